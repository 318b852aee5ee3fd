"""Long stirred runs: time-averaged energy spectra E(k) (Sec. 4).

Chaotic trajectories of different precisions decorrelate, so long runs are
compared through time-averaged spectra over the inertial range (k below the
driven shell), 2% per shell:

* 128 x 128 against the FP64 oracle itself (4000 steps, spectra averaged
  every 100 steps over the second half);
* 1024 x 1024 with the stirred workload's parameters (tau = 0.52, shell
  4..6, amplitude 1e-5): FP32 form against the FP64 form, whose every 100
  steps are pinned to the oracle at 1e-12 by the parity tests (the oracle
  itself cannot run 20k steps of a 1024^2 lattice in test time);
* 1024 x 1024 with the precision workload's band (shell 8..10, tau = 0.51):
  BF16 and FP16 deviation storage against the FP64 form, 2% per shell, each
  with its default rounding (BF16 stochastic, FP16 nearest).  BF16 with
  round-to-nearest misses the bar: its rounding error is a deterministic
  function of the smooth deviation field and shifts every low-k shell by
  about 4% (checked below as a property of that rounding, not hidden).
"""
import os

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2101_06187_gb300 as rl  # noqa: E402

oracle.set_threads(os.cpu_count() or 4)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def gpu_mean_spectrum(n, tau, forcing, dtype, steps, start, every, nshells, rounding="default"):
    lat = rl.Lattice(n, n, tau, dtype=dtype, forcing=forcing, rounding=rounding)
    lat.init_fields()
    lat.step(start)
    acc = np.zeros(nshells)
    count = 0
    for _ in range((steps - start) // every):
        lat.step(every)
        acc += lat.energy_spectrum(nshells)
        count += 1
    lat.close()
    return acc / count


def test_time_averaged_spectrum_matches_oracle_128():
    n, tau, steps, start, every, nsh = 128, 0.52, 4000, 2000, 100, 12
    fz = dict(kmin=4, kmax=6, amp=1e-4, seed=4242, redraw_period=100)
    E_g = gpu_mean_spectrum(n, tau, fz, "f32", steps, start, every, nsh)
    f = oracle.init(n, n)
    oracle.run(f, tau, start, kmin=4, kmax=6, amp=1e-4, seed=4242, redraw=100)
    acc = np.zeros(nsh)
    cnt = 0
    for k in range((steps - start) // every):
        oracle.run(f, tau, every, step0=start + k * every, kmin=4, kmax=6, amp=1e-4, seed=4242, redraw=100)
        _, vx, vy = oracle.fields(f)
        acc += oracle.energy_spectrum(vx, vy, nsh)
        cnt += 1
    E_o = acc / cnt
    rel = np.abs(E_g[1:4] - E_o[1:4]) / E_o[1:4]
    assert np.all(rel < 0.02), rel


def test_time_averaged_spectrum_fp32_vs_fp64_1024():
    w = workloads.STIRRED_1024
    fz = dict(kmin=w.kmin, kmax=w.kmax, amp=w.amp, seed=w.seed, redraw_period=w.redraw)
    args = (w.nx, w.tau, fz)
    E64 = gpu_mean_spectrum(*args, "f64", 20000, 10000, 500, 8)
    E32 = gpu_mean_spectrum(*args, "f32", 20000, 10000, 500, 8)
    rel = np.abs(E32[1:4] - E64[1:4]) / E64[1:4]
    assert np.all(rel < 0.02), rel


@pytest.fixture(scope="module")
def precision_fp64_spectrum():
    w = workloads.PRECISION_4096
    fz = dict(kmin=w.kmin, kmax=w.kmax, amp=w.amp, seed=w.seed, redraw_period=w.redraw)
    return w, fz, gpu_mean_spectrum(1024, w.tau, fz, "f64", 10000, 5000, 500, 10)


@pytest.mark.parametrize("dtype,rounding", [("bf16", "default"), ("f16", "default"), ("bf16", "stochastic"),
                                            ("f16", "stochastic")])
def test_time_averaged_spectrum_16bit_vs_fp64_1024(precision_fp64_spectrum, dtype, rounding):
    w, fz, E64 = precision_fp64_spectrum
    E16 = gpu_mean_spectrum(1024, w.tau, fz, dtype, 10000, 5000, 500, 10, rounding=rounding)
    rel = np.abs(E16[1:8] - E64[1:8]) / E64[1:8]
    assert np.all(rel < 0.02), rel


def test_nearest_rounding_biases_the_bf16_spectrum(precision_fp64_spectrum):
    """Why BF16 rounds stochastically by default: with round-to-nearest the
    time-averaged low-k spectrum is shifted by several percent, beyond the
    2% bar."""
    w, fz, E64 = precision_fp64_spectrum
    E16 = gpu_mean_spectrum(1024, w.tau, fz, "bf16", 10000, 5000, 500, 10, rounding="nearest")
    rel = (E16[1:8] - E64[1:8]) / E64[1:8]
    assert np.max(np.abs(rel)) > 0.02, rel


def test_large_workload_compensated_spectrum_fp32_vs_fp64_2048():
    """The 8192^2 workload's parameters (tau = 0.505, shell 16..18, amplitude
    2e-6, redraw every 100 steps) on its 2048^2 oracle lattice: the
    compensated spectrum k^{5/3} E(k), time-averaged over steps 5000..10000
    and normalised over 1 <= k < 16, of the FP32 form against the FP64 form
    (whose every 100 steps the parity tests pin to the oracle at 1e-12),
    2% per shell; the shell energies themselves agree to 2% as well."""
    from paper_2101_06187_gb300 import analysis
    w = workloads.LARGE_8192
    fz = dict(kmin=w.kmin, kmax=w.kmax, amp=w.amp, seed=w.seed, redraw_period=w.redraw)
    n, nsh = 2048, 17
    E64 = gpu_mean_spectrum(n, w.tau, fz, "f64", 10000, 5000, 1000, nsh)
    E32 = gpu_mean_spectrum(n, w.tau, fz, "f32", 10000, 5000, 1000, nsh)
    c64, c32 = analysis.compensated(E64)[:15], analysis.compensated(E32)[:15]
    c64, c32 = c64 / c64.mean(), c32 / c32.mean()
    assert np.all(np.abs(c32 - c64) / c64 < 0.02), (c32, c64)
    rel = np.abs(E32[1:16] - E64[1:16]) / E64[1:16]
    assert np.all(rel < 0.02), rel
