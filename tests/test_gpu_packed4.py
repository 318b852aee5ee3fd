"""Four nodes per thread (RLBM_KERNEL_PACKED4): the packed stream + collide +
force step of Sec. 3.2 for two node pairs per thread, each class row read as
one aligned run of four values plus at most one side value.  Per lane it runs
the packed kernel's taps, weights, operation order and store rounding, so its
populations must equal RLBM_KERNEL_PACKED's bit for bit: every launch shape
and register budget, FP32 / BF16 / FP16 storage, round-to-nearest and
stochastic rounding, the FP32 and the refined FP64-accurate Landau frame,
forced and unforced runs, lattices where one run of four is the whole row
width apart from its periodic neighbours (nx = 4, 8) and rows whose run count
leaves the last block ragged.  Plus parity with the FP64 oracle and the
conditions the kernel refuses (nx not divisible by 4, cfl != 1, FP64
storage).
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

SHAPES = [(128, 1, 4), (64, 2, 4), (32, 4, 4), (128, 1, 3), (64, 2, 3), (32, 4, 3)]
FORCING = dict(kmin=1, kmax=2, amp=2e-4, seed=987654321, redraw_period=7)
FORCING_TINY = dict(kmin=1, kmax=1, amp=2e-3, seed=5, redraw_period=3)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _run(kernel, nx, ny, dtype, fields, shape=None, steps=(5, 1, 9), forced=True, **kw):
    forcing = (FORCING if min(nx, ny) > 8 else FORCING_TINY) if forced else None
    lat = rl.Lattice(nx, ny, 0.6, dtype=dtype, forcing=forcing, kernel=kernel, **kw)
    lat.init_fields(*fields)
    if shape is not None:
        lat.set_launch(kernel, *shape)
    for n in steps:
        lat.step(n)
    pops, info = lat.populations(), lat.info()
    lat.close()
    return pops, info


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("size", [(68, 40), (1100, 9), (4, 4), (8, 6)])
def test_four_node_runs_equal_packed_pairs(dtype, shape, size):
    nx, ny = size
    fields = workloads.random_smooth(nx, ny, seed=11 * nx + ny, deps=0.05, vmax=0.05)
    ref, _ = _run("packed", nx, ny, dtype, fields, rounding="nearest")
    got, info = _run("packed4", nx, ny, dtype, fields, shape=shape, rounding="nearest")
    assert info["kernel"] == rl.KERNELS["packed4"] and info["steps_per_launch"] == 1
    assert (info["block_x"], info["block_y"], info["launch_budget"]) == shape
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("forced", [True, False])
def test_stochastic_rounding_equals_packed(dtype, forced):
    """The rounding draws hash each pair's node index and updated rest
    values, so the four-node kernel rounds every pair as the packed kernel
    does."""
    nx, ny = 132, 50
    fields = workloads.random_smooth(nx, ny, seed=3, deps=0.05, vmax=0.05)
    ref, _ = _run("packed", nx, ny, dtype, fields, forced=forced, rounding="stochastic")
    got, _ = _run("packed4", nx, ny, dtype, fields, forced=forced, rounding="stochastic")
    np.testing.assert_array_equal(got, ref)
    nearest, _ = _run("packed4", nx, ny, dtype, fields, forced=forced, rounding="nearest")
    assert np.any(got != nearest)  # the stochastic path ran


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_refined_frame_equals_packed(dtype):
    """RLBM_LANDAU_FP64 on FP32 lanes: the frame refined to FP64 accuracy."""
    nx, ny = 96, 44
    fields = workloads.random_smooth(nx, ny, seed=9, deps=0.08, vmax=0.3)
    ref, _ = _run("packed", nx, ny, dtype, fields, landau="fp64", rounding="nearest")
    got, _ = _run("packed4", nx, ny, dtype, fields, landau="fp64", rounding="nearest")
    np.testing.assert_array_equal(got, ref)


def test_fp32_parity_with_the_oracle():
    """100 forced steps from smooth fields: the FP32 bar of the packed
    kernel (1e-5 relative on eps and on v against the FP64 oracle)."""
    nx, ny = 64, 48
    eps, vx, vy = workloads.random_smooth(nx, ny, seed=21, deps=0.05, vmax=0.05)
    lat = rl.Lattice(nx, ny, 0.6, dtype="f32", forcing=FORCING, kernel="packed4")
    lat.init_fields(eps, vx, vy)
    lat.step(100)
    e, u, w, _ = lat.moments()
    lat.close()
    f = oracle.init(nx, ny, eps, vx, vy)
    oracle.run(f, 0.6, 100, kmin=FORCING["kmin"], kmax=FORCING["kmax"], amp=FORCING["amp"], seed=FORCING["seed"],
               redraw=FORCING["redraw_period"])
    re, ru, rw = oracle.fields(f)
    vnorm = max(np.max(np.abs(ru)), np.max(np.abs(rw)))
    assert np.max(np.abs(e - re)) <= 1e-5 * np.max(np.abs(re))
    assert max(np.max(np.abs(u - ru)), np.max(np.abs(w - rw))) <= 1e-5 * vnorm


def test_refused_configurations():
    with pytest.raises(rl.RLBMError):
        rl.Lattice(66, 8, 0.6, dtype="f32", kernel="packed4")  # nx not divisible by 4
    with pytest.raises(rl.RLBMError):
        rl.Lattice(64, 8, 0.6, dtype="f32", kernel="packed4", cfl=0.625)
    with pytest.raises(rl.RLBMError):
        rl.Lattice(64, 8, 0.6, dtype="f64", kernel="packed4")
    lat = rl.Lattice(64, 8, 0.6, dtype="f32", kernel="packed4")
    with pytest.raises(rl.RLBMError):
        lat.set_launch("packed4", 256, 1, 4)  # at most 128 threads per block
    lat.close()


def test_autotuner_considers_four_node_runs():
    """The autotuner times the four-node shapes among its candidates; its
    choice (whatever it is) steps the lattice."""
    nx, ny = 256, 64
    fields = workloads.random_smooth(nx, ny, seed=4)
    lat = rl.Lattice(nx, ny, 0.6, dtype="bf16", forcing=FORCING, kernel="packed4")
    lat.init_fields(*fields)
    kernel, bx, by = lat.autotune(reps=3)
    assert kernel == rl.KERNELS["packed4"] and bx * by <= 128
    lat.step(3)
    lat.close()


def test_graphs_and_direct_launches_agree():
    """Step chunks replayed as CUDA graphs equal the same launches issued
    one by one (BF16, stochastic rounding, across forcing epochs)."""
    nx, ny = 132, 50
    fields = workloads.random_smooth(nx, ny, seed=6, deps=0.05, vmax=0.05)
    a, _ = _run("packed4", nx, ny, "bf16", fields, steps=(6, 9, 1), rounding="stochastic", use_graphs=True)
    b, _ = _run("packed4", nx, ny, "bf16", fields, steps=(6, 9, 1), rounding="stochastic", use_graphs=False)
    np.testing.assert_array_equal(a, b)


def test_autotuner_skips_four_node_runs_where_nx_is_not_divisible_by_4():
    """On an automatic-kernel handle whose rows do not split into runs of
    four, the four-node shapes are refused by their launcher and passed over;
    pinning one fails and leaves the handle usable."""
    nx, ny = 66, 40
    fields = workloads.random_smooth(nx, ny, seed=8)
    lat = rl.Lattice(nx, ny, 0.6, dtype="bf16", forcing=FORCING)
    lat.init_fields(*fields)
    kernel, _, _ = lat.autotune(reps=2)
    assert kernel != rl.KERNELS["packed4"]
    with pytest.raises(rl.RLBMError):
        lat.set_launch("packed4", 128, 1, 4)
    lat.step(4)
    assert lat.info()["step"] == 4
    lat.close()
