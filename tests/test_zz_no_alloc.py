"""GPU check of rlbm_moments_static, the moments entry point that allocates
nothing (for callers that cannot allocate device memory when they need the
fields: fixed memory budgets, loops that must avoid cudaMalloc's implicit
synchronisation, memory owned by another framework's pool).

It is called through the C ABI on the device state of an ordinary handle,
twice in a row (its static scratch keeps the previous call's contents, so the
second call checks that what must start at zero is cleared), and compared
with the handle's own rlbm_moments_device.  This file is collected last so
that a stop-at-first-failure run has already run every other test; it also
passes alone in a fresh process.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2101_06187_gb300 as rl  # noqa: E402

TOL = 1e-12  # the FP64 parity bar of the GPU tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_static_scratch_moments_match_handle_moments(dtype):
    nx, ny = 200, 136
    fields = workloads.random_smooth(nx, ny, seed=99, deps=0.05, vmax=0.05)
    lat = rl.Lattice(nx, ny, 0.6, dtype=dtype, forcing=dict(kmin=2, kmax=5, amp=1e-4, seed=3, redraw_period=10))
    lat.init_fields(*fields)
    lat.step(25)
    info = lat.info()
    dev = torch.device("cuda", lat.device)
    ref = [torch.empty(ny * nx, dtype=torch.float64, device=dev) for _ in range(3)]
    ref_tot = torch.empty(3, dtype=torch.float64, device=dev)
    stream = lat._torch_stream
    lat.moments_device(ref[0], ref[1], ref[2], ref_tot)
    lat.synchronize()
    for call in range(2):
        out = [torch.full((ny * nx,), float("nan"), dtype=torch.float64, device=dev) for _ in range(3)]
        tot = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
        rl.rlbm_moments_static(rl.DTYPES[dtype], info["populations"], nx, ny, info["pitch"], info["eps0"],
                               info["scale"], out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(),
                               tot.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        for a, b in zip(out, ref):
            a, b = a.cpu().numpy(), b.cpu().numpy()
            assert np.max(np.abs(a - b)) <= TOL * np.max(np.abs(b)), call
        t, r = tot.cpu().numpy(), ref_tot.cpu().numpy()
        assert np.max(np.abs(t - r)) <= TOL * abs(r[0]), call
    lat.close()


def test_static_scratch_rejects_lattices_beyond_its_size():
    lat = rl.Lattice(64, 64, 0.7, dtype="f32")
    info = lat.info()
    n = 8192  # ceil(8192/32) * ceil(8192/8) = 262144 blocks > 65536
    with pytest.raises(rl.RLBMError):
        rl.rlbm_moments_static(rl.DTYPES["f32"], info["populations"], n, n, n, 1.0, 1.0)
    lat.close()
