"""GPU check of rlbm_moments_static, the moments entry point that allocates
nothing.  It exists for callers that cannot allocate device memory when
they need the fields: applications that run on a memory budget fixed up
front, time-stepping loops that must not take cudaMalloc's implicit
synchronisation, and hosts whose device memory belongs to another
framework's pool.

It is called through the C ABI on the device state of an ordinary handle,
twice in a row (its static scratch keeps the previous call's contents: the
second call sees the first call's partial sums and failed-node count still
there), and compared with the handle's own rlbm_moments_device within the
FP64 parity tolerance of the GPU tests; on lattices that stream at cfl != 1
it is also compared with the oracle's fields of an FP64 run.  The reported
failed-node count must be 0 on both calls.  This file is collected last so
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
FORCING = dict(kmin=2, kmax=5, amp=1e-4, seed=3, redraw_period=10)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _static_moments(lat, info, cfl, sentinel_bad=-7):
    nx, ny = lat.nx, lat.ny
    dev = torch.device("cuda", lat.device)
    out = [torch.full((ny * nx,), float("nan"), dtype=torch.float64, device=dev) for _ in range(3)]
    tot = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
    bad = torch.full((1,), sentinel_bad, dtype=torch.int32, device=dev)
    stream = lat._torch_stream
    rl.rlbm_moments_static(rl.STENCILS["sph26"], rl.DTYPES[lat.dtype], info["populations"], nx, ny, info["pitch"],
                           info["eps0"], info["scale"], cfl, out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(),
                           tot.data_ptr(), bad.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return [a.cpu().numpy() for a in out], tot.cpu().numpy(), int(bad.cpu().item())


def _check_against_handle(dtype, cfl):
    nx, ny = 200, 136
    fields = workloads.random_smooth(nx, ny, seed=99, deps=0.05, vmax=0.05)
    lat = rl.Lattice(nx, ny, 0.6, dtype=dtype, forcing=FORCING, cfl=cfl)
    lat.init_fields(*fields)
    lat.step(25)
    info = lat.info()
    dev = torch.device("cuda", lat.device)
    ref = [torch.empty(ny * nx, dtype=torch.float64, device=dev) for _ in range(3)]
    ref_tot = torch.empty(3, dtype=torch.float64, device=dev)
    lat.moments_device(ref[0], ref[1], ref[2], ref_tot)
    lat.synchronize()
    ref = [a.cpu().numpy() for a in ref]
    r = ref_tot.cpu().numpy()
    for call in range(2):
        out, t, nbad = _static_moments(lat, info, cfl)
        assert nbad == 0, (call, nbad)
        for a, b in zip(out, ref):
            assert np.max(np.abs(a - b)) <= TOL * np.max(np.abs(b)), call
        assert np.max(np.abs(t - r)) <= TOL * abs(r[0]), call
    lat.close()


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_static_scratch_moments_match_handle_moments(dtype):
    _check_against_handle(dtype, 1.0)


@pytest.mark.parametrize("cfl", [0.625, 1.25])
def test_static_scratch_moments_at_other_cfl(cfl):
    """The paper's time steps on its finer lattices (Sec. 5: cfl 0.625 and
    1.25): the pull before the moments moves cfl v_i cells."""
    _check_against_handle("f32", cfl)


@pytest.mark.parametrize("cfl", [0.625, 1.25])
def test_static_scratch_moments_match_oracle_at_other_cfl(cfl):
    import oracle
    oracle.build()
    nx, ny, nsteps = 48, 40, 12
    fields = workloads.random_smooth(nx, ny, seed=17, deps=0.05, vmax=0.05)
    lat = rl.Lattice(nx, ny, 0.6, dtype="f64", forcing=FORCING, cfl=cfl)
    lat.init_fields(*fields)
    lat.step(nsteps)
    info = lat.info()
    f = oracle.init(nx, ny, *fields)
    oracle.run(f, 0.6, nsteps, kmin=FORCING["kmin"], kmax=FORCING["kmax"], amp=FORCING["amp"], seed=FORCING["seed"],
               redraw=FORCING["redraw_period"], cfl=cfl)
    want = oracle.fields(f, cfl)
    for call in range(2):
        out, _, nbad = _static_moments(lat, info, cfl)
        assert nbad == 0
        err_e = np.max(np.abs(out[0] - want[0].ravel())) / np.max(np.abs(want[0]))
        vn = max(np.max(np.abs(want[1])), np.max(np.abs(want[2])))
        err_v = max(np.max(np.abs(out[1] - want[1].ravel())), np.max(np.abs(out[2] - want[2].ravel()))) / vn
        assert err_e <= TOL and err_v <= TOL, (call, err_e, err_v)
    lat.close()


def test_static_scratch_rejects_lattices_beyond_its_size_and_other_layouts():
    lat = rl.Lattice(64, 64, 0.7, dtype="f32")
    info = lat.info()
    n = 8192  # ceil(8192/32) * ceil(8192/8) = 262144 blocks > 65536
    with pytest.raises(rl.RLBMError):
        rl.rlbm_moments_static(rl.STENCILS["sph26"], rl.DTYPES["f32"], info["populations"], n, n, n, 1.0, 1.0)
    with pytest.raises(rl.RLBMError):  # the ring's 8-plane state is not this call's layout
        rl.rlbm_moments_static(rl.STENCILS["ring8"], rl.DTYPES["f32"], info["populations"], 64, 64, info["pitch"],
                               1.0, 1.0)
    for cfl in (0.0, 2.0, float("nan")):
        with pytest.raises(rl.RLBMError):
            rl.rlbm_moments_static(rl.STENCILS["sph26"], rl.DTYPES["f32"], info["populations"], 64, 64, info["pitch"],
                                   1.0, 1.0, cfl)
    lat.close()
