"""Two lattice steps per launch (RLBM_KERNEL_FUSED2, temporal blocking of
the stream + collide + force step of Sec. 3.2): parity with the FP64 oracle,
and bit-for-bit equality with the packed single-step kernel -- both steps of
a launch run the same per-node arithmetic and the intermediate state is
rounded to the storage type as a single step stores it.  Every tile shape,
ragged lattices (nx not a multiple of the tile width, odd ny), the 4x4
minimum (the window wraps onto itself), odd step counts and chunks that
cross forcing epochs (the force changes between the two steps of no
launch), graphs on and off, and the eta/s relaxation.
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

TILES = [(64, 16, 2), (64, 8, 4), (32, 16, 4), (128, 8, 2)]
FORCING = dict(kmin=1, kmax=2, amp=2e-4, seed=987654321, redraw_period=7)
FORCING_TINY = dict(kmin=1, kmax=1, amp=2e-3, seed=5, redraw_period=3)  # 4x4: kmax < n/2
CHUNKS = (1, 6, 13, 2, 41, 4)  # odd and even chunks, across epoch boundaries (67 steps)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _run(kernel, nx, ny, dtype, fields, tile=None, graphs=True, chunks=CHUNKS, **kw):
    forcing = FORCING if min(nx, ny) > 8 else FORCING_TINY
    lat = rl.Lattice(nx, ny, 0.6, dtype=dtype, forcing=forcing, kernel=kernel, use_graphs=graphs, **kw)
    lat.init_fields(*fields)
    if tile is not None:
        lat.set_launch(kernel, *tile)
    for n in chunks:
        lat.step(n)
    pops, info = lat.populations(), lat.info()
    lat.close()
    return pops, info


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("size", [(66, 40), (130, 27), (4, 4), (200, 34)])
def test_two_step_launches_equal_packed_single_steps(dtype, tile, size):
    nx, ny = size
    fields = workloads.random_smooth(nx, ny, seed=7 * nx + ny, deps=0.05, vmax=0.05)
    ref, _ = _run("packed", nx, ny, dtype, fields)
    got, info = _run("fused2", nx, ny, dtype, fields, tile=tile)
    assert info["kernel"] == rl.KERNELS["fused2"] and info["steps_per_launch"] == 2
    assert (info["block_x"], info["block_y"], info["launch_budget"]) == tile
    assert info["step"] == sum(CHUNKS)
    np.testing.assert_array_equal(got, ref)


def test_graphs_and_direct_launches_agree():
    nx, ny = 130, 66
    fields = workloads.random_smooth(nx, ny, seed=5)
    a, _ = _run("fused2", nx, ny, "f32", fields, graphs=True)
    b, _ = _run("fused2", nx, ny, "f32", fields, graphs=False)
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("cfl", [0.625, 0.15625, 0.9])
def test_sub_unit_cfl_equals_packed(cfl, dtype, tile):
    """0 < cfl < 1 (the paper's time steps on its coarser lattices, Sec. 5):
    runtime bilinear weights, halo 1; bit for bit against the packed kernel."""
    nx, ny = 130, 27
    fields = workloads.random_smooth(nx, ny, seed=17, deps=0.05, vmax=0.05)
    kw = dict(cfl=cfl, eta_s=0.01, dt=0.05)
    ref, _ = _run("packed", nx, ny, dtype, fields, **kw)
    got, info = _run("fused2", nx, ny, dtype, fields, tile=tile, **kw)
    assert info["kernel"] == rl.KERNELS["fused2"] and info["steps_per_launch"] == 2
    np.testing.assert_array_equal(got, ref)


def test_eta_over_s_relaxation_equals_packed():
    nx, ny = 96, 40
    fields = workloads.random_smooth(nx, ny, seed=9, deps=0.05, vmax=0.05)
    ref, _ = _run("packed", nx, ny, "f32", fields, eta_s=0.01, dt=0.05)
    got, _ = _run("fused2", nx, ny, "f32", fields, eta_s=0.01, dt=0.05)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("size", [(66, 40), (130, 27), (4, 4)])
def test_two_step_run_matches_oracle(size):
    nx, ny = size
    forcing = FORCING if min(nx, ny) > 8 else FORCING_TINY
    fields = workloads.random_smooth(nx, ny, seed=nx * 1000 + ny, deps=0.05, vmax=0.05)
    lat = rl.Lattice(nx, ny, 0.7, dtype="f32", landau="fp32", forcing=forcing, kernel="fused2")
    lat.init_fields(*fields)
    lat.step(100)
    got = lat.moments()
    lat.close()
    f = oracle.init(nx, ny, *fields)
    oracle.run(f, 0.7, 100, kmin=forcing["kmin"], kmax=forcing["kmax"], amp=forcing["amp"], seed=forcing["seed"],
               redraw=forcing["redraw_period"])
    e_r, vx_r, vy_r = oracle.fields(f)
    err_e = np.max(np.abs(got[0] - e_r)) / np.max(np.abs(e_r))
    vnorm = max(np.max(np.abs(vx_r)), np.max(np.abs(vy_r)))
    err_v = max(np.max(np.abs(got[1] - vx_r)), np.max(np.abs(got[2] - vy_r))) / vnorm
    assert err_e < 1e-5 and err_v < 1e-5, (err_e, err_v)


def test_autotune_over_tiles_keeps_state():
    nx, ny = 256, 128
    fields = workloads.random_smooth(nx, ny, seed=3)
    lat = rl.Lattice(nx, ny, 0.6, dtype="f32", forcing=FORCING, kernel="fused2")
    lat.init_fields(*fields)
    lat.step(3)
    p0 = lat.populations()
    k, bx, by = lat.autotune(3)
    assert k == rl.KERNELS["fused2"] and (bx, by) in [(t[0], t[1]) for t in TILES]
    np.testing.assert_array_equal(lat.populations(), p0)
    info = lat.info()
    assert info["steps_per_launch"] == 2 and info["bytes_per_node"] == (2 * 17 * 4 + 2 * 4) // 2
    lat.close()


def test_set_launch_rejects_misfits():
    lat = rl.Lattice(64, 32, 0.6, dtype="f32", forcing=FORCING, kernel="fused2")
    lat.init_fields()
    for bad in (("fused2", 32, 32, 2), ("packed", 128, 1, 2), ("fused2", 64, 16, 3)):
        with pytest.raises(rl.RLBMError):
            lat.set_launch(*bad)
    lat.step(2)  # the handle stays usable
    assert lat.info()["step"] == 2
    lat.close()
    lat = rl.Lattice(64, 32, 0.6, dtype="f64", forcing=FORCING)  # FP64 has no packed lanes
    with pytest.raises(rl.RLBMError):
        lat.set_launch("fused2", 64, 16, 2)
    lat.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_fp64_landau_solve_on_the_packed_kernels(dtype):
    """The FP64 Landau solve of the FP32 and 16-bit forms on the packed
    kernels (the FP32 frame refined to FP64 accuracy by one double-float
    Newton step): two steps per launch equal packed single steps bit for
    bit, and the run matches the FP64 oracle within the form's tolerance."""
    nx, ny = 66, 40
    fields = workloads.random_smooth(nx, ny, seed=5 * nx + ny, deps=0.05, vmax=0.05)
    ref, info_p = _run("packed", nx, ny, dtype, fields, landau="fp64")
    got, info_f = _run("fused2", nx, ny, dtype, fields, landau="fp64")
    assert info_p["kernel"] == rl.KERNELS["packed"] and info_f["kernel"] == rl.KERNELS["fused2"]
    np.testing.assert_array_equal(got, ref)
    lat = rl.Lattice(nx, ny, 0.6, dtype=dtype, forcing=FORCING, kernel="fused2", landau="fp64")
    lat.init_fields(*fields)
    for n in CHUNKS:
        lat.step(n)
    e_g, vx_g, vy_g, _ = lat.moments()
    lat.close()
    f = oracle.init(nx, ny, *fields)
    oracle.run(f, 0.6, sum(CHUNKS), kmin=FORCING["kmin"], kmax=FORCING["kmax"], amp=FORCING["amp"],
               seed=FORCING["seed"], redraw=FORCING["redraw_period"])
    e_o, vx_o, vy_o = oracle.fields(f)
    tol = {"f32": 1e-5, "bf16": 2e-2, "f16": 2e-3}[dtype]
    vn = max(np.max(np.abs(vx_o)), np.max(np.abs(vy_o)))
    assert np.max(np.abs(e_g - e_o)) / np.max(np.abs(e_o)) < tol
    assert max(np.max(np.abs(vx_g - vx_o)), np.max(np.abs(vy_g - vy_o))) / vn < tol
