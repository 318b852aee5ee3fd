"""Domain decomposition on one GPU: a lattice split into slabs of rows
(paper_2101_06187_gb300/slab.py, SlabGroup: the slabs of one lattice in one
process, halo rows exchanged by device copies through rlbm_halo_pack /
rlbm_halo_unpack, the force drawn in the whole lattice's frame by
rlbm_set_force_frame) advances exactly like the whole lattice: the slabs'
interior populations equal the whole lattice's bit for bit, for one and two
halo rows, the packed single step and two steps per launch, ragged slab
sizes and forcing epochs crossed between exchanges."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2101_06187_gb300 as rl  # noqa: E402
from paper_2101_06187_gb300 import slab  # noqa: E402

FORCING = dict(kmin=1, kmax=3, amp=2e-4, seed=31, redraw_period=5)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("world,halo,kernel,dtype", [(2, 1, "packed", "f32"), (3, 1, "packed", "f32"),
                                                     (2, 2, "fused2", "f32"), (3, 2, "fused2", "f32"),
                                                     (2, 1, "gather", "f64")])
def test_slabs_equal_the_whole_lattice(world, halo, kernel, dtype):
    nx, ny, tau, nsteps = 64, 67, 0.6, 24
    fields = workloads.random_smooth(nx, ny, seed=8, deps=0.05, vmax=0.05)
    whole = rl.Lattice(nx, ny, tau, dtype=dtype, forcing=FORCING, kernel=kernel)
    whole.init_fields(*fields)
    whole.step(nsteps)
    ref = whole.populations()
    e_ref = whole.moments()[0]
    whole.close()
    group = slab.SlabGroup(nx, ny, tau, world, halo, dtype=dtype, forcing=FORCING, kernel=kernel)
    group.init_fields(*fields)
    group.step(nsteps)
    parts = [s.lat.populations()[:, slice(*s.rows.interior), :] for s in group.slabs]
    got = np.concatenate(parts, axis=1)
    e_got = group.moments()[0]
    group.close()
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(e_got, e_ref)


def test_force_frame_gives_the_whole_lattices_rows():
    nx, ny = 32, 48
    whole = rl.Lattice(nx, ny, 0.7, dtype="f32", forcing=FORCING)
    Fx, Fy = whole.force()
    whole.close()
    part = rl.Lattice(nx, 20, 0.7, dtype="f32", forcing=FORCING)
    part.set_force_frame(nx, ny, 0, -3)   # local rows 0..19 = global rows 45..47, 0..16
    px, py = part.force()
    g = (np.arange(20) - 3) % ny
    np.testing.assert_array_equal(px, Fx[g])
    np.testing.assert_array_equal(py, Fy[g])
    with pytest.raises(rl.RLBMError):
        part.set_force_frame(nx, 6, 0, 0)   # kmax 3 needs a frame wider than 6
    part.close()
