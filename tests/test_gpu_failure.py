"""Failure detection on the GPU without a fault: the TMA kernel's waits on
its tile copies are bounded (one second of global time).  With the test
hook that leaves the copies unissued, the wait runs out, the kernel sets the
handle's device error word and leaves; the next synchronising call reports
RLBM_ERR_TIMEOUT (sticky on that handle), and the CUDA context stays usable:
a new lattice in the same process still matches the oracle."""
import os
import time

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
FORCING = dict(kmin=2, kmax=4, amp=2e-4, seed=123456789, redraw_period=7)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_bounded_wait_runs_out_and_is_reported():
    lat = rl.Lattice(128, 64, 0.7, dtype="f32", kernel="tma", forcing=FORCING, test_unarmed_wait=True)
    lat.init_fields()
    t0 = time.time()
    lat.step(1)
    with pytest.raises(rl.RLBMError) as err:
        lat.synchronize()
    elapsed = time.time() - t0
    assert err.value.status == rl.RLBM_ERR_TIMEOUT
    assert 0.5 < elapsed < 60.0, elapsed
    with pytest.raises(rl.RLBMError) as again:  # sticky on this handle
        lat.step(1)
    assert again.value.status == rl.RLBM_ERR_TIMEOUT
    lat.close()

    # the context is intact: a new lattice on the same kernel still matches the oracle
    nx, ny = 64, 48
    fields = workloads.random_smooth(nx, ny, seed=9, deps=0.05, vmax=0.05)
    good = rl.Lattice(nx, ny, 0.7, dtype="f32", kernel="tma", forcing=FORCING)
    good.init_fields(*fields)
    good.step(20)
    e, vx, vy, _ = good.moments()
    good.synchronize()
    good.close()
    f = oracle.init(nx, ny, *fields)
    oracle.run(f, 0.7, 20, kmin=2, kmax=4, amp=2e-4, seed=123456789, redraw=7)
    E, VX, VY = oracle.fields(f)
    assert np.max(np.abs(e - E)) < 1e-5 * np.max(np.abs(E))
    assert max(np.max(np.abs(vx - VX)), np.max(np.abs(vy - VY))) < 1e-5 * max(np.max(np.abs(VX)), np.max(np.abs(VY)))


def test_failed_allocation_is_reported_and_nothing_leaks():
    """Host-side fault injection through the allocator hooks: the k-th
    allocation fails; rlbm_create returns RLBM_ERR_ALLOC and frees every
    block it obtained (the fake allocator counts them)."""
    import ctypes
    for fail_at in (0, 1, 3, 6):
        live = {}
        calls = [0]

        def _alloc(nbytes, _ctx):
            calls[0] += 1
            if calls[0] - 1 == fail_at:
                return None
            t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
            live[t.data_ptr()] = t
            return t.data_ptr()

        def _free(ptr, _nbytes, _ctx):
            live.pop(int(ptr), None)

        alloc_cb, free_cb = rl.ALLOC_FN(_alloc), rl.FREE_FN(_free)
        o = rl.rlbm_opts_default()
        o.alloc, o.free = alloc_cb, free_cb
        out = ctypes.c_void_p()
        forcing = rl.Forcing(2, 4, 1e-4, 1, 10)
        st = rl.library().rlbm_create(64, 48, 0, 0.7, ctypes.byref(forcing), ctypes.byref(o), ctypes.byref(out))
        assert st == rl.RLBM_ERR_ALLOC, (fail_at, st)
        assert out.value is None
        assert not live, (fail_at, len(live))
