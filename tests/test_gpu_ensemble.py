"""GPU tests of the ensemble (batched) step: each member must evolve exactly
like a lone lattice with the same parameters, match the oracle, and keep its
state across autotuning and graph replay."""
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

RUNS = [
    dict(nx=64, ny=64, tau=0.6, forcing=dict(kmin=2, kmax=4, amp=2e-4, seed=11, redraw_period=7)),
    dict(nx=96, ny=40, tau=0.52, forcing=dict(kmin=1, kmax=3, amp=1e-4, seed=12, redraw_period=7)),
    dict(nx=32, ny=72, tau=0.7, forcing=dict(kmin=2, kmax=3, amp=3e-4, seed=13, redraw_period=5)),
    dict(nx=128, ny=128, tau=0.51, forcing=None),
    dict(nx=8, ny=8, tau=0.9, forcing=dict(kmin=1, kmax=2, amp=1e-3, seed=14, redraw_period=3)),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _fields(r, k):
    return workloads.random_smooth(r["nx"], r["ny"], seed=500 + k, deps=0.03, vmax=0.03)


@pytest.mark.parametrize("dtype", ["f32", "f64", "bf16"])
def test_members_evolve_like_lone_lattices(dtype):
    ens = rl.Ensemble(RUNS, dtype=dtype)
    for k, r in enumerate(RUNS):
        ens.init_fields(k, *_fields(r, k))
    for n in (1, 5, 12, 3):  # chunks crossing the members' redraw epochs
        ens.step(n)
    # same per-node code in both kernels; the compiler may contract a few
    # products differently, so FP32 agrees to rounding, not bitwise
    tol = {"f64": 1e-13, "f32": 1e-6, "bf16": 1e-2}[dtype]
    for k, r in enumerate(RUNS):
        lat = rl.Lattice(r["nx"], r["ny"], r["tau"], dtype=dtype, forcing=r["forcing"], kernel="vec")
        lat.init_fields(*_fields(r, k))
        lat.step(21)
        a, b = ens.populations(k), lat.populations()
        assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(b)), k
        lat.close()
    assert ens.info()["step"] == 21
    ens.close()


def test_members_match_oracle():
    ens = rl.Ensemble(RUNS, dtype="f32")
    for k, r in enumerate(RUNS):
        ens.init_fields(k, *_fields(r, k))
    ens.step(60)
    for k in (0, 1, 4):
        r = RUNS[k]
        f = oracle.init(r["nx"], r["ny"], *_fields(r, k))
        fz = r["forcing"]
        oracle.run(f, r["tau"], 60, kmin=fz["kmin"], kmax=fz["kmax"], amp=fz["amp"], seed=fz["seed"],
                   redraw=fz["redraw_period"])
        e_o, vx_o, vy_o = oracle.fields(f)
        e_g, vx_g, vy_g, _ = ens.moments(k)
        err_e = np.max(np.abs(e_g - e_o)) / np.max(np.abs(e_o))
        vn = max(np.max(np.abs(vx_o)), np.max(np.abs(vy_o)))
        err_v = max(np.max(np.abs(vx_g - vx_o)), np.max(np.abs(vy_g - vy_o))) / vn
        assert err_e < 1e-5 and err_v < 1e-5, (k, err_e, err_v)
    ens.close()


def test_autotune_and_graphs_keep_results():
    out = []
    for tune, graphs in ((False, False), (True, True)):
        ens = rl.Ensemble(RUNS, dtype="f32", use_graphs=graphs)
        for k, r in enumerate(RUNS):
            ens.init_fields(k, *_fields(r, k))
        ens.step(4)
        if tune:
            before = [ens.populations(k) for k in range(len(RUNS))]
            bx, by, grid = ens.autotune(3)
            info = ens.info()
            # thread blocks of at most 256, or two-step tiles of at most 1024 nodes
            assert (bx * by <= 256 or (info["kernel"] == rl.KERNELS["fused2"] and bx * by <= 1024)) and grid >= 1
            for k in range(len(RUNS)):
                np.testing.assert_array_equal(ens.populations(k), before[k])
        ens.step(30)
        out.append([ens.populations(k) for k in range(len(RUNS))])
        ens.close()
    # the tuned run may use another kernel body (packed lanes): FP32 rounding, not bitwise
    for a, b in zip(*out):
        assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(a))


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("graphs", [True, False])
def test_two_step_body_equals_packed_lone_lattices(dtype, graphs):
    """The two-step ensemble body (two steps per launch through shared
    memory) against lone lattices on the packed single-step kernel: the same
    per-node arithmetic, so bit for bit; odd chunks cross the members'
    forcing epochs (an odd last step runs the packed body)."""
    ens = rl.Ensemble(RUNS, dtype=dtype, kernel="fused2", use_graphs=graphs)
    info = ens.info()
    assert info["kernel"] == rl.KERNELS["fused2"] and info["steps_per_launch"] == 2
    for k, r in enumerate(RUNS):
        ens.init_fields(k, *_fields(r, k))
    for n in (1, 6, 13, 2, 9):
        ens.step(n)
    for k, r in enumerate(RUNS):
        # ensembles round 16-bit stores to nearest by default
        lat = rl.Lattice(r["nx"], r["ny"], r["tau"], dtype=dtype, forcing=r["forcing"], kernel="packed",
                         rounding="nearest")
        lat.init_fields(*_fields(r, k))
        lat.step(31)
        np.testing.assert_array_equal(ens.populations(k), lat.populations(), err_msg=str(k))
        lat.close()
    ens.close()


def test_two_step_body_autotune_keeps_state():
    ens = rl.Ensemble(RUNS, dtype="f32", kernel="fused2")
    for k, r in enumerate(RUNS):
        ens.init_fields(k, *_fields(r, k))
    ens.step(3)
    before = [ens.populations(k) for k in range(len(RUNS))]
    bx, by, grid = ens.autotune(2)
    assert (bx, by) in ((64, 8), (64, 16), (32, 16), (128, 8)) and grid >= 1
    for k in range(len(RUNS)):
        np.testing.assert_array_equal(ens.populations(k), before[k])
    info = ens.info()
    nodes = sum(r["nx"] * r["ny"] for r in RUNS)
    forced = sum(r["nx"] * r["ny"] for r in RUNS if r["forcing"])
    assert info["bytes_per_step"] == (nodes * 2 * 17 * 4 + forced * 8) // 2
    ens.close()


def test_ensemble_workload_shape_runs():
    """The 64-member workload (sides 256..1024, tau in [0.51, 0.7], bands
    around centres in [4, 12]) steps and stays physical."""
    runs = [dict(nx=w.nx, ny=w.ny, tau=w.tau,
                 forcing=dict(kmin=w.kmin, kmax=w.kmax, amp=w.amp, seed=w.seed, redraw_period=w.redraw))
            for w in workloads.ensemble()]
    ens = rl.Ensemble(runs, dtype="f32")
    ens.autotune(2)
    ens.step(100)
    info = ens.info()
    assert info["nruns"] == 64 and info["step"] == 100
    for k in (0, 31, 63):
        e, vx, vy, tot = ens.moments(k)
        assert np.all(np.isfinite(e)) and np.max(np.hypot(vx, vy)) < 0.1
    ens.close()


def test_ensemble_workload_members_match_oracle():
    """The 64-member workload (sides 256..1024), autotuned as the benchmark
    runs it, 100 steps from seeded smooth fields; one member of each side up
    to 512 against the FP64 oracle at the FP32 bar."""
    members = workloads.ensemble()
    runs = [dict(nx=w.nx, ny=w.ny, tau=w.tau,
                 forcing=dict(kmin=w.kmin, kmax=w.kmax, amp=w.amp, seed=w.seed, redraw_period=w.redraw))
            for w in members]
    ens = rl.Ensemble(runs, dtype="f32")
    ens.autotune(2)
    picks = {}
    for k, w in enumerate(members):
        ens.init_fields(k, *workloads.random_smooth(w.nx, w.ny, seed=900 + k, deps=0.02, vmax=0.02))
        if w.nx <= 512 and w.nx not in picks:
            picks[w.nx] = k
    ens.step(100)
    assert len(picks) == 3
    for k in picks.values():
        w = members[k]
        f = oracle.init(w.nx, w.ny, *workloads.random_smooth(w.nx, w.ny, seed=900 + k, deps=0.02, vmax=0.02))
        oracle.run(f, w.tau, 100, kmin=w.kmin, kmax=w.kmax, amp=w.amp, seed=w.seed, redraw=w.redraw)
        e_o, vx_o, vy_o = oracle.fields(f)
        e_g, vx_g, vy_g, _ = ens.moments(k)
        err_e = np.max(np.abs(e_g - e_o)) / np.max(np.abs(e_o))
        vn = max(np.max(np.abs(vx_o)), np.max(np.abs(vy_o)))
        err_v = max(np.max(np.abs(vx_g - vx_o)), np.max(np.abs(vy_g - vy_o))) / vn
        assert err_e < 1e-5 and err_v < 1e-5, (k, w.nx, err_e, err_v)
    ens.close()


def test_bad_member_index_rejected():
    ens = rl.Ensemble(RUNS[:2], dtype="f32")
    buf = np.empty(64 * 64)
    with pytest.raises(rl.RLBMError):
        rl.rlbm_batch_moments(ens.handle, 5, buf, buf, buf, np.empty(3))
    with pytest.raises(rl.RLBMError):
        rl.rlbm_batch_moments(ens.handle, -1, buf, buf, buf, np.empty(3))
    ens.close()


def test_stochastic_rounding_members_equal_lone_lattices():
    """BF16 members rounding their stores stochastically (the random bits
    are hashed from each member's own node index and state) evolve bit for
    bit like lone lattices with the same rounding."""
    ens = rl.Ensemble(RUNS, dtype="bf16", kernel="fused2", rounding="stochastic")
    for k, r in enumerate(RUNS):
        ens.init_fields(k, *_fields(r, k))
    ens.step(14)
    for k, r in enumerate(RUNS):
        lat = rl.Lattice(r["nx"], r["ny"], r["tau"], dtype="bf16", forcing=r["forcing"], kernel="packed",
                         rounding="stochastic")
        lat.init_fields(*_fields(r, k))
        lat.step(14)
        np.testing.assert_array_equal(ens.populations(k), lat.populations(), err_msg=str(k))
        lat.close()
    ens.close()
