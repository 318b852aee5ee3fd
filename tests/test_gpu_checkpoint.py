"""Checkpoint and resume: a lattice saved mid-run (across forcing epochs)
and restored into a new handle created with the same arguments continues
bitwise like the uninterrupted run -- the stirring force is a counter-based
function of (seed, epoch) -- for the one-layer lattice, the 2D ring and the
3D lattice; a checkpoint of another configuration or a truncated one is
refused and leaves the state untouched."""
import os
import tempfile

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2101_06187_gb300 as rl  # noqa: E402

FORCING = dict(kmin=2, kmax=4, amp=2e-4, seed=424242, redraw_period=9)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _make(kind, **kw):
    if kind == "slab":
        return rl.Lattice(64, 48, 0.6, dtype="f32", kernel="packed", forcing=FORCING, **kw)
    if kind == "slab-fused2":  # two steps per launch: saves land between launch pairs and on odd steps
        return rl.Lattice(64, 48, 0.6, dtype="f32", kernel="fused2", forcing=FORCING, **kw)
    if kind == "slab-bf16":  # stochastic rounding of the stores: its draws are a function of the state
        return rl.Lattice(64, 48, 0.6, dtype="bf16", kernel="fused2", forcing=FORCING, rounding="stochastic", **kw)
    if kind == "ring":
        return rl.Lattice(64, 48, 0.6, dtype="f32", kernel="packed", forcing=FORCING, stencil="ring8", **kw)
    if kind == "ring-fused2":
        return rl.Lattice(64, 48, 0.6, dtype="f32", kernel="fused2", forcing=FORCING, stencil="ring8", **kw)
    return rl.Lattice3D(16, 12, 10, 0.6, dtype="f32", kernel="packed", forcing=FORCING, **kw)


def _fields(kind):
    if kind == "3d":
        return workloads.random_smooth3d(16, 12, 10, seed=5)
    return workloads.random_smooth(64, 48, seed=5)


@pytest.mark.parametrize("kind", ["slab", "slab-fused2", "slab-bf16", "ring", "ring-fused2", "3d"])
def test_resumed_run_is_bitwise_the_uninterrupted_run(kind):
    a = _make(kind)
    a.init_fields(*_fields(kind))
    a.step(40)
    ref = a.populations()
    a.close()

    b = _make(kind)
    b.init_fields(*_fields(kind))
    b.step(13)  # mid-epoch
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "state.rlbm")
        b.save(path)
        b.close()
        c = _make(kind)
        c.load(path)
    assert c.info()["step"] == 13
    c.step(27)
    np.testing.assert_array_equal(c.populations(), ref)
    c.close()


def test_mismatched_or_truncated_checkpoints_are_refused():
    a = _make("slab")
    a.init_fields(*_fields("slab"))
    a.step(5)
    ck = a.checkpoint()
    before = a.populations()
    other = rl.Lattice(64, 48, 0.6, dtype="f32", kernel="packed", forcing=dict(FORCING, seed=1))
    with pytest.raises(rl.RLBMError) as e1:
        other.restore(ck)  # another forcing seed
    assert e1.value.status == rl.RLBM_ERR_ARG
    other.close()
    bigger = rl.Lattice(64, 50, 0.6, dtype="f32", kernel="packed", forcing=FORCING)
    with pytest.raises(rl.RLBMError):
        bigger.restore(ck)  # other sizes
    bigger.close()
    with pytest.raises(rl.RLBMError):
        a.restore(ck[: len(ck) // 2])  # truncated
    np.testing.assert_array_equal(a.populations(), before)
    a.restore(ck)  # its own checkpoint is fine
    np.testing.assert_array_equal(a.populations(), before)
    a.close()
