"""Pin of the oracle's Philox4x32-10 bit pattern (the generator of the
stirring force's mode draws, Sec. 5) against an implementation it shares
nothing with: Triton's own Philox4x32 (the generator of Triton's random
number functions, from the same SC'11 definition by Salmon, Moraes, Dror and
Shaw), run on the CPU by Triton's interpreter.  The words compared are the
counters the forcing uses under the workloads' seeds, the all-zero and
all-one words, and seeded random ones; a wrong multiplier, Weyl constant,
word exchange or round count changes almost every output word.  The GPU
test tests/test_gpu_philox.py pins the same words against cuRAND's
Philox4x32-10 and the library's device generator."""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

import oracle
import workloads

HERE = os.path.dirname(os.path.abspath(__file__))


def _oracle_words(ctr, key):
    return np.stack([oracle.philox4x32_10(c, k) for c, k in zip(ctr, key)])


def test_philox_matches_triton_implementation():
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    ctr, key = workloads.philox_pin_inputs()
    with tempfile.TemporaryDirectory() as tmp:
        paths = [os.path.join(tmp, n) for n in ("ctr.npy", "key.npy", "out.npy")]
        np.save(paths[0], ctr)
        np.save(paths[1], key)
        env = dict(os.environ, TRITON_INTERPRET="1", CUDA_VISIBLE_DEVICES="")
        r = subprocess.run([sys.executable, os.path.join(HERE, "numerics", "philox_triton_check.py"), *paths],
                           env=env, capture_output=True, text=True, timeout=600)
        if r.returncode != 0 and "No module named" in r.stderr:
            pytest.skip("Triton's interpreter is not importable here: " + r.stderr.strip().splitlines()[-1])
        assert r.returncode == 0, r.stderr
        got = np.load(paths[2])
    want = _oracle_words(ctr, key)
    assert got.shape == want.shape
    bad = np.nonzero(np.any(got != want, axis=1))[0]
    assert bad.size == 0, (bad[:8], ctr[bad[:1]], key[bad[:1]], got[bad[:1]], want[bad[:1]])


def test_philox_pin_inputs_cover_the_forcing_counters():
    ctr, key = workloads.philox_pin_inputs(n_random=16)
    seed = workloads.SEED
    k = (seed & 0xFFFFFFFF, seed >> 32)
    sel = (key[:, 0] == k[0]) & (key[:, 1] == k[1])
    assert {(int(c[0]), int(c[2])) for c in ctr[sel]} >= {(e, s) for e in range(4) for s in range(2)}
    assert len({int(c[1]) for c in ctr[sel]}) == 256
