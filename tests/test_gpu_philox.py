"""Pin of the Philox4x32-10 bit pattern on the GPU (the generator of the
stirring force's mode draws, Sec. 5): cuRAND's Philox4x32-10 block function
(a library routine) and the library's own device generator, both compared
word for word with the oracle on the forcing's counters under the
workloads' seeds, the all-zero and all-one words and seeded random words."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))


def test_philox_matches_curand_and_the_library_generator():
    oracle.build()
    ctr, key = workloads.philox_pin_inputs()
    src = os.path.join(HERE, "numerics", "philox_curand_check.cu")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "philox_check")
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-o", exe, src],
                       check=True)
        paths = [os.path.join(tmp, n) for n in ("ctr.bin", "key.bin", "curand.bin", "lib.bin")]
        ctr.astype("<u4").tofile(paths[0])
        key.astype("<u4").tofile(paths[1])
        subprocess.run([exe, *paths], check=True, timeout=120)
        got_curand = np.fromfile(paths[2], dtype="<u4").reshape(-1, 4)
        got_lib = np.fromfile(paths[3], dtype="<u4").reshape(-1, 4)
    want = np.stack([oracle.philox4x32_10(c, k) for c, k in zip(ctr, key)])
    for name, got in (("curand", got_curand), ("library", got_lib)):
        bad = np.nonzero(np.any(got != want, axis=1))[0]
        assert bad.size == 0, (name, bad[:8], ctr[bad[:1]], key[bad[:1]])
