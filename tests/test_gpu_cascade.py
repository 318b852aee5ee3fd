"""The paper's qualitative physics (Sec. 4, Sec. 5, Figs. 5-7): a lattice
stirred at small scales develops an inverse energy cascade whose
time-averaged spectrum falls as k^(-5/3) between the largest scales and the
driven band.  A statistical check, not a parity pin: 512^2, FP32, tau =
0.51, stirring on the shell 20 <= |k| <= 24; after 30000 steps, E(k) is
averaged over 100 samples of the next 30000 steps (device-side statistics)
and fitted over 3 <= k <= 13.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2101_06187_gb300 as rl  # noqa: E402
from paper_2101_06187_gb300 import analysis  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_inverse_cascade_follows_the_kolmogorov_slope():
    n, nsh = 512, 128
    lat = rl.Lattice(n, n, 0.51, dtype="f32", kernel="packed",
                     forcing=dict(kmin=20, kmax=24, amp=3e-5, seed=11, redraw_period=100))
    lat.init_fields()
    lat.step(30000)
    lat.spectrum_reset()
    for _ in range(100):
        lat.step(300)
        lat.spectrum_sample(nsh)
    mean, sem, count = lat.spectrum_stats(nsh)
    lat.close()
    assert count == 100
    slope, _ = analysis.fit_slope(mean, 3, 13)
    assert -2.0 < slope < -1.35, slope
    comp = analysis.compensated(mean)  # k^(5/3) E(k), k = 1, 2, ...
    flat = comp[3:13] / comp[5]        # k = 4 .. 13, normalised at k = 6
    assert np.all((flat > 0.6) & (flat < 1.6)), flat
    # energy moves to large scales: the spectrum peaks well below the driven band
    assert int(np.argmax(mean[1:19])) + 1 <= 8
