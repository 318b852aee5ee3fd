"""Host logic of the benchmark that needs no GPU: how a step count is split
into launches of the chosen kernel (two steps per launch for the two-step
kernels, an odd remainder as one single step), and the source hashes that
keep a stored DRAM-traffic figure tied to the kernel it was measured on."""
import bench


class _FakeLattice:
    def __init__(self, spl):
        self._spl = spl

    def info(self):
        return {"steps_per_launch": self._spl}


def test_launch_units_single_step_kernels():
    assert bench.launch_units(_FakeLattice(1), 5) == [1, 1, 1, 1, 1]
    assert bench.launch_units(_FakeLattice(1), 0) == []


def test_launch_units_two_step_kernels():
    assert bench.launch_units(_FakeLattice(2), 6) == [2, 2, 2]
    assert bench.launch_units(_FakeLattice(2), 7) == [2, 2, 2, 1]   # the odd step runs alone
    assert bench.launch_units(_FakeLattice(2), 1) == [1]
    assert sum(bench.launch_units(_FakeLattice(2), 1000)) == 1000


def test_source_hashes_cover_each_variant_and_differ():
    h4, h5, h7 = (bench.step_kernel_source_hash(k) for k in (4, 5, 7))
    assert len({h4, h5, h7}) == 3 and all(len(h) == 64 for h in (h4, h5, h7))
    assert bench.step_kernel_source_hash(1) == h4   # the one-step kernels share the per-node sources
