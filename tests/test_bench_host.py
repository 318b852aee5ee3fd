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


class _RecordingLattice(_FakeLattice):
    def __init__(self, spl):
        super().__init__(spl)
        self.calls = []

    def step(self, n):
        self.calls.append(n)

    def synchronize(self):
        pass


def test_warm_up_makes_the_timed_calls_for_both_buffer_parities():
    # graphs are keyed by (step count, starting buffer): at least two calls of
    # the timed size must run before the first timed event
    for spl, warmup, want in ((2, 5, [2, 2, 2]), (2, 1, [2, 2]), (1, 3, [1, 1, 1]), (1, 0, [1, 1])):
        lat = _RecordingLattice(spl)
        done = bench.warm_up(lat, warmup)
        assert lat.calls == want and done == sum(want)


def test_flush_policy_and_shared_workload_config():
    import workloads
    assert not bench.needs_flush(8192, "f32")      # 9.7 GB of state: larger than L2
    assert bench.needs_flush(128, "f64")
    w = workloads.LARGE_8192
    c = bench.workload_config(w, 8192, "f32")
    assert c["workload"] == "stirred_8192x8192_tau0.505_shell16-18"
    assert c == bench.workload_config(w, 8192, "f32")  # both arms build it the same way
    assert "larger than L2" in c["l2"]
