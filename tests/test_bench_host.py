"""Host logic of bench.py (no GPU): clock-record parsing, the traffic figure's source check,
the algorithmic flop count and the voxel option."""
import bench


def test_clock_summary_reads_clocks_and_reasons():
    s = bench.ClockSampler(0)
    s.lines = [
        "0, 2070, 2070, 812.3, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    r = s.summary()
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_summary_flags_thermal_and_hw_slowdown():
    s = bench.ClockSampler(0)
    s.lines = ["0, 1500, 2070, 900, 0x48, Active, Not Active, Active, Not Active"]
    r = s.summary()
    assert r["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and r["sm_mhz"] == 1500.0


def test_clock_summary_without_samples():
    r = bench.ClockSampler(0).summary()
    assert r == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    sha = bench.cuda_sources_sha256()
    monkeypatch.setitem(bench.NCU_TRAFFIC, "sources_sha256", sha)
    monkeypatch.setitem(bench.NCU_TRAFFIC, "bytes_per_launch", {"barrel/fp64": 1234, "calorimeter/fp64/staged": 99})
    assert bench.measured_traffic("barrel", "fp64") == 1234
    assert bench.measured_traffic("barrel", "fp64", "staged") is None      # each schedule has its own capture
    assert bench.measured_traffic("calorimeter", "fp64", "staged") == 99
    assert bench.measured_traffic("barrel", "fp32_recheck") is None
    assert bench.measured_traffic("calorimeter", "fp64") is None
    monkeypatch.setitem(bench.NCU_TRAFFIC, "sources_sha256", "0" * 64)
    assert bench.measured_traffic("barrel", "fp64") is None


def test_source_hash_ignores_comments_only():
    """The traffic figure's source check hashes what the compiler sees: comments and spacing do not count,
    string literals and code do."""
    a = 'int a = 1;  // one\n/* block */ const char *s = "x//y"; char q = \'"\';\n'
    b = 'int a = 1;\nconst char *s = "x//y";   char q = \'"\'; // other comment\n'
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only(a) != bench.code_only(a.replace("x//y", "x/y"))
    assert bench.code_only(a) != bench.code_only(a.replace("a = 1", "a = 2"))


def test_algorithmic_flops_weights_each_counted_event():
    counts = {k: 0 for k in bench.FLOPS}
    assert bench.algorithmic_flops(counts) == 0.0
    for k in bench.FLOPS:
        c = dict(counts, **{k: 3})
        assert bench.algorithmic_flops(c) == 3.0 * bench.FLOPS[k]
    assert bench.algorithmic_flops({k: 1 for k in bench.FLOPS}) == float(sum(bench.FLOPS.values()))


def test_voxel_option():
    assert bench.parse_voxel("default") is None
    assert bench.parse_voxel("smart").mode == "smart"
    v = bench.parse_voxel("fixed:2,0:51,11")
    assert (v.mode, tuple(v.axes), tuple(v.slices)) == ("fixed", (2, 0), (51, 11))


class _Event:
    def __init__(self, **kw):
        self.t = None

    def record(self, stream=None):
        _Event.clock += 1.0
        self.t = _Event.clock

    def elapsed_time(self, end):
        return end.t - self.t


class _FakeTorch:
    class cuda:
        Event = _Event
        syncs = []

        @staticmethod
        def synchronize():
            _FakeTorch.cuda.syncs.append(len(_FakeTorch.log))

    log = []


class _FakeG4:
    def __init__(self):
        self.launches = []

    def g4n_transport_batch(self, ctx, items, seed, edep, cnt, **kw):
        self.launches.append(seed)
        _FakeTorch.log.append(("launch", seed))

    def g4n_sync(self, ctx, stream=None):
        pass

    def g4n_kernel_launches(self, ctx):
        return 5 * len(self.launches)   # as if every batch launched five kernels

    def counters_dict(self, cnt):
        return {"steps": 7}


class _Arr:
    shape = (100, 1)

    def zero_(self):
        pass

    def fill_(self, x):
        _FakeTorch.log.append(("flush", x))


def test_timed_region_is_bracketed_by_synchronize_and_barrier():
    _Event.clock = 0.0
    _FakeTorch.log, _FakeTorch.cuda.syncs = [], []
    calls = []
    barrier = lambda: calls.append(len(_FakeTorch.log))
    g4 = _FakeG4()

    class A:
        warmup, steps = 3, 4

    ms, c, _, launches = bench.time_mode(g4, _FakeTorch, None, None, 100, 0, A, _Arr(), _Arr(), _Arr(), None, {},
                                         barrier=barrier)
    assert g4.launches == [1100, 1101, 1102, 100, 101, 102, 103]     # W warm-ups, then exactly K timed launches
    assert launches == 5 * 4                                         # the kernels of the K timed batches only
    assert len(ms) == 4 and c == {"steps": 7}
    first_timed = _FakeTorch.log.index(("flush", 0.0))
    # a synchronize and a barrier right before the first timed launch and right after the last
    assert calls == [first_timed, len(_FakeTorch.log)]
    assert first_timed in _FakeTorch.cuda.syncs and len(_FakeTorch.log) in _FakeTorch.cuda.syncs
