"""Host-side helpers of bench.py that decide what a bench line reports.

The radix schedule a single capture runs (the library's choice per FFT size,
or the one asked for where the size has it), and the rule that a stored DRAM
traffic figure is reported only for the kernel it was measured on: the same
radix schedule, the same capture length and the same STFT sources.
"""
import bench


def test_schedule_of_each_size():
    # N = 16^a r: schedule 1 exists where r > 1, schedule 2 where r = 2
    assert [bench._sched_of(N, 3) for N in (256, 512, 1024, 2048, 4096, 8192)] == [0, 1, 1, 1, 0, 2]
    assert [bench._sched_of(N, -1) for N in (256, 512, 1024, 2048, 4096, 8192)] == [0, 1, 1, 1, 0, 2]
    assert [bench._sched_of(N, 2) for N in (256, 512, 1024, 2048, 4096, 8192)] == [0, 2, 0, 0, 0, 2]
    assert [bench._sched_of(N, 1) for N in (256, 512, 1024, 2048, 4096, 8192)] == [0, 1, 1, 1, 0, 1]
    assert all(bench._sched_of(N, 0) == 0 for N in (256, 512, 1024, 2048, 4096, 8192))


def test_traffic_only_for_the_measured_kernel(monkeypatch):
    entry = {"sha256": bench._sha256(bench.STFT_SOURCES), "n_samples": 1 << 20, "sched": 2, "bytes": 12345}
    monkeypatch.setitem(bench.TRAFFIC, "probe", entry)
    assert bench._traffic("probe", 1 << 20, 2) == 12345
    assert bench._traffic("probe", 1 << 20, 1) is None          # another radix schedule
    assert bench._traffic("probe", 1 << 21, 2) is None          # another capture length
    assert bench._traffic("absent", 1 << 20, 2) is None
    monkeypatch.setitem(bench.TRAFFIC, "probe", dict(entry, sha256="0" * 64))
    assert bench._traffic("probe", 1 << 20, 2) is None          # the sources changed since


def test_stored_traffic_entries_are_well_formed():
    for name, t in bench.TRAFFIC.items():
        assert name in bench.SINGLE
        gen, seed, N, hop, n, _ = bench.SINGLE[name]
        assert t["n_samples"] == n and t["sched"] == bench._sched_of(N, 3)
        assert len(t["sha256"]) == 64 and t["bytes"] > 8 * n   # at least the IQ read
