"""bench.py's host-side bookkeeping, without a GPU: the ncu traffic figures
are reported only for the workload and the kernel sources they were
captured on; the algorithmic counts are those the design states."""
import bench


def test_traffic_only_for_its_workload_and_sources():
    for k in bench.NCU_TRAFFIC:
        got = bench.ncu_traffic(k)
        assert got is None or got == bench.NCU_TRAFFIC[k]["bytes"], k   # null once the sources changed
        assert bench.ncu_traffic(k, (1_000_000, 400)) is None
        assert bench.ncu_traffic(k, (500_000, 800)) is None
    assert bench.ncu_traffic("k_composite") is None


def test_traffic_goes_null_when_a_source_changes(monkeypatch):
    k = "k_search_select"
    e = dict(bench.NCU_TRAFFIC[k])
    e["sha256"] = "0" * 64
    monkeypatch.setitem(bench.NCU_TRAFFIC, k, e)
    assert bench.ncu_traffic(k) is None


def test_decode_gather_bytes():
    # 8 K S (neighbour ids and distances) + 4 F U (feature rows) + 16 S
    assert bench.agg_gather_bytes(S=10, K=8, F=32, U=3) == 8 * 8 * 10 + 4 * 32 * 3 + 16 * 10
