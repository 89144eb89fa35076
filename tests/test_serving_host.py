"""Host-side scheduling of the serving loop, without a GPU: grouping of queued
requests by factor-cache key, the right-hand-side cap of a batch, admission by
the library's footprint and least-recently-used eviction of idle entries."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def serving():
    from paper_1504_04058_gb300 import build
    build.build()
    from paper_1504_04058_gb300 import serving
    return serving


class FakeHandle:
    def __init__(self):
        self.destroyed = False

    def destroy(self):
        self.destroyed = True


def make_req(serving, vid, k=1, rid=0, n=63):
    return serving.Request(vid, np.ones((n, n)), 8 * np.pi, 8, 4, np.zeros((n, n, k), complex), rid=rid)


def drain(srv):
    out = []
    while True:
        k, batch = srv._take_batch()
        if batch is None:
            return out
        out.append((k[0], [r.rid for r, _ in batch]))


def test_batches_group_by_key_up_to_max_rhs(serving):
    srv = serving.Server(1 << 40, workers=1, max_rhs=4, start=False)
    for rid, (vid, k) in enumerate([("A", 1), ("B", 2), ("A", 2), ("B", 2), ("A", 1), ("B", 1)]):
        srv.submit(make_req(serving, vid, k, rid))
    assert drain(srv) == [("A", [0, 2, 4]), ("B", [1, 3]), ("B", [5])]
    srv.close()


def test_no_batching_takes_one_request_at_a_time(serving):
    srv = serving.Server(1 << 40, workers=1, max_rhs=4, start=False, batching=False)
    for rid, vid in enumerate("AAB"):
        srv.submit(make_req(serving, vid, 1, rid))
    assert drain(srv) == [("A", [0]), ("A", [1]), ("B", [2])]
    srv.close()


def test_request_wider_than_max_rhs_runs_alone(serving):
    srv = serving.Server(1 << 40, workers=1, max_rhs=4, start=False)
    srv.submit(make_req(serving, "A", 6, 0))
    srv.submit(make_req(serving, "A", 1, 1))
    assert drain(srv) == [("A", [0]), ("A", [1])]
    srv.close()


def test_busy_key_is_skipped(serving):
    srv = serving.Server(1 << 40, workers=1, max_rhs=4, start=False)
    a, b = make_req(serving, "A", 1, 0), make_req(serving, "B", 1, 1)
    srv.submit(a)
    srv.submit(b)
    e = serving._Entry(FakeHandle(), 0, 4)
    e.busy = True
    srv.cache[a.key()] = e
    assert drain(srv) == [("B", [1])]
    e.busy = False
    assert drain(srv) == [("A", [0])]
    srv.close()


def test_admission_evicts_least_recently_used_idle_entry(serving):
    from paper_1504_04058_gb300 import asp_footprint_bytes
    probe = serving.Server(1 << 40, workers=1, max_rhs=4, start=False)
    fp = asp_footprint_bytes(probe._params(make_req(serving, "A")))
    probe.close()
    assert fp > 0
    srv = serving.Server(int(2.5 * fp), workers=1, max_rhs=4, start=False)
    entries = {}
    for t, vid in enumerate("AB"):
        r = make_req(serving, vid)
        assert srv._admit(r) == fp
        entries[vid] = srv.cache[r.key()] = serving._Entry(FakeHandle(), fp, 4)
        entries[vid].last_used = float(t)
    entries["A"].last_used = 5.0  # B is now the least recently used
    r = make_req(serving, "C")
    assert srv._admit(r) == fp
    assert entries["B"].handle.destroyed and not entries["A"].handle.destroyed
    assert srv.stats["evictions"] == 1 and srv.used_bytes == 2 * fp
    srv.cache[r.key()] = serving._Entry(FakeHandle(), fp, 4)
    for e in srv.cache.values():
        e.busy = True
    assert srv._admit(make_req(serving, "D")) is None  # nothing idle to evict
    assert srv.used_bytes == 2 * fp
    srv.close()


def test_request_larger_than_budget_is_refused(serving):
    srv = serving.Server(1024, workers=1, max_rhs=4, start=False)
    with pytest.raises(MemoryError):
        srv._admit(make_req(serving, "A"))
    srv.close()


def test_unsupported_size_is_refused_at_admission(serving):
    """A 2D grid above what the sweep chain takes (n = 1217 on 152 SMs) gets a
    footprint of 0 from the library and is refused before any setup."""
    srv = serving.Server(1 << 40, workers=1, max_rhs=4, start=False)
    with pytest.raises(ValueError, match="unsupported"):
        srv._admit(make_req(serving, "A", n=1217))
    assert srv.used_bytes == 0
    srv.close()


def test_percentiles(serving):
    p = serving.percentiles(np.arange(1, 101, dtype=float))
    assert p["p50"] == pytest.approx(50.5) and p["p99"] == pytest.approx(99.01)
