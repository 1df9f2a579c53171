"""Serving-form scheduler on the host: admission under the HBM budget, FIFO
order, grouping of small jobs, replay timing and shutdown.  The server runs
in dry-run mode (each run sleeps in proportion to its rows; no CUDA call), so
these tests need no GPU."""
import pytest

from paper_2603_16103_gb300 import binding as B


def fake(n, sh_dim=48):
    s = B.ngs_splats()
    s.n, s.cap, s.sh_dim = n, n, sh_dim
    return s


def server(**cfg):
    base = dict(dry_run_ns_per_splat=20.0, bytes_per_splat=1000)
    base.update(cfg)
    return B.Server(**base)


def intervals(srv, ids):
    return [(srv.info(j)["start_s"], srv.info(j)["finish_s"]) for j in ids]


def test_one_slot_is_fifo_without_overlap():
    with server(slots=1, group_small=0) as srv:
        ids = [srv.submit(fake(n), max(1, n // 2)) for n in (200_000, 50_000, 300_000, 1000)]
        for j in ids:
            srv.wait(j, 30)
        iv = intervals(srv, ids)
        starts = [a for a, _ in iv]
        assert starts == sorted(starts)
        for (a0, b0), (a1, b1) in zip(iv, iv[1:]):
            assert a1 >= b0 - 1e-9
        for j in ids:
            info = srv.info(j)
            assert info["status"] == B.NGS_JOB_DONE and info["group_size"] == 1
            assert info["n_out"] == info["target"]


def test_budget_admits_one_large_job_at_a_time():
    # each job's estimate is 60% of the budget: never two at once, on any slot count
    with server(slots=4, group_small=0, hbm_budget_bytes=100_000_000) as srv:
        ids = [srv.submit(fake(60_000), 100) for _ in range(5)]
        for j in ids:
            srv.wait(j, 30)
        iv = sorted(intervals(srv, ids))
        for (a0, b0), (a1, b1) in zip(iv, iv[1:]):
            assert a1 >= b0 - 1e-9
        assert srv.stats()["peak_reserved_bytes"] <= 100_000_000


def test_concurrent_slots_overlap_when_the_budget_allows():
    with server(slots=4, group_small=0, dry_run_ns_per_splat=200.0) as srv:
        ids = [srv.submit(fake(200_000), 1000) for _ in range(4)]
        for j in ids:
            srv.wait(j, 30)
        iv = intervals(srv, ids)
        assert max(a for a, _ in iv) < min(b for _, b in iv)   # all four ran together
        assert len({srv.info(j)["slot"] for j in ids}) == 4


def test_small_jobs_queued_behind_a_run_form_one_group():
    with server(slots=1, group_small=1, small_rows=100_000, group_rows=1_000_000,
                dry_run_ns_per_splat=100.0) as srv:
        big = srv.submit(fake(2_000_000), 1000)              # occupies the only slot
        small = [srv.submit(fake(50_000), 5000) for _ in range(6)]
        tiny = srv.submit(fake(40_000), 10)                  # target <= k: never grouped
        for j in [big] + small + [tiny]:
            srv.wait(j, 30)
        groups = {srv.info(j)["group"] for j in small}
        assert len(groups) == 1 and srv.info(small[0])["group_size"] == 6
        assert srv.info(tiny)["group_size"] == 1
        assert srv.info(tiny)["start_s"] >= srv.info(small[0])["finish_s"] - 1e-9


def test_group_rows_cap_splits_groups():
    with server(slots=1, group_small=1, small_rows=100_000, group_rows=120_000,
                dry_run_ns_per_splat=100.0) as srv:
        big = srv.submit(fake(1_000_000), 1000)
        small = [srv.submit(fake(50_000), 5000) for _ in range(5)]
        for j in [big] + small:
            srv.wait(j, 30)
        sizes = [srv.info(j)["group_size"] for j in small]
        assert sizes == [2, 2, 2, 2, 1]


def test_job_above_budget_fails_at_submit():
    with server(hbm_budget_bytes=10_000_000) as srv:
        with pytest.raises(B.NgsError) as e:
            srv.submit(fake(20_000), 100)
        assert e.value.code == B.NGS_ERR_BUDGET
        assert srv.stats()["failed"] == 1


def test_bad_job_is_rejected():
    with server() as srv:
        with pytest.raises(B.NgsError):
            srv.submit(fake(1000), 0)
        s = fake(1000)
        s.cap = 10
        with pytest.raises(B.NgsError):
            srv.submit(s, 10)


def test_replay_submits_at_the_arrival_times():
    arrivals = [0.0, 0.05, 0.06, 0.2]
    with server(slots=2) as srv:
        t0 = srv.clock()
        ids = srv.replay([fake(10_000) for _ in arrivals], [100] * 4, arrivals)
        sub = [srv.info(j)["submit_s"] - t0 for j in ids]
        for s, a in zip(sub, arrivals):
            assert a - 1e-3 <= s <= a + 0.03
        assert all(srv.info(j)["status"] == B.NGS_JOB_DONE for j in ids)
        st = srv.stats()
        assert st["submitted"] == st["finished"] == 4 and st["queued"] == 0


def test_destroy_finishes_queued_jobs():
    srv = server(slots=1, group_small=0)
    ids = [srv.submit(fake(100_000), 10) for _ in range(3)]
    srv.close()   # must not hang; the jobs run to completion first
