"""Serving runtime (include/svt_serve.h) on CPU: dry-run servers touch no device, each job sleeps
for its given duration and occupies its given footprint.  Checked: admission by slots and memory
(never more in flight than either allows), strict first-in first-out order, refusal of a job
larger than the whole budget, latency accounting from arrival (p50 / p99 by nearest rank), drain
and the throughput figure."""
import time

import pytest

from paper_0810_3286_gb300._abi import SVTError


def _server(**kw):
    from paper_0810_3286_gb300.serve import Server
    return Server(dry_run=True, **kw)


def test_slots_bound_jobs_in_flight():
    with _server(slots=3) as s:
        ids = [s.submit(100, 100, nnz=10, dry_run_us=30000, dry_run_bytes=1) for _ in range(9)]
        s.drain()
        st = s.stats()
        assert st["completed"] == 9 and st["failed"] == 0
        assert st["peak_running"] == 3
        res = [s.wait(i) for i in ids]
    # FIFO: starts in submission order
    starts = [r["t_start_ms"] for r in res]
    assert starts == sorted(starts)
    # three waves of three jobs of 30 ms: the last job cannot start before ~60 ms
    assert res[-1]["t_start_ms"] - res[0]["t_start_ms"] >= 55.0


def test_memory_budget_bounds_bytes_in_flight_and_head_of_line_waits():
    with _server(slots=8, device_budget=100) as s:
        big = s.submit(10, 10, nnz=5, dry_run_us=40000, dry_run_bytes=70)
        mid = s.submit(10, 10, nnz=5, dry_run_us=40000, dry_run_bytes=60)     # must wait for big
        small = s.submit(10, 10, nnz=5, dry_run_us=1000, dry_run_bytes=10)    # fits, but is behind mid
        s.drain()
        st = s.stats()
        r_big, r_mid, r_small = s.wait(big), s.wait(mid), s.wait(small)
    assert st["peak_bytes"] <= 100
    assert r_mid["t_start_ms"] >= r_big["t_end_ms"] - 1.0
    assert r_small["t_start_ms"] >= r_mid["t_start_ms"]            # strict FIFO
    assert r_small["t_start_ms"] < r_mid["t_end_ms"]               # ...and then it runs beside mid


def test_job_above_budget_is_refused():
    with _server(slots=2, device_budget=50) as s:
        with pytest.raises(SVTError):
            s.submit(10, 10, nnz=5, dry_run_us=10, dry_run_bytes=51)
        ok = s.submit(10, 10, nnz=5, dry_run_us=10, dry_run_bytes=50)
        assert s.wait(ok)["status"] == 0


def test_latency_percentiles_from_arrival():
    with _server(slots=1) as s:
        # one slot, ten 20 ms jobs submitted at once: latency of the k-th job is ~ 20 k ms
        ids = [s.submit(10, 10, nnz=5, dry_run_us=20000, dry_run_bytes=1) for _ in range(10)]
        s.drain()
        st = s.stats()
        lat = sorted(r["t_end_ms"] - r["t_submit_ms"] for r in (s.wait(i) for i in ids))
    assert st["p50_ms"] == pytest.approx(lat[4], abs=1e-6)      # nearest rank: ceil(0.5 * 10) = 5th
    assert st["p99_ms"] == pytest.approx(lat[9], abs=1e-6)      # ceil(0.99 * 10) = 10th
    assert 180.0 <= lat[9] <= 400.0
    # throughput: 10 jobs over (last completion - first arrival) ~ 200 ms of one slot
    assert 25.0 <= st["solves_per_s"] <= 52.0


def test_invalid_jobs_rejected():
    with _server(slots=1) as s:
        with pytest.raises(SVTError):
            s.submit(0, 10, nnz=5)
        with pytest.raises(SVTError):
            s.submit(3, 3, nnz=10)
