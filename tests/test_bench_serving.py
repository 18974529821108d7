"""The bench's serving leg against a fake server on the host: the arrival rate,
the job size scaled to the offered load, and the literal jobs (those the
footprint admits are reported, not run; the others are refused at submission)."""
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Est:
    def __init__(self, n):
        self.n = n


def _fake_mctrg(trajectories_per_job_cap=None):
    m = types.SimpleNamespace()
    m.MCTRG_OK, m.MCTRG_ETIMEDOUT, m.MCTRG_EUNREACHABLE = 0, -7, -9
    jobs = {}
    submitted = []

    def submit(srv, beta, h, L, chi, target, max_samples, seed):
        if L > 4096:                                   # beyond the fake device
            return m.MCTRG_EUNREACHABLE, 0
        j = len(jobs) + 1
        jobs[j] = max_samples
        submitted.append((L, chi, max_samples))
        return 0, j

    def wait(srv, j, timeout):
        n = jobs.pop(j)
        return (m.MCTRG_EUNREACHABLE if n < 1000 else 0), _Est(n), 1e-3

    m.mctrg_server_create = lambda: object()
    m.mctrg_server_destroy = lambda srv: None
    m.mctrg_server_submit = submit
    m.mctrg_server_wait = wait
    m.mctrg_server_footprint = lambda srv, L, chi, n: (0, 1) if L <= 4096 else (m.MCTRG_EUNREACHABLE, 0)
    m.submitted = submitted
    return m


def test_serving_leg_scales_job_size_to_the_offered_load():
    m = _fake_mctrg()
    out = bench.measure_serving(m, 0.05, load=0.7, literal_jobs=6, burst_jobs=4)
    # arrivals at the stated rate, each job capped so that they offer 70% of the capacity
    assert out["arrivals_per_s"] <= bench.SERVE_ARRIVALS_PER_S
    cap = out["capacity_trajectories_per_s"]
    expect = int(min(bench.SERVE_MAX_SAMPLES, max(4, round(0.7 * cap / bench.SERVE_ARRIVALS_PER_S))))
    assert out["sample_cap_per_job"] == expect
    mix = [s for s in m.submitted if s[0] <= 32]
    assert all(n == expect for _, _, n in mix[4 + 32:])          # after the two bursts
    assert out["jobs"] == len(mix) - 4 - 32
    assert out["latency_p50_s"] is not None and out["jobs_unfinished_after_drain"] == 0
    # literal jobs: admissible ones reported, not submitted; the rest refused at submission
    lit = out["literal_jobs"]
    assert len(lit["admissible_not_run"]) + lit["refused_at_submit"] == 6
    assert not [s for s in m.submitted if s[0] >= 256]
    assert all(x < 1.0 for x in lit["latency_s"])
