"""Serving loop: continuous batching of estimate jobs (mctrg_server_*).

Jobs that arrive while others run are admitted by device footprint as slots
and memory free up, and run concurrently on their own streams; each job's
trajectories use its own counters, so its result must be the same alone and
in any mix.  A job whose standard error, projected by 1/sqrt(N) (Sec. V, Eq.
shrunkDev), cannot reach its target within max_samples stops early."""
import math
import time

import numpy as np
import pytest

from oracle import ising
from paper_1710_03757_gb300 import build, mctrg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def _wait_all(srv, ids, timeout=300.0):
    out = {}
    for j in ids:
        st, est, lat = mctrg.mctrg_server_wait(srv, j, timeout)
        out[j] = (st, est, lat)
    return out


def test_jobs_reach_target_and_match_exact_z():
    srv = mctrg.mctrg_server_create()
    try:
        jobs = [(0.44, 0.0, 4, 2, 0.02), (0.3, 0.1, 4, 2, 0.02), (0.4, 0.0, 8, 4, 0.02), (0.5, 0.05, 4, 2, 0.01)]
        ids = []
        for b, h, L, chi, tgt in jobs:
            st, jid = mctrg.mctrg_server_submit(srv, b, h, L, chi, tgt, 1 << 18, 1000 + len(ids))
            assert st == 0
            ids.append(jid)
        res = _wait_all(srv, ids)
        for (b, h, L, chi, tgt), j in zip(jobs, ids):
            st, est, lat = res[j]
            assert st == 0, mctrg.mctrg_strerror(st)
            assert est.se_ln_Z <= tgt and lat > 0
            exact = ising.brute_force_lnZ(L, b, h) if L <= 4 else ising.kaufman_lnZ(L, b)
            z = math.exp(exact - est.ln_scale)
            assert abs(est.mean_Z_scaled - z) <= 3.5 * est.se_Z_scaled
    finally:
        mctrg.mctrg_server_destroy(srv)


def test_same_result_alone_and_in_a_mix():
    job = (0.44, 0.0, 16, 8, 0.01, 1 << 14, 77)
    srv = mctrg.mctrg_server_create()
    try:
        st, j = mctrg.mctrg_server_submit(srv, *job)
        assert st == 0
        st, alone, _ = mctrg.mctrg_server_wait(srv, j, 300.0)
        assert st == 0
    finally:
        mctrg.mctrg_server_destroy(srv)
    srv = mctrg.mctrg_server_create()
    try:
        others = []
        for k in range(6):
            st, o = mctrg.mctrg_server_submit(srv, 0.3 + 0.04 * k, 0.02 * k, 8 << (k % 2), 4 + 4 * (k % 2),
                                              0.01, 1 << 14, 500 + k)
            assert st == 0
            others.append(o)
        st, j = mctrg.mctrg_server_submit(srv, *job)
        assert st == 0
        st, mixed, _ = mctrg.mctrg_server_wait(srv, j, 300.0)
        assert st == 0
        _wait_all(srv, others)
    finally:
        mctrg.mctrg_server_destroy(srv)
    assert mixed.n == alone.n
    assert mixed.ln_mean_Z == alone.ln_mean_Z and mixed.se_ln_Z == alone.se_ln_Z
    assert mixed.sum_x == alone.sum_x and mixed.m2_x == alone.m2_x


def test_status_codes():
    srv = mctrg.mctrg_server_create()
    try:
        # the literal large configurations cannot be admitted: rejected at once
        t = time.time()
        st, _ = mctrg.mctrg_server_submit(srv, 0.44, 0.0, 65536, 32, 1e-6, 1 << 20, 1)
        assert st == mctrg.MCTRG_EUNREACHABLE and time.time() - t < 1.0
        assert mctrg.mctrg_server_submit(srv, 0.44, 0.0, 6, 4, 1e-2, 100, 1)[0] == mctrg.MCTRG_EINVAL
        assert mctrg.mctrg_server_poll(srv, 123456)[0] == mctrg.MCTRG_ENOTFOUND
        st, j = mctrg.mctrg_server_submit(srv, 0.44, 0.0, 32, 16, 1e-9, 1 << 12, 3)
        assert st == 0
        assert mctrg.mctrg_server_poll(srv, j)[0] == mctrg.MCTRG_EAGAIN
        assert mctrg.mctrg_server_wait(srv, j, 0.01)[0] == mctrg.MCTRG_ETIMEDOUT
        # a target that max_samples cannot reach: projected after the first
        # round (about half a second of work, 2 to 256 trajectories), result
        # returned, status says so
        st, est, lat = mctrg.mctrg_server_wait(srv, j, 300.0)
        assert st == mctrg.MCTRG_EUNREACHABLE and 2 <= est.n <= 256
        # destroying the server with a job still running is clean
        st, j2 = mctrg.mctrg_server_submit(srv, 0.44, 0.0, 32, 16, 1e-9, 1 << 14, 4)
        assert st == 0
    finally:
        mctrg.mctrg_server_destroy(srv)


def test_admission_by_footprint():
    # a budget of three jobs' footprints: the workers never hold more than the
    # budget (plus the shared-prefix buffers a plan does not count), all jobs
    # finish, and each equals its run on a server with room to spare
    job = lambda k: (0.3 + 0.02 * k, 0.0, 16, 8, 1e-9, 1 << 12, 900 + k)
    roomy = mctrg.mctrg_server_create()
    try:
        st, fp = mctrg.mctrg_server_footprint(roomy, 16, 8, 1 << 12)
        assert st == 0 and fp > 0
        ref = {}
        for k in range(8):
            st, j = mctrg.mctrg_server_submit(roomy, *job(k))
            ref[k] = j
        ref = {k: mctrg.mctrg_server_wait(roomy, j, 300.0)[1] for k, j in ref.items()}
    finally:
        mctrg.mctrg_server_destroy(roomy)
    budget = 3 * fp + fp // 2
    srv = mctrg.mctrg_server_create(mctrg.make_options(hbm_budget_bytes=budget))
    try:
        ids = {}
        for k in range(8):
            st, j = mctrg.mctrg_server_submit(srv, *job(k))
            assert st == 0
            ids[k] = j
        import threading
        peak, done = [0], threading.Event()

        def watch():
            while not done.is_set():
                b, r = mctrg.mctrg_server_memory(srv)
                assert b == budget
                peak[0] = max(peak[0], r)
                time.sleep(0.002)
        th = threading.Thread(target=watch)
        th.start()
        try:
            res = _wait_all(srv, list(ids.values()))
        finally:
            done.set()
            th.join()
    finally:
        mctrg.mctrg_server_destroy(srv)
    print("budget %d, peak held %d (footprint %d)" % (budget, peak[0], fp))
    assert 0 < peak[0] <= budget + (64 << 20)
    for k, j in ids.items():
        st, est, _ = res[j]
        assert st == mctrg.MCTRG_EUNREACHABLE
        assert est.n == ref[k].n and est.sum_x == ref[k].sum_x and est.m2_x == ref[k].m2_x


def test_literal_configurations_are_refused_fast():
    srv = mctrg.mctrg_server_create()
    try:
        t = time.time()
        # far beyond the device: refused at submission
        for L, chi in ((65536, 8), (4096, 32), (16384, 16)):
            assert mctrg.mctrg_server_submit(srv, 0.44, 0.0, L, chi, 1e-5, 1 << 18, 1)[0] == mctrg.MCTRG_EUNREACHABLE
        assert mctrg.mctrg_server_footprint(srv, 4096, 32, 1 << 18)[0] == mctrg.MCTRG_EUNREACHABLE
        # feasible lattices with targets far out of reach: stopped after the first round
        ids = [mctrg.mctrg_server_submit(srv, 0.44, 0.0, L, chi, tgt, 1 << 18, 2)[1]
               for L, chi, tgt in ((256, 8, 1e-5), (512, 8, 1e-6), (256, 16, 1e-6))]
        for j in ids:
            st, est, lat = mctrg.mctrg_server_wait(srv, j, 600.0)
            # one first round: about half a second of work, at most 256 trajectories
            assert st == mctrg.MCTRG_EUNREACHABLE and est.n <= 64
        print("literal jobs refused or projected out of reach in %.1f s" % (time.time() - t))
    finally:
        mctrg.mctrg_server_destroy(srv)


def test_fixed_sample_job_runs_exactly_max_samples():
    # target 0: no early stop; the rounds (256, 512, then the rest) merge to the
    # estimate of one run over the same counters (to the rounding of the merge)
    srv = mctrg.mctrg_server_create()
    try:
        st, j = mctrg.mctrg_server_submit(srv, 0.44, 0.0, 16, 8, 0.0, 1000, 21)
        assert st == 0
        st, est, _ = mctrg.mctrg_server_wait(srv, j, 300.0)
        assert st == mctrg.MCTRG_OK and est.n == 1000
    finally:
        mctrg.mctrg_server_destroy(srv)
    ctx = mctrg.mctrg_create()
    try:
        assert mctrg.mctrg_init_lattice(ctx, 0.44, 0.0, 16, 8) == 0
        st, ref = mctrg.mctrg_run(ctx, 1000, 21, 0)
    finally:
        mctrg.mctrg_destroy(ctx)
    assert abs(est.ln_mean_Z - ref.ln_mean_Z) <= 1e-13 * abs(ref.ln_mean_Z)
    assert abs(est.se_ln_Z - ref.se_ln_Z) <= 1e-10 * ref.se_ln_Z
    assert est.n_negative == ref.n_negative and est.n_flagged == ref.n_flagged
