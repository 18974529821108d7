"""Serving loop: continuous batching of estimate jobs (mctrg_server_*).

Jobs that arrive while others run are admitted as device memory frees up and
run concurrently on their own streams; each job's trajectories use its own
counters, so its result must be the same alone and in any mix."""
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
        # a target that max_samples cannot reach: result returned, status says so
        st, est, lat = mctrg.mctrg_server_wait(srv, j, 300.0)
        assert st == mctrg.MCTRG_EUNREACHABLE and est.n == 1 << 12
        # destroying the server with a job still running is clean
        st, j2 = mctrg.mctrg_server_submit(srv, 0.44, 0.0, 32, 16, 1e-9, 1 << 14, 4)
        assert st == 0
    finally:
        mctrg.mctrg_server_destroy(srv)
