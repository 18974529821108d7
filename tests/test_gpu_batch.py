"""Batching pattern: jobs of uneven lattice size and chi in one run
(mctrg_batch_run), their SVD stages in shared launches over matrices of
different sizes.

Each job's per-trajectory results and estimate must equal those of
mctrg_run with the same lattice, seed and counters, bit for bit (every
kernel treats items independently; the launch geometry the autotuner picks
does not change the arithmetic).  The autotuner's choices are kept in the
cache file and read back.
"""
import os

import numpy as np
import pytest

from paper_1710_03757_gb300 import build, mctrg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    mctrg.lib()


JOBS = [  # beta, h, L, chi, n_samples, seed, first_traj
    (0.44, 0.0, 16, 16, 24, 11, 0),
    (0.30, 0.05, 8, 4, 300, 12, 5),
    (0.50, 0.0, 32, 8, 64, 13, 0),
    (0.40, 0.1, 4, 2, 500, 14, 0),
    (0.35, 0.0, 32, 16, 8, 15, 100),
    (0.44, 0.02, 16, 8, 128, 16, 0),
    (0.60, 0.0, 2, 4, 10, 17, 0),          # every level exact
]


def solo(job, prec):
    beta, h, L, chi, n, seed, first = job
    ctx = mctrg.mctrg_create(mctrg.make_options(precision=prec))
    try:
        assert mctrg.mctrg_init_lattice(ctx, beta, h, L, chi) == 0
        ln, sg, fl = np.zeros(n), np.zeros(n, np.int8), np.zeros(n, np.uint8)
        st, est = mctrg.mctrg_run(ctx, n, seed, first, ln, sg, fl)
        return st, est, ln, sg, fl
    finally:
        mctrg.mctrg_destroy(ctx)


@pytest.mark.parametrize("prec", [mctrg.MCTRG_FP64, mctrg.MCTRG_FP64TC])
def test_batch_equals_solo_runs(tmp_path, prec):
    total = sum(j[4] for j in JOBS)
    ln, sg, fl = np.zeros(total), np.zeros(total, np.int8), np.zeros(total, np.uint8)
    cache = str(tmp_path / "tune.txt")
    st, ests = mctrg.mctrg_batch_run(JOBS, mctrg.make_options(precision=prec, autotune_cache=cache), ln, sg, fl)
    assert st == 0, mctrg.mctrg_strerror(st)
    assert os.path.exists(cache) and len(open(cache).read().split()) % 4 == 0
    off = 0
    for job, e in zip(JOBS, ests):
        n = job[4]
        st1, e1, l1, s1, f1 = solo(job, prec)
        np.testing.assert_array_equal(ln[off:off + n], l1)
        np.testing.assert_array_equal(sg[off:off + n], s1)
        np.testing.assert_array_equal(fl[off:off + n], f1)
        assert e.n == e1.n and e.sum_x == e1.sum_x and e.m2_x == e1.m2_x and e.ln_scale == e1.ln_scale
        assert e.ln_mean_Z == e1.ln_mean_Z or (np.isnan(e.ln_mean_Z) and np.isnan(e1.ln_mean_Z))
        off += n


def test_cached_choices_are_read_back(tmp_path):
    cache = tmp_path / "tune.txt"
    cache.write_text("256 16 304 1216\n64 8 152 1216\n")
    jobs = JOBS[:3]
    total = sum(j[4] for j in jobs)
    ln = np.zeros(total)
    st, ests = mctrg.mctrg_batch_run(jobs, mctrg.make_options(autotune_cache=str(cache)), ln)
    assert st == 0
    # the two shapes of these jobs were cached: nothing new was timed or written
    assert cache.read_text() == "256 16 304 1216\n64 8 152 1216\n"
    ln2 = np.zeros(total)
    st, _ = mctrg.mctrg_batch_run(jobs, mctrg.make_options(), ln2)   # no cache: tuned afresh
    assert st == 0
    np.testing.assert_array_equal(ln, ln2)


def test_batch_rejects_bad_arguments():
    assert mctrg.mctrg_batch_run([(0.4, 0.0, 8, 4, 0, 1, 0)])[0] == mctrg.MCTRG_EINVAL
    assert mctrg.mctrg_batch_run([(0.4, 0.0, 6, 4, 10, 1, 0)])[0] == mctrg.MCTRG_EINVAL
    assert mctrg.mctrg_batch_run([(0.4, 0.0, 8, 4, 10, 1, 0)],
                                 mctrg.make_options(precision=mctrg.MCTRG_TF32X3))[0] == mctrg.MCTRG_EINVAL
