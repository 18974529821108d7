"""Per-trajectory comparison of the CUDA path with the oracle (test helper).

Both sides consume the same Philox stream, so a trajectory's kept index sets,
sign and ln|Z~| agree unless a near-tie makes two correct implementations keep
different indices; such trajectories carry flags (kept and dropped singular
values closer than 1e-8 s_1, a uniform within 1e-9 of a CDF step, a kept
value below 1e-7 s_1).  The flags are computed from quantities that the two
sides know to about 1e-15 relative, against thresholds of 1e-9 and above, so
they must agree too:

  * a trajectory is flagged on both sides or on neither, and where both flag
    it, the two flag words share at least one bit (the near-tie that both saw
    first; after it the kept sets may differ and later flags with them);
  * the one stated exception: a trajectory flagged on one side only whose
    flags include a kept value below 1e-7 s_1.  That side sampled singular
    values at the rounding-noise level of a (numerically) rank-deficient
    matrix, e.g. [1, 2.7e-13, 1.2e-14, 6e-17] where the matrix has rank 1;
    the other SVD's noise values fell below the zero threshold n 2^-52 s_1,
    so it kept all its "nonzero" values without sampling and raised no flag.
    Which noise values clear the threshold is not determined by the
    mathematics, so such trajectories are counted and printed, held to at
    most 1% of the trajectories, and excluded from the value comparison;
  * every unflagged trajectory has the same sign and
    |ln|Z~|_gpu - ln|Z~|_oracle| <= 1e-10 max(1, |ln|Z~||)  (Q16: the
    tolerance of ln Z per trajectory, FP64 on both sides);
  * the count of negative trajectories agrees exactly on the unflagged ones,
    and the device estimate counts its own negative and flagged trajectories;
  * the device estimate (its reductions run in the estimator kernel) equals
    the oracle's estimator (Sec. III, Eq. infiniteEnsemble; Sec. V, Eq.
    shrunkDev) applied to the GPU's own per-trajectory outputs, to 1e-13.

min_ok is the smallest fraction of unflagged trajectories a case accepts;
each caller states where its floor comes from.
"""
import math

import numpy as np

from oracle.estimator import estimate

TOL = 1e-10
EST_TOL = 1e-13
FLAG_TINY_KEPT = 4


def _rel(a, b, scale):
    return abs(a - b) / max(scale, 1e-300)


def check_estimate(est, sign, lnabs, flags=None):
    """The device estimate against the oracle's estimator on the same outputs."""
    ref = estimate(sign, lnabs)
    assert est.n == ref['n']
    assert est.n_negative == ref['n_negative'] == int(np.sum(sign < 0))
    if flags is not None:
        assert est.n_flagged == int(np.sum(flags != 0))
    assert est.ln_scale == ref['ln_scale']
    ok = sign != 0
    x = np.where(ok, sign * np.exp(np.where(ok, lnabs, ref['ln_scale']) - ref['ln_scale']), 0.0)
    scale_x = float(np.mean(np.abs(x))) if len(x) else 1.0
    assert _rel(est.mean_Z_scaled, ref['mean_Z_scaled'], scale_x) <= EST_TOL
    assert _rel(est.sum_x, est.n * ref['mean_Z_scaled'], est.n * scale_x) <= EST_TOL
    if est.n > 1:
        m2 = ref['se_Z_scaled'] ** 2 * est.n * (est.n - 1)
        assert _rel(est.m2_x, m2, max(m2, 1e-300)) <= 1e-12
        assert _rel(est.se_Z_scaled, ref['se_Z_scaled'], ref['se_Z_scaled']) <= 1e-12
        assert _rel(est.ess, ref['ess'], ref['ess']) <= 1e-12
    if ref['mean_Z_scaled'] > 0 and math.isfinite(ref['ln_mean_Z']):
        assert _rel(est.ln_mean_Z, ref['ln_mean_Z'], max(1.0, abs(ref['ln_mean_Z']))) <= EST_TOL
        if est.n > 1:
            assert _rel(est.se_ln_Z, ref['se_ln_Z'], ref['se_ln_Z']) <= 1e-12
    else:
        assert math.isnan(est.ln_mean_Z)


def compare(gpu, orc, min_ok, label=""):
    """gpu = (estimate, lnabs, sign, flags) from mctrg_run; orc = (sign, lnabs,
    flags) from oracle.trg.run_many.  Returns the number of trajectories
    compared value by value."""
    est, gl, gs, gf = gpu
    os_, ol, of = orc
    n = len(gl)
    fg, fo = gf != 0, of != 0
    one_sided = np.flatnonzero(fg != fo)
    noise = one_sided[((gf | of)[one_sided] & FLAG_TINY_KEPT) != 0]
    other = np.setdiff1d(one_sided, noise)
    disjoint = np.flatnonzero(fg & fo & ((gf & of) == 0))
    print("%s parity: %d trajectories, %d flagged (gpu) / %d (oracle), flag rate %.3f, "
          "%d flagged on one side only with noise-level kept values %s"
          % (label, n, int(fg.sum()), int(fo.sum()), float(fg.mean()) if n else 0.0, noise.size,
             noise[:10].tolist()))
    assert other.size == 0, "flagged on one side only: %s (gpu flags %s, oracle flags %s)" % (
        other[:10].tolist(), gf[other[:10]].tolist(), of[other[:10]].tolist())
    assert noise.size <= max(1, n // 100), "noise-level one-sided flags at %s" % noise[:10].tolist()
    assert disjoint.size == 0, "flag words without a common bit at %s" % disjoint[:10].tolist()
    ok = ~fg & ~fo
    assert ok.mean() >= min_ok, "too many flagged trajectories: %d of %d" % (int((~ok).sum()), n)
    np.testing.assert_array_equal(gs[ok], os_[ok])
    nz = ok & (os_ != 0)
    if nz.any():
        err = np.abs(gl[nz] - ol[nz]) / np.maximum(1.0, np.abs(ol[nz]))
        assert err.max() <= TOL, "max rel err %.3e at %d" % (err.max(), int(np.flatnonzero(nz)[np.argmax(err)]))
    # negative trajectories: identical where unflagged; the flagged ones that differ are listed
    assert int(np.sum(gs[ok] < 0)) == int(np.sum(os_[ok] < 0))
    diff = np.flatnonzero(~ok & ((gs < 0) != (os_ < 0)))
    if diff.size:
        print("%s: sign differs on flagged trajectories %s" % (label, diff[:20].tolist()))
    check_estimate(est, gs, gl, gf)
    return int(ok.sum())
