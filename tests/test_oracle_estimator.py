"""Pins of the oracle's estimator (Sec. III Eq. infiniteEnsemble, Sec. V Eq. shrunkDev)."""
import math

import numpy as np
import pytest

from oracle.estimator import estimate


def test_matches_direct_statistics():
    rng = np.random.default_rng(0)
    z = rng.lognormal(0.0, 0.7, 500) * np.where(rng.random(500) < 0.1, -1, 1)
    e = estimate(np.sign(z), np.log(np.abs(z)))
    scale = math.exp(e['ln_scale'])
    assert e['mean_Z_scaled'] * scale == pytest.approx(z.mean(), rel=1e-13)
    assert e['se_Z_scaled'] * scale == pytest.approx(z.std(ddof=1) / math.sqrt(500), rel=1e-12)
    assert e['n_negative'] == int(np.sum(z < 0))
    assert e['ln_mean_Z'] == pytest.approx(math.log(z.mean()), rel=1e-13)
    assert e['ess'] == pytest.approx(z.sum() ** 2 / np.sum(z * z), rel=1e-12)


def test_huge_values_do_not_overflow():
    lnabs = np.array([5000.0, 5001.0, 4999.5])
    e = estimate(np.ones(3), lnabs)
    ref = 5001.0 + math.log(np.mean(np.exp(lnabs - 5001.0)))
    assert e['ln_mean_Z'] == pytest.approx(ref, rel=1e-15)


def test_zero_samples_and_negative_mean():
    e = estimate(np.array([1, 0, -1, -1]), np.array([0.0, -np.inf, 0.0, 0.0]))
    assert e['mean_Z_scaled'] == pytest.approx(-0.25)
    assert math.isnan(e['ln_mean_Z'])
