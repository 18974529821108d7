"""CPU checks of the C-ABI library: it loads, exports every declared symbol,
and its host-side logic (TRG geometry, Philox stream, estimate merging)
agrees with the oracle.  No device work is issued."""
import ctypes
import glob
import math
import os
import re

import numpy as np
import pytest

from oracle import philox
from oracle.estimator import estimate
from oracle.network import plan
from paper_1710_03757_gb300 import build, mctrg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(mctrg_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert {"mctrg_run", "mctrg_init_lattice", "mctrg_create"} <= names
    lib = ctypes.CDLL(mctrg.LIB_PATH)
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert names == set(mctrg.EXPORTS)


def test_strerror():
    assert mctrg.mctrg_strerror(0) == "ok"
    assert "invalid" in mctrg.mctrg_strerror(mctrg.MCTRG_EINVAL)


@pytest.mark.parametrize("L", [2, 4, 8, 16, 32])
def test_geometry_matches_oracle(L):
    levels = plan(L)
    for k in range(len(levels) - 1):
        par, parents = mctrg.mctrg_plan_level(L, k)
        np.testing.assert_array_equal(par, levels[k].parity)
        np.testing.assert_array_equal(parents, levels[k].children_parents)


def test_geometry_rejects_bad_sizes():
    lib = mctrg.lib()
    assert lib.mctrg_plan_level(6, 0, None, None) == mctrg.MCTRG_EINVAL
    assert lib.mctrg_plan_level(4, 4, None, None) == mctrg.MCTRG_EINVAL


def test_philox_matches_oracle():
    for seed in (0, 1, 0x4D435453, 2 ** 64 - 1):
        for traj, level, tensor in ((0, 0, 0), (123, 5, 77), (2 ** 32 - 1, 19, 65535)):
            ref = philox.uniforms(seed, traj, level, tensor, 6)
            got = [mctrg.mctrg_philox_uniform(seed, traj, level, tensor, t) for t in range(6)]
            assert got == ref


def _est_from(sign, lnabs, scale=None):
    x_scale = np.max(lnabs[sign != 0]) if scale is None else scale
    x = np.where(sign != 0, sign * np.exp(np.where(sign != 0, lnabs, x_scale) - x_scale), 0.0)
    e = mctrg.Estimate()
    e.n = len(x)
    e.ln_scale = x_scale
    e.sum_x = x.sum()
    e.m2_x = np.sum((x - x.mean()) ** 2)
    e.n_negative = int(np.sum(sign < 0))
    return e


def test_merge_matches_oracle_on_whole_sample():
    rng = np.random.default_rng(4)
    lnabs = 500.0 + rng.normal(0, 2, 3000)
    sign = np.where(rng.random(3000) < 0.05, -1, 1).astype(np.int8)
    parts = [_est_from(sign[a:b], lnabs[a:b]) for a, b in ((0, 1000), (1000, 1700), (1700, 3000))]
    out = mctrg.mctrg_merge_estimates(parts)
    ref = estimate(sign, lnabs)
    assert out.n == 3000
    assert out.ln_scale == ref['ln_scale']
    assert out.mean_Z_scaled == pytest.approx(ref['mean_Z_scaled'], rel=1e-12)
    assert out.se_Z_scaled == pytest.approx(ref['se_Z_scaled'], rel=1e-10)
    assert out.ln_mean_Z == pytest.approx(ref['ln_mean_Z'], rel=1e-14)
    assert out.ess == pytest.approx(ref['ess'], rel=1e-10)
    assert out.n_negative == ref['n_negative']


def test_merge_rejects_empty():
    with pytest.raises(mctrg.MctrgError):
        mctrg.mctrg_merge_estimates([mctrg.Estimate()])


def test_create_rejects_bad_options_before_touching_the_device():
    # option checks come first, so they hold on a host without a GPU
    import ctypes
    lib = mctrg.lib()
    h = ctypes.c_void_p()
    for bad in (dict(precision=9), dict(svd=4), dict(svd=-1), dict(zero_tol_scale=-1.0),
                dict(zero_tol_scale=float("inf")), dict(zero_tol_scale=float("nan")),
                dict(deterministic_levels=-1)):
        o = mctrg.make_options(**bad)
        assert lib.mctrg_create(ctypes.byref(o), ctypes.byref(h)) == mctrg.MCTRG_EINVAL, bad
    assert lib.mctrg_create(None, ctypes.byref(h)) == mctrg.MCTRG_EINVAL


def test_ratio_estimate_matches_first_order_propagation():
    # two estimates from the oracle's estimator on synthetic per-trajectory values
    rng = np.random.default_rng(3)
    parts = []
    for shift in (0.0, 2.5):
        ln = rng.normal(10.0 + shift, 0.3, 500)
        sg = np.ones(500, np.int8)
        e = mctrg.Estimate()
        ref = estimate(sg, ln)
        x = np.exp(ln - ref['ln_scale'])
        e.n, e.ln_scale, e.mean_Z_scaled, e.se_Z_scaled = 500, ref['ln_scale'], x.mean(), x.std(ddof=1) / math.sqrt(500)
        parts.append((e, np.exp(ln)))
    st, r, se = mctrg.mctrg_ratio_estimate(parts[1][0], parts[0][0])
    assert st == 0
    a, b = parts[1][1], parts[0][1]
    exp_r = a.mean() / b.mean()
    exp_se = exp_r * math.hypot(a.std(ddof=1) / math.sqrt(500) / a.mean(), b.std(ddof=1) / math.sqrt(500) / b.mean())
    assert r == pytest.approx(exp_r, rel=1e-12) and se == pytest.approx(exp_se, rel=1e-10)
    bad = mctrg.Estimate()
    bad.n, bad.mean_Z_scaled = 10, -1.0
    assert mctrg.mctrg_ratio_estimate(parts[0][0], bad)[0] == mctrg.MCTRG_EDOMAIN
