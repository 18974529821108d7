"""Monte Carlo estimate of Z from per-trajectory results (oracle).

Test infrastructure only: nothing on the product path may import this module.

Sec. III, Eq. infiniteEnsemble: the sample mean of Z~ estimates Z without bias;
Sec. V, Eq. shrunkDev: its error falls as 1/sqrt(N).  Per-trajectory values
arrive as (sign, ln|Z~|) because Z~ overflows double precision at large L.
With m = max ln|Z~_i| and x_i = sign_i exp(ln|Z~_i| - m):
    Z^ = e^m mean(x),  SE(Z^) = e^m std(x, ddof=1) / sqrt(N),
    ln Z^ = m + ln mean(x)  (only if mean(x) > 0),  SE(ln Z^) = SE / Z^,
    ESS = (sum x)^2 / sum x^2.
Unbiasedness holds for Z^, not for ln Z^.
"""
import math

import numpy as np


def estimate(sign, lnabs):
    sign = np.asarray(sign, dtype=np.float64)
    lnabs = np.asarray(lnabs, dtype=np.float64)
    n = len(sign)
    ok = sign != 0
    m = float(np.max(lnabs[ok])) if np.any(ok) else 0.0
    x = np.where(ok, sign * np.exp(np.where(ok, lnabs, m) - m), 0.0)
    mean = float(np.mean(x)) if n else math.nan
    sd = float(np.std(x, ddof=1)) if n > 1 else math.nan
    se = sd / math.sqrt(n) if n > 1 else math.nan
    out = {
        'n': n, 'ln_scale': m, 'mean_Z_scaled': mean, 'se_Z_scaled': se,
        'n_negative': int(np.sum(sign < 0)),
        'ess': float(np.sum(x) ** 2 / np.sum(x * x)) if np.any(x != 0) else 0.0,
    }
    if mean > 0:
        out['ln_mean_Z'] = m + math.log(mean)
        out['se_ln_Z'] = se / mean
    else:
        out['ln_mean_Z'] = math.nan
        out['se_ln_Z'] = math.nan
    return out
