"""Pins of the oracle's Philox4x32-10 stream (CPU only)."""
import os

import numpy as np

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((tuple(v[0:4]), tuple(v[4:6]), tuple(v[6:10])))
    return rows


def test_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert philox.philox4x32_10(ctr, key) == out


def test_uniform_mapping():
    # step t uses words (0,1) of block t>>1 for even t and (2,3) for odd t
    seed = 0x123456789ABCDEF
    x = philox.philox4x32_10((0, 5, 3, 11), (seed & 0xFFFFFFFF, seed >> 32))
    u = philox.uniforms(seed, 11, 3, 5, 2)
    assert u[0] == ((x[1] << 32 | x[0]) >> 11) * 2.0 ** -53
    assert u[1] == ((x[3] << 32 | x[2]) >> 11) * 2.0 ** -53


def test_uniform_statistics():
    u = np.array([v for t in range(200) for v in philox.uniforms(7, t, 1, 2, 16)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / len(u))
    # distinct counters give distinct streams
    assert philox.uniforms(7, 0, 1, 2, 4) != philox.uniforms(7, 1, 1, 2, 4)
    assert philox.uniforms(7, 0, 1, 2, 4) != philox.uniforms(7, 0, 2, 2, 4)
    assert philox.uniforms(7, 0, 1, 2, 4) != philox.uniforms(8, 0, 1, 2, 4)
