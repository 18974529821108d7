"""Philox4x32-10 counter-based generator, host side (oracle copy).

Test infrastructure only: nothing on the product path may import this module.

Written from the published definition (Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 3.3): ten rounds of
two 32x32->64 multiplies on the even words, xor with the odd words and the
round key, and a Weyl-sequence key schedule.  The paper being implemented
(Sec. II) needs independent uniforms per tensor and per trajectory; the
counter layout below makes trajectory i a pure function of (seed, i).

Counter layout used by both the oracle and the device path:
  key     = (seed mod 2^32, seed >> 32)
  counter = (t >> 1, tensor, level, trajectory)
where t is the draw step of one tensor's sampler.  Step t takes the 64-bit
word (x[2(t&1)+1] << 32 | x[2(t&1)]), keeps its top 53 bits, and scales by
2^-53, giving a uniform in [0, 1).
"""

MASK32 = 0xFFFFFFFF
_M0, _M1 = 0xD2511F53, 0xCD9E8D57          # round multipliers
_W0, _W1 = 0x9E3779B9, 0xBB67AE85          # key-schedule increments


def philox4x32_10(ctr, key):
    """One Philox4x32 block with 10 rounds; ctr = 4 words, key = 2 words."""
    x0, x1, x2, x3 = (int(c) & MASK32 for c in ctr)
    k0, k1 = (int(k) & MASK32 for k in key)
    for _ in range(10):
        p0 = _M0 * x0
        p1 = _M1 * x2
        x0, x1, x2, x3 = ((p1 >> 32) ^ x1 ^ k0, p1 & MASK32,
                          (p0 >> 32) ^ x3 ^ k1, p0 & MASK32)
        k0 = (k0 + _W0) & MASK32
        k1 = (k1 + _W1) & MASK32
    return (x0, x1, x2, x3)


def uniforms(seed, traj, level, tensor, count):
    """The first `count` sampler uniforms of one tensor (float64 in [0,1))."""
    key = (seed & MASK32, (seed >> 32) & MASK32)
    out = []
    for t in range(count):
        x = philox4x32_10((t >> 1, tensor, level, traj), key)
        lo, hi = (x[0], x[1]) if (t & 1) == 0 else (x[2], x[3])
        out.append(((hi << 32 | lo) >> 11) * 2.0 ** -53)
    return out
