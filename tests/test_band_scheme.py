"""The arithmetic the band SVD route's tensor-core products rest on, checked
on the host in plain integer arithmetic (no code shared with the kernels):

* balanced 8-bit digits of a 64-bit integer are the bytes of one sum,
  x + 0x8080808080808080, less 128 each;
* the digit products of one group g = i + j, summed over K, stay within the
  range FP32 holds exactly (2^24) for the trailing update (K = 16, every group)
  and for the first four groups of the K = 256 products;
* two biased FP32 readbacks (integer + 1.5 * 2^23) pair into G0 * 2^8 + G1
  in 32-bit two's complement after one constant subtraction;
* eight digit slices with the groups of weight >= 2^-64 reproduce a product of
  59- and 62-bit fixed-point operands more accurately than the same product
  in FP64 arithmetic, while seven slices (56 bits) fall well short of it.
"""
import numpy as np


def balanced_digits(x, nd=8):
    """digits d_0 (top) .. d_{nd-1} of x, each in [-128, 127], sum d_i 256^(nd-1-i) = x"""
    y = (x + sum(0x80 << (8 * i) for i in range(nd))) & ((1 << (8 * nd)) - 1)
    return [((y >> (8 * (nd - 1 - i))) & 0xFF) - 128 for i in range(nd)]


def test_balanced_digits_are_the_bytes_of_one_sum():
    rng = np.random.default_rng(1)
    xs = [int(v) for v in rng.integers(-(1 << 62), 1 << 62, 2000)] + [0, 1, -1, (1 << 62) - 1, -(1 << 62)]
    for x in xs:
        d = balanced_digits(x)
        assert all(-128 <= v <= 127 for v in d)
        assert sum(v * 256 ** (7 - i) for i, v in enumerate(d)) == x
        assert abs(d[0]) <= 64                       # a 62-bit value leaves a small top digit


def _group_bound(K, top_a, top_b, g):
    # |sum_K sum_{i+j=g} a_i b_j| with |a_0| <= top_a, |b_0| <= top_b, other digits <= 128
    tot = 0
    for i in range(g + 1):
        j = g - i
        tot += (top_a if i == 0 else 128) * (top_b if j == 0 else 128)
    return K * tot


def test_group_sums_stay_exact_in_fp32():
    # trailing update: both operands 62-bit (top digits <= 64), K = 16: every group below 2^22
    assert max(_group_bound(16, 64, 64, g) for g in range(8)) < 1 << 22
    # W and X: the 59-bit trailing matrix (top digit <= 8) against V or U (entries <= 1 at 61
    # bits: top digit <= 32), K <= 256: groups 0..3 at most 2^24 (exact); the later ones may round
    assert max(_group_bound(256, 8, 32, g) for g in range(4)) <= 1 << 24
    # the FP32 readback of the update, x + 1.5 2^23, is exact for |x| <= 2^22
    for G in (0, 1, -1, (1 << 21), -(1 << 21), 12345, -777777):
        f = np.float32(G) + np.float32(12582912.0)
        assert int(f.view(np.int32)) - 0x4B400000 == G


def test_biased_readbacks_pair_in_32_bits():
    rng = np.random.default_rng(2)
    B = 0x4B400000
    for _ in range(20000):
        g0, g1 = (int(v) for v in rng.integers(-(1 << 21), (1 << 21) + 1, 2))
        b0, b1 = (g0 + B) & 0xFFFFFFFF, (g1 + B) & 0xFFFFFFFF
        v = (b0 * 256 + b1 - B * 257) & 0xFFFFFFFF
        v = v - (1 << 32) if v >= 1 << 31 else v
        assert v == g0 * 256 + g1


def _digit_product(A, Bm, nd):
    """sum over groups g <= nd - 1 of the digit products, as an exact integer matrix, for integer
    matrices A (m x K) and Bm (K x n); each operand cut to its top nd digits first"""
    m, K = A.shape
    n = Bm.shape[1]
    sh = 8 * (8 - nd)
    Ad = np.array([[balanced_digits(int(v) >> sh, nd) for v in row] for row in A], dtype=np.int64)
    Bd = np.array([[balanced_digits(int(v) >> sh, nd) for v in row] for row in Bm], dtype=np.int64)
    out = [[0] * n for _ in range(m)]
    for g in range(nd):
        G = np.zeros((m, n), dtype=np.int64)
        for i in range(g + 1):
            G += Ad[:, :, i] @ Bd[:, :, g - i]
        w = 256 ** (2 * nd - 2 - g) * (1 << (2 * sh))
        for r in range(m):
            for c in range(n):
                out[r][c] += int(G[r, c]) * w
    return out


def test_eight_slices_beat_an_fp64_product_seven_do_not():
    # the same product three ways against the exact integer result, each error relative to
    # the products' normwise scale K max|a| max|b|: in FP64 arithmetic (operands rounded to
    # 53 bits, then a float64 matmul), with eight digit slices, with seven
    rng = np.random.default_rng(3)
    K = 64
    for _ in range(3):
        A = rng.integers(-(1 << 58), 1 << 58, (6, K))          # fixed-point trailing matrix
        Bm = rng.integers(-(1 << 61), 1 << 61, (K, 5))         # an FP64 operand at 62 bits
        exact = [[sum(int(A[r, k]) * int(Bm[k, c]) for k in range(K)) for c in range(5)] for r in range(6)]
        scale = K * (1 << 58) * (1 << 61)

        def err(got):
            return max(abs(a - b) for ra, rb in zip(got, exact) for a, b in zip(ra, rb)) / scale

        f64 = (A.astype(np.float64) / 2.0 ** 58) @ (Bm.astype(np.float64) / 2.0 ** 61)
        e_f64 = err([[int(round(float(v) * 2.0 ** 119)) for v in row] for row in f64])
        e8, e7 = err(_digit_product(A, Bm, 8)), err(_digit_product(A, Bm, 7))
        assert e8 < 0.25 * e_f64      # measured: about 10x below
        assert e7 > 4.0 * e_f64       # measured: about 20x above
