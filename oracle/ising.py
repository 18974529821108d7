"""2D Ising model: site tensor and exact partition functions (oracle).

Test infrastructure only: nothing on the product path may import this module.

Model (Sec. IV, Eq. ising_model, extended by a uniform field h):
    Z = sum_{sigma} exp( beta * sum_<ij> s_i s_j + beta * h * sum_i s_i )
on an L x L periodic square lattice, J = k_B = 1, beta = 1/T.

Exact references used to pin the Monte Carlo estimator:
  * brute_force_lnZ    - direct sum over all 2^(L*L) states (L <= 4)
  * transfer_lnZ       - row transfer matrix, Z = Tr T^L (L <= 10)
  * kaufman_lnZ        - Kaufman's closed form for the finite torus, h = 0
  * onsager_minus_beta_f - Onsager's free energy per site, h = 0, L -> inf
"""
import itertools
import math

import numpy as np


def site_tensor(beta, h):
    """T[l,u,r,d] = sum_s e^{beta h s} W[s,l] W[s,u] W[s,r] W[s,d].

    The bond weight e^{beta s s'} = sum_a W[s,a] W[s',a] with
    W[s,0] = sqrt(cosh beta), W[s,1] = s sqrt(sinh beta); index s = 0 is spin
    +1 and s = 1 is spin -1.  Each bond of the lattice is shared by the r leg
    of one site and the l leg of its right neighbour (d and u vertically), so
    the trace of the network of these tensors is Z.
    """
    W = np.array([[math.sqrt(math.cosh(beta)), math.sqrt(math.sinh(beta))],
                  [math.sqrt(math.cosh(beta)), -math.sqrt(math.sinh(beta))]])
    T = np.zeros((2, 2, 2, 2))
    for s, spin in enumerate((1.0, -1.0)):
        w = W[s]
        T += math.exp(beta * h * spin) * np.einsum('a,b,c,d->abcd', w, w, w, w)
    return T


def impurity_tensor(beta, h):
    """The site tensor with the site's spin inserted (the impurity of Sec. III's
    partial traces): T_imp[l,u,r,d] = sum_s s e^{beta h s} W[s,l] W[s,u] W[s,r] W[s,d].
    Replacing site i's tensor by it gives sum_sigma sigma_i e^{-beta H} = Z <sigma_i>."""
    W = np.array([[math.sqrt(math.cosh(beta)), math.sqrt(math.sinh(beta))],
                  [math.sqrt(math.cosh(beta)), -math.sqrt(math.sinh(beta))]])
    T = np.zeros((2, 2, 2, 2))
    for s, spin in enumerate((1.0, -1.0)):
        w = W[s]
        T += spin * math.exp(beta * h * spin) * np.einsum('a,b,c,d->abcd', w, w, w, w)
    return T


def brute_force_observable(L, beta, h, sites):
    """<prod_{i in sites} sigma_i> and ln Z by enumerating every configuration;
    a site is (x, y)."""
    n = L * L
    if n > 20:
        raise ValueError("brute force limited to L*L <= 20")
    idx = np.arange(1 << n, dtype=np.int64)
    spins = (1 - 2 * ((idx[:, None] >> np.arange(n)) & 1)).reshape(-1, L, L)   # [state, y, x]
    bonds = (spins * np.roll(spins, -1, axis=2)).sum(axis=(1, 2)) \
        + (spins * np.roll(spins, -1, axis=1)).sum(axis=(1, 2))
    e = beta * bonds + beta * h * spins.sum(axis=(1, 2))
    w = np.exp(e - e.max())
    obs = np.ones(len(idx))
    for x, y in sites:
        obs = obs * spins[:, y, x]
    return float(np.sum(w * obs) / np.sum(w)), _logsumexp(e)


def transfer_observable(L, beta, h, columns):
    """<prod_{x in columns} sigma_(x, 0)> on the L x L torus (L <= 10) from the row
    transfer matrix: Tr(S T^L) / Tr(T^L), S the diagonal of the product of the
    row's spins at those columns (any row: translation invariance)."""
    if L > 10:
        raise ValueError("transfer matrix limited to L <= 10")
    rows = list(itertools.product((1, -1), repeat=L))
    R = np.array(rows, dtype=np.float64)
    intra = (R * np.roll(R, -1, axis=1)).sum(axis=1)
    field = R.sum(axis=1)
    logT = beta * (R @ R.T) + beta * (intra + h * field)[:, None]
    T = np.exp(logT - logT.max())
    P = np.linalg.matrix_power(T / np.linalg.norm(T, 2), L)
    S = np.prod(R[:, list(columns)], axis=1)
    return float(np.sum(S * np.diag(P)) / np.trace(P))


def _logsumexp(x):
    m = np.max(x)
    return float(m + np.log(np.sum(np.exp(x - m))))


def brute_force_lnZ(L, beta, h=0.0):
    """ln Z by enumerating every spin configuration (2^(L^2) states)."""
    n = L * L
    if n > 20:
        raise ValueError("brute force limited to L*L <= 20")
    idx = np.arange(1 << n, dtype=np.int64)
    spins = 1 - 2 * ((idx[:, None] >> np.arange(n)) & 1)          # (states, n)
    spins = spins.reshape(-1, L, L)                                 # [state, y, x]
    bonds = (spins * np.roll(spins, -1, axis=2)).sum(axis=(1, 2)) \
        + (spins * np.roll(spins, -1, axis=1)).sum(axis=(1, 2))
    mag = spins.sum(axis=(1, 2))
    return _logsumexp(beta * bonds + beta * h * mag)


def transfer_lnZ(L, beta, h=0.0):
    """ln Z = ln Tr(T^L) with the 2^L x 2^L row-to-row transfer matrix."""
    if L > 10:
        raise ValueError("transfer matrix limited to L <= 10")
    rows = list(itertools.product((1, -1), repeat=L))
    R = np.array(rows, dtype=np.float64)                            # (2^L, L)
    intra = (R * np.roll(R, -1, axis=1)).sum(axis=1)                # horizontal bonds
    field = R.sum(axis=1)
    inter = R @ R.T                                                 # vertical bonds
    logT = beta * inter + beta * (intra + h * field)[:, None]
    # T[R,R'] carries row R's horizontal bonds and field plus the R-R' vertical bonds
    shift = logT.max()
    T = np.exp(logT - shift)
    ev = np.linalg.eigvals(T)
    s = np.sum(ev.astype(np.complex128) ** L)
    return float(L * shift + np.log(s.real))


def kaufman_lnZ(L, beta, M=None):
    """ln Z of the h = 0 Ising model on an M x L torus (M rows, default M = L).

    Kaufman, Phys. Rev. 76, 1232 (1949):
      Z = 1/2 (2 sinh 2K)^{ML/2} (Z1 + Z2 + Z3 + Z4),
      Z1 = prod_{r<L} 2 cosh(M g_{2r+1}/2),  Z2 = prod 2 sinh(M g_{2r+1}/2),
      Z3 = prod_{r<L} 2 cosh(M g_{2r}/2),    Z4 = prod 2 sinh(M g_{2r}/2),
      cosh g_k = cosh 2K coth 2K - cos(pi k / L)  (g_k > 0, k != 0),
      g_0 = 2K + ln tanh K  (signed).
    Evaluated with signed logarithms so that large L does not overflow.
    """
    if M is None:
        M = L
    K = float(beta)
    c = math.cosh(2 * K) / math.tanh(2 * K)

    def gamma(k):
        if k % (2 * L) == 0:
            return 2 * K + math.log(math.tanh(K))
        return math.acosh(c - math.cos(math.pi * k / L))

    # ln(2 cosh y) = |y| + ln(1 + e^{-2|y|}),  ln|2 sinh y| = |y| + ln(1 - e^{-2|y|})
    terms = []                      # (sign, log|Z_i|)
    for odd in (1, 0):
        g = [gamma(2 * r + odd) for r in range(L)]
        lc = sum(abs(M * x / 2) + math.log1p(math.exp(-2 * abs(M * x / 2))) for x in g)
        terms.append((1.0, lc))
        sg, ls = 1.0, 0.0
        for x in g:
            y = M * x / 2
            if y == 0.0:
                sg = 0.0
                break
            sg *= math.copysign(1.0, y)
            ls += abs(y) + math.log(-math.expm1(-2 * abs(y)))
        terms.append((sg, ls))
    m = max(t[1] for t in terms)
    tot = sum(sg * math.exp(lv - m) for sg, lv in terms)
    return math.log(0.5) + (M * L / 2) * math.log(2 * math.sinh(2 * K)) + m + math.log(tot)


def onsager_minus_beta_f(beta, npts=4096):
    """-beta f per site in the thermodynamic limit, h = 0 (Onsager 1944).

    -beta f = ln 2 + 1/(8 pi^2) Int_0^{2pi} Int_0^{2pi}
              ln[cosh^2 2K - sinh 2K (cos t1 + cos t2)] dt1 dt2,
    evaluated with the midpoint rule on a periodic grid (spectrally accurate
    away from the critical point).
    """
    K = float(beta)
    t = (np.arange(npts) + 0.5) * (2 * np.pi / npts)
    c = np.cos(t)
    a = math.cosh(2 * K) ** 2
    b = math.sinh(2 * K)
    acc = 0.0
    for c1 in c:
        acc += np.log(a - b * (c1 + c)).sum()
    return math.log(2.0) + acc / (npts * npts) / 2.0


def onsager_minus_beta_f_1d(beta):
    """Same quantity from the one-dimensional elliptic form:
    -beta f = ln(2 cosh 2K) + (1/pi) Int_0^{pi/2} ln[(1 + sqrt(1 - k^2 sin^2 t))/2] dt,
    k = 2 sinh 2K / cosh^2 2K.  Used only to cross-check the 2D integral."""
    from scipy.integrate import quad
    K = float(beta)
    k = 2 * math.sinh(2 * K) / math.cosh(2 * K) ** 2
    f = lambda t: math.log((1 + math.sqrt(max(0.0, 1 - (k * math.sin(t)) ** 2))) / 2)
    val, _ = quad(f, 0, math.pi / 2, limit=200, epsabs=1e-14, epsrel=1e-14)
    return math.log(2 * math.cosh(2 * K)) + val / math.pi


# ---------------------------------------------------------------------------
# The spins-on-bonds network of Sec. IV (Fig. 1): an L x L torus of tensors
# whose legs carry the spins; the four spins on the legs of one tensor sit
# around one plaquette of the (45-degree rotated) square lattice, and the
# tensor holds the four nearest-neighbour bonds of that plaquette.  2 L^2
# spins, 4 L^2 bonds (the L = 8 network is the paper's 128-spin lattice).
# Each spin belongs to two tensors, so a field h enters as e^{beta h s / 2}
# per leg.

def bond_spin_tensor(beta, h=0.0):
    """T[l,u,r,d] = exp(beta (s_l s_u + s_u s_r + s_r s_d + s_d s_l)
                         + beta h (s_l + s_u + s_r + s_d) / 2), index 0 = spin +1."""
    sp = np.array([1.0, -1.0])
    l, u, r, d = np.meshgrid(sp, sp, sp, sp, indexing='ij')
    return np.exp(beta * (l * u + u * r + r * d + d * l) + 0.5 * beta * h * (l + u + r + d))


def bond_spin_brute_lnZ(L, beta, h=0.0):
    """ln Z of the L x L spins-on-bonds torus by enumerating all 2^(2 L^2)
    states, from the spin geometry alone: horizontal bond spins hs[y][x] (the
    r leg of tensor (x, y) and l leg of (x+1, y)), vertical vs[y][x] (the d leg
    of (x, y) and u leg of (x, y+1)); tensor (x, y) couples its four legs
    around a plaquette."""
    n = 2 * L * L
    if n > 18:
        raise ValueError("brute force limited to 2 L^2 <= 18")
    idx = np.arange(1 << n, dtype=np.int64)
    s = 1 - 2 * ((idx[:, None] >> np.arange(n)) & 1)
    hs = s[:, :L * L].reshape(-1, L, L)            # [state, y, x]
    vs = s[:, L * L:].reshape(-1, L, L)
    E = np.zeros(len(idx))
    M = s.sum(axis=1).astype(np.float64)
    for y in range(L):
        for x in range(L):
            sl = hs[:, y, (x - 1) % L]
            su = vs[:, (y - 1) % L, x]
            sr = hs[:, y, x]
            sd = vs[:, y, x]
            E += sl * su + su * sr + sr * sd + sd * sl
    return _logsumexp(beta * E + beta * h * M)


def bond_spin_transfer_lnZ(L, beta, h=0.0):
    """ln Z of the L x L spins-on-bonds torus as ln Tr(R^L), R the 2^L x 2^L
    row transfer matrix R[(u_0..u_{L-1}), (d_0..d_{L-1})] = sum over the
    horizontal bonds of the ring of L tensors (r of x = l of x+1, periodic)."""
    if L > 10:
        raise ValueError("transfer matrix limited to L <= 10")
    T = bond_spin_tensor(beta, h)
    # ring contraction: A[l_0, U..., r_x, D...] over the first x+1 tensors
    A = T.transpose(0, 1, 3, 2)                     # [l0, u0, d0, r0]
    for _ in range(1, L):
        # A[l0, U, D, r] * T[r, u, r', d] -> [l0, (U, u), (D, d), r']
        A = np.einsum('aUDr,rusd->aUuDds', A, T)
        a, U, u, Dd, d, s_ = A.shape
        A = A.reshape(a, U * u, Dd * d, s_)
    R = np.einsum('aUDa->UD', A)
    m = R.max()
    ev = np.linalg.eigvals(R / m)
    z = np.sum(ev.astype(np.complex128) ** L)
    return float(L * math.log(m) + math.log(z.real))
