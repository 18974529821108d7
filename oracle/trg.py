"""Monte Carlo TRG trajectories (oracle), Secs. II-III.

Test infrastructure only: nothing on the product path may import this module.

One trajectory coarse-grains the whole L x L network level by level
(Levin-Nave TRG, Sec. III), replacing every truncated SVD by the stochastic
truncation of Sec. II, sampled independently for every tensor (Sec. III: the
samples of different tensors must be independent).  After 2 log2(L) levels a
single tensor remains and is traced (Sec. IV).  Its value Z~ is an unbiased
sample of Z (Sec. III, Eq. infiniteEnsemble).

With deterministic_levels = k > 0 the first k levels keep the chi largest
singular values instead of sampling (Sec. II, Eq. approxSVD: plain TRG), and
sampling starts at level k: the hybrid of deterministic coarse-graining steps
followed by Monte Carlo that Sec. V proposes for translation-invariant
systems.  Every trajectory is then an unbiased sample of the trace of the
network after those k deterministic levels (not of Z itself); with k at least
the number of levels it is plain deterministic TRG.  While every tensor of a
level is identical (the translation-invariant network before sampling starts)
one split per sublattice and one plaquette contraction stand for all of them
(the logarithmic cost of Sec. III for translation-invariant systems).

Readings of points the paper leaves open (shared with the device path by
specification):
  * the SVD is LAPACK's (numpy.linalg.svd), singular values descending;
  * every tensor is divided by its largest singular value s_1 after its SVD
    and ln s_1 is accumulated per trajectory (range control only);
  * the reweighted value s_i / r_i is split as its square root on each side;
  * bond dimension of level k+1:  D' = min(chi, nu), where nu is the larger
    nonzero count of the two sublattice matricizations when every level-k
    tensor is identical (the shared prefix), else D_k^2; halves with fewer
    kept values are zero-padded to D';
  * the result is (sign, ln|Z~|, flags); flags mark near-ties where two
    correct implementations may legitimately keep different indices.
"""
import math

import numpy as np

from . import philox
from .network import plan
from .sampler import truncate, truncate_top


def matricize(T, parity):
    """A (parity 0): M[(l,u),(r,d)];  B (parity 1): M[(u,r),(d,l)]."""
    D = T.shape[0]
    if parity == 0:
        return T.reshape(D * D, D * D)
    return T.transpose(1, 2, 3, 0).reshape(D * D, D * D)


def svd(M):
    U, s, Vt = np.linalg.svd(M, full_matrices=False)
    return U, s, Vt


def split(T, parity, Dn, choose):
    """Split one tensor into its two three-leg halves (Sec. II + Sec. III).

    choose(s, n_rows) -> (kept, reweighted values, flags).  Returns
    (left half [x,y,Dn], right half [Dn,x,y], ln s_1, flags) where the left
    half is F1[l,u,a] (A) or F2[u,r,b] (B) and the right half F3[a,r,d] (A)
    or F4[b,d,l] (B).  A zero tensor gives ln s_1 = -inf.
    """
    D = T.shape[0]
    M = matricize(T, parity)
    U, s, Vt = svd(M)
    s1 = s[0]
    if not s1 > 0.0:
        z = np.zeros((D, D, Dn))
        return z, np.zeros((Dn, D, D)), -math.inf, 0
    kept, st, flags = choose(s / s1, D * D)
    if len(kept) > Dn:
        raise AssertionError("kept more values than the bond dimension")
    root = np.sqrt(st)
    left = np.zeros((D * D, Dn))
    right = np.zeros((Dn, D * D))
    left[:, :len(kept)] = U[:, kept] * root
    right[:len(kept), :] = root[:, None] * Vt[kept, :]
    return left.reshape(D, D, Dn), right.reshape(Dn, D, D), math.log(s1), flags


def contract(F3, F4, F2, F1):
    """T'[al,be,de,ga] = sum F3[al,i,j] F4[be,k,i] F2[j,m,ga] F1[m,k,de].

    Summed pairwise in the Levin-Nave order (Sec. III): X = F3 F4 over i,
    Y = F2 F1 over m, then X Y over (j, k).  Same sum as the four-tensor
    expression, in a different rounding order.
    """
    X = np.einsum('aij,bki->abjk', F3, F4)
    Y = np.einsum('jmg,mkd->jkdg', F2, F1)
    return np.tensordot(X, Y, axes=([2, 3], [0, 1]))


class Problem:
    """A lattice: L x L torus of identical site tensors T0 (legs l,u,r,d)."""

    def __init__(self, T0, L, chi, zero_tol_scale=1.0, deterministic_levels=0, site_tensors=None):
        T0 = np.asarray(T0, dtype=np.float64)
        if T0.ndim != 4 or len(set(T0.shape)) != 1:
            raise ValueError("T0 must be D x D x D x D")
        if chi < 1:
            raise ValueError("chi >= 1")
        self.T0, self.L, self.chi = T0, int(L), int(chi)
        self.zero_tol_scale = float(zero_tol_scale)   # multiplies the zero threshold (Sec. II "nonzero")
        self.levels = plan(self.L)
        self.n_levels = len(self.levels) - 1      # SVD levels: 0 .. 2m-1
        # levels 0 .. deterministic_levels-1 keep the chi largest values (Eq. approxSVD)
        self.deterministic_levels = int(deterministic_levels)
        # {level-0 tensor id (y L + x): tensor} replacing T0 at those sites (impurities);
        # such a network is not translation invariant: every level is split tensor by tensor
        self.site_tensors = {int(k): np.asarray(v, dtype=np.float64) for k, v in (site_tensors or {}).items()}


def _stochastic_chooser(seed, traj, level, tensor, chi, zero_scale=1.0):
    def choose(s, n_rows):
        uf = lambda c: philox.uniforms(seed, traj, level, tensor, c)
        kept, st, flags, _ = truncate(s, chi, uf, n_rows, zero_scale)
        return kept, st, flags
    return choose


def _deterministic_chooser(chi, zero_scale=1.0):
    def choose(s, n_rows):
        kept, st, flags, _ = truncate_top(s, chi, n_rows, zero_scale)
        return kept, st, flags
    return choose


def run_level(prob, k, tensors, shared, chooser_for, deterministic=False):
    """Split every level-k tensor and contract the plaquettes into level k+1.

    Returns (new tensors, sum of ln s_1, flags, next-level shared?).
    chooser_for(t) gives the truncation rule for tensor t.  On a shared level
    (every tensor identical) that is exact or deterministic, one split per
    sublattice and one plaquette stand for all tensors.
    """
    lev = prob.levels[k]
    D = tensors[0].shape[0]
    n_rows = D * D
    if shared:
        # every tensor identical: the nonzero count of each matricization
        nu = 0
        for par in (0, 1):
            s = svd(matricize(tensors[0], par))[1]
            if s[0] > 0:
                nu = max(nu, int(np.sum(s / s[0] > prob.zero_tol_scale * n_rows * 2.0 ** -52)))
        Dn = max(1, min(prob.chi, nu))
        exact = nu <= prob.chi
    else:
        Dn = min(prob.chi, n_rows)
        exact = False
    if shared and (exact or deterministic):
        choose = _deterministic_chooser(prob.chi, prob.zero_tol_scale)
        part = [split(tensors[0], par, Dn, choose) for par in (0, 1)]
        n_a = int(np.sum(lev.parity == 0))
        lnacc = n_a * part[0][2] + (lev.n - n_a) * part[1][2]
        flags = part[0][3] | part[1][3]
        if lev.children_parents is None or len(lev.children_parents) == 0:
            return [], lnacc, flags, True
        # the plaquette's four halves come from A (p, p+a1+a2) and B (p+a1, p+a2)
        T = contract(part[0][1], part[1][1], part[1][0], part[0][0])
        return [T] * len(lev.children_parents), lnacc, flags, True
    halves = []
    lnacc = 0.0
    flags = 0
    for t in range(lev.n):
        left, right, lns1, f = split(tensors[t], int(lev.parity[t]), Dn, chooser_for(t))
        halves.append((left, right))
        lnacc += lns1
        flags |= f
    new = []
    for p, pa1, pa2, pa12 in lev.children_parents:
        F3 = halves[p][1]
        F4 = halves[pa1][1]
        F2 = halves[pa2][0]
        F1 = halves[pa12][0]
        new.append(contract(F3, F4, F2, F1))
    return new, lnacc, flags, (shared and exact)


def run_trajectory(prob, seed, traj):
    """One Monte Carlo trajectory -> (sign, ln|Z~|, flags)."""
    tensors = [prob.T0] * prob.levels[0].n
    for t, T in prob.site_tensors.items():
        tensors[t] = T
    shared = not prob.site_tensors
    lnacc = 0.0
    flags = 0
    for k in range(prob.n_levels):
        det = k < prob.deterministic_levels
        if det:
            chooser_for = lambda t: _deterministic_chooser(prob.chi, prob.zero_tol_scale)
        else:
            chooser_for = lambda t, k=k: _stochastic_chooser(seed, traj, k, t, prob.chi, prob.zero_tol_scale)
        tensors, lnk, f, shared = run_level(prob, k, tensors, shared, chooser_for, det)
        lnacc += lnk
        flags |= f
        if lnacc == -math.inf:
            return 0, -math.inf, flags
    T = tensors[0]
    tr = float(np.einsum('abab->', T))
    if tr == 0.0:
        return 0, -math.inf, flags
    return (1 if tr > 0 else -1), lnacc + math.log(abs(tr)), flags


def run_many(prob, seed, first_traj, n, workers=1):
    """Trajectories first_traj .. first_traj+n-1 -> arrays (sign, lnabs, flags).

    With workers > 1 the trajectories are spread over a 'spawn' process pool;
    each trajectory is computed exactly as in the serial loop.
    """
    trajs = list(range(first_traj, first_traj + n))
    if workers <= 1 or n <= 1:
        res = [run_trajectory(prob, seed, i) for i in trajs]
    else:
        import multiprocessing as mp
        import os
        # one BLAS thread per worker: the workers are the parallelism
        saved = {k: os.environ.get(k) for k in ('OMP_NUM_THREADS', 'OPENBLAS_NUM_THREADS', 'MKL_NUM_THREADS')}
        for k in saved:
            os.environ[k] = '1'
        try:
            ctx = mp.get_context('spawn')
            with ctx.Pool(workers) as pool:
                res = pool.starmap(run_trajectory, [(prob, seed, i) for i in trajs],
                                   chunksize=max(1, n // (4 * workers)))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    sign = np.array([r[0] for r in res], dtype=np.int8)
    lnabs = np.array([r[1] for r in res], dtype=np.float64)
    flags = np.array([r[2] for r in res], dtype=np.uint8)
    return sign, lnabs, flags
