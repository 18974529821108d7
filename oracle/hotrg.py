"""Monte Carlo HOTRG trajectories (oracle): the stochastic truncation of Sec. II
applied to the higher-order TRG of Xie et al. (2012), one of the other
SVD-based coarse-graining schemes to which Secs. III and V say the method
extends.

Test infrastructure only: nothing on the product path may import this module.

The paper names the generalization without spelling it out; this is the
reading both sides implement:
  * a step merges pairs of rows: the tensors at (x, 2j) (top) and (x, 2j+1)
    (bottom) contract over their shared vertical bond into
        M(x, j)[(l1 l2), u1, (r1 r2), d2] = sum_k T(x,2j)[l1,u1,r1,k] T(x,2j+1)[l2,k,r2,d2],
    whose horizontal legs are the pairs of the two rows' legs;
  * each merged horizontal bond -- the one to the right of M(x, j) -- gets its
    own random projector  P~ = sum_{i in e} u_i u_i^T / r_i.  (u_i, lambda_i)
    are the eigenpairs of the Gram matrix of M(x, j)'s right unfolding,
        G[(r1 r2), (r1' r2')] = sum_{l,u,d} M[l,u,(r1 r2),d] M[l,u,(r1' r2'),d],
    descending (lambda_i = the squared singular values of that unfolding).
    Eigenvalues at or below n 2^-52 lambda_1 (n the bond dimension, the
    rounding level of a Gram matrix's eigenvalues) are zeros.  A chi-subset e
    of the nonzero ones is drawn with p(e) ~ prod_{i in e} lambda_i -- Sec. II's
    p(e) ~ prod s_i^2 -- by the sampler of the TRG path, and r_i are its
    inclusion rates (Sec. II, Eq. r).  Then E[P~] is the projector onto the
    range of G, outside which M(x, j) vanishes, so the expected network is
    the exact one (Sec. III's argument: independent samples, each unbiased,
    enter linearly) and every trajectory is an unbiased sample of Z.  With at
    most chi nonzero eigenvalues all are kept with r = 1 (an exact bond);
  * P~ = U~ U~^T with U~ = [u_i / sqrt(r_i)] (n x kc, kc = min(chi, n),
    zero-padded); the new tensor is
        T'(x, j)[a, u1, b, d2] = sum U~_left[(l1 l2), a] M(x, j)[(l1 l2), u1, (r1 r2), d2] U~_right[(r1 r2), b]
    with U~_left the projector factor of the bond between M(x-1, j) and
    M(x, j) (periodic; the same bond on both sides when Lx = 1), divided by
    sqrt(lambda_1) of its right bond, whose logarithm is accumulated per
    trajectory (range control only);
  * the new lattice is then reflected across its diagonal (x <-> y, legs
    l <-> u and r <-> d), so that the next step again merges rows -- the
    columns of the previous orientation.  2 log2 L steps leave one tensor,
    traced as Z~ = sum_{l,u} T[l,u,l,u] (Sec. IV);
  * uniforms: Philox4x32-10, counter (t >> 1, bond, step, trajectory) with
    bond = j Lx + x, the counter layout of the TRG path.
The result is (sign, ln|Z~|, flags), the flags as in the TRG path.
"""
import math

import numpy as np

from . import philox
from .sampler import truncate


class HotrgProblem:
    """An L x L torus of identical site tensors T0 (legs l, u, r, d)."""

    def __init__(self, T0, L, chi):
        T0 = np.asarray(T0, dtype=np.float64)
        if T0.ndim != 4 or T0.shape[0] != T0.shape[2] or T0.shape[1] != T0.shape[3]:
            raise ValueError("T0 must be Dh x Dv x Dh x Dv")
        if L < 2 or (L & (L - 1)):
            raise ValueError("L must be a power of two >= 2")
        if chi < 1:
            raise ValueError("chi >= 1")
        self.T0, self.L, self.chi = T0, int(L), int(chi)
        self.n_steps = 2 * int(round(math.log2(L)))


def merge(T1, T2):
    """M[(l1 l2), u1, (r1 r2), d2] = sum_k T1[l1,u1,r1,k] T2[l2,k,r2,d2]."""
    Dh, Dv = T1.shape[0], T1.shape[1]
    M = np.einsum('aurk,bksd->abursd', T1, T2)
    return M.reshape(Dh * Dh, Dv, Dh * Dh, Dv)


def right_gram(M):
    """G = sum_{l,u,d} M[l,u,r,d] M[l,u,r',d] (the right unfolding's Gram matrix)."""
    return np.einsum('lurd,lusd->rs', M, M)


def bond_eigen(M):
    """Eigenpairs of the right Gram matrix, descending, and the nonzero count."""
    G = right_gram(M)
    lam, U = np.linalg.eigh(G)
    lam, U = lam[::-1], U[:, ::-1]
    n = G.shape[0]
    if not lam[0] > 0.0:
        return lam, U, 0
    nnz = int(np.sum(lam > n * 2.0 ** -52 * lam[0]))
    return lam, U, nnz


def stochastic_choice(seed, traj, step, bond, chi):
    """The sampler of the TRG path on s_i = sqrt(lambda_i): (kept, r) per bond."""
    def choose(lam, nnz, n):
        s = np.sqrt(lam[:nnz])
        uf = lambda c: philox.uniforms(seed, traj, step, bond, c)
        kept, st, flags, _ = truncate(s, chi, uf, n)
        r = s[kept] / st if len(kept) else np.zeros(0)
        return kept, r, flags
    return choose


def projector_factor(lam, U, nnz, kc, choose):
    """U~ = [u_i / sqrt(r_i)] for the kept i, zero-padded to kc columns."""
    n = U.shape[0]
    kept, r, flags = choose(lam, nnz, n)
    if len(kept) > kc:
        raise AssertionError("kept more values than the bond dimension")
    F = np.zeros((n, kc))
    F[:, :len(kept)] = U[:, kept] / np.sqrt(r)
    return F, flags


def run_step(tensors, Lx, Ly, chi, chooser_for):
    """One row-merging step on an Lx x Ly lattice (tensors[y Lx + x]); returns
    the reflected Ly/2 x Lx lattice of new tensors, the sum of the ln
    normalizations and the flags.  chooser_for(bond) gives the truncation."""
    Dh = tensors[0].shape[0]
    n = Dh * Dh
    kc = min(chi, n)
    Lj = Ly // 2
    Ms, lns, F = [], [], []
    flags = 0
    for j in range(Lj):
        for x in range(Lx):
            M = merge(tensors[2 * j * Lx + x], tensors[(2 * j + 1) * Lx + x])
            lam, U, nnz = bond_eigen(M)
            Ms.append(M)
            if nnz == 0:
                lns.append(-math.inf)
                F.append(np.zeros((n, kc)))
                continue
            f, fl = projector_factor(lam, U, nnz, kc, chooser_for(j * Lx + x))
            F.append(f)
            lns.append(0.5 * math.log(lam[0]))
            flags |= fl
    new = [None] * (Lx * Lj)
    lnacc = 0.0
    for j in range(Lj):
        for x in range(Lx):
            b = j * Lx + x
            left = j * Lx + (x - 1) % Lx
            lnacc += lns[b]
            if lns[b] == -math.inf:
                T = np.zeros((kc, Ms[b].shape[1], kc, Ms[b].shape[3]))
            else:
                T = np.einsum('la,lurd,rb->aubd', F[left], Ms[b], F[b]) / math.exp(lns[b])
            # reflection across the diagonal: (x, j) -> (j, x), legs (l,u,r,d) -> (u,l,d,r)
            new[x * Lj + j] = T.transpose(1, 0, 3, 2)
    return new, Lj, Lx, lnacc, flags


def run_trajectory(prob, seed, traj, chooser_factory=None):
    """One Monte Carlo HOTRG trajectory -> (sign, ln|Z~|, flags).
    chooser_factory(step, bond) overrides the sampler (for enumeration)."""
    Lx = Ly = prob.L
    tensors = [prob.T0] * (Lx * Ly)
    lnacc = 0.0
    flags = 0
    for step in range(prob.n_steps):
        if chooser_factory is None:
            cf = lambda b, step=step: stochastic_choice(seed, traj, step, b, prob.chi)
        else:
            cf = lambda b, step=step: chooser_factory(step, b)
        tensors, Lx, Ly, lnk, f = run_step(tensors, Lx, Ly, prob.chi, cf)
        lnacc += lnk
        flags |= f
        if lnacc == -math.inf:
            return 0, -math.inf, flags
    assert Lx == 1 and Ly == 1
    tr = float(np.einsum('abab->', tensors[0]))
    if tr == 0.0:
        return 0, -math.inf, flags
    return (1 if tr > 0 else -1), lnacc + math.log(abs(tr)), flags


def run_many(prob, seed, first_traj, n, workers=1):
    """Trajectories first_traj .. first_traj+n-1 -> arrays (sign, lnabs, flags),
    over a 'spawn' process pool when workers > 1 (each trajectory computed as
    in the serial loop)."""
    trajs = list(range(first_traj, first_traj + n))
    if workers <= 1 or n <= 1:
        res = [run_trajectory(prob, seed, i) for i in trajs]
    else:
        import multiprocessing as mp
        import os
        saved = {k: os.environ.get(k) for k in ('OMP_NUM_THREADS', 'OPENBLAS_NUM_THREADS', 'MKL_NUM_THREADS')}
        for k in saved:
            os.environ[k] = '1'
        try:
            with mp.get_context('spawn').Pool(workers) as pool:
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
