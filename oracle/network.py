"""Levin-Nave TRG geometry on an L x L torus, and exact network traces (oracle).

Test infrastructure only: nothing on the product path may import this module.

Conventions (the paper defers the TRG leg conventions to Levin and Nave, Sec. III;
these are this implementation's reading, shared by the oracle and the device path
through their specification only, never through code):

* Level k tensors sit at positions o_k + i*a1 + j*a2 (mod L in original
  coordinates).  Level 0: a1 = (1,0) "right", a2 = (0,1) "down", o_0 = 0.
  Every tensor has legs (l, u, r, d); its r leg is the l leg of the tensor at
  +a1 and its d leg is the u leg of the tensor at +a2.
* Sublattice A is i + j even, B is i + j odd.
* A tensors are matricized as M[(l,u),(r,d)] and split into F1[l,u,a] and
  F3[a,r,d]; B tensors as M[(u,r),(d,l)] into F2[u,r,b] and F4[b,d,l].
* Each plaquette whose top-left corner p is an A tensor becomes one level k+1
  tensor  T'[al,be,de,ga] = sum_{i,j,k,m} F3(p)[al,i,j] F4(p+a1)[be,k,i]
  F2(p+a2)[j,m,ga] F1(p+a1+a2)[m,k,de]  with legs (l,u,r,d) = (al,be,de,ga),
  at position p + (a1+a2)/2, and the next basis is a1' = a1+a2, a2' = a2-a1.
* Numbering: level 0 tensor (x, y) has id y*L + x; level k+1 tensors are
  numbered in increasing order of the level-k id of their top-left parent p.

Positions are kept in doubled integer coordinates so that the half-integer
offset of the first step stays exact.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class Level:
    n: int                 # tensors at this level
    parity: np.ndarray     # (n,) 0 = sublattice A, 1 = B
    right: np.ndarray      # (n,) id of the neighbour at +a1
    down: np.ndarray       # (n,) id of the neighbour at +a2
    left: np.ndarray       # (n,) id of the neighbour at -a1
    up: np.ndarray         # (n,) id of the neighbour at -a2
    # parents of each tensor of the NEXT level (None on the last level):
    # columns = (p, p+a1, p+a2, p+a1+a2) giving (F3, F4, F2, F1)
    children_parents: np.ndarray = None


def plan(L):
    """Geometry of all levels for an L x L torus, L = 2^m >= 2.

    Returns a list of 2m+1 Level objects; level 2m holds the single final
    tensor, whose r leg meets its own l leg and d leg its own u leg.
    """
    m = int(round(np.log2(L)))
    if L < 2 or (1 << m) != L:
        raise ValueError("L must be a power of two >= 2")
    L2 = 2 * L
    # level 0
    pos = [((2 * x) % L2, (2 * y) % L2) for y in range(L) for x in range(L)]
    ij = [(x, y) for y in range(L) for x in range(L)]
    A1, A2 = (2, 0), (0, 2)
    levels = []
    for k in range(2 * m + 1):
        n = len(pos)
        key = {p: t for t, p in enumerate(pos)}
        if len(key) != n:
            raise AssertionError("duplicate positions")

        def shift(p, v, sgn=1):
            return ((p[0] + sgn * v[0]) % L2, (p[1] + sgn * v[1]) % L2)

        right = np.array([key[shift(p, A1)] for p in pos])
        down = np.array([key[shift(p, A2)] for p in pos])
        left = np.array([key[shift(p, A1, -1)] for p in pos])
        up = np.array([key[shift(p, A2, -1)] for p in pos])
        parity = np.array([(i + j) & 1 for i, j in ij])
        lev = Level(n, parity, right, down, left, up)
        levels.append(lev)
        if n == 1:
            break
        # checkerboard consistency: every neighbour has the opposite parity
        for nb in (right, down, left, up):
            if np.any(parity[nb] == parity):
                raise AssertionError("inconsistent checkerboard at level %d" % k)
        half = ((A1[0] + A2[0]) // 2, (A1[1] + A2[1]) // 2)
        new_pos, new_ij, parents = [], [], []
        for t in range(n):
            if parity[t] != 0:
                continue
            i, j = ij[t]
            p = pos[t]
            new_pos.append(shift(p, half))
            new_ij.append(((i + j) // 2, (j - i) // 2))
            parents.append((t, right[t], down[t], right[down[t]]))
        lev.children_parents = np.array(parents, dtype=np.int64)
        pos, ij = new_pos, new_ij
        A1, A2 = (A1[0] + A2[0], A1[1] + A2[1]), (A2[0] - A1[0], A2[1] - A1[1])
    return levels


def network_trace(tensors, lev):
    """Exact trace of one level's network (all bonds summed).

    tensors[t] is the (l,u,r,d) tensor of tensor t; bond 'r of t' is shared
    with the l leg of right[t] and bond 'd of t' with the u leg of down[t].
    Tensors are absorbed one at a time in id order with pairwise einsum
    calls, summing each bond once both of its legs are present.  Meant for
    small networks only.
    """
    n = lev.n
    if n == 1:
        return float(np.einsum('abab->', tensors[0]))
    legs = []
    for t in range(n):
        legs.append([('r', int(lev.left[t])), ('d', int(lev.up[t])), ('r', t), ('d', t)])
    letters = 'abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ'
    C = np.ones(())
    open_labels = []
    for t in range(n):
        names = {}
        for lab in open_labels + legs[t]:
            if lab not in names:
                names[lab] = letters[len(names)]
        a = ''.join(names[x] for x in open_labels)
        b = ''.join(names[x] for x in legs[t])
        keep = [x for x in open_labels if x not in legs[t]] + \
               [x for x in legs[t] if x not in open_labels]
        out = ''.join(names[x] for x in keep)
        C = np.einsum(a + ',' + b + '->' + out, C, tensors[t])
        open_labels = keep
    if open_labels:
        raise AssertionError("open bonds left after the full contraction")
    return float(C)
