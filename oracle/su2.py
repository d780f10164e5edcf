"""SU(2)-symmetric tensors for the oracle: exact Clebsch-Gordan coefficients,
canonical reduced-block layout with fusion trees, dense expansion.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2: every block of a symmetric tensor is a reduced dense tensor times a
generalised CGC tensor (Eq. "tensor-cgc"); for a rank-2 tensor with one
incoming and one outgoing leg the CGC tensor is an identity, for rank 3 it is
the standard Clebsch-Gordan coefficient.  The paper fixes the CGC tensor only
for those two ranks; the reading used for every rank is

  * a block is a map from its outgoing legs to its incoming legs through one
    coupled spin J: c[m_in; m_out] = sum_M <in-tree m_in | J M>
    <out-tree m_out | J M>;
  * a tree couples its legs left to right (leg order) with Condon-Shortley
    Clebsch-Gordan coefficients: ((j_a j_b) k_1 j_c) k_2 ... -> J; with no
    leg the tree is the singlet J = 0, with one leg J is that leg's spin;
  * the block's tree labels are (intermediates of the in-tree, J,
    intermediates of the out-tree), every label written as 2k;
  * blocks are sorted by per-leg sector index (leg 0 most significant),
    then by tree labels ascending; reduced blocks are row-major;
  * inside a sector of spin j with reduced degeneracy n, the dense index of
    (reduced index r, magnetic number m) is r (2j+1) + (j - m).

Contracting an outgoing leg with an incoming leg is a plain sum over m
(the CGC of a contraction is the contraction of the CGCs, Sec. 2, text after
the contraction formula).  Spins are passed doubled (2j, 2m) throughout, so
all labels are integers.
"""
from __future__ import annotations

import functools
import itertools
from dataclasses import dataclass
from fractions import Fraction
from math import factorial, sqrt

import numpy as np


# ---------------------------------------------------------------------------
# Clebsch-Gordan coefficients (Racah's closed formula, exact rationals)

def _f(n2):
    """factorial of the integer n2/2 (n2 even and >= 0 by construction)"""
    assert n2 % 2 == 0 and n2 >= 0, n2
    return factorial(n2 // 2)


@functools.lru_cache(maxsize=None)
def cg(tj1, tm1, tj2, tm2, tJ, tM):
    """<j1 m1 j2 m2 | J M> with every argument doubled.

    Racah's formula: the square of the prefactor and the alternating sum are
    exact rationals; the square root is taken once, at the end, in FP64."""
    if tm1 + tm2 != tM:
        return 0.0
    if not (abs(tj1 - tj2) <= tJ <= tj1 + tj2) or (tj1 + tj2 + tJ) % 2:
        return 0.0
    if abs(tm1) > tj1 or abs(tm2) > tj2 or abs(tM) > tJ:
        return 0.0
    if (tj1 + tm1) % 2 or (tj2 + tm2) % 2 or (tJ + tM) % 2:
        return 0.0
    pre = Fraction((tJ + 1) * _f(tJ + tj1 - tj2) * _f(tJ - tj1 + tj2) * _f(tj1 + tj2 - tJ),
                   _f(tj1 + tj2 + tJ + 2))
    pre *= (_f(tJ + tM) * _f(tJ - tM) * _f(tj1 - tm1) * _f(tj1 + tm1) * _f(tj2 - tm2) * _f(tj2 + tm2))
    s = Fraction(0)
    for k in range(0, tj1 + tj2 + tJ + 1):
        args = (tj1 + tj2 - tJ - 2 * k, tj1 - tm1 - 2 * k, tj2 + tm2 - 2 * k,
                tJ - tj2 + tm1 + 2 * k, tJ - tj1 - tm2 + 2 * k)
        if min(args) < 0:
            continue
        den = factorial(k)
        for a in args:
            den *= _f(a)
        s += Fraction((-1) ** k, den)
    if s == 0:
        return 0.0
    mag = sqrt(float(s * s * pre))
    return mag if s > 0 else -mag


# ---------------------------------------------------------------------------
# legs and blocks

@dataclass(frozen=True)
class Leg:
    flow: int          # +1 incoming, -1 outgoing
    spins: tuple       # doubled spins 2j of the sectors, strictly ascending
    degs: tuple        # reduced degeneracy n_j of every sector

    def __post_init__(self):
        assert self.flow in (1, -1)
        assert len(self.spins) == len(self.degs)
        assert all(b > a for a, b in zip(self.spins, self.spins[1:]))
        assert all(s >= 0 for s in self.spins) and all(d > 0 for d in self.degs)

    @property
    def dim(self):
        """total dimension: sum of n_j (2j + 1)"""
        return int(sum(n * (tj + 1) for tj, n in zip(self.spins, self.degs)))

    @property
    def rdim(self):
        """reduced dimension: sum of n_j"""
        return int(sum(self.degs))

    def dual(self):
        return Leg(-self.flow, self.spins, self.degs)

    def sector_offsets(self):
        sizes = [n * (tj + 1) for tj, n in zip(self.spins, self.degs)]
        return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def _couplings(tjs):
    """All left-to-right coupling trees of spins tjs: list of
    (intermediates, J) with the intermediates after the 2nd .. (n-1)th leg."""
    if len(tjs) == 0:
        return [((), 0)]
    if len(tjs) == 1:
        return [((), tjs[0])]
    out = []

    def rec(k, i, inter):
        for kn in range(abs(k - tjs[i]), k + tjs[i] + 1, 2):
            if i == len(tjs) - 1:
                out.append((tuple(inter), kn))
            else:
                rec(kn, i + 1, inter + [kn])

    rec(tjs[0], 1, [])
    return out


def in_out(legs):
    ins = [i for i, l in enumerate(legs) if l.flow == 1]
    outs = [i for i, l in enumerate(legs) if l.flow == -1]
    return ins, outs


def blocks(legs):
    """Canonical list of (sector index tuple, tree labels)."""
    ins, outs = in_out(legs)
    res = []
    for idx in itertools.product(*[range(len(l.spins)) for l in legs]):
        tj = [l.spins[i] for l, i in zip(legs, idx)]
        tin = _couplings([tj[i] for i in ins])
        tout = _couplings([tj[i] for i in outs])
        trees = sorted(a + (J,) + b for a, J in tin for b, J2 in tout if J == J2)
        res.extend((idx, t) for t in trees)
    return res


def block_shape(legs, idx):
    return tuple(l.degs[i] for l, i in zip(legs, idx))


def nnz(legs):
    return int(sum(int(np.prod(block_shape(legs, b))) for b, _ in blocks(legs)))


def dense_shape(legs):
    return tuple(l.dim for l in legs)


def _tree_vector(tjs, inter, tJ):
    """V[m_1, ..., m_n, M] = <tree(m_1..m_n) | J M>, m indices descending."""
    if len(tjs) == 0:
        assert tJ == 0
        return np.ones((1,))  # only M = 0
    V = np.eye(tjs[0] + 1)     # [m_1, K] with K = j_1
    tk = tjs[0]
    for i in range(1, len(tjs)):
        tkn = inter[i - 1] if i < len(tjs) - 1 else tJ
        tji = tjs[i]
        W = np.zeros((tk + 1, tji + 1, tkn + 1))
        for a in range(tk + 1):
            for b in range(tji + 1):
                for c in range(tkn + 1):
                    W[a, b, c] = cg(tk, tk - 2 * a, tji, tji - 2 * b, tkn, tkn - 2 * c)
        V = np.tensordot(V, W, axes=([V.ndim - 1], [0]))
        tk = tkn
    return V


def basis(legs, idx, tree):
    """Generalised CGC tensor of a block, indexed by the legs' m (descending)."""
    ins, outs = in_out(legs)
    tj = [l.spins[i] for l, i in zip(legs, idx)]
    ni, no = len(ins), len(outs)
    n_in_inter = max(ni - 2, 0)
    inter_in = tree[:n_in_inter]
    tJ = tree[n_in_inter]
    inter_out = tree[n_in_inter + 1:]
    Vi = _tree_vector([tj[i] for i in ins], inter_in, tJ)
    Vo = _tree_vector([tj[i] for i in outs], inter_out, tJ)
    if ni == 0:
        Vi = Vi.reshape(1)
        c = Vo[..., 0] if no else np.ones(())
        c = np.asarray(c)
        order = outs
    elif no == 0:
        c = Vi[..., 0]
        order = ins
    else:
        c = np.tensordot(Vi, Vo, axes=([Vi.ndim - 1], [Vo.ndim - 1]))
        order = ins + outs
    # axes of c are in (ins, outs) order: move them to leg order
    perm = [order.index(k) for k in range(len(legs))]
    return np.transpose(c, perm) if len(legs) > 1 else c


def to_dense(legs, flat):
    """Dense expansion: every block is reduced (x) CGC (Eq. "tensor-cgc"),
    placed at its sector offsets; blocks on one sector tuple add."""
    flat = np.asarray(flat, dtype=np.float64)
    out = np.zeros(dense_shape(legs))
    offs = [l.sector_offsets() for l in legs]
    pos = 0
    R = len(legs)
    for idx, tree in blocks(legs):
        shp = block_shape(legs, idx)
        n = int(np.prod(shp))
        red = flat[pos:pos + n].reshape(shp)
        pos += n
        c = basis(legs, idx, tree)
        t = np.multiply.outer(red, c)  # axes r_0..r_{R-1}, m_0..m_{R-1}
        t = np.transpose(t, [a for k in range(R) for a in (k, R + k)])
        t = t.reshape([shp[k] * c.shape[k] for k in range(R)])
        sl = tuple(slice(o[i], o[i] + t.shape[k]) for k, (o, i) in enumerate(zip(offs, idx)))
        out[sl] += t
    assert pos == flat.size, (pos, flat.size)
    return out


def from_dense(legs, dense):
    """Reduced blocks of an invariant dense tensor: projection of each sector
    tuple onto the block's CGC tensor (the CGC tensors of different trees
    are orthogonal with squared norm 2J+1)."""
    offs = [l.sector_offsets() for l in legs]
    parts = []
    R = len(legs)
    for idx, tree in blocks(legs):
        shp = block_shape(legs, idx)
        c = basis(legs, idx, tree)
        sl = tuple(slice(o[i], o[i] + shp[k] * c.shape[k]) for k, (o, i) in enumerate(zip(offs, idx)))
        sub = dense[sl].reshape([x for k in range(R) for x in (shp[k], c.shape[k])])
        red = np.tensordot(sub, c, axes=(list(range(1, 2 * R, 2)), list(range(R))))
        parts.append((red / np.sum(c * c)).reshape(-1))
    if not parts:
        return np.zeros(0)
    return np.concatenate(parts)


def contract(legsA, a, legsB, b, la, lb):
    """Reduced result of contracting legs la of A with legs lb of B: the
    dense einsum of the expanded tensors, projected back onto the output's
    blocks.  Output legs: A's open legs, then B's open legs."""
    A = to_dense(legsA, a)
    B = to_dense(legsB, b)
    for i, j in zip(la, lb):
        assert legsA[i].flow == -legsB[j].flow
        assert legsA[i].spins == legsB[j].spins and legsA[i].degs == legsB[j].degs
    C = np.tensordot(A, B, axes=(list(la), list(lb)))
    legsC = [l for i, l in enumerate(legsA) if i not in la] + [l for j, l in enumerate(legsB) if j not in lb]
    return legsC, from_dense(legsC, C), C


# ---------------------------------------------------------------------------
# rotations (independent of the Clebsch-Gordan code: spin matrices only)

def spin_matrices(tj):
    """S_x, S_y, S_z of spin j in the m-descending basis."""
    j = tj / 2.0
    ms = [j - k for k in range(tj + 1)]
    Sz = np.diag(ms)
    Sp = np.zeros((tj + 1, tj + 1))
    for k in range(1, tj + 1):      # S+ |m> = sqrt(j(j+1) - m(m+1)) |m+1>
        m = ms[k]
        Sp[k - 1, k] = np.sqrt(j * (j + 1) - m * (m + 1))
    Sx = (Sp + Sp.T) / 2.0
    Sy = (Sp - Sp.T) / 2.0j
    return Sx, Sy, Sz


def wigner_d(tj, theta):
    """exp(-i theta . S) for spin j."""
    from scipy.linalg import expm
    Sx, Sy, Sz = spin_matrices(tj)
    return expm(-1j * (theta[0] * Sx + theta[1] * Sy + theta[2] * Sz))


def leg_rotation(leg, theta):
    """Dense rotation of a leg: identity on reduced indices, D^j on m."""
    blocks_ = [np.kron(np.eye(n), wigner_d(tj, theta)) for tj, n in zip(leg.spins, leg.degs)]
    D = np.zeros((leg.dim, leg.dim), dtype=complex)
    o = 0
    for B in blocks_:
        D[o:o + B.shape[0], o:o + B.shape[0]] = B
        o += B.shape[0]
    return D


def rotate(legs, dense, theta):
    """D on every incoming leg, conj(D) on every outgoing leg."""
    T = dense.astype(complex)
    for k, l in enumerate(legs):
        D = leg_rotation(l, theta)
        if l.flow == -1:
            D = D.conj()
        T = np.moveaxis(np.tensordot(D, T, axes=([1], [k])), 0, k)
    return T
