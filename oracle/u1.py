"""U(1)- and Z2-symmetric tensors for the oracle: legs, canonical layout, dense expansion.

TEST INFRASTRUCTURE ONLY (see the package docstring).

A rank-R tensor is a direct sum of blocks (Sec. 2, Eq. "tensor-blocks"); every
leg has a direction (Sec. 2, Sec. 3.1); for an abelian symmetry the
generalised CGC of a block is one number, non-zero exactly when the charges
satisfy the addition rule, and the rule can be enforced by hand instead of
storing it (Sec. 2, text after Eq. "tensor-cgc").  No global charge shift
is allowed (Sec. 2, end of the worked example), so the rule is
    sum_i flow_i * q_i = 0        (flow +1 incoming, -1 outgoing).
For Z2 (the paper's third symmetry, compared in Sec. 4.1) the charges are
parities 0 and 1 and the same rule holds modulo 2; a leg carries its
modulus (0 for U(1), 2 for Z2) and every rule below reduces sums by it.

Canonical layout (a reading: the paper fixes no storage order):
  * a leg's sectors have strictly ascending charges; its dense index is the
    concatenation of the sectors;
  * the blocks are all sector tuples that satisfy the rule, sorted
    lexicographically by per-leg sector index, leg 0 most significant;
  * each block is stored dense row-major (leg 0 slowest), blocks
    concatenated in canonical order.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Leg:
    flow: int           # +1 incoming, -1 outgoing
    charges: tuple      # strictly ascending sector charges
    degs: tuple         # reduced degeneracy (dimension) of each sector
    mod: int = 0        # 0: U(1) integer charges; 2: Z2 parities

    def __post_init__(self):
        assert self.flow in (1, -1)
        assert len(self.charges) == len(self.degs)
        assert all(b > a for a, b in zip(self.charges, self.charges[1:]))
        assert all(d > 0 for d in self.degs)
        assert self.mod in (0, 2)
        if self.mod:
            assert all(0 <= q < self.mod for q in self.charges)

    @property
    def dim(self):
        return int(sum(self.degs))

    def dual(self):
        return Leg(-self.flow, self.charges, self.degs, self.mod)

    def charge_vector(self):
        """Charge of every dense index of the leg."""
        return np.repeat(np.array(self.charges, dtype=np.int64), self.degs)

    def sector_offsets(self):
        return np.concatenate([[0], np.cumsum(self.degs)]).astype(np.int64)

    def same_space(self, other):
        return self.charges == other.charges and self.degs == other.degs


def leg_from_spec(spec):
    return Leg(spec["flow"], tuple(spec["charges"]), tuple(spec["degs"]), spec.get("mod", 0))


def modulus(legs):
    m = {l.mod for l in legs}
    assert len(m) == 1, "legs of one tensor share their group"
    return m.pop()


def reduce(q, mod):
    """Canonical representative of a charge sum: itself (U(1)) or its parity (Z2)."""
    return q % mod if mod else q


def blocks(legs):
    """Canonical list of allowed sector tuples (Sec. 2: blocks labelled by one
    charge per leg; forbidden blocks are identically zero)."""
    mod = modulus(legs)
    out = []
    for idx in itertools.product(*[range(len(l.charges)) for l in legs]):
        if reduce(sum(l.flow * l.charges[i] for l, i in zip(legs, idx)), mod) == 0:
            out.append(idx)
    return out


def block_shape(legs, idx):
    return tuple(l.degs[i] for l, i in zip(legs, idx))


def nnz(legs):
    return int(sum(int(np.prod(block_shape(legs, b))) for b in blocks(legs)))


def dense_shape(legs):
    return tuple(l.dim for l in legs)


def allowed_mask(legs):
    """Dense boolean mask of the entries the selection rule allows, computed
    from the per-index charges alone (independent of the block list)."""
    tot = np.zeros(dense_shape(legs), dtype=np.int64)
    for ax, l in enumerate(legs):
        shape = [1] * len(legs)
        shape[ax] = l.dim
        tot = tot + l.flow * l.charge_vector().reshape(shape)
    mod = modulus(legs)
    return (tot % mod == 0) if mod else (tot == 0)


def to_dense(legs, flat):
    """Place each reduced block at its sector offsets (Eq. "tensor-blocks-diag")."""
    flat = np.asarray(flat, dtype=np.float64)
    out = np.zeros(dense_shape(legs), dtype=np.float64)
    offs = [l.sector_offsets() for l in legs]
    pos = 0
    for b in blocks(legs):
        shp = block_shape(legs, b)
        n = int(np.prod(shp))
        sl = tuple(slice(o[i], o[i] + d) for o, i, d in zip(offs, b, shp))
        out[sl] = flat[pos:pos + n].reshape(shp)
        pos += n
    assert pos == flat.size, (pos, flat.size)
    return out


def from_dense(legs, dense):
    """Read the allowed blocks of a dense array back in canonical order."""
    offs = [l.sector_offsets() for l in legs]
    parts = []
    for b in blocks(legs):
        shp = block_shape(legs, b)
        sl = tuple(slice(o[i], o[i] + d) for o, i, d in zip(offs, b, shp))
        parts.append(np.ascontiguousarray(dense[sl]).reshape(-1))
    if not parts:
        return np.zeros(0)
    return np.concatenate(parts)


def fuse(legs):
    """Fuse several legs into one (Sec. 3.2: merging legs, used to build the
    rank-4 double layer).

    Reading (the paper fixes no order): the fused leg takes the flow of the
    first leg; its charge is sum_i flow_i q_i / flow_0; its sectors are in
    ascending charge; inside a sector the sub-sector tuples come in ascending
    lexicographic order of their per-leg sector indices, and the inner index
    of a tuple is the row-major index over the member legs.
    Returns (fused_leg, F) with F the dense 0/1 isometry F[k, i_0, i_1, ...].
    """
    f0 = legs[0].flow
    mod = modulus(legs)
    by_q = {}
    for idx in itertools.product(*[range(len(l.charges)) for l in legs]):
        q = reduce(sum(l.flow * l.charges[i] for l, i in zip(legs, idx)) * f0, mod)
        by_q.setdefault(q, []).append(idx)
    charges = tuple(sorted(by_q))
    degs = tuple(sum(int(np.prod([l.degs[i] for l, i in zip(legs, t)])) for t in by_q[q])
                 for q in charges)
    fl = Leg(f0, charges, degs, mod)
    F = np.zeros((fl.dim,) + tuple(l.dim for l in legs))
    offs = [l.sector_offsets() for l in legs]
    k = 0
    for q in charges:
        for t in sorted(by_q[q]):
            shp = [l.degs[i] for l, i in zip(legs, t)]
            for inner in itertools.product(*[range(s) for s in shp]):
                F[(k,) + tuple(int(o[i]) + j for o, i, j in zip(offs, t, inner))] = 1.0
                k += 1
    assert k == fl.dim
    return fl, F


def double_layer(A_legs, A, R_legs=None, R=None):
    """Rank-4 double layer a = sum_p A (x) A* with ket/bra legs fused pairwise
    (Sec. 3.2).  The bra tensor A* carries every flow reversed; the fused leg
    takes the ket flow, so its charge is q_ket - q_bra.

    With a remover R[r, l', s] (Sec. 3.1), its double layer
    rho = sum_s R (x) R* is absorbed on the right bond, a'[l,u,r',d] =
    sum a[l,u,r,d] rho[r, r'], making the right leg equal to the left leg.
    Returns (legs, dense) of a (or a').
    """
    kl, Fl = fuse([A_legs[1], A_legs[1].dual()])
    ku, Fu = fuse([A_legs[2], A_legs[2].dual()])
    kr, Fr = fuse([A_legs[3], A_legs[3].dual()])
    kd, Fd = fuse([A_legs[4], A_legs[4].dual()])
    # A* of a real tensor has the same entries
    a = np.einsum("plurd,pLURD,alL,buU,crR,edD->abce", A, A, Fl, Fu, Fr, Fd, optimize=True)
    legs = [kl, ku, kr, kd]
    if R is not None:
        kr_in, Fri = fuse([R_legs[0], R_legs[0].dual()])
        kl_out, Flo = fuse([R_legs[1], R_legs[1].dual()])
        rho = np.einsum("rls,RLs,arR,blL->ab", R, R, Fri, Flo, optimize=True)
        assert kr_in.same_space(kr) and kr_in.flow == -kr.flow
        a = np.einsum("lurd,rx->luxd", a, rho)
        legs = [kl, ku, kl_out, kd]
    return legs, a
