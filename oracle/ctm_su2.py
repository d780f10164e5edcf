"""Dense oracle of the SU(2) LEFT move (Sec. 3 with the SU(2) tensors of Sec. 2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The network is dense (every tensor expanded with ``su2.to_dense``); the
quarters, half systems and renormalisation are the same dense einsums as the
U(1) move (``oracle.ctm.quarters``).  The projector follows the SU(2)
structure: N = R_top^T R_bot has its right-cut legs of R_top outgoing and
those of R_bot incoming, so its reduced blocks (``su2.from_dense``) group by
the coupled spin J into reduced matrices N_J; each is decomposed with
LAPACK's SVD.  Truncation keeps whole multiplets: by descending sigma (ties:
smaller J, then index) a multiplet of dimension 2J+1 is kept while the kept
total dimension stays within chi_total, and skipped otherwise.  The reduced
right and left vectors, gauge-fixed (largest-|.| entry of each left vector
positive, lowest index on ties) and scaled by sigma^-1/2, become the reduced
blocks of V[beta'^dual..., new] and Ut[new^dual, beta^dual...]; P = R_bot V
and P~ = Ut R_top^T are dense products of their expansions.  The new leg is
incoming on P.
"""
from __future__ import annotations

import numpy as np

from . import ctm as octm
from . import su2

ROLES = octm.ROLES


def _sector_matrices(legs, red, nb):
    """Reduced matrices N_J of an SU(2) tensor whose first nb legs are the
    row legs (all outgoing) and the others the column legs (all incoming)."""
    nbp = len(legs) - nb
    nin = max(nbp - 2, 0)
    blocks = su2.blocks(legs)
    rows, cols = {}, {}
    for idx, tree in blocks:
        J = tree[nin]
        rk = tuple(idx[:nb]) + tuple(tree[nin + 1:])
        ck = tuple(idx[nb:]) + tuple(tree[:nin])
        rows.setdefault(J, {})[rk] = int(np.prod([legs[i].degs[idx[i]] for i in range(nb)]))
        cols.setdefault(J, {})[ck] = int(np.prod([legs[i].degs[idx[i]] for i in range(nb, len(legs))]))
    roff, coff, mats = {}, {}, {}
    for J in sorted(rows):
        o = 0
        roff[J] = {}
        for k in sorted(rows[J]):
            roff[J][k] = o
            o += rows[J][k]
        nr = o
        o = 0
        coff[J] = {}
        for k in sorted(cols[J]):
            coff[J][k] = o
            o += cols[J][k]
        mats[J] = np.zeros((nr, o))
    pos = 0
    for idx, tree in blocks:
        shp = su2.block_shape(legs, idx)
        n = int(np.prod(shp))
        J = tree[nin]
        rk = tuple(idx[:nb]) + tuple(tree[nin + 1:])
        ck = tuple(idx[nb:]) + tuple(tree[:nin])
        blk = red[pos:pos + n].reshape(int(np.prod(shp[:nb])), int(np.prod(shp[nb:])))
        r0, c0 = roff[J][rk], coff[J][ck]
        mats[J][r0:r0 + blk.shape[0], c0:c0 + blk.shape[1]] = blk
        pos += n
    return mats, roff, coff


def left_move(net, chi_total, rel_cutoff=1e-14, return_info=False):
    """One SU(2) LEFT move.  net[role] = (legs, dense); returns the renewed
    network (C1, T4, C4 replaced)."""
    L = {r: net[r][0] for r in ROLES}
    q = octm.quarters(net)
    Rt, Rb = q["Rt"], q["Rb"]
    beta = [L["T2"][2], L["a"][3]]
    betap = [L["T2"][0], L["a"][1]]
    N = np.einsum("abcd,abef->cdef", Rt, Rb)
    n_legs = beta + betap
    assert all(l.flow == -1 for l in beta) and all(l.flow == 1 for l in betap)
    mats, roff, coff = _sector_matrices(n_legs, su2.from_dense(n_legs, N), 2)
    svd = {J: np.linalg.svd(M, full_matrices=False) for J, M in mats.items()}
    cands = [(float(s), J, j) for J, (U, S, Vt) in svd.items() for j, s in enumerate(S)]
    smax = max(c[0] for c in cands)
    kept = {J: 0 for J in svd}
    dim = 0
    for s, J, j in sorted(cands, key=lambda c: (-c[0], c[1], c[2])):
        if not (s > rel_cutoff * smax):
            break
        if j != kept[J] or dim + J + 1 > chi_total:
            continue
        kept[J] += 1
        dim += J + 1
    Js = [J for J in sorted(kept) if kept[J] > 0]
    new = su2.Leg(1, tuple(Js), tuple(kept[J] for J in Js))
    vecs = {}
    for J in Js:
        U, S, Vt = svd[J]
        k = kept[J]
        u, v = U[:, :k].copy(), Vt[:k].T.copy()
        for j in range(k):
            i = int(np.argmax(np.abs(u[:, j])))
            if u[i, j] < 0:
                u[:, j], v[:, j] = -u[:, j], -v[:, j]
        vecs[J] = (u / np.sqrt(S[:k]), v / np.sqrt(S[:k]))
    # V[beta'^dual, new]: labels (J, beta' intermediates)
    v_legs = [l.dual() for l in betap] + [new]
    vflat = []
    for idx, tree in su2.blocks(v_legs):
        J = new.spins[idx[2]]
        c0 = coff[J][tuple(idx[:2])]
        n = int(np.prod(su2.block_shape(v_legs, idx)[:2]))
        vflat.append(vecs[J][1][c0:c0 + n].reshape(-1))
    u_legs = [new.dual()] + [l.dual() for l in beta]
    uflat = []
    for idx, tree in su2.blocks(u_legs):
        J = new.spins[idx[0]]
        r0 = roff[J][tuple(idx[1:])]
        n = int(np.prod(su2.block_shape(u_legs, idx)[1:]))
        uflat.append(vecs[J][0][r0:r0 + n].T.reshape(-1))
    Vd = su2.to_dense(v_legs, np.concatenate(vflat))
    Ud = su2.to_dense(u_legs, np.concatenate(uflat))
    P = np.einsum("abcd,cdn->abn", Rb, Vd)       # [alpha', new]
    Pt = np.einsum("nab,cdab->ncd", Ud, Rt)      # [new^dual, alpha]
    C1, T1, C2, T2, C3, T3, C4, T4, a = (net[r][1] for r in ROLES)
    e = lambda s, *x: np.einsum(s, *x, optimize=True)
    X1 = q["X1"]
    C1n = e("dkx,dkc->xc", X1, P)
    W = e("cuk,umd->ckmd", Pt, T4)
    Z = e("ckmd,mkre->cdre", W, a)
    T4n = e("cdre,dex->crx", Z, P)
    Y = e("ur,rkx->ukx", C4, T3)
    C4n = e("cuk,ukx->cx", Pt, Y)
    C1n, T4n, C4n = (t / np.linalg.norm(t) for t in (C1n, T4n, C4n))
    out = dict(net)
    out["C1"] = ([L["T1"][2], new], C1n)
    out["T4"] = ([new.dual(), L["a"][2], new], T4n)
    out["C4"] = ([new.dual(), L["T3"][2]], C4n)
    if return_info:
        svals = sorted((float(s) for J, (U, S, Vt) in svd.items() for s in S[:kept[J]]), reverse=True)
        return out, {"N": N, "n_legs": n_legs, "sectors": svd, "kept": kept, "dim": dim, "P": P, "Pt": Pt,
                     "new": new, "svals": svals}
    return out


def su2_network(cfg, seed=0):
    """Dense SU(2) network of a workload: seeded reduced blocks for the eight
    environment tensors and the site a[k, k, k^dual, k^dual] (the k legs are
    the double-layer legs of the recipe)."""
    from workloads import values
    k = su2.Leg(1, *cfg["k"])
    x = su2.Leg(1, *cfg["x"])
    X = lambda f: su2.Leg(f, x.spins, x.degs)
    legs = {"C1": [X(-1), X(-1)], "C2": [X(1), X(-1)], "C3": [X(1), X(1)], "C4": [X(1), X(-1)],
            "T1": [X(1), k.dual(), X(-1)], "T2": [X(1), k, X(-1)],
            "T3": [X(1), k, X(-1)], "T4": [X(1), k.dual(), X(-1)],
            "a": [k, k, k.dual(), k.dual()]}
    net = {}
    for r, lg in legs.items():
        name = "A" if r == "a" else r
        net[r] = (lg, su2.to_dense(lg, values(seed, name, su2.nnz(lg))))
    return net
