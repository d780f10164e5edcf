"""Dense oracle of the directional CTMRG move with SVD projectors.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The corner transfer matrix is truncated as in the reference the paper cites
for it (Sec. 3, "truncated as suggested in [corboz14]") on the rank-4 double
layer (Sec. 3.2).  One LEFT move on a one-site cell:

  Q1 = C1 T1 T4 a,  Q2 = T1 C2 a T2,  Q3 = a T2 T3 C3,  Q4 = T4 a C4 T3
  R_top = Q1 Q2 [alpha, beta],  R_bot = Q4 Q3 [alpha', beta']
  N = R_top^T R_bot  (over the left cut alpha), block diagonal in the charge
      carried through the right cut; per sector N_q = U S V^T
  keep the chi largest singular values over all sectors (ties: smaller |q|,
      then smaller q), dropping those below rel_cutoff * sigma_max
  P~ = S^-1/2 U^T R_top^T,  P = R_bot V S^-1/2         (P~ P = 1)
  C1' = (C1 T1) P,  T4' = P~ (T4 a) P,  C4' = P~ (C4 T3)
  each divided by its Frobenius norm.

Readings where the paper is silent: the contraction order above, the SVD of
N without a QR, the tie-break, the gauge (largest-|.| entry of every kept
left singular vector made positive, lowest index on ties), the new leg's
sector order (ascending charge, descending sigma inside a sector).
The other directions are the LEFT move of the network rotated by 90 degree
steps; the full move is L, R, U, D in sequence, each on the updated env.

Tensor roles and their leg directions (L, U, R, D):
  C1[R,D] C2[L,D] C3[U,L] C4[U,R]  T1[L,D,R] T2[U,L,D] T3[L,U,R] T4[U,R,D]
  a[L,U,R,D]
"""
from __future__ import annotations

import numpy as np

from .u1 import Leg, modulus, reduce

ROLE_DIRS = {"C1": "RD", "C2": "LD", "C3": "UL", "C4": "UR",
             "T1": "LDR", "T2": "ULD", "T3": "LUR", "T4": "URD", "a": "LURD"}
ROLES = ("C1", "T1", "C2", "T2", "C3", "T3", "C4", "T4", "a")
# rotating the picture by +90 degrees (counter-clockwise): a leg pointing up
# then points left, and so on; the tensor at role X moves to role ROT_ROLE[X]
ROT_DIR = {"U": "L", "L": "D", "D": "R", "R": "U"}
ROT_ROLE = {"C1": "C4", "C2": "C1", "C3": "C2", "C4": "C3",
            "T1": "T4", "T2": "T1", "T3": "T2", "T4": "T3", "a": "a"}
DIR_ROTATIONS = {"L": 0, "U": 1, "R": 2, "D": 3}


def rotate_ccw(net):
    """Network rotated by +90 degrees: net[role] = (legs, dense)."""
    out = {}
    for old, new in ROT_ROLE.items():
        legs, arr = net[old]
        old_dirs = ROLE_DIRS[old]
        new_dirs_of_old = [ROT_DIR[d] for d in old_dirs]
        perm = [new_dirs_of_old.index(d) for d in ROLE_DIRS[new]]
        out[new] = ([legs[p] for p in perm], np.ascontiguousarray(np.transpose(arr, perm)))
    return out


def rotate(net, k):
    for _ in range(k % 4):
        net = rotate_ccw(net)
    return net


def sector_keys(legs, sign):
    """Charge carried through a composite index: sign * sum_i flow_i q_i
    (Z2: its parity)."""
    tot = np.zeros([l.dim for l in legs], dtype=np.int64)
    for ax, l in enumerate(legs):
        shape = [1] * len(legs)
        shape[ax] = l.dim
        tot = tot + l.flow * l.charge_vector().reshape(shape)
    return reduce(sign * tot, modulus(legs)).reshape(-1)


def cell_quarters(ul, ur, ll, lr):
    """The four enlarged corners and the two half systems of the left cut of
    a 2 x 2 plaquette: Q1 from the upper-left site's C1, T1, T4, a, Q2 from
    the upper-right site's T1, C2, T2, a, Q4 from the lower-left site's T4,
    C4, T3, a, Q3 from the lower-right site's T2, C3, T3, a (each site's
    net holds its own environment)."""
    e = lambda s, *x: np.einsum(s, *x, optimize=True)
    g = lambda net, r: net[r][1]
    X1 = e("rd,rkx->dkx", g(ul, "C1"), g(ul, "T1"))       # [C1.D, T1.D, T1.R]
    X2 = e("dkx,dme->kxme", X1, g(ul, "T4"))              # [T1.D, T1.R, T4.R, T4.D]
    Q1 = e("kxme,mkrd->xerd", X2, g(ul, "a"))             # [T1.R, T4.D, a.R, a.D]
    Y1 = e("xkc,cd->xkd", g(ur, "T1"), g(ur, "C2"))       # [T1.L, T1.D, C2.D]
    Y2 = e("xkd,dme->xkme", Y1, g(ur, "T2"))              # [T1.L, T1.D, T2.L, T2.D]
    Q2 = e("xkme,lkmd->xeld", Y2, g(ur, "a"))             # [T1.L, T2.D, a.L, a.D]
    Rt = e("xerd,xfrg->edfg", Q1, Q2)                     # [T4.D, a.D | T2.D, a.D]
    Z1 = e("ukd,dr->ukr", g(ll, "T4"), g(ll, "C4"))       # [T4.U, T4.R, C4.R]
    Z2 = e("ukr,rmx->ukmx", Z1, g(ll, "T3"))              # [T4.U, T4.R, T3.U, T3.R]
    Q4 = e("ukmx,kwrm->uwxr", Z2, g(ll, "a"))             # [T4.U, a.U, T3.R, a.R]
    W1 = e("ukd,dl->ukl", g(lr, "T2"), g(lr, "C3"))       # [T2.U, T2.L, C3.L]
    W2 = e("ukl,xml->ukxm", W1, g(lr, "T3"))              # [T2.U, T2.L, T3.L, T3.U]
    Q3 = e("ukxm,lwkm->uwxl", W2, g(lr, "a"))             # [T2.U, a.U, T3.L, a.L]
    Rb = e("uwxr,vyxr->uwvy", Q4, Q3)                     # [T4.U, a.U | T2.U, a.U]
    return {"X1": X1, "Q1": Q1, "Q2": Q2, "Q3": Q3, "Q4": Q4, "Rt": Rt, "Rb": Rb}


def quarters(net):
    """The four enlarged corners and the two half systems of the left cut."""
    return cell_quarters(net, net, net, net)


def truncate(cands, chi, rel_cutoff):
    """cands: list of (sigma, q_new, sector_key, j).  Global top-chi with the
    tie-break (sigma descending, |q| ascending, q ascending); singular values
    below rel_cutoff * sigma_max are dropped."""
    if not cands:
        return []
    smax = max(c[0] for c in cands)
    order = sorted(cands, key=lambda c: (-c[0], abs(c[1]), c[1], c[3]))
    return [c for c in order[:chi] if c[0] > rel_cutoff * smax]


def plaquette_projector(ul, ur, ll, lr, chi, rel_cutoff=1e-14):
    """Projectors of the left cut of a 2 x 2 plaquette (upper-left,
    upper-right, lower-left, lower-right site nets): the N = R_top^T R_bot
    of Sec. 3 per sector, global top-chi truncation, gauge, P and P~.
    Returns (q, P3 [T4.U, a.U, new] of the lower-left site, Pt3 [new, T4.D,
    a.D] of the upper-left site, new_leg, info)."""
    q = cell_quarters(ul, ur, ll, lr)
    Rt, Rb = q["Rt"], q["Rb"]
    beta_legs = [ur["T2"][0][2], ur["a"][0][3]]    # T2.D, a.D  (top half, right cut)
    betap_legs = [lr["T2"][0][0], lr["a"][0][1]]   # T2.U, a.U  (bottom half, right cut)
    alpha_dims = (ul["T4"][0][2].dim, ul["a"][0][3].dim)
    alphap_dims = (ll["T4"][0][0].dim, ll["a"][0][1].dim)
    na, nap = int(np.prod(alpha_dims)), int(np.prod(alphap_dims))
    Rt_m = Rt.reshape(na, -1)                 # [alpha, beta]
    Rb_m = Rb.reshape(nap, -1)                # [alpha', beta']
    N = Rt_m.T @ Rb_m                         # [beta, beta']
    kb = sector_keys(beta_legs, -1)
    kbp = sector_keys(betap_legs, +1)
    f_new = ll["C1"][0][1].flow               # the new bond keeps C1.D's flow
    mod = modulus(beta_legs)
    secs = {}
    cands = []
    for key in sorted(set(kb.tolist()) & set(kbp.tolist())):
        rows = np.nonzero(kb == key)[0]
        cols = np.nonzero(kbp == key)[0]
        U, S, Vt = np.linalg.svd(N[np.ix_(rows, cols)], full_matrices=False)
        secs[key] = (rows, cols, U, S, Vt.T)
        for j, s in enumerate(S):
            cands.append((float(s), reduce(f_new * key, mod), key, j))
    kept = truncate(cands, chi, rel_cutoff)
    # new leg: ascending charge, descending sigma inside a sector
    by_q = {}
    for s, qn, key, j in kept:
        by_q.setdefault(qn, []).append((key, j))
    new_charges = tuple(sorted(by_q))
    new_degs = tuple(len(by_q[c]) for c in new_charges)
    n_new = sum(new_degs)
    P = np.zeros((nap, n_new))
    Pt = np.zeros((n_new, na))
    svals = np.zeros(n_new)
    col = 0
    for c in new_charges:
        for key, j in sorted(by_q[c], key=lambda t: t[1]):
            rows, cols, U, S, V = secs[key]
            u = U[:, j].copy()
            v = V[:, j].copy()
            i = int(np.argmax(np.abs(u)))
            if u[i] < 0:
                u, v = -u, -v
            s = S[j]
            # P = R_bot V S^-1/2 ;  P~ = S^-1/2 U^T R_top^T
            P[:, col] = Rb_m[:, cols] @ v / np.sqrt(s)
            Pt[col, :] = (Rt_m[:, rows] @ u) / np.sqrt(s)
            svals[col] = s
            col += 1
    new_leg = Leg(f_new, new_charges, new_degs, mod)
    P3 = P.reshape(alphap_dims + (n_new,))
    Pt3 = Pt.reshape((n_new,) + alpha_dims)
    info = {"svals": svals, "P": P, "Pt": Pt, "N": N, "kept": len(kept), "new_leg": new_leg,
            "sectors": secs, "kb": kb, "kbp": kbp}
    return q, P3, Pt3, new_leg, info


def renormalise(net, X1, P3_above, Pt3_above, leg_above, P3_below, Pt3_below, leg_below):
    """Column absorption of one site (Sec. 3): C1' = (C1 T1) P (the
    projector of the cut above the site), T4' = P~ (T4 a) P (above, below),
    C4' = P~ (C4 T3) (below); each divided by its Frobenius norm.  Returns
    the three (legs, dense) pairs and the norms."""
    L = {r: net[r][0] for r in ROLES}
    C1, T1, C2, T2, C3, T3, C4, T4, a = (net[r][1] for r in ROLES)
    e = lambda s, *x: np.einsum(s, *x, optimize=True)
    C1n = e("dkx,dkc->xc", X1, P3_above)
    W = e("cuk,umd->ckmd", Pt3_above, T4)                   # [chi, a.U, T4.R, T4.D]
    Z = e("ckmd,mkre->cdre", W, a)                          # [chi, T4.D, a.R, a.D]
    T4n = e("cdre,dex->crx", Z, P3_below)                   # [chi, a.R, chi]
    Y = e("ur,rkx->ukx", C4, T3)                            # [C4.U, T3.U, T3.R]
    C4n = e("cuk,ukx->cx", Pt3_below, Y)
    norms = []
    for t in (C1n, T4n, C4n):
        norms.append(float(np.linalg.norm(t)))
    C1n, T4n, C4n = C1n / norms[0], T4n / norms[1], C4n / norms[2]
    return (([L["T1"][2], leg_above], C1n), ([leg_above.dual(), L["a"][2], leg_below], T4n),
            ([leg_below.dual(), L["T3"][2]], C4n), norms)


def left_move(net, chi, rel_cutoff=1e-14, return_info=False):
    """One LEFT move; returns the updated network (C1, T4, C4 replaced)."""
    q, P3, Pt3, new_leg, info = plaquette_projector(net, net, net, net, chi, rel_cutoff)
    C1n, T4n, C4n, norms = renormalise(net, q["X1"], P3, Pt3, new_leg, P3, Pt3, new_leg)
    out = dict(net)
    out["C1"], out["T4"], out["C4"] = C1n, T4n, C4n
    if return_info:
        info["norms"] = norms
        return out, info
    return out


def move(net, direction, chi, rel_cutoff=1e-14, return_info=False):
    """Directional move: rotate so that `direction` is LEFT, move, rotate back."""
    k = DIR_ROTATIONS[direction]
    r = rotate(net, k)
    res = left_move(r, chi, rel_cutoff, return_info)
    if return_info:
        r2, info = res
    else:
        r2, info = res, None
    back = rotate(r2, (4 - k) % 4)
    return (back, info) if return_info else back


def full_move(net, chi, rel_cutoff=1e-14):
    """L, R, U, D moves in sequence, each on the updated environment."""
    for d in "LRUD":
        net = move(net, d, chi, rel_cutoff)
    return net


# ---------------------------------------------------------------------------
# Unit cells (Sec. 3.1 and Sec. 4.1: the 2 x 2 cell of the timings): an
# Lx x Ly cell holds a site tensor per position (x right, y down), each with
# its own environment; cell["site"][(x, y)] is that site's net (its C1..C4,
# T1..T4 and a).  The LEFT move absorbs the cell column by column: for
# column x every plaquette (x, y), (x+1, y), (x, y+1), (x+1, y+1) gives the
# projectors of the cut between rows y and y+1, and column x is absorbed
# into the left environment of column x+1 (C1' with the cut above the row,
# T4' between the cuts above and below, C4' with the cut below), as the
# directional scheme the paper cites for its CTM (Sec. 3) does.  A 1 x 1
# cell is the one-site move.

def cell_left_move(cell, chi, rel_cutoff=1e-14, return_info=False):
    Lx, Ly = cell["Lx"], cell["Ly"]
    S = {k: dict(v) for k, v in cell["site"].items()}
    infos = []
    for x in range(Lx):
        xr = (x + 1) % Lx
        proj = {}
        for y in range(Ly):
            yd = (y + 1) % Ly
            proj[y] = plaquette_projector(S[(x, y)], S[(xr, y)], S[(x, yd)], S[(xr, yd)], chi, rel_cutoff)
        new = {}
        for y in range(Ly):
            qa, P3a, Pt3a, la, _ = proj[(y - 1) % Ly]
            qb, P3b, Pt3b, lb, _ = proj[y]
            new[y] = renormalise(S[(x, y)], qb["X1"], P3a, Pt3a, la, P3b, Pt3b, lb)
        for y in range(Ly):
            C1n, T4n, C4n, norms = new[y]
            tgt = S[(xr, y)]
            tgt["C1"], tgt["T4"], tgt["C4"] = C1n, T4n, C4n
            infos.append({"x": x, "y": y, "norms": norms, "info": proj[y][4]})
    out = {"Lx": Lx, "Ly": Ly, "site": S}
    return (out, infos) if return_info else out


def rotate_cell(cell, k):
    """The cell seen after k counter-clockwise quarter turns: the site at
    (x, y) moves to (y, -x mod Lx) (right becomes up, down becomes right)
    and every net is rotated as the one-site network is."""
    for _ in range(k % 4):
        Lx, Ly = cell["Lx"], cell["Ly"]
        cell = {"Lx": Ly, "Ly": Lx,
                "site": {(y, (-x) % Lx): rotate_ccw(net) for (x, y), net in cell["site"].items()}}
    return cell


def cell_move(cell, direction, chi, rel_cutoff=1e-14):
    k = DIR_ROTATIONS[direction]
    out = cell_left_move(rotate_cell(cell, k), chi, rel_cutoff)
    return rotate_cell(out, (4 - k) % 4)


def cell_full_move(cell, chi, rel_cutoff=1e-14):
    """L, R, U, D cell moves in sequence."""
    for d in "LRUD":
        cell = cell_move(cell, d, chi, rel_cutoff)
    return cell


def row_value(cell, x, y):
    """The 3 x 4 network of row y across columns x and x+1:
    C1 T1 T1' C2' / T4 a a' T2' / C4 T3 T3' C3' (primes: column x+1)."""
    Lx = cell["Lx"]
    return _row_value(cell["site"][(x, y)], cell["site"][((x + 1) % Lx, y)])


def _row_value(s0, s1):
    C1, T1, C2, T2, C3, T3, C4, T4, a = (s0[r][1] for r in ROLES)
    T1b, C2b, T2b, C3b, T3b, ab = (s1[r][1] for r in ("T1", "C2", "T2", "C3", "T3", "a"))
    e = lambda s, *x: np.einsum(s, *x, optimize=True)
    top = e("ab,akc,clf,fd->bkld", C1, T1, T1b, C2b)        # [C1.D, T1.D, T1'.D, C2'.D]
    mid = e("bmh,mkrn,rlgs,dge->bkldhnse", T4, a, ab, T2b)  # [T4.U, a.U, a'.U, T2'.U, T4.D, a.D, a'.D, T2'.D]
    bot = e("hi,inj,jso,eo->hnse", C4, T3, T3b, C3b)        # [C4.U, T3.U, T3'.U, C3'.U]
    return float(e("bkld,bkldhnse,hnse->", top, mid, bot))


def network_value(net):
    """Full 3x3 contraction C1 T1 C2 / T4 a T2 / C4 T3 C3."""
    C1, T1, C2, T2, C3, T3, C4, T4, a = (net[r][1] for r in ROLES)
    return float(np.einsum("ab,akc,cd,dme,ef,gnf,hg,bph,pkmn->", C1, T1, C2, T2, C3, T3,
                           C4, T4, a, optimize=True))


def kappa(net):
    """Partition function per site from a converged environment:
    Z(1x1) Z(0x0) / (Z(1x0) Z(0x1))."""
    C1, T1, C2, T2, C3, T3, C4, T4, a = (net[r][1] for r in ROLES)
    z11 = network_value(net)
    z00 = np.einsum("ab,ad,de,be->", C1, C2, C3, C4, optimize=True)
    # top and bottom edges joined directly (no site)
    z10 = np.einsum("ab,akc,cd,de,gke,bg->", C1, T1, C2, C3, T3, C4, optimize=True)
    # left and right edges joined directly (no site)
    z01 = np.einsum("ab,ad,dme,ef,hf,bmh->", C1, C2, T2, C3, C4, T4, optimize=True)
    return float(z11 * z00 / (z10 * z01))


def env_legs(x_leg_charges, x_leg_degs, a_legs):
    """Leg lists of the eight environment tensors around a site with legs
    a_legs = [L, U, R, D].  Environment bonds flow left-to-right along the
    rows and top-to-bottom along the columns; an edge tensor's site leg is
    the dual of the site leg it touches."""
    X = lambda f: Leg(f, tuple(x_leg_charges), tuple(x_leg_degs), a_legs[0].mod)
    kl, ku, kr, kd = a_legs
    return {"C1": [X(-1), X(-1)], "C2": [X(1), X(-1)], "C3": [X(1), X(1)], "C4": [X(1), X(-1)],
            "T1": [X(1), ku.dual(), X(-1)], "T2": [X(1), kr.dual(), X(-1)],
            "T3": [X(1), kd.dual(), X(-1)], "T4": [X(1), kl.dual(), X(-1)]}


def u1_network(cfg, seed=0):
    """Dense network of a U(1) workload: double layer with remover plus a
    random symmetric environment, all from the seeded recipe."""
    from . import u1
    from workloads import values
    A_legs = [u1.leg_from_spec(s) for s in cfg["A"]]
    R_legs = [u1.leg_from_spec(s) for s in cfg["R"]]
    A = u1.to_dense(A_legs, values(seed, "A", u1.nnz(A_legs)))
    R = u1.to_dense(R_legs, values(seed, "R", u1.nnz(R_legs)))
    a_legs, a = u1.double_layer(A_legs, A, R_legs, R)
    net = {}
    for r, lg in env_legs(cfg["x"][0], cfg["x"][1], a_legs).items():
        net[r] = (lg, u1.to_dense(lg, values(seed, r, u1.nnz(lg))))
    net["a"] = (a_legs, a)
    return net
