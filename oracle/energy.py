"""Dense oracle of two-site observables from a CTMRG environment and of the
paper's CTM error procedure.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* Open double layer (Sec. 3.2 with the physical leg kept open): the ket A
  and the bra A* are multiplied without the sum over the physical index;
  ket/bra virtual legs are fused pairwise as in the closed double layer, and
  the remover's double layer (its extra leg s traced between ket and bra,
  Sec. 3.1) is absorbed on the right leg.  Legs [kl, ku, kr, kd, p, p'],
  p the ket's physical leg, p' the bra's (its dual).
* Two-site reduced density matrix of a horizontal bond (site i and its right
  neighbour j) from the one-site environment: the 3 x 4 network
      C1 T1 T1 C2 / T4 a_i a_j T2 / C4 T3 T3 C3
  with both sites open; legs [p_i, p_i', p_j, p_j'].  A vertical bond is the
  horizontal bond of the network turned by a quarter turn (the upper site
  becomes the left one).
* Bond energy of H_ij = S_i . S_j (the spin-1/2 Heisenberg coupling of
  Sec. 4.1) = Tr(rho H) / Tr(rho).  H conserves the total S^z, so as a
  tensor with the density matrix's legs it is a U(1)-symmetric tensor (the
  product S^+_i S^-_j of two charged operators, whose extra legs carry the
  charge between the sites, Sec. 3.1, contracted).
* The error procedure of Sec. 3 (implementation details): CTM steps at
  fixed chi until the observable changes by less than a threshold (1e-8)
  or 15 steps are done; the first error is the largest change among the
  last three steps; chi is then doubled and the procedure repeated until
  two results differ by less than the threshold or chi exceeds 128; the
  second error is the change between the last two fixed-chi results; the
  error is the larger of the two.
"""
from __future__ import annotations

import numpy as np

from . import ctm, u1


def open_double_layer(A_legs, A, R_legs=None, R=None):
    """a[kl, ku, kr, kd, p, p'] = A[p, ...] A*[p', ...] with virtual ket/bra
    legs fused (the closed double layer summed over p = p'), remover
    absorbed on the right leg.  Returns (legs, dense)."""
    kl, Fl = u1.fuse([A_legs[1], A_legs[1].dual()])
    ku, Fu = u1.fuse([A_legs[2], A_legs[2].dual()])
    kr, Fr = u1.fuse([A_legs[3], A_legs[3].dual()])
    kd, Fd = u1.fuse([A_legs[4], A_legs[4].dual()])
    a = np.einsum("plurd,PLURD,alL,buU,crR,edD->abcepP", A, A, Fl, Fu, Fr, Fd, optimize=True)
    legs = [kl, ku, kr, kd, A_legs[0], A_legs[0].dual()]
    if R is not None:
        kr_in, Fri = u1.fuse([R_legs[0], R_legs[0].dual()])
        kl_out, Flo = u1.fuse([R_legs[1], R_legs[1].dual()])
        rho = np.einsum("rls,RLs,arR,blL->ab", R, R, Fri, Flo, optimize=True)
        assert kr_in.same_space(kr) and kr_in.flow == -kr.flow
        a = np.einsum("lurdpP,rx->luxdpP", a, rho)
        legs = [kl, ku, kl_out, kd, A_legs[0], A_legs[0].dual()]
    return legs, a


def rotate_open_site(legs, a, k=1):
    """The open site seen after k counter-clockwise quarter turns: its
    virtual legs permuted as the closed site's (old U points left, ...)."""
    for _ in range(k % 4):
        perm = (1, 2, 3, 0, 4, 5)
        legs = [legs[i] for i in perm]
        a = np.ascontiguousarray(np.transpose(a, perm))
    return legs, a


def bond_rdm(net, site_legs, site, bond="h"):
    """Two-site reduced density matrix rho[p_i, p_i', p_j, p_j'] (not
    normalised) of a horizontal ("h") or vertical ("v") bond; net holds the
    environment (the closed site is not used)."""
    if bond == "v":
        if "a" not in net:  # the rotation carries a closed site along (unused here)
            net = dict(net, a=(site_legs[:4], np.einsum("lurdpp->lurd", site)))
        net = ctm.rotate(net, 1)
        site_legs, site = rotate_open_site(site_legs, site, 1)
    C1, T1, C2, T2, C3, T3, C4, T4 = (net[r][1] for r in ("C1", "T1", "C2", "T2", "C3", "T3", "C4", "T4"))
    # C1[R,D] T1[L,D,R] T1 C2[L,D] / T4[U,R,D] a_i a_j T2[U,L,D] / C4[U,R] T3[L,U,R] T3 C3[U,L],
    # contracted pairwise: the left column with site i, the right column
    # with site j, then the two halves over the three cut bonds
    def e(spec, *ops):
        return np.einsum(spec, *ops, optimize=True)
    left = e("ab,akc->bkc", C1, T1)                    # [C1.D, T1.D, T1.R]
    left = e("bkc,bmh->kcmh", left, T4)                # [T1.D, T1.R, T4.R, T4.D]
    left = e("kcmh,hg->kcmg", left, C4)                # [T1.D, T1.R, T4.R, C4.R]
    left = e("kcmg,gow->kcmow", left, T3)              # [T1.D, T1.R, T4.R, T3.U, T3.R]
    left = e("kcmow,mknoPQ->cwnPQ", left, site)        # [T1.R, T3.R, a.R, p_i, p_i']
    right = e("cjx,xd->cjd", T1, C2)                   # [T1.L, T1.D, C2.D]
    right = e("cjd,dqv->cjqv", right, T2)              # [T1.L, T1.D, T2.L, T2.D]
    right = e("cjqv,vy->cjqy", right, C3)              # [T1.L, T1.D, T2.L, C3.L]
    right = e("cjqy,wsy->cjqws", right, T3)            # [T1.L, T1.D, T2.L, T3.L, T3.U]
    right = e("cjqws,njqsRS->cwnRS", right, site)      # [T1.L, T3.L, a.L, p_j, p_j']
    return e("cwnPQ,cwnRS->PQRS", left, right)


def spin_half():
    """S^z, S^+, S^- on the physical leg with charges 2S^z = (-1, +1)
    (index 0 down, index 1 up)."""
    sz = np.diag([-0.5, 0.5])
    sp = np.array([[0.0, 0.0], [1.0, 0.0]])   # |up><down|
    return sz, sp, sp.T


def heisenberg_bond():
    """H[p_i, p_i', p_j, p_j'] = <p_i p_j| S_i . S_j |p_i' p_j'> for two
    spins 1/2: S^z S^z + (S^+ S^- + S^- S^+) / 2."""
    sz, sp, sm = spin_half()
    h = np.kron(sz, sz) + 0.5 * (np.kron(sp, sm) + np.kron(sm, sp))   # rows (p_i p_j), cols (p_i' p_j')
    return np.transpose(h.reshape(2, 2, 2, 2), (0, 2, 1, 3))


def bond_energy(rho, H):
    """Tr(rho H) / Tr(rho) with rho and H in the legs [p_i, p_i', p_j, p_j']."""
    tr = np.einsum("aabb->", rho)
    return float(np.einsum("abcd,abcd->", rho, H) / tr)


def site_energy(net, site_legs, site, H):
    """Energy per site of a one-site cell: one horizontal and one vertical
    bond."""
    return bond_energy(bond_rdm(net, site_legs, site, "h"), H) + bond_energy(bond_rdm(net, site_legs, site, "v"), H)


def converge(net, chi0, observable, tol=1e-8, max_steps=15, chi_max=128, rel_cutoff=1e-14):
    """The error procedure of Sec. 3: returns (value, error, history) where
    history lists (chi, [observable after every step]) per fixed-chi run."""
    history = []
    results = []
    chi = chi0
    err1 = 0.0
    while True:
        vals = []
        for _ in range(max_steps):
            net = ctm.full_move(net, chi, rel_cutoff)
            vals.append(observable(net))
            if len(vals) >= 2 and abs(vals[-1] - vals[-2]) < tol:
                break
        tail = vals[-3:] if len(vals) >= 3 else vals
        err1 = max([abs(x - y) for x, y in zip(tail[1:], tail[:-1])] + [0.0])
        history.append((chi, vals))
        results.append(vals[-1])
        if len(results) >= 2 and abs(results[-1] - results[-2]) < tol:
            break
        if 2 * chi > chi_max:
            break
        chi *= 2
    err2 = abs(results[-1] - results[-2]) if len(results) >= 2 else 0.0
    return results[-1], max(err1, err2), history, net
