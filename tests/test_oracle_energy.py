"""Pins of the oracle's two-site observables (open double layer, reduced
density matrix from the environment, Heisenberg bond energy) against a
brute-force state vector of a finite cluster, exact product-state values,
and the closed network; and of the paper's CTM error procedure."""
import numpy as np
import pytest

from oracle import ctm, energy, u1
from workloads import u1_config, values


def brute_force_pauli_bond():
    """S_i . S_j on two spins 1/2 from Pauli matrices (basis 0 = down,
    1 = up), rows (p_i p_j), columns (p_i' p_j')."""
    sx = np.array([[0.0, 1.0], [1.0, 0.0]]) / 2
    sy = np.array([[0.0, -1.0j], [1.0j, 0.0]]) / 2
    sz = np.array([[-1.0, 0.0], [0.0, 1.0]]) / 2   # index 0 down
    h = np.kron(sx, sx) + np.kron(sy, sy) + np.kron(sz, sz)
    assert np.abs(h.imag).max() == 0
    return h.real


def test_heisenberg_bond_matches_pauli_matrices():
    H = energy.heisenberg_bond()
    h = brute_force_pauli_bond()
    assert np.allclose(np.transpose(H, (0, 2, 1, 3)).reshape(4, 4), h, atol=1e-15)
    # singlet -3/4, triplet +1/4
    w = np.sort(np.linalg.eigvalsh(h))
    assert np.allclose(w, [-0.75, 0.25, 0.25, 0.25])
    # total S^z conserved: allowed by the U(1) rule on [p_i, p_i', p_j, p_j']
    p = u1.Leg(1, (-1, 1), (1, 1))
    legs = [p, p.dual(), p, p.dual()]
    assert np.all(H[~u1.allowed_mask(legs)] == 0.0)


def site_with_boundary(seed=0):
    """A small U(1) site, remover and boundary vectors: every environment
    bond has dimension 1 (charge 0), each edge tensor is b (x) b on the
    fused site leg it touches, so the 3 x 4 network is the 1 x 2 cluster
    with open boundaries fixed to b."""
    rng = np.random.default_rng(seed)
    p = u1.Leg(1, (-1, 1), (1, 1))
    l = u1.Leg(1, (-1, 1), (2, 1))
    e_in, e_out = u1.Leg(1, (-2, 0, 2), (1, 2, 1)), u1.Leg(-1, (-2, 0, 2), (1, 2, 1))
    A_legs = [p, l, e_in, e_out, e_out]
    R_legs = [e_in, l.dual(), u1.Leg(-1, (-1, 1), (1, 1))]
    A = u1.to_dense(A_legs, rng.standard_normal(u1.nnz(A_legs)))
    R = u1.to_dense(R_legs, rng.standard_normal(u1.nnz(R_legs)))
    # boundary vectors inside one charge sector of each virtual leg
    b_l = np.zeros(l.dim)
    b_l[:2] = rng.standard_normal(2)          # charge -1 sector
    b_e = np.zeros(e_in.dim)
    b_e[1:3] = rng.standard_normal(2)         # charge 0 sector
    return A_legs, A, R_legs, R, b_l, b_e


def boundary_network(A_legs, A, R_legs, R, b_l, b_e):
    site_legs, site = energy.open_double_layer(A_legs, A, R_legs, R)
    kl, ku, kr, kd = site_legs[:4]
    net = {}
    x = (0,), (1,)
    legs = ctm.env_legs(x[0], x[1], site_legs[:4])
    fl = u1.fuse([A_legs[1], A_legs[1].dual()])[1]
    fe = u1.fuse([A_legs[2], A_legs[2].dual()])[1]
    fr = u1.fuse([R_legs[1], R_legs[1].dual()])[1]
    vl = np.einsum("kab,a,b->k", fl, b_l, b_l)    # left boundary on k_l
    vr = np.einsum("kab,a,b->k", fr, b_l, b_l)    # right boundary on the remover's l'
    ve = np.einsum("kab,a,b->k", fe, b_e, b_e)    # top and bottom boundaries
    for r in ("C1", "C2", "C3", "C4"):
        net[r] = (legs[r], np.ones((1, 1)))
    net["T1"] = (legs["T1"], ve.reshape(1, -1, 1))
    net["T3"] = (legs["T3"], ve.reshape(1, -1, 1))
    net["T4"] = (legs["T4"], vl.reshape(1, -1, 1))
    net["T2"] = (legs["T2"], vr.reshape(1, -1, 1))
    for r in ("T1", "T2", "T3", "T4"):
        assert np.all(net[r][1][~u1.allowed_mask(net[r][0])] == 0.0), r
    return site_legs, site, net


def test_rdm_of_the_boundary_cluster_is_the_brute_force_one():
    """Horizontal bond: psi_s[p_i, p_j] = sum A_i R A_j R with the boundary
    vectors on the open legs, rho = sum over the removers' extra legs s of
    psi_s psi_s^T; the environment contraction reproduces it and the bond
    energy, for the vertical bond too."""
    A_legs, A, R_legs, R, b_l, b_e = site_with_boundary()
    site_legs, site, net = boundary_network(A_legs, A, R_legs, R, b_l, b_e)
    h = brute_force_pauli_bond()
    # horizontal: i then j, the remover of i between them, that of j at the right edge
    psi = np.einsum("plurd,l,u,d,rxs,qxvwe,v,e,wyt,y->pqst", A, b_l, b_e, b_e, R, A, b_e, b_e, R, b_l, optimize=True)
    psi = psi.reshape(4, -1)
    rho_bf = psi @ psi.T
    rho = energy.bond_rdm(net, site_legs, site, "h")
    got = np.transpose(rho, (0, 2, 1, 3)).reshape(4, 4)
    assert np.allclose(got, rho_bf, rtol=0, atol=1e-13 * np.abs(rho_bf).max())
    e_bf = np.trace(rho_bf @ h) / np.trace(rho_bf)
    assert abs(energy.bond_energy(rho, energy.heisenberg_bond()) - e_bf) < 1e-13
    # vertical: i above j (i's down leg meets j's up leg), each remover at the right edge
    psi = np.einsum("plurd,l,u,rxs,x,qmdvw,m,w,vyt,y->pqst", A, b_l, b_e, R, b_l, A, b_l, b_e, R, b_l, optimize=True)
    psi = psi.reshape(4, -1)
    rho_bf = psi @ psi.T
    rho = energy.bond_rdm(net, site_legs, site, "v")
    got = np.transpose(rho, (0, 2, 1, 3)).reshape(4, 4)
    assert np.allclose(got, rho_bf, rtol=0, atol=1e-13 * np.abs(rho_bf).max())


def test_ferromagnetic_product_state():
    """Bond dimension 1, every spin up: every bond has <S.S> = 1/4 exactly."""
    p = u1.Leg(1, (-1, 1), (1, 1))
    A_legs = [p, u1.Leg(1, (-1,), (1,)), u1.Leg(1, (0,), (1,)), u1.Leg(-1, (0,), (1,)), u1.Leg(-1, (0,), (1,))]
    R_legs = [u1.Leg(1, (0,), (1,)), u1.Leg(-1, (-1,), (1,)), u1.Leg(-1, (-1, 1), (1, 1))]
    A = u1.to_dense(A_legs, [1.3])
    R = u1.to_dense(R_legs, [0.7])
    site_legs, site = energy.open_double_layer(A_legs, A, R_legs, R)
    a_legs, a = u1.double_layer(A_legs, A, R_legs, R)
    net = {r: (lg, np.ones([l.dim for l in lg])) for r, lg in ctm.env_legs((0,), (1,), a_legs).items()}
    net["a"] = (a_legs, a)
    H = energy.heisenberg_bond()
    assert abs(energy.bond_energy(energy.bond_rdm(net, site_legs, site, "h"), H) - 0.25) < 1e-15
    assert abs(energy.site_energy(net, site_legs, site, H) - 0.5) < 1e-15


def test_rdm_trace_is_the_closed_network():
    """Tr rho = the 3 x 4 network with both sites closed (the double layer
    sums p = p'), for a random (not positive) environment too; forbidden
    charge blocks of rho are exactly zero."""
    from test_oracle_ctm import z34
    cfg = u1_config("tiny")
    net = ctm.u1_network(cfg)
    A_legs = [u1.leg_from_spec(s) for s in cfg["A"]]
    R_legs = [u1.leg_from_spec(s) for s in cfg["R"]]
    A = u1.to_dense(A_legs, values(0, "A", u1.nnz(A_legs)))
    R = u1.to_dense(R_legs, values(0, "R", u1.nnz(R_legs)))
    site_legs, site = energy.open_double_layer(A_legs, A, R_legs, R)
    assert np.allclose(np.einsum("lurdpp->lurd", site), net["a"][1], atol=1e-13)
    rho = energy.bond_rdm(net, site_legs, site, "h")
    assert abs(np.einsum("aabb->", rho) / z34(net) - 1) < 1e-12
    p = A_legs[0]
    assert np.all(rho[~u1.allowed_mask([p, p.dual(), p, p.dual()])] == 0.0)


def test_error_procedure_on_the_ising_model():
    """The error procedure stops when two fixed-chi results agree to the
    threshold; on the Ising model it reaches Onsager's value within the
    error it reports."""
    from test_oracle_ctm import onsager_kappa
    beta = 0.3
    B = np.array([[np.exp(beta), np.exp(-beta)], [np.exp(-beta), np.exp(beta)]])
    w, v = np.linalg.eigh(B)
    M = v @ np.diag(np.sqrt(w)) @ v.T
    a = np.einsum("sl,su,sr,sd->lurd", M, M, M, M)
    z = lambda f: u1.Leg(f, (0,), (2,))
    a_legs = [z(1), z(1), z(-1), z(-1)]
    net = {r: (lg, np.ones([l.dim for l in lg])) for r, lg in ctm.env_legs((0,), (1,), a_legs).items()}
    net["a"] = (a_legs, a)
    val, err, hist, _ = energy.converge(net, 4, ctm.kappa, tol=1e-8, chi_max=16)
    assert all(len(v) <= 15 for _, v in hist)
    assert [c for c, _ in hist][:2] == [4, 8]
    assert abs(val - onsager_kappa(beta)) <= max(err, 1e-8) * 10
