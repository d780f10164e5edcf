"""Pins of the oracle's CTMRG move: exactness without truncation, the
projector identities, sector-wise SVD against the dense SVD, and two lattice
models with closed-form free energies (Onsager's Ising solution and Lieb's
square ice)."""
import numpy as np
import pytest
from scipy import integrate

from oracle import ctm, u1
from workloads import u1_config


def zleg(f, d):
    return u1.Leg(f, (0,), (d,))


def dense_net(rng, D=2, X=3):
    a_legs = [zleg(1, D), zleg(1, D), zleg(-1, D), zleg(-1, D)]
    legs = ctm.env_legs((0,), (X,), a_legs)
    net = {r: (lg, rng.random([l.dim for l in lg])) for r, lg in legs.items()}
    net["a"] = (a_legs, rng.random((D,) * 4))
    return net


def z34(net):
    """3x4 network C1 T1 T1 C2 / T4 a a T2 / C4 T3 T3 C3."""
    C1, T1, C2, T2, C3, T3, C4, T4, a = (net[r][1] for r in ctm.ROLES)
    return np.einsum("ab,akc,cjx,xd,bph,pkqn,qjmy,dme,hg,gnw,wyf,ef->",
                     C1, T1, T1, C2, T4, a, a, T2, C4, T3, T3, C3, optimize=True)


def z44(net):
    """4x4 network (two rows and two columns of sites), contracted row by row."""
    C1, T1, C2, T2, C3, T3, C4, T4, a = (net[r][1] for r in ctm.ROLES)
    e = lambda s, *x: np.einsum(s, *x, optimize=True)
    row = e("ab,akc,cjx,xd->bkjd", C1, T1, T1, C2)
    for _ in range(2):
        row = e("bkjd,bph->kjdph", row, T4)
        row = e("kjdph,pkqn->jdhqn", row, a)
        row = e("jdhqn,qjmy->dhnmy", row, a)
        row = e("dhnmy,dme->hnye", row, T2)
    row = e("hnye,hg->gnye", row, C4)
    row = e("gnye,gnw->wye", row, T3)
    row = e("wye,wyf->ef", row, T3)
    return e("ef,ef->", row, C3)


def test_move_is_exact_without_truncation_full_rank():
    """Full-rank half systems and every singular value kept: P P~ is the
    identity, so the renormalised 3x3 network equals the 3x4 network with
    the absorbed column (times the normalisation factors)."""
    net = dense_net(np.random.default_rng(0))
    out, info = ctm.left_move(net, 10 ** 6, return_info=True)
    assert info["kept"] == 6
    got = ctm.network_value(out) * np.prod(info["norms"])
    assert abs(got / z34(net) - 1) < 1e-9


@pytest.mark.parametrize("name", ["tiny", "d4chi16"])
def test_projectors_preserve_the_four_by_four_network(name):
    """Tr(N) is the 4x4 network; with every non-zero singular value kept,
    inserting P P~ into the left cut leaves it unchanged."""
    net = ctm.u1_network(u1_config(name))
    out, info = ctm.left_move(net, 10 ** 6, return_info=True)
    q = ctm.quarters(net)
    na = info["Pt"].shape[1]
    Rt = q["Rt"].reshape(na, -1)
    Rb = q["Rb"].reshape(info["P"].shape[0], -1)
    ref = z44(net)
    assert abs(np.trace(info["N"]) / ref - 1) < 1e-12
    got = np.trace(Rt.T @ info["P"] @ info["Pt"] @ Rb)
    assert abs(got / ref - 1) < 1e-9


def test_projector_identities_and_sector_svd():
    net = ctm.u1_network(u1_config("d4chi16"))
    out, info = ctm.left_move(net, 16, return_info=True)
    k = info["kept"]
    assert k == 16
    assert np.abs(info["Pt"] @ info["P"] - np.eye(k)).max() < 1e-12
    # the union of the sector spectra is the spectrum of the dense N
    N = info["N"]
    dense_s = np.sort(np.linalg.svd(N, compute_uv=False))[::-1]
    sec_s = np.sort(np.concatenate([s[3] for s in info["sectors"].values()]))[::-1]
    n = len(sec_s)
    assert np.allclose(sec_s, dense_s[:n], rtol=1e-10, atol=1e-12 * dense_s[0])
    assert np.all(dense_s[n:] < 1e-10 * dense_s[0])
    # the kept values are the top-chi of the dense spectrum
    assert np.allclose(np.sort(info["svals"])[::-1], dense_s[:k], rtol=1e-12)
    # N is zero outside the charge-matched sector blocks
    mask = info["kb"][:, None] == info["kbp"][None, :]
    assert np.all(N[~mask] == 0.0)
    for r in ("C1", "T4", "C4"):
        legs, arr = out[r]
        assert np.all(arr[~u1.allowed_mask(legs)] == 0.0)
        assert abs(np.linalg.norm(arr) - 1) < 1e-13


def test_rotation_by_four_quarter_turns_is_identity():
    net = ctm.u1_network(u1_config("tiny"))
    r4 = ctm.rotate(net, 4)
    for r in ctm.ROLES:
        assert np.array_equal(r4[r][1], net[r][1])
        assert r4[r][0] == net[r][0]


def onsager_kappa(beta):
    k = 2 * beta
    f = lambda t1, t2: np.log(np.cosh(k) ** 2 - np.sinh(k) * (np.cos(t1) + np.cos(t2)))
    val, _ = integrate.dblquad(f, 0, np.pi, 0, np.pi, epsabs=1e-13, epsrel=1e-13)
    return np.exp(np.log(2) + val / (2 * np.pi ** 2))


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
@pytest.mark.parametrize("beta", [0.3, 0.6])
def test_ising_free_energy_onsager(beta):
    """Classical 2D Ising model (one sector per leg): the partition function
    per site from the converged environment equals Onsager's closed form."""
    B = np.array([[np.exp(beta), np.exp(-beta)], [np.exp(-beta), np.exp(beta)]])
    w, v = np.linalg.eigh(B)
    M = v @ np.diag(np.sqrt(w)) @ v.T
    a = np.einsum("sl,su,sr,sd->lurd", M, M, M, M)
    a_legs = [zleg(1, 2), zleg(1, 2), zleg(-1, 2), zleg(-1, 2)]
    net = {r: (lg, np.ones([l.dim for l in lg]))
           for r, lg in ctm.env_legs((0,), (1,), a_legs).items()}
    net["a"] = (a_legs, a)
    for _ in range(60):
        net = ctm.full_move(net, 8)
    assert abs(ctm.kappa(net) / onsager_kappa(beta) - 1) < 1e-10


def test_square_ice_lieb():
    """Six-vertex ice model, U(1) arrow conservation on every leg: 2x2 sites
    form one site (outer legs fused pairwise, all fused charges even), so the
    one-site environment is consistent.  Partition function per 2x2 site ->
    Lieb's W^4, W = (4/3)^(3/2); critical, so the error decays slowly in chi."""
    s = u1.Leg(1, (-1, 1), (1, 1))
    ice = u1.to_dense([s, s, s.dual(), s.dual()], np.ones(6))
    big = np.einsum("aUhV,hWbX,cViY,iXdZ->acUWbdYZ", ice, ice, ice, ice)
    fl, F = u1.fuse([s, s])
    fr, Fr = u1.fuse([s.dual(), s.dual()])
    a = np.einsum("abcdefgh,Lab,Ucd,Ref,Dgh->LURD", big, F, F, Fr, Fr)
    a_legs = [fl, fl, fr, fr]
    assert np.all(a[~u1.allowed_mask(a_legs)] == 0.0)
    net = {r: (lg, u1.to_dense(lg, np.ones(u1.nnz(lg))))
           for r, lg in ctm.env_legs((-2, 0, 2), (1, 1, 1), a_legs).items()}
    net["a"] = (a_legs, a)
    for _ in range(40):
        net = ctm.full_move(net, 32)
    W4 = (4.0 / 3.0) ** 6
    assert abs(ctm.kappa(net) / W4 - 1) < 5e-5


# One counter-clockwise quarter turn written out tensor by tensor (the
# geometry, independent of the oracle's rotation tables): after the turn a
# leg that pointed up points left, left -> down, down -> right, right -> up.
# new role <- (old role, axes of the old tensor in the new role's leg order)
HAND_CCW = {
    "C1": ("C2", (1, 0)),        # [R, D] <- C2[L, D]: old D now points R, old L now D
    "T4": ("T1", (2, 1, 0)),     # [U, R, D] <- T1[L, D, R]
    "C4": ("C1", (0, 1)),        # [U, R] <- C1[R, D]
    "T3": ("T4", (0, 1, 2)),     # [L, U, R] <- T4[U, R, D]
    "C3": ("C4", (1, 0)),        # [U, L] <- C4[U, R]
    "T2": ("T3", (2, 1, 0)),     # [U, L, D] <- T3[L, U, R]
    "C2": ("C3", (0, 1)),        # [L, D] <- C3[U, L]
    "T1": ("T2", (0, 1, 2)),     # [L, D, R] <- T2[U, L, D]
    "a": ("a", (1, 2, 3, 0)),    # [L, U, R, D] <- a[L, U, R, D]: old U now L, R now U, ...
}


def hand_ccw(net):
    out = {}
    for new, (old, ax) in HAND_CCW.items():
        legs, arr = net[old]
        out[new] = ([legs[i] for i in ax], np.ascontiguousarray(np.transpose(arr, ax)))
    return out


def hand_rotate(net, k):
    for _ in range(k % 4):
        net = hand_ccw(net)
    return net


@pytest.mark.parametrize("k", [1, 2, 3])
def test_rotation_keeps_the_network_value(k):
    """A rotated network is the same contraction: the 3x3 value of a random,
    anisotropic network (distinct environment tensors, a site without
    symmetry between its legs) does not change; the oracle's rotation equals
    the hand-written quarter turns."""
    net = ctm.u1_network(u1_config("tiny"))
    ref = ctm.network_value(net)
    rot = ctm.rotate(net, k)
    assert abs(ctm.network_value(rot) / ref - 1) < 1e-12
    hand = hand_rotate(net, k)
    for r in ctm.ROLES:
        assert rot[r][0] == hand[r][0], r
        assert np.array_equal(rot[r][1], hand[r][1]), r


@pytest.mark.parametrize("direction", ["U", "R", "D"])
def test_directional_move_is_the_left_move_of_the_turned_network(direction):
    """UP, RIGHT and DOWN moves equal a LEFT move on the network turned by
    hand (1, 2, 3 counter-clockwise quarter turns) and turned back."""
    k = {"U": 1, "R": 2, "D": 3}[direction]
    net = ctm.u1_network(u1_config("tiny"))
    chi = u1_config("tiny")["chi"]
    got = ctm.move(net, direction, chi)
    want = hand_rotate(ctm.left_move(hand_rotate(net, k), chi), 4 - k)
    renewed = {"U": ("C1", "T1", "C2"), "R": ("C2", "T2", "C3"), "D": ("C3", "T3", "C4")}[direction]
    for r in ctm.ROLES:
        assert got[r][0] == want[r][0], r
        assert np.allclose(got[r][1], want[r][1], rtol=0, atol=1e-14), r
    for r in set(ctm.ROLES) - set(renewed):
        assert np.array_equal(got[r][1], net[r][1]), r
    for r in renewed:
        assert not np.array_equal(got[r][1].shape, net[r][1].shape) or not np.allclose(got[r][1], net[r][1])
