"""Pins of the SU(2) oracle (CPU): exact Clebsch-Gordan values, the spin
algebra, the paper's rank-2 example, rotation invariance and the completeness
of the canonical block basis."""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import su2

S2 = np.sqrt(2.0)
S3 = np.sqrt(3.0)
S6 = np.sqrt(6.0)
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("args,val", [
    ((1, 1, 1, -1, 0, 0), 1 / S2),            # <1/2 1/2 1/2 -1/2|0 0>
    ((1, -1, 1, 1, 0, 0), -1 / S2),
    ((2, 0, 2, 0, 0, 0), -1 / S3),            # <1 0 1 0|0 0>
    ((2, 2, 2, -2, 0, 0), 1 / S3),
    ((2, 2, 1, -1, 1, 1), np.sqrt(2 / 3)),    # <1 1 1/2 -1/2|1/2 1/2>
    ((2, 0, 1, 1, 1, 1), -np.sqrt(1 / 3)),
    ((1, 1, 1, 1, 2, 2), 1.0),
    ((1, 1, 1, -1, 2, 0), 1 / S2),
    ((2, 2, 2, 0, 4, 2), 1 / S2),
    ((2, 2, 2, -2, 4, 0), 1 / S6),
    ((2, 0, 2, 0, 4, 0), np.sqrt(2 / 3)),
    ((2, 0, 2, 0, 2, 0), 0.0),
    ((2, 2, 2, -2, 2, 0), 1 / S2),
    ((1, 1, 1, 1, 0, 0), 0.0),                # m1 + m2 != M
    ((2, 2, 2, 2, 2, 2), 0.0),                # m1 + m2 != M
])
def test_cg_closed_forms(args, val):
    assert su2.cg(*args) == pytest.approx(val, abs=1e-15)


@pytest.mark.parametrize("tj", range(0, 9))
def test_cg_singlet_closed_form(tj):
    # <j m j -m | 0 0> = (-1)^(j-m) / sqrt(2j+1)
    for tm in range(-tj, tj + 1, 2):
        want = (-1) ** ((tj - tm) // 2) / np.sqrt(tj + 1)
        assert su2.cg(tj, tm, tj, -tm, 0, 0) == pytest.approx(want, abs=1e-15)


def coupled_states(tj1, tj2):
    """matrix U[(m1, m2), (J, M)] of CG coefficients"""
    cols = [(tJ, tM) for tJ in range(abs(tj1 - tj2), tj1 + tj2 + 1, 2) for tM in range(tJ, -tJ - 1, -2)]
    U = np.zeros(((tj1 + 1) * (tj2 + 1), len(cols)))
    for a, b in itertools.product(range(tj1 + 1), range(tj2 + 1)):
        for c, (tJ, tM) in enumerate(cols):
            U[a * (tj2 + 1) + b, c] = su2.cg(tj1, tj1 - 2 * a, tj2, tj2 - 2 * b, tJ, tM)
    return U, cols


@pytest.mark.parametrize("tj1,tj2", [(a, b) for a in range(0, 7) for b in range(0, 7)])
def test_cg_orthogonal_and_complete(tj1, tj2):
    U, _ = coupled_states(tj1, tj2)
    assert U.shape[0] == U.shape[1]
    assert np.abs(U.T @ U - np.eye(U.shape[1])).max() < 1e-14
    assert np.abs(U @ U.T - np.eye(U.shape[0])).max() < 1e-14


@pytest.mark.parametrize("tj1,tj2", [(1, 1), (2, 1), (1, 2), (2, 2), (3, 2), (4, 3), (6, 4)])
def test_cg_against_spin_algebra(tj1, tj2):
    """Coupled states are eigenvectors of the total S^2 and S_z, are linked by
    S_+ with the positive standard factor, and |J J> has a positive
    component on m1 = j1 (the Condon-Shortley phase)."""
    U, cols = coupled_states(tj1, tj2)
    X1, Y1, Z1 = su2.spin_matrices(tj1)
    X2, Y2, Z2 = su2.spin_matrices(tj2)
    I1, I2 = np.eye(tj1 + 1), np.eye(tj2 + 1)
    Sx, Sy, Sz = (np.kron(A, I2) + np.kron(I1, B) for A, B in ((X1, X2), (Y1, Y2), (Z1, Z2)))
    S2tot = (Sx @ Sx + Sy @ Sy + Sz @ Sz).real
    Sp = (Sx + 1j * Sy).real
    for c, (tJ, tM) in enumerate(cols):
        v = U[:, c]
        J, M = tJ / 2, tM / 2
        assert np.abs(S2tot @ v - J * (J + 1) * v).max() < 1e-13
        assert np.abs(Sz.real @ v - M * v).max() < 1e-13
        if tM < tJ:
            up = cols.index((tJ, tM + 2))
            f = np.sqrt(J * (J + 1) - M * (M + 1))
            assert np.abs(Sp @ v - f * U[:, up]).max() < 1e-13
        if tM == tJ:
            # component with m1 = j1 (first index block), m2 = J - j1
            tm2 = tJ - tj1
            if abs(tm2) <= tj2:
                b = (tj2 - tm2) // 2
                assert v[0 * (tj2 + 1) + b] > 0


def test_paper_rank2_example():
    with open(os.path.join(HERE, "golden", "su2_rank2_example.json")) as f:
        g = json.load(f)
    legs = [su2.Leg(1, tuple(g["spins_doubled"]), (2, 2, 2)), su2.Leg(-1, tuple(g["spins_doubled"]), (2, 2, 2))]
    bl = su2.blocks(legs)
    assert [b[0] for b in bl] == [(0, 0), (1, 1), (2, 2)]    # only the diagonal blocks are allowed
    for (idx, tree), size, ratio in zip(bl, g["cgc_size"], g["elements_ratio_t_over_m"]):
        c = su2.basis(legs, idx, tree)
        assert c.shape == (size, size)
        assert np.array_equal(c, np.eye(size))
        assert c.size == ratio


def test_rank3_basis_is_cg():
    legs = [su2.Leg(1, (1,), (1,)), su2.Leg(1, (2,), (1,)), su2.Leg(-1, (1, 3), (1, 1))]
    for idx, tree in su2.blocks(legs):
        tJ = legs[2].spins[idx[2]]
        assert tree == (tJ,)
        c = su2.basis(legs, idx, tree)
        for a, b, m in itertools.product(range(2), range(3), range(tJ + 1)):
            assert c[a, b, m] == su2.cg(1, 1 - 2 * a, 2, 2 - 2 * b, tJ, tJ - 2 * m)


VLEG = ((0, 1, 2), (1, 2, 1))


def rand_legs(rng, flows, maxspin=3, maxdeg=2):
    """random legs with at least one allowed block"""
    while True:
        legs = _rand_legs(rng, flows, maxspin, maxdeg)
        if su2.nnz(legs) > 0:
            return legs


def _rand_legs(rng, flows, maxspin, maxdeg):
    legs = []
    for f in flows:
        ns = int(rng.integers(1, 4))
        sp = tuple(sorted(rng.choice(np.arange(0, maxspin + 1), size=ns, replace=False).tolist()))
        legs.append(su2.Leg(f, sp, tuple(int(x) for x in rng.integers(1, maxdeg + 1, size=ns))))
    return legs


FLOWS = [(1, -1), (1, 1, -1), (1, -1, -1), (-1, -1, -1), (1, 1, -1, -1), (-1, -1, -1, -1), (1, 1, 1, -1),
         (1, -1, 1, -1)]


@pytest.mark.parametrize("flows", FLOWS)
def test_tree_bases_orthogonal(flows):
    rng = np.random.default_rng(len(flows) * 10 + sum(flows))
    legs = rand_legs(rng, flows)
    by_sector = {}
    for idx, tree in su2.blocks(legs):
        by_sector.setdefault(idx, []).append(tree)
    for idx, trees in by_sector.items():
        cs = [su2.basis(legs, idx, t) for t in trees]
        for a, ca in enumerate(cs):
            ins, outs = su2.in_out(legs)
            tJ = trees[a][max(len(ins) - 2, 0)]
            assert np.sum(ca * ca) == pytest.approx(tJ + 1, rel=1e-13)
            for b in range(a):
                assert abs(np.sum(ca * cs[b])) < 1e-13


@pytest.mark.parametrize("flows", FLOWS)
@pytest.mark.parametrize("seed", range(2))
def test_rotation_invariance(flows, seed):
    """Wigner D on incoming legs and its conjugate on outgoing legs leave the
    dense expansion of any reduced data unchanged."""
    rng = np.random.default_rng(seed + 7 * len(flows))
    legs = rand_legs(rng, flows)
    x = rng.standard_normal(su2.nnz(legs))
    T = su2.to_dense(legs, x)
    theta = rng.standard_normal(3)
    R = su2.rotate(legs, T, theta)
    assert np.abs(R - T).max() < 1e-12 * max(1.0, np.abs(T).max())
    # round trip through the reduced blocks
    assert np.abs(su2.from_dense(legs, T) - x).max() < 1e-12


def test_rotation_detects_a_broken_tensor():
    """Plant a non-invariant entry: the rotation check must see it."""
    legs = [su2.Leg(1, (1,), (1,)), su2.Leg(-1, (1,), (1,))]
    T = su2.to_dense(legs, [1.0])
    T[0, 0] += 0.1
    R = su2.rotate(legs, T, np.array([0.3, 0.2, 0.1]))
    assert np.abs(R - T).max() > 1e-3


@pytest.mark.parametrize("case", range(6))
def test_wigner_eckart_contraction(case):
    """The dense contraction of two invariant tensors lies in the span of the
    output's canonical blocks (a missing or wrong tree would break this),
    and reduced -> dense -> contract -> reduced reproduces it."""
    rng = np.random.default_rng(40 + case)
    fa = [(1, -1, -1), (1, 1, -1, -1), (-1, -1, -1, -1), (1, -1, 1, -1), (1, 1, -1), (-1, 1, -1, 1)][case]
    A = rand_legs(rng, fa)
    # B: in-legs matching A's first two out-legs (or one), plus random legs
    outs = [i for i, l in enumerate(A) if l.flow == -1][:2]
    B = [A[i].dual() for i in outs] + rand_legs(rng, (-1, 1))
    a = rng.standard_normal(su2.nnz(A))
    b = rng.standard_normal(su2.nnz(B))
    legsC, c, Cd = su2.contract(A, a, B, b, outs, list(range(len(outs))))
    assert np.abs(su2.to_dense(legsC, c) - Cd).max() < 1e-12 * max(1.0, np.abs(Cd).max())
    R = su2.rotate(legsC, Cd, rng.standard_normal(3))
    assert np.abs(R - Cd).max() < 1e-11 * max(1.0, np.abs(Cd).max())


def fused_spins(l1, l2):
    """multiplicities of J in j1 (x) j2 summed over the sectors of two legs"""
    n = {}
    for t1, n1 in zip(l1.spins, l1.degs):
        for t2, n2 in zip(l2.spins, l2.degs):
            for tJ in range(abs(t1 - t2), t1 + t2 + 1, 2):
                n[tJ] = n.get(tJ, 0) + n1 * n2
    ks = sorted(n)
    return su2.Leg(l1.flow, tuple(ks), tuple(n[k] for k in ks))


def test_cfg3_leg_dimensions():
    """Virtual leg of D=10 (d=5 reduced); its double-layer fusion has total
    dimension 100 and reduced dimension 42; the env bond X=150 (chi=50)."""
    from workloads import su2_config
    cfg = su2_config("D10chi150")
    v = su2.Leg(1, *cfg["virtual"])
    assert (v.dim, v.rdim) == (10, 5)
    k = fused_spins(v, v.dual())
    assert (k.dim, k.rdim) == (100, 42)
    assert (k.spins, k.degs) == tuple(cfg["k"])
    x = su2.Leg(1, *cfg["x"])
    assert (x.dim, x.rdim) == (150, 50)


# ---------------------------------------------------------------------------
# the SU(2) LEFT move of the oracle

@pytest.fixture(scope="module")
def su2_move():
    from oracle import ctm_su2
    from workloads import su2_config
    net = ctm_su2.su2_network(su2_config("medium"), seed=1)
    out, info = ctm_su2.left_move(net, 24, return_info=True)
    return net, out, info


def test_su2_move_spectrum_is_the_dense_spectrum(su2_move):
    """The reduced sector matrices carry the dense N's singular values, each
    2J+1 times (a wrong sector assembly or basis would change them)."""
    net, out, info = su2_move
    N = info["N"]
    dims = N.shape
    dense = np.linalg.svd(N.reshape(dims[0] * dims[1], dims[2] * dims[3]), compute_uv=False)
    red = []
    for J, (U, S, Vt) in info["sectors"].items():
        red.extend(list(S) * (J + 1))
    red = np.sort(np.array(red))[::-1]
    dense = np.sort(dense)[::-1][:len(red)]
    assert np.abs(dense - red).max() < 1e-10 * dense[0]
    # the rest of the dense spectrum is zero (N is fully covered by its sectors)
    assert len(red) <= dims[0] * dims[1]


def test_su2_move_projectors_and_truncation(su2_move):
    net, out, info = su2_move
    new = info["new"]
    assert info["dim"] == new.dim <= 24
    # P~ P = 1 on the new leg (full dimension)
    PtP = np.einsum("nab,abm->nm", info["Pt"], info["P"])
    assert np.abs(PtP - np.eye(new.dim)).max() < 1e-10
    # whole multiplets only: no discarded value above a kept one of the same J
    for J, (U, S, Vt) in info["sectors"].items():
        k = info["kept"][J]
        assert all(S[j] >= S[k] for j in range(k)) if k < len(S) else True


def test_su2_move_outputs_are_invariant(su2_move):
    net, out, info = su2_move
    rng = np.random.default_rng(3)
    for r in ("C1", "T4", "C4"):
        legs, dense = out[r]
        assert abs(np.linalg.norm(dense) - 1.0) < 1e-12
        assert np.abs(su2.to_dense(legs, su2.from_dense(legs, dense)) - dense).max() < 1e-12
        R = su2.rotate(legs, dense, rng.standard_normal(3))
        assert np.abs(R - dense).max() < 1e-11
