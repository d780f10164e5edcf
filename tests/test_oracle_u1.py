"""Pins of the U(1) part of the oracle against facts fixed by the paper and
by the mathematics (selection rule, invariance, brute force, fusion)."""
import itertools

import numpy as np
import pytest

from oracle import u1
from workloads import gaussian_sectors, u1_config, values


def rand_legs(rng, rank):
    legs = []
    for _ in range(rank):
        qs = sorted(rng.choice(np.arange(-3, 4), size=int(rng.integers(1, 4)), replace=False))
        legs.append(u1.Leg(int(rng.choice([1, -1])), tuple(int(q) for q in qs),
                           tuple(int(d) for d in rng.integers(1, 4, size=len(qs)))))
    return legs


def test_sector_recipe_matches_configs():
    assert gaussian_sectors(16, 4) == ((-4, -2, 0, 2, 4), (1, 4, 6, 4, 1))
    assert gaussian_sectors(72, 6) == ((-6, -4, -2, 0, 2, 4, 6), (3, 8, 15, 20, 15, 8, 3))
    assert gaussian_sectors(256, 8) == ((-8, -6, -4, -2, 0, 2, 4, 6, 8),
                                        (7, 17, 32, 46, 52, 46, 32, 17, 7))


def poly_nnz(legs):
    """Number of allowed entries = coefficient of z^0 in prod_legs sum_q deg_q z^(flow q):
    an independent count (polynomial product) of the selection rule."""
    poly = {0: 1}
    for l in legs:
        new = {}
        for e, c in poly.items():
            for q, d in zip(l.charges, l.degs):
                new[e + l.flow * q] = new.get(e + l.flow * q, 0) + c * d
        poly = new
    return poly.get(0, 0)


def test_nnz_config_site_tensors():
    legs = [u1.leg_from_spec(s) for s in u1_config("d4chi16")["A"]]
    assert u1.nnz(legs) == 140 == poly_nnz(legs)
    legs = [u1.leg_from_spec(s) for s in u1_config("d6chi72")["A"]]
    assert u1.nnz(legs) == poly_nnz(legs)


@pytest.mark.parametrize("seed", range(6))
def test_nnz_and_mask_random_layouts(seed):
    rng = np.random.default_rng(seed)
    legs = rand_legs(rng, int(rng.integers(2, 5)))
    assert u1.nnz(legs) == poly_nnz(legs) == int(u1.allowed_mask(legs).sum())


@pytest.mark.parametrize("seed", range(4))
def test_dense_expansion_zero_outside_blocks(seed):
    rng = np.random.default_rng(seed)
    legs = rand_legs(rng, 4)
    x = rng.standard_normal(u1.nnz(legs))
    T = u1.to_dense(legs, x)
    mask = u1.allowed_mask(legs)
    assert np.all(T[~mask] == 0.0)                 # forbidden entries identically zero
    assert np.count_nonzero(T[mask]) == x.size     # every stored value placed once
    assert np.array_equal(u1.from_dense(legs, T), x)


def test_block_order_is_lexicographic():
    legs = [u1.Leg(1, (-1, 1), (1, 2)), u1.Leg(1, (-1, 1), (2, 1)), u1.Leg(-1, (-2, 0, 2), (1, 1, 1))]
    bl = u1.blocks(legs)
    assert bl == sorted(bl)
    assert bl == [(0, 0, 0), (0, 1, 1), (1, 0, 1), (1, 1, 2)]


@pytest.mark.parametrize("seed", range(4))
def test_u1_phase_invariance(seed):
    """A symmetric tensor is invariant under exp(i theta flow q) on every leg."""
    rng = np.random.default_rng(seed)
    legs = rand_legs(rng, 4)
    T = u1.to_dense(legs, rng.standard_normal(u1.nnz(legs))).astype(np.complex128)
    theta = rng.uniform(0, 2 * np.pi)
    R = T.copy()
    for ax, l in enumerate(legs):
        ph = np.exp(1j * theta * l.flow * l.charge_vector())
        shp = [1] * len(legs)
        shp[ax] = l.dim
        R = R * ph.reshape(shp)
    assert np.allclose(R, T, atol=1e-14, rtol=0)


def test_contraction_brute_force_and_symmetry():
    rng = np.random.default_rng(7)
    a_legs = [u1.Leg(1, (-1, 1), (1, 2)), u1.Leg(-1, (-2, 0, 2), (1, 2, 1)), u1.Leg(1, (-1, 1), (2, 1))]
    b_legs = [u1.Leg(1, (-2, 0, 2), (1, 2, 1)), u1.Leg(-1, (-1, 1), (1, 1)), u1.Leg(-1, (0, 2), (2, 1))]
    A = u1.to_dense(a_legs, rng.standard_normal(u1.nnz(a_legs)))
    B = u1.to_dense(b_legs, rng.standard_normal(u1.nnz(b_legs)))
    C = np.einsum("ixj,xkl->ijkl", A, B)
    ref = np.zeros_like(C)
    for i, x, j, k, l in itertools.product(*[range(n) for n in (A.shape[0], A.shape[1], A.shape[2], B.shape[1], B.shape[2])]):
        ref[i, j, k, l] += A[i, x, j] * B[x, k, l]
    assert np.allclose(C, ref, atol=1e-14)
    c_legs = [a_legs[0], a_legs[2], b_legs[1], b_legs[2]]
    assert np.all(C[~u1.allowed_mask(c_legs)] == 0.0)


def test_fuse_isometry_and_charges():
    ket = u1.Leg(1, (-1, 1), (3, 3))
    fl, F = u1.fuse([ket, ket.dual()])
    assert fl.flow == 1 and fl.charges == (-2, 0, 2) and fl.degs == (9, 18, 9)
    M = F.reshape(fl.dim, -1)
    assert np.array_equal(M @ M.T, np.eye(fl.dim))
    assert np.array_equal(M.T @ M, np.eye(M.shape[1]))
    qk = ket.charge_vector()
    for k in range(fl.dim):
        i, j = np.argwhere(F[k])[0]
        assert fl.charge_vector()[k] == qk[i] - qk[j]
    even = u1.Leg(1, (-2, 0, 2), (1, 4, 1))
    fe, _ = u1.fuse([even, even.dual()])
    assert fe.charges == (-4, -2, 0, 2, 4) and fe.degs == (1, 8, 18, 8, 1)


def _site(name, seed=0):
    cfg = u1_config(name)
    A_legs = [u1.leg_from_spec(s) for s in cfg["A"]]
    R_legs = [u1.leg_from_spec(s) for s in cfg["R"]]
    A = u1.to_dense(A_legs, values(seed, "A", u1.nnz(A_legs)))
    R = u1.to_dense(R_legs, values(seed, "R", u1.nnz(R_legs)))
    return A_legs, A, R_legs, R


def test_double_layer_psd_and_symmetric():
    A_legs, A, R_legs, R = _site("tiny")
    legs, a = u1.double_layer(A_legs, A)
    assert np.all(a[~u1.allowed_mask(legs)] == 0.0)
    # a viewed as (ket legs) x (bra legs) is sum_p A_p A_p^T: positive semi-definite
    Fs = [u1.fuse([l, l.dual()])[1] for l in A_legs[1:]]
    un = np.einsum("abce,alL,buU,crR,edD->lurdLURD", a, *Fs)
    n = int(np.prod(A.shape[1:]))
    M = un.reshape(n, n)
    assert np.allclose(M, M.T, atol=1e-13)
    assert np.linalg.eigvalsh(M).min() > -1e-12
    ref = np.einsum("plurd,pLURD->lurdLURD", A, A).reshape(n, n)
    assert np.allclose(M, ref, atol=1e-13)


def test_remover_makes_right_leg_equal_left_leg():
    A_legs, A, R_legs, R = _site("d4chi16")
    legs, a = u1.double_layer(A_legs, A, R_legs, R)
    assert legs[2].same_space(legs[0]) and legs[2].flow == -legs[0].flow
    assert legs[3].same_space(legs[1]) and legs[3].flow == -legs[1].flow
    assert np.all(a[~u1.allowed_mask(legs)] == 0.0)


@pytest.mark.parametrize("name", ["tiny", "d4chi16"])
def test_remover_branch_equals_the_eight_index_sum(name):
    """Pin of the remover branch (Sec. 3.1): unfusing the result gives, for
    every ket/bra index pair, sum_{p,s,r,r~} A[p,l,u,r,d] A[p,l~,u~,r~,d~]
    R[r,x,s] R[r~,x~,s], written out here with one einsum.  A transposed
    rho, a mispaired s or a missing sum over s changes this sum."""
    A_legs, A, R_legs, R = _site(name)
    legs, a = u1.double_layer(A_legs, A, R_legs, R)
    Fs = [u1.fuse([l, l.dual()])[1] for l in (A_legs[1], A_legs[2], R_legs[1], A_legs[4])]
    un = np.einsum("abce,alL,buU,cxX,edD->lLuUxXdD", a, *Fs, optimize=True)
    direct = np.einsum("plurd,pLUtD,rxs,tXs->lLuUxXdD", A, A, R, R, optimize=True)
    assert np.allclose(un, direct, rtol=0, atol=1e-13 * np.abs(direct).max())
    # the sum over s is not separable: the product of the two separate sums
    # differs (so a mispaired s cannot pass)
    wrong = np.einsum("plurd,pLUtD,rxs,tXz->lLuUxXdD", A, A, R, R, optimize=True)
    assert np.abs(wrong - direct).max() > 1e-3 * np.abs(direct).max()


@pytest.mark.parametrize("name", ["tiny", "d4chi16"])
def test_remover_equals_double_layer_of_the_absorbed_site(name):
    """a(A, R) = a(A') with A'[(p,s), l, u, x, d] = sum_r A[p,l,u,r,d] R[r,x,s]:
    absorbing the remover into the site first and then forming the plain
    double layer gives the same tensor (the physical and remover legs are
    summed together)."""
    A_legs, A, R_legs, R = _site(name)
    legs, a = u1.double_layer(A_legs, A, R_legs, R)
    P, FP = u1.fuse([A_legs[0], R_legs[2]])
    Ap = np.einsum("Pps,plurd,rxs->Pluxd", FP, A, R, optimize=True)
    Ap_legs = [P, A_legs[1], A_legs[2], R_legs[1], A_legs[4]]
    assert np.all(Ap[~u1.allowed_mask(Ap_legs)] == 0.0)
    legs2, a2 = u1.double_layer(Ap_legs, Ap)
    assert legs2 == legs
    assert np.allclose(a2, a, rtol=0, atol=1e-13 * np.abs(a).max())
