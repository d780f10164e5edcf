"""Pins of the Z2 part of the oracle (charges are parities, the paper's third
symmetry, Sec. 4.1): the selection rule against an independent count, parity
invariance, fusion, and the 2D Ising model in the Z2 basis against
Onsager's closed form."""
import itertools

import numpy as np
import pytest

from oracle import ctm, u1

from test_oracle_ctm import onsager_kappa


def zleg(flow, d0, d1):
    return u1.Leg(flow, (0, 1), (d0, d1), 2)


def rand_z2_legs(rng, rank):
    legs = []
    for _ in range(rank):
        if rng.random() < 0.25:
            q = int(rng.integers(0, 2))
            legs.append(u1.Leg(int(rng.choice([1, -1])), (q,), (int(rng.integers(1, 4)),), 2))
        else:
            legs.append(zleg(int(rng.choice([1, -1])), int(rng.integers(1, 4)), int(rng.integers(1, 4))))
    return legs


def even_count(legs):
    """Allowed entries = the even part of prod_legs (d_0 + d_1 z) at z = 1,
    i.e. (P(1) + P(-1)) / 2: a count independent of any enumeration."""
    p1 = pm1 = 1
    for l in legs:
        d = dict(zip(l.charges, l.degs))
        p1 *= d.get(0, 0) + d.get(1, 0)
        pm1 *= d.get(0, 0) - d.get(1, 0)
    return (p1 + pm1) // 2


@pytest.mark.parametrize("seed", range(6))
def test_z2_nnz_mask_and_blocks(seed):
    rng = np.random.default_rng(seed)
    legs = rand_z2_legs(rng, int(rng.integers(2, 6)))
    assert u1.nnz(legs) == even_count(legs) == int(u1.allowed_mask(legs).sum())
    for b in u1.blocks(legs):
        assert sum(l.charges[i] for l, i in zip(legs, b)) % 2 == 0


@pytest.mark.parametrize("seed", range(4))
def test_z2_parity_invariance(seed):
    """A Z2-symmetric tensor is unchanged by the sign (-1)^q on every leg,
    and a tensor with one forbidden entry planted is not."""
    rng = np.random.default_rng(seed)
    legs = rand_z2_legs(rng, 4)
    T = u1.to_dense(legs, rng.standard_normal(u1.nnz(legs)))
    R = T.copy()
    for ax, l in enumerate(legs):
        shp = [1] * len(legs)
        shp[ax] = l.dim
        R = R * ((-1.0) ** l.charge_vector()).reshape(shp)
    assert np.array_equal(R, T)
    bad = np.argwhere(~u1.allowed_mask(legs))
    if len(bad):
        T2 = T.copy()
        T2[tuple(bad[0])] = 1.0
        R2 = T2.copy()
        for ax, l in enumerate(legs):
            shp = [1] * len(legs)
            shp[ax] = l.dim
            R2 = R2 * ((-1.0) ** l.charge_vector()).reshape(shp)
        assert not np.array_equal(R2, T2)


def test_z2_fuse_parity():
    a, b = zleg(1, 2, 3), zleg(-1, 1, 2)
    fl, F = u1.fuse([a, b])
    assert fl.mod == 2 and fl.charges == (0, 1)
    assert fl.degs == (2 * 1 + 3 * 2, 2 * 2 + 3 * 1)
    M = F.reshape(fl.dim, -1)
    assert np.array_equal(M @ M.T, np.eye(fl.dim))
    qa, qb = a.charge_vector(), b.charge_vector()
    for k in range(fl.dim):
        i, j = np.argwhere(F[k])[0]
        assert fl.charge_vector()[k] == (qa[i] - qb[j]) % 2


def ising_z2_network(beta, x=1):
    """2D Ising site in the Z2 basis: the bond weight exp(beta s s') has
    eigenvectors (1, 1)/sqrt2 (even) and (1, -1)/sqrt2 (odd); with
    M = sqrt of the weight, a = sum_s M M M M rotated into that basis
    carries parities that add up to an even number.  Environment: one even
    sector of dimension x, all ones."""
    B = np.array([[np.exp(beta), np.exp(-beta)], [np.exp(-beta), np.exp(beta)]])
    w, v = np.linalg.eigh(B)
    M = v @ np.diag(np.sqrt(w)) @ v.T
    H = np.array([[1.0, 1.0], [1.0, -1.0]]) / np.sqrt(2.0)   # column 0 even, 1 odd
    a = np.einsum("sl,su,sr,sd->lurd", M @ H, M @ H, M @ H, M @ H)
    a_legs = [zleg(1, 1, 1), zleg(1, 1, 1), zleg(-1, 1, 1), zleg(-1, 1, 1)]
    return a_legs, a


def test_z2_ising_site_is_symmetric():
    a_legs, a = ising_z2_network(0.4)
    assert np.abs(a[~u1.allowed_mask(a_legs)]).max() < 1e-15


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
@pytest.mark.parametrize("beta", [0.3, 0.6])
def test_z2_ising_free_energy_onsager(beta):
    """CTMRG in the Z2 basis (blocks by parity) converges to Onsager's free
    energy per site."""
    a_legs, a = ising_z2_network(beta)
    a = np.where(u1.allowed_mask(a_legs), a, 0.0)
    net = {r: (lg, u1.to_dense(lg, np.ones(u1.nnz(lg))))
           for r, lg in ctm.env_legs((0,), (1,), a_legs).items()}
    net["a"] = (a_legs, a)
    for _ in range(60):
        net = ctm.full_move(net, 8)
    assert abs(ctm.kappa(net) / onsager_kappa(beta) - 1) < 1e-10
