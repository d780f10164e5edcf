"""GPU parity of the SU(2) contraction (reduced blocks, X-symbol recoupling)
against the dense FP64 oracle: random structures of every flow pattern, the
enlarged-corner chain C1.T1 -> X1, X1.T4 -> X2, X2.a -> Q1 of the SU(2)
workload, and sampled output sectors of the full-size (D=10, X=150) corner."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import su2  # noqa: E402
from workloads import su2_config, values  # noqa: E402
from bst_helpers import rel_err  # noqa: E402

TOL64 = 1e-12
TOL_MIXED = 1e-11


@pytest.fixture(scope="module")
def bst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_10804_gb300 import build
    build.build()
    from paper_1808_10804_gb300 import bst as b
    return b


@pytest.fixture(scope="module")
def ctx(bst):
    c = bst.Context(0)
    yield c
    c.close()


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda:0")


def bst_legs(bst, legs):
    return [bst.Leg(l.flow, tuple(l.spins), tuple(l.degs)) for l in legs]


def rand_legs(rng, flows, maxspin=4, maxdeg=3):
    while True:
        legs = []
        for f in flows:
            ns = int(rng.integers(1, 4))
            sp = tuple(sorted(rng.choice(np.arange(0, maxspin + 1), size=ns, replace=False).tolist()))
            legs.append(su2.Leg(f, sp, tuple(int(x) for x in rng.integers(1, maxdeg + 1, size=ns))))
        if su2.nnz(legs) > 0:
            return legs


CASES = [
    # (A flows, contracted A legs, B extra flows); B's contracted legs are the duals
    ((1, -1), (1,), (-1,)),                 # matrix product
    ((1, 1, -1), (2,), (-1, -1)),
    ((-1, -1, -1), (0, 2), (1, -1)),
    ((1, 1, -1, -1), (2, 3), (-1, -1)),
    ((1, -1, 1, -1), (1, 3), (1, -1)),
    ((-1, -1, -1, -1), (0, 2), (-1, -1)),   # the corner pattern: all-out with a 2-in-2-out partner
    ((1, -1, -1), (), (1, -1)),              # outer product
    ((1, 1, 1, -1), (0, 3), (1, 1)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("ozaki", TOL_MIXED)])
def test_su2_contract_matches_oracle(bst, ctx, case, seed, prec, tol):
    fa, la, fb_extra = CASES[case]
    rng = np.random.default_rng(300 + 17 * case + seed)
    while True:
        A = rand_legs(rng, fa)
        B = [A[i].dual() for i in la] + rand_legs(rng, fb_extra)
        if su2.nnz(B) > 0:
            break
    lb = tuple(range(len(la)))
    a = rng.standard_normal(su2.nnz(A))
    b = rng.standard_normal(su2.nnz(B))
    legsC, cref, _ = su2.contract(A, a, B, b, la, lb)
    LA = ctx.layout(bst_legs(bst, A), group="su2")
    LB = ctx.layout(bst_legs(bst, B), group="su2")
    LC, c = ctx.contract(LA, dev(a), LB, dev(b), la, lb, prec=prec)
    torch.cuda.synchronize()
    assert [(l.flow, tuple(l.charges), tuple(l.degs)) for l in LC.legs] == \
        [(l.flow, l.spins, l.degs) for l in legsC]
    assert LC.nnz == cref.size
    if cref.size:
        assert rel_err(c.cpu().numpy(), cref) <= tol


def test_su2_alpha_beta(bst, ctx):
    rng = np.random.default_rng(5)
    A = rand_legs(rng, (1, 1, -1, -1))
    B = [A[2].dual(), A[3].dual()] + rand_legs(rng, (-1, 1))
    a = rng.standard_normal(su2.nnz(A))
    b = rng.standard_normal(su2.nnz(B))
    legsC, cref, _ = su2.contract(A, a, B, b, (2, 3), (0, 1))
    LA = ctx.layout(bst_legs(bst, A), group="su2")
    LB = ctx.layout(bst_legs(bst, B), group="su2")
    LC = ctx.contract_layout(LA, LB, (2, 3), (0, 1))
    c0 = rng.standard_normal(LC.nnz)
    c = dev(c0)
    ctx.contract(LA, dev(a), LB, dev(b), (2, 3), (0, 1), alpha=-0.5, beta=2.0, Cl=LC, c=c)
    torch.cuda.synchronize()
    assert rel_err(c.cpu().numpy(), -0.5 * cref + 2.0 * c0) <= TOL64


def env_legs(cfg):
    k = su2.Leg(1, *cfg["k"])
    x = su2.Leg(1, *cfg["x"])
    return {"C1": [x.dual(), x.dual()], "T1": [x, k.dual(), x.dual()], "T4": [x, k.dual(), x.dual()],
            "a": [k, k, k.dual(), k.dual()]}


def corner_inputs(cfg, seed=0):
    legs = env_legs(cfg)
    data = {n: values(seed, t, su2.nnz(legs[n])) for n, t in (("C1", "C1"), ("T1", "T1"), ("T4", "T4"),
                                                               ("a", "A"))}
    return legs, data


def gpu_corner(bst, ctx, legs, data, prec):
    L = {n: ctx.layout(bst_legs(bst, l), group="su2") for n, l in legs.items()}
    d = {n: dev(v) for n, v in data.items()}
    LX1, x1 = ctx.contract(L["C1"], d["C1"], L["T1"], d["T1"], (0,), (0,), prec=prec)
    LX2, x2 = ctx.contract(LX1, x1, L["T4"], d["T4"], (0,), (0,), prec=prec)
    LQ, q = ctx.contract(LX2, x2, L["a"], d["a"], (0, 2), (1, 0), prec=prec)
    torch.cuda.synchronize()
    return (LX1, x1), (LX2, x2), (LQ, q)


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("ozaki", TOL_MIXED)])
def test_su2_corner_chain_small(bst, ctx, prec, tol):
    """C1.T1 -> X1, X1.T4 -> X2, X2.a -> Q1 on a small SU(2) structure,
    every intermediate against the oracle."""
    legs, data = corner_inputs(su2_config("small"), seed=3)
    (LX1, x1), (LX2, x2), (LQ, q) = gpu_corner(bst, ctx, legs, data, prec)
    l1, r1, _ = su2.contract(legs["C1"], data["C1"], legs["T1"], data["T1"], (0,), (0,))
    l2, r2, _ = su2.contract(l1, r1, legs["T4"], data["T4"], (0,), (0,))
    l3, r3, _ = su2.contract(l2, r2, legs["a"], data["a"], (0, 2), (1, 0))
    for got, ref in ((x1, r1), (x2, r2), (q, r3)):
        assert got.numel() == ref.size
        assert rel_err(got.cpu().numpy(), ref) <= tol


def dense_slice(legs, flat, fixed):
    """Dense expansion restricted to one sector on each leg in `fixed`
    ({leg: sector index}); other legs stay full."""
    offs = [l.sector_offsets() for l in legs]
    shape = []
    for k, l in enumerate(legs):
        if k in fixed:
            s = fixed[k]
            shape.append(l.degs[s] * (l.spins[s] + 1))
        else:
            shape.append(l.dim)
    out = np.zeros(shape)
    pos = 0
    R = len(legs)
    for idx, tree in su2.blocks(legs):
        shp = su2.block_shape(legs, idx)
        n = int(np.prod(shp))
        if all(idx[k] == s for k, s in fixed.items()):
            red = np.asarray(flat[pos:pos + n]).reshape(shp)
            c = su2.basis(legs, idx, tree)
            t = np.multiply.outer(red, c)
            t = np.transpose(t, [a for k in range(R) for a in (k, R + k)])
            t = t.reshape([shp[k] * c.shape[k] for k in range(R)])
            sl = tuple(slice(0, t.shape[k]) if k in fixed else slice(offs[k][idx[k]], offs[k][idx[k]] + t.shape[k])
                       for k in range(R))
            out[sl] += t
        pos += n
    return out


@pytest.fixture(scope="module")
def full_corner(bst, ctx):
    cfg = su2_config("D10chi150")
    legs, data = corner_inputs(cfg, seed=0)
    r64 = gpu_corner(bst, ctx, legs, data, "fp64")
    rmx = gpu_corner(bst, ctx, legs, data, "ozaki")
    return cfg, legs, data, r64, rmx


def test_su2_full_corner_mixed_vs_fp64(full_corner):
    cfg, legs, data, r64, rmx = full_corner
    for (L64, x64), (Lmx, xmx) in zip(r64, rmx):
        assert L64 == Lmx
        assert rel_err(xmx.cpu().numpy(), x64.cpu().numpy()) <= 1e-10


@pytest.mark.parametrize("pick", range(3))
def test_su2_full_corner_sampled_oracle(full_corner, pick):
    """Output sector tuples of the full-size Q1 = X2 . a, each recomputed by
    the oracle from dense slices of X2 and a, projected on the output's
    CGC tensors."""
    cfg, legs, data, r64, rmx = full_corner
    (LX1, x1), (LX2, x2), (LQ, q) = r64
    k = su2.Leg(1, *cfg["k"])
    x = su2.Leg(1, *cfg["x"])
    X2legs = [k.dual(), x.dual(), k.dual(), x.dual()]
    Qlegs = [x.dual(), x.dual(), k.dual(), k.dual()]
    assert [(l.flow, tuple(l.charges), tuple(l.degs)) for l in LX2.legs] == [(l.flow, l.spins, l.degs) for l in X2legs]
    assert [(l.flow, tuple(l.charges), tuple(l.degs)) for l in LQ.legs] == [(l.flow, l.spins, l.degs) for l in Qlegs]
    x2 = x2.cpu().numpy()
    qv = {"fp64": r64[2][1].cpu().numpy(), "ozaki": rmx[2][1].cpu().numpy()}
    # sampled output sector tuples among those with small env sectors
    tuples = sorted({idx for idx, _ in su2.blocks(Qlegs)
                     if all(Qlegs[i].degs[idx[i]] * (Qlegs[i].spins[idx[i]] + 1) <= 14 for i in (0, 1))})
    rng = np.random.default_rng(11)
    sel = tuples[int(rng.integers(0, len(tuples)))] if pick else tuples[-1]
    if pick == 2:
        sel = tuples[len(tuples) // 2]
    xs, ys, kr, kd = sel
    X2d = dense_slice(X2legs, x2, {1: xs, 3: ys})
    ad = dense_slice(legs["a"], data["a"], {2: kr, 3: kd})
    U, Xn, L_, Yn = X2d.shape
    Zn, Wn = ad.shape[2], ad.shape[3]
    lhs = np.transpose(X2d, (1, 3, 0, 2)).reshape(Xn * Yn, U * L_)          # [(x,y), (u,l)]
    rhs = np.transpose(ad, (1, 0, 2, 3)).reshape(U * L_, Zn * Wn)           # [(u,l), (z,w)]
    Cd = (lhs @ rhs).reshape(Xn, Yn, Zn, Wn)
    pos = 0
    checked = 0
    for idx, tree in su2.blocks(Qlegs):
        shp = su2.block_shape(Qlegs, idx)
        n = int(np.prod(shp))
        if idx == sel:
            c = su2.basis(Qlegs, idx, tree)
            sub = Cd.reshape([v for kk in range(4) for v in (shp[kk], c.shape[kk])])
            red = np.tensordot(sub, c, axes=([1, 3, 5, 7], [0, 1, 2, 3])) / np.sum(c * c)
            for name, tol in (("fp64", TOL64), ("ozaki", TOL_MIXED)):
                got = qv[name][pos:pos + n].reshape(shp)
                assert np.linalg.norm(got - red) <= tol * max(np.linalg.norm(red), 1e-300), (name, idx, tree)
            checked += 1
        pos += n
    assert checked >= 1


@pytest.mark.parametrize("flows", [(1, -1, -1), (1, 1, -1, -1), (-1, 1, -1, 1), (1, 1, 1, -1, -1), (-1, -1, -1, 1)])
@pytest.mark.parametrize("seed", range(3))
def test_su2_permute_matches_oracle(bst, ctx, flows, seed):
    """Leg permutation with tree recoupling: the dense tensor of the result
    is the dense tensor of the input with its axes permuted."""
    rng = np.random.default_rng(900 + 31 * seed + len(flows))
    legs = rand_legs(rng, flows, maxspin=3)
    x = rng.standard_normal(su2.nnz(legs))
    perm = [int(i) for i in rng.permutation(len(legs))]
    L = ctx.layout(bst_legs(bst, legs), group="su2")
    DL, out = ctx.permute(L, dev(x), perm)
    ctx.sync()
    dlegs = [legs[p] for p in perm]
    assert [(l.flow, tuple(l.charges), tuple(l.degs)) for l in DL.legs] == \
        [(l.flow, tuple(l.spins), tuple(l.degs)) for l in dlegs]
    want = su2.from_dense(dlegs, np.transpose(su2.to_dense(legs, x), perm))
    assert rel_err(out.cpu().numpy(), want) < 1e-13
