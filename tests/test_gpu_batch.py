"""GPU parity of the batched contraction (many independent corner
contractions Q = X2 . a over (k_u, k_l) in one launch per stage) against the
dense FP64 oracle, against the single-contraction entry point, and under CUDA
graph capture and replay."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import u1  # noqa: E402
from workloads import batched_site_legs, batched_u1_configs, values  # noqa: E402
from bst_helpers import bf16x3_bound, rel_err  # noqa: E402

LEGS_X2 = (0, 2)   # X2[k_u, x_r, k_l, x_d]: k_u, k_l
LEGS_A = (1, 0)    # a[k_l, k_u, k_r, k_d]:  k_u, k_l
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


def small_configs(count=10):
    # D in 2..5 and chi in {6, 10, 16, 24}: the oracle's dense einsum takes
    # well under a second each, sector matrices still span several tiles
    return batched_u1_configs(count, seed=7, d_range=(2, 5), chis=(6, 10, 16, 24))


def gpu_instance(bst, ctx, cfg):
    A = ctx.layout([bst.Leg(l["flow"], l["charges"], l["degs"]) for l in batched_site_legs(cfg)])
    aL, ad = ctx.double_layer(A, dev(values(cfg["seed"], "A", A.nnz)))
    kl, ku = aL.legs[0], aL.legs[1]
    X = bst.Leg(-1, tuple(cfg["x"][0]), tuple(cfg["x"][1]))
    X2L = ctx.layout([ku.dual(), X, kl.dual(), X])
    x2 = dev(values(cfg["seed"], "X2", X2L.nnz))
    return X2L, x2, aL, ad


def oracle_instance(cfg):
    A_legs = [u1.leg_from_spec(s) for s in batched_site_legs(cfg)]
    A = u1.to_dense(A_legs, values(cfg["seed"], "A", u1.nnz(A_legs)))
    a_legs, a = u1.double_layer(A_legs, A)
    X = u1.Leg(-1, tuple(cfg["x"][0]), tuple(cfg["x"][1]))
    x2_legs = [a_legs[1].dual(), X, a_legs[0].dual(), X]
    x2 = u1.to_dense(x2_legs, values(cfg["seed"], "X2", u1.nnz(x2_legs)))
    q_legs = [X, X, a_legs[2], a_legs[3]]
    return x2_legs, x2, a_legs, a, q_legs


def same_legs(bl, ol):
    return [(int(l.flow), tuple(l.charges), tuple(l.degs)) for l in bl] == \
        [(l.flow, tuple(l.charges), tuple(l.degs)) for l in ol]


def run_batch(ctx, inst, prec, **kw):
    return ctx.contract_batched([i[0] for i in inst], [i[1] for i in inst], [i[2] for i in inst],
                                [i[3] for i in inst], LEGS_X2, LEGS_A, prec=prec, **kw)


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("ozaki", TOL_MIXED)])
def test_batched_matches_oracle(bst, ctx, prec, tol):
    cfgs = small_configs()
    inst = [gpu_instance(bst, ctx, c) for c in cfgs]
    Cls, cs = run_batch(ctx, inst, prec)
    torch.cuda.synchronize()
    for cfg, L, c in zip(cfgs, Cls, cs):
        x2_legs, x2, a_legs, a, q_legs = oracle_instance(cfg)
        ref = np.einsum("uxly,luzw->xyzw", x2, a)
        # block structure bit-exact, forbidden entries exactly zero
        assert same_legs(L.legs, q_legs)
        assert L.nnz == u1.nnz(q_legs)
        assert not np.any(ref[~u1.allowed_mask(q_legs)])
        err = rel_err(c.cpu().numpy(), u1.from_dense(q_legs, ref))
        assert err <= tol, (cfg["name"], prec, err)


@pytest.mark.parametrize("prec", ["ozaki", "bf16x3"])
def test_tensor_core_batch_launches(bst, ctx, prec):
    """A repeated tensor-core batch: operands whose last contracted leg is
    their innermost leg are packed (gathered and split by one kernel), the
    others gathered by one launch and split by one; one GEMM writes every
    output block in its epilogue.  The corner workload (open innermost
    legs) takes 3 launches, a batch contracted over innermost legs 2; the
    results equal the first call's bit for bit and the oracle's."""
    cfgs = small_configs(8)
    inst = [gpu_instance(bst, ctx, c) for c in cfgs]
    Cls, cs = run_batch(ctx, inst, prec)
    torch.cuda.synchronize()
    first = [c.clone() for c in cs]
    l0 = ctx.launches
    run_batch(ctx, inst, prec, Cls=Cls, cs=cs)
    torch.cuda.synchronize()
    assert ctx.launches - l0 == 3
    for a, b in zip(cs, first):
        assert torch.equal(a, b)
    # contracted over both operands' last legs: packed
    rng = np.random.default_rng(11)
    As, as_, Bs, bs, refs = [], [], [], [], []
    for i in range(6):
        x = u1.Leg(1, (-1, 0, 1), tuple(int(v) for v in rng.integers(1, 30, 3)))
        y = u1.Leg(1, (-1, 0, 1), tuple(int(v) for v in rng.integers(1, 30, 3)))
        k = u1.Leg(-1, (-2, -1, 0, 1, 2), tuple(int(v) for v in rng.integers(1, 40, 5)))
        al, bl = [x, k], [y, k.dual()]
        A = u1.to_dense(al, rng.standard_normal(u1.nnz(al)))
        B = u1.to_dense(bl, rng.standard_normal(u1.nnz(bl)))
        AL = ctx.layout([bst.Leg(l.flow, l.charges, l.degs) for l in al])
        BL = ctx.layout([bst.Leg(l.flow, l.charges, l.degs) for l in bl])
        As.append(AL)
        Bs.append(BL)
        as_.append(dev(u1.from_dense(al, A)))
        bs.append(dev(u1.from_dense(bl, B)))
        refs.append(([x, y], np.tensordot(A, B, axes=([1], [1]))))
    Cls2, cs2 = ctx.contract_batched(As, as_, Bs, bs, [1], [1], prec=prec)
    torch.cuda.synchronize()
    l0 = ctx.launches
    ctx.contract_batched(As, as_, Bs, bs, [1], [1], prec=prec, Cls=Cls2, cs=cs2)
    torch.cuda.synchronize()
    assert ctx.launches - l0 == 2
    tol = 1e-11 if prec == "ozaki" else 1e-6
    for (cl, ref), c in zip(refs, cs2):
        assert rel_err(c.cpu().numpy(), u1.from_dense(cl, ref)) < tol


def test_batched_bf16x3_within_bound(bst, ctx):
    """The batch in the cheaper three-slice arithmetic: every element of
    every entry within the bound of its rounding (bf16x3_bound)."""
    cfgs = small_configs(6)
    inst = [gpu_instance(bst, ctx, c) for c in cfgs]
    Cls, cs = run_batch(ctx, inst, "bf16x3")
    torch.cuda.synchronize()
    for cfg, L, c in zip(cfgs, Cls, cs):
        x2_legs, x2, a_legs, a, q_legs = oracle_instance(cfg)
        ref = np.einsum("uxly,luzw->xyzw", x2, a)
        assert same_legs(L.legs, q_legs)
        nu, nx, nl, ny = x2.shape
        Am = np.transpose(x2, (1, 3, 0, 2)).reshape(nx * ny, nu * nl)
        Bm = np.transpose(a, (1, 0, 2, 3)).reshape(nu * nl, -1)
        bound = bf16x3_bound(Am, Bm)
        got = u1.to_dense(q_legs, c.cpu().numpy()).reshape(nx * ny, -1)
        assert np.all(np.abs(got - ref.reshape(nx * ny, -1)) <= bound + 1e-300), cfg["name"]


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_batched_equals_single(bst, ctx, prec):
    """Each entry of the batch is computed exactly as the single call does
    (same sector problems, same tiles, same arithmetic); a repeated layout
    pair with different data and alpha/beta accumulation are covered."""
    cfgs = small_configs()
    inst = [gpu_instance(bst, ctx, c) for c in cfgs]
    # the same layouts again with other values
    extra = []
    for X2L, x2, aL, ad in inst[:3]:
        extra.append((X2L, torch.randn_like(x2), aL, torch.randn_like(ad)))
    inst = inst + extra
    Cls = [ctx.contract_layout(i[0], i[2], LEGS_X2, LEGS_A) for i in inst]
    c0 = [torch.randn(L.nnz, dtype=torch.float64, device="cuda:0") for L in Cls]
    cb = [c.clone() for c in c0]
    run_batch(ctx, inst, prec, alpha=0.75, beta=-1.25, Cls=Cls, cs=cb)
    for (X2L, x2, aL, ad), L, c in zip(inst, Cls, c0):
        ctx.contract(X2L, x2, aL, ad, LEGS_X2, LEGS_A, prec=prec, alpha=0.75, beta=-1.25, Cl=L, c=c)
    torch.cuda.synchronize()
    for a, b in zip(cb, c0):
        if prec == "fp64":
            assert torch.equal(a, b)
        else:
            assert rel_err(a.cpu().numpy(), b.cpu().numpy()) <= 1e-15


def test_batched_single_entry_and_errors(bst, ctx):
    cfg = small_configs(1)[0]
    inst = [gpu_instance(bst, ctx, cfg)]
    Cls, cs = run_batch(ctx, inst, "fp64")
    L1, c1 = ctx.contract(inst[0][0], inst[0][1], inst[0][2], inst[0][3], LEGS_X2, LEGS_A)
    torch.cuda.synchronize()
    assert torch.equal(cs[0], c1)
    # output layout that does not belong to the contraction
    with pytest.raises(bst.BstError):
        run_batch(ctx, inst, "fp64", Cls=[inst[0][0]], cs=[torch.empty(inst[0][0].nnz, dtype=torch.float64,
                                                                       device="cuda:0")])
    # contracted legs that do not match (k_u with k_r)
    with pytest.raises(bst.BstError):
        ctx.contract_batched([inst[0][0]], [inst[0][1]], [inst[0][2]], [inst[0][3]], LEGS_X2, (2, 0))


def test_batched_graph_replay(bst, ctx):
    """After one eager call (plan, buffers and pointer table cached) the
    batch is captured into a CUDA graph; replays with new values in the same
    input buffers give what an eager call gives."""
    cfgs = small_configs(6)
    inst = [gpu_instance(bst, ctx, c) for c in cfgs]
    for prec in ("fp64", "ozaki"):
        Cls, cs = run_batch(ctx, inst, prec)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            run_batch(ctx, inst, prec, Cls=Cls, cs=cs)
        for it in range(3):
            for X2L, x2, aL, ad in inst:
                x2.normal_()
                ad.normal_()
            g.replay()
            torch.cuda.synchronize()
            got = [c.clone() for c in cs]
            _, ref = run_batch(ctx, inst, prec, Cls=Cls)
            torch.cuda.synchronize()
            for a, b in zip(got, ref):
                assert torch.equal(a, b), (prec, it)


@pytest.fixture(scope="module")
def full_batch(bst, ctx):
    cfgs = batched_u1_configs(64)
    inst = [gpu_instance(bst, ctx, c) for c in cfgs]
    Cls, c64 = run_batch(ctx, inst, "fp64")
    _, cmx = run_batch(ctx, inst, "ozaki", Cls=Cls)
    torch.cuda.synchronize()
    return cfgs, inst, Cls, c64, cmx


def test_full_batch_mixed_vs_fp64(full_batch):
    """All 64 contractions of the D ~ U{4..8}, chi ~ U{32..128} batch: the
    mixed-precision path against the FP64 path, per contraction."""
    cfgs, inst, Cls, c64, cmx = full_batch
    errs = [rel_err(a.cpu().numpy(), b.cpu().numpy()) for a, b in zip(cmx, c64)]
    assert max(errs) <= 1e-10, max(errs)


@pytest.mark.parametrize("pick", ["largest", "smallest", "median"])
def test_full_batch_sampled_oracle(full_batch, pick):
    """Sampled output entries of full-size contractions, each computed by the
    oracle as its own dense sum over (k_u, k_l)."""
    cfgs, inst, Cls, c64, cmx = full_batch
    order = np.argsort([L.nnz for L in Cls])
    i = int({"largest": order[-1], "smallest": order[0], "median": order[len(order) // 2]}[pick])
    x2_legs, x2, a_legs, a, q_legs = oracle_instance(cfgs[i])
    assert same_legs(Cls[i].legs, q_legs)
    # dense position of every stored entry
    pos = u1.from_dense(q_legs, np.arange(np.prod(u1.dense_shape(q_legs)), dtype=np.int64)
                        .reshape(u1.dense_shape(q_legs))).astype(np.int64)
    rng = np.random.default_rng(i)
    sel = rng.choice(len(pos), size=min(4096, len(pos)), replace=False)
    xs, ys, zs, ws = np.unravel_index(pos[sel], u1.dense_shape(q_legs))
    ref = np.einsum("sul,lus->s", x2[:, xs, :, ys], a[:, :, zs, ws])
    for c, tol in ((c64[i], TOL64), (cmx[i], TOL_MIXED)):
        got = c.cpu().numpy()[sel]
        scale = np.linalg.norm(ref)
        assert np.linalg.norm(got - ref) <= tol * scale, (pick, np.linalg.norm(got - ref) / scale)


def test_autotune_changes_no_bit(bst, ctx):
    """The tuned schedule (chunk size, tile order) gives the same bits as the
    untuned default schedule, and every decision is logged."""
    cfgs = small_configs(8)
    inst = [gpu_instance(bst, ctx, c) for c in cfgs]
    plain = bst.Context(0)
    try:
        plain.set_autotune(False)
        inst2 = [gpu_instance(bst, plain, c) for c in cfgs]
        for prec in ("fp64", "ozaki"):
            _, tuned = run_batch(ctx, inst, prec)
            _, untuned = run_batch(plain, inst2, prec)
            torch.cuda.synchronize()
            for a, b in zip(tuned, untuned):
                assert torch.equal(a, b), prec
        assert plain.tuning_log() == ""
    finally:
        plain.close()
    log = ctx.tuning_log()
    assert "relayout chunk chosen" in log
    assert "gemm_f64 tile order chosen" in log and "gemm_ozaki tile order chosen" in log
