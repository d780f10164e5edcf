"""GPU parity: every call of the C ABI against the dense FP64 oracle on the
same seeded inputs.  Block structure must match bit-exactly; values within
1e-12 relative (Frobenius) for the FP64 path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ctm as octm  # noqa: E402
from oracle import u1  # noqa: E402
from workloads import u1_config, values  # noqa: E402
from bst_helpers import bf16x3_bound, check_blocks, gpu_network, matched_pair_flops, rel_err, to_bst_leg, to_oracle_leg  # noqa: E402

TOL64 = 1e-12


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


def rand_legs(rng, rank, maxdeg):
    legs = []
    for _ in range(rank):
        qs = sorted(rng.choice(np.arange(-3, 4), size=int(rng.integers(1, 4)), replace=False))
        legs.append(u1.Leg(int(rng.choice([1, -1])), tuple(int(q) for q in qs),
                           tuple(int(d) for d in rng.integers(1, maxdeg + 1, size=len(qs)))))
    return legs


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda:0")


def upload(bst, ctx, legs, dense):
    L = ctx.layout([to_bst_leg(bst, l) for l in legs])
    return L, dev(u1.from_dense(legs, dense))


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("maxdeg", [3, 40])
def test_contract_matches_oracle(bst, ctx, seed, maxdeg):
    """Random layouts; large degeneracies make sector GEMMs span several 64x64
    tiles with ragged edges."""
    rng = np.random.default_rng(100 + seed)
    shared = rand_legs(rng, 2 if maxdeg > 3 else 2, maxdeg)
    ao = rand_legs(rng, 1 if maxdeg > 3 else 2, maxdeg)
    bo = rand_legs(rng, 1 if maxdeg > 3 else 2, maxdeg)
    a_legs = [ao[0], shared[0]] + ao[1:] + [shared[1]]
    b_legs = [shared[1].dual()] + bo + [shared[0].dual()]
    A = u1.to_dense(a_legs, rng.standard_normal(u1.nnz(a_legs)))
    B = u1.to_dense(b_legs, rng.standard_normal(u1.nnz(b_legs)))
    la = [1, len(a_legs) - 1]
    lb = [len(b_legs) - 1, 0]
    ref = np.tensordot(A, B, axes=(la, lb))
    AL, ad = upload(bst, ctx, a_legs, A)
    BL, bd = upload(bst, ctx, b_legs, B)
    CL, cd = ctx.contract(AL, ad, BL, bd, la, lb)
    c_legs = [l for i, l in enumerate(a_legs) if i not in la] + [l for i, l in enumerate(b_legs) if i not in lb]
    assert [to_oracle_leg(l) for l in CL.legs] == c_legs
    got = cd.cpu().numpy()
    want = u1.from_dense(c_legs, ref)
    assert got.shape == want.shape
    assert rel_err(got, want) < 1e-13
    # alpha/beta accumulation
    c2 = cd.clone()
    ctx.contract(AL, ad, BL, bd, la, lb, alpha=2.0, beta=-0.5, Cl=CL, c=c2)
    assert rel_err(c2.cpu().numpy(), 1.5 * want) < 1e-13


TOL_OZ = 1e-11


@pytest.mark.parametrize("n", [1, 2, 7, 64, 133, 160])
@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_sym_eig_matches_lapack(bst, ctx, n, prec):
    """Small dense eigensolver of the projector against LAPACK, with a
    spectrum spread over ten decades (as in the projector's Gram matrices)."""
    rng = np.random.default_rng(n)
    batch = 3
    Hs, ws = [], []
    for _ in range(batch):
        Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
        w = np.sort(10.0 ** rng.uniform(-10, 0, size=n))[::-1]
        Hs.append((Qm * w) @ Qm.T)
        ws.append(w)
    H = np.stack(Hs)
    X, lam = ctx.sym_eig(dev(H), prec)
    X, lam = X.cpu().numpy(), lam.cpu().numpy()
    for i in range(batch):
        w_ref, V_ref = np.linalg.eigh(H[i])
        w_ref, V_ref = w_ref[::-1], V_ref[:, ::-1]
        # values below 1e-6 of the largest form one unresolved cluster (FP32
        # level); the values above 1e-4 of the largest (the ones a projector
        # keeps) are at rounding level (the mixed path carries ~44-bit
        # products: a looser bound)
        tol_all, tol_top = (1e-9, 1e-14) if prec == "fp64" else (1e-9, 1e-12)
        assert np.abs(lam[i] - w_ref).max() < tol_all * w_ref[0]
        top = w_ref >= 1e-4 * w_ref[0]
        assert np.abs(lam[i] - w_ref)[top].max() < tol_top * w_ref[0]
        # their eigenvectors up to sign, where the gap makes them well defined
        for j in np.nonzero(top)[0]:
            gap = min([abs(w_ref[j] - w_ref[k]) for k in range(n) if k != j] + [np.inf]) / w_ref[0]
            if gap < 1e-8:
                continue
            err = min(np.linalg.norm(X[i][:, j] - V_ref[:, j]), np.linalg.norm(X[i][:, j] + V_ref[:, j]))
            assert err < (1e-13 + 1e-15 / gap) * (1 if prec == "fp64" else 100), (j, err, gap)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("maxdeg", [3, 40, 90])
def test_contract_ozaki_matches_oracle(bst, ctx, seed, maxdeg):
    """Tensor-core path: sector GEMMs with M, N across several 128x64 tiles,
    K across several 32-wide chunks, ragged edges everywhere."""
    rng = np.random.default_rng(300 + seed)
    shared = rand_legs(rng, 2, maxdeg)
    ao = rand_legs(rng, 1, maxdeg)
    bo = rand_legs(rng, 1, maxdeg)
    a_legs = [ao[0], shared[0], shared[1]]
    b_legs = [shared[1].dual(), bo[0], shared[0].dual()]
    A = u1.to_dense(a_legs, rng.standard_normal(u1.nnz(a_legs)))
    B = u1.to_dense(b_legs, rng.standard_normal(u1.nnz(b_legs)))
    la, lb = [1, 2], [2, 0]
    ref = np.tensordot(A, B, axes=(la, lb))
    AL, ad = upload(bst, ctx, a_legs, A)
    BL, bd = upload(bst, ctx, b_legs, B)
    CL, cd = ctx.contract(AL, ad, BL, bd, la, lb, prec="ozaki")
    ctx.sync()
    c_legs = [a_legs[0], b_legs[1]]
    want = u1.from_dense(c_legs, ref)
    assert rel_err(cd.cpu().numpy(), want) < TOL_OZ
    # alpha/beta through the GEMM epilogue's block scatter
    c2 = cd.clone()
    ctx.contract(AL, ad, BL, bd, la, lb, prec="ozaki", alpha=2.0, beta=-0.5, Cl=CL, c=c2)
    ctx.sync()
    assert rel_err(c2.cpu().numpy(), 1.5 * want) < TOL_OZ
    # wide dynamic range inside rows: the per-row scale keeps relative accuracy
    A2 = A * np.exp(rng.uniform(-20, 20, size=A.shape[0]))[:, None, None]
    ref2 = np.tensordot(A2, B, axes=(la, lb))
    AL2, ad2 = upload(bst, ctx, a_legs, A2)
    _, cd2 = ctx.contract(AL2, ad2, BL, bd, la, lb, prec="ozaki")
    ctx.sync()
    got = cd2.cpu().numpy()
    want2 = u1.from_dense(c_legs, ref2)
    # compare row by row (rows of C follow rows of A)
    assert rel_err(got, want2) < TOL_OZ


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("maxdeg", [3, 40, 90])
def test_contract_bf16x3_within_bound(bst, ctx, seed, maxdeg):
    """The cheaper three-slice arithmetic: every element within the bound
    of its rounding (bf16x3_bound), through the plain and the alpha/beta
    epilogue, with both output tile widths in play (narrow sectors take
    128 x 32 tiles); the error is above FP64 level, so the three-slice
    kernel is the one that ran."""
    rng = np.random.default_rng(700 + seed)
    shared = rand_legs(rng, 2, maxdeg)
    ao = rand_legs(rng, 1, maxdeg)
    bo = rand_legs(rng, 1, maxdeg)
    a_legs = [ao[0], shared[0], shared[1]]
    b_legs = [shared[1].dual(), bo[0], shared[0].dual()]
    A = u1.to_dense(a_legs, rng.standard_normal(u1.nnz(a_legs)))
    B = u1.to_dense(b_legs, rng.standard_normal(u1.nnz(b_legs)))
    la, lb = [1, 2], [2, 0]
    ref = np.tensordot(A, B, axes=(la, lb))
    Am = A.reshape(A.shape[0], -1)
    Bm = np.transpose(B, (2, 0, 1)).reshape(-1, B.shape[1])
    bound = bf16x3_bound(Am, Bm)
    AL, ad = upload(bst, ctx, a_legs, A)
    BL, bd = upload(bst, ctx, b_legs, B)
    CL, cd = ctx.contract(AL, ad, BL, bd, la, lb, prec="bf16x3")
    ctx.sync()
    c_legs = [a_legs[0], b_legs[1]]
    got = u1.to_dense(c_legs, cd.cpu().numpy())
    assert np.all(np.abs(got - ref) <= bound + 1e-300)
    if np.abs(ref).max() > 0 and Am.shape[1] > 8:
        assert rel_err(got, ref) > 1e-13
    c2 = cd.clone()
    ctx.contract(AL, ad, BL, bd, la, lb, prec="bf16x3", alpha=2.0, beta=-0.5, Cl=CL, c=c2)
    ctx.sync()
    got2 = u1.to_dense(c_legs, c2.cpu().numpy())
    assert np.all(np.abs(got2 - (2.0 * ref - 0.5 * got)) <= 2.0 * bound + 1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("seed", range(4))
def test_permute_and_fuse_match_oracle(bst, ctx, seed):
    rng = np.random.default_rng(200 + seed)
    legs = rand_legs(rng, 4, 4)
    T = u1.to_dense(legs, rng.standard_normal(u1.nnz(legs)))
    L, d = upload(bst, ctx, legs, T)
    perm = [int(x) for x in rng.permutation(4)]
    PL, pd = ctx.permute(L, d, perm)
    plegs = [legs[p] for p in perm]
    assert [to_oracle_leg(l) for l in PL.legs] == plegs
    assert np.array_equal(pd.cpu().numpy(), u1.from_dense(plegs, np.transpose(T, perm)))
    FL, fd = ctx.fuse(L, d, [2, 1, 1])
    fl, F = u1.fuse(legs[:2])
    flegs = [fl, legs[2], legs[3]]
    assert [to_oracle_leg(l) for l in FL.legs] == flegs
    ref = np.einsum("kab,abcd->kcd", F, T)
    assert np.array_equal(fd.cpu().numpy(), u1.from_dense(flegs, ref))


@pytest.mark.parametrize("name", ["tiny", "d4chi16", "d6chi72"])
def test_double_layer_with_remover(bst, ctx, name):
    cfg = u1_config(name)
    A_legs = [u1.leg_from_spec(s) for s in cfg["A"]]
    R_legs = [u1.leg_from_spec(s) for s in cfg["R"]]
    A = u1.to_dense(A_legs, values(0, "A", u1.nnz(A_legs)))
    R = u1.to_dense(R_legs, values(0, "R", u1.nnz(R_legs)))
    legs, a = u1.double_layer(A_legs, A, R_legs, R)
    AL = ctx.layout(cfg["A"])
    RL = ctx.layout(cfg["R"])
    aL, ad = ctx.double_layer(AL, dev(values(0, "A", AL.nnz)), RL, dev(values(0, "R", RL.nnz)))
    assert [to_oracle_leg(l) for l in aL.legs] == legs
    assert rel_err(ad.cpu().numpy(), u1.from_dense(legs, a)) < 1e-14


def oracle_net(name, seed=0):
    return octm.u1_network(u1_config(name), seed)


def test_svd_projector_matches_oracle(bst, ctx):
    net = oracle_net("d4chi16")
    L = {r: net[r][0] for r in octm.ROLES}
    q = octm.quarters(net)
    out, info = octm.left_move(net, 16, return_info=True)
    rt_legs = [L["T4"][2], L["a"][3], L["T2"][2], L["a"][3]]
    rb_legs = [L["T4"][0], L["a"][1], L["T2"][0], L["a"][1]]
    RtL, rt = upload(bst, ctx, rt_legs, q["Rt"])
    RbL, rb = upload(bst, ctx, rb_legs, q["Rb"])
    P, p, Pt, pt, sv, kept = ctx.svd_projector(RtL, rt, RbL, rb, 2, 16, 1e-14, -1)
    assert kept == info["kept"]
    nl = info["new_leg"]
    assert to_oracle_leg(P.legs[2]) == nl
    assert np.allclose(sv, info["svals"], rtol=1e-12, atol=0)
    p_legs = [L["T4"][0], L["a"][1], nl]
    pt_legs = [nl.dual(), L["T4"][2], L["a"][3]]
    na = L["T4"][2].dim * L["a"][3].dim
    P_ref = info["P"].reshape(L["T4"][0].dim, L["a"][1].dim, -1)
    Pt_ref = info["Pt"].reshape(-1, L["T4"][2].dim, L["a"][3].dim)
    assert rel_err(p.cpu().numpy(), u1.from_dense(p_legs, P_ref)) < TOL64
    assert rel_err(pt.cpu().numpy(), u1.from_dense(pt_legs, Pt_ref)) < TOL64
    assert na * 16 >= Pt.nnz


def gpu_env(bst, ctx, name, chi_cap):
    cfg = u1_config(name)
    aL, ad, Ls, data = gpu_network(bst, ctx, cfg)
    caps = {}
    for r, Lr in Ls.items():
        dims = [l.dim for l in Lr.legs]
        # renewed tensors keep their site leg and get chi-sized env legs
        caps[r] = int(np.prod([d if i == 1 and r.startswith("T") else chi_cap for i, d in enumerate(dims)]))
        caps[r] = max(caps[r], Lr.nnz)
    return cfg, aL, ad, bst.Env(ctx, Ls, data, caps)


# per-block bound: a block's error against its own norm (floored at 1e-3 of
# the tensor norm) within OWN_FACTOR times the tensor tolerance
OWN_FACTOR = 100.0


def compare_env(env, net, roles, tol):
    """Bit-exact legs; Frobenius error of every renewed tensor below tol;
    every block's error below tol relative to the tensor norm and below
    OWN_FACTOR * tol relative to its own norm (floor 1e-3 of the tensor)."""
    errs = {}
    for r in roles:
        legs, dense = net[r]
        assert [to_oracle_leg(l) for l in env.L[r].legs] == legs, r
        got, want = env.data(r).cpu().numpy(), u1.from_dense(legs, dense)
        errs[r] = rel_err(got, want)
        check_blocks(legs, got, want, tol, OWN_FACTOR * tol)
    assert max(errs.values()) < tol, errs
    return errs


@pytest.mark.parametrize("name,direction", [("tiny", 0), ("d4chi16", 0), ("d4chi16", 1), ("d4chi16", 2),
                                            ("d4chi16", 3)])
def test_directional_move_fp64(bst, ctx, name, direction):
    cfg, aL, ad, env = gpu_env(bst, ctx, name, u1_config(name)["chi"])
    net = oracle_net(name)
    d = "LURD"[direction]
    ref = octm.move(net, d, cfg["chi"])
    ctx.ctm_move(env, aL, ad, direction, cfg["chi"])
    renewed = {"L": ("C1", "T4", "C4"), "U": ("C1", "T1", "C2"), "R": ("C2", "T2", "C3"),
               "D": ("C3", "T3", "C4")}[d]
    compare_env(env, ref, renewed, TOL64)
    ctx.sync()


def test_full_move_fp64_d4chi16(bst, ctx):
    cfg, aL, ad, env = gpu_env(bst, ctx, "d4chi16", 16)
    net = oracle_net("d4chi16")
    ref = octm.full_move(net, cfg["chi"])
    ctx.ctm_move(env, aL, ad, 4, cfg["chi"])
    compare_env(env, ref, ("C1", "C2", "C3", "C4", "T1", "T2", "T3", "T4"), TOL64)


def test_left_move_fp64_d6chi72(bst, ctx):
    """Full-size D=6, chi=72 left move (the benchmark's directional step)."""
    cfg, aL, ad, env = gpu_env(bst, ctx, "d6chi72", 72)
    net = oracle_net("d6chi72")
    ref = octm.move(net, "L", cfg["chi"])
    ctx.ctm_move(env, aL, ad, 0, cfg["chi"])
    compare_env(env, ref, ("C1", "T4", "C4"), TOL64)


TOL_MOVE_OZ = 1e-9


@pytest.mark.parametrize("name,direction", [("d4chi16", 0), ("d4chi16", 3)])
def test_directional_move_ozaki(bst, ctx, name, direction):
    """Mixed-precision path: renewed tensors within 1e-9 of the FP64 oracle."""
    cfg, aL, ad, env = gpu_env(bst, ctx, name, u1_config(name)["chi"])
    d = "LURD"[direction]
    ref = octm.move(oracle_net(name), d, cfg["chi"])
    ctx.ctm_move(env, aL, ad, direction, cfg["chi"], prec="ozaki")
    ctx.sync()
    renewed = {"L": ("C1", "T4", "C4"), "U": ("C1", "T1", "C2"), "R": ("C2", "T2", "C3"),
               "D": ("C3", "T3", "C4")}[d]
    compare_env(env, ref, renewed, TOL_MOVE_OZ)


def test_full_move_ozaki_d6chi72(bst, ctx):
    """The benchmark step in mixed precision against the FP64 oracle."""
    cfg, aL, ad, env = gpu_env(bst, ctx, "d6chi72", 72)
    ref = octm.full_move(oracle_net("d6chi72"), cfg["chi"])
    ctx.ctm_move(env, aL, ad, 4, cfg["chi"], prec="ozaki")
    ctx.sync()
    compare_env(env, ref, ("C1", "C2", "C3", "C4", "T1", "T2", "T3", "T4"), TOL_MOVE_OZ)


def test_full_move_fp64_d6chi72(bst, ctx):
    """The benchmark step on the plain FP64 path: every direction's renewed
    tensors within 1e-12 of the FP64 oracle."""
    cfg, aL, ad, env = gpu_env(bst, ctx, "d6chi72", 72)
    ref = octm.full_move(oracle_net("d6chi72"), cfg["chi"])
    ctx.ctm_move(env, aL, ad, 4, cfg["chi"], prec="fp64")
    ctx.sync()
    compare_env(env, ref, ("C1", "C2", "C3", "C4", "T1", "T2", "T3", "T4"), TOL64)


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("ozaki", TOL_MOVE_OZ)])
def test_repeated_move_same_result(bst, prec, tol):
    """A second move on the same layouts (cached plans, buffers and projector
    views) agrees with the oracle like the first."""
    c = bst.Context(0)
    try:
        cfg, aL, ad, env = gpu_env(bst, c, "d6chi72", 72)
        ref = octm.move(oracle_net("d6chi72"), "L", cfg["chi"])
        pristine = {r: env.data(r).clone() for r in env.L}
        L0 = dict(env.L)
        c.ctm_move(env, aL, ad, 0, cfg["chi"], prec=prec)
        compare_env(env, ref, ("C1", "T4", "C4"), tol)
        for r in L0:
            env.buf[r][:pristine[r].numel()].copy_(pristine[r])
        env.L = dict(L0)
        n0 = len(c.tuning_log().splitlines())
        c.ctm_move(env, aL, ad, 0, cfg["chi"], prec=prec)
        c.sync()
        compare_env(env, ref, ("C1", "T4", "C4"), tol)
        assert len(c.tuning_log().splitlines()) > n0
    finally:
        c.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("ozaki", 1e-11)])
def test_contract_many_tiles_with_empty_sectors(bst, ctx, prec, tol):
    """Output sectors with no matched block pair (K = 0) between sectors that
    have one, with several output tiles per SM: the persistent tensor-core
    GEMM walks many tiles per CTA and the K = 0 sectors come out exactly 0."""
    r = u1.Leg(1, (-2, 0, 2), (1200, 1200, 1200))
    k = u1.Leg(-1, (0,), (64,))
    c = u1.Leg(-1, (-2, 0, 2), (1200, 1200, 1200))
    rng = np.random.default_rng(11)
    A = u1.to_dense([r, k], rng.standard_normal(u1.nnz([r, k])))
    B = u1.to_dense([k.dual(), c], rng.standard_normal(u1.nnz([k.dual(), c])))
    LA, a = upload(bst, ctx, [r, k], A)
    LB, b = upload(bst, ctx, [k.dual(), c], B)
    LC, cd = ctx.contract(LA, a, LB, b, (1,), (0,), prec=prec)
    torch.cuda.synchronize()
    ref = u1.from_dense([r, c], A @ B)
    got = cd.cpu().numpy()
    assert rel_err(got, ref) <= tol
    assert np.all(got[ref == 0] == 0)
    # alpha/beta: the K = 0 sectors keep beta times their old values
    old = torch.tensor(np.random.default_rng(12).standard_normal(LC.nnz), dtype=torch.float64, device="cuda:0")
    c2 = old.clone()
    ctx.contract(LA, a, LB, b, (1,), (0,), prec=prec, alpha=-1.5, beta=0.25, Cl=LC, c=c2)
    torch.cuda.synchronize()
    assert rel_err(c2.cpu().numpy(), -1.5 * ref + 0.25 * old.cpu().numpy()) <= tol


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_work_counter_counts_matched_block_pairs(bst, ctx, seed, prec):
    """bst_ctx_work_flops grows by exactly the matched-block-pair work of a
    contraction, whatever the arithmetic."""
    rng = np.random.default_rng(500 + seed)
    shared = rand_legs(rng, 2, 6)
    ao, bo = rand_legs(rng, 1, 6), rand_legs(rng, 2, 6)
    a_legs = [ao[0], shared[0], shared[1]]
    b_legs = [shared[1].dual(), bo[0], shared[0].dual(), bo[1]]
    A = u1.to_dense(a_legs, rng.standard_normal(u1.nnz(a_legs)))
    B = u1.to_dense(b_legs, rng.standard_normal(u1.nnz(b_legs)))
    AL, ad = upload(bst, ctx, a_legs, A)
    BL, bd = upload(bst, ctx, b_legs, B)
    w0 = ctx.work_flops
    ctx.contract(AL, ad, BL, bd, [1, 2], [2, 0], prec=prec)
    assert ctx.work_flops - w0 == matched_pair_flops(a_legs, [1, 2], b_legs, [2, 0])
