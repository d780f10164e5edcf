"""GPU parity of the SU(2) LEFT move (contractions with X-symbol recoupling,
projector from the reduced SVD per coupled spin J with whole-multiplet
truncation, renormalisation, norms with the 2J+1 weights) against the dense
oracle; at the full D=10, X=150 size the mixed path against the FP64 path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ctm_su2  # noqa: E402
from oracle import su2  # noqa: E402
from workloads import su2_config, values  # noqa: E402
from bst_helpers import rel_err  # noqa: E402

ENV = ("C1", "C2", "C3", "C4", "T1", "T2", "T3", "T4")


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


def gpu_net(bst, ctx, cfg, seed, chi_total):
    k = su2.Leg(1, *cfg["k"])
    x = su2.Leg(1, *cfg["x"])
    X = lambda f: su2.Leg(f, x.spins, x.degs)
    legs = {"C1": [X(-1), X(-1)], "C2": [X(1), X(-1)], "C3": [X(1), X(1)], "C4": [X(1), X(-1)],
            "T1": [X(1), k.dual(), X(-1)], "T2": [X(1), k, X(-1)],
            "T3": [X(1), k, X(-1)], "T4": [X(1), k.dual(), X(-1)],
            "a": [k, k, k.dual(), k.dual()]}
    L = {r: ctx.layout([bst.Leg(l.flow, l.spins, l.degs) for l in lg], group="su2") for r, lg in legs.items()}
    d = {r: torch.tensor(values(seed, "A" if r == "a" else r, L[r].nnz), dtype=torch.float64, device="cuda:0")
         for r in L}
    caps = {}
    for r in ENV:
        caps[r] = max(L[r].nnz, x.rdim * chi_total * (k.rdim if r.startswith("T") else 1) * 2)
    env = bst.Env(ctx, {r: L[r] for r in ENV}, {r: d[r] for r in ENV}, caps)
    return L["a"], d["a"], env


def compare(env, ref, tol):
    errs = {}
    for r in ("C1", "T4", "C4"):
        legs, dense = ref[r]
        assert [(l.flow, tuple(l.charges), tuple(l.degs)) for l in env.L[r].legs] == \
            [(l.flow, l.spins, l.degs) for l in legs], r
        errs[r] = rel_err(env.data(r).cpu().numpy(), su2.from_dense(legs, dense))
    assert max(errs.values()) < tol, errs
    return errs


@pytest.mark.parametrize("name,chi", [("small", 6), ("medium", 24)])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("ozaki", 1e-9)])
def test_su2_left_move_matches_oracle(bst, ctx, name, chi, prec, tol):
    cfg = su2_config(name)
    ref, info = ctm_su2.left_move(ctm_su2.su2_network(cfg, seed=1), chi, return_info=True)
    aL, a, env = gpu_net(bst, ctx, cfg, 1, chi)
    stats = ctx.ctm_move(env, aL, a, 0, chi, prec=prec)
    ctx.sync()
    assert stats["kept"][0] == info["dim"]
    compare(env, ref, tol)


def test_su2_other_directions_refused(bst, ctx):
    cfg = su2_config("small")
    aL, a, env = gpu_net(bst, ctx, cfg, 1, 6)
    with pytest.raises(bst.BstError) as e:
        ctx.ctm_move(env, aL, a, 1, 6)
    assert e.value.code == 8


def test_su2_left_move_full_size_mixed_vs_fp64(bst, ctx):
    """D=10 (d=5), X=150 (chi=50): no dense oracle at this size (43 TFLOP);
    the mixed path against the FP64 path, same kept multiplets."""
    cfg = su2_config("D10chi150")
    res = {}
    for prec in ("fp64", "ozaki"):
        aL, a, env = gpu_net(bst, ctx, cfg, 0, 150)
        stats = ctx.ctm_move(env, aL, a, 0, 150, prec=prec)
        ctx.sync()
        assert 0 < stats["kept"][0] <= 150
        res[prec] = ({r: [(l.flow, l.charges, l.degs) for l in env.L[r].legs] for r in ("C1", "T4", "C4")},
                     {r: env.data(r).cpu().numpy() for r in ("C1", "T4", "C4")}, stats["kept"][0])
    (L64, d64, k64), (Lmx, dmx, kmx) = res["fp64"], res["ozaki"]
    assert k64 == kmx
    for r in d64:
        assert L64[r] == Lmx[r]
        assert rel_err(dmx[r], d64[r]) < 1e-9, r
