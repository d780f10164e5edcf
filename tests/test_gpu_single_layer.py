"""GPU parity of the single-layer CTMRG move (the double layer a is never
formed; ket and bra are contracted separately): against the dense
double-layer oracle on D=4 and D=6 workloads, and at the large U(1) workload
(D=8, chi=256) against the library's own double-layer path and between the
FP64 and mixed-precision arithmetic."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ctm as octm  # noqa: E402
from oracle import u1  # noqa: E402
from workloads import u1_config, values  # noqa: E402
from bst_helpers import check_blocks, rel_err, to_oracle_leg  # noqa: E402

TOL64 = 1e-12
TOL_MOVE_OZ = 1e-9


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


def network(ctx, name, single_layer):
    from paper_1808_10804_gb300.ctmrg import Network
    cfg = u1_config(name)
    return cfg, Network(ctx, {"A": cfg["A"], "R": cfg["R"]}, cfg["x"], cfg["chi"], lambda n, k: values(0, n, k),
                        single_layer=single_layer)


RENEWED = {"L": ("C1", "T4", "C4"), "U": ("C1", "T1", "C2"), "R": ("C2", "T2", "C3"), "D": ("C3", "T3", "C4")}


def compare(net, ref, roles, tol):
    errs = {}
    for r in roles:
        legs, dense = ref[r]
        assert [to_oracle_leg(l) for l in net.env.L[r].legs] == legs, r
        got, want = net.env.data(r).cpu().numpy(), u1.from_dense(legs, dense)
        errs[r] = rel_err(got, want)
        # per block: below tol of the tensor norm, below 100 tol of its own
        # norm (floored at 1e-3 of the tensor norm)
        check_blocks(legs, got, want, tol, 100.0 * tol)
    assert max(errs.values()) < tol, errs
    return errs


def test_single_layer_site_and_legs(bst, ctx):
    """The single-layer site A' (remover absorbed, (p, s) fused) has the
    double layer of the oracle as its double layer: the env legs agree."""
    cfg, net = network(ctx, "d4chi16", True)
    assert net.siteL.rank == 5
    onet = octm.u1_network(cfg)
    assert [to_oracle_leg(l) for l in net.aL.legs] == onet["a"][0]
    for r in ("C1", "T1", "T4", "C4"):
        assert [to_oracle_leg(l) for l in net.env.L[r].legs] == onet[r][0]


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("ozaki", TOL_MOVE_OZ)])
@pytest.mark.parametrize("direction", [0, 1, 2, 3])
def test_single_layer_directional_move_d4chi16(bst, ctx, direction, prec, tol):
    cfg, net = network(ctx, "d4chi16", True)
    d = "LURD"[direction]
    ref = octm.move(octm.u1_network(cfg), d, cfg["chi"])
    net.step(prec, direction=direction)
    ctx.sync()
    compare(net, ref, RENEWED[d], tol)


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("ozaki", TOL_MOVE_OZ)])
def test_single_layer_full_move_d6chi72(bst, ctx, prec, tol):
    cfg, net = network(ctx, "d6chi72", True)
    ref = octm.full_move(octm.u1_network(cfg), cfg["chi"])
    net.step(prec)
    ctx.sync()
    compare(net, ref, ("C1", "C2", "C3", "C4", "T1", "T2", "T3", "T4"), tol)


@pytest.fixture(scope="module")
def large_left(bst, ctx):
    """LEFT move at D=8, chi=256: single layer FP64 and mixed, double layer FP64."""
    out = {}
    full = bst.Context(0)
    full.set_projector("gesvd")
    try:
        # slmx2 repeats the mixed move in the same context: that structure
        # needed several subspace rounds, so its intermediate Rayleigh-Ritz
        # steps now run in the mixed arithmetic (then one FP64 round)
        for key, c, single, prec in (("sl64", ctx, True, "fp64"), ("slmx", ctx, True, "ozaki"),
                                     ("slmx2", ctx, True, "ozaki"), ("dl64", ctx, False, "fp64"),
                                     ("sl64_svd", full, True, "fp64")):
            cfg, net = network(c, "d8chi256", single)
            n0 = len(c.tuning_log().splitlines())
            stats = net.step(prec, direction=0)
            c.sync()
            out[key + "/log"] = c.tuning_log().splitlines()[n0:]
            out[key] = ({r: [(l.flow, l.charges, l.degs) for l in net.env.L[r].legs] for r in ("C1", "T4", "C4")},
                        {r: net.env.data(r).cpu().numpy() for r in ("C1", "T4", "C4")}, stats)
            del net
            torch.cuda.empty_cache()
    finally:
        full.close()
    return out


def test_large_single_layer_equals_double_layer(large_left):
    L1, d1, s1 = large_left["sl64"]
    L2, d2, s2 = large_left["dl64"]
    assert s1["kept"][0] == s2["kept"][0] == 256
    for r in d1:
        assert L1[r] == L2[r]
        assert rel_err(d1[r], d2[r]) < TOL64, r


def test_large_subspace_projector_vs_full_svd(large_left):
    """The subspace projector (leading candidates per sector) against the
    full FP64 SVD of every sector: same kept structure, same tensors."""
    L1, d1, s1 = large_left["sl64"]
    L2, d2, s2 = large_left["sl64_svd"]
    assert s1["kept"][0] == s2["kept"][0]
    for r in d1:
        assert L1[r] == L2[r]
        assert rel_err(d1[r], d2[r]) < TOL64, r


@pytest.mark.parametrize("key", ["slmx", "slmx2"])
def test_large_single_layer_mixed_vs_fp64(large_left, key):
    L1, d1, _ = large_left["sl64"]
    L2, d2, _ = large_left[key]
    for r in d1:
        assert L1[r] == L2[r]
        assert rel_err(d2[r], d1[r]) < TOL_MOVE_OZ, r
    mixed_rr = any("intermediate Rayleigh-Ritz" in l for l in large_left[key + "/log"])
    # the first mixed call learns that this structure needs several rounds
    assert mixed_rr == (key == "slmx2")
