"""Unit-cell CTM moves through the C ABI (bst_ctm_move_cell) against the
oracle's cell moves (Sec. 3.1 cells, Sec. 4.1's 2 x 2 cell): distinct
random sites and environments per position, every direction and the full
move, FP64 and the tensor-core arithmetic; a 1 x 1 cell equals
bst_ctm_move bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ctm as octm  # noqa: E402
from oracle import u1  # noqa: E402
from workloads import u1_config  # noqa: E402
from bst_helpers import ROLE_ORDER, check_blocks, rel_err, to_bst_leg, to_oracle_leg  # noqa: E402


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


def oracle_cell(name, Lx, Ly, seed):
    """Distinct seeded sites and environments with the legs of the
    workload's one-site network (so neighbouring sites fit)."""
    base = octm.u1_network(u1_config(name))
    rng = np.random.default_rng(seed)
    site = {}
    for x in range(Lx):
        for y in range(Ly):
            site[(x, y)] = {r: (lg, u1.to_dense(lg, rng.standard_normal(u1.nnz(lg)))) for r, (lg, _) in base.items()}
    return {"Lx": Lx, "Ly": Ly, "site": site}


def gpu_cell(bst, ctx, cell, chi):
    Lx, Ly = cell["Lx"], cell["Ly"]
    envs, aLs, ads = [], [], []
    for y in range(Ly):
        for x in range(Lx):
            net = cell["site"][(x, y)]
            Ls, data, caps = {}, {}, {}
            for r in ROLE_ORDER:
                lg, arr = net[r]
                Ls[r] = ctx.layout([to_bst_leg(bst, l) for l in lg])
                data[r] = dev(u1.from_dense(lg, arr))
                dims = [l.dim for l in lg]
                caps[r] = max(Ls[r].nnz, int(np.prod([d if (i == 1 and r.startswith("T")) else 4 * chi
                                                       for i, d in enumerate(dims)])))
            envs.append(bst.Env(ctx, Ls, data, caps))
            lg, arr = net["a"]
            aLs.append(ctx.layout([to_bst_leg(bst, l) for l in lg]))
            ads.append(dev(u1.from_dense(lg, arr)))
    return envs, aLs, ads


def compare(envs, cell, tol):
    Lx = cell["Lx"]
    for (x, y), net in cell["site"].items():
        env = envs[x + Lx * y]
        for r in ROLE_ORDER:
            legs, dense = net[r]
            assert [to_oracle_leg(l) for l in env.L[r].legs] == legs, ((x, y), r)
            got, want = env.data(r).cpu().numpy(), u1.from_dense(legs, dense)
            assert rel_err(got, want) < tol, ((x, y), r, rel_err(got, want))
            check_blocks(legs, got, want, tol, 100 * tol)


@pytest.mark.parametrize("direction", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("ozaki", 1e-9)])
def test_cell_move_matches_oracle(bst, ctx, direction, prec, tol):
    name, chi = "d4chi16", 16
    cell = oracle_cell(name, 2, 2, seed=5)
    envs, aLs, ads = gpu_cell(bst, ctx, cell, chi)
    ctx.ctm_move_cell(envs, aLs, ads, 2, 2, direction, chi, prec=prec)
    ctx.sync()
    if direction == 4:
        ref = octm.cell_full_move(cell, chi)
    else:
        ref = octm.cell_move(cell, "LURD"[direction], chi)
    compare(envs, ref, tol)


def test_rectangular_cells_match_oracle(bst, ctx):
    """2 x 1 and 1 x 3 cells, full move.  A full move of a 1 x 3 cell renews
    a site's environment through up to 2 + 3 + 3 absorptions (L and R one
    column each, U and D three rows each), each within the one-site move's
    1e-12: the bound is 1e-12 per absorption of the longest direction."""
    for Lx, Ly in ((2, 1), (1, 3)):
        cell = oracle_cell("tiny", Lx, Ly, seed=Lx + 7 * Ly)
        envs, aLs, ads = gpu_cell(bst, ctx, cell, 6)
        ctx.ctm_move_cell(envs, aLs, ads, Lx, Ly, 4, 6)
        ctx.sync()
        compare(envs, octm.cell_full_move(cell, 6), 1e-12 * max(Lx, Ly))


def test_one_site_cell_is_ctm_move(bst, ctx):
    cell = oracle_cell("d4chi16", 1, 1, seed=3)
    envs, aLs, ads = gpu_cell(bst, ctx, cell, 16)
    envs2, aLs2, ads2 = gpu_cell(bst, ctx, cell, 16)
    ctx.ctm_move_cell(envs, aLs, ads, 1, 1, 4, 16)
    ctx.ctm_move(envs2[0], aLs2[0], ads2[0], 4, 16)
    ctx.sync()
    for r in ROLE_ORDER:
        assert envs[0].L[r] == envs2[0].L[r]
        assert torch.equal(envs[0].data(r), envs2[0].data(r)), r


def checkerboard_cell(seed=3):
    """Spin-1/2 U(1) sites A and B whose virtual charges differ in parity
    (A: left leg odd, the others even; B: right leg odd): A's right leg does
    not fit its own left leg, so no one-site cell holds them, while the 2 x 2
    checkerboard A B / B A does (no remover needed)."""
    rng = np.random.default_rng(seed)
    p = u1.Leg(1, (-1, 1), (1, 1))
    odd = lambda f: u1.Leg(f, (-1, 1), (2, 2))
    even = lambda f: u1.Leg(f, (-2, 0, 2), (1, 2, 1))
    A_legs = [p, odd(1), even(1), even(-1), even(-1)]
    B_legs = [p, even(1), even(1), odd(-1), even(-1)]
    layers = []
    for legs in (A_legs, B_legs):
        layers.append(u1.double_layer(legs, u1.to_dense(legs, rng.standard_normal(u1.nnz(legs)))))
    X = ((-2, 0, 2), (2, 3, 2))
    cell = {"Lx": 2, "Ly": 2, "site": {}}
    for (x, y) in ((0, 0), (1, 0), (0, 1), (1, 1)):
        al, a = layers[(x + y) % 2]
        legs = octm.env_legs(X[0], X[1], al)
        net = {r: (lg, u1.to_dense(lg, rng.standard_normal(u1.nnz(lg)))) for r, lg in legs.items()}
        net["a"] = (al, a)
        cell["site"][(x, y)] = net
    return cell


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("ozaki", 1e-9)])
def test_checkerboard_cell_matches_oracle(bst, ctx, prec, tol):
    cell = checkerboard_cell()
    a0, a1 = cell["site"][(0, 0)]["a"][0], cell["site"][(1, 0)]["a"][0]
    assert not a0[2].dual().same_space(a0[0]) and a0[2].dual().same_space(a1[0])
    envs, aLs, ads = gpu_cell(bst, ctx, cell, 12)
    ctx.ctm_move_cell(envs, aLs, ads, 2, 2, 4, 12, prec=prec)
    ctx.sync()
    compare(envs, octm.cell_full_move(cell, 12), tol)
