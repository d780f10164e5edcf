"""The sector matching built on the device (the relayout task lists,
chunk tables, sector tables and the GEMM problem list of a contraction)
equals the host planner's entry by entry, on random U(1) and Z2 layouts
and on the contractions of a CTMRG move."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import u1  # noqa: E402
from bst_helpers import gpu_network  # noqa: E402
from workloads import u1_config  # noqa: E402


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


def rand_legs(rng, rank, z2=False):
    legs = []
    for _ in range(rank):
        if z2:
            qs = sorted(rng.choice([0, 1], size=int(rng.integers(1, 3)), replace=False))
        else:
            qs = sorted(rng.choice(np.arange(-4, 5), size=int(rng.integers(1, 5)), replace=False))
        legs.append(u1.Leg(int(rng.choice([1, -1])), tuple(int(q) for q in qs),
                           tuple(int(d) for d in rng.integers(1, 5, size=len(qs))), 2 if z2 else 0))
    return legs


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("z2", [False, True])
def test_device_planner_equals_host_planner(bst, ctx, seed, z2):
    rng = np.random.default_rng(1000 + seed)
    nshared = int(rng.integers(0, 3))
    shared = rand_legs(rng, nshared, z2)
    ao = rand_legs(rng, int(rng.integers(1, 4)), z2)
    bo = rand_legs(rng, int(rng.integers(1, 3)), z2)
    a_legs = list(ao)
    pos_a = []
    for l in shared:
        k = int(rng.integers(0, len(a_legs) + 1))
        a_legs.insert(k, l)
    pos_a = [a_legs.index(l) for l in shared] if len(set(shared)) == len(shared) else None
    if pos_a is None:
        pytest.skip("repeated leg in the random draw")
    b_legs = list(bo)
    for l in shared:
        b_legs.insert(int(rng.integers(0, len(b_legs) + 1)), l.dual())
    pos_b = [b_legs.index(l.dual()) for l in shared]
    g = "z2" if z2 else "u1"
    A = ctx.layout([bst.Leg(l.flow, l.charges, l.degs) for l in a_legs], group=g)
    B = ctx.layout([bst.Leg(l.flow, l.charges, l.degs) for l in b_legs], group=g)
    if A.nnz == 0 or B.nnz == 0:
        pytest.skip("no allowed block")
    assert ctx.plan_check(A, B, pos_a, pos_b) == 0


def test_device_planner_on_the_move_contractions(bst, ctx):
    """The contractions of a D=4 move: corner, edge and site products."""
    cfg = u1_config("d4chi16")
    aL, ad, Ls, data = gpu_network(bst, ctx, cfg)
    pairs = [(Ls["C1"], Ls["T1"], [0], [0]), (Ls["T1"], Ls["C2"], [2], [0]), (Ls["T4"], Ls["C4"], [2], [0])]
    LX1 = ctx.contract_layout(Ls["C1"], Ls["T1"], [0], [0])
    LX2 = ctx.contract_layout(LX1, Ls["T4"], [0], [0])
    pairs.append((LX2, aL, [0, 2], [1, 0]))
    for A, B, la, lb in pairs:
        assert ctx.plan_check(A, B, la, lb) == 0
