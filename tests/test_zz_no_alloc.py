"""The allocation-free contraction (bst_contract_noalloc) for callers that
cannot allocate device memory (a process whose device memory another runtime
owns and has sized in advance).  Its output must match bst_contract's on the
same inputs, for two calls in a row through the shared scratch array, and a
call after the first must leave the device's free memory unchanged; a
contraction above the scratch limit must be refused.  Kept in its own file
so it is collected last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import u1  # noqa: E402
from bst_helpers import rel_err, to_bst_leg  # noqa: E402


@pytest.fixture(scope="module")
def bst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_10804_gb300 import build
    build.build()
    from paper_1808_10804_gb300 import bst as b
    return b


def _legs(seed, maxdeg):
    rng = np.random.default_rng(seed)
    def leg(flow):
        qs = sorted(rng.choice(np.arange(-3, 4), size=3, replace=False))
        return u1.Leg(flow, tuple(int(q) for q in qs), tuple(int(d) for d in rng.integers(1, maxdeg + 1, size=3)))
    s0, s1, o0, o1 = leg(1), leg(-1), leg(1), leg(-1)
    return [o0, s0, s1], [s1.dual(), o1, s0.dual()], rng


def test_noalloc_matches_contract_two_calls(bst):
    ctx = bst.Context(0)
    a_legs, b_legs, rng = _legs(11, 30)
    A = ctx.layout([to_bst_leg(bst, l) for l in a_legs])
    B = ctx.layout([to_bst_leg(bst, l) for l in b_legs])
    la, lb = [1, 2], [2, 0]
    Cl = ctx.contract_layout(A, B, la, lb)
    for call in range(2):
        a = torch.tensor(rng.standard_normal(A.nnz), dtype=torch.float64, device="cuda:0")
        b = torch.tensor(rng.standard_normal(B.nnz), dtype=torch.float64, device="cuda:0")
        _, ref = ctx.contract(A, a, B, b, la, lb, Cl=Cl)
        c = torch.full((Cl.nnz,), float("nan"), dtype=torch.float64, device="cuda:0")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        ctx.contract_noalloc(A, a, B, b, la, lb, Cl, c)
        ctx.sync()
        if call > 0:
            # the first call may load the library's module (and with it the
            # static scratch array); later calls take no device memory
            assert torch.cuda.mem_get_info()[0] == free0
        assert rel_err(c.cpu().numpy(), ref.cpu().numpy()) < 1e-13, call
        # alpha/beta accumulate into the caller's output
        c2 = ref.clone()
        ctx.contract_noalloc(A, a, B, b, la, lb, Cl, c2, alpha=2.0, beta=-1.0)
        ctx.sync()
        assert rel_err(c2.cpu().numpy(), ref.cpu().numpy()) < 1e-13, call
    ctx.close()


def test_noalloc_rejects_contractions_above_the_limit(bst):
    ctx = bst.Context(0)
    big = u1.Leg(1, (0,), (2000,))
    A = ctx.layout([to_bst_leg(bst, big), to_bst_leg(bst, big.dual())])
    B = ctx.layout([to_bst_leg(bst, big), to_bst_leg(bst, big.dual())])
    Cl = ctx.contract_layout(A, B, [1], [0])
    a = torch.zeros(A.nnz, dtype=torch.float64, device="cuda:0")
    c = torch.zeros(Cl.nnz, dtype=torch.float64, device="cuda:0")
    with pytest.raises(bst.BstError) as e:
        ctx.contract_noalloc(A, a, B, a, [1], [0], Cl, c)
    assert e.value.code == 3
    ctx.close()
