"""Bounded device waits: the tensor-core GEMM's pipeline waits give up after
the context's wait limit, record BST_E_TIMEOUT (reported by bst_ctx_sync),
wait for the copies and products they already issued, free their tensor
memory and return; the next call on the same context runs normally.  The
timeout is made to happen by a wait limit of one poll, so nothing waits on
a flag that is never set."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import u1  # noqa: E402
from bst_helpers import to_bst_leg  # noqa: E402


@pytest.fixture(scope="module")
def bst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_10804_gb300 import build
    build.build()
    from paper_1808_10804_gb300 import bst as b
    return b


def test_pipeline_wait_timeout_is_reported_and_recovered(bst):
    ctx = bst.Context(0)
    try:
        rng = np.random.default_rng(21)
        r = u1.Leg(1, (-2, 0, 2), (300, 400, 300))
        k = u1.Leg(-1, (-2, 0, 2), (200, 256, 200))
        c = u1.Leg(-1, (-4, -2, 0, 2, 4), (50, 300, 400, 300, 50))
        a_legs, b_legs = [r, k], [k.dual(), c.dual()]
        A = ctx.layout([to_bst_leg(bst, l) for l in a_legs])
        B = ctx.layout([to_bst_leg(bst, l) for l in b_legs])
        a = torch.tensor(rng.standard_normal(A.nnz), dtype=torch.float64, device="cuda:0")
        b = torch.tensor(rng.standard_normal(B.nnz), dtype=torch.float64, device="cuda:0")
        CL, ref = ctx.contract(A, a, B, b, [1], [0], prec="ozaki")
        ctx.sync()
        ctx.set_wait_limit(1)
        out = torch.zeros_like(ref)
        ctx.contract(A, a, B, b, [1], [0], prec="ozaki", Cl=CL, c=out)
        with pytest.raises(bst.BstError) as e:
            ctx.sync()
        assert e.value.code == 6          # BST_E_TIMEOUT
        ctx.sync()                        # the error word was read and cleared
        ctx.set_wait_limit(0)
        out2 = torch.zeros_like(ref)
        ctx.contract(A, a, B, b, [1], [0], prec="ozaki", Cl=CL, c=out2)
        ctx.sync()
        assert torch.equal(out2, ref)     # same bits as before the timeout
    finally:
        ctx.close()
