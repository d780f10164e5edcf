"""Iterated CTMRG through the C ABI: the square-ice (six-vertex) network,
whose partition function per site has Lieb's closed form, converged by 40
full moves on the GPU path (FP64 and mixed precision).

The model's spin-flip symmetry makes the +q and -q sectors of every
half-system spectrum exactly degenerate, so which of two equal singular
values the truncation keeps is decided by rounding: the renewed tensors are
not compared entry by entry here, only the gauge- and truncation-invariant
partition function per site (Sec. 3's CTM environment as the observable;
the dense oracle pins the same limit on the CPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ctm as octm  # noqa: E402
from oracle import u1  # noqa: E402
from bst_helpers import ROLE_ORDER, env_legs_bst, to_bst_leg, to_oracle_leg  # noqa: E402


@pytest.fixture(scope="module")
def bst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_10804_gb300 import build
    build.build()
    from paper_1808_10804_gb300 import bst as b
    return b


def ice_site():
    """2x2 ice vertices fused into one site: every fused leg carries even
    charges {-2:1, 0:2, +2:1}, so the one-site cell is consistent."""
    s = u1.Leg(1, (-1, 1), (1, 1))
    ice = u1.to_dense([s, s, s.dual(), s.dual()], np.ones(6))
    big = np.einsum("aUhV,hWbX,cViY,iXdZ->acUWbdYZ", ice, ice, ice, ice)
    fl, F = u1.fuse([s, s])
    fr, Fr = u1.fuse([s.dual(), s.dual()])
    a = np.einsum("abcdefgh,Lab,Ucd,Ref,Dgh->LURD", big, F, F, Fr, Fr)
    return [fl, fl, fr, fr], a


@pytest.mark.parametrize("prec", ["fp64", "ozaki"])
def test_square_ice_kappa_converges_to_lieb(bst, prec):
    chi = 32
    a_legs, a = ice_site()
    ctx = bst.Context(0)
    try:
        dev = "cuda:0"
        aL = ctx.layout([to_bst_leg(bst, l) for l in a_legs])
        ad = torch.tensor(u1.from_dense(a_legs, a), dtype=torch.float64, device=dev)
        legs = env_legs_bst(bst, (-2, 0, 2), (1, 1, 1), aL.legs)
        Ls, data, caps = {}, {}, {}
        for r in ROLE_ORDER:
            Ls[r] = ctx.layout(legs[r])
            data[r] = torch.ones(Ls[r].nnz, dtype=torch.float64, device=dev)
            caps[r] = chi * chi * (4 if r.startswith("T") else 1)
        env = bst.Env(ctx, Ls, data, caps)
        for _ in range(40):
            ctx.ctm_move(env, aL, ad, 4, chi, prec=prec)
        ctx.sync()
        net = {}
        for r in ROLE_ORDER:
            ol = [to_oracle_leg(l) for l in env.L[r].legs]
            net[r] = (ol, u1.to_dense(ol, env.data(r).cpu().numpy()))
        net["a"] = (a_legs, a)
        W4 = (4.0 / 3.0) ** 6
        assert abs(octm.kappa(net) / W4 - 1) < 5e-5
        # the new bonds reached chi
        x = env.L["C1"].legs[0]
        assert x.dim == chi
    finally:
        ctx.close()
