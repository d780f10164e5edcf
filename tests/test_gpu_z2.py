"""Z2 (parity) symmetric tensors through the C ABI against the dense oracle:
random contractions, every directional CTMRG move of a random Z2 network,
and the 2D Ising model in the Z2 basis converged on the GPU path to
Onsager's free energy (FP64 and mixed precision)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ctm as octm  # noqa: E402
from oracle import u1  # noqa: E402
from bst_helpers import ROLE_ORDER, check_blocks, rel_err  # noqa: E402
from test_oracle_ctm import onsager_kappa  # noqa: E402
from test_oracle_z2 import ising_z2_network, rand_z2_legs, zleg  # noqa: E402


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


def blayout(bst, ctx, legs):
    return ctx.layout([bst.Leg(l.flow, l.charges, l.degs) for l in legs], group="z2")


def to_oracle(L):
    return [u1.Leg(int(l.flow), tuple(int(q) for q in l.charges), tuple(int(d) for d in l.degs), 2) for l in L.legs]


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("ozaki", 1e-11)])
def test_z2_contract_matches_oracle(bst, ctx, seed, prec, tol):
    rng = np.random.default_rng(700 + seed)
    shared = [zleg(1, int(rng.integers(1, 30)), int(rng.integers(1, 30))) for _ in range(2)]
    ao, bo = rand_z2_legs(rng, 1), rand_z2_legs(rng, 1)
    a_legs = [ao[0], shared[0], shared[1]]
    b_legs = [shared[1].dual(), bo[0], shared[0].dual()]
    A = u1.to_dense(a_legs, rng.standard_normal(u1.nnz(a_legs)))
    B = u1.to_dense(b_legs, rng.standard_normal(u1.nnz(b_legs)))
    ref = np.tensordot(A, B, axes=([1, 2], [2, 0]))
    AL, BL = blayout(bst, ctx, a_legs), blayout(bst, ctx, b_legs)
    CL, c = ctx.contract(AL, dev(u1.from_dense(a_legs, A)), BL, dev(u1.from_dense(b_legs, B)), [1, 2], [2, 0],
                         prec=prec)
    ctx.sync()
    c_legs = [a_legs[0], b_legs[1]]
    assert to_oracle(CL) == c_legs
    want = u1.from_dense(c_legs, ref)
    assert rel_err(c.cpu().numpy(), want) < tol
    c2 = c.clone()
    ctx.contract(AL, dev(u1.from_dense(a_legs, A)), BL, dev(u1.from_dense(b_legs, B)), [1, 2], [2, 0], prec=prec,
                 alpha=2.0, beta=-0.5, Cl=CL, c=c2)
    ctx.sync()
    assert rel_err(c2.cpu().numpy(), 1.5 * want) < tol


def z2_network(seed=3, xd=(3, 3), kd=(2, 2)):
    rng = np.random.default_rng(seed)
    k_in, k_out = zleg(1, *kd), zleg(-1, *kd)
    a_legs = [k_in, k_in, k_out, k_out]
    net = {"a": (a_legs, u1.to_dense(a_legs, rng.standard_normal(u1.nnz(a_legs))))}
    for r, lg in octm.env_legs((0, 1), xd, a_legs).items():
        net[r] = (lg, u1.to_dense(lg, rng.standard_normal(u1.nnz(lg))))
    return net


def gpu_env(bst, ctx, net, chi):
    Ls, data, caps = {}, {}, {}
    for r in ROLE_ORDER:
        legs, dense = net[r]
        Ls[r] = blayout(bst, ctx, legs)
        data[r] = dev(u1.from_dense(legs, dense))
        k = max(l.dim for l in net["a"][0])
        caps[r] = max(Ls[r].nnz, chi * chi * (k if r.startswith("T") else 1))
    aL = blayout(bst, ctx, net["a"][0])
    ad = dev(u1.from_dense(net["a"][0], net["a"][1]))
    return aL, ad, bst.Env(ctx, Ls, data, caps)


@pytest.mark.parametrize("direction", [0, 1, 2, 3])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("ozaki", 1e-9)])
def test_z2_directional_moves_match_oracle(bst, ctx, direction, prec, tol):
    chi = 5
    net = z2_network()
    d = "LURD"[direction]
    ref = octm.move(net, d, chi)
    aL, ad, env = gpu_env(bst, ctx, net, chi)
    ctx.ctm_move(env, aL, ad, direction, chi, prec=prec)
    ctx.sync()
    renewed = {"L": ("C1", "T4", "C4"), "U": ("C1", "T1", "C2"), "R": ("C2", "T2", "C3"), "D": ("C3", "T3", "C4")}[d]
    for r in renewed:
        legs, dense = ref[r]
        assert to_oracle(env.L[r]) == legs, r
        got, want = env.data(r).cpu().numpy(), u1.from_dense(legs, dense)
        assert rel_err(got, want) < tol, r
        check_blocks(legs, got, want, tol, 100 * tol)


@pytest.mark.parametrize("beta", [0.3, 0.6])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("ozaki", 1e-9)])
def test_z2_ising_onsager_on_gpu(bst, beta, prec, tol):
    """The Ising CTMRG iterated on the GPU path (60 full moves, chi = 8)
    reaches Onsager's free energy per site.  From the all-ones start the
    truncation meets singular values down to 1e-9 of the largest, whose
    projector columns scale as sigma^-1/2 and carry rounding noise of that
    size; like any practical CTMRG run this one drops values below
    1e-10 sigma_max."""
    chi = 8
    a_legs, a = ising_z2_network(beta)
    a = np.where(u1.allowed_mask(a_legs), a, 0.0)
    net = {r: (lg, u1.to_dense(lg, np.ones(u1.nnz(lg)))) for r, lg in octm.env_legs((0,), (1,), a_legs).items()}
    net["a"] = (a_legs, a)
    c = bst.Context(0)
    try:
        aL, ad, env = gpu_env(bst, c, net, chi)
        for _ in range(60):
            c.ctm_move(env, aL, ad, 4, chi, rel_cutoff=1e-10, prec=prec)
        c.sync()
        out = {r: (to_oracle(env.L[r]), u1.to_dense(to_oracle(env.L[r]), env.data(r).cpu().numpy()))
               for r in ROLE_ORDER}
        out["a"] = (a_legs, a)
        assert abs(octm.kappa(out) / onsager_kappa(beta) - 1) < tol
    finally:
        c.close()
