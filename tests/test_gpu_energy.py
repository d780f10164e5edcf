"""Two-site observables and the CTM error procedure through the C ABI
against the dense oracle: the open double layer, the bond density matrices
(horizontal and vertical) from an environment, the Heisenberg bond energy of
a boundary cluster against its brute-force state vector, and the driver of
Sec. 3's error procedure against the oracle's run of the same procedure."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import ctm as octm  # noqa: E402
from oracle import energy, u1  # noqa: E402
from workloads import u1_config, values  # noqa: E402
from bst_helpers import ROLE_ORDER, gpu_network, rel_err, to_bst_leg, to_oracle_leg  # noqa: E402
from test_oracle_energy import boundary_network, brute_force_pauli_bond, site_with_boundary  # noqa: E402


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


def site_inputs(name):
    cfg = u1_config(name)
    A_legs = [u1.leg_from_spec(s) for s in cfg["A"]]
    R_legs = [u1.leg_from_spec(s) for s in cfg["R"]]
    A = values(0, "A", u1.nnz(A_legs))
    R = values(0, "R", u1.nnz(R_legs))
    return cfg, A_legs, A, R_legs, R


@pytest.mark.parametrize("name", ["tiny", "d4chi16"])
def test_open_double_layer_matches_oracle(bst, ctx, name):
    cfg, A_legs, A, R_legs, R = site_inputs(name)
    AL, RL = ctx.layout(cfg["A"]), ctx.layout(cfg["R"])
    SL, sd = ctx.double_layer_open(AL, dev(A), RL, dev(R))
    legs, ref = energy.open_double_layer(A_legs, u1.to_dense(A_legs, A), R_legs, u1.to_dense(R_legs, R))
    assert [to_oracle_leg(l) for l in SL.legs] == legs
    assert rel_err(sd.cpu().numpy(), u1.from_dense(legs, ref)) < 1e-14


@pytest.mark.parametrize("bond", [0, 1])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("ozaki", 1e-9)])
def test_bond_rdm_matches_oracle(bst, ctx, bond, prec, tol):
    cfg, A_legs, A, R_legs, R = site_inputs("d4chi16")
    aL, ad, Ls, data = gpu_network(bst, ctx, cfg)
    env = bst.Env(ctx, Ls, data)
    SL, sd = ctx.double_layer_open(ctx.layout(cfg["A"]), dev(A), ctx.layout(cfg["R"]), dev(R))
    RL, rho = ctx.bond_rdm(env, SL, sd, bond, prec=prec)
    ctx.sync()
    net = octm.u1_network(cfg)
    legs, site = energy.open_double_layer(A_legs, u1.to_dense(A_legs, A), R_legs, u1.to_dense(R_legs, R))
    ref = energy.bond_rdm(net, legs, site, "hv"[bond])
    p = A_legs[0]
    rlegs = [p, p.dual(), p, p.dual()]
    assert [to_oracle_leg(l) for l in RL.legs] == rlegs
    assert rel_err(rho.cpu().numpy(), u1.from_dense(rlegs, ref)) < tol


def test_boundary_cluster_energy_matches_brute_force(bst, ctx):
    """The 1 x 2 cluster with fixed open boundaries (every environment bond
    of dimension 1): the GPU density matrix of both bonds against the
    brute-force state vector's."""
    A_legs, A, R_legs, R, b_l, b_e = site_with_boundary()
    site_legs, site, net = boundary_network(A_legs, A, R_legs, R, b_l, b_e)
    AL = ctx.layout([to_bst_leg(bst, l) for l in A_legs])
    RL = ctx.layout([to_bst_leg(bst, l) for l in R_legs])
    SL, sd = ctx.double_layer_open(AL, dev(u1.from_dense(A_legs, A)), RL, dev(u1.from_dense(R_legs, R)))
    Ls, data = {}, {}
    for r in ROLE_ORDER:
        lg, arr = net[r]
        Ls[r] = ctx.layout([to_bst_leg(bst, l) for l in lg])
        data[r] = dev(u1.from_dense(lg, arr))
    env = bst.Env(ctx, Ls, data)
    h = brute_force_pauli_bond()
    H = energy.heisenberg_bond()
    for bond in (0, 1):
        RLo, rho = ctx.bond_rdm(env, SL, sd, bond)
        rlegs = [to_oracle_leg(l) for l in RLo.legs]
        dense = u1.to_dense(rlegs, rho.cpu().numpy())
        m = np.transpose(dense, (0, 2, 1, 3)).reshape(4, 4)
        # brute force: psi_s over the removers' extra legs (see the oracle test)
        if bond == 0:
            psi = np.einsum("plurd,l,u,d,rxs,qxvwe,v,e,wyt,y->pqst", A, b_l, b_e, b_e, R, A, b_e, b_e, R, b_l,
                            optimize=True)
        else:
            psi = np.einsum("plurd,l,u,rxs,x,qmdvw,m,w,vyt,y->pqst", A, b_l, b_e, R, b_l, A, b_l, b_e, R, b_l,
                            optimize=True)
        psi = psi.reshape(4, -1)
        rho_bf = psi @ psi.T
        assert np.allclose(m, rho_bf, rtol=0, atol=1e-13 * np.abs(rho_bf).max())
        HL = RLo
        e = ctx.dot(HL, rho, dev(HL.from_dense(H))) / np.trace(m)
        assert abs(e - np.trace(rho_bf @ h) / np.trace(rho_bf)) < 1e-13


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("ozaki", 1e-8)])
def test_error_procedure_matches_oracle(bst, prec, tol):
    """Sec. 3's procedure (threshold, step limit, chi doubling) on the D=4
    workload from chi = 4 to 16: the driver's energies per fixed-chi run and
    its step counts match the oracle running the same procedure."""
    cfg, A_legs, A, R_legs, R = site_inputs("d4chi16")
    c = bst.Context(0)
    try:
        aL, ad, Ls, data = gpu_network(bst, c, cfg)
        caps = {r: max(L.nnz, 16 * 16 * (16 if r.startswith("T") else 1)) for r, L in Ls.items()}
        env = bst.Env(c, Ls, data, caps)
        SL, sd = c.double_layer_open(c.layout(cfg["A"]), dev(A), c.layout(cfg["R"]), dev(R))
        p = SL.legs[4]
        HL = c.layout([p, p.dual(), p, p.dual()])
        H = dev(HL.from_dense(energy.heisenberg_bond()))
        st = c.ctm_converge(env, aL, ad, SL, sd, HL, H, 4, 16, tol=1e-8, max_steps=15, prec=prec)
    finally:
        c.close()
    net = octm.u1_network(cfg)
    legs, site = energy.open_double_layer(A_legs, u1.to_dense(A_legs, A), R_legs, u1.to_dense(R_legs, R))
    Hd = energy.heisenberg_bond()
    val, err, hist, _ = energy.converge(net, 4, lambda n: energy.site_energy(n, legs, site, Hd), tol=1e-8,
                                        chi_max=16)
    assert [r[0] for r in st["runs"]] == [h[0] for h in hist]
    if prec == "fp64":
        # the same stopping decisions (the mixed path's energies differ by
        # ~1e-10, which can move a decision at the 1e-8 threshold)
        assert [r[2] for r in st["runs"]] == [len(h[1]) for h in hist]
    for (chi, v, n), (chi2, vals) in zip(st["runs"], hist):
        assert abs(v - vals[-1]) < tol * max(1.0, abs(vals[-1])), (chi, v, vals[-1])
    assert abs(st["value"] - val) < tol * max(1.0, abs(val))
    assert st["error"] == pytest.approx(err, rel=1e-3, abs=10 * tol)
