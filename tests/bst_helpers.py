"""Helpers shared by the tests: build the same seeded workload on the oracle
side and through the library's C ABI, and compare block-sparse results."""
import numpy as np

from oracle import ctm as octm
from oracle import u1
from workloads import u1_config, values

ROLE_ORDER = ("C1", "C2", "C3", "C4", "T1", "T2", "T3", "T4")


def to_oracle_leg(l):
    return u1.Leg(int(l.flow), tuple(int(q) for q in l.charges), tuple(int(d) for d in l.degs))


def to_bst_leg(bst, l):
    return bst.Leg(int(l.flow), tuple(int(q) for q in l.charges), tuple(int(d) for d in l.degs))


def env_legs_bst(bst, xq, xd, a_legs):
    """Environment leg lists (same convention as the oracle: env bonds flow
    left-to-right and top-to-bottom; edge site legs are duals)."""
    X = lambda f: bst.Leg(f, tuple(xq), tuple(xd))
    kl, ku, kr, kd = a_legs
    return {"C1": [X(-1), X(-1)], "C2": [X(1), X(-1)], "C3": [X(1), X(1)], "C4": [X(1), X(-1)],
            "T1": [X(1), ku.dual(), X(-1)], "T2": [X(1), kr.dual(), X(-1)],
            "T3": [X(1), kd.dual(), X(-1)], "T4": [X(1), kl.dual(), X(-1)]}


def gpu_network(bst, ctx, cfg, seed=0, device="cuda:0"):
    """Site double layer (with remover) and random environment through the ABI."""
    import torch
    A = ctx.layout(cfg["A"])
    R = ctx.layout(cfg["R"])
    a_ = torch.tensor(values(seed, "A", A.nnz), dtype=torch.float64, device=device)
    r_ = torch.tensor(values(seed, "R", R.nnz), dtype=torch.float64, device=device)
    aL, ad = ctx.double_layer(A, a_, R, r_)
    legs = env_legs_bst(bst, cfg["x"][0], cfg["x"][1], aL.legs)
    Ls, data = {}, {}
    for r in ROLE_ORDER:
        Ls[r] = ctx.layout(legs[r])
        data[r] = torch.tensor(values(seed, r, Ls[r].nnz), dtype=torch.float64, device=device)
    return aL, ad, Ls, data


def rel_err(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))
