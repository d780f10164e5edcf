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


def block_errors(legs, got, want):
    """Per-block errors of a flat block-sparse array against the reference
    (both in the canonical layout of `legs`): list of (||d_b||, ||ref_b||)
    in block order, with the blocks enumerated by the oracle's layout."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    out, pos = [], 0
    for b in u1.blocks(legs):
        n = int(np.prod(u1.block_shape(legs, b)))
        d = got[pos:pos + n] - want[pos:pos + n]
        out.append((float(np.linalg.norm(d)), float(np.linalg.norm(want[pos:pos + n]))))
        pos += n
    assert pos == want.size
    return out


def check_blocks(legs, got, want, tol, own_tol, floor=1e-3):
    """Every block: its error relative to the tensor norm below tol, and
    relative to its own norm (floored at `floor` times the tensor norm)
    below own_tol.  Returns the worst of each ratio."""
    tn = max(float(np.linalg.norm(want)), 1e-300)
    worst_t = worst_o = 0.0
    for i, (e, n) in enumerate(block_errors(legs, got, want)):
        rt, ro = e / tn, e / max(n, floor * tn)
        worst_t, worst_o = max(worst_t, rt), max(worst_o, ro)
        assert rt < tol and ro < own_tol, (i, rt, ro, n / tn)
    return worst_t, worst_o


def matched_pair_flops(a_legs, la, b_legs, lb):
    """2 M K N summed over every pair of allowed blocks of A and B that agree
    on the contracted legs (Sec. 2's block-pair contraction), enumerated
    from the oracle's block lists."""
    tot = 0
    bb = u1.blocks(b_legs)
    for x in u1.blocks(a_legs):
        for y in bb:
            if all(a_legs[i].charges[x[i]] == b_legs[j].charges[y[j]] for i, j in zip(la, lb)):
                sa = [a_legs[i].degs[x[i]] for i in range(len(a_legs))]
                sb = [b_legs[j].degs[y[j]] for j in range(len(b_legs))]
                k = int(np.prod([sa[i] for i in la]))
                m = int(np.prod([sa[i] for i in range(len(sa)) if i not in la]))
                n = int(np.prod([sb[j] for j in range(len(sb)) if j not in lb]))
                tot += 2 * m * k * n
    return tot


def bf16x3_bound(Am, Bm):
    """Elementwise error bound of the three-slice tensor-core product
    C = Am Bm (Am: rows x K, Bm: K x cols, dense, zeros outside the
    allowed blocks).  Each operand row (column) is scaled by 2^e with
    max|x| < 2^e <= 2 max|x| and rounded to 26 bits, |x - x^| <= 2^(e-27);
    the six kept slice products are summed exactly and the three dropped
    ones (weights 2^-27, 2^-27, 2^-36 of the leading one, digits <= 2^8 in
    magnitude) add at most 2^(ea+eb-26) per k, so every k contributes at
    most 2^(ea+eb-25) <= 2^-23 max|a_i.| max|b_.j|."""
    K = Am.shape[1]
    amax = np.abs(Am).max(axis=1)
    bmax = np.abs(Bm).max(axis=0)
    return 2.0 ** -23 * K * np.outer(amax, bmax)
