"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA path.

This module holds only workload recipes: leg charge/degeneracy lists of the
benchmark configurations and seeded normal draws.  It contains none of the
method's arithmetic (no block enumeration, fusion, contraction or SVD), so
both the oracle and the GPU path can take their inputs from here without
sharing any of the computation they are compared on.

Recipe (the readings of the configurations):
  * charges are integers 2*Sz (U(1)) or 2*j (SU(2));
  * an environment bond of total dimension chi is spread over the even
    charges -Q..Q with Gaussian weights exp(-q^2 / (2 sigma^2)),
    sigma = Q/2, rounded to the exact total by a symmetric
    largest-remainder rule (see ``gaussian_sectors``);
  * tensor entries are N(0,1) from numpy's PCG64, one independent stream
    per tensor: ``default_rng([seed, tensor_id])``; the values of a tensor
    are drawn in its canonical block order (row-major inside each block).
"""
from __future__ import annotations

import numpy as np

# tensor ids for the per-tensor random streams
TID = {"A": 0, "R": 1, "C1": 2, "C2": 3, "C3": 4, "C4": 5,
       "T1": 6, "T2": 7, "T3": 8, "T4": 9, "B": 10, "X2": 11}
IN, OUT = 1, -1


def gaussian_sectors(total, qmax, step=2, sigma=None):
    """Split `total` states over charges -qmax..qmax (in `step`s) with
    Gaussian weights, keeping the distribution symmetric under q -> -q.

    Floors of the ideal shares first; then, visiting charges by descending
    remainder (ties: smaller |q| first), a +-q pair gets one more state each
    if two are left (q = 0 takes one); what is left at the end goes to q=0.
    Returns (charges, degeneracies) with zero-degeneracy sectors dropped.
    """
    if sigma is None:
        sigma = qmax / 2.0
    qs = list(range(-qmax, qmax + 1, step))
    w = np.array([np.exp(-q * q / (2.0 * sigma * sigma)) for q in qs])
    ideal = total * w / w.sum()
    n = {q: int(np.floor(x)) for q, x in zip(qs, ideal)}
    rem = {q: x - np.floor(x) for q, x in zip(qs, ideal)}
    left = total - sum(n.values())
    for q in sorted([q for q in qs if q >= 0], key=lambda q: (-rem[q], abs(q))):
        cost = 1 if q == 0 else 2
        if cost <= left:
            n[q] += 1
            if q != 0:
                n[-q] += 1
            left -= cost
    if 0 in n:
        n[0] += left
    pairs = [(q, n[q]) for q in qs if n[q] > 0]
    return tuple(q for q, _ in pairs), tuple(d for _, d in pairs)


def values(seed, tensor, n):
    """N(0,1) float64 draws for one tensor (its canonical element order)."""
    tid = TID[tensor] if isinstance(tensor, str) else int(tensor)
    return np.random.default_rng([int(seed), tid]).standard_normal(int(n))


def leg(flow, charges, degs):
    return {"flow": int(flow), "charges": tuple(int(c) for c in charges),
            "degs": tuple(int(d) for d in degs)}


def u1_config(name):
    """Leg recipes for the U(1) CTMRG workloads.

    Site A[p, l, u, r, d]: p, l, u incoming, r, d outgoing.  The remover
    R[r, l', s] (incoming r, outgoing l' and s) sits on the right bond of
    every site and restores translation invariance of the one-site cell
    (Sec. 3.1): it removes the odd charge every spin-1/2 site adds.
    Env bonds carry the Gaussian split of chi.
    """
    if name == "d4chi16":
        phys = ((-1, 1), (1, 1))
        odd = ((-1, 1), (2, 2))
        even = ((-2, 0, 2), (1, 2, 1))
        chi, qmax = 16, 4
    elif name == "d6chi72":
        phys = ((-1, 1), (1, 1))
        odd = ((-1, 1), (3, 3))
        even = ((-2, 0, 2), (1, 4, 1))
        chi, qmax = 72, 6
    elif name == "d8chi256":
        phys = ((-3, -1, 1, 3), (1, 3, 3, 1))
        odd = ((-1, 1), (4, 4))
        even = ((-2, 0, 2), (2, 4, 2))
        chi, qmax = 256, 8
    elif name == "tiny":
        phys = ((-1, 1), (1, 1))
        odd = ((-1, 1), (1, 1))
        even = ((-2, 0, 2), (1, 1, 1))
        chi, qmax = 6, 2
    else:
        raise KeyError(name)
    xq, xd = gaussian_sectors(chi, qmax)
    spin = ((-1, 1), (1, 1))
    return {
        "name": name, "chi": chi,
        "A": [leg(IN, *phys), leg(IN, *odd), leg(IN, *even), leg(OUT, *even), leg(OUT, *even)],
        # remover: r (matches A.r), l' (matches A.l), s: spin-1/2 "physical" leg, outgoing
        "R": [leg(IN, *even), leg(OUT, *odd), leg(OUT, *spin)],
        "x": (xq, xd),
    }


def batched_u1_configs(count=64, seed=0, d_range=(4, 8), chis=(32, 64, 96, 128)):
    """Recipe for the batch of independent corner contractions: bond
    dimension D ~ U{d_range}, chi ~ U{chis}; odd leg {-1,+1} and even
    leg {-2,0,2} get a seeded random composition summing to D; the env
    bond is the Gaussian split of chi with a +-1 symmetric jitter."""
    out = []
    for i in range(count):
        rng = np.random.default_rng([seed, 1000 + i])
        D = int(rng.integers(d_range[0], d_range[1] + 1))
        chi = int(rng.choice(list(chis)))
        a = int(rng.integers(1, D))            # odd leg: a states at -1, D-a at +1
        c0 = int(rng.integers(1, D - 1)) if D > 2 else 1   # even leg: c0 at 0, rest split over +-2
        rest = D - c0
        cm = rest // 2
        cp = rest - cm
        odd = ((-1, 1), (a, D - a))
        ev = [(q, n) for q, n in ((-2, cm), (0, c0), (2, cp)) if n > 0]
        even = (tuple(q for q, _ in ev), tuple(n for _, n in ev))
        qmax = 2 * int(round(chi ** 0.5 / 3)) + 2
        xq, xd = gaussian_sectors(chi, qmax)
        xd = list(xd)
        for j in range(len(xd) // 2):
            jit = int(rng.integers(-1, 2))
            if xd[j] + jit > 0 and xd[-1 - j] + jit > 0:
                xd[j] += jit
                xd[-1 - j] += jit
        out.append({"name": f"batch{i}", "seed": seed * 100000 + i, "D": D, "chi": chi,
                    "phys": ((-1, 1), (1, 1)), "odd": odd, "even": even,
                    "x": (tuple(xq), tuple(xd))})
    return out


def batched_site_legs(cfg):
    """Site tensor A[p, l, u, r, d] of one batched instance (p, l, u
    incoming; r, d outgoing).  The instance contracts the corner-edge-edge
    block X2[k_u, x_r, k_l, x_d] (legs: the duals of the double layer's u
    and l legs, and two outgoing env bonds; values from stream "X2") with
    the double layer a[k_l, k_u, k_r, k_d] of A over (k_u, k_l)."""
    return [leg(IN, *cfg["phys"]), leg(IN, *cfg["odd"]), leg(IN, *cfg["even"]),
            leg(OUT, *cfg["even"]), leg(OUT, *cfg["even"])]


def su2_config(name):
    """Leg recipes of the SU(2) workload (spins doubled, reduced
    degeneracies): virtual bond D=10 as j=0 x1 + j=1/2 x3 + j=1 x1 (d=5),
    physical j=1/2, the double-layer leg k it fuses to (total 100, reduced
    42), and the env bond of total X=150 over j=0..3 (chi=50 reduced)."""
    if name == "D10chi150":
        return {"name": name,
                "virtual": ((0, 1, 2), (1, 3, 1)),
                "phys": ((1,), (1,)),
                "k": ((0, 1, 2, 3, 4), (11, 12, 12, 6, 1)),
                "x": ((0, 1, 2, 3, 4, 5, 6), (11, 12, 10, 7, 5, 3, 2))}
    if name == "medium":
        return {"name": name,
                "virtual": ((0, 1, 2), (1, 1, 1)),
                "phys": ((1,), (1,)),
                "k": ((0, 1, 2, 3, 4), (3, 4, 4, 2, 1)),
                "x": ((0, 1, 2, 3), (4, 4, 3, 2))}
    if name == "small":
        return {"name": name,
                "virtual": ((0, 1), (1, 1)),
                "phys": ((1,), (1,)),
                "k": ((0, 1, 2), (2, 2, 1)),
                "x": ((0, 1, 2), (2, 2, 1))}
    raise KeyError(name)
