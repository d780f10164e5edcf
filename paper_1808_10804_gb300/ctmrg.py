"""One-site U(1) CTMRG network on the device, built through the C ABI.

Leg conventions (one-site cell, Sec. 3 and Sec. 3.1): site A[p,l,u,r,d] with
p, l, u incoming and r, d outgoing; the remover R[r,l',s] on every right
bond; the double layer a[L,U,R,D] = sum_p A (x) A* with R absorbed
(bst_double_layer); environment bonds flow left-to-right along rows and
top-to-bottom along columns; an edge tensor's site leg is the dual of the
site leg it touches.  Roles: C1[R,D] C2[L,D] C3[U,L] C4[U,R]
T1[L,D,R] T2[U,L,D] T3[L,U,R] T4[U,R,D].
"""
from __future__ import annotations

import torch

from . import bst

ROLES = bst.ROLES


def env_legs(xq, xd, a_legs):
    X = lambda f: bst.Leg(f, tuple(xq), tuple(xd))
    kl, ku, kr, kd = a_legs
    return {"C1": [X(-1), X(-1)], "C2": [X(1), X(-1)], "C3": [X(1), X(1)], "C4": [X(1), X(-1)],
            "T1": [X(1), ku.dual(), X(-1)], "T2": [X(1), kr.dual(), X(-1)],
            "T3": [X(1), kd.dual(), X(-1)], "T4": [X(1), kl.dual(), X(-1)]}


class Network:
    """Site tensors, double layer and environment of one workload.

    site_specs: leg dicts of A and R; x: (charges, degeneracies) of the env
    bond; draw(name, n) -> float64 numpy array of n values for tensor `name`.
    Env buffers get capacity for renewed tensors with chi-sized env legs.

    single_layer: the double layer is never formed; the move takes the
    single-layer site A'[P, l, u, r', d] = sum_r A[p,l,u,r,d] R[r,r',s] with
    (p, s) fused into P, and contracts ket and bra separately.
    """

    def __init__(self, ctx, site_specs, x, chi, draw, device="cuda:0", single_layer=False):
        self.ctx, self.chi, self.device = ctx, chi, device
        self.single_layer = single_layer
        self.A = ctx.layout(site_specs["A"])
        self.R = ctx.layout(site_specs["R"])
        self.A_host = torch.from_numpy(draw("A", self.A.nnz)).pin_memory()
        self.R_host = torch.from_numpy(draw("R", self.R.nnz)).pin_memory()
        self.A_dev = self.A_host.to(device)
        self.R_dev = self.R_host.to(device)
        self.build_site()
        legs = env_legs(x[0], x[1], self.aL.legs)
        self.L0, self.host0 = {}, {}
        caps = {}
        for r in ROLES:
            L = ctx.layout(legs[r])
            self.L0[r] = L
            self.host0[r] = torch.from_numpy(draw(r, L.nnz)).pin_memory()
            dims = [l.dim for l in L.legs]
            cap = 1
            for i, d in enumerate(dims):
                cap *= d if (r.startswith("T") and i == 1) else chi
            caps[r] = max(cap, L.nnz)
        self.env = bst.Env(ctx, self.L0, {r: self.host0[r].to(device) for r in ROLES}, caps)
        self.pristine = {r: self.env.buf[r].clone() for r in ROLES}

    def build_site(self):
        """The site tensor the move takes: the double layer a (with the
        remover absorbed), or the single-layer A' (single_layer=True)."""
        ctx = self.ctx
        if not self.single_layer:
            self.aL, self.a = ctx.double_layer(self.A, self.A_dev, self.R, self.R_dev)
            self.siteL, self.site = self.aL, self.a
            return
        L1, t1 = ctx.contract(self.A, self.A_dev, self.R, self.R_dev, (3,), (0,))   # [p,l,u,d,r',s]
        L2, t2 = ctx.permute(L1, t1, (0, 5, 1, 2, 4, 3))                            # [p,s,l,u,r',d]
        self.siteL, self.site = ctx.fuse(L2, t2, (2, 1, 1, 1, 1))                   # [P,l,u,r',d]
        self.aL = ctx.double_layer_layout(self.siteL)

    def reset(self):
        """Restore the input environment (device to device)."""
        for r in ROLES:
            self.env.buf[r].copy_(self.pristine[r], non_blocking=True)
        self.env.L = dict(self.L0)

    def reset_from_host(self):
        """Restore the input environment and site tensors from pinned host
        memory; returns the bytes copied host to device."""
        nb = 0
        self.A_dev.copy_(self.A_host, non_blocking=True)
        self.R_dev.copy_(self.R_host, non_blocking=True)
        nb += 8 * (self.A.nnz + self.R.nnz)
        for r in ROLES:
            n = self.L0[r].nnz
            self.env.buf[r][:n].copy_(self.host0[r], non_blocking=True)
            nb += 8 * n
        self.env.L = dict(self.L0)
        return nb

    def step(self, prec, rel_cutoff=1e-14, with_double_layer=True, direction=None):
        """One pass of the hot path: the site tensor (double layer with
        remover, or the single-layer site) and the full move LEFT, RIGHT, UP,
        DOWN (or one `direction`)."""
        if with_double_layer:
            self.build_site()
        d = bst.ALL if direction is None else direction
        return self.ctx.ctm_move(self.env, self.siteL, self.site, d, self.chi, rel_cutoff, prec)
