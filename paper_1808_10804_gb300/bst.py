"""Thin ctypes binding of the C ABI in include/bst.h.

Argument marshalling only: every step of the computation runs in the CUDA
library ``libbst.so`` built in-tree (see ``build.py``).  Device buffers are
float64 CUDA tensors from PyTorch (used for memory and streams only); the
library fails loudly if it is missing -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from dataclasses import dataclass

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbst.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "bst.h")

FP64, OZAKI, BF16X3 = 0, 1, 2
PREC = {"fp64": FP64, "ozaki": OZAKI, "bf16x3": BF16X3, FP64: FP64, OZAKI: OZAKI, BF16X3: BF16X3}
LEFT, UP, RIGHT, DOWN, ALL = 0, 1, 2, 3, 4
ROLES = ("C1", "C2", "C3", "C4", "T1", "T2", "T3", "T4")

_lib = None


class BstError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bst error {code}: {msg}")
        self.code = code


class _Leg(C.Structure):
    _fields_ = [("flow", C.c_int32), ("nsect", C.c_int32),
                ("charge", C.POINTER(C.c_int32)), ("deg", C.POINTER(C.c_int64))]


class _Env(C.Structure):
    _fields_ = [("C", C.c_void_p * 4), ("T", C.c_void_p * 4),
                ("c", C.c_void_p * 4), ("t", C.c_void_p * 4),
                ("c_cap", C.c_int64 * 4), ("t_cap", C.c_int64 * 4)]


class _Stats(C.Structure):
    _fields_ = [("kept", C.c_int64 * 4), ("smin_over_smax", C.c_double * 4),
                ("trunc_weight", C.c_double * 4)]


class _ConvStats(C.Structure):
    _fields_ = [("value", C.c_double), ("error", C.c_double), ("error_steps", C.c_double),
                ("error_chi", C.c_double), ("chi_final", C.c_int64), ("steps_total", C.c_int32),
                ("nchi", C.c_int32), ("chi", C.c_int64 * 8), ("value_at_chi", C.c_double * 8),
                ("steps_at_chi", C.c_int32 * 8)]


def exported_names():
    """Function names declared in include/bst.h."""
    with open(HEADER) as f:
        txt = f.read()
    return sorted(set(re.findall(r"\b(bst_[a-z_0-9]+)\s*\(", txt)))


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1808_10804_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    P = C.POINTER
    sig = {
        "bst_ctx_create": [C.c_int, C.c_size_t, P(vp)],
        "bst_ctx_destroy": [vp],
        "bst_ctx_sync": [vp, vp],
        "bst_ctx_launch_count": [vp],
        "bst_ctx_work_flops": [vp],
        "bst_ctx_profile": [vp, i32],
        "bst_ctx_set_projector": [vp, i32, i32],
        "bst_ctx_set_autotune": [vp, i32],
        "bst_ctx_set_wait_limit": [vp, i64],
        "bst_ctx_tuning_log": [vp, C.c_char_p, C.c_size_t, P(C.c_size_t)],
        "bst_ctx_profile_read": [vp, i32, C.c_char_p, i32, P(i64), P(dbl), P(dbl), P(dbl)],
        "bst_layout_create": [vp, C.c_int, i32, P(_Leg), P(vp)],
        "bst_layout_retain": [vp],
        "bst_layout_release": [vp],
        "bst_layout_info": [vp, P(i32), P(i64), P(i64)],
        "bst_layout_leg": [vp, i32, P(i32), P(i32), P(i32), P(i64)],
        "bst_layout_block": [vp, i64, P(i32), P(i64), P(i64)],
        "bst_layout_dual": [vp, P(vp)],
        "bst_layout_tree": [vp, i64, P(i32), P(i32)],
        "bst_su2_cg": [i32, i32, i32, i32, i32, i32, P(dbl)],
        "bst_permute": [vp, vp, vp, P(i32), P(vp), vp, vp],
        "bst_fuse": [vp, vp, vp, i32, P(i32), P(vp), vp, vp],
        "bst_contract_layout": [vp, vp, vp, i32, P(i32), P(i32), P(vp)],
        "bst_contract_flops": [vp, vp, vp, i32, P(i32), P(i32), P(dbl)],
        "bst_plan_check": [vp, vp, vp, i32, P(i32), P(i32), P(i64)],
        "bst_contract": [vp, vp, vp, vp, vp, i32, P(i32), P(i32), C.c_int, dbl, dbl, vp, vp, vp],
        "bst_double_layer": [vp, vp, vp, vp, vp, P(vp), vp, vp],
        "bst_contract_noalloc": [vp, vp, vp, vp, vp, i32, P(i32), P(i32), dbl, dbl, vp, vp, vp],
        "bst_contract_batched": [vp, i32, P(vp), P(vp), P(vp), P(vp), i32, P(i32), P(i32), C.c_int, dbl, dbl,
                                 P(vp), P(vp), vp],
        "bst_svd_projector": [vp, vp, vp, vp, vp, i32, i64, dbl, i32, C.c_int, P(vp), vp, P(vp), vp,
                              P(dbl), P(i64), vp],
        "bst_ctm_move": [vp, i32, vp, vp, P(_Env), i64, dbl, C.c_int, P(_Stats), vp],
        "bst_ctm_move_cell": [vp, i32, i32, i32, P(vp), P(vp), P(_Env), i64, dbl, C.c_int, vp],
        "bst_sym_eig": [vp, i32, i32, vp, vp, vp, C.c_int, vp],
        "bst_double_layer_open": [vp, vp, vp, vp, vp, P(vp), vp, vp],
        "bst_ctm_bond_rdm": [vp, i32, vp, vp, P(_Env), C.c_int, P(vp), vp, i64, vp],
        "bst_dot": [vp, vp, vp, vp, P(dbl), vp],
        "bst_ctm_converge": [vp, vp, vp, vp, vp, vp, vp, P(_Env), i64, i64, dbl, i32, dbl, C.c_int,
                             P(_ConvStats), vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.bst_ctx_launch_count.restype = C.c_int64
    L.bst_ctx_work_flops.restype = C.c_double
    L.bst_last_error.restype = C.c_char_p
    L.bst_last_error.argtypes = []
    _lib = L
    return L


def su2_cg(tj1, tm1, tj2, tm2, tJ, tM):
    """<j1 m1 j2 m2|J M> (doubled arguments) as the library computes it."""
    v = C.c_double()
    _check(lib().bst_su2_cg(tj1, tm1, tj2, tm2, tJ, tM, C.byref(v)))
    return v.value


def _check(st):
    if st != 0:
        raise BstError(st, lib().bst_last_error().decode())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    assert t.dtype == torch.float64 and t.is_cuda and t.is_contiguous()
    return C.c_void_p(t.data_ptr())


def _i32(xs):
    xs = list(xs)
    return (C.c_int32 * max(1, len(xs)))(*xs)


@dataclass(frozen=True)
class Leg:
    flow: int
    charges: tuple
    degs: tuple

    @property
    def dim(self):
        return sum(self.degs)

    def dual(self):
        return Leg(-self.flow, self.charges, self.degs)


class Layout:
    """A reference to an interned, immutable block layout."""

    def __init__(self, ctx, handle):
        self.ctx = ctx
        self.h = C.c_void_p(handle) if not isinstance(handle, C.c_void_p) else handle
        r, nb, nz = C.c_int32(), C.c_int64(), C.c_int64()
        _check(lib().bst_layout_info(self.h, C.byref(r), C.byref(nb), C.byref(nz)))
        self.rank, self.nblocks, self.nnz = r.value, nb.value, nz.value

    def __del__(self):
        try:
            if self.h and self.ctx.h:
                lib().bst_layout_release(self.h)
        except Exception:
            pass

    def __eq__(self, other):
        return isinstance(other, Layout) and self.h.value == other.h.value

    def __hash__(self):
        return hash(self.h.value)

    @property
    def legs(self):
        out = []
        for i in range(self.rank):
            f, n = C.c_int32(), C.c_int32()
            _check(lib().bst_layout_leg(self.h, i, C.byref(f), C.byref(n), None, None))
            q = (C.c_int32 * n.value)()
            d = (C.c_int64 * n.value)()
            _check(lib().bst_layout_leg(self.h, i, None, None, q, d))
            out.append(Leg(f.value, tuple(q), tuple(d)))
        return out

    def blocks(self):
        out = []
        s = (C.c_int32 * self.rank)()
        sh = (C.c_int64 * self.rank)()
        off = C.c_int64()
        for b in range(self.nblocks):
            _check(lib().bst_layout_block(self.h, b, s, C.byref(off), sh))
            out.append((tuple(s), off.value, tuple(sh)))
        return out

    def trees(self):
        """Tree labels of every block (empty tuples for U(1))."""
        n = C.c_int32()
        _check(lib().bst_layout_tree(self.h, 0, C.byref(n), None)) if self.nblocks else None
        out = []
        lab = (C.c_int32 * max(1, n.value))()
        for b in range(self.nblocks):
            _check(lib().bst_layout_tree(self.h, b, None, lab))
            out.append(tuple(lab[:n.value]))
        return out

    def dual(self):
        h = C.c_void_p()
        _check(lib().bst_layout_dual(self.h, C.byref(h)))
        return Layout(self.ctx, h)

    def from_dense(self, dense):
        """Flat canonical-order data of a dense array (its allowed blocks,
        block by block, row-major): host-side marshalling of inputs such as
        operators."""
        import numpy as np
        dense = np.asarray(dense, dtype=np.float64)
        offs = [np.concatenate([[0], np.cumsum(l.degs)]) for l in self.legs]
        out = np.zeros(self.nnz)
        for sect, off, shape in self.blocks():
            sl = tuple(slice(int(o[s]), int(o[s]) + int(d)) for o, s, d in zip(offs, sect, shape))
            n = int(np.prod(shape))
            out[off:off + n] = dense[sl].reshape(-1)
        return out

    def empty(self, device=None):
        return torch.empty(max(self.nnz, 0), dtype=torch.float64,
                           device=device or f"cuda:{self.ctx.device}")


class Context:
    def __init__(self, device=0, workspace_bytes=0):
        self.device = device
        h = C.c_void_p()
        _check(lib().bst_ctx_create(device, workspace_bytes, C.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            _check(lib().bst_ctx_destroy(self.h))
            self.h = None

    def sync(self, stream=None):
        _check(lib().bst_ctx_sync(self.h, _stream(stream)))

    @property
    def launches(self):
        return lib().bst_ctx_launch_count(self.h)

    @property
    def work_flops(self):
        """Algorithmic flops of the method's contractions issued so far."""
        return lib().bst_ctx_work_flops(self.h)

    def set_projector(self, method="subspace", iters=9):
        m = {"gesvd": 0, "subspace": 1}[method]
        _check(lib().bst_ctx_set_projector(self.h, m, iters))

    def set_wait_limit(self, tries=0):
        """Bound of the tensor-core GEMM's pipeline waits in polls (0: default)."""
        _check(lib().bst_ctx_set_wait_limit(self.h, int(tries)))

    def set_autotune(self, enable=True):
        _check(lib().bst_ctx_set_autotune(self.h, 1 if enable else 0))

    def tuning_log(self):
        n = C.c_size_t()
        _check(lib().bst_ctx_tuning_log(self.h, None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value + 1)
        _check(lib().bst_ctx_tuning_log(self.h, buf, n.value + 1, None))
        return buf.value.decode()

    def profile(self, enable=True):
        _check(lib().bst_ctx_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        """{kernel class: (launches, ms, flops, bytes)} of the recorded launches."""
        out = {}
        i = 0
        while True:
            name = C.create_string_buffer(64)
            n, ms, fl, by = C.c_int64(), C.c_double(), C.c_double(), C.c_double()
            st = lib().bst_ctx_profile_read(self.h, i, name, 64, C.byref(n), C.byref(ms), C.byref(fl), C.byref(by))
            if st != 0:
                break
            out[name.value.decode()] = (n.value, ms.value, fl.value, by.value)
            i += 1
        return out

    def layout(self, legs, group="u1"):
        """Layout of the given legs; group "u1" (charges 2Sz), "su2"
        (charges 2j, degeneracies = multiplet counts) or "z2" (parities 0, 1)."""
        g = {"u1": 1, "su2": 2, "z2": 3}[group]
        legs = [l if isinstance(l, Leg) else Leg(int(l["flow"]), tuple(l["charges"]), tuple(l["degs"]))
                for l in legs]
        arr = (_Leg * len(legs))()
        keep = []
        for i, l in enumerate(legs):
            q = (C.c_int32 * len(l.charges))(*l.charges)
            d = (C.c_int64 * len(l.degs))(*l.degs)
            keep += [q, d]
            arr[i] = _Leg(l.flow, len(l.charges), q, d)
        h = C.c_void_p()
        _check(lib().bst_layout_create(self.h, g, len(legs), arr, C.byref(h)))
        return Layout(self, h)

    # ---- operations ------------------------------------------------------------
    def permute(self, L, x, perm, stream=None):
        h = C.c_void_p()
        # the output layout is known before the launch; allocate afterwards is
        # not possible, so size by nnz of the source (a permutation keeps nnz)
        out = torch.empty(L.nnz, dtype=torch.float64, device=x.device)
        _check(lib().bst_permute(self.h, L.h, _ptr(x), _i32(perm), C.byref(h), _ptr(out), _stream(stream)))
        return Layout(self, h), out

    def fuse(self, L, x, groups, stream=None):
        h = C.c_void_p()
        out = torch.empty(L.nnz, dtype=torch.float64, device=x.device)
        _check(lib().bst_fuse(self.h, L.h, _ptr(x), len(groups), _i32(groups), C.byref(h), _ptr(out),
                              _stream(stream)))
        return Layout(self, h), out

    def contract_layout(self, A, B, legsA, legsB):
        h = C.c_void_p()
        _check(lib().bst_contract_layout(self.h, A.h, B.h, len(legsA), _i32(legsA), _i32(legsB), C.byref(h)))
        return Layout(self, h)

    def plan_check(self, A, B, legsA, legsB):
        """Entries in which the device-built sector matching of contract(A, B)
        differs from the host planner's (0: identical)."""
        n = C.c_int64()
        _check(lib().bst_plan_check(self.h, A.h, B.h, len(legsA), _i32(legsA), _i32(legsB), C.byref(n)))
        return n.value

    def contract_flops(self, A, B, legsA, legsB):
        """2 M K N over the matched block pairs of contract(A, B) (host-side plan)."""
        f = C.c_double()
        _check(lib().bst_contract_flops(self.h, A.h, B.h, len(legsA), _i32(legsA), _i32(legsB), C.byref(f)))
        return f.value

    def contract(self, A, a, B, b, legsA, legsB, prec="fp64", alpha=1.0, beta=0.0, Cl=None, c=None,
                 stream=None):
        if Cl is None:
            Cl = self.contract_layout(A, B, legsA, legsB)
        if c is None:
            c = torch.empty(Cl.nnz, dtype=torch.float64, device=a.device)
        _check(lib().bst_contract(self.h, A.h, _ptr(a), B.h, _ptr(b), len(legsA), _i32(legsA), _i32(legsB),
                                  PREC[prec], alpha, beta, Cl.h, _ptr(c), _stream(stream)))
        return Cl, c

    def contract_noalloc(self, A, a, B, b, legsA, legsB, Cl, c, alpha=1.0, beta=0.0, stream=None):
        """FP64 contraction into a caller-provided output with no device
        allocation (scratch in the library's static device array)."""
        _check(lib().bst_contract_noalloc(self.h, A.h, _ptr(a), B.h, _ptr(b), len(legsA), _i32(legsA),
                                          _i32(legsB), alpha, beta, Cl.h, _ptr(c), _stream(stream)))
        return Cl, c

    def contract_batched(self, As, as_, Bs, bs, legsA, legsB, prec="fp64", alpha=1.0, beta=0.0, Cls=None,
                         cs=None, stream=None):
        """Independent contractions cs[i] = alpha*As[i]·Bs[i] + beta*cs[i] in
        one launch per stage (tensor cores: pack, GEMM with the output
        scatter in its epilogue; FP64: gather A, gather B, GEMM, scatter)."""
        n = len(As)
        if Cls is None:
            Cls = [self.contract_layout(A, B, legsA, legsB) for A, B in zip(As, Bs)]
        if cs is None:
            cs = [torch.empty(L.nnz, dtype=torch.float64, device=a.device) for L, a in zip(Cls, as_)]
        arr = C.c_void_p * n
        _check(lib().bst_contract_batched(
            self.h, n, arr(*[L.h for L in As]), arr(*[_ptr(x) for x in as_]), arr(*[L.h for L in Bs]),
            arr(*[_ptr(x) for x in bs]), len(legsA), _i32(legsA), _i32(legsB), PREC[prec], alpha, beta,
            arr(*[L.h for L in Cls]), arr(*[_ptr(x) for x in cs]), _stream(stream)))
        return Cls, cs

    def double_layer(self, A, a, R=None, r=None, stream=None):
        h = C.c_void_p()
        _check(lib().bst_double_layer(self.h, A.h, _ptr(a), R.h if R else None, _ptr(r) if R else None,
                                      C.byref(h), None, _stream(stream)))
        L = Layout(self, h)
        out = torch.empty(L.nnz, dtype=torch.float64, device=a.device)
        _check(lib().bst_double_layer(self.h, A.h, _ptr(a), R.h if R else None, _ptr(r) if R else None,
                                      C.byref(h), _ptr(out), _stream(stream)))
        return L, out

    def double_layer_open(self, A, a, R=None, r=None, stream=None):
        """Open double layer [L, U, R, D, p, p'] (physical legs kept open)."""
        h = C.c_void_p()
        _check(lib().bst_double_layer_open(self.h, A.h, _ptr(a), R.h if R else None, _ptr(r) if R else None,
                                           C.byref(h), None, _stream(stream)))
        L = Layout(self, h)
        out = torch.empty(L.nnz, dtype=torch.float64, device=a.device)
        _check(lib().bst_double_layer_open(self.h, A.h, _ptr(a), R.h if R else None, _ptr(r) if R else None,
                                           C.byref(h), _ptr(out), _stream(stream)))
        return L, out

    def bond_rdm(self, env, site_layout, site, bond, prec="fp64", stream=None):
        """Two-site density matrix rho[p_i, p_i', p_j, p_j'] of a horizontal
        (bond 0) or vertical (bond 1) bond."""
        h = C.c_void_p()
        dp = site_layout.legs[4].dim
        out = torch.empty(dp ** 4, dtype=torch.float64, device=site.device)  # at least nnz(rho)
        e = env.to_c()
        try:
            _check(lib().bst_ctm_bond_rdm(self.h, bond, site_layout.h, _ptr(site), C.byref(e), PREC[prec],
                                          C.byref(h), _ptr(out), out.numel(), _stream(stream)))
        finally:
            env.from_c(e)
        L = Layout(self, h)
        return L, out[:L.nnz]

    def dot(self, L, x, y, stream=None):
        out = C.c_double()
        _check(lib().bst_dot(self.h, L.h, _ptr(x), _ptr(y), C.byref(out), _stream(stream)))
        return out.value

    def ctm_converge(self, env, a_layout, a, site_layout, site, H_layout, H, chi0, chi_max, tol=1e-8, max_steps=15,
                     rel_cutoff=1e-14, prec="fp64", stream=None):
        """The CTM error procedure of Sec. 3 with the energy per site as the
        observable; returns a dict of the stats."""
        st = _ConvStats()
        e = env.to_c()
        try:
            _check(lib().bst_ctm_converge(self.h, a_layout.h, _ptr(a), site_layout.h, _ptr(site), H_layout.h,
                                          _ptr(H), C.byref(e), chi0, chi_max, tol, max_steps, rel_cutoff,
                                          PREC[prec], C.byref(st), _stream(stream)))
        finally:
            env.from_c(e)
        n = min(st.nchi, 8)
        return {"value": st.value, "error": st.error, "error_steps": st.error_steps, "error_chi": st.error_chi,
                "chi_final": st.chi_final, "steps_total": st.steps_total,
                "runs": [(st.chi[i], st.value_at_chi[i], st.steps_at_chi[i]) for i in range(n)]}

    def double_layer_layout(self, A, R=None):
        """Layout of the double layer of A (with the remover R) without
        computing it."""
        h = C.c_void_p()
        _check(lib().bst_double_layer(self.h, A.h, None, R.h if R else None, None, C.byref(h), None, None))
        return Layout(self, h)

    def svd_projector(self, Rt, rt, Rb, rb, ncut, chi, rel_cutoff=1e-14, new_flow=-1, prec="fp64",
                      stream=None):
        na = 1
        for l in Rt.legs[:ncut]:
            na *= l.dim
        nap = 1
        for l in Rb.legs[:ncut]:
            nap *= l.dim
        p = torch.empty(nap * chi, dtype=torch.float64, device=rt.device)
        pt = torch.empty(na * chi, dtype=torch.float64, device=rt.device)
        sv = (C.c_double * chi)()
        kept = C.c_int64()
        hp, hpt = C.c_void_p(), C.c_void_p()
        _check(lib().bst_svd_projector(self.h, Rt.h, _ptr(rt), Rb.h, _ptr(rb), ncut, chi, rel_cutoff, new_flow,
                                       PREC[prec], C.byref(hp), _ptr(p), C.byref(hpt), _ptr(pt), sv,
                                       C.byref(kept), _stream(stream)))
        P, Pt = Layout(self, hp), Layout(self, hpt)
        return P, p[:P.nnz], Pt, pt[:Pt.nnz], list(sv)[:kept.value], kept.value

    def sym_eig(self, H, prec="fp64", stream=None):
        """H: (batch, n, n) float64 CUDA tensor -> (X, lam), eigenvalues descending."""
        batch, n, _ = H.shape
        H = H.contiguous()
        X = torch.empty_like(H)
        lam = torch.empty((batch, n), dtype=torch.float64, device=H.device)
        _check(lib().bst_sym_eig(self.h, n, batch, _ptr(H), _ptr(X), _ptr(lam), PREC[prec], _stream(stream)))
        return X, lam

    def ctm_move(self, env, a_layout, a, direction, chi, rel_cutoff=1e-14, prec="fp64", stream=None):
        """env: Env; renewed tensors are rewritten in place."""
        e = env.to_c()
        st = _Stats()
        _check(lib().bst_ctm_move(self.h, direction, a_layout.h, _ptr(a), C.byref(e), chi, rel_cutoff,
                                  PREC[prec], C.byref(st), _stream(stream)))
        env.from_c(e)
        return {"kept": list(st.kept), "smin_over_smax": list(st.smin_over_smax),
                "trunc_weight": list(st.trunc_weight)}


    def ctm_move_cell(self, envs, a_layouts, a, Lx, Ly, direction, chi, rel_cutoff=1e-14, prec="fp64",
                      stream=None):
        """Unit-cell move: envs, a_layouts, a are lists over sites x + Lx*y;
        renewed tensors are rewritten in place."""
        n = Lx * Ly
        assert len(envs) == n and len(a_layouts) == n and len(a) == n
        earr = (_Env * n)(*[e.to_c() for e in envs])
        larr = (C.c_void_p * n)(*[L.h.value for L in a_layouts])
        darr = (C.c_void_p * n)(*[_ptr(x) for x in a])
        _check(lib().bst_ctm_move_cell(self.h, direction, Lx, Ly, larr, darr, earr, chi, rel_cutoff, PREC[prec],
                                       _stream(stream)))
        for e, ce in zip(envs, earr):
            e.from_c(ce)


class Env:
    """CTMRG environment: layouts and device buffers with capacities."""

    def __init__(self, ctx, layouts, data, caps=None):
        self.ctx = ctx
        self.L = dict(layouts)
        self.buf = {}
        for r in ROLES:
            cap = (caps or {}).get(r, self.L[r].nnz)
            b = torch.zeros(max(cap, 1), dtype=torch.float64, device=f"cuda:{ctx.device}")
            b[:self.L[r].nnz].copy_(data[r])
            self.buf[r] = b

    def data(self, r):
        return self.buf[r][:self.L[r].nnz]

    def to_c(self):
        e = _Env()
        for i in range(4):
            for kind, arr, carr, cap in (("C", e.C, e.c, e.c_cap), ("T", e.T, e.t, e.t_cap)):
                r = f"{kind}{i + 1}"
                lib().bst_layout_retain(self.L[r].h)
                arr[i] = self.L[r].h.value
                carr[i] = self.buf[r].data_ptr()
                cap[i] = self.buf[r].numel()
        return e

    def from_c(self, e):
        for i in range(4):
            for kind, arr in (("C", e.C), ("T", e.T)):
                r = f"{kind}{i + 1}"
                # the library released our extra reference on replaced layouts
                # and handed back new ones; wrap them (ownership moves here)
                self.L[r] = Layout(self.ctx, C.c_void_p(arr[i]))
