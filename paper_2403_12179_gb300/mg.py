"""Thin ctypes binding of libgbmg.so (the C ABI in include/gbmg.h).

Functions keep the C names and only marshal arguments: every computation runs in the
library's CUDA kernels.  Negative return codes raise ``MgError`` carrying the code and the
library's ``mg_last_error()`` message; ``mg_poll`` returns ``MG_PENDING`` instead of raising.
The library is loaded on first use; if it has not been built (``python -m
paper_2403_12179_gb300.build``) loading raises ``OSError`` -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libgbmg.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "gbmg.h")

MG_OK, MG_PENDING = 0, 1
MG_EINVAL, MG_ENOMEM, MG_EAGAIN, MG_NOT_CONVERGED = -1, -2, -3, -4
MG_ETIMEDOUT, MG_ECUDA, MG_ENAN = -5, -6, -7
MG_F64, MG_F32 = 0, 1
MG_BC_PERIODIC, MG_BC_DIRICHLET0 = 0, 1
MG_PREC_F64, MG_PREC_MIXED = 0, 1
MG_SMOOTH_AUTO, MG_SMOOTH_HALF, MG_SMOOTH_FUSED = 0, 1, 2
MG_SMOOTH_DIRECT_READS = 4
MG_PROLONG_CONSTANT, MG_PROLONG_TRILINEAR = 0, 1

_c_int3 = ctypes.c_int * 3


class mg_bc(ctypes.Structure):
    _fields_ = [("kind", (ctypes.c_int * 2) * 3)]


class mg_options(ctypes.Structure):
    _fields_ = [("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("precision", ctypes.c_int), ("smoother", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("fixed_vcycles", ctypes.c_int),
                ("h", ctypes.c_double), ("coarse_cells", ctypes.c_int),
                ("direct_reads", ctypes.c_int), ("prolong", ctypes.c_int),
                ("inner_cycles", ctypes.c_int)]


class mg_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("vcycles", ctypes.c_int),
                ("rel_resid", ctypes.c_double), ("seconds", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_end", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise OSError(f"libgbmg.so is not built ({LIB_PATH}); run "
                              "python -m paper_2403_12179_gb300.build")
            L = ctypes.CDLL(LIB_PATH)
            L.mg_last_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


def declared_symbols():
    """Names of the entry points declared in include/gbmg.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(mg_\w+)\s*\(", text, re.M)))


def _ck(rc):
    if rc < 0:
        raise MgError(rc, lib().mg_last_error().decode())
    return rc


def _s(stream):
    """cudaStream_t from a torch.cuda.Stream, an int handle or None."""
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def make_bc(periodic=(1, 1, 1)):
    b = mg_bc()
    for d in range(3):
        k = MG_BC_PERIODIC if periodic[d] else MG_BC_DIRICHLET0
        b.kind[d][0] = k
        b.kind[d][1] = k
    return b


def make_options(nu1=2, nu2=2, max_iter=50, precision=MG_PREC_F64, smoother=MG_SMOOTH_AUTO,
                 use_graph=1, fixed_vcycles=-1, h=0.0, coarse_cells=0, direct_reads=1,
                 prolong=MG_PROLONG_CONSTANT, inner_cycles=0):
    return mg_options(nu1, nu2, max_iter, precision, smoother, use_graph, fixed_vcycles, h,
                      coarse_cells, direct_reads, prolong, inner_cycles)


# ---- context -------------------------------------------------------------------------

def mg_init(device=0, pool_bytes=0):
    ctx = ctypes.c_void_p()
    _ck(lib().mg_init(ctypes.c_int(device), ctypes.c_size_t(pool_bytes), ctypes.byref(ctx)))
    return ctx


def mg_finalize(ctx):
    _ck(lib().mg_finalize(ctx))


def mg_last_error():
    return lib().mg_last_error().decode()


def mg_version():
    return lib().mg_version()


def mg_pool_info(ctx):
    cap, used = ctx_size(), ctx_size()
    _ck(lib().mg_pool_info(ctx, ctypes.byref(cap), ctypes.byref(used)))
    return cap.value, used.value


def ctx_size():
    return ctypes.c_size_t()


def mg_set_stream(ctx, stream):
    _ck(lib().mg_set_stream(ctx, _s(stream)))


# ---- box arrays / hierarchy ---------------------------------------------------------

def mg_box_array_create(ctx, dom_lo, dom_hi, max_box):
    out = ctypes.c_int64()
    _ck(lib().mg_box_array_create(ctx, _c_int3(*dom_lo), _c_int3(*dom_hi), _c_int3(*max_box),
                                  ctypes.byref(out)))
    return out.value


def mg_box_array_from_list(ctx, dom_lo, dom_hi, boxes):
    flat = [int(v) for b in boxes for v in b]
    arr = (ctypes.c_int * len(flat))(*flat)
    out = ctypes.c_int64()
    _ck(lib().mg_box_array_from_list(ctx, _c_int3(*dom_lo), _c_int3(*dom_hi),
                                     ctypes.c_int(len(boxes)), arr, ctypes.byref(out)))
    return out.value


def mg_box_array_info(ctx, ba):
    """(domain (lo, hi), boxes as list of 6-tuples)."""
    n = ctypes.c_int()
    dom = (ctypes.c_int * 6)()
    _ck(lib().mg_box_array_info(ctx, ctypes.c_int64(ba), ctypes.byref(n), dom, None))
    boxes = (ctypes.c_int * (6 * n.value))()
    _ck(lib().mg_box_array_info(ctx, ctypes.c_int64(ba), ctypes.byref(n), None, boxes))
    return (tuple(dom[:3]), tuple(dom[3:])), [tuple(boxes[6 * i:6 * i + 6]) for i in range(n.value)]


def mg_box_array_free(ctx, ba):
    _ck(lib().mg_box_array_free(ctx, ctypes.c_int64(ba)))


def mg_hierarchy_levels(ctx, ba):
    n = ctypes.c_int()
    _ck(lib().mg_hierarchy_levels(ctx, ctypes.c_int64(ba), ctypes.byref(n)))
    return n.value


def mg_hierarchy_level(ctx, ba, level):
    out = ctypes.c_int64()
    _ck(lib().mg_hierarchy_level(ctx, ctypes.c_int64(ba), ctypes.c_int(level), ctypes.byref(out)))
    return out.value


def mg_copy_tags(ctx, ba, bc, nghost):
    """List of tags, each a 16-int tuple (see gbmg.h)."""
    n = ctypes.c_int64()
    rc = lib().mg_copy_tags(ctx, ctypes.c_int64(ba), ctypes.byref(bc), ctypes.c_int(nghost),
                            ctypes.c_int64(0), None, ctypes.byref(n))
    if rc < 0 and n.value == 0:
        _ck(rc)
    buf = (ctypes.c_int * (16 * max(n.value, 1)))()
    _ck(lib().mg_copy_tags(ctx, ctypes.c_int64(ba), ctypes.byref(bc), ctypes.c_int(nghost),
                           ctypes.c_int64(n.value), buf, ctypes.byref(n)))
    return [tuple(buf[16 * i:16 * i + 16]) for i in range(n.value)]


def mg_bottom_matrix(n, periodic, h):
    import numpy as np
    N = int(n[0]) * int(n[1]) * int(n[2])
    M = np.zeros((N, N), np.float64)
    _ck(lib().mg_bottom_matrix(_c_int3(*n), _c_int3(*periodic), ctypes.c_double(h),
                               M.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return M


# ---- fabs ------------------------------------------------------------------------------

def mg_fab_layout(ctx, ba, ncomp, nghost, dtype):
    out = ctypes.c_size_t()
    _ck(lib().mg_fab_layout(ctx, ctypes.c_int64(ba), ctypes.c_int(ncomp), ctypes.c_int(nghost),
                            ctypes.c_int(dtype), ctypes.byref(out)))
    return out.value


def mg_fab_alloc(ctx, ba, ncomp, nghost, dtype=MG_F64):
    out = ctypes.c_int64()
    _ck(lib().mg_fab_alloc(ctx, ctypes.c_int64(ba), ctypes.c_int(ncomp), ctypes.c_int(nghost),
                           ctypes.c_int(dtype), ctypes.byref(out)))
    return out.value


def mg_fab_wrap(ctx, ba, ncomp, nghost, dtype, dptr, nbytes):
    out = ctypes.c_int64()
    _ck(lib().mg_fab_wrap(ctx, ctypes.c_int64(ba), ctypes.c_int(ncomp), ctypes.c_int(nghost),
                          ctypes.c_int(dtype), ctypes.c_void_p(dptr), ctypes.c_size_t(nbytes),
                          ctypes.byref(out)))
    return out.value


def mg_fab_ptr(ctx, fab, box):
    p = ctypes.c_void_p()
    st = (ctypes.c_int64 * 4)()
    _ck(lib().mg_fab_ptr(ctx, ctypes.c_int64(fab), ctypes.c_int(box), ctypes.byref(p), st))
    return p.value, tuple(st)


def mg_fab_info(ctx, fab):
    ba, nc, ng, dt = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _ck(lib().mg_fab_info(ctx, ctypes.c_int64(fab), ctypes.byref(ba), ctypes.byref(nc),
                          ctypes.byref(ng), ctypes.byref(dt)))
    return ba.value, nc.value, ng.value, dt.value


def mg_fab_free(ctx, fab, stream=None):
    _ck(lib().mg_fab_free(ctx, ctypes.c_int64(fab), _s(stream)))


def mg_fab_copy_from_dense(ctx, fab, src_ptr, src_on_host, stream=None):
    _ck(lib().mg_fab_copy_from_dense(ctx, ctypes.c_int64(fab), ctypes.c_void_p(src_ptr),
                                     ctypes.c_int(1 if src_on_host else 0), _s(stream)))


def mg_fab_copy_to_dense(ctx, fab, dst_ptr, dst_on_host, stream=None):
    _ck(lib().mg_fab_copy_to_dense(ctx, ctypes.c_int64(fab), ctypes.c_void_p(dst_ptr),
                                   ctypes.c_int(1 if dst_on_host else 0), _s(stream)))


def mg_fab_set_val(ctx, fab, value, include_ghosts=True, stream=None):
    _ck(lib().mg_fab_set_val(ctx, ctypes.c_int64(fab), ctypes.c_double(value),
                             ctypes.c_int(1 if include_ghosts else 0), _s(stream)))


# ---- level operations ----------------------------------------------------------------

def mg_fill_boundary(ctx, fab, bc, stream=None):
    _ck(lib().mg_fill_boundary(ctx, ctypes.c_int64(fab), ctypes.byref(bc), _s(stream)))


def mg_fill_boundary_unfused(ctx, fab, bc, stream=None):
    """The ghost fill with one launch per copy tag (the unfused baseline)."""
    _ck(lib().mg_fill_boundary_unfused(ctx, ctypes.c_int64(fab), ctypes.byref(bc), _s(stream)))


def mg_smooth(ctx, phi, rhs, bc, h, color, stream=None):
    _ck(lib().mg_smooth(ctx, ctypes.c_int64(phi), ctypes.c_int64(rhs), ctypes.byref(bc),
                        ctypes.c_double(h), ctypes.c_int(color), _s(stream)))


def mg_smooth_fused(ctx, phi_src, rhs, phi_dst, bc, h, stream=None):
    _ck(lib().mg_smooth_fused(ctx, ctypes.c_int64(phi_src), ctypes.c_int64(rhs),
                              ctypes.c_int64(phi_dst), ctypes.byref(bc), ctypes.c_double(h),
                              _s(stream)))


def mg_kernel_launches():
    n = ctypes.c_int64()
    _ck(lib().mg_kernel_launches(ctypes.byref(n)))
    return n.value


def mg_residual(ctx, phi, rhs, r=0, h=0.0, want_norm=True, stream=None):
    nrm = ctypes.c_double(0.0)
    _ck(lib().mg_residual(ctx, ctypes.c_int64(phi), ctypes.c_int64(rhs), ctypes.c_int64(r),
                          ctypes.c_double(h), ctypes.byref(nrm) if want_norm else None, _s(stream)))
    return nrm.value


def mg_residual_restrict(ctx, phi, rhs, crhs, cphi=0, h=0.0, stream=None):
    _ck(lib().mg_residual_restrict(ctx, ctypes.c_int64(phi), ctypes.c_int64(rhs),
                                   ctypes.c_int64(crhs), ctypes.c_int64(cphi), ctypes.c_double(h),
                                   _s(stream)))


def mg_restrict(ctx, fine, coarse, stream=None):
    _ck(lib().mg_restrict(ctx, ctypes.c_int64(fine), ctypes.c_int64(coarse), _s(stream)))


def mg_prolong_add(ctx, coarse, fine, stream=None):
    _ck(lib().mg_prolong_add(ctx, ctypes.c_int64(coarse), ctypes.c_int64(fine), _s(stream)))


def mg_prolong_add_trilinear(ctx, coarse, fine, stream=None):
    _ck(lib().mg_prolong_add_trilinear(ctx, ctypes.c_int64(coarse), ctypes.c_int64(fine),
                                       _s(stream)))


def mg_bottom_solve(ctx, rhs, phi, bc, h, stream=None):
    _ck(lib().mg_bottom_solve(ctx, ctypes.c_int64(rhs), ctypes.c_int64(phi), ctypes.byref(bc),
                              ctypes.c_double(h), _s(stream)))


def mg_residual_norm_noalloc(dom_lo, dom_hi, boxes, phi_ptr, phi_nghost, rhs_ptr, rhs_nghost,
                             h=0.0, stream=None):
    """Residual max-norm through the entry point that allocates no device memory (for
    callers that cannot allocate); buffers laid out as mg_fab_layout describes."""
    flat = [int(v) for b in boxes for v in b]
    arr = (ctypes.c_int * len(flat))(*flat)
    nrm = ctypes.c_double(0.0)
    _ck(lib().mg_residual_norm_noalloc(_c_int3(*dom_lo), _c_int3(*dom_hi), ctypes.c_int(len(boxes)),
                                       arr, ctypes.c_void_p(phi_ptr), ctypes.c_int(phi_nghost),
                                       ctypes.c_void_p(rhs_ptr), ctypes.c_int(rhs_nghost),
                                       ctypes.c_double(h), ctypes.byref(nrm), _s(stream)))
    return nrm.value


# ---- solves ----------------------------------------------------------------------------

def mg_solve(ctx, rhs, phi, bc, tol=1e-10, opt=None):
    res = mg_result()
    rc = lib().mg_solve(ctx, ctypes.c_int64(rhs), ctypes.c_int64(phi), ctypes.byref(bc),
                        ctypes.c_double(tol), ctypes.byref(opt) if opt is not None else None,
                        ctypes.byref(res))
    if rc < 0 and rc not in (MG_NOT_CONVERGED, MG_ENAN):
        _ck(rc)
    return res


def mg_solve_batch(ctx, rhs, phi, bcs, tol=1e-10, opt=None):
    n = len(rhs)
    R = (ctypes.c_int64 * n)(*rhs)
    P = (ctypes.c_int64 * n)(*phi)
    B = (mg_bc * n)(*bcs)
    res = (mg_result * n)()
    rc = lib().mg_solve_batch(ctx, ctypes.c_int(n), R, P, B, ctypes.c_double(tol),
                              ctypes.byref(opt) if opt is not None else None, res)
    if rc < 0 and rc not in (MG_NOT_CONVERGED, MG_ENAN):
        _ck(rc)
    return list(res)


def mg_submit(ctx, rhs, phi, bc, tol=1e-10, opt=None):
    t = ctypes.c_int64()
    _ck(lib().mg_submit(ctx, ctypes.c_int64(rhs), ctypes.c_int64(phi), ctypes.byref(bc),
                        ctypes.c_double(tol), ctypes.byref(opt) if opt is not None else None,
                        ctypes.byref(t)))
    return t.value


def mg_submit_host(ctx, dom_lo, dom_hi, max_box, bc, rhs_ptr, phi_ptr, phi_is_guess=False,
                   tol=1e-10, opt=None):
    """Queue a solve whose rhs / phi are dense FP64 host arrays (addresses; pinned memory
    recommended) that must stay alive until mg_poll reports completion."""
    t = ctypes.c_int64()
    _ck(lib().mg_submit_host(ctx, _c_int3(*dom_lo), _c_int3(*dom_hi), _c_int3(*max_box),
                             ctypes.byref(bc), ctypes.c_void_p(rhs_ptr), ctypes.c_void_p(phi_ptr),
                             ctypes.c_int(1 if phi_is_guess else 0), ctypes.c_double(tol),
                             ctypes.byref(opt) if opt is not None else None, ctypes.byref(t)))
    return t.value


def mg_server_trim(ctx):
    """Release the scheduler's idle host-memory workspaces."""
    _ck(lib().mg_server_trim(ctx))


class mg_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("max_active", ctypes.c_int64), ("admit_seconds", ctypes.c_double),
                ("plan_seconds", ctypes.c_double), ("step_seconds", ctypes.c_double),
                ("retire_seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def mg_server_stats_get(ctx):
    st = mg_server_stats()
    _ck(lib().mg_server_stats_get(ctx, ctypes.byref(st)))
    return st.as_dict()


def mg_poll(ctx, ticket, timeout_ms=-1):
    """(rc, result): rc is MG_OK or MG_PENDING."""
    res = mg_result()
    rc = lib().mg_poll(ctx, ctypes.c_int64(ticket), ctypes.c_int(timeout_ms), ctypes.byref(res))
    if rc < 0:
        _ck(rc)
    return rc, res


# ---- zero-copy views (Sec. 4.1: __cuda_array_interface__) -------------------------------

class BoxView:
    """Non-owning device view of one box of a fab (ghosts included), exposing
    ``__cuda_array_interface__`` so ``torch.as_tensor(view, device="cuda")`` (or CuPy, Numba)
    aliases the library's memory.  Shape is (ncomp, nz+2g, ny+2g, nx+2g): C order
    component, z, y, x over the library's x-fastest storage."""

    def __init__(self, ctx, fab, box):
        ba, ncomp, ng, dt = mg_fab_info(ctx, fab)
        _, boxes = mg_box_array_info(ctx, ba)
        lo, hi = boxes[box][:3], boxes[box][3:]
        ptr, st = mg_fab_ptr(ctx, fab, box)
        es = 8 if dt == MG_F64 else 4
        n = [hi[d] - lo[d] + 1 + 2 * ng for d in range(3)]
        self.shape = (ncomp, n[2], n[1], n[0])
        self.strides = (st[3] * es, st[2] * es, st[1] * es, es)
        self.typestr = "<f8" if dt == MG_F64 else "<f4"
        self.ptr = ptr
        self.lo, self.ng = lo, ng

    @property
    def __cuda_array_interface__(self):
        return {"shape": self.shape, "typestr": self.typestr, "data": (self.ptr, False),
                "strides": self.strides, "version": 3}


def mg_amr2_solve(ctx, rhs0, phi0, rhs1, phi1, bc, tol=1e-10, opt=None):
    """Two-level AMR composite solve (level 1 a refined box region of level 0)."""
    res = mg_result()
    rc = lib().mg_amr2_solve(ctx, ctypes.c_int64(rhs0), ctypes.c_int64(phi0), ctypes.c_int64(rhs1),
                             ctypes.c_int64(phi1), ctypes.byref(bc), ctypes.c_double(tol),
                             ctypes.byref(opt) if opt is not None else None, ctypes.byref(res))
    if rc < 0 and rc not in (MG_NOT_CONVERGED, MG_ENAN):
        _ck(rc)
    return res


def mg_amr2_residual(ctx, rhs0, phi0, rhs1, phi1, bc, h=0.0, r0=0, r1=0):
    """Composite residual into r0 / r1 (fabs without ghosts, or 0); returns its max-norm."""
    nrm = ctypes.c_double(0.0)
    _ck(lib().mg_amr2_residual(ctx, ctypes.c_int64(rhs0), ctypes.c_int64(phi0), ctypes.c_int64(rhs1),
                               ctypes.c_int64(phi1), ctypes.byref(bc), ctypes.c_double(h),
                               ctypes.c_int64(r0), ctypes.c_int64(r1), ctypes.byref(nrm)))
    return nrm.value


def mg_triad(ctx, a, b, c, s, per_box=False, stream=None):
    """a = b + s c on valid cells: one launch over all boxes, or one launch per box."""
    _ck(lib().mg_triad(ctx, ctypes.c_int64(a), ctypes.c_int64(b), ctypes.c_int64(c),
                       ctypes.c_double(s), ctypes.c_int(1 if per_box else 0), _s(stream)))


def mg_calib_fp64(stream, iters):
    """Enqueue the FP64 rate probe on `stream`; returns the FP64 lane operations it issues."""
    n = ctypes.c_int64()
    _ck(lib().mg_calib_fp64(_s(stream), ctypes.c_int(iters), ctypes.byref(n)))
    return n.value


def mg_sweep_timing(ctx, enable):
    """Enable / disable timing of the finest-level half-sweep inside solves; returns
    (total_ms, launches) accumulated since the previous call."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _ck(lib().mg_sweep_timing(ctx, ctypes.c_int(1 if enable else 0), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value
