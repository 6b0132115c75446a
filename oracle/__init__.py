"""CPU oracle for the cell-centered multigrid Poisson path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference legs
may import this package.  The product library never loads it and shares no code with it.

The arithmetic lives in ``mg_oracle.cpp`` (plain FP64 C++, compiled with
``-ffp-contract=off``); this module compiles it with g++ on first use and marshals numpy
arrays.  What each function computes, and which reading of the paper (AMReX/pyAMReX review,
arXiv 2403.12179, Sec. 2 "linear solvers for cell-centered data", "ghost cell exchange")
it follows, is stated in ``mg_oracle.cpp``.

Field layout used here (the oracle's own): a level field is a list of numpy arrays, one per
box, shaped ``(ncomp, nz+2g, ny+2g, nx+2g)`` (x fastest).  Boxes are int arrays
``(nbox, 6)`` = ``lo0 lo1 lo2 hi0 hi1 hi2`` with inclusive bounds.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, NOT_CONVERGED, ENAN = 0, -1, -4, -7


def build(force: bool = False) -> str:
    """Compile mg_oracle.cpp into oracle/_build/liboracle.so (OpenMP, -O2, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
    return _lib


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _fp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _i3(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.int32).reshape(3))


def _boxes(b):
    return np.ascontiguousarray(np.asarray(b, dtype=np.int32).reshape(-1, 6))


def domain_extent(dlo, dhi):
    return tuple(int(dhi[d]) - int(dlo[d]) + 1 for d in range(3))


# --------------------------------------------------------------------------------------
# Box bookkeeping

def chop(dlo, dhi, max_box):
    """Boxes of edge <= max_box per dim: pieces of max_box from lo, remainder last."""
    lib = _load()
    cap = 1
    for d in range(3):
        n = int(dhi[d]) - int(dlo[d]) + 1
        cap *= -(-n // int(max_box[d]))
    out = np.zeros((cap, 6), np.int32)
    nb = lib.orc_chop(_ip(_i3(dlo)), _ip(_i3(dhi)), _ip(_i3(max_box)), ctypes.c_int(cap), _ip(out))
    if nb < 0:
        raise ValueError("chop failed")
    return out[:nb]


def hierarchy(dlo, dhi, boxes):
    """Multigrid levels: list of (dlo, dhi, boxes) from fine to the bottom level."""
    lib = _load()
    boxes = _boxes(boxes)
    cap_l, cap_b = 64, 1 << 20
    dom = np.zeros((cap_l, 6), np.int32)
    nbo = np.zeros(cap_l, np.int32)
    lh = np.zeros((min(cap_b, 64 * max(len(boxes), 1) + 64), 6), np.int32)
    nl = lib.orc_hierarchy(_ip(_i3(dlo)), _ip(_i3(dhi)), ctypes.c_int(len(boxes)), _ip(boxes),
                           ctypes.c_int(cap_l), ctypes.c_int(lh.shape[0]), _ip(dom), _ip(nbo), _ip(lh))
    if nl < 0:
        raise ValueError("no valid multigrid hierarchy for this box array")
    levels, k = [], 0
    for l in range(nl):
        levels.append((dom[l, :3].copy(), dom[l, 3:].copy(), lh[k:k + nbo[l]].copy()))
        k += nbo[l]
    return levels


# --------------------------------------------------------------------------------------
# Level fields in the oracle layout

def box_shape(box, ng, ncomp=1):
    n = [int(box[3 + d]) - int(box[d]) + 1 for d in range(3)]
    return (ncomp, n[2] + 2 * ng, n[1] + 2 * ng, n[0] + 2 * ng)


def new_field(boxes, ng, ncomp=1, dtype=np.float64):
    return [np.zeros(box_shape(b, ng, ncomp), dtype) for b in _boxes(boxes)]


def pack(fabs, dtype=np.float64):
    return np.ascontiguousarray(np.concatenate([np.asarray(f, dtype).ravel() for f in fabs]))


def unpack(flat, like):
    out, k = [], 0
    for f in like:
        out.append(flat[k:k + f.size].reshape(f.shape).copy())
        k += f.size
    return out


def from_dense(dense, boxes, dlo, ng, ncomp=1):
    """Scatter a dense domain array shaped (nz, ny, nx) (or (ncomp, nz, ny, nx)) into fabs."""
    dense = np.asarray(dense)
    if dense.ndim == 3:
        dense = dense[None]
    fabs = new_field(boxes, ng, ncomp, dense.dtype)
    for f, b in zip(fabs, _boxes(boxes)):
        lo = [int(b[d]) - int(dlo[d]) for d in range(3)]
        hi = [int(b[3 + d]) - int(dlo[d]) + 1 for d in range(3)]
        sl = (slice(None), slice(ng, f.shape[1] - ng), slice(ng, f.shape[2] - ng), slice(ng, f.shape[3] - ng))
        f[sl] = dense[:, lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
    return fabs


def to_dense(fabs, boxes, dlo, dhi, ng):
    ncomp = fabs[0].shape[0]
    n = domain_extent(dlo, dhi)
    out = np.zeros((ncomp, n[2], n[1], n[0]), fabs[0].dtype)
    for f, b in zip(fabs, _boxes(boxes)):
        lo = [int(b[d]) - int(dlo[d]) for d in range(3)]
        hi = [int(b[3 + d]) - int(dlo[d]) + 1 for d in range(3)]
        out[:, lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = \
            f[:, ng:f.shape[1] - ng, ng:f.shape[2] - ng, ng:f.shape[3] - ng]
    return out[0] if ncomp == 1 else out


# --------------------------------------------------------------------------------------
# Operations (each returns new arrays; inputs are not modified)

def fill_boundary(dlo, dhi, periodic, boxes, fabs, ng):
    """Ghost fill by owner lookup: periodic image, or -(mirror) across a Dirichlet face,
    0 where the ghost lies outside the domain in two or more non-periodic directions."""
    lib = _load()
    boxes = _boxes(boxes)
    ncomp = fabs[0].shape[0]
    f32 = fabs[0].dtype == np.float32
    flat = pack(fabs, np.float32 if f32 else np.float64)
    fn = lib.orc_fill_f32 if f32 else lib.orc_fill
    rc = fn(_ip(_i3(dlo)), _ip(_i3(dhi)), _ip(_i3(periodic)), ctypes.c_int(len(boxes)), _ip(boxes),
            ctypes.c_int(ng), ctypes.c_int(ncomp), _fp(flat) if f32 else _dp(flat))
    if rc != OK:
        raise ValueError(f"orc_fill failed ({rc})")
    return unpack(flat, fabs)


def rbgs(dlo, dhi, boxes, h, phi, ng_phi, rhs, ng_rhs, color):
    """One red-black Gauss-Seidel half-sweep (phi ghosts used as given)."""
    lib = _load()
    boxes = _boxes(boxes)
    f32 = phi[0].dtype == np.float32
    dt = np.float32 if f32 else np.float64
    fp, fr = pack(phi, dt), pack(rhs, dt)
    fn = lib.orc_rbgs_f32 if f32 else lib.orc_rbgs
    cast = _fp if f32 else _dp
    rc = fn(_ip(_i3(dlo)), _ip(_i3(dhi)), ctypes.c_int(len(boxes)), _ip(boxes), ctypes.c_double(h),
            ctypes.c_int(ng_phi), cast(fp), ctypes.c_int(ng_rhs), cast(fr), ctypes.c_int(color))
    if rc != OK:
        raise ValueError(f"orc_rbgs failed ({rc})")
    return unpack(fp, phi)


def residual(dlo, dhi, boxes, h, phi, ng_phi, rhs, ng_rhs):
    """Residual fabs (no ghosts) and its max-norm."""
    lib = _load()
    boxes = _boxes(boxes)
    fp, fr = pack(phi), pack(rhs)
    r = new_field(boxes, 0)
    flat = pack(r)
    nrm = ctypes.c_double(0)
    rc = lib.orc_residual(_ip(_i3(dlo)), _ip(_i3(dhi)), ctypes.c_int(len(boxes)), _ip(boxes),
                          ctypes.c_double(h), ctypes.c_int(ng_phi), _dp(fp), ctypes.c_int(ng_rhs),
                          _dp(fr), ctypes.c_int(0), _dp(flat), ctypes.byref(nrm))
    if rc != OK:
        raise ValueError(f"orc_residual failed ({rc})")
    return unpack(flat, r), nrm.value


def restrict(fine_level, fine, ng_f, coarse_level, ng_c):
    """Coarse fabs (ng_c ghosts, ghosts zero) = mean of the 8 children of each coarse cell."""
    lib = _load()
    fdlo, fdhi, fb = fine_level
    cdlo, cdhi, cb = coarse_level
    fb, cb = _boxes(fb), _boxes(cb)
    ff = pack(fine)
    coarse = new_field(cb, ng_c)
    fc = pack(coarse)
    rc = lib.orc_restrict(_ip(_i3(fdlo)), _ip(_i3(fdhi)), ctypes.c_int(len(fb)), _ip(fb),
                          ctypes.c_int(ng_f), _dp(ff), _ip(_i3(cdlo)), _ip(_i3(cdhi)),
                          ctypes.c_int(len(cb)), _ip(cb), ctypes.c_int(ng_c), _dp(fc))
    if rc != OK:
        raise ValueError(f"orc_restrict failed ({rc})")
    return unpack(fc, coarse)


def prolong_add(coarse_level, coarse, ng_c, fine_level, fine, ng_f, trilinear=False):
    """fine + piecewise-constant injection of coarse (valid cells); trilinear: the trilinear
    form, which reads coarse's ghosts as they are (fill them first)."""
    lib = _load()
    fdlo, fdhi, fb = fine_level
    cdlo, cdhi, cb = coarse_level
    fb, cb = _boxes(fb), _boxes(cb)
    fc, ff = pack(coarse), pack(fine)
    rc = lib.orc_prolong(_ip(_i3(cdlo)), _ip(_i3(cdhi)), ctypes.c_int(len(cb)), _ip(cb),
                         ctypes.c_int(ng_c), _dp(fc), _ip(_i3(fdlo)), _ip(_i3(fdhi)),
                         ctypes.c_int(len(fb)), _ip(fb), ctypes.c_int(ng_f), _dp(ff),
                         ctypes.c_int(1 if trilinear else 0))
    if rc != OK:
        raise ValueError(f"orc_prolong failed ({rc})")
    return unpack(ff, fine)


def set_threads(n):
    """Threads of the oracle's parallel loops from now on; returns the count in effect."""
    return int(_load().orc_set_threads(ctypes.c_int(int(n))))


def bottom_matrix(n, periodic, h):
    """Closed-form inverse (Dirichlet) or pseudo-inverse (all periodic) of the bottom
    operator, ordered x fastest."""
    lib = _load()
    N = int(n[0]) * int(n[1]) * int(n[2])
    M = np.zeros((N, N), np.float64)
    rc = lib.orc_bottom_matrix(_ip(_i3(n)), _ip(_i3(periodic)), ctypes.c_double(h), _dp(M))
    if rc != OK:
        raise ValueError("bottom_matrix: size out of range")
    return M


def solve(dlo, dhi, periodic, boxes, h, rhs, phi0=None, tol=1e-10, max_iter=50, nu1=2, nu2=2,
          fixed_vcycles=-1, mixed=False, trilinear=False, inner_cycles=2):
    """V-cycle solve of A phi = rhs on a dense domain array (nz, ny, nx); trilinear selects
    the trilinear prolongation; inner_cycles: FP32 V-cycles per outer iteration of the mixed
    form (the library's default is 2).

    Returns (phi, status, vcycles, hist) where hist[i] is ||rhs - A phi_i||_inf / ||rhs||_inf
    before V-cycle i (and after the last one)."""
    lib = _load()
    boxes = _boxes(boxes)
    rhs = np.ascontiguousarray(rhs, np.float64)
    phi = np.zeros_like(rhs) if phi0 is None else np.ascontiguousarray(phi0, np.float64).copy()
    hist = np.full(max(max_iter, fixed_vcycles) + 2, np.nan)
    vc = ctypes.c_int(0)
    rc = lib.orc_solve(_ip(_i3(dlo)), _ip(_i3(dhi)), _ip(_i3(periodic)), ctypes.c_int(len(boxes)),
                       _ip(boxes), ctypes.c_double(h), _dp(rhs), _dp(phi), ctypes.c_double(tol),
                       ctypes.c_int(max_iter), ctypes.c_int(nu1), ctypes.c_int(nu2),
                       ctypes.c_int(fixed_vcycles), ctypes.c_int(1 if mixed else 0),
                       ctypes.byref(vc), _dp(hist), ctypes.c_int(len(hist)),
                       ctypes.c_int(1 if trilinear else 0), ctypes.c_int(inner_cycles))
    if rc == EINVAL:
        raise ValueError("orc_solve: invalid problem")
    return phi, rc, vc.value, hist[:vc.value + 1].copy()
