"""Helpers for the GPU tests: move oracle-layout fields in and out of library fabs through
zero-copy box views."""
import numpy as np
import torch

from paper_2403_12179_gb300 import mg


def to_fab(ctx, ba, fabs, ng, dt=mg.MG_F64):
    ncomp = fabs[0].shape[0]
    fab = mg.mg_fab_alloc(ctx, ba, ncomp, ng, dt)
    for b, f in enumerate(fabs):
        v = torch.as_tensor(mg.BoxView(ctx, fab, b), device="cuda")
        v.copy_(torch.from_numpy(np.ascontiguousarray(f)))
    torch.cuda.synchronize()
    return fab


def from_fab(ctx, fab, nbox):
    torch.cuda.synchronize()
    return [torch.as_tensor(mg.BoxView(ctx, fab, b), device="cuda").cpu().numpy().copy()
            for b in range(nbox)]


def valid(f, ng):
    return f[:, ng:f.shape[1] - ng, ng:f.shape[2] - ng, ng:f.shape[3] - ng]


def dense_fab(ctx, ba, dense, ng):
    """FP64 fab with the dense domain array (nz, ny, nx) in its valid cells."""
    fab = mg.mg_fab_alloc(ctx, ba, 1, ng, mg.MG_F64)
    t = torch.from_numpy(np.ascontiguousarray(dense, np.float64)).cuda()
    mg.mg_fab_copy_from_dense(ctx, fab, t.data_ptr(), False)
    torch.cuda.synchronize()
    return fab


def fab_dense(ctx, fab, shape):
    out = torch.empty(shape, dtype=torch.float64, device="cuda")
    mg.mg_fab_copy_to_dense(ctx, fab, out.data_ptr(), False)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def residual_numpy(phi, rhs, periodic, h):
    """Independent FP64 residual rhs - A phi of a dense field (numpy, own summation order)."""
    p = np.pad(phi, 1)
    for ax, per in zip((2, 1, 0), periodic):   # array axes are (z, y, x)
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        src_lo = [slice(None)] * 3
        src_hi = [slice(None)] * 3
        sl_lo[ax], sl_hi[ax] = 0, -1
        if per:
            src_lo[ax], src_hi[ax] = -2, 1
            p[tuple(sl_lo)] = p[tuple(src_lo)]
            p[tuple(sl_hi)] = p[tuple(src_hi)]
        else:
            src_lo[ax], src_hi[ax] = 1, -2
            p[tuple(sl_lo)] = -p[tuple(src_lo)]
            p[tuple(sl_hi)] = -p[tuple(src_hi)]
    c = p[1:-1, 1:-1, 1:-1]
    lap = (p[1:-1, 1:-1, :-2] + p[1:-1, 1:-1, 2:] + p[1:-1, :-2, 1:-1] + p[1:-1, 2:, 1:-1] +
           p[:-2, 1:-1, 1:-1] + p[2:, 1:-1, 1:-1] - 6 * c) / (h * h)
    return rhs - lap
