// Calibration entry points (instrumentation for the roofline, not part of the solver).
//
// mg_triad is the STREAM triad a = b + s c over every valid cell of a MultiFab-like fab, the
// example the AMReX/pyAMReX review uses to measure bandwidth (Sec. 3.1) and to compare one
// kernel launch per box with one fused launch over all boxes (Sec. 3.2).  Both forms run the
// same kernel: the fused form over the box table of all boxes, the per-box form once per box
// over a one-box table.
//
// mg_calib_fp64 launches a kernel of independent FP64 fused multiply-add chains whose lane
// operation count is known, so that a caller timing it obtains the measured FP64 rate that
// the FP64 stencil kernels (bound by that rate on GB300) are compared against.
#include <cuda_runtime.h>

#include "../../include/gbmg.h"
#include "mg_kernels.hpp"
#include "mg_runtime.hpp"

using namespace gbmg;

extern "C" {

int mg_triad(mg_ctx_t h, mg_fab_t a, mg_fab_t b, mg_fab_t c, double s, int per_box, void* stream) {
  return guard([&] {
    Ctx* ctx = (Ctx*)h;
    if (!ctx) fail(MG_EINVAL, "ctx is NULL");
    ctx->require_device();
    auto fa = ctx->get_fab(a), fb = ctx->get_fab(b), fc = ctx->get_fab(c);
    for (const auto* f : {fb.get(), fc.get()}) {
      if (f->ba->ba.boxes.size() != fa->ba->ba.boxes.size() || f->dtype != fa->dtype ||
          std::memcmp(f->ba->ba.boxes.data(), fa->ba->ba.boxes.data(),
                      fa->ba->ba.boxes.size() * sizeof(Box)) != 0)
        fail(MG_EINVAL, "mg_triad: fabs differ in box array or type");
    }
    if (fa->lay.ncomp != 1 || fb->lay.ncomp != 1 || fc->lay.ncomp != 1)
      fail(MG_EINVAL, "mg_triad: one-component fabs only");
    const BoxArray& ba = fa->ba->ba;
    const cudaStream_t st = (cudaStream_t)stream;
    auto views = [&](int bx, DRow& R) {
      R.v[0] = fa->view(bx);
      R.v[1] = fb->view(bx);
      R.v[2] = fc->view(bx);
    };
    if (!per_box) {
      const OpTable& t = op_table(*ctx, "triad", {a, b, c}, 1.0, [&] {
        return make_table(*ctx, ba, 0, 1.0, 0, views, ctx->stream);
      });
      MG_CK(launch_triad_l(fa->dtype, one_seg(t.rows(), t.nbox, 0, t.width), t.nrows, s, st));
      return MG_OK;
    }
    // one row table per box, each starting at row 0 (one launch per box)
    const OpTable& t = op_table(*ctx, "triad_box", {a, b, c}, 1.0, [&] {
      std::vector<DRow> rows;
      long long n = 0;
      append_rows(&rows, &n, ba, 0, 1.0, 0, views);
      for (DRow& R : rows) R.row0 = 0;
      return upload_table(*ctx, rows, n, ctx->stream);
    });
    for (int bx = 0; bx < t.nbox; ++bx) {
      const Box& B = ba.boxes[bx];
      MG_CK(launch_triad_l(fa->dtype, one_seg(t.rows() + bx, 1, 0, B.len(0)),
                           (long long)B.len(1) * B.len(2), s, st));
    }
    return MG_OK;
  });
}

int mg_calib_fp64(void* stream, int iters, int64_t* lane_ops) {
  return guard([&] {
    if (iters < 1 || !lane_ops) fail(MG_EINVAL, "mg_calib_fp64: iters >= 1 and lane_ops needed");
    long long n = 0;
    MG_CK(launch_fp64_probe(iters, &n, (cudaStream_t)stream));
    *lane_ops = n;
    return MG_OK;
  });
}

}  // extern "C"
