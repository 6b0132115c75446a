// Residual max-norm for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or anything that allocates on the device): code that
// runs while a memory budget is frozen, inside a framework that owns every device
// allocation, or at a point where an allocation could block on other streams.  The regular
// mg_residual needs device scratch -- its box table and the norm accumulator live in memory
// the library allocates on first use.  This file gives those callers one entry point that
// allocates nothing: its scratch is the file-scope array below, of a fixed maximum size,
// which every GPU that loads the library holds until the process exits.
//
// The array's name in host code is only a host-side stand-in for the device symbol: passing
// it to a kernel would fault (or silently use the wrong memory where the GPU can reach host
// memory).  The device address is looked up once per device with cudaGetSymbolAddress and
// cached for the life of the process (after a cudaDeviceReset the library must be loaded
// again).
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/gbmg.h"
#include "mg_kernels.hpp"
#include "mg_runtime.hpp"

namespace {

constexpr int kNoAllocMaxBoxes = 1024;
constexpr size_t kTableBytes = sizeof(gbmg::DRow) * kNoAllocMaxBoxes;
constexpr size_t kScratchBytes = kTableBytes + 256;  // box table, then the norm accumulator
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;                       // guards the cache and the host staging table
void* g_scratch_addr[kMaxDevices] = {};
gbmg::DRow g_host_rows[kNoAllocMaxBoxes];

// Device address of the scratch array on the current device (set-up on first use).
void* scratch_address(int dev) {
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    gbmg::check_cuda(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
    g_scratch_addr[dev] = p;
  }
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" int mg_residual_norm_noalloc(const int dom_lo[3], const int dom_hi[3], int nbox,
                                        const int* lo_hi, const double* phi, int phi_nghost,
                                        const double* rhs, int rhs_nghost, double h,
                                        double* norm, void* stream) {
  using namespace gbmg;
  return guard([&] {
    if (!dom_lo || !dom_hi || !lo_hi || !phi || !rhs || !norm)
      fail(MG_EINVAL, "mg_residual_norm_noalloc: NULL argument");
    if (nbox < 1 || nbox > kNoAllocMaxBoxes)
      fail(MG_EINVAL, "mg_residual_norm_noalloc: 1 to 1024 boxes supported");
    if (phi_nghost < 1 || rhs_nghost < 0)
      fail(MG_EINVAL, "mg_residual_norm_noalloc: phi needs at least one ghost layer");
    const double hv = h > 0 ? h : 1.0 / (dom_hi[0] - dom_lo[0] + 1);
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) fail(MG_EINVAL, "device index out of range");
    if (s && s != cudaStreamLegacy && s != cudaStreamPerThread) {
      // the scratch address belongs to the current device: a stream of another device
      // could not reach it
      int sdev = -1;
      check_cuda(cudaStreamGetDevice(s, &sdev), "cudaStreamGetDevice");
      if (sdev != dev)
        fail(MG_EINVAL, "mg_residual_norm_noalloc: the stream belongs to another device than "
                        "the current one");
    }
    std::lock_guard<std::mutex> lk(g_mu);
    char* scratch = (char*)scratch_address(dev);
    // Box table built in host static storage: each fab is laid out as mg_fab_layout
    // describes (FP64, 1 component, rows padded to 16 bytes, boxes 256-byte aligned).
    long long off_p = 0, off_r = 0, nrows = 0;
    for (int b = 0; b < nbox; ++b) {
      const int* q = lo_hi + 6 * b;
      int n[3];
      for (int d = 0; d < 3; ++d) {
        n[d] = q[3 + d] - q[d] + 1;
        if (n[d] < 1 || q[d] < dom_lo[d] || q[3 + d] > dom_hi[d])
          fail(MG_EINVAL, "mg_residual_norm_noalloc: box empty or outside the domain");
      }
      DRow& R = g_host_rows[b];
      std::memset(&R, 0, sizeof R);
      for (int d = 0; d < 3; ++d) { R.lo[d] = q[d]; R.n[d] = n[d]; }
      R.row0 = nrows;
      R.h2 = hv * hv;
      R.ih2 = 1.0 / (hv * hv);
      const double* base[2] = {phi, rhs};
      long long* off[2] = {&off_p, &off_r};
      const int gs[2] = {phi_nghost, rhs_nghost};
      for (int k = 0; k < 2; ++k) {
        const int g = gs[k];
        const int pitch = (n[0] + 2 * g + 1) / 2 * 2;             // 16-byte rows of doubles
        const long long plane = (long long)pitch * (n[1] + 2 * g);
        const long long cs = plane * (n[2] + 2 * g);
        *off[k] = (*off[k] + 31) / 32 * 32;                       // 256-byte box alignment
        DView& v = R.v[k];
        v.p = (void*)(base[k] + *off[k] + g * plane + (long long)g * pitch + g);
        v.plane = plane;
        v.cstride = cs;
        v.pitch = pitch;
        v.g = g;
        *off[k] += cs;
      }
      nrows += (long long)n[1] * n[2];
    }
    unsigned long long* acc = (unsigned long long*)(scratch + kTableBytes);
    check_cuda(cudaMemcpyAsync(scratch, g_host_rows, sizeof(DRow) * nbox, cudaMemcpyHostToDevice, s),
               "cudaMemcpyAsync");
    check_cuda(cudaMemsetAsync(acc, 0, sizeof(unsigned long long), s), "cudaMemsetAsync");
    check_cuda(launch_residual(DT_F64, (const DRow*)scratch, nbox, nrows, acc, s), "launch_residual");
    unsigned long long bits = 0;
    check_cuda(cudaMemcpyAsync(&bits, acc, sizeof bits, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
    check_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    std::memcpy(norm, &bits, sizeof bits);
    return MG_OK;
  });
}
