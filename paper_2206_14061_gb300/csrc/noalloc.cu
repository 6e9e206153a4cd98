// lp_fit_derivatives_noalloc: the least-squares derivative fit for callers
// that cannot allocate device memory.
//
// Some callers run where cudaMalloc is off limits: code inside a memory pool
// or allocator hook that must not re-enter the allocator, plug-ins whose host
// application owns every device allocation, or real-time loops that forbid
// allocation after start-up. They cannot create an lp_ctx (which allocates its
// workspace), so this entry point keeps the only scratch the fit needs (the
// queue of stencils sent to the pivoted-QR kernel, its counter and the
// diagnostics word) in one file-scope device array. The caller still passes
// all inputs and the output.
#include <cstring>
#include <mutex>

#include "lp_internal.cuh"

namespace lp {
void launch_fit(int prec, const FitArgs& F, cudaStream_t st);
}
using namespace lp;

namespace {

// Layout of the scratch array: fallback queue, its counter, diagnostics.
constexpr size_t kQueueBytes = sizeof(int32_t) * (size_t)LP_NOALLOC_MAX_PARTICLES;
constexpr size_t kCountOff = kQueueBytes;
constexpr size_t kDiagOff = kCountOff + 256;
constexpr size_t kScratchBytes = kDiagOff + ((sizeof(DevDiag) + 255) / 256) * 256;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `dev` (the current device). The
// symbol name is a host-side stand-in; only this address may be given to a
// kernel. Looked up once per device.
lp_status scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return LP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return LP_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return LP_OK;
}

}  // namespace

extern "C" lp_status lp_fit_derivatives_noalloc(int64_t n, const double* x, const double* y,
                                                const double* z, const int32_t* nbr,
                                                const int32_t* cnt, int32_t cap,
                                                const double* const* fields,
                                                const double* mirror_sign, int32_t nf, double h,
                                                double floor_z, double* coeffs,
                                                int32_t precision, void* stream,
                                                lp_diag* diag) {
  if (n < 0 || n > LP_NOALLOC_MAX_PARTICLES) return LP_ERR_INVALID_ARG;
  if (nf < 1 || nf > kMaxFields || cap < 1 || cap > LP_MAX_CAP || !fields || !mirror_sign ||
      !(h > 0.0) || !(h < INFINITY) || !(floor_z == floor_z) ||
      (precision != LP_FP64 && precision != LP_MIXED))
    return LP_ERR_INVALID_ARG;
  if (n > 0 && (!x || !y || !z || !nbr || !cnt || !coeffs)) return LP_ERR_INVALID_ARG;
  for (int f = 0; f < nf; ++f)
    if ((n > 0 && !fields[f]) || !(mirror_sign[f] == mirror_sign[f])) return LP_ERR_INVALID_ARG;
  if (n == 0) return LP_OK;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return LP_ERR_CUDA;
  }
  void* base = nullptr;
  lp_status s = scratch_address(dev, &base);
  if (s != LP_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* b = (unsigned char*)base;
  // the array keeps the previous call's contents: clear counter and diagnostics
  if (cudaMemsetAsync(b + kCountOff, 0, kScratchBytes - kCountOff, st) != cudaSuccess) {
    cudaGetLastError();
    return LP_ERR_CUDA;
  }
  FitArgs F{};
  F.n = (int)n; F.cap = cap; F.nf = nf;
  F.x = x; F.y = y; F.z = z;
  F.nbr = nbr; F.cnt = cnt;
  for (int f = 0; f < nf; ++f) {
    F.fields[f] = fields[f];
    F.msign[f] = mirror_sign[f];
  }
  F.inv_h = 1.0 / h; F.f2 = 2.0 * floor_z;
  F.coeffs = coeffs;
  F.fb_list = (int32_t*)b;
  F.fb_count = (int32_t*)(b + kCountOff);
  F.fb_cap = LP_NOALLOC_MAX_PARTICLES;
  F.dg = (DevDiag*)(b + kDiagOff);
  launch_fit(precision, F, st);
  if (cudaGetLastError() != cudaSuccess) return LP_ERR_CUDA;
  if (!diag) return LP_OK;
  // the caller asked for the device-side counts: wait for the fit and copy
  // the diagnostics word (a plain copy into this stack frame; no allocation)
  DevDiag d;
  if (cudaMemcpyAsync(&d, b + kDiagOff, sizeof(DevDiag), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return LP_ERR_CUDA;
  }
  std::memset(diag, 0, sizeof(*diag));
  diag->flags = d.flags;
  diag->n_fallback = (int64_t)d.n_fallback;
  // more stencils needed the QR fallback than the queue holds (cannot happen
  // while the queue holds LP_NOALLOC_MAX_PARTICLES >= n entries)
  if (d.flags & LP_FLAG_OVERFLOW) return LP_ERR_STENCIL_OVERFLOW;
  return LP_OK;
}
