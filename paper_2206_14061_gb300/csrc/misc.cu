// Small helper kernels of the LP step library.
#include "lp_internal.cuh"

namespace lp {

__global__ void k_iota(int n, int32_t* __restrict__ a) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) a[s] = s;
}

// dst[f][ids[s]] = src[f][s]: sorted order back to the caller's order
__global__ void k_scatter_state(int n, const int32_t* __restrict__ ids,
                                const double* const* __restrict__ src,
                                double* const* __restrict__ dst, int nf) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int o = ids[s];
  if ((unsigned)o >= (unsigned)n) return;  // never write outside the caller's arrays
  for (int f = 0; f < nf; ++f) dst[f][o] = src[f][s];
}

// Heun's method: y0 <- y at the start of a step, and y <- (y0 + y) / 2 at
// its end (the seven state fields)
struct State7 {
  double* f[7];
};
__global__ void k_copy_state(int n, State7 dst, State7 src) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
#pragma unroll
  for (int k = 0; k < 7; ++k) dst.f[k][s] = src.f[k][s];
}
__global__ void k_heun_combine(int n, State7 y, State7 y0) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
#pragma unroll
  for (int k = 0; k < 7; ++k) y.f[k][s] = __dmul_rn(0.5, __dadd_rn(y0.f[k][s], y.f[k][s]));
}

void launch_copy_state(int n, double* const* dst, double* const* src, cudaStream_t st) {
  State7 d, s;
  for (int k = 0; k < 7; ++k) { d.f[k] = dst[k]; s.f[k] = src[k]; }
  k_copy_state<<<(n + 255) / 256, 256, 0, st>>>(n, d, s);
}
void launch_heun_combine(int n, double* const* y, double* const* y0, cudaStream_t st) {
  State7 a, b;
  for (int k = 0; k < 7; ++k) { a.f[k] = y[k]; b.f[k] = y0[k]; }
  k_heun_combine<<<(n + 255) / 256, 256, 0, st>>>(n, a, b);
}

void launch_iota(int n, int32_t* a, cudaStream_t st) {
  k_iota<<<(n + 255) / 256, 256, 0, st>>>(n, a);
}
void launch_scatter_state(int n, const int32_t* ids, const double* const* src,
                          double* const* dst, int nf, cudaStream_t st) {
  k_scatter_state<<<(n + 255) / 256, 256, 0, st>>>(n, ids, src, dst, nf);
}

}  // namespace lp
