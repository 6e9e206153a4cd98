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

void launch_iota(int n, int32_t* a, cudaStream_t st) {
  k_iota<<<(n + 255) / 256, 256, 0, st>>>(n, a);
}
void launch_scatter_state(int n, const int32_t* ids, const double* const* src,
                          double* const* dst, int nf, cudaStream_t st) {
  k_scatter_state<<<(n + 255) / 256, 256, 0, st>>>(n, ids, src, dst, nf);
}

}  // namespace lp
