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
// (along a periodic axis, period L > 0: the mean of the two positions taken
// on the same image, moved back into [0, L))
__global__ void k_heun_combine(int n, State7 y, State7 y0, double Lx, double Ly) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    const double a = y0.f[k][s], b = y.f[k][s];
    const double L = k == 0 ? Lx : (k == 1 ? Ly : 0.0);
    y.f[k][s] = L > 0.0
                    ? wrap_pos(__dadd_rn(a, __dmul_rn(0.5, min_image(__dsub_rn(b, a), L))), L)
                    : __dmul_rn(0.5, __dadd_rn(a, b));
  }
}

// Caller positions along periodic axes mapped into [0, L) before the first
// step (values already there are kept as they are; non-finite ones too)
__device__ __forceinline__ double wrap_any(double v, double L) {
  if ((v >= 0.0 && v < L) || !isfinite(v)) return v;
  double r = fmod(v, L);  // exact, |r| < L, with the sign of v
  if (r < 0.0) r = __dadd_rn(r, L);
  return r < L ? r : 0.0;
}
__global__ void k_wrap_positions(int n, double* __restrict__ x, double* __restrict__ y,
                                 double Lx, double Ly) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  if (Lx > 0.0) x[s] = wrap_any(x[s], Lx);
  if (Ly > 0.0) y[s] = wrap_any(y[s], Ly);
}

void launch_copy_state(int n, double* const* dst, double* const* src, cudaStream_t st) {
  State7 d, s;
  for (int k = 0; k < 7; ++k) { d.f[k] = dst[k]; s.f[k] = src[k]; }
  k_copy_state<<<(n + 255) / 256, 256, 0, st>>>(n, d, s);
}
void launch_heun_combine(int n, double* const* y, double* const* y0, double Lx, double Ly,
                         cudaStream_t st) {
  State7 a, b;
  for (int k = 0; k < 7; ++k) { a.f[k] = y[k]; b.f[k] = y0[k]; }
  k_heun_combine<<<(n + 255) / 256, 256, 0, st>>>(n, a, b, Lx, Ly);
}
// Verlet lists kept across calls: flag a search if some particle moved more
// than skin/2 (squared: half_skin2) since the last one, or is not finite; the
// caller's state enters the running maximum displacements of filter skipping
// as every step's new state does (the pass-2 epilogue)
__global__ void k_need_search(int n, const double* __restrict__ x, const double* __restrict__ y,
                              const double* __restrict__ z, const double* __restrict__ xref,
                              double half_skin2, double Lx, double Ly, int* __restrict__ flag,
                              VerletSkip vs) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  float disp = 0.f;
  if (s < n) {
    const double ex = min_image(x[s] - xref[s], Lx), ey = min_image(y[s] - xref[n + s], Ly);
    const double ez = z[s] - xref[2 * n + s];
    const double e2 = ((ex * ex) + (ey * ey)) + (ez * ez);
    if (!(e2 <= half_skin2)) *flag = 1;
    if (vs.dmax) {
      disp = fmaxf(vs.dmax[s], sqrtf(__double2float_ru(e2)) * (1.f + 0x1p-21f));
      vs.dmax[s] = disp;
    }
  }
  if (vs.dmax_all) {  // (the whole warp is here: no early exit above)
    const unsigned v = __reduce_max_sync(0xffffffffu, __float_as_uint(disp));
    if ((threadIdx.x & 31) == 0 && v) atomicMax(vs.dmax_all, v);
  }
}
void launch_need_search(int n, const double* x, const double* y, const double* z,
                        const double* xref, double half_skin2, double Lx, double Ly, int* flag,
                        VerletSkip vs, cudaStream_t st) {
  k_need_search<<<(n + 255) / 256, 256, 0, st>>>(n, x, y, z, xref, half_skin2, Lx, Ly, flag, vs);
}
void launch_wrap_positions(int n, double* x, double* y, double Lx, double Ly, cudaStream_t st) {
  k_wrap_positions<<<(n + 255) / 256, 256, 0, st>>>(n, x, y, Lx, Ly);
}

// y = a x + b y over n doubles (the adjoint of Heun's average); x may be y
__global__ void k_axpby(int64_t n, double a, const double* x, double b, double* y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + b * y[i];
}
void launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st) {
  k_axpby<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a, x, b, y);
}

void launch_iota(int n, int32_t* a, cudaStream_t st) {
  k_iota<<<(n + 255) / 256, 256, 0, st>>>(n, a);
}
void launch_scatter_state(int n, const int32_t* ids, const double* const* src,
                          double* const* dst, int nf, cudaStream_t st) {
  k_scatter_state<<<(n + 255) / 256, 256, 0, st>>>(n, ids, src, dst, nf);
}

}  // namespace lp
