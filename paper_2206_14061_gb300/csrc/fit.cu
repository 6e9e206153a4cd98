// GFD least-squares fits (Sec. 3.1 item 7), mu(I) closure (Sec. 2.2-2.3) and
// the explicit update (Sec. 3.1 items 8, 10).
//
// One thread per particle. A thread walks its stencil once, accumulating the
// 31 distinct moments of the Taylor rows (the 9x9 Gram matrix has only 31
// different entries) and the right-hand sides A^T b of all fields; it then
// factors the Gram matrix (Cholesky) and solves. Stencils whose Gram matrix is
// too ill-conditioned for the normal equations (relative pivot below the
// threshold, or fewer than 9 rows) are queued for a separate FP64 pivoted-QR
// kernel, the same algorithm the paper names (QR least squares).
//
// FP64 mode: everything in FP64. MIXED mode: moments, right-hand sides and the
// Cholesky factor in FP32 on the scaled, centred offsets, followed by one FP64
// refinement sweep (residual r = b - A c and A^T r in FP64, correction solved
// with the FP32 factor).
//
// Time levels of one step: pass 1 fits u, v, w at time n and sets
// V^{n+1} = V^n + dt V^n div u^n; pass 2 fits |gdot|^n and V^{n+1} and forms
// the acceleration with V^{n+1}, its gradient and phi^{n+1} = 1/V^{n+1}.
#include "fit_bodies.cuh"

namespace lp {

// ------------------------------------------------------------ pass 1

// ------------------------------------------------------------ pass 2

// ------------------------------------------------------------ kernels

template <int PREC, bool PER>
__global__ void __launch_bounds__(kMaxBlock) k_pass1(const StepArgs A) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < A.n) pass1_body<PREC, PER>(A, s);
}

// pivoted-QR fallback of pass 1 (grid-stride over the queued particles)
__global__ void __launch_bounds__(64) k_pass1_fallback(const StepArgs A) {
  const int cnt = min(*A.fb_count, A.fb_cap);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x)
    pass1_fallback_item(A, t);
  if (blockIdx.x == 0 && threadIdx.x == 0 && cnt > 0)
    atomicAdd(&A.dg->n_fallback, (unsigned long long)cnt);
}

// pivoted-QR fallback of pass 2: gradients of |gdot|^n and V^{n+1}
__global__ void __launch_bounds__(64) k_pass2_fallback(const StepArgs A) {
  const int cnt = min(*A.fb_count, A.fb_cap);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x)
    pass2_fallback_item(A, t);
}

// float-float kernels: 128 threads per block, at most 128 registers so that
// 4 blocks (16 warps) share an SM
constexpr int kFFBlock = 128;
// Fit threads take the particles of each group of kRowGroup in order of
// stencil size: a warp's lanes then have similar row counts and fewer idle
// at the end of the row loops. perm[g kRowGroup + t] is the particle of rank
// t in group g by (rows, index); the arithmetic of each particle is
// unchanged, only the thread that does it.
#ifndef LP_ROW_GROUP
#define LP_ROW_GROUP 128
#endif
#ifndef LP_PASS2_BLOCKS
#define LP_PASS2_BLOCKS 4
#endif
constexpr int kRowGroup = LP_ROW_GROUP;
__global__ void __launch_bounds__(kRowGroup) k_row_order(int n, const int32_t* __restrict__ cnt,
                                                         int32_t* __restrict__ perm) {
  __shared__ uint32_t key[kRowGroup];
  const int base = blockIdx.x * kRowGroup, t = threadIdx.x, s = base + t;
  key[t] = s < n ? ((uint32_t)min(max(cnt[s], 0), 0xffff) << 16) | (uint32_t)t : 0xffffffffu;
  __syncthreads();
  // bitonic sort of the 128 keys, ascending (past-the-end keys sort last)
  for (int k = 2; k <= kRowGroup; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int p = t ^ j;
      if (p > t) {
        const uint32_t a = key[t], b = key[p];
        if ((a > b) == ((t & k) == 0)) {
          key[t] = b;
          key[p] = a;
        }
      }
      __syncthreads();
    }
  if (s < n) perm[s] = base + (int)(key[t] & 0xffffu);
}
__device__ __forceinline__ int fit_particle(const StepArgs& A) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  return (A.perm && t < A.n) ? A.perm[t] : t;
}

// (PER: periodic axes, offsets take their nearest image)
template <bool PER>
__global__ void __launch_bounds__(kFFBlock, 4) k_gram_ff(const StepArgs A) {
  const int s = fit_particle(A);
  if (s < A.n) gram_ff_body<PER>(A, s);
}

template <bool PER>
__global__ void __launch_bounds__(kFFBlock, 4) k_pass1_ff_rows(const StepArgs A) {
  const int s = fit_particle(A);
  if (s < A.n) pass1_ff_rows_body<PER>(A, s);
}
__global__ void __launch_bounds__(kFFBlock) k_pass1_ff_solve(const StepArgs A) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < A.n) pass1_ff_solve_body(A, s);
}

__global__ void k_split_state(const StepArgs A) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < A.n) split_state_body(A, s);
}

// rows of the entries with a ghost (free surface), ahead of the main kernels:
// a fixed grid strides over the list of particles that have such entries
// (only they have work), so that a warp's lanes are all busy
constexpr int kTwinBlocks = 4 * 152;
template <bool PER>
__global__ void k_gram_twins(const StepArgs A) {
  const int cnt = min(*A.gcount, A.n);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x)
    gram_twins_body<PER>(A, A.glist[t]);
}
template <bool PER>
__global__ void k_pass2_twins(const StepArgs A) {
  const int cnt = min(*A.gcount, A.n);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x)
    pass2_twins_body<PER>(A, A.glist[t]);
}

__global__ void k_split_p1(const StepArgs A) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < A.n) split_p1_body(A, s);
}

template <int PREC, bool PER>
__global__ void __launch_bounds__(kMaxBlock) k_pass2(const StepArgs A) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  pass2_body<PREC, PER>(A, s, s < A.n);
}

template <bool PER>
__global__ void __launch_bounds__(kFFBlock, LP_PASS2_BLOCKS) k_pass2_ff(const StepArgs A) {
  const int s = fit_particle(A);
  pass2_body<LP_MIXED_FF, PER>(A, s, s < A.n);
}

// ------------------------------------------------ lp_fit_derivatives

__device__ __forceinline__ void write_coeffs(const FitArgs& F, int s, int f, const double* c) {
  const double ih = F.inv_h, ih2 = ih * ih;
  double* o = F.coeffs + ((int64_t)s * F.nf + f) * kNB;
#pragma unroll
  for (int q = 0; q < kNB; ++q) o[q] = c[q] * (q < 3 ? ih : ih2);
}

// fields are processed in groups of 4 right-hand sides per sweep
template <int PREC>
__global__ void __launch_bounds__(kBlock) k_fit(const FitArgs F) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= F.n) return;
  const int n = F.n;
  const int m = min(F.cnt[s], F.cap);
  const double xi = F.x[s], yi = F.y[s], zi = F.z[s];
  const double ih = F.inv_h;
  using T = typename std::conditional<PREC == LP_FP64, double, float>::type;
  Moments<T> M;
  M.zero();
  int rows = 0;  // entries with an index in range
  for (int k = 0; k < m; ++k) {
    const uint32_t code = (uint32_t)F.nbr[(int64_t)k * n + s];
    const int j = code & ~kMirrorBit;
    if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
    const double zj = (code >> 31) ? F.f2 - F.z[j] : F.z[j];
    M.add(T((F.x[j] - xi) * ih), T((F.y[j] - yi) * ih), T((zj - zi) * ih));
    ++rows;
  }
  T L[kTri];
  M.gram(L);
  const bool ok = chol9(L, PREC == LP_FP64 ? T(1e-9) : T(1e-4)) && rows >= kNB;
  if (!ok) {
    const int slot = atomicAdd(F.fb_count, 1);
    if (slot < F.fb_cap) F.fb_list[slot] = s;
    else atomicOr(&F.dg->flags, (unsigned)LP_FLAG_OVERFLOW);
    return;
  }
  for (int f0 = 0; f0 < F.nf; f0 += 4) {
    const int nf = min(4, F.nf - f0);
    T R[4][kNB];
    double si[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      si[f] = f < nf ? F.fields[f0 + f][s] : 0.0;
#pragma unroll
      for (int c = 0; c < kNB; ++c) R[f][c] = T(0);
    }
    for (int k = 0; k < m; ++k) {
      const uint32_t code = (uint32_t)F.nbr[(int64_t)k * n + s];
      const int j = code & ~kMirrorBit;
      if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
      const bool mir = code >> 31;
      const double zj = mir ? F.f2 - F.z[j] : F.z[j];
      T a[kNB];
      taylor_row(T((F.x[j] - xi) * ih), T((F.y[j] - yi) * ih), T((zj - zi) * ih), a);
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        if (f < nf) {
          double vj = F.fields[f0 + f][j];
          if (mir) vj *= F.msign[f0 + f];
          const T b = T(vj - si[f]);
#pragma unroll
          for (int c = 0; c < kNB; ++c) R[f][c] += b * a[c];
        }
      }
    }
    double c[4][kNB];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      chol9_solve(L, R[f]);
#pragma unroll
      for (int q = 0; q < kNB; ++q) c[f][q] = (double)R[f][q];
    }
    if (PREC == LP_MIXED) {
      // one FP64 refinement step
      double g[4][kNB];
#pragma unroll
      for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int q = 0; q < kNB; ++q) g[f][q] = 0.0;
      for (int k = 0; k < m; ++k) {
        const uint32_t code = (uint32_t)F.nbr[(int64_t)k * n + s];
        const int j = code & ~kMirrorBit;
        if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
        const bool mir = code >> 31;
        const double zj = mir ? F.f2 - F.z[j] : F.z[j];
        double a[kNB];
        taylor_row((F.x[j] - xi) * ih, (F.y[j] - yi) * ih, (zj - zi) * ih, a);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          if (f < nf) {
            double vj = F.fields[f0 + f][j];
            if (mir) vj *= F.msign[f0 + f];
            double r = vj - si[f];
#pragma unroll
            for (int q = 0; q < kNB; ++q) r -= a[q] * c[f][q];
#pragma unroll
            for (int q = 0; q < kNB; ++q) g[f][q] += a[q] * r;
          }
        }
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        chol9_solve(L, g[f]);
#pragma unroll
        for (int q = 0; q < kNB; ++q) c[f][q] += g[f][q];
      }
    }
    for (int f = 0; f < nf; ++f) write_coeffs(F, s, f0 + f, c[f]);
  }
}

// ---- lp_fit_derivatives in float-float (LP_MIXED_FF): positions relative
// to the first particle in units of h (with the floor-mirror height) and the
// fields are split once per particle; the moments, the Cholesky factor and
// the right-hand sides then run on FP32 pairs as in the step's pass 1, with
// the same pivot test and the same pivoted-QR fallback.
__global__ void k_fit_split_ff(const FitArgs F) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= F.n) return;
  const double ox = F.x[0], oy = F.y[0], oz = F.z[0], ih = F.inv_h;
  const ff fx = ff_of((F.x[s] - ox) * ih), fy = ff_of((F.y[s] - oy) * ih);
  const ff fz = ff_of((F.z[s] - oz) * ih), fm = ff_of((F.f2 - F.z[s] - oz) * ih);
  F.xs[s].xh = make_float4(fx.h, fy.h, fz.h, fm.h);
  F.xs[s].xl = make_float4(fx.l, fy.l, fz.l, fm.l);
  for (int f = 0; f < F.nf; ++f) {
    const ff v = ff_of(F.fields[f][s]);
    F.fs[(int64_t)f * F.n + s] = make_float2(v.h, v.l);
  }
}

__global__ void __launch_bounds__(128, 4) k_fit_gram_ff(const FitArgs F) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= F.n) return;
  const int n = F.n;
  const int m = min(F.cnt[s], F.cap);
  const float4 hi = F.xs[s].xh, lo = F.xs[s].xl;
  const StepConsts K0{};  // no periodic axes
  ff mo[31];
#pragma unroll
  for (int q = 0; q < 31; ++q) mo[q] = {0.f, 0.f};
  int rows = 0;  // entries with an index in range
  // the neighbour's position one row ahead, its stencil code two rows ahead
  float4 jh = make_float4(0.f, 0.f, 0.f, 0.f), jl = jh;
  auto fetch = [&](uint32_t code) {
    int j = code & ~kMirrorBit;
    if ((unsigned)j >= (unsigned)n) j = s;  // never read outside the arrays (row skipped)
    jh = F.xs[j].xh;
    jl = F.xs[j].xl;
  };
  uint32_t code = m > 0 ? (uint32_t)F.nbr[s] : 0u;
  uint32_t nxt = m > 1 ? (uint32_t)F.nbr[(int64_t)n + s] : 0u;
  if (m > 0) fetch(code);
  for (int k = 0; k < m; ++k) {
    const uint32_t c0 = code;
    const float4 h0 = jh, l0 = jl;
    if (k + 1 < m) {
      code = nxt;
      fetch(code);
      if (k + 2 < m) nxt = (uint32_t)F.nbr[(int64_t)(k + 2) * n + s];
    }
    const int j = c0 & ~kMirrorBit;
    if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
    ff_moments_add(mo, ff_row_of<false>(hi, lo, h0, l0, c0, K0));
    ++rows;
  }
  ff G[kTri];
  ff_gram_fo(mo, G);
#pragma unroll
  for (int k = 0; k < kTri; ++k) G[k] = ff_norm(G[k]);
  if (!(ff_chol9(G, 1e-4f) && rows >= kNB)) {
    const int slot = atomicAdd(F.fb_count, 1);
    if (slot < F.fb_cap) F.fb_list[slot] = s;
    else atomicOr(&F.dg->flags, (unsigned)LP_FLAG_OVERFLOW);
    F.lf[s] = make_float2(-1.f, 0.f);  // 1/L_00 > 0 for a factored stencil
    return;
  }
#pragma unroll
  for (int k = 0; k < kTri; ++k) F.lf[(int64_t)k * n + s] = make_float2(G[k].h, G[k].l);
}

// Right-hand sides and solves of the float-float fit for the field group
// f0 .. f0 + NG - 1 (one launch per group): the group's NG x 9 sums stay in
// registers, and the neighbour's position and field values are loaded one
// row ahead of the arithmetic (its stencil code two rows ahead), as in the
// step's row kernels.
// (NG = 2: a last group of an odd field count holds one field, and its second
// solve runs on zero sums; 3 blocks of 168 registers, as at 128 the sums spill)
template <int NG>
__global__ void __launch_bounds__(128, 3) k_fit_rhs_ff(const FitArgs F, int f0) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= F.n) return;
  if (!(F.lf[s].x > 0.f)) return;  // queued for the pivoted-QR fit
  const int n = F.n;
  const int m = min(F.cnt[s], F.cap);
  const int ng = min(NG, F.nf - f0);
  const float4 hi = F.xs[s].xh, lo = F.xs[s].xl;
  const StepConsts K0{};
  ff R[NG][kNB], si[NG];
  float sg[NG];
#pragma unroll
  for (int f = 0; f < NG; ++f) {
    const float2 v = f < ng ? F.fs[(int64_t)(f0 + f) * n + s] : make_float2(0.f, 0.f);
    si[f] = ff{v.x, v.y};
    sg[f] = f < ng ? (float)F.msign[f0 + f] : 0.f;
#pragma unroll
    for (int q = 0; q < kNB; ++q) R[f][q] = {0.f, 0.f};
  }
  float4 jh = make_float4(0.f, 0.f, 0.f, 0.f), jl = jh;
  float2 jv[NG];
  auto fetch = [&](uint32_t code) {
    int j = code & ~kMirrorBit;
    if ((unsigned)j >= (unsigned)n) j = s;  // never read outside the arrays (row skipped)
    jh = F.xs[j].xh;
    jl = F.xs[j].xl;
#pragma unroll
    for (int f = 0; f < NG; ++f)
      jv[f] = f < ng ? F.fs[(int64_t)(f0 + f) * n + j] : make_float2(0.f, 0.f);
  };
  uint32_t code = m > 0 ? (uint32_t)F.nbr[s] : 0u;
  uint32_t nxt = m > 1 ? (uint32_t)F.nbr[(int64_t)n + s] : 0u;
  if (m > 0) fetch(code);
  for (int k = 0; k < m; ++k) {
    const uint32_t c0 = code;
    const float4 h0 = jh, l0 = jl;
    float2 v0[NG];
#pragma unroll
    for (int f = 0; f < NG; ++f) v0[f] = jv[f];
    if (k + 1 < m) {
      code = nxt;
      fetch(code);
      if (k + 2 < m) nxt = (uint32_t)F.nbr[(int64_t)(k + 2) * n + s];
    }
    const int j = c0 & ~kMirrorBit;
    if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
    const bool mir = c0 >> 31;
    ff a[kNB];
    ff_taylor(ff_row_of<false>(hi, lo, h0, l0, c0, K0), a);
#pragma unroll
    for (int f = 0; f < NG; ++f) {
      if (f < ng) {
        const float sj = mir ? sg[f] : 1.f;  // the field at a floor mirror
        const ff b = ff_diff(sj * v0[f].x, sj * v0[f].y, si[f].h, si[f].l);
#pragma unroll
        for (int q = 0; q < kNB; ++q) ff_acc(R[f][q], b, a[q]);
      }
    }
  }
  // one field at a time: the joint solve of a 2-D array of sums makes the
  // compiler keep them in local memory
  ff_chol_solve<1>(F.lf + s, n, R + 0);
  if (NG > 1) ff_chol_solve<1>(F.lf + s, n, R + 1);
  const double ih = F.inv_h, ih2 = ih * ih;
#pragma unroll
  for (int f = 0; f < NG; ++f) {
    if (f < ng) {
      double* o = F.coeffs + ((int64_t)s * F.nf + f0 + f) * kNB;
#pragma unroll
      for (int q = 0; q < kNB; ++q) o[q] = ff_to_double(R[f][q]) * (q < 3 ? ih : ih2);
    }
  }
}

__global__ void __launch_bounds__(64) k_fit_fallback(const FitArgs F) {
  const int cnt = min(*F.fb_count, F.fb_cap);
  double Am[LP_MAX_CAP * kNB], Bm[LP_MAX_CAP * 4], C[4 * kNB], Acopy[LP_MAX_CAP * kNB];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
    const int s = F.fb_list[t];
    const int n = F.n;
    const int m = min(F.cnt[s], F.cap);
    const double xi = F.x[s], yi = F.y[s], zi = F.z[s];
    // rows are packed: an entry whose index is out of range is dropped, as in
    // the Cholesky path, and the rows after it move up
    int rows = 0;
    for (int k = 0; k < m; ++k) {
      const uint32_t code = (uint32_t)F.nbr[(int64_t)k * n + s];
      const int j = code & ~kMirrorBit;
      if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
      const double zj = (code >> 31) ? F.f2 - F.z[j] : F.z[j];
      taylor_row((F.x[j] - xi) * F.inv_h, (F.y[j] - yi) * F.inv_h, (zj - zi) * F.inv_h,
                 &Acopy[rows * kNB]);
      ++rows;
    }
    for (int f0 = 0; f0 < F.nf; f0 += 4) {
      const int nf = min(4, F.nf - f0);
      int r = 0;
      for (int k = 0; k < m; ++k) {
        const uint32_t code = (uint32_t)F.nbr[(int64_t)k * n + s];
        const int j = code & ~kMirrorBit;
        if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
        const bool mir = code >> 31;
        for (int q = 0; q < kNB; ++q) Am[r * kNB + q] = Acopy[r * kNB + q];
        for (int f = 0; f < nf; ++f) {
          double vj = F.fields[f0 + f][j];
          if (mir) vj *= F.msign[f0 + f];
          Bm[r * nf + f] = vj - F.fields[f0 + f][s];
        }
        ++r;
      }
      qr_pivoted_solve(rows, Am, nf, Bm, C);
      for (int f = 0; f < nf; ++f) write_coeffs(F, s, f0 + f, C + f * kNB);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && cnt > 0)
    atomicAdd(&F.dg->n_fallback, (unsigned long long)cnt);
}

// ---------------------------------------------------------- lp_mui_stress

__global__ void k_mui_stress(int64_t n, ColMui mui, double phi_c, double phi_min,
                             double phi_max, double alpha, double beta,
                             const double* __restrict__ V, const double* __restrict__ gu,
                             double* gdot, double* gnorm, double* P, double* eta,
                             int8_t* regime) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* G = gu + 9 * i;
  const double div = (G[0] + G[4]) + G[8];
  const double d3 = div * (1.0 / 3.0);
  const double gxx = G[0] - d3, gyy = G[4] - d3, gzz = G[8] - d3;
  const double gxy = 0.5 * (G[1] + G[3]), gxz = 0.5 * (G[2] + G[6]), gyz = 0.5 * (G[5] + G[7]);
  const double gn =
      sqrt(0.5 * (gxx * gxx + gyy * gyy + gzz * gzz + 2.0 * (gxy * gxy + gxz * gxz + gyz * gyz)));
  if (gdot) {
    double* o = gdot + 6 * i;
    o[0] = gxx; o[1] = gyy; o[2] = gzz; o[3] = gxy; o[4] = gxz; o[5] = gyz;
  }
  if (gnorm) gnorm[i] = gn;
  const double phi = 1.0 / V[i];
  double p, e;
  int r;
  if (phi <= phi_min) {
    r = 0; p = 0.0; e = 0.0;
  } else if (phi <= phi_max) {
    r = 1;
    const double a = phi_c - phi_min;
    const double q = (2.0 * a * mui.d * gn) / (phi_c - phi);
    p = mui.rho_s * q * q;
    const Closure cl = closure_at(phi, mui, phi_c, phi_min);
    e = mui.rho_s * cl.N * gn;  // mu(I) P / |gdot|
  } else {
    r = 2; p = mui.rho_s * (alpha + beta * phi); e = 0.0;
  }
  if (P) P[i] = p;
  if (eta) eta[i] = e;
  if (regime) regime[i] = (int8_t)r;
}

// ------------------------------------------------------------- launchers

void launch_pass1(int prec, const StepArgs& A, cudaStream_t st, int bs) {
  const int nb = (A.n + bs - 1) / bs;
  const bool per = A.K.periodic != 0;
  if (prec == LP_FP64) {
    if (per) k_pass1<LP_FP64, true><<<nb, bs, 0, st>>>(A);
    else k_pass1<LP_FP64, false><<<nb, bs, 0, st>>>(A);
  } else if (prec == LP_MIXED) {
    if (per) k_pass1<LP_MIXED, true><<<nb, bs, 0, st>>>(A);
    else k_pass1<LP_MIXED, false><<<nb, bs, 0, st>>>(A);
  } else {
    k_split_state<<<(A.n + 255) / 256, 256, 0, st>>>(A);
    if (A.perm) k_row_order<<<(A.n + kRowGroup - 1) / kRowGroup, kRowGroup, 0, st>>>(A.n, A.cnt, const_cast<int32_t*>(A.perm));
    const int b = bs < kFFBlock ? bs : kFFBlock;
    const int nf = (A.n + b - 1) / b;
    if (per) {
      if (A.K.free_surface) k_gram_twins<true><<<kTwinBlocks, 128, 0, st>>>(A);
      k_gram_ff<true><<<nf, b, 0, st>>>(A);
      k_pass1_ff_rows<true><<<nf, b, 0, st>>>(A);
    } else {
      if (A.K.free_surface) k_gram_twins<false><<<kTwinBlocks, 128, 0, st>>>(A);
      k_gram_ff<false><<<nf, b, 0, st>>>(A);
      k_pass1_ff_rows<false><<<nf, b, 0, st>>>(A);
    }
    k_pass1_ff_solve<<<(A.n + kFFBlock - 1) / kFFBlock, kFFBlock, 0, st>>>(A);
  }
  k_pass1_fallback<<<152, 64, 0, st>>>(A);
}
void launch_pass2(int prec, const StepArgs& A, cudaStream_t st, int bs) {
  if (prec == LP_MIXED_FF) {
    k_split_p1<<<(A.n + 255) / 256, 256, 0, st>>>(A);
    if (A.K.free_surface) {
      if (A.K.periodic) k_pass2_twins<true><<<kTwinBlocks, 128, 0, st>>>(A);
      else k_pass2_twins<false><<<kTwinBlocks, 128, 0, st>>>(A);
    }
  }
  k_pass2_fallback<<<152, 64, 0, st>>>(A);
  const int nb = (A.n + bs - 1) / bs;
  const bool per = A.K.periodic != 0;
  if (prec == LP_FP64) {
    if (per) k_pass2<LP_FP64, true><<<nb, bs, 0, st>>>(A);
    else k_pass2<LP_FP64, false><<<nb, bs, 0, st>>>(A);
  } else if (prec == LP_MIXED) {
    if (per) k_pass2<LP_MIXED, true><<<nb, bs, 0, st>>>(A);
    else k_pass2<LP_MIXED, false><<<nb, bs, 0, st>>>(A);
  } else {
    const int b = bs < kFFBlock ? bs : kFFBlock;
    if (per) k_pass2_ff<true><<<(A.n + b - 1) / b, b, 0, st>>>(A);
    else k_pass2_ff<false><<<(A.n + b - 1) / b, b, 0, st>>>(A);
  }
}
void launch_fit(int prec, const FitArgs& F, cudaStream_t st) {
  const int nb = (F.n + kBlock - 1) / kBlock;
  if (prec == LP_FP64) {
    k_fit<LP_FP64><<<nb, kBlock, 0, st>>>(F);
  } else if (prec == LP_MIXED) {
    k_fit<LP_MIXED><<<nb, kBlock, 0, st>>>(F);
  } else {
    const int nf = (F.n + 127) / 128;
    k_fit_split_ff<<<(F.n + 255) / 256, 256, 0, st>>>(F);
    k_fit_gram_ff<<<nf, 128, 0, st>>>(F);
    for (int f0 = 0; f0 < F.nf; f0 += 2) k_fit_rhs_ff<2><<<nf, 128, 0, st>>>(F, f0);
  }
  k_fit_fallback<<<152, 64, 0, st>>>(F);
}
void launch_mui_stress(int64_t n, const ColMui& m, const lp_eos& e, const double* V,
                       const double* gu, double* gdot, double* gnorm, double* P, double* eta,
                       int8_t* regime, cudaStream_t st) {
  k_mui_stress<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, m, e.phi_c, e.phi_min, e.phi_max,
                                                            e.alpha, e.beta, V, gu, gdot, gnorm,
                                                            P, eta, regime);
}

}  // namespace lp
