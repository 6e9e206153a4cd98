// Device bodies of the two fit passes and the update, shared by the per-phase
// kernels (fit.cu) and the persistent step kernel (persistent.cu). See
// fit.cu for the method.
#pragma once

#include "lp_internal.cuh"

namespace lp {

// mirror velocity factor of component a
__device__ __forceinline__ double usign(int mode, int a) {
  return mode == LP_MIRROR_NOSLIP ? -1.0 : (mode == LP_MIRROR_FREESLIP && a == 2 ? -1.0 : 1.0);
}

// Quantities of Sec. 2.2 from the fitted coefficients of u, v, w (h-scaled):
// gdot, |gdot|, div u, (1/2) Lap u + (1/6) grad div u, and V^{n+1}.
__device__ __forceinline__ void pass1_finish(const StepArgs& A, int s, const double (*c)[kNB]) {
  const int n = A.n;
  const double ih = A.K.inv_h, ih2 = ih * ih;
  double G[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) G[a][b] = c[a][b] * ih;
  const double div = (G[0][0] + G[1][1]) + G[2][2];
  const double d3 = div * (1.0 / 3.0);
  const double gxx = G[0][0] - d3, gyy = G[1][1] - d3, gzz = G[2][2] - d3;
  const double gxy = 0.5 * (G[0][1] + G[1][0]);
  const double gxz = 0.5 * (G[0][2] + G[2][0]);
  const double gyz = 0.5 * (G[1][2] + G[2][1]);
  const double ss = gxx * gxx + gyy * gyy + gzz * gzz + 2.0 * (gxy * gxy + gxz * gxz + gyz * gyz);
  double* p = A.p1;
  p[(P1_GD + 0) * n + s] = gxx; p[(P1_GD + 1) * n + s] = gyy; p[(P1_GD + 2) * n + s] = gzz;
  p[(P1_GD + 3) * n + s] = gxy; p[(P1_GD + 4) * n + s] = gxz; p[(P1_GD + 5) * n + s] = gyz;
  p[P1_GN * n + s] = sqrt(0.5 * ss);
  // Hessian columns: 3 xx, 4 yy, 5 zz, 6 xy, 7 xz, 8 yz
  double lap[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) lap[a] = (c[a][3] + c[a][4]) + c[a][5];
  const double ddx = (c[0][3] + c[1][6]) + c[2][7];
  const double ddy = (c[0][6] + c[1][4]) + c[2][8];
  const double ddz = (c[0][7] + c[1][8]) + c[2][5];
  p[(P1_LD + 0) * n + s] = (0.5 * lap[0] + ddx * (1.0 / 6.0)) * ih2;
  p[(P1_LD + 1) * n + s] = (0.5 * lap[1] + ddy * (1.0 / 6.0)) * ih2;
  p[(P1_LD + 2) * n + s] = (0.5 * lap[2] + ddz * (1.0 / 6.0)) * ih2;
  const double Vi = A.V[s];
  p[P1_VN * n + s] = Vi + A.K.dt * (Vi * div);
  p[P1_DIV * n + s] = div;
}

__device__ __forceinline__ void push_fallback(const StepArgs& A, int s) {
  const int slot = atomicAdd(A.fb_count, 1);
  if (slot < A.fb_cap) {
    A.fb_list[slot] = s;
    A.fbslot[s] = slot;
  } else {
    A.fbslot[s] = -2;  // no room: reported as a timeout-free overflow
    atomicOr(&A.dg->flags, (unsigned)LP_FLAG_OVERFLOW);
  }
}

// Right-hand sides of a ghost row in pass 2 (free boundary, Sec. 3.1 item 9):
// |gdot|_G - |gdot|_s and V_G - V_s^{n+1}, with |gdot|_G = |gdot|_s (phi_c -
// phi_G) / (phi_c - phi_s) in the inertial regime (inertial pressure
// continuous), |gdot|_s otherwise; phi_s = 1 / V_s^{n+1}.
__device__ __forceinline__ void ghost_rhs2(const StepArgs& A, double gni, double Vi, double* bg,
                                           double* bv) {
  const double phi = 1.0 / Vi;
  const bool inertial = phi > A.K.phi_min && phi <= A.K.phi_max;
  const double gng = inertial ? gni * (A.K.ghost_num / (A.K.phi_c - phi)) : gni;
  *bg = gng - gni;
  *bv = A.K.ghost_V - Vi;
}

// ------------------------------------------------------------ pass 1

template <bool PER>
__device__ __forceinline__ void pass1_ff_body(const StepArgs& A, int s);

// PER: periodic axes (offsets take their nearest image); without it the
// periods are not read
template <bool PER>
__device__ __forceinline__ double per_off(double d, double L) {
  return PER ? min_image(d, L) : d;
}
template <int PREC, bool PER = false>
__device__ __forceinline__ void pass1_body(const StepArgs& A, int s) {
  if (PREC == LP_MIXED_FF) {
    pass1_ff_body<PER>(A, s);
    return;
  }
  const int n = A.n;
  const int m = min(A.cnt[s], A.cap);
  const double xi = A.x[s], yi = A.y[s], zi = A.z[s];
  const double ui = A.u[s], vi = A.v[s], wi = A.w[s];
  const double ih = A.K.inv_h, f2 = 2.0 * A.K.floor_z;
  const int mm = A.K.mirror_mode;
  const double su = usign(mm, 0), sv = usign(mm, 1), sw = usign(mm, 2);

  if (PREC == LP_FP64) {
    Moments<double> M;
    M.zero();
    double R[3][kNB];
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
      for (int c = 0; c < kNB; ++c) R[f][c] = 0.0;
    for (int k = 0; k < m; ++k) {
      const uint32_t code = (uint32_t)A.nbr[(int64_t)k * n + s];
      const int j = code & kIndexMask;
      if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
      const bool mir = code >> 31;
      const double zj = mir ? f2 - A.z[j] : A.z[j];
      const double dx = per_off<PER>(A.x[j] - xi, A.K.Lx) * ih;
      const double dy = per_off<PER>(A.y[j] - yi, A.K.Ly) * ih, dz = (zj - zi) * ih;
      if (code & kGhostBit) M.add(-dx, -dy, -dz);  // its ghost: reflected row, b = 0
      double uj = A.u[j], vj = A.v[j], wj = A.w[j];
      if (mir) { uj *= su; vj *= sv; wj *= sw; }
      M.add(dx, dy, dz);
      double a[kNB];
      taylor_row(dx, dy, dz, a);
      const double b[3] = {uj - ui, vj - vi, wj - wi};
#pragma unroll
      for (int f = 0; f < 3; ++f)
#pragma unroll
        for (int c = 0; c < kNB; ++c) R[f][c] += b[f] * a[c];
    }
    double L[kTri];
    M.gram(L);
    const bool ok = chol9(L, 1e-9) && m >= kNB;
    if (!ok) {
      push_fallback(A, s);
      return;
    }
    A.fbslot[s] = -1;
#pragma unroll
    for (int k = 0; k < kTri; ++k) A.fac[(int64_t)k * n + s] = L[k];
#pragma unroll
    for (int f = 0; f < 3; ++f) chol9_solve(L, R[f]);
    if (A.coef1) {
#pragma unroll
      for (int f = 0; f < 3; ++f)
#pragma unroll
        for (int q = 0; q < kNB; ++q) A.coef1[(int64_t)(f * kNB + q) * n + s] = R[f][q];
    }
    pass1_finish(A, s, R);
  } else {
    // FP32 moments on the scaled offsets
    Moments<float> M;
    M.zero();
    float Rf[3][kNB];
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
      for (int c = 0; c < kNB; ++c) Rf[f][c] = 0.f;
    for (int k = 0; k < m; ++k) {
      const uint32_t code = (uint32_t)A.nbr[(int64_t)k * n + s];
      const int j = code & kIndexMask;
      if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
      const bool mir = code >> 31;
      const double zj = mir ? f2 - A.z[j] : A.z[j];
      const float dx = (float)(per_off<PER>(A.x[j] - xi, A.K.Lx) * ih);
      const float dy = (float)(per_off<PER>(A.y[j] - yi, A.K.Ly) * ih);
      const float dz = (float)((zj - zi) * ih);
      if (code & kGhostBit) M.add(-dx, -dy, -dz);  // its ghost: reflected row, b = 0
      double uj = A.u[j], vj = A.v[j], wj = A.w[j];
      if (mir) { uj *= su; vj *= sv; wj *= sw; }
      M.add(dx, dy, dz);
      float a[kNB];
      taylor_row(dx, dy, dz, a);
      const float b[3] = {(float)(uj - ui), (float)(vj - vi), (float)(wj - wi)};
#pragma unroll
      for (int f = 0; f < 3; ++f)
#pragma unroll
        for (int c = 0; c < kNB; ++c) Rf[f][c] += b[f] * a[c];
    }
    float L[kTri];
    M.gram(L);
    const bool ok = chol9(L, 1e-4f) && m >= kNB;
    if (!ok) {
      push_fallback(A, s);
      return;
    }
    A.fbslot[s] = -1;
#pragma unroll
    for (int k = 0; k < kTri; ++k) A.facf[(int64_t)k * n + s] = L[k];
    double c[3][kNB];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      chol9_solve(L, Rf[f]);
#pragma unroll
      for (int q = 0; q < kNB; ++q) c[f][q] = (double)Rf[f][q];
    }
    // one FP64 refinement step: g = A^T (b - A c), c += G^{-1} g
    double g[3][kNB];
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
      for (int q = 0; q < kNB; ++q) g[f][q] = 0.0;
    for (int k = 0; k < m; ++k) {
      const uint32_t code = (uint32_t)A.nbr[(int64_t)k * n + s];
      const int j = code & kIndexMask;
      if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
      const bool mir = code >> 31;
      const double zj = mir ? f2 - A.z[j] : A.z[j];
      const double dx = per_off<PER>(A.x[j] - xi, A.K.Lx) * ih;
      const double dy = per_off<PER>(A.y[j] - yi, A.K.Ly) * ih, dz = (zj - zi) * ih;
      double uj = A.u[j], vj = A.v[j], wj = A.w[j];
      if (mir) { uj *= su; vj *= sv; wj *= sw; }
      // the entry's row, then (flagged entries) its ghost: reflected row, b = 0
      for (int t = 0; t < ((code & kGhostBit) ? 2 : 1); ++t) {
        const double rs = t ? -1.0 : 1.0;
        double a[kNB];
        taylor_row(rs * dx, rs * dy, rs * dz, a);
        const double b[3] = {t ? 0.0 : uj - ui, t ? 0.0 : vj - vi, t ? 0.0 : wj - wi};
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          double r = b[f];
#pragma unroll
          for (int q = 0; q < kNB; ++q) r -= a[q] * c[f][q];
#pragma unroll
          for (int q = 0; q < kNB; ++q) g[f][q] += a[q] * r;
        }
      }
    }
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      chol9_solve(L, g[f]);
#pragma unroll
      for (int q = 0; q < kNB; ++q) c[f][q] += g[f][q];
    }
    pass1_finish(A, s, c);
  }
}

// pivoted-QR fallback of pass 1 (grid-stride over the queued particles)
static __device__ __noinline__ void pass1_fallback_item(const StepArgs& A, int t) {
  double Am[LP_MAX_CAP * kNB], Bm[LP_MAX_CAP * 3], C[3 * kNB];
  {
    const int s = A.fb_list[t];
    const int n = A.n;
    const int m = min(A.cnt[s], A.cap);
    const double xi = A.x[s], yi = A.y[s], zi = A.z[s];
    const double ui = A.u[s], vi = A.v[s], wi = A.w[s];
    const double ih = A.K.inv_h, f2 = 2.0 * A.K.floor_z;
    const int mm = A.K.mirror_mode;
    int rows = 0;  // a flagged entry adds its ghost: reflected row, b = 0
    for (int k = 0; k < m; ++k) {
      const uint32_t code = (uint32_t)A.nbr[(int64_t)k * n + s];
      const int j = code & kIndexMask;
      if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
      const bool mir = code >> 31;
      const double zj = mir ? f2 - A.z[j] : A.z[j];
      const double dx = min_image(A.x[j] - xi, A.K.Lx) * ih;
      const double dy = min_image(A.y[j] - yi, A.K.Ly) * ih, dz = (zj - zi) * ih;
      double uj = A.u[j], vj = A.v[j], wj = A.w[j];
      if (mir) { uj *= usign(mm, 0); vj *= usign(mm, 1); wj *= usign(mm, 2); }
      for (int t = 0; t < ((code & kGhostBit) ? 2 : 1) && rows < LP_MAX_CAP; ++t, ++rows) {
        const double rs = t ? -1.0 : 1.0;
        taylor_row(rs * dx, rs * dy, rs * dz, &Am[rows * kNB]);
        Bm[rows * 3 + 0] = t ? 0.0 : uj - ui;
        Bm[rows * 3 + 1] = t ? 0.0 : vj - vi;
        Bm[rows * 3 + 2] = t ? 0.0 : wj - wi;
      }
    }
    qr_pivoted_solve(rows, Am, 3, Bm, C);
    double c[3][kNB];
    for (int f = 0; f < 3; ++f)
      for (int q = 0; q < kNB; ++q) c[f][q] = C[f * kNB + q];
    if (A.coef1)
      for (int f = 0; f < 3; ++f)
        for (int q = 0; q < kNB; ++q) A.coef1[(int64_t)(f * kNB + q) * n + s] = c[f][q];
    pass1_finish(A, s, c);
  }
}

// pivoted-QR fallback of pass 2: gradients of |gdot|^n and V^{n+1}
static __device__ __noinline__ void pass2_fallback_item(const StepArgs& A, int t) {
  double Am[LP_MAX_CAP * kNB], Bm[LP_MAX_CAP * 2], C[2 * kNB];
  {
    const int s = A.fb_list[t];
    const int n = A.n;
    const int m = min(A.cnt[s], A.cap);
    const double xi = A.x[s], yi = A.y[s], zi = A.z[s];
    const double ih = A.K.inv_h, f2 = 2.0 * A.K.floor_z;
    const double* gn = A.p1 + P1_GN * n;
    const double* Vn = A.K.euler ? A.V : A.p1 + P1_VN * n;  // V of the pass-2 fit
    double bg_gh = 0.0, bv_gh = 0.0;
    if (A.K.free_surface) ghost_rhs2(A, gn[s], Vn[s], &bg_gh, &bv_gh);
    int rows = 0;  // a flagged entry adds its ghost: reflected row
    for (int k = 0; k < m; ++k) {
      const uint32_t code = (uint32_t)A.nbr[(int64_t)k * n + s];
      const int j = code & kIndexMask;
      if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
      const bool mir = code >> 31;
      const double zj = mir ? f2 - A.z[j] : A.z[j];
      const double dx = min_image(A.x[j] - xi, A.K.Lx) * ih;
      const double dy = min_image(A.y[j] - yi, A.K.Ly) * ih, dz = (zj - zi) * ih;
      for (int t = 0; t < ((code & kGhostBit) ? 2 : 1) && rows < LP_MAX_CAP; ++t, ++rows) {
        const double rs = t ? -1.0 : 1.0;
        taylor_row(rs * dx, rs * dy, rs * dz, &Am[rows * kNB]);
        Bm[rows * 2 + 0] = t ? bg_gh : (mir ? 0.0 : gn[j]) - gn[s];
        Bm[rows * 2 + 1] = t ? bv_gh : Vn[j] - Vn[s];
      }
    }
    qr_pivoted_solve(rows, Am, 2, Bm, C);
    if (A.coef2)
      for (int q = 0; q < 2 * kNB; ++q) A.coef2[(int64_t)q * n + s] = C[q];
    for (int q = 0; q < 3; ++q) {
      A.fbgrad[6 * t + q] = C[q] * ih;
      A.fbgrad[6 * t + 3 + q] = C[kNB + q] * ih;
    }
  }
}

// ------------------------------------------------------ float-float mode
// LP_MIXED_FF: nothing on a stencil row touches the FP64 pipe. Positions are
// scaled and split once per particle and step (X = (x - origin)/h as hi + lo
// floats, with the floor-mirror height in w), velocities likewise; each row's
// offsets, Taylor terms, the 31 moments and the right-hand sides are carried as
// float-float. The Gram matrix is factored once per particle and step in
// float-float (Cholesky, own kernel: positions and stencil only) and both
// passes solve with that factor in float-float, so the coefficients carry
// about 2^-44 cond(G) relative error, the accuracy of the float-float G.

// scaled, split positions and velocities of the current state
// (StepArgs, or the adjoint's AdjArgs for the step it differentiates)
template <class Args>
__device__ __forceinline__ void split_state_body(const Args& A, int s) {
  const GridCol g = A.grids[A.colid[s]];
  const double ih = A.K.inv_h;
  const ff fx = ff_of((A.x[s] - g.ox) * ih), fy = ff_of((A.y[s] - g.oy) * ih);
  const ff fz = ff_of((A.z[s] - g.oz) * ih);
  const ff fm = ff_of((2.0 * A.K.floor_z - A.z[s] - g.oz) * ih);
  FF8 r;
  r.xh = make_float4(fx.h, fy.h, fz.h, fm.h);
  r.xl = make_float4(fx.l, fy.l, fz.l, fm.l);
  const ff fu = ff_of(A.u[s]), fv = ff_of(A.v[s]), fw = ff_of(A.w[s]);
  r.uh = make_float4(fu.h, fv.h, fw.h, 0.f);
  r.ul = make_float4(fu.l, fv.l, fw.l, 0.f);
  A.XU[s] = r;
}

// split |gdot|^n and V^{n+1} (pass-1 outputs, FP64) for pass 2
template <class Args>
__device__ __forceinline__ void split_p1_body(const Args& A, int s) {
  const ff g = ff_of(A.p1[P1_GN * A.n + s]);
  const ff v = ff_of(A.K.euler ? A.V[s] : A.p1[P1_VN * A.n + s]);  // V of the pass-2 fit
  A.XU[s].uh = make_float4(g.h, g.l, v.h, v.l);  // the velocity half is no longer read
}

// float-float offset between two split coordinates
__device__ __forceinline__ ff ff_diff(float jh, float jl, float ih_, float il) {
  const ff d = two_sum(jh, -ih_);
  return fast_two_sum(d.h, __fadd_rn(d.l, __fsub_rn(jl, il)));
}

// Taylor row of a float-float offset and its quadratic terms
struct FFRow {
  ff dx, dy, dz, qxx, qyy, qzz, qxy, qxz, qyz;
};
// split position of the neighbour named by a stencil code
__device__ __forceinline__ void ff_gather(const StepArgs& A, int s, uint32_t code, float4& jh,
                                          float4& jl) {
  int j = code & kIndexMask;
  if ((unsigned)j >= (unsigned)A.n) j = s;  // never read outside the arrays (zero row)
  jh = A.XU[j].xh;
  jl = A.XU[j].xl;
}
// offset along an axis of period Lh (units of h, float-float; Lh = 0: not
// periodic), taken as its nearest image
// (a branch taken only by pairs across the edge)
__device__ __forceinline__ ff ff_min_image(ff d, float Lh_h, float Lh_l) {
  if (Lh_h > 0.f && fabsf(d.h) > 0.5f * Lh_h) {
    const bool pos = d.h > 0.f;
    return ff_add(d, ff{pos ? -Lh_h : Lh_h, pos ? -Lh_l : Lh_l});
  }
  return d;
}
template <bool PER>
__device__ __forceinline__ FFRow ff_row_of(const float4& hi, const float4& lo, const float4& jh,
                                           const float4& jl, uint32_t code,
                                           const StepConsts& K) {
  const bool mir = code >> 31;
  FFRow r;
  r.dx = ff_diff(jh.x, jl.x, hi.x, lo.x);
  r.dy = ff_diff(jh.y, jl.y, hi.y, lo.y);
  if (PER) {
    r.dx = ff_min_image(r.dx, K.Lhx_h, K.Lhx_l);
    r.dy = ff_min_image(r.dy, K.Lhy_h, K.Lhy_l);
  }
  r.dz = mir ? ff_diff(jh.w, jl.w, hi.z, lo.z) : ff_diff(jh.z, jl.z, hi.z, lo.z);
  r.qxx = ff_mul(r.dx, r.dx); r.qyy = ff_mul(r.dy, r.dy); r.qzz = ff_mul(r.dz, r.dz);
  r.qxy = ff_mul(r.dx, r.dy); r.qxz = ff_mul(r.dx, r.dz); r.qyz = ff_mul(r.dy, r.dz);
  return r;
}
// Row of stencil entry `code` of particle s, gathered without pipelining.
template <bool PER>
__device__ __forceinline__ FFRow ff_entry_row(const StepArgs& A, int s, const float4& hi,
                                              const float4& lo, uint32_t code) {
  float4 jh, jl;
  ff_gather(A, s, code, jh, jl);
  return ff_row_of<PER>(hi, lo, jh, jl, code, A.K);
}
// Number of entries with a ghost (kGhostBit), at the end of the stencil of s.
__device__ __forceinline__ int ghost_count(const StepArgs& A, int s, int m) {
  return A.K.free_surface ? min(max(A.gcnt[s], 0), m) : 0;
}
__device__ __forceinline__ void ff_taylor(const FFRow& r, ff* a) {
  a[0] = r.dx; a[1] = r.dy; a[2] = r.dz;
  a[3] = ff_scale(r.qxx, 0.5f); a[4] = ff_scale(r.qyy, 0.5f); a[5] = ff_scale(r.qzz, 0.5f);
  a[6] = r.qxy; a[7] = r.qxz; a[8] = r.qyz;
}

// the 31 distinct Gram moments: deg 2 (0..5), deg 3 (6..15), deg 4 (16..30)
__device__ __forceinline__ void ff_moments_add(ff* mo, const FFRow& r) {
  ff_acc1(mo[0], r.qxx); ff_acc1(mo[1], r.qyy); ff_acc1(mo[2], r.qzz);
  ff_acc1(mo[3], r.qxy); ff_acc1(mo[4], r.qxz); ff_acc1(mo[5], r.qyz);
  ff_acc(mo[6], r.dx, r.qxx);  ff_acc(mo[7], r.dy, r.qyy);  ff_acc(mo[8], r.dz, r.qzz);
  ff_acc(mo[9], r.dy, r.qxx);  ff_acc(mo[10], r.dz, r.qxx); ff_acc(mo[11], r.dx, r.qyy);
  ff_acc(mo[12], r.dz, r.qyy); ff_acc(mo[13], r.dx, r.qzz); ff_acc(mo[14], r.dy, r.qzz);
  ff_acc(mo[15], r.dz, r.qxy);
  ff_acc(mo[16], r.qxx, r.qxx); ff_acc(mo[17], r.qyy, r.qyy); ff_acc(mo[18], r.qzz, r.qzz);
  ff_acc(mo[19], r.qxx, r.qxy); ff_acc(mo[20], r.qxx, r.qxz); ff_acc(mo[21], r.qyy, r.qxy);
  ff_acc(mo[22], r.qyy, r.qyz); ff_acc(mo[23], r.qzz, r.qxz); ff_acc(mo[24], r.qzz, r.qyz);
  ff_acc(mo[25], r.qxx, r.qyy); ff_acc(mo[26], r.qxx, r.qzz); ff_acc(mo[27], r.qyy, r.qzz);
  ff_acc(mo[28], r.qxx, r.qyz); ff_acc(mo[29], r.qyy, r.qxz); ff_acc(mo[30], r.qzz, r.qxy);
}

// Moments of an entry and its ghost (the entry reflected through the
// particle): the reflection flips the odd (degree-3) terms, so together they
// add the even moments twice and the odd ones not at all.
__device__ __forceinline__ void ff_moments_add_twin(ff* mo, const FFRow& r) {
  const ff xx2 = ff_scale(r.qxx, 2.f), yy2 = ff_scale(r.qyy, 2.f), zz2 = ff_scale(r.qzz, 2.f);
  ff_acc1(mo[0], xx2); ff_acc1(mo[1], yy2); ff_acc1(mo[2], zz2);
  ff_acc1(mo[3], ff_scale(r.qxy, 2.f)); ff_acc1(mo[4], ff_scale(r.qxz, 2.f));
  ff_acc1(mo[5], ff_scale(r.qyz, 2.f));
  ff_acc(mo[16], xx2, r.qxx); ff_acc(mo[17], yy2, r.qyy); ff_acc(mo[18], zz2, r.qzz);
  ff_acc(mo[19], xx2, r.qxy); ff_acc(mo[20], xx2, r.qxz); ff_acc(mo[21], yy2, r.qxy);
  ff_acc(mo[22], yy2, r.qyz); ff_acc(mo[23], zz2, r.qxz); ff_acc(mo[24], zz2, r.qyz);
  ff_acc(mo[25], xx2, r.qyy); ff_acc(mo[26], xx2, r.qzz); ff_acc(mo[27], yy2, r.qzz);
  ff_acc(mo[28], xx2, r.qyz); ff_acc(mo[29], yy2, r.qxz); ff_acc(mo[30], zz2, r.qxy);
}

// packed Gram matrix from the moments (same entries as Moments::gram)
// the same sums with the nine sums of terms that are never negative seeded
// (ff_acc_seeded; see gram_ff_body) and the signed ones in plain float-float
__device__ __forceinline__ void ff_moments_add_seeded(ff* mo, const FFRow& r) {
  ff_acc1_seeded(mo[0], r.qxx); ff_acc1_seeded(mo[1], r.qyy); ff_acc1_seeded(mo[2], r.qzz);
  ff_acc1(mo[3], r.qxy); ff_acc1(mo[4], r.qxz); ff_acc1(mo[5], r.qyz);
  ff_acc(mo[6], r.dx, r.qxx);  ff_acc(mo[7], r.dy, r.qyy);  ff_acc(mo[8], r.dz, r.qzz);
  ff_acc(mo[9], r.dy, r.qxx);  ff_acc(mo[10], r.dz, r.qxx); ff_acc(mo[11], r.dx, r.qyy);
  ff_acc(mo[12], r.dz, r.qyy); ff_acc(mo[13], r.dx, r.qzz); ff_acc(mo[14], r.dy, r.qzz);
  ff_acc(mo[15], r.dz, r.qxy);
  ff_acc_seeded(mo[16], r.qxx, r.qxx); ff_acc_seeded(mo[17], r.qyy, r.qyy);
  ff_acc_seeded(mo[18], r.qzz, r.qzz);
  ff_acc(mo[19], r.qxx, r.qxy); ff_acc(mo[20], r.qxx, r.qxz); ff_acc(mo[21], r.qyy, r.qxy);
  ff_acc(mo[22], r.qyy, r.qyz); ff_acc(mo[23], r.qzz, r.qxz); ff_acc(mo[24], r.qzz, r.qyz);
  ff_acc_seeded(mo[25], r.qxx, r.qyy); ff_acc_seeded(mo[26], r.qxx, r.qzz);
  ff_acc_seeded(mo[27], r.qyy, r.qzz);
  ff_acc(mo[28], r.qxx, r.qyz); ff_acc(mo[29], r.qyy, r.qxz); ff_acc(mo[30], r.qzz, r.qxy);
}
// degree (2, 3 or 4) of the monomial summed in moment q
__host__ __device__ constexpr int moment_degree(int q) { return q < 6 ? 2 : (q < 16 ? 3 : 4); }
// moments whose terms are never negative (dx^2, dy^2, dz^2, dx^4, dy^4, dz^4,
// dx^2 dy^2, dx^2 dz^2, dy^2 dz^2)
__host__ __device__ constexpr bool moment_nonneg(int q) {
  return q <= 2 || (q >= 16 && q <= 18) || (q >= 25 && q <= 27);
}
__device__ __forceinline__ void ff_gram(const ff* mo, ff* g) {
  const float h = 0.5f, q = 0.25f;
  g[tri(0, 0)] = mo[0];
  g[tri(1, 0)] = mo[3];               g[tri(1, 1)] = mo[1];
  g[tri(2, 0)] = mo[4];               g[tri(2, 1)] = mo[5];               g[tri(2, 2)] = mo[2];
  g[tri(3, 0)] = ff_scale(mo[6], h);  g[tri(3, 1)] = ff_scale(mo[9], h);  g[tri(3, 2)] = ff_scale(mo[10], h);
  g[tri(3, 3)] = ff_scale(mo[16], q);
  g[tri(4, 0)] = ff_scale(mo[11], h); g[tri(4, 1)] = ff_scale(mo[7], h);  g[tri(4, 2)] = ff_scale(mo[12], h);
  g[tri(4, 3)] = ff_scale(mo[25], q); g[tri(4, 4)] = ff_scale(mo[17], q);
  g[tri(5, 0)] = ff_scale(mo[13], h); g[tri(5, 1)] = ff_scale(mo[14], h); g[tri(5, 2)] = ff_scale(mo[8], h);
  g[tri(5, 3)] = ff_scale(mo[26], q); g[tri(5, 4)] = ff_scale(mo[27], q); g[tri(5, 5)] = ff_scale(mo[18], q);
  g[tri(6, 0)] = mo[9];               g[tri(6, 1)] = mo[11];              g[tri(6, 2)] = mo[15];
  g[tri(6, 3)] = ff_scale(mo[19], h); g[tri(6, 4)] = ff_scale(mo[21], h); g[tri(6, 5)] = ff_scale(mo[30], h);
  g[tri(6, 6)] = mo[25];
  g[tri(7, 0)] = mo[10];              g[tri(7, 1)] = mo[15];              g[tri(7, 2)] = mo[13];
  g[tri(7, 3)] = ff_scale(mo[20], h); g[tri(7, 4)] = ff_scale(mo[29], h); g[tri(7, 5)] = ff_scale(mo[23], h);
  g[tri(7, 6)] = mo[28];              g[tri(7, 7)] = mo[26];
  g[tri(8, 0)] = mo[15];              g[tri(8, 1)] = mo[12];              g[tri(8, 2)] = mo[14];
  g[tri(8, 3)] = ff_scale(mo[28], h); g[tri(8, 4)] = ff_scale(mo[22], h); g[tri(8, 5)] = ff_scale(mo[24], h);
  g[tri(8, 6)] = mo[29];              g[tri(8, 7)] = mo[30];              g[tri(8, 8)] = mo[27];
}

// Order of the unknowns in the float-float factor: the six second-derivative
// terms first, the gradient last (factor row i is unknown ff_unknown(i) of the
// column order above), so that a solve that needs only the gradient stops its
// back substitution after three rows.
__host__ __device__ constexpr int ff_unknown(int i) { return i < 6 ? i + 3 : i - 6; }

// packed Gram matrix in factor order
__device__ __forceinline__ void ff_gram_fo(const ff* mo, ff* g) {
  ff c[kTri];
  ff_gram(mo, c);
#pragma unroll
  for (int i = 0; i < kNB; ++i)
#pragma unroll
    for (int j = 0; j <= i; ++j) {
      const int a = ff_unknown(i), b = ff_unknown(j);
      g[tri(i, j)] = c[a >= b ? tri(a, b) : tri(b, a)];
    }
}

// In-place float-float Cholesky factor of a packed 9x9 Gram matrix (entries
// normalised): the strictly lower entries become L and the diagonal 1/L_jj.
// Same pivot test as chol9: the Schur complement of column j must stay above
// rel_tol times the original diagonal entry, else the stencil is too
// ill-conditioned for the normal equations.
__device__ __forceinline__ bool ff_chol9(ff* a, float rel_tol) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < kNB; ++j) {
    ff d = a[tri(j, j)];
    const float d0 = d.h;
#pragma unroll
    for (int k = 0; k < j; ++k) ff_acc(d, a[tri(j, k)], ff_neg(a[tri(j, k)]));
    d = ff_norm(d);
    const bool good = d.h > rel_tol * d0;
    ok = ok && good;
    const ff inv = good ? ff_rsqrt(d) : ff{0.f, 0.f};
    a[tri(j, j)] = inv;
#pragma unroll
    for (int i = j + 1; i < kNB; ++i) {
      ff s = a[tri(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) ff_acc(s, a[tri(i, k)], ff_neg(a[tri(j, k)]));
      a[tri(i, j)] = ff_mul(ff_norm(s), inv);
    }
  }
  return ok;
}

// Solve L L^T c = r for NF right-hand sides at once with the factor that
// gram_ff_body stored for particle s (unknowns in factor order; r and c in
// column order); each factor entry is loaded once per sweep and used for
// every right-hand side. r (unnormalised accumulators on entry) is
// overwritten by c; with GRAD_ONLY only c[0..2] (the gradient), the other
// entries are left holding intermediate values.
// (L: this particle's factor, entry k at L[k * n])
template <int NF, bool GRAD_ONLY = false>
__device__ __forceinline__ void ff_chol_solve(const float2* L, int64_t n, ff (*r)[kNB]) {
  // one 8-byte load per entry
  auto at = [&](int k) {
    const float2 v = L[k * n];
    return ff{v.x, v.y};
  };
#pragma unroll
  for (int i = 0; i < kNB; ++i) {
    const int qi = ff_unknown(i);
#pragma unroll
    for (int k = 0; k < i; ++k) {
      const ff l = at(tri(i, k));
#pragma unroll
      for (int f = 0; f < NF; ++f) ff_acc(r[f][qi], l, ff_neg(r[f][ff_unknown(k)]));
    }
    const ff inv = at(tri(i, i));
#pragma unroll
    for (int f = 0; f < NF; ++f) r[f][qi] = ff_mul(ff_norm(r[f][qi]), inv);
  }
#pragma unroll
  for (int i = kNB - 1; i >= (GRAD_ONLY ? kNB - 3 : 0); --i) {
    const int qi = ff_unknown(i);
#pragma unroll
    for (int k = i + 1; k < kNB; ++k) {
      const ff l = at(tri(k, i));
#pragma unroll
      for (int f = 0; f < NF; ++f) ff_acc(r[f][qi], l, ff_neg(r[f][ff_unknown(k)]));
    }
    const ff inv = at(tri(i, i));
#pragma unroll
    for (int f = 0; f < NF; ++f) r[f][qi] = ff_mul(ff_norm(r[f][qi]), inv);
  }
}

// Entries with a ghost sit at the end of the stencil (kGhostBit). Their rows
// are handled by the two bodies below, in kernels of their own, so that the
// main row loops keep their register allocation; the main bodies add the
// stored sums.

// Moments of the entries with a ghost together with their ghosts (even
// moments twice, odd ones cancel): Tg, 31 float-float, hi then lo, k-major.
template <bool PER>
__device__ __forceinline__ void gram_twins_body(const StepArgs& A, int s) {
  const int n = A.n;
  const int m = min(A.cnt[s], A.cap);
  const int mr = m - ghost_count(A, s, m);
  if (mr == m) return;
  const float4 hi = A.XU[s].xh, lo = A.XU[s].xl;
  ff t[31];
#pragma unroll
  for (int q = 0; q < 31; ++q) t[q] = {0.f, 0.f};
#pragma unroll 1
  for (int k = mr; k < m; ++k)
    ff_moments_add_twin(t, ff_entry_row<PER>(A, s, hi, lo, (uint32_t)A.nbr[(int64_t)k * n + s]));
#pragma unroll
  for (int q = 0; q < 31; ++q) {
    const ff v = ff_norm(t[q]);
    A.Tg[(int64_t)q * n + s] = v.h;
    A.Tg[(int64_t)(31 + q) * n + s] = v.l;
  }
}

// Pass-2 right-hand-side terms of the entries with a ghost and their ghosts
// (reflected row, right-hand sides fixed by the particle): b_j a + b_G a~,
// a~ the row with its linear terms negated. T2: 2 x 9 float-float, hi then
// lo, k-major. Needs the pass-1 outputs and their split copy (XU[].uh).
template <bool PER>
__device__ __forceinline__ void pass2_twins_body(const StepArgs& A, int s) {
  const int n = A.n;
  const int m = min(A.cnt[s], A.cap);
  const int mr = m - ghost_count(A, s, m);
  if (mr == m || A.fbslot[s] != -1) return;
  const float4 hi = A.XU[s].xh, lo = A.XU[s].xl;
  const float4 gvi = A.XU[s].uh;
  double bgd, bvd;
  ghost_rhs2(A, A.p1[P1_GN * n + s], A.K.euler ? A.V[s] : A.p1[P1_VN * n + s], &bgd, &bvd);
  const ff bgg = ff_of(bgd), bvg = ff_of(bvd);
  ff R[2][kNB];
#pragma unroll
  for (int f = 0; f < 2; ++f)
#pragma unroll
    for (int q = 0; q < kNB; ++q) R[f][q] = {0.f, 0.f};
#pragma unroll 1
  for (int k = mr; k < m; ++k) {
    const uint32_t c0 = (uint32_t)A.nbr[(int64_t)k * n + s];
    const int j = c0 & kIndexMask;
    if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
    ff a[kNB];
    ff_taylor(ff_entry_row<PER>(A, s, hi, lo, c0), a);
    const float4 gvj = A.XU[j].uh;
    const ff bg = (c0 >> 31) ? ff{-gvi.x, -gvi.y} : ff_diff(gvj.x, gvj.y, gvi.x, gvi.y);
    const ff bv = ff_diff(gvj.z, gvj.w, gvi.z, gvi.w);
    const ff lin[2] = {ff_sub(bg, bgg), ff_sub(bv, bvg)};
    const ff quad[2] = {ff_add(bg, bgg), ff_add(bv, bvg)};
#pragma unroll
    for (int q = 0; q < kNB; ++q) {
      ff_acc(R[0][q], q < 3 ? lin[0] : quad[0], a[q]);
      ff_acc(R[1][q], q < 3 ? lin[1] : quad[1], a[q]);
    }
  }
#pragma unroll
  for (int f = 0; f < 2; ++f)
#pragma unroll
    for (int q = 0; q < kNB; ++q) {
      const ff v = ff_norm(R[f][q]);
      A.T2[(int64_t)(f * kNB + q) * n + s] = v.h;
      A.T2[(int64_t)(18 + f * kNB + q) * n + s] = v.l;
    }
}

// Gram matrix of a stencil in float-float (positions only): the 31 moments,
// the Cholesky factor with the pivot test, stored for both passes. Stencils
// that fail the test (or have fewer than 9 rows) are queued for the
// pivoted-QR fit.
template <bool PER>
__device__ __forceinline__ void gram_ff_body(const StepArgs& A, int s) {
  const int n = A.n;
  const int m = min(A.cnt[s], A.cap);
  const float4 hi = A.XU[s].xh, lo = A.XU[s].xl;
  // entries with a ghost (at the end of the stencil): their moments, with
  // their ghosts', come from gram_twins_body and seed the sums
  const int mr = m - ghost_count(A, s, m);
  // The nine sums of terms that are never negative start at a power of two
  // C >= rho^d (rho >= |offset| / h, d the degree): they only grow, so each
  // row's term stays below the running sum and FastTwoSum is exact; C is
  // small against the sums (no precision is lost) and comes off with an
  // error-free TwoSum at the end. Signed sums keep TwoSum (a seed large
  // enough for them would cost precision).
  const float r2 = A.K.rho * A.K.rho, r4 = r2 * r2;
  const float Cpos[2] = {pow2_ceil(r2), pow2_ceil(r4)};
  auto seed = [&](int q) {
    return moment_nonneg(q) ? Cpos[moment_degree(q) == 2 ? 0 : 1] : 0.f;
  };
  ff mo[31];
  if (mr < m) {
#pragma unroll
    for (int q = 0; q < 31; ++q)
      mo[q] = ff_add(ff{seed(q), 0.f},
                     ff{A.Tg[(int64_t)q * n + s], A.Tg[(int64_t)(31 + q) * n + s]});
  } else {
#pragma unroll
    for (int q = 0; q < 31; ++q) mo[q] = {seed(q), 0.f};
  }
  // software pipeline: stencil codes are loaded two rows ahead and the
  // neighbour's values one row ahead, so the dependent loads of a row
  // overlap the arithmetic of the previous one (same in both passes).
  uint32_t code = mr > 0 ? (uint32_t)A.nbr[s] : 0u;
  uint32_t nxt = mr > 1 ? (uint32_t)A.nbr[(int64_t)n + s] : 0u;
  float4 jh = make_float4(0.f, 0.f, 0.f, 0.f), jl = jh;
  if (mr > 0) ff_gather(A, s, code, jh, jl);
  for (int k = 0; k < mr; ++k) {
    const uint32_t c0 = code;
    const float4 h0 = jh, l0 = jl;
    if (k + 1 < mr) {
      code = nxt;
      ff_gather(A, s, code, jh, jl);
      if (k + 2 < mr) nxt = (uint32_t)A.nbr[(int64_t)(k + 2) * n + s];
    }
    ff_moments_add_seeded(mo, ff_row_of<PER>(hi, lo, h0, l0, c0, A.K));
  }
#pragma unroll
  for (int q = 0; q < 31; ++q) {  // remove the seed (error-free)
    const ff d = two_sum(mo[q].h, -seed(q));
    mo[q] = fast_two_sum(d.h, __fadd_rn(d.l, mo[q].l));
  }
  ff G[kTri];
  ff_gram_fo(mo, G);
#pragma unroll
  for (int k = 0; k < kTri; ++k) G[k] = ff_norm(G[k]);
  const bool ok = ff_chol9(G, 1e-4f) && m >= kNB;
  if (!ok) {
    push_fallback(A, s);
    return;
  }
  A.fbslot[s] = -1;
#pragma unroll
  for (int k = 0; k < kTri; ++k) {
    A.Lff[(int64_t)k * n + s] = make_float2(G[k].h, G[k].l);
  }
}

// Derived values of pass 1 from float-float coefficients (as pass1_finish):
// gdot, |gdot|, (1/2) Lap u + (1/6) grad div u and div u are formed in
// float-float. Pass 2 takes gdot and ld as float-float (P1s); of the FP64
// outputs it reads |gdot| and V^{n+1} = V^n + dt V^n div u (FP64) only, since
// the FP64 gdot, ld and div u of a particle are read only when it was fitted
// by the QR fallback, whose kernel writes them. So the per-particle FP64 work
// is two conversions and the V update.
__device__ __forceinline__ void pass1_finish_ff(const StepArgs& A, int s, const ff (*c)[kNB]) {
  const int n = A.n;
  const ff ih{A.K.ih_h, A.K.ih_l}, ih2{A.K.ih2_h, A.K.ih2_l};
  const ff third{0x1.555556p-2f, -0x1.555556p-27f}, sixth{0x1.555556p-3f, -0x1.555556p-28f};
  ff G[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) G[a][b] = ff_mul(c[a][b], ih);
  const ff div = ff_add(ff_add(G[0][0], G[1][1]), G[2][2]);
  const ff d3 = ff_mul(div, third);
  const ff gd[6] = {ff_sub(G[0][0], d3), ff_sub(G[1][1], d3), ff_sub(G[2][2], d3),
                    ff_scale(ff_add(G[0][1], G[1][0]), 0.5f),
                    ff_scale(ff_add(G[0][2], G[2][0]), 0.5f),
                    ff_scale(ff_add(G[1][2], G[2][1]), 0.5f)};
  const ff dia = ff_add(ff_add(ff_mul(gd[0], gd[0]), ff_mul(gd[1], gd[1])), ff_mul(gd[2], gd[2]));
  const ff off = ff_add(ff_add(ff_mul(gd[3], gd[3]), ff_mul(gd[4], gd[4])), ff_mul(gd[5], gd[5]));
  const ff half = ff_add(ff_scale(dia, 0.5f), off);  // (1/2) gdot:gdot
  double gn;
  if (half.h > 0x1p-120f) {
    gn = ff_to_double(ff_mul(half, ff_rsqrt(half)));  // sqrt = x / sqrt(x)
  } else {
    gn = half.h > 0.f ? sqrt(ff_to_double(half)) : 0.0;  // (1/x^2 would overflow)
  }
  double* p = A.p1;
  p[P1_GN * n + s] = gn;
  // the float-float copy for the acceleration of pass 2
#pragma unroll
  for (int q = 0; q < 6; ++q) A.P1s[(int64_t)q * n + s] = make_float2(gd[q].h, gd[q].l);
  // Hessian columns: 3 xx, 4 yy, 5 zz, 6 xy, 7 xz, 8 yz
  const ff dd[3] = {ff_add(ff_add(c[0][3], c[1][6]), c[2][7]),
                    ff_add(ff_add(c[0][6], c[1][4]), c[2][8]),
                    ff_add(ff_add(c[0][7], c[1][8]), c[2][5])};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const ff lap = ff_add(ff_add(c[a][3], c[a][4]), c[a][5]);
    const ff ld = ff_mul(ff_add(ff_scale(lap, 0.5f), ff_mul(dd[a], sixth)), ih2);
    A.P1s[(int64_t)(6 + a) * n + s] = make_float2(ld.h, ld.l);
  }
  const double Vi = A.V[s], dv = ff_to_double(div);
  p[P1_VN * n + s] = Vi + A.K.dt * (Vi * dv);
}

// pass 1 in float-float, first half: the right-hand sides A^T b of u, v, w
// (unnormalised float-float accumulators, left in R)
template <bool PER>
__device__ __forceinline__ void pass1_ff_rhs(const StepArgs& A, int s, ff (*R)[kNB]) {
  const int n = A.n;
  const int m = min(A.cnt[s], A.cap);  // ghost rows carry b = 0: no right-hand side
  const float4 hi = A.XU[s].xh, lo = A.XU[s].xl;
  const float4 uh = A.XU[s].uh, ul = A.XU[s].ul;
  const int mm = A.K.mirror_mode;
  const float sg[3] = {mm == LP_MIRROR_NOSLIP ? -1.f : 1.f, mm == LP_MIRROR_NOSLIP ? -1.f : 1.f,
                       mm != LP_MIRROR_NONE ? -1.f : 1.f};
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int q = 0; q < kNB; ++q) R[f][q] = {0.f, 0.f};
  uint32_t code = m > 0 ? (uint32_t)A.nbr[s] : 0u;
  uint32_t nxt = m > 1 ? (uint32_t)A.nbr[(int64_t)n + s] : 0u;
  float4 xh = make_float4(0.f, 0.f, 0.f, 0.f), xl = xh, vh = xh, vl = xh;
  if (m > 0) {
    ff_gather(A, s, code, xh, xl);
    const unsigned jj = min(code & kIndexMask, (unsigned)(n - 1));
    vh = A.XU[jj].uh; vl = A.XU[jj].ul;
  }
  for (int k = 0; k < m; ++k) {
    const uint32_t c0 = code;
    const float4 h0 = xh, l0 = xl, jh = vh, jl = vl;
    if (k + 1 < m) {
      code = nxt;
      ff_gather(A, s, code, xh, xl);
      const unsigned jj = min(code & kIndexMask, (unsigned)(n - 1));
      vh = A.XU[jj].uh; vl = A.XU[jj].ul;
      if (k + 2 < m) nxt = (uint32_t)A.nbr[(int64_t)(k + 2) * n + s];
    }
    const FFRow r = ff_row_of<PER>(hi, lo, h0, l0, c0, A.K);
    ff a[kNB];
    ff_taylor(r, a);
    const int j = c0 & kIndexMask;
    if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
    const bool mir = c0 >> 31;
    const float ujh[3] = {jh.x, jh.y, jh.z}, ujl[3] = {jl.x, jl.y, jl.z};
    const float uih[3] = {uh.x, uh.y, uh.z}, uil[3] = {ul.x, ul.y, ul.z};
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      const float sj = mir ? sg[f] : 1.f;
      const ff b = ff_diff(sj * ujh[f], sj * ujl[f], uih[f], uil[f]);
#pragma unroll
      for (int q = 0; q < kNB; ++q) ff_acc(R[f][q], b, a[q]);
    }
  }
}

// pass 1 in float-float: right-hand sides, solves and derived values in one
// thread (the persistent launch)
template <bool PER>
__device__ __forceinline__ void pass1_ff_body(const StepArgs& A, int s) {
  if (A.fbslot[s] != -1) return;  // queued for the pivoted-QR fit
  ff R[3][kNB];
  pass1_ff_rhs<PER>(A, s, R);
  ff_chol_solve<3>(A.Lff + s, A.n, R);
  pass1_finish_ff(A, s, R);
}

// The same work in two kernels (the per-phase launches): the row loop stores
// its 27 accumulators as they stand (R1, hi and lo, k-major), and the solve
// kernel reloads them, so the result is the same bits. Each kernel then keeps
// one instruction stream: the unrolled row loop (about 530 instructions) or
// the unrolled three-right-hand-side solve (about 3,100).
template <bool PER>
__device__ __forceinline__ void pass1_ff_rows_body(const StepArgs& A, int s) {
  if (A.fbslot[s] != -1) return;
  ff R[3][kNB];
  pass1_ff_rhs<PER>(A, s, R);
  const int64_t n = A.n;
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int q = 0; q < kNB; ++q) A.R1[(int64_t)(f * kNB + q) * n + s] = make_float2(R[f][q].h, R[f][q].l);
}
__device__ __forceinline__ void pass1_ff_solve_body(const StepArgs& A, int s) {
  if (A.fbslot[s] != -1) return;
  const int64_t n = A.n;
  ff R[3][kNB];
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int q = 0; q < kNB; ++q) {
      const float2 v = A.R1[(int64_t)(f * kNB + q) * n + s];
      R[f][q] = ff{v.x, v.y};
    }
  // one field at a time (the same operations per field as the joint solve;
  // the joint form makes the compiler keep R in local memory here)
  ff_chol_solve<1>(A.Lff + s, A.n, R + 0);
  ff_chol_solve<1>(A.Lff + s, A.n, R + 1);
  ff_chol_solve<1>(A.Lff + s, A.n, R + 2);
  pass1_finish_ff(A, s, R);
}

// pass-2 fits in float-float: gradients of |gdot|^n and V^{n+1}
template <bool PER>
__device__ __forceinline__ void pass2_ff_grads(const StepArgs& A, int s, int m, ff* gg,
                                               ff* gV) {
  const int n = A.n;
  const float4 hi = A.XU[s].xh, lo = A.XU[s].xl;
  const float4 gvi = A.XU[s].uh;
  // entries with a ghost (at the end of the stencil): their terms, with their
  // ghosts', come from pass2_twins_body and seed the sums
  const int mg = ghost_count(A, s, m);
  m -= mg;
  ff R[2][kNB];
  if (mg) {
#pragma unroll
    for (int f = 0; f < 2; ++f)
#pragma unroll
      for (int q = 0; q < kNB; ++q)
        R[f][q] = ff{A.T2[(int64_t)(f * kNB + q) * n + s], A.T2[(int64_t)(18 + f * kNB + q) * n + s]};
  } else {
#pragma unroll
    for (int f = 0; f < 2; ++f)
#pragma unroll
      for (int q = 0; q < kNB; ++q) R[f][q] = {0.f, 0.f};
  }
  uint32_t code = m > 0 ? (uint32_t)A.nbr[s] : 0u;
  uint32_t nxt = m > 1 ? (uint32_t)A.nbr[(int64_t)n + s] : 0u;
  float4 jh = make_float4(0.f, 0.f, 0.f, 0.f), jl = jh, jg = jh;
  if (m > 0) {
    ff_gather(A, s, code, jh, jl);
    jg = A.XU[min(code & kIndexMask, (unsigned)(n - 1))].uh;
  }
  for (int k = 0; k < m; ++k) {
    const uint32_t c0 = code;
    const float4 h0 = jh, l0 = jl, gvj = jg;
    if (k + 1 < m) {
      code = nxt;
      ff_gather(A, s, code, jh, jl);
      jg = A.XU[min(code & kIndexMask, (unsigned)(n - 1))].uh;
      if (k + 2 < m) nxt = (uint32_t)A.nbr[(int64_t)(k + 2) * n + s];
    }
    const FFRow r = ff_row_of<PER>(hi, lo, h0, l0, c0, A.K);
    ff a[kNB];
    ff_taylor(r, a);
    const int j = c0 & kIndexMask;
    if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
    const bool mir = c0 >> 31;
    const ff bg = mir ? ff{-gvi.x, -gvi.y} : ff_diff(gvj.x, gvj.y, gvi.x, gvi.y);
    const ff bv = ff_diff(gvj.z, gvj.w, gvi.z, gvi.w);
#pragma unroll
    for (int q = 0; q < kNB; ++q) {
      ff_acc(R[0][q], bg, a[q]);
      ff_acc(R[1][q], bv, a[q]);
    }
  }
  ff_chol_solve<2, true>(A.Lff + s, A.n, R);  // only the gradients are used
  const ff ih{A.K.ih_h, A.K.ih_l};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    gg[q] = ff_mul(R[0][q], ih);
    gV[q] = ff_mul(R[1][q], ih);
  }
}

// Acceleration of the inertial regime (Sec. 2.3) in float-float, for a
// particle fitted in float-float: V [ -(|g|/V^2)(S |g| V_c + R g_cj V_j) +
// 2 M |g| |g|_c + N g_cj |g|_j + N |g| ld_c ] + g_c with the closure M, N,
// S, R at phi = 1/V formed in float-float from the column's constants.
// |g| and V come from the split record, gdot and ld from pass 1's
// float-float copy; the result is rounded to FP64 once per component.
__device__ __forceinline__ void accel_ff(const StepArgs& A, int s, const ff* gg, const ff* gV,
                                         double* acc) {
  const int64_t n = A.n;
  const float4 gv = A.XU[s].uh;
  const ff G{gv.x, gv.y}, V{gv.z, gv.w};
  const ColMui& cm = A.mui[A.colid[s]];
  const ff k{cm.kf[0], cm.kf[1]}, aI0{cm.aI0f[0], cm.aI0f[1]}, b{cm.bf[0], cm.bf[1]};
  const ff mu2{cm.mu2f[0], cm.mu2f[1]}, c{cm.cf[0], cm.cf[1]};
  const ff phi = ff_recip(V);
  const ff w = ff_sub(ff{A.K.phic_h, A.K.phic_l}, phi);
  const ff iw = ff_recip(w), iw2 = ff_mul(iw, iw);
  const ff iden = ff_recip(ff_add(aI0, w));
  const ff M = ff_neg(ff_mul(k, iw2));
  const ff mu = ff_mul(ff_add(b, ff_mul(mu2, w)), iden);
  const ff N = ff_neg(ff_mul(M, mu));
  const ff S = ff_scale(ff_mul(ff_mul(k, iw2), iw), -2.f);
  const ff dmu = ff_neg(ff_mul(c, ff_mul(iden, iden)));
  const ff R = ff_neg(ff_add(ff_mul(S, mu), ff_mul(M, dmu)));
  ff g3[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float2 v = A.P1s[(int64_t)q * n + s];
    g3[q] = ff{v.x, v.y};
  }
  // rows of the symmetric gdot: (xx, xy, xz), (xy, yy, yz), (xz, yz, zz)
  const int ix[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
  const ff GV2 = ff_mul(G, ff_mul(phi, phi));  // |g| / V^2
  const ff SG = ff_mul(S, G), MG2 = ff_scale(ff_mul(M, G), 2.f), NG = ff_mul(N, G);
  const double gvec[3] = {A.K.gx, A.K.gy, A.K.gz};
#pragma unroll
  for (int cc = 0; cc < 3; ++cc) {
    ff gjV = ff_mul(g3[ix[cc][0]], gV[0]), gjG = ff_mul(g3[ix[cc][0]], gg[0]);
#pragma unroll
    for (int d = 1; d < 3; ++d) {
      gjV = ff_add(gjV, ff_mul(g3[ix[cc][d]], gV[d]));
      gjG = ff_add(gjG, ff_mul(g3[ix[cc][d]], gg[d]));
    }
    const float2 l = A.P1s[(int64_t)(6 + cc) * n + s];
    const ff t1 = ff_neg(ff_mul(GV2, ff_add(ff_mul(SG, gV[cc]), ff_mul(R, gjV))));
    const ff t2 = ff_mul(MG2, gg[cc]);
    const ff t3 = ff_mul(N, gjG);
    const ff t4 = ff_mul(NG, ff{l.x, l.y});
    acc[cc] = ff_to_double(ff_mul(V, ff_add(ff_add(ff_add(t1, t2), t3), t4))) + gvec[cc];
  }
}

// ------------------------------------------------------------ pass 2

// every lane of the warp must call it (live or not)
template <int PREC, bool PER = false>
__device__ __forceinline__ void pass2_body(const StepArgs& A, int s, bool live) {
  int regime = 1;
  bool overc = false, nonfin = false, below = false;
  float disp = 0.f;  // displacement from the search positions (filter skipping)
  if (live) {
    const int n = A.n;
    const double xi = A.x[s], yi = A.y[s], zi = A.z[s];
    const double ih = A.K.inv_h, f2 = 2.0 * A.K.floor_z;
    const double* gn = A.p1 + P1_GN * n;
    // V of the fits and the closure: V^{n+1} (the paper's step) or V^n (a
    // stage of Heun's method, whose right-hand side takes one time level)
    const double* Vn = A.K.euler ? A.V : A.p1 + P1_VN * n;
    const double gni = gn[s], Vi = Vn[s];
    const double Vnext = A.p1[P1_VN * n + s];
    double gg[3], gV[3];
    ff ggf[3], gVf[3];  // float-float fit (LP_MIXED_FF, no fallback)
    bool ffit = false;
    const int slot = A.fbslot[s];
    if (slot >= 0) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        gg[q] = A.fbgrad[6 * slot + q];
        gV[q] = A.fbgrad[6 * slot + 3 + q];
      }
    } else if (slot == -1) {
      const int m = min(A.cnt[s], A.cap);
      if (PREC == LP_MIXED_FF) {
        pass2_ff_grads<PER>(A, s, m, ggf, gVf);
        ffit = true;
#pragma unroll
        for (int q = 0; q < 3; ++q) gg[q] = gV[q] = 0.0;  // set below where needed
      } else if (PREC == LP_FP64) {
        double R[2][kNB];
#pragma unroll
        for (int f = 0; f < 2; ++f)
#pragma unroll
          for (int c = 0; c < kNB; ++c) R[f][c] = 0.0;
        double bg_gh = 0.0, bv_gh = 0.0;
        if (A.K.free_surface) ghost_rhs2(A, gni, Vi, &bg_gh, &bv_gh);
        for (int k = 0; k < m; ++k) {
          const uint32_t code = (uint32_t)A.nbr[(int64_t)k * n + s];
          const int j = code & kIndexMask;
          if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
          const bool mir = code >> 31;
          const double zj = mir ? f2 - A.z[j] : A.z[j];
          const double dx = per_off<PER>(A.x[j] - xi, A.K.Lx) * ih;
          const double dy = per_off<PER>(A.y[j] - yi, A.K.Ly) * ih, dz = (zj - zi) * ih;
          // the entry's row, then (flagged entries) its ghost's reflected row
          for (int t = 0; t < ((code & kGhostBit) ? 2 : 1); ++t) {
            const double rs = t ? -1.0 : 1.0;
            double a[kNB];
            taylor_row(rs * dx, rs * dy, rs * dz, a);
            const double bg = t ? bg_gh : (mir ? 0.0 : gn[j]) - gni;
            const double bv = t ? bv_gh : Vn[j] - Vi;
#pragma unroll
            for (int c = 0; c < kNB; ++c) {
              R[0][c] += bg * a[c];
              R[1][c] += bv * a[c];
            }
          }
        }
        double L[kTri];
#pragma unroll
        for (int k = 0; k < kTri; ++k) L[k] = A.fac[(int64_t)k * n + s];
        chol9_solve(L, R[0]);
        chol9_solve(L, R[1]);
        if (A.coef2) {
#pragma unroll
          for (int q = 0; q < kNB; ++q) {
            A.coef2[(int64_t)q * n + s] = R[0][q];
            A.coef2[(int64_t)(kNB + q) * n + s] = R[1][q];
          }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          gg[q] = R[0][q] * ih;
          gV[q] = R[1][q] * ih;
        }
      } else {
        float L[kTri];
#pragma unroll
        for (int k = 0; k < kTri; ++k) L[k] = A.facf[(int64_t)k * n + s];
        float Rf[2][kNB];
#pragma unroll
        for (int f = 0; f < 2; ++f)
#pragma unroll
          for (int c = 0; c < kNB; ++c) Rf[f][c] = 0.f;
        double bg_gh = 0.0, bv_gh = 0.0;
        if (A.K.free_surface) ghost_rhs2(A, gni, Vi, &bg_gh, &bv_gh);
        for (int k = 0; k < m; ++k) {
          const uint32_t code = (uint32_t)A.nbr[(int64_t)k * n + s];
          const int j = code & kIndexMask;
          if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
          const bool mir = code >> 31;
          const double zj = mir ? f2 - A.z[j] : A.z[j];
          const float dx = (float)(per_off<PER>(A.x[j] - xi, A.K.Lx) * ih);
          const float dy = (float)(per_off<PER>(A.y[j] - yi, A.K.Ly) * ih);
          const float dz = (float)((zj - zi) * ih);
          for (int t = 0; t < ((code & kGhostBit) ? 2 : 1); ++t) {
            const float rs = t ? -1.f : 1.f;
            float a[kNB];
            taylor_row(rs * dx, rs * dy, rs * dz, a);
            const float bg = (float)(t ? bg_gh : (mir ? 0.0 : gn[j]) - gni);
            const float bv = (float)(t ? bv_gh : Vn[j] - Vi);
#pragma unroll
            for (int c = 0; c < kNB; ++c) {
              Rf[0][c] += bg * a[c];
              Rf[1][c] += bv * a[c];
            }
          }
        }
        chol9_solve(L, Rf[0]);
        chol9_solve(L, Rf[1]);
        double c2[2][kNB], g[2][kNB];
#pragma unroll
        for (int q = 0; q < kNB; ++q) {
          c2[0][q] = Rf[0][q]; c2[1][q] = Rf[1][q];
          g[0][q] = 0.0; g[1][q] = 0.0;
        }
        for (int k = 0; k < m; ++k) {
          const uint32_t code = (uint32_t)A.nbr[(int64_t)k * n + s];
          const int j = code & kIndexMask;
          if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
          const bool mir = code >> 31;
          const double zj = mir ? f2 - A.z[j] : A.z[j];
          const double dx = per_off<PER>(A.x[j] - xi, A.K.Lx) * ih;
          const double dy = per_off<PER>(A.y[j] - yi, A.K.Ly) * ih, dz = (zj - zi) * ih;
          for (int t = 0; t < ((code & kGhostBit) ? 2 : 1); ++t) {
            const double rs = t ? -1.0 : 1.0;
            double a[kNB];
            taylor_row(rs * dx, rs * dy, rs * dz, a);
            double r0 = t ? bg_gh : (mir ? 0.0 : gn[j]) - gni, r1 = t ? bv_gh : Vn[j] - Vi;
#pragma unroll
            for (int q = 0; q < kNB; ++q) {
              r0 -= a[q] * c2[0][q];
              r1 -= a[q] * c2[1][q];
            }
#pragma unroll
            for (int q = 0; q < kNB; ++q) {
              g[0][q] += a[q] * r0;
              g[1][q] += a[q] * r1;
            }
          }
        }
        chol9_solve(L, g[0]);
        chol9_solve(L, g[1]);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          gg[q] = (c2[0][q] + g[0][q]) * ih;
          gV[q] = (c2[1][q] + g[1][q]) * ih;
        }
      }
    } else {
      // no fallback slot was available: treat the stencil as empty
#pragma unroll
      for (int q = 0; q < 3; ++q) gg[q] = gV[q] = 0.0;
    }
    // ---- acceleration (pressure law of Sec. 2.2.1 at phi^{n+1})
    const double phi = 1.0 / Vi;
    const double gvec[3] = {A.K.gx, A.K.gy, A.K.gz};
    double acc[3];
    if (phi <= A.K.phi_min) {
      regime = 0;
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] = gvec[c];
    } else if (phi <= A.K.phi_max && PREC == LP_MIXED_FF && ffit) {
      regime = 1;
      accel_ff(A, s, ggf, gVf, acc);
    } else if (phi <= A.K.phi_max) {
      regime = 1;
      const Closure cl = closure_at(phi, A.mui[A.colid[s]], A.K.phi_c, A.K.phi_min);
      const double g00 = A.p1[(P1_GD + 0) * n + s], g11 = A.p1[(P1_GD + 1) * n + s];
      const double g22 = A.p1[(P1_GD + 2) * n + s], g01 = A.p1[(P1_GD + 3) * n + s];
      const double g02 = A.p1[(P1_GD + 4) * n + s], g12 = A.p1[(P1_GD + 5) * n + s];
      const double g3[3][3] = {{g00, g01, g02}, {g01, g11, g12}, {g02, g12, g22}};
      const double G = gni;
      const double GV2 = G / (Vi * Vi);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        // V [ -(|g|/V^2)(S|g| V_c + R g_cj V_j) + 2M|g| |g|_c + N g_cj |g|_j
        //     + N|g| ((1/2) Lap u_c + (1/6) d_c div u) ] + g_c
        const double gjVj = (g3[c][0] * gV[0] + g3[c][1] * gV[1]) + g3[c][2] * gV[2];
        const double gjGj = (g3[c][0] * gg[0] + g3[c][1] * gg[1]) + g3[c][2] * gg[2];
        const double t1 = -GV2 * (cl.S * G * gV[c] + cl.R * gjVj);
        const double t2 = 2.0 * cl.M * G * gg[c];
        const double t3 = cl.N * gjGj;
        const double t4 = cl.N * G * A.p1[(P1_LD + c) * n + s];
        acc[c] = Vi * (((t1 + t2) + t3) + t4) + gvec[c];
      }
    } else {
      regime = 2;
      if (PREC == LP_MIXED_FF && ffit)
#pragma unroll
        for (int q = 0; q < 3; ++q) gV[q] = ff_to_double(gVf[q]);
      // sigma = -phi_s (alpha + beta phi) I  =>  a = beta grad V / V + g
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] = (A.K.beta * gV[c]) / Vi + gvec[c];
      overc = phi > A.K.phi_c;
    }
    // ---- update (Sec. 3.1 items 8, 10)
    const double dt = A.K.dt;
    const double un = A.u[s], vn = A.v[s], wn = A.w[s];
    const double u1 = un + dt * acc[0], v1 = vn + dt * acc[1], w1 = wn + dt * acc[2];
    // x with the mean velocity (the paper's step) or with u^n (Heun stage)
    const double hx = A.K.euler ? dt : 0.5 * dt;
    double x1 = xi + hx * (A.K.euler ? un : un + u1);
    double y1 = yi + hx * (A.K.euler ? vn : vn + v1);
    if (PER) {  // periodic axes: back into [0, L)
      x1 = wrap_pos(x1, A.K.Lx);
      y1 = wrap_pos(y1, A.K.Ly);
    }
    const double z1 = zi + hx * (A.K.euler ? wn : wn + w1);
    A.uo[s] = u1; A.vo[s] = v1; A.wo[s] = w1;
    A.xo[s] = x1; A.yo[s] = y1; A.zo[s] = z1;
    A.Vo[s] = Vnext;
    nonfin = !(isfinite(u1) && isfinite(v1) && isfinite(w1) && isfinite(x1) && isfinite(y1) &&
               isfinite(z1) && isfinite(Vnext));
    if (A.xref) {
      const double ex = per_off<PER>(x1 - A.xref[s], A.K.Lx);
      const double ey = per_off<PER>(y1 - A.xref[A.n + s], A.K.Ly);
      const double ez = z1 - A.xref[2 * A.n + s];
      const double e2 = ((ex * ex) + (ey * ey)) + (ez * ez);
      if (!(e2 <= A.half_skin2)) *A.need_search = 1;
      if (A.vskip.dmax) {  // rounded up: the conversion and sqrtf err by at most 2 ulp
        disp = fmaxf(A.vskip.dmax[s], sqrtf(__double2float_ru(e2)) * (1.f + 0x1p-21f));
        A.vskip.dmax[s] = disp;
      }
    }
    below = A.K.mirror_mode != LP_MIRROR_NONE && z1 < A.K.floor_z;
  }
  warp_count(&A.dg->n_gas, live && regime == 0);
  warp_count(&A.dg->n_quasistatic, live && regime == 2);
  warp_count(&A.dg->n_over_c, live && overc);
  warp_count(&A.dg->n_nonfinite, live && nonfin);
  warp_count(&A.dg->n_below_floor, live && below);
  if (A.vskip.dmax_all) {  // one atomic per warp (floats >= 0 order as their bits)
    const unsigned v = __reduce_max_sync(0xffffffffu, __float_as_uint(live ? disp : 0.f));
    if ((threadIdx.x & 31) == 0 && v) atomicMax(A.vskip.dmax_all, v);
  }
  if (live && nonfin) atomicOr(&A.dg->flags, (unsigned)LP_FLAG_NONFINITE);
  if (live && below) atomicOr(&A.dg->flags, (unsigned)LP_FLAG_BELOW_FLOOR);
}

}  // namespace lp
