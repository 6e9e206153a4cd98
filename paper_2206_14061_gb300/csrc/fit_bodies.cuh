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

// ------------------------------------------------------------ pass 1

template <int PREC>
__device__ __forceinline__ void pass1_body(const StepArgs& A, int s) {
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
      const int j = code & ~kMirrorBit;
      const bool mir = code >> 31;
      const double zj = mir ? f2 - A.z[j] : A.z[j];
      const double dx = (A.x[j] - xi) * ih, dy = (A.y[j] - yi) * ih, dz = (zj - zi) * ih;
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
      const int j = code & ~kMirrorBit;
      const bool mir = code >> 31;
      const double zj = mir ? f2 - A.z[j] : A.z[j];
      const float dx = (float)((A.x[j] - xi) * ih), dy = (float)((A.y[j] - yi) * ih);
      const float dz = (float)((zj - zi) * ih);
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
      const int j = code & ~kMirrorBit;
      const bool mir = code >> 31;
      const double zj = mir ? f2 - A.z[j] : A.z[j];
      const double dx = (A.x[j] - xi) * ih, dy = (A.y[j] - yi) * ih, dz = (zj - zi) * ih;
      double uj = A.u[j], vj = A.v[j], wj = A.w[j];
      if (mir) { uj *= su; vj *= sv; wj *= sw; }
      double a[kNB];
      taylor_row(dx, dy, dz, a);
      const double b[3] = {uj - ui, vj - vi, wj - wi};
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        double r = b[f];
#pragma unroll
        for (int q = 0; q < kNB; ++q) r -= a[q] * c[f][q];
#pragma unroll
        for (int q = 0; q < kNB; ++q) g[f][q] += a[q] * r;
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
    for (int k = 0; k < m; ++k) {
      const uint32_t code = (uint32_t)A.nbr[(int64_t)k * n + s];
      const int j = code & ~kMirrorBit;
      const bool mir = code >> 31;
      const double zj = mir ? f2 - A.z[j] : A.z[j];
      taylor_row((A.x[j] - xi) * ih, (A.y[j] - yi) * ih, (zj - zi) * ih, &Am[k * kNB]);
      double uj = A.u[j], vj = A.v[j], wj = A.w[j];
      if (mir) { uj *= usign(mm, 0); vj *= usign(mm, 1); wj *= usign(mm, 2); }
      Bm[k * 3 + 0] = uj - ui; Bm[k * 3 + 1] = vj - vi; Bm[k * 3 + 2] = wj - wi;
    }
    qr_pivoted_solve(m, Am, 3, Bm, C);
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
    const double* Vn = A.p1 + P1_VN * n;
    for (int k = 0; k < m; ++k) {
      const uint32_t code = (uint32_t)A.nbr[(int64_t)k * n + s];
      const int j = code & ~kMirrorBit;
      const bool mir = code >> 31;
      const double zj = mir ? f2 - A.z[j] : A.z[j];
      taylor_row((A.x[j] - xi) * ih, (A.y[j] - yi) * ih, (zj - zi) * ih, &Am[k * kNB]);
      Bm[k * 2 + 0] = (mir ? 0.0 : gn[j]) - gn[s];
      Bm[k * 2 + 1] = Vn[j] - Vn[s];
    }
    qr_pivoted_solve(m, Am, 2, Bm, C);
    if (A.coef2)
      for (int q = 0; q < 2 * kNB; ++q) A.coef2[(int64_t)q * n + s] = C[q];
    for (int q = 0; q < 3; ++q) {
      A.fbgrad[6 * t + q] = C[q] * ih;
      A.fbgrad[6 * t + 3 + q] = C[kNB + q] * ih;
    }
  }
}

// ------------------------------------------------------------ pass 2

// every lane of the warp must call it (live or not)
template <int PREC>
__device__ __forceinline__ void pass2_body(const StepArgs& A, int s, bool live) {
  int regime = 1;
  bool overc = false, nonfin = false, below = false;
  if (live) {
    const int n = A.n;
    const double xi = A.x[s], yi = A.y[s], zi = A.z[s];
    const double ih = A.K.inv_h, f2 = 2.0 * A.K.floor_z;
    const double* gn = A.p1 + P1_GN * n;
    const double* Vn = A.p1 + P1_VN * n;
    const double gni = gn[s], Vi = Vn[s];
    double gg[3], gV[3];
    const int slot = A.fbslot[s];
    if (slot >= 0) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        gg[q] = A.fbgrad[6 * slot + q];
        gV[q] = A.fbgrad[6 * slot + 3 + q];
      }
    } else if (slot == -1) {
      const int m = min(A.cnt[s], A.cap);
      if (PREC == LP_FP64) {
        double R[2][kNB];
#pragma unroll
        for (int f = 0; f < 2; ++f)
#pragma unroll
          for (int c = 0; c < kNB; ++c) R[f][c] = 0.0;
        for (int k = 0; k < m; ++k) {
          const uint32_t code = (uint32_t)A.nbr[(int64_t)k * n + s];
          const int j = code & ~kMirrorBit;
          const bool mir = code >> 31;
          const double zj = mir ? f2 - A.z[j] : A.z[j];
          double a[kNB];
          taylor_row((A.x[j] - xi) * ih, (A.y[j] - yi) * ih, (zj - zi) * ih, a);
          const double bg = (mir ? 0.0 : gn[j]) - gni;
          const double bv = Vn[j] - Vi;
#pragma unroll
          for (int c = 0; c < kNB; ++c) {
            R[0][c] += bg * a[c];
            R[1][c] += bv * a[c];
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
        for (int k = 0; k < m; ++k) {
          const uint32_t code = (uint32_t)A.nbr[(int64_t)k * n + s];
          const int j = code & ~kMirrorBit;
          const bool mir = code >> 31;
          const double zj = mir ? f2 - A.z[j] : A.z[j];
          float a[kNB];
          taylor_row((float)((A.x[j] - xi) * ih), (float)((A.y[j] - yi) * ih),
                     (float)((zj - zi) * ih), a);
          const float bg = (float)((mir ? 0.0 : gn[j]) - gni);
          const float bv = (float)(Vn[j] - Vi);
#pragma unroll
          for (int c = 0; c < kNB; ++c) {
            Rf[0][c] += bg * a[c];
            Rf[1][c] += bv * a[c];
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
          const int j = code & ~kMirrorBit;
          const bool mir = code >> 31;
          const double zj = mir ? f2 - A.z[j] : A.z[j];
          double a[kNB];
          taylor_row((A.x[j] - xi) * ih, (A.y[j] - yi) * ih, (zj - zi) * ih, a);
          double r0 = (mir ? 0.0 : gn[j]) - gni, r1 = Vn[j] - Vi;
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
      // sigma = -phi_s (alpha + beta phi) I  =>  a = beta grad V / V + g
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] = (A.K.beta * gV[c]) / Vi + gvec[c];
      overc = phi > A.K.phi_c;
    }
    // ---- update (Sec. 3.1 items 8, 10)
    const double dt = A.K.dt;
    const double un = A.u[s], vn = A.v[s], wn = A.w[s];
    const double u1 = un + dt * acc[0], v1 = vn + dt * acc[1], w1 = wn + dt * acc[2];
    const double x1 = xi + (0.5 * dt) * (un + u1);
    const double y1 = yi + (0.5 * dt) * (vn + v1);
    const double z1 = zi + (0.5 * dt) * (wn + w1);
    A.uo[s] = u1; A.vo[s] = v1; A.wo[s] = w1;
    A.xo[s] = x1; A.yo[s] = y1; A.zo[s] = z1;
    A.Vo[s] = Vi;
    nonfin = !(isfinite(u1) && isfinite(v1) && isfinite(w1) && isfinite(x1) && isfinite(y1) &&
               isfinite(z1) && isfinite(Vi));
    below = A.K.mirror_mode != LP_MIRROR_NONE && z1 < A.K.floor_z;
  }
  warp_count(&A.dg->n_gas, live && regime == 0);
  warp_count(&A.dg->n_quasistatic, live && regime == 2);
  warp_count(&A.dg->n_over_c, live && overc);
  warp_count(&A.dg->n_nonfinite, live && nonfin);
  warp_count(&A.dg->n_below_floor, live && below);
  if (live && nonfin) atomicOr(&A.dg->flags, (unsigned)LP_FLAG_NONFINITE);
  if (live && below) atomicOr(&A.dg->flags, (unsigned)LP_FLAG_BELOW_FLOOR);
}

}  // namespace lp
