// Hand-written adjoint (reverse mode) of one FP64 LP step with frozen stencils.
//
// Forward step of particle i (stencil rows k, scaled offsets d_k, Taylor rows
// a_k, Gram matrix G = sum a_k a_k^T):
//   pass 1:  c_f = G^{-1} sum_k a_k b_fk,  b_fk = s_f u_f(j_k) - u_f(i)  (f = u,v,w)
//            -> velocity gradient, Hessians, div u, gdot, |gdot|,
//               ld = (1/2) Lap u + (1/6) grad div u,  V^{n+1} = V + dt V div u
//   pass 2:  c_g = G^{-1} A^T b_g (b_g from |gdot|, 0 at mirrors),
//            c_V = G^{-1} A^T b_V (b_V from V^{n+1})
//   accel:   pressure law / mu(I) stress at phi^{n+1} = 1/V^{n+1} (Sec. 2.3)
//   update:  u' = u + dt a,  x' = x + dt (u + u')/2,  V' = V^{n+1}
// Least-squares adjoint, for c = G^{-1} A^T b with residual r = b - A c:
//   z = G^{-1} cbar,  bbar = A z,  Abar = r z^T - (A z) c^T,
// and Abar reaches the positions through the offsets d_k = (p_k - p_i)/h.
// Stage of Heun's method (K.euler): x' = x + dt u and the pass-2 fits and the
// closure read V^n instead of V^{n+1}, so their V adjoint goes to V^n
// directly (lVd) rather than through V^{n+1} = V + dt V div u.
// Free-surface ghosts: a flagged entry k also stands for the row a_G =
// T(-d_k) of its point reflection. Its pass-1 right-hand sides are 0 (the
// ghost carries the particle's velocity); its pass-2 ones depend only on the
// particle's own |gdot| and V^{n+1} (the ghost state, regime frozen), so their
// adjoints return to the particle; its offset adjoint enters d_k with a minus
// sign. The flags are frozen like the stencils.
// Along a periodic axis an offset is the nearest image of p_k - p_i, a
// constant shift of it, and the position update wraps by whole periods: both
// leave the derivatives as they are.
// Regimes are frozen at their forward values; d|gdot|/dgdot is 0 where
// |gdot| = 0. Parameter gradients w.r.t. (mu_s, mu_2, I0) enter through N and
// R only. Stencils that took the pivoted-QR path in the forward step are
// full rank in all but degenerate cases; their least-squares solution is then
// G^{-1} A^T b as well, and the adjoint refactors G for them without the
// forward path's conditioning threshold. Rank-deficient stencils (fewer than
// 9 rows, or a non-positive pivot) carry no fit adjoint and are counted in
// n_fallback.
#include "fit_bodies.cuh"

namespace lp {

// Closure of Sec. 2.3 with the derivatives the adjoint needs.
struct ClosureD {
  double M, N, S, R, dS, dR;  // dS = dS/dphi, dR = dR/dphi (dM/dphi = S, dN/dphi = R)
  double dN_dth[3], dR_dth[3];
};
__device__ __forceinline__ ClosureD closure_d(double phi, const ColMui& m, double phi_c,
                                              double phi_min) {
  const double a = phi_c - phi_min;
  const double w = phi_c - phi;
  const double k = 4.0 * a * a * m.d * m.d;
  const double iw = 1.0 / w;
  ClosureD c;
  c.M = -k * iw * iw;
  c.S = -2.0 * k * iw * iw * iw;
  c.dS = -6.0 * k * iw * iw * iw * iw;
  const double den = a * m.I0 + w, iden = 1.0 / den;
  const double mu = (a * m.mu_s * m.I0 + m.mu_2 * w) * iden;
  const double dmu = m.mu_2 - m.mu_s;
  const double q = -a * m.I0 * dmu * iden * iden;          // dmu/dphi
  const double dq = -2.0 * a * m.I0 * dmu * iden * iden * iden;  // d2mu/dphi2
  c.N = -c.M * mu;
  c.R = -c.S * mu - c.M * q;
  c.dR = -c.dS * mu - 2.0 * c.S * q - c.M * dq;
  const double dmu_dth[3] = {a * m.I0 * iden, w * iden, a * w * (m.mu_s - m.mu_2) * iden * iden};
  const double dq_dth[3] = {a * m.I0 * iden * iden, -a * m.I0 * iden * iden,
                            -a * dmu * (w - a * m.I0) * iden * iden * iden};
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    c.dN_dth[t] = -c.M * dmu_dth[t];
    c.dR_dth[t] = -c.S * dmu_dth[t] - c.M * dq_dth[t];
  }
  return c;
}

__device__ __forceinline__ double usign_adj(int mode, int a) {
  return mode == LP_MIRROR_NOSLIP ? -1.0 : (mode == LP_MIRROR_FREESLIP && a == 2 ? -1.0 : 1.0);
}

// adjoint of the Taylor row: dbar = J^T abar
__device__ __forceinline__ void row_adjoint(double dx, double dy, double dz, const double* ab,
                                            double* db) {
  db[0] = ab[0] + dx * ab[3] + dy * ab[6] + dz * ab[7];
  db[1] = ab[1] + dy * ab[4] + dx * ab[6] + dz * ab[8];
  db[2] = ab[2] + dz * ab[5] + dx * ab[7] + dy * ab[8];
}
// the same in float-float
__device__ __forceinline__ void ff_row_adjoint(ff dx, ff dy, ff dz, const ff* ab, ff* db) {
  db[0] = ab[0];
  ff_acc(db[0], dx, ab[3]);
  ff_acc(db[0], dy, ab[6]);
  ff_acc(db[0], dz, ab[7]);
  db[1] = ab[1];
  ff_acc(db[1], dy, ab[4]);
  ff_acc(db[1], dx, ab[6]);
  ff_acc(db[1], dz, ab[8]);
  db[2] = ab[2];
  ff_acc(db[2], dz, ab[5]);
  ff_acc(db[2], dx, ab[7]);
  ff_acc(db[2], dy, ab[8]);
#pragma unroll
  for (int q = 0; q < 3; ++q) db[q] = ff_norm(db[q]);
}

// ---------------------------------------------------------------- R0
// which stencils carry a fit adjoint; FP64 factors for the QR-path ones
__global__ void __launch_bounds__(kBlock) k_adj_prepare(const AdjArgs A) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = s < A.n;
  bool skipped = false;
  if (live) {
    const int n = A.n;
    if (A.fbslot[s] == -1) {
      A.ok[s] = 1;
    } else {
      const int m = min(A.cnt[s], A.cap);
      const double xi = A.x[s], yi = A.y[s], zi = A.z[s];
      const double ih = A.K.inv_h, f2 = 2.0 * A.K.floor_z;
      Moments<double> M;
      M.zero();
      for (int k = 0; k < m; ++k) {
        const uint32_t code = (uint32_t)A.nbr[(int64_t)k * n + s];
        const int j = code & kIndexMask;
        if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
        const double zj = (code >> 31) ? f2 - A.z[j] : A.z[j];
        const double dx = min_image(A.x[j] - xi, A.K.Lx) * ih;
        const double dy = min_image(A.y[j] - yi, A.K.Ly) * ih, dz = (zj - zi) * ih;
        M.add(dx, dy, dz);
        if (code & kGhostBit) M.add(-dx, -dy, -dz);  // the ghost's row
      }
      double L[kTri];
      M.gram(L);
      const bool good = m >= kNB && chol9(L, 1e-15);
      A.ok[s] = good ? 1 : 0;
      skipped = !good;
      if (good)
        for (int k = 0; k < kTri; ++k) A.facx[(int64_t)k * n + s] = L[k];
    }
  }
  warp_count(&A.dg->n_fallback, live && skipped);
}

__device__ __forceinline__ const double* factor_of(const AdjArgs& A, int s) {
  return A.fbslot[s] == -1 ? A.fac : A.facx;
}

// ---------------------------------------------------------------- R1
// update and acceleration adjoints; solves for the pass-2 z vectors
__global__ void __launch_bounds__(kBlock) k_adj_accel(const AdjArgs A) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  double th[3] = {0.0, 0.0, 0.0};
  if (s < A.n) {
    const int n = A.n;
    const double dt = A.K.dt, ih = A.K.inv_h;
    const bool eu = A.K.euler;
    double lu1t[3], la[3];
    for (int c = 0; c < 3; ++c) {
      // x' = x + (dt/2)(u + u') (the paper's step) or x + dt u (Euler stage)
      lu1t[c] = A.l1[3 + c][s] + (eu ? 0.0 : 0.5 * dt * A.l1[c][s]);
      la[c] = dt * lu1t[c];
      A.l0[c][s] = A.l1[c][s];
      A.l0[3 + c][s] = lu1t[c] + (eu ? dt : 0.5 * dt) * A.l1[c][s];  // u' = u + dt a
    }
    const double lV1 = A.l1[6][s];  // V' = V^{n+1}
    double lVn = 0.0;               // adjoint of the V that the fits and the closure read
    const double Vn = eu ? A.V[s] : A.p1[P1_VN * n + s];
    const double Gn = A.p1[P1_GN * n + s];
    const double phi = 1.0 / Vn;
    const int slot = A.fbslot[s];
    const bool ok = A.ok[s];
    double gg[3], gV[3];
    if (slot == -1 || slot >= 0) {
      for (int q = 0; q < 3; ++q) {
        gg[q] = A.coef2[(int64_t)q * n + s] * ih;
        gV[q] = A.coef2[(int64_t)(kNB + q) * n + s] * ih;
      }
    } else {
      for (int q = 0; q < 3; ++q) gg[q] = gV[q] = 0.0;
    }
    double lgg[3] = {0, 0, 0}, lgV[3] = {0, 0, 0}, lld[3] = {0, 0, 0}, lGam[3][3] = {};
    double lGn = 0.0;
    if (phi <= A.K.phi_min) {
      // gas: a = g, no dependence on the state
    } else if (phi <= A.K.phi_max) {
      const ClosureD cl = closure_d(phi, A.mui[A.colid[s]], A.K.phi_c, A.K.phi_min);
      const double* p = A.p1;
      const double g00 = p[(P1_GD + 0) * n + s], g11 = p[(P1_GD + 1) * n + s];
      const double g22 = p[(P1_GD + 2) * n + s], g01 = p[(P1_GD + 3) * n + s];
      const double g02 = p[(P1_GD + 4) * n + s], g12 = p[(P1_GD + 5) * n + s];
      const double Gm[3][3] = {{g00, g01, g02}, {g01, g11, g12}, {g02, g12, g22}};
      double ld[3];
      for (int c = 0; c < 3; ++c) ld[c] = p[(P1_LD + c) * n + s];
      const double A1 = Gn / (Vn * Vn);
      double lM = 0, lN = 0, lS = 0, lR = 0;
      for (int c = 0; c < 3; ++c) {
        const double gV_c = (Gm[c][0] * gV[0] + Gm[c][1] * gV[1]) + Gm[c][2] * gV[2];
        const double gg_c = (Gm[c][0] * gg[0] + Gm[c][1] * gg[1]) + Gm[c][2] * gg[2];
        const double T1 = -A1 * (cl.S * Gn * gV[c] + cl.R * gV_c);
        const double T2 = 2.0 * cl.M * Gn * gg[c];
        const double T3 = cl.N * gg_c;
        const double T4 = cl.N * Gn * ld[c];
        const double B = ((T1 + T2) + T3) + T4;
        lVn += la[c] * B;  // a = V^{n+1} B + g
        const double lB = Vn * la[c];
        lS += -A1 * Gn * gV[c] * lB;
        lR += -A1 * gV_c * lB;
        lM += 2.0 * Gn * gg[c] * lB;
        lN += (gg_c + Gn * ld[c]) * lB;
        lgV[c] += -A1 * cl.S * Gn * lB;
        lgg[c] += 2.0 * cl.M * Gn * lB;
        for (int d = 0; d < 3; ++d) {
          lgV[d] += -A1 * cl.R * Gm[c][d] * lB;
          lgg[d] += cl.N * Gm[c][d] * lB;
          lGam[c][d] += (-A1 * cl.R * gV[d] + cl.N * gg[d]) * lB;
        }
        lld[c] += cl.N * Gn * lB;
        lGn += (-(2.0 * cl.S * Gn * gV[c] + cl.R * gV_c) / (Vn * Vn) + 2.0 * cl.M * gg[c] +
                cl.N * ld[c]) * lB;
        lVn += 2.0 * (Gn / (Vn * Vn * Vn)) * (cl.S * Gn * gV[c] + cl.R * gV_c) * lB;
      }
      // closure through phi = 1/V^{n+1}
      const double lphi = lM * cl.S + lN * cl.R + lS * cl.dS + lR * cl.dR;
      lVn += -lphi / (Vn * Vn);
      for (int t = 0; t < 3; ++t) th[t] = lN * cl.dN_dth[t] + lR * cl.dR_dth[t];
    } else {
      // quasi-static: a = beta grad V / V + g
      for (int c = 0; c < 3; ++c) {
        lgV[c] += A.K.beta * la[c] / Vn;
        lVn += -A.K.beta * gV[c] * la[c] / (Vn * Vn);
      }
    }
    A.lGn[s] = lGn;
    if (eu) {
      A.lVn[s] = lV1;
      A.lVd[s] = lVn;
    } else {
      A.lVn[s] = lV1 + lVn;
    }
    A.lG6[0 * n + s] = lGam[0][0];
    A.lG6[1 * n + s] = lGam[1][1];
    A.lG6[2 * n + s] = lGam[2][2];
    A.lG6[3 * n + s] = lGam[0][1] + lGam[1][0];
    A.lG6[4 * n + s] = lGam[0][2] + lGam[2][0];
    A.lG6[5 * n + s] = lGam[1][2] + lGam[2][1];
    for (int c = 0; c < 3; ++c) A.lld[c * n + s] = lld[c];
    // pass-2 least-squares adjoint: z = G^{-1} cbar
    double zg[kNB], zV[kNB];
    for (int q = 0; q < kNB; ++q) zg[q] = zV[q] = 0.0;
    if (ok) {
      for (int q = 0; q < 3; ++q) {
        zg[q] = lgg[q] * ih;
        zV[q] = lgV[q] * ih;
      }
      const double* F = factor_of(A, s);
      double L[kTri];
#pragma unroll
      for (int k = 0; k < kTri; ++k) L[k] = F[(int64_t)k * n + s];
      chol9_solve(L, zg);
      chol9_solve(L, zV);
    }
    for (int q = 0; q < kNB; ++q) {
      A.zz[(int64_t)q * n + s] = zg[q];
      A.zz[(int64_t)(kNB + q) * n + s] = zV[q];
    }
  }
  // parameter gradient: warp reduction, one atomic per warp and parameter
  for (int t = 0; t < 3; ++t) {
    double v = th[t];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(&A.dtheta[t], v);
  }
}

// ---------------------------------------------------------------- R2
// rows of the pass-2 adjoint: to the neighbours' |gdot| and V^{n+1}, and to
// the positions
template <bool PER>
__global__ void __launch_bounds__(kBlock) k_adj_pass2(const AdjArgs A) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= A.n || !A.ok[s]) return;
  const int n = A.n;
  // z and the forward coefficients c of the two pass-2 fits (|gdot|, V), split once
  ff zg[kNB], zV[kNB], cg[kNB], cV[kNB];
  bool any = false;
#pragma unroll
  for (int q = 0; q < kNB; ++q) {
    const double zgq = A.zz[(int64_t)q * n + s], zVq = A.zz[(int64_t)(kNB + q) * n + s];
    any = any || zgq != 0.0 || zVq != 0.0;
    zg[q] = ff_of(zgq);
    zV[q] = ff_of(zVq);
    cg[q] = ff_of(A.coef2[(int64_t)q * n + s]);
    cV[q] = ff_of(A.coef2[(int64_t)(kNB + q) * n + s]);
  }
  if (!any) return;
  const double* Gn = A.p1 + P1_GN * n;
  // V of the pass-2 fit: V^{n+1}, or V^n in an Euler stage (whose adjoint is lVd)
  const double* Vn = A.K.euler ? A.V : A.p1 + P1_VN * n;
  double* const lVfit = A.K.euler ? A.lVd : A.lVn;
  const double gni = Gn[s], Vi = Vn[s];
  // ghost rows (free surface): right-hand sides bg_G = |gdot|_G - gni and
  // bv_G = V_G - Vi with |gdot|_G = gni k / (phi_c - phi) in the inertial
  // regime; their derivatives with respect to gni and Vi (phi = 1/Vi)
  double bgG = 0.0, bvG = 0.0, dbg_dg = 0.0, dbg_dV = 0.0;
  if (A.K.free_surface) {
    const double phi = 1.0 / Vi;
    bvG = A.K.ghost_V - Vi;
    if (phi > A.K.phi_min && phi <= A.K.phi_max) {
      const double w = A.K.phi_c - phi;
      bgG = gni * (A.K.ghost_num / w) - gni;
      dbg_dg = A.K.ghost_num / w - 1.0;
      dbg_dV = -gni * A.K.ghost_num / (w * w * Vi * Vi);
    }
  }
  const ff bgGf = ff_of(bgG), bvGf = ff_of(bvG);
  // the rows in float-float, as in the pass-1 adjoint: positions and the
  // neighbours' |gdot|^n and V from the split state
  const float4 hi = A.XU[s].xh, lo = A.XU[s].xl, gvi = A.XU[s].uh;
  const ff ihf{A.K.ih_h, A.K.ih_l};
  const int m = min(A.cnt[s], A.cap);
  ff sg = {0.f, 0.f}, sV = {0.f, 0.f};
  ff sp[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  double og = 0.0, oV = 0.0;  // adjoints of the particle's own gni, Vi from ghost rows
  for (int k = 0; k < m; ++k) {
    const uint32_t code = (uint32_t)A.nbr[(int64_t)k * n + s];
    const int j = code & kIndexMask;
    if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
    const bool mir = code >> 31;
    const FF8& rj = A.XU[j];
    const FFRow row = ff_row_of<PER>(hi, lo, rj.xh, rj.xl, code, A.K);
    ff a[kNB];
    ff_taylor(row, a);
    const float4 gvj = rj.uh;
    ff rg = mir ? ff{-gvi.x, -gvi.y} : ff_diff(gvj.x, gvj.y, gvi.x, gvi.y);
    ff rV = ff_diff(gvj.z, gvj.w, gvi.z, gvi.w), bg = {0.f, 0.f}, bV = {0.f, 0.f};
#pragma unroll
    for (int q = 0; q < kNB; ++q) {
      ff_acc(rg, a[q], ff_neg(cg[q]));
      ff_acc(rV, a[q], ff_neg(cV[q]));
      ff_acc(bg, a[q], zg[q]);
      ff_acc(bV, a[q], zV[q]);
    }
    rg = ff_norm(rg);
    rV = ff_norm(rV);
    bg = ff_norm(bg);
    bV = ff_norm(bV);
    if (!mir) atomicAdd(&A.lGn[j], ffs_to_double(bg.h) + ffs_to_double(bg.l));
    sg = ff_add(sg, bg);
    atomicAdd(&lVfit[j], ffs_to_double(bV.h) + ffs_to_double(bV.l));  // the mirror of j carries V_j
    sV = ff_add(sV, bV);
    ff ab[kNB];
    const ff nbg = ff_neg(bg), nbV = ff_neg(bV);
#pragma unroll
    for (int q = 0; q < kNB; ++q) {
      ab[q] = {0.f, 0.f};
      ff_acc(ab[q], rg, zg[q]);
      ff_acc(ab[q], nbg, cg[q]);
      ff_acc(ab[q], rV, zV[q]);
      ff_acc(ab[q], nbV, cV[q]);
    }
    ff db[3];
    ff_row_adjoint(row.dx, row.dy, row.dz, ab, db);
    if (code & kGhostBit) {  // the ghost's row T(-d)
#pragma unroll
      for (int q = 0; q < 3; ++q) a[q] = ff_neg(a[q]);  // T(-d): linear terms flip
      ff rgG = bgGf, rVG = bvGf, bgb = {0.f, 0.f}, bVb = {0.f, 0.f};
#pragma unroll
      for (int q = 0; q < kNB; ++q) {
        ff_acc(rgG, a[q], ff_neg(cg[q]));
        ff_acc(rVG, a[q], ff_neg(cV[q]));
        ff_acc(bgb, a[q], zg[q]);
        ff_acc(bVb, a[q], zV[q]);
      }
      rgG = ff_norm(rgG);
      rVG = ff_norm(rVG);
      bgb = ff_norm(bgb);
      bVb = ff_norm(bVb);
      const double bgbd = ffs_to_double(bgb.h) + ffs_to_double(bgb.l);
      og += bgbd * dbg_dg;
      oV += bgbd * dbg_dV - (ffs_to_double(bVb.h) + ffs_to_double(bVb.l));
      const ff nbgb = ff_neg(bgb), nbVb = ff_neg(bVb);
#pragma unroll
      for (int q = 0; q < kNB; ++q) {
        ab[q] = {0.f, 0.f};
        ff_acc(ab[q], rgG, zg[q]);
        ff_acc(ab[q], nbgb, cg[q]);
        ff_acc(ab[q], rVG, zV[q]);
        ff_acc(ab[q], nbVb, cV[q]);
      }
      ff dbG[3];
      ff_row_adjoint(ff_neg(row.dx), ff_neg(row.dy), ff_neg(row.dz), ab, dbG);
#pragma unroll
      for (int c = 0; c < 3; ++c) db[c] = ff_sub(db[c], dbG[c]);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const ff g = ff_mul(q == 2 && mir ? ff_neg(db[q]) : db[q], ihf);
      atomicAdd(&A.l0[q][j], ffs_to_double(g.h) + ffs_to_double(g.l));
      sp[q] = ff_add(sp[q], ff_mul(db[q], ihf));
    }
  }
  atomicAdd(&A.lGn[s], og - (ffs_to_double(sg.h) + ffs_to_double(sg.l)));
  atomicAdd(&lVfit[s], oV - (ffs_to_double(sV.h) + ffs_to_double(sV.l)));
  for (int c = 0; c < 3; ++c)
    atomicAdd(&A.l0[c][s], -(ffs_to_double(sp[c].h) + ffs_to_double(sp[c].l)));
}

// ---------------------------------------------------------------- R3
// the state of step n split into float-float pairs for the adjoint's rows:
// positions relative to the column's grid origin in units of h (with the
// floor-mirror height), and velocities, as the forward step splits them (GV:
// the velocity half then holds |gdot|^n and the V of the pass-2 fit, as the
// forward step's pass 2 reads them)
template <bool GV>
__global__ void k_adj_split(const AdjArgs A) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= A.n) return;
  split_state_body(A, s);
  if (GV) split_p1_body(A, s);
}

// pass-1 adjoint: |gdot| and ld to the velocity gradient and Hessians, then
// the least-squares rows to the neighbours' velocities and the positions
template <bool PER>
__global__ void __launch_bounds__(kBlock) k_adj_pass1(const AdjArgs A) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= A.n) return;
  const int n = A.n;
  const double dt = A.K.dt, ih = A.K.inv_h, ih2 = ih * ih;
  const double lVn = A.lVn[s];
  const double div = A.p1[P1_DIV * n + s];
  const double Vi = A.V[s];
  // V^{n+1} = V + dt V div; an Euler stage's fits and closure read V itself
  A.l0[6][s] = lVn * (1.0 + dt * div) + (A.K.euler ? A.lVd[s] : 0.0);
  if (!A.ok[s]) return;
  const double ldiv = lVn * dt * Vi;
  const double Gn = A.p1[P1_GN * n + s];
  double lg[6];
  for (int q = 0; q < 6; ++q) lg[q] = A.lG6[q * n + s];
  const double lGn = A.lGn[s];
  if (Gn > 0.0 && lGn != 0.0) {
    const double h2 = lGn / (2.0 * Gn);
    for (int q = 0; q < 3; ++q) lg[q] += h2 * A.p1[(P1_GD + q) * n + s];
    for (int q = 3; q < 6; ++q) lg[q] += 2.0 * h2 * A.p1[(P1_GD + q) * n + s];
  }
  // gdot = sym(grad u) - div/3 I ; div = trace(grad u)
  const double tr3 = (lg[0] + lg[1] + lg[2]) * (1.0 / 3.0);
  double lc[3][kNB];
  lc[0][0] = (lg[0] - tr3 + ldiv) * ih;
  lc[1][1] = (lg[1] - tr3 + ldiv) * ih;
  lc[2][2] = (lg[2] - tr3 + ldiv) * ih;
  lc[0][1] = lc[1][0] = 0.5 * lg[3] * ih;
  lc[0][2] = lc[2][0] = 0.5 * lg[4] * ih;
  lc[1][2] = lc[2][1] = 0.5 * lg[5] * ih;
  // ld_a = (1/2) Lap u_a + (1/6) d_a div u; columns 3 xx, 4 yy, 5 zz, 6 xy, 7 xz, 8 yz
  const double lx = A.lld[0 * n + s] * ih2, ly = A.lld[1 * n + s] * ih2,
               lz = A.lld[2 * n + s] * ih2;
  const double h6 = 1.0 / 6.0;
  lc[0][3] = (0.5 + h6) * lx; lc[0][4] = 0.5 * lx; lc[0][5] = 0.5 * lx;
  lc[0][6] = h6 * ly;         lc[0][7] = h6 * lz;  lc[0][8] = 0.0;
  lc[1][3] = 0.5 * ly; lc[1][4] = (0.5 + h6) * ly; lc[1][5] = 0.5 * ly;
  lc[1][6] = h6 * lx;  lc[1][7] = 0.0;             lc[1][8] = h6 * lz;
  lc[2][3] = 0.5 * lz; lc[2][4] = 0.5 * lz; lc[2][5] = (0.5 + h6) * lz;
  lc[2][6] = 0.0;      lc[2][7] = h6 * lx;  lc[2][8] = h6 * ly;
  bool any = false;
  for (int f = 0; f < 3; ++f)
    for (int q = 0; q < kNB; ++q) any = any || lc[f][q] != 0.0;
  if (!any) return;
  {
    const double* F = factor_of(A, s);
    double L[kTri];
#pragma unroll
    for (int k = 0; k < kTri; ++k) L[k] = F[(int64_t)k * n + s];
    for (int f = 0; f < 3; ++f) chol9_solve(L, lc[f]);  // lc becomes z_f
  }
  // The rows in float-float (the forward step's coefficients c_f and the z_f
  // split once; the offsets and velocity differences from the split state):
  // the rows' residuals, b = a . z and the row adjoints run on the FP32 pipe,
  // and only the scattered sums are FP64, converted exactly from float-float.
  ff cf[3][kNB], zf[3][kNB];
#pragma unroll
  for (int f = 0; f < 3; ++f)
#pragma unroll
    for (int q = 0; q < kNB; ++q) {
      cf[f][q] = ff_of(A.coef1[(int64_t)(f * kNB + q) * n + s]);
      zf[f][q] = ff_of(lc[f][q]);
    }
  const int mm = A.K.mirror_mode;
  const float sgn[3] = {(float)usign_adj(mm, 0), (float)usign_adj(mm, 1),
                        (float)usign_adj(mm, 2)};
  const float4 hi = A.XU[s].xh, lo = A.XU[s].xl, uh = A.XU[s].uh, ul = A.XU[s].ul;
  const float uih[3] = {uh.x, uh.y, uh.z}, uil[3] = {ul.x, ul.y, ul.z};
  const ff ihf{A.K.ih_h, A.K.ih_l};
  const int m = min(A.cnt[s], A.cap);
  ff su[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}, sp[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  for (int k = 0; k < m; ++k) {
    const uint32_t code = (uint32_t)A.nbr[(int64_t)k * n + s];
    const int j = code & kIndexMask;
    if ((unsigned)j >= (unsigned)n) continue;  // stale or corrupt stencil entry
    const bool mir = code >> 31;
    const FF8& rj = A.XU[j];
    const FFRow row = ff_row_of<PER>(hi, lo, rj.xh, rj.xl, code, A.K);
    ff a[kNB];
    ff_taylor(row, a);
    const float ujh[3] = {rj.uh.x, rj.uh.y, rj.uh.z}, ujl[3] = {rj.ul.x, rj.ul.y, rj.ul.z};
    ff ab[kNB];
#pragma unroll
    for (int q = 0; q < kNB; ++q) ab[q] = {0.f, 0.f};
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      const float sj = mir ? sgn[f] : 1.f;
      ff r = ff_diff(sj * ujh[f], sj * ujl[f], uih[f], uil[f]), b = {0.f, 0.f};
#pragma unroll
      for (int q = 0; q < kNB; ++q) {
        ff_acc(r, a[q], ff_neg(cf[f][q]));
        ff_acc(b, a[q], zf[f][q]);
      }
      r = ff_norm(r);
      b = ff_norm(b);
      atomicAdd(&A.l0[3 + f][j], ffs_to_double(sj * b.h) + ffs_to_double(sj * b.l));
      su[f] = ff_add(su[f], b);
      const ff nb = ff_neg(b);
#pragma unroll
      for (int q = 0; q < kNB; ++q) {
        ff_acc(ab[q], r, zf[f][q]);
        ff_acc(ab[q], nb, cf[f][q]);
      }
    }
    ff db[3];
    ff_row_adjoint(row.dx, row.dy, row.dz, ab, db);
    if (code & kGhostBit) {  // the ghost's row T(-d), right-hand sides 0
      const ff ndx = ff_neg(row.dx), ndy = ff_neg(row.dy), ndz = ff_neg(row.dz);
#pragma unroll
      for (int q = 0; q < 3; ++q) a[q] = ff_neg(a[q]);  // T(-d): linear terms flip
#pragma unroll
      for (int q = 0; q < kNB; ++q) ab[q] = {0.f, 0.f};
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        ff r = {0.f, 0.f}, b = {0.f, 0.f};
#pragma unroll
        for (int q = 0; q < kNB; ++q) {
          ff_acc(r, a[q], ff_neg(cf[f][q]));
          ff_acc(b, a[q], zf[f][q]);
        }
        r = ff_norm(r);
        b = ff_norm(b);
        const ff nb = ff_neg(b);
#pragma unroll
        for (int q = 0; q < kNB; ++q) {
          ff_acc(ab[q], r, zf[f][q]);
          ff_acc(ab[q], nb, cf[f][q]);
        }
      }
      ff dbG[3];
      ff_row_adjoint(ndx, ndy, ndz, ab, dbG);
#pragma unroll
      for (int q = 0; q < 3; ++q) db[q] = ff_sub(db[q], dbG[q]);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const ff g = ff_mul(q == 2 && mir ? ff_neg(db[q]) : db[q], ihf);
      atomicAdd(&A.l0[q][j], ffs_to_double(g.h) + ffs_to_double(g.l));
      sp[q] = ff_add(sp[q], ff_mul(db[q], ihf));
    }
  }
  for (int f = 0; f < 3; ++f)
    atomicAdd(&A.l0[3 + f][s], -(ffs_to_double(su[f].h) + ffs_to_double(su[f].l)));
  for (int q = 0; q < 3; ++q)
    atomicAdd(&A.l0[q][s], -(ffs_to_double(sp[q].h) + ffs_to_double(sp[q].l)));
}

// dst[f][s] = src[f][idx[s]] (caller order to sorted order)
__global__ void k_gather_fields(int n, const int32_t* __restrict__ idx,
                                const double* const* __restrict__ src,
                                double* const* __restrict__ dst, int nf) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int o = idx[s];
  if ((unsigned)o >= (unsigned)n) return;
  for (int f = 0; f < nf; ++f) dst[f][s] = src[f][o];
}

void launch_gather_fields(int n, const int32_t* idx, const double* const* src, double* const* dst,
                          int nf, cudaStream_t st) {
  k_gather_fields<<<(n + 255) / 256, 256, 0, st>>>(n, idx, src, dst, nf);
}

void launch_adjoint_step(const AdjArgs& A, cudaStream_t st) {
  const int nb = (A.n + kBlock - 1) / kBlock;
  k_adj_prepare<<<nb, kBlock, 0, st>>>(A);
  k_adj_accel<<<nb, kBlock, 0, st>>>(A);
  k_adj_split<true><<<nb, kBlock, 0, st>>>(A);
  if (A.K.periodic) k_adj_pass2<true><<<nb, kBlock, 0, st>>>(A);
  else k_adj_pass2<false><<<nb, kBlock, 0, st>>>(A);
  k_adj_split<false><<<nb, kBlock, 0, st>>>(A);
  if (A.K.periodic) k_adj_pass1<true><<<nb, kBlock, 0, st>>>(A);
  else k_adj_pass1<false><<<nb, kBlock, 0, st>>>(A);
}

}  // namespace lp
