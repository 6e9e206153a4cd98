// Internal device-side definitions shared by the CUDA translation units of the
// LP step library. Nothing here is part of the C ABI (see include/lp.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "lp.h"
#include "ff_split.cuh"

namespace lp {

constexpr uint32_t kMirrorBit = 0x80000000u;
// ghost particle: point reflection, through the particle, of the entry in the
// low bits (free boundary, Sec. 3.1 item 9); indices are below 2^30
constexpr uint32_t kGhostBit = 0x40000000u;
constexpr uint32_t kIndexMask = 0x3fffffffu;
constexpr int kNB = 9;            // quadratic Taylor basis in 3D, no constant term
constexpr int kTri = 45;          // packed lower triangle of a 9x9 matrix
constexpr int kMaxColumns = 4096;
constexpr int kBlock = 128;       // default threads per block of the per-particle kernels
constexpr int kMaxBlock = 256;    // largest block size the tuner may pick
#ifndef LP_FILTER_CHUNK
#define LP_FILTER_CHUNK 8
#endif
constexpr int kFilterChunk = LP_FILTER_CHUNK;  // candidates whose gathers the filter issues together
#ifndef LP_ROW_ORDER
#define LP_ROW_ORDER 1  // fit threads take particles sorted by stencil size (k_row_order)
#endif
#ifndef LP_SEARCH_CHUNK
#define LP_SEARCH_CHUNK 4
#endif
constexpr int kSearchChunk = LP_SEARCH_CHUNK;  // cell-range entries the search loads together
constexpr int kMaxFields = 16;    // lp_fit_derivatives
constexpr int kMaxCand = 128;     // candidate buffer of the keep-nearest search

// Uniform cell grid of one column. Cell edge >= the largest stencil radius,
// cell coordinates clamped into the grid (clamping keeps any two points within
// one cell of each other per axis when they are within one cell edge).
struct GridCol {
  double ox, oy, oz;     // origin
  double icx, icy, icz;  // 1 / cell edge per axis
  double Lx, Ly;         // periods (0: not periodic); a periodic axis has origin 0 and
                         // whole cells over [0, L), and its neighbour cells wrap
  float Lxf, Lyf;        // the periods rounded to float (FP32 prefilter)
  int nx, ny, nz;
  int64_t cell_off;      // first global cell id of this column
};

// per-column material parameters
struct ColMui {
  double mu_s, mu_2, I0, d, rho_s;
  // float-float (hi, lo) constants of the inertial closure for pass 2 of
  // LP_MIXED_FF, a = phi_c - phi_min: k = 4 a^2 d^2, a I0, a mu_s I0, mu_2,
  // a I0 (mu_2 - mu_s)
  float kf[2], aI0f[2], bf[2], mu2f[2], cf[2];
};

// constants of one step
struct StepConsts {
  double phi_c, phi_min, phi_max, alpha, beta;
  double h, inv_h, radius, r2;
  double gx, gy, gz, floor_z, dt;
  int mirror_mode;
  int cap;
  // free-surface ghosts: fixed-point grid K (power of two, K r <= 8192),
  // round((K r)^2), K h, round((K h / 2)^2), 1/phi_G, phi_c - phi_G
  int free_surface;
  int euler;  // Heun stage: pass 2 takes V^n, x advances with u^n
  // periodic boundaries: periods (0: not periodic), their float-float copies
  // in units of h, and the integer periods round(K L) of the ghost test
  int periodic;
  double Lx, Ly;
  float Lhx_h, Lhx_l, Lhy_h, Lhy_l;
  float ih_h, ih_l, ih2_h, ih2_l;  // 1/h and 1/h^2 as float-float
  float phic_h, phic_l;            // phi_c as float-float
  float rho;                       // bound on |offset| / h of a stencil entry (r/h, rounded up)
  long long ghost_PX, ghost_PY;
  double ghost_grid, ghost_hk, ghost_V, ghost_num;
  long long ghost_R2, ghost_clear2;
};

// device diagnostics, accumulated until lp_ctx_sync
struct DevDiag {
  unsigned int flags;
  int min_stencil, max_stencil;
  int pad;
  unsigned long long n_overflow, n_fallback, n_gas, n_quasistatic, n_over_c, n_nonfinite,
      n_below_floor, n_stencil_rows, n_stencils, n_ghosts;
};

__host__ __device__ constexpr int tri(int r, int c) { return r * (r + 1) / 2 + c; }

// Periodic boundaries (Sec. 3.1 item 9): the offset d along an axis of period
// L (0: not periodic) taken as its nearest image, and a position moved back
// into [0, L) (a step moves a particle far less than L). Both in FP64 with
// rounded operations in a fixed order.
__device__ __forceinline__ double min_image(double d, double L) {
  if (L > 0.0) {
    if (d > __dmul_rn(0.5, L)) return __dsub_rn(d, L);
    if (d < -__dmul_rn(0.5, L)) return __dadd_rn(d, L);
  }
  return d;
}
__device__ __forceinline__ double wrap_pos(double x, double L) {
  if (L > 0.0) {
    if (x >= L) return __dsub_rn(x, L);
    if (x < 0.0) return __dadd_rn(x, L);
  }
  return x;
}

// split position (x, y, z, mirror height) and velocity of one particle, hi
// and lo, in one 64-byte record: a row of pass 1 gathers one cache line, the
// Gram kernel the first 32-byte sector. Once pass 1 is done the velocity half
// is dead and uh holds the split |gdot|^n and V of pass 2 instead (gv: hi,
// lo, hi, lo), so a row of pass 2 gathers one line as well.
struct __align__(64) FF8 {
  float4 xh, xl, uh, ul;
};

// ------------------------------------------------------------ float-float
// Unevaluated sums hi + lo of two floats (about 48 significant bits), built
// from the error-free transformations TwoSum (Knuth) and TwoProduct (an FMA
// gives the exact rounding error of a product). The _rn intrinsics keep the
// compiler from contracting or reordering these steps.
struct ff {
  float h, l;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, {-b.h, -b.l}); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_scale(ff a, float s) { return {a.h * s, a.l * s}; }  // s = 2^k
// acc += a b, keeping acc unnormalised (lo collects all low-order terms)
__device__ __forceinline__ void ff_acc(ff& acc, ff a, ff b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const ff s = two_sum(acc.h, p);
  acc.h = s.h;
  acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, e));
}
// Seeded sums: when |acc.h| >= |a.h b.h| is known (the sum starts at a large
// power of two, see gram_ff_body), the error of the high-part addition is
// captured exactly by FastTwoSum (3 operations instead of TwoSum's 6).
__device__ __forceinline__ void ff_acc_seeded(ff& acc, ff a, ff b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const ff s = fast_two_sum(acc.h, p);
  acc.h = s.h;
  acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, e));
}
__device__ __forceinline__ void ff_acc1_seeded(ff& acc, ff a) {
  const ff s = fast_two_sum(acc.h, a.h);
  acc.h = s.h;
  acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, a.l));
}
// smallest power of two >= v (v positive and normal)
__device__ __forceinline__ float pow2_ceil(float v) {
  return __int_as_float((__float_as_int(v) + 0x007fffff) & 0x7f800000);
}
// acc += a
__device__ __forceinline__ void ff_acc1(ff& acc, ff a) {
  const ff s = two_sum(acc.h, a.h);
  acc.h = s.h;
  acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, a.l));
}
__device__ __forceinline__ ff ff_norm(ff a) { return fast_two_sum(a.h, a.l); }
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }
// 1/sqrt(d) in float-float: the correctly rounded FP32 value refined by one
// Newton-Raphson step y + (y/2)(1 - d y^2), whose residual is formed exactly
// enough in float-float (y^2 is split exactly with an FMA).
__device__ __forceinline__ ff ff_rsqrt(ff d) {
  const float y = __frsqrt_rn(d.h);
  const float p = __fmul_rn(y, y);
  const ff t = ff_mul(d, ff{p, __fmaf_rn(y, y, -p)});
  const float delta = __fsub_rn(__fsub_rn(1.f, t.h), t.l);
  return fast_two_sum(y, __fmul_rn(__fmul_rn(0.5f, y), delta));
}
// 1/d in float-float: the rounded FP32 reciprocal refined by one Newton step
// y + y (1 - d y), the residual formed in float-float
__device__ __forceinline__ ff ff_recip(ff d) {
  const float y = __frcp_rn(d.h);
  const ff t = ff_mul(d, ff{y, 0.f});
  const float e = __fsub_rn(__fsub_rn(1.f, t.h), t.l);
  return fast_two_sum(y, __fmul_rn(y, e));
}
// (RN(d), RN(d - RN(d))): integer split on the fast range (ff_split.cuh), FP64
// conversions elsewhere; the same bits either way
__device__ __forceinline__ ff ff_of(double d) {
  float h, l;
  if (ff_split_fast(d, &h, &l)) return {h, l};
  h = __double2float_rn(d);
  return {h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.h + (double)a.l; }

// clamped cell coordinate; NaN maps to 0 (fmax returns the non-NaN operand)
__device__ __forceinline__ int cell_coord(double p, double o, double inv_c, int n) {
  double t = (p - o) * inv_c;
  t = fmin(fmax(t, 0.0), (double)(n - 1));
  return (int)t;
}

__device__ __forceinline__ int64_t cell_id(const GridCol& g, int cx, int cy, int cz) {
  return g.cell_off + ((int64_t)cz * g.ny + cy) * g.nx + cx;
}

// warp-aggregated counter increment (one atomic per warp)
__device__ __forceinline__ void warp_count(unsigned long long* ctr, bool pred) {
  unsigned int b = __ballot_sync(0xffffffffu, pred);
  if (b && (threadIdx.x & 31) == (__ffs(b) - 1)) atomicAdd(ctr, (unsigned long long)__popc(b));
}

// indices of the per-particle pass-1 outputs in the SoA block p1[k*n + s]
enum { P1_GD = 0, P1_GN = 6, P1_LD = 7, P1_VN = 10, P1_DIV = 11, P1_N = 12 };

// Filter skipping between Verlet searches. A particle whose stencil was
// computed at step t_c keeps it while every candidate stays on the same side
// of the radius: the pair distance moves by at most the two particles'
// displacements since t_c, each at most twice the running maximum of their
// displacement from the search positions. So with marg_i the smallest
// distance of a candidate of i from the radius at t_c (a lower bound, net of
// the FP32 rounding) and dmax the running maxima since the search,
// 2 (dmax_i + max_j dmax_j) < marg_i means the exact test would keep the same
// candidates, in the same order. All members NULL: the filter always runs.
struct VerletSkip {
  float* marg;          // per particle, at its last filter; < 0 forces the filter
  float* dmax;          // per particle, running maximum displacement since the search
  unsigned* dmax_all;   // maximum of dmax over all particles (bits of a float >= 0)
};

struct StepArgs {
  int n, cap;
  const double *x, *y, *z, *u, *v, *w, *V;  // state at time n (sorted order)
  double *xo, *yo, *zo, *uo, *vo, *wo, *Vo; // state at n+1
  const int32_t *nbr, *cnt, *colid;
  const ColMui* mui;
  double* fac;      // FP64 Cholesky factors, 45 * n (k-major)
  float* facf;      // FP32 Cholesky factors, 45 * n (k-major)
  int32_t* fbslot;  // per particle: fallback slot or -1
  int32_t* fb_list; // fallback particles
  int32_t* fb_count;
  int fb_cap;
  double* p1;       // pass-1 outputs, P1_N * n
  double* fbgrad;   // pass-2 fallback results, 6 per slot
  DevDiag* dg;
  StepConsts K;
  double* coef1;    // optional (FP64 only): pass-1 coefficients, 27 * n (k-major)
  double* coef2;    // optional (FP64 only): pass-2 coefficients of |gdot|, V^{n+1}, 18 * n
  // float-float mode (LP_MIXED_FF): scaled positions X = (x - origin)/h split
  // into hi and lo floats (w = mirror height), velocities split likewise,
  // |gdot| and V^{n+1} split (hi, lo, hi, lo), Gram matrices in float-float
  const GridCol* grids;
  FF8* XU;  // split positions and velocities
  float2* R1;   // LP_MIXED_FF: pass 1's right-hand sides (27 float-float, k-major)
  float2* P1s;  // LP_MIXED_FF: gdot (6) and ld (3) of pass 1 as float-float, k-major
                // (null in the other modes)

  int4* Xfix;       // free surface: round(K (x, y, z, 2 floor_z - z)) per particle,
                    // relative to the column's fixed-point origin
  int32_t* gcnt;    // free surface: entries with a ghost, at the end of each stencil
  const int32_t* glist;  // free surface: the particles with ghost entries (compact), and
  const int* gcount;     // their number (set by the ghost kernel of the same stencils)
  float *Tg, *T2;   // free surface: sums over those entries and their ghosts
                    // (Gram moments 62 x n, pass-2 right-hand sides 36 x n)
  float2* Lff;      // 45 * n: float-float Cholesky factor of the Gram matrix,
                    // (hi, lo) pairs, k-major; the diagonal holds 1/L_jj
  const int32_t* perm;  // LP_MIXED_FF: particle of each fit thread (stencil
                        // sizes sorted within groups of 128), or NULL
  // Verlet candidate lists: positions at the last search and the flag that
  // requests a new search when a particle has moved more than skin/2
  const double* xref;  // 3 * n, or NULL when candidate lists are off
  double half_skin2;
  int* need_search;
  VerletSkip vskip;    // running maximum displacements for filter skipping
};

struct FitArgs {
  int n, cap, nf;
  const double *x, *y, *z;
  const int32_t *nbr, *cnt;
  const double* fields[kMaxFields];
  double msign[kMaxFields];
  double inv_h, f2;
  double* coeffs;     // n x nf x 9
  // LP_MIXED_FF: split positions (xh, xl of each record), split fields
  // (nf x n, k-major) and the float-float factors (45 x n)
  FF8* xs;
  float2* fs;
  float2* lf;
  int32_t* fb_list;
  int32_t* fb_count;
  int fb_cap;
  DevDiag* dg;
};

// arguments of the persistent step kernel (persistent.cu)
struct PersistArgs {
  StepArgs S;  // pass 1 / pass 2 (state pointers of the sorted order)
  int n;
  int rebuild;
  int64_t ncell;
  // sort phases
  const double *xs, *ys, *zs;  // positions before the sort
  const int32_t *colid_in, *ids_in;
  int32_t *colid_out, *ids_out;
  const GridCol* grids;
  uint32_t *key, *count, *fill, *start, *tile;
  int ntiles;
  int32_t* tmp;
  const double* const* src;
  double* const* dst;
  int nsrc;
  float4* pf;
  // neighbour phase
  double radius, floor_z;
  int mirror_mode, cap;
  int32_t *nbr, *cnt;
  // Verlet candidate lists (search != nullptr): the sort and a search within
  // radius + skin run only when *search is set, the exact filter every
  // rebuild step; otherwise the gather is the identity (iota)
  int* search;
  const int32_t* iota;
  int32_t *cand, *ccnt;
  int capc;
  double rsearch;
  double* xref;
  // Heun's method, first stage: copy the (sorted) state here before pass 1
  double* y0[7];
  int save_y0;
  // barrier: [0] arrivals, [1] generation
  unsigned* bar;
  unsigned long long max_spins;
  unsigned extra_arrivals;  // 0 in production; > 0 only to test the bounded wait
  // profiling (lp_ctx_profile): nanoseconds per phase (LP_PHASE_*), added by
  // thread 0 of block 0 after the grid barrier that closes each phase, and
  // the last mark in [LP_NPHASES]; NULL when profiling is off
  unsigned long long* phase_ns;
};

// arguments of the adjoint kernels (adjoint.cu)
struct AdjArgs {
  int n, cap;
  const double *x, *y, *z, *u, *v, *w, *V;  // forward state at step n (sorted order)
  const GridCol* grids;  // the columns' cell grids (origins of the split positions)
  FF8* XU;               // the state of step n split into float-float pairs
  const int32_t *nbr, *cnt, *colid, *fbslot;
  const ColMui* mui;
  const double* fac;     // FP64 Cholesky factors, 45 * n
  const double* p1;      // pass-1 outputs (P1_*)
  const double* coef1;   // pass-1 coefficients, 27 * n
  const double* coef2;   // pass-2 coefficients, 18 * n
  const double* fbgrad;  // pass-2 gradients of QR-path stencils, 6 per slot
  StepConsts K;
  const double* l1[7];   // adjoint of the state at n+1: x, y, z, u, v, w, V
  double* l0[7];         // adjoint of the state at n (output)
  double* lGn;           // adjoint of |gdot|^n (accumulated)
  double* lVn;           // adjoint of V^{n+1} (accumulated)
  double* lVd;           // Euler stage (K.euler): adjoint of the V^n that the fits and
                         // the closure read (accumulated; added to l0 V directly)
  double* lG6;           // adjoint of gdot from the acceleration, 6 * n
  double* lld;           // adjoint of ld, 3 * n
  double* zz;            // G^{-1} cbar of pass 2 (|gdot|, V^{n+1}), 18 * n
  double* dtheta;        // dL/d(mu_s, mu_2, I0), accumulated
  DevDiag* dg;
  uint8_t* ok;           // per particle: 1 if the fit adjoint is available
  double* facx;          // FP64 factors of the QR-path stencils, 45 * n
};

// ------------------------------------------------------------------ closure
// mu(I) closure of Sec. 2.3 at solid fraction phi (inertial regime):
//   M = -4 a^2 d^2/(phi_c-phi)^2, N = -M mu, S = dM/dphi, R = dN/dphi,
//   mu = (a mu_s I0 + mu_2 (phi_c-phi)) / (a I0 + phi_c - phi).
struct Closure {
  double M, N, S, R, mu;
};
__device__ __forceinline__ Closure closure_at(double phi, const ColMui& m, double phi_c,
                                              double phi_min) {
  const double a = phi_c - phi_min;
  const double w = phi_c - phi;
  const double k = 4.0 * a * a * m.d * m.d;
  Closure c;
  const double iw = 1.0 / w;
  c.M = -k * iw * iw;
  const double den = a * m.I0 + w;
  const double iden = 1.0 / den;
  c.mu = (a * m.mu_s * m.I0 + m.mu_2 * w) * iden;
  c.N = -c.M * c.mu;
  c.S = -2.0 * k * iw * iw * iw;
  const double dmu = -(a * m.I0 * (m.mu_2 - m.mu_s)) * iden * iden;
  c.R = -c.S * c.mu - c.M * dmu;
  return c;
}

// ---------------------------------------------------------- 9x9 Cholesky
// In-place factorisation of a packed SPD matrix (lower triangle). On return
// a[tri(i,j)] = L_ij for j < i and a[tri(j,j)] = 1/L_jj. Returns false if a
// pivot falls below rel_tol times the original diagonal entry (then the
// caller falls back to pivoted QR).
template <typename T>
__device__ __forceinline__ bool chol9(T* a, T rel_tol) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < kNB; ++j) {
    T d = a[tri(j, j)];
    const T d0 = d;
#pragma unroll
    for (int k = 0; k < j; ++k) d -= a[tri(j, k)] * a[tri(j, k)];
    const bool good = d > rel_tol * d0;
    ok = ok && good;
    const T inv = good ? T(1) / sqrt(d) : T(0);
    a[tri(j, j)] = inv;
#pragma unroll
    for (int i = j + 1; i < kNB; ++i) {
      T s = a[tri(i, j)];
#pragma unroll
      for (int k = 0; k < j; ++k) s -= a[tri(i, k)] * a[tri(j, k)];
      a[tri(i, j)] = s * inv;
    }
  }
  return ok;
}

// Solve L L^T c = b with a factor from chol9 (b overwritten by c).
template <typename T, typename TB>
__device__ __forceinline__ void chol9_solve(const T* L, TB* b) {
#pragma unroll
  for (int i = 0; i < kNB; ++i) {
    TB s = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s -= TB(L[tri(i, k)]) * b[k];
    b[i] = s * TB(L[tri(i, i)]);
  }
#pragma unroll
  for (int i = kNB - 1; i >= 0; --i) {
    TB s = b[i];
#pragma unroll
    for (int k = i + 1; k < kNB; ++k) s -= TB(L[tri(k, i)]) * b[k];
    b[i] = s * TB(L[tri(i, i)]);
  }
}

// Taylor-row moments of one stencil: the 31 distinct moments of the 9x9 Gram
// matrix (degree 2, 3 and 4 in the scaled offsets).
template <typename T>
struct Moments {
  T xx, yy, zz, xy, xz, yz;                                 // degree 2
  T xxx, yyy, zzz, xxy, xxz, xyy, yyz, xzz, yzz, xyz;      // degree 3
  T xxxx, yyyy, zzzz, xxxy, xxxz, xyyy, yyyz, xzzz, yzzz,  // degree 4
      xxyy, xxzz, yyzz, xxyz, xyyz, xyzz;
  __device__ __forceinline__ void zero() {
    xx = yy = zz = xy = xz = yz = T(0);
    xxx = yyy = zzz = xxy = xxz = xyy = yyz = xzz = yzz = xyz = T(0);
    xxxx = yyyy = zzzz = xxxy = xxxz = xyyy = yyyz = xzzz = yzzz = T(0);
    xxyy = xxzz = yyzz = xxyz = xyyz = xyzz = T(0);
  }
  __device__ __forceinline__ void add(T dx, T dy, T dz) {
    const T qxx = dx * dx, qyy = dy * dy, qzz = dz * dz;
    const T qxy = dx * dy, qxz = dx * dz, qyz = dy * dz;
    xx += qxx; yy += qyy; zz += qzz; xy += qxy; xz += qxz; yz += qyz;
    xxx += dx * qxx; yyy += dy * qyy; zzz += dz * qzz;
    xxy += dy * qxx; xxz += dz * qxx; xyy += dx * qyy;
    yyz += dz * qyy; xzz += dx * qzz; yzz += dy * qzz; xyz += dz * qxy;
    xxxx += qxx * qxx; yyyy += qyy * qyy; zzzz += qzz * qzz;
    xxxy += qxx * qxy; xxxz += qxx * qxz; xyyy += qyy * qxy;
    yyyz += qyy * qyz; xzzz += qzz * qxz; yzzz += qzz * qyz;
    xxyy += qxx * qyy; xxzz += qxx * qzz; yyzz += qyy * qzz;
    xxyz += qxx * qyz; xyyz += qyy * qxz; xyzz += qzz * qxy;
  }
  // Gram matrix of the columns [dx, dy, dz, dx^2/2, dy^2/2, dz^2/2, dx dy,
  // dx dz, dy dz], packed lower triangle.
  __device__ __forceinline__ void gram(T* g) const {
    const T h = T(0.5), q = T(0.25);
    g[tri(0, 0)] = xx;
    g[tri(1, 0)] = xy;       g[tri(1, 1)] = yy;
    g[tri(2, 0)] = xz;       g[tri(2, 1)] = yz;       g[tri(2, 2)] = zz;
    g[tri(3, 0)] = h * xxx;  g[tri(3, 1)] = h * xxy;  g[tri(3, 2)] = h * xxz;
    g[tri(3, 3)] = q * xxxx;
    g[tri(4, 0)] = h * xyy;  g[tri(4, 1)] = h * yyy;  g[tri(4, 2)] = h * yyz;
    g[tri(4, 3)] = q * xxyy; g[tri(4, 4)] = q * yyyy;
    g[tri(5, 0)] = h * xzz;  g[tri(5, 1)] = h * yzz;  g[tri(5, 2)] = h * zzz;
    g[tri(5, 3)] = q * xxzz; g[tri(5, 4)] = q * yyzz; g[tri(5, 5)] = q * zzzz;
    g[tri(6, 0)] = xxy;      g[tri(6, 1)] = xyy;      g[tri(6, 2)] = xyz;
    g[tri(6, 3)] = h * xxxy; g[tri(6, 4)] = h * xyyy; g[tri(6, 5)] = h * xyzz;
    g[tri(6, 6)] = xxyy;
    g[tri(7, 0)] = xxz;      g[tri(7, 1)] = xyz;      g[tri(7, 2)] = xzz;
    g[tri(7, 3)] = h * xxxz; g[tri(7, 4)] = h * xyyz; g[tri(7, 5)] = h * xzzz;
    g[tri(7, 6)] = xxyz;     g[tri(7, 7)] = xxzz;
    g[tri(8, 0)] = xyz;      g[tri(8, 1)] = yyz;      g[tri(8, 2)] = yzz;
    g[tri(8, 3)] = h * xxyz; g[tri(8, 4)] = h * yyyz; g[tri(8, 5)] = h * yzzz;
    g[tri(8, 6)] = xyyz;     g[tri(8, 7)] = xyzz;     g[tri(8, 8)] = yyzz;
  }
};

// Taylor row of a scaled offset.
template <typename T>
__device__ __forceinline__ void taylor_row(T dx, T dy, T dz, T* a) {
  a[0] = dx; a[1] = dy; a[2] = dz;
  a[3] = T(0.5) * dx * dx; a[4] = T(0.5) * dy * dy; a[5] = T(0.5) * dz * dz;
  a[6] = dx * dy; a[7] = dx * dz; a[8] = dy * dz;
}

// ------------------------------------------------ pivoted Householder QR
// Least-squares solve of A c = B by Householder QR with column pivoting
// (largest remaining column norm, ties to the lower column), rank =
// #{|R_kk| > 1e-8 |R_00|}, basic solution (coefficients beyond the rank are
// zero). A: m x 9 row-major, B: m x nf row-major (both overwritten), C: nf x 9.
__device__ inline int qr_pivoted_solve(int m, double* A, int nf, double* B, double* C) {
  int perm[kNB];
  double rdiag[kNB];
  for (int j = 0; j < kNB; ++j) perm[j] = j;
  const int kmax = m < kNB ? m : kNB;
  int steps = 0;
  for (int k = 0; k < kmax; ++k) {
    int best = k;
    double bestn = -1.0;
    for (int j = k; j < kNB; ++j) {
      double s = 0.0;
      for (int i = k; i < m; ++i) s += A[i * kNB + j] * A[i * kNB + j];
      if (s > bestn) { bestn = s; best = j; }
    }
    if (best != k) {
      for (int i = 0; i < m; ++i) {
        double t = A[i * kNB + k]; A[i * kNB + k] = A[i * kNB + best]; A[i * kNB + best] = t;
      }
      int t = perm[k]; perm[k] = perm[best]; perm[best] = t;
    }
    double ss = 0.0;
    for (int i = k; i < m; ++i) ss += A[i * kNB + k] * A[i * kNB + k];
    const double alpha = sqrt(ss);
    if (alpha == 0.0) break;
    const double sgn = A[k * kNB + k] >= 0.0 ? 1.0 : -1.0;
    // Householder vector v = x + sgn |x| e_1 kept in column k, rows k..m-1
    const double v0 = A[k * kNB + k] + sgn * alpha;
    double vtv = v0 * v0;
    for (int i = k + 1; i < m; ++i) vtv += A[i * kNB + k] * A[i * kNB + k];
    for (int j = k + 1; j < kNB; ++j) {
      double s = v0 * A[k * kNB + j];
      for (int i = k + 1; i < m; ++i) s += A[i * kNB + k] * A[i * kNB + j];
      const double f = 2.0 * s / vtv;
      A[k * kNB + j] -= f * v0;
      for (int i = k + 1; i < m; ++i) A[i * kNB + j] -= f * A[i * kNB + k];
    }
    for (int q = 0; q < nf; ++q) {
      double s = v0 * B[k * nf + q];
      for (int i = k + 1; i < m; ++i) s += A[i * kNB + k] * B[i * nf + q];
      const double f = 2.0 * s / vtv;
      B[k * nf + q] -= f * v0;
      for (int i = k + 1; i < m; ++i) B[i * nf + q] -= f * A[i * kNB + k];
    }
    rdiag[k] = -sgn * alpha;
    A[k * kNB + k] = rdiag[k];
    steps = k + 1;
  }
  int rank = 0;
  if (steps > 0) {
    const double r0 = fabs(rdiag[0]);
    for (int k = 0; k < steps; ++k) {
      if (fabs(rdiag[k]) > 1e-8 * r0) rank = k + 1;
      else break;
    }
  }
  for (int q = 0; q < nf; ++q) {
    double y[kNB];
    for (int k = rank - 1; k >= 0; --k) {
      double s = B[k * nf + q];
      for (int j = k + 1; j < rank; ++j) s -= A[k * kNB + j] * y[j];
      y[k] = s / rdiag[k];
    }
    for (int j = 0; j < kNB; ++j) C[q * kNB + j] = 0.0;
    for (int k = 0; k < rank; ++k) C[q * kNB + perm[k]] = y[k];
  }
  return rank;
}

}  // namespace lp
