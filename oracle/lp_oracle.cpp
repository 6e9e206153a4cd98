// Plain FP64 CPU oracle of the Lagrangian-particle (LP) granular-flow time step
// (Zepeda & Samulyak, "Computational Model for Granular Flows based on the
// Lagrangian Particle Method", arXiv 2206.14061).
//
// TEST INFRASTRUCTURE ONLY. This file is the slow, obviously-correct reference
// that the CUDA path is checked against. Only tests, the smoke check and the
// CPU-baseline leg of the benchmark may load it. It shares no code, header,
// table or constant with the CUDA library, and the CUDA library never calls it.
//
// Built with -ffp-contract=off so that every a*b+c is two rounded operations.
//
// What it computes, step by step, in the paper's order (Sec. 3.1):
//   * neighbour search (Sec. 3.1 items 5-6): all j != i with
//     ((dx*dx)+(dy*dy))+(dz*dz) <= r_i*r_i, by brute force over all pairs or by
//     an independent uniform-grid scan; plus floor mirror particles (Sec. 3.1
//     item 9, solid boundary) j* = (x_j, y_j, 2 f - z_j), tested with the same
//     predicate (the particle's own mirror included);
//   * optionally (free_surface = 1) ghost particles at free boundaries (Sec. 3.1
//     items 6 and 9): a particle whose stencil is one-sided gets the point
//     reflections of its inner entries; a ghost carries the particle's velocity,
//     a solid fraction just below phi_min and the |gdot| that keeps the
//     inertial pressure continuous (see add_ghosts for the test and placement
//     the paper leaves open);
//   * optionally (period_x / period_y > 0) periodic boundaries along x and/or
//     y (Sec. 3.1 item 9): offsets are nearest images, positions stay in
//     [0, L);
//   * GFD least-squares fit (Sec. 3.1 item 7): 3D form of the 2D Taylor matrix
//     with rows  [dx, dy, dz, dx^2/2, dy^2/2, dz^2/2, dx dy, dx dz, dy dz]
//     (offsets divided by h), right-hand side s_k - s_i, solved by Householder
//     QR with column pivoting; rank = #{|R_kk| > 1e-8 |R_00|}; basic solution;
//   * strain-rate tensor, divergence, |gdot| = sqrt(gdot:gdot / 2)  (Sec. 2.2);
//   * mu(I) closure M, N, S, R of Sec. 2.3, with R = dN/dphi (the printed R has
//     the sign of its second term flipped; see the R function below);
//   * three-regime pressure law (Sec. 2.2.1) and the explicit update of
//     V, u (Sec. 3.1 item 8) and x (Sec. 3.1 item 10).
//
// A forward-mode dual number with three directions (mu_s, mu_2, I0) runs the
// same templated step to give the tangent-linear reference for the adjoint.
// Regimes, pivots and neighbour topology are taken from the value part.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

// ---------------------------------------------------------------- scalars ---

struct Dual3 {
  double v;
  double d[3];
  Dual3() : v(0.0), d{0.0, 0.0, 0.0} {}
  Dual3(double x) : v(x), d{0.0, 0.0, 0.0} {}  // NOLINT: implicit promotion
};
static inline Dual3 operator+(const Dual3& a, const Dual3& b) {
  Dual3 r(a.v + b.v);
  for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
static inline Dual3 operator-(const Dual3& a, const Dual3& b) {
  Dual3 r(a.v - b.v);
  for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
static inline Dual3 operator-(const Dual3& a) {
  Dual3 r(-a.v);
  for (int k = 0; k < 3; ++k) r.d[k] = -a.d[k];
  return r;
}
static inline Dual3 operator*(const Dual3& a, const Dual3& b) {
  Dual3 r(a.v * b.v);
  for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
static inline Dual3 operator/(const Dual3& a, const Dual3& b) {
  Dual3 r(a.v / b.v);
  for (int k = 0; k < 3; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) / b.v;
  return r;
}
static inline Dual3& operator+=(Dual3& a, const Dual3& b) { return a = a + b; }
static inline Dual3& operator-=(Dual3& a, const Dual3& b) { return a = a - b; }
// sqrt: the derivative at exactly 0 is taken as 0 (non-smooth point of |gdot|).
static inline Dual3 sqrt(const Dual3& a) {
  Dual3 r(std::sqrt(a.v));
  double k = r.v > 0.0 ? 0.5 / r.v : 0.0;
  for (int j = 0; j < 3; ++j) r.d[j] = k * a.d[j];
  return r;
}
static inline double val(double x) { return x; }
static inline double val(const Dual3& x) { return x.v; }
using std::sqrt;

// ------------------------------------------------------------- parameters ---

extern "C" {

// Material, EOS and numerical parameters of one particle set (one column).
typedef struct {
  double mu_s, mu_2, I0, d, rho_s;            // mu(I) law, Sec. 2.2 (rho_s = phi_s)
  double phi_c, phi_min, phi_max, alpha, beta;  // pressure law, Sec. 2.2.1
  double h, radius;                           // lattice spacing, stencil radius
  double gx, gy, gz;                          // body force
  double floor_z, dt;
  int32_t mirror_mode;  // 0 none, 1 no-slip (u* = -u), 2 free-slip (w* = -w)
  int32_t free_surface;  // 1: ghost particles complete free-surface stencils
  int32_t time_scheme;   // 0: the paper's step (V first), 1: Heun's method (RK2)
  int32_t pad;
  double period_x, period_y;  // > 0: periodic in x / y with positions in [0, L)
} orc_params;

typedef struct {
  int64_t n_gas, n_inertial, n_quasistatic, n_over_c, n_below_floor,
      n_rank_deficient, min_stencil, max_stencil, n_ghosts;
} orc_diag;

}  // extern "C"

static const uint32_t MIRROR_BIT = 0x80000000u;
// Ghost particle (free boundary, Sec. 3.1 item 9): the point reflection,
// through particle i, of the stencil entry (j, mirror flag) of i.
static const uint32_t GHOST_BIT = 0x40000000u;
static const uint32_t INDEX_MASK = 0x3fffffffu;

// ------------------------------------------------------- neighbour search ---

// Periodic boundaries (Sec. 3.1 item 9): offset d along an axis of period L
// (L = 0: not periodic), taken as its nearest periodic image; unique when
// L > 2 r.
static inline double min_image(double d, double L) {
  if (L > 0.0) {
    if (d > 0.5 * L) d = d - L;
    else if (d < -0.5 * L) d = d + L;
  }
  return d;
}
struct Periods {
  double Lx = 0.0, Ly = 0.0;
};
template <class T>
static inline T min_image_t(const T& d, double L) {
  if (L > 0.0) {
    if (val(d) > 0.5 * L) return d - T(L);
    if (val(d) < -0.5 * L) return d + T(L);
  }
  return d;
}
// position moved back into [0, L) (a step moves a particle far less than L)
template <class T>
static inline T wrap_t(const T& x, double L) {
  if (L > 0.0) {
    if (val(x) >= L) return x - T(L);
    if (val(x) < 0.0) return x + T(L);
  }
  return x;
}

// Inclusion predicate: d^2 <= r^2, evaluated in FP64 left to right with no
// contraction; r*r is formed once by the caller. Offsets along periodic axes
// are nearest images.
// *oct receives the octant of the offset: bit 0 set for dx >= 0, bit 1 for
// dy >= 0, bit 2 for dz >= 0.
static inline bool in_ball(double xi, double yi, double zi, double xj, double yj,
                           double zj, double r2, double* d2out, const Periods& P,
                           uint8_t* oct) {
  double dx = min_image(xj - xi, P.Lx), dy = min_image(yj - yi, P.Ly), dz = zj - zi;
  double d2 = ((dx * dx) + (dy * dy)) + (dz * dz);
  *d2out = d2;
  *oct = (uint8_t)((dx >= 0.0 ? 1 : 0) | (dy >= 0.0 ? 2 : 0) | (dz >= 0.0 ? 4 : 0));
  return d2 <= r2;
}

struct Cand {
  double d2;
  uint32_t code;  // j, with MIRROR_BIT for the floor mirror of j
  uint8_t oct;    // octant of the offset x_j - x_i (see in_ball)
};
static bool cand_near_less(const Cand& a, const Cand& b) {
  // nearest first; ties by particle index, then real before mirror
  if (a.d2 != b.d2) return a.d2 < b.d2;
  uint32_t ja = a.code & ~MIRROR_BIT, jb = b.code & ~MIRROR_BIT;
  if (ja != jb) return ja < jb;
  return (a.code & MIRROR_BIT) < (b.code & MIRROR_BIT);
}
static bool cand_canon_less(const Cand& a, const Cand& b) {
  // canonical order of a stored stencil: real particles by index, then mirrors
  bool ma = a.code & MIRROR_BIT, mb = b.code & MIRROR_BIT;
  if (ma != mb) return !ma;
  return (a.code & ~MIRROR_BIT) < (b.code & ~MIRROR_BIT);
}

// Finalise a stencil: optional truncation to `cap` entries, canonical order,
// store. Returns 1 if the list did not fit (and was not truncated).
// keep_nearest 1: the cap nearest. keep_nearest 2: octant-balanced ordering
// (Sec. 3.1 item 6: the first entries of a list should lie in all
// directions, in every neighbouring octant, rather than be the nearest ones
// only): each candidate's rank among the candidates of its own octant,
// nearest first, is its round; the list takes round 0 (the nearest of every
// octant), then round 1, and so on, nearest first within a round, and keeps
// the first cap.
static int store_stencil(std::vector<Cand>& c, int32_t cap, int keep_nearest,
                         int32_t* row, int32_t* cnt) {
  int over = 0;
  if (keep_nearest && (int64_t)c.size() > cap) {
    std::sort(c.begin(), c.end(), cand_near_less);
    if (keep_nearest == 2) {
      std::vector<int32_t> round(c.size());
      int32_t seen[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (size_t k = 0; k < c.size(); ++k) round[k] = seen[c[k].oct]++;
      std::vector<size_t> ord(c.size());
      for (size_t k = 0; k < ord.size(); ++k) ord[k] = k;
      std::stable_sort(ord.begin(), ord.end(),
                       [&](size_t a, size_t b) { return round[a] < round[b]; });
      std::vector<Cand> kept;
      for (int32_t k = 0; k < cap; ++k) kept.push_back(c[ord[k]]);
      c.swap(kept);
    } else {
      c.resize(cap);
    }
  }
  std::sort(c.begin(), c.end(), cand_canon_less);
  int64_t m = (int64_t)c.size();
  if (m > cap) over = 1;
  for (int64_t k = 0; k < m && k < cap; ++k) row[k] = (int32_t)c[k].code;
  *cnt = (int32_t)m;
  return over;
}

// Brute force over all pairs (the definition itself).
static int neighbors_brute(int64_t n, const double* x, const double* y, const double* z,
                           const double* radius, double r_const, int mirror_mode,
                           double floor_z, int32_t cap, int keep_nearest, int32_t* nbr,
                           int32_t* cnt, const Periods& P = Periods()) {
  int over = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : over)
  for (int64_t i = 0; i < n; ++i) {
    double r = radius ? radius[i] : r_const;
    double r2 = r * r;
    std::vector<Cand> c;
    double d2;
    uint8_t oc;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      if (in_ball(x[i], y[i], z[i], x[j], y[j], z[j], r2, &d2, P, &oc))
        c.push_back({d2, (uint32_t)j, oc});
    }
    if (mirror_mode != 0) {
      for (int64_t j = 0; j < n; ++j) {
        double zm = 2.0 * floor_z - z[j];
        if (in_ball(x[i], y[i], z[i], x[j], y[j], zm, r2, &d2, P, &oc))
          c.push_back({d2, (uint32_t)j | MIRROR_BIT, oc});
      }
    }
    over += store_stencil(c, cap, keep_nearest, nbr + i * (int64_t)cap, cnt + i);
  }
  return over;
}

// Independent uniform-grid scan (cell edge >= largest radius); used to make
// large-N oracle runs affordable. Cell indices are clamped to the grid, which
// keeps every pair within one cell of each other in each axis; a periodic
// axis covers [0, L) with floor(L / r) cells and wraps (at least 3 cells, else
// the brute-force scan is used).
static int neighbors_grid(int64_t n, const double* x, const double* y, const double* z,
                          const double* radius, double r_const, int mirror_mode,
                          double floor_z, int32_t cap, int keep_nearest, int32_t* nbr,
                          int32_t* cnt, const Periods& P = Periods()) {
  if (n == 0) return 0;
  double rmax = r_const;
  if (radius) {
    rmax = 0.0;
    for (int64_t i = 0; i < n; ++i) rmax = std::max(rmax, radius[i]);
  }
  double lo[3] = {x[0], y[0], z[0]}, hi[3] = {x[0], y[0], z[0]};
  for (int64_t i = 0; i < n; ++i) {
    lo[0] = std::min(lo[0], x[i]); hi[0] = std::max(hi[0], x[i]);
    lo[1] = std::min(lo[1], y[i]); hi[1] = std::max(hi[1], y[i]);
    lo[2] = std::min(lo[2], z[i]); hi[2] = std::max(hi[2], z[i]);
  }
  double cell = rmax * (1.0 + 1e-9);
  if (!(cell > 0.0)) cell = 1.0;
  int64_t dim[3];
  double ce[3] = {cell, cell, cell};
  const double per[3] = {P.Lx, P.Ly, 0.0};
  for (int a = 0; a < 3; ++a) {
    if (per[a] > 0.0) {  // periodic: whole cells over [0, L)
      dim[a] = (int64_t)std::floor(per[a] / cell);
      if (dim[a] < 3)
        return neighbors_brute(n, x, y, z, radius, r_const, mirror_mode, floor_z, cap,
                               keep_nearest, nbr, cnt, P);
      lo[a] = 0.0;
      ce[a] = per[a] / (double)dim[a];
      continue;
    }
    dim[a] = (int64_t)std::floor((hi[a] - lo[a]) / cell) + 1;
    dim[a] = std::max<int64_t>(1, std::min<int64_t>(dim[a], 512));
  }
  auto cidx = [&](double p, int a) {
    int64_t c = (int64_t)std::floor((p - lo[a]) / ce[a]);
    return std::max<int64_t>(0, std::min<int64_t>(c, dim[a] - 1));
  };
  int64_t ncell = dim[0] * dim[1] * dim[2];
  std::vector<int64_t> key(n), order(n), start(ncell + 1, 0);
  for (int64_t i = 0; i < n; ++i) {
    key[i] = (cidx(z[i], 2) * dim[1] + cidx(y[i], 1)) * dim[0] + cidx(x[i], 0);
    start[key[i] + 1]++;
  }
  for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
  {
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int64_t i = 0; i < n; ++i) order[fill[key[i]]++] = i;
  }
  int over = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : over)
  for (int64_t i = 0; i < n; ++i) {
    double r = radius ? radius[i] : r_const;
    double r2 = r * r;
    std::vector<Cand> c;
    double d2;
    uint8_t oc;
    for (int pass = 0; pass < (mirror_mode ? 2 : 1); ++pass) {
      // pass 0: around x_i; pass 1: around the reflected point, for mirrors
      double qz = pass == 0 ? z[i] : 2.0 * floor_z - z[i];
      int64_t c0[3] = {cidx(x[i], 0), cidx(y[i], 1), cidx(qz, 2)};
      int64_t a0[3], a1[3];
      for (int a = 0; a < 3; ++a) {
        a0[a] = per[a] > 0.0 ? c0[a] - 1 : std::max<int64_t>(0, c0[a] - 1);
        a1[a] = per[a] > 0.0 ? c0[a] + 1 : std::min<int64_t>(dim[a] - 1, c0[a] + 1);
      }
      auto wrap = [&](int64_t v, int a) { return per[a] > 0.0 ? (v + dim[a]) % dim[a] : v; };
      for (int64_t czz = a0[2]; czz <= a1[2]; ++czz)
        for (int64_t cyy = a0[1]; cyy <= a1[1]; ++cyy)
          for (int64_t cxx = a0[0]; cxx <= a1[0]; ++cxx) {
            const int64_t cz = wrap(czz, 2), cy = wrap(cyy, 1), cx = wrap(cxx, 0);
            int64_t cc = (cz * dim[1] + cy) * dim[0] + cx;
            for (int64_t t = start[cc]; t < start[cc + 1]; ++t) {
              int64_t j = order[t];
              if (pass == 0) {
                if (j == i) continue;
                if (in_ball(x[i], y[i], z[i], x[j], y[j], z[j], r2, &d2, P, &oc))
                  c.push_back({d2, (uint32_t)j, oc});
              } else {
                double zm = 2.0 * floor_z - z[j];
                if (in_ball(x[i], y[i], z[i], x[j], y[j], zm, r2, &d2, P, &oc))
                  c.push_back({d2, (uint32_t)j | MIRROR_BIT, oc});
              }
            }
          }
    }
    over += store_stencil(c, cap, keep_nearest, nbr + i * (int64_t)cap, cnt + i);
  }
  return over;
}

// ---------------------------------------------------------- GFD LS fitting ---

static const int NB = 9;  // quadratic Taylor basis in 3D, no constant term

// Row of the Taylor matrix for an h-scaled offset (Sec. 3.1 item 7, 3D form).
template <class T>
static inline void taylor_row(const T& dx, const T& dy, const T& dz, T* a) {
  a[0] = dx; a[1] = dy; a[2] = dz;
  a[3] = 0.5 * (dx * dx); a[4] = 0.5 * (dy * dy); a[5] = 0.5 * (dz * dz);
  a[6] = dx * dy; a[7] = dx * dz; a[8] = dy * dz;
}

// Least-squares solve of A c = B (A is m x 9, row-major; B is m x nf,
// row-major) by Householder QR with column pivoting (largest remaining column
// norm, ties to the lower column). A and B are overwritten. Returns the rank.
template <class T>
static int lsq_qrcp(int m, T* A, int nf, T* B, T* C /* nf x 9 */) {
  int perm[NB];
  for (int j = 0; j < NB; ++j) perm[j] = j;
  int kmax = std::min(m, NB);
  T Rdiag[NB];
  int steps = 0;
  for (int k = 0; k < kmax; ++k) {
    int best = k;
    double bestn = -1.0;
    for (int j = k; j < NB; ++j) {
      double s = 0.0;
      for (int i = k; i < m; ++i) s += val(A[i * NB + j]) * val(A[i * NB + j]);
      if (s > bestn) { bestn = s; best = j; }
    }
    if (best != k) {
      for (int i = 0; i < m; ++i) std::swap(A[i * NB + k], A[i * NB + best]);
      std::swap(perm[k], perm[best]);
    }
    T ss = 0.0;
    for (int i = k; i < m; ++i) ss += A[i * NB + k] * A[i * NB + k];
    T alpha = sqrt(ss);
    if (val(alpha) == 0.0) break;
    double sgn = val(A[k * NB + k]) >= 0.0 ? 1.0 : -1.0;
    // v = x + sgn*|x| e_1 stored in place of column k (rows k..m-1)
    std::vector<T> v(m - k);
    for (int i = k; i < m; ++i) v[i - k] = A[i * NB + k];
    v[0] = v[0] + sgn * alpha;
    T vtv = 0.0;
    for (int i = 0; i < m - k; ++i) vtv += v[i] * v[i];
    for (int j = k; j < NB; ++j) {
      T s = 0.0;
      for (int i = k; i < m; ++i) s += v[i - k] * A[i * NB + j];
      T f = (2.0 * s) / vtv;
      for (int i = k; i < m; ++i) A[i * NB + j] -= f * v[i - k];
    }
    for (int q = 0; q < nf; ++q) {
      T s = 0.0;
      for (int i = k; i < m; ++i) s += v[i - k] * B[i * nf + q];
      T f = (2.0 * s) / vtv;
      for (int i = k; i < m; ++i) B[i * nf + q] -= f * v[i - k];
    }
    Rdiag[k] = A[k * NB + k];
    steps = k + 1;
  }
  int rank = 0;
  if (steps > 0) {
    double r0 = std::fabs(val(Rdiag[0]));
    for (int k = 0; k < steps; ++k) {
      if (std::fabs(val(Rdiag[k])) > 1e-8 * r0) rank = k + 1;
      else break;
    }
  }
  for (int q = 0; q < nf; ++q) {
    T y[NB];
    for (int k = rank - 1; k >= 0; --k) {
      T s = B[k * nf + q];
      for (int j = k + 1; j < rank; ++j) s -= A[k * NB + j] * y[j];
      y[k] = s / A[k * NB + k];
    }
    for (int j = 0; j < NB; ++j) C[q * NB + j] = 0.0;
    for (int k = 0; k < rank; ++k) C[q * NB + perm[k]] = y[k];
  }
  return rank;
}

// Fit nf fields on the stencil of particle i. `field(q, j, mirror, ghost)`
// returns the value of field q at neighbour j, at its floor mirror, or at the
// ghost particle that reflects entry j through i (whose row takes the entry's
// offset negated). Outputs the unscaled coefficients (gradient * h, second
// derivatives * h^2) in C[nf][9].
template <class T, class FieldFn>
static int fit_particle(int64_t i, const T* x, const T* y, const T* z, const int32_t* row,
                        int32_t m, double h, double floor_z, int nf, FieldFn field, T* C,
                        const Periods& P = Periods()) {
  std::vector<T> A((size_t)std::max(m, 1) * NB), B((size_t)std::max(m, 1) * nf);
  for (int32_t k = 0; k < m; ++k) {
    uint32_t code = (uint32_t)row[k];
    bool mir = code & MIRROR_BIT;
    bool ghost = code & GHOST_BIT;
    int64_t j = code & INDEX_MASK;
    T zj = mir ? T(2.0 * floor_z) - z[j] : z[j];
    T dx = min_image_t(x[j] - x[i], P.Lx) / h, dy = min_image_t(y[j] - y[i], P.Ly) / h;
    T dz = (zj - z[i]) / h;
    if (ghost) {
      dx = -dx;
      dy = -dy;
      dz = -dz;
    }
    taylor_row(dx, dy, dz, &A[(size_t)k * NB]);
    for (int q = 0; q < nf; ++q)
      B[(size_t)k * nf + q] = field(q, j, mir, ghost) - field(q, i, false, false);
  }
  return lsq_qrcp<T>(m, A.data(), nf, B.data(), C);
}

// ------------------------------------------------------------ mu(I) law ---

// Closure functions of Sec. 2.3 at solid fraction phi (inertial regime).
template <class T>
struct Closure {
  T M, N, S, R, mu;
};
template <class T>
static Closure<T> closure_at(const T& phi, const T& mu_s, const T& mu_2, const T& I0,
                             double d, double phi_c, double phi_min) {
  double a = phi_c - phi_min;
  T w = T(phi_c) - phi;
  double k = 4.0 * a * a * d * d;
  Closure<T> c;
  c.M = T(-k) / (w * w);
  // mu as a function of phi: mu(I) = mu_s + (mu_2 - mu_s)/(I0/I + 1) with
  // I = (phi_c - phi)/a, i.e. (a mu_s I0 + mu_2 w)/(a I0 + w)   (Sec. 2.3)
  T den = T(a) * I0 + w;
  c.mu = (T(a) * mu_s * I0 + mu_2 * w) / den;
  c.N = -(c.M * c.mu);                    // = 4a^2d^2/w^2 * mu
  c.S = T(-2.0 * k) / ((w * w) * w);      // dM/dphi
  // R = dN/dphi = -S mu - M dmu/dphi,  dmu/dphi = -a I0 (mu_2 - mu_s)/(a I0 + w)^2
  T dmu = -((T(a) * I0) * (mu_2 - mu_s)) / (den * den);
  c.R = -(c.S * c.mu) - c.M * dmu;
  return c;
}

enum { REG_GAS = 0, REG_INERTIAL = 1, REG_QS = 2 };
// Pressure law of Sec. 2.2.1, chosen from the particle's own solid fraction.
static inline int regime_of(double phi, double phi_min, double phi_max) {
  if (phi <= phi_min) return REG_GAS;
  if (phi <= phi_max) return REG_INERTIAL;
  return REG_QS;
}

// ------------------------------------------------------------- LP step ---

template <class T>
struct PState {
  std::vector<T> x, y, z, u, v, w, V;
  explicit PState(int64_t n) : x(n), y(n), z(n), u(n), v(n), w(n), V(n) {}
};

template <class T>
struct TParams {
  T mu_s, mu_2, I0;
  const orc_params* p;
};

struct Stencils {
  int32_t cap = 0;
  std::vector<int32_t> nbr, cnt;
};

static void add_ghosts(int64_t n, const double* x, const double* y, const double* z,
                       const orc_params* p, Stencils& st);

static void build_stencils(int64_t n, const double* x, const double* y, const double* z,
                           const orc_params* p, int brute, Stencils& st) {
  // the step never truncates; lists are sized for any lattice stencil
  st.cap = 256;
  st.nbr.assign((size_t)n * st.cap, 0);
  st.cnt.assign(n, 0);
  Periods P;
  P.Lx = p->period_x;
  P.Ly = p->period_y;
  if (brute)
    neighbors_brute(n, x, y, z, nullptr, p->radius, p->mirror_mode, p->floor_z, st.cap, 0,
                    st.nbr.data(), st.cnt.data(), P);
  else
    neighbors_grid(n, x, y, z, nullptr, p->radius, p->mirror_mode, p->floor_z, st.cap, 0,
                   st.nbr.data(), st.cnt.data(), P);
  if (p->free_surface) add_ghosts(n, x, y, z, p, st);
}

// ------------------------------------------------------- free boundary ---
// Sec. 3.1 items 6 and 9: a particle that cannot find neighbours in some
// directions gets ghost particles that complete its neighbourhood. The paper
// leaves the test and the placement open; here:
//  - positions are taken in fixed point on a power-of-two grid, X = round(K x)
//    with K the largest power of two such that K r <= 2^13 (so the scaling is
//    exact and every offset, square and pair sum below fits 32-bit integers),
//    and offsets are the exact integer differences o_k = X_k - X_i (along a
//    periodic axis the nearest image modulo round(K L)): every sum below is an
//    exact integer, independent of the entry order;
//  - each entry is weighted by w_k = max(0, R2 - |o_k|^2), R2 = round((K r)^2),
//    which fades entries out at the stencil radius (an unweighted mean is
//    dominated by which lattice points of the outermost shell happen to fall
//    inside r);
//  - the stencil is one-sided when the weighted summed offset S = sum w_k o_k
//    satisfies |S| > kSurfaceTilt K h sum w_k (lattice with 0.05-0.2 h jitter
//    and r = 2.2 h: interior and second-layer particles stay below 0.16 h,
//    free-surface particles above 0.29 h);
//  - every entry k with o_k . S >= kGhostDepth K h |S| (at least h/2 on the
//    inner side) whose reflection -o_k has no stencil entry within h/2 gets a
//    ghost at that reflection, except below the floor when floor mirrors are
//    on (the solid boundary is the mirrors' side: (z_i + z_i) - z_k < floor_z).
// The dot products o_k . S are exact 64-bit integers; only the squared
// comparisons are formed in FP64, in a fixed order, so the decisions are
// reproducible bit for bit.
static const double kSurfaceTilt = 0.22, kGhostDepth = 0.5;

static double ghost_grid(double r) {  // K: largest power of two with K r <= 8192
  double K = 1.0;
  while (K * r > 8192.0) K *= 0.5;
  while (2.0 * K * r <= 8192.0) K *= 2.0;
  return K;
}

static void add_ghosts(int64_t n, const double* x, const double* y, const double* z,
                       const orc_params* p, Stencils& st) {
  const double h = p->h, K = ghost_grid(p->radius);
  const double rk = p->radius * K;
  const int64_t R2 = std::llrint(rk * rk);
  const double hk = h * K;
  const int64_t clear2 = std::llrint((0.5 * hk) * (0.5 * hk));
  auto fix = [&](double v) { return (int64_t)std::llrint(v * K); };
  // periodic axes: integer period round(K L); offsets take their nearest image
  const int64_t PX = p->period_x > 0.0 ? std::llrint(K * p->period_x) : 0;
  const int64_t PY = p->period_y > 0.0 ? std::llrint(K * p->period_y) : 0;
  auto wrap_fix = [](int64_t o, int64_t P) {
    if (P > 0) {
      if (2 * o > P) return o - P;
      if (2 * o < -P) return o + P;
    }
    return o;
  };
  for (int64_t i = 0; i < n; ++i) {
    int32_t* row = st.nbr.data() + i * (int64_t)st.cap;
    const int32_t m = st.cnt[i];
    if (m == 0) continue;
    const int64_t Xi[3] = {fix(x[i]), fix(y[i]), fix(z[i])};
    std::vector<int64_t> o(3 * (size_t)m);
    std::vector<double> zk((size_t)m);
    int64_t S[3] = {0, 0, 0}, Wsum = 0;
    for (int32_t k = 0; k < m; ++k) {
      const uint32_t code = (uint32_t)row[k];
      const int64_t j = code & INDEX_MASK;
      const double zj = (code & MIRROR_BIT) ? 2.0 * p->floor_z - z[j] : z[j];
      zk[k] = zj;
      o[3 * k] = wrap_fix(fix(x[j]) - Xi[0], PX);
      o[3 * k + 1] = wrap_fix(fix(y[j]) - Xi[1], PY);
      o[3 * k + 2] = fix(zj) - Xi[2];
      const int64_t q = (o[3 * k] * o[3 * k] + o[3 * k + 1] * o[3 * k + 1]) +
                        o[3 * k + 2] * o[3 * k + 2];
      const int64_t w = q < R2 ? R2 - q : 0;
      for (int a = 0; a < 3; ++a) S[a] += w * o[3 * k + a];
      Wsum += w;
    }
    const double sx = (double)S[0], sy = (double)S[1], sz = (double)S[2];
    const double s2 = ((sx * sx) + (sy * sy)) + (sz * sz);
    const double lim = (kSurfaceTilt * hk) * (double)Wsum;
    if (!(s2 > lim * lim)) continue;
    const double dep = kGhostDepth * hk;
    int32_t c = m;
    for (int32_t k = 0; k < m; ++k) {
      // o_k . S exactly (|o| <= 2^13 + 1, |S| < 2^46), then one rounding
      const double ds = (double)((o[3 * k] * S[0] + o[3 * k + 1] * S[1]) + o[3 * k + 2] * S[2]);
      if (!(ds > 0.0 && ds * ds >= (dep * dep) * s2)) continue;
      if (p->mirror_mode != 0 && (z[i] + z[i]) - zk[k] < p->floor_z) continue;
      bool clear = true;
      for (int32_t l = 0; l < m && clear; ++l) {
        const int64_t ex = o[3 * l] + o[3 * k], ey = o[3 * l + 1] + o[3 * k + 1];
        const int64_t ez = o[3 * l + 2] + o[3 * k + 2];
        clear = (ex * ex + ey * ey) + ez * ez >= clear2;
      }
      if (clear && c < st.cap) row[c++] = (int32_t)((uint32_t)row[k] | GHOST_BIT);
    }
    st.cnt[i] = c;
  }
}

// Solid fraction of a ghost particle: just below phi_min (gas side of the
// pressure law), 1e-3 relative.
static inline double ghost_phi(const orc_params* p) { return p->phi_min * (1.0 - 1e-3); }

// |gdot| of a ghost of particle F (Sec. 3.1 item 9): the value that keeps the
// inertial pressure phi_s (2 a d |gdot| / (phi_c - phi))^2 continuous,
// |gdot|_G = |gdot|_F (phi_c - phi_G) / (phi_c - phi_F); outside the inertial
// regime F's own value (its acceleration does not use grad |gdot|).
template <class T>
static inline T ghost_gn(const orc_params* p, const T& phi_f, const T& gn_f);

// Per-particle intermediates of one step, exported for kernel-level parity.
template <class T>
struct Detail {
  std::vector<T> gd, gn, gV, lapdiv, div, gg, acc, Vnew;
  std::vector<int8_t> reg;
  explicit Detail(int64_t n)
      : gd(6 * n), gn(n), gV(3 * n), lapdiv(3 * n), div(n), gg(3 * n), acc(3 * n), Vnew(n),
        reg(n) {}
};

template <class T>
static inline T ghost_gn(const orc_params* p, const T& phi_f, const T& gn_f) {
  if (regime_of(val(phi_f), p->phi_min, p->phi_max) != REG_INERTIAL) return gn_f;
  return gn_f * ((p->phi_c - ghost_phi(p)) / (T(p->phi_c) - phi_f));
}

// One explicit step (Sec. 3.1 items 7, 8 and 10).
// Time levels: the difference equations of item 8 print V, V_X, ... on their
// right-hand sides without a level. Here V is advanced first from div u^n,
//   V^{n+1} = V^n + dt V^n DIV(u^n),
// and the momentum right-hand side then takes V^{n+1} (its value, its fitted
// gradient, the closure and the regime at phi^{n+1} = 1/V^{n+1}) together with
// the time-n velocity quantities gdot^n, |gdot|^n, grad |gdot|^n, LAP u^n and
// grad DIV u^n. Pass 1 fits u, v, w; pass 2 fits |gdot|^n and V^{n+1}.
// With euler = true, pass 2 takes V^n (not V^{n+1}): the right-hand side
// of the semi-discrete system at one time level, for Heun's method.
template <class T>
static void lp_rhs(int64_t n, const PState<T>& s, const TParams<T>& tp, const Stencils& st,
                   Detail<T>& o, int64_t* n_rank_deficient, bool euler = false) {
  const orc_params* p = tp.p;
  const double h = p->h;
  const double dt = p->dt;
  Periods Pp;
  Pp.Lx = p->period_x;
  Pp.Ly = p->period_y;
  auto usgn = [&](int comp) -> double {  // mirror velocity sign per component
    if (p->mirror_mode == 1) return -1.0;
    if (p->mirror_mode == 2) return comp == 2 ? -1.0 : 1.0;
    return 1.0;
  };
  int64_t n_rd = 0;
  // ---- pass 1: fits of u, v, w at time n
#pragma omp parallel for schedule(dynamic, 32) reduction(+ : n_rd)
  for (int64_t i = 0; i < n; ++i) {
    const int32_t* row = st.nbr.data() + i * (int64_t)st.cap;
    int32_t m = st.cnt[i];
    auto field = [&](int q, int64_t j, bool mir, bool ghost) -> T {
      if (ghost) j = i;  // free surface: the ghost carries the velocity of i
      switch (q) {
        case 0: return mir && !ghost ? usgn(0) * s.u[j] : s.u[j];
        case 1: return mir && !ghost ? usgn(1) * s.v[j] : s.v[j];
        default: return mir && !ghost ? usgn(2) * s.w[j] : s.w[j];
      }
    };
    T C[3 * NB];
    int rank = fit_particle<T>(i, s.x.data(), s.y.data(), s.z.data(), row, m, h, p->floor_z,
                               3, field, C, Pp);
    if (rank < NB) n_rd++;
    // velocity gradient G[a][b] = d u_a / d x_b ; second derivatives H[a][.]
    // in the column order xx, yy, zz, xy, xz, yz
    T G[3][3], H[3][6];
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) G[a][b] = C[a * NB + b] / h;
      for (int b = 0; b < 6; ++b) H[a][b] = C[a * NB + 3 + b] / (h * h);
    }
    // strain rate D, divergence, shear-rate tensor gdot = D - div/3 I (Sec. 2.2)
    T div = (G[0][0] + G[1][1]) + G[2][2];
    T g[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        T D = 0.5 * (G[a][b] + G[b][a]);
        g[a][b] = a == b ? D - div / 3.0 : D;
      }
    T ss = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) ss += g[a][b] * g[a][b];
    o.gn[i] = sqrt(0.5 * ss);
    o.gd[6 * i + 0] = g[0][0]; o.gd[6 * i + 1] = g[1][1]; o.gd[6 * i + 2] = g[2][2];
    o.gd[6 * i + 3] = g[0][1]; o.gd[6 * i + 4] = g[0][2]; o.gd[6 * i + 5] = g[1][2];
    o.div[i] = div;
    // (1/2) Lap u_a + (1/6) d_a div u   (divergence of gdot)
    T lap[3], ddiv[3];
    for (int a = 0; a < 3; ++a) lap[a] = (H[a][0] + H[a][1]) + H[a][2];
    ddiv[0] = (H[0][0] + H[1][3]) + H[2][4];
    ddiv[1] = (H[0][3] + H[1][1]) + H[2][5];
    ddiv[2] = (H[0][4] + H[1][5]) + H[2][2];
    for (int a = 0; a < 3; ++a) o.lapdiv[3 * i + a] = 0.5 * lap[a] + ddiv[a] / 6.0;
    // specific volume at n+1 (item 8, first difference equation)
    o.Vnew[i] = s.V[i] + dt * (s.V[i] * div);
  }
  // ---- pass 2: fits of |gdot|^n (mirrors carry |gdot| = 0, item 9) and
  //      V^{n+1} (mirrors keep the density), then the acceleration
#pragma omp parallel for schedule(dynamic, 32)
  for (int64_t i = 0; i < n; ++i) {
    const int32_t* row = st.nbr.data() + i * (int64_t)st.cap;
    int32_t m = st.cnt[i];
    // free surface (Sec. 3.1 item 9): a ghost has solid fraction phi_G just
    // below phi_min and the |gdot| that keeps the inertial pressure of i
    // continuous, |gdot|_G = |gdot|_i (phi_c - phi_G) / (phi_c - phi_i)
    const std::vector<T>& Vf = euler ? s.V : o.Vnew;  // V of the closure and the fit
    const double phi_g = ghost_phi(p);
    const T gn_ghost = ghost_gn<T>(p, T(1.0) / Vf[i], o.gn[i]);
    auto field = [&](int q, int64_t j, bool mir, bool ghost) -> T {
      if (ghost) return q == 0 ? gn_ghost : T(1.0 / phi_g);
      if (q == 0) return mir ? T(0.0) : o.gn[j];
      return Vf[j];
    };
    T C[2 * NB];
    fit_particle<T>(i, s.x.data(), s.y.data(), s.z.data(), row, m, h, p->floor_z, 2, field, C,
                    Pp);
    T gg[3] = {C[0] / h, C[1] / h, C[2] / h};
    T gV[3] = {C[NB + 0] / h, C[NB + 1] / h, C[NB + 2] / h};
    for (int c = 0; c < 3; ++c) {
      o.gg[3 * i + c] = gg[c];
      o.gV[3 * i + c] = gV[c];
    }
    const T Vi = Vf[i];
    const T phi = T(1.0) / Vi;
    int r = regime_of(val(phi), p->phi_min, p->phi_max);
    o.reg[i] = (int8_t)r;
    const double gvec[3] = {p->gx, p->gy, p->gz};
    T a[3];
    if (r == REG_GAS) {
      // zero pressure: motion by inertia and body force only
      for (int c = 0; c < 3; ++c) a[c] = T(gvec[c]);
    } else if (r == REG_QS) {
      // sigma = -phi_s (alpha + beta phi) delta  =>  a = beta grad V / V + g
      for (int c = 0; c < 3; ++c) a[c] = (p->beta * gV[c]) / Vi + gvec[c];
    } else {
      Closure<T> cl = closure_at<T>(phi, tp.mu_s, tp.mu_2, tp.I0, p->d, p->phi_c, p->phi_min);
      const T* gd = &o.gd[6 * i];
      T g3[3][3] = {{gd[0], gd[3], gd[4]}, {gd[3], gd[1], gd[5]}, {gd[4], gd[5], gd[2]}};
      T G = o.gn[i];
      for (int c = 0; c < 3; ++c) {
        // V [ -(|g|/V^2)(S |g| V_c + R g_cj V_j) + 2M|g| |g|_c + N g_cj |g|_j
        //     + N |g| ((1/2) Lap u_c + (1/6) d_c div) ] + g_c
        T gjVj = (g3[c][0] * gV[0] + g3[c][1] * gV[1]) + g3[c][2] * gV[2];
        T gjGj = (g3[c][0] * gg[0] + g3[c][1] * gg[1]) + g3[c][2] * gg[2];
        T t1 = -(G / (Vi * Vi)) * (cl.S * G * gV[c] + cl.R * gjVj);
        T t2 = 2.0 * cl.M * G * gg[c];
        T t3 = cl.N * gjGj;
        T t4 = cl.N * G * o.lapdiv[3 * i + c];
        a[c] = Vi * (((t1 + t2) + t3) + t4) + gvec[c];
      }
    }
    for (int c = 0; c < 3; ++c) o.acc[3 * i + c] = a[c];
  }
  if (n_rank_deficient) *n_rank_deficient += n_rd;
}

// Explicit update (Sec. 3.1 item 8 for V and u, item 10 for x).
template <class T>
static void lp_update(int64_t n, PState<T>& s, const Detail<T>& o, double dt, double Lx,
                      double Ly) {
  for (int64_t i = 0; i < n; ++i) {
    T un = s.u[i], vn = s.v[i], wn = s.w[i];
    s.V[i] = o.Vnew[i];
    s.u[i] = un + dt * o.acc[3 * i + 0];
    s.v[i] = vn + dt * o.acc[3 * i + 1];
    s.w[i] = wn + dt * o.acc[3 * i + 2];
    s.x[i] = wrap_t(s.x[i] + (0.5 * dt) * (un + s.u[i]), Lx);
    s.y[i] = wrap_t(s.y[i] + (0.5 * dt) * (vn + s.v[i]), Ly);
    s.z[i] = s.z[i] + (0.5 * dt) * (wn + s.w[i]);
  }
}

// Forward-Euler update of the semi-discrete system (stage of Heun's method):
// x advances with u^n.
template <class T>
static void lp_update_euler(int64_t n, PState<T>& s, const Detail<T>& o, double dt, double Lx,
                            double Ly) {
  for (int64_t i = 0; i < n; ++i) {
    T un = s.u[i], vn = s.v[i], wn = s.w[i];
    s.V[i] = o.Vnew[i];
    s.u[i] = un + dt * o.acc[3 * i + 0];
    s.v[i] = vn + dt * o.acc[3 * i + 1];
    s.w[i] = wn + dt * o.acc[3 * i + 2];
    s.x[i] = wrap_t(s.x[i] + dt * un, Lx);
    s.y[i] = wrap_t(s.y[i] + dt * vn, Ly);
    s.z[i] = s.z[i] + dt * wn;
  }
}

template <class T>
static void values_of(const std::vector<T>& a, std::vector<double>& out) {
  out.resize(a.size());
  for (size_t i = 0; i < a.size(); ++i) out[i] = val(a[i]);
}

// nsteps explicit steps; neighbour lists rebuilt from the current positions
// whenever step % rebuild_every == 0 and held fixed in between.
template <class T>
static void lp_run(int64_t n, PState<T>& s, const TParams<T>& tp, int nsteps, int rebuild_every,
                   int brute, orc_diag* dg) {
  const orc_params* p = tp.p;
  Stencils st;
  Detail<T> o(n);
  std::vector<double> vx, vy, vz;
  if (rebuild_every < 1) rebuild_every = 1;
  for (int step = 0; step < nsteps; ++step) {
    if (step % rebuild_every == 0) {
      values_of(s.x, vx); values_of(s.y, vy); values_of(s.z, vz);
      build_stencils(n, vx.data(), vy.data(), vz.data(), p, brute, st);
    }
    int64_t nrd = 0;
    const bool heun = p->time_scheme == 1;
    PState<T> s0 = heun ? s : PState<T>(0);
    lp_rhs<T>(n, s, tp, st, o, &nrd, heun);
    if (dg) {
      dg->n_rank_deficient += nrd;
      for (int64_t i = 0; i < n; ++i) {
        int r = o.reg[i];
        if (r == REG_GAS) dg->n_gas++;
        else if (r == REG_INERTIAL) dg->n_inertial++;
        else dg->n_quasistatic++;
        if (1.0 / val(o.Vnew[i]) > p->phi_c) dg->n_over_c++;
        dg->min_stencil = std::min<int64_t>(dg->min_stencil, st.cnt[i]);
        dg->max_stencil = std::max<int64_t>(dg->max_stencil, st.cnt[i]);
        if (step % rebuild_every == 0)
          for (int32_t k = 0; k < st.cnt[i]; ++k)
            if ((uint32_t)st.nbr[i * (int64_t)st.cap + k] & GHOST_BIT) dg->n_ghosts++;
      }
    }
    if (heun) {
      // Heun's method (second order; the paper plans a second-order scheme,
      // Sec. 3.1 item 8): y* = y + dt F(y), y** = y* + dt F(y*) on the same
      // stencils, y^{n+1} = (y + y**) / 2
      lp_update_euler<T>(n, s, o, p->dt, p->period_x, p->period_y);
      lp_rhs<T>(n, s, tp, st, o, &nrd, true);
      lp_update_euler<T>(n, s, o, p->dt, p->period_x, p->period_y);
      for (int64_t i = 0; i < n; ++i) {
        // periodic axes: the mean of the two positions taken on the same image
        if (p->period_x > 0.0)
          s.x[i] = wrap_t(s0.x[i] + 0.5 * min_image_t(s.x[i] - s0.x[i], p->period_x), p->period_x);
        else
          s.x[i] = 0.5 * (s0.x[i] + s.x[i]);
        if (p->period_y > 0.0)
          s.y[i] = wrap_t(s0.y[i] + 0.5 * min_image_t(s.y[i] - s0.y[i], p->period_y), p->period_y);
        else
          s.y[i] = 0.5 * (s0.y[i] + s.y[i]);
        s.z[i] = 0.5 * (s0.z[i] + s.z[i]); s.u[i] = 0.5 * (s0.u[i] + s.u[i]);
        s.v[i] = 0.5 * (s0.v[i] + s.v[i]); s.w[i] = 0.5 * (s0.w[i] + s.w[i]);
        s.V[i] = 0.5 * (s0.V[i] + s.V[i]);
      }
    } else {
      lp_update<T>(n, s, o, p->dt, p->period_x, p->period_y);
    }
    if (dg)
      for (int64_t i = 0; i < n; ++i)
        if (val(s.z[i]) < p->floor_z) dg->n_below_floor++;
  }
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

// ================================================================ C API ===

extern "C" {

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Neighbour lists. nbr is n x cap (row-major), entries j or (j | 0x80000000)
// for the floor mirror of j, real particles first, each group ascending.
// cnt[i] = stencil size (may exceed cap when keep_nearest == 0: overflow).
// keep_nearest: 0 all, 1 the cap nearest, 2 octant-balanced (store_stencil).
// Returns the number of overflowing particles.
int orc_neighbors(int64_t n, const double* x, const double* y, const double* z,
                  const double* radius, double r_const, int mirror_mode, double floor_z,
                  int32_t cap, int keep_nearest, int brute, int32_t* nbr, int32_t* cnt,
                  int nthreads) {
  set_threads(nthreads);
  if (brute)
    return neighbors_brute(n, x, y, z, radius, r_const, mirror_mode, floor_z, cap, keep_nearest,
                           nbr, cnt);
  return neighbors_grid(n, x, y, z, radius, r_const, mirror_mode, floor_z, cap, keep_nearest,
                        nbr, cnt);
}

// GFD fits of nf fields (fields[q*n + j]); mirror_sign[q] is the factor applied
// to field q at a floor mirror (+1 even, -1 odd, 0 zero). coeffs[(i*nf+q)*9+c]
// holds d/dx, d/dy, d/dz, d2/dx2, d2/dy2, d2/dz2, d2/dxdy, d2/dxdz, d2/dydz.
int orc_fit(int64_t n, const double* x, const double* y, const double* z, const int32_t* nbr,
            const int32_t* cnt, int32_t cap, int nf, const double* fields,
            const double* mirror_sign, double h, double floor_z, double* coeffs, int32_t* rank,
            int nthreads) {
  set_threads(nthreads);
  int64_t nrd = 0;
#pragma omp parallel for schedule(dynamic, 32) reduction(+ : nrd)
  for (int64_t i = 0; i < n; ++i) {
    auto field = [&](int q, int64_t j, bool mir, bool ghost) -> double {
      double s = fields[(int64_t)q * n + (ghost ? i : j)];  // not produced by the search
      return mir && !ghost ? mirror_sign[q] * s : s;
    };
    std::vector<double> C((size_t)nf * NB);
    int m = std::min(cnt[i], cap);
    int r = fit_particle<double>(i, x, y, z, nbr + i * (int64_t)cap, m, h, floor_z, nf, field,
                                 C.data());
    if (rank) rank[i] = r;
    if (r < NB) nrd++;
    for (int q = 0; q < nf; ++q)
      for (int c = 0; c < NB; ++c)
        coeffs[((int64_t)i * nf + q) * NB + c] =
            C[q * NB + c] / (c < 3 ? h : h * h);
  }
  return (int)nrd;
}

// Closure functions at given solid fractions: out[i*5 + {0..4}] = M, N, S, R, mu.
void orc_closure(int64_t n, const double* phi, const orc_params* p, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    Closure<double> c = closure_at<double>(phi[i], p->mu_s, p->mu_2, p->I0, p->d, p->phi_c,
                                           p->phi_min);
    out[5 * i + 0] = c.M; out[5 * i + 1] = c.N; out[5 * i + 2] = c.S;
    out[5 * i + 3] = c.R; out[5 * i + 4] = c.mu;
  }
}

// Pointwise mu(I) stress from V and the velocity gradient (grad_u[i*9 + 3a+b]
// = d u_a / d x_b): gdot (xx,yy,zz,xy,xz,yz), |gdot|, pressure P, effective
// viscosity eta (tau = eta gdot) and regime (0 gas, 1 inertial, 2 quasi-static).
void orc_mui_stress(int64_t n, const orc_params* p, const double* V, const double* grad_u,
                    double* gdot, double* gnorm, double* P, double* eta, int8_t* regime) {
  const double a = p->phi_c - p->phi_min;
  for (int64_t i = 0; i < n; ++i) {
    const double* G = grad_u + 9 * i;
    double div = (G[0] + G[4]) + G[8];
    double g[3][3];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        double D = 0.5 * (G[3 * r + c] + G[3 * c + r]);
        g[r][c] = r == c ? D - div / 3.0 : D;
      }
    double ss = 0.0;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) ss += g[r][c] * g[r][c];
    double gn = std::sqrt(0.5 * ss);
    gdot[6 * i + 0] = g[0][0]; gdot[6 * i + 1] = g[1][1]; gdot[6 * i + 2] = g[2][2];
    gdot[6 * i + 3] = g[0][1]; gdot[6 * i + 4] = g[0][2]; gdot[6 * i + 5] = g[1][2];
    gnorm[i] = gn;
    double phi = 1.0 / V[i];
    int r = regime_of(phi, p->phi_min, p->phi_max);
    regime[i] = (int8_t)r;
    if (r == REG_GAS) {
      P[i] = 0.0; eta[i] = 0.0;
    } else if (r == REG_QS) {
      P[i] = p->rho_s * (p->alpha + p->beta * phi); eta[i] = 0.0;
    } else {
      double q = (2.0 * a * p->d * gn) / (p->phi_c - phi);
      P[i] = p->rho_s * (q * q);
      Closure<double> c = closure_at<double>(phi, p->mu_s, p->mu_2, p->I0, p->d, p->phi_c,
                                             p->phi_min);
      eta[i] = p->rho_s * (c.N * gn);  // mu(I) P / |gdot|
    }
  }
}

static void load_state(int64_t n, PState<double>& s, const double* x, const double* y,
                       const double* z, const double* u, const double* v, const double* w,
                       const double* V) {
  for (int64_t i = 0; i < n; ++i) {
    s.x[i] = x[i]; s.y[i] = y[i]; s.z[i] = z[i];
    s.u[i] = u[i]; s.v[i] = v[i]; s.w[i] = w[i]; s.V[i] = V[i];
  }
}

// nsteps LP steps in place. Returns 0.
// Stencils of one step (the neighbour lists plus, with p->free_surface, the
// ghost entries), in the step's own order; rows of `cap` entries.
int orc_step_stencils(int64_t n, const double* x, const double* y, const double* z,
                      const orc_params* p, int brute, int32_t cap, int32_t* nbr, int32_t* cnt,
                      int nthreads) {
  set_threads(nthreads);
  Stencils st;
  build_stencils(n, x, y, z, p, brute, st);
  int over = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int32_t m = st.cnt[i];
    if (m > cap) over = 1;
    for (int32_t k = 0; k < m && k < cap; ++k) nbr[i * (int64_t)cap + k] = st.nbr[i * (int64_t)st.cap + k];
    cnt[i] = m;
  }
  return over;
}

// Ghost-particle state of fluid particles with solid fraction phi[i] and
// |gdot| gn[i]: phi_G and |gdot|_G.
void orc_ghost_state(int64_t n, const double* phi, const double* gn, const orc_params* p,
                     double* phi_g, double* gn_g) {
  for (int64_t i = 0; i < n; ++i) {
    phi_g[i] = ghost_phi(p);
    gn_g[i] = ghost_gn<double>(p, phi[i], gn[i]);
  }
}

int orc_step(int64_t n, double* x, double* y, double* z, double* u, double* v, double* w,
             double* V, const orc_params* p, int nsteps, int rebuild_every, int brute,
             int nthreads, orc_diag* diag) {
  set_threads(nthreads);
  PState<double> s(n);
  load_state(n, s, x, y, z, u, v, w, V);
  TParams<double> tp{p->mu_s, p->mu_2, p->I0, p};
  if (diag) {
    std::memset(diag, 0, sizeof(*diag));
    diag->min_stencil = INT64_MAX;
  }
  lp_run<double>(n, s, tp, nsteps, rebuild_every, brute, diag);
  for (int64_t i = 0; i < n; ++i) {
    x[i] = s.x[i]; y[i] = s.y[i]; z[i] = s.z[i];
    u[i] = s.u[i]; v[i] = s.v[i]; w[i] = s.w[i]; V[i] = s.V[i];
  }
  return 0;
}

// Intermediates of one step at the given state (nothing is advanced):
// gdot (6n), |gdot| (n), grad V (3n), (1/2)Lap u + (1/6) grad div (3n),
// div u (n), grad |gdot| (3n), acceleration (3n), regime (n).
int orc_step_detail(int64_t n, const double* x, const double* y, const double* z,
                    const double* u, const double* v, const double* w, const double* V,
                    const orc_params* p, int brute, int nthreads, double* gd, double* gn,
                    double* gV, double* lapdiv, double* div, double* gg, double* acc,
                    int8_t* regime) {
  set_threads(nthreads);
  PState<double> s(n);
  load_state(n, s, x, y, z, u, v, w, V);
  TParams<double> tp{p->mu_s, p->mu_2, p->I0, p};
  Stencils st;
  build_stencils(n, x, y, z, p, brute, st);
  Detail<double> o(n);
  int64_t nrd = 0;
  lp_rhs<double>(n, s, tp, st, o, &nrd);
  std::memcpy(gd, o.gd.data(), sizeof(double) * 6 * n);
  std::memcpy(gn, o.gn.data(), sizeof(double) * n);
  std::memcpy(gV, o.gV.data(), sizeof(double) * 3 * n);
  std::memcpy(lapdiv, o.lapdiv.data(), sizeof(double) * 3 * n);
  std::memcpy(div, o.div.data(), sizeof(double) * n);
  std::memcpy(gg, o.gg.data(), sizeof(double) * 3 * n);
  std::memcpy(acc, o.acc.data(), sizeof(double) * 3 * n);
  std::memcpy(regime, o.reg.data(), n);
  return (int)nrd;
}

// Tangent-linear run: the same steps on dual numbers seeded with unit
// directions in (mu_s, mu_2, I0). On return the state arrays hold the final
// values and tangent[(k*7 + f)*n + i] = d state_f(i) / d theta_k with the
// field order x, y, z, u, v, w, V.
int orc_step_tangent(int64_t n, double* x, double* y, double* z, double* u, double* v,
                     double* w, double* V, const orc_params* p, int nsteps, int rebuild_every,
                     int brute, int nthreads, double* tangent) {
  set_threads(nthreads);
  PState<Dual3> s(n);
  for (int64_t i = 0; i < n; ++i) {
    s.x[i] = x[i]; s.y[i] = y[i]; s.z[i] = z[i];
    s.u[i] = u[i]; s.v[i] = v[i]; s.w[i] = w[i]; s.V[i] = V[i];
  }
  Dual3 ms(p->mu_s), m2(p->mu_2), i0(p->I0);
  ms.d[0] = 1.0; m2.d[1] = 1.0; i0.d[2] = 1.0;
  TParams<Dual3> tp{ms, m2, i0, p};
  lp_run<Dual3>(n, s, tp, nsteps, rebuild_every, brute, nullptr);
  std::vector<Dual3>* f[7] = {&s.x, &s.y, &s.z, &s.u, &s.v, &s.w, &s.V};
  double* outv[7] = {x, y, z, u, v, w, V};
  for (int q = 0; q < 7; ++q)
    for (int64_t i = 0; i < n; ++i) {
      outv[q][i] = (*f[q])[i].v;
      for (int k = 0; k < 3; ++k) tangent[((int64_t)k * 7 + q) * n + i] = (*f[q])[i].d[k];
    }
  return 0;
}

}  // extern "C"
