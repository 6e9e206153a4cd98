// Device bodies of the cell sort and the neighbour search, shared by the
// per-phase kernels (neighbors.cu) and the persistent step kernel
// (persistent.cu). See neighbors.cu for the method.
#pragma once

#include "lp_internal.cuh"

namespace lp {

// Cell key of every particle; particles with a non-finite coordinate go to
// the extra bucket `ncell`, which no search visits.
__device__ __forceinline__ void keys_body(int s, const double* __restrict__ x,
                                          const double* __restrict__ y,
                                          const double* __restrict__ z,
                                          const int32_t* __restrict__ colid,
                                          const GridCol* __restrict__ grids, uint32_t ncell,
                                          uint32_t* __restrict__ key,
                                          uint32_t* __restrict__ count) {
  if (!(isfinite(x[s]) && isfinite(y[s]) && isfinite(z[s]))) {
    key[s] = ncell;
    atomicAdd(&count[ncell], 1u);
    return;
  }
  const GridCol g = grids[colid[s]];
  const int cx = cell_coord(x[s], g.ox, g.icx, g.nx);
  const int cy = cell_coord(y[s], g.oy, g.icy, g.ny);
  const int cz = cell_coord(z[s], g.oz, g.icz, g.nz);
  const uint32_t k = (uint32_t)cell_id(g, cx, cy, cz);
  key[s] = k;
  atomicAdd(&count[k], 1u);
}

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t ws[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) ws[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    ws[lane] = wi - w;  // exclusive prefix of each warp
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  const uint32_t r = ws[wid] + inc - v;
  __syncthreads();
  return r;
}

__device__ __forceinline__ void scatter_body(int s, const uint32_t* __restrict__ key,
                                             const uint32_t* __restrict__ start,
                                             uint32_t* __restrict__ fill,
                                             int32_t* __restrict__ tmp) {
  const uint32_t k = key[s];
  const uint32_t pos = start[k] + atomicAdd(&fill[k], 1u);
  tmp[pos] = s;
}

// Order each cell's particles by original index (insertion sort; cells hold
// about (cell edge / h)^3 particles). A cell crowded beyond kSortCap (only
// after a blow-up) keeps its arrival order: the stencils stay exact, only the
// row order inside them loses its determinism.
constexpr uint32_t kSortCap = 1024;
__device__ __forceinline__ void cell_sort_body(int64_t c, const uint32_t* __restrict__ start,
                                               int32_t* __restrict__ tmp,
                                               const int32_t* __restrict__ ids) {
  const uint32_t b = start[c], e = start[c + 1];
  if (e - b > kSortCap) return;
  for (uint32_t i = b + 1; i < e; ++i) {
    const int32_t v = tmp[i];
    const int32_t kv = ids[v];
    uint32_t j = i;
    while (j > b && ids[tmp[j - 1]] > kv) {
      tmp[j] = tmp[j - 1];
      --j;
    }
    tmp[j] = v;
  }
}

// Gather the state into the new order; FP32 origin-relative positions for the
// prefilter.
__device__ __forceinline__ void gather_body(int t, int n, const int32_t* __restrict__ tmp,
                                            const double* const* __restrict__ src,
                                            double* const* __restrict__ dst, int nsrc,
                                            const int32_t* __restrict__ ids_in,
                                            int32_t* __restrict__ ids_out,
                                            const int32_t* __restrict__ col_in,
                                            int32_t* __restrict__ col_out,
                                            const GridCol* __restrict__ grids,
                                            float4* __restrict__ pf) {
  int s = tmp[t];
  if ((unsigned)s >= (unsigned)n) s = t;  // stay inside the buffers whatever tmp holds
  for (int f = 0; f < nsrc; ++f) dst[f][t] = src[f][s];
  ids_out[t] = ids_in[s];
  const int c = col_in[s];
  col_out[t] = c;
  const GridCol g = grids[c];
  pf[t] = make_float4(__double2float_rn(src[0][s] - g.ox), __double2float_rn(src[1][s] - g.oy),
                      __double2float_rn(src[2][s] - g.oz), 0.f);
}

// FP32 offset along an axis of period L (float), nearest image; with L = 0
// the value is returned unchanged (d - (+-0))
__device__ __forceinline__ float min_image_f(float d, float L) {
  return fabsf(d) > 0.5f * L ? d - copysignf(L, d) : d;
}

// exact test d^2 <= r^2 (offsets along periodic axes: nearest images)
__device__ __forceinline__ bool exact_in(double xi, double yi, double zi, double xj, double yj,
                                         double zj, double r2, double* d2out, double Lx = 0.0,
                                         double Ly = 0.0) {
  const double dx = min_image(__dsub_rn(xj, xi), Lx), dy = min_image(__dsub_rn(yj, yi), Ly);
  const double dz = __dsub_rn(zj, zi);
  const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  *d2out = d2;
  return d2 <= r2;
}

// Candidate order of the truncating searches: squared distance, then the key
// (orig id << 1) | mirror. Squared distances are never negative (nor NaN:
// such pairs fail the radius test), so the bit patterns of the doubles order
// as their values and are compared as integers, off the FP64 pipe.
__device__ __forceinline__ bool cand_less(uint64_t da, uint32_t ka, uint64_t db, uint32_t kb) {
  if (da != db) return da < db;
  return ka < kb;
}

__device__ __forceinline__ void stencil_stats(bool live, int c, int cap, DevDiag* dg);

// Stencil of particle s; every lane of the warp must call it (live or not).
// stats = false leaves the stencil-size statistics alone (candidate lists).
// PER: the grid may have periodic axes (GridCol::Lx, Ly).
// KEEP: truncate to cap entries; keep_mode 1 keeps the cap nearest,
// keep_mode 2 the first cap of the octant-balanced ordering.
template <bool KEEP, bool PER = false>
__device__ __forceinline__ void neighbors_body(
    int s, bool live, int n, const double* __restrict__ x, const double* __restrict__ y,
    const double* __restrict__ z, const float4* __restrict__ pf,
    const int32_t* __restrict__ colid, const int32_t* __restrict__ ids,
    const GridCol* __restrict__ grids, const uint32_t* __restrict__ start,
    const double* __restrict__ radius, double r_const, int mirror_mode, double floor_z, int cap,
    int32_t* __restrict__ nbr, int32_t* __restrict__ cnt, DevDiag* __restrict__ dg,
    bool stats = true, int keep_mode = 1) {
  int c = 0;
  bool over = false;
  if (live) {
    const GridCol g = grids[colid[s]];
    const double xi = x[s], yi = y[s], zi = z[s];
    const double r = radius ? radius[s] : r_const;
    const double r2 = r * r;
    const float r2f = __double2float_rn(r2);
    const float4 pi = pf[s];
    const float fz2 = __double2float_rn(2.0 * (floor_z - g.oz));
    // FP32 prefilter band. Coordinates are origin-relative floats with error
    // <= 2^-24 |coordinate|; for a pair near the sphere the squared-distance
    // error is below about (4 L + 2) 2^-23 r^2 with L the largest coordinate
    // (mirror height included) over r. Pairs inside the band take the FP64 test.
    const float rf = __double2float_rn(r);
    // (A periodic axis adds a subtraction of the period: its length joins the
    // largest coordinate.)
    const float cmax = fmaxf(fmaxf(fmaxf(fabsf(pi.x), fabsf(pi.y)), fmaxf(fabsf(pi.z), fabsf(fz2))),
                             PER ? fmaxf(g.Lxf, g.Lyf) : 0.f);
    const float L = (4.0f * cmax + 4.0f * rf) / rf;
    const float band = (1.0f + L) * 0x1p-19f;
    const float lo = r2f * (1.0f - band), hi = r2f * (1.0f + band);
    const bool exact_only = !(band < 0.25f);  // far from the origin: FP64 for every pair
    const float Lxf = g.Lxf, Lyf = g.Lyf;
    float cdf[KEEP ? kMaxCand : 1];  // FP32 squared distances (the ordering's screen)
    uint32_t cj[KEEP ? kMaxCand : 1];
    uint8_t co[KEEP ? kMaxCand : 1];  // octant: bit 0 dx >= 0, bit 1 dy >= 0, bit 2 dz >= 0
    const int ncx = g.nx, ncy = g.ny, ncz = g.nz;
    // periodic axes wrap (>= 3 cells); float tests keep the FP64 pipe free
    const bool perx = PER && g.Lxf > 0.f, pery = PER && g.Lyf > 0.f;
    const int cx = cell_coord(xi, g.ox, g.icx, ncx);
    const int cy = cell_coord(yi, g.oy, g.icy, ncy);
    // cells cx-1..cx+1 along x as contiguous ranges of the cell table: one
    // range, or on a periodic axis at the first or last cell two (the pair
    // inside the grid, then the wrapped cell)
    const bool split = perx && (cx == 0 || cx == ncx - 1);
    const int xa0 = split ? (cx == 0 ? 0 : ncx - 2) : max(cx - 1, 0);
    const int xb0 = split ? (cx == 0 ? 1 : ncx - 1) : min(cx + 1, ncx - 1);
    const int xw = cx == 0 ? ncx - 1 : 0;  // the wrapped cell (split only)
    const int y0 = pery ? cy - 1 : max(cy - 1, 0), y1 = pery ? cy + 1 : min(cy + 1, ncy - 1);
    for (int pass = 0; pass < (mirror_mode ? 2 : 1); ++pass) {
      const double qz = pass == 0 ? zi : 2.0 * floor_z - zi;
      const int cz = cell_coord(qz, g.oz, g.icz, ncz);
      const int z0 = max(cz - 1, 0), z1 = min(cz + 1, ncz - 1);
      for (int kz = z0; kz <= z1; ++kz)
        for (int kyy = y0; kyy <= y1; ++kyy)
          for (int sx = 0; sx < (split ? 2 : 1); ++sx) {
            const int ky = kyy < 0 ? kyy + ncy : (kyy >= ncy ? kyy - ncy : kyy);  // (pery)
            const int64_t c0 = cell_id(g, sx ? xw : xa0, ky, kz);
            const int64_t c1 = cell_id(g, sx ? xw : xb0, ky, kz);
            const uint32_t b = start[c0], e = start[c1 + 1];
            // the range in chunks of kSearchChunk: their loads issue together
            for (uint32_t j0 = b; j0 < e; j0 += kSearchChunk) {
              float4 pc[kSearchChunk];
#pragma unroll
              for (int t = 0; t < kSearchChunk; ++t) pc[t] = j0 + t < e ? pf[j0 + t] : pi;
#pragma unroll
              for (int t = 0; t < kSearchChunk; ++t) {
              const uint32_t j = j0 + t;
              if (j >= e || (pass == 0 && (int)j == s)) continue;
              const float4 pj = pc[t];
              float dxf = pj.x - pi.x, dyf = pj.y - pi.y;
              if (PER) {  // nearest image (exact no-op for a period of 0)
                dxf = min_image_f(dxf, Lxf);
                dyf = min_image_f(dyf, Lyf);
              }
              const float dzf = (pass == 0 ? pj.z : fz2 - pj.z) - pi.z;
              const float d2f = dxf * dxf + dyf * dyf + dzf * dzf;
              if (!exact_only && d2f > hi) continue;
              double d2 = 0.0;
              bool in;
              uint8_t oct = 0;
              // (the octant rule forms octants from the FP64 offsets, so its
              // candidates all take the FP64 test)
              if (!exact_only && d2f < lo && !(KEEP && keep_mode == 2)) {
                in = true;
              } else {
                const double zj = pass == 0 ? z[j] : __dsub_rn(2.0 * floor_z, z[j]);
                in = exact_in(xi, yi, zi, x[j], y[j], zj, r2, &d2, PER ? g.Lx : 0.0,
                              PER ? g.Ly : 0.0);
                // (caller stencils are never periodic: the sign of x_j - x_i
                // in FP64 is that of the comparison)
                if (KEEP && keep_mode == 2)
                  oct = (uint8_t)((x[j] >= xi ? 1 : 0) | (y[j] >= yi ? 2 : 0) | (zj >= zi ? 4 : 0));
              }
              if (!in) continue;
              const uint32_t code = j | (pass ? kMirrorBit : 0u);
              if (KEEP) {
                if (c < kMaxCand) {
                  cdf[c] = d2f;
                  cj[c] = code;
                  co[c] = oct;
                } else {
                  over = true;
                }
              } else if (c < cap) {
                nbr[(int64_t)c * n + s] = (int32_t)code;
              }
              ++c;
              }
            }
          }
    }
    if (KEEP) {
      int m = c < kMaxCand ? c : kMaxCand;
      if (m > cap) {
        // tie-break keys (original index, then real before mirror), read once
        uint32_t kk[kMaxCand];
        for (int t = 0; t < m; ++t)
          kk[t] = ((uint32_t)ids[cj[t] & ~kMirrorBit] << 1) | (cj[t] >> 31);
        // The order is by the FP64 squared distance, then the key. The FP32
        // distances are within band r^2 of it (the prefilter's bound, for
        // every pair within the radius), so two candidates whose FP32
        // distances differ by more than twice that are in that order; only
        // closer pairs recompute their FP64 distances (as the test above)
        // and compare them exactly.
        const float gap = exact_only ? INFINITY : 2.0f * band * r2f;
        auto exact_bits = [&](uint32_t code) {
          const int j = code & ~kMirrorBit;
          const double zj = (code >> 31) ? __dsub_rn(2.0 * floor_z, z[j]) : z[j];
          double d2 = 0.0;
          exact_in(xi, yi, zi, x[j], y[j], zj, r2, &d2);
          return (uint64_t)__double_as_longlong(d2);
        };
        auto d_less = [&](int a, int b) {
          if (cdf[a] + gap < cdf[b]) return true;
          if (cdf[b] + gap < cdf[a]) return false;
          return cand_less(exact_bits(cj[a]), kk[a], exact_bits(cj[b]), kk[b]);
        };
        // octant-balanced: each candidate's round is its nearest-first rank
        // among the candidates of its own octant (stored over co[])
        if (keep_mode == 2) {
          uint8_t rk[kMaxCand];
          for (int t = 0; t < m; ++t) {
            int r = 0;
            for (int u = 0; u < m; ++u)
              r += (u != t && co[u] == co[t] && d_less(u, t));
            rk[t] = (uint8_t)r;
          }
          for (int t = 0; t < m; ++t) co[t] = rk[t];
        }
        // the first cap of the ordering (keys are unique, so it is one set in
        // one order): a max-heap of cap candidate indices, in which a
        // candidate that precedes the top replaces it; then heapsort, so that
        // hp[0 .. cap-1] lists them in ascending order
        auto before = [&](int a, int b) {
          if (keep_mode == 2 && co[a] != co[b]) return co[a] < co[b];  // round first
          return d_less(a, b);
        };
        uint8_t hp[LP_MAX_CAP];
        auto sift_down = [&](int i, int len) {
          for (;;) {
            const int l = 2 * i + 1;
            if (l >= len) break;
            int big = l;
            if (l + 1 < len && before(hp[l], hp[l + 1])) big = l + 1;
            if (!before(hp[i], hp[big])) break;
            const uint8_t t = hp[i]; hp[i] = hp[big]; hp[big] = t;
            i = big;
          }
        };
        for (int t = 0; t < cap; ++t) hp[t] = (uint8_t)t;
        for (int i = cap / 2 - 1; i >= 0; --i) sift_down(i, cap);
        for (int t = cap; t < m; ++t)
          if (before(t, hp[0])) {
            hp[0] = (uint8_t)t;
            sift_down(0, cap);
          }
        for (int e = cap - 1; e > 0; --e) {
          const uint8_t t = hp[0]; hp[0] = hp[e]; hp[e] = t;
          sift_down(0, e);
        }
        uint32_t kept[LP_MAX_CAP];
        for (int t = 0; t < cap; ++t) kept[t] = cj[hp[t]];
        for (int t = 0; t < cap; ++t) cj[t] = kept[t];
        m = cap;
      }
      for (int t = 0; t < m; ++t) nbr[(int64_t)t * n + s] = (int32_t)cj[t];
      c = m;
    } else {
      over = c > cap;
    }
    cnt[s] = c;
  }
  warp_count(&dg->n_overflow, live && over);
  if (live && over) atomicOr(&dg->flags, (unsigned)LP_FLAG_OVERFLOW);
  if (stats) stencil_stats(live, c, cap, dg);
}

// Stencil size statistics of one warp (every lane calls it): total rows,
// stencils, smallest and largest stencil.
__device__ __forceinline__ void stencil_stats(bool live, int c, int cap, DevDiag* dg) {
  {
    // total stencil rows and stencils (warp-reduced)
    unsigned long long rows = live ? (unsigned long long)min(c, cap) : 0ull;
    for (int o = 16; o > 0; o >>= 1) rows += __shfl_xor_sync(0xffffffffu, rows, o);
    const unsigned live_n = __popc(__ballot_sync(0xffffffffu, live));
    if ((threadIdx.x & 31) == 0 && live_n) {
      atomicAdd(&dg->n_stencil_rows, rows);
      atomicAdd(&dg->n_stencils, (unsigned long long)live_n);
    }
  }
  // stencil size range (warp-reduced)
  int mn = live ? c : INT32_MAX, mx = live ? c : 0;
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (mn != INT32_MAX) atomicMin(&dg->min_stencil, mn);
    atomicMax(&dg->max_stencil, mx);
  }
}

// Verlet filter of particle s: the stencil of this step is every candidate
// (found within radius + skin at the last search) that passes the exact
// radius test, in candidate order. Same FP32 prefilter and uncontracted FP64
// test as the search. Every lane of the warp must call it (live or not).
// With vs.marg set, a particle whose candidates provably all kept their side
// of the radius since its last filter (VerletSkip) keeps its stencil, and a
// filtered particle records its margin, a lower bound of min |d - r| over its
// candidates: with m a lower bound of |d^2 - r^2|, |d - r| = m / (d + r) >=
// m r / (2 r^2 + m), increasing in m, so the smallest m bounds every
// candidate (one beyond 2r has |d - r| > r, above any such bound). m is the
// exact FP64 |d^2 - r^2| where the filter computes it (the prefilter band),
// else the FP32 one net of its error bound e2f: each FP32 offset is within
// ec = 2^-24 (6 cmax + 6 r) of the exact one (rounded positions, the
// difference, the mirror height or the period), so the FP32 d^2 of a pair
// within 2r is within ec (7 r + 3 ec) plus 16 roundings of r^2 (the sums,
// r^2 itself and the subtractions that form m).
// (TRACK: vs is set; without it the kernel is the plain filter)
template <bool PER = false, bool TRACK = false>
__device__ __forceinline__ void filter_body(
    int s, bool live, int n, const double* __restrict__ x, const double* __restrict__ y,
    const double* __restrict__ z, const float4* __restrict__ pf,
    const int32_t* __restrict__ cand, const int32_t* __restrict__ ccnt, int capc,
    const GridCol* __restrict__ grids, const int32_t* __restrict__ colid, double r,
    double floor_z, int cap, int32_t* __restrict__ nbr, int32_t* __restrict__ cnt,
    DevDiag* __restrict__ dg, VerletSkip vs = VerletSkip{}) {
  int c = 0;
  bool over = false, built = live;
  if (TRACK && live) {
    const float mg = vs.marg[s];
    if (mg > 0.f && 2.f * (vs.dmax[s] + __uint_as_float(*vs.dmax_all)) < mg) {  // (no NaN)
      c = cnt[s];
      over = c > cap || ccnt[s] > capc;
      built = false;
    }
  }
  if (built) {
    const GridCol g = grids[colid[s]];
    const double xi = x[s], yi = y[s], zi = z[s];
    const double r2 = r * r;
    const float r2f = __double2float_rn(r2);
    const float4 pi = pf[s];
    const float fz2 = __double2float_rn(2.0 * (floor_z - g.oz));
    // FP32 prefilter band, as in neighbors_body
    const float rf = __double2float_rn(r);
    const float cmax = fmaxf(fmaxf(fmaxf(fabsf(pi.x), fabsf(pi.y)), fmaxf(fabsf(pi.z), fabsf(fz2))),
                             PER ? fmaxf(g.Lxf, g.Lyf) : 0.f);
    const float L = (4.0f * cmax + 4.0f * rf) / rf;
    const float Lxf = g.Lxf, Lyf = g.Lyf;
    const float band = (1.0f + L) * 0x1p-19f;
    const float lo = r2f * (1.0f - band), hi = r2f * (1.0f + band);
    const bool exact_only = !(band < 0.25f);  // far from the origin: FP64 for every pair
    const int m = min(ccnt[s], capc);
    float m2 = 3.f * r2f;  // lower bound of min |d^2 - r^2| (at most 3 r^2: see above)
    const float ec = 0x1p-24f * (6.f * cmax + 6.f * rf);
    const float e2f = (ec * (7.f * rf + 3.f * ec) + 16.f * 0x1p-24f * r2f) * (1.f + 0x1p-10f);
    // Candidates in chunks of kFilterChunk: the chunk's position gathers are
    // issued together and the next chunk's codes load while this one is
    // tested, so each thread keeps several gathers in flight. The stencil
    // keeps the candidates' order.
    uint32_t code[kFilterChunk];
#pragma unroll
    for (int t = 0; t < kFilterChunk; ++t)
      code[t] = t < m ? (uint32_t)cand[(int64_t)t * n + s] : 0u;
    for (int k0 = 0; k0 < m; k0 += kFilterChunk) {
      float4 pj[kFilterChunk];
#pragma unroll
      for (int t = 0; t < kFilterChunk; ++t)
        pj[t] = k0 + t < m ? pf[min(code[t] & ~kMirrorBit, (uint32_t)(n - 1))] : pi;
      uint32_t next[kFilterChunk];
#pragma unroll
      for (int t = 0; t < kFilterChunk; ++t) {
        const int k = k0 + kFilterChunk + t;
        next[t] = k < m ? (uint32_t)cand[(int64_t)k * n + s] : 0u;
      }
#pragma unroll
      for (int t = 0; t < kFilterChunk; ++t) {
        const uint32_t cd = code[t];
        const int j = cd & ~kMirrorBit;
        // past the list, or a stale or corrupt stencil entry
        if (k0 + t >= m || (unsigned)j >= (unsigned)n) continue;
        const bool mir = cd >> 31;
        float dxf = pj[t].x - pi.x, dyf = pj[t].y - pi.y;
        if (PER) {  // nearest image (exact no-op for a period of 0)
          dxf = min_image_f(dxf, Lxf);
          dyf = min_image_f(dyf, Lyf);
        }
        const float dzf = (mir ? fz2 - pj[t].z : pj[t].z) - pi.z;
        const float d2f = dxf * dxf + dyf * dyf + dzf * dzf;
        if (!exact_only && d2f > hi) {
          if (TRACK) m2 = fminf(m2, (d2f - r2f) - e2f);
          continue;
        }
        bool in;
        if (!exact_only && d2f < lo) {
          in = true;
          if (TRACK) m2 = fminf(m2, (r2f - d2f) - e2f);
        } else {
          double d2;
          const double zj = mir ? __dsub_rn(2.0 * floor_z, z[j]) : z[j];
          in = exact_in(xi, yi, zi, x[j], y[j], zj, r2, &d2, PER ? g.Lx : 0.0, PER ? g.Ly : 0.0);
          // (the FP64 d^2 errs by far less than 2^-40 r^2)
          if (TRACK) m2 = fminf(m2, __double2float_rd(fabs(d2 - r2) - 0x1p-40 * r2));
        }
        if (!in) continue;
        if (c < cap) nbr[(int64_t)c * n + s] = (int32_t)cd;
        ++c;
      }
#pragma unroll
      for (int t = 0; t < kFilterChunk; ++t) code[t] = next[t];
    }
    over = c > cap || ccnt[s] > capc;
    cnt[s] = c;
    if (TRACK) {  // rounded down (1 - 2^-20: the FP32 evaluation and rf, r2f)
      const float mm = fmaxf(0.f, m2);
      vs.marg[s] = mm * rf / (2.f * r2f + mm) * (1.f - 0x1p-20f);
    }
  }
  warp_count(&dg->n_overflow, live && over);
  if (live && over) atomicOr(&dg->flags, (unsigned)LP_FLAG_OVERFLOW);
  stencil_stats(built, c, cap, dg);  // (stencils built this step)
}

// ------------------------------------------------------- free boundary
// Ghost particles (Sec. 3.1 items 6 and 9). The paper leaves the test and the
// placement open; the reading, also the oracle's:
//  - positions in fixed point, X = round(K x) on a power-of-two grid K with
//    K r <= 8192, offsets o_k = X_k - X_i (exact integers, along a periodic
//    axis the nearest image modulo round(K L); for stencil entries
//    |o| <= 8193, so squares and pair sums fit 32 bits);
//  - weights w_k = max(0, R2 - |o_k|^2), R2 = round((K r)^2);
//  - one-sided stencil: |S| > 0.22 K h sum w_k with S = sum w_k o_k;
//  - a ghost at -o_k for every entry with o_k . S >= (K h / 2) |S| (o_k . S
//    exact in 64 bits) whose reflection has no entry within h/2 and, with
//    floor mirrors, does not lie below the floor ((z_i + z_i) - z_k <
//    floor_z).
// The FP64 operations are _rn intrinsics in the oracle's order, so the
// decisions are the oracle's bit for bit.
//
// A ghost is the reflection of an existing entry, so it is stored as a flag
// (kGhostBit) on that entry: the entry stands for two rows, itself and its
// reflection. Flagged entries are moved to the end of the stencil and
// gcnt[s] counts them; the stencil size is unchanged, but entries plus
// ghosts must fit in cap (else LP_FLAG_OVERFLOW). Positions are stored
// relative to the column's fixed-point origin (an exact integer shift), as
// 32-bit integers.

// offset along an axis of integer period P (0: none), nearest image
__device__ __forceinline__ int wrap_fix(int o, int P) {
  return P > 0 ? (2 * o > P ? o - P : (2 * o < -P ? o + P : o)) : o;
}

// fixed-point position (x, y, z, floor-mirror height) of particle s
__device__ __forceinline__ void ghost_fix_body(int s, const double* __restrict__ x,
                                               const double* __restrict__ y,
                                               const double* __restrict__ z,
                                               const int32_t* __restrict__ colid,
                                               const GridCol* __restrict__ grids, double grid,
                                               double floor_z, int4* __restrict__ X) {
  const GridCol g = grids[colid[s]];
  const long long ox = __double2ll_rn(__dmul_rn(g.ox, grid));
  const long long oy = __double2ll_rn(__dmul_rn(g.oy, grid));
  const long long oz = __double2ll_rn(__dmul_rn(g.oz, grid));
  const double zm = __dsub_rn(__dmul_rn(2.0, floor_z), z[s]);
  X[s] = make_int4((int)(__double2ll_rn(__dmul_rn(x[s], grid)) - ox),
                   (int)(__double2ll_rn(__dmul_rn(y[s], grid)) - oy),
                   (int)(__double2ll_rn(__dmul_rn(z[s], grid)) - oz),
                   (int)(__double2ll_rn(__dmul_rn(zm, grid)) - oz));
}

// Flags the entries of particle s whose reflections are ghosts; every lane of
// the warp must call it (live or not).
// The sums of the one-sided test over the entries of particle s (weights
// r^2 - d^2 in fixed point): S = sum w o, W = sum w; with STORE the offsets o
// are kept for the clearance check. False if an entry is out of range or
// already carries a ghost (the stencil is then left alone).
template <bool STORE>
__device__ __forceinline__ bool ghost_sums(int s, int n, const int4* __restrict__ X,
                                           const int32_t* __restrict__ nbr, int m, int4 xi,
                                           const StepConsts& K, short (*o)[LP_MAX_CAP],
                                           long long& S0, long long& S1, long long& S2,
                                           long long& W) {
  S0 = S1 = S2 = W = 0;
  const int R2 = (int)K.ghost_R2;
  const int PX = (int)K.ghost_PX, PY = (int)K.ghost_PY;  // integer periods (0: none)
  bool ok = m > 0;
  // software pipeline: codes two entries ahead, positions one ahead
  uint32_t nc = m > 0 ? (uint32_t)nbr[s] : 0u;
  uint32_t nn = m > 1 ? (uint32_t)nbr[(int64_t)n + s] : 0u;
  int4 nx = m > 0 ? X[min(nc & kIndexMask, (uint32_t)(n - 1))] : xi;
  for (int k = 0; k < m; ++k) {
    const uint32_t code = nc;
    const int4 xj = nx;
    if (k + 1 < m) {
      nc = nn;
      nx = X[min(nc & kIndexMask, (uint32_t)(n - 1))];
      if (k + 2 < m) nn = (uint32_t)nbr[(int64_t)(k + 2) * n + s];
    }
    if ((code & kIndexMask) >= (uint32_t)n || (code & kGhostBit)) { ok = false; break; }
    const int o0 = wrap_fix(xj.x - xi.x, PX), o1 = wrap_fix(xj.y - xi.y, PY);
    const int o2 = ((code & kMirrorBit) ? xj.w : xj.z) - xi.z;
    if (STORE) { o[0][k] = (short)o0; o[1][k] = (short)o1; o[2][k] = (short)o2; }
    const int q = (o0 * o0 + o1 * o1) + o2 * o2;
    const int w = q < R2 ? R2 - q : 0;
    S0 += (long long)w * o0;
    S1 += (long long)w * o1;
    S2 += (long long)w * o2;
    W += w;
  }
  return ok;
}
// the one-sided test: |S| > 0.22 h W (in the fixed-point units)
__device__ __forceinline__ bool ghost_one_sided(long long S0, long long S1, long long S2,
                                                long long W, const StepConsts& K,
                                                double* s2out) {
  const double sx = (double)S0, sy = (double)S1, sz = (double)S2;
  const double s2 = __dadd_rn(__dadd_rn(__dmul_rn(sx, sx), __dmul_rn(sy, sy)), __dmul_rn(sz, sz));
  const double lim = __dmul_rn(__dmul_rn(0.22, K.ghost_hk), (double)W);
  *s2out = s2;
  return s2 > __dmul_rn(lim, lim);
}

// First half of the ghost kernels (every particle): the one-sided test
// alone. A one-sided particle is appended, in no set order, at
// olist[(*ocount)++] for ghost_body; the others get no ghosts (gcnt 0). Every
// lane of the warp must call it (live or not).
__device__ __forceinline__ void ghost_scan_body(int s, bool live, int n,
                                                const int4* __restrict__ X,
                                                const int32_t* __restrict__ nbr,
                                                const int32_t* __restrict__ cnt,
                                                int32_t* __restrict__ gcnt, const StepConsts& K,
                                                int32_t* __restrict__ olist,
                                                int* __restrict__ ocount) {
  bool side = false;
  if (live) {
    const int m = min(cnt[s], K.cap);
    long long S0, S1, S2, W;
    double s2;
    side = ghost_sums<false>(s, n, X, nbr, m, X[s], K, nullptr, S0, S1, S2, W) &&
           ghost_one_sided(S0, S1, S2, W, K, &s2);
    if (!side) gcnt[s] = 0;
  }
  const unsigned has = __ballot_sync(0xffffffffu, side);
  if (has) {
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0) base = atomicAdd(ocount, __popc(has));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (side) olist[base + __popc(has & ((1u << lane) - 1u))] = s;
  }
}

// glist (optional): every particle with ghosts is appended, in no set order,
// at glist[(*gcount)++], so that the twin kernels need visit only those.
__device__ __forceinline__ void ghost_body(int s, bool live, int n, const double* __restrict__ z,
                                           const int4* __restrict__ X,
                                           int32_t* __restrict__ nbr, const int32_t* __restrict__ cnt,
                                           int32_t* __restrict__ gcnt, const StepConsts& K,
                                           DevDiag* __restrict__ dg,
                                           int32_t* __restrict__ glist = nullptr,
                                           int* __restrict__ gcount = nullptr) {
  int twins = 0;
  bool over = false;
  if (live) {
    const int m = min(cnt[s], K.cap);
    const int4 xi = X[s];
    short o[3][LP_MAX_CAP];  // offsets of the entries (|o| <= 8193)
    long long S0, S1, S2, W;
    const bool ok = ghost_sums<true>(s, n, X, nbr, m, xi, K, o, S0, S1, S2, W);
    double s2;
    const bool side = ghost_one_sided(S0, S1, S2, W, K, &s2);
    if (ok && side) {
      const double dep = __dmul_rn(0.5, K.ghost_hk);
      const double dep2s2 = __dmul_rn(__dmul_rn(dep, dep), s2);
      const double zi = z[s];
      const double f2 = __dmul_rn(2.0, K.floor_z);
      const int clear2 = (int)K.ghost_clear2;
      unsigned long long tw = 0ull;
      for (int k = 0; k < m; ++k) {
        const int o0 = o[0][k], o1 = o[1][k], o2 = o[2][k];
        const double ds = (double)(((long long)o0 * S0 + (long long)o1 * S1) + (long long)o2 * S2);
        if (!(ds > 0.0 && __dmul_rn(ds, ds) >= dep2s2)) continue;
        if (K.mirror_mode != LP_MIRROR_NONE) {
          const uint32_t code = (uint32_t)nbr[(int64_t)k * n + s];
          const int j = code & kIndexMask;
          const double zk = (code & kMirrorBit) ? __dsub_rn(f2, z[j]) : z[j];
          if (__dsub_rn(__dadd_rn(zi, zi), zk) < K.floor_z) continue;
        }
        int hits = 0;  // entries within h/2 of the reflection
        for (int l = 0; l < m; ++l) {
          const int e0 = o[0][l] + o0, e1 = o[1][l] + o1, e2 = o[2][l] + o2;
          hits += (e0 * e0 + e1 * e1) + e2 * e2 < clear2;
        }
        if (!hits) tw |= 1ull << k;
      }
      twins = __popcll(tw);
      if (twins) {
        over = m + twins > K.cap;
        // entries without a ghost first (in their order), then the flagged ones
        int32_t cd[LP_MAX_CAP];
        for (int k = 0; k < m; ++k) cd[k] = nbr[(int64_t)k * n + s];
        int w = 0;
        for (int k = 0; k < m; ++k)
          if (!((tw >> k) & 1ull)) nbr[(int64_t)(w++) * n + s] = cd[k];
        for (int k = 0; k < m; ++k)
          if ((tw >> k) & 1ull) nbr[(int64_t)(w++) * n + s] = (int32_t)((uint32_t)cd[k] | kGhostBit);
      }
    }
    gcnt[s] = twins;
  }
  if (glist) {  // one atomic per warp for the warp's particles with ghosts
    const unsigned has = __ballot_sync(0xffffffffu, live && twins > 0);
    if (has) {
      const int lane = threadIdx.x & 31;
      int base = 0;
      if (lane == 0) base = atomicAdd(gcount, __popc(has));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (live && twins > 0) glist[base + __popc(has & ((1u << lane) - 1u))] = s;
    }
  }
  unsigned long long a = (unsigned long long)twins;
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0 && a) atomicAdd(&dg->n_ghosts, a);
  warp_count(&dg->n_overflow, live && over);
  if (live && over) atomicOr(&dg->flags, (unsigned)LP_FLAG_OVERFLOW);
}

}  // namespace lp
