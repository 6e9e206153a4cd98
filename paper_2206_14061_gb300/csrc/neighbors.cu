// Cell sort and neighbour search (Sec. 3.1 items 4-6 and the solid-boundary
// mirrors of item 9).
//
// The paper stores particles in a distributed adaptive octree (p4est). On one
// GPU a uniform grid with cell edge >= the largest stencil radius does the same
// job: particles are counting-sorted by cell (stable by original index inside
// a cell, so the order is a deterministic function of the positions), and each
// particle scans the 3x3x3 block of cells around itself (and around its
// reflection in the floor, for mirror neighbours).
//
// The inclusion test is exact: ((dx*dx)+(dy*dy))+(dz*dz) <= r*r in FP64 with
// no contraction (__dmul_rn/__dadd_rn), dx = x_j - x_i. An FP32 prefilter on
// origin-relative coordinates decides every pair whose squared distance is
// farther than 2^-6 r^2 from r^2; only pairs in that band pay for the FP64 test.
#include "lp_internal.cuh"

namespace lp {

// ---------------------------------------------------------------- helpers

__global__ void k_fill_colid(int n, const int32_t* __restrict__ offs, int ncol,
                             int32_t* __restrict__ colid) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  int lo = 0, hi = ncol - 1;  // last c with offs[c] <= s
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (offs[mid] <= s) lo = mid; else hi = mid - 1;
  }
  colid[s] = lo;
}

// Per-column bounding box and largest radius: block c reduces column c.
__global__ void k_bbox(const double* __restrict__ x, const double* __restrict__ y,
                       const double* __restrict__ z, const double* __restrict__ radius,
                       const int32_t* __restrict__ offs, double* __restrict__ out) {
  const int c = blockIdx.x;
  const int b = offs[c], e = offs[c + 1];
  double v[7] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY, 0.0};
  for (int s = b + threadIdx.x; s < e; s += blockDim.x) {
    const double px = x[s], py = y[s], pz = z[s];
    // non-finite positions do not widen the grid; they are clamped into it
    if (isfinite(px) && isfinite(py) && isfinite(pz)) {
      v[0] = fmin(v[0], px); v[1] = fmin(v[1], py); v[2] = fmin(v[2], pz);
      v[3] = fmax(v[3], px); v[4] = fmax(v[4], py); v[5] = fmax(v[5], pz);
    }
    if (radius) v[6] = fmax(v[6], radius[s]);
  }
  __shared__ double sh[7][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    double t = v[k];
    for (int o = 16; o > 0; o >>= 1) {
      double u = __shfl_xor_sync(0xffffffffu, t, o);
      t = (k < 3) ? fmin(t, u) : fmax(t, u);
    }
    if (lane == 0) sh[k][wid] = t;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    const int k = threadIdx.x;
    double t = sh[k][0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      t = (k < 3) ? fmin(t, sh[k][w]) : fmax(t, sh[k][w]);
    out[7 * c + k] = t;
  }
}

// Cell key of every particle; particles with a non-finite coordinate go to
// the extra bucket `ncell`, which no search visits.
__global__ void k_keys(int n, const double* __restrict__ x, const double* __restrict__ y,
                       const double* __restrict__ z, const int32_t* __restrict__ colid,
                       const GridCol* __restrict__ grids, uint32_t ncell,
                       uint32_t* __restrict__ key, uint32_t* __restrict__ count) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  if (!(isfinite(x[s]) && isfinite(y[s]) && isfinite(z[s]))) {
    key[s] = ncell;
    atomicAdd(&count[ncell], 1u);
    return;
  }
  const GridCol g = grids[colid[s]];
  const int cx = cell_coord(x[s], g.ox, g.inv_c, g.nx);
  const int cy = cell_coord(y[s], g.oy, g.inv_c, g.ny);
  const int cz = cell_coord(z[s], g.oz, g.inv_c, g.nz);
  const uint32_t k = (uint32_t)cell_id(g, cx, cy, cz);
  key[s] = k;
  atomicAdd(&count[k], 1u);
}

// --------------------------------------------------- exclusive scan (u32)
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

__global__ void k_scan_tiles(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                             uint32_t* __restrict__ tile_sum, int64_t n) {
  __shared__ uint32_t tot;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t t = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    t += v[k];
  }
  uint32_t ex = block_exclusive_scan(t, &tot);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = ex;
    ex += v[k];
  }
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// exclusive scan of the tile sums by one block, in chunks
__global__ void k_scan_top(uint32_t* __restrict__ tile_sum, int ntiles) {
  __shared__ uint32_t tot;
  uint32_t carry = 0;
  for (int b = 0; b < ntiles; b += kScanThreads) {
    const int i = b + threadIdx.x;
    const uint32_t v = i < ntiles ? tile_sum[i] : 0u;
    const uint32_t ex = block_exclusive_scan(v, &tot);
    if (i < ntiles) tile_sum[i] = ex + carry;
    carry += tot;
    __syncthreads();
  }
}

__global__ void k_scan_add(uint32_t* __restrict__ out, const uint32_t* __restrict__ tile_sum,
                           int64_t n) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  const uint32_t add = tile_sum[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) out[base + k] += add;
}

void exclusive_scan(const uint32_t* in, uint32_t* out, uint32_t* tile_sum, int64_t n,
                    cudaStream_t st) {
  const int ntiles = (int)((n + kScanTile - 1) / kScanTile);
  k_scan_tiles<<<ntiles, kScanThreads, 0, st>>>(in, out, tile_sum, n);
  k_scan_top<<<1, kScanThreads, 0, st>>>(tile_sum, ntiles);
  k_scan_add<<<ntiles, kScanThreads, 0, st>>>(out, tile_sum, n);
}

int64_t scan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

// ------------------------------------------------------------ scatter/sort

__global__ void k_scatter(int n, const uint32_t* __restrict__ key,
                          const uint32_t* __restrict__ start, uint32_t* __restrict__ fill,
                          int32_t* __restrict__ tmp) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint32_t k = key[s];
  const uint32_t pos = start[k] + atomicAdd(&fill[k], 1u);
  tmp[pos] = s;
}

// Order each cell's particles by original index (insertion sort; cells hold
// about (cell edge / h)^3 particles). A cell crowded beyond kSortCap (only
// after a blow-up) keeps its arrival order: the stencils stay exact, only the
// row order inside them loses its determinism.
constexpr uint32_t kSortCap = 1024;
__global__ void k_cell_sort(int64_t ncell, const uint32_t* __restrict__ start,
                            int32_t* __restrict__ tmp, const int32_t* __restrict__ ids) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
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
__global__ void k_gather(int n, const int32_t* __restrict__ tmp, const double* const* __restrict__ src,
                         double* const* __restrict__ dst, int nsrc,
                         const int32_t* __restrict__ ids_in, int32_t* __restrict__ ids_out,
                         const int32_t* __restrict__ col_in, int32_t* __restrict__ col_out,
                         const GridCol* __restrict__ grids, float4* __restrict__ pf) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int s = tmp[t];
  for (int f = 0; f < nsrc; ++f) dst[f][t] = src[f][s];
  ids_out[t] = ids_in[s];
  const int c = col_in[s];
  col_out[t] = c;
  const GridCol g = grids[c];
  pf[t] = make_float4(__double2float_rn(src[0][s] - g.ox), __double2float_rn(src[1][s] - g.oy),
                      __double2float_rn(src[2][s] - g.oz), 0.f);
}

// ------------------------------------------------------- neighbour search

__device__ __forceinline__ bool exact_in(double xi, double yi, double zi, double xj, double yj,
                                         double zj, double r2, double* d2out) {
  const double dx = __dsub_rn(xj, xi), dy = __dsub_rn(yj, yi), dz = __dsub_rn(zj, zi);
  const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  *d2out = d2;
  return d2 <= r2;
}

// ordering of keep-nearest candidates: nearest first, then original index,
// then real before mirror
__device__ __forceinline__ bool cand_less(double da, uint32_t ka, double db, uint32_t kb) {
  if (da != db) return da < db;
  return ka < kb;  // ka = (orig id << 1) | mirror
}

template <bool KEEP>
__global__ void __launch_bounds__(kBlock)
k_neighbors(int n, const double* __restrict__ x, const double* __restrict__ y,
            const double* __restrict__ z, const float4* __restrict__ pf,
            const int32_t* __restrict__ colid, const int32_t* __restrict__ ids,
            const GridCol* __restrict__ grids, const uint32_t* __restrict__ start,
            const double* __restrict__ radius, double r_const, int mirror_mode, double floor_z,
            int cap, int32_t* __restrict__ nbr, int32_t* __restrict__ cnt,
            DevDiag* __restrict__ dg) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = s < n;
  int c = 0;
  bool over = false;
  if (live) {
    const GridCol g = grids[colid[s]];
    const double xi = x[s], yi = y[s], zi = z[s];
    const double r = radius ? radius[s] : r_const;
    const double r2 = r * r;
    const float r2f = __double2float_rn(r2);
    const float lo = r2f * (1.0f - 0.015625f), hi = r2f * (1.0f + 0.015625f);
    const float4 pi = pf[s];
    const float lim = 4096.0f * __double2float_rn(r);
    const bool exact_only = !(fabsf(pi.x) <= lim && fabsf(pi.y) <= lim && fabsf(pi.z) <= lim);
    const float fz2 = __double2float_rn(2.0 * (floor_z - g.oz));
    double cd2[KEEP ? kMaxCand : 1];
    uint32_t cj[KEEP ? kMaxCand : 1];
    const int ncx = g.nx, ncy = g.ny, ncz = g.nz;
    const int cx = cell_coord(xi, g.ox, g.inv_c, ncx);
    const int cy = cell_coord(yi, g.oy, g.inv_c, ncy);
    const int x0 = max(cx - 1, 0), x1 = min(cx + 1, ncx - 1);
    const int y0 = max(cy - 1, 0), y1 = min(cy + 1, ncy - 1);
    for (int pass = 0; pass < (mirror_mode ? 2 : 1); ++pass) {
      const double qz = pass == 0 ? zi : 2.0 * floor_z - zi;
      const int cz = cell_coord(qz, g.oz, g.inv_c, ncz);
      const int z0 = max(cz - 1, 0), z1 = min(cz + 1, ncz - 1);
      for (int kz = z0; kz <= z1; ++kz)
        for (int ky = y0; ky <= y1; ++ky) {
          // cells kx = x0..x1 are contiguous in the cell table
          const int64_t c0 = cell_id(g, x0, ky, kz), c1 = cell_id(g, x1, ky, kz);
          const uint32_t b = start[c0], e = start[c1 + 1];
          for (uint32_t j = b; j < e; ++j) {
            if (pass == 0 && (int)j == s) continue;
            const float4 pj = pf[j];
            const float dxf = pj.x - pi.x, dyf = pj.y - pi.y;
            const float dzf = (pass == 0 ? pj.z : fz2 - pj.z) - pi.z;
            const float d2f = dxf * dxf + dyf * dyf + dzf * dzf;
            if (!exact_only && d2f > hi) continue;
            double d2 = 0.0;
            bool in;
            if (!exact_only && d2f < lo && !KEEP) {
              in = true;
            } else {
              const double zj = pass == 0 ? z[j] : __dsub_rn(2.0 * floor_z, z[j]);
              in = exact_in(xi, yi, zi, x[j], y[j], zj, r2, &d2);
            }
            if (!in) continue;
            const uint32_t code = j | (pass ? kMirrorBit : 0u);
            if (KEEP) {
              if (c < kMaxCand) {
                cd2[c] = d2;
                cj[c] = code;
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
    if (KEEP) {
      int m = c < kMaxCand ? c : kMaxCand;
      if (m > cap) {
        // partial selection sort: the cap nearest to the front
        for (int t = 0; t < cap; ++t) {
          int best = t;
          uint32_t kb = ((uint32_t)ids[cj[t] & ~kMirrorBit] << 1) | (cj[t] >> 31);
          for (int u = t + 1; u < m; ++u) {
            const uint32_t ku = ((uint32_t)ids[cj[u] & ~kMirrorBit] << 1) | (cj[u] >> 31);
            if (cand_less(cd2[u], ku, cd2[best], kb)) { best = u; kb = ku; }
          }
          const double td = cd2[t]; cd2[t] = cd2[best]; cd2[best] = td;
          const uint32_t tj = cj[t]; cj[t] = cj[best]; cj[best] = tj;
        }
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
  if (live && over) atomicOr(&dg->flags, (unsigned)LP_FLAG_OVERFLOW);
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

// Stencils from sorted indices to caller indices.
__global__ void k_nbr_to_caller(int n, int cap, const int32_t* __restrict__ ids,
                                const int32_t* __restrict__ nbr_s, const int32_t* __restrict__ cnt_s,
                                int32_t* __restrict__ nbr_o, int32_t* __restrict__ cnt_o) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int o = ids[s];
  const int c = cnt_s[s];
  cnt_o[o] = c;
  const int m = c < cap ? c : cap;
  for (int k = 0; k < m; ++k) {
    const uint32_t code = (uint32_t)nbr_s[(int64_t)k * n + s];
    nbr_o[(int64_t)k * n + o] = (int32_t)(((uint32_t)ids[code & ~kMirrorBit]) | (code & kMirrorBit));
  }
}

// ----------------------------------------------------------- host wrappers

void launch_fill_colid(int n, const int32_t* offs, int ncol, int32_t* colid, cudaStream_t st) {
  k_fill_colid<<<(n + 255) / 256, 256, 0, st>>>(n, offs, ncol, colid);
}
void launch_bbox(int ncol, const double* x, const double* y, const double* z, const double* radius,
                 const int32_t* offs, double* out, cudaStream_t st) {
  k_bbox<<<ncol, 256, 0, st>>>(x, y, z, radius, offs, out);
}
void launch_keys(int n, const double* x, const double* y, const double* z, const int32_t* colid,
                 const GridCol* grids, int64_t ncell, uint32_t* key, uint32_t* count,
                 cudaStream_t st) {
  k_keys<<<(n + 255) / 256, 256, 0, st>>>(n, x, y, z, colid, grids, (uint32_t)ncell, key, count);
}
void launch_scatter(int n, const uint32_t* key, const uint32_t* start, uint32_t* fill,
                    int32_t* tmp, cudaStream_t st) {
  k_scatter<<<(n + 255) / 256, 256, 0, st>>>(n, key, start, fill, tmp);
}
void launch_cell_sort(int64_t ncell, const uint32_t* start, int32_t* tmp, const int32_t* ids,
                      cudaStream_t st) {
  k_cell_sort<<<(unsigned)((ncell + 255) / 256), 256, 0, st>>>(ncell, start, tmp, ids);
}
void launch_gather(int n, const int32_t* tmp, const double* const* src, double* const* dst,
                   int nsrc, const int32_t* ids_in, int32_t* ids_out, const int32_t* col_in,
                   int32_t* col_out, const GridCol* grids, float4* pf, cudaStream_t st) {
  k_gather<<<(n + 255) / 256, 256, 0, st>>>(n, tmp, src, dst, nsrc, ids_in, ids_out, col_in,
                                            col_out, grids, pf);
}
void launch_neighbors(bool keep, int n, const double* x, const double* y, const double* z,
                      const float4* pf, const int32_t* colid, const int32_t* ids,
                      const GridCol* grids, const uint32_t* start, const double* radius,
                      double r_const, int mirror_mode, double floor_z, int cap, int32_t* nbr,
                      int32_t* cnt, DevDiag* dg, cudaStream_t st) {
  const int nb = (n + kBlock - 1) / kBlock;
  if (keep)
    k_neighbors<true><<<nb, kBlock, 0, st>>>(n, x, y, z, pf, colid, ids, grids, start, radius,
                                              r_const, mirror_mode, floor_z, cap, nbr, cnt, dg);
  else
    k_neighbors<false><<<nb, kBlock, 0, st>>>(n, x, y, z, pf, colid, ids, grids, start, radius,
                                               r_const, mirror_mode, floor_z, cap, nbr, cnt, dg);
}
void launch_nbr_to_caller(int n, int cap, const int32_t* ids, const int32_t* nbr_s,
                          const int32_t* cnt_s, int32_t* nbr_o, int32_t* cnt_o, cudaStream_t st) {
  k_nbr_to_caller<<<(n + 255) / 256, 256, 0, st>>>(n, cap, ids, nbr_s, cnt_s, nbr_o, cnt_o);
}

}  // namespace lp
