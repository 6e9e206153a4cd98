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
#include "nbr_bodies.cuh"

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

// Per-column bounding box and largest radius. Doubles are reduced through an
// order-preserving map to uint64 (atomicMin/atomicMax): a block whose
// particles all belong to one column reduces in shared memory first and
// issues 7 atomics; a block that straddles columns issues them per thread.
__device__ __forceinline__ unsigned long long ord_key(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void k_bbox_init(int ncol, unsigned long long* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 7 * ncol) return;
  out[i] = (i % 7) < 3 ? ~0ull : 0ull;  // min slots start high, max slots low
}

__global__ void k_bbox(int n, const double* __restrict__ x, const double* __restrict__ y,
                       const double* __restrict__ z, const double* __restrict__ radius,
                       const int32_t* __restrict__ colid, unsigned long long* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long v[7] = {~0ull, ~0ull, ~0ull, 0ull, 0ull, 0ull, 0ull};
  int c = -1;
  if (s < n) {
    c = colid[s];
    const double px = x[s], py = y[s], pz = z[s];
    // non-finite positions do not widen the grid (they go to their own bucket)
    if (isfinite(px) && isfinite(py) && isfinite(pz)) {
      v[0] = v[3] = ord_key(px);
      v[1] = v[4] = ord_key(py);
      v[2] = v[5] = ord_key(pz);
    }
    if (radius && isfinite(radius[s])) v[6] = ord_key(radius[s]);
  }
  const int first = blockIdx.x * blockDim.x;
  const int last = min(first + (int)blockDim.x, n) - 1;
  const bool one_col = colid[first] == colid[last];
  if (!one_col) {
    if (c >= 0)
      for (int k = 0; k < 7; ++k) {
        if (k < 3) atomicMin(&out[7 * c + k], v[k]);
        else atomicMax(&out[7 * c + k], v[k]);
      }
    return;
  }
  __shared__ unsigned long long sh[7][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    unsigned long long t = v[k];
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long u = __shfl_xor_sync(0xffffffffu, t, o);
      t = k < 3 ? min(t, u) : max(t, u);
    }
    if (lane == 0) sh[k][wid] = t;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    const int k = threadIdx.x;
    unsigned long long t = sh[k][0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = k < 3 ? min(t, sh[k][w]) : max(t, sh[k][w]);
    const int col = colid[first];
    if (k < 3) atomicMin(&out[7 * col + k], t);
    else atomicMax(&out[7 * col + k], t);
  }
}

// `search` (may be NULL: always) gates the sort kernels on a device flag
__device__ __forceinline__ bool searching(const int* search) { return !search || *search; }

__global__ void k_keys(int n, const double* __restrict__ x, const double* __restrict__ y,
                       const double* __restrict__ z, const int32_t* __restrict__ colid,
                       const GridCol* __restrict__ grids, uint32_t ncell,
                       uint32_t* __restrict__ key, uint32_t* __restrict__ count,
                       const int* search) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n && searching(search)) keys_body(s, x, y, z, colid, grids, ncell, key, count);
}

// --------------------------------------------------- exclusive scan (u32)
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
                          int32_t* __restrict__ tmp, const int* search) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n && searching(search)) scatter_body(s, key, start, fill, tmp);
}

__global__ void k_cell_sort(int64_t ncell, const uint32_t* __restrict__ start,
                            int32_t* __restrict__ tmp, const int32_t* __restrict__ ids,
                            const int* search) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncell && searching(search)) cell_sort_body(c, start, tmp, ids);
}

// without a search (flag clear) the gather keeps the order: an identity copy
__global__ void k_gather(int n, const int32_t* __restrict__ tmp, const double* const* __restrict__ src,
                         double* const* __restrict__ dst, int nsrc,
                         const int32_t* __restrict__ ids_in, int32_t* __restrict__ ids_out,
                         const int32_t* __restrict__ col_in, int32_t* __restrict__ col_out,
                         const GridCol* __restrict__ grids, float4* __restrict__ pf,
                         const int32_t* __restrict__ iota, const int* search) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n)
    gather_body(t, n, searching(search) ? tmp : iota, src, dst, nsrc, ids_in, ids_out, col_in,
                col_out, grids, pf);
}

// ------------------------------------------------------- neighbour search

template <bool KEEP, bool PER>
__global__ void __launch_bounds__(kMaxBlock)
k_neighbors(int n, const double* __restrict__ x, const double* __restrict__ y,
            const double* __restrict__ z, const float4* __restrict__ pf,
            const int32_t* __restrict__ colid, const int32_t* __restrict__ ids,
            const GridCol* __restrict__ grids, const uint32_t* __restrict__ start,
            const double* __restrict__ radius, double r_const, int mirror_mode, double floor_z,
            int cap, int32_t* __restrict__ nbr, int32_t* __restrict__ cnt,
            DevDiag* __restrict__ dg, const int* search, double* __restrict__ xref,
            int keep_mode, VerletSkip vs) {
  if (!searching(search)) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (xref && s < n) {  // positions of this search, for the displacement test
    xref[s] = x[s];
    xref[n + s] = y[s];
    xref[2 * n + s] = z[s];
    if (vs.marg) {  // new candidates: filter every particle, displacements from here
      vs.marg[s] = -1.f;
      vs.dmax[s] = 0.f;
      if (s == 0) *vs.dmax_all = 0u;
    }
  }
  neighbors_body<KEEP, PER>(s, s < n, n, x, y, z, pf, colid, ids, grids, start, radius, r_const,
                            mirror_mode, floor_z, cap, nbr, cnt, dg, xref == nullptr, keep_mode);
}

// Verlet filter (filter_body). Thread 0 clears the search flag for the
// displacement test of this step's update.
template <bool PER, bool TRACK>
__global__ void __launch_bounds__(kMaxBlock)
k_filter(int n, const double* __restrict__ x, const double* __restrict__ y,
         const double* __restrict__ z, const float4* __restrict__ pf,
         const int32_t* __restrict__ cand, const int32_t* __restrict__ ccnt, int capc,
         const GridCol* __restrict__ grids, const int32_t* __restrict__ colid, double r,
         double floor_z, int cap, int32_t* __restrict__ nbr, int32_t* __restrict__ cnt,
         DevDiag* __restrict__ dg, int* search, VerletSkip vs) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s == 0) *search = 0;
  filter_body<PER, TRACK>(s, s < n, n, x, y, z, pf, cand, ccnt, capc, grids, colid, r, floor_z,
                          cap, nbr, cnt, dg, vs);
}

// Free-surface ghosts (ghost_body): fixed-point positions, then completion of
// the stencils of one-sided particles.
__global__ void k_ghost_fix(int n, const double* __restrict__ x, const double* __restrict__ y,
                            const double* __restrict__ z, const int32_t* __restrict__ colid,
                            const GridCol* __restrict__ grids, double grid, double floor_z,
                            int4* __restrict__ X, int* __restrict__ gcount) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s == 0) gcount[0] = gcount[1] = 0;  // the two lists the ghost kernels fill next
  if (s < n) ghost_fix_body(s, x, y, z, colid, grids, grid, floor_z, X);
}

// first half: the one-sided test of every particle (gcount[1]: one-sided ones)
__global__ void __launch_bounds__(kMaxBlock)
k_ghost_scan(int n, const int4* __restrict__ X, const int32_t* __restrict__ nbr,
             const int32_t* __restrict__ cnt, int32_t* __restrict__ gcnt, const StepConsts K,
             int32_t* __restrict__ olist, int* __restrict__ gcount) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  ghost_scan_body(s, s < n, n, X, nbr, cnt, gcnt, K, olist, gcount + 1);
}

// second half: the one-sided particles of the list, in full warps (a fixed
// grid strides over the list a warp at a time, so every lane calls the body)
constexpr int kGhostBlocks = 4 * 152;
__global__ void __launch_bounds__(128)
k_ghosts(int n, const double* __restrict__ z, const int4* __restrict__ X,
         int32_t* __restrict__ nbr, const int32_t* __restrict__ cnt, int32_t* __restrict__ gcnt,
         const StepConsts K, DevDiag* __restrict__ dg, int32_t* __restrict__ glist,
         int* __restrict__ gcount, const int32_t* __restrict__ olist) {
  const int m = min(gcount[1], n);
  const int lane = threadIdx.x & 31;
  const int stride = gridDim.x * blockDim.x;
  for (int base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; base < m; base += stride) {
    const int t = base + lane;
    const bool live = t < m;
    ghost_body(live ? olist[t] : 0, live, n, z, X, nbr, cnt, gcnt, K, dg, glist, gcount);
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
void launch_bbox(int n, int ncol, const double* x, const double* y, const double* z,
                 const double* radius, const int32_t* colid, unsigned long long* out,
                 cudaStream_t st) {
  k_bbox_init<<<(7 * ncol + 255) / 256, 256, 0, st>>>(ncol, out);
  k_bbox<<<(n + 255) / 256, 256, 0, st>>>(n, x, y, z, radius, colid, out);
}
void launch_keys(int n, const double* x, const double* y, const double* z, const int32_t* colid,
                 const GridCol* grids, int64_t ncell, uint32_t* key, uint32_t* count,
                 cudaStream_t st, const int* search) {
  k_keys<<<(n + 255) / 256, 256, 0, st>>>(n, x, y, z, colid, grids, (uint32_t)ncell, key, count,
                                          search);
}
void launch_scatter(int n, const uint32_t* key, const uint32_t* start, uint32_t* fill,
                    int32_t* tmp, cudaStream_t st, const int* search) {
  k_scatter<<<(n + 255) / 256, 256, 0, st>>>(n, key, start, fill, tmp, search);
}
void launch_cell_sort(int64_t ncell, const uint32_t* start, int32_t* tmp, const int32_t* ids,
                      cudaStream_t st, const int* search) {
  k_cell_sort<<<(unsigned)((ncell + 255) / 256), 256, 0, st>>>(ncell, start, tmp, ids, search);
}
void launch_gather(int n, const int32_t* tmp, const double* const* src, double* const* dst,
                   int nsrc, const int32_t* ids_in, int32_t* ids_out, const int32_t* col_in,
                   int32_t* col_out, const GridCol* grids, float4* pf, cudaStream_t st,
                   const int32_t* iota, const int* search) {
  k_gather<<<(n + 255) / 256, 256, 0, st>>>(n, tmp, src, dst, nsrc, ids_in, ids_out, col_in,
                                            col_out, grids, pf, iota, search);
}
// keep: 0 every neighbour (overflow past cap), 1 the cap nearest, 2 the first
// cap of the octant-balanced ordering
void launch_neighbors(int keep, int n, const double* x, const double* y, const double* z,
                      const float4* pf, const int32_t* colid, const int32_t* ids,
                      const GridCol* grids, const uint32_t* start, const double* radius,
                      double r_const, int mirror_mode, double floor_z, int cap, int32_t* nbr,
                      int32_t* cnt, DevDiag* dg, cudaStream_t st, int bs, const int* search,
                      double* xref, bool periodic, VerletSkip vs) {
  const int nb = (n + bs - 1) / bs;
  if (keep)  // (stencils for callers: never periodic)
    k_neighbors<true, false><<<nb, bs, 0, st>>>(n, x, y, z, pf, colid, ids, grids, start, radius,
                                                 r_const, mirror_mode, floor_z, cap, nbr, cnt, dg,
                                                 search, xref, keep, vs);
  else if (periodic)
    k_neighbors<false, true><<<nb, bs, 0, st>>>(n, x, y, z, pf, colid, ids, grids, start, radius,
                                                 r_const, mirror_mode, floor_z, cap, nbr, cnt, dg,
                                                 search, xref, 0, vs);
  else
    k_neighbors<false, false><<<nb, bs, 0, st>>>(n, x, y, z, pf, colid, ids, grids, start,
                                                  radius, r_const, mirror_mode, floor_z, cap, nbr,
                                                  cnt, dg, search, xref, 0, vs);
}
void launch_filter(int n, const double* x, const double* y, const double* z, const float4* pf,
                   const int32_t* cand, const int32_t* ccnt, int capc, const GridCol* grids,
                   const int32_t* colid, double r, double floor_z, int cap, int32_t* nbr,
                   int32_t* cnt, DevDiag* dg, int* search, cudaStream_t st, int bs,
                   bool periodic, VerletSkip vs) {
  const int nb = (n + bs - 1) / bs;
  const bool track = vs.marg != nullptr;
  if (periodic && track)
    k_filter<true, true><<<nb, bs, 0, st>>>(n, x, y, z, pf, cand, ccnt, capc, grids, colid, r,
                                            floor_z, cap, nbr, cnt, dg, search, vs);
  else if (periodic)
    k_filter<true, false><<<nb, bs, 0, st>>>(n, x, y, z, pf, cand, ccnt, capc, grids, colid, r,
                                             floor_z, cap, nbr, cnt, dg, search, vs);
  else if (track)
    k_filter<false, true><<<nb, bs, 0, st>>>(n, x, y, z, pf, cand, ccnt, capc, grids, colid, r,
                                             floor_z, cap, nbr, cnt, dg, search, vs);
  else
    k_filter<false, false><<<nb, bs, 0, st>>>(n, x, y, z, pf, cand, ccnt, capc, grids, colid, r,
                                              floor_z, cap, nbr, cnt, dg, search, vs);
}
void launch_ghosts(int n, const double* x, const double* y, const double* z,
                   const int32_t* colid, const GridCol* grids, int4* X, int32_t* nbr,
                   const int32_t* cnt, int32_t* gcnt, const StepConsts& K, DevDiag* dg,
                   cudaStream_t st, int bs, int32_t* glist, int* gcount, int32_t* olist) {
  k_ghost_fix<<<(n + 255) / 256, 256, 0, st>>>(n, x, y, z, colid, grids, K.ghost_grid, K.floor_z,
                                               X, gcount);
  k_ghost_scan<<<(n + bs - 1) / bs, bs, 0, st>>>(n, X, nbr, cnt, gcnt, K, olist, gcount);
  k_ghosts<<<kGhostBlocks, 128, 0, st>>>(n, z, X, nbr, cnt, gcnt, K, dg, glist, gcount, olist);
}
void launch_nbr_to_caller(int n, int cap, const int32_t* ids, const int32_t* nbr_s,
                          const int32_t* cnt_s, int32_t* nbr_o, int32_t* cnt_o, cudaStream_t st) {
  k_nbr_to_caller<<<(n + 255) / 256, 256, 0, st>>>(n, cap, ids, nbr_s, cnt_s, nbr_o, cnt_o);
}

}  // namespace lp
