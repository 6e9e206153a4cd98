// C ABI of the LP step library: context, workspace, argument checks and the
// host-side orchestration of the kernels in neighbors.cu and fit.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lp_internal.cuh"

namespace lp {
// neighbors.cu
void launch_fill_colid(int n, const int32_t* offs, int ncol, int32_t* colid, cudaStream_t st);
void launch_bbox(int n, int ncol, const double* x, const double* y, const double* z,
                 const double* radius, const int32_t* colid, unsigned long long* out,
                 cudaStream_t st);
void launch_keys(int n, const double* x, const double* y, const double* z, const int32_t* colid,
                 const GridCol* grids, int64_t ncell, uint32_t* key, uint32_t* count,
                 cudaStream_t st, const int* search = nullptr);
void exclusive_scan(const uint32_t* in, uint32_t* out, uint32_t* tile_sum, int64_t n,
                    cudaStream_t st);
int64_t scan_tiles(int64_t n);
void launch_scatter(int n, const uint32_t* key, const uint32_t* start, uint32_t* fill,
                    int32_t* tmp, cudaStream_t st, const int* search = nullptr);
void launch_cell_sort(int64_t ncell, const uint32_t* start, int32_t* tmp, const int32_t* ids,
                      cudaStream_t st, const int* search = nullptr);
void launch_gather(int n, const int32_t* tmp, const double* const* src, double* const* dst,
                   int nsrc, const int32_t* ids_in, int32_t* ids_out, const int32_t* col_in,
                   int32_t* col_out, const GridCol* grids, float4* pf, cudaStream_t st,
                   const int32_t* iota = nullptr, const int* search = nullptr);
void launch_neighbors(int keep, int n, const double* x, const double* y, const double* z,
                      const float4* pf, const int32_t* colid, const int32_t* ids,
                      const GridCol* grids, const uint32_t* start, const double* radius,
                      double r_const, int mirror_mode, double floor_z, int cap, int32_t* nbr,
                      int32_t* cnt, DevDiag* dg, cudaStream_t st, int bs = kBlock,
                      const int* search = nullptr, double* xref = nullptr,
                      bool periodic = false, VerletSkip vs = VerletSkip{});
void launch_filter(int n, const double* x, const double* y, const double* z, const float4* pf,
                   const int32_t* cand, const int32_t* ccnt, int capc, const GridCol* grids,
                   const int32_t* colid, double r, double floor_z, int cap, int32_t* nbr,
                   int32_t* cnt, DevDiag* dg, int* search, cudaStream_t st, int bs,
                   bool periodic = false, VerletSkip vs = VerletSkip{});
void launch_ghosts(int n, const double* x, const double* y, const double* z,
                   const int32_t* colid, const GridCol* grids, int4* X, int32_t* nbr,
                   const int32_t* cnt, int32_t* gcnt, const StepConsts& K, DevDiag* dg,
                   cudaStream_t st, int bs, int32_t* glist, int* gcount, int32_t* olist);
void launch_copy_state(int n, double* const* dst, double* const* src, cudaStream_t st);
void launch_heun_combine(int n, double* const* y, double* const* y0, double Lx, double Ly,
                         cudaStream_t st);
void launch_wrap_positions(int n, double* x, double* y, double Lx, double Ly, cudaStream_t st);
void launch_axpby(int64_t n, double a, const double* x, double b, double* y, cudaStream_t st);
void launch_need_search(int n, const double* x, const double* y, const double* z,
                        const double* xref, double half_skin2, double Lx, double Ly, int* flag,
                        VerletSkip vs, cudaStream_t st);
void launch_nbr_to_caller(int n, int cap, const int32_t* ids, const int32_t* nbr_s,
                          const int32_t* cnt_s, int32_t* nbr_o, int32_t* cnt_o, cudaStream_t st);
// fit.cu
void launch_pass1(int prec, const StepArgs& A, cudaStream_t st, int bs = kBlock);
void launch_pass2(int prec, const StepArgs& A, cudaStream_t st, int bs = kBlock);
void launch_fit(int prec, const FitArgs& F, cudaStream_t st);
void launch_mui_stress(int64_t n, const ColMui& m, const lp_eos& e, const double* V,
                       const double* gu, double* gdot, double* gnorm, double* P, double* eta,
                       int8_t* regime, cudaStream_t st);
// adjoint.cu
void launch_adjoint_step(const AdjArgs& A, cudaStream_t st);
void launch_gather_fields(int n, const int32_t* idx, const double* const* src, double* const* dst,
                          int nf, cudaStream_t st);
// persistent.cu
cudaError_t launch_persistent(int prec, const PersistArgs& P, cudaStream_t st);
int64_t persistent_scan_tiles(int64_t len);
// misc.cu
void launch_iota(int n, int32_t* a, cudaStream_t st);
void launch_scatter_state(int n, const int32_t* ids, const double* const* src,
                          double* const* dst, int nf, cudaStream_t st);
}  // namespace lp

using namespace lp;

// gather tables: [direction][kind][field]; kind 0 = step state
// (x,y,z,u,v,w,V), kind 1 = search (x,y,z,radius)
enum { kTabFields = 8 };

struct lp_ctx {
  int device = 0;
  int64_t cap_n = 0;
  int cap_cols = 0;
  int cap = 0;
  double* X[2][kTabFields] = {};  // state fields 0..6 and radius (7)
  int32_t* ids[2] = {};
  int32_t* colid[2] = {};
  float4* pf = nullptr;
  uint32_t* key = nullptr;
  int32_t* tmp = nullptr;
  int32_t* nbr = nullptr;
  int32_t* cnt = nullptr;
  int32_t* nbr_o = nullptr;
  int32_t* cnt_o = nullptr;
  double* p1 = nullptr;
  double* fac = nullptr;
  float* facf = nullptr;
  int32_t* fbslot = nullptr;
  int32_t* fb_list = nullptr;
  int32_t* fb_count = nullptr;
  double* fbgrad = nullptr;
  int fb_cap = 0;
  uint32_t* cells = nullptr;  // count | fill | start, cell_capacity entries each
  uint32_t* tile = nullptr;
  int64_t cell_capacity = 0;
  GridCol* d_grids = nullptr;
  ColMui* d_mui = nullptr;
  int32_t* d_offs = nullptr;
  double* d_bbox = nullptr;
  double* h_bbox = nullptr;
  DevDiag* dg = nullptr;
  DevDiag* h_dg = nullptr;
  double** d_tab = nullptr;  // [2 dir][2 kind][2 src/dst][8]
  // Verlet lists kept across lp_step calls (lp_params.keep_lists): the
  // candidate lists, their reference positions and the sorted order of the
  // last call stay valid for the same particle count, columns and search
  // parameters until another entry point uses the context
  bool lists_valid = false;
  bool marg_valid = false;   // with lists_valid: the filter margins (vmarg) still hold
  int64_t lists_n = 0;
  std::vector<int32_t> lists_offs;
  double lists_sig[6] = {};
  double** d_ptr = nullptr;  // caller pointers for the final scatter
  double** h_ptr = nullptr;  // pinned staging of d_ptr
  unsigned* bar = nullptr;   // grid barrier of the persistent kernel
  FF8* XU = nullptr;  // split positions and velocities (LP_MIXED_FF)
  float2* P1s = nullptr;  // float-float gdot and ld of pass 1 (LP_MIXED_FF)
  float2* R1 = nullptr;   // float-float right-hand sides of pass 1 (LP_MIXED_FF)
  float2* fit_fs = nullptr;  // split fields of lp_fit_derivatives (LP_MIXED_FF), lazily
  int4* Xfix = nullptr;       // fixed-point positions of the free-surface test
  int32_t* gcnt = nullptr;    // ghost entries per stencil
  int32_t* glist = nullptr;   // particles with ghost entries (compact, any order)
  int32_t* olist = nullptr;   // particles with one-sided stencils (compact, any order)
  int* gcount = nullptr;      // the two lists' lengths
  int32_t* perm = nullptr;    // fit thread -> particle (LP_MIXED_FF)
  float *Tg = nullptr, *T2 = nullptr;  // twin sums (allocated on first free-surface step)
  double* Y0[7] = {};                  // Heun: state at the start of the step (on first use)
  double* stage = nullptr;             // lp_step on host arrays: 7 x cap_n (on first use)
  float2* Lff = nullptr;     // float-float Cholesky factors (LP_MIXED_FF), (hi, lo) pairs
  unsigned long long* phase_ns = nullptr;  // persistent-launch phase times (profiling)
  // Verlet candidate lists (lp_params.skin)
  int32_t* cand = nullptr;   // capc x n, k-major
  int32_t* ccnt = nullptr;
  int capc = 0;
  double* xref = nullptr;    // positions at the last search, 3 x n
  float* vmarg = nullptr;    // filter skipping (VerletSkip): margins, n
  float* vdmax = nullptr;    // running maximum displacements since the search, n
  unsigned* vdall = nullptr; // their maximum
  int* d_search = nullptr;   // device flag: search at the next step
  int32_t* iota = nullptr;   // 0..n-1 (identity gather)
  double skin = 0.0;         // skin of the current lp_step call (0: off)
  int cx = 0, ci = 0;
  int64_t ncell = 0;
  std::vector<GridCol> h_grids;
  std::vector<void*> allocs;
  // profiling: event pairs per phase, launch and step counters
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<int> ev_phase;  // phase of each recorded pair
  int64_t launches = 0;
  int64_t steps = 0;
  // bounded waits of the persistent kernel (lp_ctx_set_wait_limit)
  unsigned long long max_spins = 1ull << 25;
  unsigned extra_arrivals = 0;
  // device memory lp_step_adjoint may keep for whole-run data (< 0: half of
  // the free memory; 0: always recompute from checkpoints)
  int64_t adj_keep_bytes = -1;
  // launch configuration (lp_ctx_set_tuning / lp_autotune)
  int bs_nbr = kBlock, bs_p1 = kBlock, bs_p2 = kBlock;
};

namespace {

const char* kVersion = "lp-gb300 0.1 (sm_103a)";

template <typename T>
lp_status dalloc(lp_ctx* c, T** p, size_t count) {
  void* q = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return LP_ERR_OOM;
  }
  c->allocs.push_back(q);
  *p = (T*)q;
  return LP_OK;
}

lp_status cuda_status() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

#define LP_TRY(expr)                 \
  do {                               \
    lp_status _s = (expr);           \
    if (_s != LP_OK) return _s;      \
  } while (0)

lp_status reset_diag(lp_ctx* c, cudaStream_t st) {
  DevDiag z{};
  z.min_stencil = INT32_MAX;
  *c->h_dg = z;
  if (cudaMemcpyAsync(c->dg, c->h_dg, sizeof(DevDiag), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return LP_ERR_CUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

lp_status ensure_cells(lp_ctx* c, int64_t ncell) {
  if (ncell + 2 <= c->cell_capacity) return LP_OK;
  int64_t want = std::max<int64_t>(ncell + 2, c->cell_capacity * 2);
  if (c->cells) {
    cudaFree(c->cells);
    cudaFree(c->tile);
    c->allocs.erase(std::remove(c->allocs.begin(), c->allocs.end(), (void*)c->cells), c->allocs.end());
    c->allocs.erase(std::remove(c->allocs.begin(), c->allocs.end(), (void*)c->tile), c->allocs.end());
    c->cells = nullptr;
    c->tile = nullptr;
  }
  LP_TRY(dalloc(c, &c->cells, (size_t)want * 3));
  LP_TRY(dalloc(c, &c->tile,
                (size_t)std::max(scan_tiles(want), persistent_scan_tiles(want)) + 1));
  c->cell_capacity = want;
  return LP_OK;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// Per-column grids from the bounding boxes (host), uploaded to the device.
// A periodic axis (period Lx or Ly > 0) has whole cells over [0, L), at least
// three, each at least rmax wide.
lp_status setup_grids(lp_ctx* c, int ncol, double rmax, cudaStream_t st, double Lx = 0.0,
                      double Ly = 0.0) {
  const int margin = 4;
  const double base = rmax * (1.0 + 0x1p-20);
  const int64_t budget = std::max<int64_t>(4 * c->cap_n, (int64_t)1 << 20);
  c->h_grids.resize(ncol);
  int64_t total = 0;
  double cell = base;
  for (int attempt = 0; attempt < 64; ++attempt) {
    total = 0;
    for (int k = 0; k < ncol; ++k) {
      const double* b = c->h_bbox + 7 * k;
      GridCol g{};
      double lo[3], ext[3];
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::isfinite(b[a]) ? b[a] : 0.0;
        ext[a] = (std::isfinite(b[a]) && std::isfinite(b[3 + a])) ? b[3 + a] - b[a] : 0.0;
      }
      int dims[3];
      double org[3], edge[3];
      const double per[3] = {Lx, Ly, 0.0};
      for (int a = 0; a < 3; ++a) {
        if (per[a] > 0.0) {
          dims[a] = (int)std::min(1024.0, std::max(3.0, std::floor(per[a] / cell)));
          org[a] = 0.0;
          edge[a] = per[a] / dims[a];
          if (!(edge[a] >= base)) return LP_ERR_INVALID_ARG;  // period below 3 rmax
          continue;
        }
        double d = std::floor(ext[a] / cell) + 1 + 2 * margin;
        dims[a] = (int)std::min(1024.0, std::max(1.0, d));
        org[a] = lo[a] - margin * cell;
        edge[a] = cell;
      }
      g.ox = org[0]; g.oy = org[1]; g.oz = org[2];
      g.icx = 1.0 / edge[0]; g.icy = 1.0 / edge[1]; g.icz = 1.0 / edge[2];
      g.Lx = Lx; g.Ly = Ly;
      g.Lxf = (float)Lx; g.Lyf = (float)Ly;
      g.nx = dims[0]; g.ny = dims[1]; g.nz = dims[2];
      g.cell_off = total;
      total += (int64_t)dims[0] * dims[1] * dims[2];
      c->h_grids[k] = g;
    }
    if (total <= budget) break;
    cell *= 1.25;  // coarser cells keep the grid within budget (still >= rmax)
  }
  if (total > ((int64_t)1 << 31) - 2) return LP_ERR_INVALID_ARG;
  LP_TRY(ensure_cells(c, total));
  c->ncell = total;
  if (cudaMemcpyAsync(c->d_grids, c->h_grids.data(), sizeof(GridCol) * ncol,
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return LP_ERR_CUDA;
  return LP_OK;
}

// True if every column's bounding box (h_bbox) lies inside its current grid
// with at least one cell to spare on each non-periodic side.
bool grids_cover(const lp_ctx* c, int ncol) {
  if ((int)c->h_grids.size() < ncol) return false;
  for (int k = 0; k < ncol; ++k) {
    const GridCol& g = c->h_grids[k];
    const double* b = c->h_bbox + 7 * k;
    const double org[3] = {g.ox, g.oy, g.oz}, ic[3] = {g.icx, g.icy, g.icz};
    const int dims[3] = {g.nx, g.ny, g.nz};
    const double per[3] = {g.Lx, g.Ly, 0.0};
    for (int a = 0; a < 3; ++a) {
      if (per[a] > 0.0) continue;
      if (!(b[a] <= b[3 + a])) continue;  // empty column
      const double lo = (b[a] - org[a]) * ic[a], hi = (b[3 + a] - org[a]) * ic[a];
      if (!(lo >= 1.0 && hi <= dims[a] - 1.0)) return false;
    }
  }
  return true;
}

// Upload offsets and column ids; compute the bounding boxes (synchronises).
// (fill_colid false: the slots keep the column ids of the previous call)
lp_status begin_columns(lp_ctx* c, const lp_particles* p, const double* radius_dev, int buf,
                        std::vector<int32_t>& offs, cudaStream_t st, bool fill_colid = true) {
  const int ncol = p->ncolumns;
  if (cudaMemcpyAsync(c->d_offs, offs.data(), sizeof(int32_t) * (ncol + 1), cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
    return LP_ERR_CUDA;
  if (fill_colid) launch_fill_colid((int)p->n, c->d_offs, ncol, c->colid[c->ci], st);
  launch_bbox((int)p->n, ncol, c->X[buf][0], c->X[buf][1], c->X[buf][2], radius_dev,
              c->colid[c->ci], (unsigned long long*)c->d_bbox, st);
  if (cudaMemcpyAsync(c->h_bbox, c->d_bbox, sizeof(double) * 7 * ncol, cudaMemcpyDeviceToHost,
                      st) != cudaSuccess)
    return LP_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return LP_ERR_CUDA;
  // decode the order-preserving keys; empty columns keep +-inf
  for (int k = 0; k < 7 * ncol; ++k) {
    unsigned long long u;
    std::memcpy(&u, &c->h_bbox[k], 8);
    const bool empty = (k % 7) < 3 ? u == ~0ull : u == 0ull;
    if (empty) {
      c->h_bbox[k] = (k % 7) < 3 ? INFINITY : ((k % 7) == 6 ? 0.0 : -INFINITY);
      continue;
    }
    const unsigned long long b = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
    std::memcpy(&c->h_bbox[k], &b, 8);
  }
  return cuda_status();
}

lp_status check_particles(const lp_ctx* c, const lp_particles* p, std::vector<int32_t>& offs,
                          bool need_state) {
  if (!p || p->n < 0 || p->n > c->cap_n || p->ncolumns < 1 || p->ncolumns > c->cap_cols)
    return LP_ERR_INVALID_ARG;
  if (p->n > 0 && (!p->x || !p->y || !p->z)) return LP_ERR_INVALID_ARG;
  if (p->n > 0 && need_state && (!p->u || !p->v || !p->w || !p->V)) return LP_ERR_INVALID_ARG;
  offs.assign(p->ncolumns + 1, 0);
  if (p->column_offsets) {
    for (int k = 0; k <= p->ncolumns; ++k) offs[k] = p->column_offsets[k];
    if (offs[0] != 0 || offs[p->ncolumns] != p->n) return LP_ERR_INVALID_ARG;
    for (int k = 0; k < p->ncolumns; ++k)
      if (offs[k + 1] < offs[k]) return LP_ERR_INVALID_ARG;
  } else {
    if (p->ncolumns != 1) return LP_ERR_INVALID_ARG;
    offs[1] = (int32_t)p->n;
  }
  return LP_OK;
}

// Record the start or end event of a phase (profiling only).
void phase_mark(lp_ctx* c, int phase, bool start, cudaStream_t st) {
  if (!c->profile) return;
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->ev_pool.push_back(e);
  }
  cudaEventRecord(c->ev_pool[c->ev_used++], st);
  if (start) c->ev_phase.push_back(phase);
}

// Counting sort by cell (stable by original index) from buffer c->cx into
// the other buffer; nsrc fields of table `kind`.
void sort_particles(lp_ctx* c, int n, int kind, int nsrc, cudaStream_t st,
                    const int* search = nullptr) {
  const int d = c->cx;
  uint32_t* count = c->cells;
  uint32_t* fill = c->cells + c->cell_capacity;
  uint32_t* start = c->cells + 2 * c->cell_capacity;
  cudaMemsetAsync(c->cells, 0, sizeof(uint32_t) * 2 * c->cell_capacity, st);
  launch_keys(n, c->X[d][0], c->X[d][1], c->X[d][2], c->colid[c->ci], c->d_grids, c->ncell,
              c->key, count, st, search);
  // cells 0..ncell-1, the bucket of non-finite particles (ncell), the total
  exclusive_scan(count, start, c->tile, c->ncell + 2, st);
  launch_scatter(n, c->key, start, fill, c->tmp, st, search);
  launch_cell_sort(c->ncell, start, c->tmp, c->ids[c->ci], st, search);
  const double* const* src = (const double* const*)(c->d_tab + ((d * 2 + kind) * 2 + 0) * kTabFields);
  double* const* dst = c->d_tab + ((d * 2 + kind) * 2 + 1) * kTabFields;
  launch_gather(n, c->tmp, src, dst, nsrc, c->ids[c->ci], c->ids[1 - c->ci], c->colid[c->ci],
                c->colid[1 - c->ci], c->d_grids, c->pf, st, c->iota, search);
  c->cx ^= 1;
  c->ci ^= 1;
  c->launches += 7;
}

// Filter skipping between searches (VerletSkip); off with free-surface ghosts,
// whose kernel rewrites the stencils after the filter
VerletSkip verlet_skip(lp_ctx* c, const StepConsts& K) {
  if (K.free_surface || !c->vmarg) return VerletSkip{};
  return VerletSkip{c->vmarg, c->vdmax, c->vdall};
}

StepArgs step_args(lp_ctx* c, int n, const StepConsts& K) {
  StepArgs A{};
  A.n = n;
  A.cap = c->cap;
  const int d = c->cx;
  A.x = c->X[d][0]; A.y = c->X[d][1]; A.z = c->X[d][2];
  A.u = c->X[d][3]; A.v = c->X[d][4]; A.w = c->X[d][5]; A.V = c->X[d][6];
  A.xo = c->X[1 - d][0]; A.yo = c->X[1 - d][1]; A.zo = c->X[1 - d][2];
  A.uo = c->X[1 - d][3]; A.vo = c->X[1 - d][4]; A.wo = c->X[1 - d][5]; A.Vo = c->X[1 - d][6];
  A.nbr = c->nbr; A.cnt = c->cnt; A.colid = c->colid[c->ci];
  A.mui = c->d_mui;
  A.fac = c->fac; A.facf = c->facf;
  A.fbslot = c->fbslot; A.fb_list = c->fb_list; A.fb_count = c->fb_count; A.fb_cap = c->fb_cap;
  A.p1 = c->p1; A.fbgrad = c->fbgrad; A.dg = c->dg;
  A.K = K;
  A.grids = c->d_grids;
  A.XU = c->XU; A.Lff = c->Lff; A.P1s = c->P1s; A.R1 = c->R1;
  A.perm = LP_ROW_ORDER ? c->perm : nullptr;
  A.Xfix = c->Xfix;
  A.gcnt = c->gcnt;
  A.glist = c->glist; A.gcount = c->gcount;
  A.Tg = c->Tg; A.T2 = c->T2;
  if (c->skin > 0.0) {
    A.xref = c->xref;
    const double hs = 0.5 * c->skin;
    A.half_skin2 = hs * hs * (1.0 - 0x1p-20);
    A.need_search = c->d_search;
    A.vskip = verlet_skip(c, K);
  }
  return A;
}

// Twin sums of the float-float free-surface path (62 + 36 floats per
// particle) and the saved state of Heun's method (7 doubles per particle),
// allocated on first use.
lp_status ensure_twin_buffers(lp_ctx* c, const lp_params* q) {
  if (q->time_scheme == LP_TIME_HEUN && !c->Y0[0])
    for (int f = 0; f < 7; ++f) LP_TRY(dalloc(c, &c->Y0[f], (size_t)c->cap_n));
  if (!q->free_surface || c->Tg) return LP_OK;
  LP_TRY(dalloc(c, &c->Tg, (size_t)c->cap_n * 62));
  return dalloc(c, &c->T2, (size_t)c->cap_n * 36);
}

// One LP step on the context's internal (sorted) state.
// save_y0: copy the (sorted) state to c->Y0 once the stencils are built
// (first stage of Heun's method).
void run_step(lp_ctx* c, int n, const StepConsts& K, int prec, bool rebuild, cudaStream_t st,
              bool save_y0 = false) {
  if (rebuild && c->skin > 0.0) {
    // Verlet candidate lists: search (radius + skin) only when flagged, then
    // the exact filter every step
    phase_mark(c, LP_PHASE_SORT, true, st);
    sort_particles(c, n, 0, 7, st, c->d_search);
    phase_mark(c, LP_PHASE_SORT, false, st);
    phase_mark(c, LP_PHASE_NEIGHBORS, true, st);
    const int e = c->cx;
    launch_neighbors(false, n, c->X[e][0], c->X[e][1], c->X[e][2], c->pf, c->colid[c->ci],
                     c->ids[c->ci], c->d_grids, c->cells + 2 * c->cell_capacity, nullptr,
                     K.radius + c->skin, K.mirror_mode, K.floor_z, c->capc, c->cand, c->ccnt,
                     c->dg, st, c->bs_nbr, c->d_search, c->xref, K.periodic != 0,
                     verlet_skip(c, K));
    launch_filter(n, c->X[e][0], c->X[e][1], c->X[e][2], c->pf, c->cand, c->ccnt, c->capc,
                  c->d_grids, c->colid[c->ci], K.radius, K.floor_z, c->cap, c->nbr, c->cnt,
                  c->dg, c->d_search, st, c->bs_nbr, K.periodic != 0, verlet_skip(c, K));
    if (K.free_surface) {
      launch_ghosts(n, c->X[e][0], c->X[e][1], c->X[e][2], c->colid[c->ci], c->d_grids, c->Xfix,
                    c->nbr, c->cnt, c->gcnt, K, c->dg, st, c->bs_nbr, c->glist, c->gcount, c->olist);
      c->launches += 3;
    }
    phase_mark(c, LP_PHASE_NEIGHBORS, false, st);
    c->launches += 2;
  } else if (rebuild) {
    phase_mark(c, LP_PHASE_SORT, true, st);
    sort_particles(c, n, 0, 7, st);
    phase_mark(c, LP_PHASE_SORT, false, st);
    phase_mark(c, LP_PHASE_NEIGHBORS, true, st);
    launch_neighbors(false, n, c->X[c->cx][0], c->X[c->cx][1], c->X[c->cx][2], c->pf,
                     c->colid[c->ci], c->ids[c->ci], c->d_grids, c->cells + 2 * c->cell_capacity,
                     nullptr, K.radius, K.mirror_mode, K.floor_z, c->cap, c->nbr, c->cnt, c->dg,
                     st, c->bs_nbr, nullptr, nullptr, K.periodic != 0);
    if (K.free_surface) {
      launch_ghosts(n, c->X[c->cx][0], c->X[c->cx][1], c->X[c->cx][2], c->colid[c->ci],
                    c->d_grids, c->Xfix, c->nbr, c->cnt, c->gcnt, K, c->dg, st, c->bs_nbr,
                    c->glist, c->gcount, c->olist);
      c->launches += 3;
    }
    phase_mark(c, LP_PHASE_NEIGHBORS, false, st);
    c->launches += 1;
  }
  if (save_y0) {
    launch_copy_state(n, c->Y0, c->X[c->cx], st);
    c->launches += 1;
  }
  cudaMemsetAsync(c->fb_count, 0, sizeof(int32_t), st);
  StepArgs A = step_args(c, n, K);
  phase_mark(c, LP_PHASE_PASS1, true, st);
  launch_pass1(prec, A, st, c->bs_p1);
  phase_mark(c, LP_PHASE_PASS1, false, st);
  phase_mark(c, LP_PHASE_PASS2, true, st);
  launch_pass2(prec, A, st, c->bs_p2);
  phase_mark(c, LP_PHASE_PASS2, false, st);
  c->launches += prec == LP_MIXED_FF ? (K.free_surface ? 9 : 7) + (A.perm ? 1 : 0) : 4;
  c->steps += 1;
  c->cx ^= 1;
}

// One step of the chosen time scheme: the paper's step, or Heun's method as
// two stages on the step's stencils and the average y <- (y0 + y**) / 2.
void one_step(lp_ctx* c, int n, const StepConsts& K, int prec, bool rebuild, cudaStream_t st) {
  if (!K.euler) {
    run_step(c, n, K, prec, rebuild, st);
    return;
  }
  run_step(c, n, K, prec, rebuild, st, true);
  run_step(c, n, K, prec, false, st);
  launch_heun_combine(n, c->X[c->cx], c->Y0, K.Lx, K.Ly, st);
  c->launches += 1;
  c->steps -= 1;  // two stages, one step
}

// One LP step as a single persistent cooperative launch (same buffers and
// toggles as run_step).
lp_status run_step_persistent(lp_ctx* c, int n, const StepConsts& K, int prec, bool rebuild,
                              cudaStream_t st, bool save_y0 = false) {
  PersistArgs P{};
  P.n = n;
  if (save_y0) {
    for (int f = 0; f < 7; ++f) P.y0[f] = c->Y0[f];
    P.save_y0 = 1;
  }
  P.rebuild = rebuild ? 1 : 0;
  P.ncell = c->ncell;
  const int d = c->cx;
  if (rebuild) {
    P.xs = c->X[d][0]; P.ys = c->X[d][1]; P.zs = c->X[d][2];
    P.colid_in = c->colid[c->ci]; P.ids_in = c->ids[c->ci];
    P.colid_out = c->colid[1 - c->ci]; P.ids_out = c->ids[1 - c->ci];
    P.grids = c->d_grids;
    P.key = c->key;
    P.count = c->cells;
    P.fill = c->cells + c->cell_capacity;
    P.start = c->cells + 2 * c->cell_capacity;
    P.tile = c->tile;
    P.ntiles = (int)persistent_scan_tiles(c->ncell + 2);
    P.tmp = c->tmp;
    P.src = (const double* const*)(c->d_tab + ((d * 2 + 0) * 2 + 0) * kTabFields);
    P.dst = c->d_tab + ((d * 2 + 0) * 2 + 1) * kTabFields;
    P.nsrc = 7;
    P.pf = c->pf;
    P.radius = K.radius; P.floor_z = K.floor_z; P.mirror_mode = K.mirror_mode; P.cap = c->cap;
    P.nbr = c->nbr; P.cnt = c->cnt;
    if (c->skin > 0.0) {
      P.search = c->d_search;
      P.iota = c->iota;
      P.cand = c->cand; P.ccnt = c->ccnt; P.capc = c->capc;
      P.rsearch = K.radius + c->skin;
      P.xref = c->xref;
    }
    c->cx ^= 1;  // the gather fills the other buffer
    c->ci ^= 1;
  }
  P.S = step_args(c, n, K);
  P.bar = c->bar;
  P.max_spins = c->max_spins;  // default about 2 s of __nanosleep(64)
  P.extra_arrivals = c->extra_arrivals;
  if (c->profile) {
    if (!c->phase_ns) {
      LP_TRY(dalloc(c, &c->phase_ns, (size_t)LP_NPHASES + 1));
      cudaMemsetAsync(c->phase_ns, 0, sizeof(unsigned long long) * (LP_NPHASES + 1), st);
    }
    P.phase_ns = c->phase_ns;
  }
  cudaMemsetAsync(c->bar, 0, 2 * sizeof(unsigned), st);
  if (launch_persistent(prec, P, st) != cudaSuccess) {
    cudaGetLastError();
    return LP_ERR_CUDA;
  }
  c->launches += 1;
  c->steps += 1;
  c->cx ^= 1;
  return LP_OK;
}

// nsteps steps on the internal state with the given launch mode (the loop of
// lp_step; also timed by lp_autotune).
lp_status run_steps(lp_ctx* c, int n, const StepConsts& K, int prec, int R, int launch_mode,
                    int nsteps, cudaStream_t st) {
  int done = 0;
  const int period = 2 * R;  // buffer toggles repeat after 2R steps
  if (launch_mode == LP_LAUNCH_PERSISTENT) {
    for (int k = 0; k < nsteps; ++k) {
      const lp_status r = run_step_persistent(c, n, K, prec, (k % R) == 0, st, K.euler);
      if (r != LP_OK) return r;
      if (K.euler) {  // Heun's method: second stage on the same stencils, average
        const lp_status r2 = run_step_persistent(c, n, K, prec, false, st);
        if (r2 != LP_OK) return r2;
        launch_heun_combine(n, c->X[c->cx], c->Y0, K.Lx, K.Ly, st);
        c->launches += 1;
        c->steps -= 1;
      }
    }
    done = nsteps;
  } else if (launch_mode == LP_LAUNCH_GRAPH && !c->profile && st != nullptr &&
             nsteps >= 2 * period) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return LP_ERR_CUDA;
    const int cx0 = c->cx, ci0 = c->ci;
    const int64_t launches0 = c->launches, steps0 = c->steps;
    c->launches = 0;
    c->steps = 0;
    for (int k = 0; k < period; ++k) one_step(c, n, K, prec, k % R == 0, st);
    if (cudaStreamEndCapture(st, &g) != cudaSuccess || c->cx != cx0 || c->ci != ci0) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return LP_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) {
      cudaGraphDestroy(g);
      cudaGetLastError();
      return LP_ERR_CUDA;
    }
    const int reps = nsteps / period;
    // the capture counted one period of launches and steps
    const int64_t per_launch = c->launches, per_steps = c->steps;
    for (int r = 0; r < reps; ++r) cudaGraphLaunch(ge, st);
    c->launches = launches0 + per_launch * reps;
    c->steps = steps0 + per_steps * reps;
    done = reps * period;
    cudaGraphExecDestroy(ge);
    cudaGraphDestroy(g);
  }
  for (int k = done; k < nsteps; ++k) one_step(c, n, K, prec, (k % R) == 0, st);
  return LP_OK;
}

bool valid_params(const lp_params* q, const lp_eos* e, double dt) {
  if (!q || !e) return false;
  if (!finite_pos(q->h) || !finite_pos(q->radius) || !std::isfinite(dt) || dt < 0) return false;
  if (q->mirror_mode < 0 || q->mirror_mode > 2) return false;
  if (q->precision != LP_FP64 && q->precision != LP_MIXED && q->precision != LP_MIXED_FF)
    return false;
  if (q->rebuild_every < 1) return false;
  if (q->launch_mode < LP_LAUNCH_KERNELS || q->launch_mode > LP_LAUNCH_PERSISTENT) return false;
  if (!(q->skin >= 0.0) || !std::isfinite(q->skin) || q->skin > q->radius) return false;
  if (q->free_surface != 0 && q->free_surface != 1) return false;
  if (q->time_scheme != LP_TIME_PAPER && q->time_scheme != LP_TIME_HEUN) return false;
  // periods: 0, or finite and at least three stencil radii (plus the skin);
  // the fixed-point ghost test needs K L < 2^30
  for (const double L : {q->period_x, q->period_y}) {
    if (L == 0.0) continue;
    if (!std::isfinite(L) || !(L >= 3.0 * (q->radius + q->skin) * (1.0 + 0x1p-16))) return false;
    if (q->free_surface && !(L * (8192.0 / q->radius) < 0x1p29)) return false;
  }
  if (!(e->phi_min < e->phi_max && e->phi_max < e->phi_c)) return false;
  return true;
}

}  // namespace

// ================================================================= C ABI

extern "C" {

const char* lp_version(void) { return kVersion; }

const char* lp_status_string(lp_status s) {
  switch (s) {
    case LP_OK: return "ok";
    case LP_ERR_INVALID_ARG: return "invalid argument";
    case LP_ERR_STENCIL_OVERFLOW: return "stencil overflow";
    case LP_ERR_NONFINITE: return "non-finite value";
    case LP_ERR_TIMEOUT: return "device wait timed out";
    case LP_ERR_CUDA: return "CUDA error";
    case LP_ERR_OOM: return "out of device memory";
    case LP_ERR_UNIMPLEMENTED: return "not implemented";
    default: return "unknown status";
  }
}

lp_status lp_ctx_create(const lp_ctx_desc* desc, lp_ctx** out) {
  if (!desc || !out || desc->max_particles < 1 || desc->max_particles > ((int64_t)1 << 30) ||
      desc->cap < 1 || desc->cap > LP_MAX_CAP || desc->max_columns < 1 ||
      desc->max_columns > kMaxColumns)
    return LP_ERR_INVALID_ARG;
  *out = nullptr;
  if (cudaSetDevice(desc->device) != cudaSuccess) {
    cudaGetLastError();
    return LP_ERR_CUDA;
  }
  lp_ctx* c = new lp_ctx();
  c->device = desc->device;
  c->cap_n = desc->max_particles;
  c->cap_cols = desc->max_columns;
  c->cap = desc->cap;
  const size_t n = (size_t)c->cap_n;
  lp_status s = LP_OK;
  for (int d = 0; d < 2 && s == LP_OK; ++d) {
    for (int f = 0; f < kTabFields && s == LP_OK; ++f) s = dalloc(c, &c->X[d][f], n);
    if (s == LP_OK) s = dalloc(c, &c->ids[d], n);
    if (s == LP_OK) s = dalloc(c, &c->colid[d], n);
  }
  c->fb_cap = (int)std::min<int64_t>(c->cap_n, 1 << 20);
  if (s == LP_OK) s = dalloc(c, &c->pf, n);
  if (s == LP_OK) s = dalloc(c, &c->key, n);
  if (s == LP_OK) s = dalloc(c, &c->tmp, n);
  if (s == LP_OK) s = dalloc(c, &c->nbr, n * c->cap);
  if (s == LP_OK) s = dalloc(c, &c->cnt, n);
  if (s == LP_OK) s = dalloc(c, &c->p1, n * P1_N);
  if (s == LP_OK) s = dalloc(c, &c->fac, n * kTri);
  if (s == LP_OK) s = dalloc(c, &c->facf, n * kTri);
  if (s == LP_OK) s = dalloc(c, &c->fbslot, n);
  if (s == LP_OK) s = dalloc(c, &c->fb_list, (size_t)c->fb_cap);
  if (s == LP_OK) s = dalloc(c, &c->fb_count, 1);
  if (s == LP_OK) s = dalloc(c, &c->fbgrad, (size_t)c->fb_cap * 6);
  if (s == LP_OK) s = dalloc(c, &c->d_grids, (size_t)c->cap_cols);
  if (s == LP_OK) s = dalloc(c, &c->d_mui, (size_t)c->cap_cols);
  if (s == LP_OK) s = dalloc(c, &c->d_offs, (size_t)c->cap_cols + 1);
  if (s == LP_OK) s = dalloc(c, &c->d_bbox, (size_t)c->cap_cols * 7);
  if (s == LP_OK) s = dalloc(c, &c->dg, 1);
  if (s == LP_OK) s = dalloc(c, &c->d_tab, 2 * 2 * 2 * kTabFields);
  if (s == LP_OK) s = dalloc(c, &c->d_ptr, kTabFields);
  if (s == LP_OK) s = dalloc(c, &c->bar, 2);
  if (s == LP_OK) s = dalloc(c, &c->XU, n);
  if (s == LP_OK) s = dalloc(c, &c->P1s, n * 9);
  if (s == LP_OK) s = dalloc(c, &c->R1, n * 27);
  if (s == LP_OK) s = dalloc(c, &c->Lff, n * kTri);
  if (s == LP_OK) s = dalloc(c, &c->Xfix, n);
  if (s == LP_OK) s = dalloc(c, &c->gcnt, n);
  if (s == LP_OK) s = dalloc(c, &c->glist, n);
  if (s == LP_OK) s = dalloc(c, &c->olist, n);
  if (s == LP_OK) s = dalloc(c, &c->gcount, 2);
  if (s == LP_OK) s = dalloc(c, &c->perm, n);
  c->capc = std::min(c->cap + 32, 96);
  if (s == LP_OK) s = dalloc(c, &c->cand, n * c->capc);
  if (s == LP_OK) s = dalloc(c, &c->ccnt, n);
  if (s == LP_OK) s = dalloc(c, &c->xref, 3 * n);
  if (s == LP_OK) s = dalloc(c, &c->vmarg, n);
  if (s == LP_OK) s = dalloc(c, &c->vdmax, n);
  if (s == LP_OK) s = dalloc(c, &c->vdall, 1);
  if (s == LP_OK) s = dalloc(c, &c->d_search, 1);
  if (s == LP_OK) s = dalloc(c, &c->iota, n);
  if (s == LP_OK) {
    // every index buffer starts valid: identity permutations, empty stencils
    launch_iota((int)n, c->iota, 0);
    launch_iota((int)n, c->ids[0], 0);
    launch_iota((int)n, c->ids[1], 0);
    launch_iota((int)n, c->tmp, 0);
    cudaMemset(c->colid[0], 0, n * sizeof(int32_t));
    cudaMemset(c->colid[1], 0, n * sizeof(int32_t));
    cudaMemset(c->cnt, 0, n * sizeof(int32_t));
    cudaMemset(c->nbr, 0, n * c->cap * sizeof(int32_t));
    cudaMemset(c->gcount, 0, 2 * sizeof(int));  // no particle with ghosts yet
    cudaMemset(c->ccnt, 0, n * sizeof(int32_t));
    cudaMemset(c->cand, 0, n * c->capc * sizeof(int32_t));
    cudaMemset(c->key, 0, n * sizeof(uint32_t));
    cudaMemset(c->fbslot, 0xff, n * sizeof(int32_t));
    if (cudaDeviceSynchronize() != cudaSuccess) s = LP_ERR_CUDA;
  }
  if (s == LP_OK && cudaMemset(c->bar, 0, 2 * sizeof(unsigned)) != cudaSuccess) s = LP_ERR_CUDA;
  if (s == LP_OK) s = ensure_cells(c, 1 << 16);
  if (s == LP_OK) {
    if (cudaMallocHost(&c->h_bbox, sizeof(double) * 7 * c->cap_cols) != cudaSuccess ||
        cudaMallocHost(&c->h_dg, sizeof(DevDiag)) != cudaSuccess ||
        cudaMallocHost(&c->h_ptr, sizeof(double*) * kTabFields) != cudaSuccess) {
      cudaGetLastError();
      s = LP_ERR_OOM;
    }
  }
  if (s == LP_OK) {
    // gather tables: kind 0 gathers the 7 state fields, kind 1 x, y, z, radius
    double* tab[2 * 2 * 2 * kTabFields] = {};
    const int order[2][kTabFields] = {{0, 1, 2, 3, 4, 5, 6, 7}, {0, 1, 2, 7, 3, 4, 5, 6}};
    for (int d = 0; d < 2; ++d)
      for (int kind = 0; kind < 2; ++kind)
        for (int f = 0; f < kTabFields; ++f) {
          tab[((d * 2 + kind) * 2 + 0) * kTabFields + f] = c->X[d][order[kind][f]];
          tab[((d * 2 + kind) * 2 + 1) * kTabFields + f] = c->X[1 - d][order[kind][f]];
        }
    if (cudaMemcpy(c->d_tab, tab, sizeof(tab), cudaMemcpyHostToDevice) != cudaSuccess) s = LP_ERR_CUDA;
  }
  if (s == LP_OK) s = reset_diag(c, 0);
  if (s != LP_OK) {
    lp_ctx_destroy(c);
    return s;
  }
  *out = c;
  return LP_OK;
}

lp_status lp_ctx_destroy(lp_ctx* c) {
  if (!c) return LP_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  for (void* p : c->allocs) cudaFree(p);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->h_bbox) cudaFreeHost(c->h_bbox);
  if (c->h_dg) cudaFreeHost(c->h_dg);
  if (c->h_ptr) cudaFreeHost(c->h_ptr);
  delete c;
  return cuda_status();
}

lp_status lp_ctx_sync(lp_ctx* c, void* stream, lp_diag* diag) {
  if (!c) return LP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(c->device);
  if (cudaMemcpyAsync(c->h_dg, c->dg, sizeof(DevDiag), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return LP_ERR_CUDA;
  }
  const DevDiag d = *c->h_dg;
  if (diag) {
    std::memset(diag, 0, sizeof(*diag));
    diag->flags = d.flags;
    diag->min_stencil = d.min_stencil == INT32_MAX ? 0 : d.min_stencil;
    diag->max_stencil = d.max_stencil;
    diag->n_overflow = (int64_t)d.n_overflow;
    diag->n_fallback = (int64_t)d.n_fallback;
    diag->n_gas = (int64_t)d.n_gas;
    diag->n_quasistatic = (int64_t)d.n_quasistatic;
    diag->n_over_c = (int64_t)d.n_over_c;
    diag->n_nonfinite = (int64_t)d.n_nonfinite;
    diag->n_below_floor = (int64_t)d.n_below_floor;
    diag->n_stencil_rows = (int64_t)d.n_stencil_rows;
    diag->n_stencils = (int64_t)d.n_stencils;
    diag->n_ghosts = (int64_t)d.n_ghosts;
  }
  LP_TRY(reset_diag(c, st));
  if (d.flags & LP_FLAG_TIMEOUT) return LP_ERR_TIMEOUT;
  if (d.flags & LP_FLAG_OVERFLOW) return LP_ERR_STENCIL_OVERFLOW;
  if (d.flags & LP_FLAG_NONFINITE) return LP_ERR_NONFINITE;
  return LP_OK;
}

lp_status lp_ctx_set_adjoint_memory(lp_ctx* c, int64_t max_bytes) {
  if (!c) return LP_ERR_INVALID_ARG;
  c->adj_keep_bytes = max_bytes < 0 ? -1 : max_bytes;
  return LP_OK;
}

lp_status lp_ctx_set_wait_limit(lp_ctx* c, int64_t max_spins, int32_t extra_arrivals) {
  if (!c || max_spins < 1 || extra_arrivals < 0 || extra_arrivals > 1024)
    return LP_ERR_INVALID_ARG;
  c->max_spins = (unsigned long long)max_spins;
  c->extra_arrivals = (unsigned)extra_arrivals;
  return LP_OK;
}

lp_status lp_ctx_profile(lp_ctx* c, int32_t enable) {
  if (!c) return LP_ERR_INVALID_ARG;
  c->profile = enable != 0;
  return LP_OK;
}

lp_status lp_ctx_phase_times(lp_ctx* c, void* stream, double* ms, int64_t* launches,
                             int64_t* steps) {
  if (!c || !ms) return LP_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return LP_ERR_CUDA;
  }
  for (int k = 0; k < LP_NPHASES; ++k) ms[k] = 0.0;
  for (size_t r = 0; r < c->ev_phase.size(); ++r) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, c->ev_pool[2 * r], c->ev_pool[2 * r + 1]) == cudaSuccess)
      ms[c->ev_phase[r]] += t;
  }
  cudaGetLastError();
  if (c->phase_ns) {  // phases of persistent launches (profiling)
    unsigned long long ns[LP_NPHASES];
    if (cudaMemcpy(ns, c->phase_ns, sizeof(ns), cudaMemcpyDeviceToHost) == cudaSuccess &&
        cudaMemset(c->phase_ns, 0, sizeof(ns)) == cudaSuccess) {
      for (int k = 0; k < LP_NPHASES; ++k) ms[k] += 1e-6 * (double)ns[k];
    }
    cudaGetLastError();
  }
  c->ev_phase.clear();
  c->ev_used = 0;
  if (launches) *launches = c->launches;
  if (steps) *steps = c->steps;
  c->launches = 0;
  c->steps = 0;
  return LP_OK;
}

lp_status lp_build_neighbors(lp_ctx* c, const lp_particles* p, const double* radius,
                             double r_const, int32_t mirror_mode, double floor_z, int32_t cap,
                             int32_t keep_nearest, lp_neighbors* out, void* stream) {
  if (!c || !out) return LP_ERR_INVALID_ARG;
  c->lists_valid = false;  // uses the buffers the kept Verlet lists live in
  std::vector<int32_t> offs;
  LP_TRY(check_particles(c, p, offs, false));
  if (cap < 1 || cap > c->cap || mirror_mode < 0 || mirror_mode > 2 || !std::isfinite(floor_z) ||
      keep_nearest < LP_KEEP_ALL || keep_nearest > LP_KEEP_OCTANTS)
    return LP_ERR_INVALID_ARG;
  if (!radius && !finite_pos(r_const)) return LP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(c->device);
  const int n = (int)p->n;
  if (!c->nbr_o) {
    LP_TRY(dalloc(c, &c->nbr_o, (size_t)c->cap_n * c->cap));
    LP_TRY(dalloc(c, &c->cnt_o, (size_t)c->cap_n));
  }
  out->nbr = c->nbr_o; out->cnt = c->cnt_o; out->n = n; out->cap = cap;
  if (n == 0) return LP_OK;
  const int d = c->cx;
  cudaMemcpyAsync(c->X[d][0], p->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(c->X[d][1], p->y, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(c->X[d][2], p->z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  if (radius)
    cudaMemcpyAsync(c->X[d][7], radius, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  launch_iota(n, c->ids[c->ci], st);
  LP_TRY(begin_columns(c, p, radius ? c->X[d][7] : nullptr, d, offs, st));
  double rmax = r_const;
  if (radius) {
    rmax = 0.0;
    for (int k = 0; k < p->ncolumns; ++k) rmax = std::max(rmax, c->h_bbox[7 * k + 6]);
    if (!finite_pos(rmax)) return LP_ERR_INVALID_ARG;
  }
  LP_TRY(setup_grids(c, p->ncolumns, rmax, st));
  sort_particles(c, n, 1, radius ? 4 : 3, st);
  const int e = c->cx;
  launch_neighbors(keep_nearest, n, c->X[e][0], c->X[e][1], c->X[e][2], c->pf,
                   c->colid[c->ci], c->ids[c->ci], c->d_grids, c->cells + 2 * c->cell_capacity,
                   radius ? c->X[e][7] : nullptr, r_const, mirror_mode, floor_z, cap, c->nbr,
                   c->cnt, c->dg, st);
  launch_nbr_to_caller(n, cap, c->ids[c->ci], c->nbr, c->cnt, c->nbr_o, c->cnt_o, st);
  return cuda_status();
}

lp_status lp_neighbors_export(lp_ctx* c, const lp_neighbors* nb, int32_t* host_nbr,
                              int32_t* host_cnt, void* stream) {
  if (!c || !nb || !host_nbr || !host_cnt || !nb->nbr || !nb->cnt || nb->n < 0 || nb->cap < 1)
    return LP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(c->device);
  const int64_t n = nb->n;
  const int cap = nb->cap;
  std::vector<int32_t> kn((size_t)n * cap), cn((size_t)n);
  if (n > 0) {
    if (cudaMemcpyAsync(kn.data(), nb->nbr, sizeof(int32_t) * n * cap, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(cn.data(), nb->cnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return LP_ERR_CUDA;
    }
  }
  std::vector<uint32_t> row;
  for (int64_t i = 0; i < n; ++i) {
    const int m = std::min(cn[i], cap);
    row.assign(m, 0);
    for (int k = 0; k < m; ++k) row[k] = (uint32_t)kn[(size_t)k * n + i];
    // real neighbours first, then mirrors; each ascending
    std::sort(row.begin(), row.end(), [](uint32_t a, uint32_t b) {
      if ((a >> 31) != (b >> 31)) return (a >> 31) < (b >> 31);
      return (a & 0x7fffffffu) < (b & 0x7fffffffu);
    });
    for (int k = 0; k < cap; ++k) host_nbr[i * cap + k] = k < m ? (int32_t)row[k] : 0;
    host_cnt[i] = m;
  }
  return LP_OK;
}

lp_status lp_fit_derivatives(lp_ctx* c, const lp_particles* p, const lp_neighbors* nb,
                             const double* const* fields, const double* mirror_sign, int32_t nf,
                             double h, double floor_z, double* coeffs, int32_t precision,
                             void* stream) {
  if (!c || !nb || !fields || !mirror_sign) return LP_ERR_INVALID_ARG;
  c->lists_valid = false;  // uses the buffers the kept Verlet lists live in
  std::vector<int32_t> offs;
  LP_TRY(check_particles(c, p, offs, false));
  if (p->n > 0 && !coeffs) return LP_ERR_INVALID_ARG;  // (empty arrays may be NULL)
  if (nf < 1 || nf > kMaxFields || !finite_pos(h) || !std::isfinite(floor_z) ||
      (precision != LP_FP64 && precision != LP_MIXED && precision != LP_MIXED_FF) ||
      nb->n != p->n || !nb->nbr || !nb->cnt ||
      nb->cap < 1 || nb->cap > LP_MAX_CAP)
    return LP_ERR_INVALID_ARG;
  for (int f = 0; f < nf; ++f)
    if ((p->n > 0 && !fields[f]) || !std::isfinite(mirror_sign[f])) return LP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(c->device);
  if (p->n == 0) return LP_OK;
  FitArgs F{};
  F.n = (int)p->n; F.cap = nb->cap; F.nf = nf;
  F.x = p->x; F.y = p->y; F.z = p->z;
  F.nbr = nb->nbr; F.cnt = nb->cnt;
  for (int f = 0; f < nf; ++f) {
    F.fields[f] = fields[f];
    F.msign[f] = mirror_sign[f];
  }
  F.inv_h = 1.0 / h; F.f2 = 2.0 * floor_z;
  F.coeffs = coeffs;
  F.fb_list = c->fb_list; F.fb_count = c->fb_count; F.fb_cap = c->fb_cap;
  F.dg = c->dg;
  if (precision == LP_MIXED_FF) {  // the step's split and factor buffers serve as scratch
    if (!c->fit_fs) LP_TRY(dalloc(c, &c->fit_fs, (size_t)kMaxFields * c->cap_n));
    F.xs = c->XU; F.fs = c->fit_fs; F.lf = c->Lff;
  }
  cudaMemsetAsync(c->fb_count, 0, sizeof(int32_t), st);
  launch_fit(precision, F, st);
  return cuda_status();
}

lp_status lp_mui_stress(lp_ctx* c, const lp_mui* mui, const lp_eos* eos, int64_t n,
                        const double* V, const double* grad_u, double* gdot, double* gdot_norm,
                        double* P, double* eta, int8_t* regime, void* stream) {
  if (!c || !mui || !eos || n < 0 || (n > 0 && (!V || !grad_u))) return LP_ERR_INVALID_ARG;
  if (!(eos->phi_min < eos->phi_max && eos->phi_max < eos->phi_c)) return LP_ERR_INVALID_ARG;
  cudaSetDevice(c->device);
  if (n == 0) return LP_OK;
  ColMui m{mui->mu_s, mui->mu_2, mui->I0, mui->d, mui->rho_s};
  launch_mui_stress(n, m, *eos, V, grad_u, gdot, gdot_norm, P, eta, regime,
                    (cudaStream_t)stream);
  return cuda_status();
}

namespace {
StepConsts step_consts(const lp_eos* eos, const lp_params* q, double dt, int cap) {
  StepConsts K{};
  K.phi_c = eos->phi_c; K.phi_min = eos->phi_min; K.phi_max = eos->phi_max;
  K.alpha = eos->alpha; K.beta = eos->beta;
  K.h = q->h; K.inv_h = 1.0 / q->h; K.radius = q->radius; K.r2 = q->radius * q->radius;
  K.gx = q->gx; K.gy = q->gy; K.gz = q->gz; K.floor_z = q->floor_z; K.dt = dt;
  K.mirror_mode = q->mirror_mode; K.cap = cap;
  K.free_surface = q->free_surface != 0;
  K.euler = q->time_scheme == LP_TIME_HEUN;
  // periodic boundaries (Sec. 3.1 item 9)
  K.Lx = q->period_x; K.Ly = q->period_y;
  K.periodic = (K.Lx > 0.0 || K.Ly > 0.0) ? 1 : 0;
  const double lhx = K.Lx * K.inv_h, lhy = K.Ly * K.inv_h;
  K.Lhx_h = (float)lhx; K.Lhx_l = (float)(lhx - (double)K.Lhx_h);
  K.Lhy_h = (float)lhy; K.Lhy_l = (float)(lhy - (double)K.Lhy_h);
  const double ih2 = K.inv_h * K.inv_h;
  K.ih_h = (float)K.inv_h; K.ih_l = (float)(K.inv_h - (double)K.ih_h);
  K.ih2_h = (float)ih2; K.ih2_l = (float)(ih2 - (double)K.ih2_h);
  K.phic_h = (float)K.phi_c; K.phic_l = (float)(K.phi_c - (double)K.phic_h);
  K.rho = (float)(q->radius / q->h * (1.0 + 0x1p-10));
  if (K.free_surface) {
    // ghost particles (Sec. 3.1 items 6 and 9): fixed-point grid K r <= 8192
    double g = 1.0;
    while (g * q->radius > 8192.0) g *= 0.5;
    while (2.0 * g * q->radius <= 8192.0) g *= 2.0;
    K.ghost_grid = g;
    const double rk = q->radius * g;
    K.ghost_R2 = std::llrint(rk * rk);
    K.ghost_hk = q->h * g;
    K.ghost_clear2 = std::llrint((0.5 * K.ghost_hk) * (0.5 * K.ghost_hk));
    const double phi_g = eos->phi_min * (1.0 - 1e-3);
    K.ghost_V = 1.0 / phi_g;
    K.ghost_num = eos->phi_c - phi_g;
    K.ghost_PX = K.Lx > 0.0 ? std::llrint(g * K.Lx) : 0;
    K.ghost_PY = K.Ly > 0.0 ? std::llrint(g * K.Ly) : 0;
  }
  return K;
}

// caller state -> internal buffer in caller order; per-column mu(I) upload
// Column record: the mu(I) parameters and the float-float constants of the
// inertial closure used by pass 2 of LP_MIXED_FF (a = phi_c - phi_min).
ColMui col_mui(const lp_mui& m, const lp_eos* e) {
  ColMui r{m.mu_s, m.mu_2, m.I0, m.d, m.rho_s};
  auto split = [](double v, float* f) {
    f[0] = (float)v;
    f[1] = (float)(v - (double)f[0]);
  };
  const double a = e->phi_c - e->phi_min;
  split(4.0 * a * a * m.d * m.d, r.kf);
  split(a * m.I0, r.aI0f);
  split(a * m.mu_s * m.I0, r.bf);
  split(m.mu_2, r.mu2f);
  split(a * m.I0 * (m.mu_2 - m.mu_s), r.cf);
  return r;
}

// (periods Lx, Ly > 0: positions along those axes mapped into [0, L);
// gather: into the sorted order of the previous call, kept in ids)
lp_status load_state(lp_ctx* c, const lp_particles* p, const lp_mui* mui, const lp_eos* eos,
                     cudaStream_t st, double Lx = 0.0, double Ly = 0.0, bool gather = false) {
  const int n = (int)p->n;
  std::vector<ColMui> hm(p->ncolumns);
  for (int k = 0; k < p->ncolumns; ++k) hm[k] = col_mui(mui[k], eos);
  if (cudaMemcpyAsync(c->d_mui, hm.data(), sizeof(ColMui) * p->ncolumns, cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
    return LP_ERR_CUDA;
  const int d = c->cx;
  double* const src[7] = {p->x, p->y, p->z, p->u, p->v, p->w, p->V};
  if (gather) {
    std::memcpy(c->h_ptr, src, sizeof(src));
    if (cudaMemcpyAsync(c->d_ptr, c->h_ptr, sizeof(src), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      return LP_ERR_CUDA;
    launch_gather_fields(n, c->ids[c->ci], (const double* const*)c->d_ptr,
                         c->d_tab + ((d * 2 + 0) * 2 + 0) * kTabFields, 7, st);
  } else {
    for (int f = 0; f < 7; ++f)
      cudaMemcpyAsync(c->X[d][f], src[f], sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    launch_iota(n, c->ids[c->ci], st);
  }
  if (Lx > 0.0 || Ly > 0.0) launch_wrap_positions(n, c->X[d][0], c->X[d][1], Lx, Ly, st);
  // mu(I) parameters are read back from pageable memory only once the copy ran
  return cudaStreamSynchronize(st) == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

int log2_bucket(int64_t v) {
  int b = 0;
  while (v > 1) { v >>= 1; ++b; }
  return b;
}
}  // namespace

namespace {
// 1: the kernels can read the array in place (device or managed memory);
// 0: host memory (pinned, registered or pageable)
int device_readable(const void* ptr) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? 1 : 0;
}
}  // namespace

lp_status lp_step(lp_ctx* c, lp_particles* p, const lp_mui* mui, const lp_eos* eos,
                  const lp_params* q, double dt, int32_t nsteps, void* stream) {
  if (!c || !mui || nsteps < 0) return LP_ERR_INVALID_ARG;
  std::vector<int32_t> offs;
  LP_TRY(check_particles(c, p, offs, true));
  if (!valid_params(q, eos, dt)) return LP_ERR_INVALID_ARG;
  if (q->radius * (1.0 / q->h) > 64.0) return LP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(c->device);
  const int n = (int)p->n;
  if (n == 0 || nsteps == 0) return LP_OK;
  {
    // Host arrays (all seven): copied in on the stream, stepped in the
    // context's staging block, copied back. Seven host arrays laid out one
    // after the other (x, y, z, u, v, w, V, each of n) move in one copy each
    // way.
    double* f7[7] = {p->x, p->y, p->z, p->u, p->v, p->w, p->V};
    int on_device = 0;
    for (int f = 0; f < 7; ++f) on_device += device_readable(f7[f]);
    if (on_device != 0 && on_device != 7) return LP_ERR_INVALID_ARG;  // mixed
    if (on_device == 0) {
      if (!c->stage) LP_TRY(dalloc(c, &c->stage, (size_t)7 * c->cap_n));
      bool packed = true;
      for (int f = 1; f < 7; ++f) packed = packed && f7[f] == f7[0] + (size_t)f * n;
      const size_t bytes = sizeof(double) * (size_t)n;
      if (packed) {
        if (cudaMemcpyAsync(c->stage, f7[0], 7 * bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
          return LP_ERR_CUDA;
      } else {
        for (int f = 0; f < 7; ++f)
          if (cudaMemcpyAsync(c->stage + (size_t)f * n, f7[f], bytes, cudaMemcpyHostToDevice,
                              st) != cudaSuccess)
            return LP_ERR_CUDA;
      }
      lp_particles d = *p;
      double** dp[7] = {&d.x, &d.y, &d.z, &d.u, &d.v, &d.w, &d.V};
      for (int f = 0; f < 7; ++f) *dp[f] = c->stage + (size_t)f * n;
      const lp_status r = lp_step(c, &d, mui, eos, q, dt, nsteps, stream);
      if (r != LP_OK) return r;
      if (packed) {
        if (cudaMemcpyAsync(f7[0], c->stage, 7 * bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
          return LP_ERR_CUDA;
      } else {
        for (int f = 0; f < 7; ++f)
          if (cudaMemcpyAsync(f7[f], c->stage + (size_t)f * n, bytes, cudaMemcpyDeviceToHost,
                              st) != cudaSuccess)
            return LP_ERR_CUDA;
      }
      return cuda_status();
    }
  }
  const StepConsts K = step_consts(eos, q, dt, c->cap);
  // Verlet candidate lists: the grid must hold radius + skin in one cell. The
  // lists live for one call unless keep_lists asks to keep them for the next
  // one; without that, the wider first search only pays off from about three
  // steps on and fewer steps search with the radius alone (the stencils are
  // the same either way).
  const bool keep = q->keep_lists != 0 && q->skin > 0.0 && q->rebuild_every == 1;
  const double skin =
      (q->skin > 0.0 && q->rebuild_every == 1 && (nsteps >= 3 || keep)) ? q->skin : 0.0;
  const double sig[6] = {q->radius, q->skin, q->floor_z, (double)q->mirror_mode, q->period_x,
                         q->period_y};
  const bool reuse = keep && c->lists_valid && c->lists_n == n && c->lists_offs == offs &&
                     std::memcmp(sig, c->lists_sig, sizeof(sig)) == 0;
  c->lists_valid = false;  // until this call has completed
  LP_TRY(load_state(c, p, mui, eos, st, q->period_x, q->period_y, reuse));
  const int d = c->cx;
  LP_TRY(begin_columns(c, p, nullptr, d, offs, st, !reuse));
  // kept lists keep their grid while the particles fit in it (the split
  // positions of the float-float fits are taken relative to its origin)
  if (!reuse || !grids_cover(c, p->ncolumns))
    LP_TRY(setup_grids(c, p->ncolumns, q->radius + skin, st, q->period_x, q->period_y));
  LP_TRY(ensure_twin_buffers(c, q));
  if (skin > 0.0) {
    // a search on the first step, or (kept lists) only if some particle moved
    // more than skin/2 since the last one
    const int first = reuse ? 0 : 1;
    if (cudaMemcpyAsync(c->d_search, &first, sizeof(int), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
      return LP_ERR_CUDA;
    // filter margins carry over only with the kept lists of a call that kept
    // them up to date (no ghosts, no persistent launch): nothing else has
    // written the stencils since, and the need-search test below adds the
    // caller's new state to the displacement bounds; otherwise NaN margins,
    // so that every particle is filtered on the first step
    if (!(reuse && c->marg_valid) &&
        cudaMemsetAsync(c->vmarg, 0xff, sizeof(float) * n, st) != cudaSuccess)
      return LP_ERR_CUDA;
    if (reuse) {
      const double hs = 0.5 * skin;
      launch_need_search(n, c->X[d][0], c->X[d][1], c->X[d][2], c->xref,
                         hs * hs * (1.0 - 0x1p-20), q->period_x, q->period_y, c->d_search,
                         VerletSkip{c->vmarg, c->vdmax, c->vdall}, st);
      c->launches += 2;  // gather, displacement test
    }
  }
  c->skin = skin;
  const lp_status rs = run_steps(c, n, K, q->precision, q->rebuild_every, q->launch_mode, nsteps,
                                 st);
  c->skin = 0.0;
  LP_TRY(rs);
  // after a bounded wait gave up, the internal state is incomplete: leave the
  // caller's arrays as they were (lp_ctx_sync reports LP_ERR_TIMEOUT)
  if (q->launch_mode == LP_LAUNCH_PERSISTENT) {
    unsigned flags = 0;
    if (cudaMemcpyAsync(&c->h_dg->flags, &c->dg->flags, sizeof(unsigned),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return LP_ERR_CUDA;
    flags = c->h_dg->flags;
    if (flags & LP_FLAG_TIMEOUT) return LP_OK;
  }
  if (keep && skin > 0.0) {  // lists, reference positions and order stay for the next call
    c->lists_valid = true;
    c->marg_valid = !K.free_surface && q->launch_mode != LP_LAUNCH_PERSISTENT;
    c->lists_n = n;
    c->lists_offs = offs;
    std::memcpy(c->lists_sig, sig, sizeof(sig));
  }
  // internal state -> caller arrays (original order)
  {
    const int e = c->cx;
    const double* const* dsrc = (const double* const*)(c->d_tab + ((e * 2 + 0) * 2 + 0) * kTabFields);
    double* hp[7] = {p->x, p->y, p->z, p->u, p->v, p->w, p->V};
    std::memcpy(c->h_ptr, hp, sizeof(hp));
    cudaMemcpyAsync(c->d_ptr, c->h_ptr, sizeof(hp), cudaMemcpyHostToDevice, st);
    launch_scatter_state(n, c->ids[c->ci], dsrc, c->d_ptr, 7, st);
    c->launches += 4;  // fill_colid, bbox, iota, scatter_state
    if (cudaStreamSynchronize(st) != cudaSuccess) return LP_ERR_CUDA;
  }
  return cuda_status();
}

lp_status lp_ctx_set_tuning(lp_ctx* c, const lp_tuning* t) {
  if (!c || !t) return LP_ERR_INVALID_ARG;
  for (int b : {t->block_neighbors, t->block_pass1, t->block_pass2})
    if (b != 64 && b != 128 && b != 256) return LP_ERR_INVALID_ARG;
  c->bs_nbr = t->block_neighbors;
  c->bs_p1 = t->block_pass1;
  c->bs_p2 = t->block_pass2;
  return LP_OK;
}

lp_status lp_autotune(lp_ctx* c, const lp_particles* p, const lp_mui* mui, const lp_eos* eos,
                      const lp_params* q, double dt, int32_t steps_per_trial,
                      const char* table_path, lp_tuning* out, void* stream) {
  if (!c || !mui || !out || steps_per_trial < 1 || steps_per_trial > 1000)
    return LP_ERR_INVALID_ARG;
  c->lists_valid = false;  // uses the buffers the kept Verlet lists live in
  std::vector<int32_t> offs;
  LP_TRY(check_particles(c, p, offs, true));
  if (!valid_params(q, eos, dt) || p->n < 1) return LP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(c->device);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) return LP_ERR_CUDA;
  // table key: device, log2 n, log2 columns, precision, stencil radius in h/10
  std::string dev = prop.name;
  for (char& ch : dev)
    if (ch == ' ' || ch == '|') ch = '_';
  char key[256];
  std::snprintf(key, sizeof(key), "%s|n2^%d|c2^%d|p%d|r%d", dev.c_str(), log2_bucket(p->n),
                log2_bucket(p->ncolumns), q->precision, (int)std::lround(10.0 * q->radius / q->h));
  if (table_path) {
    if (FILE* fp = std::fopen(table_path, "r")) {
      char line[512];
      while (std::fgets(line, sizeof(line), fp)) {
        char k[256];
        lp_tuning t{};
        if (std::sscanf(line, "%255s %d %d %d %d %lf", k, &t.block_neighbors, &t.block_pass1,
                        &t.block_pass2, &t.launch_mode, &t.ms_per_step) == 6 &&
            std::strcmp(k, key) == 0) {
          std::fclose(fp);
          t.from_table = 1;
          LP_TRY(lp_ctx_set_tuning(c, &t));
          *out = t;
          return LP_OK;
        }
      }
      std::fclose(fp);
    }
  }
  const int n = (int)p->n;
  const StepConsts K = step_consts(eos, q, dt, c->cap);
  const int R = q->rebuild_every;
  // every trial starts from the caller's state (which is never modified)
  auto restart = [&]() -> lp_status {
    LP_TRY(load_state(c, p, mui, eos, st, q->period_x, q->period_y));
    launch_fill_colid(n, c->d_offs, p->ncolumns, c->colid[c->ci], st);
    return LP_OK;
  };
  LP_TRY(load_state(c, p, mui, eos, st, q->period_x, q->period_y));
  LP_TRY(begin_columns(c, p, nullptr, c->cx, offs, st));
  LP_TRY(setup_grids(c, p->ncolumns, q->radius, st, q->period_x, q->period_y));
  LP_TRY(ensure_twin_buffers(c, q));
  // block sizes: per-phase device time of each candidate
  const int cand[3] = {64, 128, 256};
  double best_ms[LP_NPHASES];
  int best_bs[LP_NPHASES];
  for (int k = 0; k < LP_NPHASES; ++k) {
    best_ms[k] = 1e300;
    best_bs[k] = kBlock;
  }
  const bool prof0 = c->profile;
  double ms[LP_NPHASES];
  for (int bs : cand) {
    LP_TRY(restart());
    c->bs_nbr = c->bs_p1 = c->bs_p2 = bs;
    lp_ctx_phase_times(c, st, ms, nullptr, nullptr);  // reset
    c->profile = true;
    const lp_status r = run_steps(c, n, K, q->precision, R, LP_LAUNCH_KERNELS, steps_per_trial, st);
    c->profile = prof0;
    LP_TRY(r);
    LP_TRY(lp_ctx_phase_times(c, st, ms, nullptr, nullptr));
    for (int k = 0; k < LP_NPHASES; ++k)
      if (ms[k] < best_ms[k]) {
        best_ms[k] = ms[k];
        best_bs[k] = bs;
      }
  }
  lp_tuning t{};
  t.block_neighbors = best_bs[LP_PHASE_NEIGHBORS];
  t.block_pass1 = best_bs[LP_PHASE_PASS1];
  t.block_pass2 = best_bs[LP_PHASE_PASS2];
  LP_TRY(lp_ctx_set_tuning(c, &t));
  // launch mode: whole-step time of graph replay vs one persistent launch
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int modes[2] = {LP_LAUNCH_GRAPH, LP_LAUNCH_PERSISTENT};
  double mode_ms[2] = {1e300, 1e300};
  const int steps = std::max(steps_per_trial, 4 * R);
  for (int m = 0; m < 2; ++m) {
    if (modes[m] == LP_LAUNCH_GRAPH && st == nullptr) continue;
    LP_TRY(restart());
    cudaEventRecord(e0, st);
    const lp_status r = run_steps(c, n, K, q->precision, R, modes[m], steps, st);
    cudaEventRecord(e1, st);
    if (r != LP_OK || cudaEventSynchronize(e1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    float el = 0.f;
    cudaEventElapsedTime(&el, e0, e1);
    mode_ms[m] = el / steps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const int pick = mode_ms[1] < mode_ms[0] ? 1 : 0;
  if (mode_ms[pick] >= 1e299) return LP_ERR_CUDA;
  t.launch_mode = modes[pick];
  t.ms_per_step = mode_ms[pick];
  t.from_table = 0;
  lp_diag dummy;
  lp_ctx_sync(c, st, &dummy);  // trial steps may flag a blow-up; not the caller's state
  if (table_path) {
    if (FILE* fp = std::fopen(table_path, "a")) {
      std::fprintf(fp, "%s %d %d %d %d %.6f\n", key, t.block_neighbors, t.block_pass1,
                   t.block_pass2, t.launch_mode, t.ms_per_step);
      std::fclose(fp);
    }
  }
  *out = t;
  return LP_OK;
}

lp_status lp_step_adjoint(lp_ctx* c, const lp_particles* initial, const lp_mui* mui,
                          const lp_eos* eos, const lp_params* q, double dt, int32_t nsteps,
                          int32_t checkpoint_every, const lp_particles* seed, double* dL_dmui,
                          lp_particles* dL_dinitial, void* stream) {
  if (!c || !mui || !seed || !dL_dmui || nsteps < 0 || checkpoint_every < 1)
    return LP_ERR_INVALID_ARG;
  c->lists_valid = false;  // uses the buffers the kept Verlet lists live in
  std::vector<int32_t> offs;
  LP_TRY(check_particles(c, initial, offs, true));
  if (!valid_params(q, eos, dt) || q->precision != LP_FP64) return LP_ERR_INVALID_ARG;
  if (seed->n != initial->n || (initial->n > 0 && (!seed->x || !seed->y || !seed->z || !seed->u ||
                                                   !seed->v || !seed->w || !seed->V)))
    return LP_ERR_INVALID_ARG;
  if (dL_dinitial && (dL_dinitial->n != initial->n ||
                      (initial->n > 0 && (!dL_dinitial->x || !dL_dinitial->y || !dL_dinitial->z ||
                                          !dL_dinitial->u || !dL_dinitial->v || !dL_dinitial->w ||
                                          !dL_dinitial->V))))
    return LP_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaSetDevice(c->device);
  const int n = (int)initial->n;
  cudaMemsetAsync(dL_dmui, 0, 3 * sizeof(double), st);
  if (n == 0 || nsteps == 0) {
    if (dL_dinitial && n > 0) {
      double* const dst[7] = {dL_dinitial->x, dL_dinitial->y, dL_dinitial->z, dL_dinitial->u,
                              dL_dinitial->v, dL_dinitial->w, dL_dinitial->V};
      const double* const src[7] = {seed->x, seed->y, seed->z, seed->u, seed->v, seed->w, seed->V};
      for (int f = 0; f < 7; ++f)
        cudaMemcpyAsync(dst[f], src[f], sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    }
    return cuda_status();
  }
  const int C = checkpoint_every;
  const int nseg = (nsteps + C - 1) / C;
  std::vector<ColMui> hm(initial->ncolumns);
  for (int k = 0; k < initial->ncolumns; ++k) hm[k] = col_mui(mui[k], eos);
  if (cudaMemcpyAsync(c->d_mui, hm.data(), sizeof(ColMui) * initial->ncolumns,
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return LP_ERR_CUDA;
  const StepConsts K = step_consts(eos, q, dt, c->cap);  // periods, time scheme included
  LP_TRY(ensure_twin_buffers(c, q));  // the saved state of Heun's method
  // Heun's method: a segment keeps y^k and the first stage's y*_k of each step
  const bool heun = q->time_scheme == LP_TIME_HEUN;
  const int nkept = heun ? 2 * C + 1 : C + 1;
  const size_t N = (size_t)n;

  // Per-step fit data (the paper's step; Heun's method keeps recomputing):
  // each step's factors, pass-1 outputs, coefficients and QR-fallback slots
  // and gradients, so that the reverse sweep reads them instead of computing
  // each step again. Two ways to get them:
  //  - keep: with room for every segment's states, fit data and stencils
  //    (within the context's adjoint memory limit), the forward sweep runs
  //    each segment as below and keeps it all; the reverse sweep recomputes
  //    nothing;
  //  - recompute: the forward sweep keeps only the checkpoints, and the
  //    reverse sweep re-runs each segment from its checkpoint, keeping that
  //    segment's data; without room even for that, each reverse step
  //    recomputes its own.
  const size_t per_step = N * (size_t)(P1_N + kTri + 27 + 18) + (size_t)c->fb_cap * 6;
  const size_t nsnap = (size_t)c->cap + 3;  // a segment's stencils: nbr, cnt, ids, colid
  bool keep = false;
  if (!heun && c->adj_keep_bytes != 0) {
    const size_t need =
        sizeof(double) * (7 * N * (size_t)(nseg - 1) * nkept + per_step * (size_t)nsteps) +
        sizeof(int32_t) * N * ((size_t)nsteps + nsnap * nseg);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
      const size_t lim =
          c->adj_keep_bytes < 0 ? fr / 2 : std::min((size_t)c->adj_keep_bytes, fr);
      keep = need <= lim;
    } else {
      cudaGetLastError();
    }
  }
  double* Wk = nullptr;
  int32_t* Fk = nullptr;
  auto alloc_fit_data = [&](int steps_kept, size_t extra_i32) {
    if (cudaMalloc(&Wk, per_step * (size_t)steps_kept * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&Fk, (N * (size_t)steps_kept + extra_i32) * sizeof(int32_t)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(Wk);
      Wk = nullptr;
      Fk = nullptr;
      return false;
    }
    return true;
  };
  if (keep) keep = alloc_fit_data(nsteps, nsnap * N * (size_t)nseg);
  if (!heun && !keep) alloc_fit_data(C, 0);
  const int nsegk = keep ? nseg : 1;  // segments whose states the workspace holds
  struct StepData {
    double *p1, *fac, *coef1, *coef2, *fbgrad;
    int32_t* fbslot;
  };
  // fit data of step k of segment s2
  auto step_data = [&](int s2, int k) {
    const size_t i = keep ? (size_t)s2 * C + k : (size_t)k;
    double* b = Wk + per_step * i;
    return StepData{b, b + N * P1_N, b + N * (P1_N + kTri), b + N * (P1_N + kTri + 27),
                    b + N * (P1_N + kTri + 45), Fk + N * i};
  };
  // stencils of segment s2 (keep) in the segment's sorted order
  struct Stencils {
    const int32_t *nbr, *cnt, *ids, *colid;
  };
  auto snapshot = [&](int s2) {
    int32_t* b = Fk + N * (size_t)nsteps + nsnap * N * (size_t)s2;
    return b;
  };

  // workspace of this call: checkpoints, segment states, coefficients, adjoints
  const size_t nd = N * (7 * (size_t)nseg + 7 * (size_t)nkept * nsegk + 27 + 18 + 14 + 2 + 6 +
                         3 + 18 + 7 + 45 + 1 + 1 + (heun ? 14 : 0)) +
                    3;
  double* W = nullptr;
  if (cudaMalloc(&W, nd * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(Wk);
    cudaFree(Fk);
    return LP_ERR_OOM;
  }
  double* p = W;
  auto take = [&](size_t k) { double* r = p; p += k; return r; };
  double* ckpt = take(7 * N * nseg);
  double* seg = take(7 * N * nkept * nsegk);
  double* coef1 = take(27 * N);
  double* coef2 = take(18 * N);
  double* lam[2] = {take(7 * N), take(7 * N)};
  double* lGn = take(N);
  double* lVn = take(N);
  double* lVd = take(N);
  double* lamH = heun ? take(7 * N) : nullptr;  // Heun: half the adjoint, for y**
  double* lamS = heun ? take(7 * N) : nullptr;  // Heun: adjoint of y*
  double* lG6 = take(6 * N);
  double* lld = take(3 * N);
  double* zz = take(18 * N);
  double* scratch = take(7 * N);
  double* facx = take(45 * N);
  uint8_t* okf = (uint8_t*)take(N);  // N bytes used of N doubles
  double* dth = take(3);
  // device pointer tables: checkpoints (nseg x 7), segment states (nsegk x
  // nkept x 7), lam[0], lam[1], seed, caller initial, dL_dinitial, internal
  // X[0], X[1]
  const int nstates = nkept * nsegk;
  const int ntab = 7 * nseg + 7 * nstates + 7 * 7;
  std::vector<double*> tab(ntab);
  for (int s2 = 0; s2 < nseg; ++s2)
    for (int f = 0; f < 7; ++f) tab[7 * s2 + f] = ckpt + (size_t)(7 * s2 + f) * N;
  const int tseg = 7 * nseg;
  for (int k = 0; k < nstates; ++k)
    for (int f = 0; f < 7; ++f) tab[tseg + 7 * k + f] = seg + (size_t)(7 * k + f) * N;
  const int tlam = tseg + 7 * nstates;
  for (int b = 0; b < 2; ++b)
    for (int f = 0; f < 7; ++f) tab[tlam + 7 * b + f] = lam[b] + (size_t)f * N;
  const int tseed = tlam + 14;
  double* const sd[7] = {seed->x, seed->y, seed->z, seed->u, seed->v, seed->w, seed->V};
  for (int f = 0; f < 7; ++f) tab[tseed + f] = sd[f];
  const int tinit = tseed + 7;
  double* const in[7] = {initial->x, initial->y, initial->z, initial->u, initial->v, initial->w,
                         initial->V};
  for (int f = 0; f < 7; ++f) tab[tinit + f] = in[f];
  const int tout = tinit + 7;
  for (int f = 0; f < 7; ++f) tab[tout + f] = dL_dinitial ? (&dL_dinitial->x)[f] : lam[0];
  const int tX = tout + 7;
  for (int d = 0; d < 2; ++d)
    for (int f = 0; f < 7; ++f) tab[tX + 7 * d + f] = c->X[d][f];
  double** dtab = nullptr;
  if (cudaMalloc(&dtab, sizeof(double*) * ntab) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(W);
    cudaFree(Wk);
    cudaFree(Fk);
    return LP_ERR_OOM;
  }
  // state i of segment s2 (host table; the device copy at the same offset)
  auto kept_at = [&](int s2, int i) { return tseg + 7 * ((keep ? s2 : 0) * nkept + i); };
  StepArgs S{};
  auto one_pass = [&](double* const* in, double* const* out) {
    S.x = in[0]; S.y = in[1]; S.z = in[2]; S.u = in[3]; S.v = in[4]; S.w = in[5]; S.V = in[6];
    S.xo = out[0]; S.yo = out[1]; S.zo = out[2]; S.uo = out[3]; S.vo = out[4]; S.wo = out[5];
    S.Vo = out[6];
    cudaMemsetAsync(c->fb_count, 0, sizeof(int32_t), st);
    launch_pass1(LP_FP64, S, st);
    launch_pass2(LP_FP64, S, st);
  };
  // segment s2 from its checkpoint: the stencils rebuilt exactly as the
  // forward run built them, then every step, keeping each state (Heun's
  // method: the state y^k at 2k, the first stage's y*_k at 2k + 1) and, with
  // room for it, each step's fit data
  auto run_segment = [&](int s2) {
    const int steps = std::min(C, nsteps - s2 * C);
    for (int f = 0; f < 7; ++f)
      cudaMemcpyAsync(c->X[c->cx][f], tab[7 * s2 + f], sizeof(double) * N,
                      cudaMemcpyDeviceToDevice, st);
    launch_iota(n, c->ids[c->ci], st);
    launch_fill_colid(n, c->d_offs, initial->ncolumns, c->colid[c->ci], st);
    sort_particles(c, n, 0, 7, st);
    launch_neighbors(false, n, c->X[c->cx][0], c->X[c->cx][1], c->X[c->cx][2], c->pf,
                     c->colid[c->ci], c->ids[c->ci], c->d_grids,
                     c->cells + 2 * c->cell_capacity, nullptr, K.radius, K.mirror_mode,
                     K.floor_z, c->cap, c->nbr, c->cnt, c->dg, st, kBlock, nullptr, nullptr,
                     K.periodic != 0);
    if (K.free_surface)  // the same ghost flags as the forward run
      launch_ghosts(n, c->X[c->cx][0], c->X[c->cx][1], c->X[c->cx][2], c->colid[c->ci],
                    c->d_grids, c->Xfix, c->nbr, c->cnt, c->gcnt, K, c->dg, st, kBlock,
                    c->glist, c->gcount, c->olist);
    for (int f = 0; f < 7; ++f)
      cudaMemcpyAsync(tab[kept_at(s2, 0) + f], c->X[c->cx][f], sizeof(double) * N,
                      cudaMemcpyDeviceToDevice, st);
    S = step_args(c, n, K);
    auto kept = [&](int i) { return &tab[kept_at(s2, i)]; };
    for (int k = 0; k < steps; ++k) {
      if (!heun) {
        if (Wk) {
          const StepData d = step_data(s2, k);
          S.p1 = d.p1; S.fac = d.fac; S.coef1 = d.coef1; S.coef2 = d.coef2;
          S.fbslot = d.fbslot; S.fbgrad = d.fbgrad;
        }
        one_pass(kept(k), kept(k + 1));
      } else {  // two stages on the segment's stencils, then the average
        one_pass(kept(2 * k), kept(2 * k + 1));
        one_pass(kept(2 * k + 1), kept(2 * k + 2));
        launch_heun_combine(n, kept(2 * k + 2), kept(2 * k), K.Lx, K.Ly, st);
      }
    }
    S.p1 = c->p1; S.fac = c->fac; S.coef1 = S.coef2 = nullptr;
    S.fbslot = c->fbslot; S.fbgrad = c->fbgrad;
  };
  lp_status rs = LP_OK;
  do {
    if (cudaMemcpy(dtab, tab.data(), sizeof(double*) * ntab, cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      rs = LP_ERR_CUDA;
      break;
    }
    cudaMemsetAsync(dth, 0, 3 * sizeof(double), st);
    // ---- forward sweep: checkpoints at segment starts (caller order)
    for (int f = 0; f < 7; ++f) {
      cudaMemcpyAsync(c->X[c->cx][f], in[f], sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(tab[f], in[f], sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
    }
    if (K.periodic) {  // positions along periodic axes into [0, L), as lp_step
      launch_wrap_positions(n, c->X[c->cx][0], c->X[c->cx][1], K.Lx, K.Ly, st);
      launch_wrap_positions(n, tab[0], tab[1], K.Lx, K.Ly, st);
    }
    launch_iota(n, c->ids[c->ci], st);
    rs = begin_columns(c, initial, nullptr, c->cx, offs, st);
    if (rs != LP_OK) break;
    rs = setup_grids(c, initial->ncolumns, q->radius, st, q->period_x, q->period_y);
    if (rs != LP_OK) break;
    if (keep) {
      // every segment as the reverse sweep's re-run would run it, kept whole:
      // its stencils, and its last state (caller order) as the next checkpoint
      for (int s2 = 0; s2 < nseg; ++s2) {
        run_segment(s2);
        int32_t* sn = snapshot(s2);
        cudaMemcpyAsync(sn, c->nbr, sizeof(int32_t) * N * c->cap, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(sn + N * c->cap, c->cnt, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice,
                        st);
        cudaMemcpyAsync(sn + N * (c->cap + 1), c->ids[c->ci], sizeof(int32_t) * N,
                        cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(sn + N * (c->cap + 2), c->colid[c->ci], sizeof(int32_t) * N,
                        cudaMemcpyDeviceToDevice, st);
        if (s2 + 1 < nseg)
          launch_scatter_state(n, c->ids[c->ci],
                               (const double* const*)(dtab + kept_at(s2, std::min(C, nsteps - s2 * C))),
                               dtab + 7 * (s2 + 1), 7, st);
      }
    } else {
      for (int k = 0; k < nsteps; ++k) {
        if (k > 0 && k % C == 0)
          launch_scatter_state(n, c->ids[c->ci], (const double* const*)(dtab + tX + 7 * c->cx),
                               dtab + 7 * (k / C), 7, st);
        one_step(c, n, K, LP_FP64, k % C == 0, st);
      }
    }
    // ---- reverse sweep
    int cur = 0;  // lam[cur] holds the adjoint (caller order between segments)
    for (int f = 0; f < 7; ++f)
      cudaMemcpyAsync(lam[cur] + f * N, sd[f], sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
    for (int s2 = nseg - 1; s2 >= 0; --s2) {
      const int steps = std::min(C, nsteps - s2 * C);
      Stencils sten{c->nbr, c->cnt, c->ids[c->ci], c->colid[c->ci]};
      if (keep) {
        const int32_t* sn = snapshot(s2);
        sten = Stencils{sn, sn + N * c->cap, sn + N * (c->cap + 1), sn + N * (c->cap + 2)};
      } else {
        run_segment(s2);
        sten = Stencils{c->nbr, c->cnt, c->ids[c->ci], c->colid[c->ci]};
      }
      auto kept = [&](int i) { return &tab[kept_at(s2, i)]; };
      // adjoint to the sorted order of this segment
      launch_gather_fields(n, sten.ids, (const double* const*)(dtab + tlam + 7 * cur),
                           dtab + tlam + 7 * (1 - cur), 7, st);
      cur = 1 - cur;
      // adjoint of one step (the paper's) or one stage (Heun's method) from
      // state `sk`: l0 = J^T l1, with the step's kept fit data (k_stored >= 0:
      // its step within the segment) or recomputed here
      auto adjoint_at = [&](double* const* sk, const double* l1, double* l0, int k_stored) {
        AdjArgs J{};
        J.n = n; J.cap = c->cap;
        J.x = sk[0]; J.y = sk[1]; J.z = sk[2]; J.u = sk[3]; J.v = sk[4]; J.w = sk[5];
        J.V = sk[6];
        J.nbr = sten.nbr; J.cnt = sten.cnt; J.colid = sten.colid; J.mui = c->d_mui;
        J.grids = c->d_grids; J.XU = c->XU;  // (free: the FP64 re-runs do not split)
        if (k_stored >= 0) {
          const StepData d = step_data(s2, k_stored);
          J.fbslot = d.fbslot; J.fac = d.fac; J.p1 = d.p1; J.coef1 = d.coef1;
          J.coef2 = d.coef2; J.fbgrad = d.fbgrad;
        } else {
          double* const out[7] = {scratch,         scratch + N,     scratch + 2 * N,
                                  scratch + 3 * N, scratch + 4 * N, scratch + 5 * N,
                                  scratch + 6 * N};
          S.coef1 = coef1;
          S.coef2 = coef2;
          one_pass(sk, out);
          S.coef1 = S.coef2 = nullptr;
          J.fbslot = c->fbslot; J.fac = c->fac; J.p1 = c->p1; J.coef1 = coef1; J.coef2 = coef2;
          J.fbgrad = c->fbgrad;
        }
        J.K = K;
        for (int f = 0; f < 7; ++f) {
          J.l1[f] = l1 + f * N;
          J.l0[f] = l0 + f * N;
        }
        J.lGn = lGn; J.lVn = lVn; J.lVd = lVd; J.lG6 = lG6; J.lld = lld; J.zz = zz;
        J.dtheta = dth; J.dg = c->dg; J.ok = okf; J.facx = facx;
        launch_adjoint_step(J, st);
      };
      for (int k = steps - 1; k >= 0; --k) {
        if (!heun) {
          adjoint_at(kept(k), lam[cur], lam[1 - cur], Wk ? k : -1);
        } else {
          // y^{k+1} = (y^k + y**) / 2: half the adjoint to each; then the second
          // stage (from y*) and the first (from y^k), and the direct half
          launch_axpby((int64_t)(7 * N), 0.0, lam[cur], 0.5, lam[cur], st);
          cudaMemcpyAsync(lamH, lam[cur], sizeof(double) * 7 * N, cudaMemcpyDeviceToDevice, st);
          adjoint_at(kept(2 * k + 1), lamH, lamS, -1);
          adjoint_at(kept(2 * k), lamS, lam[1 - cur], -1);
          launch_axpby((int64_t)(7 * N), 1.0, lam[cur], 1.0, lam[1 - cur], st);
        }
        cur = 1 - cur;
      }
      // back to caller order
      launch_scatter_state(n, sten.ids, (const double* const*)(dtab + tlam + 7 * cur),
                           dtab + tlam + 7 * (1 - cur), 7, st);
      cur = 1 - cur;
    }
    if (dL_dinitial)
      for (int f = 0; f < 7; ++f)
        cudaMemcpyAsync(tab[tout + f], lam[cur] + f * N, sizeof(double) * N,
                        cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(dL_dmui, dth, 3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) rs = LP_ERR_CUDA;
    if (rs == LP_OK) rs = cuda_status();
  } while (0);
  cudaFree(dtab);
  cudaFree(Wk);
  cudaFree(Fk);
  cudaFree(W);
  return rs;
}

}  // extern "C"
