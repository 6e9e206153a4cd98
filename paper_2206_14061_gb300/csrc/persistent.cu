// One LP step as a single persistent, cooperative launch over all particles
// of all columns: cell sort, neighbour search, pass 1 and pass 2 run as
// phases of one kernel, separated by a grid barrier. The same device bodies
// as the per-phase kernels are used, so results are identical. The kernel
// takes the bodies' periodic variants (PER) in every run: with both periods 0
// they reduce to exactly the arithmetic of the non-periodic ones.
//
// The barrier is a generation counter in global memory. A block that waits
// longer than the spin limit sets LP_FLAG_TIMEOUT and leaves the kernel, so
// the launch always ends; the host reads the flag with lp_ctx_sync. The
// launch is cooperative, so all blocks are resident and the limit is never
// reached by a correct run.
#include "fit_bodies.cuh"
#include "nbr_bodies.cuh"

namespace lp {

constexpr int kPTile = kBlock * kScanItems;  // scan tile of one persistent block

int64_t persistent_scan_tiles(int64_t len) { return (len + kPTile - 1) / kPTile; }

// Grid barrier with a bounded wait. Returns false if this block gave up.
__device__ __forceinline__ bool grid_sync(unsigned* bar, unsigned long long max_spins,
                                          unsigned extra, DevDiag* dg) {
  __shared__ int gave_up;
  __syncthreads();
  if (threadIdx.x == 0) {
    gave_up = 0;
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    if (arrived == gridDim.x + extra) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned long long spins = 0;
      while (*vgen == gen) {
        if (++spins > max_spins) {
          gave_up = 1;
          atomicOr(&dg->flags, (unsigned)LP_FLAG_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return !gave_up;
}

#define LP_SYNC_OR_LEAVE()                                  \
  do {                                                      \
    if (!grid_sync(P.bar, P.max_spins, P.extra_arrivals, P.S.dg)) return; \
  } while (0)

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Profiling only: thread 0 of block 0 adds the time since the last mark
// (kept in phase_ns[LP_NPHASES]) to phase `ph`; called right after a grid
// barrier, so the mark is the moment every block has finished the phase.
__device__ __forceinline__ void phase_stamp(const PersistArgs& P, int ph) {
  if (P.phase_ns && blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long t = global_ns();
    if (ph >= 0) P.phase_ns[ph] += t - P.phase_ns[LP_NPHASES];
    P.phase_ns[LP_NPHASES] = t;
  }
}

// float-float: at most 128 registers (4 blocks per SM), as the per-phase
// float-float kernels; FP64 and MIXED at 3 blocks per SM (168 registers),
// where their bodies do not spill much
template <int PREC>
__global__ void __launch_bounds__(kBlock, PREC == LP_MIXED_FF ? 4 : 3)
    k_step_persistent(const PersistArgs P) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  const int n = P.n;
  const StepArgs& S = P.S;
  phase_stamp(P, -1);  // start mark
  // The search flag is read before the first barrier and cleared only by the
  // filter phase, after several barriers, so every block takes the same
  // branch. Without candidate lists every rebuild searches.
  const bool skin = P.search != nullptr;
  const bool srch = P.rebuild && (!skin || *(volatile int*)P.search != 0);
  if (srch) {
    // cell counts and fill counters start at zero
    for (int64_t i = tid; i < 2 * (P.ncell + 2); i += nth) {
      if (i < P.ncell + 2) P.count[i] = 0u;
      else P.fill[i - (P.ncell + 2)] = 0u;
    }
    LP_SYNC_OR_LEAVE();
    for (int s = tid; s < n; s += nth)
      keys_body(s, P.xs, P.ys, P.zs, P.colid_in, P.grids, (uint32_t)P.ncell, P.key, P.count);
    LP_SYNC_OR_LEAVE();
    // exclusive scan of ncell + 2 counts: tiles of kPTile, tile sums, add
    {
      __shared__ uint32_t tot;
      const int64_t len = P.ncell + 2;
      for (int tl = blockIdx.x; tl < P.ntiles; tl += gridDim.x) {
        const int64_t base = (int64_t)tl * kPTile + (int64_t)threadIdx.x * kScanItems;
        uint32_t v[kScanItems];
        uint32_t t = 0;
        for (int k = 0; k < kScanItems; ++k) {
          v[k] = (base + k < len) ? P.count[base + k] : 0u;
          t += v[k];
        }
        uint32_t ex = block_exclusive_scan(t, &tot);
        for (int k = 0; k < kScanItems; ++k) {
          if (base + k < len) P.start[base + k] = ex;
          ex += v[k];
        }
        if (threadIdx.x == 0) P.tile[tl] = tot;
      }
      LP_SYNC_OR_LEAVE();
      if (blockIdx.x == 0) {
        uint32_t carry = 0;
        for (int b = 0; b < P.ntiles; b += blockDim.x) {
          const int i = b + threadIdx.x;
          const uint32_t v = i < P.ntiles ? P.tile[i] : 0u;
          const uint32_t ex = block_exclusive_scan(v, &tot);
          if (i < P.ntiles) P.tile[i] = ex + carry;
          carry += tot;
          __syncthreads();
        }
      }
      LP_SYNC_OR_LEAVE();
      for (int tl = blockIdx.x; tl < P.ntiles; tl += gridDim.x) {
        const int64_t base = (int64_t)tl * kPTile;
        const uint32_t add = P.tile[tl];
        for (int k = threadIdx.x; k < kPTile; k += blockDim.x)
          if (base + k < len) P.start[base + k] += add;
      }
    }
    LP_SYNC_OR_LEAVE();
    for (int s = tid; s < n; s += nth) scatter_body(s, P.key, P.start, P.fill, P.tmp);
    LP_SYNC_OR_LEAVE();
    for (int64_t c = tid; c < P.ncell; c += nth) cell_sort_body(c, P.start, P.tmp, P.ids_in);
    LP_SYNC_OR_LEAVE();
  }
  if (P.rebuild) {
    for (int t = tid; t < n; t += nth) {
      gather_body(t, n, srch ? P.tmp : P.iota, P.src, P.dst, P.nsrc, P.ids_in, P.ids_out,
                  P.colid_in, P.colid_out, P.grids, P.pf);
      // free surface: fixed-point position of the slot this thread just wrote
      if (S.K.free_surface)
        ghost_fix_body(t, S.x, S.y, S.z, S.colid, S.grids, S.K.ghost_grid, S.K.floor_z, S.Xfix);
    }
    LP_SYNC_OR_LEAVE();
    phase_stamp(P, LP_PHASE_SORT);
  }
  if (srch) {
    // every lane of a warp runs the same number of rounds (warp-wide reductions)
    for (int base = 0; base < n; base += nth) {
      const int s = base + tid;
      if (skin) {
        if (s < n) {  // positions of this search, for the displacement test
          P.xref[s] = S.x[s];
          P.xref[n + s] = S.y[s];
          P.xref[2 * n + s] = S.z[s];
        }
        neighbors_body<false, true>(s, s < n, n, S.x, S.y, S.z, P.pf, S.colid, P.ids_out,
                                    P.grids, P.start, nullptr, P.rsearch, P.mirror_mode,
                                    P.floor_z, P.capc, P.cand, P.ccnt, S.dg, false);
      } else {
        neighbors_body<false, true>(s, s < n, n, S.x, S.y, S.z, P.pf, S.colid, P.ids_out,
                                    P.grids, P.start, nullptr, P.radius, P.mirror_mode,
                                    P.floor_z, P.cap, P.nbr, P.cnt, S.dg);
      }
    }
  }
  // the filter of particle s reads only the candidate list that this thread
  // wrote for it above (same particle-to-thread map): no barrier needed
  if (P.rebuild && skin) {
    if (tid == 0) *P.search = 0;
    for (int base = 0; base < n; base += nth) {
      const int s = base + tid;
      filter_body<true>(s, s < n, n, S.x, S.y, S.z, P.pf, P.cand, P.ccnt, P.capc, P.grids,
                        S.colid, P.radius, P.floor_z, P.cap, P.nbr, P.cnt, S.dg);
    }
  }
  // ghosts complete the stencils this thread just built (positions of all
  // particles were fixed before the last barrier)
  if (P.rebuild && S.K.free_surface) {
    for (int base = 0; base < n; base += nth) {
      const int s = base + tid;
      ghost_body(s, s < n, n, S.z, S.Xfix, P.nbr, P.cnt, S.gcnt, S.K, S.dg);
    }
  }
  if (P.phase_ns) {  // profiling: close the neighbour phase (same branch in every block)
    LP_SYNC_OR_LEAVE();
    phase_stamp(P, LP_PHASE_NEIGHBORS);
  }
  if (tid == 0) *S.fb_count = 0;
  if (P.save_y0) {  // Heun's method: the state at the start of the step
    const double* src[7] = {S.x, S.y, S.z, S.u, S.v, S.w, S.V};
    for (int s = tid; s < n; s += nth)
#pragma unroll
      for (int f = 0; f < 7; ++f) P.y0[f][s] = src[f][s];
  }
  if (PREC == LP_MIXED_FF)
    for (int s = tid; s < n; s += nth) split_state_body(S, s);
  LP_SYNC_OR_LEAVE();
  if (PREC == LP_MIXED_FF) {
    for (int s = tid; s < n; s += nth) {
      if (S.K.free_surface) gram_twins_body<true>(S, s);  // read back by the same thread
      gram_ff_body<true>(S, s);
    }
    LP_SYNC_OR_LEAVE();
  }
  for (int s = tid; s < n; s += nth) pass1_body<PREC, true>(S, s);
  LP_SYNC_OR_LEAVE();
  const int nfb = min(*S.fb_count, S.fb_cap);
  for (int t = tid; t < nfb; t += nth) pass1_fallback_item(S, t);
  if (tid == 0 && nfb > 0) atomicAdd(&S.dg->n_fallback, (unsigned long long)nfb);
  LP_SYNC_OR_LEAVE();
  phase_stamp(P, LP_PHASE_PASS1);
  if (PREC == LP_MIXED_FF) {
    for (int s = tid; s < n; s += nth) split_p1_body(S, s);
    LP_SYNC_OR_LEAVE();
  }
  for (int t = tid; t < nfb; t += nth) pass2_fallback_item(S, t);
  LP_SYNC_OR_LEAVE();
  for (int base = 0; base < n; base += nth) {
    const int s = base + tid;
    if (PREC == LP_MIXED_FF && S.K.free_surface && s < n) pass2_twins_body<true>(S, s);
    pass2_body<PREC, true>(S, s, s < n);
  }
  if (P.phase_ns) {  // profiling: close pass 2
    LP_SYNC_OR_LEAVE();
    phase_stamp(P, LP_PHASE_PASS2);
  }
}

// Largest co-resident grid for the persistent kernel (cached per precision).
template <int PREC>
int blocks_of() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_step_persistent<PREC>, kBlock, 0);
  return per > 0 ? per * sms : 0;
}

int persistent_blocks(int prec) {
  static int cached[3] = {0, 0, 0};
  const int k = prec < 0 || prec > 2 ? 0 : prec;
  if (!cached[k])
    cached[k] = prec == LP_FP64 ? blocks_of<LP_FP64>()
                                : (prec == LP_MIXED ? blocks_of<LP_MIXED>() : blocks_of<LP_MIXED_FF>());
  return cached[k];
}

cudaError_t launch_persistent(int prec, const PersistArgs& P, cudaStream_t st) {
  const int nb = persistent_blocks(prec);
  if (nb <= 0) return cudaErrorLaunchFailure;
  void* args[] = {(void*)&P};
  void* fn = prec == LP_FP64 ? (void*)k_step_persistent<LP_FP64>
             : prec == LP_MIXED ? (void*)k_step_persistent<LP_MIXED>
                                : (void*)k_step_persistent<LP_MIXED_FF>;
  return cudaLaunchCooperativeKernel(fn, dim3(nb), dim3(kBlock), args, 0, st);
}

}  // namespace lp
