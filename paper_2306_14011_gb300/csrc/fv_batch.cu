// Batched grids: many independent 2D problems of different sizes advanced
// together by one persistent, cooperative kernel.
//
// The kernel runs every step of a call: per step, a time-step phase (each
// problem's CFL maximum, reduced exactly with atomicMax on bit patterns) and
// the three SSP-RK3 stage phases.  Within a phase the work items --
// (problem, cell chunk) or (problem, tile) -- are spread round-robin over all
// co-resident CTAs; a grid-wide barrier separates the phases.  Each problem
// keeps its own time step.  Tiles are processed by the same tile_work routine
// as the single-grid stage kernels -- TMA tile loads where the problem's grid
// allows them, plain loads elsewhere -- so every problem's results are
// bitwise those of a single-grid run.
#include "fv_stage.cuh"

namespace fvk {

namespace {

constexpr uint64_t kBarrierWaitNs = 2000000000ull;  // 2 s bound on a grid-barrier wait

// Grid-wide barrier of a cooperative launch: CTA-local barrier, then thread 0
// arrives on a counter; the last arrival resets it and advances the
// generation, the others wait for the generation to move (bounded).
// Returns false in every thread of the CTA if the wait timed out.
__device__ bool grid_barrier(unsigned *count, unsigned *gen, unsigned *flags) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned *vgen = gen;
    const unsigned g = *vgen;
    __threadfence();
    if (atomicAdd(count, 1u) == gridDim.x - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else if (!spin_while_equal(vgen, g, kBarrierWaitNs)) {
      atomicOr(flags, FLAG_TIMEOUT);
      ok = 0;
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Index of the problem whose [begin[p], begin[p+1]) range holds item.
__device__ __forceinline__ int find_problem(const int *begin, int nprob, int item) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (begin[mid] <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// The CTA's mbarrier for TMA tile loads completes one phase per load;
// `phase` is the parity of the next one.
template <int MODE>
__device__ __forceinline__ bool stage_phase(const BatchArgs &b, int slot, double *tile, uint64_t *mbar,
                                            uint32_t &phase, double *s_coef, double (*red)[32]) {
  const double *Us = MODE == MODE_STAGE1 ? b.U : (MODE == MODE_STAGE2 ? b.U1 : b.U2);
  double *out = MODE == MODE_STAGE1 ? b.U1 : (MODE == MODE_STAGE2 ? b.U2 : b.U);
  const int src = MODE == MODE_STAGE1 ? 0 : (MODE == MODE_STAGE2 ? 1 : 2);
  for (int item = blockIdx.x; item < b.total_tiles; item += gridDim.x) {
    const int p = find_problem(b.tile_begin, b.nprob, item);
    const BatchProblem &P = b.prob[p];
    StageArgs a;
    a.Us = Us + P.off;
    a.Un = b.U + P.off;
    a.out = out + P.off;
    a.norm_part = nullptr;
    a.n[0] = P.n[0];
    a.n[1] = P.n[1];
    a.n[2] = 1;
    a.tile[0] = b.tile[0];
    a.tile[1] = b.tile[1];
    a.tile[2] = 1;
    a.ntile[0] = P.ntile[0];
    a.ntile[1] = P.ntile[1];
    a.ntile[2] = 1;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      a.bc[d][0] = P.bc[d][0];
      a.bc[d][1] = P.bc[d][1];
      a.ds[d] = 0.0;
      a.inv_h[d] = d < 2 ? P.inv_h[d] : 0.0;
    }
    const CUtensorMap *map = b.tmaps ? b.tmaps + (size_t)src * b.nprob + p : nullptr;
    a.use_tma = (map && b.tma_ok[(size_t)src * b.nprob + p]) ? 1 : 0;
    a.limiter = FV_LIM_MINMOD;
    a.recon = FV_RECON_CONSERVED;
    a.cL = a.cR = 0.0;
    a.g1 = b.g1;
    a.half_eps = b.half_eps;
    a.efix = b.efix;
    a.inv2efix = b.inv2efix;
    a.smax = b.dt_fixed > 0.0 ? nullptr : b.smax + (long long)slot * b.nprob + p;
    a.cfl = b.cfl;
    a.dt_fixed = b.dt_fixed;
    a.t_acc = nullptr;
    a.flags = b.flags;
    a.S = nullptr;
    a.vol = 0.0;
    const int local = item - b.tile_begin[p];
    if (!tile_work<2, MODE>(map, a, local % P.ntile[0], local / P.ntile[0], 0, tile, mbar, phase, s_coef, red))
      return false;  // a tile load timed out (flagged); the other CTAs' barrier waits run out
    if (a.use_tma) phase ^= 1u;
    // the next item reuses the shared buffers: this item's generic-proxy
    // accesses of the tile box are ordered before the next TMA write to it
    fence_proxy_async_smem();
    __syncthreads();
  }
  return grid_barrier(b.bar_count, b.bar_gen, b.flags);
}

// Per problem, the largest certified FP32 lower bound of the wave-speed sum
// (as in dt_bound_kernel), for problems where the pre-selection applies, and
// per 32-cell chunk (one warp) of each item the largest certified upper
// bound (+inf when a cell of the chunk is not certified).
__device__ __forceinline__ void dt_bound_phase(const BatchArgs &b, int slot) {
  __shared__ unsigned wmax[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int per_item = (int)(b.chunk_cells / 32);
  for (int item = blockIdx.x; item < b.total_chunks; item += gridDim.x) {
    const int p = find_problem(b.chunk_begin, b.nprob, item);
    const BatchProblem &P = b.prob[p];
    if (!P.bounded) continue;  // uniform over the CTA
    const long long N = (long long)P.n[0] * P.n[1];
    const long long c0 = (long long)(item - b.chunk_begin[p]) * b.chunk_cells;
    const long long c1 = c0 + b.chunk_cells < N ? c0 + b.chunk_cells : N;
    const int nsub = (int)((c1 - c0 + 31) / 32);
    const double *U = b.U + P.off;
    unsigned best = 0u;
    for (int q = warp; q < nsub; q += nw) {
      const long long c = c0 + (long long)q * 32 + lane;
      unsigned hi = 0u;
      if (c < c1) {
        float s32, rel;
        if (wave_sum32<2>(U, N, c, b.g1f, b.gammaf, P.inv_hf, s32, rel)) {
          const unsigned lo = __float_as_uint(__fmul_rd(s32, __fsub_rd(1.0f, rel)));
          best = lo > best ? lo : best;
          hi = __float_as_uint(__fmul_ru(s32, __fadd_ru(1.0f, rel)));
        } else {
          hi = 0x7f800000u;  // +inf: the chunk must be evaluated
        }
      }
      hi = __reduce_max_sync(0xffffffffu, hi);
      if (lane == 0) b.chunk_hi[(long long)item * per_item + q] = hi;
    }
    best = __reduce_max_sync(0xffffffffu, best);
    if (lane == 0) wmax[warp] = best;
    __syncthreads();
    if (warp == 0) {
      const unsigned m = __reduce_max_sync(0xffffffffu, lane < nw ? wmax[lane] : 0u);
      if (lane == 0) atomicMax(b.lbound + (long long)slot * b.nprob + p, m);
    }
    __syncthreads();
  }
}

// Per problem max over its cells of sum_d (|u_d| + c) / dx_d (as in dt_kernel:
// a 32-cell chunk whose certified FP32 upper bound is below the problem's
// certified lower bound cannot hold the maximum and is skipped without
// reading it; every other cell is evaluated in FP64).
__device__ __forceinline__ void dt_phase(const BatchArgs &b, int slot) {
  __shared__ unsigned long long wmax[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int per_item = (int)(b.chunk_cells / 32);
  for (int item = blockIdx.x; item < b.total_chunks; item += gridDim.x) {
    const int p = find_problem(b.chunk_begin, b.nprob, item);
    const BatchProblem &P = b.prob[p];
    const long long N = (long long)P.n[0] * P.n[1];
    const long long c0 = (long long)(item - b.chunk_begin[p]) * b.chunk_cells;
    const long long c1 = c0 + b.chunk_cells < N ? c0 + b.chunk_cells : N;
    const int nsub = (int)((c1 - c0 + 31) / 32);
    const double *U = b.U + P.off;
    const unsigned L = P.bounded ? b.lbound[(long long)slot * b.nprob + p] : 0u;
    unsigned long long best = 0ull;
    bool bad = false;
    for (int q = warp; q < nsub; q += nw) {
      // non-negative float bits order like the values
      if (P.bounded && b.chunk_hi[(long long)item * per_item + q] < L) continue;
      const long long c = c0 + (long long)q * 32 + lane;
      if (c >= c1) continue;
      const double rho = U[c];
      if (not_positive_finite(rho)) {
        bad = true;
        continue;
      }
      const double tr = rsqrt_fp64(rho);
      const double r = tr * tr;
      const double m0 = U[N + c], m1 = U[2 * N + c];
      const double u0 = m0 * r, u1 = m1 * r;
      const double k = fma(m1, u1, m0 * u0);
      const double pr = b.g1 * fma(-0.5, k, U[3 * N + c]);
      if (not_positive_finite(pr)) {
        bad = true;
        continue;
      }
      const double c2 = (b.gamma * pr) * r;
      const double cs = c2 * rsqrt_fp64(c2);
      const double s = fma(iabs(u1) + cs, P.inv_h[1], (iabs(u0) + cs) * P.inv_h[0]);
      const unsigned long long sb = (unsigned long long)dbits(s);
      best = sb > best ? sb : best;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off);
      best = o > best ? o : best;
    }
    if (lane == 0) wmax[warp] = best;
    const int anybad = __syncthreads_or(bad);
    if (warp == 0) {
      unsigned long long m = lane < nw ? wmax[lane] : 0ull;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, m, off);
        m = o > m ? o : m;
      }
      if (lane == 0) {
        atomicMax(b.smax + (long long)slot * b.nprob + p, m);
        if (anybad) atomicOr(b.flags, FLAG_NONPHYSICAL);
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256, FV_STAGE_MIN_BLOCKS) batch_run_kernel(const BatchArgs b) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ double s_coef[5];
  __shared__ double red[4][32];
  double *tile = aligned_smem(smem_raw);
  StageArgs ga;  // only the tile shape, for the mbarrier's place after the stage buffers
  ga.tile[0] = b.tile[0];
  ga.tile[1] = b.tile[1];
  ga.tile[2] = 1;
  uint64_t *mbar = stage_mbar<2>(tile, ga);
  uint32_t phase = 0u;
  if (b.tmaps) {
    if (threadIdx.x == 0) {
      mbar_init(smem_u32(mbar), 1);
      fence_mbar_init();
    }
    __syncthreads();
  }
  for (int step = 0; step < b.nsteps; ++step) {
    const int slot = step & 1;
    if (b.dt_fixed <= 0.0) {
      // clear the other slot for the next step (nobody reads it during this step)
      if (blockIdx.x == 0)
        for (int p = threadIdx.x; p < b.nprob; p += blockDim.x) {
          b.smax[(long long)(slot ^ 1) * b.nprob + p] = 0ull;
          b.lbound[(long long)(slot ^ 1) * b.nprob + p] = 0u;
        }
      dt_bound_phase(b, slot);
      if (!grid_barrier(b.bar_count, b.bar_gen, b.flags)) return;
      dt_phase(b, slot);
      if (!grid_barrier(b.bar_count, b.bar_gen, b.flags)) return;
    }
    if (blockIdx.x == 0 && b.t_acc)
      for (int p = threadIdx.x; p < b.nprob; p += blockDim.x)
        b.t_acc[p] += b.dt_fixed > 0.0 ? b.dt_fixed
                                       : b.cfl / __longlong_as_double((long long)b.smax[(long long)slot * b.nprob + p]);
    if (!stage_phase<MODE_STAGE1>(b, slot, tile, mbar, phase, s_coef, red)) return;
    if (!stage_phase<MODE_STAGE2>(b, slot, tile, mbar, phase, s_coef, red)) return;
    if (!stage_phase<MODE_STAGE3>(b, slot, tile, mbar, phase, s_coef, red)) return;
  }
}

}  // namespace

size_t batch_smem_bytes(const int tile[2]) {
  const int t3[3] = {tile[0], tile[1], 1};
  return stage_smem_bytes(2, t3);
}

cudaError_t batch_max_blocks(int threads, size_t smem, int *blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute((const void *)batch_run_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_run_kernel, threads, smem);
}

cudaError_t launch_batch_run(const BatchArgs &b, int blocks, int threads, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_run_kernel, b);
}

}  // namespace fvk
