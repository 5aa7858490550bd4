// Grid reductions of libfv: the CFL time step and the residual norms, plus
// the device-arithmetic diagnostic.
#include "fv_device.cuh"
#include "fv_internal.h"
#include "fv_stage.cuh"

namespace fvk {

size_t stage_smem_bytes(int dim, const int tile[3]) {
  const TileGeom G = tile_geom(dim, tile);
  const int nv = dim + 2;
  return 128 + sizeof(double) * (size_t)nv * (G.plane + G.fmax + G.cells) + 16;
}

cudaError_t launch_stage_2d(int, const CUtensorMap *, const StageArgs &, int, cudaStream_t);
cudaError_t launch_stage_2d_wide(int, const CUtensorMap *, const StageArgs &, int, cudaStream_t);
cudaError_t launch_stage_3d(int, const CUtensorMap *, const StageArgs &, int, cudaStream_t);
cudaError_t set_stage_attributes_2d(size_t);
cudaError_t set_stage_attributes_2d_wide(size_t);
cudaError_t set_stage_attributes_3d(size_t);

cudaError_t launch_stage(int dim, int mode, const CUtensorMap *tmap, const StageArgs &a, int threads,
                         cudaStream_t st) {
  if (dim == 2)
    return threads > kStage2dMaxThreads ? launch_stage_2d_wide(mode, tmap, a, threads, st)
                                        : launch_stage_2d(mode, tmap, a, threads, st);
  return a.march ? launch_march(mode, tmap, a, threads, st) : launch_stage_3d(mode, tmap, a, threads, st);
}

cudaError_t stage_kernel_attributes(int dim, size_t smem) {
  if (dim == 2) {
    const cudaError_t e = set_stage_attributes_2d(smem);
    return e == cudaSuccess ? set_stage_attributes_2d_wide(smem) : e;
  }
  const cudaError_t e = set_stage_attributes_3d(smem);
  return e == cudaSuccess ? set_march_attributes(smem) : e;
}

// Cells are handled in chunks of 32 consecutive cells, one warp per chunk
// (the same chunks in both passes, whatever the launch shape).
constexpr int kDtChunk = 32;

// Pass 1: the largest certified lower bound s32 (1 - rel), rounded down, over
// all cells (atomicMax on the bits of a non-negative float), and per chunk the
// largest certified upper bound s32 (1 + rel), rounded up (+inf when a cell of
// the chunk is not certified).
template <int DIM>
__global__ void __launch_bounds__(1024) dt_bound_kernel(const DtArgs a) {
  const long long N = a.ncells;
  const long long nchunk = (N + kDtChunk - 1) / kDtChunk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long wstride = (long long)gridDim.x * (blockDim.x >> 5);
  unsigned best = 0u;
  for (long long ch = (long long)blockIdx.x * (blockDim.x >> 5) + warp; ch < nchunk; ch += wstride) {
    const long long c = ch * kDtChunk + lane;
    unsigned hi = 0u;
    if (c < N) {
      float s32, rel;
      if (wave_sum32<DIM>(a.U, N, c, a.g1f, a.gammaf, a.inv_hf, s32, rel)) {
        const unsigned lo = __float_as_uint(__fmul_rd(s32, __fsub_rd(1.0f, rel)));
        best = lo > best ? lo : best;
        hi = __float_as_uint(__fmul_ru(s32, __fadd_ru(1.0f, rel)));
      } else {
        hi = 0x7f800000u;  // +inf: the chunk must be evaluated
      }
    }
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) a.chunk_hi[ch] = hi;
  }
  best = __reduce_max_sync(0xffffffffu, best);
  __shared__ unsigned wmax[32];
  if (lane == 0) wmax[warp] = best;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    const unsigned m = __reduce_max_sync(0xffffffffu, lane < nw ? wmax[lane] : 0u);
    if (lane == 0) atomicMax(a.lbound, m);
  }
}

// Pass 2 (the whole reduction when a.bounded = 0): maximum over cells of
// sum_d (|u_d| + c) / dx_d, c = sqrt(gamma p / rho), in FP64, reduced exactly
// (max of non-negative doubles = max of their bit patterns): per thread, warp
// shuffle, CTA, then one atomicMax per CTA.  Cells with rho <= 0, p <= 0 or
// NaN raise FLAG_NONPHYSICAL and are left out.  With the pre-selection, a
// chunk whose certified upper bound is below the certified lower bound L of
// pass 1 cannot hold the maximum and is skipped without reading it; chunks
// with an uncertified cell are always evaluated.  The chunk holding the
// maximum is never skipped (its upper bound is at least the maximum, which
// is at least L), so the result is the exact FP64 maximum.
template <int DIM>
__global__ void __launch_bounds__(1024) dt_kernel(const DtArgs a) {
  constexpr int NV = DIM + 2;
  const long long N = a.ncells;
  const long long nchunk = (N + kDtChunk - 1) / kDtChunk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long wstride = (long long)gridDim.x * (blockDim.x >> 5);
  const unsigned L = a.bounded ? *a.lbound : 0u;
  unsigned long long best = 0ull;
  bool bad = false;
  for (long long ch = (long long)blockIdx.x * (blockDim.x >> 5) + warp; ch < nchunk; ch += wstride) {
    if (a.bounded && a.chunk_hi[ch] < L) continue;  // non-negative float bits order like the values
    const long long c = ch * kDtChunk + lane;
    if (c >= N) continue;
    const double rho = a.U[c];
    if (not_positive_finite(rho)) {
      bad = true;
      continue;
    }
    const double tr = rsqrt_fp64(rho);
    const double r = tr * tr;
    double u[DIM];
    double k = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const double m = a.U[(1 + d) * N + c];
      u[d] = m * r;
      k = (d == 0) ? m * u[d] : fma(m, u[d], k);
    }
    const double p = a.g1 * fma(-0.5, k, a.U[(NV - 1) * N + c]);
    if (not_positive_finite(p)) {
      bad = true;
      continue;
    }
    const double c2 = (a.gamma * p) * r;
    const double cs = c2 * rsqrt_fp64(c2);
    double s = (iabs(u[0]) + cs) * a.inv_h[0];
#pragma unroll
    for (int d = 1; d < DIM; ++d) s = fma(iabs(u[d]) + cs, a.inv_h[d], s);
    const unsigned long long sb = (unsigned long long)dbits(s);
    best = sb > best ? sb : best;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off);
    best = o > best ? o : best;
  }
  __shared__ unsigned long long wmax[32];
  if (lane == 0) wmax[warp] = best;
  const int anybad = __syncthreads_or(bad);
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    unsigned long long m = lane < nw ? wmax[lane] : 0ull;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, m, off);
      m = o > m ? o : m;
    }
    if (lane == 0) {
      atomicMax(a.smax, m);
      if (anybad) atomicOr(a.flags, FLAG_NONPHYSICAL);
    }
  }
}

// Failure-path check of the bounded waits: kind 0 waits on an mbarrier that
// no copy completes (the tile-load wait), kind 1 on a word that nothing
// changes (the grid-barrier wait); both give up after limit_ns, raise
// FLAG_TIMEOUT in *flags and return.
__global__ void debug_wait_kernel(int kind, unsigned long long limit_ns, unsigned *word, unsigned *flags) {
  __shared__ __align__(8) uint64_t bar;
  bool ok;
  if (kind == 0) {
    if (threadIdx.x == 0) {
      mbar_init(smem_u32(&bar), 1);
      fence_mbar_init();
    }
    __syncthreads();
    ok = mbar_wait_bounded(smem_u32(&bar), 0u, limit_ns);
  } else {
    ok = spin_while_equal(word, 0u, limit_ns);
  }
  if (!ok && threadIdx.x == 0) atomicOr(flags, FLAG_TIMEOUT);
}

cudaError_t launch_debug_wait(int kind, unsigned long long limit_ns, unsigned *word, unsigned *flags,
                              cudaStream_t st) {
  debug_wait_kernel<<<1, 32, 0, st>>>(kind, limit_ns, word, flags);
  return cudaGetLastError();
}

// Stage 1 from the flux differences dF_d of every axis: the fused stage-1
// kernel's accumulation, with its operands formed as that kernel forms them
// (dt by one division, the axis scales -w dt / dx_d with w = 1, the start
// value U or fma(dt, S, U)) and added in its axis order, so both give the
// same bits.  Elementwise and coalesced; HBM-bound.
template <int DIM>
__global__ void __launch_bounds__(256) stage1_from_fd_kernel(const StageArgs a) {
  constexpr int NV = DIM + 2;
  const long long N = (long long)a.n[0] * a.n[1] * a.n[2];
  const double w = 1.0;
  const double dt = a.smax ? a.cfl / __longlong_as_double((long long)*a.smax) : a.dt_fixed;
  double coef[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) coef[d] = -w * dt * a.inv_h[d];
  const double src = w * dt;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double r = a.Us[v * N + i];
      if (a.S) r = fma(src, a.S[v * N + i], r);
#pragma unroll
      for (int d = 0; d < DIM; ++d) r = fma(coef[d], a.fd[((long long)d * NV + v) * N + i], r);
      a.out[v * N + i] = r;
    }
  }
}

cudaError_t launch_stage1_from_fd(int dim, const StageArgs &a, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long N = (long long)a.n[0] * a.n[1] * a.n[2];
  long long blocks = (N + 255) / 256;
  if (blocks > 8ll * sms) blocks = 8ll * sms;  // 2048 threads per SM, grid-stride beyond
  if (blocks < 1) blocks = 1;
  if (dim == 2)
    stage1_from_fd_kernel<2><<<(unsigned)blocks, 256, 0, st>>>(a);
  else
    stage1_from_fd_kernel<3><<<(unsigned)blocks, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dt(const DtArgs &a, int blocks, int threads, cudaStream_t st) {
  if (a.dim == 2) {
    if (a.bounded) dt_bound_kernel<2><<<blocks, threads, 0, st>>>(a);
    dt_kernel<2><<<blocks, threads, 0, st>>>(a);
  } else {
    if (a.bounded) dt_bound_kernel<3><<<blocks, threads, 0, st>>>(a);
    dt_kernel<3><<<blocks, threads, 0, st>>>(a);
  }
  return cudaGetLastError();
}

// Sum of per-CTA partials, one warp per variable, in a fixed order (strided
// lane sums, then a fixed shuffle tree), so the result is run-to-run exact.
__global__ void norm_finalize_kernel(const double *part, int nparts, int nvar, double *out) {
  const int v = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (v >= nvar) return;
  double s = 0.0;
  for (int q = lane; q < nparts; q += 32) s += part[(long long)q * nvar + v];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) out[v] = s;
}

cudaError_t launch_norm_finalize(const double *part, int nparts, int nvar, double *out, cudaStream_t st) {
  norm_finalize_kernel<<<1, 32 * nvar, 0, st>>>(part, nparts, nvar, out);
  return cudaGetLastError();
}

// dt = cfl / smax on the device (for a device-pointer dt_out).
__global__ void dt_finalize_kernel(const unsigned long long *smax, double cfl, double *out) {
  *out = cfl / __longlong_as_double((long long)*smax);
}

cudaError_t launch_dt_finalize(const unsigned long long *smax, double cfl, double *out, cudaStream_t st) {
  dt_finalize_kernel<<<1, 1, 0, st>>>(smax, cfl, out);
  return cudaGetLastError();
}

__global__ void debug_math_kernel(const double *x, double *o1, double *o2, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    o1[i] = rsqrt_fp64(x[i]);
    o2[i] = rcp_fp64(x[i]);
  }
}

// The integer-pipe helpers on arbitrary inputs: out[i] = op(x[i], y[i]) with
// op 0: half_nonneg(x), 1: scale_pow2<-2>(x), 2: scale_pow2<-1>(x),
// 3: scale_pow2<1>(x), 4: minmod(x, y), 5: iabs(x).
__global__ void debug_bits_kernel(int op, const double *x, const double *y, double *out, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double v = x[i];
    double r;
    switch (op) {
      case 0: r = half_nonneg(v); break;
      case 1: r = scale_pow2<-2>(v); break;
      case 2: r = scale_pow2<-1>(v); break;
      case 3: r = scale_pow2<1>(v); break;
      case 4: r = minmod(v, y[i]); break;
      case 6:
      case 7: {  // the flux kernels' products: on the integer path, else FP64
        bool ok = true;
        r = op == 6 ? pmul<true, false>(v, y[i], ok) : pmul<true, true>(v, y[i], ok);
        if (!ok) r = v * y[i];
        break;
      }
      default: r = iabs(v); break;
    }
    out[i] = r;
  }
}

cudaError_t launch_debug_bits(int op, const double *x, const double *y, double *out, long n, cudaStream_t st) {
  long blocks = (n + 255) / 256;
  if (blocks > 1216) blocks = 1216;
  if (blocks < 1) blocks = 1;
  debug_bits_kernel<<<(unsigned)blocks, 256, 0, st>>>(op, x, y, out, n);
  return cudaGetLastError();
}

// FP64 issue-rate reference: every thread runs 8 independent chains of
// `iters` operations -- kind 0: DFMA, kind 1: DADD, kind 2: products on the
// integer pipe (pmul, the flux kernels' products), kind 3: 4 DFMA chains
// beside 4 integer-pipe product chains -- and out receives one sum per
// thread so nothing is optimised away (NaN if a product left the integer
// path, which the factors near 1 never make it do).
template <int KIND>
__global__ void __launch_bounds__(256) fp64_stream_kernel(double a, double b, int iters, double *out) {
  double x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = a + threadIdx.x * 1e-9 + i;
  bool ok = true;
  // factors just above and below 1 (alternating, selected on the integer
  // pipe), so that product chains stay near their start
  const long long up = __double_as_longlong(1.0000000001234), down = __double_as_longlong(0.9999999998766);
  for (int it = 0; it < iters; ++it) {
    const double f = __longlong_as_double((it & 1) ? down : up);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (KIND == 0 || (KIND == 3 && i < 4))
        x[i] = fma(x[i], a, b);
      else if (KIND == 1)
        x[i] = x[i] + b;
      else
        x[i] = pmul<true>(x[i], f, ok);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  out[(long)blockIdx.x * blockDim.x + threadIdx.x] = ok ? s : __longlong_as_double(0x7ff8000000000000ll);
}

cudaError_t launch_fp64_stream(int kind, int blocks, int iters, double *out, cudaStream_t st) {
  const double a = 1.0000001, b = 1e-7;
  switch (kind) {
    case 0: fp64_stream_kernel<0><<<blocks, 256, 0, st>>>(a, b, iters, out); break;
    case 1: fp64_stream_kernel<1><<<blocks, 256, 0, st>>>(a, b, iters, out); break;
    case 2: fp64_stream_kernel<2><<<blocks, 256, 0, st>>>(a, b, iters, out); break;
    default: fp64_stream_kernel<3><<<blocks, 256, 0, st>>>(a, b, iters, out); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_debug_math(const double *x, double *o1, double *o2, long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  debug_math_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, o1, o2, n);
  return cudaGetLastError();
}

}  // namespace fvk
