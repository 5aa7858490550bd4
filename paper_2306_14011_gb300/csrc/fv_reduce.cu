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
cudaError_t launch_stage_3d(int, const CUtensorMap *, const StageArgs &, int, cudaStream_t);
cudaError_t set_stage_attributes_2d(size_t);
cudaError_t set_stage_attributes_3d(size_t);

cudaError_t launch_stage(int dim, int mode, const CUtensorMap *tmap, const StageArgs &a, int threads,
                         cudaStream_t st) {
  if (dim == 2) return launch_stage_2d(mode, tmap, a, threads, st);
  return a.march ? launch_march(mode, tmap, a, threads, st) : launch_stage_3d(mode, tmap, a, threads, st);
}

cudaError_t stage_kernel_attributes(int dim, size_t smem) {
  if (dim == 2) return set_stage_attributes_2d(smem);
  const cudaError_t e = set_stage_attributes_3d(smem);
  return e == cudaSuccess ? set_march_attributes(smem) : e;
}

// ---- FP32 pre-selection for the time-step reduction.
//
// FP64 -> FP32 on the integer pipe by truncating the mantissa: relative error
// below 2^-23 for |x| in the FP32 normal range; smaller values flush to
// (signed) zero, larger ones and NaN become infinite.
__device__ __forceinline__ float f32_trunc(double x) {
  const unsigned long long b = (unsigned long long)dbits(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  const unsigned sign = hi & 0x80000000u;
  unsigned f = sign | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  f = e <= 0 ? sign : f;
  f = e >= 255 ? (sign | 0x7f800000u) : f;
  return __uint_as_float(f);
}

// The wave-speed sum of cell c evaluated in FP32 (round-to-nearest operations
// that are never contracted), and a certified relative error bound rel of it.
// Returns false when no bound is certified.  Certification needs rho, E in
// [2^-30, 2^30] and |m_d| <= 2^30 (no FP32 overflow or underflow on the way)
// and a pressure p = (gamma-1)(E - k) free of strong cancellation,
// kappa = (E + k)/(E - k) <= 1024.  A first-order bound of the FP32 error is
// then (6 kappa + 11) 2^-24 (conversions 2^-23 each, every operation 2^-24,
// the relative error of E - k amplified by kappa); rel = (16 kappa32 + 32)
// 2^-24 exceeds twice that, kappa32 being kappa evaluated in FP32 (within
// 0.1% of it when kappa <= 1024).
template <int DIM>
__device__ __forceinline__ bool wave_sum32(const DtArgs &a, long long c, float &s32, float &rel) {
  constexpr int NV = DIM + 2;
  const long long N = a.ncells;
  const float rho = f32_trunc(a.U[c]);
  const float E = f32_trunc(a.U[(NV - 1) * N + c]);
  bool ok = rho >= 0x1p-30f && rho <= 0x1p30f && E >= 0x1p-30f && E <= 0x1p30f;
  const float r = __frcp_rn(rho);
  float u[DIM];
  float k = 0.0f;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const float m = f32_trunc(a.U[(1 + d) * N + c]);
    ok = ok && fabsf(m) <= 0x1p30f;
    u[d] = __fmul_rn(m, r);
    k = __fadd_rn(k, __fmul_rn(m, u[d]));
  }
  k = 0.5f * k;
  const float em = __fsub_rn(E, k), ep = __fadd_rn(E, k);
  ok = ok && em > 0.0f && ep <= __fmul_rn(1024.0f, em);
  const float c2 = __fmul_rn(__fmul_rn(a.gammaf, __fmul_rn(a.g1f, em)), r);
  const float cs = __fsqrt_rn(c2);
  float s = 0.0f;
#pragma unroll
  for (int d = 0; d < DIM; ++d) s = __fadd_rn(s, __fmul_rn(__fadd_rn(fabsf(u[d]), cs), a.inv_hf[d]));
  s32 = s;
  rel = __fmaf_ru(__fmul_ru(16.0f, __fmul_ru(ep, __frcp_ru(em))), 0x1p-24f, 32.0f * 0x1p-24f);
  return ok;
}

// Pass 1: the largest certified lower bound s32 (1 - rel), rounded down, over
// all cells (atomicMax on the bits of a non-negative float).
template <int DIM>
__global__ void __launch_bounds__(1024) dt_bound_kernel(const DtArgs a) {
  const long long N = a.ncells;
  unsigned best = 0u;
#pragma unroll 4
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    float s32, rel;
    if (wave_sum32<DIM>(a, c, s32, rel)) {
      const unsigned lo = __float_as_uint(__fmul_rd(s32, __fsub_rd(1.0f, rel)));
      best = lo > best ? lo : best;
    }
  }
  best = __reduce_max_sync(0xffffffffu, best);
  __shared__ unsigned wmax[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
// cell whose certified upper bound s32 (1 + rel) (rounded up) is below the
// certified lower bound L of pass 1 cannot hold the maximum and is skipped;
// uncertified cells are always evaluated.  The cell attaining the maximum is
// never skipped (its upper bound is at least its sum, which is at least L),
// so the result is the exact FP64 maximum.
template <int DIM>
__global__ void __launch_bounds__(1024) dt_kernel(const DtArgs a) {
  constexpr int NV = DIM + 2;
  const long long N = a.ncells;
  const float L = a.bounded ? __uint_as_float(*a.lbound) : 0.0f;
  unsigned long long best = 0ull;
  bool bad = false;
#pragma unroll 4
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    if (a.bounded) {
      float s32, rel;
      if (wave_sum32<DIM>(a, c, s32, rel) && __fmul_ru(s32, __fadd_ru(1.0f, rel)) < L) continue;
    }
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
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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

cudaError_t launch_debug_math(const double *x, double *o1, double *o2, long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  debug_math_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, o1, o2, n);
  return cudaGetLastError();
}

}  // namespace fvk
