// The split kernel structure (fv_launch.mode = FV_SPLIT): the stage computed
// the way the paper's solver organises it (Sec. 3.4) -- separate limiter and
// flux kernels per axis, a source kernel, a right-hand-side kernel and an
// update kernel -- each a grid-stride loop whose grid (the paper's gang
// count) and CTA size (its vector length) are launch parameters.  Face
// states, face fluxes and the residual go through device memory between the
// kernels.  The arithmetic per face and per cell is that of the fused kernel
// (same MUSCL, primitive-conversion and Roe routines), without its carried
// stencil differences; the update follows Eq. (4) as L = -R / |Omega|.
#include "fv_stage.cuh"

namespace fvk {
namespace {

static_assert(kSplitMaxThreads == 512, "split kernels: up to 128 registers per thread");

__device__ __forceinline__ long long first_item() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long item_stride() { return (long long)gridDim.x * blockDim.x; }

// (rho, m, E) -> (rho, u, p) of one cell, in the order of box_to_primitive.
template <int DIM>
__device__ __forceinline__ void cell_to_primitive(double (&w)[DIM + 2], double g1) {
  const double r = rcp_fp64(w[0]);
  double k = 0.0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    const double m = w[1 + d];
    const double u = m * r;
    k = (d == 0) ? m * u : fma(m, u, k);
    w[1 + d] = u;
  }
  w[DIM + 1] = g1 * fma(-0.5, k, w[DIM + 1]);
}

// Limiter kernel of axis D: the MUSCL face states of Eq. (6) of every face
// normal to D from the four cells m-2..m+1 along D (ghosts by index map).
template <int DIM, int D, int LIM>
__global__ void __launch_bounds__(kSplitMaxThreads) limiter_kernel(const SplitArgs a) {
  constexpr int NV = DIM + 2;
  const int fe0 = a.n[0] + (D == 0), fe1 = a.n[1] + (D == 1);
  const long long nf = a.nface[D], N = a.ncells;
  for (long long f = first_item(); f < nf; f += item_stride()) {
    int c3[3];
    c3[0] = (int)(f % fe0);
    const long long r = f / fe0;
    c3[1] = (int)(r % fe1);
    c3[2] = (int)(r / fe1);
    const int m = c3[D];
    double q[4][NV];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      int cc[3] = {c3[0], c3[1], c3[2]};
      cc[D] = ghost_source(m - 2 + t, a.n[D], a.bc[D][0], a.bc[D][1]);
      const long long idx = ((long long)cc[2] * a.n[1] + cc[1]) * a.n[0] + cc[0];
#pragma unroll
      for (int v = 0; v < NV; ++v) q[t][v] = a.Us[v * N + idx];
      if (a.recon == FV_RECON_PRIMITIVE) cell_to_primitive<DIM>(q[t], a.g1);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double QL, QR;
      muscl_states<LIM>(q[0][v], q[1][v], q[2][v], q[3][v], a.half_eps, a.cL, a.cR, QL, QR);
      a.QL[D][v * nf + f] = QL;
      a.QR[D][v * nf + f] = QR;
    }
  }
}

// Flux kernel of axis D: the Roe flux at every face normal to D.
template <int DIM, int D>
__global__ void __launch_bounds__(kSplitMaxThreads) flux_kernel(const SplitArgs a) {
  constexpr int NV = DIM + 2, NT = DIM - 1, E = NV - 1;
  const long long nf = a.nface[D];
  for (long long f = first_item(); f < nf; f += item_stride()) {
    double QL[NV], QR[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      QL[v] = a.QL[D][v * nf + f];
      QR[v] = a.QR[D][v * nf + f];
    }
    if (a.recon == FV_RECON_PRIMITIVE) {
      to_conserved<DIM>(QL, a.inv_g1);
      to_conserved<DIM>(QR, a.inv_g1);
    }
    // normal-first ordering: (rho, m_D, tangential momenta, E)
    double qL[NV], qR[NV], G[NV];
    qL[0] = QL[0];
    qR[0] = QR[0];
    qL[1] = QL[1 + D];
    qR[1] = QR[1 + D];
    int t = 0;
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
      if (ax == D) continue;
      qL[2 + t] = QL[1 + ax];
      qR[2 + t] = QR[1 + ax];
      ++t;
    }
    qL[E] = QL[E];
    qR[E] = QR[E];
    roe_F<NT>(qL, qR, a.g1, a.efix, a.inv2efix, G);
    double *F = a.F[D];
    F[f] = G[0];
    F[(1 + D) * nf + f] = G[1];
    t = 0;
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
      if (ax == D) continue;
      F[(1 + ax) * nf + f] = G[2 + t];
      ++t;
    }
    F[E * nf + f] = G[E];
  }
}

// Source kernel: R = -|Omega| S (0 without a source).
template <int DIM>
__global__ void __launch_bounds__(kSplitMaxThreads) source_kernel(const SplitArgs a) {
  constexpr int NV = DIM + 2;
  const long long N = a.ncells;
  const double src = -a.vol;
  for (long long c = first_item(); c < N; c += item_stride()) {
#pragma unroll
    for (int v = 0; v < NV; ++v) a.R[v * N + c] = a.S ? src * a.S[v * N + c] : 0.0;
  }
}

// Right-hand-side kernel: R += sum_d ds_d (F_{m+1/2} - F_{m-1/2}) per cell,
// axes in order; optional per-CTA sums of R_v^2 (lanes, then warps).
template <int DIM>
__global__ void __launch_bounds__(kSplitMaxThreads) rhs_kernel(const SplitArgs a) {
  constexpr int NV = DIM + 2;
  const long long N = a.ncells;
  double nrm[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) nrm[v] = 0.0;
  for (long long c = first_item(); c < N; c += item_stride()) {
    const int i = (int)(c % a.n[0]);
    const long long rr = c / a.n[0];
    const int j = (int)(rr % a.n[1]);
    const int k = (int)(rr / a.n[1]);
    long long flo[DIM], fst[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const long long fe0 = a.n[0] + (d == 0), fe1 = a.n[1] + (d == 1);
      flo[d] = ((long long)k * fe1 + j) * fe0 + i;
      fst[d] = (d == 0) ? 1 : ((d == 1) ? fe0 : fe0 * fe1);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double r = a.R[v * N + c];
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const double *F = a.F[d] + v * a.nface[d];
        r = fma(a.ds[d], F[flo[d] + fst[d]] - F[flo[d]], r);
      }
      a.R[v * N + c] = r;
      if (a.norm_part) nrm[v] = fma(r, r, nrm[v]);
    }
  }
  if (a.norm_part) {
    __shared__ double red[NV][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double sum = nrm[v];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, off);
      if (lane == 0) red[v][warp] = sum;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
      double sum = 0.0;
      const int nw = (blockDim.x + 31) >> 5;
      for (int q = 0; q < nw; ++q) sum += red[threadIdx.x][q];
      a.norm_part[(long long)blockIdx.x * NV + threadIdx.x] = sum;
    }
  }
}

// Update kernel: the SSP-RK3 stage of Eq. (4) with L = -R / |Omega|:
// Us + dt L (stage 1), 3/4 Un + 1/4 (Us + dt L) (2), 1/3 Un + 2/3 (Us + dt L) (3).
template <int DIM, int MODE>
__global__ void __launch_bounds__(kSplitMaxThreads) update_kernel(const SplitArgs a) {
  constexpr int NV = DIM + 2;
  __shared__ double s_dt;
  if (threadIdx.x == 0) s_dt = a.smax ? a.cfl / __longlong_as_double((long long)*a.smax) : a.dt_fixed;
  __syncthreads();
  const double dt = s_dt;
  const long long N = a.ncells;
  for (long long c = first_item(); c < N; c += item_stride()) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const long long e = v * N + c;
      const double s = fma(dt, -a.R[e] * a.inv_vol, a.Us[e]);
      double u;
      if (MODE == MODE_STAGE1)
        u = s;
      else if (MODE == MODE_STAGE2)
        u = fma(0.75, a.Un[e], 0.25 * s);
      else
        u = fma(1.0 / 3.0, a.Un[e], (2.0 / 3.0) * s);
      a.out[e] = u;
    }
  }
  if (MODE == MODE_STAGE3 && a.t_acc && blockIdx.x == 0 && threadIdx.x == 0) *a.t_acc += dt;
}

// CTAs of a grid-stride launch over `items`: the requested count, or enough
// for one item per thread.
unsigned blocks_for(long long items, int grid, int threads) {
  long long b = grid > 0 ? grid : (items + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 0x7fffffffLL) b = 0x7fffffffLL;
  return (unsigned)b;
}

template <int DIM, int LIM>
cudaError_t launch_limiters(const SplitArgs &a, const int *grid, const int *threads, cudaStream_t st) {
  limiter_kernel<DIM, 0, LIM><<<blocks_for(a.nface[0], grid[FV_SK_LIMITER], threads[FV_SK_LIMITER]),
                                threads[FV_SK_LIMITER], 0, st>>>(a);
  limiter_kernel<DIM, 1, LIM><<<blocks_for(a.nface[1], grid[FV_SK_LIMITER + 1], threads[FV_SK_LIMITER + 1]),
                                threads[FV_SK_LIMITER + 1], 0, st>>>(a);
  if constexpr (DIM == 3)
    limiter_kernel<DIM, 2, LIM><<<blocks_for(a.nface[2], grid[FV_SK_LIMITER + 2], threads[FV_SK_LIMITER + 2]),
                                  threads[FV_SK_LIMITER + 2], 0, st>>>(a);
  return cudaGetLastError();
}

template <int DIM>
cudaError_t launch_split_dim(int mode, const SplitArgs &a, const int *grid, const int *threads, int *rhs_blocks,
                             cudaStream_t st) {
  cudaError_t e;
  if (a.limiter == FV_LIM_VANLEER)
    e = launch_limiters<DIM, FV_LIM_VANLEER>(a, grid, threads, st);
  else if (a.limiter == FV_LIM_NONE)
    e = launch_limiters<DIM, FV_LIM_NONE>(a, grid, threads, st);
  else
    e = launch_limiters<DIM, FV_LIM_MINMOD>(a, grid, threads, st);
  if (e != cudaSuccess) return e;
  flux_kernel<DIM, 0><<<blocks_for(a.nface[0], grid[FV_SK_FLUX], threads[FV_SK_FLUX]), threads[FV_SK_FLUX], 0,
                        st>>>(a);
  flux_kernel<DIM, 1><<<blocks_for(a.nface[1], grid[FV_SK_FLUX + 1], threads[FV_SK_FLUX + 1]),
                        threads[FV_SK_FLUX + 1], 0, st>>>(a);
  if constexpr (DIM == 3)
    flux_kernel<DIM, 2><<<blocks_for(a.nface[2], grid[FV_SK_FLUX + 2], threads[FV_SK_FLUX + 2]),
                          threads[FV_SK_FLUX + 2], 0, st>>>(a);
  source_kernel<DIM><<<blocks_for(a.ncells, grid[FV_SK_SOURCE], threads[FV_SK_SOURCE]), threads[FV_SK_SOURCE], 0,
                       st>>>(a);
  const unsigned rb = blocks_for(a.ncells, grid[FV_SK_RHS], threads[FV_SK_RHS]);
  *rhs_blocks = (int)rb;
  rhs_kernel<DIM><<<rb, threads[FV_SK_RHS], 0, st>>>(a);
  if (mode != MODE_RESIDUAL) {
    const unsigned ub = blocks_for(a.ncells, grid[FV_SK_UPDATE], threads[FV_SK_UPDATE]);
    const int ut = threads[FV_SK_UPDATE];
    if (mode == MODE_STAGE1)
      update_kernel<DIM, MODE_STAGE1><<<ub, ut, 0, st>>>(a);
    else if (mode == MODE_STAGE2)
      update_kernel<DIM, MODE_STAGE2><<<ub, ut, 0, st>>>(a);
    else
      update_kernel<DIM, MODE_STAGE3><<<ub, ut, 0, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_split(int mode, const SplitArgs &a, const int *grid, const int *threads, int *rhs_blocks,
                         cudaStream_t st) {
  return a.dim == 2 ? launch_split_dim<2>(mode, a, grid, threads, rhs_blocks, st)
                    : launch_split_dim<3>(mode, a, grid, threads, rhs_blocks, st);
}

}  // namespace fvk
