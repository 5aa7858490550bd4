// z-marching fused residual / SSP-RK3 stage kernel for 3D grids.
//
// One CTA owns an x-y tile of tile[0] x tile[1] cell columns and a chunk of
// tile[2] consecutive z-planes, and walks the chunk plane by plane:
//   * the planes z-2 .. z+1 around the current plane z sit in a ring of four
//     shared-memory slots, each holding one plane of the tile plus its 2-cell
//     x-y halo for all five conserved variables; a slot is refilled by one TMA
//     box (x, y, 1, var) as soon as its plane is dead, so the copy overlaps the
//     current plane's x and y flux work.  A plane outside [0, nz) is fetched
//     from the cell it stands for (periodic wrap or transmissive copy), so no
//     z-ghost fix-up is needed; x-y halo cells outside the domain are
//     patched with plain loads (TMA fills them with zeros);
//   * the z-face flux above each column is computed once and kept in a
//     shared-memory buffer owned by the thread that owns that column, so it
//     serves as the lower face of the next plane (no z-face is evaluated twice
//     inside a chunk);
//   * x and y faces of the current plane go to shared-memory face buffers;
//     after a barrier each column forms R = cx dFx, then + cy dFy, then
//     + cz dFz (the order of the box-tiled kernel, so both give identical
//     bits) and writes the residual or the RK stage combination.
// Per cell the face work is (1 + 1/tile[0]) + (1 + 1/tile[1]) + (1 + 1/tile[2])
// fluxes (3.16 at 16 x 16 columns and 32-plane chunks) against 3.375 for an
// 8 x 8 x 8 box tile, whose depth shared memory bounds; in exchange the CTA
// synchronises twice per plane.  Two 256-thread CTAs fit on an SM.  Stages 2
// and 3 copy U^n of each plane's columns into shared memory asynchronously
// while the plane's faces are evaluated.
#include "fv_stage.cuh"

namespace fvk {

namespace {

constexpr int kRing = 4;
constexpr int NV3 = 5;

struct MarchGeom {
  int BX, BY;  // plane box with halo
  int plane;   // doubles per variable per plane
  int slot;    // doubles per ring slot (the plane of all five variables, padded to 128 bytes)
  int cols;    // tile[0] * tile[1]
  int nfx, nfy;  // x and y faces of a full plane
};

__host__ __device__ inline MarchGeom march_geom(const int tile[3]) {
  MarchGeom g;
  g.BX = tile[0] + 4;
  g.BY = tile[1] + 4;
  g.plane = g.BX * g.BY;
  g.slot = (NV3 * g.plane + 15) & ~15;
  g.cols = tile[0] * tile[1];
  g.nfx = (tile[0] + 1) * tile[1];
  g.nfy = tile[0] * (tile[1] + 1);
  return g;
}

// Plain loads of a whole plane box (interior and x-y halo) of plane zsrc.
__device__ __forceinline__ void load_plane_plain(double *slot, const StageArgs &a, const int o[2], int ext0,
                                                 int ext1, int zsrc, const MarchGeom &G) {
  const long long N = (long long)a.n[0] * a.n[1] * a.n[2];
  const int w = ext0 + 4, h = ext1 + 4;
  for (int q = threadIdx.x; q < w * h; q += blockDim.x) {
    const int lx = q % w, ly = q / w;
    const int gx = ghost_source(o[0] - 2 + lx, a.n[0], a.bc[0][0], a.bc[0][1]);
    const int gy = ghost_source(o[1] - 2 + ly, a.n[1], a.bc[1][0], a.bc[1][1]);
    const long long src = ((long long)zsrc * a.n[1] + gy) * a.n[0] + gx;
    const int dst = ly * G.BX + lx;
#pragma unroll
    for (int v = 0; v < NV3; ++v) slot[v * G.plane + dst] = a.Us[v * N + src];
  }
}

// After a TMA load: patch the x-y halo cells that lie outside the domain
// (the stencil never reads the corners).  Tile-uniform early exit.
__device__ __forceinline__ void fix_plane_halo(double *slot, const StageArgs &a, const int o[2], int ext0, int ext1,
                                               int zsrc, const MarchGeom &G) {
  const long long N = (long long)a.n[0] * a.n[1] * a.n[2];
  bool wrote = false;
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    const int e = d == 0 ? ext0 : ext1, eo = d == 0 ? ext1 : ext0;
    if (o[d] >= 2 && o[d] + e + 2 <= a.n[d]) continue;
    wrote = true;
    for (int q = threadIdx.x; q < 4 * eo; q += blockDim.x) {
      const int layer = q & 3, r = q >> 2;
      const int ld = layer < 2 ? layer : e + layer;  // local coordinate along d
      const int g = o[d] - 2 + ld;
      if (g >= 0 && g < a.n[d]) continue;
      const int gs = ghost_source(g, a.n[d], a.bc[d][0], a.bc[d][1]);
      const int gx = d == 0 ? gs : o[0] + r, gy = d == 0 ? o[1] + r : gs;
      const int lx = d == 0 ? ld : r + 2, ly = d == 0 ? r + 2 : ld;
      const long long src = ((long long)zsrc * a.n[1] + gy) * a.n[0] + gx;
#pragma unroll
      for (int v = 0; v < NV3; ++v) slot[v * G.plane + ly * G.BX + lx] = a.Us[v * N + src];
    }
  }
  if (wrote) fence_proxy_async_smem();  // order these writes before the slot's next TMA refill
}

// One face normal to axis D from the stencil values p[0..3][v] (v stride
// `vs`), written into F (variable stride fs) at index f.  Same arithmetic as
// the box-tiled kernel's face pass.
template <int D, int LIM>
__device__ __forceinline__ void march_face(const double *p0, const double *p1, const double *p2, const double *p3,
                                           int vs, const StageArgs &a, double *F, int fs, int f) {
  double QL[NV3], QR[NV3];
#pragma unroll
  for (int v = 0; v < NV3; ++v)
    muscl_states<LIM>(p0[v * vs], p1[v * vs], p2[v * vs], p3[v * vs], a.half_eps, a.cL, a.cR, QL[v], QR[v]);
  double qL[5], qR[5], Gf[5];
  qL[0] = QL[0];
  qR[0] = QR[0];
  qL[1] = QL[1 + D];
  qR[1] = QR[1 + D];
  int t = 0;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if (ax == D) continue;
    qL[2 + t] = QL[1 + ax];
    qR[2 + t] = QR[1 + ax];
    ++t;
  }
  qL[4] = QL[4];
  qR[4] = QR[4];
  roe_F<2>(qL, qR, a.g1, a.efix, a.inv2efix, Gf);
  F[f] = Gf[0];
  F[(1 + D) * fs + f] = Gf[1];
  t = 0;
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if (ax == D) continue;
    F[(1 + ax) * fs + f] = Gf[2 + t];
    ++t;
  }
  F[4 * fs + f] = Gf[4];
}

// z-faces above the columns this thread owns, between ring planes r and r+1
// (stencil planes r-1 .. r+2), into Fz (variable stride cols).
template <int LIM>
__device__ __forceinline__ void z_faces(const double *ring, int r, const StageArgs &a, int ext0, int ncol,
                                        const MarchGeom &G, double *Fz) {
  const double *s0 = ring + ((r - 1) & 3) * G.slot, *s1 = ring + (r & 3) * G.slot;
  const double *s2 = ring + ((r + 1) & 3) * G.slot, *s3 = ring + ((r + 2) & 3) * G.slot;
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
    const int i = c % ext0, j = c / ext0;
    const int lc = (j + 2) * G.BX + (i + 2);
    march_face<2, LIM>(s0 + lc, s1 + lc, s2 + lc, s3 + lc, G.plane, a, Fz, G.cols, c);
  }
}

// Issue (TMA) or perform (plain loads) the load of ring plane r.
__device__ __forceinline__ void fetch_plane(const CUtensorMap *tmap, double *ring, uint64_t *mbar, int r,
                                            const StageArgs &a, const int o[2], int ext0, int ext1, int z0,
                                            const MarchGeom &G) {
  const int zsrc = ghost_source(z0 - 2 + r, a.n[2], a.bc[2][0], a.bc[2][1]);
  double *slot = ring + (r & 3) * G.slot;
  if (a.use_tma) {
    if (threadIdx.x == 0) {
      const uint32_t bar = smem_u32(mbar + (r & 3));
      mbar_expect_tx(bar, (uint32_t)(NV3 * G.plane * sizeof(double)));
      tma_load_4d(smem_u32(slot), tmap, o[0] - 2, o[1] - 2, zsrc, 0, bar);
    }
  } else {
    load_plane_plain(slot, a, o, ext0, ext1, zsrc, G);
  }
}

// Wait (bounded) for ring plane r's TMA; false on a timeout.
__device__ __forceinline__ bool wait_plane(uint64_t *mbar, int r, const StageArgs &a) {
  if (!a.use_tma) return true;
  return mbar_wait_bounded(smem_u32(mbar + (r & 3)), (uint32_t)((r >> 2) & 1), kTmaWaitNs);
}

// CTA-wide barrier that also reports whether any thread's wait timed out.  On
// a timeout thread 0 raises the flag and waits once more for each copy still
// in flight (ring planes first .. last), so none lands after the CTA exits.
__device__ __forceinline__ bool sync_timed_out(bool ok, uint64_t *mbar, int first, int last, const StageArgs &a) {
  if (!__syncthreads_or(!ok)) return false;
  if (threadIdx.x == 0) {
    atomicOr(a.flags, FLAG_TIMEOUT);
    for (int q = first; q <= last; ++q)
      mbar_wait_bounded(smem_u32(mbar + (q & 3)), (uint32_t)((q >> 2) & 1), kTmaWaitNs);
  }
  return true;
}

template <int MODE, int LIM>
__global__ void __launch_bounds__(256, 2) march_kernel(const __grid_constant__ CUtensorMap tmap, const StageArgs a) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ double s_coef[5];
  __shared__ double red[NV3][32];
  const MarchGeom G = march_geom(a.tile);
  double *ring = aligned_smem(smem_raw);
  double *Fx = ring + kRing * G.slot;
  double *Fy = Fx + NV3 * G.nfx;
  double *Fz0 = Fy + NV3 * G.nfy;
  double *Fz1 = Fz0 + NV3 * G.cols;
  double *Unb = Fz1 + NV3 * G.cols;  // stages 2 and 3: U^n of the current plane's columns
  uint64_t *mbar = reinterpret_cast<uint64_t *>(Unb + NV3 * G.cols);

  const long long tix = a.tile_begin + blockIdx.x;  // linear tile index
  long long b = tix;
  const int bx = (int)(b % a.ntile[0]);
  b /= a.ntile[0];
  const int by = (int)(b % a.ntile[1]);
  const int bz = (int)(b / a.ntile[1]);
  const int o[2] = {bx * a.tile[0], by * a.tile[1]};
  const int ext0 = min(a.tile[0], a.n[0] - o[0]), ext1 = min(a.tile[1], a.n[1] - o[1]);
  const int z0 = bz * a.tile[2];
  const int nzc = min(a.tile[2], a.n[2] - z0);
  const int ncol = ext0 * ext1;
  const long long N = (long long)a.n[0] * a.n[1] * a.n[2];
  const int last = nzc + 3;  // ring planes 0 .. last stand for z0-2 .. z0+nzc+1

  if (threadIdx.x == 0) {
    if (a.use_tma) {
#pragma unroll
      for (int s = 0; s < kRing; ++s) mbar_init(smem_u32(mbar + s), 1);
      fence_mbar_init();
    }
    double dt = 0.0, w = 0.0;
    if (MODE != MODE_RESIDUAL) {
      dt = a.smax ? a.cfl / __longlong_as_double((long long)*a.smax) : a.dt_fixed;
      w = (MODE == MODE_STAGE1) ? 1.0 : ((MODE == MODE_STAGE2) ? 0.25 : 2.0 / 3.0);
    }
    s_coef[0] = dt;
#pragma unroll
    for (int d = 0; d < 3; ++d) s_coef[1 + d] = (MODE == MODE_RESIDUAL) ? a.ds[d] : -w * dt * a.inv_h[d];
    s_coef[4] = (MODE == MODE_RESIDUAL) ? -a.vol : w * dt;
  }
  __syncthreads();
  const double dt = s_coef[0], cx = s_coef[1], cy = s_coef[2], cz = s_coef[3], src = s_coef[4];

  // ---- prologue: planes z0-2 .. z0+1, the z-face below z0, then plane z0+2
  for (int r = 0; r < kRing; ++r) fetch_plane(&tmap, ring, mbar, r, a, o, ext0, ext1, z0, G);
  bool ok = true;
  for (int r = 0; r < kRing; ++r) ok = ok && wait_plane(mbar, r, a);
  if (sync_timed_out(ok, mbar, 0, kRing - 1, a)) return;  // also publishes plain loads
  double *Fzp = Fz0, *Fzc = Fz1;
  z_faces<LIM>(ring, 1, a, ext0, ncol, G, Fzp);
  __syncthreads();  // plane 0 dead
  fetch_plane(&tmap, ring, mbar, kRing, a, o, ext0, ext1, z0, G);
  __syncthreads();

  const bool want_norm = (MODE == MODE_RESIDUAL) && a.norm_part != nullptr;
  double nrm[NV3];
#pragma unroll
  for (int v = 0; v < NV3; ++v) nrm[v] = 0.0;
  const int zsx = ext0 + 1;  // x-face row length
  const int nfx = zsx * ext1, nfy = ext0 * (ext1 + 1);

  for (int k = 0; k < nzc; ++k) {
    const int r = k + 2;  // ring index of the current plane z0 + k
    double *cur = ring + (r & 3) * G.slot;
    // stages 2 and 3: U^n of this plane's columns into Unb with asynchronous
    // copies, issued by the thread that reads them in E, so their latency
    // hides behind the plane's face work (E of the previous plane, the only
    // reader of these entries, came before in this thread's program order)
    if (MODE == MODE_STAGE2 || MODE == MODE_STAGE3)
      for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
        const int i = c % ext0, j = c / ext0;
        const long long gi = ((long long)(z0 + k) * a.n[1] + (o[1] + j)) * a.n[0] + (o[0] + i);
#pragma unroll
        for (int v = 0; v < NV3; ++v) cp_async8(smem_u32(Unb + v * G.cols + c), a.Un + v * N + gi);
      }
    // A. wait for plane r+2; patch the current plane's x-y halo
    ok = wait_plane(mbar, r + 2, a);
    if (a.use_tma) fix_plane_halo(cur, a, o, ext0, ext1, z0 + k, G);
    // B. z-faces above the current plane (stencil planes r-1 .. r+2; after a
    // timeout the values read are discarded)
    z_faces<LIM>(ring, r, a, ext0, ncol, G, Fzc);
    if (sync_timed_out(ok, mbar, r + 2, r + 2, a)) return;  // plane r-1 dead; halo patch visible
    // C. refill plane r-1's slot with plane r+3
    if (r + 3 <= last) {
      if (a.use_tma && threadIdx.x == 0) fence_proxy_async_smem();
      fetch_plane(&tmap, ring, mbar, r + 3, a, o, ext0, ext1, z0, G);
    }
    // D. x and y faces of the current plane
    for (int f = threadIdx.x; f < nfx + nfy; f += blockDim.x) {
      if (f < nfx) {
        const int i = f % zsx, j = f / zsx;
        const double *p = cur + (j + 2) * G.BX + i;
        march_face<0, LIM>(p, p + 1, p + 2, p + 3, G.plane, a, Fx, G.nfx, f);
      } else {
        const int g = f - nfx;
        const int i = g % ext0, j = g / ext0;
        const double *p = cur + j * G.BX + i + 2;
        march_face<1, LIM>(p, p + G.BX, p + 2 * G.BX, p + 3 * G.BX, G.plane, a, Fy, G.nfy, g);
      }
    }
    __syncthreads();
    // E. residual of the current plane and the epilogue
    if (MODE == MODE_STAGE2 || MODE == MODE_STAGE3) cp_async_wait_all();  // this thread's U^n copies
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
      const int i = c % ext0, j = c / ext0;
      const int fx = j * zsx + i, fy = j * ext0 + i;
      const long long gi = ((long long)(z0 + k) * a.n[1] + (o[1] + j)) * a.n[0] + (o[0] + i);
      const int lc = (j + 2) * G.BX + (i + 2);
#pragma unroll
      for (int v = 0; v < NV3; ++v) {
        // same accumulation as the box-tiled kernel: the stage base, then x, y, z
        const double dFx = Fx[v * G.nfx + fx + 1] - Fx[v * G.nfx + fx];
        const double un = (MODE == MODE_STAGE2 || MODE == MODE_STAGE3) ? Unb[v * G.cols + c] : 0.0;
        double rv = (MODE == MODE_RESIDUAL && !a.S)
                        ? cx * dFx
                        : fma(cx, dFx, start_value<MODE>(a, cur[v * G.plane + lc], un, v * N + gi, src));
        rv = fma(cy, Fy[v * G.nfy + fy + ext0] - Fy[v * G.nfy + fy], rv);
        rv = fma(cz, Fzc[v * G.cols + c] - Fzp[v * G.cols + c], rv);
        if (MODE == MODE_RESIDUAL && want_norm) nrm[v] = fma(rv, rv, nrm[v]);
        a.out[v * N + gi] = rv;
      }
    }
    double *t = Fzp;  // each column's z-face buffer entries belong to one thread
    Fzp = Fzc;
    Fzc = t;
  }
  if (MODE == MODE_STAGE3 && a.t_acc && tix == 0 && threadIdx.x == 0) *a.t_acc += dt;

  if (want_norm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV3; ++v) {
      double sum = nrm[v];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, off);
      if (lane == 0) red[v][warp] = sum;
    }
    __syncthreads();
    if (threadIdx.x < NV3) {
      double sum = 0.0;
      const int nw = (blockDim.x + 31) >> 5;
      for (int q = 0; q < nw; ++q) sum += red[threadIdx.x][q];
      a.norm_part[tix * NV3 + threadIdx.x] = sum;
    }
  }
}

template <int LIM>
cudaError_t launch_march_lim(int mode, const CUtensorMap *tmap, const StageArgs &a, int threads, cudaStream_t st) {
  const size_t smem = march_smem_bytes(a.tile);
  const long long nblk = a.tile_count > 0 ? a.tile_count : (long long)a.ntile[0] * a.ntile[1] * a.ntile[2] - a.tile_begin;
  const dim3 grid((unsigned)nblk), block(threads);
  switch (mode) {
    case MODE_RESIDUAL: march_kernel<MODE_RESIDUAL, LIM><<<grid, block, smem, st>>>(*tmap, a); break;
    case MODE_STAGE1: march_kernel<MODE_STAGE1, LIM><<<grid, block, smem, st>>>(*tmap, a); break;
    case MODE_STAGE2: march_kernel<MODE_STAGE2, LIM><<<grid, block, smem, st>>>(*tmap, a); break;
    case MODE_STAGE3: march_kernel<MODE_STAGE3, LIM><<<grid, block, smem, st>>>(*tmap, a); break;
    default: return cudaErrorInvalidValue;  // the flux-difference mode runs on box tiles only
  }
  return cudaGetLastError();
}

template <int LIM>
cudaError_t set_march_attributes_lim(size_t smem_optin) {
  cudaError_t e = cudaSuccess;
  const void *k[4] = {(const void *)march_kernel<MODE_RESIDUAL, LIM>, (const void *)march_kernel<MODE_STAGE1, LIM>,
                      (const void *)march_kernel<MODE_STAGE2, LIM>, (const void *)march_kernel<MODE_STAGE3, LIM>};
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k[i]);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem_optin - fa.sharedSizeBytes));
  }
  return e;
}

}  // namespace

size_t march_smem_bytes(const int tile[3]) {
  const MarchGeom G = march_geom(tile);
  return 128 + sizeof(double) * ((size_t)kRing * G.slot + (size_t)NV3 * (G.nfx + G.nfy + 3 * G.cols)) +
         sizeof(uint64_t) * kRing;
}

cudaError_t launch_march(int mode, const CUtensorMap *tmap, const StageArgs &a, int threads, cudaStream_t st) {
  if (a.limiter == FV_LIM_VANLEER) return launch_march_lim<FV_LIM_VANLEER>(mode, tmap, a, threads, st);
  if (a.limiter == FV_LIM_NONE) return launch_march_lim<FV_LIM_NONE>(mode, tmap, a, threads, st);
  return launch_march_lim<FV_LIM_MINMOD>(mode, tmap, a, threads, st);
}

cudaError_t set_march_attributes(size_t smem_optin) {
  cudaError_t e = set_march_attributes_lim<FV_LIM_MINMOD>(smem_optin);
  if (e == cudaSuccess) e = set_march_attributes_lim<FV_LIM_VANLEER>(smem_optin);
  if (e == cudaSuccess) e = set_march_attributes_lim<FV_LIM_NONE>(smem_optin);
  return e;
}

}  // namespace fvk
