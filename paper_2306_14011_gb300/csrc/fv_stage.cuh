// Fused residual / SSP-RK3 stage kernel for 2D and 3D uniform Cartesian grids.
//
// One CTA owns a tile of cells.  It
//   1. stages the tile plus a 2-cell halo of every conserved variable into
//      shared memory: one TMA box (x, y[, z], var) completing on an mbarrier,
//      then plain loads for the halo cells that lie outside the domain
//      (periodic wrap or transmissive copy) -- TMA fills those with zeros;
//      without a tensor map (odd nx, tiny grids) every cell is a plain load;
//   2. per axis d, computes every face flux of the tile exactly once: MUSCL
//      face states of Eq. (6) (eps/2 * minmod slope) and the Roe flux, into a
//      shared-memory face buffer; each thread takes a run of consecutive faces
//      along the normal, carrying the stencil differences from face to face;
//   3. accumulates per cell, in shared memory, sum_d coef_d (F_{k+1/2} -
//      F_{k-1/2}) -- the flux-difference form of Eq. (5) -- starting, in the
//      RK modes, from the stage's base value (U^s, 3/4 U^n + 1/4 U^s or
//      1/3 U^n + 2/3 U^s), so the accumulator ends as the SSP-RK3 stage of
//      Eq. (4) discretised in time;
//   4. writes the residual or the new stage state for its cells (coalesced
//      along x).
// Faces on a tile boundary are computed by both neighbouring CTAs (a
// 1/tile_x + 1/tile_y [+ 1/tile_z] overhead); inside a tile each face is
// evaluated once.
#pragma once
#include "../../include/fv.h"
#include "fv_device.cuh"
#include "fv_internal.h"

namespace fvk {

constexpr uint64_t kTmaWaitNs = 2000000000ull;  // 2 s bound on the tile-load wait

struct TileGeom {
  int BX, BY, BZ;   // tile box with halo
  int plane;        // doubles per variable in the box
  int fmax;         // face-buffer length per variable
  int cells;        // cells per full tile
};

__host__ __device__ inline TileGeom tile_geom(int dim, const int tile[3]) {
  TileGeom g;
  const int tx = tile[0], ty = tile[1], tz = (dim == 3) ? tile[2] : 1;
  g.BX = tx + 4;
  g.BY = ty + 4;
  g.BZ = (dim == 3) ? tz + 4 : 1;
  g.plane = g.BX * g.BY * g.BZ;
  const int fx = (tx + 1) * ty * tz, fy = tx * (ty + 1) * tz, fz = (dim == 3) ? tx * ty * (tz + 1) : 0;
  g.fmax = fx > fy ? fx : fy;
  g.fmax = g.fmax > fz ? g.fmax : fz;
  g.cells = tx * ty * tz;
  return g;
}

// Interior index that ghost coordinate c of an axis with n cells reads.
__device__ __forceinline__ int ghost_source(int c, int n, int bclo, int bchi) {
  if (c < 0) return bclo == 0 ? ((c % n) + n) % n : 0;
  if (c >= n) return bchi == 0 ? c % n : n - 1;
  return c;
}

// Load halo cells of the tile box (the 4 layers along each axis next to the
// valid tile, over the valid extent of the other axes).  only_outside: skip
// cells inside the domain (already staged by TMA).
template <int DIM>
__device__ __forceinline__ void load_halo(double *tile, const StageArgs &a, const int o[3], const int ext[3],
                                          const TileGeom &G, bool only_outside) {
  constexpr int NV = DIM + 2;
  const long long N = (long long)a.n[0] * a.n[1] * a.n[2];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    if (only_outside && o[d] >= 2 && o[d] + ext[d] + 2 <= a.n[d]) continue;
    const int a1 = (d == 0) ? 1 : 0, a2 = (d == 2) ? 1 : 2;  // the other two axes
    const int e1 = ext[a1], e2 = (DIM == 3) ? ext[a2] : 1;
    const int cnt = 4 * e1 * e2;
    for (int h = threadIdx.x; h < cnt; h += blockDim.x) {
      const int layer = h & 3;
      const int r = h >> 2;
      int l[3];
      l[d] = (layer < 2) ? layer : ext[d] + layer;
      l[a1] = r % e1 + 2;
      l[a2] = (DIM == 3) ? r / e1 + 2 : 0;
      int gc[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) gc[q] = o[q] - 2 + l[q];
      if (DIM == 2) gc[2] = 0;
      const bool outside = gc[d] < 0 || gc[d] >= a.n[d];
      if (only_outside && !outside) continue;
      gc[d] = ghost_source(gc[d], a.n[d], a.bc[d][0], a.bc[d][1]);
      const long long src = ((long long)gc[2] * a.n[1] + gc[1]) * a.n[0] + gc[0];
      const int dst = (l[2] * G.BY + l[1]) * G.BX + l[0];
#pragma unroll
      for (int v = 0; v < NV; ++v) tile[v * G.plane + dst] = a.Us[v * N + src];
    }
  }
}

// All face fluxes of the tile along axis D into F, then their differences
// into the cell accumulator R (R = coef * dF for the first axis, += after).
// MUSCL face states of Eq. (6) on the stencil q0..q3 for limiter LIM.  Both
// limiters are symmetric (Psi(r) = r Psi(1/r)), so the two kappa-weighted
// limited slopes coincide and the states are q -+ eps/2 * slope; without a
// limiter the kappa weights cL = eps(1-kappa)/4, cR = eps(1+kappa)/4 apply.
// muscl_from_diffs takes the stencil's three differences dm = q1 - q0,
// d0 = q2 - q1, dp = q3 - q2 (consecutive faces share two of them).
template <int LIM>
__device__ __forceinline__ void muscl_from_diffs(double q1, double q2, double dm, double d0, double dp, double h,
                                                 double cL, double cR, double &QL, double &QR) {
  if (LIM == FV_LIM_NONE) {
    QL = fma(cL, dm, fma(cR, d0, q1));
    QR = fma(-cR, d0, fma(-cL, dp, q2));
  } else if (LIM == FV_LIM_VANLEER) {
    QL = fma(h, vanleer(dm, d0), q1);
    QR = fma(-h, vanleer(d0, dp), q2);
  } else {
    QL = fma(h, minmod(dm, d0), q1);
    QR = fma(-h, minmod(d0, dp), q2);
  }
}

template <int LIM>
__device__ __forceinline__ void muscl_states(double q0, double q1, double q2, double q3, double h, double cL,
                                             double cR, double &QL, double &QR) {
  muscl_from_diffs<LIM>(q1, q2, q1 - q0, q2 - q1, q3 - q2, h, cL, cR, QL, QR);
}

// Conserved state (rho, m, E) of primitive variables (rho, u, p), in place:
// m = rho u, E = p / (gamma - 1) + rho |u|^2 / 2.
template <int DIM>
__device__ __forceinline__ void to_conserved(double (&w)[DIM + 2], double inv_g1) {
  double q2 = w[1] * w[1];
#pragma unroll
  for (int d = 1; d < DIM; ++d) q2 = fma(w[1 + d], w[1 + d], q2);
  const double e = fma(scale_pow2<-1>(w[0]), q2, w[DIM + 1] * inv_g1);
#pragma unroll
  for (int d = 0; d < DIM; ++d) w[1 + d] = w[0] * w[1 + d];
  w[DIM + 1] = e;
}

// Every cell of the staged box from conserved to primitive variables, in
// place: u = m / rho, p = (gamma - 1)(E - m.u / 2).  Corner cells the stencils
// never read may hold zeros; whatever they turn into is never used.
template <int DIM>
__device__ __forceinline__ void box_to_primitive(double *tile, const TileGeom &G, double g1) {
  for (int c = threadIdx.x; c < G.plane; c += blockDim.x) {
    const double rho = tile[c];
    const double r = rcp_fp64(rho);
    double k = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const double m = tile[(1 + d) * G.plane + c];
      const double u = m * r;
      k = (d == 0) ? m * u : fma(m, u, k);
      tile[(1 + d) * G.plane + c] = u;
    }
    tile[(DIM + 1) * G.plane + c] = g1 * fma(-0.5, k, tile[(DIM + 1) * G.plane + c]);
  }
}

// The part of a stage update that does not depend on the fluxes: Us (stage
// 1), 3/4 Un + 1/4 Us (stage 2), 1/3 Un + 2/3 Us (stage 3); 0 for the residual.
template <int MODE>
__device__ __forceinline__ double stage_base(double us, double un) {
  if (MODE == MODE_RESIDUAL) return 0.0;
  if (MODE == MODE_STAGE1) return us;
  if (MODE == MODE_STAGE2) return fma(0.75, un, quarter(us));
  return fma(1.0 / 3.0, un, (2.0 / 3.0) * us);
}

// The value a cell's accumulation starts from: the stage base, plus the
// source term of Eq. (5) when one is set (src = -|Omega| for the residual,
// w dt for an RK stage, since dU/dt = -R/|Omega| has +S).
template <int MODE>
__device__ __forceinline__ double start_value(const StageArgs &a, double us, double un, long long idx, double src) {
  double b = stage_base<MODE>(us, un);
  if (a.S) b = (MODE == MODE_RESIDUAL) ? src * a.S[idx] : fma(src, a.S[idx], b);
  return b;
}

template <int DIM, int D, int LIM, int MODE>
__device__ __forceinline__ void face_pass(const double *__restrict__ tile, double *__restrict__ F,
                                          double *__restrict__ R, const StageArgs &a, const int o[3],
                                          const int ext[3], const TileGeom &G, double coef, double src) {
  constexpr int NV = DIM + 2;
  constexpr int NT = DIM - 1;
  constexpr int E = NV - 1;
  const int fe0 = ext[0] + (D == 0), fe1 = ext[1] + (D == 1), fe2 = (DIM == 3) ? ext[2] + (D == 2) : 1;
  // Faces form lines along the normal axis D (fn faces each); a work item is a
  // run of up to K consecutive faces of one line, so each face after the first
  // takes one new stencil value and one new difference per variable.  Items
  // are numbered with the line fastest (neighbouring threads, neighbouring
  // lines); K = ceil(faces / threads) keeps one item per thread when the
  // lines split evenly.
  const int fn = (D == 0) ? fe0 : ((D == 1) ? fe1 : fe2);
  const int la = (D == 0) ? fe1 : fe0;  // line index = a + la * b over the two other axes
  const int nline = fe0 * fe1 * fe2 / fn;
  const int K = (fn * nline + (int)blockDim.x - 1) / (int)blockDim.x;
  const int nrun = (fn + K - 1) / K;
  const int sstride = (D == 0) ? 1 : ((D == 1) ? G.BX : G.BX * G.BY);
  const int fstr = (D == 0) ? 1 : ((D == 1) ? fe0 : fe0 * fe1);  // face-index stride along the normal
  const double h = a.half_eps;
  for (int item = threadIdx.x; item < nrun * nline; item += blockDim.x) {
    const int run = item / nline, line = item - run * nline;
    const int ca = line % la, cb = line / la;  // the line's two other-axis coordinates
    const int m0 = run * K, m1 = min(m0 + K, fn);
    int lx, ly, lz, f;  // box coordinates of stencil start of face m0, and its face index
    if (D == 0) {
      lx = m0, ly = ca + 2, lz = cb + 2;
      f = (cb * fe1 + ca) * fe0 + m0;
    } else if (D == 1) {
      lx = ca + 2, ly = m0, lz = cb + 2;
      f = (cb * fe1 + m0) * fe0 + ca;
    } else {
      lx = ca + 2, ly = cb + 2, lz = m0;
      f = (m0 * fe1 + cb) * fe0 + ca;
    }
    if (DIM == 2) lz = 0;
    const double *p = tile + (lz * G.BY + ly) * G.BX + lx;
    // carried from face to face: the two leading differences (stencil values
    // are re-read from shared memory, which keeps the carried state small)
    double dm[NV], d0[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double *pv = p + v * G.plane;
      dm[v] = pv[sstride] - pv[0];
      d0[v] = pv[2 * sstride] - pv[sstride];
    }
    for (int m = m0; m < m1; ++m, p += sstride, f += fstr) {
      double QL[NV], QR[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double *pv = p + v * G.plane;
        const double q1 = pv[sstride], q2 = pv[2 * sstride];
        const double dp = pv[3 * sstride] - q2;
        muscl_from_diffs<LIM>(q1, q2, dm[v], d0[v], dp, h, a.cL, a.cR, QL[v], QR[v]);
        dm[v] = d0[v];
        d0[v] = dp;
      }
      if (a.recon == FV_RECON_PRIMITIVE) {  // (rho, u, p) face states -> (rho, m, E)
        to_conserved<DIM>(QL, a.inv_g1);
        to_conserved<DIM>(QR, a.inv_g1);
      }
      // normal-first ordering: (rho, m_D, tangential momenta, E)
      double qL[NT + 3], qR[NT + 3], Gf[NT + 3];
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
      roe_F<NT>(qL, qR, a.g1, a.efix, a.inv2efix, Gf);
      F[f] = Gf[0];
      F[(1 + D) * G.fmax + f] = Gf[1];
      t = 0;
#pragma unroll
      for (int ax = 0; ax < DIM; ++ax) {
        if (ax == D) continue;
        F[(1 + ax) * G.fmax + f] = Gf[2 + t];
        ++t;
      }
      F[E * G.fmax + f] = Gf[E];
    }
  }
  if (D == 0 && (MODE == MODE_STAGE2 || MODE == MODE_STAGE3)) cp_async_wait_all();  // this thread's U^n copies
  __syncthreads();
  // R accumulates the new value of each cell: the first axis starts from the
  // stage base (RK modes) or from 0 (residual), so the update needs no
  // separate addition.
  const int ncell = ext[0] * ext[1] * ((DIM == 3) ? ext[2] : 1);
  const int fstride = (D == 0) ? 1 : ((D == 1) ? fe0 : fe0 * fe1);
  const long long N = (long long)a.n[0] * a.n[1] * a.n[2];
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    const int i = c % ext[0];
    const int rr = c / ext[0];
    const int j = rr % ext[1];
    const int k = rr / ext[1];
    const int flo = (k * fe1 + j) * fe0 + i;
    long long gi = 0;
    int lc = 0;
    if (D == 0 && MODE != MODE_FLUXDIFF && (MODE != MODE_RESIDUAL || a.S)) {
      gi = ((long long)(o[2] + k) * a.n[1] + (o[1] + j)) * a.n[0] + (o[0] + i);
      lc = (((DIM == 3) ? k + 2 : 0) * G.BY + (j + 2)) * G.BX + (i + 2);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double dF = F[v * G.fmax + flo + fstride] - F[v * G.fmax + flo];
      if (MODE == MODE_FLUXDIFF) {  // this axis's differences alone, written out after the pass
        R[v * G.cells + c] = dF;
      } else if (D == 0) {
        if (MODE == MODE_RESIDUAL && !a.S)
          R[v * G.cells + c] = coef * dF;
        else  // stages 2 and 3: R holds U^n, copied in by prefetch_un
          R[v * G.cells + c] =
              fma(coef, dF, start_value<MODE>(a, a.recon == FV_RECON_PRIMITIVE ? a.Us[v * N + gi] : tile[v * G.plane + lc],
                                              (MODE == MODE_STAGE2 || MODE == MODE_STAGE3) ? R[v * G.cells + c] : 0.0,
                                              v * N + gi, src));
      } else {
        R[v * G.cells + c] = fma(coef, dF, R[v * G.cells + c]);
      }
    }
  }
  __syncthreads();
}

// The tile's cells of the accumulator R into the SoA array dst (the
// flux-difference mode's per-axis output).  R is not written again before the
// next face pass's barrier, so no barrier is needed here.
template <int DIM>
__device__ __forceinline__ void store_cells(const double *R, double *dst, const StageArgs &a, const int o[3],
                                            const int ext[3], const TileGeom &G) {
  constexpr int NV = DIM + 2;
  const long long N = (long long)a.n[0] * a.n[1] * a.n[2];
  const int ncell = ext[0] * ext[1] * ext[2];
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    const int i = c % ext[0];
    const int rr = c / ext[0];
    const int j = rr % ext[1];
    const int k = rr / ext[1];
    const long long gi = ((long long)(o[2] + k) * a.n[1] + (o[1] + j)) * a.n[0] + (o[0] + i);
#pragma unroll
    for (int v = 0; v < NV; ++v) dst[v * N + gi] = R[v * G.cells + c];
  }
}

// Stages 2 and 3: U^n of the tile's cells into the accumulator R, with
// asynchronous copies issued before the tile load completes, so their latency
// hides behind the load and the first axis's fluxes; the first axis's
// accumulation (same cell-to-thread map) waits for the thread's own copies and
// reads U^n there before overwriting it.
template <int DIM, int MODE>
__device__ __forceinline__ void prefetch_un(double *R, const StageArgs &a, const int o[3], const int ext[3],
                                            const TileGeom &G) {
  if (MODE != MODE_STAGE2 && MODE != MODE_STAGE3) return;
  constexpr int NV = DIM + 2;
  const long long N = (long long)a.n[0] * a.n[1] * a.n[2];
  const int ncell = ext[0] * ext[1] * ext[2];
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    const int i = c % ext[0];
    const int rr = c / ext[0];
    const int j = rr % ext[1];
    const int k = rr / ext[1];
    const long long gi = ((long long)(o[2] + k) * a.n[1] + (o[1] + j)) * a.n[0] + (o[0] + i);
#pragma unroll
    for (int v = 0; v < NV; ++v) cp_async8(smem_u32(R + v * G.cells + c), a.Un + v * N + gi);
  }
}

// All the work of one tile: stage the tile (TMA with mbarrier `bar` at parity
// `phase`, or plain loads), compute the face fluxes axis by axis, accumulate
// the residual (or the new stage state) and write it.  `tile` is the CTA's dynamic shared
// memory (128-byte aligned); s_coef (5 doubles) and red are static shared
// scratch.
// Returns false (uniformly across the CTA) if the tile load timed out.
template <int DIM, int MODE, int LIM = FV_LIM_MINMOD>
__device__ __forceinline__ bool tile_work(const CUtensorMap *tmap, const StageArgs &a, int bx, int by, int bz,
                                          double *tile, uint64_t *mbar, uint32_t phase, double *s_coef,
                                          double (*red)[32]) {
  constexpr int NV = DIM + 2;
  const TileGeom G = tile_geom(DIM, a.tile);
  double *F = tile + NV * G.plane;
  double *R = F + NV * G.fmax;
  const int o[3] = {bx * a.tile[0], by * a.tile[1], (DIM == 3) ? bz * a.tile[2] : 0};
  int ext[3];
  ext[0] = min(a.tile[0], a.n[0] - o[0]);
  ext[1] = min(a.tile[1], a.n[1] - o[1]);
  ext[2] = (DIM == 3) ? min(a.tile[2], a.n[2] - o[2]) : 1;
  const long long N = (long long)a.n[0] * a.n[1] * a.n[2];

  // ---- 1. stage the tile and its halo (and, stages 2-3, U^n into R)
  if (a.use_tma) {
    const uint32_t bar = smem_u32(mbar);
    if (threadIdx.x == 0) {
      mbar_expect_tx(bar, (uint32_t)(NV * G.plane * sizeof(double)));
      if (DIM == 2)
        tma_load_3d(smem_u32(tile), tmap, o[0] - 2, o[1] - 2, 0, bar);
      else
        tma_load_4d(smem_u32(tile), tmap, o[0] - 2, o[1] - 2, o[2] - 2, 0, bar);
    }
    prefetch_un<DIM, MODE>(R, a, o, ext, G);
    const bool ok = mbar_wait_bounded(bar, phase, kTmaWaitNs);
    if (__syncthreads_or(!ok)) {
      if (MODE == MODE_STAGE2 || MODE == MODE_STAGE3) cp_async_wait_all();
      if (threadIdx.x == 0) {
        atomicOr(a.flags, FLAG_TIMEOUT);
        mbar_wait_bounded(bar, phase, kTmaWaitNs);  // let a late copy land before the CTA moves on
      }
      return false;
    }
    load_halo<DIM>(tile, a, o, ext, G, true);
  } else {
    prefetch_un<DIM, MODE>(R, a, o, ext, G);
    const int ncell = ext[0] * ext[1] * ext[2];
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
      const int i = c % ext[0];
      const int rr = c / ext[0];
      const int j = rr % ext[1];
      const int k = rr / ext[1];
      const long long src = ((long long)(o[2] + k) * a.n[1] + (o[1] + j)) * a.n[0] + (o[0] + i);
      const int dst = (((DIM == 3) ? k + 2 : 0) * G.BY + (j + 2)) * G.BX + (i + 2);
#pragma unroll
      for (int v = 0; v < NV; ++v) tile[v * G.plane + dst] = a.Us[v * N + src];
    }
    load_halo<DIM>(tile, a, o, ext, G, false);
  }

  // ---- 2./3. face fluxes and their differences per axis.  The step and the
  // per-axis scales are formed once per CTA (an FP64 division per thread
  // would cost ~2% of the kernel's FP64 work).
  if (threadIdx.x == 0) {
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
  if (a.recon == FV_RECON_PRIMITIVE) {  // Eq. (6) on (rho, u, p)
    box_to_primitive<DIM>(tile, G, a.g1);
    __syncthreads();
  }
  const double dt = s_coef[0];
  face_pass<DIM, 0, LIM, MODE>(tile, F, R, a, o, ext, G, s_coef[1], s_coef[4]);
  if (MODE == MODE_FLUXDIFF) store_cells<DIM>(R, a.fd, a, o, ext, G);
  face_pass<DIM, 1, LIM, MODE>(tile, F, R, a, o, ext, G, s_coef[2], s_coef[4]);
  if (MODE == MODE_FLUXDIFF) store_cells<DIM>(R, a.fd + (long long)NV * N, a, o, ext, G);
  if constexpr (DIM == 3) {
    face_pass<DIM, 2, LIM, MODE>(tile, F, R, a, o, ext, G, s_coef[3], s_coef[4]);
    if (MODE == MODE_FLUXDIFF) store_cells<DIM>(R, a.fd + 2ll * NV * N, a, o, ext, G);
  }
  if (MODE == MODE_FLUXDIFF) return true;

  // ---- 4. epilogue
  const int ncell = ext[0] * ext[1] * ext[2];
  const bool want_norm = (MODE == MODE_RESIDUAL) && a.norm_part != nullptr;
  double nrm[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) nrm[v] = 0.0;
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    const int i = c % ext[0];
    const int rr = c / ext[0];
    const int j = rr % ext[1];
    const int k = rr / ext[1];
    const long long gi = ((long long)(o[2] + k) * a.n[1] + (o[1] + j)) * a.n[0] + (o[0] + i);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double r = R[v * G.cells + c];  // the residual, or the cell's new value
      if (MODE == MODE_RESIDUAL && want_norm) nrm[v] = fma(r, r, nrm[v]);
      a.out[v * N + gi] = r;
    }
  }
  if (MODE == MODE_STAGE3 && a.t_acc && bx == 0 && by == 0 && bz == 0 && threadIdx.x == 0) *a.t_acc += dt;

  if (want_norm) {
    // CTA partial sums of R_v^2 (fixed reduction order: lanes, then warps)
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
      const long long tix = ((long long)bz * a.ntile[1] + by) * a.ntile[0] + bx;
      a.norm_part[tix * NV + threadIdx.x] = sum;
    }
  }
  return true;
}

// Dynamic shared memory of the stage kernels: tile box, face buffer, residual
// accumulator, then one mbarrier.
template <int DIM>
__device__ __forceinline__ uint64_t *stage_mbar(double *tile, const StageArgs &a) {
  constexpr int NV = DIM + 2;
  const TileGeom G = tile_geom(DIM, a.tile);
  return reinterpret_cast<uint64_t *>(tile + NV * (G.plane + G.fmax + G.cells));
}

__device__ __forceinline__ double *aligned_smem(unsigned char *raw) {
  return reinterpret_cast<double *>((reinterpret_cast<uintptr_t>(raw) + 127) & ~uintptr_t(127));
}

// One CTA per tile of the grid.  Register budget: FV_STAGE_MIN_BLOCKS resident
// CTAs of MAXT threads per SM (2 by default; the default tiles' shared memory
// also allows two CTAs per SM).  2D kernels come in two sizes: up to
// kStage2dMaxThreads threads (170 registers per thread for the face runs and
// their integer-pipe products) and up to 256 (128 registers); 3D box kernels
// take up to kStage3dMaxThreads threads (168 registers: the five-variable
// runs would spill at 128).
#ifndef FV_STAGE_MIN_BLOCKS
#define FV_STAGE_MIN_BLOCKS 2
#endif
template <int DIM, int MODE, int LIM, int MAXT>
__global__ void __launch_bounds__(MAXT, FV_STAGE_MIN_BLOCKS)
    stage_kernel(const __grid_constant__ CUtensorMap tmap, const StageArgs a) {
  constexpr int NV = DIM + 2;
  extern __shared__ unsigned char smem_raw[];
  __shared__ double s_coef[5];
  __shared__ double red[NV][32];
  double *tile = aligned_smem(smem_raw);
  uint64_t *mbar = stage_mbar<DIM>(tile, a);
  if (a.use_tma) {
    if (threadIdx.x == 0) {
      mbar_init(smem_u32(mbar), 1);
      fence_mbar_init();
    }
    __syncthreads();
  }
  long long b = a.tile_begin + blockIdx.x;
  const int bx = (int)(b % a.ntile[0]);
  b /= a.ntile[0];
  const int by = (int)(b % a.ntile[1]);
  const int bz = (int)(b / a.ntile[1]);
  tile_work<DIM, MODE, LIM>(&tmap, a, bx, by, bz, tile, mbar, 0u, s_coef, red);
}

template <int DIM, int LIM, int MAXT>
cudaError_t launch_stage_lim(int mode, const CUtensorMap *tmap, const StageArgs &a, int threads, cudaStream_t st) {
  const size_t smem = stage_smem_bytes(DIM, a.tile);
  const long long nblk = a.tile_count > 0 ? a.tile_count : (long long)a.ntile[0] * a.ntile[1] * a.ntile[2] - a.tile_begin;
  const dim3 grid((unsigned)nblk), block(threads);
  switch (mode) {
    case MODE_RESIDUAL: stage_kernel<DIM, MODE_RESIDUAL, LIM, MAXT><<<grid, block, smem, st>>>(*tmap, a); break;
    case MODE_STAGE1: stage_kernel<DIM, MODE_STAGE1, LIM, MAXT><<<grid, block, smem, st>>>(*tmap, a); break;
    case MODE_STAGE2: stage_kernel<DIM, MODE_STAGE2, LIM, MAXT><<<grid, block, smem, st>>>(*tmap, a); break;
    case MODE_STAGE3: stage_kernel<DIM, MODE_STAGE3, LIM, MAXT><<<grid, block, smem, st>>>(*tmap, a); break;
    default: stage_kernel<DIM, MODE_FLUXDIFF, LIM, MAXT><<<grid, block, smem, st>>>(*tmap, a); break;
  }
  return cudaGetLastError();
}

template <int DIM, int MAXT>
cudaError_t launch_stage_dim(int mode, const CUtensorMap *tmap, const StageArgs &a, int threads, cudaStream_t st) {
  if (a.limiter == FV_LIM_VANLEER) return launch_stage_lim<DIM, FV_LIM_VANLEER, MAXT>(mode, tmap, a, threads, st);
  if (a.limiter == FV_LIM_NONE) return launch_stage_lim<DIM, FV_LIM_NONE, MAXT>(mode, tmap, a, threads, st);
  return launch_stage_lim<DIM, FV_LIM_MINMOD, MAXT>(mode, tmap, a, threads, st);
}

// Allow each stage kernel the largest dynamic shared memory the device offers
// (opt-in limit minus the kernel's static shared memory), so contexts with
// different tile shapes never lower each other's limit.  `smem_optin` is the
// device's per-block opt-in limit.
template <int DIM, int LIM, int MAXT>
cudaError_t set_stage_attributes_lim(size_t smem_optin) {
  cudaError_t e = cudaSuccess;
  const void *k[5] = {(const void *)stage_kernel<DIM, MODE_RESIDUAL, LIM, MAXT>,
                      (const void *)stage_kernel<DIM, MODE_STAGE1, LIM, MAXT>,
                      (const void *)stage_kernel<DIM, MODE_STAGE2, LIM, MAXT>,
                      (const void *)stage_kernel<DIM, MODE_STAGE3, LIM, MAXT>,
                      (const void *)stage_kernel<DIM, MODE_FLUXDIFF, LIM, MAXT>};
  for (int i = 0; i < 5 && e == cudaSuccess; ++i) {
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k[i]);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(smem_optin - fa.sharedSizeBytes));
  }
  return e;
}

template <int DIM, int MAXT>
cudaError_t set_stage_attributes_dim(size_t smem_optin) {
  cudaError_t e = set_stage_attributes_lim<DIM, FV_LIM_MINMOD, MAXT>(smem_optin);
  if (e == cudaSuccess) e = set_stage_attributes_lim<DIM, FV_LIM_VANLEER, MAXT>(smem_optin);
  if (e == cudaSuccess) e = set_stage_attributes_lim<DIM, FV_LIM_NONE, MAXT>(smem_optin);
  return e;
}

}  // namespace fvk
