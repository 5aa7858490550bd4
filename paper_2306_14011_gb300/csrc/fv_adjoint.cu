// Discrete adjoint of the residual: out = sum_d scale_d J_d(U)^T lam, with J_d
// the Jacobian of the axis-d flux differences, plus a linear combination of up
// to three arrays (the reverse of the SSP-RK3 stage combinations).
//
// lam^T R = sum over faces f of ds (lam_{f-1} - lam_f) . F_f, F_f the flux
// between cells f-1 and f from the MUSCL states of cells f-2..f+1.  One CTA
// per tile computes, for every face whose stencil touches the tile, the
// cotangents of its left/right states (roe_F_vjp) and pushes them through the
// reconstruction to the four stencil cells; each cell then gathers what its
// faces sent it, so no atomics are needed.  Halos: 3 cells of U, 2 of lam.
// With transmissive boundaries the faces outside [0, n] do not exist and the
// boundary cells also collect what was sent to their ghost copies.
#include "../../include/fv.h"
#include "fv_adjoint.cuh"
#include "fv_stage.cuh"

namespace fvk {

namespace {

struct AdjGeom {
  int UX, UY, UZ, uplane;  // U box with halo 3
  int LX, LY, LZ, lplane;  // lam box with halo 2
  int fmax, cells;
};

__host__ __device__ inline AdjGeom adj_geom(int dim, const int tile[3]) {
  AdjGeom g;
  const int tx = tile[0], ty = tile[1], tz = dim == 3 ? tile[2] : 1;
  g.UX = tx + 6;
  g.UY = ty + 6;
  g.UZ = dim == 3 ? tz + 6 : 1;
  g.uplane = g.UX * g.UY * g.UZ;
  g.LX = tx + 4;
  g.LY = ty + 4;
  g.LZ = dim == 3 ? tz + 4 : 1;
  g.lplane = g.LX * g.LY * g.LZ;
  const int fx = (tx + 3) * ty * tz, fy = tx * (ty + 3) * tz, fz = dim == 3 ? tx * ty * (tz + 3) : 0;
  g.fmax = fx > fy ? fx : fy;
  g.fmax = g.fmax > fz ? g.fmax : fz;
  g.cells = tx * ty * tz;
  return g;
}

// Box of `halo` cells around the valid tile, every variable, plain loads with
// the boundary index map (corners included; they are never read).  With
// zero_transmissive, cells beyond a transmissive side are 0 instead: they are
// ghosts, which carry no residual and hence no cotangent.
template <int DIM>
__device__ void load_box(double *dst, const double *src, const AdjArgs &a, const int o[3], const int ext[3],
                         int halo, int BX, int BY, int plane, bool zero_transmissive) {
  constexpr int NV = DIM + 2;
  const long long N = (long long)a.n[0] * a.n[1] * a.n[2];
  const int ex = ext[0] + 2 * halo, ey = ext[1] + 2 * halo, ez = DIM == 3 ? ext[2] + 2 * halo : 1;
  const int cnt = ex * ey * ez;
  for (int c = threadIdx.x; c < cnt; c += blockDim.x) {
    const int i = c % ex, r = c / ex, j = r % ey, k = r / ey;
    const int cx = o[0] - halo + i, cy = o[1] - halo + j, cz = DIM == 3 ? o[2] - halo + k : 0;
    bool ghost_zero = false;
    if (zero_transmissive) {
      const int cc[3] = {cx, cy, cz};
#pragma unroll
      for (int d = 0; d < DIM; ++d)
        ghost_zero = ghost_zero || (cc[d] < 0 && a.bc[d][0] == FV_BC_TRANSMISSIVE) ||
                     (cc[d] >= a.n[d] && a.bc[d][1] == FV_BC_TRANSMISSIVE);
    }
    const int gx = ghost_source(cx, a.n[0], a.bc[0][0], a.bc[0][1]);
    const int gy = ghost_source(cy, a.n[1], a.bc[1][0], a.bc[1][1]);
    const int gz = DIM == 3 ? ghost_source(cz, a.n[2], a.bc[2][0], a.bc[2][1]) : 0;
    const long long s = ((long long)gz * a.n[1] + gy) * a.n[0] + gx;
    const int d = (k * BY + j) * BX + i;
#pragma unroll
    for (int v = 0; v < NV; ++v) dst[v * plane + d] = ghost_zero ? 0.0 : src[v * N + s];
  }
}

// pick3(d, x, y, z): x, y or z for d = 0, 1, 2 (register selects, so that an
// axis chosen at run time needs no indexed local array).
__device__ __forceinline__ int pick3(int d, int x, int y, int z) { return d == 0 ? x : (d == 1 ? y : z); }

// Faces along axis D: per face the cotangents sent to its four stencil cells
// (c0..c3 for cells f-2 .. f+1), stored as 4*NV doubles; then every tile cell
// gathers and accumulates scale * (sum) into acc.  The axis is a run-time
// argument: the kernel runs one copy of this (long) code for every axis, half
// (2D) or a third (3D) of the instruction footprint of one copy per axis,
// and the normal-first ordering of the flux's variables is formed with
// selects.
// HALF: the MUSCL factor eps/2 is 1/2 (eps = 1), so h * x is an exponent
// decrement on the integer pipe (scale_pow2) instead of an FP64 product.
template <int DIM, bool HALF>
__device__ void adj_face_pass(const double *Ubox, const double *Lbox, double *Fb, double *acc, const AdjArgs &a,
                              const int o[3], const int ext[3], const AdjGeom &G, double scale, int D) {
  constexpr int NV = DIM + 2;
  constexpr int NT = DIM - 1;
  constexpr int E = NV - 1;
  const int fe0 = ext[0] + (D == 0 ? 3 : 0), fe1 = ext[1] + (D == 1 ? 3 : 0);
  const int fe2 = DIM == 3 ? ext[2] + (D == 2 ? 3 : 0) : 1;
  const int nf = fe0 * fe1 * fe2;
  const int us = pick3(D, 1, G.UX, G.UX * G.UY);  // U stencil stride
  const int ls = pick3(D, 1, G.LX, G.LX * G.LY);  // lam stride
  const int oD = pick3(D, o[0], o[1], o[2]), nD = pick3(D, a.n[0], a.n[1], a.n[2]);
  const double h = a.half_eps;
  const bool lo_trans = a.bc[D][0] == FV_BC_TRANSMISSIVE, hi_trans = a.bc[D][1] == FV_BC_TRANSMISSIVE;
  for (int f = threadIdx.x; f < nf; f += blockDim.x) {
    const int i = f % fe0, rr = f / fe0, j = rr % fe1, k = rr / fe1;
    // face index along D (global): between cells fg-1 and fg
    const int fg = oD - 1 + pick3(D, i, j, k);
    double *out = Fb + f;  // 4*NV values at stride G.fmax
    const bool real = !((lo_trans && fg < 0) || (hi_trans && fg > nD));
    if (!real) {
#pragma unroll
      for (int q = 0; q < 4 * NV; ++q) out[q * G.fmax] = 0.0;
      continue;
    }
    // U stencil: cells fg-2 .. fg+1 -> U box coordinate along D: (fg-2) - (o[D]-3) = loc[D]
    const int ux = D == 0 ? i : i + 3, uy = D == 1 ? j : j + 3, uz = DIM == 3 ? (D == 2 ? k : k + 3) : 0;
    const double *pu = Ubox + (uz * G.UY + uy) * G.UX + ux;
    // lam at cells fg-1 and fg -> lam box coordinate along D: (fg-1) - (o[D]-2) = loc[D]
    const int lx = D == 0 ? i : i + 2, ly = D == 1 ? j : j + 2, lz = DIM == 3 ? (D == 2 ? k : k + 2) : 0;
    const double *pl = Lbox + (lz * G.LY + ly) * G.LX + lx;
    double QL[NV], QR[NV], gb[NV];
    int pL[NV], pR[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double *q = pu + v * G.uplane;
      const double q0 = q[0], q1 = q[us], q2 = q[2 * us], q3 = q[3 * us];
      const double dm = q1 - q0, d0 = q2 - q1, dp = q3 - q2;
      QL[v] = fma(h, minmod(dm, d0), q1);
      QR[v] = fma(-h, minmod(d0, dp), q2);
      pL[v] = minmod_pick(dm, d0);
      pR[v] = minmod_pick(d0, dp);
      gb[v] = pl[v * G.lplane] - pl[v * G.lplane + ls];
    }
    // normal-first ordering (rho, m_D, tangential momenta in axis order, E)
    double qL[NT + 3], qR[NT + 3], Gb[NT + 3], bL[NT + 3], bR[NT + 3];
    qL[0] = QL[0];
    qR[0] = QR[0];
    Gb[0] = gb[0];
    qL[E] = QL[E];
    qR[E] = QR[E];
    Gb[E] = gb[E];
    if (DIM == 2) {
      const bool x = D == 0;
      qL[1] = isel(x, QL[1], QL[2]);
      qL[2] = isel(x, QL[2], QL[1]);
      qR[1] = isel(x, QR[1], QR[2]);
      qR[2] = isel(x, QR[2], QR[1]);
      Gb[1] = isel(x, gb[1], gb[2]);
      Gb[2] = isel(x, gb[2], gb[1]);
    } else {
      // normal m_D; tangential (m_1, m_2), (m_0, m_2) or (m_0, m_1)
      const bool d0 = D == 0, d2 = D == 2;
      qL[1] = isel(d0, QL[1], isel(d2, QL[3], QL[2]));
      qL[2] = isel(d0, QL[2], QL[1]);
      qL[3] = isel(d2, QL[2], QL[3]);
      qR[1] = isel(d0, QR[1], isel(d2, QR[3], QR[2]));
      qR[2] = isel(d0, QR[2], QR[1]);
      qR[3] = isel(d2, QR[2], QR[3]);
      Gb[1] = isel(d0, gb[1], isel(d2, gb[3], gb[2]));
      Gb[2] = isel(d0, gb[2], gb[1]);
      Gb[3] = isel(d2, gb[2], gb[3]);
    }
    roe_F_vjp<NT>(qL, qR, a.g1, a.efix, a.inv2efix, Gb, bL, bR);
    // back to the natural variable order
    double QLb[NV], QRb[NV];
    QLb[0] = bL[0];
    QRb[0] = bR[0];
    QLb[E] = bL[E];
    QRb[E] = bR[E];
    if (DIM == 2) {
      const bool x = D == 0;
      QLb[1] = isel(x, bL[1], bL[2]);
      QLb[2] = isel(x, bL[2], bL[1]);
      QRb[1] = isel(x, bR[1], bR[2]);
      QRb[2] = isel(x, bR[2], bR[1]);
    } else {
      const bool d0 = D == 0, d1 = D == 1, d2 = D == 2;
      QLb[1] = isel(d0, bL[1], bL[2]);
      QLb[2] = isel(d1, bL[1], isel(d0, bL[2], bL[3]));
      QLb[3] = isel(d2, bL[1], bL[3]);
      QRb[1] = isel(d0, bR[1], bR[2]);
      QRb[2] = isel(d1, bR[1], isel(d0, bR[2], bR[3]));
      QRb[3] = isel(d2, bR[1], bR[3]);
    }
    // through the reconstruction: QL = q1 + h mm(q1-q0, q2-q1), QR = q2 - h mm(q2-q1, q3-q2).
    // The picked slope's derivative is +-1 on its two cells; the selections and
    // sign flips run on the integer pipe (isel, mul_sign), only the sums in FP64.
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double hl = HALF ? scale_pow2<-1>(QLb[v]) : h * QLb[v];
      const double hr = HALF ? scale_pow2<-1>(QRb[v]) : h * QRb[v];
      const double nhl = mul_sign(hl, -1.0), nhr = mul_sign(hr, -1.0);
      const double c0 = isel(pL[v] == 1, nhl, 0.0);
      const double c3 = isel(pR[v] == 2, nhr, 0.0);
      // c1 = QLb + (pL: +hl if a, -hl if b) + (pR: +hr if a)
      // c2 = QRb + (pR: -hr if a, +hr if b) + (pL: +hl if b)
      const double l1 = isel(pL[v] == 1, hl, isel(pL[v] == 2, nhl, 0.0));
      const double r2 = isel(pR[v] == 1, nhr, isel(pR[v] == 2, hr, 0.0));
      const double c1 = (QLb[v] + l1) + isel(pR[v] == 1, hr, 0.0);
      const double c2 = (QRb[v] + r2) + isel(pL[v] == 2, hl, 0.0);
      out[(4 * v + 0) * G.fmax] = c0;
      out[(4 * v + 1) * G.fmax] = c1;
      out[(4 * v + 2) * G.fmax] = c2;
      out[(4 * v + 3) * G.fmax] = c3;
    }
  }
  __syncthreads();
  // gather: cell c (local index m along D) receives c0 of face m+2, c1 of m+1,
  // c2 of m, c3 of m-1 (local face index = global face - (o[D]-1)); boundary
  // cells of transmissive sides also collect what was sent to their ghosts.
  const int ncell = ext[0] * ext[1] * (DIM == 3 ? ext[2] : 1);
  const int fstride = pick3(D, 1, fe0, fe0 * fe1);
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    const int i = c % ext[0], rr = c / ext[0], j = rr % ext[1], k = rr / ext[1];
    const int m = pick3(D, i, j, k);
    // local index of the face between cells m-1 and m (global face o[D]+m) along D
    const int fi = D == 0 ? m + 1 : i, fj = D == 1 ? m + 1 : j, fk = D == 2 ? m + 1 : k;
    const int fc = (fk * fe1 + fj) * fe0 + fi;  // face "m" (global o[D]+m)
    const int gcell = oD + m;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double *P = Fb + (4 * v) * G.fmax;
      double s = P[0 * G.fmax + fc + 2 * fstride]   // c0 of face m+2
                 + P[1 * G.fmax + fc + fstride]     // c1 of face m+1
                 + P[2 * G.fmax + fc]               // c2 of face m
                 + P[3 * G.fmax + fc - fstride];    // c3 of face m-1
      if (lo_trans && gcell == 0) {
        // ghosts -2, -1 are copies of cell 0: face 0 sends c0 (cell -2) and c1
        // (cell -1), face 1 sends c0 (cell -1)
        s += P[0 * G.fmax + fc] + P[1 * G.fmax + fc] + P[0 * G.fmax + fc + fstride];
      }
      if (hi_trans && gcell == nD - 1) {
        // ghosts n, n+1 are copies of cell n-1: face n sends c2 (cell n) and c3
        // (cell n+1), face n-1 sends c3 (cell n)
        s += P[2 * G.fmax + fc + fstride] + P[3 * G.fmax + fc + fstride] + P[3 * G.fmax + fc];
      }
      if (D == 0)
        acc[v * G.cells + c] = scale * s;
      else
        acc[v * G.cells + c] = fma(scale, s, acc[v * G.cells + c]);
    }
  }
  __syncthreads();
}

// Register budget: two CTAs of kAdjThreads2d threads per SM in 2D (170
// registers per thread for the reverse pass and its integer-pipe products);
// in 3D the 8x4x4 tile's shared memory (128 KB) allows one CTA per SM
// anyway, so the kernel may use the whole register file.
template <int DIM, bool HALF>
__global__ void __launch_bounds__(DIM == 2 ? kAdjThreads2d : 256, DIM == 2 ? 2 : 1) adjoint_kernel(const AdjArgs a) {
  constexpr int NV = DIM + 2;
  extern __shared__ unsigned char smem_raw[];
  double *Ubox = aligned_smem(smem_raw);
  const AdjGeom G = adj_geom(DIM, a.tile);
  double *Lbox = Ubox + NV * G.uplane;
  double *Fb = Lbox + NV * G.lplane;
  double *acc = Fb + 4 * NV * G.fmax;
  int b = blockIdx.x;
  const int bx = b % a.ntile[0];
  b /= a.ntile[0];
  const int by = b % a.ntile[1];
  const int bz = b / a.ntile[1];
  const int o[3] = {bx * a.tile[0], by * a.tile[1], DIM == 3 ? bz * a.tile[2] : 0};
  int ext[3];
  ext[0] = min(a.tile[0], a.n[0] - o[0]);
  ext[1] = min(a.tile[1], a.n[1] - o[1]);
  ext[2] = DIM == 3 ? min(a.tile[2], a.n[2] - o[2]) : 1;
  load_box<DIM>(Ubox, a.U, a, o, ext, 3, G.UX, G.UY, G.uplane, false);
  load_box<DIM>(Lbox, a.lam, a, o, ext, 2, G.LX, G.LY, G.lplane, true);
  __syncthreads();
#pragma unroll 1
  for (int D = 0; D < DIM; ++D) adj_face_pass<DIM, HALF>(Ubox, Lbox, Fb, acc, a, o, ext, G, a.scale[D], D);
  const long long N = (long long)a.n[0] * a.n[1] * a.n[2];
  const int ncell = ext[0] * ext[1] * ext[2];
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    const int i = c % ext[0], rr = c / ext[0], j = rr % ext[1], k = rr / ext[1];
    const long long gi = ((long long)(o[2] + k) * a.n[1] + (o[1] + j)) * a.n[0] + (o[0] + i);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double r = acc[v * G.cells + c];
      if (a.A) r = fma(a.cA, a.A[v * N + gi], r);
      if (a.B) r = fma(a.cB, a.B[v * N + gi], r);
      if (a.C) r = fma(a.cC, a.C[v * N + gi], r);
      a.out[v * N + gi] = r;
    }
  }
}

}  // namespace

size_t adjoint_smem_bytes(int dim, const int tile[3]) {
  const AdjGeom G = adj_geom(dim, tile);
  const int nv = dim + 2;
  return 128 + sizeof(double) * (size_t)nv * (G.uplane + G.lplane + 4 * G.fmax + G.cells);
}

template <int DIM, bool HALF>
cudaError_t launch_adjoint_kernel(const AdjArgs &a, unsigned blocks, int threads, size_t smem, cudaStream_t st) {
  const cudaError_t e = cudaFuncSetAttribute((const void *)adjoint_kernel<DIM, HALF>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) adjoint_kernel<DIM, HALF><<<blocks, threads, smem, st>>>(a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_adjoint(int dim, const AdjArgs &a, int threads, cudaStream_t st) {
  const size_t smem = adjoint_smem_bytes(dim, a.tile);
  const unsigned blocks = (unsigned)((long long)a.ntile[0] * a.ntile[1] * a.ntile[2]);
  const bool half = a.half_eps == 0.5;
  if (dim == 2)
    return half ? launch_adjoint_kernel<2, true>(a, blocks, threads, smem, st)
                : launch_adjoint_kernel<2, false>(a, blocks, threads, smem, st);
  return half ? launch_adjoint_kernel<3, true>(a, blocks, threads, smem, st)
              : launch_adjoint_kernel<3, false>(a, blocks, threads, smem, st);
}

}  // namespace fvk
