// CPU oracle for the finite-volume Euler solver: TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, obviously-correct FP64 restatement of the method, written from
// the paper's equations.  Only the test suite, the package's smoke check and the
// benchmark's CPU-baseline leg may load it; the GPU library never does, and the
// two share no code, headers or tables.
//
// What it computes (paper sections in brackets):
//   * conserved vector Q and the inviscid normal flux F_{i,n}      [Eq. (2)]
//   * MUSCL kappa-extrapolation of conserved variables to faces,
//     limiter Psi = minmod, eps and kappa as parameters              [Eq. (6)]
//   * Roe approximate Riemann flux with Harten's entropy fix on the
//     acoustic waves (the paper leaves the flux function unnamed)
//   * spatial residual R_h = sum over faces of F*ds - |Omega| S     [Eq. (5)]
//   * semi-discrete form |Omega| dU/dt + R_h = 0                    [Eq. (4)]
//     advanced with the three-stage SSP Runge-Kutta scheme of Shu-Osher
//     (the paper says "explicit Runge-Kutta", Sec. 3.2)
//   * a CFL time step (the paper: "provided stability conditions are met")
//
// Everything is templated on the scalar type T so that one source gives the
// FP64 reference (T = double), a forward-mode directional derivative
// (T = a dual number) and an operation count (T = a counting double).
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace orc {

enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1 };

struct Grid {
  int dim;           // 2 or 3
  int n[3];          // cells per axis; n[2] = 1 in 2D
  double len[3];     // domain extent per axis
  int bc[3][2];      // per axis, (low, high) side
};

enum { LIM_MINMOD = 0, LIM_VANLEER = 1, LIM_NONE = 2 };

struct Scheme {
  double gamma;  // ratio of specific heats (1.4)
  double cfl;    // CFL number of the time-step rule (0.5)
  double eps;    // MUSCL eps of Eq. (6): 1 -> second order
  double kappa;  // MUSCL kappa of Eq. (6): -1 -> fully upwind
  double efix;   // Harten entropy-fix width as a fraction of the Roe sound speed
  int limiter;   // Psi of Eq. (6): LIM_MINMOD, LIM_VANLEER or LIM_NONE (Psi = 1)
  int recon;     // variables Eq. (6) extrapolates: RECON_CONSERVED (Sec. 3.1) or RECON_PRIMITIVE
};
enum { RECON_CONSERVED = 0, RECON_PRIMITIVE = 1 };

// Primitive variables (rho, u_1..u_dim, p) of a conserved state
// (rho, m_1..m_dim, E), and back: u = m / rho, p = (gamma-1)(E - rho |u|^2 / 2).
template <class T>
void to_primitive(const Scheme &s, int dim, const T *q, T *w) {
  w[0] = q[0];
  T q2 = T(0.0);
  for (int a = 0; a < dim; ++a) {
    w[1 + a] = q[1 + a] / q[0];
    q2 = q2 + w[1 + a] * w[1 + a];
  }
  w[dim + 1] = (s.gamma - 1.0) * (q[dim + 1] - 0.5 * q[0] * q2);
}
template <class T>
void to_conserved(const Scheme &s, int dim, const T *w, T *q) {
  q[0] = w[0];
  T q2 = T(0.0);
  for (int a = 0; a < dim; ++a) {
    q[1 + a] = w[0] * w[1 + a];
    q2 = q2 + w[1 + a] * w[1 + a];
  }
  q[dim + 1] = w[dim + 1] / (s.gamma - 1.0) + 0.5 * w[0] * q2;
}

// ---------------------------------------------------------------- scalar helpers
inline double value(double x) { return x; }
inline double value(long double x) { return (double)x; }
using std::sqrt;
using std::fabs;

// Minmod of two slopes (the limiter of Eq. (6), in "limited difference" form):
// both positive -> the smaller, both negative -> the larger, otherwise 0.
template <class T>
T minmod(const T &a, const T &b) {
  if (value(a) > 0.0 && value(b) > 0.0) return value(a) < value(b) ? a : b;
  if (value(a) < 0.0 && value(b) < 0.0) return value(a) > value(b) ? a : b;
  return T(0.0);
}

// van Leer's limiter in limited-difference form: Psi(r) = (r + |r|) / (1 + |r|)
// with r = d_neighbour / d gives Psi(r) d = 2 d d_neighbour / (d + d_neighbour)
// when d and d_neighbour have one strict sign, else 0.
template <class T>
T vanleer(const T &a, const T &b) {
  if ((value(a) > 0.0 && value(b) > 0.0) || (value(a) < 0.0 && value(b) < 0.0)) return 2.0 * a * b / (a + b);
  return T(0.0);
}

// Psi^{+}_{k-1/2} times (Q_k - Q_{k-1}) and Psi^{-}_{k+1/2} times (Q_{k+1} - Q_k):
// Psi evaluated at r, the ratio of the neighbouring difference to this one,
// times this difference.  For minmod, Psi(r) = max(0, min(1, r)), the product
// equals minmod(d, d_neighbour) exactly; this division-free form avoids 0/0
// when a difference vanishes.  Without a limiter, Psi = 1.
template <class T>
T limited(int lim, const T &d, const T &d_neighbour) {
  if (lim == LIM_VANLEER) return vanleer(d, d_neighbour);
  if (lim == LIM_NONE) return d;
  return minmod(d, d_neighbour);
}

// MUSCL extrapolation, Eq. (6), for one scalar component on the stencil
// q0 = Q_{k-1}, q1 = Q_k, q2 = Q_{k+1}, q3 = Q_{k+2}; returns Q^L_{k+1/2} and
// Q^R_{k+1/2}.
template <class T>
void muscl(const Scheme &s, const T &q0, const T &q1, const T &q2, const T &q3, T &QL, T &QR) {
  T dm = q1 - q0;  // Q_k - Q_{k-1}
  T d0 = q2 - q1;  // Q_{k+1} - Q_k
  T dp = q3 - q2;  // Q_{k+2} - Q_{k+1}
  T psi_p_km = limited(s.limiter, dm, d0);  // Psi^+_{k-1/2} (Q_k - Q_{k-1})
  T psi_m_kp = limited(s.limiter, d0, dm);  // Psi^-_{k+1/2} (Q_{k+1} - Q_k)
  T psi_p_kp = limited(s.limiter, d0, dp);  // Psi^+_{k+1/2} (Q_{k+1} - Q_k)
  T psi_m_k3 = limited(s.limiter, dp, d0);  // Psi^-_{k+3/2} (Q_{k+2} - Q_{k+1})
  // Eq. (6); a term whose weight (1 -+ kappa) is zero is left out (with
  // kappa = -1 the two (1 + kappa) terms vanish), which changes no result.
  const double e4 = s.eps / 4.0, wm = 1.0 - s.kappa, wp = 1.0 + s.kappa;
  T sumL = T(0.0), sumR = T(0.0);
  if (wm != 0.0) { sumL = sumL + wm * psi_p_km; sumR = sumR + wm * psi_m_k3; }
  if (wp != 0.0) { sumL = sumL + wp * psi_m_kp; sumR = sumR + wp * psi_p_kp; }
  QL = q1 + e4 * sumL;
  QR = q2 - e4 * sumR;
}

// Inviscid flux normal to axis d (Eq. (2) with n = e_d) of conserved state Q.
template <class T>
void physical_flux(const Scheme &s, int dim, int d, const T *Q, T *F) {
  const int nv = dim + 2;
  T rho = Q[0];
  T u[3] = {T(0.0), T(0.0), T(0.0)};
  for (int i = 0; i < dim; ++i) u[i] = Q[1 + i] / rho;
  T q2 = T(0.0);
  for (int i = 0; i < dim; ++i) q2 = q2 + u[i] * u[i];
  T p = (s.gamma - 1.0) * (Q[nv - 1] - 0.5 * rho * q2);
  T vn = u[d];
  F[0] = rho * vn;
  for (int i = 0; i < dim; ++i) F[1 + i] = rho * u[i] * vn + (i == d ? p : T(0.0));
  F[nv - 1] = (Q[nv - 1] + p) * vn;  // rho h_t V_n with rho h_t = rho e_t + p
}

// Harten's entropy fix: |lambda| replaced by (lambda^2 + delta^2) / (2 delta)
// where |lambda| < delta.
template <class T>
T entropy_fixed_abs(const T &lambda, const T &delta) {
  T a = fabs(lambda);
  if (value(delta) > 0.0 && value(a) < value(delta)) return (lambda * lambda + delta * delta) / (2.0 * delta);
  return a;
}

// Roe's approximate Riemann flux across a face normal to axis d:
//   F = 1/2 (F(Q_L) + F(Q_R)) - 1/2 sum_w |lambda_w| alpha_w r_w
// with Roe (sqrt(rho)-weighted) averages, wave strengths alpha_w, eigenvalues
// lambda_w and right eigenvectors r_w of the Euler flux Jacobian at the Roe
// state.  Acoustic waves get Harten's entropy fix with delta = efix * c~.
template <class T>
void roe_flux(const Scheme &s, int dim, int d, const T *QL, const T *QR, T *F) {
  const int nv = dim + 2;
  const double g1 = s.gamma - 1.0;
  // primitive variables of each side
  T rhoL = QL[0], rhoR = QR[0];
  T uL[3] = {T(0.0), T(0.0), T(0.0)}, uR[3] = {T(0.0), T(0.0), T(0.0)};
  T q2L = T(0.0), q2R = T(0.0);
  for (int i = 0; i < dim; ++i) {
    uL[i] = QL[1 + i] / rhoL;
    uR[i] = QR[1 + i] / rhoR;
    q2L = q2L + uL[i] * uL[i];
    q2R = q2R + uR[i] * uR[i];
  }
  T pL = g1 * (QL[nv - 1] - 0.5 * rhoL * q2L);
  T pR = g1 * (QR[nv - 1] - 0.5 * rhoR * q2R);
  T HL = (QL[nv - 1] + pL) / rhoL;
  T HR = (QR[nv - 1] + pR) / rhoR;

  // Roe averages
  T sL = sqrt(rhoL), sR = sqrt(rhoR);
  T rho_t = sL * sR;
  T u_t[3] = {T(0.0), T(0.0), T(0.0)};
  T q2_t = T(0.0);
  for (int i = 0; i < dim; ++i) {
    u_t[i] = (sL * uL[i] + sR * uR[i]) / (sL + sR);
    q2_t = q2_t + u_t[i] * u_t[i];
  }
  T H_t = (sL * HL + sR * HR) / (sL + sR);
  T c_t = sqrt(g1 * (H_t - 0.5 * q2_t));
  T un_t = u_t[d];

  // jumps and wave strengths
  T drho = rhoR - rhoL;
  T dp = pR - pL;
  T du[3] = {T(0.0), T(0.0), T(0.0)};
  for (int i = 0; i < dim; ++i) du[i] = uR[i] - uL[i];
  T c2 = c_t * c_t;
  T alpha1 = (dp - rho_t * c_t * du[d]) / (2.0 * c2);  // u - c wave
  T alpha2 = drho - dp / c2;                            // entropy wave
  T alpha3 = (dp + rho_t * c_t * du[d]) / (2.0 * c2);  // u + c wave
  T beta[3];                                            // shear waves
  for (int i = 0; i < dim; ++i) beta[i] = rho_t * du[i];

  // eigenvalues, with the entropy fix on the acoustic pair
  T delta = s.efix * c_t;
  T l1 = entropy_fixed_abs(un_t - c_t, delta);
  T l2 = fabs(un_t);
  T l3 = entropy_fixed_abs(un_t + c_t, delta);

  // right eigenvectors
  T r1[5], r2[5], r3[5];
  r1[0] = T(1.0);
  r2[0] = T(1.0);
  r3[0] = T(1.0);
  for (int i = 0; i < dim; ++i) {
    r1[1 + i] = u_t[i] - (i == d ? c_t : T(0.0));
    r2[1 + i] = u_t[i];
    r3[1 + i] = u_t[i] + (i == d ? c_t : T(0.0));
  }
  r1[nv - 1] = H_t - un_t * c_t;
  r2[nv - 1] = 0.5 * q2_t;
  r3[nv - 1] = H_t + un_t * c_t;

  T FL[5], FR[5];
  physical_flux(s, dim, d, QL, FL);
  physical_flux(s, dim, d, QR, FR);

  for (int k = 0; k < nv; ++k) {
    T diss = l1 * alpha1 * r1[k] + l2 * alpha2 * r2[k] + l3 * alpha3 * r3[k];
    // shear wave for tangential direction i: r = (0, e_i, u~_i)
    for (int i = 0; i < dim; ++i) {
      if (i == d) continue;
      T ri = (k == 1 + i) ? T(1.0) : (k == nv - 1 ? u_t[i] : T(0.0));
      diss = diss + l2 * beta[i] * ri;
    }
    F[k] = 0.5 * (FL[k] + FR[k]) - 0.5 * diss;
  }
}

// ---------------------------------------------------------------- grid helpers
struct Layout {
  int dim, nv;
  int n[3];      // interior cells (n[2] = 1 in 2D)
  int ng[3];     // ghost layers per axis (2 on active axes, 0 on the z axis in 2D)
  int m[3];      // padded extents
  double h[3];   // spacing
  explicit Layout(const Grid &g) {
    dim = g.dim;
    nv = g.dim + 2;
    for (int a = 0; a < 3; ++a) {
      n[a] = (a < dim) ? g.n[a] : 1;
      ng[a] = (a < dim) ? 2 : 0;
      m[a] = n[a] + 2 * ng[a];
      h[a] = (a < dim) ? g.len[a] / g.n[a] : 1.0;
    }
  }
  size_t cells() const { return (size_t)n[0] * n[1] * n[2]; }
  size_t padded() const { return (size_t)m[0] * m[1] * m[2]; }
  // interior index of cell (i, j, k) in U[v][k][j][i]
  size_t idx(int v, int i, int j, int k) const { return (((size_t)v * n[2] + k) * n[1] + j) * n[0] + i; }
  // padded index; i, j, k are interior coordinates (may be -2 .. n+1)
  size_t pidx(int v, int i, int j, int k) const {
    return (((size_t)v * m[2] + (k + ng[2])) * m[1] + (j + ng[1])) * m[0] + (i + ng[0]);
  }
};

// Index of the interior cell that ghost coordinate c (-2..n+1) on an axis with
// n cells maps to: periodic wrap, or the nearest interior cell (transmissive,
// a zero-gradient extrapolation).
inline int ghost_source(int c, int n, const int bc[2]) {
  if (c < 0) return bc[0] == BC_PERIODIC ? ((c % n) + n) % n : 0;
  if (c >= n) return bc[1] == BC_PERIODIC ? c % n : n - 1;
  return c;
}

// Copy the interior state into a ghost-padded array and fill 2 ghost layers on
// every active axis.  (Corner ghosts are filled too but never read: every face
// stencil runs along a single axis.)
template <class T>
void pad(const Grid &g, const Layout &L, const T *U, std::vector<T> &P) {
  P.assign(L.padded() * L.nv, T(0.0));
  for (int v = 0; v < L.nv; ++v)
    for (int k = -L.ng[2]; k < L.n[2] + L.ng[2]; ++k)
      for (int j = -L.ng[1]; j < L.n[1] + L.ng[1]; ++j)
        for (int i = -L.ng[0]; i < L.n[0] + L.ng[0]; ++i) {
          int si = ghost_source(i, L.n[0], g.bc[0]);
          int sj = ghost_source(j, L.n[1], g.bc[1]);
          int sk = (L.dim == 3) ? ghost_source(k, L.n[2], g.bc[2]) : k;
          P[L.pidx(v, i, j, k)] = U[L.idx(v, si, sj, sk)];
        }
}

// Flux across the face between Q_k and Q_{k+1} normal to axis d, from the
// four-cell stencil q = (Q_{k-1}, Q_k, Q_{k+1}, Q_{k+2}) along that axis:
// the MUSCL face states of Eq. (6), applied to each conserved component
// (Sec. 3.1) or, with RECON_PRIMITIVE, to (rho, u, p) and converted back to
// conserved variables, then the Roe flux between them.
template <class T>
void stencil_flux(const Scheme &s, int dim, int d, const T (&q)[4][5], T *F) {
  const int nv = dim + 2;
  T QL[5], QR[5];
  if (s.recon == RECON_PRIMITIVE) {
    T w[4][5], WL[5], WR[5];
    for (int m = 0; m < 4; ++m) to_primitive(s, dim, q[m], w[m]);
    for (int v = 0; v < nv; ++v) muscl(s, w[0][v], w[1][v], w[2][v], w[3][v], WL[v], WR[v]);
    to_conserved(s, dim, WL, QL);
    to_conserved(s, dim, WR, QR);
  } else {
    for (int v = 0; v < nv; ++v) muscl(s, q[0][v], q[1][v], q[2][v], q[3][v], QL[v], QR[v]);
  }
  roe_flux(s, dim, d, QL, QR, F);
}

// Spatial residual of Eq. (5): for every cell,
//   R_k = sum over its faces of F.n ds - |Omega| S_k
//       = sum_d ds_d (F_{k+1/2,d} - F_{k-1/2,d}) - |Omega| S_k,
// where ds_d is the area of a face normal to axis d (dy in 2D for x-faces,
// dy*dz in 3D), F_{k+1/2,d} the Roe flux between the MUSCL states of Eq. (6)
// (inviscid: no viscous flux) and S the cell-averaged source (S = NULL: 0).
// Each face flux is evaluated once, stored, and read by both cells that share it.
// TERMS = true instead accumulates the magnitudes of the terms that sum:
// sum_d ds_d (|F_{k+1/2,d}| + |F_{k-1/2,d}|) + |Omega| |S_k| (the scale of
// the residual's rounding error, the tolerance floor for residuals that vanish).
template <class T, bool TERMS = false>
void residual(const Grid &g, const Scheme &s, const T *U, T *R, const double *S = nullptr) {
  Layout L(g);
  std::vector<T> P;
  pad(g, L, U, P);
  const int nv = L.nv;
  const long ncell = (long)L.cells();
  for (long c = 0; c < ncell * nv; ++c) R[c] = T(0.0);
  for (int d = 0; d < L.dim; ++d) {
    double ds = 1.0;
    for (int a = 0; a < L.dim; ++a)
      if (a != d) ds *= L.h[a];
    int e[3] = {0, 0, 0};
    e[d] = 1;
    // face f (0 .. n_d) along axis d lies between cells f-1 and f
    int fn[3] = {L.n[0], L.n[1], L.n[2]};
    fn[d] += 1;
    const long nface = (long)fn[0] * fn[1] * fn[2];
    std::vector<T> F((size_t)nface * nv);
#pragma omp parallel for schedule(static)
    for (long f = 0; f < nface; ++f) {
      int i = (int)(f % fn[0]), j = (int)((f / fn[0]) % fn[1]), k = (int)(f / ((long)fn[0] * fn[1]));
      // the cells left of the face: (i,j,k) - e_d
      int a = i - e[0], b = j - e[1], c = k - e[2];
      T q[4][5], Ff[5];  // the stencil Q_{k-1}, Q_k, Q_{k+1}, Q_{k+2}
      for (int v = 0; v < nv; ++v) {
        q[0][v] = P[L.pidx(v, a - e[0], b - e[1], c - e[2])];
        q[1][v] = P[L.pidx(v, a, b, c)];
        q[2][v] = P[L.pidx(v, i, j, k)];
        q[3][v] = P[L.pidx(v, i + e[0], j + e[1], k + e[2])];
      }
      stencil_flux(s, L.dim, d, q, Ff);
      for (int v = 0; v < nv; ++v) F[(size_t)v * nface + f] = Ff[v];
    }
#pragma omp parallel for schedule(static)
    for (long cidx = 0; cidx < ncell; ++cidx) {
      int i = (int)(cidx % L.n[0]), j = (int)((cidx / L.n[0]) % L.n[1]), k = (int)(cidx / ((long)L.n[0] * L.n[1]));
      long lo = ((long)k * fn[1] + j) * fn[0] + i;                             // face k-1/2
      long hi = ((long)(k + e[2]) * fn[1] + (j + e[1])) * fn[0] + (i + e[0]);  // face k+1/2
      for (int v = 0; v < nv; ++v) {
        const T Fh = F[(size_t)v * nface + hi], Fl = F[(size_t)v * nface + lo];
        if constexpr (TERMS)
          R[(size_t)v * ncell + cidx] += (std::fabs(Fh) + std::fabs(Fl)) * ds;
        else
          R[(size_t)v * ncell + cidx] += (Fh - Fl) * ds;
      }
    }
  }
  if (S) {
    double vol = 1.0;
    for (int a = 0; a < L.dim; ++a) vol *= L.h[a];
    for (long c = 0; c < ncell * nv; ++c) {
      if constexpr (TERMS)
        R[c] = R[c] + vol * std::fabs(T(S[c]));
      else
        R[c] = R[c] - vol * T(S[c]);
    }
  }
}

// The residual of Eq. (5) at a list of cells only (flat interior indices
// k*ny*nx + j*nx + i), for sampled checks on grids too large for the full
// residual.  Per cell and axis it evaluates the two faces k-1/2 and k+1/2
// from their stencils, each cell of which is read through the boundary map
// (no ghost-padded copy of the grid), and sums the differences in the order
// `residual` does, so both give the same doubles.  S: the cell-averaged
// source of the whole grid (layout of U) or NULL.  out: [ncells][nv].
template <class T>
void residual_cells(const Grid &g, const Scheme &s, const double *U, long ncells, const long *cells, double *out,
                    const double *S = nullptr) {
  Layout L(g);
  const int nv = L.nv;
  double vol = 1.0;
  for (int a = 0; a < L.dim; ++a) vol *= L.h[a];
#pragma omp parallel for schedule(dynamic, 64)
  for (long c = 0; c < ncells; ++c) {
    const long id = cells[c];
    const int i = (int)(id % L.n[0]), j = (int)((id / L.n[0]) % L.n[1]);
    const int k = (int)(id / ((long)L.n[0] * L.n[1]));
    T R[5] = {T(0.0), T(0.0), T(0.0), T(0.0), T(0.0)};
    for (int d = 0; d < L.dim; ++d) {
      double ds = 1.0;
      for (int a = 0; a < L.dim; ++a)
        if (a != d) ds *= L.h[a];
      T Fside[2][5];
      for (int side = 0; side < 2; ++side) {  // side 0: face k-1/2, side 1: face k+1/2
        // the face between cells k-1+side and k+side has the stencil
        // k-2+side .. k+1+side along axis d
        T q[4][5];
        for (int t = 0; t < 4; ++t) {
          int c3[3] = {i, j, k};
          c3[d] += side + t - 2;
          const int si = ghost_source(c3[0], L.n[0], g.bc[0]);
          const int sj = ghost_source(c3[1], L.n[1], g.bc[1]);
          const int sk = (L.dim == 3) ? ghost_source(c3[2], L.n[2], g.bc[2]) : 0;
          for (int v = 0; v < nv; ++v) q[t][v] = T(U[L.idx(v, si, sj, sk)]);
        }
        stencil_flux(s, L.dim, d, q, Fside[side]);
      }
      for (int v = 0; v < nv; ++v) R[v] += (Fside[1][v] - Fside[0][v]) * ds;
    }
    if (S)
      for (int v = 0; v < nv; ++v) R[v] = R[v] - vol * T(S[(size_t)v * L.cells() + (size_t)id]);
    for (int v = 0; v < nv; ++v) out[c * nv + v] = value(R[v]);
  }
}

// Largest stable time step of the explicit scheme,
//   dt = CFL / max_k sum_d (|u_d| + c) / dx_d,   c = sqrt(gamma p / rho).
// Returns -1 if any cell has rho <= 0, p <= 0 or a NaN.
template <class T>
double time_step(const Grid &g, const Scheme &s, const T *U) {
  Layout L(g);
  double smax = 0.0;
  bool bad = false;
  for (int k = 0; k < L.n[2]; ++k)
    for (int j = 0; j < L.n[1]; ++j)
      for (int i = 0; i < L.n[0]; ++i) {
        T rho = U[L.idx(0, i, j, k)];
        T q2 = T(0.0), u[3] = {T(0.0), T(0.0), T(0.0)};
        for (int a = 0; a < L.dim; ++a) {
          u[a] = U[L.idx(1 + a, i, j, k)] / rho;
          q2 = q2 + u[a] * u[a];
        }
        T p = (s.gamma - 1.0) * (U[L.idx(L.nv - 1, i, j, k)] - 0.5 * rho * q2);
        if (!(value(rho) > 0.0) || !(value(p) > 0.0)) { bad = true; continue; }
        T c = sqrt(s.gamma * p / rho);
        T sum = T(0.0);
        for (int a = 0; a < L.dim; ++a) sum = sum + (fabs(u[a]) + c) / L.h[a];
        if (value(sum) > smax) smax = value(sum);
      }
  if (bad) return -1.0;
  return s.cfl / smax;
}

// One step of the three-stage SSP Runge-Kutta scheme applied to Eq. (4),
// dU/dt = L(U) = -R_h(U) / |Omega|:
//   U1 = U + dt L(U)
//   U2 = 3/4 U + 1/4 (U1 + dt L(U1))
//   U  = 1/3 U + 2/3 (U2 + dt L(U2))
template <class T>
void rk3_step(const Grid &g, const Scheme &s, T *U, double dt, const double *S = nullptr) {
  Layout L(g);
  const size_t N = L.cells() * L.nv;
  double vol = 1.0;
  for (int a = 0; a < L.dim; ++a) vol *= L.h[a];
  std::vector<T> R(N), U1(N), U2(N);
  residual(g, s, U, R.data(), S);
  for (size_t c = 0; c < N; ++c) U1[c] = U[c] + dt * (-R[c] / vol);
  residual(g, s, U1.data(), R.data(), S);
  for (size_t c = 0; c < N; ++c) U2[c] = 0.75 * U[c] + 0.25 * (U1[c] + dt * (-R[c] / vol));
  residual(g, s, U2.data(), R.data(), S);
  for (size_t c = 0; c < N; ++c) U[c] = (1.0 / 3.0) * U[c] + (2.0 / 3.0) * (U2[c] + dt * (-R[c] / vol));
}

}  // namespace orc
