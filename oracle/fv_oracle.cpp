// C ABI of the CPU oracle: TEST INFRASTRUCTURE ONLY (see fv_oracle.hpp).
// Loaded through ctypes by the test suite, the smoke check and the benchmark's
// CPU-baseline leg; nothing on the GPU path links it.
#include "fv_oracle.hpp"

#include <atomic>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

// Forward-mode dual number: value and one directional derivative.
struct Dual {
  double v, d;
  Dual(double x = 0.0) : v(x), d(0.0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
  Dual &operator+=(const Dual &o) { v += o.v; d += o.d; return *this; }
  Dual &operator-=(const Dual &o) { v -= o.v; d -= o.d; return *this; }
};
inline double value(const Dual &x) { return x.v; }
inline Dual operator+(const Dual &a, const Dual &b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(const Dual &a, const Dual &b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(const Dual &a) { return Dual(-a.v, -a.d); }
inline Dual operator*(const Dual &a, const Dual &b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(const Dual &a, const Dual &b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline Dual operator*(double a, const Dual &b) { return Dual(a * b.v, a * b.d); }
inline Dual operator*(const Dual &a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual operator/(const Dual &a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual operator+(double a, const Dual &b) { return Dual(a + b.v, b.d); }
inline Dual operator-(double a, const Dual &b) { return Dual(a - b.v, -b.d); }
inline Dual sqrt(const Dual &a) { double r = std::sqrt(a.v); return Dual(r, a.d / (2.0 * r)); }
inline Dual fabs(const Dual &a) { return a.v < 0.0 ? -a : a; }

// A double that counts the floating-point operations applied to it (+, -, *,
// /, sqrt each count one; negation, fabs and comparisons count none).
struct OpCount { std::atomic<long> add{0}, mul{0}, div{0}, sqrt{0}; };
static OpCount g_ops;
struct Counted {
  double v;
  Counted(double x = 0.0) : v(x) {}
  Counted &operator+=(const Counted &o) { g_ops.add++; v += o.v; return *this; }
  Counted &operator-=(const Counted &o) { g_ops.add++; v -= o.v; return *this; }
};
inline double value(const Counted &x) { return x.v; }
inline Counted operator+(const Counted &a, const Counted &b) { g_ops.add++; return Counted(a.v + b.v); }
inline Counted operator-(const Counted &a, const Counted &b) { g_ops.add++; return Counted(a.v - b.v); }
inline Counted operator-(const Counted &a) { return Counted(-a.v); }
inline Counted operator*(const Counted &a, const Counted &b) { g_ops.mul++; return Counted(a.v * b.v); }
inline Counted operator/(const Counted &a, const Counted &b) { g_ops.div++; return Counted(a.v / b.v); }
inline Counted operator*(double a, const Counted &b) { g_ops.mul++; return Counted(a * b.v); }
inline Counted operator*(const Counted &a, double b) { g_ops.mul++; return Counted(a.v * b); }
inline Counted operator/(const Counted &a, double b) { g_ops.div++; return Counted(a.v / b); }
inline Counted operator+(double a, const Counted &b) { g_ops.add++; return Counted(a + b.v); }
inline Counted operator-(double a, const Counted &b) { g_ops.add++; return Counted(a - b.v); }
inline Counted sqrt(const Counted &a) { g_ops.sqrt++; return Counted(std::sqrt(a.v)); }
inline Counted fabs(const Counted &a) { return Counted(std::fabs(a.v)); }

}  // namespace orc

using namespace orc;

extern "C" {

// Spatial residual R_h of Eq. (5) (face areas included; S: the cell-averaged
// source, same layout as U, or NULL for S = 0).
// U, R: [nv][nz][ny][nx] float64.  Returns 0.
int orc_residual(const Grid *g, const Scheme *s, const double *U, double *R, const double *S) {
  residual(*g, *s, U, R, S);
  return 0;
}

// The residual evaluated in extended precision (long double: 64-bit or
// 113-bit significand depending on the host) from the same double inputs,
// for measuring the rounding error of FP64 evaluations.
// Per cell and variable, sum_d ds_d (|F_{k+1/2,d}| + |F_{k-1/2,d}|) + |Omega| |S|:
// the magnitude of the terms the residual of Eq. (5) adds up.
int orc_residual_terms(const Grid *g, const Scheme *s, const double *U, double *R, const double *S) {
  residual<double, true>(*g, *s, U, R, S);
  return 0;
}

int orc_residual_ext(const Grid *g, const Scheme *s, const double *U, double *R, const double *S) {
  Layout L(*g);
  size_t N = L.cells() * L.nv;
  std::vector<long double> X(N), Y(N);
  for (size_t c = 0; c < N; ++c) X[c] = U[c];
  residual(*g, *s, X.data(), Y.data(), S);
  for (size_t c = 0; c < N; ++c) R[c] = (double)Y[c];
  return 0;
}

// CFL time step; -1 when a cell is non-physical.
double orc_time_step(const Grid *g, const Scheme *s, const double *U) { return time_step(*g, *s, U); }

// One SSP-RK3 step in place.  dt <= 0: use the CFL step of U.
// Returns the dt used, or -1 when the state is non-physical.
double orc_rk3_step(const Grid *g, const Scheme *s, double *U, double dt, const double *S) {
  if (dt <= 0.0) dt = time_step(*g, *s, U);
  if (dt <= 0.0) return -1.0;
  rk3_step(*g, *s, U, dt, S);
  return dt;
}

// nsteps SSP-RK3 steps.  dt_fixed > 0 holds the step fixed; otherwise each step
// takes the CFL step of its starting state, and with t_end > 0 the last step
// is shortened to land on t_end (steps stop there).  Returns the time reached,
// or -1 when the state became non-physical.
double orc_run(const Grid *g, const Scheme *s, double *U, int nsteps, double dt_fixed, double t_end, const double *S) {
  double t = 0.0;
  for (int n = 0; n < nsteps; ++n) {
    if (t_end > 0.0 && t >= t_end) break;
    double dt = dt_fixed > 0.0 ? dt_fixed : time_step(*g, *s, U);
    if (dt <= 0.0) return -1.0;
    if (t_end > 0.0 && t + dt > t_end) dt = t_end - t;
    rk3_step(*g, *s, U, dt, S);
    t += dt;
  }
  return t;
}

}  // extern "C"

extern "C" {

// The residual of Eq. (5) at the listed cells (flat interior indices), equal
// to the matching entries of orc_residual.  S: the source of the whole grid,
// or NULL.  out: [ncells][nv].  Returns 0, or -1 for an index outside the grid.
static bool cells_in_grid(const Grid *g, long ncells, const long *cells) {
  Layout L(*g);
  for (long c = 0; c < ncells; ++c)
    if (cells[c] < 0 || cells[c] >= (long)L.cells()) return false;
  return true;
}

int orc_residual_cells(const Grid *g, const Scheme *s, const double *U, long ncells, const long *cells, double *out,
                       const double *S) {
  if (!cells_in_grid(g, ncells, cells)) return -1;
  residual_cells<double>(*g, *s, U, ncells, cells, out, S);
  return 0;
}

// The same in extended precision (long double), rounded to double at the end.
int orc_residual_cells_ext(const Grid *g, const Scheme *s, const double *U, long ncells, const long *cells,
                           double *out, const double *S) {
  if (!cells_in_grid(g, ncells, cells)) return -1;
  residual_cells<long double>(*g, *s, U, ncells, cells, out, S);
  return 0;
}

// Point functions for unit tests.
void orc_roe_flux(const Scheme *s, int dim, int d, const double *QL, const double *QR, double *F) {
  roe_flux(*s, dim, d, QL, QR, F);
}
void orc_physical_flux(const Scheme *s, int dim, int d, const double *Q, double *F) { physical_flux(*s, dim, d, Q, F); }
void orc_muscl(const Scheme *s, const double *q4, double *QL, double *QR) { muscl(*s, q4[0], q4[1], q4[2], q4[3], *QL, *QR); }

// Directional derivative (Jacobian-vector product) of the residual: dR = (dR/dU) dU.
int orc_residual_jvp(const Grid *g, const Scheme *s, const double *U, const double *dU, double *R, double *dR) {
  Layout L(*g);
  size_t N = L.cells() * L.nv;
  std::vector<Dual> X(N), Y(N);
  for (size_t c = 0; c < N; ++c) X[c] = Dual(U[c], dU[c]);
  residual(*g, *s, X.data(), Y.data());
  for (size_t c = 0; c < N; ++c) { if (R) R[c] = Y[c].v; dR[c] = Y[c].d; }
  return 0;
}

// Directional derivative of nsteps SSP-RK3 steps with a fixed dt:
// on return U holds the state after the steps and dU its derivative.
int orc_rk3_jvp(const Grid *g, const Scheme *s, double *U, double *dU, int nsteps, double dt) {
  Layout L(*g);
  size_t N = L.cells() * L.nv;
  std::vector<Dual> X(N);
  for (size_t c = 0; c < N; ++c) X[c] = Dual(U[c], dU[c]);
  for (int n = 0; n < nsteps; ++n) rk3_step(*g, *s, X.data(), dt);
  for (size_t c = 0; c < N; ++c) { U[c] = X[c].v; dU[c] = X[c].d; }
  return 0;
}

// Floating-point operations of one residual evaluation, one time-step
// evaluation and one SSP-RK3 step with a given dt, counted while running the
// oracle on U: counts[0..3] = (add/sub, mul, div, sqrt) per call type, laid
// out as [residual 4][time_step 4][rk3_step 4].
int orc_count_ops(const Grid *g, const Scheme *s, const double *U, double dt, long *counts) {
  Layout L(*g);
  size_t N = L.cells() * L.nv;
  std::vector<Counted> X(N), Y(N);
  for (size_t c = 0; c < N; ++c) X[c] = Counted(U[c]);
  auto grab = [&](long *dst) {
    dst[0] = g_ops.add.exchange(0);
    dst[1] = g_ops.mul.exchange(0);
    dst[2] = g_ops.div.exchange(0);
    dst[3] = g_ops.sqrt.exchange(0);
  };
  long dummy[4];
  grab(dummy);
  residual(*g, *s, X.data(), Y.data());
  grab(counts + 0);
  time_step(*g, *s, X.data());
  grab(counts + 4);
  rk3_step(*g, *s, X.data(), dt);
  grab(counts + 8);
  return 0;
}

// Threads the oracle's OpenMP loops use.
int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
