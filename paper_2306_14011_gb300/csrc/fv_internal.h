// Host/device shared definitions of libfv (internal; not part of the C ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

namespace fvk {

// Work of one launch of the fused stage kernel.
enum StageMode : int {
  MODE_RESIDUAL = 0,  // out = R_h (Eq. (5), face areas included)
  MODE_STAGE1 = 1,    // out = Us + dt L(Us)
  MODE_STAGE2 = 2,    // out = 3/4 Un + 1/4 (Us + dt L(Us))
  MODE_STAGE3 = 3     // out = 1/3 Un + 2/3 (Us + dt L(Us))
};

struct StageArgs {
  const double *Us;    // state whose residual is evaluated (SoA, interior cells)
  const double *Un;    // U^n for stages 2 and 3
  double *out;         // residual or next state (must not alias Us)
  double *norm_part;   // residual mode: per-CTA partial sums of R_v^2, or null
  int n[3];            // cells per axis (n[2] = 1 in 2D)
  int tile[3];         // cells per CTA tile (tile[2] = 1 in 2D)
  int ntile[3];        // tiles per axis
  int bc[3][2];        // FV_BC_* per axis side
  int use_tma;         // 1: stage tiles with TMA (tensor map valid), 0: plain loads
  double g1;           // gamma - 1
  double half_eps;     // eps / 2 (MUSCL slope weight)
  double efix;         // entropy-fix width / c~
  double inv2efix;     // 1 / (2 efix), 0 when efix = 0
  double half_ds[3];   // residual mode: face area / 2 per axis
  double half_inv_h[3];  // stage modes: 1 / (2 dx_d)
  const unsigned long long *smax;  // CFL mode: bits of max wave-speed sum, else null
  double cfl;          // CFL number (with smax)
  double dt_fixed;     // step when smax is null
  double *t_acc;       // stage 3: simulated time accumulator (one thread adds dt), or null
  unsigned *flags;     // device flags (FLAG_*)
};

struct DtArgs {
  const double *U;
  long long ncells;
  int dim;
  double g1, gamma;
  double inv_h[3];
  unsigned long long *smax;  // atomicMax target (bits of a non-negative double)
  unsigned *flags;
};

// Dynamic shared memory of a stage-kernel CTA for a tile shape.
size_t stage_smem_bytes(int dim, const int tile[3]);

// Kernel launchers (return the launch error).
cudaError_t launch_stage(int dim, int mode, const CUtensorMap *tmap, const StageArgs &a, int threads,
                         cudaStream_t st);
cudaError_t launch_dt(const DtArgs &a, int blocks, int threads, cudaStream_t st);
cudaError_t launch_dt_finalize(const unsigned long long *smax, double cfl, double *out, cudaStream_t st);
cudaError_t launch_norm_finalize(const double *part, int nparts, int nvar, double *out, cudaStream_t st);
cudaError_t launch_debug_math(const double *x, double *o1, double *o2, long n, cudaStream_t st);
// Raise the stage kernels' dynamic shared-memory limit to the device maximum
// (smem_optin = cudaDeviceProp::sharedMemPerBlockOptin of the current device).
cudaError_t stage_kernel_attributes(int dim, size_t smem_optin);

}  // namespace fvk
