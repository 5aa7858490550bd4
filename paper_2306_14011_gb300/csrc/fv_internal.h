// Host/device shared definitions of libfv (internal; not part of the C ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/fv.h"

namespace fvk {

// Largest CTA of the 3D box-tiled stage kernel (its register budget).
constexpr int kStage3dMaxThreads = 192;
// 2D stage kernels are built twice: for CTAs of up to this many threads (two
// resident CTAs leave 170 registers per thread for the face runs and their
// integer-pipe products) and for larger CTAs up to 256 (128 registers).
constexpr int kStage2dMaxThreads = 192;
// CTA size of the 2D adjoint kernel (the 3D one takes 256).
constexpr int kAdjThreads2d = 192;
// Largest CTA of the split kernels (FV_SPLIT; their register budget).
constexpr int kSplitMaxThreads = 512;

// Work of one launch of the fused stage kernel.
enum StageMode : int {
  MODE_RESIDUAL = 0,  // out = R_h (Eq. (5), face areas included)
  MODE_STAGE1 = 1,    // out = Us + dt L(Us)
  MODE_STAGE2 = 2,    // out = 3/4 Un + 1/4 (Us + dt L(Us))
  MODE_STAGE3 = 3,    // out = 1/3 Un + 2/3 (Us + dt L(Us))
  MODE_FLUXDIFF = 4   // fd[d] = the axis-d flux differences F_{k+1/2} - F_{k-1/2} (no face areas)
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
  int march;           // 3D: 1 = x-y tiles marching along z in chunks of tile[2] planes
  long long tile_begin;  // first tile of this launch (linear tile index, x fastest)
  long long tile_count;  // tiles of this launch (0: all from tile_begin)
  const double *S;     // cell-averaged source of Eq. (5) (layout of U), or null
  double vol;          // cell volume |Omega| (with S)
  int limiter;         // FV_LIM_* of Eq. (6)
  int recon;           // FV_RECON_*: the variables Eq. (6) extrapolates
  double inv_g1;       // 1 / (gamma - 1) (primitive reconstruction)
  double cL, cR;       // unlimited kappa-scheme weights eps (1 -+ kappa) / 4
  double g1;           // gamma - 1
  double half_eps;     // eps / 2 (MUSCL slope weight)
  double efix;         // entropy-fix width / c~
  double inv2efix;     // 1 / (2 efix), 0 when efix = 0
  double ds[3];        // residual mode: face area per axis
  double inv_h[3];     // stage modes: 1 / dx_d
  const unsigned long long *smax;  // CFL mode: bits of max wave-speed sum, else null
  double cfl;          // CFL number (with smax)
  double dt_fixed;     // step when smax is null
  double *t_acc;       // stage 3: simulated time accumulator (one thread adds dt), or null
  unsigned *flags;     // device flags (FLAG_*)
  double *fd;          // flux-difference mode: [dim][nvar][cells] output
};

struct DtArgs {
  const double *U;
  long long ncells;
  int dim;
  double g1, gamma;
  double inv_h[3];
  unsigned long long *smax;  // atomicMax target (bits of a non-negative double)
  unsigned *flags;
  // FP32 pre-selection (bounded = 1): lbound receives the bits of the largest
  // certified lower bound of a cell's wave-speed sum; the exact pass then
  // evaluates in FP64 only the cells whose certified upper bound reaches it
  int bounded;
  unsigned *lbound;
  unsigned *chunk_hi;  // per 32-cell chunk: bits of its certified FP32 upper bound
  float g1f, gammaf, inv_hf[3];
};

// One problem of a batched context (2D).
struct BatchProblem {
  long long off;         // offset (doubles) of its SoA block in the packed state
  int n[2];              // cells along x, y
  int ntile[2];          // tiles along x, y
  int bc[3][2];          // FV_BC_* per axis side
  double inv_h[2];       // 1 / dx_d
  float inv_hf[2];       // 1 / dx_d in FP32 (time-step pre-selection)
  int bounded;           // 1: FP32 pre-selection of the time-step reduction applies
};

struct BatchArgs {
  const BatchProblem *prob;
  const int *tile_begin;   // [nprob + 1] first tile item of each problem
  const int *chunk_begin;  // [nprob + 1] first time-step chunk of each problem
  int nprob, total_tiles, total_chunks, nsteps;
  long long chunk_cells;    // cells per time-step item (a multiple of 32)
  unsigned *chunk_hi;       // [total_chunks][chunk_cells / 32] certified upper bound per 32-cell chunk
  int tile[2];
  double *U, *U1, *U2;           // packed states
  unsigned long long *smax;      // [2][nprob] bits of each problem's max wave-speed sum
  unsigned *lbound;              // [2][nprob] bits of its certified FP32 lower bound
  double *t_acc;                 // [nprob] simulated time, or null
  unsigned *flags;
  unsigned *bar_count, *bar_gen; // grid barrier words
  const CUtensorMap *tmaps;      // [3][nprob] tile-load maps over U, U1, U2 per problem, or null
  const int *tma_ok;             // [3][nprob] 1 where that map exists (else plain loads)
  double g1, gamma, half_eps, efix, inv2efix, cfl, dt_fixed;
  float g1f, gammaf;
};

// The split kernel structure (fv_launch.mode = FV_SPLIT): per axis a limiter
// kernel writing the MUSCL face states QL, QR and a flux kernel writing the
// Roe flux F, then source, right-hand-side and update
// kernels.  Face arrays of axis d are [nvar][nface[d]] with faces indexed x
// fastest over (n[0] + (d == 0)) x (n[1] + (d == 1)) x (n[2] + (d == 2)); face
// m along d lies between cells m - 1 and m.
struct SplitArgs {
  int dim;
  int n[3];
  int bc[3][2];
  long long ncells;
  long long nface[3];
  const double *Us;          // state whose residual is evaluated
  const double *Un;          // U^n for stages 2 and 3
  double *out;               // the next stage state (stage modes)
  double *QL[3], *QR[3];     // face states per axis
  double *F[3];              // Roe flux per axis
  double *R;                 // the residual (the output in residual mode)
  double *norm_part;         // residual mode: per-CTA partial sums of R_v^2 of the RHS kernel, or null
  const double *S;           // source of Eq. (5), or null
  double vol, inv_vol;       // |Omega| and 1 / |Omega|
  int limiter, recon;        // FV_LIM_*, FV_RECON_*
  double inv_g1, cL, cR, g1, half_eps, efix, inv2efix;
  double ds[3];              // face area per axis
  const unsigned long long *smax;  // CFL mode: bits of the max wave-speed sum, else null
  double cfl, dt_fixed;
  double *t_acc;             // stage 3: simulated time (one thread adds dt), or null
};
// Launch the split kernels of one residual evaluation (mode MODE_RESIDUAL) or
// RK stage: grid[k], threads[k] for slot k of FV_SK_* (grid 0: one item per
// thread).  *rhs_blocks receives the RHS kernel's CTA count (the number of
// norm partials).
cudaError_t launch_split(int mode, const SplitArgs &a, const int *grid, const int *threads, int *rhs_blocks,
                         cudaStream_t st);

// Adjoint (vector-Jacobian product) kernel: out = sum_d scale_d J_d(U)^T lam
// + cA A + cB B + cC C (A, B, C may be null).
struct AdjArgs {
  const double *U, *lam;
  double *out;
  const double *A, *B, *C;
  double cA, cB, cC;
  double scale[3];
  int n[3], tile[3], ntile[3], bc[3][2];
  double g1, half_eps, efix, inv2efix;
};
size_t adjoint_smem_bytes(int dim, const int tile[3]);
cudaError_t launch_adjoint(int dim, const AdjArgs &a, int threads, cudaStream_t st);

size_t batch_smem_bytes(const int tile[2]);
cudaError_t batch_max_blocks(int threads, size_t smem, int *blocks_per_sm);
cudaError_t launch_batch_run(const BatchArgs &b, int blocks, int threads, size_t smem, cudaStream_t st);

// Dynamic shared memory of a stage-kernel CTA for a tile shape.
size_t stage_smem_bytes(int dim, const int tile[3]);
// ... and of the z-marching 3D kernel (tile[2] = planes per chunk, unused here).
size_t march_smem_bytes(const int tile[3]);

// The z-marching 3D stage kernel (StageArgs.march = 1): launcher and the
// dynamic shared-memory attribute of its instantiations.
cudaError_t launch_march(int mode, const CUtensorMap *tmap, const StageArgs &a, int threads, cudaStream_t st);
cudaError_t set_march_attributes(size_t smem_optin);

// Kernel launchers (return the launch error).
cudaError_t launch_stage(int dim, int mode, const CUtensorMap *tmap, const StageArgs &a, int threads,
                         cudaStream_t st);
cudaError_t launch_dt(const DtArgs &a, int blocks, int threads, cudaStream_t st);
// SSP-RK3 stage 1 from the per-axis flux differences of the flux-difference
// mode (a.fd): a.out = a.Us + dt L(a.Us), bit for bit the fused stage-1 kernel.
cudaError_t launch_stage1_from_fd(int dim, const StageArgs &a, cudaStream_t st);
cudaError_t launch_dt_finalize(const unsigned long long *smax, double cfl, double *out, cudaStream_t st);
cudaError_t launch_norm_finalize(const double *part, int nparts, int nvar, double *out, cudaStream_t st);
cudaError_t launch_debug_math(const double *x, double *o1, double *o2, long n, cudaStream_t st);
// blocks x 256 threads, 8 chains of `iters` DFMA (kind 0) / DADD (kind 1) each; out: blocks x 256 doubles.
cudaError_t launch_fp64_stream(int kind, int blocks, int iters, double *out, cudaStream_t st);
cudaError_t launch_debug_bits(int op, const double *x, const double *y, double *out, long n, cudaStream_t st);
cudaError_t launch_debug_wait(int kind, unsigned long long limit_ns, unsigned *word, unsigned *flags,
                              cudaStream_t st);
// Raise the stage kernels' dynamic shared-memory limit to the device maximum
// (smem_optin = cudaDeviceProp::sharedMemPerBlockOptin of the current device).
cudaError_t stage_kernel_attributes(int dim, size_t smem_optin);

// Argument checks shared by the entry points (fv_api.cu).
// validate_grid: FV_OK or FV_EINVAL (dimension, extents, boundary pairs, size).
int validate_grid(const fv_grid *g);
// Where a caller's array lives: host memory (pageable or pinned; the call
// stages it), memory of device `dev` or managed memory (used in place), or
// memory of another GPU (rejected: the kernels would reach it only through
// peer access).
enum PtrKind { PTR_HOST = 0, PTR_DEVICE = 1, PTR_OTHER_DEVICE = 2 };
PtrKind pointer_kind(const void *p, int dev);

}  // namespace fvk

struct fv_ctx;
struct fv_launch;

namespace fvk {
// Tuner support (fv_api.cu).  ctx_work_state: copy U (device or host) into the
// context's staging buffer and return it, so timing runs never touch the
// caller's state.  ctx_time_launch: with launch l, one warm-up SSP-RK3 step
// then `steps` timed steps on Uw (CFL dt, direct launches), `repeats` times;
// *sec = median seconds per step.  Returns FV_EINVAL for an invalid l (nothing
// launched).  ctx_sm_count: multiprocessors of the context's device.
int ctx_work_state(fv_ctx *c, const double *U, double **Uw);
int ctx_time_launch(fv_ctx *c, double *Uw, const fv_launch *l, int steps, int repeats, double *sec);
int ctx_sm_count(const fv_ctx *c);
int ctx_validate_launch(const fv_ctx *c, const fv_launch *l);
int ctx_default_launch(const fv_ctx *c, fv_launch *l);
int ctx_dim(const fv_ctx *c);
}  // namespace fvk
