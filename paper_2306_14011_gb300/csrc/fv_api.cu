// Host side of the libfv C ABI (declared in include/fv.h): contexts, argument
// validation, TMA tensor maps, host-pointer staging and the CUDA-graph step
// driver.  Every numerical step runs in the kernels of fv_stage*.cu and
// fv_reduce.cu.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/fv.h"
#include "fv_device.cuh"
#include "fv_internal.h"

using namespace fvk;

namespace {

#define FV_CK(call)                                 \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(e_);    \
  } while (0)

int cuda_fail(cudaError_t e) {
  (void)cudaGetLastError();  // clear a sticky launch error so the next call can proceed
  return e == cudaErrorMemoryAllocation ? FV_ENOMEM : FV_ECUDA;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

typedef CUresult (*PointerAttributeFn)(void *, CUpointer_attribute, CUdeviceptr);

PointerAttributeFn pointer_attribute_fn() {
  static PointerAttributeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PointerAttributeFn>(p);
  });
  return fn;
}

// The device address of host memory [p, p + bytes) when the whole range lies
// in one page-locked allocation mapped into the current device's address
// space, so that kernels may store to it directly; nullptr otherwise
// (pageable memory, or a range the CUDA driver does not report as one allocation).
double *mapped_host_range(double *p, size_t bytes) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
  PointerAttributeFn get = pointer_attribute_fn();
  if (!get) return nullptr;
  CUdeviceptr start = 0;
  size_t size = 0;
  const CUdeviceptr d = reinterpret_cast<CUdeviceptr>(at.devicePointer);
  if (get(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, d) != CUDA_SUCCESS ||
      get(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, d) != CUDA_SUCCESS)
    return nullptr;
  if (d < start || bytes > size || d - start > size - bytes) return nullptr;
  return static_cast<double *>(at.devicePointer);
}

}  // namespace

namespace fvk {

int validate_grid(const fv_grid *g) {
  if (!g || (g->dim != 2 && g->dim != 3)) return FV_EINVAL;
  for (int d = 0; d < 3; ++d) {
    const bool active = d < g->dim;
    if (active) {
      if (g->n[d] < 1 || !(g->len[d] > 0.0)) return FV_EINVAL;
      for (int s = 0; s < 2; ++s)
        if (g->bc[d][s] != FV_BC_PERIODIC && g->bc[d][s] != FV_BC_TRANSMISSIVE) return FV_EINVAL;
      if ((g->bc[d][0] == FV_BC_PERIODIC) != (g->bc[d][1] == FV_BC_PERIODIC)) return FV_EINVAL;
    } else if (g->n[d] != 1) {
      return FV_EINVAL;
    }
  }
  const long long cells = (long long)g->n[0] * g->n[1] * g->n[2];
  if (cells * (g->dim + 2) >= (1ll << 40)) return FV_EINVAL;
  return FV_OK;
}

PtrKind pointer_kind(const void *p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return PTR_HOST;
  }
  if (at.type == cudaMemoryTypeManaged) return PTR_DEVICE;
  if (at.type == cudaMemoryTypeDevice) return at.device == dev ? PTR_DEVICE : PTR_OTHER_DEVICE;
  return PTR_HOST;
}

}  // namespace fvk

namespace {

struct GraphEntry {
  const double *U;
  long long dt_bits;  // fixed dt bits, or 0 for CFL steps
  int steps;
  cudaGraphExec_t exec;
  void *aux = nullptr;  // device memory the graph reads (batched tile-load maps), freed with it
};

}  // namespace

struct fv_ctx {
  fv_grid grid;
  fv_scheme scheme;
  fv_launch launch;
  cudaStream_t stream;
  cudaStream_t cap;  // capture stream for graphs
  int device, sms;
  size_t smem_optin;
  int nv;
  long long ncells;
  size_t state_bytes;
  double *U1, *U2;            // RK stage buffers
  double *stage_in, *stage_out;  // host-pointer staging (lazy)
  unsigned long long *smax;   // scratch: bits of the max wave-speed sum
  unsigned *lbound;           // scratch: bits of its certified FP32 lower bound
  unsigned *chunk_hi;         // per 32-cell chunk: bits of its certified upper bound
  unsigned *flags;            // scratch: device flags
  double *t_acc;              // scratch: simulated time
  double *dt_dev;             // scratch: dt for device outputs
  double *norm_out;           // scratch: nvar norms
  double *norm_part;          // scratch: per-CTA partials (lazy)
  long long norm_part_cap;
  double *X1, *X2;            // adjoint work states (lazy)
  double *split_buf;          // FV_SPLIT face states, fluxes and residual (lazy)
  double *fd;                 // host-state runs: per-axis flux differences of the first stage (lazy)
  std::vector<cudaEvent_t> h2d_events;  // host-state runs: per-band copy-in events (lazy)
  std::vector<GraphEntry> graphs;
  const double *source;        // caller's cell-averaged source of Eq. (5), or null
  // host-pointer runs: copy-back stream and per-band events (lazy)
  cudaStream_t copy_stream;
  cudaStream_t aux_stream;  // host-state runs: second stream of the first stage's bands (lazy)
  std::vector<cudaEvent_t> band_events;
  // batched contexts (ngrids > 1)
  int ngrids;
  std::vector<fv_grid> grids;
  std::vector<long long> offsets;  // ngrids + 1, in doubles
  BatchProblem *b_prob;
  int *b_tile_begin, *b_chunk_begin;
  unsigned long long *b_smax;      // [2][ngrids], then the FP32 lower bounds [2][ngrids]
  double *b_tacc;                  // [ngrids]
  unsigned *b_bar;                 // count, generation
  unsigned *b_chunk_hi;            // per 32-cell chunk of each time-step item: its certified upper bound
  int b_total_tiles, b_total_chunks, b_blocks;
};

namespace {

// Shared memory the stage kernels declare statically (the residual kernel's
// norm reduction buffer, 5 x 32 doubles), kept free of the dynamic budget.
constexpr size_t kStaticSmemReserve = 2048;

// *host: whether p is host memory (staged by the call).  FV_EINVAL for memory
// of a GPU other than the context's.
int where(const fv_ctx *c, const void *p, bool *host) {
  const PtrKind k = pointer_kind(p, c->device);
  *host = k == PTR_HOST;
  return k == PTR_OTHER_DEVICE ? FV_EINVAL : FV_OK;
}

int validate_scheme(const fv_scheme *s) {
  if (!s || !(s->gamma > 1.0) || !(s->cfl > 0.0) || !(s->eps >= 0.0) || !(s->eps <= 2.0) || !(s->efix >= 0.0) ||
      !(s->efix < 1.0))
    return FV_EINVAL;
  if (s->limiter != FV_LIM_MINMOD && s->limiter != FV_LIM_VANLEER && s->limiter != FV_LIM_NONE) return FV_EINVAL;
  if (s->recon != FV_RECON_CONSERVED && s->recon != FV_RECON_PRIMITIVE) return FV_EINVAL;
  return FV_OK;
}

int validate_launch(const fv_grid *g, const fv_scheme *sch, const fv_launch *l, size_t smem_optin) {
  if (l->mode != FV_FUSED && l->mode != FV_SPLIT) return FV_EINVAL;
  if (l->mode == FV_SPLIT)
    for (int k = 0; k < FV_SK_COUNT; ++k) {
      const fv_kernel_cfg &q = l->split[k];
      if (q.threads < 32 || q.threads > kSplitMaxThreads || q.threads % 32 || q.grid < 0) return FV_EINVAL;
    }
  for (int s = 0; s < 3; ++s) {
    const fv_kernel_cfg &k = l->stage[s];
    if (k.march != 0 && (k.march != 1 || g->dim != 3)) return FV_EINVAL;
    if (k.march && sch->recon != FV_RECON_CONSERVED) return FV_EINVAL;  // z-marching: conserved only
    for (int d = 0; d < 3; ++d) {
      if (d == 2 && k.march) {
        if (k.tile[2] < 1 || k.tile[2] > (1 << 24)) return FV_EINVAL;  // planes per chunk
      } else if (d < g->dim) {
        if (k.tile[d] < 2 || k.tile[d] > 252) return FV_EINVAL;
      } else if (k.tile[d] != 1) {
        return FV_EINVAL;
      }
    }
    if (k.tile[0] % 2) return FV_EINVAL;  // TMA boxes start on 16-byte boundaries
    if (k.threads < 32 || k.threads > 256 || k.threads % 32) return FV_EINVAL;
    if (g->dim == 3 && !k.march && k.threads > kStage3dMaxThreads) return FV_EINVAL;
    if (k.grid != 0) return FV_EINVAL;  // tiled kernels cover the domain
    if (k.loader != FV_LOADER_TMA && k.loader != FV_LOADER_PLAIN) return FV_EINVAL;
    const size_t smem = k.march ? march_smem_bytes(k.tile) : stage_smem_bytes(g->dim, k.tile);
    if (smem + kStaticSmemReserve > smem_optin) return FV_EINVAL;
  }
  if (l->dt.threads < 32 || l->dt.threads > 1024 || l->dt.threads % 32 || l->dt.grid < 0) return FV_EINVAL;
  return FV_OK;
}

void ntiles(const fv_grid &g, const int tile[3], int nt[3]) {
  for (int d = 0; d < 3; ++d) nt[d] = (d < g.dim) ? (g.n[d] + tile[d] - 1) / tile[d] : 1;
}

// TMA tensor map over the state array U (nv variables) of grid g: dims
// (x, y[, z], var), box = tile + halo (one z-plane for the z-marching kernel).
bool make_tmap_grid(const fv_grid &g, int nv, const double *U, const int tile[3], int march, CUtensorMap *map) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  if (g.n[0] % 2) return false;                          // row stride must be a multiple of 16 bytes
  if (reinterpret_cast<uintptr_t>(U) % 16) return false;  // base address alignment
  const int box[3] = {tile[0] + 4, tile[1] + 4, march ? 1 : tile[2] + 4};
  for (int d = 0; d < g.dim; ++d)
    if (box[d] > 256 || box[d] > g.n[d]) return false;
  cuuint64_t dims[4], strides[3];
  cuuint32_t boxd[4], estr[4] = {1, 1, 1, 1};
  const int rank = g.dim + 1;
  cuuint64_t stride = sizeof(double);
  for (int d = 0; d < g.dim; ++d) {
    dims[d] = (cuuint64_t)g.n[d];
    boxd[d] = (cuuint32_t)box[d];
    stride *= (cuuint64_t)g.n[d];
    strides[d] = stride;  // byte stride of dimension d+1
  }
  dims[g.dim] = (cuuint64_t)nv;
  boxd[g.dim] = (cuuint32_t)nv;
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, (cuuint32_t)rank, const_cast<double *>(U), dims, strides,
                   boxd, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_tmap(const fv_ctx *c, const double *U, const int tile[3], int march, CUtensorMap *map) {
  return make_tmap_grid(c->grid, c->nv, U, tile, march, map);
}

// Faces per axis of the split kernels: (n_d + 1) x the other extents.
long long split_faces(const fv_grid &g, int d) {
  long long f = 1;
  for (int a = 0; a < 3; ++a) f *= (long long)g.n[a] + (a == d && d < g.dim ? 1 : 0);
  return f;
}

int ensure_split(fv_ctx *c) {
  if (c->split_buf) return FV_OK;
  size_t doubles = (size_t)c->nv * (size_t)c->ncells;  // residual
  for (int d = 0; d < c->grid.dim; ++d) doubles += 3 * (size_t)c->nv * (size_t)split_faces(c->grid, d);
  FV_CK(cudaMalloc(&c->split_buf, sizeof(double) * doubles));
  return FV_OK;
}

// CTAs of the split RHS kernel (= its norm partials) for the current launch.
long long split_rhs_blocks(const fv_ctx *c) {
  const fv_kernel_cfg &k = c->launch.split[FV_SK_RHS];
  long long b = k.grid > 0 ? k.grid : (c->ncells + k.threads - 1) / k.threads;
  return std::min<long long>(std::max<long long>(b, 1), 0x7fffffffLL);
}

// One residual evaluation or RK stage with the split kernels (FV_SPLIT).
int split_stage(fv_ctx *c, int mode, const double *Us, const double *Un, double *out,
                const unsigned long long *smax, double dt_fixed, double *norm_part, double *t_acc, cudaStream_t st) {
  int r;
  if ((r = ensure_split(c))) return r;
  const fv_grid &g = c->grid;
  SplitArgs a;
  memset(&a, 0, sizeof(a));
  a.dim = g.dim;
  a.ncells = c->ncells;
  for (int d = 0; d < 3; ++d) {
    a.n[d] = g.n[d];
    a.bc[d][0] = g.bc[d][0];
    a.bc[d][1] = g.bc[d][1];
  }
  double *p = c->split_buf;
  a.R = mode == MODE_RESIDUAL ? out : p;
  p += (size_t)c->nv * c->ncells;
  for (int d = 0; d < g.dim; ++d) {
    a.nface[d] = split_faces(g, d);
    const size_t fsz = (size_t)c->nv * a.nface[d];
    a.QL[d] = p;
    a.QR[d] = p + fsz;
    a.F[d] = p + 2 * fsz;
    p += 3 * fsz;
  }
  a.Us = Us;
  a.Un = Un;
  a.out = out;
  a.norm_part = norm_part;
  a.S = c->source;
  double h[3];
  a.vol = 1.0;
  for (int d = 0; d < 3; ++d) {
    h[d] = (d < g.dim) ? g.len[d] / g.n[d] : 1.0;
    a.vol *= h[d];
  }
  a.inv_vol = 1.0 / a.vol;
  for (int d = 0; d < 3; ++d) {
    double ds = 1.0;
    for (int e = 0; e < g.dim; ++e)
      if (e != d) ds *= h[e];
    a.ds[d] = ds;
  }
  a.limiter = c->scheme.limiter;
  a.recon = c->scheme.recon;
  a.inv_g1 = 1.0 / (c->scheme.gamma - 1.0);
  a.cL = 0.25 * c->scheme.eps * (1.0 - c->scheme.kappa);
  a.cR = 0.25 * c->scheme.eps * (1.0 + c->scheme.kappa);
  a.g1 = c->scheme.gamma - 1.0;
  a.half_eps = 0.5 * c->scheme.eps;
  a.efix = c->scheme.efix;
  a.inv2efix = c->scheme.efix > 0.0 ? 0.5 / c->scheme.efix : 0.0;
  a.smax = smax;
  a.cfl = c->scheme.cfl;
  a.dt_fixed = dt_fixed;
  a.t_acc = t_acc;
  int grid[FV_SK_COUNT], threads[FV_SK_COUNT], rb = 0;
  for (int k = 0; k < FV_SK_COUNT; ++k) {
    grid[k] = c->launch.split[k].grid;
    threads[k] = c->launch.split[k].threads;
  }
  FV_CK(launch_split(mode, a, grid, threads, &rb, st));
  return FV_OK;
}

int stage(fv_ctx *c, int mode, int sidx, const double *Us, const double *Un, double *out,
          const unsigned long long *smax, double dt_fixed, double *norm_part, double *t_acc, cudaStream_t st,
          long long tile_begin = 0, long long tile_count = 0) {
  if (c->launch.mode == FV_SPLIT)  // whole-grid launches only (no tile ranges)
    return split_stage(c, mode, Us, Un, out, smax, dt_fixed, norm_part, t_acc, st);
  const fv_grid &g = c->grid;
  const fv_kernel_cfg &k = c->launch.stage[sidx];
  StageArgs a;
  memset(&a, 0, sizeof(a));
  a.tile_begin = tile_begin;
  a.tile_count = tile_count;
  a.S = c->source;
  a.vol = 1.0;
  for (int d = 0; d < g.dim; ++d) a.vol *= g.len[d] / g.n[d];
  a.Us = Us;
  a.Un = Un;
  a.out = out;
  a.norm_part = norm_part;
  for (int d = 0; d < 3; ++d) {
    a.n[d] = g.n[d];
    a.tile[d] = k.tile[d];
    a.bc[d][0] = g.bc[d][0];
    a.bc[d][1] = g.bc[d][1];
  }
  ntiles(g, k.tile, a.ntile);
  double h[3];
  for (int d = 0; d < 3; ++d) h[d] = (d < g.dim) ? g.len[d] / g.n[d] : 1.0;
  for (int d = 0; d < 3; ++d) {
    double ds = 1.0;  // area of a face normal to axis d
    for (int e = 0; e < g.dim; ++e)
      if (e != d) ds *= h[e];
    a.ds[d] = ds;
    a.inv_h[d] = (d < g.dim) ? g.n[d] / g.len[d] : 1.0;  // as the batched kernel's n / len
  }
  a.limiter = c->scheme.limiter;
  a.recon = c->scheme.recon;
  a.inv_g1 = 1.0 / (c->scheme.gamma - 1.0);
  a.cL = 0.25 * c->scheme.eps * (1.0 - c->scheme.kappa);
  a.cR = 0.25 * c->scheme.eps * (1.0 + c->scheme.kappa);
  a.g1 = c->scheme.gamma - 1.0;
  a.half_eps = 0.5 * c->scheme.eps;
  a.efix = c->scheme.efix;
  a.inv2efix = c->scheme.efix > 0.0 ? 0.5 / c->scheme.efix : 0.0;
  a.smax = smax;
  a.cfl = c->scheme.cfl;
  a.dt_fixed = dt_fixed;
  a.t_acc = t_acc;
  a.flags = c->flags;
  a.fd = c->fd;
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  a.march = k.march;
  a.use_tma = (k.loader == FV_LOADER_TMA && make_tmap(c, Us, k.tile, k.march, &map)) ? 1 : 0;
  FV_CK(launch_stage(g.dim, mode, &map, a, k.threads, st));
  return FV_OK;
}

int dt_launch(fv_ctx *c, const double *U, cudaStream_t st) {
  DtArgs a;
  memset(&a, 0, sizeof(a));
  a.U = U;
  a.ncells = c->ncells;
  a.dim = c->grid.dim;
  a.g1 = c->scheme.gamma - 1.0;
  a.gamma = c->scheme.gamma;
  for (int d = 0; d < 3; ++d) a.inv_h[d] = (d < c->grid.dim) ? c->grid.n[d] / c->grid.len[d] : 0.0;
  a.smax = c->smax;
  a.flags = c->flags;
  // FP32 pre-selection where its error bound applies (1/dx within [2^-30, 2^30],
  // 2^-20 <= gamma - 1 and gamma < 1e6: no FP32 overflow or underflow)
  bool b = c->scheme.gamma < 1e6 && a.g1 >= 0x1p-20;
  for (int d = 0; d < c->grid.dim; ++d) b = b && a.inv_h[d] >= 0x1p-30 && a.inv_h[d] <= 0x1p30;
  a.bounded = b ? 1 : 0;
  a.lbound = c->lbound;
  a.chunk_hi = c->chunk_hi;
  a.g1f = (float)a.g1;
  a.gammaf = (float)a.gamma;
  for (int d = 0; d < 3; ++d) a.inv_hf[d] = (float)a.inv_h[d];
  // grid 0: enough CTAs to fill every SM with 2048 threads (both passes read
  // the state from HBM and need loads in flight)
  int blocks = c->launch.dt.grid > 0 ? c->launch.dt.grid : std::max(1, 2048 / c->launch.dt.threads) * c->sms;
  const long long need = (c->ncells + c->launch.dt.threads - 1) / c->launch.dt.threads;
  if (blocks > need) blocks = (int)(need > 0 ? need : 1);
  FV_CK(cudaMemsetAsync(c->smax, 0, 16, st));  // smax and the FP32 bound
  FV_CK(launch_dt(a, blocks, c->launch.dt.threads, st));
  return FV_OK;
}

// One SSP-RK3 step on device state U (stream st).  smax_mode: dt from CFL.
int rk_step_device(fv_ctx *c, double *U, double dt_fixed, bool cfl, double *t_acc, cudaStream_t st) {
  int r;
  const unsigned long long *sm = nullptr;
  if (cfl) {
    if ((r = dt_launch(c, U, st))) return r;
    sm = c->smax;
  }
  if ((r = stage(c, MODE_STAGE1, 0, U, U, c->U1, sm, dt_fixed, nullptr, nullptr, st))) return r;
  if ((r = stage(c, MODE_STAGE2, 1, c->U1, U, c->U2, sm, dt_fixed, nullptr, nullptr, st))) return r;
  if ((r = stage(c, MODE_STAGE3, 2, c->U2, U, U, sm, dt_fixed, nullptr, t_acc, st))) return r;
  return FV_OK;
}

int ensure_staging(fv_ctx *c) {
  if (!c->stage_in) FV_CK(cudaMalloc(&c->stage_in, c->state_bytes));
  if (!c->stage_out) FV_CK(cudaMalloc(&c->stage_out, c->state_bytes));
  return FV_OK;
}

int read_flags(fv_ctx *c) {
  unsigned f = 0;
  FV_CK(cudaMemcpyAsync(&f, c->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  FV_CK(cudaStreamSynchronize(c->stream));
  if (f) FV_CK(cudaMemsetAsync(c->flags, 0, sizeof(unsigned), c->stream));
  if (f & FLAG_TIMEOUT) return FV_ETIMEOUT;
  if (f & FLAG_NONPHYSICAL) return FV_ENONPHYSICAL;
  return FV_OK;
}

int set_attributes(fv_ctx *c) {
  FV_CK(stage_kernel_attributes(c->grid.dim, c->smem_optin));
  return FV_OK;
}

// Callers make sure no launch of the graph is still queued when it owns
// device memory (cudaFree also waits for the device).
void destroy_graph(GraphEntry &g) {
  cudaGraphExecDestroy(g.exec);
  if (g.aux) cudaFree(g.aux);
}

void drop_graphs(fv_ctx *c) {
  for (auto &g : c->graphs) destroy_graph(g);
  c->graphs.clear();
}

// Graphs are keyed by the state pointer; callers that allocate a new state
// per call would grow the cache without bound, so keep the newest entries.
constexpr size_t kMaxGraphs = 16;
void remember_graph(fv_ctx *c, const GraphEntry &e) {
  // evict the oldest entries of other states (the caller may hold a sibling
  // graph of e.U that it is about to launch)
  for (size_t i = 0; c->graphs.size() >= kMaxGraphs && i < c->graphs.size();) {
    if (c->graphs[i].U != e.U) {
      if (c->graphs[i].aux) cudaStreamSynchronize(c->stream);  // its last launch may be queued
      destroy_graph(c->graphs[i]);
      c->graphs.erase(c->graphs.begin() + i);
    } else {
      ++i;
    }
  }
  c->graphs.push_back(e);
}

}  // namespace

namespace {

constexpr long long kBatchChunk = 4096;  // cells per time-step work item

// Device tables of a batch for the current launch tile; cooperative grid size.
int batch_setup(fv_ctx *c) {
  const int *tile = c->launch.stage[0].tile;
  const int n = c->ngrids;
  std::vector<BatchProblem> P(n);
  std::vector<int> tb(n + 1), cb(n + 1);
  int tiles = 0, chunks = 0;
  for (int g = 0; g < n; ++g) {
    const fv_grid &G = c->grids[g];
    BatchProblem &p = P[g];
    memset(&p, 0, sizeof(p));
    p.off = c->offsets[g];
    for (int d = 0; d < 2; ++d) {
      p.n[d] = G.n[d];
      p.ntile[d] = (G.n[d] + tile[d] - 1) / tile[d];
      const double h = G.len[d] / G.n[d];
      p.inv_h[d] = G.n[d] / G.len[d];
      p.inv_hf[d] = (float)p.inv_h[d];
    }
    // the FP32 pre-selection's conditions (as for single grids)
    p.bounded = c->scheme.gamma < 1e6 && c->scheme.gamma - 1.0 >= 0x1p-20 && p.inv_h[0] >= 0x1p-30 &&
                p.inv_h[0] <= 0x1p30 && p.inv_h[1] >= 0x1p-30 && p.inv_h[1] <= 0x1p30;
    for (int d = 0; d < 3; ++d) {
      p.bc[d][0] = G.bc[d][0];
      p.bc[d][1] = G.bc[d][1];
    }
    tb[g] = tiles;
    cb[g] = chunks;
    tiles += p.ntile[0] * p.ntile[1];
    chunks += (int)(((long long)G.n[0] * G.n[1] + kBatchChunk - 1) / kBatchChunk);
  }
  tb[n] = tiles;
  cb[n] = chunks;
  c->b_total_tiles = tiles;
  c->b_total_chunks = chunks;
  FV_CK(cudaMemcpy(c->b_prob, P.data(), sizeof(BatchProblem) * n, cudaMemcpyHostToDevice));
  FV_CK(cudaMemcpy(c->b_tile_begin, tb.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
  FV_CK(cudaMemcpy(c->b_chunk_begin, cb.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
  int per_sm = 0;
  FV_CK(batch_max_blocks(c->launch.stage[0].threads, batch_smem_bytes(tile), &per_sm));
  if (per_sm < 1) return FV_EINVAL;
  c->b_blocks = per_sm * c->sms;
  return FV_OK;
}

int batch_init(fv_ctx *c, const fv_grid *grids, int ngrids) {
  c->ngrids = ngrids;
  c->grids.assign(grids, grids + ngrids);
  c->offsets.assign(ngrids + 1, 0);
  long long off = 0;
  for (int g = 0; g < ngrids; ++g) {
    if (grids[g].dim != 2) return FV_EUNSUPPORTED;
    if (validate_grid(&grids[g])) return FV_EINVAL;
    c->offsets[g] = off;
    off += 4ll * grids[g].n[0] * grids[g].n[1];
    off = (off + 31) / 32 * 32;  // 256-byte aligned blocks
  }
  c->offsets[ngrids] = off;
  c->state_bytes = sizeof(double) * (size_t)off;
  FV_CK(cudaMalloc(&c->b_prob, sizeof(BatchProblem) * ngrids));
  FV_CK(cudaMalloc(&c->b_tile_begin, sizeof(int) * (ngrids + 1)));
  FV_CK(cudaMalloc(&c->b_chunk_begin, sizeof(int) * (ngrids + 1)));
  FV_CK(cudaMalloc(&c->b_smax, (sizeof(unsigned long long) + sizeof(unsigned)) * 2 * ngrids));
  FV_CK(cudaMalloc(&c->b_tacc, sizeof(double) * ngrids));
  FV_CK(cudaMalloc(&c->b_bar, sizeof(unsigned) * 2));
  FV_CK(cudaMemset(c->b_bar, 0, sizeof(unsigned) * 2));
  long long chunks = 0;  // time-step items, as batch_setup counts them
  for (int g = 0; g < ngrids; ++g) chunks += ((long long)grids[g].n[0] * grids[g].n[1] + kBatchChunk - 1) / kBatchChunk;
  FV_CK(cudaMalloc(&c->b_chunk_hi, sizeof(unsigned) * (size_t)chunks * (kBatchChunk / 32)));
  return FV_OK;
}

// nsteps steps of a batch in one cooperative launch, captured in a graph.
int batch_run(fv_ctx *c, double *Ud, int nsteps, double dt_fixed, bool want_t) {
  if (nsteps == 0) return FV_OK;
  const int n = c->ngrids;
  long long dbits = 0;
  if (dt_fixed > 0.0) memcpy(&dbits, &dt_fixed, sizeof(dbits));
  cudaGraphExec_t exec = nullptr;
  for (auto &g : c->graphs)
    if (g.U == Ud && g.dt_bits == dbits && g.steps == nsteps) exec = g.exec;
  if (!exec) {
    BatchArgs b;
    memset(&b, 0, sizeof(b));
    b.prob = c->b_prob;
    b.tile_begin = c->b_tile_begin;
    b.chunk_begin = c->b_chunk_begin;
    b.nprob = n;
    b.total_tiles = c->b_total_tiles;
    b.total_chunks = c->b_total_chunks;
    b.nsteps = nsteps;
    b.chunk_cells = kBatchChunk;
    b.chunk_hi = c->b_chunk_hi;
    b.tile[0] = c->launch.stage[0].tile[0];
    b.tile[1] = c->launch.stage[0].tile[1];
    b.U = Ud;
    b.U1 = c->U1;
    b.U2 = c->U2;
    b.smax = c->b_smax;
    b.lbound = reinterpret_cast<unsigned *>(c->b_smax + 2 * c->ngrids);
    b.g1f = (float)(c->scheme.gamma - 1.0);
    b.gammaf = (float)c->scheme.gamma;
    b.t_acc = c->b_tacc;
    b.flags = c->flags;
    b.bar_count = c->b_bar;
    b.bar_gen = c->b_bar + 1;
    b.g1 = c->scheme.gamma - 1.0;
    b.gamma = c->scheme.gamma;
    b.half_eps = 0.5 * c->scheme.eps;
    b.efix = c->scheme.efix;
    b.inv2efix = c->scheme.efix > 0.0 ? 0.5 / c->scheme.efix : 0.0;
    b.cfl = c->scheme.cfl;
    b.dt_fixed = dt_fixed > 0.0 ? dt_fixed : 0.0;
    // TMA tile loads: per stage source (Ud, U1, U2) and problem a tensor map
    // over that problem's block, where its grid allows one (the conditions of
    // single grids); the others load with plain loads.  The maps hold Ud's
    // address, so they belong to this graph and are freed with it.
    void *aux = nullptr;
    if (c->launch.stage[0].loader == FV_LOADER_TMA) {
      const int t3[3] = {b.tile[0], b.tile[1], 1};
      std::vector<CUtensorMap> maps(3 * (size_t)n);
      std::vector<int> ok(3 * (size_t)n, 0);
      const double *src[3] = {Ud, c->U1, c->U2};
      int any = 0;
      for (int k = 0; k < 3; ++k)
        for (int g = 0; g < n; ++g) {
          memset(&maps[(size_t)k * n + g], 0, sizeof(CUtensorMap));
          ok[(size_t)k * n + g] = make_tmap_grid(c->grids[g], 4, src[k] + c->offsets[g], t3, 0, &maps[(size_t)k * n + g]);
          any |= ok[(size_t)k * n + g];
        }
      if (any) {
        const size_t mb = sizeof(CUtensorMap) * maps.size();
        FV_CK(cudaMalloc(&aux, mb + sizeof(int) * ok.size()));
        cudaError_t em = cudaMemcpy(aux, maps.data(), mb, cudaMemcpyHostToDevice);
        if (em == cudaSuccess)
          em = cudaMemcpy(static_cast<char *>(aux) + mb, ok.data(), sizeof(int) * ok.size(), cudaMemcpyHostToDevice);
        if (em != cudaSuccess) {
          cudaFree(aux);
          return cuda_fail(em);
        }
        b.tmaps = static_cast<const CUtensorMap *>(aux);
        b.tma_ok = reinterpret_cast<const int *>(static_cast<char *>(aux) + mb);
      }
    }
    const int blocks = c->b_blocks < c->b_total_tiles ? c->b_blocks : c->b_total_tiles;
    cudaGraph_t graph;
    FV_CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(c->b_smax, 0, (sizeof(unsigned long long) + sizeof(unsigned)) * 2 * n, c->cap);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->b_tacc, 0, sizeof(double) * n, c->cap);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->b_bar, 0, sizeof(unsigned), c->cap);
    if (e == cudaSuccess)
      e = launch_batch_run(b, blocks, c->launch.stage[0].threads, batch_smem_bytes(b.tile), c->cap);
    cudaError_t ec = cudaStreamEndCapture(c->cap, &graph);
    if (e != cudaSuccess) {
      if (ec == cudaSuccess) cudaGraphDestroy(graph);
      if (aux) cudaFree(aux);
      return cuda_fail(e);
    }
    if (ec != cudaSuccess) {
      if (aux) cudaFree(aux);
      return cuda_fail(ec);
    }
    cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      if (aux) cudaFree(aux);
      return cuda_fail(ei);
    }
    GraphEntry ge{Ud, dbits, nsteps, exec};
    ge.aux = aux;
    remember_graph(c, ge);
  }
  FV_CK(cudaGraphLaunch(exec, c->stream));
  (void)want_t;
  return FV_OK;
}

}  // namespace

namespace fvk {

int ctx_work_state(fv_ctx *c, const double *U, double **Uw) {
  int r;
  if ((r = ensure_staging(c))) return r;
  FV_CK(cudaMemcpyAsync(c->stage_in, U, c->state_bytes, cudaMemcpyDefault, c->stream));
  FV_CK(cudaStreamSynchronize(c->stream));
  *Uw = c->stage_in;
  return FV_OK;
}

int ctx_time_launch(fv_ctx *c, double *Uw, const fv_launch *l, int steps, int repeats, double *sec) {
  int r = validate_launch(&c->grid, &c->scheme, l, c->smem_optin);
  if (r) return r;
  const fv_launch saved = c->launch;
  c->launch = *l;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  std::vector<double> t;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) r = FV_ECUDA;
  if (!r) r = rk_step_device(c, Uw, 0.0, true, nullptr, c->stream);  // warm-up
  for (int rep = 0; rep < repeats && !r; ++rep) {
    if (cudaEventRecord(e0, c->stream) != cudaSuccess) r = FV_ECUDA;
    for (int s = 0; s < steps && !r; ++s) r = rk_step_device(c, Uw, 0.0, true, nullptr, c->stream);
    float ms = 0.f;
    if (!r && (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
               cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      r = FV_ECUDA;
    if (!r) t.push_back(1e-3 * ms / steps);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  c->launch = saved;
  if (r) {
    (void)cudaGetLastError();
    return r;
  }
  std::sort(t.begin(), t.end());
  *sec = t[t.size() / 2];
  return read_flags(c);
}

int ctx_sm_count(const fv_ctx *c) { return c->sms; }
int ctx_validate_launch(const fv_ctx *c, const fv_launch *l) {
  return validate_launch(&c->grid, &c->scheme, l, c->smem_optin);
}
int ctx_default_launch(const fv_ctx *c, fv_launch *l) {
  const int r = fv_default_launch(&c->grid, l);
  l->mode = c->launch.mode;  // the default of the context's kernel structure
  return r;
}
int ctx_dim(const fv_ctx *c) { return c->grid.dim; }

}  // namespace fvk

extern "C" {

const char *fv_strerror(int status) {
  switch (status) {
    case FV_OK: return "success";
    case FV_EINVAL: return "invalid argument";
    case FV_ENOMEM: return "out of memory";
    case FV_ECUDA: return "CUDA error";
    case FV_ENONPHYSICAL: return "non-physical state (rho <= 0, p <= 0 or NaN)";
    case FV_ETIMEOUT: return "device-side wait timed out";
    case FV_EUNSUPPORTED: return "valid request the library does not support";
    default: return "unknown status";
  }
}

int fv_default_launch(const fv_grid *g, fv_launch *l) {
  if (!l || validate_grid(g)) return FV_EINVAL;
  memset(l, 0, sizeof(*l));
  for (int s = 0; s < 3; ++s) {
    fv_kernel_cfg &k = l->stage[s];
    if (g->dim == 2) {
      k.tile[0] = 64;  // two CTAs per SM (shared memory)
      k.tile[1] = 16;
      k.tile[2] = 1;
    } else {
      k.tile[0] = 8;  // 9 x 8 x 8 faces per axis: three full rounds of 192 threads
      k.tile[1] = 8;
      k.tile[2] = 8;
    }
    // 2D: 192 threads take the 17 faces of each of the 64 y-lines of a 64x16
    // tile in runs of 6 (one run per thread) and the 65 faces of each of its
    // 16 x-lines in 11 runs of 6 or fewer
    k.threads = 192;
    k.grid = 0;
  }
  l->dt.threads = 512;  // 1024 threads per SM keep enough loads in flight
  l->dt.grid = 0;
  l->mode = FV_FUSED;
  for (int k = 0; k < FV_SK_COUNT; ++k) {
    l->split[k].threads = 128;
    l->split[k].grid = 0;
  }
  return FV_OK;
}

int fv_init(fv_ctx **out, const fv_grid *grids, int ngrids, const fv_scheme *s, const fv_launch *l, void *stream) {
  if (!out) return FV_EINVAL;
  *out = nullptr;
  if (ngrids < 1 || !grids) return FV_EINVAL;
  if (validate_grid(grids) || validate_scheme(s)) return FV_EINVAL;
  fv_ctx *c = new (std::nothrow) fv_ctx();
  if (!c) return FV_ENOMEM;
  c->grid = grids[0];
  c->scheme = *s;
  c->stream = static_cast<cudaStream_t>(stream);
  c->nv = grids[0].dim + 2;
  c->ncells = (long long)grids[0].n[0] * grids[0].n[1] * grids[0].n[2];
  c->state_bytes = sizeof(double) * (size_t)c->nv * (size_t)c->ncells;
  c->ngrids = 1;
  int r = FV_OK;
  auto fail = [&](int code) {
    fv_destroy(c);
    return code;
  };
  if (ngrids > 1 && (s->limiter != FV_LIM_MINMOD || s->recon != FV_RECON_CONSERVED)) return fail(FV_EUNSUPPORTED);
  if (ngrids > 1 && (r = batch_init(c, grids, ngrids))) return fail(r);
  if (cudaGetDevice(&c->device) != cudaSuccess) return fail(cuda_fail(cudaErrorNoDevice));
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) return fail(FV_ECUDA);
  c->sms = prop.multiProcessorCount;
  c->smem_optin = prop.sharedMemPerBlockOptin;
  if (l) {
    c->launch = *l;
  } else {
    fv_default_launch(&c->grid, &c->launch);
    // the batched persistent kernel also runs its CFL phases with these
    // threads: it keeps 32x32 tiles and 256 threads per CTA (measured 8%
    // faster than 160 on the 96-grid Sod batch)
    if (ngrids > 1)
      for (int s = 0; s < 3; ++s) {
        c->launch.stage[s].tile[0] = c->launch.stage[s].tile[1] = 32;
        c->launch.stage[s].threads = 256;
      }
  }
  if ((r = validate_launch(&c->grid, &c->scheme, &c->launch, c->smem_optin))) return fail(r);
  if (ngrids > 1 && c->launch.mode != FV_FUSED) return fail(FV_EUNSUPPORTED);
  if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) return fail(FV_ECUDA);
  if (cudaMalloc(&c->U1, c->state_bytes) != cudaSuccess || cudaMalloc(&c->U2, c->state_bytes) != cudaSuccess)
    return fail(cuda_fail(cudaErrorMemoryAllocation));
  // scratch: smax (8) | FP32 lower bound (4) + pad | flags (8) | t_acc (8) | dt (8) | norms (8 * 5)
  char *scr = nullptr;
  if (cudaMalloc(&scr, 256) != cudaSuccess) return fail(cuda_fail(cudaErrorMemoryAllocation));
  c->smax = reinterpret_cast<unsigned long long *>(scr);
  c->lbound = reinterpret_cast<unsigned *>(scr + 8);
  c->flags = reinterpret_cast<unsigned *>(scr + 16);
  c->t_acc = reinterpret_cast<double *>(scr + 24);
  c->dt_dev = reinterpret_cast<double *>(scr + 32);
  c->norm_out = reinterpret_cast<double *>(scr + 40);
  if (cudaMemset(scr, 0, 256) != cudaSuccess) return fail(FV_ECUDA);
  if (cudaMalloc(&c->chunk_hi, sizeof(unsigned) * (size_t)((c->ncells + 31) / 32)) != cudaSuccess)
    return fail(cuda_fail(cudaErrorMemoryAllocation));
  if ((r = set_attributes(c))) return fail(r);
  if (c->ngrids > 1 && (r = batch_setup(c))) return fail(r);
  if (c->launch.mode == FV_SPLIT && (r = ensure_split(c))) return fail(r);  // never inside a graph capture
  *out = c;
  return FV_OK;
}

int fv_layout(const fv_ctx *c, long long *offsets, int ngrids) {
  if (!c || !offsets || ngrids != c->ngrids) return FV_EINVAL;
  if (c->ngrids == 1) {
    offsets[0] = 0;
    offsets[1] = (long long)c->nv * c->ncells;
    return FV_OK;
  }
  for (int g = 0; g <= c->ngrids; ++g) offsets[g] = c->offsets[g];
  return FV_OK;
}

int fv_set_launch(fv_ctx *c, const fv_launch *l) {
  if (!c || !l) return FV_EINVAL;
  int r = validate_launch(&c->grid, &c->scheme, l, c->smem_optin);
  if (r) return r;
  if (c->ngrids > 1 && l->mode != FV_FUSED) return FV_EUNSUPPORTED;
  if (l->mode == FV_SPLIT && (r = ensure_split(c))) return r;
  // queued work may still read the graphs' tile-load maps and the batch tables
  FV_CK(cudaStreamSynchronize(c->stream));
  c->launch = *l;
  drop_graphs(c);
  if ((r = set_attributes(c))) return r;
  if (c->ngrids > 1) return batch_setup(c);
  return FV_OK;
}

int fv_set_source(fv_ctx *c, const double *S) {
  if (!c) return FV_EINVAL;
  if (c->ngrids > 1) return FV_EUNSUPPORTED;
  if (S && pointer_kind(S, c->device) != PTR_DEVICE) return FV_EINVAL;
  if (S != c->source) {
    FV_CK(cudaStreamSynchronize(c->stream));  // launches queued with the old source finish first
    drop_graphs(c);                           // captured graphs hold the old pointer
    c->source = S;
  }
  return FV_OK;
}

int fv_get_launch(const fv_ctx *c, fv_launch *l) {
  if (!c || !l) return FV_EINVAL;
  *l = c->launch;
  return FV_OK;
}

int fv_residual(fv_ctx *c, const double *U, double *R, double *rnorm2) {
  if (!c || !U || !R || U == R) return FV_EINVAL;
  if (c->ngrids > 1) return FV_EUNSUPPORTED;
  int r;
  bool hostU, hostR, hostN = false;
  if (where(c, U, &hostU) || where(c, R, &hostR) || (rnorm2 && where(c, rnorm2, &hostN))) return FV_EINVAL;
  if ((hostU || hostR) && (r = ensure_staging(c))) return r;
  const double *Ud = U;
  double *Rd = R;
  if (hostU) {
    FV_CK(cudaMemcpyAsync(c->stage_in, U, c->state_bytes, cudaMemcpyHostToDevice, c->stream));
    Ud = c->stage_in;
  }
  if (hostR) Rd = c->stage_out;
  double *part = nullptr;
  int nt[3];
  ntiles(c->grid, c->launch.stage[0].tile, nt);
  const long long nblk = c->launch.mode == FV_SPLIT ? split_rhs_blocks(c) : (long long)nt[0] * nt[1] * nt[2];
  if (rnorm2) {
    if (c->norm_part_cap < nblk) {
      if (c->norm_part) cudaFree(c->norm_part);
  if (c->X1) cudaFree(c->X1);
  if (c->X2) cudaFree(c->X2);
  if (c->b_prob) cudaFree(c->b_prob);
  if (c->b_tile_begin) cudaFree(c->b_tile_begin);
  if (c->b_chunk_begin) cudaFree(c->b_chunk_begin);
  if (c->b_smax) cudaFree(c->b_smax);
  if (c->b_tacc) cudaFree(c->b_tacc);
  if (c->b_bar) cudaFree(c->b_bar);
  if (c->b_chunk_hi) cudaFree(c->b_chunk_hi);
      c->norm_part = nullptr;
      c->norm_part_cap = 0;
      FV_CK(cudaMalloc(&c->norm_part, sizeof(double) * c->nv * nblk));
      c->norm_part_cap = nblk;
    }
    part = c->norm_part;
  }
  if ((r = stage(c, MODE_RESIDUAL, 0, Ud, Ud, Rd, nullptr, 0.0, part, nullptr, c->stream))) return r;
  if (rnorm2) {
    FV_CK(launch_norm_finalize(part, (int)nblk, c->nv, c->norm_out, c->stream));
    FV_CK(cudaMemcpyAsync(rnorm2, c->norm_out, sizeof(double) * c->nv,
                          hostN ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream));
  }
  if (hostR) FV_CK(cudaMemcpyAsync(R, Rd, c->state_bytes, cudaMemcpyDeviceToHost, c->stream));
  if (hostU || hostR || hostN) FV_CK(cudaStreamSynchronize(c->stream));
  return FV_OK;
}

int fv_time_step(fv_ctx *c, const double *U, double *dt_out) {
  if (!c || !U || !dt_out) return FV_EINVAL;
  if (c->ngrids > 1) return FV_EUNSUPPORTED;
  int r;
  bool hostU, hostD;
  if (where(c, U, &hostU) || where(c, dt_out, &hostD)) return FV_EINVAL;
  const double *Ud = U;
  if (hostU) {
    if ((r = ensure_staging(c))) return r;
    FV_CK(cudaMemcpyAsync(c->stage_in, U, c->state_bytes, cudaMemcpyHostToDevice, c->stream));
    Ud = c->stage_in;
  }
  if ((r = dt_launch(c, Ud, c->stream))) return r;
  if (!hostD) {
    FV_CK(launch_dt_finalize(c->smax, c->scheme.cfl, dt_out, c->stream));
    return hostU ? read_flags(c) : FV_OK;
  }
  unsigned long long bits = 0;
  FV_CK(cudaMemcpyAsync(&bits, c->smax, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
  if ((r = read_flags(c))) return r;
  double smax;
  memcpy(&smax, &bits, sizeof(smax));
  *dt_out = c->scheme.cfl / smax;
  return FV_OK;
}

int fv_rk_step(fv_ctx *c, double *U, double dt, double *dt_used) {
  if (!c || !U) return FV_EINVAL;
  if (c->ngrids > 1) return fv_run(c, U, 1, dt, dt_used);
  int r;
  bool hostU;
  if (where(c, U, &hostU)) return FV_EINVAL;
  double *Ud = U;
  if (hostU) {
    if ((r = ensure_staging(c))) return r;
    FV_CK(cudaMemcpyAsync(c->stage_in, U, c->state_bytes, cudaMemcpyHostToDevice, c->stream));
    Ud = c->stage_in;
  }
  const bool cfl = !(dt > 0.0);
  if (dt_used) FV_CK(cudaMemsetAsync(c->t_acc, 0, sizeof(double), c->stream));
  if ((r = rk_step_device(c, Ud, cfl ? 0.0 : dt, cfl, dt_used ? c->t_acc : nullptr, c->stream))) return r;
  if (hostU) FV_CK(cudaMemcpyAsync(U, Ud, c->state_bytes, cudaMemcpyDeviceToHost, c->stream));
  if (dt_used) {
    FV_CK(cudaMemcpyAsync(dt_used, c->t_acc, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return read_flags(c);
  }
  if (hostU) FV_CK(cudaStreamSynchronize(c->stream));
  return FV_OK;
}

// Host-state runs are split into bands of whole tile rows (2D) or tile
// planes (3D) of stage launch sidx: band b holds tile rows [r0, r1) and the
// grid rows [u0, u1) along the banded axis.
struct Bands {
  int slow;                 // banded axis: y in 2D, z in 3D
  long long per_row;        // tiles per tile row / plane
  int rows, nb;             // tile rows, bands
  long long cells_per_unit; // cells per grid row / plane
  int r0(int b) const { return (int)((long long)rows * b / nb); }
};

Bands make_bands(const fv_ctx *c, int sidx, int max_bands) {
  const fv_grid &g = c->grid;
  int nt[3];
  ntiles(g, c->launch.stage[sidx].tile, nt);
  Bands B;
  B.slow = g.dim - 1;
  B.per_row = (long long)nt[0] * (B.slow == 2 ? nt[1] : 1);
  B.rows = nt[B.slow];
  B.nb = B.rows < max_bands ? B.rows : max_bands;
  B.cells_per_unit = (long long)g.n[0] * (B.slow == 2 ? g.n[1] : 1);
  return B;
}

int ensure_events(std::vector<cudaEvent_t> &ev, int n) {
  while ((int)ev.size() < n) {
    cudaEvent_t e;
    FV_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ev.push_back(e);
  }
  return FV_OK;
}

// Whether the first stage of a host-state run may overlap the copy in: fused
// box-tile stage 1 (the flux-difference mode has no z-marching variant) on a
// grid whose tile rows (planes) are at least two cells high, so that a band's
// 2-cell halo lies in its neighbours.
bool overlap_first_stage(const fv_ctx *c) {
  const fv_kernel_cfg &k1 = c->launch.stage[0];
  return c->launch.mode == FV_FUSED && k1.march == 0 && k1.tile[c->grid.dim - 1] >= 2;
}

// Stage 1 of the first step of a run on a host state, overlapped with the
// state's copy to the device: the copy runs band by band (whole tile rows in
// 2D, tile planes in 3D) on the copy stream; as soon as a band and its
// neighbours have arrived, the flux-difference kernel computes that band's
// per-axis flux differences; the CFL reduction runs on the copy stream once
// the last band is in; then an elementwise kernel forms U1 = U + dt L(U) from
// the differences with the fused stage-1 kernel's operations in its order
// (the same bits).
int first_stage_from_host(fv_ctx *c, const double *Uh, double *Ud, double dt_fixed, bool cfl) {
  const fv_grid &g = c->grid;
  const Bands B = make_bands(c, 0, 1);  // geometry only: the bands are set here
  const fv_kernel_cfg &k1 = c->launch.stage[0];
  const long long N = c->ncells;
  // bands of 1, 1, 1, 2, 4, 8 and then 16 tile rows: the first flux
  // differences start once 3 tile rows are in, and the copy (about twice as
  // fast as the flux kernel) stays ahead of the bands after them
  std::vector<int> rb{0};
  const int ramp[6] = {1, 1, 1, 2, 4, 8};
  for (int q = 0; rb.back() < B.rows; ++q) rb.push_back(std::min(B.rows, rb.back() + (q < 6 ? ramp[q] : 16)));
  const int nb = (int)rb.size() - 1;
  if (!c->fd) return FV_EINVAL;  // allocated by the caller's check
  if (!c->copy_stream) FV_CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  if (!c->aux_stream) FV_CK(cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking));
  int r;
  if ((r = ensure_events(c->h2d_events, nb + 3))) return r;
  // the copy in and the second band stream start after the compute stream's
  // earlier work (which may still read Ud)
  FV_CK(cudaEventRecord(c->h2d_events[nb + 1], c->stream));
  FV_CK(cudaStreamWaitEvent(c->copy_stream, c->h2d_events[nb + 1], 0));
  FV_CK(cudaStreamWaitEvent(c->aux_stream, c->h2d_events[nb + 1], 0));
  for (int b = 0; b < nb; ++b) {
    const long long u0 = (long long)rb[b] * k1.tile[B.slow];
    const long long u1 = std::min<long long>((long long)rb[b + 1] * k1.tile[B.slow], g.n[B.slow]);
    for (int v = 0; v < c->nv; ++v) {
      const long long off = v * N + u0 * B.cells_per_unit;
      FV_CK(cudaMemcpyAsync(Ud + off, Uh + off, sizeof(double) * (u1 - u0) * B.cells_per_unit,
                            cudaMemcpyHostToDevice, c->copy_stream));
    }
    FV_CK(cudaEventRecord(c->h2d_events[b], c->copy_stream));
  }
  if (cfl && (r = dt_launch(c, Ud, c->copy_stream))) return r;
  FV_CK(cudaEventRecord(c->h2d_events[nb], c->copy_stream));
  // band b reads the rows of bands b-1..b+1 (the 2-cell halo; across a
  // periodic boundary band 0 reads the last band and the last band band 0):
  // bands 1..nb-2 start once band b+1 is in (the copies complete in order),
  // the last band and band 0 once everything is.  Consecutive bands go to
  // two streams, so that a band's last partial wave of CTAs overlaps the
  // next band.
  int nlaunch = 0;
  auto band = [&](int b) {
    cudaStream_t st = (nlaunch++ & 1) ? c->aux_stream : c->stream;
    const int wait = (b == 0 || b + 1 >= nb) ? nb - 1 : b + 1;
    const cudaError_t e = cudaStreamWaitEvent(st, c->h2d_events[wait], 0);
    if (e != cudaSuccess) return cuda_fail(e);
    return stage(c, MODE_FLUXDIFF, 0, Ud, Ud, nullptr, nullptr, 0.0, nullptr, nullptr, st,
                 (long long)rb[b] * B.per_row, (long long)(rb[b + 1] - rb[b]) * B.per_row);
  };
  for (int b = 1; b + 1 < nb; ++b)
    if ((r = band(b))) return r;
  if (nb > 1 && (r = band(nb - 1))) return r;
  if ((r = band(0))) return r;
  // U1 = U + dt L(U), after every band and the CFL reduction
  FV_CK(cudaEventRecord(c->h2d_events[nb + 2], c->aux_stream));
  FV_CK(cudaStreamWaitEvent(c->stream, c->h2d_events[nb + 2], 0));
  FV_CK(cudaStreamWaitEvent(c->stream, c->h2d_events[nb], 0));
  StageArgs a;
  memset(&a, 0, sizeof(a));
  a.Us = Ud;
  a.out = c->U1;
  a.fd = c->fd;
  a.S = c->source;
  for (int d = 0; d < 3; ++d) {
    a.n[d] = g.n[d];
    a.inv_h[d] = (d < g.dim) ? g.n[d] / g.len[d] : 1.0;  // as stage() forms it
  }
  a.smax = cfl ? c->smax : nullptr;
  a.cfl = c->scheme.cfl;
  a.dt_fixed = dt_fixed;
  FV_CK(launch_stage1_from_fd(g.dim, a, c->stream));
  return FV_OK;
}

// Stage 3 of the last SSP-RK3 step of a run on a host state.  On page-locked
// host memory mapped into the device's address space, stage 3 stores the new
// state straight to the host over the host link (its ~120 GB/s of stores stay
// below the link's rate, so the copy back costs no time of its own).
// Otherwise stage 3 runs in bands of whole tile rows (2D) or tile planes (3D),
// each band's cells copied back to the host on a second stream while the
// next band computes, so most of the device-to-host copy overlaps the last
// kernel.
int last_stage_to_host(fv_ctx *c, double *Ud, double *Uh, const unsigned long long *sm, double dt_fixed) {
  const fv_grid &g = c->grid;
  if (double *Uh_dev = mapped_host_range(Uh, c->state_bytes))
    return stage(c, MODE_STAGE3, 2, c->U2, Ud, Uh_dev, sm, dt_fixed, nullptr, c->t_acc, c->stream);
  const Bands B = make_bands(c, 2, 8);
  const fv_kernel_cfg &k3 = c->launch.stage[2];
  if (!c->copy_stream) FV_CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  int r;
  if ((r = ensure_events(c->band_events, B.nb + 1))) return r;
  const long long N = c->ncells;
  for (int b = 0; b < B.nb; ++b) {
    const int r0 = B.r0(b), r1 = B.r0(b + 1);
    if ((r = stage(c, MODE_STAGE3, 2, c->U2, Ud, Ud, sm, dt_fixed, nullptr, c->t_acc, c->stream, r0 * B.per_row,
                   (long long)(r1 - r0) * B.per_row)))
      return r;
    FV_CK(cudaEventRecord(c->band_events[b], c->stream));
    FV_CK(cudaStreamWaitEvent(c->copy_stream, c->band_events[b], 0));
    const long long u0 = (long long)r0 * k3.tile[B.slow];
    const long long u1 = std::min<long long>((long long)r1 * k3.tile[B.slow], g.n[B.slow]);
    for (int v = 0; v < c->nv; ++v) {
      const long long off = v * N + u0 * B.cells_per_unit;
      FV_CK(cudaMemcpyAsync(Uh + off, Ud + off, sizeof(double) * (u1 - u0) * B.cells_per_unit,
                            cudaMemcpyDeviceToHost, c->copy_stream));
    }
  }
  FV_CK(cudaEventRecord(c->band_events[B.nb], c->copy_stream));
  FV_CK(cudaStreamWaitEvent(c->stream, c->band_events[B.nb], 0));
  return FV_OK;
}

int fv_run(fv_ctx *c, double *U, int nsteps, double dt_fixed, double *t_out) {
  if (!c || !U || nsteps < 0) return FV_EINVAL;
  int r;
  bool hostU;
  if (where(c, U, &hostU)) return FV_EINVAL;
  double *Ud = U;
  // a host state's first step overlaps its stage 1 with the copy in (when
  // the buffer of its flux differences can be had; else the copy comes first)
  bool overlap = hostU && c->ngrids == 1 && nsteps > 0 && overlap_first_stage(c);
  if (overlap && !c->fd &&
      cudaMalloc(&c->fd, sizeof(double) * (size_t)c->grid.dim * c->state_bytes / sizeof(double)) != cudaSuccess) {
    (void)cudaGetLastError();
    c->fd = nullptr;
    overlap = false;
  }
  if (hostU) {
    if ((r = ensure_staging(c))) return r;
    if (!overlap) FV_CK(cudaMemcpyAsync(c->stage_in, U, c->state_bytes, cudaMemcpyHostToDevice, c->stream));
    Ud = c->stage_in;
  }
  if (c->ngrids > 1) {
    if ((r = batch_run(c, Ud, nsteps, dt_fixed, t_out != nullptr))) return r;
    if (hostU) FV_CK(cudaMemcpyAsync(U, Ud, c->state_bytes, cudaMemcpyDeviceToHost, c->stream));
    if (t_out) {
      if (nsteps == 0) {
        for (int g = 0; g < c->ngrids; ++g) t_out[g] = 0.0;
      } else {
        FV_CK(cudaMemcpyAsync(t_out, c->b_tacc, sizeof(double) * c->ngrids, cudaMemcpyDeviceToHost, c->stream));
      }
      return read_flags(c);
    }
    if (hostU) FV_CK(cudaStreamSynchronize(c->stream));
    return FV_OK;
  }
  const bool cfl = !(dt_fixed > 0.0);
  long long dbits = 0;
  if (!cfl) memcpy(&dbits, &dt_fixed, sizeof(dbits));
  FV_CK(cudaMemsetAsync(c->t_acc, 0, sizeof(double), c->stream));
  // Graphs of K steps and of one step, both captured on the first call for
  // this (U, dt mode) so that later calls only replay.
  const int K = 16;
  cudaGraphExec_t gK = nullptr, g1 = nullptr;
  for (auto &g : c->graphs)
    if (g.U == Ud && g.dt_bits == dbits) (g.steps == K ? gK : g1) = g.exec;
  for (int pass = 0; pass < 2 && nsteps > 0; ++pass) {
    const int steps = pass == 0 ? K : 1;
    if ((pass == 0 ? gK : g1) != nullptr) continue;
    cudaGraph_t graph;
    cudaGraphExec_t exec = nullptr;
    r = FV_OK;
    FV_CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    for (int s = 0; s < steps && r == FV_OK; ++s) r = rk_step_device(c, Ud, dt_fixed, cfl, c->t_acc, c->cap);
    cudaError_t ec = cudaStreamEndCapture(c->cap, &graph);
    if (r) {
      if (ec == cudaSuccess) cudaGraphDestroy(graph);
      return r;
    }
    FV_CK(ec);
    cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    FV_CK(ei);
    remember_graph(c, GraphEntry{Ud, dbits, steps, exec});
    (pass == 0 ? gK : g1) = exec;
  }
  // On a host state the first step (overlapping its stage 1 with the copy
  // in) and the last step (its stage 3 writing to the host, or overlapping
  // its copy back: fused kernels, they run by tile rows) run outside the
  // graphs.
  const bool to_host = hostU && c->launch.mode == FV_FUSED;
  const unsigned long long *sm = cfl ? c->smax : nullptr;
  int left = nsteps;
  bool copied_back = false;
  if (overlap) {
    if ((r = first_stage_from_host(c, U, Ud, dt_fixed, cfl))) return r;
    if ((r = stage(c, MODE_STAGE2, 1, c->U1, Ud, c->U2, sm, dt_fixed, nullptr, nullptr, c->stream))) return r;
    if (nsteps == 1) {
      if ((r = last_stage_to_host(c, Ud, U, sm, dt_fixed))) return r;
      copied_back = true;
    } else if ((r = stage(c, MODE_STAGE3, 2, c->U2, Ud, Ud, sm, dt_fixed, nullptr, c->t_acc, c->stream))) {
      return r;
    }
    --left;
  }
  for (int l = (to_host && left > 0) ? left - 1 : left; l > 0;) {
    const int steps = l >= K ? K : 1;
    FV_CK(cudaGraphLaunch(steps == K ? gK : g1, c->stream));
    l -= steps;
  }
  if (hostU && !copied_back) {
    if (to_host && left > 0) {
      // the last step: CFL reduction and stages 1-2 as usual, then stage 3 to the host
      if (cfl && (r = dt_launch(c, Ud, c->stream))) return r;
      if ((r = stage(c, MODE_STAGE1, 0, Ud, Ud, c->U1, sm, dt_fixed, nullptr, nullptr, c->stream))) return r;
      if ((r = stage(c, MODE_STAGE2, 1, c->U1, Ud, c->U2, sm, dt_fixed, nullptr, nullptr, c->stream))) return r;
      if ((r = last_stage_to_host(c, Ud, U, sm, dt_fixed))) return r;
    } else {
      FV_CK(cudaMemcpyAsync(U, Ud, c->state_bytes, cudaMemcpyDeviceToHost, c->stream));
    }
  }
  if (t_out) {
    FV_CK(cudaMemcpyAsync(t_out, c->t_acc, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return read_flags(c);
  }
  if (hostU) FV_CK(cudaStreamSynchronize(c->stream));
  return FV_OK;
}

namespace {

// One adjoint launch over the whole grid.
int adjoint(fv_ctx *c, const double *U, const double *lam, double *out, double w_dt, const double *A, double cA,
            const double *B, double cB, const double *Cc, double cC) {
  const fv_grid &g = c->grid;
  AdjArgs a;
  memset(&a, 0, sizeof(a));
  a.U = U;
  a.lam = lam;
  a.out = out;
  a.A = A;
  a.B = B;
  a.C = Cc;
  a.cA = cA;
  a.cB = cB;
  a.cC = cC;
  // 2D: 16x20 tiles, 380 x-faces and 368 y-faces, each about two full
  // rounds of the 192 threads (16x16 left 304 faces per axis, 1.6 rounds)
  const int tile2[3] = {16, 20, 1}, tile3[3] = {8, 4, 4};
  const int *tile = g.dim == 2 ? tile2 : tile3;
  for (int d = 0; d < 3; ++d) {
    a.n[d] = g.n[d];
    a.tile[d] = tile[d];
    a.ntile[d] = (d < g.dim) ? (g.n[d] + tile[d] - 1) / tile[d] : 1;
    a.bc[d][0] = g.bc[d][0];
    a.bc[d][1] = g.bc[d][1];
  }
  double h[3];
  for (int d = 0; d < 3; ++d) h[d] = (d < g.dim) ? g.len[d] / g.n[d] : 1.0;
  for (int d = 0; d < 3; ++d) {
    if (w_dt == 0.0) {  // residual: the face area
      double ds = 1.0;
      for (int e = 0; e < g.dim; ++e)
        if (e != d) ds *= h[e];
      a.scale[d] = ds;
    } else {  // RK stage: -w dt / dx_d, the transposed stage update
      a.scale[d] = -w_dt / h[d];
    }
  }
  a.g1 = c->scheme.gamma - 1.0;
  a.half_eps = 0.5 * c->scheme.eps;
  a.efix = c->scheme.efix;
  a.inv2efix = c->scheme.efix > 0.0 ? 0.5 / c->scheme.efix : 0.0;
  FV_CK(launch_adjoint(g.dim, a, g.dim == 2 ? kAdjThreads2d : 256, c->stream));
  return FV_OK;
}

}  // namespace

namespace {

// The reverse of one SSP-RK3 step at fixed dt, given its stage states U1, U2:
// three residual VJPs with the transposed stage combinations.
int rk_step_reverse(fv_ctx *c, const double *U, const double *U1, const double *U2, const double *lam, double dt,
                    double *out) {
  int r;
  // X2 = dJ/dU2 = 2/3 lam + 2/3 dt (dL/dU2)^T lam
  if ((r = adjoint(c, U2, lam, c->X2, (2.0 / 3.0) * dt, lam, 2.0 / 3.0, nullptr, 0.0, nullptr, 0.0))) return r;
  // X1 = dJ/dU1 = 1/4 X2 + 1/4 dt (dL/dU1)^T X2
  if ((r = adjoint(c, U1, c->X2, c->X1, 0.25 * dt, c->X2, 0.25, nullptr, 0.0, nullptr, 0.0))) return r;
  // out = 1/3 lam + 3/4 X2 + X1 + dt (dL/dU)^T X1
  return adjoint(c, U, c->X1, out, dt, lam, 1.0 / 3.0, c->X2, 0.75, c->X1, 1.0);
}

}  // namespace

extern "C" int fv_adjoint_vjp(fv_ctx *c, int what, const double *U, const double *lam, double dt, double *out) {
  if (!c || !U || !lam || !out || out == U || out == lam) return FV_EINVAL;
  if (c->ngrids > 1 || c->scheme.limiter != FV_LIM_MINMOD || c->scheme.recon != FV_RECON_CONSERVED)
    return FV_EUNSUPPORTED;
  if (pointer_kind(U, c->device) != PTR_DEVICE || pointer_kind(lam, c->device) != PTR_DEVICE ||
      pointer_kind(out, c->device) != PTR_DEVICE)
    return FV_EINVAL;
  if (what == FV_VJP_RESIDUAL) return adjoint(c, U, lam, out, 0.0, nullptr, 0.0, nullptr, 0.0, nullptr, 0.0);
  if (what != FV_VJP_RKSTEP || !(dt > 0.0)) return FV_EINVAL;
  if (!c->X1) FV_CK(cudaMalloc(&c->X1, c->state_bytes));
  if (!c->X2) FV_CK(cudaMalloc(&c->X2, c->state_bytes));
  int r;
  // forward stage states of the step: U1 = U + dt L(U), U2 = 3/4 U + 1/4 (U1 + dt L(U1))
  if ((r = stage(c, MODE_STAGE1, 0, U, U, c->U1, nullptr, dt, nullptr, nullptr, c->stream))) return r;
  if ((r = stage(c, MODE_STAGE2, 1, c->U1, U, c->U2, nullptr, dt, nullptr, nullptr, c->stream))) return r;
  return rk_step_reverse(c, U, c->U1, c->U2, lam, dt, out);
}

int fv_rk_step_stages(fv_ctx *c, double *U, double dt, double *U1, double *U2) {
  if (!c || !U || !U1 || !U2 || U1 == U || U2 == U || U1 == U2 || !(dt > 0.0)) return FV_EINVAL;
  if (c->ngrids > 1) return FV_EUNSUPPORTED;
  if (pointer_kind(U, c->device) != PTR_DEVICE || pointer_kind(U1, c->device) != PTR_DEVICE ||
      pointer_kind(U2, c->device) != PTR_DEVICE)
    return FV_EINVAL;
  // the stage launches of fv_rk_step at a fixed step, into the caller's stage arrays
  int r;
  if ((r = stage(c, MODE_STAGE1, 0, U, U, U1, nullptr, dt, nullptr, nullptr, c->stream))) return r;
  if ((r = stage(c, MODE_STAGE2, 1, U1, U, U2, nullptr, dt, nullptr, nullptr, c->stream))) return r;
  return stage(c, MODE_STAGE3, 2, U2, U, U, nullptr, dt, nullptr, nullptr, c->stream);
}

int fv_adjoint_vjp_stages(fv_ctx *c, const double *U, const double *U1, const double *U2, const double *lam,
                          double dt, double *out) {
  if (!c || !U || !U1 || !U2 || !lam || !out || out == U || out == lam || out == U1 || out == U2 || !(dt > 0.0))
    return FV_EINVAL;
  if (c->ngrids > 1 || c->scheme.limiter != FV_LIM_MINMOD || c->scheme.recon != FV_RECON_CONSERVED)
    return FV_EUNSUPPORTED;
  if (pointer_kind(U, c->device) != PTR_DEVICE || pointer_kind(U1, c->device) != PTR_DEVICE ||
      pointer_kind(U2, c->device) != PTR_DEVICE || pointer_kind(lam, c->device) != PTR_DEVICE ||
      pointer_kind(out, c->device) != PTR_DEVICE)
    return FV_EINVAL;
  if (!c->X1) FV_CK(cudaMalloc(&c->X1, c->state_bytes));
  if (!c->X2) FV_CK(cudaMalloc(&c->X2, c->state_bytes));
  return rk_step_reverse(c, U, U1, U2, lam, dt, out);
}

int fv_sync(fv_ctx *c) {
  if (!c) return FV_EINVAL;
  return read_flags(c);
}

void fv_destroy(fv_ctx *c) {
  if (!c) return;
  if (c->stream || c->U1) cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  if (c->U1) cudaFree(c->U1);
  if (c->U2) cudaFree(c->U2);
  if (c->stage_in) cudaFree(c->stage_in);
  if (c->stage_out) cudaFree(c->stage_out);
  if (c->chunk_hi) cudaFree(c->chunk_hi);
  for (cudaEvent_t e : c->band_events) cudaEventDestroy(e);
  for (cudaEvent_t e : c->h2d_events) cudaEventDestroy(e);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
  if (c->fd) cudaFree(c->fd);
  if (c->smax) cudaFree(c->smax);  // start of the scratch block
  if (c->norm_part) cudaFree(c->norm_part);
  if (c->X1) cudaFree(c->X1);
  if (c->X2) cudaFree(c->X2);
  if (c->split_buf) cudaFree(c->split_buf);
  if (c->b_prob) cudaFree(c->b_prob);
  if (c->b_tile_begin) cudaFree(c->b_tile_begin);
  if (c->b_chunk_begin) cudaFree(c->b_chunk_begin);
  if (c->b_smax) cudaFree(c->b_smax);
  if (c->b_tacc) cudaFree(c->b_tacc);
  if (c->b_bar) cudaFree(c->b_bar);
  if (c->b_chunk_hi) cudaFree(c->b_chunk_hi);
  if (c->cap) cudaStreamDestroy(c->cap);
  delete c;
}

int fv_debug_wait(int kind, double limit_seconds, void *stream) {
  if ((kind != 0 && kind != 1) || !(limit_seconds > 0.0) || !(limit_seconds <= 10.0)) return FV_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned *buf = nullptr;  // [0] the word nobody changes, [1] flags
  if (cudaMalloc(&buf, 2 * sizeof(unsigned)) != cudaSuccess) return cuda_fail(cudaErrorMemoryAllocation);
  int r = FV_OK;
  unsigned flags = 0;
  if (cudaMemsetAsync(buf, 0, 2 * sizeof(unsigned), st) != cudaSuccess ||
      launch_debug_wait(kind, (unsigned long long)(limit_seconds * 1e9), buf, buf + 1, st) != cudaSuccess ||
      cudaMemcpyAsync(&flags, buf + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    (void)cudaGetLastError();
    r = FV_ECUDA;
  } else if (flags & FLAG_TIMEOUT) {
    r = FV_ETIMEOUT;
  }
  cudaFree(buf);
  return r;
}

int fv_debug_bits(int op, const double *x, const double *y, double *out, long n, void *stream) {
  if (op < 0 || op > 7 || !x || !out || n < 0 || ((op == 4 || op >= 6) && !y)) return FV_EINVAL;
  FV_CK(launch_debug_bits(op, x, y, out, n, static_cast<cudaStream_t>(stream)));
  return FV_OK;
}

int fv_debug_fp64_rate(int kind, double *lane_ops_per_s, void *stream) {
  if (kind < 0 || kind > 3 || !lane_ops_per_s) return FV_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  FV_CK(cudaGetDevice(&dev));
  FV_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = 8 * sms, iters = 4096;  // 2048 threads per SM, ~20 ms
  double *out = nullptr;
  FV_CK(cudaMalloc(&out, sizeof(double) * 256 * (size_t)blocks));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int r = FV_OK;
  float ms = 0.f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      launch_fp64_stream(kind, blocks, iters / 8, out, st) != cudaSuccess ||  // warm-up
      cudaEventRecord(e0, st) != cudaSuccess || launch_fp64_stream(kind, blocks, iters, out, st) != cudaSuccess ||
      cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
    (void)cudaGetLastError();
    r = FV_ECUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (r == FV_OK) *lane_ops_per_s = (double)blocks * 256 * iters * 8 / (1e-3 * ms);
  return r;
}

int fv_debug_math(const double *x, double *out_rsqrt, double *out_rcp, long n, void *stream) {
  if (!x || !out_rsqrt || !out_rcp || n < 0) return FV_EINVAL;
  FV_CK(launch_debug_math(x, out_rsqrt, out_rcp, n, static_cast<cudaStream_t>(stream)));
  return FV_OK;
}

}  // extern "C"
