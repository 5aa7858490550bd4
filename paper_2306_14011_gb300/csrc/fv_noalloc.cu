// fv_residual_noalloc: the residual and its norms without any allocation.
//
// For callers that cannot allocate device memory at the time they call, and
// therefore cannot create an fv_ctx: services that fix their device-memory
// budget at start-up, plug-ins running inside an application that owns the
// device's memory, or hosts that cannot afford the device-wide
// synchronisation cudaFree implies.  The only scratch the residual needs,
// the per-CTA partial sums of R_v^2, lives in a fixed array below.
#include <cstring>
#include <mutex>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/fv.h"
#include "fv_internal.h"

using namespace fvk;

namespace {

// Layout: kCtrl doubles of control words (word 0: device flags), then the
// partial sums, nvar per CTA.  1 MiB + 256 B; every GPU that loads the library
// holds it until the process exits.
constexpr long long kCtrl = 32;
constexpr long long kPartials = 131072;
static __device__ __align__(256) double g_noalloc_scratch[kCtrl + kPartials];

constexpr int kMaxDevices = 64;
struct DeviceSetup {
  bool ready;
  double *scratch;  // device address of g_noalloc_scratch on this device
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

// Once per device, with that device current: the device address of the
// scratch array (its name in host code is only a host-side stand-in) and the
// stage kernels' shared-memory limit.
int setup_device(int dev, double **scratch) {
  if (dev < 0 || dev >= kMaxDevices) return FV_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_setup[dev].ready) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      (void)cudaGetLastError();
      return FV_ECUDA;
    }
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        stage_kernel_attributes(2, (size_t)optin) != cudaSuccess ||
        stage_kernel_attributes(3, (size_t)optin) != cudaSuccess) {
      (void)cudaGetLastError();
      return FV_ECUDA;
    }
    g_setup[dev].scratch = static_cast<double *>(p);
    g_setup[dev].ready = true;
  }
  *scratch = g_setup[dev].scratch;
  return FV_OK;
}

}  // namespace

extern "C" int fv_residual_noalloc(const fv_grid *g, const fv_scheme *s, const double *U, double *R,
                                   double *rnorm2, void *stream) {
  if (validate_grid(g) != FV_OK || !s || !(s->gamma > 1.0) || !(s->eps >= 0.0) || !(s->eps <= 2.0) || !(s->efix >= 0.0) ||
      !(s->efix < 1.0) || s->limiter < FV_LIM_MINMOD || s->limiter > FV_LIM_NONE ||
      (s->recon != FV_RECON_CONSERVED && s->recon != FV_RECON_PRIMITIVE))
    return FV_EINVAL;
  if (!U || !R || U == R) return FV_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return FV_ECUDA;
  }
  // device (or managed) memory of the current GPU only
  if (pointer_kind(U, dev) != PTR_DEVICE || pointer_kind(R, dev) != PTR_DEVICE ||
      (rnorm2 && pointer_kind(rnorm2, dev) != PTR_DEVICE))
    return FV_EINVAL;
  fv_launch l;
  if (fv_default_launch(g, &l) != FV_OK) return FV_EINVAL;
  const fv_kernel_cfg &k = l.stage[0];
  const int nv = g->dim + 2;
  int nt[3];
  for (int d = 0; d < 3; ++d) nt[d] = (d < g->dim) ? (g->n[d] + k.tile[d] - 1) / k.tile[d] : 1;
  const long long nblk = (long long)nt[0] * nt[1] * nt[2];
  if (nblk >= (1ll << 31)) return FV_EINVAL;
  if (rnorm2 && nblk * nv > kPartials) return FV_EINVAL;  // grid too large for the fixed scratch
  double *scratch = nullptr;
  int r = setup_device(dev, &scratch);
  if (r) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The flags word is where a kernel would raise a timed-out tile-load wait;
  // plain tile loads have no such wait, and nothing reads it back.  It must
  // start at zero; the partials are all rewritten by this call.
  unsigned *flags = reinterpret_cast<unsigned *>(scratch);
  if (cudaMemsetAsync(flags, 0, sizeof(unsigned), st) != cudaSuccess) {
    (void)cudaGetLastError();
    return FV_ECUDA;
  }
  StageArgs a;
  memset(&a, 0, sizeof(a));
  a.Us = U;
  a.Un = U;
  a.out = R;
  a.norm_part = rnorm2 ? scratch + kCtrl : nullptr;
  double h[3];
  for (int d = 0; d < 3; ++d) {
    a.n[d] = g->n[d];
    a.tile[d] = k.tile[d];
    a.ntile[d] = nt[d];
    a.bc[d][0] = g->bc[d][0];
    a.bc[d][1] = g->bc[d][1];
    h[d] = (d < g->dim) ? g->len[d] / g->n[d] : 1.0;
  }
  for (int d = 0; d < 3; ++d) {
    double ds = 1.0;
    for (int e = 0; e < g->dim; ++e)
      if (e != d) ds *= h[e];
    a.ds[d] = ds;
    a.inv_h[d] = (d < g->dim) ? g->n[d] / g->len[d] : 1.0;  // as the batched kernel's n / len
  }
  a.use_tma = 0;  // plain loads: no tensor map, results identical to the TMA loader
  a.march = k.march;
  a.limiter = s->limiter;
  a.recon = s->recon;
  a.inv_g1 = 1.0 / (s->gamma - 1.0);
  a.cL = 0.25 * s->eps * (1.0 - s->kappa);
  a.cR = 0.25 * s->eps * (1.0 + s->kappa);
  a.g1 = s->gamma - 1.0;
  a.half_eps = 0.5 * s->eps;
  a.efix = s->efix;
  a.inv2efix = s->efix > 0.0 ? 0.5 / s->efix : 0.0;
  a.flags = flags;
  CUtensorMap unused;
  memset(&unused, 0, sizeof(unused));
  if (launch_stage(g->dim, MODE_RESIDUAL, &unused, a, k.threads, st) != cudaSuccess) {
    (void)cudaGetLastError();
    return FV_ECUDA;
  }
  if (rnorm2 && launch_norm_finalize(a.norm_part, (int)nblk, nv, rnorm2, st) != cudaSuccess) {
    (void)cudaGetLastError();
    return FV_ECUDA;
  }
  return FV_OK;
}
