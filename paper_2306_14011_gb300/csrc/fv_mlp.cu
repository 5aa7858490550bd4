// Surrogate network of the autotuner (paper Sec. 3.3, Table "para-setting"):
// a fully connected FP64 regressor with ReLU hidden layers and an identity
// output, trained by minibatch Adam on 1/2 mean squared error plus an L2
// penalty alpha/(2B) ||W||^2.  The layers are tiny (widths <= 1024, batches of
// 200), so each kernel maps one thread to one output element and sums in a
// fixed order: results are deterministic run to run.  (Tensor cores do not
// apply: FP64 tensor throughput on this part is far below its FP32 rates and
// the work is microseconds per batch.)
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fv.h"
#include "fv_internal.h"

namespace fvk {

namespace {

constexpr int kMaxLayers = 8;
constexpr int kMaxWidth = 1024;

// out[r][j] = act(sum_i in[row(r)][i] W[i][j] + b[j]); row(r) = idx[r] if idx.
__global__ void dense_forward(const double *in, const int *idx, long rows, int fin, int fout, const double *W,
                              const double *b, double *out, int relu) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= rows * fout) return;
  const long r = t / fout;
  const int j = (int)(t - r * fout);
  const long src = idx ? (long)idx[r] : r;
  const double *x = in + src * fin;
  double acc = b[j];
  for (int i = 0; i < fin; ++i) acc = fma(x[i], W[(long)i * fout + j], acc);
  out[t] = (relu && acc < 0.0) ? 0.0 : acc;
}

// delta[r] = out[r] - y[idx[r]] (identity output, width 1).
__global__ void output_delta(const double *out, const double *y, const int *idx, int rows, double *delta) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < rows) delta[r] = out[r] - y[idx[r]];
}

// gW[i][j] = (sum_r A[row(r)][i] delta[r][j] + alpha W[i][j]) / B;  gb[j] = sum_r delta[r][j] / B
__global__ void dense_grads(const double *A, const int *idx, int rows, int fin, int fout, const double *delta,
                            const double *W, double alpha, double *gW, double *gb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nW = fin * fout;
  if (t < nW) {
    const int i = t / fout, j = t - (t / fout) * fout;
    double acc = 0.0;
    for (int r = 0; r < rows; ++r) {
      const long src = idx ? (long)idx[r] : r;
      acc = fma(A[src * fin + i], delta[(long)r * fout + j], acc);
    }
    gW[t] = (acc + alpha * W[t]) / rows;
  } else if (t < nW + fout) {
    const int j = t - nW;
    double acc = 0.0;
    for (int r = 0; r < rows; ++r) acc += delta[(long)r * fout + j];
    gb[j] = acc / rows;
  }
}

// dprev[r][i] = (sum_j delta[r][j] W[i][j]) * [A[r][i] > 0]   (ReLU derivative)
__global__ void dense_backprop(const double *delta, const double *W, const double *A, int rows, int fin, int fout,
                               double *dprev) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * fin) return;
  const int r = t / fin, i = t - (t / fin) * fin;
  double acc = 0.0;
  for (int j = 0; j < fout; ++j) acc = fma(delta[(long)r * fout + j], W[(long)i * fout + j], acc);
  dprev[t] = A[t] > 0.0 ? acc : 0.0;
}

// Adam (Kingma & Ba), efficient form: lr_t carries the bias corrections.
__global__ void adam_update(double *p, const double *g, double *m, double *v, long n, double b1, double b2,
                            double lr_t, double eps) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double gt = g[t];
  const double mt = b1 * m[t] + (1.0 - b1) * gt;
  const double vt = b2 * v[t] + (1.0 - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  p[t] -= lr_t * mt / (sqrt(vt) + eps);
}

// acc += B * (1/2 mean(delta^2) + alpha/(2B) sum_l ||W_l||^2)  (one CTA, fixed order)
__global__ void batch_loss(const double *delta, int rows, const double *params, const long *woff, const long *wlen,
                           int nl, double alpha, double *acc) {
  __shared__ double red[256];
  double s = 0.0, w2 = 0.0;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) s = fma(delta[r], delta[r], s);
  for (int l = 0; l < nl; ++l)
    for (long k = threadIdx.x; k < wlen[l]; k += blockDim.x) {
      const double w = params[woff[l] + k];
      w2 = fma(w, w, w2);
    }
  red[threadIdx.x] = 0.5 * s + 0.5 * alpha * w2;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) *acc += red[0];
}

inline unsigned nblocks(long work, int threads) { return (unsigned)((work + threads - 1) / threads); }

struct Net {
  int nl;
  int sizes[kMaxLayers + 1];
  long woff[kMaxLayers], boff[kMaxLayers];
  long nparams;
};

bool make_net(int nl, const int *sizes, Net &net) {
  if (nl < 1 || nl > kMaxLayers || !sizes) return false;
  net.nl = nl;
  long off = 0;
  for (int l = 0; l <= nl; ++l) {
    if (sizes[l] < 1 || sizes[l] > kMaxWidth) return false;
    net.sizes[l] = sizes[l];
  }
  if (sizes[nl] != 1) return false;
  for (int l = 0; l < nl; ++l) {
    net.woff[l] = off;
    off += (long)sizes[l] * sizes[l + 1];
    net.boff[l] = off;
    off += sizes[l + 1];
  }
  net.nparams = off;
  return true;
}

}  // namespace

// Forward pass over `rows` inputs in chunks; act0/act1: ping-pong buffers of
// chunk * max width doubles.
cudaError_t mlp_forward(const Net &net, const double *params, const double *X, long n, double *out, double *act0,
                        double *act1, long chunk, cudaStream_t st) {
  for (long r0 = 0; r0 < n; r0 += chunk) {
    const long rows = (n - r0 < chunk) ? n - r0 : chunk;
    const double *in = X + r0 * net.sizes[0];
    for (int l = 0; l < net.nl; ++l) {
      const bool last = l == net.nl - 1;
      double *dst = last ? out + r0 : ((l & 1) ? act1 : act0);
      const int fo = net.sizes[l + 1];
      dense_forward<<<nblocks(rows * fo, 256), 256, 0, st>>>(in, nullptr, rows, net.sizes[l], fo,
                                                             params + net.woff[l], params + net.boff[l], dst,
                                                             last ? 0 : 1);
      in = dst;
    }
  }
  return cudaGetLastError();
}

}  // namespace fvk

using namespace fvk;

extern "C" int fv_mlp_predict(int nl, const int *sizes, const double *params, const double *X, long n, double *out,
                              void *stream) {
  Net net;
  if (!make_net(nl, sizes, net) || !params || !X || !out || n < 0) return FV_EINVAL;
  if (n == 0) return FV_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int maxw = 1;
  for (int l = 1; l < nl; ++l) maxw = sizes[l] > maxw ? sizes[l] : maxw;
  const long chunk = n < 65536 ? n : 65536;
  double *buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * 2 * chunk * maxw) != cudaSuccess) {
    (void)cudaGetLastError();
    return FV_ENOMEM;
  }
  cudaError_t e = mlp_forward(net, params, X, n, out, buf, buf + chunk * maxw, chunk, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return FV_ECUDA;
  }
  return FV_OK;
}

extern "C" int fv_mlp_train(int nl, const int *sizes, double *params, const double *X, const double *y, long n,
                            const int *order, int epochs, const fv_mlp_hyper *h, double *loss_out,
                            int *epochs_run, void *stream) {
  Net net;
  if (!make_net(nl, sizes, net) || !params || !X || !y || !order || !h || n < 1 || epochs < 0 || h->batch < 1 ||
      !(h->lr > 0.0) || !(h->beta1 >= 0.0 && h->beta1 < 1.0) || !(h->beta2 >= 0.0 && h->beta2 < 1.0) ||
      !(h->eps > 0.0) || !(h->alpha >= 0.0))
    return FV_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int B = h->batch < n ? h->batch : (int)n;
  long acts = 0;
  for (int l = 1; l <= nl; ++l) acts += (long)B * sizes[l];
  int maxw = 1;
  for (int l = 0; l <= nl; ++l) maxw = sizes[l] > maxw ? sizes[l] : maxw;
  // workspace: activations, two delta buffers, grads, Adam m and v, loss, layer tables
  const size_t nd = (size_t)acts + 2 * (size_t)B * maxw + 3 * (size_t)net.nparams + 1;
  double *ws = nullptr;
  long *tab = nullptr;
  if (cudaMalloc(&ws, sizeof(double) * nd) != cudaSuccess || cudaMalloc(&tab, sizeof(long) * 2 * kMaxLayers) !=
                                                                  cudaSuccess) {
    if (ws) cudaFree(ws);
    (void)cudaGetLastError();
    return FV_ENOMEM;
  }
  double *A[kMaxLayers + 1];
  A[0] = nullptr;  // layer-0 activations are rows of X through the index array
  double *p = ws;
  for (int l = 1; l <= nl; ++l) {
    A[l] = p;
    p += (long)B * sizes[l];
  }
  double *d0 = p, *d1 = p + (size_t)B * maxw;
  p += 2 * (size_t)B * maxw;
  double *grad = p, *m = p + net.nparams, *v = p + 2 * net.nparams;
  double *loss = v + net.nparams;
  long htab[2 * kMaxLayers];
  for (int l = 0; l < nl; ++l) {
    htab[l] = net.woff[l];
    htab[kMaxLayers + l] = (long)sizes[l] * sizes[l + 1];
  }
  cudaError_t e = cudaMemcpyAsync(tab, htab, sizeof(htab), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m, 0, sizeof(double) * 2 * net.nparams, st);
  long t = 0;
  int ran = 0;
  double best = INFINITY;
  int bad = 0;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    e = cudaMemsetAsync(loss, 0, sizeof(double), st);
    const int *ord = order + (long)ep * n;
    for (long s0 = 0; s0 < n && e == cudaSuccess; s0 += B) {
      const int rows = (int)((n - s0 < B) ? n - s0 : B);
      const int *idx = ord + s0;
      // forward
      for (int l = 0; l < nl; ++l) {
        const int fo = sizes[l + 1];
        dense_forward<<<nblocks((long)rows * fo, 256), 256, 0, st>>>(
            l == 0 ? X : A[l], l == 0 ? idx : nullptr, rows, sizes[l], fo, params + net.woff[l],
            params + net.boff[l], A[l + 1], l < nl - 1 ? 1 : 0);
      }
      output_delta<<<nblocks(rows, 256), 256, 0, st>>>(A[nl], y, idx, rows, d0);
      batch_loss<<<1, 256, 0, st>>>(d0, rows, params, tab, tab + kMaxLayers, nl, h->alpha, loss);
      // backward
      double *dcur = d0, *dnext = d1;
      for (int l = nl - 1; l >= 0; --l) {
        const int fi = sizes[l], fo = sizes[l + 1];
        dense_grads<<<nblocks((long)fi * fo + fo, 256), 256, 0, st>>>(
            l == 0 ? X : A[l], l == 0 ? idx : nullptr, rows, fi, fo, dcur, params + net.woff[l], h->alpha,
            grad + net.woff[l], grad + net.boff[l]);
        if (l > 0) {
          dense_backprop<<<nblocks((long)rows * fi, 256), 256, 0, st>>>(dcur, params + net.woff[l], A[l], rows, fi,
                                                                       fo, dnext);
          double *tmp = dcur;
          dcur = dnext;
          dnext = tmp;
        }
      }
      ++t;
      const double lr_t = h->lr * std::sqrt(1.0 - std::pow(h->beta2, (double)t)) / (1.0 - std::pow(h->beta1, (double)t));
      adam_update<<<nblocks(net.nparams, 256), 256, 0, st>>>(params, grad, m, v, net.nparams, h->beta1, h->beta2,
                                                            lr_t, h->eps);
      e = cudaGetLastError();
    }
    double lh = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&lh, loss, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) break;
    lh /= (double)n;
    if (loss_out) loss_out[ep] = lh;
    ++ran;
    // stop once the epoch loss failed to improve by tol for more than n_iter_no_change epochs
    if (lh > best - h->tol)
      ++bad;
    else
      bad = 0;
    if (lh < best) best = lh;
    if (h->n_iter_no_change > 0 && bad > h->n_iter_no_change) break;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(ws);
  cudaFree(tab);
  if (epochs_run) *epochs_run = ran;
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return FV_ECUDA;
  }
  return FV_OK;
}
