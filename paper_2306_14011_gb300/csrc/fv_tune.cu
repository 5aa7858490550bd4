// fv_tune: the paper's machine-learning autotuner (Sec. 3.3-3.6) over the
// launch parameters of this library's kernels.
//
// The paper tunes gang and vector length of seven OpenACC kernels (14
// parameters, Table "tuning-parameters") by timing a random sample of
// configurations, fitting a fully connected ReLU network (Adam, Table
// "para-setting") to run time on standardised features, and using the model
// to find fast configurations.  Two spaces, after the context's kernel
// structure: FV_SPLIT is the paper's own -- gang count (CTAs) and vector
// length (threads) of each split kernel over the Table's value sets, 14
// parameters in 2D, 18 in 3D; FV_FUSED tunes the three fused RK-stage kernels
// and the time-step reduction -- tile shape, threads per CTA and tile loader
// per stage (and the 3D kernel kind), plus the reduction's threads and grid:
// 14 parameters in 2D, 20 in 3D.  Random numbers come from SplitMix64
// (Steele, Lea and Flood, 2014).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <set>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/fv.h"
#include "fv_internal.h"

using namespace fvk;

namespace {

struct SplitMix64 {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
  int below(int n) { return (int)(uniform() * n); }
};

struct Space {
  int dim, mode, per_stage, nparams;
  std::vector<std::vector<int>> vals;
  std::vector<int> slots;  // FV_SPLIT: the split kernel of each (gang, vector) pair
};

Space make_space(int dim, int mode) {
  Space sp;
  sp.dim = dim;
  sp.mode = mode;
  sp.per_stage = 0;
  if (mode == FV_SPLIT) {
    // Table "tuning-parameters": gang 100..1000 step 100, vector 32..384 step 32
    std::vector<int> gang, vector;
    for (int g = 100; g <= 1000; g += 100) gang.push_back(g);
    for (int v = 32; v <= 384; v += 32) vector.push_back(v);
    for (int d = 0; d < dim; ++d) sp.slots.push_back(FV_SK_LIMITER + d);
    for (int d = 0; d < dim; ++d) sp.slots.push_back(FV_SK_FLUX + d);
    sp.slots.insert(sp.slots.end(), {FV_SK_SOURCE, FV_SK_RHS, FV_SK_UPDATE});
    for (size_t q = 0; q < sp.slots.size(); ++q) {
      sp.vals.push_back(gang);
      sp.vals.push_back(vector);
    }
    sp.nparams = (int)sp.vals.size();
    return sp;
  }
  const std::vector<int> threads = {64, 96, 128, 160, 192, 224, 256};
  for (int s = 0; s < 3; ++s) {
    if (dim == 2) {
      sp.vals.push_back({8, 16, 32, 64, 128});
      sp.vals.push_back({2, 4, 8, 16, 32});
    } else {
      sp.vals.push_back({8, 16, 32});
      sp.vals.push_back({4, 8, 16});
      sp.vals.push_back({2, 4, 8});
    }
    sp.vals.push_back(threads);
    sp.vals.push_back({FV_LOADER_TMA, FV_LOADER_PLAIN});
    if (dim == 3) sp.vals.push_back({0, 1});  // box tiles / z-marching (chunk = 8 x tile-z value)
  }
  sp.per_stage = dim == 2 ? 4 : 6;
  sp.vals.push_back({128, 256, 512, 1024});  // time-step kernel threads
  sp.vals.push_back({1, 2, 4, 8});           // time-step kernel CTAs per SM
  sp.nparams = (int)sp.vals.size();
  return sp;
}

typedef std::vector<int> Cfg;  // index into each value set

// The launch of configuration c; `base` supplies what the space leaves fixed
// (FV_SPLIT: the fused stage and time-step fields).
fv_launch to_launch(const Space &sp, const Cfg &c, int sms, const fv_launch &base) {
  fv_launch l;
  if (sp.mode == FV_SPLIT) {
    l = base;
    l.mode = FV_SPLIT;
    for (size_t q = 0; q < sp.slots.size(); ++q) {
      l.split[sp.slots[q]].grid = sp.vals[2 * q][c[2 * q]];
      l.split[sp.slots[q]].threads = sp.vals[2 * q + 1][c[2 * q + 1]];
    }
    return l;
  }
  l = base;
  l.mode = FV_FUSED;
  for (int s = 0; s < 3; ++s) {
    const int b = s * sp.per_stage;
    fv_kernel_cfg &k = l.stage[s];
    k.tile[0] = sp.vals[b][c[b]];
    k.tile[1] = sp.vals[b + 1][c[b + 1]];
    k.tile[2] = sp.dim == 3 ? sp.vals[b + 2][c[b + 2]] : 1;
    const int o = sp.dim == 3 ? 3 : 2;
    k.threads = sp.vals[b + o][c[b + o]];
    k.loader = sp.vals[b + o + 1][c[b + o + 1]];
    k.march = sp.dim == 3 ? sp.vals[b + o + 2][c[b + o + 2]] : 0;
    if (k.march) k.tile[2] *= 8;  // planes per chunk: 16, 32 or 64
    k.grid = 0;
  }
  const int b = 3 * sp.per_stage;
  l.dt.threads = sp.vals[b][c[b]];
  l.dt.grid = sp.vals[b + 1][c[b + 1]] * sms;
  return l;
}

// Features: log2 of the numeric parameters (tiles, thread counts, grid
// multiplier, gang counts), the loader and the 3D kernel choice as 0/1.
void features(const Space &sp, const Cfg &c, double *f) {
  for (int p = 0; p < sp.nparams; ++p) {
    const int v = sp.vals[p][c[p]];
    f[p] = (sp.vals[p].size() == 2 && sp.vals[p][0] == 0) ? (double)v : std::log2((double)v);
  }
}

uint64_t key(const Space &sp, const Cfg &c) {
  uint64_t k = 0;
  for (int p = 0; p < sp.nparams; ++p) k = k * (uint64_t)sp.vals[p].size() + (uint64_t)c[p];
  return k;
}

// The index vector of launch l in the space, if every value is in it.
bool cfg_of(const Space &sp, const fv_launch &l, int sms, Cfg *out) {
  Cfg c(sp.nparams);
  auto find = [&](int p, int v) {
    for (int i = 0; i < (int)sp.vals[p].size(); ++i)
      if (sp.vals[p][i] == v) {
        c[p] = i;
        return true;
      }
    return false;
  };
  if (sp.mode == FV_SPLIT) {
    if (l.mode != FV_SPLIT) return false;
    for (size_t q = 0; q < sp.slots.size(); ++q)
      if (!find((int)(2 * q), l.split[sp.slots[q]].grid) || !find((int)(2 * q + 1), l.split[sp.slots[q]].threads))
        return false;
    *out = c;
    return true;
  }
  if (l.mode != FV_FUSED) return false;
  for (int s = 0; s < 3; ++s) {
    const int b = s * sp.per_stage;
    const fv_kernel_cfg &k = l.stage[s];
    const int o = sp.dim == 3 ? 3 : 2;
    if (!find(b, k.tile[0]) || !find(b + 1, k.tile[1])) return false;
    if (sp.dim == 3 && (!find(b + 2, k.march ? k.tile[2] / 8 : k.tile[2]) || !find(b + o + 2, k.march) ||
                        (k.march && k.tile[2] % 8)))
      return false;
    if (!find(b + o, k.threads) || !find(b + o + 1, k.loader)) return false;
  }
  const int b = 3 * sp.per_stage;
  if (!find(b, l.dt.threads)) return false;
  const int mult = l.dt.grid == 0 ? std::max(1, 2048 / l.dt.threads) : l.dt.grid / sms;  // grid 0: SMs filled
  if (l.dt.grid != 0 && l.dt.grid % sms) return false;
  if (!find(b + 1, mult)) return false;
  *out = c;
  return true;
}

Cfg random_cfg(const Space &sp, SplitMix64 &rng) {
  Cfg c(sp.nparams);
  for (int p = 0; p < sp.nparams; ++p) c[p] = rng.below((int)sp.vals[p].size());
  return c;
}

double r2_score(const std::vector<double> &y, const std::vector<double> &yh) {
  double mean = 0.0;
  for (double v : y) mean += v;
  mean /= (double)y.size();
  double ss_res = 0.0, ss_tot = 0.0;
  for (size_t i = 0; i < y.size(); ++i) {
    ss_res += (y[i] - yh[i]) * (y[i] - yh[i]);
    ss_tot += (y[i] - mean) * (y[i] - mean);
  }
  return ss_tot > 0.0 ? 1.0 - ss_res / ss_tot : 0.0;
}

struct DevBuf {
  void *p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  bool alloc(size_t bytes) { return cudaMalloc(&p, bytes) == cudaSuccess; }
  template <class T>
  T *as() { return static_cast<T *>(p); }
};

}  // namespace

extern "C" int fv_tune_space(int dim, int mode, int *n_params, double *size) {
  if ((dim != 2 && dim != 3) || (mode != FV_FUSED && mode != FV_SPLIT) || !n_params || !size) return FV_EINVAL;
  const Space sp = make_space(dim, mode);
  double points = 1.0;
  for (auto &v : sp.vals) points *= (double)v.size();
  *n_params = sp.nparams;
  *size = points;
  return FV_OK;
}

extern "C" int fv_tune(fv_ctx *ctx, const double *U, const fv_tune_opts *opts_in, fv_launch *best,
                       fv_tune_report *rep) {
  if (!ctx || !U || !best) return FV_EINVAL;
  fv_tune_opts o;
  memset(&o, 0, sizeof(o));
  if (opts_in) o = *opts_in;
  if (o.samples <= 0) o.samples = 1000;
  if (o.steps <= 0) o.steps = 2;
  if (o.repeats <= 0) o.repeats = 1;
  if (o.candidates <= 0) o.candidates = 200000;
  if (o.top <= 0) o.top = 16;
  if (o.final_repeats <= 0) o.final_repeats = 5;
  if (o.rounds <= 0) o.rounds = 3;
  if (o.refine == 0) o.refine = 2;
  if (o.refine < 0) o.refine = 0;
  if (o.seed == 0) o.seed = 1;
  if (o.samples < 8) return FV_EINVAL;
  fv_mlp_hyper h = o.mlp;
  if (!(h.alpha > 0.0)) h.alpha = 1e-4;
  if (!(h.beta1 > 0.0)) h.beta1 = 0.95;
  if (!(h.beta2 > 0.0)) h.beta2 = 0.90;
  if (!(h.lr > 0.0)) h.lr = 9e-4;
  if (!(h.eps > 0.0)) h.eps = 1e-9;
  if (!(h.tol > 0.0)) h.tol = 1e-6;
  if (h.batch <= 0) h.batch = 200;
  if (h.max_epochs <= 0) h.max_epochs = 200;
  if (h.n_iter_no_change <= 0) h.n_iter_no_change = 10;
  const int dim = ctx_dim(ctx), sms = ctx_sm_count(ctx);
  fv_launch deflt;  // the library default: the analogue of the compiler's default launch
  int r;
  if ((r = ctx_default_launch(ctx, &deflt))) return r;
  const Space sp = make_space(dim, deflt.mode);
  const int nf = sp.nparams;
  std::vector<int> sizes;
  sizes.push_back(nf);
  for (int i = 0; i < 4 && o.hidden[i] > 0; ++i) sizes.push_back(o.hidden[i]);
  if (sizes.size() == 1) sizes.insert(sizes.end(), {128, 64, 32});
  sizes.push_back(1);
  const int nl = (int)sizes.size() - 1;

  double *Uw = nullptr;
  if ((r = ctx_work_state(ctx, U, &Uw))) return r;
  SplitMix64 rng{o.seed};

  // every measured configuration, its time, and whether it is held out
  std::vector<Cfg> cfgs;
  std::vector<double> times;
  std::vector<char> held;
  std::set<uint64_t> seen;
  int best_i = -1;
  auto measure = [&](const Cfg &c, bool holdout, int *outcome) -> int {
    *outcome = 0;
    if (!seen.insert(key(sp, c)).second) return FV_OK;
    const fv_launch l = to_launch(sp, c, sms, deflt);
    double t = 0.0;
    const int rr = ctx_time_launch(ctx, Uw, &l, o.steps, o.repeats, &t);
    if (rr == FV_EINVAL) return FV_OK;  // outside the device limits (shared memory)
    if (rr) return rr;
    cfgs.push_back(c);
    times.push_back(t);
    held.push_back(holdout ? 1 : 0);
    if (best_i < 0 || t < times[best_i]) {
      best_i = (int)times.size() - 1;
      *outcome = 2;
    } else {
      *outcome = 1;
    }
    return FV_OK;
  };

  // ---- 1. time the default launch (a training sample) and a random sample of
  // valid configurations (25% held out)
  int outcome;
  {
    Cfg c0;
    if (cfg_of(sp, deflt, sms, &c0) && (r = measure(c0, false, &outcome))) return r;
  }
  const int n_default_samples = (int)cfgs.size();
  for (int attempts = 0; (int)cfgs.size() < o.samples + n_default_samples && attempts < 50 * o.samples;
       ++attempts) {
    const bool hold = (rng.uniform() < 0.25);
    if ((r = measure(random_cfg(sp, rng), hold, &outcome))) return r;
  }
  if ((int)cfgs.size() < 8) return FV_EINVAL;
  double best_sampled = INFINITY;  // best of the random sample (the default excluded)
  for (size_t i = n_default_samples; i < times.size(); ++i) best_sampled = std::min(best_sampled, times[i]);

  // ---- 2. surrogate rounds
  DevBuf dP, dOut;
  long np = 0;
  for (int l = 0; l < nl; ++l) np += (long)sizes[l] * sizes[l + 1] + sizes[l + 1];
  if (!dP.alloc(sizeof(double) * np)) return FV_ENOMEM;
  std::vector<double> mu(nf), sd(nf);
  double ymu = 0.0, ysd = 1.0, r2_tr = 0.0, r2_te = 0.0;
  int epochs = 0, ntr = 0, nte = 0, rounds_run = 0;
  std::vector<Cfg> cand;
  std::vector<double> CFraw;
  {  // candidate pool, fixed for all rounds
    std::set<uint64_t> cseen;
    cand.reserve(o.candidates);
    for (int attempts = 0; (int)cand.size() < o.candidates && attempts < 4 * o.candidates; ++attempts) {
      Cfg c = random_cfg(sp, rng);
      if (!cseen.insert(key(sp, c)).second) continue;
      const fv_launch l = to_launch(sp, c, sms, deflt);
      if (ctx_validate_launch(ctx, &l) != FV_OK) continue;  // cannot launch (shared memory)
      cand.push_back(c);
    }
    CFraw.resize(cand.size() * (size_t)nf);
    for (size_t q = 0; q < cand.size(); ++q) features(sp, cand[q], &CFraw[q * nf]);
  }
  DevBuf dC, dCo;
  const long nc = (long)cand.size();
  if (nc > 0 && (!dC.alloc(sizeof(double) * CFraw.size()) || !dCo.alloc(sizeof(double) * nc))) return FV_ENOMEM;
  for (int round = 0; round < o.rounds; ++round) {
    const int n = (int)cfgs.size();
    std::vector<int> tr, te;
    for (int i = 0; i < n; ++i) (held[i] ? te : tr).push_back(i);
    ntr = (int)tr.size();
    nte = (int)te.size();
    if (ntr < 4) break;
    // standardisation on the training rows
    std::vector<double> Fall((size_t)n * nf);
    for (int i = 0; i < n; ++i) features(sp, cfgs[i], &Fall[(size_t)i * nf]);
    for (int p = 0; p < nf; ++p) {
      double m = 0.0, v = 0.0;
      for (int i : tr) m += Fall[(size_t)i * nf + p];
      m /= ntr;
      for (int i : tr) v += (Fall[(size_t)i * nf + p] - m) * (Fall[(size_t)i * nf + p] - m);
      v /= ntr;
      mu[p] = m;
      sd[p] = v > 0.0 ? std::sqrt(v) : 1.0;
    }
    ymu = 0.0;
    for (int i : tr) ymu += std::log(times[i]);
    ymu /= ntr;
    double yv = 0.0;
    for (int i : tr) yv += (std::log(times[i]) - ymu) * (std::log(times[i]) - ymu);
    ysd = yv > 0.0 ? std::sqrt(yv / ntr) : 1.0;
    // rows: training rows first, then held-out rows
    std::vector<double> X((size_t)n * nf), z(n);
    std::vector<int> rows(tr);
    rows.insert(rows.end(), te.begin(), te.end());
    for (int q = 0; q < n; ++q) {
      const int i = rows[q];
      for (int p = 0; p < nf; ++p) X[(size_t)q * nf + p] = (Fall[(size_t)i * nf + p] - mu[p]) / sd[p];
      z[q] = (std::log(times[i]) - ymu) / ysd;
    }
    std::vector<double> params(np);
    {
      long k = 0;
      for (int l = 0; l < nl; ++l) {
        const double bound = std::sqrt(6.0 / (sizes[l] + sizes[l + 1]));
        for (long q = 0; q < (long)sizes[l] * sizes[l + 1] + sizes[l + 1]; ++q)
          params[k++] = (2.0 * rng.uniform() - 1.0) * bound;
      }
    }
    std::vector<int> order((size_t)h.max_epochs * ntr);
    for (int e = 0; e < h.max_epochs; ++e) {
      int *ord = &order[(size_t)e * ntr];
      std::iota(ord, ord + ntr, 0);
      for (int i = ntr - 1; i > 0; --i) std::swap(ord[i], ord[rng.below(i + 1)]);
    }
    DevBuf dX, dy, dO, dPr;
    if (!dX.alloc(sizeof(double) * X.size()) || !dy.alloc(sizeof(double) * n) ||
        !dO.alloc(sizeof(int) * order.size()) || !dPr.alloc(sizeof(double) * n))
      return FV_ENOMEM;
    if (cudaMemcpy(dX.p, X.data(), sizeof(double) * X.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dy.p, z.data(), sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dP.p, params.data(), sizeof(double) * np, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dO.p, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return FV_ECUDA;
    if ((r = fv_mlp_train(nl, sizes.data(), dP.as<double>(), dX.as<double>(), dy.as<double>(), ntr, dO.as<int>(),
                          h.max_epochs, &h, nullptr, &epochs, nullptr)))
      return r;
    if ((r = fv_mlp_predict(nl, sizes.data(), dP.as<double>(), dX.as<double>(), n, dPr.as<double>(), nullptr)))
      return r;
    std::vector<double> pz(n);
    if (cudaMemcpy(pz.data(), dPr.p, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess) return FV_ECUDA;
    std::vector<double> ytr, ptr_, yte, pte;
    for (int q = 0; q < n; ++q) {
      const double tt = times[rows[q]], pt = std::exp(ymu + ysd * pz[q]);
      (q < ntr ? ytr : yte).push_back(tt);
      (q < ntr ? ptr_ : pte).push_back(pt);
    }
    r2_tr = r2_score(ytr, ptr_);
    r2_te = nte > 1 ? r2_score(yte, pte) : 0.0;
    ++rounds_run;
    // score the candidate pool and measure the best predicted not yet measured
    if (nc == 0) break;
    std::vector<double> CF(CFraw.size());
    for (size_t q = 0; q < CF.size(); ++q) CF[q] = (CFraw[q] - mu[q % nf]) / sd[q % nf];
    if (cudaMemcpy(dC.p, CF.data(), sizeof(double) * CF.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return FV_ECUDA;
    if ((r = fv_mlp_predict(nl, sizes.data(), dP.as<double>(), dC.as<double>(), nc, dCo.as<double>(), nullptr)))
      return r;
    std::vector<double> pc(nc);
    if (cudaMemcpy(pc.data(), dCo.p, sizeof(double) * nc, cudaMemcpyDeviceToHost) != cudaSuccess) return FV_ECUDA;
    std::vector<long> ix(nc);
    std::iota(ix.begin(), ix.end(), 0);
    std::sort(ix.begin(), ix.end(), [&](long a, long b) { return pc[a] < pc[b]; });
    int taken = 0;
    for (long q = 0; q < nc && taken < o.top; ++q) {
      if (seen.count(key(sp, cand[ix[q]]))) continue;
      if ((r = measure(cand[ix[q]], false, &outcome))) return r;
      if (outcome) ++taken;
    }
  }

  // ---- 3. coordinate-descent refinement of the best measured configuration
  int n_refined = 0;
  for (int sweep = 0; sweep < o.refine; ++sweep) {
    bool improved = false;
    for (int p = 0; p < nf; ++p) {
      for (int v = 0; v < (int)sp.vals[p].size(); ++v) {
        Cfg c = cfgs[best_i];
        if (c[p] == v) continue;
        c[p] = v;
        const size_t before = times.size();
        if ((r = measure(c, false, &outcome))) return r;
        if (times.size() > before) ++n_refined;
        if (outcome == 2) improved = true;
      }
    }
    if (!improved) break;
  }
  fv_launch tuned = to_launch(sp, cfgs[best_i], sms, deflt);

  // ---- 4. exhaustive search of the reduced space (shared tile and threads)
  fv_launch exh_best;
  memset(&exh_best, 0, sizeof(exh_best));
  int n_exh = 0;
  if (o.exhaustive && sp.mode == FV_SPLIT) {  // one shared (gang, vector) for every split kernel
    double t_exh = INFINITY;
    for (int gang : sp.vals[0])
      for (int vec : sp.vals[1]) {
        fv_launch l = deflt;
        for (int slot : sp.slots) {
          l.split[slot].grid = gang;
          l.split[slot].threads = vec;
        }
        double t = 0.0;
        r = ctx_time_launch(ctx, Uw, &l, o.steps, o.repeats, &t);
        if (r == FV_EINVAL) continue;
        if (r) return r;
        ++n_exh;
        if (t < t_exh) {
          t_exh = t;
          exh_best = l;
        }
      }
  } else if (o.exhaustive) {
    std::vector<std::vector<int>> axes;
    if (dim == 2)
      axes = {sp.vals[0], sp.vals[1], {1}, sp.vals[2]};
    else
      axes = {sp.vals[0], sp.vals[1], sp.vals[2], sp.vals[3]};
    double t_exh = INFINITY;
    for (int a : axes[0])
      for (int b : axes[1])
        for (int cz : axes[2])
          for (int th : axes[3]) {
            fv_launch l = deflt;
            for (int s = 0; s < 3; ++s) {
              l.stage[s].tile[0] = a;
              l.stage[s].tile[1] = b;
              l.stage[s].tile[2] = dim == 3 ? cz : 1;
              l.stage[s].threads = th;
              l.stage[s].loader = FV_LOADER_TMA;
              l.stage[s].march = 0;
            }
            double t = 0.0;
            r = ctx_time_launch(ctx, Uw, &l, o.steps, o.repeats, &t);
            if (r == FV_EINVAL) continue;
            if (r) return r;
            ++n_exh;
            if (t < t_exh) {
              t_exh = t;
              exh_best = l;
            }
          }
  }

  // ---- 5. final comparison, interleaved measurements
  double tf_def = 0.0, tf_tun = 0.0, tf_exh = 0.0;
  {
    std::vector<double> a, b, cc;
    for (int q = 0; q < o.final_repeats; ++q) {
      double t;
      if ((r = ctx_time_launch(ctx, Uw, &deflt, o.steps, 1, &t))) return r;
      a.push_back(t);
      if ((r = ctx_time_launch(ctx, Uw, &tuned, o.steps, 1, &t))) return r;
      b.push_back(t);
      if (n_exh > 0) {
        if ((r = ctx_time_launch(ctx, Uw, &exh_best, o.steps, 1, &t))) return r;
        cc.push_back(t);
      }
    }
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    std::sort(cc.begin(), cc.end());
    tf_def = a[a.size() / 2];
    tf_tun = b[b.size() / 2];
    tf_exh = cc.empty() ? 0.0 : cc[cc.size() / 2];
  }
  // the fastest of the three by median (the search's pick wins ties)
  int chosen = 0;
  double t_ret = tf_tun;
  fv_launch ret = tuned;
  if (tf_def < t_ret) {
    chosen = 1;
    t_ret = tf_def;
    ret = deflt;
  }
  if (n_exh > 0 && tf_exh < t_ret) {
    chosen = 2;
    t_ret = tf_exh;
    ret = exh_best;
  }
  if ((r = fv_set_launch(ctx, &ret))) return r;
  *best = ret;
  if (rep) {
    memset(rep, 0, sizeof(*rep));
    rep->t_default = tf_def;
    rep->t_tuned = t_ret;
    rep->t_search = tf_tun;
    rep->chosen = chosen;
    rep->t_best_sampled = best_sampled;
    rep->t_exhaustive = tf_exh;
    rep->r2_train = r2_tr;
    rep->r2_test = r2_te;
    double space = 1.0;
    for (auto &v : sp.vals) space *= (double)v.size();
    rep->space_size = space;
    rep->n_params = sp.nparams;
    rep->n_train = ntr;
    rep->n_test = nte;
    rep->epochs = epochs;
    rep->n_measured = (int)times.size();
    rep->n_exhaustive = n_exh;
    rep->rounds = rounds_run;
    rep->n_refined = n_refined;
    rep->exhaustive_best = exh_best;
    rep->search_best = tuned;
  }
  return FV_OK;
}
