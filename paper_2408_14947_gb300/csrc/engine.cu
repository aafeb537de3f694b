// Host engine and C ABI of the ERX per-line step (include/erx.h).
//
// A context owns the FP64 background state (mu: d, K: packed lower d x d) and
// the scratch for one block of T lines.  erx_push_lines cuts the caller's
// lines into blocks and, per block, enqueues on the context's stream:
//   [S1 project] -> S2 stats -> S3 EMA scan -> S4 chol + inverse -> S5 scores -> S6 normalise
// The per-line statistics of a block are independent, so S2, S4 and S5 run
// all T lines at once; only S3 is sequential in t, as a d^2-wide scan.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/erx.h"
#include "erx_internal.cuh"

using namespace erx;

struct erx_ctx {
  erx_config cfg{};
  int B = 0, W = 0, d = 0, T = 0;
  int device = 0;
  int n_sm = 1;
  bool tc_stats = false;
  cudaStream_t stream = nullptr;
  bool int_stats = false;
  bool fp64 = true;
  bool failed = false;
  int64_t t = 0;
  std::vector<double> w_host;   // b x d projection (empty without projection)
  // device buffers
  double* mu_state = nullptr;
  double* K_state = nullptr;
  double* mu_t = nullptr;
  double* K_t = nullptr;
  double* Linv = nullptr;
  float* Linv32 = nullptr;
  uint64_t* S1i = nullptr;
  uint64_t* S2i = nullptr;
  double* mu_hat = nullptr;
  double* shift = nullptr;
  double* S2f = nullptr;
  void* Z = nullptr;
  int* colptr = nullptr;
  int* rows = nullptr;
  double* vals = nullptr;
  unsigned long long* err = nullptr;
  double* ema_scratch = nullptr;
  double* imc_mprev = nullptr;   // IMC: per-line deltas, constants and chunk sums of a block
  float2* L2 = nullptr;          // FP64E: the blocked factor and mu_t as hi/lo floats
  float2* mu2 = nullptr;
  // pushes of several blocks: block b+1's statistics, update and factor (stream A)
  // overlap block b's score (stream B); the buffers that pass from A to B have
  // one copy per slot (b & 1).  Stream A, the chain every block waits on, has
  // the greatest priority and B the least, so that SMs freed by the scores go
  // to the statistics, EMA and factor kernels first; both fork from and join
  // back into the context's stream.
  bool overlap = false;
  cudaStream_t sA = nullptr, sB = nullptr;
  cudaEvent_t ev_fac[2] = {}, ev_fin[2] = {}, ev_join = nullptr, ev_fork = nullptr,
              ev_joinA = nullptr;
  double* mu_t_s[2] = {};
  double* Linv_s[2] = {};
  float* Linv32_s[2] = {};
  void* Z_s[2] = {};
  // ERX_FLAG_PIPELINE: the factor of the current state, made ahead for the next
  // single-line push, and the second stream that defers each line's update
  bool pipeline = false;
  bool have_pre = false;
  double* mu_pre = nullptr;
  double* Lf_pre = nullptr;
  float* Lf32_pre = nullptr;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_start = nullptr, ev_stats = nullptr, ev_scored = nullptr, ev_ready = nullptr;
  // host staging for erx_push_lines_host
  void* h_in[2] = {nullptr, nullptr};
  void* d_in[2] = {nullptr, nullptr};
  void* h_out = nullptr;
  void* d_out = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr};
  cudaEvent_t ev_used[2] = {nullptr, nullptr};
  std::vector<void*> allocs;
  // per-kernel launch counts and event-bracketed timing
  bool profiling = false;
  int64_t launches[ERX_K_COUNT] = {};
  int64_t timed[ERX_K_COUNT] = {};
  double total_ms[ERX_K_COUNT] = {};
  struct Pending { int k; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> spare_events;
  // learned projection and its drift monitor
  erx_encoder* enc = nullptr;
  int audit_every = 0;
  double min_corr_thr = 0.0;
  erx_ctx* audit = nullptr;
  bool fallback = false;
  double last_corr = NAN, min_corr = NAN;
  int64_t audits = 0;
  void* audit_delta = nullptr;       // device, up to T lines of scores
  std::vector<char> h_learned, h_full;
};

namespace {

size_t elem_size(int dt) { return dt == ERX_U16 ? 2 : dt == ERX_F32 ? 4 : 8; }

template <typename T>
erx_status dalloc(erx_ctx* c, T** p, size_t n) {
  void* q = nullptr;
  if (n == 0) n = 1;
  if (cudaMalloc(&q, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return ERX_ENOMEM;
  }
  c->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return ERX_OK;
}

void free_all(erx_ctx* c) {
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  for (int i = 0; i < 2; ++i) {
    if (c->h_in[i]) cudaFreeHost(c->h_in[i]);
    if (c->ev_in[i]) cudaEventDestroy(c->ev_in[i]);
    if (c->ev_used[i]) cudaEventDestroy(c->ev_used[i]);
  }
  if (c->h_out) cudaFreeHost(c->h_out);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  for (cudaEvent_t* e : {&c->ev_start, &c->ev_stats, &c->ev_scored, &c->ev_ready, &c->ev_fac[0],
                        &c->ev_fac[1], &c->ev_fin[0], &c->ev_fin[1], &c->ev_join, &c->ev_fork,
                        &c->ev_joinA})
    if (*e) cudaEventDestroy(*e), *e = nullptr;
  if (c->sA) cudaStreamDestroy(c->sA), c->sA = nullptr;
  if (c->sB) cudaStreamDestroy(c->sB), c->sB = nullptr;
  if (c->side) cudaStreamDestroy(c->side), c->side = nullptr;
  if (c->audit) erx_destroy(c->audit), c->audit = nullptr;
  for (auto& p : c->pending) cudaEventDestroy(p.a), cudaEventDestroy(p.b);
  for (auto e : c->spare_events) cudaEventDestroy(e);
  c->pending.clear();
  c->spare_events.clear();
}

cudaEvent_t take_event(erx_ctx* c) {
  if (!c->spare_events.empty()) {
    cudaEvent_t e = c->spare_events.back();
    c->spare_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets one kernel launch: counts it and, when profiling, records events around it.
struct KernelScope {
  erx_ctx* c;
  int k;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  KernelScope(erx_ctx* c_, int k_, cudaStream_t s_ = nullptr)
      : c(c_), k(k_), st(s_ ? s_ : c_->stream) {
    c->launches[k]++;
    if (c->profiling) {
      a = take_event(c);
      if (a) cudaEventRecord(a, st);
    }
  }
  ~KernelScope() {
    if (a) {
      cudaEvent_t b = take_event(c);
      if (b) {
        cudaEventRecord(b, st);
        c->pending.push_back({k, a, b});
      } else {
        c->spare_events.push_back(a);
      }
    }
  }
};

void resolve_pending(erx_ctx* c) {
  for (auto& p : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->total_ms[p.k] += ms;
      c->timed[p.k]++;
    }
    c->spare_events.push_back(p.a);
    c->spare_events.push_back(p.b);
  }
  c->pending.clear();
  cudaGetLastError();
}

uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

erx_status check_cuda(erx_ctx* c, cudaError_t e) {
  if (e == cudaSuccess) return ERX_OK;
  if (c) c->failed = true;
  return ERX_ECUDA;
}

erx_status validate(const erx_config* cfg) {
  if (!cfg) return ERX_EINVAL;
  if (cfg->bands < 1 || cfg->width < 2) return ERX_EINVAL;
  if (!(cfg->momentum > 0.0 && cfg->momentum <= 1.0)) return ERX_EINVAL;
  if (!(cfg->ridge >= 0.0) || !std::isfinite(cfg->ridge)) return ERX_EINVAL;
  if (cfg->proj != ERX_PROJ_NONE && cfg->proj != ERX_PROJ_SRP && cfg->proj != ERX_PROJ_LEARNED)
    return ERX_EINVAL;
  if (cfg->proj == ERX_PROJ_LEARNED &&
      (cfg->in_dtype != ERX_F32 || cfg->proj_dim < 2 || cfg->proj_dim > 32))
    return ERX_EINVAL;
  if (cfg->proj == ERX_PROJ_SRP && (cfg->proj_dim < 1 || cfg->proj_dim > cfg->bands))
    return ERX_EINVAL;
  if (cfg->order != ERX_UPDATE_THEN_SCORE && cfg->order != ERX_SCORE_THEN_UPDATE)
    return ERX_EINVAL;
  if (cfg->averaging != ERX_AVG_EMA && cfg->averaging != ERX_AVG_IMC &&
      cfg->averaging != ERX_AVG_POOLED)
    return ERX_EINVAL;
  if ((cfg->flags & ERX_FLAG_PIPELINE) &&
      (cfg->order != ERX_SCORE_THEN_UPDATE || cfg->proj == ERX_PROJ_LEARNED))
    return ERX_EINVAL;
  if (cfg->in_dtype < ERX_U16 || cfg->in_dtype > ERX_F64) return ERX_EINVAL;
  if (cfg->in_dtype == ERX_U16 && (cfg->in_bits < 1 || cfg->in_bits > 16)) return ERX_EINVAL;
  if (cfg->form < ERX_FORM_FP64 || cfg->form > ERX_FORM_FP64E) return ERX_EINVAL;
  if (cfg->form == ERX_FORM_FP64E &&
      (cfg->proj != ERX_PROJ_NONE || (cfg->in_dtype != ERX_U16 && cfg->in_dtype != ERX_F32)))
    return ERX_EUNSUPPORTED;
  if (cfg->block_lines < 0 || cfg->warmup_lines < 0) return ERX_EINVAL;
  const int d = cfg->proj != ERX_PROJ_NONE ? cfg->proj_dim : cfg->bands;
  if (d > kMaxDim || cfg->width > (1 << 20) || cfg->bands > 65536) return ERX_EUNSUPPORTED;
  return ERX_OK;
}

// operand format of the tensor-core kernels for a form: 1 BF16, 2 TF32, 3 3xTF32; 0: none
int tc_format(int form) {
  return form == ERX_FORM_TF32 ? 2 : form == ERX_FORM_BF16 ? 1 : form == ERX_FORM_TF32X3 ? 3 : 0;
}

// Enqueue the whole step for `n` lines at `x` (device), outputs at line offset 0 of the given
// pointers.
erx_status audit_block(erx_ctx* c, const void* x, int64_t n, int64_t stride_elems, void* delta);

void enqueue_stats(erx_ctx* c, const void* x, int64_t stride_elems, const void* zsrc, int ztype,
                   int64_t zstride, int ps, int T, cudaStream_t st);
void enqueue_update(erx_ctx* c, int T, cudaStream_t st);
void enqueue_score(erx_ctx* c, const void* zsrc, int ztype, int64_t zstride, int ps, int T,
                   const double* mu, const double* Lf, const float* Lf32, void* delta, void* dn,
                   uint8_t* mask, uint8_t* det, cudaStream_t st);

erx_status run_block(erx_ctx* c, const void* x, int64_t n, int64_t stride_elems, void* delta,
                     void* dn, uint8_t* mask, uint8_t* det, int slot = -1) {
  const int T = (int)n, W = c->W, d = c->d, B = c->B;
  if (slot >= 0) {
    // this block's copies of the buffers stream B reads; wait until B is done
    // with them (block b-2)
    c->mu_t = c->mu_t_s[slot];
    c->Linv = c->Linv_s[slot];
    c->Linv32 = c->Linv32_s[slot];
    c->Z = c->Z_s[slot];
    cudaStreamWaitEvent(c->stream, c->ev_fin[slot], 0);
  }
  const bool learned = c->cfg.proj == ERX_PROJ_LEARNED;
  if (learned && !c->enc) return ERX_ESTATE;
  if (learned && c->fallback) {
    // full-band ERX for every line from here on
    const size_t es = elem_size(c->cfg.in_dtype);
    erx_status s = erx_push_lines(c->audit, x, n, stride_elems * (int64_t)es, delta, dn, mask, det);
    c->t += n;
    return s;
  }
  const int in_t = c->cfg.in_dtype;
  cudaStream_t st = c->stream;
  const void* zsrc = x;
  int ztype = in_t;
  int64_t zstride = stride_elems;
  int ps = B;
  if (!c->w_host.empty()) {
    KernelScope ks(c, ERX_K_PROJECT);
    launch_project(in_t, x, stride_elems, B, W, d, T, c->colptr, c->rows, c->vals, c->fp64,
                   c->Z, st);
    zsrc = c->Z;
    ztype = c->fp64 ? ERX_F64 : ERX_F32;
    zstride = (int64_t)W * d;
    ps = d;
  } else if (learned) {
    KernelScope ks(c, ERX_K_ENCODE);
    const float* xf = (const float*)x;
    if (stride_elems == (int64_t)W * B) {
      encoder_forward_on(c->enc, xf, (int64_t)T * W, (float*)c->Z, st);
    } else {
      for (int j = 0; j < T; ++j)
        encoder_forward_on(c->enc, xf + j * stride_elems, W, (float*)c->Z + (int64_t)j * W * d,
                           st);
    }
    zsrc = c->Z;
    ztype = ERX_F32;
    zstride = (int64_t)W * d;
    ps = d;
  }
  enqueue_stats(c, x, stride_elems, zsrc, ztype, zstride, ps, T, st);
  enqueue_update(c, T, st);
  {
    KernelScope ks(c, ERX_K_CHOL);
    launch_chol_inv(c->K_t, d, T, c->cfg.ridge, c->Linv, c->fp64 ? nullptr : c->Linv32, c->err,
                    c->t, st, c->fp64,
                    // FP64E: the previous block's score runs on the FP32 pipe beside the
                    // FP64 factor (measured +7 %); the other forms gain nothing from it
                    slot >= 0 && c->cfg.form == ERX_FORM_FP64E);
  }
  cudaStream_t sb = st;
  if (slot >= 0) {
    cudaEventRecord(c->ev_fac[slot], st);
    sb = c->sB;
    cudaStreamWaitEvent(sb, c->ev_fac[slot], 0);
  }
  if (!c->fp64) {
    KernelScope ks(c, ERX_K_TRINV, sb);
    launch_trinv32(c->Linv32, d, T, sb);
  }
  enqueue_score(c, zsrc, ztype, zstride, ps, T, c->mu_t, c->Linv, c->Linv32, delta, dn, mask,
                det, sb);
  if (slot >= 0) cudaEventRecord(c->ev_fin[slot], sb);
  const erx_status rs = check_cuda(c, cudaGetLastError());
  if (rs == ERX_OK && learned && c->audit_every > 0) {
    const erx_status as = audit_block(c, x, n, stride_elems, delta);
    c->t += n;
    return as;
  }
  c->t += n;
  return rs;
}

// S2 of T lines (x: the raw lines; z: what S2 takes, the lines or their projection)
void enqueue_stats(erx_ctx* c, const void* x, int64_t stride_elems, const void* zsrc, int ztype,
                   int64_t zstride, int ps, int T, cudaStream_t st) {
  const int W = c->W, d = c->d;
  if (c->int_stats && c->tc_stats) {
    KernelScope ks(c, ERX_K_STATS_TC, st);
    launch_stats_tc((const uint16_t*)x, stride_elems, W, d, (1u << c->cfg.in_bits) - 1u, T,
                    c->n_sm, c->S1i, c->S2i, c->err, c->t, st);
  } else if (c->int_stats) {
    KernelScope ks(c, ERX_K_STATS_INT, st);
    launch_stats_int((const uint16_t*)x, stride_elems, W, d, (1u << c->cfg.in_bits) - 1u, T,
                     c->S1i, c->S2i, c->err, c->t, st);
  } else {
    {
      KernelScope ks(c, ERX_K_MEAN, st);
      launch_mean(ztype, zsrc, zstride, ps, W, d, T, !c->fp64, c->mu_hat, c->shift, st);
    }
    // TF32 / BF16 forms: S2 on the tensor cores.  The 3xTF32 form keeps the FP32
    // SIMT scatter: its scatter on the tensor cores measured 3.5e-6 (relative
    // to sqrt(K_aa K_bb)) against 1e-7 for FP32, from accumulating ~200 MMA
    // steps per line in tensor memory, which puts its scores 10x off FP32's.
    const int fmt = tc_format(c->cfg.form);
    if ((fmt == 1 || fmt == 2) && ztype == ERX_F32 && !(c->cfg.flags & ERX_FLAG_SIMT_STATS) &&
        syrk_tc_supported(zsrc, zstride, ps, W, d)) {
      KernelScope ks(c, ERX_K_SYRK_TC, st);
      launch_syrk_tc(fmt, (const float*)zsrc, zstride, W, d, T, c->n_sm, c->shift, c->S2f, c->err,
                     c->t, st);
    } else {
      KernelScope ks(c, ERX_K_STATS_FP, st);
      launch_stats_fp(ztype, c->fp64, zsrc, zstride, ps, W, d, T, c->shift, c->S2f, st);
    }
  }
}

// S3 over T lines: per-line statistics to score with (mu_t, K_t) and the state
// advanced.  EMA; IMC; or pooled: IMC over the warm-up lines, EMA afterwards (a
// block that straddles the end of the warm-up is scanned in two parts).
void enqueue_update(erx_ctx* c, int T, cudaStream_t st) {
  const int W = c->W, d = c->d;
  const int64_t P = packed_size(d);
  int k = 0;   // leading lines of the block averaged with equal weight
  if (c->cfg.averaging == ERX_AVG_IMC)
    k = T;
  else if (c->cfg.averaging == ERX_AVG_POOLED && c->t < c->cfg.warmup_lines)
    k = (int)std::min<int64_t>(T, c->cfg.warmup_lines - c->t);
  if (k > 0) {
    KernelScope ks(c, ERX_K_EMA, st);
    launch_imc_scan(c->int_stats, c->S1i, c->S2i, c->mu_hat, c->shift, c->S2f, k, d, W, c->t,
                    c->cfg.order, c->mu_state, c->K_state, c->mu_t, c->K_t, c->imc_mprev,
                    c->ema_scratch, st, (c->int_stats ? (1u << c->cfg.in_bits) - 1u : 0xffffu));
  }
  if (k < T) {
    const int64_t dd = (int64_t)d * d;
    KernelScope ks(c, ERX_K_EMA, st);
    launch_ema_scan(c->int_stats, c->S1i ? c->S1i + k * d : nullptr,
                    c->S2i ? c->S2i + k * dd : nullptr, c->mu_hat ? c->mu_hat + k * d : nullptr,
                    c->shift ? c->shift + k * d : nullptr, c->S2f ? c->S2f + k * dd : nullptr,
                    T - k, d, W, c->cfg.momentum, c->t + k, c->cfg.order, c->mu_state,
                    c->K_state, c->mu_t + k * d, c->K_t + k * P, c->ema_scratch, st,
                    (c->int_stats ? (1u << c->cfg.in_bits) - 1u : 0xffffu));
  }
}

// S5 and S6 of T lines against (mu_t, factor) per line
void enqueue_score(erx_ctx* c, const void* zsrc, int ztype, int64_t zstride, int ps, int T,
                   const double* mu, const double* Lf, const float* Lf32, void* delta, void* dn,
                   uint8_t* mask, uint8_t* det, cudaStream_t st) {
  const int W = c->W, d = c->d;
  if (c->cfg.form == ERX_FORM_FP64E) {
    KernelScope ks(c, ERX_K_SOLVE_DF, st);
    launch_solve_df(ztype, zsrc, zstride, ps, W, d, T, mu, Lf, c->mu2, c->L2, (double*)delta,
                    st);
  } else if (c->fp64) {
    KernelScope ks(c, ERX_K_SOLVE_FP64, st);
    launch_solve_fp64(ztype, zsrc, zstride, ps, W, d, T, mu, Lf, (double*)delta, st);
  } else if (tc_format(c->cfg.form) > 0) {
    KernelScope ks(c, ERX_K_SOLVE_TC, st);
    launch_solve_tc(tc_format(c->cfg.form), ztype, zsrc, zstride, ps, W, d, T, mu, Lf32,
                    (float*)delta, c->err, c->t, st);
  } else {
    KernelScope ks(c, ERX_K_SOLVE_FP32, st);
    launch_solve_fp32(ztype, zsrc, zstride, ps, W, d, T, mu, Lf32, (float*)delta, st);
  }
  {
    KernelScope ks(c, ERX_K_NORMALISE, st);
    launch_normalise(c->fp64, delta, W, T, c->cfg.threshold, c->t, c->cfg.warmup_lines, dn,
                     mask, det, st);
  }
}

// ERX_FLAG_PIPELINE: the factor of the current state (the one the next line is
// scored with in score-then-update order), on stream st
void enqueue_prefactor(erx_ctx* c, cudaStream_t st) {
  const int d = c->d;
  {
    KernelScope ks(c, ERX_K_CHOL, st);
    launch_chol_inv(c->K_state, d, 1, c->cfg.ridge, c->Lf_pre, c->fp64 ? nullptr : c->Lf32_pre,
                    c->err, c->t, st, c->fp64);
  }
  if (!c->fp64) {
    KernelScope ks(c, ERX_K_TRINV, st);
    launch_trinv32(c->Lf32_pre, d, 1, st);
  }
  cudaMemcpyAsync(c->mu_pre, c->mu_state, sizeof(double) * d, cudaMemcpyDeviceToDevice, st);
}

// One line in score-then-update order with the update deferred (ERX_FLAG_PIPELINE).
// On the context's stream: the line is scored against the factor made at the
// end of the previous push, and its delta_N written.  On the second stream,
// concurrently: the line's statistics and the state's update, then (once the
// score has read the old factor) the factor of the new state for the next
// line.  The next push's score waits for that factor; the context's stream
// waits for the statistics (so the line's buffer is free once it passes).
erx_status run_line_pipelined(erx_ctx* c, const void* x, int64_t stride_elems, void* delta,
                              void* dn, uint8_t* mask, uint8_t* det) {
  const int W = c->W, d = c->d, B = c->B;
  cudaStream_t st = c->stream, sd = c->side;
  cudaStreamWaitEvent(st, c->ev_ready, 0);
  const void* zsrc = x;
  int ztype = c->cfg.in_dtype;
  int64_t zstride = stride_elems;
  int ps = B;
  if (!c->w_host.empty()) {
    KernelScope ks(c, ERX_K_PROJECT, st);
    launch_project(c->cfg.in_dtype, x, stride_elems, B, W, d, 1, c->colptr, c->rows, c->vals,
                   c->fp64, c->Z, st);
    zsrc = c->Z;
    ztype = c->fp64 ? ERX_F64 : ERX_F32;
    zstride = (int64_t)W * d;
    ps = d;
  }
  cudaEventRecord(c->ev_start, st);
  enqueue_score(c, zsrc, ztype, zstride, ps, 1, c->mu_pre, c->Lf_pre, c->Lf32_pre, delta, dn,
                mask, det, st);
  cudaStreamWaitEvent(sd, c->ev_start, 0);
  enqueue_stats(c, x, stride_elems, zsrc, ztype, zstride, ps, 1, sd);
  cudaEventRecord(c->ev_stats, sd);
  enqueue_update(c, 1, sd);
  cudaStreamWaitEvent(st, c->ev_stats, 0);
  cudaEventRecord(c->ev_scored, st);
  cudaStreamWaitEvent(sd, c->ev_scored, 0);
  c->t += 1;
  enqueue_prefactor(c, sd);
  cudaEventRecord(c->ev_ready, sd);
  return check_cuda(c, cudaGetLastError());
}

// ERX_FLAG_PIPELINE, around pushes that take the ordinary path: first the
// deferred update of the last pipelined line must be done (join), afterwards
// the factor of the new state is made for the next single-line push (refresh).
void pipeline_join(erx_ctx* c) {
  if (c->pipeline) cudaStreamWaitEvent(c->stream, c->ev_ready, 0);
}

erx_status pipeline_refresh(erx_ctx* c) {
  if (!c->pipeline) return ERX_OK;
  c->have_pre = false;
  if (c->t == 0) return ERX_OK;
  enqueue_prefactor(c, c->stream);
  cudaEventRecord(c->ev_ready, c->stream);
  const erx_status s = check_cuda(c, cudaGetLastError());
  c->have_pre = s == ERX_OK;
  return s;
}

// every stream of the context idle
cudaError_t sync_all(erx_ctx* c) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess && c->side) e = cudaStreamSynchronize(c->side);
  if (e == cudaSuccess && c->sB) e = cudaStreamSynchronize(c->sB);
  return e;
}

double spearman(const double* a, const double* b, int n) {
  auto ranks = [n](const double* v) {
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [v](int x, int y) { return v[x] < v[y]; });
    std::vector<double> r(n);
    for (int i = 0; i < n;) {          // mid-ranks for ties
      int j = i;
      while (j + 1 < n && v[idx[j + 1]] == v[idx[i]]) ++j;
      for (int q = i; q <= j; ++q) r[idx[q]] = 0.5 * (i + j);
      i = j + 1;
    }
    return r;
  };
  const std::vector<double> ra = ranks(a), rb = ranks(b);
  double ma = 0, mb = 0;
  for (int i = 0; i < n; ++i) ma += ra[i], mb += rb[i];
  ma /= n, mb /= n;
  double sab = 0, saa = 0, sbb = 0;
  for (int i = 0; i < n; ++i) {
    sab += (ra[i] - ma) * (rb[i] - mb);
    saa += (ra[i] - ma) * (ra[i] - ma);
    sbb += (rb[i] - mb) * (rb[i] - mb);
  }
  return (saa > 0 && sbb > 0) ? sab / std::sqrt(saa * sbb) : 1.0;
}

// Score every audit_every-th line of the block with the full-band context and
// compare the two rankings of that line's pixels.
erx_status audit_block(erx_ctx* c, const void* x, int64_t n, int64_t stride_elems, void* delta) {
  const int64_t N = c->audit_every;
  const int64_t j0 = (N - (c->t % N)) % N;
  if (j0 >= n) return ERX_OK;
  const int64_t m = (n - 1 - j0) / N + 1;
  const int W = c->W;
  const size_t es = elem_size(c->cfg.in_dtype);
  const size_t ss = c->fp64 ? 8 : 4;
  const char* xa = (const char*)x + j0 * stride_elems * (int64_t)es;
  erx_status s = erx_push_lines(c->audit, xa, m, N * stride_elems * (int64_t)es, c->audit_delta,
                                nullptr, nullptr, nullptr);
  if (s != ERX_OK) return s;
  c->h_learned.resize((size_t)m * W * ss);
  c->h_full.resize((size_t)m * W * ss);
  if (cudaStreamSynchronize(c->audit->stream) != cudaSuccess ||
      cudaMemcpy2DAsync(c->h_learned.data(), W * ss, (const char*)delta + j0 * W * ss, N * W * ss,
                        W * ss, (size_t)m, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->h_full.data(), c->audit_delta, (size_t)m * W * ss,
                      cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return check_cuda(c, cudaGetLastError());
  std::vector<double> a(W), b(W);
  for (int64_t j = 0; j < m; ++j) {
    for (int i = 0; i < W; ++i) {
      const size_t o = (size_t)j * W + i;
      a[i] = ss == 8 ? ((const double*)c->h_learned.data())[o] : ((const float*)c->h_learned.data())[o];
      b[i] = ss == 8 ? ((const double*)c->h_full.data())[o] : ((const float*)c->h_full.data())[o];
    }
    const double rc = spearman(a.data(), b.data(), W);
    c->last_corr = rc;
    c->min_corr = std::isnan(c->min_corr) ? rc : std::min(c->min_corr, rc);
    c->audits += 1;
    if (rc < c->min_corr_thr && !c->fallback) {
      c->fallback = true;
      c->audit->cfg.momentum = c->cfg.momentum;
      c->audit->t = c->t + n;       // next line the fallback scores is global line t + n
    }
  }
  return ERX_OK;
}

}  // namespace

extern "C" {

void erx_config_default(erx_config* cfg, int32_t bands, int32_t width) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->bands = bands;
  cfg->width = width;
  cfg->momentum = 0.1;
  cfg->proj = ERX_PROJ_NONE;
  cfg->proj_dim = 5;
  cfg->seed = 0;
  cfg->ridge = 1e-5;
  cfg->warmup_lines = 99;
  cfg->order = ERX_UPDATE_THEN_SCORE;
  cfg->averaging = ERX_AVG_EMA;
  cfg->in_dtype = ERX_F32;
  cfg->in_bits = 16;
  cfg->form = ERX_FORM_FP64;
  cfg->threshold = 3.0;
  cfg->block_lines = 0;
  cfg->flags = 0;
  cfg->srp_weights = nullptr;
}

erx_status erx_srp_weights(int32_t bands, int32_t dim, uint64_t seed, double* w) {
  if (bands < 1 || dim < 1 || !w) return ERX_EINVAL;
  const double s = std::sqrt((double)bands);
  const double p_half = 1.0 / (2.0 * s), p_nz = 1.0 / s;
  const double mag = std::sqrt(s) / std::sqrt((double)dim);
  for (int64_t i = 0; i < bands; ++i)
    for (int64_t j = 0; j < dim; ++j) {
      const uint64_t z = splitmix64_at(seed, (uint64_t)(i * dim + j));
      const double u = (double)(z >> 11) * 0x1.0p-53;
      w[i * dim + j] = u < p_half ? mag : (u < p_nz ? -mag : 0.0);
    }
  return ERX_OK;
}

erx_status erx_create(const erx_config* cfg, void* cuda_stream, erx_ctx** out) {
  if (!out) return ERX_EINVAL;
  *out = nullptr;
  erx_status s = validate(cfg);
  if (s != ERX_OK) return s;
  erx_ctx* c = new (std::nothrow) erx_ctx();
  if (!c) return ERX_ENOMEM;
  c->cfg = *cfg;
  c->cfg.srp_weights = nullptr;
  c->B = cfg->bands;
  c->W = cfg->width;
  c->d = cfg->proj != ERX_PROJ_NONE ? cfg->proj_dim : cfg->bands;
  c->stream = (cudaStream_t)cuda_stream;
  c->fp64 = cfg->form == ERX_FORM_FP64 || cfg->form == ERX_FORM_FP64E;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return ERX_ECUDA;
  }
  const int B = c->B, W = c->W, d = c->d;
  if (cfg->proj == ERX_PROJ_SRP) {
    c->w_host.resize((size_t)B * d);
    if (cfg->srp_weights)
      std::memcpy(c->w_host.data(), cfg->srp_weights, sizeof(double) * B * d);
    else
      erx_srp_weights(B, d, cfg->seed, c->w_host.data());
  }
  // exact integer statistics: u16 samples, no projection, and p^2 maxv^2 < 2^62
  const double maxv = std::ldexp(1.0, cfg->in_bits) - 1.0;
  c->int_stats = cfg->in_dtype == ERX_U16 && cfg->proj == ERX_PROJ_NONE &&
                 (double)W * maxv < 2.1e9;
  c->tc_stats = c->int_stats && !(cfg->flags & ERX_FLAG_SIMT_STATS) &&
                stats_tc_supported(d, W, cfg->in_bits);
  if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device) !=
      cudaSuccess) {
    cudaGetLastError();
    delete c;
    return ERX_ECUDA;
  }
  // block size: keep the per-block scratch near 256 MiB
  const int64_t P = packed_size(d);
  const bool learned = cfg->proj == ERX_PROJ_LEARNED;
  size_t per_line = (size_t)P * 8 * 2 + (size_t)d * 8 * 4 + (size_t)d * d * 8 +
                    (c->fp64 ? 0 : (size_t)P * 4) +
                    (c->w_host.empty() && !learned ? 0 : (size_t)W * d * 8);
  int T = cfg->block_lines > 0 ? cfg->block_lines
                               : (int)std::max<size_t>(1, (256ull << 20) / per_line);
  T = std::min(T, 4096);
  c->T = T;
  if (configure_factor_kernels() != cudaSuccess || configure_solve_kernels() != cudaSuccess ||
      configure_stats_tc_kernel() != cudaSuccess || configure_solve_tc_kernels() != cudaSuccess ||
      configure_syrk_tc_kernels() != cudaSuccess || configure_solve_df_kernels() != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return ERX_ECUDA;
  }
  s = ERX_OK;
#define ERX_A(p, n) \
  if (s == ERX_OK) s = dalloc(c, &c->p, (size_t)(n))
  ERX_A(mu_state, d);
  ERX_A(K_state, P);
  ERX_A(mu_t, (size_t)T * d);
  ERX_A(K_t, (size_t)T * P);
  ERX_A(Linv, (size_t)T * P);
  if (!c->fp64) ERX_A(Linv32, (size_t)T * P);
  if (c->int_stats) {
    ERX_A(S1i, (size_t)T * d);
    ERX_A(S2i, (size_t)T * d * d);
  } else {
    ERX_A(mu_hat, (size_t)T * d);
    ERX_A(shift, (size_t)T * d);
    ERX_A(S2f, (size_t)T * d * d);
  }
  ERX_A(err, kErrSlots);
  if (ema_scratch_doubles(d, T) > 0) ERX_A(ema_scratch, ema_scratch_doubles(d, T));
  if (cfg->averaging != ERX_AVG_EMA) ERX_A(imc_mprev, imc_work_doubles(d, T));
  if (cfg->form == ERX_FORM_FP64E) {
    ERX_A(L2, (size_t)T * P);
    ERX_A(mu2, (size_t)T * d);
  }
  c->pipeline = (cfg->flags & ERX_FLAG_PIPELINE) != 0;
  if (c->pipeline) {
    ERX_A(mu_pre, d);
    ERX_A(Lf_pre, P);
    if (!c->fp64) ERX_A(Lf32_pre, P);
    if (s == ERX_OK &&
        (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_start, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_stats, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_scored, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_ready, cudaEventDisableTiming) != cudaSuccess))
      s = ERX_ECUDA;
  }
  // block overlap (stream B): second copies of what passes from A to B.  Not in
  // the FP64 form: both halves are bound by the same FP64 pipe there, and the
  // overlap only adds contention.
  c->overlap = !learned && cfg->form != ERX_FORM_FP64;
  c->mu_t_s[0] = c->mu_t;
  c->Linv_s[0] = c->Linv;
  c->Linv32_s[0] = c->Linv32;
  if (c->overlap) {
    if (s == ERX_OK) s = dalloc(c, &c->mu_t_s[1], (size_t)T * d);
    if (s == ERX_OK) s = dalloc(c, &c->Linv_s[1], (size_t)T * P);
    if (s == ERX_OK && !c->fp64) s = dalloc(c, &c->Linv32_s[1], (size_t)T * P);
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (s == ERX_OK &&
        (cudaStreamCreateWithPriority(&c->sA, cudaStreamNonBlocking, greatest) != cudaSuccess ||
         cudaStreamCreateWithPriority(&c->sB, cudaStreamNonBlocking, least) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_joinA, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_fac[0], cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_fac[1], cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_fin[0], cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_fin[1], cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess))
      s = ERX_ECUDA;
  }
#undef ERX_A
  if (s == ERX_OK && learned) {
    float* zp = nullptr;
    s = dalloc(c, &zp, (size_t)T * W * d);
    c->Z = zp;
  }
  if (s == ERX_OK && !c->w_host.empty()) {
    std::vector<int> cp(d + 1, 0), rw;
    std::vector<double> vl;
    for (int j = 0; j < d; ++j) {
      for (int i = 0; i < B; ++i) {
        const double v = c->w_host[(size_t)i * d + j];
        if (v != 0.0) rw.push_back(i), vl.push_back(v);
      }
      cp[j + 1] = (int)rw.size();
    }
    s = dalloc(c, &c->colptr, cp.size());
    if (s == ERX_OK) s = dalloc(c, &c->rows, std::max<size_t>(1, rw.size()));
    if (s == ERX_OK) s = dalloc(c, &c->vals, std::max<size_t>(1, vl.size()));
    void* zp = nullptr;
    if (s == ERX_OK) {
      s = c->fp64 ? dalloc(c, (double**)&zp, (size_t)T * W * d)
                  : dalloc(c, (float**)&zp, (size_t)T * W * d);
      c->Z = zp;
      c->Z_s[0] = zp;
    }
    if (s == ERX_OK && c->overlap) {
      s = c->fp64 ? dalloc(c, (double**)&zp, (size_t)T * W * d)
                  : dalloc(c, (float**)&zp, (size_t)T * W * d);
      c->Z_s[1] = zp;
    }
    if (s == ERX_OK) {
      cudaMemcpy(c->colptr, cp.data(), cp.size() * sizeof(int), cudaMemcpyHostToDevice);
      if (!rw.empty()) {
        cudaMemcpy(c->rows, rw.data(), rw.size() * sizeof(int), cudaMemcpyHostToDevice);
        cudaMemcpy(c->vals, vl.data(), vl.size() * sizeof(double), cudaMemcpyHostToDevice);
      }
    }
  }
  if (s == ERX_OK) {
    if (cudaMemset(c->mu_state, 0, sizeof(double) * d) != cudaSuccess ||
        cudaMemset(c->K_state, 0, sizeof(double) * P) != cudaSuccess ||
        cudaMemset(c->err, 0xff, sizeof(unsigned long long) * kErrSlots) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess)
      s = ERX_ECUDA;
  }
  if (s != ERX_OK) {
    cudaGetLastError();
    free_all(c);
    delete c;
    return s;
  }
  *out = c;
  return ERX_OK;
}

erx_status erx_push_lines(erx_ctx* c, const void* lines, int64_t n, int64_t stride_bytes,
                          void* delta, void* dn, uint8_t* mask, uint8_t* det) {
  if (!c) return ERX_EINVAL;
  if (c->failed) return ERX_ECUDA;
  if (n < 0 || (n > 0 && (!lines || !delta))) return ERX_EINVAL;
  const size_t es = elem_size(c->cfg.in_dtype);
  const int64_t line_elems = (int64_t)c->W * c->B;
  if (stride_bytes == 0) stride_bytes = line_elems * (int64_t)es;
  if (stride_bytes < line_elems * (int64_t)es || stride_bytes % (int64_t)es) return ERX_EINVAL;
  const int64_t stride = stride_bytes / (int64_t)es;
  const size_t ss = c->fp64 ? 8 : 4;
  if (c->pipeline && n == 1 && c->have_pre)
    return run_line_pipelined(c, lines, stride, delta, dn, mask, det);
  pipeline_join(c);
  const bool two = c->overlap && n > c->T;
  cudaStream_t user = c->stream;
  if (two) {
    // the blocks' stream A work runs on the internal stream of the greatest
    // priority, after what the context's stream holds
    cudaEventRecord(c->ev_fork, user);
    cudaStreamWaitEvent(c->sA, c->ev_fork, 0);
    c->stream = c->sA;
  }
  erx_status s = ERX_OK;
  for (int64_t b = 0; b < n && s == ERX_OK; b += c->T) {
    const int64_t m = std::min<int64_t>(c->T, n - b);
    const char* x = (const char*)lines + b * stride_bytes;
    s = run_block(c, x, m, stride, (char*)delta + (size_t)b * c->W * ss,
                  dn ? (char*)dn + (size_t)b * c->W * ss : nullptr,
                  mask ? mask + (size_t)b * c->W : nullptr, det ? det + b : nullptr,
                  two ? (int)((b / c->T) & 1) : -1);
  }
  if (two) {
    // the context's stream waits for both streams' last work; slot 0's buffers
    // are the ones the single-stream path uses
    c->stream = user;
    cudaEventRecord(c->ev_joinA, c->sA);
    cudaStreamWaitEvent(user, c->ev_joinA, 0);
    cudaEventRecord(c->ev_join, c->sB);
    cudaStreamWaitEvent(user, c->ev_join, 0);
    c->mu_t = c->mu_t_s[0];
    c->Linv = c->Linv_s[0];
    c->Linv32 = c->Linv32_s[0];
    c->Z = c->Z_s[0];
    const erx_status js = check_cuda(c, cudaGetLastError());
    if (s == ERX_OK) s = js;
  }
  if (s != ERX_OK) return s;
  return pipeline_refresh(c);
}

erx_status erx_push_lines_host(erx_ctx* c, const void* lines, int64_t n, int64_t stride_bytes,
                               void* delta, void* dn, uint8_t* mask, uint8_t* det) {
  if (!c) return ERX_EINVAL;
  if (c->failed) return ERX_ECUDA;
  if (n < 0 || (n > 0 && (!lines || !delta))) return ERX_EINVAL;
  const size_t es = elem_size(c->cfg.in_dtype);
  const int64_t line_elems = (int64_t)c->W * c->B;
  const size_t line_bytes = (size_t)line_elems * es;
  if (stride_bytes == 0) stride_bytes = (int64_t)line_bytes;
  if (stride_bytes < (int64_t)line_bytes || stride_bytes % (int64_t)es) return ERX_EINVAL;
  const int T = c->T, W = c->W;
  const size_t ss = c->fp64 ? 8 : 4;
  // per line outputs: delta, delta_n (ss each), mask (1); detecting (1) per line
  const size_t out_line = (size_t)W * (2 * ss + 1) + 1;
  if (!c->copy_stream) {
    erx_status s = ERX_OK;
    if (cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
      return check_cuda(c, cudaGetLastError());
    for (int i = 0; i < 2 && s == ERX_OK; ++i) {
      if (cudaMallocHost(&c->h_in[i], (size_t)T * line_bytes) != cudaSuccess) s = ERX_ENOMEM;
      if (s == ERX_OK) s = dalloc(c, (char**)&c->d_in[i], (size_t)T * line_bytes);
      if (s == ERX_OK && (cudaEventCreateWithFlags(&c->ev_in[i], cudaEventDisableTiming) !=
                              cudaSuccess ||
                          cudaEventCreateWithFlags(&c->ev_used[i], cudaEventDisableTiming) !=
                              cudaSuccess))
        s = ERX_ECUDA;
    }
    if (s == ERX_OK && cudaMallocHost(&c->h_out, (size_t)T * out_line) != cudaSuccess)
      s = ERX_ENOMEM;
    if (s == ERX_OK) s = dalloc(c, (char**)&c->d_out, (size_t)T * out_line);
    if (s != ERX_OK) {
      cudaGetLastError();
      return s;
    }
  }
  pipeline_join(c);
  // Input: pinned caller memory is copied directly; pageable memory through h_in.
  cudaPointerAttributes pa{};
  const bool pinned = cudaPointerGetAttributes(&pa, lines) == cudaSuccess &&
                      (pa.type == cudaMemoryTypeHost);
  cudaGetLastError();
  const int64_t nb = (n + T - 1) / T;
  auto stage = [&](int64_t b) -> erx_status {
    const int slot = (int)(b & 1);
    const int64_t m = std::min<int64_t>(T, n - b * T);
    const char* src = (const char*)lines + b * T * stride_bytes;
    // the slot's previous block must have been consumed by the compute stream
    if (cudaStreamWaitEvent(c->copy_stream, c->ev_used[slot], 0) != cudaSuccess)
      return check_cuda(c, cudaGetLastError());
    if (pinned && stride_bytes == (int64_t)line_bytes) {
      if (cudaMemcpyAsync(c->d_in[slot], src, (size_t)m * line_bytes, cudaMemcpyHostToDevice,
                          c->copy_stream) != cudaSuccess)
        return check_cuda(c, cudaGetLastError());
    } else {
      if (cudaEventSynchronize(c->ev_in[slot]) != cudaSuccess)
        return check_cuda(c, cudaGetLastError());
      for (int64_t j = 0; j < m; ++j)
        std::memcpy((char*)c->h_in[slot] + j * line_bytes, src + j * stride_bytes, line_bytes);
      if (cudaMemcpyAsync(c->d_in[slot], c->h_in[slot], (size_t)m * line_bytes,
                          cudaMemcpyHostToDevice, c->copy_stream) != cudaSuccess)
        return check_cuda(c, cudaGetLastError());
    }
    if (cudaEventRecord(c->ev_in[slot], c->copy_stream) != cudaSuccess)
      return check_cuda(c, cudaGetLastError());
    return ERX_OK;
  };
  if (nb > 0) {
    erx_status s = stage(0);
    if (s != ERX_OK) return s;
  }
  for (int64_t b = 0; b < nb; ++b) {
    const int slot = (int)(b & 1);
    const int64_t m = std::min<int64_t>(T, n - b * T);
    if (b + 1 < nb) {
      erx_status s = stage(b + 1);
      if (s != ERX_OK) return s;
    }
    if (cudaStreamWaitEvent(c->stream, c->ev_in[slot], 0) != cudaSuccess)
      return check_cuda(c, cudaGetLastError());
    char* o = (char*)c->d_out;
    void* d_delta = o;
    void* d_dn = o + (size_t)T * W * ss;
    uint8_t* d_mask = (uint8_t*)(o + (size_t)T * W * ss * 2);
    uint8_t* d_det = d_mask + (size_t)T * W;
    erx_status s = run_block(c, c->d_in[slot], m, (int64_t)(line_bytes / es), d_delta,
                             dn ? d_dn : nullptr, mask ? d_mask : nullptr,
                             det ? d_det : nullptr);
    if (s != ERX_OK) return s;
    if (cudaEventRecord(c->ev_used[slot], c->stream) != cudaSuccess)
      return check_cuda(c, cudaGetLastError());
    // results of this block back to the caller
    const size_t off = (size_t)b * T;
    cudaError_t e = cudaMemcpyAsync((char*)delta + off * W * ss, d_delta, (size_t)m * W * ss,
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && dn)
      e = cudaMemcpyAsync((char*)dn + off * W * ss, d_dn, (size_t)m * W * ss,
                          cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && mask)
      e = cudaMemcpyAsync(mask + off * W, d_mask, (size_t)m * W, cudaMemcpyDeviceToHost,
                          c->stream);
    if (e == cudaSuccess && det)
      e = cudaMemcpyAsync(det + off, d_det, (size_t)m, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return check_cuda(c, e);
  }
  erx_status s = pipeline_refresh(c);
  if (s == ERX_OK) s = check_cuda(c, cudaStreamSynchronize(c->copy_stream));
  if (s == ERX_OK) s = check_cuda(c, sync_all(c));
  return s;
}

erx_status erx_sync(erx_ctx* c, int64_t* bad_line) {
  if (bad_line) *bad_line = -1;
  if (!c) return ERX_EINVAL;
  if (c->failed) return ERX_ECUDA;
  unsigned long long e[kErrSlots];
  if (sync_all(c) != cudaSuccess ||
      cudaMemcpy(e, c->err, sizeof(e), cudaMemcpyDeviceToHost) != cudaSuccess)
    return check_cuda(c, cudaGetLastError());
  if (cudaMemset(c->err, 0xff, sizeof(e)) != cudaSuccess) return check_cuda(c, cudaGetLastError());
  if (e[kErrTimeout] != ~0ull) {
    if (bad_line) *bad_line = (int64_t)e[kErrTimeout];
    return ERX_ETIMEOUT;
  }
  if (e[kErrNotPD] != ~0ull) {
    if (bad_line) *bad_line = (int64_t)e[kErrNotPD];
    return ERX_ENOTPD;
  }
  if (e[kErrRange] != ~0ull) {
    if (bad_line) *bad_line = (int64_t)e[kErrRange];
    return ERX_ERANGE;
  }
  return ERX_OK;
}

erx_status erx_reset(erx_ctx* c) {
  if (!c) return ERX_EINVAL;
  if (c->failed) return ERX_ECUDA;
  c->t = 0;
  c->have_pre = false;
  return ERX_OK;
}

erx_status erx_get_state(erx_ctx* c, int64_t* t, double* mu, double* K) {
  if (!c) return ERX_EINVAL;
  if (c->failed) return ERX_ECUDA;
  const int d = c->d;
  const int64_t P = packed_size(d);
  std::vector<double> kp((size_t)P);
  if (sync_all(c) != cudaSuccess) return check_cuda(c, cudaGetLastError());
  if (mu && cudaMemcpy(mu, c->mu_state, sizeof(double) * d, cudaMemcpyDeviceToHost) != cudaSuccess)
    return check_cuda(c, cudaGetLastError());
  if (K) {
    if (cudaMemcpy(kp.data(), c->K_state, sizeof(double) * P, cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return check_cuda(c, cudaGetLastError());
    for (int a = 0; a < d; ++a)
      for (int b = 0; b <= a; ++b) {
        const double v = kp[(size_t)a * (a + 1) / 2 + b];
        K[(size_t)a * d + b] = v;
        K[(size_t)b * d + a] = v;
      }
  }
  if (t) *t = c->t;
  return ERX_OK;
}

erx_status erx_set_state(erx_ctx* c, int64_t t, const double* mu, const double* K) {
  if (!c || t < 0 || (t > 0 && (!mu || !K))) return ERX_EINVAL;
  if (c->failed) return ERX_ECUDA;
  const int d = c->d;
  const int64_t P = packed_size(d);
  if (t > 0) {
    std::vector<double> kp((size_t)P);
    for (int a = 0; a < d; ++a)
      for (int b = 0; b <= a; ++b) kp[(size_t)a * (a + 1) / 2 + b] = K[(size_t)a * d + b];
    if (sync_all(c) != cudaSuccess ||
        cudaMemcpy(c->mu_state, mu, sizeof(double) * d, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->K_state, kp.data(), sizeof(double) * P, cudaMemcpyHostToDevice) !=
            cudaSuccess)
      return check_cuda(c, cudaGetLastError());
  }
  c->t = t;
  c->have_pre = false;   // the next push takes the ordinary path and refactors
  return ERX_OK;
}

int32_t erx_dim(const erx_ctx* c) { return c ? c->d : -1; }

erx_status erx_get_projection(const erx_ctx* c, double* w) {
  if (!c || !w) return ERX_EINVAL;
  const int B = c->B, d = c->d;
  if (c->w_host.empty()) {
    for (int i = 0; i < B; ++i)
      for (int j = 0; j < d; ++j) w[(size_t)i * d + j] = i == j ? 1.0 : 0.0;
  } else {
    std::memcpy(w, c->w_host.data(), sizeof(double) * B * d);
  }
  return ERX_OK;
}

erx_status erx_set_encoder(erx_ctx* c, erx_encoder* enc, int32_t audit_every,
                           double min_rank_corr) {
  if (!c || !enc || audit_every < 0) return ERX_EINVAL;
  if (c->cfg.proj != ERX_PROJ_LEARNED) return ERX_ESTATE;
  if (encoder_k(enc) != c->d || encoder_bands(enc) != c->B) return ERX_EINVAL;
  c->enc = enc;
  c->audit_every = audit_every;
  c->min_corr_thr = min_rank_corr;
  if (audit_every > 0 && !c->audit) {
    erx_config a = c->cfg;
    a.proj = ERX_PROJ_NONE;
    a.block_lines = std::max(1, c->T / audit_every + 1);
    a.momentum = 1.0 - std::pow(1.0 - c->cfg.momentum, (double)audit_every);
    erx_status s = erx_create(&a, c->stream, &c->audit);
    if (s != ERX_OK) return s;
    void* p = nullptr;
    const size_t ss = c->fp64 ? 8 : 4;
    s = dalloc(c, (char**)&p, (size_t)(c->T / audit_every + 1) * c->W * ss);
    if (s != ERX_OK) return s;
    c->audit_delta = p;
  }
  return ERX_OK;
}

erx_status erx_get_drift(erx_ctx* c, double* last_corr, double* min_corr, int64_t* audits,
                         int32_t* fallback) {
  if (!c) return ERX_EINVAL;
  if (last_corr) *last_corr = c->last_corr;
  if (min_corr) *min_corr = c->min_corr;
  if (audits) *audits = c->audits;
  if (fallback) *fallback = c->fallback ? 1 : 0;
  return ERX_OK;
}

erx_status erx_profile_enable(erx_ctx* c, int32_t on) {
  if (!c) return ERX_EINVAL;
  c->profiling = on != 0;
  return ERX_OK;
}

erx_status erx_profile_read(erx_ctx* c, int32_t k, int32_t reset, double* total_ms,
                            int64_t* timed, int64_t* launches) {
  if (!c || k < 0 || k >= ERX_K_COUNT) return ERX_EINVAL;
  if (c->failed) return ERX_ECUDA;
  if (sync_all(c) != cudaSuccess) return check_cuda(c, cudaGetLastError());
  resolve_pending(c);
  if (total_ms) *total_ms = c->total_ms[k];
  if (timed) *timed = c->timed[k];
  if (launches) *launches = c->launches[k];
  if (reset) {
    for (int i = 0; i < ERX_K_COUNT; ++i) c->total_ms[i] = 0.0, c->timed[i] = 0, c->launches[i] = 0;
  }
  return ERX_OK;
}

const char* erx_kernel_name(int32_t k) {
  static const char* names[ERX_K_COUNT] = {"project",    "stats_int",  "mean",
                                           "stats_fp",   "ema_scan",   "chol",
                                           "solve_fp64", "solve_fp32", "normalise",
                                           "stats_tc",   "solve_tc",   "encode",
                                           "trinv32",    "syrk_tc",    "solve_df"};
  return (k >= 0 && k < ERX_K_COUNT) ? names[k] : nullptr;
}

erx_status erx_destroy(erx_ctx* c) {
  if (!c) return ERX_OK;
  sync_all(c);
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
  cudaGetLastError();
  free_all(c);
  delete c;
  return ERX_OK;
}

const char* erx_status_str(erx_status s) {
  switch (s) {
    case ERX_OK: return "ERX_OK";
    case ERX_EINVAL: return "ERX_EINVAL: invalid argument";
    case ERX_ENOMEM: return "ERX_ENOMEM: allocation failed";
    case ERX_ECUDA: return "ERX_ECUDA: CUDA error; context failed";
    case ERX_ENOTPD: return "ERX_ENOTPD: K_t + ridge I not positive definite";
    case ERX_ERANGE: return "ERX_ERANGE: input sample above 2^in_bits - 1";
    case ERX_ESTATE: return "ERX_ESTATE: call not valid in this state";
    case ERX_EUNSUPPORTED: return "ERX_EUNSUPPORTED: beyond this library's limits";
    case ERX_ETIMEOUT: return "ERX_ETIMEOUT: a bounded wait in a kernel gave up";
    case ERX_EIO: return "ERX_EIO: file not readable or writable, or not a checkpoint";
  }
  return "ERX_?: unknown status";
}

}  // extern "C"
