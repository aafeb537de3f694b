// Batched form: many independent line streams, with their own widths and band
// counts, each advanced by one line per step.
//
// A step is six phase kernels over the whole batch (line means, centred
// scatter, EMA update, FP64 factor, scores, normalisation), each launched once
// for all streams with a work list that maps its CTAs to (stream, tile); the
// per-stream parameters, including the line count, live in a device table, so
// the step is captured once in a CUDA graph and replayed.  The score kernel of
// each band count is chosen by an autotuner that times the candidate kernels
// on the batch itself.  Streams on learned codes share one encoder: their raw
// lines sit in one contiguous buffer and their codes in another, so a single
// encoder forward over all their pixels opens the step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/erx.h"
#include "erx_batch.cuh"
#include "erx_internal.cuh"

using namespace erx;

namespace erx {
int batch_stats_tiles(int d, int W, bool fp64);
int batch_scatter_chunks(int d, int W);
int batch_solve_tiles(int route, int W, int layout);
void launch_batch_solve_simt(const BStream* S, const BItem* items, int n_items, int dmax,
                             cudaStream_t st);
void launch_batch_solve_fp64(int layout, const BStream* S, const BItem* items, int n_items,
                             int dmax, cudaStream_t st);
void launch_batch_solve_tc(int fmt, const BStream* S, const BItem* items, int n_items, int dmax,
                           unsigned long long* err, cudaStream_t st);
}  // namespace erx

namespace {

__global__ void gather_kernel(const float* const* __restrict__ src, const BStream* __restrict__ S) {
  const BStream& s = S[blockIdx.y];
  const float* p = src[blockIdx.y];
  if (!p) return;
  float* dst = s.xin ? s.xin : const_cast<float*>(s.x);
  const int64_t n = (int64_t)s.W * (s.xin ? s.b_in : s.d);
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  if ((((uintptr_t)p | (uintptr_t)dst) & 15) == 0 && (n & 3) == 0) {
    // 16-byte copies where both ends allow them
    const float4* p4 = reinterpret_cast<const float4*>(p);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int64_t i = t0; i < (n >> 2); i += step) d4[i] = __ldg(p4 + i);
  } else {
    for (int64_t i = t0; i < n; i += step) dst[i] = p[i];
  }
}

}  // namespace

// a run of work items for one launch: items [off, off + n) of a list, dmax the
// largest d among their streams
struct Seg {
  int off = 0, n = 0, dmax = 1;
};

struct erx_batch {
  int n = 0;
  int form = ERX_FORM_FP64;
  int dmax = 1;
  cudaStream_t stream = nullptr;
  bool failed = false;
  std::vector<erx_config> cfg;
  std::vector<BStream> host;      // host mirror of the table (pointers, shapes, routes)
  BStream* table = nullptr;       // device table
  std::vector<void*> allocs;
  // Work lists.  The step runs as two chains side by side inside its graph:
  // chain 0, the streams above 128 dimensions (their single-SM factors are the
  // step's long pole), on the batch's stream; chain 1, all others, on a second
  // stream.  Every list is ordered by chain, and each chain's part is a run of
  // segments (one per launch) recorded below.
  BItem* stream_items = nullptr;  // mean and normalise: one item per stream
  Seg seg_stream[2];
  BItem* stats_items = nullptr;
  Seg seg_stats[2];
  BItem* ema_items = nullptr;
  Seg seg_ema[2];
  BItem* solve_items[kRoutes] = {};
  Seg seg_solve[kRoutes][2][3];   // route, chain, FP64 layout (layout 0 for routes 1..4)
  // factor and FP32 inverse: per chain, the look-ahead schedule group, then the
  // column group, each largest d first
  BItem* chol_items = nullptr;
  Seg seg_chol[2][2];             // chain, schedule (0 look-ahead, 1 column)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  unsigned long long* err = nullptr;
  // learned streams: raw lines [sum W][b_in] and codes [sum W][k], stream order
  int n_learned = 0, learned_b = 0, learned_k = 0;
  int64_t learned_pix = 0;
  float* xin = nullptr;
  float* codes = nullptr;
  erx_encoder* enc = nullptr;
  // graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // push staging
  const float** ptr_host[2] = {nullptr, nullptr};
  const float** ptr_dev = nullptr;
  cudaEvent_t ptr_ev[2] = {nullptr, nullptr};
  int ptr_slot = 0;
};

namespace {

template <typename T>
erx_status balloc(erx_batch* b, T** p, size_t n) {
  void* q = nullptr;
  if (cudaMalloc(&q, std::max<size_t>(1, n) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return ERX_ENOMEM;
  }
  b->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return ERX_OK;
}

void bfree(erx_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  for (void* p : b->allocs) cudaFree(p);
  for (int i = 0; i < 2; ++i) {
    if (b->ptr_host[i]) cudaFreeHost(b->ptr_host[i]);
    if (b->ptr_ev[i]) cudaEventDestroy(b->ptr_ev[i]);
  }
  b->allocs.clear();
}

bool route_allowed(int form, int route) {
  switch (form) {
    case ERX_FORM_FP64: return route == 0;
    case ERX_FORM_FP32: return route == 1;
    case ERX_FORM_TF32: return route == 1 || route == 2;
    case ERX_FORM_BF16: return route == 1 || route == 3;
    case ERX_FORM_TF32X3: return route == 1 || route == 4;
  }
  return false;
}

int native_route(int form) {
  return form == ERX_FORM_FP64 ? 0 : form == ERX_FORM_FP32 ? 1 : form == ERX_FORM_TF32 ? 2
         : form == ERX_FORM_BF16 ? 3 : 4;
}

// operand format of a tensor-core route: 2 TF32, 1 BF16, 3 3xTF32
int route_format(int route) {
  return route == 2 ? 2 : route == 3 ? 1 : 3;
}

int least_priority() {
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  return least;
}

// chain of a stream in the step's graph: 0 above 128 dimensions, else 1
int chain_of(const BStream& e) { return e.d > 128 ? 0 : 1; }

// Sort `items` by (chain, sub(stream)) and record the runs in segs[chain][sub]:
// offsets in that order, counts and each run's largest d.  `then` orders items
// within a run.
template <int NS, typename Sub, typename Then>
void order_segments(const erx_batch* b, std::vector<BItem>& items, Seg (&segs)[2][NS], Sub sub,
                    Then then) {
  std::stable_sort(items.begin(), items.end(), [&](const BItem& x, const BItem& y) {
    const BStream &u = b->host[x.s], &v = b->host[y.s];
    if (chain_of(u) != chain_of(v)) return chain_of(u) < chain_of(v);
    if (sub(u) != sub(v)) return sub(u) < sub(v);
    return then(x, y);
  });
  for (int c = 0; c < 2; ++c)
    for (int k = 0; k < NS; ++k) segs[c][k] = Seg{};
  for (const BItem& it : items) {
    const BStream& e = b->host[it.s];
    Seg& g = segs[chain_of(e)][sub(e)];
    g.n += 1;
    g.dmax = std::max(g.dmax, e.d);
  }
  int off = 0;
  for (int c = 0; c < 2; ++c)
    for (int k = 0; k < NS; ++k) segs[c][k].off = off, off += segs[c][k].n;
}

// copy a work list to the device, allocating it on first use with `cap` items
erx_status upload_items(erx_batch* b, BItem** dev, const std::vector<BItem>& items, size_t cap) {
  if (!*dev) {
    erx_status st = balloc(b, dev, std::max(cap, items.size()));
    if (st != ERX_OK) return st;
  }
  if (!items.empty() && cudaMemcpy(*dev, items.data(), items.size() * sizeof(BItem),
                                   cudaMemcpyHostToDevice) != cudaSuccess)
    return ERX_ECUDA;
  return ERX_OK;
}

// (Re)build the score-kernel work lists from the routes (and FP64 layouts) in
// the host table: per route, by chain, then FP64 layout, largest d first.
erx_status build_solve_items(erx_batch* b) {
  for (int r = 0; r < kRoutes; ++r) {
    std::vector<BItem> items;
    for (int s = 0; s < b->n; ++s)
      if (b->host[s].route == r)
        for (int k = 0; k < batch_solve_tiles(r, b->host[s].W, b->host[s].layout); ++k)
          items.push_back({s, k});
    order_segments(
        b, items, b->seg_solve[r], [&](const BStream& e) { return r == 0 ? e.layout : 0; },
        [&](const BItem& x, const BItem& y) { return b->host[x.s].d > b->host[y.s].d; });
    // capacity: every stream's tiles for this route at the finest tiling
    size_t cap = 0;
    for (int s = 0; s < b->n; ++s) cap += (size_t)batch_solve_tiles(r, b->host[s].W, 2);
    erx_status st = upload_items(b, &b->solve_items[r], items, cap);
    if (st != ERX_OK) return st;
  }
  return ERX_OK;
}

// (Re)build the factor work list from the schedules in the host table.
erx_status build_chol_items(erx_batch* b) {
  std::vector<BItem> items;
  for (int i = 0; i < b->n; ++i) items.push_back({i, 0});
  order_segments(
      b, items, b->seg_chol, [](const BStream& e) { return e.fac ? 0 : 1; },
      [&](const BItem& x, const BItem& y) { return b->host[x.s].d > b->host[y.s].d; });
  return upload_items(b, &b->chol_items, items, items.size());
}

// The per-stream, scatter and EMA work lists (fixed for the batch's life).
erx_status build_step_items(erx_batch* b, std::vector<BItem> st_items,
                            std::vector<BItem> ema_items) {
  std::vector<BItem> str;
  for (int i = 0; i < b->n; ++i) str.push_back({i, 0});
  Seg sg[2][1], ss[2][1], se[2][1];
  auto none = [](const BStream&) { return 0; };
  order_segments(b, str, sg, none, [&](const BItem& x, const BItem& y) {
    return b->host[x.s].d > b->host[y.s].d;
  });
  order_segments(b, st_items, ss, none, [&](const BItem& x, const BItem& y) {
    const BStream &u = b->host[x.s], &v = b->host[y.s];
    return (int64_t)u.W * u.d > (int64_t)v.W * v.d;
  });
  order_segments(b, ema_items, se, none, [](const BItem&, const BItem&) { return false; });
  for (int c = 0; c < 2; ++c)
    b->seg_stream[c] = sg[c][0], b->seg_stats[c] = ss[c][0], b->seg_ema[c] = se[c][0];
  erx_status s = upload_items(b, &b->stream_items, str, str.size());
  if (s == ERX_OK) s = upload_items(b, &b->stats_items, st_items, st_items.size());
  if (s == ERX_OK) s = upload_items(b, &b->ema_items, ema_items, ema_items.size());
  return s;
}

// The device table's line counts advance on the device; pull them into the
// host mirror before the mirror is uploaded again.
erx_status refresh_host(erx_batch* b) {
  std::vector<BStream> dev(b->n);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess ||
      cudaMemcpy(dev.data(), b->table, sizeof(BStream) * b->n, cudaMemcpyDeviceToHost) !=
          cudaSuccess)
    return ERX_ECUDA;
  for (int i = 0; i < b->n; ++i) b->host[i].t = dev[i].t;
  return ERX_OK;
}

erx_status upload_table(erx_batch* b) {
  if (cudaMemcpy(b->table, b->host.data(), sizeof(BStream) * b->n, cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return ERX_ECUDA;
  return ERX_OK;
}

// One chain's share of a step: every phase for the chain's streams, in order.
void enqueue_chain(erx_batch* b, int c, cudaStream_t st) {
  const bool fp64 = b->form == ERX_FORM_FP64;
  const Seg& sg = b->seg_stream[c];
  launch_batch_mean(b->table, b->stream_items + sg.off, sg.n, !fp64, st);
  launch_batch_stats(b->table, b->stats_items + b->seg_stats[c].off, b->seg_stats[c].n, fp64, st);
  launch_batch_ema(b->table, b->ema_items + b->seg_ema[c].off, b->seg_ema[c].n, st);
  for (int f = 0; f < 2; ++f) {   // look-ahead group, then column group
    const Seg& g = b->seg_chol[c][f];
    launch_batch_chol(b->table, b->chol_items + g.off, g.n, g.dmax, f == 0, !fp64, b->err, st);
    if (!fp64) launch_batch_trinv32(b->table, b->chol_items + g.off, g.n, g.dmax, st);
  }
  for (int r = 0; r < kRoutes; ++r) {
    for (int l = 0; l < (r == 0 ? 3 : 1); ++l) {
      const Seg& g = b->seg_solve[r][c][l];
      if (!g.n) continue;
      const BItem* it = b->solve_items[r] + g.off;
      if (r == 0) launch_batch_solve_fp64(l, b->table, it, g.n, g.dmax, st);
      else if (r == 1) launch_batch_solve_simt(b->table, it, g.n, g.dmax, st);
      else launch_batch_solve_tc(route_format(r), b->table, it, g.n, g.dmax, b->err, st);
    }
  }
  launch_batch_normalise(b->table, b->stream_items + sg.off, sg.n, fp64, st);
}

void enqueue_step(erx_batch* b, cudaStream_t st) {
  if (b->enc && b->learned_pix > 0)
    encoder_forward_on(b->enc, b->xin, b->learned_pix, b->codes, st);
  // chain 0 (streams above 128 dimensions) on st, chain 1 beside it
  const bool fork = b->seg_stream[0].n > 0 && b->seg_stream[1].n > 0;
  if (fork) {
    cudaEventRecord(b->ev_fork, st);
    cudaStreamWaitEvent(b->side, b->ev_fork, 0);
  }
  enqueue_chain(b, 0, st);
  enqueue_chain(b, 1, fork ? b->side : st);
  if (fork) {
    cudaEventRecord(b->ev_join, b->side);
    cudaStreamWaitEvent(st, b->ev_join, 0);
  }
}

erx_status capture(erx_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec), b->exec = nullptr;
  if (b->graph) cudaGraphDestroy(b->graph), b->graph = nullptr;
  // chain 0 is captured from a stream of the greatest priority, chain 1 from
  // one of the least, and the graph keeps each node's priority: whenever SMs
  // free up, the waiting CTAs of the long chain are placed first
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithPriority(&cs, cudaStreamNonBlocking, greatest) != cudaSuccess)
    return ERX_ECUDA;
  erx_status s = ERX_OK;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    s = ERX_ECUDA;
  } else {
    enqueue_step(b, cs);
    if (cudaStreamEndCapture(cs, &b->graph) != cudaSuccess ||
        cudaGraphInstantiateWithFlags(&b->exec, b->graph,
                                      cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess)
      s = ERX_ECUDA;
  }
  cudaStreamDestroy(cs);
  if (s != ERX_OK) cudaGetLastError();
  return s;
}

}  // namespace

extern "C" {

erx_status erx_batch_create(int32_t n, const erx_config* cfgs, void* cuda_stream,
                            erx_batch** out) {
  if (!out || n < 1 || !cfgs) return ERX_EINVAL;
  *out = nullptr;
  const int form = cfgs[0].form;
  if (form < ERX_FORM_FP64 || form > ERX_FORM_TF32X3) return ERX_EINVAL;
  for (int i = 0; i < n; ++i) {
    const erx_config& c = cfgs[i];
    if (c.bands < 1 || c.width < 2 || !(c.momentum > 0.0 && c.momentum <= 1.0) ||
        !(c.ridge >= 0.0) || !std::isfinite(c.ridge) || c.warmup_lines < 0 ||
        (c.order != ERX_UPDATE_THEN_SCORE && c.order != ERX_SCORE_THEN_UPDATE) ||
        c.form != form)
      return ERX_EINVAL;
    if (c.averaging != ERX_AVG_EMA) return ERX_EUNSUPPORTED;
    if (c.proj == ERX_PROJ_LEARNED) {
      // one encoder for the batch: all learned streams share bands and k
      if (c.proj_dim < 1 || c.proj_dim > kMaxDim || c.bands > (1 << 16)) return ERX_EINVAL;
      for (int j = 0; j < i; ++j)
        if (cfgs[j].proj == ERX_PROJ_LEARNED &&
            (cfgs[j].bands != c.bands || cfgs[j].proj_dim != c.proj_dim))
          return ERX_EINVAL;
    } else if (c.proj != ERX_PROJ_NONE || c.bands > kMaxDim) {
      return ERX_EUNSUPPORTED;
    }
    if (c.in_dtype != ERX_F32 || c.width > (1 << 20)) return ERX_EUNSUPPORTED;
  }
  erx_batch* b = new (std::nothrow) erx_batch();
  if (!b) return ERX_ENOMEM;
  b->n = n;
  b->form = form;
  b->stream = (cudaStream_t)cuda_stream;
  b->cfg.assign(cfgs, cfgs + n);
  b->host.resize(n);
  size_t nx = 0, nd = 0, np = 0, ndd = 0, nw = 0;
  auto dim = [&](int i) {   // ERX dimension of stream i
    return cfgs[i].proj == ERX_PROJ_LEARNED ? cfgs[i].proj_dim : cfgs[i].bands;
  };
  for (int i = 0; i < n; ++i) {
    const int d = dim(i), W = cfgs[i].width;
    b->dmax = std::max(b->dmax, d);
    if (cfgs[i].proj == ERX_PROJ_LEARNED) {
      b->n_learned += 1;
      b->learned_b = cfgs[i].bands;
      b->learned_k = d;
      b->learned_pix += W;
    }
    nx += (size_t)W * d;
    nd += d;
    np += (size_t)packed_size(d);
    ndd += (size_t)d * d * batch_scatter_chunks(d, W);
    nw += W;
  }
  const size_t ss = form == ERX_FORM_FP64 ? 8 : 4;
  erx_status s = ERX_OK;
  float* ax = nullptr;
  double *amu, *amh, *ash, *amt, *aks, *akt, *alf, *as2;
  float* alf32 = nullptr;
  char *adl = nullptr, *adn = nullptr;
  uint8_t *amk = nullptr, *adt = nullptr;
  if (configure_batch_kernels() != cudaSuccess) s = ERX_ECUDA;
#define BA(p, cnt) \
  if (s == ERX_OK) s = balloc(b, &p, cnt)
  BA(ax, nx);
  if (b->n_learned) BA(b->xin, (size_t)b->learned_pix * b->learned_b);
  BA(amu, nd);
  BA(amh, nd);
  BA(ash, nd);
  BA(amt, nd);
  BA(aks, np);
  BA(akt, np);
  BA(alf, np);
  BA(alf32, np);
  BA(as2, ndd);
  BA(adl, nw * ss);
  BA(adn, nw * ss);
  BA(amk, nw);
  BA(adt, (size_t)n);
  BA(b->table, (size_t)n);
  BA(b->err, (size_t)kErrSlots);
  BA(b->ptr_dev, (size_t)n);
#undef BA
  if (s == ERX_OK) {
    // line buffers: the learned streams' codes first, contiguous in stream
    // order (one encoder forward writes them all), then the other streams
    size_t ox = (size_t)b->learned_pix * b->learned_k, oc = 0, oin = 0;
    size_t od = 0, op = 0, odd = 0, ow = 0;
    b->codes = ax;
    std::vector<BItem> st_items, ema_items;
    for (int i = 0; i < n; ++i) {
      const erx_config& c = cfgs[i];
      const int d = dim(i), W = c.width;
      BStream& e = b->host[i];
      if (c.proj == ERX_PROJ_LEARNED) {
        e.x = ax + oc;
        e.xin = b->xin + oin;
        e.b_in = c.bands;
        oc += (size_t)W * d;
        oin += (size_t)W * c.bands;
      } else {
        e.x = ax + ox;
        e.xin = nullptr;
        e.b_in = 0;
        ox += (size_t)W * d;
      }
      e.W = W;
      e.d = d;
      e.route = native_route(form);
      e.layout = d > 128 ? 1 : 0;
      e.fac = d > 128 ? 1 : 0;
      e.order = c.order;
      e.alpha = c.momentum;
      e.ridge = c.ridge;
      e.threshold = c.threshold;
      e.warmup = c.warmup_lines;
      e.t = 0;
      e.mu_state = amu + od;
      e.mu_hat = amh + od;
      e.shift = ash + od;
      e.mu_t = amt + od;
      e.K_state = aks + op;
      e.K_t = akt + op;
      e.Lf = alf + op;
      e.Lf32 = alf32 + op;
      e.S2f = as2 + odd;
      e.nch = batch_scatter_chunks(d, W);
      e.delta = adl + ow * ss;
      e.dn = adn + ow * ss;
      e.mask = amk + ow;
      e.det = adt + i;
      for (int k = 0; k < batch_stats_tiles(d, W, form == ERX_FORM_FP64); ++k)
        st_items.push_back({i, k});
      const int64_t ne = packed_size(d) + d;
      for (int k = 0; k < (int)((ne + 127) / 128); ++k) ema_items.push_back({i, k});
      od += d;
      op += (size_t)packed_size(d);
      odd += (size_t)d * d * e.nch;
      ow += W;
    }
    if (s == ERX_OK) s = build_step_items(b, std::move(st_items), std::move(ema_items));
    if (s == ERX_OK) s = build_chol_items(b);
    if (s == ERX_OK &&
        (cudaStreamCreateWithPriority(&b->side, cudaStreamNonBlocking, least_priority()) !=
             cudaSuccess ||
         cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess))
      s = ERX_ECUDA;
  }
  if (s == ERX_OK) s = build_solve_items(b);
  if (s == ERX_OK) s = upload_table(b);
  for (int i = 0; i < 2 && s == ERX_OK; ++i) {
    if (cudaMallocHost(&b->ptr_host[i], sizeof(float*) * n) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ptr_ev[i], cudaEventDisableTiming) != cudaSuccess)
      s = ERX_ENOMEM;
  }
  if (s == ERX_OK && (cudaMemset(b->err, 0xff, sizeof(unsigned long long) * kErrSlots) !=
                          cudaSuccess ||
                      cudaDeviceSynchronize() != cudaSuccess))
    s = ERX_ECUDA;
  // a batch with learned streams is captured when its encoder is attached
  if (s == ERX_OK && !b->n_learned) s = capture(b);
  if (s != ERX_OK) {
    cudaGetLastError();
    bfree(b);
    delete b;
    return s;
  }
  *out = b;
  return ERX_OK;
}

erx_status erx_batch_set_encoder(erx_batch* b, erx_encoder* enc) {
  if (!b || !enc || !b->n_learned || encoder_bands(enc) != b->learned_b ||
      encoder_k(enc) != b->learned_k)
    return ERX_EINVAL;
  if (b->failed) return ERX_ECUDA;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
    cudaGetLastError();
    b->failed = true;
    return ERX_ECUDA;
  }
  b->enc = enc;
  const erx_status s = capture(b);
  if (s != ERX_OK) b->failed = true;   // no step graph: the batch cannot run
  return s;
}

erx_status erx_batch_buffers(erx_batch* b, int32_t i, float** line_dev, void** delta_dev,
                             void** delta_norm_dev, uint8_t** mask_dev, uint8_t** detecting_dev) {
  if (!b || i < 0 || i >= b->n) return ERX_EINVAL;
  const BStream& e = b->host[i];
  if (line_dev) *line_dev = e.xin ? e.xin : const_cast<float*>(e.x);
  if (delta_dev) *delta_dev = e.delta;
  if (delta_norm_dev) *delta_norm_dev = e.dn;
  if (mask_dev) *mask_dev = e.mask;
  if (detecting_dev) *detecting_dev = e.det;
  return ERX_OK;
}

erx_status erx_batch_push(erx_batch* b, const float* const* lines_dev) {
  if (!b) return ERX_EINVAL;
  if (b->failed) return ERX_ECUDA;
  if (b->n_learned && !b->enc) return ERX_ESTATE;
  if (lines_dev) {
    const int slot = b->ptr_slot;
    b->ptr_slot ^= 1;
    // the pointer array of this slot may still feed a copy two pushes back
    if (cudaEventSynchronize(b->ptr_ev[slot]) != cudaSuccess) {
      b->failed = true;
      return ERX_ECUDA;
    }
    std::memcpy(b->ptr_host[slot], lines_dev, sizeof(float*) * b->n);
    int wmax = 1;
    for (int i = 0; i < b->n; ++i) {
      const BStream& h = b->host[i];
      wmax = std::max<int64_t>(wmax, ((int64_t)h.W * (h.xin ? h.b_in : h.d) + 255) / 256);
    }
    if (cudaMemcpyAsync(b->ptr_dev, b->ptr_host[slot], sizeof(float*) * b->n,
                        cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaEventRecord(b->ptr_ev[slot], b->stream) != cudaSuccess) {
      b->failed = true;
      return ERX_ECUDA;
    }
    dim3 grid((unsigned)std::min(wmax, 64), (unsigned)b->n);
    gather_kernel<<<grid, 256, 0, b->stream>>>(b->ptr_dev, b->table);
  }
  if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) {
    cudaGetLastError();
    b->failed = true;
    return ERX_ECUDA;
  }
  return ERX_OK;
}

erx_status erx_batch_sync(erx_batch* b, int64_t* bad_stream) {
  if (bad_stream) *bad_stream = -1;
  if (!b) return ERX_EINVAL;
  if (b->failed) return ERX_ECUDA;
  unsigned long long e[kErrSlots];
  if (cudaStreamSynchronize(b->stream) != cudaSuccess ||
      cudaMemcpy(e, b->err, sizeof(e), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(b->err, 0xff, sizeof(e)) != cudaSuccess) {
    cudaGetLastError();
    b->failed = true;
    return ERX_ECUDA;
  }
  for (int k : {(int)kErrTimeout, (int)kErrNotPD}) {
    if (e[k] != ~0ull) {
      if (bad_stream) *bad_stream = (int64_t)e[k];
      return k == kErrTimeout ? ERX_ETIMEOUT : ERX_ENOTPD;
    }
  }
  return ERX_OK;
}

erx_status erx_batch_get_state(erx_batch* b, int32_t i, int64_t* t, double* mu, double* K) {
  if (!b || i < 0 || i >= b->n) return ERX_EINVAL;
  if (b->failed) return ERX_ECUDA;
  BStream e;
  const BStream& h = b->host[i];
  const int d = h.d;
  const int64_t P = packed_size(d);
  std::vector<double> kp((size_t)P);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess ||
      cudaMemcpy(&e, b->table + i, sizeof(BStream), cudaMemcpyDeviceToHost) != cudaSuccess ||
      (mu && cudaMemcpy(mu, h.mu_state, sizeof(double) * d, cudaMemcpyDeviceToHost) !=
                 cudaSuccess) ||
      cudaMemcpy(kp.data(), h.K_state, sizeof(double) * P, cudaMemcpyDeviceToHost) !=
          cudaSuccess) {
    cudaGetLastError();
    b->failed = true;
    return ERX_ECUDA;
  }
  if (K)
    for (int a = 0; a < d; ++a)
      for (int c = 0; c <= a; ++c) K[(size_t)a * d + c] = K[(size_t)c * d + a] = kp[(size_t)a * (a + 1) / 2 + c];
  if (t) *t = e.t;
  return ERX_OK;
}

erx_status erx_batch_route(const erx_batch* b, int32_t i, int32_t* route) {
  if (!b || i < 0 || i >= b->n || !route) return ERX_EINVAL;
  *route = b->host[i].route;
  return ERX_OK;
}

erx_status erx_batch_tune(erx_batch* b, int32_t reps, const char* cache_path) {
  if (!b || reps < 1) return ERX_EINVAL;
  if (b->failed) return ERX_ECUDA;
  const bool fp64 = b->form == ERX_FORM_FP64;
  // band counts present and the routes the form allows
  std::map<int, std::vector<int>> classes;
  for (int s = 0; s < b->n; ++s) classes[b->host[s].d].push_back(s);
  std::vector<int> routes;
  for (int r = 0; r < kRoutes; ++r)
    if (route_allowed(b->form, r)) routes.push_back(r);
  char dev_name[256] = "gpu";
  {
    int dev = 0;
    cudaDeviceProp p{};
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&p, dev) == cudaSuccess)
      std::snprintf(dev_name, sizeof dev_name, "%s", p.name);
    cudaGetLastError();
  }
  std::string cache;
  if (cache_path) {
    if (FILE* f = std::fopen(cache_path, "r")) {
      char buf[4096];
      size_t k;
      while ((k = std::fread(buf, 1, sizeof buf, f)) > 0) cache.append(buf, k);
      std::fclose(f);
    }
  }
  // keys: device, form, band count, width bucket and what was chosen
  auto key_of = [&](int d, int wbucket, const char* what) {
    char k[352];
    std::snprintf(k, sizeof k, "\"%s|form%d|d%d|w%d%s\"", dev_name, b->form, d, wbucket, what);
    return std::string(k);
  };
  auto cached = [&](const std::string& key) {
    const size_t pos = cache.find(key + ":");
    return pos == std::string::npos ? -1 : std::atoi(cache.c_str() + pos + key.size() + 1);
  };
  // The candidates rerun the last step's factor and score kernels, which read
  // only per-step inputs (K_t, mu_t, the line) and rewrite per-step outputs: the
  // state does not move.  A step must therefore have run once.
  bool need_run = true;
  {
    BStream e;
    if (cudaStreamSynchronize(b->stream) == cudaSuccess &&
        cudaMemcpy(&e, b->table, sizeof(BStream), cudaMemcpyDeviceToHost) == cudaSuccess)
      need_run = (e.t == 0);
    cudaGetLastError();
  }
  if (need_run) return ERX_ESTATE;
  if (refresh_host(b) != ERX_OK) {
    b->failed = true;
    return ERX_ECUDA;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return ERX_ECUDA;
  // time `launch` (reps runs after one warm-up pass) on a scratch copy of `items`
  BItem* dit = nullptr;
  size_t dit_cap = 0;
  auto timed = [&](const std::vector<BItem>& items, auto&& launch) -> float {
    if (items.size() > dit_cap) {
      if (dit) cudaFree(dit);
      dit = nullptr;
      if (cudaMalloc(&dit, items.size() * sizeof(BItem)) != cudaSuccess) {
        cudaGetLastError();
        dit_cap = 0;
        return 1e30f;
      }
      dit_cap = items.size();
    }
    cudaMemcpy(dit, items.data(), items.size() * sizeof(BItem), cudaMemcpyHostToDevice);
    float ms = 1e30f;
    for (int pass = 0; pass < 2; ++pass) {
      cudaEventRecord(e0, b->stream);
      for (int k = 0; k < reps; ++k) launch(dit, (int)items.size());
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
    }
    return ms;
  };
  std::string new_entries;
  auto remember = [&](const std::string& key, int v) {
    char line[420];
    std::snprintf(line, sizeof line, "%s%s: %d", new_entries.empty() && cache.empty() ? "" : ",\n ",
                  key.c_str(), v);
    new_entries += line;
  };
  for (auto& kv : classes) {
    const int d = kv.first;
    const std::vector<int>& ss = kv.second;
    int wsum = 0;
    for (int s : ss) wsum += b->host[s].W;
    const int wbucket = 1 << (int)std::ceil(std::log2(std::max(1, wsum / (int)ss.size())));
    std::vector<BItem> per_stream;
    for (int s : ss) per_stream.push_back({s, 0});

    // (1) factor schedule: column (256 threads) or look-ahead (512), same bits
    const std::string kf = key_of(d, wbucket, "|factor");
    int fac = cached(kf);
    if (fac != 0 && fac != 1) {
      float best = 1e30f;
      for (int f = 0; f < 2; ++f) {
        const float ms = timed(per_stream, [&](const BItem* it, int n) {
          launch_batch_chol(b->table, it, n, d, f == 1, !fp64, b->err, b->stream);
        });
        if (ms < best) best = ms, fac = f;
      }
      remember(kf, fac);
    }
    // the FP32 routes' factor copy is inverted in place by trinv32: redo it
    if (!fp64) {
      timed(per_stream, [&](const BItem*, int) {});   // uploads the list
      launch_batch_trinv32(b->table, dit, (int)per_stream.size(), d, b->stream);
    }
    for (int s : ss) b->host[s].fac = fac;

    // (2) score route (forms that allow two)
    int best_r = b->host[ss[0]].route;
    if (routes.size() > 1) {
      const std::string kr = key_of(d, wbucket, "");
      best_r = cached(kr);
      if (!route_allowed(b->form, best_r)) {
        best_r = -1;
        float best = 1e30f;
        for (int r : routes) {
          std::vector<BItem> it;
          for (int s : ss)
            for (int k = 0; k < batch_solve_tiles(r, b->host[s].W, 0); ++k) it.push_back({s, k});
          // the route's score type must match the table's: routes 1 to 4 all write float
          std::vector<BStream> tmp = b->host;
          for (int s : ss) tmp[s].route = r;
          cudaMemcpy(b->table, tmp.data(), sizeof(BStream) * b->n, cudaMemcpyHostToDevice);
          const float ms = timed(it, [&](const BItem* di, int n) {
            if (r == 1) launch_batch_solve_simt(b->table, di, n, d, b->stream);
            else launch_batch_solve_tc(route_format(r), b->table, di, n, d, b->err, b->stream);
          });
          if (ms < best) best = ms, best_r = r;
        }
        remember(kr, best_r);
      }
    }
    for (int s : ss) b->host[s].route = best_r;

    // (3) FP64 score: threads per pixel and pixels per CTA, same bits
    if (best_r == 0) {
      const std::string kl = key_of(d, wbucket, "|fp64layout");
      int lay = cached(kl);
      if (lay < 0 || lay > 2) {
        float best = 1e30f;
        for (int l = 0; l < 3; ++l) {
          std::vector<BItem> it;
          for (int s : ss)
            for (int k = 0; k < batch_solve_tiles(0, b->host[s].W, l); ++k) it.push_back({s, k});
          const float ms = timed(it, [&](const BItem* di, int n) {
            launch_batch_solve_fp64(l, b->table, di, n, d, b->stream);
          });
          if (ms < best) best = ms, lay = l;
        }
        remember(kl, lay);
      }
      for (int s : ss) b->host[s].layout = lay;
    }
  }
  if (dit) cudaFree(dit);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  erx_status s = upload_table(b);
  if (s == ERX_OK) s = build_solve_items(b);
  if (s == ERX_OK) s = build_chol_items(b);
  if (s == ERX_OK) s = capture(b);
  if (s == ERX_OK && cache_path && !new_entries.empty()) {
    std::string body = cache;
    const size_t close = body.rfind('}');
    if (close == std::string::npos) body = "{" + new_entries + "\n}\n";
    else body = body.substr(0, close) + new_entries + "\n}\n";
    if (FILE* f = std::fopen(cache_path, "w")) {
      std::fwrite(body.data(), 1, body.size(), f);
      std::fclose(f);
    }
  }
  if (cudaGetLastError() != cudaSuccess) s = ERX_ECUDA;
  if (s != ERX_OK) b->failed = true;
  return s;
}

erx_status erx_batch_destroy(erx_batch* b) {
  if (!b) return ERX_OK;
  cudaStreamSynchronize(b->stream);
  cudaGetLastError();
  bfree(b);
  delete b;
  return ERX_OK;
}

}  // extern "C"

namespace erx {
cudaError_t configure_batch_kernels() {
  cudaError_t e = configure_factor_kernels();
  if (e == cudaSuccess) e = configure_solve_kernels();
  if (e == cudaSuccess) e = configure_solve_tc_kernels();
  return e;
}
}  // namespace erx
