// erx_push_lines_static: the ERX line step with no device allocation at all.
//
// Some callers cannot call cudaMalloc: a real-time pipeline that is forbidden
// to allocate once it is running (allocation can block or fail at any
// moment), a host that handed all device memory to its own pool, or an
// embedding runtime that only lends out device buffers it already owns.  For
// them this entry point runs the same kernels as erx_push_lines, but keeps the
// per-line intermediates in one fixed array compiled into the library
// (g_scratch below) instead of in context-owned allocations, and keeps the
// background state in buffers the caller passes in.
//
// g_scratch is a file-scope __device__ array: every GPU that loads this
// library reserves it until the process exits.  Host code cannot use its name
// as a device address (on the host it names a shadow variable), so on the
// first call on each device, with that device current, we ask the runtime for
// its device address with cudaGetSymbolAddress and pass that pointer to the
// kernels.  That first call also raises the shared-memory limit of the large
// kernels on the device; make it before any stream capture.
//
// All calls in the process share the one array and it keeps whatever the last
// call left there.  The error slots are reset at the start of every call;
// everything else is fully written before it is read.  Two calls whose GPU
// work overlaps (different streams, or different host threads) race on the
// array and corrupt each other's results: serialise them.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/erx.h"
#include "erx_internal.cuh"

using namespace erx;

namespace {

constexpr int kStaticMaxDim = kMaxDim;  // d <= 224
constexpr size_t kAlign = 256;

constexpr size_t round_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Layout of the scratch for one line at the largest d (bytes).
constexpr size_t kVecB = round_up(sizeof(double) * kStaticMaxDim);
constexpr size_t kMatB = round_up(sizeof(double) * kStaticMaxDim * kStaticMaxDim);
constexpr size_t kPackB = round_up(sizeof(double) * kStaticMaxDim * (kStaticMaxDim + 1) / 2);
constexpr size_t kPack32B = round_up(sizeof(float) * kStaticMaxDim * (kStaticMaxDim + 1) / 2);
constexpr size_t kErrB = round_up(sizeof(unsigned long long) * kErrSlots);
constexpr size_t kOffS1 = 0;                       // sum x (u64) | line mean
constexpr size_t kOffShift = kOffS1 + kVecB;       // centring shift
constexpr size_t kOffS2 = kOffShift + kVecB;       // sum x x^T (u64) | centred scatter (double)
constexpr size_t kOffMuT = kOffS2 + kMatB;         // mu the line is scored with
constexpr size_t kOffKT = kOffMuT + kVecB;         // K the line is scored with (packed)
constexpr size_t kOffLinv = kOffKT + kPackB;       // blocked factor (packed)
constexpr size_t kOffLinv32 = kOffLinv + kPackB;   // its float copy, then L^{-1} in FP32
constexpr size_t kOffErr = kOffLinv32 + kPack32B;  // deferred error slots
constexpr size_t kScratchBytes = kOffErr + kErrB;  // about 0.9 MiB

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device, set up on first use.
erx_status scratch_for_current_device(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return ERX_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return ERX_ECUDA;
    }
    if (configure_factor_kernels() != cudaSuccess || configure_solve_kernels() != cudaSuccess) {
      cudaGetLastError();
      return ERX_ECUDA;
    }
    g_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_ptr[dev];
  return ERX_OK;
}

size_t sample_bytes(int dt) { return dt == ERX_U16 ? 2 : dt == ERX_F32 ? 4 : 8; }

}  // namespace

extern "C" erx_status erx_push_lines_static(const erx_config* cfg, void* cuda_stream,
                                            double* mu_dev, double* K_dev, int64_t* t_host,
                                            const void* lines_dev, int64_t n_lines,
                                            int64_t line_stride_bytes, void* delta_dev,
                                            void* delta_norm_dev, uint8_t* mask_dev,
                                            uint8_t* detecting_dev) {
  if (!cfg || !mu_dev || !K_dev || !t_host || *t_host < 0 || n_lines < 0) return ERX_EINVAL;
  if (n_lines > 0 && (!lines_dev || !delta_dev)) return ERX_EINVAL;
  if (cfg->bands < 1 || cfg->width < 2 || !(cfg->momentum > 0.0 && cfg->momentum <= 1.0) ||
      !(cfg->ridge >= 0.0) || !std::isfinite(cfg->ridge) ||
      (cfg->order != ERX_UPDATE_THEN_SCORE && cfg->order != ERX_SCORE_THEN_UPDATE) ||
      cfg->in_dtype < ERX_U16 || cfg->in_dtype > ERX_F64 ||
      (cfg->in_dtype == ERX_U16 && (cfg->in_bits < 1 || cfg->in_bits > 16)) ||
      (cfg->form != ERX_FORM_FP64 && cfg->form != ERX_FORM_FP32) || cfg->warmup_lines < 0 ||
      (cfg->proj != ERX_PROJ_NONE && cfg->proj != ERX_PROJ_SRP))
    return ERX_EINVAL;
  // limits of the fixed scratch: no projection, d = b <= 224, p <= 2^20; EMA averaging
  if (cfg->proj != ERX_PROJ_NONE || cfg->bands > kStaticMaxDim || cfg->width > (1 << 20) ||
      cfg->averaging != ERX_AVG_EMA)
    return ERX_EUNSUPPORTED;
  const size_t es = sample_bytes(cfg->in_dtype);
  const int W = cfg->width, d = cfg->bands;
  const int64_t line_elems = (int64_t)W * d;
  if (line_stride_bytes == 0) line_stride_bytes = line_elems * (int64_t)es;
  if (line_stride_bytes < line_elems * (int64_t)es || line_stride_bytes % (int64_t)es)
    return ERX_EINVAL;
  if (n_lines == 0) return ERX_OK;

  unsigned char* s = nullptr;
  erx_status st_ = scratch_for_current_device(&s);
  if (st_ != ERX_OK) return st_;
  uint64_t* S1i = reinterpret_cast<uint64_t*>(s + kOffS1);
  double* mu_hat = reinterpret_cast<double*>(s + kOffS1);
  double* shift = reinterpret_cast<double*>(s + kOffShift);
  uint64_t* S2i = reinterpret_cast<uint64_t*>(s + kOffS2);
  double* S2f = reinterpret_cast<double*>(s + kOffS2);
  double* mu_t = reinterpret_cast<double*>(s + kOffMuT);
  double* K_t = reinterpret_cast<double*>(s + kOffKT);
  double* Linv = reinterpret_cast<double*>(s + kOffLinv);
  float* Linv32 = reinterpret_cast<float*>(s + kOffLinv32);
  unsigned long long* err = reinterpret_cast<unsigned long long*>(s + kOffErr);

  cudaStream_t st = (cudaStream_t)cuda_stream;
  const bool fp64 = cfg->form == ERX_FORM_FP64;
  const double maxv = std::ldexp(1.0, cfg->in_bits) - 1.0;
  const bool int_stats = cfg->in_dtype == ERX_U16 && (double)W * maxv < 2.1e9;
  const int64_t stride = line_stride_bytes / (int64_t)es;
  const size_t ss = fp64 ? 8 : 4;
  int64_t t = *t_host;

  if (cudaMemsetAsync(err, 0xff, sizeof(unsigned long long) * kErrSlots, st) != cudaSuccess) {
    cudaGetLastError();
    return ERX_ECUDA;
  }
  for (int64_t j = 0; j < n_lines; ++j, ++t) {
    const void* x = (const char*)lines_dev + j * line_stride_bytes;
    void* delta = (char*)delta_dev + (size_t)j * W * ss;
    void* dn = delta_norm_dev ? (char*)delta_norm_dev + (size_t)j * W * ss : nullptr;
    uint8_t* mask = mask_dev ? mask_dev + (size_t)j * W : nullptr;
    uint8_t* det = detecting_dev ? detecting_dev + j : nullptr;
    if (int_stats) {
      launch_stats_int((const uint16_t*)x, stride, W, d, (1u << cfg->in_bits) - 1u, 1, S1i, S2i,
                       err, t, st);
    } else {
      launch_mean(cfg->in_dtype, x, stride, d, W, d, 1, !fp64, mu_hat, shift, st);
      launch_stats_fp(cfg->in_dtype, fp64, x, stride, d, W, d, 1, shift, S2f, st);
    }
    launch_ema_scan(int_stats, S1i, S2i, mu_hat, shift, S2f, 1, d, W, cfg->momentum, t,
                    cfg->order, mu_dev, K_dev, mu_t, K_t, nullptr, st,
                    int_stats ? (1u << cfg->in_bits) - 1u : 0xffffu);
    launch_chol_inv(K_t, d, 1, cfg->ridge, Linv, fp64 ? nullptr : Linv32, err, t, st, fp64);
    if (!fp64) launch_trinv32(Linv32, d, 1, st);
    if (fp64)
      launch_solve_fp64(cfg->in_dtype, x, stride, d, W, d, 1, mu_t, Linv, (double*)delta, st);
    else
      launch_solve_fp32(cfg->in_dtype, x, stride, d, W, d, 1, mu_t, Linv32, (float*)delta, st);
    launch_normalise(fp64, delta, W, 1, cfg->threshold, t, cfg->warmup_lines, dn, mask, det, st);
  }
  unsigned long long e[kErrSlots];
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess ||
      cudaMemcpy(e, err, sizeof(e), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return ERX_ECUDA;
  }
  *t_host = t;
  if (e[kErrNotPD] != ~0ull) return ERX_ENOTPD;
  if (e[kErrRange] != ~0ull) return ERX_ERANGE;
  return ERX_OK;
}
