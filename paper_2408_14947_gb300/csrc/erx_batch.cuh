// Device-side description of a batch of independent line streams advanced one
// line each per step (the batched form).  One table entry per stream; work
// items map a CTA of a phase kernel to (stream, tile).
#pragma once

#include <cstdint>

namespace erx {

constexpr int kRoutes = 5;   // score kernels a stream can be routed to

struct BStream {
  const float* x;        // the stream's current line, [W][d] float32 (device); codes if learned
  float* xin;            // learned streams: the raw line [W][b_in] the gather writes; else null
  int b_in;
  int W, d;
  int route;             // score kernel: 0 FP64, 1 FP32 SIMT, 2 TF32 MMA, 3 BF16 MMA,
                         // 4 3xTF32 MMA
  int layout;            // route 0: threads per pixel x pixels per CTA, 0 (1, 64),
                         // 1 (2, 64), 2 (16, 8); all give the same bits
  int fac;               // factor schedule: 0 column (256 threads), 1 look-ahead (512)
  int order;
  double alpha, ridge, threshold;
  int64_t warmup;
  int64_t t;             // lines seen; advanced on the device at the end of each step
  double* mu_state;      // d
  double* K_state;       // d(d+1)/2 packed
  double* mu_hat;        // d
  double* shift;         // d
  double* S2f;           // nch x d x d: the scatter's 256-pixel chunk sums
  int nch;               // chunk sums in S2f
  double* mu_t;          // d
  double* K_t;           // d(d+1)/2
  double* Lf;            // d(d+1)/2 blocked factor
  float* Lf32;           // its float copy
  void* delta;           // W scores (double for route 0, float otherwise)
  void* dn;              // W normalised scores (same type)
  uint8_t* mask;         // W
  uint8_t* det;          // 1 flag
};

struct BItem {
  int s;      // stream
  int tile;   // tile index within the stream's work for this phase
};

// Batched phase launchers: each CTA takes items[blockIdx.x].
void launch_batch_mean(const BStream* S, const BItem* items, int n, bool float_shift,
                       cudaStream_t st);
void launch_batch_stats(const BStream* S, const BItem* items, int n_items, bool fp64,
                        cudaStream_t st);
void launch_batch_ema(const BStream* S, const BItem* items, int n_items, cudaStream_t st);
void launch_batch_trinv32(const BStream* S, const BItem* items, int n, int dmax,
                          cudaStream_t st);
// the factor of the streams in items[0 .. n): big = all have d > 128 (look-ahead
// schedule, one CTA per SM), else all d <= 128; dmax = their largest d
void launch_batch_chol(const BStream* S, const BItem* items, int n, int dmax, bool big,
                       bool want32, unsigned long long* err, cudaStream_t st);
void launch_batch_solve(int route, const BStream* S, const BItem* items, int n_items, int dmax,
                        unsigned long long* err, cudaStream_t st);
void launch_batch_normalise(const BStream* S, const BItem* items, int n, bool fp64,
                            cudaStream_t st);
cudaError_t configure_batch_kernels();

}  // namespace erx
