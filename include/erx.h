/*
 * erx.h - C ABI of the GB300 (sm_103a) ERX per-line engine.
 *
 * ERX (Garske et al., "ERX: A fast real-time anomaly detection algorithm for
 * hyperspectral line scanning", Sec. III) scores every pixel of each incoming
 * line of a line-scan cube by its Mahalanobis distance to an exponentially
 * moving background mean and covariance, then normalises the scores per line.
 * One call of erx_push_lines runs, for every line t it is given:
 *
 *   S1 project     Z_t = X_t W  (sparse random projection, Sec. III-B), or Z_t = X_t
 *   S2 line stats  mu_hat_t = mean of the pixels, K_hat_t = 1/(p-1) centred scatter (Sec. III-C)
 *   S3 EMA         mu_t = (1-a) mu_{t-1} + a mu_hat_t, K_t likewise; t = 0 starts from line 0 (Sec. III-C)
 *   S4 factor      L_t L_t^T = K_t + ridge I (Sec. III-D)
 *   S5 score       L_t m_i = z_i - mu_t, delta_i = sqrt(m_i . m_i) (Sec. III-D)
 *   S6 normalise   delta_N,i = (delta_i - mean) / std (population std), mask = delta_N >= tau (Sec. III-E)
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are device pointers owned by the caller; they must
 *    stay valid until the work enqueued on the context's stream has finished.
 *    Pointers named *_host are host pointers.
 *  - All work is enqueued on the CUDA stream given to erx_create and the call
 *    returns after enqueueing (erx_push_lines) unless stated otherwise.
 *  - Errors found on the device (a non-positive or non-finite pivot, an input
 *    value above the declared bit depth) are deferred: they are reported by
 *    erx_sync or by the next call on the context.
 *  - ERX_EINVAL leaves the context unchanged.  After ERX_ECUDA the context is
 *    failed and only erx_destroy may be called.
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - No C++ exception crosses this interface.
 */
#ifndef ERX_H
#define ERX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct erx_ctx erx_ctx;

typedef enum {
  ERX_OK = 0,
  ERX_EINVAL = 1,       /* invalid argument; nothing was done */
  ERX_ENOMEM = 2,       /* device or host allocation failed */
  ERX_ECUDA = 3,        /* a CUDA call failed; the context is failed */
  ERX_ENOTPD = 4,       /* K_t + ridge I was not positive definite at some line */
  ERX_ERANGE = 5,       /* an integer input sample exceeded 2^in_bits - 1 */
  ERX_ESTATE = 6,       /* call not valid in the context's current state */
  ERX_EUNSUPPORTED = 7, /* valid request this library does not implement */
  ERX_ETIMEOUT = 8,     /* a bounded wait inside a kernel gave up; results of the call are invalid */
  ERX_EIO = 9           /* a file could not be read or written, or is not a valid checkpoint */
} erx_status;

/* projection (Sec. III-B): none, sparse random projection, or a trained
 * band encoder (erx_encoder, attached with erx_set_encoder) */
enum { ERX_PROJ_NONE = 0, ERX_PROJ_SRP = 1, ERX_PROJ_LEARNED = 2 };
/* order of update and scoring (Sec. III-C/III-D: the paper scores with mu_t, L_t) */
enum { ERX_UPDATE_THEN_SCORE = 0, ERX_SCORE_THEN_UPDATE = 1 };
/* background averaging: ERX_AVG_EMA, the exponentially moving averages of
 * Sec. III-C (momentum alpha); ERX_AVG_IMC, the equal-weight ablation of
 * Sec. IV-C, a batch version of Welford's update: the state is the mean and the
 * 1/(n-1) covariance of all n pixels seen (momentum unused); ERX_AVG_POOLED,
 * the other reading of the warm-up buffer of Sec. IV-B: the warmup_lines first
 * lines are pooled with equal weight (as IMC) into the estimate the EMAs start
 * from, the EMAs of Sec. III-C afterwards */
enum { ERX_AVG_EMA = 0, ERX_AVG_IMC = 1, ERX_AVG_POOLED = 2 };
/* input sample type, lines laid out [pixel][band] (band-interleaved-by-pixel) */
enum { ERX_U16 = 0, ERX_F32 = 1, ERX_F64 = 2 };
/* flags: ERX_FLAG_SIMT_STATS keeps S2 off the tensor cores: exact integer
 * sums by 32-bit integer multiply-adds for u16 lines (identical results), the
 * FP32 SIMT scatter for floating-point lines in the tensor-core forms.
 * ERX_FLAG_PIPELINE (score-then-update order only; not with a learned
 * projection): a single-line push scores its line against the factor of the
 * state made at the end of the previous push, writes delta / delta_N on the
 * context's stream, and defers the line's statistics, the state update and
 * the next factor to a second stream, so a line's latency is its score and
 * normalisation alone.  Results are identical to score-then-update without
 * the flag.  The line's buffer is free once the context's stream has passed
 * the push; erx_sync, erx_get_state and erx_destroy wait for both streams. */
enum { ERX_FLAG_SIMT_STATS = 1, ERX_FLAG_PIPELINE = 2 };
/* arithmetic form of S5 (and of S2 for floating input); S3 and S4 are FP64 in
 * every form, and u16 input without projection always gets exact integer S2.
 * FP64: FP64 arithmetic.  FP32: FP32 SIMT arithmetic.  TF32 / BF16: tensor-core
 * MMAs with TF32 / BF16 operands and FP32 accumulation.  TF32X3: tensor-core
 * MMAs on split operands v = hi + lo (both TF32), accumulating
 * hi hi' + hi lo' + lo hi' in FP32 (near-FP32 products at three MMAs each).
 * In the tensor-core forms, S2 of floating-point lines runs on the tensor
 * cores too (unless ERX_FLAG_SIMT_STATS is set, or the lines are not 16-byte
 * aligned with p * d a multiple of 4: then FP32 SIMT).  FP64E: as FP64
 * (statistics, state, factor and delta in FP64), but S5 in double-float
 * arithmetic on the FP32 pipe (each value a sum of two floats, about 48
 * significant bits, error-free sums and products), held to the FP64 form's
 * error bar; u16 or f32 lines without projection (ERX_EUNSUPPORTED otherwise). */
enum {
  ERX_FORM_FP64 = 0,
  ERX_FORM_FP32 = 1,
  ERX_FORM_TF32 = 2,
  ERX_FORM_BF16 = 3,
  ERX_FORM_TF32X3 = 4,
  ERX_FORM_FP64E = 5
};

typedef struct {
  int32_t bands;        /* b >= 1 */
  int32_t width;        /* p >= 2 pixels per line (K_hat needs p - 1 > 0) */
  double momentum;      /* alpha in (0, 1]; paper default 0.1 (Sec. III-C) */
  int32_t proj;         /* ERX_PROJ_NONE (d = b) or ERX_PROJ_SRP */
  int32_t proj_dim;     /* d for SRP, 1 <= d <= b; paper default 5 (Sec. III-B) */
  uint64_t seed;        /* seed of the SRP matrix when srp_weights is NULL */
  double ridge;         /* added to the diagonal at factorisation only; 1e-5 (Sec. III-D) */
  int32_t warmup_lines; /* lines flagged not-detecting at the start; 99 (Sec. IV-B) */
  int32_t order;        /* ERX_UPDATE_THEN_SCORE (paper) or ERX_SCORE_THEN_UPDATE */
  int32_t in_dtype;     /* ERX_U16, ERX_F32 or ERX_F64 */
  int32_t in_bits;      /* for ERX_U16: samples are < 2^in_bits (1..16); else ignored */
  int32_t form;         /* ERX_FORM_* */
  double threshold;     /* tau_N for the mask (Sec. III-E) */
  int32_t block_lines;  /* lines processed per internal block; 0 = automatic */
  int32_t flags;        /* ERX_FLAG_* bits */
  const double* srp_weights; /* optional b x d row-major host matrix replacing the drawn SRP */
  int32_t averaging;    /* ERX_AVG_EMA (paper), ERX_AVG_IMC or ERX_AVG_POOLED; the
                         * batch and the no-allocation entry point take
                         * ERX_AVG_EMA only */
} erx_config;

/* Fill *cfg with the paper's defaults for a b-band, p-pixel line:
 * alpha 0.1, no projection, ridge 1e-5, warm-up 99, update-then-score,
 * ERX_F32 input, FP64 form, threshold 3.0, SRP d = 5 when proj is set. */
void erx_config_default(erx_config* cfg, int32_t bands, int32_t width);

/* Create a context.  cuda_stream is a cudaStream_t (NULL: the legacy default
 * stream).  Allocates the FP64 state (mu: d, K: d x d) and per-block scratch
 * on the current device.  Limits: d <= 224 (the factor of K_t + ridge I is
 * held in one SM's shared memory), p <= 1 << 20.  Returns ERX_EINVAL on a bad
 * config, ERX_EUNSUPPORTED beyond the limits, ERX_ENOMEM / ERX_ECUDA on
 * allocation failure. */
erx_status erx_create(const erx_config* cfg, void* cuda_stream, erx_ctx** out);

/* Process n_lines consecutive lines, in order, continuing the context's stream
 * of lines.  lines_dev: n_lines lines, line j at lines_dev + j*line_stride_bytes,
 * each p x b samples of in_dtype, row-major [pixel][band]; line_stride_bytes
 * = 0 means p*b*sizeof(sample).  Outputs (device, caller-owned, row-major
 * [line][pixel]):
 *   delta_dev       delta (Sec. III-D); double for ERX_FORM_FP64 and ERX_FORM_FP64E, float
 *                   for the other forms
 *   delta_norm_dev  delta_N (Sec. III-E), same type as delta; may be NULL
 *   mask_dev        uint8 delta_N >= threshold; may be NULL
 *   detecting_dev   uint8 per line, 1 once the warm-up lines have passed; may be NULL
 * Asynchronous on the context's stream. */
erx_status erx_push_lines(erx_ctx* ctx, const void* lines_dev, int64_t n_lines,
                          int64_t line_stride_bytes, void* delta_dev, void* delta_norm_dev,
                          uint8_t* mask_dev, uint8_t* detecting_dev);

/* As erx_push_lines, with every buffer in HOST memory (pageable or pinned).
 * Lines are staged to the device in blocks through library-owned pinned and
 * device buffers, the copies overlapping the compute of the previous block.
 * Synchronous: returns when the results are in the host buffers. */
erx_status erx_push_lines_host(erx_ctx* ctx, const void* lines_host, int64_t n_lines,
                               int64_t line_stride_bytes, void* delta_host,
                               void* delta_norm_host, uint8_t* mask_host,
                               uint8_t* detecting_host);

/* Wait for the context's stream and report deferred device errors
 * (ERX_ETIMEOUT, ERX_ENOTPD, ERX_ERANGE) raised since the last erx_sync.  *bad_line (may be
 * NULL) receives the global index of the first offending line or -1. */
erx_status erx_sync(erx_ctx* ctx, int64_t* bad_line);

/* Forget every line seen: the next line pushed is line 0 again. */
erx_status erx_reset(erx_ctx* ctx);

/* Copy the state out (host pointers): *t = lines seen, mu (d), K (d x d
 * row-major, symmetric).  Synchronises the context's stream. */
erx_status erx_get_state(erx_ctx* ctx, int64_t* t, double* mu_host, double* K_host);

/* Replace the state (host pointers): t lines seen, mu (d), K (d x d, the
 * lower triangle is used).  t = 0 makes the next line initialise the state. */
erx_status erx_set_state(erx_ctx* ctx, int64_t t, const double* mu_host, const double* K_host);

/* Projected dimension d of the context (b without projection). */
int32_t erx_dim(const erx_ctx* ctx);

/* Copy the context's b x d projection matrix (row-major) to w_host. */
erx_status erx_get_projection(const erx_ctx* ctx, double* w_host);

/* Draw the b x d SRP matrix of Sec. III-B (host only, no GPU needed): entry
 * (i, j) is sqrt(sqrt(b)/d) times +1, -1 or 0 with probabilities
 * 1/(2 sqrt b), 1/(2 sqrt b), 1 - 1/sqrt b, decided by output k = i*d + j of
 * SplitMix64 (Steele, Lea and Flood, 2014) seeded with seed: u = (z >> 11)
 * 2^-53, +1 if u < 1/(2s), -1 if u < 1/s. */
erx_status erx_srp_weights(int32_t bands, int32_t dim, uint64_t seed, double* w_host);

/* erx_push_lines without any device allocation (the paper has no
 * counterpart; it serves callers that are not allowed to allocate).
 *
 * A context (erx_create) allocates its state and scratch with cudaMalloc.
 * Some callers cannot do that: a real-time pipeline that must not allocate
 * once running (an allocation can block or fail at any moment), a host whose
 * device memory is all owned by its own pool, or a runtime that only lends
 * out buffers it already holds.  This call needs no context: the caller owns
 * the background state, and the per-line intermediates live in one fixed
 * scratch array compiled into the library (about 0.9 MiB, reserved on every
 * GPU that loads the library until the process exits).  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *
 *  cfg           as for erx_create, within these limits: proj ERX_PROJ_NONE,
 *                bands <= 224 (the fixed scratch is sized for one line at
 *                d = 224), width <= 2^20 and averaging ERX_AVG_EMA, else the
 *                call returns ERX_EUNSUPPORTED; form ERX_FORM_FP64 or
 *                ERX_FORM_FP32, else ERX_EINVAL.  Either way it does nothing.
 *                Both orders and all three input types are supported.
 *                cfg->srp_weights, cfg->block_lines and cfg->flags are ignored.
 *  cuda_stream   cudaStream_t the work runs on (NULL: legacy default stream).
 *  mu_dev        device, d doubles: background mean, read and updated in place.
 *  K_dev         device, d(d+1)/2 doubles: background covariance, packed lower
 *                triangle (row j at offset j(j+1)/2), read and updated in place.
 *  t_host        host, in: lines seen so far (0: the first line initialises the
 *                state, whatever mu_dev / K_dev hold); out: advanced by n_lines.
 *  lines_dev ... detecting_dev   exactly as erx_push_lines.
 *
 * Processes the lines one at a time and returns when the GPU work has
 * finished (synchronises cuda_stream), reporting ERX_ENOTPD / ERX_ERANGE
 * directly.  Those two come after every line has been processed: the state
 * in mu_dev / K_dev and *t_host have advanced by n_lines all the same (the
 * scores of the offending line are NaN or meaningless), so a retry must not
 * push the same lines again.  The first call on each device looks up the scratch array's
 * device address and raises the shared-memory limit of the large kernels on
 * that device; make that first call before any stream capture.  Every call
 * shares the one scratch array: calls whose GPU work overlaps (from several
 * streams or host threads) race on it and corrupt each other's results. */
erx_status erx_push_lines_static(const erx_config* cfg, void* cuda_stream, double* mu_dev,
                                 double* K_dev, int64_t* t_host, const void* lines_dev,
                                 int64_t n_lines, int64_t line_stride_bytes, void* delta_dev,
                                 void* delta_norm_dev, uint8_t* mask_dev, uint8_t* detecting_dev);

/* ---- Learned band encoder --------------------------------------------------
 *
 * A learned counterpart of the sparse random projection (Sec. III-B; the paper
 * names learning-based extensions as future work, Sec. V): an MLP from b bands
 * to k codes, c = W2 relu(W1 xn + b1) + b2 with xn = (x - shift) * scale,
 * trained on the GPU so that ERX on the codes ranks pixels as full-band ERX
 * does.  Weights are kept in FP32 (master) with bf16 copies; the forward and
 * the backward products run on the tensor cores with bf16 operands (the
 * normalised spectra, the hidden activations relu(W1 xn + b1), dL/dc and
 * dL/dh rounded to bf16) and FP32 accumulation, the same forward for training
 * and inference.  Parameters are laid out as one vector
 * [W1 (k1 = hidden x bands, row-major) | b1 | W2 (k x hidden) | b2]. */
typedef struct erx_encoder erx_encoder;

typedef struct {
  double momentum;     /* alpha of the code-space EMA during training (Sec. III-C) */
  double ridge;        /* eps of the code-space factor (Sec. III-D) */
  float lr, beta1, beta2, eps, weight_decay;   /* AdamW */
} erx_train_opts;

/* alpha 0.1, ridge 1e-5, lr 1e-3, betas (0.9, 0.999), eps 1e-8, weight decay 1e-4 */
void erx_train_opts_default(erx_train_opts* o);

/* Create an encoder bands -> hidden -> k (bands <= 256, hidden <= 128: one
 * tensor-core tile of hidden units, 2 <= k <= 32; ERX_EUNSUPPORTED otherwise)
 * on the current device, initial weights He-scaled normal draws from
 * SplitMix64(seed) (Box-Muller), biases 0, input normalisation identity.  All
 * its work runs on cuda_stream. */
erx_status erx_encoder_create(int32_t bands, int32_t hidden, int32_t k, uint64_t seed,
                              void* cuda_stream, erx_encoder** out);

/* Per-band input normalisation xn = (x - shift) * scale (host arrays, bands each). */
erx_status erx_encoder_set_norm(erx_encoder* e, const float* shift_host, const float* scale_host);

/* Copy the parameter vector out (theta_out, may be NULL) and/or replace it
 * (theta_in, may be NULL; also resets the AdamW moments).  Host arrays of
 * erx_encoder_nparams(e) floats.  Synchronises. */
erx_status erx_encoder_params(erx_encoder* e, float* theta_out, const float* theta_in);
int64_t erx_encoder_nparams(const erx_encoder* e);
/* k; *bands and *hidden (may be NULL) receive the other sizes; -1 for NULL. */
int32_t erx_encoder_dims(const erx_encoder* e, int32_t* bands, int32_t* hidden);

/* Forget the code-space EMA used by training (the next line initialises it). */
erx_status erx_encoder_reset_stats(erx_encoder* e);

/* Codes of n_pix pixels: x_dev [n_pix][bands] float -> codes_dev [n_pix][k] float. */
erx_status erx_encoder_forward(erx_encoder* e, const float* x_dev, int64_t n_pix,
                               float* codes_dev);

/* Train on n_lines consecutive lines (lines_dev [n][width][bands] float,
 * targets_dev [n][width] double: full-band ERX delta of those lines), one
 * AdamW step per line in order, continuing the code-space EMA.  loss_host (may
 * be NULL): per-line loss, which synchronises every line. */
erx_status erx_encoder_train(erx_encoder* e, const float* lines_dev, int64_t n_lines,
                             int32_t width, const double* targets_dev, const erx_train_opts* o,
                             float* loss_host);

/* Gradient of one line's loss (host vector of nparams) without updating the
 * weights; advances the code-space EMA like a training step.  Synchronises. */
erx_status erx_encoder_line_grad(erx_encoder* e, const float* line_dev, int32_t width,
                                 const double* target_dev, const erx_train_opts* o,
                                 float* grad_host, float* loss_host);

erx_status erx_encoder_destroy(erx_encoder* e);

/* Checkpoint an encoder to a file and restore it (no counterpart in the
 * paper, whose learning-based extension is future work, Sec. V).  The file is
 * a flat little-endian binary:
 *   char[8] "ERXENC01"; int32 bands, hidden, k, reserved (0); int64 AdamW
 *   step count, code-space line count t;
 *   float shift[bands], scale[bands];   input normalisation
 *   float theta[n], m[n], v[n];         weights and AdamW moments, n = nparams
 *   double mu_e[k], K_e[k(k+1)/2];      code-space EMA state (packed lower)
 * so a loaded encoder computes the same codes bit for bit and resumes
 * training exactly where the saved one stopped.  erx_encoder_save synchronises
 * the encoder's stream; ERX_EIO if the file cannot be written.
 * erx_encoder_load creates a new encoder on the current device, its work on
 * cuda_stream; ERX_EIO if the file cannot be read or is not such a
 * checkpoint (wrong magic, sizes beyond erx_encoder_create's limits, or a
 * length that does not match them). */
erx_status erx_encoder_save(erx_encoder* e, const char* path);
erx_status erx_encoder_load(const char* path, void* cuda_stream, erx_encoder** out);

/* Attach a trained encoder to a context created with proj = ERX_PROJ_LEARNED
 * (proj_dim = the encoder's k, in_dtype ERX_F32, bands = the encoder's bands):
 * its codes replace S1.  The encoder must outlive the context's use of it.
 * audit_every > 0 turns on the drift monitor: every audit_every-th line is
 * also scored by an internal full-band context of the same form (fed only the
 * audited lines, with momentum 1 - (1 - alpha)^audit_every), and the Spearman
 * rank correlation between the two score vectors of that line is recorded; once
 * it falls below min_rank_corr the context falls back to full-band ERX for
 * every later line (the internal context then takes every line with alpha). */
erx_status erx_set_encoder(erx_ctx* ctx, erx_encoder* enc, int32_t audit_every,
                           double min_rank_corr);

/* Drift monitor readout: last and lowest audited rank correlation (NaN before
 * the first audit), number of audits, and whether the fallback is active. */
erx_status erx_get_drift(erx_ctx* ctx, double* last_corr, double* min_corr, int64_t* audits,
                         int32_t* fallback);

/* ---- Batched form: many independent streams, one line each per step ------
 *
 * A batch holds n independent ERX streams, each with its own width, band
 * count and parameters, and advances every one of them by one line per step.
 * A step is six phase kernels launched once for the whole batch (line means,
 * centred scatter, EMA update, FP64 factor, scores, normalisation) with work
 * lists mapping CTAs to (stream, tile); it is captured once in a CUDA graph and
 * replayed.  Limits: float32 input, bands <= 224, one form for the whole batch.
 * Projection: none, or the learned codes of one encoder shared by the batch
 * (streams with proj ERX_PROJ_LEARNED; see erx_batch_set_encoder). */
typedef struct erx_batch erx_batch;

/* Create a batch of n streams from cfgs[0..n-1] (all with the same form and
 * in_dtype ERX_F32; proj ERX_PROJ_NONE, or ERX_PROJ_LEARNED with proj_dim = the
 * encoder's code count k, every learned stream with the same bands and k).
 * Allocates per-stream state, one input line and one output line per stream on
 * the current device; learned streams also get a codes line (width x k). */
erx_status erx_batch_create(int32_t n, const erx_config* cfgs, void* cuda_stream,
                            erx_batch** out);

/* The batch-owned device buffers of stream i: the input line (width x bands
 * float, written by the caller or by erx_batch_push; the raw spectra for a
 * learned stream) and the scores of the
 * last step (delta and delta_N: double for ERX_FORM_FP64, float otherwise;
 * mask: width bytes; detecting: 1 byte).  Any out pointer may be NULL. */
erx_status erx_batch_buffers(erx_batch* b, int32_t i, float** line_dev, void** delta_dev,
                             void** delta_norm_dev, uint8_t** mask_dev, uint8_t** detecting_dev);

/* One step: every stream takes one line.  lines_dev: NULL, or a host array of
 * n device pointers (an entry may be NULL) whose lines are first copied into
 * the streams' input buffers by one gather kernel.  Asynchronous. */
erx_status erx_batch_push(erx_batch* b, const float* const* lines_dev);

/* Attach the band encoder of the batch's learned streams (Sec. V names learned
 * band reduction as future work; the encoder is this library's extension):
 * each step first maps every learned stream's line to its codes with one
 * encoder forward over all of them (tensor cores, BF16 operands, FP32
 * results), and ERX then runs on the codes.  enc must have bands and k equal to
 * the learned streams' bands and proj_dim (ERX_EINVAL otherwise, and when the
 * batch has no learned stream) and must outlive the batch or be replaced.
 * Re-captures the step.  A batch with learned streams returns ERX_ESTATE from
 * erx_batch_push until an encoder is attached. */
erx_status erx_batch_set_encoder(erx_batch* b, erx_encoder* enc);

/* Wait for the batch's stream; report ERX_ENOTPD / ERX_ETIMEOUT raised since
 * the last call, with the index of the first offending stream. */
erx_status erx_batch_sync(erx_batch* b, int64_t* bad_stream);

/* State of stream i (host pointers, as erx_get_state).  Synchronises. */
erx_status erx_batch_get_state(erx_batch* b, int32_t i, int64_t* t, double* mu, double* K);

/* Score kernel chosen for stream i: 0 FP64, 1 FP32 SIMT, 2 TF32 MMA, 3 BF16 MMA,
 * 4 3xTF32 MMA. */
erx_status erx_batch_route(const erx_batch* b, int32_t i, int32_t* route);

/* Autotuner: for every band count in the batch (with its width bucket), time
 * on the batch itself, `reps` runs each with CUDA events, and keep the fastest
 *  - factor schedule: column (256 threads, several CTAs per SM) or look-ahead
 *    (512 threads, one CTA per SM);
 *  - score kernel, where the form allows two (TF32 form: TF32 MMA or FP32
 *    SIMT; BF16: BF16 MMA or FP32 SIMT; TF32X3: 3xTF32 MMA or FP32 SIMT);
 *  - FP64 score layout: 1, 2 or 16 threads per pixel over 64, 64 or 8 pixel
 *    tiles;
 * then re-capture the step.  The schedules and layouts give the same bits;
 * only the score kernel choice changes the arithmetic.  Needs one step pushed
 * before (ERX_ESTATE otherwise); overwrites the last step's scores, not the
 * state.  cache_path (may be NULL): a JSON object of earlier choices keyed by
 * device, form, band count, width bucket and the choice ("|factor",
 * "|fp64layout", none for the score kernel); hits skip the timing and new
 * choices are appended. */
erx_status erx_batch_tune(erx_batch* b, int32_t reps, const char* cache_path);

/* Release the batch.  NULL is a no-op. */
erx_status erx_batch_destroy(erx_batch* b);

/* Kernels of the line step, for erx_profile_read. */
enum {
  ERX_K_PROJECT = 0,    /* S1 sparse projection */
  ERX_K_STATS_INT = 1,  /* S2 exact integer sums (u16, no projection) */
  ERX_K_MEAN = 2,       /* S2 line means */
  ERX_K_STATS_FP = 3,   /* S2 centred scatter, floating point */
  ERX_K_EMA = 4,        /* S3 EMA scan */
  ERX_K_CHOL = 5,       /* S4 Cholesky and inverse */
  ERX_K_SOLVE_FP64 = 6, /* S5 scores, FP64 */
  ERX_K_SOLVE_FP32 = 7, /* S5 scores, FP32 */
  ERX_K_NORMALISE = 8,  /* S6 normalisation */
  ERX_K_STATS_TC = 9,   /* S2 exact integer sums on the tensor cores */
  ERX_K_SOLVE_TC = 10,  /* S5 scores on the tensor cores (TF32 / BF16 / 3xTF32) */
  ERX_K_ENCODE = 11,    /* S1 learned band encoder (codes) */
  ERX_K_TRINV = 12,     /* S4 full inverse of the factor in FP32 (non-FP64 forms) */
  ERX_K_SYRK_TC = 13,   /* S2 centred scatter of floating lines on the tensor cores */
  ERX_K_SOLVE_DF = 14,  /* S5 scores in double-float (FP64E form) */
  ERX_K_COUNT = 15
};

/* Per-kernel timing.  While enabled (on != 0), every kernel the context
 * launches is bracketed by two CUDA events recorded on the context's stream.
 * Launch counts are kept whether or not timing is enabled. */
erx_status erx_profile_enable(erx_ctx* ctx, int32_t on);

/* Totals since the last call with reset != 0: *launches kernel launches of
 * kind `kernel` (ERX_K_*) and, for launches made while timing was enabled,
 * *total_ms their summed device time.  Synchronises the context's stream. */
erx_status erx_profile_read(erx_ctx* ctx, int32_t kernel, int32_t reset, double* total_ms,
                            int64_t* timed_launches, int64_t* launches);

/* Static name of kernel kind `kernel`, or NULL. */
const char* erx_kernel_name(int32_t kernel);

/* Release the context and everything it allocated.  NULL is a no-op. */
erx_status erx_destroy(erx_ctx* ctx);

/* Static string naming a status code. */
const char* erx_status_str(erx_status s);


/* ---- Detection quality (Sec. IV-B), a tooling call outside the per-line step ----
 * Scores a detection map (n scores, device, float or double) against anomaly
 * labels (n bytes, device, nonzero = anomaly):
 *   auc          area under the ROC curve (TPR against FPR over all thresholds),
 *                of the map min-max normalised in FP64, v = (s - min) / (max - min),
 *                and quantised to `bins` levels, q = min(floor(v * bins), bins - 1):
 *                the Mann-Whitney statistic, ties within a level counting one half
 *                (|auc - exact| <= 1 / bins for a continuous map);
 *   auc_tpr_tau  area under TPR against the threshold tau in [0, 1] of the
 *                normalised map (= the anomalies' mean normalised score);
 *   auc_fpr_tau  the same for FPR (= the background's mean normalised score);
 *   auc_td = (auc + auc_tpr_tau) / 2,  auc_bs = (auc - auc_fpr_tau + 1) / 2;
 *   u2           2U, the exact integer statistic behind auc.
 * A non-finite score counts in level 0 (the sums then carry it).
 * Synchronous on cuda_stream; allocates its scratch (cudaMalloc) per call.
 * ERX_EINVAL if n <= 0, bins outside [2, 2^24], score_dtype not ERX_F32 / ERX_F64,
 * or the labels hold no anomaly or no background pixel. */
typedef struct {
  double auc, auc_tpr_tau, auc_fpr_tau, auc_td, auc_bs;
  int64_t positives, negatives;
  uint64_t u2;
} erx_roc;
erx_status erx_roc_metrics(const void* scores_dev, int32_t score_dtype, const uint8_t* labels_dev,
                           int64_t n, int32_t bins, void* cuda_stream, erx_roc* out);

/* ---- Self-test of the bounded device waits ------------------------------
 *
 * Every device-side wait of the library (an mbarrier of an asynchronous copy
 * or of a tensor-core commit) polls at most a fixed number of times; when the
 * limit runs out the kernel records ERX_ETIMEOUT, waits once more (bounded)
 * for its work in flight, releases its tensor memory and returns, so the
 * context stays usable.  This entry point runs that path on purpose without
 * any fault: one thread waits on an mbarrier that nothing arrives at, at most
 * `limit` polls (1 <= limit <= 2^20; each poll returns within the hardware's
 * suspend window), on cuda_stream.  Returns ERX_ETIMEOUT when the wait ran out
 * as designed, ERX_OK if it completed (a defect), ERX_EINVAL for a limit out of
 * range, ERX_ECUDA on a launch error.  Synchronises. */
erx_status erx_selftest_bounded_wait(uint32_t limit, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* ERX_H */
