/*
 * libstda — Radar-STDA on GB300 (sm_103a): C-ABI.
 *
 * Radar-STDA (arXiv 2307.09063) denoises the newest of three consecutive
 * FMCW range-Doppler (RD) maps. This library runs its forward pass (Sec. IV:
 * Eq. "concat_operation", Eqs. "mobile_encoder_stage1/2",
 * "mobile_decoder_stage1/2", "eca_process_equation", the two skip
 * connections of Sec. IV-D), the synthetic RD generator of Sec. III (Eqs.
 * "discrete signal", "IF signal", "column transform", "row transform"), and
 * the SINR metric of Sec. V-B, as CUDA kernels on the GPU.
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are device pointers owned by the caller; they must
 *    stay valid until the work queued on `stream` has finished. Host
 *    pointers are named host_*.
 *  - Work is queued on `stream` (NULL = the legacy default stream) and the
 *    call returns without waiting, except stda_create, stda_destroy,
 *    stda_get_*, stda_set_* and stda_device_status, which synchronise.
 *  - Errors are returned as a status code; nothing aborts. The message of
 *    the last failure of a context is in stda_last_error().
 *  - A context is not thread-safe: calls on one context must not overlap in
 *    host threads.
 *  - Map layout: a window is [3][H][W] float (STDA_FP32) or bfloat16
 *    (the other precisions), frames ordered t, t-1, t-2 (channel order
 *    of Eq. "concat_operation"); H = range bins, W = Doppler bins, both
 *    positive multiples of 8 (the three stride-2 stages halve the map three
 *    times). A batch is [B][3][H][W], the output [B][1][H][W] in the same
 *    element type, values in (0, 1).
 */
#ifndef STDA_H
#define STDA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st; /* cudaStream_t */
struct CUevent_st;  /* cudaEvent_t  */

typedef struct stda_ctx stda_ctx; /* opaque, owned by the library */

typedef enum {
  STDA_OK = 0,
  STDA_ERR_INVALID_ARG = 1, /* null pointer, bad count, bad enum          */
  STDA_ERR_SHAPE = 2,       /* H or W not a positive multiple of 8, B out
                               of [0, max_batch], map larger than created */
  STDA_ERR_OOM = 3,         /* device allocation failed                   */
  STDA_ERR_CUDA = 4,        /* a CUDA runtime call failed                 */
  STDA_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up         */
  STDA_ERR_BUSY = 6,        /* serving: no slot or memory free right now  */
  STDA_ERR_UNSUPPORTED = 7, /* not available for this precision / device  */
  STDA_WARMUP = 8           /* serving: fewer than three frames buffered  */
} stda_status;

/* Arithmetic of the forward pass (accumulation is FP32 in every case):
 *  STDA_FP32          FP32 FMA on the CUDA cores, float I/O.
 *  STDA_BF16          bf16 tensor-core operands (tcgen05 kind::f16), bf16 I/O.
 *  STDA_FP8_E4M3      E4M3 tensor-core operands (kind::f8f6f4) for the dense
 *                     convolutions of blocks 2-6, weights with per-output-
 *                     channel scales; every operand is a two-term E4M3 sum
 *                     (high part + E4M3 of its rounding remainder) and each
 *                     tap issues three MMAs (hi*hi, lo*hi, hi*lo), which keeps
 *                     the error at the bf16 level. Block 1 (8 input channels)
 *                     runs in bf16. bf16 I/O.
 *  STDA_FP8_E4M3_FAST as STDA_FP8_E4M3 with one E4M3 term per operand (one
 *                     MMA per tap); about 16x the bf16 error (3-bit mantissa),
 *                     outside the bf16 tolerance. */
typedef enum {
  STDA_FP32 = 0,
  STDA_BF16 = 1,
  STDA_FP8_E4M3 = 2,
  STDA_FP8_E4M3_FAST = 3
} stda_precision;

typedef struct {
  int H, W;          /* largest map size the context serves (multiples of 8) */
  int max_batch;     /* largest batch of windows per call                    */
  stda_precision prec;
  uint64_t weight_seed;    /* random initialisation of the weights          */
  size_t mem_budget_bytes; /* serving admission limit; 0 = no limit         */
  int frames;              /* maps stacked per window (Sec. IV-A, Eq.
                              "concat_operation"): 3 as in the paper (0
                              also means 3), or 2 / 4 for the fusion
                              variants, which change only the stem's
                              input channels. stda_backward, stda_submit and
                              stda_forward_static need 3 (else
                              STDA_ERR_UNSUPPORTED).                       */
} stda_config;

/* ---------------------------------------------------------------- context */

/* Allocates the context, its folded weights and its activation scratch for
 * max_batch windows of H x W, and initialises the weights from weight_seed
 * (uniform draws of a SplitMix64 hash; see stda_get_params). Uses the
 * current CUDA device. */
stda_status stda_create(const stda_config* cfg, stda_ctx** out);
stda_status stda_destroy(stda_ctx* ctx);

/* 137,915: the learnable parameters in canonical order (stem; per block
 * dw1x1, BN1, dw3x3, BN2, BN3, stage-2 weight, BN, residual weight and bias,
 * ECA kernel; output conv weight and bias). Table "performance_radar_stda"
 * prints 0.14 M. */
size_t stda_num_params(void);
/* 1,360: batch-norm running means and variances (per BN: mean[C], var[C]). */
size_t stda_num_buffers(void);

/* Host only (no GPU needed): the parameters and BN buffers that
 * stda_create draws from `seed`. host_params[137915], host_buffers[1360]. */
stda_status stda_init_params(uint64_t seed, float* host_params,
                             float* host_buffers);

/* The same for a context of `frames` (1..4) stacked maps: the stem weight
 * is W[8][frames][3][3], so the parameter count is 137915 + 72 (frames - 3);
 * every other tensor has the same values as for three maps. */
size_t stda_num_params_frames(int frames);
stda_status stda_init_params_frames(uint64_t seed, int frames, float* host_params,
                                    float* host_buffers);

/* Structural re-parameterisation for deployment (host only, no GPU). The
 * paper's blocks train as multi-branch MobileOne-style units (Sec. IV-B,
 * Eqs. "mobile_encoder_stage1/2", "mobile_decoder_stage1/2": dw 1x1 + BN,
 * dw 3x3 + BN and an identity BN summed before a ReLU; a conv + BN main
 * branch) and collapse at inference into one conv + bias per branch. This
 * writes that inference network, with every BN folded in FP64 and rounded
 * to float once, in PyTorch weight layouts, concatenated in this order:
 *   stem.weight [8][T][3][3], stem.bias [8]      Conv2d(T, 8, 3, padding 1) + ReLU
 *   for each block b = 0..5 (Cin 8,16,32,64,32,16; Cout 16,32,64,32,16,8):
 *     dw.weight [Cin][1][3][3], dw.bias [Cin]    depthwise Conv2d(padding 1,
 *                                                groups Cin) + ReLU (the
 *                                                decoder's stride-1 transposed
 *                                                conv written as a correlation)
 *     main.weight, main.bias [Cout]              encoder: Conv2d [Cout][Cin][3][3],
 *                                                stride 2, padding 1; decoder:
 *                                                ConvTranspose2d [Cin][Cout][4][4],
 *                                                stride 2, padding 1; then ReLU
 *     res.weight, res.bias [Cout]                the same conv shape, no ReLU;
 *                                                y = ReLU(main) + res
 *     eca.weight [1][1][3]                       Conv1d(1, 1, 3, padding 1, no
 *                                                bias) on the channel means,
 *                                                sigmoid, scales y
 *   out.weight [1][8][3][3], out.bias [1]        Conv2d(8, 1, 3, padding 1) + sigmoid
 * with the skips D1 += E2 (input of block 4) and D2 += E1 (input of block 5)
 * after ECA; T = frames stacked maps (1..4; 3 in the paper). host_params /
 * host_buffers as for stda_init_params_frames; host_out holds
 * n = stda_reparam_count(frames) floats. Returns STDA_ERR_INVALID_ARG on a
 * null pointer, frames outside 1..4 or a wrong n. */
size_t stda_reparam_count(int frames);
stda_status stda_reparam_export(const float* host_params, const float* host_buffers, int frames,
                                float* host_out, size_t n);

/* Copies the FP32 parameters / BN buffers to or from host memory (n must
 * equal the count above). stda_set_* refolds BN into the convolutions in
 * FP64 on the host and re-uploads every precision's weights. */
stda_status stda_get_params(stda_ctx* ctx, float* host_dst, size_t n);
stda_status stda_set_params(stda_ctx* ctx, const float* host_src, size_t n);
stda_status stda_get_buffers(stda_ctx* ctx, float* host_dst, size_t n);
stda_status stda_set_buffers(stda_ctx* ctx, const float* host_src, size_t n);

/* ---------------------------------------------------------------- forward */

/* Denoises B windows: d_in [B][frames][H][W] -> d_out [B][1][H][W] (Sec. IV-A,
 * Eqs. "encoder_stda", "decoder_stda"). H, W may be smaller than the
 * context's, but B*H*W may not exceed max_batch*H_ctx*W_ctx. B == 0 is a
 * no-op. d_in and d_out must be 16-byte aligned (STDA_ERR_INVALID_ARG
 * otherwise). */
stda_status stda_forward(stda_ctx* ctx, const void* d_in, void* d_out, int B,
                         int H, int W, struct CUstream_st* stream);

/* The same forward pass on host buffers, end to end: h_in [B][frames][H][W]
 * and h_out [B][1][H][W] in host memory, element type as for stda_forward
 * (page-locked memory lets the copies overlap kernels; pageable memory works
 * but its copies do not overlap). The input is copied to one of two device
 * staging buffers on an internal stream that waits only for the forward that
 * last read that buffer (two calls back), so a call's input copy overlaps the
 * previous call's kernels; the forward runs on `stream` once its input has
 * landed. Where h_out is page-locked and mapped into the device's address
 * space (cudaHostAlloc / cudaHostRegister memory with the context's device
 * current, e.g. a pinned torch tensor) and 16-byte aligned, the forward's
 * last kernel stores the result straight into it (NVLink-C2C on
 * Grace-Blackwell, no copy back); otherwise the output is copied back from
 * a staging buffer on a second internal stream, which `stream` then waits
 * for. So: h_in must hold its final contents when the call is made (it is
 * not ordered after work already queued on `stream`); h_out is complete
 * once `stream` has been synchronised; work queued on `stream` after the
 * call follows the output. Calls on one context must
 * use one stream. The first call allocates the staging buffers (two pairs of
 * max_batch windows of the context's H x W). Shapes as for stda_forward. */
stda_status stda_forward_host(stda_ctx* ctx, const void* h_in, void* h_out, int B,
                              int H, int W, struct CUstream_st* stream);

/* Training step (adjoint of the forward pass): runs the network's forward
 * pass with a tape and its exact adjoint, in FP32 on the CUDA cores, with
 * batch normalisation in inference form (frozen running statistics;
 * gamma and beta receive gradients; stda_backward_bn below selects training
 * mode). Weight and BN gradients are reduced
 * in FP32 over slices of the batch's pixels and across slices in FP64 (in a
 * fixed order); the loss is an FP64 sum.
 *   d_in      [B][3][H][W] in the context's element type
 *   d_target  [B][1][H][W] clean maps in the context's element type; the
 *             loss is their mean squared error (Sec. V-C trains the
 *             denoiser against interference-free maps), or NULL
 *   d_gout    [B][1][H][W] float dL/dz, used when d_target is NULL
 *   d_gparams [137915] float dL/dtheta in canonical order (required)
 *   d_loss    double, the loss (target mode), or NULL
 *   d_gin     [B][3][H][W] float dL/dx, or NULL
 *   d_out     [B][1][H][W] float forward output of the training graph, or NULL
 * The first call allocates the context's training workspace (for
 * max_batch windows of the context's H x W). */
stda_status stda_backward(stda_ctx* ctx, const void* d_in, const void* d_target,
                          const float* d_gout, float* d_gparams, double* d_loss,
                          float* d_gin, float* d_out, int B, int H, int W,
                          struct CUstream_st* stream);

/* BN modes of the training step. */
typedef enum {
  STDA_BN_RUNNING = 0, /* inference form: the running statistics (frozen) */
  STDA_BN_BATCH = 1    /* training mode: each BN normalises with the mean and
                          biased variance of its input over the whole batch
                          (all B windows and pixels of a channel), and the
                          adjoint carries the dependence of those statistics
                          on the input:
                          dx = gamma/sigma (dy - [sum dy + xhat sum dy xhat]/N) */
} stda_bn_mode;

/* stda_backward with a BN mode. d_bn_stats (optional, [1360] float, device)
 * receives the mean and variance each BN normalised with, in the layout of
 * the BN buffers (per BN: mean[C] then var[C]; stem, then per block BN1,
 * BN2, BN3, BN), from which a caller updates the running statistics (e.g.
 * running = (1 - m) running + m batch). The statistics are two-pass
 * (mean, then mean squared deviation), FP32 over slices of the batch's
 * pixels and FP64 across slices. STDA_ERR_INVALID_ARG on an unknown mode. */
stda_status stda_backward_bn(stda_ctx* ctx, const void* d_in, const void* d_target,
                             const float* d_gout, float* d_gparams, double* d_loss,
                             float* d_gin, float* d_out, int B, int H, int W,
                             stda_bn_mode bn_mode, float* d_bn_stats,
                             struct CUstream_st* stream);

/* ---------------------------------------------------------------- serving */

/* Continuous batching of radar streams (the online pattern of Sec. IV-B:
 * each new frame t is denoised with frames t-1 and t-2 of the same radar).
 * Frames and outputs are bfloat16 [H][W] device buffers, 16-byte aligned;
 * serving runs the tensor-core forward of the context's precision (bf16 for
 * an STDA_FP32 context). Every radar keeps its last three frames in a
 * device ring owned by the context.
 *
 * stda_submit copies d_frame into radar `radar_id`'s ring on `stream` and
 * returns STDA_WARMUP while the radar has fewer than three frames. From the
 * third frame on, the window (t, t-1, t-2) joins the pending batch of its
 * map size; the denoised frame t is written to d_out and `done` (if not
 * NULL) is recorded once it is there. A new radar is refused with
 * STDA_ERR_BUSY when its ring (3 H W bf16) plus, for a map size not seen
 * before, that size's batch buffers would exceed the context's
 * mem_budget_bytes (0 = no limit); H and W must stay the same for a radar
 * (else STDA_ERR_SHAPE). A radar whose previous window is still pending
 * flushes that window's batch first. Batches of 64 windows launch by
 * themselves. Use one stream for all serving calls of a context. */
stda_status stda_submit(stda_ctx* ctx, int radar_id, int H, int W,
                        const void* d_frame, void* d_out,
                        struct CUevent_st* done, struct CUstream_st* stream);
/* Launches every pending window: per map size one batch (its own stream,
 * so sizes overlap), ordered after the frames copied on `stream`. */
stda_status stda_flush(stda_ctx* ctx, struct CUstream_st* stream);
/* Releases radar_id's ring (after its pending window has run); blocks until
 * its size's batches in flight have finished. */
stda_status stda_serve_close(stda_ctx* ctx, int radar_id,
                             struct CUstream_st* stream);
/* Device bytes held by serving (rings and per-size batch buffers), and the
 * number of open radars. */
size_t stda_serve_bytes(stda_ctx* ctx);
int stda_serve_radars(stda_ctx* ctx);

/* Device-side error word of the context (STDA_OK or STDA_ERR_TIMEOUT):
 * synchronises the context's last stream and every serving stream, returns
 * the word and clears it, so a later call reports only errors raised after
 * this one. A kernel that gives up on a bounded wait finishes the work it
 * has queued on the tensor cores, frees its tensor memory and returns, so
 * the context stays usable after a timeout. */
stda_status stda_device_status(stda_ctx* ctx);
/* Bound of the tensor-core kernels' waits for their tiles' MMAs, in polls
 * of an mbarrier (each poll may itself suspend briefly); default 2^22, far
 * above any tile's latency. 0 makes every such wait give up at once, so the
 * next forward reports STDA_ERR_TIMEOUT through stda_device_status: a hook
 * for tests of the timeout path (its output is then undefined). The waits
 * for MMAs already issued, before tensor memory is freed, keep the default
 * bound. */
stda_status stda_set_wait_limit(stda_ctx* ctx, uint32_t polls);
const char* stda_last_error(stda_ctx* ctx);
const char* stda_status_string(stda_status s);

/* ------------------------------------------------------- no-allocation path */

/* The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory: real-time pipelines that forbid allocation
 * after start-up (cudaMalloc can synchronise the device and stall for
 * milliseconds), plug-ins whose host application owns every device buffer,
 * and code that must stay inside a fixed memory budget.
 *
 * The same FP32 forward pass as stda_forward on a context of precision
 * STDA_FP32, but with no context and no allocation of any kind: the caller
 * passes the canonical parameters and BN buffers already in device memory
 *   d_params  [137915] float, d_buffers [1360] float (stda_init_params order)
 * and the input / output windows (d_in [B][3][H][W], d_out [B][1][H][W],
 * float). The folded weights (BN folded in FP32 on the GPU at every call)
 * and all activation scratch live in one file-scope device array of 8 MiB
 * that every GPU loading the library holds until the process exits. A call
 * takes at most 65,536 map pixels (B*H*W; e.g. one 256 x 256 window or
 * sixteen 64 x 64 windows); larger calls return STDA_ERR_SHAPE without
 * launching anything.
 *
 * The first call on a device looks up the array's device address on that
 * device (cudaGetSymbolAddress). With CUDA's lazy module loading that first
 * call (or the library's first kernel launch on the device) is also when
 * the module is loaded and the 8 MiB are placed in device memory, so a
 * caller that cannot allocate later should make one call at start-up, and
 * before any stream capture. Every call on a device shares the one array
 * and overwrites it: calls whose work overlaps on the GPU (different
 * streams, or different host threads without ordering) race and corrupt
 * each other's results. Nothing in the array needs to start at zero: each
 * call writes every value it later reads. */
stda_status stda_forward_static(const float* d_params, const float* d_buffers,
                                const float* d_in, float* d_out, int B, int H,
                                int W, struct CUstream_st* stream);

/* ------------------------------------------------------------ measurement */

/* Per-kernel timing: while enabled, every kernel the context launches is
 * bracketed by a CUDA event pair recorded on the launch's own stream.
 * Enabling or disabling synchronises the device and clears the records. */
stda_status stda_profile(stda_ctx* ctx, int enable);
/* Synchronises on the last record, then fills, per kernel of the forward
 * pass (up to `max`): its name, total milliseconds and launch count since
 * the last read, and clears the records. Returns the number of kernels, or
 * -1 on error. Any output array may be NULL. */
int stda_profile_read(stda_ctx* ctx, const char** names, double* total_ms,
                      int* launches, int max);
/* Number of kernels the context has launched since it was created. */
uint64_t stda_launch_count(stda_ctx* ctx);

/* -------------------------------------------------------------- generator */

typedef struct {
  int N, M;          /* fast-time samples per chirp, chirps per frame       */
  int P, Q;          /* range / Doppler DFT points (P >= N, Q >= M, powers
                        of two, P*Q <= 2^20): the map is H = P by W = Q     */
  int tmin, tmax;    /* point targets per window, uniform integer, <= 16   */
  int imin, imax;    /* interferers per frame, uniform integer, <= 4       */
  double snr_min, snr_max; /* per-sample target SNR [dB]                    */
  double inr_min, inr_max; /* interferer power above a target [dB]          */
  double kmin, kmax;       /* interferer / victim chirp slope ratio         */
} stda_gen_config;

/* Synthesises windows w0 .. w0+B-1 of workload `cid` from `seed` (Sec. III:
 * point targets per Eq. "discrete signal", dechirped interfering chirps and
 * complex Gaussian noise per Eq. "IF signal", Hann window, 2-D DFT per Eqs.
 * "column transform"/"row transform", Doppler axis centred, 20 log10
 * magnitude min-max normalised per map), computed in FP64 on the GPU.
 *   d_noisy  [B][3][P][Q] out, element type `bf16` ? bfloat16 : float
 *   d_clean  [B][P][Q]    out (targets + the same noise, no interferers), or NULL
 *   d_bins   [B][16][2]   out int32 frame-t peak cells (p*, q*), or NULL
 *   d_ntgt   [B]          out int32 target count, or NULL
 * Allocates temporary device memory for the duration of the call (freed in
 * stream order). */
stda_status stda_generate(const stda_gen_config* g, uint64_t seed,
                          uint64_t cid, int w0, int B, int bf16,
                          void* d_noisy, void* d_clean, int* d_bins,
                          int* d_ntgt, struct CUstream_st* stream);

/* ------------------------------------------------------------- evaluation */

/* Per-window evaluation of B maps (Sec. V-B), no context needed:
 *   d_maps   [B][H][W] denoised (or any) maps, bfloat16 if bf16 else float
 *   d_clean  [B][H][W] interference-free maps (same type), or NULL
 *   d_bins   [B][16][2] int32 target peak cells (as stda_generate writes)
 *   d_ntgt   [B] int32 target counts
 *   d_sinr   [B] double: Eq. (SINR), 10 log10 of the mean z^2 over the
 *            distinct peak cells over the mean z^2 over the cells outside
 *            every (2 guard + 1)^2 box around a peak; FP64 sums. Or NULL.
 *   d_evm    [B] double: Eq. (EVM), mean over the peak cells of
 *            |clean - z| / |clean| (needs d_clean), or NULL
 *   d_det    [B][H][W] uint8 CA-CFAR detections, or NULL: cell power z^2
 *            against alpha times the mean power of the training cells (the
 *            (2 (cfar_guard + cfar_train) + 1)^2 square minus the
 *            (2 cfar_guard + 1)^2 guard square, clipped at the edges),
 *            alpha = N (pfa^(-1/N) - 1) for N training cells
 *   d_det_rate [B] float: fraction of distinct targets with a detection
 *            within +-1 cell (the paper's AP without its clustering step),
 *            or NULL
 * May allocate temporary device memory (stream-ordered); synchronises the
 * stream when CA-CFAR runs. */
stda_status stda_metrics(const void* d_maps, const void* d_clean, int bf16,
                         const int* d_bins, const int* d_ntgt, int B, int H,
                         int W, int guard, int cfar_guard, int cfar_train,
                         double pfa, double* d_sinr, double* d_evm,
                         float* d_det_rate, unsigned char* d_det,
                         struct CUstream_st* stream);

#ifdef __cplusplus
}
#endif
#endif /* STDA_H */
