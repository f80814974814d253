/*
 * Radar-STDA oracle — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, double-precision CPU implementation of what the Radar-STDA
 * hot path computes: the synthetic range-Doppler (RD) generator of Sec. III
 * (Eqs. "discrete signal", "IF signal", "column transform", "row transform")
 * and the denoising autoencoder of Sec. IV (Eqs. "concat_operation",
 * "mobile_encoder_stage1/2", "mobile_decoder_stage1/2",
 * "eca_process_equation"), plus the SINR/EVM metrics of Sec. V-B.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this code. It shares nothing with the CUDA library: no headers,
 * no helpers, no tables. Convolutions are direct sums, batch normalisation
 * is kept unfolded, the DFT is a direct sum.
 */
#ifndef STDA_ORACLE_H
#define STDA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- counter-based random numbers (SplitMix64, Steele/Lea/Flood 2014) ---- */
uint64_t orc_splitmix64(uint64_t x);
uint64_t orc_key(uint64_t seed, uint64_t cid, uint64_t w, uint64_t tag,
                 uint64_t i1, uint64_t i2);
double orc_u01(uint64_t key); /* (key >> 11) * 2^-53, in [0, 1) */

/* ---- generator configuration (one per workload) ---- */
typedef struct {
  int N, M;        /* fast-time samples per chirp, chirps per frame        */
  int P, Q;        /* range / Doppler DFT points (zero padding if > N, M)  */
  int tmin, tmax;  /* number of point targets, uniform integer            */
  int imin, imax;  /* number of interferers per frame, uniform integer    */
  double snr_min, snr_max; /* per-sample SNR of a target [dB]            */
  double inr_min, inr_max; /* interferer power above a target [dB]       */
  double kmin, kmax;       /* interferer/victim chirp-slope ratio        */
} orc_gen_cfg;

#define ORC_MAX_TGT 16
#define ORC_MAX_INT 4

typedef struct {
  int n_tgt;
  double r[ORC_MAX_TGT];        /* range bin at frame t, in [2, N-2)      */
  double d[ORC_MAX_TGT];        /* Doppler bin, cycles per M chirps       */
  double delta[ORC_MAX_TGT];    /* range-bin drift per frame              */
  double phase[3][ORC_MAX_TGT]; /* per-frame carrier phase                */
  int n_int[3];
  double kappa[3][ORC_MAX_INT];
  double nx[3][ORC_MAX_INT];
  double amp_i[3][ORC_MAX_INT];
  double snr_db;
  double sigma; /* noise standard deviation, sigma^2 = 10^(-SNR/10) */
} orc_scene;

void orc_draw_scene(uint64_t seed, uint64_t cid, uint64_t w,
                    const orc_gen_cfg* cfg, orc_scene* sc);

/* Complex IF samples s(n, m) of frame f (0 = t, 1 = t-1, 2 = t-2), Eq. "IF
 * signal". Layout [N][M] (row n = fast time). with_int=0 drops interferers,
 * with_noise=0 drops v(n, m). */
void orc_if_signal(uint64_t seed, uint64_t cid, uint64_t w,
                   const orc_gen_cfg* cfg, const orc_scene* sc, int f,
                   int with_int, int with_noise, double* s_re, double* s_im);

/* Hann-windowed 2-D DFT of s[N][M] into Y[P][Q] (Eqs. "column transform",
 * "row transform"), Doppler axis shifted so zero velocity sits at Q/2. */
void orc_rd_complex(const double* s_re, const double* s_im, int N, int M,
                    int P, int Q, double* y_re, double* y_im);

/* 20 log10 magnitude, min-max normalised to [0, 1] per map. */
void orc_lognorm(const double* y_re, const double* y_im, int n, double* z);

/* Closed-form frame-t peak cells of every target: bins[2*o] = p*, [2*o+1] = q*. */
int orc_peak_bins(const orc_gen_cfg* cfg, const orc_scene* sc, int* bins);

/* One whole window: noisy[3][P][Q], clean[P][Q] (targets + same noise, no
 * interferers), bins of frame t. Returns the target count. */
int orc_gen_window(uint64_t seed, uint64_t cid, uint64_t w,
                   const orc_gen_cfg* cfg, double* noisy, double* clean,
                   int* bins);

/* Physical helpers for the victim radar of the paper's Table (victim
 * parameters): returns range resolution, max range, max velocity,
 * velocity resolution in m and m/s for N samples and M chirps. */
void orc_radar_helpers(int N, int M, double out[4]);

/* ---- network ---- */
int orc_num_params(void);  /* learnable parameters, canonical order */
int orc_num_buffers(void); /* BN running means and variances        */

/* Whole forward pass for one window, FP64. in[3][H][W] (frames t, t-1, t-2).
 * out[H][W]. blocks (optional) receives the six block outputs E1, E2, E3,
 * D1, D2, D3 (after ECA and skip additions), concatenated, each [C][h][w]. */
int orc_forward(const float* params, const float* buffers, const float* in,
                int H, int W, double* out, double* blocks);

/* The fusion variant with T (1..4) stacked maps in[T][H][W] (frames t,
 * t-1, ...): the stem takes T input channels; params hold
 * orc_num_params_frames(T) values in the canonical order. */
int orc_num_params_frames(int frames);
int orc_forward_frames(const float* params, const float* buffers, const float* in, int frames, int H, int W,
                       double* out);

/* Batch forward with nthreads POSIX threads; out[B][H][W]. */
int orc_forward_batch(const float* params, const float* buffers,
                      const float* in, int B, int H, int W, double* out,
                      int nthreads);

/* Training step with BN in training mode (mode 1: each BN normalises with
 * the mean and biased variance of its input over the whole batch) or with
 * the running statistics (mode 0, equal to orc_loss_grad): MSE over B
 * windows in[B][3][H][W] against target[B][H][W]; gparams[num_params];
 * stats (optional, [num_buffers]) receives each BN's mean and variance in
 * the BN-buffer layout. Returns the loss (NAN on a bad shape). */
double orc_loss_grad_bn(const float* params, const float* buffers, const float* in, const float* target, int B,
                        int H, int W, int mode, double* gparams, double* stats);

/* Primitive operations, exposed for pins. */
void orc_conv2d(const double* x, int Ci, int H, int W, const double* w,
                const double* bias, int Co, int k, int stride, int pad,
                int groups, double* y);
void orc_conv_transpose2d(const double* x, int Ci, int H, int W,
                          const double* w, const double* bias, int Co, int k,
                          int stride, int pad, int groups, double* y);
void orc_eca(double* m, int C, int h, int w, const double* k3);

/* Adjoint of the forward pass for one window: given dL/dz (gout [H][W]),
 * writes dL/dtheta (gparams[num_params], canonical order) and, if gin is not
 * NULL, dL/dx (gin [3][H][W]). */
int orc_adjoint(const float* params, const float* buffers, const float* in,
                const double* gout, int H, int W, double* gparams,
                double* gin);

/* Mean squared error over B windows against target maps [B][H][W] and its
 * gradient with respect to every parameter. Returns the loss. */
double orc_loss_grad(const float* params, const float* buffers,
                     const float* in, const float* target, int B, int H,
                     int W, double* gparams, int nthreads);

/* ---- metrics (Sec. V-B) ---- */
double orc_sinr_db(const double* z, int P, int Q, const int* bins, int nb,
                   int guard);
double orc_evm(const double* clean, const double* est, int P, int Q,
               const int* bins, int nb);

/* CA-CFAR detections det[P][Q] (0/1) on map z; returns their number. */
int orc_cacfar(const double* z, int P, int Q, int guard, int train, double pfa,
               unsigned char* det);
/* Fraction of distinct target cells with a detection within +-1 cell. */
double orc_detect_rate(const unsigned char* det, int P, int Q, const int* bins,
                       int nb);

#ifdef __cplusplus
}
#endif
#endif
