/*
 * Radar-STDA oracle — TEST INFRASTRUCTURE ONLY (see stda_oracle.h).
 *
 * Plain FP64 restatement of the paper's generator (Sec. III), network
 * (Sec. IV) and metrics (Sec. V-B). Everything is a direct sum in the
 * paper's order; nothing is blocked, fused or reordered. Compile with
 * -ffp-contract=off so that every product and sum rounds on its own: the
 * integer peak bins are then the same on any IEEE-754 host.
 *
 * Readings of the paper where it is silent or garbled (layer widths, the
 * stem, the output module, depthwise stage-1 convolutions, the decoder
 * residual, ECA kernel size, generator details) are listed beside each
 * function.
 */
#include "stda_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define BN_EPS 1e-5

/* ======================================================================== */
/* Counter-based random numbers.                                            */
/* ======================================================================== */

/* SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014), applied as
 * a stateless hash: one call maps one 64-bit counter to one 64-bit value. */
uint64_t orc_splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}

/* Key of one draw: hash chain over (seed, workload id, window, tag, i1, i2). */
uint64_t orc_key(uint64_t seed, uint64_t cid, uint64_t w, uint64_t tag,
                 uint64_t i1, uint64_t i2) {
  uint64_t h = orc_splitmix64(seed);
  h = orc_splitmix64(h ^ cid);
  h = orc_splitmix64(h ^ w);
  h = orc_splitmix64(h ^ tag);
  h = orc_splitmix64(h ^ i1);
  h = orc_splitmix64(h ^ i2);
  return h;
}

double orc_u01(uint64_t key) {
  return (double)(key >> 11) * (1.0 / 9007199254740992.0); /* 2^-53 */
}

enum {
  TAG_TGT_COUNT = 1,
  TAG_TGT_R = 2,
  TAG_TGT_D = 3,
  TAG_TGT_PHASE = 4,
  TAG_INT_COUNT = 5,
  TAG_INT_KAPPA = 6,
  TAG_INT_NX = 7,
  TAG_INT_INR = 8,
  TAG_INT_PHASE = 9,
  TAG_SNR = 10,
  TAG_NOISE = 11
};

static double draw(uint64_t seed, uint64_t cid, uint64_t w, uint64_t tag,
                   uint64_t i1, uint64_t i2) {
  return orc_u01(orc_key(seed, cid, w, tag, i1, i2));
}

static int draw_int(int lo, int hi, double u) {
  return lo + (int)floor(u * (double)(hi - lo + 1));
}

/* ======================================================================== */
/* Generator (Sec. III).                                                    */
/* ======================================================================== */

/* Victim radar of the paper's Table "victim parameters": carrier 77 GHz,
 * sampling 12.5 MHz, chirp slope over the ADC window 153.6 MHz / 5.12 us =
 * 30 MHz/us, chirp repetition 2 x 21.12 us (two TX, TDM), 30 frames/s. */
static const double C_LIGHT = 299792458.0;
static const double F_CARRIER = 77e9;
static const double SLOPE = 30e12; /* Hz/s */
static const double F_SAMPLE = 12.5e6;
static const double T_REP = 2.0 * 21.12e-6;
static const double T_FRAME = 1.0 / 30.0;

void orc_radar_helpers(int N, int M, double out[4]) {
  double ts = 1.0 / F_SAMPLE;
  double bw = SLOPE * (double)N * ts;        /* swept bandwidth in the ADC window */
  double lambda = C_LIGHT / F_CARRIER;
  out[0] = C_LIGHT / (2.0 * bw);             /* range resolution */
  out[1] = F_SAMPLE * C_LIGHT / (2.0 * SLOPE); /* max range (complex IF) */
  out[2] = lambda / (4.0 * T_REP);           /* max unambiguous velocity */
  out[3] = lambda / (2.0 * (double)M * T_REP); /* velocity resolution */
}

/* Range-bin drift per frame per Doppler bin: dv * T_frame / dR. */
static double drift_per_doppler_bin(int N, int M) {
  double h[4];
  orc_radar_helpers(N, M, h);
  return h[3] * T_FRAME / h[0];
}

/* Scene draws for one window. Targets: count uniform in [tmin, tmax];
 * range bin r ~ U(2, N-2), Doppler bin d ~ U(-M/2+1, M/2-1), amplitude 1,
 * phase ~ U(0, 2 pi) per frame; the range moves by d * drift per frame.
 * Interferers are drawn independently for each of the three frames. */
void orc_draw_scene(uint64_t seed, uint64_t cid, uint64_t w,
                    const orc_gen_cfg* cfg, orc_scene* sc) {
  memset(sc, 0, sizeof(*sc));
  int N = cfg->N, M = cfg->M;
  double mv = drift_per_doppler_bin(N, M);
  sc->n_tgt = draw_int(cfg->tmin, cfg->tmax, draw(seed, cid, w, TAG_TGT_COUNT, 0, 0));
  for (int o = 0; o < sc->n_tgt; ++o) {
    sc->r[o] = 2.0 + (double)(N - 4) * draw(seed, cid, w, TAG_TGT_R, o, 0);
    sc->d[o] = (double)(-M / 2 + 1) + (double)(M - 2) * draw(seed, cid, w, TAG_TGT_D, o, 0);
    sc->delta[o] = sc->d[o] * mv;
    for (int f = 0; f < 3; ++f)
      sc->phase[f][o] = 2.0 * ORC_PI * draw(seed, cid, w, TAG_TGT_PHASE, o, f);
  }
  for (int f = 0; f < 3; ++f) {
    sc->n_int[f] = draw_int(cfg->imin, cfg->imax, draw(seed, cid, w, TAG_INT_COUNT, f, 0));
    for (int i = 0; i < sc->n_int[f]; ++i) {
      sc->kappa[f][i] = cfg->kmin + (cfg->kmax - cfg->kmin) * draw(seed, cid, w, TAG_INT_KAPPA, f, i);
      sc->nx[f][i] = (double)N * draw(seed, cid, w, TAG_INT_NX, f, i);
      double inr = cfg->inr_min + (cfg->inr_max - cfg->inr_min) * draw(seed, cid, w, TAG_INT_INR, f, i);
      sc->amp_i[f][i] = pow(10.0, inr / 20.0);
    }
  }
  sc->snr_db = cfg->snr_min + (cfg->snr_max - cfg->snr_min) * draw(seed, cid, w, TAG_SNR, 0, 0);
  sc->sigma = pow(10.0, -sc->snr_db / 20.0);
}

/* Eq. "IF signal": s(n,m) = sum_o s_B,o(n,m) + sum_i s_I,i(n,m) + v(n,m).
 *  - s_B (Eq. "discrete signal") in bin units: exp(j 2 pi (r n / N + d m / M)
 *    + j phi): beat frequency r/N cycles per sample, Doppler d/M cycles per
 *    chirp, phi the range-dependent carrier phase.
 *  - s_I: the dechirped interferer is a chirp whose instantaneous frequency
 *    gamma (n - n_x) crosses zero at sample n_x, gamma = (kappa - 1) * slope
 *    * Ts^2 cycles/sample^2; only the part inside the IF band |f| <= fs/2
 *    passes the low-pass filter. A fresh phase per chirp.
 *  - v: complex white Gaussian noise of variance sigma^2 (Box-Muller). */
void orc_if_signal(uint64_t seed, uint64_t cid, uint64_t w,
                   const orc_gen_cfg* cfg, const orc_scene* sc, int f,
                   int with_int, int with_noise, double* s_re, double* s_im) {
  int N = cfg->N, M = cfg->M;
  double a_ts2 = SLOPE / (F_SAMPLE * F_SAMPLE);
  for (int n = 0; n < N; ++n) {
    for (int m = 0; m < M; ++m) {
      double re = 0.0, im = 0.0;
      for (int o = 0; o < sc->n_tgt; ++o) {
        double rf = sc->r[o] - (double)f * sc->delta[o];
        double ph = 2.0 * ORC_PI * (rf * (double)n / (double)N + sc->d[o] * (double)m / (double)M) +
                    sc->phase[f][o];
        re += cos(ph);
        im += sin(ph);
      }
      if (with_int) {
        for (int i = 0; i < sc->n_int[f]; ++i) {
          double g = (sc->kappa[f][i] - 1.0) * a_ts2;
          double x = (double)n - sc->nx[f][i];
          if (fabs(g * x) <= 0.5) {
            double ph = ORC_PI * g * x * x +
                        2.0 * ORC_PI * draw(seed, cid, w, TAG_INT_PHASE, f, (uint64_t)(i * M + m));
            re += sc->amp_i[f][i] * cos(ph);
            im += sc->amp_i[f][i] * sin(ph);
          }
        }
      }
      if (with_noise) {
        uint64_t k = (uint64_t)n * (uint64_t)M + (uint64_t)m;
        double u1 = 1.0 - draw(seed, cid, w, TAG_NOISE, f, 2 * k);
        double u2 = draw(seed, cid, w, TAG_NOISE, f, 2 * k + 1);
        double rad = sqrt(-2.0 * log(u1));
        double sd = sc->sigma * sqrt(0.5);
        re += sd * rad * cos(2.0 * ORC_PI * u2);
        im += sd * rad * sin(2.0 * ORC_PI * u2);
      }
      s_re[n * M + m] = re;
      s_im[n * M + m] = im;
    }
  }
}

static double hann(int n, int N) {
  if (N == 1) return 1.0;
  return 0.5 - 0.5 * cos(2.0 * ORC_PI * (double)n / (double)(N - 1));
}

/* Eqs. "column transform" and "row transform" as direct sums (0-based
 * indices), after a symmetric Hann window on each axis; P >= N, Q >= M means
 * zero padding. The Doppler axis is shifted by Q/2. */
void orc_rd_complex(const double* s_re, const double* s_im, int N, int M,
                    int P, int Q, double* y_re, double* y_im) {
  double* cp = malloc(sizeof(double) * P);
  double* sp = malloc(sizeof(double) * P);
  double* cq = malloc(sizeof(double) * Q);
  double* sq = malloc(sizeof(double) * Q);
  double* t_re = malloc(sizeof(double) * P * M);
  double* t_im = malloc(sizeof(double) * P * M);
  for (int k = 0; k < P; ++k) {
    cp[k] = cos(2.0 * ORC_PI * (double)k / (double)P);
    sp[k] = sin(2.0 * ORC_PI * (double)k / (double)P);
  }
  for (int k = 0; k < Q; ++k) {
    cq[k] = cos(2.0 * ORC_PI * (double)k / (double)Q);
    sq[k] = sin(2.0 * ORC_PI * (double)k / (double)Q);
  }
  /* y(p, m) = sum_n w_n s(n, m) exp(-j 2 pi n p / P) */
  for (int p = 0; p < P; ++p) {
    for (int m = 0; m < M; ++m) {
      double re = 0.0, im = 0.0;
      for (int n = 0; n < N; ++n) {
        int k = (int)(((long long)n * p) % P);
        double wr = hann(n, N) * s_re[n * M + m];
        double wi = hann(n, N) * s_im[n * M + m];
        /* (wr + j wi)(cos - j sin) */
        re += wr * cp[k] + wi * sp[k];
        im += wi * cp[k] - wr * sp[k];
      }
      t_re[p * M + m] = re;
      t_im[p * M + m] = im;
    }
  }
  /* Y(p, q) = sum_m w_m y(p, m) exp(-j 2 pi m q / Q), stored at (q + Q/2) mod Q */
  for (int p = 0; p < P; ++p) {
    for (int q = 0; q < Q; ++q) {
      double re = 0.0, im = 0.0;
      for (int m = 0; m < M; ++m) {
        int k = (int)(((long long)m * q) % Q);
        double wr = hann(m, M) * t_re[p * M + m];
        double wi = hann(m, M) * t_im[p * M + m];
        re += wr * cq[k] + wi * sq[k];
        im += wi * cq[k] - wr * sq[k];
      }
      int qs = (q + Q / 2) % Q;
      y_re[p * Q + qs] = re;
      y_im[p * Q + qs] = im;
    }
  }
  free(cp); free(sp); free(cq); free(sq); free(t_re); free(t_im);
}

/* 20 log10 |Y| (floored at 1e-12), then (L - min) / (max - min) per map. */
void orc_lognorm(const double* y_re, const double* y_im, int n, double* z) {
  double lo = INFINITY, hi = -INFINITY;
  for (int i = 0; i < n; ++i) {
    double mag = sqrt(y_re[i] * y_re[i] + y_im[i] * y_im[i]);
    if (mag < 1e-12) mag = 1e-12;
    z[i] = 20.0 * log10(mag);
    if (z[i] < lo) lo = z[i];
    if (z[i] > hi) hi = z[i];
  }
  for (int i = 0; i < n; ++i) z[i] = (hi > lo) ? (z[i] - lo) / (hi - lo) : 0.0;
}

static int pos_mod(long long a, int m) {
  long long r = a % m;
  return (int)(r < 0 ? r + m : r);
}

/* A beat tone of r cycles per N samples peaks at DFT bin r * P / N (Sec.
 * III-B: the range peak sits at the beat frequency); the Doppler tone of d
 * cycles per M chirps at bin d * Q / M, moved by the Q/2 shift. */
int orc_peak_bins(const orc_gen_cfg* cfg, const orc_scene* sc, int* bins) {
  for (int o = 0; o < sc->n_tgt; ++o) {
    double pr = sc->r[o] * (double)cfg->P / (double)cfg->N;
    double qd = sc->d[o] * (double)cfg->Q / (double)cfg->M;
    long long p = (long long)floor(pr + 0.5);
    long long q = (long long)floor(qd + 0.5);
    bins[2 * o] = pos_mod(p, cfg->P);
    bins[2 * o + 1] = pos_mod((long long)pos_mod(q, cfg->Q) + cfg->Q / 2, cfg->Q);
  }
  return sc->n_tgt;
}

int orc_gen_window(uint64_t seed, uint64_t cid, uint64_t w,
                   const orc_gen_cfg* cfg, double* noisy, double* clean,
                   int* bins) {
  orc_scene sc;
  orc_draw_scene(seed, cid, w, cfg, &sc);
  int N = cfg->N, M = cfg->M, P = cfg->P, Q = cfg->Q;
  double* s_re = malloc(sizeof(double) * N * M);
  double* s_im = malloc(sizeof(double) * N * M);
  double* y_re = malloc(sizeof(double) * P * Q);
  double* y_im = malloc(sizeof(double) * P * Q);
  for (int f = 0; f < 3; ++f) {
    orc_if_signal(seed, cid, w, cfg, &sc, f, 1, 1, s_re, s_im);
    orc_rd_complex(s_re, s_im, N, M, P, Q, y_re, y_im);
    orc_lognorm(y_re, y_im, P * Q, noisy + (size_t)f * P * Q);
  }
  if (clean) {
    orc_if_signal(seed, cid, w, cfg, &sc, 0, 0, 1, s_re, s_im);
    orc_rd_complex(s_re, s_im, N, M, P, Q, y_re, y_im);
    orc_lognorm(y_re, y_im, P * Q, clean);
  }
  free(s_re); free(s_im); free(y_re); free(y_im);
  if (bins) orc_peak_bins(cfg, &sc, bins);
  return sc.n_tgt;
}

/* ======================================================================== */
/* Network (Sec. IV).                                                       */
/* ======================================================================== */

/* 2-D convolution (cross-correlation, as in every DL framework), direct sum:
 * y[o][Y][X] = b[o] + sum_{i in group(o)} sum_{ky,kx}
 *              x[i][Y*s - p + ky][X*s - p + kx] * w[o][i - group base][ky][kx],
 * zero outside the map. w is [Co][Ci/groups][k][k]. */
void orc_conv2d(const double* x, int Ci, int H, int W, const double* w,
                const double* bias, int Co, int k, int stride, int pad,
                int groups, double* y) {
  int Ho = (H + 2 * pad - k) / stride + 1;
  int Wo = (W + 2 * pad - k) / stride + 1;
  int cig = Ci / groups, cog = Co / groups;
  for (int o = 0; o < Co; ++o) {
    int g = o / cog;
    for (int Y = 0; Y < Ho; ++Y) {
      for (int X = 0; X < Wo; ++X) {
        double acc = bias ? bias[o] : 0.0;
        for (int il = 0; il < cig; ++il) {
          int i = g * cig + il;
          for (int ky = 0; ky < k; ++ky) {
            int yy = Y * stride - pad + ky;
            if (yy < 0 || yy >= H) continue;
            for (int kx = 0; kx < k; ++kx) {
              int xx = X * stride - pad + kx;
              if (xx < 0 || xx >= W) continue;
              acc += x[((size_t)i * H + yy) * W + xx] * w[(((size_t)o * cig + il) * k + ky) * k + kx];
            }
          }
        }
        y[((size_t)o * Ho + Y) * Wo + X] = acc;
      }
    }
  }
}

/* Transposed convolution ("DeConv"), as a scatter: every input value
 * x[i][yi][xi] adds x * w[i][o - group base][ky][kx] to output
 * (yi*s - p + ky, xi*s - p + kx). w is [Ci][Co/groups][k][k].
 * Output size (H - 1) s - 2p + k. */
void orc_conv_transpose2d(const double* x, int Ci, int H, int W,
                          const double* w, const double* bias, int Co, int k,
                          int stride, int pad, int groups, double* y) {
  int Ho = (H - 1) * stride - 2 * pad + k;
  int Wo = (W - 1) * stride - 2 * pad + k;
  int cig = Ci / groups, cog = Co / groups;
  for (int o = 0; o < Co; ++o)
    for (int t = 0; t < Ho * Wo; ++t) y[(size_t)o * Ho * Wo + t] = bias ? bias[o] : 0.0;
  for (int i = 0; i < Ci; ++i) {
    int g = i / cig;
    for (int yi = 0; yi < H; ++yi) {
      for (int xi = 0; xi < W; ++xi) {
        double v = x[((size_t)i * H + yi) * W + xi];
        for (int ol = 0; ol < cog; ++ol) {
          int o = g * cog + ol;
          for (int ky = 0; ky < k; ++ky) {
            int Y = yi * stride - pad + ky;
            if (Y < 0 || Y >= Ho) continue;
            for (int kx = 0; kx < k; ++kx) {
              int X = xi * stride - pad + kx;
              if (X < 0 || X >= Wo) continue;
              y[((size_t)o * Ho + Y) * Wo + X] += v * w[(((size_t)i * cog + ol) * k + ky) * k + kx];
            }
          }
        }
      }
    }
  }
}

/* Batch normalisation in inference form, per channel. */
static void batchnorm(double* x, int C, int n, const double* gam,
                      const double* bet, const double* mean, const double* var) {
  for (int c = 0; c < C; ++c) {
    double s = gam[c] / sqrt(var[c] + BN_EPS);
    for (int t = 0; t < n; ++t) x[(size_t)c * n + t] = s * (x[(size_t)c * n + t] - mean[c]) + bet[c];
  }
}

static void relu(double* x, size_t n) {
  for (size_t t = 0; t < n; ++t) x[t] = x[t] > 0.0 ? x[t] : 0.0;
}

/* Eq. "eca_process_equation": m_tilde = GAP(m); W_m = sigmoid(Conv1D(m_tilde));
 * m_hat = W_m * m. Reading: the 1-D convolution has kernel size 3 (ECA-Net's
 * adaptive size for 8..64 channels), zero padding 1, no bias. */
void orc_eca(double* m, int C, int h, int w, const double* k3) {
  size_t n = (size_t)h * w;
  double* g = malloc(sizeof(double) * C);
  for (int c = 0; c < C; ++c) {
    double s = 0.0;
    for (size_t t = 0; t < n; ++t) s += m[c * n + t];
    g[c] = s / (double)n;
  }
  for (int c = 0; c < C; ++c) {
    double z = 0.0;
    for (int j = 0; j < 3; ++j) {
      int cc = c + j - 1;
      if (cc >= 0 && cc < C) z += k3[j] * g[cc];
    }
    double sc = 1.0 / (1.0 + exp(-z));
    for (size_t t = 0; t < n; ++t) m[c * n + t] *= sc;
  }
  free(g);
}

/* ---- parameter table (canonical order) ----
 * stem:  W[8][3][3][3], BN(gamma[8], beta[8])
 * block: W1[c] (depthwise 1x1), BN1, W3[c][1][3][3] (depthwise 3x3), BN2,
 *        BN3 (identity branch), W2 (stage 2), BN, Wres, bres[cout], eca[3]
 *        encoder: W2, Wres are [2c][c][3][3] (stride 2, pad 1)
 *        decoder: W2, Wres are [c][c/2][4][4] (transposed, stride 2, pad 1)
 * out:   W[1][8][3][3], b[1]
 * Buffers: per BN, running mean[C] then running var[C]; order stem, then per
 * block BN1, BN2, BN3, BN. */
typedef struct {
  int enc, cin, cout;
  const double *w1, *g1, *b1, *w3, *g2, *b2, *g3, *b3, *w2, *g, *b, *rw, *rb, *eca;
  const double *m1, *v1, *m2, *v2, *m3, *v3, *m, *v;
} orc_blk;

typedef struct {
  double* pmem;
  double* bmem;
  int frames; /* input maps per window: stem input channels */
  const double *stem_w, *stem_g, *stem_b, *stem_m, *stem_v;
  orc_blk blk[6];
  const double *out_w, *out_b;
} orc_net;

static const int BLK_ENC[6] = {1, 1, 1, 0, 0, 0};
static const int BLK_CIN[6] = {8, 16, 32, 64, 32, 16};

static int blk_cout(int b) { return BLK_ENC[b] ? 2 * BLK_CIN[b] : BLK_CIN[b] / 2; }
static int blk_dense(int b) {
  int ci = BLK_CIN[b], co = blk_cout(b);
  return BLK_ENC[b] ? co * ci * 9 : ci * co * 16;
}

/* The stem weight W[8][T][3][3] grows with the number T of stacked maps;
 * every other tensor is independent of T. */
int orc_num_params_frames(int frames) {
  int n = 8 * frames * 9 + 16;
  for (int b = 0; b < 6; ++b) {
    int ci = BLK_CIN[b], co = blk_cout(b);
    n += ci + 2 * ci + 9 * ci + 2 * ci + 2 * ci + blk_dense(b) + 2 * co + blk_dense(b) + co + 3;
  }
  return n + 72 + 1;
}

int orc_num_params(void) { return orc_num_params_frames(3); }

int orc_num_buffers(void) {
  int n = 16;
  for (int b = 0; b < 6; ++b) n += 2 * (3 * BLK_CIN[b] + blk_cout(b));
  return n;
}

static void net_load_frames(orc_net* net, const float* params, const float* buffers, int frames) {
  int np = orc_num_params_frames(frames), nb = orc_num_buffers();
  net->frames = frames;
  net->pmem = malloc(sizeof(double) * np);
  net->bmem = malloc(sizeof(double) * nb);
  for (int i = 0; i < np; ++i) net->pmem[i] = (double)params[i];
  for (int i = 0; i < nb; ++i) net->bmem[i] = (double)buffers[i];
  const double* p = net->pmem;
  const double* q = net->bmem;
  net->stem_w = p; p += 8 * frames * 9;
  net->stem_g = p; p += 8;
  net->stem_b = p; p += 8;
  net->stem_m = q; q += 8;
  net->stem_v = q; q += 8;
  for (int b = 0; b < 6; ++b) {
    orc_blk* k = &net->blk[b];
    int ci = BLK_CIN[b], co = blk_cout(b);
    k->enc = BLK_ENC[b]; k->cin = ci; k->cout = co;
    k->w1 = p; p += ci;
    k->g1 = p; p += ci;
    k->b1 = p; p += ci;
    k->w3 = p; p += 9 * ci;
    k->g2 = p; p += ci;
    k->b2 = p; p += ci;
    k->g3 = p; p += ci;
    k->b3 = p; p += ci;
    k->w2 = p; p += blk_dense(b);
    k->g = p; p += co;
    k->b = p; p += co;
    k->rw = p; p += blk_dense(b);
    k->rb = p; p += co;
    k->eca = p; p += 3;
    k->m1 = q; q += ci;
    k->v1 = q; q += ci;
    k->m2 = q; q += ci;
    k->v2 = q; q += ci;
    k->m3 = q; q += ci;
    k->v3 = q; q += ci;
    k->m = q; q += co;
    k->v = q; q += co;
  }
  net->out_w = p; p += 72;
  net->out_b = p; p += 1;
}

static void net_load(orc_net* net, const float* params, const float* buffers) {
  net_load_frames(net, params, buffers, 3);
}

static void net_free(orc_net* net) {
  free(net->pmem);
  free(net->bmem);
}

/* One mobile encoder or decoder block followed by ECA.
 * Stage 1 (Eqs. "mobile_encoder_stage1", "mobile_decoder_stage1"):
 *   x1 = ReLU(BN1(Conv1x1 x) + BN2(Conv3x3 x) + BN3(x)); reading: both
 *   convolutions are depthwise (groups = channels), as in MobileOne and the
 *   paper's "depthwise separable" remark; the decoder uses transposed
 *   convolutions of stride 1.
 * Stage 2 (Eqs. "mobile_encoder_stage2", "mobile_decoder_stage2"):
 *   y = ReLU(BN(Conv3x3-s2 x1)) + Conv3x3-s2(x) for the encoder;
 *   y = ReLU(BN(DeConv4x4-s2 x1)) + DeConv4x4-s2(x) for the decoder (reading:
 *   the printed residual cannot double the map, so it mirrors the main
 *   branch). The residual convolution carries a bias, the main one does not.
 * Then ECA on the block output. x is [cin][h][w]; returns a fresh buffer
 * [cout][ho][wo]. */
static double* block_forward(const orc_blk* k, const double* x, int h, int w,
                             int* ho, int* wo) {
  int ci = k->cin, co = k->cout;
  size_t n = (size_t)h * w;
  double* t1 = malloc(sizeof(double) * ci * n);
  double* t2 = malloc(sizeof(double) * ci * n);
  double* x1 = malloc(sizeof(double) * ci * n);
  if (k->enc) {
    orc_conv2d(x, ci, h, w, k->w1, NULL, ci, 1, 1, 0, ci, t1);
    orc_conv2d(x, ci, h, w, k->w3, NULL, ci, 3, 1, 1, ci, t2);
  } else {
    orc_conv_transpose2d(x, ci, h, w, k->w1, NULL, ci, 1, 1, 0, ci, t1);
    orc_conv_transpose2d(x, ci, h, w, k->w3, NULL, ci, 3, 1, 1, ci, t2);
  }
  batchnorm(t1, ci, (int)n, k->g1, k->b1, k->m1, k->v1);
  batchnorm(t2, ci, (int)n, k->g2, k->b2, k->m2, k->v2);
  memcpy(x1, x, sizeof(double) * ci * n);
  batchnorm(x1, ci, (int)n, k->g3, k->b3, k->m3, k->v3);
  for (size_t t = 0; t < ci * n; ++t) x1[t] += t1[t] + t2[t];
  relu(x1, ci * n);
  int H2 = k->enc ? h / 2 : 2 * h, W2 = k->enc ? w / 2 : 2 * w;
  size_t n2 = (size_t)H2 * W2;
  double* mn = malloc(sizeof(double) * co * n2);
  double* rs = malloc(sizeof(double) * co * n2);
  if (k->enc) {
    orc_conv2d(x1, ci, h, w, k->w2, NULL, co, 3, 2, 1, 1, mn);
    orc_conv2d(x, ci, h, w, k->rw, k->rb, co, 3, 2, 1, 1, rs);
  } else {
    orc_conv_transpose2d(x1, ci, h, w, k->w2, NULL, co, 4, 2, 1, 1, mn);
    orc_conv_transpose2d(x, ci, h, w, k->rw, k->rb, co, 4, 2, 1, 1, rs);
  }
  batchnorm(mn, co, (int)n2, k->g, k->b, k->m, k->v);
  relu(mn, co * n2);
  for (size_t t = 0; t < co * n2; ++t) mn[t] += rs[t];
  orc_eca(mn, co, H2, W2, k->eca);
  free(t1); free(t2); free(x1); free(rs);
  *ho = H2;
  *wo = W2;
  return mn;
}

/* Sec. IV-A..D. Input module (reading): the three maps are stacked as
 * channels (Eq. "concat_operation", order t, t-1, t-2), then a 3x3
 * convolution 3 -> 8 with BN and ReLU. Encoder widths 8 -> 16 -> 32 -> 64,
 * decoder 64 -> 32 -> 16 -> 8; the two skip connections (Sec. IV-D) add the
 * encoder outputs of the same size to the outputs of decoder blocks 1 and 2.
 * Output module (reading): 3x3 convolution 8 -> 1 with bias, then sigmoid. */
static int forward_one(const orc_net* net, const float* in, int H, int W,
                       double* out, double* blocks) {
  if (H <= 0 || W <= 0 || H % 8 || W % 8) return -1;
  size_t n = (size_t)H * W;
  const int T = net->frames;
  double* x = malloc(sizeof(double) * T * n);
  for (size_t t = 0; t < T * n; ++t) x[t] = (double)in[t];
  double* a = malloc(sizeof(double) * 8 * n);
  orc_conv2d(x, T, H, W, net->stem_w, NULL, 8, 3, 1, 1, 1, a);
  batchnorm(a, 8, (int)n, net->stem_g, net->stem_b, net->stem_m, net->stem_v);
  relu(a, 8 * n);
  free(x);
  double* skip[2] = {NULL, NULL};
  int h = H, w = W;
  size_t boff = 0;
  for (int b = 0; b < 6; ++b) {
    int ho, wo;
    double* y = block_forward(&net->blk[b], a, h, w, &ho, &wo);
    size_t sz = (size_t)net->blk[b].cout * ho * wo;
    if (b == 3 || b == 4) {
      const double* s = skip[4 - b]; /* D1 + E2, D2 + E1 */
      for (size_t t = 0; t < sz; ++t) y[t] += s[t];
    }
    if (b == 0 || b == 1) {
      skip[b] = malloc(sizeof(double) * sz);
      memcpy(skip[b], y, sizeof(double) * sz);
    }
    if (blocks) {
      memcpy(blocks + boff, y, sizeof(double) * sz);
      boff += sz;
    }
    free(a);
    a = y;
    h = ho;
    w = wo;
  }
  double* z = malloc(sizeof(double) * n);
  orc_conv2d(a, 8, H, W, net->out_w, net->out_b, 1, 3, 1, 1, 1, z);
  for (size_t t = 0; t < n; ++t) out[t] = 1.0 / (1.0 + exp(-z[t]));
  free(z);
  free(a);
  free(skip[0]);
  free(skip[1]);
  return 0;
}

int orc_forward(const float* params, const float* buffers, const float* in,
                int H, int W, double* out, double* blocks) {
  orc_net net;
  net_load(&net, params, buffers);
  int rc = forward_one(&net, in, H, W, out, blocks);
  net_free(&net);
  return rc;
}

/* The fusion variants of Sec. IV-A: T = 2, 3 or 4 maps (frames t, t-1, ...)
 * stacked as channels in place of three. */
int orc_forward_frames(const float* params, const float* buffers, const float* in, int frames, int H, int W,
                       double* out) {
  if (frames < 1 || frames > 4) return -1;
  orc_net net;
  net_load_frames(&net, params, buffers, frames);
  int rc = forward_one(&net, in, H, W, out, NULL);
  net_free(&net);
  return rc;
}

typedef struct {
  const orc_net* net;
  const float* in;
  double* out;
  int B, H, W, tid, nt, rc;
} fwd_job;

static void* fwd_worker(void* arg) {
  fwd_job* j = (fwd_job*)arg;
  size_t n = (size_t)j->H * j->W;
  for (int b = j->tid; b < j->B; b += j->nt) {
    int rc = forward_one(j->net, j->in + (size_t)b * 3 * n, j->H, j->W, j->out + (size_t)b * n, NULL);
    if (rc) j->rc = rc;
  }
  return NULL;
}

int orc_forward_batch(const float* params, const float* buffers,
                      const float* in, int B, int H, int W, double* out,
                      int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > B) nthreads = B;
  orc_net net;
  net_load(&net, params, buffers);
  pthread_t th[256];
  fwd_job jobs[256];
  if (nthreads > 256) nthreads = 256;
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = (fwd_job){&net, in, out, B, H, W, t, nthreads, 0};
    pthread_create(&th[t], NULL, fwd_worker, &jobs[t]);
  }
  int rc = 0;
  for (int t = 0; t < nthreads; ++t) {
    pthread_join(th[t], NULL);
    if (jobs[t].rc) rc = jobs[t].rc;
  }
  net_free(&net);
  return rc;
}

/* ======================================================================== */
/* Gradient (adjoint of the forward pass), FP64.                            */
/* ======================================================================== */

/* Adjoints of the primitives, direct sums (accumulate into dx / dw / db). */
static void conv2d_bwd(const double* x, int Ci, int H, int W, const double* w, int Co, int k, int stride,
                       int pad, int groups, const double* dy, double* dx, double* dw, double* db) {
  int Ho = (H + 2 * pad - k) / stride + 1;
  int Wo = (W + 2 * pad - k) / stride + 1;
  int cig = Ci / groups, cog = Co / groups;
  for (int o = 0; o < Co; ++o) {
    int g = o / cog;
    for (int Y = 0; Y < Ho; ++Y)
      for (int X = 0; X < Wo; ++X) {
        double d = dy[((size_t)o * Ho + Y) * Wo + X];
        if (db) db[o] += d;
        for (int il = 0; il < cig; ++il) {
          int i = g * cig + il;
          for (int ky = 0; ky < k; ++ky) {
            int yy = Y * stride - pad + ky;
            if (yy < 0 || yy >= H) continue;
            for (int kx = 0; kx < k; ++kx) {
              int xx = X * stride - pad + kx;
              if (xx < 0 || xx >= W) continue;
              size_t wi = (((size_t)o * cig + il) * k + ky) * k + kx;
              size_t xi = ((size_t)i * H + yy) * W + xx;
              if (dw) dw[wi] += d * x[xi];
              if (dx) dx[xi] += d * w[wi];
            }
          }
        }
      }
  }
}

static void conv_transpose2d_bwd(const double* x, int Ci, int H, int W, const double* w, int Co, int k,
                                 int stride, int pad, int groups, const double* dy, double* dx, double* dw,
                                 double* db) {
  int Ho = (H - 1) * stride - 2 * pad + k;
  int Wo = (W - 1) * stride - 2 * pad + k;
  int cig = Ci / groups, cog = Co / groups;
  if (db)
    for (int o = 0; o < Co; ++o)
      for (int t = 0; t < Ho * Wo; ++t) db[o] += dy[(size_t)o * Ho * Wo + t];
  for (int i = 0; i < Ci; ++i) {
    int g = i / cig;
    for (int yi = 0; yi < H; ++yi)
      for (int xi = 0; xi < W; ++xi) {
        size_t xo = ((size_t)i * H + yi) * W + xi;
        for (int ol = 0; ol < cog; ++ol) {
          int o = g * cog + ol;
          for (int ky = 0; ky < k; ++ky) {
            int Y = yi * stride - pad + ky;
            if (Y < 0 || Y >= Ho) continue;
            for (int kx = 0; kx < k; ++kx) {
              int X = xi * stride - pad + kx;
              if (X < 0 || X >= Wo) continue;
              double d = dy[((size_t)o * Ho + Y) * Wo + X];
              size_t wi = (((size_t)i * cog + ol) * k + ky) * k + kx;
              if (dw) dw[wi] += d * x[xo];
              if (dx) dx[xo] += d * w[wi];
            }
          }
        }
      }
  }
}

/* BN in inference form: y = gam (x - mean) / sqrt(var + eps) + bet. Given dy,
 * accumulates dgam, dbet and (if dx) dx. */
static void batchnorm_bwd(const double* x, int C, int n, const double* gam, const double* mean,
                          const double* var, const double* dy, double* dx, double* dgam, double* dbet) {
  for (int c = 0; c < C; ++c) {
    double is = 1.0 / sqrt(var[c] + BN_EPS);
    for (int t = 0; t < n; ++t) {
      double d = dy[(size_t)c * n + t];
      dgam[c] += d * (x[(size_t)c * n + t] - mean[c]) * is;
      dbet[c] += d;
      if (dx) dx[(size_t)c * n + t] += d * gam[c] * is;
    }
  }
}

/* Saved tensors of one block (for the adjoint). */
typedef struct {
  int h, w, H2, W2;
  double *x, *t1, *t2, *x1, *u, *y, *g, *s;
} blk_tape;

/* Gradient pointers of one block, in the canonical blob. */
typedef struct {
  double *w1, *g1, *b1, *w3, *g2, *b2, *g3, *b3, *w2, *g, *b, *rw, *rb, *eca;
} blk_grad;

static double* dup(const double* a, size_t n) {
  double* r = malloc(sizeof(double) * n);
  memcpy(r, a, sizeof(double) * n);
  return r;
}

/* Forward of one block keeping its intermediates (same arithmetic as
 * block_forward). Returns the post-ECA output. */
static double* block_forward_tape(const orc_blk* k, const double* x, int h, int w, blk_tape* T) {
  int ci = k->cin, co = k->cout;
  size_t n = (size_t)h * w;
  T->h = h;
  T->w = w;
  T->x = dup(x, ci * n);
  T->t1 = malloc(sizeof(double) * ci * n);
  T->t2 = malloc(sizeof(double) * ci * n);
  if (k->enc) {
    orc_conv2d(x, ci, h, w, k->w1, NULL, ci, 1, 1, 0, ci, T->t1);
    orc_conv2d(x, ci, h, w, k->w3, NULL, ci, 3, 1, 1, ci, T->t2);
  } else {
    orc_conv_transpose2d(x, ci, h, w, k->w1, NULL, ci, 1, 1, 0, ci, T->t1);
    orc_conv_transpose2d(x, ci, h, w, k->w3, NULL, ci, 3, 1, 1, ci, T->t2);
  }
  double* b1 = dup(T->t1, ci * n);
  double* b2 = dup(T->t2, ci * n);
  double* b3 = dup(x, ci * n);
  batchnorm(b1, ci, (int)n, k->g1, k->b1, k->m1, k->v1);
  batchnorm(b2, ci, (int)n, k->g2, k->b2, k->m2, k->v2);
  batchnorm(b3, ci, (int)n, k->g3, k->b3, k->m3, k->v3);
  T->x1 = malloc(sizeof(double) * ci * n);
  for (size_t t = 0; t < ci * n; ++t) T->x1[t] = b1[t] + b2[t] + b3[t];
  relu(T->x1, ci * n);
  free(b1); free(b2); free(b3);
  int H2 = k->enc ? h / 2 : 2 * h, W2 = k->enc ? w / 2 : 2 * w;
  size_t n2 = (size_t)H2 * W2;
  T->H2 = H2;
  T->W2 = W2;
  T->u = malloc(sizeof(double) * co * n2);
  double* rs = malloc(sizeof(double) * co * n2);
  if (k->enc) {
    orc_conv2d(T->x1, ci, h, w, k->w2, NULL, co, 3, 2, 1, 1, T->u);
    orc_conv2d(x, ci, h, w, k->rw, k->rb, co, 3, 2, 1, 1, rs);
  } else {
    orc_conv_transpose2d(T->x1, ci, h, w, k->w2, NULL, co, 4, 2, 1, 1, T->u);
    orc_conv_transpose2d(x, ci, h, w, k->rw, k->rb, co, 4, 2, 1, 1, rs);
  }
  T->y = dup(T->u, co * n2);
  batchnorm(T->y, co, (int)n2, k->g, k->b, k->m, k->v);
  relu(T->y, co * n2);
  for (size_t t = 0; t < co * n2; ++t) T->y[t] += rs[t];
  free(rs);
  /* ECA, keeping g and s */
  T->g = malloc(sizeof(double) * co);
  T->s = malloc(sizeof(double) * co);
  for (int c = 0; c < co; ++c) {
    double a = 0.0;
    for (size_t t = 0; t < n2; ++t) a += T->y[c * n2 + t];
    T->g[c] = a / (double)n2;
  }
  double* out = malloc(sizeof(double) * co * n2);
  for (int c = 0; c < co; ++c) {
    double z = 0.0;
    for (int j = 0; j < 3; ++j) {
      int cc = c + j - 1;
      if (cc >= 0 && cc < co) z += k->eca[j] * T->g[cc];
    }
    T->s[c] = 1.0 / (1.0 + exp(-z));
    for (size_t t = 0; t < n2; ++t) out[c * n2 + t] = T->s[c] * T->y[c * n2 + t];
  }
  return out;
}

/* Adjoint of one block: dout (gradient of the post-ECA output) -> dx
 * (gradient of the block input, accumulated) and the parameter gradients. */
static void block_backward(const orc_blk* k, const blk_tape* T, const double* dout, double* dx, blk_grad* G) {
  int ci = k->cin, co = k->cout, h = T->h, w = T->w, H2 = T->H2, W2 = T->W2;
  size_t n = (size_t)h * w, n2 = (size_t)H2 * W2;
  /* ECA: out = s * y, s = sigmoid(z), z = conv1d(g), g = mean(y) */
  double* dy = malloc(sizeof(double) * co * n2);
  double* dz = calloc(co, sizeof(double));
  for (int c = 0; c < co; ++c) {
    double ds = 0.0;
    for (size_t t = 0; t < n2; ++t) {
      ds += dout[c * n2 + t] * T->y[c * n2 + t];
      dy[c * n2 + t] = T->s[c] * dout[c * n2 + t];
    }
    dz[c] = ds * T->s[c] * (1.0 - T->s[c]);
  }
  for (int c = 0; c < co; ++c)
    for (int j = 0; j < 3; ++j) {
      int cc = c + j - 1;
      if (cc < 0 || cc >= co) continue;
      G->eca[j] += dz[c] * T->g[cc];
      /* dg[cc] += dz[c] * k[j]; g = mean(y) */
      double dg = dz[c] * k->eca[j] / (double)n2;
      for (size_t t = 0; t < n2; ++t) dy[cc * n2 + t] += dg;
    }
  free(dz);
  /* y = ReLU(BN(u)) + res(x) */
  double* dbn = malloc(sizeof(double) * co * n2);
  for (int c = 0; c < co; ++c) {
    double is = 1.0 / sqrt(k->v[c] + BN_EPS);
    for (size_t t = 0; t < n2; ++t) {
      double bn = k->g[c] * (T->u[c * n2 + t] - k->m[c]) * is + k->b[c];
      dbn[c * n2 + t] = bn > 0.0 ? dy[c * n2 + t] : 0.0;
    }
  }
  double* du = calloc(co * n2, sizeof(double));
  batchnorm_bwd(T->u, co, (int)n2, k->g, k->m, k->v, dbn, du, G->g, G->b);
  free(dbn);
  double* dx1 = calloc(ci * n, sizeof(double));
  if (k->enc) {
    conv2d_bwd(T->x1, ci, h, w, k->w2, co, 3, 2, 1, 1, du, dx1, G->w2, NULL);
    conv2d_bwd(T->x, ci, h, w, k->rw, co, 3, 2, 1, 1, dy, dx, G->rw, G->rb);
  } else {
    conv_transpose2d_bwd(T->x1, ci, h, w, k->w2, co, 4, 2, 1, 1, du, dx1, G->w2, NULL);
    conv_transpose2d_bwd(T->x, ci, h, w, k->rw, co, 4, 2, 1, 1, dy, dx, G->rw, G->rb);
  }
  free(du);
  free(dy);
  /* x1 = ReLU(BN1(t1) + BN2(t2) + BN3(x)) */
  for (size_t t = 0; t < ci * n; ++t)
    if (T->x1[t] <= 0.0) dx1[t] = 0.0;
  double* dt1 = calloc(ci * n, sizeof(double));
  double* dt2 = calloc(ci * n, sizeof(double));
  batchnorm_bwd(T->t1, ci, (int)n, k->g1, k->m1, k->v1, dx1, dt1, G->g1, G->b1);
  batchnorm_bwd(T->t2, ci, (int)n, k->g2, k->m2, k->v2, dx1, dt2, G->g2, G->b2);
  batchnorm_bwd(T->x, ci, (int)n, k->g3, k->m3, k->v3, dx1, dx, G->g3, G->b3);
  if (k->enc) {
    conv2d_bwd(T->x, ci, h, w, k->w1, ci, 1, 1, 0, ci, dt1, dx, G->w1, NULL);
    conv2d_bwd(T->x, ci, h, w, k->w3, ci, 3, 1, 1, ci, dt2, dx, G->w3, NULL);
  } else {
    conv_transpose2d_bwd(T->x, ci, h, w, k->w1, ci, 1, 1, 0, ci, dt1, dx, G->w1, NULL);
    conv_transpose2d_bwd(T->x, ci, h, w, k->w3, ci, 3, 1, 1, ci, dt2, dx, G->w3, NULL);
  }
  free(dt1); free(dt2); free(dx1);
}

static void tape_free(blk_tape* T) {
  free(T->x); free(T->t1); free(T->t2); free(T->x1); free(T->u); free(T->y); free(T->g); free(T->s);
}

/* dL/dtheta and dL/dx of one window given dL/dz (gout [H][W]); the
 * gradients are accumulated into gparams (canonical order) and gin
 * ([3][H][W], may be NULL). */
static int adjoint_one(const orc_net* net, const float* in, const double* gout, int H, int W, double* gp,
                       double* gin) {
  if (H <= 0 || W <= 0 || H % 8 || W % 8) return -1;
  size_t n = (size_t)H * W;
  /* gradient pointers mirror the parameter layout */
  double* q = gp;
  double *gstem_w = q, *gstem_g = q + 216, *gstem_b = q + 224;
  q += 232;
  blk_grad G[6];
  for (int b = 0; b < 6; ++b) {
    int ci = BLK_CIN[b], co = blk_cout(b);
    G[b].w1 = q; q += ci;
    G[b].g1 = q; q += ci;
    G[b].b1 = q; q += ci;
    G[b].w3 = q; q += 9 * ci;
    G[b].g2 = q; q += ci;
    G[b].b2 = q; q += ci;
    G[b].g3 = q; q += ci;
    G[b].b3 = q; q += ci;
    G[b].w2 = q; q += blk_dense(b);
    G[b].g = q; q += co;
    G[b].b = q; q += co;
    G[b].rw = q; q += blk_dense(b);
    G[b].rb = q; q += co;
    G[b].eca = q; q += 3;
  }
  double *gout_w = q, *gout_b = q + 72;
  /* forward with tape */
  double* x = malloc(sizeof(double) * 3 * n);
  for (size_t t = 0; t < 3 * n; ++t) x[t] = (double)in[t];
  double* su = malloc(sizeof(double) * 8 * n); /* stem conv output */
  orc_conv2d(x, 3, H, W, net->stem_w, NULL, 8, 3, 1, 1, 1, su);
  double* a = dup(su, 8 * n);
  batchnorm(a, 8, (int)n, net->stem_g, net->stem_b, net->stem_m, net->stem_v);
  relu(a, 8 * n);
  blk_tape T[6];
  double* outs[6];
  double* stem_out = a;
  int h = H, w = W;
  for (int b = 0; b < 6; ++b) {
    outs[b] = block_forward_tape(&net->blk[b], a, h, w, &T[b]);
    size_t sz = (size_t)net->blk[b].cout * T[b].H2 * T[b].W2;
    if (b == 3 || b == 4) {
      const double* s = outs[4 - b];
      for (size_t t = 0; t < sz; ++t) outs[b][t] += s[t];
    }
    a = outs[b];
    h = T[b].H2;
    w = T[b].W2;
  }
  free(stem_out);
  /* outs[0..5] hold the block outputs (post ECA, post skip); a == outs[5] */
  double* zl = malloc(sizeof(double) * n);
  orc_conv2d(a, 8, H, W, net->out_w, net->out_b, 1, 3, 1, 1, 1, zl);
  /* output: z = sigmoid(zl) */
  double* dzl = malloc(sizeof(double) * n);
  for (size_t t = 0; t < n; ++t) {
    double z = 1.0 / (1.0 + exp(-zl[t]));
    dzl[t] = gout[t] * z * (1.0 - z);
  }
  double* dcur = calloc(8 * n, sizeof(double));
  conv2d_bwd(a, 8, H, W, net->out_w, 1, 3, 1, 1, 1, dzl, dcur, gout_w, gout_b);
  free(zl); free(dzl);
  /* blocks in reverse; skip sources collect extra gradient */
  double* dskip[2] = {calloc((size_t)16 * (H / 2) * (W / 2), sizeof(double)),
                      calloc((size_t)32 * (H / 4) * (W / 4), sizeof(double))};
  for (int b = 5; b >= 0; --b) {
    size_t osz = (size_t)net->blk[b].cout * T[b].H2 * T[b].W2;
    if (b == 0 || b == 1)
      for (size_t t = 0; t < osz; ++t) dcur[t] += dskip[b][t];
    if (b == 3 || b == 4)
      for (size_t t = 0; t < osz; ++t) dskip[4 - b][t] += dcur[t];
    size_t isz = (size_t)net->blk[b].cin * T[b].h * T[b].w;
    double* dx = calloc(isz, sizeof(double));
    block_backward(&net->blk[b], &T[b], dcur, dx, &G[b]);
    free(dcur);
    dcur = dx;
  }
  /* stem: a0 = ReLU(BN(su)) */
  for (size_t t = 0; t < 8 * n; ++t)
    if (T[0].x[t] <= 0.0) dcur[t] = 0.0;
  double* dsu = calloc(8 * n, sizeof(double));
  batchnorm_bwd(su, 8, (int)n, net->stem_g, net->stem_m, net->stem_v, dcur, dsu, gstem_g, gstem_b);
  conv2d_bwd(x, 3, H, W, net->stem_w, 8, 3, 1, 1, 1, dsu, gin, gstem_w, NULL);
  free(dsu); free(dcur); free(su); free(x);
  for (int b = 0; b < 6; ++b) {
    tape_free(&T[b]);
    free(outs[b]);
  }
  free(dskip[0]);
  free(dskip[1]);
  return 0;
}

int orc_adjoint(const float* params, const float* buffers, const float* in, const double* gout, int H, int W,
                double* gparams, double* gin) {
  orc_net net;
  net_load(&net, params, buffers);
  memset(gparams, 0, sizeof(double) * orc_num_params());
  if (gin) memset(gin, 0, sizeof(double) * 3 * H * W);
  int rc = adjoint_one(&net, in, gout, H, W, gparams, gin);
  net_free(&net);
  return rc;
}

typedef struct {
  const orc_net* net;
  const float *in, *target;
  int B, H, W, tid, nt, rc;
  double loss;
  double* gp;
} grad_job;

static void* grad_worker(void* arg) {
  grad_job* j = (grad_job*)arg;
  size_t n = (size_t)j->H * j->W;
  double* z = malloc(sizeof(double) * n);
  double* gz = malloc(sizeof(double) * n);
  double N = (double)j->B * (double)n;
  for (int b = j->tid; b < j->B; b += j->nt) {
    int rc = forward_one(j->net, j->in + (size_t)b * 3 * n, j->H, j->W, z, NULL);
    if (rc) { j->rc = rc; continue; }
    for (size_t t = 0; t < n; ++t) {
      double e = z[t] - (double)j->target[(size_t)b * n + t];
      j->loss += e * e / N;
      gz[t] = 2.0 * e / N;
    }
    rc = adjoint_one(j->net, j->in + (size_t)b * 3 * n, gz, j->H, j->W, j->gp, NULL);
    if (rc) j->rc = rc;
  }
  free(z);
  free(gz);
  return NULL;
}

/* Mean squared error over B windows against the clean maps, and its
 * gradient with respect to every parameter (canonical order). Threads
 * accumulate into private buffers that are summed in a fixed order. */
double orc_loss_grad(const float* params, const float* buffers, const float* in, const float* target, int B,
                     int H, int W, double* gparams, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > B) nthreads = B;
  if (nthreads > 256) nthreads = 256;
  orc_net net;
  net_load(&net, params, buffers);
  int np = orc_num_params();
  pthread_t th[256];
  grad_job jobs[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = (grad_job){&net, in, target, B, H, W, t, nthreads, 0, 0.0, calloc(np, sizeof(double))};
    pthread_create(&th[t], NULL, grad_worker, &jobs[t]);
  }
  double loss = 0.0;
  memset(gparams, 0, sizeof(double) * np);
  int rc = 0;
  for (int t = 0; t < nthreads; ++t) {
    pthread_join(th[t], NULL);
    loss += jobs[t].loss;
    for (int i = 0; i < np; ++i) gparams[i] += jobs[t].gp[i];
    free(jobs[t].gp);
    if (jobs[t].rc) rc = jobs[t].rc;
  }
  net_free(&net);
  return rc ? NAN : loss;
}

/* ======================================================================== */
/* Training-mode BatchNorm (batch statistics), FP64.                        */
/* ======================================================================== */

/* In training mode a BN normalises with the mean and the biased variance of
 * its input over the whole batch (every window and pixel of a channel), so
 * each window's forward pass and adjoint depend on all the others. The
 * batch network below holds every layer's tensors for all B windows
 * ([B][C][n]) and takes the convolutions window by window with the
 * primitives above. mode 0 normalises with the running statistics instead
 * and then computes the same loss and gradient as orc_loss_grad. */

/* Per-channel mean and biased variance of x[B][C][n] (two passes). */
static void bnb_stats(const double* x, int B, int C, size_t n, double* mean, double* var) {
  double N = (double)B * (double)n;
  for (int c = 0; c < C; ++c) {
    double s = 0.0;
    for (int b = 0; b < B; ++b)
      for (size_t t = 0; t < n; ++t) s += x[((size_t)b * C + c) * n + t];
    double m = s / N, q = 0.0;
    for (int b = 0; b < B; ++b)
      for (size_t t = 0; t < n; ++t) {
        double d = x[((size_t)b * C + c) * n + t] - m;
        q += d * d;
      }
    mean[c] = m;
    var[c] = q / N;
  }
}

/* One BN on x[B][C][n] in place. The statistics it normalises with go to
 * mean / var: the batch's (mode 1) or the running ones (mode 0). */
static void bnb_forward(double* x, int B, int C, size_t n, const double* gam, const double* bet,
                        const double* rmean, const double* rvar, int mode, double* mean, double* var) {
  if (mode) {
    bnb_stats(x, B, C, n, mean, var);
  } else {
    memcpy(mean, rmean, sizeof(double) * C);
    memcpy(var, rvar, sizeof(double) * C);
  }
  for (int b = 0; b < B; ++b)
    for (int c = 0; c < C; ++c) {
      double sc = gam[c] / sqrt(var[c] + BN_EPS);
      double* p = x + ((size_t)b * C + c) * n;
      for (size_t t = 0; t < n; ++t) p[t] = sc * (p[t] - mean[c]) + bet[c];
    }
}

/* Adjoint of one BN given its input x and the statistics it used: dgam +=
 * sum dy xhat, dbet += sum dy, dx += gam / sigma (dy - [sum dy + xhat sum dy
 * xhat] / N), the bracket only with batch statistics (mode 1), where the
 * mean and variance are functions of x. */
static void bnb_backward(const double* x, int B, int C, size_t n, const double* gam, const double* mean,
                         const double* var, const double* dy, double* dx, double* dgam, double* dbet, int mode) {
  double N = (double)B * (double)n;
  for (int c = 0; c < C; ++c) {
    double is = 1.0 / sqrt(var[c] + BN_EPS), sdy = 0.0, sdx = 0.0;
    for (int b = 0; b < B; ++b)
      for (size_t t = 0; t < n; ++t) {
        size_t i = ((size_t)b * C + c) * n + t;
        sdy += dy[i];
        sdx += dy[i] * (x[i] - mean[c]) * is;
      }
    dgam[c] += sdx;
    dbet[c] += sdy;
    if (!dx) continue;
    for (int b = 0; b < B; ++b)
      for (size_t t = 0; t < n; ++t) {
        size_t i = ((size_t)b * C + c) * n + t;
        double d = dy[i];
        if (mode) d -= (sdy + (x[i] - mean[c]) * is * sdx) / N;
        dx[i] += gam[c] * is * d;
      }
  }
}

/* Saved tensors of one block for all windows, and the statistics each BN
 * used (m1, v1: BN1 ... m, v: main BN). */
typedef struct {
  int h, w, H2, W2;
  double *x, *t1, *t2, *x1, *u, *y, *g, *s;
  double *m1, *v1, *m2, *v2, *m3, *v3, *m, *v;
} bblk_tape;

static void conv_batch(int tr, const double* x, int B, int Ci, int H, int W, const double* w, const double* bias,
                       int Co, int k, int stride, int pad, int groups, double* y, int Ho, int Wo) {
  for (int b = 0; b < B; ++b) {
    const double* xb = x + (size_t)b * Ci * H * W;
    double* yb = y + (size_t)b * Co * Ho * Wo;
    if (tr)
      orc_conv_transpose2d(xb, Ci, H, W, w, bias, Co, k, stride, pad, groups, yb);
    else
      orc_conv2d(xb, Ci, H, W, w, bias, Co, k, stride, pad, groups, yb);
  }
}

static void conv_batch_bwd(int tr, const double* x, int B, int Ci, int H, int W, const double* w, int Co, int k,
                           int stride, int pad, int groups, const double* dy, double* dx, double* dw, double* db,
                           int Ho, int Wo) {
  for (int b = 0; b < B; ++b) {
    const double* xb = x + (size_t)b * Ci * H * W;
    const double* dyb = dy + (size_t)b * Co * Ho * Wo;
    double* dxb = dx ? dx + (size_t)b * Ci * H * W : NULL;
    if (tr)
      conv_transpose2d_bwd(xb, Ci, H, W, w, Co, k, stride, pad, groups, dyb, dxb, dw, db);
    else
      conv2d_bwd(xb, Ci, H, W, w, Co, k, stride, pad, groups, dyb, dxb, dw, db);
  }
}

/* Block forward over the batch (the arithmetic of block_forward_tape). */
static double* bblk_forward(const orc_blk* k, const double* x, int B, int h, int w, int mode, bblk_tape* T) {
  int ci = k->cin, co = k->cout, tr = !k->enc;
  size_t n = (size_t)h * w, sz = (size_t)B * ci * n;
  T->h = h;
  T->w = w;
  T->H2 = k->enc ? h / 2 : 2 * h;
  T->W2 = k->enc ? w / 2 : 2 * w;
  size_t n2 = (size_t)T->H2 * T->W2, sz2 = (size_t)B * co * n2;
  T->m1 = malloc(sizeof(double) * ci); T->v1 = malloc(sizeof(double) * ci);
  T->m2 = malloc(sizeof(double) * ci); T->v2 = malloc(sizeof(double) * ci);
  T->m3 = malloc(sizeof(double) * ci); T->v3 = malloc(sizeof(double) * ci);
  T->m = malloc(sizeof(double) * co); T->v = malloc(sizeof(double) * co);
  T->x = dup(x, sz);
  T->t1 = malloc(sizeof(double) * sz);
  T->t2 = malloc(sizeof(double) * sz);
  conv_batch(tr, x, B, ci, h, w, k->w1, NULL, ci, 1, 1, 0, ci, T->t1, h, w);
  conv_batch(tr, x, B, ci, h, w, k->w3, NULL, ci, 3, 1, 1, ci, T->t2, h, w);
  double* b1 = dup(T->t1, sz);
  double* b2 = dup(T->t2, sz);
  double* b3 = dup(x, sz);
  bnb_forward(b1, B, ci, n, k->g1, k->b1, k->m1, k->v1, mode, T->m1, T->v1);
  bnb_forward(b2, B, ci, n, k->g2, k->b2, k->m2, k->v2, mode, T->m2, T->v2);
  bnb_forward(b3, B, ci, n, k->g3, k->b3, k->m3, k->v3, mode, T->m3, T->v3);
  T->x1 = malloc(sizeof(double) * sz);
  for (size_t t = 0; t < sz; ++t) T->x1[t] = b1[t] + b2[t] + b3[t];
  relu(T->x1, sz);
  free(b1); free(b2); free(b3);
  T->u = malloc(sizeof(double) * sz2);
  double* rs = malloc(sizeof(double) * sz2);
  conv_batch(tr, T->x1, B, ci, h, w, k->w2, NULL, co, k->enc ? 3 : 4, 2, 1, 1, T->u, T->H2, T->W2);
  conv_batch(tr, x, B, ci, h, w, k->rw, k->rb, co, k->enc ? 3 : 4, 2, 1, 1, rs, T->H2, T->W2);
  T->y = dup(T->u, sz2);
  bnb_forward(T->y, B, co, n2, k->g, k->b, k->m, k->v, mode, T->m, T->v);
  relu(T->y, sz2);
  for (size_t t = 0; t < sz2; ++t) T->y[t] += rs[t];
  free(rs);
  /* ECA per window */
  T->g = malloc(sizeof(double) * B * co);
  T->s = malloc(sizeof(double) * B * co);
  double* out = malloc(sizeof(double) * sz2);
  for (int b = 0; b < B; ++b) {
    const double* yb = T->y + (size_t)b * co * n2;
    double *g = T->g + (size_t)b * co, *sc = T->s + (size_t)b * co;
    for (int c = 0; c < co; ++c) {
      double a = 0.0;
      for (size_t t = 0; t < n2; ++t) a += yb[c * n2 + t];
      g[c] = a / (double)n2;
    }
    for (int c = 0; c < co; ++c) {
      double z = 0.0;
      for (int j = 0; j < 3; ++j) {
        int cc = c + j - 1;
        if (cc >= 0 && cc < co) z += k->eca[j] * g[cc];
      }
      sc[c] = 1.0 / (1.0 + exp(-z));
      for (size_t t = 0; t < n2; ++t) out[(size_t)b * co * n2 + c * n2 + t] = sc[c] * yb[c * n2 + t];
    }
  }
  return out;
}

/* Block adjoint over the batch (the arithmetic of block_backward, with the
 * batch-statistics BN adjoint when mode is 1). dx accumulates. */
static void bblk_backward(const orc_blk* k, const bblk_tape* T, int B, const double* dout, double* dx, blk_grad* G,
                          int mode) {
  int ci = k->cin, co = k->cout, h = T->h, w = T->w, H2 = T->H2, W2 = T->W2, tr = !k->enc;
  size_t n = (size_t)h * w, n2 = (size_t)H2 * W2, sz = (size_t)B * ci * n, sz2 = (size_t)B * co * n2;
  double* dy = malloc(sizeof(double) * sz2);
  for (int b = 0; b < B; ++b) {
    const double* ob = dout + (size_t)b * co * n2;
    const double* yb = T->y + (size_t)b * co * n2;
    const double *g = T->g + (size_t)b * co, *sc = T->s + (size_t)b * co;
    double* dyb = dy + (size_t)b * co * n2;
    double* dz = calloc(co, sizeof(double));
    for (int c = 0; c < co; ++c) {
      double ds = 0.0;
      for (size_t t = 0; t < n2; ++t) {
        ds += ob[c * n2 + t] * yb[c * n2 + t];
        dyb[c * n2 + t] = sc[c] * ob[c * n2 + t];
      }
      dz[c] = ds * sc[c] * (1.0 - sc[c]);
    }
    for (int c = 0; c < co; ++c)
      for (int j = 0; j < 3; ++j) {
        int cc = c + j - 1;
        if (cc < 0 || cc >= co) continue;
        G->eca[j] += dz[c] * g[cc];
        double dg = dz[c] * k->eca[j] / (double)n2;
        for (size_t t = 0; t < n2; ++t) dyb[cc * n2 + t] += dg;
      }
    free(dz);
  }
  /* y = ReLU(BN(u)) + res(x) */
  double* dbn = malloc(sizeof(double) * sz2);
  for (int b = 0; b < B; ++b)
    for (int c = 0; c < co; ++c) {
      double is = 1.0 / sqrt(T->v[c] + BN_EPS);
      for (size_t t = 0; t < n2; ++t) {
        size_t i = ((size_t)b * co + c) * n2 + t;
        double bn = k->g[c] * (T->u[i] - T->m[c]) * is + k->b[c];
        dbn[i] = bn > 0.0 ? dy[i] : 0.0;
      }
    }
  double* du = calloc(sz2, sizeof(double));
  bnb_backward(T->u, B, co, n2, k->g, T->m, T->v, dbn, du, G->g, G->b, mode);
  free(dbn);
  double* dx1 = calloc(sz, sizeof(double));
  int kk = k->enc ? 3 : 4;
  conv_batch_bwd(tr, T->x1, B, ci, h, w, k->w2, co, kk, 2, 1, 1, du, dx1, G->w2, NULL, H2, W2);
  conv_batch_bwd(tr, T->x, B, ci, h, w, k->rw, co, kk, 2, 1, 1, dy, dx, G->rw, G->rb, H2, W2);
  free(du);
  free(dy);
  /* x1 = ReLU(BN1(t1) + BN2(t2) + BN3(x)) */
  for (size_t t = 0; t < sz; ++t)
    if (T->x1[t] <= 0.0) dx1[t] = 0.0;
  double* dt1 = calloc(sz, sizeof(double));
  double* dt2 = calloc(sz, sizeof(double));
  bnb_backward(T->t1, B, ci, n, k->g1, T->m1, T->v1, dx1, dt1, G->g1, G->b1, mode);
  bnb_backward(T->t2, B, ci, n, k->g2, T->m2, T->v2, dx1, dt2, G->g2, G->b2, mode);
  bnb_backward(T->x, B, ci, n, k->g3, T->m3, T->v3, dx1, dx, G->g3, G->b3, mode);
  conv_batch_bwd(tr, T->x, B, ci, h, w, k->w1, ci, 1, 1, 0, ci, dt1, dx, G->w1, NULL, h, w);
  conv_batch_bwd(tr, T->x, B, ci, h, w, k->w3, ci, 3, 1, 1, ci, dt2, dx, G->w3, NULL, h, w);
  free(dt1); free(dt2); free(dx1);
}

static void bblk_free(bblk_tape* T) {
  free(T->x); free(T->t1); free(T->t2); free(T->x1); free(T->u); free(T->y); free(T->g); free(T->s);
  free(T->m1); free(T->v1); free(T->m2); free(T->v2); free(T->m3); free(T->v3); free(T->m); free(T->v);
}

/* Gradient pointers mirroring the canonical parameter layout. */
static double* grad_layout(double* q, blk_grad* G) {
  q += 232; /* stem W, gamma, beta */
  for (int b = 0; b < 6; ++b) {
    int ci = BLK_CIN[b], co = blk_cout(b);
    G[b].w1 = q; q += ci;
    G[b].g1 = q; q += ci;
    G[b].b1 = q; q += ci;
    G[b].w3 = q; q += 9 * ci;
    G[b].g2 = q; q += ci;
    G[b].b2 = q; q += ci;
    G[b].g3 = q; q += ci;
    G[b].b3 = q; q += ci;
    G[b].w2 = q; q += blk_dense(b);
    G[b].g = q; q += co;
    G[b].b = q; q += co;
    G[b].rw = q; q += blk_dense(b);
    G[b].rb = q; q += co;
    G[b].eca = q; q += 3;
  }
  return q; /* output conv W, b */
}

/* MSE training loss over B windows against the targets and its gradient
 * (canonical order) with BN in training mode (mode 1: batch statistics) or
 * inference mode (mode 0: running statistics). stats (optional) receives,
 * in the order and layout of the BN buffers, the mean and variance each BN
 * normalised with (mode 1: the batch's, biased). Returns NAN on a bad
 * shape. */
double orc_loss_grad_bn(const float* params, const float* buffers, const float* in, const float* target, int B,
                        int H, int W, int mode, double* gparams, double* stats) {
  if (B < 1 || H <= 0 || W <= 0 || H % 8 || W % 8) return NAN;
  orc_net net;
  net_load(&net, params, buffers);
  int np = orc_num_params();
  memset(gparams, 0, sizeof(double) * np);
  blk_grad G[6];
  double* gout_w = grad_layout(gparams, G);
  double *gout_b = gout_w + 72, *gstem_w = gparams, *gstem_g = gparams + 216, *gstem_b = gparams + 224;
  size_t n = (size_t)H * W;
  double* x = malloc(sizeof(double) * B * 3 * n);
  for (size_t t = 0; t < (size_t)B * 3 * n; ++t) x[t] = (double)in[t];
  double* su = malloc(sizeof(double) * B * 8 * n);
  conv_batch(0, x, B, 3, H, W, net.stem_w, NULL, 8, 3, 1, 1, 1, su, H, W);
  double sm[8], sv[8];
  double* a0 = dup(su, (size_t)B * 8 * n);
  bnb_forward(a0, B, 8, n, net.stem_g, net.stem_b, net.stem_m, net.stem_v, mode, sm, sv);
  relu(a0, (size_t)B * 8 * n);
  bblk_tape T[6];
  double* outs[6];
  const double* a = a0;
  int h = H, w = W;
  for (int b = 0; b < 6; ++b) {
    outs[b] = bblk_forward(&net.blk[b], a, B, h, w, mode, &T[b]);
    size_t sz = (size_t)B * net.blk[b].cout * T[b].H2 * T[b].W2;
    if (b == 3 || b == 4) {
      const double* s = outs[4 - b];
      for (size_t t = 0; t < sz; ++t) outs[b][t] += s[t];
    }
    a = outs[b];
    h = T[b].H2;
    w = T[b].W2;
  }
  /* output conv, sigmoid, MSE */
  double* zl = malloc(sizeof(double) * B * n);
  conv_batch(0, a, B, 8, H, W, net.out_w, net.out_b, 1, 3, 1, 1, 1, zl, H, W);
  double loss = 0.0, N = (double)B * (double)n;
  double* dzl = malloc(sizeof(double) * B * n);
  for (size_t t = 0; t < (size_t)B * n; ++t) {
    double z = 1.0 / (1.0 + exp(-zl[t])), e = z - (double)target[t];
    loss += e * e / N;
    dzl[t] = 2.0 * e / N * z * (1.0 - z);
  }
  double* dcur = calloc((size_t)B * 8 * n, sizeof(double));
  conv_batch_bwd(0, a, B, 8, H, W, net.out_w, 1, 3, 1, 1, 1, dzl, dcur, gout_w, gout_b, H, W);
  free(zl);
  free(dzl);
  double* dskip[2] = {calloc((size_t)B * 16 * (H / 2) * (W / 2), sizeof(double)),
                      calloc((size_t)B * 32 * (H / 4) * (W / 4), sizeof(double))};
  for (int b = 5; b >= 0; --b) {
    size_t osz = (size_t)B * net.blk[b].cout * T[b].H2 * T[b].W2;
    if (b == 0 || b == 1)
      for (size_t t = 0; t < osz; ++t) dcur[t] += dskip[b][t];
    if (b == 3 || b == 4)
      for (size_t t = 0; t < osz; ++t) dskip[4 - b][t] += dcur[t];
    double* dx = calloc((size_t)B * net.blk[b].cin * T[b].h * T[b].w, sizeof(double));
    bblk_backward(&net.blk[b], &T[b], B, dcur, dx, &G[b], mode);
    free(dcur);
    dcur = dx;
  }
  /* stem: a0 = ReLU(BN(su)) */
  for (size_t t = 0; t < (size_t)B * 8 * n; ++t)
    if (a0[t] <= 0.0) dcur[t] = 0.0;
  double* dsu = calloc((size_t)B * 8 * n, sizeof(double));
  bnb_backward(su, B, 8, n, net.stem_g, sm, sv, dcur, dsu, gstem_g, gstem_b, mode);
  conv_batch_bwd(0, x, B, 3, H, W, net.stem_w, 8, 3, 1, 1, 1, dsu, NULL, gstem_w, NULL, H, W);
  if (stats) {
    double* q = stats;
    memcpy(q, sm, sizeof(sm)); q += 8;
    memcpy(q, sv, sizeof(sv)); q += 8;
    for (int b = 0; b < 6; ++b) {
      int ci = BLK_CIN[b], co = blk_cout(b);
      const double* mv[8] = {T[b].m1, T[b].v1, T[b].m2, T[b].v2, T[b].m3, T[b].v3, T[b].m, T[b].v};
      for (int j = 0; j < 8; ++j) {
        int c = j < 6 ? ci : co;
        memcpy(q, mv[j], sizeof(double) * c);
        q += c;
      }
    }
  }
  free(dsu); free(dcur); free(su); free(a0); free(x);
  for (int b = 0; b < 6; ++b) {
    bblk_free(&T[b]);
    free(outs[b]);
  }
  free(dskip[0]);
  free(dskip[1]);
  net_free(&net);
  return loss;
}

/* ======================================================================== */
/* Metrics (Sec. V-B).                                                      */
/* ======================================================================== */

/* Eq. (SINR): 10 log10 of the mean power over the target-peak cells O
 * divided by the mean power over the noise cells N. Reading: O = the
 * distinct closed-form peak cells; N = every cell outside a (2 guard + 1)^2
 * box around each O cell; the map value itself is the magnitude. */
double orc_sinr_db(const double* z, int P, int Q, const int* bins, int nb,
                   int guard) {
  char* mask = calloc((size_t)P * Q, 1); /* 1 = peak, 2 = guard */
  for (int o = 0; o < nb; ++o) {
    int p = bins[2 * o], q = bins[2 * o + 1];
    for (int dp = -guard; dp <= guard; ++dp)
      for (int dq = -guard; dq <= guard; ++dq) {
        int pp = p + dp, qq = q + dq;
        if (pp < 0 || pp >= P || qq < 0 || qq >= Q) continue;
        if (mask[pp * Q + qq] == 0) mask[pp * Q + qq] = 2;
      }
  }
  for (int o = 0; o < nb; ++o) mask[bins[2 * o] * Q + bins[2 * o + 1]] = 1;
  double so = 0.0, sn = 0.0;
  long no = 0, nn = 0;
  for (int i = 0; i < P * Q; ++i) {
    double e = z[i] * z[i];
    if (mask[i] == 1) { so += e; ++no; }
    else if (mask[i] == 0) { sn += e; ++nn; }
  }
  free(mask);
  if (no == 0 || nn == 0) return NAN;
  return 10.0 * log10((so / (double)no) / (sn / (double)nn));
}

/* Eq. (EVM): mean over the distinct peak cells of |clean - est| / |clean|. */
double orc_evm(const double* clean, const double* est, int P, int Q,
               const int* bins, int nb) {
  char* seen = calloc((size_t)P * Q, 1);
  double s = 0.0;
  int cnt = 0;
  for (int o = 0; o < nb; ++o) {
    int i = bins[2 * o] * Q + bins[2 * o + 1];
    if (seen[i]) continue;
    seen[i] = 1;
    s += fabs(clean[i] - est[i]) / fabs(clean[i]);
    ++cnt;
  }
  free(seen);
  return cnt ? s / cnt : NAN;
}

/* Cell-averaging CFAR (Sec. V-B: CA-CFAR as the peak detector on RD maps).
 * Reading: the cell power is z^2 (as in Eq. (SINR)); the cell under test is
 * compared with the mean power of the training cells, i.e. the cells of the
 * (2 (guard + train) + 1)^2 square around it minus the (2 guard + 1)^2 guard
 * square, clipped at the map edge; detection when
 * z^2 > alpha * mean, alpha = N (pfa^(-1/N) - 1) for N training cells (the
 * textbook CA-CFAR factor for exponentially distributed noise power). */
int orc_cacfar(const double* z, int P, int Q, int guard, int train, double pfa, unsigned char* det) {
  int count = 0;
  int R = guard + train;
  for (int p = 0; p < P; ++p)
    for (int q = 0; q < Q; ++q) {
      double s = 0.0;
      int n = 0;
      for (int dp = -R; dp <= R; ++dp)
        for (int dq = -R; dq <= R; ++dq) {
          if (dp >= -guard && dp <= guard && dq >= -guard && dq <= guard) continue;
          int pp = p + dp, qq = q + dq;
          if (pp < 0 || pp >= P || qq < 0 || qq >= Q) continue;
          s += z[pp * Q + qq] * z[pp * Q + qq];
          ++n;
        }
      double alpha = (double)n * (pow(pfa, -1.0 / (double)n) - 1.0);
      double c = z[p * Q + q] * z[p * Q + q];
      unsigned char d = n > 0 && c > alpha * (s / (double)n);
      det[p * Q + q] = d;
      count += d;
    }
  return count;
}

/* Fraction of distinct target cells with a detection within +-1 cell
 * (Sec. V-B: AP = N_cd / N, without the clustering step). */
double orc_detect_rate(const unsigned char* det, int P, int Q, const int* bins, int nb) {
  int hit = 0, cnt = 0;
  for (int o = 0; o < nb; ++o) {
    int dup = 0;
    for (int k = 0; k < o; ++k) dup |= bins[2 * k] == bins[2 * o] && bins[2 * k + 1] == bins[2 * o + 1];
    if (dup) continue;
    ++cnt;
    int found = 0;
    for (int dp = -1; dp <= 1; ++dp)
      for (int dq = -1; dq <= 1; ++dq) {
        int pp = bins[2 * o] + dp, qq = bins[2 * o + 1] + dq;
        if (pp >= 0 && pp < P && qq >= 0 && qq < Q && det[pp * Q + qq]) found = 1;
      }
    hit += found;
  }
  return cnt ? (double)hit / cnt : NAN;
}
