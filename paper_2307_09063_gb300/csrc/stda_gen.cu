// Synthetic range-Doppler windows on the GPU (Sec. III), in FP64.
//
//  1. k_scene: one thread per window draws the scene from a SplitMix64 hash
//     keyed by (seed, workload, window, tag, i1, i2): point targets (range
//     bin r, Doppler bin d, per-frame phase), per-frame interferers (slope
//     ratio, crossing sample, power) and the noise level. Every quantity
//     that decides an integer (counts, peak bins) is computed with
//     explicitly rounded FP64 operations, never contracted into an FMA.
//  2. k_signal: one thread per (map, n, m) evaluates Eq. "IF signal" (sum of
//     Eq. "discrete signal" targets, dechirped interferer bursts inside the
//     IF band, complex Gaussian noise by Box-Muller) times the Hann windows.
//     Maps 0..2 are frames t, t-1, t-2; map 3 is the interference-free frame t.
//  3. k_fft_range / k_fft_doppler: radix-2 FFTs in shared memory (Eqs.
//     "column transform", "row transform"), zero padded to P x Q, Doppler
//     axis shifted by Q/2.
//  4. k_lognorm: 20 log10 magnitude, min-max normalised per map.
#include <cuda_bf16.h>

#include "stda_internal.h"

namespace stda {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxTgt = 16, kMaxInt = 4;

enum : uint64_t {
  TAG_TGT_COUNT = 1, TAG_TGT_R = 2, TAG_TGT_D = 3, TAG_TGT_PHASE = 4, TAG_INT_COUNT = 5,
  TAG_INT_KAPPA = 6, TAG_INT_NX = 7, TAG_INT_INR = 8, TAG_INT_PHASE = 9, TAG_SNR = 10, TAG_NOISE = 11
};

struct Scene {
  int n_tgt;
  int n_int[3];
  double r[kMaxTgt], d[kMaxTgt], delta[kMaxTgt], phase[3][kMaxTgt];
  double kappa[3][kMaxInt], nx[3][kMaxInt], amp[3][kMaxInt];
  double sigma;
};

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}

struct Keyer {
  uint64_t base;  // hash of (seed, workload, window)
  __device__ Keyer(uint64_t seed, uint64_t cid, uint64_t w) { base = mix64(mix64(mix64(seed) ^ cid) ^ w); }
  __device__ double u(uint64_t tag, uint64_t i1, uint64_t i2) const {
    uint64_t h = mix64(mix64(mix64(base ^ tag) ^ i1) ^ i2);
    return (double)(h >> 11) * (1.0 / 9007199254740992.0);
  }
};

__device__ __forceinline__ int uniform_int(int lo, int hi, double u) {
  return lo + (int)floor(__dmul_rn(u, (double)(hi - lo + 1)));
}

__device__ __forceinline__ int wrap(long long a, int m) {
  long long r = a % m;
  return (int)(r < 0 ? r + m : r);
}

struct GenParams {
  int N, M, P, Q, logP, logQ;
  int tmin, tmax, imin, imax;
  double snr_min, snr_max, inr_min, inr_max, kmin, kmax;
  double drift;   // range bins per frame per Doppler bin
  double a_ts2;   // victim slope * Ts^2 [cycles / sample^2]
};

__global__ void k_scene(GenParams g, uint64_t seed, uint64_t cid, int w0, int B, Scene* sc, int* bins,
                        int* ntgt) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  Keyer k(seed, cid, (uint64_t)(w0 + b));
  Scene s;
  s.n_tgt = uniform_int(g.tmin, g.tmax, k.u(TAG_TGT_COUNT, 0, 0));
  for (int o = 0; o < kMaxTgt; ++o) {
    s.r[o] = s.d[o] = s.delta[o] = 0.0;
    for (int f = 0; f < 3; ++f) s.phase[f][o] = 0.0;
  }
  for (int o = 0; o < s.n_tgt; ++o) {
    s.r[o] = __dadd_rn(2.0, __dmul_rn((double)(g.N - 4), k.u(TAG_TGT_R, o, 0)));
    s.d[o] = __dadd_rn((double)(-g.M / 2 + 1), __dmul_rn((double)(g.M - 2), k.u(TAG_TGT_D, o, 0)));
    s.delta[o] = s.d[o] * g.drift;
    for (int f = 0; f < 3; ++f) s.phase[f][o] = 2.0 * kPi * k.u(TAG_TGT_PHASE, o, f);
    // frame-t peak cell (Sec. III-B): range bin r P / N, Doppler bin d Q / M
    double pr = __ddiv_rn(__dmul_rn(s.r[o], (double)g.P), (double)g.N);
    double qd = __ddiv_rn(__dmul_rn(s.d[o], (double)g.Q), (double)g.M);
    long long p = (long long)floor(__dadd_rn(pr, 0.5));
    long long q = (long long)floor(__dadd_rn(qd, 0.5));
    if (bins) {
      bins[(b * kMaxTgt + o) * 2] = wrap(p, g.P);
      bins[(b * kMaxTgt + o) * 2 + 1] = wrap((long long)wrap(q, g.Q) + g.Q / 2, g.Q);
    }
  }
  if (bins)
    for (int o = s.n_tgt; o < kMaxTgt; ++o) bins[(b * kMaxTgt + o) * 2] = bins[(b * kMaxTgt + o) * 2 + 1] = -1;
  for (int f = 0; f < 3; ++f) {
    s.n_int[f] = uniform_int(g.imin, g.imax, k.u(TAG_INT_COUNT, f, 0));
    for (int i = 0; i < kMaxInt; ++i) s.kappa[f][i] = s.nx[f][i] = s.amp[f][i] = 0.0;
    for (int i = 0; i < s.n_int[f]; ++i) {
      s.kappa[f][i] = g.kmin + (g.kmax - g.kmin) * k.u(TAG_INT_KAPPA, f, i);
      s.nx[f][i] = (double)g.N * k.u(TAG_INT_NX, f, i);
      double inr = g.inr_min + (g.inr_max - g.inr_min) * k.u(TAG_INT_INR, f, i);
      s.amp[f][i] = pow(10.0, inr / 20.0);
    }
  }
  double snr = g.snr_min + (g.snr_max - g.snr_min) * k.u(TAG_SNR, 0, 0);
  s.sigma = pow(10.0, -snr / 20.0);
  sc[b] = s;
  if (ntgt) ntgt[b] = s.n_tgt;
}

__device__ __forceinline__ double hann(int n, int N) {
  return N == 1 ? 1.0 : 0.5 - 0.5 * cos(2.0 * kPi * (double)n / (double)(N - 1));
}

// X: [B][4][P][Q] complex (row = fast-time sample n, column = chirp m),
// zero where n >= N or m >= M (the caller clears it first).
__global__ void k_signal(GenParams g, uint64_t seed, uint64_t cid, int w0, const Scene* sc, double2* X) {
  int bm = blockIdx.y;  // window * 4 + map
  int b = bm >> 2, map = bm & 3;
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.N * g.M) return;
  int n = idx / g.M, m = idx % g.M;
  const Scene& s = sc[b];
  int f = map < 3 ? map : 0;
  bool with_int = map < 3;
  Keyer k(seed, cid, (uint64_t)(w0 + b));
  double re = 0.0, im = 0.0;
  for (int o = 0; o < s.n_tgt; ++o) {
    double rf = s.r[o] - (double)f * s.delta[o];
    double ph = 2.0 * kPi * (rf * (double)n / (double)g.N + s.d[o] * (double)m / (double)g.M) + s.phase[f][o];
    double sn, cs;
    sincos(ph, &sn, &cs);
    re += cs;
    im += sn;
  }
  if (with_int) {
    for (int i = 0; i < s.n_int[f]; ++i) {
      double gm = (s.kappa[f][i] - 1.0) * g.a_ts2;
      double x = (double)n - s.nx[f][i];
      if (fabs(gm * x) <= 0.5) {
        double ph = kPi * gm * x * x + 2.0 * kPi * k.u(TAG_INT_PHASE, f, (uint64_t)(i * g.M + m));
        double sn, cs;
        sincos(ph, &sn, &cs);
        re += s.amp[f][i] * cs;
        im += s.amp[f][i] * sn;
      }
    }
  }
  uint64_t kk = (uint64_t)n * (uint64_t)g.M + (uint64_t)m;
  double u1 = 1.0 - k.u(TAG_NOISE, f, 2 * kk);
  double u2 = k.u(TAG_NOISE, f, 2 * kk + 1);
  double rad = sqrt(-2.0 * log(u1)) * s.sigma * sqrt(0.5);
  double sn, cs;
  sincos(2.0 * kPi * u2, &sn, &cs);
  re += rad * cs;
  im += rad * sn;
  double wgt = hann(n, g.N) * hann(m, g.M);
  X[((size_t)bm * g.P + n) * g.Q + m] = make_double2(re * wgt, im * wgt);
}

// In-place radix-2 decimation-in-time FFT (forward, e^{-j...}) of nseq
// sequences of length L = 2^logL, stored one after another in shared memory
// in bit-reversed order.
__device__ void fft_stages(double2* x, int nseq, int L) {
  for (int half = 1; half < L; half <<= 1) {
    for (int j = threadIdx.x; j < nseq * (L / 2); j += blockDim.x) {
      int s = j / (L / 2), k = j % (L / 2);
      int pos = k % half, i0 = (k / half) * 2 * half + pos, i1 = i0 + half;
      double sn, cs;
      sincospi((double)pos / (double)half, &sn, &cs);
      double2 a = x[s * L + i0], c = x[s * L + i1];
      double2 t = make_double2(c.x * cs + c.y * sn, c.y * cs - c.x * sn);
      x[s * L + i0] = make_double2(a.x + t.x, a.y + t.y);
      x[s * L + i1] = make_double2(a.x - t.x, a.y - t.y);
    }
    __syncthreads();
  }
}

constexpr int kFftCols = 4;

__global__ void k_fft_range(GenParams g, double2* X) {
  extern __shared__ double2 buf[];  // [kFftCols][P]
  double2* base = X + (size_t)blockIdx.y * g.P * g.Q;
  int m0 = blockIdx.x * kFftCols, P = g.P;
  for (int i = threadIdx.x; i < kFftCols * P; i += blockDim.x) {
    int c = i % kFftCols, p = i / kFftCols;
    double2 v = (m0 + c < g.M) ? base[(size_t)p * g.Q + m0 + c] : make_double2(0.0, 0.0);
    buf[c * P + (__brev(p) >> (32 - g.logP))] = v;
  }
  __syncthreads();
  fft_stages(buf, kFftCols, P);
  for (int i = threadIdx.x; i < kFftCols * P; i += blockDim.x) {
    int c = i % kFftCols, p = i / kFftCols;
    if (m0 + c < g.M) base[(size_t)p * g.Q + m0 + c] = buf[c * P + p];
  }
}

constexpr int kFftRows = 4;

__global__ void k_fft_doppler(GenParams g, double2* X) {
  extern __shared__ double2 buf[];  // [kFftRows][Q]
  double2* base = X + (size_t)blockIdx.y * g.P * g.Q;
  int p0 = blockIdx.x * kFftRows, Q = g.Q;
  for (int i = threadIdx.x; i < kFftRows * Q; i += blockDim.x) {
    int r = i / Q, q = i % Q;
    buf[r * Q + (__brev(q) >> (32 - g.logQ))] = base[(size_t)(p0 + r) * Q + q];
  }
  __syncthreads();
  fft_stages(buf, kFftRows, Q);
  for (int i = threadIdx.x; i < kFftRows * Q; i += blockDim.x) {
    int r = i / Q, q = i % Q;
    base[(size_t)(p0 + r) * Q + (q + Q / 2) % Q] = buf[r * Q + q];
  }
}

__device__ __forceinline__ double level_db(double2 y) {
  double mag = sqrt(y.x * y.x + y.y * y.y);
  return 20.0 * log10(mag < 1e-12 ? 1e-12 : mag);
}

template <typename T>
__device__ __forceinline__ T to_out(double v);
template <>
__device__ __forceinline__ float to_out<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_out<__nv_bfloat16>(double v) { return __double2bfloat16(v); }

template <typename T>
__global__ void __launch_bounds__(1024) k_lognorm(GenParams g, const double2* X, T* noisy, T* clean) {
  __shared__ double s_lo[32], s_hi[32];
  int bm = blockIdx.x, b = bm >> 2, map = bm & 3;
  int PQ = g.P * g.Q;
  const double2* x = X + (size_t)bm * PQ;
  double lo = 1e300, hi = -1e300;
  for (int i = threadIdx.x; i < PQ; i += blockDim.x) {
    double l = level_db(x[i]);
    lo = fmin(lo, l);
    hi = fmax(hi, l);
  }
  for (int o = 16; o; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_lo[warp] = lo;
    s_hi[warp] = hi;
  }
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
    lo = lane < nw ? s_lo[lane] : 1e300;
    hi = lane < nw ? s_hi[lane] : -1e300;
    for (int o = 16; o; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      s_lo[0] = lo;
      s_hi[0] = hi;
    }
  }
  __syncthreads();
  lo = s_lo[0];
  hi = s_hi[0];
  T* dst;
  if (map < 3)
    dst = noisy + ((size_t)b * 3 + map) * PQ;
  else if (clean)
    dst = clean + (size_t)b * PQ;
  else
    return;
  for (int i = threadIdx.x; i < PQ; i += blockDim.x)
    dst[i] = to_out<T>(hi > lo ? (level_db(x[i]) - lo) / (hi - lo) : 0.0);
}

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return (1 << l) == v ? l : -1;
}

}  // namespace

cudaError_t generate(const stda_gen_config* c, uint64_t seed, uint64_t cid, int w0, int B, int bf16,
                     void* noisy, void* clean, int* bins, int* ntgt, cudaStream_t st) {
  GenParams g;
  g.N = c->N; g.M = c->M; g.P = c->P; g.Q = c->Q;
  g.logP = ilog2(c->P);
  g.logQ = ilog2(c->Q);
  g.tmin = c->tmin; g.tmax = c->tmax; g.imin = c->imin; g.imax = c->imax;
  g.snr_min = c->snr_min; g.snr_max = c->snr_max; g.inr_min = c->inr_min; g.inr_max = c->inr_max;
  g.kmin = c->kmin; g.kmax = c->kmax;
  // victim radar (Table "victim parameters"): slope 30 MHz/us over the ADC
  // window, fs = 12.5 MHz, 77 GHz, chirp repetition 2 x 21.12 us, 30 frames/s
  const double c0 = 299792458.0, fc = 77e9, slope = 30e12, fs = 12.5e6, trep = 2.0 * 21.12e-6,
               tframe = 1.0 / 30.0;
  double rres = c0 / (2.0 * slope * (double)g.N / fs);
  double vres = (c0 / fc) / (2.0 * (double)g.M * trep);
  g.drift = vres * tframe / rres;
  g.a_ts2 = slope / (fs * fs);

  const size_t per_window = (size_t)4 * g.P * g.Q * sizeof(double2);
  int chunk = (int)((size_t)512 << 20) / per_window;
  if (chunk < 1) chunk = 1;
  if (chunk > B) chunk = B;
  Scene* sc = nullptr;
  double2* X = nullptr;
  cudaError_t e;
  if ((e = cudaMallocAsync((void**)&sc, sizeof(Scene) * (size_t)B, st))) return e;
  if ((e = cudaMallocAsync((void**)&X, per_window * chunk, st))) {
    cudaFreeAsync(sc, st);
    return e;
  }
  cudaFuncSetAttribute(k_fft_range, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(kFftCols * g.P * sizeof(double2)));
  cudaFuncSetAttribute(k_fft_doppler, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(kFftRows * g.Q * sizeof(double2)));
  k_scene<<<(B + 127) / 128, 128, 0, st>>>(g, seed, cid, w0, B, sc, bins, ntgt);
  for (int c0w = 0; c0w < B && !e; c0w += chunk) {
    int nb = B - c0w < chunk ? B - c0w : chunk;
    cudaMemsetAsync(X, 0, per_window * nb, st);
    k_signal<<<dim3((g.N * g.M + 255) / 256, nb * 4), 256, 0, st>>>(g, seed, cid, w0 + c0w, sc + c0w, X);
    k_fft_range<<<dim3((g.M + kFftCols - 1) / kFftCols, nb * 4), 256, kFftCols * g.P * sizeof(double2), st>>>(g, X);
    k_fft_doppler<<<dim3(g.P / kFftRows, nb * 4), 256, kFftRows * g.Q * sizeof(double2), st>>>(g, X);
    if (bf16)
      k_lognorm<__nv_bfloat16><<<nb * 4, 1024, 0, st>>>(
          g, X, (__nv_bfloat16*)noisy + (size_t)c0w * 3 * g.P * g.Q,
          clean ? (__nv_bfloat16*)clean + (size_t)c0w * g.P * g.Q : nullptr);
    else
      k_lognorm<float><<<nb * 4, 1024, 0, st>>>(g, X, (float*)noisy + (size_t)c0w * 3 * g.P * g.Q,
                                                clean ? (float*)clean + (size_t)c0w * g.P * g.Q : nullptr);
    e = cudaGetLastError();
  }
  cudaFreeAsync(X, st);
  cudaFreeAsync(sc, st);
  return e ? e : cudaGetLastError();
}

}  // namespace stda
