// Training step of Radar-STDA on the GPU: forward with a tape, mean squared
// error against the clean maps (or a given dL/dz), and the adjoint of every
// operation, producing dL/dtheta for all 137,915 parameters.
//
// The graph keeps batch normalisation unfolded (inference form with frozen
// running statistics, or the batch's statistics in training mode; gamma and
// beta are trained), so every tensor of the taped forward is the one the
// adjoint needs. Tensors are NCHW float32, arithmetic FP32 on the CUDA cores:
// dense stride-2 convs and their input gradients as direct convolutions over
// cp.async-staged tiles, their weight gradients as split-K GEMMs, stride-1
// depthwise / stem / output convs and their weight gradients by register
// windows, elementwise passes four elements per thread. Weight and BN
// gradients are first reduced over slices of the batch's pixels in FP32
// (warp shuffles), then the slices are summed in FP64 in a fixed order; the
// loss is an FP64 sum.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "stda_internal.h"
#include "stda_train.h"

namespace stda {
namespace {

constexpr int kT = 256;

inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }
// grid of the per-plane elementwise kernels: x over the n pixels of a plane,
// y over the planes (each block loops over planes y, y + gridDim.y, ...)
inline dim3 gridp(long total, long n) { return dim3(cdiv(n, kT), (unsigned)std::min(total / n, 65535L)); }
inline int planes(long total, long n) { return (int)(total / n); }

// Reductions over the B windows' pixels are split into slices of at least
// kMinSlice pixels, enough of them for about kSliceBlocks blocks per SM, the
// partial sums of one launch holding at most kPartCap floats.
constexpr int kMinSlice = 1024;
constexpr int kSliceBlocks = 8;
constexpr long kPartCap = 1L << 22;

int device_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// Slicing of `total` pixels for a launch of `width` blocks per slice whose
// partials are `outputs` floats per slice: {pixels per slice, slices}.
struct Slices {
  int S, n;
};
Slices slices(long total, long width, long outputs, int align, int blocks_per_sm, int min_slice = kMinSlice) {
  long want = ((long)device_sms() * blocks_per_sm + width - 1) / width;
  want = std::max(1L, std::min(want, kPartCap / std::max(1L, outputs)));
  long S = std::max((long)min_slice, (total + want - 1) / want);
  S = (S + align - 1) / align * align;
  return Slices{(int)S, (int)cdiv(total, S)};
}

// The elementwise kernels take V = 4 consecutive elements per thread
// (16-byte loads and stores; the plane size is then a multiple of 4) or V = 1.
template <int V>
__device__ __forceinline__ void ldv(const float* p, float (&v)[V]) {
  if constexpr (V == 4) {
    const float4 f = *(const float4*)p;
    v[0] = f.x;
    v[1] = f.y;
    v[2] = f.z;
    v[3] = f.w;
  } else {
#pragma unroll
    for (int e = 0; e < V; ++e) v[e] = p[e];
  }
}
template <int V>
__device__ __forceinline__ void stv(float* p, const float (&v)[V]) {
  if constexpr (V == 4) {
    *(float4*)p = make_float4(v[0], v[1], v[2], v[3]);
  } else {
#pragma unroll
    for (int e = 0; e < V; ++e) p[e] = v[e];
  }
}

// a BN layer: gamma, beta, and the mean and variance it normalises with
struct BnP {
  const float *g, *b, *m, *v;
};
__device__ __forceinline__ float bnv(const BnP& q, int c, float x) {
  return q.g[c] * (x - q.m[c]) * rsqrtf(q.v[c] + 1e-5f) + q.b[c];
}

// ----------------------------------------------------------- forward ops
// Each thread computes NT consecutive output channels (forward) or input
// channels (input gradient) of one pixel, so every activation load feeds NT
// FMAs; NT divides the channels per group (NT = 1 for depthwise convs).
// Strided transposed taps: only ky = Y + p (mod s) reach an input row
// (likewise kx), so the loops step by s from that residue.

// y[b][o][Y][X] = bias[o] + sum_{i in group(o), ky, kx} x[b][i][Y s - p + ky][X s - p + kx] w[o][i'][ky][kx]
template <int NT>
__global__ void k_conv(const float* __restrict__ x, const float* __restrict__ w, const float* __restrict__ bias,
                       float* __restrict__ y, int B, int Ci, int H, int W, int Co, int k, int s, int p, int g,
                       int Ho, int Wo) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Ho * Wo) return;
  const int Y = q / Wo, X = q - Y * Wo, o0 = blockIdx.y * NT, b = blockIdx.z;
  int cig = Ci / g, gi = o0 / (Co / g);
  float acc[NT];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j] = bias ? bias[o0 + j] : 0.f;
  for (int il = 0; il < cig; ++il) {
    const float* xp = x + ((size_t)b * Ci + gi * cig + il) * H * W;
    const float* wp = w + ((size_t)o0 * cig + il) * k * k;
    for (int ky = 0; ky < k; ++ky) {
      int yy = Y * s - p + ky;
      if (yy < 0 || yy >= H) continue;
      for (int kx = 0; kx < k; ++kx) {
        int xx = X * s - p + kx;
        if (xx < 0 || xx >= W) continue;
        const float v = xp[yy * W + xx];
#pragma unroll
        for (int j = 0; j < NT; ++j) acc[j] += v * wp[(size_t)j * cig * k * k + ky * k + kx];
      }
    }
  }
  const size_t plane = (size_t)Ho * Wo;
  float* yp = y + ((size_t)b * Co + o0) * plane + (size_t)Y * Wo + X;
#pragma unroll
  for (int j = 0; j < NT; ++j) yp[j * plane] = acc[j];
}

// transposed: y[b][o][Y][X] = bias[o] + sum x[b][i][yi][xi] w[i][o'][ky][kx], Y = yi s - p + ky
template <int NT>
__global__ void k_convT(const float* __restrict__ x, const float* __restrict__ w, const float* __restrict__ bias,
                        float* __restrict__ y, int B, int Ci, int H, int W, int Co, int k, int s, int p, int g,
                        int Ho, int Wo) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Ho * Wo) return;
  const int Y = q / Wo, X = q - Y * Wo, o0 = blockIdx.y * NT, b = blockIdx.z;
  int cig = Ci / g, cog = Co / g, gi = o0 / cog, ol0 = o0 % cog;
  float acc[NT];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j] = bias ? bias[o0 + j] : 0.f;
  for (int il = 0; il < cig; ++il) {
    int i = gi * cig + il;
    const float* xp = x + ((size_t)b * Ci + i) * H * W;
    const float* wp = w + ((size_t)i * cog + ol0) * k * k;
    for (int ky = (Y + p) % s; ky < k; ky += s) {
      int yi = (Y + p - ky) / s;
      if (yi < 0 || yi >= H) continue;
      for (int kx = (X + p) % s; kx < k; kx += s) {
        int xi = (X + p - kx) / s;
        if (xi < 0 || xi >= W) continue;
        const float v = xp[yi * W + xi];
#pragma unroll
        for (int j = 0; j < NT; ++j) acc[j] += v * wp[(size_t)j * k * k + ky * k + kx];
      }
    }
  }
  const size_t plane = (size_t)Ho * Wo;
  float* yp = y + ((size_t)b * Co + o0) * plane + (size_t)Y * Wo + X;
#pragma unroll
  for (int j = 0; j < NT; ++j) yp[j * plane] = acc[j];
}

// dx[b][i][yy][xx] += sum over (o, ky, kx) with yy = Y s - p + ky of dy w (adjoint of k_conv)
template <int NT>
__global__ void k_conv_dgrad(const float* __restrict__ dy, const float* __restrict__ w, float* __restrict__ dx,
                             int B, int Ci, int H, int W, int Co, int k, int s, int p, int g, int Ho, int Wo) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= H * W) return;
  const int yy = q / W, xx = q - yy * W, i0 = blockIdx.y * NT, b = blockIdx.z;
  int cig = Ci / g, cog = Co / g, gi = i0 / cig, il0 = i0 % cig;
  float acc[NT];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j] = 0.f;
  for (int ol = 0; ol < cog; ++ol) {
    int o = gi * cog + ol;
    const float* dp = dy + ((size_t)b * Co + o) * Ho * Wo;
    const float* wp = w + ((size_t)o * cig + il0) * k * k;
    for (int ky = (yy + p) % s; ky < k; ky += s) {
      int Y = (yy + p - ky) / s;
      if (Y < 0 || Y >= Ho) continue;
      for (int kx = (xx + p) % s; kx < k; kx += s) {
        int X = (xx + p - kx) / s;
        if (X < 0 || X >= Wo) continue;
        const float d = dp[Y * Wo + X];
#pragma unroll
        for (int j = 0; j < NT; ++j) acc[j] += d * wp[(size_t)j * k * k + ky * k + kx];
      }
    }
  }
  const size_t plane = (size_t)H * W;
  float* xp = dx + ((size_t)b * Ci + i0) * plane + (size_t)yy * W + xx;
#pragma unroll
  for (int j = 0; j < NT; ++j) xp[j * plane] += acc[j];
}

// dx[b][i][yi][xi] += sum_{o', ky, kx} dy[b][o][yi s - p + ky][xi s - p + kx] w[i][o'][ky][kx]
template <int NT>
__global__ void k_convT_dgrad(const float* __restrict__ dy, const float* __restrict__ w, float* __restrict__ dx,
                              int B, int Ci, int H, int W, int Co, int k, int s, int p, int g, int Ho, int Wo) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= H * W) return;
  const int yi = q / W, xi = q - yi * W, i0 = blockIdx.y * NT, b = blockIdx.z;
  int cig = Ci / g, cog = Co / g, gi = i0 / cig;
  float acc[NT];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j] = 0.f;
  for (int ol = 0; ol < cog; ++ol) {
    int o = gi * cog + ol;
    const float* dp = dy + ((size_t)b * Co + o) * Ho * Wo;
    const float* wp = w + ((size_t)i0 * cog + ol) * k * k;
    for (int ky = 0; ky < k; ++ky) {
      int Y = yi * s - p + ky;
      if (Y < 0 || Y >= Ho) continue;
      for (int kx = 0; kx < k; ++kx) {
        int X = xi * s - p + kx;
        if (X < 0 || X >= Wo) continue;
        const float d = dp[Y * Wo + X];
#pragma unroll
        for (int j = 0; j < NT; ++j) acc[j] += d * wp[(size_t)j * cog * k * k + ky * k + kx];
      }
    }
  }
  const size_t plane = (size_t)H * W;
  float* xp = dx + ((size_t)b * Ci + i0) * plane + (size_t)yi * W + xi;
#pragma unroll
  for (int j = 0; j < NT; ++j) xp[j * plane] += acc[j];
}

// ------------------------------------------ depthwise stride-1 convs
// The per-channel (groups = channels) K x K convs of the blocks' first stage,
// stride 1, pad P = (K - 1) / 2, and their transposed twins are one
// correlation per channel, dst[c][Y][X] (+)= bias[c] + sum_{ky,kx}
// src[c][Y + d ky - d P][X + d kx - d P] w[c][ky][kx] with d = +1, or d = -1
// (FLIP) for the kernel flipped:
//   conv forward, transposed-conv input gradient: d = +1
//   transposed-conv forward, conv input gradient: d = -1
// One thread per output pixel; grid (pixels / 256, C, B).
template <int K, bool FLIP>
__global__ void __launch_bounds__(256) k_dw(const float* __restrict__ src, const float* __restrict__ w,
                                            const float* __restrict__ bias, float* __restrict__ dst, int C, int H,
                                            int W, int accumulate) {
  constexpr int P = (K - 1) / 2;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= H * W) return;
  const int c = blockIdx.y, Y = q / W, X = q - Y * W;
  const size_t plane = ((size_t)blockIdx.z * C + c) * H * W;
  const float* sp = src + plane;
  float wk[K * K];
#pragma unroll
  for (int t = 0; t < K * K; ++t) wk[t] = w[c * K * K + t];
  float acc = bias ? bias[c] : 0.f;
#pragma unroll
  for (int ky = 0; ky < K; ++ky) {
    const int sy = FLIP ? Y + P - ky : Y - P + ky;
    if ((unsigned)sy >= (unsigned)H) continue;
#pragma unroll
    for (int kx = 0; kx < K; ++kx) {
      const int sx = FLIP ? X + P - kx : X - P + kx;
      if ((unsigned)sx < (unsigned)W) acc += sp[sy * W + sx] * wk[ky * K + kx];
    }
  }
  float* dp = dst + plane + q;
  *dp = accumulate ? *dp + acc : acc;
}

// k_dw with four horizontally adjacent outputs per thread (W a multiple of
// 4): each source row is read as one 16-byte load plus the two neighbours.
template <int K, bool FLIP>
__global__ void __launch_bounds__(256) k_dw4(const float* __restrict__ src, const float* __restrict__ w,
                                             const float* __restrict__ bias, float* __restrict__ dst, int C, int H,
                                             int W, int accumulate) {
  constexpr int P = (K - 1) / 2;
  const int W4 = W >> 2, q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= H * W4) return;
  const int c = blockIdx.y, Y = q / W4, X0 = (q - Y * W4) * 4;
  const size_t plane = ((size_t)blockIdx.z * C + c) * H * W;
  const float* sp = src + plane;
  float wk[K * K];
#pragma unroll
  for (int t = 0; t < K * K; ++t) wk[t] = w[c * K * K + t];
  const float b0 = bias ? bias[c] : 0.f;
  float acc[4] = {b0, b0, b0, b0};
#pragma unroll
  for (int ky = 0; ky < K; ++ky) {
    const int sy = FLIP ? Y + P - ky : Y - P + ky;
    if ((unsigned)sy >= (unsigned)H) continue;
    const float* row = sp + (size_t)sy * W + X0;
    float v[4 + 2 * P];  // columns X0 - P .. X0 + 3 + P
    const float4 m = *(const float4*)row;
    v[P] = m.x;
    v[P + 1] = m.y;
    v[P + 2] = m.z;
    v[P + 3] = m.w;
    if (P) {
      v[0] = X0 > 0 ? row[-1] : 0.f;
      v[4 + 2 * P - 1] = X0 + 4 < W ? row[4] : 0.f;
    }
#pragma unroll
    for (int o = 0; o < 4; ++o)
#pragma unroll
      for (int kx = 0; kx < K; ++kx) acc[o] += v[o + (FLIP ? K - 1 - kx : kx)] * wk[ky * K + kx];
  }
  float* dp = dst + plane + (size_t)Y * W + X0;
  if (accumulate) {
    const float4 o = *(const float4*)dp;
    acc[0] += o.x;
    acc[1] += o.y;
    acc[2] += o.z;
    acc[3] += o.w;
  }
  *(float4*)dp = make_float4(acc[0], acc[1], acc[2], acc[3]);
}

// Full 3x3 stride-1 pad-1 convs of few channels (the stem 3 -> 8, the output
// conv 8 -> 1) and their input gradients, four horizontally adjacent pixels
// per thread (W a multiple of 4): dst[n][Y][X] (+)= bias[n] + sum_{m,ky,kx}
// W(n, m, ky, kx) src[m][Y + d ky - d][X + d kx - d], d = -1 when FLIP (the
// input gradient of a conv), W(n, m) = w[n][m] or, when WT, w[m][n].
template <int M, int N, bool FLIP, bool WT>
__global__ void __launch_bounds__(256) k_cs1(const float* __restrict__ src, const float* __restrict__ w,
                                             const float* __restrict__ bias, float* __restrict__ dst, int H, int W,
                                             int accumulate) {
  __shared__ float ws[M * N * 9];
  for (int i = threadIdx.x; i < M * N * 9; i += blockDim.x) ws[i] = w[i];
  __syncthreads();
  const int W4 = W >> 2, q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= H * W4) return;
  const int Y = q / W4, X0 = (q - Y * W4) * 4, b = blockIdx.y;
  const size_t plane = (size_t)H * W;
  float acc[N][4];
#pragma unroll
  for (int n = 0; n < N; ++n)
#pragma unroll
    for (int o = 0; o < 4; ++o) acc[n][o] = bias ? bias[n] : 0.f;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const float* sp = src + ((size_t)b * M + m) * plane;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int sy = FLIP ? Y + 1 - ky : Y - 1 + ky;
      if ((unsigned)sy >= (unsigned)H) continue;
      const float* row = sp + (size_t)sy * W + X0;
      const float4 c4 = *(const float4*)row;
      const float v[6] = {X0 > 0 ? row[-1] : 0.f, c4.x, c4.y, c4.z, c4.w, X0 + 4 < W ? row[4] : 0.f};
#pragma unroll
      for (int n = 0; n < N; ++n)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const float wv = ws[(WT ? m * N + n : n * M + m) * 9 + ky * 3 + kx];
#pragma unroll
          for (int o = 0; o < 4; ++o) acc[n][o] += v[o + (FLIP ? 2 - kx : kx)] * wv;
        }
    }
  }
#pragma unroll
  for (int n = 0; n < N; ++n) {
    float* dp = dst + ((size_t)b * N + n) * plane + (size_t)Y * W + X0;
    float4 r = make_float4(acc[n][0], acc[n][1], acc[n][2], acc[n][3]);
    if (accumulate) {
      const float4 o = *(const float4*)dp;
      r.x += o.x;
      r.y += o.y;
      r.z += o.z;
      r.w += o.w;
    }
    *(float4*)dp = r;
  }
}

// Weight gradients of the stride-1, pad (K - 1) / 2 convs: the per-channel
// ones (DW: dW[c][t] = sum_p A[c][p] G[c][p + t - P]) and the full ones of
// few channels (dW[a][g][t] = sum_p A[a][p] G[g][p + t - P], A = dy with CA
// output channels, G = x with CG input channels; index (a CG + g) K^2 + t).
// For a conv A = dy and G = x; for a transposed depthwise conv A = x and
// G = dy. A thread walks down L rows of one column X of one window, keeping
// the K x K window of G (NG channels) in registers and loading one new G row
// per step; it accumulates NA x NG x K^2 sums. Group blockIdx.y selects the
// channels (DW: channel y; full: A channels (y / ngg) NA + a, G channels
// (y % ngg) NG + j). Each block sums its threads (warp shuffles, then one
// pass over the warps) into part[blockIdx.x][output index].
template <int K, int NA, int NG, bool DW>
__global__ void __launch_bounds__(256) k_wgrad_s1(const float* __restrict__ A, const float* __restrict__ G,
                                                  float* __restrict__ part, int B, int H, int W, int CA, int CG,
                                                  int L, int nseg, int nout) {
  constexpr int P = (K - 1) / 2, KK = K * K, NV = NA * NG * KK;
  __shared__ float sh[8][NV];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = blockIdx.y, ngg = DW ? 1 : CG / NG;
  const int a0 = DW ? grp : (grp / ngg) * NA, g0 = DW ? grp : (grp % ngg) * NG;
  const int task = blockIdx.x * blockDim.x + tid;
  float acc[NA][NG][KK];
#pragma unroll
  for (int i = 0; i < NA; ++i)
#pragma unroll
    for (int j = 0; j < NG; ++j)
#pragma unroll
      for (int t = 0; t < KK; ++t) acc[i][j][t] = 0.f;
  if (task < B * nseg * W) {
    const int X = task % W, r = task / W, yseg = r % nseg, b = r / nseg;
    const int y0 = yseg * L, y1 = min(H, y0 + L);
    const size_t plane = (size_t)H * W;
    const float* ap = A + ((size_t)b * CA + a0) * plane + X;
    const float* gp = G + ((size_t)b * (DW ? CA : CG) + g0) * plane;
    float win[NG][K][K];  // win[j][ry][kx] = G[g0 + j][Y - P + ry][X - P + kx]
    auto load_row = [&](int gy, int ry) {
#pragma unroll
      for (int j = 0; j < NG; ++j)
#pragma unroll
        for (int kx = 0; kx < K; ++kx) {
          const int gx = X - P + kx;
          win[j][ry][kx] = (unsigned)gy < (unsigned)H && (unsigned)gx < (unsigned)W
                               ? gp[j * plane + (size_t)gy * W + gx]
                               : 0.f;
        }
    };
#pragma unroll
    for (int ry = 1; ry < K; ++ry) load_row(y0 - P + ry - 1, ry);
    for (int Y = y0; Y < y1; ++Y) {
#pragma unroll
      for (int ry = 0; ry + 1 < K; ++ry)
#pragma unroll
        for (int j = 0; j < NG; ++j)
#pragma unroll
          for (int kx = 0; kx < K; ++kx) win[j][ry][kx] = win[j][ry + 1][kx];
      load_row(Y + P, K - 1);
      float av[NA];
#pragma unroll
      for (int i = 0; i < NA; ++i) av[i] = ap[i * plane + (size_t)Y * W];
#pragma unroll
      for (int i = 0; i < NA; ++i)
#pragma unroll
        for (int j = 0; j < NG; ++j)
#pragma unroll
          for (int ry = 0; ry < K; ++ry)
#pragma unroll
            for (int kx = 0; kx < K; ++kx) acc[i][j][ry * K + kx] += av[i] * win[j][ry][kx];
    }
  }
#pragma unroll
  for (int i = 0; i < NA; ++i)
#pragma unroll
    for (int j = 0; j < NG; ++j)
#pragma unroll
      for (int t = 0; t < KK; ++t) {
        float v = acc[i][j][t];
#pragma unroll
        for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) sh[warp][(i * NG + j) * KK + t] = v;
      }
  __syncthreads();
  const int nw = blockDim.x >> 5;
  for (int v = tid; v < NV; v += blockDim.x) {
    float r = 0.f;
    for (int k = 0; k < nw; ++k) r += sh[k][v];
    const int i = v / (NG * KK), j = (v / KK) % NG, t = v % KK;
    const int o = DW ? grp * KK + t : ((a0 + i) * CG + g0 + j) * KK + t;
    part[(size_t)blockIdx.x * nout + o] = r;
  }
}

// ------------------------------------- dense stride-2 convs, direct form
// The dense (one-group) stride-2, pad-1 convs of the blocks and their input
// gradients, as direct convolutions with the source tile staged in shared
// memory (kDcMC channels a stage, with the K x K weights of the block's
// output channels), each thread holding NP pixels x NO output channels:
//   k_sconv  (conv, K = 3 encoder forward, K = 4 decoder input gradient):
//     out[n][Y][X] (+)= bias[n] + sum_{m,ky,kx} w[n][m][ky][kx] src[m][2Y-1+ky][2X-1+kx]
//   k_stconv (transposed, K = 4 decoder forward, K = 3 encoder input gradient):
//     out[n][Y][X] (+)= bias[n] + sum w[m][n][ky][kx] src[m][yi][xi] over Y = 2yi-1+ky, X = 2xi-1+kx
// Stages are copied with cp.async (zero-filled outside the source) into two
// shared-memory buffers, the next stage in flight while the current one is
// used; the weights come re-laid as wT[m][ky kx][n] (k_wt), 16 bytes a copy,
// as do the transposed form's source rows. 256 threads: warp w = (row group or output phase, channel group);
// lane = (row in the warp, column), TX columns per warp row. Sums run in FP32
// over m, then ky, kx; a thread's output channels 2 j and 2 j + 1 share one
// packed FMA (fma.rn.f32x2: two IEEE FMAs, the same results).
constexpr int kDcMC = 4;  // source channels per stage
constexpr long kDcWT = 32768;  // largest dense conv weight tensor (64 x 32 x 4 x 4)

__device__ __forceinline__ void cp_async4(float* sdst, const float* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(gsrc), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async16(float* sdst, const float* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Weights of a dense conv re-laid as wT[m][ky kx][n] (m source, n output
// channel), so a block's output channels of one (m, tap) are contiguous:
// from w[m][n][t] (T) or w[n][m][t].
__global__ void k_wt(const float* __restrict__ w, float* __restrict__ wT, int M, int N, int KK, int T) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * KK * N) return;
  const int n = e % N, t = (e / N) % KK, m = e / (N * KK);
  wT[e] = T ? w[((size_t)m * N + n) * KK + t] : w[((size_t)n * M + m) * KK + t];
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int NO>
__device__ __forceinline__ void load_w(const float* p, float (&wv)[NO]) {
#pragma unroll
  for (int q = 0; q < NO / 4; ++q) {
    const float4 f = *(const float4*)&p[4 * q];
    wv[4 * q] = f.x;
    wv[4 * q + 1] = f.y;
    wv[4 * q + 2] = f.z;
    wv[4 * q + 3] = f.w;
  }
}

template <int K, int NO, int TX, int NPP>
struct SconvGeo {
  static constexpr int NP = NPP, KK = K * K, RW = 32 / TX, TY = 4 * NP * RW, R = 2 * TY + K - 2;
  static constexpr int PW = TX == 32 ? 33 : 20;  // parity-plane row (TX + 1, padded against conflicts)
  static constexpr int RS = 2 * PW, CS = R * RS, NB = 2 * NO;
  static constexpr int NX = kDcMC * CS, NW = kDcMC * KK * NB, STAGE = NX + NW;
  static constexpr size_t smem() { return sizeof(float) * 2 * STAGE; }
};

template <int K, int NO, int TX, int NP_>
__global__ void __launch_bounds__(256) k_sconv(const float* __restrict__ src, const float* __restrict__ w,
                                               const float* __restrict__ bias, float* __restrict__ out, int M,
                                               int Hs, int Ws, int N, int accumulate) {
  using G = SconvGeo<K, NO, TX, NP_>;
  constexpr int KK = G::KK, RW = G::RW, NP = G::NP, TY = G::TY, R = G::R, PW = G::PW, RS = G::RS, CS = G::CS;
  constexpr int NB = G::NB;
  extern __shared__ __align__(16) float dsm[];
  const int Ho = Hs / 2, Wo = Ws / 2;
  const int tilesx = (Wo + TX - 1) / TX;
  const int X0 = (blockIdx.x % tilesx) * TX, Y0 = (blockIdx.x / tilesx) * TY;
  const int n0 = blockIdx.y * NB, b = blockIdx.z;
  const int tid = threadIdx.x, lane = tid & 31, wq = tid >> 5, cg = wq & 1, rg = wq >> 1;
  const int x = lane % TX, ry = lane / TX;
  const size_t splane = (size_t)Hs * Ws;
  const float* sb = src + (size_t)b * M * splane;
  auto issue = [&](int m0, float* buf) {
    for (int e = tid; e < kDcMC * R * 2 * PW; e += 256) {
      const int m = e / (R * 2 * PW), r = (e / (2 * PW)) % R, u = e % (2 * PW);
      const int gy = 2 * Y0 - 1 + r, gx = 2 * X0 - 1 + u;
      const bool ok = m0 + m < M && (unsigned)gy < (unsigned)Hs && (unsigned)gx < (unsigned)Ws && u < 2 * TX + K - 2;
      cp_async4(buf + m * CS + r * RS + (u & 1) * PW + (u >> 1),
                ok ? sb + (size_t)(m0 + m) * splane + (size_t)gy * Ws + gx : src, ok);
    }
    float* wsb = buf + G::NX;
    for (int e = tid; e < G::NW / 4; e += 256) {  // 16-byte runs of wT[m][t][n0 ..]
      const int q = e % (NB / 4), t = (e / (NB / 4)) % KK, m = e / ((NB / 4) * KK);
      const bool ok = m0 + m < M;
      cp_async16(wsb + (m * KK + t) * NB + 4 * q, ok ? w + ((size_t)(m0 + m) * KK + t) * N + n0 + 4 * q : w, ok);
    }
    cp_async_commit();
  };
  float2 acc[NP][NO / 2];
#pragma unroll
  for (int i = 0; i < NP; ++i)
#pragma unroll
    for (int j = 0; j < NO / 2; ++j) acc[i][j] = make_float2(0.f, 0.f);
  issue(0, dsm);
  int stage = 0;
  for (int m0 = 0; m0 < M; m0 += kDcMC, ++stage) {
    const float* xs = dsm + (stage & 1) * G::STAGE;
    const float* ws = xs + G::NX;
    if (m0 + kDcMC < M) {
      issue(m0 + kDcMC, dsm + ((stage + 1) & 1) * G::STAGE);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* xb = xs + (2 * (rg * NP * RW + ry)) * RS + x;
#pragma unroll
    for (int m = 0; m < kDcMC; ++m) {
#pragma unroll
      for (int ky = 0; ky < K; ++ky)
#pragma unroll
        for (int kx = 0; kx < K; ++kx) {
          float wv[NO];
          load_w<NO>(ws + (m * KK + ky * K + kx) * NB + cg * NO, wv);
#pragma unroll
          for (int i = 0; i < NP; ++i) {
            const float xv = xb[m * CS + (2 * i * RW + ky) * RS + (kx & 1) * PW + (kx >> 1)];
#pragma unroll
            for (int j = 0; j < NO / 2; ++j)  // output channels 2 j, 2 j + 1: two FMAs in one instruction
              acc[i][j] = __ffma2_rn(make_float2(xv, xv), make_float2(wv[2 * j], wv[2 * j + 1]), acc[i][j]);
          }
        }
    }
    __syncthreads();  // this buffer is refilled two stages on
  }
  const size_t oplane = (size_t)Ho * Wo;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    const int Y = Y0 + (rg * NP + i) * RW + ry, X = X0 + x;
    if (Y >= Ho || X >= Wo) continue;
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      const int n = n0 + cg * NO + j;
      if (n >= N) continue;
      float* o = out + ((size_t)b * N + n) * oplane + (size_t)Y * Wo + X;
      const float v = (j & 1) ? acc[i][j >> 1].y : acc[i][j >> 1].x;
      *o = accumulate ? *o + v : v + (bias ? bias[n] : 0.f);
    }
  }
}

template <int K, int NO, int TX, int NPP>
struct StconvGeo {
  static constexpr int NP = NPP, KK = K * K, RW = 32 / TX, TU = NP * RW, R = TU + 2;
  static constexpr int RS = TX == 32 ? 40 : 48;  // source tile row (TX + 8, padded against conflicts)
  static constexpr int CS = R * RS, NB = 2 * NO;
  static constexpr int NX = kDcMC * CS, NW = kDcMC * KK * NB, STAGE = NX + NW;
  static constexpr size_t smem() { return sizeof(float) * 2 * STAGE; }
};

// the taps of output phase (PY, PX) of k_stconv: ky = ky0 + 2 sy < K with
// ky0 = (PY + 1) mod 2, source row offset (PY + 1 - ky) / 2 (likewise x)
template <int K, int NO, int TX, int NP, int PY, int PX>
__device__ __forceinline__ void stconv_phase(const float* xb, const float* wb, float2 (&acc)[NP][NO / 2]) {
  using G = StconvGeo<K, NO, TX, NP>;
  constexpr int KY0 = (PY + 1) & 1, KX0 = (PX + 1) & 1;
  constexpr int NTY = KY0 + 2 < K ? 2 : 1, NTX = KX0 + 2 < K ? 2 : 1;
#pragma unroll
  for (int m = 0; m < kDcMC; ++m)
#pragma unroll
    for (int sy = 0; sy < NTY; ++sy)
#pragma unroll
      for (int sx = 0; sx < NTX; ++sx) {
        const int ky = KY0 + 2 * sy, kx = KX0 + 2 * sx;
        const int dy = (PY + 1 - ky) / 2, dx = (PX + 1 - kx) / 2;
        float wv[NO];
        load_w<NO>(wb + (m * G::KK + ky * K + kx) * G::NB, wv);
#pragma unroll
        for (int i = 0; i < G::NP; ++i) {
          const float xv = xb[m * G::CS + (i * G::RW + 1 + dy) * G::RS + 1 + dx];
#pragma unroll
          for (int j = 0; j < NO / 2; ++j)  // output channels 2 j, 2 j + 1: two FMAs in one instruction
            acc[i][j] = __ffma2_rn(make_float2(xv, xv), make_float2(wv[2 * j], wv[2 * j + 1]), acc[i][j]);
        }
      }
}

template <int K, int NO, int TX, int NP_>
__global__ void __launch_bounds__(256) k_stconv(const float* __restrict__ src, const float* __restrict__ w,
                                                const float* __restrict__ bias, float* __restrict__ out, int M,
                                                int Hs, int Ws, int N, int accumulate) {
  using G = StconvGeo<K, NO, TX, NP_>;
  constexpr int KK = G::KK, RW = G::RW, NP = G::NP, TU = G::TU, R = G::R, RS = G::RS, NB = G::NB;
  extern __shared__ __align__(16) float dsm[];
  const int Ho = 2 * Hs, Wo = 2 * Ws;
  const int tilesx = (Ws + TX - 1) / TX;
  const int V0 = (blockIdx.x % tilesx) * TX, U0 = (blockIdx.x / tilesx) * TU;
  const int n0 = blockIdx.y * NB, b = blockIdx.z;
  const int tid = threadIdx.x, lane = tid & 31, wq = tid >> 5, ph = wq & 3, cg = wq >> 2;
  const int py = ph >> 1, px = ph & 1, v = lane % TX, ru = lane / TX;
  const size_t splane = (size_t)Hs * Ws;
  const float* sb = src + (size_t)b * M * splane;
  auto issue = [&](int m0, float* buf) {
    // tile row r, column c holds source (U0 - 1 + r, V0 - 4 + c): 16-byte
    // runs that lie wholly inside or outside the map (Ws, V0 multiples of 4)
    constexpr int CH = (TX + 8) / 4;
    for (int e = tid; e < kDcMC * R * CH; e += 256) {
      const int j = e % CH, r = (e / CH) % R, m = e / (CH * R);
      const int gy = U0 - 1 + r, gx = V0 - 4 + 4 * j;
      const bool ok = m0 + m < M && (unsigned)gy < (unsigned)Hs && (unsigned)gx < (unsigned)Ws;
      cp_async16(buf + m * G::CS + r * RS + 4 * j, ok ? sb + (size_t)(m0 + m) * splane + (size_t)gy * Ws + gx : src,
                 ok);
    }
    float* wsb = buf + G::NX;
    for (int e = tid; e < G::NW / 4; e += 256) {  // 16-byte runs of wT[m][t][n0 ..]
      const int q = e % (NB / 4), t = (e / (NB / 4)) % KK, m = e / ((NB / 4) * KK);
      const bool ok = m0 + m < M;
      cp_async16(wsb + (m * KK + t) * NB + 4 * q, ok ? w + ((size_t)(m0 + m) * KK + t) * N + n0 + 4 * q : w, ok);
    }
    cp_async_commit();
  };
  float2 acc[NP][NO / 2];
#pragma unroll
  for (int i = 0; i < NP; ++i)
#pragma unroll
    for (int j = 0; j < NO / 2; ++j) acc[i][j] = make_float2(0.f, 0.f);
  issue(0, dsm);
  int stage = 0;
  for (int m0 = 0; m0 < M; m0 += kDcMC, ++stage) {
    const float* xs = dsm + (stage & 1) * G::STAGE;
    const float* ws = xs + G::NX;
    if (m0 + kDcMC < M) {
      issue(m0 + kDcMC, dsm + ((stage + 1) & 1) * G::STAGE);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* xb = xs + ru * RS + v + 3;  // + 1 + dx: column V0 + v + dx
    const float* wb = ws + cg * NO;
    switch (ph) {
      case 0: stconv_phase<K, NO, TX, NP, 0, 0>(xb, wb, acc); break;
      case 1: stconv_phase<K, NO, TX, NP, 0, 1>(xb, wb, acc); break;
      case 2: stconv_phase<K, NO, TX, NP, 1, 0>(xb, wb, acc); break;
      default: stconv_phase<K, NO, TX, NP, 1, 1>(xb, wb, acc); break;
    }
    __syncthreads();  // this buffer is refilled two stages on
  }
  const size_t oplane = (size_t)Ho * Wo;
#pragma unroll
  for (int i = 0; i < NP; ++i) {
    const int Y = 2 * (U0 + i * RW + ru) + py, X = 2 * (V0 + v) + px;
    if (Y >= Ho || X >= Wo) continue;
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      const int n = n0 + cg * NO + j;
      if (n >= N) continue;
      float* o = out + ((size_t)b * N + n) * oplane + (size_t)Y * Wo + X;
      const float v = (j & 1) ? acc[i][j >> 1].y : acc[i][j >> 1].x;
      *o = accumulate ? *o + v : v + (bias ? bias[n] : 0.f);
    }
  }
}

// ------------------------------------------- dense stride-2 convs as GEMMs
// The dense convolutions of the blocks (3x3 stride 2 in the encoder, 4x4
// stride-2 transposed in the decoder, pad 1, one group) and their input
// gradients as tiled FP32 implicit GEMMs on the CUDA cores:
//   ENC_FWD   y[b][n][Y][X]      = bias[n] + sum_{i,ky,kx} W[n][i][ky][kx] x[b][i][2Y-1+ky][2X-1+kx]
//   DEC_FWD   y[b][n][2yo+py][2xo+px] = bias[n] + sum_{i,sy,sx} W[i][n][ky][kx] x[b][i][yo+py-sy][xo+px-sx],
//             ky = 1 - py + 2 sy (the four taps of output phase (py, px))
//   ENC_DGRAD dx[b][n][yy][xx]  += sum_{o,ky,kx} W[o][n][ky][kx] dy[b][o][(yy+1-ky)/2][(xx+1-kx)/2]
//             over the taps of parity ky = yy + 1 (mod 2) (one or two per axis)
//   DEC_DGRAD dx[b][n][yi][xi]  += sum_{o,ky,kx} W[n][o][ky][kx] dy[b][o][2yi-1+ky][2xi-1+kx]
// GEMM rows m are pixels (of one output phase: blockIdx.z), columns n output
// channels, K runs over (input channel, tap). A block computes BM x BN
// outputs (4 x 4 per thread, BM * BN = 4096) in K-steps of 8 staged in shared
// memory. Sums run in FP32 in increasing k.
enum { ENC_FWD = 0, DEC_FWD = 1, ENC_DGRAD = 2, DEC_DGRAD = 3 };

struct GemmArgs {
  const float* src;   // x (forward) or dy (input gradient), NCHW
  const float* w;     // the conv's weights in PyTorch layout
  const float* bias;  // forward only, or null
  float* out;         // y (written) or dx (accumulated)
  int B, Cs, Hs, Ws;  // source tensor
  int N, Ho, Wo;      // output channels and output map
  int Cw;             // the weight tensor's other channel count
};

template <int CASE, int BN>
__global__ void __launch_bounds__(256) k_igemm(GemmArgs a) {
  constexpr int BM = 4096 / BN, BK = 8, KPT = BK * BM / 256;
  __shared__ __align__(16) float As[BK][BM];
  __shared__ __align__(16) float Bs[BK][BN];
  const int tid = threadIdx.x, py = blockIdx.z >> 1, px = blockIdx.z & 1;
  // phase grid of the GEMM rows: pixels (b, r, c) of an Hr x Wr map
  int Hr, Wr, ty = 1, tx = 1, K;
  if (CASE == ENC_FWD) { Hr = a.Ho; Wr = a.Wo; K = a.Cs * 9; }
  else if (CASE == DEC_FWD) { Hr = a.Hs; Wr = a.Ws; K = a.Cs * 4; }
  else if (CASE == ENC_DGRAD) { Hr = a.Ho / 2; Wr = a.Wo / 2; ty = py ? 2 : 1; tx = px ? 2 : 1; K = a.Cs * ty * tx; }
  else { Hr = a.Ho; Wr = a.Wo; K = a.Cs * 16; }
  const long M = (long)a.B * Hr * Wr;
  const long m0 = (long)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;
  // this thread's A row and K slice for the tile loads
  const int ml = tid % BM, kg = tid / BM;
  const long mrow = m0 + ml;
  const bool mok = mrow < M;
  int bb = 0, rr = 0, cc = 0;
  if (mok) {
    bb = (int)(mrow / ((long)Hr * Wr));
    const int q = (int)(mrow % ((long)Hr * Wr));
    rr = q / Wr;
    cc = q % Wr;
  }
  const int tn = tid % (BN / 4), tm = tid / (BN / 4);
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
      const int kl = kg * KPT + j, k = k0 + kl;
      float v = 0.f;
      if (mok && k < K) {
        if (CASE == ENC_FWD) {
          const int i = k / 9, t = k % 9, y = 2 * rr - 1 + t / 3, x = 2 * cc - 1 + t % 3;
          if (y >= 0 && y < a.Hs && x >= 0 && x < a.Ws) v = a.src[(((size_t)bb * a.Cs + i) * a.Hs + y) * a.Ws + x];
        } else if (CASE == DEC_FWD) {
          const int i = k >> 2, sy = (k >> 1) & 1, sx = k & 1, y = rr + py - sy, x = cc + px - sx;
          if (y >= 0 && y < a.Hs && x >= 0 && x < a.Ws) v = a.src[(((size_t)bb * a.Cs + i) * a.Hs + y) * a.Ws + x];
        } else if (CASE == ENC_DGRAD) {
          const int o = k / (ty * tx), t = k % (ty * tx);
          const int ky = py ? 2 * (t / tx) : 1, kx = px ? 2 * (t % tx) : 1;
          const int y = (2 * rr + py + 1 - ky) / 2, x = (2 * cc + px + 1 - kx) / 2;
          if (y >= 0 && y < a.Hs && x >= 0 && x < a.Ws) v = a.src[(((size_t)bb * a.Cs + o) * a.Hs + y) * a.Ws + x];
        } else {
          const int o = k >> 4, ky = (k >> 2) & 3, kx = k & 3, y = 2 * rr - 1 + ky, x = 2 * cc - 1 + kx;
          if (y >= 0 && y < a.Hs && x >= 0 && x < a.Ws) v = a.src[(((size_t)bb * a.Cs + o) * a.Hs + y) * a.Ws + x];
        }
      }
      As[kl][ml] = v;
    }
    for (int e = tid; e < BK * BN; e += 256) {
      const int kl = e / BN, nl = e % BN, k = k0 + kl, n = n0 + nl;
      float v = 0.f;
      if (k < K && n < a.N) {
        if (CASE == ENC_FWD) {
          v = a.w[(size_t)n * K + k];
        } else if (CASE == DEC_FWD) {
          const int i = k >> 2, sy = (k >> 1) & 1, sx = k & 1, ky = 1 - py + 2 * sy, kx = 1 - px + 2 * sx;
          v = a.w[(((size_t)i * a.N + n) * 4 + ky) * 4 + kx];
        } else if (CASE == ENC_DGRAD) {
          const int o = k / (ty * tx), t = k % (ty * tx);
          const int ky = py ? 2 * (t / tx) : 1, kx = px ? 2 * (t % tx) : 1;
          v = a.w[(((size_t)o * a.N + n) * 3 + ky) * 3 + kx];
        } else {
          v = a.w[((size_t)n * a.Cs) * 16 + k];
        }
      }
      Bs[kl][nl] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 av = *(const float4*)&As[kk][tm * 4];
      const float4 bv = *(const float4*)&Bs[kk][tn * 4];
      const float am[4] = {av.x, av.y, av.z, av.w}, bn[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += am[i] * bn[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long m = m0 + tm * 4 + i;
    if (m >= M) continue;
    const int b = (int)(m / ((long)Hr * Wr)), q = (int)(m % ((long)Hr * Wr)), r = q / Wr, c = q % Wr;
    int Y = r, X = c;
    if (CASE == DEC_FWD) { Y = 2 * r + py; X = 2 * c + px; }
    if (CASE == ENC_DGRAD) { Y = 2 * r + py; X = 2 * c + px; }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tn * 4 + j;
      if (n >= a.N) continue;
      float* o = a.out + (((size_t)b * a.N + n) * a.Ho + Y) * a.Wo + X;
      if (CASE == ENC_FWD || CASE == DEC_FWD)
        *o = acc[i][j] + (a.bias ? a.bias[n] : 0.f);
      else
        *o += acc[i][j];
    }
  }
}

// Weight gradients of the full (one-group) convs as split-K FP32 GEMMs:
//   conv:       dW[o][i][ky][kx] = sum_{b,Y,X} dy[b][o][Y][X] x[b][i][sY-p+ky][sX-p+kx]
//   transposed: dW[i][o][ky][kx] = sum_{b,y,x} x[b][i][y][x] dy[b][o][sy-p+ky][sx-p+kx]
// Both are part[slice][r][c] = sum over the slice's pixels m of A[m][r] G[m][c]:
// A the row operand (dy of a conv, x of a transposed conv) on its own map
// Hp x Wp, r its channel (M rows, padded with zero rows to MP, a multiple of
// 4); G the gathered operand on its map Hg x Wg, c = channel * KS^2 + tap (N
// columns). A block owns columns [n0, n0 + BN) of one slice (S pixels, a
// multiple of 32) and stages 32 pixels at a time in shared memory, one row
// or column per warp pass with lane = pixel, in 16-byte groups XOR-swizzled
// by (row / 4) mod 8 so that the lane-per-pixel stores and the per-thread
// 4 x 4 float4 reads are free of bank conflicts. The next stage's values are
// loaded into registers while the current one is multiplied. KG groups of
// P = (MP / 4) (BN / 4) threads take the 4-pixel groups of a stage in turn;
// their 4 x 4 sums are added in group order at the end.
struct WgArgs {
  const float* a;  // row operand, [B][M][Hp][Wp]
  const float* g;  // gathered operand, [B][CG][Hg][Wg]
  float* part;     // [slices][M][N]
  int B, M, MP, N, CG, Hp, Wp, Hg, Wg, s, p;
  int BN, KG, S;
};
// values of one stage each lane loads: rows wq + i nw (i < kWgRows), columns
// wq + j nw (j < kWgCols)
constexpr int kWgRows = 8, kWgCols = 16;

__device__ __forceinline__ int wg_swz(int row, int grp) { return row * 32 + ((grp ^ ((row >> 2) & 7)) << 2); }

template <int KS>
__global__ void __launch_bounds__(256, 3) k_wgemm(WgArgs a) {
  constexpr int KK = KS * KS;
  extern __shared__ __align__(16) float wsm[];
  float* As = wsm;                 // [MP][32], swizzled
  float* Gs = wsm + 32 * a.MP;     // [BN][32], swizzled
  int* tab = (int*)(Gs + 32 * a.BN);
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, wq = tid >> 5, nw = nth >> 5;
  const int P = (a.MP >> 2) * (a.BN >> 2), kg = tid / P, pos = tid % P;
  const int tm = pos / (a.BN >> 2), tn = pos % (a.BN >> 2);
  const bool act = kg < a.KG;
  const int n0 = blockIdx.y * a.BN;
  const int np = a.Hp * a.Wp;
  const int K = a.B * np, k0 = blockIdx.x * a.S, k1 = min(K, k0 + a.S);
  const int gplane = a.Hg * a.Wg;
  // column c: offset of its (channel, ky, kx) in a window of G << 4 | ky << 2 | kx
  for (int c = tid; c < a.BN; c += nth) {
    const int col = n0 + c, ch = col / KK, t = col % KK, ky = t / KS, kx = t % KS;
    tab[c] = col < a.N ? ((ch * gplane + ky * a.Wg + kx) << 4) | (ky << 2) | kx : -1;
  }
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  float ra[kWgRows], rg[kWgCols];
  auto fetch = [&](int s0) {
    const int m = s0 + lane;
    const bool mok = m < k1;
    int b = 0, q = 0, Y = 0, X = 0;
    if (mok) {
      b = (unsigned)m / (unsigned)np;
      q = m - b * np;
      Y = (unsigned)q / (unsigned)a.Wp;
      X = q - Y * a.Wp;
    }
    const float* ab = a.a + (size_t)b * a.M * np + q;
#pragma unroll
    for (int i = 0; i < kWgRows; ++i) {
      const int r = wq + i * nw;
      ra[i] = mok && r < a.M ? ab[(size_t)r * np] : 0.f;
    }
    const int gy0 = a.s * Y - a.p, gx0 = a.s * X - a.p;
    const float* gb = a.g + (size_t)b * a.CG * gplane + (gy0 * a.Wg + gx0);
#pragma unroll
    for (int j = 0; j < kWgCols; ++j) {
      const int c = wq + j * nw;
      float v = 0.f;
      if (mok && c < a.BN) {
        const int e = tab[c];
        if (e >= 0 && (unsigned)(gy0 + ((e >> 2) & 3)) < (unsigned)a.Hg && (unsigned)(gx0 + (e & 3)) < (unsigned)a.Wg)
          v = gb[e >> 4];
      }
      rg[j] = v;
    }
  };
  __syncthreads();  // the column table
  if (k0 < k1) fetch(k0);
  const int so = lane & 3, sg = lane >> 2;
  for (int s0 = k0; s0 < k1; s0 += 32) {
    __syncthreads();  // the previous stage's reads are done
#pragma unroll
    for (int i = 0; i < kWgRows; ++i) {
      const int r = wq + i * nw;
      if (r < a.MP) As[wg_swz(r, sg) + so] = ra[i];
    }
#pragma unroll
    for (int j = 0; j < kWgCols; ++j) {
      const int c = wq + j * nw;
      if (c < a.BN) Gs[wg_swz(c, sg) + so] = rg[j];
    }
    __syncthreads();
    if (s0 + 32 < k1) fetch(s0 + 32);
    if (act) {
      for (int grp = kg; grp < 8; grp += a.KG) {
        float4 av[4], gv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = *(const float4*)&As[wg_swz(tm * 4 + i, grp)];
#pragma unroll
        for (int j = 0; j < 4; ++j) gv[j] = *(const float4*)&Gs[wg_swz(tn * 4 + j, grp)];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[i][j] += av[i].x * gv[j].x;
            acc[i][j] += av[i].y * gv[j].y;
            acc[i][j] += av[i].z * gv[j].z;
            acc[i][j] += av[i].w * gv[j].w;
          }
      }
    }
  }
  // k-group sums, in group order: red[(kg * 16 + v) * P + pos]
  if (a.KG > 1) {
    __syncthreads();
    if (act) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) wsm[(kg * 16 + i * 4 + j) * P + pos] = acc[i][j];
    }
    __syncthreads();
    if (kg == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float r = wsm[(i * 4 + j) * P + pos];
          for (int k = 1; k < a.KG; ++k) r += wsm[(k * 16 + i * 4 + j) * P + pos];
          acc[i][j] = r;
        }
    }
  }
  if (kg == 0) {
    float* out = a.part + (size_t)blockIdx.x * a.M * a.N;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int row = tm * 4 + i, col = n0 + tn * 4 + j;
        if (row < a.M && col < a.N) out[(size_t)row * a.N + col] = acc[i][j];
      }
  }
}

// k_wgemm with the block shape fixed at compile time (the six dense convs of
// the network): MP rows, BN columns per block, KG k-groups of
// P = (MP / 4) (BN / 4) threads, 256 threads (8 warps) in all. Every stage
// index, swizzle and loop bound is then a constant: each lane fills MP / 8
// rows and BN / 8 columns of a 32-pixel stage.
template <int KS, int MP, int BN, int KG>
__global__ void __launch_bounds__(256, 2) k_wgemm_t(WgArgs a) {
  constexpr int KK = KS * KS, P = (MP / 4) * (BN / 4), RA = MP / 8, RG = BN / 8;
  static_assert(P * KG <= 256 && MP % 8 == 0 && BN % 8 == 0, "block shape");
  constexpr int NGRP = (8 + KG - 1) / KG;  // 4-pixel groups per k-group and stage
  __shared__ __align__(16) float As[MP * 32];
  __shared__ __align__(16) float Gs[BN * 32];
  __shared__ int tab[BN];
  __shared__ __align__(16) float red[KG > 1 ? KG * 16 * P : 1];
  const int tid = threadIdx.x, lane = tid & 31, wq = tid >> 5;
  const int kg = tid / P, pos = tid % P, tm = pos / (BN / 4), tn = pos % (BN / 4);
  const bool act = kg < KG;
  const int n0 = blockIdx.y * BN;
  const int np = a.Hp * a.Wp;
  const int K = a.B * np, k0 = blockIdx.x * a.S, k1 = min(K, k0 + a.S);
  const int gplane = a.Hg * a.Wg;
  for (int c = tid; c < BN; c += 256) {
    const int col = n0 + c, ch = col / KK, t = col % KK, ky = t / KS, kx = t % KS;
    tab[c] = col < a.N ? ((ch * gplane + ky * a.Wg + kx) << 4) | (ky << 2) | kx : -1;
  }
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  float ra[RA], rg[RG];
  const size_t rstride = (size_t)8 * np;  // rows wq, wq + 8, ...
  auto fetch = [&](int s0) {
    const int m = s0 + lane;
    const bool mok = m < k1;
    int b = 0, q = 0, Y = 0, X = 0;
    if (mok) {
      b = (unsigned)m / (unsigned)np;
      q = m - b * np;
      Y = (unsigned)q / (unsigned)a.Wp;
      X = q - Y * a.Wp;
    }
    const float* ab = a.a + ((size_t)b * a.M + wq) * np + q;
#pragma unroll
    for (int i = 0; i < RA; ++i) ra[i] = mok && wq + 8 * i < a.M ? ab[i * rstride] : 0.f;
    const int gy0 = a.s * Y - a.p, gx0 = a.s * X - a.p;
    const float* gb = a.g + (size_t)b * a.CG * gplane + (gy0 * a.Wg + gx0);
#pragma unroll
    for (int j = 0; j < RG; ++j) {
      const int e = tab[wq + 8 * j];
      rg[j] = mok && e >= 0 && (unsigned)(gy0 + ((e >> 2) & 3)) < (unsigned)a.Hg &&
                      (unsigned)(gx0 + (e & 3)) < (unsigned)a.Wg
                  ? gb[e >> 4]
                  : 0.f;
    }
  };
  __syncthreads();  // the column table
  if (k0 < k1) fetch(k0);
  // this lane's stage slots: row wq + 8 i sits in 16-byte group (lane / 4) ^ ((row / 4) mod 8)
  const int so = lane & 3, sg = lane >> 2;
  const int xa = tm & 7, xg = tn & 7;
  for (int s0 = k0; s0 < k1; s0 += 32) {
    __syncthreads();  // the previous stage's reads are done
#pragma unroll
    for (int i = 0; i < RA; ++i) {
      const int r = wq + 8 * i;
      As[r * 32 + ((sg ^ ((r >> 2) & 7)) << 2) + so] = ra[i];
    }
#pragma unroll
    for (int j = 0; j < RG; ++j) {
      const int c = wq + 8 * j;
      Gs[c * 32 + ((sg ^ ((c >> 2) & 7)) << 2) + so] = rg[j];
    }
    __syncthreads();
    if (s0 + 32 < k1) fetch(s0 + 32);
    if (act) {
#pragma unroll
      for (int g2 = 0; g2 < NGRP; ++g2) {
        const int grp = kg + g2 * KG;
        if (grp >= 8) break;
        const float* ap = As + tm * 128 + ((grp ^ xa) << 2);
        const float* gp = Gs + tn * 128 + ((grp ^ xg) << 2);
        float4 av[4], gv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = *(const float4*)(ap + 32 * i);
#pragma unroll
        for (int j = 0; j < 4; ++j) gv[j] = *(const float4*)(gp + 32 * j);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[i][j] += av[i].x * gv[j].x;
            acc[i][j] += av[i].y * gv[j].y;
            acc[i][j] += av[i].z * gv[j].z;
            acc[i][j] += av[i].w * gv[j].w;
          }
      }
    }
  }
  if (KG > 1) {
    if (act) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) red[(kg * 16 + i * 4 + j) * P + pos] = acc[i][j];
    }
    __syncthreads();
    if (kg == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float r = red[(i * 4 + j) * P + pos];
#pragma unroll
          for (int k = 1; k < KG; ++k) r += red[(k * 16 + i * 4 + j) * P + pos];
          acc[i][j] = r;
        }
    }
  }
  if (kg == 0) {
    float* out = a.part + (size_t)blockIdx.x * a.M * a.N;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int row = tm * 4 + i, col = n0 + tn * 4 + j;
        if (row < a.M && col < a.N) out[(size_t)row * a.N + col] = acc[i][j];
      }
  }
}

__device__ float block_sum(float v, float* sh) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  float r = 0.f;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
  return r;  // valid in thread 0
}

// Weight gradient of NT channel pairs of a conv (or of a transposed conv
// when TR) over one slice of the flattened (window, pixel) domain: pixels
// [blockIdx.y S, blockIdx.y S + S) of the B n pixels (n = Ho Wo for a conv,
// H W for a transposed conv). One block per pair tile, the shared operand
// (dy of output o for a conv, x of input i for a transposed conv) loaded once
// per pixel for the NT pairs; per value a warp shuffle reduction, then one
// pass over the warps; part[slice][pair * k * k + tap].
// K is the kernel size (1, 3 or 4) as a template argument, so the sums stay
// in registers.
template <bool TR, int K, int NT>
__global__ void k_wgrad(const float* __restrict__ x, const float* __restrict__ dy, float* __restrict__ part,
                        int B, int Ci, int H, int W, int Co, int s, int p, int g, int Ho, int Wo,
                        int npairs, int S) {
  constexpr int k = K, KK = K * K, NV = NT * KK;
  __shared__ float sh[32 * NV];
  const int tile = blockIdx.x, chunk = blockIdx.y;
  const int cig = Ci / g, cog = Co / g;
  const long npix = TR ? (long)H * W : (long)Ho * Wo;
  const long e0 = (long)chunk * S, e1 = min((long)B * npix, e0 + S);
  int i, o, pair0;
  if (!TR) {  // pairs o * cig + il, il = il0 .. il0 + NT - 1
    o = tile / (cig / NT);
    const int il0 = (tile % (cig / NT)) * NT;
    i = (o / cog) * cig + il0;
    pair0 = o * cig + il0;
  } else {    // pairs i * cog + ol, ol = ol0 .. ol0 + NT - 1
    i = tile / (cog / NT);
    const int ol0 = (tile % (cog / NT)) * NT;
    o = (i / cig) * cog + ol0;
    pair0 = i * cog + ol0;
  }
  float acc[NT][KK];
#pragma unroll
  for (int j = 0; j < NT; ++j)
#pragma unroll
    for (int t = 0; t < KK; ++t) acc[j][t] = 0.f;
  if (!TR) {
    const int n = Ho * Wo;
    for (int b = (int)(e0 / n); (long)b * n < e1; ++b) {
      const float* xp = x + ((size_t)b * Ci + i) * H * W;
      const float* dp = dy + ((size_t)b * Co + o) * n;
      const int q0 = (int)max(e0 - (long)b * n, 0L), q1 = (int)min(e1 - (long)b * n, (long)n);
      for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        int Y = q / Wo, X = q % Wo;
        float d = dp[q];
#pragma unroll
        for (int ky = 0; ky < k; ++ky) {
          int yy = Y * s - p + ky;
          if (yy < 0 || yy >= H) continue;
#pragma unroll
          for (int kx = 0; kx < k; ++kx) {
            int xx = X * s - p + kx;
            if (xx < 0 || xx >= W) continue;
#pragma unroll
            for (int j = 0; j < NT; ++j) acc[j][ky * k + kx] += d * xp[(size_t)j * H * W + yy * W + xx];
          }
        }
      }
    }
  } else {
    const int n = H * W;
    for (int b = (int)(e0 / n); (long)b * n < e1; ++b) {
      const float* xp = x + ((size_t)b * Ci + i) * n;
      const float* dp = dy + ((size_t)b * Co + o) * Ho * Wo;
      const int q0 = (int)max(e0 - (long)b * n, 0L), q1 = (int)min(e1 - (long)b * n, (long)n);
      for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        int yi = q / W, xi = q % W;
        float v = xp[q];
#pragma unroll
        for (int ky = 0; ky < k; ++ky) {
          int Y = yi * s - p + ky;
          if (Y < 0 || Y >= Ho) continue;
#pragma unroll
          for (int kx = 0; kx < k; ++kx) {
            int X = xi * s - p + kx;
            if (X < 0 || X >= Wo) continue;
#pragma unroll
            for (int j = 0; j < NT; ++j) acc[j][ky * k + kx] += v * dp[(size_t)j * Ho * Wo + Y * Wo + X];
          }
        }
      }
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < NT; ++j)
#pragma unroll
    for (int t = 0; t < KK; ++t) {
      float v = acc[j][t];
#pragma unroll
      for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) sh[warp * NV + j * KK + t] = v;
    }
  __syncthreads();
  for (int v = threadIdx.x; v < NV; v += blockDim.x) {
    float r = 0.f;
    for (int w = 0; w < nw; ++w) r += sh[w * NV + v];
    part[(size_t)chunk * npairs * KK + (size_t)pair0 * KK + v] = r;
  }
}

// Per-channel sums over one slice (pixels [chunk S, chunk S + S) of the B n):
// S1 = sum a, S2 = sum a (v - mean) / sqrt(var + eps) (S2 only if v);
// part[chunk][c][2].
template <int V>
__global__ void k_chan_sums(const float* __restrict__ a, const float* __restrict__ v, const float* __restrict__ mean,
                            const float* __restrict__ var, float* __restrict__ part, int B, int C, int n, int S) {
  __shared__ float sh[32];
  const int c = blockIdx.x, chunk = blockIdx.y;
  const long e0 = (long)chunk * S, e1 = min((long)B * n, e0 + S);
  float s1 = 0.f, s2 = 0.f;
  float m = v ? mean[c] : 0.f, is = v ? rsqrtf(var[c] + 1e-5f) : 0.f;
  for (int b = (int)(e0 / n); (long)b * n < e1; ++b) {
    const float* ap = a + ((size_t)b * C + c) * n;
    const float* vp = v ? v + ((size_t)b * C + c) * n : nullptr;
    const int q0 = (int)max(e0 - (long)b * n, 0L), q1 = (int)min(e1 - (long)b * n, (long)n);
    for (int q = q0 + V * threadIdx.x; q < q1; q += V * blockDim.x) {
      float d[V], u[V];
      ldv<V>(ap + q, d);
      if (vp) ldv<V>(vp + q, u);
#pragma unroll
      for (int e = 0; e < V; ++e) {
        s1 += d[e];
        if (vp) s2 += d[e] * (u[e] - m) * is;
      }
    }
  }
  float r1 = block_sum(s1, sh);
  float r2 = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    part[((size_t)chunk * C + c) * 2] = r1;
    part[((size_t)chunk * C + c) * 2 + 1] = r2;
  }
}

// Stage 1 of a block, adjoint side, in one pass: dv = dx1 [x1 > 0] (written
// back into dx1) and per channel over one slice of the pixels the four sums
// S0 = sum dv and Sk = sum dv (u_k - mean_k) / sqrt(var_k + eps) for the
// inputs u_1 = t1, u_2 = t2, u_3 = x of the three BNs (dbeta_k = S0,
// dgamma_k = Sk); part[chunk][c][4].
struct Bn3 {
  const float *m1, *v1, *m2, *v2, *m3, *v3;
};
template <int V>
__global__ void k_stage1_sums(float* __restrict__ dx1, const float* __restrict__ x1, const float* __restrict__ t1,
                              const float* __restrict__ t2, const float* __restrict__ x, Bn3 bn,
                              float* __restrict__ part, int B, int C, int n, int S) {
  __shared__ float sh[32];
  const int c = blockIdx.x, chunk = blockIdx.y;
  const long e0 = (long)chunk * S, e1 = min((long)B * n, e0 + S);
  const float m1 = bn.m1[c], i1 = rsqrtf(bn.v1[c] + 1e-5f), m2 = bn.m2[c], i2 = rsqrtf(bn.v2[c] + 1e-5f);
  const float m3 = bn.m3[c], i3 = rsqrtf(bn.v3[c] + 1e-5f);
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  for (int b = (int)(e0 / n); (long)b * n < e1; ++b) {
    const size_t base = ((size_t)b * C + c) * n;
    const int q0 = (int)max(e0 - (long)b * n, 0L), q1 = (int)min(e1 - (long)b * n, (long)n);
    for (int q = q0 + V * threadIdx.x; q < q1; q += V * blockDim.x) {
      float d[V], a[V], u1[V], u2[V], u3[V];
      ldv<V>(dx1 + base + q, d);
      ldv<V>(x1 + base + q, a);
      ldv<V>(t1 + base + q, u1);
      ldv<V>(t2 + base + q, u2);
      ldv<V>(x + base + q, u3);
#pragma unroll
      for (int e = 0; e < V; ++e) {
        d[e] = a[e] > 0.f ? d[e] : 0.f;
        s0 += d[e];
        s1 += d[e] * (u1[e] - m1) * i1;
        s2 += d[e] * (u2[e] - m2) * i2;
        s3 += d[e] * (u3[e] - m3) * i3;
      }
      stv<V>(dx1 + base + q, d);
    }
  }
  const float r0 = block_sum(s0, sh), r1 = block_sum(s1, sh), r2 = block_sum(s2, sh), r3 = block_sum(s3, sh);
  if (threadIdx.x == 0) {
    float* o = part + ((size_t)chunk * C + c) * 4;
    o[0] = r0;
    o[1] = r1;
    o[2] = r2;
    o[3] = r3;
  }
}
// Stage 2 of a block, adjoint side, in one pass: dbn = dy [BN(u) > 0], per
// channel over one slice S1 = sum dbn and S2 = sum dbn (u - mean) / sqrt(var
// + eps) (dbeta, dgamma; part[chunk][c][2]), and out = dbn, or (scale: BN
// with running statistics) out = dbn gam / sqrt(var + eps), the BN input's
// adjoint.
template <int V>
__global__ void k_stage2_sums(const float* __restrict__ dy, const float* __restrict__ u, BnP bn,
                              float* __restrict__ out, float* __restrict__ part, int B, int C, int n, int S,
                              int scale) {
  __shared__ float sh[32];
  const int c = blockIdx.x, chunk = blockIdx.y;
  const long e0 = (long)chunk * S, e1 = min((long)B * n, e0 + S);
  const float is = rsqrtf(bn.v[c] + 1e-5f), m = bn.m[c], g = bn.g[c], be = bn.b[c], f = scale ? g * is : 1.f;
  float s1 = 0.f, s2 = 0.f;
  for (int b = (int)(e0 / n); (long)b * n < e1; ++b) {
    const size_t base = ((size_t)b * C + c) * n;
    const int q0 = (int)max(e0 - (long)b * n, 0L), q1 = (int)min(e1 - (long)b * n, (long)n);
    for (int q = q0 + V * threadIdx.x; q < q1; q += V * blockDim.x) {
      float d[V], a[V];
      ldv<V>(dy + base + q, d);
      ldv<V>(u + base + q, a);
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const float xh = (a[e] - m) * is;
        d[e] = g * xh + be > 0.f ? d[e] : 0.f;
        s1 += d[e];
        s2 += d[e] * xh;
        d[e] *= f;
      }
      stv<V>(out + base + q, d);
    }
  }
  const float r1 = block_sum(s1, sh), r2 = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    part[((size_t)chunk * C + c) * 2] = r1;
    part[((size_t)chunk * C + c) * 2 + 1] = r2;
  }
}
// part[chunk][c][4] of k_stage1_sums summed over chunks in FP64, one warp per
// (c, k) as k_reduce_few: S0 is added to the three dbeta, Sk to dgamma_k.
__global__ void __launch_bounds__(256) k_reduce_stage1(const float* __restrict__ part, int nchunks, int C,
                                                       double* __restrict__ acc, long b1, long b2, long b3, long g1,
                                                       long g2, long g3) {
  const int lane = threadIdx.x & 31, j = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (j >= 4 * C) return;
  double s = 0.0;
  for (int ch = lane; ch < nchunks; ch += 32) s += (double)part[(size_t)ch * 4 * C + j];
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane) return;
  const int c = j >> 2, k = j & 3;
  if (k == 0) {
    acc[b1 + c] += s;
    acc[b2 + c] += s;
    acc[b3 + c] += s;
  } else {
    acc[(k == 1 ? g1 : k == 2 ? g2 : g3) + c] += s;
  }
}

// Sums partials over chunks in FP64 and adds them into the gradient
// accumulator, acc[dst + j] += sum_chunk part[chunk][j * stride + off], or
// (fout) writes fout[j] = scale * that sum. 256 threads: lane = output j of a
// group of 32, warp w sums chunks w, w + 8, ...; the 8 warp sums are added in
// warp order, so the result does not depend on timing.
__global__ void __launch_bounds__(256) k_reduce(const float* __restrict__ part, int nchunks, int n, int stride,
                                                int off, double* __restrict__ acc, long dst,
                                                float* __restrict__ fout, double scale) {
  __shared__ double sh[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, j = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (j < n) {
    const float* src = part + (size_t)j * stride + off;
    const size_t cs = (size_t)n * stride;
    int c = w;
    for (; c + 24 < nchunks; c += 32) {
      const float v0 = src[c * cs], v1 = src[(c + 8) * cs], v2 = src[(c + 16) * cs], v3 = src[(c + 24) * cs];
      s += (double)v0;
      s += (double)v1;
      s += (double)v2;
      s += (double)v3;
    }
    for (; c < nchunks; c += 8) s += (double)src[c * cs];
  }
  sh[w][lane] = s;
  __syncthreads();
  if (w == 0 && j < n) {
    double r = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) r += sh[k][lane];
    if (fout)
      fout[j] = (float)(r * scale);
    else
      acc[dst + j] += r;
  }
}

// The same for few outputs: one warp per output j (of n), its lanes summing
// chunks lane, lane + 32, ... in order, then a fixed shuffle tree. With
// dst_odd >= 0 the partials are [chunk][n / 2][2] pairs: even j go to
// acc[dst + j / 2], odd j to acc[dst_odd + j / 2].
__global__ void __launch_bounds__(256) k_reduce_few(const float* __restrict__ part, int nchunks, int n, int stride,
                                                    int off, double* __restrict__ acc, long dst, long dst_odd,
                                                    float* __restrict__ fout, double scale) {
  const int lane = threadIdx.x & 31, j = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (j >= n) return;
  const float* src = part + (size_t)j * stride + off;
  const size_t cs = (size_t)n * stride;
  double s = 0.0;
  for (int c = lane; c < nchunks; c += 32) s += (double)src[c * cs];
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane) return;
  if (fout)
    fout[j] = (float)(s * scale);
  else if (dst_odd >= 0)
    acc[((j & 1) ? dst_odd : dst) + (j >> 1)] += s;
  else
    acc[dst + j] += s;
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ out, int n) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = (float)a[j];
}

// y = relu?(gam (x - mean) / sqrt(var + eps) + bet) per channel
template <int V>
__global__ void k_bn(const float* __restrict__ x, float* __restrict__ y, const float* __restrict__ gam,
                     const float* __restrict__ bet, const float* __restrict__ mean, const float* __restrict__ var,
                     int planes, int C, int n, int relu) {
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) * V;
  if (q >= n) return;
  for (int pl = blockIdx.y; pl < planes; pl += gridDim.y) {
    const int c = pl % C;
    const size_t idx = (size_t)pl * n + q;
    const float g = gam[c] * rsqrtf(var[c] + 1e-5f), m = mean[c], b = bet[c];
    float v[V];
    ldv<V>(x + idx, v);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const float o = g * (v[e] - m) + b;
      v[e] = relu ? fmaxf(o, 0.f) : o;
    }
    stv<V>(y + idx, v);
  }
}

// stage 1: x1 = ReLU(BN1(t1) + BN2(t2) + BN3(x))
template <int V>
__global__ void k_stage1(const float* t1, const float* t2, const float* x, float* x1, BnP b1, BnP b2, BnP b3,
                         int planes, int C, int n) {
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) * V;
  if (q >= n) return;
  for (int pl = blockIdx.y; pl < planes; pl += gridDim.y) {
    const int c = pl % C;
    const size_t idx = (size_t)pl * n + q;
    float a1[V], a2[V], a3[V];
    ldv<V>(t1 + idx, a1);
    ldv<V>(t2 + idx, a2);
    ldv<V>(x + idx, a3);
#pragma unroll
    for (int e = 0; e < V; ++e) a1[e] = fmaxf(bnv(b1, c, a1[e]) + bnv(b2, c, a2[e]) + bnv(b3, c, a3[e]), 0.f);
    stv<V>(x1 + idx, a1);
  }
}
// y = ReLU(BN(u)) + r
template <int V>
__global__ void k_stage2(const float* u, const float* r, float* y, BnP bn, int planes, int C, int n) {
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) * V;
  if (q >= n) return;
  for (int pl = blockIdx.y; pl < planes; pl += gridDim.y) {
    const int c = pl % C;
    const size_t idx = (size_t)pl * n + q;
    float a[V], b[V];
    ldv<V>(u + idx, a);
    ldv<V>(r + idx, b);
#pragma unroll
    for (int e = 0; e < V; ++e) a[e] = fmaxf(bnv(bn, c, a[e]), 0.f) + b[e];
    stv<V>(y + idx, a);
  }
}

// per (b, c): g = mean over the map
template <int V>
__global__ void k_gap(const float* __restrict__ y, float* __restrict__ g, int n) {
  __shared__ float sh[32];
  const float* p = y + (size_t)blockIdx.x * n;
  float s = 0.f;
  for (int q = V * threadIdx.x; q < n; q += V * blockDim.x) {
    float v[V];
    ldv<V>(p + q, v);
#pragma unroll
    for (int e = 0; e < V; ++e) s += v[e];
  }
  float r = block_sum(s, sh);
  if (threadIdx.x == 0) g[blockIdx.x] = r / (float)n;
}
// per (b, c): s = sigmoid(conv1d_k3(g))
__global__ void k_eca_s(const float* g, const float* k3, float* sc, int B, int C) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * C) return;
  int c = idx % C;
  const float* gb = g + (idx - c);
  float z = k3[1] * gb[c];
  if (c > 0) z += k3[0] * gb[c - 1];
  if (c + 1 < C) z += k3[2] * gb[c + 1];
  sc[idx] = 1.f / (1.f + expf(-z));
}
// out = s * y (+ skip)
template <int V>
__global__ void k_scale(const float* y, const float* sc, const float* skip, float* out, int planes, int n) {
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) * V;
  if (q >= n) return;
  for (int pl = blockIdx.y; pl < planes; pl += gridDim.y) {
    const size_t idx = (size_t)pl * n + q;
    const float s = sc[pl];
    float a[V], b[V];
    ldv<V>(y + idx, a);
    if (skip) ldv<V>(skip + idx, b);
#pragma unroll
    for (int e = 0; e < V; ++e) a[e] = skip ? s * a[e] + b[e] : s * a[e];
    stv<V>(out + idx, a);
  }
}

// output: z = sigmoid(logit); MSE gradient (or given gout) -> dlogit;
// per-block FP64 loss partials
__global__ void k_out_loss(const float* logit, const float* target, const float* gout, float* z, float* dlogit,
                           double* loss_part, long total, double inv_n) {
  __shared__ double sh[32];
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double e2 = 0.0;
  if (idx < total) {
    float zz = 1.f / (1.f + expf(-logit[idx]));
    z[idx] = zz;
    float g;
    if (target) {
      double e = (double)zz - (double)target[idx];
      e2 = e * e * inv_n;
      g = (float)(2.0 * e * inv_n);
    } else {
      g = gout[idx];
    }
    dlogit[idx] = g * zz * (1.f - zz);
  }
  for (int o = 16; o; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[warp] = e2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
    loss_part[blockIdx.x] = s;
  }
}
// *out = sum of part[0 .. n), one block of 256 threads: thread t sums
// t, t + 256, ... in order, then a fixed tree over the threads.
__global__ void __launch_bounds__(256) k_sum_f64(const double* part, int n, double* out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += part[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h; h >>= 1) {
    if ((int)threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// ---------------------------------------------------------- backward ops
// per (b, c): ds = sum dout * y
template <int V>
__global__ void k_eca_ds(const float* dout, const float* y, float* ds, int n) {
  __shared__ float sh[32];
  const float* a = dout + (size_t)blockIdx.x * n;
  const float* v = y + (size_t)blockIdx.x * n;
  float s = 0.f;
  for (int q = V * threadIdx.x; q < n; q += V * blockDim.x) {
    float x[V], z[V];
    ldv<V>(a + q, x);
    ldv<V>(v + q, z);
#pragma unroll
    for (int e = 0; e < V; ++e) s += x[e] * z[e];
  }
  float r = block_sum(s, sh);
  if (threadIdx.x == 0) ds[blockIdx.x] = r;
}
// per window b (one block, thread = channel c < C <= 64): dz = ds s (1 - s);
// dg[c] = sum_j dz[c + 1 - j] k3[j] / n (the mean's adjoint); dk partial
// dk[j] = sum_c dz[c] g[c + j - 1], summed over the block in a fixed order
__global__ void k_eca_back(const float* ds, const float* sc, const float* g, const float* k3, float* dgm,
                           float* dk_part, int B, int C, int n) {
  __shared__ float dz[64];
  __shared__ float sh[32];
  const int b = blockIdx.x, c = threadIdx.x;
  if (c < C) {
    const float s = sc[b * C + c];
    dz[c] = ds[b * C + c] * s * (1.f - s);
  }
  __syncthreads();
  if (c < C) {
    float v = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int cc = c + 1 - j;
      if (cc >= 0 && cc < C) v += dz[cc] * k3[j];
    }
    dgm[b * C + c] = v / (float)n;
  }
  for (int j = 0; j < 3; ++j) {
    const int cg = c + j - 1;
    const float t = block_sum(c < C && cg >= 0 && cg < C ? dz[c] * g[b * C + cg] : 0.f, sh);
    if (c == 0) dk_part[b * 3 + j] = t;
  }
}
// dy = s * dout + dg (the mean's adjoint, already divided by n)
template <int V>
__global__ void k_eca_dy(const float* dout, const float* sc, const float* dgm, float* dy, int planes, int n) {
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) * V;
  if (q >= n) return;
  for (int pl = blockIdx.y; pl < planes; pl += gridDim.y) {
    const size_t idx = (size_t)pl * n + q;
    const float s = sc[pl], d = dgm[pl];
    float a[V];
    ldv<V>(dout + idx, a);
#pragma unroll
    for (int e = 0; e < V; ++e) a[e] = s * a[e] + d;
    stv<V>(dy + idx, a);
  }
}
// out (+)= a * gam / sqrt(var + eps)
template <int V>
__global__ void k_bn_dx(const float* a, BnP bn, float* out, int planes, int C, int n, int accumulate) {
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) * V;
  if (q >= n) return;
  for (int pl = blockIdx.y; pl < planes; pl += gridDim.y) {
    const int c = pl % C;
    const size_t idx = (size_t)pl * n + q;
    const float g = bn.g[c] * rsqrtf(bn.v[c] + 1e-5f);
    float v[V], o[V];
    ldv<V>(a + idx, v);
    if (accumulate) ldv<V>(out + idx, o);
#pragma unroll
    for (int e = 0; e < V; ++e) v[e] = accumulate ? o[e] + v[e] * g : v[e] * g;
    stv<V>(out + idx, v);
  }
}
// Batch statistics of a BN input x[B][C][n]: part[chunk][c] = sum over the
// slice's pixels (chunk S .. chunk S + S of the B n) of x (mean == null) or
// of (x - mean[c])^2.
template <int V>
__global__ void k_bn_part(const float* __restrict__ x, const float* __restrict__ mean, float* __restrict__ part,
                          int B, int C, int n, int S) {
  __shared__ float sh[32];
  const int c = blockIdx.x, chunk = blockIdx.y;
  const long e0 = (long)chunk * S, e1 = min((long)B * n, e0 + S);
  const float m = mean ? mean[c] : 0.f;
  float s = 0.f;
  for (int b = (int)(e0 / n); (long)b * n < e1; ++b) {
    const float* p = x + ((size_t)b * C + c) * n;
    const int q0 = (int)max(e0 - (long)b * n, 0L), q1 = (int)min(e1 - (long)b * n, (long)n);
    for (int q = q0 + V * threadIdx.x; q < q1; q += V * blockDim.x) {
      float u[V];
      ldv<V>(p + q, u);
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const float d = u[e] - m;
        s += mean ? d * d : u[e];
      }
    }
  }
  const float r = block_sum(s, sh);
  if (threadIdx.x == 0) part[(size_t)chunk * C + c] = r;
}
// Batch-statistics BN adjoint: out (+)= gam / sigma (dy - (sum dy + xhat sum
// dy xhat) / N), the two sums of this BN being gacc[dbet + c], gacc[dgam + c];
// invN = 1 / N.
template <int V>
__global__ void k_bn_dx_batch(const float* dy, const float* x, BnP bn, const double* __restrict__ gacc, long dgam,
                              long dbet, float invN, float* out, int planes, int C, int n, int accumulate) {
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) * V;
  if (q >= n) return;
  for (int pl = blockIdx.y; pl < planes; pl += gridDim.y) {
    const int c = pl % C;
    const size_t idx = (size_t)pl * n + q;
    const float is = rsqrtf(bn.v[c] + 1e-5f), m = bn.m[c], g = bn.g[c] * is;
    // (sum dy + xhat sum dy xhat) / N as cb + xhat cg, the two channel means in FP32
    const float cb = (float)gacc[dbet + c] * invN, cg = (float)gacc[dgam + c] * invN;
    float d[V], xv[V], o[V];
    ldv<V>(dy + idx, d);
    ldv<V>(x + idx, xv);
    if (accumulate) ldv<V>(out + idx, o);
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const float xh = (xv[e] - m) * is;
      const float v = g * (d[e] - (cb + xh * cg));
      d[e] = accumulate ? o[e] + v : v;
    }
    stv<V>(out + idx, d);
  }
}
// dv = dx1 [x1 > 0]
template <int V>
__global__ void k_relu_mask(const float* d, const float* act, float* out, long total) {
  const long idx = ((long)blockIdx.x * blockDim.x + threadIdx.x) * V;
  if (idx >= total) return;
  float a[V], b[V];
  ldv<V>(d + idx, a);
  ldv<V>(act + idx, b);
#pragma unroll
  for (int e = 0; e < V; ++e) a[e] = b[e] > 0.f ? a[e] : 0.f;
  stv<V>(out + idx, a);
}
template <int V>
__global__ void k_add(float* a, const float* b, long total) {
  const long idx = ((long)blockIdx.x * blockDim.x + threadIdx.x) * V;
  if (idx >= total) return;
  float x[V], y[V];
  ldv<V>(a + idx, x);
  ldv<V>(b + idx, y);
#pragma unroll
  for (int e = 0; e < V; ++e) x[e] += y[e];
  stv<V>(a + idx, x);
}
__global__ void k_bf16_to_f32(const __nv_bfloat16* a, float* out, long total) {
  const long idx = ((long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (idx + 4 <= total && ((total & 3) == 0) && ((uintptr_t)a & 7) == 0) {
    const uint2 u = *(const uint2*)(a + idx);
    *(float4*)(out + idx) = make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xFFFF0000u),
                                        __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xFFFF0000u));
  } else {
    for (long i = idx; i < min(idx + 4, total); ++i) out[i] = __bfloat162float(a[i]);
  }
}

}  // namespace

// ---------------------------------------------------------------- host
// Canonical parameter and buffer offsets (same order as the parameter blob).
struct Canon {
  int stem_w, stem_g, stem_b, stem_m, stem_v;
  int w1[6], g1[6], b1[6], w3[6], g2[6], b2[6], g3[6], b3[6], w2[6], g[6], be[6], rw[6], rb[6], eca[6];
  int m1[6], v1[6], m2[6], v2[6], m3[6], v3[6], m[6], v[6];
  int out_w, out_b;
};

static Canon canon() {
  Canon o;
  int p = 0, q = 0;
  o.stem_w = p; p += 216;
  o.stem_g = p; p += 8;
  o.stem_b = p; p += 8;
  o.stem_m = q; q += 8;
  o.stem_v = q; q += 8;
  for (int b = 0; b < kNumBlocks; ++b) {
    int ci = kBlkCin[b], co = kBlkCout[b], dense = (kBlkEnc[b] ? 9 : 16) * ci * co;
    o.w1[b] = p; p += ci;
    o.g1[b] = p; p += ci;
    o.b1[b] = p; p += ci;
    o.w3[b] = p; p += 9 * ci;
    o.g2[b] = p; p += ci;
    o.b2[b] = p; p += ci;
    o.g3[b] = p; p += ci;
    o.b3[b] = p; p += ci;
    o.w2[b] = p; p += dense;
    o.g[b] = p; p += co;
    o.be[b] = p; p += co;
    o.rw[b] = p; p += dense;
    o.rb[b] = p; p += co;
    o.eca[b] = p; p += 3;
    o.m1[b] = q; q += ci;
    o.v1[b] = q; q += ci;
    o.m2[b] = q; q += ci;
    o.v2[b] = q; q += ci;
    o.m3[b] = q; q += ci;
    o.v3[b] = q; q += ci;
    o.m[b] = q; q += co;
    o.v[b] = q; q += co;
  }
  o.out_w = p; p += 72;
  o.out_b = p;
  return o;
}

namespace {
// Bump allocator over one device buffer.
struct Arena {
  char* base;
  size_t off, cap;
  float* f(size_t n) { return (float*)take(n * sizeof(float)); }
  double* d(size_t n) { return (double*)take(n * sizeof(double)); }
  void* take(size_t bytes) {
    size_t o = (off + 255) / 256 * 256;
    off = o + bytes;
    return base ? base + o : nullptr;
  }
};

struct BlkTape {
  int h, w, H2, W2;
  float *x, *t1, *t2, *x1, *u, *r, *y, *g, *s, *out;
};
}  // namespace

size_t train_workspace_bytes(int B, int H, int W) {
  TrainArgs a{};
  a.B = B;
  a.H = H;
  a.W = W;
  Arena ar{nullptr, 0, 0};
  return train_step_plan(a, &ar);
}

// Plans (base == nullptr) or runs the whole training step. Returns the
// workspace bytes used.
size_t train_step_plan(const TrainArgs& a, void* arena_v) {
  Arena& ar = *(Arena*)arena_v;
  const bool run = ar.base != nullptr;
  const Canon C = canon();
  const int B = a.B, H = a.H, W = a.W;
  const size_t n0 = (size_t)H * W;
  cudaStream_t st = a.stream;
  const float* P = a.params;
  // elementwise launches: 4 elements per thread where the plane (or the
  // whole tensor) holds a multiple of 4
  auto plane_launch = [&](long tot, long n, auto k4, auto k1, auto... args) {
    if (n % 4 == 0)
      k4<<<dim3(cdiv(n / 4, kT), (unsigned)std::min(tot / n, 65535L)), kT, 0, st>>>(args...);
    else
      k1<<<gridp(tot, n), kT, 0, st>>>(args...);
  };
  auto lin_launch = [&](long tot, auto k4, auto k1, auto... args) {
    if (tot % 4 == 0)
      k4<<<cdiv(tot / 4, kT), kT, 0, st>>>(args...);
    else
      k1<<<cdiv(tot, kT), kT, 0, st>>>(args...);
  };
  // per-slice partial sums of the reductions (weight gradients, channel
  // sums, batch statistics), one launch at a time
  float* part = ar.f(kPartCap);
  double* gacc = ar.d(kNumParams);  // gradient accumulator
  // adds sum_chunk part[chunk][j * stride + off] to gacc[dst + j] (fout:
  // writes fout[j] = scale * that sum)
  auto reduce = [&](const float* pp, int nch, int n, int stride, int off, long dst, float* fout = nullptr,
                    double scale = 1.0) {
    if (n <= 1024)
      k_reduce_few<<<cdiv(n, 8), 256, 0, st>>>(pp, nch, n, stride, off, gacc, dst, -1, fout, scale);
    else
      k_reduce<<<cdiv(n, 32), 256, 0, st>>>(pp, nch, n, stride, off, gacc, dst, fout, scale);
  };
  // BN statistics: the running ones, or (training mode) the batch's, computed
  // into `bst` (same layout as the running buffers) right before each BN
  float* bst = ar.f(kNumBuffers);
  const float* Q = a.bn_batch ? bst : a.buffers;
  auto bnp = [&](int g, int b, int m, int v) { return BnP{P + g, P + b, Q + m, Q + v}; };
  auto batch_stats = [&](const float* x, int Cc, int n, int moff, int voff) {
    if (!run || !a.bn_batch) return;
    const double N = (double)B * n;
    const Slices sl = slices((long)B * n, Cc, Cc, 4, kSliceBlocks);
    auto bn_part = n % 4 == 0 ? k_bn_part<4> : k_bn_part<1>;
    bn_part<<<dim3(Cc, sl.n), kT, 0, st>>>(x, nullptr, part, B, Cc, n, sl.S);
    reduce(part, sl.n, Cc, 1, 0, 0, bst + moff, 1.0 / N);
    bn_part<<<dim3(Cc, sl.n), kT, 0, st>>>(x, bst + moff, part, B, Cc, n, sl.S);
    reduce(part, sl.n, Cc, 1, 0, 0, bst + voff, 1.0 / N);
  };

  // ---- forward with tape
  float* xin = ar.f((size_t)B * 3 * n0);
  if (run) {
    if (a.in_bf16)
      k_bf16_to_f32<<<cdiv((long)B * 3 * n0, 4 * kT), kT, 0, st>>>((const __nv_bfloat16*)a.in, xin, (long)B * 3 * n0);
    else
      cudaMemcpyAsync(xin, a.in, sizeof(float) * B * 3 * n0, cudaMemcpyDeviceToDevice, st);
  }
  // dense stride-2 convs (and their input gradients) as tiled GEMMs
  auto igemm = [&](int cse, const float* src, const float* w, const float* bias, float* out, int Cs, int Hs,
                   int Ws, int N, int Ho, int Wo) {
    GemmArgs ga{src, w, bias, out, B, Cs, Hs, Ws, N, Ho, Wo, 0};
    const long rows = cse == ENC_FWD ? (long)Ho * Wo
                      : cse == DEC_FWD ? (long)Hs * Ws
                      : cse == ENC_DGRAD ? (long)(Ho / 2) * (Wo / 2)
                                         : (long)Ho * Wo;
    const int bn = N >= 64 ? 64 : N >= 32 ? 32 : 16, bm = 4096 / bn;
    dim3 grid(cdiv((long)B * rows, bm), cdiv(N, bn), (cse == DEC_FWD || cse == ENC_DGRAD) ? 4 : 1);
    auto go = [&](auto kern) { kern<<<grid, 256, 0, st>>>(ga); };
#define STDA_IGEMM(C)                                                  \
  (bn == 64 ? go(k_igemm<C, 64>) : bn == 32 ? go(k_igemm<C, 32>) : go(k_igemm<C, 16>))
    if (cse == ENC_FWD) STDA_IGEMM(ENC_FWD);
    else if (cse == DEC_FWD) STDA_IGEMM(DEC_FWD);
    else if (cse == ENC_DGRAD) STDA_IGEMM(ENC_DGRAD);
    else STDA_IGEMM(DEC_DGRAD);
#undef STDA_IGEMM
  };
  auto dense_s2 = [](int k, int s, int p, int g, bool tr) { return g == 1 && s == 2 && p == 1 && k == (tr ? 4 : 3); };
  // direct stride-2 conv (T: transposed) of src [B][M][Hs][Ws] into N channels
  float* wT = ar.f(kDcWT);  // a dense conv's weights as [m][tap][n]
  // the direct form applies: N a multiple of the block's channels, even maps,
  // and for the transposed form a source width that is a multiple of 4
  auto dconv_ok = [](bool T, int M, int Hs, int Ws, int N, int K) {
    const int no = N >= 32 ? 16 : N >= 16 ? 8 : 4;
    return N % (2 * no) == 0 && Hs % 2 == 0 && Ws % 2 == 0 && (!T || Ws % 4 == 0) && (long)M * N * K * K <= kDcWT;
  };
  auto dconv = [&](bool T, int K, const float* src, const float* w, const float* bias, float* out, int M, int Hs,
                   int Ws, int N, int accumulate) {
    k_wt<<<cdiv((long)M * K * K * N, kT), kT, 0, st>>>(w, wT, M, N, K * K, T ? 1 : 0);
    const int no = N >= 32 ? 16 : N >= 16 ? 8 : 4;
    const int tx = (T ? Ws : Ws / 2) >= 32 ? 32 : 16;
    // pixels per thread: 2 with 16 channels; with 4 or 8 channels 4 (the
    // weights feed more FMAs) where that still gives about six blocks per SM
    auto tiles_for = [&](int np) {
      const int rw = 32 / tx;
      return T ? cdiv(Ws, tx) * cdiv(Hs, np * rw) : cdiv(Ws / 2, tx) * cdiv(Hs / 2, 4 * np * rw);
    };
    const long want = (long)device_sms() * 6;
    const int np = no < 16 && (long)tiles_for(4) * cdiv(N, 2 * no) * B >= want ? 4 : 2;
    const dim3 grid(tiles_for(np), cdiv(N, 2 * no), B);
    auto go = [&](auto kern, size_t smem) {
      if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      kern<<<grid, 256, smem, st>>>(src, wT, bias, out, M, Hs, Ws, N, accumulate);
    };
#define STDA_DC2(KERN, GEO, KS, NO, TX)                                                            \
  (NO < 16 && np == 4 ? go(KERN<KS, NO, TX, (NO < 16 ? 4 : 2)>, GEO<KS, NO, TX, (NO < 16 ? 4 : 2)>::smem()) \
                      : go(KERN<KS, NO, TX, 2>, GEO<KS, NO, TX, 2>::smem()))
#define STDA_DC(KERN, GEO, KS)                                                                              \
  (no == 16 ? (tx == 32 ? STDA_DC2(KERN, GEO, KS, 16, 32) : STDA_DC2(KERN, GEO, KS, 16, 16))                \
            : no == 8 ? (tx == 32 ? STDA_DC2(KERN, GEO, KS, 8, 32) : STDA_DC2(KERN, GEO, KS, 8, 16))        \
                      : (tx == 32 ? STDA_DC2(KERN, GEO, KS, 4, 32) : STDA_DC2(KERN, GEO, KS, 4, 16)))
    if (T)
      K == 4 ? STDA_DC(k_stconv, StconvGeo, 4) : STDA_DC(k_stconv, StconvGeo, 3);
    else
      K == 4 ? STDA_DC(k_sconv, SconvGeo, 4) : STDA_DC(k_sconv, SconvGeo, 3);
#undef STDA_DC
#undef STDA_DC2
  };
  auto conv = [&](const float* x, const float* w, const float* bias, float* y, int Ci, int h, int wd, int Co,
                  int k, int s, int p, int g, bool tr, int Ho, int Wo) {
    if (!run) return;
    if (dense_s2(k, s, p, g, tr) && dconv_ok(tr, Ci, h, wd, Co, k)) {
      dconv(tr, k, x, w, bias, y, Ci, h, wd, Co, 0);
      return;
    }
    if (g == 1 && s == 1 && p == 1 && k == 3 && !tr && wd % 4 == 0 &&
        ((Ci == 3 && Co == 8) || (Ci == 8 && Co == 1))) {
      const dim3 grid(cdiv((long)h * wd / 4, kT), B);
      if (Ci == 3)
        k_cs1<3, 8, false, false><<<grid, kT, 0, st>>>(x, w, bias, y, h, wd, 0);
      else
        k_cs1<8, 1, false, false><<<grid, kT, 0, st>>>(x, w, bias, y, h, wd, 0);
      return;
    }
    if (dense_s2(k, s, p, g, tr)) {
      igemm(tr ? DEC_FWD : ENC_FWD, x, w, bias, y, Ci, h, wd, Co, Ho, Wo);
      return;
    }
    if (g == Ci && g == Co && s == 1 && p == (k - 1) / 2 && (k == 1 || k == 3)) {
      if (wd % 4 == 0) {
        const dim3 grid(cdiv((long)h * wd / 4, kT), Ci, B);
        if (k == 1)
          k_dw4<1, false><<<grid, kT, 0, st>>>(x, w, bias, y, Ci, h, wd, 0);
        else if (tr)
          k_dw4<3, true><<<grid, kT, 0, st>>>(x, w, bias, y, Ci, h, wd, 0);
        else
          k_dw4<3, false><<<grid, kT, 0, st>>>(x, w, bias, y, Ci, h, wd, 0);
        return;
      }
      const dim3 grid(cdiv((long)h * wd, kT), Ci, B);
      if (k == 1)
        k_dw<1, false><<<grid, kT, 0, st>>>(x, w, bias, y, Ci, h, wd, 0);
      else if (tr)
        k_dw<3, true><<<grid, kT, 0, st>>>(x, w, bias, y, Ci, h, wd, 0);
      else
        k_dw<3, false><<<grid, kT, 0, st>>>(x, w, bias, y, Ci, h, wd, 0);
      return;
    }
    const int nt = (Co / g) % 8 == 0 ? 8 : (Co / g) % 4 == 0 ? 4 : 1;
    const dim3 grid(cdiv((long)Ho * Wo, kT), Co / nt, B);
    auto go = [&](auto kern) { kern<<<grid, kT, 0, st>>>(x, w, bias, y, B, Ci, h, wd, Co, k, s, p, g, Ho, Wo); };
    if (tr)
      nt == 8 ? go(k_convT<8>) : nt == 4 ? go(k_convT<4>) : go(k_convT<1>);
    else
      nt == 8 ? go(k_conv<8>) : nt == 4 ? go(k_conv<4>) : go(k_conv<1>);
  };
  float* su = ar.f((size_t)B * 8 * n0);
  float* a0 = ar.f((size_t)B * 8 * n0);
  conv(xin, P + C.stem_w, nullptr, su, 3, H, W, 8, 3, 1, 1, 1, false, H, W);
  batch_stats(su, 8, (int)n0, C.stem_m, C.stem_v);
  if (run) {
    long n = (long)B * 8 * n0;
    plane_launch(n, (long)n0, k_bn<4>, k_bn<1>, su, a0, P + C.stem_g, P + C.stem_b, Q + C.stem_m, Q + C.stem_v,
                 planes(n, n0), 8, (int)n0, 1);
  }
  BlkTape T[6];
  const float* cur = a0;
  int h = H, w = W;
  for (int b = 0; b < 6; ++b) {
    const int ci = kBlkCin[b], co = kBlkCout[b];
    const bool enc = kBlkEnc[b];
    BlkTape& t = T[b];
    t.h = h;
    t.w = w;
    t.H2 = enc ? h / 2 : 2 * h;
    t.W2 = enc ? w / 2 : 2 * w;
    const size_t n = (size_t)h * w, n2 = (size_t)t.H2 * t.W2;
    t.x = (float*)cur;
    t.t1 = ar.f((size_t)B * ci * n);
    t.t2 = ar.f((size_t)B * ci * n);
    t.x1 = ar.f((size_t)B * ci * n);
    t.u = ar.f((size_t)B * co * n2);
    t.r = ar.f((size_t)B * co * n2);
    t.y = ar.f((size_t)B * co * n2);
    t.g = ar.f((size_t)B * co);
    t.s = ar.f((size_t)B * co);
    t.out = ar.f((size_t)B * co * n2);
    conv(t.x, P + C.w1[b], nullptr, t.t1, ci, h, w, ci, 1, 1, 0, ci, !enc, h, w);
    conv(t.x, P + C.w3[b], nullptr, t.t2, ci, h, w, ci, 3, 1, 1, ci, !enc, h, w);
    batch_stats(t.t1, ci, (int)n, C.m1[b], C.v1[b]);
    batch_stats(t.t2, ci, (int)n, C.m2[b], C.v2[b]);
    batch_stats(t.x, ci, (int)n, C.m3[b], C.v3[b]);
    if (run)
      plane_launch((long)B * ci * n, (long)n, k_stage1<4>, k_stage1<1>, t.t1, t.t2, t.x, t.x1,
                   bnp(C.g1[b], C.b1[b], C.m1[b], C.v1[b]), bnp(C.g2[b], C.b2[b], C.m2[b], C.v2[b]),
                   bnp(C.g3[b], C.b3[b], C.m3[b], C.v3[b]), B * ci, ci, (int)n);
    if (enc) {
      conv(t.x1, P + C.w2[b], nullptr, t.u, ci, h, w, co, 3, 2, 1, 1, false, t.H2, t.W2);
      conv(t.x, P + C.rw[b], P + C.rb[b], t.r, ci, h, w, co, 3, 2, 1, 1, false, t.H2, t.W2);
    } else {
      conv(t.x1, P + C.w2[b], nullptr, t.u, ci, h, w, co, 4, 2, 1, 1, true, t.H2, t.W2);
      conv(t.x, P + C.rw[b], P + C.rb[b], t.r, ci, h, w, co, 4, 2, 1, 1, true, t.H2, t.W2);
    }
    batch_stats(t.u, co, (int)n2, C.m[b], C.v[b]);
    if (run) {
      long tot = (long)B * co * n2;
      plane_launch(tot, (long)n2, k_stage2<4>, k_stage2<1>, t.u, t.r, t.y, bnp(C.g[b], C.be[b], C.m[b], C.v[b]),
                   planes(tot, n2), co, (int)n2);
      (n2 % 4 == 0 ? k_gap<4> : k_gap<1>)<<<B * co, kT, 0, st>>>(t.y, t.g, (int)n2);
      k_eca_s<<<cdiv(B * co, kT), kT, 0, st>>>(t.g, P + C.eca[b], t.s, B, co);
      const float* skip = b == 3 ? T[1].out : b == 4 ? T[0].out : nullptr;
      plane_launch(tot, (long)n2, k_scale<4>, k_scale<1>, t.y, t.s, skip, t.out, planes(tot, n2), (int)n2);
    }
    cur = t.out;
    h = t.H2;
    w = t.W2;
  }
  float* logit = ar.f((size_t)B * n0);
  float* z = ar.f((size_t)B * n0);
  float* dlogit = ar.f((size_t)B * n0);
  const int nlb = cdiv((long)B * n0, kT);
  double* lpart = ar.d(nlb);
  conv(cur, P + C.out_w, P + C.out_b, logit, 8, H, W, 1, 3, 1, 1, 1, false, H, W);
  if (run) {
    k_out_loss<<<nlb, kT, 0, st>>>(logit, a.target, a.gout, z, dlogit, lpart, (long)B * n0, 1.0 / ((double)B * n0));
    if (a.loss) k_sum_f64<<<1, 256, 0, st>>>(lpart, nlb, a.loss);
    if (a.z_out) cudaMemcpyAsync(a.z_out, z, sizeof(float) * B * n0, cudaMemcpyDeviceToDevice, st);
  }

  // ---- backward
  if (run) cudaMemsetAsync(gacc, 0, sizeof(double) * kNumParams, st);
  auto wgrad = [&](const float* x, const float* dy, int Ci, int hh, int ww, int Co, int k, int s, int p, int g,
                   bool tr, int Ho, int Wo, int dst) {
    if (!run) return;
    // stride-1 convs: depthwise ones, and full ones of few channels (stem,
    // output conv), by column walks with a register window
    const bool dw = g == Ci && g == Co && s == 1 && p == (k - 1) / 2 && (k == 1 || k == 3);
    const bool full3 = g == 1 && s == 1 && k == 3 && p == 1 && !tr && ((Ci == 3 && Co % 2 == 0) || Ci % 4 == 0);
    if (dw || full3) {
      const int groups = dw ? Ci : Ci == 3 ? Co / 2 : Co * (Ci / 4);
      const long cols = (long)B * ww;
      const long target = (long)device_sms() * 4 * 256 / groups;
      int nseg = (int)std::max(1L, std::min((target + cols - 1) / cols, (long)std::max(1, hh / 8)));
      const int L = cdiv(hh, nseg);
      nseg = cdiv(hh, L);
      const dim3 grid(cdiv(cols * nseg, 256), groups);
      const int nout = (dw ? Ci : Ci * Co) * k * k;
      if ((long)grid.x * nout <= kPartCap) {
        const float* A = tr ? x : dy;
        const float* G = tr ? dy : x;
        if (dw && k == 1)
          k_wgrad_s1<1, 1, 1, true><<<grid, 256, 0, st>>>(A, G, part, B, hh, ww, Ci, Ci, L, nseg, nout);
        else if (dw)
          k_wgrad_s1<3, 1, 1, true><<<grid, 256, 0, st>>>(A, G, part, B, hh, ww, Ci, Ci, L, nseg, nout);
        else if (Ci == 3)
          k_wgrad_s1<3, 2, 3, false><<<grid, 256, 0, st>>>(dy, x, part, B, hh, ww, Co, Ci, L, nseg, nout);
        else
          k_wgrad_s1<3, 1, 4, false><<<grid, 256, 0, st>>>(dy, x, part, B, hh, ww, Co, Ci, L, nseg, nout);
        reduce(part, grid.x, nout, 1, 0, dst);
        return;
      }
    }
    if (g == 1 && (k == 3 || k == 4)) {
      WgArgs wa;
      wa.a = tr ? x : dy;
      wa.g = tr ? dy : x;
      wa.part = part;
      wa.B = B;
      wa.M = tr ? Ci : Co;
      wa.MP = cdiv(wa.M, 4) * 4;
      wa.CG = tr ? Co : Ci;
      wa.N = wa.CG * k * k;
      wa.Hp = tr ? hh : Ho;
      wa.Wp = tr ? ww : Wo;
      wa.Hg = tr ? Ho : hh;
      wa.Wg = tr ? Wo : ww;
      wa.s = s;
      wa.p = p;
      // column tiles of at most 4096 / MP columns (<= 256 threads of 4 x 4)
      int nt = cdiv((long)wa.MP * wa.N, 4096);
      wa.BN = cdiv(cdiv(wa.N, nt), 4) * 4;
      while ((wa.MP / 4) * (wa.BN / 4) > 256) wa.BN = cdiv(cdiv(wa.N, ++nt), 4) * 4;
      nt = cdiv(wa.N, wa.BN);
      const int P = (wa.MP / 4) * (wa.BN / 4);
      wa.KG = std::min(8, 256 / P);
      const int threads = cdiv((long)P * wa.KG, 32) * 32, nw = threads / 32;
      // the network's six shapes: fixed-shape kernels (MP, BN, KG)
      const bool fits = (long)B * wa.Hp * wa.Wp < (1L << 30) && (long)wa.CG * wa.Hg * wa.Wg < (1L << 27);
      auto fixed = [&](auto kern, int bn) {
        const int ntf = cdiv(wa.N, bn);
        const Slices sl = slices((long)B * wa.Hp * wa.Wp, ntf, (long)wa.M * wa.N, 32, 2, 256);
        wa.S = sl.S;
        kern<<<dim3(sl.n, ntf), 256, 0, st>>>(wa);
        reduce(part, sl.n, wa.M * wa.N, 1, 0, dst);
      };
      if (fits && wa.MP == wa.M) {
        const int key = k * 10000 + wa.M * 1000 + wa.N;
        switch (key) {
          case 3 * 10000 + 16 * 1000 + 72: fixed(k_wgemm_t<3, 16, 72, 3>, 72); return;
          case 3 * 10000 + 32 * 1000 + 144: fixed(k_wgemm_t<3, 32, 48, 2>, 48); return;
          case 3 * 10000 + 64 * 1000 + 288: fixed(k_wgemm_t<3, 64, 32, 2>, 32); return;
          case 4 * 10000 + 64 * 1000 + 512: fixed(k_wgemm_t<4, 64, 64, 1>, 64); return;
          case 4 * 10000 + 32 * 1000 + 256: fixed(k_wgemm_t<4, 32, 128, 1>, 128); return;
          case 4 * 10000 + 16 * 1000 + 128: fixed(k_wgemm_t<4, 16, 128, 2>, 128); return;
          default: break;
        }
      }
      if (wa.MP <= kWgRows * nw && wa.BN <= kWgCols * nw && fits) {
        const Slices sl = slices((long)B * wa.Hp * wa.Wp, nt, (long)wa.M * wa.N, 32, 4, 256);
        wa.S = sl.S;
        const size_t smem = std::max(sizeof(float) * (32 * (wa.MP + wa.BN) + wa.BN),
                                     wa.KG > 1 ? sizeof(float) * 16 * P * wa.KG : (size_t)0);
        if (k == 3)
          k_wgemm<3><<<dim3(sl.n, nt), threads, smem, st>>>(wa);
        else
          k_wgemm<4><<<dim3(sl.n, nt), threads, smem, st>>>(wa);
        reduce(part, sl.n, wa.M * wa.N, 1, 0, dst);
        return;
      }
    }
    int npairs = tr ? Ci * (Co / g) : Co * (Ci / g);
    // pairs per block: 4 where the tiled dimension (Ci / g for a conv,
    // Co / g for a transposed conv) allows
    // (2 for the 4x4 kernels, whose 16 sums per pair cost registers)
    const int tdim = tr ? Co / g : Ci / g;
    const int nt = tdim % 4 == 0 ? (k == 4 ? 2 : 4) : 1;
    const Slices sl = slices((long)B * (tr ? (long)hh * ww : (long)Ho * Wo), npairs / nt, (long)npairs * k * k, 1,
                             kSliceBlocks);
    dim3 grid(npairs / nt, sl.n);
    auto go = [&](auto kern) {
      kern<<<grid, kT, 0, st>>>(x, dy, part, B, Ci, hh, ww, Co, s, p, g, Ho, Wo, npairs, sl.S);
    };
    if (nt == 4) {
      if (k == 1) tr ? go(k_wgrad<true, 1, 4>) : go(k_wgrad<false, 1, 4>);
      else tr ? go(k_wgrad<true, 3, 4>) : go(k_wgrad<false, 3, 4>);
    } else if (nt == 2) {
      tr ? go(k_wgrad<true, 4, 2>) : go(k_wgrad<false, 4, 2>);
    } else {
      if (k == 1) tr ? go(k_wgrad<true, 1, 1>) : go(k_wgrad<false, 1, 1>);
      else if (k == 3) tr ? go(k_wgrad<true, 3, 1>) : go(k_wgrad<false, 3, 1>);
      else tr ? go(k_wgrad<true, 4, 1>) : go(k_wgrad<false, 4, 1>);
    }
    reduce(part, sl.n, npairs * k * k, 1, 0, dst);
  };
  auto dgrad = [&](const float* dy, const float* w, float* dx, int Ci, int hh, int ww, int Co, int k, int s, int p,
                   int g, bool tr, int Ho, int Wo) {
    if (!run) return;
    if (dense_s2(k, s, p, g, tr) && dconv_ok(!tr, Co, Ho, Wo, Ci, k)) {
      // encoder: transposed 3x3 of dy; decoder: 4x4 stride-2 conv of dy
      dconv(!tr, k, dy, w, nullptr, dx, Co, Ho, Wo, Ci, 1);
      return;
    }
    if (g == 1 && s == 1 && p == 1 && k == 3 && !tr && ww % 4 == 0 &&
        ((Ci == 3 && Co == 8) || (Ci == 8 && Co == 1))) {
      const dim3 grid(cdiv((long)hh * ww / 4, kT), B);
      if (Ci == 3)
        k_cs1<8, 3, true, true><<<grid, kT, 0, st>>>(dy, w, nullptr, dx, hh, ww, 1);
      else
        k_cs1<1, 8, true, true><<<grid, kT, 0, st>>>(dy, w, nullptr, dx, hh, ww, 1);
      return;
    }
    if (dense_s2(k, s, p, g, tr)) {
      igemm(tr ? DEC_DGRAD : ENC_DGRAD, dy, w, nullptr, dx, Co, Ho, Wo, Ci, hh, ww);
      return;
    }
    if (g == Ci && g == Co && s == 1 && p == (k - 1) / 2 && (k == 1 || k == 3)) {
      if (ww % 4 == 0) {
        const dim3 grid(cdiv((long)hh * ww / 4, kT), Ci, B);
        if (k == 1)
          k_dw4<1, false><<<grid, kT, 0, st>>>(dy, w, nullptr, dx, Ci, hh, ww, 1);
        else if (tr)
          k_dw4<3, false><<<grid, kT, 0, st>>>(dy, w, nullptr, dx, Ci, hh, ww, 1);
        else
          k_dw4<3, true><<<grid, kT, 0, st>>>(dy, w, nullptr, dx, Ci, hh, ww, 1);
        return;
      }
      const dim3 grid(cdiv((long)hh * ww, kT), Ci, B);
      if (k == 1)
        k_dw<1, false><<<grid, kT, 0, st>>>(dy, w, nullptr, dx, Ci, hh, ww, 1);
      else if (tr)
        k_dw<3, false><<<grid, kT, 0, st>>>(dy, w, nullptr, dx, Ci, hh, ww, 1);
      else
        k_dw<3, true><<<grid, kT, 0, st>>>(dy, w, nullptr, dx, Ci, hh, ww, 1);
      return;
    }
    const int nt = (Ci / g) % 8 == 0 ? 8 : (Ci / g) % 4 == 0 ? 4 : 1;
    const dim3 grid(cdiv((long)hh * ww, kT), Ci / nt, B);
    auto go = [&](auto kern) { kern<<<grid, kT, 0, st>>>(dy, w, dx, B, Ci, hh, ww, Co, k, s, p, g, Ho, Wo); };
    if (tr)
      nt == 8 ? go(k_convT_dgrad<8>) : nt == 4 ? go(k_convT_dgrad<4>) : go(k_convT_dgrad<1>);
    else
      nt == 8 ? go(k_conv_dgrad<8>) : nt == 4 ? go(k_conv_dgrad<4>) : go(k_conv_dgrad<1>);
  };
  // per-channel sums of (a) and (a * normalised v) -> dbeta / dgamma (and bias)
  auto chan = [&](const float* av, const float* v, const float* mean, const float* var, int Cc, int n,
                  int dgam, int dbet) {
    if (!run) return;
    const Slices sl = slices((long)B * n, Cc, 2L * Cc, 4, kSliceBlocks);
    (n % 4 == 0 ? k_chan_sums<4> : k_chan_sums<1>)<<<dim3(Cc, sl.n), kT, 0, st>>>(av, v, mean, var, part, B, Cc, n,
                                                                                 sl.S);
    if (dbet >= 0 && dgam >= 0)  // both sums in one launch
      k_reduce_few<<<cdiv(2 * Cc, 8), 256, 0, st>>>(part, sl.n, 2 * Cc, 1, 0, gacc, dbet, dgam, nullptr, 1.0);
    else if (dbet >= 0)
      reduce(part, sl.n, Cc, 2, 0, dbet);
    else if (dgam >= 0)
      reduce(part, sl.n, Cc, 2, 1, dgam);
  };
  // out (+)= dBN input: gam / sigma dy (running statistics), or the batch
  // adjoint, whose sums of this BN chan() has just added to gacc
  auto bn_dx = [&](const float* d, const float* x, BnP bn, int dgam, int dbet, float* out, long tot, int Cc, int n,
                   int accumulate) {
    if (!run) return;
    if (a.bn_batch)
      plane_launch(tot, (long)n, k_bn_dx_batch<4>, k_bn_dx_batch<1>, d, x, bn, gacc, dgam, dbet,
                   (float)(1.0 / ((double)B * n)), out, planes(tot, n), Cc, n, accumulate);
    else
      plane_launch(tot, (long)n, k_bn_dx<4>, k_bn_dx<1>, d, bn, out, planes(tot, n), Cc, n, accumulate);
  };
  // output conv
  float* dcur = ar.f((size_t)B * 8 * n0);
  if (run) cudaMemsetAsync(dcur, 0, sizeof(float) * B * 8 * n0, st);
  wgrad(cur, dlogit, 8, H, W, 1, 3, 1, 1, 1, false, H, W, C.out_w);
  chan(dlogit, nullptr, nullptr, nullptr, 1, (int)n0, -1, C.out_b);
  dgrad(dlogit, P + C.out_w, dcur, 8, H, W, 1, 3, 1, 1, 1, false, H, W);
  float* dskip0 = ar.f((size_t)B * 16 * (H / 2) * (W / 2));
  float* dskip1 = ar.f((size_t)B * 32 * (H / 4) * (W / 4));
  if (run) {
    cudaMemsetAsync(dskip0, 0, sizeof(float) * B * 16 * (H / 2) * (W / 2), st);
    cudaMemsetAsync(dskip1, 0, sizeof(float) * B * 32 * (H / 4) * (W / 4), st);
  }
  // scratch for one block's adjoint (largest block sizes)
  size_t big = (size_t)B * 8 * n0;  // every block map holds at most 8 H W values per window
  float* dy = ar.f(big);
  float* dtmp = ar.f(big);
  float* dx1 = ar.f(big);
  float* dt = ar.f(big);
  float* ds = ar.f((size_t)B * 64);
  float* dgm = ar.f((size_t)B * 64);
  float* dkp = ar.f((size_t)B * 3);
  float* dxs[2] = {ar.f(big), ar.f(big)};
  for (int b = 5; b >= 0; --b) {
    const BlkTape& t = T[b];
    const int ci = kBlkCin[b], co = kBlkCout[b];
    const bool enc = kBlkEnc[b];
    const int n = t.h * t.w, n2 = t.H2 * t.W2;
    const long tot2 = (long)B * co * n2, tot = (long)B * ci * n;
    float* dx = dxs[b & 1];
    if (run) {
      if (b == 0) lin_launch(tot2, k_add<4>, k_add<1>, dcur, dskip0, tot2);
      if (b == 1) lin_launch(tot2, k_add<4>, k_add<1>, dcur, dskip1, tot2);
      if (b == 3) lin_launch(tot2, k_add<4>, k_add<1>, dskip1, dcur, tot2);
      if (b == 4) lin_launch(tot2, k_add<4>, k_add<1>, dskip0, dcur, tot2);
      // ECA
      (n2 % 4 == 0 ? k_eca_ds<4> : k_eca_ds<1>)<<<B * co, kT, 0, st>>>(dcur, t.y, ds, n2);
      k_eca_back<<<B, 64, 0, st>>>(ds, t.s, t.g, P + C.eca[b], dgm, dkp, B, co, n2);
      reduce(dkp, B, 3, 1, 0, C.eca[b]);
      plane_launch(tot2, (long)n2, k_eca_dy<4>, k_eca_dy<1>, dcur, t.s, dgm, dy, planes(tot2, n2), n2);
      // main branch: dbn = dy [BN(u) > 0] and its dbeta, dgamma sums; du =
      // dbn gam / sigma (scaled in the same pass with running statistics)
      BnP bn = bnp(C.g[b], C.be[b], C.m[b], C.v[b]);
      const Slices sl = slices((long)B * n2, co, 2L * co, 4, kSliceBlocks);
      (n2 % 4 == 0 ? k_stage2_sums<4> : k_stage2_sums<1>)<<<dim3(co, sl.n), kT, 0, st>>>(
          dy, t.u, bn, dtmp, part, B, co, (int)n2, sl.S, a.bn_batch ? 0 : 1);
      k_reduce_few<<<cdiv(2L * co, 8), 256, 0, st>>>(part, sl.n, 2 * co, 1, 0, gacc, C.be[b], C.g[b], nullptr, 1.0);
    }
    if (a.bn_batch)
      bn_dx(dtmp, t.u, bnp(C.g[b], C.be[b], C.m[b], C.v[b]), C.g[b], C.be[b], dtmp, tot2, co, n2, 0);
    if (run) {
      cudaMemsetAsync(dx1, 0, sizeof(float) * tot, st);
      cudaMemsetAsync(dx, 0, sizeof(float) * tot, st);
    }
    const int kk = enc ? 3 : 4;
    wgrad(t.x1, dtmp, ci, t.h, t.w, co, kk, 2, 1, 1, !enc, t.H2, t.W2, C.w2[b]);
    dgrad(dtmp, P + C.w2[b], dx1, ci, t.h, t.w, co, kk, 2, 1, 1, !enc, t.H2, t.W2);
    // residual branch
    wgrad(t.x, dy, ci, t.h, t.w, co, kk, 2, 1, 1, !enc, t.H2, t.W2, C.rw[b]);
    chan(dy, nullptr, nullptr, nullptr, co, n2, -1, C.rb[b]);
    dgrad(dy, P + C.rw[b], dx, ci, t.h, t.w, co, kk, 2, 1, 1, !enc, t.H2, t.W2);
    // stage 1: dv = dx1 [x1 > 0] and the sums of its three BNs, one pass
    if (run) {
      const Slices sl = slices((long)B * n, ci, 4L * ci, 4, kSliceBlocks);
      const Bn3 b3{Q + C.m1[b], Q + C.v1[b], Q + C.m2[b], Q + C.v2[b], Q + C.m3[b], Q + C.v3[b]};
      (n % 4 == 0 ? k_stage1_sums<4> : k_stage1_sums<1>)<<<dim3(ci, sl.n), kT, 0, st>>>(dx1, t.x1, t.t1, t.t2, t.x,
                                                                                      b3, part, B, ci, n, sl.S);
      k_reduce_stage1<<<cdiv(4L * ci, 8), 256, 0, st>>>(part, sl.n, ci, gacc, C.b1[b], C.b2[b], C.b3[b], C.g1[b],
                                                        C.g2[b], C.g3[b]);
    }
    bn_dx(dx1, t.x, bnp(C.g3[b], C.b3[b], C.m3[b], C.v3[b]), C.g3[b], C.b3[b], dx, tot, ci, n, 1);
    // dt1 = dv gam1 / sigma1 -> dw1, dx
    bn_dx(dx1, t.t1, bnp(C.g1[b], C.b1[b], C.m1[b], C.v1[b]), C.g1[b], C.b1[b], dt, tot, ci, n, 0);
    wgrad(t.x, dt, ci, t.h, t.w, ci, 1, 1, 0, ci, !enc, t.h, t.w, C.w1[b]);
    dgrad(dt, P + C.w1[b], dx, ci, t.h, t.w, ci, 1, 1, 0, ci, !enc, t.h, t.w);
    bn_dx(dx1, t.t2, bnp(C.g2[b], C.b2[b], C.m2[b], C.v2[b]), C.g2[b], C.b2[b], dt, tot, ci, n, 0);
    wgrad(t.x, dt, ci, t.h, t.w, ci, 3, 1, 1, ci, !enc, t.h, t.w, C.w3[b]);
    dgrad(dt, P + C.w3[b], dx, ci, t.h, t.w, ci, 3, 1, 1, ci, !enc, t.h, t.w);
    dcur = dx;
  }
  // stem: a0 = ReLU(BN(su))
  const long tot0 = (long)B * 8 * n0;
  if (run) lin_launch(tot0, k_relu_mask<4>, k_relu_mask<1>, dcur, a0, dtmp, tot0);
  chan(dtmp, su, Q + C.stem_m, Q + C.stem_v, 8, (int)n0, C.stem_g, C.stem_b);
  bn_dx(dtmp, su, bnp(C.stem_g, C.stem_b, C.stem_m, C.stem_v), C.stem_g, C.stem_b, dtmp, tot0, 8, (int)n0, 0);
  wgrad(xin, dtmp, 3, H, W, 8, 3, 1, 1, 1, false, H, W, C.stem_w);
  if (a.gin) {
    float* gin = ar.f((size_t)B * 3 * n0);
    if (run) {
      cudaMemsetAsync(gin, 0, sizeof(float) * B * 3 * n0, st);
      dgrad(dtmp, P + C.stem_w, gin, 3, H, W, 8, 3, 1, 1, 1, false, H, W);
      cudaMemcpyAsync(a.gin, gin, sizeof(float) * B * 3 * n0, cudaMemcpyDeviceToDevice, st);
    }
  }
  if (run) {
    if (a.bn_stats)
      cudaMemcpyAsync(a.bn_stats, Q, sizeof(float) * kNumBuffers, cudaMemcpyDeviceToDevice, st);
    if (a.gparams_f64) cudaMemcpyAsync(a.gparams_f64, gacc, sizeof(double) * kNumParams, cudaMemcpyDeviceToDevice, st);
    if (a.gparams) k_to_f32<<<cdiv(kNumParams, kT), kT, 0, st>>>(gacc, a.gparams, kNumParams);
  }
  return ar.off;
}

cudaError_t train_step(const TrainArgs& a, void* workspace, size_t bytes) {
  Arena ar{(char*)workspace, 0, bytes};
  size_t need = train_workspace_bytes(a.B, a.H, a.W) + (a.gin ? (size_t)a.B * 3 * a.H * a.W * 4 + 256 : 0);
  if (need > bytes) return cudaErrorInvalidValue;
  train_step_plan(a, &ar);
  return cudaGetLastError();
}

}  // namespace stda
