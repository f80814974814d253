// Training step of Radar-STDA on the GPU: forward with a tape, mean squared
// error against the clean maps (or a given dL/dz), and the adjoint of every
// operation, producing dL/dtheta for all 137,915 parameters.
//
// The graph keeps batch normalisation unfolded (inference form with frozen
// running statistics; gamma and beta are trained), so every tensor of the
// taped forward is the one the adjoint needs. Tensors are NCHW float32.
// Weight and BN gradients are first reduced per batch chunk in FP32 (one
// thread block per (output, input) channel pair, warp shuffles), then the
// chunks are summed in FP64 in a fixed order; the loss is an FP64 sum.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "stda_internal.h"
#include "stda_train.h"

namespace stda {
namespace {

constexpr int kT = 256;
constexpr int kChunkWin = 4;  // windows per weight-gradient partial

inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }
inline dim3 grid1(long n) { return dim3(cdiv(n, kT)); }

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
  const int CoT = Co / NT;
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)B * CoT * Ho * Wo) return;
  int X = idx % Wo, Y = (idx / Wo) % Ho, o0 = (int)((idx / ((long)Wo * Ho)) % CoT) * NT,
      b = idx / ((long)Wo * Ho * CoT);
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
  const int CoT = Co / NT;
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)B * CoT * Ho * Wo) return;
  int X = idx % Wo, Y = (idx / Wo) % Ho, o0 = (int)((idx / ((long)Wo * Ho)) % CoT) * NT,
      b = idx / ((long)Wo * Ho * CoT);
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
  const int CiT = Ci / NT;
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)B * CiT * H * W) return;
  int xx = idx % W, yy = (idx / W) % H, i0 = (int)((idx / ((long)W * H)) % CiT) * NT,
      b = idx / ((long)W * H * CiT);
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
  const int CiT = Ci / NT;
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)B * CiT * H * W) return;
  int xi = idx % W, yi = (idx / W) % H, i0 = (int)((idx / ((long)W * H)) % CiT) * NT,
      b = idx / ((long)W * H * CiT);
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
// when TR) over the windows of one chunk: one block per pair tile, the
// shared operand (dy of output o for a conv, x of input i for a transposed
// conv) loaded once per pixel for the NT pairs; per value a warp shuffle
// reduction, then one pass over the warps; part[chunk][pair * k * k + tap].
// K is the kernel size (1, 3 or 4) as a template argument, so the sums stay
// in registers.
template <bool TR, int K, int NT>
__global__ void k_wgrad(const float* __restrict__ x, const float* __restrict__ dy, float* __restrict__ part,
                        int B, int Ci, int H, int W, int Co, int s, int p, int g, int Ho, int Wo,
                        int npairs) {
  constexpr int k = K, KK = K * K, NV = NT * KK;
  __shared__ float sh[32 * NV];
  const int tile = blockIdx.x, chunk = blockIdx.y;
  const int cig = Ci / g, cog = Co / g;
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
  const int b0 = chunk * kChunkWin, b1 = min(B, b0 + kChunkWin);
  if (!TR) {
    const int n = Ho * Wo;
    for (int b = b0; b < b1; ++b) {
      const float* xp = x + ((size_t)b * Ci + i) * H * W;
      const float* dp = dy + ((size_t)b * Co + o) * n;
      for (int q = threadIdx.x; q < n; q += blockDim.x) {
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
    for (int b = b0; b < b1; ++b) {
      const float* xp = x + ((size_t)b * Ci + i) * n;
      const float* dp = dy + ((size_t)b * Co + o) * Ho * Wo;
      for (int q = threadIdx.x; q < n; q += blockDim.x) {
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

// Per-channel sums over one chunk of windows: S1 = sum a, S2 = sum a (v - mean) / sqrt(var + eps)
// (S2 only if v); part[chunk][c][2].
__global__ void k_chan_sums(const float* __restrict__ a, const float* __restrict__ v, const float* __restrict__ mean,
                            const float* __restrict__ var, float* __restrict__ part, int B, int C, int n) {
  __shared__ float sh[32];
  const int c = blockIdx.x, chunk = blockIdx.y;
  const int b0 = chunk * kChunkWin, b1 = min(B, b0 + kChunkWin);
  float s1 = 0.f, s2 = 0.f;
  float m = v ? mean[c] : 0.f, is = v ? rsqrtf(var[c] + 1e-5f) : 0.f;
  for (int b = b0; b < b1; ++b) {
    const float* ap = a + ((size_t)b * C + c) * n;
    const float* vp = v ? v + ((size_t)b * C + c) * n : nullptr;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      float d = ap[q];
      s1 += d;
      if (vp) s2 += d * (vp[q] - m) * is;
    }
  }
  float r1 = block_sum(s1, sh);
  float r2 = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    part[((size_t)chunk * C + c) * 2] = r1;
    part[((size_t)chunk * C + c) * 2 + 1] = r2;
  }
}

// Sums partials over chunks in FP64 (fixed order) and adds them into the
// gradient accumulator: acc[dst + j] += sum_chunk part[chunk][j * stride + off].
__global__ void k_reduce(const float* __restrict__ part, int nchunks, int n, int stride, int off,
                         double* __restrict__ acc, long dst) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c) s += (double)part[(size_t)c * n * stride + (size_t)j * stride + off];
  acc[dst + j] += s;
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ out, int n) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = (float)a[j];
}

// y = relu?(gam (x - mean) / sqrt(var + eps) + bet) per channel
__global__ void k_bn(const float* __restrict__ x, float* __restrict__ y, const float* __restrict__ gam,
                     const float* __restrict__ bet, const float* __restrict__ mean, const float* __restrict__ var,
                     long total, int C, int n, int relu) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int c = (idx / n) % C;
  float v = gam[c] * (x[idx] - mean[c]) * rsqrtf(var[c] + 1e-5f) + bet[c];
  y[idx] = relu ? fmaxf(v, 0.f) : v;
}

// stage 1: x1 = ReLU(BN1(t1) + BN2(t2) + BN3(x))
struct BnP {
  const float *g, *b, *m, *v;
};
__device__ __forceinline__ float bnv(const BnP& q, int c, float x) {
  return q.g[c] * (x - q.m[c]) * rsqrtf(q.v[c] + 1e-5f) + q.b[c];
}
__global__ void k_stage1(const float* t1, const float* t2, const float* x, float* x1, BnP b1, BnP b2, BnP b3,
                         long total, int C, int n) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int c = (idx / n) % C;
  x1[idx] = fmaxf(bnv(b1, c, t1[idx]) + bnv(b2, c, t2[idx]) + bnv(b3, c, x[idx]), 0.f);
}
// y = ReLU(BN(u)) + r
__global__ void k_stage2(const float* u, const float* r, float* y, BnP bn, long total, int C, int n) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int c = (idx / n) % C;
  y[idx] = fmaxf(bnv(bn, c, u[idx]), 0.f) + r[idx];
}

// per (b, c): g = mean over the map
__global__ void k_gap(const float* __restrict__ y, float* __restrict__ g, int n) {
  __shared__ float sh[32];
  const float* p = y + (size_t)blockIdx.x * n;
  float s = 0.f;
  for (int q = threadIdx.x; q < n; q += blockDim.x) s += p[q];
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
__global__ void k_scale(const float* y, const float* sc, const float* skip, float* out, long total, int n) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  float v = sc[idx / n] * y[idx];
  out[idx] = skip ? v + skip[idx] : v;
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
__global__ void k_sum_f64(const double* part, int n, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *out = s;
  }
}

// ---------------------------------------------------------- backward ops
// per (b, c): ds = sum dout * y
__global__ void k_eca_ds(const float* dout, const float* y, float* ds, int n) {
  __shared__ float sh[32];
  const float* a = dout + (size_t)blockIdx.x * n;
  const float* v = y + (size_t)blockIdx.x * n;
  float s = 0.f;
  for (int q = threadIdx.x; q < n; q += blockDim.x) s += a[q] * v[q];
  float r = block_sum(s, sh);
  if (threadIdx.x == 0) ds[blockIdx.x] = r;
}
// per window b (one thread per b): dz = ds s (1 - s); dk partial; dg
__global__ void k_eca_back(const float* ds, const float* sc, const float* g, const float* k3, float* dgm,
                           float* dk_part, int B, int C, int n) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float *dsb = ds + b * C, *sb = sc + b * C, *gb = g + b * C;
  float* dg = dgm + b * C;
  float dk[3] = {0.f, 0.f, 0.f};
  for (int c = 0; c < C; ++c) dg[c] = 0.f;
  for (int c = 0; c < C; ++c) {
    float dz = dsb[c] * sb[c] * (1.f - sb[c]);
    for (int j = 0; j < 3; ++j) {
      int cc = c + j - 1;
      if (cc < 0 || cc >= C) continue;
      dk[j] += dz * gb[cc];
      dg[cc] += dz * k3[j] / (float)n;
    }
  }
  for (int j = 0; j < 3; ++j) dk_part[b * 3 + j] = dk[j];
}
// dy = s * dout + dg (the mean's adjoint, already divided by n)
__global__ void k_eca_dy(const float* dout, const float* sc, const float* dgm, float* dy, long total, int n) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  dy[idx] = sc[idx / n] * dout[idx] + dgm[idx / n];
}
// dbn = dy [BN(u) > 0]
__global__ void k_relu_bn_mask(const float* dy, const float* u, BnP bn, float* dbn, long total, int C, int n) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int c = (idx / n) % C;
  dbn[idx] = bnv(bn, c, u[idx]) > 0.f ? dy[idx] : 0.f;
}
// out (+)= a * gam / sqrt(var + eps)
__global__ void k_bn_dx(const float* a, BnP bn, float* out, long total, int C, int n, int accumulate) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int c = (idx / n) % C;
  float v = a[idx] * bn.g[c] * rsqrtf(bn.v[c] + 1e-5f);
  out[idx] = accumulate ? out[idx] + v : v;
}
// Batch statistics of a BN input x[B][C][n]: part[chunk][c] = sum over the
// chunk's windows of x (mean == null) or of (x - mean[c])^2.
__global__ void k_bn_part(const float* __restrict__ x, const float* __restrict__ mean, float* __restrict__ part,
                          int B, int C, int n) {
  __shared__ float sh[32];
  const int c = blockIdx.x, chunk = blockIdx.y;
  const int b0 = chunk * kChunkWin, b1 = min(B, b0 + kChunkWin);
  const float m = mean ? mean[c] : 0.f;
  float s = 0.f;
  for (int b = b0; b < b1; ++b) {
    const float* p = x + ((size_t)b * C + c) * n;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const float d = p[q] - m;
      s += mean ? d * d : p[q];
    }
  }
  const float r = block_sum(s, sh);
  if (threadIdx.x == 0) part[(size_t)chunk * C + c] = r;
}
// out[c] = (sum over chunks of part[chunk][c]) / N, summed in FP64
__global__ void k_bn_fin(const float* __restrict__ part, int nchunks, int C, double N, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double s = 0.0;
  for (int k = 0; k < nchunks; ++k) s += (double)part[(size_t)k * C + c];
  out[c] = (float)(s / N);
}
// Batch-statistics BN adjoint: out (+)= gam / sigma (dy - (sum dy + xhat sum
// dy xhat) / N), the two sums of this BN being gacc[dbet + c], gacc[dgam + c].
__global__ void k_bn_dx_batch(const float* dy, const float* x, BnP bn, const double* __restrict__ gacc, long dgam,
                              long dbet, double N, float* out, long total, int C, int n, int accumulate) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int c = (idx / n) % C;
  const float is = rsqrtf(bn.v[c] + 1e-5f), xh = (x[idx] - bn.m[c]) * is;
  const float corr = (float)((gacc[dbet + c] + (double)xh * gacc[dgam + c]) / N);
  const float v = bn.g[c] * is * (dy[idx] - corr);
  out[idx] = accumulate ? out[idx] + v : v;
}
// dv = dx1 [x1 > 0]
__global__ void k_relu_mask(const float* d, const float* act, float* out, long total) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  out[idx] = act[idx] > 0.f ? d[idx] : 0.f;
}
__global__ void k_add(float* a, const float* b, long total) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < total) a[idx] += b[idx];
}
__global__ void k_bf16_to_f32(const __nv_bfloat16* a, float* out, long total) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < total) out[idx] = __bfloat162float(a[idx]);
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
  const int nchunk = cdiv(B, kChunkWin);
  // BN statistics: the running ones, or (training mode) the batch's, computed
  // into `bst` (same layout as the running buffers) right before each BN
  float* bst = ar.f(kNumBuffers);
  float* spart = ar.f((size_t)64 * nchunk);
  const float* Q = a.bn_batch ? bst : a.buffers;
  auto bnp = [&](int g, int b, int m, int v) { return BnP{P + g, P + b, Q + m, Q + v}; };
  auto batch_stats = [&](const float* x, int Cc, int n, int moff, int voff) {
    if (!run || !a.bn_batch) return;
    const double N = (double)B * n;
    k_bn_part<<<dim3(Cc, nchunk), kT, 0, st>>>(x, nullptr, spart, B, Cc, n);
    k_bn_fin<<<cdiv(Cc, kT), kT, 0, st>>>(spart, nchunk, Cc, N, bst + moff);
    k_bn_part<<<dim3(Cc, nchunk), kT, 0, st>>>(x, bst + moff, spart, B, Cc, n);
    k_bn_fin<<<cdiv(Cc, kT), kT, 0, st>>>(spart, nchunk, Cc, N, bst + voff);
  };

  // ---- forward with tape
  float* xin = ar.f((size_t)B * 3 * n0);
  if (run) {
    if (a.in_bf16)
      k_bf16_to_f32<<<grid1((long)B * 3 * n0), kT, 0, st>>>((const __nv_bfloat16*)a.in, xin, (long)B * 3 * n0);
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
  auto conv = [&](const float* x, const float* w, const float* bias, float* y, int Ci, int h, int wd, int Co,
                  int k, int s, int p, int g, bool tr, int Ho, int Wo) {
    if (!run) return;
    if (dense_s2(k, s, p, g, tr)) {
      igemm(tr ? DEC_FWD : ENC_FWD, x, w, bias, y, Ci, h, wd, Co, Ho, Wo);
      return;
    }
    const int nt = (Co / g) % 8 == 0 ? 8 : (Co / g) % 4 == 0 ? 4 : 1;
    long n = (long)B * (Co / nt) * Ho * Wo;
    auto go = [&](auto kern) { kern<<<grid1(n), kT, 0, st>>>(x, w, bias, y, B, Ci, h, wd, Co, k, s, p, g, Ho, Wo); };
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
    k_bn<<<grid1(n), kT, 0, st>>>(su, a0, P + C.stem_g, P + C.stem_b, Q + C.stem_m, Q + C.stem_v, n, 8, (int)n0, 1);
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
      k_stage1<<<grid1((long)B * ci * n), kT, 0, st>>>(t.t1, t.t2, t.x, t.x1, bnp(C.g1[b], C.b1[b], C.m1[b], C.v1[b]),
                                                     bnp(C.g2[b], C.b2[b], C.m2[b], C.v2[b]),
                                                     bnp(C.g3[b], C.b3[b], C.m3[b], C.v3[b]), (long)B * ci * n, ci,
                                                     (int)n);
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
      k_stage2<<<grid1(tot), kT, 0, st>>>(t.u, t.r, t.y, bnp(C.g[b], C.be[b], C.m[b], C.v[b]), tot, co, (int)n2);
      k_gap<<<B * co, kT, 0, st>>>(t.y, t.g, (int)n2);
      k_eca_s<<<cdiv(B * co, kT), kT, 0, st>>>(t.g, P + C.eca[b], t.s, B, co);
      const float* skip = b == 3 ? T[1].out : b == 4 ? T[0].out : nullptr;
      k_scale<<<grid1(tot), kT, 0, st>>>(t.y, t.s, skip, t.out, tot, (int)n2);
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
    if (a.loss) k_sum_f64<<<1, 32, 0, st>>>(lpart, nlb, a.loss);
    if (a.z_out) cudaMemcpyAsync(a.z_out, z, sizeof(float) * B * n0, cudaMemcpyDeviceToDevice, st);
  }

  // ---- backward
  double* gacc = ar.d(kNumParams);
  if (run) cudaMemsetAsync(gacc, 0, sizeof(double) * kNumParams, st);
  // largest partial buffer: pairs * k * k per chunk
  size_t part_max = 0;
  for (int b = 0; b < 6; ++b) {
    size_t dense = (size_t)(kBlkEnc[b] ? 9 : 16) * kBlkCin[b] * kBlkCout[b];
    part_max = std::max(part_max, dense);
  }
  part_max = std::max(part_max, (size_t)216);
  float* part = ar.f(part_max * nchunk);
  auto wgrad = [&](const float* x, const float* dy, int Ci, int hh, int ww, int Co, int k, int s, int p, int g,
                   bool tr, int Ho, int Wo, int dst) {
    if (!run) return;
    int npairs = tr ? Ci * (Co / g) : Co * (Ci / g);
    // pairs per block: 4 where the tiled dimension (Ci / g for a conv,
    // Co / g for a transposed conv) allows
    // (2 for the 4x4 kernels, whose 16 sums per pair cost registers)
    const int tdim = tr ? Co / g : Ci / g;
    const int nt = tdim % 4 == 0 ? (k == 4 ? 2 : 4) : 1;
    dim3 grid(npairs / nt, nchunk);
    auto go = [&](auto kern) { kern<<<grid, kT, 0, st>>>(x, dy, part, B, Ci, hh, ww, Co, s, p, g, Ho, Wo, npairs); };
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
    int n = npairs * k * k;
    k_reduce<<<cdiv(n, kT), kT, 0, st>>>(part, nchunk, n, 1, 0, gacc, dst);
  };
  auto dgrad = [&](const float* dy, const float* w, float* dx, int Ci, int hh, int ww, int Co, int k, int s, int p,
                   int g, bool tr, int Ho, int Wo) {
    if (!run) return;
    if (dense_s2(k, s, p, g, tr)) {
      igemm(tr ? DEC_DGRAD : ENC_DGRAD, dy, w, nullptr, dx, Co, Ho, Wo, Ci, hh, ww);
      return;
    }
    const int nt = (Ci / g) % 8 == 0 ? 8 : (Ci / g) % 4 == 0 ? 4 : 1;
    long n = (long)B * (Ci / nt) * hh * ww;
    auto go = [&](auto kern) { kern<<<grid1(n), kT, 0, st>>>(dy, w, dx, B, Ci, hh, ww, Co, k, s, p, g, Ho, Wo); };
    if (tr)
      nt == 8 ? go(k_convT_dgrad<8>) : nt == 4 ? go(k_convT_dgrad<4>) : go(k_convT_dgrad<1>);
    else
      nt == 8 ? go(k_conv_dgrad<8>) : nt == 4 ? go(k_conv_dgrad<4>) : go(k_conv_dgrad<1>);
  };
  // per-channel sums of (a) and (a * normalised v) -> dbeta / dgamma (and bias)
  auto chan = [&](const float* av, const float* v, const float* mean, const float* var, int Cc, int n,
                  int dgam, int dbet) {
    if (!run) return;
    k_chan_sums<<<dim3(Cc, nchunk), kT, 0, st>>>(av, v, mean, var, part, B, Cc, n);
    if (dbet >= 0) k_reduce<<<cdiv(Cc, kT), kT, 0, st>>>(part, nchunk, Cc, 2, 0, gacc, dbet);
    if (dgam >= 0) k_reduce<<<cdiv(Cc, kT), kT, 0, st>>>(part, nchunk, Cc, 2, 1, gacc, dgam);
  };
  // out (+)= dBN input: gam / sigma dy (running statistics), or the batch
  // adjoint, whose sums of this BN chan() has just added to gacc
  auto bn_dx = [&](const float* d, const float* x, BnP bn, int dgam, int dbet, float* out, long tot, int Cc, int n,
                   int accumulate) {
    if (!run) return;
    if (a.bn_batch)
      k_bn_dx_batch<<<grid1(tot), kT, 0, st>>>(d, x, bn, gacc, dgam, dbet, (double)B * n, out, tot, Cc, n,
                                               accumulate);
    else
      k_bn_dx<<<grid1(tot), kT, 0, st>>>(d, bn, out, tot, Cc, n, accumulate);
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
      if (b == 0) k_add<<<grid1(tot2), kT, 0, st>>>(dcur, dskip0, tot2);
      if (b == 1) k_add<<<grid1(tot2), kT, 0, st>>>(dcur, dskip1, tot2);
      if (b == 3) k_add<<<grid1(tot2), kT, 0, st>>>(dskip1, dcur, tot2);
      if (b == 4) k_add<<<grid1(tot2), kT, 0, st>>>(dskip0, dcur, tot2);
      // ECA
      k_eca_ds<<<B * co, kT, 0, st>>>(dcur, t.y, ds, n2);
      k_eca_back<<<cdiv(B, 64), 64, 0, st>>>(ds, t.s, t.g, P + C.eca[b], dgm, dkp, B, co, n2);
      k_reduce<<<1, 32, 0, st>>>(dkp, B, 3, 1, 0, gacc, C.eca[b]);
      k_eca_dy<<<grid1(tot2), kT, 0, st>>>(dcur, t.s, dgm, dy, tot2, n2);
      // main branch: dbn = dy [BN(u) > 0]; du = dbn gam / sigma
      BnP bn = bnp(C.g[b], C.be[b], C.m[b], C.v[b]);
      k_relu_bn_mask<<<grid1(tot2), kT, 0, st>>>(dy, t.u, bn, dtmp, tot2, co, n2);
    }
    chan(dtmp, t.u, Q + C.m[b], Q + C.v[b], co, n2, C.g[b], C.be[b]);
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
    // stage 1: dv = dx1 [x1 > 0]
    if (run) k_relu_mask<<<grid1(tot), kT, 0, st>>>(dx1, t.x1, dx1, tot);
    chan(dx1, t.t1, Q + C.m1[b], Q + C.v1[b], ci, n, C.g1[b], C.b1[b]);
    chan(dx1, t.t2, Q + C.m2[b], Q + C.v2[b], ci, n, C.g2[b], C.b2[b]);
    chan(dx1, t.x, Q + C.m3[b], Q + C.v3[b], ci, n, C.g3[b], C.b3[b]);
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
  if (run) k_relu_mask<<<grid1(tot0), kT, 0, st>>>(dcur, a0, dtmp, tot0);
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
