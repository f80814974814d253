// Radar-STDA forward pass with the dense convolutions on the tcgen05 tensor
// cores (BF16 operands, FP32 accumulation in tensor memory).
//
// One kernel per network level; one CTA per band of rows of one window,
// always spanning the full map width. Per CTA:
//  1. Stage the block input x (previous block output x ECA weights, plus the
//     skip operand for decoders; for encoder block 1 the stem conv computed
//     from the three raw frames) into shared memory as bf16 "planes" in the
//     no-swizzle K-major core-matrix layout [channel group][pixel][8 ch]
//     with zero margins. Encoder inputs are split into four polyphase planes
//     (even/odd row x even/odd column), so that the stride-2 3x3 convolution
//     reads each tap at a unit-stride shifted pixel.
//  2. Stage 1 (Eqs. mobile_*_stage1, BN folded into one depthwise 3x3 +
//     bias + ReLU) on the CUDA cores into a second set of planes.
//  3. Stage 2 (Eqs. mobile_*_stage2) on the tensor cores: the GEMM rows are
//     128 consecutive pixels of the padded plane; every tap (encoder 3x3
//     stride 2; decoder 2x2 sub-pixel taps of the 4x4 stride-2 transposed
//     convolution, one accumulator per output phase) is an MMA whose A
//     descriptor starts at the tap's shifted pixel, so no im2col copy exists.
//     Main and residual branches accumulate into separate TMEM columns.
//  4. Epilogue: TMEM -> registers, ReLU(main + BN shift) + residual + bias,
//     bf16 NHWC store, per-band channel sums for the next ECA.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <tuple>

#include "stda_internal.h"
#include "stda_tc.h"
#include "umma.h"

namespace stda {
namespace {

using namespace umma;
constexpr int kThreads = 256;

__device__ __forceinline__ void bf16x8_to_f32(uint4 u, float* f) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float2 t = __bfloat1622float2(h[i]);
    f[2 * i] = t.x;
    f[2 * i + 1] = t.y;
  }
}
__device__ __forceinline__ uint4 f32_to_bf16x8(const float* f) {
  uint4 u;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
  return u;
}

// ECA weights of one window (same arithmetic as the CUDA-core path).
__device__ void eca_scales(const float* __restrict__ part, int ntiles, int C, float inv_n,
                           const float* __restrict__ k3, float* s_g, float* s_s) {
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    float a = 0.f;
    for (int t = 0; t < ntiles; ++t) a += part[t * C + c];
    s_g[c] = a * inv_n;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    float z = k3[1] * s_g[c];
    if (c > 0) z += k3[0] * s_g[c - 1];
    if (c + 1 < C) z += k3[2] * s_g[c + 1];
    s_s[c] = 1.f / (1.f + expf(-z));
  }
  __syncthreads();
}

__device__ __forceinline__ void warp_sum_to(float v, float* dst) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) *dst += v;
}

// Issues every MMA of one CTA (one thread). Accumulator (tile i, acc a) sits
// at TMEM column (i * nacc + a) * NP; K-steps of accumulator a are
// ks[(a % nph) * nsteps ...] for the main branch (a < nph) and the same
// table for the residual branch (a >= nph).
__device__ void issue_mmas(uint32_t tmem, const KStep* ks, int nsteps, int nph, int NP, int ntile, int m_lo,
                           int WP, int PIXA, uint32_t x1_base, uint32_t x0_base, uint32_t wm_base,
                           uint32_t wr_base) {
  const uint32_t idesc = idesc_bf16(128, NP);
  const uint32_t wstep = 2u * NP * 16u;  // bytes per packed K-step
  for (int i = 0; i < ntile; ++i) {
    int m0 = m_lo + 128 * i;
    for (int a = 0; a < 2 * nph; ++a) {
      bool res = a >= nph;
      int ph = res ? a - nph : a;
      uint32_t xb = res ? x0_base : x1_base, wb = res ? wr_base : wm_base;
      uint32_t d = tmem + (uint32_t)((i * 2 * nph + a) * NP);
      for (int j = 0; j < nsteps; ++j) {
        KStep k = ks[ph * nsteps + j];
        int p0 = k.pl0 * PIXA + m0 + k.dr0 * WP + k.dc0;
        int p1 = k.pl1 * PIXA + m0 + k.dr1 * WP + k.dc1;
        uint64_t ad = desc(xb + (uint32_t)p0 * 16u, (uint32_t)(p1 - p0) * 16u, 128);
        uint64_t bd = desc(wb + (uint32_t)(ph * nsteps + j) * wstep, (uint32_t)NP * 16u, 128);
        mma_bf16(d, ad, bd, idesc, j > 0);
      }
    }
  }
}

// Shared-memory carve-up, identical on host and device.
struct Smem {
  int wbytes, planes_bytes, in_bytes;
  int off_wm, off_wr, off_x0, off_x1, off_in, off_misc, total;
};
__host__ __device__ inline Smem smem_layout(int nsteps_total, int NP, int nplanes, int PIXA, int in_bytes) {
  Smem s;
  s.wbytes = nsteps_total * 2 * NP * 16;
  s.planes_bytes = nplanes * PIXA * 16;
  s.in_bytes = (in_bytes + 127) / 128 * 128;
  s.off_wm = 0;
  s.off_wr = s.wbytes;
  s.off_x0 = 2 * s.wbytes;
  s.off_x1 = s.off_x0 + s.planes_bytes;
  s.off_in = s.off_x1 + s.planes_bytes;
  s.off_misc = s.off_in + s.in_bytes;
  s.total = s.off_misc + kTcMiscBytes;
  return s;
}

// Misc area: [0, 512) K-step table, [512, 1024) ECA g / s (input),
// [1024, 1536) ECA s (skip), [1536, 4096) stage-1 weights + bias,
// [4096, 5120) stem weights + bias, [5120, 7168) per-warp channel sums,
// [7168] mbarrier, [7176] TMEM slot.
struct Misc {
  KStep* ks;
  float *g, *sa, *ss, *dw, *dwb, *stw, *stb, *red;
  uint64_t* bar;
  uint32_t* tslot;
  __device__ Misc(unsigned char* p, int CI) {
    ks = (KStep*)p;
    g = (float*)(p + 512);
    sa = g + 64;
    ss = (float*)(p + 1024);
    dw = (float*)(p + 1536);
    dwb = dw + 9 * CI;
    stw = (float*)(p + 4096);
    stb = stw + 216;
    red = (float*)(p + 5120);
    bar = (uint64_t*)(p + 7168);
    tslot = (uint32_t*)(p + 7176);
  }
};

__device__ void copy_to_smem(void* dst, const void* src, int bytes) {
  const uint4* s = (const uint4*)src;
  uint4* d = (uint4*)dst;
  for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = s[i];
}

__device__ void zero_smem(void* dst, int bytes) {
  uint4* d = (uint4*)dst;
  for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = make_uint4(0, 0, 0, 0);
}

// Waits for the MMAs, reads one accumulator row (16 columns) per call.
__device__ __forceinline__ uint32_t lane_addr(uint32_t tmem, int warp, int col) {
  return tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)col;
}

// ---------------------------------------------------------------- encoder
template <int CI, bool STEM>
__global__ void __launch_bounds__(kThreads) k_enc_tc(TcArgs a) {
  constexpr int CO = 2 * CI, G = CI / 8, NP = CO;
  extern __shared__ __align__(1024) unsigned char sm[];
  const int nsteps = (CI == 8) ? 5 : 9 * CI / 16;
  const int in_bytes = STEM ? 3 * (2 * a.band + 6) * (a.w + 6) * 2 : 0;
  const Smem L = smem_layout(nsteps, NP, 4 * G, a.PIXA, in_bytes);
  Misc M(sm + L.off_misc, CI);
  __nv_bfloat16* x0 = (__nv_bfloat16*)(sm + L.off_x0);
  __nv_bfloat16* x1 = (__nv_bfloat16*)(sm + L.off_x1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.y, band = blockIdx.x, TY = a.band;
  const int h = a.h, w = a.w, ho = h / 2, wo = w / 2;
  const int oy0 = band * TY, WP = a.WP, PIXA = a.PIXA;

  if (warp == 0) tmem_alloc(M.tslot, a.tmem_cols);
  if (tid == 0) {
    mbar_init(M.bar, 1);
    mbar_fence_init();
  }
  copy_to_smem(sm + L.off_wm, a.L.wm, L.wbytes);
  copy_to_smem(sm + L.off_wr, a.L.wr, L.wbytes);
  zero_smem(sm + L.off_x0, 2 * L.planes_bytes);
  for (int i = tid; i < nsteps; i += blockDim.x) M.ks[i] = a.L.ks[i];
  for (int i = tid; i < 9 * CI; i += blockDim.x) M.dw[i] = a.dw[i];
  for (int i = tid; i < CI; i += blockDim.x) M.dwb[i] = a.dwb[i];
  for (int i = tid; i < 8 * CO; i += blockDim.x) M.red[i] = 0.f;
  if (STEM) {
    for (int i = tid; i < 216; i += blockDim.x) M.stw[i] = a.stem_w[i];
    for (int i = tid; i < 8; i += blockDim.x) M.stb[i] = a.stem_b[i];
  } else {
    eca_scales(a.ppart + (size_t)b * a.ptiles * CI, a.ptiles, CI, 1.f / (float)(h * w), a.pk3, M.g, M.sa);
  }
  __syncthreads();

  // 1. block input x into the four phase planes: plane (py, px) holds
  // x[2r + py][2s + px] at local row r - (oy0 - 1), column s + 1.
  const int y_lo = max(0, 2 * oy0 - 2), y_hi = min(h - 1, 2 * oy0 + 2 * TY + 1);
  if (STEM) {
    const int RI = 2 * TY + 6, CW = w + 6, yi0 = 2 * oy0 - 3;
    __nv_bfloat16* sin = (__nv_bfloat16*)(sm + L.off_in);
    const __nv_bfloat16* in = a.in + (size_t)b * 3 * h * w;
    for (int i = tid; i < 3 * RI * CW; i += blockDim.x) {
      int c = i / (RI * CW), r = (i / CW) % RI, q = i % CW, y = yi0 + r, x = q - 3;
      sin[i] = (y >= 0 && y < h && x >= 0 && x < w) ? in[((size_t)c * h + y) * w + x] : __float2bfloat16(0.f);
    }
    __syncthreads();
    for (int i = tid; i < (y_hi - y_lo + 1) * w; i += blockDim.x) {
      int y = y_lo + i / w, x = i % w;
      float acc[8];
#pragma unroll
      for (int o = 0; o < 8; ++o) acc[o] = M.stb[o];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int t = 0; t < 9; ++t) {
          float v = __bfloat162float(sin[(c * RI + y - yi0 + t / 3 - 1) * CW + x + 3 + t % 3 - 1]);
#pragma unroll
          for (int o = 0; o < 8; ++o) acc[o] += v * M.stw[(c * 9 + t) * 8 + o];
        }
#pragma unroll
      for (int o = 0; o < 8; ++o) acc[o] = fmaxf(acc[o], 0.f);
      int pl = (y & 1) * 2 + (x & 1), p = ((y >> 1) - oy0 + 1) * WP + (x >> 1) + 1;
      *(uint4*)(x0 + ((size_t)pl * PIXA + p) * 8) = f32_to_bf16x8(acc);
    }
  } else {
    const __nv_bfloat16* in = a.in + (size_t)b * h * w * CI;
    for (int i = tid; i < (y_hi - y_lo + 1) * w * G; i += blockDim.x) {
      int g = i % G, pos = i / G, y = y_lo + pos / w, x = pos % w;
      float f[8];
      bf16x8_to_f32(*(const uint4*)(in + ((size_t)y * w + x) * CI + g * 8), f);
#pragma unroll
      for (int c = 0; c < 8; ++c) f[c] *= M.sa[g * 8 + c];
      int pl = ((y & 1) * 2 + (x & 1)) * G + g, p = ((y >> 1) - oy0 + 1) * WP + (x >> 1) + 1;
      *(uint4*)(x0 + ((size_t)pl * PIXA + p) * 8) = f32_to_bf16x8(f);
    }
  }
  __syncthreads();
  // 2. stage 1 at the rows the stride-2 taps read: y in [2 oy0 - 1, 2 oy0 + 2 TY - 1]
  {
    const int y1_lo = max(0, 2 * oy0 - 1), y1_hi = min(h - 1, 2 * oy0 + 2 * TY - 1);
    for (int i = tid; i < (y1_hi - y1_lo + 1) * w * G; i += blockDim.x) {
      int g = i % G, pos = i / G, y = y1_lo + pos / w, x = pos % w;
      float acc[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[c] = M.dwb[g * 8 + c];
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
        int pl = ((yy & 1) * 2 + (xx & 1)) * G + g, p = ((yy >> 1) - oy0 + 1) * WP + (xx >> 1) + 1;
        float f[8];
        bf16x8_to_f32(*(const uint4*)(x0 + ((size_t)pl * PIXA + p) * 8), f);
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] += M.dw[t * CI + g * 8 + c] * f[c];
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[c] = fmaxf(acc[c], 0.f);
      int pl = ((y & 1) * 2 + (x & 1)) * G + g, p = ((y >> 1) - oy0 + 1) * WP + (x >> 1) + 1;
      *(uint4*)(x1 + ((size_t)pl * PIXA + p) * 8) = f32_to_bf16x8(acc);
    }
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *M.tslot;
  const int m_lo = WP + 1;
  // 3. stage 2 on the tensor cores
  if (tid == 0) {
    issue_mmas(tmem, M.ks, nsteps, 1, NP, a.ntile, m_lo, WP, PIXA, smem_u32(x1), smem_u32(x0),
               smem_u32(sm + L.off_wm), smem_u32(sm + L.off_wr));
    commit(M.bar);
  }
  const bool ok = mbar_wait(M.bar, 0);
  fence_after_sync();
  if (!ok) {
    if (tid == 0) atomicExch(a.status, (int)STDA_ERR_TIMEOUT);
    mbar_wait(M.bar, 0);  // bounded: let issued MMAs drain before TMEM is freed
  } else {
    // 4. epilogue: warps w and w + 4 share TMEM lanes; they take alternate tiles
    for (int i = warp >> 2; i < a.ntile; i += 2) {
      int m = m_lo + 128 * i + (warp & 3) * 32 + lane;
      int lr = m / WP, lc = m % WP, oy = oy0 + lr - 1, ox = lc - 1;
      bool valid = lr >= 1 && lr <= TY && oy < ho && ox >= 0 && ox < wo;
      __nv_bfloat16* dst = a.out + (((size_t)b * ho + oy) * wo + ox) * CO;
#pragma unroll
      for (int c = 0; c < CO; c += 16) {
        float mv[16], rv[16];
        ld16(lane_addr(tmem, warp, i * 2 * NP + c), mv);
        ld16(lane_addr(tmem, warp, i * 2 * NP + NP + c), rv);
        ld_wait();
        float o[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) o[j] = valid ? fmaxf(mv[j] + a.b2[c + j], 0.f) + rv[j] + a.rb[c + j] : 0.f;
        if (valid) {
          *(uint4*)(dst + c) = f32_to_bf16x8(o);
          *(uint4*)(dst + c + 8) = f32_to_bf16x8(o + 8);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) warp_sum_to(o[j], &M.red[warp * CO + c + j]);
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, a.tmem_cols);
  float* part = a.part + ((size_t)b * gridDim.x + band) * CO;
  for (int c = tid; c < CO; c += blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < 8; ++k) s += M.red[k * CO + c];
    part[c] = s;
  }
}

// ---------------------------------------------------------------- decoder
template <int CI, bool SKIP>
__global__ void __launch_bounds__(kThreads) k_dec_tc(TcArgs a) {
  constexpr int CO = CI / 2, G = CI / 8, NP = CO < 16 ? 16 : CO;
  extern __shared__ __align__(1024) unsigned char sm[];
  const int nsteps = 4 * CI / 16;  // per output phase
  const Smem L = smem_layout(4 * nsteps, NP, G, a.PIXA, 0);
  Misc M(sm + L.off_misc, CI);
  __nv_bfloat16* x0 = (__nv_bfloat16*)(sm + L.off_x0);
  __nv_bfloat16* x1 = (__nv_bfloat16*)(sm + L.off_x1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.y, band = blockIdx.x, TA = a.band;
  const int h = a.h, w = a.w, Ho = 2 * h, Wo = 2 * w;
  const int a0 = band * TA, WP = a.WP, PIXA = a.PIXA;

  if (warp == 0) tmem_alloc(M.tslot, a.tmem_cols);
  if (tid == 0) {
    mbar_init(M.bar, 1);
    mbar_fence_init();
  }
  copy_to_smem(sm + L.off_wm, a.L.wm, L.wbytes);
  copy_to_smem(sm + L.off_wr, a.L.wr, L.wbytes);
  zero_smem(sm + L.off_x0, 2 * L.planes_bytes);
  for (int i = tid; i < 4 * nsteps; i += blockDim.x) M.ks[i] = a.L.ks[i];
  for (int i = tid; i < 9 * CI; i += blockDim.x) M.dw[i] = a.dw[i];
  for (int i = tid; i < CI; i += blockDim.x) M.dwb[i] = a.dwb[i];
  for (int i = tid; i < 8 * CO; i += blockDim.x) M.red[i] = 0.f;
  const float inv_n = 1.f / (float)(h * w);
  eca_scales(a.ppart + (size_t)b * a.ptiles * CI, a.ptiles, CI, inv_n, a.pk3, M.g, M.sa);
  if (SKIP) eca_scales(a.spart + (size_t)b * a.stiles * CI, a.stiles, CI, inv_n, a.sk3, M.g, M.ss);
  __syncthreads();

  // 1. x = ECA(A) (+ ECA(skip)) at rows a0 - 2 .. a0 + TA + 1; plane pixel
  // (r - a0 + 2) * WP + (c + 2)
  {
    const int r_lo = max(0, a0 - 2), r_hi = min(h - 1, a0 + TA + 1);
    const __nv_bfloat16* A = a.in + (size_t)b * h * w * CI;
    const __nv_bfloat16* S = SKIP ? a.skip + (size_t)b * h * w * CI : nullptr;
    for (int i = tid; i < (r_hi - r_lo + 1) * w * G; i += blockDim.x) {
      int g = i % G, pos = i / G, r = r_lo + pos / w, c = pos % w;
      size_t off = ((size_t)r * w + c) * CI + g * 8;
      float f[8];
      bf16x8_to_f32(*(const uint4*)(A + off), f);
#pragma unroll
      for (int k = 0; k < 8; ++k) f[k] *= M.sa[g * 8 + k];
      if (SKIP) {
        float s[8];
        bf16x8_to_f32(*(const uint4*)(S + off), s);
#pragma unroll
        for (int k = 0; k < 8; ++k) f[k] += M.ss[g * 8 + k] * s[k];
      }
      int p = (r - a0 + 2) * WP + c + 2;
      *(uint4*)(x0 + ((size_t)g * PIXA + p) * 8) = f32_to_bf16x8(f);
    }
  }
  __syncthreads();
  // 2. stage 1 at rows a0 - 1 .. a0 + TA (the sub-pixel taps reach +-1)
  {
    const int r_lo = max(0, a0 - 1), r_hi = min(h - 1, a0 + TA);
    for (int i = tid; i < (r_hi - r_lo + 1) * w * G; i += blockDim.x) {
      int g = i % G, pos = i / G, r = r_lo + pos / w, c = pos % w;
      int p = (r - a0 + 2) * WP + c + 2;
      float acc[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = M.dwb[g * 8 + k];
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        float f[8];
        bf16x8_to_f32(*(const uint4*)(x0 + ((size_t)g * PIXA + p + (t / 3 - 1) * WP + t % 3 - 1) * 8), f);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += M.dw[t * CI + g * 8 + k] * f[k];
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = fmaxf(acc[k], 0.f);
      *(uint4*)(x1 + ((size_t)g * PIXA + p) * 8) = f32_to_bf16x8(acc);
    }
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *M.tslot;
  const int m_lo = 2 * WP + 2;
  if (tid == 0) {
    issue_mmas(tmem, M.ks, nsteps, 4, NP, a.ntile, m_lo, WP, PIXA, smem_u32(x1), smem_u32(x0),
               smem_u32(sm + L.off_wm), smem_u32(sm + L.off_wr));
    commit(M.bar);
  }
  const bool ok = mbar_wait(M.bar, 0);
  fence_after_sync();
  if (!ok) {
    if (tid == 0) atomicExch(a.status, (int)STDA_ERR_TIMEOUT);
    mbar_wait(M.bar, 0);  // bounded: let issued MMAs drain before TMEM is freed
  } else {
    for (int i = warp >> 2; i < a.ntile; i += 2) {
      int m = m_lo + 128 * i + (warp & 3) * 32 + lane;
      int lr = m / WP, lc = m % WP, r = a0 + lr - 2, c = lc - 2;
      bool valid = lr >= 2 && lr < TA + 2 && r < h && c >= 0 && c < w;
#pragma unroll 1
      for (int ph = 0; ph < 4; ++ph) {
        int Y = 2 * r + (ph >> 1), X = 2 * c + (ph & 1);
        __nv_bfloat16* dst = a.out + (((size_t)b * Ho + Y) * Wo + X) * CO;
#pragma unroll
        for (int cc = 0; cc < CO; cc += 8) {
          float mv[8], rv[8], o[8];
          ld8(lane_addr(tmem, warp, (i * 8 + ph) * NP + cc), mv);
          ld8(lane_addr(tmem, warp, (i * 8 + 4 + ph) * NP + cc), rv);
          ld_wait();
#pragma unroll
          for (int j = 0; j < 8; ++j) o[j] = valid ? fmaxf(mv[j] + a.b2[cc + j], 0.f) + rv[j] + a.rb[cc + j] : 0.f;
          if (valid) *(uint4*)(dst + cc) = f32_to_bf16x8(o);
#pragma unroll
          for (int j = 0; j < 8; ++j) warp_sum_to(o[j], &M.red[warp * CO + cc + j]);
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, a.tmem_cols);
  float* part = a.part + ((size_t)b * gridDim.x + band) * CO;
  for (int c = tid; c < CO; c += blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < 8; ++k) s += M.red[k * CO + c];
    part[c] = s;
  }
}

uint32_t pow2_cols(int cols) {
  uint32_t n = 32;
  while ((int)n < cols) n <<= 1;
  return n;
}

int cdiv(int a, int b) { return (a + b - 1) / b; }

// Band geometry of one level: the largest band (8, 4, 2 or 1 rows) whose
// accumulators fit the 512 TMEM columns and whose planes fit shared memory.
struct Geo {
  int band, ntile, WP, PIXA, smem;
  uint32_t cols;
};

Geo encoder_geo(int CI, bool stem, int h, int w) {
  const int CO = 2 * CI, G = CI / 8, wo = w / 2, nsteps = CI == 8 ? 5 : 9 * CI / 16;
  Geo g{};
  for (int TY = 8; TY >= 1; TY >>= 1) {
    g.band = TY;
    g.WP = wo + 2;
    int m_lo = g.WP + 1, count = TY * g.WP + wo - m_lo + 1;
    g.ntile = cdiv(count, 128);
    g.PIXA = std::max((TY + 2) * g.WP, m_lo + 128 * g.ntile + 1);
    g.PIXA = (g.PIXA + 7) / 8 * 8;
    int in_bytes = stem ? 3 * (2 * TY + 6) * (w + 6) * 2 : 0;
    g.smem = smem_layout(nsteps, CO, 4 * G, g.PIXA, in_bytes).total;
    g.cols = pow2_cols(g.ntile * 2 * CO);
    if (g.ntile * 2 * CO <= 512 && g.smem <= kTcMaxSmem) return g;
  }
  g.band = 0;
  return g;
}

Geo decoder_geo(int CI, int h, int w) {
  const int CO = CI / 2, G = CI / 8, NP = CO < 16 ? 16 : CO, nsteps = 4 * CI / 16;
  Geo g{};
  for (int TA = 8; TA >= 1; TA >>= 1) {
    g.band = TA;
    g.WP = w + 4;
    int m_lo = 2 * g.WP + 2, count = (TA - 1) * g.WP + w;
    g.ntile = cdiv(count, 128);
    g.PIXA = std::max((TA + 4) * g.WP, m_lo + 128 * g.ntile + g.WP + 1);
    g.PIXA = (g.PIXA + 7) / 8 * 8;
    g.smem = smem_layout(4 * nsteps, NP, G, g.PIXA, 0).total;
    g.cols = pow2_cols(g.ntile * 8 * NP);
    if (g.ntile * 8 * NP <= 512 && g.smem <= kTcMaxSmem) return g;
  }
  g.band = 0;
  return g;
}

template <typename K>
cudaError_t launch(K kern, const Geo& g, int B, const TcArgs& a, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, g.smem);
  if (e) return e;
  kern<<<dim3(a.tiles_per_window, B), kThreads, g.smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

// ------------------------------------------------------------ host packing
namespace {
// Encoder tap (ky, kx) of the stride-2 3x3 conv -> polyphase plane and
// shift: input row 2 oy - 1 + ky lies in the odd plane one row up (ky = 0),
// the even plane (ky = 1) or the odd plane (ky = 2).
int tap_phase(int k) { return k == 1 ? 0 : 1; }
int tap_shift(int k) { return k == 0 ? -1 : 0; }
}  // namespace

void pack_tc(const float* folded, const FoldedOffsets& off, std::vector<unsigned char>* blob, TcPackOffsets* po) {
  std::vector<__nv_bfloat16> w;
  std::vector<KStep> ks_all;
  std::vector<size_t> ks_start(6);
  size_t wm_elems[6], wr_elems[6];
  for (int b = 0; b < kNumBlocks; ++b) {
    const int ci = kBlkCin[b], co = kBlkCout[b], G = ci / 8;
    const bool enc = kBlkEnc[b];
    const int NP = enc ? co : (co < 16 ? 16 : co);
    std::vector<KStep> ks;
    // each K-step: two (tap, channel group) halves; weights w(tap, ci, co)
    struct Half {
      int tap, g;  // tap < 0: zero half
    };
    std::vector<std::pair<Half, Half>> halves;
    if (enc) {
      auto tap_ks = [&](int t, int g) {
        int ky = t / 3, kx = t % 3;
        return std::make_tuple((tap_phase(ky) * 2 + tap_phase(kx)) * G + g, tap_shift(ky), tap_shift(kx));
      };
      if (ci == 8) {
        const int pairs[5][2] = {{0, 2}, {6, 8}, {1, 7}, {3, 5}, {4, -1}};
        for (auto& pr : pairs) {
          auto [p0, r0, c0] = tap_ks(pr[0], 0);
          KStep k{(int8_t)p0, (int8_t)r0, (int8_t)c0, (int8_t)p0, (int8_t)r0, (int8_t)(c0 + 1), 0, 0};
          if (pr[1] >= 0) {
            auto [p1, r1, c1] = tap_ks(pr[1], 0);
            k.pl1 = (int8_t)p1;
            k.dr1 = (int8_t)r1;
            k.dc1 = (int8_t)c1;
          }
          ks.push_back(k);
          halves.push_back({{pr[0], 0}, {pr[1], 0}});
        }
      } else {
        for (int t = 0; t < 9; ++t)
          for (int kg = 0; kg < G / 2; ++kg) {
            auto [p0, r0, c0] = tap_ks(t, 2 * kg);
            ks.push_back({(int8_t)p0, (int8_t)r0, (int8_t)c0, (int8_t)(p0 + 1), (int8_t)r0, (int8_t)c0, 0, 0});
            halves.push_back({{t, 2 * kg}, {t, 2 * kg + 1}});
          }
      }
    } else {
      for (int ph = 0; ph < 4; ++ph) {
        int py = ph >> 1, px = ph & 1;
        for (int st = 0; st < 4; ++st)
          for (int kg = 0; kg < G / 2; ++kg) {
            int dy = (st >> 1) - 1 + py, dx = (st & 1) - 1 + px;
            ks.push_back({(int8_t)(2 * kg), (int8_t)dy, (int8_t)dx, (int8_t)(2 * kg + 1), (int8_t)dy, (int8_t)dx, 0,
                          0});
            halves.push_back({{ph * 4 + st, 2 * kg}, {ph * 4 + st, 2 * kg + 1}});
          }
      }
    }
    // packed [step][half][n < NP][8]
    for (int br = 0; br < 2; ++br) {
      const float* src = folded + (br == 0 ? off.w2[b] : off.rw[b]);
      (br == 0 ? wm_elems[b] : wr_elems[b]) = w.size();
      for (auto& hh : halves)
        for (int hf = 0; hf < 2; ++hf) {
          Half h = hf == 0 ? hh.first : hh.second;
          for (int n = 0; n < NP; ++n)
            for (int c = 0; c < 8; ++c) {
              float v = 0.f;
              if (h.tap >= 0 && n < co) v = src[((size_t)h.tap * ci + h.g * 8 + c) * co + n];
              w.push_back(__float2bfloat16(v));
            }
        }
      while (w.size() % 64) w.push_back(__float2bfloat16(0.f));  // 128-byte alignment
    }
    ks_start[b] = ks_all.size();
    ks_all.insert(ks_all.end(), ks.begin(), ks.end());
  }
  size_t wbytes = w.size() * sizeof(__nv_bfloat16);
  blob->assign(wbytes + ks_all.size() * sizeof(KStep), 0);
  std::memcpy(blob->data(), w.data(), wbytes);
  std::memcpy(blob->data() + wbytes, ks_all.data(), ks_all.size() * sizeof(KStep));
  for (int b = 0; b < kNumBlocks; ++b) {
    po->wm[b] = wm_elems[b] * sizeof(__nv_bfloat16);
    po->wr[b] = wr_elems[b] * sizeof(__nv_bfloat16);
    po->ks[b] = wbytes + ks_start[b] * sizeof(KStep);
  }
  po->total = blob->size();
}

TcWeights tc_weights_from(const unsigned char* base, const TcPackOffsets& po) {
  TcWeights t;
  for (int b = 0; b < kNumBlocks; ++b)
    t.layer[b] = TcLayer{(const __nv_bfloat16*)(base + po.wm[b]), (const __nv_bfloat16*)(base + po.wr[b]),
                         (const KStep*)(base + po.ks[b])};
  return t;
}

cudaError_t forward_tc(const NetW& w, const TcWeights& tw, const __nv_bfloat16* in, __nv_bfloat16* out, int B,
                       int H, int W, const FwdScratch& s, int* status, cudaStream_t st, KernelHook* hook,
                       int* tiles_out) {
  cudaError_t e = cudaSuccess;
  int tiles[6];
  const void* prev = nullptr;
  for (int l = 0; l < 6; ++l) {
    const int ci = kBlkCin[l];
    static const int in_div[6] = {1, 2, 4, 8, 4, 2};
    const int h = H / in_div[l], wd = W / in_div[l];
    Geo g = kBlkEnc[l] ? encoder_geo(ci, l == 0, h, wd) : decoder_geo(ci, h, wd);
    if (g.band == 0) return cudaErrorInvalidConfiguration;
    TcArgs a{};
    a.in = (const __nv_bfloat16*)(l == 0 ? (const void*)in : prev);
    if (l > 0) {
      a.ppart = s.part[l - 1];
      a.pk3 = w.blk[l - 1].eca;
      a.ptiles = tiles[l - 1];
    }
    if (l == 4 || l == 5) {  // D2 += E2 -> input of D2 is D1 + E2; input of D3 is D2 + E1
      int sk = l == 4 ? 1 : 0;
      a.skip = (const __nv_bfloat16*)s.act[sk];
      a.spart = s.part[sk];
      a.sk3 = w.blk[sk].eca;
      a.stiles = tiles[sk];
    }
    a.h = h;
    a.w = wd;
    a.band = g.band;
    a.ntile = g.ntile;
    a.WP = g.WP;
    a.PIXA = g.PIXA;
    a.tmem_cols = g.cols;
    a.stem_w = w.stem_w;
    a.stem_b = w.stem_b;
    a.dw = w.blk[l].dw;
    a.dwb = w.blk[l].dwb;
    a.b2 = w.blk[l].b2;
    a.rb = w.blk[l].rb;
    a.L = tw.layer[l];
    a.out = (__nv_bfloat16*)s.act[l];
    a.part = s.part[l];
    a.status = status;
    const int rows = kBlkEnc[l] ? h / 2 : h;
    a.tiles_per_window = cdiv(rows, g.band);
    tiles[l] = a.tiles_per_window;
    hook->begin(K_ENC1 + l, st);
    switch (l) {
      case 0: e = launch(k_enc_tc<8, true>, g, B, a, st); break;
      case 1: e = launch(k_enc_tc<16, false>, g, B, a, st); break;
      case 2: e = launch(k_enc_tc<32, false>, g, B, a, st); break;
      case 3: e = launch(k_dec_tc<64, false>, g, B, a, st); break;
      case 4: e = launch(k_dec_tc<32, true>, g, B, a, st); break;
      case 5: e = launch(k_dec_tc<16, true>, g, B, a, st); break;
    }
    hook->end(st);
    if (e) return e;
    prev = s.act[l];
  }
  if (tiles_out)
    for (int l = 0; l < 6; ++l) tiles_out[l] = tiles[l];
  return cudaSuccess;
}

}  // namespace stda
