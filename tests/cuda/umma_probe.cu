// Unit probes of the tcgen05 primitives in csrc/umma.h (test-only library).
//
// probe_gemm: D[128][N] = A[128][K] * B[N][K]^T, A and B staged in shared
//   memory in the no-swizzle K-major core-matrix layout the forward kernels
//   use; one thread issues K/16 MMAs into TMEM; the result is read back with
//   tcgen05.ld. Shared buffers are sized so that the tensor core stays in
//   bounds even if the LBO / SBO roles were the other way round.
// probe_conv: a 3x3 convolution (16 -> 32 channels) on a padded plane, one
//   M-tile of 128 consecutive plane pixels, each tap an MMA whose A operand
//   starts at the tap's shifted pixel (16-byte granular start addresses).
// Both return 0, or 1 if a bounded wait gave up.
#include <cuda_bf16.h>

#include "../../paper_2307_09063_gb300/csrc/umma.h"

using namespace stda::umma;

namespace {

constexpr int kA = 48 * 1024, kB = 16 * 1024;

__global__ void k_probe_gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, float* D, int N, int K,
                             int* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __nv_bfloat16* sA = (__nv_bfloat16*)sm;
  __nv_bfloat16* sB = (__nv_bfloat16*)(sm + kA);
  uint64_t* bar = (uint64_t*)(sm + kA + kB);
  uint32_t* tslot = (uint32_t*)(sm + kA + kB + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < (kA + kB) / 2; i += blockDim.x) ((__nv_bfloat16*)sm)[i] = __float2bfloat16(0.f);
  __syncthreads();
  // element (m, k) -> core matrix (k/8, m/8): ((k/8) * 16 + m/8) * 64 + (m%8) * 8 + k%8
  for (int i = tid; i < 128 * K; i += blockDim.x) {
    int m = i / K, k = i % K;
    sA[((k / 8) * 16 + m / 8) * 64 + (m % 8) * 8 + k % 8] = A[i];
  }
  for (int i = tid; i < N * K; i += blockDim.x) {
    int n = i / K, k = i % K;
    sB[((k / 8) * (N / 8) + n / 8) * 64 + (n % 8) * 8 + k % 8] = B[i];
  }
  if (warp == 0) tmem_alloc(tslot, 64);
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t lboA = 16 * 128, lboB = (N / 8) * 128;
  if (tid == 0) {
    for (int ks = 0; ks < K / 16; ++ks) {
      uint64_t a = desc(smem_u32(sA) + ks * 2 * lboA, lboA, 128);
      uint64_t b = desc(smem_u32(sB) + ks * 2 * lboB, lboB, 128);
      mma_bf16(tmem, a, b, idesc_bf16(128, N), ks > 0);
    }
    commit(bar);
  }
  bool ok = mbar_wait(bar, 0);
  fence_after_sync();
  if (!ok) {
    if (tid == 0) atomicExch(status, 1);
  } else if (warp < 4) {
    for (int c = 0; c < N; c += 16) {
      float v[16];
      ld16(tmem + ((uint32_t)(warp * 32) << 16) + c, v);
      ld_wait();
      for (int j = 0; j < 16; ++j) D[(warp * 32 + lane) * N + c + j] = v[j];
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 64);
}

// Plane: 10 rows x 16 columns (1-pixel margin around an 8 x 14 image),
// two channel groups of 8; tail padding so every shifted M-tile read stays
// inside the plane buffer. The shared buffer is padded to 100 KB so that
// reads stay inside it under either reading of LBO / SBO.
constexpr int kWp = 16, kRows = 10, kPix = 320;
constexpr int kWBytes = 9 * 2 * 32 * 16, kConvSmem = 100 * 1024;

__global__ void k_probe_conv(const __nv_bfloat16* X /*[kRows*kWp][16]*/, const __nv_bfloat16* Wt /*[9][32][16]*/,
                             float* D /*[128][32]*/, int* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __nv_bfloat16* sW = (__nv_bfloat16*)sm;             // [9 taps][2 halves][32][8]
  __nv_bfloat16* sX = (__nv_bfloat16*)(sm + kWBytes); // [2 groups][kPix][8]
  uint64_t* bar = (uint64_t*)(sm + kConvSmem);
  uint32_t* tslot = (uint32_t*)(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < kConvSmem / 2; i += blockDim.x) ((__nv_bfloat16*)sm)[i] = __float2bfloat16(0.f);
  __syncthreads();
  for (int i = tid; i < 2 * kPix * 8; i += blockDim.x) {
    int g = i / (kPix * 8), p = (i / 8) % kPix, c = i % 8;
    sX[i] = p < kRows * kWp ? X[p * 16 + g * 8 + c] : __float2bfloat16(0.f);
  }
  for (int i = tid; i < 9 * 32 * 16; i += blockDim.x) {
    int t = i / 512, n = (i / 16) % 32, k = i % 16;
    sW[((t * 2 + k / 8) * 32 + n) * 8 + k % 8] = Wt[i];
  }
  if (warp == 0) tmem_alloc(tslot, 32);
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  fence_proxy_async();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  const int m0 = kWp + 1;
  if (tid == 0) {
    for (int t = 0; t < 9; ++t) {
      int dy = t / 3 - 1, dx = t % 3 - 1;
      uint64_t a = desc(smem_u32(sX) + (m0 + dy * kWp + dx) * 16, kPix * 16, 128);
      uint64_t b = desc(smem_u32(sW) + t * 2 * 32 * 16, 32 * 16, 128);
      mma_bf16(tmem, a, b, idesc_bf16(128, 32), t > 0);
    }
    commit(bar);
  }
  bool ok = mbar_wait(bar, 0);
  fence_after_sync();
  if (!ok) {
    if (tid == 0) atomicExch(status, 1);
  } else if (warp < 4) {
    for (int c = 0; c < 32; c += 16) {
      float v[16];
      ld16(tmem + ((uint32_t)(warp * 32) << 16) + c, v);
      ld_wait();
      for (int j = 0; j < 16; ++j) D[(warp * 32 + lane) * 32 + c + j] = v[j];
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 32);
}

}  // namespace

extern "C" int probe_gemm(const void* A, const void* B, float* D, int N, int K, int* status) {
  if (N < 16 || N > 64 || N % 16 || K < 16 || K > 64 || K % 16) return -1;
  size_t smem = kA + kB + 64;
  cudaFuncSetAttribute(k_probe_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_probe_gemm<<<1, 128, smem>>>((const __nv_bfloat16*)A, (const __nv_bfloat16*)B, D, N, K, status);
  return (int)cudaDeviceSynchronize();
}

extern "C" int probe_conv(const void* X, const void* Wt, float* D, int* status) {
  size_t smem = kConvSmem + 64;
  cudaFuncSetAttribute(k_probe_conv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_probe_conv<<<1, 128, smem>>>((const __nv_bfloat16*)X, (const __nv_bfloat16*)Wt, D, status);
  return (int)cudaDeviceSynchronize();
}
