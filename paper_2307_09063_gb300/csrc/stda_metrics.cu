// Evaluation of denoised maps on the GPU (Sec. V-B): SINR and EVM at the
// targets' peak cells with FP64 sums, and a cell-averaging CFAR detector
// with the fraction of targets it finds.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "stda_internal.h"

namespace stda {
namespace {

constexpr int kMaxTgt = 16;

__device__ __forceinline__ double val(const void* p, int bf16, size_t i) {
  return bf16 ? (double)__bfloat162float(((const __nv_bfloat16*)p)[i]) : (double)((const float*)p)[i];
}

// 0 = noise cell, 1 = peak cell, 2 = guard cell of some peak
__device__ __forceinline__ int cell_kind(const int* bins, int nb, int p, int q, int guard) {
  int kind = 0;
  for (int o = 0; o < nb; ++o) {
    int dp = p - bins[2 * o], dq = q - bins[2 * o + 1];
    if (dp == 0 && dq == 0) return 1;
    if (dp >= -guard && dp <= guard && dq >= -guard && dq <= guard) kind = 2;
  }
  return kind;
}

// One block per window. Eq. (SINR): 10 log10(mean_O z^2 / mean_N z^2);
// Eq. (EVM): mean over peak cells of |clean - est| / |clean|.
__global__ void k_sinr_evm(const void* maps, const void* clean, int bf16, const int* bins, const int* ntgt, int H,
                           int W, int guard, double* sinr, double* evm) {
  const int b = blockIdx.x;
  const int nb = min(ntgt[b], kMaxTgt);
  const int* bb = bins + (size_t)b * kMaxTgt * 2;
  const size_t n = (size_t)H * W, base = (size_t)b * n;
  double so = 0.0, sn = 0.0, no = 0.0, nn = 0.0, ev = 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
    int p = (int)(i / W), q = (int)(i % W);
    int k = cell_kind(bb, nb, p, q, guard);
    double z = val(maps, bf16, base + i), e = z * z;
    if (k == 1) {
      so += e;
      no += 1.0;
      if (clean) {
        double c = val(clean, bf16, base + i);
        ev += fabs(c - z) / fabs(c);
      }
    } else if (k == 0) {
      sn += e;
      nn += 1.0;
    }
  }
  double v[5] = {so, sn, no, nn, ev};
  for (int j = 0; j < 5; ++j)
    for (int o = 16; o; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
  __shared__ double acc[5][32];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int j = 0; j < 5; ++j) acc[j][warp] = v[j];
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[5] = {0, 0, 0, 0, 0};
    for (int j = 0; j < 5; ++j)
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t[j] += acc[j][k];
    sinr[b] = (t[2] > 0 && t[3] > 0) ? 10.0 * log10((t[0] / t[2]) / (t[1] / t[3])) : nan("");
    if (evm) evm[b] = t[2] > 0 ? t[4] / t[2] : nan("");
  }
}

// One thread per cell: training-cell power summed in FP64 in a fixed order,
// factor alpha[N] (N training cells) from a host table.
__global__ void k_cacfar(const void* maps, int bf16, int B, int H, int W, int guard, int train,
                         const double* alpha, unsigned char* det) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)B * H * W) return;
  const int q = idx % W, p = (idx / W) % H;
  const size_t base = (size_t)(idx / ((long)H * W)) * H * W;
  const int R = guard + train;
  double s = 0.0;
  int n = 0;
  for (int dp = -R; dp <= R; ++dp)
    for (int dq = -R; dq <= R; ++dq) {
      if (dp >= -guard && dp <= guard && dq >= -guard && dq <= guard) continue;
      int pp = p + dp, qq = q + dq;
      if (pp < 0 || pp >= H || qq < 0 || qq >= W) continue;
      double z = val(maps, bf16, base + (size_t)pp * W + qq);
      s += z * z;
      ++n;
    }
  double z = val(maps, bf16, idx), c = z * z;
  det[idx] = n > 0 && c > alpha[n] * (s / (double)n);
}

// One thread per window: fraction of distinct targets with a detection
// within +-1 cell.
__global__ void k_detect_rate(const unsigned char* det, const int* bins, const int* ntgt, int B, int H, int W,
                              float* rate) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int nb = min(ntgt[b], kMaxTgt);
  const int* bb = bins + (size_t)b * kMaxTgt * 2;
  const unsigned char* d = det + (size_t)b * H * W;
  int hit = 0, cnt = 0;
  for (int o = 0; o < nb; ++o) {
    bool dup = false;
    for (int k = 0; k < o; ++k) dup |= bb[2 * k] == bb[2 * o] && bb[2 * k + 1] == bb[2 * o + 1];
    if (dup) continue;
    ++cnt;
    bool found = false;
    for (int dp = -1; dp <= 1; ++dp)
      for (int dq = -1; dq <= 1; ++dq) {
        int pp = bb[2 * o] + dp, qq = bb[2 * o + 1] + dq;
        if (pp >= 0 && pp < H && qq >= 0 && qq < W && d[(size_t)pp * W + qq]) found = true;
      }
    hit += found;
  }
  rate[b] = cnt ? (float)hit / (float)cnt : nanf("");
}

}  // namespace

cudaError_t metrics(const void* maps, const void* clean, int bf16, const int* bins, const int* ntgt, int B, int H,
                    int W, int guard, int cfar_guard, int cfar_train, double pfa, double* sinr, double* evm,
                    float* det_rate, unsigned char* det, cudaStream_t st) {
  if (sinr || evm) {
    double* s = sinr;
    if (!s && cudaMallocAsync((void**)&s, sizeof(double) * B, st)) return cudaErrorMemoryAllocation;
    k_sinr_evm<<<B, 256, 0, st>>>(maps, clean, bf16, bins, ntgt, H, W, guard, s, evm);
    if (!sinr) cudaFreeAsync(s, st);
  }
  if (det || det_rate) {
    const int R = cfar_guard + cfar_train, nmax = (2 * R + 1) * (2 * R + 1);
    std::vector<double> a(nmax + 1, 0.0);
    for (int n = 1; n <= nmax; ++n) a[n] = (double)n * (std::pow(pfa, -1.0 / (double)n) - 1.0);
    double* d_alpha;
    unsigned char* d = det;
    if (cudaMallocAsync((void**)&d_alpha, sizeof(double) * (nmax + 1), st)) return cudaErrorMemoryAllocation;
    if (!d && cudaMallocAsync((void**)&d, (size_t)B * H * W, st)) return cudaErrorMemoryAllocation;
    cudaMemcpyAsync(d_alpha, a.data(), sizeof(double) * (nmax + 1), cudaMemcpyHostToDevice, st);
    long n = (long)B * H * W;
    k_cacfar<<<(int)((n + 255) / 256), 256, 0, st>>>(maps, bf16, B, H, W, cfar_guard, cfar_train, d_alpha, d);
    if (det_rate) k_detect_rate<<<(B + 63) / 64, 64, 0, st>>>(d, bins, ntgt, B, H, W, det_rate);
    cudaStreamSynchronize(st);  // the host table must outlive the copy
    cudaFreeAsync(d_alpha, st);
    if (!det) cudaFreeAsync(d, st);
  }
  return cudaGetLastError();
}

}  // namespace stda
