// stda_forward_static: the FP32 forward pass without any device allocation.
//
// Some callers cannot call cudaMalloc: real-time radar pipelines that forbid
// allocation after start-up (an allocation can synchronise the device and
// take milliseconds), plug-ins whose host application owns all device memory,
// and code that must not perturb a memory budget. This entry point lets them
// run the denoiser with only the buffers they already hold: the parameters,
// the input windows and the output maps. The folded weights and the
// activation scratch live in one file-scope __device__ array that every GPU
// loading the library holds until the process exits.
//
// The array's name is only a host-side stand-in in host code; the device
// address is fetched once per device with cudaGetSymbolAddress, with that
// device current, on the first call made on it.
#include <cuda_runtime.h>

#include <mutex>

#include "stda_internal.h"

namespace stda {
namespace {

constexpr size_t kStaticBytes = (size_t)8 << 20;  // 8 MiB
constexpr size_t kStaticMaxPixels = 65536;          // B * H * W per call
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices];

// Offsets of every tensor in the canonical parameter blob and BN buffers.
struct CanonOffsets {
  int stem_w, stem_g, stem_b, stem_m, stem_v;
  int w1[6], g1[6], b1[6], w3[6], g2[6], b2[6], g3[6], b3[6], w2[6], g[6], be[6], rw[6], rb[6], eca[6];
  int m1[6], v1[6], m2[6], v2[6], m3[6], v3[6], m[6], v[6];
  int out_w, out_b;
};

CanonOffsets canon_offsets() {
  CanonOffsets o;
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

// BN in inference form as an affine map: scale and shift of channel c
// (FP32, like the forward it feeds).
__device__ float bn_scale(const float* P, const float* Bf, int g, int v, int c) {
  return P[g + c] / sqrtf(Bf[v + c] + 1e-5f);
}
__device__ float bn_shift(const float* P, const float* Bf, int g, int be, int m, int v, int c) {
  return P[be + c] - Bf[m + c] * bn_scale(P, Bf, g, v, c);
}

// Folds the canonical parameters into the kernels' layout (the same layout
// and the same algebra as the host path of stda_set_params, which folds in
// FP64), in FP32, grid-stride.
__global__ void k_fold(const float* __restrict__ P, const float* __restrict__ Bf, float* __restrict__ F,
                       CanonOffsets co, FoldedOffsets fo) {
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  for (int i = t0; i < 216; i += nt) {
    int o = i / 27, r = i % 27;
    F[fo.stem_w + r * 8 + o] = P[co.stem_w + i] * bn_scale(P, Bf, co.stem_g, co.stem_v, o);
  }
  for (int i = t0; i < 8; i += nt)
    F[fo.stem_b + i] = bn_shift(P, Bf, co.stem_g, co.stem_b, co.stem_m, co.stem_v, i);
  const int cins[6] = {8, 16, 32, 64, 32, 16}, couts[6] = {16, 32, 64, 32, 16, 8};
  for (int b = 0; b < 6; ++b) {
    const int ci = cins[b], cout = couts[b];
    const bool enc = b < 3;
    for (int i = t0; i < 9 * ci; i += nt) {
      int t = i / ci, ch = i % ci;
      float k = bn_scale(P, Bf, co.g2[b], co.v2[b], ch) * P[co.w3[b] + ch * 9 + (enc ? t : 8 - t)];
      if (t == 4)
        k += bn_scale(P, Bf, co.g1[b], co.v1[b], ch) * P[co.w1[b] + ch] + bn_scale(P, Bf, co.g3[b], co.v3[b], ch);
      F[fo.dw[b] + i] = k;
    }
    for (int ch = t0; ch < ci; ch += nt)
      F[fo.dwb[b] + ch] = bn_shift(P, Bf, co.g1[b], co.b1[b], co.m1[b], co.v1[b], ch) +
                          bn_shift(P, Bf, co.g2[b], co.b2[b], co.m2[b], co.v2[b], ch) +
                          bn_shift(P, Bf, co.g3[b], co.b3[b], co.m3[b], co.v3[b], ch);
    const int dense = (enc ? 9 : 16) * ci * cout;
    for (int d = t0; d < dense; d += nt) {
      int o = d % cout, i = (d / cout) % ci, kk = d / (cout * ci);  // kk = tap, or phase * 4 + sub-tap
      size_t s;
      if (enc) {
        s = ((size_t)o * ci + i) * 9 + kk;
      } else {
        int ph = kk / 4, st = kk % 4, py = ph >> 1, px = ph & 1, sy = st >> 1, sx = st & 1;
        int ky = py + 1 - 2 * (sy - 1 + py), kx = px + 1 - 2 * (sx - 1 + px);
        s = (((size_t)i * cout + o) * 4 + ky) * 4 + kx;
      }
      F[fo.w2[b] + d] = P[co.w2[b] + s] * bn_scale(P, Bf, co.g[b], co.v[b], o);
      F[fo.rw[b] + d] = P[co.rw[b] + s];
    }
    for (int o = t0; o < cout; o += nt) {
      F[fo.b2[b] + o] = bn_shift(P, Bf, co.g[b], co.be[b], co.m[b], co.v[b], o);
      F[fo.rb[b] + o] = P[co.rb[b] + o];
    }
    for (int j = t0; j < 3; j += nt) F[fo.eca[b] + j] = P[co.eca[b] + j];
  }
  for (int i = t0; i < 72; i += nt) {
    int ch = i / 9, t = i % 9;
    F[fo.out_w + t * 8 + ch] = P[co.out_w + i];
  }
  if (t0 == 0) F[fo.out_b] = P[co.out_b];
}

// Device address of the static array on the current device (set up once
// per device).
cudaError_t static_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

struct NoHook : KernelHook {
  void begin(int, cudaStream_t) override {}
  void end(cudaStream_t) override {}
};

}  // namespace
}  // namespace stda

extern "C" stda_status stda_forward_static(const float* d_params, const float* d_buffers, const float* d_in,
                                           float* d_out, int B, int H, int W, cudaStream_t stream) {
  using namespace stda;
  if (B < 0 || H <= 0 || W <= 0 || H % 8 || W % 8) return STDA_ERR_SHAPE;
  if (B == 0) return STDA_OK;
  if (!d_params || !d_buffers || !d_in || !d_out) return STDA_ERR_INVALID_ARG;
  if ((size_t)B * H * W > kStaticMaxPixels) return STDA_ERR_SHAPE;
  const FoldedOffsets fo = folded_layout();
  const size_t wbytes = (fo.total * sizeof(float) + 255) / 256 * 256;
  if (wbytes + scratch_bytes(B, H, W, sizeof(float)) > kStaticBytes) return STDA_ERR_SHAPE;
  void* base = nullptr;
  cudaError_t e = static_address(&base);
  if (e) {
    cudaGetLastError();
    return STDA_ERR_CUDA;
  }
  float* folded = (float*)base;
  k_fold<<<64, 256, 0, stream>>>(d_params, d_buffers, folded, canon_offsets(), fo);
  FwdScratch s;
  scratch_carve((unsigned char*)base + wbytes, B, H, W, sizeof(float), &s);
  NoHook hook;
  e = forward_simt<float>(net_from(folded, fo), d_in, d_out, B, H, W, s, stream, &hook);
  if (e) {
    cudaGetLastError();
    return STDA_ERR_CUDA;
  }
  return STDA_OK;
}
