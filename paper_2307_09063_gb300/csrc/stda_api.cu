// libstda C-ABI: context, parameters, BN folding, dispatch.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "stda_internal.h"
#include "stda_tc.h"
#include "stda_train.h"
#include "stda_serve.h"

namespace stda {

// ----------------------------------------------------------------------------
// Parameter initialisation: every value is U(lo, hi) from a SplitMix64 hash
// of (seed, 0, 0, tag, tensor id, element), in FP64, rounded to FP32.
// Distributions: conv / deconv weights U(+-sqrt(6 / fan)) with fan = Cin/g *
// k^2 (conv) or Cin/g * k^2 / s^2 (transposed conv); biases U(+-0.05); BN
// gamma U(0.8, 1.2), beta U(+-0.1), running mean U(+-0.1), running variance
// U(0.8, 1.2); ECA kernels U(+-0.577); the output conv weights carry a gain
// of 3 so that the sigmoid output is spread out.
// ----------------------------------------------------------------------------
namespace {

uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ULL;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
  return x ^ (x >> 31);
}

double u01(uint64_t seed, uint64_t tag, uint64_t i1, uint64_t i2) {
  uint64_t h = mix64(seed);
  h = mix64(h ^ 0);
  h = mix64(h ^ 0);
  h = mix64(h ^ tag);
  h = mix64(h ^ i1);
  h = mix64(h ^ i2);
  return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

constexpr uint64_t TAG_WEIGHT = 20, TAG_BN_MEAN = 21, TAG_BN_VAR = 22;
constexpr double kOutGain = 3.0;
constexpr double kBnEps = 1e-5;

struct Tensor {
  int size;
  double lo, hi;
  bool out_w;
};

std::vector<Tensor> param_table(int frames) {
  std::vector<Tensor> t;
  auto conv = [&](int size, int fan) {
    double b = std::sqrt(6.0 / fan);
    t.push_back({size, -b, b, false});
  };
  auto bn = [&](int c) {
    t.push_back({c, 0.8, 1.2, false});
    t.push_back({c, -0.1, 0.1, false});
  };
  conv(8 * frames * 9, frames * 9);
  bn(8);
  for (int b = 0; b < kNumBlocks; ++b) {
    int ci = kBlkCin[b], co = kBlkCout[b];
    conv(ci, 1);
    bn(ci);
    conv(9 * ci, 9);
    bn(ci);
    bn(ci);
    int dense = kBlkEnc[b] ? co * ci * 9 : ci * co * 16;
    int fan = kBlkEnc[b] ? ci * 9 : ci * 16 / 4;
    conv(dense, fan);
    bn(co);
    conv(dense, fan);
    t.push_back({co, -0.05, 0.05, false});
    t.push_back({3, -0.577, 0.577, false});
  }
  conv(72, 72);
  t.back().out_w = true;
  t.push_back({1, -0.05, 0.05, false});
  return t;
}

std::vector<int> bn_channels() {
  std::vector<int> c{8};
  for (int b = 0; b < kNumBlocks; ++b) {
    c.push_back(kBlkCin[b]);
    c.push_back(kBlkCin[b]);
    c.push_back(kBlkCin[b]);
    c.push_back(kBlkCout[b]);
  }
  return c;
}

}  // namespace

size_t num_params(int frames) {
  size_t n = 0;
  for (const Tensor& t : param_table(frames)) n += t.size;
  return n;
}

void init_params(uint64_t seed, float* params, float* buffers, int frames) {
  auto tab = param_table(frames);
  size_t off = 0;
  for (size_t tid = 0; tid < tab.size(); ++tid) {
    const Tensor& t = tab[tid];
    for (int i = 0; i < t.size; ++i) {
      double u = u01(seed, TAG_WEIGHT, tid, (uint64_t)i);
      double v = t.lo + (t.hi - t.lo) * u;
      if (t.out_w) v = v * kOutGain;
      params[off++] = (float)v;
    }
  }
  auto ch = bn_channels();
  size_t q = 0;
  for (size_t bid = 0; bid < ch.size(); ++bid) {
    for (int i = 0; i < ch[bid]; ++i) buffers[q + i] = (float)(-0.1 + 0.2 * u01(seed, TAG_BN_MEAN, bid, i));
    for (int i = 0; i < ch[bid]; ++i)
      buffers[q + ch[bid] + i] = (float)(0.8 + 0.4 * u01(seed, TAG_BN_VAR, bid, i));
    q += 2 * ch[bid];
  }
}

// ----------------------------------------------------------------------------
// BN folding (inference form): BN(y) = s * y + t, s = gamma / sqrt(var + eps),
// t = beta - mean * s. Stage 1 of a block is BN1(dw1x1 x) + BN2(dw3x3 x) +
// BN3(x): one depthwise 3x3 cross-correlation whose centre tap gathers
// s1 * w1 + s3, bias t1 + t2 + t3. The decoder's stride-1 transposed 3x3 is
// the cross-correlation with the kernel flipped in both axes.
// ----------------------------------------------------------------------------
FoldedOffsets folded_layout(int frames) {
  FoldedOffsets o;
  size_t p = 0;
  auto take = [&](size_t n) {
    size_t r = p;
    p += (n + 63) / 64 * 64;
    return r;
  };
  o.stem_w = take(frames * 9 * 8);
  o.stem_b = take(8);
  for (int b = 0; b < kNumBlocks; ++b) {
    int ci = kBlkCin[b], co = kBlkCout[b];
    size_t dense = (size_t)(kBlkEnc[b] ? 9 : 16) * ci * co;
    o.dw[b] = take(9 * ci);
    o.dwb[b] = take(ci);
    o.w2[b] = take(dense);
    o.b2[b] = take(co);
    o.rw[b] = take(dense);
    o.rb[b] = take(co);
    o.eca[b] = take(3);
  }
  o.out_w = take(72);
  o.out_b = take(1);
  o.total = p;
  return o;
}

namespace {
struct Cursor {
  const float* p;
  std::vector<double> take(int n) {
    std::vector<double> v(p, p + n);
    p += n;
    return v;
  }
};
struct BnFold {
  std::vector<double> s, t;
};
BnFold bn_fold(const std::vector<double>& g, const std::vector<double>& be, const float*& buf, int c) {
  BnFold r;
  r.s.resize(c);
  r.t.resize(c);
  for (int i = 0; i < c; ++i) {
    double mean = buf[i], var = buf[c + i];
    r.s[i] = g[i] / std::sqrt(var + kBnEps);
    r.t[i] = be[i] - mean * r.s[i];
  }
  buf += 2 * c;
  return r;
}
}  // namespace

void fold_params(const float* params, const float* buffers, float* dst, FoldedOffsets* off, int frames) {
  *off = folded_layout(frames);
  std::memset(dst, 0, sizeof(float) * off->total);
  Cursor c{params};
  const float* bq = buffers;
  {
    auto w = c.take(8 * frames * 9);
    auto g = c.take(8);
    auto be = c.take(8);
    BnFold f = bn_fold(g, be, bq, 8);
    for (int o = 0; o < 8; ++o)
      for (int ci = 0; ci < frames; ++ci)
        for (int t = 0; t < 9; ++t)
          dst[off->stem_w + (ci * 9 + t) * 8 + o] = (float)(w[(o * frames + ci) * 9 + t] * f.s[o]);
    for (int o = 0; o < 8; ++o) dst[off->stem_b + o] = (float)f.t[o];
  }
  for (int b = 0; b < kNumBlocks; ++b) {
    int ci = kBlkCin[b], co = kBlkCout[b];
    bool enc = kBlkEnc[b];
    int dense = enc ? co * ci * 9 : ci * co * 16;
    auto w1 = c.take(ci);
    auto g1 = c.take(ci), b1 = c.take(ci);
    auto w3 = c.take(9 * ci);
    auto g2 = c.take(ci), b2 = c.take(ci);
    auto g3 = c.take(ci), b3 = c.take(ci);
    auto w2 = c.take(dense);
    auto g = c.take(co), be = c.take(co);
    auto rw = c.take(dense);
    auto rb = c.take(co);
    auto eca = c.take(3);
    BnFold f1 = bn_fold(g1, b1, bq, ci), f2 = bn_fold(g2, b2, bq, ci), f3 = bn_fold(g3, b3, bq, ci);
    BnFold fm = bn_fold(g, be, bq, co);
    for (int ch = 0; ch < ci; ++ch) {
      for (int t = 0; t < 9; ++t) {
        double k = f2.s[ch] * w3[ch * 9 + (enc ? t : 8 - t)];
        if (t == 4) k += f1.s[ch] * w1[ch] + f3.s[ch];
        dst[off->dw[b] + t * ci + ch] = (float)k;
      }
      dst[off->dwb[b] + ch] = (float)(f1.t[ch] + f2.t[ch] + f3.t[ch]);
    }
    if (enc) {
      for (int o = 0; o < co; ++o)
        for (int i = 0; i < ci; ++i)
          for (int t = 0; t < 9; ++t) {
            size_t d = ((size_t)t * ci + i) * co + o;
            dst[off->w2[b] + d] = (float)(w2[((size_t)o * ci + i) * 9 + t] * fm.s[o]);
            dst[off->rw[b] + d] = (float)rw[((size_t)o * ci + i) * 9 + t];
          }
    } else {
      for (int py = 0; py < 2; ++py)
        for (int px = 0; px < 2; ++px)
          for (int sy = 0; sy < 2; ++sy)
            for (int sx = 0; sx < 2; ++sx) {
              int dy = sy - 1 + py, dx = sx - 1 + px;
              int ky = py + 1 - 2 * dy, kx = px + 1 - 2 * dx;
              int ph = py * 2 + px, st = sy * 2 + sx;
              for (int i = 0; i < ci; ++i)
                for (int o = 0; o < co; ++o) {
                  size_t s = (((size_t)i * co + o) * 4 + ky) * 4 + kx;
                  size_t d = (((size_t)ph * 4 + st) * ci + i) * co + o;
                  dst[off->w2[b] + d] = (float)(w2[s] * fm.s[o]);
                  dst[off->rw[b] + d] = (float)rw[s];
                }
            }
    }
    for (int o = 0; o < co; ++o) {
      dst[off->b2[b] + o] = (float)fm.t[o];
      dst[off->rb[b] + o] = (float)rb[o];
    }
    for (int j = 0; j < 3; ++j) dst[off->eca[b] + j] = (float)eca[j];
  }
  auto ow = c.take(72);
  auto ob = c.take(1);
  for (int ch = 0; ch < 8; ++ch)
    for (int t = 0; t < 9; ++t) dst[off->out_w + t * 8 + ch] = (float)ow[ch * 9 + t];
  dst[off->out_b] = (float)ob[0];
}

// Inference network in PyTorch weight layouts (the order documented with
// stda_reparam_export), BN folded in FP64 exactly as fold_params does.
size_t reparam_count(int frames) {
  size_t n = 8 * frames * 9 + 8 + 72 + 1;
  for (int b = 0; b < kNumBlocks; ++b) {
    const size_t ci = kBlkCin[b], co = kBlkCout[b], dense = (kBlkEnc[b] ? 9 : 16) * ci * co;
    n += 9 * ci + ci + 2 * dense + 2 * co + 3;
  }
  return n;
}

void reparam_export(const float* params, const float* buffers, int frames, float* out) {
  Cursor c{params};
  const float* bq = buffers;
  float* o = out;
  {
    auto w = c.take(8 * frames * 9);
    auto g = c.take(8);
    auto be = c.take(8);
    BnFold f = bn_fold(g, be, bq, 8);
    for (int oc = 0; oc < 8; ++oc)
      for (int k = 0; k < frames * 9; ++k) *o++ = (float)(w[oc * frames * 9 + k] * f.s[oc]);
    for (int oc = 0; oc < 8; ++oc) *o++ = (float)f.t[oc];
  }
  for (int b = 0; b < kNumBlocks; ++b) {
    const int ci = kBlkCin[b], co = kBlkCout[b];
    const bool enc = kBlkEnc[b];
    const int dense = enc ? co * ci * 9 : ci * co * 16;
    auto w1 = c.take(ci);
    auto g1 = c.take(ci), b1 = c.take(ci);
    auto w3 = c.take(9 * ci);
    auto g2 = c.take(ci), b2 = c.take(ci);
    auto g3 = c.take(ci), b3 = c.take(ci);
    auto w2 = c.take(dense);
    auto g = c.take(co), be = c.take(co);
    auto rw = c.take(dense);
    auto rb = c.take(co);
    auto eca = c.take(3);
    BnFold f1 = bn_fold(g1, b1, bq, ci), f2 = bn_fold(g2, b2, bq, ci), f3 = bn_fold(g3, b3, bq, ci);
    BnFold fm = bn_fold(g, be, bq, co);
    for (int ch = 0; ch < ci; ++ch)
      for (int t = 0; t < 9; ++t) {
        double k = f2.s[ch] * w3[ch * 9 + (enc ? t : 8 - t)];
        if (t == 4) k += f1.s[ch] * w1[ch] + f3.s[ch];
        *o++ = (float)k;
      }
    for (int ch = 0; ch < ci; ++ch) *o++ = (float)(f1.t[ch] + f2.t[ch] + f3.t[ch]);
    // main conv: the output channel is the first index of a Conv2d weight,
    // the second of a ConvTranspose2d weight
    for (int i = 0; i < dense; ++i) {
      const int oc = enc ? i / (ci * 9) : (i / 16) % co;
      *o++ = (float)(w2[i] * fm.s[oc]);
    }
    for (int oc = 0; oc < co; ++oc) *o++ = (float)fm.t[oc];
    for (int i = 0; i < dense; ++i) *o++ = (float)rw[i];
    for (int oc = 0; oc < co; ++oc) *o++ = (float)rb[oc];
    for (int j = 0; j < 3; ++j) *o++ = (float)eca[j];
  }
  auto ow = c.take(72);
  auto ob = c.take(1);
  for (int k = 0; k < 72; ++k) *o++ = (float)ow[k];
  *o++ = (float)ob[0];
}

const char* const kKernelNames[K_NUM_IDS] = {"enc1_stem", "enc2", "enc3", "dec1", "dec2", "dec3", "out"};

NetW net_from(const float* base, const FoldedOffsets& o, int frames) {
  NetW n;
  n.frames = frames;
  n.stem_w = base + o.stem_w;
  n.stem_b = base + o.stem_b;
  for (int b = 0; b < kNumBlocks; ++b)
    n.blk[b] = BlockW{base + o.dw[b], base + o.dwb[b], base + o.w2[b], base + o.b2[b],
                      base + o.rw[b], base + o.rb[b], base + o.eca[b]};
  n.out_w = base + o.out_w;
  n.out_b = base + o.out_b;
  return n;
}

}  // namespace stda

// ============================================================================
// C-ABI
// ============================================================================
namespace {
// Counts launches; when enabled, records a CUDA event pair around every
// launch on the launch's own stream.
struct Profiler : stda::KernelHook {
  bool on = false;
  uint64_t launches = 0;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  int cur_id = 0;
  cudaEvent_t cur = nullptr;
  struct Rec {
    int id;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  cudaEvent_t next() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  void begin(int id, cudaStream_t st) override {
    ++launches;
    if (!on) return;
    cur_id = id;
    cur = next();
    cudaEventRecord(cur, st);
  }
  void end(cudaStream_t st) override {
    if (!on) return;
    cudaEvent_t e = next();
    cudaEventRecord(e, st);
    recs.push_back({cur_id, cur, e});
  }
  void reset() {
    recs.clear();
    used = 0;
  }
  ~Profiler() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};
}  // namespace

struct stda_ctx {
  Profiler prof;
  stda_config cfg;
  int frames = 3;  // stacked maps per window
  int device = 0;
  std::vector<float> params, buffers;
  stda::FoldedOffsets off;
  float* d_folded = nullptr;
  stda::NetW net;
  unsigned char* d_tc = nullptr;  // packed tensor-core weights and K-step tables
  size_t d_tc_bytes = 0;
  stda::TcPackOffsets tc_off;
  stda::TcWeights tcw;
  float* d_canon = nullptr;  // canonical parameters + BN buffers (training graph)
  void* d_train = nullptr;   // training workspace
  size_t train_bytes = 0;
  float* d_target32 = nullptr;  // float copy of bf16 targets
  stda::Serve* serve = nullptr;
  void* d_scratch = nullptr;
  size_t scratch_size = 0;
  int* d_status = nullptr;
  uint32_t wait_polls = stda::kWaitPolls;  // bound of the tensor-core kernels' tile waits
  cudaStream_t last_stream = nullptr;
  // forward passes and training steps captured as CUDA graphs, by their
  // buffers and shape, most recent last; replayed on the caller's stream. A
  // call is captured the second time its key is seen (one-off calls run
  // directly); exec is null for a key seen once.
  struct GraphKey {
    uintptr_t p[10];
    int i[5];
    bool operator==(const GraphKey& o) const {
      for (int k = 0; k < 10; ++k)
        if (p[k] != o.p[k]) return false;
      for (int k = 0; k < 5; ++k)
        if (i[k] != o.i[k]) return false;
      return true;
    }
  };
  struct Graph {
    GraphKey key;
    int launches;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  cudaStream_t cap = nullptr;  // private stream the captures run on
  // host-buffer forward: two staging pairs (max_batch windows each), copy
  // streams, and per pair the events input copied / forward done / output copied
  void* d_hin[2] = {};
  void* d_hout[2] = {};
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t ev_h[2] = {}, ev_f[2] = {}, ev_d[2] = {};
  bool f_recorded[2] = {};
  uint64_t host_calls = 0;
  std::string err;
};

namespace {

stda_status fail(stda_ctx* c, stda_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

stda_status cuda_fail(stda_ctx* c, cudaError_t e, const char* where) {
  cudaGetLastError();
  return fail(c, e == cudaErrorMemoryAllocation ? STDA_ERR_OOM : STDA_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

size_t elem_size(stda_precision p) { return p == STDA_FP32 ? 4 : 2; }

// Captured forwards hold the weight, scratch and status pointers and the
// wait bound as kernel parameters: drop them whenever one of those changes.
void drop_graphs(stda_ctx* c) {
  for (auto& g : c->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
}

stda_status upload_weights(stda_ctx* c) {
  drop_graphs(c);
  std::vector<float> host(stda::folded_layout(c->frames).total);
  stda::fold_params(c->params.data(), c->buffers.data(), host.data(), &c->off, c->frames);
  cudaError_t e = cudaMemcpy(c->d_folded, host.data(), host.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e) return cuda_fail(c, e, "upload weights");
  c->net = stda::net_from(c->d_folded, c->off, c->frames);
  std::vector<unsigned char> blob;
  // FP8: E4M3 stage-2 operands in every block but the first (8 input channels)
  bool f8[6];
  const bool fp8 = c->cfg.prec == STDA_FP8_E4M3 || c->cfg.prec == STDA_FP8_E4M3_FAST;
  for (int b = 0; b < 6; ++b) f8[b] = fp8 && b > 0;
  stda::pack_tc(host.data(), c->off, c->frames, f8, c->cfg.prec == STDA_FP8_E4M3_FAST ? 1 : 2, &blob, &c->tc_off);
  if (c->d_tc && blob.size() > c->d_tc_bytes) {
    cudaFree(c->d_tc);
    c->d_tc = nullptr;
  }
  if (!c->d_tc) {
    if ((e = cudaMalloc((void**)&c->d_tc, blob.size()))) return cuda_fail(c, e, "alloc tc weights");
    c->d_tc_bytes = blob.size();
  }
  if ((e = cudaMemcpy(c->d_tc, blob.data(), blob.size(), cudaMemcpyHostToDevice)))
    return cuda_fail(c, e, "upload tc weights");
  c->tcw = stda::tc_weights_from(c->d_tc, c->tc_off);
  if (c->frames != 3) return STDA_OK;  // the training graph is the three-map network
  if (!c->d_canon &&
      (e = cudaMalloc((void**)&c->d_canon, sizeof(float) * (stda::kNumParams + stda::kNumBuffers))))
    return cuda_fail(c, e, "alloc canonical parameters");
  if ((e = cudaMemcpy(c->d_canon, c->params.data(), sizeof(float) * stda::kNumParams, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(c->d_canon + stda::kNumParams, c->buffers.data(), sizeof(float) * stda::kNumBuffers,
                      cudaMemcpyHostToDevice)))
    return cuda_fail(c, e, "upload canonical parameters");
  return STDA_OK;
}

bool shape_ok(int H, int W) { return H > 0 && W > 0 && H % 8 == 0 && W % 8 == 0; }

// The forward pass's kernels on `st` (seven launches; per-kernel hooks).
cudaError_t run_forward(stda_ctx* c, const void* d_in, void* d_out, int B, int H, int W, cudaStream_t st,
                        stda::KernelHook* hook) {
  const size_t es = elem_size(c->cfg.prec);
  stda::FwdScratch s;
  stda::scratch_carve(c->d_scratch, B, H, W, es, &s);
  cudaError_t e;
  if (c->cfg.prec == STDA_FP32)
    return stda::forward_simt<float>(c->net, (const float*)d_in, (float*)d_out, B, H, W, s, st, hook);
  int tiles[6];
  e = stda::forward_tc(c->net, c->tcw, (const __nv_bfloat16*)d_in, (__nv_bfloat16*)d_out, B, H, W, s, c->d_status,
                       st, hook, tiles, c->wait_polls);
  if (!e)
    e = stda::launch_out_bf16(c->net, (const __nv_bfloat16*)s.act[5], s.part[5], tiles[5], (__nv_bfloat16*)d_out, B,
                              H, W, st, hook);
  return e;
}

// Counts the launches of a captured forward.
struct Counter : stda::KernelHook {
  int n = 0;
  void begin(int, cudaStream_t) override { ++n; }
  void end(cudaStream_t) override {}
};
constexpr size_t kMaxGraphs = 8;

// Runs body(stream, hook) for `key`: directly the first time the key is
// seen, then captured once as a CUDA graph on the private stream and
// replayed on `st` (launch counts of the captured forward kernels added).
template <typename Body>
stda_status run_cached(stda_ctx* c, const stda_ctx::GraphKey& key, cudaStream_t st, const char* what, Body body) {
  cudaError_t e;
  size_t gi = 0;
  while (gi < c->graphs.size() && !(c->graphs[gi].key == key)) ++gi;
  if (gi == c->graphs.size()) {
    if (c->graphs.size() == kMaxGraphs) {
      if (c->graphs.front().exec) cudaGraphExecDestroy(c->graphs.front().exec);
      c->graphs.erase(c->graphs.begin());
    }
    c->graphs.push_back({key, 0, nullptr});
    if ((e = body(st, &c->prof))) return cuda_fail(c, e, what);
    return STDA_OK;
  }
  if (!c->graphs[gi].exec) {
    if (!c->cap && (e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking))) return cuda_fail(c, e, what);
    Counter cnt;
    if ((e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal))) return cuda_fail(c, e, what);
    const cudaError_t fe = body(c->cap, &cnt);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(c->cap, &graph);
    if (fe || e) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(c, fe ? fe : e, what);
    }
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e) return cuda_fail(c, e, what);
    c->graphs[gi].exec = exec;
    c->graphs[gi].launches = cnt.n;
  }
  if ((e = cudaGraphLaunch(c->graphs[gi].exec, st))) return cuda_fail(c, e, what);
  c->prof.launches += (uint64_t)c->graphs[gi].launches;
  return STDA_OK;
}

}  // namespace

extern "C" {


const char* stda_status_string(stda_status s) {
  switch (s) {
    case STDA_OK: return "ok";
    case STDA_ERR_INVALID_ARG: return "invalid argument";
    case STDA_ERR_SHAPE: return "invalid shape";
    case STDA_ERR_OOM: return "out of device memory";
    case STDA_ERR_CUDA: return "CUDA error";
    case STDA_ERR_TIMEOUT: return "device wait timed out";
    case STDA_ERR_BUSY: return "busy";
    case STDA_ERR_UNSUPPORTED: return "unsupported";
    case STDA_WARMUP: return "warming up (fewer than three frames)";
  }
  return "unknown status";
}

size_t stda_num_params(void) { return stda::kNumParams; }
size_t stda_num_buffers(void) { return stda::kNumBuffers; }

stda_status stda_create(const stda_config* cfg, stda_ctx** out) {
  if (!cfg || !out) return STDA_ERR_INVALID_ARG;
  *out = nullptr;
  if (!shape_ok(cfg->H, cfg->W) || cfg->max_batch < 1) return STDA_ERR_SHAPE;
  if (cfg->prec != STDA_FP32 && cfg->prec != STDA_BF16 && cfg->prec != STDA_FP8_E4M3 &&
      cfg->prec != STDA_FP8_E4M3_FAST)
    return STDA_ERR_INVALID_ARG;
  const int frames = cfg->frames == 0 ? 3 : cfg->frames;
  if (frames < 1 || frames > stda::kMaxFrames) return STDA_ERR_INVALID_ARG;
  stda_ctx* c = new stda_ctx;
  c->cfg = *cfg;
  c->frames = frames;
  cudaGetDevice(&c->device);
  c->params.resize(stda::num_params(frames));
  c->buffers.resize(stda::kNumBuffers);
  stda::init_params(cfg->weight_seed, c->params.data(), c->buffers.data(), frames);
  if (cudaMalloc((void**)&c->d_folded, stda::folded_layout(frames).total * sizeof(float))) {
    cudaGetLastError();
    stda_destroy(c);
    return STDA_ERR_OOM;
  }
  c->scratch_size = stda::scratch_bytes(cfg->max_batch, cfg->H, cfg->W, elem_size(cfg->prec));
  if (cudaMalloc(&c->d_scratch, c->scratch_size)) {
    cudaGetLastError();
    stda_destroy(c);
    return STDA_ERR_OOM;
  }
  if (cudaMalloc((void**)&c->d_status, sizeof(int)) || cudaMemset(c->d_status, 0, sizeof(int))) {
    cudaGetLastError();
    stda_destroy(c);
    return STDA_ERR_OOM;
  }
  stda_status s = upload_weights(c);
  if (s != STDA_OK) {
    stda_destroy(c);
    return s;
  }
  *out = c;
  return STDA_OK;
}

stda_status stda_destroy(stda_ctx* c) {
  if (!c) return STDA_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  if (c->d_folded) cudaFree(c->d_folded);
  if (c->d_scratch) cudaFree(c->d_scratch);
  if (c->d_status) cudaFree(c->d_status);
  if (c->d_tc) cudaFree(c->d_tc);
  if (c->d_canon) cudaFree(c->d_canon);
  if (c->d_train) cudaFree(c->d_train);
  if (c->d_target32) cudaFree(c->d_target32);
  if (c->serve) stda::serve_delete(c->serve);
  for (int k = 0; k < 2; ++k) {
    if (c->d_hin[k]) cudaFree(c->d_hin[k]);
    if (c->d_hout[k]) cudaFree(c->d_hout[k]);
    if (c->ev_h[k]) cudaEventDestroy(c->ev_h[k]);
    if (c->ev_f[k]) cudaEventDestroy(c->ev_f[k]);
    if (c->ev_d[k]) cudaEventDestroy(c->ev_d[k]);
  }
  if (c->h2d) cudaStreamDestroy(c->h2d);
  if (c->d2h) cudaStreamDestroy(c->d2h);
  drop_graphs(c);
  if (c->cap) cudaStreamDestroy(c->cap);
  delete c;
  return STDA_OK;
}

stda_status stda_init_params(uint64_t seed, float* params, float* buffers) {
  if (!params || !buffers) return STDA_ERR_INVALID_ARG;
  stda::init_params(seed, params, buffers);
  return STDA_OK;
}

size_t stda_reparam_count(int frames) {
  return frames >= 1 && frames <= stda::kMaxFrames ? stda::reparam_count(frames) : 0;
}

stda_status stda_reparam_export(const float* params, const float* buffers, int frames, float* out, size_t n) {
  if (!params || !buffers || !out || frames < 1 || frames > stda::kMaxFrames || n != stda::reparam_count(frames))
    return STDA_ERR_INVALID_ARG;
  stda::reparam_export(params, buffers, frames, out);
  return STDA_OK;
}

size_t stda_num_params_frames(int frames) {
  return frames >= 1 && frames <= stda::kMaxFrames ? stda::num_params(frames) : 0;
}

stda_status stda_init_params_frames(uint64_t seed, int frames, float* params, float* buffers) {
  if (!params || !buffers || frames < 1 || frames > stda::kMaxFrames) return STDA_ERR_INVALID_ARG;
  stda::init_params(seed, params, buffers, frames);
  return STDA_OK;
}

stda_status stda_get_params(stda_ctx* c, float* dst, size_t n) {
  if (!c || !dst || n != c->params.size()) return fail(c, STDA_ERR_INVALID_ARG, "get_params: bad arguments");
  std::memcpy(dst, c->params.data(), n * sizeof(float));
  return STDA_OK;
}

stda_status stda_set_params(stda_ctx* c, const float* src, size_t n) {
  if (!c || !src || n != c->params.size()) return fail(c, STDA_ERR_INVALID_ARG, "set_params: bad arguments");
  cudaDeviceSynchronize();
  std::memcpy(c->params.data(), src, n * sizeof(float));
  return upload_weights(c);
}

stda_status stda_get_buffers(stda_ctx* c, float* dst, size_t n) {
  if (!c || !dst || n != c->buffers.size()) return fail(c, STDA_ERR_INVALID_ARG, "get_buffers: bad arguments");
  std::memcpy(dst, c->buffers.data(), n * sizeof(float));
  return STDA_OK;
}

stda_status stda_set_buffers(stda_ctx* c, const float* src, size_t n) {
  if (!c || !src || n != c->buffers.size()) return fail(c, STDA_ERR_INVALID_ARG, "set_buffers: bad arguments");
  cudaDeviceSynchronize();
  std::memcpy(c->buffers.data(), src, n * sizeof(float));
  return upload_weights(c);
}

stda_status stda_forward(stda_ctx* c, const void* d_in, void* d_out, int B, int H, int W, cudaStream_t st) {
  if (!c) return STDA_ERR_INVALID_ARG;
  if (B < 0 || B > c->cfg.max_batch) return fail(c, STDA_ERR_SHAPE, "forward: batch out of range");
  if (!shape_ok(H, W)) return fail(c, STDA_ERR_SHAPE, "forward: H and W must be positive multiples of 8");
  if (B == 0) return STDA_OK;
  if (!d_in || !d_out) return fail(c, STDA_ERR_INVALID_ARG, "forward: null pointer");
  if (((uintptr_t)d_in | (uintptr_t)d_out) & 15)
    return fail(c, STDA_ERR_INVALID_ARG, "forward: buffers must be 16-byte aligned");
  size_t es = elem_size(c->cfg.prec);
  if (stda::scratch_bytes(B, H, W, es) > c->scratch_size)
    return fail(c, STDA_ERR_SHAPE, "forward: B*H*W exceeds the context's scratch");
  c->last_stream = st;
  cudaError_t e;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (c->prof.on || cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    // per-kernel timing, or the caller is capturing the stream: launch directly
    cudaGetLastError();
    e = run_forward(c, d_in, d_out, B, H, W, st, &c->prof);
    if (e) return cuda_fail(c, e, "forward");
    return STDA_OK;
  }
  stda_ctx::GraphKey key{};
  key.p[0] = (uintptr_t)d_in;
  key.p[1] = (uintptr_t)d_out;
  key.i[0] = B;
  key.i[1] = H;
  key.i[2] = W;
  key.i[3] = 1;  // forward
  return run_cached(c, key, st, "forward", [&](cudaStream_t s, stda::KernelHook* h) {
    return run_forward(c, d_in, d_out, B, H, W, s, h);
  });
}

stda_status stda_forward_host(stda_ctx* c, const void* h_in, void* h_out, int B, int H, int W, cudaStream_t st) {
  if (!c) return STDA_ERR_INVALID_ARG;
  if (B < 0 || B > c->cfg.max_batch) return fail(c, STDA_ERR_SHAPE, "forward_host: batch out of range");
  if (!shape_ok(H, W)) return fail(c, STDA_ERR_SHAPE, "forward_host: H and W must be positive multiples of 8");
  if ((size_t)B * H * W > (size_t)c->cfg.max_batch * c->cfg.H * c->cfg.W)
    return fail(c, STDA_ERR_SHAPE, "forward_host: B*H*W exceeds the context");
  if (B == 0) return STDA_OK;
  if (!h_in || !h_out) return fail(c, STDA_ERR_INVALID_ARG, "forward_host: null pointer");
  const size_t es = elem_size(c->cfg.prec);
  const size_t cap = (size_t)c->cfg.max_batch * c->cfg.H * c->cfg.W * es;
  cudaError_t e = cudaSuccess;
  if (!c->h2d) {
    for (int k = 0; k < 2 && !e; ++k)
      if (!(e = cudaMalloc(&c->d_hin[k], cap * c->frames))) e = cudaMalloc(&c->d_hout[k], cap);
    if (!e) e = cudaStreamCreateWithFlags(&c->h2d, cudaStreamNonBlocking);
    if (!e) e = cudaStreamCreateWithFlags(&c->d2h, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && !e; ++k)
      if (!(e = cudaEventCreateWithFlags(&c->ev_h[k], cudaEventDisableTiming)) &&
          !(e = cudaEventCreateWithFlags(&c->ev_f[k], cudaEventDisableTiming)))
        e = cudaEventCreateWithFlags(&c->ev_d[k], cudaEventDisableTiming);
    if (e) return cuda_fail(c, e, "forward_host: staging");
  }
  // staging pair k alternates between calls: this call's input copy only
  // waits for the forward that last read pair k (two calls back)
  const int k = (int)(c->host_calls++ & 1);
  const size_t nin = (size_t)B * c->frames * H * W * es, nout = (size_t)B * H * W * es;
  if (c->f_recorded[k] && (e = cudaStreamWaitEvent(c->h2d, c->ev_f[k], 0))) return cuda_fail(c, e, "forward_host");
  if ((e = cudaMemcpyAsync(c->d_hin[k], h_in, nin, cudaMemcpyHostToDevice, c->h2d)) ||
      (e = cudaEventRecord(c->ev_h[k], c->h2d)) || (e = cudaStreamWaitEvent(st, c->ev_h[k], 0)))
    return cuda_fail(c, e, "forward_host: input copy");
  // page-locked, device-mapped h_out (16-byte aligned, allocated or
  // registered with this device current): the output kernel stores the
  // result straight into it over the host link, so no copy back is queued
  // and the next call's forward need not wait for one
  void* direct = nullptr;
  cudaPointerAttributes pa{};
  int dev = -1;
  if (cudaPointerGetAttributes(&pa, h_out) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess) {
    if (pa.type == cudaMemoryTypeHost && pa.device == dev && pa.devicePointer &&
        ((uintptr_t)pa.devicePointer & 15) == 0)
      direct = pa.devicePointer;
  } else {
    cudaGetLastError();  // an unknown pointer is not an error here: the staged copy serves it
  }
  const stda_status r = stda_forward(c, c->d_hin[k], direct ? direct : c->d_hout[k], B, H, W, st);
  if (r != STDA_OK) return r;
  if ((e = cudaEventRecord(c->ev_f[k], st))) return cuda_fail(c, e, "forward_host");
  c->f_recorded[k] = true;
  if (direct) return STDA_OK;
  if ((e = cudaStreamWaitEvent(c->d2h, c->ev_f[k], 0)) ||
      (e = cudaMemcpyAsync(h_out, c->d_hout[k], nout, cudaMemcpyDeviceToHost, c->d2h)) ||
      (e = cudaEventRecord(c->ev_d[k], c->d2h)) || (e = cudaStreamWaitEvent(st, c->ev_d[k], 0)))
    return cuda_fail(c, e, "forward_host: output copy");
  return STDA_OK;
}

namespace {
__global__ void k_bf16_to_f32_flat(const __nv_bfloat16* a, float* o, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = __bfloat162float(a[i]);
}
}  // namespace

stda_status stda_backward(stda_ctx* c, const void* d_in, const void* d_target, const float* d_gout,
                          float* d_gparams, double* d_loss, float* d_gin, float* d_out, int B, int H, int W,
                          cudaStream_t st) {
  return stda_backward_bn(c, d_in, d_target, d_gout, d_gparams, d_loss, d_gin, d_out, B, H, W, STDA_BN_RUNNING,
                          nullptr, st);
}

stda_status stda_backward_bn(stda_ctx* c, const void* d_in, const void* d_target, const float* d_gout,
                             float* d_gparams, double* d_loss, float* d_gin, float* d_out, int B, int H, int W,
                             stda_bn_mode bn_mode, float* d_bn_stats, cudaStream_t st) {
  if (c && c->frames != 3) return fail(c, STDA_ERR_UNSUPPORTED, "backward: the training step takes three maps");
  if (!c) return STDA_ERR_INVALID_ARG;
  if (bn_mode != STDA_BN_RUNNING && bn_mode != STDA_BN_BATCH)
    return fail(c, STDA_ERR_INVALID_ARG, "backward: unknown BN mode");
  if (B < 0 || B > c->cfg.max_batch) return fail(c, STDA_ERR_SHAPE, "backward: batch out of range");
  if (!shape_ok(H, W)) return fail(c, STDA_ERR_SHAPE, "backward: H and W must be positive multiples of 8");
  if ((size_t)B * H * W > (size_t)c->cfg.max_batch * c->cfg.H * c->cfg.W)
    return fail(c, STDA_ERR_SHAPE, "backward: B*H*W exceeds the context");
  if (!d_in || !d_gparams || (!d_target && !d_gout))
    return fail(c, STDA_ERR_INVALID_ARG, "backward: null pointer");
  cudaError_t e;
  if (!c->d_train) {
    size_t need = stda::train_workspace_bytes(c->cfg.max_batch, c->cfg.H, c->cfg.W) +
                  (size_t)c->cfg.max_batch * 3 * c->cfg.H * c->cfg.W * sizeof(float) + 256;
    if ((e = cudaMalloc(&c->d_train, need))) return cuda_fail(c, e, "backward: workspace");
    c->train_bytes = need;
  }
  const bool bf = c->cfg.prec != STDA_FP32;
  const float* target = (const float*)d_target;
  if (d_target && bf) {
    if (!c->d_target32 &&
        (e = cudaMalloc((void**)&c->d_target32, sizeof(float) * c->cfg.max_batch * c->cfg.H * c->cfg.W)))
      return cuda_fail(c, e, "backward: target buffer");
    target = c->d_target32;
  }
  stda::TrainArgs a{};
  a.params = c->d_canon;
  a.buffers = c->d_canon + stda::kNumParams;
  a.in = d_in;
  a.in_bf16 = bf;
  a.target = target;
  a.gout = d_target ? nullptr : d_gout;
  a.gparams = d_gparams;
  a.loss = d_target ? d_loss : nullptr;
  a.gin = d_gin;
  a.z_out = d_out;
  a.bn_batch = bn_mode == STDA_BN_BATCH;
  a.bn_stats = d_bn_stats;
  a.B = B;
  a.H = H;
  a.W = W;
  c->last_stream = st;
  if (B == 0) return STDA_OK;
  // the step's ~270 launches (conversion of bf16 targets, taped forward,
  // adjoint, reductions) replay as one CUDA graph from a key's second use
  stda_ctx::GraphKey key{};
  const void* ptrs[9] = {d_in, d_target, d_gout, d_gparams, d_loss, d_gin, d_out, d_bn_stats, c->d_train};
  for (int k = 0; k < 9; ++k) key.p[k] = (uintptr_t)ptrs[k];
  key.i[0] = B;
  key.i[1] = H;
  key.i[2] = W;
  key.i[3] = 2 + (int)bn_mode;  // training step
  return run_cached(c, key, st, "backward", [&](cudaStream_t s, stda::KernelHook*) {
    if (d_target && bf) {
      long n = (long)B * H * W;
      k_bf16_to_f32_flat<<<(int)((n + 255) / 256), 256, 0, s>>>((const __nv_bfloat16*)d_target, c->d_target32, n);
    }
    stda::TrainArgs t = a;
    t.stream = s;
    const cudaError_t te = stda::train_step(t, c->d_train, c->train_bytes);
    return te ? te : cudaGetLastError();
  });
}

stda_status stda_submit(stda_ctx* c, int radar, int H, int W, const void* d_frame, void* d_out, cudaEvent_t done,
                        cudaStream_t st) {
  if (c && c->frames != 3) return fail(c, STDA_ERR_UNSUPPORTED, "submit: serving takes three maps per window");
  if (!c) return STDA_ERR_INVALID_ARG;
  if (!shape_ok(H, W)) return fail(c, STDA_ERR_SHAPE, "submit: H and W must be positive multiples of 8");
  if (!d_frame || !d_out) return fail(c, STDA_ERR_INVALID_ARG, "submit: null pointer");
  if (((uintptr_t)d_frame | (uintptr_t)d_out) & 15) return fail(c, STDA_ERR_INVALID_ARG, "submit: unaligned buffer");
  if (!c->serve) c->serve = stda::serve_new(c->d_status);
  c->last_stream = st;
  cudaError_t e;
  stda_status s = stda::serve_submit(c->serve, c->net, c->tcw, c->cfg.mem_budget_bytes, radar, H, W, d_frame, d_out,
                                     done, st, &e);
  if (e) return cuda_fail(c, e, "submit");
  if (s == STDA_ERR_BUSY) return fail(c, s, "submit: memory budget exhausted");
  if (s == STDA_ERR_SHAPE) return fail(c, s, "submit: radar changed its map size");
  return s;
}

stda_status stda_flush(stda_ctx* c, cudaStream_t st) {
  if (!c) return STDA_ERR_INVALID_ARG;
  if (!c->serve) return STDA_OK;
  c->last_stream = st;
  cudaError_t e = stda::serve_flush(c->serve, c->net, c->tcw, st);
  if (e) return cuda_fail(c, e, "flush");
  return STDA_OK;
}

stda_status stda_serve_close(stda_ctx* c, int radar, cudaStream_t st) {
  if (!c) return STDA_ERR_INVALID_ARG;
  if (!c->serve) return fail(c, STDA_ERR_INVALID_ARG, "serve_close: unknown radar");
  cudaError_t e;
  stda_status s = stda::serve_close(c->serve, c->net, c->tcw, radar, st, &e);
  if (e) return cuda_fail(c, e, "serve_close");
  if (s != STDA_OK) return fail(c, s, "serve_close: unknown radar");
  return s;
}

size_t stda_serve_bytes(stda_ctx* c) { return c && c->serve ? stda::serve_used(c->serve) : 0; }
int stda_serve_radars(stda_ctx* c) { return c && c->serve ? stda::serve_radars(c->serve) : 0; }

stda_status stda_device_status(stda_ctx* c) {
  if (!c) return STDA_ERR_INVALID_ARG;
  int h = 0;
  cudaError_t e = cudaStreamSynchronize(c->last_stream);
  if (!e && c->serve) e = stda::serve_sync(c->serve);
  if (e) return cuda_fail(c, e, "device_status");
  e = cudaMemcpy(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (!e && h != STDA_OK) e = cudaMemset(c->d_status, 0, sizeof(int));
  if (e) return cuda_fail(c, e, "device_status");
  return (stda_status)h;
}

stda_status stda_set_wait_limit(stda_ctx* c, uint32_t polls) {
  if (!c) return STDA_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  drop_graphs(c);
  c->wait_polls = polls;
  return STDA_OK;
}

const char* stda_last_error(stda_ctx* c) { return c ? c->err.c_str() : "null context"; }

stda_status stda_profile(stda_ctx* c, int enable) {
  if (!c) return STDA_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  c->prof.on = enable != 0;
  c->prof.reset();
  return STDA_OK;
}

int stda_profile_read(stda_ctx* c, const char** names, double* total_ms, int* launches, int max) {
  if (!c || max < 0) return -1;
  int n = stda::K_NUM_IDS < max ? stda::K_NUM_IDS : max;
  std::vector<double> t(stda::K_NUM_IDS, 0.0);
  std::vector<int> k(stda::K_NUM_IDS, 0);
  if (!c->prof.recs.empty() && cudaEventSynchronize(c->prof.recs.back().b)) {
    cudaGetLastError();
    return -1;
  }
  for (auto& r : c->prof.recs) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    t[r.id] += ms;
    k[r.id] += 1;
  }
  for (int i = 0; i < n; ++i) {
    if (names) names[i] = stda::kKernelNames[i];
    if (total_ms) total_ms[i] = t[i];
    if (launches) launches[i] = k[i];
  }
  c->prof.reset();
  return n;
}

uint64_t stda_launch_count(stda_ctx* c) { return c ? c->prof.launches : 0; }

stda_status stda_generate(const stda_gen_config* g, uint64_t seed, uint64_t cid, int w0, int B, int bf16,
                          void* d_noisy, void* d_clean, int* d_bins, int* d_ntgt, cudaStream_t st) {
  if (!g || B < 0 || w0 < 0) return STDA_ERR_INVALID_ARG;
  if (B == 0) return STDA_OK;
  if (!d_noisy) return STDA_ERR_INVALID_ARG;
  auto pow2 = [](int v) { return v >= 8 && v <= 1024 && (v & (v - 1)) == 0; };
  if (!pow2(g->P) || !pow2(g->Q) || g->N < 4 || g->M < 2 || g->N > g->P || g->M > g->Q) return STDA_ERR_SHAPE;
  if (g->tmin < 0 || g->tmax < g->tmin || g->tmax > 16 || g->imin < 0 || g->imax < g->imin || g->imax > 4)
    return STDA_ERR_INVALID_ARG;
  cudaError_t e = stda::generate(g, seed, cid, w0, B, bf16, d_noisy, d_clean, d_bins, d_ntgt, st);
  if (e) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? STDA_ERR_OOM : STDA_ERR_CUDA;
  }
  return STDA_OK;
}

stda_status stda_metrics(const void* maps, const void* clean, int bf16, const int* bins, const int* ntgt, int B,
                         int H, int W, int guard, int cfar_guard, int cfar_train, double pfa, double* sinr,
                         double* evm, float* det_rate, unsigned char* det, cudaStream_t st) {
  if (B < 0 || H <= 0 || W <= 0 || guard < 0 || cfar_guard < 0 || cfar_train < 1 || !(pfa > 0.0 && pfa < 1.0))
    return STDA_ERR_INVALID_ARG;
  if (B == 0) return STDA_OK;
  if (!maps || !bins || !ntgt || (evm && !clean)) return STDA_ERR_INVALID_ARG;
  cudaError_t e = stda::metrics(maps, clean, bf16, bins, ntgt, B, H, W, guard, cfar_guard, cfar_train, pfa, sinr,
                                evm, det_rate, det, st);
  if (e) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? STDA_ERR_OOM : STDA_ERR_CUDA;
  }
  return STDA_OK;
}

}  // extern "C"
