// Serving: continuous batching of per-radar frame streams.
//
// Every radar keeps its last three range-Doppler frames in a device ring
// (the online pattern of Sec. IV-B: the window of frame t is t, t-1, t-2).
// A submitted frame is copied into the ring; from the third frame on it
// makes a window, which waits in the pending list of its map size. A flush
// launches, per map size, one batch: a gather kernel assembles the windows
// from the rings, then a CUDA graph (captured once per batch bucket of 1,
// 2, 4, ... windows) runs the forward pass and scatters each output map to
// its request. Each map size has its own stream, so batches of different
// sizes run at the same time; a radar that submits again while its previous
// window is still pending flushes that window's batch first, and the
// caller's stream waits until the gather has read the ring before the next
// frame overwrites the oldest slot. Admission: a new radar is refused
// (STDA_ERR_BUSY) when its ring, plus a new size class's buffers, would
// exceed the context's memory budget; closing a radar frees its ring.
#include <cuda_bf16.h>

#include <map>
#include <vector>

#include "stda_internal.h"
#include "stda_serve.h"
#include "stda_tc.h"

namespace stda {
namespace {

constexpr int kMaxBucket = 64;  // windows per serving batch

struct Req {
  const __nv_bfloat16* f[3];  // frames t, t-1, t-2 in the radar's ring
  __nv_bfloat16* out;
};

// windows i < count: copy the three ring frames; i >= count (bucket
// padding): zeros
__global__ void k_gather(const Req* __restrict__ reqs, const int* __restrict__ count, __nv_bfloat16* in, int n) {
  const int i = blockIdx.y, f = blockIdx.z;
  uint4* dst = (uint4*)(in + ((size_t)i * 3 + f) * n);
  const bool live = i < *count;
  const uint4* src = live ? (const uint4*)reqs[i].f[f] : nullptr;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n / 8; q += gridDim.x * blockDim.x)
    dst[q] = live ? src[q] : make_uint4(0, 0, 0, 0);
}

__global__ void k_scatter(const Req* __restrict__ reqs, const int* __restrict__ count,
                          const __nv_bfloat16* out, int n) {
  const int i = blockIdx.y;
  if (i >= *count) return;
  const uint4* src = (const uint4*)(out + (size_t)i * n);
  uint4* dst = (uint4*)reqs[i].out;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n / 8; q += gridDim.x * blockDim.x) dst[q] = src[q];
}

struct NoHook : KernelHook {
  void begin(int, cudaStream_t) override {}
  void end(cudaStream_t) override {}
};

}  // namespace

struct Radar {
  int H = 0, W = 0;
  __nv_bfloat16* ring = nullptr;  // [3][H][W]
  long count = 0;                 // frames received
  bool pending = false;
};

struct Pending {
  int radar;
  Req req;
  cudaEvent_t done;
};

struct SizeClass {
  int H = 0, W = 0;
  __nv_bfloat16* in = nullptr;   // [kMaxBucket][3][H][W]
  __nv_bfloat16* out = nullptr;  // [kMaxBucket][H][W]
  void* scratch = nullptr;
  FwdScratch s;
  Req* d_reqs = nullptr;  // device request table
  int* d_count = nullptr;
  Req* h_reqs[4] = {};    // pinned staging ring
  int* h_count[4] = {};
  cudaEvent_t staged[4] = {};
  int stage = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t gathered = nullptr, ready = nullptr;
  std::map<int, cudaGraphExec_t> graphs;  // by bucket
  std::vector<Pending> pending;
  size_t bytes = 0;
};

struct Serve {
  std::map<int, Radar> radars;
  std::map<long, SizeClass*> classes;  // key H * 65536 + W
  size_t used = 0;
  int* status = nullptr;
  ~Serve() {
    for (auto& r : radars) cudaFree(r.second.ring);
    for (auto& kv : classes) {
      SizeClass* c = kv.second;
      for (auto& g : c->graphs) cudaGraphExecDestroy(g.second);
      cudaFree(c->in);
      cudaFree(c->out);
      cudaFree(c->scratch);
      cudaFree(c->d_reqs);
      cudaFree(c->d_count);
      for (int k = 0; k < 4; ++k) {
        cudaFreeHost(c->h_reqs[k]);
        cudaFreeHost(c->h_count[k]);
        cudaEventDestroy(c->staged[k]);
      }
      cudaEventDestroy(c->gathered);
      cudaEventDestroy(c->ready);
      cudaStreamDestroy(c->stream);
      delete c;
    }
  }
};

Serve* serve_new(int* status) {
  Serve* s = new Serve;
  s->status = status;
  return s;
}
void serve_delete(Serve* s) { delete s; }

static size_t class_bytes(int H, int W) {
  size_t px = (size_t)H * W;
  return kMaxBucket * px * 4 * sizeof(__nv_bfloat16) + scratch_bytes(kMaxBucket, H, W, 2) +
         sizeof(Req) * kMaxBucket + 256;
}

static cudaError_t class_create(Serve* sv, int H, int W, SizeClass** out) {
  SizeClass* c = new SizeClass;
  c->H = H;
  c->W = W;
  size_t px = (size_t)H * W;
  cudaError_t e;
  if ((e = cudaMalloc((void**)&c->in, kMaxBucket * 3 * px * 2)) || (e = cudaMalloc((void**)&c->out, kMaxBucket * px * 2)) ||
      (e = cudaMalloc(&c->scratch, scratch_bytes(kMaxBucket, H, W, 2))) ||
      (e = cudaMalloc((void**)&c->d_reqs, sizeof(Req) * kMaxBucket)) || (e = cudaMalloc((void**)&c->d_count, sizeof(int))))
    return e;
  for (int k = 0; k < 4; ++k) {
    if ((e = cudaMallocHost((void**)&c->h_reqs[k], sizeof(Req) * kMaxBucket)) ||
        (e = cudaMallocHost((void**)&c->h_count[k], sizeof(int))) ||
        (e = cudaEventCreateWithFlags(&c->staged[k], cudaEventDisableTiming)))
      return e;
  }
  if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) ||
      (e = cudaEventCreateWithFlags(&c->gathered, cudaEventDisableTiming)) ||
      (e = cudaEventCreateWithFlags(&c->ready, cudaEventDisableTiming)))
    return e;
  scratch_carve(c->scratch, kMaxBucket, H, W, 2, &c->s);
  c->bytes = class_bytes(H, W);
  sv->classes[(long)H * 65536 + W] = c;
  *out = c;
  return cudaSuccess;
}

// Forward of `bucket` windows of one class (inside a graph capture).
static cudaError_t class_forward(const NetW& w, const TcWeights& tw, SizeClass* c, int bucket, int* status) {
  NoHook hook;
  int tiles[6];
  cudaError_t e = forward_tc(w, tw, c->in, c->out, bucket, c->H, c->W, c->s, status, c->stream, &hook, tiles);
  if (e) return e;
  e = launch_out_bf16(w, (const __nv_bfloat16*)c->s.act[5], c->s.part[5], tiles[5], c->out, bucket, c->H, c->W,
                      c->stream, &hook);
  if (e) return e;
  int n = c->H * c->W;
  k_scatter<<<dim3(std::max(1, std::min(64, n / 8 / 256)), bucket), 256, 0, c->stream>>>(c->d_reqs, c->d_count,
                                                                                          c->out, n);
  return cudaGetLastError();
}

static cudaError_t class_flush(Serve* sv, const NetW& w, const TcWeights& tw, SizeClass* c, cudaStream_t caller) {
  int B = (int)c->pending.size();
  if (!B) return cudaSuccess;
  int bucket = 1;
  while (bucket < B) bucket <<= 1;
  cudaError_t e;
  // stage the request table (pinned ring; wait until the slot's last copy ran)
  int k = c->stage;
  c->stage = (c->stage + 1) % 4;
  if ((e = cudaEventSynchronize(c->staged[k]))) return e;
  for (int i = 0; i < B; ++i) c->h_reqs[k][i] = c->pending[i].req;
  *c->h_count[k] = B;
  // order after the caller's ring copies
  if ((e = cudaEventRecord(c->ready, caller)) || (e = cudaStreamWaitEvent(c->stream, c->ready, 0))) return e;
  if ((e = cudaMemcpyAsync(c->d_reqs, c->h_reqs[k], sizeof(Req) * B, cudaMemcpyHostToDevice, c->stream)) ||
      (e = cudaMemcpyAsync(c->d_count, c->h_count[k], sizeof(int), cudaMemcpyHostToDevice, c->stream)) ||
      (e = cudaEventRecord(c->staged[k], c->stream)))
    return e;
  int n = c->H * c->W;
  k_gather<<<dim3(std::max(1, std::min(64, n / 8 / 256)), bucket, 3), 256, 0, c->stream>>>(c->d_reqs, c->d_count,
                                                                                           c->in, n);
  if ((e = cudaGetLastError()) || (e = cudaEventRecord(c->gathered, c->stream)) ||
      (e = cudaStreamWaitEvent(caller, c->gathered, 0)))
    return e;
  auto it = c->graphs.find(bucket);
  if (it == c->graphs.end()) {
    cudaGraph_t g;
    if ((e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed))) return e;
    cudaError_t fe = class_forward(w, tw, c, bucket, sv->status);
    e = cudaStreamEndCapture(c->stream, &g);
    if (fe) return fe;
    if (e) return e;
    cudaGraphExec_t ex;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e) return e;
    it = c->graphs.emplace(bucket, ex).first;
  }
  if ((e = cudaGraphLaunch(it->second, c->stream))) return e;
  for (auto& p : c->pending) {
    if (p.done && (e = cudaEventRecord(p.done, c->stream))) return e;
    sv->radars[p.radar].pending = false;
  }
  c->pending.clear();
  return cudaSuccess;
}

cudaError_t serve_flush(Serve* sv, const NetW& w, const TcWeights& tw, cudaStream_t st) {
  for (auto& kv : sv->classes) {
    cudaError_t e = class_flush(sv, w, tw, kv.second, st);
    if (e) return e;
  }
  return cudaSuccess;
}

stda_status serve_submit(Serve* sv, const NetW& w, const TcWeights& tw, size_t budget, int radar, int H, int W,
                         const void* frame, void* out, cudaEvent_t done, cudaStream_t st, cudaError_t* err) {
  *err = cudaSuccess;
  auto rit = sv->radars.find(radar);
  long key = (long)H * 65536 + W;
  auto cit = sv->classes.find(key);
  if (rit == sv->radars.end()) {
    size_t need = (size_t)3 * H * W * sizeof(__nv_bfloat16) + (cit == sv->classes.end() ? class_bytes(H, W) : 0);
    if (budget && sv->used + need > budget) return STDA_ERR_BUSY;
    Radar r;
    r.H = H;
    r.W = W;
    if ((*err = cudaMalloc((void**)&r.ring, (size_t)3 * H * W * sizeof(__nv_bfloat16)))) return STDA_ERR_OOM;
    sv->used += (size_t)3 * H * W * sizeof(__nv_bfloat16);
    rit = sv->radars.emplace(radar, r).first;
  } else if (rit->second.H != H || rit->second.W != W) {
    return STDA_ERR_SHAPE;
  }
  if (cit == sv->classes.end()) {
    SizeClass* c;
    if ((*err = class_create(sv, H, W, &c))) return STDA_ERR_OOM;
    sv->used += c->bytes;
    cit = sv->classes.find(key);
  }
  Radar& r = rit->second;
  SizeClass* c = cit->second;
  // a window of this radar is still pending: launch it before its oldest
  // frame is overwritten
  if (r.pending && (*err = class_flush(sv, w, tw, c, st))) return STDA_ERR_CUDA;
  const size_t fbytes = (size_t)H * W * sizeof(__nv_bfloat16);
  __nv_bfloat16* slot = r.ring + (size_t)(r.count % 3) * H * W;
  if ((*err = cudaMemcpyAsync(slot, frame, fbytes, cudaMemcpyDeviceToDevice, st))) return STDA_ERR_CUDA;
  r.count += 1;
  if (r.count < 3) return STDA_WARMUP;
  Pending p;
  p.radar = radar;
  for (int f = 0; f < 3; ++f) p.req.f[f] = r.ring + (size_t)((r.count - 1 - f) % 3) * H * W;
  p.req.out = (__nv_bfloat16*)out;
  p.done = done;
  c->pending.push_back(p);
  r.pending = true;
  if ((int)c->pending.size() == kMaxBucket && (*err = class_flush(sv, w, tw, c, st))) return STDA_ERR_CUDA;
  return STDA_OK;
}

stda_status serve_close(Serve* sv, const NetW& w, const TcWeights& tw, int radar, cudaStream_t st, cudaError_t* err) {
  *err = cudaSuccess;
  auto it = sv->radars.find(radar);
  if (it == sv->radars.end()) return STDA_ERR_INVALID_ARG;
  if (it->second.pending) {
    SizeClass* c = sv->classes[(long)it->second.H * 65536 + it->second.W];
    if ((*err = class_flush(sv, w, tw, c, st))) return STDA_ERR_CUDA;
  }
  // the ring may still be read by a batch in flight on its class stream
  SizeClass* c = sv->classes[(long)it->second.H * 65536 + it->second.W];
  if ((*err = cudaStreamSynchronize(c->stream))) return STDA_ERR_CUDA;
  cudaFree(it->second.ring);
  sv->used -= (size_t)3 * it->second.H * it->second.W * sizeof(__nv_bfloat16);
  sv->radars.erase(it);
  return STDA_OK;
}

size_t serve_used(const Serve* sv) { return sv->used; }

cudaError_t serve_sync(Serve* sv) {
  for (auto& kv : sv->classes)
    if (cudaError_t e = cudaStreamSynchronize(kv.second->stream)) return e;
  return cudaSuccess;
}
int serve_radars(const Serve* sv) { return (int)sv->radars.size(); }

}  // namespace stda
