// Serving: continuous batching of per-radar frame streams.
//
// Every radar keeps its last three range-Doppler frames in a device ring
// (the online pattern of Sec. IV-B: the window of frame t is t, t-1, t-2).
// A submitted frame is copied into the ring; from the third frame on it
// makes a window, which waits in the pending list of its map size.
//
// A flush launches every pending window of every map size as ONE CUDA graph:
// per size class a branch gathers the windows from the rings, runs the
// forward pass over a fixed batch of up to 64 windows whose actual count the
// kernels read from device memory, and scatters each output map to its
// request. The branches of the different sizes are independent nodes of the
// graph, so their kernels overlap on the device. The graph is captured once
// per set of size classes and replayed for every flush; only the request
// tables (pinned staging ring, copied in stream order before the launch)
// change. An event recorded inside the graph once every gather has read the
// rings orders the caller's next ring copies after it, so frames keep
// arriving while the forward runs. A radar that submits again while its
// previous window is still pending flushes first. Admission: a new radar is
// refused (STDA_ERR_BUSY) when its ring, plus a new size class's buffers,
// would exceed the context's memory budget; closing a radar frees its ring.
#include <cuda_bf16.h>

#include <map>
#include <vector>

#include "stda_internal.h"
#include "stda_serve.h"
#include "stda_tc.h"

namespace stda {
namespace {

constexpr int kMaxBucket = 64;  // windows per size class and flush
constexpr int kStages = 4;      // pinned request-table slots in flight

struct Req {
  const __nv_bfloat16* f[3];  // frames t, t-1, t-2 in the radar's ring
  __nv_bfloat16* out;
};

// windows i < count: copy the three ring frames (the rest of the fixed
// batch is not read by the forward kernels)
__global__ void k_gather(const Req* __restrict__ reqs, const int* __restrict__ count, __nv_bfloat16* in, int n) {
  const int i = blockIdx.y, f = blockIdx.z;
  if (i >= *count) return;
  uint4* dst = (uint4*)(in + ((size_t)i * 3 + f) * n);
  const uint4* src = (const uint4*)reqs[i].f[f];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n / 8; q += gridDim.x * blockDim.x) dst[q] = src[q];
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
  int* d_count = nullptr; // windows of this class in the current flush
  Req* h_reqs[kStages] = {};
  int* h_count[kStages] = {};
  cudaStream_t stream = nullptr;  // the class's branch while a graph is captured
  cudaEvent_t gdone = nullptr, join = nullptr;
  std::vector<Pending> pending;
  size_t bytes = 0;
};

struct Serve {
  std::map<int, Radar> radars;
  std::map<long, SizeClass*> classes;  // key H * 65536 + W
  size_t used = 0;
  int* status = nullptr;
  cudaStream_t s0 = nullptr;  // the flushes' stream: staging copies and graph launches
  cudaEvent_t fork = nullptr, ready = nullptr, gathered = nullptr;
  cudaEvent_t staged[kStages] = {};
  int stage = 0;
  cudaGraphExec_t graph = nullptr;  // one branch per size class
  size_t graph_classes = 0;
  ~Serve();
};

static void class_free(SizeClass* c) {
  if (c->stream) cudaStreamSynchronize(c->stream);
  cudaFree(c->in);
  cudaFree(c->out);
  cudaFree(c->scratch);
  cudaFree(c->d_reqs);
  cudaFree(c->d_count);
  for (int k = 0; k < kStages; ++k) {
    if (c->h_reqs[k]) cudaFreeHost(c->h_reqs[k]);
    if (c->h_count[k]) cudaFreeHost(c->h_count[k]);
  }
  if (c->gdone) cudaEventDestroy(c->gdone);
  if (c->join) cudaEventDestroy(c->join);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

Serve::~Serve() {
  if (s0) cudaStreamSynchronize(s0);
  if (graph) cudaGraphExecDestroy(graph);
  for (auto& r : radars) cudaFree(r.second.ring);
  for (auto& kv : classes) class_free(kv.second);
  for (int k = 0; k < kStages; ++k)
    if (staged[k]) cudaEventDestroy(staged[k]);
  if (fork) cudaEventDestroy(fork);
  if (ready) cudaEventDestroy(ready);
  if (gathered) cudaEventDestroy(gathered);
  if (s0) cudaStreamDestroy(s0);
}

Serve* serve_new(int* status) {
  Serve* s = new Serve;
  s->status = status;
  return s;
}
void serve_delete(Serve* s) { delete s; }

static cudaError_t serve_init(Serve* sv) {
  if (sv->s0) return cudaSuccess;
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&sv->s0, cudaStreamNonBlocking)) ||
      (e = cudaEventCreateWithFlags(&sv->fork, cudaEventDisableTiming)) ||
      (e = cudaEventCreateWithFlags(&sv->ready, cudaEventDisableTiming)) ||
      (e = cudaEventCreateWithFlags(&sv->gathered, cudaEventDisableTiming)))
    return e;
  for (int k = 0; k < kStages; ++k)
    if ((e = cudaEventCreateWithFlags(&sv->staged[k], cudaEventDisableTiming))) return e;
  return cudaSuccess;
}

static size_t class_bytes(int H, int W) {
  size_t px = (size_t)H * W;
  return kMaxBucket * px * 4 * sizeof(__nv_bfloat16) + scratch_bytes(kMaxBucket, H, W, 2) +
         sizeof(Req) * kMaxBucket + 256;
}

static cudaError_t class_alloc(SizeClass* c, int H, int W) {
  c->H = H;
  c->W = W;
  size_t px = (size_t)H * W;
  cudaError_t e;
  if ((e = cudaMalloc((void**)&c->in, kMaxBucket * 3 * px * 2)) || (e = cudaMalloc((void**)&c->out, kMaxBucket * px * 2)) ||
      (e = cudaMalloc(&c->scratch, scratch_bytes(kMaxBucket, H, W, 2))) ||
      (e = cudaMalloc((void**)&c->d_reqs, sizeof(Req) * kMaxBucket)) || (e = cudaMalloc((void**)&c->d_count, sizeof(int))) ||
      (e = cudaMemset(c->d_count, 0, sizeof(int))))
    return e;
  for (int k = 0; k < kStages; ++k) {
    if ((e = cudaMallocHost((void**)&c->h_reqs[k], sizeof(Req) * kMaxBucket)) ||
        (e = cudaMallocHost((void**)&c->h_count[k], sizeof(int))))
      return e;
  }
  if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) ||
      (e = cudaEventCreateWithFlags(&c->gdone, cudaEventDisableTiming)) ||
      (e = cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming)))
    return e;
  scratch_carve(c->scratch, kMaxBucket, H, W, 2, &c->s);
  c->bytes = class_bytes(H, W);
  return cudaSuccess;
}

static cudaError_t class_create(Serve* sv, int H, int W, SizeClass** out) {
  SizeClass* c = new SizeClass;
  const cudaError_t e = class_alloc(c, H, W);
  if (e) {
    cudaGetLastError();
    class_free(c);
    return e;
  }
  sv->classes[(long)H * 65536 + W] = c;
  *out = c;
  return cudaSuccess;
}

// One size class's branch of the flush graph (captured): gather, forward of
// the fixed batch with the window count read on the device, scatter.
static cudaError_t class_branch(const NetW& w, const TcWeights& tw, SizeClass* c, int* status) {
  NoHook hook;
  const int n = c->H * c->W, gx = std::max(1, std::min(64, n / 8 / 256));
  k_gather<<<dim3(gx, kMaxBucket, 3), 256, 0, c->stream>>>(c->d_reqs, c->d_count, c->in, n);
  cudaError_t e = cudaGetLastError();
  if (e || (e = cudaEventRecord(c->gdone, c->stream))) return e;
  int tiles[6];
  e = forward_tc(w, tw, c->in, c->out, kMaxBucket, c->H, c->W, c->s, status, c->stream, &hook, tiles, kWaitPolls,
                 c->d_count);
  if (e) return e;
  e = launch_out_bf16(w, (const __nv_bfloat16*)c->s.act[5], c->s.part[5], tiles[5], c->out, kMaxBucket, c->H, c->W,
                      c->stream, &hook, c->d_count);
  if (e) return e;
  k_scatter<<<dim3(gx, kMaxBucket), 256, 0, c->stream>>>(c->d_reqs, c->d_count, c->out, n);
  if ((e = cudaGetLastError())) return e;
  return cudaEventRecord(c->join, c->stream);
}

// Captures the flush graph: fork from s0 into one branch per size class,
// an event recorded once every gather is done (the caller's ring copies wait
// for it), join back into s0.
static cudaError_t capture_graph(Serve* sv, const NetW& w, const TcWeights& tw) {
  cudaError_t e;
  if (sv->graph) {
    if ((e = cudaStreamSynchronize(sv->s0))) return e;  // the old graph has finished
    cudaGraphExecDestroy(sv->graph);
    sv->graph = nullptr;
  }
  e = cudaStreamBeginCapture(sv->s0, cudaStreamCaptureModeRelaxed);
  if (e) return e;
  cudaError_t fe = cudaEventRecord(sv->fork, sv->s0);
  for (auto& kv : sv->classes) {
    if (fe) break;
    if (!(fe = cudaStreamWaitEvent(kv.second->stream, sv->fork, 0))) fe = class_branch(w, tw, kv.second, sv->status);
  }
  for (auto& kv : sv->classes)
    if (!fe) fe = cudaStreamWaitEvent(sv->s0, kv.second->gdone, 0);
  if (!fe) fe = cudaEventRecordWithFlags(sv->gathered, sv->s0, cudaEventRecordExternal);
  for (auto& kv : sv->classes)
    if (!fe) fe = cudaStreamWaitEvent(sv->s0, kv.second->join, 0);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(sv->s0, &g);
  if (fe || e) {
    if (g) cudaGraphDestroy(g);
    return fe ? fe : e;
  }
  e = cudaGraphInstantiate(&sv->graph, g, 0);
  cudaGraphDestroy(g);
  if (e) return e;
  sv->graph_classes = sv->classes.size();
  return cudaSuccess;
}

// Launches every pending window: the request tables of all size classes
// (empty classes get count 0) are copied on s0 after the caller's ring
// copies, then the flush graph runs; the caller's stream waits only until
// the gathers have read the rings.
cudaError_t serve_flush(Serve* sv, const NetW& w, const TcWeights& tw, cudaStream_t caller) {
  bool any = false;
  for (auto& kv : sv->classes) any = any || !kv.second->pending.empty();
  if (!any) return cudaSuccess;
  cudaError_t e;
  if (!sv->graph || sv->graph_classes != sv->classes.size())
    if ((e = capture_graph(sv, w, tw))) return e;
  const int k = sv->stage;
  sv->stage = (sv->stage + 1) % kStages;
  if ((e = cudaEventSynchronize(sv->staged[k]))) return e;  // slot k's last copies have run
  if ((e = cudaEventRecord(sv->ready, caller)) || (e = cudaStreamWaitEvent(sv->s0, sv->ready, 0))) return e;
  for (auto& kv : sv->classes) {
    SizeClass* c = kv.second;
    const int n = (int)c->pending.size();
    for (int i = 0; i < n; ++i) c->h_reqs[k][i] = c->pending[i].req;
    *c->h_count[k] = n;
    if ((n && (e = cudaMemcpyAsync(c->d_reqs, c->h_reqs[k], sizeof(Req) * n, cudaMemcpyHostToDevice, sv->s0))) ||
        (e = cudaMemcpyAsync(c->d_count, c->h_count[k], sizeof(int), cudaMemcpyHostToDevice, sv->s0)))
      return e;
  }
  if ((e = cudaEventRecord(sv->staged[k], sv->s0)) || (e = cudaGraphLaunch(sv->graph, sv->s0)) ||
      (e = cudaStreamWaitEvent(caller, sv->gathered, 0)))
    return e;
  for (auto& kv : sv->classes) {
    for (auto& p : kv.second->pending) {
      if (p.done && (e = cudaEventRecord(p.done, sv->s0))) return e;
      sv->radars[p.radar].pending = false;
    }
    kv.second->pending.clear();
  }
  return cudaSuccess;
}

stda_status serve_submit(Serve* sv, const NetW& w, const TcWeights& tw, size_t budget, int radar, int H, int W,
                         const void* frame, void* out, cudaEvent_t done, cudaStream_t st, cudaError_t* err) {
  *err = cudaSuccess;
  if ((*err = serve_init(sv))) return STDA_ERR_CUDA;
  auto rit = sv->radars.find(radar);
  long key = (long)H * 65536 + W;
  auto cit = sv->classes.find(key);
  if (rit == sv->radars.end()) {
    size_t need = (size_t)3 * H * W * sizeof(__nv_bfloat16) + (cit == sv->classes.end() ? class_bytes(H, W) : 0);
    if (budget && sv->used + need > budget) return STDA_ERR_BUSY;
  } else if (rit->second.H != H || rit->second.W != W) {
    return STDA_ERR_SHAPE;
  }
  if (cit == sv->classes.end()) {
    SizeClass* c;
    if ((*err = class_create(sv, H, W, &c))) return STDA_ERR_OOM;
    sv->used += c->bytes;
    cit = sv->classes.find(key);
  }
  if (rit == sv->radars.end()) {
    Radar r;
    r.H = H;
    r.W = W;
    if ((*err = cudaMalloc((void**)&r.ring, (size_t)3 * H * W * sizeof(__nv_bfloat16)))) return STDA_ERR_OOM;
    sv->used += (size_t)3 * H * W * sizeof(__nv_bfloat16);
    rit = sv->radars.emplace(radar, r).first;
  }
  Radar& r = rit->second;
  SizeClass* c = cit->second;
  // a window of this radar is still pending: launch it before its oldest
  // frame is overwritten
  if (r.pending && (*err = serve_flush(sv, w, tw, st))) return STDA_ERR_CUDA;
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
  if ((int)c->pending.size() == kMaxBucket && (*err = serve_flush(sv, w, tw, st))) return STDA_ERR_CUDA;
  return STDA_OK;
}

stda_status serve_close(Serve* sv, const NetW& w, const TcWeights& tw, int radar, cudaStream_t st, cudaError_t* err) {
  *err = cudaSuccess;
  auto it = sv->radars.find(radar);
  if (it == sv->radars.end()) return STDA_ERR_INVALID_ARG;
  if (it->second.pending && (*err = serve_flush(sv, w, tw, st))) return STDA_ERR_CUDA;
  // the ring may still be read by a flush in flight
  if (sv->s0 && (*err = cudaStreamSynchronize(sv->s0))) return STDA_ERR_CUDA;
  cudaFree(it->second.ring);
  sv->used -= (size_t)3 * it->second.H * it->second.W * sizeof(__nv_bfloat16);
  sv->radars.erase(it);
  return STDA_OK;
}

size_t serve_used(const Serve* sv) { return sv->used; }
int serve_radars(const Serve* sv) { return (int)sv->radars.size(); }

cudaError_t serve_sync(Serve* sv) { return sv->s0 ? cudaStreamSynchronize(sv->s0) : cudaSuccess; }

}  // namespace stda
