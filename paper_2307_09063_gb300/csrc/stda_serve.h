// Serving (continuous batching of per-radar frame streams): internal API.
#pragma once
#include <cuda_runtime.h>

#include "stda_internal.h"
#include "stda_tc.h"

namespace stda {

struct Serve;
Serve* serve_new(int* status);
void serve_delete(Serve* s);
stda_status serve_submit(Serve* sv, const NetW& w, const TcWeights& tw, size_t budget, int radar, int H, int W,
                         const void* frame, void* out, cudaEvent_t done, cudaStream_t st, cudaError_t* err);
cudaError_t serve_flush(Serve* sv, const NetW& w, const TcWeights& tw, cudaStream_t st);
stda_status serve_close(Serve* sv, const NetW& w, const TcWeights& tw, int radar, cudaStream_t st,
                        cudaError_t* err);
size_t serve_used(const Serve* sv);
// Waits for every batch in flight on the size classes' streams.
cudaError_t serve_sync(Serve* sv);
int serve_radars(const Serve* sv);

}  // namespace stda
