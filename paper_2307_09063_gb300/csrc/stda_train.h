// Training step (forward with tape + adjoint) on the GPU: internal API.
#pragma once
#include <cuda_runtime.h>

#include "stda_internal.h"

namespace stda {

struct TrainArgs {
  const float* params;   // canonical parameters [137915] (device)
  const float* buffers;  // BN running statistics [1360] (device)
  const void* in;        // [B][3][H][W], float or bf16
  bool in_bf16;
  const float* target;   // [B][H][W] clean maps (MSE), or null
  const float* gout;     // [B][H][W] dL/dz when target is null
  float* gparams;        // [137915] dL/dtheta (FP64-accumulated), or null
  double* gparams_f64;   // the same in FP64, or null
  double* loss;          // MSE (target mode), or null
  float* gin;            // [B][3][H][W] dL/dx, or null
  float* z_out;          // [B][H][W] forward output of the training graph, or null
  bool bn_batch;         // BN in training mode: normalise with the batch's statistics
  float* bn_stats;       // [1360] the statistics each BN used (BN-buffer layout), or null
  int B, H, W;
  cudaStream_t stream;
};

// Workspace of one training step for B windows of H x W (without gin).
size_t train_workspace_bytes(int B, int H, int W);
size_t train_step_plan(const TrainArgs& a, void* arena);
cudaError_t train_step(const TrainArgs& a, void* workspace, size_t bytes);

}  // namespace stda
