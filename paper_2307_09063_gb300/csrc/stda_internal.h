// Internal declarations of libstda (not part of the C-ABI).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/stda.h"

namespace stda {

// Network shape (Sec. IV; widths are the canonical reading: stem 3 -> 8,
// encoder 8 -> 16 -> 32 -> 64, decoder 64 -> 32 -> 16 -> 8).
constexpr int kNumBlocks = 6;
constexpr int kBlkEnc[6] = {1, 1, 1, 0, 0, 0};
constexpr int kBlkCin[6] = {8, 16, 32, 64, 32, 16};
constexpr int kBlkCout[6] = {16, 32, 64, 32, 16, 8};
constexpr int kNumParams = 137915;
constexpr int kNumBuffers = 1360;

// Folded weights of one block (BN folded into the convolutions, FP32).
//  dw [9][Cin]   stage-1: the three branches of Eqs. mobile_*_stage1 as one
//                depthwise 3x3 cross-correlation (tap = (dy+1)*3 + (dx+1)),
//  dwb[Cin]      its bias (sum of the three BN shifts),
//  w2            stage-2 main branch, scaled by its BN:
//                  encoder [9 taps][Cin][Cout]
//                  decoder [4 phases][4 sub-taps][Cin][Cout] (sub-pixel form
//                  of the stride-2 4x4 transposed convolution),
//  b2 [Cout]     its BN shift,
//  rw, rb        residual branch weight (same layout as w2) and bias,
//  eca[3]        the ECA 1-D kernel.
struct BlockW {
  const float *dw, *dwb, *w2, *b2, *rw, *rb, *eca;
};

constexpr int kMaxFrames = 4;  // stacked maps per window (3 in the paper)

struct NetW {
  int frames;           // stacked input maps = stem input channels
  const float* stem_w;  // [frames * 9 = ci*9 + tap][8]
  const float* stem_b;  // [8]
  BlockW blk[6];
  const float* out_w;  // [9 taps][8]
  const float* out_b;  // [1]
};

// Host-side folding of the canonical parameters (FP64 arithmetic).
// Returns the flat folded buffer and fills offsets into it.
struct FoldedOffsets {
  size_t stem_w, stem_b, out_w, out_b;
  size_t dw[6], dwb[6], w2[6], b2[6], rw[6], rb[6], eca[6];
  size_t total;
};
void fold_params(const float* params, const float* buffers, float* dst,
                 FoldedOffsets* off, int frames = 3);
FoldedOffsets folded_layout(int frames = 3);
NetW net_from(const float* dev_base, const FoldedOffsets& off, int frames = 3);

// Parameter initialisation from a seed (SplitMix64 uniform draws).
size_t num_params(int frames);
void init_params(uint64_t seed, float* params, float* buffers, int frames = 3);

// Activation scratch of one forward pass for B windows of H x W.
struct FwdScratch {
  void* act[6];   // block pre-activations (before ECA), NHWC
  float* part[6]; // per-tile channel sums of each block output [B][tiles][C]
  int tiles[6];   // tiles per window of each block's producing kernel
};

// Optional per-kernel CUDA-event timing and launch counting; every kernel
// launch of the library is bracketed by begin(id) / end().
enum KernelId { K_ENC1 = 0, K_ENC2, K_ENC3, K_DEC1, K_DEC2, K_DEC3, K_OUT, K_NUM_IDS };
extern const char* const kKernelNames[K_NUM_IDS];
struct KernelHook {
  virtual void begin(int id, cudaStream_t st) = 0;
  virtual void end(cudaStream_t st) = 0;
  virtual ~KernelHook() {}
};

// Forward pass on the CUDA cores (FP32 arithmetic and storage; T = float,
// the STDA_FP32 path). Returns cudaSuccess or the launch error.
template <typename T>
cudaError_t forward_simt(const NetW& w, const T* in, T* out, int B, int H,
                         int W, const FwdScratch& s, cudaStream_t st,
                         KernelHook* hook);
size_t scratch_bytes(int B, int H, int W, size_t elem);
void scratch_carve(void* base, int B, int H, int W, size_t elem,
                   FwdScratch* s);

// Evaluation of denoised maps (SINR, EVM, CA-CFAR).
cudaError_t metrics(const void* maps, const void* clean, int bf16, const int* bins, const int* ntgt, int B, int H,
                    int W, int guard, int cfar_guard, int cfar_train, double pfa, double* sinr, double* evm,
                    float* det_rate, unsigned char* det, cudaStream_t st);

// Generator.
cudaError_t generate(const stda_gen_config* g, uint64_t seed, uint64_t cid,
                     int w0, int B, int bf16, void* noisy, void* clean,
                     int* bins, int* ntgt, cudaStream_t st);

}  // namespace stda
