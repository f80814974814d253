// Tensor-core forward path: shared declarations (host and device).
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include <vector>

#include "stda_internal.h"

namespace stda {

// One K-step (K = 16 bf16) of an implicit-GEMM accumulator: the two 8-wide
// K halves read plane pl0 / pl1 of the staged activations at pixel offset
// (dr, dc) from the GEMM row's own pixel.
struct KStep {
  int8_t pl0, dr0, dc0, pl1, dr1, dc1, pad0, pad1;
};

// Packed stage-2 weights of one block in the MMA's K-major core-matrix
// order, [accumulator phase][K-step][K half][N padded][8] bf16, and the
// K-step table ([phase][K-step]).
struct TcLayer {
  const unsigned char* wm;
  const unsigned char* wr;
  const KStep* ks;
  const float* swm;  // E4M3 per-output-channel weight scales (main, residual)
  const float* swr;
  bool f8;           // E4M3 operands (kind::f8f6f4) instead of bf16
  int terms;         // E4M3 terms per operand: 1, or 2 (high + rounding remainder)
  int nsteps;        // K-steps per accumulator
};
struct TcWeights {
  const unsigned char* stem;
  TcLayer layer[6];
};

constexpr int kTcMaxSmem = 227 * 1024;
constexpr int kTcHalfSmem = 113 * 1024;  // two CTAs per SM

struct TcArgs {
  const __nv_bfloat16* in;  // block 1: raw frames [B][3][H][W]; else previous block [B][h][w][CI]
  const float* ppart;
  const float* pk3;
  int ptiles;
  const __nv_bfloat16* skip;  // decoder skip operand [B][h][w][CI] (pre-ECA) or null
  const float* spart;
  const float* sk3;
  int stiles;
  int h, w;       // input map of this block
  int band;       // encoder: output rows per CTA; decoder: input rows per CTA
  int ntile;      // 128-row GEMM tiles per CTA
  int WP, PIXA;   // plane pitch and pixels per plane
  int tiles_per_window;
  int nwin;  // windows in the batch (items = windows x bands)
  int nbuf;   // TMEM buffers that run tiles (1 .. 4), one MMA issuer each
  int nslot;  // TMEM accumulator slots per buffer (2: next tile queued before the drain)
  int gpb;    // warp groups per TMEM buffer (2: the drain is split between them)
  int nsteps;
  uint32_t tmem_cols;
  const float *stem_w, *stem_b, *dw, *dwb, *b2, *rb;
  TcLayer L;
  __nv_bfloat16* out;
  float* part;
  int* status;
  uint32_t wait_polls;  // polls of the tile barrier before a drain wait gives up
  // encoder block 1 (stem on the tensor cores): stem GEMM tiles per item,
  // pixel-pair plane stride, TMA boxes per input row and their width
  // (elements), staged raw bytes per item, packed stem weights
  int ntile_s, PS, nbox, BW, raw_bytes;
  const unsigned char* stem_pk;
  const int* d_nwin;  // windows to process, read on the device (<= nwin), or null for nwin
};

// Host: packs the folded FP32 weights of every block for the tensor cores.
// Returns byte offsets (into one device buffer) of each block's tensors.
struct TcPackOffsets {
  size_t stem;  // stem weights as tcgen05 B operand: [dy 3][K half 2][N 16][8] bf16
  size_t wm[6], wr[6], ks[6], swm[6], swr[6];
  bool f8[6];
  int terms[6];
  int nsteps[6];
  size_t total;
};
// f8[b]: block b's stage-2 operands in E4M3 (needs 16 or more input
// channels), with f8_terms (1 or 2) E4M3 terms per operand.
void pack_tc(const float* folded, const FoldedOffsets& off, int frames, const bool* f8, int f8_terms,
             std::vector<unsigned char>* blob, TcPackOffsets* po);
TcWeights tc_weights_from(const unsigned char* dev_base, const TcPackOffsets& po);

// Default bound of the device-side waits for a tile's MMAs (mbarrier polls,
// each of which may itself suspend briefly): far above any tile's latency.
constexpr uint32_t kWaitPolls = 1u << 22;

// Forward of the six blocks on the tensor cores (output conv excluded);
// tiles_out receives the ECA partial-sum tiles per window of each block.
// wait_polls bounds the epilogue's wait for each tile (0: give up at once,
// which only tests of the timeout path use); on a timeout the kernel still
// waits, with the default bound, for the MMAs it issued before it frees its
// tensor memory, and sets *status to STDA_ERR_TIMEOUT. With d_nwin the
// kernels read the number of windows (at most B) from device memory when
// they start, so a captured graph serves any batch up to B.
cudaError_t forward_tc(const NetW& w, const TcWeights& tw, const __nv_bfloat16* in, __nv_bfloat16* out, int B,
                       int H, int W, const FwdScratch& s, int* status, cudaStream_t st, KernelHook* hook,
                       int* tiles_out, uint32_t wait_polls = kWaitPolls, const int* d_nwin = nullptr);

// Output conv (CUDA cores) over the decoder-3 map, bf16 I/O (windows
// beyond *d_nwin skipped when d_nwin is given).
cudaError_t launch_out_bf16(const NetW& w, const __nv_bfloat16* d3, const float* part5, int tiles5,
                            __nv_bfloat16* out, int B, int H, int W, cudaStream_t st, KernelHook* hook,
                            const int* d_nwin = nullptr);

}  // namespace stda
