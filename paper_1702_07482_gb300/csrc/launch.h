// Internal interface between the C ABI (api.cu) and the kernel translation
// units.  Every launcher returns the CUDA error of its launch.
#pragma once
#include <cuda_runtime.h>
#include "args.cuh"

namespace tnrd {

// Tile heights compiled for the fused forward stage (tiles are TH x 32).
constexpr int kFusedTH[] = {16, 24, 32};
constexpr int kNumFusedTH = 3;

// Shared memory bytes / threads of one fused-forward CTA, 0 if not built.
size_t fused_fwd_smem(int ks, int nk, int th);
int fused_fwd_threads(int ks, int nk, int th);
// Blocks of the fused forward kernel resident per SM (occupancy query).
int fused_fwd_occupancy(int ks, int nk, int th);

cudaError_t launch_fused_fwd(int ks, int nk, int th, const StageArgs& a, int N, cudaStream_t s);
cudaError_t launch_unfused_fwd(int ks, const UnfArgs& a, int N, cudaStream_t s);

}  // namespace tnrd
