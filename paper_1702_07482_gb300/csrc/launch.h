// Internal interface between the C ABI (api.cu) and the kernel translation
// units.  Every launcher returns the CUDA error of its launch.
#pragma once
#include <cuda_runtime.h>
#include "args.cuh"
#include "tnrd.h"

namespace tnrd {

// Records `msg` for tnrd_last_error() on this host thread and returns s.
tnrd_status set_error(tnrd_status s, const char* msg);

// Launches a forward stage kernel with programmatic stream serialization, so
// that it may start while the previous kernel of the stream finishes (the
// stage kernels wait with griddepcontrol.wait before touching u).
// TNRD_PDL=0 launches plainly (comparison runs).
bool pdl_enabled();
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args)
{
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// Tile heights compiled for the fused forward stage, per filter size (tiles are
// TH x (32 - 2R)); 0 terminates a list.
inline const int* fused_th_list(int ks)
{
    static const int k3[] = {17, 23, 29, 0};
    static const int k5[] = {17, 22, 27, 32, 0};
    static const int k7[] = {16, 23, 30, 32, 37, 45, 0};
    return ks == 3 ? k3 : ks == 5 ? k5 : k7;
}

// Shared memory bytes / threads of one fused-forward CTA, 0 if not built.
size_t fused_fwd_smem(int ks, int nk, int th, int nrbf);
int fused_fwd_threads(int ks, int nk, int th);
// Blocks of the fused forward kernel resident per SM (occupancy query).
int fused_fwd_occupancy(int ks, int nk, int th, int nrbf);

cudaError_t launch_fused_fwd(int ks, int nk, int th, const StageArgs& a, int N, cudaStream_t s);
cudaError_t launch_unfused_fwd(int ks, const UnfArgs& a, int N, cudaStream_t s);

// Tensor-core forward stage: tile height for NB row blocks, launcher, and the
// device error word (read and cleared).
int tc_tile_h(int ks, int nb);
// Operand precision of the tensor-core stage: TF32, BF16, or TF32 with split
// (high + low) operands.
enum TcPrec { TC_TF32 = 0, TC_BF16 = 1, TC_TF32X3 = 2 };
cudaError_t launch_tc_fwd(int ks, int nk, int nb, int prec, const StageArgs& a, int N,
                          cudaStream_t s);
cudaError_t tc_take_error(int* out);
// Address of that word on the current device (null if it cannot be had); the
// fused stages record a tile copy that never landed there too.  Looked up
// again whenever the current context changes (after a device reset the
// module, and with it the word, can sit at another address).
int* device_status_word();
// Unique id of the current CUDA context (cuCtxGetId), 0 if there is none or
// it cannot be read.
unsigned long long current_context_id();

// Bulk-tensor-copy staging of u_{t-1} tiles: TNRD_TMA=0 turns it off (the
// kernels gather instead); a 3-D [N][H][pitch] float32 tensor map with a
// box_w x box_h x 1 box; and StageArgs set-up for a kernel whose staged tile is
// box_w x box_h (falls back to the gather if a map cannot be encoded).
bool tma_staging_enabled();
bool encode_tile_map(CUtensorMap* map, const float* base, int W, int H, int N, int pitch,
                     long long img_stride, int box_w, int box_h);
void stage_args_tma(StageArgs& a, int N, int box_w, int box_h);
// Test hook behind tnrd_stage_wait_test (process-wide), and the wait limit it
// sets (SM cycles per bounded wait of the fused stages).
void set_stage_wait_test(long long cycles, int never_complete);
long long stage_wait_limit();
// Staged tile (columns x rows) of the fused forward kernel of tile height th.
bool fused_fwd_box(int ks, int nk, int th, int* box_w, int* box_h);
// One stage t of a batched plan on the tensor cores (all images' tiles in one launch).
cudaError_t launch_tc_batch(int ks, int nk, int nb, int prec, const BatchArgs& a, int t,
                            int ntiles, cudaStream_t s);

// Column-pair fused forward (two z-columns per lane, TW = 64 - 2R); nsplit 2
// runs each tile on a cluster of two CTAs with half of the filters each.
const int* pair_th_list(int ks);
cudaError_t launch_pair_fwd(int ks, int nk, int th, int nsplit, const StageArgs& a, int N,
                            cudaStream_t s);
// The same kernel on clusters of nsplit = 4 or 8 CTAs per tile (small images),
// compiled for the tile heights of pair_cluster_th_list.
const int* pair_cluster_th_list(int ks);
cudaError_t launch_pair_cluster_fwd(int ks, int nk, int th, int nsplit, const StageArgs& a, int N,
                                    cudaStream_t s);
// All T stages of that kernel in one launch with grid barriers between them,
// and whether all `clusters` clusters of such a launch can be resident at once.
cudaError_t launch_pair_cascade(int ks, int nk, int th, int nsplit, const CascadeArgs& c, int N,
                                cudaStream_t s);
bool pair_cascade_fits(int ks, int nk, int th, int nsplit, long long clusters);

// Persistent batched forward.
cudaError_t launch_batch_fwd(int ks, int nk, int th, const BatchArgs& a, int grid, cudaStream_t s);
int batch_fwd_occupancy(int ks, int nk, int th, int nrbf);
// The same plan one stage per launch (T launches, no waits between tiles).
cudaError_t launch_batch_stages(int ks, int nk, int th, const BatchArgs& a, cudaStream_t s);
// One launch per stage on the column-pair kernel's tiles (two-CTA clusters;
// the plan's tile table in that geometry), and that kernel's staged tile.
cudaError_t launch_batch_pairs(int ks, int nk, int th, const BatchArgs& a, cudaStream_t s);
bool pair_fwd_box(int ks, int nk, int th, int* box_w, int* box_h);

// Backward: tile height of bwd_zb / bwd_adj, one stage's prep + zb + adj +
// filter-gradient launches, and the fixed-order partial reduce (three sets).
int bwd_tile_h(int ks);
// One backward stage (prep, zb, adjoint, dk).  adj_prec < 0: the adjoint and the
// filter gradient on the CUDA cores (bwd_adj, bwd_dk); TC_TF32X3: the adjoint on
// the tensor cores (tc_bwd_adj); TC_TF32: the adjoint and the filter gradient
// (tc_bwd_dk) on the tensor cores.  A tensor-core wait that gave up is recorded
// in the status word err.
cudaError_t launch_bwd_stage(int ks, int nk, const BwdArgs& a, int N, cudaStream_t s,
                             int adj_prec = -1, int* err = nullptr);
cudaError_t launch_tc_bwd_adj(int ks, int nk, int prec, const BwdArgs& a, int N, int* err,
                              cudaStream_t s);
// dL/dk partials on the tensor cores (tc_bwd_dk): one row of part_k per tile of
// 32 x 16 pixels, tc_dk_tiles(H, W) tiles per image.
cudaError_t launch_tc_bwd_dk(int ks, int nk, int prec, const BwdArgs& a, int N, int* err,
                             cudaStream_t s);
int tc_dk_tiles(int H, int W);
cudaError_t launch_bwd_reduce(const RedArgs& r, cudaStream_t s);

// Quality indexes: tiles per image, and the partials + finish launches.
int quality_tiles(int H, int W);
cudaError_t launch_quality(const QualityArgs& a, int N, cudaStream_t s);

}  // namespace tnrd
