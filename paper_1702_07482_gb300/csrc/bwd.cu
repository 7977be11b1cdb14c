// Instantiations and launchers of the backward stage kernels.
#include "launch.h"
#include "bwd.cuh"

namespace tnrd {

// bwd_zb and bwd_adj tile heights: TH + 2R is a multiple of ksize, so that
// the walks of interior tiles end on a whole group of steps.
int bwd_tile_h(int ks) { return ks == 3 ? 34 : 36; }

namespace {

template <int KS, int NK, int TH>
cudaError_t launch_stage(const BwdArgs& a, int N, cudaStream_t s)
{
    using Z = ZbCfg<KS, NK, TH>;
    using A = AdjCfg<KS, NK, TH>;
    cudaError_t e = cudaFuncSetAttribute(bwd_zb<KS, NK, TH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Z::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(bwd_adj<KS, NK, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)A::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    bwd_zb<KS, NK, TH><<<dim3(a.zb_tiles_x * a.zb_tiles_y, N), Z::NTHREADS, Z::SMEM_BYTES, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bwd_adj<KS, NK, TH><<<dim3(a.tiles_x * a.tiles_y, N), A::NTHREADS, A::SMEM_BYTES, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bwd_dk<KS, NK, TH><<<dim3(a.dk_tiles_x * a.dk_tiles_y, N), 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_bwd_stage(int ks, int nk, const BwdArgs& a, int N, cudaStream_t s)
{
    bwd_prep<<<dim3(a.prep_blocks, N), 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ks == 3 && nk == 4) return launch_stage<3, 4, 34>(a, N, s);
    if (ks == 5 && nk == 24) return launch_stage<5, 24, 36>(a, N, s);
    if (ks == 7 && nk == 48) return launch_stage<7, 48, 36>(a, N, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_bwd_reduce(const RedArgs& r, cudaStream_t s)
{
    int blocks = 1;
    for (const RedSet& g : r.s) {
        const int b = g.nparam >= 32 ? (g.nparam + 31) / 32 : g.nparam;
        blocks = b > blocks ? b : blocks;
    }
    bwd_reduce<<<dim3(blocks, 3), RED_THREADS, 0, s>>>(r);
    return cudaGetLastError();
}

}  // namespace tnrd
