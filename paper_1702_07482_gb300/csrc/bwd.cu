// Instantiations and launchers of the backward stage kernels.
#include "launch.h"
#include "bwd.cuh"

namespace tnrd {

int bwd_tile_h(int ks) { return ks == 3 ? 23 : ks == 5 ? 22 : 30; }

namespace {

template <int KS, int NK, int TH>
cudaError_t launch_bank(const BwdArgs& a, int N, cudaStream_t s)
{
    using C = BwdCfg<KS, NK, TH>;
    cudaError_t e = cudaFuncSetAttribute(bwd_bank<KS, NK, TH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    bwd_bank<KS, NK, TH><<<dim3(a.tiles_x * a.tiles_y, N), C::NTHREADS, C::SMEM_BYTES, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    bwd_dk<KS, NK><<<dim3(a.dk_tiles_x * a.dk_tiles_y, N), 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_bwd_stage(int ks, int nk, const BwdArgs& a, int N, cudaStream_t s)
{
    bwd_prep<<<dim3(a.prep_blocks, N), 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ks == 3 && nk == 4) return launch_bank<3, 4, 23>(a, N, s);
    if (ks == 5 && nk == 24) return launch_bank<5, 24, 22>(a, N, s);
    if (ks == 7 && nk == 48) return launch_bank<7, 48, 30>(a, N, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_bwd_reduce(const float* part, int nrows, int nparam, float* out, cudaStream_t s)
{
    bwd_reduce<<<(nparam + 255) / 256, 256, 0, s>>>(part, nrows, nparam, out);
    return cudaGetLastError();
}

}  // namespace tnrd
