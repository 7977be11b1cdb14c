// Instantiations and launcher of the fused FP32 forward stage kernel.
#include "launch.h"
#include "fused_fwd.cuh"

namespace tnrd {

namespace {

template <int KS, int NK, int TH>
cudaError_t launch_one(const StageArgs& a, int N, cudaStream_t s)
{
    using C = FusedCfg<KS, NK, TH>;
    cudaError_t e = cudaFuncSetAttribute(fused_stage_fwd<KS, NK, TH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    dim3 grid(a.tiles_x * a.tiles_y, N);
    fused_stage_fwd<KS, NK, TH><<<grid, C::NTHREADS, C::SMEM_BYTES, s>>>(a);
    return cudaGetLastError();
}

template <int KS, int NK, int TH>
int occupancy_one()
{
    using C = FusedCfg<KS, NK, TH>;
    if (cudaFuncSetAttribute(fused_stage_fwd<KS, NK, TH>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)C::SMEM_BYTES) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fused_stage_fwd<KS, NK, TH>,
                                                      C::NTHREADS, C::SMEM_BYTES) != cudaSuccess)
        return 0;
    return nb;
}

#define TNRD_FUSED_CASES(X)                                                         \
    X(3, 4, 16) X(3, 4, 24) X(3, 4, 32) X(5, 24, 16) X(5, 24, 24) X(5, 24, 32)     \
    X(7, 48, 16) X(7, 48, 24) X(7, 48, 32)

}  // namespace

size_t fused_fwd_smem(int ks, int nk, int th)
{
#define X(K, N, T) if (ks == K && nk == N && th == T) return FusedCfg<K, N, T>::SMEM_BYTES;
    TNRD_FUSED_CASES(X)
#undef X
    return 0;
}

int fused_fwd_threads(int ks, int nk, int th)
{
#define X(K, N, T) if (ks == K && nk == N && th == T) return FusedCfg<K, N, T>::NTHREADS;
    TNRD_FUSED_CASES(X)
#undef X
    return 0;
}

int fused_fwd_occupancy(int ks, int nk, int th)
{
#define X(K, N, T) if (ks == K && nk == N && th == T) return occupancy_one<K, N, T>();
    TNRD_FUSED_CASES(X)
#undef X
    return 0;
}

cudaError_t launch_fused_fwd(int ks, int nk, int th, const StageArgs& a, int N, cudaStream_t s)
{
#define X(K, NN, T) if (ks == K && nk == NN && th == T) return launch_one<K, NN, T>(a, N, s);
    TNRD_FUSED_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace tnrd
