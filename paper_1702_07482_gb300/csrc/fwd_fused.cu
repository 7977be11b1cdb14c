// Instantiations and launcher of the fused FP32 forward stage kernel.
#include "launch.h"
#include "fused_fwd.cuh"

namespace tnrd {

namespace {

template <int KS, int NK, int TH>
cudaError_t launch_one(const StageArgs& a, int N, cudaStream_t s)
{
    using C = FusedCfg<KS, NK, TH>;
    if (a.th > TH || a.te > a.th || a.te < 0) return cudaErrorInvalidValue;   // buffers hold TH rows
    const size_t smem = C::smem_bytes(a.nrbf);
    cudaError_t e = cudaFuncSetAttribute(fused_stage_fwd<KS, NK, TH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    StageArgs b = a;
    stage_args_tma(b, N, C::UP, C::UH);
    dim3 grid(a.tiles_x * a.tiles_y, N);
    return launch_pdl(fused_stage_fwd<KS, NK, TH>, grid, dim3(C::NTHREADS), smem, s, b);
}

template <int KS, int NK, int TH>
int occupancy_one(int nrbf)
{
    using C = FusedCfg<KS, NK, TH>;
    const size_t smem = C::smem_bytes(nrbf);
    if (cudaFuncSetAttribute(fused_stage_fwd<KS, NK, TH>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fused_stage_fwd<KS, NK, TH>,
                                                      C::NTHREADS, smem) != cudaSuccess)
        return 0;
    return nb;
}

// Tile heights per filter size.  Most have TH + 4R a multiple of ksize (the
// walk of an interior tile has no partial group of steps); 7x7 also has 32,
// which tiles 512 rows in 16 (a single 512^2 image in one wave), and 45 (the
// largest with two CTAs per SM: four tile rows for 180-row crops).
#define TNRD_FUSED_CASES(X)                                                         \
    X(3, 4, 17) X(3, 4, 23) X(3, 4, 29) X(5, 24, 17) X(5, 24, 22) X(5, 24, 27)     \
    X(5, 24, 32) X(7, 48, 16) X(7, 48, 23) X(7, 48, 30) X(7, 48, 32) X(7, 48, 37)  \
    X(7, 48, 45)

}  // namespace

size_t fused_fwd_smem(int ks, int nk, int th, int nrbf)
{
#define X(K, N, T) if (ks == K && nk == N && th == T) return FusedCfg<K, N, T>::smem_bytes(nrbf);
    TNRD_FUSED_CASES(X)
#undef X
    return 0;
}

bool fused_fwd_box(int ks, int nk, int th, int* box_w, int* box_h)
{
#define X(K, N, T)                                                                  \
    if (ks == K && nk == N && th == T) {                                            \
        *box_w = FusedCfg<K, N, T>::UP;                                             \
        *box_h = FusedCfg<K, N, T>::UH;                                             \
        return true;                                                                \
    }
    TNRD_FUSED_CASES(X)
#undef X
    return false;
}

int fused_fwd_threads(int ks, int nk, int th)
{
#define X(K, N, T) if (ks == K && nk == N && th == T) return FusedCfg<K, N, T>::NTHREADS;
    TNRD_FUSED_CASES(X)
#undef X
    return 0;
}

int fused_fwd_occupancy(int ks, int nk, int th, int nrbf)
{
#define X(K, N, T) if (ks == K && nk == N && th == T) return occupancy_one<K, N, T>(nrbf);
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
