// Instantiations and launcher of the column-pair fused FP32 forward stage
// (one CTA per tile, or a cluster of two CTAs per tile).
#include "launch.h"
#include "fused_pair.cuh"

namespace tnrd {

namespace {

template <int KS, int NK, int TH>
cudaError_t launch_one(const StageArgs& a, int N, int nsplit, cudaStream_t s)
{
    if (a.th > TH || a.te > a.th || a.te < 0) return cudaErrorInvalidValue;   // buffers hold TH rows
    if (nsplit == 2) {
        using C = PairCfg<KS, NK, TH, 2>;
        cudaError_t e = cudaFuncSetAttribute(fused_pair2_fwd<KS, NK, TH>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        StageArgs b = a;
        stage_args_tma(b, N, C::UP, C::UH);
        e = launch_pdl(fused_pair2_fwd<KS, NK, TH>, dim3(2 * a.tiles_x * a.tiles_y, N),
                       dim3(C::NTHREADS), C::SMEM_BYTES, s, b);
        if (e != cudaSuccess) return e;
    } else {
        using C = PairCfg<KS, NK, TH, 1>;
        cudaError_t e = cudaFuncSetAttribute(fused_pair_fwd<KS, NK, TH>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        StageArgs b = a;
        stage_args_tma(b, N, C::UP, C::UH);
        e = launch_pdl(fused_pair_fwd<KS, NK, TH>, dim3(a.tiles_x * a.tiles_y, N), dim3(C::NTHREADS),
                       C::SMEM_BYTES, s, b);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// Tile heights per filter size (as for the one-column kernel).
#define TNRD_PAIR_CASES(X)                                                         \
    X(3, 4, 17) X(3, 4, 23) X(3, 4, 29) X(5, 24, 17) X(5, 24, 22) X(5, 24, 27)    \
    X(5, 24, 32) X(7, 48, 16) X(7, 48, 23) X(7, 48, 30) X(7, 48, 32) X(7, 48, 37)

}  // namespace

const int* pair_th_list(int ks)
{
    static const int l3[] = {17, 23, 29, 0}, l5[] = {17, 22, 27, 32, 0},
                     l7[] = {16, 23, 30, 32, 37, 0};
    static const int none[] = {0};
    return ks == 3 ? l3 : ks == 5 ? l5 : ks == 7 ? l7 : none;
}

cudaError_t launch_pair_fwd(int ks, int nk, int th, int nsplit, const StageArgs& a, int N,
                            cudaStream_t s)
{
#define X(K, NN, T) if (ks == K && nk == NN && th == T) return launch_one<K, NN, T>(a, N, nsplit, s);
    TNRD_PAIR_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace tnrd
