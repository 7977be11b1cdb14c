// Instantiations and launcher of the column-pair fused FP32 forward stage on
// clusters of four or eight CTAs per tile (small images; see fused_pair.cuh).
#include "launch.h"
#include "fused_pair.cuh"

namespace tnrd {

namespace {

template <int KS, int NK, int TH, int NS>
cudaError_t launch_ns(const StageArgs& a, int N, cudaStream_t s)
{
    if constexpr (NK % NS != 0) {
        return cudaErrorInvalidValue;
    } else {
        using C = PairCfg<KS, NK, TH, NS>;
        if (a.th > TH || a.te > a.th || a.te < 0) return cudaErrorInvalidValue;   // buffers hold TH rows
        cudaError_t e = cudaFuncSetAttribute(fused_pairc_fwd<KS, NK, TH, NS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        StageArgs b = a;
        stage_args_tma(b, N, C::UP, C::UH);
        return launch_pdl(fused_pairc_fwd<KS, NK, TH, NS>, dim3(NS * a.tiles_x * a.tiles_y, N),
                          dim3(C::NTHREADS), C::SMEM_BYTES, s, b);
    }
}

template <int KS, int NK, int TH, int NS>
cudaError_t launch_cascade_ns(const CascadeArgs& c, int N, cudaStream_t s)
{
    if constexpr (NK % NS != 0) {
        return cudaErrorInvalidValue;
    } else {
        using C = PairCfg<KS, NK, TH, NS>;
        if (c.th > TH || c.te > c.th || c.te < 0) return cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(fused_pairc_cascade<KS, NK, TH, NS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        return launch_pdl(fused_pairc_cascade<KS, NK, TH, NS>, dim3(NS * c.tiles_x * c.tiles_y, N),
                          dim3(C::NTHREADS), C::SMEM_BYTES, s, c);
    }
}

// Whether every cluster of the cascade launch can be resident at once.
template <int KS, int NK, int TH, int NS>
bool cascade_fits_ns(long long clusters)
{
    if constexpr (NK % NS != 0) {
        return false;
    } else {
        using C = PairCfg<KS, NK, TH, NS>;
        if (cudaFuncSetAttribute(fused_pairc_cascade<KS, NK, TH, NS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)C::SMEM_BYTES) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(NS * clusters), 1, 1);
        cfg.blockDim = dim3(C::NTHREADS);
        cfg.dynamicSmemBytes = C::SMEM_BYTES;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = NS;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, fused_pairc_cascade<KS, NK, TH, NS>, &cfg) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        return clusters <= (long long)n;
    }
}

// Tile heights compiled for the cluster splits (the small tiles small images need;
// on the 128^2, 5x5x24 image 12-row tiles measured 259.8 Mpixel/s against 212.0
// with 17 rows and 229.0 with 8).
#define TNRD_PAIRC_CASES(X) \
    X(3, 4, 17) X(3, 4, 23) X(5, 24, 12) X(5, 24, 17) X(5, 24, 22) X(7, 48, 12) X(7, 48, 16) \
    X(7, 48, 23)

}  // namespace

const int* pair_cluster_th_list(int ks)
{
    static const int l3[] = {17, 23, 0}, l5[] = {12, 17, 22, 0}, l7[] = {12, 16, 23, 0};
    static const int none[] = {0};
    return ks == 3 ? l3 : ks == 5 ? l5 : ks == 7 ? l7 : none;
}

cudaError_t launch_pair_cascade(int ks, int nk, int th, int nsplit, const CascadeArgs& c, int N,
                                cudaStream_t s)
{
#define X(K, NN, T)                                                          \
    if (ks == K && nk == NN && th == T) {                                    \
        if (nsplit == 4) return launch_cascade_ns<K, NN, T, 4>(c, N, s);     \
        if (nsplit == 8) return launch_cascade_ns<K, NN, T, 8>(c, N, s);     \
    }
    TNRD_PAIRC_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

bool pair_cascade_fits(int ks, int nk, int th, int nsplit, long long clusters)
{
#define X(K, NN, T)                                                          \
    if (ks == K && nk == NN && th == T) {                                    \
        if (nsplit == 4) return cascade_fits_ns<K, NN, T, 4>(clusters);      \
        if (nsplit == 8) return cascade_fits_ns<K, NN, T, 8>(clusters);      \
    }
    TNRD_PAIRC_CASES(X)
#undef X
    return false;
}

cudaError_t launch_pair_cluster_fwd(int ks, int nk, int th, int nsplit, const StageArgs& a, int N,
                                    cudaStream_t s)
{
#define X(K, NN, T)                                                          \
    if (ks == K && nk == NN && th == T) {                                    \
        if (nsplit == 4) return launch_ns<K, NN, T, 4>(a, N, s);             \
        if (nsplit == 8) return launch_ns<K, NN, T, 8>(a, N, s);             \
    }
    TNRD_PAIRC_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace tnrd
