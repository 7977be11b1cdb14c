// Instantiations and launcher of the tensor-core forward stage.
#include <atomic>

#include "launch.h"
#include "tc_fwd.cuh"

namespace tnrd {

namespace {

template <int KS, int NK, int NB, bool BF>
cudaError_t launch_one(const StageArgs& a, int N, cudaStream_t s)
{
    using C = TcCfg<KS, NK, NB, BF>;
    cudaError_t e = cudaFuncSetAttribute(tc_stage_fwd<KS, NK, NB, BF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    tc_stage_fwd<KS, NK, NB, BF><<<dim3(a.tiles_x * a.tiles_y, N), C::NTHREADS, C::SMEM_BYTES, s>>>(a);
    return cudaGetLastError();
}

template <int KS, int NK, int NB, bool BF>
cudaError_t launch_batch_one(const BatchArgs& a, int t, int ntiles, cudaStream_t s)
{
    using C = TcCfg<KS, NK, NB, BF>;
    cudaError_t e = cudaFuncSetAttribute(tc_batch_fwd<KS, NK, NB, BF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    tc_batch_fwd<KS, NK, NB, BF><<<ntiles, C::NTHREADS, C::SMEM_BYTES, s>>>(a, t);
    return cudaGetLastError();
}

#define TNRD_TC_CASES(X) \
    X(3, 4, 2) X(3, 4, 3) X(5, 24, 2) X(5, 24, 3) X(7, 48, 2) X(7, 48, 3)

}  // namespace

int tc_tile_h(int ks, int nb) { return 16 * nb - 2 * (ks / 2); }

cudaError_t launch_tc_fwd(int ks, int nk, int nb, bool bf16, const StageArgs& a, int N,
                          cudaStream_t s)
{
#define X(K, NN, B)                                                                  \
    if (ks == K && nk == NN && nb == B)                                              \
        return bf16 ? launch_one<K, NN, B, true>(a, N, s) : launch_one<K, NN, B, false>(a, N, s);
    TNRD_TC_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_tc_batch(int ks, int nk, int nb, bool bf16, const BatchArgs& a, int t,
                            int ntiles, cudaStream_t s)
{
#define X(K, NN, B)                                                                     \
    if (ks == K && nk == NN && nb == B)                                                 \
        return bf16 ? launch_batch_one<K, NN, B, true>(a, t, ntiles, s)                 \
                    : launch_batch_one<K, NN, B, false>(a, t, ntiles, s);
    TNRD_TC_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

int* device_status_word()
{
    constexpr int MAXDEV = 64;
    static std::atomic<int*> words[MAXDEV] = {};   // per device, filled on first use
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) return nullptr;
    int* w = words[dev].load(std::memory_order_acquire);
    if (!w) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_tc_error) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        w = static_cast<int*>(p);
        words[dev].store(w, std::memory_order_release);   // every thread stores the same address
    }
    return w;
}

cudaError_t tc_take_error(int* out)
{
    int v = 0, zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_tc_error, sizeof v);
    if (e == cudaSuccess && v != 0) e = cudaMemcpyToSymbol(g_tc_error, &zero, sizeof zero);
    *out = v;
    return e;
}

}  // namespace tnrd
