// Instantiations and launcher of the tensor-core forward stage.
#include <algorithm>
#include <mutex>

#include "launch.h"
#include "tc_fwd.cuh"

namespace tnrd {

namespace {

int sm_count()
{
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return nsm > 0 ? nsm : 1;
}

// Persistent grid: at most one CTA per SM, and no more CTAs than there are
// tiles for their warpgroups.
template <int KS, int NK, int NB, bool BF, bool X3>
int tc_grid(long long ntiles)
{
    using C = TcCfg<KS, NK, NB, BF, X3>;
    const long long need = (ntiles + C::NWG - 1) / C::NWG;
    return (int)std::max(1LL, std::min((long long)sm_count(), need));
}

template <int KS, int NK, int NB, bool BF, bool X3>
cudaError_t launch_one(const StageArgs& a, int N, cudaStream_t s)
{
    using C = TcCfg<KS, NK, NB, BF, X3>;
    cudaError_t e = cudaFuncSetAttribute(tc_stage_fwd<KS, NK, NB, BF, X3>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int grid = tc_grid<KS, NK, NB, BF, X3>((long long)N * a.tiles_x * a.tiles_y);
    return launch_pdl(tc_stage_fwd<KS, NK, NB, BF, X3>, dim3(grid), dim3(C::NTHREADS), C::SMEM_BYTES,
                      s, a, N);
}

template <int KS, int NK, int NB, bool BF, bool X3>
cudaError_t launch_batch_one(const BatchArgs& a, int t, int ntiles, cudaStream_t s)
{
    using C = TcCfg<KS, NK, NB, BF, X3>;
    cudaError_t e = cudaFuncSetAttribute(tc_batch_fwd<KS, NK, NB, BF, X3>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    tc_batch_fwd<KS, NK, NB, BF, X3><<<tc_grid<KS, NK, NB, BF, X3>(ntiles), C::NTHREADS,
                                       C::SMEM_BYTES, s>>>(a, t);
    return cudaGetLastError();
}

#define TNRD_TC_CASES(X) \
    X(3, 4, 2) X(3, 4, 3) X(5, 24, 2) X(5, 24, 3) X(7, 48, 2) X(7, 48, 3)
// split-operand TF32 (two row blocks: the operand copies leave room for no more)
#define TNRD_TC_X3_CASES(X) X(3, 4, 2) X(5, 24, 2) X(7, 48, 2)

}  // namespace

int tc_tile_h(int ks, int nb) { return 16 * nb - 2 * (ks / 2); }

cudaError_t launch_tc_fwd(int ks, int nk, int nb, int prec, const StageArgs& a, int N,
                          cudaStream_t s)
{
#define X(K, NN, B)                                                                  \
    if (ks == K && nk == NN && nb == B && prec != TC_TF32X3)                         \
        return prec == TC_BF16 ? launch_one<K, NN, B, true, false>(a, N, s)          \
                               : launch_one<K, NN, B, false, false>(a, N, s);
    TNRD_TC_CASES(X)
#undef X
#define X(K, NN, B)                                                                  \
    if (ks == K && nk == NN && nb == B && prec == TC_TF32X3)                         \
        return launch_one<K, NN, B, false, true>(a, N, s);
    TNRD_TC_X3_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_tc_batch(int ks, int nk, int nb, int prec, const BatchArgs& a, int t,
                            int ntiles, cudaStream_t s)
{
#define X(K, NN, B)                                                                     \
    if (ks == K && nk == NN && nb == B && prec != TC_TF32X3)                            \
        return prec == TC_BF16 ? launch_batch_one<K, NN, B, true, false>(a, t, ntiles, s) \
                               : launch_batch_one<K, NN, B, false, false>(a, t, ntiles, s);
    TNRD_TC_CASES(X)
#undef X
#define X(K, NN, B)                                                                     \
    if (ks == K && nk == NN && nb == B && prec == TC_TF32X3)                            \
        return launch_batch_one<K, NN, B, false, true>(a, t, ntiles, s);
    TNRD_TC_X3_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

int* device_status_word()
{
    // Per device: the word's address and the context it was looked up in.  A
    // new context (e.g. after cudaDeviceReset) means a new lookup.
    constexpr int MAXDEV = 64;
    struct Slot {
        unsigned long long ctx;
        int* word;
    };
    static std::mutex mu;
    static Slot slots[MAXDEV] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) {
        (void)cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    const unsigned long long ctx = current_context_id();
    Slot& s = slots[dev];
    if (!s.word || ctx == 0 || ctx != s.ctx) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_tc_error) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            s.word = nullptr;
            return nullptr;
        }
        s.word = static_cast<int*>(p);
        s.ctx = current_context_id();   // the lookup may have made the context current
    }
    return s.word;
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
