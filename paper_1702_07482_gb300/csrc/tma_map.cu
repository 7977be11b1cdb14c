// Host side of the bulk tensor copies that stage u_{t-1} tiles: tensor-map
// encoding (through the driver entry point the runtime hands out, so the
// library needs no link against the driver library) and the device status
// word the kernels report a copy that never landed to.
#include <cudaTypedefs.h>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include "launch.h"

namespace tnrd {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            (void)cudaGetLastError();
    });
    return fn;
}

template <class F>
F driver_fn(const char* name, int version)
{
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, version, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        return reinterpret_cast<F>(p);
    (void)cudaGetLastError();
    return nullptr;
}

}  // namespace

unsigned long long current_context_id()
{
    static std::once_flag once;
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    std::call_once(once, [] {
        get_current = driver_fn<PFN_cuCtxGetCurrent_v4000>("cuCtxGetCurrent", 4000);
        get_id = driver_fn<PFN_cuCtxGetId_v12000>("cuCtxGetId", 12000);
    });
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

bool pdl_enabled()
{
    const char* env = std::getenv("TNRD_PDL");   // "0": plain launches (comparison runs)
    return !(env && std::strcmp(env, "0") == 0);
}

bool tma_staging_enabled()
{
    const char* env = std::getenv("TNRD_TMA");   // "0": symmetric gather instead (comparison runs)
    return !(env && std::strcmp(env, "0") == 0);
}

bool encode_tile_map(CUtensorMap* map, const float* base, int W, int H, int N, int pitch,
                     long long img_stride, int box_w, int box_h)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn || !base || W < 1 || H < 1 || N < 1 || pitch < W || (pitch & 3) ||
        ((uintptr_t)base & 15) || box_w < 4 || box_w > 256 || (box_w & 3) || box_h < 1 ||
        box_h > 256 || img_stride < (long long)H * pitch || (img_stride & 3))
        return false;
    const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * sizeof(float),
                                   (cuuint64_t)img_stride * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    std::memset(map, 0, sizeof *map);
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {
std::atomic<long long> g_wait_limit{1ll << 31};
std::atomic<int> g_tx_extra{0};
}  // namespace

void set_stage_wait_test(long long cycles, int never_complete)
{
    g_wait_limit.store(cycles);
    g_tx_extra.store(never_complete ? 16 : 0);
}

long long stage_wait_limit() { return g_wait_limit.load(); }

void stage_args_tma(StageArgs& a, int N, int box_w, int box_h)
{
    a.wait_limit = g_wait_limit.load();
    a.tx_extra = g_tx_extra.load();
    a.err = device_status_word();
    a.use_tma = a.err != nullptr && tma_staging_enabled() &&
                encode_tile_map(&a.umap, a.u_in, a.W, a.H, N, a.pitch, a.img_stride, box_w, box_h);
}

}  // namespace tnrd
