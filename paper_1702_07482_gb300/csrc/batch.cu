// Persistent batched forward: all stages of all images of a plan in one
// launch.  CTAs take (stage, image, tile) items from a stage-major queue.  The
// tile of stage t reads u_{t-1} over its tile plus a 3R/2R halo and writes u_t
// over its own rows/columns, so it must wait until the 3 x 3 neighbouring tiles
// have finished stage t-1: they wrote the halo it reads (read after write) and
// they were the last readers of the buffer it overwrites (write after read).
// Items of stage t-1 precede every item of stage t in the queue and are held
// only by running CTAs, so every wait ends; each wait is also bounded by a
// clock budget, after which the CTA records TNRD_ERR_TIMEOUT, skips its item
// and leaves its tile unfinished (so its dependants give up too).
#include "launch.h"
#include "fused_fwd.cuh"

namespace tnrd {

namespace {

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

}  // namespace

template <int KS, int NK, int TH>
__global__ void __launch_bounds__(FusedCfg<KS, NK, TH>::NTHREADS, FusedCfg<KS, NK, TH>::MINB)
batch_persistent_fwd(const __grid_constant__ BatchArgs a)
{
    extern __shared__ __align__(128) float smem[];
    __shared__ int s_item, s_ok;
    const long long limit = *a.wait_limit;
    const int total = a.ntiles * a.T;
#pragma unroll 1
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.work_counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total) break;
        const int t = item / a.ntiles, gt = item - t * a.ntiles;
        const int2 ti = a.tile_img[gt];
        const BatchImg& im = a.imgs[ti.x];
        const int ty = ti.y / im.tiles_x, tx = ti.y - (ti.y / im.tiles_x) * im.tiles_x;
        if (threadIdx.x == 0) {
            int ok = 1;
            if (t > 0) {
                const long long t0 = clock64();
                for (int dy = -1; dy <= 1 && ok; ++dy) {
                    const int yy = ty + dy;
                    if (yy < 0 || yy >= im.tiles_y) continue;
                    for (int dx = -1; dx <= 1 && ok; ++dx) {
                        const int xx = tx + dx;
                        if (xx < 0 || xx >= im.tiles_x) continue;
                        const int* c = a.tile_done + im.tile_base + yy * im.tiles_x + xx;
                        while (ld_acquire(c) < t) {
                            if (clock64() - t0 > limit) {
                                ok = 0;
                                break;
                            }
                            __nanosleep(100);
                        }
                    }
                }
                if (!ok) atomicExch(a.status, 4 /* TNRD_ERR_TIMEOUT */);
            }
            s_ok = ok;
        }
        __syncthreads();
        if (s_ok) {
            const BatchSet& ps = a.sets[im.set];
            TileJob j;
            // stage t writes u when (T-1-t) is even, so that stage T-1 lands in u
            float* cur = ((a.T - 1 - t) % 2 == 0) ? im.u : im.tmp;
            const float* prev = ((a.T - t) % 2 == 0) ? im.u : im.tmp;
            j.u_in = (t == 0) ? im.f : prev;
            j.u_out = cur;
            j.f = im.f;
            j.H = im.H;
            j.W = im.W;
            j.pitch = im.pitch;
            j.tiles_x = im.tiles_x;
            j.tiles_y = im.tiles_y;
            j.th = TH;
            j.te = 0;
            j.ty = ty;
            j.tx = tx;
            j.k = ps.k + (size_t)t * NK * KS * KS;
            j.w = ps.w + (size_t)t * NK * a.nrbf;
            j.lam = ps.lam + t;
            j.nrbf = a.nrbf;
            j.dterm = ps.dterm;
            j.proj_c = ps.proj_c;
            j.rc = &ps.rc;
            stage_tile<KS, NK, TH>(j, smem);   // ends with a CTA barrier after the stores
            if (threadIdx.x == 0) {
                __threadfence();
                st_release(a.tile_done + im.tile_base + ti.y, t + 1);
            }
        }
        __syncthreads();
    }
}

// The same tiles one stage at a time: stage t of every image's tiles in one
// launch (grid = tiles of all images), the stages ordered by the stream, so no
// tile waits for another.  The plan's autotuner times this schedule against
// the persistent one.
template <int KS, int NK, int TH>
__global__ void __launch_bounds__(FusedCfg<KS, NK, TH>::NTHREADS, FusedCfg<KS, NK, TH>::MINB)
batch_stage_fwd(const __grid_constant__ BatchArgs a, int t)
{
    extern __shared__ __align__(128) float smem[];
    const int2 ti = a.tile_img[blockIdx.x];
    const BatchImg& im = a.imgs[ti.x];
    const BatchSet& ps = a.sets[im.set];
    TileJob j;
    // stage t writes u when (T-1-t) is even, so that stage T-1 lands in u
    const int src = (t == 0) ? 0 : (((a.T - t) % 2 == 0) ? 1 : 2);   // f, u, tmp
    j.u_out = ((a.T - 1 - t) % 2 == 0) ? im.u : im.tmp;
    j.u_in = src == 0 ? im.f : (src == 1 ? im.u : im.tmp);
    j.umap = a.maps ? a.maps + 3 * ti.x + src : nullptr;
    j.img = 0;
    j.err = a.err;
    j.wait_limit = *a.wait_limit;
    j.f = im.f;
    j.H = im.H;
    j.W = im.W;
    j.pitch = im.pitch;
    j.tiles_x = im.tiles_x;
    j.tiles_y = im.tiles_y;
    j.th = TH;
    j.te = 0;
    j.ty = ti.y / im.tiles_x;
    j.tx = ti.y - j.ty * im.tiles_x;
    j.k = ps.k + (size_t)t * NK * KS * KS;
    j.w = ps.w + (size_t)t * NK * a.nrbf;
    j.lam = ps.lam + t;
    j.nrbf = a.nrbf;
    j.dterm = ps.dterm;
    j.proj_c = ps.proj_c;
    j.rc = &ps.rc;
    stage_tile<KS, NK, TH>(j, smem);
}

namespace {

template <int KS, int NK, int TH>
cudaError_t launch_stages_one(const BatchArgs& a, cudaStream_t s)
{
    using C = FusedCfg<KS, NK, TH>;
    const size_t smem = C::smem_bytes(a.nrbf);
    cudaError_t e = cudaFuncSetAttribute(batch_stage_fwd<KS, NK, TH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    for (int t = 0; t < a.T && e == cudaSuccess; ++t) {
        batch_stage_fwd<KS, NK, TH><<<a.ntiles, C::NTHREADS, smem, s>>>(a, t);
        e = cudaGetLastError();
    }
    return e;
}

template <int KS, int NK, int TH>
cudaError_t launch_one(const BatchArgs& a, int grid, cudaStream_t s)
{
    using C = FusedCfg<KS, NK, TH>;
    const size_t smem = C::smem_bytes(a.nrbf);
    cudaError_t e = cudaFuncSetAttribute(batch_persistent_fwd<KS, NK, TH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    batch_persistent_fwd<KS, NK, TH><<<grid, C::NTHREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template <int KS, int NK, int TH>
int occupancy_one(int nrbf)
{
    using C = FusedCfg<KS, NK, TH>;
    const size_t smem = C::smem_bytes(nrbf);
    if (cudaFuncSetAttribute(batch_persistent_fwd<KS, NK, TH>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_persistent_fwd<KS, NK, TH>,
                                                      C::NTHREADS, smem) != cudaSuccess)
        return 0;
    return nb;
}

#define TNRD_BATCH_CASES(X)                                                         \
    X(3, 4, 17) X(3, 4, 23) X(3, 4, 29) X(5, 24, 17) X(5, 24, 22) X(5, 24, 27)     \
    X(5, 24, 32) X(7, 48, 16) X(7, 48, 23) X(7, 48, 30) X(7, 48, 32) X(7, 48, 37)  \
    X(7, 48, 45)

}  // namespace

cudaError_t launch_batch_fwd(int ks, int nk, int th, const BatchArgs& a, int grid, cudaStream_t s)
{
#define X(K, N, T) if (ks == K && nk == N && th == T) return launch_one<K, N, T>(a, grid, s);
    TNRD_BATCH_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_stages(int ks, int nk, int th, const BatchArgs& a, cudaStream_t s)
{
#define X(K, N, T) if (ks == K && nk == N && th == T) return launch_stages_one<K, N, T>(a, s);
    TNRD_BATCH_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

int batch_fwd_occupancy(int ks, int nk, int th, int nrbf)
{
#define X(K, N, T) if (ks == K && nk == N && th == T) return occupancy_one<K, N, T>(nrbf);
    TNRD_BATCH_CASES(X)
#undef X
    return 0;
}

}  // namespace tnrd
