// Batched forward, one launch per stage, on the column-pair kernel's tiles
// (two z-columns per lane, tiles of 64 - 2R columns, each on a cluster of two
// CTAs with half of the filters): the plan's third schedule, weighed by its
// autotuner against the one-column schedules of batch.cu.  Each tile's bits
// are those of fused_pair2_fwd at the same tile height (uniform tiles).
#include "launch.h"
#include "fused_pair.cuh"

namespace tnrd {

// Stage t of every image's tiles; grid 2 x the plan's tiles.
template <int KS, int NK, int TH>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(PairCfg<KS, NK, TH, 2>::NTHREADS, 2)
batch_pair2_fwd(const __grid_constant__ BatchArgs a, int t)
{
    namespace cg = cooperative_groups;
    using C = PairCfg<KS, NK, TH, 2>;
    extern __shared__ __align__(128) float smem[];
    __shared__ int s_xoff;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int2 ti = a.tile_img[blockIdx.x >> 1];
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
    const int xoff = pair_tile_walk<KS, NK, TH, 2>(j, smem, rank);
    if (threadIdx.x == 0) s_xoff = xoff;
    cl.sync();   // both CTAs' h buffers complete and visible in the cluster
    const float* remote = cl.map_shared_rank(smem, rank ^ 1) + ((C::U_FL + 3) & ~3);
    if (xoff >= 0 && *cl.map_shared_rank(&s_xoff, rank ^ 1) >= 0)
        pair_tile_epilogue<KS, NK, TH, 2>(j, smem, remote, rank * C::NTHREADS + threadIdx.x,
                                          2 * C::NTHREADS, xoff);
    cl.sync();   // keep this CTA's shared memory alive until the other has read it
}

namespace {

template <int KS, int NK, int TH>
cudaError_t launch_pairs_one(const BatchArgs& a, cudaStream_t s)
{
    using C = PairCfg<KS, NK, TH, 2>;
    cudaError_t e = cudaFuncSetAttribute(batch_pair2_fwd<KS, NK, TH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM_BYTES);
    for (int t = 0; t < a.T && e == cudaSuccess; ++t) {
        batch_pair2_fwd<KS, NK, TH><<<2 * a.ntiles, C::NTHREADS, C::SMEM_BYTES, s>>>(a, t);
        e = cudaGetLastError();
    }
    return e;
}

#define TNRD_BPAIR_CASES(X)                                                        \
    X(3, 4, 17) X(3, 4, 23) X(3, 4, 29) X(5, 24, 17) X(5, 24, 22) X(5, 24, 27)    \
    X(5, 24, 32) X(7, 48, 16) X(7, 48, 23) X(7, 48, 30) X(7, 48, 32) X(7, 48, 37)

}  // namespace

cudaError_t launch_batch_pairs(int ks, int nk, int th, const BatchArgs& a, cudaStream_t s)
{
#define X(K, N, T) if (ks == K && nk == N && th == T) return launch_pairs_one<K, N, T>(a, s);
    TNRD_BPAIR_CASES(X)
#undef X
    return cudaErrorInvalidValue;
}

bool pair_fwd_box(int ks, int nk, int th, int* box_w, int* box_h)
{
#define X(K, N, T)                                                                  \
    if (ks == K && nk == N && th == T) {                                            \
        *box_w = PairCfg<K, N, T, 2>::UP;                                           \
        *box_h = PairCfg<K, N, T, 2>::UH;                                           \
        return true;                                                                \
    }
    TNRD_BPAIR_CASES(X)
#undef X
    return false;
}

}  // namespace tnrd
