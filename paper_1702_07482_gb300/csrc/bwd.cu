// Instantiations and launchers of the backward stage kernels.
#include "launch.h"
#include "bwd.cuh"

#include <cstdio>
#include <cstdlib>

namespace tnrd {

// bwd_zb and bwd_adj tile heights: TH + 2R is a multiple of ksize, so that
// the walks of interior tiles end on a whole group of steps.
int bwd_tile_h(int ks) { return ks == 3 ? 34 : 36; }

namespace {

// Filter split S of a kernel whose warps walk fpw filters each per tile: S
// CTAs of a tile share them out (a divisor of fpw).  Picks the S of least
// estimated duration, in filter walks: ceil(ctas S / slots) waves of
// fpw / S walks plus a per-CTA overhead (staging the tile, partials) of 0.3
// walk, the value that ranks the measured splits of the 32 x 180^2 training
// step as measured (3 and 3 best for bwd_zb and bwd_dk; none for large batches).
int filter_split(long long tiles, int fpw, long long slots)
{
    int best = 1;
    double best_cost = 1e300;
    for (int sp = 1; sp <= fpw; ++sp) {
        if (fpw % sp) continue;
        const long long waves = (tiles * sp + slots - 1) / slots;
        const double cost = (double)waves * ((double)fpw / sp + 0.3);
        if (cost < best_cost * 0.999) {
            best_cost = cost;
            best = sp;
        }
    }
    return best;
}

int sm_count()
{
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return nsm;
}

template <int KS, int NK, int TH>
cudaError_t launch_stage(const BwdArgs& a, int N, cudaStream_t s, int adj_prec, int* err)
{
    using Z = ZbCfg<KS, NK, TH>;
    using A = AdjCfg<KS, NK, TH>;
    cudaError_t e = cudaFuncSetAttribute(bwd_zb<KS, NK, TH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Z::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(bwd_adj<KS, NK, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)A::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    // resident CTAs per SM of bwd_zb and bwd_dk (for the filter split)
    static const int occ_zb = [] {
        int b = 0;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, bwd_zb<KS, NK, TH>, Z::NTHREADS,
                                                             Z::SMEM_BYTES) == cudaSuccess && b > 0 ? b : 1;
    }();
    static const int occ_dk = [] {
        int b = 0;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, bwd_dk<KS, NK, TH>, 128, 0) ==
                       cudaSuccess && b > 0 ? b : 1;
    }();
    const long long nsm = sm_count();
    const long long zb_tiles = (long long)a.zb_tiles_x * a.zb_tiles_y * N;
    const long long dk_tiles = (long long)a.dk_tiles_x * a.dk_tiles_y * N;
    int zs = filter_split(zb_tiles, Z::FPW, nsm * occ_zb);
    int ds = filter_split(dk_tiles, NK / 4, nsm * occ_dk);
    if (const char* env = std::getenv("TNRD_BWD_SPLIT")) {   // tuning override "zb,dk"
        int z = 0, d = 0;
        if (std::sscanf(env, "%d,%d", &z, &d) == 2 && z >= 1 && d >= 1 && Z::FPW % z == 0 &&
            (NK / 4) % d == 0) {
            zs = z;
            ds = d;
        }
    }
    bwd_zb<KS, NK, TH><<<dim3(a.zb_tiles_x * a.zb_tiles_y, N, zs), Z::NTHREADS, Z::SMEM_BYTES, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (adj_prec >= 0) {
        e = launch_tc_bwd_adj(KS, NK, adj_prec, a, N, err, s);
    } else {
        bwd_adj<KS, NK, TH><<<dim3(a.tiles_x * a.tiles_y, N), A::NTHREADS, A::SMEM_BYTES, s>>>(a);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    // the filter gradient on the tensor cores with TF32 operands; with split TF32
    // the CUDA-core kernel is faster (the doubled operands leave one or two CTAs
    // per SM for a kernel that hides its loads with CTAs)
    if (adj_prec == TC_TF32) return launch_tc_bwd_dk(KS, NK, adj_prec, a, N, err, s);
    bwd_dk<KS, NK, TH><<<dim3(a.dk_tiles_x * a.dk_tiles_y, N, ds), 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_bwd_stage(int ks, int nk, const BwdArgs& a, int N, cudaStream_t s,
                             int adj_prec, int* err)
{
    bwd_prep<<<dim3(a.prep_blocks, N), 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ks == 3 && nk == 4) return launch_stage<3, 4, 34>(a, N, s, adj_prec, err);
    if (ks == 5 && nk == 24) return launch_stage<5, 24, 36>(a, N, s, adj_prec, err);
    if (ks == 7 && nk == 48) return launch_stage<7, 48, 36>(a, N, s, adj_prec, err);
    return cudaErrorInvalidValue;
}

cudaError_t launch_bwd_reduce(const RedArgs& r, cudaStream_t s)
{
    int blocks = 1;
    for (const RedSet& g : r.s) {
        const int b = g.nparam >= 32 ? (g.nparam + 31) / 32 : g.nparam;
        blocks = b > blocks ? b : blocks;
    }
    bwd_reduce<<<dim3(blocks, 3), RED_THREADS, 0, s>>>(r);
    return cudaGetLastError();
}

}  // namespace tnrd
