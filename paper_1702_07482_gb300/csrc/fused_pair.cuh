// Fused FP32 forward stage of TRDMD (Eq. diffusionprocessfinal), column-pair
// variant: u_t = prox(u_{t-1} - sum_i K_i^T phi_i(K_i u_{t-1})) in one kernel
// per stage, with the filter responses kept in registers and only u_t
// written to HBM (as fused_stage_fwd).
//
// Lane j owns the two z-columns c0 = x0 - R + 2j and c1 = c0 + 1, so a warp
// covers 64 z-columns and the tile TW = 64 - 2R output columns.  Against one
// column per lane this
//   * reads the 2R + 2 u values of both columns as R + 1 float2 loads,
//   * gathers the 2R + 2 neighbouring v values with 2R shuffles,
//   * accumulates h as float2 rows,
//   * and spends 2R of every 64 z-columns on the halo instead of 2R of 32.
// Each warp walks down its columns once per filter (rolling z and h
// accumulators as in fused_stage_fwd) and keeps h in a private buffer; the
// epilogue sums the buffers, folds the border (exact transpose of the
// symmetric-padded convolution) and applies the prox.
//
// NSPLIT = 2 runs one tile on a cluster of two CTAs, each with half of the
// filters; the epilogue of each CTA covers half of the tile and adds the
// other CTA's h buffers through distributed shared memory.  This doubles the
// CTAs of small images (one 512 x 512 image is ~150 tiles for 152 SMs).
// NSPLIT = 4 or 8 (fused_pairc_fwd) spreads one tile over a cluster of four or
// eight CTAs in the same way, for images too small to give every SM a CTA
// otherwise; each CTA's epilogue adds all ranks' h buffers in rank order.
#pragma once
#include <cooperative_groups.h>
#include "args.cuh"
#include "fused_fwd.cuh"   // shfl_rel

namespace tnrd {

template <int KS, int NK, int TH, int NSPLIT>
struct PairCfg {
    static constexpr int R = KS / 2;
    static constexpr int TW = 64 - 2 * R;          // output columns per tile
    static constexpr int NK_CTA = NK / NSPLIT;
    static_assert(NK % NSPLIT == 0, "filters must split evenly over the cluster");
    static constexpr int NWARP = pair_nwarp(NK_CTA);
    static constexpr int NTHREADS = NWARP * 32;
    static constexpr int FPW = NK_CTA / NWARP;
    static constexpr int GROUPS_EXT = (TH + 6 * R + KS - 1) / KS;
    static constexpr int GROUPS_INT = (TH + 4 * R + KS - 1) / KS;
    static constexpr int UH_EXT = GROUPS_EXT * KS;
    static constexpr int UH_INT = R + GROUPS_INT * KS;
    static constexpr int UH = UH_EXT > UH_INT ? UH_EXT : UH_INT;   // u rows from y0 - 3R
    static constexpr int UW = 64 + 2 * R;          // u cols from x0 - 2R
    static constexpr int UP = staged_pitch(UW);    // staged row pitch (16-byte aligned box)
    static constexpr int U_FL = UH * UP;
    static constexpr int H_FL = (TH + 2 * R) * 64; // h rows from y0 - R, two columns per lane
    static constexpr int KPAD = (KS * KS + 3) & ~3;
    static constexpr int WPADN = (MAX_NRBF + 2 * RBF_WPAD + 3) & ~3;
    static constexpr int PW_FL = H_FL + KPAD + WPADN;
    static constexpr int SMEM_FL = ((U_FL + 3) & ~3) + NWARP * PW_FL;
    static constexpr size_t SMEM_BYTES = sizeof(float) * (size_t)SMEM_FL;
};

// vw[t] = v at column c0 - R + t (t = 0 .. 2R+1) from the (v0, v1) pairs of
// lanes j + floor((t - R) / 2).
template <int KS, int T, bool EDGE>
__device__ __forceinline__ void gather_pair(float (&vw)[KS + 1], float v0, float v1, int lane)
{
    if constexpr (T < KS + 1) {
        constexpr int R = KS / 2;
        constexpr int d = T - R;
        constexpr int D = d >= 0 ? d / 2 : -((1 - d) / 2);
        constexpr int E = d - 2 * D;
        vw[T] = shfl_rel<D, EDGE>(E ? v1 : v0, lane);
        gather_pair<KS, T + 1, EDGE>(vw, v0, v1, lane);
    }
}

// One group of KS walk steps (see walk_group of fused_stage_fwd for the
// row bookkeeping); urow points at this lane's first u column (2j) of the
// step-0 row, hrow at its float2 of the h row completed at step 0.  FIRST as
// in walk_group: the first 2R steps only prime the z accumulators.
template <int KS, int UP, bool INTERIOR, bool FIRST = false, bool LAST = false>
__device__ __forceinline__ void pair_group(const float* __restrict__ urow, float2* __restrict__ hrow,
                                           const float (&kr)[KS][KS], float (&za0)[KS],
                                           float (&za1)[KS], float (&ha0)[KS], float (&ha1)[KS],
                                           int m0, int zrow0, int H, bool col_in0, bool col_in1,
                                           int mz_lo, int mh_lo, int mh_hi, int lane,
                                           const float* __restrict__ wp, const RbfConst& rc)
{
    constexpr int R = KS / 2;
#pragma unroll
    for (int mm = 0; mm < KS; ++mm) {
        const int m = m0 + mm;
        if constexpr (LAST) {
            if (m >= mh_hi) break;   // partial last group
        }
        const float2* row = reinterpret_cast<const float2*>(urow + m * UP);
        float in[2 * R + 2];   // in[t] = u(row, c0 - R + t)
#pragma unroll
        for (int t2 = 0; t2 <= R; ++t2) {
            const float2 p = row[t2];
            in[2 * t2] = p.x;
            in[2 * t2 + 1] = p.y;
        }
        // z(c) = sum_{a,b} k[a][b] u(i + R - a, c + R - b): the row feeds slots (step + a) mod KS
#pragma unroll
        for (int b = 0; b < KS; ++b) {
#pragma unroll
            for (int a = 0; a < KS; ++a) {
                if (FIRST && mm + a < 2 * R) continue;
                const int s = (mm + a) % KS;
                za0[s] = fmaf(kr[a][b], in[2 * R - b], za0[s]);
                za1[s] = fmaf(kr[a][b], in[2 * R + 1 - b], za1[s]);
            }
        }
        const float z0 = za0[mm], z1 = za1[mm];
        za0[mm] = 0.0f;
        za1[mm] = 0.0f;
        if constexpr (FIRST) {
            if (mm < 2 * R) continue;
        }
        float v0 = rbf_phi_w(z0, wp, rc);
        float v1 = rbf_phi_w(z1, wp, rc);
        if constexpr (!INTERIOR) {
            const int zi = zrow0 + m;
            const bool row_ok = (m >= mz_lo) && ((unsigned)zi < (unsigned)H);
            v0 = (row_ok && col_in0) ? v0 : 0.0f;
            v1 = (row_ok && col_in1) ? v1 : 0.0f;
        }
        float vw[KS + 1];
        gather_pair<KS, 0, !INTERIOR>(vw, v0, v1, lane);
        // h(c) = sum_{a,b} k[a][b] v(i - R + a, c - R + b): slots (step - a) mod KS
#pragma unroll
        for (int b = 0; b < KS; ++b) {
#pragma unroll
            for (int a = 0; a < KS; ++a) {
                const int s = (mm - a + 2 * KS) % KS;
                ha0[s] = fmaf(kr[a][b], vw[b], ha0[s]);
                ha1[s] = fmaf(kr[a][b], vw[b + 1], ha1[s]);
            }
        }
        const int sf = (mm - 2 * R + 2 * KS) % KS;
        if (m >= mh_lo && m < mh_hi) {
            float2 h = hrow[m * 32];
            h.x += ha0[sf];
            h.y += ha1[sf];
            hrow[m * 32] = h;
        }
        ha0[sf] = 0.0f;
        ha1[sf] = 0.0f;
    }
}

// One stage on one tile.  rank selects the CTA's half of the filters and of
// the epilogue when NSPLIT = 2 (the two CTAs of a cluster share the tile);
// remote_h is then the other CTA's h buffers (distributed shared memory).
// The haloed u_{t-1} tile is staged by a bulk tensor copy (j.umap set, start
// column even) or gathered through L2.  Returns the staged column of x0 - 2R,
// or -1 (uniform over the CTA) if the copy never landed.
template <int KS, int NK, int TH, int NSPLIT>
__device__ __forceinline__ int pair_tile_walk(const TileJob& j, float* smem, int rank)
{
    using C = PairCfg<KS, NK, TH, NSPLIT>;
    constexpr int R = C::R;
    constexpr int TW = C::TW;
    float* sU = smem;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* myH = smem + ((C::U_FL + 3) & ~3) + warp * C::PW_FL;
    float* myK = myH + C::H_FL;
    float* myW = myK + C::KPAD;
    const int ty = j.ty, tx = j.tx;
    const int H = j.H, W = j.W;
    const RowTile rt = row_tile(ty, j.tiles_y, H, min(j.th, TH), min(j.te, TH), R);
    const int y0 = rt.y0, x0 = tile_origin(tx, TW, W);
    const bool ext = (ty == 0) || (ty == j.tiles_y - 1);
    const bool border = ext || (tx == 0) || (tx == j.tiles_x - 1);
    const RbfConst& rc = *j.rc;

    for (int e = lane; e < C::H_FL; e += 32) myH[e] = 0.0f;
    for (int e = lane; e < C::WPADN; e += 32) myW[e] = 0.0f;
    // float2 row reads: the staged column of x0 - 2R must be even (ends with a CTA barrier)
    const int xoff = stage_u_tile<C::UH, C::UW, C::NTHREADS, 2>(j, sU, y0 - 3 * R, x0 - 2 * R);
    if (xoff < 0) return -1;

    const int hy0 = ext ? y0 - R : y0;
    const int nh = ext ? rt.h + 2 * R : rt.h;
    const int nsteps = nh + 4 * R;
    const int ub0 = ext ? 0 : R;
    const float* urow = sU + ub0 * C::UP + xoff + 2 * lane;
    float2* hrow = reinterpret_cast<float2*>(myH) + (hy0 - 4 * R - (y0 - R)) * 32 + lane;
    const int zrow0 = hy0 - 3 * R;
    const int c0 = x0 - R + 2 * lane;
    const bool col_in0 = (unsigned)c0 < (unsigned)W;
    const bool col_in1 = (unsigned)(c0 + 1) < (unsigned)W;

#pragma unroll 1
    for (int fl = 0; fl < C::FPW; ++fl) {
        const int fi = rank * C::NK_CTA + warp * C::FPW + fl;
        for (int e = lane; e < KS * KS; e += 32) myK[e] = __ldg(j.k + fi * KS * KS + e);
        for (int e = lane; e < j.nrbf; e += 32) myW[RBF_WPAD + e] = __ldg(j.w + fi * j.nrbf + e);
        __syncwarp();
        float kr[KS][KS];
#pragma unroll
        for (int p = 0; p < KS; ++p)
#pragma unroll
            for (int q = 0; q < KS; ++q) kr[p][q] = myK[p * KS + q];
        float za0[KS], za1[KS], ha0[KS], ha1[KS];
#pragma unroll
        for (int s = 0; s < KS; ++s) za0[s] = za1[s] = ha0[s] = ha1[s] = 0.0f;
        // whole groups of KS steps, then the partial last one (if any)
        int m0 = KS;
        if (!border) {
            pair_group<KS, C::UP, true, true>(urow, hrow, kr, za0, za1, ha0, ha1, 0, zrow0, H,
                                              col_in0, col_in1, 2 * R, 4 * R, nsteps, lane, myW, rc);
#pragma unroll 1
            for (; m0 + KS <= nsteps; m0 += KS)
                pair_group<KS, C::UP, true>(urow, hrow, kr, za0, za1, ha0, ha1, m0, zrow0, H,
                                            col_in0, col_in1, 2 * R, 4 * R, nsteps, lane, myW, rc);
            if (m0 < nsteps)
                pair_group<KS, C::UP, true, false, true>(urow, hrow, kr, za0, za1, ha0, ha1, m0,
                                                         zrow0, H, col_in0, col_in1, 2 * R, 4 * R,
                                                         nsteps, lane, myW, rc);
        } else {
            pair_group<KS, C::UP, false, true>(urow, hrow, kr, za0, za1, ha0, ha1, 0, zrow0, H,
                                               col_in0, col_in1, 2 * R, 4 * R, nsteps, lane, myW, rc);
#pragma unroll 1
            for (; m0 + KS <= nsteps; m0 += KS)
                pair_group<KS, C::UP, false>(urow, hrow, kr, za0, za1, ha0, ha1, m0, zrow0, H,
                                             col_in0, col_in1, 2 * R, 4 * R, nsteps, lane, myW, rc);
            if (m0 < nsteps)
                pair_group<KS, C::UP, false, false, true>(urow, hrow, kr, za0, za1, ha0, ha1, m0,
                                                          zrow0, H, col_in0, col_in1, 2 * R, 4 * R,
                                                          nsteps, lane, myW, rc);
        }
        __syncwarp();
    }
    return xoff;
}

// Epilogue over the tile's own pixels idx = first, first + step, ...:
// g = fold(sum of the h buffers), u_t = prox(u_{t-1} - g).  xoff: staged
// column of x0 - 2R.
template <int KS, int NK, int TH, int NSPLIT>
__device__ __forceinline__ void pair_tile_epilogue(const TileJob& j, const float* smem,
                                                   const float* remote, int first, int step,
                                                   int xoff)
{
    using C = PairCfg<KS, NK, TH, NSPLIT>;
    constexpr int R = C::R;
    constexpr int TW = C::TW;
    const float* sU = smem;
    const float* sH = smem + ((C::U_FL + 3) & ~3);
    const int ty = j.ty, tx = j.tx;
    const int H = j.H, W = j.W;
    const RowTile rt = row_tile(ty, j.tiles_y, H, min(j.th, TH), min(j.te, TH), R);
    const int y0 = rt.y0, x0 = tile_origin(tx, TW, W);
    const bool ext = (ty == 0) || (ty == j.tiles_y - 1);
    const bool border = ext || (tx == 0) || (tx == j.tiles_x - 1);
    const float lam = __ldg(j.lam);
    const int wy0 = rt.wy0, wy1 = rt.wy1;
    const int wx0 = tile_split(tx, TW, W, j.tiles_x, R), wx1 = tile_split(tx + 1, TW, W, j.tiles_x, R);
    for (int idx = first; idx < rt.h * TW; idx += step) {
        const int qy = y0 + idx / TW, qx = x0 + idx % TW;
        if (qy < wy0 || qy >= wy1 || qx < wx0 || qx >= wx1) continue;
        int sy[2], sx[2];
        int nsy = 1, nsx = 1;
        sy[0] = qy;
        sx[0] = qx;
        if (border) {
            if (qy < R) sy[nsy++] = -1 - qy;
            else if (qy >= H - R) sy[nsy++] = 2 * H - 1 - qy;
            if (qx < R) sx[nsx++] = -1 - qx;
            else if (qx >= W - R) sx[nsx++] = 2 * W - 1 - qx;
        }
        float g = 0.0f;
        for (int p = 0; p < nsy; ++p) {
            for (int q = 0; q < nsx; ++q) {
                const int o = (sy[p] - (y0 - R)) * 64 + sx[q] - (x0 - R);
                float hs = 0.0f;
#pragma unroll
                for (int wq = 0; wq < C::NWARP; ++wq) hs += sH[wq * C::PW_FL + o];
                if constexpr (NSPLIT == 2) {
                    // the other CTA's filters summed apart and added last: the
                    // result (a + b = b + a) does not depend on which CTA of the
                    // cluster finishes the pixel, i.e. not on the tiling
                    float hr = 0.0f;
#pragma unroll
                    for (int wq = 0; wq < C::NWARP; ++wq) hr += remote[wq * C::PW_FL + o];
                    hs += hr;
                }
                g += hs;
            }
        }
        const float up = sU[(qy - y0 + 3 * R) * C::UP + (qx - x0 + 2 * R) + xoff];
        const float fv = __ldg(j.f + (size_t)qy * j.pitch + qx);
        j.u_out[(size_t)qy * j.pitch + qx] = stage_out(up, g, fv, lam, j.dterm, j.proj_c);
    }
}

// As pair_tile_epilogue for a cluster of NS CTAs: g sums the h buffers of
// every rank (hb[r], rank r's buffers) in rank order, so a pixel's bits do not
// depend on which CTA of the cluster finishes it.
template <int KS, int NK, int TH, int NS>
__device__ __forceinline__ void pair_tile_epilogue_cluster(const TileJob& j, const float* smem,
                                                           const float* const (&hb)[NS],
                                                           int first, int step, int xoff)
{
    using C = PairCfg<KS, NK, TH, NS>;
    constexpr int R = C::R;
    constexpr int TW = C::TW;
    const float* sU = smem;
    const int ty = j.ty, tx = j.tx;
    const int H = j.H, W = j.W;
    const RowTile rt = row_tile(ty, j.tiles_y, H, min(j.th, TH), min(j.te, TH), R);
    const int y0 = rt.y0, x0 = tile_origin(tx, TW, W);
    const bool ext = (ty == 0) || (ty == j.tiles_y - 1);
    const bool border = ext || (tx == 0) || (tx == j.tiles_x - 1);
    const float lam = __ldg(j.lam);
    const int wy0 = rt.wy0, wy1 = rt.wy1;
    const int wx0 = tile_split(tx, TW, W, j.tiles_x, R), wx1 = tile_split(tx + 1, TW, W, j.tiles_x, R);
    for (int idx = first; idx < rt.h * TW; idx += step) {
        const int qy = y0 + idx / TW, qx = x0 + idx % TW;
        if (qy < wy0 || qy >= wy1 || qx < wx0 || qx >= wx1) continue;
        int sy[2], sx[2];
        int nsy = 1, nsx = 1;
        sy[0] = qy;
        sx[0] = qx;
        if (border) {
            if (qy < R) sy[nsy++] = -1 - qy;
            else if (qy >= H - R) sy[nsy++] = 2 * H - 1 - qy;
            if (qx < R) sx[nsx++] = -1 - qx;
            else if (qx >= W - R) sx[nsx++] = 2 * W - 1 - qx;
        }
        float g = 0.0f;
        for (int p = 0; p < nsy; ++p) {
            for (int q = 0; q < nsx; ++q) {
                const int o = (sy[p] - (y0 - R)) * 64 + sx[q] - (x0 - R);
                float hs = 0.0f;
#pragma unroll
                for (int r = 0; r < NS; ++r) {
                    float hr = 0.0f;
#pragma unroll
                    for (int wq = 0; wq < C::NWARP; ++wq) hr += hb[r][wq * C::PW_FL + o];
                    hs += hr;
                }
                g += hs;
            }
        }
        const float up = sU[(qy - y0 + 3 * R) * C::UP + (qx - x0 + 2 * R) + xoff];
        const float fv = __ldg(j.f + (size_t)qy * j.pitch + qx);
        j.u_out[(size_t)qy * j.pitch + qx] = stage_out(up, g, fv, lam, j.dterm, j.proj_c);
    }
}

__device__ __forceinline__ TileJob pair_job(const StageArgs& a, int tile, int th_kernel)
{
    const int n = blockIdx.y;
    TileJob j;
    j.u_in = a.u_in + (size_t)n * a.img_stride;
    j.u_out = a.u_out + (size_t)n * a.img_stride;
    j.f = a.f + (size_t)n * a.img_stride;
    j.H = a.H;
    j.W = a.W;
    j.pitch = a.pitch;
    j.tiles_x = a.tiles_x;
    j.tiles_y = a.tiles_y;
    j.th = a.th > 0 ? a.th : th_kernel;
    j.te = a.te;
    j.ty = tile / a.tiles_x;
    j.tx = tile - j.ty * a.tiles_x;
    j.k = a.k;
    j.w = a.w;
    j.lam = a.lam;
    j.nrbf = a.nrbf;
    j.dterm = a.dterm;
    j.proj_c = a.proj_c;
    j.rc = &a.rc;
    j.umap = a.use_tma ? &a.umap : nullptr;
    j.img = n;
    j.err = a.err;
    j.wait_limit = a.wait_limit;
    j.tx_extra = a.tx_extra;
    return j;
}

// One CTA per tile; grid (tiles_x * tiles_y, N).
template <int KS, int NK, int TH>
__global__ void __launch_bounds__(PairCfg<KS, NK, TH, 1>::NTHREADS, 2)
fused_pair_fwd(const __grid_constant__ StageArgs a)
{
    extern __shared__ __align__(128) float smem[];
    tc::pdl_launch_dependents();   // the next stage may launch; it waits before touching u
    const TileJob j = pair_job(a, blockIdx.x, TH);
    const int xoff = pair_tile_walk<KS, NK, TH, 1>(j, smem, 0);
    if (xoff < 0) return;
    __syncthreads();
    pair_tile_epilogue<KS, NK, TH, 1>(j, smem, nullptr, threadIdx.x,
                                      PairCfg<KS, NK, TH, 1>::NTHREADS, xoff);
}

// A cluster of two CTAs per tile; grid (2 * tiles_x * tiles_y, N).
template <int KS, int NK, int TH>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(PairCfg<KS, NK, TH, 2>::NTHREADS, 2)
fused_pair2_fwd(const __grid_constant__ StageArgs a)
{
    namespace cg = cooperative_groups;
    using C = PairCfg<KS, NK, TH, 2>;
    extern __shared__ __align__(128) float smem[];
    __shared__ int s_xoff;
    tc::pdl_launch_dependents();   // the next stage may launch; it waits before touching u
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const TileJob j = pair_job(a, blockIdx.x >> 1, TH);
    const int xoff = pair_tile_walk<KS, NK, TH, 2>(j, smem, rank);
    if (threadIdx.x == 0) s_xoff = xoff;
    cl.sync();   // both CTAs' h buffers complete and visible in the cluster
    const float* remote = cl.map_shared_rank(smem, rank ^ 1) + ((C::U_FL + 3) & ~3);
    // both CTAs pass both cluster barriers; the epilogue runs only if both tiles staged
    if (xoff >= 0 && *cl.map_shared_rank(&s_xoff, rank ^ 1) >= 0)
        pair_tile_epilogue<KS, NK, TH, 2>(j, smem, remote, rank * C::NTHREADS + threadIdx.x,
                                          2 * C::NTHREADS, xoff);
    cl.sync();   // keep this CTA's shared memory alive until the other has read it
}

// A cluster of NS (4 or 8) CTAs per tile; grid (NS * tiles_x * tiles_y, N).
template <int KS, int NK, int TH, int NS>
__global__ void __cluster_dims__(NS, 1, 1) __launch_bounds__(PairCfg<KS, NK, TH, NS>::NTHREADS, 2)
fused_pairc_fwd(const __grid_constant__ StageArgs a)
{
    namespace cg = cooperative_groups;
    using C = PairCfg<KS, NK, TH, NS>;
    extern __shared__ __align__(128) float smem[];
    __shared__ int s_xoff;
    tc::pdl_launch_dependents();   // the next stage may launch; it waits before touching u
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const TileJob j = pair_job(a, blockIdx.x / NS, TH);
    const int xoff = pair_tile_walk<KS, NK, TH, NS>(j, smem, rank);
    if (threadIdx.x == 0) s_xoff = xoff;
    cl.sync();   // every CTA's h buffers complete and visible in the cluster
    const float* hb[NS];
    bool all = xoff >= 0;
#pragma unroll
    for (int r = 0; r < NS; ++r) {
        hb[r] = cl.map_shared_rank(smem, r) + ((C::U_FL + 3) & ~3);
        all = all && *cl.map_shared_rank(&s_xoff, r) >= 0;
    }
    // every CTA passes both cluster barriers; the epilogue runs only if all tiles staged
    if (all)
        pair_tile_epilogue_cluster<KS, NK, TH, NS>(j, smem, hb, rank * C::NTHREADS + threadIdx.x,
                                                   NS * C::NTHREADS, xoff);
    cl.sync();   // keep this CTA's shared memory alive until the others have read it
}

// Grid-wide barrier of a single-launch cascade: every CTA adds one to
// *counter and waits until it reaches `target` (all CTAs of the launch are
// resident: the host checks that before it uses the cascade).  The wait is
// bounded by `limit` SM cycles; false if it ran out.  Writes before the barrier
// are visible to loads through L2 after it (fence, then release/acquire on the
// counter).
__device__ __forceinline__ bool cascade_barrier(int* counter, int target, long long limit)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(counter, 1);
        const long long t0 = clock64();
        int ok = 1;
        for (;;) {
            int v;
            asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(counter) : "memory");
            if (v >= target) break;
            if (clock64() - t0 > limit) {
                ok = 0;
                break;
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// All T stages on clusters of NS CTAs per tile (grid NS * tiles_x * tiles_y,
// N), one launch: the small images whose per-stage launches are dominated by
// start-up (cold instruction cache, tile copy, cluster barriers).  Each stage
// is the column-pair walk and the cluster epilogue of fused_pairc_fwd with the
// tile gathered through L2 (its u was written by other CTAs in this launch);
// a grid barrier separates the stages.  If a barrier wait runs out, the status
// word gets TNRD_ERR_TIMEOUT and the CTAs still run every stage and barrier
// (each wait bounded), so that no cluster barrier is left waiting.
template <int KS, int NK, int TH, int NS>
__global__ void __cluster_dims__(NS, 1, 1) __launch_bounds__(PairCfg<KS, NK, TH, NS>::NTHREADS, 2)
fused_pairc_cascade(const __grid_constant__ CascadeArgs c)
{
    namespace cg = cooperative_groups;
    using C = PairCfg<KS, NK, TH, NS>;
    extern __shared__ __align__(128) float smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int n = blockIdx.y;
    const int tile = blockIdx.x / NS;
    const int nctas = (int)(gridDim.x * gridDim.y);
    const float* hb[NS];
#pragma unroll
    for (int r = 0; r < NS; ++r) hb[r] = cl.map_shared_rank(smem, r) + ((C::U_FL + 3) & ~3);
    bool ok = true;
#pragma unroll 1
    for (int t = 0; t < c.T; ++t) {
        const float* in;
        float* out;
        if (c.keep) {
            in = (t == 0) ? c.f : c.u + (size_t)t * c.batch;
            out = c.u + (size_t)(t + 1) * c.batch;
        } else {
            // stage t writes u when (T-1-t) is even, so the last stage lands in u
            float* cur = ((c.T - 1 - t) % 2 == 0) ? c.u : c.pp;
            float* prev = ((c.T - t) % 2 == 0) ? c.u : c.pp;
            in = (t == 0) ? c.f : prev;
            out = cur;
        }
        TileJob j;
        j.u_in = in + (size_t)n * c.img_stride;
        j.u_out = out + (size_t)n * c.img_stride;
        j.f = c.f + (size_t)n * c.img_stride;
        j.H = c.H;
        j.W = c.W;
        j.pitch = c.pitch;
        j.tiles_x = c.tiles_x;
        j.tiles_y = c.tiles_y;
        j.th = c.th > 0 ? c.th : TH;
        j.te = c.te;
        j.ty = tile / c.tiles_x;
        j.tx = tile - j.ty * c.tiles_x;
        j.k = c.k + (size_t)t * NK * KS * KS;
        j.w = c.w + (size_t)t * NK * c.nrbf;
        j.lam = c.lam + t;
        j.nrbf = c.nrbf;
        j.dterm = c.dterm;
        j.proj_c = c.proj_c;
        j.rc = &c.rc;
        j.umap = nullptr;   // gather through L2: the tile was written in this launch
        j.img = n;
        j.err = c.err;
        const int xoff = pair_tile_walk<KS, NK, TH, NS>(j, smem, rank);
        cl.sync();   // every CTA's h buffers complete and visible in the cluster
        pair_tile_epilogue_cluster<KS, NK, TH, NS>(j, smem, hb, rank * C::NTHREADS + threadIdx.x,
                                                   NS * C::NTHREADS, xoff);
        cl.sync();   // the other CTAs have read this CTA's h buffers
        if (t + 1 < c.T) ok = cascade_barrier(c.counter, (t + 1) * nctas, c.wait_limit) && ok;
    }
    if (!ok && threadIdx.x == 0) atomicExch(c.err, 4 /* TNRD_ERR_TIMEOUT */);
}

}  // namespace tnrd
