// Fused FP32 forward stage of TRDMD (Eq. diffusionprocessfinal):
//   u_t = prox(u_{t-1} - sum_i K_i^T phi_i(K_i u_{t-1}))
// in ONE kernel per stage.  The N_k filter responses z_i, v_i = phi_i(z_i)
// live only in registers; u_{t-1} is staged once per tile in shared memory and
// only u_t is written to HBM.
//
// Tile: th rows (runtime, at most the compiled TH; the first and last tile
// rows may be shorter, see row_tile) x TW = 32 - 2R output columns, R =
// ksize/2.  Warp lane j owns
// z-column x0 - R + j, so the 32 lanes cover the tile plus the R-wide column
// halo that the adjoint needs.  Each warp owns nfilt/NWARP filters; for each
// filter it walks down its columns once ("walk"), one input row per step:
//   1. z rows:   z(i) = sum_{a,b} k[a][b] u(i + R - a, x + R - b), kept in ksize
//                rolling accumulators; row i is complete after input row i + R.
//   2. v = phi(z) for the completed row (0 outside the image).
//   3. the 2R+1 v values of the neighbouring columns come from warp shuffles,
//   4. h rows:   h(i) = sum_{a,b} k[a][b] v(i - R + a, x - R + b), again ksize
//                rolling accumulators; row i is complete after v row i + R,
//                and is added into the warp's h buffer in shared memory.
// h is the adjoint of the zero-extended convolution; the exact transpose of
// the symmetric-padded convolution folds it back at the border:
//   (K^T v)(q) = sum_{q' : sym(q') = q} h(q').
// Tiles on the top/bottom row of tiles walk R extra h rows on each side (the
// mirror sources); on the left/right the extra columns are the halo lanes,
// whose missing neighbours lie outside the image where v = 0.
// The epilogue sums the warps' h, folds, applies the prox and stores u_t.
#pragma once
#include "args.cuh"
#include "tile_stage.cuh"

namespace tnrd {

// Value of lane + D's x.  With EDGE, 0 when lane + D falls outside the warp;
// without, whatever the shuffle returns there (used only by halo lanes whose
// h values an interior tile never reads).
template <int D, bool EDGE>
__device__ __forceinline__ float shfl_rel(float x, int lane)
{
    if constexpr (D == 0) {
        return x;
    } else if constexpr (D > 0) {
        const float y = __shfl_down_sync(0xffffffffu, x, D);
        return (!EDGE || lane + D < 32) ? y : 0.0f;
    } else {
        const float y = __shfl_up_sync(0xffffffffu, x, -D);
        return (!EDGE || lane + D >= 0) ? y : 0.0f;
    }
}

template <int KS, int B, bool EDGE>
__device__ __forceinline__ void gather_row(float (&vw)[KS], float v, int lane)
{
    if constexpr (B < KS) {
        vw[B] = shfl_rel<B - KS / 2, EDGE>(v, lane);
        gather_row<KS, B + 1, EDGE>(vw, v, lane);
    }
}

// One group of KS walk steps starting at step m0 (see the file comment).
//   urow  : shared-memory pointer to u row of step 0 at this lane's z-column
//           minus 2R columns (u(step m, column offset c - R) = urow[m*UP + c + R])
//   hrow  : this warp's h buffer at the h row completed at step 0, this lane
//   zrow0 : image row of the z row completed at step 0
// INTERIOR: the tile touches no image border, so every z of a valid step is
// inside the image and no v needs masking (partial z rows of the first 2R
// steps only reach h rows above the tile, which are never stored).
// FIRST: the group of steps 0 .. KS-1, whose first 2R steps only prime the z
// accumulators -- their phi, shuffles and h updates would reach no stored h
// row, and the z updates of rows completing before step 2R no used z, so they
// are left out (the stored values are the same bits).
// LAST: the walk's final group, which may be partial: steps from mh_hi (the
// walk's step count) on are not taken.
template <int KS, int UP, bool INTERIOR, bool FIRST = false, bool LAST = false>
__device__ __forceinline__ void walk_group(const float* __restrict__ urow, float* __restrict__ hrow,
                                           const float (&kr)[KS][KS], float (&za)[KS],
                                           float (&ha)[KS], int m0, int zrow0, int H, bool col_in,
                                           int mz_lo, int mh_lo, int mh_hi, int lane,
                                           const float* __restrict__ tab, const RbfConst& rc)
{
    constexpr int R = KS / 2;
#pragma unroll
    for (int mm = 0; mm < KS; ++mm) {
        const int m = m0 + mm;
        if constexpr (LAST) {
            if (m >= mh_hi) break;
        }
        const float* row = urow + m * UP;
        float in[KS];
#pragma unroll
        for (int b = 0; b < KS; ++b) in[b] = row[2 * R - b];
        // z: the input row feeds z slots (step + a) mod KS; slot mm completes (a = 0)
#pragma unroll
        for (int b = 0; b < KS; ++b) {
#pragma unroll
            for (int a = 0; a < KS; ++a) {
                if (FIRST && mm + a < 2 * R) continue;
                const int s = (mm + a) % KS;
                za[s] = fmaf(kr[a][b], in[b], za[s]);
            }
        }
        const float z = za[mm];
        za[mm] = 0.0f;
        if constexpr (FIRST) {
            if (mm < 2 * R) continue;
        }
        float v = rbf_phi_tab(z, tab, rc);
        if constexpr (!INTERIOR) {
            const int zi = zrow0 + m;
            const bool v_ok = col_in && (m >= mz_lo) && ((unsigned)zi < (unsigned)H);
            v = v_ok ? v : 0.0f;
        }
        float vw[KS];
        gather_row<KS, 0, !INTERIOR>(vw, v, lane);
        // h: the v row feeds h slots (step - a) mod KS; slot (mm - 2R) completes (a = 2R)
#pragma unroll
        for (int b = 0; b < KS; ++b) {
#pragma unroll
            for (int a = 0; a < KS; ++a) {
                const int s = (mm - a + 2 * KS) % KS;
                ha[s] = fmaf(kr[a][b], vw[b], ha[s]);
            }
        }
        const int sf = (mm - 2 * R + 2 * KS) % KS;
        if (m >= mh_lo && m < mh_hi) hrow[m * 32] += ha[sf];
        ha[sf] = 0.0f;
    }
}

// One stage on one tile (the whole CTA).  The haloed u_{t-1} tile is staged by
// a bulk tensor copy when j.umap is set, else gathered through L2
// (ld.global.cg), which lets a persistent kernel read tiles that other CTAs
// wrote earlier in the same launch; ends with a CTA barrier after the stores.
template <int KS, int NK, int TH>
__device__ __forceinline__ void stage_tile(const TileJob& j, float* smem)
{
    using C = FusedCfg<KS, NK, TH>;
    constexpr int R = C::R;
    constexpr int TW = C::TW;
    float* sU = smem;                          // rows [y0-3R, ...) x cols [x0-2R, x0+TW+2R)
    float* sH = sU + C::U_FL;                  // per warp: rows [y0-R, y0+TH+R) x 32 lanes
    float* sKW = sH + C::NWARP * C::H_FL;
    float* sTab = smem + C::TAB_OFF;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ty = j.ty, tx = j.tx;
    const int H = j.H, W = j.W;
    // rows of this tile (runtime height th <= TH; border tile rows te, if set)
    const RowTile rt = row_tile(ty, j.tiles_y, H, min(j.th, TH), min(j.te, TH), R);
    const int y0 = rt.y0, x0 = tile_origin(tx, TW, W);
    const bool ext = (ty == 0) || (ty == j.tiles_y - 1);
    const bool border = ext || (tx == 0) || (tx == j.tiles_x - 1);
    const RbfConst& rc = *j.rc;

    float* myH = sH + warp * C::H_FL;
    float* myK = sKW + warp * C::KW_FL;
    float* myW = myK + C::KPAD;
    float* myT = sTab + warp * RBF_TP * RBF_NCOEF;
    for (int e = lane; e < C::H_FL; e += 32) myH[e] = 0.0f;
    for (int e = lane; e < C::WPADN; e += 32) myW[e] = 0.0f;
    // staged column of x0 - 2R (ends with a CTA barrier)
    const int xoff = stage_u_tile<C::UH, C::UW, C::NTHREADS, 1>(j, sU, y0 - 3 * R, x0 - 2 * R);
    if (xoff < 0) return;   // the copy never landed (status recorded)

    // Walk geometry.  h rows [hy0, hy0 + nh); step m reads u row hy0 - 2R + m,
    // completes z row hy0 - 3R + m (valid from m = 2R) and h row hy0 - 4R + m
    // (valid for m in [4R, nh + 4R)).  Steps run in groups of KS, the last one
    // stopping at step nh + 4R; the U buffer has rows for a whole last group.
    const int hy0 = ext ? y0 - R : y0;
    const int nh = ext ? rt.h + 2 * R : rt.h;
    const int nsteps = nh + 4 * R;
    const int ub0 = ext ? 0 : R;                         // U buffer row of step 0
    const float* urow = sU + ub0 * C::UP + xoff + lane;
    float* hrow = myH + (hy0 - 4 * R - (y0 - R)) * 32 + lane;
    const int zrow0 = hy0 - 3 * R;
    const bool col_in = (unsigned)(x0 - R + lane) < (unsigned)W;

#pragma unroll 1
    for (int fl = 0; fl < C::FPW; ++fl) {
        const int fi = warp * C::FPW + fl;
        for (int e = lane; e < KS * KS; e += 32) myK[e] = __ldg(j.k + fi * KS * KS + e);
        for (int e = lane; e < j.nrbf; e += 32) myW[RBF_WPAD + e] = __ldg(j.w + fi * j.nrbf + e);
        __syncwarp();
        rbf_build_table(myT, myW, j.nrbf, rc, lane);
        float kr[KS][KS];
#pragma unroll
        for (int p = 0; p < KS; ++p)
#pragma unroll
            for (int q = 0; q < KS; ++q) kr[p][q] = myK[p * KS + q];
        __syncwarp();
        float za[KS], ha[KS];
#pragma unroll
        for (int s = 0; s < KS; ++s) za[s] = ha[s] = 0.0f;
        // whole groups of KS steps, then the partial last one (if any)
        int m0 = KS;
        if (!border) {
            walk_group<KS, C::UP, true, true>(urow, hrow, kr, za, ha, 0, zrow0, H, col_in, 2 * R,
                                              4 * R, nsteps, lane, myT, rc);
#pragma unroll 1
            for (; m0 + KS <= nsteps; m0 += KS)
                walk_group<KS, C::UP, true>(urow, hrow, kr, za, ha, m0, zrow0, H, col_in, 2 * R,
                                            4 * R, nsteps, lane, myT, rc);
            if (m0 < nsteps)
                walk_group<KS, C::UP, true, false, true>(urow, hrow, kr, za, ha, m0, zrow0, H,
                                                         col_in, 2 * R, 4 * R, nsteps, lane, myT, rc);
        } else {
            walk_group<KS, C::UP, false, true>(urow, hrow, kr, za, ha, 0, zrow0, H, col_in, 2 * R,
                                               4 * R, nsteps, lane, myT, rc);
#pragma unroll 1
            for (; m0 + KS <= nsteps; m0 += KS)
                walk_group<KS, C::UP, false>(urow, hrow, kr, za, ha, m0, zrow0, H, col_in, 2 * R,
                                             4 * R, nsteps, lane, myT, rc);
            if (m0 < nsteps)
                walk_group<KS, C::UP, false, false, true>(urow, hrow, kr, za, ha, m0, zrow0, H,
                                                          col_in, 2 * R, 4 * R, nsteps, lane, myT, rc);
        }
        __syncwarp();
    }
    __syncthreads();

    // Epilogue: g = fold(sum over warps of h), u_t = prox(u_{t-1} - g).
    const float lam = __ldg(j.lam);
    const int wy0 = rt.wy0, wy1 = rt.wy1;
    const int wx0 = tile_split(tx, TW, W, j.tiles_x, R), wx1 = tile_split(tx + 1, TW, W, j.tiles_x, R);
    for (int idx = threadIdx.x; idx < rt.h * TW; idx += C::NTHREADS) {
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
                const int hi = sy[p] - (y0 - R), hj = sx[q] - (x0 - R);
                float hs = 0.0f;
#pragma unroll
                for (int wq = 0; wq < C::NWARP; ++wq) hs += sH[wq * C::H_FL + hi * 32 + hj];
                g += hs;
            }
        }
        const float up = sU[(qy - y0 + 3 * R) * C::UP + (qx - x0 + 2 * R) + xoff];
        const float fv = __ldg(j.f + (size_t)qy * j.pitch + qx);
        j.u_out[(size_t)qy * j.pitch + qx] = stage_out(up, g, fv, lam, j.dterm, j.proj_c);
    }
    __syncthreads();
}

template <int KS, int NK, int TH>
__global__ void __launch_bounds__(FusedCfg<KS, NK, TH>::NTHREADS, FusedCfg<KS, NK, TH>::MINB)
fused_stage_fwd(const __grid_constant__ StageArgs a)
{
    extern __shared__ __align__(128) float smem[];
    tc::pdl_launch_dependents();   // the next stage may launch; it waits before touching u
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
    j.th = a.th > 0 ? a.th : TH;
    j.te = a.te;
    j.ty = blockIdx.x / a.tiles_x;
    j.tx = blockIdx.x - j.ty * a.tiles_x;
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
    stage_tile<KS, NK, TH>(j, smem);
}

}  // namespace tnrd
