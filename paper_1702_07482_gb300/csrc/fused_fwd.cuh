// Fused FP32 forward stage of TRDMD (Eq. diffusionprocessfinal):
//   u_t = prox(u_{t-1} - sum_i K_i^T phi_i(K_i u_{t-1}))
// in ONE kernel per stage.  A CTA owns a TH x 32 output tile; the N_k filter
// responses z_i and v_i = phi_i(z_i) never leave shared memory/registers and
// only u_t is written to HBM.
//
// Tile geometry ("buffer" coordinates have their origin at image pixel
// (y0 - 2R, x0 - 2R), R = ksize/2):
//   U : u_{t-1} over rows [0, TH+4R) x cols [0, 32+4R), symmetric-padded
//   z-region (where z_i, v_i are needed): rows [R, TH+3R) x cols [R, 32+3R)
//   tile (outputs): rows [2R, TH+2R) x cols [2R, 34+... ) i.e. 32 columns
//   V : v_i over the same extents as U; zero outside the image and outside
//       the z-region (the zero margin lets the adjoint read without tests)
//   h = sum_i C_i^T v_i, the zero-extended adjoint, over the "extended region"
//       (= z-region) for tiles on the image border, over the tile otherwise.
// The exact transpose of the symmetric-padded convolution folds h back:
//   (K^T v)(q) = sum_{q' : sym(q') = q} h(q'),
// so border pixels add the h values of their mirror images outside the image.
//
// Work split: 4 warps, each owning nfilt/4 filters for the whole tile, so the
// filter loop needs no CTA barrier.  Inside a warp each lane owns one column
// and walks it top to bottom ("strip"), keeping ksize rolling accumulators;
// every input row read from shared memory (ksize values) feeds ksize^2 FMAs.
#pragma once
#include "args.cuh"

namespace tnrd {

// z strip: lane column j (buffer coords), outputs rows [i0, i1).
//   z(i, j) = sum_{a,b} k[a][b] U[i + R - a][j + R - b]
// Input row rho = i0 - R + m feeds output i with a = (i - i0) + 2R - m; output
// i is complete after a = 0.  Accumulator slot of output i: (i - i0) mod KS.
template <int KS, int UP>
__device__ __forceinline__ void z_strip(const float* __restrict__ sU, float* __restrict__ sV,
                                        const float (&kr)[KS][KS], int j, int i0, int i1,
                                        int img_y0, int img_x0, int H, int W,
                                        const float* wp, const RbfConst& rc)
{
    constexpr int R = KS / 2;
    float acc[KS];
#pragma unroll
    for (int s = 0; s < KS; ++s) acc[s] = 0.0f;
    const int nsteps = (i1 - i0) + 2 * R;
    const int x_img = img_x0 + j;
    const bool col_in = (unsigned)x_img < (unsigned)W;
    const float* src = sU + (i0 - R) * UP + j + R;
#pragma unroll 1
    for (int m0 = 0; m0 < nsteps; m0 += KS) {
#pragma unroll
        for (int mm = 0; mm < KS; ++mm) {
            const int m = m0 + mm;
            if (m < nsteps) {
                const float* row = src + m * UP;
                float in[KS];
#pragma unroll
                for (int b = 0; b < KS; ++b) in[b] = row[-b];
#pragma unroll
                for (int a = 0; a < KS; ++a) {
                    const int s = (mm + a + 2 * KS - 2 * R) % KS;
#pragma unroll
                    for (int b = 0; b < KS; ++b) acc[s] = fmaf(kr[a][b], in[b], acc[s]);
                }
                const int sf = (mm + 2 * KS - 2 * R) % KS;
                if (m >= 2 * R) {
                    const int i = i0 + m - 2 * R;
                    const int y_img = img_y0 + i;
                    float v = 0.0f;
                    if (col_in && (unsigned)y_img < (unsigned)H) v = rbf_phi(acc[sf], wp, rc);
                    sV[i * UP + j] = v;
                }
                acc[sf] = 0.0f;
            }
        }
    }
}

// h strip: lane column j, outputs rows [i0, i1), accumulated into sH.
//   h(i, j) = sum_{a,b} k[a][b] V[i - R + a][j - R + b]
// Input row rho = i0 - R + m feeds output i with a = m - (i - i0); output i is
// complete after a = 2R.
template <int KS, int UP, int HP>
__device__ __forceinline__ void h_strip(const float* __restrict__ sV, float* __restrict__ sH,
                                        const float (&kr)[KS][KS], int j, int i0, int i1)
{
    constexpr int R = KS / 2;
    float acc[KS];
#pragma unroll
    for (int s = 0; s < KS; ++s) acc[s] = 0.0f;
    const int nsteps = (i1 - i0) + 2 * R;
    const float* src = sV + (i0 - R) * UP + j - R;
    float* dst = sH + (i0 - R) * HP + (j - R);
#pragma unroll 1
    for (int m0 = 0; m0 < nsteps; m0 += KS) {
#pragma unroll
        for (int mm = 0; mm < KS; ++mm) {
            const int m = m0 + mm;
            if (m < nsteps) {
                const float* row = src + m * UP;
                float in[KS];
#pragma unroll
                for (int b = 0; b < KS; ++b) in[b] = row[b];
#pragma unroll
                for (int a = 0; a < KS; ++a) {
                    const int s = (mm - a + 2 * KS) % KS;
#pragma unroll
                    for (int b = 0; b < KS; ++b) acc[s] = fmaf(kr[a][b], in[b], acc[s]);
                }
                const int sf = (mm - 2 * R + 2 * KS) % KS;
                if (m >= 2 * R) {
                    float* o = dst + (m - 2 * R) * HP;
                    *o += acc[sf];
                }
                acc[sf] = 0.0f;
            }
        }
    }
}

template <int KS, int NK, int TH>
__global__ void __launch_bounds__(FusedCfg<KS, NK, TH>::NTHREADS, 3)
fused_stage_fwd(const StageArgs a)
{
    using C = FusedCfg<KS, NK, TH>;
    constexpr int R = C::R;
    extern __shared__ __align__(16) float smem[];
    float* sU = smem;
    float* sV = sU + C::U_FL;
    float* sH = sV + C::NWARP * C::V_FL;
    float* sKW = sH + C::NWARP * C::H_FL;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = blockIdx.y;
    const int ty = blockIdx.x / a.tiles_x, tx = blockIdx.x - ty * a.tiles_x;
    const int H = a.H, W = a.W;
    const int y0 = tile_origin(ty, TH, H), x0 = tile_origin(tx, 32, W);
    const bool border = (ty == 0) || (ty == a.tiles_y - 1) || (tx == 0) || (tx == a.tiles_x - 1);
    const float* uin = a.u_in + (size_t)n * a.img_stride;

    for (int i = threadIdx.x; i < C::NWARP * (C::V_FL + C::H_FL + C::KW_FL); i += C::NTHREADS)
        sV[i] = 0.0f;
    for (int idx = threadIdx.x; idx < C::UH * C::UW; idx += C::NTHREADS) {
        const int i = idx / C::UW, j = idx - i * C::UW;
        const int yy = sym_idx(y0 - 2 * R + i, H), xx = sym_idx(x0 - 2 * R + j, W);
        sU[i * C::UP + j] = uin[(size_t)yy * a.pitch + xx];
    }
    __syncthreads();

    float* myV = sV + warp * C::V_FL;
    float* myH = sH + warp * C::H_FL;
    float* myK = sKW + warp * C::KW_FL;
    float* myW = myK + C::KPAD;
    const int img_y0 = y0 - 2 * R, img_x0 = x0 - 2 * R;

#pragma unroll 1
    for (int fl = 0; fl < C::FPW; ++fl) {
        const int fi = warp * C::FPW + fl;
        for (int e = lane; e < KS * KS; e += 32) myK[e] = __ldg(a.k + fi * KS * KS + e);
        for (int e = lane; e < a.nrbf; e += 32) myW[RBF_WPAD + e] = __ldg(a.w + fi * a.nrbf + e);
        __syncwarp();
        float kr[KS][KS];
#pragma unroll
        for (int p = 0; p < KS; ++p)
#pragma unroll
            for (int q = 0; q < KS; ++q) kr[p][q] = myK[p * KS + q];

        // z_i and v_i over the z-region: 32 full columns, then the 2R
        // remaining columns in row chunks spread over the lanes.
        z_strip<KS, C::UP>(sU, myV, kr, R + lane, R, R + C::ZH, img_y0, img_x0, H, W, myW, a.rc);
        if (lane < C::XC * C::NCH) {
            const int c = lane % C::XC, ch = lane / C::XC;
            const int i0 = R + ch * C::CHT, i1 = min(i0 + C::CHT, R + C::ZH);
            if (i0 < i1)
                z_strip<KS, C::UP>(sU, myV, kr, R + 32 + c, i0, i1, img_y0, img_x0, H, W, myW, a.rc);
        }
        __syncwarp();

        // h += C_i^T v_i over the tile, or over the extended region on a border tile.
        if (!border) {
            h_strip<KS, C::UP, C::HP>(myV, myH, kr, 2 * R + lane, 2 * R, 2 * R + TH);
        } else {
            h_strip<KS, C::UP, C::HP>(myV, myH, kr, R + lane, R, R + C::ZH);
            if (lane < C::XC * C::NCH) {
                const int c = lane % C::XC, ch = lane / C::XC;
                const int i0 = R + ch * C::CHT, i1 = min(i0 + C::CHT, R + C::ZH);
                if (i0 < i1) h_strip<KS, C::UP, C::HP>(myV, myH, kr, R + 32 + c, i0, i1);
            }
        }
        __syncwarp();
    }
    __syncthreads();

    // Epilogue: g = fold(sum over warps of h), u_t = prox(u_{t-1} - g).
    const float lam = __ldg(a.lam);
    const int tiles_y = a.tiles_y, tiles_x = a.tiles_x;
    const int wy0 = tile_split(ty, TH, H, tiles_y, R), wy1 = tile_split(ty + 1, TH, H, tiles_y, R);
    const int wx0 = tile_split(tx, 32, W, tiles_x, R), wx1 = tile_split(tx + 1, 32, W, tiles_x, R);
    const float* fimg = a.f + (size_t)n * a.img_stride;
    float* uout = a.u_out + (size_t)n * a.img_stride;
    for (int idx = threadIdx.x; idx < TH * 32; idx += C::NTHREADS) {
        const int qy = y0 + idx / 32, qx = x0 + (idx & 31);
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
                const int hi = sy[p] - y0 + R, hj = sx[q] - x0 + R;  // H-buffer coords
                float hs = 0.0f;
#pragma unroll
                for (int wq = 0; wq < C::NWARP; ++wq) hs += sH[wq * C::H_FL + hi * C::HP + hj];
                g += hs;
            }
        }
        const float up = sU[(qy - y0 + 2 * R) * C::UP + (qx - x0 + 2 * R)];
        const float fv = __ldg(fimg + (size_t)qy * a.pitch + qx);
        uout[(size_t)qy * a.pitch + qx] = prox_idiv(up - g, fv, lam);
    }
}

}  // namespace tnrd
