// Backward stage of TRDMD (Sec. 3.2, Eqs. iterstep, derv1, derv1-1, derv2,
// derv4).  For stage t with e = dL/du_t:
//   d        = y .* e,          y = du_t/du~_t              (Eqs. derv1, derv2)
//   dL/dlam  = sum_p x_p e_p,   x = du_t/dlam_t             (Eq. derv4)
//   b_i      = K_i d
//   c_i      = -phi_i'(z_i) .* b_i,   z_i = K_i u_{t-1}
//   dL/dw_ij = -sum_p b_i(p) G_j(z_i(p))      (phi_i is linear in w_i)
//   dL/dk_i  = sum_p c_i(p) u(p + R - (a,b)) - v_i(p) d(p + R - (a,b)),  v_i = phi_i(z_i)
//   dL/du_{t-1} = d + sum_i K_i^T c_i                       (Eq. derv1-1)
// (K_i^T of the symmetric-padded convolution is the rotated-kernel
// convolution with the border folded back, as in the forward stage.)
//
// y and x need u~ and S = sqrt(u~^2 + 8 a lam f^2), a = 1 + 2 lam.  The prox
// output u_t > 0 satisfies a u^2 - u~ u - 2 lam f^2 = 0, so both follow from
// the stored u_t exactly, without recomputing the stage:
//   u~ = a u - 2 lam f^2 / u,   S = a u + 2 lam f^2 / u,
//   y = u / S,   x = (2/a) (f^2 (1 + 4 lam) / S - u).
// u_t = 0 happens only when f = 0 and u~ <= 0, where y = x = 0.
#pragma once
#include "args.cuh"
#include "fused_fwd.cuh"   // shfl_rel / gather_row

namespace tnrd {

// grid (prep_blocks, N), 256 threads
__global__ void __launch_bounds__(256) bwd_prep(const BwdArgs a)
{
    const int n = blockIdx.y;
    const int p = blockIdx.x * 256 + threadIdx.x;
    float xe = 0.0f;
    if (p < a.H * a.W) {
        const int y = p / a.W, x = p - y * a.W;
        const size_t o = (size_t)n * a.img_stride + (size_t)y * a.pitch + x;
        const float lam = __ldg(a.lam);
        const float u = a.u_cur[o], fv = a.f[o], e = a.e_cur[o];
        const float av = fmaf(2.0f, lam, 1.0f);
        float yv = 0.0f, xv = 0.0f;
        if (u > 0.0f) {
            const float f2 = fv * fv;
            const float r = 2.0f * lam * f2 / u;
            const float S = fmaf(av, u, r);
            yv = u / S;
            xv = (2.0f / av) * (f2 * fmaf(4.0f, lam, 1.0f) / S - u);
        }
        a.d[o] = yv * e;
        xe = xv * e;
    }
    // deterministic block sum: warp shuffles, then warp 0 over the 8 warp sums
    __shared__ float ws[8];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) xe += __shfl_down_sync(0xffffffffu, xe, off);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = xe;
    __syncthreads();
    if (threadIdx.x < 32) {
        float s = threadIdx.x < 8 ? ws[threadIdx.x] : 0.0f;
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) a.part_l[n * a.prep_blocks + blockIdx.x] = s;
    }
}

// One group of KS walk steps of the backward bank kernel (geometry as in
// walk_group of the forward stage; urow/drow index the u and d buffers).
template <int KS, int UP>
__device__ __forceinline__ void bwd_walk_group(
    const float* __restrict__ urow, const float* __restrict__ drow, float* __restrict__ hrow,
    const float (&kr)[KS][KS], float (&za)[KS], float (&ba)[KS], float (&ha)[KS], int m0,
    int zrow0, int H, bool col_in, bool col_own, int wy0, int wy1, int mh_lo, int mh_hi, int lane,
    const float* __restrict__ tab, float* __restrict__ hist, int nrbf, const RbfConst& rc,
    float* __restrict__ cpl_col, float* __restrict__ vpl_col, int pitch)
{
    constexpr int R = KS / 2;
#pragma unroll
    for (int mm = 0; mm < KS; ++mm) {
        const int m = m0 + mm;
        const float* ur = urow + m * UP;
        const float* dr = drow + m * UP;
        float in[KS], dn[KS];
#pragma unroll
        for (int b = 0; b < KS; ++b) {
            in[b] = ur[2 * R - b];
            dn[b] = dr[2 * R - b];
        }
#pragma unroll
        for (int b = 0; b < KS; ++b) {
#pragma unroll
            for (int q = 0; q < KS; ++q) {
                const int s = (mm + q) % KS;
                za[s] = fmaf(kr[q][b], in[b], za[s]);
                ba[s] = fmaf(kr[q][b], dn[b], ba[s]);
            }
        }
        const float z = za[mm], bv = ba[mm];
        za[mm] = 0.0f;
        ba[mm] = 0.0f;
        const int zi = zrow0 + m;
        const bool inside = col_in && (m >= 2 * R) && ((unsigned)zi < (unsigned)H);
        float v, dphi;
        RbfWin2 win;
        rbf_phi_dphi_tab(z, tab, rc, v, dphi, win);
        const float c = inside ? -dphi * bv : 0.0f;
        v = inside ? v : 0.0f;
        if (col_own && zi >= wy0 && zi < wy1) {
            // own pixel: keep c and v for the filter gradient, and add
            // -b G_j(z) to the lane's bins j = j0 - RBF_WIN .. j0 + RBF_WIN
            cpl_col[(size_t)zi * pitch] = c;
            vpl_col[(size_t)zi * pitch] = v;
            float g = -bv * win.pre;
            const int j_lo = win.row - 2 * RBF_WIN;     // j of coefficient n = 0
#pragma unroll
            for (int nn = 0; nn <= 2 * RBF_WIN; ++nn) {
                const int mdev = nn - RBF_WIN;
                const int j = j_lo + nn;
                if (j >= 0 && j < nrbf) hist[j * 32 + lane] += g * rc.E[mdev < 0 ? -mdev : mdev];
                g *= win.q;
            }
        }
        float cw[KS];
        gather_row<KS, 0, true>(cw, c, lane);
#pragma unroll
        for (int b = 0; b < KS; ++b) {
#pragma unroll
            for (int q = 0; q < KS; ++q) {
                const int s = (mm - q + 2 * KS) % KS;
                ha[s] = fmaf(kr[q][b], cw[b], ha[s]);
            }
        }
        const int sf = (mm - 2 * R + 2 * KS) % KS;
        if (m >= mh_lo && m < mh_hi) hrow[m * 32] += ha[sf];
        ha[sf] = 0.0f;
    }
}

// grid (tiles_x * tiles_y, N), BwdCfg::NTHREADS threads
template <int KS, int NK, int TH>
__global__ void __launch_bounds__(BwdCfg<KS, NK, TH>::NTHREADS)
bwd_bank(const BwdArgs a)
{
    using C = BwdCfg<KS, NK, TH>;
    constexpr int R = C::R;
    constexpr int TW = C::TW;
    extern __shared__ __align__(16) float smem[];
    float* sU = smem;
    float* sD = sU + C::UH * C::UP;
    float* sW = sD + C::UH * C::UP;   // per-warp blocks: H | KW | HIST | TAB

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = blockIdx.y;
    const int ty = blockIdx.x / a.tiles_x, tx = blockIdx.x - ty * a.tiles_x;
    const int H = a.H, W = a.W;
    const int y0 = tile_origin(ty, TH, H), x0 = tile_origin(tx, TW, W);
    const bool ext = (ty == 0) || (ty == a.tiles_y - 1);
    const bool border = ext || (tx == 0) || (tx == a.tiles_x - 1);
    const size_t ioff = (size_t)n * a.img_stride;

    for (int idx = threadIdx.x; idx < C::UH * C::UW; idx += C::NTHREADS) {
        const int i = idx / C::UW, j = idx - i * C::UW;
        const int yy = sym_idx(y0 - 3 * R + i, H), xx = sym_idx(x0 - 2 * R + j, W);
        const size_t o = ioff + (size_t)yy * a.pitch + xx;
        sU[i * C::UP + j] = a.u_prev[o];
        sD[i * C::UP + j] = a.d[o];
    }
    float* myH = sW + warp * (C::H_FL + C::KW_FL + C::HIST_FL + C::TAB_FL);
    float* myK = myH + C::H_FL;
    float* myWp = myK + C::KPAD;
    float* myHist = myK + C::KW_FL;
    float* myT = myHist + C::HIST_FL;
    for (int e = lane; e < C::H_FL; e += 32) myH[e] = 0.0f;
    for (int e = lane; e < C::WPADN; e += 32) myWp[e] = 0.0f;
    for (int e = lane; e < C::HIST_FL; e += 32) myHist[e] = 0.0f;
    __syncthreads();

    const int wy0 = tile_split(ty, TH, H, a.tiles_y, R), wy1 = tile_split(ty + 1, TH, H, a.tiles_y, R);
    const int wx0 = tile_split(tx, TW, W, a.tiles_x, R), wx1 = tile_split(tx + 1, TW, W, a.tiles_x, R);
    const int hy0 = ext ? y0 - R : y0;
    const int nh = ext ? TH + 2 * R : TH;
    const int nsteps = nh + 4 * R;
    const int ub0 = ext ? 0 : R;
    const float* urow = sU + ub0 * C::UP + lane;
    const float* drow = sD + ub0 * C::UP + lane;
    float* hrow = myH + (hy0 - 4 * R - (y0 - R)) * 32 + lane;
    const int zrow0 = hy0 - 3 * R;
    const int xcol = x0 - R + lane;
    const bool col_in = (unsigned)xcol < (unsigned)W;
    const bool col_own = xcol >= wx0 && xcol < wx1;
    const int cta = n * (a.tiles_x * a.tiles_y) + blockIdx.x;

#pragma unroll 1
    for (int fl = 0; fl < C::FPW; ++fl) {
        const int fi = warp * C::FPW + fl;
        for (int e = lane; e < KS * KS; e += 32) myK[e] = __ldg(a.k + fi * KS * KS + e);
        for (int e = lane; e < a.nrbf; e += 32) myWp[RBF_WPAD + e] = __ldg(a.w + fi * a.nrbf + e);
        __syncwarp();
        rbf_build_table(myT, myWp, a.nrbf, a.rc, lane);
        float kr[KS][KS];
#pragma unroll
        for (int p = 0; p < KS; ++p)
#pragma unroll
            for (int q = 0; q < KS; ++q) kr[p][q] = myK[p * KS + q];
        __syncwarp();
        const size_t plane = ioff * (size_t)a.nfilt + (size_t)fi * a.img_stride;
        float* cpl_col = a.cpl + plane + (col_own ? xcol : 0);
        float* vpl_col = a.vpl + plane + (col_own ? xcol : 0);
        float za[KS], ba[KS], ha[KS];
#pragma unroll
        for (int s = 0; s < KS; ++s) za[s] = ba[s] = ha[s] = 0.0f;
#pragma unroll 1
        for (int m0 = 0; m0 < nsteps; m0 += KS)
            bwd_walk_group<KS, C::UP>(urow, drow, hrow, kr, za, ba, ha, m0, zrow0, H, col_in,
                                      col_own, wy0, wy1, 4 * R, nsteps, lane, myT, myHist,
                                      a.nrbf, a.rc, cpl_col, vpl_col, a.pitch);
        __syncwarp();
        // per-tile dL/dw_i: sum the lanes' bins (skewed reads avoid bank conflicts)
        for (int j = lane; j < a.nrbf; j += 32) {
            float s = 0.0f;
#pragma unroll 8
            for (int l = 0; l < 32; ++l) s += myHist[j * 32 + ((l + j) & 31)];
            a.part_w[((size_t)cta * a.nfilt + fi) * a.nrbf + j] = s;
        }
        __syncwarp();
        for (int e = lane; e < C::HIST_FL; e += 32) myHist[e] = 0.0f;
        __syncwarp();
    }
    __syncthreads();

    // e_{t-1} = d + fold(sum over warps of h)
    const float* sH0 = sW;
    constexpr int WSTRIDE = C::H_FL + C::KW_FL + C::HIST_FL + C::TAB_FL;
    for (int idx = threadIdx.x; idx < TH * TW; idx += C::NTHREADS) {
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
                for (int wq = 0; wq < C::NWARP; ++wq) hs += sH0[wq * WSTRIDE + hi * 32 + hj];
                g += hs;
            }
        }
        const float dv = sD[(qy - y0 + 3 * R) * C::UP + (qx - x0 + 2 * R)];
        a.e_prev[ioff + (size_t)qy * a.pitch + qx] = dv + g;
    }
}

// grid (dk_tiles_x * dk_tiles_y, N), 4 warps.  Per warp and filter: lane =
// pixel column, walk over the u/d rows of the tile plus R above and below,
// with rolling windows of the 2R+1 c and v rows that meet each u/d row r:
//   acc[a][b] += c(r - R + a) u(r, x + R - b) - v(r - R + a) d(r, x + R - b)
// (u, d symmetric-padded); rows and columns outside the tile or the image carry
// c = v = 0, so every pixel's product is counted by exactly one tile.
template <int KS, int NK>
__global__ void __launch_bounds__(128) bwd_dk(const BwdArgs a)
{
    constexpr int R = KS / 2;
    constexpr int NW = 4;
    constexpr int FPW = NK / NW;
    static_assert(NK % NW == 0, "");
    constexpr int UHD = DK_TH + 2 * R, UWD = DK_TW + 2 * R;
    __shared__ float sU[UHD * UWD];
    __shared__ float sD[UHD * UWD];
    __shared__ float sRed[NW][KS * KS][33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = blockIdx.y;
    const int ty = blockIdx.x / a.dk_tiles_x, tx = blockIdx.x - ty * a.dk_tiles_x;
    const int y0 = ty * DK_TH, x0 = tx * DK_TW;
    const int H = a.H, W = a.W;
    const size_t ioff = (size_t)n * a.img_stride;
    for (int idx = threadIdx.x; idx < UHD * UWD; idx += 128) {
        const int i = idx / UWD, j = idx - i * UWD;
        const int yy = sym_idx(y0 - R + i, H), xx = sym_idx(x0 - R + j, W);
        const size_t o = ioff + (size_t)yy * a.pitch + xx;
        sU[idx] = a.u_prev[o];
        sD[idx] = a.d[o];
    }
    __syncthreads();
    const int x = x0 + lane;
    const bool col_ok = x < W;
    const int rows_here = min(DK_TH, H - y0);
    const int cta = n * (a.dk_tiles_x * a.dk_tiles_y) + blockIdx.x;
#pragma unroll 1
    for (int fl = 0; fl < FPW; ++fl) {
        const int fi = warp * FPW + fl;
        const size_t plane = ioff * (size_t)a.nfilt + (size_t)fi * a.img_stride;
        const float* cp = a.cpl + plane + (col_ok ? x : 0);
        const float* vp = a.vpl + plane + (col_ok ? x : 0);
        float acc[KS][KS];
#pragma unroll
        for (int p = 0; p < KS; ++p)
#pragma unroll
            for (int q = 0; q < KS; ++q) acc[p][q] = 0.0f;
        // Step m handles u/d buffer row m (image row y0 - R + m).  The c/v rows
        // that meet it are tile rows m - 2R + a, a = 0..2R: window slot a.
        float cw[KS], vw[KS];
#pragma unroll
        for (int s = 0; s < KS; ++s) cw[s] = vw[s] = 0.0f;
#pragma unroll 1
        for (int m = 0; m < DK_TH + 2 * R; ++m) {
#pragma unroll
            for (int s = 0; s < KS - 1; ++s) {
                cw[s] = cw[s + 1];
                vw[s] = vw[s + 1];
            }
            float cn = 0.0f, vn = 0.0f;
            if (col_ok && m < rows_here) {
                cn = cp[(size_t)(y0 + m) * a.pitch];
                vn = vp[(size_t)(y0 + m) * a.pitch];
            }
            cw[KS - 1] = cn;
            vw[KS - 1] = vn;
            const float* ur = sU + m * UWD + lane;
            const float* dr = sD + m * UWD + lane;
            float in[KS], dn[KS];
#pragma unroll
            for (int b = 0; b < KS; ++b) {
                in[b] = ur[2 * R - b];
                dn[b] = dr[2 * R - b];
            }
#pragma unroll
            for (int p = 0; p < KS; ++p)
#pragma unroll
                for (int q = 0; q < KS; ++q)
                    acc[p][q] = fmaf(cw[p], in[q], fmaf(-vw[p], dn[q], acc[p][q]));
        }
        // reduce over the 32 lanes (columns) through shared memory
#pragma unroll
        for (int p = 0; p < KS; ++p)
#pragma unroll
            for (int q = 0; q < KS; ++q) sRed[warp][p * KS + q][lane] = acc[p][q];
        __syncwarp();
        for (int e = lane; e < KS * KS; e += 32) {
            float s = 0.0f;
#pragma unroll 8
            for (int l = 0; l < 32; ++l) s += sRed[warp][e][l];
            a.part_k[((size_t)cta * a.nfilt + fi) * (KS * KS) + e] = s;
        }
        __syncwarp();
    }
}

// Fixed-order sums of the per-tile partials into the gradients of one stage.
// grid ceil(nparam / 256): thread e sums parameter e over all partial rows.
__global__ void __launch_bounds__(256) bwd_reduce(const float* __restrict__ part, int nrows,
                                                  int nparam, float* __restrict__ out)
{
    const int e = blockIdx.x * 256 + threadIdx.x;
    if (e >= nparam) return;
    float s = 0.0f;
    for (int r = 0; r < nrows; ++r) s += part[(size_t)r * nparam + e];
    out[e] = s;
}

}  // namespace tnrd
