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
#include <type_traits>
#include "args.cuh"
#include "fused_fwd.cuh"   // shfl_rel / gather_row

namespace tnrd {

// grid (prep_blocks, N), 256 threads.  Per pixel, with s = du_t/du~ and psi the
// explicit data term's reaction (zero for the prox), writes d = s e, for the
// explicit data terms also the identity-path cotangent d_id = (1 - psi'(u)) d,
// and sums e du_t/dlam per block:
//   dterm 0: s = y, du_t/dlam = x (Eqs. derv2, derv4; from u_t as above);
//   dterm 1: s = 1, psi = lam (u - f), psi' = lam, du_t/dlam = -(u - f);
//   dterm 2: s = [u_t > c] (u_t = max(u~, c); derivative 0 at the floor),
//            psi = lam (u - f)(u + f) / u^3, psi' = lam (3 f^2 - u^2) / u^4,
//            du_t/dlam = -s psi / lam.
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
        if (a.dterm == 0) {
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
        } else {
            const float up = a.u_prev[o];
            float dv, dpsi, dlam;
            if (a.dterm == 1) {
                dv = e;
                dpsi = lam;
                dlam = -(up - fv);
            } else {
                dv = (u > a.proj_c) ? e : 0.0f;
                const float u2 = up * up;
                dpsi = lam * (3.0f * fv * fv - u2) / (u2 * u2);
                dlam = -((up - fv) * (up + fv)) / (u2 * up);
            }
            a.d[o] = dv;
            a.d_id[o] = (1.0f - dpsi) * dv;
            xe = dlam * dv;
        }
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

// One group of KS walk steps of bwd_zb starting at step m0.  Step m takes
// u and d row y0 - R + m (shared-memory rows m); z and b of image row
// y0 - 2R + m complete there (rolling accumulators, slot (step + a) mod KS).
// FIRST: the group of steps 0 .. KS-1; updates of rows completing before step
// 2R (above the tile) are left out.
template <int KS, int UP, bool FIRST = false>
__device__ __forceinline__ void zb_group(
    const float2* __restrict__ udrow, const float (&kr)[KS][KS],
    float (&za)[KS], float (&ba)[KS], int m0, int y0, int H, int TH, bool col_in, int lane,
    const float* __restrict__ wp, float* __restrict__ hist_lane, const RbfConst& rc,
    float* __restrict__ cpl_col, float* __restrict__ vpl_col, int pitch)
{
    constexpr int R = KS / 2;
#pragma unroll
    for (int mm = 0; mm < KS; ++mm) {
        const int m = m0 + mm;
        const float2* udr = udrow + m * UP;
        float in[KS], dn[KS];
#pragma unroll
        for (int b = 0; b < KS; ++b) {
            const float2 ud = udr[2 * R - b];   // (u, d) interleaved: one 64-bit load
            in[b] = ud.x;
            dn[b] = ud.y;
        }
#pragma unroll
        for (int b = 0; b < KS; ++b) {
#pragma unroll
            for (int q = 0; q < KS; ++q) {
                if (FIRST && mm + q < 2 * R) continue;
                const int s = (mm + q) % KS;
                za[s] = fmaf(kr[q][b], in[b], za[s]);
                ba[s] = fmaf(kr[q][b], dn[b], ba[s]);
            }
        }
        const float z = za[mm], bv = ba[mm];
        za[mm] = 0.0f;
        ba[mm] = 0.0f;
        const int zr = m - 2 * R;            // tile row of the completed z
        const int zi = y0 + zr;
        if (col_in && zr >= 0 && zr < TH && zi < H) {
            float v, dphi;
            RbfWin2 win;
            rbf_phi_dphi_w(z, wp, rc, v, dphi, win);
            const float c = -dphi * bv;
            cpl_col[(size_t)zi * pitch] = c;
            vpl_col[(size_t)zi * pitch] = v;
            // dL/dw_j += -b G_j(z) for the window bins j = j0 - RBF_WIN + nn,
            // stored at histogram row j + 2 RBF_WIN = win.row + nn
            float g = -bv * win.pre;
            float* hp = hist_lane + win.row * 32;
#pragma unroll
            for (int nn = 0; nn <= 2 * RBF_WIN; ++nn) {
                const int md = nn - RBF_WIN;
                hp[nn * 32] = fmaf(g, rc.E[md < 0 ? -md : md], hp[nn * 32]);
                g *= win.q;
            }
        }
    }
}

// grid (zb_tiles_x * zb_tiles_y, N, S), ZbCfg::NTHREADS threads, 2 CTAs per SM;
// the S CTAs of a tile share out each warp's filters (fl = blockIdx.z, + S, ...).
template <int KS, int NK, int TH>
__global__ void __launch_bounds__(ZbCfg<KS, NK, TH>::NTHREADS, 2)
bwd_zb(const __grid_constant__ BwdArgs a)
{
    using C = ZbCfg<KS, NK, TH>;
    constexpr int R = C::R;
    extern __shared__ __align__(16) float smem[];
    float2* sUD = reinterpret_cast<float2*>(smem);   // (u_{t-1}, d) interleaved
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* myHist = smem + 2 * C::U_FL + warp * C::PW_FL;
    float* myK = myHist + C::HIST_FL;
    float* myWp = myK + C::KPAD;

    const int n = blockIdx.y;
    const int ty = blockIdx.x / a.zb_tiles_x, tx = blockIdx.x - ty * a.zb_tiles_x;
    const int H = a.H, W = a.W;
    const int y0 = ty * TH, x0 = tx * 32;
    const size_t ioff = (size_t)n * a.img_stride;

    for (int idx = threadIdx.x; idx < C::U_FL; idx += C::NTHREADS) {
        const int i = idx / C::UW, j = idx - i * C::UW;
        const int yy = sym_idx(y0 - R + i, H), xx = sym_idx(x0 - R + j, W);
        const size_t o = ioff + (size_t)yy * a.pitch + xx;
        sUD[idx] = make_float2(a.u_prev[o], a.d[o]);
    }
    for (int e = lane; e < C::HIST_FL; e += 32) myHist[e] = 0.0f;
    for (int e = lane; e < C::WPADN; e += 32) myWp[e] = 0.0f;
    __syncthreads();

    const int x = x0 + lane;
    const bool col_in = x < W;
    const float2* udrow = sUD + lane;
    const int cta = n * (a.zb_tiles_x * a.zb_tiles_y) + blockIdx.x;

#pragma unroll 1
    for (int fl = blockIdx.z; fl < C::FPW; fl += gridDim.z) {
        const int fi = warp * C::FPW + fl;
        for (int e = lane; e < KS * KS; e += 32) myK[e] = __ldg(a.k + fi * KS * KS + e);
        for (int e = lane; e < a.nrbf; e += 32) myWp[RBF_WPAD + e] = __ldg(a.w + fi * a.nrbf + e);
        __syncwarp();
        float kr[KS][KS];
#pragma unroll
        for (int p = 0; p < KS; ++p)
#pragma unroll
            for (int q = 0; q < KS; ++q) kr[p][q] = myK[p * KS + q];
        const size_t plane = ioff * (size_t)a.nfilt + (size_t)fi * a.img_stride;
        float* cpl_col = a.cpl + plane + (col_in ? x : 0);
        float* vpl_col = a.vpl + plane + (col_in ? x : 0);
        float za[KS], ba[KS];
#pragma unroll
        for (int s = 0; s < KS; ++s) za[s] = ba[s] = 0.0f;
        zb_group<KS, C::UP, true>(udrow, kr, za, ba, 0, y0, H, TH, col_in, lane, myWp,
                                  myHist + lane, a.rc, cpl_col, vpl_col, a.pitch);
#pragma unroll 1
        for (int g = 1; g < C::GROUPS; ++g)
            zb_group<KS, C::UP>(udrow, kr, za, ba, g * KS, y0, H, TH, col_in, lane, myWp,
                                myHist + lane, a.rc, cpl_col, vpl_col, a.pitch);
        __syncwarp();
        // per-tile dL/dw_i: sum the lanes' bins (skewed reads avoid bank conflicts)
        for (int j = lane; j < a.nrbf; j += 32) {
            const float* hb = myHist + (j + 2 * RBF_WIN) * 32;
            float s = 0.0f;
#pragma unroll 8
            for (int l = 0; l < 32; ++l) s += hb[(l + j) & 31];
            a.part_w[((size_t)cta * a.nfilt + fi) * a.nrbf + j] = s;
        }
        __syncwarp();
        for (int e = lane; e < C::HIST_FL; e += 32) myHist[e] = 0.0f;
        __syncwarp();
    }
}

// One group of KS walk steps of bwd_adj starting at step m0.  Step m takes c
// row hy0 - R + m (cv[mm], this lane's column); h row hy0 - 2R + m completes
// there and is added to the warp's buffer at hrow[m * 32].  FIRST: the group
// of steps 0 .. KS-1, where kernel rows a > step reach only h rows above the
// first stored one and are left out.
template <int KS, bool FIRST = false>
__device__ __forceinline__ void adj_group(const float (&cv)[KS], float* __restrict__ hrow,
                                          const float (&kr)[KS][KS], float (&ha)[KS], int m0,
                                          int mh_lo, int mh_hi, int lane)
{
    constexpr int R = KS / 2;
#pragma unroll
    for (int mm = 0; mm < KS; ++mm) {
        const int m = m0 + mm;
        float cw[KS];
        gather_row<KS, 0, true>(cw, cv[mm], lane);   // cw[b] = c(row, x - R + b)
        // h(q, x) += k[a][b] c(q - R + a, x - R + b): this c row feeds h rows
        // q = row + R - a, slot (step + 2R - a) mod KS; slot mm completes (a = 2R)
#pragma unroll
        for (int b = 0; b < KS; ++b) {
#pragma unroll
            for (int q = 0; q < KS; ++q) {
                if (FIRST && q > mm) continue;
                const int s = (mm + 2 * R - q) % KS;
                ha[s] = fmaf(kr[q][b], cw[b], ha[s]);
            }
        }
        if (m >= mh_lo && m < mh_hi) hrow[m * 32] += ha[mm];
        ha[mm] = 0.0f;
    }
}

// grid (tiles_x * tiles_y, N), AdjCfg::NTHREADS threads.  Tiles, own regions
// and the border fold as in the fused forward stage.
template <int KS, int NK, int TH>
__global__ void __launch_bounds__(AdjCfg<KS, NK, TH>::NTHREADS, 2)
bwd_adj(const __grid_constant__ BwdArgs a)
{
    using C = AdjCfg<KS, NK, TH>;
    constexpr int R = C::R;
    constexpr int TW = C::TW;
    extern __shared__ __align__(16) float smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* myH = smem + warp * C::H_FL;   // h rows y0 - R .. y0 + TH + R - 1

    const int n = blockIdx.y;
    const int ty = blockIdx.x / a.tiles_x, tx = blockIdx.x - ty * a.tiles_x;
    const int H = a.H, W = a.W;
    const int y0 = tile_origin(ty, TH, H), x0 = tile_origin(tx, TW, W);
    const bool ext = (ty == 0) || (ty == a.tiles_y - 1);
    const bool border = ext || (tx == 0) || (tx == a.tiles_x - 1);
    const size_t ioff = (size_t)n * a.img_stride;
    for (int e = lane; e < C::H_FL; e += 32) myH[e] = 0.0f;

    const int hy0 = ext ? y0 - R : y0;           // first h row walked
    const int nh = ext ? TH + 2 * R : TH;
    const int nsteps = nh + 2 * R;               // c rows hy0 - R .. hy0 + nh + R - 1
    const int ngroups = (nsteps + KS - 1) / KS;
    const int xcol = x0 - R + lane;
    const bool col_in = (unsigned)xcol < (unsigned)W;
    // h row of step m is hy0 - 2R + m: buffer row hy0 - 2R + m - (y0 - R)
    float* hrow = myH + (hy0 - R - y0) * 32 + lane;

#pragma unroll 1
    for (int fl = 0; fl < C::FPW; ++fl) {
        const int fi = warp * C::FPW + fl;
        float kr[KS][KS];
#pragma unroll
        for (int p = 0; p < KS; ++p)
#pragma unroll
            for (int q = 0; q < KS; ++q) kr[p][q] = __ldg(a.k + (fi * KS + p) * KS + q);
        const float* cpl = a.cpl + ioff * (size_t)a.nfilt + (size_t)fi * a.img_stride +
                           (col_in ? xcol : 0);
        float ha[KS];
#pragma unroll
        for (int s = 0; s < KS; ++s) ha[s] = 0.0f;
        // c rows of group g; the next group's loads are issued before the
        // current group's arithmetic
        auto load_group = [&](int g, float (&cv)[KS]) {
#pragma unroll
            for (int mm = 0; mm < KS; ++mm) {
                const int m = g * KS + mm, r = hy0 - R + m;
                cv[mm] = (col_in && (unsigned)r < (unsigned)H && m < nsteps)
                             ? __ldcg(cpl + (size_t)r * a.pitch) : 0.0f;
            }
        };
        float cv[KS];
        load_group(0, cv);
        {
            float cn[KS];
            load_group(1, cn);
            adj_group<KS, true>(cv, hrow, kr, ha, 0, 2 * R, nsteps, lane);
#pragma unroll
            for (int mm = 0; mm < KS; ++mm) cv[mm] = cn[mm];
        }
#pragma unroll 1
        for (int g = 1; g < ngroups; ++g) {
            float cn[KS];
            load_group(g + 1, cn);
            adj_group<KS>(cv, hrow, kr, ha, g * KS, 2 * R, nsteps, lane);
#pragma unroll
            for (int mm = 0; mm < KS; ++mm) cv[mm] = cn[mm];
        }
    }
    __syncthreads();

    // e_{t-1} = d + fold(sum over warps of h)
    const int wy0 = tile_split(ty, TH, H, a.tiles_y, R), wy1 = tile_split(ty + 1, TH, H, a.tiles_y, R);
    const int wx0 = tile_split(tx, TW, W, a.tiles_x, R), wx1 = tile_split(tx + 1, TW, W, a.tiles_x, R);
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
                for (int wq = 0; wq < C::NWARP; ++wq) hs += smem[wq * C::H_FL + hi * 32 + hj];
                g += hs;
            }
        }
        const size_t o = ioff + (size_t)qy * a.pitch + qx;
        a.e_prev[o] = a.d_id[o] + g;
    }
}

// grid (dk_tiles_x * dk_tiles_y, N, S), 4 warps (the S CTAs of a tile share out
// each warp's filters: fl = blockIdx.z, + S, ...); tiles of 32 columns x TH rows
// (TH + 2R a multiple of KS).  Per warp and filter: lane = pixel column, walk
// over the u/d rows of the tile plus R above and below; step m takes u/d row
// y0 - R + m and the 2R+1 c and v rows y0 + m - 2R + a (a = 0..2R) that meet it:
//   acc[a][b] += c(y0 + m - 2R + a) u(y0 - R + m, x + R - b)
//              - v(y0 + m - 2R + a) d(y0 - R + m, x + R - b)
// (u, d symmetric-padded); rows and columns outside the tile or the image carry
// c = v = 0, so every pixel's product is counted by exactly one tile.  The c
// and v rows of a group of KS steps sit in registers (cur), with those of the
// previous group (prev); the next group's loads are issued one group ahead.
template <int KS, int NK, int TH>
__global__ void __launch_bounds__(128) bwd_dk(const __grid_constant__ BwdArgs a)
{
    constexpr int R = KS / 2;
    constexpr int NW = 4;
    constexpr int FPW = NK / NW;
    static_assert(NK % NW == 0, "");
    constexpr int STEPS = TH + 2 * R;
    static_assert(STEPS % KS == 0, "the walk must end on a whole group");
    constexpr int NG = STEPS / KS;
    constexpr int UWD = 32 + 2 * R;
    __shared__ float2 sUD[STEPS * UWD];   // (u_{t-1}, d) interleaved
    __shared__ float sRed[NW][KS * KS][33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = blockIdx.y;
    const int ty = blockIdx.x / a.dk_tiles_x, tx = blockIdx.x - ty * a.dk_tiles_x;
    const int y0 = ty * TH, x0 = tx * 32;
    const int H = a.H, W = a.W;
    const size_t ioff = (size_t)n * a.img_stride;
    for (int idx = threadIdx.x; idx < STEPS * UWD; idx += 128) {
        const int i = idx / UWD, j = idx - i * UWD;
        const int yy = sym_idx(y0 - R + i, H), xx = sym_idx(x0 - R + j, W);
        const size_t o = ioff + (size_t)yy * a.pitch + xx;
        sUD[idx] = make_float2(a.u_prev[o], a.d[o]);
    }
    __syncthreads();
    const int x = x0 + lane;
    const bool col_ok = x < W;
    const int rows_here = min(TH, H - y0);
    const int cta = n * (a.dk_tiles_x * a.dk_tiles_y) + blockIdx.x;
#pragma unroll 1
    for (int fl = blockIdx.z; fl < FPW; fl += gridDim.z) {
        const int fi = warp * FPW + fl;
        const size_t plane = ioff * (size_t)a.nfilt + (size_t)fi * a.img_stride;
        const float* cp = a.cpl + plane + (size_t)y0 * a.pitch + (col_ok ? x : 0);
        const float* vp = a.vpl + plane + (size_t)y0 * a.pitch + (col_ok ? x : 0);
        auto load_group = [&](int g, float (&cg)[KS], float (&vg)[KS]) {
#pragma unroll
            for (int mm = 0; mm < KS; ++mm) {
                const int r = g * KS + mm;   // tile row
                const bool ok = col_ok && r < rows_here;
                cg[mm] = ok ? __ldcg(cp + (size_t)r * a.pitch) : 0.0f;
                vg[mm] = ok ? __ldcg(vp + (size_t)r * a.pitch) : 0.0f;
            }
        };
        float acc[KS][KS];
#pragma unroll
        for (int p = 0; p < KS; ++p)
#pragma unroll
            for (int q = 0; q < KS; ++q) acc[p][q] = 0.0f;
        float cprev[KS], vprev[KS], ccur[KS], vcur[KS];
#pragma unroll
        for (int s = 0; s < KS; ++s) cprev[s] = vprev[s] = 0.0f;
        load_group(0, ccur, vcur);
        // one group of KS steps; in the first group the slots of c/v rows above
        // the tile, in the last those below it, are zero and left out
        auto group = [&](int g, auto first_tag, auto last_tag) {
            constexpr bool FIRST = decltype(first_tag)::value, LAST = decltype(last_tag)::value;
            float cnext[KS], vnext[KS];
            load_group(g + 1, cnext, vnext);
#pragma unroll
            for (int mm = 0; mm < KS; ++mm) {
                const float2* udr = sUD + (g * KS + mm) * UWD + lane;
                float in[KS], dn[KS];
#pragma unroll
                for (int b = 0; b < KS; ++b) {
                    const float2 ud = udr[2 * R - b];
                    in[b] = ud.x;
                    dn[b] = ud.y;
                }
#pragma unroll
                for (int p = 0; p < KS; ++p) {
                    // c/v row m - 2R + p: slot mm - 2R + p of this group or the last
                    const int sl = mm - 2 * R + p;
                    if (FIRST && sl < 0) continue;         // rows above the tile
                    if (LAST && sl >= KS - 2 * R) continue; // rows at or below y0 + TH
                    const float cv = sl >= 0 ? ccur[sl] : cprev[sl + KS];
                    const float vv = sl >= 0 ? vcur[sl] : vprev[sl + KS];
#pragma unroll
                    for (int q = 0; q < KS; ++q)
                        acc[p][q] = fmaf(cv, in[q], fmaf(-vv, dn[q], acc[p][q]));
                }
            }
#pragma unroll
            for (int s = 0; s < KS; ++s) {
                cprev[s] = ccur[s];
                vprev[s] = vcur[s];
                ccur[s] = cnext[s];
                vcur[s] = vnext[s];
            }
        };
        using T_ = std::true_type;
        using F_ = std::false_type;
        static_assert(NG >= 2, "the walk has a first and a last group");
        group(0, T_{}, F_{});
#pragma unroll 1
        for (int g = 1; g < NG - 1; ++g) group(g, F_{}, F_{});
        group(NG - 1, F_{}, T_{});
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
// grid (blocks, 3), 512 threads; blockIdx.y picks the partial set.  Sets of
// 32 or more parameters: block x takes parameters 32x .. 32x + 31 (lane), and
// warp w sums rows w, w + 16, ...; the 16 warp sums are then added in warp
// order.  Smaller sets: block x takes parameter x, thread i sums rows i,
// i + 512, ..., followed by a fixed pairwise tree.  Either way the order of
// every addition is fixed by the launch shape alone.
constexpr int RED_THREADS = 512;
__global__ void __launch_bounds__(RED_THREADS) bwd_reduce(const __grid_constant__ RedArgs a)
{
    const RedSet g = a.s[blockIdx.y];
    __shared__ float red[RED_THREADS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NWR = RED_THREADS / 32;
    if (g.nparam >= 32) {
        const int e = blockIdx.x * 32 + lane;
        if (blockIdx.x * 32 >= g.nparam) return;
        float s = 0.0f;
        if (e < g.nparam) {
#pragma unroll 4
            for (int r = warp; r < g.nrows; r += NWR) s += g.part[(size_t)r * g.nparam + e];
        }
        red[warp * 32 + lane] = s;
        __syncthreads();
        if (warp == 0 && e < g.nparam) {
            float t = 0.0f;
#pragma unroll
            for (int w = 0; w < NWR; ++w) t += red[w * 32 + lane];
            g.out[e] = t;
        }
    } else {
        const int e = blockIdx.x;
        if (e >= g.nparam) return;
        float s = 0.0f;
#pragma unroll 4
        for (int r = tid; r < g.nrows; r += RED_THREADS) s += g.part[(size_t)r * g.nparam + e];
        red[tid] = s;
        for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
            __syncthreads();
            if (tid < w) red[tid] += red[tid + w];
        }
        if (tid == 0) g.out[e] = red[0];
    }
}

}  // namespace tnrd
