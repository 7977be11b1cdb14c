// Tensor-core adjoint of the backward stage (Sec. 3.2, Eq. derv1-1):
//   dL/du_{t-1} = d + fold(sum_i K_i^T c_i)
// as the forward stage's adjoint: Y[p][tap] = sum_i c_i(p) k_i[tap] is one
// tcgen05 GEMM per group of 128 positions (M = 128, N = 64 taps, K = the
// filters), h(q) = sum_tap Y[q + off(tap)][tap] is scattered on the CUDA cores
// into the warpgroup's h buffer in kernel-row phases, and the epilogue folds the
// border (the exact transpose of the symmetric-padded convolution) and adds d.
//
// The c planes come from bwd_zb in HBM; each thread loads its position's c
// values, 16 filters per round, one round ahead, and writes them as the A
// operand (TF32, or X3: TF32 high part and TF32 remainder, three MMAs per
// product -- lo*hi + hi*lo + hi*hi -- for FP32 accuracy).  Tiles are those of
// the forward's tensor-core stage, (16 NB - 2R) x (32 - 2R) outputs over a
// region of 16 NB x 32 positions; a group is 4 rows x 32 columns of it, warp w
// one row, lane l one column, so a warp's loads are 128 contiguous bytes.  The
// scatter sums each kernel row within the warp first: lane l adds
// Y[row][l - R + b][tap (a, b)] over b (shuffles), the one h element of column
// l + R the row feeds through kernel row a, then one read-modify-write per
// kernel row (the warps' h rows are disjoint within a phase; a warpgroup barrier
// between phases).  One persistent CTA per SM of NWG warpgroups; the filter
// matrix is staged once per CTA.  Every wait on the tensor core is bounded; a
// timeout sets the status word and the CTA still frees its TMEM.
#include <algorithm>

#include "args.cuh"
#include "launch.h"
#include "tc_bwd_cfg.cuh"
#include "tc_ptx.cuh"

namespace tnrd {


template <int KS, int NK, int NB, bool X3>
__global__ void __launch_bounds__(TcAdjCfg<KS, NK, NB, X3>::NTHREADS, 1)
tc_bwd_adj(const __grid_constant__ BwdArgs a, int n_img, int tiles_x, int tiles_y, int* err)
{
    using C = TcAdjCfg<KS, NK, NB, X3>;
    constexpr int R = C::R, TW = C::TW, TH = C::TH;
    constexpr long long WAIT_LIMIT = 1ll << 31;          // SM cycles, about one second
    constexpr uint32_t ID_Y = tc::idesc(tc::FMT_TF32, 128, C::NT);
    constexpr uint32_t LBO_KM = (C::NT / 8) * 128;
    constexpr int NG = C::ZR / 4;                        // groups of 4 position rows
    constexpr int NY8 = (KS * KS + 7) / 8;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, wg = tid >> 7, wt = tid & 127, warp = wt >> 5, lane = wt & 31;
    const int bar = 1 + wg;
    unsigned char* wgs = smem + C::OFF_WG + (size_t)wg * C::WG_BYTES;
    float* sV = reinterpret_cast<float*>(wgs + C::WG_V);
    float* sH = reinterpret_cast<float*>(wgs + C::WG_H);
    uint64_t* mb = reinterpret_cast<uint64_t*>(wgs + C::WG_MISC);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + C::OFF_TMEM);

    // filter matrix B[tap][i] = k_i[tap], core matrices [i/4][tap/8][tap%8][i%4]
    // (X3: the TF32 remainders KM_BYTES on)
    {
        float* sKm = reinterpret_cast<float*>(smem + C::OFF_KM);
        for (int e = tid; e < C::NT * C::NKP; e += C::NTHREADS) {
            const int tap = e / C::NKP, i = e - tap * C::NKP;
            const float v = (tap < KS * KS && i < NK) ? __ldg(a.k + i * KS * KS + tap) : 0.0f;
            const int o = ((i / 4) * (C::NT / 8) + tap / 8) * 32 + (tap % 8) * 4 + (i % 4);
            const float hi = tc::to_tf32(v);
            sKm[o] = hi;
            if constexpr (X3) sKm[C::KM_BYTES / 4 + o] = tc::to_tf32(v - hi);
        }
    }
    if (wt == 0) tc::mbar_init(mb, 1);
    tc::fence_async_smem();
    if (tid < 32) tc::tmem_alloc(tslot, C::TMEM_COLS);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t ybuf = tbase + (uint32_t)(128 * wg);
    const uint32_t sKm = tc::smem_u32(smem + C::OFF_KM);
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const int g = wt >> 3, mp = wt & 7;

    uint32_t ph = 0;       // parity of the next phase of mb
    bool pend = false;     // a commit on mb not yet waited for
    int ok = 1;
    auto wait_mma = [&]() {
        const bool got = ok && tc::mbar_wait(mb, ph, WAIT_LIMIT);
        if (got) {
            ph ^= 1u;
            pend = false;
        }
        ok = tc::wg_and(bar, got);
    };

    const int H = a.H, W = a.W, P = a.pitch;
    const long long plane = a.img_stride;
    const int tpi = tiles_x * tiles_y, nt = n_img * tpi;
    const int per = (nt + (int)gridDim.x - 1) / (int)gridDim.x;
    const int c0 = min(nt, (int)blockIdx.x * per), c1 = min(nt, c0 + per);
#pragma unroll 1
    for (int s = c0 + wg; s < c1 && ok; s += C::NWG) {
        const int n = s / tpi, ti = s - n * tpi, ty = ti / tiles_x, tx = ti - ty * tiles_x;
        const int y0 = tile_origin(ty, TH, H), x0 = tile_origin(tx, TW, W);
        const bool border = (ty == 0) || (ty == tiles_y - 1) || (tx == 0) || (tx == tiles_x - 1);
        const float* cimg = a.cpl + (size_t)n * plane * a.nfilt;
        tc::wg_sync(bar);   // the previous tile's epilogue has read h
        for (int e = wt; e < C::HROWS * C::HPITCH; e += 128) sH[e] = 0.0f;

        // c values of round rr of group gi at this thread's position (0 outside
        // the image and for filters beyond NK)
        auto load_round = [&](int gi, int rr, float (&c)[16]) {
            const int yy = y0 - R + 4 * gi + warp, xx = x0 - R + lane;
            const bool in = (unsigned)yy < (unsigned)H && (unsigned)xx < (unsigned)W;
            const float* p = cimg + (in ? (size_t)yy * P + xx : 0);
#pragma unroll
            for (int f = 0; f < 16; ++f) {
                const int i = 16 * rr + f;
                c[f] = (in && i < NK) ? __ldcg(p + (size_t)i * plane) : 0.0f;
            }
        };
        float cur[16];
        load_round(0, 0, cur);
#pragma unroll 1
        for (int gi = 0; gi < NG; ++gi) {
#pragma unroll 1
            for (int rr = 0; rr < C::NR; ++rr) {
                float nxt[16];
                if (rr + 1 < C::NR) load_round(gi, rr + 1, nxt);
                else if (gi + 1 < NG) load_round(gi + 1, 0, nxt);
                // the previous round's MMAs have read the V slot
                if (rr > 0) wait_mma();
                if (ok) {
                    // A layout [filter/4][g][mp][filter%4], high parts then low parts
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        if (16 * rr + 4 * q4 >= C::NKP) continue;
                        float hi[4], lo[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            hi[k] = tc::to_tf32(cur[4 * q4 + k]);
                            lo[k] = tc::to_tf32(cur[4 * q4 + k] - hi[k]);
                        }
                        float* dst = sV + (q4 * 16 + g) * 32 + mp * 4;
                        *reinterpret_cast<float4*>(dst) = make_float4(hi[0], hi[1], hi[2], hi[3]);
                        if constexpr (X3)
                            *reinterpret_cast<float4*>(dst + C::VLO / 4) = make_float4(lo[0], lo[1], lo[2], lo[3]);
                    }
                }
                tc::fence_async_smem();
                tc::fence_before();
                tc::wg_sync(bar);
                tc::fence_after();
                if (ok && wt == 0) {
                    // Y += C_rr Kmat_rr, per 8 filters (X3: c_lo k_hi + c_hi k_lo + c_hi k_hi)
                    const int nks = min(2, (C::NKP - 16 * rr) / 8);
                    for (int s8 = 0; s8 < nks; ++s8) {
                        const uint32_t va = tc::smem_u32(sV) + (uint32_t)(s8 * 4096);
                        const uint32_t kh = sKm + (uint32_t)((2 * rr + s8) * 2 * LBO_KM);
                        const uint64_t dvh = tc::sdesc(va, 16 * 128, 128);
                        const uint64_t dkh = tc::sdesc(kh, LBO_KM, 128);
                        const uint32_t acc0 = (rr > 0 || s8 > 0) ? 1u : 0u;
                        if constexpr (X3) {
                            tc::mma_tf32(ybuf, tc::sdesc(va + (uint32_t)C::VLO, 16 * 128, 128), dkh, ID_Y, acc0);
                            tc::mma_tf32(ybuf, dvh, tc::sdesc(kh + (uint32_t)C::KM_BYTES, LBO_KM, 128), ID_Y, 1);
                            tc::mma_tf32(ybuf, dvh, dkh, ID_Y, 1);
                        } else {
                            tc::mma_tf32(ybuf, dvh, dkh, ID_Y, acc0);
                        }
                    }
                    tc::commit(mb);
                }
                if (ok) pend = true;
#pragma unroll
                for (int f = 0; f < 16; ++f) cur[f] = nxt[f];
            }
            wait_mma();
            tc::fence_after();
            uint32_t yr[NY8][8];
            if (ok) {
#pragma unroll
                for (int c = 0; c < NY8; ++c) tc::tmem_ld8_nowait(ybuf + lane_base + 8 * c, yr[c]);
                tc::tmem_wait_ld();
            }
            tc::fence_before();
            tc::wg_sync(bar);
            tc::fence_after();
            // h(p - off(tap)) += Y[p][tap]: h index (prow + 2R - a, pcol + 2R - b) for
            // the position (prow, pcol) of the region; lane l owns h column l + R,
            // fed by the positions l - R + b of its warp's row (outside the 32
            // columns: outside the image, or h columns no output reads)
            if (ok) {
                const int hrow0 = 4 * gi + warp + 2 * R;
#pragma unroll
                for (int ka = 0; ka < KS; ++ka) {
                    if (ka > 0) tc::wg_sync(bar);
                    float acc = 0.0f;
#pragma unroll
                    for (int b = 0; b < KS; ++b) {
                        const int t = ka * KS + b;
                        const int src = lane - R + b;
                        const float v = __shfl_sync(0xffffffffu, __uint_as_float(yr[t / 8][t % 8]), src & 31);
                        acc += (src >= 0 && src < 32) ? v : 0.0f;
                    }
                    sH[(hrow0 - ka) * C::HPITCH + lane + R] += acc;
                }
            }
        }

        // ---- e_{t-1} = d + fold(h) over the pixels this tile owns ----
        tc::wg_sync(bar);
        if (ok) {
            const int wy0 = tile_split(ty, TH, H, tiles_y, R), wy1 = tile_split(ty + 1, TH, H, tiles_y, R);
            const int wx0 = tile_split(tx, TW, W, tiles_x, R), wx1 = tile_split(tx + 1, TW, W, tiles_x, R);
            const size_t ioff = (size_t)n * plane;
            for (int idx = wt; idx < TH * TW; idx += 128) {
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
                float gsum = 0.0f;
                for (int pp = 0; pp < nsy; ++pp)
                    for (int q = 0; q < nsx; ++q)
                        gsum += sH[(sy[pp] - (y0 - 2 * R)) * C::HPITCH + sx[q] - (x0 - 2 * R)];
                const size_t o = ioff + (size_t)qy * P + qx;
                a.e_prev[o] = a.d_id[o] + gsum;
            }
        }
    }
    if (!ok) {
        if (pend) tc::mbar_wait(mb, ph, WAIT_LIMIT);
        if (wt == 0) atomicExch(err, 4);
    }
    tc::fence_before();
    __syncthreads();
    if (tid < 32) tc::tmem_dealloc(tbase, C::TMEM_COLS);
}

// Filter gradient of the backward stage (Sec. 3.2, Eq. derv1-1 differentiated
// in k), per tile of 32 columns x TPR rows of pixels p:
//   dL/dk_i[a][b] += sum_p c_i(p) u(p + (R - a, R - b)) - v_i(p) d(p + (R - a, R - b))
// (u = u_{t-1}, d as in bwd_prep, both symmetric-padded; c = v = 0 outside the
// image) as one tcgen05 GEMM with the pixels as K: D[tap row][filter] (M = 128,
// N = the filters padded to 16, FP32 in TMEM), K = 8 pixels per MMA.
//   A (taps x pixels) needs no im2col: each u row is kept as its four column
//   residues interleaved in 16-byte chunks, IL[q][r][j] = u(x0 - R + 4q + r + j),
//   so for the 4 pixels of quad q0 the 8 tap rows b'' = 0..7 of one kernel row
//   (tap column b = KS - 1 - b'') are the chunks IL[q0 + b''/4][b'' % 4], 16 bytes
//   apart: one K-major core matrix as the MMA reads it; the next 4 pixels start
//   64 bytes on, the next kernel row (a = KS - 1 - a'') one IL row on.  Rows
//   a'', b'' >= KS of the 128 are padding whose D rows are not stored.
//   B (filters x pixels) is one pixel row of c (and, for the second GEMM, of -v)
//   staged as [quad][filter][4 pixels] (quad pitch padded by 16 bytes: the
//   staging stores of a warp fall in distinct banks).
// X3: every operand as TF32 high part and TF32 remainder, three MMAs per
// product.  Per pixel row one barrier: the row's staging buffer (NBUF, used in
// turn) is written -- the next row's values already loaded into registers --
// and one thread issues the row's MMAs; the buffer is written again NBUF rows
// later, once those MMAs have completed.  One buffer: a second one halves the
// CTAs per SM, and the kernel hides its load latency with CTAs, not buffers
// (measured: 226 against 214 us per launch on the 32 x 180^2 batch, TF32).
// At the end each thread reads its tap row of D and writes the tile's partial
// dL/dk, which bwd_reduce sums over the tiles in a fixed order.

int tc_dk_tiles(int H, int W) { return ((W + 31) / 32) * ((H + 15) / 16); }

template <int KS, int NK, bool X3>
__global__ void __launch_bounds__(128)
tc_bwd_dk(const __grid_constant__ BwdArgs a, int tiles_x, int* err)
{
    using C = TcDkCfg<KS, NK, X3>;
    constexpr int R = C::R, TPR = C::TPR, NP = C::NP;
    constexpr long long WAIT_LIMIT = 1ll << 31;
    constexpr uint32_t ID = tc::idesc(tc::FMT_TF32, 128, NP);
    constexpr int FPT = (NK + 3) / 4;                    // filters per thread and pixel row
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint64_t* mb = reinterpret_cast<uint64_t*>(smem + C::OFF_MISC);   // one per staging buffer
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + C::OFF_MISC + 16);
    const int n = blockIdx.y, tile = blockIdx.x;
    const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const int y0 = ty * TPR, x0 = tx * 32;
    const int H = a.H, W = a.W, P = a.pitch;
    const size_t ioff = (size_t)n * a.img_stride;

    // interleaved residue rows of u and d (symmetric padding; rows past the
    // tile's last kernel row are read but only feed padding taps)
    {
        float* il = reinterpret_cast<float*>(smem);
        constexpr int NIL = C::ILR_REAL * C::NCOLQ * 16;
        for (int e = tid; e < NIL; e += 128) {
            const int ir = e / (C::NCOLQ * 16), rem = e - ir * (C::NCOLQ * 16);
            const int q = rem >> 4, r = (rem >> 2) & 3, j = rem & 3;
            const int yy = sym_idx(y0 - R + ir, H), xx = sym_idx(x0 - R + 4 * q + r + j, W);
            const size_t o = ioff + (size_t)yy * P + xx;
            const float uv = a.u_prev[o], dv = a.d[o];
            const float uh = tc::to_tf32(uv), dh = tc::to_tf32(dv);
            il[C::OFF_ILU / 4 + e] = uh;
            il[C::OFF_ILD / 4 + e] = dh;
            if constexpr (X3) {
                il[(C::OFF_ILU + C::IL_BYTES) / 4 + e] = tc::to_tf32(uv - uh);
                il[(C::OFF_ILD + C::IL_BYTES) / 4 + e] = tc::to_tf32(dv - dh);
            }
        }
        // padding filters of the staging stay zero
        if constexpr (NP > NK) {
            float* st = reinterpret_cast<float*>(smem + C::OFF_ST);
            for (int e = tid; e < 2 * C::NBUF * C::NSPL * 8 * (NP - NK) * 4; e += 128) {
                const int part = e / (8 * (NP - NK) * 4), rem = e - part * (8 * (NP - NK) * 4);
                const int q = rem / ((NP - NK) * 4), f = NK + (rem / 4) % (NP - NK), j = rem & 3;
                st[(part * C::STG_BYTES + (size_t)q * C::QB) / 4 + f * 4 + j] = 0.0f;
            }
        }
    }
    if (tid == 0)
        for (int b = 0; b < C::NBUF; ++b) tc::mbar_init(mb + b, 1);
    if (warp == 0) tc::tmem_alloc(tslot, C::TMEM_COLS);
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;

    // c and v of pixel row pr: lane = pixel column, filters warp, warp + 4, ...
    const int xx = x0 + lane;
    auto load_row = [&](int pr, float (&cr)[FPT], float (&vr)[FPT]) {
        const int yy = y0 + pr;
        const bool in = yy < H && xx < W;
        const size_t o = ioff * (size_t)a.nfilt + (in ? (size_t)yy * P + xx : 0);
#pragma unroll
        for (int k = 0; k < FPT; ++k) {
            const int f = warp + 4 * k;
            const bool v = in && f < NK;
            cr[k] = v ? __ldcg(a.cpl + o + (size_t)f * a.img_stride) : 0.0f;
            vr[k] = v ? __ldcg(a.vpl + o + (size_t)f * a.img_stride) : 0.0f;
        }
    };
    const uint32_t s_il_u = tc::smem_u32(smem + C::OFF_ILU), s_il_d = tc::smem_u32(smem + C::OFF_ILD);
    const uint32_t s_st = tc::smem_u32(smem + C::OFF_ST);
    uint32_t ph = 0;       // bit s: parity of the next phase of mb[s]
    uint32_t pend = 0;     // bit s: a commit on mb[s] not yet waited for
    int ok = 1;
    float cur_c[FPT], cur_v[FPT];
    load_row(0, cur_c, cur_v);
    const int rows = min(TPR, H - y0);
#pragma unroll 1
    for (int pr = 0; pr < rows; ++pr) {
        float nxt_c[FPT], nxt_v[FPT];
        if (pr + 1 < rows) load_row(pr + 1, nxt_c, nxt_v);
        const int sb = pr % C::NBUF;
        // the MMAs of row pr - NBUF have read this staging buffer
        bool mine = ok != 0;
        if (pr >= C::NBUF) {
            mine = ok && tc::mbar_wait(mb + sb, (ph >> sb) & 1u, WAIT_LIMIT);
            if (mine) {
                ph ^= 1u << sb;
                pend &= ~(1u << sb);
            }
        }
        if (mine) {
            float* st = reinterpret_cast<float*>(smem);
            const int q = lane >> 2, j = lane & 3;
            const size_t bufo = C::OFF_ST + sb * C::BUF_BYTES + (size_t)q * C::QB;
#pragma unroll
            for (int k = 0; k < FPT; ++k) {
                const int f = warp + 4 * k;
                if (f >= NK) continue;
                const size_t oc = bufo / 4 + f * 4 + j;
                const size_t ov = (bufo + C::NSPL * C::STG_BYTES) / 4 + f * 4 + j;
                const float ch = tc::to_tf32(cur_c[k]), vh = tc::to_tf32(-cur_v[k]);
                st[oc] = ch;
                st[ov] = vh;
                if constexpr (X3) {
                    st[oc + C::STG_BYTES / 4] = tc::to_tf32(cur_c[k] - ch);
                    st[ov + C::STG_BYTES / 4] = tc::to_tf32(-cur_v[k] - vh);
                }
            }
        }
        tc::fence_async_smem();
        tc::fence_before();
        ok = __syncthreads_and(mine);
        tc::fence_after();
        if (ok && tid == 0) {
            const uint32_t s_st_c = s_st + (uint32_t)(sb * C::BUF_BYTES);
            const uint32_t s_st_v = s_st_c + (uint32_t)(C::NSPL * C::STG_BYTES);
#pragma unroll
            for (int kc = 0; kc < 4; ++kc) {
                const uint32_t ao = (uint32_t)(pr * C::ILP + 2 * kc * 64);
                const uint32_t bo = (uint32_t)(2 * kc * C::QB);
                const bool first = pr == 0 && kc == 0;
                // u row terms with c, then d row terms with -v
#pragma unroll
                for (int term = 0; term < 2; ++term) {
                    const uint32_t A = (term ? s_il_d : s_il_u) + ao, B = (term ? s_st_v : s_st_c) + bo;
                    const uint64_t dah = tc::sdesc(A, 64, C::ILP), dbh = tc::sdesc(B, C::QB, 128);
                    const uint32_t acc0 = (first && term == 0) ? 0u : 1u;
                    if constexpr (X3) {
                        tc::mma_tf32(tmem, tc::sdesc(A + (uint32_t)C::IL_BYTES, 64, C::ILP), dbh, ID, acc0);
                        tc::mma_tf32(tmem, dah, tc::sdesc(B + (uint32_t)C::STG_BYTES, C::QB, 128), ID, 1);
                        tc::mma_tf32(tmem, dah, dbh, ID, 1);
                    } else {
                        tc::mma_tf32(tmem, dah, dbh, ID, acc0);
                    }
                }
            }
            tc::commit(mb + sb);
        }
        if (ok) pend |= 1u << sb;
        if (pr + 1 < rows) {
#pragma unroll
            for (int k = 0; k < FPT; ++k) {
                cur_c[k] = nxt_c[k];
                cur_v[k] = nxt_v[k];
            }
        }
    }
    // D complete (the last row's commit covers every earlier MMA): tap row
    // m = tid -> partial dL/dk of the tile
    {
        bool got = ok != 0;
        for (int i = 1; i <= C::NBUF && i <= rows; ++i) {   // the last rows' commits
            const int sb = (rows - i) % C::NBUF;
            got = got && tc::mbar_wait(mb + sb, (ph >> sb) & 1u, WAIT_LIMIT);
            if (got) {
                ph ^= 1u << sb;
                pend &= ~(1u << sb);
            }
        }
        ok = __syncthreads_and(got);
    }
    tc::fence_after();
    const int ai = tid >> 3, bi = tid & 7;   // kernel-row slot a'', column slot b''
    const size_t prow = (size_t)n * gridDim.x + tile;   // partial row: image n, tile
    float* part = a.part_k + prow * a.nfilt * (KS * KS);
    const int e = (KS - 1 - ai) * KS + (KS - 1 - bi);
    const bool store = ai < KS && bi < KS;
    if (ok) {
        const uint32_t lb = (uint32_t)(32 * warp) << 16;
#pragma unroll
        for (int c8 = 0; c8 < NP / 8; ++c8) {
            uint32_t v[8];
            tc::tmem_ld8_nowait(tmem + lb + 8 * c8, v);
            tc::tmem_wait_ld();
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int f = 8 * c8 + k;
                if (store && f < NK) part[(size_t)f * (KS * KS) + e] = __uint_as_float(v[k]);
            }
        }
    } else if (store) {
        // a wait gave up: the tile contributes nothing (the status word says so)
        for (int f = 0; f < NK; ++f) part[(size_t)f * (KS * KS) + e] = 0.0f;
    }
    if (!ok) {
        for (int b = 0; b < C::NBUF; ++b)
            if (pend & (1u << b)) tc::mbar_wait(mb + b, (ph >> b) & 1u, WAIT_LIMIT);
        if (tid == 0) atomicExch(err, 4);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, C::TMEM_COLS);
}

namespace {

int sm_count()
{
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return nsm > 0 ? nsm : 1;
}

template <int KS, int NK, bool X3>
cudaError_t launch_adj(const BwdArgs& a, int N, int* err, cudaStream_t s)
{
    using C = TcAdjCfg<KS, NK, 2, X3>;
    cudaError_t e = cudaFuncSetAttribute(tc_bwd_adj<KS, NK, 2, X3>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int tx = (a.W + C::TW - 1) / C::TW, ty = (a.H + C::TH - 1) / C::TH;
    const long long tiles = (long long)N * tx * ty;
    const int grid = (int)std::max(1LL, std::min((long long)sm_count(), (tiles + C::NWG - 1) / C::NWG));
    tc_bwd_adj<KS, NK, 2, X3><<<grid, C::NTHREADS, C::SMEM_BYTES, s>>>(a, N, tx, ty, err);
    return cudaGetLastError();
}

}  // namespace

template <int KS, int NK, bool X3>
cudaError_t launch_dk(const BwdArgs& a, int N, int* err, cudaStream_t s)
{
    using C = TcDkCfg<KS, NK, X3>;
    cudaError_t e = cudaFuncSetAttribute(tc_bwd_dk<KS, NK, X3>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int tx = (a.W + 31) / 32, ty = (a.H + C::TPR - 1) / C::TPR;
    tc_bwd_dk<KS, NK, X3><<<dim3(tx * ty, N), 128, C::SMEM_BYTES, s>>>(a, tx, err);
    return cudaGetLastError();
}

cudaError_t launch_tc_bwd_dk(int ks, int nk, int prec, const BwdArgs& a, int N, int* err,
                             cudaStream_t s)
{
    const bool x3 = prec == TC_TF32X3;
    if (prec != TC_TF32 && !x3) return cudaErrorInvalidValue;
#define X(K, NN)                                                                          \
    if (ks == K && nk == NN) return x3 ? launch_dk<K, NN, true>(a, N, err, s)             \
                                       : launch_dk<K, NN, false>(a, N, err, s);
    X(3, 4) X(5, 24) X(7, 48)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t launch_tc_bwd_adj(int ks, int nk, int prec, const BwdArgs& a, int N, int* err,
                              cudaStream_t s)
{
    const bool x3 = prec == TC_TF32X3;
    if (prec != TC_TF32 && !x3) return cudaErrorInvalidValue;
#define X(K, NN)                                                                          \
    if (ks == K && nk == NN) return x3 ? launch_adj<K, NN, true>(a, N, err, s)            \
                                       : launch_adj<K, NN, false>(a, N, err, s);
    X(3, 4) X(5, 24) X(7, 48)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace tnrd
