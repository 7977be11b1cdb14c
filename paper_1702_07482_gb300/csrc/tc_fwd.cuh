// Tensor-core forward stage (TNRD_ALGO_TC_TF32):
//   z = K u      as an implicit GEMM  D_z[pixel][filter] (tcgen05, TF32 in, FP32 acc)
//   v = phi(z)   on the CUDA cores (FP32), each thread one pixel, all filters
//   Y = V Kmat   as a GEMM            D_Y[pixel][tap] = sum_i v_i(pixel) k_i[tap]
//   h(q) = sum_tap Y[q + off(tap)][tap]   (adjoint; scattered on the CUDA cores)
//   u_t = prox(u_{t-1} - fold(h))         (FP32, IEEE sqrt/div)
//
// Tile: TH = 16 NB - 2R rows x TW = 32 - 2R columns of output; its z-region is
// 16 NB rows x 32 columns.  One MMA group = 128 z positions: 16 rows of one
// row block x 8 columns of one residue class (columns r, r+4, .., r+28).
//
// Filter-bank operand A needs no im2col: for residue r the tile of u is kept
// as a copy shifted by r columns (u_r[i][j] = u[i][j + r], TF32-rounded).  A
// K-major core matrix is 8 rows of 16 bytes, rows 16 bytes apart, so reading
// u_r with rows 4 floats apart gives A[m][b'] = u_r[row][4 m + b'] directly:
// row m of the core matrix is pixel column r + 4 m, K index b' is the tap
// column.  The second K core matrix (taps 4..7) starts 16 bytes later
// (leading offset 16 B, overlapping the first); the next 8-pixel group is the
// next image row (stride offset = the copy's row pitch).  Kernel row a is one
// MMA of K = 8 with the start row shifted by a; taps b' >= ksize are zero in B.
//
// TNRD_ALGO_TC_BF16 (BF = true) runs the same tile and groups with BF16
// operands (kind::f16, K = 16 per MMA, FP32 accumulation).  A BF16 core-matrix
// row is 8 values, so residue r of u is kept as overlapping chunks of 8:
// chunk c of a row holds u columns 4c + r .. 4c + r + 7.  Core row m is chunk
// m (pixel column r + 4m, taps 0..7) and the second K core (taps 8..15) is
// chunk m + 2, 32 bytes on.  V and the adjoint's filter matrix are BF16 too;
// phi, the scatter, the fold and the prox stay FP32.
#pragma once
#include "args.cuh"
#include "tc_ptx.cuh"

namespace tnrd {

// Device-side failure word of the tensor-core kernels (0 = none); read and
// cleared by tnrd_device_status().  Defined here: only tc_fwd.cu includes this
// header (the library is built without relocatable device code).
__device__ int g_tc_error = 0;

// One stage on one tile (the whole CTA).  err receives TNRD_ERR_TIMEOUT (4)
// when a wait on the tensor core gives up (the tile's output is then not written).
template <int KS, int NK, int NB, bool BF>
__device__ __forceinline__ void tc_tile(const TileJob& a, unsigned char* smem, int* err)
{
    using C = TcCfg<KS, NK, NB, BF>;
    constexpr int R = C::R, TW = C::TW, TH = C::TH;
    constexpr long long WAIT_LIMIT = 1ll << 31;   // SM cycles, about one second
    float* sU = reinterpret_cast<float*>(smem + C::OFF_U);
    float* sBz = reinterpret_cast<float*>(smem + C::OFF_BZ);
    float* sKm = reinterpret_cast<float*>(smem + C::OFF_KM);
    float* sV = reinterpret_cast<float*>(smem + C::OFF_V);
    float* sW = reinterpret_cast<float*>(smem + C::OFF_W);
    float* sH = reinterpret_cast<float*>(smem + C::OFF_H);
    uint64_t* mbz = reinterpret_cast<uint64_t*>(smem + C::OFF_MISC);       // 2 barriers
    uint64_t* mby = reinterpret_cast<uint64_t*>(smem + C::OFF_MISC + 16);
    uint32_t* tbase = reinterpret_cast<uint32_t*>(smem + C::OFF_MISC + 24);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int ty = a.ty, tx = a.tx;
    const int H = a.H, W = a.W;
    const int y0 = tile_origin(ty, TH, H), x0 = tile_origin(tx, TW, W);
    const bool border = (ty == 0) || (ty == a.tiles_y - 1) || (tx == 0) || (tx == a.tiles_x - 1);
    const float* uin = a.u_in;

    // ---- stage operands in shared memory ----------------------------------
    if constexpr (!BF) {
        constexpr int UCOPY = C::UROWS * C::UPITCH;
        for (int idx = tid; idx < 4 * UCOPY; idx += 128) {
            const int r = idx / UCOPY, rem = idx - r * UCOPY;
            const int i = rem / C::UPITCH, j = rem - i * C::UPITCH;
            const int yy = sym_idx(y0 - 2 * R + i, H), xx = sym_idx(x0 - 2 * R + j + r, W);
            sU[idx] = tc::to_tf32(__ldcg(uin + (size_t)yy * a.pitch + xx));
        }
        // B of the filter bank, per kernel row ka: B[nn][b'] = k_nn[ka][KS-1-b'],
        // K-major core matrices [nn/8][b'/4][nn%8][b'%4]
        for (int e = tid; e < KS * C::NPAD * 8; e += 128) {
            const int ka = e / (C::NPAD * 8), rem = e - ka * (C::NPAD * 8);
            const int nn = rem / 8, k = rem - nn * 8;
            const float v = (nn < NK && k < KS) ? __ldg(a.k + (nn * KS + ka) * KS + (KS - 1 - k)) : 0.0f;
            sBz[ka * C::NPAD * 8 + ((nn / 8) * 2 + k / 4) * 32 + (nn % 8) * 4 + (k % 4)] = tc::to_tf32(v);
        }
        // B of the adjoint GEMM: B[tap][i] = k_i[tap], core matrices [i/4][tap/8][tap%8][i%4]
        for (int e = tid; e < C::NT * C::NKP; e += 128) {
            const int tap = e / C::NKP, i = e - tap * C::NKP;
            const float v = (tap < KS * KS && i < NK) ? __ldg(a.k + i * KS * KS + tap) : 0.0f;
            sKm[((i / 4) * (C::NT / 8) + tap / 8) * 32 + (tap % 8) * 4 + (i % 4)] = tc::to_tf32(v);
        }
    } else {
        // u chunks, two values per 32-bit store: [r][row][chunk][8]
        uint32_t* sU2 = reinterpret_cast<uint32_t*>(sU);
        constexpr int PAIRS = 4 * C::UROWS * C::UCHUNKS * 4;
        for (int idx = tid; idx < PAIRS; idx += 128) {
            const int e2 = idx & 3, c = (idx >> 2) % C::UCHUNKS, ri = (idx >> 2) / C::UCHUNKS;
            const int r = ri / C::UROWS, i = ri - r * C::UROWS;
            const int yy = sym_idx(y0 - 2 * R + i, H);
            const int x = x0 - 2 * R + 4 * c + r + 2 * e2;
            const float* ur = uin + (size_t)yy * a.pitch;
            sU2[idx] = tc::pack_bf16x2(__ldcg(ur + sym_idx(x, W)), __ldcg(ur + sym_idx(x + 1, W)));
        }
        // B of the filter bank, per kernel row ka: B[nn][b'] = k_nn[ka][KS-1-b'] (b' < 16),
        // core matrices [nn/8][b'/8][nn%8][b'%8]
        uint32_t* sBz2 = reinterpret_cast<uint32_t*>(sBz);
        for (int e = tid; e < KS * C::NPAD * 8; e += 128) {
            const int ka = e / (C::NPAD * 8), rem = e - ka * (C::NPAD * 8);
            const int nn = rem / 8, k = 2 * (rem - nn * 8);
            const float v0 = (nn < NK && k < KS) ? __ldg(a.k + (nn * KS + ka) * KS + (KS - 1 - k)) : 0.0f;
            const float v1 = (nn < NK && k + 1 < KS) ? __ldg(a.k + (nn * KS + ka) * KS + (KS - 2 - k)) : 0.0f;
            sBz2[(ka * C::NPAD * 16 + ((nn / 8) * 2 + k / 8) * 64 + (nn % 8) * 8 + (k % 8)) / 2] =
                tc::pack_bf16x2(v0, v1);
        }
        // B of the adjoint GEMM: B[tap][i] = k_i[tap], core matrices [i/8][tap/8][tap%8][i%8]
        uint32_t* sKm2 = reinterpret_cast<uint32_t*>(sKm);
        for (int e = tid; e < C::NT * C::NKP / 2; e += 128) {
            const int tap = e / (C::NKP / 2), i = 2 * (e - tap * (C::NKP / 2));
            const bool tok = tap < KS * KS;
            const float v0 = (tok && i < NK) ? __ldg(a.k + i * KS * KS + tap) : 0.0f;
            const float v1 = (tok && i + 1 < NK) ? __ldg(a.k + (i + 1) * KS * KS + tap) : 0.0f;
            sKm2[(((i / 8) * (C::NT / 8) + tap / 8) * 64 + (tap % 8) * 8 + (i % 8)) / 2] =
                tc::pack_bf16x2(v0, v1);
        }
    }
    for (int e = tid; e < NK * C::WPADN; e += 128) {
        const int i = e / C::WPADN, jj = e - i * C::WPADN - RBF_WPAD;
        sW[e] = (jj >= 0 && jj < a.nrbf) ? __ldg(a.w + i * a.nrbf + jj) : 0.0f;
    }
    for (int e = tid; e < C::ESZ * 128 * C::NKP / 4; e += 128) sV[e] = 0.0f;
    for (int e = tid; e < 4 * C::HROWS * C::HPITCH; e += 128) sH[e] = 0.0f;
    if (tid == 0) {
        tc::mbar_init(mbz + 0, 1);
        tc::mbar_init(mbz + 1, 1);
        tc::mbar_init(mby, 1);
    }
    if (warp == 0) tc::tmem_alloc(tbase, C::TMEM_COLS);
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tbase;
    // TMEM columns: z of even groups at 0, z of odd groups at 64, Y at 128
    const uint32_t tyv = tmem + 128;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    constexpr uint32_t FMT = BF ? tc::FMT_BF16 : tc::FMT_TF32;
    constexpr uint32_t ID_Z = tc::idesc(FMT, 128, C::NPAD);
    constexpr uint32_t ID_Y = tc::idesc(FMT, 128, C::NT);
    constexpr uint32_t LBO_KM = (C::NT / 8) * 128;
    const RbfConst& rc = *a.rc;

    const int g = tid >> 3, mp = tid & 7;       // this thread's pixel in every group
    float* myh = sH + warp * (C::HROWS * C::HPITCH);
    uint32_t phz = 0u, phy = 0u;   // bit b of phz: parity of z buffer b's next phase
    int ok = 1;
    constexpr int NG = 4 * NB;                  // groups (row block, residue) per tile

    // z = K u of group gi into TMEM buffer zb: one MMA (K = 32 bytes) per kernel row
    auto issue_z = [&](int gi, int zb) {
        const int nb = gi >> 2, r = gi & 3;
        const uint32_t ur = tc::smem_u32(sU) + (uint32_t)(r * C::UROWS * C::UROWB);
#pragma unroll
        for (int ka = 0; ka < KS; ++ka) {
            const uint64_t da = tc::sdesc(ur + (uint32_t)((16 * nb + 2 * R - ka) * C::UROWB),
                                          BF ? 32 : 16, C::UROWB);
            const uint64_t db = tc::sdesc(tc::smem_u32(sBz) + (uint32_t)(ka * C::NPAD * 32), 128, 256);
            if constexpr (BF) tc::mma_f16(tmem + 64u * zb, da, db, ID_Z, ka > 0);
            else tc::mma_tf32(tmem + 64u * zb, da, db, ID_Z, ka > 0);
        }
        tc::commit(mbz + zb);
    };
    if (tid == 0) issue_z(0, 0);

#pragma unroll 1
    for (int gi = 0; gi < NG; ++gi) {
        const int nb = gi >> 2, r = gi & 3, zb = gi & 1;
        if (ok) {
            ok = tc::mbar_wait(mbz + zb, (phz >> zb) & 1u, WAIT_LIMIT);
            phz ^= 1u << zb;
            tc::fence_after();
        }
        ok = __syncthreads_and(ok);
        // the next group's filter bank runs on the tensor core during phi
        if (ok && tid == 0 && gi + 1 < NG) issue_z(gi + 1, zb ^ 1);
        // ---- v = phi(z) into the A operand of the adjoint GEMM -------------------
        const int yy = y0 - R + 16 * nb + g, xx = x0 - R + r + 4 * mp;
        const bool inside = (unsigned)yy < (unsigned)H && (unsigned)xx < (unsigned)W;
        if (ok) {
#pragma unroll 1
            for (int c8 = 0; c8 < NK; c8 += 8) {
                float z[8], v[8];
                tc::tmem_ld8(tmem + 64u * zb + lane_base + c8, z);
                // branch-free: the 8 evaluations are independent and interleave
                // (z is finite everywhere: u is mirror-loaded), then masked
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int i = c8 + q;
                    const float ph = rbf_phi_w(z[q], sW + (i < NK ? i : 0) * C::WPADN, rc);
                    v[q] = (i < NK && inside) ? ph : 0.0f;
                }
                if constexpr (!BF) {
                    // A layout [filter/4][g][mp][filter%4]: core matrices of 8 positions x 4 filters
                    float4* d0 = reinterpret_cast<float4*>(sV + ((c8 / 4) * 16 + g) * 32 + mp * 4);
                    *d0 = make_float4(tc::to_tf32(v[0]), tc::to_tf32(v[1]), tc::to_tf32(v[2]), tc::to_tf32(v[3]));
                    if (c8 + 4 < C::NKP) {
                        float4* d1 = reinterpret_cast<float4*>(sV + ((c8 / 4 + 1) * 16 + g) * 32 + mp * 4);
                        *d1 = make_float4(tc::to_tf32(v[4]), tc::to_tf32(v[5]), tc::to_tf32(v[6]), tc::to_tf32(v[7]));
                    }
                } else {
                    // A layout [filter/8][g][mp][filter%8]: core matrices of 8 positions x 8 filters
                    uint4* d0 = reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(sV) +
                                                         ((c8 / 8) * 16 + g) * 128 + mp * 16);
                    *d0 = make_uint4(tc::pack_bf16x2(v[0], v[1]), tc::pack_bf16x2(v[2], v[3]),
                                     tc::pack_bf16x2(v[4], v[5]), tc::pack_bf16x2(v[6], v[7]));
                }
            }
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        // ---- Y = V Kmat ----------------------------------------------------------
        if (ok) {
            if (tid == 0) {
                // one MMA per two K cores (8 filters TF32, 16 filters BF16): 4 KB of V
                // and 2 LBO_KM of the filter matrix apart
#pragma unroll
                for (int s = 0; s < C::NKP / C::KMMA; ++s) {
                    const uint64_t da = tc::sdesc(tc::smem_u32(sV) + (uint32_t)(s * 4096), 16 * 128, 128);
                    const uint64_t db = tc::sdesc(tc::smem_u32(sKm) + (uint32_t)(s * 2 * LBO_KM), LBO_KM, 128);
                    if constexpr (BF) tc::mma_f16(tyv, da, db, ID_Y, s > 0);
                    else tc::mma_tf32(tyv, da, db, ID_Y, s > 0);
                }
                tc::commit(mby);
            }
            ok = tc::mbar_wait(mby, phy & 1, WAIT_LIMIT);
            ++phy;
            tc::fence_after();
        }
        ok = __syncthreads_and(ok);
        // ---- scatter: h(p - off(tap)) += Y[p][tap] into this warp's partial ------
        // (tcgen05.ld is warp-collective: every lane loads; lanes outside the
        // image have v = 0, hence Y = 0, and add zeros at in-range indices)
        // Two lanes of a warp, (g, mp) and (g', mp'), update the same h element
        // through taps (a, b) and (a', b') when g - a = g' - a' and
        // 4 mp - b = 4 mp' - b', i.e. only for taps with different kernel rows,
        // or with the same row and b - b' = +-4.  Taps of one row with b in
        // [0, 4) or in [4, 8) never collide, so a warp barrier (which also
        // orders the lanes' shared-memory accesses) before each such run keeps
        // every read-modify-write of h whole.
        if (ok) {
            const int base = (16 * nb + g + 2 * R) * C::HPITCH + (r + 4 * mp + 2 * R);
#pragma unroll
            for (int c8 = 0; c8 < KS * KS; c8 += 8) {
                float y[8];
                tc::tmem_ld8(tyv + lane_base + c8, y);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int t = c8 + q;
                    if (t < KS * KS) {
                        if ((t % KS) % 4 == 0) __syncwarp();
                        myh[base - (t / KS) * C::HPITCH - (t % KS)] += y[q];
                    }
                }
            }
            __syncwarp();
        }
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
    }
    if (!ok) {
        // give the MMAs in flight a bounded chance to finish before TMEM is freed
        tc::mbar_wait(mbz + 0, phz & 1u, WAIT_LIMIT);
        tc::mbar_wait(mbz + 1, (phz >> 1) & 1u, WAIT_LIMIT);
    }

    // ---- epilogue: g = fold(sum of the warps' h), u_t = prox(u_{t-1} - g) ------
    if (ok) {
        const float lam = __ldg(a.lam);
        const int wy0 = tile_split(ty, TH, H, a.tiles_y, R), wy1 = tile_split(ty + 1, TH, H, a.tiles_y, R);
        const int wx0 = tile_split(tx, TW, W, a.tiles_x, R), wx1 = tile_split(tx + 1, TW, W, a.tiles_x, R);
        const float* fimg = a.f;
        float* uout = a.u_out;
        for (int idx = tid; idx < TH * TW; idx += 128) {
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
            for (int p = 0; p < nsy; ++p) {
                for (int q = 0; q < nsx; ++q) {
                    const int hi = sy[p] - (y0 - 2 * R), hj = sx[q] - (x0 - 2 * R);
                    float hs = 0.0f;
#pragma unroll
                    for (int wq = 0; wq < 4; ++wq) hs += sH[wq * (C::HROWS * C::HPITCH) + hi * C::HPITCH + hj];
                    gsum += hs;
                }
            }
            const float up = __ldcg(uin + (size_t)qy * a.pitch + qx);
            const float fv = __ldg(fimg + (size_t)qy * a.pitch + qx);
            uout[(size_t)qy * a.pitch + qx] = stage_out(up, gsum, fv, lam, a.dterm, a.proj_c);
        }
    } else if (tid == 0) {
        atomicExch(err, 4);
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, C::TMEM_COLS);
}

// Per-call stage: grid (tiles_x * tiles_y, N), one tile per CTA.
template <int KS, int NK, int NB, bool BF>
__global__ void __launch_bounds__(128, 2) tc_stage_fwd(const __grid_constant__ StageArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
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
    j.ty = blockIdx.x / a.tiles_x;
    j.tx = blockIdx.x - j.ty * a.tiles_x;
    j.k = a.k;
    j.w = a.w;
    j.lam = a.lam;
    j.nrbf = a.nrbf;
    j.dterm = a.dterm;
    j.proj_c = a.proj_c;
    j.rc = &a.rc;
    tc_tile<KS, NK, NB, BF>(j, smem, &g_tc_error);
}

// Stage t of a batched plan: grid (all images' tiles), the tile table of the
// plan gives each CTA its (image, tile); each image's parameter set, buffers
// and data term come from the plan.  Stage t writes u when (T-1-t) is even
// and the plan's inter-stage image otherwise, so the last stage lands in u.
template <int KS, int NK, int NB, bool BF>
__global__ void __launch_bounds__(128, 2) tc_batch_fwd(const __grid_constant__ BatchArgs a, int t)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int2 ti = a.tile_img[blockIdx.x];
    const BatchImg& im = a.imgs[ti.x];
    const BatchSet& ps = a.sets[im.set];
    TileJob j;
    j.u_out = ((a.T - 1 - t) % 2 == 0) ? im.u : im.tmp;
    j.u_in = (t == 0) ? im.f : (((a.T - t) % 2 == 0) ? im.u : im.tmp);
    j.f = im.f;
    j.H = im.H;
    j.W = im.W;
    j.pitch = im.pitch;
    j.tiles_x = im.tiles_x;
    j.tiles_y = im.tiles_y;
    j.ty = ti.y / im.tiles_x;
    j.tx = ti.y - j.ty * im.tiles_x;
    j.k = ps.k + (size_t)t * NK * KS * KS;
    j.w = ps.w + (size_t)t * NK * a.nrbf;
    j.lam = ps.lam + t;
    j.nrbf = a.nrbf;
    j.dterm = ps.dterm;
    j.proj_c = ps.proj_c;
    j.rc = &ps.rc;
    tc_tile<KS, NK, NB, BF>(j, smem, a.status);
}

}  // namespace tnrd
