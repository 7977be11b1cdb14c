// Tensor-core forward stage (TNRD_ALGO_TC_TF32 / _BF16) of Eq. diffusionprocessfinal:
//   z = K u      as an implicit GEMM  D_z[pixel][filter] (tcgen05, FP32 accumulation)
//   v = phi(z)   on the CUDA cores (FP32), each thread one pixel, all filters
//   Y = V Kmat   as a GEMM            D_Y[pixel][tap] = sum_i v_i(pixel) k_i[tap]
//   h(q) = sum_tap Y[q + off(tap)][tap]   (adjoint; scattered on the CUDA cores)
//   u_t = prox(u_{t-1} - fold(h))         (FP32, IEEE sqrt/div)
//
// Launch: one persistent CTA per SM made of NWG independent warpgroups (three
// for TF32, four for BF16).  The CTA takes a contiguous run of the launch's
// tiles; its warpgroups work through them in turn, each with its own tile
// buffers, TMEM columns and mbarriers and its own elected thread issuing the
// MMAs.  The filter operands of both GEMMs and the RBF weights are staged once
// per CTA and parameter set (a batch may change sets between images).
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
// The raw u rows of the tile are read from global memory once and the four
// residue copies built from them in shared memory.
//
// BF16 (BF = true) runs the same tile and groups with BF16 operands
// (kind::f16, K = 16 per MMA, FP32 accumulation).  A BF16 core-matrix row is 8
// values, so residue r of u is kept as overlapping chunks of 8: chunk c of a
// row holds u columns 4c + r .. 4c + r + 7.  Core row m is chunk m (pixel
// column r + 4m, taps 0..7) and the second K core (taps 8..15) is chunk m + 2,
// 32 bytes on.  V and the adjoint's filter matrix are BF16 too; phi, the
// scatter, the fold and the prox stay FP32.
//
// X3 (TNRD_ALGO_TC_TF32X3) keeps FP32 accuracy on the TF32 tensor cores: every
// operand x is held as hi = tf32(x) and lo = tf32(x - hi) (x - hi is exact in
// FP32), and each GEMM is taken as lo*hi + hi*lo + hi*hi, three TF32 MMAs into
// the same FP32 accumulator; the dropped lo*lo term is below 2^-22 of the
// product.  To keep three warpgroups per CTA with the doubled operands, a
// warpgroup holds the u copies of two residues only (a ring; the groups run
// residue-major and the next residue is built from the tile's raw rows while
// the current one is in use), V holds one round of 16 filters (high and low
// parts) at a time -- the adjoint MMAs of round rr accumulate Y in its own TMEM
// buffer while phi works on round rr + 1, and the next round's V is written
// once they have read the slot -- and z has one TMEM buffer: z(gi + 1) is
// issued once phi has read z(gi), and runs under gi's adjoint and scatter.
//
// TMEM: each warpgroup owns 128 columns, two buffers of 64.  Group g's z lands
// in buffer g & 1; once phi has read it, the same buffer receives group g's Y,
// and once Y has been read, group g + 2's z.  So the filter bank of the next
// group always runs on the tensor core while phi of this one runs on the SM.
//
// Adjoint scatter into ONE h buffer per warpgroup, in kernel-row phases: lane
// (g, mp) of warp w (pixel row 4w + g' of the row block, g = 4w + g') adds its
// tap (a, b) value at h row (row - a).  In one phase all warps use the same a,
// so their rows are disjoint; a warpgroup barrier separates the phases.  Within
// a warp two lanes reach the same element only through taps b and b +- 4 of the
// same row, so a warp barrier before each run of taps with b in [0, 4) or
// [4, 8) keeps every read-modify-write whole.  The sums are in a fixed order:
// repeated runs give the same bits.
#pragma once
#include "args.cuh"
#include "tc_ptx.cuh"

namespace tnrd {

// Device-side failure word of the tensor-core kernels (0 = none); read and
// cleared by tnrd_device_status().  Defined here: only tc_fwd.cu includes this
// header (the library is built without relocatable device code).
__device__ int g_tc_error = 0;

// What one tile needs besides the shared filter operands.
struct TcTile {
    const float* u_in;
    float* u_out;
    const float* f;
    int H, W, pitch;
    int tiles_x, tiles_y, ty, tx;
    const float* lam;
    int dterm;
    float proj_c;
};

// One parameter set of the stage.
struct TcSet {
    const float* k;       // [NK][KS][KS]
    const float* w;       // [NK][nrbf]
    int nrbf;
    const RbfConst* rc;
};

// Tiles of a per-call stage: N images of tiles_x * tiles_y tiles, one set.
struct TcCallSrc {
    const StageArgs* a;
    int n_img;
    __device__ int ntiles() const { return n_img * a->tiles_x * a->tiles_y; }
    __device__ int set_of(int) const { return 0; }
    __device__ int seg_end(int, int c1) const { return c1; }
    __device__ TcSet params(int) const { return TcSet{a->k, a->w, a->nrbf, &a->rc}; }
    __device__ TcTile tile(int s) const
    {
        const int tpi = a->tiles_x * a->tiles_y;
        const int n = s / tpi, ti = s - n * tpi;
        TcTile j;
        j.u_in = a->u_in + (size_t)n * a->img_stride;
        j.u_out = a->u_out + (size_t)n * a->img_stride;
        j.f = a->f + (size_t)n * a->img_stride;
        j.H = a->H;
        j.W = a->W;
        j.pitch = a->pitch;
        j.tiles_x = a->tiles_x;
        j.tiles_y = a->tiles_y;
        j.ty = ti / a->tiles_x;
        j.tx = ti - j.ty * a->tiles_x;
        j.lam = a->lam;
        j.dterm = a->dterm;
        j.proj_c = a->proj_c;
        return j;
    }
};

// Tiles of stage t of a batched plan: the plan's tile table gives each global
// tile its (image, tile); each image its buffers, parameter set and data
// term.  Stage t writes u when (T-1-t) is even and the plan's inter-stage
// image otherwise, so the last stage lands in u.
template <int KS, int NK>
struct TcBatchSrc {
    const BatchArgs* a;
    int t;
    __device__ int ntiles() const { return a->ntiles; }
    __device__ int set_of(int s) const { return a->imgs[a->tile_img[s].x].set; }
    __device__ int seg_end(int s, int c1) const
    {
        const int set = set_of(s);
        int e = s + 1;
        while (e < c1 && set_of(e) == set) ++e;
        return e;
    }
    __device__ TcSet params(int set) const
    {
        const BatchSet& ps = a->sets[set];
        return TcSet{ps.k + (size_t)t * NK * KS * KS, ps.w + (size_t)t * NK * a->nrbf, a->nrbf, &ps.rc};
    }
    __device__ TcTile tile(int s) const
    {
        const int2 ti = a->tile_img[s];
        const BatchImg& im = a->imgs[ti.x];
        const BatchSet& ps = a->sets[im.set];
        TcTile j;
        j.u_out = ((a->T - 1 - t) % 2 == 0) ? im.u : im.tmp;
        j.u_in = (t == 0) ? im.f : (((a->T - t) % 2 == 0) ? im.u : im.tmp);
        j.f = im.f;
        j.H = im.H;
        j.W = im.W;
        j.pitch = im.pitch;
        j.tiles_x = im.tiles_x;
        j.tiles_y = im.tiles_y;
        j.ty = ti.y / im.tiles_x;
        j.tx = ti.y - j.ty * im.tiles_x;
        j.lam = ps.lam + t;
        j.dterm = ps.dterm;
        j.proj_c = ps.proj_c;
        return j;
    }
};

// Filter operands of both GEMMs and the padded RBF weights of one parameter
// set, by all threads of the CTA.
template <int KS, int NK, int NB, bool BF, bool X3>
__device__ __forceinline__ void tc_stage_consts(const TcSet& ps, unsigned char* smem, int tid)
{
    using C = TcCfg<KS, NK, NB, BF, X3>;
    constexpr int NTH = C::NTHREADS;
    if constexpr (!BF) {
        float* sBz = reinterpret_cast<float*>(smem + C::OFF_BZ);
        float* sKm = reinterpret_cast<float*>(smem + C::OFF_KM);
        // B of the filter bank, per kernel row ka: B[nn][b'] = k_nn[ka][KS-1-b'],
        // K-major core matrices [nn/8][b'/4][nn%8][b'%4]
        for (int e = tid; e < KS * C::NPAD * 8; e += NTH) {
            const int ka = e / (C::NPAD * 8), rem = e - ka * (C::NPAD * 8);
            const int nn = rem / 8, k = rem - nn * 8;
            const float v = (nn < NK && k < KS) ? __ldg(ps.k + (nn * KS + ka) * KS + (KS - 1 - k)) : 0.0f;
            const int o = ka * C::NPAD * 8 + ((nn / 8) * 2 + k / 4) * 32 + (nn % 8) * 4 + (k % 4);
            const float hi = tc::to_tf32(v);
            sBz[o] = hi;
            if constexpr (X3) sBz[C::BZ_BYTES / 4 + o] = tc::to_tf32(v - hi);
        }
        // B of the adjoint GEMM: B[tap][i] = k_i[tap], core matrices [i/4][tap/8][tap%8][i%4]
        for (int e = tid; e < C::NT * C::NKP; e += NTH) {
            const int tap = e / C::NKP, i = e - tap * C::NKP;
            const float v = (tap < KS * KS && i < NK) ? __ldg(ps.k + i * KS * KS + tap) : 0.0f;
            const int o = ((i / 4) * (C::NT / 8) + tap / 8) * 32 + (tap % 8) * 4 + (i % 4);
            const float hi = tc::to_tf32(v);
            sKm[o] = hi;
            if constexpr (X3) sKm[C::KM_BYTES / 4 + o] = tc::to_tf32(v - hi);
        }
    } else {
        // B of the filter bank, per kernel row ka: B[nn][b'] = k_nn[ka][KS-1-b'] (b' < 16),
        // core matrices [nn/8][b'/8][nn%8][b'%8]
        uint32_t* sBz2 = reinterpret_cast<uint32_t*>(smem + C::OFF_BZ);
        for (int e = tid; e < KS * C::NPAD * 8; e += NTH) {
            const int ka = e / (C::NPAD * 8), rem = e - ka * (C::NPAD * 8);
            const int nn = rem / 8, k = 2 * (rem - nn * 8);
            const float v0 = (nn < NK && k < KS) ? __ldg(ps.k + (nn * KS + ka) * KS + (KS - 1 - k)) : 0.0f;
            const float v1 = (nn < NK && k + 1 < KS) ? __ldg(ps.k + (nn * KS + ka) * KS + (KS - 2 - k)) : 0.0f;
            sBz2[(ka * C::NPAD * 16 + ((nn / 8) * 2 + k / 8) * 64 + (nn % 8) * 8 + (k % 8)) / 2] =
                tc::pack_bf16x2(v0, v1);
        }
        // B of the adjoint GEMM: B[tap][i] = k_i[tap], core matrices [i/8][tap/8][tap%8][i%8]
        uint32_t* sKm2 = reinterpret_cast<uint32_t*>(smem + C::OFF_KM);
        for (int e = tid; e < C::NT * C::NKP / 2; e += NTH) {
            const int tap = e / (C::NKP / 2), i = 2 * (e - tap * (C::NKP / 2));
            const bool tok = tap < KS * KS;
            const float v0 = (tok && i < NK) ? __ldg(ps.k + i * KS * KS + tap) : 0.0f;
            const float v1 = (tok && i + 1 < NK) ? __ldg(ps.k + (i + 1) * KS * KS + tap) : 0.0f;
            sKm2[(((i / 8) * (C::NT / 8) + tap / 8) * 64 + (tap % 8) * 8 + (i % 8)) / 2] =
                tc::pack_bf16x2(v0, v1);
        }
    }
    // RBF weights in the bank-conflict-free pair table of rbf_phi_col:
    // [round][row][column], filters beyond NK all zeros
    float2* sW2 = reinterpret_cast<float2*>(smem + C::OFF_W);
    for (int e = tid; e < C::NR * TC_ROWS * 16; e += NTH) {
        const int c = e & 15, row = (e >> 4) % TC_ROWS, r = (e >> 4) / TC_ROWS, f = 16 * r + c;
        const int j0 = row - RBF_WPAD;   // weight index of the pair's first element
        const bool ok0 = f < NK && j0 >= 0 && j0 < ps.nrbf, ok1 = f < NK && j0 + 1 >= 0 && j0 + 1 < ps.nrbf;
        sW2[e] = make_float2(ok0 ? __ldg(ps.w + f * ps.nrbf + j0) : 0.0f,
                             ok1 ? __ldg(ps.w + f * ps.nrbf + j0 + 1) : 0.0f);
    }
}

// Per-warpgroup pipeline state: parity of each mbarrier's next phase (bit 0, 1:
// z buffers, bit 2: Y) and which of them have a commit outstanding.
struct TcPipe {
    uint32_t ph = 0, pend = 0;
};

// One stage on one tile, by one warpgroup (bar: its named barrier).  Returns
// 0 if a wait on the tensor core gave up (the tile's output is then not
// written); uniform over the warpgroup.
template <int KS, int NK, int NB, bool BF, bool X3>
__device__ __forceinline__ int tc_tile(const TcTile& a, const RbfConst& rc, unsigned char* smem,
                                       unsigned char* wgs, uint32_t tmem, uint64_t* mb, TcPipe& pp,
                                       int wt, int bar)
{
    using C = TcCfg<KS, NK, NB, BF, X3>;
    constexpr int R = C::R, TW = C::TW, TH = C::TH;
    constexpr long long WAIT_LIMIT = 1ll << 31;   // SM cycles, about one second
    float* sU = reinterpret_cast<float*>(wgs + C::WG_U);
    float* sV = reinterpret_cast<float*>(wgs + C::WG_V);
    float* sH = reinterpret_cast<float*>(wgs + C::WG_H);
    const float* sW = reinterpret_cast<const float*>(smem + C::OFF_W);
    const uint32_t sBz = tc::smem_u32(smem + C::OFF_BZ);
    const uint32_t sKm = tc::smem_u32(smem + C::OFF_KM);

    const int warp = wt >> 5;
    const int H = a.H, W = a.W;
    const int y0 = tile_origin(a.ty, TH, H), x0 = tile_origin(a.tx, TW, W);
    const bool border = (a.ty == 0) || (a.ty == a.tiles_y - 1) || (a.tx == 0) || (a.tx == a.tiles_x - 1);
    // the whole z-region inside the image: no v needs masking
    const bool zin = y0 - R >= 0 && y0 - R + C::ZR <= H && x0 - R >= 0 && x0 - R + 32 <= W;
    const float* uin = a.u_in;

    // ---- stage u: raw rows (in the V area; X3: their own area, kept for the
    // tile), then the residue operands (X3: residue 0; the others as the groups
    // reach them) --------
    float* const sRaw = C::RING ? reinterpret_cast<float*>(wgs + C::WG_RAW) : sV;
    // ring layout: residue rres of u (X3: high and low parts) into ring slot rres & 1
    auto build_res = [&](int rres) {
        constexpr int UCOPY = C::UROWS * C::UPITCH;
        float* dst = sU + (rres & 1) * C::NSPL * (C::U_SLOT / 4);
        for (int idx = wt; idx < UCOPY; idx += 128) {
            const int i = idx / C::UPITCH, j = idx - i * C::UPITCH;
            const float v = sRaw[i * C::RAWP + j + rres];
            const float hi = tc::to_tf32(v);
            dst[idx] = hi;
            if constexpr (X3) dst[C::U_SLOT / 4 + idx] = tc::to_tf32(v - hi);
        }
    };
    tc::wg_sync(bar);   // the previous tile's epilogue has read h
    {
        float* raw = sRaw;
        const int ry = y0 - 2 * R, rx = x0 - 2 * R;
        const bool inner = ry >= 0 && ry + C::UROWS <= H && rx >= 0 && rx + C::RAWC <= W;
        constexpr int NRAW = C::UROWS * C::RAWC;
        // four loads in flight per thread before their stores
#pragma unroll 1
        for (int i0 = 0; i0 < NRAW; i0 += 4 * 128) {
            float v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int idx = i0 + k * 128 + wt;
                const int i = idx / C::RAWC, j = idx - i * C::RAWC;
                const int yy = inner ? ry + i : sym_idx(ry + i, H);
                const int xx = inner ? rx + j : sym_idx(rx + j, W);
                v[k] = idx < NRAW ? __ldcg(uin + (size_t)yy * a.pitch + xx) : 0.0f;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int idx = i0 + k * 128 + wt;
                const int i = idx / C::RAWC, j = idx - i * C::RAWC;
                if (idx < NRAW) raw[i * C::RAWP + j] = v[k];
            }
        }
        for (int e = wt; e < C::HROWS * C::HPITCH; e += 128) sH[e] = 0.0f;
        tc::wg_sync(bar);
        if constexpr (C::RING) {
            build_res(0);
        } else if constexpr (!BF) {
            constexpr int UCOPY = C::UROWS * C::UPITCH;
            for (int idx = wt; idx < 4 * UCOPY; idx += 128) {
                const int r = idx / UCOPY, rem = idx - r * UCOPY;
                const int i = rem / C::UPITCH, j = rem - i * C::UPITCH;
                sU[idx] = tc::to_tf32(raw[i * C::RAWP + j + r]);
            }
        } else {
            // u chunks, two values per 32-bit store: [r][row][chunk][8]
            uint32_t* sU2 = reinterpret_cast<uint32_t*>(sU);
            constexpr int PAIRS = 4 * C::UROWS * C::UCHUNKS * 4;
            for (int idx = wt; idx < PAIRS; idx += 128) {
                const int e2 = idx & 3, c = (idx >> 2) % C::UCHUNKS, ri = (idx >> 2) / C::UCHUNKS;
                const int r = ri / C::UROWS, i = ri - r * C::UROWS;
                const float* rr = raw + i * C::RAWP + 4 * c + r + 2 * e2;
                sU2[idx] = tc::pack_bf16x2(rr[0], rr[1]);
            }
        }
        tc::fence_async_smem();
        tc::fence_before();
        tc::wg_sync(bar);   // operands complete; the raw rows are no longer needed (but X3's)
        tc::fence_after();
    }

    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    constexpr uint32_t FMT = BF ? tc::FMT_BF16 : tc::FMT_TF32;
    constexpr uint32_t ID_Z = tc::idesc(FMT, 128, C::NPAD);
    constexpr uint32_t ID_Y = tc::idesc(FMT, 128, C::NT);
    constexpr uint32_t LBO_KM = (C::NT / 8) * 128;
    constexpr int NG = 4 * NB;                  // groups (row block, residue) per tile
    const int g = wt >> 3, mp = wt & 7;         // this thread's pixel in every group

    // z = K u of group gi into TMEM buffer gi & 1: one MMA (K = 32 bytes) per kernel
    // row.  Ring layout: groups residue-major (gi = NB r + nb), residue r in ring slot
    // r & 1, one z buffer (0); X3: three MMAs per kernel row.
    constexpr bool RING = C::RING;
    auto issue_z = [&](int gi) {
        const int nb = RING ? gi % NB : gi >> 2, r = RING ? gi / NB : gi & 3, zb = RING ? 0 : gi & 1;
        const uint32_t ur = tc::smem_u32(sU) +
                            (uint32_t)(RING ? (r & 1) * C::NSPL * C::U_SLOT : r * C::UROWS * C::UROWB);
#pragma unroll
        for (int ka = 0; ka < KS; ++ka) {
            const uint32_t ua = ur + (uint32_t)((16 * nb + 2 * R - ka) * C::UROWB);
            const uint32_t ba = sBz + (uint32_t)(ka * C::NPAD * 32);
            const uint64_t da = tc::sdesc(ua, BF ? 32 : 16, C::UROWB);
            const uint64_t db = tc::sdesc(ba, 128, 256);
            if constexpr (BF) {
                tc::mma_f16(tmem + 64u * zb, da, db, ID_Z, ka > 0);
            } else if constexpr (X3) {
                // u_lo k_hi + u_hi k_lo + u_hi k_hi
                tc::mma_tf32(tmem + 64u * zb, tc::sdesc(ua + (uint32_t)C::U_SLOT, 16, C::UROWB), db,
                             ID_Z, ka > 0);
                tc::mma_tf32(tmem + 64u * zb, da, tc::sdesc(ba + (uint32_t)C::BZ_BYTES, 128, 256),
                             ID_Z, 1);
                tc::mma_tf32(tmem + 64u * zb, da, db, ID_Z, 1);
            } else {
                tc::mma_tf32(tmem + 64u * zb, da, db, ID_Z, ka > 0);
            }
        }
        tc::commit(mb + zb);
    };
    if (wt == 0) {
        issue_z(0);
        if constexpr (!RING) issue_z(1);
    }
    pp.pend |= RING ? 1u : 3u;
    int ok = 1;

    // phi of round rr (filters 16 rr .. 16 rr + 15) of the group in TMEM buffer
    // tbuf: x[4q + t] = v of filter 16 rr + 4((q + a) mod 4) + t, a = (wt >> 2) & 3.
    // Lane j = 4a + b of each half-warp takes the round's filter
    // 4((q + a) mod 4) + ((t + b) mod 4) at step s = 4q + t: at every step the
    // half-warp's 16 lanes evaluate 16 different filters, so their weight loads
    // fall in 16 distinct bank pairs.  Filters beyond NK have zero weights (v = 0).
    const int ja = (wt >> 2) & 3, jb = wt & 3;
    auto phi_round = [&](int rr, uint32_t tbuf, bool inside, float (&x)[16]) {
        const float2* sW2 = reinterpret_cast<const float2*>(smem + C::OFF_W);
        {
            uint32_t zr0[8], zr1[8];
            tc::tmem_ld8_nowait(tbuf + lane_base + 16 * rr, zr0);
            tc::tmem_ld8_nowait(tbuf + lane_base + 16 * rr + 8, zr1);
            tc::tmem_wait_ld();
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                x[k] = __uint_as_float(zr0[k]);
                x[k + 8] = __uint_as_float(zr1[k]);
            }
        }
        rotl16(x, 4 * ja);                   // groups of four rotated by a
        rotl4x4(x, jb);                      // within the group by b
        const float2* tab_r = sW2 + rr * TC_ROWS * 16;
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            const int col = (4 * ((s >> 2) + ja) & 12) | (((s & 3) + jb) & 3);
            x[s] = rbf_phi_col(x[s], tab_r, col, rc);
        }
        rotl4x4(x, (4 - jb) & 3);            // x[4q + t] = v of filter 4((q + a) mod 4) + t
        if (!zin) {
#pragma unroll
            for (int m = 0; m < 16; ++m) x[m] = inside ? x[m] : 0.0f;
        }
    };
    // scatter h(p - off(tap)) += Y[p][tap] of group (nb, r), one kernel row per phase
    constexpr int NY8 = (KS * KS + 7) / 8;
    auto scatter = [&](int nb, int r, const uint32_t (&yr)[NY8][8]) {
        const int base = (16 * nb + g + 2 * R) * C::HPITCH + (r + 4 * mp + 2 * R);
#pragma unroll
        for (int ka = 0; ka < KS; ++ka) {
            if (ka > 0) tc::wg_sync(bar);
#pragma unroll
            for (int b = 0; b < KS; ++b) {
                if (b % 4 == 0) __syncwarp();
                const int t = ka * KS + b;
                sH[base - ka * C::HPITCH - b] += __uint_as_float(yr[t / 8][t % 8]);
            }
        }
        __syncwarp();
    };
    // wait on mbarrier b (z buffers 0, 1; Y 2), uniform over the warpgroup
    auto wait_mb = [&](int b) {
        const bool got = ok && tc::mbar_wait(mb + b, (pp.ph >> b) & 1u, WAIT_LIMIT);
        if (got) {
            pp.ph ^= 1u << b;
            pp.pend &= ~(1u << b);
        }
        ok = tc::wg_and(bar, got);
    };

    if constexpr (RING) {
        // one z buffer (columns 0..63) and Y (64..127); z(gi + 1) is issued once
        // phi has read z(gi) and runs under the adjoint and the scatter of gi
        const uint32_t tbuf = tmem, ybuf = tmem + 64u;
#pragma unroll 1
        for (int gi = 0; gi < NG; ++gi) {
            const int nb = gi % NB, r = gi / NB;
            wait_mb(0);
            tc::fence_after();
            // the next residue into the slot of residue r - 1, whose z are all done
            if ((gi + 1) % NB == 0 && gi + 1 < NG) build_res((gi + 1) / NB);
            const int yy = y0 - R + 16 * nb + g, xx = x0 - R + r + 4 * mp;
            const bool inside = (unsigned)yy < (unsigned)H && (unsigned)xx < (unsigned)W;
#pragma unroll 1
            for (int rr = 0; rr < C::NR; ++rr) {
                float x[16];
                if (ok) phi_round(rr, tbuf, inside, x);
                // the previous round's adjoint MMAs have read the V slot
                if (rr > 0) wait_mb(2);
                if (ok) {
                    // A layout [filter/4][g][mp][filter%4] of the round's 16 filters,
                    // high parts, then low parts VLO bytes on
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        const int f0 = 4 * ((q4 + ja) & 3);
                        if (16 * rr + f0 < C::NKP) {
                            float hi[4], lo[4];
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                hi[k] = tc::to_tf32(x[4 * q4 + k]);
                                lo[k] = tc::to_tf32(x[4 * q4 + k] - hi[k]);
                            }
                            float* dst = sV + ((f0 / 4) * 16 + g) * 32 + mp * 4;
                            *reinterpret_cast<float4*>(dst) = make_float4(hi[0], hi[1], hi[2], hi[3]);
                            if constexpr (X3)
                                *reinterpret_cast<float4*>(dst + C::VLO / 4) = make_float4(lo[0], lo[1], lo[2], lo[3]);
                        }
                    }
                }
                tc::fence_async_smem();
                tc::fence_before();
                tc::wg_sync(bar);
                tc::fence_after();
                const bool last = rr == C::NR - 1;
                if (ok && wt == 0) {
                    // Y += V_rr Kmat_rr: per 8 filters v_lo k_hi + v_hi k_lo + v_hi k_hi
                    const int nks = min(2, (C::NKP - 16 * rr) / 8);
                    for (int s = 0; s < nks; ++s) {
                        const uint32_t va = tc::smem_u32(sV) + (uint32_t)(s * 4096);
                        const uint32_t kh = sKm + (uint32_t)((2 * rr + s) * 2 * LBO_KM);
                        const uint64_t dvh = tc::sdesc(va, 16 * 128, 128);
                        const uint64_t dkh = tc::sdesc(kh, LBO_KM, 128);
                        if constexpr (X3) {
                            tc::mma_tf32(ybuf, tc::sdesc(va + (uint32_t)C::VLO, 16 * 128, 128), dkh, ID_Y,
                                         rr > 0 || s > 0);
                            tc::mma_tf32(ybuf, dvh, tc::sdesc(kh + (uint32_t)C::KM_BYTES, LBO_KM, 128),
                                         ID_Y, 1);
                            tc::mma_tf32(ybuf, dvh, dkh, ID_Y, 1);
                        } else {
                            tc::mma_tf32(ybuf, dvh, dkh, ID_Y, rr > 0 || s > 0);
                        }
                    }
                    tc::commit(mb + 2);
                    // every lane has read z(gi) and written the next residue: z(gi + 1)
                    if (last && gi + 1 < NG) issue_z(gi + 1);
                }
                if (ok) {
                    pp.pend |= 4u;
                    if (last && gi + 1 < NG) pp.pend |= 1u;
                }
            }
            wait_mb(2);
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
            if (ok) scatter(nb, r, yr);
        }
    } else {
#pragma unroll 1
    for (int gi = 0; gi < NG; ++gi) {
        const int nb = gi >> 2, r = gi & 3, zb = gi & 1;
        const uint32_t tbuf = tmem + 64u * zb;
        wait_mb(zb);
        tc::fence_after();
        // ---- v = phi(z) into the A operand of the adjoint GEMM -------------------
        const int yy = y0 - R + 16 * nb + g, xx = x0 - R + r + 4 * mp;
        const bool inside = (unsigned)yy < (unsigned)H && (unsigned)xx < (unsigned)W;
        if (ok) {
#pragma unroll 1
            for (int rr = 0; rr < C::NR; ++rr) {
                float x[16];
                phi_round(rr, tbuf, inside, x);
                if constexpr (!BF) {
                    // A layout [filter/4][g][mp][filter%4]: core matrices of 8 positions x 4
                    // filters; group q of this lane is the round's filter group (q + a) mod 4
                    // (16-byte stores at lane-dependent groups: 8 lanes of a quarter-warp
                    // differ in mp, so they still hit 8 distinct 16-byte bank groups)
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        const int f0 = 16 * rr + 4 * ((q4 + ja) & 3);
                        if (16 * rr + 16 <= C::NKP || f0 < C::NKP)
                            *reinterpret_cast<float4*>(sV + ((f0 / 4) * 16 + g) * 32 + mp * 4) =
                                make_float4(tc::to_tf32(x[4 * q4]), tc::to_tf32(x[4 * q4 + 1]),
                                            tc::to_tf32(x[4 * q4 + 2]), tc::to_tf32(x[4 * q4 + 3]));
                    }
                } else {
                    rotl16(x, (16 - 4 * ja) & 15);   // filter order: x[m] = v of filter 16 rr + m
                    // A layout [filter/8][g][mp][filter%8]: core matrices of 8 positions x 8 filters
#pragma unroll
                    for (int q8 = 0; q8 < 2; ++q8) {
                        const int f0 = 16 * rr + 8 * q8;
                        if (f0 < C::NKP)
                            *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(sV) +
                                                      ((f0 / 8) * 16 + g) * 128 + mp * 16) =
                                make_uint4(tc::pack_bf16x2(x[8 * q8], x[8 * q8 + 1]),
                                           tc::pack_bf16x2(x[8 * q8 + 2], x[8 * q8 + 3]),
                                           tc::pack_bf16x2(x[8 * q8 + 4], x[8 * q8 + 5]),
                                           tc::pack_bf16x2(x[8 * q8 + 6], x[8 * q8 + 7]));
                    }
                }
            }
        }
        tc::fence_async_smem();
        tc::fence_before();
        tc::wg_sync(bar);
        tc::fence_after();
        // ---- Y = V Kmat into the same buffer (z has been read) -------------------
        if (ok && wt == 0) {
            // one MMA per two K cores (8 filters TF32, 16 filters BF16): 4 KB of V
            // and 2 LBO_KM of the filter matrix apart
#pragma unroll
            for (int s = 0; s < C::NKP / C::KMMA; ++s) {
                const uint64_t da = tc::sdesc(tc::smem_u32(sV) + (uint32_t)(s * 4096), 16 * 128, 128);
                const uint64_t db = tc::sdesc(sKm + (uint32_t)(s * 2 * LBO_KM), LBO_KM, 128);
                if constexpr (BF) tc::mma_f16(tbuf, da, db, ID_Y, s > 0);
                else tc::mma_tf32(tbuf, da, db, ID_Y, s > 0);
            }
            tc::commit(mb + 2);
        }
        if (ok) pp.pend |= 4u;
        wait_mb(2);
        tc::fence_after();
        // ---- this pixel's Y row, then the buffer takes group gi + 2's z ----------
        // (tcgen05.ld is warp-collective: every lane loads; lanes outside the
        // image have v = 0, hence Y = 0, and add zeros at in-range indices)
        uint32_t yr[NY8][8];
        if (ok) {
#pragma unroll
            for (int c = 0; c < NY8; ++c) tc::tmem_ld8_nowait(tbuf + lane_base + 8 * c, yr[c]);
            tc::tmem_wait_ld();
        }
        tc::fence_before();
        tc::wg_sync(bar);
        tc::fence_after();
        if (ok && gi + 2 < NG) {
            if (wt == 0) issue_z(gi + 2);
            pp.pend |= 1u << zb;
        }
        // ---- scatter h(p - off(tap)) += Y[p][tap], one kernel row per phase ------
        if (ok) scatter(nb, r, yr);
    }
    }

    // ---- epilogue: g = fold(h), u_t = prox(u_{t-1} - g) ---------------------------
    tc::wg_sync(bar);
    if (ok) {
        const float lam = __ldg(a.lam);
        const int wy0 = tile_split(a.ty, TH, H, a.tiles_y, R), wy1 = tile_split(a.ty + 1, TH, H, a.tiles_y, R);
        const int wx0 = tile_split(a.tx, TW, W, a.tiles_x, R), wx1 = tile_split(a.tx + 1, TW, W, a.tiles_x, R);
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
            for (int p = 0; p < nsy; ++p)
                for (int q = 0; q < nsx; ++q)
                    gsum += sH[(sy[p] - (y0 - 2 * R)) * C::HPITCH + sx[q] - (x0 - 2 * R)];
            const float up = __ldcg(uin + (size_t)qy * a.pitch + qx);
            const float fv = __ldg(a.f + (size_t)qy * a.pitch + qx);
            a.u_out[(size_t)qy * a.pitch + qx] = stage_out(up, gsum, fv, lam, a.dterm, a.proj_c);
        }
    }
    return ok;
}

// The persistent CTA: a contiguous run of the source's tiles, split into runs
// of one parameter set; per run the CTA stages the set's operands and its
// warpgroups take the run's tiles in turn.  err receives TNRD_ERR_TIMEOUT (4)
// when a warpgroup gave up waiting for its MMAs (it then skips its remaining
// tiles, waits a bounded time for the MMAs still in flight, and the CTA frees
// its TMEM as usual).
template <int KS, int NK, int NB, bool BF, bool X3, class Src>
__device__ __forceinline__ void tc_run(const Src& src, unsigned char* smem, int* err)
{
    using C = TcCfg<KS, NK, NB, BF, X3>;
    constexpr long long WAIT_LIMIT = 1ll << 31;
    const int tid = threadIdx.x, wg = tid >> 7, wt = tid & 127;
    const int bar = 1 + wg;   // named barrier of this warpgroup (0 is the CTA's)
    unsigned char* wgs = smem + C::OFF_WG + (size_t)wg * C::WG_BYTES;
    uint64_t* mb = reinterpret_cast<uint64_t*>(wgs + C::WG_MISC);   // z buffers 0, 1; Y
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + C::OFF_TMEM);
    if (wt == 0) {
        tc::mbar_init(mb + 0, 1);
        tc::mbar_init(mb + 1, 1);
        tc::mbar_init(mb + 2, 1);
    }
    if (tid < 32) tc::tmem_alloc(tslot, C::TMEM_COLS);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t tmem = tbase + (uint32_t)(C::TMEM_WG * wg);

    TcPipe pp;
    int ok = 1;
    const int nt = src.ntiles();
    const int per = (nt + (int)gridDim.x - 1) / (int)gridDim.x;
    const int c0 = min(nt, (int)blockIdx.x * per), c1 = min(nt, c0 + per);
#pragma unroll 1
    for (int s0 = c0; s0 < c1;) {
        const int set = src.set_of(s0);
        const int s1 = src.seg_end(s0, c1);
        const TcSet ps = src.params(set);
        __syncthreads();   // every warpgroup's MMAs of the previous set have completed
        tc_stage_consts<KS, NK, NB, BF, X3>(ps, smem, tid);
        tc::fence_async_smem();
        __syncthreads();
        // the tiles read u_{t-1} (the previous stage's output) and overwrite the
        // buffer that stage read: wait for it (programmatic dependent launch)
        tc::pdl_wait();
        const RbfConst rc = *ps.rc;
#pragma unroll 1
        for (int s = s0 + wg; s < s1 && ok; s += C::NWG)
            ok = tc_tile<KS, NK, NB, BF, X3>(src.tile(s), rc, smem, wgs, tmem, mb, pp, wt, bar);
        s0 = s1;
    }
    if (!ok) {
        // give the MMAs in flight a bounded chance to finish before TMEM is freed
        for (int b = 0; b < 3; ++b)
            if (pp.pend & (1u << b)) tc::mbar_wait(mb + b, (pp.ph >> b) & 1u, WAIT_LIMIT);
        if (wt == 0) atomicExch(err, 4);
    }
    tc::fence_before();
    __syncthreads();
    if (tid < 32) tc::tmem_dealloc(tbase, C::TMEM_COLS);
}

// Per-call stage: a persistent grid of at most one CTA per SM over the N
// images' tiles.
template <int KS, int NK, int NB, bool BF, bool X3>
__global__ void __launch_bounds__(TcCfg<KS, NK, NB, BF, X3>::NTHREADS, 1)
tc_stage_fwd(const __grid_constant__ StageArgs a, int n_img)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    tc::pdl_launch_dependents();   // the next stage may launch; it waits before touching u
    const TcCallSrc src{&a, n_img};
    tc_run<KS, NK, NB, BF, X3>(src, smem, &g_tc_error);
}

// Stage t of a batched plan over every image's tiles.
template <int KS, int NK, int NB, bool BF, bool X3>
__global__ void __launch_bounds__(TcCfg<KS, NK, NB, BF, X3>::NTHREADS, 1)
tc_batch_fwd(const __grid_constant__ BatchArgs a, int t)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const TcBatchSrc<KS, NK> src{&a, t};
    tc_run<KS, NK, NB, BF, X3>(src, smem, a.status);
}

}  // namespace tnrd
