// Kernel argument structs and compile-time tile configurations, shared by
// the kernel translation units and the host-side dispatcher.
#pragma once
#include <cuda.h>
#include "common.cuh"

namespace tnrd {

struct StageArgs {
    const float* u_in;     // [N][H][pitch]  u_{t-1}
    float* u_out;          // [N][H][pitch]  u_t
    const float* f;        // [N][H][pitch]
    long long img_stride;  // floats between images
    int H, W, pitch;
    int tiles_x, tiles_y;
    const float* k;        // [nfilt][ks][ks] of this stage
    const float* w;        // [nfilt][nrbf] of this stage
    const float* lam;      // &lambda[t]
    int nrbf;
    int dterm;             // tnrd_data_term of the model
    float proj_c;          // projection floor (dterm 2)
    RbfConst rc;
    int th, te;            // row tiling (row_tile): tile height <= the kernel's TH, short border tiles
    int use_tma;           // umap describes u_in: stage tiles with bulk tensor copies
    int* err;              // device status word (TNRD_ERR_TIMEOUT on a copy that never landed)
    long long wait_limit;  // SM cycles per wait on a tile copy
    int tx_extra;          // test hook: extra bytes the copy's mbarrier expects (0)
    CUtensorMap umap;      // [N][H][pitch] float32 view of u_in, box of the kernel's staged tile
};

// All T stages of a small image batch in one launch (fused_pairc_cascade):
// stage t reads u_{t-1} (f for t = 0) and writes u_t to `stage_out(t)`; the
// CTAs meet at a grid-wide barrier (counter, zeroed before the launch)
// between stages.
struct CascadeArgs {
    const float* f;        // [N][H][pitch]  u_0
    float* u;              // u_T, or [T+1][N][H][pitch] all stages (keep)
    float* pp;             // ping-pong batch (keep == 0, T >= 2)
    long long img_stride;  // floats between images
    long long batch;       // floats of one [N][H][pitch] batch
    int H, W, pitch;
    int tiles_x, tiles_y;
    int th, te;
    int T, keep;
    const float* k;        // [T][nfilt][ks][ks]
    const float* w;        // [T][nfilt][nrbf]
    const float* lam;      // [T]
    int nrbf;
    int dterm;
    float proj_c;
    RbfConst rc;
    int* counter;          // grid barrier (one int, zero at launch)
    int* err;              // status word: TNRD_ERR_TIMEOUT if a barrier wait ran out
    long long wait_limit;  // SM cycles per barrier wait
};

// One tile of one stage for stage_tile(): pointers already offset to the image.
struct TileJob {
    const float* u_in;
    float* u_out;
    const float* f;
    int H, W, pitch;
    int tiles_x, tiles_y, ty, tx;
    const float* k;
    const float* w;
    const float* lam;
    int nrbf;
    int dterm;
    float proj_c;
    const RbfConst* rc;
    int th = 0, te = 0;                  // row tiling (row_tile); th <= the kernel's TH
    const CUtensorMap* umap = nullptr;   // tensor map of u_in (null: symmetric gather)
    int img = 0;                         // z coordinate of this image in umap
    int* err = nullptr;                  // status word for a copy that timed out
    long long wait_limit = 1ll << 31;    // SM cycles per wait on the copy (about one second)
    int tx_extra = 0;                    // test hook: extra bytes the copy's mbarrier expects
};

// Warps of a column-pair CTA holding nk_cta filters (each warp walks
// nk_cta / warps of them).
__host__ __device__ constexpr int pair_nwarp(int nk_cta)
{
    return nk_cta % 8 == 0 ? 8 : nk_cta % 6 == 0 ? 6 : nk_cta % 4 == 0 ? 4 : nk_cta % 3 == 0 ? 3
         : nk_cta % 2 == 0 ? 2 : 1;
}

template <int KS, int NK, int TH>
struct FusedCfg {
    static constexpr int R = KS / 2;
    static constexpr int TW = 32 - 2 * R;          // output columns per tile
    static constexpr int NWARP = NK >= 8 ? 8 : NK;
    static constexpr int NTHREADS = NWARP * 32;
    static constexpr int MINB = 2;                 // CTAs per SM the registers are sized for
    static constexpr int FPW = NK / NWARP;
    static_assert(NK % NWARP == 0, "filters must split evenly over the warps");
    static constexpr int GROUPS_EXT = (TH + 6 * R + KS - 1) / KS;
    static constexpr int GROUPS_INT = (TH + 4 * R + KS - 1) / KS;
    static constexpr int UH_EXT = GROUPS_EXT * KS;
    static constexpr int UH_INT = R + GROUPS_INT * KS;
    static constexpr int UH = UH_EXT > UH_INT ? UH_EXT : UH_INT;   // u rows from y0 - 3R
    static constexpr int UW = 32 + 2 * R;          // u cols from x0 - 2R
    static constexpr int UP = staged_pitch(UW);    // staged row pitch (16-byte aligned box)
    static constexpr int H_FL = (TH + 2 * R) * 32; // h rows from y0 - R, one column per lane
    static constexpr int KPAD = (KS * KS + 3) & ~3;
    static constexpr int WPADN = MAX_NRBF + 2 * RBF_WPAD;
    static constexpr int U_FL = UH * UP;
    static constexpr int KW_FL = KPAD + WPADN;
    static constexpr int SMEM_FL = U_FL + NWARP * (H_FL + KW_FL);
    static constexpr int TAB_OFF = (SMEM_FL + 3) & ~3;   // 16-byte aligned table base
    // dynamic shared memory: the fixed part plus one RBF coefficient table per warp
    static constexpr size_t smem_bytes(int nrbf)
    {
        (void)nrbf;
        return sizeof(float) * ((size_t)TAB_OFF + (size_t)NWARP * RBF_TP * RBF_NCOEF);
    }
};

// Tile origin along one axis: tiles of size T cover [0, n); the last tile is
// shifted back to end at n (when n >= T) so that every tile lies inside the
// image and only the first and the last tile touch a border.
__host__ __device__ __forceinline__ int tile_origin(int t, int T, int n)
{
    return (n >= T) ? min(t * T, n - T) : 0;
}

// Start of the range of rows (or columns) that tile t writes; tile t writes
// [tile_split(t), tile_split(t+1)).  Rows within R of a border need the mirror
// images of their adjoint values, which only the first (top) and the last
// (bottom) tile compute, so the split between the last two tiles is moved to
// at most n - R, and never below R when there are only two tiles (n >= 2R).
__host__ __device__ __forceinline__ int tile_split(int t, int T, int n, int nt, int R)
{
    if (t <= 0) return 0;
    if (t >= nt) return n;
    if (t == nt - 1) return min(t * T, n - R);
    return t * T;
}

// Row range of tile t of nt along an image axis of n rows.
//   te == 0: uniform tiles of th rows, the last shifted back to end at n
//            (tile_origin / tile_split).
//   te > 0 (short border tiles; requires n >= 2 te + th): the first tile is
//            [0, te), the last [n - te, n), the others th rows from te on, the
//            last of them shifted back to end at n - te.  With te = th - 2R a
//            border tile walks as many steps as an interior one (th + 4R).
// Tile t covers [y0, y0 + h) and writes [wy0, wy1); the written ranges
// partition [0, n), rows within R of a border go to the border tiles, and the
// last interior tile writes at least 2R rows.
struct RowTile {
    int y0, h, wy0, wy1;
};

__host__ __device__ __forceinline__ int row_tiles(int n, int th, int te)
{
    return te > 0 ? 2 + (n - 2 * te + th - 1) / th : (n + th - 1) / th;
}

__host__ __device__ __forceinline__ int row_split_short(int s, int nt, int n, int th, int te, int R)
{
    if (s <= 0) return 0;
    if (s >= nt) return n;
    if (s == nt - 1) return n - te;
    const int v = te + (s - 1) * th;
    return (s == nt - 2) ? min(v, n - te - 2 * R) : v;
}

__host__ __device__ __forceinline__ RowTile row_tile(int t, int nt, int n, int th, int te, int R)
{
    RowTile r;
    if (te <= 0) {
        r.y0 = tile_origin(t, th, n);
        r.h = th;
        r.wy0 = tile_split(t, th, n, nt, R);
        r.wy1 = tile_split(t + 1, th, n, nt, R);
        return r;
    }
    if (t == 0) {
        r.y0 = 0;
        r.h = te;
    } else if (t == nt - 1) {
        r.y0 = n - te;
        r.h = te;
    } else {
        r.y0 = min(te + (t - 1) * th, n - te - th);
        r.h = th;
    }
    r.wy0 = row_split_short(t, nt, n, th, te, R);
    r.wy1 = row_split_short(t + 1, nt, n, th, te, R);
    return r;
}

struct UnfArgs {
    const float* u_in;
    float* u_out;
    const float* f;
    float* v;              // [N][nfilt][H][pitch]
    float* g;              // [N][H][pitch]
    long long img_stride;  // floats between images of u/f/g
    int H, W, pitch;
    int nfilt;
    const float* k;        // [nfilt][ks][ks]
    const float* w;        // [nfilt][nrbf]
    const float* lam;
    int nrbf;
    int dterm;
    float proj_c;
    RbfConst rc;
};


// ---------------------------------------------------------------------------
// Backward stage (Sec. 3.2).  One stage t is five launches:
//   bwd_prep  : d = y .* e (Eq. derv2), per-block sums of x .* e (Eq. derv4)
//   bwd_zb    : z_i = K_i u, b_i = K_i d, c_i = -phi_i'(z_i) .* b_i, v_i = phi_i(z_i)
//               on each tile's own pixels, written to the c and v planes, and
//               per-tile dL/dw partials
//   bwd_adj   : e_{t-1} = d + sum_i K_i^T c_i (Eq. derv1-1) from the c planes
//   bwd_dk    : per-tile dL/dk partials sum_p c_i(p) u(p+.) - v_i(p) d(p+.)
//   bwd_reduce: fixed-order sums of all partials into this stage's gradients
// ---------------------------------------------------------------------------
struct BwdArgs {
    const float* u_prev;   // u_{t-1}   [N][H][pitch]
    const float* u_cur;    // u_t       [N][H][pitch]
    const float* f;        //           [N][H][pitch]
    const float* e_cur;    // dL/du_t   [N][H][pitch]
    float* d;              // s .* e    [N][H][pitch] (s = du_t/du~; y for dterm 0)
    float* d_id;           // (1 - psi') d [N][H][pitch]: identity path (dterm != 0)
    float* e_prev;         // dL/du_{t-1} [N][H][pitch]
    float* cpl;            // c planes  [N][nfilt][H][pitch]
    float* vpl;            // v planes  [N][nfilt][H][pitch]
    float* part_w;         // [N * zb tiles][nfilt][nrbf]
    float* part_k;         // [N * dk tiles][nfilt][ks*ks]
    float* part_l;         // [N * prep blocks]
    long long img_stride;  // floats between images of a plane set
    int H, W, pitch;
    int zb_tiles_x, zb_tiles_y;    // bwd_zb tiling (32 x ZB_TH, plain)
    int tiles_x, tiles_y;          // bwd_adj tiling (as the fused forward)
    int dk_tiles_x, dk_tiles_y;
    int prep_blocks;               // per image
    const float* k;
    const float* w;
    const float* lam;
    int nfilt, nrbf;
    int dterm;
    float proj_c;
    RbfConst rc;
};

// bwd_zb: tiles of 32 columns (one per lane) x TH rows that do not overlap;
// u and d are staged with an R-wide symmetric halo.  Each warp owns nfilt /
// NWARP filters and keeps, per filter, a private dL/dw histogram per lane with
// 2 RBF_WIN guard bins on each side (bin j at row j + 2 RBF_WIN), so that the
// 13 window bins of any clamped z need no bounds test.
template <int KS, int NK, int TH>
struct ZbCfg {
    static constexpr int R = KS / 2;
    static constexpr int NWARP = NK >= 8 ? 8 : NK;
    static constexpr int NTHREADS = NWARP * 32;
    static constexpr int FPW = NK / NWARP;
    static_assert(NK % NWARP == 0, "filters must split evenly over the warps");
    static constexpr int GROUPS = (TH + 2 * R + KS - 1) / KS;   // walk groups of KS steps
    static constexpr int UH = GROUPS * KS;                       // u/d rows from y0 - R
    static constexpr int UW = 32 + 2 * R;                        // u/d cols from x0 - R
    static constexpr int UP = UW;
    static constexpr int U_FL = UH * UP;
    static constexpr int HIST_ROWS = MAX_NRBF + 4 * RBF_WIN;
    static constexpr int HIST_FL = HIST_ROWS * 32;
    static constexpr int KPAD = (KS * KS + 3) & ~3;
    static constexpr int WPADN = (MAX_NRBF + 2 * RBF_WPAD + 3) & ~3;
    static constexpr int PW_FL = HIST_FL + KPAD + WPADN;         // per warp
    static constexpr int SMEM_FL = 2 * U_FL + NWARP * PW_FL;
    static constexpr size_t SMEM_BYTES = sizeof(float) * (size_t)SMEM_FL;
};

// bwd_adj: tiles as the fused forward stage (TH rows x 32 - 2R columns, lane j
// on column x0 - R + j); each warp accumulates the zero-extended adjoint h of
// its filters in a private buffer of TH + 2R rows.
template <int KS, int NK, int TH>
struct AdjCfg {
    static constexpr int R = KS / 2;
    static constexpr int TW = 32 - 2 * R;
    static constexpr int NWARP = NK >= 8 ? 8 : NK;
    static constexpr int NTHREADS = NWARP * 32;
    static constexpr int FPW = NK / NWARP;
    static_assert(NK % NWARP == 0, "filters must split evenly over the warps");
    static constexpr int H_FL = (TH + 2 * R) * 32;
    static constexpr size_t SMEM_BYTES = sizeof(float) * (size_t)NWARP * H_FL;
};

// Quality indexes (tnrd_quality): per-tile FP64 partial sums, then the indexes.
enum QualitySum {
    Q_SE = 0,      // sum (x - y)^2
    Q_SSIM,        // sum of the SSIM of the tile's windows
    Q_LA, Q_LB,    // sums of the Laplacians of x and y
    Q_LAA, Q_LBB, Q_LAB,
    Q_R, Q_RR,     // sums of f / y and its square
    Q_SY, Q_SYY,   // sums of y and y^2
    QSUMS
};
constexpr int QOUT = 6;   // psnr, mssim, ec, ri_mean, ri_var, cv
struct QualityArgs {
    const float* ref;      // [N][H][pitch] or null
    const float* img;      // [N][H][pitch] despeckled
    const float* noisy;    // [N][H][pitch] or null
    long long img_stride;
    int H, W, pitch;
    int tiles_x, tiles_y;
    float peak;
    double* part;          // [N][tiles][QSUMS]
    double* out;           // [N][QOUT]
    float g1[11];          // normalised 1-D SSIM window, sigma = 1.5
    float g2[121];         // its outer product (the 2-D window), row-major
};

// Gradient reduction: up to three (partials, rows, parameters, output) sets in
// one launch, blockIdx.y selecting the set.
struct RedSet {
    const float* part;   // [nrows][nparam]
    int nrows, nparam;
    float* out;          // [nparam]
};
struct RedArgs {
    RedSet s[3];
};

// ---------------------------------------------------------------------------
// Persistent batched forward (tnrd_batch_forward).
// ---------------------------------------------------------------------------
struct BatchImg {
    const float* f;
    float* u;          // final output u_T
    float* tmp;        // inter-stage image (ping-pong partner of u)
    int H, W, pitch;
    int tiles_x, tiles_y, tile_base;   // tiles of this image: [tile_base, +tiles_x*tiles_y)
    int set;
};

struct BatchSet {
    const float* k;    // [T][nfilt][ks][ks]
    const float* w;    // [T][nfilt][nrbf]
    const float* lam;  // [T]
    int dterm;         // tnrd_data_term of this parameter set
    float proj_c;
    RbfConst rc;
};

struct BatchArgs {
    const BatchImg* imgs;
    const BatchSet* sets;
    const int2* tile_img;        // global tile -> (image, tile within the image)
    int* work_counter;
    int* tile_done;              // per global tile: stages completed
    int* status;                 // 0, or TNRD_ERR_TIMEOUT
    const long long* wait_limit; // cycles
    int ntiles;                  // tiles per stage over all images
    int T;
    int nfilt, ksize, nrbf;
    const CUtensorMap* maps;     // per image: f, u, tmp views for the per-stage kernel (or null)
    int* err;                    // status word for the per-stage kernel's copies (the plan's)
};

// ---------------------------------------------------------------------------
// Tensor-core stage (TNRD_ALGO_TC_TF32 / _BF16 / _TF32X3): filter bank and
// adjoint as implicit GEMMs on tcgen05, phi and the prox on the CUDA cores.
// One persistent CTA per SM of NWG independent warpgroups; each warpgroup works
// through its own tiles, the GEMMs' filter operands and the RBF weights are
// staged once per CTA (per parameter set) and shared.  X3: every operand is
// kept as its TF32 high part and the TF32 rounding of the remainder, and each
// product is taken as lo*hi + hi*lo + hi*hi (three TF32 MMAs).
// ---------------------------------------------------------------------------
template <int KS, int NK, int NB, bool BF, bool X3 = false>
struct TcCfg {
    static_assert(!(BF && X3), "split operands are TF32 only");
    static constexpr int R = KS / 2;
    static constexpr int TW = 32 - 2 * R;        // output columns per tile
    static constexpr int ZR = 16 * NB;           // z rows per tile (NB blocks of 16)
    static constexpr int TH = ZR - 2 * R;        // output rows per tile
    static constexpr int ESZ = BF ? 2 : 4;       // bytes per operand element
    static constexpr int KMMA = BF ? 16 : 8;     // K of one MMA (32 bytes)
    static constexpr int KCORE = BF ? 8 : 4;     // K elements of one core matrix row (16 bytes)
    static constexpr int NSPL = X3 ? 2 : 1;      // copies of each operand (X3: high, low part)
    // ring layout (a two-residue ring of u copies, one z buffer, V one round of
    // 16 filters): split TF32, and TF32 with three row blocks, whose taller tiles
    // fit three warpgroups only so
    static constexpr bool RING = X3 || (!BF && NB == 3);
    static constexpr int NPAD = (NK + 15) / 16 * 16;                 // N of the filter-bank GEMM
    static constexpr int NKP = (NK + KMMA - 1) / KMMA * KMMA;        // K of the adjoint GEMM
    static constexpr int NT = (KS * KS + 15) / 16 * 16;  // N of the adjoint GEMM (taps)
    static_assert(NPAD <= 64 && NT <= 64, "TMEM: one 64-column buffer holds z or Y");
    static constexpr int UROWS = ZR + 2 * R;     // u rows from y0 - 2R
    // u operand row of one residue class r, in bytes:
    //  TF32: a copy shifted by r columns, 36 floats (A core row m = floats 4m..4m+3);
    //  BF16: 10 chunks of 8 values, chunk c = u columns 4c + r .. 4c + r + 7
    //        (A core row m = chunk m; the second K core, taps 8..15, is chunk m + 2)
    static constexpr int UPITCH = 36;            // TF32 floats per row
    static constexpr int UCHUNKS = 10;           // BF16 chunks per row
    static constexpr int UROWB = BF ? UCHUNKS * 16 : UPITCH * 4;
    // raw u rows of the tile (columns x0 - 2R ..), staged once per tile and
    // copied into the residue operands: TF32 reads 39 columns, BF16 47
    static constexpr int RAWC = BF ? 47 : 39;
    static constexpr int RAWP = BF ? 48 : 40;
    static constexpr int HROWS = ZR + 2 * R;     // h rows from y0 - 2R
    static constexpr int HPITCH = 41;            // h columns from x0 - 2R (41 = 1 mod 4: no bank conflicts)
    static constexpr int WPADN = MAX_NRBF + 2 * RBF_WPAD;
    static constexpr size_t al(size_t x) { return (x + 127) / 128 * 128; }
    static constexpr size_t mx(size_t a, size_t b) { return a > b ? a : b; }
    // shared by the CTA's warpgroups (X3: the low parts right after the high parts)
    static constexpr size_t BZ_BYTES = (size_t)ESZ * KS * NPAD * KMMA;
    static constexpr size_t KM_BYTES = (size_t)ESZ * NT * NKP;
    static constexpr size_t OFF_BZ = 0;
    static constexpr size_t OFF_KM = al(OFF_BZ + NSPL * BZ_BYTES);
    static constexpr size_t OFF_W = al(OFF_KM + NSPL * KM_BYTES);
    static constexpr int NR = (NK + 15) / 16;    // rounds of 16 filters (RBF weight table)
    static constexpr size_t OFF_WG = al(OFF_W + 8ull * NR * TC_ROWS * 16);
    // per warpgroup: u operands, V (the raw u rows before the first group), h, barriers.
    // U holds the four residue copies of u, or (X3) a ring of two residues, each
    // as high and low parts, built from the raw rows that stay for the whole tile.
    // V holds all NKP filters of a group, or (X3) one round of 16 filters, high and
    // low parts: the round's adjoint MMAs run while phi works on the next round.
    static constexpr size_t U_SLOT = (size_t)UROWS * UROWB;     // one residue copy
    static constexpr size_t U_BYTES = (RING ? 2 * NSPL : 4) * U_SLOT;
    static constexpr size_t RAW_BYTES = 4ull * UROWS * RAWP;
    static constexpr int VF = RING ? 16 : NKP;   // filters of V held at once
    static constexpr size_t VLO = (size_t)ESZ * 128 * VF;   // byte offset of V's low parts
    static constexpr size_t WG_U = 0;
    static constexpr size_t WG_RAW = al(WG_U + U_BYTES);    // ring layout only
    static constexpr size_t WG_V = RING ? al(WG_RAW + RAW_BYTES) : WG_RAW;
    static constexpr size_t WG_H = al(WG_V + (RING ? NSPL * VLO : mx(VLO, RAW_BYTES)));
    static constexpr size_t WG_MISC = al(WG_H + 4ull * HROWS * HPITCH);
    static constexpr size_t WG_BYTES = al(WG_MISC + 32);
    static constexpr size_t SMEM_MAX = 227 * 1024;
    static constexpr int fit_wg(int n) { return (n > 1 && OFF_WG + (size_t)n * WG_BYTES + 16 > SMEM_MAX) ? fit_wg(n - 1) : n; }
    // warpgroups per CTA; TMEM columns of one (128): two z buffers that also
    // take Y, or (ring) one z buffer at 0..63 and the adjoint's Y at 64..127
    static constexpr int NWG = fit_wg(RING ? 3 : 4);   // ring: at most three (registers)
    static constexpr int TMEM_WG = 128;
    static constexpr int NTHREADS = 128 * NWG;
    static constexpr size_t OFF_TMEM = OFF_WG + (size_t)NWG * WG_BYTES;
    static constexpr size_t SMEM_BYTES = OFF_TMEM + 16;
    static constexpr uint32_t TMEM_COLS = NWG * TMEM_WG <= 256 ? 256 : 512;
    static_assert(NWG * TMEM_WG <= 512, "TMEM");
    static_assert(SMEM_BYTES <= SMEM_MAX, "shared memory");
};

}  // namespace tnrd
