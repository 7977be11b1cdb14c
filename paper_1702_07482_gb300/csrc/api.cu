// C ABI of libtnrd.so (declared in include/tnrd.h): argument validation,
// workspace layout, stage scheduling and kernel selection.  No allocation and
// no host synchronisation happens here.
#include "tnrd.h"
#include "launch.h"

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

namespace {

thread_local std::string g_err;

tnrd_status fail(tnrd_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

}  // namespace

namespace tnrd {

tnrd_status set_error(tnrd_status s, const char* msg)
{
    g_err = msg;
    return s;
}

}  // namespace tnrd

namespace {

tnrd_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(TNRD_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

bool supported_model(int ks, int nk)
{
    return (ks == 3 && nk == 4) || (ks == 5 && nk == 24) || (ks == 7 && nk == 48);
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

tnrd_status check_params(const tnrd_params* p)
{
    if (!p) return fail(TNRD_ERR_INVALID_ARG, "params is null");
    if (p->T < 1) return fail(TNRD_ERR_INVALID_ARG, "T = %d < 1", p->T);
    if (!supported_model(p->ksize, p->nfilt))
        return fail(TNRD_ERR_UNSUPPORTED, "(ksize, nfilt) = (%d, %d) not built; "
                    "supported: (3,4), (5,24), (7,48)", p->ksize, p->nfilt);
    if (p->nrbf < 1 || p->nrbf > tnrd::MAX_NRBF)
        return fail(TNRD_ERR_UNSUPPORTED, "nrbf = %d outside [1, %d]", p->nrbf, tnrd::MAX_NRBF);
    if (!(p->rbf_gamma > 0.0f) || !(p->rbf_delta >= p->rbf_gamma) || !std::isfinite(p->rbf_mu0))
        return fail(TNRD_ERR_UNSUPPORTED, "RBF spacing must satisfy delta >= gamma > 0 "
                    "(delta = %g, gamma = %g)", p->rbf_delta, p->rbf_gamma);
    if (!p->filters || !p->rbf_w || !p->lambda)
        return fail(TNRD_ERR_INVALID_ARG, "null parameter array");
    if (p->data_term != TNRD_DATA_IDIV && p->data_term != TNRD_DATA_GAUSS &&
        p->data_term != TNRD_DATA_PROJ)
        return fail(TNRD_ERR_INVALID_ARG, "data_term = %d is not a tnrd_data_term", p->data_term);
    if (p->data_term == TNRD_DATA_PROJ && !(p->proj_c > 0.0f && std::isfinite(p->proj_c)))
        return fail(TNRD_ERR_INVALID_ARG, "proj_c = %g must be a positive number", p->proj_c);
    return TNRD_OK;
}

tnrd_status check_images(int N, int H, int W, int pitch, int ks)
{
    if (N < 0) return fail(TNRD_ERR_INVALID_ARG, "N = %d < 0", N);
    if (H < ks || W < ks)
        return fail(TNRD_ERR_INVALID_ARG, "image %d x %d smaller than the %d x %d filter", H, W, ks, ks);
    if (pitch < W || pitch % 4 != 0)
        return fail(TNRD_ERR_INVALID_ARG, "pitch %d must be >= W = %d and a multiple of 4", pitch, W);
    if ((long long)H * (long long)pitch >= (1LL << 31))
        return fail(TNRD_ERR_INVALID_ARG, "image of %d x %d (pitch %d) too large", H, W, pitch);
    if (N > 65535) return fail(TNRD_ERR_INVALID_ARG, "N = %d > 65535", N);
    return TNRD_OK;
}

tnrd::RbfConst make_rbf(const tnrd_params* p)
{
    tnrd::RbfConst rc{};
    const double mu0 = p->rbf_mu0, d = p->rbf_delta, g = p->rbf_gamma;
    const int W = tnrd::RBF_WIN;
    rc.mu0 = (float)mu0;
    rc.delta = (float)d;
    rc.inv_delta = (float)(1.0 / d);
    rc.zlo = (float)(mu0 - (W + 0.49) * d);
    rc.zhi = (float)(mu0 + (p->nrbf - 1 + W + 0.49) * d);
    rc.t_off = (float)(-mu0 / d);
    rc.tmax = (float)(p->nrbf - 1 + W);
    const double log2e = 1.4426950408889634;
    rc.c_q2 = (float)(log2e * d / (g * g));
    rc.c_p2a = (float)(log2e / (2.0 * g * g));
    rc.c_p2b = (float)(log2e * W * d / (g * g));
    rc.c_p2b_tc = (float)(log2e * tnrd::TC_WIN * d / (g * g));
    rc.cq = (float)(d / (g * g));
    rc.half_inv_g2 = (float)(1.0 / (2.0 * g * g));
    rc.inv_g2 = (float)(1.0 / (g * g));
    rc.jmax = p->nrbf - 1 + W;
    for (int m = 0; m <= W; ++m) rc.E[m] = (float)std::exp(-(double)m * m * d * d / (2.0 * g * g));
    return rc;
}

// Estimated duration, in walk steps of one CTA, of one fused stage launch over
// N images of H x W: tiles of th x tw pixels (border tile rows te, 0: th; see
// row_tile), `split` CTAs per tile, `slots` CTAs resident at once (two per
// SM).  A tile in the first or last tile row walks te + 6R steps, the others
// th + 4R.  When every CTA is resident at once the launch lasts as long as its
// longest CTA; otherwise the work spreads over the slots, plus half the
// longest CTA for the tail.
double fused_cost(int N, int H, int W, int th, int te, int tw, int R, int split, int slots)
{
    const long long ty = tnrd::row_tiles(H, th, te), tx = (W + tw - 1) / tw;
    const long long n_ext = ty >= 2 ? 2 : 1;
    const double w_ext = (te > 0 ? te : th) + 6 * R, w_int = th + 4 * R;
    const double w_max = ty > n_ext ? std::max(w_ext, w_int) : w_ext;
    const long long ctas = (long long)N * ty * tx * split;
    if (ctas <= slots) return w_max;
    const double per_col = n_ext * w_ext + (double)(ty - n_ext) * w_int;
    return (double)N * tx * split * per_col / slots + 0.5 * w_max;
}

// Row tiling of a fused launch: runtime tile height th, border tile rows te
// (0: uniform tiles), and the compiled kernel tile height kth >= th.
struct RowChoice {
    int th = 0, te = 0, kth = 0;
    double cost = 1e300;
};

// The row tiling of least estimated duration over th from the largest
// compiled tile height down to the smallest, uniform or with border tiles 2R
// shorter (so that they walk as many steps as interior ones).  Overrides:
// TNRD_FUSED_TH pins th, TNRD_FUSED_ROWS=uniform|short pins the tiling.
RowChoice pick_rows(const int* list, int R, int N, int H, int W, int tw, int split, int nsm)
{
    int kmin = 1 << 30, kmax = 0;
    for (const int* p = list; *p; ++p) {
        kmin = std::min(kmin, *p);
        kmax = std::max(kmax, *p);
    }
    int want = 0, rows = -1;   // rows: -1 either, 0 uniform, 1 short border tiles
    if (const char* env = std::getenv("TNRD_FUSED_TH")) want = std::atoi(env);
    if (const char* env = std::getenv("TNRD_FUSED_ROWS"))
        rows = !std::strcmp(env, "uniform") ? 0 : !std::strcmp(env, "short") ? 1 : -1;
    if (want > kmax || (want > 0 && want < 2 * R + 1)) want = 0;
    RowChoice best;
    for (int th = want ? want : kmax; th >= (want ? want : kmin); --th) {
        int kth = 0;
        for (const int* p = list; *p; ++p)
            if (*p >= th && (kth == 0 || *p < kth)) kth = *p;
        for (int shrt = 0; shrt < 2; ++shrt) {
            if (rows >= 0 && shrt != rows) continue;
            const int te = shrt ? th - 2 * R : 0;
            if (shrt && (te < 2 * R || H < 2 * te + th)) continue;
            const double cost = fused_cost(N, H, W, th, te, tw, R, split, 2 * nsm);
            if (cost < best.cost * 0.999) {
                best.th = th;
                best.te = te;
                best.kth = kth;
                best.cost = cost;
            }
        }
    }
    if (best.kth == 0) {   // the overrides allow nothing: uniform tiles of the pinned (or largest) height
        best.th = want ? want : kmax;
        best.te = 0;
        for (const int* p = list; *p; ++p)
            if (*p >= best.th && (best.kth == 0 || *p < best.kth)) best.kth = *p;
    }
    return best;
}

int device_sm_count()
{
    int nsm = 148;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return nsm;
}

// Fused forward kernel choice.  The one-column-per-lane kernel
// (fused_stage_fwd) is the default.  When it cannot give every SM two CTAs
// (a single small image), the column-pair kernel on two-CTA clusters
// (fused_pair2_fwd, half of the filters per CTA) spreads the same work over
// more CTAs; when even that leaves SMs without a CTA (a small image), clusters
// of four or eight CTAs per tile (fused_pairc_fwd) are weighed against it.
// Either way the row tiling minimises the estimated duration (pick_rows).
// TNRD_FUSED_KERNEL=lane|pair|pair2|pair4|pair8, TNRD_FUSED_TH and
// TNRD_FUSED_ROWS override the choice (tuning and measurement).
struct FusedChoice {
    int pair = 0;     // 0: one column per lane; 1: column pairs
    int th = 0;       // runtime tile height
    int te = 0;       // border tile rows (0: uniform tiles)
    int kth = 0;      // compiled tile height of the kernel (>= th)
    int nsplit = 1;
    int tw = 0;
};

// Estimated duration, in filter-walk steps, of a column-pair launch on
// clusters of `split` CTAs with row tiling rc: the longer of the longest
// CTA's sequential walks (fused_cost counts steps, each warp walks fpw
// filters) and the whole launch's warp-steps over the SMs at ten warps' worth
// of issue each (plus a per-CTA overhead of 8 steps per warp: staging, the
// cluster barriers and the epilogue).
double pair_split_cost(int nk, int split, const RowChoice& rc, int R, int N, int H, int W, int tw,
                       int nsm)
{
    const int nw = tnrd::pair_nwarp(nk / split), fpw = nk / split / nw;
    const long long tiles = (long long)N * tnrd::row_tiles(H, rc.th, rc.te) * ((W + tw - 1) / tw);
    const double walk = fused_cost(N, H, W, rc.th, rc.te, tw, R, split, 2 * nsm) * fpw;
    const double issue = (double)tiles * split * nw * (fpw * (rc.th + 4.0 * R) + 8.0) / (10.0 * nsm);
    return std::max(walk, issue);
}

FusedChoice pick_fused(int ks, int nk, int N, int H, int W)
{
    FusedChoice c;
    int force = -1;   // -1 auto, 0 lane, 1 pair, 2 pair2, 4 pair4, 8 pair8
    if (const char* env = std::getenv("TNRD_FUSED_KERNEL")) {
        if (!std::strcmp(env, "lane")) force = 0;
        else if (!std::strcmp(env, "pair")) force = 1;
        else if (!std::strcmp(env, "pair2")) force = 2;
        else if (!std::strcmp(env, "pair4") && nk % 4 == 0) force = 4;
        else if (!std::strcmp(env, "pair8") && nk % 8 == 0) force = 8;
    }
    const int R = ks / 2;
    const int nsm = device_sm_count();
    c.tw = 32 - 2 * R;
    RowChoice rc = pick_rows(tnrd::fused_th_list(ks), R, N, H, W, c.tw, 1, nsm);
    c.th = rc.th;
    c.te = rc.te;
    c.kth = rc.kth;
    const long long lane_ctas = (long long)N * tnrd::row_tiles(H, c.th, c.te) * ((W + c.tw - 1) / c.tw);
    if (force == 0) return c;
    if (force < 0 && lane_ctas >= 2LL * nsm) {
        // Enough tiles for the one-column kernel.  The two-CTA column-pair kernel
        // does the same work in fewer instructions (a pair step, two columns a
        // lane, costs 1.9 one-column steps: fitted to 16 x 2048^2 and 32 x 180^2 at
        // 7x7x48, where it measured 0.89x and 1.10x the one-column time) but its
        // 64 - 2R column tiles waste more of narrow images; the estimated
        // durations (walk steps x filters per warp x step cost) decide.
        if (ks != 7) return c;
        const int tw2 = 64 - 2 * R;
        const RowChoice r2 = pick_rows(tnrd::pair_th_list(ks), R, N, H, W, tw2, 2, nsm);
        const int fpw_lane = nk / std::min(8, nk);
        const int fpw_pair = nk / 2 / tnrd::pair_nwarp(nk / 2);
        const double lane_cost = rc.cost * fpw_lane, pair_cost = r2.cost * fpw_pair * 1.9;
        if (r2.kth == 0 || !(pair_cost < 0.95 * lane_cost)) return c;
        c.pair = 1;
        c.nsplit = 2;
        c.tw = tw2;
        c.th = r2.th;
        c.te = r2.te;
        c.kth = r2.kth;
        return c;
    }
    c.pair = 1;
    c.tw = 64 - 2 * R;
    if (force == 4 || force == 8) {
        c.nsplit = force;
        rc = pick_rows(tnrd::pair_cluster_th_list(ks), R, N, H, W, c.tw, force, nsm);
    } else {
        c.nsplit = (force == 1) ? 1 : 2;
        rc = pick_rows(tnrd::pair_th_list(ks), R, N, H, W, c.tw, c.nsplit, nsm);
        const long long ctas2 = 2LL * N * tnrd::row_tiles(H, rc.th, rc.te) * ((W + c.tw - 1) / c.tw);
        if (force < 0 && ctas2 < nsm) {
            double best = pair_split_cost(nk, 2, rc, R, N, H, W, c.tw, nsm);
            for (int split : {4, 8}) {
                if (nk % split) continue;
                const RowChoice rs = pick_rows(tnrd::pair_cluster_th_list(ks), R, N, H, W, c.tw, split, nsm);
                if (rs.kth == 0) continue;
                const double cost = pair_split_cost(nk, split, rs, R, N, H, W, c.tw, nsm);
                if (cost < 0.85 * best) {
                    best = cost;
                    rc = rs;
                    c.nsplit = split;
                }
            }
        }
    }
    c.th = rc.th;
    c.te = rc.te;
    c.kth = rc.kth;
    return c;
}

// Row blocks of 16 z rows per tensor-core tile: 3 for BF16 (its smaller
// operands leave room for three warpgroups with the taller tile), 2 for TF32
// (with three it runs the ring layout on three warpgroups, measured 3 % slower)
// and for split TF32 (built with two only).  TNRD_TC_NB=2|3 overrides for TF32
// and BF16.
bool is_tc(tnrd_algo algo)
{
    return algo == TNRD_ALGO_TC_TF32 || algo == TNRD_ALGO_TC_BF16 || algo == TNRD_ALGO_TC_TF32X3;
}

int tc_prec(tnrd_algo algo)
{
    return algo == TNRD_ALGO_TC_BF16 ? tnrd::TC_BF16 : algo == TNRD_ALGO_TC_TF32X3 ? tnrd::TC_TF32X3
                                                                                    : tnrd::TC_TF32;
}

const char* tc_name(tnrd_algo algo)
{
    return algo == TNRD_ALGO_TC_BF16 ? "bf16" : algo == TNRD_ALGO_TC_TF32X3 ? "tf32x3" : "tf32";
}

int pick_tc_nb(tnrd_algo algo)
{
    int nb = (algo == TNRD_ALGO_TC_BF16) ? 3 : 2;
    if (algo == TNRD_ALGO_TC_TF32X3) return 2;
    if (const char* env = std::getenv("TNRD_TC_NB")) {
        const int v = std::atoi(env);
        if (v == 2 || v == 3) nb = v;
    }
    return nb;
}

// Whether tnrd_forward runs all T stages in one launch (fused_pairc_cascade):
// the fused algorithm on images small enough for the cluster splits, T >= 2,
// and every cluster of the launch resident at once (occupancy query; false
// without a GPU).  TNRD_CASCADE=0 turns it off (comparison runs).
bool use_cascade(const tnrd_params* p, int N, int H, int W, tnrd_algo algo, FusedChoice* out)
{
    if (algo != TNRD_ALGO_FUSED || p->T < 2) return false;
    if (const char* env = std::getenv("TNRD_CASCADE"))
        if (!std::strcmp(env, "0")) return false;
    const FusedChoice fc = pick_fused(p->ksize, p->nfilt, N, H, W);
    if (!fc.pair || fc.nsplit <= 2) return false;
    const long long clusters = (long long)N * tnrd::row_tiles(H, fc.th, fc.te) * ((W + fc.tw - 1) / fc.tw);
    if (!tnrd::pair_cascade_fits(p->ksize, p->nfilt, fc.kth, fc.nsplit, clusters)) return false;
    if (out) *out = fc;
    return true;
}

struct FwdLayout {
    size_t pingpong = 0;   // offset of the ping-pong image batch
    size_t v = 0, g = 0;   // unfused response planes and adjoint plane
    size_t counter = 0;    // grid-barrier counter of the one-launch cascade
    bool cascade = false;
    size_t total = 0;
};

FwdLayout fwd_layout(const tnrd_params* p, int N, int H, int W, int pitch, int keep, tnrd_algo algo)
{
    FwdLayout L;
    const size_t batch = sizeof(float) * (size_t)N * H * pitch;
    size_t off = 0;
    if (!keep && p->T >= 2) {
        L.pingpong = off;
        off = align_up(off + batch, 256);
    }
    if (N > 0 && use_cascade(p, N, H, W, algo, nullptr)) {
        L.cascade = true;
        L.counter = off;
        off = align_up(off + sizeof(int), 256);
    }
    if (algo == TNRD_ALGO_UNFUSED) {
        L.v = off;
        off = align_up(off + batch * (size_t)p->nfilt, 256);
        L.g = off;
        off = align_up(off + batch, 256);
    }
    L.total = off;
    return L;
}

struct BwdLayout {
    size_t d = 0, did = 0, e0 = 0, e1 = 0, c = 0, v = 0, pw = 0, pk = 0, pl = 0, total = 0;
    int zb_tiles_x = 0, zb_tiles_y = 0, tiles_x = 0, tiles_y = 0, dk_tiles_x = 0,
        dk_tiles_y = 0, prep_blocks = 0;
};

BwdLayout bwd_layout(const tnrd_params* p, int N, int H, int W, int pitch)
{
    BwdLayout L;
    const int ks = p->ksize, R = ks / 2, tw = 32 - 2 * R, th = tnrd::bwd_tile_h(ks);
    L.zb_tiles_x = (W + 31) / 32;
    L.zb_tiles_y = (H + th - 1) / th;
    L.tiles_x = (W + tw - 1) / tw;
    L.tiles_y = (H + th - 1) / th;
    L.dk_tiles_x = (W + 31) / 32;
    L.dk_tiles_y = (H + th - 1) / th;
    L.prep_blocks = (H * W + 255) / 256;
    const size_t batch = sizeof(float) * (size_t)N * H * pitch;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off = align_up(off + bytes, 256); return o; };
    L.d = take(batch);
    if (p->data_term != TNRD_DATA_IDIV) L.did = take(batch);
    L.e0 = take(batch);
    L.e1 = take(batch);
    L.c = take(batch * (size_t)p->nfilt);
    L.v = take(batch * (size_t)p->nfilt);
    L.pw = take(sizeof(float) * (size_t)N * L.zb_tiles_x * L.zb_tiles_y * p->nfilt * p->nrbf);
    // dL/dk partials: the CUDA-core kernel's tiles or the tensor-core kernel's
    const size_t dk_rows = std::max((size_t)L.dk_tiles_x * L.dk_tiles_y, (size_t)tnrd::tc_dk_tiles(H, W));
    L.pk = take(sizeof(float) * (size_t)N * dk_rows * p->nfilt * ks * ks);
    L.pl = take(sizeof(float) * (size_t)N * L.prep_blocks);
    L.total = off;
    return L;
}

}  // namespace

extern "C" {

const char* tnrd_last_error(void) { return g_err.c_str(); }

tnrd_status tnrd_device_status(void)
{
    int v = 0;
    cudaError_t e = tnrd::tc_take_error(&v);
    if (e != cudaSuccess) return cuda_fail(e, "device status read");
    if (v != 0) return fail((tnrd_status)v, "a stage gave up waiting for its MMAs or its tile copy");
    return TNRD_OK;
}

tnrd_status tnrd_stage_wait_test(long long cycles, int never_complete)
{
    if (cycles < 0) return fail(TNRD_ERR_INVALID_ARG, "negative wait limit");
    tnrd::set_stage_wait_test(cycles, never_complete);
    return TNRD_OK;
}

int tnrd_version(void) { return 1 * 10000 + 0 * 100 + 0; }

size_t tnrd_workspace_size(tnrd_op op, const tnrd_params* params, int N, int H, int W,
                           int pitch, int keep_stages, tnrd_algo algo)
{
    if (check_params(params) != TNRD_OK) return 0;
    if (check_images(N, H, W, pitch, params->ksize) != TNRD_OK) return 0;
    if (op == TNRD_OP_FORWARD) return fwd_layout(params, N, H, W, pitch, keep_stages, algo).total;
    if (op == TNRD_OP_BACKWARD) return bwd_layout(params, N, H, W, pitch).total;
    return 0;
}

tnrd_status tnrd_forward_kernel(const tnrd_params* p, int N, int H, int W, tnrd_algo algo,
                                char* buf, size_t len)
{
    if (!buf || len == 0) return fail(TNRD_ERR_INVALID_ARG, "null or empty buffer");
    buf[0] = '\0';
    tnrd_status st = check_params(p);
    if (st != TNRD_OK) return st;
    st = check_images(N, H, W, (W + 3) & ~3, p->ksize);
    if (st != TNRD_OK) return st;
    const int ks = p->ksize, nk = p->nfilt, R = ks / 2;
    if (algo == TNRD_ALGO_FUSED) {
        const FusedChoice c = pick_fused(ks, nk, N, H, W);
        const char* staging = tnrd::tma_staging_enabled() ? "tma" : "gather";
        char rows[40] = "";
        if (c.te > 0) std::snprintf(rows, sizeof rows, " (border rows %d)", c.te);
        if (use_cascade(p, N, H, W, algo, nullptr)) {
            std::snprintf(buf, len, "fused_pairc_cascade<%d,%d,%d,%d> tiles %dx%d%s, all %d stages in "
                          "one launch, gather staging", ks, nk, c.kth, c.nsplit, c.th, c.tw, rows, p->T);
        } else {
            std::snprintf(buf, len, "%s<%d,%d,%d> tiles %dx%d%s, %s staging",
                          !c.pair ? "fused_stage_fwd" : c.nsplit == 2 ? "fused_pair2_fwd"
                          : c.nsplit == 4 ? "fused_pair4_fwd" : c.nsplit == 8 ? "fused_pair8_fwd"
                          : "fused_pair_fwd",
                          ks, nk, c.kth, c.th, c.tw, rows, staging);
        }
    } else if (algo == TNRD_ALGO_UNFUSED) {
        std::snprintf(buf, len, "unf_bank_phi + unf_adjoint + unf_prox <%d,%d>", ks, nk);
    } else if (is_tc(algo)) {
        const int nb = pick_tc_nb(algo);
        std::snprintf(buf, len, "tc_stage_fwd<%d,%d,%d,%s> tiles %dx%d", ks, nk, nb, tc_name(algo),
                      tnrd::tc_tile_h(ks, nb), 32 - 2 * R);
    } else {
        return fail(TNRD_ERR_INVALID_ARG, "unknown algo");
    }
    return TNRD_OK;
}

tnrd_status tnrd_forward(const tnrd_params* p, int N, int H, int W, int pitch,
                         const float* f, float* u, int keep_stages, tnrd_algo algo,
                         void* workspace, size_t workspace_bytes, cudaStream_t stream)
{
    tnrd_status st = check_params(p);
    if (st != TNRD_OK) return st;
    st = check_images(N, H, W, pitch, p->ksize);
    if (st != TNRD_OK) return st;
    if (algo != TNRD_ALGO_FUSED && algo != TNRD_ALGO_UNFUSED && !is_tc(algo))
        return fail(TNRD_ERR_UNSUPPORTED, "algo %d not available in tnrd_forward", (int)algo);
    if (N == 0) return TNRD_OK;
    if (!f || !u) return fail(TNRD_ERR_INVALID_ARG, "null image pointer");
    if (!aligned16(f) || !aligned16(u)) return fail(TNRD_ERR_INVALID_ARG, "f and u must be 16-byte aligned");
    const size_t plane = (size_t)H * pitch;
    const size_t batch = plane * (size_t)N;
    const size_t u_len = keep_stages ? batch * (size_t)(p->T + 1) : batch;
    if ((const float*)u < f + batch && f < (const float*)u + u_len)
        return fail(TNRD_ERR_INVALID_ARG, "u overlaps f");
    const FwdLayout L = fwd_layout(p, N, H, W, pitch, keep_stages, algo);
    if (L.total > 0 && (!workspace || workspace_bytes < L.total))
        return fail(TNRD_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", L.total,
                    workspace ? workspace_bytes : (size_t)0);
    char* ws = (char*)workspace;
    float* pp = L.total ? (float*)(ws + L.pingpong) : nullptr;

    if (keep_stages) {
        cudaError_t e = cudaMemcpyAsync(u, f, sizeof(float) * batch, cudaMemcpyDeviceToDevice, stream);
        if (e != cudaSuccess) return cuda_fail(e, "copy of u_0");
    }
    const tnrd::RbfConst rc = make_rbf(p);
    const int ks = p->ksize, nk = p->nfilt;
    const FusedChoice fc = (algo == TNRD_ALGO_FUSED) ? pick_fused(ks, nk, N, H, W) : FusedChoice{};
    const int tc_nb = pick_tc_nb(algo);

    if (L.cascade) {
        // all stages in one launch: zero the grid-barrier counter, then launch
        const FusedChoice& cc = fc;
        int* counter = (int*)(ws + L.counter);
        cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
        if (e != cudaSuccess) return cuda_fail(e, "cascade counter");
        tnrd::CascadeArgs c{};
        c.f = f;
        c.u = u;
        c.pp = pp;
        c.img_stride = (long long)plane;
        c.batch = (long long)batch;
        c.H = H;
        c.W = W;
        c.pitch = pitch;
        c.tiles_x = (W + cc.tw - 1) / cc.tw;
        c.tiles_y = tnrd::row_tiles(H, cc.th, cc.te);
        c.th = cc.th;
        c.te = cc.te;
        c.T = p->T;
        c.keep = keep_stages ? 1 : 0;
        c.k = p->filters;
        c.w = p->rbf_w;
        c.lam = p->lambda;
        c.nrbf = p->nrbf;
        c.dterm = p->data_term;
        c.proj_c = p->proj_c;
        c.rc = rc;
        c.counter = counter;
        c.err = tnrd::device_status_word();
        c.wait_limit = tnrd::stage_wait_limit();
        if (!c.err) return fail(TNRD_ERR_CUDA, "device status word unavailable");
        e = tnrd::launch_pair_cascade(ks, nk, cc.kth, cc.nsplit, c, N, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cascade launch");
        return TNRD_OK;
    }

    for (int t = 0; t < p->T; ++t) {
        const float* in;
        float* out;
        if (keep_stages) {
            in = (t == 0) ? f : u + (size_t)t * batch;
            out = u + (size_t)(t + 1) * batch;
        } else {
            // stage t writes u when (T-1-t) is even, so the last stage lands in u
            float* cur = ((p->T - 1 - t) % 2 == 0) ? u : pp;
            float* prev = ((p->T - t) % 2 == 0) ? u : pp;
            in = (t == 0) ? f : prev;
            out = cur;
        }
        const float* kt = p->filters + (size_t)t * nk * ks * ks;
        const float* wt = p->rbf_w + (size_t)t * nk * p->nrbf;
        cudaError_t e;
        if (algo == TNRD_ALGO_FUSED) {
            tnrd::StageArgs a{};
            a.u_in = in;
            a.u_out = out;
            a.f = f;
            a.img_stride = (long long)plane;
            a.H = H;
            a.W = W;
            a.pitch = pitch;
            a.tiles_x = (W + fc.tw - 1) / fc.tw;
            a.tiles_y = tnrd::row_tiles(H, fc.th, fc.te);
            a.th = fc.th;
            a.te = fc.te;
            a.k = kt;
            a.w = wt;
            a.lam = p->lambda + t;
            a.nrbf = p->nrbf;
            a.dterm = p->data_term;
            a.proj_c = p->proj_c;
            a.rc = rc;
            e = (fc.pair && fc.nsplit > 2) ? tnrd::launch_pair_cluster_fwd(ks, nk, fc.kth, fc.nsplit, a, N, stream)
              : fc.pair ? tnrd::launch_pair_fwd(ks, nk, fc.kth, fc.nsplit, a, N, stream)
                        : tnrd::launch_fused_fwd(ks, nk, fc.kth, a, N, stream);
        } else if (is_tc(algo)) {
            tnrd::StageArgs a{};
            const int tw = 32 - 2 * (ks / 2), tth = tnrd::tc_tile_h(ks, tc_nb);
            a.u_in = in;
            a.u_out = out;
            a.f = f;
            a.img_stride = (long long)plane;
            a.H = H;
            a.W = W;
            a.pitch = pitch;
            a.tiles_x = (W + tw - 1) / tw;
            a.tiles_y = (H + tth - 1) / tth;
            a.k = kt;
            a.w = wt;
            a.lam = p->lambda + t;
            a.nrbf = p->nrbf;
            a.dterm = p->data_term;
            a.proj_c = p->proj_c;
            a.rc = rc;
            e = tnrd::launch_tc_fwd(ks, nk, tc_nb, tc_prec(algo), a, N, stream);
        } else {
            tnrd::UnfArgs a{};
            a.u_in = in;
            a.u_out = out;
            a.f = f;
            a.v = (float*)(ws + L.v);
            a.g = (float*)(ws + L.g);
            a.img_stride = (long long)plane;
            a.H = H;
            a.W = W;
            a.pitch = pitch;
            a.nfilt = nk;
            a.k = kt;
            a.w = wt;
            a.lam = p->lambda + t;
            a.nrbf = p->nrbf;
            a.dterm = p->data_term;
            a.proj_c = p->proj_c;
            a.rc = rc;
            e = tnrd::launch_unfused_fwd(ks, a, N, stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "stage launch");
    }
    return TNRD_OK;
}

tnrd_status tnrd_backward(const tnrd_params* p, int N, int H, int W, int pitch,
                          const float* f, const float* u_stages, const float* grad_uT,
                          float* grad_u0, float* grad_filters, float* grad_rbf_w,
                          float* grad_lambda, tnrd_algo algo,
                          void* workspace, size_t workspace_bytes, cudaStream_t stream)
{
    tnrd_status st = check_params(p);
    if (st != TNRD_OK) return st;
    st = check_images(N, H, W, pitch, p->ksize);
    if (st != TNRD_OK) return st;
    if (algo != TNRD_ALGO_FUSED && algo != TNRD_ALGO_TC_TF32 && algo != TNRD_ALGO_TC_TF32X3)
        return fail(TNRD_ERR_UNSUPPORTED, "tnrd_backward supports TNRD_ALGO_FUSED, _TC_TF32 and _TC_TF32X3");
    if (!grad_filters || !grad_rbf_w || !grad_lambda)
        return fail(TNRD_ERR_INVALID_ARG, "null gradient output");
    const int T = p->T, ks = p->ksize, nk = p->nfilt, nrbf = p->nrbf;
    if (N == 0) {
        // no images: every gradient is zero
        cudaError_t e = cudaMemsetAsync(grad_filters, 0, sizeof(float) * (size_t)T * nk * ks * ks, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(grad_rbf_w, 0, sizeof(float) * (size_t)T * nk * nrbf, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(grad_lambda, 0, sizeof(float) * (size_t)T, stream);
        return e == cudaSuccess ? TNRD_OK : cuda_fail(e, "zeroing gradients");
    }
    if (!f || !u_stages || !grad_uT) return fail(TNRD_ERR_INVALID_ARG, "null image pointer");
    if (!aligned16(f) || !aligned16(u_stages) || !aligned16(grad_uT) ||
        (grad_u0 && !aligned16(grad_u0)))
        return fail(TNRD_ERR_INVALID_ARG, "image pointers must be 16-byte aligned");
    const BwdLayout L = bwd_layout(p, N, H, W, pitch);
    if (!workspace || workspace_bytes < L.total)
        return fail(TNRD_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", L.total,
                    workspace ? workspace_bytes : (size_t)0);
    char* ws = (char*)workspace;
    const size_t batch = (size_t)N * H * pitch;
    float* ebuf[2] = {(float*)(ws + L.e0), (float*)(ws + L.e1)};

    tnrd::BwdArgs a{};
    a.f = f;
    a.d = (float*)(ws + L.d);
    a.d_id = (p->data_term != TNRD_DATA_IDIV) ? (float*)(ws + L.did) : a.d;
    a.cpl = (float*)(ws + L.c);
    a.vpl = (float*)(ws + L.v);
    a.part_w = (float*)(ws + L.pw);
    a.part_k = (float*)(ws + L.pk);
    a.part_l = (float*)(ws + L.pl);
    a.img_stride = (long long)H * pitch;
    a.H = H;
    a.W = W;
    a.pitch = pitch;
    a.zb_tiles_x = L.zb_tiles_x;
    a.zb_tiles_y = L.zb_tiles_y;
    a.tiles_x = L.tiles_x;
    a.tiles_y = L.tiles_y;
    a.dk_tiles_x = L.dk_tiles_x;
    a.dk_tiles_y = L.dk_tiles_y;
    a.prep_blocks = L.prep_blocks;
    a.nfilt = nk;
    a.nrbf = nrbf;
    a.dterm = p->data_term;
    a.proj_c = p->proj_c;
    a.rc = make_rbf(p);
    // the adjoint on the tensor cores (TF32 or split TF32), the rest as FUSED
    const int adj_prec = algo == TNRD_ALGO_FUSED ? -1 : tc_prec(algo);
    int* err = nullptr;
    if (adj_prec >= 0 && !(err = tnrd::device_status_word()))
        return fail(TNRD_ERR_CUDA, "device status word unavailable");

    for (int t = T - 1; t >= 0; --t) {
        a.u_prev = u_stages + (size_t)t * batch;
        a.u_cur = u_stages + (size_t)(t + 1) * batch;
        a.e_cur = (t == T - 1) ? grad_uT : ebuf[(t + 1) & 1];
        a.e_prev = (t == 0 && grad_u0) ? grad_u0 : ebuf[t & 1];
        a.k = p->filters + (size_t)t * nk * ks * ks;
        a.w = p->rbf_w + (size_t)t * nk * nrbf;
        a.lam = p->lambda + t;
        cudaError_t e = tnrd::launch_bwd_stage(ks, nk, a, N, stream, adj_prec, err);
        if (e != cudaSuccess) return cuda_fail(e, "backward stage launch");
        tnrd::RedArgs r{};
        r.s[0] = {a.part_k, N * (adj_prec == tnrd::TC_TF32 ? tnrd::tc_dk_tiles(H, W)
                                                          : L.dk_tiles_x * L.dk_tiles_y),
                  nk * ks * ks,
                  grad_filters + (size_t)t * nk * ks * ks};
        r.s[1] = {a.part_w, N * L.zb_tiles_x * L.zb_tiles_y, nk * nrbf,
                  grad_rbf_w + (size_t)t * nk * nrbf};
        r.s[2] = {a.part_l, N * L.prep_blocks, 1, grad_lambda + t};
        e = tnrd::launch_bwd_reduce(r, stream);
        if (e != cudaSuccess) return cuda_fail(e, "gradient reduce launch");
    }
    return TNRD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Quality indexes.
// ---------------------------------------------------------------------------
extern "C" {

size_t tnrd_quality_workspace_size(int N, int H, int W)
{
    if (N < 1 || H < 1 || W < 1) return 0;
    return sizeof(double) * (size_t)N * tnrd::quality_tiles(H, W) * tnrd::QSUMS;
}

tnrd_status tnrd_quality(const float* ref, const float* img, const float* noisy, int N, int H,
                         int W, int pitch, float peak, double* out, void* workspace,
                         size_t workspace_bytes, cudaStream_t stream)
{
    if (N < 1 || H < 1 || W < 1 || pitch < W)
        return fail(TNRD_ERR_INVALID_ARG, "quality: N, H, W >= 1 and pitch >= W required");
    if ((long long)H * (long long)pitch >= (1LL << 31) || N > 65535)
        return fail(TNRD_ERR_INVALID_ARG, "quality: images too large");
    if (!img || !out) return fail(TNRD_ERR_INVALID_ARG, "quality: null img or out");
    if (!(peak > 0.0f) || !std::isfinite(peak))
        return fail(TNRD_ERR_INVALID_ARG, "quality: peak must be a positive number");
    const size_t need = tnrd_quality_workspace_size(N, H, W);
    if (!workspace || workspace_bytes < need)
        return fail(TNRD_ERR_WORKSPACE, "quality: workspace of %zu bytes needed", need);
    tnrd::QualityArgs a{};
    a.ref = ref;
    a.img = img;
    a.noisy = noisy;
    a.img_stride = (long long)H * pitch;
    a.H = H;
    a.W = W;
    a.pitch = pitch;
    a.tiles_x = (W + 31) / 32;
    a.tiles_y = (H + 31) / 32;
    a.peak = peak;
    a.part = (double*)workspace;
    a.out = out;
    double g[11], sum = 0.0;
    for (int b = 0; b < 11; ++b) {
        const double d = b - 5;
        g[b] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
        sum += g[b];
    }
    for (int b = 0; b < 11; ++b) a.g1[b] = (float)(g[b] / sum);
    for (int r = 0; r < 11; ++r)
        for (int b = 0; b < 11; ++b) a.g2[r * 11 + b] = (float)(g[r] * g[b] / (sum * sum));
    const cudaError_t e = tnrd::launch_quality(a, N, stream);
    return e == cudaSuccess ? TNRD_OK : cuda_fail(e, "quality launch");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched forward: plans.
// ---------------------------------------------------------------------------
struct tnrd_plan {
    int device = 0;
    tnrd_algo algo = TNRD_ALGO_FUSED;   // FUSED: fused stage kernel; TC_*: tensor-core stage
    int tc_nb = 2;
    int stages = 0;   // FUSED: 0 one persistent launch, 1 one launch per stage, 2 one launch
                      // per stage on column-pair tiles (autotuned)
    int ks = 0, nk = 0, nrbf = 0, T = 0;
    int th = 0;
    int nimg = 0, nsets = 0, ntiles = 0, ntiles_max = 0;
    int grid = 0;
    std::vector<tnrd_image> imgs;
    std::vector<tnrd_params> sets;
    char* block = nullptr;          // the plan's one device allocation
    size_t off_imgs = 0, off_sets = 0, off_tiles = 0, off_counters = 0, off_limit = 0, off_tmp = 0;
    size_t off_maps = 0;            // per image: tensor maps of f, u, tmp (per-stage fused kernel)
    std::vector<size_t> tmp_off;    // per image, offset of its inter-stage image
    tnrd::BatchArgs args{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// Tiles of one image in a plan: th rows x (32 - 2R) columns, or x (64 - 2R)
// columns for the column-pair schedule.
int batch_tiles(const tnrd_image& im, int ks, int th, int* tx, int* ty, bool pair = false)
{
    const int tw = (pair ? 64 : 32) - 2 * (ks / 2);
    *tx = (im.W + tw - 1) / tw;
    *ty = (im.H + th - 1) / th;
    return *tx * *ty;
}

// Uploads the image/tile tables of tile height th and points plan->args at them.
tnrd_status plan_build(tnrd_plan* P, int th, cudaStream_t s)
{
    std::vector<tnrd::BatchImg> bi(P->nimg);
    std::vector<int2> tiles;
    int base = 0;
    for (int i = 0; i < P->nimg; ++i) {
        const tnrd_image& im = P->imgs[i];
        int tx, ty;
        const int n = batch_tiles(im, P->ks, th, &tx, &ty, P->stages == 2);
        bi[i].f = im.f;
        bi[i].u = im.u;
        bi[i].tmp = (float*)(P->block + P->tmp_off[i]);
        bi[i].H = im.H;
        bi[i].W = im.W;
        bi[i].pitch = im.pitch;
        bi[i].tiles_x = tx;
        bi[i].tiles_y = ty;
        bi[i].tile_base = base;
        bi[i].set = im.param_set;
        for (int k = 0; k < n; ++k) tiles.push_back(make_int2(i, k));
        base += n;
    }
    P->th = th;
    P->ntiles = base;
    // tensor maps of every image's f, u and tmp for the per-stage fused kernel's
    // tile copies (boxes of this tile height); none if any cannot be encoded
    std::vector<CUtensorMap> maps;
    int bw = 0, bh = 0;
    const bool box = P->stages == 2 ? tnrd::pair_fwd_box(P->ks, P->nk, th, &bw, &bh)
                                    : tnrd::fused_fwd_box(P->ks, P->nk, th, &bw, &bh);
    if (P->algo == TNRD_ALGO_FUSED && tnrd::tma_staging_enabled() && box) {
        maps.resize(3 * (size_t)P->nimg);
        for (int i = 0; i < P->nimg && !maps.empty(); ++i) {
            const float* src[3] = {bi[i].f, bi[i].u, bi[i].tmp};
            for (int k = 0; k < 3; ++k) {
                if (!tnrd::encode_tile_map(&maps[3 * i + k], src[k], bi[i].W, bi[i].H, 1, bi[i].pitch,
                                           (long long)bi[i].H * bi[i].pitch, bw, bh)) {
                    maps.clear();
                    break;
                }
            }
        }
    }
    cudaError_t e = cudaMemcpyAsync(P->block + P->off_imgs, bi.data(), sizeof(tnrd::BatchImg) * bi.size(),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !maps.empty())
        e = cudaMemcpyAsync(P->block + P->off_maps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P->block + P->off_tiles, tiles.data(), sizeof(int2) * tiles.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "plan upload");
    tnrd::BatchArgs& A = P->args;
    A.imgs = (const tnrd::BatchImg*)(P->block + P->off_imgs);
    A.sets = (const tnrd::BatchSet*)(P->block + P->off_sets);
    A.tile_img = (const int2*)(P->block + P->off_tiles);
    A.work_counter = (int*)(P->block + P->off_counters);
    A.status = A.work_counter + 1;
    A.tile_done = A.work_counter + 2;
    A.wait_limit = (const long long*)(P->block + P->off_limit);
    A.ntiles = P->ntiles;
    A.maps = maps.empty() ? nullptr : (const CUtensorMap*)(P->block + P->off_maps);
    A.err = A.status;   // a tile copy that never landed is a plan failure (tnrd_plan_status)
    A.T = P->T;
    A.nfilt = P->nk;
    A.ksize = P->ks;
    A.nrbf = P->nrbf;
    if (P->algo == TNRD_ALGO_FUSED) {
        const int occ = tnrd::batch_fwd_occupancy(P->ks, P->nk, th, P->nrbf);
        int nsm = 1;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P->device);
        P->grid = std::max(1, nsm * std::max(occ, 1));
    } else {
        P->grid = P->ntiles;   // one CTA per tile and stage
    }
    return TNRD_OK;
}

cudaError_t plan_enqueue(const tnrd_plan* P, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(P->block + P->off_counters, 0, sizeof(int) * (2 + (size_t)P->ntiles), s);
    if (e != cudaSuccess) return e;
    if (P->algo == TNRD_ALGO_FUSED)
        return P->stages == 2 ? tnrd::launch_batch_pairs(P->ks, P->nk, P->th, P->args, s)
             : P->stages ? tnrd::launch_batch_stages(P->ks, P->nk, P->th, P->args, s)
                         : tnrd::launch_batch_fwd(P->ks, P->nk, P->th, P->args, P->grid, s);
    for (int t = 0; t < P->T && e == cudaSuccess; ++t)
        e = tnrd::launch_tc_batch(P->ks, P->nk, P->tc_nb, tc_prec(P->algo), P->args, t, P->ntiles, s);
    return e;
}

}  // namespace

extern "C" {

tnrd_status tnrd_plan_create(tnrd_plan** out, const tnrd_image* images, int nimg,
                             const tnrd_params* sets, int nsets, tnrd_algo algo, int autotune,
                             cudaStream_t stream)
{
    if (!out) return fail(TNRD_ERR_INVALID_ARG, "plan pointer is null");
    *out = nullptr;
    if (!images || nimg < 1 || !sets || nsets < 1)
        return fail(TNRD_ERR_INVALID_ARG, "need at least one image and one parameter set");
    if (algo != TNRD_ALGO_FUSED && !is_tc(algo))
        return fail(TNRD_ERR_UNSUPPORTED, "batched forward supports the fused and tensor-core stages");
    for (int s = 0; s < nsets; ++s) {
        tnrd_status st = check_params(&sets[s]);
        if (st != TNRD_OK) return st;
        if (sets[s].T != sets[0].T || sets[s].ksize != sets[0].ksize || sets[s].nfilt != sets[0].nfilt ||
            sets[s].nrbf != sets[0].nrbf)
            return fail(TNRD_ERR_INVALID_ARG, "parameter sets differ in T, ksize, nfilt or nrbf");
    }
    const int ks = sets[0].ksize;
    for (int i = 0; i < nimg; ++i) {
        const tnrd_image& im = images[i];
        tnrd_status st = check_images(1, im.H, im.W, im.pitch, ks);
        if (st != TNRD_OK) return st;
        if (!im.f || !im.u || !aligned16(im.f) || !aligned16(im.u))
            return fail(TNRD_ERR_INVALID_ARG, "image %d: null or misaligned pointer", i);
        if (im.param_set < 0 || im.param_set >= nsets)
            return fail(TNRD_ERR_INVALID_ARG, "image %d: param_set %d out of range", i, im.param_set);
        const size_t n = (size_t)im.H * im.pitch;
        if ((const float*)im.u < im.f + n && im.f < (const float*)im.u + n)
            return fail(TNRD_ERR_INVALID_ARG, "image %d: u overlaps f", i);
    }
    tnrd_plan* P = new tnrd_plan();
    cudaGetDevice(&P->device);
    P->ks = ks;
    P->nk = sets[0].nfilt;
    P->nrbf = sets[0].nrbf;
    P->T = sets[0].T;
    P->nimg = nimg;
    P->nsets = nsets;
    P->imgs.assign(images, images + nimg);
    P->sets.assign(sets, sets + nsets);
    P->algo = algo;
    P->tc_nb = pick_tc_nb(algo);
    // tensor-core plans: the stage kernel's one tile height; fused plans: the list
    const int tc_th[2] = {tnrd::tc_tile_h(ks, P->tc_nb), 0};
    const int* ths = (algo == TNRD_ALGO_FUSED) ? tnrd::fused_th_list(ks) : tc_th;
    int tmax = 0;
    for (int pair = 0; pair < (algo == TNRD_ALGO_FUSED ? 2 : 1); ++pair) {
        for (const int* p = pair ? tnrd::pair_th_list(ks) : ths; *p; ++p) {
            int n = 0;
            for (int i = 0; i < nimg; ++i) {
                int tx, ty;
                n += batch_tiles(images[i], ks, *p, &tx, &ty, pair != 0);
            }
            tmax = std::max(tmax, n);
        }
    }
    P->ntiles_max = tmax;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off = align_up(off + bytes, 256); return o; };
    P->off_imgs = take(sizeof(tnrd::BatchImg) * nimg);
    P->off_sets = take(sizeof(tnrd::BatchSet) * nsets);
    P->off_tiles = take(sizeof(int2) * tmax);
    P->off_counters = take(sizeof(int) * (2 + (size_t)tmax));
    P->off_limit = take(sizeof(long long));
    P->off_maps = take(sizeof(CUtensorMap) * 3 * (size_t)nimg);
    P->tmp_off.resize(nimg);
    for (int i = 0; i < nimg; ++i) P->tmp_off[i] = take(sizeof(float) * (size_t)images[i].H * images[i].pitch);
    cudaError_t e = cudaMalloc((void**)&P->block, off);
    if (e != cudaSuccess) {
        delete P;
        return cuda_fail(e, "plan allocation");
    }
    std::vector<tnrd::BatchSet> bs(nsets);
    for (int s = 0; s < nsets; ++s) {
        bs[s].k = sets[s].filters;
        bs[s].w = sets[s].rbf_w;
        bs[s].lam = sets[s].lambda;
        bs[s].dterm = sets[s].data_term;
        bs[s].proj_c = sets[s].proj_c;
        bs[s].rc = make_rbf(&sets[s]);
    }
    const long long limit = 2000000000LL;
    e = cudaMemcpyAsync(P->block + P->off_sets, bs.data(), sizeof(tnrd::BatchSet) * nsets,
                        cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P->block + P->off_limit, &limit, sizeof limit, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        tnrd_plan_destroy(P);
        return cuda_fail(e, "plan upload");
    }

    // tile height (and, for the fused stage, the schedule: one persistent launch
    // or one launch per stage): timed on the data (autotune) or, without
    // autotune, the persistent launch with the tile height of least total work
    // including halos
    int best = ths[0], best_stages = 0;
    if (autotune) {
        float best_ms = 1e30f;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        // candidates: every tile height of the one-column schedules (persistent,
        // per stage) and of the column-pair schedule (per stage)
        std::vector<std::pair<int, int>> cand;   // (mode, tile height)
        for (const int* p = ths; *p; ++p) {
            cand.push_back({0, *p});
            if (algo == TNRD_ALGO_FUSED) cand.push_back({1, *p});
        }
        if (algo == TNRD_ALGO_FUSED)
            for (const int* p = tnrd::pair_th_list(ks); *p; ++p) cand.push_back({2, *p});
        for (const auto& cd : cand) {
            const int mode = cd.first;
            const int* p = &cd.second;
            P->stages = mode;
            tnrd_status st = plan_build(P, *p, stream);
            if (st != TNRD_OK) { tnrd_plan_destroy(P); return st; }
            {
                float ms = 0.0f;
                e = plan_enqueue(P, stream);   // warm-up
                for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
                    cudaEventRecord(e0, stream);
                    e = plan_enqueue(P, stream);
                    cudaEventRecord(e1, stream);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    float m = 0.0f;
                    cudaEventElapsedTime(&m, e0, e1);
                    ms += m;
                }
                if (e != cudaSuccess) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    tnrd_plan_destroy(P);
                    return cuda_fail(e, "autotune run");
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    best = *p;
                    best_stages = mode;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    } else {
        const int R = ks / 2;
        double best_cost = 1e300;
        for (const int* p = ths; *p; ++p) {
            double cost = 0.0;
            for (int i = 0; i < nimg; ++i) {
                int tx, ty;
                cost += (double)batch_tiles(images[i], ks, *p, &tx, &ty) * (*p + 4 * R);
            }
            if (cost < best_cost * 0.999) {
                best_cost = cost;
                best = *p;
            }
        }
    }
    P->stages = best_stages;
    if (const char* env = std::getenv("TNRD_BATCH_SCHEDULE")) {   // tuning override
        int want = -1;
        if (std::strcmp(env, "persistent") == 0) want = 0;
        if (algo == TNRD_ALGO_FUSED && std::strcmp(env, "stages") == 0) want = 1;
        if (algo == TNRD_ALGO_FUSED && std::strcmp(env, "pairs") == 0) want = 2;
        if (want >= 0 && want != P->stages) {
            if ((want == 2) != (P->stages == 2)) {
                // other tile geometry: its tile height of least total work with halos
                const int R = ks / 2;
                double best_cost = 1e300;
                for (const int* p = want == 2 ? tnrd::pair_th_list(ks) : ths; *p; ++p) {
                    double cost = 0.0;
                    for (int i = 0; i < nimg; ++i) {
                        int tx, ty;
                        cost += (double)batch_tiles(images[i], ks, *p, &tx, &ty, want == 2) * (*p + 4 * R);
                    }
                    if (cost < best_cost * 0.999) {
                        best_cost = cost;
                        best = *p;
                    }
                }
            }
            P->stages = want;
        }
    }
    tnrd_status st = plan_build(P, best, stream);
    if (st != TNRD_OK) { tnrd_plan_destroy(P); return st; }

    // record the launch in a graph
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = plan_enqueue(P, cs);
            e = cudaStreamEndCapture(cs, &P->graph);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&P->exec, P->graph, 0);
        cudaStreamDestroy(cs);
    }
    if (e != cudaSuccess) {
        tnrd_plan_destroy(P);
        return cuda_fail(e, "plan graph capture");
    }
    *out = P;
    return TNRD_OK;
}

tnrd_status tnrd_batch_forward(const tnrd_plan* P, cudaStream_t stream)
{
    if (!P) return fail(TNRD_ERR_INVALID_ARG, "plan is null");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "stream query");
    if (cap == cudaStreamCaptureStatusActive) e = plan_enqueue(P, stream);
    else e = cudaGraphLaunch(P->exec, stream);
    return e == cudaSuccess ? TNRD_OK : cuda_fail(e, "batch launch");
}

tnrd_status tnrd_plan_status(const tnrd_plan* P)
{
    if (!P) return fail(TNRD_ERR_INVALID_ARG, "plan is null");
    int st = 0;
    cudaError_t e = cudaMemcpy(&st, P->block + P->off_counters + sizeof(int), sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (st == TNRD_ERR_TIMEOUT) return fail(TNRD_ERR_TIMEOUT, "a tile gave up waiting for its neighbours");
    return st == 0 ? TNRD_OK : fail((tnrd_status)st, "device status %d", st);
}

tnrd_status tnrd_plan_set_wait_limit(tnrd_plan* P, long long cycles)
{
    if (!P || cycles < 0) return fail(TNRD_ERR_INVALID_ARG, "bad plan or negative limit");
    cudaError_t e = cudaMemcpy(P->block + P->off_limit, &cycles, sizeof cycles, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? TNRD_OK : cuda_fail(e, "wait limit");
}

int tnrd_plan_tile_height(const tnrd_plan* P) { return P ? P->th : 0; }

int tnrd_plan_tile_width(const tnrd_plan* P)
{
    if (!P) return 0;
    return ((P->algo == TNRD_ALGO_FUSED && P->stages == 2) ? 64 : 32) - 2 * (P->ks / 2);
}

int tnrd_plan_launches(const tnrd_plan* P)
{
    if (!P) return 0;
    return (P->algo == TNRD_ALGO_FUSED && !P->stages) ? 1 : P->T;
}

void tnrd_plan_destroy(tnrd_plan* P)
{
    if (!P) return;
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    if (P->block) {
        cudaDeviceSynchronize();
        cudaFree(P->block);
    }
    delete P;
}

}  // extern "C"
