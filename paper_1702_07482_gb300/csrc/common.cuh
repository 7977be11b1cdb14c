// Shared device helpers of the TRDMD stage kernels: the symmetric boundary
// index, the influence function phi (a sum of Gaussian RBFs) and the prox of
// the I-divergence data term.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tnrd {

// phi_i(z) = sum_j w_ij exp(-(z - mu_j)^2 / (2 gamma^2)), mu_j = mu0 + j delta.
// Only the RBF_TERMS centres nearest to z are summed.  With delta >= gamma the
// nearest centre is within delta/2 of z, every dropped centre is at least
// (RBF_WIN + 1/2) delta = 6.5 gamma away, and the dropped terms total less than
// 2 * exp(-21.1) * max|w| < 1.4e-9 * max|w| -- far below FP32 rounding of phi.
constexpr int RBF_WIN = 6;
constexpr int RBF_TERMS = 2 * RBF_WIN + 1;
constexpr int MAX_NRBF = 64;
// The tensor-core stages sum the 2*TC_WIN+1 = 11 nearest centres: every dropped
// centre is at least (TC_WIN + 1/2) delta = 5.5 gamma away, so the dropped
// terms total less than 2 * exp(-15.1) * max|w| < 5.4e-7 * max|w|, three
// orders of magnitude below the rounding of v to the adjoint GEMM's operand
// precision (TF32: 2^-11 relative, BF16: 2^-8).
constexpr int TC_WIN = 5;
// w is staged in shared memory with 2*RBF_WIN zeros on each side, so that the
// 13-term window never needs a bounds test: wp[j + 2*RBF_WIN] = w_j.
constexpr int RBF_WPAD = 2 * RBF_WIN;

struct RbfConst {
    float mu0;          // first centre
    float delta;        // centre spacing
    float inv_delta;
    float zlo, zhi;     // z is clamped to [mu_0 - 6.49 delta, mu_last + 6.49 delta]
    float t_off;        // -mu0 / delta
    float tmax;         // nrbf - 1 + RBF_WIN: largest window centre index
    float cq;           // delta / gamma^2
    float half_inv_g2;  // 1 / (2 gamma^2)
    float inv_g2;       // 1 / gamma^2
    float c_q2;         // log2(e) delta / gamma^2
    float c_p2a;        // log2(e) / (2 gamma^2)
    float c_p2b;        // log2(e) RBF_WIN delta / gamma^2
    float c_p2b_tc;     // log2(e) TC_WIN delta / gamma^2 (window of the tensor-core stages)
    int jmax;           // nrbf - 1 + RBF_WIN
    float E[RBF_WIN + 1];  // exp(-m^2 delta^2 / (2 gamma^2)), m = 0..RBF_WIN
};

// Window coefficient table of one influence function, built in shared memory
// per filter, coefficient-major: entry (n, r) at tab[n * rows + r] with
// r = j0 + RBF_WIN (j0 = -RBF_WIN .. nrbf-1+RBF_WIN) and
//   C(n, r) = w_{j0 - RBF_WIN + n} * E[|n - RBF_WIN|],  n = 0 .. 2 RBF_WIN
// (w_j = 0 outside [0, nrbf)).  Each lane gathers the 13 entries of its own
// row; with this layout two lanes collide on a bank only when their rows
// differ by a multiple of 32 centres.
constexpr int RBF_NCOEF = RBF_TERMS;
// Table pitch (rows) fixed at compile time so that the 13 gathers of a lane use
// immediate offsets; tables hold up to MAX_NRBF centres.
constexpr int RBF_TP = MAX_NRBF + 2 * RBF_WIN;

__device__ __host__ __forceinline__ int rbf_table_rows(int nrbf) { return nrbf + 2 * RBF_WIN; }

// 2^x with the SFU's ex2.approx (max relative error about 2^-22).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Half-sample symmetric index into [0, n), any integer i (period 2n).
// Row pitch (floats) of a staged tile of uw columns: room for a start column
// rounded down to 16 bytes (up to 3 floats earlier), a multiple of 4 floats.
__host__ __device__ constexpr int staged_pitch(int uw) { return (uw + 3 + 3) & ~3; }

__device__ __forceinline__ int sym_idx(int i, int n)
{
    const int p = 2 * n;
    int m = i % p;
    m = (m < 0) ? m + p : m;
    return (m < n) ? m : (p - 1 - m);
}

// Window set-up shared by phi and phi': z = mu_{j0} + s with j0 the nearest
// centre (clamped), q = exp(s delta / gamma^2) and
// pre = exp(-s^2 / (2 gamma^2) - RBF_WIN s delta / gamma^2).  Then
//   exp(-(z - mu_{j0+m})^2 / (2 gamma^2)) = pre * q^(m + RBF_WIN) * E[|m|]
// exactly, which turns the window sum into one polynomial in q (Horner).
struct RbfWindow {
    float s, q, pre;
    int j0;
};

__device__ __forceinline__ RbfWindow rbf_window(float z, const RbfConst& rc)
{
    RbfWindow r;
    const float zc = fminf(fmaxf(z, rc.zlo), rc.zhi);
    int j0 = __float2int_rn((zc - rc.mu0) * rc.inv_delta);
    j0 = min(max(j0, -RBF_WIN), rc.jmax);
    r.j0 = j0;
    r.s = zc - fmaf((float)j0, rc.delta, rc.mu0);
    r.q = expf(r.s * rc.cq);
    r.pre = expf(-r.s * fmaf(r.s, rc.half_inv_g2, (float)RBF_WIN * rc.cq));
    return r;
}

// phi(z) with weights wp (padded as described above, in shared memory).
__device__ __forceinline__ float rbf_phi(float z, const float* wp, const RbfConst& rc)
{
    const RbfWindow win = rbf_window(z, rc);
    const float* wr = wp + (win.j0 + RBF_WIN);   // wr[n] = w_{j0 - RBF_WIN + n}
    float p = wr[2 * RBF_WIN] * rc.E[RBF_WIN];
#pragma unroll
    for (int n = 2 * RBF_WIN - 1; n >= 0; --n) {
        const int m = n - RBF_WIN;
        p = fmaf(p, win.q, wr[n] * rc.E[m < 0 ? -m : m]);
    }
    return win.pre * p;
}

// Window set-up from the table's point of view: j0 (clamped nearest centre),
// q = exp(s delta / gamma^2) and pre = exp(-s^2/(2 gamma^2) - RBF_WIN s delta / gamma^2)
// computed as powers of two with pre-scaled arguments; the nearest centre is
// found with the 1.5 * 2^23 rounding trick (exact for |t| < 2^22).
struct RbfWin2 {
    float s, q, pre;
    int row;   // table row j0 + RBF_WIN
};

__device__ __forceinline__ RbfWin2 rbf_win2(float z, const RbfConst& rc)
{
    RbfWin2 r;
    const float zc = fminf(fmaxf(z, rc.zlo), rc.zhi);
    // zc within 6.49 spacings of the grid: t rounds into [-RBF_WIN, nrbf-1+RBF_WIN]
    const float t = fmaf(zc, rc.inv_delta, rc.t_off);
    const float tm = t + 12582912.0f;
    const float jf = tm - 12582912.0f;
    r.row = __float_as_int(tm) - 0x4B400000 + RBF_WIN;
    r.s = zc - fmaf(jf, rc.delta, rc.mu0);
    r.q = ex2_approx(r.s * rc.c_q2);
    r.pre = ex2_approx(-r.s * fmaf(r.s, rc.c_p2a, rc.c_p2b));
    return r;
}

// Horner evaluation in q of the 13 window coefficients of table row `row`
// (coefficient-major table of pitch RBF_TP).
__device__ __forceinline__ float rbf_horner(const float* __restrict__ tab, int row, float q)
{
    const float* c = tab + row;
    float p = c[(2 * RBF_WIN) * RBF_TP];
#pragma unroll
    for (int n = 2 * RBF_WIN - 1; n >= 0; --n) p = fmaf(p, q, c[n * RBF_TP]);
    return p;
}

// Horner evaluation of P(q) = sum_n C_n q^n and of q P'(q) = sum_n n C_n q^n
// from one pass over the table row (the derivative recurrence of Horner).
__device__ __forceinline__ void rbf_horner_d(const float* __restrict__ tab, int row, float q,
                                             float& P, float& QdP)
{
    const float* c = tab + row;
    float p = c[(2 * RBF_WIN) * RBF_TP];
    float dp = 0.0f;
#pragma unroll
    for (int n = 2 * RBF_WIN - 1; n >= 0; --n) {
        dp = fmaf(dp, q, p);
        p = fmaf(p, q, c[n * RBF_TP]);
    }
    P = p;
    QdP = q * dp;
}

// phi(z) and phi'(z) from a coefficient table.  With z = mu_{j0} + s,
//   phi'(z) = -(1/gamma^2) sum_j w_j (z - mu_j) G_j(z)
//           = -(1/gamma^2) (s phi(z) - delta pre sum_n (n - RBF_WIN) C_n q^n).
__device__ __forceinline__ void rbf_phi_dphi_tab(float z, const float* __restrict__ tab,
                                                 const RbfConst& rc, float& phi, float& dphi,
                                                 RbfWin2& win)
{
    win = rbf_win2(z, rc);
    float P, QdP;
    rbf_horner_d(tab, win.row, win.q, P, QdP);
    phi = win.pre * P;
    const float m1 = win.pre * fmaf(-(float)RBF_WIN, P, QdP);   // pre sum (n - W) C_n q^n
    dphi = -rc.inv_g2 * fmaf(win.s, phi, -rc.delta * m1);
}

// phi(z) straight from the padded weights wp (wp[j + RBF_WPAD] = w_j): the
// same window and Horner evaluation as rbf_phi_tab, with each coefficient
// formed as w_j * E[|m|] on the fly instead of read from a table.
__device__ __forceinline__ float rbf_phi_w(float z, const float* __restrict__ wp, const RbfConst& rc)
{
    const RbfWin2 w = rbf_win2(z, rc);
    const float* wr = wp + w.row;   // wr[n] = wp[j0 + RBF_WIN + n] = w_{j0 - RBF_WIN + n}
    float p = wr[2 * RBF_WIN] * rc.E[RBF_WIN];
#pragma unroll
    for (int n = 2 * RBF_WIN - 1; n >= 0; --n) {
        const int m = n - RBF_WIN;
        p = fmaf(p, w.q, wr[n] * rc.E[m < 0 ? -m : m]);
    }
    return w.pre * p;
}

// phi(z) and phi'(z) straight from the padded weights wp, as rbf_phi_dphi_tab
// with the window coefficients w_j E[|m|] formed on the fly.
__device__ __forceinline__ void rbf_phi_dphi_w(float z, const float* __restrict__ wp,
                                               const RbfConst& rc, float& phi, float& dphi,
                                               RbfWin2& win)
{
    win = rbf_win2(z, rc);
    const float* wr = wp + win.row;
    float p = wr[2 * RBF_WIN] * rc.E[RBF_WIN];
    float dp = 0.0f;
#pragma unroll
    for (int n = 2 * RBF_WIN - 1; n >= 0; --n) {
        const int m = n - RBF_WIN;
        dp = fmaf(dp, win.q, p);
        p = fmaf(p, win.q, wr[n] * rc.E[m < 0 ? -m : m]);
    }
    phi = win.pre * p;
    const float m1 = win.pre * fmaf(-(float)RBF_WIN, p, win.q * dp);
    dphi = -rc.inv_g2 * fmaf(win.s, phi, -rc.delta * m1);
}

// RBF weights of the tensor-core stages, laid out so that the 16 lanes of a
// half-warp never collide on a shared-memory bank.  Filters go in rounds of 16
// (filter f = 16 r + c, column c); with wp filter f's padded weights (wp[j +
// RBF_WPAD] = w_j, zeros elsewhere), entry (r, row, c) holds the 8-byte pair
// (wp[row], wp[row + 1]) at pair index (r * TC_ROWS + row) * 16 + c.  Every
// entry of column c lies in bank pair c, so when the lanes of a half-warp
// evaluate 16 different filters of one round at once, their loads hit 16
// distinct bank pairs whatever their window rows: no conflicts.  The window's
// 11 weights start at wp index row = j0 + RBF_WPAD - TC_WIN and are the pairs
// of rows row, row + 2, .., row + 10.
constexpr int TC_ROWS = MAX_NRBF + 2 * RBF_WPAD;

// phi(z) over the TC_WIN window of the filter in column `col` of the round
// whose entries start at tab_r (tab + r * TC_ROWS * 16).  Horner in q as
// rbf_phi_w.
__device__ __forceinline__ float rbf_phi_col(float z, const float2* __restrict__ tab_r, int col,
                                             const RbfConst& rc)
{
    const float zc = fminf(fmaxf(z, rc.zlo), rc.zhi);
    const float t = fmaf(zc, rc.inv_delta, rc.t_off);
    const float tm = t + 12582912.0f;
    const float jf = tm - 12582912.0f;
    const int row = __float_as_int(tm) - 0x4B400000 + (RBF_WPAD - TC_WIN);   // wp index of w_{j0-TC_WIN}
    const float s = zc - fmaf(jf, rc.delta, rc.mu0);
    const float q = ex2_approx(s * rc.c_q2);
    const float pre = ex2_approx(-s * fmaf(s, rc.c_p2a, rc.c_p2b_tc));
    const float2* wr = tab_r + row * 16 + col;
    float c[2 * TC_WIN + 2];
#pragma unroll
    for (int k = 0; k <= TC_WIN; ++k) {
        const float2 v = wr[32 * k];
        c[2 * k] = v.x;
        c[2 * k + 1] = v.y;
    }
    float p = c[2 * TC_WIN] * rc.E[TC_WIN];
#pragma unroll
    for (int n = 2 * TC_WIN - 1; n >= 0; --n) {
        const int m = n - TC_WIN;
        p = fmaf(p, q, c[n] * rc.E[m < 0 ? -m : m]);
    }
    return pre * p;
}

// Within each aligned group of four: x[4q + t] <- x[4q + ((t + k) mod 4)]
// for a per-thread k in [0, 4) (two stages of selects).
__device__ __forceinline__ void rotl4x4(float (&x)[16], int k)
{
#pragma unroll
    for (int b = 2; b >= 1; b >>= 1) {
        const bool on = (k & b) != 0;
        float y[16];
#pragma unroll
        for (int s = 0; s < 16; ++s) y[s] = on ? x[(s & ~3) | ((s + b) & 3)] : x[s];
#pragma unroll
        for (int s = 0; s < 16; ++s) x[s] = y[s];
    }
}

// x[s] <- x[(s + k) mod 16] for a per-thread k in [0, 16): four stages of
// selects (no register indexing, no memory).
__device__ __forceinline__ void rotl16(float (&x)[16], int k)
{
#pragma unroll
    for (int b = 8; b >= 1; b >>= 1) {
        const bool on = (k & b) != 0;
        float y[16];
#pragma unroll
        for (int s = 0; s < 16; ++s) y[s] = on ? x[(s + b) & 15] : x[s];
#pragma unroll
        for (int s = 0; s < 16; ++s) x[s] = y[s];
    }
}

// phi(z) from a coefficient table.
__device__ __forceinline__ float rbf_phi_tab(float z, const float* __restrict__ tab,
                                             const RbfConst& rc)
{
    const RbfWin2 w = rbf_win2(z, rc);
    return w.pre * rbf_horner(tab, w.row, w.q);
}

// Builds the coefficient table of one filter from its padded weights wp
// (wp[j + RBF_WPAD] = w_j, zeros elsewhere); cooperative over the 32 lanes.
__device__ __forceinline__ void rbf_build_table(float* tab, const float* wp, int nrbf,
                                                const RbfConst& rc, int lane)
{
    const int rows = rbf_table_rows(nrbf);
    for (int e = lane; e < RBF_NCOEF * rows; e += 32) {
        const int n = e / rows, r = e - n * rows;
        const int m = n - RBF_WIN;
        tab[n * RBF_TP + r] = wp[r + n] * rc.E[m < 0 ? -m : m];
    }
}

// Prox of G(u) = lam (u^2 - 2 f^2 log u) at u~ (Eq. subproblemGIdiv).  For
// u~ < 0 the same root is written 4 lam f^2 / (S - u~), free of cancellation.
// sqrtf and '/' are the IEEE round-to-nearest operations (no fast-math).
__device__ __forceinline__ float prox_idiv(float ut, float f, float lam)
{
    const float a = fmaf(2.0f, lam, 1.0f);
    const float f2 = f * f;
    const float S = sqrtf(fmaf(ut, ut, 8.0f * a * lam * f2));
    return (ut >= 0.0f) ? (ut + S) / (2.0f * a) : (4.0f * lam * f2) / (S - ut);
}

// Stage output from u_{t-1} = up, the diffusion force g, f and lam, for the
// data terms of tnrd_data_term (mode):
//   0: prox of the I-divergence term at u~ = up - g (Eq. subproblemGIdiv);
//   1: TNRD Gaussian denoising, u~ - lam (up - f) (Sec. 2.2.1, G = 0);
//   2: max(u~ - psi, c), psi = (lam / up) (1 - f^2 / up^2) (Eq. diffusion_backP),
//      written lam (up - f)(up + f) / up^3 to avoid the cancellation in 1 - f^2/up^2.
__device__ __forceinline__ float stage_out(float up, float g, float f, float lam, int mode,
                                           float c)
{
    const float ut = up - g;
    if (mode == 0) return prox_idiv(ut, f, lam);
    if (mode == 1) return fmaf(-lam, up - f, ut);
    const float psi = lam * ((up - f) * (up + f)) / (up * up * up);
    return fmaxf(ut - psi, c);
}

}  // namespace tnrd
