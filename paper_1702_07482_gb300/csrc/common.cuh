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
constexpr int MAX_NRBF = 128;
// w is staged in shared memory with 2*RBF_WIN zeros on each side, so that the
// 13-term window never needs a bounds test: wp[j + 2*RBF_WIN] = w_j.
constexpr int RBF_WPAD = 2 * RBF_WIN;

struct RbfConst {
    float mu0;          // first centre
    float delta;        // centre spacing
    float inv_delta;
    float zlo, zhi;     // z is clamped to [mu_0 - 6.5 delta, mu_last + 6.5 delta]
    float cq;           // delta / gamma^2
    float half_inv_g2;  // 1 / (2 gamma^2)
    float inv_g2;       // 1 / gamma^2
    int jmax;           // nrbf - 1 + RBF_WIN: largest window centre index
    float E[RBF_WIN + 1];  // exp(-m^2 delta^2 / (2 gamma^2)), m = 0..RBF_WIN
};

// Half-sample symmetric index into [0, n), any integer i (period 2n).
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

}  // namespace tnrd
