// Unfused three-kernel FP32 stage, the baseline the fused kernel is measured
// against.  Same arithmetic per output, but the N_k response planes
// v_i = phi_i(K_i u) make a round trip through HBM:
//   K1 unf_bank_phi : v_i = phi_i(K_i u_{t-1})           -> N_k planes
//   K2 unf_adjoint  : g = sum_i K_i^T v_i (gather form, border folded) -> 1 plane
//   K3 unf_prox     : u_t = prox(u_{t-1} - g)
#pragma once
#include "args.cuh"

namespace tnrd {

// grid (ceil(H*W/256), nfilt, N)
template <int KS>
__global__ void __launch_bounds__(256) unf_bank_phi(const UnfArgs a)
{
    constexpr int R = KS / 2;
    __shared__ float sk[KS * KS];
    __shared__ float swp[MAX_NRBF + 2 * RBF_WPAD];
    const int fi = blockIdx.y, n = blockIdx.z;
    for (int e = threadIdx.x; e < KS * KS; e += blockDim.x) sk[e] = a.k[fi * KS * KS + e];
    for (int e = threadIdx.x; e < MAX_NRBF + 2 * RBF_WPAD; e += blockDim.x) {
        const int j = e - RBF_WPAD;
        swp[e] = (j >= 0 && j < a.nrbf) ? a.w[fi * a.nrbf + j] : 0.0f;
    }
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.H * a.W) return;
    const int y = p / a.W, x = p - y * a.W;
    const float* u = a.u_in + (size_t)n * a.img_stride;
    float z = 0.0f;
#pragma unroll
    for (int ia = 0; ia < KS; ++ia) {
        const int yy = sym_idx(y + R - ia, a.H);
#pragma unroll
        for (int ib = 0; ib < KS; ++ib) {
            const int xx = sym_idx(x + R - ib, a.W);
            z = fmaf(sk[ia * KS + ib], u[(size_t)yy * a.pitch + xx], z);
        }
    }
    a.v[((size_t)n * a.nfilt + fi) * ((size_t)a.H * a.pitch) + (size_t)y * a.pitch + x] =
        rbf_phi(z, swp, a.rc);
}

// grid (ceil(H*W/256), N); dynamic smem nfilt*KS*KS floats
template <int KS>
__global__ void __launch_bounds__(256) unf_adjoint(const UnfArgs a)
{
    constexpr int R = KS / 2;
    extern __shared__ float sk_all[];
    const int n = blockIdx.y;
    for (int e = threadIdx.x; e < a.nfilt * KS * KS; e += blockDim.x) sk_all[e] = a.k[e];
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.H * a.W) return;
    const int y = p / a.W, x = p - y * a.W;
    const int H = a.H, W = a.W;
    // mirror sources of (y, x) in the zero-extended adjoint: (K^T v)(q) =
    // sum_{q': sym(q') = q} sum_{a,b} k[a][b] v(q' - R + (a, b)).
    int sy[2], sx[2], nsy = 1, nsx = 1;
    sy[0] = y;
    sx[0] = x;
    if (y < R) sy[nsy++] = -1 - y;
    else if (y >= H - R) sy[nsy++] = 2 * H - 1 - y;
    if (x < R) sx[nsx++] = -1 - x;
    else if (x >= W - R) sx[nsx++] = 2 * W - 1 - x;
    const size_t plane = (size_t)H * a.pitch;
    const float* vbase = a.v + (size_t)n * a.nfilt * plane;
    float g = 0.0f;
    for (int fi = 0; fi < a.nfilt; ++fi) {
        const float* v = vbase + fi * plane;
        const float* k = sk_all + fi * KS * KS;
        for (int ps = 0; ps < nsy; ++ps) {
            for (int qs = 0; qs < nsx; ++qs) {
#pragma unroll
                for (int ia = 0; ia < KS; ++ia) {
                    const int yy = sy[ps] - R + ia;
                    if (yy < 0 || yy >= H) continue;
#pragma unroll
                    for (int ib = 0; ib < KS; ++ib) {
                        const int xx = sx[qs] - R + ib;
                        if (xx < 0 || xx >= W) continue;
                        g = fmaf(k[ia * KS + ib], v[(size_t)yy * a.pitch + xx], g);
                    }
                }
            }
        }
    }
    a.g[(size_t)n * a.img_stride + (size_t)y * a.pitch + x] = g;
}

// grid (ceil(H*W/256), N)
__global__ void __launch_bounds__(256) unf_prox(const UnfArgs a)
{
    const int n = blockIdx.y;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.H * a.W) return;
    const int y = p / a.W, x = p - y * a.W;
    const size_t o = (size_t)n * a.img_stride + (size_t)y * a.pitch + x;
    a.u_out[o] = stage_out(a.u_in[o], a.g[o], a.f[o], __ldg(a.lam), a.dterm, a.proj_c);
}

}  // namespace tnrd
