// Kernel argument structs and compile-time tile configurations, shared by
// the kernel translation units and the host-side dispatcher.
#pragma once
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
    RbfConst rc;
};

template <int KS, int NK, int TH>
struct FusedCfg {
    static constexpr int R = KS / 2;
    static constexpr int TW = 32;
    static constexpr int NWARP = 4;
    static constexpr int NTHREADS = NWARP * 32;
    static constexpr int FPW = NK / NWARP;
    static_assert(NK % NWARP == 0, "filters must split evenly over the warps");
    static constexpr int UH = TH + 4 * R, UW = TW + 4 * R;
    static constexpr int UP = UW | 1;          // odd pitch spreads column chunks over banks
    static constexpr int ZH = TH + 2 * R, ZW = TW + 2 * R;
    static constexpr int HP = ZW | 1;
    static constexpr int XC = ZW - 32;         // columns beyond the 32 lanes (= 2R)
    static constexpr int NCH = 32 / XC;        // row chunks for them
    static constexpr int CHT = (ZH + NCH - 1) / NCH;
    static constexpr int KPAD = (KS * KS + 3) & ~3;
    static constexpr int WPADN = MAX_NRBF + 2 * RBF_WPAD;
    static constexpr int U_FL = UH * UP;
    static constexpr int V_FL = UH * UP;
    static constexpr int H_FL = ZH * HP;
    static constexpr int KW_FL = KPAD + WPADN;
    static constexpr int SMEM_FL = U_FL + NWARP * (V_FL + H_FL + KW_FL);
    static constexpr size_t SMEM_BYTES = sizeof(float) * (size_t)SMEM_FL;
};

// Tile origin along one axis: tiles of size T cover [0, n); the last tile is
// shifted back to end at n (when n >= T) so that every tile lies inside the
// image and only the first and the last tile touch a border.
__device__ __forceinline__ int tile_origin(int t, int T, int n)
{
    return (n >= T) ? min(t * T, n - T) : 0;
}

// Start of the range of rows (or columns) that tile t writes; tile t writes
// [tile_split(t), tile_split(t+1)).  Rows within R of a border need the mirror
// images of their adjoint values, which only the first (top) and the last
// (bottom) tile compute, so the split between the last two tiles is moved to
// at most n - R, and never below R when there are only two tiles (n >= 2R).
__device__ __forceinline__ int tile_split(int t, int T, int n, int nt, int R)
{
    if (t <= 0) return 0;
    if (t >= nt) return n;
    if (t == nt - 1) return min(t * T, n - R);
    return t * T;
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
    RbfConst rc;
};

}  // namespace tnrd
