// Tile configurations of the backward's tensor-core kernels (csrc/tc_bwd.cu):
// shared-memory layout, TMEM columns and threads.  Host-visible so that the
// layout checks can see them.
#pragma once
#include <cstddef>
#include <cstdint>

namespace tnrd {

// tc_bwd_adj: the adjoint dL/du_{t-1} = d + fold(sum_i K_i^T c_i) per tile of
// (16 NB - 2R) x (32 - 2R) outputs over 16 NB x 32 positions; four warpgroups,
// each with one round of V (16 filters, high then low parts), its h buffer and
// an mbarrier; the filter matrix (high, low) shared.
template <int KS, int NK, int NB, bool X3>
struct TcAdjCfg {
    static constexpr int R = KS / 2;
    static constexpr int TW = 32 - 2 * R;
    static constexpr int ZR = 16 * NB;                   // position rows per tile
    static constexpr int TH = ZR - 2 * R;
    static constexpr int NKP = (NK + 7) / 8 * 8;         // K of the GEMM (TF32: 8 per MMA)
    static constexpr int NT = (KS * KS + 15) / 16 * 16;  // N (taps)
    static constexpr int NR = (NK + 15) / 16;            // rounds of 16 filters
    static constexpr int NSPL = X3 ? 2 : 1;
    static constexpr int HROWS = ZR + 2 * R;
    static constexpr int HPITCH = 41;
    static constexpr size_t al(size_t x) { return (x + 127) / 128 * 128; }
    static constexpr size_t KM_BYTES = 4ull * NT * NKP;
    static constexpr size_t OFF_KM = 0;
    static constexpr size_t OFF_WG = al(OFF_KM + NSPL * KM_BYTES);
    static constexpr size_t VLO = 4ull * 128 * 16;       // one round, high parts; low parts after
    static constexpr size_t WG_V = 0;
    static constexpr size_t WG_H = al(WG_V + NSPL * VLO);
    static constexpr size_t WG_MISC = al(WG_H + 4ull * HROWS * HPITCH);
    static constexpr size_t WG_BYTES = al(WG_MISC + 32);
    static constexpr int NWG = 4;
    static constexpr int NTHREADS = 128 * NWG;
    static constexpr size_t OFF_TMEM = OFF_WG + (size_t)NWG * WG_BYTES;
    static constexpr size_t SMEM_BYTES = OFF_TMEM + 16;
    static constexpr uint32_t TMEM_COLS = 512;           // 128 per warpgroup, Y in the first 64
    static_assert(NT <= 64, "Y fits one 64-column buffer");
    static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
};

// tc_bwd_dk: the filter gradient per tile of 32 columns x TPR rows of pixels;
// interleaved residue rows of u and d (high, low parts), NBUF staging buffers
// of one pixel row of c and -v, two mbarriers and the TMEM slot.
template <int KS, int NK, bool X3>
struct TcDkCfg {
    static constexpr int R = KS / 2;
    static constexpr int TPR = 16;                       // pixel rows per tile
    static constexpr int NP = (NK + 15) / 16 * 16;       // N (filters, padded)
    static constexpr int NCOLQ = 10;                     // quads of an IL row (pixel quads 0..7 + 2)
    static constexpr int ILP = NCOLQ * 64;               // bytes per IL row
    static constexpr int ILR = TPR + 16;                 // IL rows the MMAs address (16 slots per pixel row)
    static constexpr int ILR_REAL = TPR + 2 * R;         // IL rows real taps read (the rest stay unwritten)
    static constexpr int NBUF = 1;                       // staging buffers
    static constexpr int NSPL = X3 ? 2 : 1;
    static constexpr size_t IL_BYTES = (size_t)ILR * ILP;
    static constexpr int QB = NP * 16 + 16;              // staging bytes per quad
    static constexpr size_t STG_BYTES = 8ull * QB;       // one pixel row of c (or -v)
    static constexpr size_t OFF_ILU = 0;                 // u: high parts, then low
    static constexpr size_t OFF_ILD = OFF_ILU + NSPL * IL_BYTES;
    // staging buffer s (0, 1) at OFF_ST + s BUF_BYTES: c high, c low, -v high, -v low
    static constexpr size_t OFF_ST = OFF_ILD + NSPL * IL_BYTES;
    static constexpr size_t BUF_BYTES = 2 * NSPL * STG_BYTES;
    static constexpr size_t OFF_MISC = OFF_ST + NBUF * BUF_BYTES;
    static constexpr size_t SMEM_BYTES = OFF_MISC + 32;
    static constexpr uint32_t TMEM_COLS = NP <= 32 ? 32 : 64;
    static_assert(ILP % 16 == 0 && QB % 16 == 0, "descriptor strides");
    static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
};

}  // namespace tnrd
