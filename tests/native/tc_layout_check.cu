// Host-side check of the tensor-core stage's shared-memory and TMEM layout
// (TcCfg in args.cuh) for every configuration the library instantiates: TF32
// and BF16 with two and three row blocks, split TF32 with two, for 3x3x4,
// 5x5x24 and 7x7x48.  For each it re-derives, from the operand shapes, the
// byte range every MMA descriptor and every staging loop addresses, and checks
// that the range lies inside its own region, that the regions are disjoint and
// in order, and that shared memory and TMEM fit:
//   - filter-bank B (per kernel row: NPAD/8 core matrices 256 B apart, two K
//     cores 128 B apart), adjoint B (two K cores per MMA, LBO_KM apart), the RBF
//     weight table with its window rows;
//   - per warpgroup: the u operand copies (four residues, or the two-slot ring
//     with high and low parts) as the filter-bank A reads them (16 rows of a row
//     block from row 16 nb + 2R - ka, core rows 16 B apart, second K core at +16
//     or +32 B), the raw rows the copies are built from, V (the adjoint's A: 16
//     M groups 128 B apart, two K cores 2 KB apart per MMA), h, the mbarriers;
//   - TMEM: the z buffer(s) and Y inside the warpgroup's columns.
// The backward's kernels (tc_bwd_cfg.cuh) likewise: tc_bwd_adj's filter matrix,
// V rounds, h buffers and TMEM; tc_bwd_dk's interleaved residue rows as its A
// descriptors read them (16 kernel-row groups one row apart from pixel row pr,
// core rows 16 B apart, second K core at +64 B) and its staged B rows (core
// matrices of 8 filters 128 B apart, second K core one quad on).
// Prints "ok <configs>" and exits 0, or prints the first violation and exits 1.
#include <cstdio>
#include "args.cuh"
#include "tc_bwd_cfg.cuh"

static int fails = 0;
#define CHECK(cond, ...)                                                   \
    do {                                                                   \
        if (!(cond)) {                                                     \
            std::printf("KS %d NK %d NB %d BF %d X3 %d: ", KS, NK, NB, BF, X3); \
            std::printf(__VA_ARGS__);                                      \
            std::printf("\n");                                             \
            ++fails;                                                       \
            return;                                                        \
        }                                                                  \
    } while (0)

template <int KS, int NK, int NB, bool BF, bool X3>
void check_cfg()
{
    using C = tnrd::TcCfg<KS, NK, NB, BF, X3>;
    constexpr int R = C::R;
    // ---- totals ----
    CHECK(C::NWG >= 1, "no warpgroup fits");
    CHECK(C::SMEM_BYTES <= 227 * 1024, "shared memory %zu", C::SMEM_BYTES);
    CHECK(C::NWG * C::TMEM_WG <= (int)C::TMEM_COLS && C::TMEM_COLS <= 512, "TMEM %d x %d > %u",
          C::NWG, C::TMEM_WG, C::TMEM_COLS);
    CHECK(C::TMEM_COLS >= 32 && (C::TMEM_COLS & (C::TMEM_COLS - 1)) == 0, "TMEM allocation %u",
          C::TMEM_COLS);
    // ---- shared regions of the CTA ----
    CHECK(C::OFF_BZ + C::NSPL * C::BZ_BYTES <= C::OFF_KM, "filter bank B overlaps Kmat");
    CHECK(C::OFF_KM + C::NSPL * C::KM_BYTES <= C::OFF_W, "Kmat overlaps the weight table");
    CHECK(C::OFF_W + 8ull * C::NR * tnrd::TC_ROWS * 16 <= C::OFF_WG, "weight table overlaps the warpgroups");
    CHECK(C::OFF_WG + (size_t)C::NWG * C::WG_BYTES <= C::OFF_TMEM, "warpgroups overlap the TMEM slot");
    for (size_t off : {C::OFF_BZ, C::OFF_KM, C::OFF_W, C::OFF_WG, C::WG_BYTES})
        CHECK(off % 16 == 0, "offset %zu not 16-byte aligned", off);
    // filter-bank B: kernel row ka at ka NPAD 32 bytes; NPAD / 8 core matrices
    // (SBO 256) of two K cores (LBO 128) of 128 bytes
    {
        const size_t last = (size_t)(KS - 1) * C::NPAD * 32 + (size_t)(C::NPAD / 8 - 1) * 256 + 128 + 128;
        CHECK(last <= C::BZ_BYTES, "filter-bank B reads to %zu of %zu", last, C::BZ_BYTES);
    }
    // adjoint B: k-step s at s 2 LBO_KM; two K cores LBO_KM apart, NT / 8 core
    // matrices 128 B apart
    {
        const size_t lbo = (C::NT / 8) * 128;
        const int steps = C::NKP / C::KMMA;
        const size_t last = (size_t)(steps - 1) * 2 * lbo + lbo + (size_t)(C::NT / 8 - 1) * 128 + 128;
        CHECK(last <= C::KM_BYTES, "adjoint B reads to %zu of %zu", last, C::KM_BYTES);
    }
    // weight table: window rows row .. row + 2 TC_WIN + 1 for the nearest centre
    // j0 in [0, MAX_NRBF), row = j0 + RBF_WPAD - TC_WIN
    CHECK(tnrd::RBF_WPAD - tnrd::TC_WIN >= 0, "window starts before the table");
    CHECK(tnrd::MAX_NRBF - 1 + tnrd::RBF_WPAD - tnrd::TC_WIN + 2 * tnrd::TC_WIN + 1 < tnrd::TC_ROWS,
          "window ends after the table");
    // ---- per warpgroup ----
    CHECK(C::WG_U + C::U_BYTES <= C::WG_RAW, "u copies overlap the raw rows");
    if (C::RING) CHECK(C::WG_RAW + C::RAW_BYTES <= C::WG_V, "raw rows overlap V");
    {
        const size_t v_area = C::RING ? C::NSPL * C::VLO : (C::VLO > C::RAW_BYTES ? C::VLO : C::RAW_BYTES);
        CHECK(C::WG_V + v_area <= C::WG_H, "V overlaps h");
        if (!C::RING) CHECK(C::RAW_BYTES <= v_area, "raw rows do not fit the V area");
    }
    CHECK(C::WG_H + 4ull * C::HROWS * C::HPITCH <= C::WG_MISC, "h overlaps the mbarriers");
    CHECK(C::WG_MISC + 3 * 8 <= C::WG_BYTES, "mbarriers leave the warpgroup");
    for (size_t off : {C::WG_U, C::WG_RAW, C::WG_V, C::WG_H, C::WG_MISC})
        CHECK(off % 16 == 0, "warpgroup offset %zu not 16-byte aligned", off);
    // filter-bank A: group (nb, r), kernel row ka: 16 rows UROWB apart from row
    // 16 nb + 2R - ka; 8 core rows 16 B apart; the second K core at +16 (TF32)
    // or +32 (BF16); in slot s of the copies (high part; X3 low part + U_SLOT)
    {
        const int slots = C::RING ? 2 : 4;
        const size_t slot_stride = C::RING ? C::NSPL * C::U_SLOT : C::U_SLOT;
        for (int s = 0; s < slots; ++s)
            for (int part = 0; part < C::NSPL; ++part)
                for (int nb = 0; nb < NB; ++nb)
                    for (int ka = 0; ka < KS; ++ka) {
                        const int row0 = 16 * nb + 2 * R - ka;
                        CHECK(row0 >= 0, "A starts above the copy");
                        const size_t base = s * slot_stride + part * C::U_SLOT;
                        const size_t end = base + (size_t)(row0 + 15) * C::UROWB + 7 * 16 + (BF ? 32 : 16) + 16;
                        CHECK(end <= base - part * C::U_SLOT + (part + 1) * C::U_SLOT &&
                                  end <= C::U_BYTES,
                              "A of slot %d part %d nb %d ka %d reads to %zu", s, part, nb, ka, end);
                    }
    }
    // residue copies built from the raw rows: TF32 column j + r (j < 36, r < 4);
    // BF16 chunk c covers raw columns 4c + r .. 4c + r + 7 (c < 10)
    {
        const int last_col = BF ? 4 * (C::UCHUNKS - 1) + 3 + 7 : (C::UPITCH - 1) + 3;
        CHECK(last_col < C::RAWC && C::RAWC <= C::RAWP, "copies read raw column %d of %d", last_col, C::RAWC);
        CHECK(C::UROWB * 1 >= (BF ? C::UCHUNKS * 16 : C::UPITCH * 4), "copy row pitch");
    }
    // adjoint A (V): k-step s at s 4096 (+ VLO for the low parts): 16 M groups
    // 128 B apart, two K cores 2048 B apart
    {
        const int steps_held = C::VF / C::KMMA;
        const size_t end = (size_t)(steps_held - 1) * 4096 + 2048 + 15 * 128 + 128;
        CHECK(end <= C::VLO, "V reads to %zu of %zu per part", end, C::VLO);
    }
    // TMEM: z (NPAD columns) and Y (NT columns) inside the warpgroup's columns
    if (C::RING) {
        CHECK(C::NPAD <= 64 && 64 + C::NT <= C::TMEM_WG, "ring TMEM layout");
    } else {
        CHECK(64 + C::NPAD <= C::TMEM_WG && 64 + C::NT <= C::TMEM_WG, "two-buffer TMEM layout");
    }
}

#define CHECKB(cond, ...)                                                  \
    do {                                                                   \
        if (!(cond)) {                                                     \
            std::printf("%s KS %d NK %d X3 %d: ", what, KS, NK, X3);      \
            std::printf(__VA_ARGS__);                                      \
            std::printf("\n");                                             \
            ++fails;                                                       \
            return;                                                        \
        }                                                                  \
    } while (0)

template <int KS, int NK, bool X3>
void check_adj()
{
    const char* what = "tc_bwd_adj";
    using C = tnrd::TcAdjCfg<KS, NK, 2, X3>;
    CHECKB(C::SMEM_BYTES <= 227 * 1024, "shared memory %zu", C::SMEM_BYTES);
    CHECKB(C::NWG * 128 <= (int)C::TMEM_COLS && C::TMEM_COLS <= 512, "TMEM");
    CHECKB(C::OFF_KM + C::NSPL * C::KM_BYTES <= C::OFF_WG, "filter matrix overlaps the warpgroups");
    CHECKB(C::WG_V + C::NSPL * C::VLO <= C::WG_H, "V overlaps h");
    CHECKB(C::WG_H + 4ull * C::HROWS * C::HPITCH <= C::WG_MISC, "h overlaps the mbarrier");
    CHECKB(C::WG_MISC + 8 <= C::WG_BYTES, "mbarrier leaves the warpgroup");
    CHECKB(C::OFF_WG + (size_t)C::NWG * C::WG_BYTES <= C::OFF_TMEM, "warpgroups overlap the TMEM slot");
    // B: k-step (2 rr + s) at (2 rr + s) 2 LBO; two K cores LBO apart, NT / 8 core
    // matrices 128 B apart
    const size_t lbo = (C::NT / 8) * 128;
    const size_t endb = (size_t)(C::NKP / 8 - 1) * 2 * lbo + lbo + (size_t)(C::NT / 8 - 1) * 128 + 128;
    CHECKB(endb <= C::KM_BYTES, "filter matrix read to %zu of %zu", endb, C::KM_BYTES);
    // A (V, one round): two k-steps of 4096 B, 16 M groups 128 B apart, two K cores 2048 B apart
    const size_t enda = 4096 + 2048 + 15 * 128 + 128;
    CHECKB(enda <= C::VLO, "V read to %zu of %zu", enda, C::VLO);
    CHECKB(C::NT <= 64, "Y columns");
}

template <int KS, int NK, bool X3>
void check_dk()
{
    const char* what = "tc_bwd_dk";
    using C = tnrd::TcDkCfg<KS, NK, X3>;
    CHECKB(C::SMEM_BYTES <= 227 * 1024, "shared memory %zu", C::SMEM_BYTES);
    CHECKB(C::NP <= (int)C::TMEM_COLS, "TMEM columns");
    CHECKB(C::OFF_ILD == C::OFF_ILU + C::NSPL * C::IL_BYTES && C::OFF_ST == C::OFF_ILD + C::NSPL * C::IL_BYTES &&
               C::OFF_MISC == C::OFF_ST + C::NBUF * C::BUF_BYTES && C::OFF_MISC + 16 + 4 <= C::SMEM_BYTES,
           "regions out of order");
    CHECKB(C::NBUF <= 2, "mbarriers: two slots");
    // A: pixel row pr, 8-pixel chunk kc: start pr ILP + 2 kc 64; 16 groups ILP
    // apart; 8 core rows 16 B apart; the second K core at +64
    for (int pr = 0; pr < C::TPR; ++pr)
        for (int kc = 0; kc < 4; ++kc) {
            const size_t end = (size_t)(pr + 15) * C::ILP + 2 * kc * 64 + 64 + 7 * 16 + 16;
            CHECKB(end <= C::IL_BYTES, "A of row %d chunk %d reads to %zu of %zu", pr, kc, end, C::IL_BYTES);
            // within one IL row: quads up to 2 kc + 1 + 1 (taps b'' < 8)
            CHECKB(2 * kc * 64 + 64 + 7 * 16 + 16 <= C::ILP, "A leaves its IL row");
        }
    CHECKB(C::ILR_REAL <= C::ILR, "built IL rows");
    // the IL rows real taps read (kernel-row slots a'' < KS) are the built ones
    CHECKB(C::TPR - 1 + KS - 1 < C::ILR_REAL, "real taps read unbuilt IL rows");
    // B: chunk kc at 2 kc QB; NP / 8 core matrices 128 B apart; second K core at +QB
    const size_t endb = (size_t)(2 * 3 + 1) * C::QB + (size_t)(C::NP / 8 - 1) * 128 + 128;
    CHECKB(endb <= C::STG_BYTES, "B reads to %zu of %zu", endb, C::STG_BYTES);
    CHECKB(C::QB % 16 == 0 && (C::QB / 4) % 32 == 4, "staging quad pitch (banks)");
}

int main()
{
    int n = 0;
#define X(K, NN, B)                        \
    check_cfg<K, NN, B, false, false>();   \
    check_cfg<K, NN, B, true, false>();    \
    n += 2;
    X(3, 4, 2) X(3, 4, 3) X(5, 24, 2) X(5, 24, 3) X(7, 48, 2) X(7, 48, 3)
#undef X
    check_cfg<3, 4, 2, false, true>();
    check_cfg<5, 24, 2, false, true>();
    check_cfg<7, 48, 2, false, true>();
    n += 3;
#define Y(K, NN)                 \
    check_adj<K, NN, false>();   \
    check_adj<K, NN, true>();    \
    check_dk<K, NN, false>();    \
    check_dk<K, NN, true>();     \
    n += 4;
    Y(3, 4) Y(5, 24) Y(7, 48)
#undef Y
    if (fails) return 1;
    std::printf("ok %d\n", n);
    return 0;
}
