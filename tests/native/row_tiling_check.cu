// Host-side exhaustive check of the fused stage's row tiling (row_tile in
// args.cuh, the function every fused kernel uses to place its tile and pick
// the rows it writes).  For every image height, tile height and border-tile
// height the per-call kernels can be given, and both tilings (uniform and
// short border rows), checks that
//   - the written ranges of the tiles partition [0, H) in order,
//   - each tile writes only rows it covers, and covers only image rows
//     (when the image holds a whole tile),
//   - rows within R of a border are written by a border tile (the first or
//     the last), which computes their mirror contributions,
//   - with short border rows, the last interior tile writes at least 2R rows,
//   - row_tiles() gives the tile count the host launches with.
// Prints "ok <cases>" and exits 0, or prints the first violation and exits 1.
#include <cstdio>
#include "args.cuh"

using tnrd::RowTile;

static int check(int H, int th, int te, int R)
{
    const int nt = tnrd::row_tiles(H, th, te);
    if (nt < 1) return std::printf("H %d th %d te %d: %d tiles\n", H, th, te, nt), 1;
    int next = 0;
    for (int t = 0; t < nt; ++t) {
        const RowTile r = tnrd::row_tile(t, nt, H, th, te, R);
        const bool border = (t == 0) || (t == nt - 1);
        if (r.wy0 != next || r.wy1 < r.wy0)
            return std::printf("H %d th %d te %d R %d tile %d: writes [%d, %d), expected from %d\n",
                               H, th, te, R, t, r.wy0, r.wy1, next), 1;
        next = r.wy1;
        if (r.wy1 > r.wy0 && (r.wy0 < r.y0 || r.wy1 > r.y0 + r.h))
            return std::printf("H %d th %d te %d R %d tile %d: writes [%d, %d) outside its rows [%d, %d)\n",
                               H, th, te, R, t, r.wy0, r.wy1, r.y0, r.y0 + r.h), 1;
        if (H >= r.h && (r.y0 < 0 || r.y0 + r.h > H))
            return std::printf("H %d th %d te %d tile %d: rows [%d, %d) leave the image\n",
                               H, th, te, t, r.y0, r.y0 + r.h), 1;
        if (!border && r.wy1 > r.wy0 && (r.wy0 < R || r.wy1 > H - R))
            return std::printf("H %d th %d te %d R %d tile %d: interior tile writes border rows [%d, %d)\n",
                               H, th, te, R, t, r.wy0, r.wy1), 1;
        if (te > 0 && t == nt - 2 && t > 0 && r.wy1 - r.wy0 < 2 * R)
            return std::printf("H %d th %d te %d R %d: last interior tile writes %d rows\n",
                               H, th, te, R, r.wy1 - r.wy0), 1;
    }
    if (next != H) return std::printf("H %d th %d te %d: rows end at %d\n", H, th, te, next), 1;
    return 0;
}

int main()
{
    long cases = 0;
    for (int R = 1; R <= 3; ++R) {
        const int ks = 2 * R + 1;
        for (int th = 2 * R + 1; th <= 45; ++th) {
            for (int H = ks; H <= 700; ++H) {
                if (check(H, th, 0, R)) return 1;
                ++cases;
                const int te = th - 2 * R;   // the short border rows the host picks
                if (te >= 2 * R && H >= 2 * te + th) {
                    if (check(H, th, te, R)) return 1;
                    ++cases;
                }
            }
        }
    }
    std::printf("ok %ld\n", cases);
    return 0;
}
