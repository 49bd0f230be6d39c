// Host check of the stream-K GEMM's work split (stream_k.cuh): for many
// (tiles, K slices, grid) combinations, every iteration is computed exactly
// once, partial tiles only occur at the ends of a CTA's range, workspace
// slots are unique and in range, and the summing kernel's view of each tile
// (sk_tile_ctas, sk_piece_slot) names exactly the pieces that were written.
// Prints "ok <cases>" and exits 0, or reports the first violation and exits 1.
#include <cstdio>
#include <map>
#include <set>
#include <utility>
#include <vector>

#include "../paper_2104_04609_gb300/csrc/stream_k.cuh"

static int fail(const char *what, int tiles, int KB, int G) {
    std::printf("FAIL %s tiles=%d KB=%d G=%d\n", what, tiles, KB, G);
    return 1;
}

static int check(int tiles, int KB, int G) {
    const long long iters = (long long)tiles * KB;
    if (G < 1 || G > iters) return 0;
    if (sk_begin(0, iters, G) != 0 || sk_begin(G, iters, G) != iters) return fail("range ends", tiles, KB, G);
    std::vector<std::vector<int>> cover(tiles, std::vector<int>(KB, 0));
    std::map<int, std::vector<std::pair<int, int>>> pieces;  // tile -> (cta, slot)
    std::vector<int> whole(tiles, 0);
    std::set<int> slots;
    for (int c = 0; c < G; ++c) {
        const long long b = sk_begin(c, iters, G), e = sk_begin(c + 1, iters, G);
        if (e <= b) return fail("empty range", tiles, KB, G);
        int seg = 0;
        for (long long it = b; it < e; ++seg) {
            const SkSeg s = sk_next(it, e, KB);
            if (s.n < 1 || s.kb0 < 0 || s.kb0 + s.n > KB || s.tile < 0 || s.tile >= tiles)
                return fail("segment bounds", tiles, KB, G);
            for (int k = s.kb0; k < s.kb0 + s.n; ++k) ++cover[s.tile][k];
            const bool is_whole = s.kb0 == 0 && s.n == KB;
            const bool last = it + s.n == e;
            if (is_whole) {
                ++whole[s.tile];
            } else {
                if (seg != 0 && !last) return fail("partial segment inside a range", tiles, KB, G);
                const int slot = sk_slot(c, seg);
                if (slot < 0 || slot >= 2 * G || !slots.insert(slot).second)
                    return fail("slot out of range or reused", tiles, KB, G);
                pieces[s.tile].push_back({c, slot});
            }
            it += s.n;
        }
    }
    for (int t = 0; t < tiles; ++t) {
        for (int k = 0; k < KB; ++k)
            if (cover[t][k] != 1) return fail("iteration not covered exactly once", tiles, KB, G);
        int lo, hi;
        sk_tile_ctas(t, KB, iters, G, &lo, &hi);
        if (lo < 0 || hi >= G || lo > hi) return fail("tile CTA range", tiles, KB, G);
        if (lo == hi) {
            if (whole[t] != 1 || pieces.count(t)) return fail("single-CTA tile not whole", tiles, KB, G);
            continue;
        }
        if (whole[t] != 0) return fail("split tile also written whole", tiles, KB, G);
        std::vector<std::pair<int, int>> want;
        for (int c = lo; c <= hi; ++c) want.push_back({c, sk_piece_slot(c, t, KB, iters, G)});
        if (want != pieces[t]) return fail("summed pieces differ from written pieces", tiles, KB, G);
    }
    return 0;
}

int main() {
    long long cases = 0;
    const int tile_list[] = {1, 2, 3, 5, 7, 16, 47, 63, 125, 152, 153, 304, 400, 800};
    const int kb_list[] = {1, 2, 3, 5, 8, 64, 125, 128, 188, 500};
    for (int tiles : tile_list)
        for (int KB : kb_list) {
            const long long iters = (long long)tiles * KB;
            std::set<int> grids = {1, 2, 3, 7, 48, 85, 151, 152, 153, 304};
            long long g = iters / 48;  // the library's choice: one CTA per SM, 48 slices at least
            if (g > 152) g = 152;
            if (g < 1) g = 1;
            grids.insert((int)g);
            if (iters <= 400) grids.insert((int)iters);
            for (int G : grids) {
                if (check(tiles, KB, G)) return 1;
                ++cases;
            }
        }
    std::printf("ok %lld\n", cases);
    return 0;
}
