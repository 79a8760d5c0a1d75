// Host-side checks of the two gridding tables the plan builds (no GPU needed):
//  * build_gather_table: every (cell, antenna, tap) contribution of every footprint appears
//    exactly once, under the lane that owns its cell pair (an entry's tap pair expanded to the
//    covered cells); every cell of a touched row is written exactly once per sample (by a pair's
//    store or a zero step); block offsets stay inside the block; the warps' list steps are
//    balanced;
//  * build_reg64_schedule: every footprint row segment appears once; no two segments of a round
//    share a cell; the 16 lanes of a half-warp start on distinct (y + x0) mod 16 bank pairs;
//    the first-write masks mark exactly one tap per touched cell.
// Usage: schedule_tables_check A K N C P   (exit status 0 when every check holds)
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <set>
#include <vector>

#include "epic_internal.cuh"

static long g_bad = 0;
#define CHECK(cond, ...)                  \
    do {                                  \
        if (!(cond)) {                    \
            if (g_bad < 10) {             \
                std::printf(__VA_ARGS__); \
                std::printf("\n");        \
            }                             \
            g_bad++;                      \
        }                                 \
    } while (0)

int main(int argc, char **argv)
{
    if (argc != 6) return 2;
    const int A = std::atoi(argv[1]), K = std::atoi(argv[2]), N = std::atoi(argv[3]), C = std::atoi(argv[4]),
              P = std::atoi(argv[5]);
    const int M = N == 96 ? 48 : N == 32 ? 32 : 64, h = (K - 1) / 2, S = M + 1;
    std::mt19937 rng(20230120u + A + N);
    std::vector<short2> cells(static_cast<size_t>(C) * A);
    for (auto &c : cells) {   // a centrally condensed layout, as real arrays are
        std::normal_distribution<double> nd(N / 2.0, N / 7.0);
        int x, y;
        do {
            x = static_cast<int>(nd(rng));
            y = static_cast<int>(nd(rng));
        } while (x < h || x >= N - h || y < h || y >= N - h);
        c = make_short2(static_cast<short>(x), static_cast<short>(y));
    }
    std::vector<int> chans(C);
    for (int i = 0; i < C; i++) chans[i] = i;

    // ---- gather table
    std::vector<uint32_t> tab;
    std::vector<int4> idx;
    std::vector<int2> chan;
    std::vector<unsigned long long> rows;
    CHECK(epic::build_gather_table(cells, A, K, M, P, chans, tab, idx, chan, rows) == EPIC_OK, "gather build failed");
    for (int ci = 0; ci < C && g_bad == 0; ci++) {
        std::multiset<long long> want, got;
        unsigned long long want_rows = 0;
        for (int a = 0; a < A; a++) {
            const short2 k = cells[static_cast<size_t>(ci) * A + a];
            for (int dyi = 0; dyi < K; dyi++)
                for (int dx = 0; dx < K; dx++) {
                    const int y = ((k.y % M + dyi - h) % M + M) % M, x = ((k.x % M + dx - h) % M + M) % M;
                    want_rows |= 1ull << y;
                    want.insert((static_cast<long long>(y * S + x) << 32) | (static_cast<long long>(a) << 8) |
                                (dyi * K + dx));
                }
        }
        CHECK(rows[ci] == want_rows, "channel %d: touched-row mask", ci);
        std::map<uint32_t, int> written;
        const long long base = chan[ci].x, end = base + chan[ci].y;
        long long wmin = 1LL << 40, wmax = 0, dmax = 0;
        for (int w = 0; w < 8; w++) {
            const int4 ix = idx[ci * 8 + w];
            for (int r = 0; r < ix.y; r++)
                for (int l = 0; l < 32; l++) {
                    const long long at = base + ix.x + r * 32 + l;
                    CHECK(at < end, "channel %d warp %d: zero list outside its block", ci, w);
                    if (at < end && tab[at] != ~0u) written[tab[at]]++;
                }
            long long off = base + ix.z, steps = 0;
            for (int b = 0; b < ix.w && off < end; b++) {
                const int d = static_cast<int>(tab[off]);
                CHECK(off + 33 + 32LL * d <= end, "channel %d warp %d: batch outside its block", ci, w);
                if (off + 33 + 32LL * d > end) break;
                for (int l = 0; l < 32; l++) {
                    const uint32_t cell = tab[off + 1 + l];   // left cell of the pair
                    if (cell != ~0u) {
                        CHECK((cell % S) % 2 == 0, "channel %d: pair not starting at an even column", ci);
                        written[cell]++;
                        written[cell + 1]++;
                    }
                    for (int j = 0; j < d; j++) {
                        const uint32_t e = tab[off + 33 + 32LL * j + l];
                        if (e == ~0u) continue;
                        CHECK(cell != ~0u, "channel %d: entry under an empty lane", ci);
                        const long long a = e >> 8;
                        const int tp = e & 0xFF, dyi = tp / (K + 1), dxl = tp % (K + 1) - 1;
                        CHECK(dyi < K && (dxl >= 0 || dxl + 1 < K), "channel %d: tap pair %d", ci, tp);
                        if (dxl >= 0)
                            got.insert((static_cast<long long>(cell) << 32) | (a << 8) | (dyi * K + dxl));
                        if (dxl + 1 < K)
                            got.insert((static_cast<long long>(cell + 1) << 32) | (a << 8) | (dyi * K + dxl + 1));
                    }
                }
                off += 33 + 32LL * d;
                steps += d;
                dmax = std::max(dmax, static_cast<long long>(d));
            }
            wmin = std::min(wmin, steps);
            wmax = std::max(wmax, steps);
        }
        CHECK(want == got, "channel %d: contributions differ (%zu wanted, %zu listed)", ci, want.size(), got.size());
        for (int y = 0; y < M; y++)
            for (int x = 0; x < M; x++) {
                const uint32_t cell = static_cast<uint32_t>(y * S + x);
                const int n = written.count(cell) ? written[cell] : 0;
                CHECK(n == (((want_rows >> y) & 1ull) ? 1 : 0), "channel %d: cell (%d, %d) written %d times", ci, y,
                      x, n);
            }
        // balance (longest batch first to the least-loaded warp): the warps' list steps differ by at
        // most one batch
        CHECK(wmax - wmin <= dmax, "channel %d: warp list steps %lld .. %lld (longest batch %lld)", ci, wmin,
              wmax, dmax);
    }

    // ---- round schedule (tensor kernels)
    if (M == 64 || M == 48) {
        std::vector<uint32_t> desc;
        std::vector<int> nr;
        int rmax = 0;
        std::vector<unsigned long long> rows2;
        std::vector<uint16_t> first;
        CHECK(epic::build_reg64_schedule(cells, A, K, M, chans, desc, nr, rmax, rows2, first) == EPIC_OK,
              "round schedule build failed");
        for (int ci = 0; ci < C && g_bad == 0; ci++) {
            CHECK(rows2[ci] == rows[ci], "channel %d: row masks of the two tables differ", ci);
            std::multiset<long long> want, got;
            for (int a = 0; a < A; a++) {
                const short2 k = cells[static_cast<size_t>(ci) * A + a];
                for (int dyi = 0; dyi < K; dyi++) want.insert((static_cast<long long>(a) << 8) | dyi);
            }
            std::map<int, int> first_taps;
            for (int w = 0; w < 8; w++)
                for (int r = 0; r < nr[ci * 8 + w]; r++) {
                    std::set<int> used;
                    int res_seen[2][16] = {};
                    for (int l = 0; l < 32; l++) {
                        const size_t at = ((static_cast<size_t>(ci) * 8 + w) * rmax + r) * 32 + l;
                        const uint32_t d = desc[at];
                        if (!(d >> 31)) continue;
                        const int a = d & 0xFFF, dyi = (d >> 12) & 0xF, y = (d >> 16) & 0x3F, x0 = (d >> 22) & 0x3F;
                        got.insert((static_cast<long long>(a) << 8) | dyi);
                        CHECK(y % 8 == w, "channel %d: row %d in warp %d", ci, y, w);
                        CHECK(res_seen[l / 16][(y + x0) % 16]++ == 0, "channel %d: bank residue repeated", ci);
                        for (int dx = 0; dx < K; dx++) {
                            const int cell = y * M + (x0 + dx) % M;
                            CHECK(used.insert(cell).second, "channel %d: two segments of a round share a cell", ci);
                            if ((first[at] >> dx) & 1u) first_taps[cell]++;
                        }
                    }
                }
            CHECK(want == got, "channel %d: row segments differ", ci);
            for (auto &kv : first_taps) CHECK(kv.second == 1, "channel %d: cell with %d first writes", ci, kv.second);
        }
    }
    std::printf("%s: A=%d K=%d N=%d C=%d P=%d, %zu table words, %ld failures\n", g_bad ? "FAIL" : "ok", A, K, N, C,
                P, tab.size(), g_bad);
    return g_bad ? 1 : 0;
}
