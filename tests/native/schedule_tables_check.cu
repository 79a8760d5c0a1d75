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
#include "tc_common.cuh"

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
    {   // the same table from one host thread and from three
        for (int nt : {1, 3}) {
            std::vector<uint32_t> tab1;
            std::vector<int4> idx1;
            std::vector<int2> chan1;
            std::vector<unsigned long long> rows1;
            CHECK(epic::build_gather_table(cells, A, K, M, P, chans, tab1, idx1, chan1, rows1, nt) == EPIC_OK,
                  "gather build on %d threads failed", nt);
            bool same = tab1 == tab && rows1 == rows && idx1.size() == idx.size() && chan1.size() == chan.size();
            for (size_t i = 0; same && i < idx.size(); i++)
                same = idx1[i].x == idx[i].x && idx1[i].y == idx[i].y && idx1[i].z == idx[i].z && idx1[i].w == idx[i].w;
            for (size_t i = 0; same && i < chan.size(); i++) same = chan1[i].x == chan[i].x && chan1[i].y == chan[i].y;
            CHECK(same, "gather table built on %d threads differs from the default build", nt);
        }
    }
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
    // ---- pair lists of the grid-side-128 tensor kernel, for a layout whose rows fold without
    // overlap (a 60-row band): the same (cell pair, antenna, tap pair) entries as the FP32 table,
    // each warp's batches split in two halves that cover them once, offsets inside the block, the
    // upper-row mask, and no list for a layout whose rows overlap after folding
    long long pair_words = -1;
    if ((N == 128 || N == 96) && P == 2 && K * (K + 1) <= 63 && A <= 1024) {
        // the pair kernel's lists (folded side M = 64 or 48): an aperture band of M - 4 rows
        const int span = M - 4;
        std::vector<short2> band(cells);
        for (auto &c : band) c.y = static_cast<short>(M - span / 2 + ((c.y - h) % (span - 2 * h)) + h);
        std::vector<uint32_t> t32;
        std::vector<int4> i32, pidx;
        std::vector<int2> c32, pchan;
        std::vector<unsigned long long> r32, upper;
        std::vector<uint16_t> ptab;
        CHECK(epic::build_gather_table(band, A, K, M, P, chans, t32, i32, c32, r32) == EPIC_OK, "band table");
        // every schedule the autotuner tries deals the same batches: same sizes, same per-channel blocks
        const epic::PairSchedule scheds[] = {{90, 80}, {0, 0}, {150, 67}, {60, 100}};
        for (const epic::PairSchedule &ps : scheds) {
            std::vector<int4> pidx_s;
            std::vector<int2> pchan_s;
            std::vector<unsigned long long> upper_s;
            std::vector<uint16_t> ptab_s;
            CHECK(epic::build_pair_tables(band, A, K, chans, t32, i32, c32, ptab_s, pidx_s, pchan_s, upper_s, ps, M) ==
                      EPIC_OK,
                  "pair lists build failed (schedule %d/%d)", ps.tmem_load, ps.first_pct);
            if (ps.tmem_load == 90 && ps.first_pct == 80) {
                ptab = ptab_s;
                pidx = pidx_s;
                pchan = pchan_s;
                upper = upper_s;
                continue;
            }
            bool same = ptab_s.size() == ptab.size() && pidx_s.size() == pidx.size() && upper_s == upper;
            for (size_t i = 0; same && i < pchan.size(); i++) same = pchan_s[i].x == pchan[i].x && pchan_s[i].y == pchan[i].y;
            std::multiset<uint16_t> a(ptab.begin(), ptab.end()), b(ptab_s.begin(), ptab_s.end());
            CHECK(same && a == b, "schedule %d/%d changes the lists' sizes or content", ps.tmem_load, ps.first_pct);
        }
        CHECK(!ptab.empty(), "pair lists build failed");
        for (int ci = 0; ci < C && g_bad == 0; ci++) {
            unsigned long long up = 0;
            for (int a = 0; a < A; a++)
                for (int dy = -h; dy <= h; dy++) {
                    const int ky = band[static_cast<size_t>(ci) * A + a].y + dy;
                    if (ky >= M) up |= 1ull << (ky - M);
                }
            CHECK(up == upper[ci], "channel %d: upper-row mask", ci);
            std::multiset<long long> want, got;
            const uint32_t *blk = t32.data() + c32[ci].x;
            for (int w = 0; w < 8; w++) {
                const int4 q = i32[static_cast<size_t>(ci) * 8 + w];
                long long off = q.z;
                for (int b = 0; b < q.w; b++) {
                    const int d = static_cast<int>(blk[off]);
                    for (int l = 0; l < 32; l++) {
                        const uint32_t cw = blk[off + 1 + l];
                        for (int j = 0; j < d; j++) {
                            const uint32_t e = blk[off + 33 + 32LL * j + l];
                            if (e == ~0u || cw == ~0u) continue;
                            const long long pos = (cw / S) * 32 + (cw % S) / 2;
                            want.insert((pos << 24) | ((e >> 8) << 8) | (e & 0xFF));
                        }
                    }
                    off += 33 + 32LL * d;
                }
            }
            const uint16_t *pb = ptab.data() + pchan[ci].x;
            for (int w = 0; w < epic::kPairGatherWarps; w++) {
                const int4 q = pidx[static_cast<size_t>(ci) * epic::kPairGatherWarps + w];
                CHECK(w < 8 || q.w == 0, "channel %d: a gridding-only warp with a second list", ci);
                for (int half = 0; half < 2; half++) {
                    long long off = half ? q.z : q.x;
                    const int nb = half ? q.w : q.y;
                    for (int b = 0; b < nb; b++) {
                        CHECK(off + 33 <= pchan[ci].y, "channel %d: batch header outside the block", ci);
                        const int d = pb[off];
                        CHECK(off + 33 + 32LL * d <= pchan[ci].y, "channel %d: batch outside the block", ci);
                        for (int l = 0; l < 32; l++) {
                            // the lane's G16 byte offset (pol 0, Re, hi part) back to its cell pair
                            const uint16_t go = pb[off + 1 + l];
                            const int y = (go / 2048) * 8 + (go % 128) / 16;
                            const int k = ((go % 2048) / 128) * 8 + (go % 16) / 2;
                            const bool lane_ok = go != 0xFFFFu && y < M && k < M && k % 2 == 0 &&
                                                 epic::tcc::k_off(y, k) == go;
                            for (int j = 0; j < d; j++) {
                                const uint16_t e = pb[off + 33 + 32LL * j + l];
                                const long long a = e & 1023, tp = e >> 10;
                                CHECK(a < A && tp <= K * (K + 1), "channel %d: entry out of range", ci);
                                if (tp == K * (K + 1)) continue;   // an empty step: the zero tap slot (any antenna)
                                CHECK(lane_ok, "channel %d: entry under an empty or bad lane offset", ci);
                                const long long pos = y * 32 + k / 2;
                                got.insert((pos << 24) | (a << 8) | tp);
                            }
                        }
                        off += 33 + 32LL * d;
                    }
                }
            }
            CHECK(want == got, "channel %d: pair lists differ from the FP32 table (%zu vs %zu)", ci, want.size(),
                  got.size());
            pair_words = std::max<long long>(pair_words, pchan[ci].y);
        }
        // rows that overlap after folding (one footprint in rows 0.., one in rows 64..): no pair lists
        if (A > 1) {
            std::vector<short2> wide(band);
            for (int ci = 0; ci < C; ci++) {
                wide[static_cast<size_t>(ci) * A].y = static_cast<short>(h);
                wide[static_cast<size_t>(ci) * A + 1].y = static_cast<short>(M + h);
            }
            std::vector<uint32_t> t2;
            std::vector<int4> i2, pidx2;
            std::vector<int2> c2, pchan2;
            std::vector<unsigned long long> r2, up2;
            std::vector<uint16_t> pt2;
            CHECK(epic::build_gather_table(wide, A, K, M, P, chans, t2, i2, c2, r2) == EPIC_OK, "wide table");
            CHECK(epic::build_pair_tables(wide, A, K, chans, t2, i2, c2, pt2, pidx2, pchan2, up2, epic::PairSchedule(), M) ==
                      EPIC_ERR_UNSUPPORTED,
                  "rows that overlap after folding were accepted");
        }
    }
    std::printf("%s: A=%d K=%d N=%d C=%d P=%d, %zu table words, %lld pair words, %ld failures\n", g_bad ? "FAIL" : "ok",
                A, K, N, C, P, tab.size(), pair_words, g_bad);
    return g_bad ? 1 : 0;
}
