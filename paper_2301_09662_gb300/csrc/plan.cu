// Plan construction and the C entry points of libepic.
//
// epic_plan validates the geometry, maps antennas to grid cells (Sec. 3.1),
// builds the kernel image |W^(l)|^2 used by the autocorrelation subtraction
// (Sec. 2.2, Eq. 4), the FP32 twiddle tables, and the workspace.  Everything
// here runs once per plan; the per-integration work is in the kernels.
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <thread>
#include <map>
#include <new>

#include "epic_internal.cuh"

using epic::GroupCfg;

namespace {

bool supported_n(int n) { return n == 32 || n == 64 || n == 96 || n == 128 || n == 256 || n == 512; }

// Folding factor per grid side for the FP32 kernel (folded side M = N / Q1).
int fold_for(int n)
{
    switch (n) {
    case 32: return 1;    // M = 32
    case 64: return 1;    // M = 64
    case 96: return 2;    // M = 48
    case 128: return 2;   // M = 64
    case 256: return 4;   // M = 64
    case 512: return 8;   // M = 64
    default: return 0;
    }
}

template <class T>
int dev_upload(T **dst, const T *src, size_t n)
{
    *dst = nullptr;
    if (n == 0) return EPIC_OK;
    if (cudaMalloc(reinterpret_cast<void **>(dst), n * sizeof(T)) != cudaSuccess) {
        *dst = nullptr;
        return EPIC_ERR_NOMEM;
    }
    if (src && cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return EPIC_ERR_CUDA;
    return EPIC_OK;
}

void free_plan(epic_plan_s *p)
{
    if (!p) return;
    for (auto e : p->events) cudaEventDestroy(e);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    for (auto st : p->side) cudaStreamDestroy(st);
    for (auto e : p->ev_join) cudaEventDestroy(e);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_auto) cudaEventDestroy(p->ev_auto);
    if (p->cap) cudaStreamDestroy(p->cap);
    cudaFree(p->d_cells);
    cudaFree(p->d_kernel);
    cudaFree(p->d_dft);
    cudaFree(p->d_dft48);
    cudaFree(p->d_bauto);
    cudaFree(p->d_autoint);
    cudaFree(p->d_status);
    cudaFree(p->d_dfreq);
    cudaFree(p->d_dtab);
    cudaFree(p->d_stage_v);
    cudaFree(p->d_stage_g);
    cudaFree(p->d_stage_out);
    if (p->s_up) cudaStreamSynchronize(p->s_up);
    if (p->s_down) cudaStreamSynchronize(p->s_down);
    for (int i = 0; i < 2; i++) {
        cudaFree(p->d_ring_v[i]);
        cudaFree(p->d_ring_g[i]);
        cudaFree(p->d_ring_out[i]);
        for (cudaEvent_t e : {p->ev_up[i], p->ev_in_free[i], p->ev_img[i], p->ev_out_free[i]})
            if (e) cudaEventDestroy(e);
    }
    if (p->s_up) cudaStreamDestroy(p->s_up);
    if (p->s_down) cudaStreamDestroy(p->s_down);
    for (auto &g : p->groups) {
        cudaFree(g.d_chans);
        cudaFree(g.d_out_off);
        cudaFree(g.d_wpow);
        cudaFree(g.d_twN);
        cudaFree(g.d_partial);
        cudaFree(g.d_sched);
        cudaFree(g.d_first);
        cudaFree(g.d_nrounds);
        cudaFree(g.d_gf);
        cudaFree(g.d_j0);
        cudaFree(g.d_bseg);
        cudaFree(g.d_boff);
        cudaFree(g.d_rowmask);
        cudaFree(g.d_gtab);
        cudaFree(g.d_gidx);
        cudaFree(g.d_gchan);
        cudaFree(g.d_tw64);
        cudaFree(g.d_Y);
        cudaFree(g.d_ptab);
        cudaFree(g.d_pchan);
        cudaFree(g.d_pidx);
        cudaFree(g.d_upper);
        cudaFree(g.d_ef_off);
    }
    delete p;
}

// |W^(l)|^2, W^(l) = sum_d W(d) exp(+2 pi i d.l / N), on the shifted layout
// out[i][j] with l = (j - N/2, i - N/2).  FP64, separable phase tables.
void kernel_power(const float *kern, int K, int N, std::vector<double> &out)
{
    const int h = (K - 1) / 2;
    std::vector<std::complex<double>> ph(static_cast<size_t>(K) * N);  // [d + h][l index]
    for (int d = -h; d <= h; d++)
        for (int i = 0; i < N; i++) {
            const int l = i - N / 2;
            const long e = (((long)d * l) % N + N) % N;
            const double ang = 2.0 * M_PI * static_cast<double>(e) / N;
            ph[static_cast<size_t>(d + h) * N + i] = {std::cos(ang), std::sin(ang)};
        }
    out.assign(static_cast<size_t>(N) * N, 0.0);
    std::vector<std::complex<double>> rowsum(static_cast<size_t>(K) * N);  // [dy][j]
    for (int dy = 0; dy < K; dy++)
        for (int j = 0; j < N; j++) {
            std::complex<double> s = 0;
            for (int dx = 0; dx < K; dx++) {
                std::complex<double> w(kern[2 * (dy * K + dx)], kern[2 * (dy * K + dx) + 1]);
                s += w * ph[static_cast<size_t>(dx) * N + j];
            }
            rowsum[static_cast<size_t>(dy) * N + j] = s;
        }
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            std::complex<double> s = 0;
            for (int dy = 0; dy < K; dy++) s += rowsum[static_cast<size_t>(dy) * N + j] * ph[static_cast<size_t>(dy) * N + i];
            out[static_cast<size_t>(i) * N + j] = std::norm(s);
        }
}

}  // namespace

namespace epic {

int host_cell_map(const double *ant_xy_m, int n_ant, const double *freq_hz, int n_chan, const int *grid_n,
                  double du, int K, std::vector<short2> &cells)
{
    double sx = 0, sy = 0;
    for (int a = 0; a < n_ant; a++) { sx += ant_xy_m[2 * a]; sy += ant_xy_m[2 * a + 1]; }
    const double cx = sx / n_ant, cy = sy / n_ant;
    const int h = (K - 1) / 2;
    cells.assign(static_cast<size_t>(n_chan) * n_ant, make_short2(0, 0));
    for (int c = 0; c < n_chan; c++) {
        const int N = grid_n[c];
        for (int a = 0; a < n_ant; a++) {
            const double x = ant_xy_m[2 * a] - cx, y = ant_xy_m[2 * a + 1] - cy;
            const double fx = (x * freq_hz[c]) / (kC0 * du);
            const double fy = (y * freq_hz[c]) / (kC0 * du);
            if (std::fabs(fx) > 1e6 || std::fabs(fy) > 1e6) return EPIC_ERR_OUT_OF_GRID;
            const long long kx = std::llround(fx) + N / 2;
            const long long ky = std::llround(fy) + N / 2;
            if (kx - h < 0 || kx + h >= N || ky - h < 0 || ky + h >= N) return EPIC_ERR_OUT_OF_GRID;
            cells[static_cast<size_t>(c) * n_ant + a] = make_short2(static_cast<short>(kx), static_cast<short>(ky));
        }
    }
    return EPIC_OK;
}

void host_kernel_power(const float *kern, int K, int N, std::vector<double> &out) { kernel_power(kern, K, N, out); }

// A kernel's dynamic shared-memory cap holds for the whole process, so it is
// raised to the most the device allows beside the kernel's static shared
// memory rather than to one caller's size: a later plan or call that needs
// less must not lower it under one that needs more.
int raise_dyn_smem_cap(const void *kfn, size_t need)
{
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, kfn) != cudaSuccess)
        return EPIC_ERR_CUDA;
    const long long cap = static_cast<long long>(optin) - static_cast<long long>(fa.sharedSizeBytes);
    if (cap < 0 || need > static_cast<size_t>(cap)) return EPIC_ERR_UNSUPPORTED;
    return cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(cap)) ==
                   cudaSuccess
               ? EPIC_OK
               : EPIC_ERR_UNSUPPORTED;
}

// Gridding schedule of the register-transform kernels (fold side M = 64 or 48).
// Each antenna footprint is cut into K row segments (one per dy) of K cells on
// the folded M x M grid.  Warp w owns rows y = w (mod 8); its segments are
// packed greedily into rounds of 32 lanes such that (a) no two segments of a
// round share a cell, so a round can read-add-write without atomics, and (b)
// the 16 lanes of each half-warp start at distinct (y + x) mod 16, which with
// the row stride of M + 1 float2 (65 or 49, both 1 mod 16) puts every lane of
// a half-warp on its own pair of banks for each of the K cells.
int build_reg64_schedule(const std::vector<short2> &cells, int A, int K, int M, const std::vector<int> &chans,
                         std::vector<uint32_t> &desc, std::vector<int> &nrounds, int &rmax,
                         std::vector<unsigned long long> &rowmask, std::vector<uint16_t> &first)
{
    constexpr int W = 8;
    const int h = (K - 1) / 2;
    if (A > 4096 || K > 15 || (M != 64 && M != 48)) return EPIC_ERR_UNSUPPORTED;
    struct Round {
        uint32_t lane[32];
        uint64_t rowmask[64 / W];
    };
    const int nc = static_cast<int>(chans.size());
    std::vector<std::vector<std::vector<Round>>> all(nc, std::vector<std::vector<Round>>(W));
    rowmask.assign(nc, 0ull);
    rmax = 0;
    for (int ci = 0; ci < nc; ci++) {
        const int c = chans[ci];
        for (int a = 0; a < A; a++) {
            const short2 k = cells[static_cast<size_t>(c) * A + a];
            const int jx = k.x % M, jy = k.y % M;
            const int x0 = ((jx - h) % M + M) % M;
            uint64_t mask = 0;
            for (int dx = 0; dx < K; dx++) mask |= 1ull << ((x0 + dx) % M);
            for (int dyi = 0; dyi < K; dyi++) {
                const int y = ((jy + dyi - h) % M + M) % M;
                const int w = y % W, res = (y + x0) % 16;
                rowmask[ci] |= 1ull << y;
                const uint32_t d = (1u << 31) | (static_cast<uint32_t>(x0) << 22) | (static_cast<uint32_t>(y) << 16) |
                                   (static_cast<uint32_t>(dyi) << 12) | static_cast<uint32_t>(a);
                auto &rounds = all[ci][w];
                bool placed = false;
                for (auto &r : rounds) {
                    if (r.rowmask[y / W] & mask) continue;
                    int ln = -1;
                    if (!r.lane[res]) ln = res;
                    else if (!r.lane[16 + res]) ln = 16 + res;
                    if (ln < 0) continue;
                    r.lane[ln] = d;
                    r.rowmask[y / W] |= mask;
                    placed = true;
                    break;
                }
                if (!placed) {
                    Round r{};
                    r.lane[res] = d;
                    r.rowmask[y / W] = mask;
                    rounds.push_back(r);
                }
            }
        }
        for (int w = 0; w < W; w++) rmax = std::max(rmax, static_cast<int>(all[ci][w].size()));
    }
    if (rmax == 0) rmax = 1;
    desc.assign(static_cast<size_t>(nc) * W * rmax * 32, 0u);
    first.assign(desc.size(), 0);
    nrounds.assign(static_cast<size_t>(nc) * W, 0);
    for (int ci = 0; ci < nc; ci++) {
        // first[.] bit dx: tap dx of that segment is the first write of its cell in round order
        // (each warp owns its rows, so per channel one pass over the warps' rounds decides it)
        std::vector<uint8_t> touched(M * M, 0);
        for (int w = 0; w < W; w++) {
            const auto &rounds = all[ci][w];
            nrounds[ci * W + w] = static_cast<int>(rounds.size());
            for (size_t r = 0; r < rounds.size(); r++)
                for (int l = 0; l < 32; l++) {
                    const uint32_t d = rounds[r].lane[l];
                    const size_t at = ((static_cast<size_t>(ci) * W + w) * rmax + r) * 32 + l;
                    desc[at] = d;
                    if (!(d >> 31)) continue;
                    const int y = static_cast<int>((d >> 16) & 0x3Fu), x0 = static_cast<int>((d >> 22) & 0x3Fu);
                    uint16_t m = 0;
                    for (int dx = 0; dx < K; dx++) {
                        uint8_t &tc = touched[y * M + ((x0 + dx) % M)];
                        if (!tc) m |= static_cast<uint16_t>(1u << dx);
                        tc = 1;
                    }
                    first[at] = m;
                }
        }
    }
    return EPIC_OK;
}

// Gather table of the FP32 register-transform kernel (fold side M = 64 or 48).
// A lane owns a pair of horizontally adjacent folded cells (x = 2 xp, 2 xp + 1)
// and sums, in registers, the (antenna, tap pair) entries whose footprints cover
// either cell: one voltage load serves both cells, and an antenna whose row
// segment covers only one of them brings a zero weight for the other.  Each
// pair is stored once per plane, so the gridding reads no grid cell and needs
// no cleared grid.  Pairs are sorted by list length and dealt in batches of 32
// lanes (one list step per warp iteration; a batch runs as long as its longest
// list).  Within each group of lanes that one shared-memory request serves (8
// for the 16-byte dual-polarisation voltage loads, 16 for the 8-byte
// single-polarisation ones) the list order is chosen greedily so that one step
// reads distinct banks (a greedy order, then a local search of swaps within a
// lane's list on the wavefronts).  Cells of touched rows that no listed pair writes get
// zeros, from per-warp lists of 32 cells per step; rows nobody touches are
// skipped by the transform and need nothing.  Batches go to the warps longest
// first, each to the warp with the least work so far, then the zero steps.
//   entry: a << 8 | tp, tp = dyi (K + 1) + dxl + 1, dxl in [-1, K - 1] the tap column of the left
//          cell (-1: only the right cell is covered; K - 1: only the left one)
//   channel block: [zero lists of warps 0..7][gather batches of warps 0..7]
//   gather batch:  [length d][32 left-cell offsets y (M + 1) + 2 xp, or ~0][d x 32 entries, or ~0]
//   idx[ci * 8 + w] = (zero list offset, zero steps, first batch offset, batches), offsets from the
//   channel block's start; chan[ci] = (block start, block words)
// Channels are built in parallel on up to `threads` host threads (0: up to 16, or the hardware's
// count); the table does not depend on the thread count.  A host allocation failure returns
// EPIC_ERR_NOMEM, a layout the format cannot hold EPIC_ERR_UNSUPPORTED.
int build_gather_table(const std::vector<short2> &cells, int A, int K, int M, int P, const std::vector<int> &chans,
                       std::vector<uint32_t> &tab, std::vector<int4> &idx, std::vector<int2> &chan,
                       std::vector<unsigned long long> &rowmask, int threads)
{
    constexpr int W = 8;
    const int h = (K - 1) / 2, S = M + 1, MP = M / 2;
    if (A > 4096 || K > 15 || (M != 64 && M != 48)) return EPIC_ERR_UNSUPPORTED;
    const int nc = static_cast<int>(chans.size());
    const int grp = P == 2 ? 8 : 16;    // lanes per request; bank slot = a mod grp
    tab.clear();
    idx.assign(static_cast<size_t>(nc) * W, make_int4(0, 0, 0, 0));
    chan.assign(nc, make_int2(0, 0));
    rowmask.assign(nc, 0ull);
    // channels are independent: each builds its own block (offsets relative to the block), in
    // parallel over host threads; the blocks are then laid end to end in channel order, so the
    // table does not depend on the thread count
    std::vector<std::vector<uint32_t>> blocks(nc);
    auto build_one = [&](int ci) -> bool {
        const int c = chans[ci];
        std::vector<std::vector<uint32_t>> list(M * MP);   // per pair: a << 8 | tp
        for (int a = 0; a < A; a++) {
            const short2 k = cells[static_cast<size_t>(c) * A + a];
            const int jx = k.x % M, jy = k.y % M;
            const int x0 = ((jx - h) % M + M) % M;
            for (int dyi = 0; dyi < K; dyi++) {
                const int y = ((jy + dyi - h) % M + M) % M;
                rowmask[ci] |= 1ull << y;
                int last = -1;
                for (int dx = 0; dx < K; dx++) {
                    const int x = (x0 + dx) % M, pr = x >> 1;
                    if (pr == last) continue;   // the right cell of a pair already listed
                    last = pr;
                    const int dxl = dx - (x & 1);
                    list[y * MP + pr].push_back((static_cast<uint32_t>(a) << 8) |
                                                static_cast<uint32_t>(dyi * (K + 1) + dxl + 1));
                }
            }
        }
        std::vector<int> touched, zero;
        for (int i = 0; i < M * MP; i++)
            if (!list[i].empty()) touched.push_back(i);
        for (int i = 0; i < M * M; i++) {
            const int y = i / M, x = i % M;
            if (((rowmask[ci] >> y) & 1ull) && list[y * MP + x / 2].empty()) zero.push_back(i);
        }
        std::stable_sort(touched.begin(), touched.end(),
                         [&](int u, int v) { return list[u].size() > list[v].size(); });
        auto cell_word = [&](int i) { return static_cast<uint32_t>((i / M) * S + i % M); };
        auto pair_word = [&](int i) { return static_cast<uint32_t>((i / MP) * S + 2 * (i % MP)); };
        std::vector<std::vector<uint32_t>> batches;
        for (size_t b0 = 0; b0 < touched.size(); b0 += 32) {
            const int nl = static_cast<int>(std::min<size_t>(32, touched.size() - b0));
            int d = 0;
            for (int l = 0; l < nl; l++) d = std::max(d, static_cast<int>(list[touched[b0 + l]].size()));
            std::vector<uint32_t> words(1 + 32 + static_cast<size_t>(d) * 32, ~0u);
            words[0] = static_cast<uint32_t>(d);
            for (int l = 0; l < nl; l++) words[1 + l] = pair_word(touched[b0 + l]);
            for (int g0 = 0; g0 < 32; g0 += grp) {
                std::vector<std::vector<uint32_t>> rem(grp);
                for (int l = 0; l < grp; l++)
                    if (g0 + l < nl) rem[l] = list[touched[b0 + g0 + l]];
                for (int j = 0; j < d; j++) {
                    std::vector<int> order(grp);
                    for (int l = 0; l < grp; l++) order[l] = l;
                    std::stable_sort(order.begin(), order.end(),
                                     [&](int u, int v) { return rem[u].size() > rem[v].size(); });
                    std::vector<int> slot(grp, -1);   // antenna already reading that bank slot this step
                    for (int l : order) {
                        auto &r = rem[l];
                        if (r.empty()) continue;
                        const bool must = static_cast<int>(r.size()) >= d - j;
                        int pick = -1;
                        for (size_t q = 0; q < r.size() && pick < 0; q++) {
                            const int a = static_cast<int>(r[q] >> 8), sl = a % grp;
                            if (slot[sl] < 0 || slot[sl] == a) pick = static_cast<int>(q);
                        }
                        if (pick < 0 && must) pick = 0;
                        if (pick < 0) continue;
                        const uint32_t e = r[pick];
                        r.erase(r.begin() + pick);
                        slot[static_cast<int>(e >> 8) % grp] = static_cast<int>(e >> 8);
                        words[1 + 32 + static_cast<size_t>(j) * 32 + g0 + l] = e;
                    }
                }
                // then a local search over each lane's order (two of its steps swapped, empty ones
                // included) while the group's voltage loads need fewer wavefronts: a step costs the
                // most distinct antennas any bank slot (a mod grp) receives
                auto at = [&](int j, int l) -> uint32_t & { return words[1 + 32 + static_cast<size_t>(j) * 32 + g0 + l]; };
                auto step_cost = [&](int j) {
                    int seen[16], ns = 0, cnt[16] = {}, mx = 0;
                    for (int l = 0; l < grp; l++) {
                        const uint32_t e = at(j, l);
                        if (e == ~0u) continue;
                        const int a = static_cast<int>(e >> 8);
                        bool dup = false;
                        for (int q = 0; q < ns; q++) dup = dup || seen[q] == a;
                        if (dup) continue;
                        seen[ns++] = a;
                        mx = std::max(mx, ++cnt[a % grp]);
                    }
                    return mx;
                };
                bool improved = d <= 24;   // (bounded: plan time grows as d^2 per pass)
                for (int pass = 0; pass < 4 && improved; pass++) {
                    improved = false;
                    for (int l = 0; l < grp; l++)
                        for (int j1 = 0; j1 < d; j1++)
                            for (int j2 = j1 + 1; j2 < d; j2++) {
                                uint32_t &x = at(j1, l), &y = at(j2, l);
                                if (x == y) continue;
                                const int before = step_cost(j1) + step_cost(j2);
                                std::swap(x, y);
                                if (step_cost(j1) + step_cost(j2) < before) improved = true;
                                else std::swap(x, y);
                            }
                }
            }
            batches.push_back(std::move(words));
        }
        // longest first, each to the least-loaded warp (cost ~ list steps; a store step ~ 1/4)
        std::vector<int> ord(batches.size());
        for (size_t i = 0; i < ord.size(); i++) ord[i] = static_cast<int>(i);
        std::stable_sort(ord.begin(), ord.end(), [&](int u, int v) { return batches[u][0] > batches[v][0]; });
        std::vector<std::vector<int>> per_warp(W);
        std::vector<long long> load(W, 0);
        for (int b : ord) {
            const int w = static_cast<int>(std::min_element(load.begin(), load.end()) - load.begin());
            per_warp[w].push_back(b);
            load[w] += 4 * static_cast<long long>(batches[b][0]) + 2;
        }
        std::vector<int> zsteps(W, 0);
        for (size_t z0 = 0; z0 < zero.size(); z0 += 32) {
            const int w = static_cast<int>(std::min_element(load.begin(), load.end()) - load.begin());
            zsteps[w]++;
            load[w] += 1;
        }
        std::vector<uint32_t> &blk = blocks[ci];
        size_t zi = 0;   // zero cells dealt in natural order: consecutive cells, distinct banks
        for (int w = 0; w < W; w++) {
            idx[static_cast<size_t>(ci) * W + w].x = static_cast<int>(blk.size());
            idx[static_cast<size_t>(ci) * W + w].y = zsteps[w];
            for (int st = 0; st < zsteps[w]; st++)
                for (int l = 0; l < 32; l++, zi++) blk.push_back(zi < zero.size() ? cell_word(zero[zi]) : ~0u);
        }
        for (int w = 0; w < W; w++) {
            idx[static_cast<size_t>(ci) * W + w].z = static_cast<int>(blk.size());
            idx[static_cast<size_t>(ci) * W + w].w = static_cast<int>(per_warp[w].size());
            for (int b : per_warp[w]) blk.insert(blk.end(), batches[b].begin(), batches[b].end());
            if (blk.size() > 0x7FFFFFFFull) return false;
        }
        return true;
    };
    std::atomic<int> next{0};
    std::atomic<bool> ok{true}, nomem{false};
    auto worker = [&]() {
        for (int ci; ok && (ci = next++) < nc;) {
            try {
                if (!build_one(ci)) ok = false;
            } catch (const std::bad_alloc &) {
                nomem = true;
                ok = false;
            } catch (...) {
                ok = false;
            }
        }
    };
    const int nt = threads > 0 ? std::min(nc, threads)
                               : std::max(1, std::min({nc, 16, static_cast<int>(std::thread::hardware_concurrency())}));
    std::vector<std::thread> pool;
    for (int i = 1; i < nt; i++) {
        try {
            pool.emplace_back(worker);
        } catch (...) {
            break;   // fewer threads: the calling thread takes the rest
        }
    }
    worker();
    for (auto &th : pool) th.join();
    if (!ok) return nomem ? EPIC_ERR_NOMEM : EPIC_ERR_UNSUPPORTED;
    for (int ci = 0; ci < nc; ci++) {
        const size_t start = tab.size();
        if (start + blocks[ci].size() > 0x7FFFFFFFull) return EPIC_ERR_UNSUPPORTED;
        chan[ci] = make_int2(static_cast<int>(start), static_cast<int>(blocks[ci].size()));
        tab.insert(tab.end(), blocks[ci].begin(), blocks[ci].end());
        std::vector<uint32_t>().swap(blocks[ci]);
    }
    if (tab.empty()) tab.push_back(0);
    return EPIC_OK;
}

void prof_begin(epic_plan_s *plan)
{
    if (plan->profiling) plan->n_recorded = 0;
}

void prof_mark(epic_plan_s *plan, cudaStream_t stream, int stage, bool start)
{
    if (!plan->profiling) return;
    while (static_cast<int>(plan->events.size()) < 2 * (stage + 1)) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            plan->profiling = false;
            return;
        }
        plan->events.push_back(e);
    }
    // External records become event-record nodes when the stream is being
    // captured (a plain record would only mark a dependency)
    cudaEventRecordWithFlags(plan->events[2 * stage + (start ? 0 : 1)], stream, cudaEventRecordExternal);
    if (!start && stage + 1 > plan->n_recorded) plan->n_recorded = stage + 1;
}

// One integration on `stream`: replay the plan's CUDA graph (captured on the
// first call and again whenever T, a pointer or the profiling state changes),
// or launch directly when graphs are disabled.
int run_image(epic_plan_s *p, const uint8_t *v, const float2 *gains, int T, float2 *out, cudaStream_t stream)
{
    if (!p->use_graph) return image_fp32(p, v, gains, T, out, stream, false);
    if (!p->gexec || p->g_v != v || p->g_gains != gains || p->g_delays != p->delays || p->g_out != out ||
        p->g_T != T || p->g_prof != p->profiling) {
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return EPIC_ERR_CUDA;
        const int rc = image_fp32(p, v, gains, T, out, p->cap, true);
        const cudaError_t ce = cudaStreamEndCapture(p->cap, &graph);
        if (rc != EPIC_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (ce != cudaSuccess || !graph) return EPIC_ERR_CUDA;
        bool updated = false;
        if (p->gexec) {
            cudaGraphExecUpdateResultInfo info;
            updated = cudaGraphExecUpdate(p->gexec, graph, &info) == cudaSuccess;
            if (!updated) {
                cudaGetLastError();
                cudaGraphExecDestroy(p->gexec);
                p->gexec = nullptr;
            }
        }
        if (!updated && cudaGraphInstantiate(&p->gexec, graph, 0) != cudaSuccess) {
            cudaGraphDestroy(graph);
            p->gexec = nullptr;
            return EPIC_ERR_CUDA;
        }
        cudaGraphDestroy(graph);
        p->g_v = v;
        p->g_gains = gains;
        p->g_delays = p->delays;
        p->g_out = out;
        p->g_T = T;
        p->g_prof = p->profiling;
    }
    return cudaGraphLaunch(p->gexec, stream) == cudaSuccess ? EPIC_OK : EPIC_ERR_CUDA;
}

}  // namespace epic

extern "C" {

const char *epic_strerror(int code)
{
    switch (code) {
    case EPIC_OK: return "ok";
    case EPIC_ERR_ARG: return "invalid argument";
    case EPIC_ERR_OUT_OF_GRID: return "antenna footprint outside the grid";
    case EPIC_ERR_UNSUPPORTED: return "unsupported configuration";
    case EPIC_ERR_CUDA: return "CUDA runtime error";
    case EPIC_ERR_TIMEOUT: return "device-side wait timed out";
    case EPIC_ERR_NOMEM: return "out of memory";
    case EPIC_ERR_DEVICE: return "device-side consistency check failed";
    case EPIC_ERR_TOO_LARGE: return "request exceeds the fixed scratch of epic_image_static";
    default: return "unknown error";
    }
}

int epic_plan(epic_plan_t *out, const double *ant_xy_m, int n_ant, int n_pol,
              const float *kernel_c64, int K, const int *grid_n, const double *freq_hz,
              int n_chan, double du, int max_spectra, int precision, unsigned flags)
{
    if (!out) return EPIC_ERR_ARG;
    *out = nullptr;
    if (!ant_xy_m || !kernel_c64 || !grid_n || !freq_hz) return EPIC_ERR_ARG;
    if (n_ant < 1 || (n_pol != 1 && n_pol != 2) || K < 1 || (K % 2) == 0 || K > epic::kMaxK ||
        n_chan < 1 || !(du > 0.0) || du > 0.5 || max_spectra < 0)
        return EPIC_ERR_ARG;
    constexpr unsigned kUser = EPIC_MEAN | EPIC_NO_AUTOSUB | EPIC_KERNEL_TAPER | EPIC_STOKES | EPIC_ANTENNA_KERNELS;
    constexpr unsigned kDiag = EPIC_DIAG_NO_GRAPH | EPIC_DIAG_GATHER_GLOBAL | EPIC_DIAG_NO_ALIAS |
                               EPIC_DIAG_WITHHOLD_MMA | EPIC_DIAG_ALIAS_BATCH(255) | EPIC_DIAG_NO_PAIR;
    if (flags & ~(kUser | kDiag)) return EPIC_ERR_ARG;
    const unsigned diag = flags & kDiag;
    flags &= kUser;
    if ((flags & EPIC_STOKES) && n_pol != 2) return EPIC_ERR_ARG;
    const bool ant_kernels = (flags & EPIC_ANTENNA_KERNELS) != 0;
    if (ant_kernels && (flags & EPIC_KERNEL_TAPER)) return EPIC_ERR_ARG;
    if (ant_kernels && precision != EPIC_FP32) return EPIC_ERR_UNSUPPORTED;
    if (precision < EPIC_FP32 || precision > EPIC_TC_SPLIT_BF16) return EPIC_ERR_ARG;
    const bool tensor = precision != EPIC_FP32;
    if (tensor) {
        // the tensor form runs on 64-point transforms: sides 64, 128, 256, 512 fold to them and
        // side 32 is transformed zero-padded; side 96 (48-point transforms in the same operands)
        // only on the dual-polarisation pair kernel, else it runs the FP32 kernel in the same
        // plan, and then at least one group must be of another side (checked again once the
        // groups are built)
        if ((n_ant * n_pol) % 4 != 0) return EPIC_ERR_UNSUPPORTED;
        bool any = n_pol == 2 && !ant_kernels;
        for (int c = 0; c < n_chan; c++) any = any || grid_n[c] != 96;
        if (!any) return EPIC_ERR_UNSUPPORTED;
    }
    if (static_cast<long long>(n_ant) * n_pol > epic::kMaxAP) return EPIC_ERR_UNSUPPORTED;
    for (int c = 0; c < n_chan; c++) {
        if (!(freq_hz[c] > 0.0) || !std::isfinite(freq_hz[c])) return EPIC_ERR_ARG;
        if (!supported_n(grid_n[c])) return EPIC_ERR_UNSUPPORTED;
    }
    for (int a = 0; a < n_ant; a++)
        if (!std::isfinite(ant_xy_m[2 * a]) || !std::isfinite(ant_xy_m[2 * a + 1])) return EPIC_ERR_ARG;

    // antenna -> cell map: per channel, per axis, llround((x - x_c) f / (c0 du)) + N/2
    double sx = 0, sy = 0;
    for (int a = 0; a < n_ant; a++) { sx += ant_xy_m[2 * a]; sy += ant_xy_m[2 * a + 1]; }
    const double cx = sx / n_ant, cy = sy / n_ant;
    const int h = (K - 1) / 2;
    std::vector<short2> cells(static_cast<size_t>(n_chan) * n_ant);
    for (int c = 0; c < n_chan; c++) {
        const int N = grid_n[c];
        for (int a = 0; a < n_ant; a++) {
            const double x = ant_xy_m[2 * a] - cx, y = ant_xy_m[2 * a + 1] - cy;
            const double fx = (x * freq_hz[c]) / (epic::kC0 * du);
            const double fy = (y * freq_hz[c]) / (epic::kC0 * du);
            if (std::fabs(fx) > 1e6 || std::fabs(fy) > 1e6) return EPIC_ERR_OUT_OF_GRID;
            const long long kx = std::llround(fx) + N / 2;
            const long long ky = std::llround(fy) + N / 2;
            if (kx - h < 0 || kx + h >= N || ky - h < 0 || ky + h >= N) return EPIC_ERR_OUT_OF_GRID;
            cells[static_cast<size_t>(c) * n_ant + a] = make_short2(static_cast<short>(kx), static_cast<short>(ky));
        }
    }

    auto *p = new (std::nothrow) epic_plan_s();
    if (!p) return EPIC_ERR_NOMEM;
    if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return EPIC_ERR_CUDA; }
    if (cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
        delete p;
        return EPIC_ERR_CUDA;
    }
    p->A = n_ant;
    p->P = n_pol;
    p->NP = n_pol == 2 ? 4 : 1;
    p->C = n_chan;
    // gridding kernel: the caller's W, or a single unit tap when W is applied
    // as an image-domain taper
    const bool taper = (flags & EPIC_KERNEL_TAPER) != 0;
    p->K = taper ? 1 : K;
    p->nker = ant_kernels ? n_ant : 1;
    const float unit_tap[2] = {1.f, 0.f};
    p->max_spectra = max_spectra;
    p->precision = precision;
    p->du = du;
    p->flags = flags;
    p->grid_n.assign(grid_n, grid_n + n_chan);
    p->out_off.resize(n_chan);
    long long off = 0;
    for (int c = 0; c < n_chan; c++) {
        p->out_off[c] = off;
        off += static_cast<long long>(p->NP) * grid_n[c] * grid_n[c];
    }
    p->out_floats = static_cast<size_t>(off) * 2;
    std::vector<long long> ef_off(n_chan);     // E-field images: channel offsets within one sample
    for (int c = 0; c < n_chan; c++) {
        ef_off[c] = p->ef_stride;
        p->ef_stride += static_cast<long long>(n_pol) * grid_n[c] * grid_n[c];
    }

    int smem_optin = 0;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device) != cudaSuccess) {
        delete p;
        return EPIC_ERR_CUDA;
    }
    int rc = dev_upload(&p->d_cells, cells.data(), cells.size());
    if (rc == EPIC_OK)
        rc = taper ? dev_upload(&p->d_kernel, reinterpret_cast<const float2 *>(unit_tap), 1)
                   : dev_upload(&p->d_kernel, reinterpret_cast<const float2 *>(kernel_c64),
                                static_cast<size_t>(p->nker) * K * K);
    if (rc == EPIC_OK && ant_kernels) {
        // B_aa(rho) = sum_d W_a(d) W_a^*(d - rho), rho in [-(K-1), K-1]^2, FP64
        const int R = 2 * K - 1, hh = (K - 1) / 2;
        std::vector<double2> bauto(static_cast<size_t>(n_ant) * R * R);
        for (int a = 0; a < n_ant; a++) {
            const float *Wa = kernel_c64 + static_cast<size_t>(a) * K * K * 2;
            for (int ry = -(K - 1); ry <= K - 1; ry++)
                for (int rx = -(K - 1); rx <= K - 1; rx++) {
                    std::complex<double> acc = 0;
                    for (int dy = -hh; dy <= hh; dy++)
                        for (int dx = -hh; dx <= hh; dx++) {
                            const int ey = dy - ry, ex = dx - rx;
                            if (ey < -hh || ey > hh || ex < -hh || ex > hh) continue;
                            const int i0 = (dy + hh) * K + (dx + hh), i1 = (ey + hh) * K + (ex + hh);
                            acc += std::complex<double>(Wa[2 * i0], Wa[2 * i0 + 1]) *
                                   std::conj(std::complex<double>(Wa[2 * i1], Wa[2 * i1 + 1]));
                        }
                    bauto[(static_cast<size_t>(a) * R + (ry + K - 1)) * R + (rx + K - 1)] =
                        make_double2(acc.real(), acc.imag());
                }
        }
        rc = dev_upload(&p->d_bauto, bauto.data(), bauto.size());
    }

    if (rc == EPIC_OK) rc = dev_upload(&p->d_status, static_cast<const int *>(nullptr), 1);
    if (rc == EPIC_OK) {
        // delay phases: FP64 turns at a mid-band reference once per (t, antenna),
        // the per-channel remainder (f_c - f_ref) tau in FP32 inside the kernels
        double fmin = freq_hz[0], fmax = freq_hz[0];
        for (int c = 1; c < n_chan; c++) {
            fmin = std::min(fmin, freq_hz[c]);
            fmax = std::max(fmax, freq_hz[c]);
        }
        p->f_ref = 0.5 * (fmin + fmax);
        std::vector<float> dfreq(n_chan);
        for (int c = 0; c < n_chan; c++) dfreq[c] = static_cast<float>(freq_hz[c] - p->f_ref);
        rc = dev_upload(&p->d_dfreq, dfreq.data(), dfreq.size());
        if (rc == EPIC_OK)
            rc = dev_upload(&p->d_dtab, static_cast<const float4 *>(nullptr),
                            static_cast<size_t>(max_spectra) * static_cast<size_t>(n_ant));
    }
    if (rc == EPIC_OK && cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) rc = EPIC_ERR_CUDA;

    // channel groups by grid side
    std::map<int, std::vector<int>> by_n;
    for (int c = 0; c < n_chan; c++) by_n[grid_n[c]].push_back(c);
    const int npf = n_pol == 2 ? 4 : 1;
    for (auto &kv : by_n) {
        if (rc != EPIC_OK) break;
        GroupCfg g;
        g.N = kv.first;
        g.Q1 = fold_for(g.N);
        g.M = g.N / g.Q1;
        if (tensor && g.N == 32) {
            // the tensor kernel's 64-point DFT of the zero-padded 32 x 32 grid: its even
            // frequencies 2 l are the 32-point transform at l (cells lie in [0, 32))
            g.M = 64;
            g.up = 2;
        }
        g.Q = g.Q1 * g.Q1;
        g.chans = kv.second;
        g.n_chan = static_cast<int>(g.chans.size());
        g.n_items = g.n_chan * g.Q;
        std::vector<long long> offs(g.n_chan);
        for (int i = 0; i < g.n_chan; i++) offs[i] = p->out_off[g.chans[i]];
        std::vector<double> wpow;
        kernel_power(kernel_c64, K, g.N, wpow);
        std::vector<float2> tw(g.N);
        for (int k = 0; k < g.N; k++) {
            const double ang = 2.0 * M_PI * k / g.N;
            tw[k] = make_float2(static_cast<float>(std::cos(ang)), static_cast<float>(std::sin(ang)));
        }
        g.tau_cap = epic::fp32_pick_tau(g.n_items, max_spectra, p->sm_count);
        if (g.tau_cap < 1) g.tau_cap = 1;
        g.R1 = 8;
        g.R2 = g.M / 8;
        const int ap = n_ant * n_pol;
        g.tensor = tensor && g.M == 64;
        // (the tensor kernel's fold path is written for dual polarisation)
        const bool fold_ok = g.Q1 == 8 && p->nker == 1 && p->K > 1 && !(diag & EPIC_DIAG_NO_ALIAS) &&
                             !(tensor && n_pol == 1);
        if (g.tensor) {
            // + static shared memory of the kernel (barriers, TMEM slot, alignment); a large side
            // that can take the fold path needs only the operands and the grid there
            g.tc_regular = epic::tc_dual_smem_bytes(n_ant, p->K) + 2048 <= static_cast<size_t>(smem_optin);
            if (!g.tc_regular && !(fold_ok && epic::tc_dual_fold_smem_bytes() + 2048 <= static_cast<size_t>(smem_optin)))
                rc = EPIC_ERR_UNSUPPORTED;
            g.reg64 = true;   // same gridding schedule and natural pixel order
            g.ts = 1;
        } else if ((g.M == 64 || g.M == 48) && (ap % 4) == 0) {
            for (int ts = 2; ts >= 1 && !g.reg64; ts--) {
                if (epic::reg64_smem_bytes(g.M, n_pol, ts, n_ant, p->K, p->nker) <= static_cast<size_t>(smem_optin)) {
                    g.reg64 = true;
                    g.ts = ts;
                }
            }
        }
        if (g.reg64) {
            g.R1 = 1;
            g.R2 = g.M;
            std::vector<uint32_t> desc;
            std::vector<int> nr;
            std::vector<unsigned long long> rows;
            std::vector<uint16_t> first;
            if (g.tensor) {
                // the tensor kernels grid by scheduled rounds into a cleared-once grid
                rc = epic::build_reg64_schedule(cells, n_ant, p->K, g.M, g.chans, desc, nr, g.rmax, rows, first);
                if (rc == EPIC_OK) rc = dev_upload(&g.d_sched, desc.data(), desc.size());
                if (rc == EPIC_OK) rc = dev_upload(&g.d_first, first.data(), first.size());
                if (rc == EPIC_OK) rc = dev_upload(&g.d_nrounds, nr.data(), nr.size());
            } else {
                std::vector<uint32_t> tab;
                std::vector<int4> gidx;
                std::vector<int2> gchan;
                rc = epic::build_gather_table(cells, n_ant, p->K, g.M, n_pol, g.chans, tab, gidx, gchan, rows);
                if (rc == EPIC_OK) rc = dev_upload(&g.d_gtab, tab.data(), tab.size());
                if (rc == EPIC_OK) rc = dev_upload(&g.d_gidx, gidx.data(), gidx.size());
                if (rc == EPIC_OK) rc = dev_upload(&g.d_gchan, gchan.data(), gchan.size());
                // a channel's whole table in shared memory when it fits beside the grids
                g.gwords = 0;
                for (const int2 &ch : gchan) g.gwords = std::max(g.gwords, ch.y);
                g.gstage = epic::reg64_smem_bytes(g.M, n_pol, g.ts, n_ant, p->K, p->nker) +
                               sizeof(uint32_t) * static_cast<size_t>(g.gwords) <=
                           static_cast<size_t>(smem_optin);
                if (diag & EPIC_DIAG_GATHER_GLOBAL) g.gstage = false;   // the unstaged form
            }
            if (rc == EPIC_OK) rc = dev_upload(&g.d_rowmask, rows.data(), rows.size());
            // large sides with one shared kernel of more than one tap: grid once per (channel,
            // sample) and fold all classes (alias_fold.cu), for the FP32 and the two-stage tensor
            // kernel.  With one tap (the taper) re-gridding per class is cheaper than moving the
            // folded grids through HBM (measured at N = 512: 0.24 s against 0.44 s per dense
            // integration).  EPIC_NO_ALIAS=1 keeps the per-class gridding.
            if (rc == EPIC_OK && fold_ok) {
                std::vector<short2> j0;
                std::vector<uint32_t> bseg;
                std::vector<int> boff;
                if (epic::build_alias_tables(cells, n_ant, p->K, g.N, g.chans, j0, bseg, boff) == EPIC_OK) {
                    const size_t per_sample = static_cast<size_t>(g.n_items) * n_pol * 64 * 64 * sizeof(float2);
                    constexpr size_t kBudget = size_t(4) << 30;   // folded grids of one time batch
                    g.alias_tb = static_cast<int>(std::max<size_t>(1, std::min<size_t>(max_spectra, kBudget / per_sample)));
                    // a diagnostic cap on the time batch (tests: several batches on a small case)
                    const int cap_tb = static_cast<int>((diag >> 16) & 255u);
                    if (cap_tb > 0) g.alias_tb = std::min(g.alias_tb, cap_tb);
                    rc = dev_upload(&g.d_j0, j0.data(), j0.size());
                    if (rc == EPIC_OK) rc = dev_upload(&g.d_bseg, bseg.data(), std::max<size_t>(1, bseg.size()));
                    if (rc == EPIC_OK) rc = dev_upload(&g.d_boff, boff.data(), boff.size());
                    if (rc == EPIC_OK)
                        rc = dev_upload(&g.d_gf, static_cast<const float2 *>(nullptr), per_sample / sizeof(float2) * g.alias_tb);
                    g.alias = rc == EPIC_OK;
                }
            }
            if (rc == EPIC_OK && g.tensor && !g.tc_regular && !g.alias) rc = EPIC_ERR_UNSUPPORTED;
            // grid sides 128 and 96 in a tensor plan: two pixel classes per CTA from one gridding when
            // the aperture's rows fold without overlap and the lists fit in shared memory (side 96:
            // 48-point DFTs in the 64-point operands; without the pair kernel it stays on the FP32
            // kernel); grid side 64: the same kernel with its one class
            const bool pair_side = (g.tensor && (g.N == 128 || g.N == 64)) || (tensor && g.N == 96 && g.reg64);
            if (rc == EPIC_OK && pair_side && n_pol == 2 && p->nker == 1 && !(diag & EPIC_DIAG_NO_PAIR)) {
                std::vector<uint32_t> tab32;
                std::vector<int4> idx32, pidx;
                std::vector<int2> chan32, pchan;
                std::vector<unsigned long long> rows32, upper;
                std::vector<uint16_t> ptab;
                if (epic::build_gather_table(cells, n_ant, p->K, g.M, 2, g.chans, tab32, idx32, chan32, rows32) ==
                        EPIC_OK &&
                    epic::build_pair_tables(cells, n_ant, p->K, g.chans, tab32, idx32, chan32, ptab, pidx, pchan,
                                            upper, epic::PairSchedule(), g.M) == EPIC_OK) {
                    int words = 0;
                    for (const int2 &ch : pchan) words = std::max(words, ch.y);
                    if (epic::tc_pair_smem_bytes(n_ant, p->K, words) + 2048 <= static_cast<size_t>(smem_optin)) {
                        g.pair = true;
                        g.pwords = words;
                        if (g.M == 48) {   // side 96 leaves the FP32 kernel for the pair kernel
                            g.tensor = true;
                            g.tc_regular = true;
                        }
                        g.h_tab32 = std::move(tab32);
                        g.h_idx32 = std::move(idx32);
                        g.h_chan32 = std::move(chan32);
                        if (p->h_cells.empty()) p->h_cells = cells;
                        g.ptab_n = ptab.size();
                        g.pidx_n = pidx.size();
                        rc = dev_upload(&g.d_ptab, ptab.data(), ptab.size());
                        if (rc == EPIC_OK) rc = dev_upload(&g.d_pidx, pidx.data(), pidx.size());
                        if (rc == EPIC_OK) rc = dev_upload(&g.d_pchan, pchan.data(), pchan.size());
                        if (rc == EPIC_OK) rc = dev_upload(&g.d_upper, upper.data(), upper.size());
                    }
                }
            }
        }
        g.launch_items = g.pair ? g.n_chan * (g.Q1 == 2 ? 2 : 1) : g.n_items;
        if (g.pair) g.tau_cap = std::max(g.tau_cap, epic::fp32_pick_tau(g.launch_items, max_spectra, p->sm_count));
        if (rc == EPIC_OK) rc = dev_upload(&g.d_chans, g.chans.data(), g.chans.size());
        if (rc == EPIC_OK) rc = dev_upload(&g.d_out_off, offs.data(), offs.size());
        if (rc == EPIC_OK) {
            std::vector<long long> eo(g.n_chan);
            for (int i = 0; i < g.n_chan; i++) eo[i] = ef_off[g.chans[i]];
            rc = dev_upload(&g.d_ef_off, eo.data(), eo.size());
        }
        if (rc == EPIC_OK) rc = dev_upload(&g.d_wpow, wpow.data(), wpow.size());
        if (rc == EPIC_OK) rc = dev_upload(&g.d_twN, tw.data(), tw.size());
        if (rc == EPIC_OK && ant_kernels) {
            std::vector<double2> tw64(g.N);
            for (int k = 0; k < g.N; k++) {
                const double ang = 2.0 * M_PI * k / g.N;
                tw64[k] = make_double2(std::cos(ang), std::sin(ang));
            }
            rc = dev_upload(&g.d_tw64, tw64.data(), tw64.size());
            if (rc == EPIC_OK)
                rc = dev_upload(&g.d_Y, static_cast<const double2 *>(nullptr),
                                static_cast<size_t>(g.n_chan) * 3 * (2 * K - 1) * g.N);
        }
        if (rc == EPIC_OK)
            rc = dev_upload(&g.d_partial, static_cast<const float *>(nullptr),
                            static_cast<size_t>(g.tau_cap) * g.n_items * g.M * g.M * npf);
        p->groups.push_back(g);
    }
    if (rc == EPIC_OK && tensor) {   // a tensor plan runs at least one group on the tensor cores
        bool any = false;
        for (const auto &g : p->groups) any = any || g.tensor;
        if (!any) rc = EPIC_ERR_UNSUPPORTED;
    }
    // exact auto sums: one set per image of a series batch (slot 0 for epic_image)
    p->series_cap = epic::kMaxTau;
    for (const auto &g : p->groups) p->series_cap = std::min(p->series_cap, g.tau_cap);
    p->series_cap = std::max(p->series_cap, 1);
    if (rc == EPIC_OK)
        rc = dev_upload(&p->d_autoint, static_cast<const int *>(nullptr),
                        static_cast<size_t>(p->series_cap) * n_chan * n_ant * 4);
    if (rc == EPIC_OK && tensor) {
        // both 64-point DFT stages on the tensor cores (tc_dual64.cu)
        std::vector<uint16_t> ops;
        epic::build_dft_operand(precision == EPIC_TC_SPLIT_BF16, ops);
        rc = dev_upload(&p->d_dft, reinterpret_cast<const uint8_t *>(ops.data()), ops.size() * 2);
        bool side48 = false;
        for (const auto &g : p->groups) side48 = side48 || (g.pair && g.M == 48);
        if (rc == EPIC_OK && side48) {
            epic::build_dft_operand(precision == EPIC_TC_SPLIT_BF16, ops, 48);
            rc = dev_upload(&p->d_dft48, reinterpret_cast<const uint8_t *>(ops.data()), ops.size() * 2);
        }
        // the dual kernel's dynamic shared memory: the largest any of its groups needs (a
        // large side on the fold path needs the operands and the grid only)
        size_t dual = 0;
        for (const auto &g : p->groups)
            if (g.tensor && !g.pair)
                dual = std::max(dual, g.tc_regular ? epic::tc_dual_smem_bytes(n_ant, p->K)
                                                   : epic::tc_dual_fold_smem_bytes());
        if (rc == EPIC_OK && dual) rc = epic::prepare_tc_dual(p, dual);
        size_t pair = 0;
        for (const auto &g : p->groups)
            if (g.pair) pair = std::max(pair, epic::tc_pair_smem_bytes(n_ant, p->K, g.pwords));
        if (rc == EPIC_OK && pair) rc = epic::prepare_tc_pair(p, pair);
    }
    for (const auto &g : p->groups) {
        if (rc != EPIC_OK) break;
        if (!g.tensor) rc = epic::prepare_fp32(p, g);
        if (rc == EPIC_OK && g.alias) rc = epic::prepare_alias(p);
    }
    if (rc == EPIC_OK) {
        p->use_graph = !(diag & EPIC_DIAG_NO_GRAPH);
        // Fault injection for the failure-detection test: the tensor kernel
        // issues no MMA, so its completion wait runs out after a short budget
        // and the plan's status word reports EPIC_ERR_TIMEOUT.
        if (diag & EPIC_DIAG_WITHHOLD_MMA) {
            p->test_withhold_mma = 1;
            p->wait_budget = 2000000;   // ~1 ms
        }
        if (cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->ev_auto, cudaEventDisableTiming) != cudaSuccess)
            rc = EPIC_ERR_CUDA;
        if (p->groups.size() > 1) {
            for (size_t i = 0; i < p->groups.size() && rc == EPIC_OK; i++) {
                cudaStream_t st;
                cudaEvent_t ev;
                if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
                    rc = EPIC_ERR_CUDA;
                    break;
                }
                p->side.push_back(st);
                if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
                    rc = EPIC_ERR_CUDA;
                    break;
                }
                p->ev_join.push_back(ev);
            }
        }
    }
    if (rc != EPIC_OK) {
        free_plan(p);
        return rc;
    }
    *out = p;
    return EPIC_OK;
}

size_t epic_out_floats(epic_plan_t plan) { return plan ? plan->out_floats : 0; }

int epic_image(epic_plan_t plan, const uint8_t *ci4, const float *gains, int n_spectra,
               float *out, void *stream)
{
    if (!plan || !out) return EPIC_ERR_ARG;
    if (n_spectra < 0 || n_spectra > plan->max_spectra) return EPIC_ERR_ARG;
    if (n_spectra > 0 && !ci4) return EPIC_ERR_ARG;
    auto s = static_cast<cudaStream_t>(stream);
    plan->delays = nullptr;
    return epic::run_image(plan, ci4, reinterpret_cast<const float2 *>(gains), n_spectra,
                           reinterpret_cast<float2 *>(out), s);
}

int epic_image_ex(epic_plan_t plan, const uint8_t *ci4, const float *gains, const double *delays_s, int n_spectra,
                  float *out, void *stream)
{
    if (!plan || !out) return EPIC_ERR_ARG;
    if (n_spectra < 0 || n_spectra > plan->max_spectra) return EPIC_ERR_ARG;
    if (n_spectra > 0 && !ci4) return EPIC_ERR_ARG;
    auto s = static_cast<cudaStream_t>(stream);
    plan->delays = delays_s;
    const int rc = epic::run_image(plan, ci4, reinterpret_cast<const float2 *>(gains), n_spectra,
                                   reinterpret_cast<float2 *>(out), s);
    plan->delays = nullptr;
    return rc;
}

// Autotuner: for each channel group, time the imaging and epilogue launches of
// an n_spectra integration (zero voltages, unit gains, scratch buffers) at a few
// time-chunk counts -- the cost model's choice, its neighbours, and the counts
// that fill whole waves of SMs -- and keep the fastest (min of three timed runs).
namespace {

// Deal a pair group's lists again with schedule ps and replace its device lists (same sizes:
// the batches do not depend on the dealing), after the work queued on s.
int repack_pair(epic_plan_s *plan, epic::GroupCfg &g, const epic::PairSchedule &ps, cudaStream_t s)
{
    std::vector<int4> pidx;
    std::vector<int2> pchan;
    std::vector<unsigned long long> upper;
    std::vector<uint16_t> ptab;
    int rc = epic::build_pair_tables(plan->h_cells, plan->A, plan->K, g.chans, g.h_tab32, g.h_idx32, g.h_chan32,
                                     ptab, pidx, pchan, upper, ps, g.M);
    if (rc != EPIC_OK) return rc;
    if (ptab.size() != g.ptab_n || pidx.size() != g.pidx_n) return EPIC_ERR_UNSUPPORTED;
    if (cudaStreamSynchronize(s) != cudaSuccess ||
        cudaMemcpy(g.d_ptab, ptab.data(), ptab.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g.d_pidx, pidx.data(), pidx.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess)
        return EPIC_ERR_CUDA;
    g.psched = ps;
    return EPIC_OK;
}

}  // namespace

int epic_autotune(epic_plan_t plan, int n_spectra, void *stream)
{
    if (!plan || n_spectra < 1 || n_spectra > plan->max_spectra) return EPIC_ERR_ARG;
    auto s = static_cast<cudaStream_t>(stream);
    const size_t vbytes = static_cast<size_t>(n_spectra) * plan->C * plan->A * plan->P;
    uint8_t *v = nullptr;
    float2 *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = EPIC_OK;
    if (cudaMalloc(&v, vbytes) != cudaSuccess || cudaMalloc(&out, plan->out_floats * sizeof(float)) != cudaSuccess)
        rc = EPIC_ERR_NOMEM;
    if (rc == EPIC_OK && (cudaMemsetAsync(v, 0, vbytes, s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
                          cudaEventCreate(&e1) != cudaSuccess))
        rc = EPIC_ERR_CUDA;
    const double *saved_delays = plan->delays;
    plan->delays = nullptr;
    const bool autosub = !(plan->flags & EPIC_NO_AUTOSUB);
    if (rc == EPIC_OK && autosub) rc = epic::launch_autopower(plan, v, n_spectra, s);
    for (auto &g : plan->groups) {
        if (rc != EPIC_OK) break;
        if (g.alias) continue;               // one time chunk, batched by the plan: nothing to tune
        const int cap = std::max(1, std::min(g.tau_cap, n_spectra));
        std::vector<int> cand;
        auto add = [&](int n) {
            if (n >= 1 && n <= cap && std::find(cand.begin(), cand.end(), n) == cand.end()) cand.push_back(n);
        };
        const int c0 = epic::fp32_pick_tau(g.launch_items, n_spectra, plan->sm_count);
        for (int d = -2; d <= 2; d++) add(c0 + d);
        for (int waves = 1; waves <= 4; waves++)
            add(static_cast<int>((static_cast<long long>(waves) * plan->sm_count) / std::max(1, g.launch_items)));
        float best = 1e30f;
        int best_n = c0;
        for (int n : cand) {
            g.tuned_tau = n;
            g.tuned_T = n_spectra;
            float t_min = 1e30f;
            for (int rep = 0; rep < 4 && rc == EPIC_OK; rep++) {
                int nt = 0;
                if (cudaEventRecord(e0, s) != cudaSuccess) rc = EPIC_ERR_CUDA;
                if (rc == EPIC_OK) rc = epic::launch_imaging(plan, g, v, nullptr, n_spectra, &nt, s);
                if (rc == EPIC_OK) rc = epic::launch_epilogue(plan, g, nullptr, n_spectra, nt, out, s);
                if (rc == EPIC_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
                    rc = EPIC_ERR_CUDA;
                float ms = 0;
                if (rc == EPIC_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = EPIC_ERR_CUDA;
                if (rc == EPIC_OK && rep > 0) t_min = std::min(t_min, ms);   // the first run warms up
            }
            if (rc != EPIC_OK) break;
            if (t_min < best) {
                best = t_min;
                best_n = n;
            }
        }
        g.tuned_tau = best_n;
        g.tuned_T = n_spectra;
        // pair kernel: how its lists are dealt to the warps, measured at the chosen time chunks
        if (g.pair && rc == EPIC_OK) {
            const epic::PairSchedule cands[] = {{90, 80}, {60, 80}, {120, 80}, {90, 67}, {60, 90}, {150, 67}};
            epic::PairSchedule best_s = g.psched;
            float best_t = best;
            for (const epic::PairSchedule &ps : cands) {
                if (rc != EPIC_OK) break;
                if (ps.tmem_load == g.psched.tmem_load && ps.first_pct == g.psched.first_pct) continue;
                rc = repack_pair(plan, g, ps, s);
                float t_min = 1e30f;
                for (int rep = 0; rep < 4 && rc == EPIC_OK; rep++) {
                    int nt = 0;
                    if (cudaEventRecord(e0, s) != cudaSuccess) rc = EPIC_ERR_CUDA;
                    if (rc == EPIC_OK) rc = epic::launch_imaging(plan, g, v, nullptr, n_spectra, &nt, s);
                    if (rc == EPIC_OK) rc = epic::launch_epilogue(plan, g, nullptr, n_spectra, nt, out, s);
                    if (rc == EPIC_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
                        rc = EPIC_ERR_CUDA;
                    float ms = 0;
                    if (rc == EPIC_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = EPIC_ERR_CUDA;
                    if (rc == EPIC_OK && rep > 0) t_min = std::min(t_min, ms);
                }
                if (rc == EPIC_OK && t_min < best_t) {
                    best_t = t_min;
                    best_s = ps;
                }
            }
            if (rc == EPIC_OK) rc = repack_pair(plan, g, best_s, s);
        }
    }
    plan->delays = saved_delays;
    plan->g_T = -1;                      // the next epic_image re-captures its graph
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(v);
    cudaFree(out);
    if (rc == EPIC_OK && cudaGetLastError() != cudaSuccess) rc = EPIC_ERR_CUDA;
    return rc;
}

int epic_image_series_ex(epic_plan_t plan, const uint8_t *ci4, const float *gains, const double *delays_s,
                         int n_spectra, int spi, float *out, void *stream)
{
    if (!plan || !out || spi < 1) return EPIC_ERR_ARG;
    if (n_spectra < 0 || n_spectra > plan->max_spectra || n_spectra % spi != 0) return EPIC_ERR_ARG;
    if (n_spectra > 0 && !ci4) return EPIC_ERR_ARG;
    if (plan->nker > 1) return EPIC_ERR_UNSUPPORTED;
    auto s = static_cast<cudaStream_t>(stream);
    const int n_img = n_spectra / spi;
    const size_t img_floats = plan->out_floats;
    const size_t row_bytes = static_cast<size_t>(plan->C) * plan->A * plan->P;
    auto *out2 = reinterpret_cast<float2 *>(out);
    const auto *g2 = reinterpret_cast<const float2 *>(gains);
    int rc = EPIC_OK;
    for (int i0 = 0; i0 < n_img && rc == EPIC_OK; i0 += plan->series_cap) {
        const int b = std::min(plan->series_cap, n_img - i0);
        const uint8_t *vb = ci4 + static_cast<size_t>(i0) * spi * row_bytes;
        float2 *ob = out2 + static_cast<size_t>(i0) * (img_floats / 2);
        if (!(plan->flags & EPIC_NO_AUTOSUB)) rc = epic::launch_autopower_series(plan, vb, spi, b, s);
        // the batch's delays, time-indexed from the batch's first spectrum like its voltages
        plan->delays = delays_s ? delays_s + static_cast<size_t>(i0) * spi * plan->A : nullptr;
        if (rc == EPIC_OK && plan->delays) rc = epic::launch_delay_prep(plan, spi * b, s);
        plan->force_tau = b;   // one time chunk per image
        for (const auto &g : plan->groups) {
            if (rc != EPIC_OK) break;
            int n_tau = 0;
            rc = epic::launch_imaging(plan, g, vb, g2, spi * b, &n_tau, s);
            if (rc == EPIC_OK) rc = epic::launch_epilogue_series(plan, g, g2, spi, b, ob, s);
        }
        plan->force_tau = 0;
        plan->delays = nullptr;
    }
    return rc;
}

size_t epic_efield_floats(epic_plan_t plan) { return plan ? static_cast<size_t>(plan->ef_stride) * 2 : 0; }

int epic_image_efield(epic_plan_t plan, const uint8_t *ci4, const float *gains, int n_spectra, float *out, void *stream)
{
    if (!plan || !out) return EPIC_ERR_ARG;
    if (n_spectra < 0 || n_spectra > plan->max_spectra) return EPIC_ERR_ARG;
    if (n_spectra > 0 && !ci4) return EPIC_ERR_ARG;
    if (plan->precision != EPIC_FP32) return EPIC_ERR_UNSUPPORTED;
    for (const auto &g : plan->groups)
        if (!g.reg64 || g.tensor) return EPIC_ERR_UNSUPPORTED;
    if (n_spectra == 0) return EPIC_OK;
    auto s = static_cast<cudaStream_t>(stream);
    auto *o = reinterpret_cast<float2 *>(out);
    const auto *g2 = reinterpret_cast<const float2 *>(gains);
    plan->delays = nullptr;
    for (const auto &g : plan->groups) {
        const int rc = epic::launch_reg64_efield(plan, g, ci4, g2, n_spectra, o, plan->ef_stride, s);
        if (rc != EPIC_OK) return rc;
    }
    return EPIC_OK;
}

int epic_image_series(epic_plan_t plan, const uint8_t *ci4, const float *gains, int n_spectra, int spi, float *out,
                      void *stream)
{
    return epic_image_series_ex(plan, ci4, gains, nullptr, n_spectra, spi, out, stream);
}

namespace {

// the device staging of the host-buffer entry points (the imaging graph's fixed pointers)
int ensure_stage(epic_plan_s *plan)
{
    if (plan->d_stage_out) return EPIC_OK;
    const size_t vbytes = static_cast<size_t>(plan->max_spectra) * plan->C * plan->A * plan->P;
    const size_t gfloats = static_cast<size_t>(plan->C) * plan->A * plan->P * 2;
    if (cudaMalloc(&plan->d_stage_v, vbytes ? vbytes : 16) != cudaSuccess ||
        cudaMalloc(&plan->d_stage_g, gfloats * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&plan->d_stage_out, plan->out_floats * sizeof(float)) != cudaSuccess) {
        cudaFree(plan->d_stage_v);
        cudaFree(plan->d_stage_g);
        cudaFree(plan->d_stage_out);
        plan->d_stage_v = nullptr;
        plan->d_stage_g = nullptr;
        plan->d_stage_out = nullptr;
        return EPIC_ERR_NOMEM;
    }
    return EPIC_OK;
}

// the two upload / download slots, streams and events of epic_image_host_async
int ensure_ring(epic_plan_s *plan)
{
    if (plan->s_down) return EPIC_OK;
    const size_t vbytes = static_cast<size_t>(plan->max_spectra) * plan->C * plan->A * plan->P;
    const size_t gfloats = static_cast<size_t>(plan->C) * plan->A * plan->P * 2;
    bool ok = true;
    for (int i = 0; i < 2 && ok; i++) {
        ok = cudaMalloc(&plan->d_ring_v[i], vbytes ? vbytes : 16) == cudaSuccess &&
             cudaMalloc(&plan->d_ring_g[i], gfloats * sizeof(float)) == cudaSuccess &&
             cudaMalloc(&plan->d_ring_out[i], plan->out_floats * sizeof(float)) == cudaSuccess;
        for (cudaEvent_t *e : {&plan->ev_up[i], &plan->ev_in_free[i], &plan->ev_img[i], &plan->ev_out_free[i]})
            ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    }
    ok = ok && cudaStreamCreateWithFlags(&plan->s_up, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&plan->s_down, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) return EPIC_OK;
    for (int i = 0; i < 2; i++) {
        cudaFree(plan->d_ring_v[i]);
        cudaFree(plan->d_ring_g[i]);
        cudaFree(plan->d_ring_out[i]);
        plan->d_ring_v[i] = nullptr;
        plan->d_ring_g[i] = nullptr;
        plan->d_ring_out[i] = nullptr;
        for (cudaEvent_t *e : {&plan->ev_up[i], &plan->ev_in_free[i], &plan->ev_img[i], &plan->ev_out_free[i]})
            if (*e) {
                cudaEventDestroy(*e);
                *e = nullptr;
            }
    }
    if (plan->s_up) cudaStreamDestroy(plan->s_up);
    plan->s_up = nullptr;
    if (plan->s_down) cudaStreamDestroy(plan->s_down);
    plan->s_down = nullptr;
    return EPIC_ERR_NOMEM;
}

}  // namespace

int epic_image_host(epic_plan_t plan, const uint8_t *ci4, const float *gains, int n_spectra,
                    float *out, void *stream)
{
    if (!plan || !out) return EPIC_ERR_ARG;
    if (n_spectra < 0 || n_spectra > plan->max_spectra) return EPIC_ERR_ARG;
    if (n_spectra > 0 && !ci4) return EPIC_ERR_ARG;
    auto s = static_cast<cudaStream_t>(stream);
    const size_t gfloats = static_cast<size_t>(plan->C) * plan->A * plan->P * 2;
    if (const int rc = ensure_stage(plan); rc != EPIC_OK) return rc;
    const size_t nbytes = static_cast<size_t>(n_spectra) * plan->C * plan->A * plan->P;
    if (nbytes && cudaMemcpyAsync(plan->d_stage_v, ci4, nbytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return EPIC_ERR_CUDA;
    if (gains && cudaMemcpyAsync(plan->d_stage_g, gains, gfloats * sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return EPIC_ERR_CUDA;
    int rc = epic::run_image(plan, plan->d_stage_v, gains ? reinterpret_cast<const float2 *>(plan->d_stage_g) : nullptr,
                             n_spectra, reinterpret_cast<float2 *>(plan->d_stage_out), s);
    if (rc != EPIC_OK) return rc;
    if (cudaMemcpyAsync(out, plan->d_stage_out, plan->out_floats * sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return EPIC_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return EPIC_ERR_CUDA;
    return EPIC_OK;
}

int epic_image_host_async(epic_plan_t plan, const uint8_t *ci4, const float *gains, int n_spectra, float *out,
                          void *stream)
{
    if (!plan || !out) return EPIC_ERR_ARG;
    if (n_spectra < 0 || n_spectra > plan->max_spectra) return EPIC_ERR_ARG;
    if (n_spectra > 0 && !ci4) return EPIC_ERR_ARG;
    if (const int rc = ensure_stage(plan); rc != EPIC_OK) return rc;
    if (const int rc = ensure_ring(plan); rc != EPIC_OK) return rc;
    auto s = static_cast<cudaStream_t>(stream);
    const int k = static_cast<int>(plan->n_async++ & 1);
    const size_t nbytes = static_cast<size_t>(n_spectra) * plan->C * plan->A * plan->P;
    const size_t gbytes = static_cast<size_t>(plan->C) * plan->A * plan->P * 2 * sizeof(float);
    const size_t obytes = plan->out_floats * sizeof(float);
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    // upload into slot k once the imaging two calls back has taken its inputs out of it
    if (!ok(cudaStreamWaitEvent(plan->s_up, plan->ev_in_free[k], 0)) ||
        (nbytes && !ok(cudaMemcpyAsync(plan->d_ring_v[k], ci4, nbytes, cudaMemcpyHostToDevice, plan->s_up))) ||
        (gains && !ok(cudaMemcpyAsync(plan->d_ring_g[k], gains, gbytes, cudaMemcpyHostToDevice, plan->s_up))) ||
        !ok(cudaEventRecord(plan->ev_up[k], plan->s_up)))
        return EPIC_ERR_CUDA;
    // on the caller's stream: inputs into the imaging graph's fixed buffers, image, result into
    // slot k once the download two calls back has emptied it
    if (!ok(cudaStreamWaitEvent(s, plan->ev_up[k], 0)) ||
        (nbytes && !ok(cudaMemcpyAsync(plan->d_stage_v, plan->d_ring_v[k], nbytes, cudaMemcpyDeviceToDevice, s))) ||
        (gains && !ok(cudaMemcpyAsync(plan->d_stage_g, plan->d_ring_g[k], gbytes, cudaMemcpyDeviceToDevice, s))) ||
        !ok(cudaEventRecord(plan->ev_in_free[k], s)))
        return EPIC_ERR_CUDA;
    int rc = epic::run_image(plan, plan->d_stage_v, gains ? reinterpret_cast<const float2 *>(plan->d_stage_g) : nullptr,
                             n_spectra, reinterpret_cast<float2 *>(plan->d_stage_out), s);
    if (rc != EPIC_OK) return rc;
    if (!ok(cudaStreamWaitEvent(s, plan->ev_out_free[k], 0)) ||
        !ok(cudaMemcpyAsync(plan->d_ring_out[k], plan->d_stage_out, obytes, cudaMemcpyDeviceToDevice, s)) ||
        !ok(cudaEventRecord(plan->ev_img[k], s)))
        return EPIC_ERR_CUDA;
    // download slot k into the caller's host buffer
    if (!ok(cudaStreamWaitEvent(plan->s_down, plan->ev_img[k], 0)) ||
        !ok(cudaMemcpyAsync(out, plan->d_ring_out[k], obytes, cudaMemcpyDeviceToHost, plan->s_down)) ||
        !ok(cudaEventRecord(plan->ev_out_free[k], plan->s_down)))
        return EPIC_ERR_CUDA;
    return EPIC_OK;
}

int epic_host_wait(epic_plan_t plan)
{
    if (!plan) return EPIC_ERR_ARG;
    if (!plan->s_down) return EPIC_OK;
    if (cudaStreamSynchronize(plan->s_up) != cudaSuccess || cudaStreamSynchronize(plan->s_down) != cudaSuccess)
        return EPIC_ERR_CUDA;
    return EPIC_OK;
}

int epic_status(epic_plan_t plan)
{
    if (!plan) return EPIC_ERR_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return EPIC_ERR_CUDA;
    int st = 0;
    if (cudaMemcpy(&st, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return EPIC_ERR_CUDA;
    if (cudaMemset(plan->d_status, 0, sizeof(int)) != cudaSuccess) return EPIC_ERR_CUDA;
    if (st & epic::kStatusTimeout) return EPIC_ERR_TIMEOUT;
    if (st & epic::kStatusDevice) return EPIC_ERR_DEVICE;
    return EPIC_OK;
}

int epic_set_profiling(epic_plan_t plan, int enable)
{
    if (!plan) return EPIC_ERR_ARG;
    plan->profiling = enable != 0;
    plan->n_recorded = 0;
    return EPIC_OK;
}

int epic_stage_times(epic_plan_t plan, float *ms, int max_stages)
{
    if (!plan || !ms || max_stages < 0) return EPIC_ERR_ARG;
    if (!plan->profiling || plan->n_recorded == 0) return EPIC_ERR_ARG;
    const int n = plan->n_recorded < max_stages ? plan->n_recorded : max_stages;
    for (int i = 0; i < plan->n_recorded; i++)
        if (cudaEventSynchronize(plan->events[2 * i + 1]) != cudaSuccess) return EPIC_ERR_CUDA;
    for (int i = 0; i < n; i++)
        if (cudaEventElapsedTime(&ms[i], plan->events[2 * i], plan->events[2 * i + 1]) != cudaSuccess)
            return EPIC_ERR_CUDA;
    return n;
}

void epic_destroy(epic_plan_t plan)
{
    if (!plan) return;
    cudaDeviceSynchronize();
    free_plan(plan);
}

}  // extern "C"
