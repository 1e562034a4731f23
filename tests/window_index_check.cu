// Host-side check of the windowed stage kernel's index arithmetic
// (k_mixed_fused in hsgn_fused.cuh): every tile geometry the library launches,
// single grids (tile rows for several co-resident CTA counts) and batch
// instances (one CTA slot) on both the large (256 threads) and the small (128
// threads) windowed kernel, both boundary conditions. It evaluates the same
// __host__ __device__ helpers the kernel calls and checks that every global
// cell index lies in [0, n), every shared-memory index within the arrays, that
// tiles cover the grid once, that the rows kept from a window lie HW - 1 rows
// or more inside it, and that the two tiles beside a face build the same
// mini-window, and that the four cells per thread of the cell, row and solve
// phases cover the window within the arrays. The same for the double-float
// stage (k_df_stage in hsgn_dfstage.cuh, 96-row overlap): in addition, the
// faces its flux phase writes (four per thread, plus face 4T from the last
// thread when the window is full) cover every face its cell phase reads.
// Exit status 0 when every check passes.
#include <cstdio>
#include <cstdlib>
#include "../paper_2510_07539_gb300/csrc/hsgn_dfstage.cuh"

using namespace hsgn;
constexpr int M = 4;

#define CHECK(c)                                                                               \
    do {                                                                                       \
        if (!(c)) {                                                                            \
            printf("FAIL %s n=%lld S=%d p=%lld bc=%d line %d\n", #c, (long long)n, S,          \
                   (long long)p, BC, __LINE__);                                                \
            exit(1);                                                                           \
        }                                                                                      \
    } while (0)

static long long checked_windows = 0;

template <int T, int BC, int HW = 64>
void check(int64_t n, int S) {
    using G = FusedGeom<T, M, HW>;
    int64_t p = -1;
    CHECK(S >= 1 && S <= G::S);
    // cell, row and solve phases: thread t reads the cell arrays at 4t .. 4t + 7
    // as two float4 (arrays 16-byte aligned), dh at 4t + 8, and writes the
    // padded rows pd(4t + k)
    CHECK(G::NC % 4 == 0 && 4 * T + 5 <= G::NC && pd(4 * T - 1) < G::NC);
    const int64_t P = (n + S - 1) / S;
    int64_t covered = 0;
    for (p = 0; p < P; ++p) {
        ++checked_windows;
        const Window w = window_of<BC>(p, n, S, HW);
        CHECK(w.sp >= 1 && w.sp <= S);
        CHECK(w.t0 == covered);
        covered += w.sp;
        CHECK(w.W >= 1 && w.W + 1 <= T * M);  // rows of the block solve, closing row included
        CHECK(w.W + 2 <= 4 * T);  // the cells c = -1 .. W, four per thread
        CHECK(w.lo >= 0 && w.lo + w.sp <= w.W);
        // load phase: j < W + 6, both cells in range on either path
        CHECK(w.W + 6 <= G::NC);
        const bool inner = inner_window(w.wl, w.W, n);
        for (int j = 0; j < w.W + 6; ++j) {
            int64_t gi, gn, ci, cn;
            load_cells<BC>(inner, w.wl, j, n, gi, gn);
            load_cells<BC>(false, w.wl, j, n, ci, cn);
            CHECK(gi >= 0 && gi < n && gn >= 0 && gn < n);
            CHECK(gi == ci && gn == cn);  // the direct path reads the cells the general one does
            if (BC == BC_PERIODIC) CHECK(((w.wl - 3 + j) % n + n) % n == gi);
            if (inner) {
                // the direct path: cells b + j - 1 (j in [2, W + 3]) .. b + j + 1 and
                // faces b + j .. b + j + 2 from b = wl - 3; the face left of cell
                // b + j is read at b + j, so cell 0 (periodic face n - 1/2) is excluded
                const int64_t b = w.wl - 3;
                CHECK(b + j >= 1 && b + j + 1 < n);
                if (j >= 2 && j <= w.W + 3) CHECK(b + j - 1 >= 0 && cell_at<BC>(w.wl - 4 + j, n) == b + j - 1);
                CHECK(b + j + 2 <= n);  // G1 has n + 1 faces
            }
        }
        // padded stores: face couplings pd(j), j <= W; dh at pd(r + 1), r <= W
        CHECK(pd(w.W + 1) < G::NC);
        // back-substitution reads rows r - 1 .. r + 1 of the tile rows r
        if (!(BC == BC_TRANSMISSIVE && w.lend)) CHECK(w.lo >= HW);
        if (!(BC == BC_TRANSMISSIVE && w.rend)) CHECK(w.W - (w.lo + w.sp) >= HW);
        CHECK(pd(w.lo + w.sp + 1) < G::NC && w.lo + w.sp + 3 < G::NC);
        // dh of window row r at r + 4 (r = -1 .. W; thread t stores rows 4t .. 4t + 3)
        CHECK(w.W + 4 < G::NC);
        // next-wave L2 prefetch of this tile's window (clamped to [0, n)): the
        // first (R + 21) / 16 threads, one line of 16 pairs each, cover it
        {
            const int64_t c0 = w.wl - 3 < 0 ? 0 : w.wl - 3;
            const int64_t c1 = w.wl + w.W + 3 > n ? n : w.wl + w.W + 3;
            CHECK(c0 >= 0 && c1 <= n && c0 < c1);
            CHECK(c1 - c0 <= 16 * ((G::R + 6 + 15) / 16));
        }
        CHECK(w.t0 + w.sp <= n);
        // mini-windows of the tile faces
        const bool lface = !(BC == BC_TRANSMISSIVE && w.t0 == 0);
        const bool rface = !(BC == BC_TRANSMISSIVE && w.t0 + w.sp == n);
        for (int side = 0; side < 2; ++side) {
            if (!(side == 0 ? lface : rface)) continue;
            const int64_t tf = side == 0 ? w.t0 : w.t0 + w.sp;
            const MiniWindow m = mini_of<BC>(tf, n, G::HB);
            const int ms = (int)(m.ml - w.wl);
            CHECK(ms >= 0 && ms + m.mw <= w.W);
            CHECK(m.mw + 1 <= 32 * G::MB);
            const int kr = (int)(tf - m.ml);
            CHECK(kr - 1 >= 0 && kr < m.mw);
            if (BC == BC_TRANSMISSIVE) {
                if (m.lend) CHECK(m.ml == 0);
                if (m.rend) CHECK(m.ml + m.mw == n);
            }
            // the tile on the other side of the face builds the same mini-window
            const int64_t q = side == 0 ? (p == 0 ? P - 1 : p - 1) : (p + 1 == P ? 0 : p + 1);
            const Window wq = window_of<BC>(q, n, S, HW);
            const int64_t tq = side == 0 ? wq.t0 + wq.sp : wq.t0;
            if (BC == BC_PERIODIC)
                CHECK(((tq - tf) % n + n) % n == 0);
            else
                CHECK(tq == tf);
            const MiniWindow mq = mini_of<BC>(tq, n, G::HB);
            CHECK(mq.mw == m.mw && mq.lend == m.lend && mq.rend == m.rend);
            if (BC == BC_PERIODIC) CHECK(((mq.ml - m.ml) % n + n) % n == 0);
            const int msq = (int)(mq.ml - wq.wl);
            CHECK(msq >= 0 && msq + mq.mw <= wq.W);
        }
    }
    CHECK(covered == n);
}

// The double-float stage: T = 256 threads, four rows each, overlap DHW.
constexpr int DT = 256, DHW = 96, DHW_MIN = 48;

// One window of the double-float stage (tile rows [w.t0, w.t0 + w.sp)).
template <int BC>
void check_df_window(const Window& w, int64_t n) {
    using G = DfGeom<DT, M, DHW>;
    const int S = w.sp;          // (reported by CHECK)
    const int64_t p = w.t0;
    ++checked_windows;
    CHECK(w.sp >= 1);
    CHECK(w.W >= 1 && w.W <= G::R && w.W + 1 <= DT * M);
    CHECK(w.lo >= 0 && w.lo + w.sp <= w.W);
    CHECK(w.W + 6 <= G::NC);  // loaded cells -3 .. W + 2
    const bool inner = inner_window(w.wl, w.W, n);
    for (int j = 0; j < w.W + 6; ++j) {
        const int64_t gi = inner ? w.wl - 3 + j : cell_at<BC>(w.wl - 3 + j, n);
        CHECK(gi >= 0 && gi < n);
        CHECK(gi == cell_at<BC>(w.wl - 3 + j, n));
    }
    // flux phase: thread t writes faces 4t .. 4t + 3; the last thread also
    // face 4T when W + 3 > 4T. The cell phase reads faces 0 .. W + 2 (cells
    // c = -1 .. W, faces j and j + 1 of cell j - 1); a face f is built from
    // the loaded cells at index f .. f + 3
    const int top = (w.W + 3 > 4 * DT) ? 4 * DT : 4 * DT - 1;  // highest face written
    CHECK(w.W + 2 <= top);
    CHECK(top + 3 < G::NC);
    for (int f = 0; f <= w.W + 2; ++f) CHECK(f + 3 < w.W + 6);
    // cell phase: cell j (j < W + 2) reads state index j + 2 (loaded) and
    // writes per-cell index j; row phase: row i < W reads per-cell indices
    // i .. i + 2 and state indices i + 2 .. i + 4; back-substitution: tile row
    // r reads dh at r + 3 .. r + 5 (rows -1 .. W, index 3 a ghost only at a
    // transmissive left end, where lo = 0)
    CHECK(w.W + 1 + 2 < w.W + 6);
    CHECK(w.W - 1 + 4 < w.W + 6);
    CHECK(w.lo + w.sp - 1 + 5 <= w.W + 4 && w.W + 4 < G::NC);
    CHECK(w.lo >= 1 || (BC == BC_TRANSMISSIVE && w.lend));
}

// The wide tiling (tiles of S rows, overlap DHW) and a narrower one (tiles of
// Sn rows, overlap hwn: 48 .. 88 in steps of 8) of an n-cell grid: the windows
// of every tile, and of the pieces (wide overlap) that a narrower tile is redone
// in when its window misses the decay bound; both tilings cover the grid once.
template <int BC>
void check_df(int64_t n, int S, int Sn = 0, int hwn = 0) {
    using G = DfGeom<DT, M, DHW>;
    int64_t p = -1;
    CHECK(G::NC % 4 == 0 && 4 * DT + 4 <= G::NC);  // get4 at 4t + 4 reads up to 4T + 3
    CHECK(S >= 1 && S <= G::S);
    const int64_t P = (n + S - 1) / S;
    int64_t covered = 0;
    for (p = 0; p < P; ++p) {
        const Window w = window_of<BC>(p, n, S, DHW);
        const Window wa = window_at<BC>(p * (int64_t)S, w.sp, n, DHW);
        CHECK(w.t0 == wa.t0 && w.wl == wa.wl && w.W == wa.W && w.lo == wa.lo && w.sp == wa.sp);
        CHECK(w.sp >= 1 && w.sp <= S && w.t0 == covered);
        covered += w.sp;
        check_df_window<BC>(w, n);
    }
    CHECK(covered == n);
    if (Sn == 0) return;
    CHECK(hwn >= DHW_MIN && hwn < DHW && hwn % 8 == 0);
    CHECK(Sn >= S && Sn <= G::R - 2 * hwn);
    const int64_t Pn = (n + Sn - 1) / Sn;
    covered = 0;
    for (p = 0; p < Pn; ++p) {
        const int64_t t0 = p * (int64_t)Sn;
        const int sp = (int)(n - t0 < Sn ? n - t0 : Sn);
        CHECK(sp >= 1 && t0 == covered);
        covered += sp;
        check_df_window<BC>(window_at<BC>(t0, sp, n, hwn), n);
        const int np = (sp + G::S - 1) / G::S;
        const int pr = (sp + np - 1) / np;
        int64_t pc = t0;
        for (int k = 0; k < np; ++k) {
            const int psp = pr < sp - k * pr ? pr : sp - k * pr;
            CHECK(psp >= 1 && psp <= G::S);
            const Window w = window_at<BC>(t0 + (int64_t)k * pr, psp, n, DHW);
            CHECK(w.t0 == pc);
            pc += psp;
            check_df_window<BC>(w, n);
        }
        CHECK(pc == t0 + sp);
    }
    CHECK(covered == n);
}

template <int BC>
void check_grid(int64_t n) {
    using G = FusedGeom<256, M, 64>;
    using Gs = FusedGeom<128, M, 64>;
    for (int64_t slots : {1, 2, 152, 304, 456, 608})
        check<256, BC>(n, (int)fused_tile_rows(n, G::S, slots));
    check<128, BC>(n, (int)fused_tile_rows(n, Gs::S, 1));
    // the narrow-overlap batch variants (32 rows)
    check<256, BC, 32>(n, (int)fused_tile_rows(n, FusedGeom<256, M, 32>::S, 1));
    check<128, BC, 32>(n, (int)fused_tile_rows(n, FusedGeom<128, M, 32>::S, 1));
    using D = DfGeom<DT, M, DHW>;
    for (int64_t slots : {1, 2, 152, 304})
        for (int hw = DHW_MIN; hw < DHW; hw += 8)
            check_df<BC>(n, (int)fused_tile_rows(n, D::S, slots),
                         (int)fused_tile_rows(n, D::R - 2 * hw, slots), hw);
}

int main() {
    const int64_t big[] = {1000, 1278, 1279, 1280, 1281, 2557, 2558, 2559, 70001, 388800,
                           388801, 1048576, 3000000, 16777216, 16777217};
    for (int64_t n = 3; n <= 9000; ++n) {
        check_grid<BC_PERIODIC>(n);
        check_grid<BC_TRANSMISSIVE>(n);
    }
    for (int64_t n : big) {
        check_grid<BC_PERIODIC>(n);
        check_grid<BC_TRANSMISSIVE>(n);
    }
    // windows ending 3 or 4 cells before the domain end (the edge of the direct path)
    using G = FusedGeom<256, M, 64>;
    using Gs = FusedGeom<128, M, 64>;
    for (int64_t k = 1; k <= 40; ++k)
        for (int64_t e = 60; e <= 72; ++e) {
            check<256, BC_PERIODIC>(k * G::S + e, G::S);
            check<256, BC_TRANSMISSIVE>(k * G::S + e, G::S);
            check<128, BC_PERIODIC>(k * Gs::S + e, Gs::S);
            check<128, BC_TRANSMISSIVE>(k * Gs::S + e, Gs::S);
        }
    // full double-float windows (tiles of the largest size, as a 2^16 grid gets)
    using D = DfGeom<DT, M, DHW>;
    for (int64_t k = 1; k <= 80; ++k)
        for (int hw = DHW_MIN; hw < DHW; hw += 8) {
            const int sn = D::R - 2 * hw;
            check_df<BC_PERIODIC>(k * D::S, D::S, sn, hw);
            check_df<BC_TRANSMISSIVE>(k * D::S + 1, D::S, sn, hw);
            check_df<BC_PERIODIC>(k * sn, D::S, sn, hw);
            check_df<BC_TRANSMISSIVE>(k * sn + 1, D::S, sn, hw);
        }
    printf("large: R=%d S=%d NC=%d; small: R=%d S=%d NC=%d; double-float: R=%d S=%d NC=%d; "
           "windows=%lld\nall index checks passed\n", G::R, G::S, G::NC, Gs::R, Gs::S, Gs::NC,
           D::R, D::S, D::NC, checked_windows);
    return 0;
}
