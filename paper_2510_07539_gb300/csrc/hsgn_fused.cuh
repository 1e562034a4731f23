// hsgn_fused.cuh -- the mixed-precision stage in one launch (sm_103a).
//
// Same arithmetic as hsgn_mixed.cuh (Sec. 4.2, eq. (GN_hyp_eq_semi_fully_discrete),
// increment form; Sec. 3.2, efficient form of the tableau), but the depth
// system A dh = d - A h_b is solved on overlapping windows instead of through
// a global separator system, so that fluxes, rows, solve and back-substitution
// of a tile run in one CTA and nothing per row goes through HBM except the
// stage inputs and outputs:
//  * CTA p owns the tile of rows [t0, t0 + sp) and solves the rows of the
//    window [t0 - HW, t0 + sp + HW) with the coupling to the rows outside the
//    window dropped. Periodic: indices are taken modulo n, so a window longer
//    than the grid is the periodic system unrolled, whose solution is the
//    periodic one. Transmissive: the window is clipped at the domain ends,
//    where the Neumann rows are the exact ones.
//  * A has diagonal 1 + l_i + r_i and off-diagonals -l_i, -r_i with
//    l_i = tau^2/dx^2 beta_{i-1/2}, r_i = tau^2/dx^2 beta_{i+1/2} > 0. The
//    error e caused by the dropped value x beyond the left edge solves the
//    window system with one forcing term at row 0, so e_i = rho_i e_{i-1} with
//    rho_i = l_i / (1 + l_i + r_i (1 - rho_{i+1})), starting from the right
//    edge. With kappa <= l_i, r_i <= K over the window every rho_i stays below
//    the smaller root rho* = 2K / (B + sqrt(B^2 - 4 kappa K)), B = 1 + K + kappa,
//    of rho = K / (1 + K + kappa (1 - rho)) (the iteration from the edge rises
//    monotonically towards it), hence |e_i| <= rho*^(i+1) |x|; the same holds
//    from the right. The tile rows and the rows of a tile-face mini window lie
//    HB = HW - 1 rows or more inside their window. Each CTA evaluates rho* from
//    the min and max of tau^2 beta / dx^2 over its cells and raises
//    HSGN_DEV_ERR_TRUNCATION when rho*^HB > 2^-30 (the single-precision
//    increments themselves carry 2^-24). For a uniform state rho* is the decay
//    rate of the inverse, about 0.55 at CFL_IMEX = 4.
//  * Mass: in stage 2 the face flux at a tile boundary is used by the two CTAs
//    on either side. Both solve the same mini-window of 2 HB rows centred on
//    that face with the same code path and evaluate the face flux from it, so
//    the two values are bitwise equal and the flux-form depth update stays
//    conservative. Stage 1 updates no depth: each face of G1 is written once,
//    by the tile on its left (periodic face -1/2 is read as face n-1/2).
//  * Stage 2 cannot update U in place (the windows of neighbouring tiles still
//    read U^n), so it writes U^{n+1} to a second state buffer.
//  * The state is held as double-float pairs x = hi + lo (hi = x rounded to
//    single precision, |lo| <= half an ulp of hi: a 48-bit significand), so
//    that no step of the stage needs the double-precision datapath, which on
//    sm_103a runs at 1/58 of the single-precision rate:
//      - hi is the single-precision value the stage works with;
//      - differences of neighbouring values are (hi1 - hi0) + (lo1 - lo0),
//        where hi1 - hi0 is exact for values within a factor 2 (Sterbenz);
//      - h^2 - m uses the exact product hi*hi = p + e (one fma);
//      - the accumulation U + dU is TwoSum (Knuth) followed by a renormalising
//        TwoSum, and the depth subtracts the exact difference of the two face
//        fluxes (TwoSum again), so the depth update stays conservative up to
//        the 2^-49 rounding of the pair.
#pragma once

#include "hsgn_mixed.cuh"

namespace hsgn {

// s + e = a + b exactly (Knuth's TwoSum, no ordering assumption).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) + (x + y) with x + y given exactly as two floats; renormalised by
// Dekker's FastTwoSum (hi' = s + e rounded is exact to rounding whatever the
// ordering; lo' loses accuracy only where the pair's lowest bits do not matter).
__device__ __forceinline__ float2 df_add(float2 a, float x, float y) {
    float s, e;
    two_sum(a.x, x, s, e);
    e = __fadd_rn(e, __fadd_rn(a.y, y));
    const float h = __fadd_rn(s, e);
    return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}

// (hi, lo) + x for one float x (df_add with y = 0).
__device__ __forceinline__ float2 df_add1(float2 a, float x) {
    float s, e;
    two_sum(a.x, x, s, e);
    e = __fadd_rn(e, a.y);
    const float h = __fadd_rn(s, e);
    return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}

// Hint: bring the 128-byte line holding *a into L2 (a must point into an allocation).
__device__ __forceinline__ void prefetch_l2(const void* a) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

// Pair of a double (state conversion, off the stepping path).
__device__ __forceinline__ float2 df_of(double x) {
    const float hi = __double2float_rn(x);
    return make_float2(hi, __double2float_rn(x - (double)hi));
}

struct FusedParams {
    int64_t n;
    int32_t stage;        // 1: writes G1, dq1, dm1, dr1; 2: writes U^{n+1} to out
    int32_t local_speed;
    int32_t track_speed;  // stage 1 clears *speed_next, stage 2 folds max |u| into it
    int32_t S;            // tile rows (<= the kernel's capacity)
    int32_t slots;        // co-resident CTAs of this launch (0: no prefetch of the next wave)
    float g, lam, tau, tdx, fq, Cc, fd, lt2, ltau, wl1, wb1;
    const float2* U[4];             // U^n (double-float pairs)
    float *G1, *dq1, *dm1, *dr1;    // stage-1 increments; G1 has n+1 faces (face i+1/2 at i+1)
    float2* out[4];                 // U^{n+1} (stage 2; not aliased with U)
    const double* speed;            // global Rusanov speed of the step
    double* speed_next;             // max |u^{n+1}|
    unsigned* err;
    // a batch of independent instances (batched != 0): tile b belongs to instance
    // tile_inst[b]; for that instance inst[] gives the packed cell offset, n, dx,
    // lambda, dt, its tile rows (`base`), tile count (`P`) and first tile (`blk0`);
    // speed / speed_next are then per-instance arrays. The fields n, S, tau and
    // the constants derived from it above are used for a single instance only.
    int32_t batched;
    const InstInfo* inst;
    const int32_t* tile_inst;
    const float2* bathy;  // bottom b per cell as double-float pairs (bottom form only)
};

// Window of tile p: tile rows [t0, t0 + sp); window rows [wl, wl + W) (global,
// periodic ones not yet reduced modulo n); the tile starts at window row lo.
// lend / rend: the window ends at the domain end (transmissive only).
struct Window {
    int64_t t0, wl;
    int sp, W, lo;
    bool lend, rend;
};

template <int BC>
__host__ __device__ inline Window window_of(int64_t p, int64_t n, int S, int HW) {
    Window w;
    w.t0 = p * (int64_t)S;
    const int64_t rest = n - w.t0;
    w.sp = (int)(rest < S ? rest : S);
    if (BC == BC_PERIODIC) {
        w.wl = w.t0 - HW;
        w.W = w.sp + 2 * HW;
        w.lend = w.rend = false;
    } else {
        w.wl = w.t0 - HW < 0 ? 0 : w.t0 - HW;
        const int64_t wr = w.t0 + w.sp + HW > n ? n : w.t0 + w.sp + HW;
        w.W = (int)(wr - w.wl);
        w.lend = w.wl == 0;
        w.rend = wr == n;
    }
    w.lo = (int)(w.t0 - w.wl);
    return w;
}

// Mini-window of the face between global rows t-1 and t: rows [ml, ml + mw)
// (global, unreduced), clipped at transmissive domain ends; the face's right
// row is mini row t - ml.
struct MiniWindow {
    int64_t ml;
    int mw;
    bool lend, rend;
};

template <int BC>
__host__ __device__ inline MiniWindow mini_of(int64_t t, int64_t n, int HB) {
    MiniWindow m;
    if (BC == BC_PERIODIC) {
        m.ml = t - HB;
        m.mw = 2 * HB;
        m.lend = m.rend = false;
    } else {
        m.ml = t - HB < 0 ? 0 : t - HB;
        const int64_t mr = t + HB > n ? n : t + HB;
        m.mw = (int)(mr - m.ml);
        m.lend = m.ml == 0;
        m.rend = mr == n;
    }
    return m;
}

// Cell of global index x: modulo n (periodic, any x) or clamped (transmissive).
template <int BC>
__host__ __device__ __forceinline__ int64_t cell_at(int64_t x, int64_t n) {
    if (BC == BC_PERIODIC) {
        if (x >= 0 && x < n) return x;
        if (x < 0 && x >= -n) return x + n;
        if (x >= n && x < 2 * n) return x - n;
        const int64_t r = x % n;
        return r < 0 ? r + n : r;
    }
    return x < 0 ? 0 : (x >= n ? n - 1 : x);
}

// Cells read by the load phase for window cell index j (window cell j - 3):
// the cell itself (gi) and its right neighbour (gn), j = 0 .. W + 5. A window
// whose cells -3 .. W + 3 all lie in [1, n) (`inner`) indexes them directly,
// as offsets j and j + 1 from cell wl - 3 (cell 0 is left out: the face left
// of it is read as the periodic face n - 1/2).
__host__ __device__ inline bool inner_window(int64_t wl, int W, int64_t n) {
    return wl - 3 >= 1 && wl + W + 3 < n;
}

template <int BC>
__host__ __device__ __forceinline__ void load_cells(bool inner, int64_t wl, int j, int64_t n,
                                                    int64_t& gi, int64_t& gn) {
    gi = inner ? wl - 3 + j : cell_at<BC>(wl - 3 + j, n);
    gn = inner ? gi + 1 : cell_at<BC>(wl - 2 + j, n);
}

// Tile rows of an n-row grid for a kernel of tiles of at most smax rows:
// equal tiles, as many as fill `slots` co-resident CTAs in whole waves.
__host__ inline int64_t fused_tile_rows(int64_t n, int64_t smax, int64_t slots) {
    const int64_t pmin = (n + smax - 1) / smax;
    if (pmin >= slots) {
        const int64_t waves = (pmin + slots - 1) / slots;
        return (n + waves * slots - 1) / (waves * slots);
    }
    return (n + pmin - 1) / pmin;
}

// Capacity of the fused kernel: T threads, M = 4 rows per thread, overlap HW.
// Thread t owns the window cells and rows 4t .. 4t + 3 in the flux,
// coefficient, row and solve phases; the W + 2 cells c = -1 .. W whose
// coefficients are formed must fit, hence R = T M - 2 window rows (the
// elimination adds one identity row). The cell arrays have a multiple of 4
// entries so that every array starts on a 16-byte boundary.
template <int T, int M, int HW>
struct FusedGeom {
    static constexpr int R = T * M - 2;      // window rows
    static constexpr int S = R - 2 * HW;     // largest tile
    static constexpr int HB = HW - 1;        // half-width of a tile-boundary mini-window
    static constexpr int NC = (pd_size(R + 6) + 3) & ~3;
    static constexpr int MB = (2 * HB + 1 + 31) / 32;  // rows per lane of the mini solve
    static_assert(M == 4, "the cell phases move four cells per thread as one float4");
    static_assert(S > 0, "overlap too wide for the window");
};

// Shared-memory vectors of four consecutive cells (16-byte aligned).
__device__ __forceinline__ void lds4(const float* a, float* v) {
    const float4 x = *reinterpret_cast<const float4*>(a);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
}
__device__ __forceinline__ void sts4(float* a, const float* v) {
    *reinterpret_cast<float4*>(a) = make_float4(v[0], v[1], v[2], v[3]);
}

// Single-precision reciprocal: the hardware approximation (hsgn_tridiag.cuh).
__device__ __forceinline__ float rcpa(float x) { return rcp(x); }

// Shared memory. Arrays are reused once their phase is over (cell c of the
// window at index c+3 in the U arrays, c+1 in the per-cell arrays):
//   phase 0: hl, ql, ml, rl (U_l), qb, mb, rb (U_b), Dh, Dq, Dm (differences
//            of U_b at the face to the right of a cell);
//   phases 1+2 (fluxes in registers): dq -> ql, dm -> X0, dr -> rl,
//            beta -> hl, delta -> ml;
//   phase 3 (rows in registers): for the stage-2 mini solves the face couplings
//            tau^2 beta_{f+1/2}/dx^2 -> rb and the right-hand sides -> mb
//            (both padded: a lane of the mini solve reads rows at a stride);
//   phase 4: dh -> Dq (window row r at r + 4); face mass fluxes of the tile -> rb.
// The bottom form (WB) reuses Dh for the jump of h_l - h_b at the face, Dm for
// P_l = h_l^2 - m_l and then beta (hl keeps h_l), ml for the non-gravity part
// of the pressure, mb for p~, and adds the free-surface jump Z (which becomes
// the face force Psi in phase 3), the bottom jump Db, the bottom source Sb
// and m_b - m_l = (w_b - w_l) dm1 taken from the increment (the single-
// precision m_b and m_l round it away, and lambda alpha amplifies it).
template <int NC, bool WB>
struct FusedWb {
    float Z[NC], Db[NC], Sb[NC], Mbl[NC];
};
template <int NC>
struct FusedWb<NC, false> {};

template <int T, int M, int HW, bool WB = false>
struct FusedShared {
    static constexpr int NC = FusedGeom<T, M, HW>::NC;
    float hl[NC], ql[NC], ml[NC], rl[NC];
    float qb[NC], mb[NC], rb[NC];
    float Dh[NC], Dq[NC], Dm[NC];
    float X0[NC];
    FusedWb<NC, WB> wb;
    SepShared<T, float> sep;
    float bnd[2][2];       // dh of the two rows at the left / right tile face (mini solves)
    unsigned kmax, kmin;   // bits of max / min tau^2 beta / dx^2 (positive floats order as integers)
};

// WB selects the well-balanced bottom form (the flat printed scheme otherwise):
// the m^dag bottom source -(3/2) tau q_l b_x, and in place of the delta terms
// the face forces Phi_{f+1/2} of the bottom form, used in the increment form
//   Psi_f = Phi_f + beta_f (h_b jump) = g hbar_f (h_l + b jump) + (pi jump)
//           + (3/2) p~_f (b jump) - beta_f (h_l - h_b jump),
// with pi = eta p~ + lambda alpha (m^dag b_1 - m_l) the non-gravity part of
// p^ (g/2 (h_l^2 jump) + g hbar_f (b jump) = g hbar_f (h_l + b jump) exactly).
// The free-surface jump comes from the double-float h and b, and p~ and
// m^dag b_1 - m_l from P_l = h_l^2 - m_l of the pairs, so that a lake at rest
// stays at rest to the pairs' precision rather than to single precision.
// STAGE (1 or 2, equal to p.stage) specialises the kernel for its stage.
template <int T, int M, int HW, int BC, bool WB, int STAGE>
__global__ void __launch_bounds__(T, (WB ? 768 : 1024) / T) k_mixed_fused(const FusedParams p) {
    static_assert(STAGE == 1 || STAGE == 2, "two stages");
    using Gm = FusedGeom<T, M, HW>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<FusedShared<T, M, HW, WB>*>(smem_raw);
    const int tid = threadIdx.x;
    // the instance of this tile: its size, offsets, constants and speeds
    int64_t n = p.n, cell0 = 0, face0 = 0, tile = blockIdx.x;
    int S = p.S;
    float c_tau = p.tau, c_lam = p.lam, c_tdx = p.tdx, c_fq = p.fq, c_Cc = p.Cc, c_fd = p.fd;
    float c_lt2 = p.lt2, c_ltau = p.ltau;
    const double* spd_in = p.speed;
    double* spd_out = p.speed_next;
    if (p.batched) {
        const int k = p.tile_inst[blockIdx.x];
        const InstInfo I = p.inst[k];
        n = I.n;
        S = (int)I.base;
        tile = blockIdx.x - I.blk0;
        cell0 = I.cell0;
        face0 = I.cell0 + k;  // instance k's n+1 faces follow those of instances < k
        // the instance's stage constants (set on the host with its time step)
        c_tau = I.tau;
        c_lam = I.lamf;
        c_tdx = I.tdx;
        c_fq = I.fq;
        c_Cc = I.Cc;
        c_fd = I.fd;
        c_lt2 = I.lt2;
        c_ltau = I.ltau;
        spd_in = p.speed + k;
        spd_out = p.speed_next + k;
    }
    const Window win = window_of<BC>(tile, n, S, HW);
    const int W = win.W;
    const int64_t wl = win.wl;
    constexpr bool two = STAGE == 2;
    const float wl1 = p.wl1, wb1 = p.wb1;
    const float2* __restrict__ U0 = p.U[0] + cell0;
    const float2* __restrict__ U1 = p.U[1] + cell0;
    const float2* __restrict__ U2 = p.U[2] + cell0;
    const float2* __restrict__ U3 = p.U[3] + cell0;
    const float* __restrict__ G1 = p.G1 + face0;
    float* const G1w = p.G1 + face0;
    float* const dq1p = p.dq1 + cell0;
    float* const dm1p = p.dm1 + cell0;
    float* const dr1p = p.dr1 + cell0;
    // (G1: the face left of cell i at i, right of it at i + 1; the periodic
    // face -1/2 is read as face n-1/2, which only the last tile writes)
    if (tid == 0) {
        sm.kmax = 0u;
        sm.kmin = 0x7F7FFFFFu;
    }
    if (p.track_speed && !two && tile == 0 && tid == 0) *spd_out = 0.0;

    // ---- 0. window cells -3 .. W+2 (index c + 3)
    constexpr int NL = (Gm::R + 6 + T - 1) / T;
    // windows away from the domain ends read cells wl-3 .. wl+W+3 directly
    const bool inner = inner_window(wl, W, n);
    // one window cell: its loads come from `at` (cell itself, offset 0, or its
    // right neighbour, offset 1, of U^n and the stage-1 increments; faces
    // left / right of either); the direct path indexes from cell wl - 3 with
    // 32-bit offsets, the general one maps every cell through cell_at
    auto load_cell = [&](const int j, const auto& at) {
        const float2 h0 = at.u(U0, 0), q0 = at.u(U1, 0);
        const float2 m0 = at.u(U2, 0), rr0 = at.u(U3, 0);
        const float2 h1 = at.u(U0, 1), q1 = at.u(U1, 1), m1 = at.u(U2, 1);
        float dh1 = 0.f, dq1 = 0.f, dm1 = 0.f, dr1 = 0.f, dh1n = 0.f, dq1n = 0.f, dm1n = 0.f;
        if constexpr (two) {
            const float g0 = at.face_left(G1, 0), g1 = at.face_right(G1, 0);
            const float g2 = at.face_left(G1, 1), g3 = at.face_right(G1, 1);
            dq1 = at.f(dq1p, 0);
            dm1 = at.f(dm1p, 0);
            dr1 = at.f(dr1p, 0);
            dq1n = at.f(dq1p, 1);
            dm1n = at.f(dm1p, 1);
            dh1 = g0 - g1;
            dh1n = g2 - g3;
        }
        // x + w d with the stage-1 increments (stage 1 has none: x itself)
        auto inc = [](float w, float d, float x) {
            if constexpr (two) return fmaf(w, d, x);
            else return x;
        };
        const float hf = h0.x, qf = q0.x, mf = m0.x, rf = rr0.x;
        sm.hl[j] = inc(wl1, dh1, hf);
        sm.ql[j] = inc(wl1, dq1, qf);
        sm.ml[j] = inc(wl1, dm1, mf);
        sm.rl[j] = inc(wl1, dr1, rf);
        sm.qb[j] = inc(wb1, dq1, qf);
        if constexpr (two) {  // stage 1: U_b = U_l = U^n, read from ml, rl in the cell phase
            sm.mb[j] = fmaf(wb1, dm1, mf);
            sm.rb[j] = fmaf(wb1, dr1, rf);
        }
        // differences of U^n at the face to the right: (hi1 - hi0) + (lo1 - lo0)
        const float Dhn = __fadd_rn(__fsub_rn(h1.x, h0.x), __fsub_rn(h1.y, h0.y));
        const float Dqn = __fadd_rn(__fsub_rn(q1.x, q0.x), __fsub_rn(q1.y, q0.y));
        sm.Dq[j] = inc(wb1, dq1n - dq1, Dqn);
        if constexpr (!WB) {
            const float Dmn = __fadd_rn(__fsub_rn(m1.x, m0.x), __fsub_rn(m1.y, m0.y));
            sm.Dh[j] = inc(wb1, dh1n - dh1, Dhn);
            sm.Dm[j] = inc(wb1, dm1n - dm1, Dmn);
        } else {
            (void)dm1n;  // the bottom form carries P_l instead of the m difference
            const float2 b0 = at.u(p.bathy + cell0, 0), b1 = at.u(p.bathy + cell0, 1);
            // free-surface jump (h_l + b) at the face right of the cell:
            // hi1 - hi0 of h is exact, that of b is taken exactly by TwoSum
            float sb, eb;
            two_sum(b1.x, -b0.x, sb, eb);
            const float lo = __fadd_rn(__fadd_rn(__fsub_rn(h1.y, h0.y), __fsub_rn(b1.y, b0.y)), eb);
            const float hz = __fadd_rn(__fsub_rn(h1.x, h0.x), sb);
            sm.wb.Z[j] = inc(wl1, dh1n - dh1, __fadd_rn(hz, lo));
            sm.wb.Db[j] = __fadd_rn(sb, __fadd_rn(__fsub_rn(b1.y, b0.y), eb));
            sm.Dh[j] = two ? (wl1 - wb1) * (dh1n - dh1) : 0.f;  // (h_l - h_b) jump
            // P_l = h_l^2 - m_l: hi^2 = pp + pe exactly, pp - m.hi exact for m close to h^2
            const float pp = __fmul_rn(hf, hf);
            const float pe = fmaf(hf, hf, -pp);
            const float P0 = __fadd_rn(__fsub_rn(pp, m0.x), fmaf(2.f * hf, h0.y, __fsub_rn(pe, m0.y)));
            sm.Dm[j] = inc(wl1, fmaf(dh1, fmaf(wl1, dh1, 2.f * hf), -dm1), P0);
            // (3/2) q_l (b_{c+1} - b_{c-1}) of the cells c = -1 .. W whose m^dag is formed
            float src = 0.f;
            if (j >= 2 && j <= W + 3)
                src = 1.5f * inc(wl1, dq1, qf) * (b1.x - at.u(p.bathy + cell0, -1).x);
            sm.wb.Sb[j] = src;
            sm.wb.Mbl[j] = two ? (wb1 - wl1) * dm1 : 0.f;
        }
    };
    if (inner) {
        // cells wl - 3 + j + d for d = -1, 0, 1: all in [0, n) for j in [2, W + 3]
        // (d = -1) and j <= W + 5 (d = 0, 1), by the window test above
        const int64_t b = wl - 3;
        // (a + b) is the same for every cell of the CTA; only the 32-bit
        // offset j + d varies
        struct Direct {
            int64_t b;
            int j;
            __device__ float2 u(const float2* a, int d) const { return __ldg((a + b) + (j + d)); }
            __device__ float f(const float* a, int d) const { return __ldg((a + b) + (j + d)); }
            __device__ float face_left(const float* a, int d) const {
                return __ldg((a + b) + (j + d));
            }
            __device__ float face_right(const float* a, int d) const {
                return __ldg((a + b) + (j + d + 1));
            }
        };
#pragma unroll
        for (int it = 0; it < NL; ++it) {
            const int j = tid + it * T;
            if (j < W + 6) load_cell(j, Direct{b, j});
        }
    } else {
        struct General {
            int64_t gi, gn, gp, n;
            __device__ int64_t cell(int d) const { return d == 0 ? gi : (d > 0 ? gn : gp); }
            __device__ float2 u(const float2* a, int d) const { return __ldg(a + cell(d)); }
            __device__ float f(const float* a, int d) const { return __ldg(a + cell(d)); }
            // G1 index of the face left of cell i: periodic face -1/2 is face n-1/2
            __device__ float face_left(const float* a, int d) const {
                const int64_t c = cell(d);
                return __ldg(a + ((BC == BC_PERIODIC && c == 0) ? n : c));
            }
            __device__ float face_right(const float* a, int d) const {
                return __ldg(a + cell(d) + 1);
            }
        };
#pragma unroll
        for (int it = 0; it < NL; ++it) {
            const int j = tid + it * T;
            if (j < W + 6) {
                int64_t gi, gn;
                load_cells<BC>(false, wl, j, n, gi, gn);
                const int64_t gp = cell_at<BC>(wl - 4 + j, n);
                load_cell(j, General{gi, gn, gp, n});
            }
        }
    }
    // L2 prefetch of the tile that the next wave of CTAs starts on this slot
    // (tile blockIdx.x + slots of this launch: CTAs are dispatched in index
    // order as slots free up; in a batch it may belong to another instance):
    // one 128-byte line per thread and array over the cells of its window that
    // lie in [0, n) of its instance; PF threads cover the widest window
    constexpr int PF = (Gm::R + 6 + 15) / 16;
    if (p.slots > 0 && tid < PF) {
        const int64_t ts = (int64_t)blockIdx.x + p.slots;
        if (ts < (int64_t)gridDim.x) {
            int64_t sn = p.n, sc = 0, sf = 0, st = ts;
            int sS = p.S;
            if (p.batched) {
                const int k = p.tile_inst[ts];
                const InstInfo& I = p.inst[k];
                sn = I.n;
                sS = (int)I.base;
                st = ts - I.blk0;
                sc = I.cell0;
                sf = I.cell0 + k;
            }
            const Window ws = window_of<BC>(st, sn, sS, HW);
            const int64_t c0 = ws.wl - 3 < 0 ? 0 : ws.wl - 3;
            const int64_t c1 = ws.wl + ws.W + 3 > sn ? sn : ws.wl + ws.W + 3;
            const int64_t c = c0 + 16 * (int64_t)tid;  // 16 pairs per line
            if (c < c1) {
#pragma unroll
                for (int v = 0; v < 4; ++v) prefetch_l2(p.U[v] + sc + c);
                if constexpr (WB) prefetch_l2(p.bathy + sc + c);
            }
            if constexpr (two) {
                const int64_t f = c0 + 32 * (int64_t)tid;  // 32 floats per line
                if (f < c1) {
                    prefetch_l2(p.G1 + sf + f);
                    prefetch_l2(p.dq1 + sc + f);
                    prefetch_l2(p.dm1 + sc + f);
                    prefetch_l2(p.dr1 + sc + f);
                }
            }
        }
    }
    __syncthreads();

    const float tau = c_tau, lam = c_lam, g = p.g;
    const float gspeed = p.local_speed ? 0.f : (float)(*spd_in);
    unsigned bad = 0;

    // ---- 1+2. Thread t owns the cells j = 4t .. 4t + 3 (window cell c = j - 1;
    //           c = -1 .. W are formed). In registers it evaluates the Rusanov
    //           fluxes of U_l (Sec. 4.1) at the five faces jf = 4t .. 4t + 4 around
    //           them (face jf lies between cells jf - 2 and jf - 1) from the
    //           cells 4t - 3 .. 4t + 4 (array index 4t .. 4t + 7, two float4 per
    //           variable), then the increments and coefficients of its cells:
    //           r^dag = r_b + dr' + lambda tau, m^dag = m_b + dm' + lambda tau^2,
    //           q^dag = q_b + dq. The results are stored after the barrier
    //           (they reuse the arrays the other threads still read).
    const float lt2 = c_lt2, Cc = c_Cc, htdx = 0.5f * c_tdx;
    const int j0 = 4 * tid;
    float dq_[4], dm_[4], dr_[4], be_[4], de_[4];
    float pt_[WB ? 4 : 1];
    float kloc = 0.f, kmin = 3.0e38f;
    {
        float H[8], Q[8], Mv[8], Rv[8];
        lds4(sm.hl + j0, H); lds4(sm.hl + j0 + 4, H + 4);
        lds4(sm.ql + j0, Q); lds4(sm.ql + j0 + 4, Q + 4);
        lds4(sm.ml + j0, Mv); lds4(sm.ml + j0 + 4, Mv + 4);
        lds4(sm.rl + j0, Rv); lds4(sm.rl + j0 + 4, Rv + 4);
        float FQ[5], FM[5], FR[5];
#pragma unroll
        for (int e = 0; e < 5; ++e) {
            const float hm = H[e], h0 = H[e + 1], h1 = H[e + 2], h2 = H[e + 3];
            const float qm = Q[e], q0 = Q[e + 1], q1 = Q[e + 2], q2 = Q[e + 3];
            const float mm = Mv[e], m0 = Mv[e + 1], m1 = Mv[e + 2], m2 = Mv[e + 3];
            const float rm = Rv[e], r0_ = Rv[e + 1], r1 = Rv[e + 2], r2 = Rv[e + 3];
            const float hL = fmaf(0.25f, h1 - hm, h0), hR = fmaf(-0.25f, h2 - h0, h1);
            const float qL = fmaf(0.25f, q1 - qm, q0), qR = fmaf(-0.25f, q2 - q0, q1);
            const float mL = fmaf(0.25f, m1 - mm, m0), mR = fmaf(-0.25f, m2 - m0, m1);
            const float rL = fmaf(0.25f, r1 - rm, r0_), rR = fmaf(-0.25f, r2 - r0_, r1);
            if (j0 + e < W + 3 && !pos_finite(fminf(hL, hR))) bad |= HSGN_DEV_ERR_DEPTH;
            const float ip = rcpa(hL * hR);
            const float uL = qL * hR * ip, uR = qR * hL * ip;
            const float s = p.local_speed ? fmaxf(fabsf(uL), fabsf(uR)) : gspeed;
            // twice the flux: the 1/2 is folded into htdx below (halving is exact)
            FQ[e] = fmaf(uL, qL, uR * qR) - s * (qR - qL);
            FM[e] = fmaf(uL, mL, uR * mR) - s * (mR - mL);
            FR[e] = fmaf(uL, rL, uR * rR) - s * (rR - rL);
        }
        // cells j at array index j + 2: rb, mb (and the bottom-form arrays) of
        // 4t + 2 .. 4t + 5 from two float4 each; hl, ml from the registers above
        float RB[8], MB[8];
        if constexpr (two) {
            lds4(sm.rb + j0, RB); lds4(sm.rb + j0 + 4, RB + 4);
            lds4(sm.mb + j0, MB); lds4(sm.mb + j0 + 4, MB + 4);
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                RB[i] = Rv[i];
                MB[i] = Mv[i];
            }
        }
        float SB[WB ? 8 : 1], PL[WB ? 8 : 1], MBL[WB ? 8 : 1];
        if constexpr (WB) {
            lds4(sm.wb.Sb + j0, SB); lds4(sm.wb.Sb + j0 + 4, SB + 4);
            lds4(sm.Dm + j0, PL); lds4(sm.Dm + j0 + 4, PL + 4);
            lds4(sm.wb.Mbl + j0, MBL); lds4(sm.wb.Mbl + j0 + 4, MBL + 4);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            dq_[k] = dm_[k] = dr_[k] = be_[k] = de_[k] = 0.f;
            if constexpr (WB) pt_[k] = 0.f;
            if (j0 + k < W + 2) {
                const float drv = -htdx * (FR[k + 1] - FR[k]);
                float dmv = fmaf(tau, RB[k + 2] + drv, -htdx * (FM[k + 1] - FM[k]));
                // bottom source of the (h eta) equation, -(3/2) h u b_x (Sec. 2.3, eq. (hSGNb_eq)), from U_l
                if constexpr (WB) dmv = fmaf(-c_fq, SB[k + 2], dmv);
                const float dqv = -htdx * (FQ[k + 1] - FQ[k]);
                const float msv = MB[k + 2] + dmv + lt2;
                const float h = H[k + 2];
                if (!pos_finite(h)) bad |= HSGN_DEV_ERR_DEPTH;
                const float Dh_ = fmaf(h, h, lt2);
                const float Rr = rcpa(h * Dh_);
                const float ih = Dh_ * Rr;
                const float iD = h * Rr;
                const float eta = Mv[k + 2] * ih;
                const float e = eta * ih;
                const float alpha = fmaf(2.f, e, -1.f) * ih * (-1.f / 3.f);
                const float c2 = fmaf(g, h, (lam * (1.f / 3.f)) * e * e);
                const float a2 = fmaf(-lam * eta, alpha, c2);
                const float ib1 = h * h * iD;
                const float beta2 = (2.f * lt2) * h * iD * iD;
                const float beta = fmaf(lam * alpha * beta2, msv, a2);
                if (!pos_finite(beta)) bad |= HSGN_DEV_ERR_COERCIVE;
                dq_[k] = dqv;
                dm_[k] = dmv;
                dr_[k] = drv;
                be_[k] = beta;
                if constexpr (!WB) {
                    de_[k] = alpha * ib1;
                } else {
                    // p~ = (lambda/3)(1 - m_l/h_l^2) = (lambda/3) P_l / h_l^2;
                    // m^dag b_1 - m_l = (h^2 (m_b - m_l + dm) + lambda tau^2 P_l) / (h^2 + lambda tau^2)
                    const float Pl = PL[k + 2];
                    const float ptil = (lam * (1.f / 3.f)) * Pl * ih * ih;
                    const float X = fmaf(h * h, MBL[k + 2] + dmv, lt2 * Pl) * iD;
                    de_[k] = fmaf(eta, ptil, lam * alpha * X);  // pi = eta p~ + lambda alpha X
                    pt_[k] = ptil;
                }
                kloc = fmaxf(kloc, Cc * beta);
                kmin = fminf(kmin, Cc * beta);
            }
        }
    }
    __syncthreads();
    float* const dqa = sm.ql;
    float* const dma = sm.X0;
    float* const dra = sm.rl;
    float* const bea = WB ? sm.Dm : sm.hl;
    float* const dea = sm.ml;  // delta (flat) or pi (bottom form)
    float* const pta = sm.mb;  // p~ (bottom form)
    sts4(dqa + j0, dq_);
    sts4(dma + j0, dm_);
    sts4(dra + j0, dr_);
    sts4(bea + j0, be_);
    sts4(dea + j0, de_);
    if constexpr (WB) sts4(pta + j0, pt_);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kloc = fmaxf(kloc, __shfl_xor_sync(0xffffffffu, kloc, o));
        kmin = fminf(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
    }
    if ((tid & 31) == 0) {
        if (pos_finite(kloc)) atomicMax(&sm.kmax, __float_as_uint(kloc));
        if (pos_finite(kmin)) atomicMin(&sm.kmin, __float_as_uint(kmin));
    }
    __syncthreads();
    if (BC == BC_TRANSMISSIVE && (win.lend || win.rend)) {  // (uniform over the CTA)
        // zero-order ghost copies at the domain ends
        if (tid == 0 && win.lend) {
            dqa[0] = dqa[1]; dma[0] = dma[1]; dra[0] = dra[1]; bea[0] = bea[1]; dea[0] = dea[1];
            if constexpr (WB) pta[0] = pta[1];
        }
        if (tid == 0 && win.rend) {
            const int a = W + 1, c = W;
            dqa[a] = dqa[c]; dma[a] = dma[c]; dra[a] = dra[c]; bea[a] = bea[c]; dea[a] = dea[c];
            if constexpr (WB) pta[a] = pta[c];
        }
        __syncthreads();
    }

    // ---- 3. rows i = 4t .. 4t + 3 of A dh = d - A h_b, in the registers of
    //         thread t: face couplings k_j = tau^2/dx^2 beta at the faces j = 4t ..
    //         4t + 4 (face j between rows j - 1 and j; zero across a transmissive
    //         domain end, which makes the end rows the Neumann rows) and the
    //         right-hand sides d_i (cell c of the per-cell arrays at c + 1, the face
    //         right of cell c of the difference arrays at c + 3). The couplings and
    //         right-hand sides also go to shared memory for the tile-face mini
    //         solves of stage 2 (face j at pd(j), row i at pd(i)), the bottom
    //         form's face forces Psi for the face fluxes (face j at j + 2).
    const float fq = c_fq, hfd = 0.5f * c_fd, hCc = 0.5f * Cc;
    float* const BF = sm.rb;
    float* const RD = sm.mb;
    float* Psi = nullptr;  // face forces of the bottom form, face j at j + 2
    if constexpr (WB) Psi = sm.wb.Z;
    float KF[5], rd[4];
    float PS[WB ? 5 : 1];
    {
        float B[8], DQ[8], QA[8], DH[8];
        lds4(bea + j0, B); lds4(bea + j0 + 4, B + 4);
        lds4(sm.Dq + j0, DQ); lds4(sm.Dq + j0 + 4, DQ + 4);
        lds4(dqa + j0, QA); lds4(dqa + j0 + 4, QA + 4);
        lds4(sm.Dh + j0, DH); lds4(sm.Dh + j0 + 4, DH + 4);
        if constexpr (WB) {
            float H[8], PT[8], DE[8], Z[8], DB[8];
            lds4(sm.hl + j0, H); lds4(sm.hl + j0 + 4, H + 4);
            lds4(pta + j0, PT); lds4(pta + j0 + 4, PT + 4);
            lds4(dea + j0, DE); lds4(dea + j0 + 4, DE + 4);
            lds4(sm.wb.Z + j0, Z); lds4(sm.wb.Z + j0 + 4, Z + 4);
            lds4(sm.wb.Db + j0, DB); lds4(sm.wb.Db + j0 + 4, DB + 4);
#pragma unroll
            for (int e = 0; e < 5; ++e) {
                const int j = j0 + e;
                const float bf = 0.5f * (B[e] + B[e + 1]);
                const float hbar = 0.5f * (H[e + 2] + H[e + 3]);
                const float ptf = 0.5f * (PT[e] + PT[e + 1]);
                float psi = fmaf(g * hbar, Z[e + 2], DE[e + 1] - DE[e]);
                psi = fmaf(1.5f * ptf, DB[e + 2], psi);
                psi = fmaf(-bf, DH[e + 2], psi);
                float kf = __fmul_rn(Cc, bf);
                if (BC == BC_TRANSMISSIVE && ((j == 0 && win.lend) || (j == W && win.rend))) {
                    kf = 0.f;
                    psi = 0.f;
                }
                KF[e] = kf;
                PS[e] = psi;
            }
            // d_i - (A h_b)_i = -tau/(2dx) (q^dag_{i+1} - q^dag_{i-1}) + tau^2/dx^2 (Psi_{i+1/2} - Psi_{i-1/2})
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float dqc = DQ[k + 2] + DQ[k + 3] + (QA[k + 2] - QA[k]);
                rd[k] = fmaf(-fq, dqc, Cc * (PS[k + 1] - PS[k]));
            }
        } else {
            float DE[8], MA[8], DM[8];
            lds4(dea + j0, DE); lds4(dea + j0 + 4, DE + 4);
            lds4(dma + j0, MA); lds4(dma + j0 + 4, MA + 4);
            lds4(sm.Dm + j0, DM); lds4(sm.Dm + j0 + 4, DM + 4);
#pragma unroll
            for (int e = 0; e < 5; ++e) {
                const int j = j0 + e;
                float kf = __fmul_rn(hCc, B[e] + B[e + 1]);
                if (BC == BC_TRANSMISSIVE && ((j == 0 && win.lend) || (j == W && win.rend))) kf = 0.f;
                KF[e] = kf;
            }
            // Every product is rounded explicitly (fmaf / __fmul_rn): neighbouring
            // rows share products (the right face of row k is the left face of
            // row k + 1), and a shared product left to the compiler is not fused
            // where a single-use one is, so a row's bits would depend on its
            // position in the thread's four rows. The rows of a tile-face mini
            // window must come out bitwise equal in the two windows that hold
            // them. The face averages' 1/2 is folded into hfd and hCc.
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float bm = B[k] + B[k + 1], bp = B[k + 1] + B[k + 2];      // 2 beta_face
                const float dmn = DE[k] + DE[k + 1], dpl = DE[k + 1] + DE[k + 2];  // 2 delta_face
                const float dqc = DQ[k + 2] + DQ[k + 3] + (QA[k + 2] - QA[k]);
                const float dmp = DM[k + 3] + (MA[k + 2] - MA[k + 1]);
                const float dmm = DM[k + 2] + (MA[k + 1] - MA[k]);
                const float dd = fmaf(dpl, dmp, -__fmul_rn(dmn, dmm));
                const float hd = fmaf(bm, DH[k + 2], -__fmul_rn(bp, DH[k + 3]));
                rd[k] = fmaf(-fq, dqc, fmaf(hfd, dd, -__fmul_rn(hCc, hd)));
            }
        }
    }
    __syncthreads();
    // (the stores below overwrite arrays read above by the neighbouring threads)
    if constexpr (WB) {
#pragma unroll
        for (int e = 0; e < 4; e += 2)
            *reinterpret_cast<float2*>(Psi + j0 + e + 2) = make_float2(PS[e], PS[e + 1]);
    }
    // tile-boundary mini solves (the last two warps, while the others solve
    // the separator system of the window; wid = 1, 2 selects the face)
    // (stage 2 only: stage 1 writes every face of G1 once, from the tile on
    // its left, and updates no depth)
    const bool lface = two && !(BC == BC_TRANSMISSIVE && win.t0 == 0);
    const bool rface = two && !(BC == BC_TRANSMISSIVE && win.t0 + win.sp == n);
    if (two) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            BF[pd(j0 + k)] = KF[k];
            RD[pd(j0 + k)] = rd[k];
        }
    }
    auto mini = [&](int wid) {
        const int side = wid - 1;
        if (side < 0 || side > 1 || !(side == 0 ? lface : rface)) return;
        const int64_t tf = side == 0 ? win.t0 : win.t0 + win.sp;  // right row of the face
        const MiniWindow mwn = mini_of<BC>(tf, n, Gm::HB);
        const int ms = (int)(mwn.ml - wl);                         // first mini row in the window
        const int mw = mwn.mw;
        // mini row k (window row ms + k); its first / last row drops its outer coupling
        auto rowm = [&](int k, float& a, float& bb, float& c, float& d) {
            if (k >= mw) {
                a = 0.f; bb = 1.f; c = 0.f; d = 0.f;
                return;
            }
            const int i = ms + k;
            const float kl = BF[pd(i)], kr = BF[pd(i + 1)];
            a = (k == 0 && !mwn.lend) ? 0.f : -kl;
            c = (k == mw - 1 && !mwn.rend) ? 0.f : -kr;
            bb = 1.f + kl + kr;
            d = RD[pd(i)];
        };
        float y[Gm::MB], v[Gm::MB], w[Gm::MB], last[4];
        int cs, m;
        warp_block_solve<Gm::MB>(mw + 1, rowm, y, v, w, cs, m, last, p.err);
        const int kr = (int)(tf - mwn.ml);  // mini row of the face's right row
#pragma unroll
        for (int k = 0; k < Gm::MB; ++k) {
            if (k < m) {
                if (cs + k == kr - 1) sm.bnd[side][0] = y[k];
                if (cs + k == kr) sm.bnd[side][1] = y[k];
            }
        }
    };
    float* const dha = sm.Dq;  // dh of window row r at r + 4, r = -1 .. W (rows 4t.. as a float4)
    {
        // row 4t + k of the window; the first / last window row drops its outer
        // coupling; the rows from W on close the window (identity)
        auto roww = [&](int k, int i, float& a, float& bb, float& c, float& d) {
            if (i >= W) {
                a = 0.f; bb = 1.f; c = 0.f; d = 0.f;
                return;
            }
            const float kl = KF[k], kr = KF[k + 1];
            a = (i == 0 && !win.lend) ? 0.f : -kl;
            c = (i == W - 1 && !win.rend) ? 0.f : -kr;
            bb = 1.f + kl + kr;
            d = rd[k];
        };
        float y[M];
        if constexpr (two) {
            // the separators by cyclic reduction over all warps but the last
            // two, which solve the tile-face mini windows meanwhile
            cta_window_solve<T, M, T - 64>(W + 1, roww, sm.sep, y, p.err, mini);
        } else {
            // no mini windows in stage 1: the separators by cyclic reduction over all threads
            cta_window_solve<T, M>(W + 1, roww, sm.sep, y, p.err);
        }
#pragma unroll
        for (int k = 0; k < M; ++k)
            if (!(j0 + k < W)) y[k] = 0.f;
        // dh = y: the values outside the window (and the closing row) are taken as 0
        sts4(dha + j0 + 4, y);
    }
    __syncthreads();
    if (BC == BC_TRANSMISSIVE && (win.lend || win.rend)) {  // (uniform over the CTA)
        if (tid == 0 && win.lend) dha[3] = dha[4];
        if (tid == 0 && win.rend) dha[W + 4] = dha[W + 3];
        __syncthreads();
    }

    // truncation bound of this window: rho*^HB <= 2^-30
    if (tid == 0) {
        const bool cut = BC == BC_PERIODIC || !(win.lend && win.rend);
        const float K = __uint_as_float(sm.kmax), kap = fminf(__uint_as_float(sm.kmin), K);
        if (cut && K > 0.f) {
            const float B = 1.f + K + kap;
            const float rho = 2.f * K / (B + sqrtf(fmaxf(B * B - 4.f * kap * K, 0.f)));
            if ((float)Gm::HB * __log2f(rho) > -30.f) bad |= HSGN_DEV_ERR_TRUNCATION;
        }
    }
    __syncthreads();

    // ---- 4a. face mass fluxes (divided by dx) of the tile's faces, each evaluated
    //          once: thread t takes the window faces jf = 4t .. 4t + 3 (face jf
    //          between rows jf - 1 and jf) that belong to the tile, jf = lo .. lo + sp;
    //          at a tile face both rows come from the shared mini solve
    //   G = tau/(2dx) (q^dag_L + q^dag_R) - lambda tau^2/dx^2 delta_face (m^dag_R - m^dag_L)
    //       - tau^2/dx^2 beta_face (hbar_R - hbar_L)
    const int lo = win.lo, sp = win.sp;
    float* const Gt = sm.rb;   // face jf at jf - lo
    float* const dQa = sm.mb;  // momentum increment of window row r at r
    if (j0 + 3 >= lo && j0 <= lo + sp) {
        float QB[8], QA[8], B[8];
        lds4(sm.qb + j0, QB); lds4(sm.qb + j0 + 4, QB + 4);
        lds4(dqa + j0, QA); lds4(dqa + j0 + 4, QA + 4);
        lds4(bea + j0, B); lds4(bea + j0 + 4, B + 4);
        float DW[6];  // dh of the rows j0 - 1 .. j0 + 4
        DW[0] = dha[j0 + 3];
        lds4(dha + j0 + 4, DW + 1);
        DW[5] = dha[j0 + 8];
        float DE[WB ? 1 : 8], MA[WB ? 1 : 8], DM[WB ? 1 : 8], DH[WB ? 1 : 8], PV[WB ? 8 : 1];
        if constexpr (WB) {
            lds4(Psi + j0, PV); lds4(Psi + j0 + 4, PV + 4);
        } else {
            lds4(dea + j0, DE); lds4(dea + j0 + 4, DE + 4);
            lds4(dma + j0, MA); lds4(dma + j0 + 4, MA + 4);
            lds4(sm.Dm + j0, DM); lds4(sm.Dm + j0 + 4, DM + 4);
            lds4(sm.Dh + j0, DH); lds4(sm.Dh + j0 + 4, DH + 4);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = j0 + e - lo;  // tile face j = 0 .. sp
            if (j >= 0 && j <= sp) {
                float dL = DW[e], dR = DW[e + 1];
                if (j == 0 && lface) { dL = sm.bnd[0][0]; dR = sm.bnd[0][1]; }
                if (j == sp && rface) { dL = sm.bnd[1][0]; dR = sm.bnd[1][1]; }
                const float qsum = (QB[e + 2] + QB[e + 3]) + (QA[e] + QA[e + 1]);
                // (rounded explicitly: a tile face's flux is evaluated by both
                // tiles beside it, at different positions among the four faces)
                float G;
                if constexpr (WB) {
                    // G = tau/(2dx) (q^dag_L + q^dag_R) - tau^2/dx^2 (Psi_f + beta_face (dh_R - dh_L))
                    G = fmaf(-Cc, fmaf(0.5f * (B[e] + B[e + 1]), dR - dL, PV[e + 2]),
                             __fmul_rn(fq, qsum));
                } else {
                    const float dmf = DM[e + 2] + (MA[e + 1] - MA[e]);
                    const float dhf = DH[e + 2] + (dR - dL);
                    G = fmaf(-__fmul_rn(hCc, B[e] + B[e + 1]), dhf,
                             fmaf(-__fmul_rn(hfd, DE[e] + DE[e + 1]), dmf,
                                  __fmul_rn(fq, qsum)));
                }
                if (!isfinite(G)) bad |= HSGN_DEV_ERR_NONFINITE;
                Gt[j] = G;
            }
        }
        // momentum increment of the rows 4t .. 4t + 3 (those of the tile are used)
        float dq4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float dhL = DW[k], dhC = DW[k + 1], dhR = DW[k + 2];
            if constexpr (WB) {
                // q = q^dag - tau/(2dx) (F_{i+1/2} + F_{i-1/2}), F = Psi + beta_face (dh jump)
                const float Fp = fmaf(0.5f * (B[k + 1] + B[k + 2]), dhR - dhC, PV[k + 3]);
                const float Fl = fmaf(0.5f * (B[k] + B[k + 1]), dhC - dhL, PV[k + 2]);
                dq4[k] = QA[k + 1] - fq * (Fp + Fl);
            } else {
                // q: tau/(2dx) beta (hbar_{i+1} - hbar_{i-1}), lambda tau/(2dx) delta (m^dag_{i+1} - m^dag_{i-1})
                const float dhc = (DH[k + 2] + DH[k + 3]) + (dhR - dhL);  // faces r-1/2, r+1/2
                const float dmc = (DM[k + 2] + DM[k + 3]) + (MA[k + 2] - MA[k]);
                dq4[k] = QA[k + 1] - fq * B[k + 1] * dhc - lam * fq * DE[k + 1] * dmc;
            }
        }
        sts4(dQa + j0, dq4);
    }
    __syncthreads();

    // ---- 4b. back-substitution of the tile rows
    float umax = 0.f;
    // the tile's cells and faces from its first cell: 32-bit offsets t
    const int64_t t0 = win.t0;
    const float2* const U0t = U0 + t0;
    const float2* const U1t = U1 + t0;
    const float2* const U2t = U2 + t0;
    const float2* const U3t = U3 + t0;
    const float* const G1t = G1 + t0;  // face left of cell t at t, right of it at t + 1
    float* const dq1t = dq1p + t0;
    float* const dm1t = dm1p + t0;
    float* const dr1t = dr1p + t0;
    // stage 1 writes the tile's faces 1 .. sp of G1 here and face 0 only at a
    // transmissive left domain end (face i+1/2 of cell i at i + 1; every other
    // face 0 is the previous tile's face sp)
    float* const G1wt = G1w + t0;
    if (!two && BC == BC_TRANSMISSIVE && t0 == 0 && tid == 0) G1wt[0] = Gt[0];
    float2* const o0t = two ? p.out[0] + cell0 + t0 : nullptr;
    float2* const o1t = two ? p.out[1] + cell0 + t0 : nullptr;
    float2* const o2t = two ? p.out[2] + cell0 + t0 : nullptr;
    float2* const o3t = two ? p.out[3] + cell0 + t0 : nullptr;
    // periodic face -1/2 is face n-1/2 (for the first cell of the first tile)
    const bool wrap0 = BC == BC_PERIODIC && t0 == 0;
    for (int t = tid; t < sp; t += T) {
        const int r = lo + t;            // window row
        const float dhC = dha[r + 4], dmC = dma[r + 1], dQ = dQa[r];
        // base depth (rounded) and P0 = h_b^2 - m_b of this cell
        const float2 h0 = U0t[t], m0 = U2t[t];
        const float hf = h0.x;
        // (h^2 - m)^n: hi^2 = p + e exactly; p - m.hi is exact for m close to h^2
        const float pp = __fmul_rn(hf, hf);
        const float pe = fmaf(hf, hf, -pp);
        float hbf = hf;
        float P0 = __fadd_rn(__fsub_rn(pp, m0.x), fmaf(2.f * hf, h0.y, __fsub_rn(pe, m0.y)));
        float g1l = 0.f, g1r = 0.f;
        if constexpr (two) {
            g1l = (wrap0 && t == 0) ? G1[n] : G1t[t];
            g1r = G1t[t + 1];
            const float dh1 = g1l - g1r, dm1 = dm1t[t];
            hbf = fmaf(wb1, dh1, hf);
            P0 = fmaf(wb1, fmaf(dh1, fmaf(wb1, dh1, 2.f * hf), -dm1), P0);
        }
        const float hbar = hbf + dhC;
        const float P = fmaf(dhC, 2.f * hbf + dhC, P0);  // hbar^2 - m_b
        const float E = P - dmC;                          // hbar^2 - m^
        const float h2 = hbar * hbar;
        const float iDen = rcpa(h2 + c_lt2);
        const float dR = fmaf(c_ltau * E, iDen, dra[r + 1]);
        const float dM = P - E * h2 * iDen;
        unsigned b2 = 0;
        if (!pos_finite(hbar)) b2 |= HSGN_DEV_ERR_DEPTH;
        if (!isfinite(dQ) || !isfinite(dM) || !isfinite(dR)) b2 |= HSGN_DEV_ERR_NONFINITE;
        bad |= b2;
        if (!two) {
            dq1t[t] = dQ;
            dm1t[t] = dM;
            dr1t[t] = dR;
            G1wt[t + 1] = Gt[t + 1];
        } else {
            const float Tp = fmaf(wb1, g1r, Gt[t + 1]);
            const float Tm = fmaf(wb1, g1l, Gt[t]);
            float d, de;
            two_sum(Tm, -Tp, d, de);  // exact Tm - Tp
            o0t[t] = df_add(h0, d, de);
            o1t[t] = df_add1(U1t[t], fmaf(wb1, dq1t[t], dQ));
            o2t[t] = df_add1(m0, fmaf(wb1, dm1t[t], dM));
            o3t[t] = df_add1(U3t[t], fmaf(wb1, dr1t[t], dR));
            if (p.track_speed && !b2) umax = fmaxf(umax, fabsf(sm.qb[r + 3] + dQ) * rcpa(hbar));
        }
    }
    if (bad) flag_error(p.err, bad);
    if (p.track_speed && two) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, o));
        if ((tid & 31) == 0 && umax > 0.f)
            atomicMax(reinterpret_cast<unsigned long long*>(spd_out),
                      (unsigned long long)__double_as_longlong(f64_of(umax)));
    }
}

// State conversions of the windowed path (off the stepping path).
__global__ void k_df_from_f64(int64_t n, const double* __restrict__ src, float2* __restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = df_of(src[i]);
}

__global__ void k_f64_from_df(int64_t n, const float2* __restrict__ src, double* __restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = src[i];
        dst[i] = (double)v.x + (double)v.y;  // exact: the pair has 48 significant bits
    }
}

// k_speeds (hsgn_kernels.cuh) for a double-float state.
__global__ void k_speeds_df(int64_t n, const float2* h, const float2* q, const float2* m, double g,
                            double lam, double* out, unsigned* err) {
    double um = 0.0, nm = 0.0;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 hv = h[i], qv = q[i], mv = m[i];
        const double hh = (double)hv.x + (double)hv.y;
        if (!(hh > 0.0)) {
            bad = true;
            continue;
        }
        const double u = fabs(((double)qv.x + (double)qv.y) / hh);
        const double e = ((double)mv.x + (double)mv.y) / (hh * hh);
        const double nu = u + sqrt(g * hh + (lam / 3.0) * e * e);
        um = fmax(um, u);
        nm = fmax(nm, nu);
    }
    if (bad) flag_error(err, HSGN_DEV_ERR_DEPTH);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        um = fmax(um, __shfl_xor_sync(0xffffffffu, um, o));
        nm = fmax(nm, __shfl_xor_sync(0xffffffffu, nm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (um > 0.0)
            atomicMax(reinterpret_cast<unsigned long long*>(out),
                      (unsigned long long)__double_as_longlong(um));
        if (nm > 0.0)
            atomicMax(reinterpret_cast<unsigned long long*>(out + 1),
                      (unsigned long long)__double_as_longlong(nm));
    }
}

// Global Rusanov speed max |u| of a double-float state in single precision,
// u = |q.hi| / h.hi rounded once: the stage kernels use the speed in single
// precision. Cheaper than k_speeds_df, whose double-precision divisions and
// square root run on the slow FP64 pipe; that kernel stays for the time-step
// rule. out must be zero on entry.
__global__ void k_umax_df(int64_t n, const float2* __restrict__ h, const float2* __restrict__ q,
                          double* out, unsigned* err) {
    float um = 0.f;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float hv = h[i].x;
        if (!pos_finite(hv)) {
            bad = true;
            continue;
        }
        um = fmaxf(um, __fdiv_rn(fabsf(q[i].x), hv));
    }
    if (bad) flag_error(err, HSGN_DEV_ERR_DEPTH);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) um = fmaxf(um, __shfl_xor_sync(0xffffffffu, um, o));
    if ((threadIdx.x & 31) == 0 && um > 0.f)
        atomicMax(reinterpret_cast<unsigned long long*>(out),
                  (unsigned long long)__double_as_longlong(f64_of(um)));
}

// k_umax_df per instance of a batch: one CTA per instance, out[k] = max |u|.
__global__ void __launch_bounds__(256) k_umax_batched_df(const InstInfo* inst, const float2* h,
                                                         const float2* q, double* out,
                                                         unsigned* err) {
    __shared__ float ru[8];
    const InstInfo I = inst[blockIdx.x];
    float um = 0.f;
    bool bad = false;
    for (int64_t i = I.cell0 + threadIdx.x; i < I.cell0 + I.n; i += blockDim.x) {
        const float hv = h[i].x;
        if (!pos_finite(hv)) {
            bad = true;
            continue;
        }
        um = fmaxf(um, __fdiv_rn(fabsf(q[i].x), hv));
    }
    if (bad) flag_error(err, HSGN_DEV_ERR_DEPTH);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) um = fmaxf(um, __shfl_xor_sync(0xffffffffu, um, o));
    if ((threadIdx.x & 31) == 0) ru[threadIdx.x >> 5] = um;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) um = fmaxf(um, ru[w]);
        out[blockIdx.x] = f64_of(um);
    }
}

// k_speeds_batched (hsgn_mixed.cuh) for a batch held as double-float pairs:
// per-instance max |u| and max nu, one CTA per instance.
__global__ void __launch_bounds__(256) k_speeds_batched_df(const InstInfo* inst, const float2* h,
                                                           const float2* q, const float2* m,
                                                           double g, double* out_u, double* out_nu,
                                                           unsigned* err) {
    __shared__ double ru[8], rn[8];
    const InstInfo I = inst[blockIdx.x];
    double um = 0.0, nm = 0.0;
    bool bad = false;
    for (int64_t i = I.cell0 + threadIdx.x; i < I.cell0 + I.n; i += blockDim.x) {
        const float2 hv = h[i], qv = q[i], mv = m[i];
        const double hh = (double)hv.x + (double)hv.y;
        if (!pos_finite(hh)) {
            bad = true;
            continue;
        }
        const double u = fabs(((double)qv.x + (double)qv.y) / hh);
        const double e = ((double)mv.x + (double)mv.y) / (hh * hh);
        um = fmax(um, u);
        nm = fmax(nm, u + sqrt(g * hh + (I.lam / 3.0) * e * e));
    }
    if (bad) flag_error(err, HSGN_DEV_ERR_DEPTH);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        um = fmax(um, __shfl_xor_sync(0xffffffffu, um, o));
        nm = fmax(nm, __shfl_xor_sync(0xffffffffu, nm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        ru[threadIdx.x >> 5] = um;
        rn[threadIdx.x >> 5] = nm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            um = fmax(um, ru[w]);
            nm = fmax(nm, rn[w]);
        }
        out_u[blockIdx.x] = um;
        if (out_nu) out_nu[blockIdx.x] = nm;
    }
}

}  // namespace hsgn
