// hsgn_dfstage.cuh -- the FP64-class stage in one launch: double-float
// arithmetic on the single-precision pipe (sm_103a).
//
// One stage of Sec. 4.2, eq. (GN_hyp_eq_semi_fully_discrete), inside the
// two-stage tableau of Sec. 3.2 (efficient form), computed with every value a
// double-float pair (hsgn_dfloat.cuh: 48-bit significand, each operation a
// few single-precision instructions; sm_103a issues 58 single-precision
// operations per double-precision one). Same tiling as the windowed mixed
// stage (hsgn_fused.cuh): CTA p owns the tile [t0, t0 + sp) of rows and solves
// the depth system on the window [t0 - HWt, t0 + sp + HWt), dropping the
// coupling beyond it. The overlap HWt (48 .. 96 rows) is a launch parameter
// that the host sets from the coupling stage 2 recorded; the decay bound of
// the truncation is checked per CTA against 2^-50 (the pairs carry about
// 2^-47), a tile whose window misses it is redone in pieces with the widest
// overlap HW, and beyond that the stage reports HSGN_ERR_TRUNCATION. The flat
// bottom and the well-balanced bottom form (WB) share the kernel.
//
// Increment form, as in the mixed stage but with the increments kept as pairs:
//  * stage 1 (U_b = U_l = U^n) writes dU1 = U_I^(1) - U^n;
//  * stage 2 forms U_l = U^n + (c/gamma) dU1 and U_b = U^n + ((1-gamma)/gamma) dU1
//    on load and writes U^{n+1} = U_b + dU2 into the other state buffer;
//  * the depth system A dh = d - A h_b is solved for the increment dh, so its
//    rounding scales with the increment rather than with the depth.
// Accuracy choices (each measured against the FP64 oracle: without them the
// h w error per stage was 4e-13, with them under 1e-13):
//  * differences of neighbouring state values (the U_b parts of q^dag and
//    m^dag, h_b, h_l, the bottom, pi) use the cancellation-accurate sum add_acc;
//    so do the fluxes of h eta and h w, the face terms Phi and the dm^
//    differences inside them, whose errors reach h w through the relaxation's
//    lambda tau. The plain pair sum add_u (rounding about 2^-47 of its
//    operands) takes the differences that reach the depth system only through
//    tau/(2dx) twice (the flux of q; the dq increments of the rows) or reach
//    only q (the dh and dm^ increments of the back-substitution);
//  * hbar^2 - m_b = (h_b^2 - m_b) + dh (2 h_b + dh), with h_b^2 - m_b formed
//    exactly (sq_minus), so that the relaxation update
//    (hw)bar = r_b + dr + lambda tau (hbar^2 - m^)/(hbar^2 + lambda tau^2),
//    which amplifies errors in hbar^2 - m by lambda tau, sees no rounding of hbar.
// Mass: hbar = h_b + dh with dh from the window solve (no flux form): the
// pairs' rounding of dh is 2^-47 of the increment, far below the 1e-13
// conservation bound.
#pragma once

#include "hsgn_fused.cuh"
#include "hsgn_dfloat.cuh"

namespace hsgn {

// The block elimination of hsgn_tridiag.cuh instantiated for pairs needs these.
__device__ __forceinline__ bool pos_finite(dfl x) { return pos_finite(x.hi); }
__device__ __forceinline__ float hi_of(dfl x) { return x.hi; }
__device__ __forceinline__ dfl shfl_up_d(dfl x, int s) {
    return dfl(__shfl_up_sync(0xffffffffu, x.hi, s), __shfl_up_sync(0xffffffffu, x.lo, s));
}
__device__ __forceinline__ dfl shfl_down_d(dfl x, int s) {
    return dfl(__shfl_down_sync(0xffffffffu, x.hi, s), __shfl_down_sync(0xffffffffu, x.lo, s));
}
__device__ __forceinline__ dfl shfl_xor_d(dfl x, int s) {
    return dfl(__shfl_xor_sync(0xffffffffu, x.hi, s), __shfl_xor_sync(0xffffffffu, x.lo, s));
}

// Single-precision versions of the pair helpers (the FP32-flux split runs the
// flux and coefficient phases on floats).
__device__ __forceinline__ float scale(float a, float pow2) { return a * pow2; }
__device__ __forceinline__ float sub_acc(float a, float b) { return a - b; }
__device__ __forceinline__ float add_f(float a, float x) { return a + x; }
__device__ __forceinline__ float dabs(float a) { return fabsf(a); }
__device__ __forceinline__ float dmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float add_u(float a, float b) { return a + b; }
__device__ __forceinline__ float sub_u(float a, float b) { return a - b; }
__device__ __forceinline__ dfl to_dfl(dfl x) { return x; }
__device__ __forceinline__ dfl to_dfl(float x) { return dfl(x); }
__device__ __forceinline__ dfl as_R(dfl x, dfl) { return x; }
__device__ __forceinline__ float as_R(dfl x, float) { return f_add(x.hi, x.lo); }

// Number type of the flux and coefficient phases of k_df_stage.
template <bool F32>
struct FluxReal {
    using type = dfl;
};
template <>
struct FluxReal<true> {
    using type = float;
};

// A shared-memory array of pairs, high and low parts in separate planes so
// that four consecutive entries are two 128-bit loads (lanes 16 bytes apart:
// no bank conflicts).
template <int NC>
struct DArr {
    float hi[NC], lo[NC];
    __device__ __forceinline__ dfl get(int i) const { return dfl(hi[i], lo[i]); }
    __device__ __forceinline__ void set(int i, dfl v) {
        hi[i] = v.hi;
        lo[i] = v.lo;
    }
    // entries i .. i+3 (i a multiple of 4)
    __device__ __forceinline__ void get4(int i, dfl* v) const {
        const float4 h = *reinterpret_cast<const float4*>(hi + i);
        const float4 l = *reinterpret_cast<const float4*>(lo + i);
        v[0] = dfl(h.x, l.x);
        v[1] = dfl(h.y, l.y);
        v[2] = dfl(h.z, l.z);
        v[3] = dfl(h.w, l.w);
    }
    __device__ __forceinline__ void set4(int i, const dfl* v) {
        *reinterpret_cast<float4*>(hi + i) = make_float4(v[0].hi, v[1].hi, v[2].hi, v[3].hi);
        *reinterpret_cast<float4*>(lo + i) = make_float4(v[0].lo, v[1].lo, v[2].lo, v[3].lo);
    }
};

// Four consecutive entries (i a multiple of 4) as pairs or as their high parts.
template <int NC>
__device__ __forceinline__ void ld4(const DArr<NC>& a, int i, dfl* v) { a.get4(i, v); }
template <int NC>
__device__ __forceinline__ void ld4(const DArr<NC>& a, int i, float* v) {
    const float4 h = *reinterpret_cast<const float4*>(a.hi + i);
    v[0] = h.x; v[1] = h.y; v[2] = h.z; v[3] = h.w;
}
template <int NC>
__device__ __forceinline__ void ld1(const DArr<NC>& a, int i, dfl& v) { v = a.get(i); }
template <int NC>
__device__ __forceinline__ void ld1(const DArr<NC>& a, int i, float& v) { v = a.hi[i]; }
template <int NC>
__device__ __forceinline__ void st1(DArr<NC>& a, int i, dfl v) { a.set(i, v); }
template <int NC>
__device__ __forceinline__ void st1(DArr<NC>& a, int i, float v) { a.set(i, dfl(v)); }
template <int NC>
__device__ __forceinline__ void st4(DArr<NC>& a, int i, const dfl* v) { a.set4(i, v); }
template <int NC>
__device__ __forceinline__ void st4(DArr<NC>& a, int i, const float* v) {
    const dfl d[4] = {dfl(v[0]), dfl(v[1]), dfl(v[2]), dfl(v[3])};
    a.set4(i, d);
}

// Window of the tile rows [t0, t0 + sp) with overlap HW (window_of for a run
// of rows that need not start at a multiple of the tile size).
template <int BC>
__host__ __device__ inline Window window_at(int64_t t0, int sp, int64_t n, int HW) {
    Window w;
    w.t0 = t0;
    w.sp = sp;
    if (BC == BC_PERIODIC) {
        w.wl = t0 - HW;
        w.W = sp + 2 * HW;
        w.lend = w.rend = false;
    } else {
        w.wl = t0 - HW < 0 ? 0 : t0 - HW;
        const int64_t wr = t0 + sp + HW > n ? n : t0 + sp + HW;
        w.W = (int)(wr - w.wl);
        w.lend = w.wl == 0;
        w.rend = wr == n;
    }
    w.lo = (int)(t0 - w.wl);
    return w;
}

// Rows between a kept row and the window edge that bring the decay bound
// rho*^rows under 2^-50, from log2 rho* (0xFFFF when the coupling does not decay).
__host__ __device__ inline unsigned df_rows_needed(float lg) {
    if (!(lg < 0.f)) return 0xFFFFu;
    const float r = ceilf(-50.f / lg);
    return r < 65535.f ? (unsigned)r : 0xFFFFu;
}

// Geometry: T threads, M = 4 rows per thread, overlap HW (as FusedGeom).
template <int T, int M, int HW>
struct DfGeom {
    static constexpr int R = T * M - 2;          // window rows (one identity row closes it)
    static constexpr int S = R - 2 * HW;         // largest tile
    static constexpr int HB = HW - 1;            // rows between a kept row and the window edge
    static constexpr int NC = (R + 6 + 3) & ~3;  // cells -3 .. W+2 at c + 3
    static_assert(M == 4, "four cells per thread");
    static_assert(S > 0, "overlap too wide for the window");
};

// The bottom of the window (bottom form only).
template <int NC, bool WB>
struct DfWb {
    DArr<NC> bb;
};
template <int NC>
struct DfWb<NC, false> {};

// Shared memory. Cell c of the window at c + 3 in the state arrays, at c + 1
// in the per-cell arrays; face jf (between window cells jf - 2 and jf - 1) at
// jf. After the cell phase the U_l arrays and the flux arrays are reused:
// flat: dq -> hl, dm^ -> ql, dr -> ml, beta -> rl, delta -> fq; dh of row r
// -> fm at r + 4. Bottom form (h_l stays in hl for the face forces): dq -> ql,
// dm^ -> ml, dr -> rl, beta -> fq, pi -> fm, p~ -> fr; after the solve the
// face forces Psi -> fm (face jf at jf) and dh -> fr.

template <int T, int M, int HW, bool WB = false>
struct DfShared {
    static constexpr int NC = DfGeom<T, M, HW>::NC;
    DArr<NC> hl, ql, ml, rl;  // U_l
    DArr<NC> hb, qb, mb, rb;  // U_b
    DArr<NC> fq, fm, fr;      // twice the Rusanov fluxes of q, h eta, h w
    DfWb<NC, WB> wb;          // the bottom b, cells -3 .. W+2 at c + 3
    SepShared<T, dfl> sep;
    unsigned kmax, kmin;      // bits of max / min tau^2 beta / dx^2 (positive floats order as integers)
    dfl kc[7];                // per-step constants of an adaptive step
};

// The constants of a stage that depend on the time step (tau = gamma dt).
struct DfStepConst {
    dfl tau, lt2, ltau, fq, lfq, Cc, fd;
};

__device__ __forceinline__ DfStepConst df_step_const(double dt, double dx, double lam) {
    const double tau = (1.0 - 1.0 / sqrt(2.0)) * dt;  // gamma dt, Sec. 3.2
    DfStepConst k;
    k.tau = dfl_of(tau);
    k.lt2 = dfl_of(lam * tau * tau);
    k.ltau = dfl_of(lam * tau);
    k.fq = dfl_of(tau / (2.0 * dx));
    k.lfq = dfl_of(lam * tau / (2.0 * dx));
    k.Cc = dfl_of(tau * tau / (dx * dx));
    k.fd = dfl_of(lam * tau * tau / (dx * dx));
    return k;
}

// sqrt(a) of a positive pair: the single-precision root refined by one
// Newton step, s + (a - s^2)/(2 s) with s^2 formed exactly.
__device__ __forceinline__ dfl dsqrt(dfl a) {
    const float s = sqrtf(a.hi);
    const float p = f_mul(s, s);
    const float pe = f_fma(s, s, -p);
    const float r = f_add(f_sub(f_sub(a.hi, p), pe), a.lo);
    return dfl_make(s, f_mul(r, f_rcp(f_add(s, s))));
}

struct DfParams {
    int64_t n;
    int32_t stage;        // 1: writes dU1; 2: writes U^{n+1} to out
    int32_t local_speed;  // Rusanov speed max(|u^L|, |u^R|) per face instead of *speed
    int32_t track_speed;  // stage 1 clears *speed_next, stage 2 folds max |u^{n+1}| into it
    int32_t S;            // tile rows (one CTA per tile)
    // overlap of a tile's window, HWt <= HW of the kernel; a tile whose window
    // misses the decay bound with HWt < HW is redone in pieces with overlap HW
    int32_t HWt;
    int32_t slots;        // co-resident CTAs of the launch (next-wave L2 prefetch; 0: none)
    unsigned* need_out;   // stage 1 clears it, stage 2 records the overlap rows its
                          // windows needed (df_rows_needed; or nullptr)
    // bottom form: the bottom b per cell (pairs), and wb1 - wl1, the weight of
    // m_b - m_l = (wb1 - wl1) dm1 in stage 2
    const float2* bathy;
    dfl wmd;
    // constants of the stage as pairs (tau = gamma dt): tau, lambda tau^2,
    // lambda tau, tau/(2 dx), lambda tau/(2 dx), tau^2/dx^2, lambda tau^2/dx^2,
    // g, lambda, lambda/3, 1/3, and the stage-2 weights c/gamma, (1-gamma)/gamma
    dfl tau, lt2, ltau, fq, lfq, Cc, fd, g, lam, lam3, third, wl1, wb1;
    // per-step time step (adaptive != 0): stage 1 takes dt = min(cfl dx / nu_max,
    // mcfl dx / u_max) from speed[0] = max |u| and speed[1] = max nu of U^n, writes it
    // to dtp[0] and adds it to dtp[1]; stage 2 reads dtp[0]; both derive the
    // constants above that depend on dt themselves; stage 2 folds max nu of
    // U^{n+1} into speed_next[1] (Sec. 3.3 eq. (eq:MCFL), Sec. 5)
    int32_t adaptive;
    double cfl, mcfl, dx, lam_d, g_d;
    double* dtp;
    const float2* U[4];   // U^n (pairs)
    float2* D1[4];        // stage-1 increments dU1 (written by stage 1, read by stage 2)
    float2* out[4];       // U^{n+1} (stage 2; not aliased with U)
    const double* speed;  // global Rusanov speed of the step
    double* speed_next;   // max |u^{n+1}|
    unsigned* err;
};

// F32 selects the precision split of the mixed FP64-solve form
// (HSGN_MIXED | HSGN_DOUBLE_FLOAT): fluxes, starred increments and coefficients
// in single precision, rows, depth solve, back-substitution and the
// accumulation of the state in pairs.
// WB selects the well-balanced bottom form (reading R7 of the oracle): the
// (h eta) equation's bottom source -(3/2) tau q_l b_x in m^dag, and in place of
// the delta term the face forces
//   Psi_f = Phi_f + beta_f (h_b jump) = g hbar_f (h_l + b jump) + (pi jump)
//           + (3/2) p~_f (b jump) - beta_f (h_l - h_b jump),
// p~ = (lambda/3)(1 - eta/h), pi = eta p~ + lambda alpha (m^dag b_1 - m_l)
// (p^ of the scheme less g h^2/2, whose jump is g hbar_f (h_l jump)), with
// m^dag b_1 - m_l = (h^2 (m_b - m_l + dm^) + lambda tau^2 (h^2 - m_l)) / (h^2 + lambda tau^2)
// and m_b - m_l = (wb1 - wl1) dm1 taken from the stage-1 increment; the
// momentum then takes q = q^dag - tau/(2dx) (F_{i+1/2} + F_{i-1/2}) with
// F_f = Psi_f + beta_f (dh jump).
template <int T, int M, int HW, int BC, int STAGE, bool F32 = false, bool WB = false>
__global__ void __launch_bounds__(T, 2) k_df_stage(const DfParams p) {
    static_assert(STAGE == 1 || STAGE == 2, "two stages");
    static_assert(!(F32 && WB), "the bottom form computes every phase in pairs");
    using Gm = DfGeom<T, M, HW>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<DfShared<T, M, HW, WB>*>(smem_raw);
    constexpr bool two = STAGE == 2;
    const int tid = threadIdx.x;
    const int64_t n = p.n;
    if (p.track_speed && !two && blockIdx.x == 0 && tid == 0) {
        p.speed_next[0] = 0.0;
        if (p.adaptive) p.speed_next[1] = 0.0;
    }
    if (!two && p.need_out && blockIdx.x == 0 && tid == 0) *p.need_out = 0u;
    const int S0 = p.S;
    const int HW0 = p.HWt < HW ? p.HWt : HW;
    const int64_t tile0 = (int64_t)blockIdx.x * S0;
    const int sp0 = (int)(n - tile0 < S0 ? n - tile0 : S0);
    // the time step: fixed (from the parameters) or from the CFL rule
    DfStepConst kc{p.tau, p.lt2, p.ltau, p.fq, p.lfq, p.Cc, p.fd};
    if (p.adaptive) {
        if (tid == 0) {
            double dt;
            if (!two) {
                const double u = p.speed[0], nu = p.speed[1];
                dt = p.cfl * p.dx / nu;
                if (p.mcfl > 0.0 && u > 0.0 && u * dt / p.dx > p.mcfl) dt = p.mcfl * p.dx / u;
                if (blockIdx.x == 0) {
                    p.dtp[0] = dt;
                    p.dtp[1] += dt;
                }
            } else {
                dt = p.dtp[0];
            }
            const DfStepConst k = df_step_const(dt, p.dx, p.lam_d);
            sm.kc[0] = k.tau; sm.kc[1] = k.lt2; sm.kc[2] = k.ltau; sm.kc[3] = k.fq;
            sm.kc[4] = k.lfq; sm.kc[5] = k.Cc; sm.kc[6] = k.fd;
        }
        __syncthreads();
        kc = DfStepConst{sm.kc[0], sm.kc[1], sm.kc[2], sm.kc[3], sm.kc[4], sm.kc[5], sm.kc[6]};
    }

    unsigned bad = 0;
    dfl umax(0.f), numax(0.f);
    // pass -1: the tile with the overlap HW0; if its window misses the decay
    // bound with HW0 < HW, passes 0 .. npieces-1 redo the tile in pieces of
    // pr rows with the wide overlap HW
    int npieces = 0, pr = 0;
    for (int piece = -1;;) {
    if (piece >= 0) __syncthreads();  // (the previous pass's shared reads are done)
    const int HWc = piece < 0 ? HW0 : HW;
    const Window win = piece < 0 ? window_at<BC>(tile0, sp0, n, HW0)
                                 : window_at<BC>(tile0 + (int64_t)piece * pr,
                                                 min(pr, sp0 - piece * pr), n, HW);
    const int W = win.W;
    const int64_t wl = win.wl;
    if (tid == 0) {
        sm.kmax = 0u;
        sm.kmin = 0x7F7FFFFFu;
    }

    // ---- 0. window cells -3 .. W+2 (index c + 3): U_l and U_b (stage 2:
    //         formed from U^n and dU1 with the efficient-form weights)
    {
        const bool inner = inner_window(wl, W, n);
        constexpr int NL = (Gm::R + 6 + T - 1) / T;
#pragma unroll
        for (int it = 0; it < NL; ++it) {
            const int j = tid + it * T;
            if (j < W + 6) {
                const int64_t gi = inner ? wl - 3 + j : cell_at<BC>(wl - 3 + j, n);
                DArr<Gm::NC>* const L[4] = {&sm.hl, &sm.ql, &sm.ml, &sm.rl};
                DArr<Gm::NC>* const B[4] = {&sm.hb, &sm.qb, &sm.mb, &sm.rb};
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float2 a = __ldg(p.U[v] + gi);
                    const dfl u(a.x, a.y);
                    if constexpr (two) {
                        const float2 d = __ldg(p.D1[v] + gi);
                        const dfl dv(d.x, d.y);
                        L[v]->set(j, fma_u(p.wl1, dv, u));
                        B[v]->set(j, fma_u(p.wb1, dv, u));
                    } else {
                        L[v]->set(j, u);
                        B[v]->set(j, u);
                    }
                }
                if constexpr (WB) {
                    const float2 b = __ldg(p.bathy + gi);
                    sm.wb.bb.set(j, dfl(b.x, b.y));
                }
            }
        }
        // L2 prefetch of the window of the tile that the next wave of CTAs
        // starts on this slot (tile blockIdx.x + slots: CTAs are dispatched in
        // index order as slots free up), one 128-byte line (16 pairs) per
        // thread and array over the cells of that window inside [0, n)
        constexpr int PF = (Gm::R + 6 + 15) / 16;
        if (piece < 0 && p.slots > 0 && tid < PF) {
            const int64_t ts = (int64_t)blockIdx.x + p.slots;
            if (ts < (int64_t)gridDim.x) {
                const int64_t nt0 = ts * S0;
                const Window ws = window_at<BC>(nt0, (int)(n - nt0 < S0 ? n - nt0 : S0), n, HW0);
                const int64_t c0 = ws.wl - 3 < 0 ? 0 : ws.wl - 3;
                const int64_t c1 = ws.wl + ws.W + 3 > n ? n : ws.wl + ws.W + 3;
                const int64_t c = c0 + 16 * (int64_t)tid;
                if (c < c1) {
#pragma unroll
                    for (int v = 0; v < 4; ++v) prefetch_l2(p.U[v] + c);
                    if constexpr (two) {
#pragma unroll
                        for (int v = 0; v < 4; ++v) prefetch_l2(p.D1[v] + c);
                    }
                    if constexpr (WB) prefetch_l2(p.bathy + c);
                }
            }
        }
    }
    __syncthreads();

    const int j0 = 4 * tid;

    // ---- A. twice the Rusanov fluxes of U_l (Sec. 4.1) at the faces
    //         jf = 4t .. 4t+3 (face jf between window cells jf - 2 and jf - 1,
    //         reconstructed from the cells at index jf .. jf + 3): centred
    //         unlimited linear reconstruction of (h, q, h eta, h w),
    //         u = q/h on either side, 2F = u^L X^L + u^R X^R - s (X^R - X^L)
    //         (a cell's quarter centred difference serves the faces on both of
    //         its sides; the flux is taken as (u^L + s) X^L + (u^R - s) X^R, the
    //         two speed sums shared by the three variables).
    //         R is the number type of phases A and B: pairs, or single
    //         precision for the FP32-flux split (F32).
    using R = typename FluxReal<F32>::type;
    const R spd = p.local_speed ? R(0.f) : as_R(dfl_of(*p.speed), R());
    {
        // the quarter centred difference of cell c = 1 .. 5 of the 8 loaded
        auto quarter = [](const R* X, R* D) {
#pragma unroll
            for (int c = 1; c <= 5; ++c) D[c - 1] = scale(sub_u(X[c + 1], X[c - 1]), 0.25f);
        };
        R wL[4], wR[4];  // u^L + s, u^R - s
        {
            R H[8], Q[8], DH[5], DQ[5];
            ld4(sm.hl, j0, H);
            ld4(sm.hl, j0 + 4, H + 4);
            ld4(sm.ql, j0, Q);
            ld4(sm.ql, j0 + 4, Q + 4);
            quarter(H, DH);
            quarter(Q, DQ);
            R Fq[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const R hL = add_u(H[e + 1], DH[e]), hR = sub_u(H[e + 2], DH[e + 1]);
                const R qL = add_u(Q[e + 1], DQ[e]), qR = sub_u(Q[e + 2], DQ[e + 1]);
                if (j0 + e < W + 3 && !(pos_finite(hL) && pos_finite(hR))) bad |= HSGN_DEV_ERR_DEPTH;
                const R uL = qL / hL, uR = qR / hR;
                const R s = p.local_speed ? dmax(dabs(uL), dabs(uR)) : spd;
                wL[e] = add_u(uL, s);
                wR[e] = sub_u(uR, s);
                // the momentum flux from the same reconstruction of q
                Fq[e] = fma_u(wL[e], qL, wR[e] * qR);
            }
            st4(sm.fq, j0, Fq);
        }
        DArr<Gm::NC>* const X[2] = {&sm.ml, &sm.rl};
        DArr<Gm::NC>* const F[2] = {&sm.fm, &sm.fr};
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            R Xv[8], Dv[5];
            ld4(*X[v], j0, Xv);
            ld4(*X[v], j0 + 4, Xv + 4);
            quarter(Xv, Dv);
            R Fv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const R xL = add_u(Xv[e + 1], Dv[e]);
                const R xR = sub_u(Xv[e + 2], Dv[e + 1]);
                Fv[e] = fma_u(wL[e], xL, wR[e] * xR);
            }
            st4(*F[v], j0, Fv);
        }
        // the faces 4t .. 4t + 3 stop at 4T - 1; a full window (W = R) also
        // needs face W + 2 = 4T (right of cell W): the last thread adds it
        if (tid == T - 1 && W + 3 > 4 * T) {
            const int f = 4 * T;  // cells at index f .. f + 3, all loaded (< W + 6)
            auto face = [&](const DArr<Gm::NC>& A, R& xl, R& xr) {
                R x0, x1, x2, x3;
                ld1(A, f, x0);
                ld1(A, f + 1, x1);
                ld1(A, f + 2, x2);
                ld1(A, f + 3, x3);
                xl = add_u(x1, scale(sub_u(x2, x0), 0.25f));
                xr = sub_u(x2, scale(sub_u(x3, x1), 0.25f));
            };
            R hL, hR, qL, qR, mL, mR, rL, rR;
            face(sm.hl, hL, hR);
            face(sm.ql, qL, qR);
            face(sm.ml, mL, mR);
            face(sm.rl, rL, rR);
            if (!(pos_finite(hL) && pos_finite(hR))) bad |= HSGN_DEV_ERR_DEPTH;
            const R uL = qL / hL, uR = qR / hR;
            const R s = p.local_speed ? dmax(dabs(uL), dabs(uR)) : spd;
            const R wl = add_u(uL, s), wr = sub_u(uR, s);
            st1(sm.fq, f, fma_u(wl, qL, wr * qR));
            st1(sm.fm, f, fma_u(wl, mL, wr * mR));
            st1(sm.fr, f, fma_u(wl, rL, wr * rR));
        }
    }
    __syncthreads();

    // ---- B. per cell c = j - 1, j = 4t .. 4t+3 (c = -1 .. W are formed):
    //         increments of the starred values (lines 1-3 of the scheme, the
    //         lambda tau and lambda tau^2 terms kept apart),
    //           dr = -tau/dx (F^r_{c+1/2} - F^r_{c-1/2}),        r^dag = r_b + dr + lambda tau
    //           dm^ = tau (r_b + dr) - tau/dx (F^m ...),         m^dag = m_b + dm^ + lambda tau^2
    //           dq = -tau/dx (F^q ...),                          q^dag = q_b + dq
    //         and the coefficients of U_l (eq. (eq:hSGN_alpha) and the scheme):
    //           eta = m/h, alpha = -(2 eta/h - 1)/(3h), c^2 = g h + (lambda/3) eta^2/h^2,
    //           a^2 = c^2 - lambda eta alpha, beta_1 = 1 + lambda tau^2/h^2,
    //           beta_2 = 2 lambda tau^2/(beta_1^2 h^3), beta = a^2 + lambda alpha beta_2 m^dag,
    //           delta = alpha/beta_1
    //         Bottom form: m^dag also takes -(3/2) tau q_l b_x, and per cell
    //           p~ = (lambda/3) P_l/h^2, P_l = h^2 - m_l (h = h_l),
    //           pi = eta p~ + lambda alpha (h^2 (m_b - m_l + dm^) + lambda tau^2 P_l)/(h^2 + lambda tau^2)
    //         take the place of delta
    dfl dq_[4], dm_[4], dr_[4], be_[4], de_[4], pt_[WB ? 4 : 1];
    float kloc = 0.f, kmin = 3.0e38f;
    {
        const R c_fq = as_R(kc.fq, R()), c_tau = as_R(kc.tau, R()), c_lt2 = as_R(kc.lt2, R());
        const R c_third = as_R(p.third, R()), c_g = as_R(p.g, R()), c_lam3 = as_R(p.lam3, R());
        const R c_lam = as_R(p.lam, R());
        R FQ[8], FM[8], FR[8];
        ld4(sm.fq, j0, FQ);
        ld4(sm.fq, j0 + 4, FQ + 4);
        ld4(sm.fm, j0, FM);
        ld4(sm.fm, j0 + 4, FM + 4);
        ld4(sm.fr, j0, FR);
        ld4(sm.fr, j0 + 4, FR + 4);
        R HL[8], ML[8], MB[8], RB[8];
        ld4(sm.hl, j0, HL);
        ld4(sm.hl, j0 + 4, HL + 4);
        ld4(sm.ml, j0, ML);
        ld4(sm.ml, j0 + 4, ML + 4);
        ld4(sm.mb, j0, MB);
        ld4(sm.mb, j0 + 4, MB + 4);
        ld4(sm.rb, j0, RB);
        ld4(sm.rb, j0 + 4, RB + 4);
        // bottom form: m_b - m_l = (wb1 - wl1) dm1 from the stage-1 increments
        // (zero in stage 1), read per cell inside the loop with q_l and b
        const bool inner = WB && two && inner_window(wl, W, n);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            dq_[k] = dm_[k] = dr_[k] = be_[k] = de_[k] = dfl(0.f);
            if constexpr (WB) pt_[k] = dfl(0.f);
            if (j0 + k < W + 2) {
                const R dr = -(c_fq * sub_acc(FR[k + 1], FR[k]));
                R dm = fma_u(c_tau, add_u(RB[k + 2], dr), -(c_fq * sub_acc(FM[k + 1], FM[k])));
                // bottom source of the (h eta) equation, -(3/2) tau q_l (b_{c+1} - b_{c-1})/(2 dx)
                // (Sec. 2.3, eq. (hSGNb_eq))
                if constexpr (WB)
                    dm = sub_u(dm, mul_f(c_fq * (sm.ql.get(j0 + k + 2) *
                                                 sub_acc(sm.wb.bb.get(j0 + k + 3),
                                                         sm.wb.bb.get(j0 + k + 1))),
                                         1.5f));
                // (the q flux difference reaches the depth system only through
                // tau/(2dx) twice: the plain pair sum)
                const R dq = -(c_fq * sub_u(FQ[k + 1], FQ[k]));
                const R ms = add_u(add_u(MB[k + 2], dm), c_lt2);
                const R h = HL[k + 2];
                if (!pos_finite(h)) bad |= HSGN_DEV_ERR_DEPTH;
                const R ih = rcp(h);
                const R eta = ML[k + 2] * ih;
                const R e = eta * ih;
                const R alpha = -(add_f(scale(e, 2.f), -1.f) * ih * c_third);
                const R c2 = fma_u(c_g, h, c_lam3 * (e * e));
                const R a2 = sub_u(c2, c_lam * (eta * alpha));
                const R h2 = h * h;
                const R iD = rcp(add_u(h2, c_lt2));  // 1/(beta_1 h^2)
                const R ib1 = h2 * iD;              // 1/beta_1
                const R beta2 = scale(c_lt2, 2.f) * (h * (iD * iD));
                const R beta = fma(c_lam * alpha, beta2 * ms, a2);
                if (!pos_finite(beta)) bad |= HSGN_DEV_ERR_COERCIVE;
                dq_[k] = to_dfl(dq);
                dm_[k] = to_dfl(dm);
                dr_[k] = to_dfl(dr);
                be_[k] = to_dfl(beta);
                if constexpr (!WB) {
                    de_[k] = to_dfl(alpha * ib1);
                } else {
                    dfl mbl(0.f);
                    if (two) {
                        // per-cell index j is window cell j - 1, global cell wl + j - 1
                        const int64_t gi = inner ? wl + j0 + k - 1 : cell_at<BC>(wl + j0 + k - 1, n);
                        const float2 d = __ldg(p.D1[2] + gi);
                        mbl = p.wmd * dfl(d.x, d.y);
                    }
                    const dfl Pl = sq_minus(h, ML[k + 2]);
                    const dfl ptil = c_lam3 * (Pl * (ih * ih));
                    const dfl X = fma_u(h2, add_u(mbl, dm), c_lt2 * Pl) * iD;
                    de_[k] = fma_u(eta, ptil, (c_lam * alpha) * X);  // pi
                    pt_[k] = ptil;
                }
                const float kb = f_mul(kc.Cc.hi, hi_of(beta));
                kloc = fmaxf(kloc, kb);
                kmin = fminf(kmin, kb);
            }
        }
    }
    __syncthreads();
    DArr<Gm::NC>& DQ = WB ? sm.ql : sm.hl;
    DArr<Gm::NC>& DM = WB ? sm.ml : sm.ql;
    DArr<Gm::NC>& DR = WB ? sm.rl : sm.ml;
    DArr<Gm::NC>& BE = WB ? sm.fq : sm.rl;
    DArr<Gm::NC>& DE = WB ? sm.fm : sm.fq;  // delta, or pi of the bottom form
    DArr<Gm::NC>& PT = sm.fr;               // p~ of the bottom form
    DArr<Gm::NC>& DH = WB ? sm.fr : sm.fm;  // (after the solve)
    DArr<Gm::NC>& PSI = sm.fm;              // face forces of the bottom form (after the solve)
    DQ.set4(j0, dq_);
    DM.set4(j0, dm_);
    DR.set4(j0, dr_);
    BE.set4(j0, be_);
    DE.set4(j0, de_);
    if constexpr (WB) PT.set4(j0, pt_);
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
    // truncation bound of this window, rho*^(HWc - 1) <= 2^-50, from the
    // coupling bounds of its rows (every thread evaluates the same words: the
    // decision below is uniform over the CTA)
    {
        const bool cut = BC == BC_PERIODIC || !(win.lend && win.rend);
        const float K = __uint_as_float(sm.kmax), kap = fminf(__uint_as_float(sm.kmin), K);
        float lg = -INFINITY;
        if (cut && K > 0.f) {
            const float Bq = 1.f + K + kap;
            const float rho = 2.f * K / (Bq + sqrtf(fmaxf(Bq * Bq - 4.f * kap * K, 0.f)));
            lg = __log2f(rho);
        }
        if (two && piece < 0 && p.need_out && tid == 0 && lg > -INFINITY)
            atomicMax(p.need_out, df_rows_needed(lg));
        const bool misses = (float)(HWc - 1) * lg > -50.f;
        if (misses && piece < 0 && HWc < HW) {
            npieces = (sp0 + Gm::S - 1) / Gm::S;
            pr = (sp0 + npieces - 1) / npieces;
            piece = 0;
            continue;
        }
        if (misses && tid == 0) bad |= HSGN_DEV_ERR_TRUNCATION;
    }
    if (BC == BC_TRANSMISSIVE && (win.lend || win.rend)) {  // (uniform over the CTA)
        // zero-order ghost copies of the per-cell values at the domain ends
        if (tid == 0 && win.lend) {
            DQ.set(0, DQ.get(1)); DM.set(0, DM.get(1)); DR.set(0, DR.get(1));
            BE.set(0, BE.get(1)); DE.set(0, DE.get(1));
            if constexpr (WB) PT.set(0, PT.get(1));
        }
        if (tid == 0 && win.rend) {
            const int a = W + 1, c = W;
            DQ.set(a, DQ.get(c)); DM.set(a, DM.get(c)); DR.set(a, DR.get(c));
            BE.set(a, BE.get(c)); DE.set(a, DE.get(c));
            if constexpr (WB) PT.set(a, PT.get(c));
        }
        __syncthreads();
    }

    // ---- C. rows i = 4t .. 4t+3 of A dh = d - A h_b (lines 8-10 of the
    //         scheme in increment form; interface values are means, reading
    //         R2, and the delta term carries factor 1 with means, reading R3):
    //           coupling of face f (rows f-1, f): K_f = tau^2/dx^2 beta_f
    //             (zero across a transmissive domain end: Neumann rows);
    //           Phi_f = lambda tau^2/dx^2 delta_f (m^dag_f - m^dag_{f-1}) + K_f (h_b,f - h_b,f-1);
    //           d_i - (A h_b)_i = -tau/(2 dx) (q^dag_{i+1} - q^dag_{i-1}) + Phi_{i+1} - Phi_i.
    //         Bottom form: Phi_f = tau^2/dx^2 Psi_f with the face forces Psi_f above.
    dfl KF[5], rd[4], PSv[WB ? 4 : 1];
    if constexpr (WB) {
        dfl Phi[5];
        {
            // face by face, each face's values read as it goes (left cell:
            // per-cell index f, state f + 2; right cell: f + 1, f + 3), so that
            // the six per-cell arrays are not all held in registers at once
            dfl bL = BE.get(j0), eL = DE.get(j0), pL = PT.get(j0);
            dfl hlL = sm.hl.get(j0 + 2), hbL = sm.hb.get(j0 + 2), bbL = sm.wb.bb.get(j0 + 2);
#pragma unroll
            for (int e = 0; e < 5; ++e) {
                const int f = j0 + e;  // rows f - 1 | f: per-cell index f, f + 1; state f + 2, f + 3
                const dfl bR = BE.get(f + 1), eR = DE.get(f + 1), pR = PT.get(f + 1);
                const dfl hlR = sm.hl.get(f + 3), hbR = sm.hb.get(f + 3), bbR = sm.wb.bb.get(f + 3);
                const dfl bf = scale(add_u(bL, bR), 0.5f);
                dfl kf = kc.Cc * bf;
                const dfl dhl = sub_acc(hlR, hlL);
                const dfl db = sub_acc(bbR, bbL);
                const dfl hbar = scale(add_u(hlL, hlR), 0.5f);
                const dfl ptf = scale(add_u(pL, pR), 0.5f);
                // g hbar_f (h_l + b jump) + (pi jump) + (3/2) p~_f (b jump) - beta_f (h_l - h_b jump)
                dfl psi = add_u(add_u(p.g * (hbar * add_u(dhl, db)), sub_acc(eR, eL)),
                                sub_u(mul_f(ptf * db, 1.5f), bf * sub_u(dhl, sub_acc(hbR, hbL))));
                if (BC == BC_TRANSMISSIVE && ((f == 0 && win.lend) || (f == W && win.rend))) {
                    kf = dfl(0.f);
                    psi = dfl(0.f);
                }
                KF[e] = kf;
                Phi[e] = kc.Cc * psi;
                if (e < 4) PSv[e] = psi;
                bL = bR; eL = eR; pL = pR;
                hlL = hlR; hbL = hbR; bbL = bbR;
            }
        }
        dfl Q8[8], QU[8];
        DQ.get4(j0, Q8);
        DQ.get4(j0 + 4, Q8 + 4);
        sm.qb.get4(j0, QU);
        sm.qb.get4(j0 + 4, QU + 4);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const dfl dqc = add_u(sub_acc(QU[k + 4], QU[k + 2]), sub_u(Q8[k + 2], Q8[k]));
            rd[k] = sub_u(sub_acc(Phi[k + 1], Phi[k]), kc.fq * dqc);
        }
    } else {
        dfl Phi[5];
        {
            dfl B8[8], E8[8];
            BE.get4(j0, B8);
            BE.get4(j0 + 4, B8 + 4);
            DE.get4(j0, E8);
            DE.get4(j0 + 4, E8 + 4);
            dfl M8[8], MU[8], H8[8];
            DM.get4(j0, M8);
            DM.get4(j0 + 4, M8 + 4);
            sm.mb.get4(j0, MU);
            sm.mb.get4(j0 + 4, MU + 4);
            sm.hb.get4(j0, H8);
            sm.hb.get4(j0 + 4, H8 + 4);
#pragma unroll
            for (int e = 0; e < 5; ++e) {
                const int f = j0 + e;  // rows f - 1 | f: per-cell index f, f + 1; state f + 2, f + 3
                const dfl bf = scale(add_u(B8[e], B8[e + 1]), 0.5f);
                const dfl df = scale(add_u(E8[e], E8[e + 1]), 0.5f);
                dfl kf = kc.Cc * bf;
                if (BC == BC_TRANSMISSIVE && ((f == 0 && win.lend) || (f == W && win.rend)))
                    kf = dfl(0.f);
                const dfl dmf = add_u(sub_acc(MU[e + 3], MU[e + 2]), sub_acc(M8[e + 1], M8[e]));
                const dfl dhf = sub_acc(H8[e + 3], H8[e + 2]);
                KF[e] = kf;
                Phi[e] = fma_u(kc.fd * df, dmf, kf * dhf);
            }
        }
        dfl Q8[8], QU[8];
        DQ.get4(j0, Q8);
        DQ.get4(j0 + 4, Q8 + 4);
        sm.qb.get4(j0, QU);
        sm.qb.get4(j0 + 4, QU + 4);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            // q^dag of cells i+1 and i-1: state index i + 4, i + 2; per-cell index i + 2, i
            const dfl dqc = add_u(sub_acc(QU[k + 4], QU[k + 2]), sub_u(Q8[k + 2], Q8[k]));
            rd[k] = sub_u(sub_acc(Phi[k + 1], Phi[k]), kc.fq * dqc);
        }
    }
    {
        // row 4t + k of the window; the first / last window row drops its outer
        // coupling; the rows from W on close the window (identity)
        auto roww = [&](int k, int i, dfl& a, dfl& bb, dfl& c, dfl& d) {
            if (i >= W) {
                a = dfl(0.f); bb = dfl(1.f); c = dfl(0.f); d = dfl(0.f);
                return;
            }
            const dfl kl = KF[k], kr = KF[k + 1];
            a = (i == 0 && !win.lend) ? dfl(0.f) : -kl;
            c = (i == W - 1 && !win.rend) ? dfl(0.f) : -kr;
            bb = add_f(add_u(kl, kr), 1.f);
            d = rd[k];
        };
        dfl y[M];
        cta_window_solve<T, M>(W + 1, roww, sm.sep, y, p.err);
        // dh = y: the values outside the window (and the closing row) are taken as 0
#pragma unroll
        for (int k = 0; k < M; ++k)
            if (!(j0 + k < W)) y[k] = dfl(0.f);
        DH.set4(j0 + 4, y);
        // the face forces of the bottom form for the back-substitution (their
        // array held pi, last read before the solve's first barrier)
        if constexpr (WB) PSI.set4(j0, PSv);
    }
    __syncthreads();
    if (BC == BC_TRANSMISSIVE && (win.lend || win.rend)) {  // (uniform over the CTA)
        if (tid == 0 && win.lend) DH.set(3, DH.get(4));
        if (tid == 0 && win.rend) DH.set(W + 4, DH.get(W + 3));
        __syncthreads();
    }

    // ---- E. back-substitution of the tile rows (lines 11-13 of the scheme;
    //         h w with h^2 implicit, Sec. 6.3.1), in increment form:
    //           dQ = dq - tau/(2dx) beta (hbar_{i+1} - hbar_{i-1})
    //                   - lambda tau/(2dx) delta (m^dag_{i+1} - m^dag_{i-1}),
    //           P = hbar^2 - m_b, E = hbar^2 - m^ = P - dm^, D = hbar^2 + lambda tau^2,
    //           (h eta)bar - m_b = P - E hbar^2/D,  (h w)bar - r_b = dr + lambda tau E/D
    //         (m^dag hbar^2/D and r^dag - lambda tau (h eta)bar/hbar^2 without the
    //         cancellation of their lambda tau terms)
    const int lo = win.lo, sp = win.sp;
    const int64_t t0 = win.t0;
    for (int t = tid; t < sp; t += T) {
        const int r = lo + t;  // window row; state index r + 3, per-cell index r + 1, dh index r + 4
        const dfl dh = DH.get(r + 4);
        const dfl hb = sm.hb.get(r + 3), mb = sm.mb.get(r + 3);
        const dfl dhc = add_u(sub_acc(sm.hb.get(r + 4), sm.hb.get(r + 2)),
                              sub_u(DH.get(r + 5), DH.get(r + 3)));
        const dfl dmv = DM.get(r + 1);
        dfl dQ;
        if constexpr (!WB) {
            const dfl dmc = add_u(sub_acc(sm.mb.get(r + 4), sm.mb.get(r + 2)),
                                  sub_u(DM.get(r + 2), DM.get(r)));
            dQ = sub_u(DQ.get(r + 1),
                       add_u(kc.fq * (BE.get(r + 1) * dhc), kc.lfq * (DE.get(r + 1) * dmc)));
        } else {
            // q = q^dag - tau/(2dx) (F_{r+1/2} + F_{r-1/2}), F_f = Psi_f + beta_f (dh jump)
            (void)dhc;
            const dfl bp = scale(add_u(BE.get(r + 1), BE.get(r + 2)), 0.5f);
            const dfl bm = scale(add_u(BE.get(r), BE.get(r + 1)), 0.5f);
            const dfl Fp = fma_u(bp, sub_u(DH.get(r + 5), dh), PSI.get(r + 1));
            const dfl Fm = fma_u(bm, sub_u(dh, DH.get(r + 3)), PSI.get(r));
            dQ = sub_u(DQ.get(r + 1), kc.fq * add_u(Fp, Fm));
        }
        const dfl P = add_u(sq_minus(hb, mb), dh * add_u(scale(hb, 2.f), dh));
        const dfl E = sub_u(P, dmv);
        // (renormalised where it is written as the new state)
        const dfl hbar = two ? hb + dh : add_u(hb, dh);
        const dfl h2 = hbar * hbar;
        const dfl iDen = rcp(add_u(h2, kc.lt2));
        const dfl Ei = E * iDen;
        const dfl dR = fma_u(kc.ltau, Ei, DR.get(r + 1));
        const dfl dM = sub_u(P, Ei * h2);
        unsigned b2 = 0;
        if (!pos_finite(hbar)) b2 |= HSGN_DEV_ERR_DEPTH;
        if (!isfinite(dQ.hi) || !isfinite(dM.hi) || !isfinite(dR.hi)) b2 |= HSGN_DEV_ERR_NONFINITE;
        bad |= b2;
        const int64_t gc = t0 + t;
        if constexpr (!two) {
            p.D1[0][gc] = make_float2(dh.hi, dh.lo);
            p.D1[1][gc] = make_float2(dQ.hi, dQ.lo);
            p.D1[2][gc] = make_float2(dM.hi, dM.lo);
            p.D1[3][gc] = make_float2(dR.hi, dR.lo);
        } else {
            const dfl qn = sm.qb.get(r + 3) + dQ;
            const dfl mn = mb + dM;
            const dfl rn = sm.rb.get(r + 3) + dR;
            p.out[0][gc] = make_float2(hbar.hi, hbar.lo);
            p.out[1][gc] = make_float2(qn.hi, qn.lo);
            p.out[2][gc] = make_float2(mn.hi, mn.lo);
            p.out[3][gc] = make_float2(rn.hi, rn.lo);
            if (p.track_speed && !b2) {
                const dfl ua = dabs(qn) / hbar;
                umax = dmax(umax, ua);
                if (p.adaptive) {
                    // nu = |u| + sqrt(g h + (lambda/3) eta^2/h^2) of U^{n+1} (reading R9)
                    const dfl e = mn / (hbar * hbar);
                    numax = dmax(numax, ua + dsqrt(fma(p.g, hbar, p.lam3 * (e * e))));
                }
            }
        }
    }
    if (piece < 0 || ++piece >= npieces) break;
    }  // passes
    if (bad) flag_error(p.err, bad);
    if (p.track_speed && two) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) umax = dmax(umax, shfl_xor_d(umax, o));
        if ((tid & 31) == 0 && umax.hi > 0.f)
            atomicMax(reinterpret_cast<unsigned long long*>(p.speed_next),
                      (unsigned long long)__double_as_longlong(dfl_to_double(umax)));
        if (p.adaptive) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) numax = dmax(numax, shfl_xor_d(numax, o));
            if ((tid & 31) == 0 && numax.hi > 0.f)
                atomicMax(reinterpret_cast<unsigned long long*>(p.speed_next + 1),
                          (unsigned long long)__double_as_longlong(dfl_to_double(numax)));
        }
    }
}

// Pairs of base and lin - base (hsgn_stage on the double-float form): the
// stage-2 kernel with weights 1 and 0 then runs the stage from U_b = base,
// U_l = lin.
__global__ void k_df_stage_inputs(int64_t n, const double* __restrict__ base,
                                  const double* __restrict__ lin, float2* __restrict__ ub,
                                  float2* __restrict__ dl) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double b = base[i];
        ub[i] = df_of(b);
        dl[i] = df_of(lin[i] - b);
    }
}

// Pairs to doubles in place (the pair and the double of entry i share its 8 bytes).
__global__ void k_f64_from_df_inplace(int64_t n, void* buf) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = reinterpret_cast<const float2*>(buf)[i];
        reinterpret_cast<double*>(buf)[i] = (double)v.x + (double)v.y;
    }
}

}  // namespace hsgn
