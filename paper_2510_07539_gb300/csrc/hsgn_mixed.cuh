// hsgn_mixed.cuh -- the stage in mixed precision: FP32 increments, FP64 state.
//
// Same scheme as hsgn_kernels.cuh (Sec. 4.2, eq. (GN_hyp_eq_semi_fully_discrete);
// Sec. 3.2 efficient form of the tableau), rearranged so that every quantity
// computed in single precision is an increment or a coefficient, never a
// difference of two large numbers:
//  * the stage-1 result is kept as FP32 increments (q, h eta, h w) and FP32
//    face mass fluxes G (depth increment = G_{i-1/2} - G_{i+1/2});
//  * differences of the FP64 base state are formed in FP64 before rounding;
//  * the depth system is solved for dh = hbar - h_b:  A dh = d - A h_b
//    (A has row sums 1, so the right side is a sum of differences);
//  * hbar is then rebuilt in FP64 in flux form, hbar_i = h_b,i - (G_{i+1/2} -
//    G_{i-1/2}), with G_{i+1/2} = tau/(2dx)(q^dag_i + q^dag_{i+1}) -
//    lambda tau^2/dx^2 delta_{i+1/2} (m^dag_{i+1} - m^dag_i) - tau^2/dx^2
//    beta_{i+1/2} (hbar_{i+1} - hbar_i): the face fluxes are shared by both
//    neighbours, so the mass is conserved to FP64 rounding;
//  * the relaxation update without the cancellation of the two lambda tau terms:
//    with m^ = m^dag - lambda tau^2 and E = hbar^2 - m^,
//      (h w)bar = r_b + dr' + lambda tau E / (hbar^2 + lambda tau^2),
//      (h eta)bar = hbar^2 - E hbar^2 / (hbar^2 + lambda tau^2),
//    which equal r^dag - lambda tau mbar/hbar^2 and m^dag/(1 + lambda tau^2/hbar^2).
// FP64 work per cell and stage: three base-state differences, one h^2 - m, and
// the final additions (stage 2 only). Conversions between the two formats are
// done with integer operations: on sm_103a the cvt instructions run on the slow
// double-precision datapath.
#pragma once

#include "hsgn_kernels.cuh"

namespace hsgn {

// Double to single by truncating the significand (relative error below 2^-23);
// magnitudes below the single normal range give a signed zero, above it (and
// NaN) an infinity.
__device__ __forceinline__ float f32_of(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned s = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu) - 1023 + 127;
    const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    unsigned r;
    if (e <= 0)
        r = s;
    else if (e >= 255)
        r = s | 0x7F800000u;
    else
        r = s | ((unsigned)e << 23) | m;
    return __uint_as_float(r);
}

// Single to double, exact (subnormal singles flush to zero).
__device__ __forceinline__ double f64_of(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned s = u & 0x80000000u, e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
    unsigned hi, lo;
    if (e == 0) {
        hi = s;
        lo = 0u;
    } else if (e == 255u) {
        hi = s | 0x7FF00000u | (m >> 3);
        lo = m << 29;
    } else {
        hi = s | ((e + 896u) << 20) | (m >> 3);
        lo = m << 29;
    }
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

struct MixedParams {
    int64_t n;
    int32_t bc;
    int32_t local_speed;
    int32_t stage;  // 1: writes the stage-1 increments; 2: writes U^{n+1}
    int32_t track_speed;
    float g, lam, tau;
    float tdx;   // tau / dx
    float fq;    // tau / (2 dx)
    float Cc;    // tau^2 / dx^2
    float fd;    // lambda tau^2 / dx^2
    float lt2;   // lambda tau^2
    float ltau;  // lambda tau
    float wl1, wb1;  // U_l = U^n + wl1 dU1, U_b = U^n + wb1 dU1
    const double* U[4];                  // U^n (FP64)
    float *G1, *dq1, *dm1, *dr1;         // stage-1 increments: G1 has n+1 faces
    double* speed;                       // global Rusanov speed of the step
    BlockSplit split;
    // per-row results of the assembly kernel, three float4 records per row:
    //   rec[3i]   = (y, v, w, q_b)       block elimination triple, base momentum
    //   rec[3i+1] = (dq, dm', dr', beta) increments and coefficient of the cell
    //   rec[3i+2] = (delta, Dh, Dm, P0)  coefficient, base differences at face
    //                                    i+1/2, h_b^2 - m_b
    float4* rec;
    float* blk;
    float* s;                            // block separators (after the separator solve)
    double* out[4];                      // U^{n+1} (stage 2)
    unsigned* err;
    // batch of independent instances (batched != 0): the fields n, split, the
    // dt-dependent constants and speed above are replaced per block by the
    // instance's entries
    int32_t batched;
    const struct InstInfo* inst;         // per instance
    const int32_t* blk_inst;             // instance of every global block
    double* speeds;                      // per-instance Rusanov speed
};

// One instance of a batch: packed cell offset, size, block split, first global
// block, grid spacing, relaxation parameter and time step, and the stage
// constants in single precision that follow from them (tau = gamma dt: tau,
// tau/dx, tau/(2dx), tau^2/dx^2, lambda tau^2/dx^2, lambda tau^2, lambda tau,
// lambda), set on the host with the time step exactly as for one instance
// (the FP64 pipe would otherwise spend every CTA's start on them).
struct InstInfo {
    int64_t cell0;
    int64_t n;
    int64_t base;
    int32_t P, rem;
    int32_t blk0, pad;
    double dx, lam, dt;
    float tau, tdx, fq, Cc, fd, lt2, ltau, lamf;
};

// Geometry and constants of the instance that owns a block.
struct BlockCtx {
    int64_t cell0, face0;  // packed offsets of the instance's cell 0 and face -1/2
    int64_t n;             // cells of the instance
    BlockSplit split;      // the instance's blocks
    int64_t lb, blk0;      // local block index, global index of block 0
    int64_t r0;            // first local row of the block
    int nb;                // rows of the block
    float tau, tdx, fq, Cc, fd, lt2, ltau, lam;
    double* speed;
};

__device__ __forceinline__ BlockCtx make_ctx(const MixedParams& p, int64_t b) {
    BlockCtx c;
    if (!p.batched) {
        c.cell0 = 0;
        c.face0 = 0;
        c.n = p.n;
        c.split = p.split;
        c.lb = b;
        c.blk0 = 0;
        c.tau = p.tau; c.tdx = p.tdx; c.fq = p.fq; c.Cc = p.Cc; c.fd = p.fd;
        c.lt2 = p.lt2; c.ltau = p.ltau; c.lam = p.lam;
        c.speed = p.speed;
    } else {
        const int k = p.blk_inst[b];
        const InstInfo I = p.inst[k];
        c.cell0 = I.cell0;
        c.face0 = I.cell0 + k;  // instance k's n+1 faces follow those of instances < k
        c.n = I.n;
        c.split.n = I.n;
        c.split.base = I.base;
        c.split.P = I.P;
        c.split.rem = I.rem;
        c.lb = b - I.blk0;
        c.blk0 = I.blk0;
        c.tau = I.tau; c.tdx = I.tdx; c.fq = I.fq; c.Cc = I.Cc; c.fd = I.fd;
        c.lt2 = I.lt2; c.ltau = I.ltau; c.lam = I.lamf;
        c.speed = p.speeds + k;
    }
    c.r0 = c.split.start(c.lb);
    c.nb = (int)c.split.size(c.lb);
    return c;
}

// Face index of G1: face i+1/2 is stored at i+1 (i = -1 .. n-1).
// Shared memory of the mixed assembly for blocks of at most S = T*M rows; the
// arrays read in the chunk mapping use the padded index pd().
template <int T, int M>
struct MixedShared {
    static constexpr int S = T * M;
    static constexpr int NC = pd_size(S + 6);
    float hl[NC], ql[NC], ml[NC], rl[NC];   // U_l, cells -3 .. S+2 (later: y, v, w)
    float qb[NC], mb[NC], rb[NC];           // U_b (rounded)
    float Dh[NC], Dq[NC], Dm[NC];           // face between local cells j-3, j-2
    float P0[NC];
    float Fq[S + 3], Fm[S + 3], Fr[S + 3];  // faces -2 .. S
    float dq[NC], dm[NC], dr[NC], be[NC], de[NC];  // cells -1 .. S
    SepShared<T, float> sep;
    float lastrow[4];
};

template <int T, int M, int BC>
__global__ void __launch_bounds__(T) k_mixed_assemble(const MixedParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<MixedShared<T, M>*>(smem_raw);
    const int tid = threadIdx.x;
    const int64_t b = blockIdx.x;
    const BlockCtx X = make_ctx(p, b);
    const int64_t r0 = X.r0;
    const int nb = X.nb;
    const int64_t n = X.n;
    const bool two = p.stage == 2;
    const float wl1 = p.wl1, wb1 = p.wb1;
    const double* __restrict__ U0 = p.U[0] + X.cell0;
    const double* __restrict__ U1 = p.U[1] + X.cell0;
    const double* __restrict__ U2 = p.U[2] + X.cell0;
    const double* __restrict__ U3 = p.U[3] + X.cell0;
    const float* __restrict__ G1 = p.G1 + X.face0;
    const float* __restrict__ dq1p = p.dq1 + X.cell0;
    const float* __restrict__ dm1p = p.dm1 + X.cell0;
    const float* __restrict__ dr1p = p.dr1 + X.cell0;
    float4* __restrict__ rec = p.rec + 3 * X.cell0;

    // ---- 0. stage inputs with a 3-cell halo; FP64 differences of U^n. At most
    //         ceil((S+6)/T) cells per thread; all loads of a cell are issued
    //         before any of its shared-memory stores.
    constexpr int NL = (T * M + 6 + T - 1) / T;
#pragma unroll
    for (int it = 0; it < NL; ++it) {
        const int j = tid + it * T;
        if (j < nb + 6) {
            const int64_t gi = wrap_index(r0 + j - 3, n, BC);
            const int64_t gn = wrap_index(r0 + j - 2, n, BC);
            const double h0 = __ldg(U0 + gi), q0 = __ldg(U1 + gi);
            const double m0 = __ldg(U2 + gi), rr0 = __ldg(U3 + gi);
            const double h1 = __ldg(U0 + gn), q1 = __ldg(U1 + gn), m1 = __ldg(U2 + gn);
            float dh1 = 0.f, dq1 = 0.f, dm1 = 0.f, dr1 = 0.f, dh1n = 0.f, dq1n = 0.f, dm1n = 0.f;
            if (two) {
                const float g0 = __ldg(G1 + gi), g1 = __ldg(G1 + gi + 1);
                const float g2 = __ldg(G1 + gn), g3 = __ldg(G1 + gn + 1);
                dq1 = __ldg(dq1p + gi);
                dm1 = __ldg(dm1p + gi);
                dr1 = __ldg(dr1p + gi);
                dq1n = __ldg(dq1p + gn);
                dm1n = __ldg(dm1p + gn);
                dh1 = g0 - g1;
                dh1n = g2 - g3;
            }
            const float hf = f32_of(h0), qf = f32_of(q0), mf = f32_of(m0), rf = f32_of(rr0);
            const int jp = pd(j);
            sm.hl[jp] = fmaf(wl1, dh1, hf);
            sm.ql[jp] = fmaf(wl1, dq1, qf);
            sm.ml[jp] = fmaf(wl1, dm1, mf);
            sm.rl[jp] = fmaf(wl1, dr1, rf);
            sm.qb[jp] = fmaf(wb1, dq1, qf);
            sm.mb[jp] = fmaf(wb1, dm1, mf);
            sm.rb[jp] = fmaf(wb1, dr1, rf);
            sm.Dh[jp] = fmaf(wb1, dh1n - dh1, f32_of(h1 - h0));
            sm.Dq[jp] = fmaf(wb1, dq1n - dq1, f32_of(q1 - q0));
            sm.Dm[jp] = fmaf(wb1, dm1n - dm1, f32_of(m1 - m0));
            // h_b^2 - m_b = (h^2 - m)^n + wb1 dh1 (2 h^n + wb1 dh1) - wb1 dm1
            sm.P0[jp] = fmaf(wb1, fmaf(dh1, fmaf(wb1, dh1, 2.f * hf), -dm1),
                             f32_of(fma(h0, h0, -m0)));
        }
    }
    __syncthreads();

    const float tau = X.tau, lam = X.lam, g = p.g;
    const float gspeed = p.local_speed ? 0.f : (float)(*X.speed);
    unsigned bad = 0;

    // ---- 1. Rusanov fluxes of U_l at faces f = -2 .. nb (Sec. 4.1)
    for (int j = tid; j < nb + 3; j += T) {
        const int a0 = pd(j), a1 = pd(j + 1), a2 = pd(j + 2), a3 = pd(j + 3);
        const float hm = sm.hl[a0], h0 = sm.hl[a1], h1 = sm.hl[a2], h2 = sm.hl[a3];
        const float qm = sm.ql[a0], q0 = sm.ql[a1], q1 = sm.ql[a2], q2 = sm.ql[a3];
        const float mm = sm.ml[a0], m0 = sm.ml[a1], m1 = sm.ml[a2], m2 = sm.ml[a3];
        const float rm = sm.rl[a0], r0_ = sm.rl[a1], r1 = sm.rl[a2], r2 = sm.rl[a3];
        const float hL = fmaf(0.25f, h1 - hm, h0), hR = fmaf(-0.25f, h2 - h0, h1);
        const float qL = fmaf(0.25f, q1 - qm, q0), qR = fmaf(-0.25f, q2 - q0, q1);
        const float mL = fmaf(0.25f, m1 - mm, m0), mR = fmaf(-0.25f, m2 - m0, m1);
        const float rL = fmaf(0.25f, r1 - rm, r0_), rR = fmaf(-0.25f, r2 - r0_, r1);
        if (!pos_finite(hL) || !pos_finite(hR)) bad |= HSGN_DEV_ERR_DEPTH;
        const float ip = __frcp_rn(hL * hR);
        const float uL = qL * hR * ip, uR = qR * hL * ip;
        const float s = p.local_speed ? fmaxf(fabsf(uL), fabsf(uR)) : gspeed;
        sm.Fq[j] = 0.5f * (fmaf(uL, qL, uR * qR) - s * (qR - qL));
        sm.Fm[j] = 0.5f * (fmaf(uL, mL, uR * mR) - s * (mR - mL));
        sm.Fr[j] = 0.5f * (fmaf(uL, rL, uR * rR) - s * (rR - rL));
    }
    __syncthreads();

    // ---- 2. increments and coefficients at cells c = -1 .. nb:
    //         r^dag = r_b + dr' + lambda tau, m^dag = m_b + dm' + lambda tau^2, q^dag = q_b + dq
    const float lt2 = X.lt2, tdx = X.tdx;
    for (int j = tid; j < nb + 2; j += T) {
        const int c3 = pd(j + 2);
        const float drv = -tdx * (sm.Fr[j + 1] - sm.Fr[j]);
        const float dmv = fmaf(tau, sm.rb[c3] + drv, -tdx * (sm.Fm[j + 1] - sm.Fm[j]));
        const float dqv = -tdx * (sm.Fq[j + 1] - sm.Fq[j]);
        const float msv = sm.mb[c3] + dmv + lt2;
        const float h = sm.hl[c3];
        if (!pos_finite(h)) bad |= HSGN_DEV_ERR_DEPTH;
        const float Dh_ = fmaf(h, h, lt2);
        const float R = __frcp_rn(h * Dh_);
        const float ih = Dh_ * R;
        const float iD = h * R;
        const float eta = sm.ml[c3] * ih;
        const float e = eta * ih;
        const float alpha = fmaf(2.f, e, -1.f) * ih * (-1.f / 3.f);
        const float c2 = fmaf(g, h, (lam * (1.f / 3.f)) * e * e);
        const float a2 = fmaf(-lam * eta, alpha, c2);
        const float ib1 = h * h * iD;
        const float beta2 = (2.f * lt2) * h * iD * iD;
        const float beta = fmaf(lam * alpha * beta2, msv, a2);
        if (!pos_finite(beta)) bad |= HSGN_DEV_ERR_COERCIVE;
        const int jp = pd(j);
        sm.dq[jp] = dqv;
        sm.dm[jp] = dmv;
        sm.dr[jp] = drv;
        sm.be[jp] = beta;
        sm.de[jp] = alpha * ib1;
    }
    __syncthreads();
    if (BC == BC_TRANSMISSIVE && tid == 0) {
        if (r0 == 0) {
            sm.dq[0] = sm.dq[1]; sm.dm[0] = sm.dm[1]; sm.dr[0] = sm.dr[1];
            sm.be[0] = sm.be[1]; sm.de[0] = sm.de[1];
        }
        if (r0 + nb == n) {
            const int a = pd(nb + 1), c = pd(nb);
            sm.dq[a] = sm.dq[c]; sm.dm[a] = sm.dm[c]; sm.dr[a] = sm.dr[c];
            sm.be[a] = sm.be[c]; sm.de[a] = sm.de[c];
        }
    }
    __syncthreads();

    // per-row results used by the back-substitution
    for (int i = tid; i < nb; i += T) {
        const int64_t gi = r0 + i;
        const int c1 = pd(i + 1), f3 = pd(i + 3);
        rec[3 * gi + 1] = make_float4(sm.dq[c1], sm.dm[c1], sm.dr[c1], sm.be[c1]);
        rec[3 * gi + 2] = make_float4(sm.de[c1], sm.Dh[f3], sm.Dm[f3], sm.P0[f3]);
    }

    // ---- 3. rows of A dh = d - A h_b (face i+1/2 of cell i is index i+3)
    const float Cc = X.Cc, fq = X.fq, fd = X.fd;
    auto row = [&](int i, float& a, float& bb, float& c, float& d) {
        const int c0 = pd(i), c1 = pd(i + 1), c2 = pd(i + 2), f2 = pd(i + 2), f3 = pd(i + 3);
        const float bm = 0.5f * (sm.be[c0] + sm.be[c1]);
        const float bp = 0.5f * (sm.be[c1] + sm.be[c2]);
        const float dmn = 0.5f * (sm.de[c0] + sm.de[c1]);
        const float dpl = 0.5f * (sm.de[c1] + sm.de[c2]);
        const float dqc = sm.Dq[f2] + sm.Dq[f3] + (sm.dq[c2] - sm.dq[c0]);
        const float dmp = sm.Dm[f3] + (sm.dm[c2] - sm.dm[c1]);
        const float dmm = sm.Dm[f2] + (sm.dm[c1] - sm.dm[c0]);
        d = -fq * dqc + fd * (dpl * dmp - dmn * dmm) - Cc * (bm * sm.Dh[f2] - bp * sm.Dh[f3]);
        a = -Cc * bm;
        c = -Cc * bp;
        bb = fmaf(Cc, bm + bp, 1.f);
        if (BC == BC_TRANSMISSIVE) {
            const int64_t gi = r0 + i;
            if (gi == 0) { bb = fmaf(Cc, bp, 1.f); a = 0.f; }
            if (gi == n - 1) { bb = fmaf(Cc, bm, 1.f); c = 0.f; }
        }
    };
    float y[M], v[M], w[M], last[4];
    int cs, m;
    cta_block_solve<T, M>(nb, row, sm.sep, y, v, w, cs, m, last, p.err);
    if (bad) flag_error(p.err, bad);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < M; ++k) {
        if (k < m) {
            const int a = pd(cs + k);
            sm.hl[a] = y[k];
            sm.ql[a] = v[k];
            sm.ml[a] = w[k];
        }
    }
    if (m > 0 && cs + m == nb) {
        sm.lastrow[0] = last[0]; sm.lastrow[1] = last[1];
        sm.lastrow[2] = last[2]; sm.lastrow[3] = last[3];
    }
    __syncthreads();
    for (int i = tid; i < nb; i += T) {
        const int a = pd(i);
        rec[3 * (r0 + i)] = make_float4(sm.hl[a], sm.ql[a], sm.ml[a], sm.qb[pd(i + 3)]);
    }
    if (tid == 0) {
        float* s = p.blk + (X.blk0 + X.lb) * BLK_STRIDE;
        s[0] = sm.lastrow[0]; s[1] = sm.lastrow[1]; s[2] = sm.lastrow[2]; s[3] = sm.lastrow[3];
        s[4] = sm.hl[0]; s[5] = sm.ql[0]; s[6] = sm.ml[0];
        if (nb >= 2) {
            const int a = pd(nb - 2);
            s[7] = sm.hl[a]; s[8] = sm.ql[a]; s[9] = sm.ml[a];
        } else {
            s[7] = 0.f; s[8] = -1.f; s[9] = 0.f;
        }
    }
}

// Everything the back-substitution needs about one cell (read from the
// assembly results only: U^n itself is overwritten in place by stage 2).
struct MixedCell {
    float dh;          // hbar - h_b
    float qb;          // base momentum (rounded)
    float dq, dm, dr, be, de;
    float Dh, Dm;      // base differences at the face to the right
};

__device__ __forceinline__ MixedCell mixed_cell(const float4* __restrict__ rec, int64_t j,
                                                float sl, float sr, bool ghost, float& P0) {
    MixedCell c;
    const float4 r0 = rec[3 * j], r1 = rec[3 * j + 1], r2 = rec[3 * j + 2];
    c.dh = r0.x - sl * r0.y - sr * r0.z;
    c.qb = r0.w;
    c.dq = r1.x;
    c.dm = r1.y;
    c.dr = r1.z;
    c.be = r1.w;
    c.de = r2.x;
    // a transmissive ghost is a copy of the boundary cell: no jump across its face
    c.Dh = ghost ? 0.f : r2.y;
    c.Dm = ghost ? 0.f : r2.z;
    P0 = r2.w;
    return c;
}

// Face mass flux (divided by dx) between cells L and R; the face differences
// are those stored with L. Both neighbours evaluate it identically.
__device__ __forceinline__ float face_flux(const BlockCtx& X, const MixedCell& L,
                                           const MixedCell& R) {
    const float qsum = (L.qb + R.qb) + (L.dq + R.dq);
    const float dmf = L.Dm + (R.dm - L.dm);
    const float dhf = L.Dh + (R.dh - L.dh);
    return X.fq * qsum - X.fd * (0.5f * (L.de + R.de)) * dmf - X.Cc * (0.5f * (L.be + R.be)) * dhf;
}

// One CTA per block; each thread handles rows of the block.
template <int BC>
__global__ void __launch_bounds__(256) k_mixed_backsub(const MixedParams p) {
    __shared__ float red[8];
    const BlockCtx X = make_ctx(p, blockIdx.x);
    const int64_t n = X.n;
    const BlockSplit& sp = X.split;
    const float* __restrict__ s = p.s + X.blk0;
    const float4* __restrict__ rec = p.rec + 3 * X.cell0;
    const float* __restrict__ G1 = p.G1 + X.face0;
    const int64_t lb = X.lb;
    const int64_t lbl = lb == 0 ? sp.P - 1 : lb - 1, lbr = lb + 1 == sp.P ? 0 : lb + 1;
    const float s_ll = s[lbl == 0 ? sp.P - 1 : lbl - 1];  // separators around the block
    const float s_l = s[lbl], s_c = s[lb], s_r = s[lbr];
    float umax = 0.f;
    for (int t = threadIdx.x; t < X.nb; t += blockDim.x) {
        const int64_t i = X.r0 + t;  // local row
        const int64_t il = wrap_index(i - 1, n, BC), ir = wrap_index(i + 1, n, BC);
        const bool gl = (BC == BC_TRANSMISSIVE) && i == 0;
        const bool gr = (BC == BC_TRANSMISSIVE) && i == n - 1;
        // separators (s_{B-1}, s_B) of the block B of each of the three cells
        const bool lin = (il == i - 1 && t > 0) || il == i;          // left cell in this block
        const bool rin = (ir == i + 1 && t + 1 < X.nb) || ir == i;   // right cell in this block
        float P0, P0l, P0r;
        const MixedCell C = mixed_cell(rec, i, s_l, s_c, gr, P0);
        const MixedCell Lc = lin ? mixed_cell(rec, il, s_l, s_c, gl, P0l)
                                 : mixed_cell(rec, il, s_ll, s_l, gl, P0l);
        const MixedCell Rc = rin ? mixed_cell(rec, ir, s_l, s_c, gr, P0r)
                                 : mixed_cell(rec, ir, s_c, s_r, gr, P0r);
        // own base depth (rounded): U^n of this cell is read here, before this
        // thread overwrites it
        const int64_t pi = X.cell0 + i;
        float hbf = f32_of(p.U[0][pi]);
        if (p.stage == 2) hbf = fmaf(p.wb1, G1[i] - G1[i + 1], hbf);
        const float Gp = face_flux(X, C, Rc);  // face i+1/2
        const float Gm = face_flux(X, Lc, C);  // face i-1/2
        // q: tau/(2dx) beta (hbar_{i+1} - hbar_{i-1}), lambda tau/(2dx) delta (m^dag_{i+1} - m^dag_{i-1})
        const float dhc = (Lc.Dh + C.Dh) + (Rc.dh - Lc.dh);
        const float dmc = (Lc.Dm + C.Dm) + (Rc.dm - Lc.dm);
        const float dQ = C.dq - X.fq * C.be * dhc - X.lam * X.fq * C.de * dmc;
        // relaxation pair
        const float hbar = hbf + C.dh;
        const float P = fmaf(C.dh, 2.f * hbf + C.dh, P0);  // hbar^2 - m_b
        const float E = P - C.dm;                           // hbar^2 - m^
        const float h2 = hbar * hbar;
        const float iDen = __frcp_rn(h2 + X.lt2);
        const float dR = fmaf(X.ltau * E, iDen, C.dr);
        const float dM = P - E * h2 * iDen;
        unsigned bad = 0;
        if (!pos_finite(hbar)) bad |= HSGN_DEV_ERR_DEPTH;
        if (!isfinite(Gp) || !isfinite(Gm) || !isfinite(dQ) || !isfinite(dM) || !isfinite(dR))
            bad |= HSGN_DEV_ERR_NONFINITE;
        if (bad) flag_error(p.err, bad);
        if (p.stage == 1) {
            p.G1[X.face0 + i + 1] = Gp;
            if (i == 0) p.G1[X.face0] = Gm;
            p.dq1[pi] = dQ;
            p.dm1[pi] = dM;
            p.dr1[pi] = dR;
        } else {
            const float wb1 = p.wb1;
            const float Tp = fmaf(wb1, G1[i + 1], Gp);
            const float Tm = fmaf(wb1, G1[i], Gm);
            const double h = p.U[0][pi] - (f64_of(Tp) - f64_of(Tm));
            const double q = p.U[1][pi] + f64_of(fmaf(wb1, p.dq1[pi], dQ));
            const double m = p.U[2][pi] + f64_of(fmaf(wb1, p.dm1[pi], dM));
            const double r = p.U[3][pi] + f64_of(fmaf(wb1, p.dr1[pi], dR));
            p.out[0][pi] = h;
            p.out[1][pi] = q;
            p.out[2][pi] = m;
            p.out[3][pi] = r;
            if (p.track_speed && !bad) umax = fmaxf(umax, fabsf((C.qb + dQ) / hbar));
        }
    }
    if (p.track_speed) {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, o));
        if (lane == 0) red[wid] = umax;
        __syncthreads();
        if (threadIdx.x == 0) {
            float v = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmaxf(v, red[w]);
            if (v > 0.f)
                atomicMax(reinterpret_cast<unsigned long long*>(X.speed),
                          (unsigned long long)__double_as_longlong(f64_of(v)));
        }
    }
}

// Per-instance max |u| and max nu = |u| + sqrt(g h + (lambda/3) eta^2/h^2) of a
// batch (Sec. 5 time-step rule): one CTA per instance.
__global__ void __launch_bounds__(256) k_speeds_batched(const InstInfo* inst, const double* h,
                                                        const double* q, const double* m,
                                                        double g, double* out_u, double* out_nu,
                                                        unsigned* err) {
    __shared__ double ru[8], rn[8];
    const InstInfo I = inst[blockIdx.x];
    double um = 0.0, nm = 0.0;
    bool bad = false;
    for (int64_t i = I.cell0 + threadIdx.x; i < I.cell0 + I.n; i += blockDim.x) {
        const double hh = h[i];
        if (!pos_finite(hh)) {
            bad = true;
            continue;
        }
        const double u = fabs(q[i] / hh);
        const double e = m[i] / (hh * hh);
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

// Separator systems of a batch: one warp per instance, cyclic system of the
// instance's blocks (at most SEP_ROWS of them).
__global__ void __launch_bounds__(32) k_sep_batched(const MixedParams p, int reset_speed) {
    const int k = blockIdx.x;
    const InstInfo I = p.inst[k];
    if (reset_speed && threadIdx.x == 0) p.speeds[k] = 0.0;
    warp_cyclic_solve((int)I.P, BlkRowsT<float>{p.blk + (int64_t)I.blk0 * BLK_STRIDE, I.P},
                      p.s + I.blk0, p.err);
}

}  // namespace hsgn
