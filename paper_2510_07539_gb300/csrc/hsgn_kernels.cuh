// hsgn_kernels.cuh -- CUDA kernels of one semi-implicit IMEX stage (sm_103a).
//
// Paper: Macca, Boscheri, Ricchiuto, arXiv 2510.07539.
//   stage update:  Sec. 4.2, eq. (GN_hyp_eq_semi_fully_discrete)
//   fluxes:        Sec. 4.1 (Rusanov flux hat D_x, centred linear reconstruction)
//   coefficients:  eqs. (eq:hSGN_alpha), (eq:b1), (eq:hnew)
//   stage states:  Sec. 3.2, eq. (tableau) in its efficient form
//
// One stage is three launches:
//   k_stage_assemble  one CTA per block of rows: loads the two stage inputs
//                     with a 3-cell halo, forms U_l and U_b on load, computes
//                     face fluxes, starred values, coefficients and matrix rows
//                     in shared memory, and eliminates the block (separator
//                     method, hsgn_tridiag.cuh). Stores per row (y, v, w) and
//                     the back-substitution inputs; per block a summary row.
//   k_reduced_cyclic  one CTA: the cyclic system of the block separators.
//   k_backsub         one thread per cell: hbar = y - s_L v - s_R w, then
//                     qbar, (h eta)bar, (h w)bar.
#pragma once

#include <cstdint>

#include "hsgn_tridiag.cuh"

namespace hsgn {

constexpr int BC_PERIODIC = 0;
constexpr int BC_TRANSMISSIVE = 1;

// Number of doubles in a block summary: separator row (a, b, c, d), then the
// triples of the first row (F) and of the last interior row (L).
constexpr int BLK_STRIDE = 10;

// Neighbour index for offsets |i - j| <= n of an in-range j (all stencils here
// reach at most 3 cells and n >= 3): one conditional add or subtract.
__device__ __forceinline__ int64_t wrap_index(int64_t i, int64_t n, int bc) {
    if (bc == BC_PERIODIC) return i < 0 ? i + n : (i >= n ? i - n : i);
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}


// Even split of n rows into P blocks: block b starts at b*base + min(b, rem)
// and has base + (b < rem) rows.
struct BlockSplit {
    int64_t n, base;
    int32_t P, rem;
    __host__ __device__ int64_t start(int64_t b) const { return b * base + (b < rem ? b : rem); }
    __host__ __device__ int64_t size(int64_t b) const { return base + (b < rem ? 1 : 0); }
    __host__ __device__ int64_t block_of(int64_t i) const {
        const int64_t big = (int64_t)rem * (base + 1);
        if (n < ((int64_t)1 << 31)) {  // 32-bit division is several times cheaper
            const unsigned ui = (unsigned)i, ub = (unsigned)base, ubig = (unsigned)big;
            return ui < ubig ? ui / (ub + 1u) : (unsigned)rem + (ui - ubig) / ub;
        }
        return i < big ? i / (base + 1) : rem + (i - big) / base;
    }
    // block of row j = i - 1 or i + 1 given the block b of row i (cyclic)
    __host__ __device__ int64_t left_of(int64_t b, int64_t j) const {
        if (j < 0) return P - 1;
        return j < start(b) ? b - 1 : b;
    }
    __host__ __device__ int64_t right_of(int64_t b, int64_t j) const {
        if (j >= n) return 0;
        return j >= start(b) + size(b) ? b + 1 : b;
    }
};

struct StageParams {
    int64_t n;
    int32_t bc;
    int32_t local_speed;  // 1: Rusanov speed max(|u^L|,|u^R|); 0: global *speed
    double dx, g, lam, tau;
    const double* A[4];  // first input state (h, q, m, r)
    const double* B[4];  // second input state, may be null when wl1 == wb1 == 0
    double wl0, wl1;     // U_l = wl0 A + wl1 B   (linearisation state)
    double wb0, wb1;     // U_b = wb0 A + wb1 B   (base state)
    const double* C[4];  // optional third state (null: none): U_l += wl2 C
    double wl2;
    int32_t recon;       // 1: centred linear reconstruction; 0: none (first order)
    const double* speed; // device scalar: global Rusanov speed of the step
    BlockSplit split;
    // per-row outputs
    double *y, *v, *w;
    double *qs, *ms, *rs, *be, *de;
    double* blk;          // P * BLK_STRIDE
    unsigned* err;
    // well-balanced bathymetry form: bottom per cell, face forces Phi_{i+1/2}
    const double* bathy;
    double* phi;
};

// Arrays of the well-balanced form only; empty for the flat-bottom kernel so
// that its shared memory (and occupancy) is unchanged.
template <int S, bool WB>
struct WbShared {
    double bb[S + 6];             // bottom, cells -3 .. S+2
    double ph[S + 2], pt[S + 2];  // p^ and p~, cells -1 .. S
    double Phi[S + 1];            // faces -1/2 .. S-1/2
};
template <int S>
struct WbShared<S, false> {};

// Shared memory of k_stage_assemble for blocks of at most S = T*M rows.
template <int T, int M, bool WB = false>
struct AssembleShared {
    static constexpr int S = T * M;
    double hl[S + 6], ql[S + 6], ml[S + 6], rl[S + 6];  // U_l, cells -3 .. S+2
    double hb[S + 6], qb[S + 6], mb[S + 6], rb[S + 6];  // U_b, same indexing
    double Fq[S + 3], Fm[S + 3], Fr[S + 3];             // faces -2 .. S
    double qs[S + 2], ms[S + 2], rs[S + 2], be[S + 2], de[S + 2];  // cells -1 .. S
    SepShared<T> sep;
    double lastrow[4];
    WbShared<S, WB> wb;
};

// T threads per CTA, M rows per thread in the block elimination. WB selects
// the well-balanced bathymetry form (the printed flat scheme otherwise).
template <int T, int M, int BC, bool WB>
__global__ void __launch_bounds__(T) k_stage_assemble(const StageParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto& sm = *reinterpret_cast<AssembleShared<T, M, WB>*>(smem_raw);
    const int tid = threadIdx.x;
    const int64_t b = blockIdx.x;
    const int64_t r0 = p.split.start(b);
    const int nb = (int)p.split.size(b);
    const int64_t n = p.n;
    const bool two = (p.B[0] != nullptr);
    const bool three = (p.C[0] != nullptr);

    // ---- 0. stage inputs with a 3-cell halo; U_l and U_b formed on load
    for (int j = tid; j < nb + 6; j += T) {
        const int64_t gi = wrap_index(r0 + j - 3, n, BC);
        const double ah = p.A[0][gi], aq = p.A[1][gi], am = p.A[2][gi], ar = p.A[3][gi];
        if (two) {
            const double bh = p.B[0][gi], bq = p.B[1][gi], bm = p.B[2][gi], br = p.B[3][gi];
            sm.hl[j] = p.wl0 * ah + p.wl1 * bh;
            sm.ql[j] = p.wl0 * aq + p.wl1 * bq;
            sm.ml[j] = p.wl0 * am + p.wl1 * bm;
            sm.rl[j] = p.wl0 * ar + p.wl1 * br;
            sm.hb[j] = p.wb0 * ah + p.wb1 * bh;
            sm.qb[j] = p.wb0 * aq + p.wb1 * bq;
            sm.mb[j] = p.wb0 * am + p.wb1 * bm;
            sm.rb[j] = p.wb0 * ar + p.wb1 * br;
        } else {
            sm.hl[j] = ah; sm.ql[j] = aq; sm.ml[j] = am; sm.rl[j] = ar;
            sm.hb[j] = ah; sm.qb[j] = aq; sm.mb[j] = am; sm.rb[j] = ar;
        }
        if (three) {
            sm.hl[j] = fma(p.wl2, p.C[0][gi], sm.hl[j]);
            sm.ql[j] = fma(p.wl2, p.C[1][gi], sm.ql[j]);
            sm.ml[j] = fma(p.wl2, p.C[2][gi], sm.ml[j]);
            sm.rl[j] = fma(p.wl2, p.C[3][gi], sm.rl[j]);
        }
        if constexpr (WB) sm.wb.bb[j] = p.bathy ? p.bathy[gi] : 0.0;
    }
    __syncthreads();

    const double dx = p.dx, tau = p.tau, lam = p.lam, g = p.g;
    const double gspeed = p.local_speed ? 0.0 : *p.speed;
    unsigned bad = 0;

    // ---- 1. Rusanov fluxes at faces f = -2 .. nb (face f between cells f, f+1),
    //         centred unlimited reconstruction of the conserved variables of U_l.
    for (int j = tid; j < nb + 3; j += T) {
        const int c = j;  // face f = j-2; its stencil cells f-1 .. f+2 sit at smem j .. j+3
        const double hm = sm.hl[c], h0 = sm.hl[c + 1], h1 = sm.hl[c + 2], h2 = sm.hl[c + 3];
        const double qm = sm.ql[c], q0 = sm.ql[c + 1], q1 = sm.ql[c + 2], q2 = sm.ql[c + 3];
        const double mm = sm.ml[c], m0 = sm.ml[c + 1], m1 = sm.ml[c + 2], m2 = sm.ml[c + 3];
        const double rm = sm.rl[c], r0_ = sm.rl[c + 1], r1 = sm.rl[c + 2], r2 = sm.rl[c + 3];
        const double sl = p.recon ? 0.25 : 0.0;  // reconstruction slope factor
        const double hL = fma(sl, h1 - hm, h0), hR = fma(-sl, h2 - h0, h1);
        const double qL = fma(sl, q1 - qm, q0), qR = fma(-sl, q2 - q0, q1);
        const double mL = fma(sl, m1 - mm, m0), mR = fma(-sl, m2 - m0, m1);
        const double rL = fma(sl, r1 - rm, r0_), rR = fma(-sl, r2 - r0_, r1);
        if (!pos_finite(hL) || !pos_finite(hR)) bad |= HSGN_DEV_ERR_DEPTH;
        const double ip = rcp(hL * hR);  // one reciprocal for both velocities
        const double uL = qL * hR * ip, uR = qR * hL * ip;
        const double s = p.local_speed ? fmax(fabs(uL), fabs(uR)) : gspeed;
        sm.Fq[j] = 0.5 * (fma(uL, qL, uR * qR) - s * (qR - qL));
        sm.Fm[j] = 0.5 * (fma(uL, mL, uR * mR) - s * (mR - mL));
        sm.Fr[j] = 0.5 * (fma(uL, rL, uR * rR) - s * (rR - rL));
    }
    __syncthreads();

    // ---- 2. starred values and coefficients at cells c = -1 .. nb
    const double lt2 = lam * tau * tau;
    const double tdx = tau / dx;
    for (int j = tid; j < nb + 2; j += T) {
        const int c3 = j + 2;  // smem index of cell c = j-1 in the U arrays
        const double rsv = fma(-tdx, sm.Fr[j + 1] - sm.Fr[j], sm.rb[c3]) + lam * tau;
        double msv = fma(tau, rsv, fma(-tdx, sm.Fm[j + 1] - sm.Fm[j], sm.mb[c3]));
        if constexpr (WB)  // -(3/2) h u b_x of the (h eta) equation (Sec. 2.3, eq. (hSGNb_eq)), from U_l
            msv -= tau * 1.5 * sm.ql[c3] * (sm.wb.bb[c3 + 1] - sm.wb.bb[c3 - 1]) / (2.0 * dx);
        const double qsv = fma(-tdx, sm.Fq[j + 1] - sm.Fq[j], sm.qb[c3]);
        // coefficients with one reciprocal R = 1/(h (h^2 + lambda tau^2)):
        //   1/h = (h^2 + lambda tau^2) R,  1/beta_1 = h^2/(h^2 + lambda tau^2) = h^3 R,
        //   beta_2 = 2 lambda tau^2 h / (h^2 + lambda tau^2)^2
        const double h = sm.hl[c3];
        if (!pos_finite(h)) bad |= HSGN_DEV_ERR_DEPTH;
        const double Dh = fma(h, h, lt2);
        const double R = rcp(h * Dh);
        const double ih = Dh * R;
        const double iD = h * R;
        const double eta = sm.ml[c3] * ih;
        const double e = eta * ih;
        const double alpha = fma(2.0, e, -1.0) * ih * (-1.0 / 3.0);
        const double c2 = fma(g, h, (lam * (1.0 / 3.0)) * e * e);
        const double a2 = fma(-lam * eta, alpha, c2);
        const double ib1 = h * h * iD;
        const double beta2 = (2.0 * lt2) * h * iD * iD;
        const double beta = fma(lam * alpha * beta2, msv, a2);
        if (!pos_finite(beta)) bad |= HSGN_DEV_ERR_COERCIVE;
        sm.qs[j] = qsv;
        sm.ms[j] = msv;
        sm.rs[j] = rsv;
        sm.be[j] = beta;
        sm.de[j] = alpha * ib1;
        if constexpr (WB) {
            // p^ = p(h_l, m_l) + lambda alpha (m^dag b_1(h_l) - m_l), p = g h^2/2 + eta p~,
            // p~ = (lambda/3)(1 - eta/h) (e = eta/h), b_1 = h^2 / (h^2 + lambda tau^2)
            const double ptil = (lam * (1.0 / 3.0)) * (1.0 - e);
            sm.wb.pt[j] = ptil;
            sm.wb.ph[j] = fma(0.5 * g * h, h, eta * ptil) + lam * alpha * fma(msv, h * h * iD, -sm.ml[c3]);
        }
    }
    __syncthreads();
    if (BC == BC_TRANSMISSIVE && tid == 0) {
        // zero-order ghost copies of the per-cell quantities at the domain ends
        if (r0 == 0) {
            sm.qs[0] = sm.qs[1]; sm.ms[0] = sm.ms[1]; sm.rs[0] = sm.rs[1];
            sm.be[0] = sm.be[1]; sm.de[0] = sm.de[1];
        }
        if (r0 + nb == n) {
            sm.qs[nb + 1] = sm.qs[nb]; sm.ms[nb + 1] = sm.ms[nb]; sm.rs[nb + 1] = sm.rs[nb];
            sm.be[nb + 1] = sm.be[nb]; sm.de[nb + 1] = sm.de[nb];
        }
    }
    __syncthreads();

    if constexpr (WB) {
        // explicit face forces Phi_{f+1/2}, f = -1 .. nb-1 (smem index f+1):
        //   p^ jump + (g h + (3/2) p~)_{face} (b jump) - beta_{face} (h_l jump).
        // Transmissive: both cells of an end face are the same ghost copy, so
        // every jump and Phi vanish there.
        for (int f1 = tid; f1 < nb + 1; f1 += T) {
            const int c0 = f1, c1 = f1 + 1;        // cells f, f+1 in the -1 .. nb arrays
            const int u0 = f1 + 2, u1 = f1 + 3;    // the same cells in the U_l arrays
            const double db = sm.wb.bb[u1] - sm.wb.bb[u0];
            const double dhl = sm.hl[u1] - sm.hl[u0];
            const double hbar_f = 0.5 * (sm.hl[u0] + sm.hl[u1]);
            const double ptf = 0.5 * (sm.wb.pt[c0] + sm.wb.pt[c1]);
            const double bf = 0.5 * (sm.be[c0] + sm.be[c1]);
            double phi = (sm.wb.ph[c1] - sm.wb.ph[c0]) + fma(g, hbar_f, 1.5 * ptf) * db - bf * dhl;
            if (BC == BC_TRANSMISSIVE) {
                const int64_t gf = r0 + f1 - 1;    // face between global cells gf, gf+1
                if (gf < 0 || gf + 1 > n - 1) phi = 0.0;
            }
            sm.wb.Phi[f1] = phi;
        }
        __syncthreads();
        for (int i = tid; i < nb; i += T) p.phi[r0 + i] = sm.wb.Phi[i + 1];
    }

    // back-substitution inputs of the block's own rows
    for (int i = tid; i < nb; i += T) {
        const int64_t gi = r0 + i;
        p.qs[gi] = sm.qs[i + 1];
        p.ms[gi] = sm.ms[i + 1];
        p.rs[gi] = sm.rs[i + 1];
        p.be[gi] = sm.be[i + 1];
        p.de[gi] = sm.de[i + 1];
    }

    // ---- 3. rows of Delta[hbar] = h^dagger and the block elimination
    const double Cc = tau * tau / (dx * dx);
    const double fq = tau / (2.0 * dx);
    const double fd = lam * tau * tau / (dx * dx);
    auto row = [&](int i, double& a, double& bb, double& c, double& d) {
        const double bm = 0.5 * (sm.be[i] + sm.be[i + 1]);
        const double bp = 0.5 * (sm.be[i + 1] + sm.be[i + 2]);
        const double dm = 0.5 * (sm.de[i] + sm.de[i + 1]);
        const double dp = 0.5 * (sm.de[i + 1] + sm.de[i + 2]);
        const double msc = sm.ms[i + 1];
        if constexpr (WB)
            d = fma(-fq, sm.qs[i + 2] - sm.qs[i], sm.hb[i + 3]) + Cc * (sm.wb.Phi[i + 1] - sm.wb.Phi[i]);
        else
            d = fma(-fq, sm.qs[i + 2] - sm.qs[i], sm.hb[i + 3]) +
                fd * (dp * (sm.ms[i + 2] - msc) - dm * (msc - sm.ms[i]));
        a = -Cc * bm;
        c = -Cc * bp;
        bb = fma(Cc, bm + bp, 1.0);
        if (BC == BC_TRANSMISSIVE) {
            const int64_t gi = r0 + i;
            if (gi == 0) { bb = fma(Cc, bp, 1.0); a = 0.0; }
            if (gi == n - 1) { bb = fma(Cc, bm, 1.0); c = 0.0; }
        }
    };
    double y[M], v[M], w[M], last[4];
    int cs, m;
    cta_block_solve<T, M>(nb, row, sm.sep, y, v, w, cs, m, last, p.err);
    // ---- 4. stage (y, v, w) in the U_l arrays, which the row function no
    //         longer reads, for coalesced stores
    __syncthreads();
#pragma unroll
    for (int k = 0; k < M; ++k) {
        if (k < m) {
            sm.hl[cs + k] = y[k];
            sm.ql[cs + k] = v[k];
            sm.ml[cs + k] = w[k];
        }
    }
    if (m > 0 && cs + m == nb) {
        sm.lastrow[0] = last[0]; sm.lastrow[1] = last[1];
        sm.lastrow[2] = last[2]; sm.lastrow[3] = last[3];
    }
    if (bad) flag_error(p.err, bad);
    __syncthreads();
    for (int i = tid; i < nb; i += T) {
        p.y[r0 + i] = sm.hl[i];
        p.v[r0 + i] = sm.ql[i];
        p.w[r0 + i] = sm.ml[i];
    }
    if (tid == 0) {
        double* s = p.blk + b * BLK_STRIDE;
        s[0] = sm.lastrow[0]; s[1] = sm.lastrow[1]; s[2] = sm.lastrow[2]; s[3] = sm.lastrow[3];
        s[4] = sm.hl[0]; s[5] = sm.ql[0]; s[6] = sm.ml[0];
        if (nb >= 2) {
            s[7] = sm.hl[nb - 2]; s[8] = sm.ql[nb - 2]; s[9] = sm.ml[nb - 2];
        } else {
            s[7] = 0.0; s[8] = -1.0; s[9] = 0.0;
        }
    }
}

// Row source of the block-separator system: row b couples s_{b-1}, s_b, s_{b+1}
// (cyclic in b). With x_{sep-1} = y_L - s_{b-1} v_L - s_b w_L (last interior
// row of block b) and x_{sep+1} = y_F - s_b v_F - s_{b+1} w_F (first row of
// block b+1), the separator row a x_{sep-1} + b x_sep + c x_{sep+1} = d gives
//   (-a v_L) s_{b-1} + (b - a w_L - c v_F) s_b + (-c w_F) s_{b+1} = d - a y_L - c y_F.
template <class R>
struct BlkRowsT {
    using Real = R;
    const R* blk;
    int64_t P;
    __device__ void operator()(int64_t i, R& A, R& B, R& C, R& D) const {
        const R* s = blk + i * BLK_STRIDE;
        const R* f = blk + (i + 1 == P ? 0 : i + 1) * BLK_STRIDE;
        const R a = s[0], bb = s[1], c = s[2], d = s[3];
        A = -a * s[8];
        B = bb - a * s[9] - c * f[5];
        C = -c * f[6];
        D = d - a * s[7] - c * f[4];
    }
};
using BlkRows = BlkRowsT<double>;

// Row source reading explicit arrays (cyclic: a[0] couples x[n-1], c[n-1] couples x[0]).
struct ArrayRows {
    using Real = double;
    const double *a, *b, *c, *d;
    int periodic;
    int64_t n;  // total rows of the system
    __device__ void operator()(int64_t k, double& A, double& B, double& C, double& D) const {
        A = a[k];
        B = b[k];
        C = c[k];
        D = d[k];
        if (!periodic) {
            if (k == 0) A = 0.0;
            if (k == n - 1) C = 0.0;
        }
    }
};

// Rows per block of the separator levels: one warp, 4 rows per lane (short
// dependent chains: these small systems are latency-bound, not throughput-bound).
constexpr int SEP_MS = 4;
constexpr int SEP_ROWS = 32 * SEP_MS;

// Cyclic tridiagonal system of nrows <= SEP_ROWS rows in one warp. The last
// row's unknown x_{n-1} is the external unknown on BOTH sides of rows
// 0 .. n-2 (the cyclic couplings a_0 and c_{n-2}), so x_i = y_i - x_{n-1}
// (v_i + w_i), and the last row a x_{n-2} + b x_{n-1} + c x_0 = d closes it.
template <class RowSrc>
__device__ __forceinline__ void warp_cyclic_solve(int nrows, RowSrc rows,
                                                  typename RowSrc::Real* x, unsigned* err) {
    using Real = typename RowSrc::Real;
    __shared__ Real sh[8];
    const int t = threadIdx.x;
    if (nrows == 1) {
        if (t == 0) {
            Real A, B, C, D;
            rows(0, A, B, C, D);
            const Real den = A + B + C;
            if (!pos_finite(den)) flag_error(err, HSGN_DEV_ERR_COERCIVE);
            x[0] = D / den;
        }
        return;
    }
    Real y[SEP_MS], v[SEP_MS], w[SEP_MS], last[4];
    int cs, m;
    auto rf = [&](int i, Real& A, Real& B, Real& C, Real& D) { rows(i, A, B, C, D); };
    warp_block_solve<SEP_MS>(nrows, rf, y, v, w, cs, m, last, err);
#pragma unroll
    for (int k = 0; k < SEP_MS; ++k) {
        if (k < m) {
            const int i = cs + k;
            if (i == 0) { sh[0] = y[k]; sh[1] = v[k] + w[k]; }
            if (i == nrows - 2) { sh[2] = y[k]; sh[3] = v[k] + w[k]; }
        }
    }
    if (m > 0 && cs + m == nrows) {
        sh[4] = last[0]; sh[5] = last[1]; sh[6] = last[2]; sh[7] = last[3];
    }
    __syncwarp();
    const Real a = sh[4], b = sh[5], c = sh[6], d = sh[7];
    const Real den = b - a * sh[3] - c * sh[1];
    if (t == 0 && !pos_finite(den)) flag_error(err, HSGN_DEV_ERR_COERCIVE);
    const Real xl = (d - a * sh[2] - c * sh[0]) / den;
#pragma unroll
    for (int k = 0; k < SEP_MS; ++k) {
        if (k < m) {
            const int i = cs + k;
            x[i] = (i == nrows - 1) ? xl : y[k] - xl * (v[k] + w[k]);
        }
    }
}

template <class RowSrc>
__global__ void __launch_bounds__(32) k_cyclic_onewarp(int nrows, RowSrc rows,
                                                      typename RowSrc::Real* x,
                                                      double* speed_reset, unsigned* err) {
    if (speed_reset && threadIdx.x == 0) *speed_reset = 0.0;
    warp_cyclic_solve(nrows, rows, x, err);
}

// Cyclic system of at most T*M rows in one CTA (the CTA block machinery); used
// for the single-precision separator systems, where the parallel cyclic
// reduction over T chunk separators is cheap.
template <int T, int M, class RowSrc>
__global__ void __launch_bounds__(T) k_cyclic_onecta(int nrows, RowSrc rows,
                                                     typename RowSrc::Real* x,
                                                     double* speed_reset, unsigned* err) {
    using Real = typename RowSrc::Real;
    __shared__ SepShared<T, Real> sep;
    __shared__ Real sh[8];
    const int t = threadIdx.x;
    if (speed_reset && t == 0) *speed_reset = 0.0;
    if (nrows == 1) {
        if (t == 0) {
            Real A, B, C, D;
            rows(0, A, B, C, D);
            const Real den = A + B + C;
            if (!pos_finite(den)) flag_error(err, HSGN_DEV_ERR_COERCIVE);
            x[0] = D / den;
        }
        return;
    }
    Real y[M], v[M], w[M], last[4];
    int cs, m;
    auto rf = [&](int i, Real& A, Real& B, Real& C, Real& D) { rows(i, A, B, C, D); };
    cta_block_solve<T, M>(nrows, rf, sep, y, v, w, cs, m, last, err);
#pragma unroll
    for (int k = 0; k < M; ++k) {
        if (k < m) {
            const int i = cs + k;
            if (i == 0) { sh[0] = y[k]; sh[1] = v[k] + w[k]; }
            if (i == nrows - 2) { sh[2] = y[k]; sh[3] = v[k] + w[k]; }
        }
    }
    if (m > 0 && cs + m == nrows) {
        sh[4] = last[0]; sh[5] = last[1]; sh[6] = last[2]; sh[7] = last[3];
    }
    __syncthreads();
    const Real a = sh[4], b = sh[5], c = sh[6], d = sh[7];
    const Real den = b - a * sh[3] - c * sh[1];
    if (t == 0 && !pos_finite(den)) flag_error(err, HSGN_DEV_ERR_COERCIVE);
    const Real xl = (d - a * sh[2] - c * sh[0]) / den;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        if (k < m) {
            const int i = cs + k;
            x[i] = (i == nrows - 1) ? xl : y[k] - xl * (v[k] + w[k]);
        }
    }
}

// One level of the multi-block elimination of a row source: one warp per
// block of at most SEP_ROWS rows; per row (y, v, w) and a block summary.
template <class Real>
struct ReduceShared {
    Real ys[SEP_ROWS], vs[SEP_ROWS], ws[SEP_ROWS];
    Real lastrow[4];
};

template <class RowSrc>
__global__ void __launch_bounds__(32) k_block_reduce(RowSrc rows, BlockSplit split,
                                                     typename RowSrc::Real* yo,
                                                     typename RowSrc::Real* vo,
                                                     typename RowSrc::Real* wo,
                                                     typename RowSrc::Real* blk, unsigned* err) {
    using Real = typename RowSrc::Real;
    __shared__ ReduceShared<Real> sh;
    const int64_t b = blockIdx.x;
    const int64_t r0 = split.start(b);
    const int nb = (int)split.size(b);
    auto rf = [&](int i, Real& A, Real& B, Real& C, Real& D) { rows(r0 + i, A, B, C, D); };
    Real y[SEP_MS], v[SEP_MS], w[SEP_MS], last[4];
    int cs, m;
    warp_block_solve<SEP_MS>(nb, rf, y, v, w, cs, m, last, err);
#pragma unroll
    for (int k = 0; k < SEP_MS; ++k) {
        if (k < m) {
            sh.ys[cs + k] = y[k];
            sh.vs[cs + k] = v[k];
            sh.ws[cs + k] = w[k];
        }
    }
    if (m > 0 && cs + m == nb) {
        sh.lastrow[0] = last[0]; sh.lastrow[1] = last[1];
        sh.lastrow[2] = last[2]; sh.lastrow[3] = last[3];
    }
    __syncwarp();
    for (int i = threadIdx.x; i < nb; i += 32) {
        yo[r0 + i] = sh.ys[i];
        vo[r0 + i] = sh.vs[i];
        wo[r0 + i] = sh.ws[i];
    }
    if (threadIdx.x == 0) {
        Real* s = blk + b * BLK_STRIDE;
        s[0] = sh.lastrow[0]; s[1] = sh.lastrow[1]; s[2] = sh.lastrow[2]; s[3] = sh.lastrow[3];
        s[4] = sh.ys[0]; s[5] = sh.vs[0]; s[6] = sh.ws[0];
        if (nb >= 2) {
            s[7] = sh.ys[nb - 2]; s[8] = sh.vs[nb - 2]; s[9] = sh.ws[nb - 2];
        } else {
            s[7] = Real(0); s[8] = Real(-1); s[9] = Real(0);
        }
    }
}

// x_i = y_i - s_{b-1} v_i - s_b w_i for every row of a multi-block solve.
template <class Real>
__global__ void k_block_backout(BlockSplit split, const Real* y, const Real* v, const Real* w,
                                const Real* s, Real* x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= split.n) return;
    const int64_t b = split.block_of(i);
    const Real sl = s[b == 0 ? split.P - 1 : b - 1];
    const Real sr = s[b];
    x[i] = y[i] - sl * v[i] - sr * w[i];
}

struct BacksubParams {
    int64_t n;
    int32_t bc;
    int32_t track_speed;  // 1: atomically fold max |u| of the result into *speed
    double dx, lam, tau;
    BlockSplit split;
    const double *y, *v, *w, *s;
    const double *qs, *ms, *rs, *be, *de;
    const double* phi;    // face forces Phi_{i+1/2} (well-balanced form)
    double* out[4];
    double* speed;
    unsigned* err;
};

__device__ __forceinline__ double hbar_at(const BacksubParams& p, int64_t i, int64_t b) {
    const double sl = p.s[b == 0 ? p.split.P - 1 : b - 1];
    const double sr = p.s[b];
    return p.y[i] - sl * p.v[i] - sr * p.w[i];
}

// Back-substitution of Sec. 4.2 (the fourth equation with h^2 implicit, the
// "second version" of Sec. 6.3.1):
//   qbar = q^dag - tau/(2dx) beta (hbar_{i+1} - hbar_{i-1})
//                - lambda tau/(2dx) delta (m^dag_{i+1} - m^dag_{i-1}),
//   mbar = m^dag / (1 + lambda tau^2 / hbar^2),  rbar = r^dag - lambda tau mbar / hbar^2,
// i.e. with D = hbar^2 + lambda tau^2: mbar = m^dag hbar^2 / D, rbar = r^dag - lambda tau m^dag / D.
// The neighbours' hbar come from the adjacent lanes; the lanes at the ends of
// a warp compute their outer neighbour themselves.
template <int BC, bool WB>
__global__ void k_backsub(const BacksubParams p) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool live = i < p.n;
    const int64_t bi = live ? p.split.block_of(i) : 0;
    const double h = live ? hbar_at(p, i, bi) : 0.0;
    const double hl_s = __shfl_up_sync(0xffffffffu, h, 1);
    const double hr_s = __shfl_down_sync(0xffffffffu, h, 1);
    double umax = 0.0;
    if (live) {
        const int64_t il = wrap_index(i - 1, p.n, BC), ir = wrap_index(i + 1, p.n, BC);
        // block of the neighbour actually used: the next block, the same cell
        // (transmissive clamp) or the cyclic wrap
        const int64_t bl = il == i - 1 ? p.split.left_of(bi, i - 1) : (il == i ? bi : p.split.P - 1);
        const int64_t br = ir == i + 1 ? p.split.right_of(bi, i + 1) : (ir == i ? bi : 0);
        const double hl = (lane == 0 || il != i - 1) ? hbar_at(p, il, bl) : hl_s;
        const double hr = (lane == 31 || ir != i + 1) ? hbar_at(p, ir, br) : hr_s;
        const double fq = p.tau / (2.0 * p.dx);
        double q;
        if constexpr (WB) {
            // q = q^dag - tau/(2dx) (F_{i+1/2} + F_{i-1/2}), F = Phi + beta_{face} (hbar jump)
            const double phr = p.phi[i];
            const double phl = (i > 0) ? p.phi[i - 1] : (BC == BC_PERIODIC ? p.phi[p.n - 1] : 0.0);
            const double Fp = fma(0.5 * (p.be[i] + p.be[ir]), hr - h, phr);
            const double Fm = fma(0.5 * (p.be[il] + p.be[i]), h - hl, phl);
            q = p.qs[i] - fq * (Fp + Fm);
        } else {
            q = p.qs[i] - fq * p.be[i] * (hr - hl) - p.lam * fq * p.de[i] * (p.ms[ir] - p.ms[il]);
        }
        const double h2 = h * h;
        const double D = fma(h, h, p.lam * p.tau * p.tau);
        const double R = rcp(h * D);  // 1/D = h R, 1/h = D R
        const double iD = h * R;
        const double msv = p.ms[i];
        const double m = msv * h2 * iD;
        const double r = p.rs[i] - p.lam * p.tau * msv * iD;
        unsigned bad = 0;
        if (!pos_finite(h)) bad |= HSGN_DEV_ERR_DEPTH;
        if (!finite_bits(q) || !finite_bits(m) || !finite_bits(r)) bad |= HSGN_DEV_ERR_NONFINITE;
        if (bad) flag_error(p.err, bad);
        p.out[0][i] = h;
        p.out[1][i] = q;
        p.out[2][i] = m;
        p.out[3][i] = r;
        if (p.track_speed && !bad) umax = fabs(q * (D * R));
    }
    if (p.track_speed) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) umax = fmax(umax, __shfl_xor_sync(0xffffffffu, umax, o));
        if (lane == 0 && umax > 0.0)
            atomicMax(reinterpret_cast<unsigned long long*>(p.speed),
                      (unsigned long long)__double_as_longlong(umax));
    }
}

// ---------------------------------------------------------------------------
// Explicit hSGN operator (Sec. 4.4, eq. (GN_hyp_eq_explicit)) at the state Us,
//   L_h = -D_x(q),  L_q = -hat D_x(q u) - a^2 D_x(h) - lambda alpha D_x(h eta),
//   L_m = -hat D_x(h u eta) + h w,  L_r = -hat D_x(h u w) - lambda ((h eta)/h^2 - 1),
// D_x central over 2 dx, hat D_x the Rusanov difference of the (reconstructed)
// face fluxes. One thread per cell; each face flux is evaluated by both of its
// cells. Writes out1 = a1 U0 + b1 Us + c1 L(Us) and, if out2 is set, out2 =
// a2 U0 + b2 Us + c2 L(Us) (U0 is read at the own cell only, so out1 may
// alias U0); Euler, Heun and the explicit stage of ARS(2,2,2) are
// combinations of this form.
// ---------------------------------------------------------------------------
struct ExplicitParams {
    int64_t n;
    int32_t recon;        // 1: centred linear reconstruction; 0: none
    int32_t local_speed;  // 1: Rusanov speed max(|u^L|,|u^R|); 0: global *speed
    int32_t track_speed;  // 1: fold max |u| of out1 into *speed_next
    int32_t spectral;     // with track_speed: fold max(|u| + c) instead (explicit schemes)
    double dx, g, lam;
    double idx, i2dx;     // 1/dx, 1/(2 dx)
    const double* Us[4];
    const double* U0[4];  // may be null when a1 == a2 == 0
    double a1, b1, c1, a2, b2, c2;
    double* out1[4];
    double* out2[4];      // may be null
    const double* speed;
    double* speed_next;
    unsigned* err;
};

// Rusanov fluxes of q u, h u eta, h u w at the face between cells 0 and 1
// from cells -1 .. 2 (Sec. 4.1).
__device__ __forceinline__ void explicit_face(const double* h, const double* q, const double* m,
                                              const double* r, double sl, bool local,
                                              double gspeed, double& Fq, double& Fm, double& Fr,
                                              unsigned& bad) {
    const double hL = fma(sl, h[2] - h[0], h[1]), hR = fma(-sl, h[3] - h[1], h[2]);
    const double qL = fma(sl, q[2] - q[0], q[1]), qR = fma(-sl, q[3] - q[1], q[2]);
    const double mL = fma(sl, m[2] - m[0], m[1]), mR = fma(-sl, m[3] - m[1], m[2]);
    const double rL = fma(sl, r[2] - r[0], r[1]), rR = fma(-sl, r[3] - r[1], r[2]);
    if (!pos_finite(hL) || !pos_finite(hR)) bad |= HSGN_DEV_ERR_DEPTH;
    const double ip = rcp(hL * hR);
    const double uL = qL * hR * ip, uR = qR * hL * ip;
    const double s = local ? fmax(fabs(uL), fabs(uR)) : gspeed;
    Fq = 0.5 * (fma(uL, qL, uR * qR) - s * (qR - qL));
    Fm = 0.5 * (fma(uL, mL, uR * mR) - s * (mR - mL));
    Fr = 0.5 * (fma(uL, rL, uR * rR) - s * (rR - rL));
}

// One CTA of ET threads per ET consecutive cells: cells -2 .. ET+1 of the
// block are staged in shared memory, each of the ET+1 faces is evaluated once.
constexpr int ET = 256;

template <int BC>
__global__ void __launch_bounds__(ET) k_explicit(const ExplicitParams p) {
    __shared__ double sh[4][ET + 4];      // cells c0-2 .. c0+ET+1
    __shared__ double sf[3][ET + 1];      // faces c0-1/2 .. c0+ET-1/2
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int64_t c0 = (int64_t)blockIdx.x * ET;
    const int64_t n = p.n;
    for (int j = tid; j < ET + 4; j += ET) {
        const int64_t c = wrap_index(c0 + j - 2 < 2 * n ? c0 + j - 2 : n - 1, n, BC);
        sh[0][j] = p.Us[0][c];
        sh[1][j] = p.Us[1][c];
        sh[2][j] = p.Us[2][c];
        sh[3][j] = p.Us[3][c];
    }
    __syncthreads();
    unsigned bad = 0;
    const double sl = p.recon ? 0.25 : 0.0;
    const bool local = p.local_speed != 0;
    const double gspeed = local ? 0.0 : *p.speed;
    for (int f = tid; f < ET + 1; f += ET) {  // face f - 1/2 of the block: cells f-2 .. f+1
        double Fq, Fm, Fr;
        explicit_face(&sh[0][f], &sh[1][f], &sh[2][f], &sh[3][f], sl, local, gspeed, Fq, Fm, Fr,
                      bad);
        sf[0][f] = Fq;
        sf[1][f] = Fm;
        sf[2][f] = Fr;
    }
    __syncthreads();
    const int64_t i = c0 + tid;
    double umax = 0.0;
    if (i < n) {
        const int j = tid + 2;  // own cell in sh
        const double hc = sh[0][j], hlft = sh[0][j - 1], hrgt = sh[0][j + 1];
        const double qlft = sh[1][j - 1], qrgt = sh[1][j + 1];
        const double mc = sh[2][j], mlft = sh[2][j - 1], mrgt = sh[2][j + 1];
        const double rc = sh[3][j];
        if (!pos_finite(hc)) bad |= HSGN_DEV_ERR_DEPTH;
        const double ih = rcp(hc);
        const double eta = mc * ih;
        const double e = eta * ih;
        const double alpha = fma(2.0, e, -1.0) * ih * (-1.0 / 3.0);
        const double c2 = fma(p.g, hc, (p.lam * (1.0 / 3.0)) * e * e);
        const double a2 = fma(-p.lam * eta, alpha, c2);
        const double idx = p.idx, i2dx = p.i2dx;
        double L[4];
        L[0] = -(qrgt - qlft) * i2dx;
        L[1] = -(sf[0][tid + 1] - sf[0][tid]) * idx - a2 * (hrgt - hlft) * i2dx -
               p.lam * alpha * (mrgt - mlft) * i2dx;
        L[2] = -(sf[1][tid + 1] - sf[1][tid]) * idx + rc;
        L[3] = -(sf[2][tid + 1] - sf[2][tid]) * idx - p.lam * (e - 1.0);
        const double cur[4] = {hc, sh[1][j], mc, rc};
        double o1[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double u0 = p.U0[0] ? p.U0[k][i] : 0.0;
            o1[k] = fma(p.c1, L[k], fma(p.b1, cur[k], p.a1 * u0));
            if (p.out2[0]) p.out2[k][i] = fma(p.c2, L[k], fma(p.b2, cur[k], p.a2 * u0));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) p.out1[k][i] = o1[k];
        if (!finite_bits(o1[0]) || !finite_bits(o1[1]) || !finite_bits(o1[2]) ||
            !finite_bits(o1[3]))
            bad |= HSGN_DEV_ERR_NONFINITE;
        if (p.track_speed && !bad) {
            // |u|, or the spectral radius |u| + c, c^2 = g h + (lambda/3) eta^2/h^2
            // (Sec. 2.2, eq. (eq:hSGN_eigenvalues)) of the new state
            const double ihn = rcp(o1[0]);
            umax = fabs(o1[1] * ihn);
            if (p.spectral) {
                const double en = o1[2] * ihn * ihn;
                umax += sqrt(fma(p.g, o1[0], (p.lam * (1.0 / 3.0)) * en * en));
            }
        }
    }
    if (bad) flag_error(p.err, bad);
    if (p.track_speed) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) umax = fmax(umax, __shfl_xor_sync(0xffffffffu, umax, o));
        if (lane == 0 && umax > 0.0)
            atomicMax(reinterpret_cast<unsigned long long*>(p.speed_next),
                      (unsigned long long)__double_as_longlong(umax));
    }
}

// max |u| and max nu = |u| + sqrt(g h + (lambda/3) eta^2/h^2) over the state
// (Sec. 5 time-step rule); out[0] = max |u|, out[1] = max nu. Non-negative
// doubles order like their bit patterns, so atomicMax on the bits is exact.
__global__ void k_speeds(int64_t n, const double* h, const double* q, const double* m, double g,
                         double lam, double* out, unsigned* err) {
    double um = 0.0, nm = 0.0;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double hh = h[i];
        if (!(hh > 0.0)) {
            bad = true;
            continue;
        }
        const double u = fabs(q[i] / hh);
        const double e = m[i] / (hh * hh);
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

}  // namespace hsgn
