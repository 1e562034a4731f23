// hsgn_adjoint.cuh -- discrete adjoint of one stage (FP64, well-balanced form).
//
// Given dJ/dU_out of a stage U_out = S(U_b, U_l, tau) (Sec. 4.2, eq.
// (GN_hyp_eq_semi_fully_discrete) with the bottom form of the library), the
// kernels below add dJ/dU_b, dJ/dU_l, dJ/db and dJ/ds (s the global Rusanov
// speed) to their accumulators. Each kernel reverses one group of forward
// operations, in reverse order of the forward stage:
//   k_adj_backsub   q, m, r of the back-substitution and the face forces
//                   F = Phi + beta_face (hbar jump) (one thread per cell)
//   k_adj_rows      rows of the transposed depth matrix (the matrix is
//                   symmetric) for dJ/dD = M^{-T} dJ/dhbar, solved by the
//                   library's tridiagonal solve
//   k_adj_rowsadj   dJ/dM_ij = -(dJ/dD)_i hbar_j through beta_face, and the
//                   right-hand side D (base depth, q^dag, Phi)
//   k_adj_phi       face forces Phi (p^ jumps, bottom force, beta_face dh_l)
//                   (one thread per face)
//   k_adj_cell      p^ and p~, then beta, per cell (functions of h_l, m_l, m^dag)
//   k_adj_starred   m^dag (with the bottom source), r^dag, q^dag
//   k_adj_flux      Rusanov fluxes, the reconstruction of U_l and the speed
// Scatters to a neighbour use atomicAdd (a cell or face receives at most a
// few contributions), so sums are not ordered. The forward quantities q^dag,
// m^dag, r^dag, beta come from the forward stage kernel's work arrays, hbar
// and mbar from its output; everything else is recomputed.
#pragma once

#include "hsgn_kernels.cuh"

namespace hsgn {

struct AdjParams {
    int64_t n;
    int32_t bc;
    double dx, g, lam, tau;
    const double* speed;            // global Rusanov speed of the step
    const double* Ub[4];            // base state
    const double* Ul[4];            // linearisation state
    const double* bathy;            // bottom (may be null: flat)
    const double *qs, *ms, *rs, *be;  // forward per-cell quantities
    const double *hbar, *mbar;      // forward stage output (h, h eta)
    const double* Ao[4];            // dJ/dU_out
    double* Ab[4];                  // += dJ/dU_b
    double* Al[4];                  // += dJ/dU_l
    double* Abathy;                 // += dJ/db (may be null)
    double* Aspeed;                 // += dJ/ds (device scalar)
    // work (zeroed before the first kernel): per cell
    double *qs_a, *ms_a, *rs_a, *be_a, *ph_a, *pt_a, *hbar_a, *D_a;
    double *ra, *rb, *rc;           // rows of the transposed matrix
    // per face index k+1 (face k+1/2, k = -1 .. n-1): n+1 entries
    double *Phi_a, *Fq_a, *Fm_a, *Fr_a;
};

template <int BC>
__device__ __forceinline__ int64_t adj_nb(int64_t i, int64_t n) {
    return wrap_index(i, n, BC);
}

// ---- back-substitution: r = r^dag - lambda tau m/h^2, m = m^dag h^2/(h^2 +
//      lambda tau^2), q = q^dag - tau/(2dx) (F_{i+1/2} + F_{i-1/2})
template <int BC>
__global__ void __launch_bounds__(256) k_adj_backsub(const AdjParams p) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const int64_t n = p.n;
    const int64_t il = adj_nb<BC>(i - 1, n), ir = adj_nb<BC>(i + 1, n);
    const double lam = p.lam, tau = p.tau, lt2 = lam * tau * tau, f2 = tau / (2.0 * p.dx);
    const double h = p.hbar[i], den = h * h + lt2;
    const double ho_a = p.Ao[0][i], qo_a = p.Ao[1][i], mo_a = p.Ao[2][i], ro_a = p.Ao[3][i];
    atomicAdd(p.rs_a + i, ro_a);
    const double m_a = mo_a - ro_a * lam * tau / (h * h);
    atomicAdd(p.hbar_a + i, ho_a + ro_a * 2.0 * lam * tau * p.mbar[i] / (h * h * h) +
                                m_a * p.ms[i] * 2.0 * h * lt2 / (den * den));
    atomicAdd(p.ms_a + i, m_a * h * h / den);
    atomicAdd(p.qs_a + i, qo_a);
    const double a = -f2 * qo_a;
    const double bp = 0.5 * (p.be[i] + p.be[ir]), bm = 0.5 * (p.be[il] + p.be[i]);
    const double jp = p.hbar[ir] - p.hbar[i], jm = p.hbar[i] - p.hbar[il];
    atomicAdd(p.Phi_a + i + 1, a);
    atomicAdd(p.be_a + i, 0.5 * a * jp);
    atomicAdd(p.be_a + ir, 0.5 * a * jp);
    atomicAdd(p.hbar_a + ir, a * bp);
    atomicAdd(p.hbar_a + i, -a * bp);
    atomicAdd(p.Phi_a + i, a);
    atomicAdd(p.be_a + il, 0.5 * a * jm);
    atomicAdd(p.be_a + i, 0.5 * a * jm);
    atomicAdd(p.hbar_a + i, a * bm);
    atomicAdd(p.hbar_a + il, -a * bm);
}

// Row i of the forward depth matrix: A_i x_{i-1} + B_i x_i + C_i x_{i+1}.
template <int BC>
__device__ __forceinline__ void adj_row(const AdjParams& p, int64_t i, double& A, double& B,
                                        double& C) {
    const int64_t n = p.n;
    const int64_t il = adj_nb<BC>(i - 1, n), ir = adj_nb<BC>(i + 1, n);
    const double Cc = p.tau * p.tau / (p.dx * p.dx);
    const double bm = 0.5 * (p.be[il] + p.be[i]), bp = 0.5 * (p.be[i] + p.be[ir]);
    A = -Cc * bm;
    C = -Cc * bp;
    B = 1.0 + Cc * (bm + bp);
    if (BC == BC_TRANSMISSIVE) {
        if (i == 0) { B = 1.0 + Cc * bp; A = 0.0; }
        if (i == n - 1) { B = 1.0 + Cc * bm; C = 0.0; }
    }
}

// rows of M^T: (a^T)_i = C_{i-1}, (c^T)_i = A_{i+1} (cyclic when periodic)
template <int BC>
__global__ void __launch_bounds__(256) k_adj_rows(const AdjParams p) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const int64_t n = p.n;
    double A, B, C, Al_, Bl, Cl, Ar, Br, Cr;
    adj_row<BC>(p, i, A, B, C);
    adj_row<BC>(p, i > 0 ? i - 1 : n - 1, Al_, Bl, Cl);
    adj_row<BC>(p, i < n - 1 ? i + 1 : 0, Ar, Br, Cr);
    p.ra[i] = i > 0 ? Cl : (BC == BC_PERIODIC ? Cl : 0.0);
    p.rb[i] = B;
    p.rc[i] = i < n - 1 ? Ar : (BC == BC_PERIODIC ? Ar : 0.0);
}

// dJ/dM and the right-hand side D_i = h_b,i - tau/(2dx)(q^dag_{i+1} - q^dag_{i-1})
// + tau^2/dx^2 (Phi_{i+1/2} - Phi_{i-1/2})
template <int BC>
__global__ void __launch_bounds__(256) k_adj_rowsadj(const AdjParams p) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const int64_t n = p.n;
    const int64_t il = adj_nb<BC>(i - 1, n), ir = adj_nb<BC>(i + 1, n);
    const double Cc = p.tau * p.tau / (p.dx * p.dx), f2 = p.tau / (2.0 * p.dx);
    const double Da = p.D_a[i];
    const double A_a = -Da * p.hbar[il], B_a = -Da * p.hbar[i], C_a = -Da * p.hbar[ir];
    double bm_a = -Cc * A_a + Cc * B_a, bp_a = -Cc * C_a + Cc * B_a;
    if (BC == BC_TRANSMISSIVE && i == 0) bm_a = 0.0;
    if (BC == BC_TRANSMISSIVE && i == n - 1) bp_a = 0.0;
    atomicAdd(p.be_a + il, 0.5 * bm_a);
    atomicAdd(p.be_a + i, 0.5 * bm_a + 0.5 * bp_a);
    atomicAdd(p.be_a + ir, 0.5 * bp_a);
    atomicAdd(p.Ab[0] + i, Da);
    atomicAdd(p.qs_a + ir, -f2 * Da);
    atomicAdd(p.qs_a + il, f2 * Da);
    atomicAdd(p.Phi_a + i + 1, Cc * Da);
    atomicAdd(p.Phi_a + i, -Cc * Da);
}

__device__ __forceinline__ double adj_ptil(double lam, double h, double m) {
    return (lam / 3.0) * (1.0 - (m / h) / h);
}

// face forces Phi_{k+1/2} = (p^_{i1} - p^_{i0}) + (g hbar_face + (3/2) p~_face)(b_{i1} - b_{i0})
//                           - beta_face (h_l,i1 - h_l,i0),  k = -1 .. n-1
template <int BC>
__global__ void __launch_bounds__(256) k_adj_phi(const AdjParams p) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // k + 1
    if (f > p.n) return;
    const int64_t n = p.n, k = f - 1;
    const int64_t i0 = adj_nb<BC>(k, n), i1 = adj_nb<BC>(k + 1, n);
    const double g = p.g, lam = p.lam;
    const double* hl = p.Ul[0];
    const double* ml = p.Ul[2];
    const double a = p.Phi_a[f];
    const double db = p.bathy ? p.bathy[i1] - p.bathy[i0] : 0.0;
    const double pt0 = adj_ptil(lam, hl[i0], ml[i0]), pt1 = adj_ptil(lam, hl[i1], ml[i1]);
    const double G = g * 0.5 * (hl[i0] + hl[i1]) + 1.5 * 0.5 * (pt0 + pt1);
    const double bbar = 0.5 * (p.be[i0] + p.be[i1]), dhl = hl[i1] - hl[i0];
    atomicAdd(p.ph_a + i1, a);
    atomicAdd(p.ph_a + i0, -a);
    const double G_a = a * db;
    atomicAdd(p.Al[0] + i0, 0.5 * g * G_a);
    atomicAdd(p.Al[0] + i1, 0.5 * g * G_a);
    atomicAdd(p.pt_a + i0, 0.75 * G_a);
    atomicAdd(p.pt_a + i1, 0.75 * G_a);
    if (p.bathy && p.Abathy) {
        atomicAdd(p.Abathy + i1, a * G);
        atomicAdd(p.Abathy + i0, -a * G);
    }
    atomicAdd(p.be_a + i0, 0.5 * (-a * dhl));
    atomicAdd(p.be_a + i1, 0.5 * (-a * dhl));
    atomicAdd(p.Al[0] + i1, -a * bbar);
    atomicAdd(p.Al[0] + i0, a * bbar);
}

// p^ = g h^2/2 + eta p~ + lambda alpha (m^dag b_1 - m_l) and p~ = (lambda/3)(1 - e)
// (e = m_l/h^2, eta = m_l/h, alpha = -(2e - 1)/(3h), b_1 = h^2/(h^2 + lambda tau^2)),
// then beta = a^2 + lambda alpha beta_2 m^dag (eq. (eq:hSGN_alpha)), per cell
__global__ void __launch_bounds__(256) k_adj_cell(const AdjParams p) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const double g = p.g, lam = p.lam, tau = p.tau, lt2 = lam * tau * tau;
    const double h = p.Ul[0][i], m = p.Ul[2][i], msv = p.ms[i];
    double h_acc = 0.0, m_acc = 0.0, ms_acc = 0.0;
    {
        const double e = m / (h * h), eta = m / h;
        const double alpha = -(2.0 * e - 1.0) / (3.0 * h);
        const double den = h * h + lt2, b1 = h * h / den;
        const double wv = msv * b1 - m;
        const double ptil = (lam / 3.0) * (1.0 - e);
        const double a = p.ph_a[i];
        const double ptot_a = p.pt_a[i] + a * eta;
        const double eta_a = a * ptil;
        const double alpha_a = a * lam * wv;
        const double w_a = a * lam * alpha;
        double h_a = a * g * h, m_a = -w_a, e_a = 0.0;
        ms_acc += w_a * b1;
        const double b1_a = w_a * msv;
        h_a += b1_a * 2.0 * h * lt2 / (den * den);
        e_a += alpha_a * (-2.0 / (3.0 * h));
        h_a += alpha_a * (2.0 * e - 1.0) / (3.0 * h * h);
        e_a += -(lam / 3.0) * ptot_a;
        m_a += eta_a / h;
        h_a += -eta_a * m / (h * h);
        m_a += e_a / (h * h);
        h_a += -2.0 * e_a * m / (h * h * h);
        h_acc += h_a;
        m_acc += m_a;
    }
    {
        const double eta = m / h;
        const double alpha = -(2.0 * eta / h - 1.0) / (3.0 * h);
        const double beta1 = 1.0 + lt2 / (h * h);
        const double beta2 = 2.0 * lt2 / (beta1 * beta1 * h * h * h);
        const double a = p.be_a[i];
        const double a2_a = a;
        double alpha_a = a * lam * beta2 * msv;
        const double beta2_a = a * lam * alpha * msv;
        ms_acc += a * lam * alpha * beta2;
        const double beta1_a = beta2_a * (-2.0 * beta2 / beta1);
        double h_a = beta2_a * (-3.0 * beta2 / h);
        h_a += beta1_a * (-2.0 * lt2 / (h * h * h));
        const double c2_a = a2_a;
        double eta_a = -a2_a * lam * alpha;
        alpha_a += -a2_a * lam * eta;
        h_a += c2_a * (g - (2.0 * lam / 3.0) * eta * eta / (h * h * h));
        eta_a += c2_a * (2.0 * lam / 3.0) * eta / (h * h);
        eta_a += alpha_a * (-2.0 / (3.0 * h * h));
        h_a += alpha_a * (4.0 * eta / (3.0 * h * h * h) - 1.0 / (3.0 * h * h));
        m_acc += eta_a / h;
        h_a += -eta_a * m / (h * h);
        h_acc += h_a;
    }
    atomicAdd(p.Al[0] + i, h_acc);
    atomicAdd(p.Al[2] + i, m_acc);
    atomicAdd(p.ms_a + i, ms_acc);
}

// m^dag = m_b - tau/dx (F^m_{i+1/2} - F^m_{i-1/2}) + tau r^dag - tau (3/2) q_l b_x,
// then r^dag = r_b - tau/dx (F^r ...) + lambda tau, q^dag = q_b - tau/dx (F^q ...)
template <int BC>
__global__ void __launch_bounds__(256) k_adj_starred(const AdjParams p) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const int64_t n = p.n;
    const int64_t il = adj_nb<BC>(i - 1, n), ir = adj_nb<BC>(i + 1, n);
    const double tau = p.tau, fd = tau / p.dx;
    const double a = p.ms_a[i];
    atomicAdd(p.Ab[2] + i, a);
    atomicAdd(p.Fm_a + i + 1, -fd * a);
    atomicAdd(p.Fm_a + i, fd * a);
    const double rs_a = p.rs_a[i] + tau * a;
    if (p.bathy) {
        const double k = -tau * 1.5 / (2.0 * p.dx);
        const double ql = p.Ul[1][i];
        atomicAdd(p.Al[1] + i, k * (p.bathy[ir] - p.bathy[il]) * a);
        if (p.Abathy) {
            atomicAdd(p.Abathy + ir, k * ql * a);
            atomicAdd(p.Abathy + il, -k * ql * a);
        }
    }
    atomicAdd(p.Ab[3] + i, rs_a);
    atomicAdd(p.Fr_a + i + 1, -fd * rs_a);
    atomicAdd(p.Fr_a + i, fd * rs_a);
    const double qa = p.qs_a[i];
    atomicAdd(p.Ab[1] + i, qa);
    atomicAdd(p.Fq_a + i + 1, -fd * qa);
    atomicAdd(p.Fq_a + i, fd * qa);
}

// Rusanov fluxes of the reconstructed U_l at face k+1/2 (index f = k+1) and the
// speed s: F = (u_L X_L + u_R X_R - s (X_R - X_L))/2
template <int BC>
__global__ void __launch_bounds__(256) k_adj_flux(const AdjParams p) {
    __shared__ double red[8];
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double sp_a = 0.0;
    if (f <= p.n) {
        const int64_t n = p.n, k = f - 1;
        const int64_t im = adj_nb<BC>(k - 1, n), i0 = adj_nb<BC>(k, n);
        const int64_t i1 = adj_nb<BC>(k + 1, n), i2 = adj_nb<BC>(k + 2, n);
        const double* hl = p.Ul[0];
        const double* ql = p.Ul[1];
        const double* ml = p.Ul[2];
        const double* rl = p.Ul[3];
        const double s = *p.speed;
        const double hL = hl[i0] + (hl[i1] - hl[im]) / 4.0, hR = hl[i1] - (hl[i2] - hl[i0]) / 4.0;
        const double qL = ql[i0] + (ql[i1] - ql[im]) / 4.0, qR = ql[i1] - (ql[i2] - ql[i0]) / 4.0;
        const double mL = ml[i0] + (ml[i1] - ml[im]) / 4.0, mR = ml[i1] - (ml[i2] - ml[i0]) / 4.0;
        const double rL = rl[i0] + (rl[i1] - rl[im]) / 4.0, rR = rl[i1] - (rl[i2] - rl[i0]) / 4.0;
        const double uL = qL / hL, uR = qR / hR;
        const double aq = p.Fq_a[f], am = p.Fm_a[f], ar = p.Fr_a[f];
        const double uL_a = 0.5 * (aq * qL + am * mL + ar * rL);
        const double uR_a = 0.5 * (aq * qR + am * mR + ar * rR);
        double qL_a = 0.5 * aq * (uL + s), qR_a = 0.5 * aq * (uR - s);
        const double mL_a = 0.5 * am * (uL + s), mR_a = 0.5 * am * (uR - s);
        const double rL_a = 0.5 * ar * (uL + s), rR_a = 0.5 * ar * (uR - s);
        sp_a = -0.5 * (aq * (qR - qL) + am * (mR - mL) + ar * (rR - rL));
        qL_a += uL_a / hL;
        qR_a += uR_a / hR;
        const double hL_a = -uL_a * uL / hL, hR_a = -uR_a * uR / hR;
        const double vL[4] = {hL_a, qL_a, mL_a, rL_a}, vR[4] = {hR_a, qR_a, mR_a, rR_a};
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            atomicAdd(p.Al[v] + i0, vL[v] + 0.25 * vR[v]);
            atomicAdd(p.Al[v] + i1, 0.25 * vL[v] + vR[v]);
            atomicAdd(p.Al[v] + im, -0.25 * vL[v]);
            atomicAdd(p.Al[v] + i2, -0.25 * vR[v]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sp_a += __shfl_xor_sync(0xffffffffu, sp_a, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sp_a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(p.Aspeed, t);
    }
}

// ---- helpers of the run adjoint ---------------------------------------------

// four device arrays passed by value
struct Ptr4 {
    const double* p[4];
};
struct MutPtr4 {
    double* p[4];
};

// out_k = a X_k + b Y_k (+ c Z_k when Z.p[0] is set), 4 arrays of n; out may
// alias an input (each element is read before it is written)
__global__ void __launch_bounds__(256) k_adj_axpby(int64_t n, double a, Ptr4 X, double b, Ptr4 Y,
                                                   double c, Ptr4 Z, MutPtr4 out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double v = a * X.p[k][i] + b * Y.p[k][i];
        if (Z.p[0]) v += c * Z.p[k][i];
        out.p[k][i] = v;
    }
}

// max_i |q_i/h_i| (as the ordered bits of a non-negative double) ...
__global__ void __launch_bounds__(256) k_adj_umax(int64_t n, const double* h, const double* q,
                                                  unsigned long long* bits) {
    double um = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        um = fmax(um, fabs(q[i] / h[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) um = fmax(um, __shfl_xor_sync(0xffffffffu, um, o));
    if ((threadIdx.x & 31) == 0) atomicMax(bits, (unsigned long long)__double_as_longlong(um));
}

// ... and the first cell attaining it
__global__ void __launch_bounds__(256) k_adj_argmax(int64_t n, const double* h, const double* q,
                                                    const unsigned long long* bits,
                                                    unsigned long long* idx) {
    const double um = __longlong_as_double((long long)*bits);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (fabs(q[i] / h[i]) == um) atomicMin(idx, (unsigned long long)i);
}

// the adjoint of s = |q/h| at the argmax cell
__global__ void k_adj_speed(const double* h, const double* q, const unsigned long long* idx,
                            const double* s_a, double* Ah, double* Aq) {
    const int64_t i = (int64_t)*idx;
    const double hh = h[i], qq = q[i];
    const double sg = qq > 0.0 ? 1.0 : (qq < 0.0 ? -1.0 : 0.0);
    Aq[i] += *s_a * sg / hh;
    Ah[i] += -*s_a * fabs(qq) / (hh * hh);
}

// gauge misfit after a step: J += dt/2 sum_g (h_{c_g} - d_g)^2, and the adjoint seed
// A_h[c_g] += dt (h_{c_g} - d_g)
__global__ void k_adj_gauges(int64_t n_gauges, const int64_t* cells, const double* data,
                             const double* h, double dt, double* J, double* Ah) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_gauges) return;
    const double e = h[cells[k]] - data[k];
    if (J) atomicAdd(J, 0.5 * e * e * dt);
    if (Ah) atomicAdd(Ah + cells[k], e * dt);
}

}  // namespace hsgn
