/*
 * hsgn_oracle.c -- plain, serial, FP64 CPU restatement of the semi-implicit
 * IMEX time step of the hyperbolic Serre-Green-Naghdi (hSGN) system.
 *
 * TEST INFRASTRUCTURE. This is the oracle the CUDA library is checked
 * against. Only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark load it. It shares no code, header, table or helper with the
 * CUDA library and never calls it.
 *
 * Source: E. Macca, W. Boscheri, M. Ricchiuto, "Semi-implicit strategies for
 * the Serre-Green-Naghdi equations in hyperbolic form" (arXiv 2510.07539).
 *   hSGN system, pressure:          Sec. 2.2, eqs. (hSGN_eq), (eq:hSGN_p)
 *   eigenvalues / celerity:         eqs. (eq:hSGN_eigenvalues), (eq:hSGN_c)
 *   pressure-gradient split:        eqs. (eq:hSGN_px), (eq:hSGN_alpha)
 *   splitting and h-elimination:    Sec. 3.1, eqs. (hSGN_eq-split) .. (eq:hnew)
 *   IMEX stages and tableau:        Sec. 3.2, eq. (tableau) and its efficient form
 *   time-step rule:                 Sec. 3.3 eq. (eq:MCFL), Sec. 5 (CFL definitions)
 *   D_x, hat D_x, reconstruction:   Sec. 4.1
 *   fully-discrete stage:           Sec. 4.2, eq. (GN_hyp_eq_semi_fully_discrete)
 *
 * Readings where the paper is silent or ambiguous (each restated at its use):
 *   R1  the printed 2-stage tableau (implicit first stage) is the scheme;
 *   R2  interface coefficients beta_{i+1/2}, delta_{i+1/2} are arithmetic means;
 *   R3  the "1/2" in front of the delta term of h^dagger pairs with a SUM of the
 *       two cell values, i.e. the term uses the mean with factor 1 (the literal
 *       reading is kept behind a flag, used only by a test that shows it gives
 *       the wrong linear dispersion);
 *   R4  in a stage, the additive "old" values come from the base state U_b and
 *       every flux and coefficient from the linearisation state U_l = U_E^(i);
 *   R5  reconstruction acts on the conserved variables (h, q, m, r). The
 *       Rusanov speed "alpha ~ |u|" (Sec. 4.1) is read as the global speed
 *       max_i |u_i^n| of the step (the same u_max the time-step rule of Sec. 5
 *       computes at t^n), used by both stages (rusanov = 1, default). The
 *       local speed max(|u^L|, |u^R|) is kept as rusanov = 0. Reason: at rest
 *       the local speed is zero, the explicit flux of h eta is then linear in
 *       q (coefficient eta) with no dissipation, and the linearised step
 *       amplifies grid-scale modes (spectral radius 1.02-1.14 per step on the
 *       paper's grids); the global speed damps them;
 *   R6  periodic: indices wrap and the matrix is cyclic; transmissive:
 *       zero-order ghost copies of every per-cell quantity, so the end rows of
 *       the matrix are Neumann rows;
 *   R7  bathymetry (form 1): the paper writes the model with a bottom (Sec.
 *       2.3, eq. (hSGNb_eq)) but derives the semi-implicit scheme only for a
 *       flat one. Form 1 keeps the splitting and the tridiagonal structure and
 *       is well balanced. With b_t = 0 the third equation of (hSGNb_eq) is
 *       (h eta)_t + (h u eta)_x = h w - (3/2) h u b_x (explicit source), the
 *       pressure p = g h^2/2 + eta p~ is the flat one, and the momentum gets the
 *       source -(g h + (3/2) p~) b_x. The implicit pressure is linearised about
 *       the linearisation state: p^ + beta (hbar - h_l) with
 *       p^ = p(h_l, m_l) + lambda alpha_l (m^dag b_1(h_l) - m_l); face forces
 *       F_{i+1/2} = p^_{i+1} - p^_i + (g h + (3/2) p~)_{i+1/2} (b_{i+1} - b_i)
 *                 + beta_{i+1/2} ((hbar_{i+1} - hbar_i) - (h_l,i+1 - h_l,i))
 *       drive both the depth rows, Delta[hbar]_i = h_b,i - tau/(2dx)
 *       (q^dag_{i+1} - q^dag_{i-1}) + tau^2/dx^2 (Phi_{i+1/2} - Phi_{i-1/2})
 *       with Phi = F - beta (hbar_{i+1} - hbar_i), and the momentum,
 *       qbar_i = q^dag_i - tau/(2dx) (F_{i+1/2} + F_{i-1/2}). At a lake at rest
 *       (u = 0, eta = h, w = 0, h + b = const) every term cancels exactly;
 *   R9  nu = |u| + sqrt(g h + (lambda/3) eta^2/h^2) (the form of eq. (eq:hSGN_c)).
 *
 * State layout: four arrays of n cells each, h, q = h u, m = h eta, r = h w.
 * Every routine returns 0 on success or a positive error code (see below).
 *
 * Parity status of each function (what pins it, in the test-suite):
 *   oracle_tridiag_solve   dense LU of the same matrix (library routine)
 *   oracle_imex_scalar     stability function from the unreduced tableau,
 *                          Taylor expansion 1 + z + z^2/2 + O(z^3)
 *   oracle_stage/step/run  exact mass conservation, constant-state
 *                          preservation, mirror symmetry, periodic shift,
 *                          linear hSGN dispersion relation (with Doppler
 *                          shift), lambda = 0 shallow-water limit, solitary
 *                          wave closed form (convergence trend), temporal
 *                          order 2
 *   oracle_assemble        row sums 1 (Delta[const] = const), symmetry,
 *                          diagonal dominance
 *   oracle_suggest_dt      the CFL_SW / CFL_IMEX ratios printed for the
 *                          Gaussian-bell test (Sec. 6.1)
 *   oracle_explicit_rhs    the continuous hSGN right-hand side differentiated
 *                          spectrally (second-order consistency, first order
 *                          without reconstruction), zero at rest, mass
 *   oracle_run schemes     ARS(2,2,2) against its double tableau on the
 *                          scalar split equation; SI1 / Euler / Heun against
 *                          their one-line definitions; temporal orders 2, 1,
 *                          2, 1 on hSGN; dispersion relation and solitary
 *                          wave at second order (ARS(2,2,2), Heun); mass and
 *                          constant states for every scheme
 *   oracle_stage_adjoint   central finite differences of oracle_stage along
 *                          random smooth directions in U_b, U_l, b and the
 *                          speed (both BCs)
 *   oracle_adjoint         central finite differences of the gauge misfit of
 *                          a run (initial state and bottom); zero gradient for
 *                          a lake at rest with matching data
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARG 1
#define ORACLE_ERR_DEPTH 2      /* a depth used as a divisor was <= 0 */
#define ORACLE_ERR_COERCIVE 3   /* beta <= 0 or a zero pivot */
#define ORACLE_ERR_NONFINITE 4
#define ORACLE_ERR_NOMEM 5

#define BC_PERIODIC 0
#define BC_TRANSMISSIVE 1

typedef struct {
    int64_t n;          /* number of cells, >= 3 */
    double dx;          /* uniform cell width */
    int32_t bc;         /* BC_PERIODIC or BC_TRANSMISSIVE */
    int32_t delta_half; /* 0: reading R3 (default); 1: literal factor 1/2 */
    double g;           /* gravity */
    double lambda;      /* relaxation parameter, >= 0 */
    int32_t rusanov;    /* 0: local speed max(|u^L|,|u^R|); 1: global speed (R5) */
    int32_t form;       /* 0: the printed flat-bottom scheme; 1: well-balanced form (R7) */
    double speed;       /* global Rusanov speed of the current step (rusanov == 1) */
    const double* bathy; /* bottom b per cell (form 1; NULL = flat) */
    int32_t recon;      /* 1: centred linear reconstruction (Sec. 4.1); 0: none (first order) */
    int32_t scheme;     /* time stepping of oracle_run, see ORACLE_SCHEME_* */
} oracle_params;

/* Time-stepping schemes of oracle_run (the first is the method of the paper;
 * the others are the comparisons it reports or names):
 *   PRINTED  the two-stage IMEX tableau of Sec. 3.2, eq. (tableau) (R1)
 *   ARS222   the three-stage Ascher-Ruuth-Spiteri ARS(2,2,2) double tableau
 *            (explicit first stage), in the generic stage form of Sec. 3.2
 *   SI1      first-order semi-implicit: one stage with tau = dt
 *            (eq. (GN_hyp_eq_semi_fully_discrete) as printed)
 *   EX_HEUN  explicit hSGN, eq. (GN_hyp_eq_explicit), with Heun's method
 *   EX_EULER explicit hSGN, eq. (GN_hyp_eq_explicit), forward Euler */
#define ORACLE_SCHEME_PRINTED 0
#define ORACLE_SCHEME_ARS222 1
#define ORACLE_SCHEME_SI1 2
#define ORACLE_SCHEME_EX_HEUN 3
#define ORACLE_SCHEME_EX_EULER 4

/* Neighbour index: wrap (periodic) or clamp to the boundary cell
 * (transmissive, zero-order ghost copies, reading R6). */
static int64_t nb(const oracle_params* p, int64_t i) {
    if (p->bc == BC_PERIODIC) {
        int64_t k = i % p->n;
        return k < 0 ? k + p->n : k;
    }
    if (i < 0) return 0;
    if (i >= p->n) return p->n - 1;
    return i;
}

/* ------------------------------------------------------------------------
 * Tridiagonal solve. Row i reads a[i] x[i-1] + b[i] x[i] + c[i] x[i+1] = d[i].
 * periodic == 0: a[0] and c[n-1] are ignored (plain Thomas elimination).
 * periodic != 0: a[0] couples x[n-1] and c[n-1] couples x[0] (cyclic
 * matrix); solved by writing the matrix as a tridiagonal matrix plus a rank-one
 * correction u v^T and applying the Sherman-Morrison formula
 *   x = y - z (v.y) / (1 + v.z),   T y = d,  T z = u.
 * Choice: u = (s, 0..0, c[n-1]), v = (1, 0..0, a[0]/s) with s = -b[0], so T
 * has T[0][0] = b[0] - s and T[n-1][n-1] = b[n-1] - a[0] c[n-1] / s.
 * ------------------------------------------------------------------------ */
static int thomas(int64_t n, const double* a, const double* b, const double* c,
                  const double* d, double* x, double* work) {
    /* forward elimination: work holds the modified super-diagonal */
    double piv = b[0];
    if (!(piv != 0.0)) return ORACLE_ERR_COERCIVE;
    work[0] = c[0] / piv;
    x[0] = d[0] / piv;
    for (int64_t i = 1; i < n; ++i) {
        piv = b[i] - a[i] * work[i - 1];
        if (!(piv != 0.0)) return ORACLE_ERR_COERCIVE;
        work[i] = (i < n - 1) ? c[i] / piv : 0.0;
        x[i] = (d[i] - a[i] * x[i - 1]) / piv;
    }
    /* back substitution */
    for (int64_t i = n - 2; i >= 0; --i) x[i] = x[i] - work[i] * x[i + 1];
    return ORACLE_OK;
}

int oracle_tridiag_solve(int64_t n, int32_t periodic, const double* a, const double* b,
                         const double* c, const double* d, double* x) {
    if (n < 1 || !a || !b || !c || !d || !x) return ORACLE_ERR_ARG;
    if (n == 1) {
        double diag = b[0] + (periodic ? a[0] + c[0] : 0.0);
        if (!(diag != 0.0)) return ORACLE_ERR_COERCIVE;
        x[0] = d[0] / diag;
        return ORACLE_OK;
    }
    if (!periodic || n == 2) {
        double* work = (double*)malloc((size_t)n * sizeof(double));
        if (!work) return ORACLE_ERR_NOMEM;
        int rc;
        if (!periodic) {
            rc = thomas(n, a, b, c, d, x, work);
        } else {
            /* n == 2: both couplings of each row hit the other unknown */
            double bb[2] = {b[0], b[1]};
            double aa[2] = {0.0, a[1] + c[1]};
            double cc[2] = {a[0] + c[0], 0.0};
            rc = thomas(2, aa, bb, cc, d, x, work);
        }
        free(work);
        return rc;
    }
    double* bt = (double*)malloc((size_t)n * sizeof(double));
    double* u = (double*)malloc((size_t)n * sizeof(double));
    double* z = (double*)malloc((size_t)n * sizeof(double));
    double* work = (double*)malloc((size_t)n * sizeof(double));
    if (!bt || !u || !z || !work) {
        free(bt); free(u); free(z); free(work);
        return ORACLE_ERR_NOMEM;
    }
    const double s = -b[0];
    const double corner_lo = c[n - 1]; /* A[n-1][0] */
    const double corner_hi = a[0];     /* A[0][n-1] */
    memcpy(bt, b, (size_t)n * sizeof(double));
    bt[0] = b[0] - s;
    bt[n - 1] = b[n - 1] - corner_hi * corner_lo / s;
    for (int64_t i = 0; i < n; ++i) u[i] = 0.0;
    u[0] = s;
    u[n - 1] = corner_lo;
    int rc = thomas(n, a, bt, c, d, x, work);
    if (rc == ORACLE_OK) rc = thomas(n, a, bt, c, u, z, work);
    if (rc == ORACLE_OK) {
        const double vy = x[0] + (corner_hi / s) * x[n - 1];
        const double vz = z[0] + (corner_hi / s) * z[n - 1];
        const double den = 1.0 + vz;
        if (!(den != 0.0)) {
            rc = ORACLE_ERR_COERCIVE;
        } else {
            const double f = vy / den;
            for (int64_t i = 0; i < n; ++i) x[i] -= f * z[i];
        }
    }
    free(bt); free(u); free(z); free(work);
    return rc;
}

/* ------------------------------------------------------------------------
 * One implicit stage of the semi-implicit scheme, Sec. 4.2, eq.
 * (GN_hyp_eq_semi_fully_discrete), with Delta t replaced by the stage step tau
 * and the state roles of reading R4:
 *   base state U_b: the additive old values h, q, h eta, h w;
 *   linearisation state U_l: the reconstructed fluxes (Sec. 4.1) and every
 *   coefficient (a^2, alpha, beta_1, beta_2, beta, delta).
 * The full set of per-cell quantities is returned through `asm_out` when it is
 * not NULL (used by the tests of the assembled matrix).
 * ------------------------------------------------------------------------ */
typedef struct {
    double *qs, *ms, *rs;          /* q^dagger, (h eta)^dagger, (h w)^dagger */
    double *beta, *delta;          /* cell coefficients */
    double *a, *b, *c, *d;         /* rows of Delta[h] = h^dagger */
} oracle_assembly;

static double sqr(double x) { return x * x; }

/* ------------------------------------------------------------------------
 * Rusanov fluxes of hu^2, hu eta, hu w at every face (Sec. 4.1, hat D_x),
 * shared by the semi-implicit stage and the explicit scheme. Index k + 1
 * holds the face between cells k and k+1, k = -1 .. n-1. With p->recon the
 * conserved variables are reconstructed by the unlimited centred slope,
 *   v^L_{k+1/2} = v_k + (v_{k+1} - v_{k-1})/4,
 *   v^R_{k+1/2} = v_{k+1} - (v_{k+2} - v_k)/4,
 * without it the face values are the cell values (first order).
 * ------------------------------------------------------------------------ */
static int rusanov_fluxes(const oracle_params* p, const double* hl, const double* ql,
                          const double* ml, const double* rl, double* Fq, double* Fm,
                          double* Fr) {
    const int64_t n = p->n;
    for (int64_t k = -1; k < n; ++k) {
        const int64_t im = nb(p, k - 1), i0 = nb(p, k), i1 = nb(p, k + 1), i2 = nb(p, k + 2);
        double hL = hl[i0], hR = hl[i1], qL = ql[i0], qR = ql[i1];
        double mL = ml[i0], mR = ml[i1], rL = rl[i0], rR = rl[i1];
        if (p->recon) {
            hL = hl[i0] + (hl[i1] - hl[im]) / 4.0;
            hR = hl[i1] - (hl[i2] - hl[i0]) / 4.0;
            qL = ql[i0] + (ql[i1] - ql[im]) / 4.0;
            qR = ql[i1] - (ql[i2] - ql[i0]) / 4.0;
            mL = ml[i0] + (ml[i1] - ml[im]) / 4.0;
            mR = ml[i1] - (ml[i2] - ml[i0]) / 4.0;
            rL = rl[i0] + (rl[i1] - rl[im]) / 4.0;
            rR = rl[i1] - (rl[i2] - rl[i0]) / 4.0;
        }
        if (!(hL > 0.0) || !(hR > 0.0)) return ORACLE_ERR_DEPTH;
        const double uL = qL / hL, uR = qR / hR;
        const double s = p->rusanov ? p->speed : fmax(fabs(uL), fabs(uR));
        Fq[k + 1] = 0.5 * (uL * qL + uR * qR - s * (qR - qL));
        Fm[k + 1] = 0.5 * (uL * mL + uR * mR - s * (mR - mL));
        Fr[k + 1] = 0.5 * (uL * rL + uR * rR - s * (rR - rL));
    }
    return ORACLE_OK;
}

static int stage_impl(const oracle_params* p,
                      const double* hb, const double* qb, const double* mb, const double* rb,
                      const double* hl, const double* ql, const double* ml, const double* rl,
                      double tau, double* ho, double* qo, double* mo, double* ro,
                      oracle_assembly* keep) {
    const int64_t n = p->n;
    if (n < 3 || !(p->dx > 0.0) || !(tau >= 0.0) || !(p->lambda >= 0.0)) return ORACLE_ERR_ARG;
    const double dx = p->dx, g = p->g, lam = p->lambda;
    int rc = ORACLE_OK;
    double* Phi = NULL; /* face forces of form 1 (freed on every exit path) */

    /* face fluxes: index k + 1 holds the face between cells k and k+1, k = -1..n-1 */
    double* Fq = (double*)malloc((size_t)(n + 1) * sizeof(double));
    double* Fm = (double*)malloc((size_t)(n + 1) * sizeof(double));
    double* Fr = (double*)malloc((size_t)(n + 1) * sizeof(double));
    double* qs = (double*)malloc((size_t)n * sizeof(double));
    double* ms = (double*)malloc((size_t)n * sizeof(double));
    double* rs = (double*)malloc((size_t)n * sizeof(double));
    double* beta = (double*)malloc((size_t)n * sizeof(double));
    double* delta = (double*)malloc((size_t)n * sizeof(double));
    double* A = (double*)malloc((size_t)n * sizeof(double));
    double* B = (double*)malloc((size_t)n * sizeof(double));
    double* C = (double*)malloc((size_t)n * sizeof(double));
    double* D = (double*)malloc((size_t)n * sizeof(double));
    double* hbar = (double*)malloc((size_t)n * sizeof(double));
    if (!Fq || !Fm || !Fr || !qs || !ms || !rs || !beta || !delta || !A || !B || !C || !D || !hbar) {
        rc = ORACLE_ERR_NOMEM;
        goto done;
    }

    /* (1) Rusanov fluxes of hu^2, hu eta, hu w at every face (Sec. 4.1, hat D_x) */
    rc = rusanov_fluxes(p, hl, ql, ml, rl, Fq, Fm, Fr);
    if (rc != ORACLE_OK) goto done;

    /* (2) starred values and the coefficients of eqs. (eq:hSGN_alpha) and
     * (GN_hyp_eq_semi_fully_discrete), per cell. */
    const int wb = p->form == 1;
    const double* bb = p->bathy;
    for (int64_t i = 0; i < n; ++i) {
        rs[i] = rb[i] - (tau / dx) * (Fr[i + 1] - Fr[i]) + lam * tau;
        ms[i] = mb[i] - (tau / dx) * (Fm[i + 1] - Fm[i]) + tau * rs[i];
        if (wb && bb) /* -(3/2) h u b_x of the (h eta) equation, from U_l */
            ms[i] -= tau * 1.5 * ql[i] * (bb[nb(p, i + 1)] - bb[nb(p, i - 1)]) / (2.0 * dx);
        qs[i] = qb[i] - (tau / dx) * (Fq[i + 1] - Fq[i]);
        const double h = hl[i];
        if (!(h > 0.0)) { rc = ORACLE_ERR_DEPTH; goto done; }
        const double eta = ml[i] / h;
        const double alpha = -(2.0 * eta / h - 1.0) / (3.0 * h);
        const double c2 = g * h + (lam / 3.0) * eta * eta / (h * h);
        const double a2 = c2 - lam * eta * alpha;
        const double beta1 = 1.0 + lam * tau * tau / (h * h);
        const double beta2 = 2.0 * lam * tau * tau / (beta1 * beta1 * h * h * h);
        beta[i] = a2 + lam * alpha * beta2 * ms[i];
        delta[i] = alpha / beta1;
        if (!(beta[i] > 0.0)) { rc = ORACLE_ERR_COERCIVE; goto done; }
    }

    /* (3) rows of Delta[h]_i = h^dagger_i. Interface values are means (R2);
     * the delta term carries factor 1 with means (R3). Form 1 (R7) replaces
     * the delta term by the explicit face forces Phi. */
    if (wb) {
        Phi = (double*)malloc((size_t)(n + 1) * sizeof(double)); /* face k+1/2 at k+1 */
        double* ph = (double*)malloc((size_t)n * sizeof(double));
        double* pt = (double*)malloc((size_t)n * sizeof(double));
        if (!Phi || !ph || !pt) { free(ph); free(pt); rc = ORACLE_ERR_NOMEM; goto done; }
        for (int64_t i = 0; i < n; ++i) {
            const double h = hl[i], eta = ml[i] / h;
            const double ptil = (lam / 3.0) * (1.0 - eta / h);
            const double alpha = -(2.0 * eta / h - 1.0) / (3.0 * h);
            const double b1 = h * h / (h * h + lam * tau * tau);
            ph[i] = g * h * h / 2.0 + eta * ptil + lam * alpha * (ms[i] * b1 - ml[i]);
            pt[i] = ptil;
        }
        for (int64_t k = -1; k < n; ++k) {
            const int64_t i0 = nb(p, k), i1 = nb(p, k + 1);
            const double db = bb ? bb[i1] - bb[i0] : 0.0;
            const double bbar = 0.5 * (beta[i0] + beta[i1]);
            Phi[k + 1] = (ph[i1] - ph[i0]) + (g * 0.5 * (hl[i0] + hl[i1]) + 1.5 * 0.5 * (pt[i0] + pt[i1])) * db
                       - bbar * (hl[i1] - hl[i0]);
        }
        free(ph); free(pt);
    }
    {
        const double Cc = tau * tau / (dx * dx);
        const double fd = (p->delta_half ? 0.5 : 1.0) * lam * tau * tau / (dx * dx);
        for (int64_t i = 0; i < n; ++i) {
            const int64_t il = nb(p, i - 1), ir = nb(p, i + 1);
            const double bm = 0.5 * (beta[il] + beta[i]);   /* beta_{i-1/2} */
            const double bp = 0.5 * (beta[i] + beta[ir]);   /* beta_{i+1/2} */
            const double dm = 0.5 * (delta[il] + delta[i]);
            const double dp = 0.5 * (delta[i] + delta[ir]);
            if (wb)
                D[i] = hb[i] - (tau / (2.0 * dx)) * (qs[ir] - qs[il]) + Cc * (Phi[i + 1] - Phi[i]);
            else
                D[i] = hb[i] - (tau / (2.0 * dx)) * (qs[ir] - qs[il])
                     + fd * (dp * (ms[ir] - ms[i]) - dm * (ms[i] - ms[il]));
            A[i] = -Cc * bm;
            C[i] = -Cc * bp;
            B[i] = 1.0 + Cc * (bm + bp);
            if (p->bc == BC_TRANSMISSIVE) {
                /* Neumann rows: the ghost h_{-1} = h_0 (resp. h_n = h_{n-1}) */
                if (i == 0) { B[i] = 1.0 + Cc * bp; A[i] = 0.0; }
                if (i == n - 1) { B[i] = 1.0 + Cc * bm; C[i] = 0.0; }
            }
        }
    }

    /* (4) solve Delta[hbar] = h^dagger (cyclic when periodic) */
    rc = oracle_tridiag_solve(n, p->bc == BC_PERIODIC, A, B, C, D, hbar);
    if (rc != ORACLE_OK) goto done;

    /* (5) back-substitution for qbar, (h eta)bar, (h w)bar; the fourth
     * equation treats h^2 implicitly (Sec. 6.3.1, "second version"). */
    for (int64_t i = 0; i < n; ++i) {
        const int64_t il = nb(p, i - 1), ir = nb(p, i + 1);
        const double h = hbar[i];
        if (!(h > 0.0)) { rc = ORACLE_ERR_DEPTH; goto done; }
        double q;
        if (wb) {
            /* face forces F = Phi + beta_{face} (hbar jump) on both sides */
            const double Fp = Phi[i + 1] + 0.5 * (beta[i] + beta[ir]) * (hbar[ir] - hbar[i]);
            const double Fm_ = Phi[i] + 0.5 * (beta[il] + beta[i]) * (hbar[i] - hbar[il]);
            q = qs[i] - (tau / (2.0 * dx)) * (Fp + Fm_);
        } else {
            q = qs[i] - (tau / (2.0 * dx)) * beta[i] * (hbar[ir] - hbar[il])
              - (lam * tau / (2.0 * dx)) * delta[i] * (ms[ir] - ms[il]);
        }
        const double m = ms[i] / (1.0 + lam * tau * tau / (h * h));
        const double r = rs[i] - lam * tau * m / (h * h);
        if (!isfinite(h) || !isfinite(q) || !isfinite(m) || !isfinite(r)) {
            rc = ORACLE_ERR_NONFINITE;
            goto done;
        }
        ho[i] = h; qo[i] = q; mo[i] = m; ro[i] = r;
    }

    if (keep) {
        memcpy(keep->qs, qs, (size_t)n * sizeof(double));
        memcpy(keep->ms, ms, (size_t)n * sizeof(double));
        memcpy(keep->rs, rs, (size_t)n * sizeof(double));
        memcpy(keep->beta, beta, (size_t)n * sizeof(double));
        memcpy(keep->delta, delta, (size_t)n * sizeof(double));
        memcpy(keep->a, A, (size_t)n * sizeof(double));
        memcpy(keep->b, B, (size_t)n * sizeof(double));
        memcpy(keep->c, C, (size_t)n * sizeof(double));
        memcpy(keep->d, D, (size_t)n * sizeof(double));
    }

done:
    free(Phi);
    free(Fq); free(Fm); free(Fr); free(qs); free(ms); free(rs); free(beta); free(delta);
    free(A); free(B); free(C); free(D); free(hbar);
    return rc;
}

int oracle_stage(const oracle_params* p,
                 const double* hb, const double* qb, const double* mb, const double* rb,
                 const double* hl, const double* ql, const double* ml, const double* rl,
                 double tau, double* ho, double* qo, double* mo, double* ro) {
    if (!p) return ORACLE_ERR_ARG;
    return stage_impl(p, hb, qb, mb, rb, hl, ql, ml, rl, tau, ho, qo, mo, ro, NULL);
}

/* The assembled quantities of one stage (same arguments as oracle_stage);
 * outputs are n-long arrays. */
int oracle_assemble(const oracle_params* p,
                    const double* hb, const double* qb, const double* mb, const double* rb,
                    const double* hl, const double* ql, const double* ml, const double* rl,
                    double tau, double* qs, double* ms, double* rs, double* beta,
                    double* delta, double* a, double* b, double* c, double* d) {
    if (!p) return ORACLE_ERR_ARG;
    const int64_t n = p->n;
    if (n < 3) return ORACLE_ERR_ARG;
    double* tmp = (double*)malloc((size_t)(4 * n) * sizeof(double));
    if (!tmp) return ORACLE_ERR_NOMEM;
    oracle_assembly keep = {qs, ms, rs, beta, delta, a, b, c, d};
    int rc = stage_impl(p, hb, qb, mb, rb, hl, ql, ml, rl, tau,
                        tmp, tmp + n, tmp + 2 * n, tmp + 3 * n, &keep);
    free(tmp);
    return rc;
}

/* ------------------------------------------------------------------------
 * Right-hand side of the explicit hSGN scheme, eq. (GN_hyp_eq_explicit)
 * (Sec. 4.4), with every term evaluated at the given state U:
 *   L_h = -D_x(q)
 *   L_q = -hat D_x(q u) - a^2 D_x(h) - lambda alpha D_x(h eta)
 *   L_m = -hat D_x(h u eta) + h w
 *   L_r = -hat D_x(h u w) - lambda ((h eta)/h^2 - 1)
 * D_x(F)_i = (F_{i+1} - F_{i-1})/(2 dx) (the mean face values of Sec. 4.4),
 * hat D_x the Rusanov flux difference, a^2 and alpha of eq. (eq:hSGN_alpha)
 * at the cell. The forward Euler step U + dt L(U) is the scheme as printed;
 * L(U) is also the explicit evaluation H(U, U) of the IMEX right-hand side.
 * Flat bottom only.
 * ------------------------------------------------------------------------ */
int oracle_explicit_rhs(const oracle_params* p, const double* h, const double* q,
                        const double* m, const double* r, double* Lh, double* Lq, double* Lm,
                        double* Lr) {
    if (!p || p->n < 3 || !(p->dx > 0.0) || p->form != 0) return ORACLE_ERR_ARG;
    const int64_t n = p->n;
    const double dx = p->dx, g = p->g, lam = p->lambda;
    double* Fq = (double*)malloc((size_t)(n + 1) * sizeof(double));
    double* Fm = (double*)malloc((size_t)(n + 1) * sizeof(double));
    double* Fr = (double*)malloc((size_t)(n + 1) * sizeof(double));
    int rc = ORACLE_OK;
    if (!Fq || !Fm || !Fr) { rc = ORACLE_ERR_NOMEM; goto done; }
    rc = rusanov_fluxes(p, h, q, m, r, Fq, Fm, Fr);
    if (rc != ORACLE_OK) goto done;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t il = nb(p, i - 1), ir = nb(p, i + 1);
        if (!(h[i] > 0.0)) { rc = ORACLE_ERR_DEPTH; goto done; }
        const double eta = m[i] / h[i];
        const double alpha = -(2.0 * eta / h[i] - 1.0) / (3.0 * h[i]);
        const double c2 = g * h[i] + (lam / 3.0) * eta * eta / (h[i] * h[i]);
        const double a2 = c2 - lam * eta * alpha;
        Lh[i] = -(q[ir] - q[il]) / (2.0 * dx);
        Lq[i] = -(Fq[i + 1] - Fq[i]) / dx - a2 * (h[ir] - h[il]) / (2.0 * dx)
              - lam * alpha * (m[ir] - m[il]) / (2.0 * dx);
        Lm[i] = -(Fm[i + 1] - Fm[i]) / dx + r[i];
        Lr[i] = -(Fr[i + 1] - Fr[i]) / dx - lam * (m[i] / (h[i] * h[i]) - 1.0);
        if (!isfinite(Lh[i]) || !isfinite(Lq[i]) || !isfinite(Lm[i]) || !isfinite(Lr[i])) {
            rc = ORACLE_ERR_NONFINITE;
            goto done;
        }
    }
done:
    free(Fq); free(Fm); free(Fr);
    return rc;
}

/* ------------------------------------------------------------------------
 * IMEX Runge-Kutta step of Sec. 3.2 with the double Butcher tableau of eq.
 * (tableau) (reading R1: two stages, implicit first stage),
 *   gamma = 1 - 1/sqrt(2),  c = 1/(2 gamma),
 * written in the efficient form given right after the tableau:
 *   U_I^(1) = U^n + dt gamma H(U_E^(1), U_I^(1)),           U_E^(1) = U^n
 *   U_E^(2) = (1 - c/gamma) U^n + (c/gamma) U_I^(1)
 *   U_I^(2) = (1 - (1-gamma)/gamma) U^n + ((1-gamma)/gamma) U_I^(1)
 *             + dt gamma H(U_E^(2), U_I^(2)),
 *   U^{n+1} = U_I^(2) (stiffly accurate).
 * Each implicit stage is a call S(U_b, U_l, tau = gamma dt) of a stage
 * operator; the generic driver below is shared by the hSGN step and by the
 * scalar split test equation.
 * ------------------------------------------------------------------------ */
typedef int (*stage_fn)(void* ctx, int64_t len, const double* Ub, const double* Ul,
                        double tau, double* Uout);

static int imex2_step(void* ctx, stage_fn S, int64_t len, double* U, double dt, double* work) {
    const double gamma = 1.0 - 1.0 / sqrt(2.0);
    const double c = 1.0 / (2.0 * gamma);
    double* U1 = work;
    double* Ue = work + len;
    double* Ub = work + 2 * len;
    int rc = S(ctx, len, U, U, gamma * dt, U1);
    if (rc != ORACLE_OK) return rc;
    for (int64_t k = 0; k < len; ++k) {
        Ue[k] = (1.0 - c / gamma) * U[k] + (c / gamma) * U1[k];
        Ub[k] = (1.0 - (1.0 - gamma) / gamma) * U[k] + ((1.0 - gamma) / gamma) * U1[k];
    }
    return S(ctx, len, Ub, Ue, gamma * dt, U);
}

/* Explicit evaluation F(U) = H(U, U) of the full right-hand side. */
typedef int (*rhs_fn)(void* ctx, int64_t len, const double* U, double* L);

/* ARS(2,2,2) (Ascher, Ruuth, Spiteri 1997) in the generic stage form of
 * Sec. 3.2 (U_E^(i) = U^n + dt sum_{j<i} aE_ij H_j, U_I^(i) = U^n +
 * dt (sum_{j<i} aI_ij H_j + aI_ii H(U_E^(i), U_I^(i))), H_j = H(U_E^(j),
 * U_I^(j))), with the double tableau
 *   explicit: aE_21 = gamma, aE_31 = delta, aE_32 = 1 - delta
 *   implicit: aI_22 = gamma, aI_32 = 1 - gamma, aI_33 = gamma,
 * gamma = 1 - 1/sqrt(2), delta = 1 - 1/(2 gamma), U^{n+1} = U_I^(3).
 * Stage 1 is explicit (U_E^(1) = U_I^(1) = U^n, H_1 = F(U^n)); an implicit
 * stage is the stage operator with base U^n + dt sum_{j<i} aI_ij H_j,
 * linearisation state U_E^(i) and tau = gamma dt, and H_i is recovered from
 * its result as (U_I^(i) - base)/(gamma dt). */
static int ars222_step(void* ctx, stage_fn S, rhs_fn F, int64_t len, double* U, double dt,
                       double* work) {
    const double gamma = 1.0 - 1.0 / sqrt(2.0);
    const double delta = 1.0 - 1.0 / (2.0 * gamma);
    double* H1 = work;
    double* H2 = work + len;
    double* Ue = work + 2 * len;
    double* Ub = work + 3 * len;
    double* Ui = work + 4 * len;
    int rc = F(ctx, len, U, H1);
    if (rc != ORACLE_OK) return rc;
    for (int64_t k = 0; k < len; ++k) Ue[k] = U[k] + dt * gamma * H1[k];
    rc = S(ctx, len, U, Ue, gamma * dt, Ui); /* stage 2: base U^n */
    if (rc != ORACLE_OK) return rc;
    for (int64_t k = 0; k < len; ++k) {
        H2[k] = (Ui[k] - U[k]) / (gamma * dt);
        Ue[k] = U[k] + dt * (delta * H1[k] + (1.0 - delta) * H2[k]);
        Ub[k] = U[k] + dt * (1.0 - gamma) * H2[k];
    }
    return S(ctx, len, Ub, Ue, gamma * dt, U); /* stage 3 */
}

/* First-order semi-implicit step: one stage with tau = dt. */
static int si1_step(void* ctx, stage_fn S, int64_t len, double* U, double dt, double* work) {
    double* Ui = work;
    const int rc = S(ctx, len, U, U, dt, Ui);
    if (rc == ORACLE_OK) memcpy(U, Ui, (size_t)len * sizeof(double));
    return rc;
}

/* Explicit steps: forward Euler U + dt F(U), and Heun's method
 * U* = U + dt F(U), U^{n+1} = (U + U* + dt F(U*))/2. */
static int euler_step(void* ctx, rhs_fn F, int64_t len, double* U, double dt, double* work) {
    double* L = work;
    const int rc = F(ctx, len, U, L);
    if (rc != ORACLE_OK) return rc;
    for (int64_t k = 0; k < len; ++k) U[k] = U[k] + dt * L[k];
    return ORACLE_OK;
}

static int heun_step(void* ctx, rhs_fn F, int64_t len, double* U, double dt, double* work) {
    double* L = work;
    double* Us = work + len;
    int rc = F(ctx, len, U, L);
    if (rc != ORACLE_OK) return rc;
    for (int64_t k = 0; k < len; ++k) Us[k] = U[k] + dt * L[k];
    rc = F(ctx, len, Us, L);
    if (rc != ORACLE_OK) return rc;
    for (int64_t k = 0; k < len; ++k) U[k] = 0.5 * (U[k] + Us[k] + dt * L[k]);
    return ORACLE_OK;
}

/* One step of the selected scheme (work holds 5 len values). */
static int scheme_step(int32_t scheme, void* ctx, stage_fn S, rhs_fn F, int64_t len, double* U,
                       double dt, double* work) {
    switch (scheme) {
        case ORACLE_SCHEME_PRINTED: return imex2_step(ctx, S, len, U, dt, work);
        case ORACLE_SCHEME_ARS222: return ars222_step(ctx, S, F, len, U, dt, work);
        case ORACLE_SCHEME_SI1: return si1_step(ctx, S, len, U, dt, work);
        case ORACLE_SCHEME_EX_HEUN: return heun_step(ctx, F, len, U, dt, work);
        case ORACLE_SCHEME_EX_EULER: return euler_step(ctx, F, len, U, dt, work);
        default: return ORACLE_ERR_ARG;
    }
}

/* hSGN stage on a packed state [h | q | m | r] of 4 n values */
static int hsgn_stage_packed(void* ctx, int64_t len, const double* Ub, const double* Ul,
                             double tau, double* Uo) {
    const oracle_params* p = (const oracle_params*)ctx;
    const int64_t n = p->n;
    (void)len;
    return stage_impl(p, Ub, Ub + n, Ub + 2 * n, Ub + 3 * n, Ul, Ul + n, Ul + 2 * n, Ul + 3 * n,
                      tau, Uo, Uo + n, Uo + 2 * n, Uo + 3 * n, NULL);
}

/* explicit right-hand side on a packed state */
static int hsgn_rhs_packed(void* ctx, int64_t len, const double* U, double* L) {
    const oracle_params* p = (const oracle_params*)ctx;
    const int64_t n = p->n;
    (void)len;
    return oracle_explicit_rhs(p, U, U + n, U + 2 * n, U + 3 * n, L, L + n, L + 2 * n, L + 3 * n);
}

/* n_steps steps of size dt (scheme p->scheme) on the state arrays (in place). */
int oracle_run(const oracle_params* p, double* h, double* q, double* m, double* r,
               double dt, int64_t n_steps) {
    if (!p || !h || !q || !m || !r || p->n < 3 || n_steps < 0) return ORACLE_ERR_ARG;
    const int64_t n = p->n;
    double* U = (double*)malloc((size_t)(4 * n) * sizeof(double));
    double* work = (double*)malloc((size_t)(20 * n) * sizeof(double));
    if (!U || !work) { free(U); free(work); return ORACLE_ERR_NOMEM; }
    memcpy(U, h, (size_t)n * sizeof(double));
    memcpy(U + n, q, (size_t)n * sizeof(double));
    memcpy(U + 2 * n, m, (size_t)n * sizeof(double));
    memcpy(U + 3 * n, r, (size_t)n * sizeof(double));
    int rc = ORACLE_OK;
    oracle_params ps = *p;
    for (int64_t s = 0; s < n_steps && rc == ORACLE_OK; ++s) {
        if (ps.rusanov) {
            /* global Rusanov speed of this step: max over cells of |u^n| (R5).
             * The fully explicit schemes treat every wave explicitly, so their
             * Rusanov speed is the spectral radius of the system, max of
             * |u| + c with c^2 = g h + (lambda/3) eta^2/h^2 (Sec. 2.2, eq.
             * (eq:hSGN_eigenvalues); reading R12) */
            const int spectral = ps.scheme == ORACLE_SCHEME_EX_HEUN ||
                                 ps.scheme == ORACLE_SCHEME_EX_EULER;
            double umax = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                if (!(U[i] > 0.0)) return free(U), free(work), ORACLE_ERR_DEPTH;
                double u = fabs(U[n + i] / U[i]);
                if (spectral) {
                    const double e = U[2 * n + i] / (U[i] * U[i]);
                    u += sqrt(ps.g * U[i] + (ps.lambda / 3.0) * e * e);
                }
                if (u > umax) umax = u;
            }
            ps.speed = umax;
        }
        rc = scheme_step(ps.scheme, (void*)&ps, hsgn_stage_packed, hsgn_rhs_packed, 4 * n, U, dt,
                         work);
    }
    if (rc == ORACLE_OK) {
        memcpy(h, U, (size_t)n * sizeof(double));
        memcpy(q, U + n, (size_t)n * sizeof(double));
        memcpy(m, U + 2 * n, (size_t)n * sizeof(double));
        memcpy(r, U + 3 * n, (size_t)n * sizeof(double));
    }
    free(U); free(work);
    return rc;
}

int oracle_step(const oracle_params* p, double* h, double* q, double* m, double* r, double dt) {
    return oracle_run(p, h, q, m, r, dt, 1);
}

/* Scalar split linear test equation y' = aE y + aI y: H(y_E, y_I) =
 * aE y_E + aI y_I, so a stage solves y = y_b + tau (aE y_l + aI y). */
typedef struct { double aE, aI; } scalar_ctx;

static int scalar_stage(void* ctx, int64_t len, const double* Ub, const double* Ul,
                        double tau, double* Uo) {
    const scalar_ctx* s = (const scalar_ctx*)ctx;
    for (int64_t k = 0; k < len; ++k) {
        const double den = 1.0 - tau * s->aI;
        if (!(den != 0.0)) return ORACLE_ERR_COERCIVE;
        Uo[k] = (Ub[k] + tau * s->aE * Ul[k]) / den;
    }
    return ORACLE_OK;
}

static int scalar_rhs(void* ctx, int64_t len, const double* U, double* L) {
    const scalar_ctx* s = (const scalar_ctx*)ctx;
    for (int64_t k = 0; k < len; ++k) L[k] = (s->aE + s->aI) * U[k];
    return ORACLE_OK;
}

int oracle_imex_scalar_scheme(int32_t scheme, double aE, double aI, double y, double dt,
                              int64_t n_steps, double* out) {
    if (!out || n_steps < 0) return ORACLE_ERR_ARG;
    scalar_ctx s = {aE, aI};
    double U[1] = {y};
    double work[5];
    for (int64_t k = 0; k < n_steps; ++k) {
        int rc = scheme_step(scheme, &s, scalar_stage, scalar_rhs, 1, U, dt, work);
        if (rc != ORACLE_OK) return rc;
    }
    *out = U[0];
    return ORACLE_OK;
}

int oracle_imex_scalar(double aE, double aI, double y, double dt, int64_t n_steps, double* out) {
    return oracle_imex_scalar_scheme(ORACLE_SCHEME_PRINTED, aE, aI, y, dt, n_steps, out);
}

/* ------------------------------------------------------------------------
 * Time step rule of Sec. 5: dt_bar = CFL dx / nu_max, then the material
 * condition MCFL = u_max dt / dx must not exceed `mcfl`; otherwise dt =
 * mcfl dx / u_max. nu = |u| + sqrt(g h + (lambda/3) eta^2/h^2) (reading R9).
 * Also returns nu_max and u_max.
 * ------------------------------------------------------------------------ */
int oracle_suggest_dt(const oracle_params* p, const double* h, const double* q,
                      const double* m, double cfl, double mcfl,
                      double* dt_out, double* nu_max_out, double* u_max_out) {
    if (!p || !h || !q || !m || !dt_out || p->n < 1 || !(cfl > 0.0)) return ORACLE_ERR_ARG;
    double numax = 0.0, umax = 0.0;
    for (int64_t i = 0; i < p->n; ++i) {
        if (!(h[i] > 0.0)) return ORACLE_ERR_DEPTH;
        const double u = q[i] / h[i];
        const double eta = m[i] / h[i];
        const double nu = fabs(u) + sqrt(p->g * h[i] + (p->lambda / 3.0) * sqr(eta / h[i]));
        if (nu > numax) numax = nu;
        if (fabs(u) > umax) umax = fabs(u);
    }
    double dt = cfl * p->dx / numax;
    if (mcfl > 0.0 && umax > 0.0 && umax * dt / p->dx > mcfl) dt = mcfl * p->dx / umax;
    *dt_out = dt;
    if (nu_max_out) *nu_max_out = numax;
    if (u_max_out) *u_max_out = umax;
    return ORACLE_OK;
}

/* ========================================================================
 * Discrete adjoint of the step (well-balanced form 1, global Rusanov speed).
 *
 * For a misfit J(U_out), the adjoint of a stage maps dJ/dU_out to dJ/dU_b,
 * dJ/dU_l, dJ/db and dJ/ds (s the Rusanov speed) by running the stage's
 * operations backwards: every forward formula of stage_impl (form 1) is
 * differentiated by the chain rule, each operation in reverse order of the
 * forward one:
 *   back-substitution  (q, m, r outputs; face forces Phi + beta_face dhbar)
 *   solve              dJ/dD = M^{-T} dJ/dhbar,  dJ/dM_ij = -(dJ/dD)_i hbar_j
 *   rows, right-hand side
 *   face forces Phi    (p^ jumps, bottom force, beta_face dh_l)
 *   p^, p~ per cell    (functions of h_l, m_l, m^dag)
 *   beta per cell      (functions of h_l, m_l, m^dag, eq. (eq:hSGN_alpha))
 *   starred values     (r^dag, m^dag with the bottom source, q^dag)
 *   Rusanov fluxes     (reconstruction of U_l, the speed s)
 * The adjoints of inputs are ADDED to the given arrays (callers zero them).
 * Requires form 1 (a zero bottom gives the flat-bottom variant of the form),
 * rusanov = 1 and recon = 1.
 * ======================================================================== */
static int stage_adjoint(const oracle_params* p, const double* const Ub[4],
                         const double* const Ul[4], double tau, const double* const Ao[4],
                         double* const Ab[4], double* const Al[4], double* Abathy,
                         double* Aspeed) {
    const int64_t n = p->n;
    if (p->form != 1 || !p->rusanov || !p->recon || n < 3) return ORACLE_ERR_ARG;
    const double dx = p->dx, g = p->g, lam = p->lambda, s = p->speed;
    const double* hl = Ul[0]; const double* ql = Ul[1];
    const double* ml = Ul[2]; const double* rl = Ul[3];
    const double* hb = Ub[0];
    const double* bb = p->bathy;
    const double Cc = tau * tau / (dx * dx), f2 = tau / (2.0 * dx), fd = tau / dx;
    const double lt2 = lam * tau * tau;
    int rc = ORACLE_OK;
    const int nn = 34;  /* work arrays below */
    double* w = (double*)calloc((size_t)nn * (size_t)(n + 1), sizeof(double));
    if (!w) return ORACLE_ERR_NOMEM;
    double* Fq = w;             double* Fm = w + (n + 1);   double* Fr = w + 2 * (n + 1);
    double* qs = w + 3 * (n + 1); double* ms = w + 4 * (n + 1); double* rs = w + 5 * (n + 1);
    double* be = w + 6 * (n + 1); double* ph = w + 7 * (n + 1); double* pt = w + 8 * (n + 1);
    double* Phi = w + 9 * (n + 1); double* A = w + 10 * (n + 1); double* B = w + 11 * (n + 1);
    double* C = w + 12 * (n + 1); double* D = w + 13 * (n + 1); double* hbar = w + 14 * (n + 1);
    double* mbar = w + 15 * (n + 1);
    double* Fq_a = w + 16 * (n + 1); double* Fm_a = w + 17 * (n + 1); double* Fr_a = w + 18 * (n + 1);
    double* qs_a = w + 19 * (n + 1); double* ms_a = w + 20 * (n + 1); double* rs_a = w + 21 * (n + 1);
    double* be_a = w + 22 * (n + 1); double* ph_a = w + 23 * (n + 1); double* pt_a = w + 24 * (n + 1);
    double* Phi_a = w + 25 * (n + 1); double* hbar_a = w + 26 * (n + 1); double* D_a = w + 27 * (n + 1);
    double* aT = w + 28 * (n + 1); double* cT = w + 29 * (n + 1);
    const int periodic = p->bc == BC_PERIODIC;
    double bsum = 0.0;
    (void)bsum;

    /* ---- forward recomputation (the operations of stage_impl, form 1) */
    rc = rusanov_fluxes(p, hl, ql, ml, rl, Fq, Fm, Fr);
    if (rc != ORACLE_OK) goto done;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t il = nb(p, i - 1), ir = nb(p, i + 1);
        rs[i] = Ub[3][i] - (tau / dx) * (Fr[i + 1] - Fr[i]) + lam * tau;
        ms[i] = Ub[2][i] - (tau / dx) * (Fm[i + 1] - Fm[i]) + tau * rs[i];
        if (bb) ms[i] -= tau * 1.5 * ql[i] * (bb[ir] - bb[il]) / (2.0 * dx);
        qs[i] = Ub[1][i] - (tau / dx) * (Fq[i + 1] - Fq[i]);
        const double h = hl[i];
        if (!(h > 0.0)) { rc = ORACLE_ERR_DEPTH; goto done; }
        const double eta = ml[i] / h;
        const double alpha = -(2.0 * eta / h - 1.0) / (3.0 * h);
        const double c2 = g * h + (lam / 3.0) * eta * eta / (h * h);
        const double a2 = c2 - lam * eta * alpha;
        const double beta1 = 1.0 + lam * tau * tau / (h * h);
        const double beta2 = 2.0 * lam * tau * tau / (beta1 * beta1 * h * h * h);
        be[i] = a2 + lam * alpha * beta2 * ms[i];
        const double ptil = (lam / 3.0) * (1.0 - eta / h);
        const double b1 = h * h / (h * h + lt2);
        pt[i] = ptil;
        ph[i] = g * h * h / 2.0 + eta * ptil + lam * alpha * (ms[i] * b1 - ml[i]);
    }
    for (int64_t k = -1; k < n; ++k) {
        const int64_t i0 = nb(p, k), i1 = nb(p, k + 1);
        const double db = bb ? bb[i1] - bb[i0] : 0.0;
        const double bbar = 0.5 * (be[i0] + be[i1]);
        Phi[k + 1] = (ph[i1] - ph[i0]) + (g * 0.5 * (hl[i0] + hl[i1]) + 1.5 * 0.5 * (pt[i0] + pt[i1])) * db
                   - bbar * (hl[i1] - hl[i0]);
    }
    for (int64_t i = 0; i < n; ++i) {
        const int64_t il = nb(p, i - 1), ir = nb(p, i + 1);
        const double bm = 0.5 * (be[il] + be[i]), bp = 0.5 * (be[i] + be[ir]);
        D[i] = hb[i] - f2 * (qs[ir] - qs[il]) + Cc * (Phi[i + 1] - Phi[i]);
        A[i] = -Cc * bm;
        C[i] = -Cc * bp;
        B[i] = 1.0 + Cc * (bm + bp);
        if (!periodic) {
            if (i == 0) { B[i] = 1.0 + Cc * bp; A[i] = 0.0; }
            if (i == n - 1) { B[i] = 1.0 + Cc * bm; C[i] = 0.0; }
        }
    }
    rc = oracle_tridiag_solve(n, periodic, A, B, C, D, hbar);
    if (rc != ORACLE_OK) goto done;
    for (int64_t i = 0; i < n; ++i) mbar[i] = ms[i] / (1.0 + lt2 / (hbar[i] * hbar[i]));

    /* ---- back-substitution */
    for (int64_t i = 0; i < n; ++i) {
        const int64_t il = nb(p, i - 1), ir = nb(p, i + 1);
        const double h = hbar[i], den = h * h + lt2;
        const double ho_a = Ao[0][i], qo_a = Ao[1][i], mo_a = Ao[2][i], ro_a = Ao[3][i];
        /* r = r^dag - lambda tau m / h^2 */
        rs_a[i] += ro_a;
        const double m_a = mo_a - ro_a * lam * tau / (h * h);
        hbar_a[i] += ho_a + ro_a * 2.0 * lam * tau * mbar[i] / (h * h * h);
        /* m = m^dag h^2 / (h^2 + lambda tau^2) */
        ms_a[i] += m_a * h * h / den;
        hbar_a[i] += m_a * ms[i] * 2.0 * h * lt2 / (den * den);
        /* q = q^dag - tau/(2dx) (F_{i+1/2} + F_{i-1/2}), F = Phi + beta_face (hbar jump) */
        qs_a[i] += qo_a;
        const double a = -f2 * qo_a;
        const double bp = 0.5 * (be[i] + be[ir]), bm = 0.5 * (be[il] + be[i]);
        const double jp = hbar[ir] - hbar[i], jm = hbar[i] - hbar[il];
        Phi_a[i + 1] += a;
        be_a[i] += 0.5 * a * jp;
        be_a[ir] += 0.5 * a * jp;
        hbar_a[ir] += a * bp;
        hbar_a[i] -= a * bp;
        Phi_a[i] += a;
        be_a[il] += 0.5 * a * jm;
        be_a[i] += 0.5 * a * jm;
        hbar_a[i] += a * bm;
        hbar_a[il] -= a * bm;
    }

    /* ---- solve: dJ/dD = M^{-T} dJ/dhbar (rows of the transposed matrix) */
    for (int64_t i = 0; i < n; ++i) {
        aT[i] = i > 0 ? C[i - 1] : (periodic ? C[n - 1] : 0.0);
        cT[i] = i < n - 1 ? A[i + 1] : (periodic ? A[0] : 0.0);
    }
    rc = oracle_tridiag_solve(n, periodic, aT, B, cT, hbar_a, D_a);
    if (rc != ORACLE_OK) goto done;

    /* ---- rows and right-hand side */
    for (int64_t i = 0; i < n; ++i) {
        const int64_t il = nb(p, i - 1), ir = nb(p, i + 1);
        const double A_a = -D_a[i] * hbar[il], B_a = -D_a[i] * hbar[i], C_a = -D_a[i] * hbar[ir];
        double bm_a = -Cc * A_a + Cc * B_a, bp_a = -Cc * C_a + Cc * B_a;
        if (!periodic && i == 0) bm_a = 0.0;
        if (!periodic && i == n - 1) bp_a = 0.0;
        be_a[il] += 0.5 * bm_a;
        be_a[i] += 0.5 * bm_a + 0.5 * bp_a;
        be_a[ir] += 0.5 * bp_a;
        Ab[0][i] += D_a[i];
        qs_a[ir] -= f2 * D_a[i];
        qs_a[il] += f2 * D_a[i];
        Phi_a[i + 1] += Cc * D_a[i];
        Phi_a[i] -= Cc * D_a[i];
    }

    /* ---- face forces Phi_{k+1/2}, k = -1 .. n-1 */
    for (int64_t k = -1; k < n; ++k) {
        const int64_t i0 = nb(p, k), i1 = nb(p, k + 1);
        const double a = Phi_a[k + 1];
        const double db = bb ? bb[i1] - bb[i0] : 0.0;
        const double G = g * 0.5 * (hl[i0] + hl[i1]) + 1.5 * 0.5 * (pt[i0] + pt[i1]);
        const double bbar = 0.5 * (be[i0] + be[i1]), dhl = hl[i1] - hl[i0];
        ph_a[i1] += a;
        ph_a[i0] -= a;
        const double G_a = a * db;
        Al[0][i0] += 0.5 * g * G_a;
        Al[0][i1] += 0.5 * g * G_a;
        pt_a[i0] += 0.75 * G_a;
        pt_a[i1] += 0.75 * G_a;
        if (bb && Abathy) {
            Abathy[i1] += a * G;
            Abathy[i0] -= a * G;
        }
        be_a[i0] += 0.5 * (-a * dhl);
        be_a[i1] += 0.5 * (-a * dhl);
        Al[0][i1] -= a * bbar;
        Al[0][i0] += a * bbar;
    }

    /* ---- p^ and p~ per cell:
     *   e = m_l/h^2, eta = m_l/h, p~ = (lambda/3)(1 - e), alpha = -(2e - 1)/(3h),
     *   b_1 = h^2/(h^2 + lambda tau^2), w = m^dag b_1 - m_l,
     *   p^ = g h^2/2 + eta p~ + lambda alpha w */
    for (int64_t i = 0; i < n; ++i) {
        const double h = hl[i], m = ml[i];
        const double e = m / (h * h), eta = m / h;
        const double alpha = -(2.0 * e - 1.0) / (3.0 * h);
        const double den = h * h + lt2, b1 = h * h / den;
        const double wv = ms[i] * b1 - m;
        const double a = ph_a[i];
        const double ptot_a = pt_a[i] + a * eta;
        const double eta_a = a * pt[i];
        const double alpha_a = a * lam * wv;
        const double w_a = a * lam * alpha;
        double h_a = a * g * h, m_a = -w_a, e_a = 0.0;
        ms_a[i] += w_a * b1;
        const double b1_a = w_a * ms[i];
        h_a += b1_a * 2.0 * h * lt2 / (den * den);
        e_a += alpha_a * (-2.0 / (3.0 * h));
        h_a += alpha_a * (2.0 * e - 1.0) / (3.0 * h * h);
        e_a += -(lam / 3.0) * ptot_a;
        m_a += eta_a / h;
        h_a += -eta_a * m / (h * h);
        m_a += e_a / (h * h);
        h_a += -2.0 * e_a * m / (h * h * h);
        Al[0][i] += h_a;
        Al[2][i] += m_a;
    }

    /* ---- beta per cell (eq. (eq:hSGN_alpha) and the semi-discrete beta):
     *   eta = m_l/h, alpha = -(2 eta/h - 1)/(3h), c^2 = g h + (lambda/3) eta^2/h^2,
     *   a^2 = c^2 - lambda eta alpha, beta_1 = 1 + lambda tau^2/h^2,
     *   beta_2 = 2 lambda tau^2/(beta_1^2 h^3), beta = a^2 + lambda alpha beta_2 m^dag */
    for (int64_t i = 0; i < n; ++i) {
        const double h = hl[i], m = ml[i];
        const double eta = m / h;
        const double alpha = -(2.0 * eta / h - 1.0) / (3.0 * h);
        const double beta1 = 1.0 + lt2 / (h * h);
        const double beta2 = 2.0 * lt2 / (beta1 * beta1 * h * h * h);
        const double a = be_a[i];
        const double a2_a = a;
        double alpha_a = a * lam * beta2 * ms[i];
        const double beta2_a = a * lam * alpha * ms[i];
        ms_a[i] += a * lam * alpha * beta2;
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
        Al[2][i] += eta_a / h;
        h_a += -eta_a * m / (h * h);
        Al[0][i] += h_a;
    }

    /* ---- starred values: m^dag first (it feeds r^dag), then r^dag, q^dag */
    for (int64_t i = 0; i < n; ++i) {
        const int64_t il = nb(p, i - 1), ir = nb(p, i + 1);
        const double a = ms_a[i];
        Ab[2][i] += a;
        Fm_a[i + 1] -= fd * a;
        Fm_a[i] += fd * a;
        rs_a[i] += tau * a;
        if (bb) {
            const double k = -tau * 1.5 / (2.0 * dx);
            Al[1][i] += k * (bb[ir] - bb[il]) * a;
            if (Abathy) {
                Abathy[ir] += k * ql[i] * a;
                Abathy[il] -= k * ql[i] * a;
            }
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        Ab[3][i] += rs_a[i];
        Fr_a[i + 1] -= fd * rs_a[i];
        Fr_a[i] += fd * rs_a[i];
        Ab[1][i] += qs_a[i];
        Fq_a[i + 1] -= fd * qs_a[i];
        Fq_a[i] += fd * qs_a[i];
    }

    /* ---- Rusanov fluxes and the reconstruction of U_l (face k+1/2 at k+1) */
    for (int64_t k = -1; k < n; ++k) {
        const int64_t im = nb(p, k - 1), i0 = nb(p, k), i1 = nb(p, k + 1), i2 = nb(p, k + 2);
        const double hL = hl[i0] + (hl[i1] - hl[im]) / 4.0, hR = hl[i1] - (hl[i2] - hl[i0]) / 4.0;
        const double qL = ql[i0] + (ql[i1] - ql[im]) / 4.0, qR = ql[i1] - (ql[i2] - ql[i0]) / 4.0;
        const double mL = ml[i0] + (ml[i1] - ml[im]) / 4.0, mR = ml[i1] - (ml[i2] - ml[i0]) / 4.0;
        const double rL = rl[i0] + (rl[i1] - rl[im]) / 4.0, rR = rl[i1] - (rl[i2] - rl[i0]) / 4.0;
        const double uL = qL / hL, uR = qR / hR;
        const double aq = Fq_a[k + 1], am = Fm_a[k + 1], ar = Fr_a[k + 1];
        const double uL_a = 0.5 * (aq * qL + am * mL + ar * rL);
        const double uR_a = 0.5 * (aq * qR + am * mR + ar * rR);
        double qL_a = 0.5 * aq * (uL + s), qR_a = 0.5 * aq * (uR - s);
        const double mL_a = 0.5 * am * (uL + s), mR_a = 0.5 * am * (uR - s);
        const double rL_a = 0.5 * ar * (uL + s), rR_a = 0.5 * ar * (uR - s);
        if (Aspeed) *Aspeed += -0.5 * (aq * (qR - qL) + am * (mR - mL) + ar * (rR - rL));
        qL_a += uL_a / hL;
        qR_a += uR_a / hR;
        const double hL_a = -uL_a * uL / hL, hR_a = -uR_a * uR / hR;
        const double vL_a[4] = {hL_a, qL_a, mL_a, rL_a}, vR_a[4] = {hR_a, qR_a, mR_a, rR_a};
        for (int v = 0; v < 4; ++v) {
            Al[v][i0] += vL_a[v] + 0.25 * vR_a[v];
            Al[v][i1] += 0.25 * vL_a[v] + vR_a[v];
            Al[v][im] -= 0.25 * vL_a[v];
            Al[v][i2] -= 0.25 * vR_a[v];
        }
    }
done:
    free(w);
    return rc;
}

/* Adjoint of a stage on caller arrays (test entry point): the adjoints are
 * added to Ab (4 arrays), Al (4 arrays), *Abathy (n, may be NULL) and
 * *Aspeed (may be NULL). */
int oracle_stage_adjoint(const oracle_params* p, const double* hb, const double* qb,
                         const double* mb, const double* rb, const double* hl, const double* ql,
                         const double* ml, const double* rl, double tau, const double* ho_a,
                         const double* qo_a, const double* mo_a, const double* ro_a,
                         double* hb_a, double* qb_a, double* mb_a, double* rb_a, double* hl_a,
                         double* ql_a, double* ml_a, double* rl_a, double* bathy_a,
                         double* speed_a) {
    if (!p) return ORACLE_ERR_ARG;
    const double* Ub[4] = {hb, qb, mb, rb};
    const double* Ul[4] = {hl, ql, ml, rl};
    const double* Ao[4] = {ho_a, qo_a, mo_a, ro_a};
    double* Ab[4] = {hb_a, qb_a, mb_a, rb_a};
    double* Al[4] = {hl_a, ql_a, ml_a, rl_a};
    return stage_adjoint(p, Ub, Ul, tau, Ao, Ab, Al, bathy_a, speed_a);
}

/* ------------------------------------------------------------------------
 * Gradient of the gauge misfit
 *   J = 1/2 sum_{s=1..n_steps} sum_g (h_{c_g}^s - d_{s,g})^2 dt
 * (h^s the depth after step s, c_g the gauge cells, d the data, n_steps x
 * n_gauges row-major) with respect to the initial state and the bottom, for
 * the paper's two-stage step (efficient form) in form 1 with the global
 * Rusanov speed s^n = max_i |q_i/h_i| of each step (its subgradient goes to
 * the first cell attaining the maximum). All states of the run are kept (the
 * oracle serves small cases). On return U holds the final state, *misfit J
 * and gU (4 arrays) / gb (n, may be NULL) the gradient.
 * ------------------------------------------------------------------------ */
int oracle_adjoint(const oracle_params* p, double* h, double* q, double* m, double* r, double dt,
                   int64_t n_steps, int64_t n_gauges, const int64_t* gauge_cells,
                   const double* gauge_data, double* misfit, double* gh, double* gq, double* gm,
                   double* gr, double* gb) {
    if (!p || !h || !q || !m || !r || !misfit || !gh || !gq || !gm || !gr || n_steps < 0 ||
        n_gauges < 0 || (n_gauges > 0 && (!gauge_cells || !gauge_data)) || p->form != 1 ||
        !p->rusanov || !p->recon || p->scheme != ORACLE_SCHEME_PRINTED)
        return ORACLE_ERR_ARG;
    const int64_t n = p->n;
    for (int64_t k = 0; k < n_gauges; ++k)
        if (gauge_cells[k] < 0 || gauge_cells[k] >= n) return ORACLE_ERR_ARG;
    const double gam = 1.0 - 1.0 / sqrt(2.0), c = 1.0 / (2.0 * gam);
    const double wl0 = 1.0 - c / gam, wl1 = c / gam;
    const double wb0 = 1.0 - (1.0 - gam) / gam, wb1 = (1.0 - gam) / gam;
    const double tau = gam * dt;
    const size_t st = (size_t)(4 * n);
    double* S = (double*)malloc((size_t)(n_steps + 1) * st * sizeof(double)); /* states */
    double* sp = (double*)malloc((size_t)(n_steps + 1) * sizeof(double));
    int64_t* am = (int64_t*)malloc((size_t)(n_steps + 1) * sizeof(int64_t));
    double* wk = (double*)calloc(24 * (size_t)n, sizeof(double));
    if (!S || !sp || !am || !wk) { free(S); free(sp); free(am); free(wk); return ORACLE_ERR_NOMEM; }
    int rc = ORACLE_OK;
    memcpy(S, h, (size_t)n * sizeof(double));
    memcpy(S + n, q, (size_t)n * sizeof(double));
    memcpy(S + 2 * n, m, (size_t)n * sizeof(double));
    memcpy(S + 3 * n, r, (size_t)n * sizeof(double));
    oracle_params ps = *p;
    double J = 0.0;
    /* forward, keeping every state, its speed and its argmax cell */
    for (int64_t s = 0; s < n_steps; ++s) {
        double* U = S + (size_t)s * st;
        double umax = 0.0;
        int64_t imax = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (!(U[i] > 0.0)) { rc = ORACLE_ERR_DEPTH; goto done; }
            const double u = fabs(U[n + i] / U[i]);
            if (u > umax) { umax = u; imax = i; }
        }
        sp[s] = umax;
        am[s] = imax;
        ps.speed = umax;
        memcpy(U + st, U, st * sizeof(double));
        double work[1];
        (void)work;
        double* W = (double*)malloc(12 * (size_t)n * sizeof(double));
        if (!W) { rc = ORACLE_ERR_NOMEM; goto done; }
        rc = imex2_step((void*)&ps, hsgn_stage_packed, 4 * n, U + st, dt, W);
        free(W);
        if (rc != ORACLE_OK) goto done;
        for (int64_t k = 0; k < n_gauges; ++k) {
            const double e = U[st + gauge_cells[k]] - gauge_data[s * n_gauges + k];
            J += 0.5 * e * e * dt;
        }
    }
    /* reverse */
    {
        double* Ua = wk;                 /* dJ/dU^s (4n) */
        double* Ua1 = wk + 4 * n;        /* dJ/dU_I^(1) */
        double* Ab = wk + 8 * n;         /* stage base adjoint */
        double* Al = wk + 12 * n;        /* stage linearisation adjoint */
        double* U1 = wk + 16 * n;        /* U_I^(1) */
        double* Ue = wk + 20 * n;        /* stage-2 linearisation state */
        double* Ubs = (double*)malloc(st * sizeof(double));
        double* Ab2 = (double*)malloc(st * sizeof(double));
        if (!Ubs || !Ab2) { free(Ubs); free(Ab2); rc = ORACLE_ERR_NOMEM; goto done; }
        memset(Ua, 0, st * sizeof(double));
        if (gb) memset(gb, 0, (size_t)n * sizeof(double));
        for (int64_t s = n_steps - 1; s >= 0 && rc == ORACLE_OK; --s) {
            const double* U = S + (size_t)s * st;
            const double* Un = S + (size_t)(s + 1) * st;
            for (int64_t k = 0; k < n_gauges; ++k)
                Ua[gauge_cells[k]] += (Un[gauge_cells[k]] - gauge_data[s * n_gauges + k]) * dt;
            ps.speed = sp[s];
            /* recompute the stage-1 result and the stage-2 states */
            const double* Uv[4] = {U, U + n, U + 2 * n, U + 3 * n};
            double* U1v[4] = {U1, U1 + n, U1 + 2 * n, U1 + 3 * n};
            rc = stage_impl(&ps, Uv[0], Uv[1], Uv[2], Uv[3], Uv[0], Uv[1], Uv[2], Uv[3], tau,
                            U1v[0], U1v[1], U1v[2], U1v[3], NULL);
            if (rc != ORACLE_OK) break;
            for (size_t k = 0; k < st; ++k) {
                Ue[k] = wl0 * U[k] + wl1 * U1[k];
                Ubs[k] = wb0 * U[k] + wb1 * U1[k];
            }
            double speed_a = 0.0;
            /* stage 2 */
            memset(Ab, 0, st * sizeof(double));
            memset(Al, 0, st * sizeof(double));
            {
                const double* Ubv[4] = {Ubs, Ubs + n, Ubs + 2 * n, Ubs + 3 * n};
                const double* Ulv[4] = {Ue, Ue + n, Ue + 2 * n, Ue + 3 * n};
                const double* Aov[4] = {Ua, Ua + n, Ua + 2 * n, Ua + 3 * n};
                double* Abv[4] = {Ab, Ab + n, Ab + 2 * n, Ab + 3 * n};
                double* Alv[4] = {Al, Al + n, Al + 2 * n, Al + 3 * n};
                rc = stage_adjoint(&ps, Ubv, Ulv, tau, Aov, Abv, Alv, gb, &speed_a);
                if (rc != ORACLE_OK) break;
            }
            for (size_t k = 0; k < st; ++k) {
                Ua1[k] = wl1 * Al[k] + wb1 * Ab[k];
                Ua[k] = wl0 * Al[k] + wb0 * Ab[k];
            }
            /* stage 1: U_b = U_l = U^s */
            memset(Ab2, 0, st * sizeof(double));
            memset(Al, 0, st * sizeof(double));
            {
                const double* Aov[4] = {Ua1, Ua1 + n, Ua1 + 2 * n, Ua1 + 3 * n};
                double* Abv[4] = {Ab2, Ab2 + n, Ab2 + 2 * n, Ab2 + 3 * n};
                double* Alv[4] = {Al, Al + n, Al + 2 * n, Al + 3 * n};
                rc = stage_adjoint(&ps, Uv, Uv, tau, Aov, Abv, Alv, gb, &speed_a);
                if (rc != ORACLE_OK) break;
            }
            for (size_t k = 0; k < st; ++k) Ua[k] += Ab2[k] + Al[k];
            /* the step's speed s = |q/h| at its argmax cell */
            {
                const int64_t i = am[s];
                const double hh = U[i], qq = U[n + i];
                const double sg = qq > 0.0 ? 1.0 : (qq < 0.0 ? -1.0 : 0.0);
                Ua[n + i] += speed_a * sg / hh;
                Ua[i] += -speed_a * fabs(qq) / (hh * hh);
            }
        }
        free(Ubs);
        free(Ab2);
        if (rc == ORACLE_OK) {
            memcpy(gh, Ua, (size_t)n * sizeof(double));
            memcpy(gq, Ua + n, (size_t)n * sizeof(double));
            memcpy(gm, Ua + 2 * n, (size_t)n * sizeof(double));
            memcpy(gr, Ua + 3 * n, (size_t)n * sizeof(double));
            const double* Uf = S + (size_t)n_steps * st;
            memcpy(h, Uf, (size_t)n * sizeof(double));
            memcpy(q, Uf + n, (size_t)n * sizeof(double));
            memcpy(m, Uf + 2 * n, (size_t)n * sizeof(double));
            memcpy(r, Uf + 3 * n, (size_t)n * sizeof(double));
            *misfit = J;
        }
    }
done:
    free(S); free(sp); free(am); free(wk);
    return rc;
}
