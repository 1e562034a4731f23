// hsgn_tridiag.cuh -- block-partitioned tridiagonal elimination for one CTA.
//
// The depth system of the semi-implicit stage (Sec. 4.2, eq.
// (GN_hyp_eq_semi_fully_discrete), "Delta[hbar]_i = h^dagger_i") is a
// symmetric, strictly diagonally dominant tridiagonal matrix (cyclic when
// periodic). It is solved exactly by a separator (Schur-complement) method:
//
//  * A block of `nrows` consecutive rows is owned by one CTA. Its LAST row is
//    the block separator x_R; the row before the block is x_L (the previous
//    block's separator). For every other row the CTA computes (y, v, w) with
//        x_i = y_i - x_L v_i - x_R w_i .
//  * Inside the CTA each thread owns a contiguous chunk of rows; the chunk's
//    last row is a thread separator. The chunk interior is eliminated by the
//    Thomas algorithm with three right-hand sides (d, the coupling to the left
//    separator, the coupling to the right separator).
//  * The thread separators satisfy a tridiagonal system of their own (the
//    Schur complement), solved by parallel cyclic reduction in shared memory,
//    again with three right-hand sides.
//
// Cost per row: one reciprocal and about ten multiply-adds in the chunk sweep
// plus six in the recombination; the cyclic reduction touches one row in
// `rows per thread`. No pivoting: pivots of an M-matrix stay positive; a
// non-positive pivot sets HSGN_DEV_ERR_COERCIVE.
#pragma once

#include <cstdint>

#define HSGN_DEV_ERR_DEPTH 1u
#define HSGN_DEV_ERR_COERCIVE 2u
#define HSGN_DEV_ERR_NONFINITE 4u

namespace hsgn {

__device__ __forceinline__ void flag_error(unsigned* err, unsigned bits) {
    if (err) atomicOr(err, bits);
}

// x > 0 and finite, tested on the bit pattern (integer pipe; false for +-0,
// negatives, +Inf and NaN).
__device__ __forceinline__ bool pos_finite(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b - 1ull) < 0x7FEFFFFFFFFFFFFFull;
}

__device__ __forceinline__ bool finite_bits(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b & 0x7FF0000000000000ull) != 0x7FF0000000000000ull;
}

// Reciprocal. The IEEE division is used: on sm_103a it outruns a Newton-Raphson
// reciprocal seeded in single precision (77 vs 65 Gop/s measured), because the
// single/double conversions of the seed cost more than the division's own
// refinement steps.
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

// Shared memory of the separator system of a CTA with T threads.
template <int T>
struct SepShared {
    double A[T], B[T], C[T], D1[T], D2[T], D3[T];
    double YF[T], VF[T], WF[T];
};

// Chunk of rows [cs, cs + m) owned by thread t when `nrows` rows are split as
// evenly as possible over min(T, nrows) threads.
template <int T>
__device__ __forceinline__ void chunk_of(int nrows, int t, int& cs, int& m, int& teff) {
    teff = nrows < T ? nrows : T;
    if (t >= teff) {
        cs = nrows;
        m = 0;
        return;
    }
    const int base = nrows / teff, extra = nrows % teff;
    m = base + (t < extra ? 1 : 0);
    cs = t * base + (t < extra ? t : extra);
}

// Eliminate a block of `nrows` rows (1 <= nrows <= T*M). All T threads of the
// CTA must call it. `row(i, a, b, c, d)` returns local row i (0 <= i < nrows).
// On return thread t holds, for k < m, the triple (y, v, w) of row cs + k; the
// block separator (row nrows - 1) gets (0, 0, -1). The thread that owns the
// last row also returns its coefficients in last[0..3].
template <int T, int M, class RowFn>
__device__ __forceinline__ void cta_block_solve(int nrows, RowFn row, SepShared<T>& sh,
                                                double (&y)[M], double (&v)[M], double (&w)[M],
                                                int& cs, int& m, double (&last)[4],
                                                unsigned* err) {
    const int t = threadIdx.x;
    int teff;
    chunk_of<T>(nrows, t, cs, m, teff);
    const int nint = m - 1;  // interior rows of the chunk (the last row is its separator)

    // ---- 1. Thomas sweep of the chunk interior with three right-hand sides:
    //         y <- d, v <- a_first e_first, w <- c_last e_last.
    //         Forward: w holds c', y holds g (rhs d), v holds gv (rhs a e_0).
    double sa = 0.0, sb = 1.0, sc = 0.0, sd = 0.0;  // separator row of the chunk
    bool bad = false;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        if (k < nint) {
            double a, b, c, d;
            row(cs + k, a, b, c, d);
            double p, ip;
            if (k == 0) {
                p = b;
                ip = rcp(p);
                y[k] = d * ip;
                v[k] = a * ip;
            } else {
                p = fma(-a, w[k - 1], b);
                ip = rcp(p);
                y[k] = fma(-a, y[k - 1], d) * ip;
                v[k] = -a * v[k - 1] * ip;
            }
            bad |= !pos_finite(p);
            w[k] = c * ip;
        }
    }
    if (m > 0) row(cs + m - 1, sa, sb, sc, sd);
    // backward substitution: Y_k = g_k - c'_k Y_{k+1}, V likewise, W_k = -c'_k W_{k+1}.
    // The last interior values (YL, VL, WL) are kept in scalars; an empty
    // interior means the row before the separator is the previous separator.
    double YL = 0.0, VL = -1.0, WL = 0.0;
    {
        // seeds make the first executed row (k = nint-1) give Y = g, V = gv, W = c'
        double Yn = 0.0, Vn = 0.0, Wn = -1.0;
#pragma unroll
        for (int k = M - 1; k >= 0; --k) {
            if (k < nint) {
                const double Y = fma(-w[k], Yn, y[k]);
                const double V = fma(-w[k], Vn, v[k]);
                const double W = -w[k] * Wn;
                if (k == nint - 1) {
                    YL = Y;
                    VL = V;
                    WL = W;
                }
                y[k] = Y;
                v[k] = V;
                w[k] = W;
                Yn = Y;
                Vn = V;
                Wn = W;
            }
        }
    }
    if (bad) flag_error(err, HSGN_DEV_ERR_COERCIVE);

    // first-interior values of the chunk; an empty interior means the row
    // after the previous separator is this chunk's separator: (0, 0, -1)
    if (t < teff) {
        sh.YF[t] = nint > 0 ? y[0] : 0.0;
        sh.VF[t] = nint > 0 ? v[0] : 0.0;
        sh.WF[t] = nint > 0 ? w[0] : -1.0;
    }
    __syncthreads();

    // ---- 2. separator system: sigma_t for t < teff - 1, with external
    //         sigma_{-1} = x_L and sigma_{teff-1} = x_R moved to the right side.
    const int ns = teff - 1;
    if (t < ns) {
        const double YF1 = sh.YF[t + 1], VF1 = sh.VF[t + 1], WF1 = sh.WF[t + 1];
        const double At = -sa * VL;
        const double Bt = sb - sa * WL - sc * VF1;
        const double Ct = -sc * WF1;
        const double Dt = sd - sa * YL - sc * YF1;
        sh.A[t] = (t == 0) ? 0.0 : At;
        sh.C[t] = (t == ns - 1) ? 0.0 : Ct;
        sh.B[t] = Bt;
        sh.D1[t] = Dt;
        sh.D2[t] = (t == 0) ? At : 0.0;
        sh.D3[t] = (t == ns - 1) ? Ct : 0.0;
    }
    if (t == teff - 1) {
        last[0] = sa;
        last[1] = sb;
        last[2] = sc;
        last[3] = sd;
    }
    __syncthreads();

    // parallel cyclic reduction over the ns separator rows; each level first
    // stores 1/B of every row so that both neighbours reuse it
    bool badp = false;
    for (int s = 1; s < ns; s <<= 1) {
        if (t < ns) sh.YF[t] = rcp(sh.B[t]);
        __syncthreads();
        double nA = 0.0, nB = 0.0, nC = 0.0, n1 = 0.0, n2 = 0.0, n3 = 0.0;
        if (t < ns) {
            nB = sh.B[t];
            n1 = sh.D1[t];
            n2 = sh.D2[t];
            n3 = sh.D3[t];
            if (t - s >= 0) {
                const double k1 = sh.A[t] * sh.YF[t - s];
                nA = -sh.A[t - s] * k1;
                nB = fma(-sh.C[t - s], k1, nB);
                n1 = fma(-sh.D1[t - s], k1, n1);
                n2 = fma(-sh.D2[t - s], k1, n2);
                n3 = fma(-sh.D3[t - s], k1, n3);
            }
            if (t + s < ns) {
                const double k2 = sh.C[t] * sh.YF[t + s];
                nC = -sh.C[t + s] * k2;
                nB = fma(-sh.A[t + s], k2, nB);
                n1 = fma(-sh.D1[t + s], k2, n1);
                n2 = fma(-sh.D2[t + s], k2, n2);
                n3 = fma(-sh.D3[t + s], k2, n3);
            }
        }
        __syncthreads();
        if (t < ns) {
            sh.A[t] = nA;
            sh.B[t] = nB;
            sh.C[t] = nC;
            sh.D1[t] = n1;
            sh.D2[t] = n2;
            sh.D3[t] = n3;
        }
        __syncthreads();
    }
    if (t < ns) {
        const double Bt = sh.B[t];
        badp = !pos_finite(Bt);
        const double iB = rcp(Bt);
        sh.D1[t] *= iB;  // Ys
        sh.D2[t] *= iB;  // Vs
        sh.D3[t] *= iB;  // Ws
    }
    if (badp) flag_error(err, HSGN_DEV_ERR_COERCIVE);
    __syncthreads();

    // ---- 3. recombination: sigma_t = Ys_t - x_L Vs_t - x_R Ws_t, with the
    //         externals sigma_{-1} = x_L -> (0, -1, 0), sigma_{teff-1} = x_R -> (0, 0, -1)
    if (t < teff) {
        double YsL, VsL, WsL, YsR, VsR, WsR;
        if (t == 0) {
            YsL = 0.0;
            VsL = -1.0;
            WsL = 0.0;
        } else {
            YsL = sh.D1[t - 1];
            VsL = sh.D2[t - 1];
            WsL = sh.D3[t - 1];
        }
        if (t == teff - 1) {
            YsR = 0.0;
            VsR = 0.0;
            WsR = -1.0;
        } else {
            YsR = sh.D1[t];
            VsR = sh.D2[t];
            WsR = sh.D3[t];
        }
#pragma unroll
        for (int k = 0; k < M; ++k) {
            if (k < nint) {
                const double Y = y[k], V = v[k], W = w[k];
                y[k] = Y - YsL * V - YsR * W;
                v[k] = -(VsL * V + VsR * W);
                w[k] = -(WsL * V + WsR * W);
            } else if (k == nint) {
                y[k] = YsR;
                v[k] = VsR;
                w[k] = WsR;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The same elimination done by one warp: lane t owns a chunk of at most M rows,
// the separator system of the chunks (at most 31 rows) is solved by parallel
// cyclic reduction in registers with warp shuffles, so no shared memory and no
// block barrier is involved. Same contract as cta_block_solve with T = 32;
// nrows <= 32 * M. All 32 lanes of the warp must call it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double shfl_up_d(double x, int s) {
    return __shfl_up_sync(0xffffffffu, x, s);
}
__device__ __forceinline__ double shfl_down_d(double x, int s) {
    return __shfl_down_sync(0xffffffffu, x, s);
}

template <int M, class RowFn>
__device__ __forceinline__ void warp_block_solve(int nrows, RowFn row, double (&y)[M],
                                                 double (&v)[M], double (&w)[M], int& cs, int& m,
                                                 double (&last)[4], unsigned* err) {
    const int t = threadIdx.x & 31;
    int teff;
    chunk_of<32>(nrows, t, cs, m, teff);
    const int nint = m - 1;

    double sa = 0.0, sb = 1.0, sc = 0.0, sd = 0.0;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        if (k < nint) {
            double a, b, c, d;
            row(cs + k, a, b, c, d);
            double p, ip;
            if (k == 0) {
                p = b;
                ip = rcp(p);
                y[k] = d * ip;
                v[k] = a * ip;
            } else {
                p = fma(-a, w[k - 1], b);
                ip = rcp(p);
                y[k] = fma(-a, y[k - 1], d) * ip;
                v[k] = -a * v[k - 1] * ip;
            }
            bad |= !pos_finite(p);
            w[k] = c * ip;
        }
    }
    if (m > 0) row(cs + m - 1, sa, sb, sc, sd);
    double YL = 0.0, VL = -1.0, WL = 0.0;
    {
        double Yn = 0.0, Vn = 0.0, Wn = -1.0;
#pragma unroll
        for (int k = M - 1; k >= 0; --k) {
            if (k < nint) {
                const double Y = fma(-w[k], Yn, y[k]);
                const double V = fma(-w[k], Vn, v[k]);
                const double W = -w[k] * Wn;
                if (k == nint - 1) {
                    YL = Y;
                    VL = V;
                    WL = W;
                }
                y[k] = Y;
                v[k] = V;
                w[k] = W;
                Yn = Y;
                Vn = V;
                Wn = W;
            }
        }
    }
    if (bad) flag_error(err, HSGN_DEV_ERR_COERCIVE);

    // first-interior values of the next lane's chunk
    const double YF0 = nint > 0 ? y[0] : 0.0;
    const double VF0 = nint > 0 ? v[0] : 0.0;
    const double WF0 = nint > 0 ? w[0] : -1.0;
    const double YF1 = shfl_down_d(YF0, 1), VF1 = shfl_down_d(VF0, 1), WF1 = shfl_down_d(WF0, 1);

    const int ns = teff - 1;
    double A = 0.0, B = 1.0, C = 0.0, D1 = 0.0, D2 = 0.0, D3 = 0.0;
    if (t < ns) {
        const double At = -sa * VL;
        const double Bt = sb - sa * WL - sc * VF1;
        const double Ct = -sc * WF1;
        const double Dt = sd - sa * YL - sc * YF1;
        A = (t == 0) ? 0.0 : At;
        C = (t == ns - 1) ? 0.0 : Ct;
        B = Bt;
        D1 = Dt;
        D2 = (t == 0) ? At : 0.0;
        D3 = (t == ns - 1) ? Ct : 0.0;
    }
    if (t == teff - 1) {
        last[0] = sa;
        last[1] = sb;
        last[2] = sc;
        last[3] = sd;
    }
    // cyclic reduction; lanes >= ns hold decoupled identity rows
    for (int s = 1; s < ns; s <<= 1) {
        const double iB = rcp(B);
        const double lA = shfl_up_d(A, s), lB = shfl_up_d(iB, s), lC = shfl_up_d(C, s);
        const double l1 = shfl_up_d(D1, s), l2 = shfl_up_d(D2, s), l3 = shfl_up_d(D3, s);
        const double rA = shfl_down_d(A, s), rB = shfl_down_d(iB, s), rC = shfl_down_d(C, s);
        const double r1 = shfl_down_d(D1, s), r2 = shfl_down_d(D2, s), r3 = shfl_down_d(D3, s);
        if (t < ns) {
            double nA = 0.0, nB = B, nC = 0.0, n1 = D1, n2 = D2, n3 = D3;
            if (t - s >= 0) {
                const double k1 = A * lB;
                nA = -lA * k1;
                nB = fma(-lC, k1, nB);
                n1 = fma(-l1, k1, n1);
                n2 = fma(-l2, k1, n2);
                n3 = fma(-l3, k1, n3);
            }
            if (t + s < ns) {
                const double k2 = C * rB;
                nC = -rC * k2;
                nB = fma(-rA, k2, nB);
                n1 = fma(-r1, k2, n1);
                n2 = fma(-r2, k2, n2);
                n3 = fma(-r3, k2, n3);
            }
            A = nA;
            B = nB;
            C = nC;
            D1 = n1;
            D2 = n2;
            D3 = n3;
        }
    }
    double Ys = 0.0, Vs = 0.0, Ws = 0.0;
    if (t < ns) {
        if (!pos_finite(B)) flag_error(err, HSGN_DEV_ERR_COERCIVE);
        const double iB = rcp(B);
        Ys = D1 * iB;
        Vs = D2 * iB;
        Ws = D3 * iB;
    }
    const double YsL0 = shfl_up_d(Ys, 1), VsL0 = shfl_up_d(Vs, 1), WsL0 = shfl_up_d(Ws, 1);
    if (t < teff) {
        double YsL, VsL, WsL, YsR, VsR, WsR;
        if (t == 0) {
            YsL = 0.0;
            VsL = -1.0;
            WsL = 0.0;
        } else {
            YsL = YsL0;
            VsL = VsL0;
            WsL = WsL0;
        }
        if (t == teff - 1) {
            YsR = 0.0;
            VsR = 0.0;
            WsR = -1.0;
        } else {
            YsR = Ys;
            VsR = Vs;
            WsR = Ws;
        }
#pragma unroll
        for (int k = 0; k < M; ++k) {
            if (k < nint) {
                const double Y = y[k], V = v[k], W = w[k];
                y[k] = Y - YsL * V - YsR * W;
                v[k] = -(VsL * V + VsR * W);
                w[k] = -(WsL * V + WsR * W);
            } else if (k == nint) {
                y[k] = YsR;
                v[k] = VsR;
                w[k] = WsR;
            }
        }
    }
}

}  // namespace hsgn
