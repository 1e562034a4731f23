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
#define HSGN_DEV_ERR_TRUNCATION 8u  // windowed solve: coupling decays too slowly

namespace hsgn {

// Shared-memory index with one pad word every 32: rows read by threads at a
// stride of 4 or 8 words (the chunk mapping) then fall in distinct banks.
__host__ __device__ __forceinline__ int pd(int i) { return i + (i >> 5); }
__host__ __device__ constexpr int pd_size(int n) { return n + (n >> 5) + 1; }

// No extra work for the warps that wait while warp 0 solves a separator system.
struct NoSide {
    __device__ void operator()(int) const {}
};

__device__ __forceinline__ void flag_error(unsigned* err, unsigned bits) {
    if (err) atomicOr(err, bits);
}

// x > 0 and finite, tested on the bit pattern (integer pipe; false for +-0,
// negatives, +Inf and NaN).
__device__ __forceinline__ bool pos_finite(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b - 1ull) < 0x7FEFFFFFFFFFFFFFull;
}

__device__ __forceinline__ bool pos_finite(float x) {
    const unsigned b = __float_as_uint(x);
    return (b - 1u) < 0x7F7FFFFFu;
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
// Single precision: the hardware approximation refined by one Newton-Raphson
// step for 1/x (e = 1 - x r, r' = r + r e), which brings it to about one ulp
// with three branch-free instructions.
__device__ __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return fmaf(r, fmaf(-x, r, 1.f), r);
}

// a * b + c in one rounding; the double-float pairs have an overload of the
// same name that skips the final renormalisation.
__device__ __forceinline__ float fma_u(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_u(double a, double b, double c) { return ::fma(a, b, c); }

// Barrier of the first n threads of the CTA (n a multiple of 32) on hardware
// barrier id (1 .. 15; __syncthreads uses 0), and the same barrier returning
// whether any of them passed a true predicate.
__device__ __forceinline__ void group_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ bool group_or(int id, int n, bool pred) {
    int r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\tsetp.ne.s32 pi, %1, 0;\n\t"
        "bar.red.or.pred po, %2, %3, pi;\n\tselp.s32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"((int)pred), "r"(id), "r"(n)
        : "memory");
    return r != 0;
}

// Leading single-precision value of a number (magnitude tests).
__device__ __forceinline__ float hi_of(float x) { return x; }
__device__ __forceinline__ float hi_of(double x) { return (float)x; }

// Shared memory of the separator system of a CTA with T threads.
// Indexed with pd(): warp 0 reads the rows at a stride of T/32.
template <int T, class Real = double>
struct SepShared {
    static constexpr int NP = pd_size(T);
    Real A[NP], B[NP], C[NP], D1[NP];
    Real YF[NP], VF[NP], WF[NP];  // first-interior values, then the separator triples
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
    // teff = T (a power of two: shift and mask) or teff = nrows (one row each)
    static_assert((T & (T - 1)) == 0, "T must be a power of two");
    const int base = nrows >= T ? nrows / T : 1, extra = nrows >= T ? nrows % T : 0;
    m = base + (t < extra ? 1 : 0);
    cs = t * base + (t < extra ? t : extra);
}

// ---------------------------------------------------------------------------
// The same elimination done by one warp: lane t owns a chunk of at most M rows,
// the separator system of the chunks (at most 31 rows) is solved by parallel
// cyclic reduction in registers with warp shuffles, so no shared memory and no
// block barrier is involved. Same contract as cta_block_solve with T = 32;
// nrows <= 32 * M. All 32 lanes of the warp must call it.
// ---------------------------------------------------------------------------
template <class Real>
__device__ __forceinline__ Real shfl_up_d(Real x, int s) {
    return __shfl_up_sync(0xffffffffu, x, s);
}
template <class Real>
__device__ __forceinline__ Real shfl_down_d(Real x, int s) {
    return __shfl_down_sync(0xffffffffu, x, s);
}

template <int M, class RowFn, class Real>
__device__ __forceinline__ void warp_block_solve(int nrows, RowFn row, Real (&y)[M],
                                                 Real (&v)[M], Real (&w)[M], int& cs, int& m,
                                                 Real (&last)[4], unsigned* err) {
    const int t = threadIdx.x & 31;
    int teff;
    chunk_of<32>(nrows, t, cs, m, teff);
    const int nint = m - 1;

    Real sa = Real(0), sb = Real(1), sc = Real(0), sd = Real(0);
    bool bad = false;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        if (k < nint) {
            Real a, b, c, d;
            row(cs + k, a, b, c, d);
            Real p, ip;
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
    Real YL = Real(0), VL = -Real(1), WL = Real(0);
    {
        Real Yn = Real(0), Vn = Real(0), Wn = -Real(1);
#pragma unroll
        for (int k = M - 1; k >= 0; --k) {
            if (k < nint) {
                const Real Y = fma(-w[k], Yn, y[k]);
                const Real V = fma(-w[k], Vn, v[k]);
                const Real W = -w[k] * Wn;
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
    const Real YF0 = nint > 0 ? y[0] : Real(0);
    const Real VF0 = nint > 0 ? v[0] : Real(0);
    const Real WF0 = nint > 0 ? w[0] : -Real(1);
    const Real YF1 = shfl_down_d(YF0, 1), VF1 = shfl_down_d(VF0, 1), WF1 = shfl_down_d(WF0, 1);

    const int ns = teff - 1;
    Real A = Real(0), B = Real(1), C = Real(0), D1 = Real(0), D2 = Real(0), D3 = Real(0);
    if (t < ns) {
        const Real At = -sa * VL;
        const Real Bt = sb - sa * WL - sc * VF1;
        const Real Ct = -sc * WF1;
        const Real Dt = sd - sa * YL - sc * YF1;
        A = (t == 0) ? Real(0) : At;
        C = (t == ns - 1) ? Real(0) : Ct;
        B = Bt;
        D1 = Dt;
        D2 = (t == 0) ? At : Real(0);
        D3 = (t == ns - 1) ? Ct : Real(0);
    }
    if (t == teff - 1) {
        last[0] = sa;
        last[1] = sb;
        last[2] = sc;
        last[3] = sd;
    }
    // cyclic reduction; lanes >= ns hold decoupled identity rows
    for (int s = 1; s < ns; s <<= 1) {
        const Real iB = rcp(B);
        const Real lA = shfl_up_d(A, s), lB = shfl_up_d(iB, s), lC = shfl_up_d(C, s);
        const Real l1 = shfl_up_d(D1, s), l2 = shfl_up_d(D2, s), l3 = shfl_up_d(D3, s);
        const Real rA = shfl_down_d(A, s), rB = shfl_down_d(iB, s), rC = shfl_down_d(C, s);
        const Real r1 = shfl_down_d(D1, s), r2 = shfl_down_d(D2, s), r3 = shfl_down_d(D3, s);
        if (t < ns) {
            Real nA = Real(0), nB = B, nC = Real(0), n1 = D1, n2 = D2, n3 = D3;
            if (t - s >= 0) {
                const Real k1 = A * lB;
                nA = -lA * k1;
                nB = fma(-lC, k1, nB);
                n1 = fma(-l1, k1, n1);
                n2 = fma(-l2, k1, n2);
                n3 = fma(-l3, k1, n3);
            }
            if (t + s < ns) {
                const Real k2 = C * rB;
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
    Real Ys = Real(0), Vs = Real(0), Ws = Real(0);
    if (t < ns) {
        if (!pos_finite(B)) flag_error(err, HSGN_DEV_ERR_COERCIVE);
        const Real iB = rcp(B);
        Ys = D1 * iB;
        Vs = D2 * iB;
        Ws = D3 * iB;
    }
    const Real YsL0 = shfl_up_d(Ys, 1), VsL0 = shfl_up_d(Vs, 1), WsL0 = shfl_up_d(Ws, 1);
    if (t < teff) {
        Real YsL, VsL, WsL, YsR, VsR, WsR;
        if (t == 0) {
            YsL = Real(0);
            VsL = -Real(1);
            WsL = Real(0);
        } else {
            YsL = YsL0;
            VsL = VsL0;
            WsL = WsL0;
        }
        if (t == teff - 1) {
            YsR = Real(0);
            VsR = Real(0);
            WsR = -Real(1);
        } else {
            YsR = Ys;
            VsR = Vs;
            WsR = Ws;
        }
#pragma unroll
        for (int k = 0; k < M; ++k) {
            if (k < nint) {
                const Real Y = y[k], V = v[k], W = w[k];
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


// Eliminate a block of `nrows` rows (1 <= nrows <= T*M). All T threads of the
// CTA must call it. `row(k, i, a, b, c, d)` returns local row i = cs + k
// (0 <= i < nrows) of the calling thread's chunk. FIXED: thread t owns the
// rows [M t, M t + M) (the rows in its registers; the last chunk may be
// shorter, the threads past it none), k is a compile-time index; otherwise
// the rows are split as evenly as possible (chunk_of).
// On return thread t holds, for k < m, the triple (y, v, w) of row cs + k; the
// block separator (row nrows - 1) gets (0, 0, -1). The thread that owns the
// last row also returns its coefficients in last[0..3].
// While warp 0 solves the separator system, every other warp w calls side(w).
template <int T, int M, bool FIXED, class RowK, class Real, class Side>
__device__ __forceinline__ void cta_block_solve_impl(int nrows, RowK row, SepShared<T, Real>& sh,
                                                     Real (&y)[M], Real (&v)[M], Real (&w)[M],
                                                     int& cs, int& m, Real (&last)[4],
                                                     unsigned* err, Side side) {
    const int t = threadIdx.x;
    int teff;
    if constexpr (FIXED) {
        teff = (nrows + M - 1) / M;
        cs = t < teff ? M * t : nrows;
        m = t < teff ? min(M, nrows - M * t) : 0;
    } else {
        chunk_of<T>(nrows, t, cs, m, teff);
    }
    const int nint = m - 1;  // interior rows of the chunk (the last row is its separator)

    // ---- 1. Thomas sweep of the chunk interior with three right-hand sides:
    //         y <- d, v <- a_first e_first, w <- c_last e_last.
    //         Forward: w holds c', y holds g (rhs d), v holds gv (rhs a e_0).
    Real sa = Real(0), sb = Real(1), sc = Real(0), sd = Real(0);  // separator row of the chunk
    bool bad = false;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        if (k < nint) {
            Real a, b, c, d;
            row(k, cs + k, a, b, c, d);
            Real p, ip;
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
    if constexpr (FIXED) {
#pragma unroll
        for (int k = 0; k < M; ++k)
            if (k == m - 1) row(k, cs + k, sa, sb, sc, sd);
    } else if (m > 0) {
        row(m - 1, cs + m - 1, sa, sb, sc, sd);
    }
    // backward substitution: Y_k = g_k - c'_k Y_{k+1}, V likewise, W_k = -c'_k W_{k+1}.
    // The last interior values (YL, VL, WL) are kept in scalars; an empty
    // interior means the row before the separator is the previous separator.
    Real YL = Real(0), VL = -Real(1), WL = Real(0);
    {
        // seeds make the first executed row (k = nint-1) give Y = g, V = gv, W = c'
        Real Yn = Real(0), Vn = Real(0), Wn = -Real(1);
#pragma unroll
        for (int k = M - 1; k >= 0; --k) {
            if (k < nint) {
                const Real Y = fma(-w[k], Yn, y[k]);
                const Real V = fma(-w[k], Vn, v[k]);
                const Real W = -w[k] * Wn;
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
        sh.YF[pd(t)] = nint > 0 ? y[0] : Real(0);
        sh.VF[pd(t)] = nint > 0 ? v[0] : Real(0);
        sh.WF[pd(t)] = nint > 0 ? w[0] : -Real(1);
    }
    __syncthreads();

    // ---- 2. separator system: sigma_t for t < teff - 1 couples sigma_{t-1},
    //         sigma_t, sigma_{t+1}, with sigma_{-1} = x_L and sigma_{teff-1} = x_R.
    //         It has the form of a block (its own last row being x_R), so warp 0
    //         eliminates it with warp_block_solve: the returned triple of row t
    //         is (Ys, Vs, Ws) with sigma_t = Ys - x_L Vs - x_R Ws.
    const int ns = teff - 1;
    if (t < ns) {
        sh.A[pd(t)] = -sa * VL;
        sh.B[pd(t)] = sb - sa * WL - sc * sh.VF[pd(t + 1)];
        sh.C[pd(t)] = -sc * sh.WF[pd(t + 1)];
        sh.D1[pd(t)] = sd - sa * YL - sc * sh.YF[pd(t + 1)];
    }
    if (t == teff - 1) {
        last[0] = sa;
        last[1] = sb;
        last[2] = sc;
        last[3] = sd;
    }
    __syncthreads();
    if (t >= 32) side(t >> 5);
    if (ns > 0 && t < 32) {
        constexpr int MW = (T + 31) / 32;
        auto srow = [&](int r, Real& a, Real& b, Real& c, Real& d) {
            if (r < ns) {
                a = sh.A[pd(r)];
                b = sh.B[pd(r)];
                c = sh.C[pd(r)];
                d = sh.D1[pd(r)];
            } else {  // the external x_R: never eliminated
                a = Real(0);
                b = Real(1);
                c = Real(0);
                d = Real(0);
            }
        };
        Real ys[MW], vs[MW], ws[MW], ls[4];
        int c2, m2;
        warp_block_solve<MW>(ns + 1, srow, ys, vs, ws, c2, m2, ls, err);
#pragma unroll
        for (int k = 0; k < MW; ++k) {
            if (k < m2 && c2 + k < ns) {
                sh.YF[pd(c2 + k)] = ys[k];
                sh.VF[pd(c2 + k)] = vs[k];
                sh.WF[pd(c2 + k)] = ws[k];
            }
        }
    }
    __syncthreads();

    // ---- 3. recombination: sigma_t = Ys_t - x_L Vs_t - x_R Ws_t, with the
    //         externals sigma_{-1} = x_L -> (0, -1, 0), sigma_{teff-1} = x_R -> (0, 0, -1)
    if (t < teff) {
        Real YsL, VsL, WsL, YsR, VsR, WsR;
        if (t == 0) {
            YsL = Real(0);
            VsL = -Real(1);
            WsL = Real(0);
        } else {
            YsL = sh.YF[pd(t - 1)];
            VsL = sh.VF[pd(t - 1)];
            WsL = sh.WF[pd(t - 1)];
        }
        if (t == teff - 1) {
            YsR = Real(0);
            VsR = Real(0);
            WsR = -Real(1);
        } else {
            YsR = sh.YF[pd(t)];
            VsR = sh.VF[pd(t)];
            WsR = sh.WF[pd(t)];
        }
#pragma unroll
        for (int k = 0; k < M; ++k) {
            if (k < nint) {
                const Real Y = y[k], V = v[k], W = w[k];
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
// Depth solve of one window: nrows rows (the last one closes the window) with
// the couplings beyond the window dropped, i.e. x_L = x_R = 0 in the notation
// of hsgn_tridiag.cuh. Thread t holds the rows M t .. M t + M - 1 in its
// registers (row(k, i, a, b, c, d) gives row i = M t + k); its last row is a
// thread separator sigma_t. As in cta_block_solve_impl each thread first
// eliminates its interior rows with three right-hand sides, so that
// x_i = y_i - sigma_{t-1} v_i - sigma_t w_i. The separators then satisfy a
// tridiagonal system of teff - 1 rows (the last thread's separator is the
// closing row), which here is solved by parallel cyclic reduction over all
// threads in shared memory, one row per thread and one right-hand side (the
// window has no external couplings), instead of by one warp: log2 of the
// row count levels, each a constant number of operations per thread, so no
// warp idles while one works. On return x[k] holds the solution of row
// M t + k (zero for the closing row and for rows past nrows).
// TP < T: only the first TP threads (TP = T - 64) reduce the separators, two
// rows each, on their own barrier, while the last two warps run
// side(1) and side(2) (other work of the CTA that needs no barrier).
// ---------------------------------------------------------------------------
template <int T, int M, int TP = T, class RowK, class Real, class Side = NoSide>
__device__ __forceinline__ void cta_window_solve(int nrows, RowK row, SepShared<T, Real>& sh,
                                                 Real (&x)[M], unsigned* err,
                                                 Side side = Side()) {
    const int t = threadIdx.x;
    const int teff = (nrows + M - 1) / M;
    const int cs = t < teff ? M * t : nrows;
    const int m = t < teff ? min(M, nrows - M * t) : 0;
    const int nint = m - 1;
    Real y[M], v[M], w[M];
    // ---- 1. Thomas sweep of the chunk interior (three right-hand sides)
    Real sa = Real(0), sb = Real(1), sc = Real(0), sd = Real(0);
    bool bad = false;
#pragma unroll
    for (int k = 0; k < M; ++k) {
        if (k < nint) {
            Real a, b, c, d;
            row(k, cs + k, a, b, c, d);
            Real p, ip;
            if (k == 0) {
                p = b;
                ip = rcp(p);
                y[k] = d * ip;
                v[k] = a * ip;
            } else {
                p = fma_u(-a, w[k - 1], b);
                ip = rcp(p);
                y[k] = fma_u(-a, y[k - 1], d) * ip;
                v[k] = -a * v[k - 1] * ip;
            }
            bad |= !pos_finite(p);
            w[k] = c * ip;
        }
    }
#pragma unroll
    for (int k = 0; k < M; ++k)
        if (k == m - 1) row(k, cs + k, sa, sb, sc, sd);
    Real YL = Real(0), VL = -Real(1), WL = Real(0);
    {
        Real Yn = Real(0), Vn = Real(0), Wn = -Real(1);
#pragma unroll
        for (int k = M - 1; k >= 0; --k) {
            if (k < nint) {
                const Real Y = fma_u(-w[k], Yn, y[k]);
                const Real V = fma_u(-w[k], Vn, v[k]);
                const Real W = -w[k] * Wn;
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
    if (t < teff) {
        sh.YF[pd(t)] = nint > 0 ? y[0] : Real(0);
        sh.VF[pd(t)] = nint > 0 ? v[0] : Real(0);
        sh.WF[pd(t)] = nint > 0 ? w[0] : -Real(1);
    }
    __syncthreads();

    // ---- 2. separator rows sigma_t, t < ns = teff - 1 (sigma_{-1} = x_L and
    //         sigma_{ns} = x_R are zero, so their couplings drop)
    const int ns = teff - 1;
    Real A = Real(0), B = Real(1), C = Real(0), D = Real(0);
    if (t < ns) {
        A = t == 0 ? Real(0) : -sa * VL;
        B = sb - sa * WL - sc * sh.VF[pd(t + 1)];
        C = t == ns - 1 ? Real(0) : -sc * sh.WF[pd(t + 1)];
        D = sd - sa * YL - sc * sh.YF[pd(t + 1)];
    }
    __syncthreads();  // (the first-interior values are read above)
    // ---- 3. parallel cyclic reduction: after the level of stride s, row t
    //         couples sigma_t to sigma_{t-2s} and sigma_{t+2s} only; rows
    //         outside [0, ns) are identity rows. The couplings of a diagonally
    //         dominant system shrink geometrically with the stride: once every
    //         row's remaining couplings are below `drop` of its diagonal (they
    //         multiply separators no larger than the solution), the levels left
    //         would change no separator beyond that and are skipped.
    const float drop = sizeof(Real) == sizeof(float) ? 0x1p-26f : 0x1p-52f;
    auto coupled_row = [&](const Real& a, const Real& b, const Real& c) {
        return fabsf(hi_of(a)) + fabsf(hi_of(c)) > drop * fabsf(hi_of(b));
    };
    // row r of the level of stride s from its neighbours' rows in shared memory
    auto reduce_row = [&](int r, int s, Real& a, Real& b, Real& c, Real& d) {
        Real nA = Real(0), nC = Real(0), nB = b, nD = d;
        if (r - s >= 0) {
            const Real k1 = a * rcp(sh.B[pd(r - s)]);
            nA = -k1 * sh.A[pd(r - s)];
            nB = fma_u(-k1, sh.C[pd(r - s)], nB);
            nD = fma_u(-k1, sh.D1[pd(r - s)], nD);
        }
        if (r + s < ns) {
            const Real k2 = c * rcp(sh.B[pd(r + s)]);
            nC = -k2 * sh.C[pd(r + s)];
            nB = fma_u(-k2, sh.A[pd(r + s)], nB);
            nD = fma_u(-k2, sh.D1[pd(r + s)], nD);
        }
        a = nA;
        b = nB;
        c = nC;
        d = nD;
    };
    auto store_row = [&](int r, const Real& a, const Real& b, const Real& c, const Real& d) {
        sh.A[pd(r)] = a;
        sh.B[pd(r)] = b;
        sh.C[pd(r)] = c;
        sh.D1[pd(r)] = d;
    };
    if constexpr (TP == T) {
        for (int s = 1; s < ns; s <<= 1) {
            const bool coupled = t < ns && coupled_row(A, B, C);
            if (!__syncthreads_or(coupled)) break;
            if (t < ns) store_row(t, A, B, C, D);
            __syncthreads();
            if (t < ns) reduce_row(t, s, A, B, C, D);
            __syncthreads();
        }
        if (t < ns) {
            if (!pos_finite(B)) bad = true;
            sh.YF[pd(t)] = D * rcp(B);
        }
    } else {
        static_assert(TP == T - 64 && TP % 32 == 0 && 2 * TP >= T, "the group leaves two warps");
        // the rows of the last two warps go to the group: thread t < TP takes
        // rows t and t + TP
        if (t >= TP && t < ns) store_row(t, A, B, C, D);
        __syncthreads();
        if (t < TP) {
            const int t2 = t + TP;
            Real A2 = Real(0), B2 = Real(1), C2 = Real(0), D2 = Real(0);
            if (t2 < ns) {
                A2 = sh.A[pd(t2)];
                B2 = sh.B[pd(t2)];
                C2 = sh.C[pd(t2)];
                D2 = sh.D1[pd(t2)];
            }
            for (int s = 1; s < ns; s <<= 1) {
                const bool coupled =
                    (t < ns && coupled_row(A, B, C)) || (t2 < ns && coupled_row(A2, B2, C2));
                if (!group_or(1, TP, coupled)) break;
                if (t < ns) store_row(t, A, B, C, D);
                if (t2 < ns) store_row(t2, A2, B2, C2, D2);
                group_sync(1, TP);
                if (t < ns) reduce_row(t, s, A, B, C, D);
                if (t2 < ns) reduce_row(t2, s, A2, B2, C2, D2);
                group_sync(1, TP);
            }
            if (t < ns) {
                if (!pos_finite(B)) bad = true;
                sh.YF[pd(t)] = D * rcp(B);
            }
            if (t2 < ns) {
                if (!pos_finite(B2)) bad = true;
                sh.YF[pd(t2)] = D2 * rcp(B2);
            }
        } else {
            side(t / 32 - TP / 32 + 1);
        }
    }
    if (bad) flag_error(err, HSGN_DEV_ERR_COERCIVE);
    __syncthreads();

    // ---- 4. recombination: x_i = y_i - sigma_{t-1} v_i - sigma_t w_i
    const Real sL = (t > 0 && t - 1 < ns) ? sh.YF[pd(t - 1)] : Real(0);
    const Real sR = t < ns ? sh.YF[pd(t)] : Real(0);
#pragma unroll
    for (int k = 0; k < M; ++k) {
        if (k < nint)
            x[k] = y[k] - sL * v[k] - sR * w[k];
        else if (k == nint)
            x[k] = sR;
        else
            x[k] = Real(0);
    }
}

// cta_block_solve_impl with rows split evenly; row(i, a, b, c, d) returns row i.
template <int T, int M, class RowFn, class Real, class Side = NoSide>
__device__ __forceinline__ void cta_block_solve(int nrows, RowFn row, SepShared<T, Real>& sh,
                                                Real (&y)[M], Real (&v)[M], Real (&w)[M],
                                                int& cs, int& m, Real (&last)[4],
                                                unsigned* err, Side side = Side()) {
    cta_block_solve_impl<T, M, false>(
        nrows, [&](int, int i, Real& a, Real& b, Real& c, Real& d) { row(i, a, b, c, d); }, sh, y,
        v, w, cs, m, last, err, side);
}

// cta_block_solve_impl with M rows per thread held in its registers:
// row(k, i, a, b, c, d) returns the k-th row of the thread (row i = M t + k).
template <int T, int M, class RowK, class Real, class Side = NoSide>
__device__ __forceinline__ void cta_block_solve_fixed(int nrows, RowK row, SepShared<T, Real>& sh,
                                                      Real (&y)[M], Real (&v)[M], Real (&w)[M],
                                                      int& cs, int& m, Real (&last)[4],
                                                      unsigned* err, Side side = Side()) {
    cta_block_solve_impl<T, M, true>(nrows, row, sh, y, v, w, cs, m, last, err, side);
}

}  // namespace hsgn
