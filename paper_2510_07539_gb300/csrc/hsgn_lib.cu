// hsgn_lib.cu -- host runtime and C ABI of the hSGN semi-implicit IMEX library.
//
// Declarations, argument meaning, ownership and error behaviour: include/hsgn.h.
// Paper: Macca, Boscheri, Ricchiuto, arXiv 2510.07539 (Sec. 3.2 time stepping,
// Sec. 4.2 fully-discrete stage, Sec. 5 time-step rule).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/hsgn.h"
#include "hsgn_kernels.cuh"
#include "hsgn_fused.cuh"
#include "hsgn_adjoint.cuh"
#include "hsgn_dfstage.cuh"

using namespace hsgn;

namespace {

// Stage block: AT threads per CTA, AM rows per thread in the block elimination
// (FP64 path); the mixed path uses more threads with shorter chunks.
constexpr int AT = 64, AM = 8, AS = AT * AM;
constexpr int XT = 128, XM = 4;
static_assert(XT * XM == AS, "both precision forms use the same block split");
// One CTA solves single-precision separator systems of up to OT*OM rows.
constexpr int OT = 256, OM = 16;
// Windowed mixed stage: FT threads, FM rows per thread, FHW overlap rows.
constexpr int FT = 256, FM = 4, FHW = 64;
// Double-float windowed stage: DT threads, FM rows per thread, DHW overlap rows
// (wider than the mixed stage's: the truncation bound is 2^-50, not 2^-30, and
// 95 rows keep it up to CFL_IMEX of about 7 for smooth states). The overlap a
// step takes follows the coupling: stage 2 records the rows its windows
// needed, and every synchronising call sets the overlap of the next steps to
// that need plus DF_MARGIN rows, rounded up to a multiple of 8 within
// [DHW_MIN, DHW] (DHW_START while nothing is recorded); a tile whose window
// misses the bound all the same is redone with DHW rows (k_df_stage).
constexpr int DT = 256, DHW = 96, DHW_MIN = 48, DHW_START = 64, DF_MARGIN = 4;

// Overlap rows of the double-float windows for a recorded need (0: none).
int df_overlap_for(unsigned need) {
    if (need == 0) return DHW_START;
    const unsigned want = need + DF_MARGIN + 1;
    const int hw = (int)((want + 7) / 8 * 8);
    return hw < DHW_MIN ? DHW_MIN : (hw > DHW ? DHW : hw);
}
// Variants of the windowed stage for batches, chosen per instance by
// hsgn_batched_set_tiles / hsgn_batched_autotune: v = 0 and 1 take FT = 256 and
// FTS = 128 threads (tiles of up to 894 / 382 rows) with the FHW-row overlap,
// v = 2 and 3 the same thread counts with a narrow FHWN-row overlap (tiles of
// up to 958 / 446 rows), which meets the 2^-30 truncation bound where the
// depth coupling decays fast (small CFL numbers) and reports
// HSGN_ERR_TRUNCATION elsewhere.
constexpr int FTS = 128, FHWN = 32, kBV = 4;
// Separator levels: one warp per block of GS rows; one warp solves up to RMAX rows.
constexpr int GS = SEP_ROWS, RMAX = SEP_ROWS;

constexpr size_t kAlign = 256;

// Tile rows of the windowed path: as few tiles of at most smax rows as
// possible, evened out so that a grid larger than one wave of `slots`
// resident CTAs ends in full waves.
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Rows per block of a single grid's FP64 / exact mixed stage for `slots`
// co-resident CTAs: as many rows as one wave needs, within [64, AS].
int64_t stage_block_rows(int64_t n, int64_t slots) {
    const int64_t r = (n + slots - 1) / slots;
    return r < 64 ? 64 : (r > AS ? AS : r);
}

BlockSplit make_split(int64_t n, int64_t rows_per_block) {
    BlockSplit s;
    s.n = n;
    s.P = (int32_t)((n + rows_per_block - 1) / rows_per_block);
    s.base = n / s.P;
    s.rem = (int32_t)(n % s.P);
    return s;
}

// Workspace (in bytes, excluding the error word) of the recursive solve of n
// rows: per level the row triples (3n), the block summaries and separators.
constexpr size_t rows_ws_bytes(int64_t n) {
    if (n <= RMAX) return 0;
    const int64_t P = (n + GS - 1) / GS;  // blocks of the even split
    return align_up(3 * n * sizeof(double)) + align_up(BLK_STRIDE * P * sizeof(double)) +
           align_up(P * sizeof(double)) + rows_ws_bytes(P);
}

template <class K>
cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Recursive cyclic solve of n rows given by a row source, with workspace `ws`:
// at most RMAX rows in one warp, otherwise one level of block elimination
// (a warp per GS rows), the cyclic system of the block separators, and the
// back-out of every row. Works in the row source's precision.
template <class RowSrc>
cudaError_t solve_src(int64_t n, RowSrc rows, typename RowSrc::Real* x, unsigned char* ws,
                      unsigned* err, double* speed_reset, cudaStream_t st) {
    using Real = typename RowSrc::Real;
    if (n <= RMAX) {
        k_cyclic_onewarp<RowSrc><<<1, 32, 0, st>>>((int)n, rows, x, speed_reset, err);
        return cudaGetLastError();
    }
    if constexpr (sizeof(Real) == sizeof(float)) {
        if (n <= OT * OM) {
            k_cyclic_onecta<OT, OM, RowSrc><<<1, OT, 0, st>>>((int)n, rows, x, speed_reset, err);
            return cudaGetLastError();
        }
    }
    const BlockSplit s = make_split(n, GS);
    const int64_t P = s.P;
    Real* y = reinterpret_cast<Real*>(ws);
    ws += align_up(3 * n * sizeof(double));
    Real* blk = reinterpret_cast<Real*>(ws);
    ws += align_up(BLK_STRIDE * P * sizeof(double));
    Real* sv = reinterpret_cast<Real*>(ws);
    ws += align_up(P * sizeof(double));
    k_block_reduce<RowSrc><<<(unsigned)P, 32, 0, st>>>(rows, s, y, y + n, y + 2 * n, blk, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = solve_src(P, BlkRowsT<Real>{blk, P}, sv, ws, err, speed_reset, st);
    if (e != cudaSuccess) return e;
    k_block_backout<Real><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s, y, y + n, y + 2 * n, sv, x);
    return cudaGetLastError();
}

cudaError_t solve_rows(int64_t n, int periodic, const double* a, const double* b, const double* c,
                       const double* d, double* x, unsigned char* ws, unsigned* err,
                       double* speed_reset, cudaStream_t st) {
    return solve_src(n, ArrayRows{a, b, c, d, periodic, n}, x, ws, err, speed_reset, st);
}

int map_error_bits(unsigned bits) {
    // the root cause first: a bad depth or coefficient produces the non-finite values
    if (bits & HSGN_DEV_ERR_DEPTH) return HSGN_ERR_NONPOSITIVE_DEPTH;
    if (bits & HSGN_DEV_ERR_COERCIVE) return HSGN_ERR_NOT_COERCIVE;
    if (bits & HSGN_DEV_ERR_NONFINITE) return HSGN_ERR_NONFINITE;
    if (bits & HSGN_DEV_ERR_TRUNCATION) return HSGN_ERR_TRUNCATION;
    return HSGN_OK;
}

__global__ void k_set_scalar(double* p, double v) { *p = v; }

}  // namespace

struct hsgn_s {
    int64_t n = 0;
    int32_t bc = 0, flags = 0;
    double dx = 0, g = 0, lam = 0;
    int device = 0;
    BlockSplit split{};
    unsigned char* mem = nullptr;  // one allocation for state and workspace
    double* U[4] = {};
    double* U1[4] = {};
    double *y = nullptr, *v = nullptr, *w = nullptr;
    double *qs = nullptr, *ms = nullptr, *rs = nullptr, *be = nullptr, *de = nullptr;
    double* blk = nullptr;
    double* s = nullptr;
    // time-stepping scheme (HSGN_SCHEME_*) and its extra state buffers
    int32_t scheme = HSGN_SCHEME_PRINTED;
    double* E2[4] = {};              // ARS(2,2,2): U^n + gamma dt L(U^n)
    double* Wd[4] = {};              // ARS(2,2,2): U^n + delta dt L(U^n)
    // well-balanced bathymetry form (HSGN_WELL_BALANCED)
    bool wb = false;
    double* bathy = nullptr;         // bottom per cell, null for a flat bottom
    float2* bathy_df = nullptr;      // the bottom as double-float pairs (windowed bottom form)
    double* phi = nullptr;           // face forces Phi_{i+1/2}
    unsigned char* rws = nullptr;    // workspace of the separator-system solve
    double* spd = nullptr;           // [0] global Rusanov speed, [1] stage speed, [2..3] scratch,
                                     // [4] global Rusanov speed while the state is in V
    // windowed mixed stage (HSGN_MIXED without HSGN_EXACT_SOLVE): one launch per
    // stage; U^{n+1} goes to the other of the two state buffers U, V
    bool windowed = false;
    int32_t tileS = 0;               // tile rows per CTA
    int32_t dfhw = 0;                // double-float: window overlap of the next steps (tileS follows it)
    int32_t ghw[2] = {};             // double-float: the overlap each captured step graph holds
    unsigned* dfneed = nullptr;      // double-float: overlap rows the coupling needed, per state buffer
    int32_t tileSlots = 0;           // co-resident CTAs of the windowed kernel
    int32_t vslots[4] = {};          // co-resident CTAs of each batch variant
    double* V[4] = {};
    int cur = 0;                     // 1: the state is in V
    // mixed precision (HSGN_MIXED): FP32 stage-1 increments and per-row results
    bool mixed = false;
    float *G1 = nullptr, *dq1 = nullptr, *dm1 = nullptr, *dr1 = nullptr;
    float4* mrec = nullptr;          // three float4 records per row
    // double-float windowed stage (HSGN_DOUBLE_FLOAT): stage-1 increments as pairs
    bool dfloat = false;
    bool df_f32 = false;             // with HSGN_MIXED: fluxes and coefficients in FP32
    float2* D1[4] = {};
    // batch (hsgn_create_batched)
    int32_t count = 1;
    bool batched = false;
    int64_t total_blocks = 0;
    InstInfo* inst = nullptr;        // device table
    int32_t* blk_inst = nullptr;     // device table
    double* speeds = nullptr;        // per-instance Rusanov speed (device)
    double* speeds_tmp = nullptr;    // 2 per instance (device), for suggest_dt
    double* speeds_next = nullptr;   // windowed batch: per-instance speed while the state is in V
    int32_t* tile_inst = nullptr;    // windowed batch: instance of every large tile (device)
    int64_t total_tiles = 0;
    int32_t* vtile[4] = {};          // windowed batch: instance of every tile of each
    int64_t vtiles[4] = {};          //   batch variant (vtile[0] is tile_inst), tile counts
    std::vector<int8_t> variant;     // per instance: its batch variant, 0 .. 3
    std::vector<InstInfo> inst_h;    // host copy
    float *mblk = nullptr, *ms_ = nullptr;
    unsigned* err = nullptr;
    cudaStream_t cap = nullptr;      // private stream used for graph capture
    cudaGraphExec_t gexec[2] = {};   // one step, per state buffer
    double gdt[2] = {};
    cudaGraphExec_t gcfl[2] = {};    // one step with the device-side CFL time step
    double gcfl_rule[2][2] = {};     // its (cfl, mcfl)
    int32_t gcfl_hw[2] = {};         // its double-float window overlap
    // event-pair profiler (hsgn_profile)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    double prof_ms[HSGN_PROF_KINDS] = {};
    int64_t prof_n[HSGN_PROF_KINDS] = {};
};

namespace {

bool local_speed(const hsgn_s* H) { return (H->flags & HSGN_RUSANOV_LOCAL) != 0; }
// Explicit Heun / Euler: every wave explicit, Rusanov speed max(|u| + c)
bool explicit_scheme(const hsgn_s* H) {
    return H->scheme == HSGN_SCHEME_EX_HEUN || H->scheme == HSGN_SCHEME_EX_EULER;
}

// The buffer holding the current state, and the global Rusanov speed of the
// state in buffer `which` (0: U, 1: V).
double* const* state(const hsgn_s* H) { return H->cur ? H->V : H->U; }
double* speed_of(const hsgn_s* H, int which) {
    if (H->batched) return which ? H->speeds_next : H->speeds;  // per instance
    return H->spd + (which ? 4 : 0);
}

cudaEvent_t take_event(hsgn_s* H) {
    if (!H->ev_pool.empty()) {
        cudaEvent_t e = H->ev_pool.back();
        H->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Records an event pair around one kernel launch when profiling is on.
struct ProfScope {
    hsgn_s* H;
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    ProfScope(hsgn_s* h, int k, cudaStream_t s) : H(h), kind(k), st(s) {
        if (H->prof) {
            a = take_event(H);
            cudaEventRecord(a, st);
        }
    }
    ~ProfScope() {
        if (a) {
            cudaEvent_t b = take_event(H);
            cudaEventRecord(b, st);
            H->recs.push_back({kind, a, b});
        }
    }
};

cudaError_t launch_stage(hsgn_s* H, const double* const A[4], const double* const B[4], double wl0,
                         double wl1, double wb0, double wb1, double tau, const double* speed_ptr,
                         double* const out[4], bool reset_and_track, cudaStream_t st,
                         const double* const C[4] = nullptr, double wl2 = 0.0) {
    StageParams p;
    for (int k = 0; k < 4; ++k) p.C[k] = C ? C[k] : nullptr;
    p.wl2 = wl2;
    p.recon = H->scheme == HSGN_SCHEME_SI1 ? 0 : 1;
    p.n = H->n;
    p.bc = H->bc;
    p.local_speed = local_speed(H) ? 1 : 0;
    p.dx = H->dx;
    p.g = H->g;
    p.lam = H->lam;
    p.tau = tau;
    for (int k = 0; k < 4; ++k) {
        p.A[k] = A[k];
        p.B[k] = B ? B[k] : nullptr;
    }
    p.wl0 = wl0;
    p.wl1 = wl1;
    p.wb0 = wb0;
    p.wb1 = wb1;
    p.speed = speed_ptr;
    p.split = H->split;
    p.y = H->y;
    p.v = H->v;
    p.w = H->w;
    p.qs = H->qs;
    p.ms = H->ms;
    p.rs = H->rs;
    p.be = H->be;
    p.de = H->de;
    p.blk = H->blk;
    p.err = H->err;
    p.bathy = H->bathy;
    p.phi = H->phi;
    const unsigned P = (unsigned)H->split.P;
    {
        ProfScope ps(H, HSGN_PROF_ASSEMBLE, st);
        if (H->wb) {
            const size_t smem = sizeof(AssembleShared<AT, AM, true>);
            if (H->bc == BC_PERIODIC)
                k_stage_assemble<AT, AM, BC_PERIODIC, true><<<P, AT, smem, st>>>(p);
            else
                k_stage_assemble<AT, AM, BC_TRANSMISSIVE, true><<<P, AT, smem, st>>>(p);
        } else {
            const size_t smem = sizeof(AssembleShared<AT, AM>);
            if (H->bc == BC_PERIODIC)
                k_stage_assemble<AT, AM, BC_PERIODIC, false><<<P, AT, smem, st>>>(p);
            else
                k_stage_assemble<AT, AM, BC_TRANSMISSIVE, false><<<P, AT, smem, st>>>(p);
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;

    const bool track = reset_and_track && !local_speed(H);
    double* reset = track ? H->spd : nullptr;
    {
        ProfScope ps(H, HSGN_PROF_REDUCED, st);
        e = solve_src(P, BlkRows{H->blk, (int64_t)P}, H->s, H->rws, H->err, reset, st);
    }
    if (e != cudaSuccess) return e;

    BacksubParams q;
    q.n = H->n;
    q.bc = H->bc;
    q.track_speed = track ? 1 : 0;
    q.dx = H->dx;
    q.lam = H->lam;
    q.tau = tau;
    q.split = H->split;
    q.y = H->y;
    q.v = H->v;
    q.w = H->w;
    q.s = H->s;
    q.qs = H->qs;
    q.ms = H->ms;
    q.rs = H->rs;
    q.be = H->be;
    q.de = H->de;
    q.phi = H->phi;
    for (int k = 0; k < 4; ++k) q.out[k] = out[k];
    q.speed = H->spd;
    q.err = H->err;
    const unsigned nb = (unsigned)((H->n + 255) / 256);
    {
        ProfScope ps(H, HSGN_PROF_BACKSUB, st);
        if (H->wb) {
            if (H->bc == BC_PERIODIC)
                k_backsub<BC_PERIODIC, true><<<nb, 256, 0, st>>>(q);
            else
                k_backsub<BC_TRANSMISSIVE, true><<<nb, 256, 0, st>>>(q);
        } else {
            if (H->bc == BC_PERIODIC)
                k_backsub<BC_PERIODIC, false><<<nb, 256, 0, st>>>(q);
            else
                k_backsub<BC_TRANSMISSIVE, false><<<nb, 256, 0, st>>>(q);
        }
    }
    return cudaGetLastError();
}

// One stage in mixed precision (hsgn_mixed.cuh). Stage 1 writes the FP32
// increments dU1 = U_I^(1) - U^n; stage 2 reads them (U_l = U^n + (c/gamma) dU1,
// U_b = U^n + ((1-gamma)/gamma) dU1) and writes U^{n+1} in place.
cudaError_t launch_stage_mixed(hsgn_s* H, int stage, double tau, cudaStream_t st) {
    const double gam = 1.0 - 1.0 / std::sqrt(2.0);
    const double c = 1.0 / (2.0 * gam);
    MixedParams p;
    p.n = H->n;
    p.bc = H->bc;
    p.local_speed = local_speed(H) ? 1 : 0;
    p.stage = stage;
    const bool track = stage == 2 && !local_speed(H);
    p.track_speed = track ? 1 : 0;
    const double dx = H->dx, lam = H->lam;
    p.g = (float)H->g;
    p.lam = (float)lam;
    p.tau = (float)tau;
    p.tdx = (float)(tau / dx);
    p.fq = (float)(tau / (2.0 * dx));
    p.Cc = (float)(tau * tau / (dx * dx));
    p.fd = (float)(lam * tau * tau / (dx * dx));
    p.lt2 = (float)(lam * tau * tau);
    p.ltau = (float)(lam * tau);
    p.wl1 = stage == 2 ? (float)(c / gam) : 0.f;
    p.wb1 = stage == 2 ? (float)((1.0 - gam) / gam) : 0.f;
    for (int k = 0; k < 4; ++k) {
        p.U[k] = H->U[k];
        p.out[k] = H->U[k];
    }
    p.G1 = H->G1;
    p.dq1 = H->dq1;
    p.dm1 = H->dm1;
    p.dr1 = H->dr1;
    p.speed = H->spd;
    p.split = H->split;
    p.rec = H->mrec;
    p.blk = H->mblk;
    p.s = H->ms_;
    p.err = H->err;
    p.batched = H->batched ? 1 : 0;
    p.inst = H->inst;
    p.blk_inst = H->blk_inst;
    p.speeds = H->speeds;
    const unsigned P = (unsigned)(H->batched ? H->total_blocks : H->split.P);
    const size_t smem = sizeof(MixedShared<XT, XM>);
    {
        ProfScope ps(H, HSGN_PROF_ASSEMBLE, st);
        if (H->bc == BC_PERIODIC)
            k_mixed_assemble<XT, XM, BC_PERIODIC><<<P, XT, smem, st>>>(p);
        else
            k_mixed_assemble<XT, XM, BC_TRANSMISSIVE><<<P, XT, smem, st>>>(p);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    {
        ProfScope ps(H, HSGN_PROF_REDUCED, st);
        if (H->batched) {
            k_sep_batched<<<(unsigned)H->count, 32, 0, st>>>(p, track ? 1 : 0);
            e = cudaGetLastError();
        } else {
            e = solve_src(P, BlkRowsT<float>{H->mblk, (int64_t)P}, H->ms_, H->rws, H->err,
                          track ? H->spd : nullptr, st);
        }
    }
    if (e != cudaSuccess) return e;
    {
        ProfScope ps(H, HSGN_PROF_BACKSUB, st);
        if (H->bc == BC_PERIODIC)
            k_mixed_backsub<BC_PERIODIC><<<P, 256, 0, st>>>(p);
        else
            k_mixed_backsub<BC_TRANSMISSIVE><<<P, 256, 0, st>>>(p);
    }
    return cudaGetLastError();
}

// One launch of the windowed stage kernel specialised for p.stage.
template <int T, int BC, bool WB, int HW = FHW>
void launch_fused(unsigned P, const FusedParams& p, cudaStream_t st) {
    const size_t smem = sizeof(FusedShared<T, FM, HW, WB>);
    if (p.stage == 2)
        k_mixed_fused<T, FM, HW, BC, WB, 2><<<P, T, smem, st>>>(p);
    else
        k_mixed_fused<T, FM, HW, BC, WB, 1><<<P, T, smem, st>>>(p);
}

// Dynamic shared-memory limit of both stage kernels of one variant.
template <int T, int BC, bool WB, int HW = FHW>
cudaError_t set_smem_fused() {
    const size_t smem = sizeof(FusedShared<T, FM, HW, WB>);
    cudaError_t e = set_smem(k_mixed_fused<T, FM, HW, BC, WB, 1>, smem);
    if (e == cudaSuccess) e = set_smem(k_mixed_fused<T, FM, HW, BC, WB, 2>, smem);
    return e;
}

// Batch variant v (flat bottom): launch, largest tile, co-resident CTAs per SM.
template <int BC>
void launch_batch_variant(int v, unsigned P, const FusedParams& p, cudaStream_t st) {
    switch (v) {
        case 0: launch_fused<FT, BC, false, FHW>(P, p, st); break;
        case 1: launch_fused<FTS, BC, false, FHW>(P, p, st); break;
        case 2: launch_fused<FT, BC, false, FHWN>(P, p, st); break;
        default: launch_fused<FTS, BC, false, FHWN>(P, p, st); break;
    }
}

int64_t batch_variant_smax(int v) {
    switch (v) {
        case 0: return FusedGeom<FT, FM, FHW>::S;
        case 1: return FusedGeom<FTS, FM, FHW>::S;
        case 2: return FusedGeom<FT, FM, FHWN>::S;
        default: return FusedGeom<FTS, FM, FHWN>::S;
    }
}

template <int T, int HW>
cudaError_t batch_variant_slots(int sms, int32_t& slots) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, k_mixed_fused<T, FM, HW, BC_PERIODIC, false, 2>, T, sizeof(FusedShared<T, FM, HW>));
    slots = sms * (per_sm > 0 ? per_sm : 1);
    return e;
}

// One stage of the windowed mixed path (hsgn_fused.cuh): one launch. Stage 1
// writes the FP32 increments, stage 2 writes U^{n+1} into the other buffer.
cudaError_t launch_stage_fused(hsgn_s* H, int stage, double tau, cudaStream_t st) {
    const double gam = 1.0 - 1.0 / std::sqrt(2.0);
    const double c = 1.0 / (2.0 * gam);
    FusedParams p;
    p.n = H->n;
    p.stage = stage;
    p.local_speed = local_speed(H) ? 1 : 0;
    p.track_speed = local_speed(H) ? 0 : 1;
    p.S = H->tileS;
    p.slots = H->tileSlots;
    const double dx = H->dx, lam = H->lam;
    p.g = (float)H->g;
    p.lam = (float)lam;
    p.tau = (float)tau;
    p.tdx = (float)(tau / dx);
    p.fq = (float)(tau / (2.0 * dx));
    p.Cc = (float)(tau * tau / (dx * dx));
    p.fd = (float)(lam * tau * tau / (dx * dx));
    p.lt2 = (float)(lam * tau * tau);
    p.ltau = (float)(lam * tau);
    p.wl1 = stage == 2 ? (float)(c / gam) : 0.f;
    p.wb1 = stage == 2 ? (float)((1.0 - gam) / gam) : 0.f;
    double* const* Uc = state(H);
    double* const* Un = H->cur ? H->U : H->V;
    for (int k = 0; k < 4; ++k) {
        p.U[k] = reinterpret_cast<const float2*>(Uc[k]);
        p.out[k] = stage == 2 ? reinterpret_cast<float2*>(Un[k]) : nullptr;
    }
    p.G1 = H->G1;
    p.dq1 = H->dq1;
    p.dm1 = H->dm1;
    p.dr1 = H->dr1;
    p.speed = speed_of(H, H->cur);
    p.speed_next = speed_of(H, 1 - H->cur);
    p.err = H->err;
    p.batched = H->batched ? 1 : 0;
    p.inst = H->inst;
    p.tile_inst = H->tile_inst;
    p.bathy = H->bathy_df;
    const unsigned P = (unsigned)((H->n + H->tileS - 1) / H->tileS);
    {
        ProfScope ps(H, HSGN_PROF_ASSEMBLE, st);
        if (H->batched) {
            // one launch per variant in use, each over its own tile table
            for (int v = 0; v < kBV; ++v) {
                if (H->vtiles[v] == 0) continue;
                FusedParams pv = p;
                pv.tile_inst = H->vtile[v];
                pv.slots = H->vslots[v];
                if (H->bc == BC_PERIODIC)
                    launch_batch_variant<BC_PERIODIC>(v, (unsigned)H->vtiles[v], pv, st);
                else
                    launch_batch_variant<BC_TRANSMISSIVE>(v, (unsigned)H->vtiles[v], pv, st);
            }
        } else if (H->wb) {
            if (H->bc == BC_PERIODIC)
                launch_fused<FT, BC_PERIODIC, true>(P, p, st);
            else
                launch_fused<FT, BC_TRANSMISSIVE, true>(P, p, st);
        } else {
            if (H->bc == BC_PERIODIC)
                launch_fused<FT, BC_PERIODIC, false>(P, p, st);
            else
                launch_fused<FT, BC_TRANSMISSIVE, false>(P, p, st);
        }
    }
    return cudaGetLastError();
}

// One launch of the double-float stage kernel specialised for p.stage.
template <int BC, bool F32, bool WB>
void launch_df(unsigned P, const DfParams& p, cudaStream_t st) {
    const size_t smem = sizeof(DfShared<DT, FM, DHW, WB>);
    if (p.stage == 2)
        k_df_stage<DT, FM, DHW, BC, 2, F32, WB><<<P, DT, smem, st>>>(p);
    else
        k_df_stage<DT, FM, DHW, BC, 1, F32, WB><<<P, DT, smem, st>>>(p);
}

// the kernel of the handle's boundary condition, precision split and bottom form
void launch_df(const hsgn_s* H, unsigned P, const DfParams& p, cudaStream_t st) {
    if (H->bc == BC_PERIODIC) {
        if (H->wb) launch_df<BC_PERIODIC, false, true>(P, p, st);
        else if (H->df_f32) launch_df<BC_PERIODIC, true, false>(P, p, st);
        else launch_df<BC_PERIODIC, false, false>(P, p, st);
    } else {
        if (H->wb) launch_df<BC_TRANSMISSIVE, false, true>(P, p, st);
        else if (H->df_f32) launch_df<BC_TRANSMISSIVE, true, false>(P, p, st);
        else launch_df<BC_TRANSMISSIVE, false, false>(P, p, st);
    }
}

template <int BC>
cudaError_t set_smem_df() {
    const size_t smem = sizeof(DfShared<DT, FM, DHW>);
    const size_t smem_wb = sizeof(DfShared<DT, FM, DHW, true>);
    cudaError_t e = set_smem(k_df_stage<DT, FM, DHW, BC, 1, false>, smem);
    if (e == cudaSuccess) e = set_smem(k_df_stage<DT, FM, DHW, BC, 2, false>, smem);
    if (e == cudaSuccess) e = set_smem(k_df_stage<DT, FM, DHW, BC, 1, true>, smem);
    if (e == cudaSuccess) e = set_smem(k_df_stage<DT, FM, DHW, BC, 2, true>, smem);
    if (e == cudaSuccess) e = set_smem(k_df_stage<DT, FM, DHW, BC, 1, false, true>, smem_wb);
    if (e == cudaSuccess) e = set_smem(k_df_stage<DT, FM, DHW, BC, 2, false, true>, smem_wb);
    return e;
}

// The window overlap of the next double-float steps and its tile rows.
void set_df_overlap(hsgn_s* H, int hw) {
    H->dfhw = hw;
    H->tileS = (int32_t)fused_tile_rows(H->n, DfGeom<DT, FM, DHW>::R - 2 * hw,
                                        H->tileSlots > 0 ? H->tileSlots : 1);
}

// Constants of a double-float stage of step tau; stage 2 gets the efficient-form
// weights (wl1, wb1) unless given.
DfParams df_params(const hsgn_s* H, int stage, double tau, double wl1, double wb1) {
    DfParams p;
    p.n = H->n;
    p.stage = stage;
    p.local_speed = local_speed(H) ? 1 : 0;
    p.track_speed = local_speed(H) ? 0 : 1;
    p.S = H->tileS;
    p.HWt = H->dfhw;
    p.slots = H->tileSlots;
    p.need_out = nullptr;
    const double dx = H->dx, lam = H->lam;
    p.tau = dfl_of(tau);
    p.lt2 = dfl_of(lam * tau * tau);
    p.ltau = dfl_of(lam * tau);
    p.fq = dfl_of(tau / (2.0 * dx));
    p.lfq = dfl_of(lam * tau / (2.0 * dx));
    p.Cc = dfl_of(tau * tau / (dx * dx));
    p.fd = dfl_of(lam * tau * tau / (dx * dx));
    p.g = dfl_of(H->g);
    p.lam = dfl_of(lam);
    p.lam3 = dfl_of(lam / 3.0);
    p.third = dfl_of(1.0 / 3.0);
    p.wl1 = dfl_of(wl1);
    p.wb1 = dfl_of(wb1);
    p.bathy = H->bathy_df;
    p.wmd = dfl_of(wb1 - wl1);
    p.adaptive = 0;
    p.cfl = p.mcfl = 0.0;
    p.dx = dx;
    p.lam_d = lam;
    p.g_d = H->g;
    p.dtp = H->spd + 6;
    for (int k = 0; k < 4; ++k) {
        p.U[k] = nullptr;
        p.D1[k] = H->D1[k];
        p.out[k] = nullptr;
    }
    p.speed = nullptr;
    p.speed_next = nullptr;
    p.err = H->err;
    return p;
}

unsigned df_tiles(const hsgn_s* H) { return (unsigned)((H->n + H->tileS - 1) / H->tileS); }

// One stage of the double-float path (hsgn_dfstage.cuh): one launch. Stage 1
// writes the increments dU1, stage 2 writes U^{n+1} into the other buffer.
// cfl > 0: the step's dt from the CFL rule of the current state, on the
// device (DfParams::adaptive); tau is then unused.
cudaError_t launch_stage_df(hsgn_s* H, int stage, double tau, cudaStream_t st, double cfl = 0.0,
                            double mcfl = 0.0) {
    const double gam = 1.0 - 1.0 / std::sqrt(2.0);
    const double c = 1.0 / (2.0 * gam);
    DfParams p = df_params(H, stage, tau, stage == 2 ? c / gam : 0.0,
                           stage == 2 ? (1.0 - gam) / gam : 0.0);
    if (cfl > 0.0) {
        p.adaptive = 1;
        p.cfl = cfl;
        p.mcfl = mcfl;
    }
    double* const* Uc = state(H);
    double* const* Un = H->cur ? H->U : H->V;
    for (int k = 0; k < 4; ++k) {
        p.U[k] = reinterpret_cast<const float2*>(Uc[k]);
        p.out[k] = stage == 2 ? reinterpret_cast<float2*>(Un[k]) : nullptr;
    }
    p.speed = speed_of(H, H->cur);
    p.speed_next = speed_of(H, 1 - H->cur);
    // stage 2 records the coupling of the state it writes (read at the next
    // synchronising call, which sets the overlap of the steps after it)
    p.need_out = H->dfneed + (1 - H->cur);
    {
        ProfScope ps(H, HSGN_PROF_ASSEMBLE, st);
        launch_df(H, df_tiles(H), p, st);
    }
    return cudaGetLastError();
}

// Explicit operator (k_explicit): out1 = a1 U0 + b1 Us + c1 L(Us), optional out2.
cudaError_t launch_explicit(hsgn_s* H, const double* const Us[4], const double* const U0[4],
                            double a1, double b1, double c1, double* const out1[4],
                            double a2, double b2, double c2, double* const out2[4],
                            bool track, cudaStream_t st) {
    ExplicitParams p;
    p.n = H->n;
    p.recon = H->scheme == HSGN_SCHEME_EX_EULER ? 0 : 1;
    p.local_speed = local_speed(H) ? 1 : 0;
    p.track_speed = track && !local_speed(H) ? 1 : 0;
    p.spectral = explicit_scheme(H) ? 1 : 0;
    p.dx = H->dx;
    p.g = H->g;
    p.lam = H->lam;
    p.idx = 1.0 / H->dx;
    p.i2dx = 0.5 / H->dx;
    for (int k = 0; k < 4; ++k) {
        p.Us[k] = Us[k];
        p.U0[k] = U0 ? U0[k] : nullptr;
        p.out1[k] = out1[k];
        p.out2[k] = out2 ? out2[k] : nullptr;
    }
    p.a1 = a1; p.b1 = b1; p.c1 = c1;
    p.a2 = a2; p.b2 = b2; p.c2 = c2;
    p.speed = H->spd;
    p.speed_next = H->spd + 4;
    p.err = H->err;
    const unsigned nb = (unsigned)((H->n + 255) / 256);
    ProfScope ps(H, HSGN_PROF_ASSEMBLE, st);
    if (H->bc == BC_PERIODIC)
        k_explicit<BC_PERIODIC><<<nb, 256, 0, st>>>(p);
    else
        k_explicit<BC_TRANSMISSIVE><<<nb, 256, 0, st>>>(p);
    return cudaGetLastError();
}

// The comparison schemes of the FP64 form (HSGN_SCHEME_*, see hsgn.h).
cudaError_t enqueue_step_scheme(hsgn_s* H, double dt, cudaStream_t st) {
    const double gam = 1.0 - 1.0 / std::sqrt(2.0);
    const double del = 1.0 - 1.0 / (2.0 * gam);
    const double* U[4] = {H->U[0], H->U[1], H->U[2], H->U[3]};
    const double* U1c[4] = {H->U1[0], H->U1[1], H->U1[2], H->U1[3]};
    cudaError_t e = cudaSuccess;
    switch (H->scheme) {
        case HSGN_SCHEME_SI1:  // one stage with tau = dt, no reconstruction
            return launch_stage(H, U, nullptr, 1.0, 0.0, 1.0, 0.0, dt, H->spd, H->U, true, st);
        case HSGN_SCHEME_ARS222: {
            // explicit stage: E2 = U + gamma dt L(U), W = U + delta dt L(U)
            e = launch_explicit(H, U, nullptr, 0.0, 1.0, gam * dt, H->E2, 0.0, 1.0, del * dt, H->Wd,
                                false, st);
            if (e != cudaSuccess) return e;
            // stage 2: base U^n, linearisation E2
            const double* E2c[4] = {H->E2[0], H->E2[1], H->E2[2], H->E2[3]};
            e = launch_stage(H, U, E2c, 0.0, 1.0, 1.0, 0.0, gam * dt, H->spd, H->U1, false, st);
            if (e != cudaSuccess) return e;
            // stage 3: base U + ((1-gamma)/gamma)(U_I2 - U), linearisation
            // W + ((1-delta)/gamma)(U_I2 - U)
            const double* Wc[4] = {H->Wd[0], H->Wd[1], H->Wd[2], H->Wd[3]};
            const double k3 = (1.0 - del) / gam, kb = (1.0 - gam) / gam;
            return launch_stage(H, U, U1c, -k3, k3, 1.0 - kb, kb, gam * dt, H->spd, H->U, true, st,
                                Wc, 1.0);
        }
        case HSGN_SCHEME_EX_HEUN:
        case HSGN_SCHEME_EX_EULER: {
            const bool heun = H->scheme == HSGN_SCHEME_EX_HEUN;
            e = cudaMemsetAsync(H->spd + 4, 0, sizeof(double), st);
            if (e != cudaSuccess) return e;
            // U* = U + dt L(U)
            e = launch_explicit(H, U, nullptr, 0.0, 1.0, dt, H->U1, 0.0, 0.0, 0.0, nullptr, !heun,
                                st);
            if (e != cudaSuccess) return e;
            if (heun) {  // U^{n+1} = (U + U* + dt L(U*))/2
                e = launch_explicit(H, U1c, U, 0.5, 0.5, 0.5 * dt, H->U, 0.0, 0.0, 0.0, nullptr,
                                    true, st);
            } else {
                for (int k = 0; k < 4 && e == cudaSuccess; ++k)
                    e = cudaMemcpyAsync(H->U[k], H->U1[k], H->n * sizeof(double),
                                        cudaMemcpyDeviceToDevice, st);
            }
            if (e != cudaSuccess) return e;
            // the next step's Rusanov speed
            if (!local_speed(H))
                e = cudaMemcpyAsync(H->spd, H->spd + 4, sizeof(double), cudaMemcpyDeviceToDevice,
                                    st);
            return e;
        }
        default:
            return cudaErrorInvalidValue;
    }
}

// IMEX step of Sec. 3.2 in efficient form:
//   U1 = S(U, U, gamma dt);
//   U  <- S(U_b, U_l, gamma dt), U_l = (1-c/gamma) U + (c/gamma) U1,
//                                U_b = (1-(1-gamma)/gamma) U + ((1-gamma)/gamma) U1.
cudaError_t enqueue_step(hsgn_s* H, double dt, cudaStream_t st) {
    const double gam = 1.0 - 1.0 / std::sqrt(2.0);
    const double c = 1.0 / (2.0 * gam);
    const double tau = gam * dt;
    if (H->dfloat) {
        cudaError_t e = launch_stage_df(H, 1, tau, st);
        if (e == cudaSuccess) e = launch_stage_df(H, 2, tau, st);
        if (e == cudaSuccess) H->cur ^= 1;
        return e;
    }
    if (H->windowed) {
        cudaError_t e = launch_stage_fused(H, 1, tau, st);
        if (e == cudaSuccess) e = launch_stage_fused(H, 2, tau, st);
        if (e == cudaSuccess) H->cur ^= 1;
        return e;
    }
    if (H->mixed) {
        const cudaError_t e = launch_stage_mixed(H, 1, tau, st);
        if (e != cudaSuccess) return e;
        return launch_stage_mixed(H, 2, tau, st);
    }
    if (H->scheme != HSGN_SCHEME_PRINTED) return enqueue_step_scheme(H, dt, st);
    const double* A[4] = {H->U[0], H->U[1], H->U[2], H->U[3]};
    const double* B[4] = {H->U1[0], H->U1[1], H->U1[2], H->U1[3]};
    cudaError_t e = launch_stage(H, A, nullptr, 1.0, 0.0, 1.0, 0.0, tau, H->spd, H->U1, false, st);
    if (e != cudaSuccess) return e;
    return launch_stage(H, A, B, 1.0 - c / gam, c / gam, 1.0 - (1.0 - gam) / gam,
                        (1.0 - gam) / gam, tau, H->spd, H->U, true, st);
}

int read_error(hsgn_s* H, cudaStream_t st) {
    unsigned bits = 0, need = 0;
    if (cudaMemcpyAsync(&bits, H->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return HSGN_ERR_CUDA;
    // the double-float form: the coupling the last step recorded sets the
    // window overlap of the steps enqueued from here on
    if (H->dfneed && cudaMemcpyAsync(&need, H->dfneed + H->cur, sizeof(unsigned),
                                     cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return HSGN_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HSGN_ERR_CUDA;
    if (H->dfneed && need) set_df_overlap(H, df_overlap_for(need));
    if (bits) {
        if (cudaMemsetAsync(H->err, 0, sizeof(unsigned), st) != cudaSuccess) return HSGN_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return HSGN_ERR_CUDA;
    }
    return map_error_bits(bits);
}

// max |u| and max nu of the current state into out[0..1] (which must be zero).
void launch_speeds(hsgn_s* H, double* out, cudaStream_t st) {
    double* const* U = state(H);
    if (H->windowed)
        k_speeds_df<<<304, 256, 0, st>>>(H->n, reinterpret_cast<const float2*>(U[0]),
                                         reinterpret_cast<const float2*>(U[1]),
                                         reinterpret_cast<const float2*>(U[2]), H->g, H->lam, out,
                                         H->err);
    else
        k_speeds<<<304, 256, 0, st>>>(H->n, U[0], U[1], U[2], H->g, H->lam, out, H->err);
}

// Recompute the global Rusanov speed max |u| of the current state.
// A caller buffer the state conversions can address directly: memory of
// this handle's device. Host memory (page-locked or not) goes through
// cudaMemcpyAsync and the idle state buffer: the copy engines move it as fast
// as kernels reading the host link would, and leave the SMs free for the work
// of other streams.
const void* device_view(const hsgn_s* H, const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice && a.device == H->device) return p;
    return nullptr;
}

// Grid of the state conversions and of the speed refresh.
unsigned convert_blocks(const hsgn_s* H) {
    const int64_t want = (H->n + 255) / 256;
    return (unsigned)(want < 4864 ? (want > 0 ? want : 1) : 4864);
}

cudaError_t refresh_speed(hsgn_s* H, cudaStream_t st) {
    if (H->batched) {
        if (H->windowed) {
            double* const* U = state(H);
            k_umax_batched_df<<<(unsigned)H->count, 256, 0, st>>>(
                H->inst, reinterpret_cast<const float2*>(U[0]), reinterpret_cast<const float2*>(U[1]),
                speed_of(H, H->cur), H->err);
        } else {
            k_speeds_batched<<<(unsigned)H->count, 256, 0, st>>>(H->inst, H->U[0], H->U[1],
                                                                 H->U[2], H->g, H->speeds, nullptr,
                                                                 H->err);
        }
        return cudaGetLastError();
    }
    double* out = speed_of(H, H->cur);
    cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    // a new state: no coupling recorded yet
    if (H->dfneed) {
        e = cudaMemsetAsync(H->dfneed, 0, 2 * sizeof(unsigned), st);
        set_df_overlap(H, DHW_START);
    }
    if (e != cudaSuccess) return e;
    if (explicit_scheme(H) && !local_speed(H)) {
        // the fully explicit schemes step with the spectral radius max(|u| + c)
        launch_speeds(H, out, st);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out, out + 1, sizeof(double), cudaMemcpyDeviceToDevice, st);
        return e;
    }
    if (H->windowed && !H->dfloat) {
        // (the double-float form takes max |u| in double precision below)
        double* const* U = state(H);
        k_umax_df<<<convert_blocks(H), 256, 0, st>>>(H->n, reinterpret_cast<const float2*>(U[0]),
                                                     reinterpret_cast<const float2*>(U[1]), out,
                                                     H->err);
    } else {
        launch_speeds(H, out, st);
    }
    return cudaGetLastError();
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }


// Tiles of a windowed batch: instance k runs on batch variant var[k] with
// equal tiles of at most that variant's rows; instance info and the tile
// tables are rewritten (the device must be idle) and the captured step graphs
// dropped, since the launches change.
int64_t batch_variant_tiles(int v, int64_t n) {
    const int64_t s = fused_tile_rows(n, batch_variant_smax(v), 1);
    return (n + s - 1) / s;
}

cudaError_t assign_tiles(hsgn_s* H, const std::vector<int8_t>& var) {
    std::vector<int32_t> t[kBV];
    for (int32_t k = 0; k < H->count; ++k) {
        InstInfo& I = H->inst_h[(size_t)k];
        const int v = var[(size_t)k];
        I.base = fused_tile_rows(I.n, batch_variant_smax(v), 1);
        I.P = (int32_t)((I.n + I.base - 1) / I.base);
        I.blk0 = (int32_t)t[v].size();
        for (int32_t b = 0; b < I.P; ++b) t[v].push_back(k);
    }
    cudaError_t e = cudaMemcpy(H->inst, H->inst_h.data(), H->count * sizeof(InstInfo),
                               cudaMemcpyHostToDevice);
    for (int v = 0; v < kBV && e == cudaSuccess; ++v)
        if (!t[v].empty())
            e = cudaMemcpy(H->vtile[v], t[v].data(), t[v].size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    H->variant = var;
    for (int v = 0; v < kBV; ++v) H->vtiles[v] = (int64_t)t[v].size();
    H->total_tiles = H->vtiles[0];
    for (int c = 0; c < 2; ++c)
        if (H->gexec[c]) {
            cudaGraphExecDestroy(H->gexec[c]);
            H->gexec[c] = nullptr;
        }
    return cudaSuccess;
}

}  // namespace

extern "C" {

const char* hsgn_error_string(int code) {
    switch (code) {
        case HSGN_OK: return "ok";
        case HSGN_ERR_INVALID_ARG: return "invalid argument";
        case HSGN_ERR_CUDA: return "CUDA runtime error";
        case HSGN_ERR_NONPOSITIVE_DEPTH: return "non-positive depth";
        case HSGN_ERR_NOT_COERCIVE: return "not coercive (beta <= 0 or non-positive pivot)";
        case HSGN_ERR_NONFINITE: return "non-finite value";
        case HSGN_ERR_UNIMPLEMENTED: return "not implemented";
        case HSGN_ERR_OUT_OF_MEMORY: return "out of device memory";
        case HSGN_ERR_TRUNCATION:
            return "windowed depth solve: coupling decays too slowly for the overlap (reduce dt "
                   "or use HSGN_EXACT_SOLVE)";
        default: return "unknown error code";
    }
}

int hsgn_create(const hsgn_grid_t* grid, double g, double lambda, const double* bathymetry,
                int32_t flags, hsgn_handle_t* out) {
    if (!out) return HSGN_ERR_INVALID_ARG;
    *out = nullptr;
    if (!grid || grid->n < 3 || grid->reserved != 0) return HSGN_ERR_INVALID_ARG;
    if (grid->bc != HSGN_BC_PERIODIC && grid->bc != HSGN_BC_TRANSMISSIVE) return HSGN_ERR_INVALID_ARG;
    if (!(grid->x_right > grid->x_left) || !std::isfinite(grid->x_left) ||
        !std::isfinite(grid->x_right))
        return HSGN_ERR_INVALID_ARG;
    if (!(g > 0.0) || !std::isfinite(g) || !(lambda >= 0.0) || !std::isfinite(lambda))
        return HSGN_ERR_INVALID_ARG;
    if (flags & ~(int32_t)(HSGN_RUSANOV_LOCAL | HSGN_MIXED | HSGN_WELL_BALANCED | HSGN_EXACT_SOLVE |
                           HSGN_DOUBLE_FLOAT | HSGN_SCHEME_MASK))
        return HSGN_ERR_UNIMPLEMENTED;
    // the double-float form (alone, or with HSGN_MIXED for the FP32-flux split):
    // the paper's scheme; the bottom form in pairs throughout (not with the split)
    if ((flags & HSGN_DOUBLE_FLOAT) && (flags & (HSGN_EXACT_SOLVE | HSGN_SCHEME_MASK)))
        return HSGN_ERR_UNIMPLEMENTED;
    if ((flags & HSGN_DOUBLE_FLOAT) && (flags & HSGN_WELL_BALANCED) && (flags & HSGN_MIXED))
        return HSGN_ERR_UNIMPLEMENTED;
    const int32_t scheme = flags & HSGN_SCHEME_MASK;
    if (scheme > HSGN_SCHEME_EX_EULER) return HSGN_ERR_INVALID_ARG;
    // the comparison schemes exist in the flat FP64 form only
    if (scheme != HSGN_SCHEME_PRINTED && (flags & (HSGN_MIXED | HSGN_WELL_BALANCED)))
        return HSGN_ERR_UNIMPLEMENTED;
    if (bathymetry && !(flags & HSGN_WELL_BALANCED)) return HSGN_ERR_INVALID_ARG;
    // the bottom form in mixed precision exists on the windowed kernel only
    if ((flags & HSGN_WELL_BALANCED) && (flags & HSGN_MIXED) && (flags & HSGN_EXACT_SOLVE))
        return HSGN_ERR_UNIMPLEMENTED;
    if (grid->n > ((int64_t)1 << 40)) return HSGN_ERR_INVALID_ARG;

    hsgn_s* H = new (std::nothrow) hsgn_s;
    if (!H) return HSGN_ERR_OUT_OF_MEMORY;
    H->n = grid->n;
    H->bc = grid->bc;
    H->flags = flags;
    H->dx = (grid->x_right - grid->x_left) / (double)grid->n;
    H->g = g;
    H->lam = lambda;
    cudaGetDevice(&H->device);
    {
        // rows per block of the FP64 stage: AS when the grid
        // fills a wave of co-resident CTAs; for smaller grids shorter blocks
        // (down to 64 rows, one per thread), which shortens the serial chunk
        // elimination of each CTA (a division per row on the FP64 pipe)
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, H->device);
        // the occupancy query needs the opt-in shared-memory size set first
        set_smem(k_stage_assemble<AT, AM, BC_PERIODIC, false>, sizeof(AssembleShared<AT, AM>));
        set_smem(k_stage_assemble<AT, AM, BC_PERIODIC, true>, sizeof(AssembleShared<AT, AM, true>));
        if (H->wb)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, k_stage_assemble<AT, AM, BC_PERIODIC, true>, AT,
                sizeof(AssembleShared<AT, AM, true>));
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, k_stage_assemble<AT, AM, BC_PERIODIC, false>, AT,
                sizeof(AssembleShared<AT, AM>));
        cudaGetLastError();
        // (the exact mixed form keeps AS rows, as its batches do, so that an
        // instance evolves bitwise alike alone and in a batch)
        H->split = make_split(H->n, (flags & HSGN_MIXED) ? (int64_t)AS
                                    : stage_block_rows(H->n, (int64_t)(sms > 0 ? sms : 1) *
                                                                 (per_sm > 0 ? per_sm : 1)));
    }
    const int64_t n = H->n, P = H->split.P;

    H->dfloat = (flags & HSGN_DOUBLE_FLOAT) != 0;
    H->df_f32 = H->dfloat && (flags & HSGN_MIXED) != 0;
    H->mixed = (flags & HSGN_MIXED) != 0 && !H->dfloat;
    H->windowed = (H->mixed && !(flags & HSGN_EXACT_SOLVE)) || H->dfloat;
    H->wb = (flags & HSGN_WELL_BALANCED) != 0;
    H->scheme = scheme;
    const size_t vec = align_up(n * sizeof(double));
    const size_t fvec = align_up((n + 1) * sizeof(float));
    const size_t recb = align_up(3 * n * sizeof(float4));
    size_t total = H->dfloat   ? 12 * vec                      // U, V; dU1 (pairs)
                   : H->windowed ? 8 * vec + 4 * fvec            // U, V; G1 dq1 dm1 dr1
                   : H->mixed  ? 4 * vec + 4 * fvec + recb     // U; G1 dq1 dm1 dr1; row records
                               : 16 * vec;                     // U, U1, y v w, 5 back-sub arrays
    if (H->wb) total += H->windowed ? vec : (bathymetry ? 2 : 1) * vec;  // pairs; Phi, bottom
    if (scheme == HSGN_SCHEME_ARS222) total += 8 * vec;    // E2, W
    total += align_up(BLK_STRIDE * P * sizeof(double)) + align_up(P * sizeof(double));
    const size_t rws = rows_ws_bytes(P);
    total += rws + align_up(8 * sizeof(double)) + align_up(sizeof(unsigned));
    if (H->dfloat) total += align_up(2 * sizeof(unsigned));
    if (cudaMalloc(&H->mem, total) != cudaSuccess) {
        cudaGetLastError();
        delete H;
        return HSGN_ERR_OUT_OF_MEMORY;
    }
    unsigned char* p = H->mem;
    auto take = [&](size_t bytes) {
        unsigned char* r = p;
        p += bytes;
        return r;
    };
    for (int k = 0; k < 4; ++k) H->U[k] = reinterpret_cast<double*>(take(vec));
    if (H->dfloat) {
        for (int k = 0; k < 4; ++k) H->V[k] = reinterpret_cast<double*>(take(vec));
        for (int k = 0; k < 4; ++k) H->D1[k] = reinterpret_cast<float2*>(take(vec));
        if (H->wb) H->bathy_df = reinterpret_cast<float2*>(take(vec));
    } else if (H->windowed) {
        for (int k = 0; k < 4; ++k) H->V[k] = reinterpret_cast<double*>(take(vec));
        H->G1 = reinterpret_cast<float*>(take(fvec));
        H->dq1 = reinterpret_cast<float*>(take(fvec));
        H->dm1 = reinterpret_cast<float*>(take(fvec));
        H->dr1 = reinterpret_cast<float*>(take(fvec));
        if (H->wb) H->bathy_df = reinterpret_cast<float2*>(take(vec));
    } else if (H->mixed) {
        H->G1 = reinterpret_cast<float*>(take(fvec));
        H->dq1 = reinterpret_cast<float*>(take(fvec));
        H->dm1 = reinterpret_cast<float*>(take(fvec));
        H->dr1 = reinterpret_cast<float*>(take(fvec));
        H->mrec = reinterpret_cast<float4*>(take(recb));
        H->mblk = reinterpret_cast<float*>(take(align_up(BLK_STRIDE * P * sizeof(double))));
        H->ms_ = reinterpret_cast<float*>(take(align_up(P * sizeof(double))));
    } else {
        for (int k = 0; k < 4; ++k) H->U1[k] = reinterpret_cast<double*>(take(vec));
        H->y = reinterpret_cast<double*>(take(vec));
        H->v = reinterpret_cast<double*>(take(vec));
        H->w = reinterpret_cast<double*>(take(vec));
        H->qs = reinterpret_cast<double*>(take(vec));
        H->ms = reinterpret_cast<double*>(take(vec));
        H->rs = reinterpret_cast<double*>(take(vec));
        H->be = reinterpret_cast<double*>(take(vec));
        H->de = reinterpret_cast<double*>(take(vec));
        H->blk = reinterpret_cast<double*>(take(align_up(BLK_STRIDE * P * sizeof(double))));
        H->s = reinterpret_cast<double*>(take(align_up(P * sizeof(double))));
        if (H->wb) {
            H->phi = reinterpret_cast<double*>(take(vec));
            if (bathymetry) H->bathy = reinterpret_cast<double*>(take(vec));
        }
        if (scheme == HSGN_SCHEME_ARS222)
            for (int k = 0; k < 4; ++k) {
                H->E2[k] = reinterpret_cast<double*>(take(vec));
                H->Wd[k] = reinterpret_cast<double*>(take(vec));
            }
    }
    H->rws = rws ? take(rws) : nullptr;
    H->spd = reinterpret_cast<double*>(take(align_up(8 * sizeof(double))));
    if (H->dfloat) H->dfneed = reinterpret_cast<unsigned*>(take(align_up(2 * sizeof(unsigned))));
    H->err = reinterpret_cast<unsigned*>(take(align_up(sizeof(unsigned))));

    cudaError_t e = cudaMemset(H->mem, 0, total);
    if (e == cudaSuccess && H->dfloat) {
        e = set_smem_df<BC_PERIODIC>();
        if (e == cudaSuccess) e = set_smem_df<BC_TRANSMISSIVE>();
        int sms = 0, per_sm = 0;
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, H->device);
        if (e == cudaSuccess)
            e = H->wb ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                            &per_sm, k_df_stage<DT, FM, DHW, BC_PERIODIC, 2, false, true>, DT,
                            sizeof(DfShared<DT, FM, DHW, true>))
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                            &per_sm, k_df_stage<DT, FM, DHW, BC_PERIODIC, 2, false>, DT,
                            sizeof(DfShared<DT, FM, DHW>));
        const int64_t slots = (int64_t)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
        H->tileSlots = (int32_t)slots;
        set_df_overlap(H, DHW_START);
    } else if (e == cudaSuccess && H->windowed) {
        e = set_smem_fused<FT, BC_PERIODIC, false>();
        if (e == cudaSuccess) e = set_smem_fused<FT, BC_TRANSMISSIVE, false>();
        if (e == cudaSuccess) e = set_smem_fused<FT, BC_PERIODIC, true>();
        if (e == cudaSuccess) e = set_smem_fused<FT, BC_TRANSMISSIVE, true>();
        int sms = 0, per_sm = 0;
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, H->device);
        if (e == cudaSuccess)
            e = H->wb ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                            &per_sm, k_mixed_fused<FT, FM, FHW, BC_PERIODIC, true, 2>, FT,
                            sizeof(FusedShared<FT, FM, FHW, true>))
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                            &per_sm, k_mixed_fused<FT, FM, FHW, BC_PERIODIC, false, 2>, FT,
                            sizeof(FusedShared<FT, FM, FHW>));
        const int64_t slots = (int64_t)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
        H->tileS = (int32_t)fused_tile_rows(n, FusedGeom<FT, FM, FHW>::S, slots);
        H->tileSlots = (int32_t)slots;
    }
    // the bottom: host or device memory, copied once (cudaMemcpyDefault infers which);
    // the windowed form keeps it as double-float pairs, converted through V[0]
    if (e == cudaSuccess && H->bathy)
        e = cudaMemcpy(H->bathy, bathymetry, n * sizeof(double), cudaMemcpyDefault);
    if (e == cudaSuccess && H->bathy_df && bathymetry) {
        e = cudaMemcpy(H->V[0], bathymetry, n * sizeof(double), cudaMemcpyDefault);
        if (e == cudaSuccess) {
            k_df_from_f64<<<1216, 256>>>(n, H->V[0], H->bathy_df);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e == cudaSuccess)
        e = set_smem(k_stage_assemble<AT, AM, BC_PERIODIC, false>, sizeof(AssembleShared<AT, AM>));
    if (e == cudaSuccess)
        e = set_smem(k_stage_assemble<AT, AM, BC_TRANSMISSIVE, false>, sizeof(AssembleShared<AT, AM>));
    if (e == cudaSuccess)
        e = set_smem(k_stage_assemble<AT, AM, BC_PERIODIC, true>, sizeof(AssembleShared<AT, AM, true>));
    if (e == cudaSuccess)
        e = set_smem(k_stage_assemble<AT, AM, BC_TRANSMISSIVE, true>,
                     sizeof(AssembleShared<AT, AM, true>));
    if (e == cudaSuccess)
        e = set_smem(k_mixed_assemble<XT, XM, BC_PERIODIC>, sizeof(MixedShared<XT, XM>));
    if (e == cudaSuccess)
        e = set_smem(k_mixed_assemble<XT, XM, BC_TRANSMISSIVE>, sizeof(MixedShared<XT, XM>));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&H->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (H->cap) cudaStreamDestroy(H->cap);
        cudaFree(H->mem);
        delete H;
        return HSGN_ERR_CUDA;
    }
    *out = H;
    return HSGN_OK;
}

void hsgn_destroy(hsgn_handle_t H) {
    if (!H) return;
    for (const auto& r : H->recs) {
        cudaEventSynchronize(r.b);
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : H->ev_pool) cudaEventDestroy(e);
    for (int c = 0; c < 2; ++c) {
        if (H->gexec[c]) cudaGraphExecDestroy(H->gexec[c]);
        if (H->gcfl[c]) cudaGraphExecDestroy(H->gcfl[c]);
    }
    if (H->cap) cudaStreamDestroy(H->cap);
    cudaFree(H->mem);
    delete H;
}

int hsgn_set_state(hsgn_handle_t H, const double* depth, const double* q, const double* heta,
                   const double* hw, void* stream) {
    if (!H || !depth || !q || !heta || !hw) return HSGN_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    const double* src[4] = {depth, q, heta, hw};
    if (!H->windowed) {
        for (int k = 0; k < 4; ++k)
            if (cudaMemcpyAsync(state(H)[k], src[k], H->n * sizeof(double), cudaMemcpyDefault,
                                st) != cudaSuccess)
                return HSGN_ERR_CUDA;
        return refresh_speed(H, st) == cudaSuccess ? HSGN_OK : HSGN_ERR_CUDA;
    }
    // the windowed path holds double-float pairs: converted straight from the
    // caller's buffer when the device can address it (device memory of this
    // device, page-locked host memory mapped into the device's address space),
    // else copied to the idle buffer first. The copies are issued back to back
    // and the conversions after them, so that the copy engine does not wait
    // for a conversion between two arrays.
    double* const* idle = H->cur ? H->U : H->V;
    const double* v[4];
    for (int k = 0; k < 4; ++k) {
        v[k] = static_cast<const double*>(device_view(H, src[k]));
        if (!v[k]) {
            if (cudaMemcpyAsync(idle[k], src[k], H->n * sizeof(double), cudaMemcpyDefault, st) !=
                cudaSuccess)
                return HSGN_ERR_CUDA;
            v[k] = idle[k];
        }
    }
    for (int k = 0; k < 4; ++k)
        k_df_from_f64<<<convert_blocks(H), 256, 0, st>>>(H->n, v[k],
                                                         reinterpret_cast<float2*>(state(H)[k]));
    if (cudaGetLastError() != cudaSuccess) return HSGN_ERR_CUDA;
    return refresh_speed(H, st) == cudaSuccess ? HSGN_OK : HSGN_ERR_CUDA;
}

int hsgn_get_state(hsgn_handle_t H, double* depth, double* q, double* heta, double* hw,
                   void* stream) {
    const int rc = hsgn_copy_state_out(H, depth, q, heta, hw, stream);
    if (rc != HSGN_OK) return rc;
    return read_error(H, as_stream(stream));
}

int hsgn_copy_state_out(hsgn_handle_t H, double* depth, double* q, double* heta, double* hw,
                        void* stream) {
    if (!H || !depth || !q || !heta || !hw) return HSGN_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    double* dst[4] = {depth, q, heta, hw};
    double* const* src = state(H);
    if (H->windowed) {
        // pairs to doubles: straight into the caller's buffer when the device
        // can address it, else through the idle buffer and a copy (the four
        // conversions first, then the copies back to back)
        double* const* tmp = H->cur ? H->U : H->V;
        double* v[4];
        for (int k = 0; k < 4; ++k) {
            v[k] = static_cast<double*>(const_cast<void*>(device_view(H, dst[k])));
            k_f64_from_df<<<convert_blocks(H), 256, 0, st>>>(
                H->n, reinterpret_cast<const float2*>(src[k]), v[k] ? v[k] : tmp[k]);
        }
        if (cudaGetLastError() != cudaSuccess) return HSGN_ERR_CUDA;
        for (int k = 0; k < 4; ++k)
            if (!v[k] && cudaMemcpyAsync(dst[k], tmp[k], H->n * sizeof(double), cudaMemcpyDefault,
                                         st) != cudaSuccess)
                return HSGN_ERR_CUDA;
        return HSGN_OK;
    }
    for (int k = 0; k < 4; ++k)
        if (cudaMemcpyAsync(dst[k], src[k], H->n * sizeof(double), cudaMemcpyDefault, st) !=
            cudaSuccess)
            return HSGN_ERR_CUDA;
    return HSGN_OK;
}

// dt of a step: positive and finite for one instance, 0 for a batch (which
// takes each instance's step from its table).
bool valid_dt(const hsgn_s* H, double dt) {
    return H->batched ? dt == 0.0 : (dt > 0.0 && std::isfinite(dt));
}

int hsgn_step(hsgn_handle_t H, double dt, void* stream) {
    if (!H || !valid_dt(H, dt)) return HSGN_ERR_INVALID_ARG;
    return enqueue_step(H, dt, as_stream(stream)) == cudaSuccess ? HSGN_OK : HSGN_ERR_CUDA;
}

int hsgn_enqueue(hsgn_handle_t H, double dt, int64_t n_steps, void* stream) {
    if (!H || !valid_dt(H, dt) || n_steps < 0) return HSGN_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    // one captured step per state buffer (the windowed path alternates them)
    for (int64_t k = 0; k < n_steps; ++k) {
        const int c = H->cur;
        if (!H->gexec[c] || H->gdt[c] != dt || H->ghw[c] != H->dfhw) {
            const bool prof = H->prof;
            H->prof = false;  // events are not captured into the graph
            if (H->gexec[c]) {
                cudaGraphExecDestroy(H->gexec[c]);
                H->gexec[c] = nullptr;
            }
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(H->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                H->prof = prof;
                return HSGN_ERR_CUDA;
            }
            const cudaError_t e1 = enqueue_step(H, dt, H->cap);
            const cudaError_t e2 = cudaStreamEndCapture(H->cap, &graph);
            H->prof = prof;
            H->cur = c;  // capturing does not advance the state
            if (e1 != cudaSuccess || e2 != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                return HSGN_ERR_CUDA;
            }
            const cudaError_t e3 = cudaGraphInstantiate(&H->gexec[c], graph, 0);
            cudaGraphDestroy(graph);
            if (e3 != cudaSuccess) {
                H->gexec[c] = nullptr;
                cudaGetLastError();
                return HSGN_ERR_CUDA;
            }
            H->gdt[c] = dt;
            H->ghw[c] = H->dfhw;
        }
        if (cudaGraphLaunch(H->gexec[c], st) != cudaSuccess) return HSGN_ERR_CUDA;
        if (H->windowed) H->cur ^= 1;
    }
    return HSGN_OK;
}

int hsgn_df_overlap(hsgn_handle_t H, int32_t* rows_needed, int32_t* overlap, void* stream) {
    if (!H || !rows_needed || !overlap) return HSGN_ERR_INVALID_ARG;
    if (!H->dfloat || !H->dfneed) return HSGN_ERR_UNIMPLEMENTED;
    cudaStream_t st = as_stream(stream);
    unsigned need = 0;
    if (cudaMemcpyAsync(&need, H->dfneed + H->cur, sizeof(unsigned), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return HSGN_ERR_CUDA;
    set_df_overlap(H, df_overlap_for(need));
    *rows_needed = (int32_t)need;
    *overlap = H->dfhw;
    return HSGN_OK;
}

int hsgn_run_cfl(hsgn_handle_t H, double cfl, double mcfl, int64_t n_steps, double* t_advanced,
                 void* stream) {
    if (!H || !t_advanced || !(cfl > 0.0) || !std::isfinite(cfl) || !(mcfl >= 0.0) ||
        !std::isfinite(mcfl) || n_steps < 0)
        return HSGN_ERR_INVALID_ARG;
    if (!H->dfloat || H->batched || local_speed(H)) return HSGN_ERR_UNIMPLEMENTED;
    cudaStream_t st = as_stream(stream);
    // max |u| and max nu of the current state (set_state and fixed steps keep
    // only max |u|), and the time advanced so far
    double* const cur = speed_of(H, H->cur);
    if (cudaMemsetAsync(cur, 0, 2 * sizeof(double), st) != cudaSuccess ||
        cudaMemsetAsync(H->spd + 6, 0, 2 * sizeof(double), st) != cudaSuccess)
        return HSGN_ERR_CUDA;
    launch_speeds(H, cur, st);
    if (cudaGetLastError() != cudaSuccess) return HSGN_ERR_CUDA;
    for (int64_t k = 0; k < n_steps; ++k) {
        const int c = H->cur;
        if (!H->gcfl[c] || H->gcfl_rule[c][0] != cfl || H->gcfl_rule[c][1] != mcfl ||
            H->gcfl_hw[c] != H->dfhw) {
            const bool prof = H->prof;
            H->prof = false;
            if (H->gcfl[c]) {
                cudaGraphExecDestroy(H->gcfl[c]);
                H->gcfl[c] = nullptr;
            }
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(H->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                H->prof = prof;
                return HSGN_ERR_CUDA;
            }
            cudaError_t e1 = launch_stage_df(H, 1, 0.0, H->cap, cfl, mcfl);
            if (e1 == cudaSuccess) e1 = launch_stage_df(H, 2, 0.0, H->cap, cfl, mcfl);
            const cudaError_t e2 = cudaStreamEndCapture(H->cap, &graph);
            H->prof = prof;
            if (e1 != cudaSuccess || e2 != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
                return HSGN_ERR_CUDA;
            }
            const cudaError_t e3 = cudaGraphInstantiate(&H->gcfl[c], graph, 0);
            cudaGraphDestroy(graph);
            if (e3 != cudaSuccess) {
                H->gcfl[c] = nullptr;
                cudaGetLastError();
                return HSGN_ERR_CUDA;
            }
            H->gcfl_rule[c][0] = cfl;
            H->gcfl_rule[c][1] = mcfl;
            H->gcfl_hw[c] = H->dfhw;
        }
        if (cudaGraphLaunch(H->gcfl[c], st) != cudaSuccess) return HSGN_ERR_CUDA;
        H->cur ^= 1;
    }
    if (cudaMemcpyAsync(t_advanced, H->spd + 7, sizeof(double), cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return HSGN_ERR_CUDA;
    return read_error(H, st);
}

int hsgn_run(hsgn_handle_t H, double dt, int64_t n_steps, void* stream) {
    if (!H || !valid_dt(H, dt) || n_steps < 0) return HSGN_ERR_INVALID_ARG;
    const int rc = hsgn_enqueue(H, dt, n_steps, stream);
    if (rc != HSGN_OK) return rc;
    return read_error(H, as_stream(stream));
}

int hsgn_profile(hsgn_handle_t H, int32_t enable) {
    if (!H) return HSGN_ERR_INVALID_ARG;
    H->prof = enable != 0;
    return HSGN_OK;
}

int hsgn_profile_read(hsgn_handle_t H, double* ms, int64_t* launches, int32_t reset) {
    if (!H) return HSGN_ERR_INVALID_ARG;
    int rc = HSGN_OK;
    for (const auto& r : H->recs) {
        float t = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess)
            rc = HSGN_ERR_CUDA;
        H->prof_ms[r.kind] += t;
        H->prof_n[r.kind] += 1;
        H->ev_pool.push_back(r.a);
        H->ev_pool.push_back(r.b);
    }
    H->recs.clear();
    for (int k = 0; k < HSGN_PROF_KINDS; ++k) {
        if (ms) ms[k] = H->prof_ms[k];
        if (launches) launches[k] = H->prof_n[k];
    }
    if (reset)
        for (int k = 0; k < HSGN_PROF_KINDS; ++k) {
            H->prof_ms[k] = 0.0;
            H->prof_n[k] = 0;
        }
    return rc;
}

int hsgn_check(hsgn_handle_t H, void* stream) {
    if (!H) return HSGN_ERR_INVALID_ARG;
    return read_error(H, as_stream(stream));
}

int hsgn_suggest_dt(hsgn_handle_t H, double cfl, double mcfl, double* dt_out, void* stream) {
    if (!H || !dt_out || !(cfl > 0.0)) return HSGN_ERR_INVALID_ARG;
    if (H->batched) return HSGN_ERR_UNIMPLEMENTED;
    cudaStream_t st = as_stream(stream);
    double* tmp = H->spd + 2;
    if (cudaMemsetAsync(tmp, 0, 2 * sizeof(double), st) != cudaSuccess) return HSGN_ERR_CUDA;
    launch_speeds(H, tmp, st);
    if (cudaGetLastError() != cudaSuccess) return HSGN_ERR_CUDA;
    double hv[2];
    if (cudaMemcpyAsync(hv, tmp, sizeof(hv), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return HSGN_ERR_CUDA;
    const int rc = read_error(H, st);
    if (rc != HSGN_OK) return rc;
    const double umax = hv[0], numax = hv[1];
    if (!(numax > 0.0)) return HSGN_ERR_INVALID_ARG;
    double dt = cfl * H->dx / numax;
    if (mcfl > 0.0 && umax > 0.0 && umax * dt / H->dx > mcfl) dt = mcfl * H->dx / umax;
    *dt_out = dt;
    return HSGN_OK;
}

int hsgn_stage(hsgn_handle_t H, const double* const base[4], const double* const lin[4],
               double tau, double speed, double* const out[4], void* stream) {
    if (!H || !base || !lin || !out || !(tau > 0.0) || !(speed >= 0.0)) return HSGN_ERR_INVALID_ARG;
    if (H->mixed || H->batched) return HSGN_ERR_UNIMPLEMENTED;
    for (int k = 0; k < 4; ++k)
        if (!base[k] || !lin[k] || !out[k]) return HSGN_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    if (H->dfloat) {
        // the stage-2 kernel with weights 1 and 0 from U_b = base (pairs, in the
        // idle state buffer) and U_l - U_b (pairs, in the increment buffers);
        // the pairs are written into `out` and converted to doubles in place
        double* const* idle = H->cur ? H->U : H->V;
        for (int k = 0; k < 4; ++k)
            k_df_stage_inputs<<<convert_blocks(H), 256, 0, st>>>(
                H->n, base[k], lin[k], reinterpret_cast<float2*>(idle[k]), H->D1[k]);
        double* spd = H->spd + 1;
        k_set_scalar<<<1, 1, 0, st>>>(spd, speed);
        DfParams p = df_params(H, 2, tau, 1.0, 0.0);
        p.track_speed = 0;
        for (int k = 0; k < 4; ++k) {
            p.U[k] = reinterpret_cast<const float2*>(idle[k]);
            p.out[k] = reinterpret_cast<float2*>(out[k]);
        }
        p.speed = spd;
        launch_df(H, df_tiles(H), p, st);
        for (int k = 0; k < 4; ++k)
            k_f64_from_df_inplace<<<convert_blocks(H), 256, 0, st>>>(H->n, out[k]);
        return cudaGetLastError() == cudaSuccess ? HSGN_OK : HSGN_ERR_CUDA;
    }
    k_set_scalar<<<1, 1, 0, st>>>(H->spd + 1, speed);
    if (cudaGetLastError() != cudaSuccess) return HSGN_ERR_CUDA;
    // A = base, B = lin: U_l = lin, U_b = base
    return launch_stage(H, base, lin, 0.0, 1.0, 1.0, 0.0, tau, H->spd + 1, out, false, st) ==
                   cudaSuccess
               ? HSGN_OK
               : HSGN_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Discrete adjoint of a run (declared in include/hsgn.h): the paper's step in
// the FP64 bottom form, states kept at checkpoints and recomputed per segment.
// ---------------------------------------------------------------------------
namespace {

struct AdjWork {
    unsigned char* mem = nullptr;
    int64_t n = 0, K = 0, nck = 0;
    double* ck = nullptr;       // checkpoints, nck x 4n
    double* seg = nullptr;      // states of a segment, (K+1) x 4n
    double* U1 = nullptr;       // stage-1 result
    double* Ue = nullptr;       // stage-2 linearisation state
    double* Ubs = nullptr;      // stage-2 base state
    double* O2 = nullptr;       // stage-2 output
    double* Ua = nullptr;       // dJ/dU of the current step boundary
    double* Ua1 = nullptr;      // dJ/dU_I^(1)
    double* Ab = nullptr;       // stage adjoints
    double* Al = nullptr;
    double* cellw = nullptr;    // 11 x n per-cell work
    double* facew = nullptr;    // 4 x (n+1) per-face work
    unsigned char* sws = nullptr;  // tridiagonal solve workspace
    unsigned long long* sbits = nullptr;  // speed of the step (bits of a double), argmax
    double* Aspeed = nullptr;
    double* J = nullptr;
    int64_t* cells = nullptr;
    double* data = nullptr;
    double* dseg = nullptr;     // gauge data of the current segment, K x n_gauges
    double* fw1 = nullptr;      // q^dag, m^dag, r^dag, beta of the step's stage 1, 4 x n
    size_t work_bytes = 0;      // cellw + facew, zeroed per stage adjoint
    // a full segment of K steps is the same launch sequence for every segment
    // once its checkpoint is in seg[0] and its gauge data in dseg: captured
    // once per kind (forward with the misfit, forward, reverse) and replayed
    cudaGraphExec_t g_fwd_misfit = nullptr, g_fwd = nullptr, g_rev = nullptr;
};

Ptr4 cp4(const double* b, int64_t n) {
    return Ptr4{{b, b + n, b + 2 * n, b + 3 * n}};
}
MutPtr4 mp4(double* b, int64_t n) {
    return MutPtr4{{b, b + n, b + 2 * n, b + 3 * n}};
}

unsigned grid_of(int64_t m) { return (unsigned)((m + 255) / 256); }

// global Rusanov speed max |q/h| of a state and its first argmax cell
cudaError_t adj_speed(AdjWork& W, const double* U, cudaStream_t st) {
    const int64_t n = W.n;
    cudaError_t e = cudaMemsetAsync(W.sbits, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(W.sbits + 1, 0xFF, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_adj_umax<<<304, 256, 0, st>>>(n, U, U + n, W.sbits);
    k_adj_argmax<<<304, 256, 0, st>>>(n, U, U + n, W.sbits, W.sbits + 1);
    return cudaGetLastError();
}

// one step of the paper's scheme on packed arrays in -> out (4n each)
cudaError_t adj_forward_step(hsgn_s* H, AdjWork& W, const double* in, double* out, double dt,
                             cudaStream_t st) {
    const int64_t n = W.n;
    const double gam = 1.0 - 1.0 / std::sqrt(2.0), c = 1.0 / (2.0 * gam);
    cudaError_t e = adj_speed(W, in, st);
    if (e != cudaSuccess) return e;
    const double* speed = reinterpret_cast<const double*>(W.sbits);
    const double* A[4] = {in, in + n, in + 2 * n, in + 3 * n};
    double* U1[4] = {W.U1, W.U1 + n, W.U1 + 2 * n, W.U1 + 3 * n};
    const double* B[4] = {W.U1, W.U1 + n, W.U1 + 2 * n, W.U1 + 3 * n};
    double* O[4] = {out, out + n, out + 2 * n, out + 3 * n};
    e = launch_stage(H, A, nullptr, 1.0, 0.0, 1.0, 0.0, gam * dt, speed, U1, false, st);
    if (e != cudaSuccess) return e;
    return launch_stage(H, A, B, 1.0 - c / gam, c / gam, 1.0 - (1.0 - gam) / gam,
                        (1.0 - gam) / gam, gam * dt, speed, O, false, st);
}

// adjoint of one stage whose forward was just run by launch_stage (the work
// arrays of the handle hold its q^dag, m^dag, r^dag, beta)
// fw: q^dag, m^dag, r^dag and beta of that stage's forward (the handle's work
// arrays right after it, or a copy of them)
cudaError_t adj_stage(hsgn_s* H, AdjWork& W, const double* Ub, const double* Ul, double tau,
                      const double* out, const double* Ao, double* Ab, double* Al,
                      double* Abathy, const double* const fw[4], cudaStream_t st) {
    const int64_t n = W.n;
    AdjParams p;
    p.n = n;
    p.bc = H->bc;
    p.dx = H->dx;
    p.g = H->g;
    p.lam = H->lam;
    p.tau = tau;
    p.speed = reinterpret_cast<const double*>(W.sbits);
    for (int v = 0; v < 4; ++v) {
        p.Ub[v] = Ub + v * n;
        p.Ul[v] = Ul + v * n;
        p.Ao[v] = Ao + v * n;
        p.Ab[v] = Ab + v * n;
        p.Al[v] = Al + v * n;
    }
    p.bathy = H->bathy;
    p.qs = fw[0];
    p.ms = fw[1];
    p.rs = fw[2];
    p.be = fw[3];
    p.hbar = out;
    p.mbar = out + 2 * n;
    p.Abathy = Abathy;
    p.Aspeed = W.Aspeed;
    double* c = W.cellw;
    p.qs_a = c; p.ms_a = c + n; p.rs_a = c + 2 * n; p.be_a = c + 3 * n; p.ph_a = c + 4 * n;
    p.pt_a = c + 5 * n; p.hbar_a = c + 6 * n; p.D_a = c + 7 * n;
    p.ra = c + 8 * n; p.rb = c + 9 * n; p.rc = c + 10 * n;
    double* f = W.facew;
    p.Phi_a = f; p.Fq_a = f + (n + 1); p.Fm_a = f + 2 * (n + 1); p.Fr_a = f + 3 * (n + 1);
    cudaError_t e = cudaMemsetAsync(W.cellw, 0, W.work_bytes, st);
    if (e != cudaSuccess) return e;
    const unsigned gc = grid_of(n), gf = grid_of(n + 1);
    const bool per = H->bc == BC_PERIODIC;
    if (per) k_adj_backsub<BC_PERIODIC><<<gc, 256, 0, st>>>(p);
    else k_adj_backsub<BC_TRANSMISSIVE><<<gc, 256, 0, st>>>(p);
    if (per) k_adj_rows<BC_PERIODIC><<<gc, 256, 0, st>>>(p);
    else k_adj_rows<BC_TRANSMISSIVE><<<gc, 256, 0, st>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = solve_rows(n, per ? 1 : 0, p.ra, p.rb, p.rc, p.hbar_a, p.D_a, W.sws, H->err, nullptr, st);
    if (e != cudaSuccess) return e;
    if (per) k_adj_rowsadj<BC_PERIODIC><<<gc, 256, 0, st>>>(p);
    else k_adj_rowsadj<BC_TRANSMISSIVE><<<gc, 256, 0, st>>>(p);
    if (per) k_adj_phi<BC_PERIODIC><<<gf, 256, 0, st>>>(p);
    else k_adj_phi<BC_TRANSMISSIVE><<<gf, 256, 0, st>>>(p);
    k_adj_cell<<<gc, 256, 0, st>>>(p);
    if (per) k_adj_starred<BC_PERIODIC><<<gc, 256, 0, st>>>(p);
    else k_adj_starred<BC_TRANSMISSIVE><<<gc, 256, 0, st>>>(p);
    if (per) k_adj_flux<BC_PERIODIC><<<gf, 256, 0, st>>>(p);
    else k_adj_flux<BC_TRANSMISSIVE><<<gf, 256, 0, st>>>(p);
    return cudaGetLastError();
}

// dJ/dU^s from dJ/dU^{s+1} (in W.Ua, updated in place) for the step from U
cudaError_t adj_step(hsgn_s* H, AdjWork& W, const double* U, double dt, double* Abathy,
                     cudaStream_t st) {
    const int64_t n = W.n;
    const double gam = 1.0 - 1.0 / std::sqrt(2.0), c = 1.0 / (2.0 * gam);
    const double wl0 = 1.0 - c / gam, wl1 = c / gam;
    const double wb0 = 1.0 - (1.0 - gam) / gam, wb1 = (1.0 - gam) / gam;
    const double tau = gam * dt;
    const unsigned gc = grid_of(n);
    const Ptr4 none{{nullptr, nullptr, nullptr, nullptr}};
    cudaError_t e = adj_speed(W, U, st);
    if (e != cudaSuccess) return e;
    const double* speed = reinterpret_cast<const double*>(W.sbits);
    const double* A[4] = {U, U + n, U + 2 * n, U + 3 * n};
    double* U1m[4] = {W.U1, W.U1 + n, W.U1 + 2 * n, W.U1 + 3 * n};
    // stage-1 forward (its q^dag, m^dag, r^dag, beta kept for its adjoint),
    // the stage-2 states, stage-2 forward
    e = launch_stage(H, A, nullptr, 1.0, 0.0, 1.0, 0.0, tau, speed, U1m, false, st);
    if (e != cudaSuccess) return e;
    const double* const hw[4] = {H->qs, H->ms, H->rs, H->be};
    const double* const fw1[4] = {W.fw1, W.fw1 + n, W.fw1 + 2 * n, W.fw1 + 3 * n};
    for (int v = 0; v < 4 && e == cudaSuccess; ++v)
        e = cudaMemcpyAsync(W.fw1 + v * n, hw[v], n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    k_adj_axpby<<<gc, 256, 0, st>>>(n, wl0, cp4(U, n), wl1, cp4(W.U1, n), 0.0, none, mp4(W.Ue, n));
    k_adj_axpby<<<gc, 256, 0, st>>>(n, wb0, cp4(U, n), wb1, cp4(W.U1, n), 0.0, none, mp4(W.Ubs, n));
    const double* Bb[4] = {W.Ubs, W.Ubs + n, W.Ubs + 2 * n, W.Ubs + 3 * n};
    const double* Bl[4] = {W.Ue, W.Ue + n, W.Ue + 2 * n, W.Ue + 3 * n};
    double* O2m[4] = {W.O2, W.O2 + n, W.O2 + 2 * n, W.O2 + 3 * n};
    e = launch_stage(H, Bb, Bl, 0.0, 1.0, 1.0, 0.0, tau, speed, O2m, false, st);
    if (e != cudaSuccess) return e;
    // stage-2 adjoint
    e = cudaMemsetAsync(W.Ab, 0, 8 * (size_t)n * sizeof(double), st);  // Ab and Al
    if (e == cudaSuccess) e = cudaMemsetAsync(W.Aspeed, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    e = adj_stage(H, W, W.Ubs, W.Ue, tau, W.O2, W.Ua, W.Ab, W.Al, Abathy, hw, st);
    if (e != cudaSuccess) return e;
    k_adj_axpby<<<gc, 256, 0, st>>>(n, wl1, cp4(W.Al, n), wb1, cp4(W.Ab, n), 0.0, none,
                                    mp4(W.Ua1, n));
    k_adj_axpby<<<gc, 256, 0, st>>>(n, wl0, cp4(W.Al, n), wb0, cp4(W.Ab, n), 0.0, none,
                                    mp4(W.Ua, n));
    // stage-1 adjoint
    e = cudaMemsetAsync(W.Ab, 0, 8 * (size_t)n * sizeof(double), st);
    if (e != cudaSuccess) return e;
    e = adj_stage(H, W, U, U, tau, W.U1, W.Ua1, W.Ab, W.Al, Abathy, fw1, st);
    if (e != cudaSuccess) return e;
    k_adj_axpby<<<gc, 256, 0, st>>>(n, 1.0, cp4(W.Ua, n), 1.0, cp4(W.Ab, n), 1.0, cp4(W.Al, n),
                                    mp4(W.Ua, n));
    // the step's speed
    k_adj_speed<<<1, 1, 0, st>>>(U, U + n, W.sbits + 1, W.Aspeed, W.Ua, W.Ua + n);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int hsgn_adjoint(hsgn_handle_t H, double dt, int64_t n_steps, int64_t n_gauges,
                 const int64_t* gauge_cells, const double* gauge_data, int64_t checkpoint_every,
                 double* const grad_state[4], double* grad_bathymetry, double* misfit,
                 void* stream) {
    if (!H || !(dt > 0.0) || !std::isfinite(dt) || n_steps < 1 || n_gauges < 0 || !misfit ||
        checkpoint_every < 1 || (n_gauges > 0 && (!gauge_cells || !gauge_data)))
        return HSGN_ERR_INVALID_ARG;
    if (H->batched || H->mixed || H->dfloat || !H->wb || H->scheme != HSGN_SCHEME_PRINTED ||
        local_speed(H))
        return HSGN_ERR_UNIMPLEMENTED;
    const int64_t n = H->n;
    for (int64_t k = 0; k < n_gauges; ++k)
        if (gauge_cells[k] < 0 || gauge_cells[k] >= n) return HSGN_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    AdjWork W;
    W.n = n;
    W.K = checkpoint_every < n_steps ? checkpoint_every : n_steps;
    W.nck = (n_steps + W.K - 1) / W.K;
    const size_t s4 = align_up(4 * (size_t)n * sizeof(double));
    const size_t cellb = align_up(11 * (size_t)n * sizeof(double));
    const size_t faceb = align_up(4 * (size_t)(n + 1) * sizeof(double));
    const size_t swsb = rows_ws_bytes(n);
    const size_t gcb = align_up((size_t)(n_gauges > 0 ? n_gauges : 1) * sizeof(int64_t));
    const size_t gdb = align_up((size_t)(n_gauges > 0 ? n_gauges : 1) * (size_t)n_steps *
                                sizeof(double));
    const size_t dsb = align_up((size_t)(n_gauges > 0 ? n_gauges : 1) * (size_t)W.K *
                                sizeof(double));
    const size_t total = (size_t)W.nck * s4 + (size_t)(W.K + 1) * s4 + 9 * s4 + cellb + faceb +
                         swsb + align_up(4 * sizeof(unsigned long long)) + gcb + gdb + dsb;
    if (cudaMalloc(&W.mem, total) != cudaSuccess) {
        cudaGetLastError();
        return HSGN_ERR_OUT_OF_MEMORY;
    }
    unsigned char* p = W.mem;
    auto take = [&](size_t b) { unsigned char* r = p; p += b; return r; };
    W.ck = reinterpret_cast<double*>(take((size_t)W.nck * s4));
    W.seg = reinterpret_cast<double*>(take((size_t)(W.K + 1) * s4));
    W.U1 = reinterpret_cast<double*>(take(s4));
    W.Ue = reinterpret_cast<double*>(take(s4));
    W.Ubs = reinterpret_cast<double*>(take(s4));
    W.O2 = reinterpret_cast<double*>(take(s4));
    W.Ua = reinterpret_cast<double*>(take(s4));
    W.Ua1 = reinterpret_cast<double*>(take(s4));
    W.fw1 = reinterpret_cast<double*>(take(s4));
    // Ab and Al are contiguous (one memset clears both)
    W.Ab = reinterpret_cast<double*>(take(2 * s4));
    W.Al = W.Ab + 4 * n;
    W.cellw = reinterpret_cast<double*>(take(cellb));
    W.facew = reinterpret_cast<double*>(take(faceb));
    W.work_bytes = cellb + faceb;  // contiguous
    W.sws = swsb ? take(swsb) : nullptr;
    W.sbits = reinterpret_cast<unsigned long long*>(take(align_up(4 * sizeof(unsigned long long))));
    W.Aspeed = reinterpret_cast<double*>(W.sbits + 2);
    W.J = reinterpret_cast<double*>(W.sbits + 3);
    W.cells = reinterpret_cast<int64_t*>(take(gcb));
    W.data = reinterpret_cast<double*>(take(gdb));
    W.dseg = reinterpret_cast<double*>(take(dsb));
    // Ab/Al: 2*s4 holds 8n doubles only when s4 has no padding between the halves
    int rc = HSGN_OK;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (x != cudaSuccess && e == cudaSuccess) e = x; };
    if (n_gauges > 0) {
        chk(cudaMemcpyAsync(W.cells, gauge_cells, (size_t)n_gauges * sizeof(int64_t),
                            cudaMemcpyHostToDevice, st));
        chk(cudaMemcpyAsync(W.data, gauge_data, (size_t)n_gauges * n_steps * sizeof(double),
                            cudaMemcpyDefault, st));
    }
    chk(cudaMemsetAsync(W.J, 0, sizeof(double), st));
    const size_t sd = s4 / sizeof(double);
    const unsigned gg = (unsigned)((n_gauges + 255) / 256);
    double* const seg = W.seg;
    // L steps from seg[0] into seg[1..L], with the misfit of each new state
    auto fwd_segment = [&](int64_t L, bool misfit, cudaStream_t s) -> cudaError_t {
        for (int64_t j = 0; j < L; ++j) {
            cudaError_t x = adj_forward_step(H, W, seg + (size_t)j * sd, seg + (size_t)(j + 1) * sd,
                                             dt, s);
            if (x != cudaSuccess) return x;
            if (misfit && n_gauges > 0)
                k_adj_gauges<<<gg, 256, 0, s>>>(n_gauges, W.cells, W.dseg + j * n_gauges,
                                                seg + (size_t)(j + 1) * sd, dt, W.J, nullptr);
        }
        return cudaGetLastError();
    };
    // the adjoints of steps L-1 .. 0 of the segment, seg[0..L] holding its states
    auto rev_segment = [&](int64_t L, cudaStream_t s) -> cudaError_t {
        for (int64_t j = L - 1; j >= 0; --j) {
            if (n_gauges > 0)
                k_adj_gauges<<<gg, 256, 0, s>>>(n_gauges, W.cells, W.dseg + j * n_gauges,
                                                seg + (size_t)(j + 1) * sd, dt, nullptr, W.Ua);
            cudaError_t x = adj_step(H, W, seg + (size_t)j * sd, dt, grad_bathymetry, s);
            if (x != cudaSuccess) return x;
        }
        return cudaGetLastError();
    };
    // run a full segment through its graph (captured on first use)
    auto replay = [&](cudaGraphExec_t& g, auto body) -> cudaError_t {
        if (!g) {
            const bool prof = H->prof;
            H->prof = false;  // events are not captured into graphs
            cudaGraph_t graph = nullptr;
            cudaError_t x = cudaStreamBeginCapture(H->cap, cudaStreamCaptureModeThreadLocal);
            if (x == cudaSuccess) {
                const cudaError_t xb = body(H->cap);
                x = cudaStreamEndCapture(H->cap, &graph);
                if (x == cudaSuccess) x = xb;
            }
            H->prof = prof;
            if (x == cudaSuccess) x = cudaGraphInstantiate(&g, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (x != cudaSuccess) {
                g = nullptr;
                return x;
            }
        }
        return cudaGraphLaunch(g, st);
    };
    auto stage_data = [&](int64_t s0, int64_t L) {
        if (n_gauges > 0)
            chk(cudaMemcpyAsync(W.dseg, W.data + s0 * n_gauges,
                                (size_t)L * n_gauges * sizeof(double), cudaMemcpyDeviceToDevice,
                                st));
    };
    // forward: checkpoints every K steps, the misfit after every step
    for (int k = 0; k < 4; ++k)
        chk(cudaMemcpyAsync(seg + k * n, H->U[k], n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    for (int64_t cix = 0; cix < W.nck && e == cudaSuccess; ++cix) {
        const int64_t s0 = cix * W.K, L = std::min(W.K, n_steps - s0);
        chk(cudaMemcpyAsync(W.ck + (size_t)cix * sd, seg, 4 * n * sizeof(double),
                            cudaMemcpyDeviceToDevice, st));
        stage_data(s0, L);
        if (e != cudaSuccess) break;
        if (L == W.K)
            chk(replay(W.g_fwd_misfit, [&](cudaStream_t s) { return fwd_segment(L, true, s); }));
        else
            chk(fwd_segment(L, true, st));
        chk(cudaMemcpyAsync(seg, seg + (size_t)L * sd, 4 * n * sizeof(double),
                            cudaMemcpyDeviceToDevice, st));
    }
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        chk(cudaMemcpyAsync(H->U[k], seg + k * n, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    // reverse, one segment at a time: its states recomputed from the checkpoint
    chk(cudaMemsetAsync(W.Ua, 0, 4 * n * sizeof(double), st));
    if (grad_bathymetry) chk(cudaMemsetAsync(grad_bathymetry, 0, n * sizeof(double), st));
    for (int64_t cix = W.nck - 1; cix >= 0 && e == cudaSuccess; --cix) {
        const int64_t s0 = cix * W.K, L = std::min(W.K, n_steps - s0);
        chk(cudaMemcpyAsync(seg, W.ck + (size_t)cix * sd, 4 * n * sizeof(double),
                            cudaMemcpyDeviceToDevice, st));
        stage_data(s0, L);
        if (e != cudaSuccess) break;
        if (L == W.K) {
            chk(replay(W.g_fwd, [&](cudaStream_t s) { return fwd_segment(L, false, s); }));
            chk(replay(W.g_rev, [&](cudaStream_t s) { return rev_segment(L, s); }));
        } else {
            chk(fwd_segment(L, false, st));
            chk(rev_segment(L, st));
        }
    }
    if (grad_state)
        for (int k = 0; k < 4 && e == cudaSuccess; ++k)
            if (grad_state[k])
                chk(cudaMemcpyAsync(grad_state[k], W.Ua + k * n, n * sizeof(double),
                                    cudaMemcpyDeviceToDevice, st));
    chk(cudaMemcpyAsync(misfit, W.J, sizeof(double), cudaMemcpyDeviceToHost, st));
    chk(refresh_speed(H, st));
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) rc = read_error(H, st);  // synchronises
    else rc = HSGN_ERR_CUDA;
    cudaStreamSynchronize(st);
    for (cudaGraphExec_t g : {W.g_fwd_misfit, W.g_fwd, W.g_rev})
        if (g) cudaGraphExecDestroy(g);
    cudaFree(W.mem);
    return rc;
}

// The single-precision stage constants of an instance from its time step,
// rounded exactly as the single-instance path rounds them (tau = gamma dt,
// gamma = 1 - 1/sqrt(2), Sec. 3.2; each constant formed in double precision).
void set_inst_constants(InstInfo& I) {
    const double gam = 1.0 - 1.0 / std::sqrt(2.0);
    const double tau = gam * I.dt, dx = I.dx, lam = I.lam;
    I.tau = (float)tau;
    I.tdx = (float)(tau / dx);
    I.fq = (float)(tau / (2.0 * dx));
    I.Cc = (float)(tau * tau / (dx * dx));
    I.fd = (float)(lam * tau * tau / (dx * dx));
    I.lt2 = (float)(lam * tau * tau);
    I.ltau = (float)(lam * tau);
    I.lamf = (float)lam;
}

int hsgn_create_batched(int32_t count, const int64_t* n, const double* x_left,
                        const double* x_right, const double* lambda, double g, int32_t bc,
                        int32_t flags, hsgn_handle_t* out) {
    if (!out) return HSGN_ERR_INVALID_ARG;
    *out = nullptr;
    if (count < 1 || !n || !x_left || !x_right || !lambda) return HSGN_ERR_INVALID_ARG;
    if (bc != HSGN_BC_PERIODIC && bc != HSGN_BC_TRANSMISSIVE) return HSGN_ERR_INVALID_ARG;
    if (!(g > 0.0) || !std::isfinite(g)) return HSGN_ERR_INVALID_ARG;
    if (flags & ~(int32_t)(HSGN_RUSANOV_LOCAL | HSGN_MIXED | HSGN_EXACT_SOLVE))
        return HSGN_ERR_UNIMPLEMENTED;
    const bool windowed = !(flags & HSGN_EXACT_SOLVE);
    std::vector<InstInfo> info((size_t)count);
    std::vector<int32_t> binst;
    int64_t cells = 0;
    int64_t blocks = 0, vcap[kBV] = {0, 0, 0, 0};
    for (int32_t k = 0; k < count; ++k) {
        const int64_t nk = n[k];
        if (nk < 3 || (!windowed && nk > (int64_t)SEP_ROWS * AS) || nk > ((int64_t)1 << 31))
            return HSGN_ERR_INVALID_ARG;
        if (!(x_right[k] > x_left[k]) || !std::isfinite(x_left[k]) || !std::isfinite(x_right[k]))
            return HSGN_ERR_INVALID_ARG;
        if (!(lambda[k] >= 0.0) || !std::isfinite(lambda[k])) return HSGN_ERR_INVALID_ARG;
        InstInfo& I = info[(size_t)k];
        I.cell0 = cells;
        I.n = nk;
        I.blk0 = (int32_t)blocks;
        I.pad = 0;
        I.dx = (x_right[k] - x_left[k]) / (double)nk;
        I.lam = lambda[k];
        I.dt = 0.0;
        set_inst_constants(I);
        if (windowed) {
            // tiles of the windowed stage (set by assign_tiles below); the tile
            // tables hold every instance on either variant
            I.base = fused_tile_rows(nk, FusedGeom<FT, FM, FHW>::S, 1);
            I.P = (int32_t)((nk + I.base - 1) / I.base);
            I.rem = 0;
            for (int v = 1; v < kBV; ++v) vcap[v] += batch_variant_tiles(v, nk);
        } else {
            const BlockSplit s = make_split(nk, AS);
            I.base = s.base;
            I.P = s.P;
            I.rem = s.rem;
        }
        for (int32_t b = 0; b < I.P; ++b) binst.push_back(k);
        cells += nk;
        blocks += I.P;
    }
    hsgn_s* H = new (std::nothrow) hsgn_s;
    if (!H) return HSGN_ERR_OUT_OF_MEMORY;
    H->n = cells;
    H->bc = bc;
    H->flags = flags | HSGN_MIXED;
    H->mixed = true;
    H->batched = true;
    H->windowed = windowed;
    H->count = count;
    H->total_blocks = windowed ? 0 : blocks;
    H->total_tiles = windowed ? blocks : 0;
    H->g = g;
    H->lam = 0.0;
    H->dx = 0.0;
    H->inst_h = info;
    cudaGetDevice(&H->device);
    const size_t vec = align_up(cells * sizeof(double));
    const size_t fvec = align_up((cells + count) * sizeof(float));
    const size_t recb = windowed ? 0 : align_up(3 * cells * sizeof(float4));
    size_t total = (windowed ? 8 : 4) * vec + 4 * fvec + recb;
    if (!windowed)
        total += align_up(BLK_STRIDE * blocks * sizeof(float)) + align_up(blocks * sizeof(float));
    total += align_up(count * sizeof(InstInfo)) + align_up(blocks * sizeof(int32_t));
    if (windowed)
        for (int v = 1; v < kBV; ++v) total += align_up(vcap[v] * sizeof(int32_t));
    total += 4 * align_up(count * sizeof(double));
    total += align_up(8 * sizeof(double)) + align_up(sizeof(unsigned));
    if (cudaMalloc(&H->mem, total) != cudaSuccess) {
        cudaGetLastError();
        delete H;
        return HSGN_ERR_OUT_OF_MEMORY;
    }
    unsigned char* p = H->mem;
    auto take = [&](size_t bytes) {
        unsigned char* r = p;
        p += bytes;
        return r;
    };
    for (int k = 0; k < 4; ++k) H->U[k] = reinterpret_cast<double*>(take(vec));
    if (windowed)
        for (int k = 0; k < 4; ++k) H->V[k] = reinterpret_cast<double*>(take(vec));
    H->G1 = reinterpret_cast<float*>(take(fvec));
    H->dq1 = reinterpret_cast<float*>(take(fvec));
    H->dm1 = reinterpret_cast<float*>(take(fvec));
    H->dr1 = reinterpret_cast<float*>(take(fvec));
    if (!windowed) {
        H->mrec = reinterpret_cast<float4*>(take(recb));
        H->mblk = reinterpret_cast<float*>(take(align_up(BLK_STRIDE * blocks * sizeof(float))));
        H->ms_ = reinterpret_cast<float*>(take(align_up(blocks * sizeof(float))));
    }
    H->inst = reinterpret_cast<InstInfo*>(take(align_up(count * sizeof(InstInfo))));
    H->blk_inst = reinterpret_cast<int32_t*>(take(align_up(blocks * sizeof(int32_t))));
    if (windowed) {
        H->tile_inst = H->blk_inst;
        H->vtile[0] = H->blk_inst;
        for (int v = 1; v < kBV; ++v)
            H->vtile[v] = reinterpret_cast<int32_t*>(take(align_up(vcap[v] * sizeof(int32_t))));
    }
    H->speeds = reinterpret_cast<double*>(take(align_up(count * sizeof(double))));
    H->speeds_tmp = reinterpret_cast<double*>(take(2 * align_up(count * sizeof(double))));
    H->speeds_next = reinterpret_cast<double*>(take(align_up(count * sizeof(double))));
    H->spd = reinterpret_cast<double*>(take(align_up(8 * sizeof(double))));
    H->err = reinterpret_cast<unsigned*>(take(align_up(sizeof(unsigned))));
    cudaError_t e = cudaMemset(H->mem, 0, total);
    if (e == cudaSuccess)
        e = cudaMemcpy(H->inst, info.data(), count * sizeof(InstInfo), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(H->blk_inst, binst.data(), blocks * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = set_smem(k_mixed_assemble<XT, XM, BC_PERIODIC>, sizeof(MixedShared<XT, XM>));
    if (e == cudaSuccess)
        e = set_smem(k_mixed_assemble<XT, XM, BC_TRANSMISSIVE>, sizeof(MixedShared<XT, XM>));
    if (e == cudaSuccess)
        e = set_smem_fused<FT, BC_PERIODIC, false>();
    if (e == cudaSuccess) e = set_smem_fused<FT, BC_TRANSMISSIVE, false>();
    if (e == cudaSuccess) e = set_smem_fused<FTS, BC_PERIODIC, false>();
    if (e == cudaSuccess) e = set_smem_fused<FTS, BC_TRANSMISSIVE, false>();
    if (e == cudaSuccess) e = set_smem_fused<FT, BC_PERIODIC, false, FHWN>();
    if (e == cudaSuccess) e = set_smem_fused<FT, BC_TRANSMISSIVE, false, FHWN>();
    if (e == cudaSuccess) e = set_smem_fused<FTS, BC_PERIODIC, false, FHWN>();
    if (e == cudaSuccess) e = set_smem_fused<FTS, BC_TRANSMISSIVE, false, FHWN>();
    if (e == cudaSuccess && windowed) {
        // co-resident CTAs of each variant (the next-wave L2 prefetch)
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, H->device);
        if (e == cudaSuccess) e = batch_variant_slots<FT, FHW>(sms, H->vslots[0]);
        if (e == cudaSuccess) e = batch_variant_slots<FTS, FHW>(sms, H->vslots[1]);
        if (e == cudaSuccess) e = batch_variant_slots<FT, FHWN>(sms, H->vslots[2]);
        if (e == cudaSuccess) e = batch_variant_slots<FTS, FHWN>(sms, H->vslots[3]);
        H->tileSlots = H->vslots[0];
    }
    if (e == cudaSuccess && windowed) e = assign_tiles(H, std::vector<int8_t>((size_t)count, 0));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&H->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (H->cap) cudaStreamDestroy(H->cap);
        cudaFree(H->mem);
        delete H;
        return HSGN_ERR_CUDA;
    }
    *out = H;
    return HSGN_OK;
}

int hsgn_batched_set_dt(hsgn_handle_t H, const double* dt) {
    if (!H || !H->batched || !dt) return HSGN_ERR_INVALID_ARG;
    for (int32_t k = 0; k < H->count; ++k)
        if (!(dt[k] > 0.0) || !std::isfinite(dt[k])) return HSGN_ERR_INVALID_ARG;
    for (int32_t k = 0; k < H->count; ++k) {
        H->inst_h[(size_t)k].dt = dt[k];
        set_inst_constants(H->inst_h[(size_t)k]);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return HSGN_ERR_CUDA;
    if (cudaMemcpy(H->inst, H->inst_h.data(), H->count * sizeof(InstInfo), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return HSGN_ERR_CUDA;
    return HSGN_OK;
}

int hsgn_batched_suggest_dt(hsgn_handle_t H, double cfl, double mcfl, double* dt_out,
                            void* stream) {
    if (!H || !H->batched || !dt_out || !(cfl > 0.0)) return HSGN_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    const int32_t c = H->count;
    double* um = H->speeds_tmp;
    double* nm = H->speeds_tmp + align_up(c * sizeof(double)) / sizeof(double);
    if (H->windowed) {
        double* const* U = state(H);
        k_speeds_batched_df<<<(unsigned)c, 256, 0, st>>>(
            H->inst, reinterpret_cast<const float2*>(U[0]), reinterpret_cast<const float2*>(U[1]),
            reinterpret_cast<const float2*>(U[2]), H->g, um, nm, H->err);
    } else {
        k_speeds_batched<<<(unsigned)c, 256, 0, st>>>(H->inst, H->U[0], H->U[1], H->U[2], H->g, um,
                                                      nm, H->err);
    }
    if (cudaGetLastError() != cudaSuccess) return HSGN_ERR_CUDA;
    std::vector<double> hu((size_t)c), hn((size_t)c);
    if (cudaMemcpyAsync(hu.data(), um, c * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(hn.data(), nm, c * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return HSGN_ERR_CUDA;
    const int rc = read_error(H, st);
    if (rc != HSGN_OK) return rc;
    for (int32_t k = 0; k < c; ++k) {
        const double dx = H->inst_h[(size_t)k].dx;
        if (!(hn[(size_t)k] > 0.0)) return HSGN_ERR_INVALID_ARG;
        double dt = cfl * dx / hn[(size_t)k];
        if (mcfl > 0.0 && hu[(size_t)k] > 0.0 && hu[(size_t)k] * dt / dx > mcfl)
            dt = mcfl * dx / hu[(size_t)k];
        dt_out[k] = dt;
    }
    return HSGN_OK;
}

int hsgn_batched_set_tiles(hsgn_handle_t H, const int32_t* variant) {
    if (!H || !H->batched || !variant) return HSGN_ERR_INVALID_ARG;
    if (!H->windowed) return HSGN_ERR_UNIMPLEMENTED;
    std::vector<int8_t> var((size_t)H->count);
    for (int32_t k = 0; k < H->count; ++k) {
        if (variant[k] < 0 || variant[k] >= kBV) return HSGN_ERR_INVALID_ARG;
        var[(size_t)k] = (int8_t)variant[k];
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return HSGN_ERR_CUDA;
    return assign_tiles(H, var) == cudaSuccess ? HSGN_OK : HSGN_ERR_CUDA;
}

int hsgn_batched_get_tiles(hsgn_handle_t H, int32_t* variant_out) {
    if (!H || !H->batched || !variant_out) return HSGN_ERR_INVALID_ARG;
    if (!H->windowed) return HSGN_ERR_UNIMPLEMENTED;
    for (int32_t k = 0; k < H->count; ++k) variant_out[k] = H->variant[(size_t)k];
    return HSGN_OK;
}

// Autotuner of the batch's tiles: times `steps` steps from the current state
// (restored after every trial) with every instance on each batch variant in
// turn; a variant whose windows report HSGN_ERR_TRUNCATION for this batch (its
// overlap too narrow for the coupling) is ruled out. From the times a cost per
// tile of each variant (ms / tiles launched) assigns each instance the variant
// with the smallest predicted cost (tiles x cost per tile); that assignment is
// timed as well when it mixes variants. The fastest timed assignment stays.
int hsgn_batched_autotune(hsgn_handle_t H, int32_t steps, double* ms_out, int32_t* choice_out,
                          void* stream) {
    if (!H || !H->batched || steps < 1) return HSGN_ERR_INVALID_ARG;
    if (!H->windowed) return HSGN_ERR_UNIMPLEMENTED;
    for (int32_t k = 0; k < H->count; ++k)
        if (!(H->inst_h[(size_t)k].dt > 0.0)) return HSGN_ERR_INVALID_ARG;  // set_dt first
    cudaStream_t st = as_stream(stream);
    const int64_t n = H->n;
    // the state, kept as doubles (exact: the pairs carry 48 bits)
    double* keep = nullptr;
    if (cudaMalloc(&keep, 4 * n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return HSGN_ERR_OUT_OF_MEMORY;
    }
    double* kp[4] = {keep, keep + n, keep + 2 * n, keep + 3 * n};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = HSGN_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = HSGN_ERR_CUDA;
    if (rc == HSGN_OK) rc = hsgn_get_state(H, kp[0], kp[1], kp[2], kp[3], stream);
    const std::vector<int8_t> start = H->variant;
    const double nan = std::nan("");
    // one timed assignment; a truncation report rules it out (ms stays NaN)
    auto trial = [&](const std::vector<int8_t>& var, double& ms) -> int {
        ms = nan;
        if (cudaDeviceSynchronize() != cudaSuccess || assign_tiles(H, var) != cudaSuccess)
            return HSGN_ERR_CUDA;
        // two warm-up steps capture the graphs of both state buffers
        int r = hsgn_run(H, 0.0, 2, stream);
        if (r == HSGN_OK) r = hsgn_set_state(H, kp[0], kp[1], kp[2], kp[3], stream);
        if (r == HSGN_OK) {
            if (cudaEventRecord(e0, st) != cudaSuccess) return HSGN_ERR_CUDA;
            r = hsgn_enqueue(H, 0.0, steps, stream);
            if (r != HSGN_OK) return r;
            float t = 0.f;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
                return HSGN_ERR_CUDA;
            r = read_error(H, st);
            if (r == HSGN_OK) ms = (double)t / steps;
        }
        if (r != HSGN_OK && r != HSGN_ERR_TRUNCATION) return r;
        return hsgn_set_state(H, kp[0], kp[1], kp[2], kp[3], stream);
    };
    const size_t c = (size_t)H->count;
    double tv[kBV + 1] = {nan, nan, nan, nan, nan};
    std::vector<int8_t> vm(c, 0);
    int32_t choice = -1;
    for (int v = 0; v < kBV && rc == HSGN_OK; ++v) {
        rc = trial(std::vector<int8_t>(c, (int8_t)v), tv[v]);
        if (rc == HSGN_OK && !std::isnan(tv[v]) && (choice < 0 || tv[v] < tv[choice])) choice = v;
    }
    if (rc == HSGN_OK && choice < 0) rc = HSGN_ERR_TRUNCATION;  // no variant fits this batch
    if (rc == HSGN_OK) {
        double cost[kBV];
        for (int v = 0; v < kBV; ++v) {
            int64_t tiles = 0;
            for (size_t k = 0; k < c; ++k) tiles += batch_variant_tiles(v, H->inst_h[k].n);
            cost[v] = tv[v] / (double)tiles;
        }
        bool mixed = false;
        for (size_t k = 0; k < c; ++k) {
            const int64_t nk = H->inst_h[k].n;
            int best = choice;
            for (int v = 0; v < kBV; ++v)
                if (!std::isnan(cost[v]) &&
                    (double)batch_variant_tiles(v, nk) * cost[v] <
                        (double)batch_variant_tiles(best, nk) * cost[best])
                    best = v;
            vm[k] = (int8_t)best;
            mixed |= vm[k] != vm[0];
        }
        if (mixed) {
            rc = trial(vm, tv[kBV]);
            if (rc == HSGN_OK && !std::isnan(tv[kBV]) && tv[kBV] < tv[choice]) choice = kBV;
        }
    }
    if (rc == HSGN_OK) {
        if (cudaDeviceSynchronize() != cudaSuccess ||
            assign_tiles(H, choice == kBV ? vm : std::vector<int8_t>(c, (int8_t)choice)) !=
                cudaSuccess)
            rc = HSGN_ERR_CUDA;
    } else {
        cudaDeviceSynchronize();
        cudaGetLastError();
        assign_tiles(H, start);
    }
    if (ms_out)
        for (int v = 0; v <= kBV; ++v) ms_out[v] = tv[v];
    if (choice_out) *choice_out = choice;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(keep);
    return rc;
}

int hsgn_tridiag_workspace_bytes(int64_t n, size_t* bytes) {
    if (n < 1 || !bytes) return HSGN_ERR_INVALID_ARG;
    *bytes = align_up(sizeof(unsigned)) + rows_ws_bytes(n);
    return HSGN_OK;
}

int hsgn_tridiag_solve(int64_t n, int32_t periodic, const double* a, const double* b,
                       const double* c, const double* d, double* x, void* workspace,
                       size_t workspace_bytes, void* stream) {
    if (n < 1 || !a || !b || !c || !d || !x || !workspace) return HSGN_ERR_INVALID_ARG;
    size_t need = 0;
    hsgn_tridiag_workspace_bytes(n, &need);
    if (workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0)
        return HSGN_ERR_INVALID_ARG;
    cudaStream_t st = as_stream(stream);
    unsigned* err = reinterpret_cast<unsigned*>(workspace);
    unsigned char* ws = reinterpret_cast<unsigned char*>(workspace) + align_up(sizeof(unsigned));
    if (cudaMemsetAsync(err, 0, sizeof(unsigned), st) != cudaSuccess) return HSGN_ERR_CUDA;
    if (solve_rows(n, periodic ? 1 : 0, a, b, c, d, x, ws, err, nullptr, st) != cudaSuccess)
        return HSGN_ERR_CUDA;
    unsigned bits = 0;
    if (cudaMemcpyAsync(&bits, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return HSGN_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HSGN_ERR_CUDA;
    return map_error_bits(bits);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Arithmetic peaks of the device (hsgn_fma_peak): independent fused
// multiply-add chains, eight per thread, over every SM.
// ---------------------------------------------------------------------------
namespace {

constexpr int kPeakChains = 8;

__device__ __forceinline__ float peak_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double peak_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <class R>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, R b, R c, R* out) {
    R a[kPeakChains];
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) a[k] = (R)(threadIdx.x + k) * (R)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kPeakChains; ++k) a[k] = peak_fma(a[k], b, c);
    }
    R s = 0;
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) s += a[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

template <class R>
int fma_peak(double* tflops, cudaStream_t st) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<R>, 256, 0) !=
            cudaSuccess) {
        cudaGetLastError();
        return HSGN_ERR_CUDA;
    }
    const unsigned blocks = (unsigned)(sms * (per_sm > 0 ? per_sm : 1));
    // FP32 runs about 58 times as many operations per clock as FP64 on sm_103a:
    // each timed run takes some tens of milliseconds (launch ramps negligible)
    const int iters = sizeof(R) == 4 ? 1 << 18 : 1 << 14;
    R* out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    int rc = HSGN_OK;
    if (cudaMallocAsync(&out, (size_t)blocks * 256 * sizeof(R), st) != cudaSuccess ||
        cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        rc = HSGN_ERR_CUDA;
    } else {
        k_fma_peak<R><<<blocks, 256, 0, st>>>(iters / 8, (R)0.999, (R)1e-3, out);  // warm-up
        cudaEventRecord(a, st);
        k_fma_peak<R><<<blocks, 256, 0, st>>>(iters, (R)0.999, (R)1e-3, out);
        cudaEventRecord(b, st);
        float ms = 0.f;
        if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess ||
            !(ms > 0.f))
            rc = HSGN_ERR_CUDA;
        else
            *tflops = 2.0 * kPeakChains * (double)iters * blocks * 256 / (ms * 1e-3) / 1e12;
    }
    if (out) cudaFreeAsync(out, st);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = HSGN_ERR_CUDA;
    cudaGetLastError();
    return rc;
}

}  // namespace

extern "C" int hsgn_fma_peak(int32_t bits, double* tflops, void* stream) {
    if (!tflops || (bits != 32 && bits != 64)) return HSGN_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    return bits == 32 ? fma_peak<float>(tflops, st) : fma_peak<double>(tflops, st);
}

// ---------------------------------------------------------------------------
// No-allocation variant of the tridiagonal solve (declared in include/hsgn.h).
// The scratch is a file-scope device array; host code looks up its device
// address once per device (the array's name is only a host-side stand-in).
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoAllocMaxN = HSGN_TRIDIAG_NOALLOC_MAX_N;
// error word + the workspace of the recursive solve of the largest size
constexpr size_t kNoAllocBytes = kAlign + rows_ws_bytes(kNoAllocMaxN);
static_assert(kNoAllocBytes < (size_t)8 << 20, "fixed scratch must stay modest");
static_assert(kNoAllocBytes == HSGN_TRIDIAG_NOALLOC_SCRATCH_BYTES,
              "the size stated in hsgn.h must match the array");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on
// the first call per device).
int noalloc_scratch(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return HSGN_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return HSGN_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return HSGN_OK;
}

}  // namespace

extern "C" int hsgn_tridiag_solve_noalloc(int64_t n, int32_t periodic, const double* a,
                                          const double* b, const double* c, const double* d,
                                          double* x, void* stream) {
    if (n < 1 || n > kNoAllocMaxN || !a || !b || !c || !d || !x) return HSGN_ERR_INVALID_ARG;
    size_t need = 0;
    if (hsgn_tridiag_workspace_bytes(n, &need) != HSGN_OK || need > kNoAllocBytes)
        return HSGN_ERR_INVALID_ARG;
    void* ws = nullptr;
    const int rc = noalloc_scratch(&ws);
    if (rc != HSGN_OK) return rc;
    // same launch sequence as hsgn_tridiag_solve; it clears the error word first
    return hsgn_tridiag_solve(n, periodic, a, b, c, d, x, ws, kNoAllocBytes, stream);
}
