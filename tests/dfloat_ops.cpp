// Host build of the double-float operations of the FP64-class stage
// (paper_2510_07539_gb300/csrc/hsgn_dfloat.cuh), exported with plain float
// arguments so that a test can compare them with exact rational arithmetic.
// Built with -ffp-contract=off: the header spells every rounding explicitly and
// the host build must not fuse a*b + c behind its back.
#include "../paper_2510_07539_gb300/csrc/hsgn_dfloat.cuh"

using hsgn::dfl;

namespace {
inline void out2(dfl r, float* o) {
    o[0] = r.hi;
    o[1] = r.lo;
}
}  // namespace

extern "C" {
void dfo_add(float ah, float al, float bh, float bl, float* o) { out2(dfl(ah, al) + dfl(bh, bl), o); }
void dfo_add_u(float ah, float al, float bh, float bl, float* o) {
    out2(hsgn::add_u(dfl(ah, al), dfl(bh, bl)), o);
}
void dfo_add_acc(float ah, float al, float bh, float bl, float* o) {
    out2(hsgn::add_acc(dfl(ah, al), dfl(bh, bl)), o);
}
void dfo_add_f(float ah, float al, float x, float* o) { out2(hsgn::add_f(dfl(ah, al), x), o); }
void dfo_mul(float ah, float al, float bh, float bl, float* o) { out2(dfl(ah, al) * dfl(bh, bl), o); }
void dfo_mul_f(float ah, float al, float x, float* o) { out2(hsgn::mul_f(dfl(ah, al), x), o); }
void dfo_fma(float ah, float al, float bh, float bl, float ch, float cl, float* o) {
    out2(hsgn::fma(dfl(ah, al), dfl(bh, bl), dfl(ch, cl)), o);
}
void dfo_fma_u(float ah, float al, float bh, float bl, float ch, float cl, float* o) {
    out2(hsgn::fma_u(dfl(ah, al), dfl(bh, bl), dfl(ch, cl)), o);
}
void dfo_rcp(float ah, float al, float* o) { out2(hsgn::rcp(dfl(ah, al)), o); }
void dfo_div(float ah, float al, float bh, float bl, float* o) { out2(dfl(ah, al) / dfl(bh, bl), o); }
void dfo_sq_minus(float hh, float hl, float mh, float ml, float* o) {
    out2(hsgn::sq_minus(dfl(hh, hl), dfl(mh, ml)), o);
}
void dfo_of(double x, float* o) { out2(hsgn::dfl_of(x), o); }
}
