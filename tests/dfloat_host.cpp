// Host build of the double-float header for test_dfloat_cpu.py (compiled with -ffp-contract=off).
#include "dfloat.cuh"

extern "C" {
static void put(ck::df r, float *o) { o[0] = r.hi; o[1] = r.lo; }
void dfh_from_double(double d, float *o) { put(ck::df(d), o); }
void dfh_add(float ah, float al, float bh, float bl, float *o) { put(ck::df(ah, al) + ck::df(bh, bl), o); }
void dfh_sub(float ah, float al, float bh, float bl, float *o) { put(ck::df(ah, al) - ck::df(bh, bl), o); }
void dfh_mul(float ah, float al, float bh, float bl, float *o) { put(ck::df(ah, al) * ck::df(bh, bl), o); }
void dfh_mulf(float ah, float al, float b, float *o) { put(ck::df(ah, al) * b, o); }
void dfh_rcp(float ah, float al, float *o) { put(ck::rcp_nr(ck::df(ah, al)), o); }
void dfh_rsqrt(float ah, float al, float *o) { put(ck::rsqrt_nr(ck::df(ah, al)), o); }
}
