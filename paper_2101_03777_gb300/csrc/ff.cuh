// Float-float ("double-FP32") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi)/2, about 48 significant bits.  The building blocks are the
// error-free transformations of Knuth (TwoSum), Dekker (FastTwoSum) and the
// FMA form of Dekker's TwoProduct; sums of products follow the compensated
// dot product Dot2 of Ogita, Rump and Oishi ("Accurate sum and dot product",
// SIAM J. Sci. Comput. 26, 2005), whose result is as accurate as if it were
// computed in twice the working precision and then rounded.
//
// GB300 issues FP64 at a small fraction of its FP32 rate, so the inner Krylov
// iteration runs in this format: the same 8 bytes per value as FP64 in
// memory, but every arithmetic instruction on the FP32 pipes.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace crhyb {

// a + b = s + e exactly (any magnitudes)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// a + b = s + e exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// a * b = p + e exactly (barring underflow)
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Accumulator of a sum of products: s + c, where c gathers the rounding
// errors of the running sum and of the products (Dot2).
struct FFAcc {
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    // += (ah + al) * (bh + bl), the al*bl term (below 2^-48 relative) dropped
    __device__ __forceinline__ void mad(float ah, float al, float bh, float bl) {
        float p, e, t;
        two_prod(ah, bh, p, e);
        e = __fmaf_rn(ah, bl, e);
        e = __fmaf_rn(al, bh, e);
        two_sum(s, p, s, t);
        c = __fadd_rn(c, __fadd_rn(t, e));
    }
    // += a * (bh + bl) with a plain FP32 a
    __device__ __forceinline__ void mad1(float a, float bh, float bl) {
        float p, e, t;
        two_prod(a, bh, p, e);
        e = __fmaf_rn(a, bl, e);
        two_sum(s, p, s, t);
        c = __fadd_rn(c, __fadd_rn(t, e));
    }
    // += (bh + bl)
    __device__ __forceinline__ void add(float bh, float bl) {
        float t;
        two_sum(s, bh, s, t);
        c = __fadd_rn(c, __fadd_rn(t, bl));
    }
    // normalised result
    __device__ __forceinline__ float2 result() const {
        float h, l;
        fast_two_sum(s, c, h, l);
        return make_float2(h, l);
    }
};

// a + b (float-float, accurate addition: both halves are added error free)
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    float s, e, t, f;
    two_sum(a.x, b.x, s, e);
    two_sum(a.y, b.y, t, f);
    e = __fadd_rn(e, t);
    fast_two_sum(s, e, s, e);
    e = __fadd_rn(e, f);
    fast_two_sum(s, e, s, e);
    return make_float2(s, e);
}

// a * b (float-float)
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
    float p, e;
    two_prod(a.x, b.x, p, e);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    fast_two_sum(p, e, p, e);
    return make_float2(p, e);
}

// a * b for a plain FP32 a
__device__ __forceinline__ float2 ff_mul1(float a, float2 b) {
    float p, e;
    two_prod(a, b.x, p, e);
    e = __fmaf_rn(a, b.y, e);
    fast_two_sum(p, e, p, e);
    return make_float2(p, e);
}

// a * b + c (float-float)
__device__ __forceinline__ float2 ff_fma(float2 a, float2 b, float2 c) { return ff_add(ff_mul(a, b), c); }

__device__ __forceinline__ float2 ff_neg(float2 a) { return make_float2(-a.x, -a.y); }

// FP64 <-> float-float (used outside the iteration only: these convert on the FP64 unit)
__device__ __forceinline__ float2 ff_from_double(double v) {
    const float h = __double2float_rn(v);
    const float l = __double2float_rn(v - double(h));
    return make_float2(h, l);
}
__device__ __forceinline__ double ff_to_double(float2 a) { return double(a.x) + double(a.y); }

// the low part of a matrix value, FP32 or BF16
__device__ __forceinline__ float lo_val(const float* p) { return __ldcs(p); }
__device__ __forceinline__ float lo_val(const __nv_bfloat16* p) {
    const unsigned short u = __ldcs(reinterpret_cast<const unsigned short*>(p));
    return __uint_as_float(unsigned(u) << 16);
}

// (hi, lo) of matrix value idx: an interleaved float-float pair (one 8-byte load;
// vh unused), or an FP32 high plane with a BF16 low plane
__device__ __forceinline__ void hl_val(const float* vh, const float2* vl, size_t idx, float& h, float& l) {
    const float2 v = __ldcs(vl + idx);
    h = v.x;
    l = v.y;
}
__device__ __forceinline__ void hl_val(const float* vh, const __nv_bfloat16* vl, size_t idx, float& h, float& l) {
    h = __ldcs(vh + idx);
    l = lo_val(vl + idx);
}

}  // namespace crhyb
