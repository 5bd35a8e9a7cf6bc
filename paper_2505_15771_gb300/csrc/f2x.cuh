// Double-float ("double-word") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with
// hi = RN(hi + lo), about 48 significant bits: FP64-class accuracy for the
// stage operator at FP32 issue rates (GB300 runs FP32 at roughly 60x its
// FP64 rate).  The building blocks are the error-free transforms
//   TwoSum   (Knuth, TAOCP vol. 2): s + t = a + b exactly,
//   Fast2Sum (Dekker 1971): the same for |a| >= |b|,
//   TwoProd  with FMA: p + e = a * b exactly,
// and the double-word operations analysed by Joldes, Muller and Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic", ACM TOMS 44(2), 2017:
//   add: SloppyDWPlusDW (TwoSum of the high parts, plain sum of the low
//        parts);
//   mul: DWTimesDW with FMA (the xl * yl term dropped);
//   fma: the DWTimesDW product added as in add;
//   div: one Newton-style correction of the FP32 quotient (Dekker 1971).
// Results are left unnormalised: the final Fast2Sum of those algorithms is
// deferred to norm(), which the kernels apply where a value is stored.  An
// unnormalised pair is still the exact sum hi + lo with |lo| of the order of
// u |operands| (u = 2^-24), so every later operation keeps its absolute error
// at O(u^2) times the magnitudes involved, as with renormalised pairs; the
// saving is three instructions per operation and a shorter dependency chain
// through each accumulator.  No step relies on FMA contraction of a separate
// multiply and add: where the exact product error is needed the FMA is
// explicit.  Nor may the compiler contract one (nvcc does by default, and a
// product fused into the TwoSum that follows it breaks the error-free
// transformation, leaving FP32-level errors): every rounded sum, difference
// and product here is an __f*_rn intrinsic, which is never contracted.  The
// type is a plain pair so that arrays of it have the layout of FP64 arrays
// (8 bytes a value).
#pragma once

#include <cuda_runtime.h>

#include "hho_internal.h"

__device__ __forceinline__ f2x f2x_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    return f2x{s, __fsub_rn(b, z)};
}

__device__ __forceinline__ f2x f2x_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float ap = __fsub_rn(s, b);
    const float bp = __fsub_rn(s, ap);
    return f2x{s, __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp))};
}

__device__ __forceinline__ f2x operator+(f2x x, f2x y) {
    const f2x s = f2x_two_sum(x.hi, y.hi);
    const float w = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return f2x{s.hi, w};
}
__device__ __forceinline__ f2x operator-(f2x x) { return f2x{-x.hi, -x.lo}; }
__device__ __forceinline__ f2x operator-(f2x x, f2x y) { return x + (-y); }
__device__ __forceinline__ f2x& operator+=(f2x& x, f2x y) { return x = x + y; }
__device__ __forceinline__ f2x& operator-=(f2x& x, f2x y) { return x = x - y; }

__device__ __forceinline__ f2x operator*(f2x x, f2x y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return f2x{p, e};
}

// x * y + z
__device__ __forceinline__ f2x fma(f2x x, f2x y, f2x z) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    const f2x s = f2x_two_sum(p, z.hi);
    const float w = __fadd_rn(s.lo, __fadd_rn(e, z.lo));
    return f2x{s.hi, w};
}

// c * x and c * x + z for an FP32 constant c (the exact small integers of
// the polynomial derivatives)
__device__ __forceinline__ f2x mulc(float c, f2x x) {
    const float p = __fmul_rn(c, x.hi);
    float e = fmaf(c, x.hi, -p);
    e = fmaf(c, x.lo, e);
    return f2x{p, e};
}
__device__ __forceinline__ f2x fmac(float c, f2x x, f2x z) {
    const float p = __fmul_rn(c, x.hi);
    float e = fmaf(c, x.hi, -p);
    e = fmaf(c, x.lo, e);
    const f2x s = f2x_two_sum(p, z.hi);
    const float w = __fadd_rn(s.lo, __fadd_rn(e, z.lo));
    return f2x{s.hi, w};
}

__device__ __forceinline__ f2x operator/(f2x x, f2x y) {
    y = f2x_fast_two_sum(y.hi, y.lo);
    const float q = __fdiv_rn(x.hi, y.hi);
    const f2x r = x - mulc(q, y);
    return f2x_fast_two_sum(q, __fdiv_rn(__fadd_rn(r.hi, r.lo), y.hi));
}

// Read-only load of a pair (one 8-byte load).
__device__ __forceinline__ f2x __ldg(const f2x* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return f2x(v.x, v.y);
}

// Renormalised pair (hi = RN(hi + lo)), applied where a value is stored.
__device__ __forceinline__ f2x norm(f2x x) { return f2x_fast_two_sum(x.hi, x.lo); }

// Scalar helpers shared by the FP64, FP32 and double-float instantiations.
__device__ __forceinline__ double norm(double x) { return x; }
__device__ __forceinline__ float norm(float x) { return x; }
__device__ __forceinline__ double mulc(float c, double x) { return (double)c * x; }
__device__ __forceinline__ float mulc(float c, float x) { return c * x; }
__device__ __forceinline__ double fmac(float c, double x, double z) { return fma((double)c, x, z); }
__device__ __forceinline__ float fmac(float c, float x, float z) { return fmaf(c, x, z); }
