// Arithmetic policies of the on-chip stencil steppers: FP32, FP64 and
// float-float (an unevaluated sum hi + lo of two FP32 values, about 48
// significant bits, evaluated on the FP32 pipe).
//
// Float-float uses the error-free transformations of Knuth (TwoSum) and
// Dekker (FastTwoSum), and the FMA form of the exact product error.  Their
// additions and products use the __fadd_rn / __fsub_rn / __fmul_rn
// intrinsics, which the compiler never contracts into FMAs (a contracted
// s = a + b*c would break the error-free property); the
// addition is the "sloppy" double-single sum (one TwoSum on the high parts,
// the low parts added, one FastTwoSum to renormalise), whose error is bounded
// by a small multiple of 2^-44 (|a| + |b|).
#pragma once

#include <cuda_runtime.h>

namespace pit {

constexpr unsigned kFullMask = 0xffffffffu;

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff{s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return ff{s, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ ff ff_from_double(double x) {
    const float h = (float)x;
    return ff{h, (float)(x - (double)h)};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// ------------------------------------------------------- FP64 <-> FP32
// Conversions between binary64 and binary32 done with integer operations,
// written from the IEEE-754 formats.  On GB300 the hardware conversion runs
// on the FP64 pipe (2 lanes per clock per SM), where a conversion per point
// per slice costs about a tenth of an FP32 stencil kernel; the integer pipe
// is 32x wider.  Normal-range values take the integer path and round to
// nearest even exactly like the hardware conversion; zeros, subnormal
// results, infinities and NaNs take the (rare) hardware path.
__device__ __forceinline__ float d2f_rn(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const int fe = (int)((hi >> 20) & 0x7ffu) - 896;     // binary32 biased exponent
    if (fe <= 0 || fe >= 255) return __double2float_rn(x);
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // top 23 mantissa bits
    const unsigned rem = lo & 0x1fffffffu;                   // 29 discarded bits
    unsigned r = (hi & 0x80000000u) | ((unsigned)fe << 23) | m;
    r += (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;  // carry may reach the exponent: still exact
    return __uint_as_float(r);
}

__device__ __forceinline__ double f2d(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)f;
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
    const unsigned lo = (u & 7u) << 29;
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

// ------------------------------------------------------------------ policies
// V: value type; the stage update is w = u + cc * (vn + vs + vw + ve - 4 vc).
template <class V>
struct Arith;

template <>
struct Arith<float> {
    static constexpr bool kUInSmem = false;
    __device__ static float from_d(double x) { return d2f_rn(x); }
    __device__ static double to_d(float v) { return f2d(v); }
    __device__ static float zero() { return 0.f; }
    __device__ static float sel(bool c, float a, float b) { return c ? a : b; }
    __device__ static float stage(float vn, float vs, float vw, float ve, float vc, float u,
                                  float cc) {
        return fmaf(cc, fmaf(-4.f, vc, (vn + vs) + (vw + ve)), u);
    }
    __device__ static float shfl_up(float v) { return __shfl_up_sync(kFullMask, v, 1); }
    __device__ static float shfl_down(float v) { return __shfl_down_sync(kFullMask, v, 1); }
    // four consecutive values to / from 16-byte aligned shared memory
    __device__ static void st4(float *p, const float (&v)[4]) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    __device__ static void ld4(const float *p, float (&v)[4]) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    }
};

template <>
struct Arith<double> {
    static constexpr bool kUInSmem = true;
    __device__ static double from_d(double x) { return x; }
    __device__ static double to_d(double v) { return v; }
    __device__ static double zero() { return 0.0; }
    __device__ static double sel(bool c, double a, double b) { return c ? a : b; }
    __device__ static double stage(double vn, double vs, double vw, double ve, double vc,
                                   double u, double cc) {
        return fma(cc, fma(-4.0, vc, (vn + vs) + (vw + ve)), u);
    }
    __device__ static double shfl_up(double v) { return __shfl_up_sync(kFullMask, v, 1); }
    __device__ static double shfl_down(double v) { return __shfl_down_sync(kFullMask, v, 1); }
    __device__ static void st4(double *p, const double (&v)[4]) {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    }
    __device__ static void ld4(const double *p, double (&v)[4]) {
        const double2 a = reinterpret_cast<const double2 *>(p)[0];
        const double2 b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = a.x;
        v[1] = a.y;
        v[2] = b.x;
        v[3] = b.y;
    }
};

// ----------------------------------------------------- packed float-float
// Two points per instruction: the same operations as Arith<ff>::stage, each
// on an f32x2 pair (__fadd2_rn, __fmul2_rn, __ffma2_rn round each lane to
// nearest like their scalar forms; a - b is the exact-product FMA
// b * (-1) + a), so a packed stage gives the scalar stage's results bit for
// bit while issuing half the FP32 instructions.
struct ff2 {
    float2 hi, lo;
};

__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e) {
    s = __fadd2_rn(a, b);
    const float2 bb = f2_sub(s, a);
    e = __fadd2_rn(f2_sub(a, f2_sub(s, bb)), f2_sub(b, bb));
}

// two float-float values as the lanes of a packed pair
__device__ __forceinline__ ff2 ff_pair(const ff &a, const ff &b) {
    return ff2{make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)};
}

// {a.hi, b.hi, a.lo, b.lo}: one 16-byte record per pair
__device__ __forceinline__ float4 ff_pack_pair(const ff &a, const ff &b) {
    return make_float4(a.hi, b.hi, a.lo, b.lo);
}

// w = u + cc (vn + vs + vw + ve - 4 vc) for two points, cc = (cch, ccl),
// ncch = -cch.  Same scheme as Arith<ff>::stage in 44 FP32 operations:
// the fourth TwoSum takes its operand -4 vc.hi as exact FMA products
// (no separate multiply), the product error term starts from -p (no
// negation), and the result is left unnormalised -- w.hi is the TwoSum of
// u.hi and p, w.lo collects the rest, a few ulp of w.hi at most -- which
// costs nothing in accuracy because every low part is summed in FP32 next
// to exact sums of the high parts; ff_renorm2 restores |lo| <= ulp(hi)/2
// once per time step.
__device__ __forceinline__ ff2 ff_stage2(const ff2 &vn, const ff2 &vs, const ff2 &vw,
                                         const ff2 &ve, const ff2 &vc, const ff2 &u,
                                         float2 cch, float2 ncch, float2 ccl) {
    const float2 m4 = make_float2(-4.f, -4.f);
    float2 ah, al, bh, bl, ch, cl;
    two_sum2(vn.hi, vs.hi, ah, al);
    two_sum2(vw.hi, ve.hi, bh, bl);
    two_sum2(ah, bh, ch, cl);
    // TwoSum(ch, -4 vc.hi): s = dh, -bb = ch - dh, e = (ch - (s - bb)) + (b - bb)
    const float2 dh = __ffma2_rn(m4, vc.hi, ch);
    const float2 nbb = f2_sub(ch, dh);
    const float2 dl = __fadd2_rn(f2_sub(ch, __fadd2_rn(dh, nbb)), __ffma2_rn(m4, vc.hi, nbb));
    const float2 lo = __ffma2_rn(
        m4, vc.lo,
        __fadd2_rn(__fadd2_rn(__fadd2_rn(al, bl), __fadd2_rn(cl, dl)),
                   __fadd2_rn(__fadd2_rn(vn.lo, vs.lo), __fadd2_rn(vw.lo, ve.lo))));
    const float2 pn = __fmul2_rn(ncch, dh);      // -p, p = cch dh
    float2 e = __ffma2_rn(cch, dh, pn);          // p's rounding error, exact
    e = __ffma2_rn(cch, lo, e);
    e = __ffma2_rn(ccl, dh, e);
    // TwoSum(u.hi, p) with p = -pn
    const float2 sh = f2_sub(u.hi, pn);
    const float2 nb2 = f2_sub(u.hi, sh);
    const float2 sl = __fadd2_rn(f2_sub(u.hi, __fadd2_rn(sh, nb2)), f2_sub(nb2, pn));
    ff2 w;
    w.hi = sh;
    w.lo = __fadd2_rn(sl, __fadd2_rn(u.lo, e));
    return w;
}

// ff_stage2 that also returns -fl(cc.hi * dh), the negated FP32 rounding of
// the first-order term cc * (vn + vs + vw + ve - 4 vc) it adds to u (the
// split RK4 step continues from it in FP32); the same operations otherwise.
__device__ __forceinline__ ff2 ff_stage2_neg_w(const ff2 &vn, const ff2 &vs, const ff2 &vw,
                                               const ff2 &ve, const ff2 &vc, const ff2 &u,
                                               float2 cch, float2 ncch, float2 ccl,
                                               float2 &neg_w) {
    const float2 m4 = make_float2(-4.f, -4.f);
    float2 ah, al, bh, bl, ch, cl;
    two_sum2(vn.hi, vs.hi, ah, al);
    two_sum2(vw.hi, ve.hi, bh, bl);
    two_sum2(ah, bh, ch, cl);
    const float2 dh = __ffma2_rn(m4, vc.hi, ch);
    const float2 nbb = f2_sub(ch, dh);
    const float2 dl = __fadd2_rn(f2_sub(ch, __fadd2_rn(dh, nbb)), __ffma2_rn(m4, vc.hi, nbb));
    const float2 lo = __ffma2_rn(
        m4, vc.lo,
        __fadd2_rn(__fadd2_rn(__fadd2_rn(al, bl), __fadd2_rn(cl, dl)),
                   __fadd2_rn(__fadd2_rn(vn.lo, vs.lo), __fadd2_rn(vw.lo, ve.lo))));
    const float2 pn = __fmul2_rn(ncch, dh);
    float2 e = __ffma2_rn(cch, dh, pn);
    e = __ffma2_rn(cch, lo, e);
    e = __ffma2_rn(ccl, dh, e);
    const float2 sh = f2_sub(u.hi, pn);
    const float2 nb2 = f2_sub(u.hi, sh);
    const float2 sl = __fadd2_rn(f2_sub(u.hi, __fadd2_rn(sh, nb2)), f2_sub(nb2, pn));
    neg_w = pn;
    ff2 w;
    w.hi = sh;
    w.lo = __fadd2_rn(sl, __fadd2_rn(u.lo, e));
    return w;
}

// ff_stage2_neg_w from the neighbours' high words alone: the exact sum of
// the high words times cc in float-float, added to the float-float centre u;
// the low words' stencil is left out (the split RK4 step applies cc to the
// centre's low word with its FP32 terms instead).  39 FP32 operations per
// point, 5 fewer than ff_stage2_neg_w.
__device__ __forceinline__ ff2 ff_stage2_neg_w_hi(float2 vn, float2 vs, float2 vw, float2 ve, const ff2 &u,
                                                  float2 cch, float2 ncch, float2 ccl, float2 &neg_w) {
    const float2 m4 = make_float2(-4.f, -4.f);
    float2 ah, al, bh, bl, ch, cl;
    two_sum2(vn, vs, ah, al);
    two_sum2(vw, ve, bh, bl);
    two_sum2(ah, bh, ch, cl);
    const float2 dh = __ffma2_rn(m4, u.hi, ch);
    const float2 nbb = f2_sub(ch, dh);
    const float2 dl = __fadd2_rn(f2_sub(ch, __fadd2_rn(dh, nbb)), __ffma2_rn(m4, u.hi, nbb));
    const float2 lo = __fadd2_rn(__fadd2_rn(al, bl), __fadd2_rn(cl, dl));
    const float2 pn = __fmul2_rn(ncch, dh);      // -p, p = cch dh
    float2 e = __ffma2_rn(cch, dh, pn);          // p's rounding error, exact
    e = __ffma2_rn(cch, lo, e);
    e = __ffma2_rn(ccl, dh, e);
    // TwoSum(u.hi, p) with p = -pn
    const float2 sh = f2_sub(u.hi, pn);
    const float2 nb2 = f2_sub(u.hi, sh);
    const float2 sl = __fadd2_rn(f2_sub(u.hi, __fadd2_rn(sh, nb2)), f2_sub(nb2, pn));
    neg_w = pn;
    ff2 w;
    w.hi = sh;
    w.lo = __fadd2_rn(sl, __fadd2_rn(u.lo, e));
    return w;
}

// s + q for two float-float values s and FP32 values q given negated
// (nq = -q): TwoSum of the high parts, the low part added, FastTwoSum
// renormalisation.  10 FP32 operations per point.
__device__ __forceinline__ ff2 ff_add_neg_f32_2(const ff2 &s, float2 nq) {
    const float2 h = f2_sub(s.hi, nq);
    const float2 bb = f2_sub(h, s.hi);                 // the -q actually added
    const float2 e = f2_sub(f2_sub(s.hi, f2_sub(h, bb)), __fadd2_rn(nq, bb));
    const float2 lo = __fadd2_rn(e, s.lo);
    ff2 w;
    w.hi = __fadd2_rn(h, lo);
    w.lo = f2_sub(lo, f2_sub(w.hi, h));
    return w;
}

// FastTwoSum renormalisation of two float-float values (|lo| <= a few ulp(hi))
__device__ __forceinline__ ff2 ff_renorm2(const ff2 &v) {
    ff2 w;
    w.hi = __fadd2_rn(v.hi, v.lo);
    w.lo = f2_sub(v.lo, f2_sub(w.hi, v.hi));
    return w;
}

template <>
struct Arith<ff> {
    static constexpr bool kUInSmem = true;
    __device__ static ff from_d(double x) { return ff_from_double(x); }
    __device__ static double to_d(ff v) { return ff_to_double(v); }
    __device__ static ff zero() { return ff{0.f, 0.f}; }
    __device__ static ff sel(bool c, ff a, ff b) { return ff{c ? a.hi : b.hi, c ? a.lo : b.lo}; }
    // w = u + cc (vn + vs + vw + ve - 4 vc): the high parts are summed with
    // exact TwoSums; their rounding errors and all low parts (each about
    // 2^-24 of the values) are summed in FP32, which costs about 2^-48 of
    // the values; the product with cc keeps its exact FMA error term; one
    // renormalisation at the end.  48 FP32 operations.
    __device__ static ff stage(ff vn, ff vs, ff vw, ff ve, ff vc, ff u, ff cc) {
        const ff a = two_sum(vn.hi, vs.hi);
        const ff b = two_sum(vw.hi, ve.hi);
        const ff c = two_sum(a.hi, b.hi);
        const ff d = two_sum(c.hi, __fmul_rn(-4.f, vc.hi));   // exact scaling by -4
        const float lo = fmaf(-4.f, vc.lo, ((a.lo + b.lo) + (c.lo + d.lo)) +
                                              ((vn.lo + vs.lo) + (vw.lo + ve.lo)));
        const float p = __fmul_rn(cc.hi, d.hi);
        float e = fmaf(cc.hi, d.hi, -p);
        e = fmaf(cc.hi, lo, e);
        e = fmaf(cc.lo, d.hi, e);
        const ff s = two_sum(u.hi, p);
        return fast_two_sum(s.hi, s.lo + (u.lo + e));
    }
    __device__ static ff shfl_up(ff v) {
        return ff{__shfl_up_sync(kFullMask, v.hi, 1), __shfl_up_sync(kFullMask, v.lo, 1)};
    }
    __device__ static ff shfl_down(ff v) {
        return ff{__shfl_down_sync(kFullMask, v.hi, 1), __shfl_down_sync(kFullMask, v.lo, 1)};
    }
    __device__ static void st4(ff *p, const ff (&v)[4]) {
        float4 *q = reinterpret_cast<float4 *>(p);
        q[0] = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
        q[1] = make_float4(v[2].hi, v[2].lo, v[3].hi, v[3].lo);
    }
    __device__ static void ld4(const ff *p, ff (&v)[4]) {
        const float4 a = reinterpret_cast<const float4 *>(p)[0];
        const float4 b = reinterpret_cast<const float4 *>(p)[1];
        v[0] = ff{a.x, a.y};
        v[1] = ff{a.z, a.w};
        v[2] = ff{b.x, b.y};
        v[3] = ff{b.z, b.w};
    }
};

}  // namespace pit
