// Arithmetic policies of the on-chip stencil steppers: FP32, FP64 and
// float-float (an unevaluated sum hi + lo of two FP32 values, about 48
// significant bits, evaluated on the FP32 pipe).
//
// Float-float uses the error-free transformations of Knuth (TwoSum) and
// Dekker (FastTwoSum), and the FMA form of the exact product error; the
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
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return ff{s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = a + b;
    const float e = b - (s - a);
    return ff{s, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = a.hi * b.hi;
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

// ------------------------------------------------------------------ policies
// V: value type; the stage update is w = u + cc * (vn + vs + vw + ve - 4 vc).
template <class V>
struct Arith;

template <>
struct Arith<float> {
    static constexpr bool kUInSmem = false;
    __device__ static float from_d(double x) { return (float)x; }
    __device__ static double to_d(float v) { return (double)v; }
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

template <>
struct Arith<ff> {
    static constexpr bool kUInSmem = true;
    __device__ static ff from_d(double x) { return ff_from_double(x); }
    __device__ static double to_d(ff v) { return ff_to_double(v); }
    __device__ static ff zero() { return ff{0.f, 0.f}; }
    __device__ static ff sel(bool c, ff a, ff b) { return ff{c ? a.hi : b.hi, c ? a.lo : b.lo}; }
    __device__ static ff stage(ff vn, ff vs, ff vw, ff ve, ff vc, ff u, ff cc) {
        const ff t = ff_add(ff_add(vn, vs), ff_add(vw, ve));
        const ff l = ff_add(t, ff{-4.f * vc.hi, -4.f * vc.lo});   // exact scaling by -4
        return ff_add(u, ff_mul(cc, l));
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
