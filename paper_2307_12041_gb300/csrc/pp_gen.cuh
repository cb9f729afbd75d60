// Arithmetic for the basis generators of the tensor-core path: packed FP32
// pairs (fma/mul/add .f32x2, two lanes of work per issue slot) and a phase
// evaluation e^{i pi m s} for a fixed-point phase coefficient s.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace pp {
namespace gen {

// ---- packed FP32 pairs ------------------------------------------------------
// Built on the float2 builtins (__ffma2_rn and friends), which the compiler
// keeps as single packed instructions on register pairs.
struct f2 {
    float2 v;
};
__device__ __forceinline__ f2 pk(float a, float b) { return f2{make_float2(a, b)}; }
__device__ __forceinline__ void upk(f2 a, float &x, float &y) {
    x = a.v.x;
    y = a.v.y;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return f2{__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return f2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return f2{__fadd2_rn(a.v, b.v)}; }

// Two complex numbers held as packed real parts and packed imaginary parts.
struct c2 {
    f2 re, im;
};
// Two independent rotations z <- z * e, e given with its negated imaginary part.
struct rot2_step {
    f2 re, im, nim;
};
__device__ __forceinline__ rot2_step make_step(float2 e0, float2 e1) {
    rot2_step s;
    s.re = pk(e0.x, e1.x);
    s.im = pk(e0.y, e1.y);
    s.nim = pk(-e0.y, -e1.y);
    return s;
}
__device__ __forceinline__ c2 make_c2(float2 z0, float2 z1) {
    c2 z;
    z.re = pk(z0.x, z1.x);
    z.im = pk(z0.y, z1.y);
    return z;
}
__device__ __forceinline__ c2 rot2(c2 z, const rot2_step &e) {
    c2 r;
    r.re = fma2(z.re, e.re, mul2(z.im, e.nim));
    r.im = fma2(z.im, e.re, mul2(z.re, e.im));
    return r;
}

// ---- phase evaluation -------------------------------------------------------
// e^{i pi m s} = (cos, sin)(pi m s) for integer m and s held as (s mod 2) * 2^62.
// m s mod 2 is exact in 64-bit integers; the phase is reduced to the nearest
// quarter turn k and a remainder x in [-1/4, 1/4] half-turns, and sin, cos of
// y = pi x (|y| <= pi/4) come from their Taylor series to y^9 and y^10
// (truncation below 2e-9 relative), then the quarter turn is applied.
__device__ __forceinline__ float2 phase_poly(unsigned long long m, unsigned long long s) {
    const unsigned long long p = (m * s) & 0x7FFFFFFFFFFFFFFFull;   // [0, 2) half-turns, 2^-62 units
    const unsigned long long kk = (p + (1ull << 60)) >> 61;           // 0..4 quarter turns
    const long long r = (long long)(p - (kk << 61));                 // [-2^60, 2^60)
    const float x = (float)(int)(r >> 32) * 0x1p-30f;                 // half-turns
    const float y = x * 3.14159265358979f;
    const float z = y * y;
    float sp = fmaf(z, 2.75573192e-6f, -1.98412698e-4f);              //  1/9!, -1/7!
    sp = fmaf(z, sp, 8.33333333e-3f);                                 //  1/5!
    sp = fmaf(z, sp, -1.66666667e-1f);                                // -1/3!
    const float sn = fmaf(y * z, sp, y);
    float cp = fmaf(z, -2.75573192e-7f, 2.48015873e-5f);              // -1/10!, 1/8!
    cp = fmaf(z, cp, -1.38888889e-3f);                                // -1/6!
    cp = fmaf(z, cp, 4.16666667e-2f);                                 //  1/4!
    cp = fmaf(z, cp, -0.5f);                                          // -1/2!
    const float cs = fmaf(z, cp, 1.0f);
    const unsigned k = (unsigned)kk & 3u;
    const float c_ = (k & 1u) ? sn : cs;
    const float s_ = (k & 1u) ? cs : sn;
    // k = 0: ( c,  s); 1: (-s,  c); 2: (-c, -s); 3: ( s, -c)
    return make_float2((k == 1u || k == 2u) ? -c_ : c_, (k >= 2u) ? -s_ : s_);
}

// e^{i pi m s} from the hardware sine and cosine (__sincosf: absolute error at most
// 2^-21.4 for arguments in [-pi, pi]); the reduced phase keeps 31 bits.  For the
// TF32 operands only, whose own rounding (2^-11 relative) is far larger.
__device__ __forceinline__ float2 phase_sfu(unsigned long long m, unsigned long long s) {
    const long long q = (long long)((m * s) << 1);      // (m s mod 2) in [-1, 1) half-turns, 2^-63 units
    const float y = (float)(int)(q >> 32) * (3.14159265358979f * 0x1p-31f);   // radians in [-pi, pi)
    float sn, cs;
    __sincosf(y, &sn, &cs);
    return make_float2(cs, sn);
}

}  // namespace gen
}  // namespace pp
