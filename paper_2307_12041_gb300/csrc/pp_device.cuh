// Device-side building blocks shared by every kernel of the library.
//
// Notation (arXiv 2307.12041, Sec. III): die [0,W] x [0,H]; mode u along x,
// p (called v here) along y; k_u = u pi / W, l_v = v pi / H.
//
// The rectangle integrals of Eq. (aup) factor as
//   X_iu = int theta_i(x) cos(k_u x) dx = f_u * Xt_iu,  f_u = 2W / (pi max(u,1)),
//   Xt_iu = c_i cos(pi u s_i) sin(pi u t_i)   (u >= 1),   Xt_i0 = c_i pi t_i,
// with s_i = x_i / W and t_i = w_i / (2W) (sin a - sin b = 2 cos((a+b)/2) sin((a-b)/2)).
// The kernels only ever build the scaled basis Xt (values of magnitude <= |c|),
// and fold f_u, g_v and the Green's weights into the coefficient operand.
//
// Phases.  pi u s is reduced modulo 2 pi exactly: s is held as a 64-bit fixed
// point number s_fix = (s mod 2) * 2^62, so u * s_fix (mod 2^63) is the phase in
// units of 2^-62 half-turns with no rounding at all.  Only the final reduced
// phase in [-1, 1) half-turns is rounded to FP32 before sincospif.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pp {

// Per-block, per-axis record written by the preparation kernel (64 bytes).
struct __align__(16) AxisRec {
    unsigned long long s;   // (centre / L) mod 2, fixed point 2^-62 half-turns
    unsigned long long t;   // (size / (2L)) mod 2, same units
    float2 es;              // (cos, sin)(pi s): one mode step of the centre phase
    float2 et;              // (cos, sin)(pi t): one mode step of the half-size phase
    float v0;               // scaled rectangle basis at mode 0: c pi t (x), pi t (y)
    float q;                // x axis: centre-sample charge c w h;  y axis: 1
    float c;                // x axis: charge density c;            y axis: 1
    float inv_l;            // pi / L (for the derivative factors -u pi / L)
    float2 es8;             // (cos, sin)(8 pi s): an 8-mode step
    float2 et8;             // (cos, sin)(8 pi t)
};
static_assert(sizeof(AxisRec) == 64, "AxisRec layout");

// e^{i pi m s} for an integer mode m and a fixed-point phase coefficient s.
// The reduced phase is split into its top 24 bits (exact in FP32, fed to
// sincospif) and a residual below 2^-23 half-turns, applied as a first-order
// rotation (the dropped second-order term is below 1e-13).
__device__ __forceinline__ float2 phase_cs(unsigned long long m, unsigned long long s) {
    unsigned long long p = m * s;                 // m s mod 2^64, units 2^-62
    long long q = (long long)(p << 1);            // (m s mod 2) -> [-1, 1), units 2^-63
    int hi = (int)(q >> 40);                      // signed top 24 bits
    long long lo = q - ((long long)hi << 40);     // [0, 2^40)
    float th = (float)hi * 0x1p-23f;              // exact
    float d = (float)(int)(lo >> 16) * (3.14159265358979f * 0x1p-47f);   // pi * residual
    float sn, cs;
    sincospif(th, &sn, &cs);
    return make_float2(fmaf(-sn, d, cs), fmaf(cs, d, sn));
}

// The gradient value v of block b as the energy kernels write it (GradOut in
// pp_internal.h): optionally combined with the value already in out[b] (weighted by
// w[b]), scaled by a device scalar and masked.
template <typename GO>
__device__ __forceinline__ float grad_out(const GO &go, const float *out, size_t b, float v) {
    if (go.acc) {
        const float wb = (go.w ? go.w[b] : 0.0f) + (go.wt ? 0.5f * (float)go.wt[0] : 0.0f);
        v = fmaf(wb, out[b], v);
    }
    if (go.scale) v *= (float)go.scale[0];
    if (go.mask && go.mask[b] == 0) v = 0.0f;
    return v;
}

// z * e (complex), one angle-addition step.
__device__ __forceinline__ float2 rot(float2 z, float2 e) {
    return make_float2(fmaf(z.x, e.x, -z.y * e.y), fmaf(z.y, e.x, z.x * e.y));
}

// (x * k) mod 2 in units of 2^-62 half-turns, for a float32 x and a positive
// normal double k, from the exact 77-bit product of the two significands
// (integer arithmetic only: FP64 is a narrow pipe on this GPU), rounded to the
// nearest unit (ties away from zero), then reduced mod 2.  Used for s = x / L and
// t = w / (2L) with k = 1/L, 1/(2L).
__device__ __forceinline__ unsigned long long fixed_halfturns(float x, double k) {
    const unsigned xb = __float_as_uint(x);
    const int xe = (int)((xb >> 23) & 0xFFu);
    if ((xb & 0x7FFFFFFFu) == 0u || xe == 0xFF) return 0ull;      // zero (or not finite)
    const unsigned long long mx = (unsigned long long)((xb & 0x7FFFFFu) | (xe ? 0x800000u : 0u));
    const unsigned long long kb = (unsigned long long)__double_as_longlong(k);
    const unsigned long long mk = (kb & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    // value * 2^62 = mx * mk * 2^sh
    const int sh = (xe ? xe : 1) - 150 + ((int)((kb >> 52) & 0x7FF) - 1075) + 62;
    const unsigned long long lo = mx * mk, hi = __umul64hi(mx, mk);   // mx * mk < 2^77
    constexpr unsigned long long M63 = 0x7FFFFFFFFFFFFFFFull;
    unsigned long long q;
    if (sh >= 0) {
        q = sh >= 63 ? 0ull : (lo << sh);
    } else {
        const int r = -sh;
        if (r >= 78) {
            q = 0ull;
        } else if (r < 64) {
            q = (lo >> r) | (r ? (hi << (64 - r)) : 0ull);
            q += (lo >> (r - 1)) & 1ull;                                // r >= 1 here
        } else {
            q = hi >> (r - 64);
            q += (r == 64 ? (lo >> 63) : (hi >> (r - 65))) & 1ull;
        }
    }
    q &= M63;
    return (xb >> 31) ? ((0ull - q) & M63) : q;
}

// Programmatic dependent launch.  A kernel launched by launch_dependent() may be
// scheduled while the kernel before it in the stream is still running; pdl_wait()
// blocks until that kernel has completed and its writes are visible (a no-op for a
// plain launch).  Every such kernel calls pdl_wait() before its first global load or
// store and before it allocates tensor memory, so that while it waits it holds
// nothing an earlier kernel still needs.  pdl_trigger() lets the next dependent
// kernel be scheduled once every CTA of this grid has issued it or exited.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... Params, typename... Args>
cudaError_t launch_dependent(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t stream, Args &&...args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

}  // namespace pp
