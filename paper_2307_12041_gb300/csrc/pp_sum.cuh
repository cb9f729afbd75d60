// Compensated float32 sums for the reductions of the placement-loop and binned-scheme
// kernels (W_LSE and HPWL, the step norms, the overflow excess, E).
//
// FP64 arithmetic (and every float -> double conversion) issues at a small fraction of
// the FP32 rate on this GPU, so accumulating each element in FP64 costs more than the
// rest of those kernels.  Instead each thread carries an unevaluated pair (s, c), the
// sum being s + c: every float add of a term is followed by the exact recovery of its
// rounding error (Knuth's TwoSum, TAOCP vol. 2, sec. 4.2.2) into c, and a product's
// rounding error comes exactly from one fused multiply-add (TwoProduct, Ogita, Rump and
// Oishi, "Accurate sum and dot product", SISC 2005).  What is lost is only the rounding
// of the small additions into c, about 2^-48 of the terms' magnitudes per term: as
// accurate as the FP64 accumulation it replaces.  The pair is merged across the warp in
// the same way and widened to double once per warp.  The _rn intrinsics keep the
// compiler from contracting a product and a sum into one FMA, which would break the
// error recovery.
#pragma once

namespace pp {

struct Sum2 {
    float s = 0.f, c = 0.f;
};

// a += v, the rounding error of the add kept in a.c
__device__ __forceinline__ void add2(Sum2 &a, float v) {
    const float t = __fadd_rn(a.s, v);
    const float bp = __fsub_rn(t, a.s);
    a.c = __fadd_rn(a.c, __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(v, bp)));
    a.s = t;
}

// a += x * y, with the rounding errors of the product and of the add
__device__ __forceinline__ void add_prod(Sum2 &a, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float e = fmaf(x, y, -p);
    add2(a, p);
    a.c = __fadd_rn(a.c, e);
}

// a += b
__device__ __forceinline__ void merge2(Sum2 &a, const Sum2 &b) {
    add2(a, b.s);
    a.c = __fadd_rn(a.c, b.c);
}

// The warp's total of its lanes' pairs, as a double (every lane gets it).
__device__ __forceinline__ double warp_total(Sum2 a) {
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        Sum2 o;
        o.s = __shfl_xor_sync(0xffffffffu, a.s, off);
        o.c = __shfl_xor_sync(0xffffffffu, a.c, off);
        merge2(a, o);
    }
    return (double)a.s + (double)a.c;
}

// scale x (the CTA's total) added to *dst with one atomic per CTA; every thread of the
// CTA must call it (it synchronises the CTA), with blockDim.x a multiple of 32.
__device__ __forceinline__ void block_add2(Sum2 a, double *dst, double scale = 1.0) {
    __shared__ double part[32];
    const double w = warp_total(a);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += part[k];
        atomicAdd(dst, scale * t);
    }
    __syncthreads();
}

}  // namespace pp
