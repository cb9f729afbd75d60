// Kernels of the placement loop around the density energy (Sec. IV: minimise
// f = W_LSE + lambda N with one Nesterov step per iteration, a penalty update and an
// overflow stop, "as in ePlace").
//
//   lse_net_kernel      per net and axis: max, min and the shifted sums
//                       sum exp((x - max) / gamma), sum exp((min - x) / gamma); the net's
//                       W_LSE and HPWL into a per-CTA sum
//   lse_cell_kernel     per cell: dW/dx = sum over its nets of softmax(x / gamma) -
//                       softmax(-x / gamma) at the cell (a gather over the cell's nets,
//                       no atomics: the result does not depend on thread timing)
//   combine_kernel      g = (dW + lambda dN) / max(1, |nets of i| + lambda q_i)
//                       (ePlace's diagonal preconditioner; fixed blocks get 0)
//   step_norms_kernel   |v - v_prev|^2 and |g - g_prev|^2 (for the step length)
//   nesterov_kernel     u' = clamp(v - alpha g), v' = clamp(u' + coef (u' - u)),
//                       alpha = |v - v_prev| / |g - g_prev| read on the device
//   overflow_kernel     sum_b max(P_b - rho_t, 0) of a bin density P
//   cell_step_kernel    the one-call iteration's cell pass: the three kernels above
//                       (per-cell wirelength gradient, combination, step norms) fused
//   place_loop_*_kernel the loop's scalar update between iterations (one thread, FP64)
//                       when the loop runs on the device (pp_place_run)
//
// The loop's scalars (lambda, gamma, alpha0, coef) come either as kernel arguments or,
// when `scal` is non-NULL, from device memory {lambda, gamma, alpha0, coef} read when
// the kernel runs (so that one captured CUDA graph serves every iteration).
#include <cmath>
#include <cstdint>

#include "pp_internal.h"
#include "pp_place.h"
#include "pp_sum.cuh"

namespace pp {
namespace {

// stats[e] = {max x, min x, 1 / sum exp((x - max)/g), 1 / sum exp((min - x)/g), same for y}
__global__ void lse_net_kernel(int n_nets, const int32_t *__restrict__ net_ptr,
                               const int32_t *__restrict__ net_pin, const float *__restrict__ x,
                               const float *__restrict__ y, float gamma, float inv_gamma,
                               const float *__restrict__ scal, float4 *__restrict__ stats,
                               double *__restrict__ out) {
    if (scal) {
        gamma = scal[1];
        inv_gamma = 1.f / gamma;
    }
    // e^{d / gamma} = 2^{d k2}: one multiply and the hardware base-2 exponential
    const float k2 = inv_gamma * 1.44269504088896341f;
    Sum2 wl, hp;
    // A net of up to KP pins is taken by its own thread: its pins gathered together (their
    // loads in flight at once) and kept in registers for the second pass.  Longer nets
    // are taken by the whole warp afterwards, one at a time, a pin per lane, with warp
    // reductions, so that no lane's long net holds its warp.  The warps run the loop in
    // step (e = base + lane), every lane reaching the warp-wide steps.
    constexpr int KP = 8;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    auto finish = [&](int e, float hx, float lx, float hy, float ly, float spx, float snx, float spy, float sny) {
        stats[2 * e] = make_float4(hx, lx, 1.f / spx, 1.f / snx);
        stats[2 * e + 1] = make_float4(hy, ly, 1.f / spy, 1.f / sny);
        add2(hp, hx - lx);
        add2(hp, hy - ly);
        add2(wl, hx - lx);
        add2(wl, hy - ly);
        add_prod(wl, gamma, logf(spx));
        add_prod(wl, gamma, logf(snx));
        add_prod(wl, gamma, logf(spy));
        add_prod(wl, gamma, logf(sny));
    };
    for (int base = ((int)(blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < n_nets; base += nwarps * 32) {
        const int e = base + lane;
        int p0 = 0, p1 = 0;
        if (e < n_nets) {
            p0 = net_ptr[e];
            p1 = net_ptr[e + 1];
        }
        const int np = p1 - p0;
        if (e < n_nets && np <= KP) {
            float hx = -INFINITY, lx = INFINITY, hy = -INFINITY, ly = INFINITY;
            float px[KP], py[KP];
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                px[k] = py[k] = 0.f;
                if (k < np) {
                    const int i = net_pin[p0 + k];
                    px[k] = x[i];
                    py[k] = y[i];
                }
            }
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                if (k < np) {
                    hx = fmaxf(hx, px[k]);
                    lx = fminf(lx, px[k]);
                    hy = fmaxf(hy, py[k]);
                    ly = fminf(ly, py[k]);
                }
            }
            float spx = 0.f, snx = 0.f, spy = 0.f, sny = 0.f;
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                if (k < np) {
                    spx += exp2f((px[k] - hx) * k2);
                    snx += exp2f((lx - px[k]) * k2);
                    spy += exp2f((py[k] - hy) * k2);
                    sny += exp2f((ly - py[k]) * k2);
                }
            }
            if (np >= 2) {
                finish(e, hx, lx, hy, ly, spx, snx, spy, sny);
            } else {   // a net of fewer than two pins adds nothing: both exponentials
                       // of its gradient terms are exp(-inf) = 0 (no inf * 0)
                stats[2 * e] = make_float4(INFINITY, -INFINITY, 0.f, 0.f);
                stats[2 * e + 1] = make_float4(INFINITY, -INFINITY, 0.f, 0.f);
            }
        }
        // the warp's long nets, one at a time over the whole warp
        unsigned todo = __ballot_sync(full, e < n_nets && np > KP);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int q0 = __shfl_sync(full, p0, src), q1 = __shfl_sync(full, p1, src);
            // pass 1: max and min; the first 32 pins stay in registers for pass 2
            float hx = -INFINITY, lx = INFINITY, hy = -INFINITY, ly = INFINITY, fx = 0.f, fy = 0.f;
            const bool first = q0 + lane < q1;
            if (first) {
                const int i = net_pin[q0 + lane];
                fx = x[i];
                fy = y[i];
                hx = lx = fx;
                hy = ly = fy;
            }
            for (int p = q0 + 32 + lane; p < q1; p += 32) {
                const int i = net_pin[p];
                const float xi = x[i], yi = y[i];
                hx = fmaxf(hx, xi);
                lx = fminf(lx, xi);
                hy = fmaxf(hy, yi);
                ly = fminf(ly, yi);
            }
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                hx = fmaxf(hx, __shfl_xor_sync(full, hx, off));
                lx = fminf(lx, __shfl_xor_sync(full, lx, off));
                hy = fmaxf(hy, __shfl_xor_sync(full, hy, off));
                ly = fminf(ly, __shfl_xor_sync(full, ly, off));
            }
            // pass 2: the shifted exponential sums
            float spx = 0.f, snx = 0.f, spy = 0.f, sny = 0.f;
            if (first) {
                spx = exp2f((fx - hx) * k2);
                snx = exp2f((lx - fx) * k2);
                spy = exp2f((fy - hy) * k2);
                sny = exp2f((ly - fy) * k2);
            }
            for (int p = q0 + 32 + lane; p < q1; p += 32) {
                const int i = net_pin[p];
                const float xi = x[i], yi = y[i];
                spx += exp2f((xi - hx) * k2);
                snx += exp2f((lx - xi) * k2);
                spy += exp2f((yi - hy) * k2);
                sny += exp2f((ly - yi) * k2);
            }
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                spx += __shfl_xor_sync(full, spx, off);
                snx += __shfl_xor_sync(full, snx, off);
                spy += __shfl_xor_sync(full, spy, off);
                sny += __shfl_xor_sync(full, sny, off);
            }
            if (lane == src) finish(base + src, hx, lx, hy, ly, spx, snx, spy, sny);
        }
    }
    block_add2(wl, out);
    block_add2(hp, out + 1);
}

__global__ void lse_cell_kernel(int n_cells, const int32_t *__restrict__ cell_ptr,
                                const int32_t *__restrict__ cell_net, const float *__restrict__ x,
                                const float *__restrict__ y, float inv_gamma, const float *__restrict__ scal,
                                const float4 *__restrict__ stats, float *__restrict__ gx,
                                float *__restrict__ gy) {
    if (scal) inv_gamma = 1.f / scal[1];
    const float k2 = inv_gamma * 1.44269504088896341f;   // e^{d / gamma} = 2^{d k2}
    // the first KC nets of a cell gathered together (their loads in flight at once)
    constexpr int KC = 4;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_cells; i += gridDim.x * blockDim.x) {
        const float xi = x[i], yi = y[i];
        const int k0 = cell_ptr[i], k1 = cell_ptr[i + 1];
        float ax = 0.f, ay = 0.f;
        float4 sxs[KC], sys[KC];
#pragma unroll
        for (int q = 0; q < KC; ++q) {
            if (k0 + q < k1) {
                const int e = cell_net[k0 + q];
                sxs[q] = stats[2 * e];
                sys[q] = stats[2 * e + 1];
            }
        }
#pragma unroll
        for (int q = 0; q < KC; ++q) {
            if (k0 + q < k1) {
                const float4 sx = sxs[q], sy = sys[q];
                ax += exp2f((xi - sx.x) * k2) * sx.z - exp2f((sx.y - xi) * k2) * sx.w;
                ay += exp2f((yi - sy.x) * k2) * sy.z - exp2f((sy.y - yi) * k2) * sy.w;
            }
        }
        for (int b = k0 + KC; b < k1; b += KC) {      // the rest KC at a time, in order
#pragma unroll
            for (int q = 0; q < KC; ++q) {
                if (b + q < k1) {
                    const int e = cell_net[b + q];
                    sxs[q] = stats[2 * e];
                    sys[q] = stats[2 * e + 1];
                }
            }
#pragma unroll
            for (int q = 0; q < KC; ++q) {
                if (b + q < k1) {
                    const float4 sx = sxs[q], sy = sys[q];
                    ax += exp2f((xi - sx.x) * k2) * sx.z - exp2f((sx.y - xi) * k2) * sx.w;
                    ay += exp2f((yi - sy.x) * k2) * sy.z - exp2f((sy.y - yi) * k2) * sy.w;
                }
            }
        }
        gx[i] = ax;
        gy[i] = ay;
    }
}

__global__ void combine_kernel(int64_t n, const float *__restrict__ gwx, const float *__restrict__ gwy,
                               const float *__restrict__ gnx, const float *__restrict__ gny,
                               const int32_t *__restrict__ cell_ptr, const float *__restrict__ q,
                               const uint8_t *__restrict__ movable, float lambda, const float *__restrict__ scal,
                               float *__restrict__ gx, float *__restrict__ gy) {
    if (scal) lambda = scal[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (movable && !movable[i]) {
            gx[i] = gy[i] = 0.f;
            continue;
        }
        const float deg = cell_ptr ? (float)(cell_ptr[i + 1] - cell_ptr[i]) : 0.f;
        const float inv = 1.f / fmaxf(1.f, deg + lambda * q[i]);
        gx[i] = (gwx[i] + lambda * gnx[i]) * inv;
        gy[i] = (gwy[i] + lambda * gny[i]) * inv;
    }
}

// The one-call iteration's cell pass: the per-cell wirelength gradient (as
// lse_cell_kernel), the preconditioned combination with the density gradient (as
// combine_kernel) and the step norms (as step_norms_kernel) in one kernel, so that the
// wirelength gradient never leaves registers.  g equals what the separate kernels
// write; the norms differ from theirs only in the order of their compensated sums.
__global__ void cell_step_kernel(int n_cells, const int32_t *__restrict__ cell_ptr,
                                 const int32_t *__restrict__ cell_net, const float *__restrict__ x,
                                 const float *__restrict__ y, float inv_gamma, float lambda,
                                 const float *__restrict__ scal, const float4 *__restrict__ stats,
                                 const float *__restrict__ gnx, const float *__restrict__ gny,
                                 const float *__restrict__ q, const uint8_t *__restrict__ movable,
                                 const float *__restrict__ vpx, const float *__restrict__ vpy,
                                 const float *__restrict__ gpx, const float *__restrict__ gpy,
                                 float *__restrict__ gx, float *__restrict__ gy, double *__restrict__ norms) {
    if (scal) {
        lambda = scal[0];
        inv_gamma = 1.f / scal[1];
    }
    const float k2 = inv_gamma * 1.44269504088896341f;   // e^{d / gamma} = 2^{d k2}
    constexpr int KC = 4;
    Sum2 dv, dg;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_cells; i += gridDim.x * blockDim.x) {
        const float xi = x[i], yi = y[i];
        const int k0 = cell_ptr[i], k1 = cell_ptr[i + 1];
        float ax = 0.f, ay = 0.f;
        float4 sxs[KC], sys[KC];
        for (int b = k0; b < k1; b += KC) {                 // the cell's nets KC at a time, in order
#pragma unroll
            for (int c = 0; c < KC; ++c) {
                if (b + c < k1) {
                    const int e = cell_net[b + c];
                    sxs[c] = stats[2 * e];
                    sys[c] = stats[2 * e + 1];
                }
            }
#pragma unroll
            for (int c = 0; c < KC; ++c) {
                if (b + c < k1) {
                    const float4 sx = sxs[c], sy = sys[c];
                    ax += exp2f((xi - sx.x) * k2) * sx.z - exp2f((sx.y - xi) * k2) * sx.w;
                    ay += exp2f((yi - sy.x) * k2) * sy.z - exp2f((sy.y - yi) * k2) * sy.w;
                }
            }
        }
        float g0 = 0.f, g1 = 0.f;
        if (!movable || movable[i]) {
            const float inv = 1.f / fmaxf(1.f, (float)(k1 - k0) + lambda * q[i]);
            g0 = (ax + lambda * gnx[i]) * inv;
            g1 = (ay + lambda * gny[i]) * inv;
        }
        gx[i] = g0;
        gy[i] = g1;
        const float a = xi - vpx[i], c = yi - vpy[i], d = g0 - gpx[i], e = g1 - gpy[i];
        add_prod(dv, a, a);
        add_prod(dv, c, c);
        add_prod(dg, d, d);
        add_prod(dg, e, e);
    }
    block_add2(dv, norms);
    block_add2(dg, norms + 1);
}

__global__ void step_norms_kernel(int64_t n, const float *__restrict__ vx, const float *__restrict__ vy,
                                  const float *__restrict__ vpx, const float *__restrict__ vpy,
                                  const float *__restrict__ gx, const float *__restrict__ gy,
                                  const float *__restrict__ gpx, const float *__restrict__ gpy,
                                  double *__restrict__ norms) {
    Sum2 dv, dg;
    // U strided elements per thread and round, their loads in flight together
    constexpr int U = 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n; b += U * stride) {
        float a[U], c[U], d[U], e[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const int64_t i = b + k * stride;
            a[k] = c[k] = d[k] = e[k] = 0.f;
            if (i < n) {
                a[k] = vx[i] - vpx[i];
                c[k] = vy[i] - vpy[i];
                d[k] = gx[i] - gpx[i];
                e[k] = gy[i] - gpy[i];
            }
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            add_prod(dv, a[k], a[k]);
            add_prod(dv, c[k], c[k]);
            add_prod(dg, d[k], d[k]);
            add_prod(dg, e[k], e[k]);
        }
    }
    block_add2(dv, norms);
    block_add2(dg, norms + 1);
}

__global__ void nesterov_kernel(int64_t n, float *__restrict__ ux, float *__restrict__ uy, float *__restrict__ vx,
                                float *__restrict__ vy, float *__restrict__ vpx, float *__restrict__ vpy,
                                const float *__restrict__ gx, const float *__restrict__ gy,
                                float *__restrict__ gpx, float *__restrict__ gpy, const float *__restrict__ w,
                                const float *__restrict__ h, float W, float H,
                                const uint8_t *__restrict__ movable, const double *__restrict__ norms,
                                float alpha0, float coef, const float *__restrict__ scal) {
    if (scal) {
        alpha0 = scal[2];
        coef = scal[3];
    }
    // step length: |v - v_prev| / |g - g_prev| from the previous iteration, else alpha0
    // (once per CTA: FP64 division and square root are slow on this GPU)
    __shared__ float s_alpha;
    if (threadIdx.x == 0) {
        float al = alpha0;
        if (norms && norms[1] > 0.0 && norms[0] > 0.0) al = (float)sqrt(norms[0] / norms[1]);
        s_alpha = al;
    }
    __syncthreads();
    const float alpha = s_alpha;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float vxi = vx[i], vyi = vy[i], gxi = gx[i], gyi = gy[i];
        vpx[i] = vxi;
        vpy[i] = vyi;
        gpx[i] = gxi;
        gpy[i] = gyi;
        if (movable && !movable[i]) continue;
        const float lx = 0.5f * w[i], hx = W - 0.5f * w[i], ly = 0.5f * h[i], hy = H - 0.5f * h[i];
        const float nux = fminf(fmaxf(vxi - alpha * gxi, lx), hx);
        const float nuy = fminf(fmaxf(vyi - alpha * gyi, ly), hy);
        const float nvx = fminf(fmaxf(nux + coef * (nux - ux[i]), lx), hx);
        const float nvy = fminf(fmaxf(nuy + coef * (nuy - uy[i]), ly), hy);
        ux[i] = nux;
        uy[i] = nuy;
        vx[i] = nvx;
        vy[i] = nvy;
    }
}

__global__ void overflow_kernel(int64_t cells, const float *__restrict__ P, float target, double *__restrict__ out) {
    Sum2 s;
    constexpr int U = 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < cells; b += U * stride) {
        float v[U];
#pragma unroll
        for (int k = 0; k < U; ++k) v[k] = b + k * stride < cells ? P[b + k * stride] : target;
#pragma unroll
        for (int k = 0; k < U; ++k) add2(s, fmaxf(v[k] - target, 0.f));
    }
    block_add2(s, out);
}

// ---- the loop's scalar update on the device (pp_place_run) ----

// The scalar update rounds every operation on its own (no contraction into FMAs),
// in the order the host loop evaluates it, so that both make the same roundings
// (pow aside).
__device__ __forceinline__ double a_next_of(double a) {
    return __dadd_rn(1.0, sqrt(__dadd_rn(__dmul_rn(__dmul_rn(4.0, a), a), 1.0))) / 2.0;
}

// ePlace's smoothing schedule gamma(tau) = 8 w_b 10^{(20/9)(tau - 0.1) - 1}
__device__ double gamma_of_tau(double tau, double bin_w) {
    const double ex = __dsub_rn(__dmul_rn(20.0 / 9.0, __dsub_rn(tau, 0.1)), 1.0);
    return __dmul_rn(__dmul_rn(8.0, bin_w), pow(10.0, ex));
}

// The next iteration's float32 scalars {lambda, gamma, alpha0 = 0, coef} from the
// state, coef = (a_k - 1) / a_{k+1}; the stop code when one is out of range.
__device__ int32_t next_scalars(pp_place_state *st) {
    const double a = st->a_k;
    const double a_next = a_next_of(a);
    const float lam = (float)st->lambda, gam = (float)st->gamma, coef = (float)((a - 1.0) / a_next);
    if (!(isfinite(lam) && lam >= 0.f && isfinite(gam) && gam > 0.f && isfinite(coef) && isfinite(a) && a >= 1.0))
        return PP_PLACE_NONFINITE;
    st->scalars[0] = lam;
    st->scalars[1] = gam;
    st->scalars[2] = 0.f;
    st->scalars[3] = coef;
    return PP_PLACE_RUNNING;
}

// Before the loop: check that the state can start and set the first scalars; the
// WHILE node's condition is 1 only if it can.
__global__ void place_loop_begin_kernel(pp_place_state *st, int32_t max_iters, cudaGraphConditionalHandle cond) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    st->run_count = 0;
    int32_t stop = st->stop;
    if (stop == PP_PLACE_RUNNING) {
        if (st->k >= max_iters)
            stop = PP_PLACE_MAX_ITERS;
        else if (!(st->k >= 1 && st->d_ref > 0.0 && isfinite(st->d_ref) && isfinite(st->hpwl_prev)))
            stop = PP_PLACE_BAD_STATE;
        else
            stop = next_scalars(st);
    }
    st->stop = stop;
    cudaGraphSetConditional(cond, stop == PP_PLACE_RUNNING ? 1u : 0u);
}

// After iteration k: its record, the penalty and smoothing updates, the stop test and
// the next scalars; the WHILE node's condition for the next body execution.
__global__ void place_loop_step_kernel(const double *__restrict__ stats, pp_place_state *st,
                                       pp_place_record *trace, pp_place_schedule sc,
                                       const unsigned *__restrict__ status, cudaGraphConditionalHandle cond) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int64_t k = st->k;
    pp_place_record r;
    r.k = k;
    r.reserved = 0;
    r.tau = __dmul_rn(stats[0], sc.bin_area) / sc.area_mov;
    r.w_lse = stats[1];
    r.hpwl = stats[2];
    r.e = stats[3];
    r.lambda = st->lambda;
    r.gamma = st->gamma;
    st->a_k = a_next_of(st->a_k);
    const double mu = pow(1.1, 1.0 - (r.hpwl - st->hpwl_prev) / st->d_ref);
    st->lambda = __dmul_rn(st->lambda, fmin(1.1, fmax(0.75, mu)));
    st->hpwl_prev = r.hpwl;
    st->tau = r.tau;
    st->gamma = gamma_of_tau(r.tau, sc.bin_w);
    st->k = k + 1;
    const int32_t runs = ++st->run_count;
    int32_t stop = PP_PLACE_RUNNING;
    if (r.tau < sc.tau_stop)
        stop = PP_PLACE_CONVERGED;
    else if (k + 1 >= sc.max_iters || runs >= sc.max_iters)
        stop = PP_PLACE_MAX_ITERS;
    else if (*status != 0u)
        stop = PP_PLACE_DEVICE_ERROR;
    else
        stop = next_scalars(st);
    st->stop = stop;
    r.stop = stop;
    if (k >= 0 && k < sc.max_iters) trace[k] = r;
    cudaGraphSetConditional(cond, stop == PP_PLACE_RUNNING ? 1u : 0u);
}

int grid_for(int64_t n, int cap) {
    int64_t b = (n + 255) / 256;
    if (b < 1) b = 1;
    return (int)(b < cap ? b : cap);
}

}  // namespace

cudaError_t launch_wirelength(int n_nets, int n_cells, const int32_t *net_ptr, const int32_t *net_pin,
                              const int32_t *cell_ptr, const int32_t *cell_net, const float *x,
                              const float *y, float gamma, const float *scal, float *stats, float *gx,
                              float *gy, double *out, int sm_count, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    if (n_nets > 0)
        lse_net_kernel<<<grid_for(n_nets, 16 * sm_count), 256, 0, st>>>(
            n_nets, net_ptr, net_pin, x, y, gamma, 1.f / gamma, scal, reinterpret_cast<float4 *>(stats), out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (n_cells > 0 && gx)
        lse_cell_kernel<<<grid_for(n_cells, 16 * sm_count), 256, 0, st>>>(
            n_cells, cell_ptr, cell_net, x, y, 1.f / gamma, scal, reinterpret_cast<const float4 *>(stats), gx,
            gy);
    return cudaGetLastError();
}

cudaError_t launch_cell_step(int n_cells, const int32_t *cell_ptr, const int32_t *cell_net, const float *x,
                             const float *y, float gamma, float lambda, const float *scal, const float *stats,
                             const float *gnx, const float *gny, const float *q, const uint8_t *movable,
                             const float *vpx, const float *vpy, const float *gpx, const float *gpy, float *gx,
                             float *gy, double *norms, int sm_count, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(norms, 0, 2 * sizeof(double), st);
    if (e != cudaSuccess || n_cells <= 0) return e;
    cell_step_kernel<<<grid_for(n_cells, 16 * sm_count), 256, 0, st>>>(
        n_cells, cell_ptr, cell_net, x, y, 1.f / gamma, lambda, scal, reinterpret_cast<const float4 *>(stats),
        gnx, gny, q, movable, vpx, vpy, gpx, gpy, gx, gy, norms);
    return cudaGetLastError();
}

cudaError_t launch_combine(int64_t n, const float *gwx, const float *gwy, const float *gnx, const float *gny,
                           const int32_t *cell_ptr, const float *q, const uint8_t *movable, float lambda,
                           const float *scal, float *gx, float *gy, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    combine_kernel<<<grid_for(n, 4096), 256, 0, st>>>(n, gwx, gwy, gnx, gny, cell_ptr, q, movable, lambda, scal, gx,
                                                      gy);
    return cudaGetLastError();
}

cudaError_t launch_step_norms(int64_t n, const float *vx, const float *vy, const float *vpx, const float *vpy,
                              const float *gx, const float *gy, const float *gpx, const float *gpy,
                              double *norms, int sm_count, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(norms, 0, 2 * sizeof(double), st);
    if (e != cudaSuccess || n <= 0) return e;
    // two CTAs per SM, grid-stride: few same-address FP64 atomics at the end
    step_norms_kernel<<<grid_for(n, 2 * sm_count), 256, 0, st>>>(n, vx, vy, vpx, vpy, gx, gy, gpx, gpy, norms);
    return cudaGetLastError();
}

cudaError_t launch_nesterov(int64_t n, float *ux, float *uy, float *vx, float *vy, float *vpx, float *vpy,
                            const float *gx, const float *gy, float *gpx, float *gpy, const float *w,
                            const float *h, float W, float H, const uint8_t *movable, const double *norms,
                            float alpha0, float coef, const float *scal, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    nesterov_kernel<<<grid_for(n, 4096), 256, 0, st>>>(n, ux, uy, vx, vy, vpx, vpy, gx, gy, gpx, gpy, w, h, W, H,
                                                       movable, norms, alpha0, coef, scal);
    return cudaGetLastError();
}

cudaError_t launch_overflow(int m, const float *P, float target, double *out, int sm_count, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    const int64_t cells = (int64_t)m * m;
    overflow_kernel<<<grid_for(cells, 2 * sm_count), 256, 0, st>>>(cells, P, target, out);
    return cudaGetLastError();
}

cudaError_t launch_place_loop_begin(pp_place_state *st, int32_t max_iters, cudaGraphConditionalHandle cond,
                                    cudaStream_t s) {
    place_loop_begin_kernel<<<1, 32, 0, s>>>(st, max_iters, cond);
    return cudaGetLastError();
}

cudaError_t launch_place_loop_step(const double *stats, pp_place_state *st, pp_place_record *trace,
                                   const pp_place_schedule &sc, const unsigned *status,
                                   cudaGraphConditionalHandle cond, cudaStream_t s) {
    place_loop_step_kernel<<<1, 32, 0, s>>>(stats, st, trace, sc, status, cond);
    return cudaGetLastError();
}

}  // namespace pp
