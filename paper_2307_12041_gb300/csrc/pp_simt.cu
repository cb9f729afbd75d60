// FP32 CUDA-core path (PP_FP32) and the precision-independent kernels:
//   prep_kernel          per-block fixed-point phases and scale factors
//   coeff_simt_kernel    St = Xt^T Yt over a slice of blocks (Eq. aup/au0/a0p sums)
//   finish_simt_kernel   a = G o S (Eq. a-a..a-d) and the energy operand K
//   energy_simt_kernel   N_i, dE/dx_i, dE/dy_i as row dots of (Xt K) with Yt, Yh
//
// Scaled quantities (f_u = 2W/(pi max(u,1)), g_v = 2H/(pi max(v,1))):
//   X = f Xt, Y = g Yt                      rectangle integrals (Eq. aup factors)
//   S = X^T Y = f St g,  a = G o S,  G_uv = e_u e_v / (W H (k_u^2 + l_v^2)), G_00 = 0
//   K = f a g  (the operand of both energy contractions)
//   N_i  = sum_uv Xt_iu K_uv Yt_iv
//   gx_i = sum_uv Xh_iu K_uv Yt_iv,  Xh_iu = -(u pi / W) c sin(pi u s) sin(pi u t)
//   gy_i = sum_uv Xt_iu K_uv Yh_iv,  Yh_iv = -(v pi / H) sin(pi v s) sin(pi v t)
#include <cmath>
#include <cstdio>

#include "pp_device.cuh"
#include "pp_internal.h"

namespace pp {

// ---------------------------------------------------------------------------
// Preparation: one record per block and axis; zero the FP64 sums and E.
// ---------------------------------------------------------------------------
__global__ void prep_kernel(const float *__restrict__ x, const float *__restrict__ y,
                            const float *__restrict__ w, const float *__restrict__ h,
                            const float *__restrict__ c, int n, double invW, double invH,
                            float piW, float piH, AxisRec *__restrict__ xr, AxisRec *__restrict__ yr,
                            double *__restrict__ S64, size_t nS, double *e_total,
                            const float *__restrict__ gw, const double *__restrict__ gt, bool weighted) {
    // FP32 and integer arithmetic only (FP64 is a narrow pipe on this GPU)
    pdl_trigger();            // a dependent coefficient or finish kernel may be scheduled now
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const double halfW = 0.5 * invW, halfH = 0.5 * invH;       // exact: powers of two
    // weighted: charge c_i (0.5 gt + gw_i), the charges whose coefficients b give the
    // second term of the adjoint of sum_i gw_i N_i + gt E
    const float ght = (weighted && gt) ? 0.5f * (float)gt[0] : 0.0f;
    // one thread per block: its x and y records (independent work, issued together)
    for (size_t b = tid; b < (size_t)n; b += stride) {
        const float px = x[b], py = y[b], lw = w[b], lh = h[b];
        float ci = c ? c[b] : 1.0f;
        if (weighted) ci *= ght + (gw ? gw[b] : 0.0f);
        AxisRec rx, ry;
        rx.s = fixed_halfturns(px, invW);
        ry.s = fixed_halfturns(py, invH);
        rx.t = fixed_halfturns(lw, halfW);
        ry.t = fixed_halfturns(lh, halfH);
        rx.es = phase_cs(1, rx.s);
        ry.es = phase_cs(1, ry.s);
        rx.et = phase_cs(1, rx.t);
        ry.et = phase_cs(1, ry.t);
        rx.es8 = phase_cs(8, rx.s);
        ry.es8 = phase_cs(8, ry.s);
        rx.et8 = phase_cs(8, rx.t);
        ry.et8 = phase_cs(8, ry.t);
        rx.inv_l = piW;
        ry.inv_l = piH;
        rx.v0 = ci * (0.5f * piW * lw);                               // c pi t
        rx.q = ci * lw * lh;
        rx.c = ci;
        ry.v0 = 0.5f * piH * lh;
        ry.q = 1.0f;
        ry.c = 1.0f;
        xr[b] = rx;
        yr[b] = ry;
    }
    for (size_t j = tid; j < nS; j += stride) S64[j] = 0.0;
    if (tid == 0 && e_total) *e_total = 0.0;
}

cudaError_t launch_prep(const Launch &L, bool zero_S, double *e_total, const ChargeWeights &cw) {
    size_t nS = zero_S ? (size_t)L.Mx * L.My : 0;
    size_t work = (size_t)L.n > nS ? (size_t)L.n : nS;
    int blocks = (int)((work + 255) / 256);
    if (blocks < 1) blocks = 1;
    if (blocks > 32 * L.sm_count) blocks = 32 * L.sm_count;
    const double PI = 3.141592653589793;
    prep_kernel<<<blocks, 256, 0, L.stream>>>(L.x, L.y, L.w, L.h, L.c, L.n, 1.0 / L.W, 1.0 / L.H,
                                              (float)(PI / L.W), (float)(PI / L.H), L.xrec, L.yrec,
                                              L.S64, nS, e_total, cw.gw, cw.gt, cw.on);
    return cudaGetLastError();
}

__global__ void round_coeffs_kernel(const double *__restrict__ a64, float *__restrict__ a_out, size_t count) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        a_out[i] = (float)a64[i];
}

cudaError_t launch_round_coeffs(const double *a64, float *a_out, size_t count, cudaStream_t stream) {
    if (count == 0) return cudaSuccess;
    size_t blocks = (count + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    round_coeffs_kernel<<<(int)blocks, 256, 0, stream>>>(a64, a_out, count);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Descent step: x <- clamp(x - lr gx + sigma n0, w/2, W - w/2), likewise y, with
// Box-Muller normals from Philox4x32-10 (Salmon et al., SC 2011) keyed by the seed
// and counted by (block, step).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__global__ void descent_step_kernel(float W, float H, int64_t n, float *__restrict__ x,
                                    float *__restrict__ y, const float *__restrict__ w,
                                    const float *__restrict__ h, const float *__restrict__ gx,
                                    const float *__restrict__ gy, const uint8_t *__restrict__ movable,
                                    float lr, float sigma, uint2 key, unsigned step) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (movable && !movable[i]) continue;
        const uint4 o = philox4x32_10(make_uint4((unsigned)i, step, 0u, 0u), key);
        const float u0 = ((float)o.x + 0.5f) * 0x1p-32f;          // (0, 1]
        const float u1 = ((float)o.y + 0.5f) * 0x1p-32f;
        const float r = sqrtf(-2.f * logf(u0));
        float sn, cs;
        sincospif(2.f * u1, &sn, &cs);
        const float wi = w[i], hi = h[i];
        const float xi = x[i] - lr * gx[i] + sigma * (r * cs);
        const float yi = y[i] - lr * gy[i] + sigma * (r * sn);
        x[i] = fminf(fmaxf(xi, 0.5f * wi), W - 0.5f * wi);
        y[i] = fminf(fmaxf(yi, 0.5f * hi), H - 0.5f * hi);
    }
}

cudaError_t launch_descent_step(float W, float H, int64_t n, float *x, float *y, const float *w,
                                const float *h, const float *gx, const float *gy,
                                const uint8_t *movable, float lr, float sigma, uint64_t seed,
                                uint64_t step, cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    const int64_t want = (n + 255) / 256;
    const int grid = (int)(want < 65535 ? want : 65535);
    descent_step_kernel<<<grid, 256, 0, stream>>>(W, H, n, x, y, w, h, gx, gy, movable, lr, sigma,
                                                  make_uint2((unsigned)seed, (unsigned)(seed >> 32)),
                                                  (unsigned)step);
    return cudaGetLastError();
}

// Eight consecutive modes m0..m0+7 of the scaled rectangle basis of one block:
// out[j] = c cos(pi m s) sin(pi m t), m = m0 + j (value v0 at m = 0).
__device__ __forceinline__ void rect_run8(const AxisRec &r, int m0, float out[8]) {
    float2 zs = phase_cs((unsigned long long)m0, r.s);
    float2 zt = phase_cs((unsigned long long)m0, r.t);
    zt.x *= r.c;
    zt.y *= r.c;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        out[j] = zs.x * zt.y;
        zs = rot(zs, r.es);
        zt = rot(zt, r.et);
    }
    if (m0 == 0) out[0] = r.v0;
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// ---------------------------------------------------------------------------
// Coefficient contraction, FP32: CTA tile 128 (u) x 128 (v), a slice of blocks.
// ---------------------------------------------------------------------------
constexpr int CT = 128;   // tile edge
constexpr int CKC = 32;   // blocks per shared-memory chunk
constexpr int CKS = 32;   // blocks summed in plain FP32 before each compensated add (divides CKC)

struct CoeffSmem {
    float Xs[2][CKC][CT];
    float Ys[2][CKC][CT];
    AxisRec Rs[2][2][CKC];
    float lo[64 * 256];      // compensation terms of the running sums, [i*8+j][thread]
};

__global__ void __launch_bounds__(256, 1)
coeff_simt_kernel(const AxisRec *__restrict__ xr, const AxisRec *__restrict__ yr, int n, int Mx,
                  int My, int slice, double *__restrict__ S64) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CoeffSmem &sm = *reinterpret_cast<CoeffSmem *>(smem_raw);
    auto &Xs = sm.Xs;
    auto &Ys = sm.Ys;
    auto &Rs = sm.Rs;
    float *lo_s = sm.lo;
    const int tiles_v = (My + CT - 1) / CT;
    const int tu = blockIdx.x / tiles_v, tv = blockIdx.x % tiles_v;
    const int u_base = tu * CT, v_base = tv * CT;
    const int b0 = blockIdx.y * slice;
    const int b1 = min(n, b0 + slice);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // 16 x 16 thread grid; a warp covers 4 (u) x 8 (v) threads so each 16-byte
    // shared load is one wavefront.
    const int ty = (warp >> 1) * 4 + (lane >> 3);
    const int tx = (warp & 1) * 8 + (lane & 7);
    // generator mapping: chunk row gk, modes gm..gm+7
    const int gk = tid >> 4, gm = (tid & 15) * 8;

    // Every CKS blocks of a chunk are summed into fresh registers, then added to a
    // compensated running sum (hi in registers, lo in shared memory; error-free
    // two-sum), so the FP32 rounding does not grow with the slice length.  Both run
    // on pairs of adjacent v (packed f32x2 FMA and add: one instruction per two
    // lanes' worth of FMA-pipe work, each half rounded exactly as the scalar
    // operation), which leaves issue slots for the loads, the generator and the sums.
    const float2 m1 = make_float2(-1.f, -1.f);            // fma(x, -1, y) = y - x, one rounding
    float2 hi[8][4];
    float2 *lo_s2 = reinterpret_cast<float2 *>(lo_s);     // [i*4+jj][thread]
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            hi[i][jj] = make_float2(0.f, 0.f);
            lo_s2[(i * 4 + jj) * 256 + tid] = make_float2(0.f, 0.f);
        }

    const int nchunks = (b1 - b0 + CKC - 1) / CKC;
    // The records of chunk ch + 1 are copied to shared memory (cp.async) while
    // chunk ch is multiplied: 32 blocks x 2 axes x 64 bytes = 256 x 16-byte pieces.
    auto fetch_recs = [&](int ch, int buf) {
        if (tid < 2 * CKC * 4) {
            const int axis = tid / (CKC * 4), r = tid % (CKC * 4);
            const int k = r / 4, piece = r % 4;
            const int b = b0 + ch * CKC + k;
            if (b < b1) {
                const AxisRec *src = (axis == 0 ? xr : yr) + b;
                cp_async16(reinterpret_cast<char *>(&Rs[buf][axis][k]) + 16 * piece,
                           reinterpret_cast<const char *>(src) + 16 * piece);
            }
        }
        cp_async_commit();
    };
    fetch_recs(0, 0);
    for (int ch = 0; ch < nchunks; ++ch) {
        const int buf = ch & 1;
        cp_async_wait_all();
        __syncthreads();
#pragma unroll
        for (int g2 = 0; g2 < CKC; g2 += 16) {             // chunk rows gk and gk + 16
            const int row = gk + g2;
            float vx[8], vy[8];
            if (b0 + ch * CKC + row < b1) {
                rect_run8(Rs[buf][0][row], u_base + gm, vx);
                rect_run8(Rs[buf][1][row], v_base + gm, vy);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) vx[j] = vy[j] = 0.f;
            }
            *reinterpret_cast<float4 *>(&Xs[buf][row][gm]) = make_float4(vx[0], vx[1], vx[2], vx[3]);
            *reinterpret_cast<float4 *>(&Xs[buf][row][gm + 4]) = make_float4(vx[4], vx[5], vx[6], vx[7]);
            *reinterpret_cast<float4 *>(&Ys[buf][row][gm]) = make_float4(vy[0], vy[1], vy[2], vy[3]);
            *reinterpret_cast<float4 *>(&Ys[buf][row][gm + 4]) = make_float4(vy[4], vy[5], vy[6], vy[7]);
        }
        if (ch + 1 < nchunks) fetch_recs(ch + 1, buf ^ 1);
        __syncthreads();
#pragma unroll 1
        for (int k0 = 0; k0 < CKC; k0 += CKS) {
            float2 acc[8][4];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[i][jj] = make_float2(0.f, 0.f);
#pragma unroll 4
            for (int k = k0; k < k0 + CKS; ++k) {
                const float4 a0 = *reinterpret_cast<const float4 *>(&Xs[buf][k][ty * 4]);
                const float4 a1 = *reinterpret_cast<const float4 *>(&Xs[buf][k][64 + ty * 4]);
                const float4 c0 = *reinterpret_cast<const float4 *>(&Ys[buf][k][tx * 4]);
                const float4 c1 = *reinterpret_cast<const float4 *>(&Ys[buf][k][64 + tx * 4]);
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float2 bp[4] = {make_float2(c0.x, c0.y), make_float2(c0.z, c0.w), make_float2(c1.x, c1.y),
                                      make_float2(c1.z, c1.w)};
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float2 ai = make_float2(av[i], av[i]);
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) acc[i][jj] = __ffma2_rn(ai, bp[jj], acc[i][jj]);
                }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const float2 h = hi[i][jj], a = acc[i][jj];
                    const float2 sum = __fadd2_rn(h, a);
                    const float2 bb = __ffma2_rn(h, m1, sum);                                // sum - hi
                    const float2 e = __fadd2_rn(__ffma2_rn(__ffma2_rn(bb, m1, sum), m1, h),  // hi - (sum - bb)
                                                __ffma2_rn(bb, m1, a));                       // + (acc - bb)
                    float2 &l = lo_s2[(i * 4 + jj) * 256 + tid];
                    l = __fadd2_rn(l, e);
                    hi[i][jj] = sum;
                }
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int u = u_base + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
        if (u >= Mx) continue;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const float2 h = hi[i][jj], l = lo_s2[(i * 4 + jj) * 256 + tid];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int j = 2 * jj + q;
                const int v = v_base + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
                if (v < My)
                    atomicAdd(&S64[(size_t)u * My + v], (double)(q ? h.y : h.x) + (double)(q ? l.y : l.x));
            }
        }
    }
}

cudaError_t launch_coeff_simt(const Launch &L) {
    if (L.n == 0) return cudaSuccess;
    const int tiles = ((L.Mx + CT - 1) / CT) * ((L.My + CT - 1) / CT);
    // Slices of at most 2048 blocks bound the FP32 accumulation length; the
    // slices are combined in FP64.
    int slice = 2048;
    int slices = (L.n + slice - 1) / slice;
    dim3 grid(tiles, slices);
    const int smem = (int)sizeof(CoeffSmem);
    cudaError_t err = cudaFuncSetAttribute(coeff_simt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err != cudaSuccess) return err;
    coeff_simt_kernel<<<grid, 256, smem, L.stream>>>(L.xrec, L.yrec, L.n, L.Mx, L.My, slice, L.S64);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Finish: a = G o (f St g) and the FP32 energy operand K = f a g, zero padded to
// (round_up(Mx, 32), Kld = round_up(My, 128)).
// ---------------------------------------------------------------------------
__global__ void finish_simt_kernel(const double *__restrict__ S64, const float *__restrict__ a_in,
                                   float *__restrict__ a_out, float *__restrict__ K, int Mx, int My,
                                   int Mxp, int Kld, double W, double H, double *__restrict__ a64) {
    const double PI = 3.141592653589793;
    const size_t total = (size_t)Mxp * Kld;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int u = (int)(idx / Kld), v = (int)(idx % Kld);
        float kv = 0.f;
        if (u < Mx && v < My) {
            const double f = 2.0 * W / (PI * (u > 0 ? u : 1));
            const double g = 2.0 * H / (PI * (v > 0 ? v : 1));
            double av;
            if (a_in) {
                av = (double)a_in[(size_t)u * My + v];
            } else {
                const double ku = u * PI / W, lv = v * PI / H;
                const double eps = (u ? 2.0 : 1.0) * (v ? 2.0 : 1.0);
                const double G = (u == 0 && v == 0) ? 0.0 : eps / (W * H * (ku * ku + lv * lv));
                av = G * f * g * S64[(size_t)u * My + v];
                if (a64) {                      // running FP64 sum over calls (chunks, ranks)
                    const double t = a64[(size_t)u * My + v] + av;
                    a64[(size_t)u * My + v] = t;
                    if (a_out) a_out[(size_t)u * My + v] = (float)t;
                } else if (a_out) {
                    a_out[(size_t)u * My + v] = (float)av;
                }
            }
            kv = (float)(f * av * g);
        }
        if (K) K[idx] = kv;
    }
}

cudaError_t launch_finish_simt(const Launch &L, const float *a_in, float *a_out, double *a64, bool with_K) {
    const int Mxp = round_up(L.Mx, kSimtKU);
    const size_t total = (size_t)Mxp * L.Kld;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 8 * L.sm_count) blocks = 8 * L.sm_count;
    finish_simt_kernel<<<blocks, 256, 0, L.stream>>>(L.S64, a_in, a_out, with_K ? (float *)L.K : nullptr,
                                                     L.Mx, L.My, Mxp, L.Kld, L.W, L.H, a64);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Energy and gradient, FP32: CTA = 64 blocks; loops over v tiles of 128 and u
// chunks of 32.  T = Xt K and T' = Xh K accumulate in registers (4 blocks x 8 v
// per thread); the row dots with Yt and Yh run at the end of each v tile.
// ---------------------------------------------------------------------------
constexpr int EB = 64;             // blocks per CTA
constexpr int EU = kSimtKU;        // u chunk
constexpr int EV = kSimtKV;        // v tile
constexpr int XLD = EB + 4;        // padded row of the basis tiles

template <int SAMPLE>
__device__ __forceinline__ void xbasis_run8(const AxisRec &r, int m0, float xt[8], float xh[8]) {
    // SAMPLE 0 (rectangle): Xt = c cos(pi u s) sin(pi u t), Xh = -(u pi/W) c sin sin
    // SAMPLE 1 (centre):    Xt = q cos(pi u s) / f_u,     Xh = -q (u pi/W) sin(pi u s) / f_u
    float2 zs = phase_cs((unsigned long long)m0, r.s);
    if (SAMPLE == 0) {
        float2 zt = phase_cs((unsigned long long)m0, r.t);
        zt.x *= r.c;
        zt.y *= r.c;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float ku = (float)(m0 + j) * r.inv_l;
            xt[j] = zs.x * zt.y;
            xh[j] = -ku * zs.y * zt.y;
            zs = rot(zs, r.es);
            zt = rot(zt, r.et);
        }
        if (m0 == 0) xt[0] = r.v0;
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int m = m0 + j;
            const float ku = (float)m * r.inv_l;
            const float inv_f = 0.5f * (float)(m > 0 ? m : 1) * r.inv_l;   // 1 / f_u
            xt[j] = r.q * zs.x * inv_f;
            xh[j] = -r.q * ku * zs.y * inv_f;
            zs = rot(zs, r.es);
        }
    }
}

template <int SAMPLE>
__device__ __forceinline__ void ybasis_run4(const AxisRec &r, int m0, float yt[4], float yh[4]) {
    // SAMPLE 0: Yt = cos(pi v s) sin(pi v t) (v0 at v = 0), Yh = -(v pi/H) sin sin
    // SAMPLE 1: Yt = cos(pi v s) / g_v,                   Yh = -(v pi/H) sin(pi v s) / g_v
    float2 zs = phase_cs((unsigned long long)m0, r.s);
    if (SAMPLE == 0) {
        float2 zt = phase_cs((unsigned long long)m0, r.t);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float lv = (float)(m0 + j) * r.inv_l;
            yt[j] = zs.x * zt.y;
            yh[j] = -lv * zs.y * zt.y;
            zs = rot(zs, r.es);
            zt = rot(zt, r.et);
        }
        if (m0 == 0) yt[0] = r.v0;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + j;
            const float lv = (float)m * r.inv_l;
            const float inv_g = 0.5f * (float)(m > 0 ? m : 1) * r.inv_l;
            yt[j] = zs.x * inv_g;
            yh[j] = -lv * zs.y * inv_g;
            zs = rot(zs, r.es);
        }
    }
}


struct EnergySmem {
    float Xs[2][EU][XLD];
    float Xh[2][EU][XLD];
    float Ks[2][EU][EV];
    double red[8];
};

template <int SAMPLE>
__global__ void __launch_bounds__(256, 1)
energy_simt_kernel(const AxisRec *__restrict__ xr, const AxisRec *__restrict__ yr, int n, int Mx,
                   int My, const float *__restrict__ K, int Kld, float *__restrict__ e_block,
                   double *__restrict__ e_total, float *__restrict__ gx, float *__restrict__ gy,
                   const GradOut go) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    EnergySmem &sm = *reinterpret_cast<EnergySmem *>(smem_raw);
    auto &Xs = sm.Xs;
    auto &Xh = sm.Xh;
    auto &Ks = sm.Ks;
    auto &red = sm.red;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int blk0 = blockIdx.x * EB;
    // compute mapping: bt = group of 4 blocks, vt = group of 8 v (two runs of 4)
    const int bt = warp * 2 + (lane >> 4);
    const int vt = lane & 15;
    // generator mapping: one block (column), 8 u's (run)
    const int g_run = warp >> 1;                 // u offset g_run*8 in the chunk
    const int g_blk = (warp & 1) * 32 + lane;    // block within the CTA

    const int nuc = (Mx + EU - 1) / EU;
    const int nvt = (My + EV - 1) / EV;
    const int total = nuc * nvt;

    float eN[4] = {0.f, 0.f, 0.f, 0.f}, eX[4] = {0.f, 0.f, 0.f, 0.f}, eY[4] = {0.f, 0.f, 0.f, 0.f};
    // T, T' on pairs of adjacent v (packed f32x2 FMAs, each half rounded as fmaf)
    float2 T[4][4], Tp[4][4];

    const bool g_valid = blk0 + g_blk < n;
    AxisRec grec;
    if (g_valid) grec = xr[blk0 + g_blk];

    // Iteration `it` visits v tiles and u chunks from the highest modes down, so
    // that the decaying terms of K are summed smallest first.
    auto coords = [&](int it, int &vtile, int &uc) {
        vtile = nvt - 1 - it / nuc;
        uc = nuc - 1 - it % nuc;
    };
    auto load_K = [&](int it, int buf) {
        int vtile, uc;
        coords(it, vtile, uc);
        const float *src = K + (size_t)(uc * EU) * Kld + vtile * EV;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = (tid + r * 256) * 4;      // float index within the 32 x 128 tile
            const int row = e / EV, col = e % EV;
            cp_async16(&Ks[buf][row][col], src + (size_t)row * Kld + col);
        }
        cp_async_commit();
    };

    load_K(0, 0);
    for (int it = 0; it < total; ++it) {
        const int buf = it & 1;
        int vtile, uc;
        coords(it, vtile, uc);
        if (uc == nuc - 1) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) T[i][jj] = Tp[i][jj] = make_float2(0.f, 0.f);
        }
        // basis chunk
        {
            float xt[8], xh[8];
            if (g_valid) {
                xbasis_run8<SAMPLE>(grec, uc * EU + g_run * 8, xt, xh);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) xt[j] = xh[j] = 0.f;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                Xs[buf][g_run * 8 + j][g_blk] = xt[j];
                Xh[buf][g_run * 8 + j][g_blk] = xh[j];
            }
        }
        cp_async_wait_all();
        __syncthreads();
        if (it + 1 < total) load_K(it + 1, buf ^ 1);
#pragma unroll 4
        for (int k = EU - 1; k >= 0; --k) {
            const float4 a = *reinterpret_cast<const float4 *>(&Xs[buf][k][bt * 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Xh[buf][k][bt * 4]);
            const float4 k0 = *reinterpret_cast<const float4 *>(&Ks[buf][k][vt * 4]);
            const float4 k1 = *reinterpret_cast<const float4 *>(&Ks[buf][k][64 + vt * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
            const float2 kp[4] = {make_float2(k0.x, k0.y), make_float2(k0.z, k0.w), make_float2(k1.x, k1.y),
                                  make_float2(k1.z, k1.w)};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 ai = make_float2(av[i], av[i]), bi = make_float2(bv[i], bv[i]);
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    T[i][jj] = __ffma2_rn(ai, kp[jj], T[i][jj]);
                    Tp[i][jj] = __ffma2_rn(bi, kp[jj], Tp[i][jj]);
                }
            }
        }
        if (uc == 0) {
            // row dots for this v tile (highest v first)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int b = blk0 + bt * 4 + i;
                if (b >= n) continue;
                const AxisRec ry = yr[b];
#pragma unroll
                for (int half = 1; half >= 0; --half) {
                    const int v0 = vtile * EV + half * 64 + vt * 4;
                    float yt[4], yh[4];
                    ybasis_run4<SAMPLE>(ry, v0, yt, yh);
#pragma unroll
                    for (int j = 3; j >= 0; --j) {
                        if (v0 + j < My) {
                            const float2 t2 = T[i][half * 2 + (j >> 1)], tp2 = Tp[i][half * 2 + (j >> 1)];
                            const float t = (j & 1) ? t2.y : t2.x, tp = (j & 1) ? tp2.y : tp2.x;
                            eN[i] = fmaf(t, yt[j], eN[i]);
                            eY[i] = fmaf(t, yh[j], eY[i]);
                            eX[i] = fmaf(tp, yt[j], eX[i]);
                        }
                    }
                }
            }
        }
    }
    // reduce over the 16 v groups (lanes differing in the low 4 bits)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int off = 8; off >= 1; off >>= 1) {
            eN[i] += __shfl_xor_sync(0xffffffffu, eN[i], off);
            eX[i] += __shfl_xor_sync(0xffffffffu, eX[i], off);
            eY[i] += __shfl_xor_sync(0xffffffffu, eY[i], off);
        }
    }
    double esum = 0.0;
    if (vt == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int b = blk0 + bt * 4 + i;
            if (b < n) {
                if (e_block) e_block[b] = eN[i];
                if (gx) gx[b] = grad_out(go, gx, b, eX[i]);
                if (gy) gy[b] = grad_out(go, gy, b, eY[i]);
                esum += (double)eN[i];
            }
        }
    }
    if (e_total) {
        esum += __shfl_xor_sync(0xffffffffu, esum, 16);
        if (lane == 0) red[warp] = esum;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int k = 0; k < 8; ++k) s += red[k];
            atomicAdd(e_total, 0.5 * s);
        }
    }
}

cudaError_t launch_energy_simt(const Launch &L, int sample, float *e_block, double *e_total,
                               float *gx, float *gy, const GradOut &go) {
    if (L.n == 0) return cudaSuccess;
    const int grid = (L.n + EB - 1) / EB;
    const float *K = (const float *)L.K;
    const int smem = (int)sizeof(EnergySmem);
    cudaError_t err;
    if (sample == 0) {
        err = cudaFuncSetAttribute(energy_simt_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (err != cudaSuccess) return err;
        energy_simt_kernel<0><<<grid, 256, smem, L.stream>>>(L.xrec, L.yrec, L.n, L.Mx, L.My, K, L.Kld,
                                                             e_block, e_total, gx, gy, go);
    } else {
        err = cudaFuncSetAttribute(energy_simt_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (err != cudaSuccess) return err;
        energy_simt_kernel<1><<<grid, 256, smem, L.stream>>>(L.xrec, L.yrec, L.n, L.Mx, L.My, K, L.Kld,
                                                             e_block, e_total, gx, gy, go);
    }
    return cudaGetLastError();
}

}  // namespace pp
