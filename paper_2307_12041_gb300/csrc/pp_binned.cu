// The paper's binned fast scheme (Sec. III-D) on the GPU:
//   bin_density_kernel    P_lj = sum_i c_i area(block i ∩ bin lj) / area(bin)
//   trig_kernel           C[u][l] = cos(u (l + 1/2) pi / m), S[u][l] = sin(...)
//   cuBLAS GEMMs          a' = Cx P Cy^T;  psi = Cx^T a Cy;  xi_x = Sx^T (k o a) Cy;
//                         xi_y = Cx^T (a o l) Sy   (Eq. disa, dis-psi1, dis-ksi)
//   scale_kernel          a = (Eq. disa prefactors) o a';  k o a;  a o l
//   interp_kernel         bilinear weighting of the bin-centre values at each block
//                         centre: N_i = q_i psi_i, grad = -q_i xi_i, E = 1/2 sum N_i
// The transforms are dense products of an m-point cosine / sine matrix with an
// m x m grid: plain GEMMs, issued to cuBLAS (FP32, or TF32 tensor cores).
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "pp_internal.h"

namespace pp {
namespace {

// x * k * 2^40 rounded to the nearest integer (ties away from zero), exact from the
// significands of the float32 x and the positive normal double k, for |x k| < 2^22:
// bin coordinates with 2^-40-bin resolution in integer arithmetic (FP64 is a
// narrow pipe on this GPU).
__device__ __forceinline__ long long fixed_bins(float x, double k) {
    const unsigned xb = __float_as_uint(x);
    const int xe = (int)((xb >> 23) & 0xFFu);
    if ((xb & 0x7FFFFFFFu) == 0u || xe == 0xFF) return 0;
    const unsigned long long mx = (unsigned long long)((xb & 0x7FFFFFu) | (xe ? 0x800000u : 0u));
    const unsigned long long kb = (unsigned long long)__double_as_longlong(k);
    const unsigned long long mk = (kb & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    const int sh = (xe ? xe : 1) - 150 + ((int)((kb >> 52) & 0x7FF) - 1075) + 40;   // value = mx mk 2^sh
    const unsigned long long lo = mx * mk, hi = __umul64hi(mx, mk);
    unsigned long long q;
    if (sh >= 0) {
        q = sh >= 63 ? 0ull : (lo << sh);
    } else {
        const int r = -sh;
        if (r >= 78) q = 0ull;
        else if (r < 64) q = ((lo >> r) | (r ? (hi << (64 - r)) : 0ull)) + ((lo >> (r - 1)) & 1ull);
        else q = (hi >> (r - 64)) + ((r == 64 ? (lo >> 63) : (hi >> (r - 65))) & 1ull);
    }
    return (xb >> 31) ? -(long long)q : (long long)q;
}

__global__ void bin_density_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                   const float *__restrict__ w, const float *__restrict__ h,
                                   const float *__restrict__ c, int n, int m, double inv_wb,
                                   double inv_hb, float *__restrict__ P) {
    constexpr int F = 40;                                 // fraction bits of a bin coordinate
    constexpr long long ONE = 1ll << F;
    const float unit = 0x1p-40f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        // block edges in bin units, exact (2^-40 bins)
        const long long cx = fixed_bins(x[i], inv_wb), hx = fixed_bins(w[i], 0.5 * inv_wb);
        const long long cy = fixed_bins(y[i], inv_hb), hy = fixed_bins(h[i], 0.5 * inv_hb);
        const long long x0 = cx - hx, x1 = cx + hx, y0 = cy - hy, y1 = cy + hy;
        const int l0 = (int)max(0ll, x0 >> F), l1 = (int)min((long long)(m - 1), (x1 - 1) >> F);
        const int j0 = (int)max(0ll, y0 >> F), j1 = (int)min((long long)(m - 1), (y1 - 1) >> F);
        const float ci = c ? c[i] : 1.f;
        for (int l = l0; l <= l1; ++l) {
            const long long ox = min(x1, (long long)(l + 1) * ONE) - max(x0, (long long)l * ONE);
            if (ox <= 0) continue;
            const float cox = ci * ((float)ox * unit);
            for (int j = j0; j <= j1; ++j) {
                const long long oy = min(y1, (long long)(j + 1) * ONE) - max(y0, (long long)j * ONE);
                if (oy <= 0) continue;
                atomicAdd(&P[(size_t)l * m + j], cox * ((float)oy * unit));   // area / bin area
            }
        }
    }
}

// C, S: M x m, angle pi u (2l + 1) / (2m) reduced exactly in integers
__global__ void trig_kernel(int M, int m, float *__restrict__ C, float *__restrict__ S) {
    const long long total = (long long)M * m;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(k / m), l = (int)(k % m);
        const long long q = ((long long)u * (2 * l + 1)) % (4LL * m);   // in units of pi / (2m)
        float s, co;
        sincospif((float)q / (float)(2 * m), &s, &co);
        C[k] = co;
        S[k] = s;
    }
}

// a = prefactor o a' (Eq. disa-a..d), ka = (u pi / W) a, al = a (p pi / H); FP32
__global__ void scale_kernel(int Mx, int My, int m, float W, float H, const float *__restrict__ ap,
                             float *__restrict__ a, float *__restrict__ ka, float *__restrict__ al) {
    const float PI = 3.14159265358979f;
    const float inv_pi3 = 1.f / (PI * PI * PI), inv_pi4 = inv_pi3 / PI;
    const long long total = (long long)Mx * My;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(k / My), p = (int)(k % My);
        const float fu = (float)u, fp = (float)p;
        const float su = sinpif(fu / (2.f * m)), sp = sinpif(fp / (2.f * m));
        float f = 0.f;
        if (u == 0 && p > 0) f = 4.f * H * H * inv_pi3 / (fp * fp * fp * (float)m) * sp;
        else if (p == 0 && u > 0) f = 4.f * W * W * inv_pi3 / (fu * fu * fu * (float)m) * su;
        else if (u > 0 && p > 0)
            f = 16.f * (W * W) * (H * H) * inv_pi4 / (fu * fp * (fu * fu * H * H + fp * fp * W * W)) * su * sp;
        const float av = f * ap[k];
        a[k] = av;
        ka[k] = (fu * PI / W) * av;
        al[k] = av * (fp * PI / H);
    }
}

__global__ void interp_kernel(const float *__restrict__ x, const float *__restrict__ y,
                              const float *__restrict__ w, const float *__restrict__ h,
                              const float *__restrict__ c, int n, int m, float inv_wb, float inv_hb,
                              const float *__restrict__ psi, const float *__restrict__ xix,
                              const float *__restrict__ xiy, float *__restrict__ e_block,
                              float *__restrict__ gx, float *__restrict__ gy, double *__restrict__ e_total) {
    double e = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float fx = fminf(fmaxf(x[i] * inv_wb - 0.5f, 0.f), (float)(m - 1));
        const float fy = fminf(fmaxf(y[i] * inv_hb - 0.5f, 0.f), (float)(m - 1));
        const int l0 = min((int)fx, m - 2), j0 = min((int)fy, m - 2);
        const float tx = fx - (float)l0, ty = fy - (float)j0;
        const size_t k00 = (size_t)l0 * m + j0, k10 = k00 + m, k01 = k00 + 1, k11 = k10 + 1;
        const float w00 = (1.f - tx) * (1.f - ty), w10 = tx * (1.f - ty), w01 = (1.f - tx) * ty, w11 = tx * ty;
        auto at = [&](const float *V) { return w00 * V[k00] + w10 * V[k10] + w01 * V[k01] + w11 * V[k11]; };
        const float q = (c ? c[i] : 1.f) * w[i] * h[i];
        const float Ni = q * at(psi);
        if (e_block) e_block[i] = Ni;
        if (gx) gx[i] = -q * at(xix);
        if (gy) gy[i] = -q * at(xiy);
        e += 0.5 * (double)Ni;
    }
    if (e_total) {
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
        if ((threadIdx.x & 31) == 0) atomicAdd(e_total, e);
    }
}

std::mutex g_cublas_mu;
cublasHandle_t g_cublas[64];

// C = op(A) op(B) on row-major matrices (C: M x N, inner K) through column-major cuBLAS:
// C^T = op(B)^T op(A)^T, the buffers read as their transposes.
cublasStatus_t gemm_rm(cublasHandle_t hd, bool tf32, bool ta, bool tb, int M, int N, int K, const float *A,
                       int lda, const float *B, int ldb, float *C, int ldc) {
    const float one = 1.f, zero = 0.f;
    return cublasGemmEx(hd, tb ? CUBLAS_OP_T : CUBLAS_OP_N, ta ? CUBLAS_OP_T : CUBLAS_OP_N, N, M, K, &one, B,
                        CUDA_R_32F, ldb, A, CUDA_R_32F, lda, &zero, C, CUDA_R_32F, ldc,
                        tf32 ? CUBLAS_COMPUTE_32F_FAST_TF32 : CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
}

}  // namespace

BinnedLayout binned_layout(int m, int Mx, int My) {
    BinnedLayout L{};
    size_t off = 0;
    auto take = [&](size_t count) {
        const size_t o = off;
        off += (count * sizeof(float) + 255) / 256 * 256;
        return o;
    };
    const size_t mm = (size_t)m * m;
    L.P = take(mm);
    L.Cx = take((size_t)Mx * m);
    L.Sx = take((size_t)Mx * m);
    L.Cy = take((size_t)My * m);
    L.Sy = take((size_t)My * m);
    L.T = take((size_t)Mx * m);
    L.ap = take((size_t)Mx * My);
    L.a = take((size_t)Mx * My);
    L.ka = take((size_t)Mx * My);
    L.al = take((size_t)Mx * My);
    L.U = take((size_t)m * My);
    L.psi = take(mm);
    L.xix = take(mm);
    L.xiy = take(mm);
    L.total = off;
    return L;
}

cudaError_t launch_bin_density(const float *x, const float *y, const float *w, const float *h, const float *c,
                               int n, int m, double W, double H, float *P, int sm_count, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    bin_density_kernel<<<8 * sm_count, 256, 0, st>>>(x, y, w, h, c, n, m, m / W, m / H, P);
    return cudaGetLastError();
}

cudaError_t run_binned(const Launch &Lc, int dev, int m, bool tf32, unsigned char *ws, float *a_out, float *e_block,
                       float *gx, float *gy, double *e_total, const char **what) {
    const int Mx = Lc.Mx, My = Lc.My, n = Lc.n;
    const BinnedLayout B = binned_layout(m, Mx, My);
    float *P = (float *)(ws + B.P), *Cx = (float *)(ws + B.Cx), *Sx = (float *)(ws + B.Sx);
    float *Cy = (float *)(ws + B.Cy), *Sy = (float *)(ws + B.Sy), *T = (float *)(ws + B.T);
    float *ap = (float *)(ws + B.ap), *a = a_out ? a_out : (float *)(ws + B.a);
    float *ka = (float *)(ws + B.ka), *al = (float *)(ws + B.al), *U = (float *)(ws + B.U);
    float *psi = (float *)(ws + B.psi), *xix = (float *)(ws + B.xix), *xiy = (float *)(ws + B.xiy);
    cudaStream_t st = Lc.stream;
    *what = "binned scheme launch";
    cudaError_t e = cudaMemsetAsync(P, 0, (size_t)m * m * sizeof(float), st);
    if (e != cudaSuccess) return e;
    if (e_total && (e = cudaMemsetAsync(e_total, 0, sizeof(double), st)) != cudaSuccess) return e;
    const int grid = 8 * Lc.sm_count;
    if (n > 0) {
        bin_density_kernel<<<grid, 256, 0, st>>>(Lc.x, Lc.y, Lc.w, Lc.h, Lc.c, n, m, m / Lc.W, m / Lc.H, P);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    trig_kernel<<<grid, 256, 0, st>>>(Mx, m, Cx, Sx);
    trig_kernel<<<grid, 256, 0, st>>>(My, m, Cy, Sy);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(g_cublas_mu);
        *what = "cuBLAS";
        if (!g_cublas[dev] && cublasCreate(&g_cublas[dev]) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
        cublasHandle_t hd = g_cublas[dev];
        if (cublasSetStream(hd, st) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
        bool ok = true;
        ok &= gemm_rm(hd, tf32, false, false, Mx, m, m, Cx, m, P, m, T, m) == CUBLAS_STATUS_SUCCESS;      // T = Cx P
        ok &= gemm_rm(hd, tf32, false, true, Mx, My, m, T, m, Cy, m, ap, My) == CUBLAS_STATUS_SUCCESS;    // a' = T Cy^T
        if (!ok) return cudaErrorUnknown;
        scale_kernel<<<grid, 256, 0, st>>>(Mx, My, m, (float)Lc.W, (float)Lc.H, ap, a, ka, al);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ok &= gemm_rm(hd, tf32, true, false, m, My, Mx, Cx, m, a, My, U, My) == CUBLAS_STATUS_SUCCESS;     // Cx^T a
        ok &= gemm_rm(hd, tf32, false, false, m, m, My, U, My, Cy, m, psi, m) == CUBLAS_STATUS_SUCCESS;    // psi
        ok &= gemm_rm(hd, tf32, true, false, m, My, Mx, Sx, m, ka, My, U, My) == CUBLAS_STATUS_SUCCESS;    // Sx^T (k a)
        ok &= gemm_rm(hd, tf32, false, false, m, m, My, U, My, Cy, m, xix, m) == CUBLAS_STATUS_SUCCESS;    // xi_x
        ok &= gemm_rm(hd, tf32, true, false, m, My, Mx, Cx, m, al, My, U, My) == CUBLAS_STATUS_SUCCESS;    // Cx^T (a l)
        ok &= gemm_rm(hd, tf32, false, false, m, m, My, U, My, Sy, m, xiy, m) == CUBLAS_STATUS_SUCCESS;    // xi_y
        if (!ok) return cudaErrorUnknown;
    }
    *what = "binned scheme launch";
    if (n > 0) {
        interp_kernel<<<grid, 256, 0, st>>>(Lc.x, Lc.y, Lc.w, Lc.h, Lc.c, n, m, (float)(m / Lc.W),
                                            (float)(m / Lc.H), psi, xix, xiy, e_block, gx, gy, e_total);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace pp
