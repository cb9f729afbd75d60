// The paper's binned fast scheme (Sec. III-D) on the GPU:
//   bin_density_kernel    P_lj = sum_i c_i area(block i ∩ bin lj) / area(bin) (the
//                         interiors of large blocks through a row difference array),
//                         by FP32 atomics, or exactly in 64-bit fixed point
//   row_prefix_add_kernel the difference array's row prefix sums added to P (FP32 path;
//                         the first row transform does it for m = 512, 1024)
//   density_finish_kernel P = the fixed-point accumulators plus the difference array's
//                         row prefix sums, as float (exact path)
//   transform kernels     the cosine / sine transforms of Eq. (disa), (dis-psi1) and
//                         (dis-ksi) along one grid axis at a time, one CTA per row:
//                           a'   = Cx P Cy^T            (DCT-II along j, then along l)
//                           psi  = Cx^T a Cy            (DCT-III along v, then along u)
//                           xi_x = Sx^T (k o a) Cy      (DCT-III along v, DST-III along u)
//                           xi_y = Cx^T (a o l) Sy      (DST-III along v, DCT-III along u)
//                         with C[u][l] = cos(pi u (2l + 1) / 2m), S likewise with sin.
//                         For m a power of two each transform is one m-point complex
//                         FFT in shared memory (the paper computes these transforms with
//                         the FFT: O(m^2 log m) per 2-D transform); other m use a direct
//                         sum over a shared-memory table of cos(pi q / 2m), q < 4m.
//                         A transform whose next step runs along the other axis
//                         writes each row's outputs down a column of that step's
//                         input (no separate transpose).
//   scale_kernel          a = (Eq. disa prefactors) o a', transposing a' to u-major
//   interp_kernel         bilinear weighting of the bin-centre values at each block
//                         centre: N_i = q_i psi_i, grad = -q_i xi_i, E = 1/2 sum N_i
// Every transform runs in FP32.
#include <cuda_runtime.h>

#include <cmath>

#include "pp_internal.h"
#include "pp_sum.cuh"

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

// Blocks covering at most kSmallBins bins are binned by their own thread; larger ones
// (macros: up to thousands of bins) by the whole warp, which takes them one at a time
// (found by a ballot) and shares out their bins, so that one large block does not
// hold its warp for thousands of serial additions.  With a difference array D, a large
// block spans at least 3 bin columns: the bins strictly inside its column range are
// covered fully along y, so row l of the block adds the same c fx(l) to each of them.
// It adds +c fx(l) at D[l][j0 + 1] and -c fx(l) at D[l][j1] instead, its two edge
// columns directly, and the prefix sums of D's rows are added to P afterwards
// (row_prefix_add_kernel, the first row transform, or density_finish_kernel): four
// additions per row of the block instead of one per bin.
constexpr int kSmallBins = 8;

// FIXED: each addition is rounded once to 2^-32 bin areas and summed in 64-bit integers
// (P and D int64), so that the sums are exact and do not depend on the order in which
// the atomics land (FP32 atomics round each partial sum, by an amount that follows that
// order); |P| < 2^31 bin areas.  Else FP32 atomics into float P and D.
constexpr float kFix = 0x1p32f, kUnfix = 0x1p-32f;

template <bool FIXED>
__device__ __forceinline__ void add_bin(void *base, size_t idx, float v) {
    if (FIXED)
        atomicAdd(reinterpret_cast<unsigned long long *>(base) + idx, (unsigned long long)__float2ll_rn(v * kFix));
    else
        atomicAdd(reinterpret_cast<float *>(base) + idx, v);
}

template <bool FIXED>
__global__ void bin_density_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                   const float *__restrict__ w, const float *__restrict__ h,
                                   const float *__restrict__ c, int n, int m, double inv_wb,
                                   double inv_hb, void *__restrict__ P, void *__restrict__ D) {
    constexpr int F = 40;                                 // fraction bits of a bin coordinate
    constexpr long long ONE = 1ll << F;
    const float unit = 0x1p-40f;
    const int lane = threadIdx.x & 31;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    // overlap of block [b0, b1) with bin k, in units of 2^-40 bins
    auto overlap = [&](long long b0, long long b1, int k) {
        return min(b1, (long long)(k + 1) * ONE) - max(b0, (long long)k * ONE);
    };
    // every lane of the warp runs every iteration (the warp-wide steps need them all)
    for (long long base = wid * 32; base < n; base += warps * 32) {
        const long long i = base + lane;
        long long x0 = 0, x1 = 0, y0 = 0, y1 = 0;
        int l0 = 0, l1 = -1, j0 = 0, j1 = -1;
        float ci = 0.f;
        if (i < n) {
            // block edges in bin units, exact (2^-40 bins)
            const long long cx = fixed_bins(x[i], inv_wb), hx = fixed_bins(w[i], 0.5 * inv_wb);
            const long long cy = fixed_bins(y[i], inv_hb), hy = fixed_bins(h[i], 0.5 * inv_hb);
            x0 = cx - hx;
            x1 = cx + hx;
            y0 = cy - hy;
            y1 = cy + hy;
            l0 = (int)max(0ll, x0 >> F);
            l1 = (int)min((long long)(m - 1), (x1 - 1) >> F);
            j0 = (int)max(0ll, y0 >> F);
            j1 = (int)min((long long)(m - 1), (y1 - 1) >> F);
            ci = c ? c[i] : 1.f;
        }
        const long long nl = l1 >= l0 ? l1 - l0 + 1 : 0, nj = j1 >= j0 ? j1 - j0 + 1 : 0;
        const bool large = nl * nj > kSmallBins;
        if (!large && nl > 0 && nj > 0) {
            // along each axis only the first and the last bin can be partly covered; the
            // bins between get the whole bin (1 in bin units), so the 2^-40-unit overlaps
            // are formed and converted twice per axis, not once per bin
            const float ax0 = (float)overlap(x0, x1, l0) * unit, ax1 = (float)overlap(x0, x1, l1) * unit;
            const float ay0 = (float)overlap(y0, y1, j0) * unit, ay1 = (float)overlap(y0, y1, j1) * unit;
            for (int l = l0; l <= l1; ++l) {
                const float fx = l == l0 ? ax0 : (l == l1 ? ax1 : 1.f);
                if (!(fx > 0.f)) continue;
                const float cox = ci * fx;
                for (int j = j0; j <= j1; ++j) {
                    const float fy = j == j0 ? ay0 : (j == j1 ? ay1 : 1.f);
                    if (!(fy > 0.f)) continue;
                    add_bin<FIXED>(P, (size_t)l * m + j, cox * fy);   // area / bin area
                }
            }
        }
        unsigned todo = __ballot_sync(0xffffffffu, large);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const long long bx0 = __shfl_sync(0xffffffffu, x0, src), bx1 = __shfl_sync(0xffffffffu, x1, src);
            const long long by0 = __shfl_sync(0xffffffffu, y0, src), by1 = __shfl_sync(0xffffffffu, y1, src);
            const int bl0 = __shfl_sync(0xffffffffu, l0, src), bj0 = __shfl_sync(0xffffffffu, j0, src);
            const int bnl = (int)__shfl_sync(0xffffffffu, nl, src), bnj = (int)__shfl_sync(0xffffffffu, nj, src);
            const float bc = __shfl_sync(0xffffffffu, ci, src);
            const int bl1 = bl0 + bnl - 1, bj1 = bj0 + bnj - 1;
            // as for small blocks, only the edge bins of each axis can be partly covered
            const float ax0 = (float)overlap(bx0, bx1, bl0) * unit, ax1 = (float)overlap(bx0, bx1, bl1) * unit;
            const float ay0 = (float)overlap(by0, by1, bj0) * unit, ay1 = (float)overlap(by0, by1, bj1) * unit;
            auto fx_of = [&](int l) { return l == bl0 ? ax0 : (l == bl1 ? ax1 : 1.f); };
            auto fy_of = [&](int j) { return j == bj0 ? ay0 : (j == bj1 ? ay1 : 1.f); };
            if (D && bnj >= 3) {
                const int ja = bj0, jb = bj1;
                const float fa = ay0, fb = ay1;
                for (int r = lane; r < bnl; r += 32) {
                    const int l = bl0 + r;
                    const float fx = fx_of(l);
                    if (!(fx > 0.f)) continue;
                    const float cx = bc * fx;
                    const size_t row = (size_t)l * m;
                    if (fa > 0.f) add_bin<FIXED>(P, row + ja, cx * fa);
                    if (fb > 0.f) add_bin<FIXED>(P, row + jb, cx * fb);
                    add_bin<FIXED>(D, row + ja + 1, cx);
                    add_bin<FIXED>(D, row + jb, -cx);
                }
                continue;
            }
            // the block's bins shared out over the lanes: rows of up to 32 bins take
            // 32 / bnj rows per round (lane = row offset * bnj + column), longer rows
            // their columns 32 at a time
            if (bnj <= 32) {
                const int per = 32 / bnj, lr = lane / bnj, j = bj0 + (lane - lr * bnj);
                if (lr < per) {
                    const float fy = fy_of(j);
                    for (int r = lr; r < bnl; r += per) {
                        const int l = bl0 + r;
                        const float fx = fx_of(l);
                        if (fx > 0.f && fy > 0.f) add_bin<FIXED>(P, (size_t)l * m + j, bc * fx * fy);
                    }
                }
            } else {
                for (int l = bl0; l <= bl1; ++l) {
                    const float fx = fx_of(l);
                    for (int j = bj0 + lane; j <= bj1; j += 32) {
                        const float fy = fy_of(j);
                        if (fx > 0.f && fy > 0.f) add_bin<FIXED>(P, (size_t)l * m + j, bc * fx * fy);
                    }
                }
            }
        }
    }
}

// P[l][j] += sum_{j' <= j} D[l][j'] (one CTA of 256 threads per row l, the row in chunks
// of 1,024 in order, each an inclusive scan: 4 values per thread, then the warp and
// block partial sums); D is left as it was.
__global__ void __launch_bounds__(256) row_prefix_add_kernel(const float *__restrict__ D, float *__restrict__ P,
                                                             int m) {
    __shared__ float wsum[8];
    const float *dr = D + (size_t)blockIdx.x * m;
    float *pr = P + (size_t)blockIdx.x * m;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    float carry = 0.f;
    for (int base = 0; base < m; base += 1024) {
        const int j = base + 4 * threadIdx.x;
        float v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = j + q < m ? dr[j + q] : 0.f;
        v[1] += v[0];
        v[2] += v[1];
        v[3] += v[2];
        float t = v[3];                                   // this thread's total; inclusive scan over the warp
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const float o = __shfl_up_sync(0xffffffffu, t, off);
            if (lane >= off) t += o;
        }
        if (lane == 31) wsum[wp] = t;
        __syncthreads();
        float before = carry;                             // chunks before, warps before, lanes before
        for (int k = 0; k < wp; ++k) before += wsum[k];
        before += t - v[3];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (j + q < m) pr[j + q] += before + v[q];
        float chunk = 0.f;
        for (int k = 0; k < 8; ++k) chunk += wsum[k];
        carry += chunk;
        __syncthreads();                                  // wsum is rewritten by the next chunk
    }
}

// P[l][j] = (Pq[l][j] + sum_{j' <= j} Dq[l][j']) 2^-32 as float (one CTA of 256 threads
// per row l, the row in chunks of 1,024 in order, each an inclusive scan of 4 values per
// thread, then the warp and block partial sums; in 64-bit integers, so exact).
__global__ void __launch_bounds__(256) density_finish_kernel(const long long *__restrict__ Pq,
                                                             const long long *__restrict__ Dq,
                                                             float *__restrict__ P, int m) {
    __shared__ long long wsum[8];
    const long long *dr = Dq + (size_t)blockIdx.x * m;
    const long long *qr = Pq + (size_t)blockIdx.x * m;
    float *pr = P + (size_t)blockIdx.x * m;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    long long carry = 0;
    for (int base = 0; base < m; base += 1024) {
        const int j = base + 4 * threadIdx.x;
        long long v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = j + q < m ? dr[j + q] : 0ll;
        v[1] += v[0];
        v[2] += v[1];
        v[3] += v[2];
        long long t = v[3];                               // this thread's total; inclusive scan over the warp
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long o = __shfl_up_sync(0xffffffffu, t, off);
            if (lane >= off) t += o;
        }
        if (lane == 31) wsum[wp] = t;
        __syncthreads();
        long long before = carry;                         // chunks before, warps before, lanes before
        for (int k = 0; k < wp; ++k) before += wsum[k];
        before += t - v[3];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (j + q < m) pr[j + q] = __ll2float_rn(qr[j + q] + before + v[q]) * kUnfix;
        long long chunk = 0;
        for (int k = 0; k < 8; ++k) chunk += wsum[k];
        carry += chunk;
        __syncthreads();                                  // wsum is rewritten by the next chunk
    }
}

// a = prefactor o a' (Eq. disa-a..d), FP32: a[u][p] = f(u, p) a'[p][u] (a' = R2 is
// [My][Mx], a leaves u-major): a transpose through a padded
// 32 x 32 shared tile (reads and writes both coalesced) with the prefactor applied on
// the way out; the sines of the tile's 32 u and 32 p are formed once per tile.
__global__ void scale_kernel(int Mx, int My, int m, float W, float H, const float *__restrict__ apt,
                             float *__restrict__ a) {
    __shared__ float t[32][33];
    __shared__ float s_u[32], s_p[32];
    const float PI = 3.14159265358979f;
    const float inv_pi3 = 1.f / (PI * PI * PI), inv_pi4 = inv_pi3 / PI;
    const int u0 = blockIdx.x * 32, p0 = blockIdx.y * 32;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    if (tid < 32) s_u[tid] = sinpif((float)(u0 + tid) / (2.f * m));
    else if (tid < 64) s_p[tid - 32] = sinpif((float)(p0 + tid - 32) / (2.f * m));
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int p = p0 + k, u = u0 + threadIdx.x;
        if (p < My && u < Mx) t[k][threadIdx.x] = apt[(size_t)p * Mx + u];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int u = u0 + k, p = p0 + threadIdx.x;
        if (u >= Mx || p >= My) continue;
        const float fu = (float)u, fp = (float)p;
        const float su = s_u[k], sp = s_p[threadIdx.x];
        float f = 0.f;
        if (u == 0 && p > 0) f = 4.f * H * H * inv_pi3 / (fp * fp * fp * (float)m) * sp;
        else if (p == 0 && u > 0) f = 4.f * W * W * inv_pi3 / (fu * fu * fu * (float)m) * su;
        else if (u > 0 && p > 0)
            f = 16.f * (W * W) * (H * H) * inv_pi4 / (fu * fp * (fu * fu * H * H + fp * fp * W * W)) * su * sp;
        a[(size_t)u * My + p] = f * t[threadIdx.x][k];
    }
}

// ---------------------------------------------------------------------------
// One-dimensional transforms along rows, one CTA per row.
//   DCT2:  X_u = sum_{l < kin} x_l cos(pi u (2l + 1) / 2m),          u < keep
//   DCT3:  T_l = sum_{u < kin} s_u c_u cos(pi u (2l + 1) / 2m),      l < m
//   DST3:  T_l = sum_{u < kin} s_u c_u sin(pi u (2l + 1) / 2m),      l < m
// with s_u = u * in_scale when in_scale != 0, else 1 (the k_u, l_p factors of
// Eq. dis-ksi applied on the fly).
// FFT form (m a power of two; Makhoul's reordering): DCT2: y_k = x_2k, y_{m-1-k} =
// x_{2k+1}, Y = DFT(y), X_u = Re(e^{-i pi u / 2m} Y_u).  DCT3: Y_u = e^{i pi u / 2m}
// (c_u - i c_{m-u}) (c_m = 0), z = unnormalised inverse DFT(Y), then m x_2k = Re z_k,
// m x_{2k+1} = Re z_{m-1-k} and T_l = (m x_l + c_0) / 2.  DST3: sin(pi u (2l + 1) /
// 2m) = (-1)^l cos(pi (m - u)(2l + 1) / 2m), i.e. the DCT3 of c'_u = c_{m-u} (c'_0 =
// 0) with alternating signs.
// ---------------------------------------------------------------------------
enum { T_DCT2 = 0, T_DCT3 = 1, T_DST3 = 2 };

// Up to three independent row passes of the same sizes in one launch of the warp FFT
// kernels (blockIdx.y picks one): each with its input, output, input scale and, for the
// inverse kernels, its kind (DCT-III, or DST-III when dst is set).  Independent passes
// side by side give the GPU several times the warps of one pass.
struct RowJobs {
    const float *in[3];
    float *out[3];
    float in_scale[3];
    int dst[3];
};
template <typename T>
__device__ __forceinline__ T pick3(const T (&v)[3], int j) {
    return j == 0 ? v[0] : (j == 1 ? v[1] : v[2]);
}
constexpr int T_THREADS = 256;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Twiddle tables of an m-point transform (m a power of two), computed once per
// evaluation: tw[k] = e^{-2 pi i k / m} (k < m/2) and qw[u] = (cos, sin)(pi u / 2m)
// (u < m), from exact arguments.
__global__ void fft_tables_kernel(int m, float2 *__restrict__ tw, float2 *__restrict__ qw) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        float sn, cs;
        if (k < m / 2) {
            sincospif(2.0f * (float)k / (float)m, &sn, &cs);
            tw[k] = make_float2(cs, -sn);
        }
        sincospif((float)k / (float)(2 * m), &sn, &cs);
        qw[k] = make_float2(cs, sn);
    }
}

template <int MODE>
__global__ void __launch_bounds__(T_THREADS) fft_rows_kernel(const float *__restrict__ in, int in_ld, int kin,
                                                           float in_scale, int m, int log2m, int keep,
                                                           float *__restrict__ out, int out_ld, int ostr,
                                                           const float2 *__restrict__ tw_g,
                                                           const float2 *__restrict__ qw) {
    extern __shared__ float2 sm2[];
    float2 *buf = sm2;                 // m values
    float2 *tw = sm2 + m;              // m / 2 twiddles e^{-2 pi i k / m}
    const float *row = in + (size_t)blockIdx.x * in_ld;
    const int half = m >> 1;
    for (int k = threadIdx.x; k < half; k += blockDim.x) tw[k] = tw_g[k];
    auto coef = [&](int u) -> float {                           // s_u c_u, 0 beyond kin
        if (u < 0 || u >= kin) return 0.f;
        const float v = row[u];
        return in_scale != 0.f ? v * ((float)u * in_scale) : v;
    };
    const int shift = 32 - log2m;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        float2 v;
        if (MODE == T_DCT2) {
            const int src = k < half ? 2 * k : 2 * (m - 1 - k) + 1;
            v = make_float2(src < kin ? row[src] : 0.f, 0.f);
        } else {
            // DCT3 of c (MODE DCT3) or of c'_u = c_{m-u}, c'_0 = 0 (MODE DST3)
            const float cu = MODE == T_DCT3 ? coef(k) : (k == 0 ? 0.f : coef(m - k));
            const float cmu = k == 0 ? 0.f : (MODE == T_DCT3 ? coef(m - k) : coef(k));
            const float2 q = qw[k];                                     // (cos, sin)(pi k / 2m)
            v = make_float2(q.x * cu + q.y * cmu, q.y * cu - q.x * cmu);   // e^{i theta} (cu - i cmu)
        }
        buf[__brev((unsigned)k) >> shift] = v;
    }
    __syncthreads();
    // iterative radix-2 decimation in time; DCT2 forward, DCT3 / DST3 inverse (conjugate twiddles)
    for (int s = 1; s <= log2m; ++s) {
        const int hs = 1 << (s - 1), step = m >> s;
        for (int b = threadIdx.x; b < half; b += blockDim.x) {
            const int pos = b & (hs - 1);
            const int i = ((b >> (s - 1)) << s) + pos, j = i + hs;
            float2 w = tw[pos * step];
            if (MODE != T_DCT2) w.y = -w.y;
            const float2 t = cmul(w, buf[j]);
            const float2 x = buf[i];
            buf[i] = make_float2(x.x + t.x, x.y + t.y);
            buf[j] = make_float2(x.x - t.x, x.y - t.y);
        }
        __syncthreads();
    }
    float *orow = out + (size_t)blockIdx.x * out_ld;
    if (MODE == T_DCT2) {
        for (int u = threadIdx.x; u < keep; u += blockDim.x) {
            const float2 q = qw[u];
            orow[(size_t)u * ostr] = buf[u].x * q.x + buf[u].y * q.y;
        }
    } else {
        const float c0 = MODE == T_DCT3 ? coef(0) : 0.f;
        for (int l = threadIdx.x; l < m; l += blockDim.x) {
            const float mx = (l & 1) ? buf[m - 1 - (l >> 1)].x : buf[l >> 1].x;
            const float t = 0.5f * (mx + c0);
            orow[(size_t)l * ostr] = (MODE == T_DST3 && (l & 1)) ? -t : t;
        }
    }
}

// The same transforms for m = 32 R (R = 16, 32), one warp per row and no block-wide
// barrier after the tables: the four-step FFT with n = R n1 + n2 and k = k1 + 32 k2,
//   Y_k = sum_n y_n W^{nk} = sum_{n2} W_R^{n2 k2} W_m^{n2 k1} sum_{n1} y_{R n1 + n2} W_32^{n1 k1}
// (W = e^{-2 pi i / m}, conjugated for the inverse transforms).  Lane n1 holds y_{R n1 + n2}
// for every n2 in registers; the 32-point transforms run across the lanes (decimation in
// frequency by shuffles, leaving lane L with k1 = bitreverse5(L)); then the twiddle, then
// an R-point decimation-in-frequency transform in registers (leaving k2 bit-reversed).
// The row comes in and the results go out through the warp's shared-memory buffer, padded
// by one word per 32 (pad()), so that global accesses are coalesced and the lanes' strided
// shared-memory accesses fall in distinct banks.  The pre- and post-processing of the
// DCT-II / DCT-III / DST-III are those of fft_rows_kernel.
__device__ __forceinline__ int pad(int i) { return i + (i >> 5); }

template <int MODE, int R>
__global__ void __launch_bounds__(128) fft_rows_warp_kernel(const RowJobs jobs, int in_ld, int kin, int nrows,
                                                           int keep, int out_ld, int ostr,
                                                           const float2 *__restrict__ tw_g,
                                                           const float2 *__restrict__ qw_g,
                                                           const float *__restrict__ dif) {
    constexpr int m = 32 * R, half = m / 2, mp = m + m / 32;
    constexpr bool INV = MODE != T_DCT2;
    const float *__restrict__ in = pick3(jobs.in, blockIdx.y);
    float *__restrict__ out = pick3(jobs.out, blockIdx.y);
    const float in_scale = pick3(jobs.in_scale, blockIdx.y);
    const bool DST = INV && pick3(jobs.dst, blockIdx.y) != 0;
    __shared__ float2 tw[m];                                 // W^k (e^{-+2 pi i k / m}), k < m
    __shared__ float2 qw[mp];                                // (cos, sin)(pi u / 2m) at pad(u)
    __shared__ float xs[4][mp];                              // one row per warp, at pad(i)
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        float2 w = k < half ? tw_g[k] : make_float2(-tw_g[k - half].x, -tw_g[k - half].y);
        if (INV) w.y = -w.y;
        tw[k] = w;
        qw[pad(k)] = qw_g[k];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int r = blockIdx.x * 4 + wp;
    const bool live = r < nrows;                             // warp-uniform
    if (live) {
        float *xw = xs[wp];
        const float *row = in + (size_t)r * in_ld;
        for (int i = lane; i < kin; i += 32) {
            const float v = row[i];
            xw[pad(i)] = (MODE != T_DCT2 && in_scale != 0.f) ? v * ((float)i * in_scale) : v;   // s_u c_u
        }
        if (MODE == T_DCT2 && dif) {
            // the bin density's row: plus the prefix sums of the difference array's row (the
            // large blocks' interiors, bin_density_kernel); lane L sums entries R L .. R L + R - 1
            __syncwarp();
            const float4 *d4 = reinterpret_cast<const float4 *>(dif + (size_t)r * in_ld + R * lane);
            float pre[R];
    #pragma unroll
            for (int q = 0; q < R / 4; ++q) {
                const float4 v = d4[q];
                pre[4 * q] = v.x;
                pre[4 * q + 1] = v.y;
                pre[4 * q + 2] = v.z;
                pre[4 * q + 3] = v.w;
            }
    #pragma unroll
            for (int q = 1; q < R; ++q) pre[q] += pre[q - 1];
            float t = pre[R - 1];                                // inclusive scan of the lanes' totals
    #pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const float o = __shfl_up_sync(0xffffffffu, t, off);
                if (lane >= off) t += o;
            }
            const float before = t - pre[R - 1];
    #pragma unroll
            for (int q = 0; q < R; ++q) xw[pad(R * lane + q)] += before + pre[q];
        }
        __syncwarp();
        auto W = [&](int j) -> float2 { return tw[j & (m - 1)]; };   // W^j, any j >= 0
        auto coef = [&](int u) -> float { return u >= 0 && u < kin ? xw[pad(u)] : 0.f; };
        float2 a[R];
    #pragma unroll
        for (int n2 = 0; n2 < R; ++n2) {
            const int n = R * lane + n2;
            if (MODE == T_DCT2) {
                const int src = n < half ? 2 * n : 2 * (m - 1 - n) + 1;
                a[n2] = make_float2(coef(src), 0.f);
            } else {
                const float cu = !DST ? coef(n) : (n == 0 ? 0.f : coef(m - n));
                const float cmu = n == 0 ? 0.f : (!DST ? coef(m - n) : coef(n));
                const float2 q = qw[pad(n)];
                a[n2] = make_float2(q.x * cu + q.y * cmu, q.y * cu - q.x * cmu);
            }
        }
        const float c0 = INV && !DST ? coef(0) : 0.f;
        // 32-point transforms across the lanes: pairs (i, i + h), i with bit h clear:
        // y_i <- y_i + y_{i+h}, y_{i+h} <- (y_i - y_{i+h}) W_{2h}^{i mod h}
    #pragma unroll
        for (int h = 16; h >= 1; h >>= 1) {
            // y_i + y_{i+h} = (o + a) * 1 on the lanes with bit h clear, (o - a) W otherwise
            const bool hi = (lane & h) != 0;
            const float sg = hi ? -1.f : 1.f;
            const float2 w = hi ? W((lane & (h - 1)) * (m / (2 * h))) : make_float2(1.f, 0.f);
    #pragma unroll
            for (int n2 = 0; n2 < R; ++n2) {
                const float ox = __shfl_xor_sync(0xffffffffu, a[n2].x, h);
                const float oy = __shfl_xor_sync(0xffffffffu, a[n2].y, h);
                a[n2] = cmul(make_float2(fmaf(sg, a[n2].x, ox), fmaf(sg, a[n2].y, oy)), w);
            }
        }
        const int k1 = (int)(__brev((unsigned)lane) >> 27);
    #pragma unroll
        for (int n2 = 1; n2 < R; ++n2) a[n2] = cmul(a[n2], W(n2 * k1));
        // R-point transforms in registers, the same butterflies with compile-time indices
    #pragma unroll
        for (int h = R / 2; h >= 1; h >>= 1) {
    #pragma unroll
            for (int i = 0; i < R; ++i) {
                if (i & h) continue;
                const float2 u = a[i], v = a[i + h];
                a[i] = make_float2(u.x + v.x, u.y + v.y);
                a[i + h] = cmul(make_float2(u.x - v.x, u.y - v.y), W((i & (h - 1)) * (m / (2 * h))));
            }
        }
        // a[j] = Y_k, k = k1 + 32 bitreverse(j) over log2 R bits: results to the warp buffer at
        // their output positions, then out in order
        constexpr int LR = R == 16 ? 4 : 5;
        __syncwarp();                                            // every lane has read its inputs
    #pragma unroll
        for (int j = 0; j < R; ++j) {
            const int k = k1 + 32 * (int)(__brev((unsigned)j) >> (32 - LR));
            if (MODE == T_DCT2) {
                const float2 q = qw[pad(k)];
                xw[pad(k)] = a[j].x * q.x + a[j].y * q.y;
            } else {
                const int l = k < half ? 2 * k : 2 * (m - 1 - k) + 1;
                const float t = 0.5f * (a[j].x + c0);
                xw[pad(l)] = (DST && (l & 1)) ? -t : t;
            }
        }
        __syncwarp();
    }
    const int nout = MODE == T_DCT2 ? keep : m;
    if (out_ld != 1) {
        if (live) {
            float *orow = out + (size_t)r * out_ld;
            for (int i = lane; i < nout; i += 32) orow[(size_t)i * ostr] = xs[wp][pad(i)];
        }
        return;
    }
    // transposed output (out_ld = 1: row r's outputs go down column r): the CTA's four
    // rows are adjacent there and are written together, 16 bytes per output index
    __syncthreads();
    const int r0 = blockIdx.x * 4;
    const bool vec = r0 + 3 < nrows && (ostr & 3) == 0 && ((uintptr_t)out & 15) == 0;
    for (int i = threadIdx.x; i < nout; i += blockDim.x) {
        float *o = out + (size_t)i * ostr + r0;
        if (vec) {
            *reinterpret_cast<float4 *>(o) = make_float4(xs[0][pad(i)], xs[1][pad(i)], xs[2][pad(i)], xs[3][pad(i)]);
        } else {
            for (int q = 0; q < 4 && r0 + q < nrows; ++q) o[q] = xs[q][pad(i)];
        }
    }
}

// m = 1024 with two warps per row (twice the warps of fft_rows_warp_kernel, half the
// registers each).  Warp h of a row holds n2 in [16 h, 16 h + 16) and runs the 32-point
// transforms across the lanes and the twiddle for those.  The 32-point transform over n2
// begins with the butterflies (n2, n2 + 16), which pair the two warps, so they exchange
// their values once through shared memory:
//   warp 0:  u_i = y_i + y_{i+16}                 -> Y_{k1 + 32 (2q)},     16-point over i
//   warp 1:  v_i = (y_i - y_{i+16}) W_32^i        -> Y_{k1 + 32 (2q + 1)}, 16-point over i
// (i < 16).  Named barrier 1 + (row within the CTA) joins the row's two warps.
template <int MODE>
__global__ void __launch_bounds__(128) fft_rows_pair_kernel(const RowJobs jobs, int in_ld, int kin, int nrows,
                                                           int keep, int out_ld, int ostr,
                                                           const float2 *__restrict__ tw_g,
                                                           const float2 *__restrict__ qw_g,
                                                           const float *__restrict__ dif) {
    constexpr int R = 32, H = 16, m = 32 * R, half = m / 2, mp = m + m / 32;
    constexpr bool INV = MODE != T_DCT2;
    const float *__restrict__ in = pick3(jobs.in, blockIdx.y);
    float *__restrict__ out = pick3(jobs.out, blockIdx.y);
    const float in_scale = pick3(jobs.in_scale, blockIdx.y);
    const bool DST = INV && pick3(jobs.dst, blockIdx.y) != 0;
    __shared__ float2 tw[m];                                 // W^k (e^{-+2 pi i k / m}), k < m
    __shared__ float2 qw[mp];                                // (cos, sin)(pi u / 2m) at pad(u)
    __shared__ float xs[2][mp];                              // one row per warp pair, at pad(i)
    __shared__ float2 xch[2][2][H][32];                      // [row][warp][i][lane]
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        float2 w = k < half ? tw_g[k] : make_float2(-tw_g[k - half].x, -tw_g[k - half].y);
        if (INV) w.y = -w.y;
        tw[k] = w;
        qw[pad(k)] = qw_g[k];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int rr = wp >> 1, h = wp & 1;                      // row within the CTA, warp within the row
    const int r = blockIdx.x * 2 + rr;
    const bool live = r < nrows;                             // the same for the row's two warps
    if (live) {
        const int bar = 1 + rr;
        auto row_sync = [&]() { asm volatile("bar.sync %0, 64;" ::"r"(bar) : "memory"); };
        float *xw = xs[rr];
        const float *row = in + (size_t)r * in_ld;
        for (int i = threadIdx.x & 63; i < kin; i += 64) {
            const float v = row[i];
            xw[pad(i)] = (MODE != T_DCT2 && in_scale != 0.f) ? v * ((float)i * in_scale) : v;   // s_u c_u
        }
        if (MODE == T_DCT2 && dif) {
            // the difference array's row prefix sums (as fft_rows_warp_kernel), by warp 0 of the row
            row_sync();
            if (h == 0) {
                const float4 *d4 = reinterpret_cast<const float4 *>(dif + (size_t)r * in_ld + R * lane);
                float pre[R];
    #pragma unroll
                for (int q = 0; q < R / 4; ++q) {
                    const float4 v = d4[q];
                    pre[4 * q] = v.x;
                    pre[4 * q + 1] = v.y;
                    pre[4 * q + 2] = v.z;
                    pre[4 * q + 3] = v.w;
                }
    #pragma unroll
                for (int q = 1; q < R; ++q) pre[q] += pre[q - 1];
                float t = pre[R - 1];
    #pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const float o = __shfl_up_sync(0xffffffffu, t, off);
                    if (lane >= off) t += o;
                }
                const float before = t - pre[R - 1];
    #pragma unroll
                for (int q = 0; q < R; ++q) xw[pad(R * lane + q)] += before + pre[q];
            }
        }
        row_sync();
        auto W = [&](int j) -> float2 { return tw[j & (m - 1)]; };   // W^j, any j >= 0
        auto coef = [&](int u) -> float { return u >= 0 && u < kin ? xw[pad(u)] : 0.f; };
        float2 a[H];
    #pragma unroll
        for (int i = 0; i < H; ++i) {
            const int n = R * lane + H * h + i;
            if (MODE == T_DCT2) {
                const int src = n < half ? 2 * n : 2 * (m - 1 - n) + 1;
                a[i] = make_float2(coef(src), 0.f);
            } else {
                const float cu = !DST ? coef(n) : (n == 0 ? 0.f : coef(m - n));
                const float cmu = n == 0 ? 0.f : (!DST ? coef(m - n) : coef(n));
                const float2 q = qw[pad(n)];
                a[i] = make_float2(q.x * cu + q.y * cmu, q.y * cu - q.x * cmu);
            }
        }
        const float c0 = INV && !DST ? coef(0) : 0.f;
    #pragma unroll
        for (int hh = 16; hh >= 1; hh >>= 1) {
            const bool hi = (lane & hh) != 0;
            const float sg = hi ? -1.f : 1.f;
            const float2 w = hi ? W((lane & (hh - 1)) * (m / (2 * hh))) : make_float2(1.f, 0.f);
    #pragma unroll
            for (int i = 0; i < H; ++i) {
                const float ox = __shfl_xor_sync(0xffffffffu, a[i].x, hh);
                const float oy = __shfl_xor_sync(0xffffffffu, a[i].y, hh);
                a[i] = cmul(make_float2(fmaf(sg, a[i].x, ox), fmaf(sg, a[i].y, oy)), w);
            }
        }
        const int k1 = (int)(__brev((unsigned)lane) >> 27);
    #pragma unroll
        for (int i = 0; i < H; ++i) {
            const int n2 = H * h + i;
            if (n2 > 0) a[i] = cmul(a[i], W(n2 * k1));
        }
        // the first butterflies of the 32-point transform over n2, across the row's two warps
    #pragma unroll
        for (int i = 0; i < H; ++i) xch[rr][h][i][lane] = a[i];
        row_sync();
    #pragma unroll
        for (int i = 0; i < H; ++i) {
            const float2 o = xch[rr][1 - h][i][lane];
            if (h == 0) a[i] = make_float2(a[i].x + o.x, a[i].y + o.y);                          // y_i + y_{i+16}
            else a[i] = cmul(make_float2(o.x - a[i].x, o.y - a[i].y), W(i * (m / 32)));          // (y_i - y_{i+16}) W_32^i
        }
        // 16-point transforms in registers (W_16 = W_m^{m/16})
    #pragma unroll
        for (int hh = H / 2; hh >= 1; hh >>= 1) {
    #pragma unroll
            for (int i = 0; i < H; ++i) {
                if (i & hh) continue;
                const float2 u = a[i], v = a[i + hh];
                a[i] = make_float2(u.x + v.x, u.y + v.y);
                a[i + hh] = cmul(make_float2(u.x - v.x, u.y - v.y), W((i & (hh - 1)) * (m / (2 * hh))));
            }
        }
        // a[j] = Y_k, k = k1 + 32 (2 bitreverse4(j) + h); every lane of both warps has read its
        // inputs (before the exchange barrier), so the row buffer takes the results
    #pragma unroll
        for (int j = 0; j < H; ++j) {
            const int k = k1 + 32 * (2 * (int)(__brev((unsigned)j) >> 28) + h);
            if (MODE == T_DCT2) {
                const float2 q = qw[pad(k)];
                xw[pad(k)] = a[j].x * q.x + a[j].y * q.y;
            } else {
                const int l = k < half ? 2 * k : 2 * (m - 1 - k) + 1;
                const float t = 0.5f * (a[j].x + c0);
                xw[pad(l)] = (DST && (l & 1)) ? -t : t;
            }
        }
        row_sync();
    }
    const int nout = MODE == T_DCT2 ? keep : m;
    if (out_ld != 1) {
        if (live) {
            float *orow = out + (size_t)r * out_ld;
            for (int i = threadIdx.x & 63; i < nout; i += 64) orow[(size_t)i * ostr] = xs[rr][pad(i)];
        }
        return;
    }
    // transposed output (out_ld = 1: row r's outputs go down column r): the CTA's two
    // rows are adjacent there and are written together, 8 bytes per output index
    __syncthreads();
    const int r0 = blockIdx.x * 2;
    const bool vec = r0 + 1 < nrows && (ostr & 1) == 0 && ((uintptr_t)out & 7) == 0;
    for (int i = threadIdx.x; i < nout; i += blockDim.x) {
        float *o = out + (size_t)i * ostr + r0;
        if (vec) {
            *reinterpret_cast<float2 *>(o) = make_float2(xs[0][pad(i)], xs[1][pad(i)]);
        } else {
            for (int q = 0; q < 2 && r0 + q < nrows; ++q) o[q] = xs[q][pad(i)];
        }
    }
}

// The same transforms for any m: direct sums over a table cos(pi q / 2m), q < 4m
// (sin(pi q / 2m) = cos(pi (q - m) / 2m)); the phase u (2l + 1) is kept mod 4m in
// integers.
template <int MODE>
__global__ void __launch_bounds__(T_THREADS) direct_rows_kernel(const float *__restrict__ in, int in_ld, int kin,
                                                              float in_scale, int m, int keep,
                                                              float *__restrict__ out, int out_ld, int ostr) {
    extern __shared__ float smf[];
    float *tab = smf;                  // 4m
    float *x = smf + 4 * m;            // the row's inputs (kin of them)
    const float *row = in + (size_t)blockIdx.x * in_ld;
    const int m4 = 4 * m;
    for (int q = threadIdx.x; q < m4; q += blockDim.x) tab[q] = cospif((float)q / (float)(2 * m));
    for (int u = threadIdx.x; u < kin; u += blockDim.x) {
        const float v = row[u];
        x[u] = (MODE != T_DCT2 && in_scale != 0.f) ? v * ((float)u * in_scale) : v;
    }
    __syncthreads();
    float *orow = out + (size_t)blockIdx.x * out_ld;
    if (MODE == T_DCT2) {
        for (int u = threadIdx.x; u < keep; u += blockDim.x) {
            float acc = 0.f;
            int q = u % m4;                          // u (2l + 1) at l = 0
            const int dq = (2 * u) % m4;
            for (int l = 0; l < kin; ++l) {
                acc = fmaf(x[l], tab[q], acc);
                q += dq;
                if (q >= m4) q -= m4;
            }
            orow[(size_t)u * ostr] = acc;
        }
    } else {
        for (int l = threadIdx.x; l < m; l += blockDim.x) {
            float acc = 0.f;
            const int dq = 2 * l + 1;                // phase step per u
            int q = MODE == T_DST3 ? m4 - m : 0;     // u (2l + 1) - m (sine) at u = 0, mod 4m
            for (int u = 0; u < kin; ++u) {
                acc = fmaf(x[u], tab[q], acc);
                q += dq;
                if (q >= m4) q -= m4;
            }
            orow[(size_t)l * ostr] = acc;
        }
    }
}

__global__ void interp_kernel(const float *__restrict__ x, const float *__restrict__ y,
                              const float *__restrict__ w, const float *__restrict__ h,
                              const float *__restrict__ c, int n, int m, float inv_wb, float inv_hb,
                              const float4 *__restrict__ V, float *__restrict__ e_block,
                              float *__restrict__ gx, float *__restrict__ gy, double *__restrict__ e_total) {
    Sum2 e;                            // sum of N_i (compensated); E = half of it
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float fx = fminf(fmaxf(x[i] * inv_wb - 0.5f, 0.f), (float)(m - 1));
        const float fy = fminf(fmaxf(y[i] * inv_hb - 0.5f, 0.f), (float)(m - 1));
        const int l0 = min((int)fx, m - 2), j0 = min((int)fy, m - 2);
        const float tx = fx - (float)l0, ty = fy - (float)j0;
        // bin-centre values (psi, xi_x, xi_y) at (l, j) are V[j * m + l]
        const size_t k00 = (size_t)j0 * m + l0, k10 = k00 + 1, k01 = k00 + m, k11 = k01 + 1;
        const float w00 = (1.f - tx) * (1.f - ty), w10 = tx * (1.f - ty), w01 = (1.f - tx) * ty, w11 = tx * ty;
        const float4 v00 = V[k00], v10 = V[k10], v01 = V[k01], v11 = V[k11];
        const float psi = w00 * v00.x + w10 * v10.x + w01 * v01.x + w11 * v11.x;
        const float xix = w00 * v00.y + w10 * v10.y + w01 * v01.y + w11 * v11.y;
        const float xiy = w00 * v00.z + w10 * v10.z + w01 * v01.z + w11 * v11.z;
        const float q = (c ? c[i] : 1.f) * w[i] * h[i];
        const float Ni = q * psi;
        if (e_block) e_block[i] = Ni;
        if (gx) gx[i] = -q * xix;
        if (gy) gy[i] = -q * xiy;
        add2(e, Ni);
    }
    if (e_total) block_add2(e, e_total, 0.5);      // one atomic per CTA
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
    L.P = take(mm);                      // the density, float
    L.D = take(4 * mm);                  // float D, or the int64 accumulators Pq, Dq (exact sums)
    L.R1t = take((size_t)My * m);
    L.R2 = take((size_t)My * Mx);
    L.a = take((size_t)Mx * My);
    L.Ut = take((size_t)m * Mx);
    L.Upt = take((size_t)m * Mx);
    L.V = take(4 * mm);
    L.tab = take(3 * (size_t)m);         // m/2 + m complex twiddles
    L.total = off;
    return L;
}

cudaError_t launch_bin_density(const float *x, const float *y, const float *w, const float *h, const float *c,
                               int n, int m, double W, double H, float *P, int sm_count, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    bin_density_kernel<false><<<8 * sm_count, 256, 0, st>>>(x, y, w, h, c, n, m, m / W, m / H, P, nullptr);
    return cudaGetLastError();
}

namespace {

bool pow2(int m) { return m > 0 && (m & (m - 1)) == 0; }
bool warp_fft(int m) { return m == 512 || m == 1024; }

// Row transforms, FFT when m is a power of two (one warp per row for m = 512, two for
// m = 1024, all jobs in one launch; one CTA per row and one launch per job otherwise).
// `fwd`: DCT-II; else each job's DCT-III or DST-III (RowJobs::dst).  Rows `nrows` of
// each job's input transformed; output element k of row r at out[r * out_ld + k * ostr].
// dif (DCT-II with the warp FFT only): row prefix sums added to the input rows.
cudaError_t rows(bool fwd, const RowJobs &J, int njobs, int in_ld, int nrows, int kin, int m, int keep,
                 int out_ld, int ostr, const float2 *tw, const float2 *qw, cudaStream_t st,
                 const float *dif = nullptr) {
    if (nrows <= 0 || njobs <= 0) return cudaSuccess;
    if (njobs > 3) return cudaErrorInvalidValue;
    if (warp_fft(m)) {
        const int per_cta = m == 512 ? 4 : 2;
        const dim3 grid((nrows + per_cta - 1) / per_cta, njobs);
        if (m == 512) {
            if (fwd) fft_rows_warp_kernel<T_DCT2, 16><<<grid, 128, 0, st>>>(J, in_ld, kin, nrows, keep, out_ld, ostr,
                                                                            tw, qw, dif);
            else fft_rows_warp_kernel<T_DCT3, 16><<<grid, 128, 0, st>>>(J, in_ld, kin, nrows, keep, out_ld, ostr, tw,
                                                                        qw, dif);
        } else {
            if (fwd) fft_rows_pair_kernel<T_DCT2><<<grid, 128, 0, st>>>(J, in_ld, kin, nrows, keep, out_ld, ostr, tw,
                                                                        qw, dif);
            else fft_rows_pair_kernel<T_DCT3><<<grid, 128, 0, st>>>(J, in_ld, kin, nrows, keep, out_ld, ostr, tw, qw,
                                                                    dif);
        }
        return cudaGetLastError();
    }
    for (int j = 0; j < njobs; ++j) {
        const int mode = fwd ? T_DCT2 : (J.dst[j] ? T_DST3 : T_DCT3);
        const float *in = J.in[j];
        float *out = J.out[j];
        const float in_scale = J.in_scale[j];
        cudaError_t e;
        if (pow2(m)) {
            int lg = 0;
            while ((1 << lg) < m) ++lg;
            const size_t smem = (size_t)(m + m / 2) * sizeof(float2);
            auto go = [&](auto kfn) {
                cudaError_t r = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (r != cudaSuccess) return r;
                kfn<<<nrows, T_THREADS, smem, st>>>(in, in_ld, kin, in_scale, m, lg, keep, out, out_ld, ostr, tw,
                                                    qw);
                return cudaGetLastError();
            };
            e = mode == T_DCT2 ? go(fft_rows_kernel<T_DCT2>)
                               : (mode == T_DCT3 ? go(fft_rows_kernel<T_DCT3>) : go(fft_rows_kernel<T_DST3>));
        } else {
            const size_t smem = (size_t)(4 * m + kin) * sizeof(float);
            auto go = [&](auto kfn) {
                cudaError_t r = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (r != cudaSuccess) return r;
                kfn<<<nrows, T_THREADS, smem, st>>>(in, in_ld, kin, in_scale, m, keep, out, out_ld, ostr);
                return cudaGetLastError();
            };
            e = mode == T_DCT2 ? go(direct_rows_kernel<T_DCT2>)
                               : (mode == T_DCT3 ? go(direct_rows_kernel<T_DCT3>) : go(direct_rows_kernel<T_DST3>));
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t run_binned(const Launch &Lc, int dev, int m, bool tf32, unsigned char *ws, float *a_out, float *e_block,
                       float *gx, float *gy, double *e_total, const char **what) {
    (void)dev;
    // the transforms are FP32 FFTs (or direct sums) in either precision; PP_FP32 sums the
    // density exactly in 64-bit fixed point (deterministic), PP_TF32 by FP32 atomics
    const bool exact = !tf32;
    const int Mx = Lc.Mx, My = Lc.My, n = Lc.n;
    const BinnedLayout B = binned_layout(m, Mx, My);
    float *P = (float *)(ws + B.P), *R1t = (float *)(ws + B.R1t);
    float *R2 = (float *)(ws + B.R2), *a = a_out ? a_out : (float *)(ws + B.a);
    float *Ut = (float *)(ws + B.Ut);
    float *Upt = (float *)(ws + B.Upt);
    float *V = (float *)(ws + B.V);
    float2 *tw = (float2 *)(ws + B.tab), *qw = tw + m / 2;
    cudaStream_t st = Lc.stream;
    *what = "binned scheme launch";
    float *D = (float *)(ws + B.D);                             // float path
    long long *Pq = (long long *)(ws + B.D), *Dq = Pq + (size_t)m * m;   // exact path
    cudaError_t e;
    const int grid = 8 * Lc.sm_count;
    if (exact) {
        // int64 accumulators (bin areas x 2^32; Dq the large blocks' row differences),
        // summed exactly, then P = float(Pq + row prefix sums of Dq) 2^-32
        if ((e = cudaMemsetAsync(Pq, 0, 2 * (size_t)m * m * sizeof(long long), st)) != cudaSuccess) return e;
        if (n > 0) {
            bin_density_kernel<true><<<grid, 256, 0, st>>>(Lc.x, Lc.y, Lc.w, Lc.h, Lc.c, n, m, m / Lc.W,
                                                           m / Lc.H, Pq, Dq);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        density_finish_kernel<<<m, 256, 0, st>>>(Pq, Dq, P, m);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else {
        // P and D are consecutive: one memset for both
        if ((e = cudaMemsetAsync(P, 0, B.D - B.P + (size_t)m * m * sizeof(float), st)) != cudaSuccess) return e;
        if (n > 0) {
            bin_density_kernel<false><<<grid, 256, 0, st>>>(Lc.x, Lc.y, Lc.w, Lc.h, Lc.c, n, m, m / Lc.W,
                                                            m / Lc.H, P, D);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if (!warp_fft(m)) {        // else added by the first row transform
                row_prefix_add_kernel<<<m, 256, 0, st>>>(D, P, m);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
        }
    }
    if (e_total && (e = cudaMemsetAsync(e_total, 0, sizeof(double), st)) != cudaSuccess) return e;
    const float kW = (float)(3.141592653589793 / Lc.W), lH = (float)(3.141592653589793 / Lc.H);
    if (pow2(m)) {
        fft_tables_kernel<<<(m + 255) / 256, 256, 0, st>>>(m, tw, qw);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
#define PP_STEP(expr)                              \
    do {                                           \
        if ((e = (expr)) != cudaSuccess) return e; \
    } while (0)
    // a' = Cx P Cy^T: along j (rows l of P, each row's outputs written down a column of
    // R1t, so that no transpose is needed), then along l
    {
        const RowJobs j1{{P}, {R1t}, {0.f}, {0}};
        PP_STEP(rows(true, j1, 1, m, m, m, m, My, 1, m, tw, qw, st, (n > 0 && !exact) ? D : nullptr));
        const RowJobs j2{{R1t}, {R2}, {0.f}, {0}};
        PP_STEP(rows(true, j2, 1, m, My, m, m, Mx, Mx, 1, tw, qw, st));
    }
    scale_kernel<<<dim3((Mx + 31) / 32, (My + 31) / 32), dim3(32, 8), 0, st>>>(Mx, My, m, (float)Lc.W, (float)Lc.H,
                                                                             R2, a);
    PP_STEP(cudaGetLastError());
    // along v (rows u of a), both in one launch: U = a Cy (psi, xi_x), Up = (a o l) Sy
    // (xi_y), written transposed (Ut[j][u], Upt[j][u])
    {
        const RowJobs j3{{a, a}, {Ut, Upt}, {0.f, lH}, {0, 1}};
        PP_STEP(rows(false, j3, 2, My, Mx, My, m, m, 1, Mx, tw, qw, st));
    }
    // along u (rows j), the three in one launch: psi = Cx^T U, xi_x = Sx^T (k o U),
    // xi_y = Cx^T Up, stored interleaved as V[j][l] = (psi, xi_x, xi_y, unused) so that the
    // interpolation reads one float4 per corner
    {
        const RowJobs j4{{Ut, Ut, Upt}, {V + 0, V + 1, V + 2}, {0.f, kW, 0.f}, {0, 1, 0}};
        PP_STEP(rows(false, j4, 3, Mx, m, Mx, m, m, 4 * m, 4, tw, qw, st));
    }
#undef PP_STEP
    if (n > 0) {
        interp_kernel<<<grid, 256, 0, st>>>(Lc.x, Lc.y, Lc.w, Lc.h, Lc.c, n, m, (float)(m / Lc.W),
                                            (float)(m / Lc.H), (const float4 *)V, e_block, gx, gy, e_total);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace pp
