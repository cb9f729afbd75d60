// Tensor-core path (PP_TF32, PP_BF16X3) for sm_103a: tcgen05 MMAs, TMEM
// accumulators, TMA-staged coefficient tiles, basis tiles generated in shared
// memory by dedicated warps.
//
//   tc_coeff_kernel   St = Xt^T Yt (contraction over blocks).  CTA tile 256 (u) x
//                     256 (v) as two M=128, N=256 accumulators that share the Yt
//                     operand; persistent over (tile, block slice) units.  A
//                     slice is contracted in chains of at most c_chain<PREC>()
//                     blocks: the tensor cores' FP32 accumulation rounds toward
//                     zero, a bias that grows with the number of MMAs
//                     accumulated into one TMEM value, so each chain starts a
//                     fresh accumulator and the epilogue adds it (round to
//                     nearest) into the unit's FP32 partial; the slices are
//                     summed with Kahan compensation by the finish kernel.
//   tc_finish_kernel  a = G o (f St g) and K = f a g in the operand precision,
//                     laid out so that one 3-D TMA box is one pipeline stage.
//   tc_energy_kernel  T = Xt K and T' = Xh K for row tiles of 128 blocks (two
//                     accumulators sharing the TMA-staged K tile), then row dots
//                     with Yt and Yh in the epilogue warps; persistent, one CTA
//                     per SM looping over row tiles.
//
// Operand layouts (no swizzle, core matrix = 8 rows x 16 bytes, LBO = K-direction
// core stride, SBO = M/N-direction core stride):
//   TF32  operands are K-major (MN-major TF32 is not used).
//   BF16  coefficient operands are MN-major (modes contiguous), energy operands
//         K-major.
// BF16x3 splits every operand into hi = bf16(x), lo = bf16(x - hi) and sums the
// three products hi*hi + hi*lo + lo*hi in the FP32 accumulator.
//
// Every wait is bounded: on a timeout the kernel raises bit 0 of the device
// status word, stops issuing work, waits (bounded) for its own MMAs to drain,
// frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cmath>
#include <type_traits>
#include <cstdio>

#include "pp_device.cuh"
#include "pp_gen.cuh"
#include "pp_internal.h"
#include "pp_tc.cuh"

namespace pp {

using namespace tc;
using gen::c2;
using gen::f2;

namespace {

constexpr uint64_t kWaitLimit = 4000000000ull;   // ns an mbarrier wait may take before giving up

__device__ __forceinline__ void raise_timeout(unsigned *status, volatile int *abort_flag) {
    *abort_flag = 1;
    if (status) atomicOr(status, 1u);
}

// Split x into bf16 hi (nearest) and lo = bf16(x - hi).
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}


// ===========================================================================
// Coefficient contraction
// ===========================================================================
constexpr int C_TILE = 256;                 // u and v edge of a CTA tile
constexpr int C_KB = 32;                    // blocks per pipeline stage
constexpr int C_STAGES = 3;
constexpr int C_STAGE_BYTES = 65536;        // A 32 KB + B 32 KB (both precisions)
constexpr int C_GEN_GROUPS = 2;            // generator groups filling alternate stages
constexpr int C_GEN_WARPS = 8 * C_GEN_GROUPS;
constexpr int C_EPI_WARPS = 8;             // two per TMEM lane quarter: one per accumulator
constexpr int C_LOADER_WARP = 1 + C_EPI_WARPS + C_GEN_WARPS;     // copies per-block records
constexpr int C_THREADS = 32 * (C_LOADER_WARP + 1);
constexpr int C_REC_BYTES = 2 * C_KB * (int)sizeof(AxisRec);    // x and y records of a stage

struct CoeffBars {
    uint64_t full[C_STAGES];
    uint64_t empty[C_STAGES];
    uint64_t recs_full[C_STAGES];
    uint64_t acc_full;
    uint64_t acc_empty;
    uint64_t drain;
    uint32_t tmem_slot;
    int abort_flag;
};
constexpr int C_SMEM = C_STAGES * (C_STAGE_BYTES + C_REC_BYTES) + 1024 + (int)sizeof(CoeffBars);

struct CoeffArgs {
    const AxisRec *xr, *yr;
    int n, tiles_v, slices, slice_len, units;
    int Mxc, Myc;         // padded (multiple of 256) extents of the partial tiles
    float *part;          // [slices][Mxc][Myc]
    unsigned *status;
};

// TF32 generator.  A sampled sinusoid y_j = f(a + j th) (f = cos or sin) obeys
// y_{j+1} = 2 cos(th) y_j - y_{j-1}.  With the signs sigma_j = +,+,-,-,+,+,...
// (period 4, so that sigma_{j+1} sigma_{j-1} = -1) the scaled values s_j =
// sigma_j y_j obey s_{j+1} = c_j s_j + s_{j-1}, c_j = +2 cos(th) for even j and
// -2 cos(th) for odd j: one FMA per step and no negation.  The cosine chain of the
// centre phase and the sine chain of the half-size phase carry the same signs, so
// their product s^Z_j s^T_j is the basis value itself.
//
// Rounding: an error d entering at step i reaches step j multiplied by
// sin((j - i) th) / sin th, at most j - i in magnitude, so after J steps the
// accumulated error is below J^2 / 2 units of FP32 rounding: 512 units (3e-5
// relative) for the 32-step chains here; the anchors come from the hardware sine
// and cosine (error 4e-7, at most 32 times that at the chain's end).  Both are far
// below the 2^-11 rounding of the TF32 operand they feed.
//
// Layout: K-major rows of 4 consecutive blocks.  Thread gg (0..127) owns the block
// pair 4*k4 + 2*pp + {0, 1} of the stage and the mode residue r; it writes the
// operand rows R = r + 8j (modes mode_base + r + 8j, j = 0..31) as 8-byte halves of
// the 16-byte core rows, the two blocks' chains advanced together in packed
// registers (step th = 8 pi s for the centre, 8 pi t for the half size; e^{i th}
// from the record).
__device__ __forceinline__ void gen_coeff_tf32(unsigned char *op, const AxisRec *recs, int nvalid,
                                               int mode_base, int gg) {
    const int lane = gg & 31, w = gg >> 5;
    const int r = lane & 7, pp = (lane >> 3) & 1, k4 = 2 * w + (lane >> 4);
    const int b0 = 4 * k4 + 2 * pp;
    const unsigned long long m0 = (unsigned long long)(mode_base + r);
    // per block: s_0, s_{-1} of both chains, 2 cos(th) of both chains
    float z0[2], zm[2], t0[2], tm[2], cz[2], ct[2], v0[2];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int k = b0 + b;
        if (k < nvalid) {
            const AxisRec &R = recs[k];
            const float2 AZ = gen::phase_sfu(m0, R.s), AT = gen::phase_sfu(m0, R.t);
            const float2 hZ = R.es8, hT = R.et8;
            z0[b] = AZ.x;                                          // cos(pi m0 s)
            zm[b] = -fmaf(AZ.x, hZ.x, AZ.y * hZ.y);                // -cos(pi (m0 - 8) s)
            t0[b] = R.c * AT.y;                                    // c sin(pi m0 t)
            tm[b] = -R.c * fmaf(AT.y, hT.x, -AT.x * hT.y);         // -c sin(pi (m0 - 8) t)
            cz[b] = 2.f * hZ.x;
            ct[b] = 2.f * hT.x;
            v0[b] = R.v0;
        } else {
            z0[b] = zm[b] = t0[b] = tm[b] = cz[b] = ct[b] = v0[b] = 0.f;
        }
    }
    f2 Z = gen::pk(z0[0], z0[1]), Zp = gen::pk(zm[0], zm[1]);
    f2 T = gen::pk(t0[0], t0[1]), Tp = gen::pk(tm[0], tm[1]);
    const f2 CZ = gen::pk(cz[0], cz[1]), NCZ = gen::pk(-cz[0], -cz[1]);
    const f2 CT = gen::pk(ct[0], ct[1]), NCT = gen::pk(-ct[0], -ct[1]);
    unsigned char *base = op + k4 * 128 + r * 16 + pp * 8;
    auto put = [&](int j) {
        float a, b;
        gen::upk(gen::mul2(Z, T), a, b);
        *reinterpret_cast<float2 *>(base + j * 1024) = make_float2(to_tf32_mma(a), to_tf32_mma(b));
    };
#pragma unroll 4
    for (int j = 0; j < 32; j += 2) {
        put(j);
        f2 nz = gen::fma2(CZ, Z, Zp), nt = gen::fma2(CT, T, Tp);     // even j: c_j = +2 cos th
        Zp = Z;
        Z = nz;
        Tp = T;
        T = nt;
        put(j + 1);
        nz = gen::fma2(NCZ, Z, Zp);                                   // odd j: c_j = -2 cos th
        nt = gen::fma2(NCT, T, Tp);
        Zp = Z;
        Z = nz;
        Tp = T;
        T = nt;
    }
    // mode 0 (the u = 0 / v = 0 column): v0 = c pi t, not the sine limit the chain
    // gives; this thread stored that slot first, so its own later store wins
    if (m0 == 0) *reinterpret_cast<float2 *>(base) = make_float2(to_tf32_mma(v0[0]), to_tf32_mma(v0[1]));
}

__device__ __forceinline__ uint32_t cvt_bf16x2(float lo_half, float hi_half) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi_half), "f"(lo_half));
    return d;
}
// (a, b) -> packed bf16 hi parts and packed bf16 lo = bf16(x - hi) parts (a in the low half)
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
    hi = cvt_bf16x2(a, b);
    const float ha = __uint_as_float(hi << 16), hb = __uint_as_float(hi & 0xFFFF0000u);
    lo = cvt_bf16x2(a - ha, b - hb);
}

// BF16 generator: MN-major rows of 8 consecutive modes of one block.  Thread
// (block k, lane group lg) writes mode groups lg + 4q (q = 0..7), 8 modes each,
// hi and lo parts; even and odd modes advance as two packed chains, the group
// anchors by complex rotation (32 modes), the modes within a group by the signed
// three-term recurrence.  Element
// (mode R, block k) at (R/8)*128 + (k/8)*4096 + (k%8)*16.
__device__ __forceinline__ void gen_coeff_bf16(unsigned char *op_hi, unsigned char *op_lo,
                                               const AxisRec *recs, int nvalid, int mode_base, int g) {
    const int lane = g & 31, wq = (g >> 5) & 3;
    const int k = (lane & 7) + 8 * wq;
    const int lg = lane >> 3;
    float2 za = make_float2(0.f, 0.f), ta = za, es = make_float2(1.f, 0.f), et = es, es8 = es, et8 = es;
    float v0 = 0.f;
    if (k < nvalid) {
        const AxisRec &R = recs[k];
        const unsigned long long m0 = (unsigned long long)(mode_base + 8 * lg);
        za = gen::phase_poly(m0, R.s);
        ta = gen::phase_poly(m0, R.t);
        ta.x *= R.c;
        ta.y *= R.c;
        es = R.es;
        et = R.et;
        es8 = R.es8;
        et8 = R.et8;
        v0 = R.v0;
    }
    // group-start chains (modes m, m+1), the 2-mode step, and the 32-mode jump
    c2 GS = gen::make_c2(za, rot(za, es)), GT = gen::make_c2(ta, rot(ta, et));
    const float2 es2 = rot(es, es), et2 = rot(et, et);
    const float2 s16 = rot(es8, es8), t16 = rot(et8, et8);
    const gen::rot2_step S32 = gen::make_step(rot(s16, s16), rot(s16, s16));
    const gen::rot2_step T32 = gen::make_step(rot(t16, t16), rot(t16, t16));
    const size_t koff = (size_t)(k >> 3) * 4096 + (k & 7) * 16;
    // groups q and q + 4 (128 modes apart) advance together: two independent chains
    const float2 s64 = rot(rot(s16, s16), rot(s16, s16)), t64 = rot(rot(t16, t16), rot(t16, t16));
    const gen::rot2_step S128 = gen::make_step(rot(s64, s64), rot(s64, s64));
    const gen::rot2_step T128 = gen::make_step(rot(t64, t64), rot(t64, t64));
    c2 HS = gen::rot2(GS, S128), HT = gen::rot2(GT, T128);
    // within a group, (m, m+1) advance by the signed three-term recurrence of the
    // TF32 generators (4 steps: rounding below 8 FP32 units), started from the
    // group's complex anchor and its value two modes back (times conj(e^{2 i pi s}))
    const f2 KZ = gen::pk(2.f * es2.x, 2.f * es2.x), NKZ = gen::pk(-2.f * es2.x, -2.f * es2.x);
    const f2 KT = gen::pk(2.f * et2.x, 2.f * et2.x), NKT = gen::pk(-2.f * et2.x, -2.f * et2.x);
    const f2 E2X = gen::pk(es2.x, es2.x), E2Y = gen::pk(es2.y, es2.y);
    const f2 F2X = gen::pk(et2.x, et2.x), NF2Y = gen::pk(-et2.y, -et2.y);
    auto start = [&](const c2 &z, const c2 &t, f2 &Z, f2 &Zp, f2 &T, f2 &Tp) {
        Z = z.re;
        T = t.im;
        // s_{-1} = -y_{-1}: -Re(z conj(e2)) = -(z.re e2.x + z.im e2.y), -Im(t conj(e2))
        const f2 zr = gen::fma2(z.re, E2X, gen::mul2(z.im, E2Y));
        const f2 ti = gen::fma2(t.im, F2X, gen::mul2(t.re, NF2Y));
        Zp = gen::pk(-zr.v.x, -zr.v.y);
        Tp = gen::pk(-ti.v.x, -ti.v.y);
    };
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
        const int grp0 = lg + 4 * q, grp1 = grp0 + 16;
        f2 Z0, Zp0, T0, Tp0, Z1, Zp1, T1, Tp1;
        start(GS, GT, Z0, Zp0, T0, Tp0);
        start(HS, HT, Z1, Zp1, T1, Tp1);
        uint32_t hi0[4], lo0[4], hi1[4], lo1[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            float a, b, c, d;
            gen::upk(gen::mul2(Z0, T0), a, b);
            gen::upk(gen::mul2(Z1, T1), c, d);
            if (jj == 0 && mode_base + 8 * grp0 == 0) a = v0;
            split2(a, b, hi0[jj], lo0[jj]);
            split2(c, d, hi1[jj], lo1[jj]);
            const f2 kz = (jj & 1) ? NKZ : KZ, kt = (jj & 1) ? NKT : KT;
            const f2 nz0 = gen::fma2(kz, Z0, Zp0), nt0 = gen::fma2(kt, T0, Tp0);
            const f2 nz1 = gen::fma2(kz, Z1, Zp1), nt1 = gen::fma2(kt, T1, Tp1);
            Zp0 = Z0;
            Z0 = nz0;
            Tp0 = T0;
            T0 = nt0;
            Zp1 = Z1;
            Z1 = nz1;
            Tp1 = T1;
            T1 = nt1;
        }
        const size_t off0 = (size_t)grp0 * 128 + koff, off1 = (size_t)grp1 * 128 + koff;
        *reinterpret_cast<uint4 *>(op_hi + off0) = make_uint4(hi0[0], hi0[1], hi0[2], hi0[3]);
        *reinterpret_cast<uint4 *>(op_lo + off0) = make_uint4(lo0[0], lo0[1], lo0[2], lo0[3]);
        *reinterpret_cast<uint4 *>(op_hi + off1) = make_uint4(hi1[0], hi1[1], hi1[2], hi1[3]);
        *reinterpret_cast<uint4 *>(op_lo + off1) = make_uint4(lo1[0], lo1[1], lo1[2], lo1[3]);
        GS = gen::rot2(GS, S32);
        GT = gen::rot2(GT, T32);
        HS = gen::rot2(HS, S32);
        HT = gen::rot2(HT, T32);
    }
}

__device__ __forceinline__ void red_add2(float *p, float a, float b) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}

// At teardown: wait (bounded) until the copies this thread issued for the last uses of
// each stage slot have landed (their completion barrier `done[s]`, completed by the
// copies' bytes alone), so that the CTA never exits while a copy still writes into
// its shared memory; `issued` copies were issued, slot it % stages, phase it / stages.
__device__ __forceinline__ void wait_copies_landed(uint64_t *done, int stages, uint32_t issued) {
    const uint32_t first = issued > (uint32_t)stages ? issued - (uint32_t)stages : 0u;
    for (uint32_t k = first; k < issued; ++k)
        mbar_wait(&done[k % stages], (k / stages) & 1, kWaitLimit, nullptr);
}

// Most blocks accumulated in one TMEM chain.  Each MMA step may truncate the FP32
// accumulator by up to one unit in the last place, in a consistent direction:
// 8192 TF32 blocks are 1024 steps of K = 8, a relative bias below 1.3e-4, small
// beside the 2^-11 rounding of TF32 operands; BF16x3 (operands good to about
// 2^-16, three MMAs per K = 16 step) keeps chains of 2048 blocks, 384 steps.
template <int PREC>
__host__ __device__ constexpr int c_chain() { return PREC == 1 ? 8192 : 2048; }

// Stages per accumulation chain for a unit of nst stages: the fewest chains of at
// most c_chain<PREC>() blocks, of equal length (the last one possibly shorter).
template <int PREC>
__device__ __forceinline__ int chain_stages(int nst) {
    constexpr int cmax = c_chain<PREC>() / C_KB;
    const int nch = (nst + cmax - 1) / cmax;
    return nch > 0 ? (nst + nch - 1) / nch : 1;
}

template <int PREC>
__global__ void __launch_bounds__(C_THREADS, 1) tc_coeff_kernel(const CoeffArgs args) {
    extern __shared__ unsigned char smem_raw[];
    // 1 KB-aligned base by pointer arithmetic on the __shared__ array, so that the
    // compiler keeps every access in the shared address space (LDS/STS)
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *recs_base = smem + C_STAGES * C_STAGE_BYTES;
    CoeffBars &bars = *reinterpret_cast<CoeffBars *>(recs_base + C_STAGES * C_REC_BYTES);
    volatile int *abort_flag = &bars.abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < C_STAGES; ++s) {
            mbar_init(&bars.full[s], (C_GEN_WARPS / C_GEN_GROUPS) * 32);   // one group per stage
            mbar_init(&bars.empty[s], 1);
            mbar_init(&bars.recs_full[s], 1);
        }
        mbar_init(&bars.acc_full, 1);
        mbar_init(&bars.acc_empty, C_EPI_WARPS * 32);
        mbar_init(&bars.drain, 1);
        bars.abort_flag = 0;
        mbar_fence_init();
    }
    pdl_wait();                        // the block records come from the preparation kernel
    if (warp == 0) {
        tmem_alloc(&bars.tmem_slot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    pdl_trigger();                     // the finish kernel may be scheduled (it waits for this one)
    const uint32_t tmem = bars.tmem_slot;

    const int tiles_v = args.tiles_v;
    if (warp == 0) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr bool BF = PREC == 2;
            const uint32_t idesc = instr_desc(BF ? kFmtBF16 : kFmtTF32, 128, 256, BF, BF);
            // stage 0's operand descriptors; the others are byte offsets from them.  The
            // issuing thread bounds the kernel, so its loop keeps to adds and compares.
            const uint32_t s0 = smem_u32(smem);
            const uint64_t dA = BF ? smem_desc(s0, 4096, 128) : smem_desc(s0, 128, 1024);
            const uint64_t dB = BF ? smem_desc(s0 + 32768, 4096, 128) : smem_desc(s0 + 32768, 128, 1024);
            uint32_t it = 0, dc = 0;     // stages issued, chains committed
            int s = 0, ph = 0;           // it % C_STAGES, (it / C_STAGES) & 1
            for (int unit = blockIdx.x; unit < args.units && !*abort_flag; unit += gridDim.x) {
                const int slice = unit % args.slices;
                const int b0 = slice * args.slice_len;
                const int b1 = min(args.n, b0 + args.slice_len);
                const int nst = (b1 - b0 + C_KB - 1) / C_KB;
                const int cst = chain_stages<PREC>(nst);
                int sc = 0;                  // stage within the chain
                for (int st = 0; st < nst; ++st, ++it, sc = (sc + 1 == cst ? 0 : sc + 1),
                         ph ^= (s + 1 == C_STAGES), s = (s + 1 == C_STAGES ? 0 : s + 1)) {
                    if (sc == 0) {
                        // the epilogue has read the previous chain out of TMEM
                        if (dc > 0 && !mbar_wait(&bars.acc_empty, (dc - 1) & 1, kWaitLimit, abort_flag)) {
                            raise_timeout(args.status, abort_flag);
                            break;
                        }
                        tc_fence_after();
                    }
                    if (!mbar_wait(&bars.full[s], ph, kWaitLimit, abort_flag)) {
                        raise_timeout(args.status, abort_flag);
                        break;
                    }
                    tc_fence_after();
                    const uint32_t so = (uint32_t)s * C_STAGE_BYTES;
                    if (!BF) {
                        // A: 256 rows x 32 blocks tf32, cores (row/8, blk/4): LBO 128, SBO 1024
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t bd = desc_add(dB, so + kk * 256);
#pragma unroll
                            for (int acc = 0; acc < 2; ++acc) {
                                const uint64_t ad = desc_add(dA, so + acc * 16384 + kk * 256);
                                mma_tf32(tmem + acc * 256, ad, bd, idesc, sc > 0 || kk > 0);
                            }
                        }
                    } else {
                        // MN-major bf16: element (mode R, blk k) at (R/8)*128 + (k/8)*4096
                        // + (k%8)*16: SBO (mode groups) 128, LBO (block groups) 4096;
                        // hi parts at +0 (A) / +32768 (B), lo parts 16 KB further
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint32_t ko = kk * 8192;
                            const uint64_t bh = desc_add(dB, so + ko);
                            const uint64_t bl = desc_add(dB, so + 16384 + ko);
#pragma unroll
                            for (int acc = 0; acc < 2; ++acc) {
                                const uint32_t mo = acc * 2048;
                                const uint64_t ah = desc_add(dA, so + mo + ko);
                                const uint64_t al = desc_add(dA, so + 16384 + mo + ko);
                                const bool accum = sc > 0 || kk > 0;
                                mma_bf16(tmem + acc * 256, al, bh, idesc, accum);
                                mma_bf16(tmem + acc * 256, ah, bl, idesc, true);
                                mma_bf16(tmem + acc * 256, ah, bh, idesc, true);
                            }
                        }
                    }
                    mma_commit(&bars.empty[s]);
                    if (sc == cst - 1 || st == nst - 1) {
                        mma_commit(&bars.acc_full);
                        ++dc;
                    }
                }
            }
            // all MMAs issued by this thread complete before the TMEM is freed
            mma_commit(&bars.drain);
            if (!mbar_wait(&bars.drain, 0, kWaitLimit, nullptr)) raise_timeout(args.status, abort_flag);
        }
        __syncwarp();
    } else if (warp <= C_EPI_WARPS) {
        // ---------------- epilogue: TMEM -> FP32 partial tile ----------------
        // Warp w reads TMEM lanes 32 (w % 4) .. + 31 of accumulator (w - 1) / 4, 16
        // lanes x 64 columns per load (16x256b shape: thread t holds rows t/4 and
        // t/4 + 8, columns 8j + 2 (t % 4) + {0, 1}), so that the four threads of a
        // row write one full 32-byte sector per store.
        const int quarter = warp & 3, acc = (warp - 1) >> 2;
        const int rsub = lane >> 2, csub = 2 * (lane & 3);
        uint32_t dc = 0;
        for (int unit = blockIdx.x; unit < args.units; unit += gridDim.x) {
            if (*abort_flag) break;
            const int tile = unit / args.slices, slice = unit % args.slices;
            const int tu = tile / tiles_v, tv = tile % tiles_v;
            const int b0 = slice * args.slice_len;
            const int nst = (min(args.n, b0 + args.slice_len) - b0 + C_KB - 1) / C_KB;
            const int nch = (nst + chain_stages<PREC>(nst) - 1) / chain_stages<PREC>(nst);
#pragma unroll 1
            for (int ch = 0; ch < nch; ++ch, ++dc) {
                if (!mbar_wait(&bars.acc_full, dc & 1, kWaitLimit, abort_flag)) {
                    raise_timeout(args.status, abort_flag);
                    break;
                }
                tc_fence_after();
#pragma unroll 1
                for (int half = 0; half < 2; ++half) {
                    const int r0 = quarter * 32 + half * 16;          // first TMEM lane of the load
                    const int u = tu * C_TILE + acc * 128 + r0 + rsub;
                    float *dst0 = args.part + ((size_t)slice * args.Mxc + u) * args.Myc + tv * C_TILE + csub;
                    float *dst1 = dst0 + (size_t)8 * args.Myc;          // row + 8
#pragma unroll 1
                    for (int c = 0; c < 256; c += 64) {
                        float v[32];
                        tmem_ld_16x256b_x8(tmem + ((uint32_t)r0 << 16) + acc * 256 + c, v);
                        tmem_ld_wait_regs32(v);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            float *p0 = dst0 + c + 8 * j, *p1 = dst1 + c + 8 * j;
                            if (ch == 0) {
                                *reinterpret_cast<float2 *>(p0) = make_float2(v[4 * j], v[4 * j + 1]);
                                *reinterpret_cast<float2 *>(p1) = make_float2(v[4 * j + 2], v[4 * j + 3]);
                            } else {    // added in L2 (round to nearest) after this thread's earlier store
                                red_add2(p0, v[4 * j], v[4 * j + 1]);
                                red_add2(p1, v[4 * j + 2], v[4 * j + 3]);
                            }
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(&bars.acc_empty);
            }
        }
    } else if (warp < C_LOADER_WARP) {
        // ---------------- basis generators ----------------
        // group gr fills the stages it with it % C_GEN_GROUPS == gr, so two stages are
        // generated at once and each group's latency is hidden behind the other's
        const int g = threadIdx.x - 32 * (1 + C_EPI_WARPS);    // 0..511
        const int gr = g >> 8;
        const int which = (g >> 7) & 1;                        // 0: Xt (A), 1: Yt (B)
        const int gg = g & 127;
        uint32_t it = 0;
        for (int unit = blockIdx.x; unit < args.units; unit += gridDim.x) {
            const int tile = unit / args.slices, slice = unit % args.slices;
            const int tu = tile / tiles_v, tv = tile % tiles_v;
            const int b0 = slice * args.slice_len;
            const int b1 = min(args.n, b0 + args.slice_len);
            const int nst = (b1 - b0 + C_KB - 1) / C_KB;
            for (int st = 0; st < nst; ++st, ++it) {
                if (*abort_flag) break;
                if ((int)(it % C_GEN_GROUPS) != gr) continue;
                const int s = it % C_STAGES;
                // empty first: the MMAs have consumed stage it - 3, so the other group
                // has filled it and its records phase is complete; only then is the
                // parity wait on recs_full unambiguous (it cannot be two phases behind)
                if ((it >= C_STAGES &&
                     !mbar_wait(&bars.empty[s], ((it / C_STAGES) - 1) & 1, kWaitLimit, abort_flag)) ||
                    !mbar_wait(&bars.recs_full[s], (it / C_STAGES) & 1, kWaitLimit, abort_flag)) {
                    raise_timeout(args.status, abort_flag);
                    break;
                }
                unsigned char *sb = smem + s * C_STAGE_BYTES;
                const AxisRec *recs =
                    reinterpret_cast<const AxisRec *>(recs_base + s * C_REC_BYTES) + which * C_KB;
                const int nvalid = min(C_KB, b1 - (b0 + st * C_KB));
                const int mode_base = (which ? tv : tu) * C_TILE;
                if (PREC == 1)
                    gen_coeff_tf32(sb + which * 32768, recs, nvalid, mode_base, gg);
                else
                    gen_coeff_bf16(sb + which * 32768, sb + which * 32768 + 16384, recs, nvalid, mode_base, gg);
                fence_proxy_async_smem();
                mbar_arrive(&bars.full[s]);
            }
            if (*abort_flag) break;
        }
    } else {
        // ---------------- record loader: x and y records of each stage ----------------
        if (lane == 0) {
            uint32_t it = 0;
            for (int unit = blockIdx.x; unit < args.units; unit += gridDim.x) {
                const int slice = unit % args.slices;
                const int b0 = slice * args.slice_len;
                const int b1 = min(args.n, b0 + args.slice_len);
                const int nst = (b1 - b0 + C_KB - 1) / C_KB;
                for (int st = 0; st < nst; ++st, ++it) {
                    if (*abort_flag) break;
                    const int s = it % C_STAGES;
                    // the generators have finished with this buffer's previous stage
                    if (it >= C_STAGES &&
                        !mbar_wait(&bars.full[s], ((it / C_STAGES) - 1) & 1, kWaitLimit, abort_flag)) {
                        raise_timeout(args.status, abort_flag);
                        break;
                    }
                    const int blk0 = b0 + st * C_KB;
                    const uint32_t bytes = (uint32_t)min(C_KB, b1 - blk0) * (uint32_t)sizeof(AxisRec);
                    unsigned char *dst = recs_base + s * C_REC_BYTES;
                    mbar_arrive_expect_tx(&bars.recs_full[s], 2 * bytes);
                    bulk_load(dst, args.xr + blk0, bytes, &bars.recs_full[s]);
                    bulk_load(dst + C_KB * sizeof(AxisRec), args.yr + blk0, bytes, &bars.recs_full[s]);
                }
                if (*abort_flag) break;
            }
            wait_copies_landed(bars.recs_full, C_STAGES, it);
        }
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ===========================================================================
// Coefficient contraction on SM pairs
// ===========================================================================
// The pair kernel runs the same contraction with the two CTAs of a cluster on two
// SMs issuing M = 256 MMAs together (cta_group::2): per MMA each CTA supplies 128
// rows of Xt (A) and half of the 256 columns of Yt (B) from its own shared memory,
// and its tensor memory receives its 128 rows of the 256 x 256 result.  A CTA pair
// covers a 512 (u) x 256 (v) tile with two such accumulators per CTA.  Compared with
// one CTA per 256 x 256 tile, each SM generates and reads only half of the Yt
// operand: 112 KB of shared-memory traffic per 32-block stage instead of 160 KB,
// which is what bounds the single-CTA kernel.
//
// Rows of the pair tile held by CTA rank rk (0 or 1), accumulator acc (TMEM lane i):
// TF32 mode tile_u0 + 256 acc + 2 i + rk (the two CTAs' rows interleaved, so that
// each CTA's 256 A rows are one progression of step 2 that one recurrence chain per
// generator thread covers), BF16x3 tile_u0 + 256 acc + 128 rk + i; its B columns are
// v = tile_v0 + 128 rk + [0, 128).  The even CTA's thread 0 of warp 0 issues every MMA; its commits
// arrive on the barriers of both CTAs (multicast).  Its `acc_empty` barrier counts the
// epilogue warps of both CTAs, which arrive through cluster addresses.  Its `full[s]`
// counts its own generator warps (local arrivals) and one relay from the odd CTA: there
// the generator warps arrive on their local `gen_done[s]` and thread 0 of warp 0 (idle
// otherwise) waits for that phase and passes it on with one cluster-scope release.  With
// a cluster-scope release by every generator warp, a per-stage trace showed ~0.8 us
// between a warp's last store of a stage and its next stage's start, on the critical
// path of the odd CTA's A generators.
constexpr int P_STAGES = 4;
constexpr int P_A_BYTES = 32768;                // 256 rows x 32 blocks
constexpr int P_B_BYTES = 16384;                // 128 rows x 32 blocks
constexpr int P_STAGE_BYTES = P_A_BYTES + P_B_BYTES;
constexpr int P_TILE_U = 512;
constexpr int P_TILE_V = 256;

struct PairBars {
    uint64_t full[P_STAGES];       // even CTA: its generator warps + the odd CTA's relay
    uint64_t empty[P_STAGES];      // both: MMA commit (multicast)
    uint64_t recs_full[P_STAGES];  // local: record copies
    uint64_t gen_done[P_STAGES];   // local: this CTA's generators are done with the records
    uint64_t acc_full;             // both: MMA commit at the end of a chain (multicast)
    uint64_t acc_empty;            // even CTA: epilogue warps of both CTAs
    uint64_t drain;                // even CTA: every MMA complete
    uint32_t tmem_slot;
    int abort_flag;
};
constexpr int P_SMEM = P_STAGES * (P_STAGE_BYTES + C_REC_BYTES) + 1024 + (int)sizeof(PairBars);
static_assert(P_SMEM <= 232448, "pair kernel shared memory");

// TF32 rows for the pair kernel: segment g (g < nseg) holds 128 consecutive modes
// from mb[g] as operand rows 128 g + r + 8 j' (j' < 16), generated as 16-step chains
// of the signed three-term recurrence (as gen_coeff_tf32, one chain per segment).
__device__ __forceinline__ void gen_pair_tf32(unsigned char *op, const AxisRec *recs, int nvalid, int mb0,
                                              int mb1, int nseg, int gg) {
    const int lane = gg & 31, w = gg >> 5;
    const int r = lane & 7, pp = (lane >> 3) & 1, k4 = 2 * w + (lane >> 4);
    const int b0 = 4 * k4 + 2 * pp;
    unsigned char *base = op + k4 * 128 + r * 16 + pp * 8;
#pragma unroll 1
    for (int g = 0; g < nseg; ++g) {
        const unsigned long long m0 = (unsigned long long)((g ? mb1 : mb0) + r);
        float z0[2], zm[2], t0[2], tm[2], cz[2], ct[2], v0[2];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int k = b0 + b;
            if (k < nvalid) {
                const AxisRec &R = recs[k];
                const float2 AZ = gen::phase_sfu(m0, R.s), AT = gen::phase_sfu(m0, R.t);
                const float2 hZ = R.es8, hT = R.et8;
                z0[b] = AZ.x;
                zm[b] = -fmaf(AZ.x, hZ.x, AZ.y * hZ.y);
                t0[b] = R.c * AT.y;
                tm[b] = -R.c * fmaf(AT.y, hT.x, -AT.x * hT.y);
                cz[b] = 2.f * hZ.x;
                ct[b] = 2.f * hT.x;
                v0[b] = R.v0;
            } else {
                z0[b] = zm[b] = t0[b] = tm[b] = cz[b] = ct[b] = v0[b] = 0.f;
            }
        }
        f2 Z = gen::pk(z0[0], z0[1]), Zp = gen::pk(zm[0], zm[1]);
        f2 T = gen::pk(t0[0], t0[1]), Tp = gen::pk(tm[0], tm[1]);
        const f2 CZ = gen::pk(cz[0], cz[1]), NCZ = gen::pk(-cz[0], -cz[1]);
        const f2 CT = gen::pk(ct[0], ct[1]), NCT = gen::pk(-ct[0], -ct[1]);
        unsigned char *sb = base + g * 16 * 1024;
        auto put = [&](int j) {
            float a, b;
            gen::upk(gen::mul2(Z, T), a, b);
            *reinterpret_cast<float2 *>(sb + j * 1024) = make_float2(to_tf32_mma(a), to_tf32_mma(b));
        };
#pragma unroll 4
        for (int j = 0; j < 16; j += 2) {
            put(j);
            f2 nz = gen::fma2(CZ, Z, Zp), nt = gen::fma2(CT, T, Tp);
            Zp = Z;
            Z = nz;
            Tp = T;
            T = nt;
            put(j + 1);
            nz = gen::fma2(NCZ, Z, Zp);
            nt = gen::fma2(NCT, T, Tp);
            Zp = Z;
            Z = nz;
            Tp = T;
            T = nt;
        }
        if (m0 == 0) *reinterpret_cast<float2 *>(sb) = make_float2(to_tf32_mma(v0[0]), to_tf32_mma(v0[1]));
    }
}

// TF32 A rows for the pair kernel with the modes interleaved between the two CTAs:
// row R of CTA rank rk holds mode mb + rk + 2 R (R < 256), so that each CTA's 256
// rows are one progression of step 2 and one chain per thread covers them: thread
// (block pair, residue r) generates rows r + 8 j (modes m0 + 16 j, m0 = mb + rk + 2 r)
// for j < 32 by the signed three-term recurrence with step 16 pi s, one anchor.
__device__ __forceinline__ void gen_pair_tf32_interleaved(unsigned char *op, const AxisRec *recs, int nvalid,
                                                          int m_first, int gg) {
    const int lane = gg & 31, w = gg >> 5;
    const int r = lane & 7, pp = (lane >> 3) & 1, k4 = 2 * w + (lane >> 4);
    const int b0 = 4 * k4 + 2 * pp;
    const unsigned long long m0 = (unsigned long long)(m_first + 2 * r);
    float z0[2], zm[2], t0[2], tm[2], cz[2], ct[2], v0[2];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int k = b0 + b;
        if (k < nvalid) {
            const AxisRec &R = recs[k];
            const float2 AZ = gen::phase_sfu(m0, R.s), AT = gen::phase_sfu(m0, R.t);
            const float2 hZ = rot(R.es8, R.es8), hT = rot(R.et8, R.et8);     // 16-mode steps
            z0[b] = AZ.x;
            zm[b] = -fmaf(AZ.x, hZ.x, AZ.y * hZ.y);                // -cos(pi (m0 - 16) s)
            t0[b] = R.c * AT.y;
            tm[b] = -R.c * fmaf(AT.y, hT.x, -AT.x * hT.y);         // -c sin(pi (m0 - 16) t)
            cz[b] = 2.f * hZ.x;
            ct[b] = 2.f * hT.x;
            v0[b] = R.v0;
        } else {
            z0[b] = zm[b] = t0[b] = tm[b] = cz[b] = ct[b] = v0[b] = 0.f;
        }
    }
    f2 Z = gen::pk(z0[0], z0[1]), Zp = gen::pk(zm[0], zm[1]);
    f2 T = gen::pk(t0[0], t0[1]), Tp = gen::pk(tm[0], tm[1]);
    const f2 CZ = gen::pk(cz[0], cz[1]), NCZ = gen::pk(-cz[0], -cz[1]);
    const f2 CT = gen::pk(ct[0], ct[1]), NCT = gen::pk(-ct[0], -ct[1]);
    unsigned char *base = op + k4 * 128 + r * 16 + pp * 8;
    auto put = [&](int j) {
        float a, b;
        gen::upk(gen::mul2(Z, T), a, b);
        *reinterpret_cast<float2 *>(base + j * 1024) = make_float2(to_tf32_mma(a), to_tf32_mma(b));
    };
#pragma unroll 4
    for (int j = 0; j < 32; j += 2) {
        put(j);
        f2 nz = gen::fma2(CZ, Z, Zp), nt = gen::fma2(CT, T, Tp);
        Zp = Z;
        Z = nz;
        Tp = T;
        T = nt;
        put(j + 1);
        nz = gen::fma2(NCZ, Z, Zp);
        nt = gen::fma2(NCT, T, Tp);
        Zp = Z;
        Z = nz;
        Tp = T;
        T = nt;
    }
    if (m0 == 0) *reinterpret_cast<float2 *>(base) = make_float2(to_tf32_mma(v0[0]), to_tf32_mma(v0[1]));
}

// BF16 rows for the pair kernel (MN-major, bf16 hi and lo): segment 0 = 128 modes from
// mb0 as mode groups 0..15, segment 1 (nseg == 2) = 128 modes from mb0 + 256 as groups
// 16..31.  Element (mode group q, block k) at q * 128 + (k / 8) * lbo + (k % 8) * 16.
__device__ __forceinline__ void gen_pair_bf16(unsigned char *op_hi, unsigned char *op_lo, const AxisRec *recs,
                                              int nvalid, int mb0, int nseg, int lbo, int g) {
    const int lane = g & 31, wq = (g >> 5) & 3;
    const int k = (lane & 7) + 8 * wq;
    const int lg = lane >> 3;
    float2 za = make_float2(0.f, 0.f), ta = za, es = make_float2(1.f, 0.f), et = es, es8 = es, et8 = es;
    float v0 = 0.f;
    if (k < nvalid) {
        const AxisRec &R = recs[k];
        const unsigned long long m0 = (unsigned long long)(mb0 + 8 * lg);
        za = gen::phase_poly(m0, R.s);
        ta = gen::phase_poly(m0, R.t);
        ta.x *= R.c;
        ta.y *= R.c;
        es = R.es;
        et = R.et;
        es8 = R.es8;
        et8 = R.et8;
        v0 = R.v0;
    }
    c2 GS = gen::make_c2(za, rot(za, es)), GT = gen::make_c2(ta, rot(ta, et));
    const float2 es2 = rot(es, es), et2 = rot(et, et);
    const float2 s16 = rot(es8, es8), t16 = rot(et8, et8);
    const gen::rot2_step S32 = gen::make_step(rot(s16, s16), rot(s16, s16));
    const gen::rot2_step T32 = gen::make_step(rot(t16, t16), rot(t16, t16));
    const size_t koff = (size_t)(k >> 3) * lbo + (k & 7) * 16;
    // segment 1 starts 256 modes after segment 0: e^{i pi 256 s} by squarings of e^{i pi 16 s}
    const float2 s64 = rot(rot(s16, s16), rot(s16, s16)), t64 = rot(rot(t16, t16), rot(t16, t16));
    const float2 s256 = rot(rot(s64, s64), rot(s64, s64)), t256 = rot(rot(t64, t64), rot(t64, t64));
    const gen::rot2_step S256 = gen::make_step(s256, s256);
    const gen::rot2_step T256 = gen::make_step(t256, t256);
    c2 HS = gen::rot2(GS, S256), HT = gen::rot2(GT, T256);
    const f2 KZ = gen::pk(2.f * es2.x, 2.f * es2.x), NKZ = gen::pk(-2.f * es2.x, -2.f * es2.x);
    const f2 KT = gen::pk(2.f * et2.x, 2.f * et2.x), NKT = gen::pk(-2.f * et2.x, -2.f * et2.x);
    const f2 E2X = gen::pk(es2.x, es2.x), E2Y = gen::pk(es2.y, es2.y);
    const f2 F2X = gen::pk(et2.x, et2.x), NF2Y = gen::pk(-et2.y, -et2.y);
    auto start = [&](const c2 &z, const c2 &t, f2 &Z, f2 &Zp, f2 &T, f2 &Tp) {
        Z = z.re;
        T = t.im;
        const f2 zr = gen::fma2(z.re, E2X, gen::mul2(z.im, E2Y));
        const f2 ti = gen::fma2(t.im, F2X, gen::mul2(t.re, NF2Y));
        Zp = gen::pk(-zr.v.x, -zr.v.y);
        Tp = gen::pk(-ti.v.x, -ti.v.y);
    };
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
        const int grp0 = lg + 4 * q, grp1 = grp0 + 16;
        f2 Z0, Zp0, T0, Tp0, Z1, Zp1, T1, Tp1;
        start(GS, GT, Z0, Zp0, T0, Tp0);
        start(HS, HT, Z1, Zp1, T1, Tp1);
        uint32_t hi0[4], lo0[4], hi1[4], lo1[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            float a, b, c, d;
            gen::upk(gen::mul2(Z0, T0), a, b);
            gen::upk(gen::mul2(Z1, T1), c, d);
            if (jj == 0 && mb0 + 8 * grp0 == 0) a = v0;
            split2(a, b, hi0[jj], lo0[jj]);
            split2(c, d, hi1[jj], lo1[jj]);
            const f2 kz = (jj & 1) ? NKZ : KZ, kt = (jj & 1) ? NKT : KT;
            const f2 nz0 = gen::fma2(kz, Z0, Zp0), nt0 = gen::fma2(kt, T0, Tp0);
            const f2 nz1 = gen::fma2(kz, Z1, Zp1), nt1 = gen::fma2(kt, T1, Tp1);
            Zp0 = Z0;
            Z0 = nz0;
            Tp0 = T0;
            T0 = nt0;
            Zp1 = Z1;
            Z1 = nz1;
            Tp1 = T1;
            T1 = nt1;
        }
        const size_t off0 = (size_t)grp0 * 128 + koff, off1 = (size_t)grp1 * 128 + koff;
        *reinterpret_cast<uint4 *>(op_hi + off0) = make_uint4(hi0[0], hi0[1], hi0[2], hi0[3]);
        *reinterpret_cast<uint4 *>(op_lo + off0) = make_uint4(lo0[0], lo0[1], lo0[2], lo0[3]);
        if (nseg > 1) {
            *reinterpret_cast<uint4 *>(op_hi + off1) = make_uint4(hi1[0], hi1[1], hi1[2], hi1[3]);
            *reinterpret_cast<uint4 *>(op_lo + off1) = make_uint4(lo1[0], lo1[1], lo1[2], lo1[3]);
        }
        GS = gen::rot2(GS, S32);
        GT = gen::rot2(GT, T32);
        HS = gen::rot2(HS, S32);
        HT = gen::rot2(HT, T32);
    }
}

struct PairArgs {
    const AxisRec *xr, *yr;
    int n, tiles_v, slices, slice_len, units;
    int Mxc, Myc;         // padded extents of the partial tiles (multiples of 512, 256)
    float *part;          // [slices][Mxc][Myc]
    unsigned *status;
};

template <int PREC>
__global__ void __launch_bounds__(C_THREADS, 1) tc_coeff_pair_kernel(const PairArgs args) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *recs_base = smem + P_STAGES * P_STAGE_BYTES;
    PairBars &bars = *reinterpret_cast<PairBars *>(recs_base + P_STAGES * C_REC_BYTES);
    volatile int *abort_flag = &bars.abort_flag;
    const uint32_t rank = cluster_ctarank();           // 0: issues the MMAs
    const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
    constexpr int GEN_WARPS_PER_GROUP = C_GEN_WARPS / C_GEN_GROUPS;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < P_STAGES; ++s) {
            mbar_init(&bars.full[s], GEN_WARPS_PER_GROUP + 1);      // even CTA's group + relay
            mbar_init(&bars.empty[s], 1);
            mbar_init(&bars.recs_full[s], 1);
            mbar_init(&bars.gen_done[s], GEN_WARPS_PER_GROUP);
        }
        mbar_init(&bars.acc_full, 1);
        mbar_init(&bars.acc_empty, 2 * C_EPI_WARPS);
        mbar_init(&bars.drain, 1);
        bars.abort_flag = 0;
        mbar_fence_init();
    }
    // both CTAs' barriers exist before any arrival from the peer
    cluster_sync();
    pdl_wait();                        // the block records come from the preparation kernel
    if (warp == 0) {
        tmem_alloc_pair(&bars.tmem_slot, 512);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    pdl_trigger();
    const uint32_t tmem = bars.tmem_slot;
    // cluster addresses of the even CTA's barriers that both CTAs arrive on
    const uint32_t acc_empty0 = mapa_shared(smem_u32(&bars.acc_empty), 0);
    const int tiles_v = args.tiles_v;

    if (warp == 0) {
        // ---------------- MMA issuer (even CTA) ----------------
        if (rank == 0 && lane == 0) {
            constexpr bool BF = PREC == 2;
            const uint32_t idesc = instr_desc(BF ? kFmtBF16 : kFmtTF32, 256, 256, BF, BF);
            // stage 0's operand descriptors; the others are byte offsets from them.  This
            // thread's issue loop bounds the kernel (a per-stage trace and a 6% gain from
            // dropping one integer division), so it keeps to adds and compares.
            const uint32_t s0 = smem_u32(smem);
            const uint64_t dA = BF ? smem_desc(s0, 4096, 128) : smem_desc(s0, 128, 1024);
            const uint64_t dB = BF ? smem_desc(s0 + P_A_BYTES, 2048, 128) : smem_desc(s0 + P_A_BYTES, 128, 1024);
            uint32_t it = 0, dc = 0;
            for (int unit = pair; unit < args.units && !*abort_flag; unit += npairs) {
                const int slice = unit % args.slices;
                const int b0 = slice * args.slice_len;
                const int b1 = min(args.n, b0 + args.slice_len);
                const int nst = (b1 - b0 + C_KB - 1) / C_KB;
                const int cst = chain_stages<PREC>(nst);
                int sc = 0;              // stage within the chain
                for (int st = 0; st < nst; ++st, ++it, sc = (sc + 1 == cst ? 0 : sc + 1)) {
                    const int s = it % P_STAGES;
                    if (sc == 0) {
                        if (dc > 0) {
                            bool ok = mbar_try_wait_cluster(&bars.acc_empty, (dc - 1) & 1);
                            const uint64_t t0 = ok ? 0 : globaltimer_ns();
                            for (uint32_t i = 1; !ok && !*abort_flag; ++i) {
                                ok = mbar_try_wait_cluster(&bars.acc_empty, (dc - 1) & 1);
                                if (!ok && (i & 63) == 0 && globaltimer_ns() - t0 > kWaitLimit) break;
                            }
                            if (!ok) {
                                raise_timeout(args.status, abort_flag);
                                break;
                            }
                        }
                        tc_fence_after();
                    }
                    {
                        bool ok = mbar_try_wait_cluster(&bars.full[s], (it / P_STAGES) & 1);
                        const uint64_t t0 = ok ? 0 : globaltimer_ns();
                        for (uint32_t i = 1; !ok && !*abort_flag; ++i) {
                            ok = mbar_try_wait_cluster(&bars.full[s], (it / P_STAGES) & 1);
                            if (!ok && (i & 63) == 0 && globaltimer_ns() - t0 > kWaitLimit) break;
                        }
                        if (!ok) {
                            raise_timeout(args.status, abort_flag);
                            break;
                        }
                    }
                    tc_fence_after();
                    const uint32_t so = (uint32_t)s * P_STAGE_BYTES;
                    if (!BF) {
                        // A: 256 rows x 32 blocks (LBO 128, SBO 1024); B: 128 rows, same layout
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t bd = desc_add(dB, so + kk * 256);
#pragma unroll
                            for (int acc = 0; acc < 2; ++acc) {
                                const uint64_t ad = desc_add(dA, so + acc * 16384 + kk * 256);
                                mma_tf32_pair(tmem + acc * 256, ad, bd, idesc, sc > 0 || kk > 0);
                            }
                        }
                    } else {
                        // MN-major bf16: A (256 modes) block groups 4096 B apart, B (128 modes) 2048;
                        // lo parts 16 KB (A) / 8 KB (B) after the hi parts
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint64_t bh = desc_add(dB, so + kk * 4096);
                            const uint64_t bl = desc_add(dB, so + 8192 + kk * 4096);
#pragma unroll
                            for (int acc = 0; acc < 2; ++acc) {
                                const uint32_t ao = acc * 2048 + kk * 8192;
                                const uint64_t ah = desc_add(dA, so + ao);
                                const uint64_t al = desc_add(dA, so + 16384 + ao);
                                const bool accum = sc > 0 || kk > 0;
                                mma_bf16_pair(tmem + acc * 256, al, bh, idesc, accum);
                                mma_bf16_pair(tmem + acc * 256, ah, bl, idesc, true);
                                mma_bf16_pair(tmem + acc * 256, ah, bh, idesc, true);
                            }
                        }
                    }
                    mma_commit_pair(&bars.empty[s], 0x3);
                    if (sc == cst - 1 || st == nst - 1) {
                        mma_commit_pair(&bars.acc_full, 0x3);
                        ++dc;
                    }
                }
            }
            mma_commit_pair(&bars.drain, 0x1);
            if (!mbar_wait(&bars.drain, 0, kWaitLimit, nullptr)) raise_timeout(args.status, abort_flag);
        } else if (rank == 1 && lane == 0) {
            // ---------------- relay (odd CTA): gen_done[s] complete -> even CTA's full[s] ----------------
            uint32_t it = 0;
            for (int unit = pair; unit < args.units && !*abort_flag; unit += npairs) {
                const int slice = unit % args.slices;
                const int b0 = slice * args.slice_len;
                const int nst = (min(args.n, b0 + args.slice_len) - b0 + C_KB - 1) / C_KB;
                for (int st = 0; st < nst; ++st, ++it) {
                    const int s = it % P_STAGES;
                    // phase it / P_STAGES of gen_done[s]: the next one needs this relay first
                    if (!mbar_wait(&bars.gen_done[s], (it / P_STAGES) & 1, kWaitLimit, abort_flag)) {
                        raise_timeout(args.status, abort_flag);
                        break;
                    }
                    mbar_arrive_cluster(mapa_shared(smem_u32(&bars.full[s]), 0));
                }
            }
        }
        __syncwarp();
    } else if (warp <= C_EPI_WARPS) {
        // ---------------- epilogue: this CTA's 128 rows of each accumulator ----------------
        const int quarter = warp & 3, acc = (warp - 1) >> 2;
        const int rsub = lane >> 2, csub = 2 * (lane & 3);
        uint32_t dc = 0;
        for (int unit = pair; unit < args.units; unit += npairs) {
            if (*abort_flag) break;
            const int tile = unit / args.slices, slice = unit % args.slices;
            const int tu = tile / tiles_v, tv = tile % tiles_v;
            const int b0 = slice * args.slice_len;
            const int nst = (min(args.n, b0 + args.slice_len) - b0 + C_KB - 1) / C_KB;
            const int nch = (nst + chain_stages<PREC>(nst) - 1) / chain_stages<PREC>(nst);
#pragma unroll 1
            for (int ch = 0; ch < nch; ++ch, ++dc) {
                if (!mbar_wait(&bars.acc_full, dc & 1, kWaitLimit, abort_flag)) {
                    raise_timeout(args.status, abort_flag);
                    break;
                }
                tc_fence_after();
#pragma unroll 1
                for (int half = 0; half < 2; ++half) {
                    const int r0 = quarter * 32 + half * 16;
                    // TMEM lane i of accumulator acc: mode tile_u0 + 256 acc + 2 i + rank (TF32,
                    // interleaved rows) or tile_u0 + 256 acc + 128 rank + i (BF16x3)
                    const int i0 = r0 + rsub;
                    const int u = PREC == 1 ? tu * P_TILE_U + acc * 256 + 2 * i0 + (int)rank
                                            : tu * P_TILE_U + acc * 256 + (int)rank * 128 + i0;
                    float *dst0 = args.part + ((size_t)slice * args.Mxc + u) * args.Myc + tv * P_TILE_V + csub;
                    float *dst1 = dst0 + (size_t)(PREC == 1 ? 16 : 8) * args.Myc;      // lane i0 + 8
#pragma unroll 1
                    for (int c = 0; c < 256; c += 64) {
                        float v[32];
                        tmem_ld_16x256b_x8(tmem + ((uint32_t)r0 << 16) + acc * 256 + c, v);
                        tmem_ld_wait_regs32(v);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            float *p0 = dst0 + c + 8 * j, *p1 = dst1 + c + 8 * j;
                            if (ch == 0) {
                                *reinterpret_cast<float2 *>(p0) = make_float2(v[4 * j], v[4 * j + 1]);
                                *reinterpret_cast<float2 *>(p1) = make_float2(v[4 * j + 2], v[4 * j + 3]);
                            } else {
                                red_add2(p0, v[4 * j], v[4 * j + 1]);
                                red_add2(p1, v[4 * j + 2], v[4 * j + 3]);
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(acc_empty0);
            }
        }
    } else if (warp < C_LOADER_WARP) {
        // ---------------- basis generators ----------------
        const int g = threadIdx.x - 32 * (1 + C_EPI_WARPS);    // 0..511
        const int gr = g >> 8;
        const int which = (g >> 7) & 1;                        // 0: Xt (A), 1: Yt (B)
        const int gg = g & 127;
        uint32_t it = 0;
        for (int unit = pair; unit < args.units; unit += npairs) {
            const int tile = unit / args.slices, slice = unit % args.slices;
            const int tu = tile / tiles_v, tv = tile % tiles_v;
            const int b0 = slice * args.slice_len;
            const int b1 = min(args.n, b0 + args.slice_len);
            const int nst = (b1 - b0 + C_KB - 1) / C_KB;
            for (int st = 0; st < nst; ++st, ++it) {
                if (*abort_flag) break;
                if ((int)(it % C_GEN_GROUPS) != gr) continue;
                const int s = it % P_STAGES;
                // empty first (the MMAs of this slot's previous use are complete, so both
                // generator groups are past it), then this use's records
                if ((it >= P_STAGES &&
                     !mbar_wait(&bars.empty[s], ((it / P_STAGES) - 1) & 1, kWaitLimit, abort_flag)) ||
                    !mbar_wait(&bars.recs_full[s], (it / P_STAGES) & 1, kWaitLimit, abort_flag)) {
                    raise_timeout(args.status, abort_flag);
                    break;
                }
                unsigned char *sb = smem + s * P_STAGE_BYTES;
                const AxisRec *recs =
                    reinterpret_cast<const AxisRec *>(recs_base + s * C_REC_BYTES) + which * C_KB;
                const int nvalid = min(C_KB, b1 - (b0 + st * C_KB));
                if (which == 0) {
                    if (PREC == 1) {
                        gen_pair_tf32_interleaved(sb, recs, nvalid, tu * P_TILE_U + (int)rank, gg);
                    } else {
                        const int mb0 = tu * P_TILE_U + (int)rank * 128;
                        gen_pair_bf16(sb, sb + 16384, recs, nvalid, mb0, 2, 4096, gg);
                    }
                } else {
                    const int mb = tv * P_TILE_V + (int)rank * 128;
                    if (PREC == 1)
                        gen_pair_tf32(sb + P_A_BYTES, recs, nvalid, mb, 0, 1, gg);
                    else
                        gen_pair_bf16(sb + P_A_BYTES, sb + P_A_BYTES + 8192, recs, nvalid, mb, 1, 2048, gg);
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&bars.gen_done[s]);          // odd CTA: relayed by warp 0
                    if (rank == 0) mbar_arrive(&bars.full[s]);
                }
            }
            if (*abort_flag) break;
        }
    } else {
        // ---------------- record loader (each CTA its own copy of the stage's records) ----------------
        if (lane == 0) {
            uint32_t it = 0;
            for (int unit = pair; unit < args.units; unit += npairs) {
                const int slice = unit % args.slices;
                const int b0 = slice * args.slice_len;
                const int b1 = min(args.n, b0 + args.slice_len);
                const int nst = (b1 - b0 + C_KB - 1) / C_KB;
                for (int st = 0; st < nst; ++st, ++it) {
                    if (*abort_flag) break;
                    const int s = it % P_STAGES;
                    if (it >= P_STAGES &&
                        !mbar_wait(&bars.gen_done[s], ((it / P_STAGES) - 1) & 1, kWaitLimit, abort_flag)) {
                        raise_timeout(args.status, abort_flag);
                        break;
                    }
                    const int blk0 = b0 + st * C_KB;
                    const uint32_t bytes = (uint32_t)min(C_KB, b1 - blk0) * (uint32_t)sizeof(AxisRec);
                    unsigned char *dst = recs_base + s * C_REC_BYTES;
                    mbar_arrive_expect_tx(&bars.recs_full[s], 2 * bytes);
                    bulk_load(dst, args.xr + blk0, bytes, &bars.recs_full[s]);
                    bulk_load(dst + C_KB * sizeof(AxisRec), args.yr + blk0, bytes, &bars.recs_full[s]);
                }
                if (*abort_flag) break;
            }
            wait_copies_landed(bars.recs_full, P_STAGES, it);
        }
        __syncwarp();
    }
    // both CTAs are done with the tensor memory and the even CTA's MMAs (which read
    // the odd CTA's shared memory) are complete before either CTA frees or exits
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, 512);
    }
}

// ===========================================================================
// Finish: FP64 sum of the slice partials -> a, K in the energy operand layout
// ===========================================================================
// Sum of one double per thread over the CTA, added to *dst (one atomic per CTA).
__device__ __forceinline__ void cta_add_double(double v, double *dst) {
    __shared__ double part_sums[32];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) part_sums[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part_sums[w];
        atomicAdd(dst, t);
    }
}

// e_total (optional, with a computed here from the partials): E = 1/2 sum_uv a_uv S_uv,
// which equals 1/2 sum_i N_i of the blocks the partials came from, in FP64 from the
// FP32 coefficients.  The per-block sums of the energy kernel use K rounded to the
// operand precision; K is shared by all blocks, so its rounding shifts every N_i
// alike and their total by up to about one TF32 unit; this sum does not.
template <int PREC>
__global__ void tc_finish_kernel(const float *__restrict__ part, int slices, int Mxc, int Myc,
                                 const float *__restrict__ a_in, float *__restrict__ a_out,
                                 void *__restrict__ Kop, void *__restrict__ Klo, int Mx, int My,
                                 int Mxe, int Mye, float piW, float piH, float invWH,
                                 double *__restrict__ e_total, unsigned *__restrict__ split_cnt,
                                 int nsplit, double *__restrict__ a64) {
    pdl_wait();                        // the slice partials come from the coefficient kernel
    pdl_trigger();                     // the energy kernel may be scheduled (it waits for this one)
    // the energy kernel that follows finds its split-tile counters at zero
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < nsplit; i += blockDim.x) split_cnt[i] = 0u;
    // FP32 throughout (FP64 is a narrow pipe on this GPU): the slice partials are
    // summed with Kahan compensation; the operand is TF32 or bf16 anyway.
    float e_acc = 0.f;                 // this thread's few terms; summed across the CTA in FP64
    // 32-bit indices (Mxe * Mye <= 4096^2); Mye is a multiple of 256
    const int total = Mxe * Mye, mye_sh = 31 - __clz(Mye & -Mye), mye_odd = Mye >> mye_sh;
    const size_t sstride = (size_t)Mxc * Myc;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        // u = idx / Mye, v = idx % Mye with Mye = mye_odd * 2^mye_sh (mye_odd is 1 for
        // the powers of two of every workload, else a 32-bit division)
        const int q = idx >> mye_sh;
        const int u = mye_odd == 1 ? q : q / mye_odd;
        const int v = idx - u * Mye;
        float kv = 0.f;
        if (u < Mx && v < My) {
            const float uf = (float)(u > 0 ? u : 1), vf = (float)(v > 0 ? v : 1);
            // f g = (2W / (pi u')) (2H / (pi v')) = 4 / (piW piH u' v'), u' v' < 2^24 exact
            const float fg = 4.0f / (piW * piH * (uf * vf));
            float av;
            if (a_in) {
                av = a_in[(size_t)u * My + v];
            } else {
                // slices in order (Kahan), their loads issued eight at a time
                float S = 0.f, comp = 0.f;
                const float *src = part + (size_t)u * Myc + v;
                int s = 0;
                for (; s + 8 <= slices; s += 8) {
                    float pv[8];
#pragma unroll
                    for (int q8 = 0; q8 < 8; ++q8) pv[q8] = __ldcg(src + (size_t)(s + q8) * sstride);
#pragma unroll
                    for (int q8 = 0; q8 < 8; ++q8) {
                        const float y = pv[q8] - comp;
                        const float t = S + y;
                        comp = (t - S) - y;
                        S = t;
                    }
                }
                for (; s < slices; ++s) {
                    const float y = __ldcg(src + (size_t)s * sstride) - comp;
                    const float t = S + y;
                    comp = (t - S) - y;
                    S = t;
                }
                const float ku = (float)u * piW, lv = (float)v * piH;
                const float eps = (u ? 2.f : 1.f) * (v ? 2.f : 1.f);
                const float G = (u == 0 && v == 0) ? 0.f : eps * invWH / (ku * ku + lv * lv);
                av = G * fg * S;
                if (a64) {                      // running FP64 sum over calls (chunks, ranks)
                    const double t = a64[(size_t)u * My + v] + (double)av;
                    a64[(size_t)u * My + v] = t;
                    if (a_out) a_out[(size_t)u * My + v] = (float)t;
                } else if (a_out) {
                    a_out[(size_t)u * My + v] = av;
                }
                e_acc = fmaf(0.5f * av, fg * S, e_acc);
            }
            kv = fg * av;
        }
        if (!Kop) continue;
        const int vb = v >> 8, vi = v & 255;
        if (PREC == 1) {
            const int off = ((vb * (Mxe >> 2) + (u >> 2)) * 256 + vi) * 4 + (u & 3);
            reinterpret_cast<float *>(Kop)[off] = to_tf32(kv);
        } else {
            const int off = ((vb * (Mxe >> 3) + (u >> 3)) * 256 + vi) * 8 + (u & 7);
            __nv_bfloat16 hi, lo;
            split_bf16(kv, hi, lo);
            reinterpret_cast<__nv_bfloat16 *>(Kop)[off] = hi;
            reinterpret_cast<__nv_bfloat16 *>(Klo)[off] = lo;
        }
    }
    if (e_total) cta_add_double((double)e_acc, e_total);
}

// ===========================================================================
// Energy and gradient
// ===========================================================================
constexpr int E_ROWS = kEnergyRows;         // blocks per row tile
constexpr int E_VC = 256;                   // v columns per accumulator pass
constexpr int E_KS = 32;                    // u per pipeline stage
constexpr int E_STAGES = 3;
constexpr int E_STAGE_BYTES = 65536;        // A (Xt, Xh) 32 KB + B (K) 32 KB
constexpr int E_GEN_WARPS = 8;              // two groups of 4 warps, alternate stages
constexpr int E_EPI_WARPS = 8;              // two per TMEM lane quarter, 128 columns each
constexpr int E_THREADS = 32 * (2 + E_EPI_WARPS + E_GEN_WARPS);
constexpr int E_DRAIN_THREADS = 32 * E_EPI_WARPS;
constexpr int E_DRAIN_COLS = E_VC / 2;

struct EnergyBars {
    uint64_t full[E_STAGES];        // generator group of the stage
    uint64_t kfull[E_STAGES];       // the stage's K tile (TMA bytes)
    uint64_t empty[E_STAGES];
    uint64_t acc_full;
    uint64_t acc_empty;
    uint64_t drain;
    uint32_t tmem_slot;
    int abort_flag;
    float red[2][E_ROWS][3];    // per segment parity: column half 1 of each row, for half 0
    unsigned split_old;         // boundary counter value seen by this CTA
};
constexpr int E_SMEM = E_STAGES * E_STAGE_BYTES + 1024 + (int)sizeof(EnergyBars);

// Row tiles of E_ROWS blocks, each a sequence of nvc accumulator passes: the
// tiles * nvc (tile, pass) units are cut into gridDim.x equal ranges, one per CTA,
// so a tile may be split between two neighbouring CTAs (never three: a range has
// at least nvc units).  The two parts of a split tile meet in `split`: the CTA that
// arrives second at the boundary counter adds head + tail and writes the outputs.
struct EnergyArgs {
    const AxisRec *xr, *yr;
    int n, tiles, Mx, My, Mxe, Mye;      // tiles: row tiles of E_ROWS blocks
    float *split;                        // [gridDim.x + 1][2][E_ROWS][3]
    unsigned *split_cnt;                 // [gridDim.x + 1], zero at launch (finish kernel)
    float *e_block, *gx, *gy;
    double *e_total;
    unsigned *status;
    GradOut go;                          // what happens to gx, gy before they are written
};

// Energy-operand generator: one block, the stage's 32 consecutive u, written as
// K-major 16-byte rows (4 tf32 or 8 bf16 u each) as they are produced.
// SAMPLE 0 (rectangle): Xt = c cos(pi u s) sin(pi u t)  (c pi t at u = 0),
//                       Xh = -(u pi/W) c sin(pi u s) sin(pi u t);
// SAMPLE 1 (centre):    Xt = q cos(pi u s)/f_u,  Xh = -q (u pi/W) sin(pi u s)/f_u.
// Rectangle mode advances (u, u+1) as two packed chains with a 2-mode step.
template <int SAMPLE>
struct EnergyChain {
    // SAMPLE 0 state
    c2 Z, T;
    gen::rot2_step S2, T2;
    f2 nku, dku;
    // SAMPLE 1 state
    float2 zs, es;
    float ku, inv_l, q;
    int u;
    bool valid;
    __device__ __forceinline__ void init(const AxisRec &R, bool v, int u0) {
        valid = v;
        u = u0;
        if (!v) return;
        if (SAMPLE == 0) {
            const float2 za = gen::phase_poly((unsigned long long)u0, R.s);
            float2 ta = gen::phase_poly((unsigned long long)u0, R.t);
            ta.x *= R.c;
            ta.y *= R.c;
            Z = gen::make_c2(za, rot(za, R.es));
            T = gen::make_c2(ta, rot(ta, R.et));
            const float2 es2 = rot(R.es, R.es), et2 = rot(R.et, R.et);
            S2 = gen::make_step(es2, es2);
            T2 = gen::make_step(et2, et2);
            nku = gen::pk(-(float)u0 * R.inv_l, -(float)(u0 + 1) * R.inv_l);
            dku = gen::pk(-2.f * R.inv_l, -2.f * R.inv_l);
        } else {
            zs = gen::phase_poly((unsigned long long)u0, R.s);
            es = R.es;
            ku = (float)u0 * R.inv_l;
            inv_l = R.inv_l;
            q = R.q;
        }
    }
    // the next two u: Xt, Xh
    __device__ __forceinline__ void next2(float &t0, float &t1, float &h0, float &h1) {
        if (!valid) {
            t0 = t1 = h0 = h1 = 0.f;
            return;
        }
        if (SAMPLE == 0) {
            gen::upk(gen::mul2(Z.re, T.im), t0, t1);
            gen::upk(gen::mul2(nku, gen::mul2(Z.im, T.im)), h0, h1);
            nku = gen::add2(nku, dku);
            Z = gen::rot2(Z, S2);
            T = gen::rot2(T, T2);
        } else {
            float tt[2], hh[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int m = u + e;
                const float inv_f = 0.5f * (float)(m > 0 ? m : 1) * inv_l;   // 1 / f_u
                tt[e] = q * zs.x * inv_f;
                hh[e] = -q * ku * zs.y * inv_f;
                zs = rot(zs, es);
                ku += inv_l;
            }
            t0 = tt[0];
            t1 = tt[1];
            h0 = hh[0];
            h1 = hh[1];
        }
        u += 2;
    }
};

// TF32, rectangle sampling: the stage's modes u0 .. u0 + 31 as two chains, u0 + j
// (lane a) and u0 + 16 + j (lane b) for j = 0..15, advanced together in packed
// registers.  cos(pi u s), sin(pi u s) and c sin(pi u t) follow the signed
// three-term recurrence of the TF32 coefficient generator (one FMA per step,
// signs +,+,-,- shared by the three chains, so that the products are the basis
// values); 16 steps keep the rounding below 128 FP32 units (8e-6) and the
// hardware sine and cosine anchors (error 4e-7) below 16 times theirs, far under
// the TF32 operand rounding.
__device__ __forceinline__ void gen_energy_tf32_rect(unsigned char *sb, const AxisRec &R, bool valid, int row,
                                                     int u0) {
    f2 C, S, T, Cp, Sp, Tp, KZ, KT, nku, dku;
    float v0 = 0.f;
    if (valid) {
        const float2 za = gen::phase_sfu((unsigned long long)u0, R.s);
        const float2 ta = gen::phase_sfu((unsigned long long)u0, R.t);
        const float2 zb = rot(za, rot(R.es8, R.es8));      // u0 + 16: times e^{i 16 pi s}
        const float2 tb = rot(ta, rot(R.et8, R.et8));
        const float2 es = R.es, et = R.et;
        C = gen::pk(za.x, zb.x);
        S = gen::pk(za.y, zb.y);
        T = gen::pk(R.c * ta.y, R.c * tb.y);
        // s_{-1} = -y_{-1}, the chains' values at u - 1 (rotation by conj(e^{i pi s}))
        Cp = gen::pk(-fmaf(za.x, es.x, za.y * es.y), -fmaf(zb.x, es.x, zb.y * es.y));
        Sp = gen::pk(-fmaf(za.y, es.x, -za.x * es.y), -fmaf(zb.y, es.x, -zb.x * es.y));
        Tp = gen::pk(-R.c * fmaf(ta.y, et.x, -ta.x * et.y), -R.c * fmaf(tb.y, et.x, -tb.x * et.y));
        KZ = gen::pk(2.f * es.x, 2.f * es.x);
        KT = gen::pk(2.f * et.x, 2.f * et.x);
        nku = gen::pk(-(float)u0 * R.inv_l, -(float)(u0 + 16) * R.inv_l);
        dku = gen::pk(-R.inv_l, -R.inv_l);
        v0 = R.v0;
    } else {
        C = S = T = Cp = Sp = Tp = KZ = KT = nku = dku = gen::pk(0.f, 0.f);
    }
    const f2 NKZ = gen::pk(-KZ.v.x, -KZ.v.y), NKT = gen::pk(-KT.v.x, -KT.v.y);
    // [128 rows x 32 u] tf32 K-major: core (row/8, u/4) at (row/8)*1024 + (u/4)*128
    unsigned char *A = sb + (size_t)(row >> 3) * 1024 + (row & 7) * 16;
    auto step = [&](const f2 &kz, const f2 &kt) {
        const f2 nc = gen::fma2(kz, C, Cp), ns = gen::fma2(kz, S, Sp), nt = gen::fma2(kt, T, Tp);
        Cp = C;
        C = nc;
        Sp = S;
        S = ns;
        Tp = T;
        T = nt;
        nku = gen::add2(nku, dku);
    };
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
        float ta[4], tb[4], ha[4], hb[4];
#pragma unroll
        for (int jj = 0; jj < 4; jj += 2) {
            gen::upk(gen::mul2(C, T), ta[jj], tb[jj]);
            gen::upk(gen::mul2(gen::mul2(S, T), nku), ha[jj], hb[jj]);
            step(KZ, KT);                                   // even j: +2 cos
            gen::upk(gen::mul2(C, T), ta[jj + 1], tb[jj + 1]);
            gen::upk(gen::mul2(gen::mul2(S, T), nku), ha[jj + 1], hb[jj + 1]);
            step(NKZ, NKT);                                 // odd j: -2 cos
        }
        if (c == 0 && u0 == 0 && valid) ta[0] = v0;        // u = 0: c pi t, not the sine limit
        *reinterpret_cast<float4 *>(A + c * 128) =
            make_float4(to_tf32_mma(ta[0]), to_tf32_mma(ta[1]), to_tf32_mma(ta[2]), to_tf32_mma(ta[3]));
        *reinterpret_cast<float4 *>(A + 16384 + c * 128) =
            make_float4(to_tf32_mma(ha[0]), to_tf32_mma(ha[1]), to_tf32_mma(ha[2]), to_tf32_mma(ha[3]));
        *reinterpret_cast<float4 *>(A + (c + 4) * 128) =
            make_float4(to_tf32_mma(tb[0]), to_tf32_mma(tb[1]), to_tf32_mma(tb[2]), to_tf32_mma(tb[3]));
        *reinterpret_cast<float4 *>(A + 16384 + (c + 4) * 128) =
            make_float4(to_tf32_mma(hb[0]), to_tf32_mma(hb[1]), to_tf32_mma(hb[2]), to_tf32_mma(hb[3]));
    }
}

template <int PREC, int SAMPLE>
__device__ __forceinline__ void gen_energy(unsigned char *sb, const AxisRec &R, bool valid, int row,
                                           int u0) {
    if (PREC == 1 && SAMPLE == 0) {
        gen_energy_tf32_rect(sb, R, valid, row, u0);
        return;
    }
    // two independent chains: u0..u0+15 (a) and u0+16..u0+31 (b)
    EnergyChain<SAMPLE> a, b;
    a.init(R, valid, u0);
    b.init(R, valid, u0 + 16);
    if (PREC == 1) {
        // [128 rows x 32 u] tf32 K-major: core (row/8, u/4) at (row/8)*1024 + (u/4)*128
        unsigned char *A = sb + (size_t)(row >> 3) * 1024 + (row & 7) * 16;
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
            float t[4], h[4], tb[4], hb[4];
            a.next2(t[0], t[1], h[0], h[1]);
            b.next2(tb[0], tb[1], hb[0], hb[1]);
            a.next2(t[2], t[3], h[2], h[3]);
            b.next2(tb[2], tb[3], hb[2], hb[3]);
            if (SAMPLE == 0 && c == 0 && u0 == 0 && valid) t[0] = R.v0;
            *reinterpret_cast<float4 *>(A + c * 128) =
                make_float4(to_tf32_mma(t[0]), to_tf32_mma(t[1]), to_tf32_mma(t[2]), to_tf32_mma(t[3]));
            *reinterpret_cast<float4 *>(A + 16384 + c * 128) =
                make_float4(to_tf32_mma(h[0]), to_tf32_mma(h[1]), to_tf32_mma(h[2]), to_tf32_mma(h[3]));
            *reinterpret_cast<float4 *>(A + (c + 4) * 128) =
                make_float4(to_tf32_mma(tb[0]), to_tf32_mma(tb[1]), to_tf32_mma(tb[2]), to_tf32_mma(tb[3]));
            *reinterpret_cast<float4 *>(A + 16384 + (c + 4) * 128) =
                make_float4(to_tf32_mma(hb[0]), to_tf32_mma(hb[1]), to_tf32_mma(hb[2]), to_tf32_mma(hb[3]));
        }
    } else {
        // [128 rows x 32 u] bf16 K-major: core (row/8, u/8) at (row/8)*512 + (u/8)*128;
        // regions Xt hi, Xt lo, Xh hi, Xh lo (8 KB each)
        unsigned char *A = sb + (size_t)(row >> 3) * 512 + (row & 7) * 16;
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
            uint32_t th[4], tl[4], hh[4], hl[4], th2[4], tl2[4], hh2[4], hl2[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float t0, t1, h0, h1, q0, q1, g0, g1;
                a.next2(t0, t1, h0, h1);
                b.next2(q0, q1, g0, g1);
                if (SAMPLE == 0 && c == 0 && j == 0 && u0 == 0 && valid) t0 = R.v0;
                split2(t0, t1, th[j], tl[j]);
                split2(h0, h1, hh[j], hl[j]);
                split2(q0, q1, th2[j], tl2[j]);
                split2(g0, g1, hh2[j], hl2[j]);
            }
            *reinterpret_cast<uint4 *>(A + c * 128) = make_uint4(th[0], th[1], th[2], th[3]);
            *reinterpret_cast<uint4 *>(A + 8192 + c * 128) = make_uint4(tl[0], tl[1], tl[2], tl[3]);
            *reinterpret_cast<uint4 *>(A + 16384 + c * 128) = make_uint4(hh[0], hh[1], hh[2], hh[3]);
            *reinterpret_cast<uint4 *>(A + 24576 + c * 128) = make_uint4(hl[0], hl[1], hl[2], hl[3]);
            *reinterpret_cast<uint4 *>(A + (c + 2) * 128) = make_uint4(th2[0], th2[1], th2[2], th2[3]);
            *reinterpret_cast<uint4 *>(A + 8192 + (c + 2) * 128) = make_uint4(tl2[0], tl2[1], tl2[2], tl2[3]);
            *reinterpret_cast<uint4 *>(A + 16384 + (c + 2) * 128) = make_uint4(hh2[0], hh2[1], hh2[2], hh2[3]);
            *reinterpret_cast<uint4 *>(A + 24576 + (c + 2) * 128) = make_uint4(hl2[0], hl2[1], hl2[2], hl2[3]);
        }
    }
}

// The y-axis fields one epilogue row needs.
struct YRec {
    unsigned long long s, t;
    float2 es, et;
    float inv_l, v0;
};
__device__ __forceinline__ YRec load_yrec(const AxisRec *yr, int b) {
    const AxisRec &R = yr[b];
    YRec y;
    y.s = R.s;
    y.t = R.t;
    y.es = R.es;
    y.et = R.et;
    y.inv_l = R.inv_l;
    y.v0 = R.v0;
    return y;
}

// Row dots of one thread's 8 columns (rectangle sampling): Yt and Yh advance as
// packed chains over column pairs.
struct EpiRect {
    c2 Z, T;
    gen::rot2_step S2, T2;
    f2 nlv, dlv, EN, EX, EY;
    __device__ __forceinline__ void init(const YRec &Ry, int vb) {
        const float2 za = gen::phase_poly((unsigned long long)vb, Ry.s);
        const float2 ta = gen::phase_poly((unsigned long long)vb, Ry.t);
        Z = gen::make_c2(za, rot(za, Ry.es));
        T = gen::make_c2(ta, rot(ta, Ry.et));
        const float2 es2 = rot(Ry.es, Ry.es), et2 = rot(Ry.et, Ry.et);
        S2 = gen::make_step(es2, es2);
        T2 = gen::make_step(et2, et2);
        nlv = gen::pk(-(float)vb * Ry.inv_l, -(float)(vb + 1) * Ry.inv_l);
        dlv = gen::pk(-2.f * Ry.inv_l, -2.f * Ry.inv_l);
        EN = EX = EY = gen::pk(0.f, 0.f);
    }
    __device__ __forceinline__ void cols8(const float t[8], const float tp[8]) {
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            const f2 tt = gen::pk(t[j], t[j + 1]), ttp = gen::pk(tp[j], tp[j + 1]);
            const f2 yt = gen::mul2(Z.re, T.im), pr = gen::mul2(Z.im, T.im);
            EN = gen::fma2(tt, yt, EN);
            EX = gen::fma2(ttp, yt, EX);
            EY = gen::fma2(gen::mul2(tt, nlv), pr, EY);
            nlv = gen::add2(nlv, dlv);
            Z = gen::rot2(Z, S2);
            T = gen::rot2(T, T2);
        }
    }
    __device__ __forceinline__ void sums(float &aN, float &aX, float &aY) const {
        float x0, x1;
        gen::upk(EN, x0, x1);
        aN = x0 + x1;
        gen::upk(EX, x0, x1);
        aX = x0 + x1;
        gen::upk(EY, x0, x1);
        aY = x0 + x1;
    }
};
// Row dots for TF32 operands (rectangle sampling): cos(pi v s), sin(pi v s) and
// sin(pi v t) over column pairs (v, v + 1) as signed three-term recurrences with a
// 2-mode step (one FMA per step, signs +,+,-,- shared by the three chains), anchored
// again from the phase (hardware sine and cosine) every 64 columns, so that no
// chain runs more than 32 steps (rounding below 512 FP32 units).  The derivative
// dot sum_k n_k a_k, with a_k = T'_k sin(pi v s) sin(pi v t) and the linear weight
// n_k = n_0 + k d (n = -l_v), is summed as n_0 A + d (K A - B) with A = sum a_k and
// B = sum of the partial sums of A (sum_k k a_k = K A - B): two operations a step
// instead of three.
struct EpiRect3 {
    f2 C, S, T, Cp, Sp, Tp, K, KT, n0, EN, EX, EA, EB;
    float dl;
    int col;
    __device__ __forceinline__ void anchor(const YRec &Ry, int v) {
        const float2 z = gen::phase_sfu((unsigned long long)v, Ry.s);
        const float2 t = gen::phase_sfu((unsigned long long)v, Ry.t);
        const float2 z1 = rot(z, Ry.es), t1 = rot(t, Ry.et);
        const float2 e2s = rot(Ry.es, Ry.es), e2t = rot(Ry.et, Ry.et);
        const float2 ce2s = make_float2(e2s.x, -e2s.y), ce2t = make_float2(e2t.x, -e2t.y);
        const float2 zp = rot(z, ce2s), zp1 = rot(z1, ce2s), tp = rot(t, ce2t), tp1 = rot(t1, ce2t);
        C = gen::pk(z.x, z1.x);
        S = gen::pk(z.y, z1.y);
        T = gen::pk(t.y, t1.y);
        Cp = gen::pk(-zp.x, -zp1.x);                        // s_{-1} = -y_{-1}
        Sp = gen::pk(-zp.y, -zp1.y);
        Tp = gen::pk(-tp.y, -tp1.y);
        K = gen::pk(2.f * e2s.x, 2.f * e2s.x);
        KT = gen::pk(2.f * e2t.x, 2.f * e2t.x);
    }
    __device__ __forceinline__ void init(const YRec &Ry, int vb) {
        anchor(Ry, vb);
        n0 = gen::pk(-(float)vb * Ry.inv_l, -(float)(vb + 1) * Ry.inv_l);
        dl = -2.f * Ry.inv_l;
        EN = EX = EA = EB = gen::pk(0.f, 0.f);
        col = 0;
    }
    __device__ __forceinline__ void cols8(const float t[8], const float tp[8], const YRec &Ry, int vb) {
        if (col > 0 && (col & 63) == 0) anchor(Ry, vb + col);
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            const f2 tt = gen::pk(t[j], t[j + 1]), ttp = gen::pk(tp[j], tp[j + 1]);
            const f2 yt = gen::mul2(C, T), pr = gen::mul2(S, T);
            EN = gen::fma2(tt, yt, EN);
            EX = gen::fma2(ttp, yt, EX);
            EA = gen::fma2(tt, pr, EA);
            EB = gen::add2(EB, EA);
            // step j / 2 of the chain: +2 cos for even, -2 cos for odd
            const f2 k = (j & 2) ? gen::pk(-K.v.x, -K.v.y) : K;
            const f2 kt = (j & 2) ? gen::pk(-KT.v.x, -KT.v.y) : KT;
            const f2 nc = gen::fma2(k, C, Cp), ns = gen::fma2(k, S, Sp), nt = gen::fma2(kt, T, Tp);
            Cp = C;
            C = nc;
            Sp = S;
            S = ns;
            Tp = T;
            T = nt;
        }
        col += 8;
    }
    __device__ __forceinline__ void sums(float &aN, float &aX, float &aY) const {
        float x0, x1;
        gen::upk(EN, x0, x1);
        aN = x0 + x1;
        gen::upk(EX, x0, x1);
        aX = x0 + x1;
        const float steps = (float)(col >> 1);
        const f2 kab = gen::fma2(gen::pk(steps, steps), EA, gen::pk(-EB.v.x, -EB.v.y));   // K A - B
        gen::upk(gen::fma2(n0, EA, gen::mul2(gen::pk(dl, dl), kab)), x0, x1);
        aY = x0 + x1;
    }
};

// Centre sampling: Yt = cos(pi v s') / g_v, Yh = -l_v sin(pi v s') / g_v, one chain.
struct EpiCenter {
    float2 zs, es;
    float lv, inv_l;
    int v;
    float aN, aX, aY;
    __device__ __forceinline__ void init(const YRec &Ry, int vb) {
        zs = gen::phase_poly((unsigned long long)vb, Ry.s);
        es = Ry.es;
        inv_l = Ry.inv_l;
        lv = (float)vb * Ry.inv_l;
        v = vb;
        aN = aX = aY = 0.f;
    }
    __device__ __forceinline__ void cols8(const float t[8], const float tp[8]) {
#pragma unroll
        for (int j = 0; j < 8; ++j, ++v) {
            const float inv_g = 0.5f * (float)(v > 0 ? v : 1) * inv_l;
            const float yt = zs.x * inv_g;
            const float yh = -lv * zs.y * inv_g;
            aN = fmaf(t[j], yt, aN);
            aY = fmaf(t[j], yh, aY);
            aX = fmaf(tp[j], yt, aX);
            zs = rot(zs, es);
            lv += inv_l;
        }
    }
    __device__ __forceinline__ void sums(float &a, float &b, float &c) const {
        a = aN;
        b = aX;
        c = aY;
    }
};

__device__ __forceinline__ void epi_cols8(EpiRect3 &ep, const float t[8], const float tp[8], const YRec &Ry,
                                          int vb) {
    ep.cols8(t, tp, Ry, vb);
}
template <class E>
__device__ __forceinline__ void epi_cols8(E &ep, const float t[8], const float tp[8], const YRec &, int) {
    ep.cols8(t, tp);
}

// One thread's share of accumulator pass pc: TMEM lane row (trow), columns
// [cb, cb + E_DRAIN_COLS) of the pass, global column base vb; adds its row dots
// to (eN, eX, eY) and releases its part of TMEM.
template <int PREC, int SAMPLE>
__device__ __forceinline__ void drain_pass(EnergyBars &bars, volatile int *abort_flag, unsigned *status,
                                           uint32_t trow, int cb, int vb, int pc, bool valid,
                                           const YRec &Ry, float &eN, float &eX, float &eY) {
    if (*abort_flag) return;
    constexpr bool R3 = PREC == 1 && SAMPLE == 0;
    typename std::conditional<R3, EpiRect3, typename std::conditional<SAMPLE == 0, EpiRect, EpiCenter>::type>::type ep;
    if (valid) ep.init(Ry, vb);          // phase anchors ahead of the wait
    if (!mbar_wait(&bars.acc_full, pc & 1, kWaitLimit, abort_flag)) {
        raise_timeout(status, abort_flag);
        return;
    }
    tc_fence_after();
    // 16-column chunks (T and T' of each): one load round per chunk, whose
    // latency is paid once per 16 columns
    float tA[16], pA[16];
    float fixN = 0.f, fixX = 0.f;
#pragma unroll 1
    for (int c = 0; c < E_DRAIN_COLS; c += 16) {
        tmem_ld16(trow + cb + c, tA);
        tmem_ld16(trow + cb + c + 256, pA);
        tmem_ld_wait_regs16(tA, pA);
        // v = 0 column (rectangle sampling): Yt = pi t there, not the sine limit 0 the
        // chain gives; Yh = 0
        if (SAMPLE == 0 && c == 0 && vb == 0) {
            fixN = tA[0] * Ry.v0;
            fixX = pA[0] * Ry.v0;
        }
        if (valid) {
            epi_cols8(ep, tA, pA, Ry, vb);
            epi_cols8(ep, tA + 8, pA + 8, Ry, vb);
        }
    }
    tc_fence_before();
    mbar_arrive(&bars.acc_empty);
    if (valid) {
        float aN, aX, aY;
        ep.sums(aN, aX, aY);
        eN += fixN + aN;
        eX += fixX + aX;
        eY += aY;
    }
}

// End of a tile segment (the passes [v0, v1] of row tile `tile`) for one epilogue
// thread: column half 1 puts its sums in shared memory (double-buffered by segment
// parity, so that a one-pass segment cannot overwrite them before they are read);
// after named barrier 1 (all epilogue threads) half 0 adds them.  A whole tile's
// outputs are written directly; a split tile's part goes to the boundary scratch
// and the second part to arrive writes head + tail (named barrier 2: half 0).
// E gets each part's share directly (it is a sum over blocks).
__device__ __forceinline__ void finish_segment(EnergyBars &bars, volatile int *abort_flag, const EnergyArgs &args,
                                               int seg, int tile, int v0, int v1, int nvc, int row, int cq,
                                               float eN, float eX, float eY) {
    if (cq != 0) {
        float *r = bars.red[seg & 1][row];
        r[0] = eN;
        r[1] = eX;
        r[2] = eY;
    }
    // both halves wait (no half can run ahead into the next segment's arrival and
    // complete a barrier phase that belongs to this one)
    asm volatile("bar.sync 1, %0;" ::"r"(E_DRAIN_THREADS) : "memory");
    if (cq != 0) return;
    const int b = tile * E_ROWS + row;
    const bool valid = b < args.n;
    eN += bars.red[seg & 1][row][0];
    eX += bars.red[seg & 1][row][1];
    eY += bars.red[seg & 1][row][2];
    const bool ok = !*abort_flag;
    double es = valid ? (double)eN : 0.0;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) es += __shfl_xor_sync(0xffffffffu, es, off);
    if ((threadIdx.x & 31) == 0 && args.e_total && ok) atomicAdd(args.e_total, 0.5 * es);
    if (v0 == 0 && v1 == nvc - 1) {
        if (valid && ok) {
            if (args.e_block) args.e_block[b] = eN;
            if (args.gx) args.gx[b] = grad_out(args.go, args.gx, b, eX);
            if (args.gy) args.gy[b] = grad_out(args.go, args.gy, b, eY);
        }
        return;
    }
    // split tile: head part (v0 == 0) ends this CTA's range, tail part starts it
    const int side = v0 == 0 ? 0 : 1;
    const int bd = side == 0 ? blockIdx.x + 1 : blockIdx.x;           // boundary index
    float *mine = args.split + (((size_t)bd * 2 + side) * E_ROWS + row) * 3;
    const float *other = args.split + (((size_t)bd * 2 + (1 - side)) * E_ROWS + row) * 3;
    mine[0] = eN;
    mine[1] = eX;
    mine[2] = eY;
    __threadfence();
    asm volatile("bar.sync 2, %0;" ::"r"(E_ROWS) : "memory");
    if (row == 0) bars.split_old = atomicAdd(&args.split_cnt[bd], 1u);
    asm volatile("bar.sync 2, %0;" ::"r"(E_ROWS) : "memory");
    if (bars.split_old == 1u) {              // the other part is in: head + tail, fixed order
        __threadfence();
        const float o0 = __ldcg(other), o1 = __ldcg(other + 1), o2 = __ldcg(other + 2);
        const float hN = side == 0 ? eN : o0, tN = side == 0 ? o0 : eN;
        const float hX = side == 0 ? eX : o1, tX = side == 0 ? o1 : eX;
        const float hY = side == 0 ? eY : o2, tY = side == 0 ? o2 : eY;
        if (valid && ok) {
            if (args.e_block) args.e_block[b] = hN + tN;
            if (args.gx) args.gx[b] = grad_out(args.go, args.gx, b, hX + tX);
            if (args.gy) args.gy[b] = grad_out(args.go, args.gy, b, hY + tY);
        }
    }
    // keep bars.split_old until every half-0 thread has read it
    asm volatile("bar.sync 2, %0;" ::"r"(E_ROWS) : "memory");
}

// Persistent: each CTA runs its range of (tile, pass) units; the generators and the
// TMA warp fill the next pass's stages while the epilogue drains the previous
// one, and TMEM is allocated once.
template <int PREC, int SAMPLE>
__global__ void __launch_bounds__(E_THREADS, 1)
tc_energy_kernel(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
                 const EnergyArgs args) {
    extern __shared__ unsigned char smem_raw[];
    // 1 KB-aligned base by pointer arithmetic on the __shared__ array, so that the
    // compiler keeps every access in the shared address space (LDS/STS)
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    EnergyBars &bars = *reinterpret_cast<EnergyBars *>(smem + E_STAGES * E_STAGE_BYTES);
    volatile int *abort_flag = &bars.abort_flag;
    constexpr bool BF = PREC == 2;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nvc = args.Mye / E_VC;
    const int nks = args.Mxe / E_KS;
    const long long U = (long long)args.tiles * nvc;              // (tile, pass) units
    const int ub = (int)(U * blockIdx.x / gridDim.x), ue = (int)(U * (blockIdx.x + 1) / gridDim.x);

    if (threadIdx.x == 0) {
        for (int s = 0; s < E_STAGES; ++s) {
            mbar_init(&bars.full[s], (E_GEN_WARPS / 2) * 32);     // one generator group (128 threads)
            mbar_init(&bars.kfull[s], 1);                         // the TMA producer + its bytes
            mbar_init(&bars.empty[s], 1);
        }
        mbar_init(&bars.acc_full, 1);
        mbar_init(&bars.acc_empty, E_DRAIN_THREADS);
        mbar_init(&bars.drain, 1);
        bars.abort_flag = 0;
        mbar_fence_init();
    }
    pdl_wait();                        // K and the split counters come from the finish kernel
    if (warp == 0) {
        tmem_alloc(&bars.tmem_slot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = bars.tmem_slot;

    if (warp == 0) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = instr_desc(BF ? kFmtBF16 : kFmtTF32, 128, 256, false, false);
            // stage 0's operand descriptors (A: LBO 128 (u cores), SBO 1024 (TF32) / 512 (bf16)
            // row groups; B: [u/T][256 v][T] K-major, LBO 4096, SBO 128); the others are byte
            // offsets from them, so that the issue loop keeps to adds and compares
            const uint32_t s0 = smem_u32(smem);
            const uint64_t dA = BF ? smem_desc(s0, 128, 512) : smem_desc(s0, 128, 1024);
            const uint64_t dB = smem_desc(s0 + 32768, 4096, 128);
            int it = 0, pc = 0;       // stages consumed, accumulator passes
            int s = 0, ph = 0;        // it % E_STAGES, (it / E_STAGES) & 1
            for (int un = ub; un < ue && !*abort_flag; ++un, ++pc) {
                {
                    if (pc > 0 && !mbar_wait(&bars.acc_empty, (pc - 1) & 1, kWaitLimit, abort_flag)) {
                        raise_timeout(args.status, abort_flag);
                        break;
                    }
                    tc_fence_after();
                    for (int ks = 0; ks < nks; ++ks, ++it, ph ^= (s + 1 == E_STAGES), s = (s + 1 == E_STAGES ? 0 : s + 1)) {
                        if (!mbar_wait(&bars.full[s], ph, kWaitLimit, abort_flag) ||
                            !mbar_wait(&bars.kfull[s], ph, kWaitLimit, abort_flag)) {
                            raise_timeout(args.status, abort_flag);
                            break;
                        }
                        tc_fence_after();
                        const uint32_t so = (uint32_t)s * E_STAGE_BYTES;
                        if (!BF) {
                            // Xt at +0, Xh at +16 KB, K at +32 KB
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t bd = desc_add(dB, so + kk * 8192);
                                const bool accum = ks > 0 || kk > 0;
                                mma_tf32(tmem, desc_add(dA, so + kk * 256), bd, idesc, accum);
                                mma_tf32(tmem + 256, desc_add(dA, so + 16384 + kk * 256), bd, idesc, accum);
                            }
                        } else {
                            // Xt hi / lo at +0 / +8 KB, Xh hi / lo at +16 / +24 KB, K hi / lo at +32 / +48 KB
#pragma unroll
                            for (int kk = 0; kk < 2; ++kk) {
                                const uint64_t bh = desc_add(dB, so + kk * 8192);
                                const uint64_t bl = desc_add(dB, so + 16384 + kk * 8192);
                                const bool accum = ks > 0 || kk > 0;
                                const uint32_t ao = so + kk * 256;
                                mma_bf16(tmem, desc_add(dA, ao + 8192), bh, idesc, accum);
                                mma_bf16(tmem, desc_add(dA, ao), bl, idesc, true);
                                mma_bf16(tmem, desc_add(dA, ao), bh, idesc, true);
                                mma_bf16(tmem + 256, desc_add(dA, ao + 24576), bh, idesc, accum);
                                mma_bf16(tmem + 256, desc_add(dA, ao + 16384), bl, idesc, true);
                                mma_bf16(tmem + 256, desc_add(dA, ao + 16384), bh, idesc, true);
                            }
                        }
                        mma_commit(&bars.empty[s]);
                    }
                    if (*abort_flag) break;
                    mma_commit(&bars.acc_full);
                }
            }
            // all MMAs issued by this thread complete before the TMEM is freed
            mma_commit(&bars.drain);
            if (!mbar_wait(&bars.drain, 0, kWaitLimit, nullptr)) raise_timeout(args.status, abort_flag);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- TMA producer: K tiles (the same sequence for every row tile) ----------------
        if (lane == 0) {
            constexpr int T = BF ? 8 : 4;                 // u per 16-byte core row
            const uint32_t bytes = BF ? 2 * 16384 : 32768;
            int it = 0;
            for (int un = ub; un < ue && !*abort_flag; ++un) {
                const int vc = un % nvc;
                {
                    for (int ks = 0; ks < nks; ++ks, ++it) {
                        if (*abort_flag) break;
                        const int s = it % E_STAGES;
                        if (it >= E_STAGES &&
                            !mbar_wait(&bars.empty[s], ((it / E_STAGES) - 1) & 1, kWaitLimit, abort_flag)) {
                            raise_timeout(args.status, abort_flag);
                            break;
                        }
                        unsigned char *sb = smem + s * E_STAGE_BYTES + 32768;
                        // stage start in 1 KB rows: ((vc*(Mxe/T) + ks*(32/T)) * 4 KB) / 1 KB
                        const int row = 4 * (vc * (args.Mxe / T) + ks * (E_KS / T));
                        mbar_arrive_expect_tx(&bars.kfull[s], bytes);
                        tma_load_2d(sb, &tm_hi, 0, row, &bars.kfull[s]);
                        if (BF) tma_load_2d(sb + 16384, &tm_lo, 0, row, &bars.kfull[s]);
                    }
                }
            }
            wait_copies_landed(bars.kfull, E_STAGES, (uint32_t)it);
        }
        __syncwarp();
    } else if (warp < 2 + E_EPI_WARPS) {
        // ---------------- epilogue: row dots with Yt, Yh ----------------
        // A warp reads TMEM lanes 32 * (warp % 4) .. + 31: its rows; two warps per
        // lane quarter take 128 columns each.  Every epilogue thread runs the same
        // tile sequence and meets named barrier 1 once per tile, also after an
        // abort (the work is then skipped).
        const int row = (warp & 3) * 32 + lane;
        const int cq = (warp - 2) >> 2;
        const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        int pc = 0, seg = 0, v0 = 0;
        bool valid = false;
        YRec Ry{};
        float eN = 0.f, eX = 0.f, eY = 0.f;
        for (int un = ub; un < ue; ++un, ++pc) {
            const int tile = un / nvc, vc = un % nvc;
            if (un == ub || vc == 0) {           // a new tile segment
                const int b = tile * E_ROWS + row;
                valid = b < args.n;
                if (valid) Ry = load_yrec(args.yr, b);
                eN = eX = eY = 0.f;
                v0 = vc;
            }
            drain_pass<PREC, SAMPLE>(bars, abort_flag, args.status, trow, cq * E_DRAIN_COLS,
                               vc * E_VC + cq * E_DRAIN_COLS, pc, valid, Ry, eN, eX, eY);
            if (vc == nvc - 1 || un == ue - 1)
                finish_segment(bars, abort_flag, args, seg++, tile, v0, vc, nvc, row, cq, eN, eX, eY);
        }
    } else {
        // ---------------- basis generators: Xt, Xh ----------------
        // group grp fills the CTA's stages it = grp, grp + 2, ..., so every stage is
        // filled by exactly one group
        const int g = threadIdx.x - 32 * (2 + E_EPI_WARPS);   // 0..255
        const int row = g & 127, grp = g >> 7;
        bool valid = false;
        AxisRec Rx;
        for (int un = ub; un < ue && !*abort_flag; ++un) {
            const int tile = un / nvc, vc = un % nvc;
            if (un == ub || vc == 0) {
                const int b = tile * E_ROWS + row;
                valid = b < args.n;
                if (valid) Rx = args.xr[b];
            }
            const int base = (un - ub) * nks;
            for (int ks = (base + grp) & 1; ks < nks; ks += 2) {
                if (*abort_flag) break;
                const int it = base + ks;
                const int s = it % E_STAGES;
                if (it >= E_STAGES &&
                    !mbar_wait(&bars.empty[s], ((it / E_STAGES) - 1) & 1, kWaitLimit, abort_flag)) {
                    raise_timeout(args.status, abort_flag);
                    break;
                }
                gen_energy<PREC, SAMPLE>(smem + s * E_STAGE_BYTES, Rx, valid, row, ks * E_KS);
                fence_proxy_async_smem();
                mbar_arrive(&bars.full[s]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    }
    return fn;
}

// 2-D map over the tiled energy operand viewed as rows of 1 KB (256 x 32-bit
// words).  The finish kernel lays K out so that one pipeline stage (32 u x 256 v,
// in the K-major core-matrix order the MMA reads) is one contiguous run of
// 32 KB (TF32) or 16 KB (each bf16 half), so a stage is one box of 32 or 16 rows.
cudaError_t make_kmap(CUtensorMap *map, void *base, bool bf16, int Mxe, int Mye) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const size_t bytes = (size_t)Mxe * Mye * (bf16 ? 2 : 4);
    cuuint64_t dims[2] = {256, (cuuint64_t)(bytes / 1024)};
    cuuint64_t strides[1] = {1024};
    cuuint32_t box[2] = {256, (cuuint32_t)(bf16 ? 16 : 32)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

namespace {
__global__ void wait_probe_kernel(uint64_t limit_ns, unsigned *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    // phase 0 never completes: nothing arrives on the barrier
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0, limit_ns, nullptr)) atomicOr(status, 1u);
}
}  // namespace

namespace {
__global__ void phase_eval_kernel(const float *__restrict__ x, double invL, const int32_t *__restrict__ m,
                                  int64_t count, int evaluator, float2 *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long s = fixed_halfturns(x[i], invL);
        const unsigned long long mm = (unsigned long long)m[i];
        out[i] = evaluator == 0 ? phase_cs(mm, s) : evaluator == 1 ? gen::phase_poly(mm, s) : gen::phase_sfu(mm, s);
    }
}
}  // namespace

cudaError_t launch_phase_eval(const float *x, double invL, const int32_t *m, int64_t count,
                              int evaluator, float *out, cudaStream_t stream) {
    if (count == 0) return cudaSuccess;
    const int64_t want = (count + 255) / 256;
    const int grid = (int)(want < 4096 ? want : 4096);
    phase_eval_kernel<<<grid, 256, 0, stream>>>(x, invL, m, count, evaluator,
                                                reinterpret_cast<float2 *>(out));
    return cudaGetLastError();
}

cudaError_t launch_wait_probe(uint64_t limit_ns, unsigned *status, cudaStream_t stream) {
    wait_probe_kernel<<<1, 32, 0, stream>>>(limit_ns, status);
    return cudaGetLastError();
}

TcPlan tc_plan(int n, int Mx, int My) {
    TcPlan p{};
    // SM pairs (512 x 256 tiles) once the u extent fills one; else one CTA per 256 x 256 tile
    p.pair = round_up(Mx, C_TILE) >= P_TILE_U ? 1 : 0;
    p.Mxc = round_up(Mx, p.pair ? P_TILE_U : C_TILE);
    p.Myc = round_up(My, C_TILE);
    p.Mxe = round_up(Mx, E_KS);
    p.Mye = round_up(My, E_VC);
    const int tiles = (p.Mxc / (p.pair ? P_TILE_U : C_TILE)) * (p.Myc / C_TILE);
    const int slots = p.pair ? kPlanSMs / 2 : kPlanSMs;      // units in flight
    // Slice count s: the kernel takes ceil(tiles * s / slots) unit times of n / s
    // blocks each, so pick the s that minimises ceil(tiles * s / slots) / s (the
    // smallest such s: fewest partial tiles to sum), with slices of >= 512 blocks.
    int max_slices = (n + 511) / 512;
    if (max_slices > 4 * kPlanSMs) max_slices = 4 * kPlanSMs;
    if (max_slices < 1) max_slices = 1;
    int slices = 1;
    double best = 1e300;
    for (int sc = 1; sc <= max_slices; ++sc) {
        const double waves = (double)(((long long)tiles * sc + slots - 1) / slots);
        const double t = waves / sc;
        if (t < best * (1.0 - 1e-9)) {
            best = t;
            slices = sc;
        }
    }
    p.slice_len = round_up((n + slices - 1) / slices > 0 ? (n + slices - 1) / slices : 1, C_KB);
    p.slices = (n + p.slice_len - 1) / p.slice_len;
    if (p.slices < 1) p.slices = 1;
    p.tiles = tiles;
    return p;
}

// Pair kernel launch: clusters of two CTAs (one per SM), as many pairs as can be
// resident at once (at most one per unit), with programmatic dependent launch.
template <int PREC>
cudaError_t launch_coeff_pair(const Launch &L, const TcPlan &P, float *part) {
    PairArgs a{};
    a.xr = L.xrec;
    a.yr = L.yrec;
    a.n = L.n;
    a.tiles_v = P.Myc / P_TILE_V;
    a.slices = P.slices;
    a.slice_len = P.slice_len;
    a.units = P.tiles * P.slices;
    a.Mxc = P.Mxc;
    a.Myc = P.Myc;
    a.part = part;
    a.status = L.status;
    auto kfn = tc_coeff_pair_kernel<PREC>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, P_SMEM);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.blockDim = dim3(C_THREADS);
    cfg.dynamicSmemBytes = P_SMEM;
    cfg.stream = L.stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int pairs = L.sm_count / 2;
    cfg.gridDim = dim3(2 * pairs);
    int active = 0;
    if (cudaOccupancyMaxActiveClusters(&active, kfn, &cfg) == cudaSuccess && active > 0 && active < pairs)
        pairs = active;
    cudaGetLastError();
    if (pairs > a.units) pairs = a.units;
    if (pairs < 1) pairs = 1;
    cfg.gridDim = dim3(2 * pairs);
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kfn, a);
}

cudaError_t launch_coeff_tc(const Launch &L, int prec, const TcPlan &P, float *part) {
    if (L.n == 0) return cudaSuccess;
    if (P.pair) return prec == 1 ? launch_coeff_pair<1>(L, P, part) : launch_coeff_pair<2>(L, P, part);
    CoeffArgs a{};
    a.xr = L.xrec;
    a.yr = L.yrec;
    a.n = L.n;
    a.tiles_v = P.Myc / C_TILE;
    a.slices = P.slices;
    a.slice_len = P.slice_len;
    a.units = P.tiles * P.slices;
    a.Mxc = P.Mxc;
    a.Myc = P.Myc;
    a.part = part;
    a.status = L.status;
    const int grid = a.units < L.sm_count ? a.units : L.sm_count;
    cudaError_t e;
    if (prec == 1) {
        e = cudaFuncSetAttribute(tc_coeff_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, C_SMEM);
        if (e != cudaSuccess) return e;
        e = launch_dependent(tc_coeff_kernel<1>, dim3(grid), dim3(C_THREADS), C_SMEM, L.stream, a);
        if (e != cudaSuccess) return e;
    } else {
        e = cudaFuncSetAttribute(tc_coeff_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, C_SMEM);
        if (e != cudaSuccess) return e;
        e = launch_dependent(tc_coeff_kernel<2>, dim3(grid), dim3(C_THREADS), C_SMEM, L.stream, a);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

__global__ void energy_from_coeffs_kernel(const float *__restrict__ a, int Mx, int My, double piW,
                                          double piH, double invWH, double *__restrict__ e_total) {
    double e = 0.0;
    const size_t total = (size_t)Mx * My;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int u = (int)(idx / My), v = (int)(idx % My);
        if (u == 0 && v == 0) continue;
        const double ku = u * piW, lv = v * piH;
        const double inv_G = (ku * ku + lv * lv) / ((u ? 2.0 : 1.0) * (v ? 2.0 : 1.0) * invWH);
        const double av = a[idx];
        e += 0.5 * av * av * inv_G;
    }
    cta_add_double(e, e_total);
}

cudaError_t launch_energy_from_coeffs(const float *a, int Mx, int My, double W, double H, double *e_total,
                                      cudaStream_t stream) {
    const size_t total = (size_t)Mx * My;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    const double PI = 3.141592653589793;
    energy_from_coeffs_kernel<<<blocks, 256, 0, stream>>>(a, Mx, My, PI / W, PI / H, 1.0 / (W * H), e_total);
    return cudaGetLastError();
}

cudaError_t launch_finish_tc(const Launch &L, int prec, const TcPlan &P, const float *part,
                             const float *a_in, float *a_out, void *Khi, void *Klo, double *e_total,
                             double *a64) {
    const size_t total = (size_t)P.Mxe * P.Mye;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 8 * L.sm_count) blocks = 8 * L.sm_count;
    if (blocks < 1) blocks = 1;
    const double PI = 3.141592653589793;
    const float piW = (float)(PI / L.W), piH = (float)(PI / L.H), invWH = (float)(1.0 / (L.W * L.H));
    auto kfn = prec == 1 ? tc_finish_kernel<1> : tc_finish_kernel<2>;
    return launch_dependent(kfn, dim3(blocks), dim3(256), 0, L.stream, part, P.slices, P.Mxc, P.Myc, a_in,
                            a_out, Khi, Klo, L.Mx, L.My, P.Mxe, P.Mye, piW, piH, invWH,
                            a_in ? nullptr : e_total, L.esplit_cnt, L.esplit_n, a_in ? nullptr : a64);
}

cudaError_t launch_energy_tc(const Launch &L, int prec, int sample, const TcPlan &P, void *Khi,
                             void *Klo, float *e_block, double *e_total, float *gx, float *gy,
                             const GradOut &go) {
    if (L.n == 0) return cudaSuccess;
    CUtensorMap mh, ml;
    const bool bf = prec == 2;
    cudaError_t e = make_kmap(&mh, Khi, bf, P.Mxe, P.Mye);
    if (e != cudaSuccess) return e;
    e = make_kmap(&ml, bf ? Klo : Khi, bf, P.Mxe, P.Mye);
    if (e != cudaSuccess) return e;
    EnergyArgs a{};
    a.xr = L.xrec;
    a.yr = L.yrec;
    a.n = L.n;
    a.Mx = L.Mx;
    a.My = L.My;
    a.Mxe = P.Mxe;
    a.Mye = P.Mye;
    a.e_block = e_block;
    a.gx = gx;
    a.gy = gy;
    a.e_total = e_total;
    a.go = go;
    a.status = L.status;
    a.tiles = (L.n + E_ROWS - 1) / E_ROWS;
    a.split = L.esplit;
    a.split_cnt = L.esplit_cnt;
    int grid = a.tiles < L.sm_count ? a.tiles : L.sm_count;           // persistent
    if (grid > kEnergyGridMax) grid = kEnergyGridMax;
    if (grid + 1 > L.esplit_n || !L.esplit || !L.esplit_cnt) return cudaErrorInvalidValue;
#define PP_ELAUNCH(PR, SA)                                                                         \
    do {                                                                                           \
        auto kfn = tc_energy_kernel<PR, SA>;                                                       \
        e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, E_SMEM);       \
        if (e != cudaSuccess) return e;                                                            \
        e = launch_dependent(kfn, dim3(grid), dim3(E_THREADS), E_SMEM, L.stream, mh, ml, a);       \
        if (e != cudaSuccess) return e;                                                            \
    } while (0)
    if (prec == 1 && sample == 0) PP_ELAUNCH(1, 0);
    else if (prec == 1) PP_ELAUNCH(1, 1);
    else if (sample == 0) PP_ELAUNCH(2, 0);
    else PP_ELAUNCH(2, 1);
#undef PP_ELAUNCH
    return cudaGetLastError();
}

}  // namespace pp
