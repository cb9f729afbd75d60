// Internal launch interface between the C ABI (pp_api.cu) and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace pp {

struct AxisRec;

// Everything a kernel launch needs about one evaluation.
struct Launch {
    double W, H;
    int n;
    int Mx, My;
    const float *x, *y, *w, *h, *c;
    AxisRec *xrec, *yrec;       // workspace: per-block records
    double *S64;                // workspace: Mx*My FP64 sums of the scaled basis
    void *K;                    // workspace: energy operand (layout per precision)
    int Kld;                    // leading dimension / padded size for K (per precision)
    unsigned *status;           // device status word
    float *esplit;              // tensor-core energy: split-tile scratch (see tc_energy_kernel)
    unsigned *esplit_cnt;       //   and its boundary counters (esplit_n of them)
    int esplit_n;
    int sm_count;
    cudaStream_t stream;
};

// What the energy kernels do with the gradient they form for block b (value v,
// either axis) before writing it: nothing (the default), or
//   v <- (w[b] + 0.5 wt[0]) * out[b] + v   when acc (out already holds a gradient;
//                                          w, wt may each be NULL = 0),
//   v <- v * scale[0]                      when scale != NULL (a device scalar),
//   v <- 0                                 when mask != NULL and mask[b] == 0.
// This is how the adjoint entry point combines its two energy passes.
struct GradOut {
    const float *w = nullptr;
    const double *wt = nullptr;
    const double *scale = nullptr;
    const uint8_t *mask = nullptr;
    bool acc = false;
};

// Per-block charge weights of the preparation kernel: the x records get charge
// c_i * (0.5 * gt[0] + gw[i]) instead of c_i (either pointer may be NULL = 0).
struct ChargeWeights {
    const float *gw = nullptr;
    const double *gt = nullptr;
    bool on = false;
};

// Padded sizes of the FP32 energy operand (u rows, v columns).
constexpr int kSimtKU = 32;     // u chunk of the FP32 energy kernel
constexpr int kSimtKV = 128;    // v tile of the FP32 energy kernel
inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Tensor-core path (pp_tc.cu).  Coefficient tiles are 256 x 256, or 512 x 256 on
// SM pairs when Mx exceeds 256 (padded extents Mxc, Myc); the energy operand is
// padded to (Mxe = 32k, Mye = 256k).  Blocks are
// cut into `slices` of slice_len for the persistent coefficient kernel; the plan
// depends only on the problem (kPlanSMs sets the target of two units per SM).
constexpr int kPlanSMs = 152;
// Energy kernel: row tiles of kEnergyRows blocks, at most kEnergyGridMax persistent
// CTAs; a tile cut between two CTAs meets in a scratch of kEnergyRows x 3 floats per
// side and boundary, with one counter per boundary.
constexpr int kEnergyRows = 128;
constexpr int kEnergyGridMax = 256;
inline int energy_boundaries(int n) {
    const int tiles = (n + kEnergyRows - 1) / kEnergyRows;
    return (tiles < kEnergyGridMax ? tiles : kEnergyGridMax) + 1;
}
struct TcPlan {
    int Mxc, Myc, Mxe, Mye, tiles, slices, slice_len;
    int pair;             // 1: the coefficient kernel runs on SM pairs (512 x 256 tiles)
};
TcPlan tc_plan(int n, int Mx, int My);
cudaError_t launch_coeff_tc(const Launch &L, int prec, const TcPlan &P, float *part);
// a64 (optional): FP64 running sum of coefficients, a64 += a; a_out then receives
// the rounded running sum instead of this call's a.  Khi == NULL: no operand.
cudaError_t launch_finish_tc(const Launch &L, int prec, const TcPlan &P, const float *part,
                             const float *a_in, float *a_out, void *Khi, void *Klo, double *e_total,
                             double *a64 = nullptr);
cudaError_t launch_energy_tc(const Launch &L, int prec, int sample, const TcPlan &P, void *Khi,
                             void *Klo, float *e_block, double *e_total, float *gx, float *gy,
                             const GradOut &go = GradOut());

// pp_api.cu: message returned by pp_last_error() for the calling thread
void set_last_error(const char *msg);
// Binned fast scheme (pp_binned.cu): workspace offsets (bytes) and the pipeline.
struct BinnedLayout {
    size_t P, D, R1t, R2, a, Ut, Upt, V, tab, total;
};
BinnedLayout binned_layout(int m, int Mx, int My);
// `what` names the failing step on error
cudaError_t run_binned(const Launch &L, int dev, int m, bool tf32, unsigned char *ws, float *a_out,
                       float *e_block, float *gx, float *gy, double *e_total, const char **what);
// P[l m + j] += sum_i c_i area(block i ∩ bin lj) / area(bin) on an m x m grid (P zeroed by the caller)
cudaError_t launch_bin_density(const float *x, const float *y, const float *w, const float *h, const float *c,
                               int n, int m, double W, double H, float *P, int sm_count, cudaStream_t st);
// E = 1/2 sum_uv a_uv^2 / G_uv (FP64) from coefficients a (Mx x My, u-major), added to *e_total
cudaError_t launch_energy_from_coeffs(const float *a, int Mx, int My, double W, double H, double *e_total,
                                      cudaStream_t stream);
cudaError_t launch_descent_step(float W, float H, int64_t n, float *x, float *y, const float *w,
                                const float *h, const float *gx, const float *gy,
                                const uint8_t *movable, float lr, float sigma, uint64_t seed,
                                uint64_t step, cudaStream_t stream);
cudaError_t launch_phase_eval(const float *x, double invL, const int32_t *m, int64_t count,
                              int evaluator, float *out, cudaStream_t stream);
// one CTA whose thread waits (bounded) on an mbarrier nothing completes
cudaError_t launch_wait_probe(uint64_t limit_ns, unsigned *status, cudaStream_t stream);

// pp_place.cu: the placement loop's launchers are declared in pp_place.h

// pp_simt.cu
cudaError_t launch_prep(const Launch &L, bool zero_S, double *e_total,
                        const ChargeWeights &cw = ChargeWeights());
cudaError_t launch_coeff_simt(const Launch &L);
// a64 as for launch_finish_tc; with_K = false skips the energy operand
cudaError_t launch_finish_simt(const Launch &L, const float *a_in, float *a_out, double *a64 = nullptr,
                               bool with_K = true);
cudaError_t launch_energy_simt(const Launch &L, int sample, float *e_block, double *e_total,
                               float *gx, float *gy, const GradOut &go = GradOut());
// a_out[i] = (float)a64[i], i < count (the rounded running sum alone)
cudaError_t launch_round_coeffs(const double *a64, float *a_out, size_t count, cudaStream_t stream);

}  // namespace pp
