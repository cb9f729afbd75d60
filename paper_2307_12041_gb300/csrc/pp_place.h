// Launchers of the placement loop's kernels (csrc/pp_place.cu), used by the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "pp.h"

namespace pp {

// pp_place.cu: the placement loop's kernels (log-sum-exp wirelength, gradient
// combination, Nesterov step, overflow)
// scal: NULL, or device {lambda, gamma, alpha0, coef} read by the kernels in place of the
// scalar arguments
cudaError_t launch_wirelength(int n_nets, int n_cells, const int32_t *net_ptr, const int32_t *net_pin,
                              const int32_t *cell_ptr, const int32_t *cell_net, const float *x,
                              const float *y, float gamma, const float *scal, float *stats, float *gx,
                              float *gy, double *out, int sm_count, cudaStream_t st);
// (launch_wirelength with gx == NULL runs the per-net pass only.)  The one-call
// iteration's cell pass: g = combination of the per-cell wirelength gradient with gn,
// written to gx, gy, and norms = {|v - vp|^2, |g - gp|^2} (zeroed here)
cudaError_t launch_cell_step(int n_cells, const int32_t *cell_ptr, const int32_t *cell_net, const float *x,
                             const float *y, float gamma, float lambda, const float *scal, const float *stats,
                             const float *gnx, const float *gny, const float *q, const uint8_t *movable,
                             const float *vpx, const float *vpy, const float *gpx, const float *gpy, float *gx,
                             float *gy, double *norms, int sm_count, cudaStream_t st);
cudaError_t launch_combine(int64_t n, const float *gwx, const float *gwy, const float *gnx, const float *gny,
                           const int32_t *cell_ptr, const float *q, const uint8_t *movable, float lambda,
                           const float *scal, float *gx, float *gy, cudaStream_t st);
cudaError_t launch_nesterov(int64_t n, float *ux, float *uy, float *vx, float *vy, float *vpx, float *vpy,
                            const float *gx, const float *gy, float *gpx, float *gpy, const float *w,
                            const float *h, float W, float H, const uint8_t *movable, const double *norms,
                            float alpha0, float coef, const float *scal, cudaStream_t st);
cudaError_t launch_step_norms(int64_t n, const float *vx, const float *vy, const float *vpx, const float *vpy,
                              const float *gx, const float *gy, const float *gpx, const float *gpy,
                              double *norms, int sm_count, cudaStream_t st);
cudaError_t launch_overflow(int m, const float *P, float target, double *out, int sm_count, cudaStream_t st);
// the loop's scalar update when the loop runs on the device (pp_place_run): the begin
// kernel sets the first scalars and the WHILE condition, the step kernel runs after
// each iteration (record, updates, stop test, next scalars, condition)
cudaError_t launch_place_loop_begin(pp_place_state *st, int32_t max_iters, cudaGraphConditionalHandle cond,
                                    cudaStream_t s);
cudaError_t launch_place_loop_step(const double *stats, pp_place_state *st, pp_place_record *trace,
                                   const pp_place_schedule &sc, const unsigned *status,
                                   cudaGraphConditionalHandle cond, cudaStream_t s);

}  // namespace pp
