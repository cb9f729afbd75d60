/*
 * pp.h -- C ABI of the GB300 library for the analytical solution of Poisson's
 * equation on a placement die (Zhu, Huang, Chen, Chang, arXiv 2307.12041).
 *
 * The die is R = [0, W] x [0, H] (Sec. II-A).  Block i has centre (x_i, y_i),
 * width w_i, height h_i and charge density c_i (unit density when c is NULL,
 * the paper's theta_i = 1 of Eq. (global density)).  With mode counts Mx, My the
 * library evaluates the truncated series of Sec. III (u = 0..Mx-1, p = 0..My-1):
 *
 *   coefficients  a_{u,p}       Eq. (a-a), (aup), (au0), (a0p)
 *   potential     psi           Eq. (psi)
 *   field         xi = -grad psi  Eq. (ksi)
 *   energy        N(v) = 1/2 sum_i N_i   (Sec. II-B)
 *   gradient      dN/d(x_i, y_i) = -(block charge) * xi   (Sec. IV, grad N = -q xi)
 *
 * Two readings of the per-block energy are offered (pp_sample):
 *   PP_RECT   N_i = c_i * (integral of psi over block i).  E = 1/2 sum N_i is then
 *             the electrostatic energy of the exact rectangle density, and the
 *             gradient is its exact derivative (minus the block-integrated field).
 *   PP_CENTER N_i = q_i psi(x_i, y_i), q_i = c_i w_i h_i, and the gradient is
 *             -q_i xi(x_i, y_i): the centre substitution of Sec. III-C.
 *
 * Conventions shared by every call
 *  - All array arguments are DEVICE pointers owned by the caller; the library
 *    allocates no device memory.  Scratch space is the caller's workspace `ws`
 *    (at least pp_workspace_size() bytes, 256-byte aligned).
 *  - Inputs x, y, w, h (and c if not NULL) are float32 arrays of n elements.
 *  - The coefficient matrix `a` is float32, Mx x My, row-major with u (the x
 *    mode) as the row index: a[u * My + p].
 *  - Calls are asynchronous on `stream` (a cudaStream_t, NULL = legacy default
 *    stream); the outputs are valid once the stream reaches the call.  Calls
 *    that share a workspace must be ordered on one stream.
 *  - The return status covers argument checks and launch errors.  Errors the
 *    GPU detects while running (a bounded wait that ran out) are recorded in a
 *    per-device status word that pp_sync_status() reads and clears.
 *  - e_total in the rectangle reading is E = 1/2 sum_i N_i.  On the tensor-core
 *    paths with a == NULL it is evaluated as the equal sum 1/2 sum_uv a_uv S_uv
 *    from the FP32 coefficients (their accuracy, not that of the TF32 / bf16 K
 *    operand shared by all blocks); with a given it is the sum of the N_i.
 *  - n = 0 is valid: outputs are zero (a all zero, *e_total = 0).
 *  - Limits: 1 <= Mx, My <= 4096; 0 <= n <= 2^31 - 1; 1e-300 <= W, H <= 1e300.
 *  - pp_last_error() describes the last non-OK status of the calling thread.
 */
#ifndef PP_H
#define PP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PP_OK = 0,
    PP_EINVAL = 1,      /* bad argument: see pp_last_error() */
    PP_ENOMEM_WS = 2,   /* workspace missing or smaller than pp_workspace_size() */
    PP_ECUDA = 3,       /* a CUDA runtime/driver call failed */
    PP_ETIMEOUT = 4,    /* a device-side bounded wait ran out (pp_sync_status) */
    PP_ENOTSUP = 5      /* precision not available on this device */
} pp_status;

/* Arithmetic of the three contractions (coefficients, X.K, X'.K):
 *  PP_FP32    CUDA-core FP32 FMA, FP64 cross-block accumulation of the coefficients.
 *  PP_TF32    tcgen05 tensor cores, TF32 operands, FP32 accumulation in TMEM.
 *  PP_BF16X3  tcgen05 tensor cores, operands split into bf16 hi + lo and
 *             multiplied as hi*hi + hi*lo + lo*hi, FP32 accumulation in TMEM.
 * In every precision the phase u*x/W is reduced modulo 2 in 64-bit fixed point
 * and the total energy is summed in FP64. */
typedef enum { PP_FP32 = 0, PP_TF32 = 1, PP_BF16X3 = 2 } pp_precision;

typedef enum { PP_RECT = 0, PP_CENTER = 1 } pp_sample;

typedef struct {
    double W, H;               /* die size (Sec. II-A) */
    int64_t n;                 /* number of blocks */
    const float *x, *y;        /* block centres, device, n each */
    const float *w, *h;        /* block widths/heights, device, n each */
    const float *c;            /* charge densities, device, n; NULL = 1 */
    int32_t Mx, My;            /* modes kept: u < Mx, p < My (Sec. III-B truncation) */
} pp_problem;

/* Bytes of workspace the calls below need for this problem and precision
 * (0 if the problem is invalid; pp_last_error() then says why). */
size_t pp_workspace_size(const pp_problem *prob, pp_precision prec);

/* Coefficient matrix of the truncated series: Eq. (a-a) a_00 = 0, Eq. (aup)
 * for u, p >= 1, Eq. (au0) for p = 0, Eq. (a0p) for u = 0, with the block sums
 * weighted by c_i.  Written to `a` (device, Mx*My float32, u-major). */
pp_status pp_coeffs(const pp_problem *prob, pp_precision prec, float *a,
                    void *ws, size_t ws_bytes, void *stream);

/* Per-block energy N_i (Sec. II-B, reading per `sample`) and total energy
 * E = 1/2 sum_i N_i.  `a` = coefficients from pp_coeffs, or NULL to compute
 * them inside this call.  e_block (device, n float32) and e_total (device,
 * one double, accumulated in FP64) may each be NULL; not both. */
pp_status pp_energy(const pp_problem *prob, pp_precision prec, pp_sample sample,
                    const float *a, float *e_block, double *e_total,
                    void *ws, size_t ws_bytes, void *stream);

/* Gradient of E = 1/2 sum_i N_i with respect to the block centres,
 * gx[i] = dE/dx_i, gy[i] = dE/dy_i (device, n float32 each; PP_RECT: exact
 * derivative, = -c_i * integral over block i of xi from Eq. (ksi); PP_CENTER:
 * -q_i xi(x_i, y_i)).  Optionally also N_i and E as in pp_energy (NULL to skip).
 * `a` = coefficients, or NULL to compute them inside this call.  With a = NULL
 * this single call is one full energy + gradient evaluation: three
 * contractions of N x Mx x My. */
pp_status pp_grad(const pp_problem *prob, pp_precision prec, pp_sample sample,
                  const float *a, float *gx, float *gy, float *e_block, double *e_total,
                  void *ws, size_t ws_bytes, void *stream);

/* pp_grad (a = NULL) for a placement held in HOST memory, results written to
 * HOST memory: the evaluation of Sec. III-C (Eq. aup, ksi) as pp_grad computes it,
 * with the transfers inside the call.
 *  - prob->x, y, w, h, c (c may be NULL) and gx, gy (required when n > 0),
 *    e_block (n float32, may be NULL), e_total (one double, may be NULL) are host
 *    pointers; device pointers of the current device are accepted as well.
 *  - Pinned (page-locked) host memory is read and written in place by the
 *    kernels, through its device mapping (each input read once, each output
 *    written once); pageable memory is copied through the workspace with
 *    cudaMemcpyAsync.  E is copied out at the end.  The caller owns every buffer
 *    and keeps it valid until `stream` has passed the call.
 *  - Workspace: pp_grad_host_workspace_size(prob, prec) bytes (pp_workspace_size,
 *    then 256 B for E and 8 staging arrays of n float32).
 *  - Errors as pp_grad (PP_EINVAL, PP_ENOMEM_WS, PP_ENOTSUP, PP_ECUDA); the
 *    outputs are defined only after synchronizing `stream`. */
size_t pp_grad_host_workspace_size(const pp_problem *prob, pp_precision prec);
pp_status pp_grad_host(const pp_problem *prob, pp_precision prec, pp_sample sample,
                       float *gx, float *gy, float *e_block, double *e_total,
                       void *ws, size_t ws_bytes, void *stream);

/* Adjoint of the energies for an upstream gradient (the backward pass of
 *   L = g_total * E + sum_i g_block_i N_i,   E = 1/2 sum_i N_i   (Sec. II-B)
 * with respect to the block centres).  N_i = sum_uv X_iu a_uv Y_iv depends on x_j
 * through block j's own basis and through the coefficients a (Eq. aup sums over
 * all blocks), so with w_i = g_total / 2 + g_block_i:
 *   dL/dx_j = w_j h_j + h^b_j,
 * where h = the gradient pp_grad returns (coefficients a of the charges c_i) and
 * h^b the same with the coefficients b of the charges c_i w_i (likewise for y).
 *  - g_total: device, one double (dL/dE), or NULL = 0.  g_block: device, n float32
 *    (dL/dN_i), or NULL = 0.  Not both NULL.
 *  - g_block == NULL: one evaluation (three contractions), gx = g_total * dE/dx in
 *    either reading (PP_CENTER: the centre-sample gradient of pp_grad scaled).
 *    g_block != NULL: PP_RECT only; two evaluations (the coefficients of both
 *    charge sets, two energy passes).
 *  - movable: device uint8 of n, or NULL: blocks with movable[i] == 0 get 0.
 *  - gx, gy: device float32 n (required when n > 0); e_block, e_total: optional,
 *    N_i and E of the placement as in pp_grad.
 *  - Workspace as pp_grad (pp_workspace_size).  PP_EINVAL as pp_grad, plus a
 *    NULL g_total and g_block, g_block with PP_CENTER, a misaligned g_total or
 *    host pointers.  Asynchronous on `stream`. */
pp_status pp_grad_adjoint(const pp_problem *prob, pp_precision prec, pp_sample sample,
                          const double *g_total, const float *g_block, const uint8_t *movable,
                          float *gx, float *gy, float *e_block, double *e_total,
                          void *ws, size_t ws_bytes, void *stream);

/* Coefficients summed over calls in FP64: a64 += a(these blocks), Eq. (aup),
 * (au0), (a0p) being sums over blocks (Eq. a-a..a-d).  For a placement cut into
 * chunks of blocks (to bound the workspace) or shared out over processes (each
 * adding its blocks, then a sum of a64 over processes), the total is a64 after
 * every part has been added.  a64: device double Mx x My (u-major), zeroed by the
 * caller before the first part.  a_out (optional): device float32 Mx x My
 * receiving the rounded running sum (float)a64 after this call; with n = 0 the
 * call adds nothing and only writes a_out.  Each part's a is formed in the
 * precision `prec` and added in FP64.  Workspace as pp_coeffs.  Asynchronous on
 * `stream`; calls that share a64 must be ordered. */
pp_status pp_coeffs_accumulate(const pp_problem *prob, pp_precision prec, double *a64, float *a_out,
                               void *ws, size_t ws_bytes, void *stream);

/* Allocation-free energy + gradient.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory where they
 * evaluate the energy (a host that fixes its device budget at start-up, a
 * plugin whose host tool owns every allocation, code inside a region where an
 * allocator call would break the caller's own memory bookkeeping).  It computes
 * the same outputs as pp_grad(prob, PP_FP32, sample, NULL, ...) -- one full
 * evaluation with the coefficients computed inside the call -- but takes no
 * workspace: its scratch is a static device array of PP_STATIC_SCRATCH_BYTES
 * inside the library, held on each GPU that uses it until the process exits.
 * The caller passes the inputs and outputs as for pp_grad (gx, gy required when
 * n > 0; e_block, e_total optional).
 *  - Limits: n <= PP_STATIC_MAX_BLOCKS, Mx, My <= PP_STATIC_MAX_MODES; larger
 *    problems are rejected with PP_EINVAL (use pp_grad with a workspace).
 *  - It allocates nothing: no cudaMalloc/cudaFree or allocating library call.
 *  - The first call on a device looks up the array's device address (set-up,
 *    once per device, with that device current); make that first call before
 *    any stream capture.  Under the CUDA runtime's default lazy module loading
 *    the array is reserved on a device by that first call (when the module that
 *    holds it is loaded), not when the library is loaded: a caller that fixes
 *    its device budget at start-up makes one call there first (n = 0 does only
 *    the set-up and zeroes *e_total).
 *  - The die size is checked as in pp_grad (W, H in [1e-300, 1e300]).
 *  - All calls share the one array and it keeps the previous call's contents;
 *    what must start at zero is cleared on `stream` by each call.  Calls whose
 *    kernels overlap on the GPU (unordered streams) race on the array. */
#define PP_STATIC_MAX_BLOCKS 32768
#define PP_STATIC_MAX_MODES 256
#define PP_STATIC_SCRATCH_BYTES 4980736
pp_status pp_grad_noalloc(const pp_problem *prob, pp_sample sample, float *gx, float *gy,
                          float *e_block, double *e_total, void *stream);

/* Waits for `stream`, then reads and clears the current device's status word:
 * PP_OK, or PP_ETIMEOUT if a kernel gave up a bounded wait since the last check. */
pp_status pp_sync_status(void *stream);

/* Phase step of the basis generators (the cos/sin factors of Eq. aup), exposed
 * for testing.  For i < count: s = x[i] * (1/L) (the float32 x times the double
 * 1/L, exact product) reduced to [0, 2) and rounded to 64-bit fixed point
 * (2^-62 half-turn units), exactly as the per-block records hold it;
 * then out[2i], out[2i+1] = cos, sin of pi * (m[i] * s mod 2), evaluated by
 * `evaluator` 0 (the records' and CUDA-core kernels' evaluator: sincospif of the
 * top 24 phase bits plus a first-order residual rotation), 1 (the BF16x3
 * generators' anchor: quarter-turn reduction and Taylor polynomials) or 2 (the
 * TF32 generators' anchor: the hardware sine and cosine of the reduced phase).
 * x (float32), m (int32, >= 0) and out (float32, 2 * count) are device arrays.
 * PP_EINVAL for L outside [1e-300, 1e300], count < 0, NULL or host pointers, or an
 * unknown evaluator; asynchronous on `stream`. */
pp_status pp_phase_eval(const float *x, double L, const int32_t *m, int64_t count, int evaluator,
                        float *out, void *stream);

/* The paper's binned fast scheme (Sec. III-D) on m x m uniform bins, for the same
 * problem description (Mx, My <= m modes, i.e. K <= m - 1):
 *   P_lj  = sum_i c_i area(block i ∩ bin lj) / area(bin)           (bin density)
 *   a     = Eq. (disa-a..d) from the cosine transform of P           (coefficients)
 *   psi, xi at the bin centres, Eq. (dis-psi1) and (dis-ksi)
 *   N_i   = q_i psi(x_i, y_i), gradient of E = 1/2 sum N_i = -q_i xi(x_i, y_i), with
 *           q_i = c_i w_i h_i and the bin-centre values weighted bilinearly at the
 *           block centre (clamped to the outermost centres).
 * The paper leaves its local-smoothness weighting of the density and its weighting
 * of the surrounding bins unstated; these are the readings taken.  The transforms
 * run along one grid axis at a time as FP32 FFTs (m a power of two; direct sums
 * otherwise) in both precisions; prec selects how the density is summed:
 * PP_FP32 exactly, in 64-bit fixed point (each addition rounded to 2^-32 bin
 * areas; the results are the same from run to run; |P| < 2^31 bin areas),
 * PP_TF32 with FP32 atomics (faster; the rounding of the sums, and so the last
 * bits of the results, follows the order the atomics land in).  PP_BF16X3 gives
 * PP_ENOTSUP.  a_out (Mx x My, optional), gx, gy (required when n > 0), e_block,
 * e_total (optional): device arrays.  2 <= m <= 4096.  Workspace: at least
 * pp_binned_workspace_size() bytes, 256-byte aligned; 0 for invalid arguments. */
size_t pp_binned_workspace_size(const pp_problem *prob, int32_t m);
pp_status pp_binned_grad(const pp_problem *prob, pp_precision prec, int32_t m, float *a_out, float *gx,
                         float *gy, float *e_block, double *e_total, void *ws, size_t ws_bytes,
                         void *stream);

/* Total energy from coefficients: *e_total = 1/2 sum_{(u,v) != (0,0)} a_uv^2 / G_uv
 * with G_uv = e_u e_v / (W H (k_u^2 + l_v^2)) (FP64 sum), i.e. 1/2 sum_uv a_uv S_uv
 * (Eq. a-a..a-d: S = a / G) = 1/2 sum_i N_i in the rectangle reading, for the
 * placement whose coefficients a are (for instance a = sum of pp_coeffs over
 * chunks of its blocks).  a: device float32 Mx x My, u-major; e_total: device
 * double.  PP_EINVAL for bad sizes or pointers.  Asynchronous on `stream`. */
pp_status pp_energy_from_coeffs(const float *a, int32_t Mx, int32_t My, double W, double H,
                                double *e_total, void *stream);

/* One position update of the descent loop (a driver around the evaluation; the
 * Nesterov loop of Sec. IV is pp_nesterov_step and its companions below).
 * For every block i with movable == NULL or movable[i] != 0:
 *   x_i <- clamp(x_i - lr * gx_i + sigma * n0_i, w_i / 2, W - w_i / 2)
 *   y_i <- clamp(y_i - lr * gy_i + sigma * n1_i, h_i / 2, H - h_i / 2)
 * where (n0_i, n1_i) are standard normals by Box-Muller from the Philox4x32-10
 * output (Salmon et al., SC 2011) for counter (i, step, 0, 0) and key (seed mod
 * 2^32, seed >> 32): u0 = (out0 + 1/2) 2^-32, u1 = (out1 + 1/2) 2^-32,
 * r = sqrt(-2 ln u0), n0 = r cos(2 pi u1), n1 = r sin(2 pi u1).
 * x, y (updated in place), w, h, gx, gy: float32 device arrays of n; movable:
 * uint8 device array of n or NULL.  PP_EINVAL for a die size outside
 * [1e-300, 1e300], n < 0, lr or sigma not finite, or a missing / host pointer
 * when n > 0.  Asynchronous on `stream`. */
pp_status pp_descent_step(double W, double H, int64_t n, float *x, float *y, const float *w,
                          const float *h, const float *gx, const float *gy, const uint8_t *movable,
                          float lr, float sigma, uint64_t seed, uint64_t step, void *stream);

/* ---- placement loop (Sec. IV: min f = W_LSE + lambda N, one Nesterov step per
 * iteration, a penalty update and an overflow stop, "as in ePlace"; the host
 * orchestrates, these entry points do the per-iteration work on the device) ---- */

/* A netlist in both orientations (device int32 arrays): net e's pins are the cells
 * net_pin[net_ptr[e] .. net_ptr[e+1]); cell i's nets are cell_net[cell_ptr[i] ..
 * cell_ptr[i+1]).  Pins sit at the cell centres.  The kernels index with these
 * arrays unchecked: every pin must lie in [0, n_cells), every net in [0, n_nets),
 * and the pointer arrays must be non-decreasing from 0 (the Python binding checks
 * this when it builds the netlist). */
typedef struct {
    int32_t n_cells, n_nets;
    const int32_t *net_ptr, *net_pin;
    const int32_t *cell_ptr, *cell_net;
} pp_netlist;

/* Bytes of workspace pp_wirelength needs: 32 per net (per-net maxima, minima and
 * the reciprocals of the shifted exponential sums), rounded up to 256. */
size_t pp_wirelength_workspace_size(int32_t n_nets);

/* Log-sum-exp wirelength (Sec. IV's W_LSE, the smooth HPWL model of ePlace):
 *   W = sum_e sum_{axis} gamma [ln sum_{i in e} e^{x_i/gamma} + ln sum_{i in e} e^{-x_i/gamma}]
 * over nets of two or more pins, each sum shifted by the net's max (min) so that no
 * exponential overflows; gx, gy (float32, n_cells) receive dW/dx, dW/dy, gathered
 * per cell from its nets (no atomics); out (device, 2 doubles) receives
 * {W, HPWL}.  x, y: float32 device arrays of n_cells.  PP_EINVAL for gamma not
 * finite or <= 0, a NULL or host pointer; PP_ENOMEM_WS for a short workspace
 * (256-byte aligned device memory).  Asynchronous on `stream`. */
pp_status pp_wirelength(const pp_netlist *netlist, const float *x, const float *y, float gamma, float *gx,
                        float *gy, double *out, void *ws, size_t ws_bytes, void *stream);

/* Objective gradient with ePlace's diagonal preconditioner:
 *   g_i = (gw_i + lambda gn_i) / max(1, deg_i + lambda q_i)
 * with deg_i = cell_ptr[i+1] - cell_ptr[i] (0 if cell_ptr is NULL) and q_i the
 * block's charge (c w h); g_i = 0 where movable[i] == 0.  float32 device arrays of
 * n; movable uint8 or NULL.  PP_EINVAL for lambda not finite or < 0 or a bad
 * pointer.  Asynchronous on `stream`. */
pp_status pp_place_combine(int64_t n, const float *gwx, const float *gwy, const float *gnx, const float *gny,
                           const int32_t *cell_ptr, const float *q, const uint8_t *movable, float lambda,
                           float *gx, float *gy, void *stream);

/* norms[0] = sum_i |v_i - vp_i|^2, norms[1] = sum_i |g_i - gp_i|^2 (both axes, FP64),
 * the quantities of the Nesterov step length.  norms: device, 2 doubles (zeroed
 * here).  Asynchronous on `stream`. */
pp_status pp_step_norms(int64_t n, const float *vx, const float *vy, const float *vpx, const float *vpy,
                        const float *gx, const float *gy, const float *gpx, const float *gpy, double *norms,
                        void *stream);

/* One Nesterov step of every movable block (in place):
 *   alpha = sqrt(norms[0] / norms[1]) when norms != NULL and both are > 0, else alpha0;
 *   vp <- v, gp <- g;
 *   u' = clamp(v - alpha g), v' = clamp(u' + coef (u' - u)),  u <- u', v <- v',
 * clamp keeping the block inside the die (x in [w/2, W - w/2], likewise y), and
 * coef = (a_k - 1) / a_{k+1} with a_{k+1} = (1 + sqrt(4 a_k^2 + 1)) / 2 from the
 * caller.  Blocks with movable[i] == 0 keep u and v.  All arrays float32 device of
 * n; movable uint8 or NULL; norms device (2 doubles) or NULL.  PP_EINVAL for a bad
 * die size, alpha0 < 0, non-finite scalars or a bad pointer.  Asynchronous. */
pp_status pp_nesterov_step(int64_t n, double W, double H, float *ux, float *uy, float *vx, float *vy, float *vpx,
                           float *vpy, const float *gx, const float *gy, float *gpx, float *gpy, const float *w,
                           const float *h, const uint8_t *movable, const double *norms, float alpha0,
                           float coef, void *stream);

/* Density overflow on an m x m grid: bins (device float32, m*m, written here)
 * receives P_b = sum_i c_i area(block i ∩ b) / area(b) (exact overlap areas, block
 * edges in 2^-40-bin fixed point; c = NULL means 1), and *out (device double)
 * = sum_b max(P_b - target, 0), the excess in bin areas; the overflow ratio is
 * *out * area(bin) / (movable area).  PP_EINVAL for m outside [1, 8192], a bad die
 * size, target < 0 or a bad pointer.  Asynchronous on `stream`. */
pp_status pp_overflow(const pp_problem *prob, int32_t m, float target, float *bins, double *out, void *stream);

/* One iteration of the loop after the first, in one call: the work of the calls
 * below, made one after the other on `stream`, with their scratch carved from one
 * workspace.  Steps 2 (its per-cell part), 3 and 4 run as one kernel: g is what
 * the separate calls give, the norms differ only in the order of their sums.
 *   1. gn, E      density gradient and energy at v: the exact series on M x M modes
 *                 (pp_grad, PP_RECT) or the binned scheme of Sec. III-D on M x M
 *                 bins (pp_binned_grad; prec PP_FP32 or PP_TF32);
 *   2. gw, W, HPWL  pp_wirelength at v with smoothing gamma;
 *   3. g          pp_place_combine(gw, gn, lambda) with the netlist's cell degrees;
 *   4. norms      pp_step_norms(v, vp, g, gp);
 *   5.            pp_nesterov_step(alpha from the norms, else alpha0; coef), in place
 *                 on u, v, vp, gp;
 *   6.            pp_overflow of the new u over the first n_overflow blocks on M x M
 *                 bins with unit charge.
 * stats (device, 4 doubles) = {overflow excess (as pp_overflow's out), W_LSE, HPWL, E}.
 * The netlist's cells are the n blocks (fillers are cells without nets); every
 * block array is float32 device memory of n_cells, movable uint8 or NULL, c NULL
 * for unit charge.  ws: at least pp_place_workspace_size(args) bytes of 256-byte
 * aligned device memory.  Errors are those of the calls above, plus PP_EINVAL
 * for a NULL args or netlist, an unknown density or n_overflow outside [0, n].
 * Sizes and scalars are checked before any step is issued; each step checks its
 * own device pointers before its launches, so a bad pointer can stop the call
 * after earlier steps were issued (u and v change only in step 5).  With
 * `scalars` set, the work of one call depends on nothing but device memory, so
 * the call can be captured once in a CUDA graph and replayed every iteration
 * after the four scalars are written to the device. */
typedef enum { PP_DENSITY_EXACT = 0, PP_DENSITY_BINNED = 1 } pp_density;

typedef struct {
    const pp_netlist *netlist;
    double W, H;                        /* die */
    int32_t M;                          /* modes per axis (exact), bins per axis (binned, overflow) */
    int32_t density;                    /* pp_density */
    int32_t prec;                       /* pp_precision of the density term */
    int32_t reserved;                   /* 0 */
    int64_t n_overflow;                 /* blocks counted in the overflow: the first n_overflow */
    const float *w, *h, *c, *q;         /* sizes, charge density (or NULL), c w h */
    const uint8_t *movable;             /* or NULL: all movable */
    float *ux, *uy, *vx, *vy;           /* Nesterov solutions u and v (in place) */
    float *vpx, *vpy, *gpx, *gpy;       /* previous v and g (in place) */
    float lambda, gamma, alpha0, coef, target;
    double *stats;
    const float *scalars;               /* NULL, or device float[4] {lambda, gamma, alpha0, coef}
                                           read by the kernels as they run, in place of the
                                           fields above (16-byte aligned; not range-checked) */
} pp_place_iteration_args;

/* Workspace bytes of pp_place_iteration (0 for invalid sizes; pp_last_error()
 * says why).  Reads only the sizes in args and its netlist. */
size_t pp_place_workspace_size(const pp_place_iteration_args *args);
pp_status pp_place_iteration(const pp_place_iteration_args *args, void *ws, size_t ws_bytes, void *stream);

/* ---- the loop itself on the device ----
 * pp_place_run runs iterations 1, 2, ... of the loop (the first, whose lambda_0 and
 * step length need reductions over the whole placement, is the caller's) without
 * returning to the host between them: one CUDA graph whose conditional WHILE node
 * repeats { pp_place_iteration; the scalar update below } until a stop condition
 * holds.  The scalar update is the loop's host arithmetic made in FP64 by one device
 * thread, in this order, after iteration k:
 *   tau      = stats[0] * bin_area / area_mov           (the overflow ratio)
 *   record k = {k, tau, W_LSE, HPWL, E, lambda, gamma}    (the values it used)
 *   a_k      <- (1 + sqrt(4 a_k^2 + 1)) / 2
 *   lambda   <- lambda * clamp(1.1^(1 - (HPWL - hpwl_prev) / d_ref), 0.75, 1.1)
 *   hpwl_prev <- HPWL;  gamma <- 8 bin_w 10^((20/9)(tau - 0.1) - 1);  k <- k + 1
 * and the next iteration's float32 scalars {lambda, gamma, 0, (a_k - 1) / a_{k+1}}.
 * The loop stops (state.stop, below) once tau < tau_stop, k reaches max_iters, a
 * scalar is not finite (or lambda < 0, gamma <= 0 in float32), or the library's
 * device status word is set (a bounded wait gave up; pp_sync_status reports it).
 * Every body execution ends in the update, and the update stops the loop after at
 * most max_iters executions of one launch, so the graph always ends. */
typedef enum {
    PP_PLACE_RUNNING = 0,
    PP_PLACE_CONVERGED = 1,     /* tau < tau_stop */
    PP_PLACE_MAX_ITERS = 2,     /* k reached max_iters */
    PP_PLACE_NONFINITE = 3,     /* a scalar of the next iteration is not finite or out of range */
    PP_PLACE_DEVICE_ERROR = 4,  /* the device status word was set */
    PP_PLACE_BAD_STATE = 5      /* the state given to pp_place_run cannot start: k < 1, d_ref <= 0, ... */
} pp_place_stop;

typedef struct {
    int32_t max_iters;          /* iterations in all (the last record is k = max_iters - 1); [1, 2^24] */
    int32_t reserved;           /* 0 */
    double tau_stop;            /* stop once the overflow ratio drops below this */
    double bin_area;            /* area of one of the M x M bins */
    double area_mov;            /* area of the movable blocks counted in the overflow (> 0) */
    double bin_w;               /* bin width, the scale of gamma */
} pp_place_schedule;

/* The loop's state in device memory (80 bytes, 16-byte aligned).  The caller writes
 * it after iteration 0; pp_place_run reads and updates it in place. */
typedef struct {
    double lambda, gamma;       /* used by the next iteration */
    double a_k;                 /* Nesterov sequence before the next iteration (>= 1) */
    double hpwl_prev;           /* HPWL of the last iteration */
    double d_ref;               /* dHPWL_ref of the penalty update (> 0) */
    double tau;                 /* overflow ratio after the last iteration */
    int64_t k;                  /* index of the next iteration (>= 1) */
    int32_t stop;               /* pp_place_stop; the run starts only from PP_PLACE_RUNNING */
    int32_t run_count;          /* iterations made by the last pp_place_run */
    float scalars[4];           /* {lambda, gamma, alpha0 = 0, coef} the kernels read */
} pp_place_state;

/* One iteration's record (64 bytes); stop is the state's stop code after it. */
typedef struct {
    int64_t k;
    int32_t stop, reserved;
    double tau, w_lse, hpwl, e, lambda, gamma;
} pp_place_record;

/* Runs the loop from `state` (device) on `stream` as described above; record k is
 * written to trace[k] (device array of max_iters records; entries before the
 * state's k are not touched).  args and ws as for pp_place_iteration; the run's
 * own state->scalars replace args->scalars.  The graph is built, instantiated and
 * launched here and released after it has run; the call returns once it is
 * launched (asynchronous like the other entry points).  PP_EINVAL for a bad
 * schedule (max_iters outside [1, 2^24], a non-finite tau_stop, bin_area,
 * area_mov or bin_w <= 0), state or trace NULL, host or misaligned; PP_ECUDA
 * when the graph cannot be built (for instance, library timing enabled: event
 * records cannot sit in a conditional body); the errors of pp_place_iteration. */
pp_status pp_place_run(const pp_place_iteration_args *args, const pp_place_schedule *sched, pp_place_state *state,
                       pp_place_record *trace, void *ws, size_t ws_bytes, void *stream);

/* Failure-path check (no counterpart in the paper).  Launches, on `stream`, one
 * kernel whose thread waits on a shared-memory mbarrier that nothing completes,
 * through the same time-bounded wait the tensor-core kernels use between their
 * pipeline stages.  After `limit_ns` nanoseconds (clamped to [1e3, 5e9]) the wait
 * gives up and the kernel records the timeout in the device status word and
 * returns, as a stalled pipeline would; the next pp_sync_status() reports
 * PP_ETIMEOUT and the context stays usable.  Returns PP_ENOTSUP below compute
 * capability 9.0, PP_ECUDA if the launch fails. */
pp_status pp_check_wait_timeout(uint64_t limit_ns, void *stream);

/* Message for the calling thread's last non-OK status ("" if none). */
const char *pp_last_error(void);

/* Library build identification string (compile flags, arch). */
const char *pp_version(void);

/* Kernel counting and timing, a benchmarking aid with no counterpart in the
 * paper.  Every kernel launch of the evaluation entry points is counted per
 * kernel class (pp_kernel).  While timing is enabled, each launch is also
 * bracketed by two CUDA events recorded on the stream it is launched on (the
 * events cost device time between launches and keep a kernel from starting
 * before the previous one has ended, so time whole steps with timing off).
 * pp_timing_collect() waits for those events, then writes per kernel class the
 * number of launches and their summed device time in milliseconds (0 for
 * launches made with timing off) since the previous collect (arrays of
 * PP_K_COUNT entries, host memory), and resets both.  At most 65536 launches are
 * timed between collects; later ones are counted in `launches` but add no time.
 * Timing assumes one device per process. */
typedef enum {
    PP_K_PREP = 0,      /* per-block phases and scale factors */
    PP_K_COEFF = 1,     /* coefficient contraction  St = Xt^T Yt */
    PP_K_FINISH = 2,    /* a = G o S and the energy operand */
    PP_K_ENERGY = 3,    /* fused energy / gradient contractions and row dots */
    PP_K_COUNT = 4
} pp_kernel;
void pp_timing_enable(int on);
pp_status pp_timing_collect(int64_t *launches, double *ms);

#ifdef __cplusplus
}
#endif

#endif /* PP_H */
