// C ABI entry points (include/pp.h): argument checks, workspace layout and the
// launch sequence of one evaluation.
//
//   pp_coeffs : prep -> coefficient contraction -> finish(a)
//   pp_energy : prep -> [coefficients -> finish(K)] or finish(K from a) -> energy
//   pp_grad   : same as pp_energy, the energy kernel also writing dE/dx, dE/dy
//   pp_grad_host : pp_grad on host buffers (pinned: read and written in place by the
//                  kernels; pageable: staged through the workspace)
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pp.h"
#include "pp_device.cuh"
#include "pp_internal.h"
#include "pp_place.h"

namespace pp {

__device__ unsigned g_status;    // bit 0: a bounded wait ran out

namespace {

thread_local std::string t_err;

pp_status fail(pp_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return st;
}

pp_status cuda_fail(cudaError_t e, const char *what) {
    return fail(PP_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

constexpr int kMaxDev = 64;
std::mutex g_mu;
int g_sm[kMaxDev];
unsigned *g_status_ptr[kMaxDev];
int g_cc_major[kMaxDev];

// Per-device constants, looked up once with that device current.
pp_status device_info(int *dev, int *sm, unsigned **status, int *cc_major) {
    cudaError_t e = cudaGetDevice(dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (*dev < 0 || *dev >= kMaxDev) return fail(PP_EINVAL, "device index %d out of range", *dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_status_ptr[*dev]) {
        int v = 0;
        e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, *dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
        g_sm[*dev] = v;
        e = cudaDeviceGetAttribute(&v, cudaDevAttrComputeCapabilityMajor, *dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
        g_cc_major[*dev] = v;
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_status);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(status)");
        g_status_ptr[*dev] = (unsigned *)p;
    }
    *sm = g_sm[*dev];
    *status = g_status_ptr[*dev];
    *cc_major = g_cc_major[*dev];
    return PP_OK;
}

struct Layout {
    size_t xrec, yrec, S64, K, Klo, part, esplit, esplit_cnt, total;
    int esplit_n;
    int Kld;
    TcPlan plan;
};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Workspace regions (byte offsets, each 256-byte aligned):
//   PP_FP32:          x/y records, S64 [Mx*My] FP64, K FP32 [round_up(Mx,32)][round_up(My,128)]
//   PP_TF32/BF16X3:   x/y records, partial tiles [slices][Mxc][Myc] FP32,
//                     K in the TMA-tiled operand layout (TF32, or bf16 hi + lo),
//                     energy split-tile scratch and counters
Layout layout(const pp_problem *p, pp_precision prec) {
    Layout L{};
    const size_t n = (size_t)p->n;
    size_t off = 0;
    L.xrec = off;
    off = align256(off + n * sizeof(AxisRec));
    L.yrec = off;
    off = align256(off + n * sizeof(AxisRec));
    if (prec == PP_FP32) {
        L.S64 = off;
        off = align256(off + (size_t)p->Mx * p->My * sizeof(double));
        L.K = off;
        const int Mxp = round_up(p->Mx, kSimtKU);
        L.Kld = round_up(p->My, kSimtKV);
        off = align256(off + (size_t)Mxp * L.Kld * sizeof(float));
        L.Klo = L.part = 0;
    } else {
        L.plan = tc_plan((int)p->n, p->Mx, p->My);
        L.part = off;
        off = align256(off + (size_t)L.plan.slices * L.plan.Mxc * L.plan.Myc * sizeof(float));
        const size_t kel = (size_t)L.plan.Mxe * L.plan.Mye;
        L.K = off;
        off = align256(off + kel * (prec == PP_TF32 ? 4 : 2));
        L.Klo = off;
        if (prec == PP_BF16X3) off = align256(off + kel * 2);
        L.esplit_n = energy_boundaries((int)p->n);
        L.esplit = off;
        off = align256(off + (size_t)L.esplit_n * 2 * kEnergyRows * 3 * sizeof(float));
        L.esplit_cnt = off;
        off = align256(off + (size_t)L.esplit_n * sizeof(unsigned));
        L.S64 = 0;
        L.Kld = L.plan.Mye;
    }
    L.total = off;
    return L;
}

pp_status check_dev_ptr(const void *ptr, int dev, const char *name) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PP_EINVAL, "%s: not a CUDA pointer (%s)", name, cudaGetErrorName(e));
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(PP_EINVAL, "%s: must be device memory", name);
    if (at.device != dev)
        return fail(PP_EINVAL, "%s: lives on device %d, current device is %d", name, at.device, dev);
    return PP_OK;
}

// Shape checks only (no pointers): die, counts, precision.
pp_status check_shape(const pp_problem *p, pp_precision prec) {
    if (!p) return fail(PP_EINVAL, "problem is NULL");
    if (!std::isfinite(p->W) || !std::isfinite(p->H) || !(p->W >= 1e-300 && p->W <= 1e300) ||
        !(p->H >= 1e-300 && p->H <= 1e300))
        return fail(PP_EINVAL, "die size W=%g H=%g must be finite and in [1e-300, 1e300]", p->W, p->H);
    if (p->n < 0 || p->n > 2147483647LL)
        return fail(PP_EINVAL, "n=%lld out of range [0, 2^31-1]", (long long)p->n);
    if (p->Mx < 1 || p->My < 1 || p->Mx > 4096 || p->My > 4096)
        return fail(PP_EINVAL, "mode counts Mx=%d My=%d must be in [1, 4096]", p->Mx, p->My);
    if (prec != PP_FP32 && prec != PP_TF32 && prec != PP_BF16X3)
        return fail(PP_EINVAL, "unknown precision %d", (int)prec);
    return PP_OK;
}

pp_status check_problem(const pp_problem *p, pp_precision prec) {
    pp_status st = check_shape(p, prec);
    if (st != PP_OK) return st;
    if (p->n > 0 && (!p->x || !p->y || !p->w || !p->h))
        return fail(PP_EINVAL, "x, y, w, h must be non-NULL when n > 0");
    return PP_OK;
}

struct Ctx {
    Launch L;
    Layout lay;
    int dev;
    int cc_major;
    pp_precision prec;
    char *base;
};

// host_io: the block arrays were already resolved by pp_grad_host to pointers the
// kernels can use (device memory, or pinned host memory mapped for the device).
pp_status setup(const pp_problem *p, pp_precision prec, void *ws, size_t ws_bytes, void *stream,
                Ctx *ctx, bool host_io = false) {
    pp_status st = check_problem(p, prec);
    if (st != PP_OK) return st;
    int sm = 0;
    unsigned *status = nullptr;
    st = device_info(&ctx->dev, &sm, &status, &ctx->cc_major);
    if (st != PP_OK) return st;
    if (prec != PP_FP32 && ctx->cc_major != 10)
        return fail(PP_ENOTSUP, "tensor-core precisions need a compute capability 10.x GPU (this is %d.x)",
                    ctx->cc_major);
    ctx->prec = prec;
    ctx->lay = layout(p, prec);
    if (!ws || ws_bytes < ctx->lay.total)
        return fail(PP_ENOMEM_WS, "workspace of %zu bytes needed, %zu given%s", ctx->lay.total,
                    ws ? ws_bytes : (size_t)0, ws ? "" : " (NULL)");
    if (((uintptr_t)ws & 255) != 0) return fail(PP_EINVAL, "workspace must be 256-byte aligned");
    if ((st = check_dev_ptr(ws, ctx->dev, "ws")) != PP_OK) return st;
    if (p->n > 0) {
        const void *ptrs[5] = {p->x, p->y, p->w, p->h, p->c};
        const char *names[5] = {"x", "y", "w", "h", "c"};
        for (int i = 0; i < 5; ++i) {
            if (!ptrs[i]) continue;
            if (((uintptr_t)ptrs[i] & 3) != 0) return fail(PP_EINVAL, "%s is not 4-byte aligned", names[i]);
            if (!host_io && (st = check_dev_ptr(ptrs[i], ctx->dev, names[i])) != PP_OK) return st;
        }
    }
    Launch &L = ctx->L;
    char *base = (char *)ws;
    ctx->base = base;
    L.W = p->W;
    L.H = p->H;
    L.n = (int)p->n;
    L.Mx = p->Mx;
    L.My = p->My;
    L.x = p->x;
    L.y = p->y;
    L.w = p->w;
    L.h = p->h;
    L.c = p->c;
    L.xrec = (AxisRec *)(base + ctx->lay.xrec);
    L.yrec = (AxisRec *)(base + ctx->lay.yrec);
    L.S64 = prec == PP_FP32 ? (double *)(base + ctx->lay.S64) : nullptr;
    L.K = base + ctx->lay.K;
    L.Kld = ctx->lay.Kld;
    L.esplit = prec == PP_FP32 ? nullptr : (float *)(base + ctx->lay.esplit);
    L.esplit_cnt = prec == PP_FP32 ? nullptr : (unsigned *)(base + ctx->lay.esplit_cnt);
    L.esplit_n = prec == PP_FP32 ? 0 : ctx->lay.esplit_n;
    L.status = status;
    L.sm_count = sm;
    L.stream = (cudaStream_t)stream;
    return PP_OK;
}

pp_status out_ptr(const void *ptr, int dev, const char *name, bool required, bool host_io = false) {
    if (!ptr) return required ? fail(PP_EINVAL, "%s must be non-NULL", name) : PP_OK;
    if (((uintptr_t)ptr & 3) != 0) return fail(PP_EINVAL, "%s is not 4-byte aligned", name);
    return host_io ? PP_OK : check_dev_ptr(ptr, dev, name);
}

// Where pp_grad_host's kernels find one caller array: device memory of this device or
// pinned host memory (its device mapping) in place; pageable host memory is staged.
struct HostArg {
    void *dev;       // what the kernels read or write
    bool staged;     // pageable: copied through the workspace
};
pp_status resolve_host_arg(const void *ptr, int dev, const char *name, void *staging, HostArg *out) {
    out->dev = nullptr;
    out->staged = false;
    if (!ptr) return PP_OK;
    if (((uintptr_t)ptr & 3) != 0) return fail(PP_EINVAL, "%s is not 4-byte aligned", name);
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        at.type = cudaMemoryTypeUnregistered;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
        if (at.device != dev)
            return fail(PP_EINVAL, "%s: lives on device %d, current device is %d", name, at.device, dev);
        out->dev = const_cast<void *>(ptr);
    } else if (at.type == cudaMemoryTypeHost && at.devicePointer) {
        out->dev = at.devicePointer;
    } else {
        out->dev = staging;
        out->staged = true;
    }
    return PP_OK;
}

// pp_grad_host's workspace: [pp_workspace_size bytes][E, 256 B][staging: x y w h c gx gy N, 4n B each]
size_t host_extra_bytes(int64_t n) { return 256 + 8 * align256((size_t)n * sizeof(float)); }

#define PP_TRY(expr, what)                                  \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return cuda_fail(_e, what);  \
    } while (0)

// ---- optional per-launch event timing (pp_timing_enable / pp_timing_collect)
struct TimedLaunch {
    cudaEvent_t a, b;
    int kind;
};
constexpr size_t kMaxTimed = 65536;
std::mutex g_tmu;
std::atomic<bool> g_timing{false};
std::vector<TimedLaunch> g_tpool;
size_t g_tused = 0;
std::atomic<int64_t> g_tcount[PP_K_COUNT];

long timed_begin(int kind, cudaStream_t s) {
    g_tcount[kind].fetch_add(1, std::memory_order_relaxed);       // every launch is counted
    if (!g_timing.load(std::memory_order_relaxed)) return -1;
    std::lock_guard<std::mutex> lk(g_tmu);
    if (g_tused >= kMaxTimed) return -1;
    if (g_tused == g_tpool.size()) {
        TimedLaunch t{};
        if (cudaEventCreate(&t.a) != cudaSuccess || cudaEventCreate(&t.b) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        g_tpool.push_back(t);
    }
    TimedLaunch &t = g_tpool[g_tused];
    t.kind = kind;
    if (cudaEventRecord(t.a, s) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return (long)g_tused++;
}

void timed_end(long idx, cudaStream_t s) {
    if (idx < 0) return;
    std::lock_guard<std::mutex> lk(g_tmu);
    cudaEventRecord(g_tpool[(size_t)idx].b, s);
}

#define PP_LAUNCH(kind, stream, expr, what)                 \
    do {                                                    \
        long _t = timed_begin((kind), (stream));            \
        cudaError_t _e = (expr);                            \
        timed_end(_t, (stream));                            \
        if (_e != cudaSuccess) return cuda_fail(_e, what);  \
    } while (0)

// Coefficients into the workspace (FP32: S64 and K; tensor cores: partial tiles
// and the tiled K operand), optionally also to a_out.
pp_status run_coefficients(Ctx &c, float *a_out, double *e_total = nullptr) {
    if (c.prec == PP_FP32) {
        PP_LAUNCH(PP_K_COEFF, c.L.stream, launch_coeff_simt(c.L), "coefficient kernel launch");
        PP_LAUNCH(PP_K_FINISH, c.L.stream, launch_finish_simt(c.L, nullptr, a_out), "finish kernel launch");
    } else {
        float *part = (float *)(c.base + c.lay.part);
        void *Khi = c.base + c.lay.K, *Klo = c.base + c.lay.Klo;
        PP_LAUNCH(PP_K_COEFF, c.L.stream, launch_coeff_tc(c.L, (int)c.prec, c.lay.plan, part),
                  "coefficient kernel launch");
        PP_LAUNCH(PP_K_FINISH, c.L.stream,
                  launch_finish_tc(c.L, (int)c.prec, c.lay.plan, part, nullptr, a_out, Khi, Klo, e_total),
                  "finish kernel launch");
    }
    return PP_OK;
}

// Energy operand K from caller-provided coefficients.
pp_status operand_from_a(Ctx &c, const float *a) {
    if (c.prec == PP_FP32) {
        PP_LAUNCH(PP_K_FINISH, c.L.stream, launch_finish_simt(c.L, a, nullptr), "finish kernel launch");
    } else {
        PP_LAUNCH(PP_K_FINISH, c.L.stream,
                  launch_finish_tc(c.L, (int)c.prec, c.lay.plan, nullptr, a, nullptr, c.base + c.lay.K,
                                   c.base + c.lay.Klo, nullptr),
                  "finish kernel launch");
    }
    return PP_OK;
}

pp_status run_energy(Ctx &c, pp_sample sample, float *e_block, double *e_total, float *gx, float *gy,
                     const GradOut &go = GradOut()) {
    if (c.prec == PP_FP32) {
        PP_LAUNCH(PP_K_ENERGY, c.L.stream, launch_energy_simt(c.L, (int)sample, e_block, e_total, gx, gy, go),
                  "energy kernel launch");
    } else {
        PP_LAUNCH(PP_K_ENERGY, c.L.stream,
                  launch_energy_tc(c.L, (int)c.prec, (int)sample, c.lay.plan, c.base + c.lay.K,
                                   c.base + c.lay.Klo, e_block, e_total, gx, gy, go),
                  "energy kernel launch");
    }
    return PP_OK;
}

// Coefficients of these blocks added into a64 (FP64, Mx x My); a_out (optional)
// receives the rounded running sum.  No energy operand is formed.
pp_status accumulate_coefficients(Ctx &c, double *a64, float *a_out) {
    if (c.prec == PP_FP32) {
        PP_LAUNCH(PP_K_COEFF, c.L.stream, launch_coeff_simt(c.L), "coefficient kernel launch");
        PP_LAUNCH(PP_K_FINISH, c.L.stream, launch_finish_simt(c.L, nullptr, a_out, a64, false),
                  "finish kernel launch");
    } else {
        float *part = (float *)(c.base + c.lay.part);
        PP_LAUNCH(PP_K_COEFF, c.L.stream, launch_coeff_tc(c.L, (int)c.prec, c.lay.plan, part),
                  "coefficient kernel launch");
        PP_LAUNCH(PP_K_FINISH, c.L.stream,
                  launch_finish_tc(c.L, (int)c.prec, c.lay.plan, part, nullptr, a_out, nullptr, nullptr,
                                   nullptr, a64),
                  "finish kernel launch");
    }
    return PP_OK;
}

pp_status energy_common(const pp_problem *p, pp_precision prec, pp_sample sample, const float *a,
                        float *gx, float *gy, float *e_block, double *e_total, void *ws,
                        size_t ws_bytes, void *stream, bool want_grad, bool host_io = false) {
    Ctx c;
    pp_status st = setup(p, prec, ws, ws_bytes, stream, &c, host_io);
    if (st != PP_OK) return st;
    if (sample != PP_RECT && sample != PP_CENTER) return fail(PP_EINVAL, "unknown sample mode %d", (int)sample);
    const bool has_blocks = p->n > 0;   // per-block arrays may be NULL when n = 0
    if (want_grad) {
        if ((st = out_ptr(gx, c.dev, "gx", has_blocks, host_io)) != PP_OK) return st;
        if ((st = out_ptr(gy, c.dev, "gy", has_blocks, host_io)) != PP_OK) return st;
    } else if (!e_block && !e_total && has_blocks) {
        return fail(PP_EINVAL, "e_block and e_total are both NULL");
    }
    if ((st = out_ptr(e_block, c.dev, "e_block", false, host_io)) != PP_OK) return st;
    if (e_total) {
        if (((uintptr_t)e_total & 7) != 0) return fail(PP_EINVAL, "e_total is not 8-byte aligned");
        if ((st = check_dev_ptr(e_total, c.dev, "e_total")) != PP_OK) return st;
    }
    if (a && (st = out_ptr(a, c.dev, "a", false)) != PP_OK) return st;
    if (p->n == 0) {
        if (e_total) PP_TRY(cudaMemsetAsync(e_total, 0, sizeof(double), c.L.stream), "memset e_total");
        return PP_OK;
    }
    const bool zero_S = a == nullptr && prec == PP_FP32;
    PP_LAUNCH(PP_K_PREP, c.L.stream, launch_prep(c.L, zero_S, e_total), "prep kernel launch");
    // Tensor-core path, rectangle sampling, coefficients of these blocks: E comes from
    // the FP32 coefficients (1/2 sum a S, FP64) in the finish kernel instead of the
    // per-block sums, whose K operand is rounded to TF32 or bf16 pairs.
    const bool e_from_a = prec != PP_FP32 && sample == PP_RECT && a == nullptr;
    st = a ? operand_from_a(c, a) : run_coefficients(c, nullptr, e_from_a ? e_total : nullptr);
    if (st != PP_OK) return st;
    st = run_energy(c, sample, e_block, e_from_a ? nullptr : e_total, want_grad ? gx : nullptr,
                    want_grad ? gy : nullptr);
    if (st != PP_OK) return st;
    return PP_OK;
}

}  // namespace

void set_last_error(const char *msg) { t_err = msg ? msg : ""; }

}  // namespace pp

using namespace pp;

extern "C" {

size_t pp_workspace_size(const pp_problem *prob, pp_precision prec) {
    if (check_shape(prob, prec) != PP_OK) return 0;
    return layout(prob, prec).total;
}

pp_status pp_coeffs(const pp_problem *prob, pp_precision prec, float *a, void *ws, size_t ws_bytes,
                    void *stream) {
    Ctx c;
    pp_status st = setup(prob, prec, ws, ws_bytes, stream, &c);
    if (st != PP_OK) return st;
    if ((st = out_ptr(a, c.dev, "a", true)) != PP_OK) return st;
    if (prob->n == 0) {
        PP_TRY(cudaMemsetAsync(a, 0, (size_t)prob->Mx * prob->My * sizeof(float), c.L.stream), "memset a");
        return PP_OK;
    }
    PP_LAUNCH(PP_K_PREP, c.L.stream, launch_prep(c.L, prec == PP_FP32, nullptr), "prep kernel launch");
    return run_coefficients(c, a);
}

pp_status pp_energy(const pp_problem *prob, pp_precision prec, pp_sample sample, const float *a,
                    float *e_block, double *e_total, void *ws, size_t ws_bytes, void *stream) {
    return energy_common(prob, prec, sample, a, nullptr, nullptr, e_block, e_total, ws, ws_bytes,
                         stream, false);
}

pp_status pp_grad(const pp_problem *prob, pp_precision prec, pp_sample sample, const float *a,
                  float *gx, float *gy, float *e_block, double *e_total, void *ws, size_t ws_bytes,
                  void *stream) {
    return energy_common(prob, prec, sample, a, gx, gy, e_block, e_total, ws, ws_bytes, stream, true);
}

size_t pp_grad_host_workspace_size(const pp_problem *prob, pp_precision prec) {
    if (check_shape(prob, prec) != PP_OK) return 0;
    return layout(prob, prec).total + host_extra_bytes(prob->n);
}

pp_status pp_grad_host(const pp_problem *prob, pp_precision prec, pp_sample sample, float *gx, float *gy,
                       float *e_block, double *e_total, void *ws, size_t ws_bytes, void *stream) {
    pp_status st = check_problem(prob, prec);
    if (st != PP_OK) return st;
    const size_t core = layout(prob, prec).total, need = core + host_extra_bytes(prob->n);
    if (!ws || ws_bytes < need)
        return fail(PP_ENOMEM_WS, "workspace of %zu bytes needed, %zu given%s", need, ws ? ws_bytes : (size_t)0,
                    ws ? "" : " (NULL)");
    if (((uintptr_t)ws & 255) != 0) return fail(PP_EINVAL, "workspace must be 256-byte aligned");
    int dev = 0, sm = 0, ccm = 0;
    unsigned *status;
    if ((st = device_info(&dev, &sm, &status, &ccm)) != PP_OK) return st;
    if ((st = check_dev_ptr(ws, dev, "ws")) != PP_OK) return st;
    const bool has_blocks = prob->n > 0;
    if (has_blocks && (!gx || !gy)) return fail(PP_EINVAL, "gx and gy must be non-NULL when n > 0");
    if (e_total && ((uintptr_t)e_total & 7) != 0) return fail(PP_EINVAL, "e_total is not 8-byte aligned");
    char *extra = (char *)ws + core;
    double *e_dev = (double *)extra;
    const size_t arr = align256((size_t)prob->n * sizeof(float)), bytes = (size_t)prob->n * sizeof(float);
    char *stg = extra + 256;
    const void *ins[5] = {prob->x, prob->y, prob->w, prob->h, prob->c};
    const char *in_names[5] = {"x", "y", "w", "h", "c"};
    HostArg in[5], out[3];
    for (int i = 0; i < 5; ++i)
        if ((st = resolve_host_arg(has_blocks ? ins[i] : nullptr, dev, in_names[i], stg + i * arr, &in[i])) != PP_OK)
            return st;
    void *outs[3] = {gx, gy, e_block};
    const char *out_names[3] = {"gx", "gy", "e_block"};
    for (int i = 0; i < 3; ++i)
        if ((st = resolve_host_arg(has_blocks ? outs[i] : nullptr, dev, out_names[i], stg + (5 + i) * arr,
                                   &out[i])) != PP_OK)
            return st;
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < 5; ++i)
        if (in[i].staged) PP_TRY(cudaMemcpyAsync(in[i].dev, ins[i], bytes, cudaMemcpyHostToDevice, s), "stage input");
    pp_problem p = *prob;
    p.x = (const float *)in[0].dev;
    p.y = (const float *)in[1].dev;
    p.w = (const float *)in[2].dev;
    p.h = (const float *)in[3].dev;
    p.c = (const float *)in[4].dev;
    st = energy_common(&p, prec, sample, nullptr, (float *)out[0].dev, (float *)out[1].dev, (float *)out[2].dev,
                       e_total ? e_dev : nullptr, ws, core, stream, true, true);
    if (st != PP_OK) return st;
    for (int i = 0; i < 3; ++i)
        if (out[i].staged) PP_TRY(cudaMemcpyAsync(outs[i], out[i].dev, bytes, cudaMemcpyDeviceToHost, s), "read output");
    if (e_total) PP_TRY(cudaMemcpyAsync(e_total, e_dev, sizeof(double), cudaMemcpyDefault, s), "read E");
    return PP_OK;
}

pp_status pp_grad_adjoint(const pp_problem *prob, pp_precision prec, pp_sample sample, const double *g_total,
                          const float *g_block, const uint8_t *movable, float *gx, float *gy, float *e_block,
                          double *e_total, void *ws, size_t ws_bytes, void *stream) {
    Ctx c;
    pp_status st = setup(prob, prec, ws, ws_bytes, stream, &c);
    if (st != PP_OK) return st;
    if (sample != PP_RECT && sample != PP_CENTER) return fail(PP_EINVAL, "unknown sample mode %d", (int)sample);
    if (!g_total && !g_block) return fail(PP_EINVAL, "g_total and g_block are both NULL");
    if (g_block && sample != PP_RECT)
        return fail(PP_EINVAL, "per-block upstream gradients (g_block) need the rectangle reading PP_RECT");
    const bool has_blocks = prob->n > 0;
    if ((st = out_ptr(gx, c.dev, "gx", has_blocks)) != PP_OK) return st;
    if ((st = out_ptr(gy, c.dev, "gy", has_blocks)) != PP_OK) return st;
    if ((st = out_ptr(e_block, c.dev, "e_block", false)) != PP_OK) return st;
    if (e_total) {
        if (((uintptr_t)e_total & 7) != 0) return fail(PP_EINVAL, "e_total is not 8-byte aligned");
        if ((st = check_dev_ptr(e_total, c.dev, "e_total")) != PP_OK) return st;
    }
    if (g_total) {
        if (((uintptr_t)g_total & 7) != 0) return fail(PP_EINVAL, "g_total is not 8-byte aligned");
        if ((st = check_dev_ptr(g_total, c.dev, "g_total")) != PP_OK) return st;
    }
    if (has_blocks && g_block && (st = out_ptr(g_block, c.dev, "g_block", true)) != PP_OK) return st;
    if (has_blocks && movable && (st = check_dev_ptr(movable, c.dev, "movable")) != PP_OK) return st;
    if (!has_blocks) {
        if (e_total) PP_TRY(cudaMemsetAsync(e_total, 0, sizeof(double), c.L.stream), "memset e_total");
        return PP_OK;
    }
    // pass 1: the placement's coefficients a and h = dE/d(x, y) (the whole answer when
    // only g_total is given: g_total * h, masked)
    PP_LAUNCH(PP_K_PREP, c.L.stream, launch_prep(c.L, prec == PP_FP32, e_total), "prep kernel launch");
    const bool e_from_a = prec != PP_FP32 && sample == PP_RECT;
    if ((st = run_coefficients(c, nullptr, e_from_a ? e_total : nullptr)) != PP_OK) return st;
    GradOut g1;
    if (!g_block) {
        g1.scale = g_total;
        g1.mask = movable;
    }
    if ((st = run_energy(c, sample, e_block, e_from_a ? nullptr : e_total, gx, gy, g1)) != PP_OK) return st;
    if (!g_block) return PP_OK;
    // pass 2: coefficients b of the charges c_i w_i, w_i = g_total / 2 + g_block_i, then
    // h^b from the records with the plain charges again, combined as w_j h_j + h^b_j
    ChargeWeights cw;
    cw.gw = g_block;
    cw.gt = g_total;
    cw.on = true;
    PP_LAUNCH(PP_K_PREP, c.L.stream, launch_prep(c.L, prec == PP_FP32, nullptr, cw), "prep kernel launch");
    if ((st = run_coefficients(c, nullptr)) != PP_OK) return st;
    PP_LAUNCH(PP_K_PREP, c.L.stream, launch_prep(c.L, false, nullptr), "prep kernel launch");
    GradOut g2;
    g2.acc = true;
    g2.w = g_block;
    g2.wt = g_total;
    g2.mask = movable;
    return run_energy(c, sample, nullptr, nullptr, gx, gy, g2);
}

pp_status pp_coeffs_accumulate(const pp_problem *prob, pp_precision prec, double *a64, float *a_out, void *ws,
                               size_t ws_bytes, void *stream) {
    Ctx c;
    pp_status st = setup(prob, prec, ws, ws_bytes, stream, &c);
    if (st != PP_OK) return st;
    if (!a64) return fail(PP_EINVAL, "a64 must be non-NULL");
    if (((uintptr_t)a64 & 7) != 0) return fail(PP_EINVAL, "a64 is not 8-byte aligned");
    if ((st = check_dev_ptr(a64, c.dev, "a64")) != PP_OK) return st;
    if ((st = out_ptr(a_out, c.dev, "a_out", false)) != PP_OK) return st;
    if (prob->n == 0) {
        if (a_out)
            PP_TRY(launch_round_coeffs(a64, a_out, (size_t)prob->Mx * prob->My, c.L.stream), "round kernel launch");
        return PP_OK;
    }
    PP_LAUNCH(PP_K_PREP, c.L.stream, launch_prep(c.L, prec == PP_FP32, nullptr), "prep kernel launch");
    return accumulate_coefficients(c, a64, a_out);
}

pp_status pp_sync_status(void *stream) {
    int dev = 0, sm = 0, ccm = 0;
    unsigned *status;
    pp_status st = device_info(&dev, &sm, &status, &ccm);
    if (st != PP_OK) return st;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    unsigned v = 0;
    e = cudaMemcpyFromSymbol(&v, g_status, sizeof v);
    if (e != cudaSuccess) return cuda_fail(e, "read status word");
    if (v) {
        const unsigned zero = 0;
        e = cudaMemcpyToSymbol(g_status, &zero, sizeof zero);
        if (e != cudaSuccess) return cuda_fail(e, "clear status word");
        return fail(PP_ETIMEOUT, "a kernel gave up a bounded wait (status 0x%x)", v);
    }
    return PP_OK;
}

pp_status pp_phase_eval(const float *x, double L, const int32_t *m, int64_t count, int evaluator,
                        float *out, void *stream) {
    int dev = 0, sm = 0, ccm = 0;
    unsigned *status;
    pp_status st = device_info(&dev, &sm, &status, &ccm);
    if (st != PP_OK) return st;
    if (!(std::isfinite(L) && L >= 1e-300 && L <= 1e300))
        return fail(PP_EINVAL, "L must be finite and in [1e-300, 1e300]");
    if (count < 0) return fail(PP_EINVAL, "count must be >= 0");
    if (evaluator < 0 || evaluator > 2) return fail(PP_EINVAL, "evaluator must be 0, 1 or 2");
    if (count == 0) return PP_OK;
    if ((st = check_dev_ptr(x, dev, "x")) != PP_OK) return st;
    if ((st = check_dev_ptr(m, dev, "m")) != PP_OK) return st;
    if ((st = check_dev_ptr(out, dev, "out")) != PP_OK) return st;
    cudaError_t e = launch_phase_eval(x, 1.0 / L, m, count, evaluator, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "phase evaluation launch");
    return PP_OK;
}

size_t pp_binned_workspace_size(const pp_problem *prob, int32_t m) {
    if (check_shape(prob, PP_FP32) != PP_OK) return 0;
    if (m < 2 || m > 4096 || prob->Mx > m || prob->My > m) {
        fail(PP_EINVAL, "bins m=%d must be in [2, 4096] and >= Mx=%d, My=%d", m, prob->Mx, prob->My);
        return 0;
    }
    return binned_layout(m, prob->Mx, prob->My).total;
}

pp_status pp_binned_grad(const pp_problem *prob, pp_precision prec, int32_t m, float *a_out, float *gx,
                         float *gy, float *e_block, double *e_total, void *ws, size_t ws_bytes, void *stream) {
    pp_status st = check_problem(prob, PP_FP32);
    if (st != PP_OK) return st;
    if (prec != PP_FP32 && prec != PP_TF32)
        return fail(prec == PP_BF16X3 ? PP_ENOTSUP : PP_EINVAL, "binned scheme: precision %d not offered",
                    (int)prec);
    const size_t need = pp_binned_workspace_size(prob, m);
    if (need == 0) return PP_EINVAL;
    int dev = 0, sm = 0, ccm = 0;
    unsigned *status;
    if ((st = device_info(&dev, &sm, &status, &ccm)) != PP_OK) return st;
    if (!ws || ws_bytes < need)
        return fail(PP_ENOMEM_WS, "workspace of %zu bytes needed, %zu given", need, ws ? ws_bytes : (size_t)0);
    if (((uintptr_t)ws & 255) != 0) return fail(PP_EINVAL, "workspace must be 256-byte aligned");
    if ((st = check_dev_ptr(ws, dev, "ws")) != PP_OK) return st;
    const bool has_blocks = prob->n > 0;
    if (has_blocks) {
        const void *ptrs[5] = {prob->x, prob->y, prob->w, prob->h, prob->c};
        const char *names[5] = {"x", "y", "w", "h", "c"};
        for (int i = 0; i < 5; ++i)
            if (ptrs[i] && (st = check_dev_ptr(ptrs[i], dev, names[i])) != PP_OK) return st;
    }
    if ((st = out_ptr(gx, dev, "gx", has_blocks)) != PP_OK) return st;
    if ((st = out_ptr(gy, dev, "gy", has_blocks)) != PP_OK) return st;
    if ((st = out_ptr(e_block, dev, "e_block", false)) != PP_OK) return st;
    if ((st = out_ptr(a_out, dev, "a_out", false)) != PP_OK) return st;
    if (e_total) {
        if (((uintptr_t)e_total & 7) != 0) return fail(PP_EINVAL, "e_total is not 8-byte aligned");
        if ((st = check_dev_ptr(e_total, dev, "e_total")) != PP_OK) return st;
    }
    Launch L{};
    L.W = prob->W;
    L.H = prob->H;
    L.n = (int)prob->n;
    L.Mx = prob->Mx;
    L.My = prob->My;
    L.x = prob->x;
    L.y = prob->y;
    L.w = prob->w;
    L.h = prob->h;
    L.c = prob->c;
    L.status = status;
    L.sm_count = sm;
    L.stream = (cudaStream_t)stream;
    const char *what = "";
    cudaError_t e = run_binned(L, dev, m, prec == PP_TF32, (unsigned char *)ws, a_out, e_block, gx, gy,
                               e_total, &what);
    if (e != cudaSuccess) return cuda_fail(e, what);
    return PP_OK;
}

pp_status pp_energy_from_coeffs(const float *a, int32_t Mx, int32_t My, double W, double H, double *e_total,
                                void *stream) {
    int dev = 0, sm = 0, ccm = 0;
    unsigned *status;
    pp_status st = device_info(&dev, &sm, &status, &ccm);
    if (st != PP_OK) return st;
    if (!(std::isfinite(W) && std::isfinite(H) && W >= 1e-300 && W <= 1e300 && H >= 1e-300 && H <= 1e300))
        return fail(PP_EINVAL, "die size W=%g H=%g must be finite and in [1e-300, 1e300]", W, H);
    if (Mx < 1 || My < 1 || Mx > 4096 || My > 4096) return fail(PP_EINVAL, "Mx=%d My=%d out of range", Mx, My);
    if ((st = check_dev_ptr(a, dev, "a")) != PP_OK) return st;
    if (((uintptr_t)e_total & 7) != 0) return fail(PP_EINVAL, "e_total is not 8-byte aligned");
    if ((st = check_dev_ptr(e_total, dev, "e_total")) != PP_OK) return st;
    PP_TRY(cudaMemsetAsync(e_total, 0, sizeof(double), (cudaStream_t)stream), "memset e_total");
    cudaError_t e = launch_energy_from_coeffs(a, Mx, My, W, H, e_total, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "energy-from-coefficients launch");
    return PP_OK;
}

pp_status pp_descent_step(double W, double H, int64_t n, float *x, float *y, const float *w,
                          const float *h, const float *gx, const float *gy, const uint8_t *movable,
                          float lr, float sigma, uint64_t seed, uint64_t step, void *stream) {
    int dev = 0, sm = 0, ccm = 0;
    unsigned *status;
    pp_status st = device_info(&dev, &sm, &status, &ccm);
    if (st != PP_OK) return st;
    if (!(std::isfinite(W) && std::isfinite(H) && W >= 1e-300 && W <= 1e300 && H >= 1e-300 && H <= 1e300))
        return fail(PP_EINVAL, "die size W=%g H=%g must be finite and in [1e-300, 1e300]", W, H);
    if (n < 0 || n > INT64_C(0x7FFFFFFF)) return fail(PP_EINVAL, "n=%lld out of range", (long long)n);
    if (!std::isfinite(lr) || !std::isfinite(sigma)) return fail(PP_EINVAL, "lr and sigma must be finite");
    if (n == 0) return PP_OK;
    const void *ptrs[6] = {x, y, w, h, gx, gy};
    const char *names[6] = {"x", "y", "w", "h", "gx", "gy"};
    for (int i = 0; i < 6; ++i)
        if ((st = check_dev_ptr(ptrs[i], dev, names[i])) != PP_OK) return st;
    if (movable && (st = check_dev_ptr(movable, dev, "movable")) != PP_OK) return st;
    cudaError_t e = launch_descent_step((float)W, (float)H, n, x, y, w, h, gx, gy, movable, lr, sigma,
                                        seed, step, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "descent step launch");
    return PP_OK;
}

// ---- placement loop (Sec. IV) -------------------------------------------------
namespace {
pp_status check_netlist(const pp_netlist *nl, int dev) {
    if (!nl) return fail(PP_EINVAL, "netlist is NULL");
    if (nl->n_cells < 0 || nl->n_nets < 0) return fail(PP_EINVAL, "negative netlist sizes");
    pp_status st;
    if (nl->n_nets > 0) {
        if ((st = check_dev_ptr(nl->net_ptr, dev, "net_ptr")) != PP_OK) return st;
        if ((st = check_dev_ptr(nl->net_pin, dev, "net_pin")) != PP_OK) return st;
    }
    if (nl->n_cells > 0) {
        if ((st = check_dev_ptr(nl->cell_ptr, dev, "cell_ptr")) != PP_OK) return st;
        if ((st = check_dev_ptr(nl->cell_net, dev, "cell_net")) != PP_OK) return st;
    }
    return PP_OK;
}
pp_status check_arrays(int dev, int count, const void *const *ptrs, const char *const *names) {
    pp_status st;
    for (int i = 0; i < count; ++i)
        if ((st = check_dev_ptr(ptrs[i], dev, names[i])) != PP_OK) return st;
    return PP_OK;
}
}  // namespace

size_t pp_wirelength_workspace_size(int32_t n_nets) {
    return n_nets <= 0 ? 256 : ((size_t)n_nets * 32 + 255) & ~(size_t)255;
}

namespace {
// The entry points of the loop with their scalars optionally on the device (`scal`,
// {lambda, gamma, alpha0, coef}, read by the kernels when they run); a by-value
// scalar is checked only when scal is NULL.
pp_status wirelength_impl(const pp_netlist *nl, const float *x, const float *y, float gamma, const float *scal,
                          float *gx, float *gy, double *out, void *ws, size_t ws_bytes, void *stream) {
    int dev = 0, sm = 0, ccm = 0;
    unsigned *status;
    pp_status st = device_info(&dev, &sm, &status, &ccm);
    if (st != PP_OK) return st;
    if ((st = check_netlist(nl, dev)) != PP_OK) return st;
    if (!scal && !(std::isfinite(gamma) && gamma > 0.f)) return fail(PP_EINVAL, "gamma must be finite and > 0");
    const size_t need = pp_wirelength_workspace_size(nl->n_nets);
    if (!ws || ws_bytes < need)
        return fail(PP_ENOMEM_WS, "workspace of %zu bytes needed, %zu given", need, ws ? ws_bytes : (size_t)0);
    if (((uintptr_t)ws & 255) != 0) return fail(PP_EINVAL, "workspace must be 256-byte aligned");
    if ((st = check_dev_ptr(ws, dev, "ws")) != PP_OK) return st;
    if ((st = check_dev_ptr(out, dev, "out")) != PP_OK) return st;
    if (((uintptr_t)out & 7) != 0) return fail(PP_EINVAL, "out is not 8-byte aligned");
    if (nl->n_cells > 0) {            // gx == gy == NULL: the per-net pass only (internal use)
        const void *ptrs[4] = {x, y, gx, gy};
        const char *names[4] = {"x", "y", "gx", "gy"};
        if ((st = check_arrays(dev, gx ? 4 : 2, ptrs, names)) != PP_OK) return st;
    }
    cudaError_t e = launch_wirelength(nl->n_nets, nl->n_cells, nl->net_ptr, nl->net_pin, nl->cell_ptr,
                                      nl->cell_net, x, y, gamma, scal, (float *)ws, gx, gy, out, sm,
                                      (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "wirelength launch");
    return PP_OK;
}

pp_status combine_impl(int64_t n, const float *gwx, const float *gwy, const float *gnx, const float *gny,
                       const int32_t *cell_ptr, const float *q, const uint8_t *movable, float lambda,
                       const float *scal, float *gx, float *gy, void *stream) {
    int dev = 0, sm = 0, ccm = 0;
    unsigned *status;
    pp_status st = device_info(&dev, &sm, &status, &ccm);
    if (st != PP_OK) return st;
    if (n < 0 || n > INT64_C(0x7FFFFFFF)) return fail(PP_EINVAL, "n=%lld out of range", (long long)n);
    if (!scal && !(std::isfinite(lambda) && lambda >= 0.f))
        return fail(PP_EINVAL, "lambda must be finite and >= 0");
    if (n == 0) return PP_OK;
    const void *ptrs[7] = {gwx, gwy, gnx, gny, q, gx, gy};
    const char *names[7] = {"gwx", "gwy", "gnx", "gny", "q", "gx", "gy"};
    if ((st = check_arrays(dev, 7, ptrs, names)) != PP_OK) return st;
    if (cell_ptr && (st = check_dev_ptr(cell_ptr, dev, "cell_ptr")) != PP_OK) return st;
    if (movable && (st = check_dev_ptr(movable, dev, "movable")) != PP_OK) return st;
    cudaError_t e = launch_combine(n, gwx, gwy, gnx, gny, cell_ptr, q, movable, lambda, scal, gx, gy,
                                   (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "combine launch");
    return PP_OK;
}

pp_status nesterov_impl(int64_t n, double W, double H, float *ux, float *uy, float *vx, float *vy, float *vpx,
                        float *vpy, const float *gx, const float *gy, float *gpx, float *gpy, const float *w,
                        const float *h, const uint8_t *movable, const double *norms, float alpha0, float coef,
                        const float *scal, void *stream) {
    int dev = 0, sm = 0, ccm = 0;
    unsigned *status;
    pp_status st = device_info(&dev, &sm, &status, &ccm);
    if (st != PP_OK) return st;
    if (!(std::isfinite(W) && std::isfinite(H) && W >= 1e-300 && W <= 1e300 && H >= 1e-300 && H <= 1e300))
        return fail(PP_EINVAL, "die size W=%g H=%g must be finite and in [1e-300, 1e300]", W, H);
    if (n < 0 || n > INT64_C(0x7FFFFFFF)) return fail(PP_EINVAL, "n=%lld out of range", (long long)n);
    if (!scal && !(std::isfinite(alpha0) && alpha0 >= 0.f && std::isfinite(coef)))
        return fail(PP_EINVAL, "alpha0 must be finite and >= 0, coef finite");
    if (n == 0) return PP_OK;
    const void *ptrs[12] = {ux, uy, vx, vy, vpx, vpy, gx, gy, gpx, gpy, w, h};
    const char *names[12] = {"ux", "uy", "vx", "vy", "vpx", "vpy", "gx", "gy", "gpx", "gpy", "w", "h"};
    if ((st = check_arrays(dev, 12, ptrs, names)) != PP_OK) return st;
    if (movable && (st = check_dev_ptr(movable, dev, "movable")) != PP_OK) return st;
    if (norms && (st = check_dev_ptr(norms, dev, "norms")) != PP_OK) return st;
    cudaError_t e = launch_nesterov(n, ux, uy, vx, vy, vpx, vpy, gx, gy, gpx, gpy, w, h, (float)W, (float)H,
                                    movable, norms, alpha0, coef, scal, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "Nesterov step launch");
    return PP_OK;
}
}  // namespace

pp_status pp_step_norms(int64_t n, const float *vx, const float *vy, const float *vpx, const float *vpy,
                        const float *gx, const float *gy, const float *gpx, const float *gpy, double *norms,
                        void *stream) {
    int dev = 0, sm = 0, ccm = 0;
    unsigned *status;
    pp_status st = device_info(&dev, &sm, &status, &ccm);
    if (st != PP_OK) return st;
    if (n < 0 || n > INT64_C(0x7FFFFFFF)) return fail(PP_EINVAL, "n=%lld out of range", (long long)n);
    if ((st = check_dev_ptr(norms, dev, "norms")) != PP_OK) return st;
    if (((uintptr_t)norms & 7) != 0) return fail(PP_EINVAL, "norms is not 8-byte aligned");
    if (n > 0) {
        const void *ptrs[8] = {vx, vy, vpx, vpy, gx, gy, gpx, gpy};
        const char *names[8] = {"vx", "vy", "vpx", "vpy", "gx", "gy", "gpx", "gpy"};
        if ((st = check_arrays(dev, 8, ptrs, names)) != PP_OK) return st;
    }
    cudaError_t e = launch_step_norms(n, vx, vy, vpx, vpy, gx, gy, gpx, gpy, norms, sm, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "step norms launch");
    return PP_OK;
}

pp_status pp_wirelength(const pp_netlist *nl, const float *x, const float *y, float gamma, float *gx, float *gy,
                        double *out, void *ws, size_t ws_bytes, void *stream) {
    if (nl && nl->n_cells > 0 && (!gx || !gy)) return fail(PP_EINVAL, "gx, gy must not be NULL");
    return wirelength_impl(nl, x, y, gamma, nullptr, gx, gy, out, ws, ws_bytes, stream);
}

pp_status pp_place_combine(int64_t n, const float *gwx, const float *gwy, const float *gnx, const float *gny,
                           const int32_t *cell_ptr, const float *q, const uint8_t *movable, float lambda,
                           float *gx, float *gy, void *stream) {
    return combine_impl(n, gwx, gwy, gnx, gny, cell_ptr, q, movable, lambda, nullptr, gx, gy, stream);
}

pp_status pp_nesterov_step(int64_t n, double W, double H, float *ux, float *uy, float *vx, float *vy, float *vpx,
                           float *vpy, const float *gx, const float *gy, float *gpx, float *gpy, const float *w,
                           const float *h, const uint8_t *movable, const double *norms, float alpha0,
                           float coef, void *stream) {
    return nesterov_impl(n, W, H, ux, uy, vx, vy, vpx, vpy, gx, gy, gpx, gpy, w, h, movable, norms, alpha0, coef,
                         nullptr, stream);
}

pp_status pp_overflow(const pp_problem *prob, int32_t m, float target, float *bins, double *out, void *stream) {
    int dev = 0, sm = 0, ccm = 0;
    unsigned *status;
    pp_status st = device_info(&dev, &sm, &status, &ccm);
    if (st != PP_OK) return st;
    if (!prob) return fail(PP_EINVAL, "problem is NULL");
    if (!(std::isfinite(prob->W) && std::isfinite(prob->H) && prob->W >= 1e-300 && prob->W <= 1e300 &&
          prob->H >= 1e-300 && prob->H <= 1e300))
        return fail(PP_EINVAL, "die size must be finite and in [1e-300, 1e300]");
    if (prob->n < 0 || prob->n > INT64_C(0x7FFFFFFF)) return fail(PP_EINVAL, "n out of range");
    if (m < 1 || m > 8192) return fail(PP_EINVAL, "bins m=%d must be in [1, 8192]", m);
    if (!(std::isfinite(target) && target >= 0.f)) return fail(PP_EINVAL, "target must be finite and >= 0");
    if ((st = check_dev_ptr(bins, dev, "bins")) != PP_OK) return st;
    if ((st = check_dev_ptr(out, dev, "out")) != PP_OK) return st;
    if (((uintptr_t)out & 7) != 0) return fail(PP_EINVAL, "out is not 8-byte aligned");
    if (prob->n > 0) {
        const void *ptrs[4] = {prob->x, prob->y, prob->w, prob->h};
        const char *names[4] = {"x", "y", "w", "h"};
        if ((st = check_arrays(dev, 4, ptrs, names)) != PP_OK) return st;
        if (prob->c && (st = check_dev_ptr(prob->c, dev, "c")) != PP_OK) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(bins, 0, (size_t)m * m * sizeof(float), s);
    if (e == cudaSuccess)
        e = launch_bin_density(prob->x, prob->y, prob->w, prob->h, prob->c, (int)prob->n, m, prob->W, prob->H,
                               bins, sm, s);
    if (e == cudaSuccess) e = launch_overflow(m, bins, target, out, sm, s);
    if (e != cudaSuccess) return cuda_fail(e, "overflow launch");
    return PP_OK;
}

namespace {
// Scratch of one placement iteration: the density and wirelength workspaces, four
// float arrays of n (gn and g per axis), the two norms and the M x M bins.
struct PlaceLayout {
    size_t dens, dens_bytes, wl, wl_bytes, vec, vec_bytes, norms, bins, total;
};

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

pp_status place_layout(const pp_place_iteration_args *a, PlaceLayout *L) {
    if (!a) return fail(PP_EINVAL, "args is NULL");
    if (!a->netlist) return fail(PP_EINVAL, "netlist is NULL");
    if (a->density != PP_DENSITY_EXACT && a->density != PP_DENSITY_BINNED)
        return fail(PP_EINVAL, "unknown density %d", (int)a->density);
    const int64_t n = a->netlist->n_cells;
    if (n < 0 || a->netlist->n_nets < 0) return fail(PP_EINVAL, "negative netlist sizes");
    if (a->n_overflow < 0 || a->n_overflow > n)
        return fail(PP_EINVAL, "n_overflow=%lld outside [0, %lld]", (long long)a->n_overflow, (long long)n);
    pp_problem prob{a->W, a->H, n, a->vx, a->vy, a->w, a->h, a->c, a->M, a->M};
    L->dens_bytes = a->density == PP_DENSITY_EXACT ? pp_workspace_size(&prob, (pp_precision)a->prec)
                                                   : pp_binned_workspace_size(&prob, a->M);
    if (L->dens_bytes == 0) return PP_EINVAL;           // the size function said why
    L->wl_bytes = pp_wirelength_workspace_size(a->netlist->n_nets);
    L->vec_bytes = round256((size_t)n * sizeof(float));
    L->dens = 0;
    L->wl = round256(L->dens_bytes);
    L->vec = L->wl + round256(L->wl_bytes);
    L->norms = L->vec + 4 * L->vec_bytes;
    L->bins = L->norms + 256;
    L->total = L->bins + round256((size_t)a->M * (size_t)a->M * sizeof(float));
    return PP_OK;
}
}  // namespace

size_t pp_place_workspace_size(const pp_place_iteration_args *a) {
    PlaceLayout L{};
    return place_layout(a, &L) == PP_OK ? L.total : 0;
}

pp_status pp_place_iteration(const pp_place_iteration_args *a, void *ws, size_t ws_bytes, void *stream) {
    PlaceLayout L{};
    pp_status st = place_layout(a, &L);
    if (st != PP_OK) return st;
    if (!ws || ws_bytes < L.total)
        return fail(PP_ENOMEM_WS, "workspace of %zu bytes needed, %zu given", L.total, ws ? ws_bytes : (size_t)0);
    if (((uintptr_t)ws & 255) != 0) return fail(PP_EINVAL, "workspace must be 256-byte aligned");
    if (!a->stats || ((uintptr_t)a->stats & 7) != 0) return fail(PP_EINVAL, "stats must be 8-byte aligned device memory");
    // the scalars are checked here, before any step is issued (each step checks its
    // own device pointers before its launches); scalars on the device are read by the
    // kernels as they run and cannot be checked here
    const float *scal = a->scalars;
    if (scal) {
        if (((uintptr_t)scal & 15) != 0) return fail(PP_EINVAL, "scalars must be 16-byte aligned");
        int dev = 0, sm = 0, ccm = 0;
        unsigned *status;
        if ((st = device_info(&dev, &sm, &status, &ccm)) != PP_OK) return st;
        if ((st = check_dev_ptr(scal, dev, "scalars")) != PP_OK) return st;
    } else {
        if (!(std::isfinite(a->gamma) && a->gamma > 0.f)) return fail(PP_EINVAL, "gamma must be finite and > 0");
        if (!(std::isfinite(a->lambda) && a->lambda >= 0.f))
            return fail(PP_EINVAL, "lambda must be finite and >= 0");
        if (!(std::isfinite(a->alpha0) && a->alpha0 >= 0.f && std::isfinite(a->coef)))
            return fail(PP_EINVAL, "alpha0 must be finite and >= 0, coef finite");
    }
    if (!(std::isfinite(a->target) && a->target >= 0.f)) return fail(PP_EINVAL, "target must be finite and >= 0");
    if (a->M < 1 || a->M > 8192) return fail(PP_EINVAL, "M=%d must be in [1, 8192]", (int)a->M);
    const pp_netlist *nl = a->netlist;
    const int64_t n = nl->n_cells;
    unsigned char *base = (unsigned char *)ws;
    float *vec[4];
    for (int k = 0; k < 4; ++k) vec[k] = (float *)(base + L.vec + k * L.vec_bytes);
    float *gnx = vec[0], *gny = vec[1], *gx = vec[2], *gy = vec[3];
    double *norms = (double *)(base + L.norms);
    float *bins = (float *)(base + L.bins);
    double *stats = a->stats;

    pp_problem prob{a->W, a->H, n, a->vx, a->vy, a->w, a->h, a->c, a->M, a->M};
    if (a->density == PP_DENSITY_EXACT)
        st = pp_grad(&prob, (pp_precision)a->prec, PP_RECT, nullptr, gnx, gny, nullptr, stats + 3, base + L.dens,
                     L.dens_bytes, stream);
    else
        st = pp_binned_grad(&prob, (pp_precision)a->prec, a->M, nullptr, gnx, gny, nullptr, stats + 3,
                            base + L.dens, L.dens_bytes, stream);
    if (st != PP_OK) return st;
    // the wirelength's per-net pass, then one kernel for its per-cell gradient, the
    // combination and the step norms (the same values as pp_wirelength,
    // pp_place_combine and pp_step_norms; gw never leaves registers)
    if ((st = wirelength_impl(nl, a->vx, a->vy, a->gamma, scal, nullptr, nullptr, stats + 1, base + L.wl,
                              L.wl_bytes, stream)) != PP_OK)
        return st;
    {
        int dev = 0, sm = 0, ccm = 0;
        unsigned *status;
        if ((st = device_info(&dev, &sm, &status, &ccm)) != PP_OK) return st;
        if (n > 0) {
            const void *ptrs[6] = {a->q, a->vpx, a->vpy, a->gpx, a->gpy, a->vx};
            const char *names[6] = {"q", "vpx", "vpy", "gpx", "gpy", "vx"};
            if ((st = check_arrays(dev, 6, ptrs, names)) != PP_OK) return st;
            if (a->movable && (st = check_dev_ptr(a->movable, dev, "movable")) != PP_OK) return st;
        }
        cudaError_t e = launch_cell_step((int)n, nl->cell_ptr, nl->cell_net, a->vx, a->vy, a->gamma, a->lambda, scal,
                                         (const float *)(base + L.wl), gnx, gny, a->q, a->movable, a->vpx, a->vpy,
                                         a->gpx, a->gpy, gx, gy, norms, sm, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "cell step launch");
    }
    if ((st = nesterov_impl(n, a->W, a->H, a->ux, a->uy, a->vx, a->vy, a->vpx, a->vpy, gx, gy, a->gpx, a->gpy,
                            a->w, a->h, a->movable, norms, a->alpha0, a->coef, scal, stream)) != PP_OK)
        return st;
    pp_problem over{a->W, a->H, a->n_overflow, a->ux, a->uy, a->w, a->h, nullptr, 1, 1};
    return pp_overflow(&over, a->M, a->target, bins, stats, stream);
}

namespace {
// The graph objects of one pp_place_run, released on every path out of it.
struct LoopGraph {
    cudaStream_t cap = nullptr;         // capture stream (nothing runs on it)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool capturing = false;
    ~LoopGraph() {
        if (capturing) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(cap, &g);
            cudaGetLastError();
        }
        if (exec) cudaGraphExecDestroy(exec);   // freed once the launched graph has run
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
    }
};
}  // namespace

pp_status pp_place_run(const pp_place_iteration_args *a, const pp_place_schedule *sc, pp_place_state *state,
                       pp_place_record *trace, void *ws, size_t ws_bytes, void *stream) {
    PlaceLayout L{};
    pp_status st = place_layout(a, &L);
    if (st != PP_OK) return st;
    if (!sc) return fail(PP_EINVAL, "schedule is NULL");
    if (sc->max_iters < 1 || sc->max_iters > (1 << 24))
        return fail(PP_EINVAL, "max_iters=%d must be in [1, 2^24]", (int)sc->max_iters);
    if (!std::isfinite(sc->tau_stop)) return fail(PP_EINVAL, "tau_stop must be finite");
    if (!(std::isfinite(sc->bin_area) && sc->bin_area > 0 && std::isfinite(sc->area_mov) && sc->area_mov > 0 &&
          std::isfinite(sc->bin_w) && sc->bin_w > 0))
        return fail(PP_EINVAL, "bin_area, area_mov and bin_w must be finite and > 0");
    if (!state || ((uintptr_t)state & 15) != 0) return fail(PP_EINVAL, "state must be 16-byte aligned device memory");
    if (!trace || ((uintptr_t)trace & 7) != 0) return fail(PP_EINVAL, "trace must be 8-byte aligned device memory");
    if (!a->stats) return fail(PP_EINVAL, "stats is NULL");
    if (!ws || ws_bytes < L.total)
        return fail(PP_ENOMEM_WS, "workspace of %zu bytes needed, %zu given", L.total, ws ? ws_bytes : (size_t)0);
    if (((uintptr_t)ws & 255) != 0) return fail(PP_EINVAL, "workspace must be 256-byte aligned");
    int dev = 0, sm = 0, ccm = 0;
    unsigned *status;
    if ((st = device_info(&dev, &sm, &status, &ccm)) != PP_OK) return st;
    if ((st = check_dev_ptr(state, dev, "state")) != PP_OK) return st;
    if ((st = check_dev_ptr(trace, dev, "trace")) != PP_OK) return st;
    pp_place_iteration_args it = *a;
    it.scalars = reinterpret_cast<const float *>(reinterpret_cast<const unsigned char *>(state) +
                                                 offsetof(pp_place_state, scalars));   // inside the state
    it.alpha0 = 0.f;

    LoopGraph G;
    cudaError_t e = cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "capture stream");
    if ((e = cudaGraphCreate(&G.graph, 0)) != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
    cudaGraphConditionalHandle cond;
    if ((e = cudaGraphConditionalHandleCreate(&cond, G.graph, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
        return cuda_fail(e, "conditional handle");
    // the begin kernel: the graph's first node
    if ((e = cudaStreamBeginCaptureToGraph(G.cap, G.graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
        return cuda_fail(e, "capture (begin)");
    G.capturing = true;
    e = launch_place_loop_begin(state, sc->max_iters, cond, G.cap);
    G.capturing = false;
    cudaGraph_t got = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(G.cap, &got);
    if (e != cudaSuccess) return cuda_fail(e, "loop begin launch");
    if (e2 != cudaSuccess) return cuda_fail(e2, "capture (begin) end");
    cudaGraphNode_t first;
    size_t n_nodes = 1;
    if ((e = cudaGraphGetNodes(G.graph, &first, &n_nodes)) != cudaSuccess || n_nodes != 1)
        return e != cudaSuccess ? cuda_fail(e, "cudaGraphGetNodes") : fail(PP_ECUDA, "loop begin: %zu nodes", n_nodes);
    // the WHILE node after it; its body is one iteration and the step kernel
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    if ((e = cudaGraphAddNode(&loop, G.graph, &first, nullptr, 1, &cp)) != cudaSuccess)
        return cuda_fail(e, "conditional node");
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(G.cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
        return cuda_fail(e, "capture (body)");
    G.capturing = true;
    st = pp_place_iteration(&it, ws, ws_bytes, G.cap);
    if (st != PP_OK) return st;                 // ~LoopGraph ends the capture
    e = launch_place_loop_step(a->stats, state, trace, *sc, status, cond, G.cap);
    G.capturing = false;
    e2 = cudaStreamEndCapture(G.cap, &got);
    if (e != cudaSuccess) return cuda_fail(e, "loop step launch");
    if (e2 != cudaSuccess) return cuda_fail(e2, "capture (body) end");
    if ((e = cudaGraphInstantiate(&G.exec, G.graph, 0)) != cudaSuccess) return cuda_fail(e, "graph instantiate");
    if ((e = cudaGraphLaunch(G.exec, (cudaStream_t)stream)) != cudaSuccess) return cuda_fail(e, "graph launch");
    return PP_OK;
}

pp_status pp_check_wait_timeout(uint64_t limit_ns, void *stream) {
    int dev = 0, sm = 0, ccm = 0;
    unsigned *status;
    pp_status st = device_info(&dev, &sm, &status, &ccm);
    if (st != PP_OK) return st;
    if (ccm < 9) return fail(PP_ENOTSUP, "mbarrier waits need compute capability 9.0 or newer");
    if (limit_ns < 1000) limit_ns = 1000;
    if (limit_ns > 5000000000ull) limit_ns = 5000000000ull;
    cudaError_t e = launch_wait_probe(limit_ns, status, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "wait probe launch");
    return PP_OK;
}

const char *pp_last_error(void) { return t_err.c_str(); }

void pp_timing_enable(int on) { g_timing.store(on != 0); }

pp_status pp_timing_collect(int64_t *launches, double *ms) {
    std::lock_guard<std::mutex> lk(g_tmu);
    double acc[PP_K_COUNT] = {0, 0, 0, 0};
    for (size_t i = 0; i < g_tused; ++i) {
        TimedLaunch &t = g_tpool[i];
        cudaError_t e = cudaEventSynchronize(t.b);
        float v = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&v, t.a, t.b);
        if (e != cudaSuccess) {
            g_tused = 0;
            return cuda_fail(e, "timing event");
        }
        acc[t.kind] += v;
    }
    for (int k = 0; k < PP_K_COUNT; ++k) {
        const int64_t cnt = g_tcount[k].exchange(0, std::memory_order_relaxed);
        if (launches) launches[k] = cnt;
        if (ms) ms[k] = acc[k];
    }
    g_tused = 0;
    return PP_OK;
}

const char *pp_version(void) {
    return "pp 0.2 (sm_103a; FP32 CUDA-core path, tcgen05 TF32/BF16x3 paths)";
}

}  // extern "C"
