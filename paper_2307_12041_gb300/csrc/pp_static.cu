// pp_grad_noalloc: the FP32 energy + gradient evaluation with its scratch in a
// fixed, file-scope device array instead of a caller-provided workspace.
//
// Who needs this: callers that cannot allocate device memory at the point where
// they evaluate the energy -- a host application that hands this library a
// fixed device budget at start-up and forbids allocation afterwards, a plugin
// called back from a tool that owns every allocation, or code running inside a
// region where an allocator call would break the caller's own bookkeeping.
// They still pass their own input and output arrays; only the scratch space
// (per-block records, the FP64 coefficient sums and the energy operand) lives
// here.
//
// The array below (PP_STATIC_SCRATCH_BYTES, about 5 MB) is reserved on a GPU
// when this file's CUDA module is loaded there and stays reserved until process
// exit.  The CUDA runtime loads modules lazily by default (CUDA_MODULE_LOADING
// = LAZY), and nothing in this module is used before the set-up below looks up
// the array's address, so in practice the first pp_grad_noalloc call on a
// device is the one that reserves it: a caller that fixes its device budget at
// start-up makes one call then (n = 0 does only the set-up).  All calls share
// the array: the contents of the previous call remain, so every part that must
// start at zero (the FP64 sums and *e_total) is cleared on the stream by the
// first kernel of each call, and two calls whose kernels overlap on the GPU
// (for example on two streams without ordering between them) race on it.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "pp.h"
#include "pp_device.cuh"
#include "pp_internal.h"

namespace pp {
namespace {

constexpr size_t kRecBytes = (size_t)PP_STATIC_MAX_BLOCKS * sizeof(AxisRec);
constexpr size_t kS64Bytes = (size_t)PP_STATIC_MAX_MODES * PP_STATIC_MAX_MODES * sizeof(double);
constexpr size_t kKBytes = (size_t)PP_STATIC_MAX_MODES * PP_STATIC_MAX_MODES * sizeof(float);
static_assert(PP_STATIC_MAX_MODES % kSimtKV == 0 && PP_STATIC_MAX_MODES % kSimtKU == 0,
              "padded FP32 operand must fit the static scratch");
static_assert(2 * kRecBytes + kS64Bytes + kKBytes == PP_STATIC_SCRATCH_BYTES,
              "scratch size stated in pp.h");

__device__ __align__(256) unsigned char g_scratch[PP_STATIC_SCRATCH_BYTES];

constexpr int kMaxDev = 64;
std::mutex g_mu;
unsigned char *g_scratch_ptr[kMaxDev];
int g_sms[kMaxDev];

pp_status err(pp_status st, const char *msg) {
    set_last_error(msg);
    return st;
}

// Set-up, once per device with that device current: the device address of the
// scratch array (in host code its name only denotes a host-side stand-in).
pp_status scratch_for_current_device(unsigned char **ptr, int *sms, int *dev) {
    if (cudaGetDevice(dev) != cudaSuccess || *dev < 0 || *dev >= kMaxDev) {
        cudaGetLastError();
        return err(PP_ECUDA, "pp_grad_noalloc: no current CUDA device");
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[*dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return err(PP_ECUDA, "pp_grad_noalloc: cudaGetSymbolAddress of the static scratch failed");
        }
        int v = 0;
        e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, *dev);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return err(PP_ECUDA, "pp_grad_noalloc: cudaDeviceGetAttribute failed");
        }
        g_sms[*dev] = v;
        g_scratch_ptr[*dev] = (unsigned char *)p;
    }
    *ptr = g_scratch_ptr[*dev];
    *sms = g_sms[*dev];
    return PP_OK;
}

pp_status device_array(const void *p, int dev, const char *what, size_t align) {
    if (((uintptr_t)p & (align - 1)) != 0) return err(PP_EINVAL, what);
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return err(PP_EINVAL, what);
    }
    if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != dev)
        return err(PP_EINVAL, what);
    return PP_OK;
}

}  // namespace
}  // namespace pp

using namespace pp;

extern "C" pp_status pp_grad_noalloc(const pp_problem *prob, pp_sample sample, float *gx, float *gy,
                                     float *e_block, double *e_total, void *stream) {
    if (!prob) return err(PP_EINVAL, "pp_grad_noalloc: problem is NULL");
    // the die range of pp_grad: 1/W and 1/H must be finite normal numbers for the
    // fixed-point phases
    if (!std::isfinite(prob->W) || !std::isfinite(prob->H) || !(prob->W >= 1e-300 && prob->W <= 1e300) ||
        !(prob->H >= 1e-300 && prob->H <= 1e300))
        return err(PP_EINVAL, "pp_grad_noalloc: die size W, H must be finite and in [1e-300, 1e300]");
    if (prob->n < 0 || prob->n > PP_STATIC_MAX_BLOCKS)
        return err(PP_EINVAL, "pp_grad_noalloc: n must be in [0, PP_STATIC_MAX_BLOCKS = 32768]");
    if (prob->Mx < 1 || prob->My < 1 || prob->Mx > PP_STATIC_MAX_MODES || prob->My > PP_STATIC_MAX_MODES)
        return err(PP_EINVAL, "pp_grad_noalloc: Mx and My must be in [1, PP_STATIC_MAX_MODES = 256]");
    if (sample != PP_RECT && sample != PP_CENTER)
        return err(PP_EINVAL, "pp_grad_noalloc: unknown sample mode");
    unsigned char *scratch = nullptr;
    int sms = 0, dev = 0;
    pp_status st = scratch_for_current_device(&scratch, &sms, &dev);
    if (st != PP_OK) return st;
    const bool blocks = prob->n > 0;
    if (blocks) {
        if (!prob->x || !prob->y || !prob->w || !prob->h || !gx || !gy)
            return err(PP_EINVAL, "pp_grad_noalloc: x, y, w, h, gx, gy must be non-NULL when n > 0");
        const void *arrays[8] = {prob->x, prob->y, prob->w, prob->h, prob->c, gx, gy, e_block};
        for (const void *a : arrays)
            if (a && (st = device_array(a, dev, "pp_grad_noalloc: every array must be 4-byte aligned "
                                                 "device memory of the current device", 4)) != PP_OK)
                return st;
    }
    if (e_total && (st = device_array(e_total, dev, "pp_grad_noalloc: e_total must be 8-byte "
                                                    "aligned device memory of the current device", 8)) != PP_OK)
        return st;

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
    L.xrec = (AxisRec *)scratch;
    L.yrec = (AxisRec *)(scratch + kRecBytes);
    L.S64 = (double *)(scratch + 2 * kRecBytes);
    L.K = scratch + 2 * kRecBytes + kS64Bytes;
    L.Kld = round_up(prob->My, kSimtKV);
    L.status = nullptr;
    L.sm_count = sms;
    L.stream = (cudaStream_t)stream;

    cudaError_t e = cudaSuccess;
    if (!blocks) {
        if (e_total) e = cudaMemsetAsync(e_total, 0, sizeof(double), L.stream);
    } else {
        // prep also zeroes the FP64 sums and *e_total left over from earlier calls
        e = launch_prep(L, true, e_total);
        if (e == cudaSuccess) e = launch_coeff_simt(L);
        if (e == cudaSuccess) e = launch_finish_simt(L, nullptr, nullptr);
        if (e == cudaSuccess) e = launch_energy_simt(L, (int)sample, e_block, e_total, gx, gy);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return err(PP_ECUDA, cudaGetErrorString(e));
    }
    return PP_OK;
}
