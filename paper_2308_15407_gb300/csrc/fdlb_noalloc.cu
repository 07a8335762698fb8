// fdlb_step_noalloc: the RK3 stepping entry point for callers that cannot allocate device
// memory (see include/fdlb.h).  All scratch -- tables, descriptors, work lists, the two
// intermediate RK buffers, per-node rows and projection table -- lives in one file-scope
// static device array; the caller passes only its distribution f (in/out) and an optional
// moments buffer.
#include "fdlb_ctx_internal.h"
#include "../../include/fdlb.h"

#include <cuda_runtime.h>

#include <mutex>
#include <string>

namespace {

// Held by every device that loads the library, until the process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[FDLB_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
constexpr int kMaxDevices = 256;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The symbol name is only a
// host-side stand-in; the address comes from cudaGetSymbolAddress, once per device.
int scratch_address(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        fdlb::set_global_error(std::string("fdlb_step_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return FDLB_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        fdlb::set_global_error("fdlb_step_noalloc: device index out of range");
        return FDLB_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            fdlb::set_global_error(std::string("fdlb_step_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return FDLB_ECUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return FDLB_OK;
}

}  // namespace

extern "C" int fdlb_step_noalloc(const fdlb_params* params, void* dev_f, size_t f_bytes, int64_t nsteps,
                                 double* dev_moments, void* stream) {
    if (!params || !dev_f || nsteps < 0) {
        fdlb::set_global_error("fdlb_step_noalloc: need params, dev_f and nsteps >= 0");
        return FDLB_EINVAL;
    }
    if (params->precision == FDLB_FP32_THEN_FP64) {
        fdlb::set_global_error("fdlb_step_noalloc: the two-phase precision form needs a context (fdlb_create)");
        return FDLB_EINVAL;
    }
    size_t need = fdlb_workspace_bytes(params, 1);
    if (need == 0) return FDLB_EINVAL;                     // message already set
    if (need > FDLB_NOALLOC_SCRATCH_BYTES) {
        fdlb::set_global_error("fdlb_step_noalloc: this instance needs " + std::to_string(need) +
                               " bytes of scratch, more than the static maximum of " +
                               std::to_string((size_t)FDLB_NOALLOC_SCRATCH_BYTES));
        return FDLB_ENOMEM;
    }
    void* ws = nullptr;
    int rc = scratch_address(&ws);
    if (rc) return rc;
    fdlb_ctx* c = nullptr;
    rc = fdlb_create(&c, params, 1, ws, FDLB_NOALLOC_SCRATCH_BYTES, stream);
    if (rc) return rc;
    fdlb_set_schedule(c, FDLB_SCHED_TILED);
    fdlb::ctx_direct_launches(c);
    cudaStream_t s = fdlb::ctx_stream(c);
    void* F = nullptr;
    size_t fb = 0;
    rc = fdlb::ctx_f_buffer(c, 0, &F, &fb);
    if (!rc && f_bytes != fb) {
        fdlb::set_global_error("fdlb_step_noalloc: f_bytes is " + std::to_string(f_bytes) + ", this instance's f has " +
                               std::to_string(fb) + " bytes");
        rc = FDLB_EINVAL;
    }
    auto cuda = [&](cudaError_t e, const char* what) {
        if (rc || e == cudaSuccess) return;
        fdlb::set_global_error(std::string("fdlb_step_noalloc: ") + what + ": " + cudaGetErrorString(e));
        rc = FDLB_ECUDA;
    };
    if (!rc) cuda(cudaMemcpyAsync(F, dev_f, fb, cudaMemcpyDeviceToDevice, s), "copy f in");
    if (!rc) rc = fdlb::ctx_reanchor(c, 0);
    if (!rc && nsteps > 0) rc = fdlb_step(c, nsteps, 0.0);
    if (!rc) cuda(cudaMemcpyAsync(dev_f, F, fb, cudaMemcpyDeviceToDevice, s), "copy f out");
    if (!rc && dev_moments) {
        const double* rows = nullptr;
        int ld = 0, nx = 0;
        rc = fdlb::ctx_moment_rows(c, 0, &rows, &ld, &nx);
        if (!rc) cuda(cudaMemcpy2DAsync(dev_moments, sizeof(double) * nx, rows, sizeof(double) * ld, sizeof(double) * nx, 8,
                                        cudaMemcpyDeviceToDevice, s), "copy moments out");
    }
    if (!rc) cuda(cudaStreamSynchronize(s), "synchronize");
    fdlb_destroy(c);
    return rc;
}
