// pat_static.cu -- pat_forward_static: the forward operator for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc: an application that hands the whole device to its own
// pool allocator and forbids any other device allocation, or a long-running service that must
// not allocate (and risk fragmentation or an allocation failure) once it is in its steady state.
// This entry point runs the same kernels as pat_forward, but every device buffer (medium tables,
// state fields, spectrum workspaces, sensor lists, the data record) is carved from one fixed
// array that the library embeds as a device global.  It calls no cudaMalloc, no cudaFree and no
// allocating library routine, and it launches the kernels directly (no CUDA graph).
#include <mutex>
#include <string>

#include "pat_host.h"

// The scratch array: PAT_STATIC_SCRATCH_BYTES bytes in every GPU's memory for as long as the
// process has the library loaded.  Every call shares it and it keeps the last call's contents;
// the forward solve initialises everything it reads (the data record is cleared, the state is
// written before it is read), so no call depends on what an earlier one left behind.
static __device__ __align__(256) unsigned char g_pat_static_scratch[PAT_STATIC_SCRATCH_BYTES];

namespace pat {

static std::mutex g_static_mu;
static void* g_static_addr[64] = {};

// Device address of the scratch array on the current device.  In host code the array's name is
// only a host-side stand-in, so the address comes from cudaGetSymbolAddress, once per device,
// with that device current.
static pat_status static_scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) {
        set_error("device ordinal above 63");
        return PAT_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        // With lazy module loading (the default), this lookup is what loads the library's device
        // module on this GPU, and with it the array: the driver reserves the array's memory here.
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_pat_static_scratch);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            set_error("cudaGetSymbolAddress (static scratch): the device has no room left to load the "
                      "library's scratch array; make the first call at start-up, before a pool takes the memory");
            return PAT_ENOMEM;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress (static scratch)");
        g_static_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_static_addr[dev]);
    return PAT_OK;
}

}  // namespace pat

using namespace pat;

extern "C" pat_status pat_forward_static(const void* p0, const double* c, const double* rho, const double* alpha0,
                                         int alpha0_is_scalar, double y, const pat_grid* grid,
                                         const pat_sensors* sensor_mask, double dt, int Nt, pat_precision prec,
                                         void* data, void* stream) {
    set_error("");
    if (!p0 || !data) {
        set_error("NULL argument");
        return PAT_EINVAL;
    }
    HostTables h;
    pat_status st = build_tables(grid, c, rho, alpha0, alpha0_is_scalar, y, sensor_mask, dt, Nt, prec, h);
    if (st != PAT_OK) return st;
    unsigned char* arena = nullptr;
    st = static_scratch_address(&arena);
    if (st != PAT_OK) return st;
    PlanBase* plan = make_plan_arena(h, arena, (size_t)PAT_STATIC_SCRATCH_BYTES, &st);
    if (!plan) return st;
    // Building the plan wrote its tables with cudaMemcpy from pageable memory and cleared the
    // spectra with cudaMemset, both on the legacy default stream: either may still be in flight
    // when it returns.  The caller's stream may be a non-blocking one that does not order after
    // the legacy stream, so wait for that work here, before the first kernel reads it.
    cudaError_t e = cudaStreamSynchronize(cudaStreamLegacy);
    if (e != cudaSuccess) {
        delete plan;
        return cuda_fail(e, "cudaStreamSynchronize (plan set-up)");
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nimg = (size_t)h.info.N * plan->elem;
    const size_t ndat = (size_t)h.Nt * h.Ns * plan->elem;
    e = cudaMemcpyAsync(plan->img_ptr, p0, nimg, cudaMemcpyDefault, s);
    if (e != cudaSuccess) st = cuda_fail(e, "copy p0");
    if (st == PAT_OK) st = plan_clear_finite(plan, s);
    if (st == PAT_OK) st = plan_forward_direct(plan, s);
    if (st == PAT_OK) st = plan_finite_check(plan, false, s);
    if (st == PAT_OK) {
        e = cudaMemcpyAsync(data, plan->data_ptr, ndat, cudaMemcpyDefault, s);
        if (e != cudaSuccess) st = cuda_fail(e, "copy data");
    }
    e = cudaStreamSynchronize(s);
    if (st == PAT_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
    if (st == PAT_OK) {
        unsigned f = 0;
        e = cudaMemcpy(&f, plan->fstat, sizeof(f), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "read status word");
        else if (f != 0) {
            set_error("the data record holds NaN or infinite values");
            st = (pat_status)f;
        }
    }
    delete plan;
    return st;
}
