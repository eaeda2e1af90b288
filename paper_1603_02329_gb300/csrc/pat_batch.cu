// pat_batch.cu -- several independent instances (uneven grids, own media and sensors) as one
// launch.  Each instance's whole per-phase solve is captured once as a graph and becomes a child
// node of one parent graph with no edges between instances, so one cudaGraphLaunch runs every
// instance and the GPU overlaps their kernels.  The persistent kernels are never batched: they spin
// on grid barriers, and two such kernels are not guaranteed to be resident at the same time.
#include <cstring>
#include <vector>

#include "pat_host.h"

struct pat_batch {
    std::vector<pat_plan*> plans;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};   // forward, adjoint
    int device = 0;
};

namespace {

using namespace pat;

pat_status fail(pat_status s, const char* msg) {
    set_error(msg);
    return s;
}

pat_status build_exec(pat_batch* b, bool adjoint) {
    int slot = adjoint ? 1 : 0;
    if (b->exec[slot]) return PAT_OK;
    cudaGraph_t parent = nullptr;
    cudaError_t e = cudaGraphCreate(&parent, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
    for (pat_plan* p : b->plans) {
        cudaGraph_t child = nullptr;
        pat_status st = plan_capture_graph(p->impl, adjoint, &child);
        if (st != PAT_OK) {
            cudaGraphDestroy(parent);
            return st;
        }
        cudaGraphNode_t node;
        e = cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, child);   // copies `child`
        cudaGraphDestroy(child);
        if (e != cudaSuccess) {
            cudaGraphDestroy(parent);
            return cuda_fail(e, "cudaGraphAddChildGraphNode");
        }
    }
    e = cudaGraphInstantiate(&b->exec[slot], parent, 0);
    cudaGraphDestroy(parent);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate (batch)");
    return PAT_OK;
}

struct Guard {
    int prev = -1;
    explicit Guard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~Guard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != prev && prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

pat_status pat_batch_create(pat_plan* const* plans, int count, pat_batch** out) {
    set_error("");
    if (!plans || !out || count < 1) return fail(PAT_EINVAL, "bad batch arguments");
    *out = nullptr;
    auto* b = new pat_batch();
    for (int i = 0; i < count; ++i) {
        pat_plan* p = plans[i];
        if (!p) {
            delete b;
            return fail(PAT_EINVAL, "NULL plan in batch");
        }
        if (p->impl->arena) {
            delete b;
            return fail(PAT_EUNSUPPORTED, "static-arena plans cannot be batched");
        }
        for (pat_plan* q : b->plans)
            if (q == p) {
                delete b;
                return fail(PAT_EINVAL, "a plan appears twice in the batch");
            }
        if (i > 0 && p->impl->device != b->device) {
            delete b;
            return fail(PAT_EINVAL, "batched plans must live on one device");
        }
        if (i == 0) b->device = p->impl->device;
        b->plans.push_back(p);
    }
    *out = b;
    return PAT_OK;
}

pat_status pat_batch_destroy(pat_batch* b) {
    set_error("");
    if (!b) return PAT_OK;
    {
        Guard g(b->device);
        cudaDeviceSynchronize();
        for (cudaGraphExec_t& x : b->exec)
            if (x) cudaGraphExecDestroy(x);
    }
    delete b;
    return PAT_OK;
}

static pat_status batch_run(pat_batch* b, bool adjoint, const void* const* in, void* const* out, void* stream) {
    set_error("");
    if (!b || !in || !out) return fail(PAT_EINVAL, "NULL argument");
    Guard g(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    pat_status st = build_exec(b, adjoint);
    if (st != PAT_OK) return st;
    for (size_t i = 0; i < b->plans.size(); ++i) {
        PlanBase* p = b->plans[i]->impl;
        if (!in[i] || !out[i]) return fail(PAT_EINVAL, "NULL instance buffer");
        const size_t nimg = (size_t)p->info.N * p->elem, ndat = (size_t)p->info.Nt * p->info.Ns * p->elem;
        cudaError_t e = adjoint ? cudaMemcpyAsync(p->data_ptr, in[i], ndat, cudaMemcpyDefault, s)
                                : cudaMemcpyAsync(p->img_ptr, in[i], nimg, cudaMemcpyDefault, s);
        if (e != cudaSuccess) return cuda_fail(e, "batch input copy");
        if (!adjoint && p->smooth) {   // p^0 = S p0 (Sec. VI.A)
            st = plan_smooth(p, p->img_ptr, s);
            if (st != PAT_OK) return st;
        }
    }
    cudaError_t e = cudaGraphLaunch(b->exec[adjoint ? 1 : 0], s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch (batch)");
    for (size_t i = 0; i < b->plans.size() && adjoint; ++i) {   // (H S)^T = S H^T
        PlanBase* p = b->plans[i]->impl;
        if (!p->smooth) continue;
        st = plan_smooth(p, p->img_ptr, s);
        if (st != PAT_OK) return st;
    }
    for (size_t i = 0; i < b->plans.size(); ++i) {
        PlanBase* p = b->plans[i]->impl;
        const size_t nimg = (size_t)p->info.N * p->elem, ndat = (size_t)p->info.Nt * p->info.Ns * p->elem;
        e = adjoint ? cudaMemcpyAsync(out[i], p->img_ptr, nimg, cudaMemcpyDefault, s)
                    : cudaMemcpyAsync(out[i], p->data_ptr, ndat, cudaMemcpyDefault, s);
        if (e != cudaSuccess) return cuda_fail(e, "batch output copy");
    }
    return PAT_OK;
}

pat_status pat_batch_forward(pat_batch* b, const void* const* p0, void* const* data, void* stream) {
    return batch_run(b, false, p0, data, stream);
}

pat_status pat_batch_adjoint(pat_batch* b, const void* const* residual, void* const* grad, void* stream) {
    return batch_run(b, true, residual, grad, stream);
}

}  // extern "C"
