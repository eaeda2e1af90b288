// pat_host.h -- FP64 host tables of a plan (computed once, then rounded to the plan precision).
#pragma once

#include <complex>
#include <vector>

#include "pat_internal.cuh"

namespace pat {

struct HostTables {
    pat_plan_info_t info;
    int d = 2, nx = 1, ny = 1, nz = 1, nxh = 1, ldh = 1;
    long long N = 0;
    int Ns = 0, Nt = 0, lossy = 0;
    double dt = 0.0, c_ref = 0.0;
    LaunchCfg cfg{};

    std::vector<double> c2, rho0, b[3], c2tau, c2eta;
    std::vector<double> a[3], au[3];
    std::vector<std::complex<double>> dp[3], dm[3], tw[3];
    std::vector<double> kv[3];
    double kap_a = 0.0, pha = 0.0, phb = 0.0, invN = 0.0;
    FftAxis fx{}, fy{}, fz{};

    // sensors (see DevSensors)
    std::vector<int> g_lineptr, g_seg_line, g_seg_sensor, g_seg_x0;
    std::vector<double> g_seg_w0, g_seg_w1;
    std::vector<int> s_lineptr, s_seg_line, s_seg_x, s_seg_e0, s_ent_sensor;
    std::vector<double> s_ent_w;
};

PlanBase* make_plan_f32(const HostTables& h, pat_status* st);
PlanBase* make_plan_f64(const HostTables& h, pat_status* st);
pat_status plan_capture(PlanBase* base, bool adjoint);
pat_status plan_capture_graph(PlanBase* base, bool adjoint, cudaGraph_t* out);
pat_status plan_run_persistent(PlanBase* base, bool adjoint, cudaStream_t s);
// x <- S x (the p0 smoothing of Sec. VI.A) in place, x a device field of the plan's precision
pat_status plan_smooth(PlanBase* base, void* x, cudaStream_t s);
// allocate the smoothing workspace (no-op when present)
pat_status plan_smooth_alloc(PlanBase* base);
// zero the plan's non-finite flag / scan the solve's output (data after H, image after H^T) into it
pat_status plan_clear_finite(PlanBase* base, cudaStream_t s);
pat_status plan_finite_check(PlanBase* base, bool adjoint, cudaStream_t s);
pat_status plan_set_fault(PlanBase* base, unsigned barrier_extra, double wait_limit_s);
pat_status plan_gradient_medium(PlanBase* base, const void* p0, const void* h, void* gc2, void* grho, void* gp0,
                                int K, cudaStream_t s);
pat_status plan_time_reversal(PlanBase* base, const void* data, void* img, int compensate, double k_cut,
                              cudaStream_t s);
pat_status plan_adjoint_atd(PlanBase* base, const void* resid, void* img, int initial_paper, cudaStream_t s);
PlanBase* make_plan_arena(const HostTables& h, unsigned char* arena, size_t cap, pat_status* st);
pat_status plan_forward_direct(PlanBase* base, cudaStream_t s);
pat_status build_tables(const pat_grid* grid, const double* c, const double* rho, const double* alpha0,
                        int alpha0_is_scalar, double y, const pat_sensors* sensors, double dt, int Nt,
                        pat_precision prec, HostTables& h);
pat_status plan_probe_read(PlanBase* b, int g, int slot, const char** name, double* mean_ms, int* samples);

}  // namespace pat
