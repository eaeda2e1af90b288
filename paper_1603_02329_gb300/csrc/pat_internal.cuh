// pat_internal.cuh -- types shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pat.h"

namespace pat {

// ------------------------------------------------------------------------------------------
// complex helpers (float2 / double2 storage)
// ------------------------------------------------------------------------------------------
template <typename T> struct CT;
template <> struct CT<float> { typedef float2 type; };
template <> struct CT<double> { typedef double2 type; };

template <typename T> using cplx = typename CT<T>::type;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mkc(T a, T b) {
    cplx<T> r;
    r.x = a;
    r.y = b;
    return r;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// a * conj(b)
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
    C r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.y * b.x - a.x * b.y;
    return r;
}
template <typename C, typename T> __host__ __device__ __forceinline__ C cscale(C a, T s) { a.x *= s; a.y *= s; return a; }

// ------------------------------------------------------------------------------------------
// FFT description of one axis (Stockham autosort, radices 2,3,4,5,7,8)
// ------------------------------------------------------------------------------------------
constexpr int kMaxStages = 16;
struct FftAxis {
    int n;
    int nst;
    int rad[kMaxStages];
    int pow2;              // n is a power of two: every index operation is a shift or a mask
    int lgn;               // log2(n) when pow2
    int lgr[kMaxStages];   // log2(rad[s]) when pow2
};

// Maximum line length handled by the shared-memory FFT.
constexpr int kMaxFftLen = 1024;

// ------------------------------------------------------------------------------------------
// Sensor lists, grouped by grid line (x-line index = z * Ny + y)
// ------------------------------------------------------------------------------------------
template <typename T> struct DevSensors {
    int Ns;
    // forward gather: segments grouped by (line, sensor); weights w0 at x0 and w1 at x0 + 1
    // (w1 = 0 for a single entry); one atomic add per segment
    const int* g_lineptr;   // [nlines + 1] -> segment range
    const int* g_seg_line;  // [nseg]
    const int* g_seg_sensor;
    const int* g_seg_x0;
    const T* g_seg_w0;
    const T* g_seg_w1;
    // adjoint scatter: segments grouped by (line, x); entries (sensor, weight)
    const int* s_lineptr;
    const int* s_seg_line;
    const int* s_seg_x;
    const int* s_seg_e0;
    const int* s_ent_sensor;
    const T* s_ent_w;
};

// ------------------------------------------------------------------------------------------
// Device-side view of a plan: passed by value to every kernel
// ------------------------------------------------------------------------------------------
template <typename T> struct DevPlan {
    int d;            // 2 or 3
    int nx, ny, nz;   // nz = 1 in 2-D
    int nxh;          // nx/2 + 1 (half spectrum along x)
    int ldh;          // row pitch of half-spectrum arrays (complex elements, >= nxh)
    int nlines;       // ny * nz x-lines
    long long N;      // nx * ny * nz
    int lossy;
    int Nt;
    T dt;

    // medium (N each)
    const T* c2;
    const T* rho0;
    const T* b[3];    // 1/rho0 at r + dx_xi / 2
    const T* c2tau;   // c0^2 tau  (lossy only)
    const T* c2eta;   // c0^2 eta  (lossy only)
    // PML factors per axis: a at normal points, au at staggered points
    const T* a[3];
    const T* au[3];
    // k-space: per-axis wavenumbers and staggered derivative symbols i k e^{+-i k dx/2}
    // (x: half spectrum 0..nx/2; y, z: full); kappa and |k|^s are evaluated from these
    const T* kv[3];
    const cplx<T>* dp[3];
    const cplx<T>* dm[3];
    T kap_a;          // c_ref dt / 2  (kappa = sinc(kap_a |k|))
    T pha, phb;       // (y - 2) / 2, (y - 1) / 2: exponents applied to |k|^2
    T invN;           // 1 / N (inverse-transform scaling)
    // FFT plans and twiddles exp(-2 pi i m / n) per axis
    FftAxis fx, fy, fz;
    const cplx<T>* twx;
    const cplx<T>* twy;
    const cplx<T>* twz;
    // per-stage twiddle tables of the power-of-two schedule (p2_stage_table; 2 n entries per axis,
    // nullptr where the axis is not a power of two of 16 .. 2048 points)
    const cplx<T>* stw[3];
    int fixed_len;    // 1: launch the kernels compiled for this plan's line lengths where they exist
    // per-stage twiddle tables of the two-stage schedule of 128- and 256-point lines (radices n/16
    // and 16; p2x_stage_table), nullptr elsewhere; spec16: which 3-D spectral passes use it
    // (0 none, 1 the plain transforms, 2 the fused multiply passes as well)
    const cplx<T>* stw16[3];
    int spec16;

    // state and workspaces (N each unless noted)
    T* u[3];
    T* rh[3];
    T* rsum;          // r = sum rho_xi (forward, lossy)
    T* pbar;          // adjoint pressure (lossy)
    cplx<T>* spec[3]; // half-spectrum workspaces [nz][ny][ldh]
    T* img;           // p0 in / gradient out
    T* data;          // [Nt][Ns]

    DevSensors<T> sens;

    // Hooks of the density-gradient sweep (readings D2-D3; nullptr = off, the default):
    //   forward: fwd_u stores g_xi = D+_xi p^n into hk_g[xi], fwd_rho stores e_xi = D-_xi u_xi^{n+1/2}
    //            into hk_e[xi] (the recomputed step's fields);
    //   adjoint: adj_rho (lossy) and the lossless adjoint tail add sum_xi e_xi (dd_bar - dt a rho_bar_xi)
    //            to hk_grho, with e_xi read from hk_ein[xi]; adj_u adds u_bar_xi (-dt au g_xi) to
    //            hk_gb[xi] (dJ/db_xi), g_xi read from hk_gin[xi], and on the final level also
    //            u_bar_xi^{-1/2} (dt/2) g_xi (the transpose of u^{-1/2} = (dt/2) b D+ p0).
    T* hk_g[3];
    T* hk_e[3];
    const T* hk_gin[3];
    const T* hk_ein[3];
    T* hk_grho;
    T* hk_gb[3];

    // Hooks of the time-reversal solve (Sec. II.B.1, readings T1-T5; off by default):
    //   tr_kc2 > 0: the absorption multiplier |k|^(y-2) becomes -W(|k| / k_c) |k|^(y-2), the reversed
    //     and band-limited absorption term (W the radial Blackman window, tr_kc2 = 1 / k_c^2);
    //   tr_node [N]: the sensor enforced at each node (-1: none); after the step the pressure there is
    //     set to tr_row[sensor] and the split densities to tr_row[sensor] / (d c0^2);
    //   tr_img: the pressure of the step launched with the last-step flag is stored there.
    T tr_kc2;
    const int* tr_node;
    const T* tr_row;
    T* tr_img;
    // Adjoint-then-discretize solve (Sec. III Eqs. (moma), (massa), (statea); readings A1-A2; atd = 1):
    // the mass update takes the source dt rho0 s / d with s = M^T atd_row, and tau, eta act before the
    // fractional Laplacians: (dd, r) = (c0^2 tau (s - sum e), c0^2 eta sum rho / rho0) and
    // p = c0^2 sum rho - rho0 L_{y-2} dd - rho0 L_{y-1} r.
    int atd;
    const T* atd_row;
    // first column tile of a spectral launch (blockIdx.x + tile0 is the tile): a 3-D spectral operation
    // may run its y / z / y passes chunk by chunk over the column tiles (0 = the whole range at once)
    int tile0;
    // Tensor-memory-access staging of the 3-D spectral tiles (8 columns): tmaps holds the tensor maps
    // of the half spectra spec[0..2] for y-pass tiles (boxes of 8 columns x ny lines) at [0..2] and for
    // z-pass tiles (8 columns x nz lines) at [3..5], in device memory; use_tma = 0 stages with cp.async.
    // fault: the plan's status word, set to PAT_ETIMEOUT when a bounded wait for a tile runs out.
    const void* tmaps;
    int use_tma;
    unsigned* fault;

    // phase-timeline trace of the persistent kernel (nullptr = off): globaltimer at entry and
    // exit of grid barriers trace_k0 .. trace_k0 + trace_nk - 1, per CTA
    unsigned long long* trace;
    int trace_k0, trace_nk;
    // grid-barrier wait bound of the persistent kernels and the test hook that makes it run out:
    // every barrier waits for bar_extra more arrivals than exist (0 in normal runs)
    unsigned bar_extra;
    unsigned long long bar_limit_ns;
};

// ------------------------------------------------------------------------------------------
// Host-side plan
// ------------------------------------------------------------------------------------------
struct LaunchCfg {
    int row_lines;    // x-lines per CTA in row kernels (even)
    int row_threads;
    int col_w;        // columns per CTA in strided-axis kernels
    int col_threads;
};

// the arguments a plan was created from (kept on the host to build coarser levels)
struct PlanInputs {
    pat_grid grid{};
    std::vector<double> c, rho, alpha0;
    int alpha0_is_scalar = 0;
    double y = 1.5, dt = 0.0;
    int Nt = 0;
    std::vector<double> pos;       // [Ns][ndim] or empty
    std::vector<int64_t> index;    // [Ns] or empty
    int Ns = 0;
    pat_precision prec = PAT_F32;
};

struct PlanBase {
    virtual ~PlanBase() {}
    PlanInputs in;
    pat_plan_info_t info;
    int device = 0;
    LaunchCfg cfg;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t fwd_exec = nullptr;
    cudaGraphExec_t adj_exec = nullptr;
    std::vector<void*> allocs;   // every device allocation owned by the plan
    // kernel-timing probe: events around the launches of sampled steps
    int probe_stride = 0;
    std::vector<cudaEvent_t> probe_ev[2];          // [graph][sample * (slots + 1) + k]
    std::vector<std::string> probe_names[2];       // slot names of one step
    int probe_samples[2] = {0, 0};
    // When `arena` is set, every device buffer of the plan is carved from that caller-provided
    // region instead of cudaMalloc, and the plan owns no stream or graph (direct launches only).
    unsigned char* arena = nullptr;
    size_t arena_cap = 0, arena_used = 0;
    void* img_ptr = nullptr;
    void* data_ptr = nullptr;
    size_t elem = 4;
    // persistent single-kernel path (2-D): grid size, barrier/status words [count, -, status, -]
    int persistent = 0;
    int persist_grid = 0;
    size_t persist_smem = 0;
    unsigned* gbar = nullptr;
    // non-finite check of the last solve's output: 0, or PAT_ENONFINITE (zeroed before each solve)
    unsigned* fstat = nullptr;
    // 1: the initial pressure is smoothed, p^0 = S p0, and the adjoint ends with S (Sec. VI.A)
    int smooth = 0;
    unsigned long long* trace = nullptr;
    int trace_k0 = 0, trace_nk = 0;
};

// error reporting (thread-local message)
void set_error(const std::string& msg);
pat_status cuda_fail(cudaError_t e, const char* what);

}  // namespace pat

struct pat_plan {
    pat::PlanBase* impl;
};
