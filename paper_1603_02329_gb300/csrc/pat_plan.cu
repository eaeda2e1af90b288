// pat_plan.cu -- FP64 host precompute of a plan and the C ABI entry points of pat.h.
//
// Everything derived from the medium and geometry is computed here once, in FP64:
//   c0^2, 1/rho0 on the staggered grids, tau and eta of Sec. II.A Eq. (Twelve) (alpha0 converted
//   from dB MHz^-y cm^-1 to Np m^-1 (rad/s)^-y), PML damping factors (Sec. VI.A: P points,
//   alpha_pml Np per point at the edge, profile (depth/P)^4), k-space symbols (staggered
//   derivatives i k exp(+-i k dx/2), kappa = sinc(c_ref |k| dt / 2), |k|^(y-2), |k|^(y-1)),
//   FFT twiddles and radix plans, and the sensor interpolation lists (Sec. III, Sec. VI.A).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <tuple>

#include "pat_host.h"

namespace pat {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

pat_status cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? PAT_ENOMEM : PAT_ECUDA;
}

static pat_status fail(pat_status s, const std::string& msg) {
    set_error(msg);
    return s;
}

// Radix plan for the Stockham FFT: 8s first, then 4, 2, 3, 5, 7.
static bool factor_axis(int n, FftAxis* ax) {
    ax->n = n;
    ax->nst = 0;
    int m = n;
    const int order[] = {8, 4, 2, 3, 5, 7};
    for (int r : order) {
        while (m % r == 0) {
            if (ax->nst >= kMaxStages) return false;
            ax->rad[ax->nst++] = r;
            m /= r;
        }
    }
    if (m != 1) return false;
    ax->pow2 = (n & (n - 1)) == 0;
    ax->lgn = 0;
    while ((1 << ax->lgn) < n) ++ax->lgn;
    for (int s = 0; s < ax->nst; ++s) {
        int l = 0;
        while ((1 << l) < ax->rad[s]) ++l;
        ax->lgr[s] = l;
    }
    return true;
}

static std::vector<std::complex<double>> twiddles(int n) {
    std::vector<std::complex<double>> t(n);
    for (int m = 0; m < n; ++m) {
        const double ang = 2.0 * M_PI * (double)m / (double)n;
        t[m] = std::complex<double>(std::cos(ang), -std::sin(ang));
    }
    return t;
}

// wavenumber of FFT bin m on an axis of n points, spacing h; Nyquist (m = n/2) positive
static double kbin(int m, int n, double h) {
    const int mm = (m > n / 2) ? m - n : m;
    return 2.0 * M_PI * (double)mm / ((double)n * h);
}

// PML damping factors (normal and staggered points) of one axis
static void pml_axis(int n, int P, double alpha, double c_ref, double h, double dt, std::vector<double>& a,
                     std::vector<double>& au) {
    a.assign(n, 1.0);
    au.assign(n, 1.0);
    if (P <= 0) return;
    auto sigma = [&](double pos) {
        double depth = std::max(std::max((double)P - pos, pos - (double)(n - 1 - P)), 0.0);
        double q = depth / (double)P;
        return alpha * (c_ref / h) * q * q * q * q;
    };
    for (int i = 0; i < n; ++i) {
        a[i] = std::exp(-sigma((double)i) * dt / 2.0);
        au[i] = std::exp(-sigma((double)i + 0.5) * dt / 2.0);
    }
}

struct SensorEntry {
    int line, x, sensor;
    double w;
};

static pat_status sensor_entries(const pat_grid& g, const pat_sensors& s, std::vector<SensorEntry>& out) {
    const int nx = g.n[0], ny = g.n[1], nz = (g.ndim == 3) ? g.n[2] : 1;
    const long long N = (long long)nx * ny * nz;
    out.clear();
    if (s.index) {
        for (int j = 0; j < s.count; ++j) {
            const long long idx = s.index[j];
            if (idx < 0 || idx >= N) return fail(PAT_EINVAL, "sensor index outside the grid");
            out.push_back({(int)(idx / nx), (int)(idx % nx), j, 1.0});
        }
        return PAT_OK;
    }
    const int d = g.ndim;
    for (int j = 0; j < s.count; ++j) {
        int i0[3] = {0, 0, 0};
        double t[3] = {0, 0, 0};
        int nc[3] = {1, 1, 1};
        for (int a = 0; a < d; ++a) {
            const double f = s.pos[(size_t)j * d + a] / g.dx[a] + (double)(g.n[a] / 2);
            if (!std::isfinite(f)) return fail(PAT_EINVAL, "non-finite sensor position");
            i0[a] = (int)std::floor(f);
            t[a] = f - (double)i0[a];
            nc[a] = (t[a] != 0.0) ? 2 : 1;
            if (i0[a] < 0 || i0[a] + nc[a] - 1 >= g.n[a]) return fail(PAT_EINVAL, "sensor position outside the grid");
        }
        for (int cz = 0; cz < nc[2]; ++cz)
            for (int cy = 0; cy < nc[1]; ++cy)
                for (int cx = 0; cx < nc[0]; ++cx) {
                    double w = (cx ? t[0] : 1.0 - t[0]) * (cy ? t[1] : 1.0 - t[1]);
                    if (d == 3) w *= (cz ? t[2] : 1.0 - t[2]);
                    if (w == 0.0) continue;
                    const int ix = i0[0] + cx, iy = i0[1] + cy, iz = (d == 3) ? i0[2] + cz : 0;
                    out.push_back({iz * ny + iy, ix, j, w});
                }
    }
    return PAT_OK;
}

static void build_sensor_lists(std::vector<SensorEntry> e, int nlines, HostTables& h) {
    // gather: segments by (line, sensor), weights at x0 and x0 + 1
    std::sort(e.begin(), e.end(), [](const SensorEntry& a, const SensorEntry& b) {
        return std::tie(a.line, a.sensor, a.x) < std::tie(b.line, b.sensor, b.x);
    });
    h.g_seg_line.clear();
    h.g_seg_sensor.clear();
    h.g_seg_x0.clear();
    h.g_seg_w0.clear();
    h.g_seg_w1.clear();
    for (size_t k = 0; k < e.size();) {
        h.g_seg_line.push_back(e[k].line);
        h.g_seg_sensor.push_back(e[k].sensor);
        h.g_seg_x0.push_back(e[k].x);
        h.g_seg_w0.push_back(e[k].w);
        if (k + 1 < e.size() && e[k + 1].line == e[k].line && e[k + 1].sensor == e[k].sensor &&
            e[k + 1].x == e[k].x + 1) {
            h.g_seg_w1.push_back(e[k + 1].w);
            k += 2;
        } else {
            h.g_seg_w1.push_back(0.0);
            k += 1;
        }
    }
    h.g_lineptr.assign(nlines + 1, 0);
    {
        size_t s = 0;
        for (int l = 0; l <= nlines; ++l) {
            while (s < h.g_seg_line.size() && h.g_seg_line[s] < l) ++s;
            h.g_lineptr[l] = (int)s;
        }
    }
    // scatter: segments by (line, x)
    std::sort(e.begin(), e.end(), [](const SensorEntry& a, const SensorEntry& b) {
        return std::tie(a.line, a.x, a.sensor) < std::tie(b.line, b.x, b.sensor);
    });
    h.s_seg_line.clear();
    h.s_seg_x.clear();
    h.s_seg_e0.clear();
    h.s_ent_sensor.clear();
    h.s_ent_w.clear();
    for (size_t k = 0; k < e.size(); ++k) {
        if (k == 0 || e[k].line != e[k - 1].line || e[k].x != e[k - 1].x) {
            h.s_seg_line.push_back(e[k].line);
            h.s_seg_x.push_back(e[k].x);
            h.s_seg_e0.push_back((int)k);
        }
        h.s_ent_sensor.push_back(e[k].sensor);
        h.s_ent_w.push_back(e[k].w);
    }
    h.s_seg_e0.push_back((int)e.size());
    h.s_lineptr.assign(nlines + 1, 0);
    {
        size_t s = 0;
        for (int l = 0; l <= nlines; ++l) {
            while (s < h.s_seg_line.size() && h.s_seg_line[s] < l) ++s;
            h.s_lineptr[l] = (int)s;
        }
    }
}

pat_status build_tables(const pat_grid* grid, const double* c, const double* rho, const double* alpha0,
                               int alpha0_is_scalar, double y, const pat_sensors* sensors, double dt, int Nt,
                               pat_precision prec, HostTables& h) {
    if (!grid || !c || !rho || !alpha0 || !sensors) return fail(PAT_EINVAL, "NULL argument");
    const pat_grid& g = *grid;
    if (g.ndim != 2 && g.ndim != 3) return fail(PAT_EINVAL, "ndim must be 2 or 3");
    if (prec != PAT_F32 && prec != PAT_F64) return fail(PAT_EINVAL, "bad precision");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(PAT_EINVAL, "dt must be positive");
    if (Nt < 1) return fail(PAT_EINVAL, "Nt must be >= 1");
    const int d = g.ndim;
    for (int a = 0; a < d; ++a) {
        if (g.n[a] < 2 || (g.n[a] & 1)) return fail(PAT_EUNSUPPORTED, "grid sizes must be even and >= 2");
        if (g.n[a] > kMaxFftLen) return fail(PAT_EUNSUPPORTED, "grid size above the FFT line limit (1024)");
        if (!(g.dx[a] > 0.0)) return fail(PAT_EINVAL, "dx must be positive");
        if (g.pml[a] < 0 || 2 * g.pml[a] > g.n[a]) return fail(PAT_EINVAL, "bad PML thickness");
    }
    if (!(g.pml_alpha >= 0.0)) return fail(PAT_EINVAL, "pml_alpha must be >= 0");
    if (sensors->count < 1) return fail(PAT_EINVAL, "need at least one sensor");
    if ((sensors->pos == nullptr) == (sensors->index == nullptr)) return fail(PAT_EINVAL, "give exactly one of sensor pos / index");

    h.d = d;
    h.nx = g.n[0];
    h.ny = g.n[1];
    h.nz = (d == 3) ? g.n[2] : 1;
    h.nxh = h.nx / 2 + 1;
    h.ldh = (h.nxh + 7) / 8 * 8;
    h.N = (long long)h.nx * h.ny * h.nz;
    // the kernels index fields and records with 32-bit offsets in places: these limits keep every
    // flat index of a field (and of a complex half spectrum) or of the record below 2^31
    if (h.N > (1LL << 27)) return fail(PAT_EUNSUPPORTED, "grid above 2^27 points (512^3)");
    if ((long long)Nt * sensors->count > 0x7fffffffLL) return fail(PAT_EUNSUPPORTED, "Nt * Ns above 2^31 - 1");
    h.Nt = Nt;
    h.Ns = sensors->count;
    h.dt = dt;
    const size_t N = (size_t)h.N;
    const int n3[3] = {h.nx, h.ny, h.nz};
    const double h3[3] = {g.dx[0], g.dx[1], d == 3 ? g.dx[2] : 1.0};
    const int p3[3] = {g.pml[0], g.pml[1], d == 3 ? g.pml[2] : 0};

    // medium
    double cmax = 0.0;
    bool lossy = false;
    for (size_t i = 0; i < N; ++i) {
        if (!(c[i] > 0.0) || !std::isfinite(c[i])) return fail(PAT_EINVAL, "sound speed must be positive");
        if (!(rho[i] > 0.0) || !std::isfinite(rho[i])) return fail(PAT_EINVAL, "density must be positive");
        const double a0 = alpha0_is_scalar ? alpha0[0] : alpha0[i];
        if (!(a0 >= 0.0) || !std::isfinite(a0)) return fail(PAT_EINVAL, "alpha0 must be >= 0");
        if (a0 != 0.0) lossy = true;
        cmax = std::max(cmax, c[i]);
    }
    if (lossy && (std::fabs(y - 1.0) < 1e-9 || !std::isfinite(y) || y <= 0.0 || y >= 3.0))
        return fail(PAT_EINVAL, "power-law exponent y must be in (0, 3) and != 1");
    h.lossy = lossy ? 1 : 0;
    h.c_ref = cmax;
    h.c2.resize(N);
    h.rho0.assign(rho, rho + N);
    for (size_t i = 0; i < N; ++i) h.c2[i] = c[i] * c[i];
    const size_t stride3[3] = {1, (size_t)h.nx, (size_t)h.nx * h.ny};
    for (int a = 0; a < d; ++a) {
        h.b[a].resize(N);
        for (size_t i = 0; i < N; ++i) {
            // neighbour at +1 along axis a, periodic
            const size_t coord = (i / stride3[a]) % (size_t)n3[a];
            const size_t j = (coord + 1 == (size_t)n3[a]) ? i - coord * stride3[a] : i + stride3[a];
            h.b[a][i] = 2.0 / (rho[i] + rho[j]);
        }
    }
    if (lossy) {
        // dB MHz^-y cm^-1 -> Np m^-1 (rad/s)^-y
        const double db_per_np = 20.0 * std::log10(std::exp(1.0));
        const double conv = 100.0 / db_per_np * std::pow(2.0 * M_PI * 1e6, -y);
        const double tn = std::tan(M_PI * y / 2.0);
        h.c2tau.resize(N);
        h.c2eta.resize(N);
        for (size_t i = 0; i < N; ++i) {
            const double a0 = (alpha0_is_scalar ? alpha0[0] : alpha0[i]) * conv;
            const double tau = -2.0 * a0 * std::pow(c[i], y - 1.0);
            const double eta = 2.0 * a0 * std::pow(c[i], y) * tn;
            h.c2tau[i] = h.c2[i] * tau;
            h.c2eta[i] = h.c2[i] * eta;
        }
    }
    // PML
    for (int a = 0; a < 3; ++a) {
        if (a < d) pml_axis(n3[a], p3[a], g.pml_alpha, cmax, h3[a], dt, h.a[a], h.au[a]);
        else {
            h.a[a].assign(1, 1.0);
            h.au[a].assign(1, 1.0);
        }
    }
    // k-space symbols
    const int klen[3] = {h.nxh, h.ny, h.nz};
    for (int a = 0; a < 3; ++a) {
        h.dp[a].resize(klen[a]);
        h.dm[a].resize(klen[a]);
        for (int m = 0; m < klen[a]; ++m) {
            const double k = (a < d) ? kbin(m, n3[a], h3[a]) : 0.0;
            const double hh = (a < d) ? h3[a] : 0.0;
            const double sn = std::sin(0.5 * k * hh), cs = std::cos(0.5 * k * hh);
            h.dp[a][m] = std::complex<double>(-k * sn, k * cs);  // i k e^{+i k h/2}
            h.dm[a][m] = std::complex<double>(k * sn, k * cs);   // i k e^{-i k h/2}
        }
    }
    for (int a = 0; a < 3; ++a) {
        h.kv[a].resize(klen[a]);
        for (int m = 0; m < klen[a]; ++m) h.kv[a][m] = (a < d) ? kbin(m, n3[a], h3[a]) : 0.0;
    }
    h.kap_a = cmax * dt / 2.0;
    h.pha = (y - 2.0) / 2.0;
    h.phb = (y - 1.0) / 2.0;
    h.invN = 1.0 / (double)h.N;
    // FFT plans
    if (!factor_axis(h.nx, &h.fx) || !factor_axis(h.ny, &h.fy) || !factor_axis(h.nz, &h.fz))
        return fail(PAT_EUNSUPPORTED, "FFT lengths must factor into 2, 3, 5, 7");
    h.tw[0] = twiddles(h.nx);
    h.tw[1] = twiddles(h.ny);
    h.tw[2] = twiddles(h.nz);
    // sensors
    std::vector<SensorEntry> ents;
    pat_status st = sensor_entries(g, *sensors, ents);
    if (st != PAT_OK) return st;
    build_sensor_lists(ents, h.ny * h.nz, h);
    // launch configuration
    h.cfg.row_lines = 2;
    h.cfg.row_threads = 128;
    h.cfg.col_threads = 256;
    const size_t cbytes = (prec == PAT_F32) ? 8 : 16;
    const int L = std::max(h.ny, h.nz);
    // columns per spectral CTA: 16-byte rows (2 complex floats or 1 complex double) keep more
    // CTAs in flight on small grids; overridable for tuning
    int w = (prec == PAT_F32) ? 2 : 1;
    if (const char* env = std::getenv("PAT_COL_W")) w = std::max(1, std::atoi(env));
    int p2 = 1;
    while (p2 * 2 <= w && p2 < 8) p2 *= 2;   // a power of two, at most 8
    w = p2;
    while (w > 1 && (size_t)(3 * L + 16 + 3 * d * L * w) * cbytes > 180 * 1024) w /= 2;
    h.cfg.col_w = w;
    // threads: one radix-8 butterfly per thread for the widest interleaved batch (d W lines)
    h.cfg.col_threads = std::min(256, std::max(64, (d * w * L / 8 + 31) / 32 * 32));
    if (const char* env = std::getenv("PAT_ROW_LINES")) {
        const int r = std::atoi(env);
        if (r >= 2 && r % 2 == 0 && (h.ny * h.nz) % r == 0) h.cfg.row_lines = r;
    }
    // info
    pat_plan_info_t& inf = h.info;
    std::memset(&inf, 0, sizeof(inf));
    inf.ndim = d;
    inf.n[0] = h.nx;
    inf.n[1] = h.ny;
    inf.n[2] = h.nz;
    inf.N = h.N;
    inf.Ns = h.Ns;
    inf.Nt = Nt;
    inf.lossy = h.lossy;
    inf.precision = prec;
    inf.dt = dt;
    inf.c_ref = cmax;
    return PAT_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace pat

using namespace pat;

extern "C" {

pat_status pat_plan_create(const pat_grid* grid, const double* c, const double* rho, const double* alpha0,
                           int alpha0_is_scalar, double y, const pat_sensors* sensors, double dt, int Nt,
                           pat_precision prec, pat_plan** out) {
    set_error("");
    if (!out) return fail(PAT_EINVAL, "out is NULL");
    *out = nullptr;
    HostTables h;
    pat_status st = build_tables(grid, c, rho, alpha0, alpha0_is_scalar, y, sensors, dt, Nt, prec, h);
    if (st != PAT_OK) return st;
    PlanBase* impl = (prec == PAT_F32) ? make_plan_f32(h, &st) : make_plan_f64(h, &st);
    if (!impl) return st;
    {
        PlanInputs& in = impl->in;
        in.grid = *grid;
        const size_t N = (size_t)h.N;
        in.c.assign(c, c + N);
        in.rho.assign(rho, rho + N);
        in.alpha0.assign(alpha0, alpha0 + (alpha0_is_scalar ? 1 : N));
        in.alpha0_is_scalar = alpha0_is_scalar;
        in.y = y;
        in.dt = dt;
        in.Nt = Nt;
        in.Ns = sensors->count;
        if (sensors->pos) in.pos.assign(sensors->pos, sensors->pos + (size_t)sensors->count * grid->ndim);
        else in.index.assign(sensors->index, sensors->index + sensors->count);
        in.prec = prec;
    }
    pat_plan* p = new pat_plan;
    p->impl = impl;
    *out = p;
    return PAT_OK;
}

pat_status pat_plan_destroy(pat_plan* plan) {
    if (!plan) return PAT_OK;
    {
        DeviceGuard g(plan->impl->device);
        if (plan->impl->trace) {
            cudaDeviceSynchronize();
            cudaFree(plan->impl->trace);
        }
        delete plan->impl;
    }
    delete plan;
    return PAT_OK;
}

pat_status pat_plan_get_info(const pat_plan* plan, pat_plan_info_t* info) {
    if (!plan || !info) return fail(PAT_EINVAL, "NULL argument");
    *info = plan->impl->info;
    return PAT_OK;
}

pat_status pat_forward_plan(pat_plan* plan, const void* p0, void* data, void* stream) {
    set_error("");
    if (!plan || !p0 || !data) return fail(PAT_EINVAL, "NULL argument");
    PlanBase* b = plan->impl;
    DeviceGuard g(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    pat_status st = b->persistent ? PAT_OK : plan_capture(b, false);
    if (st != PAT_OK) return st;
    const size_t nimg = (size_t)b->info.N * b->elem;
    const size_t ndat = (size_t)b->info.Nt * b->info.Ns * b->elem;
    cudaError_t e = cudaMemcpyAsync(b->img_ptr, p0, nimg, cudaMemcpyDefault, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy p0");
    if (b->smooth) {   // p^0 = S p0 (Sec. VI.A)
        st = plan_smooth(b, b->img_ptr, s);
        if (st != PAT_OK) return st;
    }
    st = plan_clear_finite(b, s);
    if (st != PAT_OK) return st;
    if (b->persistent) {
        st = plan_run_persistent(b, false, s);
        if (st != PAT_OK) return st;
    } else {
        e = cudaGraphLaunch(b->fwd_exec, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch (forward)");
    }
    st = plan_finite_check(b, false, s);
    if (st != PAT_OK) return st;
    e = cudaMemcpyAsync(data, b->data_ptr, ndat, cudaMemcpyDefault, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy data");
    return PAT_OK;
}

pat_status pat_adjoint(pat_plan* plan, const void* residual, void* grad, void* stream) {
    set_error("");
    if (!plan || !residual || !grad) return fail(PAT_EINVAL, "NULL argument");
    PlanBase* b = plan->impl;
    DeviceGuard g(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    pat_status st = b->persistent ? PAT_OK : plan_capture(b, true);
    if (st != PAT_OK) return st;
    const size_t nimg = (size_t)b->info.N * b->elem;
    const size_t ndat = (size_t)b->info.Nt * b->info.Ns * b->elem;
    cudaError_t e = cudaMemcpyAsync(b->data_ptr, residual, ndat, cudaMemcpyDefault, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy residual");
    st = plan_clear_finite(b, s);
    if (st != PAT_OK) return st;
    if (b->persistent) {
        st = plan_run_persistent(b, true, s);
        if (st != PAT_OK) return st;
    } else {
        e = cudaGraphLaunch(b->adj_exec, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch (adjoint)");
    }
    if (b->smooth) {   // (H S)^T = S H^T
        st = plan_smooth(b, b->img_ptr, s);
        if (st != PAT_OK) return st;
    }
    st = plan_finite_check(b, true, s);
    if (st != PAT_OK) return st;
    e = cudaMemcpyAsync(grad, b->img_ptr, nimg, cudaMemcpyDefault, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy gradient");
    return PAT_OK;
}

pat_status pat_plan_set_smoothing(pat_plan* plan, int enable) {
    set_error("");
    if (!plan || enable < 0 || enable > 1) return fail(PAT_EINVAL, "NULL plan or enable not 0 / 1");
    if (plan->impl->arena) return fail(PAT_EUNSUPPORTED, "static-arena plans do not smooth p0");
    if (enable) {
        DeviceGuard g(plan->impl->device);
        const pat_status st = plan_smooth_alloc(plan->impl);
        if (st != PAT_OK) return st;
    }
    plan->impl->smooth = enable;
    return PAT_OK;
}

pat_status pat_plan_smooth(pat_plan* plan, const void* x, void* y, void* stream) {
    set_error("");
    if (!plan || !x || !y) return fail(PAT_EINVAL, "NULL argument");
    PlanBase* b = plan->impl;
    DeviceGuard g(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (x != y) {
        const cudaError_t e = cudaMemcpyAsync(y, x, (size_t)b->info.N * b->elem, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "copy x");
    }
    return plan_smooth(b, y, s);
}

pat_status pat_plan_set_fault(pat_plan* plan, int barrier_extra, double wait_limit_s) {
    set_error("");
    if (!plan || barrier_extra < 0 || barrier_extra > 1 || !(wait_limit_s > 0.0) || wait_limit_s > 10.0)
        return fail(PAT_EINVAL, "bad fault arguments (barrier_extra 0 or 1, 0 < wait_limit_s <= 10)");
    return plan_set_fault(plan->impl, (unsigned)barrier_extra, wait_limit_s);
}

pat_status pat_gradient_c2(pat_plan* plan, const void* p0, const void* residual, void* grad_c2, void* grad_p0,
                           int checkpoint_every, void* stream) {
    set_error("");
    if (!plan || !p0 || !residual || !grad_c2) return fail(PAT_EINVAL, "NULL argument");
    if (checkpoint_every < 1) return fail(PAT_EINVAL, "checkpoint_every must be >= 1");
    PlanBase* b = plan->impl;
    if (b->arena) return fail(PAT_EUNSUPPORTED, "static-arena plans run the forward operator only");
    DeviceGuard g(b->device);
    return plan_gradient_medium(b, p0, residual, grad_c2, nullptr, grad_p0, checkpoint_every, (cudaStream_t)stream);
}

pat_status pat_gradient_rho(pat_plan* plan, const void* p0, const void* residual, void* grad_rho, void* grad_p0,
                            int checkpoint_every, void* stream) {
    set_error("");
    if (!plan || !p0 || !residual || !grad_rho) return fail(PAT_EINVAL, "NULL argument");
    if (checkpoint_every < 1) return fail(PAT_EINVAL, "checkpoint_every must be >= 1");
    PlanBase* b = plan->impl;
    if (b->arena) return fail(PAT_EUNSUPPORTED, "static-arena plans run the forward operator only");
    DeviceGuard g(b->device);
    return plan_gradient_medium(b, p0, residual, nullptr, grad_rho, grad_p0, checkpoint_every, (cudaStream_t)stream);
}

pat_status pat_gradient_medium(pat_plan* plan, const void* p0, const void* residual, void* grad_c2, void* grad_rho,
                               void* grad_p0, int checkpoint_every, void* stream) {
    set_error("");
    if (!plan || !p0 || !residual) return fail(PAT_EINVAL, "NULL argument");
    if (!grad_c2 && !grad_rho && !grad_p0) return fail(PAT_EINVAL, "no output requested");
    if (checkpoint_every < 1) return fail(PAT_EINVAL, "checkpoint_every must be >= 1");
    PlanBase* b = plan->impl;
    if (b->arena) return fail(PAT_EUNSUPPORTED, "static-arena plans run the forward operator only");
    DeviceGuard g(b->device);
    return plan_gradient_medium(b, p0, residual, grad_c2, grad_rho, grad_p0, checkpoint_every, (cudaStream_t)stream);
}

pat_status pat_time_reversal(pat_plan* plan, const void* data, void* image, int compensate, double k_cut,
                             void* stream) {
    set_error("");
    if (!plan || !data || !image) return fail(PAT_EINVAL, "NULL argument");
    if (compensate != 0 && compensate != 1) return fail(PAT_EINVAL, "compensate must be 0 or 1");
    if (compensate && !(k_cut > 0.0 && k_cut <= 1.0)) return fail(PAT_EINVAL, "k_cut must lie in (0, 1]");
    PlanBase* b = plan->impl;
    if (b->arena) return fail(PAT_EUNSUPPORTED, "static-arena plans run the forward operator only");
    DeviceGuard g(b->device);
    return plan_time_reversal(b, data, image, compensate, k_cut, (cudaStream_t)stream);
}

pat_status pat_adjoint_atd(pat_plan* plan, const void* residual, void* image, int initial_paper, void* stream) {
    set_error("");
    if (!plan || !residual || !image) return fail(PAT_EINVAL, "NULL argument");
    if (initial_paper != 0 && initial_paper != 1) return fail(PAT_EINVAL, "initial_paper must be 0 or 1");
    PlanBase* b = plan->impl;
    if (b->arena) return fail(PAT_EUNSUPPORTED, "static-arena plans run the forward operator only");
    DeviceGuard g(b->device);
    return plan_adjoint_atd(b, residual, image, initial_paper, (cudaStream_t)stream);
}

pat_status pat_forward(const void* p0, const double* c, const double* rho, const double* alpha0,
                       int alpha0_is_scalar, double y, const pat_grid* grid, const pat_sensors* sensor_mask,
                       double dt, int Nt, pat_precision prec, void* data, void* stream) {
    pat_plan* plan = nullptr;
    pat_status st = pat_plan_create(grid, c, rho, alpha0, alpha0_is_scalar, y, sensor_mask, dt, Nt, prec, &plan);
    if (st != PAT_OK) return st;
    st = pat_forward_plan(plan, p0, data, stream);
    if (st == PAT_OK) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
    }
    std::string msg = pat_last_error();
    pat_plan_destroy(plan);
    set_error(msg);
    return st;
}

pat_status pat_plan_set_probe(pat_plan* plan, int stride) {
    set_error("");
    if (!plan || stride < 0) return fail(PAT_EINVAL, "bad probe arguments");
    PlanBase* b = plan->impl;
    if (stride == b->probe_stride) return PAT_OK;
    DeviceGuard g(b->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    if (b->fwd_exec) cudaGraphExecDestroy(b->fwd_exec);
    if (b->adj_exec) cudaGraphExecDestroy(b->adj_exec);
    b->fwd_exec = b->adj_exec = nullptr;
    b->probe_stride = stride;
    return PAT_OK;
}

pat_status pat_plan_status(pat_plan* plan) {
    set_error("");
    if (!plan) return fail(PAT_EINVAL, "NULL argument");
    PlanBase* b = plan->impl;
    DeviceGuard g(b->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    if (b->gbar) {
        unsigned w[4] = {0, 0, 0, 0};
        e = cudaMemcpy(w, b->gbar, sizeof(w), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "read status word");
        if (w[2] != 0) {
            set_error("a bounded device-side wait ran out (grid barrier of the persistent kernel)");
            return (pat_status)w[2];
        }
    }
    if (b->fstat) {
        unsigned f = 0;
        e = cudaMemcpy(&f, b->fstat, sizeof(f), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "read status word");
        if (f != 0) {
            set_error(f == PAT_ETIMEOUT ? "a bounded device-side wait ran out (tensor copy of a spectral tile)"
                                        : "the last solve's output holds NaN or infinite values");
            return (pat_status)f;
        }
    }
    return PAT_OK;
}

pat_status pat_plan_set_trace(pat_plan* plan, int k0, int nk) {
    set_error("");
    if (!plan || k0 < 0 || nk < 0 || nk > 4096) return fail(PAT_EINVAL, "bad trace arguments");
    PlanBase* b = plan->impl;
    if (!b->persistent) return PAT_OK;
    DeviceGuard g(b->device);
    if (b->trace) {
        cudaDeviceSynchronize();
        cudaFree(b->trace);
        b->trace = nullptr;
    }
    b->trace_k0 = k0;
    b->trace_nk = nk;
    if (nk == 0) return PAT_OK;
    const size_t bytes = (size_t)b->persist_grid * nk * 8 * sizeof(unsigned long long);
    cudaError_t e = cudaMalloc(&b->trace, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (trace)");
    e = cudaMemset(b->trace, 0, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset (trace)");
    return PAT_OK;
}

pat_status pat_plan_read_trace(pat_plan* plan, unsigned long long* out, size_t count, int* grid) {
    set_error("");
    if (!plan || !grid) return fail(PAT_EINVAL, "NULL argument");
    PlanBase* b = plan->impl;
    *grid = 0;
    if (!b->trace) return PAT_OK;
    const size_t n = (size_t)b->persist_grid * b->trace_nk * 8;
    if (!out || count < n) return fail(PAT_EINVAL, "trace buffer too small");
    DeviceGuard g(b->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    e = cudaMemcpy(out, b->trace, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read trace");
    *grid = b->persist_grid;
    return PAT_OK;
}

int pat_plan_probe_slots(const pat_plan* plan, int adjoint) {
    if (!plan) return 0;
    return (int)plan->impl->probe_names[adjoint ? 1 : 0].size();
}

pat_status pat_plan_probe_read(pat_plan* plan, int adjoint, int slot, const char** name, double* mean_ms,
                               int* samples) {
    set_error("");
    if (!plan || !name || !mean_ms || !samples) return fail(PAT_EINVAL, "NULL argument");
    DeviceGuard g(plan->impl->device);
    pat_status st = plan_probe_read(plan->impl, adjoint ? 1 : 0, slot, name, mean_ms, samples);
    if (st == PAT_EINVAL) set_error("probe slot out of range (probe off or graph not captured yet)");
    return st;
}

const char* pat_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
