// pat_wave.cu -- device plan, launch sequence and CUDA-graph capture of the forward operator H
// and its exact transpose H^T (Sec. III).  The whole Nt-step loop of one solve is captured once
// per plan into a CUDA graph and replayed with a single cudaGraphLaunch per call.
#include <algorithm>
#include <cstdlib>
#include <cstdio>
#include <cstring>

#include <cuda.h>   // CUtensorMap and its encoder's types; the encoder is fetched from the driver at run time

#include <mutex>
#include <type_traits>

#include "pat_host.h"
#include "pat_persist.cuh"
#include "pat_p2.h"
#include "pat_smooth.h"

namespace pat {

// dJ/drho0 += the part through b_xi[j] = 2 / (rho0[j] + rho0[j + e_xi]) (periodic): with
// B_xi = dJ/db_xi * (-b_xi^2 / 2), point j receives B_xi[j] (its own b) + B_xi[j - e_xi] (the b of
// the point before it along xi) (reading D3).
template <typename T> __global__ void k_rho_chain(DevPlan<T> P, const T* gb, T* grho) {
    const long long N = P.N;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(j % P.nx);
        const long long yz = j / P.nx;
        const int y = (int)(yz % P.ny), z = (int)(yz / P.ny);
        T acc = 0;
        for (int a = 0; a < P.d; ++a) {
            long long jm;
            if (a == 0) jm = j - x + (x == 0 ? P.nx - 1 : x - 1);
            else if (a == 1) jm = j + (long long)((y == 0 ? P.ny - 1 : y - 1) - y) * P.nx;
            else jm = j + (long long)((z == 0 ? P.nz - 1 : z - 1) - z) * P.nx * P.ny;
            const T* g = gb + (size_t)a * N;
            const T b0 = P.b[a][j], b1 = P.b[a][jm];
            acc += g[j] * (T(-0.5) * b0 * b0) + g[jm] * (T(-0.5) * b1 * b1);
        }
        grho[j] += acc;
    }
}

// time reversal: p^0 = the last datum at each sensor's node (the rest of the image is zero)
template <typename T> __global__ void k_tr_start(T* img, const int* node, const T* row, int Ns) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < Ns) img[node[j]] = row[j];
}

// adjoint-then-discretize source rows: src[n] = (h^{Nt-1-n} + h^{Nt-2-n}) / 2, n = 0 .. Nt-2, the
// reversed data averaged over the half step (reading A2)
template <typename T> __global__ void k_atd_source(T* src, const T* h, int Nt, int Ns) {
    const long long cnt = (long long)(Nt - 1) * Ns;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < cnt; q += (long long)gridDim.x * blockDim.x) {
        const long long n = q / Ns, j = q - n * Ns;
        src[q] = (T)0.5 * (h[(size_t)(Nt - 1 - n) * Ns + j] + h[(size_t)(Nt - 2 - n) * Ns + j]);
    }
}

// g = sum_xi rho*_xi / rho0 (Eq. (adjj))
template <typename T> __global__ void k_atd_image(DevPlan<T> P, T* img) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < P.N; j += (long long)gridDim.x * blockDim.x) {
        T acc = 0;
        for (int a = 0; a < P.d; ++a) acc += P.rh[a][j];
        img[j] = acc / P.rho0[j];
    }
}

// reading A5, first half: x-transform of the channels (0, c0^2 eta g) into spectra 0 and 1
template <typename T, int D> __global__ void __launch_bounds__(256) k_atd_a5_fwd(DevPlan<T> P, int R) {
    RowSm<T, D> sm(P.nx, P.ldh, R);
    const int nx = P.nx, line0 = blockIdx.x * R;
    stage16(sm.tw, P.twx, (size_t)nx * sizeof(cplx<T>));
    cp_commit();
    pdl_trigger();
    pdl_wait();
    cp_wait_all();
    __syncthreads();
    for (int r = 0; r < R; ++r)
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const size_t idx = (size_t)(line0 + r) * nx + i;
            slot(sm.A, r, i, nx) = (T)0;
            slot(sm.A, R + r, i, nx) = P.c2eta[idx] * P.img[idx];
        }
    __syncthreads();
    cplx<T>* res = fft_rows<T, false>(sm.A, sm.B, P.fx, sm.tw, R);
    r2c_unpack(res, P.spec, 2, R, line0, nx, P.ldh);
}

// reading A5, second half: inverse x-transform; g <- g - L_{y-1}(c0^2 eta g) / c0^2
template <typename T, int D> __global__ void __launch_bounds__(256) k_atd_a5_inv(DevPlan<T> P, int R) {
    RowSm<T, D> sm(P.nx, P.ldh, R);
    const int nx = P.nx, line0 = blockIdx.x * R;
    stage16(sm.tw, P.twx, (size_t)nx * sizeof(cplx<T>));
    cp_commit();
    pdl_trigger();
    pdl_wait();
    stage_spectra(sm.S, P.spec, 2, line0, R, P.ldh);
    cp_commit();
    cp_wait_all();
    __syncthreads();
    c2r_pack(sm.A, sm.S, 2, R, nx, P.ldh);
    __syncthreads();
    cplx<T>* res = fft_rows<T, true>(sm.A, sm.B, P.fx, sm.tw, R);
    for (int r = 0; r < R; ++r)
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const size_t idx = (size_t)(line0 + r) * nx + i;
            P.img[idx] = P.img[idx] - slot(res, R + r, i, nx) / P.c2[idx];
        }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
    static std::mutex mu;
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    std::lock_guard<std::mutex> lock(mu);
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    }
    return fn;
}

template <typename T> struct Plan : public PlanBase {
    DevPlan<T> P{};
    HostTables H;   // kept for the FP64 tables' sizes and for rebuilding
    size_t row_smem = 0, spec_smem = 0;
    bool count_only = false;   // arena sizing pass: bump offsets, touch no memory

    template <typename U> U* dalloc(size_t count, pat_status* st) {
        void* p = nullptr;
        if (count == 0) count = 1;
        if (arena) {
            const size_t off = (arena_used + 255) & ~(size_t)255;
            const size_t bytes = count * sizeof(U);
            if (count_only) {
                arena_used = off + bytes;
                return reinterpret_cast<U*>(arena + 0);
            }
            if (off + bytes > arena_cap) {
                *st = PAT_EINVAL;
                set_error("problem too large for the static scratch array (" + std::to_string(arena_cap) +
                          " bytes): reduce the grid, Nt * Ns or the precision");
                return nullptr;
            }
            arena_used = off + bytes;
            return reinterpret_cast<U*>(arena + off);
        }
        cudaError_t e = cudaMalloc(&p, count * sizeof(U));
        if (e != cudaSuccess) {
            *st = (e == cudaErrorMemoryAllocation) ? PAT_ENOMEM : PAT_ECUDA;
            set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
            cudaGetLastError();
            return nullptr;
        }
        allocs.push_back(p);
        return static_cast<U*>(p);
    }
    template <typename U, typename V> const U* upload(const std::vector<V>& v, pat_status* st) {
        U* d = dalloc<U>(v.size(), st);
        if (!d) return nullptr;
        if (count_only) return d;
        std::vector<U> tmp(v.size());
        for (size_t i = 0; i < v.size(); ++i) tmp[i] = static_cast<U>(v[i]);
        if (!v.empty()) {
            cudaError_t e = cudaMemcpy(d, tmp.data(), v.size() * sizeof(U), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                *st = cuda_fail(e, "cudaMemcpy (plan tables)");
                return nullptr;
            }
        }
        return d;
    }
    const cplx<T>* upload_c(const std::vector<std::complex<double>>& v, pat_status* st) {
        cplx<T>* d = dalloc<cplx<T>>(v.size(), st);
        if (!d) return nullptr;
        if (count_only) return d;
        std::vector<cplx<T>> tmp(v.size());
        for (size_t i = 0; i < v.size(); ++i) tmp[i] = mkc<T>((T)v[i].real(), (T)v[i].imag());
        if (!v.empty()) {
            cudaError_t e = cudaMemcpy(d, tmp.data(), v.size() * sizeof(cplx<T>), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                *st = cuda_fail(e, "cudaMemcpy (plan tables)");
                return nullptr;
            }
        }
        return d;
    }

    ~Plan() override {
        if (arena) return;   // nothing owned on the device: the caller synchronised its stream
        if (cap_stream) cudaStreamSynchronize(cap_stream);
        cudaDeviceSynchronize();
        if (fwd_exec) cudaGraphExecDestroy(fwd_exec);
        if (adj_exec) cudaGraphExecDestroy(adj_exec);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (int g = 0; g < 2; ++g)
            for (cudaEvent_t ev : probe_ev[g]) cudaEventDestroy(ev);
        for (void* p : allocs) cudaFree(p);
    }

    pat_status build(const HostTables& h) {
        H = h;
        pat_status st = PAT_OK;
        elem = sizeof(T);
        const int D = h.d;
        P.d = D;
        P.nx = h.nx;
        P.ny = h.ny;
        P.nz = h.nz;
        P.nxh = h.nxh;
        P.ldh = h.ldh;
        P.nlines = h.ny * h.nz;
        P.N = h.N;
        P.lossy = h.lossy;
        P.dt = (T)h.dt;
        P.Nt = h.Nt;
        P.bar_extra = 0;
        P.bar_limit_ns = 2000000000ull;
        {
            const char* ef = std::getenv("PAT_P2SPEC");
            P.fixed_len = (ef && std::atoi(ef) == 0) ? 0 : 1;
        }
        const size_t N = (size_t)h.N;
        const size_t Nh = (size_t)h.nz * h.ny * h.ldh;
#define CHK(x) \
    do {       \
        if (!(x)) return st; \
    } while (0)
#define CHK2(x)                          \
    do {                                 \
        pat_status s2_ = (x);            \
        if (s2_ != PAT_OK) return s2_;   \
    } while (0)
        CHK(P.c2 = upload<T>(h.c2, &st));
        CHK(P.rho0 = upload<T>(h.rho0, &st));
        for (int a = 0; a < 3; ++a) {
            if (a < D) CHK(P.b[a] = upload<T>(h.b[a], &st));
            else P.b[a] = nullptr;
            CHK(P.a[a] = upload<T>(h.a[a], &st));
            CHK(P.au[a] = upload<T>(h.au[a], &st));
            CHK(P.dp[a] = upload_c(h.dp[a], &st));
            CHK(P.dm[a] = upload_c(h.dm[a], &st));
        }
        if (h.lossy) {
            CHK(P.c2tau = upload<T>(h.c2tau, &st));
            CHK(P.c2eta = upload<T>(h.c2eta, &st));
        }
        for (int a = 0; a < 3; ++a) CHK(P.kv[a] = upload<T>(h.kv[a], &st));
        P.kap_a = (T)h.kap_a;
        P.pha = (T)h.pha;
        P.phb = (T)h.phb;
        P.invN = (T)h.invN;
        P.fx = h.fx;
        P.fy = h.fy;
        P.fz = h.fz;
        CHK(P.twx = upload_c(h.tw[0], &st));
        CHK(P.twy = upload_c(h.tw[1], &st));
        CHK(P.twz = upload_c(h.tw[2], &st));
        {
            const FftAxis* fa[3] = {&h.fx, &h.fy, &h.fz};
            for (int a = 0; a < 3; ++a) {
                P.stw[a] = nullptr;
                if (a < D && fa[a]->pow2 && fa[a]->lgn >= 4 && fa[a]->lgn <= 11)
                    CHK(P.stw[a] = upload_c(p2_stage_table(h.tw[a], fa[a]->lgn), &st));
                P.stw16[a] = nullptr;
                if (D == 3 && a >= 1 && fa[a]->pow2 && (fa[a]->lgn == 7 || fa[a]->lgn == 8))
                    CHK(P.stw16[a] = upload_c(p2x_stage_table(h.tw[a], fa[a]->lgn), &st));
            }
            // 1 (default): the plain y passes take the two-stage schedule; 2: the fused multiply
            // passes too (measured slower at 256^3); 0: neither
            const char* e16 = std::getenv("PAT_SPEC16");
            P.spec16 = e16 ? std::max(0, std::min(3, std::atoi(e16))) : 1;
            info.schedule = (D == 3 && (P.stw16[1] || P.stw16[2])) ? P.spec16 : 0;
            const char* ech = std::getenv("PAT_SPEC_CHUNKS");
            spec_chunks = (D == 3 && ech) ? std::max(1, std::atoi(ech)) : 1;
            info.spec_chunks = 1;
        }
        for (int a = 0; a < 3; ++a) {
            if (a < D) {
                CHK(P.u[a] = dalloc<T>(N, &st));
                CHK(P.rh[a] = dalloc<T>(N, &st));
            } else {
                P.u[a] = nullptr;
                P.rh[a] = nullptr;
            }
        }
        if (h.lossy) {
            CHK(P.rsum = dalloc<T>(N, &st));
            CHK(P.pbar = dalloc<T>(N, &st));
        }
        const int nspec = std::max(D, 2);
        for (int a = 0; a < 3; ++a) {
            if (a < nspec) CHK(P.spec[a] = dalloc<cplx<T>>(Nh, &st));
            else P.spec[a] = nullptr;
        }
        CHK(P.img = dalloc<T>(N, &st));
        CHK(P.data = dalloc<T>((size_t)h.Nt * h.Ns, &st));
        CHK(fstat = dalloc<unsigned>(1, &st));
        img_ptr = P.img;
        data_ptr = P.data;
        // sensors
        DevSensors<T>& S = P.sens;
        S.Ns = h.Ns;
        CHK(S.g_lineptr = upload<int>(h.g_lineptr, &st));
        CHK(S.g_seg_line = upload<int>(h.g_seg_line, &st));
        CHK(S.g_seg_sensor = upload<int>(h.g_seg_sensor, &st));
        CHK(S.g_seg_x0 = upload<int>(h.g_seg_x0, &st));
        CHK(S.g_seg_w0 = upload<T>(h.g_seg_w0, &st));
        CHK(S.g_seg_w1 = upload<T>(h.g_seg_w1, &st));
        CHK(S.s_lineptr = upload<int>(h.s_lineptr, &st));
        CHK(S.s_seg_line = upload<int>(h.s_seg_line, &st));
        CHK(S.s_seg_x = upload<int>(h.s_seg_x, &st));
        CHK(S.s_seg_e0 = upload<int>(h.s_seg_e0, &st));
        CHK(S.s_ent_sensor = upload<int>(h.s_ent_sensor, &st));
        CHK(S.s_ent_w = upload<T>(h.s_ent_w, &st));
#undef CHK
        // launch configuration
        cfg = h.cfg;
        {
            // power-of-two y (and z) lines of 16 .. 2048 points take the register-fused spectral kernel
            const char* es2 = std::getenv("PAT_SPEC2");
            const auto ok = [](const FftAxis& a) { return a.pow2 && a.lgn >= 4 && a.lgn <= 11; };
            use_spec2 = !(es2 && std::atoi(es2) == 0) && ok(h.fy) && (D == 2 || ok(h.fz));
        }
        {
            // power-of-two x-lines of 16 .. 2048 points take the register-fused row kernels
            const char* er2 = std::getenv("PAT_ROW2");
            const int R0 = cfg.row_lines;
            use_row2 = !(er2 && std::atoi(er2) == 0) && h.fx.pow2 && h.fx.lgn >= 4 && h.fx.lgn <= 11 &&
                       (R0 & (R0 - 1)) == 0 && R0 <= 32;
            // FP32 3-D x-lines of 128 and 256 points: the u update and its transpose one velocity component
            // per CTA (PAT_ROWU1=0: all three in k_row2)
            const char* eu1 = std::getenv("PAT_ROWU1");
            use_rowu1 = use_row2 && sizeof(T) == 4 && D == 3 && P.fixed_len && (h.fx.lgn == 7 || h.fx.lgn == 8) &&
                        !(eu1 && std::atoi(eu1) == 0);
            const char* eul = std::getenv("PAT_ROWU1_LINES");
            const int ul = eul ? std::atoi(eul) : 0;
            rowu1_pin = (ul >= 2 && ul <= 32 && (ul & (ul - 1)) == 0) ? ul : 0;
            info.rowu1 = use_rowu1 ? 1 : 0;
        }
        row_smem = row_smem_bytes<T>(D, h.nx, h.ldh, cfg.row_lines);
        row2_smem = use_row2 ? row2_layout<T>(D, h.nx, h.ldh, cfg.row_lines).bytes : 0;
        spec_smem = spec_bytes(D, std::max(h.ny, h.nz), cfg.col_w);
        if (count_only) return PAT_OK;
        // padding columns of the half spectra are read (never used) by full-width tiles: zero them
        for (int a = 0; a < nspec; ++a) {
            cudaError_t e = cudaMemset(P.spec[a], 0, Nh * sizeof(cplx<T>));
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemset (spectra)");
        }
        if (D == 2) st = set_attrs<2>();
        else st = set_attrs<3>();
        if (st != PAT_OK) return st;
        P.fault = fstat;
        if (arena) return PAT_OK;
        CHK2(build_tmaps());
        cudaError_t e = cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
        CHK2(build_kap());
        CHK2(configure_persistent(h));
        info.layout[0] = persistent ? pcfg.W : cfg.col_w;
        info.layout[1] = persistent ? pcfg.ppc : cfg.row_lines;
        if (!persistent) {
            st = (D == 2) ? tune_graph<2>() : tune_graph<3>();
            if (st != PAT_OK) return st;
        }
        info.spec_chunks = (!persistent && D == 3) ? chunk_count() : 1;
        return PAT_OK;
    }

    bool use_zreg = false;
    bool zreg_all = false;
    bool use_ywide = false;
    bool use_zwide = false;
    float* kap3 = nullptr;   // kappa / N on the half spectrum, [ky][kz][ldh] (the 16-column z passes)
    float* abs3 = nullptr;   // |k|^(y-2) / N and |k|^(y-1) / N, [2][ky][kz][ldh] (absorbing plans)

    // Tensor maps of the half spectra for the 3-D spectral tiles (FP32; boxes of 8 columns x the whole
    // line: ny for y passes, nz for z passes; lines of at most 256 points): staging by tensor copies.
    // PAT_TMA=0 keeps the cp.async staging.  Without the driver's encoder, or for other plans, nothing.
    // Also the boxes of 16 columns of the plain y transforms on 128- and 256-point y-lines (k_ywide) and
    // of the field-wise z passes on 128- and 256-point z-lines (k_zwide).
    pat_status build_tmaps() {
        P.tmaps = nullptr;
        P.use_tma = 0;
        const char* ev = std::getenv("PAT_TMA");
        if (ev && std::atoi(ev) == 0) return PAT_OK;
        if (sizeof(T) != 4 || H.d != 3 || !use_spec2 || H.ny > 256 || H.nz > 256) return PAT_OK;
        EncodeTiledFn enc = encode_tiled();
        if (!enc) return PAT_OK;
        // [0..2] y-pass boxes, [3..5] z-pass boxes, [6..8] z-pass boxes under the 64-byte swizzle (the
        // register-resident z passes of 256-point lines), [9..11] y-pass boxes of 16 columns (128-byte
        // rows; 128- and 256-point y-lines), [12..14] z-pass boxes of 16 columns (128- and 256-point
        // z-lines); slots of maps a plan does not use stay zero
        CUtensorMap maps[15];
        std::memset(maps, 0, sizeof(maps));
        const bool zmaps = H.nz == 256, ymaps = H.ny == 128 || H.ny == 256, zwmaps = H.nz == 128 || H.nz == 256;
        const cuuint64_t dims[3] = {(cuuint64_t)2 * H.ldh, (cuuint64_t)H.ny, (cuuint64_t)H.nz};
        const cuuint64_t strides[2] = {(cuuint64_t)H.ldh * sizeof(cplx<T>), (cuuint64_t)H.ny * H.ldh * sizeof(cplx<T>)};
        const cuuint32_t estr[3] = {1, 1, 1};
        for (int k = 0; k < 15; ++k) {
            if ((k >= 6 && k < 9 && !zmaps) || (k >= 9 && k < 12 && !ymaps) || (k >= 12 && !zwmaps)) continue;
            const int a = k % 3;
            const void* base = (a < std::max(H.d, 2)) ? (const void*)P.spec[a] : (const void*)P.spec[0];
            const bool ypass = k < 3 || (k >= 9 && k < 12);
            const cuuint32_t box[3] = {k >= 9 ? 32u : 16u, ypass ? (cuuint32_t)H.ny : 1u, ypass ? 1u : (cuuint32_t)H.nz};
            const CUresult r = enc(&maps[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides,
                                   box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                   (k >= 6 && k < 9) ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return PAT_OK;   // keep the cp.async staging
        }
        pat_status st = PAT_OK;
        void* d = dalloc<unsigned char>(sizeof(maps), &st);
        if (!d) return st;
        const cudaError_t e = cudaMemcpy(d, maps, sizeof(maps), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy (tensor maps)");
        P.tmaps = d;
        P.use_tma = 1;
        info.tma = 1;
        // the register-resident z passes (fixed-length kernels, 256-point z-lines): by default for the D-
        // passes (DIV and its transpose), where they are faster; PAT_ZREG=0 none, 2 every multiply pass
        const char* ez = std::getenv("PAT_ZREG");
        zreg_all = ez && std::atoi(ez) >= 2;
        use_zreg = zmaps && P.fixed_len && !(ez && std::atoi(ez) == 0);
        if (use_zreg) {
            const cudaError_t ea = zreg_set_attrs();
            if (ea != cudaSuccess) return cuda_fail(ea, "cudaFuncSetAttribute (z passes)");
        }
        info.zreg = use_zreg ? 1 : 0;
        // the 16-column plain y transforms (fixed-length kernels, 128- and 256-point y-lines); PAT_YWIDE=0
        // keeps k_spec16 / k_spec2 for them
        const char* ey = std::getenv("PAT_YWIDE");
        use_ywide = ymaps && P.fixed_len && !(ey && std::atoi(ey) == 0);
        if (use_ywide) {
            const cudaError_t ea = ywide_set_attrs();
            if (ea != cudaSuccess) return cuda_fail(ea, "cudaFuncSetAttribute (y passes)");
        }
        info.ywide = use_ywide ? 1 : 0;
        // the 16-column z passes (fixed-length kernels, 128- and 256-point z-lines); PAT_ZWIDE=0 keeps
        // k_zreg / k_spec16 / k_spec2 for them.  Their multiplier tables are filled once the plan's stream
        // exists (build_kap).
        const char* ew = std::getenv("PAT_ZWIDE");
        use_zwide = zwmaps && P.fixed_len && !(ew && std::atoi(ew) == 0);
        if (use_zwide) {
            const cudaError_t ea = zwide_set_attrs();
            if (ea != cudaSuccess) return cuda_fail(ea, "cudaFuncSetAttribute (z passes)");
            pat_status st2 = PAT_OK;
            const size_t nt = (size_t)H.ny * H.nz * H.ldh;
            kap3 = dalloc<float>(nt, &st2);
            if (!kap3) return st2;
            if (P.lossy) {
                abs3 = dalloc<float>(2 * nt, &st2);
                if (!abs3) return st2;
            }
        }
        info.zwide = use_zwide ? 1 : 0;
        return PAT_OK;
    }
    pat_status build_kap() {
        if constexpr (std::is_same<T, float>::value) {
            if (!use_zwide) return PAT_OK;
            cudaError_t e = zwide_kap_table(P, kap3, cap_stream);
            if (e == cudaSuccess && abs3) e = zwide_abs_table(P, abs3, cap_stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(cap_stream);
            if (e != cudaSuccess) return cuda_fail(e, "kappa table");
        }
        return PAT_OK;
    }

    bool autotune_enabled() const {
        const char* e = std::getenv("PAT_AUTOTUNE");
        return !(e && std::atoi(e) == 0);
    }
    // device time of fn() on cap_stream: one untimed run, then the mean of `reps`
    template <class Fn> float time_on_stream(Fn&& fn, int reps) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        fn();
        cudaEventRecord(a, cap_stream);
        for (int i = 0; i < reps; ++i) fn();
        cudaEventRecord(b, cap_stream);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return ms / reps;
    }

    // FFT tile autotuner of the per-phase path: columns per spectral CTA (W) x x-lines per row CTA,
    // each feasible pair timed on one forward step and one adjoint step (the kernels do the same
    // work whatever the field values), fastest kept.  PAT_COL_W / PAT_ROW_LINES pin a dimension.
    template <int D> pat_status tune_graph() {
        if (!autotune_enabled() || H.Nt < 2) return PAT_OK;
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const bool fw = std::getenv("PAT_COL_W") != nullptr, fr = std::getenv("PAT_ROW_LINES") != nullptr;
        const int L = std::max(H.ny, H.nz);
        const LaunchCfg base = cfg;
        LaunchCfg best = cfg;
        float best_ms = 1e30f;
        int tried = 0;
        // radix schedules of the 3-D spectral passes over 128- and 256-point lines: 0 = the fixed
        // (r0, 8, ..., 8) stages everywhere, 1 = two stages (n/16, 16) for the plain y transforms,
        // 2 = two stages for every pass (PAT_SPEC16 pins one)
        std::vector<int> scheds{P.spec16};
        if (D == 3 && use_spec2 && (P.stw16[1] || P.stw16[2]) && !std::getenv("PAT_SPEC16")) scheds = {1, 0, 2, 3};
        int best_sched = P.spec16;
        // chunks of column tiles per 3-D spectral operation (PAT_SPEC_CHUNKS pins it)
        std::vector<int> chunk_cands{spec_chunks};
        if (D == 3 && !std::getenv("PAT_SPEC_CHUNKS")) chunk_cands = {1, 2, 4, 8};
        int best_chunks = spec_chunks;
        for (int nchunk : chunk_cands)
        for (int sched : scheds)
        for (int w : {1, 2, 4, 8}) {
            if (fw && w != base.col_w) continue;
            if (sizeof(T) == 8 && w > 4) continue;
            for (int r : {2, 4, 8, 16}) {
                if (fr && r != base.row_lines) continue;
                if (P.nlines % r != 0) continue;
                LaunchCfg c = base;
                c.col_w = w;
                c.row_lines = r;
                c.col_threads = std::min(256, std::max(64, (D * w * L / 8 + 31) / 32 * 32));
                if (!tile_fits(w)) continue;
                const size_t rs = row_smem_bytes<T>(D, H.nx, H.ldh, r), ss = spec_bytes(D, L, w);
                const size_t r2 = use_row2 ? row2_layout<T>(D, H.nx, H.ldh, r).bytes : 0;
                if (r2 > (size_t)optin) continue;
                if (rs > (size_t)optin || ss + 64 > (size_t)optin) continue;   // 64: the spectral kernels' static mbarrier
                cfg = c;
                row_smem = rs;
                row2_smem = r2;
                spec_smem = ss;
                P.spec16 = sched;
                spec_chunks = nchunk;
                const float ms = time_on_stream(
                    [&] {
                        fwd_step_on<D>(P, 1, P.data, (T*)nullptr, cap_stream);
                        adj_step_on<D>(1, (const T*)nullptr, (T*)nullptr, (const T*)nullptr, cap_stream);
                    },
                    2);
                ++tried;
                if (std::getenv("PAT_DEBUG"))
                    fprintf(stderr, "[pat] tune graph chunks=%d schedule=%d W=%d lines=%d: %.4f ms per step pair\n",
                            nchunk, sched, w, r, ms);
                if (ms < best_ms) {
                    best_ms = ms;
                    best = c;
                    best_sched = sched;
                    best_chunks = nchunk;
                }
            }
        }
        cudaError_t e = take_launch_err();
        if (e != cudaSuccess) return cuda_fail(e, "autotune (per-phase kernels)");
        cfg = best;
        P.spec16 = best_sched;
        info.schedule = P.spec16;
        spec_chunks = best_chunks;
        info.spec_chunks = chunk_count();
        row_smem = row_smem_bytes<T>(D, H.nx, H.ldh, cfg.row_lines);
        row2_smem = use_row2 ? row2_layout<T>(D, H.nx, H.ldh, cfg.row_lines).bytes : 0;
        spec_smem = spec_bytes(D, L, cfg.col_w);
        // the timed steps left arbitrary values in the work buffers; the solves re-initialise the
        // state, and the spectra's padding columns are cleared again
        const size_t Nh = (size_t)H.nz * H.ny * H.ldh;
        for (int a = 0; a < std::max(D, 2); ++a) cudaMemsetAsync(P.spec[a], 0, Nh * sizeof(cplx<T>), cap_stream);
        e = cudaStreamSynchronize(cap_stream);
        if (e != cudaSuccess) return cuda_fail(e, "autotune");
        info.layout[0] = cfg.col_w;
        info.layout[1] = cfg.row_lines;
        info.tuned = tried > 1;
        return PAT_OK;
    }

    // ---------------------------------------------------------------------------------------
    // persistent single-kernel path (2-D grids whose per-CTA state fits in shared memory)
    // ---------------------------------------------------------------------------------------
    PersistCfg pcfg{};
    int persist_threads = 256;
    bool persist_p2 = false;

    pat_status configure_persistent(const HostTables& h) {
        persistent = 0;
        const char* env = std::getenv("PAT_PERSIST");
        if (env && std::atoi(env) == 0) return PAT_OK;
        if (h.d != 2) return PAT_OK;
        int dev = 0, optin = 0, nsm = 0, coop = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        const bool dbg = std::getenv("PAT_DEBUG") != nullptr;
        if (!coop) return PAT_OK;
        // power-of-two axes of 16 .. 2048 points take the register-fused kernel
        const char* ep2 = std::getenv("PAT_P2");
        const bool p2 = !(ep2 && std::atoi(ep2) == 0) && h.fx.pow2 && h.fy.pow2 && h.fx.lgn >= 4 &&
                        h.fy.lgn >= 4 && h.fx.lgn <= 11 && h.fy.lgn <= 11;
        const void* kf = p2 ? p2_kernel<T>(false, h.fx.lgn, h.fy.lgn, P.fixed_len) : (const void*)k_persist<T, false>;
        const void* ka = p2 ? p2_kernel<T>(true, h.fx.lgn, h.fy.lgn, P.fixed_len) : (const void*)k_persist<T, true>;
        cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return PAT_OK;
        }
        // Candidate layouts, least work per CTA first (columns per CTA W, x-line pairs per CTA):
        // the first whose grid is co-resident wins.
        const int cands[][2] = {{2, 2}, {1, 1}, {2, 1}, {4, 2}, {4, 4}, {8, 4}, {8, 8}, {4, 1}, {8, 1}, {8, 2}};
        int forced_w = 0, forced_p = 0;
        if (const char* ew = std::getenv("PAT_PERSIST_W")) forced_w = std::atoi(ew);
        if (const char* ep = std::getenv("PAT_PERSIST_PPC")) forced_p = std::atoi(ep);
        struct Cand {
            PersistCfg c;
            int G, threads;
            size_t smem;
        };
        std::vector<Cand> ok;
        for (const auto& cnd : cands) {
            const int W = cnd[0], ppc = cnd[1];
            if (forced_w && W != forced_w) continue;
            if (forced_p && ppc != forced_p) continue;
            if (sizeof(T) == 8 && W > 4) continue;
            const int ntiles = (h.nxh + W - 1) / W;
            const int npairs = h.ny / 2;
            const int G = std::max(ntiles, (npairs + ppc - 1) / ppc);
            PersistCfg c{};
            c.W = W;
            c.lgW = (W == 1) ? 0 : (W == 2 ? 1 : (W == 4 ? 2 : 3));
            c.ntiles = ntiles;
            c.ppc = ppc;
            c.rmax = 2 * ppc;
            c.nres = 11;
            const int need = std::max(c.rmax * h.nx / 8, 2 * W * h.ny / 8);
            const int threads = std::min(256, std::max(64, (need + 31) / 32 * 32));
            const size_t smem = p2 ? p2_smem_bytes<T>(h.nx, h.ny, h.ldh, c.rmax, W, c.nres, h.lossy ? 3 : 1)
                                   : persist_smem_bytes<T>(h.nx, h.ny, h.ldh, c.rmax, W, c.nres);
            if (smem > (size_t)optin) continue;
            int per_sm = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, threads, smem);
            int per_sm_a = 0;
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_a, ka, threads, smem);
            if (dbg)
                fprintf(stderr, "[pat] persistent%s cand W=%d ppc=%d G=%d threads=%d smem=%zu per_sm=%d/%d\n",
                        p2 ? " (pow2)" : "", W, ppc, G, threads, smem, per_sm, per_sm_a);
            if (e != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            if (std::min(per_sm, per_sm_a) * nsm < G) continue;
            ok.push_back(Cand{c, G, threads, smem});
        }
        if (ok.empty()) return PAT_OK;
        pat_status st = PAT_OK;
        gbar = dalloc<unsigned>(4, &st);
        if (!gbar) return st;
        persist_p2 = p2;
        persistent = 1;
        info.path = p2 ? 2 : 1;
        auto use = [&](const Cand& k) {
            pcfg = k.c;
            persist_grid = k.G;
            persist_smem = k.smem;
            persist_threads = k.threads;
        };
        use(ok[0]);   // least work per CTA first
        if (ok.size() > 1 && autotune_enabled() && !forced_w && !forced_p && H.Nt >= 2) {
            // autotuner: time a short forward solve (at most 24 steps) with each co-resident layout
            const int Nt_full = P.Nt;
            P.Nt = std::min(Nt_full, 24);
            size_t bi = 0;
            float best = 1e30f;
            for (size_t i = 0; i < ok.size(); ++i) {
                use(ok[i]);
                const float ms = time_on_stream([&] { run_persistent(false, cap_stream); }, 2);
                if (dbg) fprintf(stderr, "[pat] tune persistent W=%d ppc=%d: %.4f ms\n", ok[i].c.W, ok[i].c.ppc, ms);
                if (ms < best) {
                    best = ms;
                    bi = i;
                }
            }
            P.Nt = Nt_full;
            use(ok[bi]);
            cudaError_t e2 = cudaStreamSynchronize(cap_stream);
            if (e2 == cudaSuccess) e2 = cudaGetLastError();
            if (e2 != cudaSuccess) return cuda_fail(e2, "autotune (persistent kernel)");
            info.tuned = 1;
        }
        return PAT_OK;
    }

    pat_status run_persistent(bool adjoint, cudaStream_t s) {
        cudaError_t e;
        if (!adjoint) {
            e = cudaMemsetAsync(P.data, 0, (size_t)H.Nt * H.Ns * sizeof(T), s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync (data)");
        }
        e = cudaMemsetAsync(gbar, 0, 4 * sizeof(unsigned), s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync (barrier)");
        const int g = adjoint ? 1 : 0;
        if (probe_stride > 0) {
            if (probe_ev[g].size() < 2) {
                for (cudaEvent_t ev : probe_ev[g]) cudaEventDestroy(ev);
                probe_ev[g].assign(2, nullptr);
                cudaEventCreate(&probe_ev[g][0]);
                cudaEventCreate(&probe_ev[g][1]);
            }
            probe_names[g].assign(1, persist_p2 ? (adjoint ? "k_persist2_adj" : "k_persist2_fwd")
                                                : (adjoint ? "k_persist_adj" : "k_persist_fwd"));
            probe_samples[g] = 1;
            cudaEventRecord(probe_ev[g][0], s);
        }
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(persist_grid);
        lc.blockDim = dim3(persist_threads);
        lc.dynamicSmemBytes = persist_smem;
        lc.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        lc.attrs = attr;
        lc.numAttrs = 1;
        P.trace = trace;
        P.trace_k0 = trace_k0;
        P.trace_nk = trace_nk;
        if (persist_p2) {
            e = p2_launch<T>(adjoint, &lc, P, pcfg, gbar);
        } else {
            if (adjoint) e = cudaLaunchKernelEx(&lc, k_persist<T, true>, P, pcfg, gbar);
            else e = cudaLaunchKernelEx(&lc, k_persist<T, false>, P, pcfg, gbar);
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchKernelEx (persistent)");
        if (probe_stride > 0) cudaEventRecord(probe_ev[g][1], s);
        return PAT_OK;
    }

    // The dynamic shared-memory limit is a property of the kernel function, shared by every plan:
    // raise it to the device's opt-in maximum (plans of different sizes coexist), after checking
    // that this plan's launches fit.
    template <int D> pat_status set_attrs() {
        cudaError_t e = cudaSuccess;
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (row_smem > (size_t)optin || spec_smem + 64 > (size_t)optin) {
            set_error("grid too large for the shared-memory kernels of this device");
            return PAT_EUNSUPPORTED;
        }
        auto seta = [&](const void* f, size_t) {
            if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        };
        seta((const void*)k_fwd_init<T, D>, row_smem);
        seta((const void*)k_fwd_u<T, D>, row_smem);
        seta((const void*)k_fwd_rho<T, D>, row_smem);
        seta((const void*)k_fwd_p<T, D>, row_smem);
        seta((const void*)k_adj_init<T, D>, row_smem);
        seta((const void*)k_adj_rho<T, D>, row_smem);
        seta((const void*)k_adj_u<T, D>, row_smem);
        seta((const void*)k_adj_p<T, D>, row_smem);
        seta((const void*)k_atd_a5_fwd<T, D>, row_smem);
        seta((const void*)k_atd_a5_inv<T, D>, row_smem);
        seta((const void*)k_spec<T, D, SPEC_PLAIN_FWD>, spec_smem);
        seta((const void*)k_spec<T, D, SPEC_PLAIN_INV>, spec_smem);
        seta((const void*)k_spec<T, D, SPEC_GRAD>, spec_smem);
        seta((const void*)k_spec<T, D, SPEC_DIV>, spec_smem);
        seta((const void*)k_spec<T, D, SPEC_ABS>, spec_smem);
        seta((const void*)k_spec<T, D, SPEC_DIVT>, spec_smem);
        seta((const void*)k_spec<T, D, SPEC_GRADT>, spec_smem);
        if (e == cudaSuccess && use_spec2) e = spec2_set_attrs<T>(optin);
        if (e == cudaSuccess && use_row2) e = row2_set_attrs<T>(optin);
        if constexpr (std::is_same<T, float>::value) {
            if (e == cudaSuccess && use_rowu1) e = rowu1_set_attrs(optin);
        }
        if (row2_smem > (size_t)optin) {
            set_error("grid too large for the shared-memory kernels of this device");
            return PAT_EINVAL;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute (shared memory)");
        return PAT_OK;
    }

    bool use_spec2 = false;
    bool use_row2 = false;
    bool use_rowu1 = false;   // the momentum row kernels with one velocity component per CTA
    int rowu1_pin = 0;        // PAT_ROWU1_LINES: x-lines per CTA of those kernels (0: rowu1_lines())
    // x-lines per CTA of the one-component momentum kernels: 16 where they divide the grid's lines (a
    // 256-thread CTA then has a butterfly per thread in every stage), else the row kernels' count
    int rowu1_lines() const {
        if (rowu1_pin > 0 && P.nlines % rowu1_pin == 0) return rowu1_pin;
        return (P.nlines % 16 == 0) ? 16 : cfg.row_lines;
    }
    size_t row2_smem = 0;

    // one step kernel of the row pass (Row2Kind): the register-fused power-of-two kernel, or the
    // generic one with its own argument list
    template <int D>
    void row_launch(int kind, const DevPlan<T>& Q, cudaStream_t s, int flag, T* data_row = nullptr,
                    const T* h_row = nullptr, T* qrow = nullptr, T* gc2 = nullptr, const T* p0c = nullptr) {
        const int R = cfg.row_lines, G = row_grid(), B = cfg.row_threads;
        if constexpr (std::is_same<T, float>::value) {
            if (use_rowu1 && D == 3 && (kind == R2_FWD_U || kind == R2_ADJ_U)) {
                cudaLaunchConfig_t lc = {};
                const int RU = rowu1_lines();
                lc.gridDim = dim3(P.nlines / RU, 3);
                lc.stream = s;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
                attr[0].val.programmaticStreamSerializationAllowed = 1;
                lc.attrs = attr;
                lc.numAttrs = 1;
                note_launch(rowu1_launch(&lc, kind == R2_ADJ_U, Q, RU, flag));
                return;
            }
        }
        if (use_row2) {
            cudaLaunchConfig_t lc = {};
            lc.gridDim = dim3(G);
            lc.blockDim = dim3(256);
            lc.dynamicSmemBytes = row2_smem;
            lc.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            lc.attrs = attr;
            lc.numAttrs = 1;
            note_launch(row2_launch<T>(&lc, D, kind, Q, R, flag, data_row, h_row, qrow, gc2, p0c));
            return;
        }
        switch (kind) {
            case R2_FWD_U: launch(k_fwd_u<T, D>, dim3(G), B, row_smem, s, Q, R, flag); break;
            case R2_FWD_RHO: launch(k_fwd_rho<T, D>, dim3(G), B, row_smem, s, Q, R, flag, data_row, qrow); break;
            case R2_FWD_P: launch(k_fwd_p<T, D>, dim3(G), B, row_smem, s, Q, R, flag, data_row, qrow); break;
            case R2_ADJ_RHO: launch(k_adj_rho<T, D>, dim3(G), B, row_smem, s, Q, R); break;
            case R2_ADJ_U: launch(k_adj_u<T, D>, dim3(G), B, row_smem, s, Q, R, flag); break;
            default: launch(k_adj_p<T, D>, dim3(G), B, row_smem, s, Q, R, flag, h_row, qrow, gc2, p0c); break;
        }
    }
    size_t spec_bytes(int D, int L, int w) const {
        return use_spec2 ? spec2_smem_bytes<T>(std::max(D, 2), L, w) : spec_smem_bytes<T>(D, L, w);
    }
    // a spectral tile of w columns stays inside the padded rows of the half spectra
    bool tile_fits(int w) const { return (size_t)((H.nxh + w - 1) / w) * w <= (size_t)H.ldh; }

    // ---------------------------------------------------------------------------------------
    // launch helpers (used while capturing, or directly on a stream)
    // ---------------------------------------------------------------------------------------
    int row_grid() const { return P.nlines / cfg.row_lines; }

    // The launchers of the power-of-two kernels return an error without touching CUDA's last-error
    // state when they have no kernel for the request; the first such error is kept here and
    // reported where the launches are checked (capture, direct runs).
    cudaError_t launch_err = cudaSuccess;
    void note_launch(cudaError_t e) {
        if (e != cudaSuccess && launch_err == cudaSuccess) launch_err = e;
    }
    cudaError_t take_launch_err() {
        const cudaError_t e = launch_err;
        launch_err = cudaSuccess;
        return e != cudaSuccess ? e : cudaGetLastError();
    }

    // Every kernel is launched with programmatic stream serialization: it may start (and run
    // its constant-data prologue) while its predecessor finishes; griddepcontrol.wait in the
    // kernel orders everything that depends on earlier kernels.
    template <typename... KArgs, typename... Args>
    void launch(void (*kern)(KArgs...), dim3 grid, int block, size_t smem, cudaStream_t s, Args... args) {
        cudaLaunchConfig_t lc = {};
        lc.gridDim = grid;
        lc.blockDim = dim3(block);
        lc.dynamicSmemBytes = smem;
        lc.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        lc.attrs = attr;
        lc.numAttrs = 1;
        cudaLaunchKernelEx(&lc, kern, args...);
    }

    // 3-D: each spectral operation runs its y / z / y passes chunk by chunk over the column tiles, so a
    // chunk's intermediate spectra can stay in L2 between the passes (1 = all tiles at once)
    int spec_chunks = 1;
    int spec_tiles() const { return (P.nxh + cfg.col_w - 1) / cfg.col_w; }
    int chunk_count() const { return std::max(1, std::min(spec_chunks, spec_tiles())); }

    template <int D, int MODE> void spec_launch(cudaStream_t s, int lax, int F, int t0 = 0, int nt = 0) {
        spec_launch_on<D, MODE>(P, s, lax, F, t0, nt);
    }
    // tiles t0 .. t0 + nt - 1 (nt = 0: all)
    template <int D, int MODE>
    void spec_launch_on(const DevPlan<T>& Q0, cudaStream_t s, int lax, int F, int t0 = 0, int nt = 0) {
        DevPlan<T> Q = Q0;
        Q.tile0 = t0;
        const int tiles = nt > 0 ? nt : (Q.nxh + cfg.col_w - 1) / cfg.col_w;
        const int outer = (lax == 1) ? Q.nz : Q.ny;
        int lgw = 0;
        while ((1 << lgw) < cfg.col_w) ++lgw;
        if (use_spec2) {
            // schedule 3: the field-wise multiply passes run their radix-16 stages with one thread per
            // butterfly of each field (128 per field of an 8-column tile)
            const bool fieldwise = (MODE == SPEC_DIV || MODE == SPEC_DIVT || MODE == SPEC_ABS);
            // (k_spec16 runs only in the kernels compiled for fixed line lengths; the others keep 256 threads)
            const bool wide = D == 3 && Q.spec16 == 3 && fieldwise && Q.stw16[lax] != nullptr && Q.fixed_len &&
                              cfg.col_w == 8;
            cudaLaunchConfig_t lc = {};
            lc.gridDim = dim3(tiles, outer);
            lc.blockDim = dim3(wide ? 128 * (MODE == SPEC_ABS ? 2 : D) : 256);
            // shared memory for the fields this launch holds (at most spec_smem)
            lc.dynamicSmemBytes = spec2_smem_bytes<T>(spec2_nf(D, MODE, F), lax == 1 ? H.ny : H.nz, cfg.col_w);
            lc.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            lc.attrs = attr;
            lc.numAttrs = 1;
            note_launch(spec2_launch<T>(&lc, D, MODE, Q, cfg.col_w, lgw, lax, F));
            return;
        }
        launch(k_spec<T, D, MODE>, dim3(tiles, outer), cfg.col_threads, spec_smem, s, Q, cfg.col_w, lgw, lax, F);
    }

    template <int D, int MODE> void spectral_on(const DevPlan<T>& Q, cudaStream_t s) {
        if (D == 2) {
            spec_launch_on<D, MODE>(Q, s, 1, 0);
            return;
        }
        spectral_chain<D, MODE>(Q, s, nullptr);
    }

    // 3-D spectral operation: y forward, z with the multiply, y inverse, chunk after chunk of the column
    // tiles; `name` != nullptr: probe marks
    // the register-resident z pass applies to this plan copy (its spectra are the ones the tensor maps
    // describe, 8-column tiles)
    bool zreg_ok(const DevPlan<T>& Q) const { return use_zreg && Q.use_tma && cfg.col_w == 8; }
    void zreg_launch_on(const DevPlan<T>& Q0, cudaStream_t s, int mode, int t0, int nt) {
        if constexpr (std::is_same<T, float>::value) {
            DevPlan<T> Q = Q0;
            Q.tile0 = t0;
            cudaLaunchConfig_t lc = {};
            lc.gridDim = dim3(nt, Q.ny);
            lc.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            lc.attrs = attr;
            lc.numAttrs = 1;
            note_launch(zreg_launch(&lc, mode, Q));
        } else {
            (void)Q0; (void)s; (void)mode; (void)t0; (void)nt;
        }
    }

    // the 16-column plain y transforms apply to this plan copy (the spectra of the tensor maps; the
    // two-stage schedule of the plain y transforms, whose arithmetic they share) when the tiles run in
    // one chunk
    bool ywide_ok(const DevPlan<T>& Q) const { return use_ywide && Q.use_tma && Q.spec16 >= 1 && chunk_count() == 1; }
    void ywide_launch_on(const DevPlan<T>& Q, cudaStream_t s, bool inverse, int F) {
        if constexpr (std::is_same<T, float>::value) {
            cudaLaunchConfig_t lc = {};
            lc.gridDim = dim3((Q.nxh + 15) / 16, Q.nz, F);
            lc.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            lc.attrs = attr;
            lc.numAttrs = 1;
            note_launch(ywide_launch(&lc, inverse, Q));
        } else {
            (void)Q; (void)s; (void)inverse; (void)F;
        }
    }

    // the 16-column z passes apply to this plan copy (the spectra of the tensor maps) when the tiles run
    // in one chunk
    bool zwide_ok(const DevPlan<T>& Q) const { return use_zwide && Q.use_tma && chunk_count() == 1; }
    // grid: one CTA per field of a tile for the field-wise passes, one per tile for D+ and its transpose;
    // the absorption pass reads its table unless the plan copy windows it (time reversal)
    void zwide_launch_on(const DevPlan<T>& Q, cudaStream_t s, int mode, int F) {
        if constexpr (std::is_same<T, float>::value) {
            const bool fieldwise = (mode == SPEC_DIV || mode == SPEC_DIVT || mode == SPEC_ABS);
            const float* mt = (mode != SPEC_ABS) ? kap3 : (Q.tr_kc2 > 0.f ? nullptr : abs3);
            cudaLaunchConfig_t lc = {};
            lc.gridDim = dim3(fieldwise ? F : 1, (Q.nxh + 15) / 16, Q.ny);
            lc.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            lc.attrs = attr;
            lc.numAttrs = 1;
            note_launch(zwide_launch(&lc, mode, Q, mt));
        } else {
            (void)Q; (void)s; (void)mode; (void)F;
        }
    }

    template <int D, int MODE> void spectral_chain(const DevPlan<T>& Q, cudaStream_t s, const char* name) {
        const int fin = (MODE == SPEC_GRAD) ? 1 : (MODE == SPEC_ABS ? 2 : D);
        const int fout = (MODE == SPEC_GRADT) ? 1 : (MODE == SPEC_ABS ? 2 : D);
        const int tiles = spec_tiles(), nc = chunk_count();
        for (int c = 0; c < nc; ++c) {
            const int t0 = (int)((long long)c * tiles / nc), t1 = (int)((long long)(c + 1) * tiles / nc);
            const bool yw = ywide_ok(Q);
            if (name) mark(s, "spec_y_fwd");
            if (yw) ywide_launch_on(Q, s, false, fin);
            else spec_launch_on<D, SPEC_PLAIN_FWD>(Q, s, 1, fin, t0, t1 - t0);
            if (name) mark(s, name);
            if (zwide_ok(Q)) zwide_launch_on(Q, s, MODE, fin);
            else if (zreg_ok(Q) && (zreg_all || MODE == SPEC_DIV || MODE == SPEC_DIVT)) zreg_launch_on(Q, s, MODE, t0, t1 - t0);
            else spec_launch_on<D, MODE>(Q, s, 2, 0, t0, t1 - t0);
            if (name) mark(s, "spec_y_inv");
            if (yw) ywide_launch_on(Q, s, true, fout);
            else spec_launch_on<D, SPEC_PLAIN_INV>(Q, s, 1, fout, t0, t1 - t0);
        }
    }

    // ---------------------------------------------------------------------------------------
    // smoothing S of the initial pressure (Sec. VI.A; pat_smooth.cu): x <- S x in place
    // ---------------------------------------------------------------------------------------
    cplx<T>* sm_Z = nullptr;   // complex workspace of N values (smooth_alloc)
    // allocate the workspace if it is missing: called when smoothing is switched on, so that the
    // solves themselves never allocate (they may run inside a caller's stream capture)
    pat_status smooth_alloc() {
        if (arena) {
            set_error("static-arena plans do not smooth p0");
            return PAT_EUNSUPPORTED;
        }
        if (!sm_Z) {
            pat_status st = PAT_OK;
            sm_Z = dalloc<cplx<T>>((size_t)P.N, &st);
            if (!sm_Z) return st;
        }
        return PAT_OK;
    }
    pat_status smooth_inplace(T* x, cudaStream_t s) {
        const pat_status ast = smooth_alloc();
        if (ast != PAT_OK) return ast;
        SmoothArgs<T> A{};
        A.d = H.d;
        A.nx = H.nx;
        A.ny = H.ny;
        A.nz = H.nz;
        A.ax[0] = P.fx;
        A.ax[1] = P.fy;
        A.ax[2] = P.fz;
        A.tw[0] = P.twx;
        A.tw[1] = P.twy;
        A.tw[2] = P.twz;
        const int n[3] = {H.nx, H.ny, H.nz};
        double kc = 0.0;
        for (int a = 0; a < 3; ++a) {
            A.dk[a] = 0.0;
            if (a >= H.d) continue;
            const double dx = in.grid.dx[a];
            A.dk[a] = 2.0 * M_PI / ((double)n[a] * dx);
            const double kn = M_PI / dx;
            kc = (a == 0) ? kn : std::min(kc, kn);
        }
        A.inv_kc2 = 1.0 / (kc * kc);
        A.invN = 1.0 / (double)P.N;
        A.Z = sm_Z;
        const cudaError_t e = smooth_apply<T>(A, x, s);
        return e == cudaSuccess ? PAT_OK : cuda_fail(e, "smoothing of p0");
    }

    // ---------------------------------------------------------------------------------------
    // medium gradient with checkpoints (direct launches of the per-phase kernels)
    // ---------------------------------------------------------------------------------------
    // forward step n -> n + 1 on the state of Q; q^{n+1} = d p^{n+1} / d c0^2 into qrow
    // (u_from_p0 = false: u^{-1/2} is the state in Q.u, not (dt/2) b D+ p^0)
    template <int D> void fwd_step_on(const DevPlan<T>& Q, int n, T* data_row, T* qrow, cudaStream_t s,
                                      bool u_from_p0 = true) {
        const int last = (n + 2 == H.Nt);
        spectral_on<D, SPEC_GRAD>(Q, s);
        row_launch<D>(R2_FWD_U, Q, s, (int)(n == 0 && u_from_p0));
        spectral_on<D, SPEC_DIV>(Q, s);
        row_launch<D>(R2_FWD_RHO, Q, s, last, data_row, nullptr, Q.lossy ? (T*)nullptr : qrow);
        if (Q.lossy) {
            spectral_on<D, SPEC_ABS>(Q, s);
            row_launch<D>(R2_FWD_P, Q, s, last, data_row, nullptr, qrow);
        }
    }
    // adjoint iteration that produces p_bar^n (the reverse of forward step n), accumulating
    // g_c2 += p_bar^n q^n (n >= 1) or, at n = 0, the initial-density term
    template <int D> void adj_step_on(int n, const T* qrow, T* gc2, const T* p0c, cudaStream_t s) {
        adj_step_q<D>(P, n, qrow, gc2, p0c, s);
    }
    // the same on the state of Q (P with the density-gradient hooks of this level set)
    template <int D> void adj_step_q(const DevPlan<T>& Q, int n, const T* qrow, T* gc2, const T* p0c, cudaStream_t s) {
        if (Q.lossy) {
            spectral_on<D, SPEC_ABS>(Q, s);
            row_launch<D>(R2_ADJ_RHO, Q, s, 0);
        }
        spectral_on<D, SPEC_DIVT>(Q, s);
        row_launch<D>(R2_ADJ_U, Q, s, (int)(n == 0));
        spectral_on<D, SPEC_GRADT>(Q, s);
        row_launch<D>(R2_ADJ_P, Q, s, (int)(n == 0), nullptr, (const T*)(Q.data + (size_t)n * H.Ns),
                      n == 0 ? (T*)nullptr : (T*)qrow, gc2, p0c);
    }

    // Medium gradients and grad_p0 = H^T h in one reverse sweep: g_c2 = d<H p0, h>/d c0^2 (readings
    // M1-M3) and g_rho = d<H p0, h>/d rho0 (readings D1-D3), either output optional.  Forward states
    // are checkpointed every K levels (levels 0, K, 2K, ...); each segment (jK, (j+1)K] is recomputed
    // from its checkpoint right before the adjoint iterations that consume it, storing q^n = dp^n/dc0^2
    // (c0^2 gradient) and g_xi = D+ p^n, e_xi = D- u^{n+1/2} of its steps (density gradient).
    //
    // The adjoint iteration of step n (level n -> n+1) reads g and e of step n; the lossless adjoint
    // tail that ends it does the density part of step n - 1 and reads e of step n - 1.  Segment j
    // recomputes steps lo .. hi-1 into slots 0 .. K-1 and its adjoint iterations run steps hi .. lo+1,
    // so step hi (slot 0 of segment j+1, recomputed earlier) is carried into slot K first.
    template <int D> pat_status gradient_medium(const void* p0, const void* h, void* gc2_out, void* grho_out,
                                                void* gp0_out, int K, cudaStream_t s) {
        const int Nt = H.Nt, Ns = H.Ns;
        const size_t N = (size_t)P.N, Nh = (size_t)H.nz * H.ny * H.ldh;
        const int nspec = std::max(D, 2);
        const int nseg = (Nt > 1) ? (Nt - 2) / K + 1 : 0;    // segments of levels 1 .. Nt-1
        const size_t ck_elems = 2 * D * N + Nh * 2;           // u, rho (real) and the p spectrum
        const bool want_c2 = gc2_out != nullptr, want_rho = grho_out != nullptr;
        const size_t ge_slot = 2 * (size_t)D * N;             // g_xi, e_xi of one step
        std::vector<void*> own;
        auto alloc = [&](size_t bytes) -> void* {
            void* ptr = nullptr;
            if (cudaMalloc(&ptr, bytes) != cudaSuccess) return nullptr;
            own.push_back(ptr);
            return ptr;
        };
        auto release = [&]() {
            cudaStreamSynchronize(s);
            for (void* ptr : own) cudaFree(ptr);
        };
        T* p0buf = (T*)alloc(N * sizeof(T));
        T* junk = (T*)alloc((size_t)std::max(Ns, 1) * sizeof(T));
        T* ckpt = (T*)alloc((size_t)std::max(nseg, 1) * ck_elems * sizeof(T));
        T* gc2 = nullptr;
        T* qbuf = nullptr;
        T* grho = nullptr;
        T* gbx = nullptr;
        T* gebuf = nullptr;
        bool ok = p0buf && junk && ckpt;
        if (ok && want_c2) {
            gc2 = (T*)alloc(N * sizeof(T));
            qbuf = (T*)alloc((size_t)std::max(1, std::min(K, Nt)) * N * sizeof(T));
            ok = gc2 && qbuf;
        }
        if (ok && want_rho) {
            grho = (T*)alloc(N * sizeof(T));
            gbx = (T*)alloc((size_t)D * N * sizeof(T));
            gebuf = (T*)alloc((size_t)(std::min(K, std::max(Nt - 1, 1)) + 1) * ge_slot * sizeof(T));
            ok = grho && gbx && gebuf;
        }
        DevPlan<T> Pf = P;
        Pf.use_tma = 0;   // its spectra are other buffers than the tensor maps describe
        for (int a = 0; a < D && ok; ++a) {
            ok = ok && (Pf.u[a] = (T*)alloc(N * sizeof(T))) && (Pf.rh[a] = (T*)alloc(N * sizeof(T)));
        }
        if (ok && P.lossy) ok = (Pf.rsum = (T*)alloc(N * sizeof(T))) != nullptr;
        for (int a = 0; a < nspec && ok; ++a) {
            ok = (Pf.spec[a] = (cplx<T>*)alloc(Nh * sizeof(cplx<T>))) != nullptr;
            if (ok) ok = cudaMemsetAsync(Pf.spec[a], 0, Nh * sizeof(cplx<T>), s) == cudaSuccess;
        }
        if (!ok) {
            cudaGetLastError();
            release();
            set_error("out of device memory for the checkpointed gradient");
            return PAT_ENOMEM;
        }
        Pf.img = p0buf;
        Pf.data = junk;
        cudaError_t e = cudaMemcpyAsync(p0buf, p0, N * sizeof(T), cudaMemcpyDefault, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(P.data, h, (size_t)Nt * Ns * sizeof(T), cudaMemcpyDefault, s);
        if (e == cudaSuccess && gc2) e = cudaMemsetAsync(gc2, 0, N * sizeof(T), s);
        if (e == cudaSuccess && grho) e = cudaMemsetAsync(grho, 0, N * sizeof(T), s);
        if (e == cudaSuccess && gbx) e = cudaMemsetAsync(gbx, 0, (size_t)D * N * sizeof(T), s);
        for (int a = 0; a < D && e == cudaSuccess; ++a) {
            e = cudaMemsetAsync(P.u[a], 0, N * sizeof(T), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(P.rh[a], 0, N * sizeof(T), s);
        }
        if (e != cudaSuccess) {
            release();
            return cuda_fail(e, "gradient setup");
        }
        if (smooth) {   // the initial pressure is S p0 (Sec. VI.A)
            const pat_status sst = smooth_inplace(p0buf, s);
            if (sst != PAT_OK) {
                release();
                return sst;
            }
        }
        const int R = cfg.row_lines, G = row_grid(), B = cfg.row_threads;
        auto save = [&](int j) {
            T* c = ckpt + (size_t)j * ck_elems;
            for (int a = 0; a < D; ++a) {
                cudaMemcpyAsync(c + (size_t)a * N, Pf.u[a], N * sizeof(T), cudaMemcpyDeviceToDevice, s);
                cudaMemcpyAsync(c + (size_t)(D + a) * N, Pf.rh[a], N * sizeof(T), cudaMemcpyDeviceToDevice, s);
            }
            cudaMemcpyAsync(c + 2 * D * N, Pf.spec[0], Nh * sizeof(cplx<T>), cudaMemcpyDeviceToDevice, s);
        };
        auto restore = [&](int j) {
            const T* c = ckpt + (size_t)j * ck_elems;
            for (int a = 0; a < D; ++a) {
                cudaMemcpyAsync(Pf.u[a], c + (size_t)a * N, N * sizeof(T), cudaMemcpyDeviceToDevice, s);
                cudaMemcpyAsync(Pf.rh[a], c + (size_t)(D + a) * N, N * sizeof(T), cudaMemcpyDeviceToDevice, s);
            }
            cudaMemcpyAsync(Pf.spec[0], c + 2 * D * N, Nh * sizeof(cplx<T>), cudaMemcpyDeviceToDevice, s);
        };
        // density hooks: slot k of gebuf holds g_xi (xi < D) then e_xi of step lo + k
        auto gslot = [&](int k, int a) { return gebuf + (size_t)k * ge_slot + (size_t)a * N; };
        auto eslot = [&](int k, int a) { return gebuf + (size_t)k * ge_slot + (size_t)(D + a) * N; };
        auto fwd_hooks = [&](DevPlan<T>& Q, int k) {
            for (int a = 0; a < 3; ++a) {
                Q.hk_g[a] = (want_rho && a < D) ? gslot(k, a) : nullptr;
                Q.hk_e[a] = (want_rho && a < D) ? eslot(k, a) : nullptr;
            }
        };
        // adjoint hooks of the iteration of step n in a segment starting at lo (lossless tails read
        // e of step n - 1)
        auto adj_hooks = [&](int n, int lo) {
            DevPlan<T> Q = P;
            if (!want_rho) return Q;
            const int ke = P.lossy ? n - lo : std::max(n - 1 - lo, 0);
            for (int a = 0; a < D; ++a) {
                Q.hk_gin[a] = gslot(n - lo, a);
                Q.hk_ein[a] = eslot(ke, a);
                Q.hk_gb[a] = gbx + (size_t)a * N;
            }
            Q.hk_grho = grho;
            return Q;
        };
        // (1) forward sweep to level (nseg - 1) K, checkpointing levels 0, K, ...
        launch(k_fwd_init<T, D>, dim3(G), B, row_smem, s, Pf, R, (int)(Nt == 1));
        if (nseg > 0) save(0);
        for (int n = 0; n < (nseg - 1) * K; ++n) {
            fwd_step_on<D>(Pf, n, junk, (T*)nullptr, s);
            if ((n + 1) % K == 0) save((n + 1) / K);
        }
        // (2) reverse sweep, segment by segment
        if (Nt == 1) {
            launch(k_adj_init<T, D>, dim3(G), B, row_smem, s, P, R, 1, (const T*)(P.data), (const T*)nullptr, gc2,
                   (const T*)p0buf);
        }
        for (int j = nseg - 1; j >= 0; --j) {
            const int lo = j * K, hi = std::min((j + 1) * K, Nt - 1);
            if (want_rho && j < nseg - 1)   // step hi = slot 0 of the segment above -> slot hi - lo
                for (int a = 0; a < 2 * D; ++a)
                    cudaMemcpyAsync(gebuf + (size_t)(hi - lo) * ge_slot + (size_t)a * N, gebuf + (size_t)a * N,
                                    N * sizeof(T), cudaMemcpyDeviceToDevice, s);
            restore(j);
            for (int n = lo; n < hi; ++n) {
                DevPlan<T> Q = Pf;
                fwd_hooks(Q, n - lo);
                fwd_step_on<D>(Q, n, junk, qbuf ? qbuf + (size_t)(n - lo) * N : (T*)nullptr, s);
            }
            int top = hi;
            if (hi == Nt - 1) {
                DevPlan<T> Q = adj_hooks(Nt - 1, lo);   // lossless tail: density part of step Nt - 2
                launch(k_adj_init<T, D>, dim3(G), B, row_smem, s, Q, R, 0, (const T*)(P.data + (size_t)(Nt - 1) * Ns),
                       (const T*)(qbuf ? qbuf + (size_t)(hi - lo - 1) * N : nullptr), gc2, (const T*)p0buf);
                top = Nt - 2;
            }
            for (int n = top; n > lo; --n)
                adj_step_q<D>(adj_hooks(n, lo), n, qbuf ? qbuf + (size_t)(n - lo - 1) * N : nullptr, gc2, p0buf, s);
        }
        if (Nt > 1) adj_step_q<D>(adj_hooks(0, 0), 0, nullptr, gc2, p0buf, s);
        if (want_rho) {   // through b_xi = 2 / (rho0 + rho0 shifted along xi) (reading D3)
            const int threads = 256;
            const int blocks = (int)std::min<size_t>((N + threads - 1) / threads, 8192);
            k_rho_chain<T><<<blocks, threads, 0, s>>>(P, (const T*)gbx, grho);
        }
        e = take_launch_err();
        if (e == cudaSuccess && gp0_out && smooth) {   // (H S)^T = S H^T
            const pat_status sst = smooth_inplace(P.img, s);
            if (sst != PAT_OK) {
                release();
                return sst;
            }
        }
        if (e == cudaSuccess && gc2_out) e = cudaMemcpyAsync(gc2_out, gc2, N * sizeof(T), cudaMemcpyDefault, s);
        if (e == cudaSuccess && grho_out) e = cudaMemcpyAsync(grho_out, grho, N * sizeof(T), cudaMemcpyDefault, s);
        if (e == cudaSuccess && gp0_out) e = cudaMemcpyAsync(gp0_out, P.img, N * sizeof(T), cudaMemcpyDefault, s);
        release();
        if (e != cudaSuccess) return cuda_fail(e, "checkpointed gradient");
        return PAT_OK;
    }

    // ---------------------------------------------------------------------------------------
    // time reversal (Sec. II.B.1, readings T1-T5) and the adjoint-then-discretize adjoint (Sec. III,
    // readings A1-A5): forward-direction solves with direct launches of the per-phase kernels on the
    // plan's own state, with the kernels' hooks set in a copy of the device plan
    // ---------------------------------------------------------------------------------------
    int* tr_node_d = nullptr;    // [N] sensor enforced at each node (-1: none), built on first use
    int* tr_list_d = nullptr;    // [Ns] node of each sensor
    T* aux_rows = nullptr;       // [max(Nt - 1, 1) + 1][Ns]: ATD source rows, then one spare row

    // the node of every sensor, when each sensor is exactly one grid node with weight 1 and no two
    // share a node (reading T2)
    pat_status tr_nodes(std::vector<int>& node) {
        const int Ns = H.Ns;
        node.assign((size_t)Ns, -1);
        std::vector<int> cnt((size_t)Ns, 0);
        for (int line = 0; line < P.nlines; ++line)
            for (int q = H.g_lineptr[line]; q < H.g_lineptr[line + 1]; ++q) {
                const int j = H.g_seg_sensor[q];
                const double w0 = H.g_seg_w0[q], w1 = H.g_seg_w1[q];
                const long long base = (long long)H.g_seg_line[q] * H.nx + H.g_seg_x0[q];
                if (w0 != 0.0) {
                    ++cnt[j];
                    if (w0 != 1.0) cnt[j] = 99;
                    node[j] = (int)base;
                }
                if (w1 != 0.0) {
                    ++cnt[j];
                    if (w1 != 1.0) cnt[j] = 99;
                    node[j] = (int)(base + 1);
                }
            }
        std::vector<char> used((size_t)P.N, 0);
        for (int j = 0; j < Ns; ++j) {
            if (cnt[j] != 1 || node[j] < 0) {
                set_error("time reversal needs every sensor on one grid node (on-grid sensors)");
                return PAT_EINVAL;
            }
            if (used[(size_t)node[j]]) {
                set_error("time reversal needs one sensor per grid node");
                return PAT_EINVAL;
            }
            used[(size_t)node[j]] = 1;
        }
        return PAT_OK;
    }

    pat_status aux_alloc(bool tr) {
        pat_status st = PAT_OK;
        if (!aux_rows) {
            aux_rows = dalloc<T>((size_t)(std::max(H.Nt - 1, 1) + 1) * std::max(H.Ns, 1), &st);
            if (!aux_rows) return st;
        }
        if (tr && !tr_node_d) {
            std::vector<int> node;
            st = tr_nodes(node);
            if (st != PAT_OK) return st;
            std::vector<int> map((size_t)P.N, -1);
            for (int j = 0; j < H.Ns; ++j) map[(size_t)node[j]] = j;
            int* m = dalloc<int>((size_t)P.N, &st);
            if (!m) return st;
            int* l = dalloc<int>((size_t)std::max(H.Ns, 1), &st);
            if (!l) return st;
            cudaError_t e = cudaMemcpy(m, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice);
            if (e == cudaSuccess && H.Ns > 0)
                e = cudaMemcpy(l, node.data(), node.size() * sizeof(int), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy (time-reversal nodes)");
            tr_node_d = m;
            tr_list_d = l;
        }
        return PAT_OK;
    }

    // image = p at the end of the reversed-time solve with the data enforced at the sensor nodes
    template <int D> pat_status time_reversal(const void* data, void* img_out, int compensate, double k_cut,
                                              cudaStream_t s) {
        pat_status st = aux_alloc(true);
        if (st != PAT_OK) return st;
        const int Nt = H.Nt, Ns = H.Ns;
        const size_t N = (size_t)P.N;
        const int R = cfg.row_lines, G = row_grid(), B = cfg.row_threads;
        T* junk = aux_rows;   // gathered samples of the solve (not used)
        cudaError_t e = cudaMemcpyAsync(P.data, data, (size_t)Nt * Ns * sizeof(T), cudaMemcpyDefault, s);
        for (int a = 0; a < D && e == cudaSuccess; ++a) e = cudaMemsetAsync(P.u[a], 0, N * sizeof(T), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(P.img, 0, N * sizeof(T), s);
        if (e != cudaSuccess) return cuda_fail(e, "time reversal setup");
        // p^0: zero except the last datum at the sensor nodes (T3)
        if (Ns > 0)
            k_tr_start<T><<<(Ns + 255) / 256, 256, 0, s>>>(P.img, tr_list_d, P.data + (size_t)(Nt - 1) * Ns, Ns);
        DevPlan<T> Q = P;
        Q.data = junk;
        Q.spec16 = std::min(Q.spec16, 1);
        if (compensate) {
            double kc = 0.0;
            for (int a = 0; a < D; ++a) {
                const double kn = M_PI / in.grid.dx[a];
                kc = (a == 0) ? kn : std::min(kc, kn);
            }
            kc *= k_cut;
            Q.tr_kc2 = (T)(1.0 / (kc * kc));
        }
        Q.tr_node = tr_node_d;
        // rho^0 = p^0 / (d c0^2), x-FFT of p^0 (its sample goes to the unused row)
        launch(k_fwd_init<T, D>, dim3(G), B, row_smem, s, Q, R, (int)(Nt == 1));
        for (int n = 0; n + 1 < Nt; ++n) {
            Q.tr_row = P.data + (size_t)(Nt - 2 - n) * Ns;
            Q.tr_img = (n + 2 == Nt) ? P.img : nullptr;
            fwd_step_on<D>(Q, n, junk, nullptr, s, false);
        }
        e = take_launch_err();
        if (e == cudaSuccess) e = cudaMemcpyAsync(img_out, P.img, N * sizeof(T), cudaMemcpyDefault, s);
        if (e != cudaSuccess) return cuda_fail(e, "time reversal");
        return PAT_OK;
    }

    // the paper's adjoint: the continuous adjoint system discretised with the same scheme, run forward
    // in adjoint time on the reversed data (A1-A2); initial_paper = 1: rho*(T) / rho0 (Eq. (adjj)),
    // 0: the gradient for the forward map's initial state (A5)
    template <int D> pat_status adjoint_atd(const void* resid, void* img_out, int initial_paper, cudaStream_t s) {
        pat_status st = aux_alloc(false);
        if (st != PAT_OK) return st;
        const int Nt = H.Nt, Ns = H.Ns;
        const size_t N = (size_t)P.N, Nh = (size_t)H.nz * H.ny * H.ldh;
        const int R = cfg.row_lines, G = row_grid(), B = cfg.row_threads;
        T* junk = aux_rows + (size_t)std::max(Nt - 1, 1) * std::max(Ns, 1);
        cudaError_t e = cudaMemcpyAsync(P.data, resid, (size_t)Nt * Ns * sizeof(T), cudaMemcpyDefault, s);
        if (e != cudaSuccess) return cuda_fail(e, "copy residual");
        // source rows s^n = (h~^n + h~^{n+1}) / 2 = (h^{Nt-1-n} + h^{Nt-2-n}) / 2 (A2)
        if (Nt > 1 && Ns > 0) {
            const long long cnt = (long long)(Nt - 1) * Ns;
            k_atd_source<T><<<(int)std::min<long long>((cnt + 255) / 256, 4096), 256, 0, s>>>(aux_rows, P.data, Nt, Ns);
        }
        // zero state: u*, rho*, p* (its spectrum feeds the first gradient)
        for (int a = 0; a < D && e == cudaSuccess; ++a) {
            e = cudaMemsetAsync(P.u[a], 0, N * sizeof(T), s);
            if (e == cudaSuccess) e = cudaMemsetAsync(P.rh[a], 0, N * sizeof(T), s);
        }
        for (int a = 0; a < std::max(D, 2) && e == cudaSuccess; ++a)
            e = cudaMemsetAsync(P.spec[a], 0, Nh * sizeof(cplx<T>), s);
        if (e != cudaSuccess) return cuda_fail(e, "adjoint-then-discretize setup");
        DevPlan<T> Q = P;
        Q.data = junk;
        Q.atd = 1;
        for (int n = 0; n + 1 < Nt; ++n) {
            Q.atd_row = aux_rows + (size_t)n * Ns;
            fwd_step_on<D>(Q, n, junk, nullptr, s, false);
        }
        // g = sum_xi rho*_xi / rho0 (Eq. (adjj)); for the forward map's initial state (A5),
        // g - L_{y-1}(c0^2 eta g) / c0^2, the fractional Laplacian by one more absorption pass
        const bool a5 = !initial_paper && P.lossy;
        const int threads = 256;
        const int blocks = (int)std::min<size_t>((N + threads - 1) / threads, 8192);
        k_atd_image<T><<<blocks, threads, 0, s>>>(P, P.img);
        if (a5) {
            // channels (0, c0^2 eta g) through x-transform, the absorption pass of the spectral kernels
            // (channel 1 gets |k|^(y-1)), inverse x-transform, then g - (channel 1) / c0^2
            launch(k_atd_a5_fwd<T, D>, dim3(G), B, row_smem, s, P, R);
            spectral_on<D, SPEC_ABS>(P, s);
            launch(k_atd_a5_inv<T, D>, dim3(G), B, row_smem, s, P, R);
        }
        e = take_launch_err();
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess && smooth) {   // (H S)^T = S H^T (reading R9)
            const pat_status sst = smooth_inplace(P.img, s);
            if (sst != PAT_OK) return sst;
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(img_out, P.img, N * sizeof(T), cudaMemcpyDefault, s);
        if (e != cudaSuccess) return cuda_fail(e, "adjoint-then-discretize");
        return PAT_OK;
    }

    // --- kernel-timing probe -----------------------------------------------------------------
    // While recording a sampled step, `mark` records one event before each launch (and one after
    // the last); names are collected on the first sampled step.
    int probe_g = -1;         // graph being recorded (0 fwd, 1 adj) when sampling, else -1
    size_t probe_next = 0;    // next event of probe_ev[probe_g]
    bool probe_first = false;
    void mark(cudaStream_t s, const char* name) {
        if (probe_g < 0) return;
        if (probe_next >= probe_ev[probe_g].size()) {
            cudaEvent_t ev;
            cudaEventCreate(&ev);
            probe_ev[probe_g].push_back(ev);
        }
        // inside stream capture only an "external" record becomes an event-record node
        cudaEventRecordWithFlags(probe_ev[probe_g][probe_next++], s, cudaEventRecordExternal);
        if (probe_first && name) probe_names[probe_g].push_back(name);
    }
    bool sampled(int n, int Nt) const {
        if (probe_stride <= 0) return false;
        return n >= probe_stride / 2 && (n - probe_stride / 2) % probe_stride == 0 && n + 1 < Nt;
    }
    void begin_sample(int g, bool first) {
        probe_g = g;
        probe_first = first;
    }
    void end_sample(cudaStream_t s) {
        mark(s, nullptr);
        probe_g = -1;
        probe_first = false;
    }

    template <int D, int MODE> void spectral_named(cudaStream_t s, const char* name) {
        if (D == 2) {
            mark(s, name);
            spec_launch<D, MODE>(s, 1, 0);
            return;
        }
        spectral_chain<D, MODE>(P, s, name);
    }

    template <int D> void record_forward(cudaStream_t s) {
        const int R = cfg.row_lines, G = row_grid(), B = cfg.row_threads;
        const int Nt = H.Nt, Ns = H.Ns;
        probe_next = 0;
        probe_names[0].clear();
        probe_samples[0] = 0;
        cudaMemsetAsync(P.data, 0, (size_t)Nt * Ns * sizeof(T), s);
        launch(k_fwd_init<T, D>, dim3(G), B, row_smem, s, P, R, (int)(Nt == 1));
        for (int n = 0; n + 1 < Nt; ++n) {
            const int last = (n + 2 == Nt);
            T* row = P.data + (size_t)(n + 1) * Ns;
            if (sampled(n, Nt)) begin_sample(0, probe_samples[0]++ == 0);
            spectral_named<D, SPEC_GRAD>(s, "spec_grad");
            mark(s, "fwd_u");
            row_launch<D>(R2_FWD_U, P, s, (int)(n == 0));
            spectral_named<D, SPEC_DIV>(s, "spec_div");
            mark(s, "fwd_rho");
            row_launch<D>(R2_FWD_RHO, P, s, last, row);
            if (P.lossy) {
                spectral_named<D, SPEC_ABS>(s, "spec_abs");
                mark(s, "fwd_p");
                row_launch<D>(R2_FWD_P, P, s, last, row);
            }
            if (probe_g >= 0) end_sample(s);
        }
    }

    template <int D> void record_adjoint(cudaStream_t s) {
        const int R = cfg.row_lines, G = row_grid(), B = cfg.row_threads;
        const int Nt = H.Nt, Ns = H.Ns;
        const size_t N = (size_t)P.N;
        for (int a = 0; a < D; ++a) {
            cudaMemsetAsync(P.u[a], 0, N * sizeof(T), s);
            cudaMemsetAsync(P.rh[a], 0, N * sizeof(T), s);
        }
        probe_next = 0;
        probe_names[1].clear();
        probe_samples[1] = 0;
        launch(k_adj_init<T, D>, dim3(G), B, row_smem, s, P, R, (int)(Nt == 1),
               (const T*)(P.data + (size_t)(Nt - 1) * Ns), (const T*)nullptr, (T*)nullptr, (const T*)nullptr);
        for (int n = Nt - 2; n >= 0; --n) {
            if (sampled(n, Nt)) begin_sample(1, probe_samples[1]++ == 0);
            if (P.lossy) {
                spectral_named<D, SPEC_ABS>(s, "spec_abs");
                mark(s, "adj_rho");
                row_launch<D>(R2_ADJ_RHO, P, s, 0);
            }
            spectral_named<D, SPEC_DIVT>(s, "spec_divt");
            mark(s, "adj_u");
            row_launch<D>(R2_ADJ_U, P, s, (int)(n == 0));
            spectral_named<D, SPEC_GRADT>(s, "spec_gradt");
            mark(s, "adj_p");
            row_launch<D>(R2_ADJ_P, P, s, (int)(n == 0), nullptr, (const T*)(P.data + (size_t)n * Ns));
            if (probe_g >= 0) end_sample(s);
        }
    }

    pat_status capture(bool adjoint, cudaGraphExec_t* out) {
        cudaGraph_t g = nullptr;
        pat_status st = capture_graph(adjoint, &g);
        if (st != PAT_OK) return st;
        cudaError_t e = cudaGraphInstantiate(out, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        return PAT_OK;
    }

    // the per-phase solve as a (not instantiated) graph; the caller owns *out
    pat_status capture_graph(bool adjoint, cudaGraph_t* out) {
        cudaError_t e = cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        if (P.d == 2) {
            if (adjoint) record_adjoint<2>(cap_stream);
            else record_forward<2>(cap_stream);
        } else {
            if (adjoint) record_adjoint<3>(cap_stream);
            else record_forward<3>(cap_stream);
        }
        cudaError_t le = take_launch_err();
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cap_stream, &g);
        if (le != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(le, "kernel launch during capture");
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        *out = g;
        return PAT_OK;
    }
};

template <typename T> PlanBase* make_plan(const HostTables& h, pat_status* st, unsigned char* arena = nullptr,
                                          size_t arena_cap = 0) {
    if (arena) {
        // sizing pass: reject a problem that does not fit before any device memory is touched
        Plan<T> sizing;
        sizing.arena = arena;
        sizing.arena_cap = arena_cap;
        sizing.count_only = true;
        *st = sizing.build(h);
        if (*st != PAT_OK) return nullptr;
        if (sizing.arena_used > arena_cap) {
            *st = PAT_EINVAL;
            set_error("problem too large for the static scratch array: needs " + std::to_string(sizing.arena_used) +
                      " bytes, the array holds " + std::to_string(arena_cap));
            return nullptr;
        }
    }
    Plan<T>* p = new Plan<T>();
    p->arena = arena;
    p->arena_cap = arena_cap;
    p->info = h.info;
    cudaGetDevice(&p->device);
    *st = p->build(h);
    if (*st != PAT_OK) {
        delete p;
        return nullptr;
    }
    return p;
}

PlanBase* make_plan_f32(const HostTables& h, pat_status* st) { return make_plan<float>(h, st); }
PlanBase* make_plan_f64(const HostTables& h, pat_status* st) { return make_plan<double>(h, st); }

PlanBase* make_plan_arena(const HostTables& h, unsigned char* arena, size_t cap, pat_status* st) {
    if (h.info.precision == PAT_F32) return make_plan<float>(h, st, arena, cap);
    return make_plan<double>(h, st, arena, cap);
}

template <typename T> static pat_status run_direct_t(Plan<T>* p, cudaStream_t s) {
    if (p->P.d == 2) p->template record_forward<2>(s);
    else p->template record_forward<3>(s);
    cudaError_t e = p->take_launch_err();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return PAT_OK;
}

pat_status plan_forward_direct(PlanBase* base, cudaStream_t s) {
    if (base->info.precision == PAT_F32) return run_direct_t(static_cast<Plan<float>*>(base), s);
    return run_direct_t(static_cast<Plan<double>*>(base), s);
}

pat_status plan_probe_read(PlanBase* b, int g, int slot, const char** name, double* mean_ms, int* samples) {
    const int slots = (int)b->probe_names[g].size();
    if (slot < 0 || slot >= slots) return PAT_EINVAL;
    const int ns = b->probe_samples[g];
    double sum = 0.0;
    int cnt = 0;
    for (int k = 0; k < ns; ++k) {
        const size_t e0 = (size_t)k * (slots + 1) + slot;
        if (e0 + 1 >= b->probe_ev[g].size()) break;
        float ms = 0.f;
        cudaError_t e = cudaEventElapsedTime(&ms, b->probe_ev[g][e0], b->probe_ev[g][e0 + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime (probe)");
        sum += ms;
        ++cnt;
    }
    *name = b->probe_names[g][slot].c_str();
    *mean_ms = cnt ? sum / cnt : 0.0;
    *samples = cnt;
    return PAT_OK;
}

pat_status plan_gradient_medium(PlanBase* base, const void* p0, const void* h, void* gc2, void* grho, void* gp0,
                                int K, cudaStream_t s) {
    if (base->info.precision == PAT_F32) {
        auto* p = static_cast<Plan<float>*>(base);
        return p->P.d == 2 ? p->template gradient_medium<2>(p0, h, gc2, grho, gp0, K, s)
                           : p->template gradient_medium<3>(p0, h, gc2, grho, gp0, K, s);
    }
    auto* p = static_cast<Plan<double>*>(base);
    return p->P.d == 2 ? p->template gradient_medium<2>(p0, h, gc2, grho, gp0, K, s)
                       : p->template gradient_medium<3>(p0, h, gc2, grho, gp0, K, s);
}

pat_status plan_time_reversal(PlanBase* base, const void* data, void* img, int compensate, double k_cut,
                              cudaStream_t s) {
    if (base->info.precision == PAT_F32) {
        auto* p = static_cast<Plan<float>*>(base);
        return p->P.d == 2 ? p->template time_reversal<2>(data, img, compensate, k_cut, s)
                           : p->template time_reversal<3>(data, img, compensate, k_cut, s);
    }
    auto* p = static_cast<Plan<double>*>(base);
    return p->P.d == 2 ? p->template time_reversal<2>(data, img, compensate, k_cut, s)
                       : p->template time_reversal<3>(data, img, compensate, k_cut, s);
}

pat_status plan_adjoint_atd(PlanBase* base, const void* resid, void* img, int initial_paper, cudaStream_t s) {
    if (base->info.precision == PAT_F32) {
        auto* p = static_cast<Plan<float>*>(base);
        return p->P.d == 2 ? p->template adjoint_atd<2>(resid, img, initial_paper, s)
                           : p->template adjoint_atd<3>(resid, img, initial_paper, s);
    }
    auto* p = static_cast<Plan<double>*>(base);
    return p->P.d == 2 ? p->template adjoint_atd<2>(resid, img, initial_paper, s)
                       : p->template adjoint_atd<3>(resid, img, initial_paper, s);
}

pat_status plan_set_fault(PlanBase* base, unsigned barrier_extra, double wait_limit_s) {
    const unsigned long long ns = (unsigned long long)(wait_limit_s * 1e9);
    if (base->info.precision == PAT_F32) {
        auto* p = static_cast<Plan<float>*>(base);
        p->P.bar_extra = barrier_extra;
        p->P.bar_limit_ns = ns;
    } else {
        auto* p = static_cast<Plan<double>*>(base);
        p->P.bar_extra = barrier_extra;
        p->P.bar_limit_ns = ns;
    }
    return PAT_OK;
}

// PAT_ENONFINITE into *flag if x[0 .. n) holds a NaN or an infinity
template <typename T> __global__ void k_finite_check(const T* x, long long n, unsigned* flag) {
    bool bad = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        bad |= !isfinite(x[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(flag, (unsigned)PAT_ENONFINITE);
}

template <typename T> static pat_status finite_check_t(PlanBase* b, bool adjoint, cudaStream_t s) {
    const long long n = adjoint ? b->info.N : (long long)b->info.Nt * b->info.Ns;
    const T* x = static_cast<const T*>(adjoint ? b->img_ptr : b->data_ptr);
    const int grid = (int)std::min<long long>(1024, (n + 255) / 256);
    k_finite_check<T><<<std::max(grid, 1), 256, 0, s>>>(x, n, b->fstat);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PAT_OK : cuda_fail(e, "non-finite check");
}

pat_status plan_clear_finite(PlanBase* b, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b->fstat, 0, sizeof(unsigned), s);
    return e == cudaSuccess ? PAT_OK : cuda_fail(e, "cudaMemsetAsync (status)");
}

pat_status plan_finite_check(PlanBase* b, bool adjoint, cudaStream_t s) {
    if (b->info.precision == PAT_F32) return finite_check_t<float>(b, adjoint, s);
    return finite_check_t<double>(b, adjoint, s);
}

pat_status plan_smooth_alloc(PlanBase* base) {
    if (base->info.precision == PAT_F32) return static_cast<Plan<float>*>(base)->smooth_alloc();
    return static_cast<Plan<double>*>(base)->smooth_alloc();
}

pat_status plan_smooth(PlanBase* base, void* x, cudaStream_t s) {
    if (base->info.precision == PAT_F32) return static_cast<Plan<float>*>(base)->smooth_inplace((float*)x, s);
    return static_cast<Plan<double>*>(base)->smooth_inplace((double*)x, s);
}

pat_status plan_run_persistent(PlanBase* base, bool adjoint, cudaStream_t s) {
    if (base->info.precision == PAT_F32) return static_cast<Plan<float>*>(base)->run_persistent(adjoint, s);
    return static_cast<Plan<double>*>(base)->run_persistent(adjoint, s);
}

pat_status plan_capture_graph(PlanBase* base, bool adjoint, cudaGraph_t* out) {
    if (base->info.precision == PAT_F32) return static_cast<Plan<float>*>(base)->capture_graph(adjoint, out);
    return static_cast<Plan<double>*>(base)->capture_graph(adjoint, out);
}

pat_status plan_capture(PlanBase* base, bool adjoint) {
    cudaGraphExec_t* slot = adjoint ? &base->adj_exec : &base->fwd_exec;
    if (*slot) return PAT_OK;
    if (base->info.precision == PAT_F32) return static_cast<Plan<float>*>(base)->capture(adjoint, slot);
    return static_cast<Plan<double>*>(base)->capture(adjoint, slot);
}

}  // namespace pat
