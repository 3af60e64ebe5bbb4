// C ABI entry points of libhmg (declared and documented in include/hmg.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/hmg.h"
#include "hmg_internal.h"
#include "hmg_runtime.h"
#include "hmg_server.h"

using namespace hmg;

namespace {

hmg_status cuda_status(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return HMG_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return HMG_CUDA_ERROR;
}

hmg_status check_launch(hmg_ctx* ctx, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return cuda_status(e, what);
}

bool check_k(double km, double ki, double kc) {
    for (double k : {km, ki, kc})
        if (!(std::isfinite(k) && k > 0.0)) return false;
    return true;
}

hmg_status check_common(hmg_ctx* ctx, int N, const void* p) {
    if (!ctx) {
        set_error("null context");
        return HMG_INVALID_ARG;
    }
    if (!valid_N(N)) {
        set_error("N = %d: need an even N = 2^a 3^b with 8 <= N <= 512", N);
        return HMG_INVALID_ARG;
    }
    if (!p) {
        set_error("null pointer argument");
        return HMG_INVALID_ARG;
    }
    return HMG_OK;
}

// Bring the phase grid onto the device and build the solve descriptor.
hmg_status prepare(hmg_ctx* ctx, const uint8_t* phase, int N, const double k[3], bool fp64, int nslots,
                   GridDesc* g, int scheme = HMG_SCHEME_EYRE_MILTON, double beta = 2.0) {
    auto gp = ctx->plan(N);
    if (!gp) {
        set_error("cannot allocate FFT tables");
        return HMG_OUT_OF_MEMORY;
    }
    if (!ctx->solve.ensure(ctx, N, fp64, nslots)) {
        set_error("cannot allocate solve state for N = %d (%zu bytes, budget %zu)", N,
                  state_bytes(N, fp64, nslots), ctx->budget);
        return HMG_OUT_OF_MEMORY;
    }
    const size_t N3 = (size_t)N * N * N;
    hmg_status st = cuda_status(copy_in(ctx->solve.phase, phase, N3, ctx->stream), "phase copy");
    if (st != HMG_OK) return st;
    *g = make_desc(*gp, fp64, k, ctx->solve.phase, nslots, scheme, beta);
    if (!fp64) {
        const int v = autotune_z(ctx, *g, &ctx->solve, ctx->stream);
        g->zvar = v & 1;
        g->xyvar = (v >> 1) & 1;
        g->nochain = (v >> 2) & 1;
        g->xpers = (v >> 3) & 1;
        g->zpers = (v >> 4) & 1;
        g->yxy = (v >> 5) & 1;
    }
    if (g->relax != 0.0) {   // relaxed schemes read the old field in every x inverse
        g->xyvar = 0;
        g->nochain = 1;
        g->xpers = 0;
        g->yxy = 0;
    }
    return HMG_OK;
}

}  // namespace

extern "C" {

const char* hmg_version(void) { return "hmg 0.1 (sm_103a)"; }

const char* hmg_last_error(void) { return g_last_error.c_str(); }

hmg_status hmg_create(hmg_ctx** out, int device, size_t budget) {
    g_last_error.clear();
    if (!out) {
        set_error("null output handle");
        return HMG_INVALID_ARG;
    }
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        set_error("no CUDA device %d (%d visible)", device, count);
        return HMG_INVALID_ARG;
    }
    DeviceGuard dg(device);
    hmg_ctx* c = new hmg_ctx();
    c->device = device;
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream64, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete c;
        return cuda_status(e, "stream create");
    }
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    c->budget = budget ? budget : (size_t)(0.9 * (double)fr);
    c->pool = std::make_shared<BudgetPool>();
    c->pool->limit = c->budget;
    *out = c;
    return HMG_OK;
}

hmg_status hmg_destroy(hmg_ctx* ctx) {
    g_last_error.clear();
    if (!ctx) return HMG_OK;
    {
        DeviceGuard dg(ctx->device);
        {
            std::lock_guard<std::mutex> lk(ctx->server_mu);
            if (ctx->server) {
                delete ctx->server;
                ctx->server = nullptr;
            }
        }
        cudaStreamSynchronize(ctx->stream);
        ctx->solve.free_all(ctx);
        ctx->plans.clear();
        cudaStreamSynchronize(ctx->stream64);
        cudaStreamDestroy(ctx->stream64);
        cudaStreamDestroy(ctx->stream);
    }
    delete ctx;
    return HMG_OK;
}

size_t hmg_footprint(int N, hmg_precision p) { return state_bytes(N, p == HMG_FP64, 3); }

hmg_status hmg_set_variant(hmg_ctx* ctx, int N, int variant) {
    g_last_error.clear();
    if (!ctx || !valid_N(N) || variant < -1 || variant > 63) {
        set_error("bad context, N or variant (-1 .. 63)");
        return HMG_INVALID_ARG;
    }
    if (variant < 0) ctx->ztune.erase(N);
    else ctx->ztune[N] = variant;
    return HMG_OK;
}

hmg_status hmg_get_variant(hmg_ctx* ctx, int N, int* variant) {
    g_last_error.clear();
    if (!ctx || !variant || !valid_N(N)) {
        set_error("bad context, N or output");
        return HMG_INVALID_ARG;
    }
    auto it = ctx->ztune.find(N);
    *variant = it == ctx->ztune.end() ? -1 : it->second;
    return HMG_OK;
}

hmg_status hmg_trace_enable(hmg_ctx* ctx, int enable) {
    g_last_error.clear();
    if (!ctx) {
        set_error("null context");
        return HMG_INVALID_ARG;
    }
    DeviceGuard dg(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (enable) ctx->tracer.reset();
    else ctx->tracer.collect();
    ctx->tracer.on = enable != 0;
    return HMG_OK;
}

hmg_status hmg_trace_read(hmg_ctx* ctx, int kind, double* total_ms, long long* launches, double* algo_bytes) {
    g_last_error.clear();
    if (!ctx || kind < 0 || kind >= HMG_K_COUNT) {
        set_error("bad context or kernel kind");
        return HMG_INVALID_ARG;
    }
    DeviceGuard dg(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    ctx->tracer.collect();
    if (total_ms) *total_ms = ctx->tracer.ms[kind];
    if (launches) *launches = ctx->tracer.launches[kind];
    if (algo_bytes) *algo_bytes = ctx->tracer.bytes[kind];
    return HMG_OK;
}

namespace {
// Spheres and cylinders into a three-phase grid: host validation and quantization, the
// sphere kernel (or zeros), then the cylinder kernel merging into the same grid.
hmg_status voxelize_impl(hmg_ctx* ctx, const hmg_sphere* spheres, size_t n, const hmg_cylinder* cylinders,
                         size_t nc, double layer, int N, uint8_t* phase_out) {
    hmg_status st = check_common(ctx, N, phase_out);
    if (st != HMG_OK) return st;
    if ((n && !spheres) || (nc && !cylinders) || n + nc == 0 || n > 100000 || nc > 100000) {
        set_error("need 1..100000 spheres or cylinders");
        return HMG_INVALID_ARG;
    }
    if (!(layer > 0.0 && layer < 1.0)) {
        set_error("layer must lie in (0, 1)");
        return HMG_INVALID_ARG;
    }
    DeviceGuard dg(ctx->device);
    std::vector<hmg_sphere> h(n);
    std::vector<hmg_cylinder> hc(nc);
    if (n) {
        if (is_device_ptr(spheres)) {
            st = cuda_status(cudaMemcpy(h.data(), spheres, n * sizeof(hmg_sphere), cudaMemcpyDeviceToHost), "sphere copy");
            if (st != HMG_OK) return st;
        } else {
            memcpy(h.data(), spheres, n * sizeof(hmg_sphere));
        }
    }
    if (nc) {
        if (is_device_ptr(cylinders)) {
            st = cuda_status(cudaMemcpy(hc.data(), cylinders, nc * sizeof(hmg_cylinder), cudaMemcpyDeviceToHost),
                             "cylinder copy");
            if (st != HMG_OK) return st;
        } else {
            memcpy(hc.data(), cylinders, nc * sizeof(hmg_cylinder));
        }
    }
    for (size_t i = 0; i < n; ++i) {
        const hmg_sphere& s = h[i];
        if (!(std::isfinite(s.cx) && std::isfinite(s.cy) && std::isfinite(s.cz) && std::isfinite(s.r)) ||
            !(s.r > 0.0 && s.r < 0.5)) {
            set_error("sphere %zu: non-finite value or radius outside (0, 0.5)", i);
            return HMG_INVALID_ARG;
        }
    }
    for (size_t i = 0; i < nc; ++i) {
        const hmg_cylinder& c = hc[i];
        const double u2 = c.ux * c.ux + c.uy * c.uy + c.uz * c.uz;
        if (!(std::isfinite(c.cx) && std::isfinite(c.cy) && std::isfinite(c.cz) && std::isfinite(u2) &&
              std::isfinite(c.r) && std::isfinite(c.h)) ||
            !(c.r > 0.0 && c.r < 0.5) || !(c.h > 0.0 && c.h <= 2.0) || !(std::fabs(u2 - 1.0) <= 1e-6)) {
            set_error("cylinder %zu: non-finite value, radius outside (0, 0.5), length outside (0, 2] or "
                      "axis not of unit length", i);
            return HMG_INVALID_ARG;
        }
    }
    // the spheres must not overlap (periodic minimum image; touching is allowed)
    for (size_t i = 0; i < n; ++i)
        for (size_t j = i + 1; j < n; ++j) {
            double d2 = 0.0;
            const double a[3] = {h[i].cx, h[i].cy, h[i].cz}, b[3] = {h[j].cx, h[j].cy, h[j].cz};
            for (int c = 0; c < 3; ++c) {
                double d = std::fabs((a[c] - std::floor(a[c])) - (b[c] - std::floor(b[c])));
                d = std::min(d, 1.0 - d);
                d2 += d * d;
            }
            const double rr = h[i].r + h[j].r;
            if (d2 < rr * rr * (1.0 - 1e-12)) {
                set_error("spheres %zu and %zu overlap", i, j);
                return HMG_INVALID_ARG;
            }
        }
    // quantization (host, FP contraction disabled at build time so that the rounding
    // of every product and sum is the plain IEEE one)
    const long long S = 2LL * N * 4096;
    const double Sd = (double)S;
    std::vector<long long> q(5 * n);
    for (size_t i = 0; i < n; ++i) {
        const double c3[3] = {h[i].cx, h[i].cy, h[i].cz};
        for (int c = 0; c < 3; ++c) {
            const double cw = c3[c] - std::floor(c3[c]);
            long long v = (long long)std::floor(cw * Sd + 0.5);
            v %= S;
            q[5 * i + c] = v;
        }
        const double t_out = h[i].r * Sd;
        const double t_in = (1.0 - layer) * h[i].r * Sd;
        q[5 * i + 3] = (long long)std::floor(t_out * t_out + 0.5);
        q[5 * i + 4] = (long long)std::floor(t_in * t_in + 0.5);
    }
    const long long Sc = 2LL * N * 256;
    const double Scd = (double)Sc;
    std::vector<long long> qc(10 * nc);
    for (size_t i = 0; i < nc; ++i) {
        const hmg_cylinder& c = hc[i];
        const double c3[3] = {c.cx, c.cy, c.cz}, u3[3] = {c.ux, c.uy, c.uz};
        for (int a = 0; a < 3; ++a) {
            const double cw = c3[a] - std::floor(c3[a]);
            qc[10 * i + a] = ((long long)std::floor(cw * Scd + 0.5)) % Sc;
            qc[10 * i + 3 + a] = (long long)std::floor(u3[a] * 1024.0 + 0.5);
        }
        const double t_out = c.r * Scd;
        const double t_in = (1.0 - layer) * c.r * Scd;
        qc[10 * i + 6] = (long long)std::floor(t_out * t_out + 0.5);
        qc[10 * i + 7] = (long long)std::floor(t_in * t_in + 0.5);
        qc[10 * i + 8] = (long long)std::floor(0.5 * c.h * Scd + 0.5);
        qc[10 * i + 9] = (long long)std::floor((0.5 * c.h - layer * c.r) * Scd + 0.5);
    }
    long long* qd = nullptr;
    uint8_t* tmp = nullptr;
    const size_t N3 = (size_t)N * N * N;
    const bool dev_out = is_device_ptr(phase_out);
    const size_t qbytes = (q.size() + qc.size()) * sizeof(long long);
    if (cudaMalloc(&qd, qbytes) != cudaSuccess || (!dev_out && cudaMalloc(&tmp, N3) != cudaSuccess)) {
        cudaGetLastError();
        if (qd) cudaFree(qd);
        set_error("cannot allocate voxelization buffers");
        return HMG_OUT_OF_MEMORY;
    }
    if (!q.empty()) cudaMemcpyAsync(qd, q.data(), q.size() * sizeof(long long), cudaMemcpyHostToDevice, ctx->stream);
    if (!qc.empty())
        cudaMemcpyAsync(qd + q.size(), qc.data(), qc.size() * sizeof(long long), cudaMemcpyHostToDevice, ctx->stream);
    uint8_t* dst = dev_out ? phase_out : tmp;
    const int ev = ctx->tracer.on ? ctx->tracer.begin(ctx->stream) : -1;
    if (n) launch_voxelize(qd, (int)n, N, S, dst, ctx->stream);
    else cudaMemsetAsync(dst, 0, N3, ctx->stream);
    if (nc) launch_voxelize_cyl(qd + q.size(), (int)nc, N, Sc, dst, ctx->stream);
    if (ev >= 0) ctx->tracer.end(ev, HMG_K_OTHER, (double)N3, ctx->stream);
    if (!dev_out) cudaMemcpyAsync(phase_out, tmp, N3, cudaMemcpyDeviceToHost, ctx->stream);
    st = check_launch(ctx, "voxelize");
    cudaFree(qd);
    if (tmp) cudaFree(tmp);
    return st;
}
}  // namespace

hmg_status hmg_voxelize(hmg_ctx* ctx, const hmg_sphere* spheres, size_t n, double layer, int N,
                        uint8_t* phase_out) {
    g_last_error.clear();
    if (n == 0) {
        set_error("need 1..100000 spheres");
        return HMG_INVALID_ARG;
    }
    return voxelize_impl(ctx, spheres, n, nullptr, 0, layer, N, phase_out);
}

hmg_status hmg_voxelize_mixed(hmg_ctx* ctx, const hmg_sphere* spheres, size_t n_spheres,
                              const hmg_cylinder* cylinders, size_t n_cylinders, double layer, int N,
                              uint8_t* phase_out) {
    g_last_error.clear();
    return voxelize_impl(ctx, spheres, n_spheres, cylinders, n_cylinders, layer, N, phase_out);
}

namespace {
hmg_status solve_impl(hmg_ctx* ctx, const uint8_t* phase, int N, double km, double ki, double kc, double tol,
                      hmg_precision precision, int scheme, double beta, int max_iter, double K_out[9],
                      hmg_info* info, double* e_out) {
    g_last_error.clear();
    auto t0 = std::chrono::steady_clock::now();
    hmg_status st = check_common(ctx, N, phase);
    if (st != HMG_OK) return st;
    if (!K_out || !check_k(km, ki, kc) || !(tol > 0.0) || (precision != HMG_FP64 && precision != HMG_FP32_BULK)) {
        set_error("bad K_out, conductivity, tolerance or precision");
        return HMG_INVALID_ARG;
    }
    if (scheme != HMG_SCHEME_EYRE_MILTON && scheme != HMG_SCHEME_BASIC &&
        scheme != HMG_SCHEME_AUGMENTED_LAGRANGIAN) {
        set_error("unknown scheme %d", scheme);
        return HMG_INVALID_ARG;
    }
    if (!(beta > 0.0 && beta <= 2.0)) {
        set_error("relaxation beta = %g outside (0, 2]", beta);
        return HMG_INVALID_ARG;
    }
    if (max_iter <= 0) max_iter = 20000;
    DeviceGuard dg(ctx->device);
    const double k[3] = {km, ki, kc};
    const bool fp64 = precision == HMG_FP64;
    GridDesc g;
    st = prepare(ctx, phase, N, k, fp64, 3, &g, scheme, beta);
    if (st != HMG_OK) return st;
    Solver sv{g, &ctx->solve, ctx->stream, ctx->tracer.on ? &ctx->tracer : nullptr};
    hmg_info local;
    memset(&local, 0, sizeof(local));
    hmg_status rs = fp64 ? sv.run_fp64(max_iter, tol, &local, K_out)
                         : sv.run_bulk(max_iter, tol, &local, K_out, ctx->stream64);
    if (rs == HMG_CUDA_ERROR) return rs;
    st = check_launch(ctx, "solve");
    if (st != HMG_OK) return st;
    if (e_out) {
        const long long N3 = g.N3;
        double* tmp = reinterpret_cast<double*>(ctx->solve.spec64);   // 9 N^3 doubles of scratch
        for (int j = 0; j < 3; ++j) launch_tau_to_e<double>(g, j, ctx->solve.tau64, tmp + 3 * j * N3, ctx->stream);
        st = cuda_status(copy_out(e_out, tmp, 9 * N3 * sizeof(double), ctx->stream), "field copy");
        if (st == HMG_OK) st = check_launch(ctx, "field copy");
        if (st != HMG_OK) return st;
    }
    local.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = local;
    return rs;
}
}  // namespace

hmg_status hmg_solve_scheme(hmg_ctx* ctx, const uint8_t* phase, int N, double km, double ki, double kc,
                            double tol, hmg_precision precision, hmg_scheme scheme, int max_iter, double K_out[9],
                            hmg_info* info, double* e_out) {
    return solve_impl(ctx, phase, N, km, ki, kc, tol, precision, (int)scheme, 2.0, max_iter, K_out, info, e_out);
}

hmg_status hmg_solve_polarization(hmg_ctx* ctx, const uint8_t* phase, int N, double km, double ki, double kc,
                                  double tol, hmg_precision precision, double beta, int max_iter, double K_out[9],
                                  hmg_info* info, double* e_out) {
    return solve_impl(ctx, phase, N, km, ki, kc, tol, precision, HMG_SCHEME_EYRE_MILTON, beta, max_iter, K_out,
                      info, e_out);
}

hmg_status hmg_solve_fields(hmg_ctx* ctx, const uint8_t* phase, int N, double km, double ki, double kc,
                            double tol, hmg_precision precision, int max_iter, double K_out[9], hmg_info* info,
                            double* e_out) {
    return hmg_solve_scheme(ctx, phase, N, km, ki, kc, tol, precision, HMG_SCHEME_EYRE_MILTON, max_iter, K_out, info,
                            e_out);
}

hmg_status hmg_solve(hmg_ctx* ctx, const uint8_t* phase, int N, double km, double ki, double kc, double tol,
                     hmg_precision precision, int max_iter, double K_out[9], hmg_info* info) {
    return hmg_solve_fields(ctx, phase, N, km, ki, kc, tol, precision, max_iter, K_out, info, nullptr);
}

hmg_status hmg_em_iterate(hmg_ctx* ctx, const uint8_t* phase, int N, double km, double ki, double kc,
                          const double grad_Theta[3], hmg_precision precision, int n_iter, double* e_inout,
                          double* eps_out) {
    g_last_error.clear();
    hmg_status st = check_common(ctx, N, phase);
    if (st != HMG_OK) return st;
    if (!e_inout || !grad_Theta || n_iter < 0 || !check_k(km, ki, kc) ||
        (precision != HMG_FP64 && precision != HMG_FP32_BULK)) {
        set_error("bad field, gradient, iteration count, conductivity or precision");
        return HMG_INVALID_ARG;
    }
    const double nE = std::sqrt(grad_Theta[0] * grad_Theta[0] + grad_Theta[1] * grad_Theta[1] +
                                grad_Theta[2] * grad_Theta[2]);
    if (!(nE > 0.0 && std::isfinite(nE))) {
        set_error("grad_Theta must be finite and nonzero");
        return HMG_INVALID_ARG;
    }
    DeviceGuard dg(ctx->device);
    const double k[3] = {km, ki, kc};
    const bool fp64 = precision == HMG_FP64;
    GridDesc g;
    st = prepare(ctx, phase, N, k, fp64, 1, &g);
    if (st != HMG_OK) return st;
    for (int c = 0; c < 3; ++c) g.E[0][c] = grad_Theta[c];
    SolveState& s = ctx->solve;
    const long long N3 = g.N3;
    double* tmp = reinterpret_cast<double*>(s.spec64);
    st = cuda_status(copy_in(tmp, e_inout, 3 * N3 * sizeof(double), ctx->stream), "field copy");
    if (st != HMG_OK) return st;
    Solver sv{g, &s, ctx->stream};
    if (fp64) launch_e_to_tau<double>(g, 0, tmp, s.tau64, ctx->stream);
    else launch_e_to_tau<float>(g, 0, tmp, s.f32buf, ctx->stream);
    for (int n = 0; n < n_iter; ++n) {
        if (fp64) sv.sweep<double>(1u, s.tau64, s.spec64, Z_ITER, XI_INPLACE_RES, nullptr, nullptr, nullptr);
        else sv.sweep<float>(1u, s.f32buf, s.spec32, Z_ITER, XI_INPLACE_RES, nullptr, nullptr, nullptr);
        double h;
        if (!sv.fetch(&h, 0, 1)) return HMG_CUDA_ERROR;
        if (eps_out) eps_out[n] = sv.eps_from_sum(h, 0);
    }
    if (fp64) launch_tau_to_e<double>(g, 0, s.tau64, tmp, ctx->stream);
    else launch_tau_to_e<float>(g, 0, s.f32buf, tmp, ctx->stream);
    st = cuda_status(copy_out(e_inout, tmp, 3 * N3 * sizeof(double), ctx->stream), "field copy");
    if (st != HMG_OK) return st;
    return check_launch(ctx, "em_iterate");
}

hmg_status hmg_equilibrium(hmg_ctx* ctx, const uint8_t* phase, int N, double km, double ki, double kc,
                           hmg_precision precision, const double* e, double* eps_eq_out, double* flux_out) {
    g_last_error.clear();
    hmg_status st = check_common(ctx, N, phase);
    if (st != HMG_OK) return st;
    if (!e || !eps_eq_out || !check_k(km, ki, kc) || (precision != HMG_FP64 && precision != HMG_FP32_BULK)) {
        set_error("bad field, output, conductivity or precision");
        return HMG_INVALID_ARG;
    }
    DeviceGuard dg(ctx->device);
    const double k[3] = {km, ki, kc};
    const bool fp64 = precision == HMG_FP64;
    GridDesc g;
    st = prepare(ctx, phase, N, k, fp64, 1, &g);
    if (st != HMG_OK) return st;
    SolveState& s = ctx->solve;
    double* tmp = reinterpret_cast<double*>(s.spec64);
    st = cuda_status(copy_in(tmp, e, 3 * g.N3 * sizeof(double), ctx->stream), "field copy");
    if (st != HMG_OK) return st;
    Solver sv{g, &s, ctx->stream};
    double eps[3], flux[3][3];
    bool ok;
    if (fp64) {
        launch_e_to_tau<double>(g, 0, tmp, s.tau64, ctx->stream);
        ok = sv.check_eq<double>(1u, s.tau64, s.spec64, eps, flux);
    } else {
        launch_e_to_tau<float>(g, 0, tmp, s.f32buf, ctx->stream);
        ok = sv.check_eq<float>(1u, s.f32buf, s.spec32, eps, flux);
    }
    if (!ok) return HMG_CUDA_ERROR;
    *eps_eq_out = eps[0];
    if (flux_out)
        for (int c = 0; c < 3; ++c) flux_out[c] = flux[0][c];
    return check_launch(ctx, "equilibrium");
}

static hmg_status fft_common(hmg_ctx* ctx, int N, int count, hmg_precision precision, const double* in,
                             double* out, bool forward) {
    g_last_error.clear();
    hmg_status st = check_common(ctx, N, in);
    if (st != HMG_OK) return st;
    if (!out || count < 1 || (precision != HMG_FP64 && precision != HMG_FP32_BULK)) {
        set_error("bad output, count or precision");
        return HMG_INVALID_ARG;
    }
    DeviceGuard dg(ctx->device);
    auto gp = ctx->plan(N);
    const bool fp64 = precision == HMG_FP64;
    if (!gp || !ctx->solve.ensure(ctx, N, fp64, 1)) {
        set_error("cannot allocate FFT state");
        return HMG_OUT_OF_MEMORY;
    }
    const double k[3] = {1.0, 1.0, 1.0};
    GridDesc g = make_desc(*gp, fp64, k, ctx->solve.phase, 1);
    if (!fp64) {
        const int v = autotune_z(ctx, g, &ctx->solve, ctx->stream);
        g.zvar = v & 1;
        g.xyvar = (v >> 1) & 1;
        g.nochain = (v >> 2) & 1;
        g.xpers = (v >> 3) & 1;
        g.zpers = (v >> 4) & 1;
        g.yxy = (v >> 5) & 1;
    }
    SolveState& s = ctx->solve;
    const long long N3 = g.N3;
    double* d64 = s.tau64;          // 3 N^3 doubles: staging of one group of three grids
    double* dsp = reinterpret_cast<double*>(s.spec64);
    for (int base = 0; base < count; base += 3) {
        const int cnt = std::min(3, count - base);
        cudaMemsetAsync(d64, 0, 3 * N3 * sizeof(double), ctx->stream);
        st = cuda_status(copy_in(d64, in + (size_t)base * N3, cnt * N3 * sizeof(double), ctx->stream), "copy in");
        if (st != HMG_OK) return st;
        if (forward) {
            if (fp64) {
                launch_x_forward<double>(g, XF_PLAIN, 1u, d64, dsp, nullptr, ctx->stream);
                launch_y_pass<double>(g, true, 1u, dsp, ctx->stream);
                launch_z_pass<double>(g, Z_FWD, 1u, dsp, nullptr, ctx->stream);
                st = cuda_status(copy_out(out + (size_t)base * N3, dsp, cnt * N3 * sizeof(double), ctx->stream), "copy out");
            } else {
                float* f = s.f32buf;
                float* sp = reinterpret_cast<float*>(s.spec32);
                launch_convert<float>(d64, f, 3 * N3, ctx->stream);
                launch_xy_forward<float>(g, XF_PLAIN, 1u, f, sp, nullptr, ctx->stream);
                launch_z_pass<float>(g, Z_FWD, 1u, sp, nullptr, ctx->stream);
                launch_convert_back<float>(sp, dsp, 3 * N3, ctx->stream);
                st = cuda_status(copy_out(out + (size_t)base * N3, dsp, cnt * N3 * sizeof(double), ctx->stream), "copy out");
            }
        } else {
            if (fp64) {
                cudaMemcpyAsync(dsp, d64, 3 * N3 * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream);
                launch_z_pass<double>(g, Z_INV, 1u, dsp, nullptr, ctx->stream);
                launch_y_pass<double>(g, false, 1u, dsp, ctx->stream);
                launch_x_inverse<double>(g, XI_PLAIN, 1u, dsp, d64, nullptr, nullptr, nullptr, nullptr, ctx->stream);
                st = cuda_status(copy_out(out + (size_t)base * N3, d64, cnt * N3 * sizeof(double), ctx->stream), "copy out");
            } else {
                float* f = s.f32buf;
                float* sp = reinterpret_cast<float*>(s.spec32);
                launch_convert<float>(d64, sp, 3 * N3, ctx->stream);
                launch_z_pass<float>(g, Z_INV, 1u, sp, nullptr, ctx->stream);
                launch_yx_inverse<float>(g, XI_PLAIN, 1u, sp, f, nullptr, nullptr, nullptr, nullptr, ctx->stream);
                launch_convert_back<float>(f, d64, 3 * N3, ctx->stream);
                st = cuda_status(copy_out(out + (size_t)base * N3, d64, cnt * N3 * sizeof(double), ctx->stream), "copy out");
            }
        }
        if (st != HMG_OK) return st;
        st = check_launch(ctx, forward ? "fft forward" : "fft inverse");
        if (st != HMG_OK) return st;
    }
    return HMG_OK;
}

hmg_status hmg_fft_forward(hmg_ctx* ctx, int N, int count, hmg_precision precision, const double* x,
                           double* X_out) {
    return fft_common(ctx, N, count, precision, x, X_out, true);
}

hmg_status hmg_fft_inverse(hmg_ctx* ctx, int N, int count, hmg_precision precision, const double* X,
                           double* x_out) {
    return fft_common(ctx, N, count, precision, X, x_out, false);
}

}  // extern "C"
