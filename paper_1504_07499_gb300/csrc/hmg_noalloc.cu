// hmg_equilibrium_noalloc: the FP64 equilibrium residual of hmg_equilibrium for callers
// that must not allocate device memory.  Every scratch buffer lives in file-scope
// static __device__ arrays sized for N <= HMG_NOALLOC_MAX_N; the call allocates
// nothing (no cudaMalloc, cudaFree, stream or event creation).
//
// In host code the names of these arrays are host-side stand-ins, not device
// addresses.  Every call looks their device addresses up with cudaGetSymbolAddress
// while the caller's device is current (a lookup that allocates nothing), so no
// address outlives the context it belongs to (cudaDeviceReset, a new primary
// context), and it writes the twiddle table of its N before using it.
// All calls share the arrays, which keep the last call's contents; the library
// serializes its calls (a lock held until the call's GPU work has finished), since
// two calls overlapping on the GPU would race on them.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/hmg.h"
#include "hmg_internal.h"
#include "hmg_runtime.h"

namespace hmg {
void make_plan(int L, FftPlan* p);
}

using namespace hmg;

namespace {

constexpr int kMaxN = HMG_NOALLOC_MAX_N;
constexpr long long kMaxN3 = (long long)kMaxN * kMaxN * kMaxN;
constexpr int kMaxPartials = 3 * kMaxN * kMaxN;   // >= CTAs of any pass at N <= kMaxN

static __device__ __align__(256) uint8_t g_phase[kMaxN3];
static __device__ __align__(256) double g_field[3 * kMaxN3];        // e, then the packed spectrum
static __device__ __align__(256) double g_spec[3 * kMaxN3];         // tau = (k + k0) e
static __device__ __align__(256) double g_partial[2 * kMaxPartials];
static __device__ __align__(256) double g_red[64];
static __device__ __align__(256) double2 g_tw[kMaxN + kMaxN / 2];

struct Addrs {
    uint8_t* phase = nullptr;
    double* field = nullptr;
    double* spec = nullptr;
    double* partial = nullptr;
    double* red = nullptr;
    double2* tw = nullptr;
};

std::mutex g_mu;

template <typename T>
bool symbol_address(T** out, const T& sym) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, sym) != cudaSuccess) return false;
    *out = static_cast<T*>(p);
    return true;
}

// With the caller's device current: the device addresses of the static arrays in the
// current context.
hmg_status lookup(Addrs* a) {
    bool ok = symbol_address(&a->phase, g_phase[0]) && symbol_address(&a->field, g_field[0]) &&
              symbol_address(&a->spec, g_spec[0]) && symbol_address(&a->partial, g_partial[0]) &&
              symbol_address(&a->red, g_red[0]) && symbol_address(&a->tw, g_tw[0]);
    if (!ok) {
        cudaError_t e = cudaGetLastError();
        set_error("cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return HMG_CUDA_ERROR;
    }
    return HMG_OK;
}

hmg_status cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return HMG_CUDA_ERROR;
}

}  // namespace

extern "C" hmg_status hmg_equilibrium_noalloc(const uint8_t* phase, int N, double km, double ki, double kc,
                                              const double* e, double* eps_eq_out, double* flux_mean_out) {
    g_last_error.clear();
    if (!phase || !e || !eps_eq_out) {
        set_error("null pointer argument");
        return HMG_INVALID_ARG;
    }
    if (!valid_N(N)) {
        set_error("N = %d: need an even N = 2^a 3^b with 8 <= N <= 512", N);
        return HMG_INVALID_ARG;
    }
    if (N > kMaxN) {
        set_error("N = %d exceeds the static scratch of hmg_equilibrium_noalloc (N <= %d)", N, kMaxN);
        return HMG_INVALID_ARG;
    }
    for (double k : {km, ki, kc})
        if (!(std::isfinite(k) && k > 0.0)) {
            set_error("conductivities must be finite and positive");
            return HMG_INVALID_ARG;
        }
    std::lock_guard<std::mutex> lk(g_mu);
    Addrs addrs;
    Addrs* a = &addrs;
    hmg_status st = lookup(a);
    if (st != HMG_OK) return st;
    cudaError_t ce = cudaSuccess;

    const cudaStream_t s = 0;   // legacy default stream of the current device
    const long long N3 = (long long)N * N * N;
    const int M = N / 2;

    // FFT schedules (host only) and the twiddle table of this N in the static array
    GridPlan gp;
    gp.N = N;
    make_plan(N, &gp.pN);
    make_plan(M, &gp.pM);
    gp.pN.tw_off = 0;
    gp.pM.tw_off = N;
    {
        double2 h[kMaxN + kMaxN / 2];
        for (int part = 0; part < 2; ++part) {
            const int L = part == 0 ? N : M, off = part == 0 ? 0 : N;
            for (int k = 0; k < L; ++k) {
                const double ang = 2.0 * M_PI * (double)k / (double)L;
                double c = std::cos(ang), sn = -std::sin(ang);
                if ((4 * k) % L == 0) {
                    const int qd = (4 * k) / L;
                    c = (qd == 0) ? 1.0 : (qd == 2 ? -1.0 : 0.0);
                    sn = (qd == 1) ? -1.0 : (qd == 3 ? 1.0 : 0.0);
                }
                h[off + k] = make_double2(c, sn);
            }
        }
        // pageable source: the copy has read h when the call returns
        ce = cudaMemcpyAsync(a->tw, h, sizeof(double2) * (N + M), cudaMemcpyHostToDevice, s);
        if (ce != cudaSuccess) return cuda_fail(ce, "twiddle upload");
    }

    // inputs into the static arrays (host or device sources)
    ce = cudaMemcpyAsync(a->phase, phase, (size_t)N3, cudaMemcpyDefault, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(a->field, e, 3 * N3 * sizeof(double), cudaMemcpyDefault, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(a->red, 0, 64 * sizeof(double), s);   // sums start at zero
    if (ce != cudaSuccess) return cuda_fail(ce, "input copy");

    const double k3[3] = {km, ki, kc};
    GridDesc g = make_desc(gp, true, k3, a->phase, 1);   // gp owns no device table
    g.tw64 = a->tw;
    // e (in g_field) -> tau = (k + k0) e (in g_spec) -> packed spectrum (in g_field)
    launch_e_to_tau<double>(g, 0, a->field, a->spec, s);
    launch_x_forward<double>(g, XF_FLUX, 1u, a->spec, a->field, a->partial, s);
    launch_reduce(a->partial, 1, x_ctas(g), 3, a->red + 16, s);
    launch_y_pass<double>(g, true, 1u, a->field, s);
    launch_z_pass<double>(g, Z_EQ, 1u, a->field, a->partial + kMaxPartials, s);
    launch_reduce(a->partial + kMaxPartials, 1, z_ctas(g), 1, a->red + 32, s);
    double h[48];
    ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h, a->red + 16, 32 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_fail(ce, "equilibrium kernels");
    double nrm = 0.0, flux[3];
    for (int c = 0; c < 3; ++c) {
        flux[c] = h[c] / (double)N3;
        nrm += flux[c] * flux[c];
    }
    *eps_eq_out = std::sqrt(h[16]) / std::sqrt(nrm);
    if (flux_mean_out)
        for (int c = 0; c < 3; ++c) flux_mean_out[c] = flux[c];
    return HMG_OK;
}
