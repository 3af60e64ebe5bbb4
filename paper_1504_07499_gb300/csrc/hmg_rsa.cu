// Seeded sphere placement on the GPU (§2: up to 100 identical, non-overlapping spheres in
// the periodic unit cube, produced by random sequential adsorption), and the RVE
// pipeline placement -> voxelization.
//
// Random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) as a counter-based
// stream: output i (i >= 1) of stream s of a seed is mix(base + i * 0x9E3779B97F4A7C15)
// with base = seed + s * 0xD1B54A32D192ED03 (mod 2^64); a uniform double is the top 53
// bits times 2^-53.  Candidate j of a placement run takes outputs 3j+1, 3j+2, 3j+3.
//
// Placement (the same steps as the library's seeded host generator):
//   1. RSA at the target radius r (stream 0): candidates are accepted in draw order when
//      their periodic minimum-image distance to every accepted centre exceeds 2r (squared
//      distances against (2r)^2); candidates are drawn in blocks of 8192 until n spheres
//      are placed or a block ends at or past the candidate cap.
//   2. Above the RSA jamming limit (step 1 fails): RSA at 0.85 r (stream 2), then
//      Monte-Carlo displacement sweeps (stream 1) that let the radius grow: each sweep
//      sets the working radius to min(r, half the smallest pair distance) and stops once
//      it reaches r with every pair farther apart than 2r; otherwise every sphere in turn
//      tries a move by step (2u - 1) per axis (step = max(r/4, 1e-3), coordinates wrapped
//      into [0, 1) as fmod(x, 1) + 1 for negative remainders), kept when it stays farther
//      than twice the working radius from all others; each sweep draws 4 uniforms per
//      sphere (the fourth is unused).
// Squared distances are (dx^2 + dy^2) + dz^2 with d = min(|a - b|, 1 - |a - b|), every
// operation rounded on its own, so the sphere lists equal the host generator's bit for
// bit.  Every loop is bounded (candidate cap, sweep cap); failure is a status, not a hang.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/hmg.h"
#include "hmg_runtime.h"

namespace hmg {
namespace rsa {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kStream = 0xD1B54A32D192ED03ull;
constexpr int kBlock = 8192;       // candidates per draw block
constexpr int kThreads = 1024;     // candidates examined per CTA round
constexpr int kMaxSpheres = 1024;  // shared-memory capacity of the kernels

__device__ __forceinline__ uint64_t mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double uniform(uint64_t base, uint64_t counter) {
    return (double)(mix(base + counter * kGamma) >> 11) * 0x1.0p-53;
}
__device__ __forceinline__ double axis_d(double a, double b) {
    const double d = fabs(__dsub_rn(a, b));
    return fmin(d, __dsub_rn(1.0, d));
}
__device__ __forceinline__ double min_image_sq(double ax, double ay, double az, double bx, double by, double bz) {
    const double dx = axis_d(ax, bx), dy = axis_d(ay, by), dz = axis_d(az, bz);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Sequential RSA in one CTA.  Each round examines kThreads consecutive candidates in
// parallel against the accepted centres, then accepts them in draw order: the first
// candidate still clear is accepted and the later ones are re-examined against it only.
// out: 3 n doubles; state[0] = spheres placed, state[1] = candidates examined.
__global__ void __launch_bounds__(kThreads) k_rsa(uint64_t base, int n, double lim, long long limit,
                                                  double* __restrict__ out, long long* __restrict__ state) {
    __shared__ double acc[3 * kMaxSpheres];
    __shared__ int wfirst[kThreads / 32];
    __shared__ int s_first, s_count;
    const int t = threadIdx.x;
    if (t == 0) s_count = 0;
    __syncthreads();
    long long used = 0;
    for (long long j0 = 0; j0 < limit && s_count < n; j0 += kThreads) {
        const long long j = j0 + t;
        const bool valid = j < limit;
        double cx = 0, cy = 0, cz = 0;
        bool ok = valid;
        if (valid) {
            cx = uniform(base, 3 * (uint64_t)j + 1);
            cy = uniform(base, 3 * (uint64_t)j + 2);
            cz = uniform(base, 3 * (uint64_t)j + 3);
            for (int a = 0; a < s_count && ok; ++a)
                ok = min_image_sq(cx, cy, cz, acc[3 * a], acc[3 * a + 1], acc[3 * a + 2]) > lim;
        }
        int start = 0;
        bool round_done = false;
        while (!round_done) {   // at most kThreads acceptances per round
            const unsigned bal = __ballot_sync(0xffffffffu, ok && t >= start);
            if ((t & 31) == 0) wfirst[t >> 5] = bal ? (t & ~31) + __ffs(bal) - 1 : kThreads;
            __syncthreads();
            if (t == 0) {
                int f = kThreads;
                for (int w = 0; w < kThreads / 32; ++w) f = min(f, wfirst[w]);
                s_first = f;
            }
            __syncthreads();
            const int f = s_first;
            if (f >= kThreads) {
                round_done = true;
            } else {
                if (t == f) {
                    const int a = s_count;
                    acc[3 * a] = cx;
                    acc[3 * a + 1] = cy;
                    acc[3 * a + 2] = cz;
                    s_count = a + 1;
                }
                __syncthreads();
                const int a = s_count - 1;
                if (ok && t > f) ok = min_image_sq(cx, cy, cz, acc[3 * a], acc[3 * a + 1], acc[3 * a + 2]) > lim;
                if (t == f) ok = false;
                start = f + 1;
                if (s_count >= n) {
                    round_done = true;
                    used = j0 + f + 1;
                }
            }
            __syncthreads();
        }
        if (s_count < n) used = min(j0 + kThreads, limit);
    }
    for (int i = t; i < 3 * s_count; i += kThreads) out[i] = acc[i];
    if (t == 0) {
        state[0] = s_count;
        state[1] = used;
    }
}

// wrap into [0, 1): fmod(x, 1) (exact), plus 1 when the remainder is negative
__device__ __forceinline__ double wrap1(double x) {
    double m = fmod(x, 1.0);
    if (m != 0.0) {
        if (m < 0.0) m = __dadd_rn(m, 1.0);
    } else {
        m = 0.0;
    }
    return m;
}

// Growth sweeps in one CTA (thread i owns sphere i for the distance checks).
// c: 3 n doubles in/out; state[0] = 1 on success, state[1] = sweeps run.
__global__ void __launch_bounds__(kThreads) k_grow(uint64_t base, int n, double r_target, double lim_target,
                                                   int max_sweeps, double* __restrict__ c,
                                                   long long* __restrict__ state) {
    __shared__ double p[3 * kMaxSpheres];
    __shared__ double wmin[kThreads / 32];
    __shared__ double s_lim;
    __shared__ int s_done;
    const int t = threadIdx.x;
    for (int i = t; i < 3 * n; i += blockDim.x) p[i] = c[i];
    if (t == 0) s_done = 0;
    __syncthreads();
    const double step = fmax(__dmul_rn(0.25, r_target), 1e-3);
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        // smallest squared pair distance (every pair, in a fixed split over threads;
        // the minimum does not depend on the order)
        double m = INFINITY;
        for (int i = t; i < n; i += blockDim.x)
            for (int k = 0; k < n; ++k)
                if (k != i) m = fmin(m, min_image_sq(p[3 * i], p[3 * i + 1], p[3 * i + 2], p[3 * k], p[3 * k + 1], p[3 * k + 2]));
        for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_down_sync(0xffffffffu, m, o));
        if ((t & 31) == 0) wmin[t >> 5] = m;
        __syncthreads();
        if (t == 0) {
            double d2 = INFINITY;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) d2 = fmin(d2, wmin[w]);
            const double half = __dmul_rn(0.5, __dsqrt_rn(d2));
            const double r_work = half < r_target ? half : r_target;
            if (r_work >= r_target && d2 > lim_target) {
                s_done = 1;
            } else {
                const double tw = __dmul_rn(2.0, r_work);
                s_lim = __dmul_rn(tw, tw);
            }
        }
        __syncthreads();
        if (s_done) break;
        const double lim = s_lim;
        const uint64_t cbase = (uint64_t)sweep * 4 * (uint64_t)n;   // counters used before this sweep
        for (int i = 0; i < n; ++i) {
            double tr[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double u = uniform(base, cbase + 4 * (uint64_t)i + a + 1);
                const double mv = __dmul_rn(step, __dsub_rn(__dmul_rn(2.0, u), 1.0));
                tr[a] = wrap1(__dadd_rn(p[3 * i + a], mv));
            }
            bool clear = true;
            for (int k = t; k < n; k += blockDim.x)
                if (k != i) clear = clear && min_image_sq(tr[0], tr[1], tr[2], p[3 * k], p[3 * k + 1], p[3 * k + 2]) > lim;
            const int all = __syncthreads_and(clear ? 1 : 0);
            if (all && t == 0) {
                p[3 * i] = tr[0];
                p[3 * i + 1] = tr[1];
                p[3 * i + 2] = tr[2];
            }
            __syncthreads();
        }
    }
    for (int i = t; i < 3 * n; i += blockDim.x) c[i] = p[i];
    if (t == 0) {
        state[0] = s_done;
        state[1] = sweep;
    }
}

}  // namespace rsa

// Runs one placement kernel; false with the error set on a CUDA failure.
static bool run_rsa(cudaStream_t st, uint64_t seed, int stream, int n, double r, long long max_candidates,
                    double* d_out, long long* d_state, long long h_state[2]) {
    const uint64_t base = seed + (uint64_t)stream * rsa::kStream;
    const double tr = 2.0 * r;
    const double lim = tr * tr;
    const long long limit = (max_candidates + rsa::kBlock - 1) / rsa::kBlock * rsa::kBlock;
    rsa::k_rsa<<<1, rsa::kThreads, 0, st>>>(base, n, lim, limit, d_out, d_state);
    cudaError_t e = cudaMemcpyAsync(h_state, d_state, 2 * sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_error("RSA kernel: %s", cudaGetErrorString(e));
        return false;
    }
    return true;
}

// The placement of steps 1-2 above into host memory (3 n centres); generator: 0 RSA,
// 1 RSA at 0.85 r + growth sweeps.
static hmg_status place(hmg_ctx* ctx, uint64_t seed, int n, double r, long long max_candidates,
                        std::vector<double>& centres, int* generator) {
    DeviceGuard dg(ctx->device);
    cudaStream_t st = ctx->stream;
    double* d_c = (double*)ctx->alloc(3 * (size_t)n * sizeof(double));
    long long* d_state = (long long*)ctx->alloc(2 * sizeof(long long));
    if (!d_c || !d_state) {
        ctx->release(d_c);
        ctx->release(d_state);
        set_error("cannot allocate placement state");
        return HMG_OUT_OF_MEMORY;
    }
    long long h[2] = {0, 0};
    hmg_status res = HMG_OK;
    int gen = 0;
    if (!run_rsa(st, seed, 0, n, r, max_candidates, d_c, d_state, h)) {
        res = HMG_CUDA_ERROR;
    } else if (h[0] < n) {
        gen = 1;
        const double r85 = 0.85 * r;
        if (!run_rsa(st, seed, 2, n, r85, max_candidates, d_c, d_state, h)) {
            res = HMG_CUDA_ERROR;
        } else if (h[0] < n) {
            set_error("RSA at the reduced radius placed %lld of %d spheres", h[0], n);
            res = HMG_NOT_CONVERGED;
        } else if (n > 1) {
            const double tr = 2.0 * r;
            const int threads = std::min(rsa::kThreads, (n + 31) / 32 * 32);   // one thread per sphere
            rsa::k_grow<<<1, threads, 0, st>>>(seed + 1 * rsa::kStream, n, r, tr * tr, 20000, d_c, d_state);
            cudaError_t e = cudaMemcpyAsync(h, d_state, 2 * sizeof(long long), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                set_error("growth kernel: %s", cudaGetErrorString(e));
                res = HMG_CUDA_ERROR;
            } else if (!h[0]) {
                set_error("growth sweeps did not reach the target radius in 20000 sweeps");
                res = HMG_NOT_CONVERGED;
            }
        }
    }
    if (res == HMG_OK) {
        centres.resize(3 * (size_t)n);
        cudaError_t e = cudaMemcpyAsync(centres.data(), d_c, 3 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error("centre copy: %s", cudaGetErrorString(e));
            res = HMG_CUDA_ERROR;
        }
    }
    ctx->release(d_c);
    ctx->release(d_state);
    if (generator) *generator = gen;
    return res;
}

static bool check_place_args(hmg_ctx* ctx, int n, double r, long long max_candidates) {
    if (!ctx || n < 1 || n > rsa::kMaxSpheres || !(r > 0.0 && r < 0.5) || max_candidates < 1) {
        set_error("need a context, 1 <= n <= %d, 0 < r < 0.5 and a positive candidate cap", rsa::kMaxSpheres);
        return false;
    }
    return true;
}

}  // namespace hmg

using namespace hmg;

extern "C" hmg_status hmg_rsa(hmg_ctx* ctx, uint64_t seed, int n, double r, long long max_candidates,
                              hmg_sphere* spheres_out, int* generator) {
    g_last_error.clear();
    if (!check_place_args(ctx, n, r, max_candidates) || !spheres_out) {
        if (!spheres_out) set_error("null output");
        return HMG_INVALID_ARG;
    }
    std::vector<double> c;
    hmg_status st = place(ctx, seed, n, r, max_candidates, c, generator);
    if (st != HMG_OK) return st;
    std::vector<hmg_sphere> h(n);
    for (int i = 0; i < n; ++i) h[i] = hmg_sphere{c[3 * i], c[3 * i + 1], c[3 * i + 2], r};
    DeviceGuard dg(ctx->device);
    if (is_device_ptr(spheres_out)) {
        if (cudaMemcpy(spheres_out, h.data(), n * sizeof(hmg_sphere), cudaMemcpyHostToDevice) != cudaSuccess) {
            set_error("sphere copy: %s", cudaGetErrorString(cudaGetLastError()));
            return HMG_CUDA_ERROR;
        }
    } else {
        for (int i = 0; i < n; ++i) spheres_out[i] = h[i];
    }
    return HMG_OK;
}

extern "C" hmg_status hmg_rve(hmg_ctx* ctx, uint64_t seed, int n, double r, long long max_candidates, double layer,
                              int N, uint8_t* phase_out, hmg_sphere* spheres_out, int* generator) {
    g_last_error.clear();
    if (!check_place_args(ctx, n, r, max_candidates)) return HMG_INVALID_ARG;
    if (!phase_out || !valid_N(N) || !(layer > 0.0 && layer < 1.0)) {
        set_error("need a phase buffer, a valid N and a layer in (0, 1)");
        return HMG_INVALID_ARG;
    }
    std::vector<double> c;
    hmg_status st = place(ctx, seed, n, r, max_candidates, c, generator);
    if (st != HMG_OK) return st;
    std::vector<hmg_sphere> h(n);
    for (int i = 0; i < n; ++i) h[i] = hmg_sphere{c[3 * i], c[3 * i + 1], c[3 * i + 2], r};
    if (spheres_out) {
        DeviceGuard dg(ctx->device);
        if (is_device_ptr(spheres_out)) {
            if (cudaMemcpy(spheres_out, h.data(), n * sizeof(hmg_sphere), cudaMemcpyHostToDevice) != cudaSuccess) {
                set_error("sphere copy: %s", cudaGetErrorString(cudaGetLastError()));
                return HMG_CUDA_ERROR;
            }
        } else {
            for (int i = 0; i < n; ++i) spheres_out[i] = h[i];
        }
    }
    return hmg_voxelize(ctx, h.data(), (size_t)n, layer, N, phase_out);
}
