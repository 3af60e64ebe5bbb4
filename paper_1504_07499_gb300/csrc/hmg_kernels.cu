// FFT passes of one Eyre-Milton sweep (§3 Algorithm, steps 2-7) and the helpers
// around them.  The 3D real transform runs as five passes over HBM:
//   x forward (real->complex, polarization of step 2 fused on load),
//   y forward,
//   z forward + Green operator of step 4 (+ macroscopic gradient at DC) + z inverse,
//   y inverse,
//   x inverse (complex->real) with the update of step 7 written out and the
//   step-6 residual accumulated in FP64.
// The sweep is written in the polarization variable tau = (k + k0) e: with
// Y = (k - k0)/(k + k0) and P the projector xi xi^T/|xi|^2 (Gamma0 = -P/k0 for
// L0 = -k0 I), steps 2-7 read tau^{n+1} = (I - 2P)(Y tau^n) + 2 k0 E, and
// e^n - e_comp^n = (tau^n - tau^{n+1}) / (2 k0), so no field but tau is stored.
// (The basic scheme runs through the same passes on e itself, with its own Y and the
// Green step -P; GridDesc carries the scheme's coefficients.)  These generic kernels
// serve FP64 and the sizes without register-resident FP32 kernels (hmg_fast.cu).
//
// Spectrum layout: after the x pass each row of N reals becomes N/2 complex values
// (x-major rows, same byte size as the real field); entry kx = 0 packs the two real
// planes kx = 0 and kx = N/2 as X(0) + i X(N/2).  The y and z passes transform that
// packed column like any other; the Green operator treats its four special modes
// (ky, kz in {0, N/2}) by real and imaginary part.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "hmg_fft.cuh"
#include "hmg_green.cuh"
#include "hmg_internal.h"

namespace hmg {

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------

template <typename R>
__device__ __forceinline__ R sel3(int ph, double a, double b, double c) {
    return R(ph == 0 ? a : (ph == 1 ? b : c));
}

// Fixed-order CTA sum of one double per thread; result valid in thread 0.
__device__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// x forward: rows of N reals -> N/2 packed complex values
// ---------------------------------------------------------------------------

template <typename R, int MODE>
__global__ void __launch_bounds__(kThreads)
k_x_forward(GridDesc g, unsigned mask, const R* __restrict__ tau, typename Cplx<R>::T* __restrict__ spec,
            double* __restrict__ partial) {
    using T2 = typename Cplx<R>::T;
    const int slot = blockIdx.y;
    if (!slot_active(g, mask, slot)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* b0 = reinterpret_cast<T2*>(smem_raw);
    const int M = g.M, N = g.N, rows = g.rows;
    T2* b1 = b0 + rows * M;
    __shared__ double red[kThreads];

    const long long row0 = (long long)blockIdx.x * rows;   // row = c*NN + z*N + y
    const T2* src = reinterpret_cast<const T2*>(tau + (long long)slot * 3 * g.N3 + row0 * N);
    double acc = 0.0;
    for (int q = threadIdx.x; q < rows * M; q += blockDim.x) {
        const int rr = q / M, n = q - rr * M;
        T2 v = src[(long long)rr * M + n];
        if (MODE != XF_PLAIN) {
            const long long prow = (row0 + rr) % g.NN;   // (z, y) row of the phase grid
            const uchar2 ph = *reinterpret_cast<const uchar2*>(g.phase + prow * N + 2 * n);
            R ca, cb;
            if (MODE == XF_POLARIZE) {
                ca = sel3<R>(ph.x, g.Y[0], g.Y[1], g.Y[2]);
                cb = sel3<R>(ph.y, g.Y[0], g.Y[1], g.Y[2]);
            } else {
                ca = sel3<R>(ph.x, g.W[0], g.W[1], g.W[2]);
                cb = sel3<R>(ph.y, g.W[0], g.W[1], g.W[2]);
            }
            v.x *= ca;
            v.y *= cb;
            if (MODE == XF_FLUX) acc += (double)v.x + (double)v.y;
        }
        b0[q] = v;
    }
    if (MODE == XF_FLUX) {
        double s = block_sum(acc, red);
        if (threadIdx.x == 0) partial[(long long)slot * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
    T2* res = fft_smem<true>(b0, b1, g.pM, TwTable<T2>::get(g), rows, M, 1);
    // real-to-complex split: X_k = E_k + w_N^k O_k with E, O the DFTs of the even and
    // odd samples, E_k = (Z_k + conj Z_{M-k})/2, O_k = (Z_k - conj Z_{M-k})/(2i)
    const T2* twN = TwTable<T2>::get(g) + g.pN.tw_off;
    T2* dst = spec + (long long)slot * 3 * g.NNM + row0 * M;
    for (int q = threadIdx.x; q < rows * M; q += blockDim.x) {
        const int rr = q / M, k = q - rr * M;
        const T2 z = res[rr * M + k];
        T2 out;
        if (k == 0) {
            out = mk(z.x + z.y, z.x - z.y);
        } else {
            const T2 zm = res[rr * M + (M - k)];
            const T2 e = mk(R(0.5) * (z.x + zm.x), R(0.5) * (z.y - zm.y));
            const T2 o = mk(R(0.5) * (z.y + zm.y), R(-0.5) * (z.x - zm.x));
            out = cadd(e, cmul(o, __ldg(&twN[k])));
        }
        dst[(long long)rr * M + k] = out;
    }
}

// ---------------------------------------------------------------------------
// x inverse: N/2 packed complex values -> N reals, with the sweep's output step
// ---------------------------------------------------------------------------

template <typename R, int MODE>
__global__ void __launch_bounds__(kThreads)
k_x_inverse(GridDesc g, unsigned mask, const typename Cplx<R>::T* __restrict__ spec, R* __restrict__ tau,
            const float* __restrict__ r32, float* __restrict__ d32, float* __restrict__ r32_out,
            double* __restrict__ partial) {
    using T2 = typename Cplx<R>::T;
    const int slot = blockIdx.y;
    if (!slot_active(g, mask, slot)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T2* b0 = reinterpret_cast<T2*>(smem_raw);
    const int M = g.M, N = g.N, rows = g.rows;
    T2* b1 = b0 + rows * M;
    __shared__ double red[kThreads];

    const long long row0 = (long long)blockIdx.x * rows;
    const T2* src = spec + (long long)slot * 3 * g.NNM + row0 * M;
    for (int q = threadIdx.x; q < rows * M; q += blockDim.x) b1[q] = src[q];
    __syncthreads();
    // complex-to-real merge: Z'_k = (X_k + conj X_{M-k}) + i w_N^{-k} (X_k - conj X_{M-k}),
    // whose length-M inverse DFT gives N x[2n] + i N x[2n+1] (unnormalized)
    const T2* twN = TwTable<T2>::get(g) + g.pN.tw_off;
    for (int q = threadIdx.x; q < rows * M; q += blockDim.x) {
        const int rr = q / M, k = q - rr * M;
        T2 xk, xm;
        if (k == 0) {
            const T2 p = b1[rr * M];
            xk = mk(p.x, R(0));
            xm = mk(p.y, R(0));
        } else {
            xk = b1[rr * M + k];
            xm = b1[rr * M + (M - k)];
        }
        const T2 s = mk(xk.x + xm.x, xk.y - xm.y);          // X_k + conj X_{M-k}
        const T2 d = mk(xk.x - xm.x, xk.y + xm.y);          // X_k - conj X_{M-k}
        const T2 dw = cmulc(d, __ldg(&twN[k]));             // d * w^{-k}
        b0[q] = mk(s.x - dw.y, s.y + dw.x);                 // s + i dw
    }
    __syncthreads();
    T2* res = fft_smem<false>(b0, b1, g.pM, TwTable<T2>::get(g), rows, M, 1);

    const long long fbase = (long long)slot * 3 * g.N3 + row0 * N;   // element offset of the tile
    T2* out = reinterpret_cast<T2*>(tau + fbase);
    // output step: add r (correction sweeps), read the old field for the residual,
    // or (XI_DIFF) write d = new - old to d32 and r32_out without touching tau
    constexpr bool kRes = MODE == XI_INPLACE_RES || MODE == XI_ADD_R_RES;
    constexpr bool kAddR = MODE == XI_ADD_R_RES || MODE == XI_ADD_R;
    const bool resid = kRes && (g.dflags ? g.resid != 0 : true);
    const bool addr = kAddR && (g.dflags ? (g.dflags[slot] & SF_ADDR) != 0 : true);
    double acc = 0.0;
    const bool relax = g.relax != 0.0;            // uniform: kernel argument
    const R wn = R(1.0 - g.relax), wo = R(g.relax);
    for (int q = threadIdx.x; q < rows * M; q += blockDim.x) {
        T2 v = res[q];
        if (relax) {   // relaxed schemes: (1 - relax) T(field) + relax field
            const T2 o = out[q];
            v = mk(wn * v.x + wo * o.x, wn * v.y + wo * o.y);
        }
        if (MODE == XI_DIFF) {
            const T2 o = out[q];
            const double da = (double)v.x - (double)o.x, db = (double)v.y - (double)o.y;
            acc += da * da + db * db;
            const float2 df = make_float2((float)da, (float)db);
            reinterpret_cast<float2*>(r32_out + fbase)[q] = df;
            reinterpret_cast<float2*>(d32 + fbase)[q] = df;
            continue;
        }
        if (addr) {
            const float2 rv = reinterpret_cast<const float2*>(r32 + fbase)[q];
            v.x += R(rv.x);
            v.y += R(rv.y);
        }
        if (resid) {
            const T2 o = out[q];
            const double da = (double)v.x - (double)o.x, db = (double)v.y - (double)o.y;
            acc += da * da + db * db;
        }
        out[q] = v;
    }
    if (kRes || MODE == XI_DIFF) {   // uniform across the CTA
        double s = block_sum(acc, red);
        if (threadIdx.x == 0 && (resid || MODE == XI_DIFF)) partial[(long long)slot * gridDim.x + blockIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------
// y pass: Py consecutive kx columns of one (component, z) plane, length N along y
// ---------------------------------------------------------------------------

template <typename R, bool FWD>
__global__ void __launch_bounds__(kThreads)
k_y_pass(GridDesc g, unsigned mask, typename Cplx<R>::T* __restrict__ spec) {
    using T2 = typename Cplx<R>::T;
    const int slot = blockIdx.y;
    if (!slot_active(g, mask, slot)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = g.N, M = g.M, P = g.Py;
    T2* b0 = reinterpret_cast<T2*>(smem_raw);
    T2* b1 = b0 + N * P;
    const int nkb = M / P;
    const int kb = blockIdx.x % nkb;
    const long long cz = blockIdx.x / nkb;                     // c*N + z
    T2* base = spec + (long long)slot * 3 * g.NNM + cz * N * M + kb * P;
    for (int q = threadIdx.x; q < N * P; q += blockDim.x) {
        const int y = q / P, p = q - y * P;
        b0[q] = base[(long long)y * M + p];
    }
    __syncthreads();
    T2* res = fft_smem<FWD>(b0, b1, g.pN, TwTable<T2>::get(g), P, 1, P);
    for (int q = threadIdx.x; q < N * P; q += blockDim.x) {
        const int y = q / P, p = q - y * P;
        base[(long long)y * M + p] = res[q];
    }
}

// ---------------------------------------------------------------------------
// z pass: Pz consecutive kx columns at one ky, all three components, length N
// along z.  Z_ITER: forward, tau_hat <- (ga - gb P) tau_hat / N^3 (+ gc E at DC;
// Eyre-Milton: (I - 2P) and 2 k0 E), inverse.  Z_EQ: forward, then sum
// |xi . phi_hat|^2 / N^6 in FP64.
// ---------------------------------------------------------------------------

template <typename R, int MODE>
__global__ void __launch_bounds__(kThreads)
k_z_pass(GridDesc g, unsigned mask, typename Cplx<R>::T* __restrict__ spec, double* __restrict__ partial) {
    using T2 = typename Cplx<R>::T;
    const int slot = blockIdx.y;
    if (!slot_active(g, mask, slot)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = g.N, M = g.M, P = g.Pz, P3 = 3 * P;
    T2* b0 = reinterpret_cast<T2*>(smem_raw);
    T2* b1 = b0 + N * P3;
    __shared__ double red[kThreads];
    const int nkb = M / P;
    const int kb = blockIdx.x % nkb;
    const int ky = blockIdx.x / nkb;
    T2* base = spec + (long long)slot * 3 * g.NNM + (long long)ky * M + kb * P;
    // SMEM layout [z][c][p]: pencil c*P + p, index stride 3P
    for (int q = threadIdx.x; q < N * P3; q += blockDim.x) {
        const int z = q / P3, cp = q - z * P3, c = cp / P, p = cp - c * P;
        b0[q] = base[(long long)c * g.NNM + (long long)z * N * M + p];
    }
    __syncthreads();
    const T2* tw = TwTable<T2>::get(g);
    T2* res = b0;
    if (MODE != Z_INV) res = fft_smem<true>(b0, b1, g.pN, tw, P3, 1, P3);
    T2* other = (res == b0) ? b1 : b0;

    if (MODE == Z_ITER || MODE == Z_ITER_NOB || MODE == Z_EQ) {
        const bool addb = g.dflags ? (g.dflags[slot] & SF_ADDB) != 0 : MODE == Z_ITER;
        const R scale = R(1.0 / (double)g.N3);
        const R cE[3] = {R(g.gc * g.E[slot][0]), R(g.gc * g.E[slot][1]), R(g.gc * g.E[slot][2])};
        const R ga = R(g.ga), gb = R(g.gb);
        double acc = 0.0;
        const double twopi_n = 6.283185307179586476925 / (double)N;
        for (int q = threadIdx.x; q < N * P; q += blockDim.x) {
            const int kz = q / P, p = q - kz * P;
            const int kx = kb * P + p;
            T2* e = res + kz * P3 + p;
            T2 s0 = e[0], s1 = e[P], s2 = e[2 * P];
            if (MODE == Z_EQ) {
                acc += eq_mode(kx, ky, kz, N, s0, s1, s2);
            } else {
                green_mode<R>(kx, ky, kz, N, scale, ga, gb, addb, cE, s0, s1, s2);
                e[0] = s0;
                e[P] = s1;
                e[2 * P] = s2;
            }
        }
        if (MODE == Z_EQ) {
            // |xi . phi_hat|^2 with xi = 2 pi m'/N and phi_hat = DFT/N^3
            const double s = block_sum(acc, red) * twopi_n * twopi_n / ((double)g.N3 * (double)g.N3);
            if (threadIdx.x == 0) partial[(long long)slot * gridDim.x + blockIdx.x] = s;
            return;
        }
        __syncthreads();
    }
    if (MODE == Z_ITER || MODE == Z_ITER_NOB || MODE == Z_INV) {
        if (MODE == Z_INV) other = b1;
        res = fft_smem<false>(res, other, g.pN, tw, P3, 1, P3);
    }
    for (int q = threadIdx.x; q < N * P3; q += blockDim.x) {
        const int z = q / P3, cp = q - z * P3, c = cp / P, p = cp - c * P;
        base[(long long)c * g.NNM + (long long)z * N * M + p] = res[q];
    }
}

// ---------------------------------------------------------------------------
// reductions and pointwise helpers
// ---------------------------------------------------------------------------

__global__ void k_reduce(const double* __restrict__ partial, int count, int groups, double* __restrict__ out) {
    __shared__ double red[kThreads];
    const int slot = blockIdx.x / groups, grp = blockIdx.x % groups;
    const int per = count / groups;
    const double* p = partial + (long long)slot * count + (long long)grp * per;
    double acc = 0.0;
    for (int i = threadIdx.x; i < per; i += blockDim.x) acc += p[i];
    double s = block_sum(acc, red);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

template <typename R>
__global__ void k_init_tau(GridDesc g, unsigned mask, R* __restrict__ tau) {
    const int slot = blockIdx.y;
    if (!slot_active(g, mask, slot)) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N3; i += (long long)gridDim.x * blockDim.x) {
        const int ph = g.phase[i];
        const double kp = ph == 0 ? g.KP[0] : (ph == 1 ? g.KP[1] : g.KP[2]);
        for (int c = 0; c < 3; ++c) tau[((long long)slot * 3 + c) * g.N3 + i] = R(kp * g.E[slot][c]);
    }
}

template <typename R>
__global__ void k_e_to_tau(GridDesc g, int slot, const double* __restrict__ e, R* __restrict__ tau) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N3; i += (long long)gridDim.x * blockDim.x) {
        const int ph = g.phase[i];
        const double kp = ph == 0 ? g.KP[0] : (ph == 1 ? g.KP[1] : g.KP[2]);
        for (int c = 0; c < 3; ++c) tau[((long long)slot * 3 + c) * g.N3 + i] = R(kp * e[c * g.N3 + i]);
    }
}

template <typename R>
__global__ void k_tau_to_e(GridDesc g, int slot, const R* __restrict__ tau, double* __restrict__ e) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N3; i += (long long)gridDim.x * blockDim.x) {
        const int ph = g.phase[i];
        const double kp = ph == 0 ? g.KP[0] : (ph == 1 ? g.KP[1] : g.KP[2]);
        for (int c = 0; c < 3; ++c) e[c * g.N3 + i] = (double)tau[((long long)slot * 3 + c) * g.N3 + i] / kp;
    }
}

__global__ void k_widen(GridDesc g, unsigned mask, const float* __restrict__ src, double* __restrict__ dst) {
    const int slot = blockIdx.y;
    if (!slot_active(g, mask, slot)) return;
    const long long n = 3 * g.N3, off = (long long)slot * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[off + i] = (double)src[off + i];
}

__global__ void k_axpy(GridDesc g, unsigned mask, const float* __restrict__ d, double* __restrict__ tau) {
    const int slot = blockIdx.y;
    if (!slot_active(g, mask, slot)) return;
    const long long n = 3 * g.N3, off = (long long)slot * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        tau[off + i] += (double)d[off + i];
}

template <typename R>
__global__ void k_convert(const double* __restrict__ s, R* __restrict__ d, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        d[i] = R(s[i]);
}

template <typename R>
__global__ void k_convert_back(const R* __restrict__ s, double* __restrict__ d, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        d[i] = (double)s[i];
}

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------

static int pointwise_blocks(long long n) {
    long long b = (n + kThreads - 1) / kThreads;
    return (int)(b < 152 * 16 ? b : 152 * 16);
}

int x_ctas(const GridDesc& g) { return (int)(3 * g.NN / g.rows); }
int z_ctas(const GridDesc& g) { return g.N * (g.M / g.Pz); }

template <> int x_ctas_for<float>(const GridDesc& g) {
    if (g.xyvar == 1 && fused_cluster(g.N)) return fused_xy_ctas(g);
    const int f = fast_x_ctas(g);
    return f ? f : x_ctas(g);
}
template <> int x_ctas_for<double>(const GridDesc& g) {
    GridDesc t = g;
    set_tiles(t, true);
    return x_ctas(t);
}
template <> int z_ctas_for<float>(const GridDesc& g) {
    const int f = fast_z_ctas(g);
    return f ? f : z_ctas(g);
}
template <> int z_ctas_for<double>(const GridDesc& g) {
    GridDesc t = g;
    set_tiles(t, true);
    return z_ctas(t);
}

template <typename R, typename K>
static void set_smem(K kern, size_t bytes) {
    // static (2 KB) plus dynamic shared memory above 48 KB needs the opt-in
    if (bytes > 32 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename R>
void launch_x_forward(const GridDesc& g, int mode, unsigned mask, const R* tau, void* spec,
                      double* partial, cudaStream_t st) {
    using T2 = typename Cplx<R>::T;
    if constexpr (std::is_same<R, float>::value) {
        if (fast_x_forward(g, mode, mask, tau, spec, partial, st)) return;
    }
    GridDesc t = g;   // FP64 passes take the FP64 tiles
    if constexpr (std::is_same<R, double>::value) set_tiles(t, true);
    const size_t sm = 2ull * t.rows * t.M * sizeof(T2);
    dim3 grid(x_ctas(t), t.nslots);
    T2* sp = reinterpret_cast<T2*>(spec);
    if (mode == XF_PLAIN) {
        set_smem<R>(k_x_forward<R, XF_PLAIN>, sm);
        k_x_forward<R, XF_PLAIN><<<grid, kThreads, sm, st>>>(t, mask, tau, sp, partial);
    } else if (mode == XF_POLARIZE) {
        set_smem<R>(k_x_forward<R, XF_POLARIZE>, sm);
        k_x_forward<R, XF_POLARIZE><<<grid, kThreads, sm, st>>>(t, mask, tau, sp, partial);
    } else {
        set_smem<R>(k_x_forward<R, XF_FLUX>, sm);
        k_x_forward<R, XF_FLUX><<<grid, kThreads, sm, st>>>(t, mask, tau, sp, partial);
    }
}

template <typename R>
void launch_y_pass(const GridDesc& g, bool forward, unsigned mask, void* spec, cudaStream_t st) {
    using T2 = typename Cplx<R>::T;
    if constexpr (std::is_same<R, float>::value) {
        if (fast_y(g, forward, mask, spec, st)) return;
    }
    GridDesc t = g;   // FP64 passes take the FP64 tiles
    if constexpr (std::is_same<R, double>::value) set_tiles(t, true);
    const size_t sm = 2ull * t.N * t.Py * sizeof(T2);
    dim3 grid(3 * t.N * (t.M / t.Py), t.nslots);
    T2* sp = reinterpret_cast<T2*>(spec);
    if (forward) {
        set_smem<R>(k_y_pass<R, true>, sm);
        k_y_pass<R, true><<<grid, kThreads, sm, st>>>(t, mask, sp);
    } else {
        set_smem<R>(k_y_pass<R, false>, sm);
        k_y_pass<R, false><<<grid, kThreads, sm, st>>>(t, mask, sp);
    }
}

template <typename R>
void launch_z_pass(const GridDesc& g, int mode, unsigned mask, void* spec, double* partial, cudaStream_t st) {
    using T2 = typename Cplx<R>::T;
    if constexpr (std::is_same<R, float>::value) {
        if (fast_z(g, mode, mask, spec, partial, st)) return;
    }
    GridDesc t = g;   // FP64 passes take the FP64 tiles
    if constexpr (std::is_same<R, double>::value) set_tiles(t, true);
    const size_t sm = 2ull * 3 * t.N * t.Pz * sizeof(T2);
    dim3 grid(z_ctas(t), t.nslots);
    T2* sp = reinterpret_cast<T2*>(spec);
    switch (mode) {
        case Z_FWD:
            set_smem<R>(k_z_pass<R, Z_FWD>, sm);
            k_z_pass<R, Z_FWD><<<grid, kThreads, sm, st>>>(t, mask, sp, partial);
            break;
        case Z_INV:
            set_smem<R>(k_z_pass<R, Z_INV>, sm);
            k_z_pass<R, Z_INV><<<grid, kThreads, sm, st>>>(t, mask, sp, partial);
            break;
        case Z_ITER:
            set_smem<R>(k_z_pass<R, Z_ITER>, sm);
            k_z_pass<R, Z_ITER><<<grid, kThreads, sm, st>>>(t, mask, sp, partial);
            break;
        case Z_ITER_NOB:
            set_smem<R>(k_z_pass<R, Z_ITER_NOB>, sm);
            k_z_pass<R, Z_ITER_NOB><<<grid, kThreads, sm, st>>>(t, mask, sp, partial);
            break;
        default:
            set_smem<R>(k_z_pass<R, Z_EQ>, sm);
            k_z_pass<R, Z_EQ><<<grid, kThreads, sm, st>>>(t, mask, sp, partial);
            break;
    }
}

template <typename R>
void launch_x_inverse(const GridDesc& g, int mode, unsigned mask, const void* spec, R* tau,
                      const float* r32, float* d32, float* r32_out, double* partial, cudaStream_t st) {
    using T2 = typename Cplx<R>::T;
    if constexpr (std::is_same<R, float>::value) {
        if (fast_x_inverse(g, mode, mask, spec, tau, r32, partial, st)) return;
    }
    GridDesc t = g;   // FP64 passes take the FP64 tiles
    if constexpr (std::is_same<R, double>::value) set_tiles(t, true);
    const size_t sm = 2ull * t.rows * t.M * sizeof(T2);
    dim3 grid(x_ctas(t), t.nslots);
    const T2* sp = reinterpret_cast<const T2*>(spec);
#define HMG_XI(MODE_)                                                                        \
    set_smem<R>(k_x_inverse<R, MODE_>, sm);                                                  \
    k_x_inverse<R, MODE_><<<grid, kThreads, sm, st>>>(t, mask, sp, tau, r32, d32, r32_out, partial)
    switch (mode) {
        case XI_PLAIN: HMG_XI(XI_PLAIN); break;
        case XI_INPLACE: HMG_XI(XI_INPLACE); break;
        case XI_INPLACE_RES: HMG_XI(XI_INPLACE_RES); break;
        case XI_ADD_R_RES: HMG_XI(XI_ADD_R_RES); break;
        case XI_ADD_R: HMG_XI(XI_ADD_R); break;
        default: HMG_XI(XI_DIFF); break;
    }
#undef HMG_XI
}

template <typename R>
bool launch_xy_forward(const GridDesc& g, int mode, unsigned mask, const R* tau, void* spec, double* partial,
                       cudaStream_t st) {
    if constexpr (std::is_same<R, float>::value) {
        if (g.xyvar == 1 && fused_xy_forward(g, mode, mask, tau, spec, partial, st)) return true;
    }
    launch_x_forward<R>(g, mode, mask, tau, spec, partial, st);
    launch_y_pass<R>(g, true, mask, spec, st);
    return false;
}

template <typename R>
bool launch_yx_inverse(const GridDesc& g, int mode, unsigned mask, const void* spec, R* tau, const float* r32,
                       float* d32, float* r32_out, double* partial, cudaStream_t st) {
    if constexpr (std::is_same<R, float>::value) {
        if (g.xyvar == 1 && fused_yx_inverse(g, mode, mask, spec, tau, r32, partial, st)) return true;
    }
    launch_y_pass<R>(g, false, mask, const_cast<void*>(spec), st);
    launch_x_inverse<R>(g, mode, mask, spec, tau, r32, d32, r32_out, partial, st);
    return false;
}

void launch_reduce(const double* partial, int nslots, int count, int groups, double* out, cudaStream_t st) {
    k_reduce<<<nslots * groups, kThreads, 0, st>>>(partial, count, groups, out);
}

template <typename R>
void launch_init_tau(const GridDesc& g, unsigned mask, R* tau, cudaStream_t st) {
    k_init_tau<R><<<dim3(pointwise_blocks(g.N3), g.nslots), kThreads, 0, st>>>(g, mask, tau);
}
template <typename R>
void launch_e_to_tau(const GridDesc& g, int slot, const double* e, R* tau, cudaStream_t st) {
    k_e_to_tau<R><<<pointwise_blocks(g.N3), kThreads, 0, st>>>(g, slot, e, tau);
}
template <typename R>
void launch_tau_to_e(const GridDesc& g, int slot, const R* tau, double* e, cudaStream_t st) {
    k_tau_to_e<R><<<pointwise_blocks(g.N3), kThreads, 0, st>>>(g, slot, tau, e);
}
void launch_widen(const GridDesc& g, unsigned mask, const float* src, double* dst, cudaStream_t st) {
    k_widen<<<dim3(pointwise_blocks(3 * g.N3), g.nslots), kThreads, 0, st>>>(g, mask, src, dst);
}
void launch_axpy(const GridDesc& g, unsigned mask, const float* d, double* tau, cudaStream_t st) {
    k_axpy<<<dim3(pointwise_blocks(3 * g.N3), g.nslots), kThreads, 0, st>>>(g, mask, d, tau);
}
template <typename R>
void launch_convert(const double* src, R* dst, long long n, cudaStream_t st) {
    k_convert<R><<<pointwise_blocks(n), kThreads, 0, st>>>(src, dst, n);
}
template <typename R>
void launch_convert_back(const R* src, double* dst, long long n, cudaStream_t st) {
    k_convert_back<R><<<pointwise_blocks(n), kThreads, 0, st>>>(src, dst, n);
}

#define HMG_INST(R)                                                                                         \
    template void launch_x_forward<R>(const GridDesc&, int, unsigned, const R*, void*, double*, cudaStream_t); \
    template void launch_y_pass<R>(const GridDesc&, bool, unsigned, void*, cudaStream_t);                   \
    template void launch_z_pass<R>(const GridDesc&, int, unsigned, void*, double*, cudaStream_t);           \
    template void launch_x_inverse<R>(const GridDesc&, int, unsigned, const void*, R*, const float*, float*, \
                                      float*, double*, cudaStream_t);                                       \
    template void launch_init_tau<R>(const GridDesc&, unsigned, R*, cudaStream_t);                          \
    template bool launch_xy_forward<R>(const GridDesc&, int, unsigned, const R*, void*, double*, cudaStream_t); \
    template bool launch_yx_inverse<R>(const GridDesc&, int, unsigned, const void*, R*, const float*, float*,   \
                                       float*, double*, cudaStream_t);                                        \
    template void launch_e_to_tau<R>(const GridDesc&, int, const double*, R*, cudaStream_t);                \
    template void launch_tau_to_e<R>(const GridDesc&, int, const R*, double*, cudaStream_t);                \
    template void launch_convert<R>(const double*, R*, long long, cudaStream_t);                            \
    template void launch_convert_back<R>(const R*, double*, long long, cudaStream_t);
HMG_INST(float)
HMG_INST(double)
#undef HMG_INST

}  // namespace hmg
