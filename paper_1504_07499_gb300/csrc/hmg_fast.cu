// Register-resident FFT passes (FP32) for the common grid sizes.
//
// A 1D transform of length L = E * TP runs as two register stages (the four-step
// factorization; n = TP n1 + n2, k = k1 + E k2):
//   stage 1: thread n2 holds x[TP n1 + n2] (n1 < E) straight from HBM, computes the
//            length-E DFT over n1 in registers and multiplies by w_L^(n2 k1);
//   exchange through shared memory (one write, one read);
//   stage 2: thread t holds, for its E/TP values of k1, all TP values of n2 and
//            computes length-TP DFTs, giving X[k1 + E k2] in registers.
// X(k1 + E k2) = sum_n1 w_E^(n1 k1) w_L^(n2 k1) sum_n2 ... is the textbook split of the
// DFT sum; the inverse runs the same stages with conjugate factors, or in reverse order
// when it starts from stage-2 registers (z pass: forward, Green operator in registers,
// inverse back to the natural layout without an extra exchange).
// Loads and stores go between HBM and registers with the pencil index fastest across
// threads, so every warp access is a run of contiguous bytes.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hmg_fft.cuh"
#include "hmg_green.cuh"
#include "hmg_internal.h"
#include "hmg_regfft.cuh"

namespace hmg {
namespace fast {

// ---------------------------------------------------------------------------
// y pass: P consecutive kx columns of one (component, z) plane; threads (p, t)
// ---------------------------------------------------------------------------

template <int L, int P, bool FWD>
__global__ void __launch_bounds__(P * Split<L>::TP, 3)
k_fy(GridDesc g, unsigned mask, float2* __restrict__ spec) {
    constexpr int E = Split<L>::E, TP = Split<L>::TP;
    const int slot = blockIdx.y;
    if (!slot_active(g, mask, slot)) return;
    extern __shared__ __align__(16) float2 sh[];   // xslots<L>() * P
    const int M = g.M;
    const int p = threadIdx.x % P, t = threadIdx.x / P;
    const int nkb = M / P;
    const int kb = blockIdx.x % nkb;
    const long long cz = blockIdx.x / nkb;
    float2* base = spec + (long long)slot * 3 * g.NNM + cz * (long long)L * M + kb * P + p;
    float2 v[E];
#pragma unroll
    for (int n1 = 0; n1 < E; ++n1) v[n1] = base[(long long)(TP * n1 + t) * M];
    const float2* twL = g.tw32 + g.pN.tw_off;
    stage1_write<L, FWD>(v, t, twL, sh + p, P);
    __syncthreads();
    stage2_read<L, FWD>(v, t, sh + p, P);
    constexpr int KPT = E / TP;
#pragma unroll
    for (int i = 0; i < KPT; ++i)
#pragma unroll
        for (int k2 = 0; k2 < TP; ++k2) base[(long long)(t * KPT + i + E * k2) * M] = v[i * TP + k2];
}

// ---------------------------------------------------------------------------
// z pass: P consecutive kx columns at one ky; three thread groups, one per
// component.  The Green operator needs, per mode, the projection d . s over the
// three components: each thread writes its component's share to shared memory,
// reads the other two, and updates its own component.
// ---------------------------------------------------------------------------

// Projector data of packed mode (kx, ky, kz) for component c, for the real part
// (plane kx, or plane 0 of the packed column) and the imaginary part (same plane,
// or plane N/2 at the four self-conjugate modes of the packed column):
// integer direction component d and |d|^2 (0 where the projector vanishes).
__device__ __forceinline__ void mode_parts(int kx, int ky, int kz, int N, int c, int& dA, int& nA, int& dB,
                                           int& nB) {
    const int my = signed_mode(ky, N), mz = signed_mode(kz, N);
    int d[3];
    if (kx == 0 && (ky == 0 || ky == N / 2) && (kz == 0 || kz == N / 2)) {
        nA = mode_dir(0, my, mz, N, d);
        dA = d[c];
        nB = mode_dir(N / 2, my, mz, N, d);
        dB = d[c];
    } else {
        nA = nB = mode_dir(kx, my, mz, N, d);
        dA = dB = d[c];
    }
}

template <int L, int P, int MODE>
__global__ void __launch_bounds__(P * Split<L>::TP, 3)
k_fz3(GridDesc g, unsigned mask, float2* __restrict__ spec, double* __restrict__ partial) {
    constexpr int E = Split<L>::E, TP = Split<L>::TP, KPT = E / TP;
    constexpr int NS = xslots<L>() * P;
    const int slot = blockIdx.y;
    if (!slot_active(g, mask, slot)) return;
    extern __shared__ __align__(16) float2 sh[];   // 3 * NS
    __shared__ double red[P * TP];
    constexpr int N = L, M = L / 2;
    constexpr long long NNM = (long long)N * N * M;
    const int p = threadIdx.x % P, t = threadIdx.x / P;
    const int nkb = M / P;
    const int kb = blockIdx.x % nkb;
    const int ky = blockIdx.x / nkb;
    const int kx = kb * P + p;
    float2* base = spec + (long long)slot * 3 * NNM + (long long)ky * M + kb * P + p;
    constexpr long long rowz = (long long)N * M;     // stride between z rows
    const float2* twL = g.tw32 + g.pN.tw_off;
    float2 v[3][E];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int n1 = 0; n1 < E; ++n1) v[c][n1] = base[c * NNM + (long long)(TP * n1 + t) * rowz];

    if (MODE == Z_INV) {
        // plain inverse transform of each component (natural order in and out)
#pragma unroll
        for (int c = 0; c < 3; ++c) stage1_write<L, false>(v[c], t, twL, sh + c * NS + p, P);
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 3; ++c) stage2_read<L, false>(v[c], t, sh + c * NS + p, P);
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) stage1_write<L, true>(v[c], t, twL, sh + c * NS + p, P);
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 3; ++c) stage2_read<L, true>(v[c], t, sh + c * NS + p, P);
    }
    if (MODE == Z_FWD || MODE == Z_INV) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int i = 0; i < KPT; ++i)
#pragma unroll
                for (int k2 = 0; k2 < TP; ++k2)
                    base[c * NNM + (long long)(t * KPT + i + E * k2) * rowz] = v[c][i * TP + k2];
        return;
    }
    if (MODE == Z_EQ) {
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < KPT; ++i)
#pragma unroll
            for (int k2 = 0; k2 < TP; ++k2)
                acc += eq_mode(kx, ky, t * KPT + i + E * k2, N, v[0][i * TP + k2], v[1][i * TP + k2], v[2][i * TP + k2]);
        const double twopi_n = 6.283185307179586476925 / (double)N;
        const double s = block_sum_d(acc, red) * twopi_n * twopi_n / ((double)g.N3 * (double)g.N3);
        if (threadIdx.x == 0) partial[(long long)slot * gridDim.x + blockIdx.x] = s;
        return;
    }
    // Green operator on the registers, then the inverse back to natural order
    const bool addb = g.dflags ? (g.dflags[slot] & SF_ADDB) != 0 : MODE == Z_ITER;
    const float scale = (float)(1.0 / (double)g.N3);
    const float twok0E[3] = {(float)(2.0 * g.k0 * g.E[slot][0]), (float)(2.0 * g.k0 * g.E[slot][1]),
                             (float)(2.0 * g.k0 * g.E[slot][2])};
#pragma unroll
    for (int i = 0; i < KPT; ++i)
#pragma unroll
        for (int k2 = 0; k2 < TP; ++k2)
            green_mode<float>(kx, ky, t * KPT + i + E * k2, N, scale, addb, twok0E, v[0][i * TP + k2],
                              v[1][i * TP + k2], v[2][i * TP + k2]);
    __syncthreads();   // every thread has read the forward exchange
#pragma unroll
    for (int c = 0; c < 3; ++c) rstage2_write<L>(v[c], t, twL, sh + c * NS + p, P);
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 3; ++c) rstage1_read<L>(v[c], t, sh + c * NS + p, P);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int n1 = 0; n1 < E; ++n1) base[c * NNM + (long long)(TP * n1 + t) * rowz] = v[c][n1];
}

// Variant 1: three thread groups, one per component; the projection d . s is summed
// through shared memory (more threads, fewer registers per thread).
template <int L, int P, int MODE>
__global__ void __launch_bounds__(3 * P * Split<L>::TP, 1)
k_fzs(GridDesc g, unsigned mask, float2* __restrict__ spec, double* __restrict__ partial) {
    constexpr int E = Split<L>::E, TP = Split<L>::TP, KPT = E / TP;
    constexpr int NS = xslots<L>() * P;
    const int slot = blockIdx.y;
    if (!slot_active(g, mask, slot)) return;
    extern __shared__ __align__(16) float2 sh[];   // 3 * NS
    __shared__ double red[3 * P * Split<L>::TP / 32 + 1];
    constexpr int N = L, M = L / 2;
    constexpr long long NNM = (long long)N * N * M;
    const int lt = threadIdx.x % (P * TP), c = threadIdx.x / (P * TP);
    const int p = lt % P, t = lt / P;
    const int nkb = M / P;
    const int kb = blockIdx.x % nkb;
    const int ky = blockIdx.x / nkb;
    const int kx = kb * P + p;
    float2* base = spec + (long long)slot * 3 * NNM + c * NNM + (long long)ky * M + kb * P + p;
    constexpr long long rowz = (long long)N * M;     // stride between z rows
    const float2* twL = g.tw32 + g.pN.tw_off;
    float2* shc = sh + c * NS + p;
    float2 v[E];
#pragma unroll
    for (int n1 = 0; n1 < E; ++n1) v[n1] = base[(long long)(TP * n1 + t) * rowz];

    if (MODE == Z_INV) {
        stage1_write<L, false>(v, t, twL, shc, P);
        __syncthreads();
        stage2_read<L, false>(v, t, shc, P);
    } else {
        stage1_write<L, true>(v, t, twL, shc, P);
        __syncthreads();
        stage2_read<L, true>(v, t, shc, P);
    }
    if (MODE == Z_FWD || MODE == Z_INV) {
#pragma unroll
        for (int i = 0; i < KPT; ++i)
#pragma unroll
            for (int k2 = 0; k2 < TP; ++k2) base[(long long)(t * KPT + i + E * k2) * rowz] = v[i * TP + k2];
        return;
    }
    // share of d . s of this component, one slot per (t, value) of the thread group
    __syncthreads();   // every thread has read the forward exchange
#pragma unroll
    for (int i = 0; i < KPT; ++i)
#pragma unroll
        for (int k2 = 0; k2 < TP; ++k2) {
            int dA, nA, dB, nB;
            mode_parts(kx, ky, t * KPT + i + E * k2, N, c, dA, nA, dB, nB);
            const float2 x = v[i * TP + k2];
            shc[((i * TP + k2) * TP + t) * P] = make_float2((float)dA * x.x, (float)dB * x.y);
        }
    __syncthreads();
    const float2* sh1 = sh + ((c + 1) % 3) * NS + p;
    const float2* sh2 = sh + ((c + 2) % 3) * NS + p;
    if (MODE == Z_EQ) {
        double acc = 0.0;
        if (c == 0) {
#pragma unroll
            for (int i = 0; i < KPT; ++i)
#pragma unroll
                for (int k2 = 0; k2 < TP; ++k2) {
                    const int q = ((i * TP + k2) * TP + t) * P;
                    const float2 a = shc[q], b = sh1[q], e = sh2[q];
                    const double dx = (double)a.x + (double)b.x + (double)e.x;
                    const double dy = (double)a.y + (double)b.y + (double)e.y;
                    const int kz = t * KPT + i + E * k2;
                    const bool special = (kx == 0) && (ky == 0 || ky == N / 2) && (kz == 0 || kz == N / 2);
                    acc += (kx == 0 || special ? 1.0 : 2.0) * (dx * dx + dy * dy);
                }
        }
        const double twopi_n = 6.283185307179586476925 / (double)N;
        const double sm = block_sum_any(acc, red) * twopi_n * twopi_n / ((double)g.N3 * (double)g.N3);
        if (threadIdx.x == 0) partial[(long long)slot * gridDim.x + blockIdx.x] = sm;
        return;
    }
    const bool addb = g.dflags ? (g.dflags[slot] & SF_ADDB) != 0 : MODE == Z_ITER;
    const float scale = (float)(1.0 / (double)g.N3);
    const float twok0E = (float)(2.0 * g.k0 * g.E[slot][c]);
#pragma unroll
    for (int i = 0; i < KPT; ++i)
#pragma unroll
        for (int k2 = 0; k2 < TP; ++k2) {
            const int kz = t * KPT + i + E * k2;
            int dA, nA, dB, nB;
            mode_parts(kx, ky, kz, N, c, dA, nA, dB, nB);
            const int q = ((i * TP + k2) * TP + t) * P;
            const float2 a = shc[q], b = sh1[q], e = sh2[q];
            const float dotA = a.x + b.x + e.x, dotB = a.y + b.y + e.y;
            const float fA = nA > 0 ? 2.0f / (float)nA : 0.0f, fB = nB > 0 ? 2.0f / (float)nB : 0.0f;
            float2& x = v[i * TP + k2];
            x.x = scale * (x.x - fA * (float)dA * dotA);
            x.y = scale * (x.y - fB * (float)dB * dotB);
            if (addb && kx == 0 && ky == 0 && kz == 0) x.x += twok0E;
        }
    __syncthreads();   // every thread has read the shares
    rstage2_write<L>(v, t, twL, shc, P);
    __syncthreads();
    rstage1_read<L>(v, t, shc, P);
#pragma unroll
    for (int n1 = 0; n1 < E; ++n1) base[(long long)(TP * n1 + t) * rowz] = v[n1];
}

// ---------------------------------------------------------------------------
// x passes: R rows per CTA, threads (t, r) with t fastest along the row
// ---------------------------------------------------------------------------

template <int M, int RW, int MODE>
__global__ void __launch_bounds__(RW * Split<M>::TP, 4)
k_fx_forward(GridDesc g, unsigned mask, const float* __restrict__ tau, float2* __restrict__ spec,
             double* __restrict__ partial) {
    constexpr int E = Split<M>::E, TP = Split<M>::TP, KPT = E / TP, RS = row_stride<M>();
    const int slot = blockIdx.y;
    if (!slot_active(g, mask, slot)) return;
    extern __shared__ __align__(16) float2 sh[];   // RW * RS
    __shared__ double red[RW * TP];
    const int N = g.N;
    const int t = threadIdx.x % TP, r = threadIdx.x / TP;
    // component fastest across CTAs, so the three components of a (z, y) block read the
    // same phase rows close together in time (L2 hits)
    const int comp = blockIdx.x % 3;
    const long long rblk = blockIdx.x / 3;
    const long long row = comp * g.NN + rblk * RW + r;              // c*NN + z*N + y
    const long long pidx = comp * (g.NN / RW) + rblk;               // component-major CTA index
    const float2* src = reinterpret_cast<const float2*>(tau + (long long)slot * 3 * g.N3 + row * N);
    const uchar2* ph = reinterpret_cast<const uchar2*>(g.phase + (row % g.NN) * N);
    float2 v[E];
#pragma unroll
    for (int n1 = 0; n1 < E; ++n1) v[n1] = src[TP * n1 + t];
    float acc = 0.f;
    if (MODE != XF_PLAIN) {
        const float c0 = (float)(MODE == XF_POLARIZE ? g.Y[0] : g.W[0]);
        const float c1 = (float)(MODE == XF_POLARIZE ? g.Y[1] : g.W[1]);
        const float c2 = (float)(MODE == XF_POLARIZE ? g.Y[2] : g.W[2]);
#pragma unroll
        for (int n1 = 0; n1 < E; ++n1) {
            const uchar2 q = ph[TP * n1 + t];
            // rounded products (never contracted into the transform's adds), as in k_fx_round
            v[n1].x = __fmul_rn(v[n1].x, sel3f(q.x, c0, c1, c2));
            v[n1].y = __fmul_rn(v[n1].y, sel3f(q.y, c0, c1, c2));
            if (MODE == XF_FLUX) acc += v[n1].x + v[n1].y;
        }
    }
    const float2* twM = g.tw32 + g.pM.tw_off;
    float2* rs = sh + r * RS;
    stage1_write<M, true>(v, t, twM, rs, 1);
    __syncthreads();
    stage2_read<M, true>(v, t, rs, 1);
    __syncthreads();
    // natural order into shared memory for the real split
#pragma unroll
    for (int i = 0; i < KPT; ++i)
#pragma unroll
        for (int k2 = 0; k2 < TP; ++k2) rs[t * KPT + i + E * k2] = v[i * TP + k2];
    if (MODE == XF_FLUX) {
        const double s = block_sum_d((double)acc, red);
        if (threadIdx.x == 0) partial[(long long)slot * gridDim.x + pidx] = s;
    } else {
        __syncthreads();
    }
    const float2* twN = g.tw32 + g.pN.tw_off;
    float2* dst = spec + (long long)slot * 3 * g.NNM + row * M;
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int k = t + TP * j;
        const float2 z = rs[k];
        float2 out;
        if (k == 0) {
            out = make_float2(z.x + z.y, z.x - z.y);
        } else {
            const float2 zm = rs[M - k];
            const float2 e = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
            const float2 o = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
            out = cadd(e, cmul(o, __ldg(&twN[k])));
        }
        dst[k] = out;
    }
}

template <int M, int RW, int MODE>
__global__ void __launch_bounds__(RW * Split<M>::TP, 3)
k_fx_inverse(GridDesc g, unsigned mask, const float2* __restrict__ spec, float* __restrict__ tau,
             const float* __restrict__ r32, double* __restrict__ partial) {
    constexpr int E = Split<M>::E, TP = Split<M>::TP, KPT = E / TP, RS = row_stride<M>();
    const int slot = blockIdx.y;
    if (!slot_active(g, mask, slot)) return;
    extern __shared__ __align__(16) float2 sh[];   // RW * RS
    __shared__ double red[RW * TP];
    const int N = g.N;
    const int t = threadIdx.x % TP, r = threadIdx.x / TP;
    const long long row = (long long)blockIdx.x * RW + r;
    const long long fbase = (long long)slot * 3 * g.N3 + row * N;
    float2* out = reinterpret_cast<float2*>(tau + fbase);
    // prefetch the old field (and r) for the output step: in flight during the FFT
    constexpr bool kRes = MODE == XI_INPLACE_RES || MODE == XI_ADD_R_RES;
    constexpr bool kAddR = MODE == XI_ADD_R_RES || MODE == XI_ADD_R;
    const bool res = kRes && (g.dflags ? g.resid != 0 : true);
    const bool addr = kAddR && (g.dflags ? (g.dflags[slot] & SF_ADDR) != 0 : true);
    float2 old[E], radd[E];
    if (res) {
#pragma unroll
        for (int j = 0; j < E; ++j) old[j] = out[t + TP * j];
    }
    if (addr) {
        const float2* rr = reinterpret_cast<const float2*>(r32 + fbase);
#pragma unroll
        for (int j = 0; j < E; ++j) radd[j] = rr[t + TP * j];
    }
    const float2* src = spec + (long long)slot * 3 * g.NNM + row * M;
    float2* rs = sh + r * RS;
#pragma unroll
    for (int j = 0; j < E; ++j) rs[t + TP * j] = src[t + TP * j];
    __syncthreads();
    // complex-to-real merge into the stage-1 layout
    const float2* twN = g.tw32 + g.pN.tw_off;
    float2 v[E];
#pragma unroll
    for (int n1 = 0; n1 < E; ++n1) {
        const int k = TP * n1 + t;
        float2 xk, xm;
        if (k == 0) {
            const float2 q = rs[0];
            xk = make_float2(q.x, 0.f);
            xm = make_float2(q.y, 0.f);
        } else {
            xk = rs[k];
            xm = rs[M - k];
        }
        const float2 s = make_float2(xk.x + xm.x, xk.y - xm.y);
        const float2 d = make_float2(xk.x - xm.x, xk.y + xm.y);
        const float2 dw = cmulc(d, __ldg(&twN[k]));
        v[n1] = make_float2(s.x - dw.y, s.y + dw.x);
    }
    __syncthreads();
    const float2* twM = g.tw32 + g.pM.tw_off;
    stage1_write<M, false>(v, t, twM, rs, 1);
    __syncthreads();
    stage2_read<M, false>(v, t, rs, 1);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < KPT; ++i)
#pragma unroll
        for (int k2 = 0; k2 < TP; ++k2) rs[t * KPT + i + E * k2] = v[i * TP + k2];
    __syncthreads();
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < E; ++j) {
        float2 x = rs[t + TP * j];
        if (addr) x = make_float2(__fadd_rn(x.x, radd[j].x), __fadd_rn(x.y, radd[j].y));
        if (res) {
            const float da = x.x - old[j].x, db = x.y - old[j].y;
            acc += da * da + db * db;
        }
        out[t + TP * j] = x;
    }
    if (kRes) {   // uniform across the CTA (kernel argument and per-slot flag)
        const double s = block_sum_d((double)acc, red);
        if (threadIdx.x == 0 && res) partial[(long long)slot * gridDim.x + blockIdx.x] = s;
    }
}

// x inverse of one sweep fused with the polarization and x forward of the next sweep
// (steps 5-7 of sweep n, steps 2-3 of sweep n + 1) over each row: the updated field
// tau^{n+1} (plus the defect r in correction sweeps) stays in registers and is written
// to memory only when WTAU is set (the field a following residual sweep compares
// against).  The spectrum is transformed in place.  Same float operations as
// k_fx_inverse followed by k_fx_forward<XF_POLARIZE>, so results are identical.
template <int M, int RW, bool ADDR, bool WTAU>
__global__ void __launch_bounds__(RW * Split<M>::TP, 2)
k_fx_round(GridDesc g, unsigned mask, float2* __restrict__ spec, float* __restrict__ tau,
           const float* __restrict__ r32) {
    constexpr int E = Split<M>::E, TP = Split<M>::TP, KPT = E / TP, RS = row_stride<M>();
    const int slot = blockIdx.y;
    if (!slot_active(g, mask, slot)) return;
    extern __shared__ __align__(16) float2 sh[];   // RW * RS
    const int N = g.N;
    const int t = threadIdx.x % TP, r = threadIdx.x / TP;
    // component fastest across CTAs (phase rows reused from L2, as in k_fx_forward)
    const int comp = blockIdx.x % 3;
    const long long rblk = blockIdx.x / 3;
    const long long row = comp * g.NN + rblk * RW + r;              // c*NN + z*N + y
    const long long fbase = (long long)slot * 3 * g.N3 + row * N;
    const bool addr = ADDR && (g.dflags ? (g.dflags[slot] & SF_ADDR) != 0 : true);
    // loads for the update and the polarization: in flight during the inverse FFT
    float2 radd[E];
    if (addr) {
        const float2* rr = reinterpret_cast<const float2*>(r32 + fbase);
#pragma unroll
        for (int j = 0; j < E; ++j) radd[j] = rr[t + TP * j];
    }
    const uchar2* ph = reinterpret_cast<const uchar2*>(g.phase + (row % g.NN) * N);
    uchar2 q[E];
#pragma unroll
    for (int j = 0; j < E; ++j) q[j] = ph[TP * j + t];
    float2* sp = spec + (long long)slot * 3 * g.NNM + row * M;
    float2* rs = sh + r * RS;
#pragma unroll
    for (int j = 0; j < E; ++j) rs[t + TP * j] = sp[t + TP * j];
    __syncthreads();
    // complex-to-real merge into the stage-1 layout
    const float2* twN = g.tw32 + g.pN.tw_off;
    const float2* twM = g.tw32 + g.pM.tw_off;
    float2 v[E];
#pragma unroll
    for (int n1 = 0; n1 < E; ++n1) {
        const int k = TP * n1 + t;
        float2 xk, xm;
        if (k == 0) {
            const float2 z = rs[0];
            xk = make_float2(z.x, 0.f);
            xm = make_float2(z.y, 0.f);
        } else {
            xk = rs[k];
            xm = rs[M - k];
        }
        const float2 s = make_float2(xk.x + xm.x, xk.y - xm.y);
        const float2 d = make_float2(xk.x - xm.x, xk.y + xm.y);
        const float2 dw = cmulc(d, __ldg(&twN[k]));
        v[n1] = make_float2(s.x - dw.y, s.y + dw.x);
    }
    __syncthreads();
    stage1_write<M, false>(v, t, twM, rs, 1);
    __syncthreads();
    stage2_read<M, false>(v, t, rs, 1);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < KPT; ++i)
#pragma unroll
        for (int k2 = 0; k2 < TP; ++k2) rs[t * KPT + i + E * k2] = v[i * TP + k2];
    __syncthreads();
    // update (step 7), optional store, polarization of the next sweep (step 2)
    const float c0 = (float)g.Y[0], c1 = (float)g.Y[1], c2 = (float)g.Y[2];
    float2* out = reinterpret_cast<float2*>(tau + fbase);
#pragma unroll
    for (int j = 0; j < E; ++j) {
        float2 x = rs[t + TP * j];
        if (addr) x = make_float2(__fadd_rn(x.x, radd[j].x), __fadd_rn(x.y, radd[j].y));
        if (WTAU) out[t + TP * j] = x;
        v[j] = make_float2(__fmul_rn(x.x, sel3f(q[j].x, c0, c1, c2)), __fmul_rn(x.y, sel3f(q[j].y, c0, c1, c2)));
    }
    __syncthreads();   // every thread has read its row values
    stage1_write<M, true>(v, t, twM, rs, 1);
    __syncthreads();
    stage2_read<M, true>(v, t, rs, 1);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < KPT; ++i)
#pragma unroll
        for (int k2 = 0; k2 < TP; ++k2) rs[t * KPT + i + E * k2] = v[i * TP + k2];
    __syncthreads();
    // real-to-complex split, written over the row it came from
#pragma unroll
    for (int j = 0; j < E; ++j) {
        const int k = t + TP * j;
        const float2 z = rs[k];
        float2 o2;
        if (k == 0) {
            o2 = make_float2(z.x + z.y, z.x - z.y);
        } else {
            const float2 zm = rs[M - k];
            const float2 e = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
            const float2 o = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
            o2 = cadd(e, cmul(o, __ldg(&twN[k])));
        }
        sp[k] = o2;
    }
}

}  // namespace fast

// ---------------------------------------------------------------------------
// dispatch: a fast kernel exists for FP32 and the lengths with a Split above
// ---------------------------------------------------------------------------

namespace {
// Launch with `bytes` of dynamic shared memory.  Static plus dynamic shared memory
// above 48 KB needs the opt-in, so it is requested whenever the two could exceed it.
template <typename K, typename... Args>
void launch_dyn(K kern, dim3 grid, int threads, size_t bytes, cudaStream_t st, Args... args) {
    if (bytes > 32 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    kern<<<grid, threads, bytes, st>>>(args...);
}
constexpr int pow2_cols(int cap, int M) {
    int p = 1;
    while (p * 2 <= cap && M % (p * 2) == 0) p *= 2;
    return p;
}
template <int L> constexpr int fy_cols() { return pow2_cols(256 / fast::Split<L>::TP, L / 2); }
template <int L> constexpr int fz_cols() { return pow2_cols(128 / fast::Split<L>::TP, L / 2); }
template <int M> constexpr int fx_rows() { return 256 / fast::Split<M>::TP; }
}  // namespace

#define HMG_FAST_LEN(L, X) \
    case L: X(L); return true;

bool fast_y(const GridDesc& g, bool fwd, unsigned mask, void* spec, cudaStream_t st) {
    float2* sp = reinterpret_cast<float2*>(spec);
#define FY(L)                                                                                     \
    {                                                                                             \
        constexpr int P = fy_cols<L>();                                                           \
        if (g.M % P) return false;                                                                \
        dim3 grid(3 * g.N * (g.M / P), g.nslots);                                                 \
        const size_t sm = sizeof(float2) * fast::xslots<L>() * P;                                 \
        if (fwd) launch_dyn(fast::k_fy<L, P, true>, grid, P * fast::Split<L>::TP, sm, st, g, mask, sp);  \
        else launch_dyn(fast::k_fy<L, P, false>, grid, P * fast::Split<L>::TP, sm, st, g, mask, sp);     \
    }
    switch (g.N) {
        HMG_FAST_LEN(64, FY)
        HMG_FAST_LEN(96, FY)
        HMG_FAST_LEN(128, FY)
        HMG_FAST_LEN(192, FY)
        HMG_FAST_LEN(256, FY)
        default: return false;
    }
#undef FY
}

int fast_z_ctas(const GridDesc& g) {
    int P = 0;
    switch (g.N) {
        case 64: P = fz_cols<64>(); break;
        case 96: P = fz_cols<96>(); break;
        case 128: P = fz_cols<128>(); break;
        case 192: P = fz_cols<192>(); break;
        case 256: P = fz_cols<256>(); break;
        default: return 0;
    }
    if (g.M % P) return 0;
    return g.N * (g.M / P);
}

bool fast_z(const GridDesc& g, int mode, unsigned mask, void* spec, double* partial, cudaStream_t st) {
    float2* sp = reinterpret_cast<float2*>(spec);
#define FZ(L)                                                                                          \
    {                                                                                                  \
        constexpr int P = fz_cols<L>();                                                                \
        if (g.M % P) return false;                                                                     \
        dim3 grid(g.N * (g.M / P), g.nslots);                                                          \
        const size_t sm = sizeof(float2) * 3 * fast::xslots<L>() * P;                                  \
        if (g.zvar == 1) {                                                                             \
            constexpr int T = 3 * P * fast::Split<L>::TP;                                              \
            switch (mode) {                                                                            \
                case Z_FWD: launch_dyn(fast::k_fzs<L, P, Z_FWD>, grid, T, sm, st, g, mask, sp, partial); break;   \
                case Z_INV: launch_dyn(fast::k_fzs<L, P, Z_INV>, grid, T, sm, st, g, mask, sp, partial); break;   \
                case Z_ITER: launch_dyn(fast::k_fzs<L, P, Z_ITER>, grid, T, sm, st, g, mask, sp, partial); break; \
                case Z_ITER_NOB: launch_dyn(fast::k_fzs<L, P, Z_ITER_NOB>, grid, T, sm, st, g, mask, sp, partial); break; \
                default: launch_dyn(fast::k_fzs<L, P, Z_EQ>, grid, T, sm, st, g, mask, sp, partial); break;       \
            }                                                                                          \
        } else {                                                                                       \
            constexpr int T = P * fast::Split<L>::TP;                                                  \
            switch (mode) {                                                                            \
                case Z_FWD: launch_dyn(fast::k_fz3<L, P, Z_FWD>, grid, T, sm, st, g, mask, sp, partial); break;   \
                case Z_INV: launch_dyn(fast::k_fz3<L, P, Z_INV>, grid, T, sm, st, g, mask, sp, partial); break;   \
                case Z_ITER: launch_dyn(fast::k_fz3<L, P, Z_ITER>, grid, T, sm, st, g, mask, sp, partial); break; \
                case Z_ITER_NOB: launch_dyn(fast::k_fz3<L, P, Z_ITER_NOB>, grid, T, sm, st, g, mask, sp, partial); break; \
                default: launch_dyn(fast::k_fz3<L, P, Z_EQ>, grid, T, sm, st, g, mask, sp, partial); break;       \
            }                                                                                          \
        }                                                                                              \
    }
    switch (g.N) {
        HMG_FAST_LEN(64, FZ)
        HMG_FAST_LEN(96, FZ)
        HMG_FAST_LEN(128, FZ)
        HMG_FAST_LEN(192, FZ)
        HMG_FAST_LEN(256, FZ)
        default: return false;
    }
#undef FZ
}

int fast_x_ctas(const GridDesc& g) {
    int RW = 0;
    switch (g.M) {
        case 32: RW = fx_rows<32>(); break;
        case 48: RW = fx_rows<48>(); break;
        case 64: RW = fx_rows<64>(); break;
        case 96: RW = fx_rows<96>(); break;
        case 128: RW = fx_rows<128>(); break;
        default: return 0;
    }
    if ((3 * g.NN) % RW || g.NN % RW) return 0;
    return (int)(3 * g.NN / RW);
}

bool fast_x_forward(const GridDesc& g, int mode, unsigned mask, const float* tau, void* spec, double* partial,
                    cudaStream_t st) {
    float2* sp = reinterpret_cast<float2*>(spec);
    if (!fast_x_ctas(g)) return false;
#define FXF(M)                                                                                                 \
    {                                                                                                          \
        constexpr int RW = fx_rows<M>();                                                                       \
        constexpr int T = RW * fast::Split<M>::TP;                                                             \
        dim3 grid(fast_x_ctas(g), g.nslots);                                                                   \
        const size_t sm = sizeof(float2) * RW * fast::row_stride<M>();                                         \
        if (mode == XF_PLAIN) launch_dyn(fast::k_fx_forward<M, RW, XF_PLAIN>, grid, T, sm, st, g, mask, tau, sp, partial); \
        else if (mode == XF_POLARIZE) launch_dyn(fast::k_fx_forward<M, RW, XF_POLARIZE>, grid, T, sm, st, g, mask, tau, sp, partial); \
        else launch_dyn(fast::k_fx_forward<M, RW, XF_FLUX>, grid, T, sm, st, g, mask, tau, sp, partial);        \
    }
    switch (g.M) {
        HMG_FAST_LEN(32, FXF)
        HMG_FAST_LEN(48, FXF)
        HMG_FAST_LEN(64, FXF)
        HMG_FAST_LEN(96, FXF)
        HMG_FAST_LEN(128, FXF)
        default: return false;
    }
#undef FXF
}

bool fast_x_inverse(const GridDesc& g, int mode, unsigned mask, const void* spec, float* tau, const float* r32,
                    double* partial, cudaStream_t st) {
    const float2* sp = reinterpret_cast<const float2*>(spec);
    if (!fast_x_ctas(g)) return false;
    if (mode != XI_PLAIN && mode != XI_INPLACE && mode != XI_INPLACE_RES && mode != XI_ADD_R_RES && mode != XI_ADD_R)
        return false;
#define FXI(M)                                                                                                         \
    {                                                                                                                  \
        constexpr int RW = fx_rows<M>();                                                                               \
        constexpr int T = RW * fast::Split<M>::TP;                                                                     \
        dim3 grid(fast_x_ctas(g), g.nslots);                                                                           \
        const size_t sm = sizeof(float2) * RW * fast::row_stride<M>();                                                 \
        if (mode == XI_INPLACE_RES) launch_dyn(fast::k_fx_inverse<M, RW, XI_INPLACE_RES>, grid, T, sm, st, g, mask, sp, tau, r32, partial); \
        else if (mode == XI_ADD_R_RES) launch_dyn(fast::k_fx_inverse<M, RW, XI_ADD_R_RES>, grid, T, sm, st, g, mask, sp, tau, r32, partial); \
        else if (mode == XI_ADD_R) launch_dyn(fast::k_fx_inverse<M, RW, XI_ADD_R>, grid, T, sm, st, g, mask, sp, tau, r32, partial); \
        else launch_dyn(fast::k_fx_inverse<M, RW, XI_INPLACE>, grid, T, sm, st, g, mask, sp, tau, r32, partial);        \
    }
    switch (g.M) {
        HMG_FAST_LEN(32, FXI)
        HMG_FAST_LEN(48, FXI)
        HMG_FAST_LEN(64, FXI)
        HMG_FAST_LEN(96, FXI)
        HMG_FAST_LEN(128, FXI)
        default: return false;
    }
#undef FXI
}

bool chain_sweeps(const GridDesc& g) {
    return !g.nochain && !(g.xyvar == 1 && fused_cluster(g.N)) && fast_x_ctas(g) > 0;
}

bool fast_x_round(const GridDesc& g, bool addr, bool wtau, unsigned mask, void* spec, float* tau, const float* r32,
                  cudaStream_t st) {
    float2* sp = reinterpret_cast<float2*>(spec);
    if (!fast_x_ctas(g)) return false;
#define FXR(M)                                                                                                      \
    {                                                                                                               \
        constexpr int RW = fx_rows<M>();                                                                            \
        constexpr int T = RW * fast::Split<M>::TP;                                                                  \
        dim3 grid(fast_x_ctas(g), g.nslots);                                                                        \
        const size_t sm = sizeof(float2) * RW * fast::row_stride<M>();                                              \
        if (addr && wtau) launch_dyn(fast::k_fx_round<M, RW, true, true>, grid, T, sm, st, g, mask, sp, tau, r32);   \
        else if (addr) launch_dyn(fast::k_fx_round<M, RW, true, false>, grid, T, sm, st, g, mask, sp, tau, r32);     \
        else if (wtau) launch_dyn(fast::k_fx_round<M, RW, false, true>, grid, T, sm, st, g, mask, sp, tau, r32);     \
        else launch_dyn(fast::k_fx_round<M, RW, false, false>, grid, T, sm, st, g, mask, sp, tau, r32);              \
    }
    switch (g.M) {
        HMG_FAST_LEN(32, FXR)
        HMG_FAST_LEN(48, FXR)
        HMG_FAST_LEN(64, FXR)
        HMG_FAST_LEN(96, FXR)
        HMG_FAST_LEN(128, FXR)
        default: return false;
    }
#undef FXR
}

#undef HMG_FAST_LEN

}  // namespace hmg
