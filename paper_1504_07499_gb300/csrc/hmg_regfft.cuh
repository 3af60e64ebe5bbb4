// Register-resident FFT building blocks (FP32) shared by the pass kernels.
//
// A 1D transform of length L = E * TP runs as two register stages (the four-step
// factorization; n = TP n1 + n2, k = k1 + E k2):
//   stage 1: thread n2 holds x[TP n1 + n2] (n1 < E), computes the length-E DFT over n1
//            in registers and multiplies by w_L^(n2 k1);
//   exchange through shared memory (one write, one read);
//   stage 2: thread t holds, for its E/TP values of k1, all TP values of n2 and
//            computes length-TP DFTs, giving X[k1 + E k2] in registers.
// X(k1 + E k2) = sum_n1 w_E^(n1 k1) w_L^(n2 k1) sum_n2 ... is the textbook split of the
// DFT sum; the inverse runs the same stages with conjugate factors, or in reverse order
// when it starts from stage-2 registers.
#pragma once

#include <cuda_runtime.h>

#include "hmg_fft.cuh"
#include "hmg_internal.h"

namespace hmg {
namespace fast {

// cos(2 pi i / 96) for i = 0..24 (first quadrant), from the power series.
__host__ __device__ constexpr double cos96_q(int i) {
    return i == 0 ? 1.0 : i == 1 ? 0.9978589232386035 : i == 2 ? 0.9914448613738104 : i == 3 ? 0.9807852804032304
         : i == 4 ? 0.9659258262890683 : i == 5 ? 0.9469301294951057 : i == 6 ? 0.9238795325112867
         : i == 7 ? 0.8968727415326883 : i == 8 ? 0.8660254037844386 : i == 9 ? 0.8314696123025452
         : i == 10 ? 0.7933533402912352 : i == 11 ? 0.7518398074789774 : i == 12 ? 0.7071067811865476
         : i == 13 ? 0.6593458151000688 : i == 14 ? 0.6087614290087207 : i == 15 ? 0.5555702330196022
         : i == 16 ? 0.5 : i == 17 ? 0.4422886902190013 : i == 18 ? 0.3826834323650898
         : i == 19 ? 0.3214394653031616 : i == 20 ? 0.25881904510252074 : i == 21 ? 0.19509032201612828
         : i == 22 ? 0.1305261922200516 : i == 23 ? 0.06540312923014306 : 0.0;
}
__host__ __device__ constexpr double cos96(int i) {
    return (i = ((i % 96) + 96) % 96, i <= 24 ? cos96_q(i) : i <= 48 ? -cos96_q(48 - i)
                                                    : i <= 72 ? -cos96_q(i - 48) : cos96_q(96 - i));
}
// w_E^m = exp(-2 pi i m / E) (forward) or its conjugate, for E dividing 96.
template <int E, bool FWD>
__device__ __forceinline__ float2 wE(int m) {
    const float c = (float)cos96(m * (96 / E));
    const float s = (float)cos96(m * (96 / E) - 24);   // sin(2 pi i / 96)
    return FWD ? make_float2(c, -s) : make_float2(c, s);
}

// x * w_E^m with the quarter turns (w = -1, +-i) done exactly by swaps and signs.
template <int E, bool FWD>
__device__ __forceinline__ float2 twiddle_E(float2 x, int m) {
    const int q = (m * 4) % E == 0 ? (m * 4 / E) % 4 : -1;   // m a multiple of E/4: quarter turns
    if (q == 0) return x;
    if (q == 2) return make_float2(-x.x, -x.y);
    if (q == 1) return FWD ? make_float2(x.y, -x.x) : make_float2(-x.y, x.x);   // w = -i (forward)
    if (q == 3) return FWD ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
    return cmul(x, wE<E, FWD>(m));
}

// Length-E DFT in registers, natural order in and out.
template <int E, bool FWD>
struct RegDFT {
    static constexpr int A = (E % 4 == 0) ? 4 : ((E % 2 == 0) ? 2 : 3);
    static constexpr int B = E / A;
    __device__ __forceinline__ static void run(float2* v) {
        float2 s[A][B];
#pragma unroll
        for (int a = 0; a < A; ++a)
#pragma unroll
            for (int j = 0; j < B; ++j) s[a][j] = v[A * j + a];
#pragma unroll
        for (int a = 0; a < A; ++a) RegDFT<B, FWD>::run(s[a]);
#pragma unroll
        for (int a = 1; a < A; ++a)
#pragma unroll
            for (int k = 1; k < B; ++k) s[a][k] = twiddle_E<E, FWD>(s[a][k], a * k);
#pragma unroll
        for (int k = 0; k < B; ++k) {
            float2 t[A];
#pragma unroll
            for (int a = 0; a < A; ++a) t[a] = s[a][k];
            RegDFT<A, FWD>::run(t);
#pragma unroll
            for (int q = 0; q < A; ++q) v[k + B * q] = t[q];
        }
    }
};
template <bool FWD> struct RegDFT<1, FWD> { __device__ __forceinline__ static void run(float2*) {} };
template <bool FWD> struct RegDFT<2, FWD> { __device__ __forceinline__ static void run(float2* v) { bfly2<FWD>(v); } };
template <bool FWD> struct RegDFT<3, FWD> { __device__ __forceinline__ static void run(float2* v) { bfly3<FWD>(v); } };
template <bool FWD> struct RegDFT<4, FWD> { __device__ __forceinline__ static void run(float2* v) { bfly4<FWD>(v); } };
template <bool FWD> struct RegDFT<8, FWD> { __device__ __forceinline__ static void run(float2* v) { bfly8<FWD>(v); } };

// Split of a length into E * TP with TP^2 dividing L (so each stage-2 thread owns
// E/TP whole length-TP transforms).
template <int L> struct Split;
template <> struct Split<16> { static constexpr int TP = 4, E = 4; };
template <> struct Split<32> { static constexpr int TP = 4, E = 8; };
template <> struct Split<48> { static constexpr int TP = 4, E = 12; };
template <> struct Split<64> { static constexpr int TP = 8, E = 8; };
template <> struct Split<96> { static constexpr int TP = 4, E = 24; };
template <> struct Split<128> { static constexpr int TP = 8, E = 16; };
template <> struct Split<192> { static constexpr int TP = 8, E = 24; };
template <> struct Split<256> { static constexpr int TP = 16, E = 16; };
template <> struct Split<512> { static constexpr int TP = 16, E = 32; };

// Shared-memory slot of (k1, n2) of one pencil: k1-major with one pad row per group of
// E/TP k1 values, so that stage-2 readers of different groups fall on different banks.
template <int L>
__device__ __forceinline__ int xslot(int k1, int n2) {
    constexpr int TP = Split<L>::TP, KPT = Split<L>::E / TP;
    return k1 * TP + n2 + (k1 / KPT);
}
template <int L> constexpr int xslots() { return L + Split<L>::E / (Split<L>::E / Split<L>::TP); }

// Twiddle load from the read-only global path, or from a table staged in shared memory
// (TWS): per-thread twiddle indices spread a warp's global loads over many L1 sectors,
// while the shared-memory table serves them in one or two wavefronts.
template <bool TWS>
__device__ __forceinline__ float2 twld(const float2* tw, int i) {
    if constexpr (TWS) return tw[i];
    else return __ldg(&tw[i]);
}

// stage 1 (+ twiddle) and the write half of the exchange
template <int L, bool FWD, bool TWS = false>
__device__ __forceinline__ void stage1_write(float2* v, int n2, const float2* __restrict__ twL, float2* sh, int pstride) {
    constexpr int E = Split<L>::E;
    RegDFT<E, FWD>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < E; ++k1) {
        const float2 w = twld<TWS>(twL, (n2 * k1) % L);
        v[k1] = FWD ? cmul(v[k1], w) : cmulc(v[k1], w);
    }
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) sh[xslot<L>(k1, n2) * pstride] = v[k1];
}

// read half of the exchange and stage 2: v[i * TP + k2] = X[(t KPT + i) + E k2]
template <int L, bool FWD>
__device__ __forceinline__ void stage2_read(float2* v, int t, const float2* sh, int pstride) {
    constexpr int E = Split<L>::E, TP = Split<L>::TP, KPT = E / TP;
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
        const int k1 = t * KPT + i;
#pragma unroll
        for (int n2 = 0; n2 < TP; ++n2) v[i * TP + n2] = sh[xslot<L>(k1, n2) * pstride];
        RegDFT<TP, FWD>::run(v + i * TP);
    }
}

// A transform that starts from the stage-2 layout, v[i * TP + m] = x[(t KPT + i) + E m]
// (the layout stage 2 leaves), runs the two stages in reverse order: length-TP DFTs over m
// in registers, twiddles w_L^(+-(t KPT + i) k_a), the exchange, and length-E DFTs, giving
// X[n2 + TP k_b] in v[k_b] of thread n2 (decimation in frequency:
// X(k_a + TP k_b) = sum_p w_E^(p k_b) w_L^(p k_a) sum_m w_TP^(m k_a) x[p + E m]).
// The inverse (FWD = false) undoes stage 2 then stage 1 of a forward transform.
template <int L, bool FWD = false, bool TWS = false>
__device__ __forceinline__ void rstage2_write(float2* v, int t, const float2* __restrict__ twL, float2* sh, int pstride) {
    constexpr int E = Split<L>::E, TP = Split<L>::TP, KPT = E / TP;
#pragma unroll
    for (int i = 0; i < KPT; ++i) {
        const int k1 = t * KPT + i;
        RegDFT<TP, FWD>::run(v + i * TP);
#pragma unroll
        for (int n2 = 0; n2 < TP; ++n2) {
            float2 x = v[i * TP + n2];
            if (n2 > 0 && k1 > 0) {
                const float2 w = twld<TWS>(twL, (n2 * k1) % L);
                x = FWD ? cmul(x, w) : cmulc(x, w);
            }
            sh[xslot<L>(k1, n2) * pstride] = x;
        }
    }
}

// read half of the reverse exchange and the length-E DFT: v[k_b] = X[n2 + TP k_b]
// (inverse: v[n1] = x[TP n1 + n2])
template <int L, bool FWD = false>
__device__ __forceinline__ void rstage1_read(float2* v, int n2, const float2* sh, int pstride) {
    constexpr int E = Split<L>::E;
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) v[k1] = sh[xslot<L>(k1, n2) * pstride];
    RegDFT<E, FWD>::run(v);
}

__device__ __forceinline__ float sel3f(int ph, float a, float b, float c) { return ph == 0 ? a : (ph == 1 ? b : c); }

static __device__ double block_sum_d(double v, double* sh) {
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

template <int M> constexpr int row_stride() {
    // slots per row, padded to an odd multiple of 8 complex values (64 B) so that
    // rows of a warp start on alternating bank halves
    return ((xslots<M>() + 15) / 16) * 16 + 8;
}

// Fixed-order CTA sum for any block size (multiple of 32); result valid in thread 0.
static __device__ double block_sum_any(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
    __syncthreads();
    return r;
}

// Variant 0: one thread holds all three components of its (column, pencil part):
// the Green operator runs entirely in registers (high register count, low occupancy).
}  // namespace fast
}  // namespace hmg
