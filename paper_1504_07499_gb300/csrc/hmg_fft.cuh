// Shared-memory mixed-radix Stockham FFT used by every pass of the 3D transform.
//
// A CTA holds `npen` pencils of length L in shared memory; element i of pencil p sits
// at p*ps + i*is.  Each stage of radix R with sub-length Ns (product of the previous
// radices) maps butterfly j in [0, L/R) of every pencil:
//   v_r = src[j + r L/R],  v_r *= w_L^(r (j mod Ns) L/(Ns R))  (r >= 1),
//   v = DFT_R(v),          dst[(j div Ns) Ns R + (j mod Ns) + r Ns] = v_r,
// the self-sorting (autosort) formulation of the Stockham algorithm, so the result
// leaves the last stage in natural order.  Buffers alternate between stages.
// Twiddles come from a host-built table w_L^k = exp(-2 pi i k / L); the inverse
// transform uses their conjugates and the conjugate butterflies (no scaling).
#pragma once

#include <cuda_runtime.h>
#include "hmg_internal.h"

namespace hmg {

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T2> __device__ __forceinline__ T2 cmulc(T2 a, T2 b) {
    return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T2> __device__ __forceinline__ T2 cconj(T2 a) { return mk(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
template <bool FWD, typename T2> __device__ __forceinline__ T2 mul_mi(T2 a) {
    return FWD ? mk(a.y, -a.x) : mk(-a.y, a.x);
}

// FP32 complex adds and subtracts as single packed two-lane FP32 instructions (sm_100
// and later); a - b is b * (-1) + a, exact product, one rounding, as the scalar form.
// Overloads of the templates above, chosen for float2.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

template <typename T2> struct TwTable;
template <> struct TwTable<float2> {
    static __device__ __forceinline__ const float2* get(const GridDesc& g) { return g.tw32; }
};
template <> struct TwTable<double2> {
    static __device__ __forceinline__ const double2* get(const GridDesc& g) { return g.tw64; }
};

// Radix-R DFT in registers, forward sign exp(-2 pi i/R) or its conjugate.
template <bool FWD, typename T2> __device__ __forceinline__ void bfly2(T2* v) {
    T2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <bool FWD, typename T2> __device__ __forceinline__ void bfly4(T2* v) {
    T2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    T2 t2 = cadd(v[1], v[3]), t3 = mul_mi<FWD>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
}

template <bool FWD, typename T2> __device__ __forceinline__ void bfly3(T2* v) {
    using S = decltype(v[0].x);
    const S h = S(0.86602540378443864676);  // sin(2 pi / 3)
    T2 t = cadd(v[1], v[2]);
    T2 u = csub(v[1], v[2]);
    T2 m = mk(v[0].x - S(0.5) * t.x, v[0].y - S(0.5) * t.y);
    // forward: X1 = m - i h u, X2 = m + i h u
    T2 iu = mul_mi<FWD>(u);  // -i u (forward) / +i u (inverse)
    v[0] = cadd(v[0], t);
    v[1] = mk(m.x + h * iu.x, m.y + h * iu.y);
    v[2] = mk(m.x - h * iu.x, m.y - h * iu.y);
}

template <bool FWD, typename T2> __device__ __forceinline__ void bfly8(T2* v) {
    using S = decltype(v[0].x);
    const S c = S(0.70710678118654752440);  // cos(pi/4)
    T2 a[4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        a[r] = cadd(v[r], v[r + 4]);
        b[r] = csub(v[r], v[r + 4]);
    }
    // b_r *= w8^r, w8 = exp(-i pi/4) forward
    b[1] = FWD ? mk(c * (b[1].x + b[1].y), c * (b[1].y - b[1].x))
               : mk(c * (b[1].x - b[1].y), c * (b[1].y + b[1].x));
    b[2] = mul_mi<FWD>(b[2]);
    b[3] = FWD ? mk(c * (b[3].y - b[3].x), -c * (b[3].x + b[3].y))
               : mk(-c * (b[3].x + b[3].y), c * (b[3].x - b[3].y));
    bfly4<FWD>(a);
    bfly4<FWD>(b);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        v[2 * r] = a[r];
        v[2 * r + 1] = b[r];
    }
}

template <int RAD, bool FWD, typename T2>
__device__ __forceinline__ void stockham_stage(const T2* __restrict__ src, T2* __restrict__ dst,
                                               int L, int Ns, int npen, int ps, int is,
                                               const T2* __restrict__ tw) {
    const int Lr = L / RAD;
    const int total = npen * Lr;
    const int tstep = L / (Ns * RAD);
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        int p, j;
        if (is == 1) {
            p = q / Lr;
            j = q - p * Lr;
        } else {
            j = q / npen;
            p = q - j * npen;
        }
        const T2* s = src + (long)p * ps;
        T2 v[RAD];
#pragma unroll
        for (int r = 0; r < RAD; ++r) v[r] = s[(j + r * Lr) * is];
        const int k = j % Ns;
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < RAD; ++r) {
                T2 w = __ldg(&tw[k * r * tstep]);
                v[r] = FWD ? cmul(v[r], w) : cmulc(v[r], w);
            }
        }
        if (RAD == 2) bfly2<FWD>(v);
        if (RAD == 3) bfly3<FWD>(v);
        if (RAD == 4) bfly4<FWD>(v);
        if (RAD == 8) bfly8<FWD>(v);
        T2* d = dst + (long)p * ps;
        const int base = (j / Ns) * Ns * RAD + k;
#pragma unroll
        for (int r = 0; r < RAD; ++r) d[(base + r * Ns) * is] = v[r];
    }
}

// Full 1D transform of `npen` pencils; returns the buffer that holds the result.
// Must be called by all threads of the CTA (contains __syncthreads).
template <bool FWD, typename T2>
__device__ T2* fft_smem(T2* b0, T2* b1, const FftPlan& pl, const T2* __restrict__ twbase,
                        int npen, int ps, int is) {
    const T2* tw = twbase + pl.tw_off;
    int Ns = 1;
    for (int s = 0; s < pl.nst; ++s) {
        const int R = pl.rad[s];
        if (R == 8) stockham_stage<8, FWD>(b0, b1, pl.L, Ns, npen, ps, is, tw);
        else if (R == 4) stockham_stage<4, FWD>(b0, b1, pl.L, Ns, npen, ps, is, tw);
        else if (R == 3) stockham_stage<3, FWD>(b0, b1, pl.L, Ns, npen, ps, is, tw);
        else stockham_stage<2, FWD>(b0, b1, pl.L, Ns, npen, ps, is, tw);
        Ns *= R;
        __syncthreads();
        T2* t = b0;
        b0 = b1;
        b1 = t;
    }
    return b0;
}

}  // namespace hmg
