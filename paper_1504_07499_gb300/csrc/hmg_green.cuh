// The Green operator of §3 applied per Fourier mode, and the per-mode term of the
// step-1 equilibrium norm, on the packed half spectrum (see hmg_kernels.cu for the
// layout).  Gamma0 = -P/k0 with P = xi xi^T / |xi|^2, so the tau-form sweep needs
// (I - 2P) s (the basic scheme, with a positive reference medium, needs -P s); the
// Nyquist rule decides xi at Nyquist components.
#pragma once

#include <cuda_runtime.h>

#include "hmg_internal.h"

namespace hmg {

__device__ __forceinline__ int signed_mode(int k, int N) { return k <= N / 2 ? k : k - N; }

// Direction m' of the projector at mode (kx >= 0, my, mz) (signed modes): Nyquist
// components are dropped unless they are the only nonzero component.  Returns |m'|^2
// (0 where P = 0: at DC and at modes made only of two or three Nyquist components).
__device__ __forceinline__ int mode_dir(int kx, int my, int mz, int N, int* d) {
    const int h = N / 2;
    const int nonzero = (kx != 0) + (my != 0) + (mz != 0);
    d[0] = (kx == h && nonzero > 1) ? 0 : kx;
    d[1] = (my == h && nonzero > 1) ? 0 : my;
    d[2] = (mz == h && nonzero > 1) ? 0 : mz;
    return d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
}

// a <- ga a - gb P a on the real mode (kx, my, mz) (P = 0 where the direction vanishes).
template <typename R>
__device__ __forceinline__ void reflect_real(R* a, int kx, int my, int mz, int N, R ga, R gb) {
    int d[3];
    const int n2 = mode_dir(kx, my, mz, N, d);
    if (n2 > 0) {
        const R f = gb / R(n2);
        const R dot = R(d[0]) * a[0] + R(d[1]) * a[1] + R(d[2]) * a[2];
        a[0] = ga * a[0] - f * R(d[0]) * dot;
        a[1] = ga * a[1] - f * R(d[1]) * dot;
        a[2] = ga * a[2] - f * R(d[2]) * dot;
    } else {
        a[0] *= ga;
        a[1] *= ga;
        a[2] *= ga;
    }
}

// s <- scale (ga s - gb P s) at packed mode (kx, ky, kz); at the DC of the kx = 0 plane
// add gc E (cE, when add_b).  kx in [0, N/2), ky, kz in [0, N).  Eyre-Milton's
// reflection (I - 2P) is ga = 1, gb = 2; the basic scheme's -P is ga = 0, gb = 1.
template <typename R, typename T2>
__device__ __forceinline__ void green_mode(int kx, int ky, int kz, int N, R scale, R ga, R gb, bool add_b,
                                           const R* cE, T2& s0, T2& s1, T2& s2) {
    const int my = signed_mode(ky, N), mz = signed_mode(kz, N);
    const bool special = (kx == 0) && (ky == 0 || ky == N / 2) && (kz == 0 || kz == N / 2);
    if (!special) {
        int d[3];
        const int n2 = mode_dir(kx, my, mz, N, d);   // > 0 at every non-special mode
        const R f = gb / R(n2);
        const R dx = R(d[0]) * s0.x + R(d[1]) * s1.x + R(d[2]) * s2.x;
        const R dy = R(d[0]) * s0.y + R(d[1]) * s1.y + R(d[2]) * s2.y;
        s0.x = scale * (ga * s0.x - f * R(d[0]) * dx);
        s0.y = scale * (ga * s0.y - f * R(d[0]) * dy);
        s1.x = scale * (ga * s1.x - f * R(d[1]) * dx);
        s1.y = scale * (ga * s1.y - f * R(d[1]) * dy);
        s2.x = scale * (ga * s2.x - f * R(d[2]) * dx);
        s2.y = scale * (ga * s2.y - f * R(d[2]) * dy);
    } else {
        R a[3] = {s0.x, s1.x, s2.x};   // plane kx = 0
        R b[3] = {s0.y, s1.y, s2.y};   // plane kx = N/2
        reflect_real(a, 0, my, mz, N, ga, gb);
        reflect_real(b, N / 2, my, mz, N, ga, gb);
        for (int c = 0; c < 3; ++c) {
            a[c] *= scale;
            b[c] *= scale;
        }
        if (add_b && ky == 0 && kz == 0)
            for (int c = 0; c < 3; ++c) a[c] += cE[c];
        s0.x = a[0];
        s0.y = b[0];
        s1.x = a[1];
        s1.y = b[1];
        s2.x = a[2];
        s2.y = b[2];
    }
}

// FP32 Green step of the register-resident z kernels: the same map as green_mode, with the
// projector factor gb / |m'|^2 from the fast reciprocal (__fdividef, error within 2 ulp)
// and the updates as packed two-lane FP32 operations on (real, imaginary) pairs:
// s_c <- scale ga s_c - (scale gb d_c / |m'|^2) (m' . s).  The four self-conjugate modes of
// the packed kx = 0 column (and the DC with its gc E) go through green_mode.
__device__ __forceinline__ void green_mode_fast(int kx, int ky, int kz, int N, float scale, float ga, float gb,
                                                bool add_b, const float* cE, float2& s0, float2& s1, float2& s2) {
    const bool special = (kx == 0) && (ky == 0 || ky == N / 2) && (kz == 0 || kz == N / 2);
    if (special) {
        green_mode<float>(kx, ky, kz, N, scale, ga, gb, add_b, cE, s0, s1, s2);
        return;
    }
    int d[3];
    const int n2 = mode_dir(kx, signed_mode(ky, N), signed_mode(kz, N), N, d);   // > 0 off the special modes
    const float gs = scale * __fdividef(gb, (float)n2);
    const float d0 = (float)d[0], d1 = (float)d[1], d2 = (float)d[2];
    const float2 dot = __ffma2_rn(make_float2(d2, d2), s2,
                                  __ffma2_rn(make_float2(d1, d1), s1, __fmul2_rn(make_float2(d0, d0), s0)));
    const float sa = scale * ga;
    const float2 sc = make_float2(sa, sa);
    const float q0 = -gs * d0, q1 = -gs * d1, q2 = -gs * d2;
    s0 = __ffma2_rn(make_float2(q0, q0), dot, __fmul2_rn(sc, s0));
    s1 = __ffma2_rn(make_float2(q1, q1), dot, __fmul2_rn(sc, s1));
    s2 = __ffma2_rn(make_float2(q2, q2), dot, __fmul2_rn(sc, s2));
}

// Weighted |m' . s|^2 of packed mode (kx, ky, kz) for the equilibrium norm (integer
// m'; the caller scales by (2 pi / N)^2 / N^6).  Modes 0 < kx < N/2 stand for kx and
// N - kx (weight 2); the kx = 0 column holds the kx = 0 and kx = N/2 planes, whose
// cross terms cancel over +-k except at the four self-conjugate modes, split here.
template <typename T2>
__device__ __forceinline__ double eq_mode(int kx, int ky, int kz, int N, const T2& s0, const T2& s1, const T2& s2) {
    const int my = signed_mode(ky, N), mz = signed_mode(kz, N);
    const bool special = (kx == 0) && (ky == 0 || ky == N / 2) && (kz == 0 || kz == N / 2);
    int d[3];
    if (!special) {
        if (mode_dir(kx, my, mz, N, d) == 0) return 0.0;
        const double dr = d[0] * (double)s0.x + d[1] * (double)s1.x + d[2] * (double)s2.x;
        const double di = d[0] * (double)s0.y + d[1] * (double)s1.y + d[2] * (double)s2.y;
        return (kx == 0 ? 1.0 : 2.0) * (dr * dr + di * di);
    }
    double acc = 0.0;
    if (mode_dir(0, my, mz, N, d) > 0) {
        const double dr = d[0] * (double)s0.x + d[1] * (double)s1.x + d[2] * (double)s2.x;
        acc += dr * dr;
    }
    if (mode_dir(N / 2, my, mz, N, d) > 0) {
        const double di = d[0] * (double)s0.y + d[1] * (double)s1.y + d[2] * (double)s2.y;
        acc += di * di;
    }
    return acc;
}

}  // namespace hmg
