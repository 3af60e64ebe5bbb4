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
// Within a block of FP32 sweeps the x inverse of one sweep and the x forward of the next
// are one kernel (k_fx_round); the y and z passes are the same in every sweep.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <algorithm>

#include "hmg_async.cuh"
#include "hmg_fft.cuh"
#include "hmg_green.cuh"
#include "hmg_internal.h"
#include "hmg_regfft.cuh"

namespace hmg {
namespace fast {

// Set by a persistent kernel whose bounded wait for a bulk copy gave up (read and
// cleared by fast_take_wait_failure).
__device__ unsigned g_wait_fail;

// ---------------------------------------------------------------------------
// y pass: P consecutive kx columns of one (component, z) plane; threads (p, t)
// ---------------------------------------------------------------------------

// CTAs per SM the register bound of a pass kernel aims at: long columns (32 values per
// thread) get more registers
template <int L, int base>
constexpr int col_min_ctas() { return Split<L>::E > 24 ? base - 1 : base; }

template <int L, int P, bool FWD>
__global__ void __launch_bounds__(P * Split<L>::TP, col_min_ctas<L, 3>())
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
    const float cE[3] = {(float)(g.gc * g.E[slot][0]), (float)(g.gc * g.E[slot][1]), (float)(g.gc * g.E[slot][2])};
    const float ga = (float)g.ga, gb = (float)g.gb;
#pragma unroll
    for (int i = 0; i < KPT; ++i)
#pragma unroll
        for (int k2 = 0; k2 < TP; ++k2)
            green_mode_fast(kx, ky, t * KPT + i + E * k2, N, scale, ga, gb, addb, cE, v[0][i * TP + k2],
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

// Variant 0 as a persistent kernel: each CTA walks the (slot, ky, column block) items in
// a fixed stride over the grid; while one item is transformed, the bulk-copy engine
// stages the next item's three component columns (a tiled tensor copy each: P kx by all
// kz at one ky) in shared memory, so HBM reads overlap the arithmetic.  Plain and
// correction sweeps only (Z_ITER, Z_ITER_NOB); same float operations as k_fz3.
// The three components' exchanges go through one component-sized buffer in turn (a third
// of the shared memory of k_fz3's exchange, so three CTAs fit on an SM beside the staging).
template <int L, int P>
struct ZSmem {
    static constexpr size_t stage_bytes = (size_t)3 * L * P * sizeof(float2);
    static constexpr size_t x_off = (stage_bytes + 127) / 128 * 128;
    static constexpr size_t total = x_off + (size_t)xslots<L>() * P * sizeof(float2);
};

template <int L, int P, int MODE>
__global__ void __launch_bounds__(P * Split<L>::TP, 3)
k_fz3_p(const __grid_constant__ CUtensorMap zmap, GridDesc g, unsigned mask, float2* __restrict__ spec, int nper) {
    constexpr int E = Split<L>::E, TP = Split<L>::TP, KPT = E / TP;
    constexpr int N = L, M = L / 2;
    constexpr long long NNM = (long long)N * N * M;
    constexpr long long rowz = (long long)N * M;     // stride between z rows
    using Z = ZSmem<L, P>;
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ int s_ok;
    const int p = threadIdx.x % P, t = threadIdx.x / P;
    const float2* stg = reinterpret_cast<const float2*>(dsm);   // [component][kz][column]
    float2* sh = reinterpret_cast<float2*>(dsm + Z::x_off) + p;  // one component at a time
    const int nkb = M / P;
    const int nitems = g.nslots * nper;
    int item = blockIdx.x;
    while (item < nitems && !slot_active(g, mask, item / nper)) item += gridDim.x;
    if (item >= nitems) return;
    const uint32_t mb = async::smem_addr(&mbar);
    if (threadIdx.x == 0) async::mbar_init(mb);
    auto issue = [&](int it) {   // thread 0: the three component columns of item `it`
        const int slot = it / nper, b = it % nper;
        async::mbar_expect(mb, (uint32_t)Z::stage_bytes);
        for (int c = 0; c < 3; ++c)
            async::tensor_g2s_4d(async::smem_addr(stg + c * L * P), &zmap, (b % nkb) * P, b / nkb, 0, slot * 3 + c, mb);
    };
    if (threadIdx.x == 0) issue(item);
    __syncthreads();
    const float2* twL = g.tw32 + g.pN.tw_off;
    const float scale = (float)(1.0 / (double)g.N3);
    const float ga = (float)g.ga, gb = (float)g.gb;
    uint32_t parity = 0;
    while (item < nitems) {
        const int slot = item / nper, b = item % nper;
        const int kb = b % nkb, ky = b / nkb;
        const int kx = kb * P + p;
        if (threadIdx.x == 0) s_ok = async::mbar_wait(mb, parity) ? 1 : 0;
        __syncthreads();
        if (!s_ok) {
            if (threadIdx.x == 0) atomicOr(&g_wait_fail, 1u);
            return;
        }
        async::mbar_wait(mb, parity);   // complete already: the copied bytes are visible here
        parity ^= 1u;
        float2 v[3][E];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int n1 = 0; n1 < E; ++n1) v[c][n1] = stg[(c * L + TP * n1 + t) * P + p];
        __syncthreads();   // every thread holds its columns: the staging takes the next item
        int nxt = item + gridDim.x;
        while (nxt < nitems && !slot_active(g, mask, nxt / nper)) nxt += gridDim.x;
        if (threadIdx.x == 0 && nxt < nitems) issue(nxt);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            stage1_write<L, true>(v[c], t, twL, sh, P);
            __syncthreads();
            stage2_read<L, true>(v[c], t, sh, P);
            __syncthreads();   // the buffer takes the next component
        }
        const bool addb = g.dflags ? (g.dflags[slot] & SF_ADDB) != 0 : MODE == Z_ITER;
        const float cE[3] = {(float)(g.gc * g.E[slot][0]), (float)(g.gc * g.E[slot][1]), (float)(g.gc * g.E[slot][2])};
#pragma unroll
        for (int i = 0; i < KPT; ++i)
#pragma unroll
            for (int k2 = 0; k2 < TP; ++k2)
                green_mode_fast(kx, ky, t * KPT + i + E * k2, N, scale, ga, gb, addb, cE, v[0][i * TP + k2],
                                v[1][i * TP + k2], v[2][i * TP + k2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rstage2_write<L>(v[c], t, twL, sh, P);
            __syncthreads();
            rstage1_read<L>(v[c], t, sh, P);
            __syncthreads();   // the buffer takes the next component
        }
        float2* base = spec + (long long)slot * 3 * NNM + (long long)ky * M + kb * P + p;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int n1 = 0; n1 < E; ++n1) base[c * NNM + (long long)(TP * n1 + t) * rowz] = v[c][n1];
        item = nxt;   // (the exchange buffer and s_ok are next written after CTA barriers)
    }
}

// Variant 1: three thread groups, one per component; the projection d . s is summed
// through shared memory (more threads, fewer registers per thread).
template <int L, int P, int MODE>
__global__ void __launch_bounds__(3 * P * Split<L>::TP, col_min_ctas<L, 2>())
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
    const float cE = (float)(g.gc * g.E[slot][c]);
    const float ga = (float)g.ga, gb = (float)g.gb;
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
            const float fA = nA > 0 ? __fdividef(gb, (float)nA) : 0.0f;
            const float fB = nB > 0 ? __fdividef(gb, (float)nB) : 0.0f;
            float2& x = v[i * TP + k2];
            x.x = scale * (ga * x.x - fA * (float)dA * dotA);
            x.y = scale * (ga * x.y - fB * (float)dB * dotB);
            if (addb && kx == 0 && ky == 0 && kz == 0) x.x += cE;
        }
    __syncthreads();   // every thread has read the shares
    rstage2_write<L>(v, t, twL, shc, P);
    __syncthreads();
    rstage1_read<L>(v, t, shc, P);
#pragma unroll
    for (int n1 = 0; n1 < E; ++n1) base[(long long)(TP * n1 + t) * rowz] = v[n1];
}

// ---------------------------------------------------------------------------
// x passes: RW rows per CTA (128 threads), threads (t, r) with t fastest along the row
// ---------------------------------------------------------------------------

// Coefficient pairs for two neighbouring voxels of phases (a, b): lut[a | b << 2] = (c_a, c_b).
__device__ __forceinline__ void coef_pairs(float2* lut, float c0, float c1, float c2) {
    if (threadIdx.x < 16) {
        const int a = threadIdx.x & 3, b = threadIdx.x >> 2;
        const float ca = a == 0 ? c0 : (a == 1 ? c1 : (a == 2 ? c2 : 0.f));
        const float cb = b == 0 ? c0 : (b == 1 ? c1 : (b == 2 ? c2 : 0.f));
        lut[threadIdx.x] = make_float2(ca, cb);
    }
}
__device__ __forceinline__ int pair_index(uchar2 q) { return q.x | (q.y << 2); }

// Stage the x pass twiddles in shared memory: tws[k] = w_M^k, tws[M + k] = w_N^k (k < M).
// The caller synchronizes the CTA before the first read.
template <int M>
__device__ __forceinline__ void stage_twiddles(float2* tws, const GridDesc& g) {
    const float2* twM = g.tw32 + g.pM.tw_off;
    const float2* twN = g.tw32 + g.pN.tw_off;
    for (int i = threadIdx.x; i < 2 * M; i += blockDim.x) tws[i] = i < M ? __ldg(&twM[i]) : __ldg(&twN[i - M]);
}

// Row values in the stage-2 layout: thread t holds complex position p = (t KPT + i) + E m
// at v[i TP + m].  With KPT even, positions t KPT + i (i even) are 16-byte aligned pairs,
// loaded and stored as float4 (and their phase ids as one uchar4).
template <int M>
__device__ __forceinline__ void s2_load(float2* v, const float2* __restrict__ row, int t) {
    constexpr int E = Split<M>::E, TP = Split<M>::TP, KPT = E / TP;
    if constexpr (KPT % 2 == 0) {
        const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
        for (int m = 0; m < TP; ++m)
#pragma unroll
            for (int i = 0; i < KPT; i += 2) {
                const float4 q = r4[(t * KPT + i + E * m) / 2];
                v[i * TP + m] = make_float2(q.x, q.y);
                v[(i + 1) * TP + m] = make_float2(q.z, q.w);
            }
    } else {
#pragma unroll
        for (int m = 0; m < TP; ++m)
#pragma unroll
            for (int i = 0; i < KPT; ++i) v[i * TP + m] = row[t * KPT + i + E * m];
    }
}
template <int M>
__device__ __forceinline__ void s2_store(float2* __restrict__ row, const float2* v, int t) {
    constexpr int E = Split<M>::E, TP = Split<M>::TP, KPT = E / TP;
    if constexpr (KPT % 2 == 0) {
        float4* r4 = reinterpret_cast<float4*>(row);
#pragma unroll
        for (int m = 0; m < TP; ++m)
#pragma unroll
            for (int i = 0; i < KPT; i += 2) {
                const float2 a = v[i * TP + m], b = v[(i + 1) * TP + m];
                r4[(t * KPT + i + E * m) / 2] = make_float4(a.x, a.y, b.x, b.y);
            }
    } else {
#pragma unroll
        for (int m = 0; m < TP; ++m)
#pragma unroll
            for (int i = 0; i < KPT; ++i) row[t * KPT + i + E * m] = v[i * TP + m];
    }
}
template <int M>
__device__ __forceinline__ void s2_load_phase(uchar2* q, const uchar2* __restrict__ row, int t) {
    constexpr int E = Split<M>::E, TP = Split<M>::TP, KPT = E / TP;
    if constexpr (KPT % 2 == 0) {
        const uchar4* r4 = reinterpret_cast<const uchar4*>(row);
#pragma unroll
        for (int m = 0; m < TP; ++m)
#pragma unroll
            for (int i = 0; i < KPT; i += 2) {
                const uchar4 b = r4[(t * KPT + i + E * m) / 2];
                q[i * TP + m] = make_uchar2(b.x, b.y);
                q[(i + 1) * TP + m] = make_uchar2(b.z, b.w);
            }
    } else {
#pragma unroll
        for (int m = 0; m < TP; ++m)
#pragma unroll
            for (int i = 0; i < KPT; ++i) q[i * TP + m] = row[t * KPT + i + E * m];
    }
}

// Lane of the same row holding the partner position M - k: a row's TP threads are TP
// consecutive lanes; thread t's values at k = t + TP j pair with thread (TP - t) mod TP.
template <int TP>
__device__ __forceinline__ int partner_lane(int t) {
    return (int)(threadIdx.x & 31u & ~(unsigned)(TP - 1)) | ((TP - t) & (TP - 1));
}
__device__ __forceinline__ float2 shfl2(float2 a, int lane) {
    return make_float2(__shfl_sync(0xffffffffu, a.x, lane), __shfl_sync(0xffffffffu, a.y, lane));
}

// Real split of a row transform held as v[kb] = Z[t + TP kb] (natural positions spread over
// the row's lanes), written to dst: X[k] = e + o w_N^k with e = (Z[k] + conj Z[M-k]) / 2,
// o = -i (Z[k] - conj Z[M-k]) / 2; X[0] packs X(0) and X(N/2).  Z[M - k] comes from the
// partner lane (v[E - 1 - kb]) or, for t = 0, from the thread itself (v[E - kb]).
// twN: w_N^k, k < M, staged in shared memory.
template <int M, int TP, int E>
__device__ __forceinline__ void r2c_split_shfl(const float2* v, int t, const float2* twN, float2* __restrict__ dst) {
    const int pl = partner_lane<TP>(t);
#pragma unroll
    for (int kb = 0; kb < E; ++kb) {
        const int k = t + TP * kb;
        const float2 z = v[kb];
        float2 zm = shfl2(v[E - 1 - kb], pl);
        if (kb > 0 && t == 0) zm = v[E - kb];
        float2 out;
        if (k == 0) {
            out = make_float2(z.x + z.y, z.x - z.y);
        } else {
            const float2 e = make_float2(0.5f * (z.x + zm.x), 0.5f * (z.y - zm.y));
            const float2 o = make_float2(0.5f * (z.y + zm.y), -0.5f * (z.x - zm.x));
            out = cadd(e, cmul(o, twN[k]));
        }
        dst[k] = out;
    }
}

// A row's TP threads are TP consecutive lanes of one warp and its exchange buffer is its
// own, so the exchanges of an x row transform synchronize the warp, not the CTA.
template <int TP>
__device__ __forceinline__ void row_sync() {
    static_assert(TP <= 32 && 32 % TP == 0, "a row's threads must lie in one warp");
    __syncwarp();
}

// Forward x transform of a row held in the stage-2 layout, ending with the real split
// written to dst: decimation-in-frequency stages (one shared-memory exchange), the split
// with the partner values exchanged by warp shuffles.  Ends without a barrier.
template <int M, int TP, int E>
__device__ __forceinline__ void row_forward_split(float2* v, int t, float2* rs, const float2* __restrict__ twM,
                                                  const float2* __restrict__ twN, float2* __restrict__ dst) {
    rstage2_write<M, true, true>(v, t, twM, rs, 1);
    row_sync<TP>();
    rstage1_read<M, true>(v, t, rs, 1);   // v[kb] = Z[t + TP kb]
    r2c_split_shfl<M, TP, E>(v, t, twN, dst);
}

template <int M, int RW, int MODE>
__global__ void __launch_bounds__(RW * Split<M>::TP, 1024 / (RW * Split<M>::TP))
k_fx_forward(GridDesc g, unsigned mask, const float* __restrict__ tau, float2* __restrict__ spec,
             double* __restrict__ partial) {
    constexpr int E = Split<M>::E, TP = Split<M>::TP, RS = row_stride<M>();
    const int slot = blockIdx.y;
    if (!slot_active(g, mask, slot)) return;
    extern __shared__ __align__(16) float2 sh[];   // RW * RS
    __shared__ double red[RW * TP];
    __shared__ float2 lut[16];
    const int N = g.N;
    const int t = threadIdx.x % TP, r = threadIdx.x / TP;
    // component fastest across CTAs, so the three components of a (z, y) block read the
    // same phase rows close together in time (L2 hits)
    const int comp = blockIdx.x % 3;
    const long long rblk = blockIdx.x / 3;
    const long long row = comp * g.NN + rblk * RW + r;              // c*NN + z*N + y
    const long long pidx = comp * (g.NN / RW) + rblk;               // component-major CTA index
    const float2* src = reinterpret_cast<const float2*>(tau + (long long)slot * 3 * g.N3 + row * N);
    __shared__ float2 tws[2 * M];
    stage_twiddles<M>(tws, g);
    if (MODE != XF_PLAIN)
        coef_pairs(lut, (float)(MODE == XF_POLARIZE ? g.Y[0] : g.W[0]), (float)(MODE == XF_POLARIZE ? g.Y[1] : g.W[1]),
                   (float)(MODE == XF_POLARIZE ? g.Y[2] : g.W[2]));
    __syncthreads();
    float2 v[E];
    s2_load<M>(v, src, t);
    float acc = 0.f;
    if (MODE != XF_PLAIN) {
        uchar2 q[E];
        s2_load_phase<M>(q, reinterpret_cast<const uchar2*>(g.phase + (row % g.NN) * N), t);
#pragma unroll
        for (int j = 0; j < E; ++j) {
            // rounded products (never contracted into the transform's adds), as in k_fx_round
            v[j] = __fmul2_rn(v[j], lut[pair_index(q[j])]);
            if (MODE == XF_FLUX) acc += v[j].x + v[j].y;
        }
    }
    if (MODE == XF_FLUX) {
        const double s = block_sum_d((double)acc, red);
        if (threadIdx.x == 0) partial[(long long)slot * gridDim.x + pidx] = s;
    }
    row_forward_split<M, TP, E>(v, t, sh + r * RS, tws, tws + M, spec + (long long)slot * 3 * g.NNM + row * M);
}

// Complex-to-real merge with the row spectrum loaded straight into the stage-1 layout
// (xk[n1] = X[TP n1 + t]); X[M - k] comes from the partner lane (xk[E - 1 - n1]) or, for
// t = 0, from the thread itself (xk[E - n1]): v[n1] = (X[k] + conj X[M-k]) + i w_N^-k
// (X[k] - conj X[M-k]), the x-transform input at k.  twN: w_N^k in shared memory.
template <int M, int TP, int E>
__device__ __forceinline__ void c2r_merge_shfl(float2* v, const float2* xk, const float2* twN, int t) {
    const int pl = partner_lane<TP>(t);
#pragma unroll
    for (int n1 = 0; n1 < E; ++n1) {
        const int k = TP * n1 + t;
        float2 a = xk[n1];
        float2 b = shfl2(xk[E - 1 - n1], pl);
        if (n1 > 0 && t == 0) b = xk[E - n1];
        if (k == 0) {   // packed X(0) + i X(N/2)
            b = make_float2(a.y, 0.f);
            a = make_float2(a.x, 0.f);
        }
        const float2 s = make_float2(a.x + b.x, a.y - b.y);
        const float2 d = make_float2(a.x - b.x, a.y + b.y);
        const float2 dw = cmulc(d, twN[k]);
        v[n1] = make_float2(s.x - dw.y, s.y + dw.x);
    }
}

// Inverse x transform of a row spectrum: load into registers, merge (warp shuffles),
// stage 1, exchange, stage 2; leaves v in the stage-2 layout (v[i TP + m] =
// x[(t KPT + i) + E m]).  The caller has synchronized the CTA after staging twN / twM.
template <int M, int TP, int E>
__device__ __forceinline__ void row_inverse(float2* v, int t, float2* rs, const float2* __restrict__ src,
                                            const float2* __restrict__ twM, const float2* __restrict__ twN) {
    float2 xk[E];
#pragma unroll
    for (int n1 = 0; n1 < E; ++n1) xk[n1] = src[TP * n1 + t];
    c2r_merge_shfl<M, TP, E>(v, xk, twN, t);
    stage1_write<M, false, true>(v, t, twM, rs, 1);
    row_sync<TP>();
    stage2_read<M, false>(v, t, rs, 1);
}

// threads per SM the register bound aims at: residual sweeps hold the old row (and r) in
// registers beside the transform
template <int M, int MODE>
constexpr int fx_inverse_min_threads() {
    return (MODE == XI_ADD_R_RES || MODE == XI_INPLACE_RES || Split<M>::E > 16) ? 512 : 768;
}

template <int M, int RW, int MODE>
__global__ void __launch_bounds__(RW * Split<M>::TP, fx_inverse_min_threads<M, MODE>() / (RW * Split<M>::TP))
k_fx_inverse(GridDesc g, unsigned mask, const float2* __restrict__ spec, float* __restrict__ tau,
             const float* __restrict__ r32, double* __restrict__ partial) {
    constexpr int E = Split<M>::E, TP = Split<M>::TP, RS = row_stride<M>();
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
    const bool relax = g.relax != 0.0;   // relaxed schemes keep a fraction of the old field
    float2 old[E], radd[E];
    if (res || relax) s2_load<M>(old, out, t);
    if (addr) s2_load<M>(radd, reinterpret_cast<const float2*>(r32 + fbase), t);
    __shared__ float2 tws[2 * M];
    stage_twiddles<M>(tws, g);
    __syncthreads();
    float2 v[E];
    row_inverse<M, TP, E>(v, t, sh + r * RS, spec + (long long)slot * 3 * g.NNM + row * M, tws, tws + M);
    float acc = 0.f;
    const float wn = (float)(1.0 - g.relax), wo = (float)g.relax;
#pragma unroll
    for (int j = 0; j < E; ++j) {
        if (relax) v[j] = make_float2(wn * v[j].x + wo * old[j].x, wn * v[j].y + wo * old[j].y);
        if (addr) v[j] = make_float2(__fadd_rn(v[j].x, radd[j].x), __fadd_rn(v[j].y, radd[j].y));
        if (res) {
            const float da = v[j].x - old[j].x, db = v[j].y - old[j].y;
            acc += da * da + db * db;
        }
    }
    s2_store<M>(out, v, t);
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
__global__ void __launch_bounds__(RW * Split<M>::TP, 512 / (RW * Split<M>::TP))
k_fx_round(GridDesc g, unsigned mask, float2* __restrict__ spec, float* __restrict__ tau,
           const float* __restrict__ r32) {
    constexpr int E = Split<M>::E, TP = Split<M>::TP, RS = row_stride<M>();
    const int slot = blockIdx.y;
    if (!slot_active(g, mask, slot)) return;
    extern __shared__ __align__(16) float2 sh[];   // RW * RS
    __shared__ float2 lut[16];
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
    if (addr) s2_load<M>(radd, reinterpret_cast<const float2*>(r32 + fbase), t);
    uchar2 q[E];
    s2_load_phase<M>(q, reinterpret_cast<const uchar2*>(g.phase + (row % g.NN) * N), t);
    coef_pairs(lut, (float)g.Y[0], (float)g.Y[1], (float)g.Y[2]);
    float2* sp = spec + (long long)slot * 3 * g.NNM + row * M;
    float2* rs = sh + r * RS;
    __shared__ float2 tws[2 * M];
    stage_twiddles<M>(tws, g);
    __syncthreads();   // tables and coefficient pairs
    const float2* twM = tws;
    const float2* twN = tws + M;
    float2 v[E];
    row_inverse<M, TP, E>(v, t, rs, sp, twM, twN);
    // update (step 7), optional store, polarization of the next sweep (step 2)
#pragma unroll
    for (int j = 0; j < E; ++j)
        if (addr) v[j] = make_float2(__fadd_rn(v[j].x, radd[j].x), __fadd_rn(v[j].y, radd[j].y));
    if (WTAU) s2_store<M>(reinterpret_cast<float2*>(tau + fbase), v, t);
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = __fmul2_rn(v[j], lut[pair_index(q[j])]);
    row_sync<TP>();   // the row's threads have read their stage-2 values from rs
    // forward transform and real split, written over the row it came from
    row_forward_split<M, TP, E>(v, t, rs, twM, twN, sp);
}

// Dynamic shared memory of k_fx_round_p: the staged spectrum rows of one block (each
// row padded by 64 bytes, so that the two rows a half-warp reads fall on different bank
// halves), the block's phase rows (each padded by 32 bytes, so that the rows of a warp
// read different banks), and the rows' exchange buffers.
template <int M, int RW>
struct RoundSmem {
    static constexpr int SROW = M + 8;
    static constexpr int PROW = 2 * M + 32;
    static constexpr size_t spec_bytes = (size_t)RW * SROW * sizeof(float2);
    static constexpr size_t phase_off = spec_bytes;
    static constexpr size_t phase_bytes = (size_t)RW * PROW;
    static constexpr size_t x_off = (phase_off + phase_bytes + 15) / 16 * 16;
    static constexpr size_t total = x_off + (size_t)RW * row_stride<M>() * sizeof(float2);
};

// k_fx_round as a persistent kernel: each CTA walks row blocks (slot, component, rows)
// in a fixed stride over the grid.  While the rows of one block are transformed, the
// bulk-copy engine stages the spectrum and phase rows of the CTA's next block in shared
// memory, so the HBM reads of a block overlap the arithmetic of the one before (the plain
// kernel exposes the load latency of its single block).  The defect r is loaded from
// global memory at the start of a block and is in flight during the inverse transform.
// Same float operations as k_fx_round, so results are identical.
template <int M, int RW, bool ADDR, bool WTAU>
__global__ void __launch_bounds__(RW * Split<M>::TP, 512 / (RW * Split<M>::TP))
k_fx_round_p(GridDesc g, unsigned mask, float2* __restrict__ spec, float* __restrict__ tau,
             const float* __restrict__ r32, int nblk) {
    constexpr int E = Split<M>::E, TP = Split<M>::TP, RS = row_stride<M>();
    using L = RoundSmem<M, RW>;
    constexpr int N = 2 * M;
    extern __shared__ __align__(128) unsigned char dsm[];
    float2* sspec = reinterpret_cast<float2*>(dsm);
    unsigned char* sphase = dsm + L::phase_off;
    __shared__ float2 lut[16];
    __shared__ float2 tws[2 * M];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ int s_ok;
    const int t = threadIdx.x % TP, r = threadIdx.x / TP;
    const int nitems = g.nslots * nblk;
    int item = blockIdx.x;
    while (item < nitems && !slot_active(g, mask, item / nblk)) item += gridDim.x;
    if (item >= nitems) return;
    const uint32_t mb = async::smem_addr(&mbar);
    if (threadIdx.x == 0) async::mbar_init(mb);
    coef_pairs(lut, (float)g.Y[0], (float)g.Y[1], (float)g.Y[2]);
    stage_twiddles<M>(tws, g);
    // thread 0: stage the spectrum rows and phase rows of block `it`
    auto issue = [&](int it) {
        const int slot = it / nblk, b = it % nblk;
        const long long row0 = (b % 3) * g.NN + (long long)(b / 3) * RW;
        const float2* src = spec + (long long)slot * 3 * g.NNM + row0 * M;
        async::mbar_expect(mb, (uint32_t)(RW * M * sizeof(float2) + RW * N));
        for (int rr = 0; rr < RW; ++rr)
            async::bulk_g2s(async::smem_addr(sspec + rr * L::SROW), src + (long long)rr * M, M * sizeof(float2), mb);
        const uint8_t* prow = g.phase + (long long)(b / 3) * RW * N;
        for (int rr = 0; rr < RW; ++rr)
            async::bulk_g2s(async::smem_addr(sphase + rr * L::PROW), prow + (long long)rr * N, N, mb);
    };
    if (threadIdx.x == 0) issue(item);
    __syncthreads();   // barrier initialized, tables staged
    const float2* twM = tws;
    const float2* twN = tws + M;
    float2* rs = reinterpret_cast<float2*>(dsm + L::x_off) + r * RS;
    uint32_t parity = 0;
    while (item < nitems) {
        const int slot = item / nblk, b = item % nblk;
        const long long row = (b % 3) * g.NN + (long long)(b / 3) * RW + r;   // c*NN + z*N + y
        const long long fbase = (long long)slot * 3 * g.N3 + row * N;
        const bool addr = ADDR && (g.dflags ? (g.dflags[slot] & SF_ADDR) != 0 : true);
        float2 radd[E];
        if (addr) s2_load<M>(radd, reinterpret_cast<const float2*>(r32 + fbase), t);
        // this block's copies: one thread decides for the CTA whether the wait succeeded
        if (threadIdx.x == 0) s_ok = async::mbar_wait(mb, parity) ? 1 : 0;
        __syncthreads();
        if (!s_ok) {
            if (threadIdx.x == 0) atomicOr(&g_wait_fail, 1u);
            return;
        }
        async::mbar_wait(mb, parity);   // complete already: the copied bytes are visible here
        parity ^= 1u;
        float2 xk[E];
#pragma unroll
        for (int n1 = 0; n1 < E; ++n1) xk[n1] = sspec[r * L::SROW + TP * n1 + t];
        uchar2 q[E];
        s2_load_phase<M>(q, reinterpret_cast<const uchar2*>(sphase + r * L::PROW), t);
        __syncthreads();   // every thread holds its rows: the buffers take the next block
        int nxt = item + gridDim.x;
        while (nxt < nitems && !slot_active(g, mask, nxt / nblk)) nxt += gridDim.x;
        if (threadIdx.x == 0 && nxt < nitems) issue(nxt);
        // x inverse (steps 5), update (step 7), optional store, polarization (step 2)
        float2 v[E];
        c2r_merge_shfl<M, TP, E>(v, xk, twN, t);
        stage1_write<M, false, true>(v, t, twM, rs, 1);
        row_sync<TP>();
        stage2_read<M, false>(v, t, rs, 1);
#pragma unroll
        for (int j = 0; j < E; ++j)
            if (addr) v[j] = make_float2(__fadd_rn(v[j].x, radd[j].x), __fadd_rn(v[j].y, radd[j].y));
        if (WTAU) s2_store<M>(reinterpret_cast<float2*>(tau + fbase), v, t);
#pragma unroll
        for (int j = 0; j < E; ++j) v[j] = __fmul2_rn(v[j], lut[pair_index(q[j])]);
        row_sync<TP>();   // the row's threads have read their stage-2 values from rs
        // forward transform (step 3) and real split, written over the rows it came from
        row_forward_split<M, TP, E>(v, t, rs, twM, twN, spec + (long long)slot * 3 * g.NNM + row * M);
        row_sync<TP>();   // rs is reused by the next block (s_ok and the staging buffers are
                          // next written after CTA barriers every thread has passed)
        item = nxt;
    }
}

// ---------------------------------------------------------------------------
// y inverse + x round trip + y forward of a (component, z) plane in one persistent kernel.
// A CTA takes whole planes: it transforms the plane's columns along y in place, then its
// rows (x inverse, update, polarization of the next sweep, x forward), then its columns
// again, the plane (N x N/2 complex values) staying in L2 between the three phases, so a
// sweep makes two HBM round trips (this pass and the z pass) instead of four.  Each phase
// runs the operations of the separate kernels (k_fy, k_fx_round, k_fy) on the same data.
// The spectrum pointer is not __restrict__: each phase reads what other threads of the CTA
// wrote in the phase before (ordered by the CTA barriers), so no load may take the
// read-only path.
// ---------------------------------------------------------------------------

template <int L>
struct YxyShape {
    static constexpr int M = L / 2;
    static constexpr int P = 256 / Split<L>::TP;        // columns per y step
    static constexpr int RW = 256 / Split<M>::TP;       // rows per x step
    static constexpr int SY = P * xslots<L>();
    static constexpr int SX = RW * row_stride<M>();
    static constexpr size_t smem = sizeof(float2) * (SY > SX ? SY : SX);
};

// P columns of a plane along y (threads (p, t), p fastest), transformed in place.
template <int L, int P, bool FWD>
__device__ __forceinline__ void y_columns(const GridDesc& g, float2* base, int t, float2* sh) {
    constexpr int E = Split<L>::E, TP = Split<L>::TP, KPT = E / TP, M = L / 2;
    float2 v[E];
#pragma unroll
    for (int n1 = 0; n1 < E; ++n1) v[n1] = base[(long long)(TP * n1 + t) * M];
    const float2* twL = g.tw32 + g.pN.tw_off;
    stage1_write<L, FWD>(v, t, twL, sh, P);
    __syncthreads();
    stage2_read<L, FWD>(v, t, sh, P);
#pragma unroll
    for (int i = 0; i < KPT; ++i)
#pragma unroll
        for (int k2 = 0; k2 < TP; ++k2) base[(long long)(t * KPT + i + E * k2) * M] = v[i * TP + k2];
}

template <int L, bool ADDR, bool WTAU>
__global__ void __launch_bounds__(256, 2)
k_yxy(GridDesc g, unsigned mask, float2* spec, float* __restrict__ tau, const float* __restrict__ r32, int nper) {
    using S = YxyShape<L>;
    constexpr int M = S::M, P = S::P, RW = S::RW;
    constexpr int N = L;
    constexpr int EX = Split<M>::E, TPX = Split<M>::TP, RS = row_stride<M>();
    extern __shared__ __align__(16) float2 sh[];
    __shared__ float2 lut[16];
    __shared__ float2 tws[2 * M];
    coef_pairs(lut, (float)g.Y[0], (float)g.Y[1], (float)g.Y[2]);
    stage_twiddles<M>(tws, g);
    __syncthreads();
    const float2* twM = tws;
    const float2* twN = tws + M;
    const int nitems = g.nslots * nper;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int slot = item / nper, pz = item % nper;   // pz = component * N + z
        if (!slot_active(g, mask, slot)) continue;         // uniform over the CTA
        float2* plane = spec + (long long)slot * 3 * g.NNM + (long long)pz * N * M;
        // y inverse (step 5, first axis), columns in place
        {
            const int p = threadIdx.x % P, t = threadIdx.x / P;
            for (int kb = 0; kb < M / P; ++kb) {
                y_columns<L, P, false>(g, plane + kb * P + p, t, sh + p);
                __syncthreads();
            }
        }
        // x inverse, update (step 7), optional store, polarization (step 2), x forward (step 3)
        {
            const int t = threadIdx.x % TPX, r = threadIdx.x / TPX;
            const bool addr = ADDR && (g.dflags ? (g.dflags[slot] & SF_ADDR) != 0 : true);
            float2* rs = sh + r * RS;
            for (int rb = 0; rb < N / RW; ++rb) {
                const int y = rb * RW + r;
                const long long row = (long long)pz * N + y;                   // c*NN + z*N + y
                const long long fbase = (long long)slot * 3 * g.N3 + row * N;
                float2 radd[EX];
                if (addr) s2_load<M>(radd, reinterpret_cast<const float2*>(r32 + fbase), t);
                uchar2 q[EX];
                s2_load_phase<M>(q, reinterpret_cast<const uchar2*>(g.phase + (row % g.NN) * N), t);
                float2* sp = plane + (long long)y * M;
                float2 v[EX];
                row_inverse<M, TPX, EX>(v, t, rs, sp, twM, twN);
#pragma unroll
                for (int j = 0; j < EX; ++j)
                    if (addr) v[j] = make_float2(__fadd_rn(v[j].x, radd[j].x), __fadd_rn(v[j].y, radd[j].y));
                if (WTAU) s2_store<M>(reinterpret_cast<float2*>(tau + fbase), v, t);
#pragma unroll
                for (int j = 0; j < EX; ++j) v[j] = __fmul2_rn(v[j], lut[pair_index(q[j])]);
                row_sync<TPX>();
                row_forward_split<M, TPX, EX>(v, t, rs, twM, twN, sp);
                row_sync<TPX>();
            }
        }
        __syncthreads();   // the rows are in memory; the exchange buffer takes the columns
        // y forward (step 3, second axis) of the next sweep, columns in place
        {
            const int p = threadIdx.x % P, t = threadIdx.x / P;
            for (int kb = 0; kb < M / P; ++kb) {
                y_columns<L, P, true>(g, plane + kb * P + p, t, sh + p);
                __syncthreads();
            }
        }
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
// Grid of a persistent kernel: as many CTAs as fit on the GPU at once (occupancy of the
// kernel at its shared memory), at most one per work item.
template <typename K>
int persistent_grid(K kern, int threads, size_t smem, int items) {
    static const int sms = [] {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return std::max(n, 1);
    }();
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem) != cudaSuccess || per < 1) per = 1;
    return std::max(1, std::min(items, per * sms));
}
// cuTensorMapEncodeTiled from the driver (looked up once; null when unavailable).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}
// Tensor map of a packed spectrum for the persistent z pass: 4D array (kx: M, ky: N,
// kz: N, slot * 3 + component) of 8-byte complex values, box of P kx by all N kz.
bool z_tensor_map(const GridDesc& g, const float2* spec, int P, CUtensorMap* out) {
    auto enc = tensor_map_encoder();
    if (!enc || g.N > 256) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)g.M, (cuuint64_t)g.N, (cuuint64_t)g.N, (cuuint64_t)(3 * g.nslots)};
    const cuuint64_t strides[3] = {(cuuint64_t)g.M * 8, (cuuint64_t)g.N * g.M * 8, (cuuint64_t)g.NNM * 8};
    const cuuint32_t box[4] = {(cuuint32_t)P, 1, (cuuint32_t)g.N, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(out, CU_TENSOR_MAP_DATA_TYPE_INT64, 4, const_cast<float2*>(spec), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
template <int L> constexpr int fz_cols() { return pow2_cols(128 / fast::Split<L>::TP, L / 2); }
// x passes run 128-thread CTAs: their barriers stall fewer warps and the load phases of
// the CTAs on an SM drift apart (x round trip 400 -> 376 us at 256^3 against 256 threads)
template <int M> constexpr int fx_rows() { return 128 / fast::Split<M>::TP; }
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
        HMG_FAST_LEN(512, FY)
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
        case 512: P = fz_cols<512>(); break;
        default: return 0;
    }
    if (g.M % P) return 0;
    return g.N * (g.M / P);
}

namespace {
template <int L, int P>
void launch_fzs(int mode, dim3 grid, size_t sm, cudaStream_t st, const GridDesc& g, unsigned mask, float2* sp,
                double* partial) {
    constexpr int T = 3 * P * fast::Split<L>::TP;
    switch (mode) {
        case Z_FWD: launch_dyn(fast::k_fzs<L, P, Z_FWD>, grid, T, sm, st, g, mask, sp, partial); break;
        case Z_INV: launch_dyn(fast::k_fzs<L, P, Z_INV>, grid, T, sm, st, g, mask, sp, partial); break;
        case Z_ITER: launch_dyn(fast::k_fzs<L, P, Z_ITER>, grid, T, sm, st, g, mask, sp, partial); break;
        case Z_ITER_NOB: launch_dyn(fast::k_fzs<L, P, Z_ITER_NOB>, grid, T, sm, st, g, mask, sp, partial); break;
        default: launch_dyn(fast::k_fzs<L, P, Z_EQ>, grid, T, sm, st, g, mask, sp, partial); break;
    }
}
// The persistent z pass (plain and correction sweeps); false when it does not apply.
template <int L, int P>
bool launch_fz3_p(int mode, cudaStream_t st, const GridDesc& g, unsigned mask, float2* sp) {
    if constexpr (L > 256) {
        return false;
    } else {
        if (mode != Z_ITER && mode != Z_ITER_NOB) return false;
        CUtensorMap map;
        if (!z_tensor_map(g, sp, P, &map)) return false;
        constexpr int T = P * fast::Split<L>::TP;
        constexpr size_t sm = fast::ZSmem<L, P>::total;
        auto kern = mode == Z_ITER ? fast::k_fz3_p<L, P, Z_ITER> : fast::k_fz3_p<L, P, Z_ITER_NOB>;
        const int nper = g.N * (g.M / P);
        const int grid = persistent_grid(kern, T, sm, nper * g.nslots);
        kern<<<grid, T, sm, st>>>(map, g, mask, sp, nper);
        return true;
    }
}
template <int L, int P>
void launch_fz3(int mode, dim3 grid, size_t sm, cudaStream_t st, const GridDesc& g, unsigned mask, float2* sp,
                double* partial) {
    constexpr int T = P * fast::Split<L>::TP;
    switch (mode) {
        case Z_FWD: launch_dyn(fast::k_fz3<L, P, Z_FWD>, grid, T, sm, st, g, mask, sp, partial); break;
        case Z_INV: launch_dyn(fast::k_fz3<L, P, Z_INV>, grid, T, sm, st, g, mask, sp, partial); break;
        case Z_ITER: launch_dyn(fast::k_fz3<L, P, Z_ITER>, grid, T, sm, st, g, mask, sp, partial); break;
        case Z_ITER_NOB: launch_dyn(fast::k_fz3<L, P, Z_ITER_NOB>, grid, T, sm, st, g, mask, sp, partial); break;
        default: launch_dyn(fast::k_fz3<L, P, Z_EQ>, grid, T, sm, st, g, mask, sp, partial); break;
    }
}
// z pass of length L: the three-components-per-thread kernel (variant 0) holds 3 E complex
// values per thread and exists up to E = 24 (L <= 256); longer columns always use the
// per-component thread groups (variant 1).
template <int L>
bool fast_z_len(const GridDesc& g, int mode, unsigned mask, float2* sp, double* partial, cudaStream_t st) {
    constexpr int P = fz_cols<L>();
    if (g.M % P) return false;
    dim3 grid(g.N * (g.M / P), g.nslots);
    const size_t sm = sizeof(float2) * 3 * fast::xslots<L>() * P;
    if constexpr (fast::Split<L>::E > 24) {
        launch_fzs<L, P>(mode, grid, sm, st, g, mask, sp, partial);
    } else {
        if (g.zvar == 1) launch_fzs<L, P>(mode, grid, sm, st, g, mask, sp, partial);
        else if (!(g.zpers && launch_fz3_p<L, P>(mode, st, g, mask, sp)))
            launch_fz3<L, P>(mode, grid, sm, st, g, mask, sp, partial);
    }
    return true;
}
}  // namespace

bool fast_z(const GridDesc& g, int mode, unsigned mask, void* spec, double* partial, cudaStream_t st) {
    float2* sp = reinterpret_cast<float2*>(spec);
    switch (g.N) {
        case 64: return fast_z_len<64>(g, mode, mask, sp, partial, st);
        case 96: return fast_z_len<96>(g, mode, mask, sp, partial, st);
        case 128: return fast_z_len<128>(g, mode, mask, sp, partial, st);
        case 192: return fast_z_len<192>(g, mode, mask, sp, partial, st);
        case 256: return fast_z_len<256>(g, mode, mask, sp, partial, st);
        case 512: return fast_z_len<512>(g, mode, mask, sp, partial, st);
        default: return false;
    }
}

int fast_x_ctas(const GridDesc& g) {
    int RW = 0;
    switch (g.M) {
        case 32: RW = fx_rows<32>(); break;
        case 48: RW = fx_rows<48>(); break;
        case 64: RW = fx_rows<64>(); break;
        case 96: RW = fx_rows<96>(); break;
        case 128: RW = fx_rows<128>(); break;
        case 256: RW = fx_rows<256>(); break;
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
        HMG_FAST_LEN(256, FXF)
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
        HMG_FAST_LEN(256, FXI)
        default: return false;
    }
#undef FXI
}

bool chain_sweeps(const GridDesc& g) {
    // a relaxed scheme needs the old field in every x inverse: its sweeps are not chained
    return !g.nochain && g.relax == 0.0 && !(g.xyvar == 1 && fused_cluster(g.N)) && fast_x_ctas(g) > 0;
}

namespace {
template <int M, bool ADDR, bool WTAU>
void launch_round_p(const GridDesc& g, unsigned mask, float2* sp, float* tau, const float* r32, cudaStream_t st) {
    constexpr int RW = fx_rows<M>();
    constexpr int T = RW * fast::Split<M>::TP;
    constexpr size_t sm = fast::RoundSmem<M, RW>::total;
    auto kern = fast::k_fx_round_p<M, RW, ADDR, WTAU>;
    const int nblk = fast_x_ctas(g);
    const int grid = persistent_grid(kern, T, sm, nblk * g.nslots);
    kern<<<grid, T, sm, st>>>(g, mask, sp, tau, r32, nblk);
}
}  // namespace

namespace {
int fast_split_e(int M) {
    switch (M) {
        case 32: return fast::Split<32>::E;
        case 48: return fast::Split<48>::E;
        case 64: return fast::Split<64>::E;
        case 96: return fast::Split<96>::E;
        case 128: return fast::Split<128>::E;
        case 256: return fast::Split<256>::E;
        default: return 0;
    }
}
}  // namespace

bool fast_take_wait_failure() {
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, fast::g_wait_fail, sizeof v) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (v) {
        const unsigned z = 0;
        cudaMemcpyToSymbol(fast::g_wait_fail, &z, sizeof z);
    }
    return v != 0;
}

bool fast_x_round(const GridDesc& g, bool addr, bool wtau, unsigned mask, void* spec, float* tau, const float* r32,
                  cudaStream_t st) {
    float2* sp = reinterpret_cast<float2*>(spec);
    if (!fast_x_ctas(g)) return false;
    // the persistent form of the correction sweeps (r added) of 24-value rows would keep
    // r in registers beside the transform and spill; those use the plain kernel
    if (g.xpers && !(addr && fast_split_e(g.M) > 16)) {
#define FXRP(M)                                                                            \
    {                                                                                      \
        if (addr && wtau) launch_round_p<M, true, true>(g, mask, sp, tau, r32, st);        \
        else if (addr) launch_round_p<M, true, false>(g, mask, sp, tau, r32, st);          \
        else if (wtau) launch_round_p<M, false, true>(g, mask, sp, tau, r32, st);          \
        else launch_round_p<M, false, false>(g, mask, sp, tau, r32, st);                   \
    }
        switch (g.M) {
            HMG_FAST_LEN(32, FXRP)
            HMG_FAST_LEN(48, FXRP)
            HMG_FAST_LEN(64, FXRP)
            HMG_FAST_LEN(96, FXRP)
            HMG_FAST_LEN(128, FXRP)
            HMG_FAST_LEN(256, FXRP)
            default: return false;
        }
#undef FXRP
    }
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
        HMG_FAST_LEN(256, FXR)
        default: return false;
    }
#undef FXR
}

namespace {
template <int L, bool ADDR, bool WTAU>
void launch_yxy(const GridDesc& g, unsigned mask, float2* sp, float* tau, const float* r32, cudaStream_t st) {
    auto kern = fast::k_yxy<L, ADDR, WTAU>;
    constexpr size_t sm = fast::YxyShape<L>::smem;
    const int nper = 3 * g.N;
    const int grid = persistent_grid(kern, 256, sm, nper * g.nslots);
    kern<<<grid, 256, sm, st>>>(g, mask, sp, tau, r32, nper);
}
}  // namespace

bool fast_yxy_available(const GridDesc& g) {
    return g.relax == 0.0 && (g.N == 64 || g.N == 128 || g.N == 192 || g.N == 256);
}

bool fast_yxy(const GridDesc& g, bool addr, bool wtau, unsigned mask, void* spec, float* tau, const float* r32,
              cudaStream_t st) {
    if (!fast_yxy_available(g)) return false;
    float2* sp = reinterpret_cast<float2*>(spec);
#define FYXY(L)                                                                        \
    {                                                                                  \
        if (addr && wtau) launch_yxy<L, true, true>(g, mask, sp, tau, r32, st);        \
        else if (addr) launch_yxy<L, true, false>(g, mask, sp, tau, r32, st);          \
        else if (wtau) launch_yxy<L, false, true>(g, mask, sp, tau, r32, st);          \
        else launch_yxy<L, false, false>(g, mask, sp, tau, r32, st);                   \
    }
    switch (g.N) {
        HMG_FAST_LEN(64, FYXY)
        HMG_FAST_LEN(128, FYXY)
        HMG_FAST_LEN(192, FYXY)
        HMG_FAST_LEN(256, FYXY)
        default: return false;
    }
#undef FYXY
}

#undef HMG_FAST_LEN

}  // namespace hmg
