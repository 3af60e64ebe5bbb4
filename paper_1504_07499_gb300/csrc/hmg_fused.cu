// Fused x + y passes (FP32) on thread-block clusters: one sweep of §3's steps 2-7 then
// moves the field through HBM three times (xy forward, z with the Green operator, yx
// inverse) instead of five.
//
// A cluster of C CTAs owns one (component, z) plane of the N x N grid.  Forward: CTA r
// loads rows y in [r N/C, (r+1) N/C), polarizes them, does the real-to-complex x
// transform of each row, and writes each row's N/2 coefficients into the shared memory
// of the CTA owning that kx block (distributed shared memory); after a cluster barrier
// CTA b transforms its N/2/C kx columns along y and stores them.  Inverse: the mirror
// image -- y transforms of a kx block, scattered to the row owners, complex-to-real x
// transforms, and the sweep's output step (add r, residual against the old field).
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "hmg_fft.cuh"
#include "hmg_internal.h"
#include "hmg_regfft.cuh"

namespace cg = cooperative_groups;

namespace hmg {
namespace fused {

using fast::RegDFT;
using fast::Split;
using fast::xslots;

template <int L, int C>
struct Geo {
    static constexpr int N = L, M = L / 2;
    static constexpr int RW = N / C;                  // rows per CTA (x stage)
    static constexpr int CW = M / C;                  // kx columns per CTA (y stage)
    static constexpr int EX = Split<M>::E, TPX = Split<M>::TP, KX = EX / TPX;
    static constexpr int EY = Split<N>::E, TPY = Split<N>::TP, KY = EY / TPY;
    static constexpr int XT = RW * TPX, YT = CW * TPY;
    static constexpr int T = XT > YT ? XT : YT;
    static constexpr int RS = fast::row_stride<M>();  // row stride of the x buffer
    static constexpr int XB = RW * RS;                // x buffer (complex values)
    static constexpr int YB = xslots<N>() * CW;      // y buffer
    static constexpr size_t SMEM = sizeof(float2) * (XB + YB);
};

// xy forward: polarize (or flux factor) on load, x R2C, DSMEM scatter, y transform
template <int L, int C, int MODE>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(Geo<L, C>::T)
k_xy_forward(GridDesc g, unsigned mask, const float* __restrict__ tau, float2* __restrict__ spec,
             double* __restrict__ partial) {
    using G = Geo<L, C>;
    constexpr int N = G::N, M = G::M, RW = G::RW, CW = G::CW;
    constexpr int EX = G::EX, TPX = G::TPX, KX = G::KX, EY = G::EY, TPY = G::TPY, KY = G::KY;
    const int slot = blockIdx.y;
    if (!slot_active(g, mask, slot)) return;   // uniform over the cluster (same slot)
    extern __shared__ __align__(16) float2 sm[];
    float2* xb = sm;
    float2* yb = sm + G::XB;
    __shared__ double red[G::T / 32 + 1];
    cg::cluster_group cluster = cg::this_cluster();
    // no CTA may write into another's shared memory before every CTA of the cluster has
    // started: arrive now, wait right before the first remote store
    auto started = cluster.barrier_arrive();
    const int rank = (int)cluster.block_rank();
    const int plane = blockIdx.x / C;          // z * 3 + c: components of a plane adjacent
    const int c = plane % 3, z = plane / 3;
    const int tid = threadIdx.x;
    const long long NN = (long long)N * N;
    const long long fbase = ((long long)slot * 3 + c) * NN * N + (long long)z * NN;   // element offset of the plane

    // ---- x stage: rows y = rank RW + r
    const int tx = tid % TPX, r = tid / TPX;
    const int y = rank * RW + r;
    float2 v[EX > EY ? EX : EY];
    float acc = 0.f;
    if (tid < G::XT) {
        const float2* src = reinterpret_cast<const float2*>(tau + fbase + (long long)y * N);
#pragma unroll
        for (int n1 = 0; n1 < EX; ++n1) v[n1] = src[TPX * n1 + tx];
        if (MODE != XF_PLAIN) {
            const uchar2* ph = reinterpret_cast<const uchar2*>(g.phase + ((long long)z * N + y) * N);
            const float c0 = (float)(MODE == XF_POLARIZE ? g.Y[0] : g.W[0]);
            const float c1 = (float)(MODE == XF_POLARIZE ? g.Y[1] : g.W[1]);
            const float c2 = (float)(MODE == XF_POLARIZE ? g.Y[2] : g.W[2]);
#pragma unroll
            for (int n1 = 0; n1 < EX; ++n1) {
                const uchar2 q = ph[TPX * n1 + tx];
                v[n1].x *= fast::sel3f(q.x, c0, c1, c2);
                v[n1].y *= fast::sel3f(q.y, c0, c1, c2);
                if (MODE == XF_FLUX) acc += v[n1].x + v[n1].y;
            }
        }
        fast::stage1_write<M, true>(v, tx, g.tw32 + g.pM.tw_off, xb + r * G::RS, 1);
    }
    __syncthreads();
    if (tid < G::XT) fast::stage2_read<M, true>(v, tx, xb + r * G::RS, 1);
    __syncthreads();
    if (tid < G::XT) {
#pragma unroll
        for (int i = 0; i < KX; ++i)
#pragma unroll
            for (int k2 = 0; k2 < TPX; ++k2) xb[r * G::RS + tx * KX + i + EX * k2] = v[i * TPX + k2];
    }
    if (MODE == XF_FLUX) {
        const double s = fast::block_sum_any((double)acc, red);
        if (tid == 0) partial[(long long)slot * gridDim.x + (long long)c * (N * C) + z * C + rank] = s;
    } else {
        __syncthreads();
    }
    // real-to-complex split and scatter of coefficient kx to the owner of its column block
    cluster.barrier_wait(std::move(started));
    if (tid < G::XT) {
        const float2* twN = g.tw32 + g.pN.tw_off;
        const float2* rs = xb + r * G::RS;
#pragma unroll
        for (int j = 0; j < EX; ++j) {
            const int k = tx + TPX * j;
            const float2 zk = rs[k];
            float2 out;
            if (k == 0) {
                out = make_float2(zk.x + zk.y, zk.x - zk.y);
            } else {
                const float2 zm = rs[M - k];
                const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
                const float2 o = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
                out = cadd(e, cmul(o, __ldg(&twN[k])));
            }
            float2* dst = cluster.map_shared_rank(yb, k / CW);
            dst[y * CW + (k % CW)] = out;   // natural layout [y][column] of the owner
        }
    }
    cluster.sync();   // every row of every CTA has arrived

    // ---- y stage: kx columns rank CW + p
    const int p = tid % CW, ty = tid / CW;
    if (tid < G::YT) {
#pragma unroll
        for (int n1 = 0; n1 < EY; ++n1) v[n1] = yb[(TPY * n1 + ty) * CW + p];
    }
    __syncthreads();
    if (tid < G::YT) fast::stage1_write<N, true>(v, ty, g.tw32 + g.pN.tw_off, yb + p, CW);
    __syncthreads();
    if (tid < G::YT) {
        fast::stage2_read<N, true>(v, ty, yb + p, CW);
        float2* dst = spec + ((long long)slot * 3 + c) * NN * M + (long long)z * N * M + rank * CW + p;
#pragma unroll
        for (int i = 0; i < KY; ++i)
#pragma unroll
            for (int k2 = 0; k2 < TPY; ++k2) dst[(long long)(ty * KY + i + EY * k2) * M] = v[i * TPY + k2];
    }
}

// yx inverse: y transform of a kx block, DSMEM scatter to the row owners, C2R x transform,
// output step (INPLACE / ADD_R / residual, as the register-resident x inverse)
template <int L, int C, int MODE>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(Geo<L, C>::T)
k_yx_inverse(GridDesc g, unsigned mask, const float2* __restrict__ spec, float* __restrict__ tau,
             const float* __restrict__ r32, double* __restrict__ partial) {
    using G = Geo<L, C>;
    constexpr int N = G::N, M = G::M, RW = G::RW, CW = G::CW;
    constexpr int EX = G::EX, TPX = G::TPX, KX = G::KX, EY = G::EY, TPY = G::TPY, KY = G::KY;
    const int slot = blockIdx.y;
    if (!slot_active(g, mask, slot)) return;
    extern __shared__ __align__(16) float2 sm[];
    float2* xb = sm;
    float2* yb = sm + G::XB;
    __shared__ double red[G::T / 32 + 1];
    cg::cluster_group cluster = cg::this_cluster();
    auto started = cluster.barrier_arrive();   // see k_xy_forward
    const int rank = (int)cluster.block_rank();
    const int plane = blockIdx.x / C;
    const int c = plane % 3, z = plane / 3;
    const int tid = threadIdx.x;
    const long long NN = (long long)N * N;

    // ---- y stage (inverse) on kx columns rank CW + p
    const int p = tid % CW, ty = tid / CW;
    float2 v[EX > EY ? EX : EY];
    if (tid < G::YT) {
        const float2* src = spec + ((long long)slot * 3 + c) * NN * M + (long long)z * N * M + rank * CW + p;
#pragma unroll
        for (int n1 = 0; n1 < EY; ++n1) v[n1] = src[(long long)(TPY * n1 + ty) * M];
        fast::stage1_write<N, false>(v, ty, g.tw32 + g.pN.tw_off, yb + p, CW);
    }
    __syncthreads();
    cluster.barrier_wait(std::move(started));
    if (tid < G::YT) {
        fast::stage2_read<N, false>(v, ty, yb + p, CW);
        // row y of column kx goes to the owner of row y
#pragma unroll
        for (int i = 0; i < KY; ++i)
#pragma unroll
            for (int k2 = 0; k2 < TPY; ++k2) {
                const int yy = ty * KY + i + EY * k2;
                float2* dst = cluster.map_shared_rank(xb, yy / RW);
                dst[(yy % RW) * G::RS + rank * CW + p] = v[i * TPY + k2];
            }
    }
    cluster.sync();

    // ---- x stage: rows y = rank RW + r
    const int tx = tid % TPX, r = tid / TPX;
    const int y = rank * RW + r;
    float2* rs = xb + r * G::RS;
    if (tid < G::XT) {
        const float2* twN = g.tw32 + g.pN.tw_off;
#pragma unroll
        for (int n1 = 0; n1 < EX; ++n1) {
            const int k = TPX * n1 + tx;
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
    }
    __syncthreads();
    if (tid < G::XT) fast::stage1_write<M, false>(v, tx, g.tw32 + g.pM.tw_off, rs, 1);
    __syncthreads();
    if (tid < G::XT) fast::stage2_read<M, false>(v, tx, rs, 1);
    __syncthreads();
    if (tid < G::XT) {
#pragma unroll
        for (int i = 0; i < KX; ++i)
#pragma unroll
            for (int k2 = 0; k2 < TPX; ++k2) rs[tx * KX + i + EX * k2] = v[i * TPX + k2];
    }
    __syncthreads();
    constexpr bool kRes = MODE == XI_INPLACE_RES || MODE == XI_ADD_R_RES;
    constexpr bool kAddR = MODE == XI_ADD_R_RES || MODE == XI_ADD_R;
    const bool res = kRes && (g.dflags ? g.resid != 0 : true);
    const bool addr = kAddR && (g.dflags ? (g.dflags[slot] & SF_ADDR) != 0 : true);
    float acc = 0.f;
    if (tid < G::XT) {
        const long long fo = ((long long)slot * 3 + c) * NN * N + (long long)z * NN + (long long)y * N;
        float2* out = reinterpret_cast<float2*>(tau + fo);
        const float2* rr = reinterpret_cast<const float2*>(r32 + fo);
#pragma unroll
        for (int j = 0; j < EX; ++j) {
            float2 x = rs[tx + TPX * j];
            if (addr) {
                const float2 a = rr[tx + TPX * j];
                x.x += a.x;
                x.y += a.y;
            }
            if (res) {
                const float2 o = out[tx + TPX * j];
                const float da = x.x - o.x, db = x.y - o.y;
                acc += da * da + db * db;
            }
            out[tx + TPX * j] = x;
        }
    }
    if (kRes) {
        const double s = fast::block_sum_any((double)acc, red);
        if (tid == 0 && res) partial[(long long)slot * gridDim.x + blockIdx.x] = s;
    }
}

}  // namespace fused

namespace {
template <typename K, typename... Args>
void launch_cluster(K kern, dim3 grid, int threads, size_t bytes, cudaStream_t st, Args... args) {
    if (bytes > 32 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    kern<<<grid, threads, bytes, st>>>(args...);
}
}  // namespace

// Cluster width per grid size (0: no fused kernels for this size).
int fused_cluster(int N) {
    switch (N) {
        case 128: return 4;
        case 192: return 4;
        case 256: return 8;
        default: return 0;
    }
}

int fused_xy_ctas(const GridDesc& g) { return fused_cluster(g.N) ? 3 * g.N * fused_cluster(g.N) : 0; }

#define HMG_FUSED_SIZES(X) X(128, 4) X(192, 4) X(256, 8)

bool fused_xy_forward(const GridDesc& g, int mode, unsigned mask, const float* tau, void* spec, double* partial,
                      cudaStream_t st) {
    float2* sp = reinterpret_cast<float2*>(spec);
#define FXY(L, C)                                                                                           \
    if (g.N == L) {                                                                                         \
        using G = fused::Geo<L, C>;                                                                         \
        dim3 grid(3 * L * C, g.nslots);                                                                     \
        if (mode == XF_PLAIN)                                                                               \
            launch_cluster(fused::k_xy_forward<L, C, XF_PLAIN>, grid, G::T, G::SMEM, st, g, mask, tau, sp, partial); \
        else if (mode == XF_POLARIZE)                                                                       \
            launch_cluster(fused::k_xy_forward<L, C, XF_POLARIZE>, grid, G::T, G::SMEM, st, g, mask, tau, sp, partial); \
        else                                                                                                \
            launch_cluster(fused::k_xy_forward<L, C, XF_FLUX>, grid, G::T, G::SMEM, st, g, mask, tau, sp, partial); \
        return true;                                                                                        \
    }
    HMG_FUSED_SIZES(FXY)
#undef FXY
    return false;
}

bool fused_yx_inverse(const GridDesc& g, int mode, unsigned mask, const void* spec, float* tau, const float* r32,
                      double* partial, cudaStream_t st) {
    const float2* sp = reinterpret_cast<const float2*>(spec);
    if (mode != XI_PLAIN && mode != XI_INPLACE && mode != XI_INPLACE_RES && mode != XI_ADD_R_RES && mode != XI_ADD_R)
        return false;
#define FYX(L, C)                                                                                                      \
    if (g.N == L) {                                                                                                    \
        using G = fused::Geo<L, C>;                                                                                    \
        dim3 grid(3 * L * C, g.nslots);                                                                                \
        if (mode == XI_INPLACE_RES)                                                                                    \
            launch_cluster(fused::k_yx_inverse<L, C, XI_INPLACE_RES>, grid, G::T, G::SMEM, st, g, mask, sp, tau, r32, partial); \
        else if (mode == XI_ADD_R_RES)                                                                                 \
            launch_cluster(fused::k_yx_inverse<L, C, XI_ADD_R_RES>, grid, G::T, G::SMEM, st, g, mask, sp, tau, r32, partial); \
        else if (mode == XI_ADD_R)                                                                                     \
            launch_cluster(fused::k_yx_inverse<L, C, XI_ADD_R>, grid, G::T, G::SMEM, st, g, mask, sp, tau, r32, partial); \
        else                                                                                                           \
            launch_cluster(fused::k_yx_inverse<L, C, XI_INPLACE>, grid, G::T, G::SMEM, st, g, mask, sp, tau, r32, partial); \
        return true;                                                                                                   \
    }
    HMG_FUSED_SIZES(FYX)
#undef FYX
    return false;
}

#undef HMG_FUSED_SIZES

}  // namespace hmg
