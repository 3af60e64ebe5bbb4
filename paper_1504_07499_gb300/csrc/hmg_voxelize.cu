// Voxelization of coated spheres into the three-phase grid (§2, Fig. 1).
// Integer rule on quantized coordinates (quantization is done on the host):
// voxel centres sit at odd multiples of G = 4096 in units of 1/(2 N G); a voxel is
// inclusion (1) if inside any core, else coating (2) if inside any sphere, else
// matrix (0), with periodic minimum-image distances and inclusive boundaries.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hmg_internal.h"

namespace hmg {

constexpr int kVoxChunk = 512;       // spheres staged in shared memory per pass
constexpr int kVoxPerThread = 4;     // consecutive x voxels per thread

__device__ __forceinline__ long long axis_d2(long long v, long long c, long long S) {
    long long d = v - c;
    if (d < 0) d += S;
    const long long e = S - d;
    d = d < e ? d : e;
    return d * d;
}

// One CTA covers a run of kThreads * kVoxPerThread voxels along x-major order.
__global__ void __launch_bounds__(kThreads)
k_voxelize(const long long* __restrict__ q, int n, int N, long long S, uint8_t* __restrict__ out) {
    __shared__ long long sq[kVoxChunk * 5];
    const long long N3 = (long long)N * N * N;
    const long long first = ((long long)blockIdx.x * kThreads + threadIdx.x) * kVoxPerThread;
    const long long G2 = 2 * 4096;
    long long d2yz[kVoxPerThread];
    long long vx[kVoxPerThread], vy[kVoxPerThread], vz[kVoxPerThread];
    int ph[kVoxPerThread];
#pragma unroll
    for (int t = 0; t < kVoxPerThread; ++t) {
        const long long i = first + t;
        const long long ii = i < N3 ? i : 0;
        const long long x = ii % N, y = (ii / N) % N, z = ii / ((long long)N * N);
        vx[t] = x * G2 + 4096;
        vy[t] = y * G2 + 4096;
        vz[t] = z * G2 + 4096;
        ph[t] = 0;
        d2yz[t] = 0;
    }
    for (int base = 0; base < n; base += kVoxChunk) {
        const int cnt = (n - base) < kVoxChunk ? (n - base) : kVoxChunk;
        __syncthreads();
        for (int k = threadIdx.x; k < cnt * 5; k += blockDim.x) sq[k] = q[(long long)base * 5 + k];
        __syncthreads();
        for (int s = 0; s < cnt; ++s) {
            const long long cx = sq[5 * s], cy = sq[5 * s + 1], cz = sq[5 * s + 2];
            const long long ro2 = sq[5 * s + 3], ri2 = sq[5 * s + 4];
#pragma unroll
            for (int t = 0; t < kVoxPerThread; ++t) {
                const long long d2 = axis_d2(vx[t], cx, S) + axis_d2(vy[t], cy, S) + axis_d2(vz[t], cz, S);
                if (d2 <= ri2) ph[t] = 1;
                else if (d2 <= ro2 && ph[t] == 0) ph[t] = 2;
            }
        }
    }
#pragma unroll
    for (int t = 0; t < kVoxPerThread; ++t) {
        const long long i = first + t;
        if (i < N3) out[i] = (uint8_t)ph[t];
    }
}

// Coated cylinders merged into a phase grid (§6: RVEs with cylinders, or spheres and
// cylinders).  Integer rule (quantization on the host): voxel centres at odd multiples of
// GC = 256 in units of 1/(2 N GC); per cylinder q holds the centre C, the axis A (integer,
// about 1024 u), R_out^2, R_in^2, H_out, H_in.  With d the signed minimum-image offset of a
// voxel centre from C and t = d . A, the voxel lies in the cylinder when
// |d|^2 |A|^2 - t^2 <= R^2 |A|^2 and t^2 <= H^2 |A|^2.  A voxel already inclusion stays so;
// a core makes it inclusion, an outer cylinder makes a matrix voxel coating.
__device__ __forceinline__ long long signed_image(long long v, long long c, long long S) {
    long long d = v - c + (S >> 1);   // in (-S/2, 3S/2)
    if (d < 0) d += S;
    if (d >= S) d -= S;
    return d - (S >> 1);              // in [-S/2, S/2)
}

__global__ void __launch_bounds__(kThreads)
k_voxelize_cyl(const long long* __restrict__ q, int n, int N, long long S, uint8_t* __restrict__ out) {
    __shared__ long long sq[kVoxChunk * 10];
    const long long N3 = (long long)N * N * N;
    const long long first = ((long long)blockIdx.x * kThreads + threadIdx.x) * kVoxPerThread;
    const long long G2 = 2 * 256;
    long long vx[kVoxPerThread], vy[kVoxPerThread], vz[kVoxPerThread];
    int ph[kVoxPerThread];
#pragma unroll
    for (int t = 0; t < kVoxPerThread; ++t) {
        const long long i = first + t;
        const long long ii = i < N3 ? i : 0;
        const long long x = ii % N, y = (ii / N) % N, z = ii / ((long long)N * N);
        vx[t] = x * G2 + 256;
        vy[t] = y * G2 + 256;
        vz[t] = z * G2 + 256;
        ph[t] = i < N3 ? out[i] : 0;
    }
    for (int base = 0; base < n; base += kVoxChunk) {
        const int cnt = (n - base) < kVoxChunk ? (n - base) : kVoxChunk;
        __syncthreads();
        for (int k = threadIdx.x; k < cnt * 10; k += blockDim.x) sq[k] = q[(long long)base * 10 + k];
        __syncthreads();
        for (int s = 0; s < cnt; ++s) {
            const long long* c = sq + 10 * s;
            const long long ax = c[3], ay = c[4], az = c[5];
            const long long a2 = ax * ax + ay * ay + az * az;
            const long long ro = c[6] * a2, ri = c[7] * a2, ho = c[8] * c[8] * a2, hi = c[9];
            const long long hi2 = hi * hi * a2;
#pragma unroll
            for (int t = 0; t < kVoxPerThread; ++t) {
                const long long dx = signed_image(vx[t], c[0], S), dy = signed_image(vy[t], c[1], S),
                                dz = signed_image(vz[t], c[2], S);
                const long long tt = dx * ax + dy * ay + dz * az;
                const long long rad = (dx * dx + dy * dy + dz * dz) * a2 - tt * tt;
                const long long t2 = tt * tt;
                if (hi > 0 && rad <= ri && t2 <= hi2) ph[t] = 1;
                else if (rad <= ro && t2 <= ho && ph[t] == 0) ph[t] = 2;
            }
        }
    }
#pragma unroll
    for (int t = 0; t < kVoxPerThread; ++t) {
        const long long i = first + t;
        if (i < N3) out[i] = (uint8_t)ph[t];
    }
}

void launch_voxelize_cyl(const long long* q, int n, int N, long long S, uint8_t* out, cudaStream_t st) {
    const long long N3 = (long long)N * N * N;
    const long long per = (long long)kThreads * kVoxPerThread;
    const int blocks = (int)((N3 + per - 1) / per);
    k_voxelize_cyl<<<blocks, kThreads, 0, st>>>(q, n, N, S, out);
}

void launch_voxelize(const long long* q, int n, int N, long long S, uint8_t* out, cudaStream_t st) {
    const long long N3 = (long long)N * N * N;
    const long long per = (long long)kThreads * kVoxPerThread;
    const int blocks = (int)((N3 + per - 1) / per);
    k_voxelize<<<blocks, kThreads, 0, st>>>(q, n, N, S, out);
}

}  // namespace hmg
