// Internal declarations shared by the libhmg translation units (host + device).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace hmg {

constexpr int kThreads = 256;      // threads per CTA in every FFT pass
constexpr int kMaxStages = 12;     // radix stages per 1D transform
constexpr int kMaxSlots = 3;       // right-hand sides (unit gradients) per RVE

// Mixed-radix Stockham schedule of one 1D length (radices 2, 3, 4, 8).
struct FftPlan {
    int L;                 // transform length
    int nst;               // number of stages
    int rad[kMaxStages];   // radix of each stage, first stage first
    int tw_off;            // offset of the length-L twiddle table exp(-2 pi i k / L)
};

// Everything a pass kernel needs about one RVE: sizes, FFT schedules, the
// per-phase coefficient table, and the device fields (FP32 or FP64 copies).
struct GridDesc {
    int N, M;              // grid size and N/2 (complex length of an x row)
    long long NN, N3;      // N*N and N^3
    long long NNM;         // complex entries per component spectrum: N*N*M
    FftPlan pN, pM;        // schedules for lengths N (y, z) and M (x)
    const float2* tw32;    // twiddle tables (all lengths, concatenated)
    const double2* tw64;
    // per-phase coefficients, k0 = sqrt(min k * max k):
    double Y[3];           // (k - k0)/(k + k0): polarization factor of the sweep
    double W[3];           // k/(k + k0): flux factor, phi = W tau
    double KP[3];          // k + k0: tau = (k + k0) e
    double k0;
    // Scheme (hmg_scheme) and its Green step s <- scale (ga s - gb P s) + gc E at the DC
    // mode; the sweep residual |e^n - e_comp^n| is epsf |field^n - field^{n+1}|.
    // Eyre-Milton (tau form): ga = 1, gb = 2, gc = 2 k0, epsf = 1 / (2 k0);
    // basic scheme (field e, Y = (k - k0) / k0, W = k, KP = 1): ga = 0, gb = 1, gc = 1, epsf = 1.
    int scheme;
    double ga, gb, gc, epsf;
    // Relaxed schemes of the Eyre-Milton family (augmented Lagrangian, polarization
    // family with relaxation beta): the x inverse keeps this fraction of the old field,
    // field^{n+1} = (1 - relax) T(field^n) + relax field^n, relax = 1 - beta / 2
    // (0: no relaxation; the sweep is then the plain map T).
    double relax;
    double E[kMaxSlots][3];  // macroscopic gradient of each right-hand side
    int nslots;            // right-hand sides held in the fields
    int rows;              // x-pass rows per CTA
    int Py, Pz;            // columns per CTA in the y and z passes
    int zvar;              // z-pass kernel variant of the register-resident path (autotuned)
    int xyvar;             // 1: fused x + y cluster kernels, 0: separate x and y passes (autotuned)
    int nochain;           // 1: FP32 sweeps of a block are not chained through k_fx_round
    int xpers;             // 1: the chained x round trip runs as a persistent kernel that
                           //    stages its next rows with bulk copies (autotuned)
    int yxy;               // 1: the chained sweeps' y inverse, x round trip and y forward run
                           //    as one persistent kernel per (component, z) plane (autotuned)
    int zpers;             // 1: the z pass of plain and correction sweeps runs as a
                           //    persistent kernel that stages its next columns with tiled
                           //    tensor copies (autotuned)
    // Per-slot flags in device memory (engine launches; nullptr = use the launch's
    // mask and template modes): SF_ACTIVE, SF_ADDB (add gc E at DC, plain sweep),
    // SF_ADDR (add the defect r, correction sweep).  `resid`: this launch of the x
    // inverse also reads the old field and sums the residual (flags mode only).
    const int* dflags;
    int resid;
    const uint8_t* phase;  // N^3 phase ids
};

enum SlotFlags { SF_ACTIVE = 1, SF_ADDB = 2, SF_ADDR = 4 };

#ifdef __CUDACC__
__device__ __forceinline__ bool slot_active(const GridDesc& g, unsigned mask, int slot) {
    return g.dflags ? (g.dflags[slot] & SF_ACTIVE) != 0 : ((mask >> slot) & 1u) != 0;
}
#endif

enum XFwdMode { XF_PLAIN = 0, XF_POLARIZE = 1, XF_FLUX = 2 };
enum XInvMode { XI_PLAIN = 0, XI_INPLACE = 1, XI_INPLACE_RES = 2, XI_ADD_R_RES = 3, XI_DIFF = 4, XI_ADD_R = 5 };
enum ZMode { Z_FWD = 0, Z_INV = 1, Z_ITER = 2, Z_ITER_NOB = 3, Z_EQ = 4 };

// Launch wrappers (hmg_kernels.cu).  `mask` selects the active right-hand sides;
// CTAs of inactive ones exit at once.  Partial-sum buffers receive one double per
// CTA and right-hand side (layout [slot][cta]).
template <typename R>
void launch_x_forward(const GridDesc& g, int mode, unsigned mask, const R* tau,
                      void* spec, double* partial, cudaStream_t st);
template <typename R>
void launch_y_pass(const GridDesc& g, bool forward, unsigned mask, void* spec, cudaStream_t st);
template <typename R>
void launch_z_pass(const GridDesc& g, int mode, unsigned mask, void* spec, double* partial,
                   cudaStream_t st);
// x inverse: writes tau (INPLACE*), adds r (ADD_R, ADD_R_RES), or writes d = new - old to
// d32 and r32 without touching tau (DIFF).  Residual modes add (new-old)^2 per CTA.
template <typename R>
void launch_x_inverse(const GridDesc& g, int mode, unsigned mask, const void* spec, R* tau,
                      const float* r32, float* d32, float* r32_out, double* partial,
                      cudaStream_t st);

// Tile sizes of the generic shared-memory passes (x rows per CTA, y and z columns per CTA)
// for FP32 or FP64 elements.  FP64 launches always take the FP64 tiles, whatever the
// descriptor says (the FP32-bulk solver runs its FP64 work on its FP32 descriptor).
void set_tiles(GridDesc& g, bool fp64);
int x_ctas(const GridDesc& g);   // CTAs per right-hand side of the generic x passes
int z_ctas(const GridDesc& g);   // CTAs per right-hand side of the generic z pass
// CTAs per right-hand side of the x / z passes that launch_* runs for precision R
// (the register-resident FP32 kernels where one exists, else the generic ones)
template <typename R> int x_ctas_for(const GridDesc& g);
template <typename R> int z_ctas_for(const GridDesc& g);

// Register-resident FP32 kernels (hmg_fast.cu); each returns false (launching
// nothing) when no specialization covers the grid size.
bool fast_y(const GridDesc& g, bool fwd, unsigned mask, void* spec, cudaStream_t st);
bool fast_z(const GridDesc& g, int mode, unsigned mask, void* spec, double* partial, cudaStream_t st);
bool fast_x_forward(const GridDesc& g, int mode, unsigned mask, const float* tau, void* spec, double* partial,
                    cudaStream_t st);
bool fast_x_inverse(const GridDesc& g, int mode, unsigned mask, const void* spec, float* tau, const float* r32,
                    double* partial, cudaStream_t st);
// x inverse of a sweep + polarization and x forward of the next, in place on the
// spectrum; adds r (addr; per-slot flag in flags mode) and stores the updated field (wtau).
bool fast_x_round(const GridDesc& g, bool addr, bool wtau, unsigned mask, void* spec, float* tau, const float* r32,
                  cudaStream_t st);
// FP32 sweeps of a block are chained (x inverse + next x forward in one kernel):
// register-resident x kernels exist for g.N, separate x and y passes, chaining not off.
bool chain_sweeps(const GridDesc& g);
// y inverse + x round trip + y forward of each plane in one persistent kernel (sizes 64,
// 128, 192, 256; not for relaxed schemes); false when it does not apply.
bool fast_yxy_available(const GridDesc& g);
bool fast_yxy(const GridDesc& g, bool addr, bool wtau, unsigned mask, void* spec, float* tau, const float* r32,
              cudaStream_t st);
// True (and cleared) when a persistent kernel's bounded wait for a bulk copy gave up
// since the last call; the results of that launch are invalid.
bool fast_take_wait_failure();
int fast_x_ctas(const GridDesc& g);
int fast_z_ctas(const GridDesc& g);

// Fused x + y passes on thread-block clusters (hmg_fused.cu, FP32); false / 0 when the
// grid size has no fused kernels.
int fused_cluster(int N);
int fused_xy_ctas(const GridDesc& g);
bool fused_xy_forward(const GridDesc& g, int mode, unsigned mask, const float* tau, void* spec, double* partial,
                      cudaStream_t st);
bool fused_yx_inverse(const GridDesc& g, int mode, unsigned mask, const void* spec, float* tau, const float* r32,
                      double* partial, cudaStream_t st);

// x then y forward (one fused launch where available), and y then x inverse.
// Return true when the fused kernels ran.
template <typename R>
bool launch_xy_forward(const GridDesc& g, int mode, unsigned mask, const R* tau, void* spec, double* partial,
                       cudaStream_t st);
template <typename R>
bool launch_yx_inverse(const GridDesc& g, int mode, unsigned mask, const void* spec, R* tau, const float* r32,
                       float* d32, float* r32_out, double* partial, cudaStream_t st);

// Sum `count` partials of each of `nslots` rows in a fixed order: out[s] = sum_i p[s*count+i].
// `groups` > 1 splits each row into that many equal consecutive groups (out[s*groups+g]).
void launch_reduce(const double* partial, int nslots, int count, int groups, double* out,
                   cudaStream_t st);

// Pointwise helpers on the fields.
template <typename R>
void launch_init_tau(const GridDesc& g, unsigned mask, R* tau, cudaStream_t st);
template <typename R>
void launch_e_to_tau(const GridDesc& g, int slot, const double* e, R* tau, cudaStream_t st);
template <typename R>
void launch_tau_to_e(const GridDesc& g, int slot, const R* tau, double* e, cudaStream_t st);
void launch_widen(const GridDesc& g, unsigned mask, const float* src, double* dst, cudaStream_t st);
void launch_axpy(const GridDesc& g, unsigned mask, const float* d, double* tau, cudaStream_t st);
template <typename R>
void launch_convert(const double* src, R* dst, long long n, cudaStream_t st);
template <typename R>
void launch_convert_back(const R* src, double* dst, long long n, cudaStream_t st);

// Voxelization (hmg_voxelize.cu): q holds n quantized spheres (cx, cy, cz, R_out^2, R_in^2).
void launch_voxelize(const long long* q, int n, int N, long long S, uint8_t* out, cudaStream_t st);
// Coated cylinders merged into a phase grid (q: 10 integers per cylinder, GC = 256 units).
void launch_voxelize_cyl(const long long* q, int n, int N, long long S, uint8_t* out, cudaStream_t st);

}  // namespace hmg
