// Host-side runtime objects of libhmg (contexts, plans, solve state, solver driver).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/hmg.h"
#include "hmg_internal.h"

namespace hmg {

void set_error(const char* fmt, ...);
extern thread_local std::string g_last_error;

bool valid_length(int L);
bool valid_N(int N);
bool is_device_ptr(const void* p);
cudaError_t copy_in(void* dst_dev, const void* src, size_t bytes, cudaStream_t st);
cudaError_t copy_out(void* dst, const void* src_dev, size_t bytes, cudaStream_t st);
size_t state_bytes(int N, bool fp64, int nslots);

// Makes `dev` current for a scope and restores the caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// FFT schedules and twiddle tables of one grid size.
struct GridPlan {
    int N = 0;
    FftPlan pN{}, pM{};
    float2* tw32 = nullptr;
    double2* tw64 = nullptr;
    ~GridPlan();
};

// Device fields of one solve: tau64/spec64 (FP64 master), f32buf/r32/spec32 (FP32 bulk).
struct SolveState {
    int N = 0;
    bool fp64 = true;
    int nslots = 0;
    uint8_t* phase = nullptr;
    double* tau64 = nullptr;
    void* spec64 = nullptr;
    float* f32buf = nullptr;
    float* r32 = nullptr;
    void* spec32 = nullptr;
    double* partial = nullptr;    // FP32 sweeps (x inverse residual)
    double* partial2 = nullptr;   // equilibrium norm (z pass)
    double* partial3 = nullptr;   // FP64 work: correction sweep residual and flux average
    double* red = nullptr;   // [0,16): FP32 sweep sums, [16,32): flux sums, [32,48): eq sums,
                             // [48,56): FP64 sweep sums
    bool ensure(::hmg_ctx* c, int N, bool fp64, int nslots);
    void free_all(::hmg_ctx* c);
};

GridDesc make_desc(const GridPlan& gp, bool fp64, const double k[3], const uint8_t* phase_d, int nslots,
                   int scheme = HMG_SCHEME_EYRE_MILTON, double beta = 2.0);

// Pick the faster z-pass variant of the FP32 register-resident path for g.N by timing
// both on the state's spectrum buffer (its contents are scratch); cached per context.
int autotune_z(::hmg_ctx* c, GridDesc g, SolveState* s, cudaStream_t st);

// Per-kernel CUDA-event timing of the solver's launches.
struct Tracer {
    bool on = false;
    double ms[HMG_K_COUNT] = {0};
    long long launches[HMG_K_COUNT] = {0};
    double bytes[HMG_K_COUNT] = {0};
    struct Pending {
        int kind;
        int ev;
        double bytes;
    };
    std::vector<cudaEvent_t> events;   // pairs (start, stop)
    std::vector<int> free_pairs;
    std::vector<Pending> pending;
    int begin(cudaStream_t st);
    void end(int ev, int kind, double bytes, cudaStream_t st);
    void collect();                    // after a stream synchronize
    void reset();
    ~Tracer();
};

// FP32 sweeps of the bulk solver run in blocks of this many; the last sweep of a
// block computes the residual and the host reads it once per block.
constexpr int kResidualEvery = 4;

// Hand-over between the phases of an FP32-bulk solve (per gradient).
// The solve stops on the FP64 equilibrium test (step 1), and at the end of a correction
// solve eps_eq is a steady multiple q of eps_comp (on the 256^3 benchmark RVE q = 3 at
// contrast 10, 8 at 200, 18-20 at 2000 and 25-33 at 20000), so a correction solve stops
// once its residual is below tol / (kEqMargin q).  q starts at kEqRatio0; after an
// equilibrium test that fails it becomes the ratio that test measured, so the next
// correction solve is aimed at the tolerance instead of creeping towards it one block of
// sweeps (and two FP64 passes) at a time.
constexpr double kEqRatio0 = 20.0;
constexpr double kEqMargin = 1.25;
// The basic and relaxed schemes start from a stop at 0.1 tol.
constexpr double kEqRatio0Slow = 8.0;

// The plain FP32 sweeps of an Eyre-Milton solve hand over to the FP64 correction once their
// residual is below this (or the tolerance, if larger): above the FP32 floor of a
// contrast-2000 solve (about 1.2e-6), so no sweeps are spent on the floor waiting for the
// stall test.  The basic and relaxed schemes, whose correction solves are limited by the
// FP32 noise of their slow contraction, keep the deeper hand-over.
constexpr double kBulkExit = 3e-6;
constexpr double kBulkExitSlow = 1e-6;

// Stop of a correction solve for a gradient whose ratio eps_eq / eps_comp is taken as q.
inline double inner_target(double tol, double q) { return tol / (kEqMargin * q); }

// Driver of one solve on one SolveState.
struct Solver {
    GridDesc g;
    SolveState* s;
    cudaStream_t st;
    Tracer* tr = nullptr;
    double* psweep = nullptr;   // partial sums of sweeps (nullptr: s->partial)
    double* pflux = nullptr;    // partial sums of the flux average (nullptr: s->partial)
    // one sweep of steps 2-7; residual modes leave the per-slot sums at red[red_off + slot]
    template <typename R>
    void sweep(unsigned mask, R* field, void* spec, int zmode, int ximode, const float* r32in, float* d32,
               float* r32out, int red_off = 0);
    // Sweep b of a block of blk FP32 sweeps on f32buf / spec32 (plain: Z_ITER without r;
    // correction: Z_ITER_NOB with r added).  Where the register-resident x kernels exist
    // the sweeps of a block are chained: the x inverse of sweep b and the x forward of
    // sweep b + 1 are one kernel and the field goes to memory only before the last sweep,
    // whose x inverse computes the residual (left at red[red_off + slot]).
    void block_sweep(unsigned mask, int b, int blk, int zmode, bool addr, const float* r32in, int red_off);
    bool chained() const;
    template <typename R>
    void equilibrium(unsigned mask, const R* field, void* spec);
    template <typename R>
    bool check_eq(unsigned mask, const R* field, void* spec, double eps_eq[3], double flux[3][3]);
    bool fetch(double* h, int off, int count);
    double eps_from_sum(double sum, int slot) const;
    hmg_status run_fp64(int max_iter, double tol, hmg_info* info, double K[9]);
    hmg_status run_bulk(int max_iter, double tol, hmg_info* info, double K[9], cudaStream_t st64);
    hmg_status finish(const int status[3], const int iters[3], const int it64[3], const double eps_comp[3],
                      const double eps_eq[3], const double flux[3][3], int rounds, hmg_info* info, double K[9]);
};

struct Request;
struct Server;

// Device-memory budget of a context, shared with the request loop's internal context
// (hmg_submit) so that the two together stay within the caller's budget.
struct BudgetPool {
    size_t limit = 0;                 // 0: no limit
    std::atomic<size_t> used{0};
};

}  // namespace hmg

struct hmg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t stream64 = nullptr;   // FP64 work overlapped with the FP32 sweeps
    size_t budget = 0;                 // pool->limit
    std::shared_ptr<hmg::BudgetPool> pool;
    std::map<void*, size_t> sizes;
    std::map<int, std::shared_ptr<hmg::GridPlan>> plans;
    hmg::SolveState solve;
    std::shared_ptr<hmg::GridPlan> plan(int N);
    void* alloc(size_t bytes);
    void release(void* p);
    hmg::Server* server = nullptr;
    std::mutex server_mu;              // guards the creation of `server`
    hmg::Tracer tracer;
    std::map<int, int> ztune;   // autotuned z-pass variant per grid size (FP32 path)
};

namespace hmg {
using Context = ::hmg_ctx;
}  // namespace hmg
