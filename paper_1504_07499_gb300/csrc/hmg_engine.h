// Many-RVE engine: advances a set of FP32-bulk solves together (hmg_solve_batch and the
// request loop behind hmg_submit/hmg_poll).
//
// Each engine tick runs, for every entry:
//   * FP64 defect-correction sweeps and equilibrium tests of the gradients that need
//     them (direct launches on a second stream, overlapping the FP32 block);
//   * one block of kResidualEvery FP32 sweeps for every gradient in the plain or the
//     correction phase.  Which gradients are active and which sweep form they use are
//     per-slot flags in device memory, so the block for all entries is one CUDA graph,
//     captured when the set of entries changes and replayed every tick: one graph launch
//     advances every RVE, each entry a branch of the graph.
// The host reads the per-gradient residuals once per tick and moves gradients between
// phases exactly as the single-RVE driver does.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <vector>

#include "../../include/hmg.h"
#include "hmg_internal.h"
#include "hmg_runtime.h"

namespace hmg {

struct SlotSM {
    int state = 0;
    int status = HMG_NOT_CONVERGED;
    int iters = 0, it64 = 0, since_best = 0;
    double eps_comp = INFINITY, eps_eq = INFINITY, eps32 = INFINITY, best = INFINITY, outer_eps = INFINITY;
    double flux[3] = {0, 0, 0};
    double qeq = kEqRatio0;   // the ratio eps_eq / eps_comp the correction solves aim for
};

struct Entry {
    long long id = 0;
    int N = 0;
    double k[3] = {0, 0, 0};
    double tol = 1e-8;
    int max_iter = 20000;
    std::shared_ptr<GridPlan> plan;
    SolveState st;
    GridDesc g{};
    SlotSM sm[3];
    int rounds = 0;
    int ticks = 0;
    bool finished = false;
    bool retired = false;   // removed by the caller; freed at the next compaction
    hmg_status result = HMG_PENDING;
    double K[9] = {0};
    hmg_info info{};
    int index = 0;        // position in the engine's flag and residual arrays
};

class Engine {
   public:
    // priority: of the engine's own streams (the CUDA stream priority; 0 is the default)
    Engine(hmg_ctx* ctx, cudaStream_t stream, cudaStream_t stream64, bool use_graph, int priority = 0);
    ~Engine();
    // Allocate device state for one RVE and copy its phase grid (host or device).
    hmg_status add(long long id, const uint8_t* phase, int N, const double k[3], double tol, int max_iter,
                   Entry** out);
    // Retire an entry (after its result has been read); its device state is freed at the
    // next compaction.  The entry must not be used afterwards.
    void remove(Entry* e);
    // Free the retired entries' state now.
    void compact();
    // One tick for all unfinished entries.
    hmg_status tick();
    bool idle() const;
    std::vector<std::unique_ptr<Entry>>& all() { return entries; }
    size_t bytes_in_use() const;
    int graph_captures = 0;
    long long graph_launches = 0;

   private:
    hmg_status tick_launch_and_update();
    hmg_status capture();
    void finish_entry(Entry* e);
    hmg_ctx* ctx;
    cudaStream_t st;
    cudaStream_t st64;     // FP64 work, overlapped with the FP32 block
    cudaEvent_t ready;
    bool use_graph;
    std::vector<std::unique_ptr<Entry>> entries;
    std::vector<cudaStream_t> side;
    int* dflags = nullptr;      // 4 ints per entry
    int* hflags = nullptr;      // pinned
    double* hred = nullptr;     // pinned, 64 doubles per entry (the entry's residual sums)
    int cap = 0;
    int nretired = 0;
    cudaGraphExec_t exec = nullptr;
    bool dirty = true;
    hmg_status grow(int need);
};

}  // namespace hmg
