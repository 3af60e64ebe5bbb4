// Many-RVE engine (see hmg_engine.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "hmg_engine.h"

namespace hmg {

namespace {
enum { PH_A = 0, PH_OUTER = 1, PH_EQ = 2, PH_INNER = 3, PH_DONE = 4 };
constexpr int kSideStreams = 16;
constexpr double kEta = 1e-4;       // correction sweeps reduce the FP64 residual by this factor
constexpr int kStall = 24;          // sweeps without a new best FP32 residual = FP32 floor

hmg_status cerr(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return HMG_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return HMG_CUDA_ERROR;
}
}  // namespace

Engine::Engine(hmg_ctx* c, cudaStream_t s, cudaStream_t s64, bool graph, int priority)
    : ctx(c), st(s), st64(s64), use_graph(graph) {
    cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
    for (int i = 0; i < kSideStreams; ++i) {
        cudaStream_t x;
        if (cudaStreamCreateWithPriority(&x, cudaStreamNonBlocking, priority) == cudaSuccess) side.push_back(x);
    }
}

Engine::~Engine() {
    cudaStreamSynchronize(st);
    cudaStreamSynchronize(st64);
    cudaEventDestroy(ready);
    for (auto& e : entries) e->st.free_all(ctx);
    if (exec) cudaGraphExecDestroy(exec);
    for (cudaStream_t x : side) cudaStreamDestroy(x);
    if (dflags) cudaFree(dflags);
    if (hflags) cudaFreeHost(hflags);
    if (hred) cudaFreeHost(hred);
}

hmg_status Engine::grow(int need) {
    if (need <= cap) return HMG_OK;
    int nc = std::max(need, std::max(8, 2 * cap));
    int* d = nullptr;
    int* hf = nullptr;
    double* hr = nullptr;
    if (cudaMalloc(&d, sizeof(int) * 4 * nc) != cudaSuccess || cudaMallocHost(&hf, sizeof(int) * 4 * nc) != cudaSuccess ||
        cudaMallocHost(&hr, sizeof(double) * 64 * nc) != cudaSuccess) {
        cudaGetLastError();
        if (d) cudaFree(d);
        if (hf) cudaFreeHost(hf);
        set_error("engine: cannot allocate flag arrays");
        return HMG_OUT_OF_MEMORY;
    }
    cudaStreamSynchronize(st);
    if (dflags) cudaFree(dflags);
    if (hflags) cudaFreeHost(hflags);
    if (hred) cudaFreeHost(hred);
    dflags = d;
    hflags = hf;
    hred = hr;
    cap = nc;
    dirty = true;
    return HMG_OK;
}

size_t Engine::bytes_in_use() const {
    size_t b = 0;
    for (const auto& e : entries) b += state_bytes(e->N, false, 3);
    return b;
}

bool Engine::idle() const {
    for (const auto& e : entries)
        if (!e->finished) return false;
    return true;
}

hmg_status Engine::add(long long id, const uint8_t* phase, int N, const double k[3], double tol, int max_iter,
                       Entry** out) {
    if (!valid_N(N)) {
        set_error("N = %d: need an even N = 2^a 3^b with 8 <= N <= 512", N);
        return HMG_INVALID_ARG;
    }
    compact();   // a new entry needs a new graph: free the retired ones first
    hmg_status s = grow((int)entries.size() + 1);
    if (s != HMG_OK) return s;
    auto e = std::make_unique<Entry>();
    e->id = id;
    e->N = N;
    memcpy(e->k, k, sizeof(e->k));
    e->tol = tol;
    e->max_iter = max_iter > 0 ? max_iter : 20000;
    e->plan = ctx->plan(N);
    if (!e->plan || !e->st.ensure(ctx, N, false, 3)) {
        set_error("engine: not enough device memory for an N = %d solve", N);
        return HMG_OUT_OF_MEMORY;
    }
    s = cerr(copy_in(e->st.phase, phase, (size_t)N * N * N, st), "phase copy");
    if (s != HMG_OK) {
        e->st.free_all(ctx);
        return s;
    }
    e->g = make_desc(*e->plan, false, k, e->st.phase, 3);
    {
        const int v = autotune_z(ctx, e->g, &e->st, st);
        e->g.zvar = v & 1;
        e->g.xyvar = (v >> 1) & 1;
        e->g.nochain = (v >> 2) & 1;
        e->g.xpers = (v >> 3) & 1;
        e->g.zpers = (v >> 4) & 1;
        e->g.yxy = (v >> 5) & 1;
    }
    launch_init_tau<float>(e->g, 7u, e->st.f32buf, st);
    e->index = (int)entries.size();
    if (out) *out = e.get();
    entries.push_back(std::move(e));
    dirty = true;
    return cerr(cudaGetLastError(), "engine add");
}

// A removed entry is retired: its graph branch stays (its flags are 0, so its kernels
// return at once) and its state is freed at the next compaction -- when retired entries
// are the majority, or before an entry is added (which needs a new graph anyway) -- so the
// graph is not rebuilt for every entry that finishes.
void Engine::remove(Entry* e) {
    if (e->retired) return;
    e->retired = true;
    ++nretired;
    if (2 * nretired > (int)entries.size()) compact();
}

void Engine::compact() {
    if (!nretired) return;
    cudaStreamSynchronize(st);
    cudaStreamSynchronize(st64);
    std::vector<std::unique_ptr<Entry>> keep;
    for (auto& up : entries) {
        if (up->retired) up->st.free_all(ctx);
        else keep.push_back(std::move(up));
    }
    entries = std::move(keep);
    for (size_t i = 0; i < entries.size(); ++i) entries[i]->index = (int)i;
    nretired = 0;
    dirty = true;
}

// The FP32 block of one entry: kResidualEvery sweeps under the per-slot flags, the last
// one with the residual, then the residual sums of the three gradients.
static void block_launches(const Entry* e, int* dflags, cudaStream_t s) {
    GridDesc gf = e->g;
    gf.dflags = dflags + 4 * e->index;
    SolveState st = e->st;
    if (chain_sweeps(gf)) {
        // chained sweeps: x inverse + next x forward in one kernel, the field stored only
        // before the last sweep (the residual sweep)
        // (with the plane kernel, the y inverse, x round trip and next y forward are one launch)
        const bool yxy = gf.yxy && fast_yxy_available(gf);
        launch_x_forward<float>(gf, XF_POLARIZE, 7u, st.f32buf, st.spec32, nullptr, s);
        for (int b = 0; b < kResidualEvery; ++b) {
            const bool last = b == kResidualEvery - 1;
            gf.resid = last;
            if (b == 0 || !yxy) launch_y_pass<float>(gf, true, 7u, st.spec32, s);
            launch_z_pass<float>(gf, Z_ITER, 7u, st.spec32, nullptr, s);
            if (!last && yxy) {
                fast_yxy(gf, true, b == kResidualEvery - 2, 7u, st.spec32, st.f32buf, st.r32, s);
                continue;
            }
            launch_y_pass<float>(gf, false, 7u, st.spec32, s);
            if (!last)
                fast_x_round(gf, true, b == kResidualEvery - 2, 7u, st.spec32, st.f32buf, st.r32, s);
            else
                launch_x_inverse<float>(gf, XI_ADD_R_RES, 7u, st.spec32, st.f32buf, st.r32, nullptr, nullptr,
                                        st.partial, s);
        }
        launch_reduce(st.partial, 3, x_ctas_for<float>(gf), 1, st.red, s);
        return;
    }
    for (int b = 0; b < kResidualEvery; ++b) {
        gf.resid = b == kResidualEvery - 1;
        launch_xy_forward<float>(gf, XF_POLARIZE, 7u, st.f32buf, st.spec32, nullptr, s);
        launch_z_pass<float>(gf, Z_ITER, 7u, st.spec32, nullptr, s);
        launch_yx_inverse<float>(gf, XI_ADD_R_RES, 7u, st.spec32, st.f32buf, st.r32, nullptr, nullptr, st.partial, s);
    }
    launch_reduce(st.partial, 3, x_ctas_for<float>(gf), 1, st.red, s);
}

hmg_status Engine::capture() {
    if (exec) {
        cudaGraphExecDestroy(exec);
        exec = nullptr;
    }
    cudaEvent_t fork;
    if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) return cerr(cudaGetLastError(), "event");
    std::vector<cudaEvent_t> joins(side.size());
    for (auto& j : joins) cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
    if (ce == cudaSuccess) {
        cudaEventRecord(fork, st);
        std::vector<bool> used(side.size(), false);
        for (auto& up : entries) {
            const size_t k = up->index % side.size();
            if (!used[k]) {
                cudaStreamWaitEvent(side[k], fork, 0);
                used[k] = true;
            }
            block_launches(up.get(), dflags, side[k]);
        }
        for (size_t k = 0; k < side.size(); ++k)
            if (used[k]) {
                cudaEventRecord(joins[k], side[k]);
                cudaStreamWaitEvent(st, joins[k], 0);
            }
        ce = cudaStreamEndCapture(st, &graph);
    }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaEventDestroy(fork);
    for (auto& j : joins) cudaEventDestroy(j);
    if (ce != cudaSuccess) {
        exec = nullptr;
        return cerr(ce, "graph capture");
    }
    ++graph_captures;
    dirty = false;
    return HMG_OK;
}

// One tick: the FP64 work of every entry (equilibrium tests, then defect-correction
// sweeps r = T tau64 + b - tau64) on the second stream, next to the FP32 block graph on
// the main stream; one synchronization; then every gradient moves on.
hmg_status Engine::tick_launch_and_update() {
    // per-slot flags of the FP32 block
    bool any32 = false, any64 = false;
    for (auto& up : entries) {
        Entry* e = up.get();
        int* f = hflags + 4 * e->index;
        f[3] = 0;
        for (int sl = 0; sl < 3; ++sl) {
            const int ph = e->finished ? PH_DONE : e->sm[sl].state;
            f[sl] = ph == PH_A ? (SF_ACTIVE | SF_ADDB) : ph == PH_INNER ? (SF_ACTIVE | SF_ADDR) : 0;
            any32 = any32 || f[sl] != 0;
            any64 = any64 || ph == PH_OUTER || ph == PH_EQ;
        }
    }
    // FP64 work after the main stream's pending phase transitions
    std::vector<unsigned> me(entries.size(), 0u), mo(entries.size(), 0u);
    if (any64) {
        cudaEventRecord(ready, st);
        cudaStreamWaitEvent(st64, ready, 0);
        for (auto& up : entries) {
            Entry* e = up.get();
            if (e->finished) continue;
            for (int sl = 0; sl < 3; ++sl) {
                if (e->sm[sl].state == PH_EQ) me[e->index] |= 1u << sl;
                if (e->sm[sl].state == PH_OUTER) mo[e->index] |= 1u << sl;
            }
            if (!me[e->index] && !mo[e->index]) continue;
            Solver sv{e->g, &e->st, st64, nullptr, e->st.partial3, e->st.partial3};
            if (me[e->index]) sv.equilibrium<double>(me[e->index], e->st.tau64, e->st.spec64);
            if (mo[e->index])
                sv.sweep<double>(mo[e->index], e->st.tau64, e->st.spec64, Z_ITER, XI_DIFF, nullptr, e->st.f32buf,
                                 e->st.r32, 48);
            cudaMemcpyAsync(hred + 64 * e->index + 16, e->st.red + 16, 40 * sizeof(double), cudaMemcpyDeviceToHost,
                            st64);
        }
    }
    if (any32) {
        hmg_status s = cerr(cudaMemcpyAsync(dflags, hflags, sizeof(int) * 4 * entries.size(), cudaMemcpyHostToDevice, st),
                            "flags");
        if (s != HMG_OK) return s;
        if (use_graph) {
            if (dirty || !exec) {
                s = capture();
                if (s != HMG_OK) return s;
            }
            s = cerr(cudaGraphLaunch(exec, st), "graph launch");
            if (s != HMG_OK) return s;
            ++graph_launches;
        } else {
            for (auto& up : entries) block_launches(up.get(), dflags, st);
        }
        for (auto& up : entries)
            cudaMemcpyAsync(hred + 64 * up->index, up->st.red, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
    }
    hmg_status s = cerr(cudaStreamSynchronize(st), "FP32 block");
    if (s == HMG_OK) s = cerr(cudaStreamSynchronize(st64), "FP64 work");
    if (s != HMG_OK) return s;
    bool pers = false;
    for (auto& up : entries) pers = pers || up->g.xpers || up->g.zpers;
    if (any32 && pers && fast_take_wait_failure()) {
        set_error("a persistent kernel gave up waiting for its bulk copies; results are invalid");
        return HMG_CUDA_ERROR;
    }
    for (auto& up : entries) {
        Entry* e = up.get();
        if (e->finished) continue;
        const double* h = hred + 64 * e->index;
        Solver sv{e->g, &e->st, st, nullptr};
        for (int sl = 0; sl < 3; ++sl) {
            SlotSM& m = e->sm[sl];
            if ((me[e->index] >> sl) & 1u) {   // equilibrium test of the FP64 master field
                double nrm = 0.0;
                for (int c = 0; c < 3; ++c) {
                    m.flux[c] = h[16 + sl * 3 + c] / (double)e->g.N3;
                    nrm += m.flux[c] * m.flux[c];
                }
                m.eps_eq = std::sqrt(h[32 + sl]) / std::sqrt(nrm);
                if (m.eps_eq < e->tol) {
                    m.status = HMG_OK;
                    m.state = PH_DONE;
                } else {
                    if (m.eps_comp > 0.0) m.qeq = std::max(m.qeq, m.eps_eq / m.eps_comp);
                    m.state = PH_INNER;
                    m.best = INFINITY;
                    m.since_best = 0;
                    ++e->rounds;
                }
            }
            if ((mo[e->index] >> sl) & 1u) {   // FP64 correction sweep
                ++m.iters;
                ++m.it64;
                m.eps_comp = sv.eps_from_sum(h[48 + sl], sl);
                m.outer_eps = m.eps_comp;
                if (!std::isfinite(m.eps_comp)) {
                    m.status = HMG_DIVERGED;
                    m.state = PH_DONE;
                } else if (m.eps_comp < e->tol) {
                    m.state = PH_EQ;
                } else {
                    m.state = PH_INNER;
                    m.best = INFINITY;
                    m.since_best = 0;
                    ++e->rounds;
                }
            }
        }
        unsigned to_a = 0, to_i = 0;
        for (int sl = 0; sl < 3; ++sl) {
            SlotSM& m = e->sm[sl];
            const int fl = hflags[4 * e->index + sl];
            if (!fl) continue;
            m.iters += kResidualEvery;
            m.eps32 = sv.eps_from_sum(h[sl], sl);
            if (!std::isfinite(m.eps32)) {
                m.status = HMG_DIVERGED;
                m.state = PH_DONE;
                continue;
            }
            if (m.eps32 < m.best * 0.999) {
                m.best = m.eps32;
                m.since_best = 0;
            } else {
                m.since_best += kResidualEvery;
            }
            if (fl & SF_ADDB) {   // plain phase
                m.eps_comp = m.eps32;
                if (m.eps32 < std::max(e->tol, kBulkExit) || m.since_best >= kStall) to_a |= 1u << sl;
            } else if (m.eps32 < std::max(kEta * m.outer_eps, inner_target(e->tol, m.qeq)) || m.since_best >= kStall) {
                to_i |= 1u << sl;
            }
        }
        if (to_a) launch_widen(e->g, to_a, e->st.f32buf, e->st.tau64, st);
        if (to_i) launch_axpy(e->g, to_i, e->st.f32buf, e->st.tau64, st);
        for (int sl = 0; sl < 3; ++sl)
            if (((to_a | to_i) >> sl) & 1u) e->sm[sl].state = PH_OUTER;
    }
    return HMG_OK;
}

void Engine::finish_entry(Entry* e) {
    Solver sv{e->g, &e->st, st, nullptr};
    unsigned left = 0;
    for (int sl = 0; sl < 3; ++sl) {
        SlotSM& m = e->sm[sl];
        if (m.status == HMG_NOT_CONVERGED) {
            if (m.state == PH_A) launch_widen(e->g, 1u << sl, e->st.f32buf, e->st.tau64, st);
            if (m.state == PH_INNER) launch_axpy(e->g, 1u << sl, e->st.f32buf, e->st.tau64, st);
            left |= 1u << sl;
        }
    }
    if (left) {
        double eps[3], flux[3][3];
        if (sv.check_eq<double>(left, e->st.tau64, e->st.spec64, eps, flux)) {
            for (int sl = 0; sl < 3; ++sl)
                if ((left >> sl) & 1u) {
                    e->sm[sl].eps_eq = eps[sl];
                    memcpy(e->sm[sl].flux, flux[sl], sizeof(flux[sl]));
                }
        } else {
            for (int sl = 0; sl < 3; ++sl) e->sm[sl].status = HMG_CUDA_ERROR;
        }
    }
    int st3[3], it[3], i64[3];
    double ec[3], ee[3], fl[3][3];
    for (int sl = 0; sl < 3; ++sl) {
        st3[sl] = e->sm[sl].status;
        it[sl] = e->sm[sl].iters;
        i64[sl] = e->sm[sl].it64;
        ec[sl] = e->sm[sl].eps_comp;
        ee[sl] = e->sm[sl].eps_eq;
        memcpy(fl[sl], e->sm[sl].flux, sizeof(fl[sl]));
    }
    e->result = sv.finish(st3, it, i64, ec, ee, fl, e->rounds, &e->info, e->K);
    e->finished = true;   // its graph branch stays (flags 0) until the entry is removed
}

hmg_status Engine::tick() {
    hmg_status s = tick_launch_and_update();
    if (s != HMG_OK) return s;
    for (auto& up : entries) {
        Entry* e = up.get();
        if (e->finished) continue;
        ++e->ticks;
        bool all_done = true;
        for (int sl = 0; sl < 3; ++sl) {
            SlotSM& m = e->sm[sl];
            if (m.state != PH_DONE && m.iters >= e->max_iter) m.state = PH_DONE;   // status stays NOT_CONVERGED
            all_done = all_done && m.state == PH_DONE;
        }
        if (all_done) finish_entry(e);
    }
    return cerr(cudaGetLastError(), "engine tick");
}

}  // namespace hmg
