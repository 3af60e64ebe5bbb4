// Request loop behind hmg_submit / hmg_poll: two lanes (large and small grids), each a
// worker thread with its own context and streams, run the queued requests.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <memory>

#include "hmg_engine.h"
#include "hmg_runtime.h"
#include "hmg_server.h"

namespace hmg {

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

Server::Server(int dev, std::shared_ptr<BudgetPool> p) : device(dev), pool(std::move(p)) {
    for (int l = 0; l < kLanes; ++l) workers[l] = std::thread([this, l] { loop(l); });
}

Server::~Server() {
    {
        std::lock_guard<std::mutex> lk(mu);
        stop = true;
    }
    cv.notify_all();
    for (auto& w : workers)
        if (w.joinable()) w.join();
}

hmg_status Server::submit(const uint8_t* phase, int N, const double k[3], double tol, hmg_precision p,
                          uint64_t* ticket) {
    Request r;
    const size_t N3 = (size_t)N * N * N;
    r.phase.resize(N3);
    if (is_device_ptr(phase)) {
        if (cudaMemcpy(r.phase.data(), phase, N3, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            set_error("phase copy failed");
            return HMG_CUDA_ERROR;
        }
    } else {
        memcpy(r.phase.data(), phase, N3);
    }
    r.N = N;
    memcpy(r.k, k, sizeof(r.k));
    r.tol = tol;
    r.prec = p;
    return enqueue(std::move(r), ticket);
}

hmg_status Server::submit_rve(uint64_t seed, int n, double radius, double layer, int N, const double k[3], double tol,
                              hmg_precision p, uint64_t* ticket) {
    Request r;
    r.rve = true;
    r.seed = seed;
    r.n_spheres = n;
    r.radius = radius;
    r.layer = layer;
    r.N = N;
    memcpy(r.k, k, sizeof(r.k));
    r.tol = tol;
    r.prec = p;
    return enqueue(std::move(r), ticket);
}

hmg_status Server::enqueue(Request&& r, uint64_t* ticket) {
    r.t_submit = now_s();
    std::lock_guard<std::mutex> lk(mu);
    std::deque<uint64_t>& queue = queues[lane_of(r.N)];
    if (queue.size() >= 4096) {
        set_error("request queue full");
        return HMG_BUSY;
    }
    r.ticket = next++;
    *ticket = r.ticket;
    ++n_submitted;
    queue.push_back(r.ticket);
    reqs.emplace(r.ticket, std::move(r));
    cv.notify_all();
    return HMG_OK;
}

// Phase grid of a request: the caller's copy, or for an RVE request the device-generated
// one (placement + voxelization on the loop's stream) in `dev`, which the caller frees.
static hmg_status request_phase(hmg_ctx* ctx, Request* r, const uint8_t** phase, uint8_t** dev) {
    *dev = nullptr;
    if (!r->rve) {
        *phase = r->phase.data();
        return HMG_OK;
    }
    uint8_t* buf = (uint8_t*)ctx->alloc((size_t)r->N * r->N * r->N);
    if (!buf) {
        set_error("cannot allocate the RVE phase grid");
        return HMG_OUT_OF_MEMORY;
    }
    int gen = 0;
    hmg_status s = hmg_rve(ctx, r->seed, r->n_spheres, r->radius, 400000, r->layer, r->N, buf, nullptr, &gen);
    if (s != HMG_OK) {
        ctx->release(buf);
        return s;
    }
    *phase = buf;
    *dev = buf;
    return HMG_OK;
}

hmg_status Server::poll(uint64_t ticket, double K[9], hmg_info* info) {
    std::lock_guard<std::mutex> lk(mu);
    auto it = reqs.find(ticket);
    if (it == reqs.end()) {
        set_error("unknown ticket %llu", (unsigned long long)ticket);
        return HMG_UNKNOWN_TICKET;
    }
    if (it->second.status == HMG_PENDING) return HMG_PENDING;
    memcpy(K, it->second.K, sizeof(double) * 9);
    if (info) *info = it->second.info;
    hmg_status s = it->second.status;
    reqs.erase(it);
    return s;
}

// Request-loop counters (summed over the lanes).
void Server::stats(long long out[6]) {
    std::lock_guard<std::mutex> lk(mu);
    out[0] = n_submitted;
    out[1] = n_completed;
    out[2] = max_resident;
    out[3] = n_ticks;
    out[4] = n_captures;
    out[5] = n_launches;
}

int Server::lane_of(int N) { return (long long)N * N * N >= kLargeN3 ? 0 : 1; }

// One lane of the request loop.  Continuous batching: every engine tick advances all
// admitted FP32-bulk requests of the lane together; between ticks, finished requests retire
// (their device state is freed) and queued ones are admitted while their footprint fits the
// budget.  FP64 requests run one at a time with the plain method.  The lanes (large and
// small grids) run on their own threads, contexts and streams, so a small request's ticks
// do not wait for a large one's and the two lanes' kernels share the GPU; they draw on one
// budget, and a request whose state does not fit while others hold memory waits in its
// queue.  The large lane runs one request at a time, in arrival order: a single 192^3 or
// 256^3 solve already keeps HBM busy, so sharing the GPU among several would only
// stretch each one's latency; small grids gain from running together (their kernels are
// short and their fields partly fit the L2 cache).
void Server::loop(int lane) {
    hmg_ctx* ctx = nullptr;
    hmg_status cs = hmg_create(&ctx, device, pool->limit);
    std::unique_ptr<Engine> eng;
    if (cs == HMG_OK) {
        ctx->pool = pool;   // one budget for the caller's context and every lane
        cudaSetDevice(device);
        eng = std::make_unique<Engine>(ctx, ctx->stream, ctx->stream64, true);
    }
    std::deque<uint64_t>& queue = queues[lane];
    std::map<Entry*, uint64_t> running;
    bool backoff = false;
    for (;;) {
        std::vector<uint64_t> admit, fp64;
        bool waiting;
        {
            std::lock_guard<std::mutex> lk(mu);
            waiting = !queue.empty();
        }
        if (waiting && eng) eng->compact();   // retired requests' memory counts for admission
        {
            std::unique_lock<std::mutex> lk(mu);
            if (backoff && running.empty())   // waiting for memory another lane or the caller holds
                cv.wait_for(lk, std::chrono::milliseconds(2), [&] { return stop; });
            cv.wait(lk, [&] { return stop || !queue.empty() || !running.empty(); });
            if (stop) break;
            // device memory held by the caller's context and by every lane together
            size_t used = pool->used.load();
            while (!queue.empty()) {
                Request& r = reqs[queue.front()];
                if (r.prec == HMG_FP64) {
                    if (!running.empty() || !fp64.empty()) break;   // plain FP64 runs alone
                    fp64.push_back(r.ticket);
                    queue.pop_front();
                    break;
                }
                const size_t need = state_bytes(r.N, false, 3);
                if ((int)running.size() + (int)admit.size() >= lane_slots[lane]) break;
                // the first request of an idle lane is always tried (it fits the budget
                // alone by the check in hmg_submit); later ones while their footprint fits
                if ((!running.empty() || !admit.empty()) && used + need > (size_t)(0.95 * (double)pool->limit)) break;
                used += need;
                admit.push_back(r.ticket);
                queue.pop_front();
            }
            for (uint64_t t : admit) reqs[t].t_start = now_s();
            for (uint64_t t : fp64) reqs[t].t_start = now_s();
        }
        backoff = false;
        // a request that cannot get its state while others hold memory goes back to the
        // front of the queue (at most kOomRetries times, then it fails)
        auto retry = [&](Request* r, hmg_status s) {
            if (s != HMG_OUT_OF_MEMORY || ++r->oom_retries > kOomRetries) return false;
            return !running.empty() || pool->used.load() > 0;
        };
        std::vector<uint64_t> requeue;
        for (uint64_t t : fp64) {
            Request* r;
            {
                std::lock_guard<std::mutex> lk(mu);
                r = &reqs[t];
            }
            double K[9] = {0};
            hmg_info info{};
            const uint8_t* ph = nullptr;
            uint8_t* dev = nullptr;
            hmg_status s = cs != HMG_OK ? cs : request_phase(ctx, r, &ph, &dev);
            if (s == HMG_OK) s = hmg_solve(ctx, ph, r->N, r->k[0], r->k[1], r->k[2], r->tol, HMG_FP64, 0, K, &info);
            if (dev) ctx->release(dev);
            if (retry(r, s)) {
                requeue.push_back(t);
                continue;
            }
            std::lock_guard<std::mutex> lk(mu);
            r->status = s == HMG_PENDING ? HMG_CUDA_ERROR : s;
            memcpy(r->K, K, sizeof(K));
            r->info = info;
            r->t_done = now_s();
            r->info.seconds = r->t_done - r->t_submit;
            ++n_completed;
        }
        for (size_t a = 0; a < admit.size(); ++a) {
            const uint64_t t = admit[a];
            Request* r;
            {
                std::lock_guard<std::mutex> lk(mu);
                r = &reqs[t];
            }
            Entry* e = nullptr;
            const uint8_t* ph = nullptr;
            uint8_t* dev = nullptr;
            hmg_status s = cs != HMG_OK ? cs : request_phase(ctx, r, &ph, &dev);
            if (s == HMG_OK) s = eng->add((long long)t, ph, r->N, r->k, r->tol, 0, &e);
            if (dev) {   // the entry holds its own copy
                cudaStreamSynchronize(ctx->stream);
                ctx->release(dev);
            }
            if (retry(r, s)) {
                requeue.insert(requeue.end(), admit.begin() + a, admit.end());
                break;
            }
            if (s != HMG_OK) {
                std::lock_guard<std::mutex> lk(mu);
                r->status = s;
                r->t_done = now_s();
                r->info.seconds = r->t_done - r->t_submit;
                ++n_completed;
                continue;
            }
            running[e] = t;
        }
        if (!requeue.empty()) {
            std::lock_guard<std::mutex> lk(mu);
            for (auto it = requeue.rbegin(); it != requeue.rend(); ++it) queue.push_front(*it);
            backoff = true;
        }
        if (running.empty()) continue;
        {
            std::lock_guard<std::mutex> lk(mu);
            resident[lane] = (long long)running.size();
            max_resident = std::max(max_resident, resident[0] + resident[1]);
        }
        const int cap0 = eng->graph_captures;
        const long long gl0 = eng->graph_launches;
        hmg_status s = eng->tick();
        {
            std::lock_guard<std::mutex> lk(mu);
            ++n_ticks;
            n_captures += eng->graph_captures - cap0;
            n_launches += eng->graph_launches - gl0;
        }
        std::vector<Entry*> done;
        for (auto& kv : running)
            if (kv.first->finished || s != HMG_OK) done.push_back(kv.first);
        for (Entry* e : done) {
            const uint64_t t = running[e];
            {
                std::lock_guard<std::mutex> lk(mu);
                Request& r = reqs[t];
                r.status = e->finished ? e->result : s;
                memcpy(r.K, e->K, sizeof(r.K));
                r.info = e->info;
                r.t_done = now_s();
                r.info.seconds = r.t_done - r.t_submit;
                r.phase.clear();
                r.phase.shrink_to_fit();
                ++n_completed;
            }
            running.erase(e);
            eng->remove(e);
        }
        std::lock_guard<std::mutex> lk(mu);
        resident[lane] = (long long)running.size();
    }
    eng.reset();
    if (ctx) hmg_destroy(ctx);
}

}  // namespace hmg

using namespace hmg;

namespace {
// The context's request loop, started by the first submission (one loop even when
// several threads submit first at once).  Starting it releases the context's own solve
// state: the loop's requests draw on the same budget.
Server* server_of(hmg_ctx* ctx) {
    std::lock_guard<std::mutex> lk(ctx->server_mu);
    if (!ctx->server) {
        DeviceGuard dg(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        ctx->solve.free_all(ctx);
        ctx->server = new Server(ctx->device, ctx->pool);
    }
    return ctx->server;
}
}  // namespace

extern "C" {

hmg_status hmg_submit(hmg_ctx* ctx, const uint8_t* phase, int N, double km, double ki, double kc, double tol,
                      hmg_precision precision, uint64_t* ticket) {
    g_last_error.clear();
    if (!ctx || !phase || !ticket || !valid_N(N) || !(km > 0 && ki > 0 && kc > 0) || !(tol > 0) ||
        (precision != HMG_FP64 && precision != HMG_FP32_BULK)) {
        set_error("bad submit arguments");
        return HMG_INVALID_ARG;
    }
    if (state_bytes(N, precision == HMG_FP64, 3) > ctx->budget) {
        set_error("request footprint exceeds the context budget");
        return HMG_OUT_OF_MEMORY;
    }
    const double k[3] = {km, ki, kc};
    return server_of(ctx)->submit(phase, N, k, tol, precision, ticket);
}

hmg_status hmg_submit_rve(hmg_ctx* ctx, uint64_t seed, int n, double r, double layer, int N, double km, double ki,
                          double kc, double tol, hmg_precision precision, uint64_t* ticket) {
    g_last_error.clear();
    if (!ctx || !ticket || !valid_N(N) || !(km > 0 && ki > 0 && kc > 0) || !(tol > 0) ||
        (precision != HMG_FP64 && precision != HMG_FP32_BULK) || n < 1 || n > 1024 || !(r > 0.0 && r < 0.5) ||
        !(layer > 0.0 && layer < 1.0)) {
        set_error("bad submit arguments");
        return HMG_INVALID_ARG;
    }
    if (state_bytes(N, precision == HMG_FP64, 3) > ctx->budget) {
        set_error("request footprint exceeds the context budget");
        return HMG_OUT_OF_MEMORY;
    }
    const double k[3] = {km, ki, kc};
    return server_of(ctx)->submit_rve(seed, n, r, layer, N, k, tol, precision, ticket);
}

hmg_status hmg_server_stats(hmg_ctx* ctx, long long out[6]) {
    g_last_error.clear();
    if (!ctx || !out) {
        set_error("bad arguments");
        return HMG_INVALID_ARG;
    }
    for (int i = 0; i < 6; ++i) out[i] = 0;
    std::lock_guard<std::mutex> lk(ctx->server_mu);
    if (ctx->server) ctx->server->stats(out);
    return HMG_OK;
}

hmg_status hmg_poll(hmg_ctx* ctx, uint64_t ticket, double K_out[9], hmg_info* info) {
    g_last_error.clear();
    if (!ctx || !K_out) {
        set_error("bad poll arguments");
        return HMG_INVALID_ARG;
    }
    Server* srv;
    {
        std::lock_guard<std::mutex> lk(ctx->server_mu);
        srv = ctx->server;
    }
    if (!srv) {
        set_error("unknown ticket");
        return HMG_UNKNOWN_TICKET;
    }
    return srv->poll(ticket, K_out, info);
}

hmg_status hmg_solve_batch(hmg_ctx* ctx, int count, const uint8_t* const* phases, const int* N_list,
                           const double* k3, double tol, hmg_precision precision, int max_iter, double* K_out,
                           hmg_info* info) {
    g_last_error.clear();
    if (!ctx || count < 1 || !phases || !N_list || !k3 || !K_out || !(tol > 0) ||
        (precision != HMG_FP64 && precision != HMG_FP32_BULK)) {
        set_error("bad batch arguments");
        return HMG_INVALID_ARG;
    }
    for (int i = 0; i < count; ++i)
        if (!phases[i] || !valid_N(N_list[i]) || !(k3[3 * i] > 0 && k3[3 * i + 1] > 0 && k3[3 * i + 2] > 0)) {
            set_error("batch entry %d: bad phase pointer, N or conductivity", i);
            return HMG_INVALID_ARG;
        }
    hmg_status worst = HMG_OK;
    if (precision == HMG_FP64) {   // the plain method, one RVE after the other
        for (int i = 0; i < count; ++i) {
            hmg_status s = hmg_solve(ctx, phases[i], N_list[i], k3[3 * i], k3[3 * i + 1], k3[3 * i + 2], tol,
                                     precision, max_iter, K_out + 9 * i, info ? info + i : nullptr);
            if (s == HMG_INVALID_ARG || s == HMG_CUDA_ERROR || s == HMG_OUT_OF_MEMORY) return s;
            if (s != HMG_OK && worst == HMG_OK) worst = s;
        }
        return worst;
    }
    cudaSetDevice(ctx->device);
    auto t0 = now_s();
    ctx->solve.free_all(ctx);   // the engine holds its own per-RVE state
    Engine eng(ctx, ctx->stream, ctx->stream64, true);
    int next = 0;
    std::map<Entry*, int> live;
    while (next < count || !live.empty()) {
        // admit as many RVEs as fit the budget (waves when the batch is larger)
        while (next < count) {
            Entry* e = nullptr;
            hmg_status s = eng.add(next, phases[next], N_list[next], k3 + 3 * next, tol, max_iter, &e);
            if (s == HMG_OUT_OF_MEMORY && !live.empty()) break;
            if (s != HMG_OK) return s;
            live[e] = next++;
        }
        hmg_status s = eng.tick();
        if (s != HMG_OK) return s;
        std::vector<Entry*> done;
        for (auto& kv : live)
            if (kv.first->finished) done.push_back(kv.first);
        for (Entry* e : done) {
            const int i = live[e];
            memcpy(K_out + 9 * i, e->K, 9 * sizeof(double));
            if (info) {
                info[i] = e->info;
                info[i].seconds = now_s() - t0;
            }
            if (e->result != HMG_OK && worst == HMG_OK) worst = e->result;
            live.erase(e);
            eng.remove(e);
        }
    }
    return worst;
}

}  // extern "C"
