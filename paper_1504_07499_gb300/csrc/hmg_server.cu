// Request loop behind hmg_submit / hmg_poll: a worker thread with its own context
// runs queued requests.
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>

#include "hmg_runtime.h"
#include "hmg_server.h"

namespace hmg {

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

Server::Server(int dev, size_t bud) : device(dev), budget(bud) { worker = std::thread([this] { loop(); }); }

Server::~Server() {
    {
        std::lock_guard<std::mutex> lk(mu);
        stop = true;
    }
    cv.notify_all();
    if (worker.joinable()) worker.join();
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
    r.t_submit = now_s();
    std::lock_guard<std::mutex> lk(mu);
    if (queue.size() >= 4096) {
        set_error("request queue full");
        return HMG_BUSY;
    }
    r.ticket = next++;
    *ticket = r.ticket;
    queue.push_back(r.ticket);
    reqs.emplace(r.ticket, std::move(r));
    cv.notify_all();
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

void Server::loop() {
    hmg_ctx* ctx = nullptr;
    hmg_status cs = hmg_create(&ctx, device, budget);
    for (;;) {
        uint64_t t;
        Request* r;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait(lk, [this] { return stop || !queue.empty(); });
            if (stop) break;
            t = queue.front();
            queue.pop_front();
            r = &reqs[t];
            r->t_start = now_s();
        }
        double K[9] = {0};
        hmg_info info{};
        hmg_status s = cs != HMG_OK ? cs
                                    : hmg_solve(ctx, r->phase.data(), r->N, r->k[0], r->k[1], r->k[2], r->tol, r->prec,
                                                0, K, &info);
        std::lock_guard<std::mutex> lk(mu);
        r->status = s == HMG_PENDING ? HMG_CUDA_ERROR : s;
        memcpy(r->K, K, sizeof(K));
        r->info = info;
        r->t_done = now_s();
        r->info.seconds = r->t_done - r->t_submit;
    }
    if (ctx) hmg_destroy(ctx);
}

}  // namespace hmg

using namespace hmg;

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
    if (!ctx->server) ctx->server = new Server(ctx->device, ctx->budget);
    const double k[3] = {km, ki, kc};
    return ctx->server->submit(phase, N, k, tol, precision, ticket);
}

hmg_status hmg_poll(hmg_ctx* ctx, uint64_t ticket, double K_out[9], hmg_info* info) {
    g_last_error.clear();
    if (!ctx || !K_out) {
        set_error("bad poll arguments");
        return HMG_INVALID_ARG;
    }
    if (!ctx->server) {
        set_error("unknown ticket");
        return HMG_UNKNOWN_TICKET;
    }
    return ctx->server->poll(ticket, K_out, info);
}

hmg_status hmg_solve_batch(hmg_ctx* ctx, int count, const uint8_t* const* phases, const int* N_list,
                           const double* k3, double tol, hmg_precision precision, int max_iter, double* K_out,
                           hmg_info* info) {
    g_last_error.clear();
    if (!ctx || count < 1 || !phases || !N_list || !k3 || !K_out) {
        set_error("bad batch arguments");
        return HMG_INVALID_ARG;
    }
    hmg_status worst = HMG_OK;
    for (int i = 0; i < count; ++i) {
        hmg_status s = hmg_solve(ctx, phases[i], N_list[i], k3[3 * i], k3[3 * i + 1], k3[3 * i + 2], tol, precision,
                                 max_iter, K_out + 9 * i, info ? info + i : nullptr);
        if (s == HMG_INVALID_ARG || s == HMG_CUDA_ERROR || s == HMG_OUT_OF_MEMORY) return s;
        if (s != HMG_OK && worst == HMG_OK) worst = s;
    }
    return worst;
}

}  // extern "C"
