// Request loop behind hmg_submit / hmg_poll.
#pragma once

#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/hmg.h"
#include "hmg_runtime.h"

namespace hmg {

struct Request {
    uint64_t ticket = 0;
    std::vector<uint8_t> phase;
    int N = 0;
    double k[3] = {0, 0, 0};
    double tol = 0;
    hmg_precision prec = HMG_FP64;
    hmg_status status = HMG_PENDING;
    double K[9] = {0};
    hmg_info info{};
    double t_submit = 0, t_start = 0, t_done = 0;
    bool admitted = false;
    // RVE generated on the device at admission (hmg_submit_rve) instead of a phase grid
    int oom_retries = 0;    // admissions put back for lack of memory
    bool rve = false;
    uint64_t seed = 0;
    int n_spheres = 0;
    double radius = 0, layer = 0;
};

struct Server {
    // The loop's own context draws on `pool`, the budget of the caller's context.
    Server(int device, std::shared_ptr<BudgetPool> pool);
    ~Server();
    hmg_status submit(const uint8_t* phase, int N, const double k[3], double tol, hmg_precision p, uint64_t* ticket);
    hmg_status submit_rve(uint64_t seed, int n, double r, double layer, int N, const double k[3], double tol,
                          hmg_precision p, uint64_t* ticket);
    hmg_status poll(uint64_t ticket, double K[9], hmg_info* info);
    // counters: submitted, completed, most requests resident at once, engine ticks,
    // graph captures, graph launches
    void stats(long long out[6]);

   private:
    // lane 0: grids of at least kLargeN3 voxels (192^3 and up); lane 1: smaller grids
    static constexpr int kLanes = 2;
    static constexpr long long kLargeN3 = 192LL * 192 * 192;
    static constexpr int kOomRetries = 5000;   // ~10 s of 2 ms waits for memory to free up
    static int lane_of(int N);
    void loop(int lane);
    hmg_status enqueue(Request&& r, uint64_t* ticket);
    int device;
    std::shared_ptr<BudgetPool> pool;
    const int lane_slots[kLanes] = {1, 64};   // requests resident per lane at once
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queues[kLanes];
    std::map<uint64_t, Request> reqs;
    uint64_t next = 1;
    bool stop = false;
    std::thread workers[kLanes];
    long long resident[kLanes] = {0, 0};
    long long n_submitted = 0, n_completed = 0, max_resident = 0, n_ticks = 0, n_captures = 0, n_launches = 0;
};

}  // namespace hmg
