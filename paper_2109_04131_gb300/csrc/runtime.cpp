// Concurrent increments of independent plans (the batched form): one increment of each of
// `count` plans, the host planning of the plans in parallel threads and their device work
// overlapping on the plans' own streams.  Plans share nothing, so each result is the one the
// plan gives alone.
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "usfft.h"

extern "C" usfft_status usfft_increment_many(usfft_plan_t* const* plans, int count, int max_threads,
                                             usfft_increment_info* infos, usfft_status* statuses) {
    if (count < 0 || (count > 0 && (!plans || !statuses))) return USFFT_EINVAL;
    for (int k = 0; k < count; ++k)
        if (!plans[k]) return USFFT_EINVAL;
    for (int k = 0; k < count; ++k)
        for (int q = k + 1; q < count; ++q)
            if (plans[k] == plans[q]) return USFFT_EINVAL;      // a plan is not thread-safe
    int hw = (int)std::thread::hardware_concurrency();
    if (hw < 1) hw = 1;
    int nt = max_threads > 0 ? max_threads : hw;
    nt = std::min(nt, count);
    std::atomic<int> next(0);
    auto worker = [&]() {
        for (;;) {
            const int k = next.fetch_add(1);
            if (k >= count) return;
            statuses[k] = usfft_increment(plans[k], infos ? infos + k : nullptr);
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
    if (nt >= 1) worker();
    for (auto& th : pool) th.join();
    usfft_status first = USFFT_OK;
    for (int k = 0; k < count && first == USFFT_OK; ++k) first = statuses[k];
    return first;
}
