// Host-side parallel loops for the setup passes (CSR builds, batch layouts).
#pragma once

#include <algorithm>
#include <cstdint>
#include <thread>
#include <vector>

namespace scs {

// Threads for a host pass over `work` entries: one below 2^20, else up to 16
// (the passes are bound by memory bandwidth well before that).
inline int host_threads(int64_t work) {
    if (work < (int64_t(1) << 20)) return 1;
    const unsigned hc = std::thread::hardware_concurrency();
    return static_cast<int>(std::min<unsigned>(16, hc > 0 ? hc : 1));
}

// f(0) .. f(T - 1): part 0 on this thread, the others on new threads; a part
// whose thread cannot be started runs here after part 0.  f must not throw.
template <typename F>
void run_parts(int T, F f) {
    std::vector<std::thread> pool;
    int started = 1;
    try {
        for (; started < T; ++started) pool.emplace_back(f, started);
    } catch (...) {
        // no more threads: the remaining parts run here
    }
    f(0);
    for (int t = started; t < T; ++t) f(t);
    for (auto &th : pool) th.join();
}

// T + 1 cut points splitting items 0..n-1 with prefix weights pre[0..n]
// (pre[0] = 0, nondecreasing) into T parts of about equal weight.
inline std::vector<int32_t> weight_cuts(const int64_t *pre, int32_t n, int T) {
    std::vector<int32_t> cut(1, 0);
    for (int t = 1; t < T; ++t) {
        const int64_t target = pre[n] * t / T;
        const int32_t j = static_cast<int32_t>(std::lower_bound(pre + cut.back(), pre + n, target) - pre);
        cut.push_back(std::max(cut.back(), std::min(j, n)));
    }
    cut.push_back(n);
    return cut;
}

}  // namespace scs
