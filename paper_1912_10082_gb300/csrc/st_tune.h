// Launch-variant tuning: for a kernel family and a problem shape, the index
// of the launch variant measured fastest on this GPU.  Host-only (no CUDA):
// the launchers consult it, st_autotune fills it, and the CPU check program
// tests the table and the selection rule.
#pragma once

#include <atomic>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <mutex>
#include <unordered_map>

namespace sttune {

// Kernel families with more than one valid launch variant for a shape.
enum Family : int {
    FOLD = 1,   // fast-diagonalisation mode product: tile edge 16, 32 or 64, or (FP32) the tensor-core tile
    LINE = 2,   // x-line tridiagonal solve: warp per row, or thread per row (64 or 16 steps a load batch)
};

struct Key {
    int family = 0, tsize = 0, a = 0, b = 0, c = 0, d = 0;
    bool operator==(const Key& o) const {
        return family == o.family && tsize == o.tsize && a == o.a && b == o.b && c == o.c && d == o.d;
    }
};

struct KeyHash {
    size_t operator()(const Key& k) const noexcept {
        uint64_t h = 1469598103934665603ull;   // FNV-1a over the six fields
        const int f[6] = {k.family, k.tsize, k.a, k.b, k.c, k.d};
        for (int v : f) {
            h ^= (uint64_t)(uint32_t)v;
            h *= 1099511628211ull;
        }
        return (size_t)h;
    }
};

// Process-wide choices, shared by every handle and thread.  Lookups skip the
// lock while the table is empty, so untuned launches pay one atomic load.
class Table {
public:
    int get(const Key& k) const {
        if (n_.load(std::memory_order_acquire) == 0) return -1;
        std::lock_guard<std::mutex> g(mu_);
        auto it = m_.find(k);
        return it == m_.end() ? -1 : it->second;
    }
    void put(const Key& k, int v) {
        std::lock_guard<std::mutex> g(mu_);
        m_[k] = v;
        n_.store((int)m_.size(), std::memory_order_release);
    }
    void clear() {
        std::lock_guard<std::mutex> g(mu_);
        m_.clear();
        n_.store(0, std::memory_order_release);
    }
    int size() const { return n_.load(std::memory_order_acquire); }
    // Calls f(key, choice) for every entry, under the lock (f must not use the table).
    template <class F>
    void for_each(F f) const {
        std::lock_guard<std::mutex> g(mu_);
        for (const auto& kv : m_) f(kv.first, kv.second);
    }

private:
    mutable std::mutex mu_;
    std::unordered_map<Key, int, KeyHash> m_;
    std::atomic<int> n_{0};
};

// Whether a stored entry can describe a launch of this library: a known
// family, element size 4 or 8, a variant index below the family's count.
inline bool plausible(const Key& k, int choice) {
    if (k.family != FOLD && k.family != LINE) return false;
    if (k.tsize != 4 && k.tsize != 8) return false;
    const int count = (k.family == FOLD && k.tsize == 4) ? 4 : 3;   // FP32 mode products: a tensor-core variant
    return choice >= 0 && choice < count;
}

inline Table& table() {
    static Table t;
    return t;
}

inline bool measured(double t) { return t >= 0.0 && std::isfinite(t); }

// Per-variant time from a rounds x n array t[r * n + c] of measurements: the
// smallest over the rounds after the first (a warm-up round, which pays for
// cold caches and first-launch costs).  A variant with any unmeasured round
// (negative: not valid for the shape) gets -1.
inline void reduce_rounds(const double* t, int rounds, int n, double* ms) {
    for (int c = 0; c < n; ++c) {
        double best = -1.0;
        bool ok = rounds > 1;
        for (int r = 1; r < rounds && ok; ++r) {
            const double v = t[(size_t)r * n + c];
            if (!measured(v)) ok = false;
            else if (best < 0.0 || v < best) best = v;
        }
        ms[c] = ok ? best : -1.0;
    }
}

// The variant to keep: the fastest measured one, unless the built-in choice
// def was measured and the fastest beats it by no more than the relative
// margin (timing noise must not move a launch off the built-in choice).
// Returns def when nothing was measured.
inline int pick(const double* ms, int n, int def, double margin) {
    int best = -1;
    for (int i = 0; i < n; ++i)
        if (measured(ms[i]) && (best < 0 || ms[i] < ms[best])) best = i;
    if (best < 0) return def;
    if (def >= 0 && def < n && measured(ms[def]) && ms[best] >= (1.0 - margin) * ms[def]) return def;
    return best;
}

}  // namespace sttune
