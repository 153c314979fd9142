// Portable seeded random numbers for host-side set-up (internal).
//
// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014) with its published constants, and what the
// library draws from it: uniform integers (multiply-shift range reduction of
// the top 32 bits), uniform doubles on (0, 1) from the top 53 bits, normal
// deviates by the Box-Muller transform, and a Fisher-Yates shuffle. Integer
// arithmetic and the C math library only, so a seed gives the same numbers on
// every platform (the distributions of <random> are implementation-defined).
#pragma once

#include <cmath>
#include <cstdint>
#include <utility>
#include <vector>

namespace bte {

struct SplitMix64 {
    uint64_t state;
    explicit SplitMix64(uint64_t seed) : state(seed) {}
    uint64_t next() {
        state += 0x9E3779B97F4A7C15ull;
        uint64_t z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    // integer in [0, n), n < 2^32
    uint32_t below(uint32_t n) { return (uint32_t)(((next() >> 32) * (uint64_t)n) >> 32); }
    // double in (0, 1)
    double open01() { return ((double)(next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    // standard normal deviate (Box-Muller, one of the pair)
    double normal() {
        const double u1 = open01(), u2 = open01();
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586476925 * u2);
    }
    template <class T>
    void shuffle(std::vector<T> &v) {
        for (size_t i = v.size(); i > 1; --i) std::swap(v[i - 1], v[below((uint32_t)i)]);
    }
};

}  // namespace bte
