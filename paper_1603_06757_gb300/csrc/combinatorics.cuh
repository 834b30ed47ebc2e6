// combinatorics.cuh -- combination indexing used by the enumerator, compiled for
// both the device (the kernels) and the host (diagnostic entry points that let the
// CPU test suite check exactly the code the kernels run).
#pragma once

#include <cstdint>

namespace mdist {

constexpr int kBn = 33;  // table C(a, b) for a, b <= 32, row-major, stride kBn

struct BinomTable64 {
    unsigned long long v[65][65];
};

// C(a, b) for a, b <= 64 by Pascal's rule, evaluated at compile time (each translation
// unit that needs it on the device keeps its own __constant__ copy).
constexpr BinomTable64 make_binom_table64() {
    BinomTable64 t{};
    for (int a = 0; a <= 64; ++a) {
        t.v[a][0] = 1;
        for (int b = 1; b <= a; ++b) t.v[a][b] = t.v[a - 1][b - 1] + (b <= a - 1 ? t.v[a - 1][b] : 0ull);
    }
    return t;
}

__host__ __device__ __forceinline__ int ffs32(uint32_t x) {
#ifdef __CUDA_ARCH__
    return __ffs((int)x);
#else
    return __builtin_ffs((int)x);
#endif
}

__host__ __device__ __forceinline__ int ffs64(unsigned long long x) {
#ifdef __CUDA_ARCH__
    return __ffsll((long long)x);
#else
    return __builtin_ffsll((long long)x);
#endif
}

// t-subset of {0..kh-1} with colex rank r, as a bit mask (combinatorial number
// system: the largest element is the largest c with C(c, t) <= r, and the rest is
// the (t-1)-subset of rank r - C(c, t)).  Requires r < C(kh, t), kh <= 32.
__host__ __device__ __forceinline__ uint32_t unrank_colex(const uint32_t *__restrict__ bn, int kh, int t, uint32_t r) {
    uint32_t mask = 0;
    int c = kh - 1;
    for (int i = t; i >= 1; --i) {
        while (bn[c * kBn + i] > r) --c;
        mask |= 1u << c;
        r -= bn[c * kBn + i];
        --c;
    }
    return mask;
}

// Next subset of the same size in colex order (Gosper's rule).  Only called when a
// successor exists within the half.
__host__ __device__ __forceinline__ uint32_t next_colex(uint32_t m) {
    const uint32_t u = m & (0u - m);
    const uint32_t v = m + u;
    return v | (((v ^ m) >> 2) >> (ffs32(m) - 1));
}

// Lexicographic rank of a g-subset of {0..k-1}, c_1 < ... < c_g:
// C(k,g) - 1 - sum_i C(k-1-c_i, g-i+1).  `C` maps (a, b) to C(a, b) for a, b <= 64.
#pragma nv_exec_check_disable
template <class Binom>
__host__ __device__ __forceinline__ unsigned long long lexrank64(unsigned long long mask, int k, int g, Binom C) {
    unsigned long long r = C(k, g) - 1ull;
    int i = 1;
    while (mask) {
        const int c = ffs64(mask) - 1;
        mask &= mask - 1;
        r -= C(k - 1 - c, g - i + 1);
        ++i;
    }
    return r;
}

}  // namespace mdist
