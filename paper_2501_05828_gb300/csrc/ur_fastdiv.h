// Unsigned 32-bit division by a divisor fixed for a kernel launch, as one multiply-high, a
// subtract and two shifts: the method of Granlund and Montgomery, "Division by invariant
// integers using multiplication" (PLDI 1994, Fig. 4.1).  For d >= 1 let l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1; then for every n < 2^32
//     q = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0),  t = floor(m n / 2^32),
// equals floor(n / d).  Plain C++ on the host (the divisor's constants) and CUDA on the device.
#ifndef UR_FASTDIV_H
#define UR_FASTDIV_H
#include <stdint.h>

#if defined(__CUDACC__)
#define UR_HD __host__ __device__
#else
#define UR_HD
#endif

namespace ur {

struct Div32 {
    uint32_t d, m, s1, s2;
};

inline Div32 make_div32(uint32_t d) {
    uint32_t l = 0;
    while (l < 32 && (1ull << l) < (uint64_t)d) ++l;
    const uint64_t m = (((uint64_t)1 << 32) * (((uint64_t)1 << l) - d)) / d + 1;
    return Div32{d, (uint32_t)m, l < 1 ? l : 1u, l > 1 ? l - 1 : 0u};
}

UR_HD inline uint32_t mulhi32(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

UR_HD inline uint32_t div32(uint32_t n, const Div32 &q) {
    const uint32_t t = mulhi32(q.m, n);
    return (t + ((n - t) >> q.s1)) >> q.s2;
}

// n / d and n % d together.
UR_HD inline uint32_t divmod32(uint32_t n, const Div32 &q, uint32_t &rem) {
    const uint32_t v = div32(n, q);
    rem = n - v * q.d;
    return v;
}

}  // namespace ur
#endif
