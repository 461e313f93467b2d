// Division of unsigned integers below 2^31 by a run-time constant d >= 2 through a
// multiply-high and a shift (Granlund and Montgomery, "Division by invariant
// integers using multiplication", PLDI 1994, Sec. 4): with l = ceil(log2 d) and
// m = ceil(2^(31+l) / d) < 2^32, floor(n / d) = floor(n * m / 2^(31+l)) for every
// 0 <= n < 2^31, because 0 <= m * d - 2^(31+l) < d <= 2^l.
#pragma once
#if defined(__CUDACC__)
#define EIG_HD __host__ __device__
#else
#define EIG_HD
#endif

namespace eig {

struct FastDiv {
    unsigned m;   // magic multiplier
    unsigned sh;  // shift after the high product: l - 1
};

inline FastDiv fastdiv_make(unsigned d) {
    unsigned l = 0;
    while ((1ull << l) < d) l++;
    const unsigned long long p = 1ull << (31 + l);
    FastDiv f;
    f.m = (unsigned)((p + d - 1) / d);
    f.sh = l - 1;
    return f;
}

EIG_HD inline unsigned fastdiv(unsigned n, FastDiv f) {
#if defined(__CUDA_ARCH__)
    return __umulhi(n, f.m) >> f.sh;
#else
    return (unsigned)(((unsigned long long)n * f.m) >> 32) >> f.sh;
#endif
}

}  // namespace eig
