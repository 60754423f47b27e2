// Quotient n / d for 0 <= n < 2^31 and a divisor d fixed for a launch, by a
// multiply and a shift (Granlund and Montgomery, division by invariant
// integers using multiplication): with k = 32 + ceil(log2 d) and
// m = floor(2^k / d) + 1, the error e = m d - 2^k lies in (0, d], and
// floor(n m / 2^k) = floor(n / d) because n e <= n d < 2^31 2^ceil(log2 d) < 2^k.
// m < 2^34 and n < 2^31, so n m fits in 64 bits.  Plain C++ on the host
// (tested there) and CUDA on the device.
#pragma once

#ifdef __CUDACC__
#define DAETI_HD __host__ __device__
#else
#define DAETI_HD
#endif

namespace daeti {

struct FastDiv {
    unsigned long long m;
    int k;
};

// d >= 1
inline FastDiv fast_div(unsigned d) {
    int c = 0;
    while ((1ull << c) < d) ++c;
    FastDiv f;
    f.k = 32 + c;
    f.m = (1ull << f.k) / d + 1;
    return f;
}

DAETI_HD inline int fdiv(int n, const FastDiv& f) {
    return (int)(((unsigned long long)(unsigned)n * f.m) >> f.k);
}

}  // namespace daeti
