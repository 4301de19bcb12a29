// Exact float -> double widening with integer operations, for kernels on GPUs whose FP64
// pipe is narrow: a normal float's exponent is rebiased by 1023 - 127 = 896 and its
// 23-bit fraction moves up 29 bits; signed zeros map to signed zeros.  Subnormal,
// infinite and NaN inputs return 0 and take the hardware conversion.  Host and
// device code share this header (the host side is checked over every float pattern).
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define TN_HD __host__ __device__ __forceinline__
#else
#define TN_HD static inline
#endif

TN_HD int tn_widen_bits(uint32_t u, uint64_t *d) {
    const uint32_t e = (u >> 23) & 0xFFu;
    const uint64_t sign = (uint64_t)(u >> 31) << 63;
    if (e == 0u) {
        if (u & 0x7FFFFFu) return 0;
        *d = sign;
        return 1;
    }
    if (e == 0xFFu) return 0;
    *d = sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29);
    return 1;
}

#ifdef __CUDACC__
__device__ __forceinline__ double tn_widen(float x) {
    uint64_t d;
    if (tn_widen_bits(__float_as_uint(x), &d)) return __longlong_as_double((long long)d);
    return (double)x;
}
#endif
