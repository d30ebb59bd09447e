// oz.cuh -- helpers of the exact-splitting (Ozaki) products: balanced digits
// of a scaled FP64 value in base 2^beta, their exact BF16 encoding, powers of
// two, and the canonical K-major layout of one 16-column operand chunk.
#pragma once

#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

// Element offset of (row, k) inside a 16-column chunk in the canonical K-major
// layout: 8 x 8 core matrices of 16-byte rows, the two core matrices of a row
// group 64 elements apart, row groups 128 elements apart.
static __host__ __device__ __forceinline__ int oz_kofs(int row, int k)
{
    return (row >> 3) * 128 + (k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}

// Balanced base-2^beta digits of I, most significant first: I = sum_s d[s] 2^(beta (S-1-s)).
static __host__ __device__ __forceinline__ int oz_digit_step(long long &I, int beta)
{
    const long long mask = (1ll << beta) - 1, half = 1ll << (beta - 1);
    long long r = I & mask;
    I >>= beta;
    if (r > half) {
        r -= (1ll << beta);
        I += 1;
    }
    return (int)r;
}

// BF16 bits of a small integer (|d| <= 256): exact.
static __host__ __device__ __forceinline__ uint16_t oz_bf16_int(int d)
{
    const float f = (float)d;
#ifdef __CUDA_ARCH__
    const uint32_t u = __float_as_uint(f);
#else
    uint32_t u;
    std::memcpy(&u, &f, 4);
#endif
    return (uint16_t)(u >> 16);
}

// 2^e as a double (normal range).
static __host__ __device__ __forceinline__ double oz_pow2(int e)
{
    const long long b = (long long)(e + 1023) << 52;
#ifdef __CUDA_ARCH__
    return __longlong_as_double(b);
#else
    double d;
    std::memcpy(&d, &b, 8);
    return d;
#endif
}

