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


// ---------------------------------------------------------------------------
// Integer-pipe versions of the two conversions around the digit products, so
// that they leave the FP64 pipe free (results bit for bit those of the FP64
// instructions they replace).

// round-half-even(v 2^k) for finite v with |v 2^k| < 2^62: the value of
// __double2ll_rn(v * 2^k) (the product being exact), from v's bit pattern.
static __host__ __device__ __forceinline__ long long oz_rint_pow2(double v, int k)
{
#ifdef __CUDA_ARCH__
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
#else
    unsigned long long b;
    std::memcpy(&b, &v, 8);
#endif
    const int e = (int)((b >> 52) & 0x7ffull);
    if (e == 0) return 0;  // zero or subnormal: far below 1/2 after any scale used here
    const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);  // v = m 2^(e - 1075)
    const int s = e - 1075 + k;
    long long r;
    if (s >= 0) {
        r = m << s;
    } else if (s < -53) {
        r = 0;  // m 2^s < 1/2
    } else {
        const int sh = -s;
        r = m >> sh;
        const long long rem = m & ((1ll << sh) - 1), half = 1ll << (sh - 1);
        if (rem > half || (rem == half && (r & 1))) r += 1;
    }
    return (b >> 63) ? -r : r;
}

// The double nearest (ties to even) to (hi 2^32 + lo) 2^p, for |hi| < 2^62,
// |lo| < 2^62 and a result in the normal range: the value of
// fma((double)hi, 2^32, (double)lo) * 2^p (one rounding, an exact power-of-two
// scale), built from the integer bits.
static __host__ __device__ __forceinline__ double oz_i64x2_scaled(long long hi, long long lo, int p)
{
    // X = hi 2^32 + lo, |X| < 2^95, as a sign and a magnitude of at most 95 bits
    const __int128 X = (__int128)hi * ((__int128)1 << 32) + (__int128)lo;
    if (X == 0) return 0.0;
    const bool neg = X < 0;
    const unsigned __int128 u = neg ? (unsigned __int128)(-X) : (unsigned __int128)X;
    const unsigned long long uh = (unsigned long long)(u >> 64), ul = (unsigned long long)u;
#ifdef __CUDA_ARCH__
    const int lz = uh ? __clzll((long long)uh) : 64 + __clzll((long long)ul);
#else
    const int lz = uh ? __builtin_clzll(uh) : 64 + __builtin_clzll(ul);
#endif
    const int nb = 128 - lz;  // bits of |X|
    unsigned long long m;
    int e2;  // |X| rounded = m 2^e2, 2^52 <= m < 2^53
    if (nb <= 53) {
        m = ul << (53 - nb);
        e2 = nb - 53;
    } else {
        int sh = nb - 53;
        const unsigned __int128 one = 1;
        m = (unsigned long long)(u >> sh);
        const unsigned __int128 rem = u & ((one << sh) - 1), half = one << (sh - 1);
        if (rem > half || (rem == half && (m & 1ull))) m += 1;
        if (m == (1ull << 53)) {
            m >>= 1;
            sh += 1;
        }
        e2 = sh;
    }
    unsigned long long bits = ((unsigned long long)(e2 + p + 52 + 1023) << 52) | (m & 0xFFFFFFFFFFFFFull);
    if (neg) bits |= 1ull << 63;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)bits);
#else
    double d;
    std::memcpy(&d, &bits, 8);
    return d;
#endif
}
