// muca_math.cuh - FP64 exp and natural logarithm evaluated by a fixed sequence of
// IEEE double operations, identical on the host and on the device, for the acceptance
// thresholds (Sec. 2.3), the weight recursion (Eq. (4)) and the Kullback-Leibler measure
// (Eq. (6)).  A table or weight vector computed by a kernel is then the same, bit for
// bit, as the one the host library computes.
//
// exp: Cody and Waite's argument reduction (x = k ln 2 + r, ln 2 split into a head whose
// integer multiples are exact and a tail), the Taylor series of exp(r) through r^13 / 13!
// by Horner's rule, and an exact scaling by 2^k.
// ln: x = 2^k m with m in [1/sqrt 2, sqrt 2]; ln m = 2 atanh(s) with s = (m-1)/(m+1),
// the odd series through s^23 / 23 by Horner's rule in s^2.
//
// On the device every addition, multiplication and division is an explicit
// round-to-nearest intrinsic (no contraction into fused multiply-adds); the host side is
// compiled with -ffp-contract=off.
#pragma once

#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

namespace muca {
namespace fp64 {

#if defined(__CUDA_ARCH__)
#define MUCA_FADD(a, b) __dadd_rn((a), (b))
#define MUCA_FSUB(a, b) __dsub_rn((a), (b))
#define MUCA_FMUL(a, b) __dmul_rn((a), (b))
#define MUCA_FDIV(a, b) __ddiv_rn((a), (b))
#else
#define MUCA_FADD(a, b) ((a) + (b))
#define MUCA_FSUB(a, b) ((a) - (b))
#define MUCA_FMUL(a, b) ((a) * (b))
#define MUCA_FDIV(a, b) ((a) / (b))
#endif

__host__ __device__ inline double from_bits(uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double d;
    std::memcpy(&d, &b, sizeof d);
    return d;
#endif
}

__host__ __device__ inline uint64_t to_bits(double d)
{
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(d);
#else
    uint64_t b;
    std::memcpy(&b, &d, sizeof b);
    return b;
#endif
}

// 2^k for -1022 <= k <= 1023.
__host__ __device__ inline double exp2i(int k) { return from_bits((uint64_t)(k + 1023) << 52); }

__host__ __device__ inline double exp(double x)
{
    const double ln2_head = 0x1.62e42fee00000p-1;   // ln 2 to 31 significant bits
    const double ln2_tail = 0x1.a39ef35793c76p-33;  // ln 2 - head, rounded
    const double inv_ln2 = 0x1.71547652b82fep+0;    // 1 / ln 2, rounded
    if (x != x)
        return x;
    if (x > 709.0)
        return from_bits(0x7FF0000000000000ull);
    if (x < -745.0)
        return 0.0;
    const double kd = floor(MUCA_FADD(MUCA_FMUL(x, inv_ln2), 0.5));
    const double r = MUCA_FSUB(MUCA_FSUB(x, MUCA_FMUL(kd, ln2_head)), MUCA_FMUL(kd, ln2_tail));
    // 1/n! for n = 13, 12, ..., 0, each the double nearest to it
    double p = 0x1.6124613a86d09p-33;
    p = MUCA_FADD(MUCA_FMUL(p, r), 0x1.1eed8eff8d898p-29);
    p = MUCA_FADD(MUCA_FMUL(p, r), 0x1.ae64567f544e4p-26);
    p = MUCA_FADD(MUCA_FMUL(p, r), 0x1.27e4fb7789f5cp-22);
    p = MUCA_FADD(MUCA_FMUL(p, r), 0x1.71de3a556c734p-19);
    p = MUCA_FADD(MUCA_FMUL(p, r), 0x1.a01a01a01a01ap-16);
    p = MUCA_FADD(MUCA_FMUL(p, r), 0x1.a01a01a01a01ap-13);
    p = MUCA_FADD(MUCA_FMUL(p, r), 0x1.6c16c16c16c17p-10);
    p = MUCA_FADD(MUCA_FMUL(p, r), 0x1.1111111111111p-7);
    p = MUCA_FADD(MUCA_FMUL(p, r), 0x1.5555555555555p-5);
    p = MUCA_FADD(MUCA_FMUL(p, r), 0x1.5555555555555p-3);
    p = MUCA_FADD(MUCA_FMUL(p, r), 0.5);
    p = MUCA_FADD(MUCA_FMUL(p, r), 1.0);
    p = MUCA_FADD(MUCA_FMUL(p, r), 1.0);
    const int k = (int)kd;
    const int k1 = k / 2;
    return MUCA_FMUL(MUCA_FMUL(p, exp2i(k1)), exp2i(k - k1));
}

__host__ __device__ inline double log(double x)
{
    const double ln2_head = 0x1.62e42fee00000p-1;
    const double ln2_tail = 0x1.a39ef35793c76p-33;
    const double sqrt2 = 0x1.6a09e667f3bcdp+0;
    if (x != x || x < 0.0)
        return from_bits(0x7FF8000000000000ull);
    if (x == 0.0)
        return -from_bits(0x7FF0000000000000ull);
    if (x == from_bits(0x7FF0000000000000ull))
        return x;
    int k = 0;
    uint64_t b = to_bits(x);
    if (((b >> 52) & 0x7FFu) == 0u) {   // subnormal: scale into the normal range first
        b = to_bits(MUCA_FMUL(x, exp2i(54)));
        k = -54;
    }
    k += (int)((b >> 52) & 0x7FFu) - 1023;
    double m = from_bits((b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull);
    if (m > sqrt2) {
        m = MUCA_FMUL(m, 0.5);
        k += 1;
    }
    const double s = MUCA_FDIV(MUCA_FSUB(m, 1.0), MUCA_FADD(m, 1.0));
    const double z = MUCA_FMUL(s, s);
    // 1/(2n+1) for n = 11, 10, ..., 0, each the double nearest to it
    double q = 0x1.642c8590b2164p-5;
    q = MUCA_FADD(MUCA_FMUL(q, z), 0x1.8618618618618p-5);
    q = MUCA_FADD(MUCA_FMUL(q, z), 0x1.af286bca1af28p-5);
    q = MUCA_FADD(MUCA_FMUL(q, z), 0x1.e1e1e1e1e1e1ep-5);
    q = MUCA_FADD(MUCA_FMUL(q, z), 0x1.1111111111111p-4);
    q = MUCA_FADD(MUCA_FMUL(q, z), 0x1.3b13b13b13b14p-4);
    q = MUCA_FADD(MUCA_FMUL(q, z), 0x1.745d1745d1746p-4);
    q = MUCA_FADD(MUCA_FMUL(q, z), 0x1.c71c71c71c71cp-4);
    q = MUCA_FADD(MUCA_FMUL(q, z), 0x1.2492492492492p-3);
    q = MUCA_FADD(MUCA_FMUL(q, z), 0x1.999999999999ap-3);
    q = MUCA_FADD(MUCA_FMUL(q, z), 0x1.5555555555555p-2);
    q = MUCA_FADD(MUCA_FMUL(q, z), 1.0);
    const double ln_m = MUCA_FMUL(MUCA_FADD(s, s), q);
    const double kd = (double)k;
    return MUCA_FADD(MUCA_FMUL(kd, ln2_head), MUCA_FADD(MUCA_FMUL(kd, ln2_tail), ln_m));
}

// Acceptance threshold of a move with weight change dw = ln W(e') - ln W(e): every
// move with dw >= 0 is accepted (0xFFFFFFFF), otherwise floor(exp(dw) 2^32) capped at
// 2^32 - 1 (Sec. 2.3 in integer form).
__host__ __device__ inline uint32_t threshold(double dw)
{
    if (dw >= 0.0)
        return 0xFFFFFFFFu;
    const double scaled = floor(MUCA_FMUL(exp(dw), 4294967296.0));
    return scaled >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)scaled;
}

}  // namespace fp64
}  // namespace muca
