// Split couplings (temperature-dependent Trotter coupling of the layered
// models of section 4): the acceptance thresholds the device evaluates itself.
//
// A swap of the states at temperatures k, k+1 has z = dbeta dE + dK dC (dE,
// dC the lower-temperature state's spatial energy and Trotter sum minus the
// upper one's).  Its threshold is T = min(floor(2^32 e^-z), 2^32 - 1), and
// 2^32 - 1 for z <= 0; the swap is taken iff T = 2^32 - 1 or u < T.  z is
// real-valued and too varied to tabulate, so e^-z is computed here with fixed
// FP64 operations, each rounded to nearest on its own (the _rn intrinsics
// keep the compiler from fusing them), which the host and any IEEE machine
// reproduce bit for bit:
//   * Cody & Waite's reduction (Software Manual for the Elementary Functions,
//     1980): x = n ln 2 + r, n = x / ln 2 rounded half to even, ln 2 split
//     into a head of 32 significant bits (n * head is exact) and a tail;
//   * e^r by its Taylor series to degree 13 in Horner order (the truncation,
//     below r^14 / 14! for |r| <= ln(2) / 2, is under 4e-18), the
//     coefficients 1/k! rounded to FP64;
//   * e^x = e^r 2^n, an exact scaling while the result is normal; x < -708
//     gives 0 (every threshold is 0 long before that).
// The functions also compile for the host (volatile temporaries instead of the
// intrinsics), where ising_split_exp exposes them for tests.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

namespace isg {
namespace split_detail {

__host__ __device__ __forceinline__ double mul_rn(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    volatile double r = a * b;
    return r;
#endif
}

__host__ __device__ __forceinline__ double add_rn(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dadd_rn(a, b);
#else
    volatile double r = a + b;
    return r;
#endif
}

__host__ __device__ __forceinline__ double sub_rn(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dsub_rn(a, b);
#else
    volatile double r = a - b;
    return r;
#endif
}

// 2^n for n in [-1022, 1023]: the biased exponent n + 1023 in bits 52..62
__host__ __device__ __forceinline__ double pow2i(int n)
{
    const long long bits = (long long)(n + 1023) << 52;
#ifdef __CUDA_ARCH__
    return __longlong_as_double(bits);
#else
    double d;
    std::memcpy(&d, &bits, sizeof d);
    return d;
#endif
}

__host__ __device__ __forceinline__ double exp_det(double x)
{
    // ln 2 = kLn2Hi + kLn2Lo: the head holds the first 32 significant bits
    constexpr double kInvLn2 = 0x1.71547652b82fep+0;
    constexpr double kLn2Hi = 0x1.62e42fee00000p-1;
    constexpr double kLn2Lo = 0x1.a39ef35793c76p-33;
    if (x < -708.0)
        return 0.0;
    if (x > 709.0)
        return INFINITY;
    const double n = rint(mul_rn(x, kInvLn2));
    const double r = sub_rn(sub_rn(x, mul_rn(n, kLn2Hi)), mul_rn(n, kLn2Lo));
    // 1/k!, k = 13 down to 0
    constexpr double c[14] = {0x1.6124613a86d09p-33, 0x1.1eed8eff8d898p-29, 0x1.ae64567f544e4p-26,
                              0x1.27e4fb7789f5cp-22, 0x1.71de3a556c734p-19, 0x1.a01a01a01a01ap-16,
                              0x1.a01a01a01a01ap-13, 0x1.6c16c16c16c17p-10, 0x1.1111111111111p-7,
                              0x1.5555555555555p-5,  0x1.5555555555555p-3,  0x1p-1,
                              0x1p+0,                0x1p+0};
    double p = c[0];
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
    for (int k = 1; k < 14; ++k)
        p = add_rn(mul_rn(p, r), c[k]);
    return mul_rn(p, pow2i(int(n)));  // n in [-1021, 1023]
}

// T = min(floor(2^32 p), 2^32 - 1) for a probability estimate p >= 0
__host__ __device__ __forceinline__ uint32_t threshold_of(double p)
{
    const double t = floor(mul_rn(p, 4294967296.0));
    return t >= 4294967295.0 ? 0xFFFFFFFFu : uint32_t(t);
}

// Swap threshold of pair (k, k+1); 2^32 - 1 means the swap is certain.
__host__ __device__ __forceinline__ uint32_t swap_threshold(double dbeta, double dK, long long dE,
                                                            long long dC)
{
    const double z = add_rn(mul_rn(dbeta, double(dE)), mul_rn(dK, double(dC)));
    if (z <= 0.0)
        return 0xFFFFFFFFu;
    return threshold_of(exp_det(-z));
}

}  // namespace split_detail
}  // namespace isg
