// Correctly rounded FP64 division and square root on the integer pipes.
//
// GB300 executes FP64 at 1/64 of the FP32 rate: a warp-wide IEEE FP64
// division or square root occupies the FP64 pipe for ~600-700 cycles of an
// SM sub-partition.  The lane-per-row dense solves of the stepwise set-up
// are made of such operations.  The routines below give the same IEEE results
// (round to nearest, ties to even) with 64-bit integer arithmetic, which
// issues at the integer rate:
//
//   quotient   Q = floor(X 2^53 / D) from a fixed-point reciprocal of the
//              divisor significand D (Newton-Raphson from an FP32 seed),
//              corrected with the exact remainder R = X 2^53 - Q D; the
//              result significand is Q >> 1 rounded with the last bit of Q
//              as round bit and R != 0 as sticky bit;
//   root       S = floor(sqrt(T)) from a fixed-point reciprocal square root
//              (Newton-Raphson from an FP32 seed), corrected with the exact
//              remainder R = T - S^2 (0 <= R <= 2S), rounded the same way.
//
// Both are the textbook digit-recurrence results, computed by the
// "reciprocal approximation + exact remainder correction" scheme (see
// e.g. Muller et al., Handbook of Floating-Point Arithmetic, on software
// division and square root); nothing of the CUDA math library is
// reproduced.  Operands outside the normal range, zeros of the square
// root, and results that would be subnormal or overflow take the hardware
// operation instead, so every input gives the IEEE result.
//
// A divisor used for several quotients (a column pivot of a Cholesky
// factor) is prepared once (make_divisor) and reused.
#pragma once

#include <cstdint>

namespace afsai {
namespace rn {

constexpr uint64_t kFrac = (uint64_t(1) << 52) - 1u;
constexpr uint64_t kHidden = uint64_t(1) << 52;
constexpr uint64_t kSign = uint64_t(1) << 63;

__device__ __forceinline__ uint64_t bits_of(double x) { return static_cast<uint64_t>(__double_as_longlong(x)); }
__device__ __forceinline__ double from_bits(uint64_t u) { return __longlong_as_double(static_cast<long long>(u)); }

// The hardware operations for the rare operands outside the integer path,
// kept out of line so that their code is not repeated at every call site.
static __device__ __noinline__ double hw_div(double a, double b) { return a / b; }
static __device__ __noinline__ double hw_sqrt(double x) { return sqrt(x); }

// A prepared divisor: its value, significand D in [2^52, 2^53), biased
// exponent and sign, and V ~ 2^116 / D (|V - 2^116 / D| <= 16).  D = 0
// marks a divisor the integer path does not handle (zero, subnormal,
// infinite, NaN).
struct Divisor {
    double b;
    uint64_t d;
    uint64_t v;
    int32_t e;
    uint32_t neg;
};

// V for a significand D: W ~ 2^115 / D by two Newton-Raphson steps
// W <- W + W (2^115 - D W) / 2^115 from the FP32 reciprocal of the top 24
// bits of D (relative error below 2^-22, so the steps reach the 64-bit
// truncation level); V = 2 W, saturated below 2^64.
__device__ __forceinline__ uint64_t recip116(uint64_t D) {
    const float f = static_cast<float>(static_cast<uint32_t>(D >> 29));  // exact: 24-bit integer
    const float r = __frcp_rn(f);                                          // 1 / f, rel. error <= 2^-24
    uint64_t W = __float2ull_rz(r * 77371252455336267181195264.0f);        // r * 2^86, <= 2^63
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const uint64_t plo = D * W;
        const uint64_t phi = __umul64hi(D, W);
        // E = 2^115 - D W as a two's complement pair (|E| < 2^94); Es = E >> 51
        const uint64_t elo = uint64_t(0) - plo;
        const uint64_t ehi = (uint64_t(1) << 51) - phi - (plo != 0 ? 1u : 0u);
        const int64_t es = static_cast<int64_t>((ehi << 13) | (elo >> 51));
        if (es >= 0)
            W += __umul64hi(W, static_cast<uint64_t>(es));
        else
            W -= __umul64hi(W, static_cast<uint64_t>(-es));
    }
    return W >= (uint64_t(1) << 63) ? ~uint64_t(0) : (W << 1);
}

static __device__ __noinline__ Divisor make_divisor(double b) {
    Divisor dv;
    dv.b = b;
    const uint64_t ub = bits_of(b);
    dv.neg = static_cast<uint32_t>(ub >> 63);
    dv.e = static_cast<int32_t>((ub >> 52) & 0x7ffu);
    if (dv.e == 0 || dv.e == 0x7ff) {
        dv.d = 0;
        dv.v = 0;
        return dv;
    }
    dv.d = (ub & kFrac) | kHidden;
    dv.v = recip116(dv.d);
    return dv;
}

// A divisor rebuilt from a stored value and its V (no Newton steps).
__device__ __forceinline__ Divisor divisor_from(double b, uint64_t v) {
    Divisor dv;
    dv.b = b;
    const uint64_t ub = bits_of(b);
    dv.neg = static_cast<uint32_t>(ub >> 63);
    dv.e = static_cast<int32_t>((ub >> 52) & 0x7ffu);
    const bool ok = dv.e != 0 && dv.e != 0x7ff;
    dv.d = ok ? ((ub & kFrac) | kHidden) : 0;
    dv.v = v;
    return dv;
}

// a / b, round to nearest even.
__device__ __forceinline__ double div_rn(double a, const Divisor& dv) {
    const uint64_t ua = bits_of(a);
    const uint64_t sign = (ua ^ (static_cast<uint64_t>(dv.neg) << 63)) & kSign;
    const int32_t ea = static_cast<int32_t>((ua >> 52) & 0x7ffu);
    if (dv.d != 0 && (ua << 1) == 0) return from_bits(sign);  // +-0 / finite nonzero
    if (dv.d == 0 || ea == 0 || ea == 0x7ff) return hw_div(a, dv.b);
    uint64_t X = (ua & kFrac) | kHidden;
    int32_t e = ea - dv.e + 1023;
    if (X < dv.d) {  // X / D in [1, 2)
        X <<= 1;
        e -= 1;
    }
    // Q ~ floor(X 2^53 / D) = floor(2X V / 2^64), within one unit
    uint64_t Q = __umul64hi(X << 1, dv.v);
    // exact remainder, |R| < 2^55, from the low words
    int64_t R = static_cast<int64_t>((X << 53) - Q * dv.d);
    const int64_t D = static_cast<int64_t>(dv.d);
    if (R < 0) {
        Q -= 1;
        R += D;
    }
    if (R < 0) {
        Q -= 1;
        R += D;
    }
    if (R >= D) {
        Q += 1;
        R -= D;
    }
    if (R >= D) {
        Q += 1;
        R -= D;
    }
    // Q in [2^53, 2^54): significand Q >> 1, round bit Q & 1, sticky R != 0
    uint64_t m = Q >> 1;
    const bool up = (Q & 1u) && (R != 0 || (m & 1u));
    m += up ? 1u : 0u;
    if (m == (uint64_t(1) << 53)) {
        m = kHidden;
        e += 1;
    }
    if (e <= 0 || e >= 0x7ff) return hw_div(a, dv.b);  // subnormal or overflowing result
    return from_bits(sign | (static_cast<uint64_t>(e) << 52) | (m & kFrac));
}

__device__ __forceinline__ double div_rn(double a, double b) { return div_rn(a, make_divisor(b)); }

// sqrt(x), round to nearest even.
static __device__ __noinline__ double sqrt_rn(double x) {
    const uint64_t ux = bits_of(x);
    const int32_t ex = static_cast<int32_t>((ux >> 52) & 0x7ffu);
    if ((ux >> 63) || ex == 0 || ex == 0x7ff) return hw_sqrt(x);
    uint64_t mx = (ux & kFrac) | kHidden;
    int32_t k = ex - 1075;  // x = mx 2^k
    if (k & 1) {            // even exponent: mx in [2^52, 2^54)
        mx <<= 1;
        k -= 1;
    }
    // Z ~ 2^89 / sqrt(mx) in (2^62, 2^63]: FP32 seed, two Newton-Raphson
    // steps Z <- Z + Z (1 - mx Z^2 / 2^178) / 2
    const float f = static_cast<float>(static_cast<uint32_t>(mx >> 30));  // exact: < 2^24
    uint64_t Z = __float2ull_rz(rsqrtf(f) * 18889465931478580854784.0f);  // * 2^74
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const uint64_t H = __umul64hi(Z, Z);  // ~ Z^2 / 2^64, < 2^62
        const uint64_t plo = mx * H;
        const uint64_t phi = __umul64hi(mx, H);
        // E = 2^114 - mx H (|E| < 2^93); correction Z E / 2^115 = umulhi(Z, E >> 51)
        const uint64_t elo = uint64_t(0) - plo;
        const uint64_t ehi = (uint64_t(1) << 50) - phi - (plo != 0 ? 1u : 0u);
        const int64_t es = static_cast<int64_t>((ehi << 13) | (elo >> 51));
        if (es >= 0)
            Z += __umul64hi(Z, static_cast<uint64_t>(es));
        else
            Z -= __umul64hi(Z, static_cast<uint64_t>(-es));
    }
    // S ~ floor(sqrt(mx 2^54)) = floor(mx Z / 2^62), within a few units
    uint64_t S = __umul64hi(mx << 2, Z);
    // exact remainder R = mx 2^54 - S^2 (|R| < 2^60) from the low words
    int64_t R = static_cast<int64_t>((mx << 54) - S * S);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        if (R < 0) {
            R += static_cast<int64_t>(2 * S - 1);
            S -= 1;
        }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        if (R > static_cast<int64_t>(2 * S)) {
            R -= static_cast<int64_t>(2 * S + 1);
            S += 1;
        }
    }
    // S in [2^53, 2^54)
    uint64_t m = S >> 1;
    int32_t e = (k >> 1) + 1049;
    const bool up = (S & 1u) && (R != 0 || (m & 1u));
    m += up ? 1u : 0u;
    if (m == (uint64_t(1) << 53)) {
        m = kHidden;
        e += 1;
    }
    return from_bits((static_cast<uint64_t>(e) << 52) | (m & kFrac));
}

}  // namespace rn
}  // namespace afsai
