// Self-check of the integer-pipe FP64 division and square root used by the
// lane-per-row dense solves of the set-up (fp64_rn.cuh) against the hardware
// IEEE operations, on operands drawn on the device from a counter-based
// generator.
#include "afsai_internal.cuh"
#include "fp64_rn.cuh"

namespace afsai {
namespace {

// splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", 2014): the finaliser of a counter
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// A finite double of random sign and significand; the biased exponent is
// drawn from [lo, lo + span).  One operand in eight gets a structured
// significand (all ones, a single bit, or a long run of ones) to reach the
// carry and boundary cases of the rounding.
__device__ __forceinline__ double draw(uint64_t r0, uint64_t r1, int lo, int span) {
    uint64_t frac = r0 & rn::kFrac;
    const uint32_t kind = static_cast<uint32_t>(r1 >> 61);
    if (kind == 0) frac = rn::kFrac;
    if (kind == 1) frac = uint64_t(1) << (r1 % 52);
    if (kind == 2) frac = rn::kFrac ^ ((uint64_t(1) << (r1 % 40)) - 1u);
    const uint64_t e = static_cast<uint64_t>(lo + static_cast<int>((r1 >> 8) % static_cast<uint64_t>(span)));
    const uint64_t sign = (r1 >> 7) & 1u;
    return rn::from_bits((sign << 63) | (e << 52) | frac);
}

__global__ void k_check_arith(int64_t n, uint64_t seed, unsigned long long* bad) {
    unsigned long long nd = 0, ns = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint64_t base = seed * 0x100000001b3ull + static_cast<uint64_t>(i) * 4u;
        const uint64_t r0 = mix64(base), r1 = mix64(base + 1), r2 = mix64(base + 2), r3 = mix64(base + 3);
        // quotients: exponents mostly near the middle (normal results), one
        // in sixteen across the whole range (subnormal and overflowing
        // results take the fallback and must still match)
        const bool wide = (r3 & 15u) == 0;
        const double a = draw(r0, r1, wide ? 1 : 900, wide ? 2046 : 250);
        const double b = draw(r2, r3, wide ? 1 : 900, wide ? 2046 : 250);
        // near-exact quotients: a2 = RN(b q) for a random q
        const double q = draw(r1 ^ r2, r0 ^ r3, 1000, 40);
        const double a2 = b * q;
        const rn::Divisor dv = rn::make_divisor(b);
        const rn::Divisor dv2 = rn::divisor_from(b, dv.v);
        if (rn::bits_of(rn::div_rn(a, dv)) != rn::bits_of(a / b)) ++nd;
        if (rn::bits_of(rn::div_rn(a2, dv2)) != rn::bits_of(a2 / b)) ++nd;
        if (rn::bits_of(rn::div_rn(1.0, dv)) != rn::bits_of(1.0 / b)) ++nd;
        if (rn::bits_of(rn::div_rn(0.0, dv)) != rn::bits_of(0.0 / b)) ++nd;
        // square roots of positive normals over the whole exponent range,
        // and of squares and their neighbours
        const double x = fabs(draw(r2 ^ r0, r1 ^ r3, 1, 2046));
        if (rn::bits_of(rn::sqrt_rn(x)) != rn::bits_of(sqrt(x))) ++ns;
        const double y = fabs(q) * fabs(q);
        const double y1 = rn::from_bits(rn::bits_of(y) + 1u), y0 = rn::from_bits(rn::bits_of(y) - 1u);
        if (rn::bits_of(rn::sqrt_rn(y)) != rn::bits_of(sqrt(y))) ++ns;
        if (rn::bits_of(rn::sqrt_rn(y1)) != rn::bits_of(sqrt(y1))) ++ns;
        if (rn::bits_of(rn::sqrt_rn(y0)) != rn::bits_of(sqrt(y0))) ++ns;
    }
    if (nd) atomicAdd(&bad[0], nd);
    if (ns) atomicAdd(&bad[1], ns);
}

}  // namespace
}  // namespace afsai

using namespace afsai;

extern "C" afsai_status afsai_check_arith(int64_t n, uint64_t seed, int64_t* mismatches, void* stream) {
    if (n < 0 || !mismatches) return fail(AFSAI_EINVAL, "invalid self-check arguments");
    auto st = static_cast<cudaStream_t>(stream);
    DevBuf<unsigned long long> bad;
    AFSAI_TRY(bad.alloc(2, st));
    AFSAI_CUDA_TRY(cudaMemsetAsync(bad.p, 0, 2 * sizeof(unsigned long long), st));
    if (n > 0) {
        const int blocks = static_cast<int>(std::min<int64_t>((n + 255) / 256, static_cast<int64_t>(num_sms()) * 16));
        k_check_arith<<<blocks, 256, 0, st>>>(n, seed, bad.p);
        AFSAI_CUDA_TRY(cudaGetLastError());
        count_launches(1);
    }
    unsigned long long h[2];
    AFSAI_CUDA_TRY(cudaMemcpyAsync(h, bad.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    AFSAI_CUDA_TRY(cudaStreamSynchronize(st));
    mismatches[0] = static_cast<int64_t>(h[0]);
    mismatches[1] = static_cast<int64_t>(h[1]);
    return AFSAI_OK;
}
