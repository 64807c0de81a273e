// philox.cuh -- inline counter-based noise for the step kernels.
//
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the
// constants 0xD2511F53 / 0xCD9E8D57 and a Weyl-sequence key schedule
// (+0x9E3779B9, +0xBB67AE85 per round).  Box & Muller (1958) turns the four
// 32-bit words of one block into four N(0,1) deviates (both the cosine and
// the sine branch of each pair).  The paper draws iid N(0,1) per face and step
// (Sec. 3, Eq. (3.7)); the counter layout that addresses a face is fixed in
// she.h.  Nothing here is ever written to device memory: each step kernel
// regenerates the deviates it needs in registers.
#pragma once
#include <cstdint>

namespace she {

constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;   // Weyl increments of the key schedule
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// The ten round keys of one key (k0 + i W0, k1 + i W1, i = 0..9), filled on
// the host and passed inside a __grid_constant__ kernel parameter, so that
// every round reads its key as a constant operand instead of re-deriving it.
struct RoundKeys {
    uint32_t k0[10];
    uint32_t k1[10];
};

inline RoundKeys make_round_keys(uint64_t seed)
{
    RoundKeys rk;
    uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
    for (int i = 0; i < 10; ++i) {
        rk.k0[i] = k0;
        rk.k1[i] = k1;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return rk;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const RoundKeys& rk)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c.x;   // 32x32 -> 64
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk.k0[round], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ rk.k1[round], (uint32_t)p0);
    }
    return c;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c.x;   // 32x32 -> 64
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return c;
}

// B independent blocks at once, round by round (round-outer order: the B
// chains interleave, and each round's key serves all of them); the same
// results as B calls of philox4x32_10.
template <int B>
__device__ __forceinline__ void philox4x32_10_batch(uint4 (&c)[B], const RoundKeys& rk)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[b].x;
            const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[b].z;
            c[b] = make_uint4((uint32_t)(p1 >> 32) ^ c[b].y ^ rk.k0[round], (uint32_t)p1,
                              (uint32_t)(p0 >> 32) ^ c[b].w ^ rk.k1[round], (uint32_t)p0);
        }
    }
}

template <int B>
__device__ __forceinline__ void philox4x32_10_batch(uint4 (&c)[B], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[b].x;
            const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[b].z;
            c[b] = make_uint4((uint32_t)(p1 >> 32) ^ c[b].y ^ k0, (uint32_t)p1,
                              (uint32_t)(p0 >> 32) ^ c[b].w ^ k1, (uint32_t)p0);
        }
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
}

// Four normals from one block, double precision: U = (u + 1/2) 2^-32,
// z0,z1 = sqrt(-2 ln U(u0)) (cos, sin)(2 pi U(u1)); z2,z3 likewise (u2, u3).
__device__ __forceinline__ void box_muller4(uint4 u, double z[4])
{
    const double scale = 2.3283064365386962890625e-10;  // 2^-32
    const double ra = sqrt(-2.0 * log(((double)u.x + 0.5) * scale));
    const double rb = sqrt(-2.0 * log(((double)u.z + 0.5) * scale));
    double sa, ca, sb, cb;
    sincospi(2.0 * (((double)u.y + 0.5) * scale), &sa, &ca);
    sincospi(2.0 * (((double)u.w + 0.5) * scale), &sb, &cb);
    z[0] = ra * ca;
    z[1] = ra * sa;
    z[2] = rb * cb;
    z[3] = rb * sb;
}

// Square root of x >= 0 by the approximate hardware instruction (relative
// error about 2^-23, sqrt(0) = 0): one instruction, no guard against x = 0.
__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Same deviates in single precision.  The radius uses the hardware base-2
// logarithm (ln U = ln 2 * log2 U); the angle is taken as
// 2 pi U - pi = 2 pi (u - 2^31 + 1/2) 2^-32, inside (-pi, pi) where the fast
// sine/cosine are accurate, and the sign flip cos(x + pi) = -cos(x) is folded
// into the radius.  U rounds to 1.0f only when the exact radius is below
// 3.5e-4; the radius is then 0 instead (max abs error 3.5e-4, probability
// 2^-25 per pair).
__device__ __forceinline__ void box_muller4(uint4 u, float z[4])
{
    const float scale = 2.3283064365386963e-10f;          // 2^-32
    const float m2ln2 = -1.38629436111989061883f;         // -2 ln 2
    const float ang = 1.46291807926715968105e-09f;        // 2 pi 2^-32
    const float ang0 = 7.31459039633579840525e-10f;       // pi 2^-32
    const float ra = -sqrt_approx(m2ln2 * __log2f(fmaf((float)u.x, scale, 0.5f * scale)));
    const float rb = -sqrt_approx(m2ln2 * __log2f(fmaf((float)u.z, scale, 0.5f * scale)));
    const float ta = fmaf((float)(int32_t)(u.y ^ 0x80000000u), ang, ang0);
    const float tb = fmaf((float)(int32_t)(u.w ^ 0x80000000u), ang, ang0);
    float sa, ca, sb, cb;
    __sincosf(ta, &sa, &ca);
    __sincosf(tb, &sb, &cb);
    z[0] = ra * ca;
    z[1] = ra * sa;
    z[2] = rb * cb;
    z[3] = rb * sb;
}

// The same single-precision deviates times a factor a > 0, free of cost: the
// radius sqrt(-2 ln U) a is sqrt(x') with x' = (-2 ln 2 a^2) log2 U, so a^2
// goes into the constant c2 = -2 ln 2 a^2 that multiplies log2 U anyway (the
// heat step takes the face noise amplitude this way).  c2 < 0.
__device__ __forceinline__ void box_muller4_scaled(uint4 u, float c2, float z[4])
{
    const float scale = 2.3283064365386963e-10f;          // 2^-32
    const float ang = 1.46291807926715968105e-09f;        // 2 pi 2^-32
    const float ang0 = 7.31459039633579840525e-10f;       // pi 2^-32
    const float ra = -sqrt_approx(c2 * __log2f(fmaf((float)u.x, scale, 0.5f * scale)));
    const float rb = -sqrt_approx(c2 * __log2f(fmaf((float)u.z, scale, 0.5f * scale)));
    const float ta = fmaf((float)(int32_t)(u.y ^ 0x80000000u), ang, ang0);
    const float tb = fmaf((float)(int32_t)(u.w ^ 0x80000000u), ang, ang0);
    float sa, ca, sb, cb;
    __sincosf(ta, &sa, &ca);
    __sincosf(tb, &sb, &cb);
    z[0] = ra * ca;
    z[1] = ra * sa;
    z[2] = rb * cb;
    z[3] = rb * sb;
}

// double precision: the deviates times a (one product each)
__device__ __forceinline__ void box_muller4_scaled(uint4 u, double a, double z[4])
{
    box_muller4(u, z);
#pragma unroll
    for (int k = 0; k < 4; ++k) z[k] *= a;
}

}  // namespace she
