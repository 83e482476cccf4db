// Device-side building blocks shared by the libsmp kernels: Philox4x32-10, the Box-Muller and 53-bit uniform
// maps, warp reductions and the device error word.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace smp {

// Device error word bits (set with atomicOr, read by the next synchronising call).
enum : int {
    DEVERR_NUMERIC = 1,   // Cholesky pivot <= 0 (not positive definite)
    DEVERR_TIMEOUT = 2,   // a bounded wait gave up
    DEVERR_BOUNDS = 4,    // an index check failed (a kernel skipped the access)
};

// Philox counter tags (fourth counter word) of the four random streams.
enum : uint32_t {
    TAG_PI = 1u,
    TAG_SAMPLE = 2u,
    TAG_SPLIT = 3u,
    TAG_INIT = 4u,
    TAG_MULTI = 5u,
    TAG_SRHT_SIGN = 6u,
    TAG_SRHT_ROW = 7u
};

struct U32x4 {
    uint32_t x, y, z, w;
};

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; in each, words 0 and 2 are multiplied by the
// two round multipliers, the high halves are xor-ed with words 1 / 3 and the round key, the low halves move to
// words 1 / 3; the key is bumped by the Weyl increments between rounds.
__device__ __forceinline__ U32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                              uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return U32x4{c0, c1, c2, c3};
}

// Hardware approximations (PTX lg2/sqrt/sin/cos .approx): the Gaussian map needs no more than binary32-level
// accuracy because M~ is invariant to a global scale of Pi and the sketch runs on TF32/BF16 operands.
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sin_approx(float x) {
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float cos_approx(float x) {
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Box-Muller on two Philox words: u1 = ((xe >> 8) + 1) 2^-24 in (0, 1], u2 = (xo >> 8) 2^-24 in [0, 1);
// rho = sqrt(-2 ln u1); (z0, z1) = rho (cos 2 pi u2, sin 2 pi u2). The angle is evaluated as theta - pi with
// theta = 2 pi u2 so the hardware sine/cosine see [-pi, pi): cos(theta) = -cos(theta - pi), same for sin.
__device__ __forceinline__ void box_muller_f32(uint32_t xe, uint32_t xo, float& z0, float& z1) {
    const float u1 = (float)((xe >> 8) + 1u) * 5.9604644775390625e-08f;
    const float u2 = (float)(xo >> 8) * 5.9604644775390625e-08f;
    const float rho = sqrt_approx(-1.3862943611198906f * lg2_approx(u1));  // -2 ln 2 * log2(u1)
    const float th = fmaf(u2, 6.2831853071795865f, -3.1415926535897932f);
    z0 = -rho * cos_approx(th);
    z1 = -rho * sin_approx(th);
}

// Binary64 Box-Muller with CUDA's accurate double log / sqrt / sincospi (the SMP_F64 path).
__device__ __forceinline__ void box_muller_f64(uint32_t xe, uint32_t xo, double& z0, double& z1) {
    const double u1 = (double)((xe >> 8) + 1u) * 5.9604644775390625e-08;
    const double u2 = (double)(xo >> 8) * 5.9604644775390625e-08;
    const double rho = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    z0 = rho * c;
    z1 = rho * s;
}

// 53-bit uniform in [0, 1): ((x0 >> 5) 2^26 + (x1 >> 6)) 2^-53; every step is exact in binary64.
__device__ __forceinline__ double uniform53(uint32_t x0, uint32_t x1) {
    return __dmul_rn(__dadd_rn(__dmul_rn((double)(x0 >> 5), 67108864.0), (double)(x1 >> 6)),
                     1.1102230246251565404e-16);
}

// Coin of Omega / split: Philox counter (i, j, 0, tag).
__device__ __forceinline__ double coin(uint32_t i, uint32_t j, uint32_t tag, uint32_t k0, uint32_t k1) {
    const U32x4 x = philox4x32_10(i, j, 0u, tag, k0, k1);
    return uniform53(x.x, x.y);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T to_acc(T v) {
    return v;
}

__device__ __forceinline__ float load_as_float(const float* p) { return *p; }
__device__ __forceinline__ float load_as_float(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ double load_as_double(const double* p) { return *p; }

__device__ __forceinline__ void set_error(int* err, int bit) {
    if (err) atomicOr(err, bit);
}

// 1/sqrt(d) in binary64 without the long-latency binary64 square root and divide: the binary32 hardware estimate
// (rsqrt.approx, relative error < 2^-22) refined by two Newton-Raphson steps y <- y (3 - d y^2) / 2, each of which
// squares the relative error (2^-44, then below binary64 rounding). Falls back to 1 / sqrt(d) outside the binary32
// range. d must be > 0.
__device__ __forceinline__ double rsqrt_refined(double d) {
    if (!(d > 1e-36 && d < 1e36)) return 1.0 / sqrt(d);
    float yf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"((float)d));
    double y = (double)yf;
    const double hd = 0.5 * d;
    y = y * fma(-hd * y, y, 1.5);
    y = y * fma(-hd * y, y, 1.5);
    return y;
}

// 1/sqrt(d) for any positive normal binary64 d, with no out-of-range branch: d = m 4^h with m in [1, 4) (exact
// exponent arithmetic), the binary32 estimate of 1/sqrt(m) refined by two Newton-Raphson steps as in rsqrt_refined,
// then scaled by 2^-h (exact). Callers keep arrays in registers across it (no call to a division or square-root
// routine).
__device__ __forceinline__ double rsqrt_scaled(double d) {
    const long long bits = __double_as_longlong(d);
    const int h = (((int)((bits >> 52) & 0x7ff)) - 1023) >> 1;   // floor(exponent / 2)
    const double m = __longlong_as_double(bits - ((long long)(2 * h) << 52));
    float yf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"((float)m));
    double y = (double)yf;
    const double hm = 0.5 * m;
    y = y * fma(-hm * y, y, 1.5);
    y = y * fma(-hm * y, y, 1.5);
    return __longlong_as_double(__double_as_longlong(y) - ((long long)h << 52));
}

// Sum of 32 per-lane vectors: afterwards lane l holds sum over lanes of v[l]. Five butterfly rounds; in the round
// with offset o each lane keeps the half of its live values selected by bit o of its lane id and adds the
// partner's matching half (o shuffles per round, 31 in total).
template <typename T>
__device__ __forceinline__ T transpose_sum32(T (&v)[32], int lane) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const T send = upper ? v[i] : v[i + o];
            const T keep = upper ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

}  // namespace smp
