// pic_device.cuh -- device building blocks of the PIC/MCC kernels: counter-
// based random numbers, own elementary functions, explicitly rounded float /
// double arithmetic. Every floating-point operation that can decide an integer
// (candidate, process, cell, fixed-point deposit) is spelled out with its
// rounding here, so the kernels compute exactly the documented sequence
// whatever the compiler's contraction settings.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pic {

// ---- explicitly rounded arithmetic, overloaded on the particle precision ----
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float div_(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float sqrt_(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ float floor_(float a) { return floorf(a); }
__device__ __forceinline__ long long rint_ll(float a) { return __float2ll_rn(a); }
__device__ __forceinline__ double add_(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul_(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double div_(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double sqrt_(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ double floor_(double a) { return floor(a); }
__device__ __forceinline__ long long rint_ll(double a) { return __double2ll_rn(a); }

template <typename T> __device__ __forceinline__ T one_minus_ulp();
template <> __device__ __forceinline__ float one_minus_ulp<float>() { return 0x1.fffffep-1f; }
template <> __device__ __forceinline__ double one_minus_ulp<double>() { return 0x1.fffffffffffffp-1; }

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ----------------------
// Ten rounds; each multiplies counter words 0 and 2 by the two Philox-4x32
// multipliers, swaps in the low halves and xors the high halves with the other
// two words and the round key; the key advances by the two Weyl increments.
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                            uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

// Stream of one particle: counter = (slot, step bits 0..31, step bits 32..47
// << 16 | species << 8 | call, discharge id), key = the 64-bit seed.
__device__ __forceinline__ U4 draw(unsigned long long seed, uint32_t slot, long long step, int species, int call,
                                   uint32_t discharge_id) {
    const unsigned long long n = (unsigned long long)step;
    const uint32_t w2 = (uint32_t)(((n >> 32) & 0xFFFFull) << 16) | ((uint32_t)species << 8) | (uint32_t)call;
    return philox4x32_10(slot, (uint32_t)n, w2, discharge_id, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// (top 23 bits + 1/2) 2^-23: in [2^-24, 1 - 2^-24], exact in float.
__device__ __forceinline__ float u01(uint32_t x) {
    return __fmul_rn(__fadd_rn(__uint2float_rn(x >> 9), 0.5f), 0x1p-23f);
}

// ---- own log and sin/cos(pi y) -------------------------------------------
// ln x for positive normal x: split x = m 2^e with m in [sqrt(1/2), sqrt(2)),
// ln m = 2 atanh(t), t = (m-1)/(m+1), Taylor series of atanh to t^9.
__device__ __forceinline__ float own_logf(float x) {
    const uint32_t b = __float_as_uint(x);
    int e = (int)((b >> 23) & 0xFFu) - 127;
    float m = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
    if (m > 0x1.6a09e6p+0f) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    const float t = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float t2 = __fmul_rn(t, t);
    float p = __fmaf_rn(t2, 0x1.c71c72p-4f, 0x1.24924ap-3f);  // 1/9, 1/7
    p = __fmaf_rn(t2, p, 0x1.99999ap-3f);                      // 1/5
    p = __fmaf_rn(t2, p, 0x1.555556p-2f);                      // 1/3
    const float t2x = __fmul_rn(2.0f, t);
    const float lm = __fmaf_rn(t2x, __fmul_rn(t2, p), t2x);
    const float ef = __int2float_rn(e);
    return __fmaf_rn(ef, 0x1.62e430p-1f, __fmaf_rn(ef, -0x1.05c610p-29f, lm));  // ln2 = hi + lo
}

// sin(pi y), cos(pi y), y in [0, 2]: y = r + q/2, q = rint(2y), |r| <= 1/4;
// Taylor series of sin(pi r) to r^9 and cos(pi r) to r^10; quadrant q mod 4.
__device__ __forceinline__ void own_sincospif(float y, float& s, float& c) {
    const float q = rintf(__fmul_rn(2.0f, y));
    const float r = __fmaf_rn(q, -0.5f, y);
    const int iq = ((int)q) & 3;
    const float r2 = __fmul_rn(r, r);
    float ps = __fmaf_rn(r2, 0x1.507834p-4f, -0x1.32d2ccp-1f);
    ps = __fmaf_rn(r2, ps, 0x1.466bc6p+1f);
    ps = __fmaf_rn(r2, ps, -0x1.4abbcep+2f);
    ps = __fmaf_rn(r2, ps, 0x1.921fb6p+1f);
    const float sn = __fmul_rn(r, ps);
    float pc = __fmaf_rn(r2, -0x1.a6d1f2p-6f, 0x1.e1f506p-3f);
    pc = __fmaf_rn(r2, pc, -0x1.55d3c8p+0f);
    pc = __fmaf_rn(r2, pc, 0x1.03c1f0p+2f);
    pc = __fmaf_rn(r2, pc, -0x1.3bd3ccp+2f);
    const float cs = __fmaf_rn(r2, pc, 1.0f);
    if (iq == 0) { s = sn; c = cs; }
    else if (iq == 1) { s = cs; c = -sn; }
    else if (iq == 2) { s = -sn; c = -cs; }
    else { s = -cs; c = sn; }
}

// Box-Muller pair of standard normals.
__device__ __forceinline__ void box_muller(float ua, float ub, float& n0, float& n1) {
    const float rr = __fsqrt_rn(__fmul_rn(-2.0f, own_logf(ua)));
    float s, c;
    own_sincospif(__fmul_rn(2.0f, ub), s, c);
    n0 = __fmul_rn(rr, c);
    n1 = __fmul_rn(rr, s);
}

// Uniform direction on the sphere, z polar: cos(theta) = 1 - 2 ua (exact),
// azimuth 2 pi ub. The double version takes sin(theta) in double and
// renormalises the float azimuth pair in double.
__device__ __forceinline__ void iso_dir(float ua, float ub, float& nx, float& ny, float& nz) {
    const float ct = __fsub_rn(1.0f, __fmul_rn(2.0f, ua));
    const float st = __fsqrt_rn(fmaxf(0.0f, __fmaf_rn(-ct, ct, 1.0f)));
    float s, c;
    own_sincospif(__fmul_rn(2.0f, ub), s, c);
    nx = __fmul_rn(st, c);
    ny = __fmul_rn(st, s);
    nz = ct;
}
__device__ __forceinline__ void iso_dir(float ua, float ub, double& nx, double& ny, double& nz) {
    const double ct = __dsub_rn(1.0, __dmul_rn(2.0, (double)ua));
    const double st = __dsqrt_rn(fmax(0.0, __fma_rn(-ct, ct, 1.0)));
    float sf, cf;
    own_sincospif(__fmul_rn(2.0f, ub), sf, cf);
    double c = (double)cf, s = (double)sf;
    const double h = __dsqrt_rn(__dadd_rn(__dmul_rn(c, c), __dmul_rn(s, s)));
    c = __ddiv_rn(c, h);
    s = __ddiv_rn(s, h);
    nx = __dmul_rn(st, c);
    ny = __dmul_rn(st, s);
    nz = ct;
}

}  // namespace pic
