// ism_device.cuh -- device helpers shared by the libism kernels.
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "ism_internal.h"

// ---------------------------------------------------------------------------
// Job lookup: the kernels of a launch set enumerate their CTAs across the
// jobs of the table; job j owns CTAs [base_j, base_{j+1}).  Bases never
// decrease; a job without CTAs of a kind shares its base with the next one,
// so the owner is the last job whose base is <= cta (binary search).
// ---------------------------------------------------------------------------
template <typename F>
__device__ __forceinline__ int ism_find_job(const JobTable& t, long long cta, F base_of)
{
    int lo = 0, hi = t.n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base_of(t.j[mid]) <= cta) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// A kernel's dynamic shared-memory limit is process-wide, so a limit set to
// each launch's own need could be lowered by another host thread launching
// the same kernel between this thread's set and its launch (which would then
// fail).  Instead the limit is raised once per device to the device's opt-in
// maximum less the kernel's static shared memory; `done` holds one bit per
// device (one flag per kernel).
inline int ism_open_smem(const void* kernel, std::atomic<unsigned long long>* done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done->load(std::memory_order_acquire) & bit) return 0;
    int mx = 0;
    if ((e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return (int)e;
    cudaFuncAttributes fa{};
    if ((e = cudaFuncGetAttributes(&fa, kernel)) != cudaSuccess) return (int)e;   // static + dynamic <= opt-in
    if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  mx - (int)fa.sharedSizeBytes)) != cudaSuccess)
        return (int)e;
    done->fetch_or(bit, std::memory_order_release);
    return 0;
}

// Reflection coefficient w of a job: from device memory when the caller keeps
// the coefficients there, else from the job table.
__device__ __forceinline__ float ism_job_beta(const JobDev& J, int w) { return J.beta_dev ? J.beta_dev[w] : J.beta[w]; }

// g2 = 6 log2(10) / (f_s T60), the log2 of the power decay per sample of the
// diffuse tail (eq. (7)-(8)).  For coefficients in device memory T60 comes
// from the Sabine formula evaluated here with the host's FP64 operations in
// the host's order, each rounded on its own (no contraction), so the value is
// bitwise the one the host computes from the same coefficients.
__device__ __forceinline__ double ism_job_g2_fp64(const JobDev& J)
{
    const double L0 = J.L[0], L1 = J.L[1], L2 = J.L[2];
    const double S[6] = {__dmul_rn(L1, L2), __dmul_rn(L1, L2), __dmul_rn(L0, L2),
                         __dmul_rn(L0, L2), __dmul_rn(L0, L1), __dmul_rn(L0, L1)};
    double den = 0.0;
    for (int i = 0; i < 6; ++i) {
        const double b = (double)J.beta_dev[i];
        den = __dadd_rn(den, __dmul_rn(S[i], __dsub_rn(1.0, __dmul_rn(b, b))));
    }
    if (!(den > 0.0)) return 0.0;
    const double T60 = __ddiv_rn(__dmul_rn(__dmul_rn(__dmul_rn(0.161, L0), L1), L2), den);
    if (!(T60 < 1.0e300)) return 0.0;
    return __ddiv_rn(J.g2_c, __dmul_rn((double)J.fs, T60));
}

// ---------------------------------------------------------------------------
// Float-float (unevaluated sum hi + lo) arithmetic on correctly rounded FP32
// operations (Dekker / Knuth two-sum).  Intrinsics keep the compiler from
// contracting or reordering the error terms.
// ---------------------------------------------------------------------------
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    float s = __fadd_rn(a.hi, b.hi);
    float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    float hi = __fadd_rn(s, e);
    float lo = __fsub_rn(e, __fsub_rn(hi, s));
    return {hi, lo};
}

// g2 of the job as a float-float pair (hi + lo is its FP64 value to ~2^-48).
__device__ __forceinline__ ff ism_job_g2(const JobDev& J)
{
    if (!J.beta_dev) return {J.g2, J.g2_lo};
    const double g = ism_job_g2_fp64(J);
    const float hi = (float)g;
    return {hi, (float)(g - (double)hi)};
}

// 2^(-g i) for a float-float rate g >= 0 and an integer 0 <= i < 2^24: the
// product x = g i keeps its rounding error (one FMA) and the low part of g,
// x is split into its nearest integer n and a remainder r in [-1/2, 1/2]
// (p - n is exact: Sterbenz), and 2^-x = 2^-n 2^-r.  The result carries
// exp2f's own error (2 ulp) and nothing from the size of x.
__device__ __forceinline__ float ism_exp2_neg(ff g, int i)
{
    const float fi = (float)i;
    const float p = __fmul_rn(g.hi, fi);
    if (!(p < 256.0f)) return 0.0f;   // below 2^-255: zero in FP32 (also catches an infinite rate)
    const float pe = __fmaf_rn(g.lo, fi, __fmaf_rn(g.hi, fi, -p));
    const float n = rintf(p);
    const float r = __fadd_rn(__fsub_rn(p, n), pe);
    return ldexpf(exp2f(-r), -(int)n);
}

// Approximate reciprocal and reciprocal square root on the special-function
// unit (max error ~1-2 ulp).
__device__ __forceinline__ float ism_rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float ism_rsqrt(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// sqrt of a positive float-float: r = a.hi / sqrt(a.hi) from the approximate
// reciprocal root, then one Newton correction from the exact residual
// a - r^2 (FMA) of the full float-float value: lo = (a - r^2) / (2 r).  The
// pair r + lo is accurate to ~2^-44 relative although r itself is not
// correctly rounded.
__device__ __forceinline__ ff ff_sqrt(ff a)
{
    float rs = ism_rsqrt(a.hi);
    float r = __fmul_rn(a.hi, rs);
    float res = __fadd_rn(__fmaf_rn(-r, r, a.hi), a.lo);
    float lo = __fmul_rn(__fmul_rn(res, 0.5f), rs);
    return {r, lo};
}

// Integer value of a float that holds an integer in [-2^22, 2^22): adding
// 1.5 * 2^23 moves it to the low mantissa bits (no rounding happens, the
// value being integral), avoiding a conversion instruction.
__device__ __forceinline__ int ism_int_of_integral(float b)
{
    return __float_as_int(__fadd_rn(b, 12582912.0f)) - 0x4B400000;
}

// Nearest integer of x for |x| < 2^22 (ties to even), same trick.
__device__ __forceinline__ int ism_round_int(float x)
{
    return __float_as_int(__fadd_rn(x, 12582912.0f)) - 0x4B400000;
}

// sin(pi f) for f in [0, 1]: g = min(f, 1 - f) in [0, 1/2] (1 - f is exact
// for f >= 1/2) and the Taylor series of sin(pi g) through (pi g)^11, whose
// remainder is below (pi/2)^13 / 13! = 5.7e-8 on [0, 1/2].
__device__ __forceinline__ float ism_sinpi01(float f)
{
    const double PI = 3.141592653589793238462643383279502884;
    const float c1 = (float)PI;
    const float c3 = (float)(-PI * PI * PI / 6.0);
    const float c5 = (float)(PI * PI * PI * PI * PI / 120.0);
    const float c7 = (float)(-PI * PI * PI * PI * PI * PI * PI / 5040.0);
    const float c9 = (float)(PI * PI * PI * PI * PI * PI * PI * PI * PI / 362880.0);
    const float c11 = (float)(-PI * PI * PI * PI * PI * PI * PI * PI * PI * PI * PI / 39916800.0);
    float g = fminf(f, __fsub_rn(1.0f, f));
    float g2 = g * g;
    float p = fmaf(g2, c11, c9);
    p = fmaf(g2, p, c7);
    p = fmaf(g2, p, c5);
    p = fmaf(g2, p, c3);
    p = fmaf(g2, p, c1);
    return p * g;
}

// cos(a), sin(a) for |a| <= pi/8 by their Taylor series through a^8 and a^9
// (remainders below a^10/10! = 2.5e-11 and a^11/11! = 7e-13).
__device__ __forceinline__ void ism_sincos_small(float a, float* s, float* c)
{
    float a2 = a * a;
    float pc = fmaf(a2, 1.0f / 40320.0f, -1.0f / 720.0f);
    pc = fmaf(a2, pc, 1.0f / 24.0f);
    pc = fmaf(a2, pc, -0.5f);
    *c = fmaf(a2, pc, 1.0f);
    float ps = fmaf(a2, 1.0f / 362880.0f, -1.0f / 5040.0f);
    ps = fmaf(a2, ps, 1.0f / 120.0f);
    ps = fmaf(a2, ps, -1.0f / 6.0f);
    *s = fmaf(a2 * a, ps, a);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each two
// 32x32 -> 64-bit products of counter words 0 and 2 with M0, M1, mixed with
// words 1, 3 and the key; the key is bumped by the Weyl constants W0, W1
// between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 ism_philox(uint4 c, uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        uint4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
        k0 += W0;
        k1 += W1;
    }
    return c;
}

// The FP32 noise transform, one correctly rounded operation at a time, in
// the order of its written specification (uniform, ratio, ln, scale):
//   u = ((x >> 9) + 1/2) 2^-23                      exact in FP32
//   r = u / (1 - u)                                 (1 - u exact)
//   ln r: r = m 2^e, m in (sqrt(1/2), sqrt(2)]; t = (m - 1)/(m + 1);
//         ln m = 2t + t^3 (2/3 + t^2 (2/5 + t^2 (2/7 + t^2 (2/9 + t^2 2/11))))
//         ln r = e ln2_hi + (e ln2_lo + ln m)
//   z = (sqrt(3)/pi) ln r                           unit-variance logistic
__device__ __forceinline__ float ism_uniform(uint32_t x)
{
    float m = __uint2float_rn(x >> 9);
    return __fmul_rn(__fadd_rn(m, 0.5f), 0x1p-23f);
}

__device__ __forceinline__ float ism_ln_spec(float x)
{
    uint32_t bits = __float_as_uint(x);
    int e = (int)((bits >> 23) & 0xFFu) - 127;
    float m = __uint_as_float((bits & 0x007FFFFFu) | 0x3F800000u);
    if (m > 1.41421353816986083984375f) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    float t = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    float t2 = __fmul_rn(t, t);
    float p = __fmaf_rn(t2, 2.0f / 11.0f, 2.0f / 9.0f);
    p = __fmaf_rn(t2, p, 2.0f / 7.0f);
    p = __fmaf_rn(t2, p, 2.0f / 5.0f);
    p = __fmaf_rn(t2, p, 2.0f / 3.0f);
    float t3 = __fmul_rn(t, t2);
    float lnm = __fmaf_rn(t3, p, __fmul_rn(2.0f, t));
    float ef = __int2float_rn(e);
    return __fmaf_rn(ef, 0.693145751953125f, __fmaf_rn(ef, 1.428606765330187e-06f, lnm));
}

__device__ __forceinline__ float ism_logistic(uint32_t x)
{
    float u = ism_uniform(x);
    float r = __fdiv_rn(u, __fsub_rn(1.0f, u));
    return __fmul_rn(0.5513288974761963f, ism_ln_spec(r));
}

// Noise of sample k of RIR `rir`: word k mod 4 of Philox(counter (k/4, rir,
// 0, 0), key (seed lo, seed hi)).  Returns the four logistic values of the
// counter block k/4.
__device__ __forceinline__ float4 ism_noise_block(uint64_t seed, uint32_t rir, uint32_t blk)
{
    uint4 w = ism_philox(make_uint4(blk, rir, 0u, 0u), (uint32_t)seed, (uint32_t)(seed >> 32));
    return make_float4(ism_logistic(w.x), ism_logistic(w.y), ism_logistic(w.z), ism_logistic(w.w));
}
