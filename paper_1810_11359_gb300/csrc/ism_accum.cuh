// ism_accum.cuh -- windowed-sinc accumulation (kernel c), the hot loop of the
// method: eq. (5) with the fractional-delay pulse of eq. (6).  The kernel is
// a template over the window length (SLOTS taps per lane), the window mask
// and the tap arithmetic (PREC); each precision is instantiated in a
// translation unit of its own (ism_accum.cu, ism_accum_fp16.cu,
// ism_accum_bf16.cu, ism_accum_lut.cu).
//
// One CTA owns ism_acc_bins(PREC) delay bins of 32 samples of one RIR, one
// warp per bin; warps share nothing but the per-axis tables, so a CTA holds few
// resources and finishes as soon as its bins do (no end-of-tile barrier: the
// schedule balances itself across many small CTAs).  An image of bin q has
// delay s = b + f (b integer,
// f in [0, 1)) with b = 32 q + rr, rr in [-1, 31] (the enumeration binned it
// by its plain-FP32 delay).  Its taps are the samples k with |k - s| < N_w/2:
// j = k - b in [-H + 1, H], H = N_w / 2.
//
// Lane l of the warp always evaluates the taps t = l + 32 s (s < SLOTS, 2H =
// 32 SLOTS), j = t - H + 1, of whatever image the warp is processing.  With j
// fixed per lane everything but two products is a lane constant:
//   sinc(j - f) = (-1)^(j+1) sin(pi f) / (pi (j - f))
//   1 + cos(2 pi (j - f) / N_w) = 1 + C_j cos(phi) + S_j sin(phi),
//                                  phi = 2 pi f / N_w,
// so with the per-image record {f, P, P cos phi, P sin phi}, P = A sin(pi f)
// / (2 pi), one tap is
//   x = sigma_j (j - f)                    (one FFMA, sigma_j = (-1)^(j+1))
//   w = P + C_j P cos phi + S_j P sin phi  (two FFMA)
//   D += w * rcp(x)                        (one MUFU + one FFMA)
// -- four FMA-pipe operations and one reciprocal per tap, the record fetched
// by one broadcast shared-memory load.
//
// Reduced-precision forms of the same tap (Section 3.3 of the paper keeps
// the sinc and the window in half precision):
//   FP16X2 / BF16X2  two images of a run per lane and instruction: x of both
//       in FP32 (the factorised sinc is ill-conditioned near x = 0 if f is
//       rounded first), packed to a half2 / bfloat162 pair; w by two packed
//       FMAs on the packed record {P, P cos phi, P sin phi}; packed
//       reciprocal; each product accumulated in FP32 by a mixed-precision FMA
//       (f16 x f16 + f32).  FP16 records are scaled by 2^e per job so that
//       late, weak images stay in the normal range; the scale is removed,
//       exactly, when a run is flushed.  f is kept in [2^-13, 1 - 2^-13] so
//       the reciprocal cannot overflow (a delay change of <= 1.2e-4 sample).
//   LUT  eq. (9): the windowed sinc tabulated every 1/Q sample and linearly
//       interpolated.  The table is polyphase: row p holds the 32 SLOTS taps
//       of the fractional delay p / Q, so lane l reads column l of two rows
//       -- conflict-free -- and a tap is two shared loads and two FFMA with
//       the record {A (1 - phi), A phi, row offset}, u = f Q, p = floor(u),
//       phi = u - p.  Q = 256 for a 32-tap window (the paper's 4096 entries
//       over [0, 16] samples, stored once per tap: 257 x 32 FP32 = 32.9 KB).
//       The mask of a non-integral window is part of the table.
//
// Tap t of an image lands at window position p = rr + 1 + t.  The warp keeps
// the window of its bin (32 (SLOTS + 1) samples from 32 q - H) in
// registers: lane l, register m holds position l + 32 m.  Images with equal
// rr are summed in the lane-per-tap accumulator D first; when rr changes the
// run total is rotated into the window with one shuffle per slot.  The ids of
// a bin are counting-sorted by their plain-FP32 offset (33 values; the exact
// rr coincides except within ~1e-3 sample of an integer) in shared memory,
// so runs are long.  The sort is stable, so the summation order -- and the
// FP32 result -- is the same on every run, with no atomics.
//
// The delay s comes from float-float arithmetic on per-axis tables of squared
// offsets (Section 2.1 factorisation), so f keeps FP32 resolution even for
// delays of tens of thousands of samples.
//
// Each warp stores its bin's window row (32 (SLOTS + 1) samples, coalesced)
// once; the finalize kernel adds, for every sample, the rows of the SLOTS + 1
// bins covering it in ascending bin order.  Every sum has a fixed order.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ism_device.cuh"

namespace {

#define ISM_PIECE 512              // ids sorted per step (shared memory per warp ~5 KB)
#define ISM_NB 33                  // delay offsets rr = -1 .. 31 inside a bin
#define ISM_CHUNK 64               // records computed per step (two per lane)
#define ISM_PAD (ISM_PIECE + 4 * ISM_NB)
#define ISM_DUMMY 0x80000000u      // sorted-list entry that carries no image

enum { PREC_FP32 = 0, PREC_FP16 = 1, PREC_BF16 = 2, PREC_LUT = 3, PREC_TEX = 4 };

struct WarpSmem {
    uint32_t sorted[ISM_PAD];      // ids sorted by plain-FP32 offset, buckets padded to 4
    uint16_t key[ISM_PIECE];       // bucket (low 6 bits) | rank in bucket << 6
    uint8_t group_bucket[ISM_PAD / 4];  // bucket of every group of 4 sorted entries
    uint32_t off[ISM_NB + 1];      // padded bucket offsets in `sorted`
    uint32_t cnt[ISM_NB + 1];      // bucket sizes
    // records of the current chunk: FP32 / LUT one float4 per image; FP16X2 /
    // BF16X2 one uint4 {f_a, f_b, P, P cos phi} per image pair at [0, 32) and
    // the pairs' packed P sin phi at [32, 40)
    float4 rec[ISM_CHUNK];
};

// Delay and amplitude of an image of bin q (eq. (2)-(4)): exact delay s = b
// + f from the float-float squared offsets, rr = b - 32 q, A = F / (4 pi d)
// = F amp_scale / s.  Branch free; an offset outside [-1, 31] (which the
// binning rules out) raises *bad and contributes nothing.
__device__ __forceinline__ void ism_delay(const float4 tx, const float4 ty, const float4 tz, int q, float amp_scale,
                                          float* f_out, float* amp_out, int* rr_out, bool* bad,
                                          const float3 o = make_float3(0.0f, 0.0f, 0.0f), float alpha = 1.0f)
{
    const ff s2 = ff_add(ff_add(ff{tx.x, tx.y}, ff{ty.x, ty.y}), ff{tz.x, tz.y});
    const ff sq = ff_sqrt(s2);
    float b = floorf(sq.hi);
    float f = __fadd_rn(__fsub_rn(sq.hi, b), sq.lo);
    // bring f into [0, 1); -tiny + 1 rounds to 1.0, hence two steps
    const bool neg = f < 0.0f;
    f = neg ? __fadd_rn(f, 1.0f) : f;
    b = neg ? b - 1.0f : b;
    const bool one = f >= 1.0f;
    f = one ? __fsub_rn(f, 1.0f) : f;
    b = one ? b + 1.0f : b;
    int rr = ism_int_of_integral(b) - ISM_SB * q;
    const float rs = ism_rcp(sq.hi);
    float amp = tx.z * ty.z * tz.z * amp_scale * rs;
    if (alpha != 1.0f)   // polar pattern: cos(theta) = o . (x_n - x_r) / d, o of unit length
        amp *= __fmaf_rn(1.0f - alpha, __fmaf_rn(o.z, tz.w, __fmaf_rn(o.y, ty.w, o.x * tx.w)) * rs, alpha);
    const bool out = rr < -1 || rr > ISM_SB - 1;
    *bad = out;
    *rr_out = out ? -1 : rr;
    *amp_out = out ? 0.0f : amp;
    *f_out = f;
}

// The per-image record of the factorised windowed sinc of eq. (6): {f, P,
// P cos(phi), P sin(phi)}, P = A sin(pi f) / (2 pi), phi = 2 pi f / N_w.
__device__ __forceinline__ float4 ism_sinc_record(float f, float amp, bool small_phase, float twopi_Nw,
                                                  float inv2Nw)
{
    const float P = amp * ism_sinpi01(f) * 0.15915494309189535f;  // A sin(pi f) / (2 pi)
    float sp, cp;
    if (small_phase) ism_sincos_small(f * twopi_Nw, &sp, &cp);
    else sincospif(f * inv2Nw, &sp, &cp);
    return make_float4(f, P, P * cp, P * sp);
}

// ---- packed half-precision helpers -------------------------------------
template <int PREC>
__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    if constexpr (PREC == PREC_FP16) {
        __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t*>(&h);
    }
}

template <int PREC>
__device__ __forceinline__ uint32_t fma2(uint32_t a, uint32_t b, uint32_t c)
{
    if constexpr (PREC == PREC_FP16) {
        __half2 r = __hfma2(*reinterpret_cast<__half2*>(&a), *reinterpret_cast<__half2*>(&b),
                            *reinterpret_cast<__half2*>(&c));
        return *reinterpret_cast<uint32_t*>(&r);
    } else {
        __nv_bfloat162 r = __hfma2(*reinterpret_cast<__nv_bfloat162*>(&a), *reinterpret_cast<__nv_bfloat162*>(&b),
                                   *reinterpret_cast<__nv_bfloat162*>(&c));
        return *reinterpret_cast<uint32_t*>(&r);
    }
}

template <int PREC>
__device__ __forceinline__ uint32_t rcp2(uint32_t a)
{
    if constexpr (PREC == PREC_FP16) {
        __half2 r = h2rcp(*reinterpret_cast<__half2*>(&a));
        return *reinterpret_cast<uint32_t*>(&r);
    } else {
        __nv_bfloat162 r = h2rcp(*reinterpret_cast<__nv_bfloat162*>(&a));
        return *reinterpret_cast<uint32_t*>(&r);
    }
}

// da += lo(w) lo(r), db += hi(w) hi(r): products of two 16-bit values
// accumulated in FP32 (mixed-precision FMA, one rounding to FP32).
template <int PREC>
__device__ __forceinline__ void mixed_fma2(float& da, float& db, uint32_t w, uint32_t r)
{
    if constexpr (PREC == PREC_FP16) {
        asm("{\n\t.reg .f16 wl, wh, rl, rh;\n\t"
            "mov.b32 {wl, wh}, %2;\n\t"
            "mov.b32 {rl, rh}, %3;\n\t"
            "fma.rn.f32.f16 %0, wl, rl, %0;\n\t"
            "fma.rn.f32.f16 %1, wh, rh, %1;\n\t}"
            : "+f"(da), "+f"(db)
            : "r"(w), "r"(r));
    } else {
        asm("{\n\t.reg .b16 wl, wh, rl, rh;\n\t"
            "mov.b32 {wl, wh}, %2;\n\t"
            "mov.b32 {rl, rh}, %3;\n\t"
            "fma.rn.f32.bf16 %0, wl, rl, %0;\n\t"
            "fma.rn.f32.bf16 %1, wh, rh, %1;\n\t}"
            : "+f"(da), "+f"(db)
            : "r"(w), "r"(r));
    }
}

// Rotates the run total D (lane = tap) into the window (lane = position);
// `scale` undoes the record scaling of the FP16 form (a power of two).
template <int SLOTS, bool SCALED>
__device__ __forceinline__ void flush_run(float (&D)[SLOTS], float (&acc)[SLOTS + 1], int rr, int lane, float scale)
{
    const int src = (lane - rr - 1) & 31;
    const bool upper = lane <= rr;
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
        float v = __shfl_sync(0xffffffffu, SCALED ? D[s] * scale : D[s], src);
        if (upper) acc[s + 1] += v;
        else acc[s] += v;
        D[s] = 0.0f;
    }
}

// Adds the taps of one FP32 record (lane = tap) directly into the window at
// its own offset rr: used, in every precision, for the rare image whose
// exact offset differs from the offset of the bucket it was sorted into.
template <int SLOTS, bool MASK>
__device__ __forceinline__ void add_single(const float4 rc, int rr, const float (&xj)[SLOTS],
                                           const float (&nsg)[SLOTS], const float (&Cj)[SLOTS],
                                           const float (&Sj)[SLOTS], const bool (&tap_ok)[SLOTS], float halfNw,
                                           float (&acc)[SLOTS + 1], int lane)
{
    const int src = (lane - rr - 1) & 31;
    const bool upper = lane <= rr;
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
        const float x = __fmaf_rn(nsg[s], rc.x, xj[s]);
        float w = __fmaf_rn(Cj[s], rc.z, __fmaf_rn(Sj[s], rc.w, rc.y));
        if (MASK) w = (tap_ok[s] && fabsf(x) < halfNw) ? w : 0.0f;
        const float v = __shfl_sync(0xffffffffu, w * ism_rcp(x), src);
        if (upper) acc[s + 1] += v;
        else acc[s] += v;
    }
}

template <int SLOTS, bool MASK>
__device__ __forceinline__ void taps(const float4 rc, const float (&xj)[SLOTS], const float (&nsg)[SLOTS],
                                     const float (&Cj)[SLOTS], const float (&Sj)[SLOTS],
                                     const bool (&tap_ok)[SLOTS], float halfNw, float (&D)[SLOTS])
{
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
        const float x = __fmaf_rn(nsg[s], rc.x, xj[s]);
        float w = __fmaf_rn(Cj[s], rc.z, __fmaf_rn(Sj[s], rc.w, rc.y));
        if (MASK) w = (tap_ok[s] && fabsf(x) < halfNw) ? w : 0.0f;
        D[s] = __fmaf_rn(w, ism_rcp(x), D[s]);
    }
}

// Taps of an image pair {f_a, f_b, P2, Pc2} + Ps2 in packed 16-bit
// arithmetic; image a accumulates into Da, image b into Db.
template <int SLOTS, bool MASK, int PREC>
__device__ __forceinline__ void taps_pair(const uint4 pr, uint32_t ps2, const float (&xj)[SLOTS],
                                          const float (&nsg)[SLOTS], const uint32_t (&C2)[SLOTS],
                                          const uint32_t (&S2)[SLOTS], const bool (&tap_ok)[SLOTS], float halfNw,
                                          float (&Da)[SLOTS], float (&Db)[SLOTS])
{
    const float fa = __uint_as_float(pr.x), fb = __uint_as_float(pr.y);
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
        const float xa = __fmaf_rn(nsg[s], fa, xj[s]);
        const float xb = __fmaf_rn(nsg[s], fb, xj[s]);
        uint32_t w = fma2<PREC>(C2[s], pr.w, fma2<PREC>(S2[s], ps2, pr.z));
        if (MASK) {
            const bool oka = tap_ok[s] && fabsf(xa) < halfNw, okb = tap_ok[s] && fabsf(xb) < halfNw;
            w &= (oka ? 0x0000FFFFu : 0u) | (okb ? 0xFFFF0000u : 0u);
        }
        mixed_fma2<PREC>(Da[s], Db[s], w, rcp2<PREC>(pack2<PREC>(xa, xb)));
    }
}

// Taps of one LUT record {A (1 - phi), A phi, row offset (int bits)}: two
// rows of the polyphase table in shared memory, column = tap.
template <int SLOTS, int ROW>
__device__ __forceinline__ void taps_lut(const float4 rc, const float* __restrict__ lut_lane, float (&D)[SLOTS])
{
    const float* p = lut_lane + __float_as_int(rc.z);
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
        D[s] = __fmaf_rn(rc.x, p[32 * s], D[s]);
        D[s] = __fmaf_rn(rc.y, p[ROW + 32 * s], D[s]);
    }
}

// Taps of one image from the windowed-sinc table read through the texture
// unit (the paper's own LUT path, Section 3.5): the table is a 2-D texture
// (x = tap, y = fractional-delay phase) with hardware linear filtering along
// y, so each tap is one filtered fetch and one FFMA with the record {A, y}.
// The filter weight has 8 fractional bits (1/256 of a phase step).
template <int SLOTS>
__device__ __forceinline__ void taps_tex(const float4 rc, unsigned long long tex, int lane, float (&D)[SLOTS])
{
#pragma unroll
    for (int s = 0; s < SLOTS; ++s)
        D[s] = __fmaf_rn(rc.x, tex2D<float>((cudaTextureObject_t)tex, (float)(lane + 32 * s) + 0.5f, rc.y), D[s]);
}

template <int SLOTS, bool MASK, int PREC>
__global__ void __launch_bounds__(ism_acc_bins(PREC) * 32) accum_kernel(const __grid_constant__ JobTable t,
                                                                  const float4* __restrict__ tbl,
                                                                  const uint32_t* __restrict__ hist,
                                                                  const uint32_t* __restrict__ ids,
                                                                  const float* __restrict__ lut_g,
                                                                  float* __restrict__ rows,
                                                                  uint32_t* __restrict__ status)
{
    constexpr bool HALF = PREC == PREC_FP16 || PREC == PREC_BF16;
    constexpr int LQ = ism_lut_phases(SLOTS);   // LUT phases per sample
    constexpr int ROW = 32 * SLOTS;             // LUT row: one entry per tap
    extern __shared__ __align__(16) unsigned char smem[];
    const long long g = blockIdx.x;
    const int jid = ism_find_job(t, g, [](const JobDev& j) { return j.acc_cta_base; });
    const JobDev& J = t.j[jid];
    const bool exact = (J.Nw == (float)(2 * J.H)) && (2 * J.H == 32 * J.slots);
    if (J.slots != SLOTS || J.use_cheb) return;                // another kernel handles this job
    if (PREC != PREC_LUT && PREC != PREC_TEX && exact == MASK) return;   // (the tables carry their own mask)

    const long long local = g - J.acc_cta_base;
    const int r = (int)(local / J.acc_groups);
    const int grp = J.acc_groups - 1 - (int)(local % J.acc_groups);  // densest (latest) bins first
    const int Nx = J.N[0], Ny = J.N[1], Nz = J.N[2];
    const int n_axis = Nx + Ny + Nz;
    const int H = J.H;
    constexpr int WIN = 32 * (SLOTS + 1);  // window registers x 32 lanes

    constexpr int BPC = ism_acc_bins(PREC);
    float4* T = reinterpret_cast<float4*>(smem);
    unsigned char* after_T = smem + (size_t)((t.max_axis_sum + 1) & ~1) * sizeof(float4);
    float* lut = reinterpret_cast<float*>(after_T);
    constexpr size_t LUT_BYTES = PREC == PREC_LUT ? (size_t)(LQ + 1) * ROW * sizeof(float) : 0;
    WarpSmem* Wall = reinterpret_cast<WarpSmem*>(after_T + LUT_BYTES);
    float* Sh = reinterpret_cast<float*>(Wall + BPC);   // plain S_hi per axis index (conflict-light keys)

    const float4* Tg = tbl + J.tbl_base + (long long)r * n_axis;
    for (int e = threadIdx.x; e < n_axis; e += blockDim.x) {
        const float4 v = Tg[e];
        T[e] = v;
        Sh[e] = v.x;
    }
    if constexpr (PREC == PREC_LUT) {
        const float4* Lg = reinterpret_cast<const float4*>(lut_g + J.lut_base);
        for (int e = threadIdx.x; e < (LQ + 1) * ROW / 4; e += blockDim.x) reinterpret_cast<float4*>(lut)[e] = Lg[e];
    }

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem& W = Wall[warp];

    // lane constants of the taps t = lane + 32 s, j = t - H + 1
    float xj[SLOTS], nsg[SLOTS], Cj[SLOTS], Sj[SLOTS], D[SLOTS], D2[SLOTS], acc[SLOTS + 1];
    uint32_t C2[SLOTS], S2[SLOTS];
    bool tap_ok[SLOTS];
    const float inv2Nw = 2.0f / J.Nw;
    const float twopi_Nw = 6.283185307179586f / J.Nw;
    const bool small_phase = J.Nw >= 16.0f;   // 2 pi f / N_w <= pi / 8
    // receiver polar pattern: the unit orientation of this RIR's receiver
    const float alpha = J.mic_alpha;
    float3 orient = make_float3(0.0f, 0.0f, 0.0f);
    if (alpha != 1.0f) {
        const float* o = J.orient_rcv + 3 * (r % J.n_rcv);
        const float ox = o[0], oy = o[1], oz = o[2];
        const float inv = 1.0f / sqrtf(__fmaf_rn(ox, ox, __fmaf_rn(oy, oy, oz * oz)));
        orient = make_float3(ox * inv, oy * inv, oz * inv);
    }
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
        const int tt = lane + 32 * s;
        const int j = tt - H + 1;
        const float sg = (j & 1) ? 1.0f : -1.0f;  // (-1)^(j+1)
        xj[s] = sg * (float)j;
        nsg[s] = -sg;
        sincospif((float)j * inv2Nw, &Sj[s], &Cj[s]);
        tap_ok[s] = tt < 2 * H;
        if constexpr (HALF) {
            C2[s] = pack2<PREC>(Cj[s], Cj[s]);
            S2[s] = pack2<PREC>(Sj[s], Sj[s]);
        }
    }
    const float halfNw = 0.5f * J.Nw;
    const unsigned lt_mask = (1u << lane) - 1u;
    // FP16 records are scaled by 2^e; f is kept away from 0 and 1 in both
    // packed forms so that the packed reciprocal stays finite
    const float rscale = (PREC == PREC_FP16) ? J.half_scale : 1.0f;
    const float dscale = (PREC == PREC_FP16) ? 1.0f / J.half_scale : 1.0f;
    const float f_lo = HALF ? 0x1p-13f : 0x1p-60f;
    const float f_hi = HALF ? 1.0f - 0x1p-13f : 1.0f;
    const float* lut_lane = lut + lane;
    __syncthreads();
    (void)lt_mask;
    (void)rscale;

    {
        const int q = grp * BPC + warp;
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
            D[s] = 0.0f;
            D2[s] = 0.0f;
        }
#pragma unroll
        for (int m = 0; m <= SLOTS; ++m) acc[m] = 0.0f;

        if (q < J.Q) {
            const long long hb = J.hist_base + ((long long)r * J.Q + q) * J.U;
            const uint32_t start = hist[hb];
            const uint32_t end = hist[hb + J.U];
            int cur_rr = -1000;
            // sparse bins (FP32): 32 images at a time in list order, no sort; each image's
            // record is computed by its lane and its taps are rotated into the window at once
            const bool sparse = PREC == PREC_FP32 && J.sparse;
            if (sparse) {
                for (uint32_t p0 = start; p0 < end; p0 += 32) {
                    const int n = (int)min(32u, end - p0);
                    float4 rc = make_float4(0.5f, 0.0f, 0.0f, 0.0f);
                    int rr = 0;
                    if (lane < n) {
                        const uint32_t pid = ids[p0 + lane];
                        const int ix = pid & 1023, iy = (pid >> 10) & 1023, iz = pid >> 20;
                        bool bad;
                        float f, amp;
                        ism_delay(T[ix], T[Nx + iy], T[Nx + Ny + iz], q, J.amp_scale, &f, &amp, &rr, &bad, orient,
                                  alpha);
                        if (bad) atomicOr(status, (uint32_t)ISM_DEVICE_FLAG_BIN);
                        f = fminf(fmaxf(f, f_lo), f_hi);
                        rc = ism_sinc_record(f, amp, small_phase, twopi_Nw, inv2Nw);   // amp = 0 if bad
                    }
                    __syncwarp();
                    W.rec[lane] = rc;
                    __syncwarp();
                    for (int l = 0; l < n; ++l)
                        add_single<SLOTS, MASK>(W.rec[l], __shfl_sync(0xffffffffu, rr, l), xj, nsg, Cj, Sj, tap_ok,
                                                halfNw, acc, lane);
                }
            }
            for (uint32_t p0 = start; !sparse && p0 < end; p0 += ISM_PIECE) {
                const int n = (int)min((uint32_t)ISM_PIECE, end - p0);
                const uint32_t* src = ids + p0;

                // ---- phase 1: stable counting sort of the piece by plain-FP32 offset
                W.cnt[lane] = 0;
                if (lane < 2) W.cnt[32 + lane] = 0;
                __syncwarp();
                for (int i0 = 0; i0 < n; i0 += 128) {
                    uint32_t pid[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {  // four loads in flight
                        const int i = i0 + 32 * u + lane;
                        pid[u] = (i < n) ? src[i] : 0u;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int i = i0 + 32 * u + lane;
                        int bucket = -1;
                        if (i < n) {
                            const int ix = pid[u] & 1023, iy = (pid[u] >> 10) & 1023, iz = pid[u] >> 20;
                            const float s2 = __fadd_rn(__fadd_rn(Sh[ix], Sh[Nx + iy]), Sh[Nx + Ny + iz]);
                            const float sp = s2 * ism_rsqrt(s2);
                            const int key = ism_round_int(sp - 0.5f) - ISM_SB * q + 1;  // ~floor(s) - 32q + 1
                            bucket = key < 0 ? 0 : (key > ISM_SB ? ISM_SB : key);
                        }
                        const unsigned peers = __match_any_sync(0xffffffffu, bucket);
                        uint32_t base = 0;
                        if (bucket >= 0) base = W.cnt[bucket];
                        __syncwarp();
                        if (bucket >= 0) {
                            if (lane == __ffs(peers) - 1) W.cnt[bucket] = base + (uint32_t)__popc(peers);
                            W.key[i] = (uint16_t)(bucket | ((base + (uint32_t)__popc(peers & lt_mask)) << 6));
                        }
                        __syncwarp();
                    }
                }
                uint32_t n_pad;
                {   // exclusive prefix over the 33 bucket sizes rounded up to 4
                    const uint32_t v = (W.cnt[lane] + 3u) & ~3u;
                    uint32_t inc = v;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t nn = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += nn;
                    }
                    const uint32_t tot32 = __shfl_sync(0xffffffffu, inc, 31);
                    n_pad = tot32 + ((W.cnt[32] + 3u) & ~3u);
                    W.off[lane] = inc - v;
                    if (lane == 0) W.off[32] = tot32;
                }
                __syncwarp();
                {   // dummies completing each bucket to a multiple of 4 (they carry their bucket)
                    for (int b = lane; b < ISM_NB; b += 32) {
                        const uint32_t c = W.cnt[b], o = W.off[b];
                        for (uint32_t k = c; k < ((c + 3u) & ~3u); ++k) W.sorted[o + k] = ISM_DUMMY | (uint32_t)b;
                        for (uint32_t k = 0; k < c; k += 4) W.group_bucket[(o + k) >> 2] = (uint8_t)b;
                    }
                }
                for (int i0 = 0; i0 < n; i0 += 128) {
                    uint32_t pid[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int i = i0 + 32 * u + lane;
                        pid[u] = (i < n) ? src[i] : 0u;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int i = i0 + 32 * u + lane;
                        if (i < n) {
                            const uint32_t k = W.key[i];
                            W.sorted[W.off[k & 63u] + (k >> 6)] = pid[u];
                        }
                    }
                }
                __syncwarp();

                // ---- phase 2: exact records, 64 at a time in sorted order; each group of 4
                // entries shares its bucket offset, so runs are checked once per group
                for (int c0 = 0; c0 < (int)n_pad; c0 += ISM_CHUNK) {
                    const int m = min(ISM_CHUNK, (int)n_pad - c0);  // a multiple of 4
                    unsigned strays[2];
                    float4 rc_l[2];
                    int rr_l[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int i = c0 + 32 * h + lane;
                        float4 rc = make_float4(0.5f, 0.0f, 0.0f, 0.0f);   // FP32 record (dummy: no amplitude)
                        float4 rl = make_float4(0.0f, 0.0f, 0.0f, 0.0f);   // LUT record
                        int rr = 0;
                        bool stray = false;
                        if (i < c0 + m) {
                            const uint32_t pid = W.sorted[i];
                            const int rr_bucket = (int)W.group_bucket[i >> 2] - 1;
                            rr = rr_bucket;
                            if (!(pid & ISM_DUMMY)) {
                                const int ix = pid & 1023, iy = (pid >> 10) & 1023, iz = pid >> 20;
                                bool bad;
                                float f, amp;
                                ism_delay(T[ix], T[Nx + iy], T[Nx + Ny + iz], q, J.amp_scale, &f, &amp, &rr, &bad,
                                          orient, alpha);
                                if (bad) atomicOr(status, (uint32_t)ISM_DEVICE_FLAG_BIN);
                                stray = rr != rr_bucket;
                                f = fminf(fmaxf(f, f_lo), f_hi);
                                if constexpr (PREC == PREC_TEX) {
                                    // texel row f Q, centred: the texture interpolates rows floor and + 1
                                    rl = make_float4(amp, __fmaf_rn(f, (float)LQ, 0.5f), 0.0f, 0.0f);
                                    if (stray) rc = ism_sinc_record(f, amp, small_phase, twopi_Nw, inv2Nw);
                                } else if constexpr (PREC == PREC_LUT) {
                                    const float u = f * (float)LQ;        // exact: LQ is a power of two
                                    const float pf = floorf(u);
                                    const float ph = u - pf;              // exact
                                    rl = make_float4(amp - amp * ph, amp * ph,
                                                     __int_as_float(ism_int_of_integral(pf) * ROW), 0.0f);
                                    if (stray) rc = ism_sinc_record(f, amp, small_phase, twopi_Nw, inv2Nw);
                                } else {
                                    rc = ism_sinc_record(f, amp, small_phase, twopi_Nw, inv2Nw);
                                }
                            }
                        }
                        if constexpr (PREC == PREC_FP32) {
                            W.rec[32 * h + lane] = stray ? make_float4(rc.x, 0.0f, 0.0f, 0.0f) : rc;
                        } else if constexpr (PREC == PREC_LUT || PREC == PREC_TEX) {
                            W.rec[32 * h + lane] = stray ? make_float4(0.0f, 0.0f, 0.0f, 0.0f) : rl;
                        } else {
                            // pack the records of lanes 2k (a) and 2k + 1 (b) into one pair
                            const float Pa = stray ? 0.0f : rc.y * rscale;
                            const float Pca = stray ? 0.0f : rc.z * rscale;
                            const float Psa = stray ? 0.0f : rc.w * rscale;
                            const float fb = __shfl_down_sync(0xffffffffu, rc.x, 1);
                            const float Pb = __shfl_down_sync(0xffffffffu, Pa, 1);
                            const float Pcb = __shfl_down_sync(0xffffffffu, Pca, 1);
                            const float Psb = __shfl_down_sync(0xffffffffu, Psa, 1);
                            if ((lane & 1) == 0) {
                                uint4* recp = reinterpret_cast<uint4*>(W.rec);
                                uint32_t* ps2 = reinterpret_cast<uint32_t*>(W.rec + 32);
                                recp[16 * h + (lane >> 1)] = make_uint4(__float_as_uint(rc.x), __float_as_uint(fb),
                                                                        pack2<PREC>(Pa, Pb), pack2<PREC>(Pca, Pcb));
                                ps2[16 * h + (lane >> 1)] = pack2<PREC>(Psa, Psb);
                            }
                        }
                        strays[h] = __ballot_sync(0xffffffffu, stray);
                        rc_l[h] = rc;
                        rr_l[h] = rr;
                    }
                    // offsets of the (up to) 16 groups of this chunk; bit g of `chg` set
                    // where group g starts a new run
                    const int ng = m >> 2;
                    const int rr_grp = (lane < ng) ? (int)W.group_bucket[(c0 >> 2) + lane] - 1 : 0;
                    const int rr_prev = __shfl_up_sync(0xffffffffu, rr_grp, 1);
                    const unsigned chg =
                        __ballot_sync(0xffffffffu, lane < ng && (lane == 0 ? rr_grp != cur_rr : rr_grp != rr_prev));
                    __syncwarp();
                    for (int g = 0; g < ng; ++g) {
                        if (chg & (1u << g)) {  // warp-uniform: a new offset starts here
                            if (cur_rr > -1000) {
#pragma unroll
                                for (int s = 0; s < SLOTS; ++s) {
                                    D[s] += D2[s];
                                    D2[s] = 0.0f;
                                }
                                flush_run<SLOTS, PREC == PREC_FP16>(D, acc, cur_rr, lane, dscale);
                            }
                            cur_rr = __shfl_sync(0xffffffffu, rr_grp, g);
                        }
                        if constexpr (PREC == PREC_FP32) {
                            const float4 r0 = W.rec[4 * g], r1 = W.rec[4 * g + 1], r2 = W.rec[4 * g + 2],
                                         r3 = W.rec[4 * g + 3];
                            // two interleaved accumulators shorten the dependent FFMA chain
                            taps<SLOTS, MASK>(r0, xj, nsg, Cj, Sj, tap_ok, halfNw, D);
                            taps<SLOTS, MASK>(r1, xj, nsg, Cj, Sj, tap_ok, halfNw, D2);
                            taps<SLOTS, MASK>(r2, xj, nsg, Cj, Sj, tap_ok, halfNw, D);
                            taps<SLOTS, MASK>(r3, xj, nsg, Cj, Sj, tap_ok, halfNw, D2);
                        } else if constexpr (PREC == PREC_TEX) {
                            const float4 r0 = W.rec[4 * g], r1 = W.rec[4 * g + 1], r2 = W.rec[4 * g + 2],
                                         r3 = W.rec[4 * g + 3];
                            taps_tex<SLOTS>(r0, J.lut_tex, lane, D);
                            taps_tex<SLOTS>(r1, J.lut_tex, lane, D2);
                            taps_tex<SLOTS>(r2, J.lut_tex, lane, D);
                            taps_tex<SLOTS>(r3, J.lut_tex, lane, D2);
                        } else if constexpr (PREC == PREC_LUT) {
                            const float4 r0 = W.rec[4 * g], r1 = W.rec[4 * g + 1], r2 = W.rec[4 * g + 2],
                                         r3 = W.rec[4 * g + 3];
                            taps_lut<SLOTS, ROW>(r0, lut_lane, D);
                            taps_lut<SLOTS, ROW>(r1, lut_lane, D2);
                            taps_lut<SLOTS, ROW>(r2, lut_lane, D);
                            taps_lut<SLOTS, ROW>(r3, lut_lane, D2);
                        } else {
                            const uint4* recp = reinterpret_cast<const uint4*>(W.rec);
                            const uint32_t* ps2 = reinterpret_cast<const uint32_t*>(W.rec + 32);
                            const uint4 p0 = recp[2 * g], p1 = recp[2 * g + 1];
                            const uint32_t s0 = ps2[2 * g], s1 = ps2[2 * g + 1];
                            taps_pair<SLOTS, MASK, PREC>(p0, s0, xj, nsg, C2, S2, tap_ok, halfNw, D, D2);
                            taps_pair<SLOTS, MASK, PREC>(p1, s1, xj, nsg, C2, S2, tap_ok, halfNw, D, D2);
                        }
                    }
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        unsigned sm = strays[h];
                        while (sm) {  // images sorted next to an integer boundary of their delay
                            const int l = __ffs(sm) - 1;
                            sm &= sm - 1;
                            const float4 rs = make_float4(__shfl_sync(0xffffffffu, rc_l[h].x, l),
                                                          __shfl_sync(0xffffffffu, rc_l[h].y, l),
                                                          __shfl_sync(0xffffffffu, rc_l[h].z, l),
                                                          __shfl_sync(0xffffffffu, rc_l[h].w, l));
                            add_single<SLOTS, MASK>(rs, __shfl_sync(0xffffffffu, rr_l[h], l), xj, nsg, Cj, Sj, tap_ok,
                                                    halfNw, acc, lane);
                        }
                    }
                    __syncwarp();
                }
            }
            if (cur_rr > -1000) {
#pragma unroll
                for (int s = 0; s < SLOTS; ++s) {
                    D[s] += D2[s];
                    D2[s] = 0.0f;
                }
                flush_run<SLOTS, PREC == PREC_FP16>(D, acc, cur_rr, lane, dscale);
            }
        }
        if (q < J.Q) {
            float* row = rows + J.rows_base + ((long long)r * J.Q + q) * WIN;
#pragma unroll
            for (int m = 0; m <= SLOTS; ++m) row[32 * m + lane] = acc[m];
        }
    }
}

template <int SLOTS, bool MASK, int PREC>
int launch_one(const JobTable& t, const WsPlan& p, char* ws, cudaStream_t s)
{
    constexpr int BPC = ism_acc_bins(PREC);
    const size_t lut_bytes =
        PREC == PREC_LUT ? (size_t)(ism_lut_phases(SLOTS) + 1) * 32 * SLOTS * sizeof(float) : 0;
    size_t sm = (size_t)((t.max_axis_sum + 1) & ~1) * sizeof(float4) + lut_bytes + BPC * sizeof(WarpSmem) +
                (size_t)t.max_axis_sum * sizeof(float);
    static std::atomic<unsigned long long> opened{0};
    int rc = ism_open_smem((const void*)accum_kernel<SLOTS, MASK, PREC>, &opened);
    if (rc) return rc;
    accum_kernel<SLOTS, MASK, PREC><<<(unsigned)p.acc_ctas, BPC * 32, sm, s>>>(
        t, reinterpret_cast<const float4*>(ws + p.tbl_off), reinterpret_cast<const uint32_t*>(ws + p.hist_off),
        reinterpret_cast<const uint32_t*>(ws + p.ids_off), reinterpret_cast<const float*>(ws + p.lut_off),
        reinterpret_cast<float*>(ws + p.rows_off), reinterpret_cast<uint32_t*>(ws + p.status_off));
    return (int)cudaGetLastError();
}

// Launches the instantiations of precision PREC that the jobs of the table
// need (one per window length and mask; the LUT form has no mask variant).
template <int PREC>
int launch_accum_prec(const JobTable& t, const WsPlan& p, char* ws, void* stream, int* launched)
{
    *launched = 0;
    if (p.acc_ctas <= 0) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    bool need[2][ISM_MAX_SLOTS + 1] = {};
    for (int i = 0; i < t.n_jobs; ++i) {
        const JobDev& J = t.j[i];
        if (J.use_cheb) continue;
        bool exact = (J.Nw == (float)(2 * J.H)) && (2 * J.H == 32 * J.slots);
        need[(exact || PREC == PREC_LUT || PREC == PREC_TEX) ? 0 : 1][J.slots] = true;
    }
    int rc = 0;
#define ISM_L(SL)                                                                            \
    if (!rc && need[0][SL]) rc = launch_one<SL, false, PREC>(t, p, ws, s), ++*launched;      \
    if constexpr (PREC != PREC_LUT && PREC != PREC_TEX)                                      \
        if (!rc && need[1][SL]) rc = launch_one<SL, true, PREC>(t, p, ws, s), ++*launched;
    ISM_L(1) ISM_L(2) ISM_L(3) ISM_L(4) ISM_L(5) ISM_L(6) ISM_L(7) ISM_L(8)
#undef ISM_L
    return rc;
}

}  // namespace
