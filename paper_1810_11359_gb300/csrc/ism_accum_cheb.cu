// ism_accum_cheb.cu -- FP32 accumulation of eq. (5) for a 32-tap window
// through a Chebyshev expansion of the windowed sinc in the fractional delay,
// fused with the enumeration of the images (Section 2.1) it accumulates.
//
// For tap j of an image with delay s = b + f (b integer, f in [0, 1)), the
// sample b + j receives A delta'(j - f) (eq. (6)).  For a window of exactly
// N_w = 32 taps every tap function g_j(f) = delta'(j - f), j = -15 .. 16, is
// an entire function of f on [0, 1] (the window's zeros fall at the ends of
// the interval, so no mask cuts it), and its Chebyshev series in u = 2f - 1
// converges fast: degree 7 reproduces each g_j to 4.2e-7 of the image's
// amplitude (degree 8: 6.4e-8; degree 9: 2.1e-9), about twice the fixed-point
// step of the moment terms (see below); together they keep an RIR within a few
// 1e-7 of its peak, far inside FP32's 1e-5, and degree 7 spares one shared-
// memory atomic per image against degree 8.  The coefficients c_{j,i},
// interpolated at the 8 Chebyshev-Gauss nodes in FP64 on the host, travel in
// the kernel's parameter table.  Hence for the images that share the integer
// delay b,
//   sum_n A_n g_j(f_n) = sum_i c_{j,i} M_i,   M_i = sum_n A_n T_i(2 f_n - 1),
// so each image costs 8 moment terms instead of 32 tap evaluations, and each
// integer delay costs 8 FMAs per tap once.
//
// Delay bins.  Bin q holds the images with b in [32 q - 1, 32 q + 31), i.e.
// offsets rr = b - 32 q in [-1, 30] (32 offsets, one per lane); its taps fall
// in the 64 samples from 32 q - 16, the bin's window row, which the finalize
// kernel sums per sample with the previous bin's row.  An image is kept iff a
// tap reaches a sample below n_ism: b <= n_ism + 14.
//
// One CTA owns B = 8 consecutive bins of one RIR -- a spherical shell of
// 256 samples around the receiver (thinner, down to one bin, when a launch
// has too few RIRs to fill the GPU) -- and enumerates the images in it itself
// (ism_shell.cuh): each candidate's exact float-float delay decides its bin,
// so every image lands in exactly one CTA, the one whose bins hold its b.
//
// Fixed point.  Every image of bin q has s >= max(s_direct, 32 q - 1) (the
// direct path is the shortest: along each axis the source's own coordinate is
// the image coordinate nearest the receiver) and at least d / L_max - 3 wall
// hits (|n| >= |x_n - x_r| / L - 1 on each axis), so |A| <= A_max = amp_scale
// beta_max^h / s_lo.  A term A T_i is scaled by 2^e and rounded to an integer
// (one FFMA against 1.5 2^23: the sum's bits hold the integer), e the largest
// integer with 2^e A_max <= min((1 - 2^-10) 2^22, 0.98 2^31 / n - 1), n first
// four times the expected number of images per integer delay, 4 pi s^2 /
// (k^3 V) (one image per room volume V), plus 64.  The sums are 32-bit
// shared-memory atomic adds of the FFMA's raw bits K + v (K = 0x4B400000, the
// bits of 1.5 2^23; v the term's integer); with n images at the integer delay
// the sum of the v is the word minus n K, modulo 2^32, exact while it stays
// below 2^31 in magnitude.  Integer addition is associative, so the sums --
// and the FP32 result -- are the same in every run, whatever the order in
// which lanes and warps add their terms.  The CTA also counts its images per (bin,
// integer delay); if some count times the largest term could reach 2^31 a sum
// may have wrapped, and the CTA redoes its shell with scales set from the exact
// counts (which do not depend on the scales), so the second pass is safe.  The
// rounding error is at most 2^-22 A_max per term wherever the counts stay below
// ~500 per integer delay; A_max falls with the distance and the wall hits.
//
// Finally each warp expands the non-empty offsets of one bin into the taps
// (lane = tap) and rotates them into the bin's register window, which it
// stores as the bin's row; the moments of an offset sit together (8 floats),
// so a warp reads them in two broadcast loads.
#include "ism_accum.cuh"
#include "ism_shell.cuh"

namespace {

#define SH_B ISM_SHELL_BINS  // delay bins per CTA (a shell of 256 samples)
#define SH_WARPS 8          // warps per CTA
#define SH_NO 32            // offsets per bin (rr = -1 .. 30)
#define SH_RS 33            // row stride of the moment table (conflict-light atomics)
#define CB_MAGIC 12582912.0f                       // 1.5 * 2^23
static_assert(ISM_CHEB_NF == 8, "the expansion reads the moments as 4 + 4");
// the expansion's moment table [bin][offset][8] overlays the sums, the counts, the scales, the
// row prefix and the column records (all dead by then), which always span more than it needs
static_assert(SH_B * SH_NO * 8 * 4 <= (SH_B * ISM_CHEB_NF * SH_RS + SH_B * SH_RS) * 4 + SH_WARPS * 32 * 32,
              "moment table larger than the tables it overlays");
#define CB_MAGIC_BITS 0x4B400000u                  // its bits

// Largest power of two 2^e with 2^e a_max <= min((1 - 2^-10) 2^22, 0.98 2^31 / n - 1):
// no term reaches 2^22 (the FFMA rounding trick) and n terms cannot sum to 2^31.
__device__ __forceinline__ float shell_scale(float a_max, float n)
{
    const float cap = fminf(4194304.0f * (1.0f - 1.0f / 1024.0f), 0.98f * 2147483648.0f / fmaxf(n, 1.0f) - 1.0f);
    const float ratio = a_max > 0.0f ? cap / a_max : 3.0e38f;
    int e = ((__float_as_int(ratio) >> 23) & 0xFF) - 127;   // floor(log2(ratio)), ratio normal
    e = max(-126, min(126, e));
    return __int_as_float((e + 127) << 23);
}

__global__ void __launch_bounds__(SH_WARPS * 32, 5) shell_kernel(const __grid_constant__ JobTable t,
                                                                  const float4* __restrict__ tbl,
                                                                  float* __restrict__ rows,
                                                                  uint32_t* __restrict__ status)
{
    constexpr int WIN = 64;   // 32 (SLOTS + 1), SLOTS = 1
    extern __shared__ __align__(16) unsigned char smem[];
    int jid, r, grp;
    if (!shell_cta(t, blockIdx.x, &jid, &r, &grp)) return;   // CTA-uniform
    const JobDev& J = t.j[jid];
    const int B = t.shell_bins;   // bins of this launch's shells: SH_B, fewer for small launch sets
    const int q0 = grp * B;
    const int nb = min(B, J.Q - q0);
    const int Nx = J.N[0], Ny = J.N[1], Nz = J.N[2];
    const int n_axis = Nx + Ny + Nz;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // shared memory: axis tables | moment sums | image counts | per-bin scales | row prefix |
    // per-warp column records
    float4* T = reinterpret_cast<float4*>(smem);
    unsigned* S = reinterpret_cast<unsigned*>(smem + (size_t)((t.max_axis_sum + 1) & ~1) * sizeof(float4));
    int* Cn = reinterpret_cast<int*>(S + SH_B * ISM_CHEB_NF * SH_RS);             // [bin][offset] images
    float* scale_s = reinterpret_cast<float*>(Cn + SH_B * SH_RS);
    float* inv_s = scale_s + SH_B;
    float* amax_s = inv_s + SH_B;                                                 // per-bin amplitude bound
    int* redo = reinterpret_cast<int*>(amax_s + SH_B);                            // [4]: retry flag
    int* rowpre = reinterpret_cast<int*>(redo + 4);                             // [Nx]: columns up to row ix
    int* rowy0 = rowpre + ((t.max_axis_sum + 4) & ~3);                          // [Nx]: first iy of row ix
    float4* recf = reinterpret_cast<float4*>(rowy0 + ((t.max_axis_sum + 4) & ~3));
    int4* reci = reinterpret_cast<int4*>(recf + SH_WARPS * 32);
    int* st = reinterpret_cast<int*>(reci + SH_WARPS * 32);                     // [warps][33]
    float4* Wf = recf + warp * 32;
    int4* Wi = reci + warp * 32;
    int* Wst = st + warp * 33;

    const float4* Tg = tbl + J.tbl_base + (long long)r * n_axis;
    for (int e = threadIdx.x; e < n_axis; e += blockDim.x) T[e] = Tg[e];
    if (threadIdx.x == 0) *redo = 0;
    __syncthreads();

    // receiver polar pattern: the unit orientation of this RIR's receiver (|g| <= 1 keeps A_max a bound)
    const int i_rcv = r - (r / J.n_rcv) * J.n_rcv;
    const float alpha = J.mic_alpha;
    float3 orient = make_float3(0.0f, 0.0f, 0.0f);
    if (alpha != 1.0f) {
        const float* o = J.orient_rcv + 3 * i_rcv;
        const float ox = o[0], oy = o[1], oz = o[2];
        const float inv = 1.0f / sqrtf(__fmaf_rn(ox, ox, __fmaf_rn(oy, oy, oz * oz)));
        orient = make_float3(ox * inv, oy * inv, oz * inv);
    }
    // exact delays b owned by this CTA: [b_lo, b_hi), b <= n_ism + 14 for H = 16
    const Shell sh = shell_setup(J, T, r, ISM_SB * q0 - 1, min(ISM_SB * (q0 + nb) - 1, J.n_ism + J.H - 1));
    const float kinv = sh.kinv;
    const float sd2 = sh.sd2;
    const bool valid = sh.valid;

    if (threadIdx.x < SH_B) {
        // fixed-point scale of bin q0 + threadIdx.x, first from the expected number of images
        // per integer delay (verified, and redone from the exact counts if it was too small)
        const int q = q0 + (int)threadIdx.x;
        float sc = 1.0f, amax = 0.0f;
        if (q < J.Q && valid) {
            const float slo = fmaxf(fmaxf(sqrtf(sd2) * (1.0f - 1.0f / 1024.0f), (float)(ISM_SB * q) - 1.0f), 1e-30f);
            float bmax = 0.0f;
            for (int w = 0; w < 6; ++w) bmax = fmaxf(bmax, fabsf(ism_job_beta(J, w)));
            const int h = max(0, (int)floorf(slo * kinv / J.Lmax - 3.0f));
            const float decay = (h == 0) ? 1.0f : (bmax > 0.0f ? exp2f((float)h * log2f(bmax)) : 0.0f);
            amax = J.amp_scale / slo * decay * 1.001f;
            // images per integer delay at s: 4 pi s^2 / (k^3 V) (one image per volume V)
            const float shi = (float)(ISM_SB * q + ISM_SB);
            const float k = 1.0f / kinv;
            const float vol = J.vol;
            const float n_est = 4.0f * (12.566371f * shi * shi / (k * k * k * vol)) + 64.0f;
            sc = shell_scale(amax, n_est);
        }
        scale_s[threadIdx.x] = sc;
        inv_s[threadIdx.x] = 1.0f / sc;   // exact: a power of two
        amax_s[threadIdx.x] = amax;
    }
    const int n_cols = shell_rows(sh, T, rowpre, rowy0);   // (synchronises the CTA)

    const float amp_scale = J.amp_scale;
    for (int pass = 0; pass < 2; ++pass) {
    for (int e = threadIdx.x; e < SH_B * ISM_CHEB_NF * SH_RS; e += blockDim.x) S[e] = 0;
    for (int e = threadIdx.x; e < SH_B * SH_RS; e += blockDim.x) Cn[e] = 0;
    __syncthreads();
    shell_walk<SH_WARPS>(sh, T, rowpre, rowy0, n_cols, make_float2(orient.x, orient.y), Wf, Wi, Wst, warp, lane,
                         [&](int b, float f, float s, const float4& cf, int, int, const float4& tz) {
        const int q = (b + 1) >> 5;
        const int ql = q - q0;
        const int o = b - ISM_SB * q + 1;   // offset index rr + 1 in [0, 32)
        const float rs = ism_rcp(s);
        float amp = cf.z * tz.z * amp_scale * rs;
        if (alpha != 1.0f)   // polar pattern: cos(theta) = o . (x_n - x_r) / d
            amp *= __fmaf_rn(1.0f - alpha, __fmaf_rn(orient.z, tz.w, cf.w) * rs, alpha);
        const float as = amp * scale_s[ql];
        const float uu = __fmaf_rn(2.0f, f, -1.0f);
        const float u2 = uu + uu;
        unsigned* Sb = S + ql * (ISM_CHEB_NF * SH_RS) + o;
        atomicAdd(Cn + ql * SH_RS + o, 1);
        atomicAdd(Sb, __float_as_uint(__fadd_rn(as, CB_MAGIC)));   // K + v: the n K go at the expansion
        atomicAdd(Sb + SH_RS, __float_as_uint(__fmaf_rn(as, uu, CB_MAGIC)));
        float tp = 1.0f, tc = uu;
#pragma unroll
        for (int k = 2; k < ISM_CHEB_NF; ++k) {
            const float tn = __fmaf_rn(u2, tc, -tp);
            atomicAdd(Sb + k * SH_RS, __float_as_uint(__fmaf_rn(as, tn, CB_MAGIC)));
            tp = tc;
            tc = tn;
        }
    });
    __syncthreads();
    // every sum of bin q holds at most Cn[q][o] terms of magnitude <= scale * A_max + 1/2:
    // below 2^31 means no sum can have wrapped; otherwise redo the shell with scales from
    // the exact counts (the counts do not depend on the scales, so the second pass is safe)
    if (pass == 0 && threadIdx.x < SH_B) {
        int mx = 0;
        for (int o = 0; o < SH_NO; ++o) mx = max(mx, Cn[threadIdx.x * SH_RS + o]);
        const float bound = (float)mx * (scale_s[threadIdx.x] * amax_s[threadIdx.x] + 0.5f);
        if (!(bound < 0.99f * 2147483648.0f)) {
            const float sc = shell_scale(amax_s[threadIdx.x], (float)mx);
            scale_s[threadIdx.x] = sc;
            inv_s[threadIdx.x] = 1.0f / sc;
            atomicOr(redo, 1);
        }
    }
    __syncthreads();
    if (!*redo || pass == 1) break;   // CTA-uniform
    }

    // ---- expansion: warp w owns bin q0 + w; lane o reads the sums of offset o
    float m[ISM_CHEB_NF];
    bool any = false;
    if (warp < nb) {
        const unsigned* Sb = S + warp * (ISM_CHEB_NF * SH_RS);
        const unsigned nk = (unsigned)Cn[warp * SH_RS + lane] * CB_MAGIC_BITS;   // n K (mod 2^32)
        const float inv = inv_s[warp];
#pragma unroll
        for (int k = 0; k < ISM_CHEB_NF; ++k) {
            const int v = (int)(Sb[k * SH_RS + lane] - nk);
            any |= v != 0;
            m[k] = __int2float_rn(v) * inv;   // exact scaling by a power of two
        }
    }
    __syncthreads();   // every sum is read before the moment table overwrites the CTA's tables
    if (warp >= nb) return;
    const int q = q0 + warp;
    // moments of (bin, offset o) at Mt + 2 (32 bin + o): {M_0..M_3}, {M_4..M_7}
    float4* Mt = reinterpret_cast<float4*>(S);
    {
        float4* mo = Mt + 2 * (32 * warp + lane);
        mo[0] = make_float4(m[0], m[1], m[2], m[3]);
        mo[1] = make_float4(m[4], m[5], m[6], m[7]);
    }
    const unsigned nonempty = __ballot_sync(0xffffffffu, any);
    __syncwarp();
    float c[ISM_CHEB_NF];   // lane = tap t: Chebyshev coefficients of g_(t - 15)
#pragma unroll
    for (int i = 0; i < ISM_CHEB_NF; ++i) c[i] = t.cheb[lane * ISM_CHEB_N + i];
    float acc[2] = {0.0f, 0.0f};
    for (int o = 0; o < SH_NO; ++o) {
        if (!((nonempty >> o) & 1u)) continue;   // warp-uniform
        const float4* mo = Mt + 2 * (32 * warp + o);
        const float4 ma = mo[0], mb = mo[1];
        const float mv[ISM_CHEB_NF] = {ma.x, ma.y, ma.z, ma.w, mb.x, mb.y, mb.z, mb.w};
        float D[1];
        D[0] = c[0] * mv[0];
#pragma unroll
        for (int k = 1; k < ISM_CHEB_NF; ++k) D[0] = __fmaf_rn(c[k], mv[k], D[0]);
        flush_run<1, false>(D, acc, o - 1, lane, 1.0f);
    }
    float* row = rows + J.rows_base + ((long long)r * J.Q + q) * WIN;
    row[lane] = acc[0];
    row[32 + lane] = acc[1];
}

size_t shell_smem(const JobTable& t)
{
    return (size_t)((t.max_axis_sum + 1) & ~1) * sizeof(float4) + (size_t)SH_B * ISM_CHEB_NF * SH_RS * sizeof(int) +
           (size_t)SH_B * SH_RS * sizeof(int) + 3 * SH_B * sizeof(float) + 4 * sizeof(int) +
           2 * (size_t)((t.max_axis_sum + 4) & ~3) * sizeof(int) +
           (size_t)SH_WARPS * 32 * (sizeof(float4) + sizeof(int4)) + (size_t)SH_WARPS * 33 * sizeof(int);
}

}  // namespace

int ism_launch_accum_cheb(const JobTable& t, const WsPlan& p, char* ws, void* stream, int* launched)
{
    *launched = 0;
    if (p.shell_ctas <= 0 || !t.any_cheb) return 0;
    const size_t sm = shell_smem(t);
    static std::atomic<unsigned long long> opened{0};
    int rc = ism_open_smem((const void*)shell_kernel, &opened);
    if (rc) return rc;
    // all of the unified L1 as shared memory: 5 CTAs of ~27 KB per SM
    cudaError_t e = cudaFuncSetAttribute(shell_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return (int)e;
    shell_kernel<<<(unsigned)p.shell_ctas, SH_WARPS * 32, sm, (cudaStream_t)stream>>>(
        t, reinterpret_cast<const float4*>(ws + p.tbl_off), reinterpret_cast<float*>(ws + p.rows_off),
        reinterpret_cast<uint32_t*>(ws + p.status_off));
    *launched = 1;
    return (int)cudaGetLastError();
}
