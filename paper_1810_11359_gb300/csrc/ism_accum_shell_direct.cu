// ism_accum_shell_direct.cu -- FP32 accumulation of eq. (5) with every tap of
// eq. (6) evaluated, for a 32-tap window, fused with the enumeration of the
// images (Section 2.1) it accumulates.
//
// The Chebyshev form (ism_accum_cheb.cu) pays for the expansion of every
// occupied integer delay; with few images per delay bin (the 48 kHz array:
// ~36 per bin) evaluating each image's 32 taps is cheaper.  Before this kernel
// such jobs went through an enumeration count, a scan and a scatter of image
// ids into delay bins; here the CTA that owns a shell of delay bins of one
// RIR enumerates the shell's images itself (ism_shell.cuh, as the Chebyshev
// form does) and adds their taps at once, so no ids, counts or sorts exist.
// The shells are 32 bins thick (1024 samples) when the bins hold few images:
// visiting the grid columns that reach a shell is what thickness amortises;
// dense rooms take 8 bins, so that their RIRs still split into many CTAs.
// The candidates of every chunk of columns form batches of 32 dealt to the
// CTA's warps in turn (ism_shell.cuh, shell_walk_cta), so no warp waits for
// another by more than one batch.
//
// Each lane that finds an image computes its record {f, P, P cos phi,
// P sin phi} (the factorised windowed sinc of ism_accum.cuh: P = A sin(pi f) /
// (2 pi), phi = 2 pi f / N_w) and the position of its first tap in the
// shell's window (32 B + 32 samples from 32 q0 - 16, B bins), and puts them
// in its warp's ring of staged records in shared memory, after the images
// already waiting, in lane order.  Whenever 32 images wait, the warp takes
// them two at a time, and lane t adds tap t of each -- sigma_t (t - 15 - f) by
// one FFMA, the window by two, one reciprocal and one product, the FMAs and
// the product issued as packed f32x2 operations on the pair -- to its warp's
// window of the shell in shared memory (consecutive lanes, consecutive
// addresses).  The order in which a warp meets and adds its images is a
// function of the geometry alone (ism_shell.cuh), so the warp windows are the
// same in every run; at the end they are summed in warp order.  No atomics:
// the output is bit-identical from run to run.
//
// The shell's window is written as the bins' window rows of the finalize
// kernel (64 samples from 32 q - 16, summed per sample with the previous
// bin's row): each bin's row holds the window's values on its first 32
// samples and zeros on the rest, except the last bin of the shell, whose
// upper half holds the 32 samples that spill into the next shell.
#include "ism_accum.cuh"
#include "ism_shell.cuh"

namespace {

// Two FP32 values in one 64-bit register pair, and the packed FP32 operations of
// sm_100-class GPUs on them (both lanes rounded as the scalar operations are).
__device__ __forceinline__ unsigned long long sd_pack(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void sd_unpack(unsigned long long r, float& a, float& b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long sd_fma2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long sd_mul2(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

#define SD_B ISM_SD_BINS             // delay bins per CTA, at most
#define SD_WARPS 8                   // warps per CTA
#define SD_RING 64                   // staged image records per warp (a ring; 32 are added at once)

// Window of a warp: the taps of b in [32 q0 - 1, 32 (q0 + B) - 1) fall in the 32 B + 32
// samples from 32 q0 - 16, then 32 samples where the padding record of an odd count adds 0.
__host__ __device__ __forceinline__ int sd_win(int B) { return 32 * B + 32; }
__host__ __device__ __forceinline__ int sd_winp(int B) { return sd_win(B) + 32; }

template <int PREC>
__global__ void __launch_bounds__(SD_WARPS * 32, 4) shell_direct_kernel(const __grid_constant__ JobTable t,
                                                                        const float4* __restrict__ tbl,
                                                                        const float* __restrict__ lut_g,
                                                                        float* __restrict__ rows, int winp)
{
    constexpr bool HALF = PREC == PREC_FP16 || PREC == PREC_BF16;
    constexpr int LQ = ism_lut_phases(1);   // table phases per sample (LUT forms)
    constexpr int WIN = 64;   // window row of a bin: 32 (SLOTS + 1), SLOTS = 1
    extern __shared__ __align__(16) unsigned char smem[];
    // CTA -> (job, RIR, shell): by the shell's rank from the outside over all RIRs of the
    // launch (every RIR's outermost, densest shell first, the lightest at the end of the
    // launch) when the jobs' shell counts are alike, else job by job, RIR by RIR, densest
    // shell first
    const long long g = blockIdx.x;
    int jid, r, grp;
    if (t.sd_rank_rirs) {
        const int k = (int)(g / t.sd_rank_rirs);
        const int rr = (int)(g - (long long)k * t.sd_rank_rirs);
        jid = ism_find_job(t, rr, [](const JobDev& d) { return (long long)d.sd_rir_base; });
        r = rr - t.j[jid].sd_rir_base;
        grp = t.j[jid].shell_groups - 1 - k;
        if (grp < 0) return;   // past the job's shells (CTA-uniform)
    } else {
        jid = ism_find_job(t, g, [](const JobDev& d) { return (long long)d.sd_cta_base; });
        const long long local = g - t.j[jid].sd_cta_base;
        r = (int)(local / t.j[jid].shell_groups);
        grp = t.j[jid].shell_groups - 1 - (int)(local % t.j[jid].shell_groups);
    }
    const JobDev& J = t.j[jid];
    const int B = J.shell_direct;   // bins per shell: 8 (dense rooms) or 32 (sparse ones)
    const int q0 = grp * B;
    const int nb = min(B, J.Q - q0);
    const int Nx = J.N[0], Ny = J.N[1], Nz = J.N[2];
    const int n_axis = Nx + Ny + Nz;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int win = sd_win(nb);   // this shell's window (the padding row follows it)

    // shared memory: axis tables | row prefix | per-warp column records | per-warp staged
    // images | per-warp windows (winp floats each: the launch's thickest shell)
    float4* T = reinterpret_cast<float4*>(smem);
    int* rowpre = reinterpret_cast<int*>(smem + (size_t)((t.max_axis_sum + 1) & ~1) * sizeof(float4));
    int* rowy0 = rowpre + ((t.max_axis_sum + 4) & ~3);
    float4* recf = reinterpret_cast<float4*>(rowy0 + ((t.max_axis_sum + 4) & ~3));
    int4* reci = reinterpret_cast<int4*>(recf + SD_WARPS * 32);
    int* st = reinterpret_cast<int*>(reci + SD_WARPS * 32);                          // [warps][33]
    float4* stage_all = reinterpret_cast<float4*>(st + SD_WARPS * 33 + 8);           // [warps][SD_RING]
    int* spos_all = reinterpret_cast<int*>(stage_all + SD_WARPS * SD_RING);           // [warps][SD_RING]
    int* wtot = spos_all + SD_WARPS * SD_RING;                                        // [warps]
    float* win_all = reinterpret_cast<float*>(wtot + SD_WARPS);                       // [warps][winp]
    float* winl = win_all + warp * winp + lane;   // lane's column of the warp's window
    float4* stage = stage_all + warp * SD_RING;
    int* spos = spos_all + warp * SD_RING;

    const float4* Tg = tbl + J.tbl_base + (long long)r * n_axis;
    for (int e = threadIdx.x; e < n_axis; e += blockDim.x) T[e] = Tg[e];
    for (int w = 0; w < SD_WARPS; ++w)
        for (int e = threadIdx.x; e < win + 32; e += blockDim.x) win_all[w * winp + e] = 0.0f;
    __syncthreads();

    // receiver polar pattern: the unit orientation of this RIR's receiver
    const int i_rcv = r - (r / J.n_rcv) * J.n_rcv;
    const float alpha = J.mic_alpha;
    float3 orient = make_float3(0.0f, 0.0f, 0.0f);
    if (alpha != 1.0f) {
        const float* o = J.orient_rcv + 3 * i_rcv;
        const float ox = o[0], oy = o[1], oz = o[2];
        const float inv = 1.0f / sqrtf(__fmaf_rn(ox, ox, __fmaf_rn(oy, oy, oz * oz)));
        orient = make_float3(ox * inv, oy * inv, oz * inv);
    }
    // lane constants of tap t = lane, j = t - 15 (see ism_accum.cuh), twice: two images
    // go through the packed FP32 pipe together (f32x2 FMA and multiply)
    const int j = lane - 15;
    const float sg = (j & 1) ? 1.0f : -1.0f;   // (-1)^(j+1)
    const float xj = sg * (float)j, nsg = -sg;
    float Sj, Cj;
    sincospif((float)j * (2.0f / 32.0f), &Sj, &Cj);
    const unsigned long long xj2 = sd_pack(xj, xj), nsg2 = sd_pack(nsg, nsg), Cj2 = sd_pack(Cj, Cj),
                             Sj2 = sd_pack(Sj, Sj);
    const float twopi_Nw = 6.283185307179586f / 32.0f, inv2Nw = 2.0f / 32.0f;
    uint32_t C2 = 0, S2 = 0;
    if constexpr (HALF) {
        C2 = pack2<PREC>(Cj, Cj);
        S2 = pack2<PREC>(Sj, Sj);
    }
    // FP16 records are scaled by 2^e (undone, exactly, on each product); f is kept away
    // from 0 and 1 in the packed forms so that the packed reciprocal stays finite
    const float rscale = (PREC == PREC_FP16) ? J.half_scale : 1.0f;
    const float dscale = (PREC == PREC_FP16) ? 1.0f / J.half_scale : 1.0f;
    const float f_lo = HALF ? 0x1p-13f : 0x1p-60f;
    const float f_hi = HALF ? 1.0f - 0x1p-13f : 1.0f;
    const float* lut = PREC == PREC_LUT ? lut_g + J.lut_base + lane : nullptr;

    const int W0 = ISM_SB * q0 - 16;   // first sample of the shell's window
    const Shell sh = shell_setup(J, T, r, ISM_SB * q0 - 1, min(ISM_SB * (q0 + nb) - 1, J.n_ism + J.H - 1));
    const int n_cols = shell_rows(sh, T, rowpre, rowy0);   // (synchronises the CTA)
    const float amp_scale = J.amp_scale;

    // Staged records: a ring of SD_RING per warp, records 2k and 2k + 1 interleaved as
    // {f_a, f_b, P_a, P_b}, {Pc_a, Pc_b, Ps_a, Ps_b}; the warp's images enter in the order
    // it meets them (batch by batch, lane by lane), and whenever 32 wait their taps are
    // added, two images at a time (lane t adds tap t of each to its column of the window).
    const ulonglong2* st2 = reinterpret_cast<const ulonglong2*>(stage);
    const int2* sp2 = reinterpret_cast<const int2*>(spos);
    int head = 0, n_st = 0;   // (warp-uniform) first pair of the ring not yet added; records waiting
    auto put = [&](int slot, const float4& rc, int pos) {
        float* sl = reinterpret_cast<float*>(stage) + 8 * (slot >> 1) + (slot & 1);
        sl[0] = rc.x;
        sl[2] = rc.y;
        sl[4] = rc.z;
        sl[6] = rc.w;
        spos[slot] = pos;
    };
    auto taps = [&](int n_pairs) {
        for (int i = 0; i < n_pairs; ++i) {
            const int k = (head + i) & (SD_RING / 2 - 1);
            const ulonglong2 fa = st2[2 * k];       // {f_a, f_b}, {P_a, P_b}
            const ulonglong2 fb = st2[2 * k + 1];   // {Pc_a, Pc_b}, {Ps_a, Ps_b}
            const int2 pp = sp2[k];
            float va, vb;
            if constexpr (PREC == PREC_FP32) {
                const unsigned long long x2 = sd_fma2(nsg2, fa.x, xj2);
                const unsigned long long w2 = sd_fma2(Cj2, fb.x, sd_fma2(Sj2, fb.y, fa.y));
                float xa, xb;
                sd_unpack(x2, xa, xb);
                sd_unpack(sd_mul2(w2, sd_pack(ism_rcp(xa), ism_rcp(xb))), va, vb);
            } else if constexpr (HALF) {
                // x in FP32, then the window and the reciprocal in packed 16-bit arithmetic;
                // the products of two 16-bit values are exact in FP32
                float xa, xb, Pa, Pb, Pca, Pcb, Psa, Psb;
                sd_unpack(sd_fma2(nsg2, fa.x, xj2), xa, xb);
                sd_unpack(fa.y, Pa, Pb);
                sd_unpack(fb.x, Pca, Pcb);
                sd_unpack(fb.y, Psa, Psb);
                const uint32_t w = fma2<PREC>(C2, pack2<PREC>(Pca, Pcb), fma2<PREC>(S2, pack2<PREC>(Psa, Psb),
                                                                                   pack2<PREC>(Pa, Pb)));
                va = 0.0f;
                vb = 0.0f;
                mixed_fma2<PREC>(va, vb, w, rcp2<PREC>(pack2<PREC>(xa, xb)));
                va *= dscale;
                vb *= dscale;
            } else if constexpr (PREC == PREC_LUT) {
                float w0a, w0b, w1a, w1b, ra, rb;
                sd_unpack(fa.x, w0a, w0b);
                sd_unpack(fa.y, w1a, w1b);
                sd_unpack(fb.x, ra, rb);
                const float* pa = lut + __float_as_int(ra);
                const float* pb = lut + __float_as_int(rb);
                va = __fmaf_rn(w1a, __ldg(pa + 32), w0a * __ldg(pa));
                vb = __fmaf_rn(w1b, __ldg(pb + 32), w0b * __ldg(pb));
            } else {   // PREC_TEX: one filtered fetch per tap
                float Aa, Ab, ya, yb;
                sd_unpack(fa.x, Aa, Ab);
                sd_unpack(fa.y, ya, yb);
                const cudaTextureObject_t tex = (cudaTextureObject_t)J.lut_tex;
                va = Aa * tex2D<float>(tex, (float)lane + 0.5f, ya);
                vb = Ab * tex2D<float>(tex, (float)lane + 0.5f, yb);
            }
            winl[pp.x] += va;
            winl[pp.y] += vb;
        }
        head = (head + n_pairs) & (SD_RING / 2 - 1);
    };

    shell_walk_cta<SD_WARPS>(
        sh, T, rowpre, rowy0, n_cols, make_float2(orient.x, orient.y), recf, reci, st, wtot, warp, lane,
        [&](bool has, int b, float f, float s, const float4& cf, const float4& tz) {
            float4 rc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (has) {
                const float rs = ism_rcp(s);
                float amp = cf.z * tz.z * amp_scale * rs;
                if (alpha != 1.0f)   // polar pattern: cos(theta) = o . (x_n - x_r) / d
                    amp *= __fmaf_rn(1.0f - alpha, __fmaf_rn(orient.z, tz.w, cf.w) * rs, alpha);
                f = fminf(fmaxf(f, f_lo), f_hi);   // keeps j - f away from 0 (the reciprocal of the tap j = 0)
                if constexpr (PREC == PREC_LUT) {
                    // eq. (9): rows floor(f Q) and + 1 of the polyphase table, weights A (1 - phi), A phi
                    const float u = f * (float)LQ;   // exact: LQ is a power of two
                    const float pf = floorf(u);
                    const float ph = u - pf;         // exact
                    rc = make_float4(amp - amp * ph, amp * ph, __int_as_float(ism_int_of_integral(pf) * 32), 0.0f);
                } else if constexpr (PREC == PREC_TEX) {
                    rc = make_float4(amp, __fmaf_rn(f, (float)LQ, 0.5f), 0.0f, 0.0f);   // texel row f Q, centred
                } else {
                    rc = ism_sinc_record(f, amp, true, twopi_Nw, inv2Nw);
                    rc.y *= rscale;
                    rc.z *= rscale;
                    rc.w *= rscale;
                }
            }
            const unsigned v = __ballot_sync(0xffffffffu, has);
            if (has)   // the images of the batch in lane order, after those waiting
                put((2 * head + n_st + __popc(v & ((1u << lane) - 1u))) & (SD_RING - 1), rc, b - 15 - W0);
            n_st += __popc(v);
            if (n_st >= 32) {
                __syncwarp();
                taps(16);
                n_st -= 32;
                __syncwarp();   // the added records are free before the next batch writes
            }
        });
    // the images still waiting (an odd count padded with a record that adds 0 past the window)
    if (n_st & 1) {
        if (lane == 0) put((2 * head + n_st) & (SD_RING - 1), make_float4(0.5f, 0.0f, 0.0f, 0.0f), win);
        ++n_st;
    }
    __syncwarp();
    taps(n_st >> 1);
    __syncthreads();

    // the bins' rows: the warps' windows summed in warp order
    for (int ql = warp; ql < nb; ql += SD_WARPS) {
        const int q = q0 + ql;
        float* row = rows + J.rows_base + ((long long)r * J.Q + q) * WIN;
        {
            const int p = 32 * ql + lane;   // lower half: samples 32 q - 16 + lane
            float v = win_all[p];
#pragma unroll
            for (int w = 1; w < SD_WARPS; ++w) v += win_all[w * winp + p];
            row[lane] = v;
        }
        {
            float v = 0.0f;
            if (ql == nb - 1) {   // the samples that spill into the next shell
                const int p = 32 * nb + lane;
                v = win_all[p];
#pragma unroll
                for (int w = 1; w < SD_WARPS; ++w) v += win_all[w * winp + p];
            }
            row[32 + lane] = v;
        }
    }
}

// the launch's thickest shell (bins)
int sd_bins_max(const JobTable& t)
{
    int bmax = 0;
    for (int i = 0; i < t.n_jobs; ++i) bmax = std::max(bmax, t.j[i].shell_direct);
    return bmax;
}

size_t shell_direct_smem(const JobTable& t)
{
    return (size_t)((t.max_axis_sum + 1) & ~1) * sizeof(float4) + 2 * (size_t)((t.max_axis_sum + 4) & ~3) * sizeof(int) +
           (size_t)SD_WARPS * 32 * (sizeof(float4) + sizeof(int4)) + ((size_t)SD_WARPS * 33 + 8) * sizeof(int) +
           (size_t)SD_WARPS * SD_RING * (sizeof(float4) + sizeof(int)) + SD_WARPS * sizeof(int) +
           (size_t)SD_WARPS * sd_winp(sd_bins_max(t)) * sizeof(float);
}

}  // namespace

template <int PREC>
static int launch_sd(const JobTable& t, const WsPlan& p, char* ws, cudaStream_t s)
{
    const size_t sm = shell_direct_smem(t);
    static std::atomic<unsigned long long> opened{0};
    int rc = ism_open_smem((const void*)shell_direct_kernel<PREC>, &opened);
    if (rc) return rc;
    cudaError_t e = cudaFuncSetAttribute(shell_direct_kernel<PREC>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return (int)e;
    shell_direct_kernel<PREC><<<(unsigned)p.sd_ctas, SD_WARPS * 32, sm, s>>>(
        t, reinterpret_cast<const float4*>(ws + p.tbl_off), reinterpret_cast<const float*>(ws + p.lut_off),
        reinterpret_cast<float*>(ws + p.rows_off), sd_winp(sd_bins_max(t)));
    return (int)cudaGetLastError();
}

int ism_launch_accum_shell_direct(const JobTable& t, const WsPlan& p, char* ws, ism_precision prec, void* stream,
                                  int* launched)
{
    *launched = 0;
    if (p.sd_ctas <= 0) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    switch (prec) {
    case ISM_PREC_FP32:
    case ISM_PREC_FP32_DIRECT: rc = launch_sd<PREC_FP32>(t, p, ws, s); break;
    case ISM_PREC_FP16X2: rc = launch_sd<PREC_FP16>(t, p, ws, s); break;
    case ISM_PREC_BF16X2: rc = launch_sd<PREC_BF16>(t, p, ws, s); break;
    case ISM_PREC_LUT: rc = launch_sd<PREC_LUT>(t, p, ws, s); break;
    case ISM_PREC_LUT_TEX: rc = launch_sd<PREC_TEX>(t, p, ws, s); break;
    default: return (int)cudaErrorInvalidValue;
    }
    *launched = rc ? 0 : 1;
    return rc;
}
