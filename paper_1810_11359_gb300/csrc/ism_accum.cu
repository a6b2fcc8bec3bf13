// ism_accum.cu -- windowed-sinc accumulation (kernel c), the hot loop of the
// method: eq. (5) with the fractional-delay pulse of eq. (6).
//
// One CTA owns a tile of 256 output samples of one RIR, i.e. 8 delay bins of
// 32 samples, one per warp.  An image of bin q has delay s = b + f (b integer,
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
// After its bins the CTA sums, for each sample, the window rows of the bins
// overlapping it in ascending bin order and stores it once.  The first and
// the last 32 SLOTS samples of the tile region also receive contributions
// from the neighbouring tiles; they go to a seam buffer that the finalize
// kernel combines, again in a fixed order.
#include "ism_device.cuh"

namespace {

#define ISM_PIECE 1024
#define ISM_NB 33                  // delay offsets rr = -1 .. 31 inside a bin
#define ISM_CHUNK 64               // records computed per step (two per lane)
#define ISM_PAD (ISM_PIECE + 4 * ISM_NB)
#define ISM_DUMMY 0x80000000u      // sorted-list entry that carries no image

struct WarpSmem {
    uint32_t sorted[ISM_PAD];      // ids sorted by plain-FP32 offset, buckets padded to 4
    uint16_t key[ISM_PIECE];       // bucket (low 6 bits) | rank in bucket << 6
    uint8_t group_bucket[ISM_PAD / 4];  // bucket of every group of 4 sorted entries
    uint32_t off[ISM_NB + 1];      // padded bucket offsets in `sorted`
    uint32_t cnt[ISM_NB + 1];      // bucket sizes
    float4 rec[ISM_CHUNK];         // f, P, P cos(phi), P sin(phi) of the current chunk
};

// The per-image record of the windowed sinc of eq. (6) for an image of bin q:
// exact delay s = b + f from the float-float squared offsets, rr = b - 32 q,
// P = A sin(pi f) / (2 pi) with A of eq. (4), and P cos(phi), P sin(phi),
// phi = 2 pi f / N_w.  Branch free; an offset outside [-1, 31] (which the
// binning rules out) raises *bad and contributes nothing.
__device__ __forceinline__ float4 ism_record(const float4 tx, const float4 ty, const float4 tz, int q,
                                             float amp_scale, bool small_phase, float twopi_Nw, float inv2Nw,
                                             int* rr_out, bool* bad)
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
    float amp = tx.z * ty.z * tz.z * amp_scale * ism_rcp(sq.hi);
    const bool out = rr < -1 || rr > ISM_SB - 1;
    *bad = out;
    rr = out ? -1 : rr;
    amp = out ? 0.0f : amp;
    f = fmaxf(f, 0x1p-60f);
    const float P = amp * ism_sinpi01(f) * 0.15915494309189535f;  // A sin(pi f) / (2 pi)
    float sp, cp;
    if (small_phase) ism_sincos_small(f * twopi_Nw, &sp, &cp);
    else sincospif(f * inv2Nw, &sp, &cp);
    *rr_out = rr;
    return make_float4(f, P, P * cp, P * sp);
}

// Rotates the run total D (lane = tap) into the window (lane = position).
template <int SLOTS>
__device__ __forceinline__ void flush_run(float (&D)[SLOTS], float (&acc)[SLOTS + 1], int rr, int lane)
{
    const int src = (lane - rr - 1) & 31;
    const bool upper = lane <= rr;
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
        float v = __shfl_sync(0xffffffffu, D[s], src);
        if (upper) acc[s + 1] += v;
        else acc[s] += v;
        D[s] = 0.0f;
    }
}

// Adds the taps of one record (lane = tap) directly into the window at its
// own offset rr: used for the rare image whose exact offset differs from the
// offset of the bucket it was sorted into.
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

template <int SLOTS, bool MASK>
__global__ void __launch_bounds__(ISM_ACC_WARPS * 32) accum_kernel(const __grid_constant__ JobTable t,
                                                                    const float4* __restrict__ tbl,
                                                                    const uint32_t* __restrict__ hist,
                                                                    const uint32_t* __restrict__ ids,
                                                                    float* __restrict__ seams,
                                                                    uint32_t* __restrict__ status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const long long g = blockIdx.x;
    const int jid = ism_find_job(t, g, [](const JobDev& j) { return j.acc_cta_base; });
    const JobDev& J = t.j[jid];
    const bool exact = (J.Nw == (float)(2 * J.H)) && (2 * J.H == 32 * J.slots);
    if (J.slots != SLOTS || exact == MASK) return;  // another instantiation handles this job

    const long long local = g - J.acc_cta_base;
    const int r = (int)(local / J.n_tiles);
    const int tile = J.n_tiles - 1 - (int)(local % J.n_tiles);  // densest (latest) tiles first
    const int Nx = J.N[0], Ny = J.N[1], Nz = J.N[2];
    const int n_axis = Nx + Ny + Nz;
    const int H = J.H;
    constexpr int WIN = 32 * (SLOTS + 1);  // window registers x 32 lanes

    float4* T = reinterpret_cast<float4*>(smem);
    WarpSmem* Wall = reinterpret_cast<WarpSmem*>(smem + (size_t)((t.max_axis_sum + 1) & ~1) * sizeof(float4));
    float* rows = reinterpret_cast<float*>(Wall + ISM_ACC_WARPS);  // [bin][WIN]

    const float4* Tg = tbl + J.tbl_base + (long long)r * n_axis;
    for (int e = threadIdx.x; e < n_axis; e += blockDim.x) T[e] = Tg[e];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem& W = Wall[warp];

    // lane constants of the taps t = lane + 32 s, j = t - H + 1
    float xj[SLOTS], nsg[SLOTS], Cj[SLOTS], Sj[SLOTS], D[SLOTS], D2[SLOTS], acc[SLOTS + 1];
    bool tap_ok[SLOTS];
    const float inv2Nw = 2.0f / J.Nw;
    const float twopi_Nw = 6.283185307179586f / J.Nw;
    const bool small_phase = J.Nw >= 16.0f;   // 2 pi f / N_w <= pi / 8
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
        const int tt = lane + 32 * s;
        const int j = tt - H + 1;
        const float sg = (j & 1) ? 1.0f : -1.0f;  // (-1)^(j+1)
        xj[s] = sg * (float)j;
        nsg[s] = -sg;
        sincospif((float)j * inv2Nw, &Sj[s], &Cj[s]);
        tap_ok[s] = tt < 2 * H;
    }
    const float halfNw = 0.5f * J.Nw;
    const unsigned lt_mask = (1u << lane) - 1u;
    const float* Sh = reinterpret_cast<const float*>(T);  // .x of the float4 entries: stride 4
    __syncthreads();
    (void)lt_mask;

    {
        const int b_in_tile = warp;
        const int q = tile * ISM_TILE_BINS + b_in_tile;
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
            for (uint32_t p0 = start; p0 < end; p0 += ISM_PIECE) {
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
                            const float s2 =
                                __fadd_rn(__fadd_rn(Sh[4 * ix], Sh[4 * (Nx + iy)]), Sh[4 * (Nx + Ny + iz)]);
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
                        float4 rc = make_float4(0.5f, 0.0f, 0.0f, 0.0f);
                        int rr = 0;
                        bool stray = false;
                        if (i < c0 + m) {
                            const uint32_t pid = W.sorted[i];
                            const int rr_bucket = (int)W.group_bucket[i >> 2] - 1;
                            rr = rr_bucket;
                            if (!(pid & ISM_DUMMY)) {
                                const int ix = pid & 1023, iy = (pid >> 10) & 1023, iz = pid >> 20;
                                bool bad;
                                rc = ism_record(T[ix], T[Nx + iy], T[Nx + Ny + iz], q, J.amp_scale, small_phase,
                                                twopi_Nw, inv2Nw, &rr, &bad);
                                if (bad) atomicOr(status, (uint32_t)ISM_DEVICE_FLAG_BIN);
                                stray = rr != rr_bucket;
                            }
                        }
                        W.rec[32 * h + lane] = stray ? make_float4(rc.x, 0.0f, 0.0f, 0.0f) : rc;
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
                                flush_run<SLOTS>(D, acc, cur_rr, lane);
                            }
                            cur_rr = __shfl_sync(0xffffffffu, rr_grp, g);
                        }
                        const float4 r0 = W.rec[4 * g], r1 = W.rec[4 * g + 1], r2 = W.rec[4 * g + 2],
                                     r3 = W.rec[4 * g + 3];
                        // two interleaved accumulators shorten the dependent FFMA chain
                        taps<SLOTS, MASK>(r0, xj, nsg, Cj, Sj, tap_ok, halfNw, D);
                        taps<SLOTS, MASK>(r1, xj, nsg, Cj, Sj, tap_ok, halfNw, D2);
                        taps<SLOTS, MASK>(r2, xj, nsg, Cj, Sj, tap_ok, halfNw, D);
                        taps<SLOTS, MASK>(r3, xj, nsg, Cj, Sj, tap_ok, halfNw, D2);
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
                flush_run<SLOTS>(D, acc, cur_rr, lane);
            }
        }
#pragma unroll
        for (int m = 0; m <= SLOTS; ++m) rows[b_in_tile * WIN + 32 * m + lane] = acc[m];
    }
    __syncthreads();

    // sample d of the tile region [256 tile - H, 256 tile - H + 256 + 32 SLOTS):
    // sum of the bins whose window covers it, in ascending bin order
    float* out = J.out + (long long)r * J.n_S;
    float* seam = seams + J.seam_base + ((long long)r * J.n_tiles + tile) * (64LL * SLOTS);
    const int base0 = ISM_TILE_SAMPLES * tile - H;
    for (int d = threadIdx.x; d < ISM_TILE_SAMPLES + 32 * SLOTS; d += blockDim.x) {
        // bins b with 0 <= d - 32 b < WIN
        const int b_lo = d >= WIN ? (d - WIN) / ISM_SB + 1 : 0;
        int b_hi = d / ISM_SB;
        if (b_hi > ISM_TILE_BINS - 1) b_hi = ISM_TILE_BINS - 1;
        float v = 0.0f;
        for (int b = b_lo; b <= b_hi; ++b) v += rows[b * WIN + (d - ISM_SB * b)];
        if (d < 32 * SLOTS) {
            seam[d] = v;
        } else if (d >= ISM_TILE_SAMPLES) {
            seam[32 * SLOTS + (d - ISM_TILE_SAMPLES)] = v;
        } else {
            const int k = base0 + d;
            if (k >= 0 && k < J.n_ism) out[k] = v;
        }
    }
}

template <int SLOTS, bool MASK>
int launch_one(const JobTable& t, const WsPlan& p, char* ws, cudaStream_t s)
{
    size_t sm = (size_t)((t.max_axis_sum + 1) & ~1) * sizeof(float4) + ISM_ACC_WARPS * sizeof(WarpSmem) +
                (size_t)ISM_TILE_BINS * 32 * (SLOTS + 1) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(accum_kernel<SLOTS, MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return (int)e;
    accum_kernel<SLOTS, MASK><<<(unsigned)p.acc_ctas, ISM_ACC_WARPS * 32, sm, s>>>(
        t, reinterpret_cast<const float4*>(ws + p.tbl_off), reinterpret_cast<const uint32_t*>(ws + p.hist_off),
        reinterpret_cast<const uint32_t*>(ws + p.ids_off), reinterpret_cast<float*>(ws + p.seam_off),
        reinterpret_cast<uint32_t*>(ws + p.status_off));
    return (int)cudaGetLastError();
}

}  // namespace

int ism_launch_accum(const JobTable& t, const WsPlan& p, char* ws, ism_precision prec, void* stream,
                     int* launched)
{
    (void)prec;
    *launched = 0;
    if (p.acc_ctas <= 0) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    bool need[2][ISM_MAX_SLOTS + 1] = {};
    for (int i = 0; i < t.n_jobs; ++i) {
        const JobDev& J = t.j[i];
        bool exact = (J.Nw == (float)(2 * J.H)) && (2 * J.H == 32 * J.slots);
        need[exact ? 0 : 1][J.slots] = true;
    }
    int rc = 0;
#define ISM_L(SL)                                                                     \
    if (!rc && need[0][SL]) rc = launch_one<SL, false>(t, p, ws, s), ++*launched;    \
    if (!rc && need[1][SL]) rc = launch_one<SL, true>(t, p, ws, s), ++*launched;
    ISM_L(1) ISM_L(2) ISM_L(3) ISM_L(4) ISM_L(5) ISM_L(6) ISM_L(7) ISM_L(8)
#undef ISM_L
    return rc;
}
