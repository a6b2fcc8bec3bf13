// ism_accum_cheb.cu -- FP32 accumulation of eq. (5) for a 32-tap window
// through a Chebyshev expansion of the windowed sinc in the fractional delay.
//
// For tap j of an image with delay s = b + f (b integer, f in [0, 1)), the
// sample b + j receives A delta'(j - f) (eq. (6)).  For a window of exactly
// N_w = 32 taps every tap function g_j(f) = delta'(j - f), j = -15 .. 16, is
// an entire function of f on [0, 1] (the window's zeros fall at the ends of
// the interval, so no mask cuts it), and its Chebyshev series in u = 2f - 1
// converges fast: degree 9 reproduces each g_j to 2e-9 (the coefficients
// c_{j,i}, interpolated at the 10 Chebyshev-Gauss nodes in FP64 on the host,
// travel in the kernel's parameter table).  Hence for the images of one delay bin that share
// the integer offset rr = b - 32 q,
//   sum_n A_n g_j(f_n) = sum_i c_{j,i} M_i,   M_i = sum_n A_n T_i(2 f_n - 1),
// so each image costs 10 moment updates on one lane instead of 32 tap
// evaluations, and each offset costs 10 FMAs per tap once per bin.
//
// One warp per bin, as in the direct kernel: the bin's ids are counting-
// sorted by their plain-FP32 offset (33 buckets) in shared memory, 512 at a
// time.  Then every lane takes every 32nd sorted entry and computes its
// exact float-float delay and amplitude (eq. (2)-(4)), storing u = 2f - 1
// and A; an entry whose exact offset differs from its bucket's (the
// plain-FP32 key is off by one within ~1e-3 sample of an integer) is added
// right away by direct evaluation of its 32 taps, in sorted order, and gets
// A = 0 for the moments.  Then lane l accumulates the moments of bucket l
// (rr = l - 1), lane 0 also those of the last, half-width bucket (rr = 31),
// in sorted order.  Finally each non-empty offset's moments are expanded
// into the taps (lane = tap) and rotated into the bin's register window,
// which is stored as the bin's row; the finalize kernel sums the rows per
// sample.  No atomics touch floating-point data; every sum has a fixed
// order.
#include "ism_accum.cuh"

namespace {

#define CB_PIECE 512
#define CB_MPAD 12      // moments of one offset, padded to three float4

struct ChebWarp {
    union {
        struct {
            uint32_t sorted[CB_PIECE];    // ids sorted by offset; then u = 2f - 1 of each entry (float bits)
            union {
                uint16_t key[CB_PIECE];   // bucket (low 6 bits) | rank in bucket << 6 (until placement)
                float amp[CB_PIECE];      // amplitude of each sorted entry (0: added directly instead)
            };
        };
        float M[ISM_NB * CB_MPAD];        // after the last piece: moments per offset
    };
    uint8_t bkt[CB_PIECE];                // bucket of each sorted entry
    uint32_t off[ISM_NB + 1];
    uint32_t cnt[ISM_NB + 1];
    float M32[CB_MPAD];                   // running moments of bucket 32 (lane 0) across pieces
};

// Moments of one bucket (entries [o, o + n) of the sorted list):
// Mx[i] += A T_i(u), T_(k) = 2u T_(k-1) - T_(k-2); two entries per step.
__device__ __forceinline__ void cheb_walk(const float* __restrict__ U, const float* __restrict__ Aw, uint32_t o,
                                          uint32_t n, float (&Mx)[ISM_CHEB_N])
{
    uint32_t i = 0;
    for (; i + 1 < n; i += 2) {
        const float ua = U[o + i], aa = Aw[o + i], ub = U[o + i + 1], ab = Aw[o + i + 1];
        const float ua2 = ua + ua, ub2 = ub + ub;
        Mx[0] += aa + ab;
        Mx[1] = __fmaf_rn(ab, ub, __fmaf_rn(aa, ua, Mx[1]));
        float pa = 1.0f, qa = ua, pb = 1.0f, qb = ub;
#pragma unroll
        for (int k = 2; k < ISM_CHEB_N; ++k) {
            const float ta = __fmaf_rn(ua2, qa, -pa), tb = __fmaf_rn(ub2, qb, -pb);
            Mx[k] = __fmaf_rn(ab, tb, __fmaf_rn(aa, ta, Mx[k]));
            pa = qa;
            qa = ta;
            pb = qb;
            qb = tb;
        }
    }
    if (i < n) {
        const float ua = U[o + i], aa = Aw[o + i];
        const float ua2 = ua + ua;
        Mx[0] += aa;
        Mx[1] = __fmaf_rn(aa, ua, Mx[1]);
        float pa = 1.0f, qa = ua;
#pragma unroll
        for (int k = 2; k < ISM_CHEB_N; ++k) {
            const float ta = __fmaf_rn(ua2, qa, -pa);
            Mx[k] = __fmaf_rn(aa, ta, Mx[k]);
            pa = qa;
            qa = ta;
        }
    }
}

__global__ void __launch_bounds__(ISM_ACC_BPC * 32) cheb_kernel(const __grid_constant__ JobTable t,
                                                                 const float4* __restrict__ tbl,
                                                                 const uint32_t* __restrict__ hist,
                                                                 const uint32_t* __restrict__ ids,
                                                                 float* __restrict__ rows,
                                                                 uint32_t* __restrict__ status)
{
    constexpr int WIN = 64;   // 32 (SLOTS + 1), SLOTS = 1
    extern __shared__ __align__(16) unsigned char smem[];
    const long long g = blockIdx.x;
    const int jid = ism_find_job(t, g, [](const JobDev& j) { return j.acc_cta_base; });
    const JobDev& J = t.j[jid];
    if (!J.use_cheb) return;   // the direct kernel handles this job

    const long long local = g - J.acc_cta_base;
    const int r = (int)(local / J.acc_groups);
    const int grp = J.acc_groups - 1 - (int)(local % J.acc_groups);  // densest (latest) bins first
    const int Nx = J.N[0], Ny = J.N[1], Nz = J.N[2];
    const int n_axis = Nx + Ny + Nz;

    float4* T = reinterpret_cast<float4*>(smem);
    ChebWarp* Wall = reinterpret_cast<ChebWarp*>(smem + (size_t)((t.max_axis_sum + 1) & ~1) * sizeof(float4));
    float* Sh = reinterpret_cast<float*>(Wall + ISM_ACC_BPC);   // plain S_hi per axis index (conflict-light keys)
    const float4* Tg = tbl + J.tbl_base + (long long)r * n_axis;
    for (int e = threadIdx.x; e < n_axis; e += blockDim.x) {
        const float4 v = Tg[e];
        T[e] = v;
        Sh[e] = v.x;
    }

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    ChebWarp& W = Wall[warp];
    const int q = grp * ISM_ACC_BPC + warp;

    // lane = tap t, j = t - 15: Chebyshev coefficients, and the constants of
    // the direct evaluation used for flagged images
    float c[ISM_CHEB_N];
#pragma unroll
    for (int i = 0; i < ISM_CHEB_N; ++i) c[i] = t.cheb[lane * ISM_CHEB_N + i];
    float xj[1], nsg[1], Cj[1], Sj[1];
    bool tap_ok[1] = {true};
    {
        const int j = lane - 15;
        const float sg = (j & 1) ? 1.0f : -1.0f;
        xj[0] = sg * (float)j;
        nsg[0] = -sg;
        sincospif((float)j * 0.0625f, &Sj[0], &Cj[0]);   // 2 j / N_w, N_w = 32
    }
    const float twopi_Nw = 6.283185307179586f / 32.0f;
    const unsigned lt_mask = (1u << lane) - 1u;
    float* U = reinterpret_cast<float*>(W.sorted);
    __syncthreads();
    if (q >= J.Q) return;

    float acc[2] = {0.0f, 0.0f};
    float M[ISM_CHEB_N];
#pragma unroll
    for (int i = 0; i < ISM_CHEB_N; ++i) M[i] = 0.0f;
    if (lane < CB_MPAD) W.M32[lane] = 0.0f;
    unsigned nonempty = 0u;     // bit b: bucket b (< 32) has had images
    bool last_nonempty = false; // bucket 32

    const long long hb = J.hist_base + ((long long)r * J.Q + q) * J.U;
    const uint32_t start = hist[hb];
    const uint32_t end = hist[hb + J.U];
    for (uint32_t p0 = start; p0 < end; p0 += CB_PIECE) {
        const int n = (int)min((uint32_t)CB_PIECE, end - p0);
        const uint32_t* src = ids + p0;

        // ---- stable counting sort of the piece by plain-FP32 offset
        W.cnt[lane] = 0;
        if (lane < 2) W.cnt[32 + lane] = 0;
        __syncwarp();
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
        {   // exclusive prefix over the 33 bucket sizes
            const uint32_t v = W.cnt[lane];
            uint32_t inc = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t nn = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += nn;
            }
            W.off[lane] = inc - v;
            if (lane == 31) W.off[32] = inc;
            nonempty |= __ballot_sync(0xffffffffu, v > 0);
        }
        __syncwarp();
        last_nonempty |= W.cnt[32] > 0;
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
                    const uint32_t dst = W.off[k & 63u] + (k >> 6);
                    W.sorted[dst] = pid[u];
                    W.bkt[dst] = (uint8_t)(k & 63u);
                }
            }
        }
        __syncwarp();

        // ---- exact delay and amplitude of every entry, one per lane (balanced);
        // entries whose exact offset differs from their bucket's are added by
        // direct evaluation of their 32 taps, in sorted order
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            float f = 0.5f, amp = 0.0f;
            int rr = 0;
            bool stray = false;
            if (i < n) {
                const uint32_t pid = W.sorted[i];
                const int bucket = W.bkt[i];
                const int ix = pid & 1023, iy = (pid >> 10) & 1023, iz = pid >> 20;
                bool bad;
                ism_delay(T[ix], T[Nx + iy], T[Nx + Ny + iz], q, J.amp_scale, &f, &amp, &rr, &bad);
                if (bad) atomicOr(status, (uint32_t)ISM_DEVICE_FLAG_BIN);
                stray = !bad && rr != bucket - 1;
                U[i] = __fmaf_rn(2.0f, f, -1.0f);
                W.amp[i] = (stray || bad) ? 0.0f : amp;
            }
            unsigned sm = __ballot_sync(0xffffffffu, stray);
            while (sm) {
                const int l = __ffs(sm) - 1;
                sm &= sm - 1;
                const float fs_ = fmaxf(__shfl_sync(0xffffffffu, f, l), 0x1p-60f);
                const float as_ = __shfl_sync(0xffffffffu, amp, l);
                const int rs_ = __shfl_sync(0xffffffffu, rr, l);
                const float4 rc = ism_sinc_record(fs_, as_, true, twopi_Nw, 0.0625f);
                add_single<1, false>(rc, rs_, xj, nsg, Cj, Sj, tap_ok, 16.0f, acc, lane);
            }
        }
        __syncwarp();

        // ---- moments: lane l walks bucket l (rr = l - 1), lane 0 also bucket 32 (rr = 31)
        cheb_walk(U, W.amp, W.off[lane], W.cnt[lane], M);
        if (lane == 0) {
            float M2[ISM_CHEB_N];
#pragma unroll
            for (int i = 0; i < ISM_CHEB_N; ++i) M2[i] = W.M32[i];
            cheb_walk(U, W.amp, W.off[32], W.cnt[32], M2);
#pragma unroll
            for (int i = 0; i < ISM_CHEB_N; ++i) W.M32[i] = M2[i];
        }
        __syncwarp();
    }

    // ---- expansion of each non-empty offset into the taps, rotated into the window
    __syncwarp();
#pragma unroll
    for (int i = 0; i < ISM_CHEB_N; ++i) W.M[lane * CB_MPAD + i] = M[i];
    if (lane < CB_MPAD) W.M[32 * CB_MPAD + lane] = W.M32[lane];
    __syncwarp();
    const float4* M4 = reinterpret_cast<const float4*>(W.M);
    for (int b = 0; b <= ISM_SB; ++b) {
        if (b < 32 ? !((nonempty >> b) & 1u) : !last_nonempty) continue;   // warp-uniform
        const float4 m0 = M4[3 * b], m1 = M4[3 * b + 1], m2 = M4[3 * b + 2];
        float D[1];
        D[0] = c[0] * m0.x;
        D[0] = __fmaf_rn(c[1], m0.y, D[0]);
        D[0] = __fmaf_rn(c[2], m0.z, D[0]);
        D[0] = __fmaf_rn(c[3], m0.w, D[0]);
        D[0] = __fmaf_rn(c[4], m1.x, D[0]);
        D[0] = __fmaf_rn(c[5], m1.y, D[0]);
        D[0] = __fmaf_rn(c[6], m1.z, D[0]);
        D[0] = __fmaf_rn(c[7], m1.w, D[0]);
        D[0] = __fmaf_rn(c[8], m2.x, D[0]);
        D[0] = __fmaf_rn(c[9], m2.y, D[0]);
        flush_run<1, false>(D, acc, b - 1, lane, 1.0f);
    }
    float* row = rows + J.rows_base + ((long long)r * J.Q + q) * WIN;
    row[lane] = acc[0];
    row[32 + lane] = acc[1];
}

}  // namespace

int ism_launch_accum_cheb(const JobTable& t, const WsPlan& p, char* ws, void* stream, int* launched)
{
    *launched = 0;
    if (p.acc_ctas <= 0 || !t.any_cheb) return 0;
    const size_t sm = (size_t)((t.max_axis_sum + 1) & ~1) * sizeof(float4) + ISM_ACC_BPC * sizeof(ChebWarp) +
                      (size_t)t.max_axis_sum * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(cheb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return (int)e;
    cheb_kernel<<<(unsigned)p.acc_ctas, ISM_ACC_BPC * 32, sm, (cudaStream_t)stream>>>(
        t, reinterpret_cast<const float4*>(ws + p.tbl_off), reinterpret_cast<const uint32_t*>(ws + p.hist_off),
        reinterpret_cast<const uint32_t*>(ws + p.ids_off), reinterpret_cast<float*>(ws + p.rows_off),
        reinterpret_cast<uint32_t*>(ws + p.status_off));
    *launched = 1;
    return (int)cudaGetLastError();
}
