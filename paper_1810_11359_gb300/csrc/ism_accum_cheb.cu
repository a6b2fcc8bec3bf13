// ism_accum_cheb.cu -- FP32 accumulation of eq. (5) for a 32-tap window
// through a Chebyshev expansion of the windowed sinc in the fractional delay.
//
// For tap j of an image with delay s = b + f (b integer, f in [0, 1)), the
// sample b + j receives A delta'(j - f) (eq. (6)).  For a window of exactly
// N_w = 32 taps every tap function g_j(f) = delta'(j - f), j = -15 .. 16, is
// an entire function of f on [0, 1] (the window's zeros fall at the ends of
// the interval, so no mask cuts it), and its Chebyshev series in u = 2f - 1
// converges fast: degree 8 reproduces each g_j to 6.4e-8 of the image's
// amplitude (degree 9: 2.1e-9; degree 7: 4.2e-7), below the fixed-point step
// of the moment terms (2^-23 of the bin's largest amplitude, see below).  The
// coefficients c_{j,i}, interpolated at the 9 Chebyshev-Gauss nodes in FP64
// on the host, travel in the kernel's parameter table.  Hence for the images
// of one delay bin that share the integer offset rr = b - 32 q,
//   sum_n A_n g_j(f_n) = sum_i c_{j,i} M_i,   M_i = sum_n A_n T_i(2 f_n - 1),
// so each image costs 9 moment terms instead of 32 tap evaluations, and each
// offset costs 9 FMAs per tap once per bin.
//
// One warp per bin.  Each lane takes every 32nd id of the bin, computes the
// image's exact float-float delay and amplitude (eq. (2)-(4)) -- so its offset
// rr in [-1, 31] is exact and no image needs special handling -- and adds its
// 9 moment terms, as integers, into the bin's moment table in shared memory
// with integer atomics.  Integer addition is associative, so the sums, and
// everything computed from them, are the same in every run whatever the order
// in which lanes and warps reach the table; no sort of the images by offset is
// needed.
//
// Fixed point.  Every image of bin q has s >= max(s_direct, 32 q - 1/2) (the
// direct path is the shortest: along each axis the source's own coordinate is
// the image coordinate nearest the receiver), so |A T_i| <= A_max = amp_scale
// / max(s_direct, 32 q - 1).  A term is A T_i scaled by 2^e, e the largest
// integer with 2^e A_max <= (1 - 2^-10) 2^22, and rounded to an integer
// (one FFMA against 1.5 2^23: the sum's bits hold the integer); |term| <
// 2^22, so the rounding error is at most 2^-23 A_max per term, the resolution
// of FP32 on the bin's largest term.  Each term is one 32-bit shared-memory
// atomic add (64-bit atomics holding two moments each measured 2.3x slower);
// after every 256 ids each lane moves the sums of its offset into FP32
// moments (x 2^-e, exact) and clears them, so no sum can exceed
// 256 x 2^22 = 2^30 in magnitude.
//
// Finally each non-empty offset's moments are expanded into the taps (lane =
// tap) and rotated into the bin's register window, which is stored as the
// bin's row; the finalize kernel sums the rows per sample.
#include "ism_accum.cuh"

namespace {

#define CB_PIECE 256    // ids between two moves of the integer sums into FP32
#define CB_MPAD 12      // moments of one offset, padded to three float4
#define CB_MAGIC 12582912.0f                       // 1.5 * 2^23
#define CB_MAGIC_BITS 0x4B400000u                  // its bits
#define CB_TERM_MAX (4194304.0f * (1.0f - 1.0f / 1024.0f))

struct __align__(16) ChebWarp {
    union {
        int P[ISM_CHEB_N * ISM_NB];         // integer sums of the moments: [moment][rr + 1]
        float M[ISM_NB * CB_MPAD];          // after the last move: FP32 moments per offset
    };
    float M32[CB_MPAD];                     // FP32 moments of offset 31 (lane 0) across pieces
};

// Moves the integer sums of one offset (index o = rr + 1) into FP32 moments
// and clears them; returns whether any sum was non-zero.
__device__ __forceinline__ bool cheb_move(int* P, int o, float inv_scale, float (&Mx)[ISM_CHEB_N])
{
    bool any = false;
#pragma unroll
    for (int k = 0; k < ISM_CHEB_N; ++k) {
        const int v = P[k * ISM_NB + o];
        P[k * ISM_NB + o] = 0;
        any |= v != 0;
        Mx[k] = __fmaf_rn(__int2float_rn(v), inv_scale, Mx[k]);
    }
    return any;
}

__global__ void __launch_bounds__(ISM_ACC_BPC * 32, 10) cheb_kernel(const __grid_constant__ JobTable t,
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
    const float4* Tg = tbl + J.tbl_base + (long long)r * n_axis;
    for (int e = threadIdx.x; e < n_axis; e += blockDim.x) T[e] = Tg[e];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    ChebWarp& W = Wall[warp];
    const int q = grp * ISM_ACC_BPC + warp;
    for (int e = lane; e < ISM_CHEB_N * ISM_NB; e += 32) W.P[e] = 0;
    if (lane < CB_MPAD) W.M32[lane] = 0.0f;
    __syncthreads();
    if (q >= J.Q) return;

    // fixed-point scale 2^e of the bin (see the header)
    float scale, inv_scale;
    {
        const float sd = sqrtf(T[-J.nlo[0]].x + T[Nx - J.nlo[1]].x + T[Nx + Ny - J.nlo[2]].x);
        const float s_lo = fmaxf(fmaxf(sd * (1.0f - 1.0f / 1024.0f), (float)(ISM_SB * q) - 1.0f), 1e-30f);
        const float ratio = CB_TERM_MAX / (J.amp_scale / s_lo);
        int e = ((__float_as_int(ratio) >> 23) & 0xFF) - 127;   // floor(log2(ratio)), ratio normal
        e = max(-126, min(126, e));
        scale = __int_as_float((e + 127) << 23);
        inv_scale = __int_as_float((127 - e) << 23);
    }

    float M[ISM_CHEB_N];
#pragma unroll
    for (int i = 0; i < ISM_CHEB_N; ++i) M[i] = 0.0f;
    unsigned nonempty = 0u;     // bit o: offset index o (< 32) has had images
    bool last_nonempty = false; // offset index 32 (rr = 31)

    const long long hb = J.hist_base + ((long long)r * J.Q + q) * J.U;
    const uint32_t start = hist[hb];
    const uint32_t end = hist[hb + J.U];
    for (uint32_t p0 = start; p0 < end; p0 += CB_PIECE) {
        const int n = (int)min((uint32_t)CB_PIECE, end - p0);
        uint32_t pid[CB_PIECE / 32];
#pragma unroll
        for (int u = 0; u < CB_PIECE / 32; ++u) {
            const int i = 32 * u + lane;
            pid[u] = (i < n) ? ids[p0 + i] : 0u;
        }
#pragma unroll
        for (int u = 0; u < CB_PIECE / 32; ++u) {
            const int i = 32 * u + lane;
            if (32 * u >= n) break;                  // warp-uniform
            if (i >= n) continue;
            const int ix = pid[u] & 1023, iy = (pid[u] >> 10) & 1023, iz = pid[u] >> 20;
            float f, amp;
            int rr;
            bool bad;
            ism_delay(T[ix], T[Nx + iy], T[Nx + Ny + iz], q, J.amp_scale, &f, &amp, &rr, &bad);
            if (bad) {
                atomicOr(status, (uint32_t)ISM_DEVICE_FLAG_BIN);
                continue;
            }
            // moment terms round(2^e A T_i(u)), T_i by the three-term recurrence
            const float as = amp * scale;
            const float uu = __fmaf_rn(2.0f, f, -1.0f);
            const float u2 = uu + uu;
            uint32_t b[ISM_CHEB_N];
            b[0] = __float_as_uint(__fadd_rn(as, CB_MAGIC));
            b[1] = __float_as_uint(__fmaf_rn(as, uu, CB_MAGIC));
            float tp = 1.0f, tc = uu;
#pragma unroll
            for (int k = 2; k < ISM_CHEB_N; ++k) {
                const float tn = __fmaf_rn(u2, tc, -tp);
                b[k] = __float_as_uint(__fmaf_rn(as, tn, CB_MAGIC));
                tp = tc;
                tc = tn;
            }
            int* Pb = W.P + (rr + 1);
#pragma unroll
            for (int k = 0; k < ISM_CHEB_N; ++k) atomicAdd(Pb + k * ISM_NB, (int)(b[k] - CB_MAGIC_BITS));
        }
        __syncwarp();
        // lane l owns offset index l (rr = l - 1); lane 0 also index 32 (rr = 31)
        nonempty |= __ballot_sync(0xffffffffu, cheb_move(W.P, lane, inv_scale, M));
        if (lane == 0) {
            float M2[ISM_CHEB_N];
#pragma unroll
            for (int i = 0; i < ISM_CHEB_N; ++i) M2[i] = W.M32[i];
            last_nonempty |= cheb_move(W.P, 32, inv_scale, M2);
#pragma unroll
            for (int i = 0; i < ISM_CHEB_N; ++i) W.M32[i] = M2[i];
        }
        __syncwarp();
    }
    last_nonempty = __shfl_sync(0xffffffffu, last_nonempty, 0);

    // ---- expansion of each non-empty offset into the taps, rotated into the window
#pragma unroll
    for (int i = 0; i < ISM_CHEB_N; ++i) W.M[lane * CB_MPAD + i] = M[i];
    if (lane < CB_MPAD) W.M[32 * CB_MPAD + lane] = W.M32[lane];
    __syncwarp();
    float acc[2] = {0.0f, 0.0f};
    const float4* M4 = reinterpret_cast<const float4*>(W.M);
    // lane = tap t: Chebyshev coefficients of g_(t - 15), live only here
    float c[ISM_CHEB_N];
#pragma unroll
    for (int i = 0; i < ISM_CHEB_N; ++i) c[i] = t.cheb[lane * ISM_CHEB_N + i];
    for (int o = 0; o <= ISM_SB; ++o) {
        if (o < 32 ? !((nonempty >> o) & 1u) : !last_nonempty) continue;   // warp-uniform
        const float4 m0 = M4[3 * o], m1 = M4[3 * o + 1], m2 = M4[3 * o + 2];
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
        flush_run<1, false>(D, acc, o - 1, lane, 1.0f);
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
    const size_t sm = (size_t)((t.max_axis_sum + 1) & ~1) * sizeof(float4) + ISM_ACC_BPC * sizeof(ChebWarp);
    cudaError_t e = cudaFuncSetAttribute(cheb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return (int)e;
    cheb_kernel<<<(unsigned)p.acc_ctas, ISM_ACC_BPC * 32, sm, (cudaStream_t)stream>>>(
        t, reinterpret_cast<const float4*>(ws + p.tbl_off), reinterpret_cast<const uint32_t*>(ws + p.hist_off),
        reinterpret_cast<const uint32_t*>(ws + p.ids_off), reinterpret_cast<float*>(ws + p.rows_off),
        reinterpret_cast<uint32_t*>(ws + p.status_off));
    *launched = 1;
    return (int)cudaGetLastError();
}
