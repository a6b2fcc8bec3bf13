// ism_accum.cu -- windowed-sinc accumulation (kernel c), the hot loop of the
// method: eq. (5) with the fractional-delay pulse of eq. (6).
//
// One CTA owns one tile of ISM_TILE_SB = 8 consecutive delay bins (8 x 32
// samples) of one RIR; warp w owns bin q.  An image of bin q has its delay
// s = b + f (b integer, f in [0,1)) with b = 32 q + rr, rr in [-1, 31].  Its
// taps are the samples k with |k - s| < N_w/2, i.e. k - b = j in [-H+1, H]
// (H = N_w/2).  The warp keeps a register window of 32 (SLOTS + 1) samples
// starting at 32 q - H: lane l, register m holds sample 32 q - H + l + 32 m.
// Every tap of an image lands in that window, each lane taking SLOTS taps
// (2H = 32 SLOTS), so the warp adds one image per step without any shared
// memory traffic and without atomics.
//
// Per tap the arithmetic is reduced to one reciprocal and four FMA-pipe
// operations by hoisting everything that depends on the image alone:
//   sin(pi (j - f)) = (-1)^(j+1) sin(pi f)                  (one sin per image)
//   cos(2 pi (p - H - s') / N_w) = C_p cos(th) + S_p sin(th)
//       with th = 2 pi (rr + f) / N_w per image and C_p, S_p per lane
//   contribution = sign_p [Q + C_p Qc + S_p Qs] / x,   x = (p - H - rr) - f
// where Q = (-1)^rr A sin(pi f) / (2 pi), Qc = Q cos th, Qs = Q sin th and
// sign_p = (-1)^(p + H + 1) is applied once when the window is stored.
//
// The delay s comes from float-float arithmetic on per-axis tables of
// squared offsets (Section 2.1 factorisation), so f keeps FP32 resolution for
// delays of tens of thousands of samples.
//
// After the bins are done the CTA sums, for each 32-sample output segment,
// the window rows of the bins that overlap it in a fixed order and stores it
// once.  Segments that straddle the tile edge go to a seam buffer that the
// finalize kernel combines, again in a fixed order.
#include "ism_device.cuh"

namespace {

struct RecSmem {
    float4 rec[ISM_TILE_SB][32];   // f, Q, Qc, Qs
    float rr[ISM_TILE_SB][32];     // bin offset as float (exact small integer)
};

template <int SLOTS, bool MASK>
__global__ void __launch_bounds__(ISM_TILE_SB * 32) accum_kernel(const __grid_constant__ JobTable t,
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

    float4* T = reinterpret_cast<float4*>(smem);
    RecSmem* R = reinterpret_cast<RecSmem*>(smem + (size_t)((t.max_axis_sum + 1) & ~1) * sizeof(float4));
    float* rows = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(R) + sizeof(RecSmem));
    // rows[w][m][lane], m in [0, SLOTS]

    const float4* Tg = tbl + J.tbl_base + (long long)r * n_axis;
    for (int e = threadIdx.x; e < n_axis; e += blockDim.x) T[e] = Tg[e];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = tile * ISM_TILE_SB + warp;

    // lane constants for window registers m = 0..SLOTS
    float xo[SLOTS + 1], Cm[SLOTS + 1], Sm[SLOTS + 1], acc[SLOTS + 1];
    const float inv2Nw = 2.0f / J.Nw;
#pragma unroll
    for (int m = 0; m <= SLOTS; ++m) {
        int p = lane + 32 * m - H;
        xo[m] = (float)p;
        sincospif((float)p * inv2Nw, &Sm[m], &Cm[m]);
        acc[m] = 0.0f;
    }
    __syncthreads();

    if (q < J.Q) {
        const long long hb = J.hist_base + ((long long)r * J.Q + q) * J.U;
        const uint32_t start = hist[hb];
        const uint32_t end = hist[hb + J.U];
        const float* Ty = reinterpret_cast<const float*>(T + Nx);
        (void)Ty;
        const float halfNw = 0.5f * J.Nw;
        for (uint32_t cb = start; cb < end; cb += 32) {
            uint32_t idx = cb + lane;
            if (idx < end) {
                uint32_t pid = ids[idx];
                int ix = pid & 1023, iy = (pid >> 10) & 1023, iz = pid >> 20;
                float4 tx = T[ix], ty = T[Nx + iy], tz = T[Nx + Ny + iz];
                ff s2 = ff_add(ff_add(ff{tx.x, tx.y}, ff{ty.x, ty.y}), ff{tz.x, tz.y});
                ff s = ff_sqrt(s2);
                float b = floorf(s.hi);
                float f = __fadd_rn(__fsub_rn(s.hi, b), s.lo);
                // bring f into [0, 1); -tiny + 1 rounds to 1.0, hence two steps
                if (f < 0.0f) {
                    f = __fadd_rn(f, 1.0f);
                    b -= 1.0f;
                }
                if (f >= 1.0f) {
                    f = __fsub_rn(f, 1.0f);
                    b += 1.0f;
                }
                int rr = (int)b - ISM_SB * q;
                float amp = tx.z * ty.z * tz.z * __fdividef(J.amp_scale, s.hi);
                if (rr < -1 || rr > ISM_SB - 1) {
                    atomicOr(status, (uint32_t)ISM_DEVICE_FLAG_BIN);
                    rr = 0;
                    amp = 0.0f;
                }
                f = fmaxf(f, 0x1p-60f);
                float P2 = amp * sinpif(f) * 0.15915494309189535f;  // A sin(pi f) / (2 pi)
                float Qv = (rr & 1) ? -P2 : P2;
                float st, ct;
                sincospif(((float)rr + f) * inv2Nw, &st, &ct);
                R->rec[warp][lane] = make_float4(f, Qv, Qv * ct, Qv * st);
                R->rr[warp][lane] = (float)rr;
            }
            __syncwarp();
            const int n = (int)min(32u, end - cb);
            for (int i = 0; i < n; ++i) {
                const float4 rc = R->rec[warp][i];
                const float rrf = R->rr[warp][i];
                const bool upper = (float)lane <= rrf;  // window register m = s + 1 instead of s
#pragma unroll
                for (int s = 0; s < SLOTS; ++s) {
                    float xb = upper ? xo[s + 1] : xo[s];
                    float C = upper ? Cm[s + 1] : Cm[s];
                    float Sn = upper ? Sm[s + 1] : Sm[s];
                    float x = __fsub_rn(__fsub_rn(xb, rrf), rc.x);
                    float term = __fmaf_rn(C, rc.z, __fmaf_rn(Sn, rc.w, rc.y));
                    if (MASK) {
                        float pos = (float)(lane + 32 * (s + (upper ? 1 : 0)));
                        bool valid = (pos <= rrf + (float)(2 * H)) && (fabsf(x) < halfNw);
                        term = valid ? term : 0.0f;
                    }
                    float v = term * ism_rcp(x);
                    if (upper) acc[s + 1] += v;
                    else acc[s] += v;
                }
            }
            __syncwarp();
        }
    }

    // store signed window rows
#pragma unroll
    for (int m = 0; m <= SLOTS; ++m) {
        int p = lane + 32 * m;
        float sg = ((p + H + 1) & 1) ? -1.0f : 1.0f;
        rows[(warp * (SLOTS + 1) + m) * 32 + lane] = sg * acc[m];
    }
    __syncthreads();

    // segment s of this tile = samples [32 (q0 + s) - H, +32)
    const int q0 = tile * ISM_TILE_SB;
    float* out = J.out + (long long)r * J.n_S;
    float* seam = seams + J.seam_base + ((long long)r * J.n_tiles + tile) * (64LL * SLOTS);
    {
        const int s = warp;
        float v = 0.0f;
#pragma unroll
        for (int m = 0; m <= SLOTS; ++m)
            if (s - m >= 0) v += rows[((s - m) * (SLOTS + 1) + m) * 32 + lane];
        if (s >= SLOTS) {
            int k = ISM_SB * (q0 + s) - H + lane;
            if (k >= 0 && k < J.n_ism) out[k] = v;
        } else {
            seam[s * 32 + lane] = v;
        }
        if (warp < SLOTS) {  // contributions spilling past the tile end
            const int s2 = warp;
            float v2 = 0.0f;
#pragma unroll
            for (int m = 1; m <= SLOTS; ++m)
                if (m >= s2 + 1) v2 += rows[((ISM_TILE_SB + s2 - m) * (SLOTS + 1) + m) * 32 + lane];
            seam[(SLOTS + s2) * 32 + lane] = v2;
        }
    }
}

template <int SLOTS, bool MASK>
int launch_one(const JobTable& t, const WsPlan& p, char* ws, cudaStream_t s)
{
    size_t sm = (size_t)((t.max_axis_sum + 1) & ~1) * sizeof(float4) + sizeof(RecSmem) +
                (size_t)ISM_TILE_SB * (SLOTS + 1) * 32 * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(accum_kernel<SLOTS, MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return (int)e;
    accum_kernel<SLOTS, MASK><<<(unsigned)p.acc_ctas, ISM_TILE_SB * 32, sm, s>>>(
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
