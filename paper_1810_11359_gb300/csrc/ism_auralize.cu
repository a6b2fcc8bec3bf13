// ism_auralize.cu -- moving sources (Section 4): the source signal is cut into
// one segment per trajectory point, each segment is filtered by the RIRs of its
// point (one per microphone) and the filtered segments are overlap-added:
//   y[m][t] = sum_p sum_{s in [a_p, a_(p+1))} x[s] h[p][m][t - s].
// The paper does this with batched FFTs; here it is a direct FP32 convolution
// on the FMA pipe (the RIRs are long, the signal is short, and the sum has a
// fixed order).
//
// One CTA owns 128 consecutive output samples and up to 8 microphones; its 4
// warps split the segments that reach the tile round-robin and add their
// partial sums in warp order at the end.  Lane l of a warp owns the outputs
// T0 + 4 l + r, r = 0 .. 3, for the 8 microphones (32 accumulators).  For one
// segment the taps k that connect it to the tile are walked in chunks of 128:
// the chunk's taps of the 8 microphones and the signal window it needs (the
// samples outside the segment zeroed) are staged in the warp's shared memory,
// the taps as [microphone][k] rows copied with 128-bit loads when every RIR
// row starts on a 16-byte boundary (n_S a multiple of 4; the chunk's first
// tap rounded down to a multiple of 4 -- the extra taps meet zeroed signal
// samples), else one float at a time.  The taps go in groups of 4: for taps
// k .. k + 3 the lane's 16 products need the 7 signal values
// x[T0 + 4 l - k - 3 .. T0 + 4 l - k + 3], two aligned float4 of the window of
// which the later one is the previous group's earlier one, so a group costs
// one 128-bit signal load (the 32 lanes read 512 contiguous bytes) and eight
// broadcast 128-bit tap loads (taps k .. k + 3 of each microphone) for 128
// FFMA; every shared address is the lane's base plus a constant.  (8 outputs per lane: fewer CTAs than SM
// slots, 13 % of the warps active, measured 10 % slower.)
#include "ism_device.cuh"

namespace {

#define AU_R 4                       // outputs per lane
#define AU_M 8                       // microphones per CTA
#define AU_KC 128                    // taps per staged chunk
#define AU_WARPS 4                   // warps per CTA (segments split round-robin)
#define AU_TILE (32 * AU_R)          // outputs per CTA
#define AU_XN (AU_TILE + AU_KC)      // signal samples per chunk (the last one is never used)

static_assert(AU_R == 4 && AU_KC % 4 == 0, "the signal window is read as float4 groups of 4 taps");

struct AuWarp {
    float4 h[AU_M][AU_KC / 4];       // taps of the chunk: [microphone][k / 4]
    float4 x[AU_XN / 4];             // signal window
};

// Segment of sample s (the largest p with a_p <= s): uniform cut when starts
// is NULL, else a binary search over the caller's start array.
__device__ __forceinline__ int au_segment(long long s, int n_x, int n_points, const int* starts)
{
    if (!starts) return (int)min((long long)n_points - 1, ((s + 1) * n_points - 1) / n_x);
    int lo = 0, hi = n_points - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((long long)starts[mid] <= s) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int au_start(int p, int n_x, int n_points, const int* starts)
{
    if (!starts) return (int)(((long long)p * n_x) / n_points);
    return min(max(starts[p], 0), n_x);
}

template <bool VEC>   // 128-bit tap staging (16-byte aligned RIR rows)
__global__ void __launch_bounds__(AU_WARPS * 32, 6) auralize_kernel(const float* __restrict__ x, int n_x,
                                                                 const float* __restrict__ h, int n_points,
                                                                 int n_mics, int n_s,
                                                                 const int* __restrict__ starts,
                                                                 float* __restrict__ y, int n_out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    AuWarp& W = reinterpret_cast<AuWarp*>(smem)[warp];
    const long long T0 = (long long)blockIdx.x * AU_TILE;
    const int m0 = blockIdx.y * AU_M;

    float acc[AU_R][AU_M];
#pragma unroll
    for (int r = 0; r < AU_R; ++r)
#pragma unroll
        for (int m = 0; m < AU_M; ++m) acc[r][m] = 0.0f;

    // samples that reach the tile: s in [T0 - n_s + 1, T0 + TILE - 1]
    const long long s_lo = max(T0 - n_s + 1, 0ll);
    const long long s_hi = min(T0 + AU_TILE - 1, (long long)n_x - 1);
    if (s_lo <= s_hi) {
        const int p_lo = au_segment(s_lo, n_x, n_points, starts);
        const int p_hi = au_segment(s_hi, n_x, n_points, starts);
        for (int p = p_lo + warp; p <= p_hi; p += AU_WARPS) {
            const int a = au_start(p, n_x, n_points, starts);
            const int b = max(a, p + 1 < n_points ? au_start(p + 1, n_x, n_points, starts) : n_x);
            if (b <= a) continue;
            // taps linking [a, b) to the tile (the vector form starts on a multiple of 4)
            const long long k_lo = VEC ? (max(T0 - b + 1, 0ll) & ~3ll) : max(T0 - b + 1, 0ll);
            const long long k_hi = min(T0 + AU_TILE - 1 - a, (long long)n_s - 1);
            const float* hp = h + (long long)p * n_mics * n_s;
            for (long long k0 = k_lo; k0 <= k_hi; k0 += AU_KC) {
                __syncwarp();
                // taps k0 .. k0 + KC - 1 of the 8 microphones (0 past k_hi or past the array)
                if (VEC) {
                    for (int e = lane; e < AU_M * AU_KC / 4; e += 32) {   // 32 lanes: 512 contiguous bytes
                        const int m = e / (AU_KC / 4), kq = e % (AU_KC / 4);
                        const long long k = k0 + 4 * kq;   // k0 % 4 == 0 and n_s % 4 == 0: k .. k + 3 < n_s
                        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        if (k <= k_hi && m0 + m < n_mics)
                            v = *reinterpret_cast<const float4*>(hp + (long long)(m0 + m) * n_s + k);
                        W.h[m][kq] = v;
                    }
                } else {
                    for (int e = lane; e < AU_KC * AU_M; e += 32) {   // coalesced along the taps
                        const int m = e / AU_KC, kk = e % AU_KC;
                        const long long k = k0 + kk;
                        float v = 0.0f;
                        if (k <= k_hi && m0 + m < n_mics) v = hp[(long long)(m0 + m) * n_s + k];
                        reinterpret_cast<float*>(&W.h[m][0])[kk] = v;
                    }
                }
                // signal window: x[T0 - k0 - KC + 1 + j], zero outside [a, b)
                const long long xb = T0 - k0 - AU_KC + 1;
                float* xw = reinterpret_cast<float*>(W.x);
                for (int j = lane; j < AU_XN; j += 32) {
                    const long long s = xb + j;
                    xw[j] = (s >= a && s < b) ? x[s] : 0.0f;
                }
                __syncwarp();
                // output r of the lane at tap kk reads window index 4 l + r + KC - 1 - kk; for the
                // group kk = 4 g + u that is element 3 + r - u of {xa, xb4}, xa = float4 at
                // 4 l + KC - 4 - 4 g, xb4 = the next float4 (the previous group's xa)
                const float4* xl = W.x + lane + (AU_KC - 4) / 4;
                float4 xb4 = xl[1];
                // the groups that hold taps <= k_hi (the last chunk of a segment is partial)
                const int ng = (int)min((long long)(AU_KC / 4), (k_hi - k0) / 4 + 1);
#pragma unroll 2
                for (int g = 0; g < ng; ++g) {
                    const float4 xa = xl[-g];
                    const float v[8] = {xa.x, xa.y, xa.z, xa.w, xb4.x, xb4.y, xb4.z, xb4.w};
                    float hv[AU_M][4];   // taps 4 g .. 4 g + 3 of each microphone
#pragma unroll
                    for (int m = 0; m < AU_M; ++m) {
                        const float4 hm = W.h[m][g];
                        hv[m][0] = hm.x;
                        hv[m][1] = hm.y;
                        hv[m][2] = hm.z;
                        hv[m][3] = hm.w;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int r = 0; r < AU_R; ++r)
#pragma unroll
                            for (int m = 0; m < AU_M; ++m)
                                acc[r][m] = __fmaf_rn(v[3 + r - u], hv[m][u], acc[r][m]);
                    xb4 = xa;
                }
            }
        }
    }

    // partial sums of the warps, added in warp order
    __syncthreads();
    float* red = reinterpret_cast<float*>(smem);   // [warps][R][M][32]
#pragma unroll
    for (int r = 0; r < AU_R; ++r)
#pragma unroll
        for (int m = 0; m < AU_M; ++m) red[((warp * AU_R + r) * AU_M + m) * 32 + lane] = acc[r][m];
    __syncthreads();
    // thread e writes output (t, m) pairs; consecutive threads take consecutive t
    for (int e = threadIdx.x; e < AU_TILE * AU_M; e += blockDim.x) {
        const int m = e / AU_TILE, i = e % AU_TILE;   // i = 8 l + r
        const int l = i / AU_R, r = i % AU_R;
        float v = red[((0 * AU_R + r) * AU_M + m) * 32 + l];
#pragma unroll
        for (int w = 1; w < AU_WARPS; ++w) v += red[((w * AU_R + r) * AU_M + m) * 32 + l];
        const long long t = T0 + i;
        if (t < n_out && m0 + m < n_mics) y[(long long)(m0 + m) * n_out + t] = v;
    }
}

}  // namespace

size_t ism_auralize_smem()
{
    const size_t stage = AU_WARPS * sizeof(AuWarp);
    const size_t red = (size_t)AU_WARPS * AU_R * AU_M * 32 * sizeof(float);
    return stage > red ? stage : red;
}

int ism_launch_auralize(const float* x, int n_x, const float* h, int n_points, int n_mics, int n_s,
                        const int* starts, float* y, void* stream)
{
    const long long n_out = (long long)n_x + n_s - 1;
    const dim3 grid((unsigned)((n_out + AU_TILE - 1) / AU_TILE), (unsigned)((n_mics + AU_M - 1) / AU_M));
    const size_t sm = ism_auralize_smem();
    // 128-bit tap rows when every row starts on a 16-byte boundary
    const bool vec = (n_s % 4 == 0) && (((uintptr_t)h & 15u) == 0);
    auto kern = vec ? auralize_kernel<true> : auralize_kernel<false>;
    static std::atomic<unsigned long long> opened[2] = {{0}, {0}};
    const int rc = ism_open_smem((const void*)kern, &opened[vec ? 1 : 0]);
    if (rc) return rc;
    kern<<<grid, AU_WARPS * 32, sm, (cudaStream_t)stream>>>(x, n_x, h, n_points, n_mics, n_s, starts, y, (int)n_out);
    return (int)cudaGetLastError();
}
