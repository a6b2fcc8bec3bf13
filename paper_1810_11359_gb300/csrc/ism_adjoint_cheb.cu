// ism_adjoint_cheb.cu -- gradients of a loss through the image-source RIR for
// a window of exactly 32 taps, through the Chebyshev expansion of the tap
// functions that the forward FP32 form uses (the paper computes forward RIRs
// only; the chain rule is that of eq. (1)-(6)).
//
// With g_k = dLoss/dh[k], an image of integer delay b = 32 q + o - 1 and
// fractional delay f has, per tap t = 0 .. 31 (sample k = 32 q - 16 + o + t,
// tap function g_t(f) = delta'(t - 15 - f) = sum_i c_{t,i} T_i(u), u = 2 f - 1):
//   ga = sum_t g_k delta'(t - 15 - f)  = sum_i Gamma_i(q, o) T_i(u)
//   ge = sum_t g_k delta''(t - 15 - f) = -2 sum_i Gamma_i(q, o) T_i'(u)
// (delta'' = d delta'/dx; d/df = -d/dx and du/df = 2), with the tables
//   Gamma_i(q, o) = sum_t c_{t,i} g[32 q - 16 + o + t].
// So each (bin, offset) costs 9 dot products of length 32 once, and each
// image two Chebyshev sums of degree 8 instead of 32 tap evaluations.  The
// truncation of the series costs 6.4e-8 of an image's amplitude in ga and, by
// Markov's inequality for the derivative of a degree-8 polynomial, at most
// 64 times that in ge.
//
// From ga and ge an image adds to its RIR's 12 gradient components
//   c = dLoss/dd = -(A / d) ga - (f_s / c) A ge       (eq. (2)-(4))
//   dLoss/dp_r  += c (p_r - p_n) / d,   dLoss/dp_s += -c (d p_n / d p_s)(p_r - p_n) / d
//   dLoss/dbeta_w += ga dA/dbeta_w      (product form of eq. (4), valid at beta = 0)
//
// One CTA owns the 8 delay bins of one shell of one RIR and enumerates its
// images itself (ism_shell.cuh), as the forward's fused kernel does: no image
// ids, no counting sort.  Warp w first builds the Gamma table of bin q0 + w
// (lane = offset o) from dLoss/dh over the bin's 64-sample window; then every
// lane accumulates the gradients of the images it is handed in 12 registers.
// The lanes' sums are reduced by a fixed butterfly per warp and the warps in
// warp order; the CTA's 12 sums go to the slot of its first bin (zeros to the
// slots of its other bins), which the reduction kernel adds per RIR in bin
// order: no atomics, bit-identical from run to run.
#include "ism_shell.cuh"

namespace {

#define SA_B ISM_SHELL_BINS   // delay bins per CTA
#define SA_WARPS 8            // warps per CTA (one per bin for the tables)
#define SA_GV 3               // float4 per Gamma row (9 terms + 3 pad)
#define SA_NG 12              // gradient components: dp_r[3], dp_s[3], dbeta[6]

__global__ void __launch_bounds__(SA_WARPS * 32, 4) shell_adjoint_kernel(const __grid_constant__ JobTable t,
                                                                          const float4* __restrict__ tbl,
                                                                          const float4* __restrict__ dtbl,
                                                                          float* __restrict__ gpart)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int jid, r, grp;
    if (!shell_cta(t, blockIdx.x, &jid, &r, &grp)) return;   // CTA-uniform
    const JobDev& J = t.j[jid];
    const int q0 = grp * SA_B;
    const int nb = min(SA_B, J.Q - q0);
    const int Nx = J.N[0], Ny = J.N[1];
    const int n_axis = Nx + Ny + J.N[2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // shared memory: axis tables | derivative tables | Gamma tables | dLoss/dh windows |
    // warp sums | row prefix | per-warp column records
    const int axis_pad = (t.max_axis_sum + 1) & ~1;
    float4* T = reinterpret_cast<float4*>(smem);
    float4* X = T + axis_pad;                                   // x_n - x_r, dF/dbeta_lo, dF/dbeta_hi, d x_n / d x_s
    float4* Gam = X + axis_pad;                                 // [bin][offset][SA_GV]: Gamma_0..8
    float* gw = reinterpret_cast<float*>(Gam + SA_B * 32 * SA_GV);   // [bin][64]
    float* red = gw + SA_B * 64;                                // [warp][SA_NG]
    int* rowpre = reinterpret_cast<int*>(red + SA_WARPS * SA_NG);
    int* rowy0 = rowpre + ((t.max_axis_sum + 4) & ~3);
    float4* recf = reinterpret_cast<float4*>(rowy0 + ((t.max_axis_sum + 4) & ~3));
    int4* reci = reinterpret_cast<int4*>(recf + SA_WARPS * 32);
    int* st = reinterpret_cast<int*>(reci + SA_WARPS * 32);     // [warps][33]

    const float4* Tg = tbl + J.tbl_base + (long long)r * n_axis;
    const float4* Xg = dtbl + J.tbl_base + (long long)r * n_axis;
    for (int e = threadIdx.x; e < n_axis; e += blockDim.x) {
        T[e] = Tg[e];
        X[e] = Xg[e];
    }
    // dLoss/dh over the windows of the CTA's bins (samples 32 q - 16 + P, P < 64; 0 outside [0, n_ism))
    const float* go = J.grad_out + (long long)r * J.n_S;
    for (int e = threadIdx.x; e < SA_B * 64; e += blockDim.x) {
        const int q = q0 + e / 64;
        const int k = ISM_SB * q - 16 + (e % 64);
        gw[e] = (q < J.Q && k >= 0 && k < J.n_ism) ? go[k] : 0.0f;
    }
    __syncthreads();
    {   // Gamma_i(q0 + warp, o = lane): 9 dot products of length 32 with the tap coefficients
        const float* gwb = gw + warp * 64;
        float acc[ISM_CHEB_N];
#pragma unroll
        for (int i = 0; i < ISM_CHEB_N; ++i) acc[i] = 0.0f;
#pragma unroll
        for (int tt = 0; tt < 32; ++tt) {
            const float gk = gwb[lane + tt];
#pragma unroll
            for (int i = 0; i < ISM_CHEB_N; ++i) acc[i] = __fmaf_rn(t.cheb[tt * ISM_CHEB_N + i], gk, acc[i]);
        }
        float4* row = Gam + (warp * 32 + lane) * SA_GV;
        row[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
        row[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
        row[2] = make_float4(acc[8], 0.0f, 0.0f, 0.0f);
    }

    // exact delays b owned by this CTA: [b_lo, b_hi), b <= n_ism + 14 (later taps miss [0, n_ism))
    const Shell sh = shell_setup(J, T, r, ISM_SB * q0 - 1, min(ISM_SB * (q0 + nb) - 1, J.n_ism + J.H - 1));
    const int n_cols = shell_rows(sh, T, rowpre, rowy0);   // (synchronises the CTA: the tables are ready)

    float G[SA_NG];
#pragma unroll
    for (int c = 0; c < SA_NG; ++c) G[c] = 0.0f;
    const float amp_scale = J.amp_scale;
    const float kfs = J.kfs_hi;   // f_s / c
    shell_walk<SA_WARPS>(sh, T, rowpre, rowy0, n_cols, make_float2(0.0f, 0.0f), recf + warp * 32, reci + warp * 32,
                         st + warp * 33, warp, lane,
                         [&](int b, float f, float s, const float4& cf, int ixy, int iz, const float4& tz) {
        const int q = (b + 1) >> 5;
        const int o = b - ISM_SB * q + 1;   // offset index rr + 1 in [0, 32)
        const float4* Gr = Gam + ((q - q0) * 32 + o) * SA_GV;
        const float4 g0 = Gr[0], g1 = Gr[1], g2 = Gr[2];
        const float Gb[ISM_CHEB_N] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w, g2.x};
        // ga = sum_i Gamma_i T_i(u), gd = sum_i Gamma_i T_i'(u)
        const float uu = __fmaf_rn(2.0f, f, -1.0f);
        const float u2 = uu + uu;
        float ga = __fmaf_rn(Gb[1], uu, Gb[0]);
        float gd = Gb[1];
        float tp = 1.0f, tc = uu, dp = 0.0f, dc = 1.0f;
#pragma unroll
        for (int i = 2; i < ISM_CHEB_N; ++i) {
            const float tn = __fmaf_rn(u2, tc, -tp);
            const float dn = __fmaf_rn(u2, dc, __fmaf_rn(2.0f, tc, -dp));   // T_i' = 2 T_(i-1) + 2 u T_(i-1)' - T_(i-2)'
            const float gi = Gb[i];
            ga = __fmaf_rn(gi, tn, ga);
            gd = __fmaf_rn(gi, dn, gd);
            tp = tc;
            tc = tn;
            dp = dc;
            dc = dn;
        }
        const int ix = ixy & 0xFFFF, iy = ixy >> 16;
        const float4 tx = T[ix], ty = T[Nx + iy];
        const float4 xx = X[ix], xy = X[Nx + iy], xz = X[Nx + Ny + iz];
        const float rs = ism_rcp(s);
        const float A = cf.z * tz.z * amp_scale * rs;        // eq. (4), as in the forward
        // c = -(A / d) ga - (f_s / c) A ge with 1 / d = (f_s / c) / s and ge = -2 gd
        const float cr = A * kfs * __fmaf_rn(2.0f, gd, -rs * ga) * rs;
        // (p_r - p_n) / d = -D / s per axis (D = signed offset in samples)
        G[0] = __fmaf_rn(-cr, tx.w, G[0]);
        G[1] = __fmaf_rn(-cr, ty.w, G[1]);
        G[2] = __fmaf_rn(-cr, tz.w, G[2]);
        G[3] = __fmaf_rn(cr, xx.w * tx.w, G[3]);
        G[4] = __fmaf_rn(cr, xy.w * ty.w, G[4]);
        G[5] = __fmaf_rn(cr, xz.w * tz.w, G[5]);
        const float gs = ga * amp_scale * rs;                // ga / (4 pi d)
        const float Fyz = ty.z * tz.z, Fxz = tx.z * tz.z, Fxy = cf.z;
        G[6] = __fmaf_rn(gs, xx.y * Fyz, G[6]);
        G[7] = __fmaf_rn(gs, xx.z * Fyz, G[7]);
        G[8] = __fmaf_rn(gs, xy.y * Fxz, G[8]);
        G[9] = __fmaf_rn(gs, xy.z * Fxz, G[9]);
        G[10] = __fmaf_rn(gs, xz.y * Fxy, G[10]);
        G[11] = __fmaf_rn(gs, xz.z * Fxy, G[11]);
    });

    // lanes (fixed butterfly; lane 0's order), then warps in order
#pragma unroll
    for (int c = 0; c < SA_NG; ++c) {
        float v = G[c];
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
        if (lane == 0) red[warp * SA_NG + c] = v;
    }
    __syncthreads();
    float* dst = gpart + J.gpart_base + ((long long)r * J.Q + q0) * SA_NG;
    if (threadIdx.x < SA_NG) {
        float v = red[threadIdx.x];
        for (int w = 1; w < SA_WARPS; ++w) v += red[w * SA_NG + threadIdx.x];
        dst[threadIdx.x] = v;
    }
    for (int e = threadIdx.x; e < (nb - 1) * SA_NG; e += blockDim.x) dst[SA_NG + e] = 0.0f;
}

size_t shell_adjoint_smem(const JobTable& t)
{
    const size_t axis_pad = (size_t)((t.max_axis_sum + 1) & ~1);
    const size_t rows = (size_t)((t.max_axis_sum + 4) & ~3);
    return 2 * axis_pad * sizeof(float4) + (size_t)SA_B * 32 * SA_GV * sizeof(float4) +
           (size_t)SA_B * 64 * sizeof(float) + (size_t)SA_WARPS * SA_NG * sizeof(float) + 2 * rows * sizeof(int) +
           (size_t)SA_WARPS * 32 * (sizeof(float4) + sizeof(int4)) + (size_t)SA_WARPS * 33 * sizeof(int);
}

}  // namespace

int ism_launch_adjoint_cheb(const JobTable& t, const WsPlan& p, char* ws, void* stream, int* launched)
{
    *launched = 0;
    if (p.shell_ctas <= 0) return 0;
    const size_t sm = shell_adjoint_smem(t);
    static std::atomic<unsigned long long> opened{0};
    int rc = ism_open_smem((const void*)shell_adjoint_kernel, &opened);
    if (rc) return rc;
    cudaError_t e = cudaFuncSetAttribute(shell_adjoint_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);   // 4 CTAs of ~32 KB per SM
    if (e != cudaSuccess) return (int)e;
    shell_adjoint_kernel<<<(unsigned)p.shell_ctas, SA_WARPS * 32, sm, (cudaStream_t)stream>>>(
        t, reinterpret_cast<const float4*>(ws + p.tbl_off), reinterpret_cast<const float4*>(ws + p.dtbl_off),
        reinterpret_cast<float*>(ws + p.gpart_off));
    *launched = 1;
    return (int)cudaGetLastError();
}
