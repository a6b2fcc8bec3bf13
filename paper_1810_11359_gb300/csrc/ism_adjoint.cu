// ism_adjoint.cu -- gradients of a loss through the image-source RIR: the
// adjoint of eq. (1)-(6) (the paper computes forward RIRs only), per tap, for
// windows other than exactly 32 taps (those take the fused Chebyshev adjoint
// of ism_adjoint_cheb.cu), and the reduction of every job's gradients.
//
// The binned image lists of the forward pass (enumeration + counting sort)
// are reused: one CTA per (RIR, tile of 8 delay bins), one warp per bin, as
// in the accumulation kernel.  The warp keeps dLoss/dh over its bin's window
// (32 (SLOTS + 1) samples from 32 q - H) in shared memory; lane l of the
// warp evaluates, for every image, the taps t = l + 32 s, j = t - H + 1,
// x = j - f:
//   delta'(x)     = w(x) sinc(x)                   w = (1 + cos(2 pi x / N_w)) / 2
//   d delta'/dx   = w'(x) sinc(x) + w(x) sinc'(x)  sinc'(x) = (cos(pi x) - sinc(x)) / x
// from the per-image values sin(pi f), cos(pi f), cos phi, sin phi (phi =
// 2 pi f / N_w) and the lane constants of j, exactly as the forward kernel
// factorises eq. (6).  With g_k = dLoss/dh[k] at the tap's sample it forms
//   a = g_k delta'(x)          (image's dLoss/dA share of this tap)
//   c = -(A / d) a - (f_s / c) A g_k delta''(x)   (dLoss/dd share, eq. (2)-(4))
// and accumulates, per lane, c (p_r - p_n) / d, -c (+-1)(p_r - p_n) / d and
// a dA/dbeta_w over all images of the bin -- the per-image factors come from a
// record computed once per image.  The lanes' sums are reduced by a fixed
// butterfly per warp, the bins of an RIR in bin order, and the RIRs of a
// source, receiver or room in index order: no atomics, bit-identical from
// run to run.
#include "ism_device.cuh"

namespace {

#define ADJ_CHUNK 32   // image records per step (one per lane)
#define ADJ_NG 12      // gradient components: dp_r[3], dp_s[3], dbeta[6]

struct AdjRec {
    float4 a;   // f, sin(pi f) / pi, cos(pi f), rr (int bits)
    float4 b;   // cos(phi), sin(phi), -A / d, -(f_s / c) A
    float4 u;   // (p_r - p_n) / d per axis
    float4 v;   // -(d p_n / d x_s)(p_r - p_n) / d per axis
    float4 q0;  // dA / d beta_w, w = 0..3
    float4 q1;  // dA / d beta_w, w = 4, 5
};

template <int SLOTS, bool MASK>
__global__ void __launch_bounds__(ISM_ACC_WARPS * 32) adjoint_kernel(const __grid_constant__ JobTable t,
                                                                      const float4* __restrict__ tbl,
                                                                      const float4* __restrict__ dtbl,
                                                                      const uint32_t* __restrict__ hist,
                                                                      const uint32_t* __restrict__ ids,
                                                                      float* __restrict__ gpart,
                                                                      uint32_t* __restrict__ status)
{
    constexpr int WIN = 32 * (SLOTS + 1);
    extern __shared__ __align__(16) unsigned char smem[];
    const long long g = blockIdx.x;
    const int jid = ism_find_job(t, g, [](const JobDev& j) { return j.adj_cta_base; });
    const JobDev& J = t.j[jid];
    const bool exact = (J.Nw == (float)(2 * J.H)) && (2 * J.H == 32 * J.slots);
    if (J.slots != SLOTS || exact == MASK) return;  // another instantiation handles this job

    const long long local = g - J.adj_cta_base;
    const int r = (int)(local / J.n_tiles);
    const int tile = J.n_tiles - 1 - (int)(local % J.n_tiles);
    const int Nx = J.N[0], Ny = J.N[1], Nz = J.N[2];
    const int n_axis = Nx + Ny + Nz;
    const int H = J.H;

    const int axis_pad = (t.max_axis_sum + 1) & ~1;
    float4* T = reinterpret_cast<float4*>(smem);      // S_hi, S_lo, F (forward tables)
    float4* X = T + axis_pad;                          // x_n - x_r, dF/dbeta_lo, dF/dbeta_hi, d x_n / d x_s
    float* gw_all = reinterpret_cast<float*>(X + axis_pad);          // [warp][WIN]
    AdjRec* rec_all = reinterpret_cast<AdjRec*>(gw_all + ISM_ACC_WARPS * WIN);  // [warp][ADJ_CHUNK]

    // forward tables and the geometry kernel's backward tables (x_n - x_r, dF/dbeta, d x_n / d x_s)
    const float4* Tg = tbl + J.tbl_base + (long long)r * n_axis;
    const float4* Xg = dtbl + J.tbl_base + (long long)r * n_axis;
    for (int e = threadIdx.x; e < n_axis; e += blockDim.x) {
        T[e] = Tg[e];
        X[e] = Xg[e];
    }

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* gw = gw_all + warp * WIN;
    AdjRec* R = rec_all + warp * ADJ_CHUNK;
    const int q = tile * ISM_TILE_BINS + warp;

    // dLoss/dh over the bin's window (samples 32 q - H + P, P < WIN; 0 outside [0, n_ism))
    {
        const float* go = J.grad_out + (long long)r * J.n_S;
        const int k0 = ISM_SB * q - H;
        for (int P = lane; P < WIN; P += 32) {
            const int k = k0 + P;
            gw[P] = (q < J.Q && k >= 0 && k < J.n_ism) ? go[k] : 0.0f;
        }
    }

    // lane constants of the taps t = lane + 32 s, j = t - H + 1
    float jf[SLOTS], sg[SLOTS], Cj[SLOTS], Sj[SLOTS];
    bool tap_ok[SLOTS];
    const float inv2Nw = 2.0f / J.Nw;
    const float twopi_Nw = 6.283185307179586f / J.Nw;
    const float pi_Nw = 3.14159265358979f / J.Nw;
    const bool small_phase = J.Nw >= 16.0f;
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
        const int tt = lane + 32 * s;
        const int j = tt - H + 1;
        jf[s] = (float)j;
        sg[s] = (j & 1) ? 1.0f : -1.0f;  // (-1)^(j+1)
        sincospif((float)j * inv2Nw, &Sj[s], &Cj[s]);
        tap_ok[s] = tt < 2 * H;
    }
    const float halfNw = 0.5f * J.Nw;
    const float kfs = J.kfs_hi;           // f_s / c
    __syncthreads();

    float G[ADJ_NG];
#pragma unroll
    for (int c = 0; c < ADJ_NG; ++c) G[c] = 0.0f;

    if (q < J.Q) {
        const long long hb = J.hist_base + ((long long)r * J.Q + q) * J.U;
        const uint32_t start = hist[hb];
        const uint32_t end = hist[hb + J.U];
        for (uint32_t c0 = start; c0 < end; c0 += ADJ_CHUNK) {
            const int m = (int)min((uint32_t)ADJ_CHUNK, end - c0);
            if (lane < m) {
                const uint32_t pid = ids[c0 + lane];
                const int ix = pid & 1023, iy = (pid >> 10) & 1023, iz = pid >> 20;
                const float4 tx = T[ix], ty = T[Nx + iy], tz = T[Nx + Ny + iz];
                const float4 xx = X[ix], xy = X[Nx + iy], xz = X[Nx + Ny + iz];
                // exact delay s = b + f (float-float), as in the forward kernel
                const ff s2 = ff_add(ff_add(ff{tx.x, tx.y}, ff{ty.x, ty.y}), ff{tz.x, tz.y});
                const ff sq = ff_sqrt(s2);
                float b = floorf(sq.hi);
                float f = __fadd_rn(__fsub_rn(sq.hi, b), sq.lo);
                if (f < 0.0f) {
                    f = __fadd_rn(f, 1.0f);
                    b -= 1.0f;
                }
                if (f >= 1.0f) {
                    f = __fsub_rn(f, 1.0f);
                    b += 1.0f;
                }
                int rr = ism_int_of_integral(b) - ISM_SB * q;
                const bool bad = rr < -1 || rr > ISM_SB - 1;
                if (bad) atomicOr(status, (uint32_t)ISM_DEVICE_FLAG_BIN);
                f = fmaxf(f, 0x1p-60f);
                const float inv_s = ism_rcp(sq.hi);
                const float Fyz = ty.z * tz.z, Fxz = tx.z * tz.z, Fxy = tx.z * ty.z;
                const float A = bad ? 0.0f : tx.z * Fyz * J.amp_scale * inv_s;    // eq. (4)
                const float inv_d = kfs * inv_s;                                  // 1 / d
                const float sc = bad ? 0.0f : J.amp_scale * inv_s;               // 1 / (4 pi d)
                float sp, cp;
                if (small_phase) ism_sincos_small(f * twopi_Nw, &sp, &cp);
                else sincospif(f * inv2Nw, &sp, &cp);
                float s1, c1;
                sincospif(f, &s1, &c1);
                AdjRec o;
                o.a = make_float4(f, s1 * 0.3183098861837907f, c1, __int_as_float(bad ? 0 : rr));
                o.b = make_float4(cp, sp, -A * inv_d, -kfs * A);
                const float ux = -xx.x * inv_d, uy = -xy.x * inv_d, uz = -xz.x * inv_d;
                o.u = make_float4(ux, uy, uz, 0.0f);
                o.v = make_float4(-xx.w * ux, -xy.w * uy, -xz.w * uz, 0.0f);
                o.q0 = make_float4(xx.y * Fyz * sc, xx.z * Fyz * sc, xy.y * Fxz * sc, xy.z * Fxz * sc);
                o.q1 = make_float4(xz.y * Fxy * sc, xz.z * Fxy * sc, 0.0f, 0.0f);
                R[lane] = o;
            }
            __syncwarp();
            for (int i = 0; i < m; ++i) {
                const float4 ra = R[i].a, rb = R[i].b;
                const int rr = __float_as_int(ra.w);
                float ga = 0.0f, ge = 0.0f;   // this lane's taps: sum g delta', sum g delta''
#pragma unroll
                for (int s = 0; s < SLOTS; ++s) {
                    const float x = jf[s] - ra.x;
                    const float rx = ism_rcp(x);
                    const float sinc = sg[s] * ra.y * rx;                  // sin(pi x) / (pi x)
                    const float cpx = -sg[s] * ra.z;                       // cos(pi x)
                    float sincp = (cpx - sinc) * rx;                       // sinc'(x)
                    const float x2 = x * x;
                    const float series = x * __fmaf_rn(x2, 3.2469697011334144f, -3.2898681336964524f);
                    sincp = fabsf(x) < 0.015625f ? series : sincp;         // -pi^2 x / 3 + pi^4 x^3 / 30
                    const float c2 = __fmaf_rn(Sj[s], rb.y, Cj[s] * rb.x); // cos(2 pi x / N_w)
                    const float s2 = __fmaf_rn(-Cj[s], rb.y, Sj[s] * rb.x);  // sin(2 pi x / N_w)
                    const float w = __fmaf_rn(0.5f, c2, 0.5f);
                    const float wp = -pi_Nw * s2;
                    float dp = w * sinc;
                    float ddp = __fmaf_rn(wp, sinc, w * sincp);
                    if (MASK) {
                        const bool ok = tap_ok[s] && fabsf(x) < halfNw;
                        dp = ok ? dp : 0.0f;
                        ddp = ok ? ddp : 0.0f;
                    }
                    const float gk = gw[rr + 1 + lane + 32 * s];
                    ga = __fmaf_rn(gk, dp, ga);
                    ge = __fmaf_rn(gk, ddp, ge);
                }
                const float c = __fmaf_rn(rb.z, ga, rb.w * ge);   // -A/d a - (f_s/c) A e
                const float4 u = R[i].u, v = R[i].v, q0 = R[i].q0, q1 = R[i].q1;
                G[0] = __fmaf_rn(c, u.x, G[0]);
                G[1] = __fmaf_rn(c, u.y, G[1]);
                G[2] = __fmaf_rn(c, u.z, G[2]);
                G[3] = __fmaf_rn(c, v.x, G[3]);
                G[4] = __fmaf_rn(c, v.y, G[4]);
                G[5] = __fmaf_rn(c, v.z, G[5]);
                G[6] = __fmaf_rn(ga, q0.x, G[6]);
                G[7] = __fmaf_rn(ga, q0.y, G[7]);
                G[8] = __fmaf_rn(ga, q0.z, G[8]);
                G[9] = __fmaf_rn(ga, q0.w, G[9]);
                G[10] = __fmaf_rn(ga, q1.x, G[10]);
                G[11] = __fmaf_rn(ga, q1.y, G[11]);
            }
            __syncwarp();
        }
#pragma unroll
        for (int c = 0; c < ADJ_NG; ++c) {
            float v = G[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            G[c] = v;
        }
        if (lane == 0) {
            float* dst = gpart + J.gpart_base + ((long long)r * J.Q + q) * ADJ_NG;
#pragma unroll
            for (int c = 0; c < ADJ_NG; ++c) dst[c] = G[c];
        }
    }
}

// Per job: bins -> RIRs, RIRs -> sources, receivers and the room (index
// order).  One CTA per job.  A warp sums the Q bin records of one (RIR,
// component): lane l adds the bins l, l + 32, ... in order, then a fixed
// butterfly adds the lanes (lane 0's order is the result), so the per-RIR sums
// take Q / 32 dependent loads instead of Q.
__global__ void __launch_bounds__(256) adjoint_reduce_kernel(const __grid_constant__ JobTable t,
                                                             const float* __restrict__ gpart,
                                                             float* __restrict__ rgrad)
{
    const JobDev& J = t.j[blockIdx.x];
    const long long R = J.n_rir;
    float* rg = rgrad + J.rgrad_base;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (long long e = warp; e < R * ADJ_NG; e += blockDim.x >> 5) {
        const long long r = e / ADJ_NG;
        const int c = (int)(e % ADJ_NG);
        const float* src = gpart + J.gpart_base + r * J.Q * ADJ_NG + c;
        float v = 0.0f;
        for (int q = lane; q < J.Q; q += 32) v += src[(long long)q * ADJ_NG];
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
        if (lane == 0) rg[e] = v;
    }
    __syncthreads();
    const int n_out = 6 + 3 * J.n_src + 3 * J.n_rcv;
    for (int e = threadIdx.x; e < n_out; e += blockDim.x) {
        float v = 0.0f;
        if (e < 6) {
            for (long long r = 0; r < R; ++r) v += rg[r * ADJ_NG + 6 + e];
            if (J.grad_beta) J.grad_beta[e] = v;
        } else if (e < 6 + 3 * J.n_src) {
            const int i = (e - 6) / 3, a = (e - 6) % 3;
            for (int j = 0; j < J.n_rcv; ++j) v += rg[((long long)i * J.n_rcv + j) * ADJ_NG + 3 + a];
            if (J.grad_src) J.grad_src[3 * i + a] = v;
        } else {
            const int j = (e - 6 - 3 * J.n_src) / 3, a = (e - 6 - 3 * J.n_src) % 3;
            for (int i = 0; i < J.n_src; ++i) v += rg[((long long)i * J.n_rcv + j) * ADJ_NG + a];
            if (J.grad_rcv) J.grad_rcv[3 * j + a] = v;
        }
    }
}

template <int SLOTS, bool MASK>
int launch_adj(const JobTable& t, const WsPlan& p, char* ws, cudaStream_t s)
{
    const size_t axis_pad = (size_t)((t.max_axis_sum + 1) & ~1);
    const size_t sm = 2 * axis_pad * sizeof(float4) + (size_t)ISM_ACC_WARPS * 32 * (SLOTS + 1) * sizeof(float) +
                      (size_t)ISM_ACC_WARPS * ADJ_CHUNK * sizeof(AdjRec);
    static std::atomic<unsigned long long> opened{0};
    int rc = ism_open_smem((const void*)adjoint_kernel<SLOTS, MASK>, &opened);
    if (rc) return rc;
    adjoint_kernel<SLOTS, MASK><<<(unsigned)p.adj_ctas, ISM_ACC_WARPS * 32, sm, s>>>(
        t, reinterpret_cast<const float4*>(ws + p.tbl_off), reinterpret_cast<const float4*>(ws + p.dtbl_off),
        reinterpret_cast<const uint32_t*>(ws + p.hist_off),
        reinterpret_cast<const uint32_t*>(ws + p.ids_off), reinterpret_cast<float*>(ws + p.gpart_off),
        reinterpret_cast<uint32_t*>(ws + p.status_off));
    return (int)cudaGetLastError();
}

}  // namespace

int ism_launch_adjoint(const JobTable& t, const WsPlan& p, char* ws, void* stream, int* launched)
{
    *launched = 0;
    cudaStream_t s = (cudaStream_t)stream;
    bool need[2][ISM_MAX_SLOTS + 1] = {};
    for (int i = 0; i < t.n_jobs && p.adj_ctas > 0; ++i) {
        const JobDev& J = t.j[i];
        if (J.adj_cheb) continue;   // the fused Chebyshev adjoint takes it
        bool exact = (J.Nw == (float)(2 * J.H)) && (2 * J.H == 32 * J.slots);
        need[exact ? 0 : 1][J.slots] = true;
    }
    int rc = 0;
#define ISM_L(SL)                                                                 \
    if (!rc && need[0][SL]) rc = launch_adj<SL, false>(t, p, ws, s), ++*launched; \
    if (!rc && need[1][SL]) rc = launch_adj<SL, true>(t, p, ws, s), ++*launched;
    ISM_L(1) ISM_L(2) ISM_L(3) ISM_L(4) ISM_L(5) ISM_L(6) ISM_L(7) ISM_L(8)
#undef ISM_L
    if (rc) return rc;
    int fused = 0;
    if ((rc = ism_launch_adjoint_cheb(t, p, ws, stream, &fused))) return rc;
    *launched += fused;
    adjoint_reduce_kernel<<<(unsigned)t.n_jobs, 256, 0, s>>>(t, reinterpret_cast<const float*>(ws + p.gpart_off),
                                                             reinterpret_cast<float*>(ws + p.rgrad_off));
    ++*launched;
    return (int)cudaGetLastError();
}
