// ism_tail.cu -- window-row sums, envelope fit and the diffuse tail (kernel d).
//
// Section 2.2 ("Diffuse reverberation") models the late RIR as logistic
// noise whose power follows the Sabine decay: 60 dB in T60 (eq. (7)) from
// the end of the image-source part t0 = n_ism / f_s (eq. (8), whose printed
// exponent log10(T60/20) is read as this decay).  Section 2.2 leaves the
// amplitude A to be fitted to the image-source part; here it is the mean over the last
// W = ceil(0.02 f_s) image-source samples of h[k]^2 2^(-g2 (n_ism - k)),
// g2 = 6 log2(10) / (f_s T60), i.e. their power brought forward to t0 along
// the same decay.  The tail is h[k] = z_k sqrt(A) 2^(-g2 (k - n_ism) / 2).
//
// The noise z_k is Philox4x32-10 (counter (k/4, rir, 0, 0), key = seed)
// through a fixed sequence of correctly rounded FP32 operations, so any
// IEEE implementation of the same specification reproduces it bit for bit.
#include "ism_device.cuh"

namespace {

// One CTA per (RIR, chunk of fin_chunk image-source samples); chunk c holds
// samples [n_ism - (c + 1) fin_chunk, n_ism - c fin_chunk), so chunk 0 holds
// the envelope-fit window and also fits the amplitude.
__global__ void __launch_bounds__(256) finalize_kernel(const __grid_constant__ JobTable t,
                                                       const float* __restrict__ rows, float* __restrict__ amp,
                                                       const float* __restrict__ env)
{
    const long long g = blockIdx.x;
    const int jid = ism_find_job(t, g, [](const JobDev& j) { return j.fin_cta_base; });
    const JobDev& J = t.j[jid];
    const long long local = g - J.fin_cta_base;
    const int r = (int)(local / J.fin_chunks);
    const int c = (int)(local % J.fin_chunks);
    const int WIN = 32 * (J.slots + 1);
    float* out = J.out + (long long)r * J.n_S;
    const float* R = rows + J.rows_base + (long long)r * J.Q * WIN;
    const int k_end = J.n_ism - c * J.fin_chunk;
    const int k_beg = max(0, k_end - J.fin_chunk);

    // eq. (5): sample k is the sum of the window rows of the bins q with
    // 0 <= k - (32 q - H) < WIN, added in ascending q
    if ((J.H & 3) == 0) {
        // four samples from a multiple of 4 share their bins (top = k + H is then a multiple
        // of 4, and top .. top + 3 lie in one 32-sample block): one 16-byte load per row,
        // the same sums in the same order
        for (int k4 = (k_beg & ~3) + 4 * (int)threadIdx.x; k4 < k_end; k4 += 4 * (int)blockDim.x) {
            const int top = k4 + J.H;
            int q_hi = top / ISM_SB;
            if (q_hi > J.Q - 1) q_hi = J.Q - 1;
            int q_lo = top - WIN + 1 <= 0 ? 0 : (top - WIN + 1 + ISM_SB - 1) / ISM_SB;
            float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            for (int q = q_lo; q <= q_hi; ++q) {
                const float4 w = *reinterpret_cast<const float4*>(R + (long long)q * WIN + (top - ISM_SB * q));
                v.x += w.x;
                v.y += w.y;
                v.z += w.z;
                v.w += w.w;
            }
            if (J.vec4 && k4 >= k_beg && k4 + 3 < k_end) {
                *reinterpret_cast<float4*>(out + k4) = v;
            } else {   // the chunk's ragged ends
                if (k4 >= k_beg && k4 < k_end) out[k4] = v.x;
                if (k4 + 1 >= k_beg && k4 + 1 < k_end) out[k4 + 1] = v.y;
                if (k4 + 2 >= k_beg && k4 + 2 < k_end) out[k4 + 2] = v.z;
                if (k4 + 3 >= k_beg && k4 + 3 < k_end) out[k4 + 3] = v.w;
            }
        }
    } else {
        for (int k = k_beg + (int)threadIdx.x; k < k_end; k += blockDim.x) {
            const int top = k + J.H;                      // k - (32 q - H) = top - 32 q
            int q_hi = top / ISM_SB;
            if (q_hi > J.Q - 1) q_hi = J.Q - 1;
            int q_lo = top - WIN + 1 <= 0 ? 0 : (top - WIN + 1 + ISM_SB - 1) / ISM_SB;
            float v = 0.0f;
            for (int q = q_lo; q <= q_hi; ++q) v += R[(long long)q * WIN + (top - ISM_SB * q)];
            out[k] = v;
        }
    }
    if (c != 0) return;
    __syncthreads();
    __shared__ float red[256];
    float A = 0.0f;
    // Lehmann-Johansson envelope: env[k] = sqrt(E(t_k) / E(t0)) from the job's table
    // (all zero when E(t0) = 0: no tail)
    const float* envt = env + J.env_base - J.env_k0;
    const bool lj = J.envelope == ISM_ENVELOPE_LJ;
    if (J.has_tail && J.W_env > 0 && !(lj && envt[J.n_ism] == 0.0f)) {
        __shared__ ff g2_s;
        if (threadIdx.x == 0) g2_s = ism_job_g2(J);
        __syncthreads();
        const ff g2 = g2_s;
        const int k0 = J.n_ism - J.W_env;
        float acc = 0.0f;
        for (int k = k0 + (int)threadIdx.x; k < J.n_ism; k += blockDim.x) {
            float h = out[k];
            if (lj) {
                const float e = envt[k];
                acc += h * h / (e * e);   // E(t0) / E(t_k): the power brought forward to t0
            } else {
                acc += h * h * ism_exp2_neg(g2, J.n_ism - k);
            }
        }
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {  // fixed-order tree
            if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        A = red[0] / (float)J.W_env;
    }
    if (threadIdx.x == 0) {
        amp[J.rir_base + r] = A;
        if (J.env_amp) J.env_amp[r] = A;
    }
}

__global__ void __launch_bounds__(256) tail_kernel(const __grid_constant__ JobTable t, const float* __restrict__ amp,
                                                   const float* __restrict__ env)
{
    const long long g = blockIdx.x;
    const int jid = ism_find_job(t, g, [](const JobDev& j) { return j.tail_cta_base; });
    const JobDev& J = t.j[jid];
    if (!J.has_tail) return;
    const int blk0 = J.n_ism >> 2, blk_last = (J.n_S - 1) >> 2;
    const int per_rir = (blk_last - blk0 + 1 + ISM_TAIL_CHUNK / 4 - 1) / (ISM_TAIL_CHUNK / 4);
    const long long local = g - J.tail_cta_base;
    const int r = (int)(local / per_rir);
    const int c = (int)(local % per_rir);
    const float sqA = sqrtf(amp[J.rir_base + r]);
    // Sabine envelope of a block of 4 samples from its first one: e_(k+d) = e_k R_d,
    // R_d = 2^(-hg d) for d = 1 .. 3 (each within 2 ulp, the product rounded once more:
    // a few 1e-7 of the sample, see ism_exp2_neg)
    __shared__ ff g2_s;
    __shared__ float R_s[4];
    if (threadIdx.x == 0) g2_s = ism_job_g2(J);
    __syncthreads();
    const ff hg = {0.5f * g2_s.hi, 0.5f * g2_s.lo};   // amplitude: half the power's rate (exact)
    if (threadIdx.x < 4) R_s[threadIdx.x] = ism_exp2_neg(hg, (int)threadIdx.x);
    __syncthreads();
    const float R1 = R_s[1], R2 = R_s[2], R3 = R_s[3];
    const bool lj = J.envelope == ISM_ENVELOPE_LJ;
    const float* envt = env + J.env_base - J.env_k0;   // sqrt(E(t_k) / E(t0)), k >= env_k0
    float* out = J.out + (long long)r * J.n_S;
    for (int i = 0; i < ISM_TAIL_CHUNK / 4 / 256; ++i) {
        int blk = blk0 + c * (ISM_TAIL_CHUNK / 4) + i * 256 + (int)threadIdx.x;
        if (blk > blk_last) break;
        float4 z = ism_noise_block(J.seed, (uint32_t)(r + J.rir_index0), (uint32_t)blk);
        int k = 4 * blk;
        float e0, e1, e2, e3;
        if (lj) {   // (k < n_S; entries below n_ism are never stored)
            e0 = sqA * envt[max(k, J.n_ism)];
            e1 = sqA * envt[min(max(k + 1, J.n_ism), J.n_S - 1)];
            e2 = sqA * envt[min(max(k + 2, J.n_ism), J.n_S - 1)];
            e3 = sqA * envt[min(max(k + 3, J.n_ism), J.n_S - 1)];
        } else if (k >= J.n_ism) {
            const float b0 = ism_exp2_neg(hg, k - J.n_ism);
            e0 = sqA * b0;
            e1 = sqA * (b0 * R1);
            e2 = sqA * (b0 * R2);
            e3 = sqA * (b0 * R3);
        } else {   // the block holding sample n_ism (only its samples >= n_ism are written)
            e0 = sqA * ism_exp2_neg(hg, max(k - J.n_ism, 0));
            e1 = sqA * ism_exp2_neg(hg, max(k + 1 - J.n_ism, 0));
            e2 = sqA * ism_exp2_neg(hg, max(k + 2 - J.n_ism, 0));
            e3 = sqA * ism_exp2_neg(hg, max(k + 3 - J.n_ism, 0));
        }
        float4 v = make_float4(z.x * e0, z.y * e1, z.z * e2, z.w * e3);
        if (J.vec4 && k >= J.n_ism && k + 3 < J.n_S) {
            *reinterpret_cast<float4*>(out + k) = v;
        } else {
            if (k >= J.n_ism && k < J.n_S) out[k] = v.x;
            if (k + 1 >= J.n_ism && k + 1 < J.n_S) out[k + 1] = v.y;
            if (k + 2 >= J.n_ism && k + 2 < J.n_S) out[k + 2] = v.z;
            if (k + 3 >= J.n_ism && k + 3 < J.n_S) out[k + 3] = v.w;
        }
    }
}

// ---------------------------------------------------------------------------
// Envelope table of a Lehmann-Johansson tail (one per job): for k in [env_k0,
// n_S), env[k] = sqrt(E(t_k) / E(t0)), t = k / f_s, t0 = n_ism / f_s, with
//   E(t) = (2 / pi) int_0^(pi/2) int_0^(pi/2) 2^(-k g(theta, phi)) sin(theta) dtheta dphi,
//   g = sum_a |u_a| gamma_a,  gamma_a = -log2 |beta_a0 beta_a1| c / (f_s L_a)
// (the average over one octant of directions u; log2 of the energy lost per
// sample along u).  One CTA per job (envelope_nodes_kernel) builds the
// Gauss-Legendre product rule (nodes by Newton's iteration on the Legendre
// recurrence, FP64), the node rates g in float-float and the weights in FP32,
// and E(t0); then four threads of envelope_kernel share each sample: each sums
// a quarter of its n^2 terms 2^(-k g) with Kahan's compensated FP32 summation
// (all terms positive: relative error ~2 ulp plus exp2f's 2 ulp), and the four
// partial sums are added in FP64 in a fixed order (E(t0) likewise).  n =
// clamp(ceil(K / 4) + 12, 16, 64) nodes per angle, K = (n_S / f_s) c
// |(-ln rho_a / L_a)_a|, the largest exponent (in nepers) over the table.  A
// job's node slot holds ISM_ENV_SLOT float4 {g hi, g lo, w, 0}, the last one
// {n (int bits), 0, E(t0) as the two halves of an FP64}.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) envelope_nodes_kernel(const __grid_constant__ JobTable t,
                                                             float4* __restrict__ nodes)
{
    const JobDev& J = t.j[blockIdx.x];
    if (!J.has_tail || J.envelope != ISM_ENVELOPE_LJ) return;   // CTA-uniform
    float4* slot = nodes + (long long)J.env_slot * ISM_ENV_SLOT;
    __shared__ double wg[ISM_ENV_MAX_NODES];
    __shared__ double sth[ISM_ENV_MAX_NODES], cth[ISM_ENV_MAX_NODES];
    __shared__ double gam[3];
    __shared__ int n_s;
    __shared__ double part[256];
    __shared__ double inv_m[ISM_ENV_MAX_NODES + 1];   // 1 / m for the Legendre recurrence
    const double PI = 3.141592653589793238462643383279502884;
    if (threadIdx.x == 0) {
        double kn = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double rho = fabs((double)ism_job_beta(J, 2 * a) * (double)ism_job_beta(J, 2 * a + 1));
            const double nep = rho > 0.0 ? -log(rho) : 1.0e30;                 // nepers per reflection pair
            gam[a] = rho > 0.0 ? nep / log(2.0) * (double)J.c / ((double)J.fs * J.L[a]) : 1.0e30;
            const double ka = nep * (double)J.c * ((double)J.n_S / (double)J.fs) / J.L[a];
            kn += ka * ka;
        }
        kn = sqrt(kn);
        n_s = kn < 4.0 * (ISM_ENV_MAX_NODES - 12) ? max(16, (int)ceil(kn / 4.0) + 12) : ISM_ENV_MAX_NODES;
    }
    if ((int)threadIdx.x <= ISM_ENV_MAX_NODES) inv_m[threadIdx.x] = threadIdx.x ? 1.0 / (double)threadIdx.x : 0.0;
    __syncthreads();
    const int n = n_s;
    // Gauss-Legendre nodes and weights on [-1, 1]: Newton on P_n from the asymptotic guess
    if ((int)threadIdx.x < n) {
        const int i = threadIdx.x;
        // Newton from a guess within ~1e-3 of the root: three steps in FP32 (to ~1e-7), then
        // two in FP64 (each doubles the correct digits); the weight takes the derivative of
        // the last step (its point differs from the root by ~1e-16)
        float xf = cospif((i + 0.75f) / (n + 0.5f));
        for (int it = 0; it < 3; ++it) {
            float p0 = 1.0f, p1 = xf;
            for (int m = 2; m <= n; ++m) {
                const float p2 = ((2.0f * m - 1.0f) * xf * p1 - (m - 1.0f) * p0) * (float)inv_m[m];
                p0 = p1;
                p1 = p2;
            }
            const float dpf = n * (xf * p1 - p0) / (xf * xf - 1.0f);
            xf -= p1 / dpf;
        }
        double x = (double)xf;
        double dp = 1.0;
        for (int it = 0; it < 2; ++it) {
            double p0 = 1.0, p1 = x;
            for (int m = 2; m <= n; ++m) {
                const double p2 = ((2.0 * m - 1.0) * x * p1 - (m - 1.0) * p0) * inv_m[m];
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            x -= p1 / dp;
        }
        wg[i] = 2.0 / ((1.0 - x * x) * dp * dp);
        const double ang = (x + 1.0) * (PI / 4.0);   // [-1, 1] -> [0, pi/2]
        sth[i] = sin(ang);
        cth[i] = cos(ang);
    }
    __syncthreads();
    // nodes (theta_i, phi_j): u = (sin t cos p, sin t sin p, cos t), weight (pi/4)^2 w_i w_j sin t (2 / pi);
    // E(t0) by the CTA's threads over the nodes, then a fixed-order tree
    const int nn = n * n;
    float s = 0.0f, comp = 0.0f;
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
        const int i = e / n, j = e - (e / n) * n;
        const double gr = sth[i] * cth[j] * gam[0] + sth[i] * sth[j] * gam[1] + cth[i] * gam[2];
        const float hi = (float)gr;
        const float lo = gr < 1.0e29 ? (float)(gr - (double)hi) : 0.0f;
        const float w = (float)(wg[i] * wg[j] * sth[i] * (PI / 8.0));
        slot[e] = make_float4(hi, lo, w, 0.0f);
        const float y = __fsub_rn(__fmul_rn(w, ism_exp2_neg(ff{hi, lo}, J.n_ism)), comp);
        const float tt = __fadd_rn(s, y);
        comp = __fsub_rn(__fsub_rn(tt, s), y);
        s = tt;
    }
    part[threadIdx.x] = (double)s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {   // the partial sums in FP64, a fixed-order tree
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double E0 = part[0];
        const unsigned long long b = (unsigned long long)__double_as_longlong(E0);
        slot[ISM_ENV_SLOT - 1] = make_float4(__int_as_float(n), 0.0f, __uint_as_float((unsigned)b),
                                             __uint_as_float((unsigned)(b >> 32)));
    }
}

__global__ void __launch_bounds__(4 * ISM_ENV_CHUNK) envelope_kernel(const __grid_constant__ JobTable t,
                                                                 const float4* __restrict__ nodes,
                                                                 float* __restrict__ env)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const long long g = blockIdx.x;
    const int jid = ism_find_job(t, g, [](const JobDev& j) { return (long long)j.env_cta_base; });
    const JobDev& J = t.j[jid];
    const int chunk = (int)(g - J.env_cta_base);
    const float4* slot = nodes + (long long)J.env_slot * ISM_ENV_SLOT;
    float4* nd = reinterpret_cast<float4*>(smem);   // [n * n] {g hi, g lo, w, 0}
    __shared__ float part[4][ISM_ENV_CHUNK];
    const float4 head = slot[ISM_ENV_SLOT - 1];
    const int n = __float_as_int(head.x);
    const double E0 = __longlong_as_double((long long)(((unsigned long long)__float_as_uint(head.w) << 32) |
                                                       __float_as_uint(head.z)));
    const int nn = n * n;
    for (int e = threadIdx.x; e < nn; e += blockDim.x) nd[e] = slot[e];
    __syncthreads();
    // sample ks of the chunk, quarter qp of the nodes (i = qp, qp + 4, ...)
    const int ks = (int)threadIdx.x % ISM_ENV_CHUNK, qp = (int)threadIdx.x / ISM_ENV_CHUNK;
    const int k = J.env_k0 + chunk * ISM_ENV_CHUNK + ks;
    float s = 0.0f, comp = 0.0f;
    if (k < J.n_S && E0 > 0.0) {
        for (int i = qp; i < nn; i += 4) {
            const float4 q = nd[i];
            const float y = __fsub_rn(__fmul_rn(q.z, ism_exp2_neg(ff{q.x, q.y}, k)), comp);
            const float tt = __fadd_rn(s, y);
            comp = __fsub_rn(__fsub_rn(tt, s), y);
            s = tt;
        }
    }
    part[qp][ks] = s;
    __syncthreads();
    if (qp != 0 || k >= J.n_S) return;
    float v = 0.0f;
    if (E0 > 0.0) {
        const double E = (((double)part[0][ks] + part[1][ks]) + part[2][ks]) + part[3][ks];
        v = (float)sqrt(E / E0);
    }
    env[J.env_base + (k - J.env_k0)] = v;
}

__global__ void noise_kernel(uint64_t seed, uint32_t rir, uint32_t k0, int n, float* z)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t k = k0 + (uint32_t)i;
    float4 b = ism_noise_block(seed, rir, k >> 2);
    float v = (k & 3u) == 0 ? b.x : ((k & 3u) == 1 ? b.y : ((k & 3u) == 2 ? b.z : b.w));
    z[i] = v;
}

}  // namespace

int ism_launch_finalize(const JobTable& t, const WsPlan& p, char* ws, void* stream)
{
    if (p.fin_ctas <= 0) return 0;
    finalize_kernel<<<(unsigned)p.fin_ctas, 256, 0, (cudaStream_t)stream>>>(
        t, reinterpret_cast<const float*>(ws + p.rows_off), reinterpret_cast<float*>(ws + p.amp_off),
        reinterpret_cast<const float*>(ws + p.env_off));
    return (int)cudaGetLastError();
}

int ism_launch_tail(const JobTable& t, const WsPlan& p, char* ws, void* stream)
{
    if (p.tail_ctas <= 0) return 0;
    tail_kernel<<<(unsigned)p.tail_ctas, 256, 0, (cudaStream_t)stream>>>(
        t, reinterpret_cast<const float*>(ws + p.amp_off), reinterpret_cast<const float*>(ws + p.env_off));
    return (int)cudaGetLastError();
}

int ism_launch_envelope(const JobTable& t, const WsPlan& p, char* ws, void* stream)
{
    if (p.env_ctas <= 0) return 0;
    float4* nodes = reinterpret_cast<float4*>(ws + p.env_nodes_off);
    envelope_nodes_kernel<<<(unsigned)t.n_jobs, 256, 0, (cudaStream_t)stream>>>(t, nodes);
    int rc = (int)cudaGetLastError();
    if (rc) return rc;
    const size_t sm = (size_t)ISM_ENV_MAX_NODES * ISM_ENV_MAX_NODES * sizeof(float4);
    static std::atomic<unsigned long long> opened{0};
    if ((rc = ism_open_smem((const void*)envelope_kernel, &opened))) return rc;
    envelope_kernel<<<(unsigned)p.env_ctas, 4 * ISM_ENV_CHUNK, sm, (cudaStream_t)stream>>>(
        t, nodes, reinterpret_cast<float*>(ws + p.env_off));
    return (int)cudaGetLastError();
}

int ism_launch_noise(uint64_t seed, uint32_t rir, uint32_t k0, int n, float* z, void* stream)
{
    if (n <= 0) return 0;
    noise_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(seed, rir, k0, n, z);
    return (int)cudaGetLastError();
}
