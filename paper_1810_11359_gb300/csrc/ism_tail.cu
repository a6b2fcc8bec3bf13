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
                                                       const float* __restrict__ rows, float* __restrict__ amp)
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
    for (int k = k_beg + (int)threadIdx.x; k < k_end; k += blockDim.x) {
        const int top = k + J.H;                      // k - (32 q - H) = top - 32 q
        int q_hi = top / ISM_SB;
        if (q_hi > J.Q - 1) q_hi = J.Q - 1;
        int q_lo = top - WIN + 1 <= 0 ? 0 : (top - WIN + 1 + ISM_SB - 1) / ISM_SB;
        float v = 0.0f;
        for (int q = q_lo; q <= q_hi; ++q) v += R[(long long)q * WIN + (top - ISM_SB * q)];
        out[k] = v;
    }
    if (c != 0) return;
    __syncthreads();
    __shared__ float red[256];
    float A = 0.0f;
    if (J.has_tail && J.W_env > 0) {
        __shared__ float g2_s;
        if (threadIdx.x == 0) g2_s = ism_job_g2(J);
        __syncthreads();
        const float g2 = g2_s;
        const int k0 = J.n_ism - J.W_env;
        float acc = 0.0f;
        for (int k = k0 + (int)threadIdx.x; k < J.n_ism; k += blockDim.x) {
            float h = out[k];
            acc += h * h * exp2f(-g2 * (float)(J.n_ism - k));
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

__global__ void __launch_bounds__(256) tail_kernel(const __grid_constant__ JobTable t, const float* __restrict__ amp)
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
    __shared__ float g2_s;
    if (threadIdx.x == 0) g2_s = ism_job_g2(J);
    __syncthreads();
    const float hg = 0.5f * g2_s;
    float* out = J.out + (long long)r * J.n_S;
    for (int i = 0; i < ISM_TAIL_CHUNK / 4 / 256; ++i) {
        int blk = blk0 + c * (ISM_TAIL_CHUNK / 4) + i * 256 + (int)threadIdx.x;
        if (blk > blk_last) break;
        float4 z = ism_noise_block(J.seed, (uint32_t)(r + J.rir_index0), (uint32_t)blk);
        int k = 4 * blk;
        float e0 = sqA * exp2f(-hg * (float)(k - J.n_ism));
        float e1 = sqA * exp2f(-hg * (float)(k + 1 - J.n_ism));
        float e2 = sqA * exp2f(-hg * (float)(k + 2 - J.n_ism));
        float e3 = sqA * exp2f(-hg * (float)(k + 3 - J.n_ism));
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
        t, reinterpret_cast<const float*>(ws + p.rows_off), reinterpret_cast<float*>(ws + p.amp_off));
    return (int)cudaGetLastError();
}

int ism_launch_tail(const JobTable& t, const WsPlan& p, char* ws, void* stream)
{
    if (p.tail_ctas <= 0) return 0;
    tail_kernel<<<(unsigned)p.tail_ctas, 256, 0, (cudaStream_t)stream>>>(t,
                                                                         reinterpret_cast<const float*>(ws + p.amp_off));
    return (int)cudaGetLastError();
}

int ism_launch_noise(uint64_t seed, uint32_t rir, uint32_t k0, int n, float* z, void* stream)
{
    if (n <= 0) return 0;
    noise_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(seed, rir, k0, n, z);
    return (int)cudaGetLastError();
}
