// ism_geometry.cu -- per-RIR geometry tables and the FP64 Sabine helper.
//
// The image grid of Section 2.1 factorises per axis: the image of index n sits
// at n L + x_s (n even) or (n + 1) L - x_s (n odd) (eq. (1)), so its offset to
// the receiver along one axis depends on n alone, and the reflection product
// of eq. (4) is a product of one factor per axis.  This kernel tabulates, for
// every RIR and every index of every axis,
//   S[n] = ((x_n - x_r) f_s / c)^2   (squared offset in samples^2, FP64, stored
//                                     as a float-float pair hi + lo)
//   F[n] = beta_0^{e0(n)} beta_1^{e1(n)}  (wall hits along that axis)
//   D[n] = (x_n - x_r) f_s / c           (signed offset, FP32: the direction
//                                          of arrival for polar patterns)
// so that image (nx, ny, nz) has s^2 = Sx + Sy + Sz and weight Fx Fy Fz.  For
// the backward pass it also tabulates x_n - x_r (metres), dF/dbeta_0,
// dF/dbeta_1 (product form, valid at beta = 0) and d x_n / d x_s = +-1
// (even / odd n).  It
// also checks that source and receiver lie strictly inside the room (and that
// a patterned receiver has a non-zero orientation); a pair that does not gets
// S = +inf everywhere, i.e. no image survives.
#include <cmath>

#include "ism_device.cuh"

namespace {

__device__ double dpow_int(double b, int e)
{
    double r = 1.0;  // 0^0 = 1: the direct path keeps weight 1
    while (e > 0) {
        if (e & 1) r *= b;
        b *= b;
        e >>= 1;
    }
    return r;
}

__global__ void __launch_bounds__(128) geometry_kernel(const __grid_constant__ JobTable t, float4* tbl,
                                                       float4* dtbl, uint32_t* status)
{
    const long long g = blockIdx.x;  // one CTA per RIR of the launch set
    const int jid = ism_find_job(t, g, [](const JobDev& j) { return j.rir_base; });
    const JobDev& J = t.j[jid];
    const int r = (int)(g - J.rir_base);
    const int i_src = r / J.n_rcv, i_rcv = r % J.n_rcv;
    const float* ps = J.pos_src + 3 * i_src;
    const float* pr = J.pos_rcv + 3 * i_rcv;

    __shared__ int ok_s;
    __shared__ double ps_s[3], pr_s[3], beta_s[6];
    if (threadIdx.x == 0) {
        int ok = 1, ok_beta = 1;
        for (int w = 0; w < 6; ++w) {
            const float b = ism_job_beta(J, w);   // checked on the host unless it lives on the device
            beta_s[w] = (double)b;
            if (J.beta_dev && !(fabsf(b) <= 1.0f)) ok_beta = 0;
        }
        if (!ok_beta) atomicOr(status, (uint32_t)ISM_DEVICE_FLAG_BETA);
        double d2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            double xs = ps[a], xr = pr[a];
            ps_s[a] = xs;
            pr_s[a] = xr;
            if (!(xs > 0.0 && xs < J.L[a] && xr > 0.0 && xr < J.L[a])) ok = 0;
            d2 += (xs - xr) * (xs - xr);
        }
        if (!(d2 > 0.0)) ok = 0;
        if (J.mic_alpha != 1.0f) {
            const float* o = J.orient_rcv + 3 * i_rcv;
            const double oo = (double)o[0] * o[0] + (double)o[1] * o[1] + (double)o[2] * o[2];
            if (!(oo > 0.0) || !(oo < 1e300)) ok = 0;
        }
        ok_s = ok && ok_beta;
        if (!ok) atomicOr(status, (uint32_t)ISM_DEVICE_FLAG_POSITION);
    }
    __syncthreads();

    const int n_axis = J.N[0] + J.N[1] + J.N[2];
    const double k = (double)J.fs / (double)J.c;
    float4* out = tbl + J.tbl_base + (long long)r * n_axis;
    for (int e = threadIdx.x; e < n_axis; e += blockDim.x) {
        int a = (e < J.N[0]) ? 0 : ((e < J.N[0] + J.N[1]) ? 1 : 2);
        int i = e - (a == 0 ? 0 : (a == 1 ? J.N[0] : J.N[0] + J.N[1]));
        int n = J.nlo[a] + i;
        bool even = (n % 2) == 0;
        // eq. (1): image coordinate minus receiver coordinate
        double m = even ? (double)n : (double)(n + 1);
        double off = even ? (ps_s[a] - pr_s[a]) : (-ps_s[a] - pr_s[a]);
        double u = (m * J.L[a] + off) * k;
        double S = u * u;
        // eq. (4): hits of the near (x0) and far (x1) wall along this axis
        int an = n < 0 ? -n : n;
        int e0 = even ? an / 2 : (n - 1 < 0 ? 1 - n : n - 1) / 2;
        int e1 = even ? an / 2 : (n + 1 < 0 ? -(n + 1) : n + 1) / 2;
        const double b0 = beta_s[2 * a], b1 = beta_s[2 * a + 1];
        double F = dpow_int(b0, e0) * dpow_int(b1, e1);
        float hi = (float)S;
        float lo = (float)(S - (double)hi);
        if (!ok_s) {
            hi = __int_as_float(0x7f800000);  // +inf: every image of this pair is culled
            lo = 0.0f;
            F = 0.0;
        }
        out[e] = make_float4(hi, lo, (float)F, (float)u);
        if (dtbl) {
            const double d0 = e0 > 0 ? (double)e0 * dpow_int(b0, e0 - 1) * dpow_int(b1, e1) : 0.0;
            const double d1 = e1 > 0 ? (double)e1 * dpow_int(b0, e0) * dpow_int(b1, e1 - 1) : 0.0;
            dtbl[J.tbl_base + (long long)r * n_axis + e] = make_float4(
                (float)(m * J.L[a] + off), ok_s ? (float)d0 : 0.0f, ok_s ? (float)d1 : 0.0f, even ? 1.0f : -1.0f);
        }
    }
}

// Inverse of eq. (7) in FP64: alpha_i = w_i alpha_0, sum_i S_i alpha_i =
// 0.161 V / T60, beta_i = +-sqrt(1 - alpha_i).
__global__ void beta_sabine_kernel(const double* L, const double* T60, const double* w, int negative,
                                   int n, double* beta_out, int* status)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double Lx = L[3 * i], Ly = L[3 * i + 1], Lz = L[3 * i + 2];
    double S[6] = {Ly * Lz, Ly * Lz, Lx * Lz, Lx * Lz, Lx * Ly, Lx * Ly};
    double wt[6];
    double sw = 0.0;
    for (int k = 0; k < 6; ++k) {
        wt[k] = w ? w[k] : 1.0;
        sw += S[k] * wt[k];
    }
    int st = 0;
    double a0 = 0.0;
    if (!(sw > 0.0) || !(T60[i] > 0.0) || !(Lx > 0.0 && Ly > 0.0 && Lz > 0.0)) st = ISM_ERR_INFEASIBLE;
    else a0 = 0.161 * Lx * Ly * Lz / (T60[i] * sw);
    for (int k = 0; k < 6 && st == 0; ++k) {
        double a = wt[k] * a0;
        if (a >= 1.0 || a < 0.0) st = ISM_ERR_INFEASIBLE;
    }
    for (int k = 0; k < 6; ++k) {
        double b = st ? 0.0 : sqrt(1.0 - wt[k] * a0);
        beta_out[6 * i + k] = negative ? -b : b;
    }
    status[i] = st;
}

}  // namespace

int ism_launch_geometry(const JobTable& t, const WsPlan& p, char* ws, void* stream)
{
    long long n_rir = p.rir_total;
    if (n_rir <= 0) return 0;
    geometry_kernel<<<(unsigned)n_rir, 128, 0, (cudaStream_t)stream>>>(
        t, reinterpret_cast<float4*>(ws + p.tbl_off), p.dtbl_off ? reinterpret_cast<float4*>(ws + p.dtbl_off) : nullptr,
        reinterpret_cast<uint32_t*>(ws + p.status_off));
    return (int)cudaGetLastError();
}

int ism_launch_beta_sabine(const double* L, const double* T60, const double* w, int negative, int n,
                           double* beta_out, int* status, void* stream)
{
    if (n <= 0) return 0;
    beta_sabine_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(L, T60, w, negative, n, beta_out,
                                                                          status);
    return (int)cudaGetLastError();
}
