// ism_accum_lut.cu -- accumulation kernel with the windowed sinc taken from a
// table (eq. (9)) and the table itself.
//
// The table of a job holds delta'(x) of eq. (6), the Hann-windowed sinc,
// at x = j - p / Q for the Q + 1 fractional delays p / Q, p = 0 .. Q, and
// the 32 SLOTS taps j = t - H + 1 of a lane-per-tap window (row p, column
// t).  It is evaluated in FP64 and stored in FP32; outside |x| < N_w / 2 the
// entry is 0, so a window of non-integral length needs no mask.
#include "ism_accum.cuh"

namespace {

__global__ void __launch_bounds__(256) lut_kernel(const __grid_constant__ JobTable t, float* __restrict__ lut)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int jid = ism_find_job(t, e, [](const JobDev& j) { return j.lut_base; });
    const JobDev& J = t.j[jid];
    const int Q = ism_lut_phases(J.slots);
    const int row = 32 * J.slots;
    const long long local = e - J.lut_base;
    if (local < 0 || local >= (long long)(Q + 1) * row) return;
    const int p = (int)(local / row), tt = (int)(local % row);
    const int j = tt - J.H + 1;
    const double x = (double)j - (double)p / (double)Q;
    const double Nw = (double)J.Nw;
    double v = 0.0;
    if (fabs(x) < 0.5 * Nw) {
        const double win = 0.5 * (1.0 + cospi(2.0 * x / Nw));
        const double sinc = x == 0.0 ? 1.0 : sinpi(x) / (3.141592653589793238462643383279502884 * x);
        v = win * sinc;
    }
    lut[e] = (float)v;
}

}  // namespace

int ism_launch_lut_tables(const JobTable& t, const WsPlan& p, char* ws, void* stream)
{
    if (p.lut_total <= 0) return 0;
    const unsigned blocks = (unsigned)((p.lut_total + 255) / 256);
    lut_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(t, reinterpret_cast<float*>(ws + p.lut_off));
    return (int)cudaGetLastError();
}

int ism_launch_accum_lut(const JobTable& t, const WsPlan& p, char* ws, void* stream, int* launched)
{
    return launch_accum_prec<PREC_LUT>(t, p, ws, stream, launched);
}
