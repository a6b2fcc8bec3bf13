// ism_accum.cu -- FP32 instantiation of the accumulation kernel (kernel c,
// eq. (5)-(6)) and the dispatch over the tap arithmetic.
#include "ism_accum.cuh"

int ism_launch_accum(const JobTable& t, const WsPlan& p, char* ws, ism_precision prec, void* stream,
                     int* launched)
{
    // the fused kernels (32-tap windows: Chebyshev moments or every tap evaluated), then
    // the per-tap kernel over binned ids for the other windows
    int a = 0, b = 0, c = 0;
    int rc = ism_launch_accum_cheb(t, p, ws, stream, &a);
    if (!rc) rc = ism_launch_accum_shell_direct(t, p, ws, prec, stream, &b);
    if (!rc) {
        switch (prec) {
        case ISM_PREC_FP32:
        case ISM_PREC_FP32_DIRECT: rc = launch_accum_prec<PREC_FP32>(t, p, ws, stream, &c); break;
        case ISM_PREC_FP16X2: rc = ism_launch_accum_fp16(t, p, ws, stream, &c); break;
        case ISM_PREC_BF16X2: rc = ism_launch_accum_bf16(t, p, ws, stream, &c); break;
        case ISM_PREC_LUT: rc = ism_launch_accum_lut(t, p, ws, stream, &c); break;
        case ISM_PREC_LUT_TEX: rc = ism_launch_accum_tex(t, p, ws, stream, &c); break;
        default: rc = (int)cudaErrorInvalidValue;
        }
    }
    *launched = a + b + c;
    return rc;
}
