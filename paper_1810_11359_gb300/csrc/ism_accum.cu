// ism_accum.cu -- FP32 instantiation of the accumulation kernel (kernel c,
// eq. (5)-(6)) and the dispatch over the tap arithmetic.
#include "ism_accum.cuh"

int ism_launch_accum(const JobTable& t, const WsPlan& p, char* ws, ism_precision prec, void* stream,
                     int* launched)
{
    switch (prec) {
    case ISM_PREC_FP32:
    case ISM_PREC_FP32_DIRECT: {
        int a = 0, b = 0, c = 0;
        int rc = ism_launch_accum_cheb(t, p, ws, stream, &a);
        if (!rc) rc = ism_launch_accum_shell_direct(t, p, ws, stream, &b);
        if (!rc) rc = launch_accum_prec<PREC_FP32>(t, p, ws, stream, &c);
        *launched = a + b + c;
        return rc;
    }
    case ISM_PREC_FP16X2: return ism_launch_accum_fp16(t, p, ws, stream, launched);
    case ISM_PREC_BF16X2: return ism_launch_accum_bf16(t, p, ws, stream, launched);
    case ISM_PREC_LUT: return ism_launch_accum_lut(t, p, ws, stream, launched);
    case ISM_PREC_LUT_TEX: return ism_launch_accum_tex(t, p, ws, stream, launched);
    }
    *launched = 0;
    return (int)cudaErrorInvalidValue;
}
