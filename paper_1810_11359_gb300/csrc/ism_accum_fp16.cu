// ism_accum_fp16.cu -- accumulation kernel with the window and the sinc in
// packed FP16 (two images per instruction), FP32 accumulation (Section 3.3).
#include "ism_accum.cuh"

int ism_launch_accum_fp16(const JobTable& t, const WsPlan& p, char* ws, void* stream, int* launched)
{
    return launch_accum_prec<PREC_FP16>(t, p, ws, stream, launched);
}
