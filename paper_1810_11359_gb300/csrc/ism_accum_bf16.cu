// ism_accum_bf16.cu -- accumulation kernel with the window and the sinc in
// packed BF16 (two images per instruction), FP32 accumulation.
#include "ism_accum.cuh"

int ism_launch_accum_bf16(const JobTable& t, const WsPlan& p, char* ws, void* stream, int* launched)
{
    return launch_accum_prec<PREC_BF16>(t, p, ws, stream, launched);
}
