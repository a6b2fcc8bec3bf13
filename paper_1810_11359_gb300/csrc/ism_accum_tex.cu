// ism_accum_tex.cu -- accumulation kernel with the windowed sinc of the
// table of eq. (9) read through the texture unit (hardware linear filtering
// between the two nearest fractional-delay phases), the paper's own LUT path
// (Section 3.5).  The table is built by lut_kernel (ism_accum_lut.cu).
#include "ism_accum.cuh"

int ism_launch_accum_tex(const JobTable& t, const WsPlan& p, char* ws, void* stream, int* launched)
{
    return launch_accum_prec<PREC_TEX>(t, p, ws, stream, launched);
}
