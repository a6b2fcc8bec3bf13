// ism_auralize_fft.cu -- moving sources (Section 4) through the frequency
// domain, the way the paper filters the source signal (batched FFTs, overlap-
// add), with FFTs written here (no FFT library on the path).
//
// The output of microphone m is a sum of linear convolutions,
//   y_m = sum_p x_p * h_{p,m},   x_p = x on [a_p, a_(p+1)), zero elsewhere,
// so with one DFT length N >= n_x + n_S - 1 (a power of two, no wrap-around)
//   Y_m[k] = sum_p X_p[k] H_{p,m}[k],   y_m = IDFT(Y_m).
// Two microphones share one complex sequence: z = h_{p,m} + i h_{p,m'} has the
// spectrum Z = H_m + i H_m', and since X_p is the spectrum of a real signal,
// sum_p X_p Z_p = Y_m + i Y_m' is the spectrum of y_m + i y_m' (both real): one
// inverse DFT per pair gives both outputs, its real and imaginary parts, with
// no unpacking.  The segments' positions ride in X_p (x_p is placed at its
// samples), so the overlap-add is the sum over p, taken in the frequency
// domain in ascending p: a fixed order, so results are identical run to run.
//
// Each length-N DFT is split four-step, N = R C, n = n1 + C n2, k = k2 + R k1:
//   Z[k2 + R k1] = sum_n1 W_C^(n1 k1) W_N^(n1 k2) sum_n2 z[n1 + C n2] W_R^(n2 k2).
//   column pass (one CTA per block of n1 columns): length-R DFTs over n2, the
//     twiddle W_N^(n1 k2), stored as A[k2][n1];
//   row pass (one CTA per block of k2 rows): length-C DFTs of the rows of A
//     for the segment and for every microphone pair, the products summed over
//     the points of the chunk; after the last chunk the inverse row DFTs and
//     the twiddle W_N^(-n1 k2) (stored as B[k2][n1]);
//   inverse column pass: length-R inverse DFTs over k2, y = result / N.
// The short DFTs run in shared memory as Stockham radix-4 stages (one radix-2
// stage first when the length is an odd power of two) in FP32, every stage
// reading its inputs into registers and writing its outputs after a barrier;
// twiddles come from sincospif of exact arguments (2 t / L), so they are
// correctly rounded to ~1 ulp.  The points are processed in chunks whose
// column-pass output fits the workspace (the row pass adds each chunk into
// the accumulated spectra Y, kept in the workspace between chunks).
#include "ism_device.cuh"

namespace {

#define AF_T 256        // threads of the column passes
#define AF_T2 256       // threads of the row pass
#define AF_COL_E 8192   // complex values per CTA of the column passes (64 KB)
#define AF_MAXPG 4      // microphone pairs per row-pass CTA (at most)
#define AF_ROW_E 2048   // complex values transformed at once by a row-pass CTA (4 radix-4 items per thread)
#define AF_MAXGRP 8     // point groups of the row pass

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(__fmaf_rn(a.x, b.x, -a.y * b.y), __fmaf_rn(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// exp(sign 2 pi i t / L) for 0 <= t < L (L a power of two): the argument 2 t / L is exact.
__device__ __forceinline__ float2 af_root(int t, int logL, float sign)
{
    float s, c;
    sincospif(sign * __int2float_rn(2 * t) * __int_as_float((127 - logL) << 23), &s, &c);
    return make_float2(c, s);
}

// Segment boundary a_p of point p (uniform cut when starts is NULL); a_P = n_x.
__device__ __forceinline__ int af_start(int p, int n_x, int P, const int* starts)
{
    if (p >= P) return n_x;
    if (!starts) return (int)(((long long)p * n_x) / P);
    return min(max(starts[p], 0), n_x);
}

// Twiddle table in shared memory: tw[t] = exp(sign 2 pi i t / L), t < n (n = L by default).
__device__ __forceinline__ void af_table(float2* tw, int logL, float sign, int n = -1)
{
    if (n < 0) n = 1 << logL;
    for (int t = threadIdx.x; t < n; t += blockDim.x) tw[t] = af_root(t, logL, sign);
}

// Radix-r DFT in registers (r = 2, 4, 8): forward when sign < 0.
__device__ __forceinline__ float2 af_mul_i(float2 d, float sign)   // (sign i) d
{
    return sign < 0.0f ? make_float2(d.y, -d.x) : make_float2(-d.y, d.x);
}

template <int RADIX>
__device__ __forceinline__ void af_dft(float2 (&v)[RADIX], float sign)
{
    if constexpr (RADIX == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (RADIX == 4) {
        const float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]), a2 = cadd(v[1], v[3]);
        const float2 a3 = af_mul_i(csub(v[1], v[3]), sign);
        v[0] = cadd(a0, a2);
        v[1] = cadd(a1, a3);
        v[2] = csub(a0, a2);
        v[3] = csub(a1, a3);
    } else {
        // decimation in frequency: a_n = x_n + x_(n+4), b_n = (x_n - x_(n+4)) W8^n, then two
        // 4-point DFTs giving the even and the odd outputs
        const float h = 0.70710678118654752440f;   // 1 / sqrt(2)
        float2 a[4], b[4];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            a[n] = cadd(v[n], v[n + 4]);
            b[n] = csub(v[n], v[n + 4]);
        }
        // W8^1 = (1 + sign i) / sqrt 2, W8^2 = sign i, W8^3 = (-1 + sign i) / sqrt 2
        b[1] = make_float2(h * (b[1].x - sign * b[1].y), h * (b[1].y + sign * b[1].x));
        b[2] = af_mul_i(b[2], sign);
        b[3] = make_float2(h * (-b[3].x - sign * b[3].y), h * (-b[3].y + sign * b[3].x));
        af_dft<4>(a, sign);
        af_dft<4>(b, sign);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[2 * k] = a[k];
            v[2 * k + 1] = b[k];
        }
    }
}

// One Stockham stage of radix RADIX on `ncol` sequences of length L = 2^logL
// in shared memory, with Ns = 2^logNs: item j of a sequence reads
// x_q = in[j + q L / RADIX] W_(RADIX Ns)^(q k), k = j mod Ns, transforms them and
// writes out[expand(j) + q Ns], expand(j) = (j div Ns) RADIX Ns + k.  All the
// reads of the stage go to registers before a barrier, then the writes, so the
// stage runs in place.  Element i of sequence c sits at buf[i ncol + c] when
// COLS (work items take consecutive sequences: conflict-free) and at
// buf[c Lp + i + i / 8], Lp = 9 L / 8, otherwise (rows, one padding element every
// 8 so that the scattered writes of the first stages spread over the banks).
// NV bounds the values a thread holds (items per thread x RADIX).
template <bool COLS, int RADIX, int NV>
__device__ __forceinline__ void af_stage(float2* buf, const float2* tw, int logL, int ncol, int logc, int logNs,
                                         float sign)
{
    constexpr int IPT = NV / RADIX;
    constexpr int LR = RADIX == 2 ? 1 : (RADIX == 4 ? 2 : 3);
    const int L = 1 << logL;
    const int T = blockDim.x;
    const int logm = logL - LR;            // items per sequence: 2^logm
    const int m = 1 << logm;
    const int Ns = 1 << logNs;
    const int tstep = L >> (logNs + LR);   // W_(RADIX Ns)^(q k) = W_L^(q k tstep)
    const int nitems = ncol << logm;
    const int Lp = L + (L >> 3);
    auto addr = [&](int i, int c) { return COLS ? (i << logc) + c : c * Lp + i + (i >> 3); };
    float2 v[IPT][RADIX];
    int jj[IPT], cc[IPT];
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
        const int w = (int)threadIdx.x + it * T;
        jj[it] = -1;
        if (w < nitems) {
            const int c = COLS ? (w & (ncol - 1)) : (w >> logm);
            const int j = COLS ? (w >> logc) : (w & (m - 1));
            const int k = j & (Ns - 1);
#pragma unroll
            for (int q = 0; q < RADIX; ++q) {
                float2 x = buf[addr(j + q * m, c)];
                if (q > 0 && k) x = cmul(x, tw[q * k * tstep]);
                v[it][q] = x;
            }
            af_dft<RADIX>(v[it], sign);
            jj[it] = j;
            cc[it] = c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
        if (jj[it] < 0) continue;
        const int j = jj[it];
        const int base = ((j >> logNs) << (logNs + LR)) + (j & (Ns - 1));
#pragma unroll
        for (int q = 0; q < RADIX; ++q) buf[addr(base + q * Ns, cc[it])] = v[it][q];
    }
    __syncthreads();
}

// In-place DFTs (forward when sign = -1, unscaled inverse when +1) of `ncol`
// sequences of length 2^logL in the layout of af_stage: radix-8 stages, then
// one radix-4 or radix-2 stage for the rest.  tw[t] = exp(sign 2 pi i t / L).
// For COLS, ncol = 2^logc.
template <bool COLS, int NV>
__device__ void af_fft(float2* buf, const float2* tw, int logL, int ncol, int logc, float sign)
{
    int logNs = 0;
    for (; logL - logNs >= 3; logNs += 3) af_stage<COLS, 8, NV>(buf, tw, logL, ncol, logc, logNs, sign);
    if (logL - logNs == 2) af_stage<COLS, 4, NV>(buf, tw, logL, ncol, logc, logNs, sign);
    else if (logL - logNs == 1) af_stage<COLS, 2, NV>(buf, tw, logL, ncol, logc, logNs, sign);
}

// The column stages with every size known at compile time (2^LOGC columns of 2^LOGL,
// AF_T threads): the same items, twiddles and arithmetic as af_stage<true, ...>, so the
// same results, with the index arithmetic folded.
template <int RADIX, int LOGL, int LOGC, int LOGNS>
__device__ __forceinline__ void af_stage_c(float2* buf, const float2* tw, float sign)
{
    constexpr int LR = RADIX == 2 ? 1 : (RADIX == 4 ? 2 : 3);
    constexpr int m = 1 << (LOGL - LR);
    constexpr int Ns = 1 << LOGNS;
    constexpr int tstep = (1 << LOGL) >> (LOGNS + LR);
    constexpr int nitems = m << LOGC;
    constexpr int IPT = (nitems + AF_T - 1) / AF_T;
    float2 v[IPT][RADIX];
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
        const int w = (int)threadIdx.x + it * AF_T;
        if (w < nitems) {
            const int c = w & ((1 << LOGC) - 1), j = w >> LOGC;
            const int k = j & (Ns - 1);
#pragma unroll
            for (int q = 0; q < RADIX; ++q) {
                float2 x = buf[((j + q * m) << LOGC) + c];
                if (q > 0 && k) x = cmul(x, tw[q * k * tstep]);
                v[it][q] = x;
            }
            af_dft<RADIX>(v[it], sign);
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
        const int w = (int)threadIdx.x + it * AF_T;
        if (w < nitems) {
            const int c = w & ((1 << LOGC) - 1), j = w >> LOGC;
            const int base = ((j >> LOGNS) << (LOGNS + LR)) + (j & (Ns - 1));
#pragma unroll
            for (int q = 0; q < RADIX; ++q) buf[((base + q * Ns) << LOGC) + c] = v[it][q];
        }
    }
    __syncthreads();
}

template <int LOGL, int LOGC, int LOGNS = 0>
__device__ __forceinline__ void af_fft_c(float2* buf, const float2* tw, float sign)
{
    if constexpr (LOGL - LOGNS >= 3) {
        af_stage_c<8, LOGL, LOGC, LOGNS>(buf, tw, sign);
        af_fft_c<LOGL, LOGC, LOGNS + 3>(buf, tw, sign);
    } else if constexpr (LOGL - LOGNS == 2) {
        af_stage_c<4, LOGL, LOGC, LOGNS>(buf, tw, sign);
    } else if constexpr (LOGL - LOGNS == 1) {
        af_stage_c<2, LOGL, LOGC, LOGNS>(buf, tw, sign);
    }
}

// ---- column pass: segments' signals and microphone-pair RIRs -> A[seq][k2][n1]
// seq = p_local (1 + n_pairs) + 0 for the segment of point p, + 1 + q for pair q.
// LOGR_T, LCB_T: log2 of the column length and of the columns per CTA when known at
// compile time (0: from the plan).
template <int LOGR_T, int LCB_T>
__global__ void __launch_bounds__(AF_T) af_cols_kernel(AfPlan pl, int p0, const float* __restrict__ x,
                                                       const float* __restrict__ h, const int* __restrict__ starts,
                                                       float2* __restrict__ A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int logR = LOGR_T ? LOGR_T : pl.logR, R = 1 << logR;
    const int lcb = LCB_T ? LCB_T : 31 - __clz(pl.cb), cb = 1 << lcb;
    float2* buf = reinterpret_cast<float2*>(smem);   // [R][cb]
    float2* tw = buf + R * cb;                       // [R]
    // W_N^t = W_N^(t_hi 2^s) W_N^(t_lo), t = t_hi 2^s + t_lo: two short tables instead of
    // one sincospif per element (the product of two correctly rounded roots: ~2 ulp)
    const int s_lo = (pl.logN + 1) >> 1;
    float2* thi = tw + R;                         // [2^(logN - s_lo)]: W_N^(j 2^s_lo)
    float2* tlo = thi + (1 << (pl.logN - s_lo));     // [2^s_lo]: W_N^j
    const int per_point = 1 + pl.n_pairs;
    const int seq = blockIdx.y;
    const int p = p0 + seq / per_point;
    const int kind = seq % per_point;   // 0: segment, 1 + q: pair q
    const int n1_0 = blockIdx.x * cb;
    af_table(tw, logR, -1.0f);
    af_table(thi, pl.logN - s_lo, -1.0f);
    af_table(tlo, pl.logN, -1.0f, 1 << s_lo);
    // the inputs, 8 loads in flight per thread: a segment of the signal (real) or
    // the RIRs of a microphone pair (real and imaginary parts)
    const int total = R * cb;
    if (kind == 0) {
        const int a = af_start(p, pl.n_x, pl.P, starts), b = max(a, af_start(p + 1, pl.n_x, pl.P, starts));
        for (int e0 = 0; e0 < total; e0 += 8 * AF_T) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * AF_T + (int)threadIdx.x;
                const int n = n1_0 + (e & (cb - 1)) + pl.C * (e >> lcb);
                v[u] = (e < total && n >= a && n < b) ? x[n] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * AF_T + (int)threadIdx.x;
                if (e < total) buf[e] = make_float2(v[u], 0.0f);
            }
        }
    } else {
        const int m = 2 * (kind - 1);
        const float* h0 = h + ((long long)p * pl.M + m) * pl.n_S;
        const float* h1 = m + 1 < pl.M ? h0 + pl.n_S : h0;
        const float im = m + 1 < pl.M ? 1.0f : 0.0f;
        for (int e0 = 0; e0 < total; e0 += 8 * AF_T) {
            float2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * AF_T + (int)threadIdx.x;
                const int n = n1_0 + (e & (cb - 1)) + pl.C * (e >> lcb);
                const bool in = e < total && n < pl.n_S;
                v[u] = make_float2(in ? h0[n] : 0.0f, in ? h1[n] * im : 0.0f);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = e0 + u * AF_T + (int)threadIdx.x;
                if (e < total) buf[e] = v[u];
            }
        }
    }
    __syncthreads();
    if constexpr (LOGR_T != 0 && LCB_T != 0) af_fft_c<LOGR_T, LCB_T>(buf, tw, -1.0f);   // sizes folded
    else af_fft<true, AF_COL_E / AF_T>(buf, tw, logR, cb, lcb, -1.0f);
    float2* out = A + (long long)seq * pl.N;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int k2 = e >> lcb, c = e & (cb - 1);
        const int n1 = n1_0 + c;
        const int t = (n1 * k2) & (pl.N - 1);
        const float2 w = cmul(thi[t >> s_lo], tlo[t & ((1 << s_lo) - 1)]);
        out[(long long)k2 * pl.C + n1] = cmul(buf[e], w);
    }
}

// ---- row pass, in two kernels.  af_rows_kernel: per block of rb rows k2 and
// group g of the points (p = g, g + G, g + 2 G, ...), the spectra of the
// chunk's points of the group -- the rows of the segment and of the (up to npg)
// microphone pairs, transformed together as 1 + nq sequences of rb rows -- and
// their products added in ascending point order to the group's partial
// spectra Yg[g], which carry over from chunk to chunk.  af_combine_kernel,
// after the last chunk: Y = Yg[0] + Yg[1] + ... in group order, the inverse
// row DFTs (over k1 -> n1) and the twiddle W_N^(-n1 k2) -> B[pair][k2][n1]
// (stored as Y).  Every sum has a fixed order that does not depend on the
// chunk size.
__global__ void __launch_bounds__(AF_T2, 3) af_rows_kernel(AfPlan pl, int p0, int n_pts, int first,
                                                           const float2* __restrict__ A, float2* __restrict__ Yg)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int E = pl.rb * pl.C;                      // elements of one sequence's rows (a power of two)
    const int logE = pl.logC + (31 - __clz(pl.rb));
    const int Lp = pl.C + (pl.C >> 3);               // padded row (see af_stage)
    const int Ep = pl.rb * Lp;
    const int q0 = blockIdx.y * pl.npg;
    const int nq = min(pl.npg, pl.n_pairs - q0);
    const int g = blockIdx.z;
    float2* buf = reinterpret_cast<float2*>(smem);   // [1 + nq][rb] padded rows: the segment's, then the pairs'
    float2* acc = buf + (1 + pl.npg) * Ep;           // [nq][rb][C]: the group's products (element e by thread e mod T)
    float2* tw = acc + pl.npg * E;                   // [C]
    const int k2_0 = blockIdx.x * pl.rb;
    const int per_point = 1 + pl.n_pairs;
    const int cmask = pl.C - 1;
    // element e of the concatenated rows (row e / C, position e mod C) in the padded layout
    auto pad = [&](int e) { return (e >> pl.logC) * Lp + (e & cmask) + ((e & cmask) >> 3); };
    af_table(tw, pl.logC, -1.0f);
    for (int e = threadIdx.x; e < nq * E; e += blockDim.x) {
        const int qq = e >> logE, i = e & (E - 1);
        acc[e] = first ? make_float2(0.0f, 0.0f) : Yg[((long long)g * pl.n_pairs + q0 + qq) * pl.N + (long long)k2_0 * pl.C + i];
    }
    const int ns = 1 + nq;
    const int tot = ns * E;   // <= AF_ROW_E
    // the chunk's points of group g: p0 + pp = g mod G
    const int pp0 = ((g - p0) % pl.n_grp + pl.n_grp) % pl.n_grp;
    for (int pp = pp0; pp < n_pts; pp += pl.n_grp) {
        const float2* Ap = A + (long long)pp * per_point * pl.N + (long long)k2_0 * pl.C;
        __syncthreads();   // the previous point's rows are read
        for (int e0 = 0; e0 < tot; e0 += 4 * AF_T2) {
            float2 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * AF_T2 + (int)threadIdx.x;
                if (e < tot) {
                    const int sq = e >> logE, i = e & (E - 1);
                    v[u] = Ap[(long long)(sq == 0 ? 0 : 1 + q0 + (sq - 1)) * pl.N + i];
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + u * AF_T2 + (int)threadIdx.x;
                if (e < tot) buf[pad(e)] = v[u];
            }
        }
        __syncthreads();
        af_fft<false, AF_ROW_E / AF_T2>(buf, tw, pl.logC, ns * pl.rb, 0, -1.0f);
        for (int e = threadIdx.x; e < nq * E; e += blockDim.x) {
            const int i = e & (E - 1);
            const float2 xs = buf[pad(i)], zs = buf[pad(E + e)];
            float2 v = acc[e];
            v.x = __fmaf_rn(xs.x, zs.x, __fmaf_rn(-xs.y, zs.y, v.x));
            v.y = __fmaf_rn(xs.x, zs.y, __fmaf_rn(xs.y, zs.x, v.y));
            acc[e] = v;
        }
    }
    for (int e = threadIdx.x; e < nq * E; e += blockDim.x) {
        const int qq = e >> logE, i = e & (E - 1);
        Yg[((long long)g * pl.n_pairs + q0 + qq) * pl.N + (long long)k2_0 * pl.C + i] = acc[e];
    }
}

// ---- row pass, one warp per sequence (rows of C = 256 or 512 points, one row per CTA):
// the Stockham stages of af_fft (same radices, items, twiddles and arithmetic) and the
// products of af_rows_kernel, so the same results, with each warp transforming its row
// alone: only warp barriers between the stages.  The row sits in registers at both
// ends of its transform -- x[v] holds element lane + 32 v on entry and spectrum element
// lane + 32 v on return: with items j = lane + 32 it and m = L / RADIX >= 32 inputs apart,
// the first stage reads only the lane's own elements and the last (Ns = m) writes only
// them, so only the stages in between go through the warp's buffer (element i at
// i + i / 8).  Warp 0 transforms the segment's row and leaves its spectrum in one of two
// buffers (alternating per point), warp 1 + qq the row of pair q0 + qq, which then adds
// the products with the segment's spectrum to its accumulators in registers; one CTA
// barrier per point.
template <int RADIX, int LOGL, bool FIRST, bool LAST>
__device__ __forceinline__ void afw_stage(float2 (&x)[(1 << LOGL) / 32], float2* buf, const float2* tw, int lane,
                                          int logNs, float sign)
{
    constexpr int LR = RADIX == 2 ? 1 : (RADIX == 4 ? 2 : 3);
    constexpr int L = 1 << LOGL;
    constexpr int m = L / RADIX;
    static_assert(m >= 32, "every stage needs at least one item per lane");
    constexpr int IPL = m / 32;
    const int Ns = 1 << logNs;
    const int tstep = L >> (logNs + LR);
    auto pad = [](int i) { return i + (i >> 3); };
    float2 v[IPL][RADIX];
#pragma unroll
    for (int it = 0; it < IPL; ++it) {
        const int j = lane + 32 * it;
        const int k = j & (Ns - 1);
#pragma unroll
        for (int q = 0; q < RADIX; ++q) {
            float2 a = FIRST ? x[it + q * IPL] : buf[pad(j + q * m)];
            if (q > 0 && k) a = cmul(a, tw[q * k * tstep]);
            v[it][q] = a;
        }
        af_dft<RADIX>(v[it], sign);
    }
    if constexpr (LAST) {
#pragma unroll
        for (int it = 0; it < IPL; ++it)
#pragma unroll
            for (int q = 0; q < RADIX; ++q) x[it + q * IPL] = v[it][q];   // base = j when Ns = m
    } else {
        __syncwarp();   // every lane has read the buffer (this stage's inputs, or the last row's)
#pragma unroll
        for (int it = 0; it < IPL; ++it) {
            const int j = lane + 32 * it;
            const int base = ((j >> logNs) << (logNs + LR)) + (j & (Ns - 1));
#pragma unroll
            for (int q = 0; q < RADIX; ++q) buf[pad(base + q * Ns)] = v[it][q];
        }
        __syncwarp();
    }
}

template <int LOGL>
__device__ __forceinline__ void afw_fft(float2 (&x)[(1 << LOGL) / 32], float2* buf, const float2* tw, int lane,
                                        float sign)
{
    static_assert(LOGL == 8 || LOGL == 9, "stages of radix 8, 8, 4 or 8, 8, 8 (as af_fft takes them)");
    afw_stage<8, LOGL, true, false>(x, buf, tw, lane, 0, sign);
    afw_stage<8, LOGL, false, false>(x, buf, tw, lane, 3, sign);
    if constexpr (LOGL == 8) afw_stage<4, LOGL, false, true>(x, buf, tw, lane, 6, sign);
    else afw_stage<8, LOGL, false, true>(x, buf, tw, lane, 6, sign);
}

template <int LOGC>
__global__ void __launch_bounds__(32 * (1 + AF_MAXPG)) af_rows_warp_kernel(AfPlan pl, int p0, int n_pts, int first,
                                                                         const float2* __restrict__ A,
                                                                         float2* __restrict__ Yg)
{
    constexpr int C = 1 << LOGC, V = C / 32, CP = C + C / 8;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* tw = reinterpret_cast<float2*>(smem);    // [C]
    float2* bufs = tw + C;                           // [2][CP]: the segment's spectrum, by point parity
    float2* bufw = bufs + 2 * CP;                    // [1 + npg][CP]: each warp's stage buffer
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k2 = blockIdx.x;
    const int q0 = blockIdx.y * pl.npg;
    const int nq = min(pl.npg, pl.n_pairs - q0);
    const int g = blockIdx.z;
    const int per_point = 1 + pl.n_pairs;
    auto pad = [](int i) { return i + (i >> 3); };
    af_table(tw, LOGC, -1.0f);
    const bool pair = warp >= 1 && warp <= nq;
    float2* buf = bufw + warp * CP;
    float2 acc[V];
    const long long yoff = ((long long)g * pl.n_pairs + q0 + (warp - 1)) * pl.N + (long long)k2 * C;
#pragma unroll
    for (int v = 0; v < V; ++v)
        acc[v] = (pair && !first) ? Yg[yoff + lane + 32 * v] : make_float2(0.0f, 0.0f);
    __syncthreads();   // the twiddle table
    const int pp0 = ((g - p0) % pl.n_grp + pl.n_grp) % pl.n_grp;
    int par = 0;
    for (int pp = pp0; pp < n_pts; pp += pl.n_grp, par ^= 1) {
        const float2* Ap = A + (long long)pp * per_point * pl.N + (long long)k2 * C;
        float2 x[V];
        if (warp == 0 || pair) {
            const float2* src = Ap + (warp == 0 ? 0 : (long long)(1 + q0 + warp - 1) * pl.N);
#pragma unroll
            for (int v = 0; v < V; ++v) x[v] = src[lane + 32 * v];
            afw_fft<LOGC>(x, buf, tw, lane, -1.0f);
            if (warp == 0) {
#pragma unroll
                for (int v = 0; v < V; ++v) bufs[par * CP + pad(lane + 32 * v)] = x[v];
            }
        }
        __syncthreads();   // the segment's spectrum of this point is complete
        if (pair) {
            const float2* xs_b = bufs + par * CP;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float2 xs = xs_b[pad(lane + 32 * v)], zs = x[v];
                float2 a = acc[v];
                a.x = __fmaf_rn(xs.x, zs.x, __fmaf_rn(-xs.y, zs.y, a.x));
                a.y = __fmaf_rn(xs.x, zs.y, __fmaf_rn(xs.y, zs.x, a.y));
                acc[v] = a;
            }
        }
    }
    if (pair) {
#pragma unroll
        for (int v = 0; v < V; ++v) Yg[yoff + lane + 32 * v] = acc[v];
    }
}

// af_combine_kernel with one warp per pair (rows of 256 or 512 points, one row per CTA):
// the same group sums, inverse Stockham stages and twiddles, so the same results.
template <int LOGC>
__global__ void __launch_bounds__(32 * AF_MAXPG) af_combine_warp_kernel(AfPlan pl, const float2* __restrict__ Yg,
                                                                      float2* __restrict__ Y)
{
    constexpr int C = 1 << LOGC, V = C / 32, CP = C + C / 8;
    extern __shared__ __align__(16) unsigned char smem[];
    float2* tw = reinterpret_cast<float2*>(smem);    // [C]
    float2* bufw = tw + C;                           // [npg][CP]: each warp's stage buffer
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k2 = blockIdx.x;
    const int q0 = blockIdx.y * pl.npg;
    const int nq = min(pl.npg, pl.n_pairs - q0);
    af_table(tw, LOGC, 1.0f);
    __syncthreads();
    if (warp >= nq) return;   // (no barrier follows)
    const long long off = (long long)(q0 + warp) * pl.N + (long long)k2 * C;
    float2 x[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        float2 a = Yg[off + lane + 32 * v];
        for (int gg = 1; gg < pl.n_grp; ++gg) a = cadd(a, Yg[(long long)gg * pl.n_pairs * pl.N + off + lane + 32 * v]);
        x[v] = a;
    }
    afw_fft<LOGC>(x, bufw + warp * CP, tw, lane, 1.0f);
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int n1 = lane + 32 * v;
        Y[off + n1] = cmul(x[v], af_root((n1 * k2) & (pl.N - 1), pl.logN, 1.0f));
    }
}

__global__ void __launch_bounds__(AF_T2) af_combine_kernel(AfPlan pl, const float2* __restrict__ Yg,
                                                           float2* __restrict__ Y)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int E = pl.rb * pl.C;
    const int logE = pl.logC + (31 - __clz(pl.rb));
    const int Lp = pl.C + (pl.C >> 3);
    const int q0 = blockIdx.y * pl.npg;
    const int nq = min(pl.npg, pl.n_pairs - q0);
    float2* acc = reinterpret_cast<float2*>(smem);   // [nq][rb] padded rows
    float2* tw = acc + pl.npg * pl.rb * Lp;          // [C]
    const int k2_0 = blockIdx.x * pl.rb;
    const int cmask = pl.C - 1;
    auto pad = [&](int e) { return (e >> pl.logC) * Lp + (e & cmask) + ((e & cmask) >> 3); };
    for (int e = threadIdx.x; e < nq * E; e += blockDim.x) {
        const int qq = e >> logE, i = e & (E - 1);
        const long long off = (long long)(q0 + qq) * pl.N + (long long)k2_0 * pl.C + i;
        float2 v = Yg[off];
        for (int gg = 1; gg < pl.n_grp; ++gg) v = cadd(v, Yg[(long long)gg * pl.n_pairs * pl.N + off]);
        acc[pad(e)] = v;
    }
    af_table(tw, pl.logC, 1.0f);
    __syncthreads();
    af_fft<false, AF_ROW_E / AF_T2>(acc, tw, pl.logC, nq * pl.rb, 0, 1.0f);
    for (int e = threadIdx.x; e < nq * E; e += blockDim.x) {
        const int qq = e >> logE, i = e & (E - 1);
        const int r = i >> pl.logC, n1 = i & cmask;
        const int k2 = k2_0 + r;
        Y[(long long)(q0 + qq) * pl.N + (long long)k2 * pl.C + n1] =
            cmul(acc[pad(e)], af_root((n1 * k2) & (pl.N - 1), pl.logN, 1.0f));
    }
}

// ---- inverse column pass: B[pair][k2][n1] -> y (real part: microphone 2q,
// imaginary part: microphone 2q + 1), scaled by 1 / N.
__global__ void __launch_bounds__(AF_T) af_icols_kernel(AfPlan pl, const float2* __restrict__ B, float* __restrict__ y)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float2* buf = reinterpret_cast<float2*>(smem);   // [R][cb3]
    float2* tw = buf + pl.R * pl.cb3;
    const int q = blockIdx.y;
    const int n1_0 = blockIdx.x * pl.cb3;
    af_table(tw, pl.logR, 1.0f);
    const float2* Bq = B + (long long)q * pl.N;
    const int total = pl.R * pl.cb3;
    const int lcb3 = 31 - __clz(pl.cb3);
    for (int e0 = 0; e0 < total; e0 += 8 * AF_T) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * AF_T + (int)threadIdx.x;
            if (e < total) v[u] = Bq[(long long)(e >> lcb3) * pl.C + n1_0 + (e & (pl.cb3 - 1))];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * AF_T + (int)threadIdx.x;
            if (e < total) buf[e] = v[u];
        }
    }
    __syncthreads();
    if (pl.logR == 9 && pl.cb3 == 4) af_fft_c<9, 2>(buf, tw, 1.0f);
    else if (pl.logR == 8 && pl.cb3 == 8) af_fft_c<8, 3>(buf, tw, 1.0f);
    else af_fft<true, AF_COL_E / AF_T>(buf, tw, pl.logR, pl.cb3, 31 - __clz(pl.cb3), 1.0f);
    const float inv_n = __int_as_float((127 - pl.logN) << 23);   // 1 / N, exact
    const int m = 2 * q;
    float* y0 = y + (long long)m * pl.n_out;
    float* y1 = m + 1 < pl.M ? y0 + pl.n_out : nullptr;
    for (int e = threadIdx.x; e < pl.R * pl.cb3; e += blockDim.x) {
        const int n2 = e >> lcb3, c = e & (pl.cb3 - 1);
        const long long n = (long long)n1_0 + c + (long long)pl.C * n2;
        if (n < pl.n_out) {
            y0[n] = buf[e].x * inv_n;
            if (y1) y1[n] = buf[e].y * inv_n;
        }
    }
}

}  // namespace

// Plan of the FFT form: sizes and the points per chunk that a workspace of
// ws_bytes holds (0: the default, about 96 MB of column-pass output per chunk).
int ism_auralize_fft_plan(int n_x, int n_points, int n_mics, int n_S, size_t ws_bytes, AfPlan* out, size_t* need)
{
    AfPlan pl{};
    const long long n_out = (long long)n_x + n_S - 1;
    int logN = 4;
    while ((1ll << logN) < n_out) ++logN;
    if (logN > 20) return -1;
    pl.N = 1 << logN;
    pl.logN = logN;
    pl.logR = (logN + 1) / 2;
    pl.logC = logN / 2;
    pl.R = 1 << pl.logR;
    pl.C = 1 << pl.logC;
    pl.n_x = n_x;
    pl.P = n_points;
    pl.M = n_mics;
    pl.n_S = n_S;
    pl.n_out = (int)n_out;
    pl.n_pairs = (n_mics + 1) / 2;
    pl.cb = std::min(pl.C, std::max(1, AF_COL_E / pl.R));
    pl.cb3 = std::min(pl.C, std::max(1, 2048 / pl.R));
    pl.rb = std::min(pl.R, std::max(1, 256 / pl.C));
    // pairs per row-pass CTA: its 1 + npg sequences of rb rows fit the 4 radix-4 items per thread
    pl.npg = std::max(1, std::min(AF_MAXPG, AF_ROW_E / (pl.rb * pl.C) - 1));
    pl.n_pg = (pl.n_pairs + pl.npg - 1) / pl.npg;
    // point groups of the row pass: enough CTAs to fill the GPU several times over
    const long long row_ctas = (long long)(pl.R / pl.rb) * pl.n_pg;
    pl.n_grp = (int)std::max(1LL, std::min((long long)AF_MAXGRP, (4LL * 152 * 4 + row_ctas - 1) / row_ctas));
    const size_t seq_bytes = (size_t)pl.N * sizeof(float2);
    const size_t per_point = (size_t)(1 + pl.n_pairs) * seq_bytes;
    const size_t y_bytes = (size_t)(1 + pl.n_grp) * pl.n_pairs * seq_bytes;   // Y and the groups' partial spectra
    // points per chunk: the column-pass output of a chunk fills the workspace (by default
    // about 96 MB, within L2), and its sequences fit one grid dimension
    const size_t max_pc = std::max<size_t>(1, 65535 / (size_t)(1 + pl.n_pairs));
    if (ws_bytes == 0) {
        pl.pc = (int)std::max<size_t>(1, std::min<size_t>((size_t)n_points, ((size_t)96 << 20) / per_point));
    } else {
        if (ws_bytes < y_bytes + per_point) return -2;
        pl.pc = (int)std::min<size_t>((size_t)n_points, (ws_bytes - y_bytes) / per_point);
    }
    pl.pc = (int)std::min<size_t>((size_t)pl.pc, max_pc);
    *out = pl;
    *need = y_bytes + (size_t)pl.pc * per_point;
    return 0;
}

static size_t af_cols_smem(const AfPlan& pl, int cb)
{
    const int s_lo = (pl.logN + 1) >> 1;
    return ((size_t)pl.R * cb + pl.R + (1u << (pl.logN - s_lo)) + (1u << s_lo)) * sizeof(float2);
}
static size_t af_rows_smem(const AfPlan& pl)
{
    return ((size_t)(1 + pl.npg) * pl.rb * (pl.C + (pl.C >> 3)) + (size_t)pl.npg * pl.rb * pl.C + pl.C) *
           sizeof(float2);
}
static size_t af_rows_warp_smem(const AfPlan& pl)
{
    const size_t cp = (size_t)pl.C + (pl.C >> 3);
    return ((size_t)pl.C + (3 + (size_t)pl.npg) * cp) * sizeof(float2);
}
static size_t af_combine_smem(const AfPlan& pl)
{
    return ((size_t)pl.npg * pl.rb * (pl.C + (pl.C >> 3)) + pl.C) * sizeof(float2);
}

int ism_launch_auralize_fft(const float* x, const float* h, const int* starts, float* y, const AfPlan& pl, char* ws,
                            void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    float2* Y = reinterpret_cast<float2*>(ws);       // the pairs' spectra, then B
    float2* Yg = Y + (size_t)pl.n_pairs * pl.N;      // the point groups' partial spectra
    float2* A = Yg + (size_t)pl.n_grp * pl.n_pairs * pl.N;
    static std::atomic<unsigned long long> o1{0}, o2{0}, o3{0}, o4{0};
    int rc;
    static std::atomic<unsigned long long> o1b{0}, o1c{0};
    if ((rc = ism_open_smem((const void*)af_cols_kernel<0, 0>, &o1))) return rc;
    if ((rc = ism_open_smem((const void*)af_cols_kernel<9, 4>, &o1b))) return rc;
    if ((rc = ism_open_smem((const void*)af_cols_kernel<8, 5>, &o1c))) return rc;
    if ((rc = ism_open_smem((const void*)af_rows_kernel, &o2))) return rc;
    if ((rc = ism_open_smem((const void*)af_icols_kernel, &o3))) return rc;
    if ((rc = ism_open_smem((const void*)af_combine_kernel, &o4))) return rc;
    const int per_point = 1 + pl.n_pairs;
    for (int p0 = 0; p0 < pl.P; p0 += pl.pc) {
        const int n_pts = std::min(pl.pc, pl.P - p0);
        const dim3 cgrid((unsigned)(pl.C / pl.cb), (unsigned)(n_pts * per_point));
        const size_t csm = af_cols_smem(pl, pl.cb);
        if (pl.logR == 9 && pl.cb == 16)
            af_cols_kernel<9, 4><<<cgrid, AF_T, csm, s>>>(pl, p0, x, h, starts, A);
        else if (pl.logR == 8 && pl.cb == 32)
            af_cols_kernel<8, 5><<<cgrid, AF_T, csm, s>>>(pl, p0, x, h, starts, A);
        else
            af_cols_kernel<0, 0><<<cgrid, AF_T, csm, s>>>(pl, p0, x, h, starts, A);
        if ((rc = (int)cudaGetLastError())) return rc;
        const dim3 rgrid((unsigned)(pl.R / pl.rb), (unsigned)pl.n_pg, (unsigned)pl.n_grp);
        if (pl.C == 256 && pl.rb == 1)
            af_rows_warp_kernel<8><<<rgrid, 32 * (1 + pl.npg), af_rows_warp_smem(pl), s>>>(pl, p0, n_pts, p0 == 0, A, Yg);
        else if (pl.C == 512 && pl.rb == 1)
            af_rows_warp_kernel<9><<<rgrid, 32 * (1 + pl.npg), af_rows_warp_smem(pl), s>>>(pl, p0, n_pts, p0 == 0, A, Yg);
        else
            af_rows_kernel<<<rgrid, AF_T2, af_rows_smem(pl), s>>>(pl, p0, n_pts, p0 == 0, A, Yg);
        if ((rc = (int)cudaGetLastError())) return rc;
    }
    const dim3 cgrid2((unsigned)(pl.R / pl.rb), (unsigned)pl.n_pg);
    const size_t wsm = ((size_t)pl.C + (size_t)pl.npg * (pl.C + (pl.C >> 3))) * sizeof(float2);
    if (pl.C == 256 && pl.rb == 1)
        af_combine_warp_kernel<8><<<cgrid2, 32 * pl.npg, wsm, s>>>(pl, Yg, Y);
    else if (pl.C == 512 && pl.rb == 1)
        af_combine_warp_kernel<9><<<cgrid2, 32 * pl.npg, wsm, s>>>(pl, Yg, Y);
    else
        af_combine_kernel<<<cgrid2, AF_T2, af_combine_smem(pl), s>>>(pl, Yg, Y);
    if ((rc = (int)cudaGetLastError())) return rc;
    af_icols_kernel<<<dim3((unsigned)(pl.C / pl.cb3), (unsigned)pl.n_pairs), AF_T, af_cols_smem(pl, pl.cb3), s>>>(
        pl, Y, y);
    return (int)cudaGetLastError();
}
