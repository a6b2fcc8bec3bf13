// ism_api.cu -- the C ABI of libism (include/ism.h): argument validation,
// planning of the launch set and of the workspace, and the launch sequence.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "ism_internal.h"

namespace {

thread_local std::string g_last_error;

ism_status fail(ism_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

ism_status cuda_fail(int e, const char* where)
{
    return fail(ISM_ERR_CUDA, "%s: %s", where, cudaGetErrorString((cudaError_t)e));
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// n = ceil(T fs (1 - 1e-6)): the relative slack absorbs the FP32 rounding of T
// (1.2 s is stored as 1.2000000477 s, which would otherwise add a sample).
int rir_len(double T, double fs) { return (int)std::ceil(T * fs * (1.0 - 1e-6)); }

bool isfin(double x) { return std::isfinite(x); }

double t60_of(const double L[3], const double beta[6])
{
    double S[6] = {L[1] * L[2], L[1] * L[2], L[0] * L[2], L[0] * L[2], L[0] * L[1], L[0] * L[1]};
    double den = 0.0;
    for (int i = 0; i < 6; ++i) den += S[i] * (1.0 - beta[i] * beta[i]);
    if (!(den > 0.0)) return INFINITY;
    return 0.161 * L[0] * L[1] * L[2] / den;
}

// Window length in taps, snapped to an integer when Tw fs is one up to the
// FP32 rounding of Tw (32 / 16000 s is not exact in FP32).
double window_taps(double Tw, double fs)
{
    double nw = Tw * fs;
    double rn = std::nearbyint(nw);
    if (std::fabs(nw - rn) <= 1e-4 * (rn > 1.0 ? rn : 1.0)) nw = rn;
    return nw;
}

struct Validated {
    ism_job job;
    double Tw, Nw;
    int n_S, n_ism, H, slots;
    int rir_index0 = 0;   // index of the first RIR in the caller's job (a sub-job of a split job)
    // backward pass only
    const float* grad_out = nullptr;
    float* grad_beta = nullptr;
    float* grad_src = nullptr;
    float* grad_rcv = nullptr;
};

ism_status validate_job(const ism_job& in, Validated& v, bool need_ptrs)
{
    v.job = in;
    ism_job& j = v.job;
    for (int a = 0; a < 3; ++a)
        if (!(j.room.L[a] > 0.0) || !isfin(j.room.L[a]))
            return fail(ISM_ERR_INVALID_ARG, "room size L[%d] = %g must be finite and > 0", a, j.room.L[a]);
    for (int w = 0; w < 6; ++w)
        if (!j.beta_dev && (!isfin(j.room.beta[w]) || std::fabs(j.room.beta[w]) > 1.0f))
            return fail(ISM_ERR_INVALID_ARG, "beta[%d] = %g must satisfy |beta| <= 1", w, (double)j.room.beta[w]);
    if (!(j.room.c > 0.0f)) j.room.c = 343.0f;
    if (!isfin(j.room.c)) return fail(ISM_ERR_INVALID_ARG, "speed of sound must be finite");
    if (!(j.fs > 0.0f) || !isfin(j.fs)) return fail(ISM_ERR_INVALID_ARG, "fs = %g must be > 0", (double)j.fs);
    if (!(j.Tmax > 0.0f) || !isfin(j.Tmax)) return fail(ISM_ERR_INVALID_ARG, "Tmax = %g must be > 0", (double)j.Tmax);
    if (!isfin(j.Tdiff) || !isfin(j.Tw)) return fail(ISM_ERR_INVALID_ARG, "Tdiff and Tw must be finite");
    if (j.n_src < 1 || j.n_rcv < 1) return fail(ISM_ERR_INVALID_ARG, "need n_src >= 1 and n_rcv >= 1");
    if ((long long)j.n_src * j.n_rcv > (1ll << 30)) return fail(ISM_ERR_UNSUPPORTED, "too many RIRs in one job");
    for (int a = 0; a < 3; ++a) {
        if (j.nb_img[a] < 1) return fail(ISM_ERR_INVALID_ARG, "nb_img[%d] = %d must be >= 1", a, j.nb_img[a]);
        if (j.nb_img[a] > ISM_MAX_AXIS)
            return fail(ISM_ERR_UNSUPPORTED, "nb_img[%d] = %d exceeds %d", a, j.nb_img[a], ISM_MAX_AXIS);
    }
    if (need_ptrs && (!j.pos_src || !j.pos_rcv || !j.out))
        return fail(ISM_ERR_INVALID_ARG, "pos_src, pos_rcv and out must be device pointers, not NULL");
    if (j.mic_pattern < ISM_MIC_OMNI || j.mic_pattern > ISM_MIC_BIDIRECTIONAL)
        return fail(ISM_ERR_INVALID_ARG, "mic_pattern = %d is not an ism_mic_pattern", j.mic_pattern);
    if (j.envelope != ISM_ENVELOPE_SABINE && j.envelope != ISM_ENVELOPE_LJ)
        return fail(ISM_ERR_INVALID_ARG, "envelope = %d is not an ism_envelope", j.envelope);
    if (need_ptrs && j.mic_pattern != ISM_MIC_OMNI && !j.orient_rcv)
        return fail(ISM_ERR_INVALID_ARG, "a polar pattern needs orient_rcv (device pointer, [n_rcv][3])");
    v.Tw = (j.Tw > 0.0f) ? (double)j.Tw : 4e-3;
    v.Nw = window_taps(v.Tw, (double)j.fs);
    if (!(v.Nw >= 2.0)) return fail(ISM_ERR_INVALID_ARG, "window of %g taps: need Tw * fs >= 2", v.Nw);
    if (v.Nw > 32.0 * ISM_MAX_SLOTS) return fail(ISM_ERR_UNSUPPORTED, "window of %g taps exceeds 256", v.Nw);
    v.n_S = rir_len(j.Tmax, j.fs);
    if (v.n_S < 1) return fail(ISM_ERR_INVALID_ARG, "Tmax * fs < 1 sample");
    v.n_ism = (j.Tdiff > 0.0f && j.Tdiff < j.Tmax) ? rir_len(j.Tdiff, j.fs) : v.n_S;
    if (v.n_ism > v.n_S) v.n_ism = v.n_S;
    if (v.n_ism < 0) v.n_ism = 0;
    if (v.n_ism > ISM_MAX_NISM)
        return fail(ISM_ERR_UNSUPPORTED, "%d image-source samples exceed %d", v.n_ism, ISM_MAX_NISM);
    v.H = (int)std::ceil(0.5 * v.Nw - 1e-9);
    if ((v.n_ism + v.H) / ISM_SB + 1 > ISM_MAX_Q)
        return fail(ISM_ERR_UNSUPPORTED, "%d image-source samples exceed the bin limit", v.n_ism);
    v.slots = (2 * v.H + 31) / 32;
    return ISM_OK;
}

// Builds the device job table and the workspace plan of one launch set.
// Chebyshev coefficients of the 32 tap functions of a 32-tap window:
// g_t(f) = delta'(t - 15 - f) (eq. (6)), f = (u + 1) / 2, interpolated at the
// Chebyshev-Gauss nodes u_k = cos(pi (k + 1/2) / N): c_i = (2 / N) sum_k
// g_t(u_k) T_i(u_k), c_0 halved.  FP64 on the host, once per process.
// Chebyshev interpolation coefficients of the 32 tap functions at N nodes (degree
// N - 1): N = ISM_CHEB_NF for the forward's moments, ISM_CHEB_N for the adjoint's
// tables; stride ISM_CHEB_N per tap either way (unused terms zero).
static void cheb_fill(float* c, int N)
{
        for (int tap = 0; tap < 32; ++tap) {
            const int j = tap - 15;
            for (int i = 0; i < N; ++i) {
                double s = 0.0;
                for (int k = 0; k < N; ++k) {
                    const double th = M_PI * (k + 0.5) / N;
                    const double x = (double)j - 0.5 * (std::cos(th) + 1.0);
                    double g = 0.0;
                    if (std::fabs(x) < 16.0) {
                        const double w = 0.5 * (1.0 + std::cos(M_PI * x / 16.0));
                        g = w * (x == 0.0 ? 1.0 : std::sin(M_PI * x) / (M_PI * x));
                    }
                    s += g * std::cos(i * th);
                }
                s *= 2.0 / N;
                if (i == 0) s *= 0.5;
                c[tap * ISM_CHEB_N + i] = (float)s;
            }
        }
}

const float* cheb_coefficients(bool forward)
{
    static float cf[32 * ISM_CHEB_N], ca[32 * ISM_CHEB_N];
    static std::once_flag once;
    std::call_once(once, [] {
        cheb_fill(cf, ISM_CHEB_NF);
        cheb_fill(ca, ISM_CHEB_N);
    });
    return forward ? cf : ca;
}

// Lays the launch set out in the workspace from byte offset `base` on (the
// status word is always at offset 0, shared by every launch set of a call).
ism_status plan(const Validated* vs, int n, ism_precision prec, bool backward, JobTable& t, WsPlan& p,
                size_t base = 0)
{
    std::memset(&t, 0, sizeof t);
    std::memset(&p, 0, sizeof p);
    t.n_jobs = n;
    long long set_cols = 0;   // grid columns x RIRs over the launch set
    for (int i = 0; i < n; ++i)
        set_cols += (long long)vs[i].job.nb_img[0] * vs[i].job.nb_img[1] * vs[i].job.n_src * vs[i].job.n_rcv;
    long long rir = 0, hist = 0, tbl = 0, ecta = 0, acta = 0, adta = 0, tcta = 0, fcta = 0, rows = 0, ids = 0, lut = 0,
              gpart = 0, srir = 0, scta = 0, env = 0, vcta = 0, sdc = 0, vslot = 0, sdrir = 0;
    int sd_gmax = 0;   // most shells of a fused direct RIR
    for (int i = 0; i < n; ++i) {
        const Validated& v = vs[i];
        const ism_job& in = v.job;
        JobDev& J = t.j[i];
        for (int a = 0; a < 3; ++a) {
            J.L[a] = in.room.L[a];
            J.N[a] = in.nb_img[a];
            J.nlo[a] = -(in.nb_img[a] / 2);
        }
        for (int w = 0; w < 6; ++w) J.beta[w] = in.room.beta[w];
        J.beta_dev = in.beta_dev;
        J.g2_c = 6.0 * std::log2(10.0);
        J.c = in.room.c;
        J.fs = in.fs;
        J.Nw = (float)v.Nw;
        double k = (double)in.fs / (double)in.room.c;
        J.kfs_hi = (float)k;
        J.kfs_lo = (float)(k - (double)J.kfs_hi);
        J.amp_scale = (float)(k / (4.0 * M_PI));
        // FP16X2: |P| <= amp_scale / 2 and |w| <= 2 |P|, so a scale of 2^e with
        // amp_scale 2^e <= 8192 keeps every packed value below the FP16 maximum
        J.half_scale = 1.0f;
        if (prec == ISM_PREC_FP16X2) {
            int e = (int)std::floor(std::log2(8192.0 / (double)J.amp_scale));
            e = e < -24 ? -24 : (e > 24 ? 24 : e);
            J.half_scale = (float)std::ldexp(1.0, e);
        }
        J.n_src = in.n_src;
        J.n_rcv = in.n_rcv;
        J.n_rir = in.n_src * in.n_rcv;
        J.n_S = v.n_S;
        J.n_ism = v.n_ism;
        J.H = v.H;
        J.slots = v.slots;
        J.Q = (v.n_ism + v.H) / ISM_SB + 1;
        J.img_per_rir = (long long)in.nb_img[0] * in.nb_img[1] * in.nb_img[2];
        // enumeration units: contiguous column ranges, about 16k warps over the
        // launch set (enough to hide the latency of the walk while keeping the
        // per-unit histogram small), at most 512 columns each
        {
            const long long cols = (long long)in.nb_img[0] * in.nb_img[1];
            long long cpu = (set_cols + 16383) / 16384;
            if (cpu < 1) cpu = 1;
            if (cpu > 512) cpu = 512;
            if (cpu > cols) cpu = cols;
            J.cols_per_unit = (int)cpu;
            J.U = (int)((cols + cpu - 1) / cpu);
        }
        J.inv_kLz = (float)(1.0 / (k * in.room.L[2]));
        for (int a = 0; a < 3; ++a) J.inv2L[a] = (float)(0.5 / in.room.L[a]);
        J.kinv = in.room.c / in.fs;   // FP32 division, as the kernels did it
        J.Lmax = (float)std::max(in.room.L[0], std::max(in.room.L[1], in.room.L[2]));
        J.vol = (float)(in.room.L[0] * in.room.L[1] * in.room.L[2]);

        J.n_tiles = (J.Q + ISM_TILE_BINS - 1) / ISM_TILE_BINS;
        double s_cut = (double)v.n_ism - 1.0 + (double)v.H + 0.5;
        J.s_cut2 = (float)(s_cut * s_cut);
        J.has_tail = v.n_ism < v.n_S;
        double beta_d[6];
        for (int w = 0; w < 6; ++w) beta_d[w] = in.room.beta[w];
        double T60 = t60_of(in.room.L, beta_d);
        {
            const double g2 = std::isfinite(T60) ? J.g2_c / ((double)in.fs * T60) : 0.0;   // (device: ism_job_g2)
            J.g2 = (float)g2;
            J.g2_lo = (float)(g2 - (double)J.g2);
        }
        J.envelope = in.envelope;
        int W = (int)std::ceil(ISM_FIT_WINDOW_S * (double)in.fs - 1e-9);
        J.W_env = W < v.n_ism ? W : v.n_ism;
        J.vec4 = (v.n_S % 4 == 0) && (((uintptr_t)in.out & 15u) == 0);
        J.seed = in.seed;
        J.rir_index0 = v.rir_index0;
        J.pos_src = in.pos_src;
        J.pos_rcv = in.pos_rcv;
        {
            static const float alpha_of[5] = {1.0f, 0.75f, 0.5f, 0.25f, 0.0f};
            J.mic_alpha = alpha_of[in.mic_pattern];
            J.orient_rcv = in.mic_pattern != ISM_MIC_OMNI ? in.orient_rcv : nullptr;
        }
        J.out = in.out;
        J.env_amp = in.env_amp;
        J.rir_base = rir;
        J.hist_base = hist;
        J.tbl_base = tbl;
        J.enum_cta_base = ecta;
        J.acc_cta_base = acta;
        J.adj_cta_base = adta;
        J.tail_cta_base = tcta;
        J.fin_cta_base = fcta;
        J.fin_chunk = std::max(2048, (J.W_env + 255) / 256 * 256);
        J.fin_chunks = std::max(1, (v.n_ism + J.fin_chunk - 1) / J.fin_chunk);
        J.rows_base = rows;
        J.lut_base = lut;
        // Chebyshev moments pay off when a delay bin holds enough images to
        // amortise the expansion of its 33 offsets and the shell's enumeration
        // set-up: estimate the images in reach per bin from the sphere of radius
        // n_ism + H samples.  Measured against the fused direct form (64 RIRs a
        // call): 84 per bin, the same time; 181, 6 % faster; 338, 31 %; 1352, 2.7x;
        // the 48 kHz array with ~36 per bin is 2.9x faster in the direct form.  The
        // crossover lies near 64-100; 64 is kept.
        {
            const double reach = ((double)v.n_ism + v.H) / k;                     // metres
            const double vol = in.room.L[0] * in.room.L[1] * in.room.L[2];
            const double in_reach = std::min((double)in.nb_img[0] * in.nb_img[1] * in.nb_img[2],
                                             4.18879020478639 * reach * reach * reach / vol);
            const double per_bin = in_reach / (double)((v.n_ism + v.H) / ISM_SB + 1);
            J.use_cheb = (prec == ISM_PREC_FP32 && !backward && v.Nw == 32.0 && v.H == 16 && v.slots == 1 &&
                          per_bin >= 64.0) ? 1 : 0;
            // sparse bins: sorting by offset and padding each offset to a group of 4
            // images costs more than adding every image's taps on its own
            J.sparse = ((prec == ISM_PREC_FP32 || prec == ISM_PREC_FP32_DIRECT) && !backward && !J.use_cheb &&
                        per_bin < 128.0) ? 1 : 0;
            // backward: a 32-tap window always takes the fused Chebyshev adjoint (an
            // image costs two degree-8 sums there, against 32 tap derivatives)
            J.adj_cheb = (backward && v.Nw == 32.0 && v.H == 16 && v.slots == 1) ? 1 : 0;
            // the other forward jobs with a 32-tap window, in every tap arithmetic: every tap
            // evaluated, the images enumerated by the CTA that accumulates them (no ids, no
            // sort); the value is the shell's thickness in bins: 32 for sparse bins, 8 for dense ones
            J.shell_direct = (!backward && !J.use_cheb && v.Nw == 32.0 && v.H == 16 && v.slots == 1)
                                 ? (per_bin < 64.0 ? ISM_SD_BINS : 8) : 0;
        }
        const bool cheb = J.use_cheb || J.adj_cheb;
        const bool fused = cheb || J.shell_direct;
        // a job takes the fused Chebyshev CTAs or the fused direct CTAs (both enumerate
        // their own images), or the direct accumulation CTAs (which read the binned ids)
        J.acc_groups = (J.use_cheb || J.shell_direct) ? 0 : (J.Q + ism_acc_bins((int)prec) - 1) / ism_acc_bins((int)prec);
        J.shell_groups = cheb ? (J.Q + ISM_SHELL_BINS - 1) / ISM_SHELL_BINS
                              : (J.shell_direct ? (J.Q + J.shell_direct - 1) / J.shell_direct : 0);
        J.shell_rir_base = srir;
        J.shell_cta_base = scta;
        J.sd_cta_base = (int)sdc;
        J.sd_rir_base = (int)sdrir;
        J.grad_out = v.grad_out;
        J.grad_beta = v.grad_beta;
        J.grad_src = v.grad_src;
        J.grad_rcv = v.grad_rcv;
        J.gpart_base = gpart;
        J.rgrad_base = rir * 12;
        const long long R = J.n_rir;
        rir += R;
        // a fused Chebyshev job enumerates its images itself: no counts, no binned ids
        if (!fused) hist += R * J.Q * J.U;
        int axis = in.nb_img[0] + in.nb_img[1] + in.nb_img[2];
        tbl += R * axis;
        if (!fused) ecta += R * ((J.U + ISM_ENUM_WARPS - 1) / ISM_ENUM_WARPS);
        acta += R * J.acc_groups;
        if (cheb) {
            srir += R;
            scta += R * J.shell_groups;
            if (J.shell_groups > t.shell_gmax) t.shell_gmax = J.shell_groups;
        }
        if (J.shell_direct) {
            sdc += R * J.shell_groups;
            sdrir += R;
            if (J.shell_groups > sd_gmax) sd_gmax = J.shell_groups;
        }
        fcta += R * J.fin_chunks;
        if (backward && !J.adj_cheb) adta += R * J.n_tiles;
        if (J.has_tail) {
            int blk0 = v.n_ism >> 2, blk_last = (v.n_S - 1) >> 2;
            tcta += R * ((blk_last - blk0 + 1 + ISM_TAIL_CHUNK / 4 - 1) / (ISM_TAIL_CHUNK / 4));
        }
        // Lehmann-Johansson tails: one envelope table per job, from the fit window to the end
        J.env_k0 = v.n_ism - J.W_env;
        J.env_base = env;
        J.env_cta_base = vcta;
        J.env_slot = (int)vslot;
        if (J.has_tail && J.envelope == ISM_ENVELOPE_LJ) {
            const long long n_env = (long long)v.n_S - J.env_k0;
            env += (n_env + 63) / 64 * 64;
            vcta += (n_env + ISM_ENV_CHUNK - 1) / ISM_ENV_CHUNK;
            ++vslot;
        }
        rows += R * J.Q * 32LL * (J.slots + 1);
        if (prec == ISM_PREC_LUT) lut += (long long)(ism_lut_phases(J.slots) + 1) * 32 * J.slots;
        // texture form: each table starts on a 512-byte boundary (texture base alignment)
        if (prec == ISM_PREC_LUT_TEX) lut += ((long long)(ism_lut_phases(J.slots) + 1) * 32 * J.slots + 127) / 128 * 128;
        if (cheb) t.any_cheb = 1;
        else if (!fused) t.any_direct = 1;
        if (backward) gpart += R * J.Q * 12;
        if (!fused) ids += R * J.img_per_rir;
        if (J.Q > t.max_Q) t.max_Q = J.Q;
        if (axis > t.max_axis_sum) t.max_axis_sum = axis;
    }
    if (hist > (long long)ISM_SCAN_BLOCK * ISM_SCAN_TOP)
        return fail(ISM_ERR_UNSUPPORTED, "delay-bin histogram of %lld entries exceeds %lld; split the batch", hist,
                    (long long)ISM_SCAN_BLOCK * ISM_SCAN_TOP);
    if (ids >= 0xFFFFFFFFll)
        return fail(ISM_ERR_UNSUPPORTED, "%lld images in one launch set exceed 2^32; split the batch", ids);
    if (rir > 0x7FFFFFFFll || ecta > 0x7FFFFFFFll || acta > 0x7FFFFFFFll || adta > 0x7FFFFFFFll ||
        tcta > 0x7FFFFFFFll || fcta > 0x7FFFFFFFll || srir * (long long)t.shell_gmax > 0x7FFFFFFFll ||
        env > 0x7FFFFFFFll || vcta > 0x7FFFFFFFll || sdrir * (long long)sd_gmax > 0x7FFFFFFFll || gpart > 0x7FFFFFFFll ||
        rir * 12 > 0x7FFFFFFFll || lut > 0x7FFFFFFFll)
        return fail(ISM_ERR_UNSUPPORTED, "launch set too large; split the batch");
    p.hist_total = hist;
    p.ids_total = ids;
    p.n_scan_blocks = (hist + ISM_SCAN_BLOCK - 1) / ISM_SCAN_BLOCK;
    if (p.n_scan_blocks < 1) p.n_scan_blocks = 1;
    p.tbl_total = tbl;
    p.rows_total = rows;
    if (t.any_cheb) std::memcpy(t.cheb, cheb_coefficients(!backward), sizeof t.cheb);
    p.rir_total = rir;
    p.lut_total = lut;
    p.gpart_total = gpart;
    p.rgrad_total = backward ? rir * 12 : 0;
    p.env_total = backward ? 0 : env;
    p.env_ctas = backward ? 0 : vcta;
    p.env_slots = backward ? 0 : vslot;
    p.enum_ctas = ecta;
    p.acc_ctas = acta;
    // Small launch sets: thinner Chebyshev shells, so that the fused launch still fills
    // the GPU (ISM_FILL_CTAS CTAs at least; a single RIR would otherwise run on ~20
    // SMs): from 8 bins down to 1.  The moment sums are exact integers and each bin's
    // fixed-point scale depends on that bin alone, so a job's result does not depend on
    // the thickness, nor on the launch set it shares.  (The direct form keeps each job's
    // own thickness: there the CTA split sets the order of the floating-point sums.)
    t.shell_bins = ISM_SHELL_BINS;
    if (!backward && scta > 0 && scta < ISM_FILL_CTAS) {
        auto ctas = [&](int bins) {
            long long c = 0;
            for (int i = 0; i < n; ++i)
                if (t.j[i].use_cheb) c += t.j[i].n_rir * (long long)((t.j[i].Q + bins - 1) / bins);
            return c;
        };
        int bc = ISM_SHELL_BINS;
        while (bc > 1 && ctas(bc) < ISM_FILL_CTAS) bc >>= 1;
        t.shell_bins = bc;
        scta = 0;
        t.shell_gmax = 0;
        for (int i = 0; i < n; ++i) {
            JobDev& J = t.j[i];
            J.shell_cta_base = scta;
            if (!J.use_cheb) continue;
            J.shell_groups = (J.Q + bc - 1) / bc;
            scta += J.n_rir * (long long)J.shell_groups;
            t.shell_gmax = std::max(t.shell_gmax, J.shell_groups);
        }
    }
    t.shell_rirs = srir;
    // shell-rank order when the jobs' shell counts are alike (at most 1/8 of the
    // rank-major grid would be CTAs past their job's shells), else job-major
    t.shell_rank_major = (srir * (long long)t.shell_gmax * 7 <= scta * 8) ? 1 : 0;
    p.shell_ctas = t.shell_rank_major ? srir * t.shell_gmax : scta;
    p.adj_ctas = adta;
    // the fused direct CTAs the same way (shells of one thickness per job: 8 or 32 bins)
    const bool sd_rank = sdrir > 0 && sdrir * (long long)sd_gmax * 7 <= sdc * 8;
    t.sd_rank_rirs = sd_rank ? (int)sdrir : 0;
    p.sd_ctas = sd_rank ? sdrir * sd_gmax : sdc;
    p.tail_ctas = tcta;
    p.fin_ctas = fcta;
    size_t off = base;
    p.status_off = 0;
    if (base == 0) off = 256;
    p.hist_off = off;
    off = align256(off + (size_t)(hist + 1) * 4);
    p.part_off = off;
    off = align256(off + (size_t)(p.n_scan_blocks + 1) * 4);
    p.ids_off = off;
    off = align256(off + (size_t)ids * 4);
    p.tbl_off = off;
    off = align256(off + (size_t)tbl * 16);
    p.dtbl_off = 0;
    if (backward) {
        p.dtbl_off = off;
        off = align256(off + (size_t)tbl * 16);
    }
    p.rows_off = off;
    off = align256(off + (size_t)rows * 4);
    p.amp_off = off;
    off = align256(off + (size_t)rir * 4);
    if (prec == ISM_PREC_LUT_TEX) off = (off + 511) & ~(size_t)511;
    p.lut_off = off;
    off = align256(off + (size_t)lut * 4);
    p.gpart_off = off;
    off = align256(off + (size_t)p.gpart_total * 4);
    p.rgrad_off = off;
    off = align256(off + (size_t)p.rgrad_total * 4);
    p.env_off = off;
    off = align256(off + (size_t)p.env_total * 4);
    p.env_nodes_off = off;
    off = align256(off + (size_t)p.env_slots * ISM_ENV_SLOT * 16);
    p.total = off;
    return ISM_OK;
}

ism_status validate_all(const ism_job* jobs, int n_jobs, std::vector<Validated>& vs, bool need_ptrs)
{
    if (!jobs || n_jobs < 1) return fail(ISM_ERR_INVALID_ARG, "need at least one job");
    vs.resize(n_jobs);
    for (int i = 0; i < n_jobs; ++i) {
        ism_status s = validate_job(jobs[i], vs[i], need_ptrs);
        if (s != ISM_OK) {
            std::string m = g_last_error;
            return fail(s, "job %d: %s", i, m.c_str());
        }
    }
    return ISM_OK;
}

// Image sources in reach of one RIR of a job: the grid, or the sphere of
// radius n_ism + H samples (its volume over the room's), whichever is smaller.
double images_in_reach(const Validated& v)
{
    const ism_job& in = v.job;
    const double k = (double)in.fs / (double)in.room.c;
    const double reach = ((double)v.n_ism + v.H) / k;
    const double vol = in.room.L[0] * in.room.L[1] * in.room.L[2];
    return std::min((double)in.nb_img[0] * in.nb_img[1] * in.nb_img[2], 4.18879020478639 * reach * reach * reach / vol);
}

// Execution schedule of a forward call: launch sets (<= ISM_MAX_JOBS jobs
// each) and the lane (internal stream) of each.  A call with enough work is
// cut into two halves by source (or by receiver for one source) that run on
// two lanes, so that one half's enumeration overlaps the other half's
// accumulation; sets alternate between the lanes.  A sub-job keeps the
// RIR index of its first RIR (the noise counter), so every RIR is computed
// exactly as in the unsplit job.
struct Schedule {
    std::vector<std::vector<Validated>> sets;
    int lanes = 1;
};

std::atomic<int> g_lanes{2};

Schedule schedule(const std::vector<Validated>& vs)
{
    Schedule sc;
    double work = 0.0;
    for (const Validated& v : vs) work += images_in_reach(v) * (double)v.job.n_src * v.job.n_rcv;
    const bool split = work >= 2.0e7 && g_lanes.load() >= 2;
    std::vector<Validated> halves[2];
    for (const Validated& v : vs) {
        const ism_job& j = v.job;
        const bool by_src = j.n_src >= 2, by_rcv = j.n_src == 1 && j.n_rcv >= 2;
        if (!split || !(by_src || by_rcv)) {
            halves[0].push_back(v);
            continue;
        }
        const int n = by_src ? j.n_src : j.n_rcv;
        const int h = n / 2;
        for (int part = 0; part < 2; ++part) {
            Validated w = v;
            const int i0 = part == 0 ? 0 : h, cnt = part == 0 ? h : n - h;
            const long long stride = by_src ? (long long)j.n_rcv * v.n_S : (long long)v.n_S;   // out elements
            if (by_src) {
                w.job.pos_src = j.pos_src ? j.pos_src + 3 * i0 : nullptr;
                w.job.n_src = cnt;
                w.rir_index0 = v.rir_index0 + i0 * j.n_rcv;
                if (j.env_amp) w.job.env_amp = j.env_amp + (long long)i0 * j.n_rcv;
            } else {
                w.job.pos_rcv = j.pos_rcv ? j.pos_rcv + 3 * i0 : nullptr;
                w.job.orient_rcv = j.orient_rcv ? j.orient_rcv + 3 * i0 : nullptr;
                w.job.n_rcv = cnt;
                w.rir_index0 = v.rir_index0 + i0;
                if (j.env_amp) w.job.env_amp = j.env_amp + i0;
            }
            if (j.out) w.job.out = j.out + (long long)i0 * stride;
            halves[part].push_back(w);
        }
    }
    for (int part = 0; part < 2; ++part)
        for (size_t g = 0; g < halves[part].size(); g += ISM_MAX_JOBS) {
            const size_t e = std::min(halves[part].size(), g + ISM_MAX_JOBS);
            sc.sets.emplace_back(halves[part].begin() + g, halves[part].begin() + e);
        }
    sc.lanes = (sc.sets.size() >= 2 && g_lanes.load() >= 2) ? 2 : 1;
    return sc;
}

// Workspace of a schedule: lane 0's sets reuse [0, base1), lane 1's sets
// [base1, need); *base1_out receives base1.
ism_status schedule_size(const Schedule& sc, ism_precision prec, size_t* bytes, size_t* base1_out)
{
    JobTable t;
    WsPlan p;
    size_t size0 = 256, size1 = 0;
    for (size_t k = 0; k < sc.sets.size(); k += sc.lanes) {
        ism_status s = plan(sc.sets[k].data(), (int)sc.sets[k].size(), prec, false, t, p, 0);
        if (s != ISM_OK) return s;
        size0 = std::max(size0, p.total);
    }
    const size_t base1 = align256(size0);
    if (sc.lanes == 2)
        for (size_t k = 1; k < sc.sets.size(); k += 2) {
            ism_status s = plan(sc.sets[k].data(), (int)sc.sets[k].size(), prec, false, t, p, base1);
            if (s != ISM_OK) return s;
            size1 = std::max(size1, p.total - base1);
        }
    *bytes = base1 + size1;
    if (base1_out) *base1_out = base1;
    return ISM_OK;
}

ism_status batch_size(const std::vector<Validated>& vs, ism_precision prec, size_t* bytes, bool backward = false)
{
    if (!backward) return schedule_size(schedule(vs), prec, bytes, nullptr);
    size_t best = 0;
    JobTable t;
    WsPlan p;
    for (size_t g = 0; g < vs.size(); g += ISM_MAX_JOBS) {
        int n = (int)std::min<size_t>(ISM_MAX_JOBS, vs.size() - g);
        ism_status s = plan(vs.data() + g, n, prec, backward, t, p);
        if (s != ISM_OK) return s;
        if (p.total > best) best = p.total;
    }
    *bytes = best;
    return ISM_OK;
}

// The two internal streams (lanes) of the calling thread on the current
// device, with the events of the fork and the join; created on first use.
struct Lanes {
    int dev = -1;
    cudaStream_t s[2] = {nullptr, nullptr};
    cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
    ~Lanes()
    {
        for (int i = 0; i < 2; ++i) {
            if (s[i]) cudaStreamDestroy(s[i]);
            if (join[i]) cudaEventDestroy(join[i]);
        }
        if (fork) cudaEventDestroy(fork);
    }
};

int lanes_of_device(Lanes** out)
{
    thread_local std::vector<Lanes> all(64);
    int d = 0;
    int e = (int)cudaGetDevice(&d);
    if (e) return e;
    if (d < 0 || d >= 64) return (int)cudaErrorInvalidDevice;
    Lanes& L = all[d];
    if (L.dev != d) {
        for (int i = 0; i < 2; ++i) {
            if ((e = (int)cudaStreamCreateWithFlags(&L.s[i], cudaStreamNonBlocking))) return e;
            if ((e = (int)cudaEventCreateWithFlags(&L.join[i], cudaEventDisableTiming))) return e;
        }
        if ((e = (int)cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming))) return e;
        L.dev = d;
    }
    *out = &L;
    return 0;
}

// ---------------------------------------------------------------------------
// Per-stage timing: event pairs recorded on the caller's stream, resolved
// when ism_profile_read() is called.
// ---------------------------------------------------------------------------
struct Profiler {
    std::mutex mu;
    bool on = false;
    struct Pending {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    double ms[ISM_N_STAGES] = {};
    long long launches[ISM_N_STAGES] = {};
    long long calls[ISM_N_STAGES] = {};

    cudaEvent_t get()
    {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void resolve()
    {
        for (auto& p : pending) {
            cudaEventSynchronize(p.b);
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) ms[p.stage] += t;
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
    }
};

Profiler& profiler()
{
    static Profiler* p = new Profiler();
    return *p;
}

bool profiling_on()
{
    Profiler& P = profiler();
    std::lock_guard<std::mutex> g(P.mu);
    return P.on;
}

// Side stream of the calling thread on the current device, with the events that fork
// it from and join it back into a launch stream (the envelope kernels run there,
// beside the enumeration and the accumulation they do not depend on).
struct Side {
    int dev = -1;
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

int side_of_device(Side** out)
{
    thread_local std::vector<Side> all(64);
    int d = 0;
    int e = (int)cudaGetDevice(&d);
    if (e) return e;
    if (d < 0 || d >= 64) return (int)cudaErrorInvalidDevice;
    Side& S = all[d];
    if (S.dev != d) {
        if ((e = (int)cudaStreamCreateWithFlags(&S.s, cudaStreamNonBlocking))) return e;
        if ((e = (int)cudaEventCreateWithFlags(&S.fork, cudaEventDisableTiming))) return e;
        if ((e = (int)cudaEventCreateWithFlags(&S.join, cudaEventDisableTiming))) return e;
        S.dev = d;
    }
    *out = &S;
    return 0;
}

// Brackets one stage; a no-op unless profiling is on.
struct StageTimer {
    int stage;
    cudaStream_t s;
    bool on;
    cudaEvent_t a = nullptr;
    StageTimer(int st, cudaStream_t stream) : stage(st), s(stream)
    {
        Profiler& P = profiler();
        std::lock_guard<std::mutex> g(P.mu);
        on = P.on;
        if (on) {
            a = P.get();
            cudaEventRecord(a, s);
        }
    }
    void done(int launched)
    {
        if (!on) return;
        Profiler& P = profiler();
        std::lock_guard<std::mutex> g(P.mu);
        cudaEvent_t b = P.get();
        cudaEventRecord(b, s);
        P.pending.push_back({stage, a, b});
        P.launches[stage] += launched;
        P.calls[stage] += 1;
    }
};

// Texture objects over the windowed-sinc tables of the texture form: a 2-D
// pitched view (x = tap, y = phase) with linear filtering, created once per
// (device, table address, shape) and kept for the life of the process (a
// texture object must outlive every kernel that reads it; tables reuse the
// same workspace addresses from call to call, so the set stays small).
bool lut_texture(float* base, int row, int rows, unsigned long long* out)
{
    static std::mutex mu;
    static std::map<std::tuple<int, uintptr_t, int, int>, unsigned long long> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const auto key = std::make_tuple(dev, (uintptr_t)base, row, rows);
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *out = it->second;
        return true;
    }
    cudaResourceDesc rd;
    std::memset(&rd, 0, sizeof rd);
    rd.resType = cudaResourceTypePitch2D;
    rd.res.pitch2D.devPtr = base;
    rd.res.pitch2D.desc = cudaCreateChannelDesc<float>();
    rd.res.pitch2D.width = (size_t)row;
    rd.res.pitch2D.height = (size_t)rows;
    rd.res.pitch2D.pitchInBytes = (size_t)row * sizeof(float);
    cudaTextureDesc td;
    std::memset(&td, 0, sizeof td);
    td.addressMode[0] = td.addressMode[1] = cudaAddressModeClamp;
    td.filterMode = cudaFilterModeLinear;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;
    cudaTextureObject_t tex = 0;
    if (cudaCreateTextureObject(&tex, &rd, &td, nullptr) != cudaSuccess) return false;
    cache[key] = (unsigned long long)tex;
    *out = (unsigned long long)tex;
    return true;
}

// The launches of one launch set, in order, on `st`.
ism_status run_set(const std::vector<Validated>& set, ism_precision prec, size_t base, char* ws, cudaStream_t st)
{
    JobTable t;
    WsPlan p;
    ism_status s = plan(set.data(), (int)set.size(), prec, false, t, p, base);
    if (s != ISM_OK) return s;
    if (prec == ISM_PREC_LUT_TEX)
        for (int i = 0; i < t.n_jobs; ++i) {
            JobDev& J = t.j[i];
            float* tb = reinterpret_cast<float*>(ws + p.lut_off) + J.lut_base;
            if (!lut_texture(tb, 32 * J.slots, ism_lut_phases(J.slots) + 1, &J.lut_tex)) {
                cudaGetLastError();
                return fail(ISM_ERR_CUDA, "texture object over the windowed-sinc table of job %d", i);
            }
        }
    void* stream = (void*)st;
    int e;
    {
        StageTimer tm(ISM_STAGE_GEOMETRY, st);
        if ((e = ism_launch_geometry(t, p, ws, stream))) return cuda_fail(e, "geometry kernel");
        tm.done(p.rir_total > 0);
    }
    // envelope tables of Lehmann-Johansson tails (read by finalize and tail): on the side
    // stream, joined back before finalize (on the launch stream while profiling, so that
    // the stage times stay those of one stream)
    Side* side = nullptr;
    if (p.env_ctas > 0) {
        if (!profiling_on()) {
            if ((e = side_of_device(&side))) return cuda_fail(e, "internal stream");
            if ((e = (int)cudaEventRecord(side->fork, st))) return cuda_fail(e, "event record");
            if ((e = (int)cudaStreamWaitEvent(side->s, side->fork, 0))) return cuda_fail(e, "stream wait");
            if ((e = ism_launch_envelope(t, p, ws, (void*)side->s))) return cuda_fail(e, "envelope kernel");
            if ((e = (int)cudaEventRecord(side->join, side->s))) return cuda_fail(e, "event record");
        } else {
            StageTimer tm(ISM_STAGE_TAIL, st);
            if ((e = ism_launch_envelope(t, p, ws, stream))) return cuda_fail(e, "envelope kernel");
            tm.done(1);
        }
    }
    {
        StageTimer tm(ISM_STAGE_ENUM_COUNT, st);
        if ((e = ism_launch_enum(t, p, ws, false, stream))) return cuda_fail(e, "enumeration (count) kernel");
        tm.done(p.enum_ctas > 0);
    }
    if (p.hist_total > 0) {
        StageTimer tm(ISM_STAGE_SCAN, st);
        if ((e = ism_launch_scan(p, ws, stream))) return cuda_fail(e, "scan kernels");
        tm.done(3);
    }
    if (t.any_direct) {
        StageTimer tm(ISM_STAGE_ENUM_SCATTER, st);
        if ((e = ism_launch_enum(t, p, ws, true, stream))) return cuda_fail(e, "enumeration (scatter) kernel");
        tm.done(p.enum_ctas > 0);
    }
    {
        StageTimer tm(ISM_STAGE_ACCUM, st);
        int launched = 0;
        if (p.lut_total > 0) {
            if ((e = ism_launch_lut_tables(t, p, ws, stream))) return cuda_fail(e, "windowed-sinc table kernel");
            ++launched;
        }
        int acc_launched = 0;
        if ((e = ism_launch_accum(t, p, ws, prec, stream, &acc_launched))) return cuda_fail(e, "accumulation kernel");
        tm.done(launched + acc_launched);
    }
    if (side && (e = (int)cudaStreamWaitEvent(st, side->join, 0))) return cuda_fail(e, "stream wait");
    {
        StageTimer tm(ISM_STAGE_FINALIZE, st);
        if ((e = ism_launch_finalize(t, p, ws, stream))) return cuda_fail(e, "finalize kernel");
        tm.done(p.rir_total > 0);
    }
    if (p.tail_ctas > 0) {
        StageTimer tm(ISM_STAGE_TAIL, st);
        if ((e = ism_launch_tail(t, p, ws, stream))) return cuda_fail(e, "tail kernel");
        tm.done(1);
    }
    return ISM_OK;
}

// Copies of the results to host memory enqueued by run_batch: every job's
// output region of the device buffer starting at d_base goes to the same
// offset from h_base, on the stream that computed it, right after it.
struct HostCopy {
    const float* d_base;
    float* h_base;
};

int copy_set_out(const std::vector<Validated>& set, const HostCopy* hc, cudaStream_t s)
{
    for (const Validated& v : set) {
        const size_t n = (size_t)v.job.n_src * v.job.n_rcv * (size_t)v.n_S;
        const size_t off = (size_t)(v.job.out - hc->d_base);
        int e = (int)cudaMemcpyAsync(hc->h_base + off, v.job.out, n * sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e) return e;
    }
    return 0;
}

ism_status run_batch(const std::vector<Validated>& vs, ism_precision prec, void* workspace, size_t ws_bytes,
                     void* stream, const HostCopy* hc = nullptr)
{
    const Schedule sc = schedule(vs);
    size_t need = 0, base1 = 0;
    ism_status s = schedule_size(sc, prec, &need, &base1);
    if (s != ISM_OK) return s;
    if (!workspace) return fail(ISM_ERR_INVALID_ARG, "workspace is NULL");
    if (((uintptr_t)workspace & 255u) != 0) return fail(ISM_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < need)
        return fail(ISM_ERR_WORKSPACE_TOO_SMALL, "workspace of %zu bytes, need %zu", ws_bytes, need);
    char* ws = static_cast<char*>(workspace);
    cudaStream_t st = (cudaStream_t)stream;
    int e = (int)cudaMemsetAsync(ws, 0, 256, st);
    if (e) return cuda_fail(e, "status reset");
    if (sc.lanes == 1) {
        for (const auto& set : sc.sets)
            if ((s = run_set(set, prec, 0, ws, st)) != ISM_OK) return s;
        for (const auto& set : sc.sets)
            if (hc && (e = copy_set_out(set, hc, st))) return cuda_fail(e, "copy of the RIRs");
        return ISM_OK;
    }
    // two lanes forked from and joined back into the caller's stream; their
    // launches interleave on the GPU (the enumeration of one half, bound by
    // scattered stores, overlaps the arithmetic of the other)
    Lanes* L = nullptr;
    if ((e = lanes_of_device(&L))) return cuda_fail(e, "internal streams");
    if ((e = (int)cudaEventRecord(L->fork, st))) return cuda_fail(e, "event record");
    for (int i = 0; i < 2; ++i)
        if ((e = (int)cudaStreamWaitEvent(L->s[i], L->fork, 0))) return cuda_fail(e, "stream wait");
    ism_status first_err = ISM_OK;
    for (size_t k = 0; k < sc.sets.size() && first_err == ISM_OK; ++k) {
        const int lane = (int)(k % 2);
        first_err = run_set(sc.sets[k], prec, lane == 0 ? 0 : base1, ws, L->s[lane]);
    }
    // each half's results leave for the host on its own stream while the other half computes
    // (enqueued after every launch, so that a copy to pageable memory cannot hold up a launch)
    for (size_t k = 0; hc && k < sc.sets.size() && first_err == ISM_OK; ++k)
        if ((e = copy_set_out(sc.sets[k], hc, L->s[k % 2]))) first_err = cuda_fail(e, "copy of the RIRs");
    // join even after an error, so that the caller's stream orders after all work enqueued
    for (int i = 0; i < 2; ++i) {
        if ((e = (int)cudaEventRecord(L->join[i], L->s[i])) && first_err == ISM_OK) first_err = cuda_fail(e, "event");
        if ((e = (int)cudaStreamWaitEvent(st, L->join[i], 0)) && first_err == ISM_OK) first_err = cuda_fail(e, "wait");
    }
    return first_err;
}

// Backward pass: the forward's geometry; for 32-tap windows the fused
// Chebyshev adjoint (which enumerates its own images), for other windows the
// forward's enumeration and binning and the per-tap adjoint; then the
// fixed-order reductions.
ism_status run_backward(const std::vector<Validated>& vs, void* workspace, size_t ws_bytes, void* stream)
{
    size_t need = 0;
    ism_status s = batch_size(vs, ISM_PREC_FP32, &need, true);
    if (s != ISM_OK) return s;
    if (!workspace) return fail(ISM_ERR_INVALID_ARG, "workspace is NULL");
    if (((uintptr_t)workspace & 255u) != 0) return fail(ISM_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < need)
        return fail(ISM_ERR_WORKSPACE_TOO_SMALL, "workspace of %zu bytes, need %zu", ws_bytes, need);
    char* ws = static_cast<char*>(workspace);
    cudaStream_t st = (cudaStream_t)stream;
    int e = (int)cudaMemsetAsync(ws, 0, 256, st);
    if (e) return cuda_fail(e, "status reset");
    JobTable t;
    WsPlan p;
    for (size_t g = 0; g < vs.size(); g += ISM_MAX_JOBS) {
        int n = (int)std::min<size_t>(ISM_MAX_JOBS, vs.size() - g);
        s = plan(vs.data() + g, n, ISM_PREC_FP32, true, t, p);
        if (s != ISM_OK) return s;
        {
            StageTimer tm(ISM_STAGE_GEOMETRY, st);
            if ((e = ism_launch_geometry(t, p, ws, stream))) return cuda_fail(e, "geometry kernel");
            tm.done(p.rir_total > 0);
        }
        {
            StageTimer tm(ISM_STAGE_ENUM_COUNT, st);
            if ((e = ism_launch_enum(t, p, ws, false, stream))) return cuda_fail(e, "enumeration (count) kernel");
            tm.done(p.enum_ctas > 0);
        }
        if (p.hist_total > 0) {
            StageTimer tm(ISM_STAGE_SCAN, st);
            if ((e = ism_launch_scan(p, ws, stream))) return cuda_fail(e, "scan kernels");
            tm.done(3);
        }
        {
            StageTimer tm(ISM_STAGE_ENUM_SCATTER, st);
            if ((e = ism_launch_enum(t, p, ws, true, stream))) return cuda_fail(e, "enumeration (scatter) kernel");
            tm.done(p.enum_ctas > 0);
        }
        {
            StageTimer tm(ISM_STAGE_ADJOINT, st);
            int launched = 0;
            if ((e = ism_launch_adjoint(t, p, ws, stream, &launched))) return cuda_fail(e, "adjoint kernel");
            tm.done(launched);
        }
    }
    return ISM_OK;
}

ism_status validate_grad_jobs(const ism_grad_job* jobs, int n_jobs, std::vector<Validated>& vs)
{
    if (!jobs || n_jobs < 1) return fail(ISM_ERR_INVALID_ARG, "need at least one job");
    std::vector<ism_job> plain(n_jobs);
    for (int i = 0; i < n_jobs; ++i) plain[i] = jobs[i].job;
    ism_status s = validate_all(plain.data(), n_jobs, vs, false);
    if (s != ISM_OK) return s;
    for (int i = 0; i < n_jobs; ++i) {
        if (jobs[i].job.mic_pattern != ISM_MIC_OMNI)
            return fail(ISM_ERR_UNSUPPORTED, "job %d: gradients are for omnidirectional receivers only", i);
        if (!jobs[i].job.pos_src || !jobs[i].job.pos_rcv || !jobs[i].grad_out)
            return fail(ISM_ERR_INVALID_ARG, "job %d: pos_src, pos_rcv and grad_out must be device pointers", i);
        vs[i].grad_out = jobs[i].grad_out;
        vs[i].grad_beta = jobs[i].grad_beta;
        vs[i].grad_src = jobs[i].grad_src;
        vs[i].grad_rcv = jobs[i].grad_rcv;
    }
    return ISM_OK;
}

ism_job make_job(const ism_room* room, const float* pos_src, int n_src, const float* pos_rcv, int n_rcv,
                 const int nb_img[3], float Tmax, float fs, float Tdiff, float Tw, uint64_t seed, float* out)
{
    ism_job j;
    std::memset(&j, 0, sizeof j);
    if (room) j.room = *room;
    j.pos_src = pos_src;
    j.n_src = n_src;
    j.pos_rcv = pos_rcv;
    j.n_rcv = n_rcv;
    if (nb_img)
        for (int a = 0; a < 3; ++a) j.nb_img[a] = nb_img[a];
    j.Tmax = Tmax;
    j.fs = fs;
    j.Tdiff = Tdiff;
    j.Tw = Tw;
    j.seed = seed;
    j.out = out;
    j.env_amp = nullptr;
    return j;
}

ism_status check_prec(ism_precision prec)
{
    if (prec != ISM_PREC_FP32 && prec != ISM_PREC_FP16X2 && prec != ISM_PREC_BF16X2 && prec != ISM_PREC_LUT &&
        prec != ISM_PREC_FP32_DIRECT && prec != ISM_PREC_LUT_TEX)
        return fail(ISM_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    return ISM_OK;
}

}  // namespace

ism_status ism_fail_message(ism_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

// Launch graphs of repeated calls.  A call whose arguments match an earlier call's
// -- every argument but the values behind the pointers (positions, outputs) --
// replays the CUDA graph of that call's launches instead of building the job tables
// and the plan and issuing the dozen launches with their 32 KB parameter tables
// again.  The graph is captured (nothing runs while capturing) after a call ran
// eagerly: the host entry captures after its first call (when the kernels write its
// page-locked result themselves), ism_simulate_batch when a key comes back (so that
// a stream of distinct batches, as the server's, pays nothing but the key).  Calls
// on a stream being captured by the caller, calls
// while the stage profiler runs, and jobs with device-resident coefficients run
// eagerly.  At most HG_MAX graphs are kept (the least recently used one goes); the
// lookup and the launch hold one lock, so no thread destroys a graph another is
// about to launch.
namespace {
#define HG_MAX 16
#define HG_SEEN 32
struct HostGraph {
    std::string key;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    size_t pos_off = 0;   // host entry: where the positions go in the workspace
    unsigned long long tick = 0;
};
std::mutex g_hg_mu;
std::vector<HostGraph> g_hg;
std::vector<std::string> g_hg_seen;   // keys met once (ism_simulate_batch), most recent last
unsigned long long g_hg_tick = 0;

template <class T>
void key_put(std::string& k, const T& v)
{
    k.append(reinterpret_cast<const char*>(&v), sizeof v);
}

void key_room(std::string& k, const ism_room& r)
{
    for (int a = 0; a < 3; ++a) key_put(k, r.L[a]);
    for (int w = 0; w < 6; ++w) key_put(k, r.beta[w]);
    key_put(k, r.c);
}

std::string host_graph_key(int dev, const ism_room* room, int n_src, int n_rcv, const int nb_img[3], float Tmax,
                           float fs, float Tdiff, float Tw, ism_precision prec, uint64_t seed, const void* out_dev,
                           const void* workspace, size_t ws_bytes)
{
    std::string k("H");
    key_put(k, dev);
    key_room(k, *room);
    key_put(k, n_src);
    key_put(k, n_rcv);
    for (int a = 0; a < 3; ++a) key_put(k, nb_img[a]);
    key_put(k, Tmax);
    key_put(k, fs);
    key_put(k, Tdiff);
    key_put(k, Tw);
    key_put(k, (int)prec);
    key_put(k, seed);
    key_put(k, out_dev);
    key_put(k, workspace);
    key_put(k, ws_bytes);
    key_put(k, g_lanes.load());
    return k;
}

std::string batch_graph_key(int dev, const ism_job* jobs, int n, ism_precision prec, const void* workspace,
                            size_t ws_bytes)
{
    std::string k("B");
    key_put(k, dev);
    key_put(k, n);
    key_put(k, (int)prec);
    key_put(k, workspace);
    key_put(k, ws_bytes);
    key_put(k, g_lanes.load());
    for (int i = 0; i < n; ++i) {
        const ism_job& j = jobs[i];
        key_room(k, j.room);
        key_put(k, j.pos_src);
        key_put(k, j.n_src);
        key_put(k, j.pos_rcv);
        key_put(k, j.n_rcv);
        for (int a = 0; a < 3; ++a) key_put(k, j.nb_img[a]);
        key_put(k, j.Tmax);
        key_put(k, j.fs);
        key_put(k, j.Tdiff);
        key_put(k, j.Tw);
        key_put(k, j.seed);
        key_put(k, j.out);
        key_put(k, j.env_amp);
        key_put(k, j.mic_pattern);
        key_put(k, j.orient_rcv);
        key_put(k, j.envelope);
    }
    return k;
}

// capture stream of the calling thread on the current device
int capture_stream(cudaStream_t* out)
{
    thread_local std::vector<cudaStream_t> cs(64, nullptr);
    int d = 0;
    int e = (int)cudaGetDevice(&d);
    if (e) return e;
    if (d < 0 || d >= 64) return (int)cudaErrorInvalidDevice;
    if (!cs[d] && (e = (int)cudaStreamCreateWithFlags(&cs[d], cudaStreamNonBlocking))) return e;
    *out = cs[d];
    return 0;
}

// The graph of `key`, if one is kept: pre(pos_off) then its launch on `st`, under the
// lock.  Returns a CUDA error (0 when all went well); *hit tells whether it launched.
template <class Pre>
int hg_replay(const std::string& key, cudaStream_t st, Pre pre, bool* hit)
{
    *hit = false;
    std::lock_guard<std::mutex> g(g_hg_mu);
    for (HostGraph& h : g_hg) {
        if (h.key != key) continue;
        h.tick = ++g_hg_tick;
        int e = pre(h.pos_off);
        if (!e) e = (int)cudaGraphLaunch(h.x, st);
        *hit = e == 0;
        return e;
    }
    return 0;
}

// Whether a batch key came before (and remember it): the batch entry captures on the
// second sighting.
bool hg_seen_before(const std::string& key)
{
    std::lock_guard<std::mutex> g(g_hg_mu);
    for (size_t i = 0; i < g_hg_seen.size(); ++i)
        if (g_hg_seen[i] == key) {
            g_hg_seen.erase(g_hg_seen.begin() + (long)i);
            return true;
        }
    if (g_hg_seen.size() >= HG_SEEN) g_hg_seen.erase(g_hg_seen.begin());
    g_hg_seen.push_back(key);
    return false;
}

// Captures run(cs) on the thread's capture stream and keeps the graph under `key`.
// A capture that fails leaves nothing behind (the call's own result is not touched).
template <class Run>
void hg_store(const std::string& key, size_t pos_off, Run run)
{
    cudaStream_t cs = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    std::lock_guard<std::mutex> lk(g_hg_mu);
    if (capture_stream(&cs) == 0 && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const ism_status sc = run(cs);
        const cudaError_t ec = cudaStreamEndCapture(cs, &g);
        if (sc == ISM_OK && ec == cudaSuccess && g && cudaGraphInstantiate(&x, g, 0) == cudaSuccess) {
            if (g_hg.size() >= HG_MAX) {
                size_t old = 0;
                for (size_t i = 1; i < g_hg.size(); ++i)
                    if (g_hg[i].tick < g_hg[old].tick) old = i;
                cudaGraphExecDestroy(g_hg[old].x);
                cudaGraphDestroy(g_hg[old].g);
                g_hg.erase(g_hg.begin() + (long)old);
            }
            HostGraph h;
            h.key = key;
            h.g = g;
            h.x = x;
            h.pos_off = pos_off;
            h.tick = ++g_hg_tick;
            g_hg.push_back(h);
        } else if (g) {
            cudaGraphDestroy(g);
        }
    }
    cudaGetLastError();
    g_last_error.clear();
}
}  // namespace

extern "C" {

const char* ism_status_string(ism_status s)
{
    switch (s) {
    case ISM_OK: return "ISM_OK";
    case ISM_ERR_INVALID_ARG: return "ISM_ERR_INVALID_ARG";
    case ISM_ERR_INFEASIBLE: return "ISM_ERR_INFEASIBLE";
    case ISM_ERR_WORKSPACE_TOO_SMALL: return "ISM_ERR_WORKSPACE_TOO_SMALL";
    case ISM_ERR_OOM: return "ISM_ERR_OOM";
    case ISM_ERR_CUDA: return "ISM_ERR_CUDA";
    case ISM_ERR_TIMEOUT: return "ISM_ERR_TIMEOUT";
    case ISM_ERR_DEVICE_CHECK: return "ISM_ERR_DEVICE_CHECK";
    case ISM_ERR_UNSUPPORTED: return "ISM_ERR_UNSUPPORTED";
    case ISM_ERR_CANCELLED: return "ISM_ERR_CANCELLED";
    }
    return "ISM_ERR_UNKNOWN";
}

const char* ism_last_error_message(void) { return g_last_error.c_str(); }

int ism_version(void) { return ISM_VERSION; }

ism_status ism_rir_length(float T, float fs, int* n_samples)
{
    if (!n_samples) return fail(ISM_ERR_INVALID_ARG, "n_samples is NULL");
    if (!(T > 0.0f) || !(fs > 0.0f) || !isfin(T) || !isfin(fs))
        return fail(ISM_ERR_INVALID_ARG, "T and fs must be finite and > 0");
    *n_samples = rir_len(T, fs);
    return ISM_OK;
}

ism_status ism_workspace_size(const ism_room* room, int n_src, int n_rcv, const int nb_img[3], float Tmax, float fs,
                              float Tdiff, float Tw, ism_precision prec, size_t* bytes)
{
    g_last_error.clear();
    if (!room || !nb_img || !bytes) return fail(ISM_ERR_INVALID_ARG, "room, nb_img and bytes must not be NULL");
    ism_status s = check_prec(prec);
    if (s != ISM_OK) return s;
    ism_job j = make_job(room, nullptr, n_src, nullptr, n_rcv, nb_img, Tmax, fs, Tdiff, Tw, 0, nullptr);
    std::vector<Validated> vs;
    if ((s = validate_all(&j, 1, vs, false)) != ISM_OK) return s;
    return batch_size(vs, prec, bytes);
}

ism_status ism_batch_workspace_size(const ism_job* jobs, int n_jobs, ism_precision prec, size_t* bytes)
{
    g_last_error.clear();
    if (!bytes) return fail(ISM_ERR_INVALID_ARG, "bytes is NULL");
    ism_status s = check_prec(prec);
    if (s != ISM_OK) return s;
    std::vector<Validated> vs;
    if ((s = validate_all(jobs, n_jobs, vs, false)) != ISM_OK) return s;
    return batch_size(vs, prec, bytes);
}

ism_status ism_simulate_batch(const ism_job* jobs, int n_jobs, ism_precision prec, void* workspace, size_t ws_bytes,
                              void* stream)
{
    g_last_error.clear();
    ism_status s = check_prec(prec);
    if (s != ISM_OK) return s;
    // a call like an earlier one replays its launch graph (see hg_replay)
    cudaStream_t st = (cudaStream_t)stream;
    std::string gkey;
    bool cacheable = jobs && n_jobs >= 1 && workspace && !profiling_on();
    for (int i = 0; cacheable && i < n_jobs; ++i) cacheable = jobs[i].beta_dev == nullptr;
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    if (cacheable && (cudaStreamIsCapturing(st, &cst) != cudaSuccess || cst != cudaStreamCaptureStatusNone)) {
        cudaGetLastError();
        cacheable = false;
    }
    if (cacheable) {
        int dev = 0;
        int e = (int)cudaGetDevice(&dev);
        if (e) return cuda_fail(e, "current device");
        gkey = batch_graph_key(dev, jobs, n_jobs, prec, workspace, ws_bytes);
        bool hit = false;
        if ((e = hg_replay(gkey, st, [](size_t) { return 0; }, &hit))) return cuda_fail(e, "graph launch");
        if (hit) return ISM_OK;
    }
    std::vector<Validated> vs;
    if ((s = validate_all(jobs, n_jobs, vs, true)) != ISM_OK) return s;
    if ((s = run_batch(vs, prec, workspace, ws_bytes, stream)) != ISM_OK) return s;
    if (!gkey.empty() && hg_seen_before(gkey))
        hg_store(gkey, 0, [&](cudaStream_t cs) { return run_batch(vs, prec, workspace, ws_bytes, cs); });
    return ISM_OK;
}

ism_status ism_simulate(const ism_room* room, const float* pos_src, int n_src, const float* pos_rcv, int n_rcv,
                        const int nb_img[3], float Tmax, float fs, float Tdiff, float Tw, ism_precision prec,
                        uint64_t seed, float* out, void* workspace, size_t ws_bytes, void* stream)
{
    g_last_error.clear();
    if (!room || !nb_img) return fail(ISM_ERR_INVALID_ARG, "room and nb_img must not be NULL");
    ism_job j = make_job(room, pos_src, n_src, pos_rcv, n_rcv, nb_img, Tmax, fs, Tdiff, Tw, seed, out);
    return ism_simulate_batch(&j, 1, prec, workspace, ws_bytes, stream);
}

ism_status ism_backward_workspace_size(const ism_grad_job* jobs, int n_jobs, size_t* bytes)
{
    g_last_error.clear();
    if (!bytes) return fail(ISM_ERR_INVALID_ARG, "bytes is NULL");
    if (!jobs || n_jobs < 1) return fail(ISM_ERR_INVALID_ARG, "need at least one job");
    std::vector<ism_job> plain(n_jobs);
    for (int i = 0; i < n_jobs; ++i) {
        if (jobs[i].job.mic_pattern != ISM_MIC_OMNI)
            return fail(ISM_ERR_UNSUPPORTED, "job %d: gradients are for omnidirectional receivers only", i);
        plain[i] = jobs[i].job;
    }
    std::vector<Validated> vs;
    ism_status s = validate_all(plain.data(), n_jobs, vs, false);
    if (s != ISM_OK) return s;
    return batch_size(vs, ISM_PREC_FP32, bytes, true);
}

ism_status ism_simulate_backward_batch(const ism_grad_job* jobs, int n_jobs, void* workspace, size_t ws_bytes,
                                       void* stream)
{
    g_last_error.clear();
    std::vector<Validated> vs;
    ism_status s = validate_grad_jobs(jobs, n_jobs, vs);
    if (s != ISM_OK) return s;
    return run_backward(vs, workspace, ws_bytes, stream);
}

ism_status ism_simulate_backward(const ism_room* room, const float* pos_src, int n_src, const float* pos_rcv,
                                 int n_rcv, const int nb_img[3], float Tmax, float fs, float Tdiff, float Tw,
                                 const float* grad_out, float* grad_beta, float* grad_src, float* grad_rcv,
                                 void* workspace, size_t ws_bytes, void* stream)
{
    g_last_error.clear();
    if (!room || !nb_img) return fail(ISM_ERR_INVALID_ARG, "room and nb_img must not be NULL");
    ism_grad_job gj;
    std::memset(&gj, 0, sizeof gj);
    gj.job = make_job(room, pos_src, n_src, pos_rcv, n_rcv, nb_img, Tmax, fs, Tdiff, Tw, 0, nullptr);
    gj.grad_out = grad_out;
    gj.grad_beta = grad_beta;
    gj.grad_src = grad_src;
    gj.grad_rcv = grad_rcv;
    return ism_simulate_backward_batch(&gj, 1, workspace, ws_bytes, stream);
}

ism_status ism_simulate_host(const ism_room* room, const float* pos_src, int n_src, const float* pos_rcv, int n_rcv,
                             const int nb_img[3], float Tmax, float fs, float Tdiff, float Tw, ism_precision prec,
                             uint64_t seed, float* out, void* workspace, size_t ws_bytes, void* stream)
{
    g_last_error.clear();
    if (!room || !nb_img || !pos_src || !pos_rcv || !out)
        return fail(ISM_ERR_INVALID_ARG, "room, nb_img, positions and out must not be NULL");
    ism_status s = check_prec(prec);
    if (s != ISM_OK) return s;
    for (int i = 0; i < n_src; ++i)
        for (int a = 0; a < 3; ++a)
            if (!(pos_src[3 * i + a] > 0.0f && (double)pos_src[3 * i + a] < room->L[a]))
                return fail(ISM_ERR_INVALID_ARG, "source %d lies outside the room", i);
    for (int i = 0; i < n_rcv; ++i)
        for (int a = 0; a < 3; ++a)
            if (!(pos_rcv[3 * i + a] > 0.0f && (double)pos_rcv[3 * i + a] < room->L[a]))
                return fail(ISM_ERR_INVALID_ARG, "receiver %d lies outside the room", i);
    cudaStream_t st = (cudaStream_t)stream;
    int e;
    // a page-locked `out` is written by the kernels themselves (over the host link, as the
    // RIRs are finished); other host memory receives a copy of the device result
    // (its address on the current device, where the kernels run: memory pinned in another
    // device's context without the portable flag has none and takes the copy)
    cudaPointerAttributes attr{};
    void* dp = nullptr;
    const bool direct = cudaPointerGetAttributes(&attr, out) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
                        cudaHostGetDevicePointer(&dp, static_cast<void*>(out), 0) == cudaSuccess && dp != nullptr;
    cudaGetLastError();   // a pageable or foreign pointer leaves an error behind
    std::string gkey;
    if (direct && workspace && !profiling_on()) {
        int dev = 0;
        if ((e = (int)cudaGetDevice(&dev))) return cuda_fail(e, "current device");
        gkey = host_graph_key(dev, room, n_src, n_rcv, nb_img, Tmax, fs, Tdiff, Tw, prec, seed, dp, workspace,
                              ws_bytes);
        bool hit = false;
        e = hg_replay(gkey, st, [&](size_t pos_off) {
            float* d_pos = reinterpret_cast<float*>(static_cast<char*>(workspace) + pos_off);
            int r = (int)cudaMemcpyAsync(d_pos, pos_src, (size_t)n_src * 3 * sizeof(float), cudaMemcpyHostToDevice, st);
            if (!r)
                r = (int)cudaMemcpyAsync(d_pos + 3 * n_src, pos_rcv, (size_t)n_rcv * 3 * sizeof(float),
                                         cudaMemcpyHostToDevice, st);
            return r;
        }, &hit);
        if (e) return cuda_fail(e, "copy of the positions or graph launch");
        if (hit) {
            if ((e = (int)cudaStreamSynchronize(st))) return cuda_fail(e, "stream synchronize");
            return ISM_OK;
        }
    }
    ism_job j = make_job(room, nullptr, n_src, nullptr, n_rcv, nb_img, Tmax, fs, Tdiff, Tw, seed, nullptr);
    std::vector<Validated> vs;
    if ((s = validate_all(&j, 1, vs, false)) != ISM_OK) return s;
    size_t sim = 0;
    if ((s = batch_size(vs, prec, &sim)) != ISM_OK) return s;
    // device layout: [simulation workspace | positions | output]
    size_t pos_off = align256(sim);
    size_t out_off = align256(pos_off + (size_t)(n_src + n_rcv) * 3 * sizeof(float));
    size_t n_out = (size_t)n_src * n_rcv * (size_t)vs[0].n_S;
    size_t need = align256(out_off + n_out * sizeof(float));
    if (!workspace) return fail(ISM_ERR_INVALID_ARG, "workspace is NULL");
    if (ws_bytes < need)
        return fail(ISM_ERR_WORKSPACE_TOO_SMALL, "workspace of %zu bytes, need %zu (ism_host_workspace_size)",
                    ws_bytes, need);
    char* ws = static_cast<char*>(workspace);
    float* d_pos = reinterpret_cast<float*>(ws + pos_off);
    float* d_out = reinterpret_cast<float*>(ws + out_off);
    if ((e = (int)cudaMemcpyAsync(d_pos, pos_src, (size_t)n_src * 3 * sizeof(float), cudaMemcpyHostToDevice, st)))
        return cuda_fail(e, "copy of source positions");
    if ((e = (int)cudaMemcpyAsync(d_pos + 3 * n_src, pos_rcv, (size_t)n_rcv * 3 * sizeof(float),
                                  cudaMemcpyHostToDevice, st)))
        return cuda_fail(e, "copy of receiver positions");
    vs[0].job.pos_src = d_pos;
    vs[0].job.pos_rcv = d_pos + 3 * n_src;
    vs[0].job.out = d_out;
    vs[0].job.seed = seed;
    if (direct) vs[0].job.out = static_cast<float*>(dp);
    const HostCopy hc{d_out, out};
    if ((s = run_batch(vs, prec, workspace, sim, stream, direct ? nullptr : &hc)) != ISM_OK) return s;
    if ((e = (int)cudaStreamSynchronize(st))) return cuda_fail(e, "stream synchronize");
    // capture this call's launches for the next identical one
    if (!gkey.empty())
        hg_store(gkey, pos_off, [&](cudaStream_t cs) { return run_batch(vs, prec, workspace, sim, cs, nullptr); });
    return ISM_OK;
}

ism_status ism_host_workspace_size(const ism_room* room, int n_src, int n_rcv, const int nb_img[3], float Tmax,
                                   float fs, float Tdiff, float Tw, ism_precision prec, size_t* bytes)
{
    size_t sim = 0;
    ism_status s = ism_workspace_size(room, n_src, n_rcv, nb_img, Tmax, fs, Tdiff, Tw, prec, &sim);
    if (s != ISM_OK) return s;
    int n_S = rir_len(Tmax, fs);
    size_t pos_off = align256(sim);
    size_t out_off = align256(pos_off + (size_t)(n_src + n_rcv) * 3 * sizeof(float));
    *bytes = align256(out_off + (size_t)n_src * n_rcv * (size_t)n_S * sizeof(float));
    return ISM_OK;
}

ism_status ism_workspace_status(const void* workspace, void* stream, uint32_t* flags)
{
    g_last_error.clear();
    if (!workspace || !flags) return fail(ISM_ERR_INVALID_ARG, "workspace and flags must not be NULL");
    uint32_t v = 0;
    int e;
    if ((e = (int)cudaMemcpyAsync(&v, workspace, sizeof v, cudaMemcpyDeviceToHost, (cudaStream_t)stream)))
        return cuda_fail(e, "status read");
    if ((e = (int)cudaStreamSynchronize((cudaStream_t)stream))) return cuda_fail(e, "stream synchronize");
    *flags = v;
    return ISM_OK;
}

ism_status ism_diffuse_noise(uint64_t seed, uint32_t rir, uint32_t k0, int n, float* z, void* stream)
{
    g_last_error.clear();
    if (n < 0 || (n > 0 && !z)) return fail(ISM_ERR_INVALID_ARG, "need n >= 0 and a device buffer");
    if ((unsigned long long)k0 + (unsigned long long)n > 0xFFFFFFFFull)
        return fail(ISM_ERR_INVALID_ARG, "sample range exceeds 2^32");
    int e = ism_launch_noise(seed, rir, k0, n, z, stream);
    if (e) return cuda_fail(e, "noise kernel");
    return ISM_OK;
}

ism_status ism_auralize(const float* signal, int n_x, const float* rirs, int n_points, int n_mics, int n_S,
                        const int* starts, float* out, void* stream)
{
    g_last_error.clear();
    if (!signal || !rirs || !out) return fail(ISM_ERR_INVALID_ARG, "signal, rirs and out must be device pointers");
    if (n_x < 1 || n_points < 1 || n_mics < 1 || n_S < 1)
        return fail(ISM_ERR_INVALID_ARG, "need n_x, n_points, n_mics, n_S >= 1");
    if ((long long)n_x + n_S - 1 > 0x7FFFFFFFll || (long long)n_points * n_mics * (long long)n_S > (1ll << 40))
        return fail(ISM_ERR_UNSUPPORTED, "signal or RIRs too long");
    if (n_points > n_x) return fail(ISM_ERR_INVALID_ARG, "more trajectory points (%d) than samples (%d)", n_points, n_x);
    int e = ism_launch_auralize(signal, n_x, rirs, n_points, n_mics, n_S, starts, out, stream);
    if (e) return cuda_fail(e, "auralization kernel");
    return ISM_OK;
}

// Operation counts deciding the automatic choice of ism_auralize_ex: the
// direct form does n_mics n_x n_S multiply-adds; the FFT form about 4 N log2 N
// lane operations per length-N DFT (one per segment, one per microphone pair
// and point, one inverse per pair) and 4 per product of spectra.  Measured on
// the 48 kHz array's filtering, the direct form runs 2.55 times as many of its
// units per second as the FFT form of its own (20.5 T multiply-adds/s against
// 8.0 T operations/s), so the FFT form is taken above that ratio.
static bool auralize_fft_pays(int n_x, int n_points, int n_mics, int n_S)
{
    const long long n_out = (long long)n_x + n_S - 1;
    int logN = 4;
    while ((1ll << logN) < n_out) ++logN;
    if (logN > 20) return false;
    const double N = (double)(1ll << logN);
    const double pairs = (double)((n_mics + 1) / 2);
    const double fft = ((double)n_points * (1.0 + pairs) + pairs) * 4.0 * N * logN + (double)n_points * pairs * 4.0 * N;
    const double direct = (double)n_mics * (double)n_x * (double)n_S;
    return direct > 2.55 * fft;
}

static ism_status auralize_args(const float* signal, int n_x, const float* rirs, int n_points, int n_mics, int n_S,
                                float* out)
{
    if (!signal || !rirs || !out) return fail(ISM_ERR_INVALID_ARG, "signal, rirs and out must be device pointers");
    if (n_x < 1 || n_points < 1 || n_mics < 1 || n_S < 1)
        return fail(ISM_ERR_INVALID_ARG, "need n_x, n_points, n_mics, n_S >= 1");
    if ((long long)n_x + n_S - 1 > 0x7FFFFFFFll || (long long)n_points * n_mics * (long long)n_S > (1ll << 40))
        return fail(ISM_ERR_UNSUPPORTED, "signal or RIRs too long");
    if (n_points > n_x) return fail(ISM_ERR_INVALID_ARG, "more trajectory points (%d) than samples (%d)", n_points, n_x);
    return ISM_OK;
}

ism_status ism_auralize_workspace_size(int n_x, int n_points, int n_mics, int n_S, int method, size_t* bytes)
{
    g_last_error.clear();
    if (!bytes) return fail(ISM_ERR_INVALID_ARG, "bytes must not be NULL");
    *bytes = 0;
    if (n_x < 1 || n_points < 1 || n_mics < 1 || n_S < 1)
        return fail(ISM_ERR_INVALID_ARG, "need n_x, n_points, n_mics, n_S >= 1");
    if (method < ISM_AURALIZE_AUTO || method > ISM_AURALIZE_FFT)
        return fail(ISM_ERR_INVALID_ARG, "method = %d is not an ism_auralize_method", method);
    const bool fft = method == ISM_AURALIZE_FFT ||
                     (method == ISM_AURALIZE_AUTO && auralize_fft_pays(n_x, n_points, n_mics, n_S));
    if (!fft) return ISM_OK;
    AfPlan pl;
    size_t need = 0;
    if (ism_auralize_fft_plan(n_x, n_points, n_mics, n_S, 0, &pl, &need))
        return fail(ISM_ERR_UNSUPPORTED, "output of %lld samples exceeds the FFT form's 2^20",
                    (long long)n_x + n_S - 1);
    *bytes = need;
    return ISM_OK;
}

ism_status ism_auralize_ex(const float* signal, int n_x, const float* rirs, int n_points, int n_mics, int n_S,
                           const int* starts, float* out, int method, void* workspace, size_t ws_bytes, void* stream)
{
    g_last_error.clear();
    ism_status st = auralize_args(signal, n_x, rirs, n_points, n_mics, n_S, out);
    if (st != ISM_OK) return st;
    if (method < ISM_AURALIZE_AUTO || method > ISM_AURALIZE_FFT)
        return fail(ISM_ERR_INVALID_ARG, "method = %d is not an ism_auralize_method", method);
    bool fft = method == ISM_AURALIZE_FFT;
    AfPlan pl;
    size_t need = 0;
    if (method == ISM_AURALIZE_AUTO && auralize_fft_pays(n_x, n_points, n_mics, n_S) && workspace &&
        ism_auralize_fft_plan(n_x, n_points, n_mics, n_S, ws_bytes, &pl, &need) == 0)
        fft = true;
    if (fft) {
        if (!workspace) return fail(ISM_ERR_INVALID_ARG, "the FFT form needs a workspace");
        if (((uintptr_t)workspace & 255u) != 0) return fail(ISM_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
        const int r = ism_auralize_fft_plan(n_x, n_points, n_mics, n_S, ws_bytes, &pl, &need);
        if (r == -1)
            return fail(ISM_ERR_UNSUPPORTED, "output of %lld samples exceeds the FFT form's 2^20",
                        (long long)n_x + n_S - 1);
        if (r == -2)
            return fail(ISM_ERR_WORKSPACE_TOO_SMALL, "workspace of %zu bytes holds no chunk of the FFT form", ws_bytes);
        int e = ism_launch_auralize_fft(signal, rirs, starts, out, pl, static_cast<char*>(workspace), stream);
        if (e) return cuda_fail(e, "auralization (FFT) kernels");
        return ISM_OK;
    }
    int e = ism_launch_auralize(signal, n_x, rirs, n_points, n_mics, n_S, starts, out, stream);
    if (e) return cuda_fail(e, "auralization kernel");
    return ISM_OK;
}

ism_status ism_t60_sabine(const double L[3], const double beta[6], double* T60)
{
    g_last_error.clear();
    if (!L || !beta || !T60) return fail(ISM_ERR_INVALID_ARG, "NULL argument");
    for (int a = 0; a < 3; ++a)
        if (!(L[a] > 0.0)) return fail(ISM_ERR_INVALID_ARG, "room size must be > 0");
    double t = t60_of(L, beta);
    if (!std::isfinite(t)) return fail(ISM_ERR_INFEASIBLE, "no absorption: T60 is infinite");
    *T60 = t;
    return ISM_OK;
}

ism_status ism_beta_sabine(const double L[3], double T60, const double abs_weights[6], int negative,
                           double beta_out[6])
{
    g_last_error.clear();
    if (!L || !beta_out) return fail(ISM_ERR_INVALID_ARG, "NULL argument");
    for (int a = 0; a < 3; ++a)
        if (!(L[a] > 0.0) || !isfin(L[a])) return fail(ISM_ERR_INVALID_ARG, "room size must be > 0");
    if (!(T60 > 0.0) || !isfin(T60)) return fail(ISM_ERR_INVALID_ARG, "T60 must be > 0");
    double S[6] = {L[1] * L[2], L[1] * L[2], L[0] * L[2], L[0] * L[2], L[0] * L[1], L[0] * L[1]};
    double w[6], sw = 0.0;
    for (int i = 0; i < 6; ++i) {
        w[i] = abs_weights ? abs_weights[i] : 1.0;
        if (!(w[i] >= 0.0) || !isfin(w[i])) return fail(ISM_ERR_INVALID_ARG, "absorption weights must be >= 0");
        sw += S[i] * w[i];
    }
    if (!(sw > 0.0)) return fail(ISM_ERR_INFEASIBLE, "all absorption weights are zero");
    double a0 = 0.161 * L[0] * L[1] * L[2] / (T60 * sw);
    for (int i = 0; i < 6; ++i)
        if (w[i] * a0 >= 1.0)
            return fail(ISM_ERR_INFEASIBLE, "T60 = %g s needs absorption %g >= 1 on wall %d", T60, w[i] * a0, i);
    for (int i = 0; i < 6; ++i) {
        double b = std::sqrt(1.0 - w[i] * a0);
        beta_out[i] = negative ? -b : b;
    }
    return ISM_OK;
}

ism_status ism_beta_sabine_device(const double* L, const double* T60, const double* abs_weights, int negative, int n,
                                  double* beta_out, int* status, void* stream)
{
    g_last_error.clear();
    if (n < 0 || (n > 0 && (!L || !T60 || !beta_out || !status)))
        return fail(ISM_ERR_INVALID_ARG, "need n >= 0 and device buffers");
    int e = ism_launch_beta_sabine(L, T60, abs_weights, negative, n, beta_out, status, stream);
    if (e) return cuda_fail(e, "Sabine kernel");
    return ISM_OK;
}

ism_status ism_nb_img_from_t(double T, const double L[3], double c, double Tw, int nb_out[3])
{
    g_last_error.clear();
    if (!L || !nb_out) return fail(ISM_ERR_INVALID_ARG, "NULL argument");
    if (!(T >= 0.0) || !isfin(T)) return fail(ISM_ERR_INVALID_ARG, "T must be >= 0");
    if (!(c > 0.0)) c = 343.0;
    if (!(Tw > 0.0)) Tw = 4e-3;
    double R = c * (T + 0.5 * Tw);
    for (int a = 0; a < 3; ++a) {
        if (!(L[a] > 0.0)) return fail(ISM_ERR_INVALID_ARG, "room size must be > 0");
        double M = std::ceil(R / L[a]) + 1.0;
        if (2.0 * M + 1.0 > 1e9) return fail(ISM_ERR_UNSUPPORTED, "image grid too large");
        nb_out[a] = (int)(2.0 * M + 1.0);
    }
    return ISM_OK;
}

ism_status ism_set_lanes(int n_lanes)
{
    g_last_error.clear();
    if (n_lanes != 1 && n_lanes != 2) return fail(ISM_ERR_INVALID_ARG, "n_lanes must be 1 or 2");
    g_lanes.store(n_lanes);
    return ISM_OK;
}

ism_status ism_profile_enable(int enable)
{
    g_last_error.clear();
    Profiler& P = profiler();
    std::lock_guard<std::mutex> g(P.mu);
    P.on = enable != 0;
    return ISM_OK;
}

ism_status ism_profile_reset(void)
{
    g_last_error.clear();
    Profiler& P = profiler();
    std::lock_guard<std::mutex> g(P.mu);
    P.resolve();
    for (int i = 0; i < ISM_N_STAGES; ++i) {
        P.ms[i] = 0.0;
        P.launches[i] = 0;
        P.calls[i] = 0;
    }
    return ISM_OK;
}

ism_status ism_profile_read(int stage, double* total_ms, long long* launches, long long* calls)
{
    g_last_error.clear();
    if (stage < 0 || stage >= ISM_N_STAGES) return fail(ISM_ERR_INVALID_ARG, "stage %d out of range", stage);
    Profiler& P = profiler();
    std::lock_guard<std::mutex> g(P.mu);
    P.resolve();
    if (total_ms) *total_ms = P.ms[stage];
    if (launches) *launches = P.launches[stage];
    if (calls) *calls = P.calls[stage];
    return ISM_OK;
}

ism_status ism_att2t_sabine(double att_dB, double T60, double* t)
{
    g_last_error.clear();
    if (!t) return fail(ISM_ERR_INVALID_ARG, "NULL argument");
    if (!(T60 > 0.0) || !isfin(att_dB)) return fail(ISM_ERR_INVALID_ARG, "T60 must be > 0");
    *t = att_dB / 60.0 * T60;
    return ISM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of ism_simulate.
//
// Some callers cannot allocate device memory at the point where they need a
// simulation: code running inside a real-time audio callback or another
// library's worker thread that must not block on the allocator, code that
// runs under a framework owning every device allocation (and forbidding raw
// cudaMalloc), or small embedded uses that cannot size and keep a workspace.
// For them the library reserves one fixed scratch area in device memory at
// module load (a file-scope __device__ array) and runs the ordinary
// simulation in it.  Every device that loads the library holds this area
// until the process exits.
// ---------------------------------------------------------------------------
#define ISM_NOALLOC_SCRATCH_BYTES (64u << 20)

static __device__ __align__(256) unsigned char g_ism_noalloc_scratch[ISM_NOALLOC_SCRATCH_BYTES];

namespace {

#define ISM_NOALLOC_MAX_DEVICES 64
std::mutex g_noalloc_mu;
void* g_noalloc_addr[ISM_NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch area for the current device; looked up once
// per device (host code only sees a stand-in symbol, never the address).
ism_status noalloc_scratch(void** out)
{
    int dev = -1;
    int e = (int)cudaGetDevice(&dev);
    if (e) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= ISM_NOALLOC_MAX_DEVICES)
        return fail(ISM_ERR_UNSUPPORTED, "device %d is beyond the %d devices this entry point serves", dev,
                    ISM_NOALLOC_MAX_DEVICES);
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = (int)cudaGetSymbolAddress(&p, g_ism_noalloc_scratch);
        if (e) return cuda_fail(e, "cudaGetSymbolAddress of the scratch area");
        if (!p) return fail(ISM_ERR_CUDA, "scratch area has no device address");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return ISM_OK;
}

}  // namespace

extern "C" ism_status ism_simulate_noalloc(const ism_room* room, const float* pos_src, int n_src,
                                           const float* pos_rcv, int n_rcv, const int nb_img[3], float Tmax,
                                           float fs, float Tdiff, float Tw, ism_precision prec, uint64_t seed,
                                           float* out, void* stream)
{
    g_last_error.clear();
    if (!room || !nb_img) return fail(ISM_ERR_INVALID_ARG, "room and nb_img must not be NULL");
    ism_status s = check_prec(prec);
    if (s != ISM_OK) return s;
    ism_job j = make_job(room, pos_src, n_src, pos_rcv, n_rcv, nb_img, Tmax, fs, Tdiff, Tw, seed, out);
    std::vector<Validated> vs;
    if ((s = validate_all(&j, 1, vs, true)) != ISM_OK) return s;
    size_t need = 0;
    if ((s = batch_size(vs, prec, &need)) != ISM_OK) return s;
    if (need > ISM_NOALLOC_SCRATCH_BYTES)
        return fail(ISM_ERR_UNSUPPORTED,
                    "this simulation needs %zu bytes of scratch, above the %u bytes of the allocation-free "
                    "entry point; use ism_simulate with a caller-owned workspace",
                    need, (unsigned)ISM_NOALLOC_SCRATCH_BYTES);
    void* scratch = nullptr;
    if ((s = noalloc_scratch(&scratch)) != ISM_OK) return s;
    return run_batch(vs, prec, scratch, ISM_NOALLOC_SCRATCH_BYTES, stream);
}
