// ism_internal.h -- definitions shared by the translation units of libism.
//
// The simulation of a batch of jobs (one job = one room with its source and
// receiver sets) runs as a fixed sequence of launches, all ordered on the
// caller's stream:
//
//   geometry  per RIR and axis: image offsets squared in samples^2 (FP64 ->
//             float-float) and wall-reflection products (Section 2.1, eq. (1),
//             eq. (4)); checks the positions.
//   enum(a)   per RIR and range of grid columns: delays of the images in
//             reach (eq. (2)-(3)), culling of those whose window misses
//             [0, n_ism), counts per 32-sample delay bin.
//   scan(b)   exclusive prefix over the counts: bin offsets (counting sort).
//   enum(a')  the same walk, scattering packed image ids into their bins in
//             a fixed order (stable counting sort).
//   accum(c)  one CTA per (RIR, ISM_ACC_BPC delay bins), one warp per bin:
//             the windowed sinc (eq. (6)) of every image of the bin into a
//             register window, stored as the bin's window row.
//   finalize  per RIR: each sample is the sum of the rows of the bins that
//             cover it, in bin order (eq. (5)); fits the envelope amplitude
//             of the diffuse tail (Section 2.2).
//   tail(d)   Philox4x32-10 logistic noise times the envelope of eq. (8).
//
// No floating-point atomic is used anywhere: every sum has a fixed order, so
// the output is bit-identical from run to run.
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/ism.h"

#define ISM_SB 32                 // samples per delay bin
#define ISM_ACC_BPC 4             // delay bins per accumulation CTA (one warp each)
#define ISM_TILE_SAMPLES 256      // samples per adjoint tile (CTA)
#define ISM_TILE_BINS (ISM_TILE_SAMPLES / ISM_SB)   // 8 bins per adjoint tile
#define ISM_ACC_WARPS ISM_TILE_BINS                 // adjoint: one warp per bin
#define ISM_ENUM_WARPS 4          // warps per enumeration CTA (one unit each)
#define ISM_MAX_JOBS 64           // jobs per launch set (kernel-parameter table, < 32 KB)
#define ISM_MAX_AXIS 1023         // images per axis (10-bit packed ids)
#define ISM_MAX_SLOTS 8           // taps per lane per image: N_w <= 256
#define ISM_MAX_NISM 131000       // image-source samples per RIR
#define ISM_MAX_Q 4104            // delay bins per RIR ((n_ism + H) / 32 + 1)
#define ISM_SCAN_BLOCK 4096       // elements per scan block
#define ISM_SCAN_TOP 16384        // max scan blocks (one top-level block)
#define ISM_FIT_WINDOW_S 0.02     // envelope fit: last 20 ms of the ISM part
#define ISM_CHEB_N 9              // Chebyshev terms of a tap function in the adjoint (degree 8); table stride
#define ISM_CHEB_NF 8             // Chebyshev terms of the forward's moments (degree 7)
#define ISM_SHELL_BINS 8          // delay bins per CTA of the fused Chebyshev accumulation
#define ISM_SD_BINS 32            // delay bins per CTA of the fused direct accumulation
#define ISM_FILL_CTAS 304         // fused CTAs a launch set should have at least (two per SM of a GB300)

// Device-side description of one job.  Everything the kernels need is here
// so that a whole launch set takes its jobs as one kernel parameter.
struct JobDev {
    double L[3];
    float beta[6];
    const float* beta_dev;    // reflection coefficients in device memory (NULL: beta)
    double g2_c;              // 6 log2(10): numerator of g2 (device-side T60)
    float c, fs, Nw;          // Nw = Tw * fs taps (real)
    float kfs_hi, kfs_lo;     // fs / c as a float-float pair
    float amp_scale;          // (fs / c) / (4 pi): A = F / (4 pi d) = F * amp_scale / s
    float s_cut2;             // cull: keep an image iff s_plain^2 < s_cut2 (samples^2)
    float g2;                 // log2 of the power decay per sample: 6 log2(10) / (fs T60)
    int N[3], nlo[3];         // images per axis, lowest index per axis
    int n_src, n_rcv, n_rir;
    int n_S, n_ism;
    int H;                    // ceil(Nw / 2): taps j in [-H + 1, H]
    int slots;                // ceil(2H / 32) taps per lane per image
    int Q;                    // delay bins per RIR
    int U;                    // enumeration units (warps) per RIR
    int cols_per_unit;        // grid columns (ix, iy) per enumeration unit
    float inv_kLz;            // 1 / ((f_s / c) L_z): samples -> z cells
    float inv2L[3];           // 1 / (2 L) per axis (rounded from FP64 on the host: no FP64 in the kernels)
    float kinv;               // c / f_s: metres per sample
    float Lmax, vol;          // longest side, volume (FP32)
    int acc_groups;           // accumulation CTAs per RIR (groups of ISM_ACC_BPC bins)
    int fin_chunk;            // samples per finalize CTA (>= the envelope-fit window)
    int fin_chunks;           // finalize CTAs per RIR (chunk 0 holds the last samples)
    int n_tiles;              // adjoint tiles (8 bins) per RIR
    int has_tail;
    int W_env;                // samples of the envelope fit window
    int vec4;                 // out rows 16-byte aligned (float4 stores allowed)
    float half_scale;         // FP16X2 records are scaled by this power of two
    int use_cheb;             // FP32 accumulation through Chebyshev moments (32-tap window)
    int shell_groups;         // fused Chebyshev CTAs per RIR (ISM_SHELL_BINS bins each; 0 otherwise)
    int sparse;               // direct FP32 form, few images per bin: no sort, each image's taps added at once
    int adj_cheb;             // backward: fused Chebyshev adjoint (32-tap window; shell_groups CTAs per RIR)
    int rir_index0;           // RIR index of the job's first RIR in its caller's job (noise counter)
    uint64_t seed;
    const float* pos_src;
    const float* pos_rcv;
    const float* orient_rcv;  // receiver orientations [n_rcv][3] (polar pattern jobs)
    float mic_alpha;          // polar pattern g = alpha + (1 - alpha) cos(theta); 1: omnidirectional
    float* out;
    float* env_amp;
    long long img_per_rir;    // N[0] N[1] N[2]
    long long rir_base;       // global RIR index of the job's first RIR
    long long hist_base;      // first counter of the job in the histogram (direct jobs)
    long long tbl_base;       // first table entry (float4) of the job
    long long enum_cta_base;  // first enumeration CTA of the job
    long long acc_cta_base;   // first accumulation CTA of the job
    long long shell_rir_base; // first RIR of the job among the launch set's fused RIRs
    long long shell_cta_base; // first fused CTA of the job (job-major order)
    long long adj_cta_base;   // first adjoint CTA of the job
    long long tail_cta_base;  // first tail CTA of the job
    long long fin_cta_base;   // first finalize CTA of the job
    long long rows_base;      // first window row (float) of the job: [n_rir][Q][32 (slots + 1)]
    // (the fields above keep their places: the register allocation of the fused kernels
    // follows the layout of what they read; the ones below are read elsewhere)
    unsigned long long lut_tex;  // texture object over the job's windowed-sinc table (texture form)
    // backward pass only
    const float* grad_out;    // dLoss/dh [n_rir][n_S]
    float* grad_beta;         // [6]
    float* grad_src;          // [n_src][3]
    float* grad_rcv;          // [n_rcv][3]
    int gpart_base;           // first per-(RIR, bin) gradient record (x 12 floats); below 2^31
    int rgrad_base;           // first per-RIR gradient (float; 12 per RIR)
    int lut_base;             // first entry (float) of the job's windowed-sinc table (LUT forms)
    // diffuse tail
    float g2_lo;              // low part of g2 (g2 + g2_lo is the FP64 value to ~2^-48)
    int envelope;             // ISM_ENVELOPE_SABINE or ISM_ENVELOPE_LJ
    int env_k0;               // first sample of the job's envelope table (n_ism - W_env)
    int env_base;             // first entry (float) of the job's envelope table [n_S - env_k0]
    int env_cta_base;         // first envelope CTA of the job
    // fused direct form (a 32-tap window, every tap evaluated, images enumerated per shell)
    int shell_direct;         // its bins per CTA (0: not this form)
    int sd_cta_base;          // first CTA of the job in its launch (shell_groups CTAs per RIR)
    int env_slot;             // the job's slot of envelope quadrature nodes (Lehmann-Johansson tails)
    int sd_rir_base;          // first RIR of the job among the launch set's fused direct RIRs
};

struct JobTable {
    int n_jobs;
    int max_Q;
    int max_axis_sum;
    int any_cheb;                      // some job accumulates through Chebyshev moments
    int any_direct;                    // some job reads delay-binned image ids
    int shell_gmax;                    // most shells of a fused RIR
    int shell_rank_major;              // fused CTAs ordered by shell rank (shell_gmax x shell_rirs) or by job
    int sd_rank_rirs;                  // fused direct CTAs ordered by shell rank over this many RIRs (0: by job)
    long long shell_rirs;              // RIRs of the fused jobs
    float cheb[32 * ISM_CHEB_N];       // Chebyshev coefficients of the 32 tap functions (32-tap window)
    JobDev j[ISM_MAX_JOBS];
    int shell_bins;                    // delay bins per CTA of the fused Chebyshev forward (<= ISM_SHELL_BINS)
};

static_assert(sizeof(JobTable) <= 32000, "the job table is passed as one kernel parameter");

// Workspace carve-up of one launch set (byte offsets into the workspace).
struct WsPlan {
    size_t status_off;     // uint32 flags (first 256 bytes)
    size_t hist_off;       // uint32 [hist_total + 1]: per (RIR, bin, unit) counts -> offsets
    size_t part_off;       // uint32 [n_scan_blocks + 1]
    size_t ids_off;        // uint32 [ids_total]
    size_t tbl_off;        // float4 [tbl_total]
    size_t dtbl_off;       // float4 [tbl_total] (backward): dF/dbeta_lo, dF/dbeta_hi, d x_n / d x_s per axis index
    size_t rows_off;       // float  [rows_total]: per-bin window rows of the accumulation
    size_t amp_off;        // float  [rir_total]
    size_t lut_off;        // float  [lut_total]: polyphase windowed-sinc tables (LUT form)
    size_t gpart_off;      // float  [gpart_total]: backward, per-(RIR, bin) gradients
    size_t rgrad_off;      // float  [rgrad_total]: backward, per-RIR gradients
    size_t env_off;        // float  [env_total]: per-job envelope tables (Lehmann-Johansson tails)
    size_t env_nodes_off;  // float4 [env_slots][ISM_ENV_SLOT]: their quadrature nodes and E(t0)
    size_t total;
    long long hist_total;
    long long ids_total;
    long long tbl_total;
    long long rows_total;
    long long rir_total;
    long long lut_total;
    long long gpart_total;
    long long rgrad_total;
    long long env_total;
    long long env_ctas;
    long long env_slots;
    long long n_scan_blocks;
    long long enum_ctas;
    long long acc_ctas;
    long long shell_ctas;
    long long sd_ctas;     // CTAs of the fused direct form (shell_direct jobs)
    long long adj_ctas;
    long long tail_ctas;
    long long fin_ctas;
};

#define ISM_TAIL_CHUNK 4096   // tail samples per CTA (256 threads x 16)
#define ISM_ENV_CHUNK 64      // envelope-table samples per CTA (four threads each)
#define ISM_ENV_MAX_NODES 64  // Gauss-Legendre nodes per angle of the envelope integral
#define ISM_ENV_SLOT (ISM_ENV_MAX_NODES * ISM_ENV_MAX_NODES + 1)   // float4 per job: nodes, then {n, E(t0)}

// Delay bins (warps) per accumulation CTA: the LUT form copies its ~33 KB
// table into shared memory once per CTA, so it takes 8 bins per CTA.
__host__ __device__ constexpr int ism_acc_bins(int prec) { return prec == 3 ? 8 : ISM_ACC_BPC; }

// Phases per sample of the polyphase windowed-sinc table of the LUT form
// (eq. (9)): 256 for windows of up to 32 taps, fewer for longer windows so
// that a table of (Q + 1) x 32 SLOTS FP32 entries stays at ~33 KB of shared
// memory.
__host__ __device__ constexpr int ism_lut_phases(int slots)
{
    return slots <= 1 ? 256 : slots == 2 ? 128 : slots <= 4 ? 64 : 32;
}

// Plan of the FFT form of the moving-source filtering (ism_auralize_fft.cu).
struct AfPlan {
    int N, logN, R, logR, C, logC;   // DFT length N = R C (powers of two)
    int n_x, P, M, n_S, n_out, n_pairs;
    int pc;             // trajectory points per chunk
    int cb;             // columns per CTA, column pass
    int cb3;            // columns per CTA, inverse column pass
    int rb;             // rows per CTA, row pass
    int npg;            // microphone pairs per CTA of the row pass
    int n_pg;           // microphone-pair groups of the row pass
    int n_grp;          // point groups of the row pass (partial spectra summed in group order)
};

// Sets the calling thread's ism_last_error_message() and returns s.
ism_status ism_fail_message(ism_status s, const char* fmt, ...);

// Launch entry points (implemented in the .cu files, called by ism_api.cu).
// Each returns 0 or a cudaError_t value.
int ism_launch_geometry(const JobTable& t, const WsPlan& p, char* ws, void* stream);
int ism_launch_enum(const JobTable& t, const WsPlan& p, char* ws, bool scatter, void* stream);
int ism_launch_scan(const WsPlan& p, char* ws, void* stream);
int ism_launch_accum(const JobTable& t, const WsPlan& p, char* ws, ism_precision prec, void* stream,
                     int* launched);
int ism_launch_accum_fp16(const JobTable& t, const WsPlan& p, char* ws, void* stream, int* launched);
int ism_launch_accum_bf16(const JobTable& t, const WsPlan& p, char* ws, void* stream, int* launched);
int ism_launch_accum_lut(const JobTable& t, const WsPlan& p, char* ws, void* stream, int* launched);
int ism_launch_accum_tex(const JobTable& t, const WsPlan& p, char* ws, void* stream, int* launched);
int ism_launch_lut_tables(const JobTable& t, const WsPlan& p, char* ws, void* stream);
int ism_launch_accum_cheb(const JobTable& t, const WsPlan& p, char* ws, void* stream, int* launched);
int ism_launch_accum_shell_direct(const JobTable& t, const WsPlan& p, char* ws, ism_precision prec, void* stream,
                                  int* launched);
int ism_launch_adjoint(const JobTable& t, const WsPlan& p, char* ws, void* stream, int* launched);
int ism_launch_adjoint_cheb(const JobTable& t, const WsPlan& p, char* ws, void* stream, int* launched);
int ism_launch_finalize(const JobTable& t, const WsPlan& p, char* ws, void* stream);
int ism_launch_tail(const JobTable& t, const WsPlan& p, char* ws, void* stream);
int ism_launch_envelope(const JobTable& t, const WsPlan& p, char* ws, void* stream);
int ism_launch_noise(uint64_t seed, uint32_t rir, uint32_t k0, int n, float* z, void* stream);
int ism_launch_auralize(const float* x, int n_x, const float* h, int n_points, int n_mics, int n_s, const int* starts,
                        float* y, void* stream);
int ism_auralize_fft_plan(int n_x, int n_points, int n_mics, int n_S, size_t ws_bytes, AfPlan* out, size_t* need);
int ism_launch_auralize_fft(const float* x, const float* h, const int* starts, float* y, const AfPlan& pl, char* ws,
                            void* stream);
int ism_launch_beta_sabine(const double* L, const double* T60, const double* w, int negative, int n,
                           double* beta_out, int* status, void* stream);
