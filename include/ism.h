/*
 * ism.h -- C ABI of libism, a GB300 (sm_103a) implementation of the
 * image-source method (ISM) for room impulse responses (RIRs) in shoebox
 * rooms, after Diaz-Guerra, Miguel and Beltran, "gpuRIR: A Python Library for
 * Room Impulse Response Simulation with GPU Acceleration".
 *
 * What the library computes (paper Section 2):
 *   For every (source, receiver) pair and every image n of the grid
 *   ceil(-N/2) <= n < ceil(N/2) per axis (Section 2.1):
 *     image position       eq. (1)
 *     distance, delay      eq. (2), eq. (3)   tau_n = d_n / c
 *     amplitude            eq. (4)            A_n = beta_n / (4 pi d_n)
 *   and accumulates Peterson's Hann-windowed sinc (eq. (6), cut-off f_s/2)
 *   of every image into the RIR (eq. (5)).  Beyond Tdiff the RIR is a
 *   logistic-noise tail with the Sabine power envelope (Section 2.2, eq. (7),
 *   eq. (8) read as a 60 dB decay over T60).
 *
 * Conventions shared by every call:
 *   - No call allocates device memory on the simulation path: the caller
 *     passes a device workspace whose size the matching *_workspace_size call
 *     returns.  Pointers are borrowed for the duration of the work.  (The
 *     launch graphs kept for repeated calls -- see ism_simulate_batch and
 *     ism_simulate_host -- hold the driver's own memory for their executable
 *     form; the allocation-free entry point keeps none.)
 *   - "device" pointers are CUDA device (or managed) memory of the current
 *     device; "host" pointers are ordinary host memory.
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL is
 *     the legacy default stream) and the call returns after the launches:
 *     results are ready when the stream reaches that point.  Apart from
 *     ism_simulate_host, ism_workspace_status and the server's waits, no call
 *     waits for the device, and internal streams fork from and join back into
 *     `stream` through events, so the device-pointer calls can be captured in
 *     a CUDA graph on `stream` (once each kernel has been launched outside a
 *     capture) and replayed.
 *   - Every call returns an ism_status.  No C++ exception crosses the ABI.
 *     On an error the outputs are not written; ism_last_error_message()
 *     describes the last error of the calling thread.
 *   - Sample counts: n_S = ceil(Tmax fs (1 - 1e-6)), n_ism = ceil(Tdiff fs (1 - 1e-6))
 *     (the relative slack absorbs the FP32 rounding of the times).
 *     Tdiff <= 0 or Tdiff >= Tmax means no diffuse tail (n_ism = n_S).
 *   - The window length Tw is in seconds (eq. (6)); N_w = Tw fs taps.
 *     Tw <= 0 selects the paper's typical 4 ms.
 *   - The library keeps per-device state for the life of the process: the
 *     kernels' raised shared-memory limits, two internal streams and three
 *     events per host thread and device, texture objects of the LUT tables
 *     and the allocation-free entry point's scratch address.  It does not
 *     survive cudaDeviceReset() or the release of a device's primary
 *     context; after either, use it from a new process.
 */
#ifndef ISM_H
#define ISM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ISM_VERSION 101

typedef enum {
    ISM_OK = 0,
    ISM_ERR_INVALID_ARG = 1,          /* argument out of its documented range           */
    ISM_ERR_INFEASIBLE = 2,           /* Sabine: some alpha >= 1, or sum S alpha = 0    */
    ISM_ERR_WORKSPACE_TOO_SMALL = 3,  /* ws_bytes below the *_workspace_size result     */
    ISM_ERR_OOM = 4,                  /* allocation failed / HBM budget exceeded        */
    ISM_ERR_CUDA = 5,                 /* a CUDA runtime call failed                     */
    ISM_ERR_TIMEOUT = 6,              /* a host-side wait ran out of time               */
    ISM_ERR_DEVICE_CHECK = 7,         /* the device reported bad input (see status)     */
    ISM_ERR_UNSUPPORTED = 8,          /* valid but outside this build's limits          */
    ISM_ERR_CANCELLED = 9             /* a served request was cancelled                 */
} ism_status;

/* Arithmetic of the windowed-sinc evaluation (Section 3.5 LUT, Section 3.6
 * mixed precision).  Image enumeration, distances and delays are always
 * FP32 (with a float-float delay, so fractional delays keep FP32 accuracy);
 * accumulation is always FP32.
 *   ISM_PREC_FP32: for a window of exactly 32 taps, the windowed sinc of tap
 *   j as a function of the fractional delay f, delta'(j - f), is expanded in
 *   Chebyshev polynomials of 2f - 1 (degree 7, error < 4.3e-7 of the image's
 *   amplitude); the images of a delay bin that share their integer offset
 *   are summed as 8 moments sum A T_i(2f - 1), each term rounded to a
 *   fixed-point integer with a step of 2^-23 of the bin's largest possible
 *   amplitude and summed exactly (so the result does not depend on the
 *   order of the images), and each offset's moments are expanded once into
 *   the 32 taps.  Other windows use the direct evaluation of
 *   ISM_PREC_FP32_DIRECT. */
typedef enum {
    ISM_PREC_FP32 = 0,        /* FP32, Chebyshev moments (32-tap windows), else direct */
    ISM_PREC_FP16X2 = 1,      /* packed FP16 window and sinc, FP32 accumulation        */
    ISM_PREC_BF16X2 = 2,      /* packed BF16 window and sinc, FP32 accumulation; BF16's
                               * 8-bit significand bounds its error only to ~1e-2 of
                               * the peak (the other reduced forms: 2e-3)            */
    ISM_PREC_LUT = 3,         /* FP32 windowed-sinc table (eq. (9)), FP32 lerp         */
    ISM_PREC_FP32_DIRECT = 4, /* FP32 sin/cos/reciprocal for every image tap (eq. (6)) */
    ISM_PREC_LUT_TEX = 5      /* the same table read through the texture unit with its
                               * hardware linear filtering (8-bit weights), as in the
                               * paper's LUT kernel (Section 3.5)                    */
} ism_precision;

/* A shoebox room (Section 2.1).  beta is ordered x0, x1, y0, y1, z0, z1:
 * x0 is the wall x = 0 (closest to the origin), x1 the wall x = L[0].
 * Negative coefficients are allowed (Section 2.2). */
typedef struct {
    double L[3];      /* room size in metres, each > 0                         */
    float beta[6];    /* reflection coefficients, |beta| <= 1                  */
    float c;          /* speed of sound in m/s, > 0 (343 if <= 0 is passed)    */
} ism_room;

/* ------------------------------------------------------------------------- */
/* Status and errors                                                          */
/* ------------------------------------------------------------------------- */
/* Static string naming a status code. */
const char* ism_status_string(ism_status s);
/* Message of the last failed call on the calling thread ("" if none).  The
 * pointer stays valid until the next library call on this thread. */
const char* ism_last_error_message(void);
/* ISM_VERSION of the loaded library. */
int ism_version(void);

/* ------------------------------------------------------------------------- */
/* Sizing                                                                     */
/* ------------------------------------------------------------------------- */
/* n_samples = ceil(T fs (1 - 1e-6)).  T > 0, fs > 0.  Host only. */
ism_status ism_rir_length(float T, float fs, int* n_samples);

/* Device workspace bytes that ism_simulate needs for these arguments (same
 * meaning as in ism_simulate).  Host only; no device work. */
ism_status ism_workspace_size(const ism_room* room, int n_src, int n_rcv, const int nb_img[3],
                              float Tmax, float fs, float Tdiff, float Tw, ism_precision prec,
                              size_t* bytes);

/* ------------------------------------------------------------------------- */
/* Forward simulation (the library call of Section 4: the room, its walls'   */
/* coefficients, the positions, the image counts, the RIR length, the switch */
/* time to the diffuse model and the sampling rate -> a 3-D tensor)          */
/* ------------------------------------------------------------------------- */
/* RIRs for all n_src x n_rcv pairs.
 *   room      host, see ism_room.
 *   pos_src   device, [n_src][3] FP32 metres; pos_rcv device, [n_rcv][3].
 *             Positions must lie strictly inside the room.  They live on the
 *             device, so they are checked there: a pair with a position
 *             outside the room, or with source == receiver, gets an all-zero
 *             RIR and raises a flag that ism_workspace_status() returns.
 *   nb_img    host, images per axis in the paper's units (Section 2.1),
 *             each in [1, 1023]; ism_nb_img_from_t() picks them from a time.
 *   Tmax      RIR length in seconds; Tdiff start of the diffuse tail (see
 *             the conventions above); Tw window length (eq. (6)).
 *   prec      windowed-sinc arithmetic (ism_precision).
 *   seed      key of the Philox4x32-10 noise of the diffuse tail; the noise
 *             of RIR r = i_src * n_rcv + i_rcv, sample k is word k mod 4 of
 *             Philox4x32-10(counter (k/4, r, 0, 0), key (seed lo, seed hi)).
 *   out       device, [n_src][n_rcv][n_S] FP32 row-major, written entirely.
 *   workspace device, >= ism_workspace_size() bytes, 256-byte aligned; its
 *             contents need no initialisation and are scratch afterwards
 *             (except the status word read by ism_workspace_status()).
 * Limits (ISM_ERR_UNSUPPORTED beyond them): N_w = Tw fs <= 256 taps,
 * n_ism <= 131000 samples, images per axis <= 1023.
 * The result is bit-identical from run to run for identical arguments
 * (no floating-point atomics; fixed summation orders). */
ism_status ism_simulate(const ism_room* room, const float* pos_src, int n_src, const float* pos_rcv,
                        int n_rcv, const int nb_img[3], float Tmax, float fs, float Tdiff, float Tw,
                        ism_precision prec, uint64_t seed, float* out, void* workspace,
                        size_t ws_bytes, void* stream);

/* Same computation from HOST buffers: copies pos_src/pos_rcv to the device,
 * runs ism_simulate and delivers the RIRs into host `out`
 * ([n_src][n_rcv][n_S] FP32): a page-locked `out` is written by the kernels
 * directly over the host link, any other host memory receives a copy of the
 * device result.  Positions are validated on the host first
 * (ISM_ERR_INVALID_ARG if one lies outside the room).  Synchronous: returns
 * when `out` holds the result.  The workspace is device memory as above.
 * Repeated calls: when `out` is page-locked (and the stage profiler is off), a
 * call whose arguments other than the positions' values -- room, counts,
 * nb_img, times, fs, prec, seed, `out`, workspace and its size, the device and
 * the ism_set_lanes() setting -- equal an earlier call's replays a CUDA graph
 * of that call's launches, captured once after it ran (the positions are copied
 * into the workspace first, as always): bit-identical results, without the
 * planning and the per-launch parameter copies.  The library keeps the 16 most
 * recently used graphs (each holds its launches' 32 KB job tables); they hold the
 * workspace and `out` addresses, so freeing either and calling again with the
 * same addresses is fine, and per-device state ends with cudaDeviceReset. */
ism_status ism_simulate_host(const ism_room* room, const float* pos_src, int n_src,
                             const float* pos_rcv, int n_rcv, const int nb_img[3], float Tmax,
                             float fs, float Tdiff, float Tw, ism_precision prec, uint64_t seed,
                             float* out, void* workspace, size_t ws_bytes, void* stream);

/* Device workspace bytes that ism_simulate_host needs: the ism_simulate
 * workspace followed by room for the positions and the RIRs. */
ism_status ism_host_workspace_size(const ism_room* room, int n_src, int n_rcv, const int nb_img[3],
                                   float Tmax, float fs, float Tdiff, float Tw, ism_precision prec,
                                   size_t* bytes);

/* Reads the device status word a previous call left in `workspace`
 * (synchronises `stream`).  *flags = 0 if the inputs were valid, otherwise a
 * bitwise OR of ISM_DEVICE_FLAG_* values. */
#define ISM_DEVICE_FLAG_POSITION 1u   /* a source/receiver outside the room or coincident */
#define ISM_DEVICE_FLAG_BIN 2u        /* an image delay fell outside its bin (internal)    */
#define ISM_DEVICE_FLAG_BETA 4u       /* a reflection coefficient read from device memory
                                         (ism_job.beta_dev) was not finite or had |beta| > 1 */
ism_status ism_workspace_status(const void* workspace, void* stream, uint32_t* flags);

/* Same computation as ism_simulate without a workspace argument, for callers
 * that cannot allocate device memory (a real-time audio callback or a
 * worker thread that must not block on the allocator, code inside a
 * framework that owns every device allocation, embedded uses that cannot
 * keep a workspace).  The paper has no counterpart: it is a deployment
 * variant of the same launches, with bitwise the same results.
 *   Scratch: a fixed 64 MiB area in device memory (a file-scope __device__
 *   array of the library); every device on which it has been set up holds it
 *   until the process exits.  This entry point never calls cudaMalloc or
 *   cudaFree.
 *   Set-up, once per device: the first call on a device looks up the area's
 *   device address (cudaGetSymbolAddress) with that device current.  With
 *   CUDA's lazy module loading (the default) that lookup is also when the
 *   driver loads the library's device code and reserves the 64 MiB, so the
 *   first call on each device can block, and can fail (ISM_ERR_CUDA, e.g.
 *   out of memory); later calls cannot fail that way.  The first call whose
 *   simulation is large enough to run as two halves (see ism_set_lanes) also
 *   creates, once per host thread and device, two internal streams and three
 *   events.  A real-time caller should therefore make one warm-up call at
 *   set-up on each device and each host thread it will call from, outside
 *   its real-time path, and before any stream capture.
 *   Limit: a simulation needing more scratch than 64 MiB (ism_workspace_size)
 *   is rejected with ISM_ERR_UNSUPPORTED and nothing is launched.
 *   Sharing: every call uses the same area and leaves its contents behind;
 *   the kernels reset what they need.  Two calls whose work overlaps on the
 *   GPU (different streams without ordering between them, or different host
 *   threads) race on the area and corrupt each other's results: order them.
 *   Checks: the device-side flags of ism_workspace_status live in the area,
 *   whose address callers never see, so they are not reported here: a source
 *   or receiver outside the room, or a source on a receiver, silently gives
 *   an all-zero RIR.  Callers of this entry point range-check their device
 *   positions themselves.
 * Arguments, layout and errors are otherwise those of ism_simulate. */
ism_status ism_simulate_noalloc(const ism_room* room, const float* pos_src, int n_src,
                                const float* pos_rcv, int n_rcv, const int nb_img[3], float Tmax,
                                float fs, float Tdiff, float Tw, ism_precision prec, uint64_t seed,
                                float* out, void* stream);

/* ------------------------------------------------------------------------- */
/* Ragged batches: many rooms in one set of launches                         */
/* ------------------------------------------------------------------------- */
/* Receiver polar patterns and orientations (Section 4 lists them among the
 * inputs of the library call).  The paper gives no formula; the
 * first-order family g(theta) = alpha + (1 - alpha) cos(theta) is used, theta
 * being the angle between the receiver's orientation and the direction from
 * the receiver to the image source; g multiplies the image's amplitude
 * (eq. (4)).  alpha: OMNI 1, SUBCARDIOID 3/4, CARDIOID 1/2, HYPERCARDIOID
 * 1/4, BIDIRECTIONAL 0. */
typedef enum {
    ISM_MIC_OMNI = 0,
    ISM_MIC_SUBCARDIOID = 1,
    ISM_MIC_CARDIOID = 2,
    ISM_MIC_HYPERCARDIOID = 3,
    ISM_MIC_BIDIRECTIONAL = 4
} ism_mic_pattern;

/* Power envelope of the diffuse tail (Section 2.2).
 *   ISM_ENVELOPE_SABINE: eq. (7)-(8), P(t) = A 10^(-6 (t - t0) / T60).
 *   ISM_ENVELOPE_LJ: the energy-decay prediction of Lehmann and Johansson,
 *   which Section 2.2 cites as the more faithful alternative.  The paper
 *   gives no formula; the one used is the energy arrival rate of the image
 *   sources of the shoebox: images have density 1/V, an image at distance r
 *   in direction u has met the walls of axis a about r |u_a| / L_a times
 *   (half of them each wall), so the energy arriving at time t follows
 *     E(t) = (1 / 4 pi) oint prod_a |beta_a0 beta_a1|^(c t |u_a| / L_a) dOmega
 *   and P(t) = A E(t) / E(t0).  It is a sum of exponentials: for equal
 *   coefficients its initial slope is Eyring's decay rate, and with unequal
 *   walls it follows the images' own energy decay where the Sabine
 *   exponential does not.  The integral is evaluated once per job on the
 *   GPU (Gauss-Legendre product rule over one octant, 16 to 64 nodes per
 *   angle chosen from c Tmax sum_a -ln|beta_a0 beta_a1| / L_a; relative
 *   quadrature error below 1e-9 while that exponent stays below 300).
 * In both, A is fitted to the last 20 ms of the image-source part (their
 * power brought forward to t0 along the envelope), and the noise is the same
 * bit-exact Philox stream. */
typedef enum {
    ISM_ENVELOPE_SABINE = 0,
    ISM_ENVELOPE_LJ = 1
} ism_envelope;

/* One independent simulation.  Meanings as in ism_simulate; pos_src,
 * pos_rcv, out and env_amp are device pointers.  env_amp may be NULL; if
 * not, it receives [n_src * n_rcv] FP32 envelope amplitudes A (eq. (8)) of
 * the diffuse tail (0 where there is no tail).  mic_pattern (an
 * ism_mic_pattern, 0 = omnidirectional) applies to every receiver of the
 * job; orient_rcv, required unless the pattern is omnidirectional, is a
 * device pointer to [n_rcv][3] FP32 orientation vectors (any non-zero
 * length; a zero vector is flagged ISM_DEVICE_FLAG_POSITION).  A zero-filled
 * job struct is omnidirectional.  The gradient calls accept only
 * omnidirectional jobs (ISM_ERR_UNSUPPORTED otherwise).
 * beta_dev (may be NULL): a device pointer to the job's 6 reflection
 * coefficients (the order of room.beta).  When set, the kernels read the
 * coefficients there and room.beta is ignored, so a caller whose
 * coefficients live on the GPU (an optimiser updating them) needs no copy to
 * the host and no synchronisation; they are checked on the device (a
 * non-finite value or |beta| > 1 flags ISM_DEVICE_FLAG_BETA and the job's
 * pairs get no image), and the Sabine T60 of the diffuse tail (eq. (7)) is
 * computed on the device with the host's FP64 operations, so the results are
 * bitwise those of the same coefficients in room.beta.  Not accepted by the
 * server (whose jobs are host-side).
 * envelope: the ism_envelope of the diffuse tail (a zero-filled job uses
 * Sabine's); ignored when the job has no tail. */
typedef struct {
    ism_room room;
    const float* pos_src;
    int n_src;
    const float* pos_rcv;
    int n_rcv;
    int nb_img[3];
    float Tmax, fs, Tdiff, Tw;
    uint64_t seed;
    float* out;
    float* env_amp;
    int mic_pattern;
    const float* orient_rcv;
    const float* beta_dev;
    int envelope;             /* an ism_envelope (0: Sabine) */
} ism_job;

/* Workspace bytes for ism_simulate_batch over these jobs. */
ism_status ism_batch_workspace_size(const ism_job* jobs, int n_jobs, ism_precision prec,
                                    size_t* bytes);

/* Simulates every job (host array `jobs`, n_jobs >= 1).  Each job's result is
 * the same as a separate ism_simulate call with the same arguments, bit for
 * bit: the jobs share launches, not arithmetic.
 * Repeated calls: a call whose jobs, precision, workspace (address and size),
 * device and ism_set_lanes() setting equal a recent call's -- the same
 * pointers, whatever the values behind them -- replays a CUDA graph of that
 * call's launches, captured (without running) after the second such call: the
 * same results without the planning and the per-launch parameter copies.  Not
 * on a stream the caller is capturing (the launches are then captured as
 * usual), not while the stage profiler runs, not for jobs with beta_dev.  The
 * graphs share the host entry's store of 16. */
ism_status ism_simulate_batch(const ism_job* jobs, int n_jobs, ism_precision prec, void* workspace,
                              size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------- */
/* Serving: continuous batching of RIR requests                              */
/* ------------------------------------------------------------------------- */
/* A request loop for RIR generation on one GPU (the paper has no serving
 * layer; each request is one ism_job, computed exactly as ism_simulate would).
 * The server holds one device allocation of `hbm_budget` bytes and one pinned
 * host allocation of `host_budget` bytes for its whole life, and carves every
 * request's positions and RIRs and every batch's workspace out of them.  A
 * launcher thread takes queued requests in arrival order and admits them into
 * a batch while memory and a stream are free (up to max_batch requests), then
 * runs the batch (ism_simulate_batch) on its own stream: up to max_inflight
 * batches run on the GPU at once, so requests arriving while others are on
 * the GPU start as soon as memory and a stream free up.  A completer thread
 * retires finished batches, copies each result to its caller's buffer, frees
 * the memory and wakes the launcher.  A request is computed with the same
 * arithmetic whatever batch it lands in: its RIRs are bit-identical alone and
 * in any mix. */
typedef struct ism_server ism_server;
typedef uint64_t ism_ticket;

typedef struct {
    size_t hbm_budget;    /* device bytes the server allocates at create (>= 16 MiB)   */
    size_t host_budget;   /* pinned host bytes for staging (0: hbm_budget / 4)        */
    int max_inflight;     /* batches on the GPU at once, one stream each (0: 3; <= 16) */
    int max_batch;        /* requests per batch (0: 32; <= 256)                       */
    int device;           /* CUDA device ordinal                                      */
    ism_precision prec;   /* tap arithmetic of every request                          */
} ism_server_config;

typedef struct {
    long long submitted, completed, failed, batches;
    size_t dev_in_use, dev_peak, host_in_use;
    int inflight, queued;
    int inflight_peak;    /* most batches seen on the GPU at once */
} ism_server_stats;

/* Creates a server (allocates its two pools, two threads and its streams).
 * ISM_ERR_OOM if the pools cannot be allocated, ISM_ERR_CUDA without a device. */
ism_status ism_server_create(const ism_server_config* cfg, ism_server** server);

/* Queues one request.  job->pos_src and job->pos_rcv are HOST pointers, copied
 * before this returns; job->out is a HOST pointer of n_src * n_rcv * n_S FP32
 * that the server writes before the request is reported done (it must stay
 * valid until then; page-locked memory is written by the kernels directly
 * over the host link, other memory through a device buffer and the
 * server's staging pool);
 * job->env_amp must be NULL.  The job is validated here
 * (arguments as for ism_simulate, positions strictly inside the room):
 * errors return at once and no ticket is issued.  A request whose memory can
 * never fit the budget is rejected with ISM_ERR_OOM. */
ism_status ism_server_submit(ism_server* server, const ism_job* job, ism_ticket* ticket);

/* Queues n_jobs requests in one call (jobs[k] as for ism_server_submit;
 * tickets: n_jobs entries).  Every job is checked before any is queued: on an
 * error nothing is queued and the message names the job.  The requests enter
 * the queue together, in array order, with one submission time. */
ism_status ism_server_submit_batch(ism_server* server, const ism_job* jobs, int n_jobs, ism_ticket* tickets);

/* *done = 1 if the request has finished (successfully or not), else 0. */
ism_status ism_server_poll(ism_server* server, ism_ticket ticket, int* done);

/* Waits up to timeout_s seconds (< 0: no limit) for the request.  Returns
 * ISM_ERR_TIMEOUT if it is still running (the ticket stays valid); otherwise
 * the request's own status (ISM_OK, or the error that failed it, or
 * ISM_ERR_CANCELLED) and releases the ticket.  latency_s (may be NULL)
 * receives the time from submission to the result being in job->out. */
ism_status ism_server_wait(ism_server* server, ism_ticket ticket, double timeout_s, double* latency_s);

/* Counters and memory use. */
ism_status ism_server_stats_read(ism_server* server, ism_server_stats* stats);

/* Finishes the batches already on the GPU, cancels the queued requests,
 * stops the threads and frees everything.  Tickets are invalid afterwards. */
ism_status ism_server_destroy(ism_server* server);

/* ------------------------------------------------------------------------- */
/* Gradients (adjoint of eq. (1)-(6))                                        */
/* ------------------------------------------------------------------------- */
/* The paper computes RIRs only; the adjoint is the chain rule through its
 * definitions.  For a loss with dLoss/dh[k] = grad_out[k] over the image-
 * source samples k < n_ism of every RIR, each image n contributes
 *   g_A = sum_k grad_out[k] delta'(k - s_n)            (eq. (5), (6))
 *   g_s = -A_n sum_k grad_out[k] d delta'/dx (k - s_n)
 * and, with s = f_s d / c (eq. (3)), A = prod beta^e / (4 pi d) (eq. (4)),
 * d = |p_r - p_n| (eq. (2)), p_n per axis = n L + x_s (n even) or
 * (n + 1) L - x_s (n odd) (eq. (1)):
 *   dLoss/d beta_w += g_A e_w beta_w^(e_w - 1) prod_(v != w) beta_v^e_v / (4 pi d)
 *   g_d = -g_A A / d + g_s f_s / c
 *   dLoss/d p_r += g_d (p_r - p_n) / d
 *   dLoss/d x_s += -g_d (x_r - x_n) / d * (+1 if n even else -1), per axis.
 * The samples of the diffuse tail (k >= n_ism) carry no gradient: the tail
 * is treated as a constant of the loss.  FP32 tap arithmetic, fixed-order
 * sums (no atomics): the result is bit-identical from run to run.
 *
 * One backward job: the forward job (its `out`, `env_amp` and `seed` are not
 * used) and device pointers
 *   grad_out   [n_src][n_rcv][n_S] FP32, dLoss/dh (read)
 *   grad_beta  [6]  FP32 (written): dLoss/d beta of the room
 *   grad_src   [n_src][3] FP32 (written)
 *   grad_rcv   [n_rcv][3] FP32 (written)
 * Outputs are written, not accumulated; any of the three may be NULL. */
typedef struct {
    ism_job job;
    const float* grad_out;
    float* grad_beta;
    float* grad_src;
    float* grad_rcv;
} ism_grad_job;

/* Workspace bytes for ism_simulate_backward_batch. */
ism_status ism_backward_workspace_size(const ism_grad_job* jobs, int n_jobs, size_t* bytes);

/* Gradients of every job (host array `jobs`); ordered on `stream`.  Errors as
 * for ism_simulate_batch; grad_out must not be NULL. */
ism_status ism_simulate_backward_batch(const ism_grad_job* jobs, int n_jobs, void* workspace,
                                       size_t ws_bytes, void* stream);

/* Single-room form: arguments of ism_simulate (FP32 tap arithmetic) plus the
 * gradient pointers of ism_grad_job. */
ism_status ism_simulate_backward(const ism_room* room, const float* pos_src, int n_src,
                                 const float* pos_rcv, int n_rcv, const int nb_img[3], float Tmax,
                                 float fs, float Tdiff, float Tw, const float* grad_out,
                                 float* grad_beta, float* grad_src, float* grad_rcv, void* workspace,
                                 size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------- */
/* Diffuse-tail noise (Section 2.2, Section 3.3)                             */
/* ------------------------------------------------------------------------- */
/* Writes the unit-variance logistic noise z of samples k0 .. k0+n-1 of RIR
 * `rir` into device `z` (FP32): z = (sqrt(3)/pi) ln(u / (1 - u)) with
 * u = ((x >> 9) + 1/2) 2^-23 and x the Philox4x32-10 word described under
 * ism_simulate; ln is evaluated by a fixed sequence of correctly rounded
 * FP32 operations, so z is reproducible bit for bit on any IEEE machine.
 * The tail of ism_simulate is z times the square root of the envelope. */
ism_status ism_diffuse_noise(uint64_t seed, uint32_t rir, uint32_t k0, int n, float* z, void* stream);

/* ------------------------------------------------------------------------- */
/* Moving sources (Section 4: a source moving along a trajectory, recorded   */
/* by a microphone array)                                                    */
/* ------------------------------------------------------------------------- */
/* Cuts the source signal into one segment per trajectory point, filters each
 * segment by the RIRs of its point (one per microphone) and overlap-adds the
 * results:
 *   out[m][t] = sum_p sum_{starts[p] <= s < end_p} signal[s] rirs[p][m][t - s],
 * end_p = starts[p + 1] (n_x for the last point), 0 <= t < n_x + n_S - 1.
 * signal: device [n_x]; rirs: device [n_points][n_mics][n_S] (the layout of
 * ism_simulate with the trajectory points as sources and the microphones as
 * receivers); starts: device [n_points] non-decreasing segment starts (values
 * are clamped to [0, n_x]; samples before starts[0] are not emitted), or NULL
 * for the uniform cut starts[p] = floor(p n_x / n_points); out: device
 * [n_mics][n_x + n_S - 1], overwritten.  FP32 multiply-adds on the GPU in a
 * fixed order (results are identical run to run).  No workspace. */
ism_status ism_auralize(const float* signal, int n_x, const float* rirs, int n_points, int n_mics, int n_S,
                        const int* starts, float* out, void* stream);

/* The same filtering with a choice of method and a caller-owned workspace.
 * The paper filters with batched FFTs and overlap-add; ISM_AURALIZE_FFT does
 * it in the frequency domain with FFTs written for this library (FP32,
 * four-step: length-N DFTs, N the power of two >= n_x + n_S - 1, at most 2^20, split
 * as N = R C into shared-memory DFTs of R and C points).  Two microphones
 * share one complex sequence (real and imaginary parts), the segment
 * spectra X_p times the pair spectra are summed over the points in ascending
 * order (the overlap-add, in the frequency domain), and one inverse DFT per
 * pair gives both outputs; results are identical run to run.  Its error is
 * that of an FP32 FFT: a few 1e-7 of the largest sum |x| * |h|, spread over
 * all outputs.  ISM_AURALIZE_DIRECT is ism_auralize (no workspace).
 * ISM_AURALIZE_AUTO takes the FFT form when its operation count is less than
 * 1 / 2.55 of the direct form's (n_mics n_x n_S multiply-adds; the ratio of the
 * two forms' measured rates on GB300) and the workspace holds at least one
 * chunk, else the direct form.
 *   workspace  device, 256-byte aligned, >= ism_auralize_workspace_size()
 *              bytes for the FFT form (scratch; may be NULL for DIRECT);
 *              a larger workspace processes more points per chunk.
 * Other arguments, layout and errors as ism_auralize; ISM_ERR_UNSUPPORTED if
 * the FFT form is asked for an output longer than 2^20 samples. */
typedef enum {
    ISM_AURALIZE_AUTO = 0,
    ISM_AURALIZE_DIRECT = 1,
    ISM_AURALIZE_FFT = 2
} ism_auralize_method;

/* Workspace bytes of ism_auralize_ex for this method (0 when it takes the
 * direct form).  Host only. */
ism_status ism_auralize_workspace_size(int n_x, int n_points, int n_mics, int n_S, int method, size_t* bytes);

ism_status ism_auralize_ex(const float* signal, int n_x, const float* rirs, int n_points, int n_mics, int n_S,
                           const int* starts, float* out, int method, void* workspace, size_t ws_bytes,
                           void* stream);

/* ------------------------------------------------------------------------- */
/* Helpers of Section 4 (FP64)                                                */
/* ------------------------------------------------------------------------- */
/* Eq. (7): T60 = 0.161 V / sum_i S_i (1 - beta_i^2).  Host. */
ism_status ism_t60_sabine(const double L[3], const double beta[6], double* T60);

/* Inverse of eq. (7): reflection coefficients giving `T60`.  alpha_i =
 * w_i alpha_0 with abs_weights w (NULL = all ones), beta_i = sqrt(1 - alpha_i),
 * negated if `negative` (Section 2.2).  ISM_ERR_INFEASIBLE if some alpha_i >= 1.
 * Host. */
ism_status ism_beta_sabine(const double L[3], double T60, const double abs_weights[6], int negative,
                           double beta_out[6]);

/* Batched inverse Sabine on the GPU in FP64: for i < n, L[i][3] and T60[i]
 * (device) -> beta_out[i][6] (device), status[i] (device int, 0 = ok,
 * ISM_ERR_INFEASIBLE otherwise; beta_out row then zero).  abs_weights is a
 * device [6] array or NULL. */
ism_status ism_beta_sabine_device(const double* L, const double* T60, const double* abs_weights,
                                  int negative, int n, double* beta_out, int* status, void* stream);

/* Images per axis so that every reflection arriving before T is simulated:
 * M = ceil(c (T + Tw/2) / L) + 1, N = 2M + 1 (an image of index n is at
 * least (|n| - 1) L away from any point of the room).  Host. */
ism_status ism_nb_img_from_t(double T, const double L[3], double c, double Tw, int nb_out[3]);

/* Time at which the Sabine decay reaches att_dB: t = att_dB / 60 * T60.  Host. */
ism_status ism_att2t_sabine(double att_dB, double T60, double* t);

/* ------------------------------------------------------------------------- */
/* Per-stage timing (the breakdown of the paper's Table 2)                    */
/* ------------------------------------------------------------------------- */
/* Stages of one simulation, in launch order. */
typedef enum {
    ISM_STAGE_GEOMETRY = 0,     /* per-RIR axis tables, position checks          */
    ISM_STAGE_ENUM_COUNT = 1,   /* image enumeration, delays, bin counts (a)     */
    ISM_STAGE_SCAN = 2,         /* prefix sum of the bin counts (b)              */
    ISM_STAGE_ENUM_SCATTER = 3, /* image enumeration, scatter into bins (a, b)   */
    ISM_STAGE_ACCUM = 4,        /* windowed-sinc accumulation, eq. (5)-(6) (c)   */
    ISM_STAGE_FINALIZE = 5,     /* tile seams and envelope fit                   */
    ISM_STAGE_TAIL = 6,         /* diffuse tail, eq. (8) (d)                     */
    ISM_STAGE_ADJOINT = 7,      /* backward: per-image gradients and reductions  */
    ISM_N_STAGES = 8
} ism_stage;

/* Internal concurrency (no counterpart in the paper; a deployment setting):
 * a forward call with enough work (about 2e7 image sources in reach) runs
 * as two halves, split by source, on two internal streams forked from and
 * joined back into the caller's stream, so that one half's enumeration
 * overlaps the other's accumulation.  n_lanes = 1 keeps every launch on the
 * caller's stream (each kernel then runs alone, e.g. for timing it); 2 is
 * the default.  The results are bit-identical either way.  Process-wide. */
ism_status ism_set_lanes(int n_lanes);

/* Turns timing on (enable != 0) or off for all later simulation calls of the
 * process.  While on, each stage is bracketed by CUDA events recorded on the
 * caller's stream (no synchronisation is added). */
ism_status ism_profile_enable(int enable);
/* Zeroes the accumulated timings and counts. */
ism_status ism_profile_reset(void);
/* Waits for the recorded events and returns, for `stage`, the summed device
 * time in milliseconds, the number of kernel launches and the number of
 * simulation calls that ran it since the last reset. */
ism_status ism_profile_read(int stage, double* total_ms, long long* launches, long long* calls);

#ifdef __cplusplus
}
#endif

#endif /* ISM_H */
