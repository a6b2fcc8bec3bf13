// ism_shell.cuh -- enumeration of the images of one RIR whose delay falls in a
// spherical shell around the receiver (Section 2.1, eq. (1)-(3)), shared by the
// fused Chebyshev accumulation (forward) and the fused Chebyshev adjoint.
//
// The image coordinates along one axis increase with the index n (eq. (1)):
// X(2m) = 2 m L + x_s and X(2m - 1) = 2 m L - x_s.  So for a grid column
// (ix, iy) the images whose distance falls in the shell [s_lo, s_hi) form at
// most two index intervals in z (below and above the receiver), found in
// closed form from the source and receiver coordinates, and the columns that
// reach the shell form one interval in iy per row ix.  A CTA's warps take the
// columns 32 at a time, compute each column's intervals and a warp prefix of
// their lengths, and process the column candidates 32 at a time (a
// candidate's column by binary search over the prefix).  Intervals are
// widened by SHELL_MARGIN sample; each candidate's exact float-float delay
// (the per-axis tables hold the squared offsets as float-float pairs) decides
// whether it belongs to the caller's range of integer delays, so every image
// lands in exactly one shell.  Candidate j of a warp's column chunk is always
// handled by lane j % 32, so the order in which a lane sees its images is a
// function of the geometry alone.
#pragma once

#include "ism_device.cuh"

#define SHELL_MARGIN 0.05f   // candidate margin (samples)

// Smallest image index n of an axis with coordinate X(n) >= Z.
__device__ __forceinline__ int ax_first(float Z, float xs, float inv2L)
{
    Z = fminf(fmaxf(Z, -1e7f), 1e7f);
    const int me = (int)ceilf((Z - xs) * inv2L);
    const int mo = (int)ceilf((Z + xs) * inv2L);
    return min(2 * me, 2 * mo - 1);
}

struct ShellAxis {
    float xs, xr, inv2L;   // source, receiver coordinate; 1 / (2 L)
    int nlo, N;
};

// Index interval [i0, i1) (0-based, clamped to the grid) of the images of an
// axis with X(n) - x_r in [D_lo, D_hi) (metres).
__device__ __forceinline__ void ax_range(const ShellAxis& a, float Dlo, float Dhi, int* i0, int* i1)
{
    const int n0 = ax_first(a.xr + Dlo, a.xs, a.inv2L);
    const int n1 = ax_first(a.xr + Dhi, a.xs, a.inv2L);
    *i0 = min(max(n0 - a.nlo, 0), a.N);
    *i1 = min(max(n1 - a.nlo, 0), a.N);
}

// CTA g of a fused launch -> (job, RIR, shell).  When the jobs' shell counts
// are alike the CTAs are ordered by the shell's rank from the outside over all
// fused RIRs of the launch set: every RIR's outermost (densest, since the
// images per delay grow as s^2) shell first, so the lightest shells fill the
// end of the launch; false for a CTA past its job's shells.  Otherwise they go
// job by job, RIR by RIR, densest shell first.
__device__ __forceinline__ bool shell_cta(const JobTable& t, long long g, int* jid, int* r, int* grp)
{
    if (!t.shell_rank_major) {
        const int j = ism_find_job(t, g, [](const JobDev& d) { return d.shell_cta_base; });
        const long long local = g - t.j[j].shell_cta_base;
        *jid = j;
        *r = (int)(local / t.j[j].shell_groups);
        *grp = t.j[j].shell_groups - 1 - (int)(local % t.j[j].shell_groups);
        return true;
    }
    const long long k = g / t.shell_rirs;   // rank from the outside
    const long long rr = g - k * t.shell_rirs;
    const int j = ism_find_job(t, rr, [](const JobDev& d) { return d.shell_rir_base; });
    *jid = j;
    *r = (int)(rr - t.j[j].shell_rir_base);
    *grp = t.j[j].shell_groups - 1 - (int)k;
    return *grp >= 0;
}

// What a CTA needs to walk the shell [b_lo, b_hi) of integer delays of RIR r.
struct Shell {
    ShellAxis ax[3];
    float kinv;            // c / f_s: metres per sample
    float s_lo2, s_hi2;    // squared shell bounds (samples^2), widened by the margin
    int b_lo, b_hi;        // integer delays owned: [b_lo, b_hi)
    float sd2;             // squared delay of the direct path (samples^2)
    int Nx, Ny;
    bool valid;            // false: the pair lies outside the room (+inf tables)
};

__device__ __forceinline__ Shell shell_setup(const JobDev& J, const float4* T, int r, int b_lo, int b_hi)
{
    Shell sh;
    const int i_src = r / J.n_rcv, i_rcv = r - (r / J.n_rcv) * J.n_rcv;
    sh.kinv = J.kinv;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        sh.ax[a].xs = J.pos_src[3 * i_src + a];
        sh.ax[a].xr = J.pos_rcv[3 * i_rcv + a];
        sh.ax[a].inv2L = J.inv2L[a];
        sh.ax[a].nlo = J.nlo[a];
        sh.ax[a].N = J.N[a];
    }
    sh.Nx = J.N[0];
    sh.Ny = J.N[1];
    sh.sd2 = T[-J.nlo[0]].x + T[J.N[0] - J.nlo[1]].x + T[J.N[0] + J.N[1] - J.nlo[2]].x;
    sh.valid = sh.sd2 < 3.0e38f;   // +inf tables: a pair outside the room (flagged by the geometry kernel)
    sh.b_lo = b_lo;
    sh.b_hi = b_hi;
    const float s_lo = fmaxf((float)b_lo - SHELL_MARGIN, 0.0f);
    const float s_hi = (float)b_hi + SHELL_MARGIN;
    sh.s_lo2 = s_lo * s_lo;
    sh.s_hi2 = s_hi * s_hi;
    return sh;
}

// Columns that reach the shell: row ix takes the iy with |y - y_r| < D_y.
// rowpre[ix] = columns in rows 0 .. ix (inclusive prefix), rowy0[ix] = first
// iy of row ix.  Every thread of the CTA calls it; returns the column count.
__device__ __forceinline__ int shell_rows(const Shell& sh, const float4* T, int* rowpre, int* rowy0)
{
    const int Nx = sh.Nx;
    for (int ix = threadIdx.x; ix < Nx; ix += blockDim.x) {
        int w = 0, y0 = 0;
        if (sh.valid) {
            const float rem = __fsub_rn(sh.s_hi2, T[ix].x);
            if (rem > 0.0f) {
                const float Dy = __fadd_rn(__fmul_rn(sqrtf(rem), sh.kinv), 1e-3f);
                int y1;
                ax_range(sh.ax[1], -Dy, Dy, &y0, &y1);
                w = max(y1 - y0, 0);
            }
        }
        rowpre[ix] = w;
        rowy0[ix] = y0;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int carry = 0;
        for (int base = 0; base < Nx; base += 32) {
            const int i = base + lane;
            int v = i < Nx ? rowpre[i] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int n = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += n;
            }
            if (i < Nx) rowpre[i] = carry + v;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
    }
    __syncthreads();
    return Nx > 0 ? rowpre[Nx - 1] : 0;
}

// Column cl of the shell (cl < n_cols): its candidate intervals in z and its
// record.  cnt = candidates; rf = {S_xy hi, S_xy lo, F_x F_y, o_x D_x + o_y D_y};
// ri = {first z index below, count below, first z index above, ix | iy << 16}.
__device__ __forceinline__ int shell_column(const Shell& sh, const float4* T, const int* rowpre, const int* rowy0,
                                            int cl, float2 orient_xy, float4* rf_out, int4* ri_out)
{
    const int Nx = sh.Nx, Ny = sh.Ny;
    int lo = 0, hi = Nx - 1;   // row: first ix with rowpre[ix] > cl
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (rowpre[mid] > cl) hi = mid;
        else lo = mid + 1;
    }
    const int ix = lo;
    const int before = ix > 0 ? rowpre[ix - 1] : 0;
    const float4 tx = T[ix];
    const int iy = min(rowy0[ix] + (cl - before), Ny - 1);
    const float4 ty = T[Nx + iy];
    const ff sxy = ff_add(ff{tx.x, tx.y}, ff{ty.x, ty.y});
    const float sxy_p = __fadd_rn(tx.x, ty.x);
    const float D1 =
        fmaxf(__fsub_rn(__fmul_rn(sqrtf(fmaxf(__fsub_rn(sh.s_lo2, sxy_p), 0.0f)), sh.kinv), 1e-3f), 0.0f);
    const float D2 = __fadd_rn(__fmul_rn(sqrtf(fmaxf(__fsub_rn(sh.s_hi2, sxy_p), 0.0f)), sh.kinv), 1e-3f);
    int d0 = 0, d1 = 0, u0 = 0, u1 = 0;
    if (sh.s_hi2 > sxy_p) {
        ax_range(sh.ax[2], -D2, -D1, &d0, &d1);   // below the receiver (closed-open in n)
        ax_range(sh.ax[2], D1, D2, &u0, &u1);     // above
        d1 = min(d1, u0);                         // disjoint, whatever the rounding
    }
    const int nd = max(d1 - d0, 0), nu = max(u1 - u0, 0);
    *rf_out = make_float4(sxy.hi, sxy.lo, tx.z * ty.z, __fmaf_rn(orient_xy.y, ty.w, orient_xy.x * tx.w));
    *ri_out = make_int4(d0, nd, u0, ix | (iy << 16));
    return nd + nu;
}

// Candidate i of a column (record cf, ci): its exact float-float delay; true
// if its integer delay b lies in [b_lo, b_hi), with b, f = the fractional part
// in [0, 1), s = the delay in samples (rounded float-float hi part), iz and tz
// = the z-axis table entry.
__device__ __forceinline__ bool shell_delay(const Shell& sh, const float4* T, const float4& cf, const int4& ci, int i,
                                            int* b_out, float* f_out, float* s_out, int* iz_out, float4* tz_out)
{
    const int iz = i < ci.y ? ci.x + i : ci.z + (i - ci.y);
    const float4 tz = T[sh.Nx + sh.Ny + iz];
    const ff s2 = ff_add(ff{cf.x, cf.y}, ff{tz.x, tz.y});
    const ff sq = ff_sqrt(s2);
    float bf = floorf(sq.hi);
    float f = __fadd_rn(__fsub_rn(sq.hi, bf), sq.lo);
    const bool neg = f < 0.0f;   // bring f into [0, 1) (see ism_delay)
    f = neg ? __fadd_rn(f, 1.0f) : f;
    bf = neg ? bf - 1.0f : bf;
    const bool one = f >= 1.0f;
    f = one ? __fsub_rn(f, 1.0f) : f;
    bf = one ? bf + 1.0f : bf;
    const int b = ism_int_of_integral(fminf(bf, 4.0e6f));
    *b_out = b;
    *f_out = f;
    *s_out = sq.hi;
    *iz_out = iz;
    *tz_out = tz;
    return b >= sh.b_lo && b < sh.b_hi;
}

// Candidate i of a column: calls on_image(b, f, s, cf, ixy, iz, tz) if it is
// an image of the shell (shell_delay).
template <class F>
__device__ __forceinline__ void shell_candidate(const Shell& sh, const float4* T, const float4& cf, const int4& ci,
                                                int i, F& on_image)
{
    int b, iz;
    float f, s;
    float4 tz;
    if (shell_delay(sh, T, cf, ci, i, &b, &f, &s, &iz, &tz)) on_image(b, f, s, cf, ci.w, iz, tz);
}

// Last index o in [0, 31] with W[o] <= j (W non-decreasing, W[0] = 0 <= j).
__device__ __forceinline__ int shell_find(const int* W, int j)
{
    int lo = 0, hi = 31;
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int mid = (lo + hi + 1) >> 1;
        if (W[mid] <= j) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The images of the shell, for the calling warp's share of the columns
// (chunks c0 = warp * 32 + k * 32 WARPS).  For each image with integer delay
// b in [b_lo, b_hi) lane calls
//   on_image(b, f, s, cf, ixy, iz, tz)
// with s = the delay in samples (rounded float-float hi part), f = its
// fractional part in [0, 1), cf = {S_xy hi, S_xy lo, F_x F_y, o_x D_x + o_y D_y}
// (column record; orient_xy = the receiver orientation's x, y), ixy = ix |
// iy << 16, iz and tz = the z-axis table entry.  Wf, Wi, Wst: the warp's
// 32-entry scratch in shared memory (33 ints for Wst).
template <int WARPS, class F>
__device__ __forceinline__ void shell_walk(const Shell& sh, const float4* T, const int* rowpre, const int* rowy0,
                                           int n_cols, float2 orient_xy, float4* Wf, int4* Wi, int* Wst, int warp,
                                           int lane, F&& on_image)
{
    for (int c0 = warp * 32; c0 < n_cols; c0 += WARPS * 32) {
        // ---- the column of this lane and its candidate intervals in z
        const int cl = c0 + lane;
        int cnt = 0;
        float4 rf = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        int4 ri = make_int4(0, 0, 0, 0);
        if (cl < n_cols) cnt = shell_column(sh, T, rowpre, rowy0, cl, orient_xy, &rf, &ri);
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int n = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += n;
        }
        const int total = __shfl_sync(0xffffffffu, inc, 31);
        __syncwarp();
        Wf[lane] = rf;
        Wi[lane] = ri;
        Wst[lane] = inc - cnt;
        if (lane == 31) Wst[32] = total;
        __syncwarp();

        // ---- the candidates, 32 at a time
        for (int j0 = 0; j0 < total; j0 += 32) {
            const int j = j0 + lane;
            if (j < total) {
                const int o = shell_find(Wst, j);
                shell_candidate(sh, T, Wf[o], Wi[o], j - Wst[o], on_image);
            }
        }
        __syncwarp();
    }
}

// The images of the shell for the whole CTA.  The candidates of every chunk of
// WARPS x 32 columns form batches of 32 (candidate c by lane c mod 32), and
// warp w takes the chunk's batches w, w + WARPS, ..: the warps differ by at
// most one batch per chunk, and only the chunk's last batch is partial.  For
// every batch the warp's 32 lanes call, converged,
//   on_lane(has, b, f, s, cf, tz)
// has = the lane's candidate is an image with integer delay b in [b_lo, b_hi)
// (shell_delay; the other arguments are unspecified when it is not), cf = its
// column record (as for shell_walk).  Which warp and lane meet an image, and in
// which order, is a function of the geometry alone.  Every thread of the CTA
// calls it.  Wf, Wi: [WARPS x 32] column records; Wst: [WARPS][33] warp
// prefixes; wtot: [WARPS].
template <int WARPS, class F>
__device__ __forceinline__ void shell_walk_cta(const Shell& sh, const float4* T, const int* rowpre, const int* rowy0,
                                               int n_cols, float2 orient_xy, float4* Wf, int4* Wi, int* Wst,
                                               int* wtot, int warp, int lane, F&& on_lane)
{
    for (int c0 = 0; c0 < n_cols; c0 += WARPS * 32) {
        const int cl = c0 + warp * 32 + lane;
        int cnt = 0;
        float4 rf = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        int4 ri = make_int4(0, 0, 0, 0);
        if (cl < n_cols) cnt = shell_column(sh, T, rowpre, rowy0, cl, orient_xy, &rf, &ri);
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int n = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += n;
        }
        Wf[warp * 32 + lane] = rf;
        Wi[warp * 32 + lane] = ri;
        Wst[warp * 33 + lane] = inc - cnt;
        if (lane == 31) {
            Wst[warp * 33 + 32] = inc;
            wtot[warp] = inc;
        }
        __syncthreads();
        int off[WARPS + 1];   // exclusive prefix of the warps' candidates
        off[0] = 0;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) off[w + 1] = off[w] + wtot[w];
        const int n_batches = (off[WARPS] + 31) >> 5;
        for (int bt = warp; bt < n_batches; bt += WARPS) {   // warp-uniform
            const int c = bt * 32 + lane;
            bool has = false;
            int b = 0;
            float f = 0.0f, s = 1.0f;
            float4 cf = make_float4(0.0f, 0.0f, 0.0f, 0.0f), tz = cf;
            if (c < off[WARPS]) {
                int wb = 0, base = 0;   // the warp whose columns hold candidate c: the last w with off[w] <= c
#pragma unroll
                for (int w = 1; w < WARPS; ++w)   // (never an empty block: off[wb + 1] > c)
                    if (off[w] <= c) {
                        wb = w;
                        base = off[w];
                    }
                const int j = c - base;
                const int o = shell_find(Wst + wb * 33, j);
                cf = Wf[wb * 32 + o];
                int iz;
                has = shell_delay(sh, T, cf, Wi[wb * 32 + o], j - Wst[wb * 33 + o], &b, &f, &s, &iz, &tz);
            }
            on_lane(has, b, f, s, cf, tz);
        }
        __syncthreads();   // the records are read before the next chunk overwrites them
    }
}
