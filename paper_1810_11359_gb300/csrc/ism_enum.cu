// ism_enum.cu -- image enumeration (kernel a) and the counting sort of the
// images into 32-sample delay bins (kernel b).
//
// Kernel (a) walks the image grid of every RIR (Section 2.1) column by
// column: one warp owns a contiguous range of columns (ix, iy) and, for each,
// only the nz range that can hold an image within reach (|n| - 1) L_z <=
// c (Tmax + Tw/2), the bound that also fixes the grid size.  For image
// (nx, ny, nz) the squared delay in samples is Sx + Sy + Sz (tables of
// ism_geometry.cu, eq. (2)-(3) with s = d f_s / c); the image is kept when its
// window (eq. (6), |t - tau| < Tw/2) can reach a sample below n_ism, and its
// delay bin is q ~ floor((s + 1/2) / 32).  The delay here is plain FP32: it
// only chooses the bin.  The accumulation kernel recomputes the delay in
// float-float and tolerates the bin being off by the FP32 error (it accepts
// offsets -1..31 inside a bin).
//
// Kernel (b) is a stable counting sort over (RIR, bin) keys:
//   count:   each warp walks its columns and counts its kept images per bin
//            (shared-memory integer adds) -> hist[rir][bin][unit]
//   scan:    exclusive prefix over hist (bin-major, unit-minor)
//   scatter: the same walk again; each image id goes to hist[rir][bin][unit]
//            + rank, the rank of images of one 32-wide step sharing a bin
//            being their lane order (match.any + popc).
// Every position is a pure function of the inputs, so the order of images
// inside a bin -- hence the FP32 summation order later -- is the same on
// every run, and each bin is one contiguous range of ids.
#include "ism_device.cuh"

namespace {

// Delay bin of an image from its plain-FP32 squared delay s2 (samples^2), or
// -1 when its window cannot reach a sample below n_ism.
__device__ __forceinline__ int bin_of(float s2, float s_cut2, int Q, uint32_t* status)
{
    if (!(s2 < s_cut2)) return -1;
    const float s = s2 * ism_rsqrt(s2);
    // nearest integer of (s + 1/2) / 32 - 1/2, i.e. ~floor((s + 1/2) / 32)
    int q = ism_round_int(__fmaf_rn(s, 1.0f / ISM_SB, 0.5f / ISM_SB - 0.5f));
    if (q >= Q || q < 0) {  // cannot happen for a consistent s_cut2; keep memory safe
        atomicOr(status, (uint32_t)ISM_DEVICE_FLAG_BIN);
        q = -1;
    }
    return q;
}

template <bool SCATTER>
__global__ void __launch_bounds__(ISM_ENUM_WARPS * 32) enum_kernel(const __grid_constant__ JobTable t,
                                                                    const float4* __restrict__ tbl,
                                                                    uint32_t* __restrict__ hist,
                                                                    uint32_t* __restrict__ ids,
                                                                    uint32_t* __restrict__ status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const long long g = blockIdx.x;
    const int jid = ism_find_job(t, g, [](const JobDev& j) { return j.enum_cta_base; });
    const JobDev& J = t.j[jid];
    const int ctas_per_rir = (J.U + ISM_ENUM_WARPS - 1) / ISM_ENUM_WARPS;
    const long long local = g - J.enum_cta_base;
    const int r = (int)(local / ctas_per_rir);
    const int c = (int)(local % ctas_per_rir);
    const int Nx = J.N[0], Ny = J.N[1], Nz = J.N[2];
    const int n_axis = Nx + Ny + Nz;
    const int Q = J.Q;

    float* S = reinterpret_cast<float*>(smem);  // [n_axis] plain FP32 squared offsets
    uint32_t* cnt_all = reinterpret_cast<uint32_t*>(smem + (size_t)((t.max_axis_sum + 3) & ~3) * 4);

    const float4* T = tbl + J.tbl_base + (long long)r * n_axis;
    for (int e = threadIdx.x; e < n_axis; e += blockDim.x) S[e] = T[e].x;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int unit = c * ISM_ENUM_WARPS + warp;
    const bool active = unit < J.U;
    uint32_t* cnt = cnt_all + (size_t)warp * t.max_Q;
    const long long hrow = J.hist_base + (long long)r * Q * J.U;  // + q * U + unit
    if (active)
        for (int q = lane; q < Q; q += 32) cnt[q] = SCATTER ? hist[hrow + (long long)q * J.U + unit] : 0u;
    __shared__ int iz_min_s;
    __syncthreads();
    if (SCATTER && warp == 0) {
        // the z index of the image plane nearest the receiver: Sz falls
        // towards it and rises beyond it (image coordinates increase with n)
        const float* Szs = S + Nx + Ny;
        float best = __int_as_float(0x7f800000);
        int bi = 0;
        for (int iz = lane; iz < Nz; iz += 32)
            if (Szs[iz] < best) {
                best = Szs[iz];
                bi = iz;
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob < best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (lane == 0) iz_min_s = bi;
    }
    __syncthreads();
    if (!active) return;
    const int iz_min = SCATTER ? iz_min_s : 0;

    const float* Sx = S;
    const float* Sy = S + Nx;
    const float* Sz = S + Nx + Ny;
    const float s_cut2 = J.s_cut2;
    const float inv_kLz = J.inv_kLz;       // 1 / (f_s / c * L_z): samples -> z cells
    const int nlo_z = J.nlo[2];
    const int col0 = unit * J.cols_per_unit;
    int col1 = col0 + J.cols_per_unit;
    if (col1 > Nx * Ny) col1 = Nx * Ny;
    const unsigned lt_mask = (1u << lane) - 1u;

    int ix = col0 / Ny, iy = col0 - (col0 / Ny) * Ny;
    for (int col = col0; col < col1; ++col, ++iy) {
        if (iy == Ny) {
            iy = 0;
            ++ix;
        }
        const float sxy = __fadd_rn(Sx[ix], Sy[iy]);
        const float rem = s_cut2 - sxy;
        if (!(rem > 0.0f)) continue;
        // |n| - 1 <= sqrt(rem) / (k L_z) bounds every kept image of the column
        const int M = (int)(rem * ism_rsqrt(rem) * inv_kLz) + 2;
        int z0 = -M - nlo_z, z1 = M - nlo_z;
        if (z0 < 0) z0 = 0;
        if (z1 > Nz - 1) z1 = Nz - 1;
        if (!SCATTER) {
            for (int base = z0; base <= z1; base += 32) {
                const int iz = base + lane;
                if (iz > z1) continue;
                const int q = bin_of(__fadd_rn(sxy, Sz[iz]), s_cut2, Q, status);
                // counts only: integer adds commute, so the order is immaterial
                if (q >= 0) atomicAdd(&cnt[q], 1u);
            }
            continue;
        }
        // scatter: the column's z range as two arms walked away from the
        // receiver's plane, along which the delay never decreases, so equal
        // bins are contiguous lanes and a lane's rank among its bin's images
        // is its distance to the first lane of its run (match.any only when
        // FP32 rounding breaks the order)
        for (int arm = 0; arm < 2; ++arm) {
            const int first = arm == 0 ? max(z0, iz_min) : min(z1, iz_min - 1);
            const int len = arm == 0 ? z1 - first + 1 : first - z0 + 1;
            for (int k0 = 0; k0 < len; k0 += 32) {
                const int k = k0 + lane;
                const int iz = arm == 0 ? first + k : first - k;
                const int q = k < len ? bin_of(__fadd_rn(sxy, Sz[iz]), s_cut2, Q, status) : -1;
                const bool valid = q >= 0;
                const unsigned vmask = __ballot_sync(0xffffffffu, valid);
                if (!vmask) break;   // the rest of the arm lies beyond the cut as well
                const int qp = __shfl_up_sync(0xffffffffu, q, 1);
                const unsigned down = __ballot_sync(0xffffffffu, valid && lane > 0 && q < qp);
                const uint32_t id = (uint32_t)ix | ((uint32_t)iy << 10) | ((uint32_t)iz << 20);
                if (down == 0u && (vmask & (vmask + 1u)) == 0u) {
                    // valid lanes are a prefix with non-decreasing bins
                    const unsigned starts = __ballot_sync(0xffffffffu, valid && (lane == 0 || q != qp));
                    const int run0 = 31 - __clz(starts & (0xffffffffu >> (31 - lane)));
                    const unsigned after = starts & ~((2u << lane) - 1u);
                    const int run1 = after ? __ffs(after) - 1 : __popc(vmask);
                    uint32_t base_cnt = 0;
                    if (valid) base_cnt = cnt[q];
                    __syncwarp();
                    if (valid) {
                        ids[base_cnt + (uint32_t)(lane - run0)] = id;
                        if (lane == run1 - 1) cnt[q] = base_cnt + (uint32_t)(run1 - run0);
                    }
                    __syncwarp();
                } else {
                    const unsigned peers = __match_any_sync(0xffffffffu, q);
                    uint32_t base_cnt = 0;
                    if (valid) base_cnt = cnt[q];
                    __syncwarp();
                    if (valid) {
                        if (lane == __ffs(peers) - 1) cnt[q] = base_cnt + (uint32_t)__popc(peers);
                        ids[base_cnt + (uint32_t)__popc(peers & lt_mask)] = id;
                    }
                    __syncwarp();
                }
            }
        }
    }
    if (!SCATTER) {
        __syncwarp();
        for (int q = lane; q < Q; q += 32) hist[hrow + (long long)q * J.U + unit] = cnt[q];
    }
}

// ---------------------------------------------------------------------------
// Exclusive scan of hist[0, n) in place; hist[n] receives the total.
// Three launches: block totals, scan of the totals (one block), apply.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread (1024 threads); returns
// the exclusive prefix and writes the block total to *total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* sh, uint32_t* total)
{
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = warp_incl_scan(v, lane);
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0u;
        uint32_t wi = warp_incl_scan(w, lane);
        sh[lane] = wi - w;
        if (lane == 31) sh[32] = wi;
    }
    __syncthreads();
    uint32_t r = sh[warp] + inc - v;
    *total = sh[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(1024) scan_partials(const uint32_t* __restrict__ a, long long n,
                                                      uint32_t* __restrict__ part)
{
    __shared__ uint32_t sh[33];
    long long i0 = (long long)blockIdx.x * ISM_SCAN_BLOCK + threadIdx.x * 4;
    uint32_t v = 0;
    for (int k = 0; k < 4; ++k)
        if (i0 + k < n) v += a[i0 + k];
    uint32_t tot;
    block_excl_scan(v, sh, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) scan_top(uint32_t* __restrict__ part, long long nb,
                                                 uint32_t* __restrict__ a, long long n)
{
    __shared__ uint32_t sh[33];
    uint32_t vals[16];
    uint32_t s = 0;
    long long i0 = (long long)threadIdx.x * 16;
    for (int k = 0; k < 16; ++k) {
        vals[k] = (i0 + k < nb) ? part[i0 + k] : 0u;
        s += vals[k];
    }
    uint32_t tot;
    uint32_t ex = block_excl_scan(s, sh, &tot);
    for (int k = 0; k < 16; ++k) {
        if (i0 + k < nb) part[i0 + k] = ex;
        ex += vals[k];
    }
    if (threadIdx.x == 0) a[n] = tot;
}

__global__ void __launch_bounds__(1024) scan_apply(uint32_t* __restrict__ a, long long n,
                                                   const uint32_t* __restrict__ part)
{
    __shared__ uint32_t sh[33];
    long long i0 = (long long)blockIdx.x * ISM_SCAN_BLOCK + threadIdx.x * 4;
    uint32_t v[4];
    uint32_t s = 0;
    for (int k = 0; k < 4; ++k) {
        v[k] = (i0 + k < n) ? a[i0 + k] : 0u;
        s += v[k];
    }
    uint32_t tot;
    uint32_t ex = block_excl_scan(s, sh, &tot) + part[blockIdx.x];
    for (int k = 0; k < 4; ++k) {
        if (i0 + k < n) a[i0 + k] = ex;
        ex += v[k];
    }
}

}  // namespace

int ism_launch_enum(const JobTable& t, const WsPlan& p, char* ws, bool scatter, void* stream)
{
    if (p.enum_ctas <= 0) return 0;
    size_t sm = (size_t)((t.max_axis_sum + 3) & ~3) * 4 + (size_t)ISM_ENUM_WARPS * t.max_Q * 4;
    auto* tbl = reinterpret_cast<const float4*>(ws + p.tbl_off);
    auto* hist = reinterpret_cast<uint32_t*>(ws + p.hist_off);
    auto* idsp = reinterpret_cast<uint32_t*>(ws + p.ids_off);
    auto* st = reinterpret_cast<uint32_t*>(ws + p.status_off);
    cudaStream_t s = (cudaStream_t)stream;
    static std::atomic<unsigned long long> opened[2] = {{0}, {0}};
    int rc;
    if (scatter) {
        if ((rc = ism_open_smem((const void*)enum_kernel<true>, &opened[1]))) return rc;
        enum_kernel<true><<<(unsigned)p.enum_ctas, ISM_ENUM_WARPS * 32, sm, s>>>(t, tbl, hist, idsp, st);
    } else {
        if ((rc = ism_open_smem((const void*)enum_kernel<false>, &opened[0]))) return rc;
        enum_kernel<false><<<(unsigned)p.enum_ctas, ISM_ENUM_WARPS * 32, sm, s>>>(t, tbl, hist, idsp, st);
    }
    return (int)cudaGetLastError();
}

int ism_launch_scan(const WsPlan& p, char* ws, void* stream)
{
    auto* hist = reinterpret_cast<uint32_t*>(ws + p.hist_off);
    auto* part = reinterpret_cast<uint32_t*>(ws + p.part_off);
    long long n = p.hist_total, nb = p.n_scan_blocks;
    cudaStream_t s = (cudaStream_t)stream;
    scan_partials<<<(unsigned)nb, 1024, 0, s>>>(hist, n, part);
    scan_top<<<1, 1024, 0, s>>>(part, nb, hist, n);
    scan_apply<<<(unsigned)nb, 1024, 0, s>>>(hist, n, part);
    return (int)cudaGetLastError();
}
