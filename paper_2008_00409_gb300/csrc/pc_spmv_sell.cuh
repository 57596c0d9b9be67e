// Sliced-ELL storage of the off-diagonal 3x3 blocks, structure of arrays, for the PCG
// product (the ELL family the paper's Sec. 3.2 argues for on GPUs, here in the SELL-C-sigma
// form: slices of C = 32 rows, rows sorted by length inside windows of sigma = 1024 rows).
//
// Layout. Rows are permuted inside each window so that long rows come first (stable sort
// by off-diagonal block count, descending); slice s holds the 32 rows at sorted positions
// 32 s .. 32 s + 31 and has width w_s = the longest of them. Block position k of slice s
// is a run of 320 32-bit words at word (base_s + k) * 320: the 32 rows' column indices,
// then component e (row-major 3x3) of the 32 rows' blocks for e = 0..8. A warp (one
// thread per row) therefore reads every word of the stream with fully coalesced 128-byte
// loads and no staging. Shorter rows are padded with their own column and zero values.
// The diagonal blocks are not stored: in the difference form the diagonal multiplies
// p_i - p_i = 0, and the plain form takes them from a dense [V][9] copy.
//
// The layout is rebuilt from the BSR matrix at the start of each solve (a sort per window,
// a scan of the slice widths, a fill): one pass over the matrix against thousands of
// products per solve.
#pragma once

#include "pc_tma.cuh"

#define SL_C 32                    // rows per slice (one warp)
#define SL_SIGMA 1024              // rows per sorting window (one CTA of the sort kernel)
#define SL_WORDS (SL_C * 10)       // 32-bit words per block position of a slice
#define SL_BUCKETS 64              // sort keys: 0 = no row, 1 + min(length, 62)
#ifndef SL_THREADS
#define SL_THREADS 256
#endif
#ifndef SL_CTAS_PER_SM
#define SL_CTAS_PER_SM 3
#endif
#ifndef SL_UNROLL
#define SL_UNROLL 2                // block positions per pipeline group
#endif

struct SellArgs {
    int nslices;
    const int32_t *perm;     // [32 nslices] sorted position -> row, -1 past V
    const int32_t *width;    // [nslices]
    const int32_t *base;     // [nslices + 1] block-position offsets
    const uint32_t *data;    // [base[nslices] * 320]
    const float *diag;       // [V][9]: dres (difference form) or the diagonal blocks
    const float4 *x4;        // p
    float4 *y4;              // q = A p
    double *partials;        // p.q partial of each CTA (slot 3)
    pc_scalars *sc;
};

// Off-diagonal block count of `row` and the position of its diagonal block (-1 if the
// row has none).
__device__ __forceinline__ int sell_row_length(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int row,
                                               int *dpos)
{
    int lo = rp[row], hi = rp[row + 1];
    const int b = lo, e = hi;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ci[mid] < row) lo = mid + 1;
        else hi = mid;
    }
    const bool has = lo < e && ci[lo] == row;
    *dpos = has ? lo : -1;
    return (e - b) - (has ? 1 : 0);
}

// One CTA of SL_SIGMA threads per window: stable counting sort of the window's rows by
// descending length, then the width of each of its 32 slices.
__global__ void __launch_bounds__(SL_SIGMA) sell_sort_kernel(int V, const int32_t *__restrict__ rp,
                                                             const int32_t *__restrict__ ci, int32_t *perm,
                                                             int32_t *width, int32_t *dpos)
{
    __shared__ int cnt[SL_SIGMA / 32][SL_BUCKETS];  // per warp and key
    __shared__ int start[SL_BUCKETS];
    __shared__ int s_len[SL_SIGMA];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int row = blockIdx.x * SL_SIGMA + t;
    int len = 0, key = 0;
    if (row < V) {
        int d;
        len = sell_row_length(rp, ci, row, &d);
        dpos[row] = d;
        key = 1 + min(len, SL_BUCKETS - 2);
    }
    for (int i = t; i < (SL_SIGMA / 32) * SL_BUCKETS; i += blockDim.x) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (rank == 0) cnt[warp][key] = __popc(peers);
    __syncthreads();
    // exclusive prefix over warps per key (one thread per key)
    if (t < SL_BUCKETS) {
        int acc = 0;
        for (int w = 0; w < SL_SIGMA / 32; ++w) {
            const int c = cnt[w][t];
            cnt[w][t] = acc;
            acc += c;
        }
        start[t] = acc;  // total of key t for now
    }
    __syncthreads();
    if (t == 0) {  // descending keys: the largest first
        int acc = 0;
        for (int k = SL_BUCKETS - 1; k >= 0; --k) {
            const int c = start[k];
            start[k] = acc;
            acc += c;
        }
    }
    __syncthreads();
    const int pos = start[key] + cnt[warp][key] + rank;
    perm[blockIdx.x * SL_SIGMA + pos] = row < V ? row : -1;
    s_len[pos] = len;
    __syncthreads();
    // slice widths: warp j takes sorted positions 32 j .. 32 j + 31
    int w = s_len[t];
    for (int o = 16; o > 0; o >>= 1) w = max(w, __shfl_xor_sync(0xffffffffu, w, o));
    const int slice = blockIdx.x * (SL_SIGMA / 32) + warp;
    if (lane == 0) width[slice] = w;
}

// One warp per slice: the rows' off-diagonal blocks in column order into the slice's
// block positions (padding: the row's own column, zero values), and each row's diagonal
// block into diag[row] (zero if absent). Fails (error bit, nothing written past `cap`
// positions) when the layout does not fit.
__global__ void sell_fill_kernel(int V, int nslices, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                 const float *__restrict__ vals, const int32_t *__restrict__ perm,
                                 const int32_t *__restrict__ width, const int32_t *__restrict__ base,
                                 const int32_t *__restrict__ dpos, int64_t cap, uint32_t *data, float *diag,
                                 uint32_t *err)
{
    const int lane = threadIdx.x & 31;
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (s >= nslices) return;
    const int w = width[s];
    const int64_t b = base[s];
    if (b + w > cap) {
        if (lane == 0) pc_set_err(err, PC_DERR_INDEX);
        return;
    }
    const int row = perm[SL_C * s + lane];
    int r0 = 0, len = 0, d = -1;
    if (row >= 0) {
        r0 = rp[row];
        len = rp[row + 1] - r0;
        d = dpos[row];
        float *dg = diag + 9ll * row;
        for (int e = 0; e < 9; ++e) dg[e] = d >= 0 ? vals[9ll * d + e] : 0.f;
    }
    const int off_len = len - (d >= 0 ? 1 : 0);
    uint32_t *out = data + b * SL_WORDS + lane;
    for (int k = 0; k < w; ++k) {
        uint32_t *o = out + (int64_t)k * SL_WORDS;
        if (k < off_len) {
            const int src = r0 + k + ((d >= 0 && r0 + k >= d) ? 1 : 0);
            o[0] = (uint32_t)ci[src];
#pragma unroll
            for (int e = 0; e < 9; ++e) o[SL_C * (1 + e)] = __float_as_uint(vals[9ll * src + e]);
        } else {
            o[0] = (uint32_t)(row >= 0 ? row : 0);
#pragma unroll
            for (int e = 0; e < 9; ++e) o[SL_C * (1 + e)] = 0u;
        }
    }
}

// Columns and values of block positions k .. k + SL_UNROLL - 1 of a slice (positions
// past the width: column -1, zero values, which contribute nothing).
__device__ __forceinline__ void sell_load_group(const uint32_t *src, int k, int w, int (&col)[SL_UNROLL],
                                                float (&B)[SL_UNROLL][9])
{
#pragma unroll
    for (int j = 0; j < SL_UNROLL; ++j) {
        if (k + j < w) {
            const uint32_t *v = src + (int64_t)(k + j) * SL_WORDS;
            col[j] = (int)__ldcs(v);
#pragma unroll
            for (int e = 0; e < 9; ++e) B[j][e] = __uint_as_float(__ldcs(v + SL_C * (1 + e)));
        } else {
            col[j] = -1;
#pragma unroll
            for (int e = 0; e < 9; ++e) B[j][e] = 0.f;
        }
    }
}

// PCG product q = A p over the sliced layout, with this CTA's p.q partial. Difference
// form: q_i = D_i p_i + sum_j A_ij (p_j - p_i); plain form: q_i = A_ii p_i + sum_j A_ij p_j.
template <bool DIFF>
__global__ void __launch_bounds__(SL_THREADS, SL_CTAS_PER_SM) spmv_sell_kernel(SellArgs a)
{
    pdl_wait();
    if (a.sc->done) return;
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    float dot = 0.f, dot_c = 0.f;  // Kahan-compensated p.q of this thread's rows
    for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < a.nslices; s += nwarps) {
        const int row = a.perm[SL_C * s + lane];
        const int w = a.width[s];
        const uint32_t *src = a.data + (int64_t)a.base[s] * SL_WORDS + lane;
        const float4 pi = row >= 0 ? __ldg(a.x4 + row) : make_float4(0.f, 0.f, 0.f, 0.f);
        float D[9];
        if (row >= 0) {
#pragma unroll
            for (int e = 0; e < 9; ++e) D[e] = __ldcs(a.diag + 9ll * row + e);
        }
        float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
        // software pipeline over groups of SL_UNROLL block positions: the next group's
        // columns and values are loaded before the current group's gathers and products,
        // so a DRAM round trip overlaps the gathers' L2 round trip
        int col[SL_UNROLL];
        float B[SL_UNROLL][9];
        sell_load_group(src, 0, w, col, B);
        for (int k = 0; k < w; k += SL_UNROLL) {
            int ncol[SL_UNROLL];
            float nB[SL_UNROLL][9];
            if (k + SL_UNROLL < w) sell_load_group(src, k + SL_UNROLL, w, ncol, nB);
            float4 u[SL_UNROLL];
#pragma unroll
            for (int j = 0; j < SL_UNROLL; ++j) u[j] = col[j] >= 0 ? __ldg(a.x4 + col[j]) : pi;
#pragma unroll
            for (int j = 0; j < SL_UNROLL; ++j) {
                float4 uj = u[j];
                if (DIFF) { uj.x -= pi.x; uj.y -= pi.y; uj.z -= pi.z; }
                acc0 = fmaf(B[j][0], uj.x, fmaf(B[j][1], uj.y, fmaf(B[j][2], uj.z, acc0)));
                acc1 = fmaf(B[j][3], uj.x, fmaf(B[j][4], uj.y, fmaf(B[j][5], uj.z, acc1)));
                acc2 = fmaf(B[j][6], uj.x, fmaf(B[j][7], uj.y, fmaf(B[j][8], uj.z, acc2)));
            }
#pragma unroll
            for (int j = 0; j < SL_UNROLL; ++j) {
                col[j] = ncol[j];
#pragma unroll
                for (int e = 0; e < 9; ++e) B[j][e] = nB[j][e];
            }
        }
        if (row >= 0) {
            acc0 = fmaf(D[0], pi.x, fmaf(D[1], pi.y, fmaf(D[2], pi.z, acc0)));
            acc1 = fmaf(D[3], pi.x, fmaf(D[4], pi.y, fmaf(D[5], pi.z, acc1)));
            acc2 = fmaf(D[6], pi.x, fmaf(D[7], pi.y, fmaf(D[8], pi.z, acc2)));
            a.y4[row] = make_float4(acc0, acc1, acc2, 0.f);
            const float term = fmaf(pi.x, acc0, fmaf(pi.y, acc1, pi.z * acc2));
            const float yk = term - dot_c;
            const float tk = dot + yk;
            dot_c = (tk - dot) - yk;
            dot = tk;
        }
    }
    pdl_trigger();
    float hi[1] = {dot}, lo[1] = {-dot_c};  // the thread's compensated sum as a pair
    pc_block_sum_df(hi, lo, 1);
    if (threadIdx.x == 0)
        reinterpret_cast<float2 *>(a.partials)[(int64_t)blockIdx.x * RED_SLOTS + 3] = make_float2(hi[0], lo[0]);
}
