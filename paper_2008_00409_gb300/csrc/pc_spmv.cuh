// Block-sparse (3x3) matrix-vector product, the dominant operator of the solve (Sec. 3.1).
//
// Persistent CTAs, five per SM when every tile fits stages of 14 blocks per row, else
// four with stages of 18 (the solve picks the shape from the matrix's largest tile). In
// each CTA a producer warp streams the CTA's 32-row
// tiles of the matrix (the tile's contiguous run of 36-byte blocks and of column
// indices) into a 2-stage shared-memory ring with 1-D bulk copies (cp.async.bulk)
// completing on mbarriers, while 4 consumer warps compute the current tile with four
// threads per row, up to four gathers in flight per thread. Row pointers, the row's own
// vector entries and the difference-form diagonal of the next tile are prefetched into
// registers before the current tile is computed, so the only latency left on a tile's
// critical path is the gather of the neighbours' vector entries. Tiles whose blocks exceed a stage (rows with many contacts)
// are read directly from global memory.
//
// PCG mode computes q = A p and this CTA's p.q partial (slot 3 of the CTA's entry in the
// partials array, as a double-float pair (float2); the update kernel that follows sums the
// partials in CTA order and forms alpha, so the SpMV ends without a grid-wide reduction
// tail), with p stored as float4 per vertex so that each gather is one 16-byte load.
// Difference form (dres given): y_j = D_j x_j + sum_i A_ji (x_i - x_j); the diagonal
// block then multiplies x_j - x_j = 0 and needs no special case.
#pragma once

#include "pc_tma.cuh"

#ifndef SP_ROWS
#define SP_ROWS 32                         // rows per tile
#endif
#ifndef SP_STAGES
#define SP_STAGES 2
#endif
#ifndef SP_CAP_PER_ROW
#define SP_CAP_PER_ROW 14                  // stage capacity in blocks per row (rows average about 12)
#endif
#ifndef SP_CTAS_PER_SM
#define SP_CTAS_PER_SM 5
#endif
#ifndef SP_TPR
#define SP_TPR 4                           // threads per row
#endif
#ifndef SP_WIN
#define SP_WIN 4                           // gathers in flight per thread
#endif
#define SP_CWARPS (SP_ROWS * SP_TPR / 32)  // consumer warps
#define SP_THREADS (32 * (SP_CWARPS + 1))  // + 1 producer warp
#define SP_CAP (SP_ROWS * SP_CAP_PER_ROW)  // blocks per stage
#define SP_VAL_BYTES ((SP_CAP * 36 + 32 + 15) / 16 * 16)
#define SP_COL_BYTES ((SP_CAP * 4 + 32 + 15) / 16 * 16)
#define SP_STAGE_BYTES (SP_VAL_BYTES + SP_COL_BYTES)
#define SP_SMEM_BYTES (SP_STAGES * SP_STAGE_BYTES)
#define SP_WAIT_BUDGET (1ll << 31)         // cycles (about a second) before a wait gives up
#define SP_CAPR_WIDE 18                    // the wider stages (blocks per row) of the product

// Stage layout and residency of spmv_kernel for stages of CAPR blocks per row: the more
// tiles in flight per SM, the more gathers of p are in flight, which is what the product
// waits on; five CTAs fit an SM with 14-block stages, four with 18-block stages.
template <int CAPR>
struct SpShape {
    static constexpr int cap = SP_ROWS * CAPR;
    static constexpr int val_bytes = (cap * 36 + 32 + 15) / 16 * 16;
    static constexpr int col_bytes = (cap * 4 + 32 + 15) / 16 * 16;
    static constexpr int stage_bytes = val_bytes + col_bytes;
    static constexpr int smem_bytes = SP_STAGES * stage_bytes;
    static constexpr int ctas_per_sm = CAPR <= SP_CAP_PER_ROW ? SP_CTAS_PER_SM : 4;
};

struct SpmvArgs {
    int V;
    const int32_t *rp;
    const int32_t *ci;
    const float *vals;
    const float *dres;    // difference-form diagonal, or null
    const float *dsc;     // optional: per row the scalar s when dres_i = s I (s > 0), else -1
    const float *xin;     // plain mode: x as float[V][3]
    const float4 *x4;     // PCG mode: the search direction p as float4[V]
    float *y;             // plain mode: result, float[V][3]
    float4 *y4;           // PCG mode: q = A p as float4[V]
    double *partials;     // PCG mode: p.q partials (slot 3 of each CTA's 4, a float2 pair)
    pc_scalars *sc;       // PCG mode: scalars
    uint32_t *err;        // error bits (timeouts)
};

template <bool PCG>
__device__ __forceinline__ float4 spmv_gather(const SpmvArgs &a, int c)
{
    if (PCG) {
        return a.x4[c];
    } else {
        return make_float4(a.xin[3ll * c], a.xin[3ll * c + 1], a.xin[3ll * c + 2], 0.f);
    }
}

__device__ __forceinline__ void spmv_fma(const float *B, float4 u, float &a0, float &a1, float &a2)
{
    a0 = fmaf(B[0], u.x, fmaf(B[1], u.y, fmaf(B[2], u.z, a0)));
    a1 = fmaf(B[3], u.x, fmaf(B[4], u.y, fmaf(B[5], u.z, a1)));
    a2 = fmaf(B[6], u.x, fmaf(B[7], u.y, fmaf(B[8], u.z, a2)));
}

// What a consumer thread needs about its own row, loaded one tile ahead.
struct SpmvRow {
    int row, rb, re;
    float4 xj;
    float D[9];
};

template <bool DIFF, bool PCG>
__device__ __forceinline__ void spmv_load_row(const SpmvArgs &a, int tile, int t, SpmvRow &r)
{
    r.row = tile * SP_ROWS + t / SP_TPR;
    r.rb = r.re = 0;
    r.xj = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r.row < a.V) {
        r.rb = a.rp[r.row];
        r.re = a.rp[r.row + 1];
        if (DIFF || PCG) r.xj = spmv_gather<PCG>(a, r.row);
        if (DIFF && (t & (SP_TPR - 1)) == 0) {
#pragma unroll
            for (int e = 0; e < 9; ++e) r.D[e] = 0.f;
            // most rows' difference diagonal is m_i I: one float instead of nine
            const float s = a.dsc ? a.dsc[r.row] : -1.f;
            if (s > 0.f) {
                r.D[0] = r.D[4] = r.D[8] = s;
            } else {
#pragma unroll
                for (int e = 0; e < 9; ++e) r.D[e] = a.dres[9ll * r.row + e];
            }
        }
    }
}

template <bool DIFF, bool PCG, int CAPR>
__global__ void __launch_bounds__(SP_THREADS, SpShape<CAPR>::ctas_per_sm) spmv_kernel(SpmvArgs a)
{
    using Sh = SpShape<CAPR>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t full_bar[SP_STAGES], empty_bar[SP_STAGES];
    __shared__ int stage_info[SP_STAGES][4];  // b0, value offset, column offset, staged
    __shared__ int s_timeout;
    if (PCG) {  // launched programmatically after the direction kernel
        pdl_wait();
        if (a.sc->done) return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < SP_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], SP_CWARPS);
        }
        s_timeout = 0;
        mbar_fence_init();
    }
    __syncthreads();
    const int ntiles = (a.V + SP_ROWS - 1) / SP_ROWS;
    // p.q of this thread's rows: FP32 with Kahan compensation (FP64 across threads)
    float dot_acc = 0.f, dot_c = 0.f;
    bool timed_out = false;

    if (warp == SP_CWARPS) {
        // ---------------- producer
        if (lane == 0) {
            int issued = 0;
            for (int k = 0;; ++k) {
                const int tile = blockIdx.x + k * gridDim.x;
                if (tile >= ntiles) break;
                const int s = k % SP_STAGES;
                const uint32_t ph = (uint32_t)(k / SP_STAGES) & 1u;
                if (k >= SP_STAGES && !mbar_wait_bounded(&empty_bar[s], ph ^ 1u, SP_WAIT_BUDGET)) {
                    timed_out = true;
                    break;
                }
                if (*(volatile int *)&s_timeout) break;
                const int r0 = tile * SP_ROWS, r1 = min(r0 + SP_ROWS, a.V);
                const int b0 = a.rp[r0], b1 = a.rp[r1];
                unsigned char *base = smem_raw + s * Sh::stage_bytes;
                if (b1 - b0 <= Sh::cap) {
                    const int64_t f0 = 9ll * b0, al0 = f0 & ~3ll, al1 = (9ll * b1 + 3) & ~3ll;
                    const int c0 = b0 & ~3, c1 = (b1 + 3) & ~3;
                    const uint32_t vbytes = (uint32_t)((al1 - al0) * 4), cbytes = (uint32_t)((c1 - c0) * 4);
                    stage_info[s][0] = b0;
                    stage_info[s][1] = (int)(f0 - al0);
                    stage_info[s][2] = b0 - c0;
                    stage_info[s][3] = 1;
                    mbar_arrive_expect_tx(&full_bar[s], vbytes + cbytes);
                    bulk_g2s(base, a.vals + al0, vbytes, &full_bar[s]);
                    bulk_g2s(base + Sh::val_bytes, a.ci + c0, cbytes, &full_bar[s]);
                } else {
                    stage_info[s][0] = b0;
                    stage_info[s][1] = 0;
                    stage_info[s][2] = 0;
                    stage_info[s][3] = 0;
                    mbar_arrive(&full_bar[s]);
                }
                ++issued;
            }
            // drain: the copies of the last stages issued must have landed before exit
            for (int k = issued - 1; k >= 0 && k >= issued - SP_STAGES; --k)
                if (!mbar_wait_bounded(&full_bar[k % SP_STAGES], (uint32_t)(k / SP_STAGES) & 1u, SP_WAIT_BUDGET))
                    timed_out = true;
        }
        __syncwarp();  // the producer warp reconverges before any block-wide barrier
    } else {
        // ---------------- consumers
        const int t = threadIdx.x;  // 0 .. SP_ROWS * SP_TPR - 1
        const int j = t & (SP_TPR - 1);
        SpmvRow nxt;
        if ((int)blockIdx.x < ntiles) spmv_load_row<DIFF, PCG>(a, blockIdx.x, t, nxt);
        for (int k = 0;; ++k) {
            const int tile = blockIdx.x + k * gridDim.x;
            if (tile >= ntiles) break;
            const SpmvRow cur = nxt;
            if (tile + (int)gridDim.x < ntiles) spmv_load_row<DIFF, PCG>(a, tile + gridDim.x, t, nxt);
            const int s = k % SP_STAGES;
            const uint32_t ph = (uint32_t)(k / SP_STAGES) & 1u;
            const bool ok = mbar_wait_bounded(&full_bar[s], ph, SP_WAIT_BUDGET);
            if (!__all_sync(0xffffffffu, ok)) {  // the whole warp leaves together
                timed_out = true;
                break;
            }
            const int b0 = stage_info[s][0], vo = stage_info[s][1], co = stage_info[s][2];
            const bool staged = stage_info[s][3] != 0;
            const float *s_vals = reinterpret_cast<const float *>(smem_raw + s * Sh::stage_bytes) + vo;
            const int32_t *s_cols = reinterpret_cast<const int32_t *>(smem_raw + s * Sh::stage_bytes + Sh::val_bytes) + co;
            float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
            const float4 xj = cur.xj;
            // up to four blocks per thread in flight (rows average about 13 blocks, so one
            // round covers most rows): all gathers are issued before the first FMA
            for (int b = cur.rb + j; b < cur.re; b += SP_WIN * SP_TPR) {
                float4 u[SP_WIN];
#pragma unroll
                for (int w = 0; w < SP_WIN; ++w) {
                    const int bw = b + w * SP_TPR;
                    if (bw < cur.re) u[w] = spmv_gather<PCG>(a, staged ? s_cols[bw - b0] : a.ci[bw]);
                }
#pragma unroll
                for (int w = 0; w < SP_WIN; ++w) {
                    const int bw = b + w * SP_TPR;
                    if (bw < cur.re) {
                        const float *B = staged ? s_vals + 9 * (bw - b0) : a.vals + 9ll * bw;
                        float4 uw = u[w];
                        if (DIFF) { uw.x -= xj.x; uw.y -= xj.y; uw.z -= xj.z; }
                        spmv_fma(B, uw, acc0, acc1, acc2);
                    }
                }
            }
            // the stage is no longer read by this warp: release it before the epilogue
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty_bar[s]);
#pragma unroll
            for (int o = 1; o < SP_TPR; o <<= 1) {
                acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
                acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
                acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
            }
            if (cur.row < a.V && j == 0) {
                if (DIFF) spmv_fma(cur.D, xj, acc0, acc1, acc2);
                if (PCG) {
                    a.y4[cur.row] = make_float4(acc0, acc1, acc2, 0.f);
                } else {
                    a.y[3ll * cur.row] = acc0;
                    a.y[3ll * cur.row + 1] = acc1;
                    a.y[3ll * cur.row + 2] = acc2;
                }
                if (PCG) {
                    const float term = fmaf(xj.x, acc0, fmaf(xj.y, acc1, xj.z * acc2));
                    const float yk = term - dot_c;
                    const float tk = dot_acc + yk;
                    dot_c = (tk - dot_acc) - yk;
                    dot_acc = tk;
                }
            }
        }
    }
    if (timed_out) {
        s_timeout = 1;
        atomicOr(a.err, PC_DERR_TIMEOUT);
        if (PCG) {
            a.sc->status = PC_ERR_TIMEOUT;
            a.sc->done = 1;
        }
    }
    if (PCG) {
        pdl_trigger();
        float hi[1] = {dot_acc}, lo[1] = {-dot_c};  // the thread's compensated sum as a pair
        pc_block_sum_df(hi, lo, 1);
        if (threadIdx.x == 0)
            reinterpret_cast<float2 *>(a.partials)[(int64_t)blockIdx.x * RED_SLOTS + 3] = make_float2(hi[0], lo[0]);
    }
}
