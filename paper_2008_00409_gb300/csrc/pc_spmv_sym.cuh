// PCG matrix-vector product on symmetric storage (Sec. 3.1's SpMV on half the matrix).
//
// The assembled matrix is bitwise symmetric (A_ji = A_ij^T). Each row keeps only its
// upper blocks (columns >= row, diagonal first), laid out like BSR; the lower part of row
// i is a list of (column j, index of block (j, i) in the upper arrays). Then
//   (A p)_i = sum over upper blocks A_ij p_j + sum over the list (A_ji)^T p_j,
// and in the difference form p_j is replaced by p_j - p_i and D_i p_i is added.
// The producer warp streams each 32-row tile's upper blocks, their columns and the
// tile's lower lists into the shared-memory ring with bulk copies; the consumers form the
// upper part from shared memory and gather each lower block from global memory (the row
// that owns it as an upper block belongs to the same band of tiles, so the block is
// found in L2 and the matrix crosses HBM once per product). Each row is reduced by its
// own four threads in a fixed order: the product is deterministic.
#pragma once

#include "pc_spmv.cuh"

#define SY_CAP_PER_ROW 12   // upper blocks per row that a stage holds
#define SY_LCAP_PER_ROW 12  // lower entries per row that a stage holds
#define SY_LWIN 2           // lower blocks per thread in flight
#define SY_CTAS_PER_SM 4    // register budget without spills
#define SY_CAP (SP_ROWS * SY_CAP_PER_ROW)
#define SY_LCAP (SP_ROWS * SY_LCAP_PER_ROW)
#define SY_VAL_BYTES ((SY_CAP * 36 + 32 + 15) / 16 * 16)
#define SY_COL_BYTES ((SY_CAP * 4 + 32 + 15) / 16 * 16)
#define SY_LBYTES ((SY_LCAP * 4 + 32 + 15) / 16 * 16)
#define SY_STAGE_BYTES (SY_VAL_BYTES + SY_COL_BYTES + 2 * SY_LBYTES)
#define SY_SMEM_BYTES (SP_STAGES * SY_STAGE_BYTES)

struct SymArgs {
    int V;
    const int32_t *urp, *uci;  // upper blocks: row pointers [V+1], columns
    const float *uvals;        // upper blocks, 9 floats each (padded by 16 floats)
    const int32_t *lrp;        // lower lists: row pointers [V+1]
    const int32_t *lcol;       // column j of each lower entry
    const int32_t *lsrc;       // index of block (j, i) in the upper arrays
    const float *dres;         // difference-form diagonal, or null
    const float4 *x4;          // p
    float4 *y4;                // q = A p
    double *partials;          // p.q partials (slot 3 of each CTA's entry)
    pc_scalars *sc;
    uint32_t *err;
};

struct SymRow {
    int row, rb, re, lb, le;
    float4 xj;
    float D[9];
};

template <bool DIFF>
__device__ __forceinline__ void sym_load_row(const SymArgs &a, int tile, int t, SymRow &r)
{
    r.row = tile * SP_ROWS + t / SP_TPR;
    r.rb = r.re = r.lb = r.le = 0;
    r.xj = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r.row < a.V) {
        r.rb = a.urp[r.row];
        r.re = a.urp[r.row + 1];
        r.lb = a.lrp[r.row];
        r.le = a.lrp[r.row + 1];
        r.xj = a.x4[r.row];
        if (DIFF && (t & (SP_TPR - 1)) == 0) {
#pragma unroll
            for (int e = 0; e < 9; ++e) r.D[e] = a.dres[9ll * r.row + e];
        }
    }
}

// acc += B^T u for a row-major 3x3 block B
__device__ __forceinline__ void spmv_fma_t(const float (&B)[9], float4 u, float &a0, float &a1, float &a2)
{
    a0 = fmaf(B[0], u.x, fmaf(B[3], u.y, fmaf(B[6], u.z, a0)));
    a1 = fmaf(B[1], u.x, fmaf(B[4], u.y, fmaf(B[7], u.z, a1)));
    a2 = fmaf(B[2], u.x, fmaf(B[5], u.y, fmaf(B[8], u.z, a2)));
}

// The 9 floats of block s of `vals` by three aligned 16-byte loads (vals is padded).
__device__ __forceinline__ void load_block9(const float *vals, int64_t s, float (&B)[9])
{
    const int64_t f = 9 * s, al = f & ~3ll;
    const int off = (int)(f - al);
    const float4 *p = reinterpret_cast<const float4 *>(vals + al);
    const float4 q0 = __ldg(p), q1 = __ldg(p + 1), q2 = __ldg(p + 2);
    const float w[12] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
#pragma unroll
    for (int k = 0; k < 9; ++k) B[k] = off == 0 ? w[k] : off == 1 ? w[k + 1] : off == 2 ? w[k + 2] : w[k + 3];
}

template <bool DIFF>
__global__ void __launch_bounds__(SP_THREADS, SY_CTAS_PER_SM) spmv_sym_kernel(SymArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t full_bar[SP_STAGES], empty_bar[SP_STAGES];
    // per stage: upper b0, value offset, column offset, upper staged, lower l0, lower offset, lower staged
    __shared__ int stage_info[SP_STAGES][8];
    __shared__ int s_timeout;
    pdl_wait();  // launched programmatically after the direction kernel
    if (a.sc->done) return;
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
    float dot_acc = 0.f, dot_c = 0.f;  // p.q of this thread's rows (Kahan; FP64 across threads)
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
                const int b0 = a.urp[r0], b1 = a.urp[r1];
                const int l0 = a.lrp[r0], l1 = a.lrp[r1];
                unsigned char *base = smem_raw + s * SY_STAGE_BYTES;
                const bool ust = b1 - b0 <= SY_CAP, lst = l1 - l0 <= SY_LCAP;
                uint32_t bytes = 0, vbytes = 0, cbytes = 0, lbytes = 0;
                int64_t al0 = 0;
                int c0 = 0, lc0 = 0;
                stage_info[s][0] = b0;
                stage_info[s][1] = 0;
                stage_info[s][2] = 0;
                stage_info[s][3] = ust ? 1 : 0;
                stage_info[s][4] = l0;
                stage_info[s][5] = 0;
                stage_info[s][6] = lst ? 1 : 0;
                if (ust) {
                    const int64_t f0 = 9ll * b0, al1 = (9ll * b1 + 3) & ~3ll;
                    al0 = f0 & ~3ll;
                    c0 = b0 & ~3;
                    const int c1 = (b1 + 3) & ~3;
                    vbytes = (uint32_t)((al1 - al0) * 4);
                    cbytes = (uint32_t)((c1 - c0) * 4);
                    stage_info[s][1] = (int)(f0 - al0);
                    stage_info[s][2] = b0 - c0;
                    bytes += vbytes + cbytes;
                }
                if (lst) {
                    lc0 = l0 & ~3;
                    const int lc1 = (l1 + 3) & ~3;
                    lbytes = (uint32_t)((lc1 - lc0) * 4);
                    stage_info[s][5] = l0 - lc0;
                    bytes += 2 * lbytes;
                }
                if (bytes > 0) {
                    mbar_arrive_expect_tx(&full_bar[s], bytes);
                    if (ust) {
                        bulk_g2s(base, a.uvals + al0, vbytes, &full_bar[s]);
                        bulk_g2s(base + SY_VAL_BYTES, a.uci + c0, cbytes, &full_bar[s]);
                    }
                    if (lst) {
                        bulk_g2s(base + SY_VAL_BYTES + SY_COL_BYTES, a.lcol + lc0, lbytes, &full_bar[s]);
                        bulk_g2s(base + SY_VAL_BYTES + SY_COL_BYTES + SY_LBYTES, a.lsrc + lc0, lbytes, &full_bar[s]);
                    }
                } else {
                    mbar_arrive(&full_bar[s]);
                }
                ++issued;
            }
            for (int k = issued - 1; k >= 0 && k >= issued - SP_STAGES; --k)
                if (!mbar_wait_bounded(&full_bar[k % SP_STAGES], (uint32_t)(k / SP_STAGES) & 1u, SP_WAIT_BUDGET))
                    timed_out = true;
        }
        __syncwarp();
    } else {
        // ---------------- consumers
        const int t = threadIdx.x;
        const int j = t & (SP_TPR - 1);
        SymRow nxt;
        if ((int)blockIdx.x < ntiles) sym_load_row<DIFF>(a, blockIdx.x, t, nxt);
        for (int k = 0;; ++k) {
            const int tile = blockIdx.x + k * gridDim.x;
            if (tile >= ntiles) break;
            const SymRow cur = nxt;
            if (tile + (int)gridDim.x < ntiles) sym_load_row<DIFF>(a, tile + gridDim.x, t, nxt);
            const int s = k % SP_STAGES;
            const uint32_t ph = (uint32_t)(k / SP_STAGES) & 1u;
            const bool ok = mbar_wait_bounded(&full_bar[s], ph, SP_WAIT_BUDGET);
            if (!__all_sync(0xffffffffu, ok)) {
                timed_out = true;
                break;
            }
            const int b0 = stage_info[s][0], vo = stage_info[s][1], co = stage_info[s][2];
            const bool ust = stage_info[s][3] != 0;
            const int l0 = stage_info[s][4], lo = stage_info[s][5];
            const bool lst = stage_info[s][6] != 0;
            const unsigned char *base = smem_raw + s * SY_STAGE_BYTES;
            const float *s_vals = reinterpret_cast<const float *>(base) + vo;
            const int32_t *s_cols = reinterpret_cast<const int32_t *>(base + SY_VAL_BYTES) + co;
            const int32_t *s_lcol = reinterpret_cast<const int32_t *>(base + SY_VAL_BYTES + SY_COL_BYTES) + lo;
            const int32_t *s_lsrc =
                reinterpret_cast<const int32_t *>(base + SY_VAL_BYTES + SY_COL_BYTES + SY_LBYTES) + lo;
            float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
            const float4 xj = cur.xj;
            // upper blocks: values from the stage, four gathers in flight
            for (int b = cur.rb + j; b < cur.re; b += SP_WIN * SP_TPR) {
                float4 u[SP_WIN];
#pragma unroll
                for (int w = 0; w < SP_WIN; ++w) {
                    const int bw = b + w * SP_TPR;
                    if (bw < cur.re) u[w] = a.x4[ust ? s_cols[bw - b0] : a.uci[bw]];
                }
#pragma unroll
                for (int w = 0; w < SP_WIN; ++w) {
                    const int bw = b + w * SP_TPR;
                    if (bw < cur.re) {
                        const float *B = ust ? s_vals + 9 * (bw - b0) : a.uvals + 9ll * bw;
                        float4 uw = u[w];
                        if (DIFF) { uw.x -= xj.x; uw.y -= xj.y; uw.z -= xj.z; }
                        spmv_fma(B, uw, acc0, acc1, acc2);
                    }
                }
            }
            // lower entries: the transposed upper block (j, i) gathered from global memory
            for (int e = cur.lb + j; e < cur.le; e += SY_LWIN * SP_TPR) {
                float4 u[SY_LWIN];
                int src[SY_LWIN];
#pragma unroll
                for (int w = 0; w < SY_LWIN; ++w) {
                    const int ew = e + w * SP_TPR;
                    if (ew < cur.le) {
                        u[w] = a.x4[lst ? s_lcol[ew - l0] : a.lcol[ew]];
                        src[w] = lst ? s_lsrc[ew - l0] : a.lsrc[ew];
                    }
                }
#pragma unroll
                for (int w = 0; w < SY_LWIN; ++w) {
                    const int ew = e + w * SP_TPR;
                    if (ew < cur.le) {
                        float B[9];
                        load_block9(a.uvals, src[w], B);
                        float4 uw = u[w];
                        if (DIFF) { uw.x -= xj.x; uw.y -= xj.y; uw.z -= xj.z; }
                        spmv_fma_t(B, uw, acc0, acc1, acc2);
                    }
                }
            }
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
                a.y4[cur.row] = make_float4(acc0, acc1, acc2, 0.f);
                const float term = fmaf(xj.x, acc0, fmaf(xj.y, acc1, xj.z * acc2));
                const float yk = term - dot_c;
                const float tk = dot_acc + yk;
                dot_c = (tk - dot_acc) - yk;
                dot_acc = tk;
            }
        }
    }
    if (timed_out) {
        s_timeout = 1;
        atomicOr(a.err, PC_DERR_TIMEOUT);
        a.sc->status = PC_ERR_TIMEOUT;
        a.sc->done = 1;
    }
    pdl_trigger();
    float hi[1] = {dot_acc}, lo[1] = {-dot_c};  // the thread's compensated sum as a pair
    pc_block_sum_df(hi, lo, 1);
    if (threadIdx.x == 0)
        reinterpret_cast<float2 *>(a.partials)[(int64_t)blockIdx.x * RED_SLOTS + 3] = make_float2(hi[0], lo[0]);
}
