// Preconditioned conjugate gradients on the assembled system (Sec. 2.5: the linear
// equations are solved with a preconditioned conjugate gradient solver; Sec. 3.1: the
// SpMV is the most expensive operator and vector operations are data parallel).
//
// Per iteration two kernels run by default:
//   spmv:           q = A p, partial p.q                             -> alpha = rz / pq
//   update + dir:   x += alpha p, r -= alpha q, z = D^-1 r, partial r.z, r.r; a grid-wide
//                   barrier; beta, stop test; p = z + beta p        (pcg_update_dir_kernel)
// or, when the rows do not fit the fused kernel's registers (or fuse = 0), three:
//   direction: p = z + beta p; spmv; update (z to memory, the last block forms beta).
// The SpMV kernel, a bulk-copy pipelined stream over the blocks, is in pc_spmv.cuh; it
// reads by default a per-solve copy of the matrix without its diagonal blocks, in stages
// of 14 blocks per row at five CTAs per SM when the matrix's largest 32-row tile fits
// them, else of 18 at four (measured per solve by tile_max_kernel).
// Dot products: FP32 within a thread, FP64 across threads; partials are summed in a fixed
// order, so every reduction is deterministic. p, q and z are float4 per vertex (each SpMV
// gather is one 16-byte load); x, r and the scalar Jacobi inverse, only ever streamed,
// are packed float[V][3].
//
// Mixed precision (PC_PREC_MIXED): the solution is an FP64 accumulator plus the FP32
// increment the iterations build; at refresh points the increment is folded into the
// accumulator and the residual is recomputed in FP64 and replaces the recurrence
// residual, keeping the search direction (residual replacement). FP64 appears only in
// that residual, the dot-product reductions and the accumulator update.
#include <math.h>
#include <string.h>


#include "pc_internal.cuh"

#define EW_THREADS 256
#define RED_SLOTS 4

// ------------------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum_d(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-reduce `n` doubles (n <= RED_SLOTS) in a fixed tree; thread 0 gets the sums.
__device__ __forceinline__ void block_sum_d(double *v, int n)
{
    __shared__ double s[RED_SLOTS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < n; ++k) {
        double w = warp_sum_d(v[k]);
        if (lane == 0) s[k][warp] = w;
    }
    __syncthreads();
    if (warp == 0) {
        for (int k = 0; k < n; ++k) {
            double w = lane < nw ? s[k][lane] : 0.0;
            v[k] = warp_sum_d(w);
        }
    }
    __syncthreads();
}

// Write this block's partial sums; returns true (in all threads) in the block that
// arrives last, with the grand totals in v[] of thread 0 (summed in block order).
static __device__ bool last_block_reduce(double *v, int n, double *partials, uint32_t *counter)
{
    __shared__ bool s_last;
    block_sum_d(v, n);
    if (threadIdx.x == 0) {
        for (int k = 0; k < n; ++k) partials[(int64_t)blockIdx.x * RED_SLOTS + k] = v[k];
        __threadfence();
        uint32_t t = atomicAdd(counter, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double acc[RED_SLOTS] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x)
        for (int k = 0; k < n; ++k) acc[k] += __ldcg(partials + (int64_t)i * RED_SLOTS + k);
    block_sum_d(acc, n);
    if (threadIdx.x == 0) {
        for (int k = 0; k < n; ++k) v[k] = acc[k];
        *counter = 0u;
    }
    return true;
}

// last_block_reduce for n <= RED_SLOTS double-float pairs (float2 partials); the totals,
// as pairs, in hi[] / lo[] of thread 0 of the last block.
static __device__ bool last_block_reduce_df(float *hi, float *lo, int n, double *partials, uint32_t *counter)
{
    __shared__ bool s_last;
    float2 *pf = reinterpret_cast<float2 *>(partials);
    pc_block_sum_df(hi, lo, n);
    if (threadIdx.x == 0) {
        for (int k = 0; k < n; ++k) pf[(int64_t)blockIdx.x * RED_SLOTS + k] = make_float2(hi[k], lo[k]);
        __threadfence();
        uint32_t t = atomicAdd(counter, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    float ah[RED_SLOTS] = {0.f, 0.f, 0.f, 0.f}, al[RED_SLOTS] = {0.f, 0.f, 0.f, 0.f};
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x)
        for (int k = 0; k < n; ++k) {
            const float2 v = __ldcg(pf + (int64_t)i * RED_SLOTS + k);
            pc_df_add(ah[k], al[k], v.x, v.y);
        }
    pc_block_sum_df(ah, al, n);
    if (threadIdx.x == 0) {
        for (int k = 0; k < n; ++k) {
            hi[k] = ah[k];
            lo[k] = al[k];
        }
        *counter = 0u;
    }
    return true;
}

#include "pc_spmv.cuh"
#include "pc_spmv_sym.cuh"
#include "pc_spmv_sell.cuh"

// ------------------------------------------------------------------------- preconditioner

// z = D^-1 r for one row. Scalar Jacobi: one float4 (three inverses) per row; block
// Jacobi: three float4 per row (the rows of the inverse 3x3 block).
template <bool BLOCK>
__device__ __forceinline__ float4 apply_precond(const float *__restrict__ dinv4, int row, float4 r)
{
    if (BLOCK) {
        const float4 *d4 = reinterpret_cast<const float4 *>(dinv4);
        const float4 a = d4[3ll * row], b = d4[3ll * row + 1], c = d4[3ll * row + 2];
        return make_float4(a.x * r.x + a.y * r.y + a.z * r.z, b.x * r.x + b.y * r.y + b.z * r.z,
                           c.x * r.x + c.y * r.y + c.z * r.z, 0.f);
    }
    const float *d = dinv4 + 3ll * row;
    return make_float4(d[0] * r.x, d[1] * r.y, d[2] * r.z, 0.f);
}

__device__ __forceinline__ float dot3(float4 a, float4 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }

// The single-system PCG keeps x, r and the Jacobi inverse packed, three floats per row
// (12 bytes instead of 16: these vectors are never gathered, only streamed).
__device__ __forceinline__ float4 ld3(const float *__restrict__ a, int row)
{
    const float *p = a + 3ll * row;
    return make_float4(p[0], p[1], p[2], 0.f);
}
__device__ __forceinline__ void st3(float *__restrict__ a, int row, float4 v)
{
    float *p = a + 3ll * row;
    p[0] = v.x;
    p[1] = v.y;
    p[2] = v.z;
}

// Inverse of the diagonal (scalar entries, or the whole 3x3 block computed in FP64).
// The same pass validates the caller's pattern before any product reads it: row pointers
// non-decreasing within [0, nnzb] and every column index in [0, V) (PC_DERR_INDEX, mapped
// to PC_ERR_ARG; a bad row's entries are not read).
template <bool BLOCK>
__global__ void dinv_kernel(int V, int64_t nnzb, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const float *__restrict__ vals, float *__restrict__ dinv, uint32_t *err)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= V) return;
    const int k0 = rp[r], k1 = rp[r + 1];
    int s = -1;
    if (k0 < 0 || k1 < k0 || (int64_t)k1 > nnzb) {
        pc_set_err(err, PC_DERR_INDEX);
    } else {
        for (int k = k0; k < k1; ++k) {
            const int c = ci[k];
            if (c < 0 || c >= V) pc_set_err(err, PC_DERR_INDEX);
            if (c == r && s < 0) s = k;
        }
    }
    double B[9];
    for (int e = 0; e < 9; ++e) B[e] = s >= 0 ? (double)vals[9ll * s + e] : 0.0;
    bool ok = s >= 0 && B[0] > 0.0 && B[4] > 0.0 && B[8] > 0.0 && isfinite(B[0] + B[4] + B[8]);
    if (!BLOCK) {
        float *d = dinv + 3ll * r;  // packed: three floats per row
        d[0] = ok ? (float)(1.0 / B[0]) : 1.f;
        d[1] = ok ? (float)(1.0 / B[4]) : 1.f;
        d[2] = ok ? (float)(1.0 / B[8]) : 1.f;
    } else {
        float4 *dinv4 = reinterpret_cast<float4 *>(dinv);
        double c00 = B[4] * B[8] - B[5] * B[7], c01 = B[2] * B[7] - B[1] * B[8], c02 = B[1] * B[5] - B[2] * B[4];
        double c10 = B[5] * B[6] - B[3] * B[8], c11 = B[0] * B[8] - B[2] * B[6], c12 = B[2] * B[3] - B[0] * B[5];
        double c20 = B[3] * B[7] - B[4] * B[6], c21 = B[1] * B[6] - B[0] * B[7], c22 = B[0] * B[4] - B[1] * B[3];
        double det = B[0] * c00 + B[1] * c10 + B[2] * c20;
        ok = ok && det > 0.0 && isfinite(det);
        if (ok) {
            dinv4[3ll * r] = make_float4((float)(c00 / det), (float)(c01 / det), (float)(c02 / det), 0.f);
            dinv4[3ll * r + 1] = make_float4((float)(c10 / det), (float)(c11 / det), (float)(c12 / det), 0.f);
            dinv4[3ll * r + 2] = make_float4((float)(c20 / det), (float)(c21 / det), (float)(c22 / det), 0.f);
        } else {
            dinv4[3ll * r] = make_float4(1.f, 0.f, 0.f, 0.f);
            dinv4[3ll * r + 1] = make_float4(0.f, 1.f, 0.f, 0.f);
            dinv4[3ll * r + 2] = make_float4(0.f, 0.f, 1.f, 0.f);
        }
    }
    if (!ok) pc_set_err(err, PC_DERR_NONFINITE);
}

// ------------------------------------------------------------------------- vector kernels
//
// Internal PCG vectors are float4 per row (x, y, z, pad): one coalesced 16-byte access
// per row and array. Each thread sums its rows' dot-product terms in FP32; the sums
// across threads and blocks are FP64 (last_block_reduce).

// alpha = r.z / p.q with p.q the sum, in CTA order, of the n_pq partials the SpMV left in
// slot 3 (every CTA computes the same value; block 0 records pq and alpha). A
// non-positive or non-finite p.q gives alpha = 0; the last block then reports it.
__device__ __forceinline__ float pcg_alpha(const double *partials, int n_pq, pc_scalars *sc)
{
    __shared__ float s_alpha;
    const float2 *pf = reinterpret_cast<const float2 *>(partials);
    float hi[1] = {0.f}, lo[1] = {0.f};
    for (int i = threadIdx.x; i < n_pq; i += blockDim.x) {
        const float2 v = __ldcg(pf + (int64_t)i * RED_SLOTS + 3);
        pc_df_add(hi[0], lo[0], v.x, v.y);
    }
    pc_block_sum_df(hi, lo, 1);
    if (threadIdx.x == 0) {
        // the quotient in FP32, the precision the iteration uses it in (an FP64 division
        // in one thread is a long dependent chain on GB300's FP64 pipe)
        const float pq = __fadd_rn(hi[0], lo[0]);
        float alpha = (float)sc->rz / pq;
        if (!(pq > 0.f) || !isfinite(alpha)) alpha = 0.f;
        s_alpha = alpha;
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->pq = pc_df_value(hi[0], lo[0]);
        sc->alpha = (double)s_alpha;
    }
    return s_alpha;
}

// Launch shape of the update kernel (measured at paper scale: 4 rows in flight per thread
// and 2 CTAs per SM beat 1 x 8 by 14 us per iteration -- fewer CTAs also means fewer
// copies of alpha's reduction)
#ifndef UPD_UNROLL
#define UPD_UNROLL 4      // rows per thread in flight
#endif
#ifndef UPD_CTAS_PER_SM
#define UPD_CTAS_PER_SM 2
#endif
// the direction kernel is fastest in the plain shape (1 row per thread, 8 CTAs per SM)
#ifndef DIR_UNROLL
#define DIR_UNROLL 1
#endif
#ifndef DIR_CTAS_PER_SM
#define DIR_CTAS_PER_SM 8
#endif

// Per row: x += alpha p; r -= alpha q; z = D^-1 r; partial (r.z, r.r); the last block
// computes beta and applies the stop tests. Each thread keeps UPD_UNROLL rows in flight
// (all loads issued before any use), and the first rows' loads are issued before
// alpha's reduction so that their latencies overlap.
template <bool BLOCK>
__global__ void __launch_bounds__(EW_THREADS) pcg_update_kernel(int V, float *__restrict__ x4,
                                                                 const float4 *__restrict__ p4,
                                                                 float *__restrict__ r4,
                                                                 const float4 *__restrict__ q4,
                                                                 const float *__restrict__ dinv4,
                                                                 float4 *__restrict__ z4, double *partials,
                                                                 int n_pq, pc_scalars *sc)
{
    pdl_wait();
    if (sc->done) return;
    const int stride = gridDim.x * blockDim.x;
    const int first = blockIdx.x * blockDim.x + threadIdx.x;
    float4 p[UPD_UNROLL], q[UPD_UNROLL], x[UPD_UNROLL], r[UPD_UNROLL];
    auto load = [&](int base) {
#pragma unroll
        for (int u = 0; u < UPD_UNROLL; ++u) {
            const int row = base + u * stride;
            if (row < V) {
                p[u] = p4[row];
                q[u] = q4[row];
                x[u] = ld3(x4, row);
                r[u] = ld3(r4, row);
            }
        }
    };
    load(first);
    const float alpha = pcg_alpha(partials, n_pq, sc);
    float rz = 0.f, rr = 0.f;
    for (int base = first; base < V; base += UPD_UNROLL * stride) {
        if (base != first) load(base);
#pragma unroll
        for (int u = 0; u < UPD_UNROLL; ++u) {
            const int row = base + u * stride;
            if (row >= V) break;
            float4 xx = x[u], rv = r[u];
            xx.x = fmaf(alpha, p[u].x, xx.x);
            xx.y = fmaf(alpha, p[u].y, xx.y);
            xx.z = fmaf(alpha, p[u].z, xx.z);
            rv.x = fmaf(-alpha, q[u].x, rv.x);
            rv.y = fmaf(-alpha, q[u].y, rv.y);
            rv.z = fmaf(-alpha, q[u].z, rv.z);
            const float4 z = apply_precond<BLOCK>(dinv4, row, rv);
            st3(x4, row, xx);
            st3(r4, row, rv);
            z4[row] = z;
            rz += dot3(rv, z);
            rr += dot3(rv, rv);
        }
    }
    pdl_trigger();
    float hi[2] = {rz, rr}, lo[2] = {0.f, 0.f};
    if (last_block_reduce_df(hi, lo, 2, partials, &sc->counter) && threadIdx.x == 0) {
        const double rz_new = pc_df_value(hi[0], lo[0]), rr_new = pc_df_value(hi[1], lo[1]);
        const double pq = sc->pq;
        sc->beta = (double)(__fadd_rn(hi[0], lo[0]) / (float)sc->rz);  // FP32, as the direction step uses it
        sc->rz = rz_new;
        sc->rr = rr_new;
        sc->iter += 1;
        double v[2] = {rz_new, rr_new};
        if (!(pq > 0.0) || !isfinite(sc->alpha)) {
            sc->status = PC_ERR_NONFINITE;
            sc->done = 1;
        } else if (!isfinite(v[1]) || !isfinite(sc->beta)) {
            sc->status = PC_ERR_NONFINITE;
            sc->done = 1;
        } else if (v[1] <= sc->tol2) {
            sc->status = PC_OK;
            sc->done = 1;
        } else if (sc->iter >= sc->max_iter) {
            sc->status = PC_ERR_NOT_CONVERGED;
            sc->done = 1;
        }
    }
}

// Per row: r = b - q (q = A x0 as float[V][3]), z = D^-1 r, p = 0, increment x = 0;
// partial (r.z, r.r, b.b); the last block initialises the scalars.
template <bool BLOCK>
__global__ void __launch_bounds__(EW_THREADS) pcg_init_kernel(int V, const float *__restrict__ b,
                                                               const float *__restrict__ q,
                                                               float *__restrict__ r4,
                                                               const float *__restrict__ dinv4,
                                                               float4 *__restrict__ z4, float4 *__restrict__ p4,
                                                               float *__restrict__ x4, double tol, int max_iter,
                                                               double *partials, pc_scalars *sc, int fused)
{
    double rz = 0.0, rr = 0.0, bb = 0.0;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < V; row += gridDim.x * blockDim.x) {
        const float b0 = b[3ll * row], b1 = b[3ll * row + 1], b2 = b[3ll * row + 2];
        const float4 r = make_float4(b0 - q[3ll * row], b1 - q[3ll * row + 1], b2 - q[3ll * row + 2], 0.f);
        const float4 z = apply_precond<BLOCK>(dinv4, row, r);
        st3(r4, row, r);
        z4[row] = z;
        // the fused update leaves p ready for the next product: start from p = z
        p4[row] = fused ? z : make_float4(0.f, 0.f, 0.f, 0.f);
        st3(x4, row, make_float4(0.f, 0.f, 0.f, 0.f));
        rz += (double)dot3(r, z);
        rr += (double)dot3(r, r);
        bb += (double)b0 * b0 + (double)b1 * b1 + (double)b2 * b2;
    }
    double v[3] = {rz, rr, bb};
    if (last_block_reduce(v, 3, partials, &sc->counter) && threadIdx.x == 0) {
        sc->rz = v[0];
        sc->rr = v[1];
        sc->bb = v[2];
        sc->tol2 = tol * tol * v[2];
        sc->alpha = 0.0;
        sc->beta = 0.0;
        sc->pq = 0.0;
        sc->iter = 0;
        sc->max_iter = max_iter;
        sc->status = PC_OK;
        sc->done = 0;
        if (!isfinite(v[2]) || !isfinite(v[1])) {
            sc->status = PC_ERR_NONFINITE;
            sc->done = 1;
        } else if (v[1] <= sc->tol2) {
            sc->done = 1;
        } else if (max_iter <= 0) {
            sc->status = PC_ERR_NOT_CONVERGED;
            sc->done = 1;
        }
    }
}

// (A x)_row in FP64 from FP32 blocks, x in FP64 or FP32 (standard or difference form).
template <typename XT, bool DIFF>
__device__ __forceinline__ void row_product64(int row, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                              const float *__restrict__ vals, const float *__restrict__ dres,
                                              const XT *__restrict__ x, double acc[3])
{
    double xj[3] = {(double)x[3ll * row], (double)x[3ll * row + 1], (double)x[3ll * row + 2]};
    acc[0] = acc[1] = acc[2] = 0.0;
    for (int k = rp[row]; k < rp[row + 1]; ++k) {
        int c = ci[k];
        if (DIFF && c == row) continue;
        const float *B = vals + 9ll * k;
        double xc[3] = {(double)x[3ll * c], (double)x[3ll * c + 1], (double)x[3ll * c + 2]};
        if (DIFF)
            for (int d = 0; d < 3; ++d) xc[d] -= xj[d];
        for (int a2 = 0; a2 < 3; ++a2)
            acc[a2] += (double)B[3 * a2] * xc[0] + (double)B[3 * a2 + 1] * xc[1] + (double)B[3 * a2 + 2] * xc[2];
    }
    if (DIFF) {
        const float *D = dres + 9ll * row;
        for (int a2 = 0; a2 < 3; ++a2)
            acc[a2] += (double)D[3 * a2] * xj[0] + (double)D[3 * a2 + 1] * xj[1] + (double)D[3 * a2 + 2] * xj[2];
    }
}

// FP64 residual of an FP32 vector x: partial (r.r, b.b) only (reporting).
template <bool DIFF>
__global__ void __launch_bounds__(EW_THREADS) residual_check_kernel(int V, const int32_t *__restrict__ rp,
                                                                    const int32_t *__restrict__ ci,
                                                                    const float *__restrict__ vals,
                                                                    const float *__restrict__ dres,
                                                                    const float *__restrict__ b,
                                                                    const float *__restrict__ x, double *partials,
                                                                    pc_scalars *sc)
{
    double rr = 0.0, bb = 0.0;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < V; row += gridDim.x * blockDim.x) {
        double acc[3];
        row_product64<float, DIFF>(row, rp, ci, vals, dres, x, acc);
        for (int a2 = 0; a2 < 3; ++a2) {
            double bv = (double)b[3ll * row + a2];
            double rv = bv - acc[a2];
            rr += rv * rv;
            bb += bv * bv;
        }
    }
    double v[2] = {rr, bb};
    if (last_block_reduce(v, 2, partials, &sc->counter) && threadIdx.x == 0) {
        sc->rr = v[0];
        sc->bb = v[1];
    }
}

// ------------------------------------------------------------------------- fused update + direction

// One kernel per iteration instead of two: the update (x += alpha p, r -= alpha q,
// z = M^-1 r, partial r.z and r.r), a grid-wide barrier, then every CTA sums the partials
// in the same order, forms beta and applies p = z + beta p to its own rows from
// registers. z never goes to memory and p is read once, so an iteration moves 48 bytes
// per row less. Each thread owns rows first + u * stride (u < R <= FU_ROWS) and keeps
// their z and p across the barrier; the grid is sized so that all CTAs are resident at
// once (checked against the occupancy on the host). The barrier's waits are bounded; a
// timeout ends the solve with PC_ERR_TIMEOUT.
#define FU_THREADS 256
#ifndef FU_ROWS
#define FU_ROWS 12  // rows a thread carries across the barrier
#endif
#ifndef FU_CTAS_PER_SM
#define FU_CTAS_PER_SM 2
#endif
#ifndef FU_GROUP
#define FU_GROUP 2  // rows whose loads are in flight together
#endif
static_assert(FU_ROWS % FU_GROUP == 0, "a thread's rows come in whole groups");

struct pc_fuse_bar {
    unsigned long long count;  // arrivals at the grid barrier (pc_grid_barrier; zeroed per solve)
    uint64_t pad;
};

template <bool BLOCK>
__global__ void __launch_bounds__(FU_THREADS, FU_CTAS_PER_SM) pcg_update_dir_kernel(
    int V, int R, float *__restrict__ x4, float4 *__restrict__ p4, float *__restrict__ r4,
    const float4 *__restrict__ q4, const float *__restrict__ dinv4, double *partials, int n_pq, pc_scalars *sc,
    pc_fuse_bar *bar, uint32_t *err, long long wait_budget)
{
    pdl_wait();
    if (sc->done) return;
    const double rz_old = sc->rz;  // read before the barrier; block 0 rewrites it after
    const int stride = gridDim.x * blockDim.x;
    const int first = blockIdx.x * blockDim.x + threadIdx.x;
    float zs[FU_ROWS][3], ps[FU_ROWS][3];
    float alpha = 0.f, rz = 0.f, rr = 0.f;
#pragma unroll
    for (int g = 0; g < FU_ROWS; g += FU_GROUP) {
        if (g >= R) break;
        float4 p[FU_GROUP], q[FU_GROUP], x[FU_GROUP], r[FU_GROUP];
#pragma unroll
        for (int u = 0; u < FU_GROUP; ++u) {
            const int row = first + (g + u) * stride;
            if (g + u < R && row < V) {
                p[u] = p4[row];
                q[u] = q4[row];
                x[u] = ld3(x4, row);
                r[u] = ld3(r4, row);
            }
        }
        if (g == 0) alpha = pcg_alpha(partials, n_pq, sc);  // overlaps the first loads
#pragma unroll
        for (int u = 0; u < FU_GROUP; ++u) {
            const int row = first + (g + u) * stride;
            zs[g + u][0] = zs[g + u][1] = zs[g + u][2] = 0.f;
            ps[g + u][0] = ps[g + u][1] = ps[g + u][2] = 0.f;
            if (g + u < R && row < V) {
                float4 xx = x[u], rv = r[u];
                xx.x = fmaf(alpha, p[u].x, xx.x);
                xx.y = fmaf(alpha, p[u].y, xx.y);
                xx.z = fmaf(alpha, p[u].z, xx.z);
                rv.x = fmaf(-alpha, q[u].x, rv.x);
                rv.y = fmaf(-alpha, q[u].y, rv.y);
                rv.z = fmaf(-alpha, q[u].z, rv.z);
                const float4 z = apply_precond<BLOCK>(dinv4, row, rv);
                st3(x4, row, xx);
                st3(r4, row, rv);
                rz += dot3(rv, z);
                rr += dot3(rv, rv);
                zs[g + u][0] = z.x;
                zs[g + u][1] = z.y;
                zs[g + u][2] = z.z;
                ps[g + u][0] = p[u].x;
                ps[g + u][1] = p[u].y;
                ps[g + u][2] = p[u].z;
            }
        }
    }
    float2 *pf = reinterpret_cast<float2 *>(partials);
    {
        float hi[2] = {rz, rr}, lo[2] = {0.f, 0.f};
        pc_block_sum_df(hi, lo, 2);
        if (threadIdx.x == 0) {
            pf[(int64_t)blockIdx.x * RED_SLOTS] = make_float2(hi[0], lo[0]);
            pf[(int64_t)blockIdx.x * RED_SLOTS + 1] = make_float2(hi[1], lo[1]);
        }
    }
    if (!pc_grid_barrier(&bar->count, wait_budget)) {
        // a timeout outranks any status block 0 may record in this launch
        if (threadIdx.x == 0) {
            atomicOr(err, PC_DERR_TIMEOUT);
            atomicExch(&sc->status, (int32_t)PC_ERR_TIMEOUT);
            sc->done = 1;
        }
        return;
    }
    // every CTA: the grid's r.z and r.r, summed in block order (the same value everywhere)
    float th[2] = {0.f, 0.f}, tl[2] = {0.f, 0.f};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const float2 a0 = __ldcg(pf + (int64_t)b * RED_SLOTS), a1 = __ldcg(pf + (int64_t)b * RED_SLOTS + 1);
        pc_df_add(th[0], tl[0], a0.x, a0.y);
        pc_df_add(th[1], tl[1], a1.x, a1.y);
    }
    pc_block_sum_df(th, tl, 2);
    __shared__ float s_beta;
    if (threadIdx.x == 0) s_beta = __fadd_rn(th[0], tl[0]) / (float)rz_old;  // FP32, as it is used
    __syncthreads();
    const float beta = s_beta;
    // the scalars' FP64 bookkeeping while the other threads take the direction step
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double rz_new = pc_df_value(th[0], tl[0]), rr = pc_df_value(th[1], tl[1]);
        const double pq = sc->pq;
        sc->beta = (double)beta;
        sc->rz = rz_new;
        sc->rr = rr;
        sc->iter += 1;
        // status changes only from PC_OK, so a timeout another CTA recorded stays
        int32_t st = PC_OK;
        if (!(pq > 0.0) || !isfinite(sc->alpha)) st = PC_ERR_NONFINITE;
        else if (!isfinite(rr) || !isfinite(beta)) st = PC_ERR_NONFINITE;
        else if (sc->iter >= sc->max_iter && !(rr <= sc->tol2)) st = PC_ERR_NOT_CONVERGED;
        if (st != PC_OK) atomicCAS(&sc->status, (int32_t)PC_OK, st);
        if (st != PC_OK || rr <= sc->tol2) sc->done = 1;
    }
    // the direction step even when this iteration stopped the solve: a residual
    // replacement that resumes it corrects p from z_old to the replaced z
    if (isfinite(beta)) {
#pragma unroll
        for (int u = 0; u < FU_ROWS; ++u) {
            if (u >= R) break;
            const int row = first + u * stride;
            if (row < V)
                p4[row] = make_float4(fmaf(beta, ps[u][0], zs[u][0]), fmaf(beta, ps[u][1], zs[u][1]),
                                      fmaf(beta, ps[u][2], zs[u][2]), 0.f);
        }
    }
    pdl_trigger();
}

// Residual replacement: r64 = b - A x64 in FP64; r = (float) r64, z = D^-1 r; partial
// (r.z, r64.r64, b.b). The last block installs r.z and the FP64 residual as the
// iteration's scalars (keeping beta and the search direction), and either starts the
// solve (`first`: p = 0) or decides whether it has converged.
template <bool DIFF, bool BLOCK>
__global__ void __launch_bounds__(EW_THREADS) residual_replace_kernel(
    int V, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const float *__restrict__ vals,
    const float *__restrict__ dres, const float *__restrict__ b, const double *__restrict__ x64,
    const float *__restrict__ dinv4, float *__restrict__ r4, float4 *__restrict__ z4, float4 *__restrict__ p4,
    int first, double tol, int max_iter, double *partials, pc_scalars *sc, int fused)
{
    double rz = 0.0, rr = 0.0, bb = 0.0;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < V; row += gridDim.x * blockDim.x) {
        double acc[3];
        row_product64<double, DIFF>(row, rp, ci, vals, dres, x64, acc);
        float rf[3];
        for (int a2 = 0; a2 < 3; ++a2) {
            double bv = (double)b[3ll * row + a2];
            double rv = bv - acc[a2];
            rr += rv * rv;
            bb += bv * bv;
            rf[a2] = (float)rv;
        }
        const float4 r = make_float4(rf[0], rf[1], rf[2], 0.f);
        const float4 z = apply_precond<BLOCK>(dinv4, row, r);
        if (fused) {
            // p already holds z_old + beta p_prev (the fused update applied the direction
            // step): swap z_old for the replaced z, p = z + beta p_prev as without fusion
            if (first) {
                p4[row] = z;
            } else {
                const float4 zo = apply_precond<BLOCK>(dinv4, row, ld3(r4, row));
                float4 pv = p4[row];
                pv.x += z.x - zo.x;
                pv.y += z.y - zo.y;
                pv.z += z.z - zo.z;
                p4[row] = pv;
            }
        } else if (first) {
            p4[row] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        st3(r4, row, r);
        z4[row] = z;
        rz += (double)dot3(r, z);
    }
    double v[3] = {rz, rr, bb};
    if (last_block_reduce(v, 3, partials, &sc->counter) && threadIdx.x == 0) {
        sc->rz = v[0];
        sc->rr = v[1];
        if (first) {
            sc->bb = v[2];
            sc->tol2 = tol * tol * v[2];
            sc->alpha = 0.0;
            sc->beta = 0.0;
            sc->pq = 0.0;
            sc->iter = 0;
            sc->max_iter = max_iter;
        }
        sc->status = PC_OK;
        sc->done = 0;
        if (!isfinite(v[1]) || !isfinite(v[2])) {
            sc->status = PC_ERR_NONFINITE;
            sc->done = 1;
        } else if (v[1] <= sc->tol2) {
            sc->done = 1;
        } else if (sc->iter >= sc->max_iter) {
            sc->status = PC_ERR_NOT_CONVERGED;
            sc->done = 1;
        }
    }
}

// x64 += increment; increment = 0 (per row, float4 increment)
__global__ void fold_kernel(int V, float *x4, double *x64)
{
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < V; row += gridDim.x * blockDim.x) {
        const float4 d = ld3(x4, row);
        x64[3ll * row] += (double)d.x;
        x64[3ll * row + 1] += (double)d.y;
        x64[3ll * row + 2] += (double)d.z;
        st3(x4, row, make_float4(0.f, 0.f, 0.f, 0.f));
    }
}
// dv += increment (FP32 solve)
__global__ void add_increment_kernel(int V, const float *x4, float *dv)
{
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < V; row += gridDim.x * blockDim.x) {
        const float4 d = ld3(x4, row);
        dv[3ll * row] += d.x;
        dv[3ll * row + 1] += d.y;
        dv[3ll * row + 2] += d.z;
    }
}
__global__ void f64_to_f32_kernel(int64_t n, const double *a, float *o)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = (float)a[i];
}
__global__ void f32_to_f64_kernel(int64_t n, const float *a, double *o)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = (double)a[i];
}
__global__ void state_update_kernel(int64_t n, float *x, float *v, const float *dv, float h)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float vi = v[i] + dv[i];
        v[i] = vi;
        x[i] = fmaf(h, vi, x[i]);
    }
}

// ------------------------------------------------------------------------- host side

static int tile_grid(const pc_ctx *c, int ctas_per_sm)
{
    int tiles = (c->V + SP_ROWS - 1) / SP_ROWS;
    int g = c->num_sms * ctas_per_sm;
    return tiles < g ? (tiles > 0 ? tiles : 1) : g;
}
// The product's grid for stages of `capr` blocks per row (SP_CAP_PER_ROW or SP_CAPR_WIDE).
static int spmv_grid(const pc_ctx *c, int capr)
{
    return tile_grid(c, capr <= SP_CAP_PER_ROW ? SpShape<SP_CAP_PER_ROW>::ctas_per_sm
                                               : SpShape<SP_CAPR_WIDE>::ctas_per_sm);
}

// Dynamic shared memory of every instantiation of the product (set once per device).
static pc_status spmv_set_smem()
{
    const int n = SpShape<SP_CAP_PER_ROW>::smem_bytes, w = SpShape<SP_CAPR_WIDE>::smem_bytes;
    PC_CUDA_TRY(cudaFuncSetAttribute(spmv_kernel<true, true, SP_CAP_PER_ROW>, cudaFuncAttributeMaxDynamicSharedMemorySize, n));
    PC_CUDA_TRY(cudaFuncSetAttribute(spmv_kernel<false, true, SP_CAP_PER_ROW>, cudaFuncAttributeMaxDynamicSharedMemorySize, n));
    PC_CUDA_TRY(cudaFuncSetAttribute(spmv_kernel<true, true, SP_CAPR_WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, w));
    PC_CUDA_TRY(cudaFuncSetAttribute(spmv_kernel<false, true, SP_CAPR_WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, w));
    PC_CUDA_TRY(cudaFuncSetAttribute(spmv_kernel<true, false, SP_CAPR_WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, w));
    PC_CUDA_TRY(cudaFuncSetAttribute(spmv_kernel<false, false, SP_CAPR_WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, w));
    return PC_OK;
}

// The largest tile (blocks in SP_ROWS consecutive rows) of a BSR pattern, into *out
// (zeroed by the caller) with one atomicMax per warp.
__global__ void tile_max_kernel(int V, const int32_t *__restrict__ rp, long long *out)
{
    const int ntiles = (V + SP_ROWS - 1) / SP_ROWS;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    long long m = 0;
    if (t < ntiles) {
        const int r0 = t * SP_ROWS, r1 = min(r0 + SP_ROWS, V);
        m = (long long)rp[r1] - rp[r0];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(out, m);
}
static int sym_grid(const pc_ctx *c) { return tile_grid(c, SY_CTAS_PER_SM); }
static int shaped_grid(const pc_ctx *c, int64_t n, int ctas_per_sm)
{
    int64_t b = (n + EW_THREADS - 1) / EW_THREADS;
    int64_t g = (int64_t)c->num_sms * ctas_per_sm;
    return (int)(b < g ? (b > 0 ? b : 1) : g);
}
static int upd_grid(const pc_ctx *c, int64_t n) { return shaped_grid(c, n, UPD_CTAS_PER_SM); }
static int dir_grid(const pc_ctx *c, int64_t n) { return shaped_grid(c, n, DIR_CTAS_PER_SM); }
static int ew_grid(const pc_ctx *c, int64_t n)
{
    int64_t b = (n + EW_THREADS - 1) / EW_THREADS;
    int64_t g = (int64_t)c->num_sms * 8;
    if (b < 1) b = 1;
    return (int)(b < g ? b : g);
}

pc_status pc_solver_alloc(pc_ctx *c)
{
    const int64_t n = 3ll * c->V;
    PC_CUDA_TRY(cudaMalloc(&c->r, sizeof(float4) * c->V));
    PC_CUDA_TRY(cudaMalloc(&c->z, sizeof(float4) * c->V));
    PC_CUDA_TRY(cudaMalloc(&c->p0, sizeof(float4) * c->V));
    PC_CUDA_TRY(cudaMalloc(&c->q, sizeof(float4) * c->V));
    PC_CUDA_TRY(cudaMalloc(&c->dinv, sizeof(float4) * 3 * c->V));
    PC_CUDA_TRY(cudaMalloc(&c->dsc, sizeof(float) * (size_t)(c->V > 0 ? c->V : 1)));
    PC_CUDA_TRY(cudaMalloc(&c->fbar, sizeof(pc_fuse_bar)));
    PC_CUDA_TRY(cudaMemset(c->fbar, 0, sizeof(pc_fuse_bar)));
    PC_CUDA_TRY(cudaMalloc(&c->dtmp, sizeof(float4) * c->V));
    PC_CUDA_TRY(cudaMalloc(&c->rhs32, sizeof(float) * n));
    PC_CUDA_TRY(cudaMalloc(&c->x64, sizeof(double) * n));
    PC_CUDA_TRY(cudaMalloc(&c->r64, sizeof(double) * n));
    c->max_red_blocks = c->num_sms * 16;
    PC_CUDA_TRY(cudaMalloc(&c->partials, sizeof(double) * RED_SLOTS * c->max_red_blocks));
    PC_CUDA_TRY(cudaMalloc(&c->sc, sizeof(pc_scalars)));
    PC_CUDA_TRY(cudaMemset(c->sc, 0, sizeof(pc_scalars)));
    PC_CUDA_TRY(cudaMallocHost(&c->sc_host, sizeof(pc_scalars)));
    PC_TRY(spmv_set_smem());
    PC_CUDA_TRY(cudaFuncSetAttribute(spmv_sym_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SY_SMEM_BYTES));
    PC_CUDA_TRY(cudaFuncSetAttribute(spmv_sym_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SY_SMEM_BYTES));
    if (c->A_cap > 0) {  // symmetric storage for systems up to the step-system capacity
        c->sym_cap = c->A_cap;
        PC_CUDA_TRY(cudaMalloc(&c->sym_urp, sizeof(int32_t) * (c->V + 2ll)));
        PC_CUDA_TRY(cudaMalloc(&c->sym_lrp, sizeof(int32_t) * (c->V + 2ll)));
        PC_CUDA_TRY(cudaMalloc(&c->sym_dpos, sizeof(int32_t) * (size_t)c->V));
        PC_CUDA_TRY(cudaMalloc(&c->sym_ucnt, sizeof(int32_t) * (c->V + 1ll)));
        PC_CUDA_TRY(cudaMalloc(&c->sym_lcnt, sizeof(int32_t) * (c->V + 1ll)));
        PC_CUDA_TRY(cudaMalloc(&c->sym_uci, sizeof(int32_t) * (size_t)(c->sym_cap + 4)));
        PC_CUDA_TRY(cudaMalloc(&c->sym_lcol, sizeof(int32_t) * (size_t)(c->sym_cap + 4)));
        PC_CUDA_TRY(cudaMalloc(&c->sym_lsrc, sizeof(int32_t) * (size_t)(c->sym_cap + 4)));
        PC_CUDA_TRY(cudaMalloc(&c->sym_uvals, sizeof(float) * (size_t)(9 * c->sym_cap + 16)));
        PC_CUDA_TRY(cudaMemset(c->sym_uvals, 0, sizeof(float) * (size_t)(9 * c->sym_cap + 16)));
        PC_CUDA_TRY(cudaMemset(c->sym_uci, 0, sizeof(int32_t) * (size_t)(c->sym_cap + 4)));
        PC_CUDA_TRY(cudaMemset(c->sym_lcol, 0, sizeof(int32_t) * (size_t)(c->sym_cap + 4)));
        PC_CUDA_TRY(cudaMemset(c->sym_lsrc, 0, sizeof(int32_t) * (size_t)(c->sym_cap + 4)));
        // sliced ELL: in a window sorted by descending length each slice is at most as wide
        // as the mean row of the slice before it, so a window needs at most its blocks / 32
        // positions plus the width of its first slice; the capacity allows 64 for that
        // (longer rows in the first slice of a window make the solve fall back to BSR)
        const int64_t nwin = (c->V + SL_SIGMA - 1) / SL_SIGMA;
        c->sell_nslices = (int32_t)(nwin * (SL_SIGMA / SL_C));
        c->sell_cap = c->A_cap / SL_C + 64 * nwin + c->sell_nslices;
        PC_CUDA_TRY(cudaMalloc(&c->sell_perm, sizeof(int32_t) * (size_t)nwin * SL_SIGMA));
        PC_CUDA_TRY(cudaMalloc(&c->sell_width, sizeof(int32_t) * (c->sell_nslices + 1ll)));
        PC_CUDA_TRY(cudaMalloc(&c->sell_base, sizeof(int32_t) * (c->sell_nslices + 1ll)));
        PC_CUDA_TRY(cudaMalloc(&c->sell_dpos, sizeof(int32_t) * (size_t)c->V));
        PC_CUDA_TRY(cudaMalloc(&c->sell_data, sizeof(uint32_t) * SL_WORDS * (size_t)c->sell_cap));
        PC_CUDA_TRY(cudaMalloc(&c->sell_diag, sizeof(float) * 9 * (size_t)c->V));
        // off-diagonal BSR: at most the step system's blocks
        c->od_cap = c->A_cap;
        PC_CUDA_TRY(cudaMalloc(&c->od_rp, sizeof(int32_t) * (c->V + 1ll)));
        PC_CUDA_TRY(cudaMalloc(&c->od_cnt, sizeof(int32_t) * (c->V + 1ll)));
        PC_CUDA_TRY(cudaMalloc(&c->od_dpos, sizeof(int32_t) * (size_t)c->V));
        PC_CUDA_TRY(cudaMalloc(&c->od_ci, sizeof(int32_t) * (size_t)(c->od_cap + 4)));
        PC_CUDA_TRY(cudaMalloc(&c->od_vals, sizeof(float) * (size_t)(9 * c->od_cap + 16)));
        PC_CUDA_TRY(cudaMemset(c->od_ci, 0, sizeof(int32_t) * (size_t)(c->od_cap + 4)));
        PC_CUDA_TRY(cudaMemset(c->od_vals, 0, sizeof(float) * (size_t)(9 * c->od_cap + 16)));
    }
    for (int i = 0; i < 8; ++i) PC_CUDA_TRY(cudaEventCreate(&c->ev[i]));
    c->ev_used = 8;
    return PC_OK;
}

static pc_status check_bsr(const pc_bsr *A, const float *vals)
{
    if (!A || !A->row_ptr || !A->col_idx || !vals) return PC_ERR_ARG;
    if ((A->cap & 3) != 0 || A->nnzb < 0 || A->nnzb > A->cap) return PC_ERR_ARG;
    if (!pc_aligned16(A->col_idx) || !pc_aligned16(vals)) return PC_ERR_ARG;
    return PC_OK;
}

// PCG products take the stage width the solve chose; plain products (y = A x) always
// the wide stages, which no tile of an assembled system outgrows in practice.
static pc_status launch_spmv(pc_ctx *c, const SpmvArgs &a, bool diff, bool pcg, cudaStream_t st,
                             int capr = SP_CAPR_WIDE)
{
    const int g = spmv_grid(c, pcg ? capr : SP_CAPR_WIDE);
    const int n = SpShape<SP_CAP_PER_ROW>::smem_bytes, w = SpShape<SP_CAPR_WIDE>::smem_bytes;
    if (pcg && capr <= SP_CAP_PER_ROW) {
        if (diff) PC_LAUNCH_PDL(c, (spmv_kernel<true, true, SP_CAP_PER_ROW>), g, SP_THREADS, n, st, a);
        else PC_LAUNCH_PDL(c, (spmv_kernel<false, true, SP_CAP_PER_ROW>), g, SP_THREADS, n, st, a);
    } else if (pcg) {
        if (diff) PC_LAUNCH_PDL(c, (spmv_kernel<true, true, SP_CAPR_WIDE>), g, SP_THREADS, w, st, a);
        else PC_LAUNCH_PDL(c, (spmv_kernel<false, true, SP_CAPR_WIDE>), g, SP_THREADS, w, st, a);
    } else {
        if (diff) PC_LAUNCH(c, (spmv_kernel<true, false, SP_CAPR_WIDE>), g, SP_THREADS, w, st, a);
        else PC_LAUNCH(c, (spmv_kernel<false, false, SP_CAPR_WIDE>), g, SP_THREADS, w, st, a);
    }
    return PC_OK;
}

extern "C" pc_status pc_bsr_spmv(pc_ctx *ctx, const pc_bsr *A, const float *vals, const float *dres, const float *x,
                                 float *y, void *stream)
{
    if (!ctx || !x || !y) return PC_ERR_ARG;
    PC_TRY(check_bsr(A, vals));
    SpmvArgs a{};
    a.V = ctx->V;
    a.rp = A->row_ptr;
    a.ci = A->col_idx;
    a.vals = vals;
    a.dres = dres;
    a.xin = x;
    a.y = y;
    a.err = ctx->d_err;
    return launch_spmv(ctx, a, dres != nullptr, false, (cudaStream_t)stream);
}

extern "C" void pc_default_solve_opts(pc_solve_opts *o)
{
    if (!o) return;
    o->tol = 1e-6;
    o->max_iter = 20000;
    o->precision = PC_PREC_FP32;
    o->refresh = 1e-2;
    o->refresh_every = 1000;
    o->check_every = 32;
    o->precond = PC_PRECOND_JACOBI;
    o->storage = PC_STORAGE_OFFDIAG;
    o->fuse = 1;
    o->schedule = PC_SCHED_AUTO;
}

struct SolveCtx {
    pc_ctx *c;
    const pc_bsr *A;
    const float *vals, *dres, *b;
    bool diff, block;
    cudaStream_t st;
    bool sym;   // the products read the symmetric storage
    bool sell;  // the products read the sliced-ELL storage
    bool offdiag;  // the products read the BSR copy without diagonal blocks
    bool fuse;     // update and direction in one kernel (pcg_update_dir_kernel)
    int fu_grid, fu_rows;
    int capr = SP_CAPR_WIDE;  // the product's stage width (blocks per row)
};

// ------------------------------------------------------------------------- symmetric storage

// Per row: the diagonal's position in the full row (binary search; missing -> error bit),
// the counts of upper (col >= row) and lower blocks.
__global__ void sym_count_kernel(int V, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                 int32_t *dpos, int32_t *ucnt, int32_t *lcnt, uint32_t *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > V) return;
    if (i == V) {
        ucnt[V] = 0;
        lcnt[V] = 0;
        return;
    }
    int lo = rp[i], hi = rp[i + 1];
    const int end = hi;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ci[mid] < i) lo = mid + 1;
        else hi = mid;
    }
    if (lo >= end || ci[lo] != i) {
        pc_set_err(err, PC_DERR_INDEX);
        lo = rp[i];
    }
    dpos[i] = lo;
    ucnt[i] = end - lo;
    lcnt[i] = lo - rp[i];
}

// Upper blocks copied in row order; each lower block (i, j) refers to block (j, i) of
// row j's upper part (binary search in row j; missing -> error bit: not symmetric).
__global__ void sym_fill_kernel(int V, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                const float *__restrict__ vals, const int32_t *__restrict__ dpos,
                                const int32_t *__restrict__ urp, const int32_t *__restrict__ lrp, int64_t cap,
                                int32_t *uci, float *uvals, int32_t *lcol, int32_t *lsrc, uint32_t *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V) return;
    const int d = dpos[i];
    if (urp[i + 1] > cap || lrp[i + 1] > cap) {
        pc_set_err(err, PC_DERR_INDEX);
        return;
    }
    for (int k = d; k < rp[i + 1]; ++k) {
        const int o = urp[i] + (k - d);
        uci[o] = ci[k];
        for (int e = 0; e < 9; ++e) uvals[9ll * o + e] = vals[9ll * k + e];
    }
    for (int k = rp[i]; k < d; ++k) {
        const int jj = ci[k];
        int lo = rp[jj], hi = rp[jj + 1];
        const int end = hi;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (ci[mid] < i) lo = mid + 1;
            else hi = mid;
        }
        const int o = lrp[i] + (k - rp[i]);
        if (lo >= end || ci[lo] != i || lo < dpos[jj]) {
            pc_set_err(err, PC_DERR_INDEX);
            lcol[o] = jj;
            lsrc[o] = urp[jj];
            continue;
        }
        lcol[o] = jj;
        lsrc[o] = urp[jj] + (lo - dpos[jj]);
    }
}

// Build the symmetric storage of A (returns false, leaving the error bits clear, when
// the pattern has no diagonal somewhere or is not symmetric).
static pc_status build_sym(pc_ctx *c, const pc_bsr *A, const float *vals, bool *ok, cudaStream_t st)
{
    *ok = false;
    const int V = c->V;
    if (c->sym_cap <= 0 || A->nnzb > c->sym_cap) return PC_OK;
    PC_LAUNCH(c, sym_count_kernel, pc_blocks(V + 1ll, 256), 256, 0, st, V, A->row_ptr, A->col_idx, c->sym_dpos,
              c->sym_ucnt, c->sym_lcnt, c->d_err);
    PC_TRY(pc_exclusive_scan(c, c->sym_ucnt, c->sym_urp, V, st));
    PC_TRY(pc_exclusive_scan(c, c->sym_lcnt, c->sym_lrp, V, st));
    PC_LAUNCH(c, sym_fill_kernel, pc_blocks(V, 128), 128, 0, st, V, A->row_ptr, A->col_idx, vals, c->sym_dpos,
              c->sym_urp, c->sym_lrp, c->sym_cap, c->sym_uci, c->sym_uvals, c->sym_lcol, c->sym_lsrc, c->d_err);
    // every lower block found its mirror (checked in the fill); equal counts of lower and
    // off-diagonal upper blocks make that map a bijection: the pattern is symmetric
    PC_CUDA_TRY(cudaMemcpyAsync(c->h_count, c->sym_urp + V, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaMemcpyAsync(reinterpret_cast<int32_t *>(c->h_count) + 1, c->sym_lrp + V, sizeof(int32_t),
                                cudaMemcpyDeviceToHost, st));
    uint32_t bits = 0;
    PC_TRY(pc_read_errors(c, st, &bits));
    const int32_t n_up = reinterpret_cast<int32_t *>(c->h_count)[0], n_lo = reinterpret_cast<int32_t *>(c->h_count)[1];
    if (bits || n_up - V != n_lo) {
        PC_CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), st));
        return PC_OK;
    }
    *ok = true;
    return PC_OK;
}

// ------------------------------------------------------------------------- sliced ELL

// Build the sliced-ELL storage of A (returns false, error bits clear, when it does not
// fit the context's capacity; the solve then reads the BSR matrix).
static pc_status build_sell(pc_ctx *c, const pc_bsr *A, const float *vals, bool *ok, cudaStream_t st)
{
    *ok = false;
    const int V = c->V;
    if (c->sell_cap <= 0 || !c->sell_data) return PC_OK;
    const int nwin = c->sell_nslices / (SL_SIGMA / SL_C);
    PC_LAUNCH(c, sell_sort_kernel, nwin, SL_SIGMA, 0, st, V, A->row_ptr, A->col_idx, c->sell_perm, c->sell_width,
              c->sell_dpos);
    PC_TRY(pc_exclusive_scan(c, c->sell_width, c->sell_base, c->sell_nslices, st));
    PC_CUDA_TRY(cudaMemcpyAsync(c->h_count, c->sell_base + c->sell_nslices, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    const int32_t total = reinterpret_cast<int32_t *>(c->h_count)[0];
    if (total < 0 || total > c->sell_cap) return PC_OK;
    PC_LAUNCH(c, sell_fill_kernel, pc_blocks((int64_t)c->sell_nslices * 32, 256), 256, 0, st, V, c->sell_nslices,
              A->row_ptr, A->col_idx, vals, c->sell_perm, c->sell_width, c->sell_base, c->sell_dpos, c->sell_cap,
              c->sell_data, c->sell_diag, c->d_err);
    uint32_t bits = 0;
    PC_TRY(pc_read_errors(c, st, &bits));
    if (bits) {
        PC_CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), st));
        return PC_OK;
    }
    *ok = true;
    return PC_OK;
}

// ------------------------------------------------------------------------- scalar diagonals

// dsc[i] = s when the difference-form diagonal of row i is exactly s I with s > 0 (every
// row away from pins: its lumped mass term), else -1 (the product then reads all nine
// entries). The product is bitwise the same either way.
__global__ void dsc_kernel(int V, const float *__restrict__ dres, float *__restrict__ dsc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V) return;
    const float *D = dres + 9ll * i;
    const bool scalar = D[1] == 0.f && D[2] == 0.f && D[3] == 0.f && D[5] == 0.f && D[6] == 0.f && D[7] == 0.f &&
                        D[0] == D[4] && D[4] == D[8] && D[0] > 0.f;
    dsc[i] = scalar ? D[0] : -1.f;
}

// ------------------------------------------------------------------------- off-diagonal BSR

// Per row: the diagonal block's position (-1 if absent) and the count of the others.
__global__ void od_count_kernel(int V, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                int32_t *dpos, int32_t *cnt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > V) return;
    if (i == V) {
        cnt[V] = 0;
        return;
    }
    int d;
    cnt[i] = sell_row_length(rp, ci, i, &d);
    dpos[i] = d;
}

// One warp per row: the row's blocks except the diagonal, in column order.
__global__ void od_fill_kernel(int V, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                               const float *__restrict__ vals, const int32_t *__restrict__ dpos,
                               const int32_t *__restrict__ od_rp, int64_t cap, int32_t *od_ci, float *od_vals,
                               uint32_t *err)
{
    const int lane = threadIdx.x & 31;
    const int row = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (row >= V) return;
    if (od_rp[row + 1] > cap) {
        if (lane == 0) pc_set_err(err, PC_DERR_INDEX);
        return;
    }
    const int r0 = rp[row], r1 = rp[row + 1], d = dpos[row], o0 = od_rp[row];
    for (int k = r0 + lane; k < r1; k += 32) {
        if (k == d) continue;
        const int o = o0 + (k - r0) - ((d >= 0 && k > d) ? 1 : 0);
        od_ci[o] = ci[k];
#pragma unroll
        for (int e = 0; e < 9; ++e) od_vals[9ll * o + e] = vals[9ll * k + e];
    }
}

// Copy A without its diagonal blocks for the difference-form products (returns false,
// error bits clear, when there is no room; the solve then reads A itself).
static pc_status build_offdiag(pc_ctx *c, const pc_bsr *A, const float *vals, bool *ok, cudaStream_t st)
{
    *ok = false;
    const int V = c->V;
    if (c->od_cap <= 0 || !c->od_vals) return PC_OK;
    PC_LAUNCH(c, od_count_kernel, pc_blocks(V + 1ll, 256), 256, 0, st, V, A->row_ptr, A->col_idx, c->od_dpos,
              c->od_cnt);
    PC_TRY(pc_exclusive_scan(c, c->od_cnt, c->od_rp, V, st));
    PC_CUDA_TRY(cudaMemcpyAsync(c->h_count, c->od_rp + V, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    const int32_t total = reinterpret_cast<int32_t *>(c->h_count)[0];
    if (total < 0 || total > c->od_cap) return PC_OK;
    PC_LAUNCH(c, od_fill_kernel, pc_blocks(32ll * V, 256), 256, 0, st, V, A->row_ptr, A->col_idx, vals, c->od_dpos,
              c->od_rp, c->od_cap, c->od_ci, c->od_vals, c->d_err);
    uint32_t bits = 0;
    PC_TRY(pc_read_errors(c, st, &bits));
    if (bits) {
        PC_CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), st));
        return PC_OK;
    }
    c->od_nnzb = total;
    *ok = true;
    return PC_OK;
}

// Launch shape of the fused update (false in *ok when a thread would need more than
// FU_ROWS rows, when the grid would not be co-resident, or without the barrier word).
static pc_status fuse_shape(pc_ctx *c, bool block, bool *ok, int *grid, int *rows)
{
    *ok = false;
    if (!c->fbar || c->V < 1) return PC_OK;
    int occ = 0;
    if (block)
        PC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pcg_update_dir_kernel<true>, FU_THREADS, 0));
    else
        PC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pcg_update_dir_kernel<false>, FU_THREADS, 0));
    if (occ < FU_CTAS_PER_SM) return PC_OK;
    const int64_t need = ((int64_t)c->V + FU_THREADS - 1) / FU_THREADS;
    const int64_t g = std::min<int64_t>((int64_t)c->num_sms * FU_CTAS_PER_SM, need);
    const int64_t r = ((int64_t)c->V + g * FU_THREADS - 1) / (g * FU_THREADS);
    if (r > FU_ROWS || g > c->max_red_blocks) return PC_OK;
    *grid = (int)g;
    *rows = (int)r;
    *ok = true;
    return PC_OK;
}

// The same copy without a host round trip (so it can be captured in a graph): valid
// whenever the matrix fits the copy's capacity, which the caller checks from nnzb.
// Also fills the scalar difference diagonals.
pc_status pc_build_offdiag_async(pc_ctx *c, const pc_bsr *A, const float *vals, const float *dres, cudaStream_t st)
{
    const int V = c->V;
    if (c->od_cap <= 0 || !c->od_vals || A->nnzb > c->od_cap) return PC_ERR_CAPACITY;
    PC_LAUNCH(c, od_count_kernel, pc_blocks(V + 1ll, 256), 256, 0, st, V, A->row_ptr, A->col_idx, c->od_dpos,
              c->od_cnt);
    PC_TRY(pc_exclusive_scan(c, c->od_cnt, c->od_rp, V, st));
    PC_LAUNCH(c, od_fill_kernel, pc_blocks(32ll * V, 256), 256, 0, st, V, A->row_ptr, A->col_idx, vals, c->od_dpos,
              c->od_rp, c->od_cap, c->od_ci, c->od_vals, c->d_err);
    if (dres && c->dsc) PC_LAUNCH(c, dsc_kernel, pc_blocks(V, 256), 256, 0, st, V, dres, c->dsc);
    return PC_OK;
}

static int sell_grid(const pc_ctx *c)
{
    const int g = c->num_sms * SL_CTAS_PER_SM;
    return g < c->max_red_blocks ? g : c->max_red_blocks;
}

static pc_status read_scalars(pc_ctx *c, cudaStream_t st)
{
    PC_CUDA_TRY(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(pc_scalars), cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    return PC_OK;
}

#define DISPATCH2(ctx, kern, diff, block, grid, thr, st, ...)                                           \
    do {                                                                                                  \
        if (diff && block) PC_LAUNCH(ctx, (kern<true, true>), grid, thr, 0, st, __VA_ARGS__);             \
        else if (diff) PC_LAUNCH(ctx, (kern<true, false>), grid, thr, 0, st, __VA_ARGS__);               \
        else if (block) PC_LAUNCH(ctx, (kern<false, true>), grid, thr, 0, st, __VA_ARGS__);              \
        else PC_LAUNCH(ctx, (kern<false, false>), grid, thr, 0, st, __VA_ARGS__);                        \
    } while (0)

// fold the FP32 increment into the FP64 accumulator and replace the residual
static pc_status replace_residual(const SolveCtx &s, float *x32, int first, double tol, int max_iter)
{
    pc_ctx *c = s.c;
    if (!first) PC_LAUNCH(c, fold_kernel, ew_grid(c, c->V), EW_THREADS, 0, s.st, c->V, x32, c->x64);
    DISPATCH2(c, residual_replace_kernel, s.diff, s.block, ew_grid(c, c->V), EW_THREADS, s.st, c->V, s.A->row_ptr,
              s.A->col_idx, s.vals, s.dres, s.b, c->x64, c->dinv, c->r, (float4 *)c->z,
              (float4 *)c->p0, first, tol, max_iter, c->partials, c->sc, (int)s.fuse);
    return PC_OK;
}

// p = z + beta p, in place (beta = 0 right after a start, where p was zeroed)
__global__ void __launch_bounds__(EW_THREADS) pcg_direction_kernel(int V, const float4 *__restrict__ z4,
                                                                    float4 *__restrict__ p4, const pc_scalars *sc)
{
    pdl_wait();
    if (sc->done) return;
    const float beta = (float)sc->beta;
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x + threadIdx.x; base < V; base += DIR_UNROLL * stride) {
        float4 z[DIR_UNROLL], p[DIR_UNROLL];
#pragma unroll
        for (int u = 0; u < DIR_UNROLL; ++u) {
            const int row = base + u * stride;
            if (row < V) {
                z[u] = z4[row];
                p[u] = p4[row];
            }
        }
#pragma unroll
        for (int u = 0; u < DIR_UNROLL; ++u) {
            const int row = base + u * stride;
            if (row < V)
                p4[row] = make_float4(fmaf(beta, p[u].x, z[u].x), fmaf(beta, p[u].y, z[u].y),
                                      fmaf(beta, p[u].z, z[u].z), 0.f);
        }
    }
    pdl_trigger();
}

// `count` PCG iterations: p = z + beta p; q = A p (and p.q -> alpha); x, r, z update
// (and r.z -> beta, stop tests). Kernels exit at once when the scalars say done.
static pc_status launch_iterations(const SolveCtx &s, float *x, int count)
{
    pc_ctx *c = s.c;
    SpmvArgs a{};
    a.V = c->V;
    a.rp = s.offdiag ? c->od_rp : s.A->row_ptr;
    a.ci = s.offdiag ? c->od_ci : s.A->col_idx;
    a.vals = s.offdiag ? c->od_vals : s.vals;
    a.dres = s.dres;
    a.dsc = (s.dres && c->dsc) ? c->dsc : nullptr;
    a.x4 = (const float4 *)c->p0;
    a.y4 = (float4 *)c->q;
    a.partials = c->partials;
    a.sc = c->sc;
    a.err = c->d_err;
    const int n_pq = s.sell ? sell_grid(c) : s.sym ? sym_grid(c) : spmv_grid(c, s.capr);
    c->ev_iter0 = c->sc_host->iter;  // the scalars were read before this chunk
    for (int k = 0; k < count; ++k) {
        // two sampled products per chunk: the first (after the host's check and the fold of
        // the increment) and one in the middle (between two updates, the steady state)
        const int slot = !c->profiling ? -1 : k == 0 ? 0 : (count > 1 && k == count / 2) ? 1 : -1;
        const bool timed = slot >= 0;
        if (slot == 1) c->ev_mid = k;
        if (!s.fuse)  // with fusion the previous update already formed p
            PC_LAUNCH_PDL(c, pcg_direction_kernel, dir_grid(c, c->V), EW_THREADS, 0, s.st, c->V,
                          (const float4 *)c->z, (float4 *)c->p0, (const pc_scalars *)c->sc);
        if (timed) PC_CUDA_TRY(cudaEventRecord(c->ev[slot ? 6 : 0], s.st));
        if (s.sym) {
            SymArgs y{};
            y.V = c->V;
            y.urp = c->sym_urp;
            y.uci = c->sym_uci;
            y.uvals = c->sym_uvals;
            y.lrp = c->sym_lrp;
            y.lcol = c->sym_lcol;
            y.lsrc = c->sym_lsrc;
            y.dres = s.dres;
            y.x4 = (const float4 *)c->p0;
            y.y4 = (float4 *)c->q;
            y.partials = c->partials;
            y.sc = c->sc;
            y.err = c->d_err;
            if (s.diff) PC_LAUNCH_PDL(c, spmv_sym_kernel<true>, n_pq, SP_THREADS, SY_SMEM_BYTES, s.st, y);
            else PC_LAUNCH_PDL(c, spmv_sym_kernel<false>, n_pq, SP_THREADS, SY_SMEM_BYTES, s.st, y);
        } else if (s.sell) {
            SellArgs y{};
            y.nslices = c->sell_nslices;
            y.perm = c->sell_perm;
            y.width = c->sell_width;
            y.base = c->sell_base;
            y.data = c->sell_data;
            y.diag = s.diff ? s.dres : c->sell_diag;
            y.x4 = (const float4 *)c->p0;
            y.y4 = (float4 *)c->q;
            y.partials = c->partials;
            y.sc = c->sc;
            if (s.diff) PC_LAUNCH_PDL(c, spmv_sell_kernel<true>, n_pq, SL_THREADS, 0, s.st, y);
            else PC_LAUNCH_PDL(c, spmv_sell_kernel<false>, n_pq, SL_THREADS, 0, s.st, y);
        } else {
            PC_TRY(launch_spmv(c, a, s.diff, true, s.st, s.capr));
        }
        if (timed) PC_CUDA_TRY(cudaEventRecord(c->ev[slot ? 7 : 1], s.st));
        if (s.fuse && s.block)
            PC_LAUNCH_PDL(c, pcg_update_dir_kernel<true>, s.fu_grid, FU_THREADS, 0, s.st, c->V, s.fu_rows,
                          x, (float4 *)c->p0, c->r, (const float4 *)c->q, c->dinv,
                          c->partials, n_pq, c->sc, c->fbar, c->d_err,
                          c->bar_wait_cycles > 0 ? (long long)c->bar_wait_cycles : SP_WAIT_BUDGET);
        else if (s.fuse)
            PC_LAUNCH_PDL(c, pcg_update_dir_kernel<false>, s.fu_grid, FU_THREADS, 0, s.st, c->V, s.fu_rows,
                          x, (float4 *)c->p0, c->r, (const float4 *)c->q, c->dinv,
                          c->partials, n_pq, c->sc, c->fbar, c->d_err,
                          c->bar_wait_cycles > 0 ? (long long)c->bar_wait_cycles : SP_WAIT_BUDGET);
        else if (s.block)
            PC_LAUNCH_PDL(c, pcg_update_kernel<true>, upd_grid(c, c->V), EW_THREADS, 0, s.st, c->V, x,
                      (const float4 *)c->p0, c->r, (const float4 *)c->q, c->dinv,
                      (float4 *)c->z, c->partials, n_pq, c->sc);
        else
            PC_LAUNCH_PDL(c, pcg_update_kernel<false>, upd_grid(c, c->V), EW_THREADS, 0, s.st, c->V, x,
                      (const float4 *)c->p0, c->r, (const float4 *)c->q, c->dinv,
                      (float4 *)c->z, c->partials, n_pq, c->sc);
        if (timed) {
            // read after the chunk's synchronisation (no stall here)
            c->ev_pending = slot ? 2 : 1;
            c->spmv_nnzb = s.offdiag ? c->od_nnzb : s.A->nnzb;
        }
    }
    return PC_OK;
}

// Fold a pending SpMV timing (events recorded by launch_iterations) into the stats; the
// caller has synchronised the stream.
static pc_status collect_spmv_timing(pc_ctx *c)
{
    // ev_pending: 1 = the chunk's first product was timed; 2 = its middle one too. The
    // middle one stands for the chunk's other products, counted from the iterations the
    // chunk ran (products launched after the solve stopped return at once and are not
    // counted; a middle one among them is not used)
    if (!c->ev_pending) return PC_OK;
    const int pending = c->ev_pending;
    c->ev_pending = 0;
    const int ran = c->sc_host->iter - c->ev_iter0;
    if (ran < 1) return PC_OK;
    float ms = 0.f;
    PC_CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
    c->spmv_ms += ms;
    c->spmv_launches += 1;
    if (pending == 2 && ran > c->ev_mid) {
        PC_CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[6], c->ev[7]));
        c->spmv_ms += (double)ms * (ran - 1);
        c->spmv_launches += ran - 1;
    }
    return PC_OK;
}

static pc_status pcg_solve_impl(pc_ctx *ctx, const pc_bsr *A, const float *vals, const float *dres,
                                const float *b, float *dv, const pc_solve_opts *opts, pc_solve_info *info,
                                void *stream);

extern "C" pc_status pc_pcg_solve(pc_ctx *ctx, const pc_bsr *A, const float *vals, const float *dres, const float *b,
                                  float *dv, const pc_solve_opts *opts, pc_solve_info *info, void *stream)
{
    return pcg_solve_impl(ctx, A, vals, dres, b, dv, opts, info, stream);
}

static pc_status pcg_solve_impl(pc_ctx *ctx, const pc_bsr *A, const float *vals, const float *dres,
                                const float *b, float *dv, const pc_solve_opts *opts, pc_solve_info *info,
                                void *stream)
{
    if (!ctx || !b || !dv || !pc_aligned16(dv)) return PC_ERR_ARG;
    PC_TRY(check_bsr(A, vals));
    pc_solve_opts o;
    pc_default_solve_opts(&o);
    if (opts) o = *opts;
    if (!(o.tol > 0.0) || o.max_iter < 0 || (o.precision != PC_PREC_FP32 && o.precision != PC_PREC_MIXED) ||
        (o.precond != PC_PRECOND_JACOBI && o.precond != PC_PRECOND_BLOCK) || !(o.refresh > 0.0 && o.refresh < 1.0) ||
        (o.schedule != PC_SCHED_AUTO && o.schedule != PC_SCHED_GRID && o.schedule != PC_SCHED_CLUSTER))
        return PC_ERR_ARG;
    if (o.check_every < 1) o.check_every = 32;
    if (o.refresh_every < 1) o.refresh_every = 1000;
    cudaStream_t st = (cudaStream_t)stream;
    const int V = ctx->V;
    const int64_t n = 3ll * V;
    SolveCtx s{ctx, A, vals, dres, b, dres != nullptr, o.precond == PC_PRECOND_BLOCK, st, false, false, false, false,
               0, 0};
    if (o.fuse) PC_TRY(fuse_shape(ctx, s.block, &s.fuse, &s.fu_grid, &s.fu_rows));
    if (s.fuse) PC_CUDA_TRY(cudaMemsetAsync(ctx->fbar, 0, sizeof(pc_fuse_bar), st));
    PC_CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), st));
    // the preconditioner's pass also validates the pattern; nothing else reads it before
    if (s.block)
        PC_LAUNCH(ctx, dinv_kernel<true>, pc_blocks(V, 256), 256, 0, st, V, A->nnzb, A->row_ptr, A->col_idx, vals,
                  ctx->dinv, ctx->d_err);
    else
        PC_LAUNCH(ctx, dinv_kernel<false>, pc_blocks(V, 256), 256, 0, st, V, A->nnzb, A->row_ptr, A->col_idx, vals,
                  ctx->dinv, ctx->d_err);
    uint32_t bits = 0;
    PC_TRY(pc_read_errors(ctx, st, &bits));  // synchronises the stream
    if (bits & PC_DERR_INDEX) return PC_ERR_ARG;
    if (bits) return PC_ERR_NONFINITE;
    if (o.schedule != PC_SCHED_GRID) {
        bool ran = false;
        const pc_status cs = pc_cluster_solve(ctx, A, vals, dres, b, dv, o, s.block, o.schedule == PC_SCHED_CLUSTER,
                                              info, st, &ran);
        if (ran || cs != PC_OK) return cs;
    }
    if (o.storage == PC_STORAGE_SYM) PC_TRY(build_sym(ctx, A, vals, &s.sym, st));
    if (o.storage == PC_STORAGE_SELL) PC_TRY(build_sell(ctx, A, vals, &s.sell, st));
    // the diagonal blocks multiply p_i - p_i = 0 in the difference form only
    if (o.storage == PC_STORAGE_OFFDIAG && s.diff) PC_TRY(build_offdiag(ctx, A, vals, &s.offdiag, st));
    if (s.diff && ctx->dsc) PC_LAUNCH(ctx, dsc_kernel, pc_blocks(V, 256), 256, 0, st, V, dres, ctx->dsc);
    // the narrower stages (more CTAs per SM) when every tile of the streamed matrix fits
    const bool tmax = !s.sym && !s.sell && ctx->d_count && ctx->h_count;
    if (tmax) {
        PC_CUDA_TRY(cudaMemsetAsync(ctx->d_count + 3, 0, sizeof(int64_t), st));
        PC_LAUNCH(ctx, tile_max_kernel, pc_blocks((V + SP_ROWS - 1) / SP_ROWS, 256), 256, 0, st, V,
                  s.offdiag ? ctx->od_rp : A->row_ptr, reinterpret_cast<long long *>(ctx->d_count + 3));
        PC_CUDA_TRY(cudaMemcpyAsync(ctx->h_count + 3, ctx->d_count + 3, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    }
    PC_TRY(pc_read_errors(ctx, st, &bits));
    if (bits) return PC_ERR_NONFINITE;
    if (tmax && ctx->h_count[3] <= (int64_t)SpShape<SP_CAP_PER_ROW>::cap) s.capr = SP_CAP_PER_ROW;

    const bool mixed = o.precision == PC_PREC_MIXED;
    // the iterations build an FP32 increment (float4 per row) on top of the initial dv:
    // mixed folds it into the FP64 accumulator, FP32 adds it to dv at the end
    float *x = ctx->dtmp;
    int replacements = 0;
    if (mixed) {
        PC_LAUNCH(ctx, f32_to_f64_kernel, ew_grid(ctx, n), EW_THREADS, 0, st, n, dv, ctx->x64);
        PC_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(float4) * V, st));
        PC_TRY(replace_residual(s, x, 1, o.tol, o.max_iter));
    } else {
        SpmvArgs a{};
        a.V = V;
        a.rp = A->row_ptr;
        a.ci = A->col_idx;
        a.vals = vals;
        a.dres = dres;
        a.xin = dv;
        a.y = ctx->rhs32;  // A dv as float[V][3]
        a.err = ctx->d_err;
        PC_TRY(launch_spmv(ctx, a, s.diff, false, st));
        if (s.block)
            PC_LAUNCH(ctx, pcg_init_kernel<true>, ew_grid(ctx, V), EW_THREADS, 0, st, V, b, ctx->rhs32,
                      ctx->r, ctx->dinv, (float4 *)ctx->z, (float4 *)ctx->p0, x,
                      o.tol, o.max_iter, ctx->partials, ctx->sc, (int)s.fuse);
        else
            PC_LAUNCH(ctx, pcg_init_kernel<false>, ew_grid(ctx, V), EW_THREADS, 0, st, V, b, ctx->rhs32,
                      ctx->r, ctx->dinv, (float4 *)ctx->z, (float4 *)ctx->p0, x,
                      o.tol, o.max_iter, ctx->partials, ctx->sc, (int)s.fuse);
    }
    PC_TRY(read_scalars(ctx, st));
    double rr_last = ctx->sc_host->rr;
    int iter_last = 0;
    int launched = 0;
    for (;;) {
        const pc_scalars h = *ctx->sc_host;
        if (h.done) {
            // mixed: a converged recurrence residual is confirmed by an FP64 replacement
            if (mixed && h.status == PC_OK && h.rr > 0.0 && h.iter > iter_last) {
                PC_TRY(replace_residual(s, x, 0, o.tol, o.max_iter));
                ++replacements;
                PC_TRY(read_scalars(ctx, st));
                rr_last = ctx->sc_host->rr;
                iter_last = ctx->sc_host->iter;
                continue;
            }
            break;
        }
        if (launched >= o.max_iter + o.check_every) break;
        if (mixed && h.iter > iter_last &&
            (h.rr <= rr_last * o.refresh * o.refresh || h.iter - iter_last >= o.refresh_every)) {
            PC_TRY(replace_residual(s, x, 0, o.tol, o.max_iter));
            ++replacements;
            PC_TRY(read_scalars(ctx, st));
            rr_last = ctx->sc_host->rr;
            iter_last = ctx->sc_host->iter;
            continue;
        }
        int chunk = o.check_every;
        if (launched == 0 && chunk > 8) chunk = 8;
        // mixed: move the FP32 increment into the FP64 accumulator at every check, so the
        // increment never grows large. Its rounding (about 6e-8 of the increment, white
        // noise that the stiff matrix amplifies) then stays far below what a residual
        // replacement measures, and replacements do not undo the iterations' progress.
        if (mixed && launched > 0)
            PC_LAUNCH(ctx, fold_kernel, ew_grid(ctx, V), EW_THREADS, 0, st, V, x, ctx->x64);
        PC_TRY(launch_iterations(s, x, chunk));
        launched += chunk;
        PC_TRY(read_scalars(ctx, st));
        PC_TRY(collect_spmv_timing(ctx));
    }
    const pc_scalars fin = *ctx->sc_host;
    if (fin.status == PC_ERR_TIMEOUT) return PC_ERR_TIMEOUT;
    pc_solve_info inf{};
    inf.iters = fin.iter;
    inf.outer = replacements;
    pc_status status = (pc_status)fin.status;
    double rr = fin.rr, bb = fin.bb;
    if (mixed) {
        if (fin.iter > iter_last) {  // stopped early (limit / breakdown): fold what there is
            PC_LAUNCH(ctx, fold_kernel, ew_grid(ctx, V), EW_THREADS, 0, st, V, x, ctx->x64);
        }
        PC_LAUNCH(ctx, f64_to_f32_kernel, ew_grid(ctx, n), EW_THREADS, 0, st, n, ctx->x64, dv);
        if (fin.iter > iter_last) {
            if (s.diff) PC_LAUNCH(ctx, residual_check_kernel<true>, ew_grid(ctx, V), EW_THREADS, 0, st, V, A->row_ptr,
                                  A->col_idx, vals, dres, b, dv, ctx->partials, ctx->sc);
            else PC_LAUNCH(ctx, residual_check_kernel<false>, ew_grid(ctx, V), EW_THREADS, 0, st, V, A->row_ptr,
                           A->col_idx, vals, dres, b, dv, ctx->partials, ctx->sc);
            PC_TRY(read_scalars(ctx, st));
            rr = ctx->sc_host->rr;
            bb = ctx->sc_host->bb;
        }
    } else {
        PC_LAUNCH(ctx, add_increment_kernel, ew_grid(ctx, V), EW_THREADS, 0, st, V, x, dv);
        if (s.diff) PC_LAUNCH(ctx, residual_check_kernel<true>, ew_grid(ctx, V), EW_THREADS, 0, st, V, A->row_ptr,
                              A->col_idx, vals, dres, b, dv, ctx->partials, ctx->sc);
        else PC_LAUNCH(ctx, residual_check_kernel<false>, ew_grid(ctx, V), EW_THREADS, 0, st, V, A->row_ptr,
                       A->col_idx, vals, dres, b, dv, ctx->partials, ctx->sc);
        PC_TRY(read_scalars(ctx, st));
        rr = ctx->sc_host->rr;
        bb = ctx->sc_host->bb;
    }
    inf.bnorm = sqrt(bb);
    inf.rel_res = bb > 0 ? sqrt(rr / bb) : 0.0;
    if (info) *info = inf;
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    return status;
}

extern "C" pc_status pc_get_solution64(pc_ctx *ctx, double *dv64, void *stream)
{
    if (!ctx || !dv64) return PC_ERR_ARG;
    PC_CUDA_TRY(cudaMemcpyAsync(dv64, ctx->x64, sizeof(double) * 3 * (size_t)ctx->V, cudaMemcpyDeviceToDevice,
                                (cudaStream_t)stream));
    return PC_OK;
}

// FP64 measures of an FP32 guess x of A x = b: |b - A x|^2, |b|^2, x.(A x) and b.x (so
// the CG energy 1/2 x.A x - b.x); the last block leaves them in the scalars' rr, bb, pq
// and rz slots (before any solve initialises them).
template <bool DIFF>
__global__ void __launch_bounds__(EW_THREADS) guess_eval_kernel(int V, const int32_t *__restrict__ rp,
                                                                const int32_t *__restrict__ ci,
                                                                const float *__restrict__ vals,
                                                                const float *__restrict__ dres,
                                                                const float *__restrict__ b,
                                                                const float *__restrict__ x, double *partials,
                                                                pc_scalars *sc)
{
    double rr = 0.0, bb = 0.0, xax = 0.0, bx = 0.0;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < V; row += gridDim.x * blockDim.x) {
        double acc[3];
        row_product64<float, DIFF>(row, rp, ci, vals, dres, x, acc);
        for (int a2 = 0; a2 < 3; ++a2) {
            const double bv = (double)b[3ll * row + a2], xv = (double)x[3ll * row + a2];
            const double rv = bv - acc[a2];
            rr += rv * rv;
            bb += bv * bv;
            xax += xv * acc[a2];
            bx += bv * xv;
        }
    }
    double v[4] = {rr, bb, xax, bx};
    if (last_block_reduce(v, 4, partials, &sc->counter) && threadIdx.x == 0) {
        sc->rr = v[0];
        sc->bb = v[1];
        sc->pq = v[2];
        sc->rz = v[3];
    }
}

// Residual and CG energy of an FP32 guess (host results; synchronizes):
// rr = |b - A x|^2, bb = |b|^2, energy = 1/2 x.(A x) - b.x.
pc_status pc_guess_eval(pc_ctx *c, const pc_bsr *A, const float *vals, const float *dres, const float *b,
                        const float *x, double *rr, double *bb, double *energy, cudaStream_t st)
{
    const int V = c->V;
    if (dres) PC_LAUNCH(c, guess_eval_kernel<true>, ew_grid(c, V), EW_THREADS, 0, st, V, A->row_ptr, A->col_idx,
                        vals, dres, b, x, c->partials, c->sc);
    else PC_LAUNCH(c, guess_eval_kernel<false>, ew_grid(c, V), EW_THREADS, 0, st, V, A->row_ptr, A->col_idx, vals,
                   dres, b, x, c->partials, c->sc);
    PC_TRY(read_scalars(c, st));
    *rr = c->sc_host->rr;
    *bb = c->sc_host->bb;
    *energy = 0.5 * c->sc_host->pq - c->sc_host->rz;
    return PC_OK;
}

// The FP64 cross term x.(A y) of two FP32 vectors (A symmetric, so it equals y.(A x)),
// left in the scalars' pq slot.
template <bool DIFF>
__global__ void __launch_bounds__(EW_THREADS) guess_cross_kernel(int V, const int32_t *__restrict__ rp,
                                                                 const int32_t *__restrict__ ci,
                                                                 const float *__restrict__ vals,
                                                                 const float *__restrict__ dres,
                                                                 const float *__restrict__ x,
                                                                 const float *__restrict__ y, double *partials,
                                                                 pc_scalars *sc)
{
    double xay = 0.0;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < V; row += gridDim.x * blockDim.x) {
        double acc[3];
        row_product64<float, DIFF>(row, rp, ci, vals, dres, y, acc);
        for (int a2 = 0; a2 < 3; ++a2) xay += (double)x[3ll * row + a2] * acc[a2];
    }
    double v[1] = {xay};
    if (last_block_reduce(v, 1, partials, &sc->counter) && threadIdx.x == 0) sc->pq = v[0];
}

pc_status pc_guess_cross(pc_ctx *c, const pc_bsr *A, const float *vals, const float *dres, const float *x,
                         const float *y, double *xay, cudaStream_t st)
{
    const int V = c->V;
    if (dres) PC_LAUNCH(c, guess_cross_kernel<true>, ew_grid(c, V), EW_THREADS, 0, st, V, A->row_ptr, A->col_idx,
                        vals, dres, x, y, c->partials, c->sc);
    else PC_LAUNCH(c, guess_cross_kernel<false>, ew_grid(c, V), EW_THREADS, 0, st, V, A->row_ptr, A->col_idx, vals,
                   dres, x, y, c->partials, c->sc);
    PC_TRY(read_scalars(c, st));
    *xay = c->sc_host->pq;
    return PC_OK;
}

// out = a x + b y (FP32 vectors of 3V entries; a and b rounded from the FP64 coefficients)
__global__ void combine_kernel(int64_t n, float *out, const float *x, const float *y, float a, float b)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = fmaf(a, x[i], b * y[i]);
}

pc_status pc_guess_combine(pc_ctx *c, float *out, const float *x, const float *y, double a, double b,
                           cudaStream_t st)
{
    const int64_t n = 3ll * c->V;
    PC_LAUNCH(c, combine_kernel, ew_grid(c, n), EW_THREADS, 0, st, n, out, x, y, (float)a, (float)b);
    return PC_OK;
}

pc_status pc_update_state(pc_ctx *c, float *x, float *v, const float *dv, float h, cudaStream_t st)
{
    const int64_t n = 3ll * c->V;
    PC_LAUNCH(c, state_update_kernel, ew_grid(c, n), EW_THREADS, 0, st, n, x, v, dv, h);
    return PC_OK;
}

// ------------------------------------------------------------------------- allocation-free solve
//
// pc_pcg_solve_static runs the same PCG kernels as pc_pcg_solve, but every scratch
// vector, reduction partial and scalar it needs lives in the file-scope array below
// instead of in a context, so the call allocates nothing. The array is sized for
// PC_STATIC_MAX_ROWS rows; each GPU that loads the library holds it (about 2.7 MB) until
// the process exits. All calls on a device share it.

#define PC_STATIC_MAX_BLOCKS 2048  // reduction partials: enough for 8 blocks per SM up to 256 SMs

struct pc_static_scratch {
    float4 r[PC_STATIC_MAX_ROWS];
    float4 z[PC_STATIC_MAX_ROWS];
    float4 p[PC_STATIC_MAX_ROWS];
    float4 q[PC_STATIC_MAX_ROWS];
    float4 dinv[3 * PC_STATIC_MAX_ROWS];
    float4 dtmp[PC_STATIC_MAX_ROWS];
    float dsc[PC_STATIC_MAX_ROWS];
    pc_fuse_bar fbar;
    float rhs32[3 * PC_STATIC_MAX_ROWS];
    double x64[3 * PC_STATIC_MAX_ROWS];
    double partials[RED_SLOTS * PC_STATIC_MAX_BLOCKS];
    int64_t count[4];  // the largest tile of the streamed matrix (slot 3), for the stage shape
    pc_scalars sc;
    uint32_t err;
};

static __device__ __align__(256) pc_static_scratch g_pcg_scratch;

// Device address of g_pcg_scratch on the current device (host code may not use the
// symbol itself as a device pointer), looked up on every call, together with the SpMV
// kernels' dynamic shared-memory limit, which pc_create sets for context-based calls.
// Both are host-side set-up without any allocation; redoing them on each call keeps them
// valid even if the device's context was reset and the module reloaded in between.
static pc_status static_scratch_address(pc_static_scratch **out, int *device)
{
    int dev = 0;
    PC_CUDA_TRY(cudaGetDevice(&dev));
    void *p = nullptr;
    PC_CUDA_TRY(cudaGetSymbolAddress(&p, g_pcg_scratch));
    PC_TRY(spmv_set_smem());
    *out = static_cast<pc_static_scratch *>(p);
    *device = dev;
    return PC_OK;
}

extern "C" pc_status pc_pcg_solve_static(int32_t V, const pc_bsr *A, const float *vals, const float *dres,
                                         const float *b, float *dv, const pc_solve_opts *opts, pc_solve_info *info,
                                         void *stream)
{
    if (V < 1 || V > PC_STATIC_MAX_ROWS) return PC_ERR_CAPACITY;
    if (!A || !vals || !b || !dv) return PC_ERR_ARG;
    pc_static_scratch *S = nullptr;
    int dev = 0;
    PC_TRY(static_scratch_address(&S, &dev));
    pc_ctx tmp;  // a view of the static scratch; owns nothing
    tmp.device = dev;
    tmp.V = V;
    PC_CUDA_TRY(cudaDeviceGetAttribute(&tmp.num_sms, cudaDevAttrMultiProcessorCount, dev));
    if (8 * tmp.num_sms > PC_STATIC_MAX_BLOCKS) return PC_ERR_CAPACITY;
    pc_scalars host_sc{};
    uint32_t host_err = 0;
    int64_t host_count[4] = {0, 0, 0, 0};
    tmp.r = reinterpret_cast<float *>(S->r);
    tmp.z = reinterpret_cast<float *>(S->z);
    tmp.p0 = reinterpret_cast<float *>(S->p);
    tmp.q = reinterpret_cast<float *>(S->q);
    tmp.dinv = reinterpret_cast<float *>(S->dinv);
    tmp.dtmp = reinterpret_cast<float *>(S->dtmp);
    tmp.dsc = S->dsc;
    tmp.fbar = &S->fbar;
    tmp.rhs32 = S->rhs32;
    tmp.x64 = S->x64;
    tmp.partials = S->partials;
    tmp.max_red_blocks = PC_STATIC_MAX_BLOCKS;
    tmp.sc = &S->sc;
    tmp.d_err = &S->err;
    tmp.sc_host = &host_sc;
    tmp.h_err = &host_err;
    tmp.d_count = S->count;
    tmp.h_count = host_count;
    // the previous call's scalars (and its reduction ticket) must not leak into this one
    PC_CUDA_TRY(cudaMemsetAsync(&S->sc, 0, sizeof(pc_scalars), (cudaStream_t)stream));
    return pcg_solve_impl(&tmp, A, vals, dres, b, dv, opts, info, stream);
}
