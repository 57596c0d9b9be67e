// Batched solve: many independent garments stored as one block-diagonal system (the
// union of their meshes), each solved to its own relative residual by ONE persistent
// PCG launch (cooperative, all CTAs co-resident), and a batched time step that captures
// value assembly, the solve and the state update in a CUDA graph.
//
// Instances own contiguous row ranges [inst_rows[k], inst_rows[k+1]) of at least 32 rows,
// so a 32-row tile touches at most two instances. Every reduction is segmented by
// instance through per-tile partial slots (first-row instance, last-row instance) that
// one CTA per instance sums in tile order, so results are deterministic. Phases are
// separated by a software grid barrier whose waits are bounded; a timeout aborts the
// launch with PC_ERR_TIMEOUT instead of hanging. Per iteration:
//   direction  p = z + beta_k p                   (rows of active instances)
//   spmv       q = A p, tile partials of p.q      (the bulk-copy pipelined SpMV)
//   alpha      alpha_k = rz_k / pq_k              (one CTA per instance)
//   update     x += alpha p, r -= alpha q, z = D^-1 r, tile partials of r.z, r.r
//   beta       beta_k, stop tests, refresh requests
// and, when some instance asks for it, FP64 residual replacement (fold the FP32
// increment into the FP64 accumulator, r = b - A x64 in FP64, new scalars).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pc_internal.cuh"

#define RED_SLOTS 4
#define BT_TILE 32  // rows per tile in every phase

// local copies of the reduction helpers used by pc_spmv.cuh's kernel (not launched here)
__device__ __forceinline__ double bt_warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ void block_sum_d(double *v, int n)
{
    __shared__ double s[RED_SLOTS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < n; ++k) {
        double w = bt_warp_sum(v[k]);
        if (lane == 0) s[k][warp] = w;
    }
    __syncthreads();
    if (warp == 0) {
        for (int k = 0; k < n; ++k) {
            double w = lane < nw ? s[k][lane] : 0.0;
            v[k] = bt_warp_sum(w);
        }
    }
    __syncthreads();
}
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

#include "pc_spmv.cuh"

// ------------------------------------------------------------------------- device state

struct bt_inst {
    double rz, rr, bb, tol2, alpha, beta, pq, rr_last;
    int32_t iter, iter_last, done, status;
    int32_t refresh, pad0, pad1, pad2;
};

struct bt_global {
    uint32_t bar_count;   // grid barrier arrivals
    uint32_t bar_gen;     // grid barrier generation
    uint32_t abort;       // set on timeout
    uint32_t n_active[2]; // instances still iterating (slot by iteration parity)
    uint32_t n_refresh[2];
    uint32_t pad;
};

struct BtArgs {
    int V, n_inst, ntiles;
    const int32_t *rp, *ci;
    const float *vals, *dres, *b;
    const int32_t *inst_rows;  // [n_inst + 1]
    const int32_t *row_inst;   // [V]
    float4 *r4, *z4, *p4, *q4, *x4;
    const float4 *dinv4;
    double *x64;
    float *dv;
    double *tp_a, *tp_b;       // tile partials [ntiles][3] for the first-row / last-row instance
    bt_inst *inst;
    bt_global *g;
    uint32_t *err;
    double tol, refresh;
    int max_iter, refresh_every;
};

// ------------------------------------------------------------------------- grid barrier

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// All CTAs of the (co-resident) grid meet; returns false everywhere once any CTA gave
// up waiting (the launch then unwinds without further waits).
__device__ bool bt_grid_sync(bt_global *g)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = ld_acquire_gpu(&g->abort) == 0u;
        if (ok) {
            const uint32_t gen = ld_acquire_gpu(&g->bar_gen);
            __threadfence();
            const uint32_t arrived = atomicAdd(&g->bar_count, 1u);
            if (arrived == gridDim.x - 1) {
                g->bar_count = 0u;
                __threadfence();
                atomicAdd(&g->bar_gen, 1u);
            } else {
                const long long t0 = clock64();
                while (ld_acquire_gpu(&g->bar_gen) == gen) {
                    if (ld_acquire_gpu(&g->abort) != 0u) { ok = 0; break; }
                    if (clock64() - t0 > SP_WAIT_BUDGET) {
                        atomicExch(&g->abort, 1u);
                        ok = 0;
                        break;
                    }
                    __nanosleep(40);
                }
            }
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ------------------------------------------------------------------------- segmented tile sums

// Warp-level: 32 lanes hold one row each (or nothing); write the tile's partial sums of
// `n` quantities split by instance into tp_a (first row's instance) and tp_b (others).
__device__ __forceinline__ void bt_tile_partials(const BtArgs &a, int tile, int row_inst_lane, bool valid,
                                                 const float *vals3, int n)
{
    const int lane = threadIdx.x & 31;
    const int first_inst = __shfl_sync(0xffffffffu, valid ? row_inst_lane : -1, 0);
    const bool in_a = valid && row_inst_lane == first_inst;
    const bool in_b = valid && row_inst_lane != first_inst;
    for (int q = 0; q < n; ++q) {
        double va = in_a ? (double)vals3[q] : 0.0, vb = in_b ? (double)vals3[q] : 0.0;
        va = bt_warp_sum(va);
        vb = bt_warp_sum(vb);
        if (lane == 0) {
            a.tp_a[3ll * tile + q] = va;
            a.tp_b[3ll * tile + q] = vb;
        }
    }
}

// Sum of quantity q over instance k's tiles, in tile order (one CTA, all threads call).
__device__ double bt_instance_sum(const BtArgs &a, int k, int q)
{
    const int r0 = a.inst_rows[k], r1 = a.inst_rows[k + 1];
    const int t0 = r0 / BT_TILE, t1 = (r1 - 1) / BT_TILE;
    double acc = 0.0;
    for (int t = t0 + threadIdx.x; t <= t1; t += blockDim.x) {
        // the tile's first-row instance is k exactly when the tile starts inside k
        const int first_row = t * BT_TILE;
        const bool a_is_k = first_row >= r0;
        acc += a_is_k ? __ldcg(a.tp_a + 3ll * t + q) : __ldcg(a.tp_b + 3ll * t + q);
    }
    double v[1] = {acc};
    block_sum_d(v, 1);
    return v[0];  // valid in thread 0
}

// ------------------------------------------------------------------------- phases

__device__ __forceinline__ bool bt_active(const BtArgs &a, int k) { return __ldcg(&a.inst[k].done) == 0; }

// p = z + beta p for active rows
__device__ void bt_phase_direction(const BtArgs &a)
{
    const int stride = gridDim.x * blockDim.x;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < a.V; row += stride) {
        const int k = a.row_inst[row];
        if (!bt_active(a, k)) continue;
        const float beta = (float)__ldcg(&a.inst[k].beta);
        const float4 z = __ldcg(a.z4 + row), p = __ldcg(a.p4 + row);
        a.p4[row] = make_float4(fmaf(beta, p.x, z.x), fmaf(beta, p.y, z.y), fmaf(beta, p.z, z.z), 0.f);
    }
}

// q = A p with the bulk-copy stage ring; tile partials of p.q. `kbase` continues the
// mbarrier phase count across calls.
template <bool DIFF>
__device__ void bt_phase_spmv(const BtArgs &a, unsigned char *smem_raw, uint64_t *full_bar, uint64_t *empty_bar,
                              int (*stage_info)[4], int kbase)
{
    __shared__ float s_rowdot[BT_TILE];
    __shared__ int s_rowinst[BT_TILE];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = a.ntiles;
    bool timed_out = false;
    if (warp == SP_CWARPS) {
        if (lane == 0) {
            int issued = 0;
            for (int k = 0;; ++k) {
                const int tile = blockIdx.x + k * gridDim.x;
                if (tile >= ntiles) break;
                const int kg = kbase + k;
                const int s = kg % SP_STAGES;
                const uint32_t ph = (uint32_t)(kg / SP_STAGES) & 1u;
                if (kg >= SP_STAGES && !mbar_wait_bounded(&empty_bar[s], ph ^ 1u, SP_WAIT_BUDGET)) {
                    timed_out = true;
                    break;
                }
                const int r0 = tile * SP_ROWS, r1 = min(r0 + SP_ROWS, a.V);
                const bool any_active = bt_active(a, a.row_inst[r0]) || bt_active(a, a.row_inst[r1 - 1]);
                const int b0 = a.rp[r0], b1 = a.rp[r1];
                unsigned char *base = smem_raw + s * SP_STAGE_BYTES;
                if (any_active && b1 - b0 <= SP_CAP) {
                    const int64_t f0 = 9ll * b0, al0 = f0 & ~3ll, al1 = (9ll * b1 + 3) & ~3ll;
                    const int c0 = b0 & ~3, c1 = (b1 + 3) & ~3;
                    const uint32_t vbytes = (uint32_t)((al1 - al0) * 4), cbytes = (uint32_t)((c1 - c0) * 4);
                    stage_info[s][0] = b0;
                    stage_info[s][1] = (int)(f0 - al0);
                    stage_info[s][2] = b0 - c0;
                    stage_info[s][3] = 1;
                    mbar_arrive_expect_tx(&full_bar[s], vbytes + cbytes);
                    bulk_g2s(base, a.vals + al0, vbytes, &full_bar[s]);
                    bulk_g2s(base + SP_VAL_BYTES, a.ci + c0, cbytes, &full_bar[s]);
                } else {
                    stage_info[s][0] = b0;
                    stage_info[s][1] = 0;
                    stage_info[s][2] = 0;
                    stage_info[s][3] = 0;
                    mbar_arrive(&full_bar[s]);
                }
                ++issued;
            }
            for (int k = issued - 1; k >= 0 && k >= issued - SP_STAGES; --k) {
                const int kg = kbase + k;
                if (!mbar_wait_bounded(&full_bar[kg % SP_STAGES], (uint32_t)(kg / SP_STAGES) & 1u, SP_WAIT_BUDGET))
                    timed_out = true;
            }
        }
        __syncwarp();  // the producer warp reconverges before any block-wide barrier
    }
    // consumers: the producer warp does not take part, so they meet on named barrier 1
    for (int k = 0; warp < SP_CWARPS; ++k) {
        const int tile = blockIdx.x + k * gridDim.x;
        if (tile >= ntiles) break;
        const int kg = kbase + k;
        const int s = kg % SP_STAGES;
        const uint32_t ph = (uint32_t)(kg / SP_STAGES) & 1u;
        const int r0 = tile * SP_ROWS;
        {
            const int t = threadIdx.x;
            const int j = t & (SP_TPR - 1);
            // after a timeout the warp stops waiting but keeps the barrier sequence
            const bool ok = timed_out ? false : mbar_wait_bounded(&full_bar[s], ph, SP_WAIT_BUDGET);
            if (!__all_sync(0xffffffffu, ok)) {
                timed_out = true;
                if ((t & (SP_TPR - 1)) == 0) {
                    s_rowdot[t / SP_TPR] = 0.f;
                    s_rowinst[t / SP_TPR] = -1;
                }
            } else {
                const int b0 = stage_info[s][0], vo = stage_info[s][1], co = stage_info[s][2];
                const bool staged = stage_info[s][3] != 0;
                const float *s_vals = reinterpret_cast<const float *>(smem_raw + s * SP_STAGE_BYTES) + vo;
                const int32_t *s_cols =
                    reinterpret_cast<const int32_t *>(smem_raw + s * SP_STAGE_BYTES + SP_VAL_BYTES) + co;
                const int row = r0 + t / SP_TPR;
                float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
                float4 xj = make_float4(0.f, 0.f, 0.f, 0.f);
                int kinst = -1;
                bool act = false;
                if (row < a.V) {
                    kinst = a.row_inst[row];
                    act = bt_active(a, kinst);
                }
                if (act) {
                    xj = __ldcg(a.p4 + row);
                    const int rb = a.rp[row], re = a.rp[row + 1];
                    for (int bb = rb + j; bb < re; bb += SP_TPR) {
                        const int c = staged ? s_cols[bb - b0] : a.ci[bb];
                        const float *B = staged ? s_vals + 9 * (bb - b0) : a.vals + 9ll * bb;
                        float4 u = __ldcg(a.p4 + c);
                        if (DIFF) { u.x -= xj.x; u.y -= xj.y; u.z -= xj.z; }
                        spmv_fma(B, u, acc0, acc1, acc2);
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
                if (j == 0) {
                    float d = 0.f;
                    if (act) {
                        if (DIFF) spmv_fma(a.dres + 9ll * row, xj, acc0, acc1, acc2);
                        a.q4[row] = make_float4(acc0, acc1, acc2, 0.f);
                        d = fmaf(xj.x, acc0, fmaf(xj.y, acc1, xj.z * acc2));
                    }
                    s_rowdot[t / SP_TPR] = d;
                    s_rowinst[t / SP_TPR] = (row < a.V) ? kinst : -1;
                }
            }
        }
        asm volatile("bar.sync 1, %0;" ::"r"(SP_CWARPS * 32) : "memory");
        if (warp == 0) {
            const int row = r0 + lane;
            const float d = s_rowdot[lane];
            const int ki = s_rowinst[lane];
            bt_tile_partials(a, tile, ki < 0 ? 0 : ki, row < a.V && ki >= 0, &d, 1);
        }
        asm volatile("bar.sync 1, %0;" ::"r"(SP_CWARPS * 32) : "memory");
    }
    if (timed_out) {
        atomicExch(&a.g->abort, 1u);
        atomicOr(a.err, PC_DERR_TIMEOUT);
    }
}

// x += alpha p; r -= alpha q; z = D^-1 r; tile partials of (r.z, r.r)
__device__ void bt_phase_update(const BtArgs &a)
{
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile < a.ntiles; tile += nwarps) {
        const int row = tile * BT_TILE + lane;
        const bool valid = row < a.V;
        int k = valid ? a.row_inst[row] : 0;
        float dots[2] = {0.f, 0.f};
        if (valid && bt_active(a, k)) {
            const float alpha = (float)__ldcg(&a.inst[k].alpha);
            const float4 p = __ldcg(a.p4 + row), q = __ldcg(a.q4 + row);
            float4 x = __ldcg(a.x4 + row), r = __ldcg(a.r4 + row);
            x.x = fmaf(alpha, p.x, x.x); x.y = fmaf(alpha, p.y, x.y); x.z = fmaf(alpha, p.z, x.z);
            r.x = fmaf(-alpha, q.x, r.x); r.y = fmaf(-alpha, q.y, r.y); r.z = fmaf(-alpha, q.z, r.z);
            const float4 d = a.dinv4[row];
            const float4 z = make_float4(d.x * r.x, d.y * r.y, d.z * r.z, 0.f);
            a.x4[row] = x;
            a.r4[row] = r;
            a.z4[row] = z;
            dots[0] = fmaf(r.x, z.x, fmaf(r.y, z.y, r.z * z.z));
            dots[1] = fmaf(r.x, r.x, fmaf(r.y, r.y, r.z * r.z));
        }
        bt_tile_partials(a, tile, k, valid, dots, 2);
    }
}

// Fold the FP32 increment into the FP64 accumulator (rows of instances asking for it)
__device__ void bt_phase_fold(const BtArgs &a)
{
    const int stride = gridDim.x * blockDim.x;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < a.V; row += stride) {
        const int k = a.row_inst[row];
        if (__ldcg(&a.inst[k].refresh) == 0) continue;
        const float4 d = __ldcg(a.x4 + row);
        a.x64[3ll * row] += (double)d.x;
        a.x64[3ll * row + 1] += (double)d.y;
        a.x64[3ll * row + 2] += (double)d.z;
        a.x4[row] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// r = b - A x64 in FP64 for rows of refreshing instances; z = D^-1 r; p = 0 when
// starting; tile partials of (r.z, r64.r64, b.b)
template <bool DIFF>
__device__ void bt_phase_residual(const BtArgs &a, bool start)
{
    const int lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    for (int tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile < a.ntiles; tile += nwarps) {
        const int row = tile * BT_TILE + lane;
        const bool valid = row < a.V;
        int k = valid ? a.row_inst[row] : 0;
        float dots[3] = {0.f, 0.f, 0.f};
        double rr64 = 0.0, bb64 = 0.0;
        if (valid && __ldcg(&a.inst[k].refresh) != 0) {
            double xj[3] = {__ldcg(a.x64 + 3ll * row), __ldcg(a.x64 + 3ll * row + 1), __ldcg(a.x64 + 3ll * row + 2)};
            double acc[3] = {0.0, 0.0, 0.0};
            for (int kk = a.rp[row]; kk < a.rp[row + 1]; ++kk) {
                const int c = a.ci[kk];
                if (DIFF && c == row) continue;
                const float *B = a.vals + 9ll * kk;
                double xc[3] = {__ldcg(a.x64 + 3ll * c), __ldcg(a.x64 + 3ll * c + 1), __ldcg(a.x64 + 3ll * c + 2)};
                if (DIFF)
                    for (int d = 0; d < 3; ++d) xc[d] -= xj[d];
                for (int q = 0; q < 3; ++q)
                    acc[q] += (double)B[3 * q] * xc[0] + (double)B[3 * q + 1] * xc[1] + (double)B[3 * q + 2] * xc[2];
            }
            if (DIFF) {
                const float *D = a.dres + 9ll * row;
                for (int q = 0; q < 3; ++q)
                    acc[q] += (double)D[3 * q] * xj[0] + (double)D[3 * q + 1] * xj[1] + (double)D[3 * q + 2] * xj[2];
            }
            float rf[3];
            for (int q = 0; q < 3; ++q) {
                const double bv = (double)a.b[3ll * row + q];
                const double rv = bv - acc[q];
                rr64 += rv * rv;
                bb64 += bv * bv;
                rf[q] = (float)rv;
            }
            const float4 d = a.dinv4[row];
            const float4 r = make_float4(rf[0], rf[1], rf[2], 0.f);
            const float4 z = make_float4(d.x * r.x, d.y * r.y, d.z * r.z, 0.f);
            a.r4[row] = r;
            a.z4[row] = z;
            if (start) a.p4[row] = make_float4(0.f, 0.f, 0.f, 0.f);
            dots[0] = fmaf(r.x, z.x, fmaf(r.y, z.y, r.z * z.z));
        }
        // rr and bb need FP64 resolution: pass them through the FP64 slots directly
        const int first_inst = __shfl_sync(0xffffffffu, valid ? k : -1, 0);
        const bool in_a = valid && k == first_inst, in_b = valid && k != first_inst;
        double v[3] = {(double)dots[0], rr64, bb64};
        for (int q = 0; q < 3; ++q) {
            double va = bt_warp_sum(in_a ? v[q] : 0.0), vb = bt_warp_sum(in_b ? v[q] : 0.0);
            if (lane == 0) {
                a.tp_a[3ll * tile + q] = va;
                a.tp_b[3ll * tile + q] = vb;
            }
        }
    }
}

// ------------------------------------------------------------------------- the persistent kernel

template <bool DIFF>
__global__ void __launch_bounds__(SP_THREADS) batched_pcg_kernel(BtArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t full_bar[SP_STAGES], empty_bar[SP_STAGES];
    __shared__ int stage_info[SP_STAGES][4];
    __shared__ int s_flag[2];
    if (threadIdx.x == 0) {
        for (int s = 0; s < SP_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], SP_CWARPS);
        }
        mbar_fence_init();
    }
    __syncthreads();
    // tiles this CTA takes in each SpMV phase (continues the mbarrier phase count)
    const int my_tiles = a.ntiles > (int)blockIdx.x ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    int kbase = 0;

    // ---- start: x64 = dv0, x = 0 (done on the host side), r = b - A x64, z, p = 0
    for (int k = blockIdx.x; k < a.n_inst; k += gridDim.x)
        if (threadIdx.x == 0) {
            a.inst[k].refresh = 1;
            a.inst[k].done = 0;
        }
    if (!bt_grid_sync(a.g)) return;
    bt_phase_residual<DIFF>(a, true);
    if (!bt_grid_sync(a.g)) return;
    for (int k = blockIdx.x; k < a.n_inst; k += gridDim.x) {
        const double rz = bt_instance_sum(a, k, 0), rr = bt_instance_sum(a, k, 1), bb = bt_instance_sum(a, k, 2);
        if (threadIdx.x == 0) {
            bt_inst &I = a.inst[k];
            I.rz = rz; I.rr = rr; I.bb = bb; I.tol2 = a.tol * a.tol * bb;
            I.alpha = 0.0; I.beta = 0.0; I.pq = 0.0; I.rr_last = rr;
            I.iter = 0; I.iter_last = 0; I.refresh = 0; I.status = PC_OK;
            I.done = (rr <= I.tol2 || !isfinite(rr)) ? 1 : 0;
            if (!isfinite(rr)) I.status = PC_ERR_NONFINITE;
            if (!I.done && a.max_iter <= 0) { I.done = 1; I.status = PC_ERR_NOT_CONVERGED; }
        }
    }
    if (!bt_grid_sync(a.g)) return;

    for (int it = 0;; ++it) {
        const int par = it & 1;
        // termination: count active instances (every CTA computes the same number)
        if (threadIdx.x == 0) {
            int active = 0;
            for (int k = 0; k < a.n_inst; ++k) active += __ldcg(&a.inst[k].done) == 0;
            s_flag[0] = active;
        }
        __syncthreads();
        if (s_flag[0] == 0) break;

        bt_phase_direction(a);
        if (!bt_grid_sync(a.g)) return;
        bt_phase_spmv<DIFF>(a, smem_raw, full_bar, empty_bar, stage_info, kbase);
        kbase += my_tiles;
        if (!bt_grid_sync(a.g)) return;
        for (int k = blockIdx.x; k < a.n_inst; k += gridDim.x) {
            if (!bt_active(a, k)) continue;
            const double pq = bt_instance_sum(a, k, 0);
            if (threadIdx.x == 0) {
                bt_inst &I = a.inst[k];
                I.pq = pq;
                double alpha = I.rz / pq;
                if (!(pq > 0.0) || !isfinite(alpha)) {
                    I.status = PC_ERR_NONFINITE;
                    I.done = 1;
                    alpha = 0.0;
                }
                I.alpha = alpha;
            }
        }
        if (!bt_grid_sync(a.g)) return;
        bt_phase_update(a);
        if (!bt_grid_sync(a.g)) return;
        for (int k = blockIdx.x; k < a.n_inst; k += gridDim.x) {
            if (!bt_active(a, k)) continue;
            const double rz = bt_instance_sum(a, k, 0), rr = bt_instance_sum(a, k, 1);
            if (threadIdx.x == 0) {
                bt_inst &I = a.inst[k];
                I.beta = rz / I.rz;
                I.rz = rz;
                I.rr = rr;
                I.iter += 1;
                if (!isfinite(rr) || !isfinite(I.beta)) {
                    I.status = PC_ERR_NONFINITE;
                    I.done = 1;
                } else if (rr <= I.tol2 || rr <= I.rr_last * a.refresh * a.refresh ||
                           I.iter - I.iter_last >= a.refresh_every) {
                    I.refresh = 1;  // confirm or refresh with an FP64 residual
                    atomicAdd(&a.g->n_refresh[par], 1u);
                } else if (I.iter >= a.max_iter) {
                    I.status = PC_ERR_NOT_CONVERGED;
                    I.done = 1;
                }
            }
        }
        if (!bt_grid_sync(a.g)) return;
        if (threadIdx.x == 0) s_flag[1] = (int)ld_acquire_gpu(&a.g->n_refresh[par]);
        __syncthreads();
        if (s_flag[1] > 0) {
            bt_phase_fold(a);
            if (!bt_grid_sync(a.g)) return;
            bt_phase_residual<DIFF>(a, false);
            if (!bt_grid_sync(a.g)) return;
            for (int k = blockIdx.x; k < a.n_inst; k += gridDim.x) {
                if (__ldcg(&a.inst[k].refresh) == 0) continue;
                const double rz = bt_instance_sum(a, k, 0), rr = bt_instance_sum(a, k, 1);
                if (threadIdx.x == 0) {
                    bt_inst &I = a.inst[k];
                    I.rz = rz;
                    I.rr = rr;
                    I.rr_last = rr;
                    I.iter_last = I.iter;
                    I.refresh = 0;
                    if (!isfinite(rr)) { I.status = PC_ERR_NONFINITE; I.done = 1; }
                    else if (rr <= I.tol2) { I.status = PC_OK; I.done = 1; }
                    else if (I.iter >= a.max_iter) { I.status = PC_ERR_NOT_CONVERGED; I.done = 1; }
                }
            }
        }
        // the counter of the other parity is free again: clear it for the next iteration
        if (blockIdx.x == 0 && threadIdx.x == 0) a.g->n_refresh[par ^ 1] = 0u;
        if (!bt_grid_sync(a.g)) return;
    }
    // ---- finish: fold what is left and write dv = x64 (FP32)
    const int stride = gridDim.x * blockDim.x;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < a.V; row += stride) {
        const float4 d = __ldcg(a.x4 + row);
        for (int q = 0; q < 3; ++q) {
            const double xv = __ldcg(a.x64 + 3ll * row + q) + (double)(&d.x)[q];
            a.x64[3ll * row + q] = xv;
            a.dv[3ll * row + q] = (float)xv;
        }
    }
}

// ------------------------------------------------------------------------- small kernels

__global__ void bt_row_inst_kernel(int n_inst, const int32_t *inst_rows, int32_t *row_inst)
{
    const int k = blockIdx.x;
    if (k >= n_inst) return;
    for (int r = inst_rows[k] + threadIdx.x; r < inst_rows[k + 1]; r += blockDim.x) row_inst[r] = k;
}

// every block (row, col) must stay inside one instance
__global__ void bt_check_blocks_kernel(int V, const int32_t *rp, const int32_t *ci, const int32_t *row_inst,
                                       uint32_t *err)
{
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= V) return;
    const int k = row_inst[row];
    for (int s = rp[row]; s < rp[row + 1]; ++s)
        if (row_inst[ci[s]] != k) { pc_set_err(err, PC_DERR_INDEX); return; }
}

__global__ void bt_dinv_kernel(int V, const int32_t *rp, const int32_t *ci, const float *vals, float4 *dinv4,
                               uint32_t *err)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= V) return;
    int s = -1;
    for (int k = rp[r]; k < rp[r + 1]; ++k)
        if (ci[k] == r) { s = k; break; }
    const float d0 = s >= 0 ? vals[9ll * s] : 0.f, d1 = s >= 0 ? vals[9ll * s + 4] : 0.f,
                d2 = s >= 0 ? vals[9ll * s + 8] : 0.f;
    const bool ok = d0 > 0.f && d1 > 0.f && d2 > 0.f && isfinite(d0 + d1 + d2);
    dinv4[r] = ok ? make_float4(1.f / d0, 1.f / d1, 1.f / d2, 0.f) : make_float4(1.f, 1.f, 1.f, 0.f);
    if (!ok) pc_set_err(err, PC_DERR_NONFINITE);
}

__global__ void bt_start_kernel(int V, const float *dv, double *x64, float4 *x4)
{
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < V; row += gridDim.x * blockDim.x) {
        for (int q = 0; q < 3; ++q) x64[3ll * row + q] = (double)dv[3ll * row + q];
        x4[row] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// ------------------------------------------------------------------------- host side

struct pc_batched_state {
    int32_t *row_inst = nullptr;   // [V]
    double *tp_a = nullptr, *tp_b = nullptr;
    bt_inst *inst = nullptr;       // [max_inst]
    bt_global *g = nullptr;
    int32_t *inst_rows = nullptr;  // [max_inst + 1]
    int max_inst = 0;
    int blocks_per_sm = 0;         // autotuned launch shape (0 = not tuned yet)
    int64_t tuned_nnzb = -1;
    int tuned_inst = -1;
    float tune_ms[5] = {0, 0, 0, 0, 0};
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream the step graph is captured on
};

static pc_batched_state *bt_state(pc_ctx *c);

#define BT_MAX_INST 4096

static pc_status bt_prepare(pc_ctx *c, pc_batched_state **out)
{
    pc_batched_state *B = bt_state(c);
    if (!B) return PC_ERR_CUDA;
    *out = B;
    return PC_OK;
}

static pc_status bt_launch(pc_ctx *c, pc_batched_state *B, const BtArgs &args, bool diff, int blocks_per_sm,
                           cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(c->num_sms * blocks_per_sm));
    cfg.blockDim = dim3(SP_THREADS);
    cfg.dynamicSmemBytes = SP_SMEM_BYTES;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    PC_CUDA_TRY(cudaMemsetAsync(B->g, 0, sizeof(bt_global), st));
    BtArgs a = args;
    if (diff) PC_CUDA_TRY(cudaLaunchKernelEx(&cfg, batched_pcg_kernel<true>, a));
    else PC_CUDA_TRY(cudaLaunchKernelEx(&cfg, batched_pcg_kernel<false>, a));
    c->launches++;
    return PC_OK;
}

static int bt_max_blocks_per_sm(bool diff)
{
    int n = 0;
    if (diff) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batched_pcg_kernel<true>, SP_THREADS, SP_SMEM_BYTES);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batched_pcg_kernel<false>, SP_THREADS, SP_SMEM_BYTES);
    return n;
}

// Solve part shared by pc_pcg_solve_batched and pc_step_batched (stream-ordered, no
// host synchronisation, so it can be captured).
static pc_status bt_enqueue(pc_ctx *c, pc_batched_state *B, const pc_bsr *A, const float *vals, const float *dres,
                            const float *b, float *dv, int n_inst, const pc_solve_opts &o, int blocks_per_sm,
                            cudaStream_t st)
{
    const int V = c->V;
    PC_LAUNCH(c, bt_dinv_kernel, pc_blocks(V, 256), 256, 0, st, V, A->row_ptr, A->col_idx, vals,
              (float4 *)c->dinv, c->d_err);
    PC_LAUNCH(c, bt_start_kernel, pc_blocks(V, 256), 256, 0, st, V, dv, c->x64, (float4 *)c->dtmp);
    BtArgs a{};
    a.V = V;
    a.n_inst = n_inst;
    a.ntiles = (V + BT_TILE - 1) / BT_TILE;
    a.rp = A->row_ptr;
    a.ci = A->col_idx;
    a.vals = vals;
    a.dres = dres;
    a.b = b;
    a.inst_rows = B->inst_rows;
    a.row_inst = B->row_inst;
    a.r4 = (float4 *)c->r;
    a.z4 = (float4 *)c->z;
    a.p4 = (float4 *)c->p0;
    a.q4 = (float4 *)c->q;
    a.x4 = (float4 *)c->dtmp;
    a.dinv4 = (const float4 *)c->dinv;
    a.x64 = c->x64;
    a.dv = dv;
    a.tp_a = B->tp_a;
    a.tp_b = B->tp_b;
    a.inst = B->inst;
    a.g = B->g;
    a.err = c->d_err;
    a.tol = o.tol;
    a.refresh = o.refresh;
    a.max_iter = o.max_iter;
    a.refresh_every = o.refresh_every;
    return bt_launch(c, B, a, dres != nullptr, blocks_per_sm, st);
}

static pc_status bt_setup_instances(pc_ctx *c, pc_batched_state *B, const pc_bsr *A, int n_inst,
                                    const int32_t *inst_rows, cudaStream_t st)
{
    if (n_inst < 1 || n_inst > B->max_inst || !inst_rows) return PC_ERR_ARG;
    if (inst_rows[0] != 0 || inst_rows[n_inst] != c->V) return PC_ERR_ARG;
    for (int k = 0; k < n_inst; ++k)
        if (inst_rows[k + 1] - inst_rows[k] < BT_TILE) return PC_ERR_ARG;
    PC_CUDA_TRY(cudaMemcpyAsync(B->inst_rows, inst_rows, sizeof(int32_t) * (n_inst + 1), cudaMemcpyHostToDevice, st));
    PC_LAUNCH(c, bt_row_inst_kernel, n_inst, 256, 0, st, n_inst, B->inst_rows, B->row_inst);
    PC_CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), st));
    PC_LAUNCH(c, bt_check_blocks_kernel, pc_blocks(c->V, 256), 256, 0, st, c->V, A->row_ptr, A->col_idx, B->row_inst,
              c->d_err);
    uint32_t bits = 0;
    PC_TRY(pc_read_errors(c, st, &bits));
    if (bits) return PC_ERR_ARG;
    return PC_OK;
}

// Autotuner: on the first solve of a given shape, time a short solve (fixed iteration
// budget) for each feasible number of co-resident CTAs per SM and keep the fastest.
static pc_status bt_autotune(pc_ctx *c, pc_batched_state *B, const pc_bsr *A, const float *vals, const float *dres,
                             const float *b, int n_inst, const pc_solve_opts &o, cudaStream_t st)
{
    if (B->blocks_per_sm > 0 && B->tuned_nnzb == A->nnzb && B->tuned_inst == n_inst) return PC_OK;
    const int maxb = std::min(4, bt_max_blocks_per_sm(dres != nullptr));
    if (maxb < 1) return PC_ERR_CUDA;
    pc_solve_opts t = o;
    t.max_iter = std::min(o.max_iter, 60);
    t.tol = 1e-30;  // run the whole budget
    float best = 1e30f;
    int best_b = maxb;
    cudaEvent_t e0, e1;
    PC_CUDA_TRY(cudaEventCreate(&e0));
    PC_CUDA_TRY(cudaEventCreate(&e1));
    float *scratch_dv = c->rhs32;  // float[V][3], a zero guess
    for (int nb = 1; nb <= maxb; ++nb) {
        PC_CUDA_TRY(cudaMemsetAsync(scratch_dv, 0, sizeof(float) * 3 * (size_t)c->V, st));
        PC_CUDA_TRY(cudaEventRecord(e0, st));
        pc_status s = bt_enqueue(c, B, A, vals, dres, b, scratch_dv, n_inst, t, nb, st);
        PC_CUDA_TRY(cudaEventRecord(e1, st));
        if (s != PC_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return s; }
        PC_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        PC_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        B->tune_ms[nb] = ms;
        if (ms < best) { best = ms; best_b = nb; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B->blocks_per_sm = best_b;
    B->tuned_nnzb = A->nnzb;
    B->tuned_inst = n_inst;
    return PC_OK;
}

static pc_status bt_collect(pc_ctx *c, pc_batched_state *B, int n_inst, pc_solve_info *info, cudaStream_t st)
{
    std::vector<bt_inst> h(n_inst);
    PC_CUDA_TRY(cudaMemcpyAsync(h.data(), B->inst, sizeof(bt_inst) * n_inst, cudaMemcpyDeviceToHost, st));
    bt_global gh{};
    PC_CUDA_TRY(cudaMemcpyAsync(&gh, B->g, sizeof(bt_global), cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    uint32_t bits = 0;
    PC_TRY(pc_read_errors(c, st, &bits));
    if (gh.abort || (bits & PC_DERR_TIMEOUT)) return PC_ERR_TIMEOUT;
    pc_status worst = PC_OK;
    for (int k = 0; k < n_inst; ++k) {
        if (info) {
            info[k].iters = h[k].iter;
            info[k].outer = 0;
            info[k].bnorm = sqrt(h[k].bb);
            info[k].rel_res = h[k].bb > 0 ? sqrt(h[k].rr / h[k].bb) : 0.0;
        }
        if (h[k].status != PC_OK && worst == PC_OK) worst = h[k].status;
    }
    return worst;
}

extern "C" pc_status pc_pcg_solve_batched(pc_ctx *ctx, const pc_bsr *A, const float *vals, const float *dres,
                                          const float *b, float *dv, int32_t n_inst, const int32_t *inst_rows,
                                          const pc_solve_opts *opts, pc_solve_info *info, void *stream)
{
    if (!ctx || !A || !A->row_ptr || !A->col_idx || !vals || !b || !dv) return PC_ERR_ARG;
    if ((A->cap & 3) != 0 || A->nnzb < 0 || A->nnzb > A->cap || !pc_aligned16(vals) || !pc_aligned16(A->col_idx))
        return PC_ERR_ARG;
    pc_solve_opts o;
    pc_default_solve_opts(&o);
    if (opts) o = *opts;
    if (!(o.tol > 0.0) || o.max_iter < 0 || !(o.refresh > 0.0 && o.refresh < 1.0)) return PC_ERR_ARG;
    if (o.refresh_every < 1) o.refresh_every = 1000;
    cudaStream_t st = (cudaStream_t)stream;
    pc_batched_state *B = nullptr;
    PC_TRY(bt_prepare(ctx, &B));
    PC_TRY(bt_setup_instances(ctx, B, A, n_inst, inst_rows, st));
    PC_TRY(bt_autotune(ctx, B, A, vals, dres, b, n_inst, o, st));
    PC_CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), st));
    PC_TRY(bt_enqueue(ctx, B, A, vals, dres, b, dv, n_inst, o, B->blocks_per_sm, st));
    return bt_collect(ctx, B, n_inst, info, st);
}

extern "C" pc_status pc_batched_config(pc_ctx *ctx, int32_t *blocks_per_sm, float *tune_ms /*[4]*/)
{
    if (!ctx) return PC_ERR_ARG;
    pc_batched_state *B = bt_state(ctx);
    if (!B) return PC_ERR_CUDA;
    if (blocks_per_sm) *blocks_per_sm = B->blocks_per_sm;
    if (tune_ms)
        for (int i = 0; i < 4; ++i) tune_ms[i] = B->tune_ms[i + 1];
    return PC_OK;
}

// A batched step: pattern (synchronous), then one CUDA graph holding value assembly,
// the persistent batched solve and the state update.
extern "C" pc_status pc_step_batched(pc_ctx *ctx, float *x, float *v, const pc_contacts *contacts, int32_t n_inst,
                                     const int32_t *inst_rows, const pc_step_opts *opts, pc_solve_info *info,
                                     void *stream)
{
    if (!ctx || !x || !v || !opts || !(opts->h > 0.0f)) return PC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    pc_solve_opts o = opts->solve;
    if (!(o.tol > 0.0) || o.max_iter < 0 || !(o.refresh > 0.0 && o.refresh < 1.0)) return PC_ERR_ARG;
    if (o.refresh_every < 1) o.refresh_every = 1000;
    pc_bsr A{ctx->A_rp, ctx->A_ci, ctx->A_cap, 0};
    PC_TRY(pc_assemble_pattern(ctx, contacts, &A, stream));
    pc_batched_state *B = nullptr;
    PC_TRY(bt_prepare(ctx, &B));
    PC_TRY(bt_setup_instances(ctx, B, &A, n_inst, inst_rows, st));
    if (opts->warm_start != PC_WARM_PREV || !ctx->has_prev_dv)
        PC_CUDA_TRY(cudaMemsetAsync(ctx->A_dv, 0, sizeof(float) * 3 * (size_t)ctx->V, st));
    if (B->blocks_per_sm == 0 || B->tuned_nnzb < 0) {
        // tune on this step's system (values assembled once outside the graph)
        PC_TRY(pc_assemble_values(ctx, &A, x, v, contacts, opts->h, ctx->A_vals, ctx->A_b, ctx->A_dres, stream));
        PC_TRY(bt_autotune(ctx, B, &A, ctx->A_vals, ctx->A_dres, ctx->A_b, n_inst, o, st));
        B->tuned_nnzb = A.nnzb;  // keep the choice for later steps of the same batch
    }
    PC_CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), st));
    // capture values, solve and update on the private stream (the caller's stream may be
    // the legacy default stream, which cannot be captured); the graph runs on `st`
    cudaGraph_t graph = nullptr;
    cudaStream_t cs = B->cap_stream;
    PC_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    pc_status s = pc_assemble_values(ctx, &A, x, v, contacts, opts->h, ctx->A_vals, ctx->A_b, ctx->A_dres, (void *)cs);
    if (s == PC_OK)
        s = bt_enqueue(ctx, B, &A, ctx->A_vals, ctx->A_dres, ctx->A_b, ctx->A_dv, n_inst, o, B->blocks_per_sm, cs);
    if (s == PC_OK) s = pc_update_state(ctx, x, v, ctx->A_dv, opts->h, cs);
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (s != PC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (ce != cudaSuccess) {
        pc_note_cuda_error(ce, "cudaStreamEndCapture", __FILE__, __LINE__);
        return PC_ERR_CUDA;
    }
    bool updated = false;
    if (B->graph_exec) {
        cudaGraphExecUpdateResultInfo res{};
        updated = cudaGraphExecUpdate(B->graph_exec, graph, &res) == cudaSuccess;
        if (!updated) {
            cudaGetLastError();
            cudaGraphExecDestroy(B->graph_exec);
            B->graph_exec = nullptr;
        }
    }
    if (!B->graph_exec) {
        cudaError_t ie = cudaGraphInstantiate(&B->graph_exec, graph, 0);
        if (ie != cudaSuccess) {
            cudaGraphDestroy(graph);
            pc_note_cuda_error(ie, "cudaGraphInstantiate", __FILE__, __LINE__);
            return PC_ERR_CUDA;
        }
    }
    cudaGraphDestroy(graph);
    PC_CUDA_TRY(cudaGraphLaunch(B->graph_exec, st));
    ctx->has_prev_dv = 1;
    return bt_collect(ctx, B, n_inst, info, st);
}

// ------------------------------------------------------------------------- state allocation

static pc_batched_state *bt_state(pc_ctx *c)
{
    return reinterpret_cast<pc_batched_state *>(c->batched);
}

pc_status pc_batched_alloc(pc_ctx *c)
{
    pc_batched_state *B = new pc_batched_state();
    c->batched = B;
    const int64_t ntiles = (c->V + BT_TILE - 1) / BT_TILE;
    B->max_inst = BT_MAX_INST;
    PC_CUDA_TRY(cudaMalloc(&B->row_inst, sizeof(int32_t) * (size_t)c->V));
    PC_CUDA_TRY(cudaMalloc(&B->tp_a, sizeof(double) * 3 * (size_t)ntiles));
    PC_CUDA_TRY(cudaMalloc(&B->tp_b, sizeof(double) * 3 * (size_t)ntiles));
    PC_CUDA_TRY(cudaMalloc(&B->inst, sizeof(bt_inst) * BT_MAX_INST));
    PC_CUDA_TRY(cudaMalloc(&B->g, sizeof(bt_global)));
    PC_CUDA_TRY(cudaMalloc(&B->inst_rows, sizeof(int32_t) * (BT_MAX_INST + 1)));
    PC_CUDA_TRY(cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking));
    PC_CUDA_TRY(cudaFuncSetAttribute(batched_pcg_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     SP_SMEM_BYTES));
    PC_CUDA_TRY(cudaFuncSetAttribute(batched_pcg_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     SP_SMEM_BYTES));
    return PC_OK;
}

void pc_batched_free(pc_ctx *c)
{
    pc_batched_state *B = bt_state(c);
    if (!B) return;
    if (B->graph_exec) cudaGraphExecDestroy(B->graph_exec);
    if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
    cudaFree(B->row_inst);
    cudaFree(B->tp_a);
    cudaFree(B->tp_b);
    cudaFree(B->inst);
    cudaFree(B->g);
    cudaFree(B->inst_rows);
    delete B;
    c->batched = nullptr;
}
