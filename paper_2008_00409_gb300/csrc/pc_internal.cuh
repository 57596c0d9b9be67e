// Internal definitions shared by the CUDA translation units of libpcloth.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/pcloth.h"

// ------------------------------------------------------------------------- error handling

#define PC_CUDA_TRY(expr)                                                                   \
    do {                                                                                    \
        cudaError_t _e = (expr);                                                            \
        if (_e != cudaSuccess) {                                                            \
            pc_note_cuda_error(_e, #expr, __FILE__, __LINE__);                              \
            return PC_ERR_CUDA;                                                             \
        }                                                                                   \
    } while (0)

#define PC_TRY(expr)                 \
    do {                             \
        pc_status _s = (expr);       \
        if (_s != PC_OK) return _s;  \
    } while (0)

void pc_note_cuda_error(cudaError_t e, const char *what, const char *file, int line);

// device error bits (ctx->d_err)
#define PC_DERR_INDEX 1u      // an index was out of range
#define PC_DERR_PAIR 2u       // a contact pair repeats a vertex
#define PC_DERR_MESH 4u       // non-manifold edge / degenerate triangle
#define PC_DERR_CAPACITY 8u   // output capacity exceeded
#define PC_DERR_NONFINITE 16u // NaN / Inf met
#define PC_DERR_TIMEOUT 32u   // a bounded device wait gave up

// element reference encoding in incidence lists: type(2) | local(2) | id(28)
#define PC_REF_TRI 0u
#define PC_REF_HINGE 1u
#define PC_REF_CONTACT 2u
__host__ __device__ inline uint32_t pc_ref(uint32_t type, uint32_t local, uint32_t id)
{
    return (type << 30) | (local << 28) | id;
}
__host__ __device__ inline uint32_t pc_ref_type(uint32_t r) { return r >> 30; }
__host__ __device__ inline uint32_t pc_ref_local(uint32_t r) { return (r >> 28) & 3u; }
__host__ __device__ inline uint32_t pc_ref_id(uint32_t r) { return r & 0x0FFFFFFFu; }

// per-element buffer strides (floats)
#define PC_TRI_STRIDE 64     // 9 forces + 6 upper 3x3 Hessian blocks (54) + 1 pad
#define PC_HINGE_STRIDE 24   // 12 forces + 12 scaled angle gradient
#define PC_CONTACT_STRIDE 20 // 12 forces + normal(3) + weights(3) + scale(1) + pad

// PCG scalar block, lives in device memory
struct pc_scalars {
    double rz;       // r.z of the current iterate
    double pq;       // p.q of the current direction
    double rr;       // r.r
    double bb;       // b.b
    double alpha, beta;
    double tol2;     // tol^2 * bb, stop threshold on rr
    int32_t iter;
    int32_t max_iter;
    int32_t done;     // 1 converged / stopped
    int32_t status;   // pc_status of the solve
    uint32_t counter; // last-block reduction ticket
    int32_t outer;    // FP64 residual replacements (the cluster solve reports them here)
};

// ------------------------------------------------------------------------- radix sort scratch
struct pc_sort_scratch {
    uint64_t *keys_alt = nullptr;
    uint32_t *vals_alt = nullptr;
    uint32_t *hist = nullptr;      // [256 * tiles]
    int64_t cap = 0;               // keys capacity
    int64_t hist_cap = 0;
};

struct pc_ctx {
    int device = 0;
    int32_t V = 0, T = 0, H = 0;
    int32_t max_contacts = 0;
    int32_t n_pins = 0;
    pc_material mat{};
    float mu = 0, lam = 0;
    int num_sms = 0;
    int64_t bar_wait_cycles = 0;   // grid-barrier wait budget of the persistent solver (0: default)

    // rest data
    int32_t *tri = nullptr;        // [T][3]
    float *rest = nullptr;         // [V][3]
    float *tri_dmi = nullptr;      // [T][4] inverse rest edge matrix
    float *tri_area = nullptr;     // [T]
    float *tri_rgram = nullptr;    // [T][6] rest Gram (11, 22, 12) as (hi, lo) float pairs
    float *mass = nullptr;         // [V]
    uint8_t *pinned = nullptr;     // [V]
    int32_t *hinge = nullptr;      // [H][4] wing0, wing1, edge0, edge1
    float *hcoef = nullptr;        // [H] 2 kb c_h
    float *hrest = nullptr;        // [H] rest angle

    // static pattern and incidence
    int64_t snnz = 0;
    int32_t *srp = nullptr;        // [V+1]
    int32_t *scol = nullptr;       // [snnz]
    int32_t *vinc_ptr = nullptr;   // [V+1]
    uint32_t *vinc = nullptr;      // [3T + 4H] element refs grouped by vertex
    int64_t enn = 0;
    int32_t *erp = nullptr;        // [V+1] edge one-rings (CSR)
    int32_t *ecol = nullptr;       // [enn] edge neighbours, sorted per vertex
    float *rest_len = nullptr;     // [V] mean rest length of the vertex's mesh edges

    // per-step contact data
    uint64_t *dkeys = nullptr;     // [6 * maxP] dynamic pattern keys (sorted)
    uint64_t *dnew = nullptr;      // [6 * maxP] keys not in the static pattern
    int32_t *dflag = nullptr;      // [6 * maxP + 1]
    int32_t *dscan = nullptr;      // [6 * maxP + 1]
    uint64_t *ckeys = nullptr;     // [4 * maxP] incidence keys (vertex)
    uint32_t *cinc = nullptr;      // [4 * maxP] contact refs grouped by vertex
    int32_t *cinc_ptr = nullptr;   // [V+1]
    int32_t n_new = 0;
    int32_t n_contacts = 0;        // contacts of the last pattern call
    const int32_t *last_pairs = nullptr;

    // element buffers
    float *tri_buf = nullptr;      // [T][PC_TRI_STRIDE]
    float *hinge_buf = nullptr;    // [H][PC_HINGE_STRIDE]
    float *cont_buf = nullptr;     // [maxP][PC_CONTACT_STRIDE]

    // solver scratch
    float *r = nullptr, *z = nullptr, *p0 = nullptr, *p1 = nullptr, *q = nullptr, *dinv = nullptr;
    float *dtmp = nullptr;         // inner solution (mixed precision)
    float *rhs32 = nullptr;        // inner right-hand side (mixed precision)
    double *x64 = nullptr, *r64 = nullptr;
    double *partials = nullptr;    // [max_blocks][4]
    pc_scalars *sc = nullptr;      // device scalars
    pc_scalars *sc_host = nullptr; // pinned host mirror
    int32_t max_red_blocks = 0;

    // symmetric storage of the system being solved (built per solve from the full BSR)
    int64_t sym_cap = 0;
    int32_t *sym_urp = nullptr, *sym_lrp = nullptr;  // [V+1]
    int32_t *sym_dpos = nullptr;                     // [V] diagonal position in the full row
    int32_t *sym_ucnt = nullptr, *sym_lcnt = nullptr;  // [V+1]
    int32_t *sym_uci = nullptr, *sym_lcol = nullptr, *sym_lsrc = nullptr;  // [sym_cap + 4]
    float *sym_uvals = nullptr;                      // [9 sym_cap + 16]
    // sliced-ELL storage (PC_STORAGE_SELL), rebuilt per solve
    int64_t sell_cap = 0;                            // block positions available
    int32_t sell_nslices = 0;
    int32_t *sell_perm = nullptr;                    // [32 sell_nslices]
    int32_t *sell_width = nullptr, *sell_base = nullptr;  // [sell_nslices + 1]
    int32_t *sell_dpos = nullptr;                    // [V]
    uint32_t *sell_data = nullptr;                   // [320 sell_cap]
    float *sell_diag = nullptr;                      // [V][9]
    // off-diagonal BSR (PC_STORAGE_OFFDIAG): the matrix without its diagonal blocks
    int64_t od_cap = 0;
    int32_t *od_rp = nullptr, *od_cnt = nullptr;     // [V+1]
    int32_t *od_dpos = nullptr;                      // [V]
    int32_t *od_ci = nullptr;                        // [od_cap + 4]
    float *od_vals = nullptr;                        // [9 od_cap + 16]
    int64_t od_nnzb = 0;                             // blocks of the last copy
    float *dsc = nullptr;                            // [V] scalar difference diagonal or -1
    struct pc_fuse_bar *fbar = nullptr;              // grid barrier of the fused PCG update
    // proximity query: cell list (8 entries per triangle) and counts
    int64_t px_cap = 0;
    uint64_t *px_keys = nullptr;
    uint32_t *px_vals = nullptr;
    int32_t *px_cnt = nullptr, *px_off = nullptr;    // [T+1]
    int32_t *px_vcnt = nullptr, *px_voff = nullptr;  // [V+1]
    uint32_t *px_max = nullptr;

    // context-owned step system
    int32_t *A_rp = nullptr, *A_ci = nullptr;
    int64_t A_cap = 0;
    float *A_vals = nullptr, *A_dres = nullptr, *A_b = nullptr, *A_dv = nullptr;
    int has_prev_dv = 0;

    // host-buffer step staging
    float *h_state = nullptr;      // device [2][V][3]
    int32_t *h_pairs = nullptr;    // device [maxP][4]
    float *h_w = nullptr;          // device [maxP][3]

    // generic scratch
    pc_sort_scratch sort;
    uint32_t *d_err = nullptr;     // device error bits
    uint32_t *h_err = nullptr;     // pinned host mirror
    int64_t *d_count = nullptr;    // device scalar (counts)
    int64_t *h_count = nullptr;    // pinned host mirror
    int32_t *scan_tmp = nullptr;   // block sums for scans
    int64_t scan_tmp_cap = 0;

    // batched solver state (pc_batched.cu)
    void *batched = nullptr;

    // learned warm start (pc_mlp.cu): caller-owned network, context-owned scratch
    const float *mlp_params = nullptr;  // device [PC_MLP_NPARAMS]
    const float *mlp_stats = nullptr;   // device [PC_MLP_NSTATS]
    float *mlp_feat = nullptr;          // [V][12]
    float *mlp_dv = nullptr;            // [V][3]

    // profiling
    int profiling = 0;
    int64_t launches = 0;
    int64_t spmv_launches = 0;
    double spmv_ms = 0.0;
    int64_t spmv_nnzb = 0;
    int64_t asm_steps = 0;         // pc_step calls timed (assembly: pattern + values)
    int cl_size = 0;               // CTAs per cluster of the cluster solve (0: not queried, -1: none)
    int64_t cl_solves = 0;         // cluster solves timed, their iterations and milliseconds
    int64_t cl_iters = 0;
    double cl_ms = 0.0;
    double asm_ms = 0.0;
    cudaEvent_t ev[2 * 64] = {};
    int ev_used = 0;
    int ev_pending = 0;            // SpMV events recorded, not yet read (1: first of the chunk, 2: and middle)
    int ev_iter0 = 0;              // PCG iterations done before the chunk
    int ev_mid = 0;                // index of the chunk's sampled middle product
};

// launch bookkeeping: every kernel launch in the library goes through this
#define PC_LAUNCH(ctx, kernel, grid, block, smem, stream, ...)                          \
    do {                                                                              \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                   \
        (ctx)->launches++;                                                            \
        cudaError_t _le = cudaGetLastError();                                         \
        if (_le != cudaSuccess) {                                                     \
            pc_note_cuda_error(_le, #kernel, __FILE__, __LINE__);                     \
            return PC_ERR_CUDA;                                                       \
        }                                                                             \
    } while (0)

// Programmatic dependent launch: the kernel may be scheduled while its predecessor in the
// stream is still running; it must call pdl_wait() before reading anything the
// predecessor writes (the wait returns once that grid has completed and its memory is
// visible), and calls pdl_trigger() to let its own successor be scheduled early.
#define PC_LAUNCH_PDL(ctx, kernel, grid, block, smem, strm, ...)                        \
    do {                                                                              \
        cudaLaunchConfig_t _cfg = {};                                                 \
        _cfg.gridDim = dim3(grid);                                                    \
        _cfg.blockDim = dim3(block);                                                  \
        _cfg.dynamicSmemBytes = (smem);                                               \
        _cfg.stream = (strm);                                                         \
        cudaLaunchAttribute _attr[1];                                                 \
        _attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;             \
        _attr[0].val.programmaticStreamSerializationAllowed = 1;                      \
        _cfg.attrs = _attr;                                                           \
        _cfg.numAttrs = 1;                                                            \
        cudaError_t _le = cudaLaunchKernelEx(&_cfg, kernel, __VA_ARGS__);             \
        (ctx)->launches++;                                                            \
        if (_le != cudaSuccess) {                                                     \
            pc_note_cuda_error(_le, #kernel, __FILE__, __LINE__);                     \
            return PC_ERR_CUDA;                                                       \
        }                                                                             \
    } while (0)

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

inline unsigned pc_blocks(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 0x7FFFFFFF) b = 0x7FFFFFFF;
    return (unsigned)b;
}

inline bool pc_aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// ------------------------------------------------------------------------- shared helpers (host side)
pc_status pc_radix_sort(pc_ctx *ctx, uint64_t *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t st);
pc_status pc_proximity_alloc(pc_ctx *ctx);
pc_status pc_build_offdiag_async(pc_ctx *c, const pc_bsr *A, const float *vals, const float *dres, cudaStream_t st);
pc_status pc_exclusive_scan(pc_ctx *ctx, const int32_t *in, int32_t *out, int64_t n, cudaStream_t st);
pc_status pc_sort_reserve(pc_ctx *ctx, int64_t n);
pc_status pc_read_errors(pc_ctx *ctx, cudaStream_t st, uint32_t *bits);
pc_status pc_setup_rest(pc_ctx *ctx, cudaStream_t st);
pc_status pc_update_state(pc_ctx *ctx, float *x, float *v, const float *dv, float h, cudaStream_t st);
pc_status pc_solver_alloc(pc_ctx *ctx);
pc_status pc_batched_alloc(pc_ctx *ctx);
void pc_batched_free(pc_ctx *ctx);
pc_status pc_guess_eval(pc_ctx *c, const pc_bsr *A, const float *vals, const float *dres, const float *b,
                        const float *x, double *rr, double *bb, double *energy, cudaStream_t st);
pc_status pc_guess_cross(pc_ctx *c, const pc_bsr *A, const float *vals, const float *dres, const float *x,
                         const float *y, double *xay, cudaStream_t st);
pc_status pc_guess_combine(pc_ctx *c, float *out, const float *x, const float *y, double a, double b,
                           cudaStream_t st);
pc_status pc_warm_guess(pc_ctx *c, const pc_bsr *A, const float *v, float h, int32_t mode, float *feat_out,
                        int32_t *guess, double *guess_res, double *guess_energy, double *guess_coef,
                        double *combo_energy, cudaStream_t st);
void pc_mlp_ctx_free(pc_ctx *c);
// The whole solve in one thread-block cluster (pc_cluster.cu). Runs when the system fits
// the cluster's shared memory (*ran = true, returns the solve's status); otherwise
// returns PC_OK with *ran = false, or PC_ERR_CAPACITY when `required`. Needs c->dinv
// filled (and the pattern validated) for this matrix; `o` is normalised by the caller.
pc_status pc_cluster_solve(pc_ctx *c, const pc_bsr *A, const float *vals, const float *dres, const float *b,
                           float *dv, const pc_solve_opts &o, bool block, bool required, pc_solve_info *info,
                           cudaStream_t st, bool *ran);

inline int pc_bits_for(int64_t n)
{
    int b = 0;
    while (b < 63 && ((int64_t)1 << b) < n) ++b;
    return b < 1 ? 1 : b;
}

// ------------------------------------------------------------------------- device helpers

__device__ __forceinline__ void pc_set_err(uint32_t *err, uint32_t bit) { atomicOr(err, bit); }

// ------------------------------------------------------------------------- software grid barrier

// Grid-wide barrier of co-resident CTAs on a 64-bit arrival counter that only grows
// (zeroed before the first launch that uses it, and every launch sharing it has the same
// grid): the k-th barrier is complete once the counter reaches k * gridDim.x. Arriving is
// one acquire-release atomic that also tells the CTA which barrier it is at, and waiting
// is one acquire load per poll: no generation word, no reset by the last CTA. Bit 63 is the
// abort flag: a CTA whose wait exceeds `budget` SM cycles sets it (pc_grid_abort), and every
// CTA that arrives or polls afterwards leaves with false, so the launch unwinds at its next
// barrier. Called by all threads of the CTA; returns the same value to all of them.
#define PC_BAR_ABORT (1ull << 63)

__device__ __forceinline__ void pc_grid_abort(unsigned long long *count)
{
    atomicOr(count, PC_BAR_ABORT);
}

__device__ __forceinline__ bool pc_grid_barrier(unsigned long long *count, long long budget)
{
    __shared__ int s_ok;
    __syncthreads();  // every thread's writes precede thread 0's release
    if (threadIdx.x == 0) {
        unsigned long long old;
        asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], 1;" : "=l"(old) : "l"(count) : "memory");
        int ok = (old & PC_BAR_ABORT) == 0ull;
        const unsigned long long n = gridDim.x;
        const unsigned long long target = ((old & ~PC_BAR_ABORT) / n + 1ull) * n;
        if (ok && (old & ~PC_BAR_ABORT) + 1ull != target) {
            const long long t0 = clock64();
            for (unsigned k = 1;; ++k) {
                // the budget is checked before the first poll and then before every 16th, so
                // a budget of a few cycles makes every CTA but the last to arrive give up
                if ((k & 15u) == 1u && clock64() - t0 > budget) {
                    pc_grid_abort(count);
                    ok = 0;
                    break;
                }
                unsigned long long c;
                asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(c) : "l"(count) : "memory");
                if (c & PC_BAR_ABORT) { ok = 0; break; }
                if (c >= target) break;
                __nanosleep(32);
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ------------------------------------------------------------------------- double-float sums
// GB300 issues FP64 at about 1/60 of its FP32 rate (and with long latency), so the
// per-iteration dot-product reductions add their partial sums as unevaluated pairs of
// floats, hi + lo (about 48 significant bits), with Knuth's error-free two-sum, and form
// an FP64 value only once, in one thread. Each pair sum is commutative bit for bit, so an
// xor butterfly leaves every lane with the same pair, and a fixed tree keeps every sum
// reproducible.
__device__ __forceinline__ void pc_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}
// (hi, lo) += (h2, l2)
__device__ __forceinline__ void pc_df_add(float &hi, float &lo, float h2, float l2)
{
    float s, e;
    pc_two_sum(hi, h2, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, l2));
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}
__device__ __forceinline__ void pc_warp_sum_df(float &hi, float &lo)
{
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        pc_df_add(hi, lo, h2, l2);
    }
}
// Block sum of n <= 4 pairs in a fixed tree (warps, then warp 0 over the warp sums);
// thread 0 gets the totals.
__device__ __forceinline__ void pc_block_sum_df(float *hi, float *lo, int n)
{
    __shared__ float2 s_df[4][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < n; ++k) {
        pc_warp_sum_df(hi[k], lo[k]);
        if (lane == 0) s_df[k][warp] = make_float2(hi[k], lo[k]);
    }
    __syncthreads();
    if (warp == 0) {
        for (int k = 0; k < n; ++k) {
            float2 w = lane < nw ? s_df[k][lane] : make_float2(0.f, 0.f);
            pc_warp_sum_df(w.x, w.y);
            hi[k] = w.x;
            lo[k] = w.y;
        }
    }
    __syncthreads();
}
__device__ __forceinline__ double pc_df_value(float hi, float lo) { return (double)hi + (double)lo; }

// lower_bound over a sorted uint64 array
__device__ __forceinline__ int64_t pc_lower_bound_u64(const uint64_t *a, int64_t n, uint64_t key)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}
