// The whole PCG solve of a small system in one launch of one thread-block cluster
// (Sec. 2.5: the linear equations are solved with a preconditioned conjugate gradient
// solver; Sec. 3.1: the SpMV and the vector operations are data parallel).
//
// A system of a few thousand vertices leaves the grid-wide solver latency-bound: each
// iteration pays kernel boundaries and grid-wide barriers for a few microseconds of work.
// Here up to 16 CTAs of one cluster (one CTA per SM) hold the whole system in their shared
// memory for the length of the solve. CTA c owns rows [c Rc, (c+1) Rc): their 3x3 blocks
// (without the diagonal block in the difference form), difference-form diagonal, Jacobi
// inverse and every vector of the iteration.
//
// Iteration: the Chronopoulos-Gear form of preconditioned CG (A. T. Chronopoulos and
// C. W. Gear, "s-step iterative methods for symmetric linear systems", J. Comput. Appl.
// Math. 25, 1989), which needs one reduction per iteration instead of two. With
// u = M^-1 r and w = A u kept alongside p and s = A p:
//     p = u + beta p,  s = w + beta s,  x += alpha p,  r -= alpha s,  u = M^-1 r,  w = A u
//     gamma = (r, u),  delta = (u, w),  beta' = gamma / gamma_old,
//     alpha' = gamma / (p', A p')  with  (p', A p') = delta + beta' ((u, s) + (p, w)) + beta'^2 (p, s)
// -- the denominator expanded exactly from the stored vectors (p' = u + beta' p, A p' =
// w + beta' s) rather than through the method's orthogonality relations, so it stays
// right after a residual replacement. One iteration: the vector update, a cluster barrier
// that publishes u, the product w = A u, and the reduction of (gamma, r.r, delta, the two
// cross terms): two cluster barriers, one reduction.
//
// Distributed shared memory: a gather from another CTA's shared memory costs far more
// than a local one (measured on GB300: six scattered 16-byte remote loads per thread take
// about 30 times as long as local ones). So every CTA keeps ghost copies of the rows it
// reads from other CTAs; set-up numbers them, tells each owner which of its rows to send
// where, and each iteration the owners push those rows' u (and, for the FP64 residual,
// x) into the consumers' ghost slots with remote stores. Every gather of the product is
// then a plain shared-memory load. Reductions: FP32 per thread, double-float pairs across
// threads (pc_df_add); each CTA's warp 0 pushes the CTA's sums into every CTA's slot
// array, and after the barrier every warp adds the C slots in rank order, so all threads
// hold bitwise the same sums and compute the same scalars and decisions with no further
// barrier. The scalars are formed in FP32 after scaling the sums by a power of two fixed at
// the start (exact), which keeps them far from the FP32 range limits.
//
// Mixed precision as in the grid-wide solver: the FP32 increment is folded into the FP64
// iterate every check_every iterations, and the residual is recomputed in FP64 when the
// recurrence residual has dropped by refresh^2, after refresh_every iterations, and to
// confirm convergence. The replacement recomputes r and u = M^-1 r, and s = A p and w = A u
// by the product (the recurrences for s and r drift); it keeps the direction p and the
// recurrence's beta, and the replaced gamma enters alpha through the expanded denominator.
// Near FP32's attainable accuracy this form needs more iterations than the two-reduction
// form (its residual recurrence goes through the recurrence for s): the same count at a
// relative residual of 1e-6 on the 64 x 64 cloth, about a quarter more at 1e-9.
//
// The kernel has no spin-waits: the cluster's CTAs are co-scheduled by the hardware and
// its barriers are hardware barriers; every branch around a barrier depends only on
// values every thread of the cluster holds identically, so all threads reach every
// barrier. The last barrier keeps each CTA resident until no other CTA can still touch
// its shared memory.
#include <math.h>

#include <algorithm>
#include <cstddef>

#include "pc_internal.cuh"

#define CL_THREADS 512
#define CL_TPR 2                         // threads per row in the products
#define CL_SL 4                          // rows per slice of the block layout (CL_SL * CL_TPR = 8 lanes)
#define CL_GROUPS (CL_THREADS / CL_TPR)  // rows in flight per CTA
#define CL_WARPS (CL_THREADS / 32)
#define CL_MAXC 16                       // CTAs per cluster at most
#define CL_NV 6                          // values per reduction at most

struct ClArgs {
    int V, Rc, cap, gcap, pcap, Vw;
    const int32_t *rp, *ci;
    const float *vals, *dres, *dinv, *b;
    float *dv;
    double *x64;  // mixed precision: the FP64 solution on exit (may be null)
    double tol, refresh;
    int max_iter, check_every, refresh_every, mixed;
    pc_scalars *sc;
    // byte offsets of the shared-memory arrays (u starts at 0)
    uint32_t o_x64, o_xv, o_r, o_w, o_p, o_s, o_dres, o_dinv, o_rs, o_bits, o_pref, o_push, o_red, o_blk;
};

struct ClRed {
    float2 warp[CL_WARPS][CL_NV];        // this CTA's warp sums
    float2 slot[2][CL_MAXC][CL_NV];      // every CTA's sums, pushed here by that CTA (by parity)
    int misc[40];                        // scan scratch (0..31), vote flags (32, 33), requests received (34)
    double rr64, bb64;                   // thread 0: FP64 r.r of the last residual pass, b.b
    float scal[12];                      // thread 0's scalars (a ClScal) for its CTA to copy
};
static_assert(offsetof(ClRed, slot) % 16 == 0 && (CL_NV * sizeof(float2)) % 16 == 0,
              "slot rows take 16-byte remote stores");
#define CL_ACT_DONE 1
#define CL_ACT_FOLD 2
#define CL_ACT_REPLACE 4

struct ClSmem {
    float4 *u;           // [Rc + gcap] M^-1 r: own rows, then ghost copies
    double *x64;         // [Rc + gcap][4] FP64 iterate: own rows, then ghost copies
    float4 *xv, *r, *w, *p, *s;  // [Rc] FP32 increment, residual, A u, direction, A p
    float *dres;         // [Rc][9]
    float *dinv;         // [Rc][9] (block) or [Rc][4] (scalar Jacobi)
    int *rl;             // [Rc] stored blocks per row
    int *sb;             // [Rc / CL_SL + 1] first record of each slice of CL_SL rows
    uint32_t *bits;      // [Vw] rows other CTAs own that this CTA reads
    int *pref;           // [Vw] ghost number of each word's first row
    uint32_t *push;      // [pcap rounded up to a power of two] rows to send:
                         // rank << 28 | ghost << 10 | local row, sorted
    ClRed *red;
    float4 *blk;         // [cap][3] each stored block: its nine values, then the index of its
                         // column into u / x64 (an int's bits) and two pad words, so that
                         // three 16-byte loads fetch a block. Sliced: the blocks of CL_SL
                         // consecutive rows interleave, block k of row l at record
                         // sb[l / CL_SL] + ((k / CL_TPR) * CL_SL + l % CL_SL) * CL_TPR + k % CL_TPR,
                         // so the eight lanes that take a step of four rows together read
                         // eight consecutive records (no shared-memory bank conflicts), and on
                         // a regular mesh the rows those blocks gather are consecutive too
};

// ------------------------------------------------------------------------- cluster primitives

__device__ __forceinline__ uint32_t cl_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_nranks()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// all threads of all CTAs of the cluster; orders shared and global memory at cluster scope
__device__ __forceinline__ void cl_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cl_smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t cl_map(uint32_t local, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}
__device__ __forceinline__ uint32_t cl_ld_u32(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t cl_atom_add(uint32_t a, uint32_t v)
{
    uint32_t old;
    asm volatile("atom.shared::cluster.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(a), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void cl_st_u32(uint32_t a, uint32_t v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void cl_st_f2(uint32_t a, float2 v)
{
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void cl_st_f4(uint32_t a, float4 v)
{
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}
__device__ __forceinline__ void cl_st_d2(uint32_t a, double x, double y)
{
    asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(a), "d"(x), "d"(y) : "memory");
}

// Block-inclusive prefix sum of one int per thread; scratch[CL_WARPS - 1] holds the total
// on return (read it before the next call, with a barrier in between).
__device__ __forceinline__ int cl_scan(int v, int *scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
    }
    if (lane == 31) scratch[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < CL_WARPS ? scratch[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int n = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += n;
        }
        scratch[lane] = w;
    }
    __syncthreads();
    if (warp > 0) incl += scratch[warp - 1];
    return incl;
}

// Every CTA learns whether any CTA raised `flag` (a barrier, then each warp reads the C
// CTAs' flags); the same answer in every thread.
__device__ __forceinline__ bool cl_vote(int *flag, int mine, uint32_t C)
{
    if (threadIdx.x == 0) *flag = mine;
    cl_sync();
    const int lane = threadIdx.x & 31;
    const uint32_t f = (uint32_t)lane < C ? cl_ld_u32(cl_map(cl_smem_addr(flag), lane)) : 0u;
    return __any_sync(0xffffffffu, f != 0u);
}

// Sum N per-thread values over the cluster; the totals land in every thread (FP32 sums) or
// in warp 0 (pairs), in every CTA bitwise the same: warp sums, warp 0 adds the warp sums
// (warp order) and pushes the CTA's sums into slot[par][rank] of every CTA, a cluster
// barrier, and the C slots added in rank order. The iterations' dot products (FP32 partials) are summed in FP32 in
// that fixed tree (13 levels for 512 threads in 16 CTAs: a relative error below 1e-6,
// far below what the CG scalars tolerate); each double-float stage cost a few hundred
// cycles of the one warp on the critical path. The FP64 residual passes' partials are
// summed as double-float pairs (PAIRS).
template <int N, bool PAIRS>
__device__ __forceinline__ void cl_reduce(const float2 (&v)[N], float2 (&tot)[N], const ClSmem &S, int &par,
                                          uint32_t C, uint32_t rank)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        float hi = v[i].x, lo = v[i].y;
        if (PAIRS) {
            pc_warp_sum_df(hi, lo);
        } else {
            for (int o = 16; o > 0; o >>= 1) hi += __shfl_xor_sync(0xffffffffu, hi, o);
        }
        if (lane == 0) S.red->warp[warp][i] = make_float2(hi, lo);
    }
    __syncthreads();
    if (warp == 0) {
        float2 cs[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            float2 w = lane < CL_WARPS ? S.red->warp[lane][i] : make_float2(0.f, 0.f);
            if (PAIRS) {
                pc_warp_sum_df(w.x, w.y);
            } else {
                for (int o = 16; o > 0; o >>= 1) w.x += __shfl_xor_sync(0xffffffffu, w.x, o);
            }
            cs[i] = w;
        }
        if ((uint32_t)lane < C) {
            // the slot row is 16-byte aligned: two pairs per 16-byte remote store
            const uint32_t dst = cl_map(cl_smem_addr(&S.red->slot[par][rank][0]), lane);
#pragma unroll
            for (int i = 0; i + 1 < N; i += 2)
                cl_st_f4(dst + 8u * i, make_float4(cs[i].x, cs[i].y, cs[i + 1].x, cs[i + 1].y));
            if (N & 1) cl_st_f2(dst + 8u * (N - 1), cs[N - 1]);
        }
    }
    cl_sync();
    // FP32 sums: every warp adds the slots (every thread then forms the scalars itself,
    // with no broadcast); pairs: warp 0 only (thread 0 uses them)
    if (!PAIRS || warp == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            float2 w = (uint32_t)lane < C ? S.red->slot[par][lane][i] : make_float2(0.f, 0.f);
            if (PAIRS) {
                pc_warp_sum_df(w.x, w.y);
            } else {
                for (int o = 16; o > 0; o >>= 1) w.x += __shfl_xor_sync(0xffffffffu, w.x, o);
            }
            tot[i] = w;
        }
    }
    // slot[par] is pushed again two reductions later, after a barrier that this CTA's warps
    // reach only once they have read it
    par ^= 1;
}

// an FP64 value as a double-float pair (the residual passes' partial sums)
__device__ __forceinline__ float2 cl_pair(double d)
{
    const float hi = (float)d;
    return make_float2(hi, (float)(d - (double)hi));
}

// ------------------------------------------------------------------------- row arithmetic

template <bool BLOCK>
__device__ __forceinline__ float4 cl_precond(const float *dinv, int l, float4 r)
{
    if (BLOCK) {
        const float *d = dinv + 9 * l;
        return make_float4(d[0] * r.x + d[1] * r.y + d[2] * r.z, d[3] * r.x + d[4] * r.y + d[5] * r.z,
                           d[6] * r.x + d[7] * r.y + d[8] * r.z, 0.f);
    }
    const float4 d = reinterpret_cast<const float4 *>(dinv)[l];
    return make_float4(d.x * r.x, d.y * r.y, d.z * r.z, 0.f);
}

__device__ __forceinline__ float cl_dot3(float4 a, float4 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }

__device__ __forceinline__ float4 cl_axpy(float a, float4 x, float4 y)  // a x + y
{
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), 0.f);
}

// Send the rows other CTAs hold ghost copies of: u (float4), or the FP64 iterate.
__device__ __forceinline__ void cl_push_u(const ClSmem &S, int Rc, int n_push)
{
    const uint32_t base = cl_smem_addr(S.u);
    for (int e = threadIdx.x; e < n_push; e += CL_THREADS) {
        const uint32_t ent = S.push[e];
        const int l = ent & 0x3FF, g = (ent >> 10) & 0x3FFFF, d = ent >> 28;
        cl_st_f4(cl_map(base + 16u * (uint32_t)(Rc + g), d), S.u[l]);
    }
}
__device__ __forceinline__ void cl_push_x64(const ClSmem &S, int Rc, int n_push)
{
    const uint32_t base = cl_smem_addr(S.x64);
    for (int e = threadIdx.x; e < n_push; e += CL_THREADS) {
        const uint32_t ent = S.push[e];
        const int l = ent & 0x3FF, g = (ent >> 10) & 0x3FFFF, d = ent >> 28;
        const uint32_t dst = cl_map(base + 32u * (uint32_t)(Rc + g), d);
        const double *x = S.x64 + 4 * l;
        cl_st_d2(dst, x[0], x[1]);
        cl_st_d2(dst + 16u, x[2], 0.0);
    }
}

// w = A u for this CTA's rows (four threads per row), with the partial dot products of
// the denominator's expansion: d += (u, w), e += (u, s) + (p, w), f += (p, s). TO_S: the
// product of whatever u holds goes to s instead, without dot products.
template <bool DIFF, bool TO_S = false>
__device__ __forceinline__ void cl_product(const ClSmem &S, int nrows, float &d, float &e, float &f)
{
    const int sub = threadIdx.x & (CL_TPR - 1), grp = threadIdx.x / CL_TPR;
    for (int l0 = 0; l0 < nrows; l0 += CL_GROUPS) {
        const int l = l0 + grp;
        const bool ok = l < nrows;
        float4 ul = make_float4(0.f, 0.f, 0.f, 0.f);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        if (ok) {
            ul = S.u[l];
            const int len = S.rl[l];
            // this thread's records: block sub, sub + CL_TPR, ... of the row, STEP float4s apart
            constexpr int STEP = 3 * CL_SL * CL_TPR;
            const float4 *q = S.blk + 3 * (S.sb[l / CL_SL] + (l % CL_SL) * CL_TPR + sub);
            // two blocks per step with their own accumulators: two independent chains of
            // shared-memory loads (block, then its column's u) in flight per thread
            float c0 = 0.f, c1 = 0.f, c2 = 0.f;
            int k = sub;
            for (; k + CL_TPR < len; k += 2 * CL_TPR, q += 2 * STEP) {
                const float4 B2 = q[2], E2 = q[STEP + 2];
                float4 uj = S.u[__float_as_int(B2.y)], vj = S.u[__float_as_int(E2.y)];
                const float4 B0 = q[0], B1 = q[1];
                const float4 E0 = q[STEP], E1 = q[STEP + 1];
                if (DIFF) {
                    uj.x -= ul.x;
                    uj.y -= ul.y;
                    uj.z -= ul.z;
                    vj.x -= ul.x;
                    vj.y -= ul.y;
                    vj.z -= ul.z;
                }
                a0 = fmaf(B0.z, uj.z, fmaf(B0.y, uj.y, fmaf(B0.x, uj.x, a0)));
                a1 = fmaf(B1.y, uj.z, fmaf(B1.x, uj.y, fmaf(B0.w, uj.x, a1)));
                a2 = fmaf(B2.x, uj.z, fmaf(B1.w, uj.y, fmaf(B1.z, uj.x, a2)));
                c0 = fmaf(E0.z, vj.z, fmaf(E0.y, vj.y, fmaf(E0.x, vj.x, c0)));
                c1 = fmaf(E1.y, vj.z, fmaf(E1.x, vj.y, fmaf(E0.w, vj.x, c1)));
                c2 = fmaf(E2.x, vj.z, fmaf(E1.w, vj.y, fmaf(E1.z, vj.x, c2)));
            }
            if (k < len) {
                const float4 B2 = q[2];
                float4 uj = S.u[__float_as_int(B2.y)];
                const float4 B0 = q[0], B1 = q[1];
                if (DIFF) {
                    uj.x -= ul.x;
                    uj.y -= ul.y;
                    uj.z -= ul.z;
                }
                a0 = fmaf(B0.z, uj.z, fmaf(B0.y, uj.y, fmaf(B0.x, uj.x, a0)));
                a1 = fmaf(B1.y, uj.z, fmaf(B1.x, uj.y, fmaf(B0.w, uj.x, a1)));
                a2 = fmaf(B2.x, uj.z, fmaf(B1.w, uj.y, fmaf(B1.z, uj.x, a2)));
            }
            a0 += c0;
            a1 += c1;
            a2 += c2;
        }
        for (int o = 1; o < CL_TPR; o <<= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (ok && sub == 0) {
            if (DIFF) {
                const float *D = S.dres + 9 * l;
                a0 = fmaf(D[2], ul.z, fmaf(D[1], ul.y, fmaf(D[0], ul.x, a0)));
                a1 = fmaf(D[5], ul.z, fmaf(D[4], ul.y, fmaf(D[3], ul.x, a1)));
                a2 = fmaf(D[8], ul.z, fmaf(D[7], ul.y, fmaf(D[6], ul.x, a2)));
            }
            const float4 w = make_float4(a0, a1, a2, 0.f);
            if (TO_S) {
                S.s[l] = w;
            } else {
                S.w[l] = w;
                const float4 p = S.p[l], s = S.s[l];
                d += cl_dot3(ul, w);
                e += cl_dot3(ul, s) + cl_dot3(p, w);
                f += cl_dot3(p, s);
            }
        }
    }
}

// FP64 residual b - A x of this CTA's rows, x gathered from the FP64 iterate (own rows
// and ghost copies). Partials (FP64): rr += |r|^2, bb += |b|^2 and, with `install`,
// r = (float) r64 and u = M^-1 r replace the recurrence's r and u (gam += r.u, FP32 dot).
template <bool DIFF, bool BLOCK>
__device__ __forceinline__ void cl_residual(const ClSmem &S, const ClArgs &a, int row0, int nrows, bool install,
                                            float &gam, double &rr, double &bb)
{
    const int sub = threadIdx.x & (CL_TPR - 1), grp = threadIdx.x / CL_TPR;
    for (int l0 = 0; l0 < nrows; l0 += CL_GROUPS) {
        const int l = l0 + grp;
        const bool ok = l < nrows;
        double xl0 = 0.0, xl1 = 0.0, xl2 = 0.0;
        if (ok && DIFF) {
            xl0 = S.x64[4 * l];
            xl1 = S.x64[4 * l + 1];
            xl2 = S.x64[4 * l + 2];
        }
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        if (ok) {
            const int len = S.rl[l];
            constexpr int STEP = 3 * CL_SL * CL_TPR;
            const float4 *q = S.blk + 3 * (S.sb[l / CL_SL] + (l % CL_SL) * CL_TPR + sub);
            for (int k = sub; k < len; k += CL_TPR, q += STEP) {
                const float4 B0 = q[0], B1 = q[1], B2 = q[2];
                const double *xj = S.x64 + 4 * __float_as_int(B2.y);
                double d0 = xj[0], d1 = xj[1], d2 = xj[2];
                if (DIFF) {
                    d0 -= xl0;
                    d1 -= xl1;
                    d2 -= xl2;
                }
                a0 += (double)B0.x * d0 + (double)B0.y * d1 + (double)B0.z * d2;
                a1 += (double)B0.w * d0 + (double)B1.x * d1 + (double)B1.y * d2;
                a2 += (double)B1.z * d0 + (double)B1.w * d1 + (double)B2.x * d2;
            }
        }
        for (int o = 1; o < CL_TPR; o <<= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (ok && sub == 0) {
            if (DIFF) {
                const float *D = S.dres + 9 * l;
                a0 += (double)D[0] * xl0 + (double)D[1] * xl1 + (double)D[2] * xl2;
                a1 += (double)D[3] * xl0 + (double)D[4] * xl1 + (double)D[5] * xl2;
                a2 += (double)D[6] * xl0 + (double)D[7] * xl1 + (double)D[8] * xl2;
            }
            const int64_t row = row0 + l;
            const double b0 = (double)a.b[3 * row], b1 = (double)a.b[3 * row + 1], b2 = (double)a.b[3 * row + 2];
            const double r0 = b0 - a0, r1 = b1 - a1, r2 = b2 - a2;
            rr += r0 * r0 + r1 * r1 + r2 * r2;
            bb += b0 * b0 + b1 * b1 + b2 * b2;
            if (install) {
                const float4 r = make_float4((float)r0, (float)r1, (float)r2, 0.f);
                const float4 u = cl_precond<BLOCK>(S.dinv, l, r);
                S.r[l] = r;
                S.u[l] = u;
                gam += cl_dot3(r, u);
            }
        }
    }
}

// x64 += increment; increment = 0 (this CTA's rows)
__device__ __forceinline__ void cl_fold(const ClSmem &S, int nrows)
{
    for (int l = threadIdx.x; l < nrows; l += CL_THREADS) {
        const float4 d = S.xv[l];
        S.x64[4 * l] += (double)d.x;
        S.x64[4 * l + 1] += (double)d.y;
        S.x64[4 * l + 2] += (double)d.z;
        S.xv[l] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// ------------------------------------------------------------------------- the scalars

// The iteration's scalars and stop state. Every thread holds a copy and updates it from
// the same sums in the same way, so all threads of the cluster take the same decisions;
// after the start and after a residual replacement thread 0 forms them (FP64 work) and the
// CTA copies them from shared memory.
struct ClScal {
    float sigma, tol2, ref2;  // scale of the sums, scaled stop threshold, refresh^2
    float gam_old, rr_last, alpha, beta;
    int iter_last, outer, status, action;
};

__device__ __forceinline__ float cl_scaled(float2 t, float sigma) { return __fadd_rn(t.x, t.y) * sigma; }

// After an iteration's reduction (gamma, r.r, delta, (u,s) + (p,w), (p,s)): the stop tests
// and, unless the solve stops or a replacement follows, the next step's alpha and beta.
__device__ __forceinline__ void cl_step(ClScal &c, const float2 (&tot)[5], int iter, const ClArgs &a)
{
    const float gam = cl_scaled(tot[0], c.sigma), rr = cl_scaled(tot[1], c.sigma);
    int act = 0;
    bool conv = false;
    if (!isfinite(rr) || !isfinite(gam)) {
        c.status = PC_ERR_NONFINITE;
        act = CL_ACT_DONE;
    } else if (rr <= c.tol2) {
        conv = true;
    } else if (iter >= a.max_iter) {
        c.status = PC_ERR_NOT_CONVERGED;
        act = CL_ACT_DONE;
    }
    if (!act) {
        if (!a.mixed) {
            act = conv ? CL_ACT_DONE : 0;
        } else if (conv) {
            // a converged recurrence residual is confirmed by an FP64 replacement
            act = (rr > 0.f && iter > c.iter_last) ? CL_ACT_REPLACE : CL_ACT_DONE;
        } else if (iter % a.check_every == 0) {
            act = CL_ACT_FOLD;
            if (rr <= c.rr_last * c.ref2 || iter - c.iter_last >= a.refresh_every) act |= CL_ACT_REPLACE;
        }
    }
    // beta' = gamma / gamma_old from the recurrence, also when a replacement follows: as in
    // the grid-wide solver the replacement keeps the direction and beta and takes the
    // replaced gamma only into alpha (with the replaced gamma in beta the iteration stalls
    // after a replacement near FP32's attainable accuracy)
    c.beta = __fdividef(gam, c.gam_old);
    if (!(act & (CL_ACT_DONE | CL_ACT_REPLACE))) {
        // alpha' = gamma / (p', A p')
        const float pap = fmaf(c.beta, fmaf(c.beta, cl_scaled(tot[4], c.sigma), cl_scaled(tot[3], c.sigma)),
                               cl_scaled(tot[2], c.sigma));
        c.alpha = __fdividef(gam, pap);
        c.gam_old = gam;
        if (!(pap > 0.f) || !isfinite(c.alpha) || !isfinite(c.beta)) {
            c.status = PC_ERR_NONFINITE;
            act = CL_ACT_DONE;
        }
    }
    c.action = act;
}

// ------------------------------------------------------------------------- the solve

template <bool DIFF, bool BLOCK>
__global__ void __launch_bounds__(CL_THREADS, 1) cluster_pcg_kernel(const ClArgs a)
{
    extern __shared__ __align__(16) unsigned char cl_smem[];
    ClSmem S;
    S.u = reinterpret_cast<float4 *>(cl_smem);
    S.x64 = reinterpret_cast<double *>(cl_smem + a.o_x64);
    S.xv = reinterpret_cast<float4 *>(cl_smem + a.o_xv);
    S.r = reinterpret_cast<float4 *>(cl_smem + a.o_r);
    S.w = reinterpret_cast<float4 *>(cl_smem + a.o_w);
    S.p = reinterpret_cast<float4 *>(cl_smem + a.o_p);
    S.s = reinterpret_cast<float4 *>(cl_smem + a.o_s);
    S.dres = reinterpret_cast<float *>(cl_smem + a.o_dres);
    S.dinv = reinterpret_cast<float *>(cl_smem + a.o_dinv);
    S.rl = reinterpret_cast<int *>(cl_smem + a.o_rs);
    S.sb = S.rl + a.Rc;
    S.bits = reinterpret_cast<uint32_t *>(cl_smem + a.o_bits);
    S.pref = reinterpret_cast<int *>(cl_smem + a.o_pref);
    S.push = reinterpret_cast<uint32_t *>(cl_smem + a.o_push);
    S.red = reinterpret_cast<ClRed *>(cl_smem + a.o_red);
    S.blk = reinterpret_cast<float4 *>(cl_smem + a.o_blk);

    const int tid = threadIdx.x;
    const uint32_t rank = cl_rank(), C = cl_nranks();
    const int Rc = a.Rc, row0 = (int)rank * Rc;
    const int nrows = max(0, min(Rc, a.V - row0));
    int *misc = S.red->misc;
    int par = 0;

    // 1. stored blocks per row (the difference form drops the diagonal block, which
    //    multiplies u_i - u_i = 0; thread l owns row l, Rc <= threads), then the records of
    //    each slice of CL_SL rows and their running sum
    if (tid < nrows) {
        const int row = row0 + tid;
        int cnt = 0;
        for (int k = a.rp[row]; k < a.rp[row + 1]; ++k) cnt += (DIFF && a.ci[k] == row) ? 0 : 1;
        S.rl[tid] = cnt;
    }
    __syncthreads();
    // records per slice: its longest row's blocks, rounded up to CL_TPR, for each of its rows
    const int nsl = (nrows + CL_SL - 1) / CL_SL;
    int ssz = 0;
    if (tid < nsl) {
        int mx = 0;
        for (int i = 0; i < CL_SL; ++i)
            if (tid * CL_SL + i < nrows) mx = max(mx, S.rl[tid * CL_SL + i]);
        ssz = (mx + CL_TPR - 1) / CL_TPR * CL_SL * CL_TPR;
    }
    const int incl = cl_scan(ssz, misc);
    if (tid < nsl) S.sb[tid + 1] = incl;
    if (tid == 0) S.sb[0] = 0;
    const int stored = misc[CL_WARPS - 1];
    // 2. the rows this CTA reads from other CTAs, as a bitmap over all rows
    for (int w = tid; w < a.Vw; w += CL_THREADS) S.bits[w] = 0u;
    __syncthreads();
    if (tid == 0) misc[34] = 0;  // requests received (other CTAs add to it after the next barrier)
    if (tid < nrows) {
        const int row = row0 + tid;
        for (int k = a.rp[row]; k < a.rp[row + 1]; ++k) {
            const int c = a.ci[k];
            if (c < row0 || c >= row0 + nrows) atomicOr(&S.bits[c >> 5], 1u << (c & 31));
        }
    }
    __syncthreads();
    // 3. ghost numbers: a prefix sum of the words' populations (Vw <= threads)
    const int pop = tid < a.Vw ? __popc(S.bits[tid]) : 0;
    const int gincl = cl_scan(pop, misc);
    if (tid < a.Vw) S.pref[tid] = gincl - pop;
    const int n_ghost = misc[CL_WARPS - 1];
    if (cl_vote(&misc[32], stored > a.cap || n_ghost > a.gcap, C)) {
        // some CTA's blocks or ghost rows exceed its shared memory: nobody runs
        if (rank == 0 && tid == 0) {
            a.sc->status = PC_ERR_CAPACITY;
            a.sc->done = 1;
            a.sc->iter = 0;
        }
        cl_sync();
        return;
    }
    // 4. ask each ghost row's owner to send it: (owner's local row, this rank, ghost number)
    for (int w = tid; w < a.Vw; w += CL_THREADS) {
        uint32_t word = S.bits[w];
        int g = S.pref[w];
        while (word) {
            const int c = 32 * w + __ffs(word) - 1;
            word &= word - 1;
            const int o = c / Rc;
            const uint32_t pos = cl_atom_add(cl_map(cl_smem_addr(&misc[34]), (uint32_t)o), 1u);
            if ((int)pos < a.pcap)
                cl_st_u32(cl_map(cl_smem_addr(&S.push[pos]), (uint32_t)o),
                          (rank << 28) | ((uint32_t)g << 10) | (uint32_t)(c - o * Rc));
            ++g;
        }
    }
    // 5. the rows into shared memory; each block's column becomes an index into u / x64
    if (tid < nrows) {
        const int row = row0 + tid;
        const int base = S.sb[tid / CL_SL] + (tid % CL_SL) * CL_TPR;
        int n = 0;  // stored blocks of the row so far
        for (int k = a.rp[row]; k < a.rp[row + 1]; ++k) {
            const int c = a.ci[k];
            if (DIFF && c == row) continue;
            const int pos = base + (n / CL_TPR) * (CL_SL * CL_TPR) + n % CL_TPR;
            int j;
            if (c >= row0 && c < row0 + nrows) {
                j = c - row0;
            } else {
                const uint32_t word = S.bits[c >> 5], below = (1u << (c & 31)) - 1u;
                j = Rc + S.pref[c >> 5] + __popc(word & below);
            }
            const float *B = a.vals + 9ll * k;
            S.blk[3 * pos] = make_float4(B[0], B[1], B[2], B[3]);
            S.blk[3 * pos + 1] = make_float4(B[4], B[5], B[6], B[7]);
            S.blk[3 * pos + 2] = make_float4(B[8], __int_as_float(j), 0.f, 0.f);
            ++n;
        }
        if (DIFF)
#pragma unroll
            for (int e = 0; e < 9; ++e) S.dres[9 * tid + e] = a.dres[9ll * row + e];
        if (BLOCK) {
            const float4 *d4 = reinterpret_cast<const float4 *>(a.dinv);
            for (int q = 0; q < 3; ++q) {
                const float4 d = d4[3ll * row + q];
                S.dinv[9 * tid + 3 * q] = d.x;
                S.dinv[9 * tid + 3 * q + 1] = d.y;
                S.dinv[9 * tid + 3 * q + 2] = d.z;
            }
        } else {
            reinterpret_cast<float4 *>(S.dinv)[tid] =
                make_float4(a.dinv[3ll * row], a.dinv[3ll * row + 1], a.dinv[3ll * row + 2], 0.f);
        }
        for (int e = 0; e < 3; ++e) S.x64[4 * tid + e] = (double)a.dv[3ll * row + e];
        S.x64[4 * tid + 3] = 0.0;
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        S.xv[tid] = zero;
        S.p[tid] = zero;
        S.s[tid] = zero;
    }
    // every request has landed after this barrier; an owner asked for more rows than it
    // can list stops everybody
    if (cl_vote(&misc[33], misc[34] > a.pcap, C)) {
        if (rank == 0 && tid == 0) {
            a.sc->status = PC_ERR_CAPACITY;
            a.sc->done = 1;
            a.sc->iter = 0;
        }
        cl_sync();
        return;
    }
    const int n_push = misc[34];
    // sort the send list by (destination, ghost number): consecutive lanes then send
    // consecutive rows into consecutive ghost slots of one CTA, and the remote stores
    // coalesce (the requests arrived in the order of the requesters' atomics). A bitonic
    // sort over the list padded to a power of two with entries that sort last.
    {
        int n2 = 1;
        while (n2 < n_push) n2 <<= 1;
        for (int i = n_push + tid; i < n2; i += CL_THREADS) S.push[i] = 0xFFFFFFFFu;
        __syncthreads();
        for (int k = 2; k <= n2; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = tid; i < n2; i += CL_THREADS) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const uint32_t x = S.push[i], y = S.push[ixj];
                        if ((i & k) == 0 ? x > y : x < y) {
                            S.push[i] = y;
                            S.push[ixj] = x;
                        }
                    }
                }
                __syncthreads();
            }
    }

    // 6. the start: r = b - A dv in FP64 (rounded to FP32), u = M^-1 r, w = A u; p = s = 0
    ClRed &K = *S.red;
    ClScal c;
    static_assert(sizeof(ClScal) <= sizeof(K.scal), "scalars fit their broadcast slot");
    auto from_thread0 = [&]() {  // thread 0's scalars to the whole CTA
        if (tid == 0) *reinterpret_cast<ClScal *>(K.scal) = c;
        __syncthreads();
        c = *reinterpret_cast<const ClScal *>(K.scal);
    };
    float2 tot[5];
    {
        cl_push_x64(S, Rc, n_push);
        cl_sync();
        float gam = 0.f, d = 0.f, e = 0.f, f = 0.f;
        double rr = 0.0, bb = 0.0;
        cl_residual<DIFF, BLOCK>(S, a, row0, nrows, true, gam, rr, bb);
        __syncthreads();
        cl_push_u(S, Rc, n_push);
        cl_sync();
        cl_product<DIFF>(S, nrows, d, e, f);
        const float2 v[4] = {make_float2(gam, 0.f), cl_pair(rr), make_float2(d, 0.f), cl_pair(bb)};
        float2 t4[4];
        cl_reduce<4, true>(v, t4, S, par, C, rank);
        if (tid == 0) {
            // a power of two that brings b.b near 1 keeps the FP32 scalars far from the
            // range limits (the scaling is exact)
            const double bbv = pc_df_value(t4[3].x, t4[3].y);
            int ex = 0;
            if (isfinite(bbv) && bbv > 0.0) frexp(bbv, &ex);
            c.sigma = ldexpf(1.f, -ex);
            c.tol2 = (float)ldexp(a.tol * a.tol * bbv, -ex);
            c.ref2 = (float)(a.refresh * a.refresh);
            K.bb64 = bbv;
            K.rr64 = pc_df_value(t4[1].x, t4[1].y);
            const float gam0 = cl_scaled(t4[0], c.sigma), rr0 = cl_scaled(t4[1], c.sigma);
            const float del0 = cl_scaled(t4[2], c.sigma);
            c.alpha = gam0 / del0;
            c.beta = 0.f;
            c.gam_old = gam0;
            c.rr_last = rr0;
            c.status = PC_OK;
            c.iter_last = 0;
            c.outer = 0;
            int act = 0;
            if (!isfinite(rr0) || !isfinite(gam0)) {
                c.status = PC_ERR_NONFINITE;
                act = CL_ACT_DONE;
            } else if (rr0 <= c.tol2) {
                act = CL_ACT_DONE;
            } else if (a.max_iter <= 0) {
                c.status = PC_ERR_NOT_CONVERGED;
                act = CL_ACT_DONE;
            } else if (!(del0 > 0.f) || !isfinite(c.alpha)) {
                c.status = PC_ERR_NONFINITE;
                act = CL_ACT_DONE;
            }
            c.action = act;
        }
        from_thread0();
    }
    int iter = 0;

    while (!(c.action & CL_ACT_DONE)) {
        const float alpha = c.alpha, beta = c.beta;
        // p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = M^-1 r; (r, u), (r, r)
        float g = 0.f, q = 0.f;
        for (int l = tid; l < nrows; l += CL_THREADS) {
            const float4 p = cl_axpy(beta, S.p[l], S.u[l]), s = cl_axpy(beta, S.s[l], S.w[l]);
            const float4 x = cl_axpy(alpha, p, S.xv[l]), r = cl_axpy(-alpha, s, S.r[l]);
            const float4 u = cl_precond<BLOCK>(S.dinv, l, r);
            S.p[l] = p;
            S.s[l] = s;
            S.xv[l] = x;
            S.r[l] = r;
            S.u[l] = u;
            g += cl_dot3(r, u);
            q += cl_dot3(r, r);
        }
        __syncthreads();
        cl_push_u(S, Rc, n_push);
        cl_sync();
        float d = 0.f, e = 0.f, f = 0.f;
        cl_product<DIFF>(S, nrows, d, e, f);
        {
            const float2 v[5] = {make_float2(g, 0.f), make_float2(q, 0.f), make_float2(d, 0.f), make_float2(e, 0.f),
                                 make_float2(f, 0.f)};
            cl_reduce<5, false>(v, tot, S, par, C, rank);
        }
        ++iter;
        cl_step(c, tot, iter, a);  // every thread, the same values
        if (c.action & (CL_ACT_FOLD | CL_ACT_REPLACE)) cl_fold(S, nrows);
        if (c.action & CL_ACT_REPLACE) {
            // r = b - A x in FP64, u = M^-1 r, and the products s = A p and w = A u anew
            // (the recurrences for s and r drift; p stays)
            __syncthreads();  // every row folded before any is sent
            cl_push_x64(S, Rc, n_push);
            cl_sync();
            float gr = 0.f, d2 = 0.f, e2 = 0.f, f2 = 0.f;
            double rr64 = 0.0, bb_unused = 0.0;
            cl_residual<DIFF, BLOCK>(S, a, row0, nrows, true, gr, rr64, bb_unused);
            __syncthreads();
            for (int l = tid; l < nrows; l += CL_THREADS) {  // u aside in w, p through the product
                S.w[l] = S.u[l];
                S.u[l] = S.p[l];
            }
            __syncthreads();
            cl_push_u(S, Rc, n_push);
            cl_sync();
            cl_product<DIFF, true>(S, nrows, d2, e2, f2);
            __syncthreads();
            for (int l = tid; l < nrows; l += CL_THREADS) S.u[l] = S.w[l];
            cl_sync();  // every CTA's product of p done before u overwrites the ghost copies
            cl_push_u(S, Rc, n_push);
            cl_sync();
            cl_product<DIFF>(S, nrows, d2, e2, f2);
            const float2 v[5] = {make_float2(gr, 0.f), cl_pair(rr64), make_float2(d2, 0.f), make_float2(e2, 0.f),
                                 make_float2(f2, 0.f)};
            cl_reduce<5, true>(v, tot, S, par, C, rank);
            if (tid == 0) {
                K.rr64 = pc_df_value(tot[1].x, tot[1].y);
                const float gam = cl_scaled(tot[0], c.sigma), rr = cl_scaled(tot[1], c.sigma);
                c.rr_last = rr;
                c.iter_last = iter;
                ++c.outer;
                int act = 0;
                if (!isfinite(rr) || !isfinite(gam)) {
                    c.status = PC_ERR_NONFINITE;
                    act = CL_ACT_DONE;
                } else if (rr <= c.tol2) {
                    act = CL_ACT_DONE;
                } else if (iter >= a.max_iter) {
                    c.status = PC_ERR_NOT_CONVERGED;
                    act = CL_ACT_DONE;
                } else {
                    // the recurrence's beta, the replaced gamma in alpha
                    const float pap = fmaf(c.beta, fmaf(c.beta, cl_scaled(tot[4], c.sigma), cl_scaled(tot[3], c.sigma)),
                                           cl_scaled(tot[2], c.sigma));
                    c.alpha = __fdividef(gam, pap);
                    c.gam_old = gam;
                    if (!(pap > 0.f) || !isfinite(c.alpha) || !isfinite(c.beta)) {
                        c.status = PC_ERR_NONFINITE;
                        act = CL_ACT_DONE;
                    }
                }
                c.action = act;
            }
            from_thread0();
        }
    }

    // 7. the solution, and its FP64 residual unless the last replacement measured it
    const bool check = a.mixed ? iter > c.iter_last : true;
    if (a.mixed) {
        if (check) cl_fold(S, nrows);
        for (int l = tid; l < nrows; l += CL_THREADS) {
            const int64_t row = row0 + l;
            for (int e = 0; e < 3; ++e) {
                const double x = S.x64[4 * l + e];
                const float d = (float)x;
                a.dv[3 * row + e] = d;
                if (a.x64) a.x64[3 * row + e] = x;
                if (check) S.x64[4 * l + e] = (double)d;
            }
        }
    } else {
        for (int l = tid; l < nrows; l += CL_THREADS) {
            const int64_t row = row0 + l;
            const float4 x = S.xv[l];
            const float d0 = a.dv[3 * row] + x.x, d1 = a.dv[3 * row + 1] + x.y, d2 = a.dv[3 * row + 2] + x.z;
            a.dv[3 * row] = d0;
            a.dv[3 * row + 1] = d1;
            a.dv[3 * row + 2] = d2;
            S.x64[4 * l] = (double)d0;
            S.x64[4 * l + 1] = (double)d1;
            S.x64[4 * l + 2] = (double)d2;
        }
    }
    if (check) {
        __syncthreads();
        cl_push_x64(S, Rc, n_push);
        cl_sync();
        float g_unused = 0.f;
        double rr64 = 0.0, bb = 0.0;
        cl_residual<DIFF, BLOCK>(S, a, row0, nrows, false, g_unused, rr64, bb);
        const float2 v[2] = {cl_pair(rr64), cl_pair(bb)};
        float2 t2[2];
        cl_reduce<2, true>(v, t2, S, par, C, rank);
        if (tid == 0) {
            K.rr64 = pc_df_value(t2[0].x, t2[0].y);
            K.bb64 = pc_df_value(t2[1].x, t2[1].y);
        }
    }
    cl_sync();
    if (rank == 0 && tid == 0) {
        pc_scalars *sc = a.sc;
        sc->rz = (double)(c.gam_old / c.sigma);
        sc->rr = K.rr64;
        sc->bb = K.bb64;
        sc->tol2 = a.tol * a.tol * K.bb64;
        sc->alpha = (double)c.alpha;
        sc->beta = (double)c.beta;
        sc->pq = 0.0;
        sc->iter = iter;
        sc->max_iter = a.max_iter;
        sc->status = c.status;
        sc->done = 1;
        sc->outer = c.outer;
    }
}

// ------------------------------------------------------------------------- host side

template <bool DIFF, bool BLOCK>
static pc_status cl_config(int C, size_t smem, cudaStream_t st, cudaLaunchConfig_t *cfg, cudaLaunchAttribute *at)
{
    auto kern = cluster_pcg_kernel<DIFF, BLOCK>;
    PC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    *cfg = cudaLaunchConfig_t{};
    cfg->gridDim = dim3((unsigned)C, 1, 1);
    cfg->blockDim = dim3(CL_THREADS, 1, 1);
    cfg->dynamicSmemBytes = smem;
    cfg->stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg->attrs = at;
    cfg->numAttrs = 1;
    return PC_OK;
}

// The largest cluster (16, else 8 CTAs) that the device can run with this shared memory.
template <bool DIFF, bool BLOCK>
static pc_status cl_size(size_t smem, int *C)
{
    *C = 0;
    for (int cand : {16, 8}) {
        cudaLaunchConfig_t cfg;
        cudaLaunchAttribute at[1];
        PC_TRY((cl_config<DIFF, BLOCK>(cand, smem, 0, &cfg, at)));
        int n = 0;
        const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, cluster_pcg_kernel<DIFF, BLOCK>, &cfg);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();  // an unsupported size is not an error of the solve
            continue;
        }
        if (n >= 1) {
            *C = cand;
            return PC_OK;
        }
    }
    return PC_OK;
}

// Shared-memory layout for V rows over C CTAs; false when the rows do not fit. The room
// left after the per-row arrays goes to the blocks (the average CTA's share and an eighth
// more) and then to ghost rows; the kernel itself refuses a CTA whose blocks, ghost rows
// or send list exceed what it got, and the automatic schedule then solves on the grid.
static bool cl_layout(int V, int C, bool diff, bool block, size_t smax, int64_t stored, ClArgs *a, size_t *smem)
{
    const int Rc = (V + C - 1) / C;
    const int Vw = (V + 31) / 32;
    if (Rc < 1 || Rc > CL_THREADS || Vw > CL_THREADS) return false;
    auto layout = [&](int gcap, int pcap, size_t *end) {
        size_t o = 0;
        auto take = [&](size_t bytes) {
            const size_t at = o;
            o += (bytes + 15) & ~(size_t)15;
            return (uint32_t)at;
        };
        take(16ull * (Rc + gcap));
        a->o_x64 = take(32ull * (Rc + gcap));
        a->o_xv = take(16ull * Rc);
        a->o_r = take(16ull * Rc);
        a->o_w = take(16ull * Rc);
        a->o_p = take(16ull * Rc);
        a->o_s = take(16ull * Rc);
        a->o_dres = take(diff ? 36ull * Rc : 0);
        a->o_dinv = take((block ? 36ull : 16ull) * Rc);
        a->o_rs = take(4ull * (Rc + Rc / CL_SL + 2));
        a->o_bits = take(4ull * Vw);
        a->o_pref = take(4ull * Vw);
        int p2 = 1;
        while (p2 < pcap) p2 <<= 1;
        a->o_push = take(4ull * p2);
        a->o_red = take(sizeof(ClRed));
        *end = o;
    };
    size_t fixed = 0;
    layout(0, 0, &fixed);
    const int64_t share = (stored + C - 1) / C;
    const int64_t want = share + share / 8 + 32;
    if ((int64_t)fixed + 48 * want >= (int64_t)smax) return false;
    // a ghost row costs 16 (u) + 32 (FP64 iterate) + 4 (a send-list entry) bytes
    const int64_t room = ((int64_t)smax - (int64_t)fixed - 48 * want) / 52;
    const int gcap = (int)std::min<int64_t>(std::min(V, 2048), room);
    const int pcap = gcap;
    size_t o = 0;
    layout(gcap, pcap, &o);
    // blocks: 48 bytes each (nine values, the column's index, two pad words)
    const int64_t cap = (int64_t)((smax - o) / 48);
    if (cap < 8 || share > cap) return false;
    a->o_blk = (uint32_t)o;
    *smem = o + 48 * (size_t)cap;
    if (*smem > smax) return false;
    a->Rc = Rc;
    a->Vw = Vw;
    a->cap = (int)cap;
    a->gcap = gcap;
    a->pcap = pcap;
    return true;
}

template <bool DIFF, bool BLOCK>
static pc_status cl_run(pc_ctx *c, const ClArgs &args, int C, size_t smem, cudaStream_t st)
{
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    PC_TRY((cl_config<DIFF, BLOCK>(C, smem, st, &cfg, at)));
    const bool timed = c->profiling && c->ev_used >= 6;
    if (timed) PC_CUDA_TRY(cudaEventRecord(c->ev[4], st));
    PC_CUDA_TRY(cudaLaunchKernelEx(&cfg, cluster_pcg_kernel<DIFF, BLOCK>, args));
    c->launches++;
    if (timed) PC_CUDA_TRY(cudaEventRecord(c->ev[5], st));
    return PC_OK;
}

pc_status pc_cluster_solve(pc_ctx *c, const pc_bsr *A, const float *vals, const float *dres, const float *b,
                           float *dv, const pc_solve_opts &o, bool block, bool required, pc_solve_info *info,
                           cudaStream_t st, bool *ran)
{
    *ran = false;
    const int V = c->V;
    const bool diff = dres != nullptr;
    int smax = 0;
    PC_CUDA_TRY(cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    int C = c->cl_size;
    if (C == 0) {
        if (diff && block) PC_TRY((cl_size<true, true>((size_t)smax, &C)));
        else if (diff) PC_TRY((cl_size<true, false>((size_t)smax, &C)));
        else if (block) PC_TRY((cl_size<false, true>((size_t)smax, &C)));
        else PC_TRY((cl_size<false, false>((size_t)smax, &C)));
        c->cl_size = C > 0 ? C : -1;
    }
    ClArgs a{};
    size_t smem = 0;
    if (C <= 0 || V < 1 || !cl_layout(V, C, diff, block, (size_t)smax, A->nnzb - (diff ? V : 0), &a, &smem))
        return required ? PC_ERR_CAPACITY : PC_OK;
    a.V = V;
    a.rp = A->row_ptr;
    a.ci = A->col_idx;
    a.vals = vals;
    a.dres = dres;
    a.dinv = c->dinv;
    a.b = b;
    a.dv = dv;
    a.x64 = o.precision == PC_PREC_MIXED ? c->x64 : nullptr;
    a.tol = o.tol;
    a.refresh = o.refresh;
    a.max_iter = o.max_iter;
    a.check_every = o.check_every;
    a.refresh_every = o.refresh_every;
    a.mixed = o.precision == PC_PREC_MIXED ? 1 : 0;
    a.sc = c->sc;
    if (diff && block) PC_TRY((cl_run<true, true>(c, a, C, smem, st)));
    else if (diff) PC_TRY((cl_run<true, false>(c, a, C, smem, st)));
    else if (block) PC_TRY((cl_run<false, true>(c, a, C, smem, st)));
    else PC_TRY((cl_run<false, false>(c, a, C, smem, st)));
    PC_CUDA_TRY(cudaMemcpyAsync(c->sc_host, c->sc, sizeof(pc_scalars), cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    if (c->profiling && c->ev_used >= 6) {
        float ms = 0.f;
        PC_CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]));
        c->cl_ms += ms;
        c->cl_solves += 1;
        c->cl_iters += c->sc_host->iter;
    }
    const pc_scalars fin = *c->sc_host;
    if (fin.status == PC_ERR_CAPACITY) return required ? PC_ERR_CAPACITY : PC_OK;
    *ran = true;
    if (info) {
        pc_solve_info inf{};
        inf.iters = fin.iter;
        inf.outer = fin.outer;
        inf.bnorm = sqrt(fin.bb);
        inf.rel_res = fin.bb > 0 ? sqrt(fin.rr / fin.bb) : 0.0;
        *info = inf;
    }
    return (pc_status)fin.status;
}
