// The whole PCG solve of a small system in one launch of one thread-block cluster
// (Sec. 2.5: the linear equations are solved with a preconditioned conjugate gradient
// solver; Sec. 3.1: the SpMV and the vector operations are data parallel).
//
// A system of a few thousand vertices leaves the grid-wide solver latency-bound: each
// iteration pays two kernel boundaries and a grid-wide barrier for a few microseconds of
// work. Here up to 16 CTAs of one cluster (one CTA per SM) hold the whole system in their
// shared memory for the length of the solve:
//   - CTA c owns rows [c Rc, (c+1) Rc). It copies its rows' 3x3 blocks (without the
//     diagonal block in the difference form), its rows' difference-form diagonal and
//     Jacobi inverse into shared memory once, and keeps x, r and q of its rows there.
//   - Per row a record (ClRec) holds what the other CTAs read: the search direction
//     (two copies, by iteration parity), z and the FP64 iterate. Each stored block keeps,
//     instead of its column index, the distributed-shared-memory address of its column's
//     record, so the product gathers p and z straight from the owning CTA's shared memory.
//   - Dot products: FP32 within a thread, FP64 across threads; each CTA's sum goes to a
//     shared slot, a cluster barrier (barrier.cluster arrive.release / wait.acquire)
//     publishes it, and every warp of every CTA then adds the C slots in the same fixed
//     order, so all threads hold bitwise the same scalars and take the same decisions.
// Per iteration two cluster barriers: after q = A p (for p.q) and after the update (for
// r.z and r.r). The direction step p = z + beta p needs no third one: the product forms
// each gathered p_j = z_j + beta p_j itself from the owner's record (bitwise the value
// the owner forms), and the owner stores its p into the record copy of the other parity,
// which nobody reads in that iteration.
//
// Mixed precision as in the grid-wide solver: the FP32 increment is folded into the FP64
// iterate every check_every iterations, and the residual is recomputed in FP64 (the
// product gathers the FP64 iterate) when the recurrence residual has dropped by
// refresh^2, after refresh_every iterations, and to confirm convergence; the replaced z
// enters the next direction step, the direction itself is kept.
//
// The kernel has no spin-waits: the cluster's CTAs are co-scheduled by the hardware and
// its barriers are hardware barriers; every branch around a barrier depends only on the
// shared scalars, so all threads of the cluster reach every barrier. The last barrier
// keeps each CTA resident until no other CTA can still read its shared memory.
#include <math.h>

#include "pc_internal.cuh"

#define CL_THREADS 1024
#define CL_TPR 4                         // threads per row in the products
#define CL_GROUPS (CL_THREADS / CL_TPR)  // rows in flight per CTA
#define CL_WARPS (CL_THREADS / 32)

// Per row, in the owning CTA's shared memory: the entries other CTAs gather.
struct __align__(16) ClRec {
    float4 p[2];   // direction of the previous iteration, by iteration parity
    float4 z;      // preconditioned residual
    double x[3];   // FP64 iterate (mixed precision); the final solution for the last residual
    double pad;
};
static_assert(sizeof(ClRec) == 80, "record layout");
#define CL_REC_Z 32
#define CL_REC_X 48

struct ClArgs {
    int V, Rc, cap;
    const int32_t *rp, *ci;
    const float *vals, *dres, *dinv, *b;
    float *dv;
    double *x64;  // mixed precision: the FP64 solution on exit (may be null)
    double tol, refresh;
    int max_iter, check_every, refresh_every, mixed;
    pc_scalars *sc;
    // byte offsets of the shared-memory arrays (the records start at 0)
    uint32_t o_x, o_r, o_q, o_dres, o_dinv, o_rs, o_red, o_addr, o_vals;
};

struct ClSmem {
    ClRec *rec;
    float4 *xv, *rv, *qv;  // FP32 increment, residual, A p
    float *dres;           // [Rc][9]
    float4 *dinv;          // [Rc] (scalar Jacobi: 3 used) or [Rc][3] (rows of the block inverse)
    int *rs;               // [Rc + 1] row starts into the stored blocks
    uint32_t *addr;        // [cap] cluster address of each block's column record
    float *vals;           // [cap][9]
    double *red_w;         // [CL_WARPS][4] warp sums
    double *red_c;         // [2][4] this CTA's sums, read by every CTA (double-buffered)
    int *misc;             // [40] scan scratch (0..31), capacity flag (32)
    struct ClBcast *bc;    // thread 0's word to its CTA
    struct ClCtl *ctl;     // thread 0's scalars
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
__device__ __forceinline__ float4 cl_ld_f4(uint32_t a)
{
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(a));
    return v;
}
__device__ __forceinline__ double2 cl_ld_d2(uint32_t a)
{
    double2 v;
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ double cl_ld_d(uint32_t a)
{
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t cl_ld_u32(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

// xor butterfly: every lane ends with bitwise the same sum (addition commutes)
__device__ __forceinline__ double cl_warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum N per-thread values over the cluster; the totals land in every lane of warp 0, in
// every CTA bitwise the same: warp sums, this CTA's sum of its warp sums (warp 0, warp
// order) into its slot of parity `par`, a cluster barrier, and the C slots added in rank
// order by warp 0. The iterations' dot products (FP32 per thread) are added as
// double-float pairs (pc_df_add: FP32 arithmetic only -- GB300 runs FP64 at about 1/60 of
// its FP32 rate, and FP64 butterflies in every thread would cost more than the iteration
// itself); the rare FP64 residual passes add doubles.
template <int N>
__device__ __forceinline__ void cl_reduce_df(const float (&v)[N], float2 (&tot)[N], const ClSmem &S, int &par,
                                             uint32_t C)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2 *red_w = reinterpret_cast<float2 *>(S.red_w);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        float hi = v[i], lo = 0.f;
        pc_warp_sum_df(hi, lo);
        if (lane == 0) red_w[4 * warp + i] = make_float2(hi, lo);
    }
    __syncthreads();
    float2 *slot = reinterpret_cast<float2 *>(S.red_c + 4 * par);
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            float2 w = red_w[4 * lane + i];
            pc_warp_sum_df(w.x, w.y);
            if (lane == 0) slot[i] = w;
        }
    }
    cl_sync();
    if (warp == 0) {
        const uint32_t base = cl_smem_addr(slot);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            float hi = 0.f, lo = 0.f;
            if ((uint32_t)lane < C) {
                const double w = cl_ld_d(cl_map(base + 8u * i, lane));  // the pair's 8 bytes
                const float2 f = *reinterpret_cast<const float2 *>(&w);
                hi = f.x;
                lo = f.y;
            }
            pc_warp_sum_df(hi, lo);
            tot[i] = make_float2(hi, lo);
        }
    }
    // the slots of this parity are rewritten two reductions later, after a barrier that
    // every CTA reaches only once it has read them
    par ^= 1;
}
template <int N>
__device__ __forceinline__ void cl_reduce_d(double (&v)[N], double (&tot)[N], const ClSmem &S, int &par, uint32_t C)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = cl_warp_sum(v[i]);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) S.red_w[4 * warp + i] = v[i];
    __syncthreads();
    double *slot = S.red_c + 4 * par;
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const double s = cl_warp_sum(S.red_w[4 * lane + i]);
            if (lane == 0) slot[i] = s;
        }
    }
    cl_sync();
    if (warp == 0) {
        const uint32_t base = cl_smem_addr(slot);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const double s = (uint32_t)lane < C ? cl_ld_d(cl_map(base + 8u * i, lane)) : 0.0;
            tot[i] = cl_warp_sum(s);
        }
    }
    par ^= 1;
}

// What thread 0 of each CTA (the same decision in every CTA) tells its CTA after a
// reduction: the step length or direction coefficient and what comes next.
struct ClBcast {
    float alpha, beta;
    int action;
    int check;
};
// Thread 0's FP64 scalars and stop state, kept in shared memory rather than in registers
// that every thread would have to reserve.
struct ClCtl {
    double rz, rr, bb, tol2, rr_last;
    float rz_f;  // rz rounded, for the FP32 quotients
    int status, iter_last, outer, bad_pq;
};
#define CL_ACT_DONE 1
#define CL_ACT_FOLD 2
#define CL_ACT_REPLACE 4

// ------------------------------------------------------------------------- row arithmetic

template <bool BLOCK>
__device__ __forceinline__ float4 cl_precond(const float4 *dinv, int l, float4 r)
{
    if (BLOCK) {
        const float4 a = dinv[3 * l], b = dinv[3 * l + 1], c = dinv[3 * l + 2];
        return make_float4(a.x * r.x + a.y * r.y + a.z * r.z, b.x * r.x + b.y * r.y + b.z * r.z,
                           c.x * r.x + c.y * r.y + c.z * r.z, 0.f);
    }
    const float4 d = dinv[l];
    return make_float4(d.x * r.x, d.y * r.y, d.z * r.z, 0.f);
}

__device__ __forceinline__ float cl_dot3(float4 a, float4 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }

// the direction step p = z + beta p_prev
__device__ __forceinline__ float4 cl_dir(float beta, float4 p, float4 z)
{
    return make_float4(fmaf(beta, p.x, z.x), fmaf(beta, p.y, z.y), fmaf(beta, p.z, z.z), 0.f);
}

// FP64 residual b - A x of this CTA's rows, x gathered from the records' FP64 iterate.
// Partials: t[1] += |r|^2, t[2] += |b|^2 and, with `install`, r = (float) r64 and
// z = D^-1 r replace the recurrence's r and z (t[0] += r.z).
template <bool DIFF, bool BLOCK>
__device__ __forceinline__ void cl_residual(const ClSmem &S, const ClArgs &a, int row0, int nrows, bool install,
                                            double t[3])
{
    const int sub = threadIdx.x & (CL_TPR - 1), grp = threadIdx.x / CL_TPR;
    t[0] = t[1] = t[2] = 0.0;
    for (int l0 = 0; l0 < nrows; l0 += CL_GROUPS) {
        const int l = l0 + grp;
        const bool ok = l < nrows;
        double xl0 = 0.0, xl1 = 0.0, xl2 = 0.0;
        if (ok && DIFF) {
            xl0 = S.rec[l].x[0];
            xl1 = S.rec[l].x[1];
            xl2 = S.rec[l].x[2];
        }
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        if (ok) {
            const int k1 = S.rs[l + 1];
            for (int k = S.rs[l] + sub; k < k1; k += CL_TPR) {
                const uint32_t ad = S.addr[k];
                const double2 x01 = cl_ld_d2(ad + CL_REC_X);
                double d0 = x01.x, d1 = x01.y, d2 = cl_ld_d(ad + CL_REC_X + 16);
                if (DIFF) {
                    d0 -= xl0;
                    d1 -= xl1;
                    d2 -= xl2;
                }
                const float *B = S.vals + 9 * k;
                a0 += (double)B[0] * d0 + (double)B[1] * d1 + (double)B[2] * d2;
                a1 += (double)B[3] * d0 + (double)B[4] * d1 + (double)B[5] * d2;
                a2 += (double)B[6] * d0 + (double)B[7] * d1 + (double)B[8] * d2;
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
            t[1] += r0 * r0 + r1 * r1 + r2 * r2;
            t[2] += b0 * b0 + b1 * b1 + b2 * b2;
            if (install) {
                const float4 r = make_float4((float)r0, (float)r1, (float)r2, 0.f);
                const float4 z = cl_precond<BLOCK>(S.dinv, l, r);
                S.rv[l] = r;
                S.rec[l].z = z;
                t[0] += (double)cl_dot3(r, z);
            }
        }
    }
}

// x64 += increment; increment = 0 (this CTA's rows)
__device__ __forceinline__ void cl_fold(const ClSmem &S, int nrows)
{
    for (int l = threadIdx.x; l < nrows; l += CL_THREADS) {
        const float4 d = S.xv[l];
        S.rec[l].x[0] += (double)d.x;
        S.rec[l].x[1] += (double)d.y;
        S.rec[l].x[2] += (double)d.z;
        S.xv[l] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// ------------------------------------------------------------------------- the solve

template <bool DIFF, bool BLOCK>
__global__ void __launch_bounds__(CL_THREADS, 1) cluster_pcg_kernel(const ClArgs a)
{
    extern __shared__ __align__(16) unsigned char cl_smem[];
    ClSmem S;
    S.rec = reinterpret_cast<ClRec *>(cl_smem);
    S.xv = reinterpret_cast<float4 *>(cl_smem + a.o_x);
    S.rv = reinterpret_cast<float4 *>(cl_smem + a.o_r);
    S.qv = reinterpret_cast<float4 *>(cl_smem + a.o_q);
    S.dres = reinterpret_cast<float *>(cl_smem + a.o_dres);
    S.dinv = reinterpret_cast<float4 *>(cl_smem + a.o_dinv);
    S.rs = reinterpret_cast<int *>(cl_smem + a.o_rs);
    S.red_w = reinterpret_cast<double *>(cl_smem + a.o_red);
    S.red_c = S.red_w + 4 * CL_WARPS;
    S.misc = reinterpret_cast<int *>(S.red_c + 8);
    S.ctl = reinterpret_cast<ClCtl *>(S.misc + 40);
    S.bc = reinterpret_cast<ClBcast *>(S.ctl + 1);
    S.addr = reinterpret_cast<uint32_t *>(cl_smem + a.o_addr);
    S.vals = reinterpret_cast<float *>(cl_smem + a.o_vals);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sub = tid & (CL_TPR - 1), grp = tid / CL_TPR;
    const uint32_t rank = cl_rank(), C = cl_nranks();
    const int Rc = a.Rc, row0 = (int)rank * Rc;
    const int nrows = max(0, min(Rc, a.V - row0));
    int par = 0;

    // 1. stored blocks per row (the difference form drops the diagonal block, which
    //    multiplies p_i - p_i = 0) and their running sum: thread l owns row l (Rc <= threads)
    int cnt = 0;
    if (tid < nrows) {
        const int row = row0 + tid;
        for (int k = a.rp[row]; k < a.rp[row + 1]; ++k) cnt += (DIFF && a.ci[k] == row) ? 0 : 1;
    }
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
    }
    if (lane == 31) S.misc[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = S.misc[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int n = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += n;
        }
        S.misc[lane] = w;
    }
    __syncthreads();
    if (warp > 0) incl += S.misc[warp - 1];
    if (tid < nrows) S.rs[tid + 1] = incl;
    if (tid == 0) {
        S.rs[0] = 0;
        S.misc[32] = S.misc[CL_WARPS - 1] > a.cap ? 1 : 0;
    }
    cl_sync();
    // every CTA learns whether any CTA's blocks exceed its stage (then nobody runs)
    const uint32_t flag = (uint32_t)lane < C ? cl_ld_u32(cl_map(cl_smem_addr(S.misc + 32), lane)) : 0u;
    if (__any_sync(0xffffffffu, flag != 0u)) {
        if (rank == 0 && tid == 0) {
            a.sc->status = PC_ERR_CAPACITY;
            a.sc->done = 1;
            a.sc->iter = 0;
        }
        cl_sync();
        return;
    }

    // 2. the rows into shared memory; each block's column becomes its record's address
    if (tid < nrows) {
        const int row = row0 + tid;
        int pos = S.rs[tid];
        const uint32_t rec0 = cl_smem_addr(S.rec);
        for (int k = a.rp[row]; k < a.rp[row + 1]; ++k) {
            const int c = a.ci[k];
            if (DIFF && c == row) continue;
            const int owner = c / Rc;
            S.addr[pos] = cl_map(rec0 + (uint32_t)(c - owner * Rc) * (uint32_t)sizeof(ClRec), (uint32_t)owner);
            const float *B = a.vals + 9ll * k;
#pragma unroll
            for (int e = 0; e < 9; ++e) S.vals[9 * pos + e] = B[e];
            ++pos;
        }
        if (DIFF)
#pragma unroll
            for (int e = 0; e < 9; ++e) S.dres[9 * tid + e] = a.dres[9ll * row + e];
        if (BLOCK) {
            const float4 *d4 = reinterpret_cast<const float4 *>(a.dinv);
            for (int j = 0; j < 3; ++j) S.dinv[3 * tid + j] = d4[3ll * row + j];
        } else {
            S.dinv[tid] = make_float4(a.dinv[3ll * row], a.dinv[3ll * row + 1], a.dinv[3ll * row + 2], 0.f);
        }
        ClRec &R = S.rec[tid];
        R.p[0] = R.p[1] = R.z = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int e = 0; e < 3; ++e) R.x[e] = (double)a.dv[3ll * row + e];
        R.pad = 0.0;
        S.xv[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    cl_sync();

    // 3. the start: r = b - A dv in FP64 (rounded to FP32), z = D^-1 r, p_prev = 0.
    // The FP64 scalars and the stop logic belong to thread 0 of each CTA (S.ctl); the CTA
    // learns alpha, beta and the next action from it (S.bc).
    ClCtl &K = *S.ctl;
    {
        double t[3], tot[3];
        cl_residual<DIFF, BLOCK>(S, a, row0, nrows, true, t);
        cl_reduce_d<3>(t, tot, S, par, C);
        if (tid == 0) {
            K.rz = tot[0];
            K.rz_f = (float)K.rz;
            K.rr = tot[1];
            K.bb = tot[2];
            K.tol2 = a.tol * a.tol * K.bb;
            K.rr_last = K.rr;
            K.status = PC_OK;
            K.iter_last = 0;
            K.outer = 0;
            K.bad_pq = 0;
            int act = 0;
            if (!isfinite(K.bb) || !isfinite(K.rr)) {
                K.status = PC_ERR_NONFINITE;
                act = CL_ACT_DONE;
            } else if (K.rr <= K.tol2) {
                act = CL_ACT_DONE;
            } else if (a.max_iter <= 0) {
                K.status = PC_ERR_NOT_CONVERGED;
                act = CL_ACT_DONE;
            }
            S.bc->action = act;
        }
        __syncthreads();
    }
    int action = S.bc->action;
    float beta = 0.f;
    int cur = 0, iter = 0;

    while (!(action & CL_ACT_DONE)) {
        // q = A p, p = z + beta p_prev formed per gathered row; p.q
        float pqf = 0.f;
        const uint32_t poff = cur ? 16u : 0u;
        for (int l0 = 0; l0 < nrows; l0 += CL_GROUPS) {
            const int l = l0 + grp;
            const bool ok = l < nrows;
            float4 pl = make_float4(0.f, 0.f, 0.f, 0.f);
            float a0 = 0.f, a1 = 0.f, a2 = 0.f;
            if (ok) {
                pl = cl_dir(beta, S.rec[l].p[cur], S.rec[l].z);
                const int k1 = S.rs[l + 1];
                for (int k = S.rs[l] + sub; k < k1; k += CL_TPR) {
                    const uint32_t ad = S.addr[k];
                    float4 d = cl_dir(beta, cl_ld_f4(ad + poff), cl_ld_f4(ad + CL_REC_Z));
                    if (DIFF) {
                        d.x -= pl.x;
                        d.y -= pl.y;
                        d.z -= pl.z;
                    }
                    const float *B = S.vals + 9 * k;
                    a0 = fmaf(B[2], d.z, fmaf(B[1], d.y, fmaf(B[0], d.x, a0)));
                    a1 = fmaf(B[5], d.z, fmaf(B[4], d.y, fmaf(B[3], d.x, a1)));
                    a2 = fmaf(B[8], d.z, fmaf(B[7], d.y, fmaf(B[6], d.x, a2)));
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
                    a0 = fmaf(D[2], pl.z, fmaf(D[1], pl.y, fmaf(D[0], pl.x, a0)));
                    a1 = fmaf(D[5], pl.z, fmaf(D[4], pl.y, fmaf(D[3], pl.x, a1)));
                    a2 = fmaf(D[8], pl.z, fmaf(D[7], pl.y, fmaf(D[6], pl.x, a2)));
                }
                const float4 q = make_float4(a0, a1, a2, 0.f);
                S.rec[l].p[cur ^ 1] = pl;
                S.qv[l] = q;
                pqf += cl_dot3(pl, q);
            }
        }
        {
            const float v[1] = {pqf};
            float2 tot[1];
            cl_reduce_df<1>(v, tot, S, par, C);
            if (tid == 0) {
                // the quotient in FP32, the precision the update uses it in
                const float pq = __fadd_rn(tot[0].x, tot[0].y);
                float alpha = K.rz_f / pq;
                K.bad_pq = !(pq > 0.f) || !isfinite(alpha);
                if (K.bad_pq) alpha = 0.f;
                S.bc->alpha = alpha;
            }
            __syncthreads();
        }
        const float alpha = S.bc->alpha;

        // x += alpha p, r -= alpha q, z = D^-1 r; r.z, r.r
        float rzf = 0.f, rrf = 0.f;
        for (int l = tid; l < nrows; l += CL_THREADS) {
            const float4 p = S.rec[l].p[cur ^ 1], q = S.qv[l];
            float4 x = S.xv[l], r = S.rv[l];
            x.x = fmaf(alpha, p.x, x.x);
            x.y = fmaf(alpha, p.y, x.y);
            x.z = fmaf(alpha, p.z, x.z);
            r.x = fmaf(-alpha, q.x, r.x);
            r.y = fmaf(-alpha, q.y, r.y);
            r.z = fmaf(-alpha, q.z, r.z);
            const float4 z = cl_precond<BLOCK>(S.dinv, l, r);
            S.xv[l] = x;
            S.rv[l] = r;
            S.rec[l].z = z;
            rzf += cl_dot3(r, z);
            rrf += cl_dot3(r, r);
        }
        {
            const float v[2] = {rzf, rrf};
            float2 tot[2];
            cl_reduce_df<2>(v, tot, S, par, C);
            if (tid == 0) {
                const float rz_new = __fadd_rn(tot[0].x, tot[0].y);
                const float beta_d = rz_new / K.rz_f;
                K.rz_f = rz_new;
                K.rz = pc_df_value(tot[0].x, tot[0].y);
                K.rr = pc_df_value(tot[1].x, tot[1].y);
                const double rr = K.rr;
                const int it = iter + 1;
                int act = 0;
                bool conv = false;
                if (K.bad_pq || !isfinite(rr) || !isfinite(beta_d)) {
                    K.status = PC_ERR_NONFINITE;
                    act = CL_ACT_DONE;
                } else if (rr <= K.tol2) {
                    conv = true;
                } else if (it >= a.max_iter) {
                    K.status = PC_ERR_NOT_CONVERGED;
                    act = CL_ACT_DONE;
                }
                if (!act) {
                    if (!a.mixed) {
                        act = conv ? CL_ACT_DONE : 0;
                    } else if (conv) {
                        // a converged recurrence residual is confirmed by an FP64 replacement
                        act = (rr > 0.0 && it > K.iter_last) ? CL_ACT_REPLACE : CL_ACT_DONE;
                    } else if (it % a.check_every == 0) {
                        act = CL_ACT_FOLD;
                        if (rr <= K.rr_last * a.refresh * a.refresh || it - K.iter_last >= a.refresh_every)
                            act |= CL_ACT_REPLACE;
                    }
                }
                S.bc->beta = beta_d;
                S.bc->action = act;
            }
            __syncthreads();
        }
        beta = S.bc->beta;
        action = S.bc->action;
        cur ^= 1;
        ++iter;
        if (action & (CL_ACT_FOLD | CL_ACT_REPLACE)) cl_fold(S, nrows);
        if (action & CL_ACT_REPLACE) {
            cl_sync();  // every CTA's folded iterate before any CTA gathers it
            double t[3], tot[3];
            cl_residual<DIFF, BLOCK>(S, a, row0, nrows, true, t);
            cl_reduce_d<3>(t, tot, S, par, C);
            if (tid == 0) {
                K.rz = tot[0];
                K.rz_f = (float)K.rz;
                K.rr = tot[1];
                K.rr_last = K.rr;
                K.iter_last = iter;
                ++K.outer;
                int act = 0;
                if (!isfinite(K.rr)) {
                    K.status = PC_ERR_NONFINITE;
                    act = CL_ACT_DONE;
                } else if (K.rr <= K.tol2) {
                    act = CL_ACT_DONE;
                } else if (iter >= a.max_iter) {
                    K.status = PC_ERR_NOT_CONVERGED;
                    act = CL_ACT_DONE;
                }
                S.bc->action = act;
            }
            __syncthreads();
            action = S.bc->action;
        }
    }

    // 4. the solution, and its FP64 residual unless the last replacement measured it
    if (tid == 0) S.bc->check = a.mixed ? (iter > K.iter_last ? 1 : 0) : 1;
    __syncthreads();
    const bool check = S.bc->check != 0;
    if (a.mixed) {
        if (check) cl_fold(S, nrows);
        for (int l = tid; l < nrows; l += CL_THREADS) {
            const int64_t row = row0 + l;
            for (int e = 0; e < 3; ++e) {
                const double x = S.rec[l].x[e];
                const float d = (float)x;
                a.dv[3 * row + e] = d;
                if (a.x64) a.x64[3 * row + e] = x;
                if (check) S.rec[l].x[e] = (double)d;
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
            S.rec[l].x[0] = (double)d0;
            S.rec[l].x[1] = (double)d1;
            S.rec[l].x[2] = (double)d2;
        }
    }
    if (check) {
        cl_sync();
        double t[3], tot[3];
        cl_residual<DIFF, BLOCK>(S, a, row0, nrows, false, t);
        cl_reduce_d<3>(t, tot, S, par, C);
        if (tid == 0) {
            K.rr = tot[1];
            K.bb = tot[2];
        }
    }
    cl_sync();
    if (rank == 0 && tid == 0) {
        pc_scalars *sc = a.sc;
        sc->rz = K.rz;
        sc->rr = K.rr;
        sc->bb = K.bb;
        sc->tol2 = K.tol2;
        sc->alpha = 0.0;
        sc->beta = (double)beta;
        sc->pq = 0.0;
        sc->iter = iter;
        sc->max_iter = a.max_iter;
        sc->status = K.status;
        sc->done = 1;
        sc->outer = K.outer;
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

// Shared-memory layout for V rows over C CTAs; false when the rows do not fit.
static bool cl_layout(int V, int C, bool diff, bool block, size_t smax, int64_t stored, ClArgs *a, size_t *smem)
{
    const int Rc = (V + C - 1) / C;
    if (Rc < 1 || Rc > CL_THREADS) return false;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += (bytes + 15) & ~(size_t)15;
        return (uint32_t)at;
    };
    take(sizeof(ClRec) * Rc);
    a->o_x = take(16ull * Rc);
    a->o_r = take(16ull * Rc);
    a->o_q = take(16ull * Rc);
    a->o_dres = take(diff ? 36ull * Rc : 0);
    a->o_dinv = take((block ? 48ull : 16ull) * Rc);
    a->o_rs = take(4ull * (Rc + 1));
    a->o_red = take(8ull * (4 * CL_WARPS + 8) + 4ull * 40 + sizeof(ClCtl) + sizeof(ClBcast));
    if (o >= smax) return false;
    const int64_t cap = (int64_t)((smax - o) / 40) & ~(int64_t)3;
    // the average CTA's blocks must fit (the kernel checks every CTA's exactly)
    if (cap < 4 || (stored + C - 1) / C > cap) return false;
    a->o_addr = (uint32_t)o;
    a->o_vals = (uint32_t)(o + 4 * cap);
    a->Rc = Rc;
    a->cap = (int)cap;
    *smem = o + 40 * (size_t)cap;
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
