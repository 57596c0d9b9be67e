// Batched solve: many independent garments stored as one block-diagonal system (the
// union of their meshes), each solved to its own relative residual by ONE persistent
// PCG launch (cooperative, all CTAs co-resident), and a batched time step that captures
// value assembly, the solve and the state update in a CUDA graph.
//
// Instances own contiguous row ranges [inst_rows[k], inst_rows[k+1]) of at least 32 rows.
// Every phase walks a work list of the instances still iterating (rebuilt by each CTA in
// shared memory when an instance finishes), one entry per (instance, 32-row tile), split
// into equal contiguous chunks, one per CTA; finished instances cost nothing. A CTA meets
// each instance in one run of its chunk and delivers one partial sum per instance; the
// CTA that delivers last sums the instance's slots in CTA order (deterministic) and sets
// the instance's scalars, so no separate scalar phase is needed. Phases are separated by
// a software grid barrier whose waits are bounded; a timeout aborts the launch with
// PC_ERR_TIMEOUT instead of hanging. Per iteration (three grid barriers):
//   direction  p = z + beta_k p                   (fold x into x64 after a refresh, and
//                                                  every 32 iterations)
//   spmv       q = A p, p.q -> alpha_k            (the bulk-copy pipelined SpMV)
//   update     x += alpha p, r -= alpha q, z = D^-1 r, r.z, r.r -> beta_k, stop tests
// and, when some instance asks for it, FP64 residual replacement for those instances
// (r = b - A (x64 + x) in FP64, new scalars).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pc_internal.cuh"

#define RED_SLOTS 4
#define BT_TILE 32  // rows per tile in every phase

__device__ __forceinline__ double bt_warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
#include "pc_spmv.cuh"

// ------------------------------------------------------------------------- device state

#define BT_MAX_INST 1024

struct bt_inst {
    double rz, rr, bb, tol2, alpha, beta, pq, rr_last;
    int32_t iter, iter_last, done, status;
    int32_t refresh;  // FP64 residual requested (set by the update phase, cleared by the next SpMV phase)
    int32_t arrive;   // CTAs that delivered their partial sums in the current phase
    int32_t pad0, pad1;
};

struct bt_global {
    unsigned long long bar; // grid barrier arrivals (pc_grid_barrier; bit 63 set on abort)
    uint32_t abort;         // set on timeout (read by the host and the state update)
    uint32_t gen;           // bumped whenever an instance finishes
    uint32_t n_refresh[2];  // refresh requests, by iteration parity
    uint32_t pad[2];
};

struct BtArgs {
    int V, n_inst;
    const int32_t *rp, *ci;
    const float *vals, *dres, *b;
    // the SpMV phase's matrix: a copy without diagonal blocks (difference form) or A itself,
    // and per row the scalar difference diagonal (s when dres_i = s I, else -1; or null)
    const int32_t *srp, *sci;
    const float *svals, *dsc;
    const int32_t *inst_rows;  // [n_inst + 1]
    float4 *p4;                // gathered by the product: one 16-byte load per row
    float *q3, *r3, *z3, *x3;  // only streamed: three floats per row (12 bytes, not 16)
    const float *dinv3;
    double *x64;
    float *dv;
    double *part;              // [(ntiles + n_inst) * 3] partial sums, one slot per (CTA, instance)
    double *part_pq;           // [(ntiles + n_inst) * SP_CWARPS] p.q per (CTA's run, consumer warp)
    bt_inst *inst;
    bt_global *g;
    uint32_t *err;
    double tol, refresh;
    int max_iter, refresh_every;
    int spmv_chunked;          // SpMV entry order: 0 strided, 1 contiguous chunks (autotuned)
    long long bar_wait;        // cycles a grid-barrier wait may take before the launch aborts
};

// Rows of the streamed vectors (three floats each).
__device__ __forceinline__ float4 bt_ld3(const float *v, int64_t row)
{
    const float *q = v + 3 * row;
    return make_float4(q[0], q[1], q[2], 0.f);
}
__device__ __forceinline__ float4 bt_ldcg3(const float *v, int64_t row)
{
    const float *q = v + 3 * row;
    return make_float4(__ldcg(q), __ldcg(q + 1), __ldcg(q + 2), 0.f);
}
__device__ __forceinline__ void bt_st3(float *v, int64_t row, float4 x)
{
    float *q = v + 3 * row;
    q[0] = x.x;
    q[1] = x.y;
    q[2] = x.z;
}

// The work list of one phase: the listed instances in order, each contributing one entry
// per 32-row tile it touches (a tile shared by two instances gives one entry to each, and
// an entry covers only its own instance's rows). Entries are split into equal contiguous
// chunks, one per CTA, so a CTA meets each instance in one run of entries and delivers
// one partial sum per instance it touches.
struct bt_list {
    int n;      // listed instances
    int total;  // entries
    int chunk;  // entries per CTA
    int pref[BT_MAX_INST + 1];
    short id[BT_MAX_INST];
};

enum { BT_LIST_ACTIVE = 0, BT_LIST_REFRESH = 1, BT_LIST_ALL = 2 };

__device__ __forceinline__ int bt_tiles_of(int r0, int r1) { return (r1 - 1) / BT_TILE - r0 / BT_TILE + 1; }

// Built by every CTA from the instance flags (all threads call; ends with a barrier).
__device__ void bt_build_list(const BtArgs &a, int mode, bt_list &L)
{
    __shared__ int s_w[2][8];
    const int n = a.n_inst, T = blockDim.x;
    const int per = (n + T - 1) / T;
    const int k0 = min(n, (int)threadIdx.x * per), k1 = min(n, k0 + per);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
    int cnt = 0, ent = 0;
    for (int k = k0; k < k1; ++k) {
        const bt_inst &I = a.inst[k];
        const bool on = mode == BT_LIST_ALL ? true
                      : mode == BT_LIST_ACTIVE ? __ldcg(&I.done) == 0
                                               : (__ldcg(&I.refresh) != 0 && __ldcg(&I.done) == 0);
        if (on) {
            ++cnt;
            ent += bt_tiles_of(a.inst_rows[k], a.inst_rows[k + 1]);
        }
    }
    // block-wide exclusive scan of (cnt, ent)
    int ic = cnt, ie = ent;
    for (int o = 1; o < 32; o <<= 1) {
        const int uc = __shfl_up_sync(0xffffffffu, ic, o), ue = __shfl_up_sync(0xffffffffu, ie, o);
        if (lane >= o) { ic += uc; ie += ue; }
    }
    if (lane == 31) { s_w[0][warp] = ic; s_w[1][warp] = ie; }
    __syncthreads();
    int bc = 0, be = 0, tc = 0, te = 0;
    for (int w = 0; w < nw; ++w) {
        if (w < warp) { bc += s_w[0][w]; be += s_w[1][w]; }
        tc += s_w[0][w];
        te += s_w[1][w];
    }
    int pos = bc + ic - cnt, e = be + ie - ent;
    for (int k = k0; k < k1; ++k) {
        const bt_inst &I = a.inst[k];
        const bool on = mode == BT_LIST_ALL ? true
                      : mode == BT_LIST_ACTIVE ? __ldcg(&I.done) == 0
                                               : (__ldcg(&I.refresh) != 0 && __ldcg(&I.done) == 0);
        if (on) {
            L.id[pos] = (short)k;
            L.pref[pos] = e;
            ++pos;
            e += bt_tiles_of(a.inst_rows[k], a.inst_rows[k + 1]);
        }
    }
    if (threadIdx.x == 0) {
        L.n = tc;
        L.total = te;
        L.pref[tc] = te;
        L.chunk = (te + gridDim.x - 1) / gridDim.x;
    }
    __syncthreads();
}

// list position holding entry j (largest m with pref[m] <= j)
__device__ __forceinline__ int bt_find(const bt_list &L, int j)
{
    int lo = 0, hi = L.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.pref[mid] <= j) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One run of entries of this CTA's chunk: list position m, entries [j, je), rows [ra, rb).
struct bt_seg {
    int m, k, j, je, ra, rb;
};

__device__ __forceinline__ void bt_seg_at(const BtArgs &a, const bt_list &L, int m, int j, int jend, bt_seg &s)
{
    s.m = m;
    s.k = L.id[m];
    s.j = j;
    s.je = min(jend, L.pref[m + 1]);
    const int r0 = a.inst_rows[s.k], r1 = a.inst_rows[s.k + 1];
    const int tb = r0 / BT_TILE;
    s.ra = max(r0, (tb + (s.j - L.pref[m])) * BT_TILE);
    s.rb = min(r1, (tb + (s.je - 1 - L.pref[m]) + 1) * BT_TILE);
}

// ------------------------------------------------------------------------- grid barrier

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Marks the launch aborted: the host and the state update read `abort`; every CTA leaves
// at its next grid barrier.
__device__ __forceinline__ void bt_abort(bt_global *g)
{
    atomicExch(&g->abort, 1u);
    pc_grid_abort(&g->bar);
}

// All CTAs of the (co-resident) grid meet; returns false everywhere once any CTA gave
// up waiting or the launch was aborted (the launch then unwinds without further waits).
__device__ bool bt_grid_sync(bt_global *g, long long budget)
{
    const bool ok = pc_grid_barrier(&g->bar, budget);
    if (!ok && threadIdx.x == 0) atomicExch(&g->abort, 1u);
    return ok;
}

// ------------------------------------------------------------------------- per-instance sums

// Barrier over the threads taking part: the whole CTA, or only the SpMV consumer warps
// (named barrier 1; the producer warp never joins it).
__device__ __forceinline__ void bt_group_bar(bool consumers)
{
    if (consumers) asm volatile("bar.sync 1, %0;" ::"r"(SP_CWARPS * 32) : "memory");
    else __syncthreads();
}

// Sum NQ values over the group's threads; the result is valid in thread 0.
template <int NQ>
__device__ void bt_group_sum(double (&v)[NQ], bool consumers)
{
    __shared__ double s[NQ][SP_CWARPS + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = consumers ? SP_CWARPS : (int)(blockDim.x >> 5);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const double w = bt_warp_sum(v[q]);
        if (lane == 0) s[q][warp] = w;
    }
    bt_group_bar(consumers);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += s[q][w];
            v[q] = t;
        }
    }
    bt_group_bar(consumers);
}

// Deliver this CTA's partial sums for the instance at list position m into the slot of
// the CTA's first entry of that instance (CTA b takes entries [b*chunk, (b+1)*chunk), so
// the instance's slots are max(b*chunk, p0) for the CTAs b whose chunk meets [p0, p1)).
// The CTA that delivers last sums the slots in CTA order (deterministic) and returns
// true with the totals in thread 0.
template <int NQ>
__device__ bool bt_deliver(const BtArgs &a, const bt_list &L, const bt_seg &sg, double (&v)[NQ], bool consumers)
{
    __shared__ int s_last;
    bt_group_sum<NQ>(v, consumers);
    const int c = L.chunk;
    const int p0 = L.pref[sg.m], p1 = L.pref[sg.m + 1];
    const int blo = p0 / c, bhi = (p1 - 1) / c;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) a.part[3ll * sg.j + q] = v[q];
        __threadfence();
        const int old = atomicAdd(&a.inst[sg.k].arrive, 1);
        const bool last = old == bhi - blo;
        if (last) {
            a.inst[sg.k].arrive = 0;
            __threadfence();
        }
        s_last = last ? 1 : 0;
    }
    bt_group_bar(consumers);
    if (!s_last) return false;
    const int nthr = consumers ? SP_CWARPS * 32 : (int)blockDim.x;
    double w[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) w[q] = 0.0;
    for (int bb = blo + (int)threadIdx.x; bb <= bhi; bb += nthr) {
        const int64_t slot = max(bb * c, p0);
#pragma unroll
        for (int q = 0; q < NQ; ++q) w[q] += __ldcg(a.part + 3 * slot + q);
    }
    bt_group_sum<NQ>(w, consumers);
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = w[q];
    return true;
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// ------------------------------------------------------------------------- phases

#ifndef BT_U
#define BT_U 2  // rows per thread in flight in the direction phase
#endif
#ifndef BT_MIN_CTAS
#define BT_MIN_CTAS 5  // register budget: five co-resident CTAs per SM (72 registers, no spills)
#endif
#define BT_WIN 3  // gathers in flight per thread in the product phase (12 blocks per row per round)

// Direction p = z + beta p over the listed rows; rows of an instance that has just
// taken an FP64 residual, or has done another 32 iterations, also fold the FP32
// increment into the FP64 accumulator.
__device__ void bt_phase_direction(const BtArgs &a, const bt_list &L)
{
    const int c = L.chunk, j0 = blockIdx.x * c, j1 = min(L.total, j0 + c);
    if (j0 >= j1) return;
    const int T = blockDim.x;
    for (int m = bt_find(L, j0), j = j0; j < j1; ++m) {
        bt_seg sg;
        bt_seg_at(a, L, m, j, j1, sg);
        j = sg.je;
        const float beta = (float)__ldcg(&a.inst[sg.k].beta);
        // fold after an FP64 residual, and every 32 iterations so the FP32 increment (and
        // its rounding, which the stiff matrix amplifies) never grows large
        const int it_k = __ldcg(&a.inst[sg.k].iter);
        const bool fold = __ldcg(&a.inst[sg.k].refresh) != 0 || (it_k > 0 && (it_k & 31) == 0);
        for (int base = sg.ra + (int)threadIdx.x; base < sg.rb; base += BT_U * T) {
            float4 z[BT_U], p[BT_U];
#pragma unroll
            for (int u = 0; u < BT_U; ++u) {
                const int row = base + u * T;
                if (row < sg.rb) {
                    z[u] = bt_ld3(a.z3, row);
                    p[u] = a.p4[row];
                }
            }
#pragma unroll
            for (int u = 0; u < BT_U; ++u) {
                const int row = base + u * T;
                if (row < sg.rb)
                    a.p4[row] = make_float4(fmaf(beta, p[u].x, z[u].x), fmaf(beta, p[u].y, z[u].y),
                                            fmaf(beta, p[u].z, z[u].z), 0.f);
            }
            if (fold) {
#pragma unroll
                for (int u = 0; u < BT_U; ++u) {
                    const int row = base + u * T;
                    if (row < sg.rb) {
                        const float4 d = bt_ld3(a.x3, row);
                        a.x64[3ll * row] += (double)d.x;
                        a.x64[3ll * row + 1] += (double)d.y;
                        a.x64[3ll * row + 2] += (double)d.z;
                        bt_st3(a.x3, row, make_float4(0.f, 0.f, 0.f, 0.f));
                    }
                }
            }
        }
    }
}

// Row bounds of a consumer thread's row, loaded one entry ahead.
struct BtRow {
    int row, rb, re;
    bool on;
};

__device__ __forceinline__ void bt_load_row(const BtArgs &a, int tile, int ra, int rb, int t, BtRow &r)
{
    r.row = tile * BT_TILE + t / SP_TPR;
    r.on = r.row >= ra && r.row < rb;
    r.rb = r.re = 0;
    if (r.on) {
        r.rb = a.srp[r.row];
        r.re = a.srp[r.row + 1];
    }
}

// Entry e of this CTA's chunk, walked in order by the producer and by the consumers.
struct bt_cursor {
    int m, k, p0, p1, r0, r1, tb;
};

__device__ __forceinline__ void bt_cursor_load(const BtArgs &a, const bt_list &L, int m, bt_cursor &cu)
{
    cu.m = m;
    cu.k = L.id[m];
    cu.p0 = L.pref[m];
    cu.p1 = L.pref[m + 1];
    cu.r0 = a.inst_rows[cu.k];
    cu.r1 = a.inst_rows[cu.k + 1];
    cu.tb = cu.r0 / BT_TILE;
}

// Entries this CTA takes in the SpMV phase: first entry, step and count. Strided order:
// b, b+G, b+2G, ... (all CTAs on one band of rows at a time); chunked order: the CTA's
// contiguous chunk. Either way a CTA meets each instance in one run of its entries.
struct bt_sched {
    int j0, step, n;
};

__device__ __forceinline__ bt_sched bt_spmv_sched(const BtArgs &a, const bt_list &L)
{
    bt_sched s;
    if (a.spmv_chunked) {
        s.j0 = (int)blockIdx.x * L.chunk;
        s.step = 1;
        s.n = max(0, min(L.total, s.j0 + L.chunk) - s.j0);
    } else {
        s.j0 = blockIdx.x;
        s.step = gridDim.x;
        s.n = (int)blockIdx.x < L.total ? (L.total - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    }
    return s;
}

// q = A p over the listed rows with the bulk-copy stage ring, entries in the order the
// autotuner chose (bt_spmv_sched). A CTA meets each instance in one run of its entries
// (an instance's entries are contiguous); each consumer warp stores its p.q over the run
// in the CTA's slot of the instance, and the slots are summed where alpha is needed
// (bt_alpha_warp). The instance's slots are contiguous from its first entry p0, one per
// CTA: strided order, the run's first entry p0 + ((b - p0) mod G), so slots p0 .. p0 +
// min(G, p1 - p0) - 1; chunked order, p0 + b - p0 / chunk for the CTAs b whose chunk meets
// [p0, p1). Contiguous slots keep the sum that every CTA of the instance makes one
// coalesced read (late in a solve one instance spans hundreds of CTAs). `kbase` continues
// the mbarrier phase count across calls.
template <bool DIFF, int CAPR>
__device__ void bt_phase_spmv(const BtArgs &a, const bt_list &L, unsigned char *smem_raw, uint64_t *full_bar,
                              uint64_t *empty_bar, int (*stage_info)[4], int kbase, int par)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bt_sched sched = bt_spmv_sched(a, L);
    const int G = sched.step, j0 = sched.j0;
    const int nent = sched.n;
    // the refresh counter of the previous iteration has been read by every CTA
    if (blockIdx.x == 0 && threadIdx.x == 0) a.g->n_refresh[par ^ 1] = 0u;
    bool timed_out = false;
    if (warp == SP_CWARPS) {
        if (lane == 0 && nent > 0) {
            bt_cursor cu;
            bt_cursor_load(a, L, bt_find(L, j0), cu);
            int issued = 0;
            for (int e = 0; e < nent; ++e) {
                const int j = j0 + e * G;
                if (j >= cu.p1) bt_cursor_load(a, L, bt_find(L, j), cu);
                const int tile = cu.tb + (j - cu.p0);
                const int ra = max(cu.r0, tile * BT_TILE), rb = min(cu.r1, tile * BT_TILE + BT_TILE);
                const int kg = kbase + e;
                const int s = kg % SP_STAGES;
                const uint32_t ph = (uint32_t)(kg / SP_STAGES) & 1u;
                if (kg >= SP_STAGES && !mbar_wait_bounded(&empty_bar[s], ph ^ 1u, SP_WAIT_BUDGET)) {
                    timed_out = true;
                    break;
                }
                const int b0 = a.srp[ra], b1 = a.srp[rb];
                unsigned char *base = smem_raw + s * SpShape<CAPR>::stage_bytes;
                if (b1 - b0 <= SpShape<CAPR>::cap) {
                    const int64_t f0 = 9ll * b0, al0 = f0 & ~3ll, al1 = (9ll * b1 + 3) & ~3ll;
                    const int c0 = b0 & ~3, c1 = (b1 + 3) & ~3;
                    const uint32_t vbytes = (uint32_t)((al1 - al0) * 4), cbytes = (uint32_t)((c1 - c0) * 4);
                    stage_info[s][0] = b0;
                    stage_info[s][1] = (int)(f0 - al0);
                    stage_info[s][2] = b0 - c0;
                    stage_info[s][3] = 1;
                    mbar_arrive_expect_tx(&full_bar[s], vbytes + cbytes);
                    bulk_g2s(base, a.svals + al0, vbytes, &full_bar[s]);
                    bulk_g2s(base + SpShape<CAPR>::val_bytes, a.sci + c0, cbytes, &full_bar[s]);
                } else {
                    stage_info[s][0] = b0;
                    stage_info[s][1] = 0;
                    stage_info[s][2] = 0;
                    stage_info[s][3] = 0;
                    mbar_arrive(&full_bar[s]);
                }
                ++issued;
            }
            // drain: the copies of the last stages issued must have landed before the phase ends
            for (int e = issued - 1; e >= 0 && e >= issued - SP_STAGES; --e) {
                const int kg = kbase + e;
                if (!mbar_wait_bounded(&full_bar[kg % SP_STAGES], (uint32_t)(kg / SP_STAGES) & 1u, SP_WAIT_BUDGET))
                    timed_out = true;
            }
        }
        __syncwarp();  // the producer warp reconverges before any block-wide barrier
    } else if (nent > 0) {
        const int t = threadIdx.x;
        const int jl = t & (SP_TPR - 1);
        bt_cursor cu;
        bt_cursor_load(a, L, bt_find(L, j0), cu);
        int seg_start = j0;
        float dot = 0.f, dot_c = 0.f;
        BtRow nxt;
        {
            const int tile = cu.tb + (j0 - cu.p0);
            bt_load_row(a, tile, max(cu.r0, tile * BT_TILE), min(cu.r1, tile * BT_TILE + BT_TILE), t, nxt);
        }
        for (int e = 0; e < nent; ++e) {
            const int j = j0 + e * G;
            const BtRow cur = nxt;
            // prefetch the next entry's rows (it may belong to the next instance)
            if (e + 1 < nent) {
                const int jn = j + G;
                int tb2 = cu.tb, p02 = cu.p0, r02 = cu.r0, r12 = cu.r1;
                if (jn >= cu.p1) {
                    const int m2 = bt_find(L, jn);
                    const int k2 = L.id[m2];
                    p02 = L.pref[m2];
                    r02 = a.inst_rows[k2];
                    r12 = a.inst_rows[k2 + 1];
                    tb2 = r02 / BT_TILE;
                }
                const int tile2 = tb2 + (jn - p02);
                bt_load_row(a, tile2, max(r02, tile2 * BT_TILE), min(r12, tile2 * BT_TILE + BT_TILE), t, nxt);
            }
            // the row's own p and the scalar of its difference-form diagonal (D = s I for all
            // but a few rows): in flight while the stage lands; a row without the scalar
            // reads its 3x3 diagonal after the gathers (holding nine floats across the loop
            // would cost the registers of the fifth CTA per SM)
            float4 xj = make_float4(0.f, 0.f, 0.f, 0.f);
            float sd = 0.f;
            if (cur.on) {
                xj = a.p4[cur.row];
                if (DIFF && jl == 0) sd = a.dsc ? a.dsc[cur.row] : -1.f;
            }
            const int kg = kbase + e;
            const int s = kg % SP_STAGES;
            const uint32_t ph = (uint32_t)(kg / SP_STAGES) & 1u;
            // after a timeout the warp stops waiting but keeps the barrier sequence
            const bool ok = timed_out ? false : mbar_wait_bounded(&full_bar[s], ph, SP_WAIT_BUDGET);
            if (!__all_sync(0xffffffffu, ok)) {
                timed_out = true;
            } else {
                const int b0 = stage_info[s][0], vo = stage_info[s][1], co = stage_info[s][2];
                const bool staged = stage_info[s][3] != 0;
                const float *s_vals = reinterpret_cast<const float *>(smem_raw + s * SpShape<CAPR>::stage_bytes) + vo;
                const int32_t *s_cols =
                    reinterpret_cast<const int32_t *>(smem_raw + s * SpShape<CAPR>::stage_bytes +
                                                      SpShape<CAPR>::val_bytes) + co;
                float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f;
                // up to BT_WIN blocks per thread in flight (rows average about 12 off-diagonal
                // blocks: one round for most); p is not written in this phase, so the gathers
                // may hit L1 (the grid barrier's acquire orders them after the direction
                // phase's writes)
                for (int bb = cur.rb + jl; bb < cur.re; bb += BT_WIN * SP_TPR) {
                    float4 u[BT_WIN];
#pragma unroll
                    for (int w = 0; w < BT_WIN; ++w) {
                        const int bw = bb + w * SP_TPR;
                        if (bw < cur.re) u[w] = a.p4[staged ? s_cols[bw - b0] : a.sci[bw]];
                    }
#pragma unroll
                    for (int w = 0; w < BT_WIN; ++w) {
                        const int bw = bb + w * SP_TPR;
                        if (bw < cur.re) {
                            const float *B = staged ? s_vals + 9 * (bw - b0) : a.svals + 9ll * bw;
                            float4 uw = u[w];
                            if (DIFF) { uw.x -= xj.x; uw.y -= xj.y; uw.z -= xj.z; }
                            spmv_fma(B, uw, acc0, acc1, acc2);
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
                if (cur.on && jl == 0) {
                    if (DIFF) {
                        if (sd > 0.f) {
                            acc0 = fmaf(sd, xj.x, acc0);
                            acc1 = fmaf(sd, xj.y, acc1);
                            acc2 = fmaf(sd, xj.z, acc2);
                        } else {
                            spmv_fma(a.dres + 9ll * cur.row, xj, acc0, acc1, acc2);
                        }
                    }
                    bt_st3(a.q3, cur.row, make_float4(acc0, acc1, acc2, 0.f));
                    kahan_add(dot, dot_c, fmaf(xj.x, acc0, fmaf(xj.y, acc1, xj.z * acc2)));
                }
            }
            // end of this instance's run: the warp's p.q goes to the run's slot
            if (j + G >= cu.p1 || e + 1 == nent) {
                const double w = bt_warp_sum((double)dot - (double)dot_c);
                // the instance's slots are contiguous from p0, one per CTA holding a run of
                // it: strided order, the run's first entry; chunked, p0 + b - p0 / chunk
                const int64_t slot = a.spmv_chunked ? cu.p0 + ((int)blockIdx.x - cu.p0 / L.chunk) : seg_start;
                if (lane == 0) a.part_pq[(int64_t)SP_CWARPS * slot + warp] = w;
                dot = 0.f;
                dot_c = 0.f;
                seg_start = j + G;
                if (e + 1 < nent) bt_cursor_load(a, L, bt_find(L, j + G), cu);
            }
        }
    }
    if (timed_out) {
        bt_abort(a.g);
        atomicOr(a.err, PC_DERR_TIMEOUT);
    }
}

#define BT_WARPS (SP_THREADS / 32)  // warps per CTA: instances a CTA's update phase handles at once
#define BT_SLOT_BATCH 4             // slot loads per lane issued together in the per-warp sums

// alpha of the instance at list position m, computed by one warp from the instance's p.q
// slots (summed in slot order, so every CTA that needs it gets the same value); the CTA
// holding the instance's first entry records it. Returns alpha in every lane.
__device__ float bt_alpha_warp(const BtArgs &a, const bt_list &L, int m, int j)
{
    const int lane = threadIdx.x & 31;
    const int k = L.id[m], p0 = L.pref[m], p1 = L.pref[m + 1];
    static_assert(SP_CWARPS == 4, "a p.q slot is four doubles (two double2)");
    bt_inst &I = a.inst[k];
    const double rz = lane == 0 ? __ldcg(&I.rz) : 0.0;  // in flight with the slot loads
    const int c = L.chunk;
    const int n = a.spmv_chunked ? (p1 - 1) / c - p0 / c + 1 : min((int)gridDim.x, p1 - p0);
    const double2 *slots = reinterpret_cast<const double2 *>(a.part_pq);
    // lane l adds slots l, l + 32, l + 64, ... in that order; the loads of BT_SLOT_BATCH
    // slots are issued before their adds (a garment late in a solve has a slot in
    // hundreds of CTAs, and one L2 round trip per slot would dominate the phase)
    double acc = 0.0;
    for (int i0 = lane; i0 < n; i0 += 32 * BT_SLOT_BATCH) {
        double v[BT_SLOT_BATCH];
#pragma unroll
        for (int u = 0; u < BT_SLOT_BATCH; ++u) {
            const int i = i0 + 32 * u;
            v[u] = 0.0;
            if (i < n) {
                const int64_t s0 = 2 * (int64_t)(p0 + i);
                const double2 x0 = __ldcg(slots + s0), x1 = __ldcg(slots + s0 + 1);
                v[u] = (x0.x + x0.y) + (x1.x + x1.y);
            }
        }
#pragma unroll
        for (int u = 0; u < BT_SLOT_BATCH; ++u)
            if (i0 + 32 * u < n) acc += v[u];
    }
    const double pq = bt_warp_sum(acc);
    float alpha32 = 0.f;
    if (lane == 0) {
        double alpha = rz / pq;
        const bool bad = !(pq > 0.0) || !isfinite(alpha);
        if (bad) alpha = 0.0;
        if (j == p0) {  // the instance's first entry is in this CTA's chunk
            I.refresh = 0;  // the direction phase has folded the increment
            I.pq = pq;
            I.alpha = alpha;
            if (bad) {
                I.status = PC_ERR_NONFINITE;
                I.done = 1;
                atomicAdd(&a.g->gen, 1u);
            }
        }
        alpha32 = (float)alpha;
    }
    return __shfl_sync(0xffffffffu, alpha32, 0);
}

// x += alpha p; r -= alpha q; z = D^-1 r; (r.z, r.r) per instance. The CTA completing an
// instance's sums sets beta and decides: go on, refresh with an FP64 residual, or stop.
// A CTA whose chunk meets several instances takes them BT_WARPS at a time: warp w finds the
// alpha of the group's instance w, all threads update the rows of the group, and warp w
// delivers instance w's sums, so the scalar steps (L2 round trips and FP64 arithmetic) of
// the instances overlap instead of adding up.
__device__ void bt_phase_update(const BtArgs &a, const bt_list &L, int par)
{
    __shared__ float s_alpha[BT_WARPS];
    __shared__ int s_row[BT_WARPS][2];
    __shared__ double s_part[BT_WARPS][BT_WARPS][2];
    const int c = L.chunk, j0 = blockIdx.x * c, j1 = min(L.total, j0 + c);
    if (j0 >= j1) return;
    const int T = blockDim.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int m0 = bt_find(L, j0), nseg = bt_find(L, j1 - 1) - m0 + 1;
    for (int g0 = 0; g0 < nseg; g0 += BT_WARPS) {
        const int gs = min(BT_WARPS, nseg - g0);
        if (warp < gs) {
            const int m = m0 + g0 + warp;
            bt_seg sg;
            bt_seg_at(a, L, m, max(j0, L.pref[m]), j1, sg);
            const float alpha = bt_alpha_warp(a, L, m, sg.j);
            if (lane == 0) {
                s_alpha[warp] = alpha;
                s_row[warp][0] = sg.ra;
                s_row[warp][1] = sg.rb;
            }
        }
        __syncthreads();
        for (int q = 0; q < gs; ++q) {
            const float alpha = s_alpha[q];
            const int rb = s_row[q][1];
            float rz = 0.f, rz_c = 0.f, rr = 0.f, rr_c = 0.f;
            // one row per thread at a time: two rows' vectors in flight would not fit the
            // persistent kernel's register budget (five CTAs per SM), which spills in every
            // phase once exceeded; prefetching them through shared memory was slower
            for (int row = s_row[q][0] + (int)threadIdx.x; row < rb; row += T) {
                const float4 p = a.p4[row], qv = bt_ld3(a.q3, row), d = bt_ld3(a.dinv3, row);
                float4 x = bt_ld3(a.x3, row), r = bt_ld3(a.r3, row);
                x.x = fmaf(alpha, p.x, x.x); x.y = fmaf(alpha, p.y, x.y); x.z = fmaf(alpha, p.z, x.z);
                r.x = fmaf(-alpha, qv.x, r.x); r.y = fmaf(-alpha, qv.y, r.y); r.z = fmaf(-alpha, qv.z, r.z);
                const float4 z = make_float4(d.x * r.x, d.y * r.y, d.z * r.z, 0.f);
                bt_st3(a.x3, row, x);
                bt_st3(a.r3, row, r);
                bt_st3(a.z3, row, z);
                kahan_add(rz, rz_c, fmaf(r.x, z.x, fmaf(r.y, z.y, r.z * z.z)));
                kahan_add(rr, rr_c, fmaf(r.x, r.x, fmaf(r.y, r.y, r.z * r.z)));
            }
            const double w0 = bt_warp_sum((double)rz - (double)rz_c), w1 = bt_warp_sum((double)rr - (double)rr_c);
            if (lane == 0) {
                s_part[q][warp][0] = w0;
                s_part[q][warp][1] = w1;
            }
        }
        __syncthreads();
        if (warp < gs) {
            // deliver into the CTA's slot of the instance, p0 + b - p0 / chunk (CTA b takes
            // entries [b*chunk, (b+1)*chunk)); the CTA that delivers last sums the slots in
            // CTA order and sets the instance's scalars
            const int m = m0 + g0 + warp;
            const int k = L.id[m], p0 = L.pref[m], p1 = L.pref[m + 1];
            const int blo = p0 / c, bhi = (p1 - 1) / c;
            const int64_t jm = p0 + ((int)blockIdx.x - blo);  // slots p0 .. p0 + bhi - blo
            int last = 0;
            if (lane == 0) {
                double v0 = 0.0, v1 = 0.0;
                for (int w = 0; w < T / 32; ++w) {
                    v0 += s_part[warp][w][0];
                    v1 += s_part[warp][w][1];
                }
                a.part[3ll * jm] = v0;
                a.part[3ll * jm + 1] = v1;
                __threadfence();
                const int old = atomicAdd(&a.inst[k].arrive, 1);
                last = old == bhi - blo;
                if (last) {
                    a.inst[k].arrive = 0;
                    __threadfence();
                }
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                double v0 = 0.0, v1 = 0.0;
                for (int b0 = blo + lane; b0 <= bhi; b0 += 32 * BT_SLOT_BATCH) {
                    double w0[BT_SLOT_BATCH], w1[BT_SLOT_BATCH];
#pragma unroll
                    for (int u = 0; u < BT_SLOT_BATCH; ++u) {
                        const int bb = b0 + 32 * u;
                        w0[u] = w1[u] = 0.0;
                        if (bb <= bhi) {
                            const int64_t slot = p0 + (bb - blo);
                            w0[u] = __ldcg(a.part + 3 * slot);
                            w1[u] = __ldcg(a.part + 3 * slot + 1);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < BT_SLOT_BATCH; ++u)
                        if (b0 + 32 * u <= bhi) {
                            v0 += w0[u];
                            v1 += w1[u];
                        }
                }
                const double rzn = bt_warp_sum(v0), rrn = bt_warp_sum(v1);
                bt_inst &I = a.inst[k];
                if (lane == 0 && !I.done) {
                    I.beta = rzn / I.rz;
                    I.rz = rzn;
                    I.rr = rrn;
                    I.iter += 1;
                    if (!isfinite(rrn) || !isfinite(I.beta)) {
                        I.status = PC_ERR_NONFINITE;
                        I.done = 1;
                        atomicAdd(&a.g->gen, 1u);
                    } else if (rrn <= I.tol2 || rrn <= I.rr_last * a.refresh * a.refresh ||
                               I.iter - I.iter_last >= a.refresh_every) {
                        I.refresh = 1;  // confirm or refresh with an FP64 residual
                        atomicAdd(&a.g->n_refresh[par], 1u);
                    } else if (I.iter >= a.max_iter) {
                        I.status = PC_ERR_NOT_CONVERGED;
                        I.done = 1;
                        atomicAdd(&a.g->gen, 1u);
                    }
                }
            }
        }
        __syncthreads();  // the group's shared arrays are reused by the next group
    }
}

// r = b - A (x64 + x) in FP64 over the listed rows; z = D^-1 r; p = 0 when starting;
// (r.z, r.r, b.b) per instance. The CTA completing an instance's sums sets its scalars
// (start) or takes the refresh result (convergence confirmed, or go on).
template <bool DIFF>
__device__ void bt_phase_residual(const BtArgs &a, const bt_list &L, bool start)
{
    const int c = L.chunk, j0 = blockIdx.x * c, j1 = min(L.total, j0 + c);
    if (j0 >= j1) return;
    const int T = blockDim.x;
    for (int m = bt_find(L, j0), j = j0; j < j1; ++m) {
        bt_seg sg;
        bt_seg_at(a, L, m, j, j1, sg);
        j = sg.je;
        double rz = 0.0, rr = 0.0, bb = 0.0;
        for (int row = sg.ra + (int)threadIdx.x; row < sg.rb; row += T) {
            const float4 xo = bt_ldcg3(a.x3, row);
            const double xj[3] = {__ldcg(a.x64 + 3ll * row) + (double)xo.x, __ldcg(a.x64 + 3ll * row + 1) + (double)xo.y,
                                  __ldcg(a.x64 + 3ll * row + 2) + (double)xo.z};
            double acc[3] = {0.0, 0.0, 0.0};
            for (int kk = a.rp[row]; kk < a.rp[row + 1]; ++kk) {
                const int col = a.ci[kk];
                if (DIFF && col == row) continue;
                const float *B = a.vals + 9ll * kk;
                const float4 xc4 = bt_ldcg3(a.x3, col);
                double xc[3] = {__ldcg(a.x64 + 3ll * col) + (double)xc4.x, __ldcg(a.x64 + 3ll * col + 1) + (double)xc4.y,
                                __ldcg(a.x64 + 3ll * col + 2) + (double)xc4.z};
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
                rr += rv * rv;
                bb += bv * bv;
                rf[q] = (float)rv;
            }
            const float4 d = bt_ld3(a.dinv3, row);
            const float4 r = make_float4(rf[0], rf[1], rf[2], 0.f);
            const float4 z = make_float4(d.x * r.x, d.y * r.y, d.z * r.z, 0.f);
            bt_st3(a.r3, row, r);
            bt_st3(a.z3, row, z);
            if (start) a.p4[row] = make_float4(0.f, 0.f, 0.f, 0.f);
            rz += (double)fmaf(r.x, z.x, fmaf(r.y, z.y, r.z * z.z));
        }
        double v[3] = {rz, rr, bb};
        if (bt_deliver<3>(a, L, sg, v, false) && threadIdx.x == 0) {
            bt_inst &I = a.inst[sg.k];
            const double rzn = v[0], rrn = v[1];
            if (start) {
                const double bbn = v[2];
                I.rz = rzn; I.rr = rrn; I.bb = bbn; I.tol2 = a.tol * a.tol * bbn;
                I.alpha = 0.0; I.beta = 0.0; I.pq = 0.0; I.rr_last = rrn;
                I.iter = 0; I.iter_last = 0; I.refresh = 0; I.status = PC_OK;
                I.done = (rrn <= I.tol2 || !isfinite(rrn)) ? 1 : 0;
                if (!isfinite(rrn)) I.status = PC_ERR_NONFINITE;
                if (!I.done && a.max_iter <= 0) { I.done = 1; I.status = PC_ERR_NOT_CONVERGED; }
            } else {
                I.rz = rzn;
                I.rr = rrn;
                I.rr_last = rrn;
                I.iter_last = I.iter;
                if (!isfinite(rrn)) { I.status = PC_ERR_NONFINITE; I.done = 1; }
                else if (rrn <= I.tol2) { I.status = PC_OK; I.done = 1; }
                else if (I.iter >= a.max_iter) { I.status = PC_ERR_NOT_CONVERGED; I.done = 1; }
                if (I.done) atomicAdd(&a.g->gen, 1u);
            }
        }
    }
}

// ------------------------------------------------------------------------- the persistent kernel

template <bool DIFF, int CAPR>
__global__ void __launch_bounds__(SP_THREADS, BT_MIN_CTAS) batched_pcg_kernel(BtArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t full_bar[SP_STAGES], empty_bar[SP_STAGES];
    __shared__ int stage_info[SP_STAGES][4];
    __shared__ bt_list L;
    __shared__ uint32_t s_gen, s_ref;
    if (threadIdx.x == 0) {
        for (int s = 0; s < SP_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], SP_CWARPS);
        }
        mbar_fence_init();
    }
    __syncthreads();
    int kbase = 0;  // entries this CTA has staged so far (mbarrier phase count)

    // ---- start: x64 = dv0 and x = 0 (set before launch); r = b - A x64, z, p = 0
    bt_build_list(a, BT_LIST_ALL, L);
    bt_phase_residual<DIFF>(a, L, true);
    if (!bt_grid_sync(a.g, a.bar_wait)) return;

    uint32_t my_gen = 0xffffffffu;
    bool stale = true;
    for (int it = 0;; ++it) {
        const int par = it & 1;
        if (threadIdx.x == 0) s_gen = ld_acquire_gpu(&a.g->gen);
        __syncthreads();
        if (stale || s_gen != my_gen) {
            bt_build_list(a, BT_LIST_ACTIVE, L);
            my_gen = s_gen;
            stale = false;
        }
        if (L.n == 0) break;

        bt_phase_direction(a, L);
        if (!bt_grid_sync(a.g, a.bar_wait)) return;
        bt_phase_spmv<DIFF, CAPR>(a, L, smem_raw, full_bar, empty_bar, stage_info, kbase, par);
        kbase += bt_spmv_sched(a, L).n;
        if (!bt_grid_sync(a.g, a.bar_wait)) return;
        bt_phase_update(a, L, par);
        if (!bt_grid_sync(a.g, a.bar_wait)) return;
        if (threadIdx.x == 0) s_ref = ld_acquire_gpu(&a.g->n_refresh[par]);
        __syncthreads();
        if (s_ref > 0) {
            bt_build_list(a, BT_LIST_REFRESH, L);
            stale = true;
            bt_phase_residual<DIFF>(a, L, false);
            if (!bt_grid_sync(a.g, a.bar_wait)) return;
        }
    }
    // ---- finish: dv = x64 + x (FP32)
    const int stride = gridDim.x * blockDim.x;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < a.V; row += stride) {
        const float4 d = bt_ldcg3(a.x3, row);
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

__global__ void bt_dinv_kernel(int V, const int32_t *rp, const int32_t *ci, const float *vals, float *dinv3,
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
    bt_st3(dinv3, r, ok ? make_float4(1.f / d0, 1.f / d1, 1.f / d2, 0.f) : make_float4(1.f, 1.f, 1.f, 0.f));
    if (!ok) pc_set_err(err, PC_DERR_NONFINITE);
}

__global__ void bt_start_kernel(int V, const float *dv, double *x64, float *x3)
{
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < V; row += gridDim.x * blockDim.x) {
        for (int q = 0; q < 3; ++q) {
            x64[3ll * row + q] = (double)dv[3ll * row + q];
            x3[3ll * row + q] = 0.f;
        }
    }
}

// v += dv, x += h v for the rows of every instance whose solve ended with PC_OK or
// PC_ERR_NOT_CONVERGED; an instance that failed keeps its state, and after an aborted
// launch no row moves.
__global__ void bt_state_update_kernel(int V, const int32_t *row_inst, const bt_inst *inst, const bt_global *g,
                                       float *x, float *v, const float *dv, float h)
{
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= V || g->abort != 0u) return;
    const int32_t st = inst[row_inst[row]].status;
    if (st != PC_OK && st != PC_ERR_NOT_CONVERGED) return;
    for (int q = 0; q < 3; ++q) {
        const int64_t i = 3ll * row + q;
        const float vi = v[i] + dv[i];
        v[i] = vi;
        x[i] = fmaf(h, vi, x[i]);
    }
}

// ------------------------------------------------------------------------- host side

#define BT_GRIDS 7  // grid candidates: 16, 32, 64 CTAs (below one per SM), then 2..5 per SM

struct pc_batched_state {
    int32_t *row_inst = nullptr;   // [V]
    double *part = nullptr;        // [(ntiles + max_inst) * 3]
    double *part_pq = nullptr;     // [(ntiles + max_inst) * SP_CWARPS]
    bt_inst *inst = nullptr;       // [max_inst]
    bt_global *g = nullptr;
    int32_t *inst_rows = nullptr;  // [max_inst + 1]
    int max_inst = 0;
    int blocks_per_sm = 0;         // autotuned launch shape: CTAs per SM, rounded up (0 = not tuned yet)
    int grid = 0;                  // autotuned launch shape: CTAs in the grid
    int spmv_order = 0;            // autotuned SpMV entry order: 0 strided, 1 chunked
    int capr = SP_CAP_PER_ROW;     // autotuned stage width of the SpMV phase (blocks per row)
    int64_t tuned_nnzb = -1;
    int tuned_inst = -1;
    int tune_grid[BT_GRIDS] = {};   // candidate grid sizes (CTAs; 0 = unused slot)
    float tune_ms[2][2][BT_GRIDS] = {};  // [stage width 14 / 18][order][grid] timings of the tuning runs
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream the step graph is captured on
};

static pc_batched_state *bt_state(pc_ctx *c);

static pc_status bt_prepare(pc_ctx *c, pc_batched_state **out)
{
    pc_batched_state *B = bt_state(c);
    if (!B) return PC_ERR_CUDA;
    *out = B;
    return PC_OK;
}

// The SpMV phase's stage widths the autotuner chooses between (blocks per row of a
// 32-row tile): the narrow one leaves more shared memory per SM, the wide one stages
// more tiles instead of reading them from global memory.
static int bt_capr(int i) { return i == 0 ? SP_CAP_PER_ROW : SP_CAPR_WIDE; }

static pc_status bt_launch(pc_ctx *c, pc_batched_state *B, const BtArgs &args, bool diff, int grid, int capr,
                           cudaStream_t st)
{
    const bool wide = capr > SP_CAP_PER_ROW;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(SP_THREADS);
    cfg.dynamicSmemBytes = wide ? SpShape<SP_CAPR_WIDE>::smem_bytes : SpShape<SP_CAP_PER_ROW>::smem_bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    PC_CUDA_TRY(cudaMemsetAsync(B->g, 0, sizeof(bt_global), st));
    PC_CUDA_TRY(cudaMemsetAsync(B->inst, 0, sizeof(bt_inst) * (size_t)args.n_inst, st));
    BtArgs a = args;
    if (diff && wide) PC_CUDA_TRY(cudaLaunchKernelEx(&cfg, batched_pcg_kernel<true, SP_CAPR_WIDE>, a));
    else if (diff) PC_CUDA_TRY(cudaLaunchKernelEx(&cfg, batched_pcg_kernel<true, SP_CAP_PER_ROW>, a));
    else if (wide) PC_CUDA_TRY(cudaLaunchKernelEx(&cfg, batched_pcg_kernel<false, SP_CAPR_WIDE>, a));
    else PC_CUDA_TRY(cudaLaunchKernelEx(&cfg, batched_pcg_kernel<false, SP_CAP_PER_ROW>, a));
    c->launches++;
    return PC_OK;
}

static int bt_max_blocks_per_sm(bool diff, int capr)
{
    int n = 0;
    const int wb = SpShape<SP_CAPR_WIDE>::smem_bytes, nb = SpShape<SP_CAP_PER_ROW>::smem_bytes;
    if (capr > SP_CAP_PER_ROW) {
        if (diff) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batched_pcg_kernel<true, SP_CAPR_WIDE>, SP_THREADS, wb);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batched_pcg_kernel<false, SP_CAPR_WIDE>, SP_THREADS, wb);
    } else {
        if (diff) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batched_pcg_kernel<true, SP_CAP_PER_ROW>, SP_THREADS, nb);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batched_pcg_kernel<false, SP_CAP_PER_ROW>, SP_THREADS, nb);
    }
    return n;
}

// Solve part shared by pc_pcg_solve_batched and pc_step_batched (stream-ordered, no
// host synchronisation, so it can be captured).
static pc_status bt_enqueue(pc_ctx *c, pc_batched_state *B, const pc_bsr *A, const float *vals, const float *dres,
                            const float *b, float *dv, int n_inst, const pc_solve_opts &o, int grid,
                            int spmv_order, int capr, cudaStream_t st)
{
    const int V = c->V;
    PC_LAUNCH(c, bt_dinv_kernel, pc_blocks(V, 256), 256, 0, st, V, A->row_ptr, A->col_idx, vals,
              c->dinv, c->d_err);
    PC_LAUNCH(c, bt_start_kernel, pc_blocks(V, 256), 256, 0, st, V, dv, c->x64, c->dtmp);
    BtArgs a{};
    a.V = V;
    a.n_inst = n_inst;
    a.rp = A->row_ptr;
    a.ci = A->col_idx;
    a.vals = vals;
    a.dres = dres;
    a.b = b;
    a.srp = A->row_ptr;
    a.sci = A->col_idx;
    a.svals = vals;
    a.dsc = nullptr;
    // difference form: the SpMV phase streams the matrix without its diagonal blocks
    // (they multiply p_i - p_i = 0) and reads one scalar per row for D_i = m_i I
    if (dres && pc_build_offdiag_async(c, A, vals, dres, st) == PC_OK) {
        a.srp = c->od_rp;
        a.sci = c->od_ci;
        a.svals = c->od_vals;
        a.dsc = c->dsc;
    }
    a.inst_rows = B->inst_rows;
    a.r3 = c->r;
    a.z3 = c->z;
    a.p4 = (float4 *)c->p0;
    a.q3 = c->q;
    a.x3 = c->dtmp;
    a.dinv3 = c->dinv;
    a.x64 = c->x64;
    a.dv = dv;
    a.part = B->part;
    a.part_pq = B->part_pq;
    a.inst = B->inst;
    a.g = B->g;
    a.err = c->d_err;
    a.tol = o.tol;
    a.refresh = o.refresh;
    a.max_iter = o.max_iter;
    a.refresh_every = o.refresh_every;
    a.spmv_chunked = spmv_order;
    a.bar_wait = c->bar_wait_cycles > 0 ? (long long)c->bar_wait_cycles : SP_WAIT_BUDGET;
    return bt_launch(c, B, a, dres != nullptr, grid, capr, st);
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
// budget) for each tile and schedule choice -- the SpMV phase's stage width (14 or 18
// blocks per row of a 32-row tile) x its entry order (strided or chunked) x the grid
// (16, 32 or 64 CTAs, where that is below one per SM: a small system's grid barriers are
// cheaper with fewer CTAs; then 2..5 co-resident CTAs per SM, as far as they fit) -- and
// keep the fastest.
static pc_status bt_autotune(pc_ctx *c, pc_batched_state *B, const pc_bsr *A, const float *vals, const float *dres,
                             const float *b, int n_inst, const pc_solve_opts &o, cudaStream_t st)
{
    if (B->grid > 0 && B->tuned_nnzb == A->nnzb && B->tuned_inst == n_inst) return PC_OK;
    pc_solve_opts t = o;
    t.max_iter = std::min(o.max_iter, 60);
    t.tol = 1e-30;  // run the whole budget
    float best = 1e30f;
    int best_b = 0, best_order = 0, best_capr = SP_CAP_PER_ROW;
    cudaEvent_t e0, e1;
    PC_CUDA_TRY(cudaEventCreate(&e0));
    PC_CUDA_TRY(cudaEventCreate(&e1));
    float *scratch_dv = c->rhs32;  // float[V][3], a zero guess
    for (int g = 0; g < BT_GRIDS; ++g) B->tune_grid[g] = 0;
    for (int g = 0; g < 3; ++g)
        if ((16 << g) < c->num_sms) B->tune_grid[g] = 16 << g;
    for (int w = 0; w < 2; ++w) {
        const int capr = bt_capr(w);
        const int maxb = std::min(5, bt_max_blocks_per_sm(dres != nullptr, capr));
        for (int order = 0; order < 2; ++order)
            for (int gi = 0; gi < BT_GRIDS; ++gi) {
                // 16, 32, 64 CTAs, then 2..5 per SM (one per SM never won: the small grids
                // serve the small systems, more CTAs the large ones)
                const int per = gi - 1;
                const int grid = gi < 3 ? B->tune_grid[gi] : (per <= maxb ? per * c->num_sms : 0);
                if (gi >= 3) B->tune_grid[gi] = per * c->num_sms;
                B->tune_ms[w][order][gi] = 0.f;
                if (grid <= 0 || maxb < 1) continue;
                PC_CUDA_TRY(cudaMemsetAsync(scratch_dv, 0, sizeof(float) * 3 * (size_t)c->V, st));
                PC_CUDA_TRY(cudaEventRecord(e0, st));
                pc_status s = bt_enqueue(c, B, A, vals, dres, b, scratch_dv, n_inst, t, grid, order, capr, st);
                PC_CUDA_TRY(cudaEventRecord(e1, st));
                if (s != PC_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return s; }
                PC_CUDA_TRY(cudaEventSynchronize(e1));
                uint32_t aborted = 0;
                PC_CUDA_TRY(cudaMemcpy(&aborted, &B->g->abort, sizeof(uint32_t), cudaMemcpyDeviceToHost));
                if (aborted) { cudaEventDestroy(e0); cudaEventDestroy(e1); return PC_ERR_TIMEOUT; }
                float ms = 0.f;
                PC_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                B->tune_ms[w][order][gi] = ms;
                if (ms < best) { best = ms; best_b = grid; best_order = order; best_capr = capr; }
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_b < 1) return PC_ERR_CUDA;  // no launch shape fits an SM
    B->grid = best_b;
    B->blocks_per_sm = (best_b + c->num_sms - 1) / c->num_sms;
    B->spmv_order = best_order;
    B->capr = best_capr;
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
    PC_TRY(bt_enqueue(ctx, B, A, vals, dres, b, dv, n_inst, o, B->grid, B->spmv_order, B->capr, st));
    return bt_collect(ctx, B, n_inst, info, st);
}

extern "C" pc_status pc_set_barrier_wait(pc_ctx *ctx, int64_t cycles)
{
    if (!ctx) return PC_ERR_ARG;
    ctx->bar_wait_cycles = cycles > 0 ? cycles : 0;
    return PC_OK;
}

extern "C" pc_status pc_batched_config(pc_ctx *ctx, int32_t *grid, int32_t *spmv_order, int32_t *stage_blocks,
                                       int32_t *grid_sizes /*[7]*/, float *tune_ms /*[28]*/)
{
    if (!ctx) return PC_ERR_ARG;
    pc_batched_state *B = bt_state(ctx);
    if (!B) return PC_ERR_CUDA;
    if (grid) *grid = B->grid;
    if (spmv_order) *spmv_order = B->spmv_order;
    if (stage_blocks) *stage_blocks = B->capr;
    if (grid_sizes)
        for (int g = 0; g < BT_GRIDS; ++g) grid_sizes[g] = B->tune_grid[g];
    if (tune_ms)
        for (int w = 0; w < 2; ++w)
            for (int order = 0; order < 2; ++order)
                for (int g = 0; g < BT_GRIDS; ++g) tune_ms[2 * BT_GRIDS * w + BT_GRIDS * order + g] = B->tune_ms[w][order][g];
    return PC_OK;
}

static pc_status bt_update_state(pc_ctx *c, pc_batched_state *B, float *x, float *v, float h, cudaStream_t st)
{
    PC_LAUNCH(c, bt_state_update_kernel, pc_blocks(c->V, 256), 256, 0, st, c->V, B->row_inst, B->inst, B->g, x, v,
              c->A_dv, h);
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
    if (B->grid == 0 || B->tuned_nnzb < 0) {
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
        s = bt_enqueue(ctx, B, &A, ctx->A_vals, ctx->A_dres, ctx->A_b, ctx->A_dv, n_inst, o, B->grid,
                       B->spmv_order, B->capr, cs);
    if (s == PC_OK) s = bt_update_state(ctx, B, x, v, opts->h, cs);
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
    PC_CUDA_TRY(cudaMalloc(&B->part, sizeof(double) * 3 * (size_t)(ntiles + BT_MAX_INST)));
    PC_CUDA_TRY(cudaMalloc(&B->part_pq, sizeof(double) * SP_CWARPS * (size_t)(ntiles + BT_MAX_INST)));
    PC_CUDA_TRY(cudaMalloc(&B->inst, sizeof(bt_inst) * BT_MAX_INST));
    PC_CUDA_TRY(cudaMalloc(&B->g, sizeof(bt_global)));
    PC_CUDA_TRY(cudaMalloc(&B->inst_rows, sizeof(int32_t) * (BT_MAX_INST + 1)));
    PC_CUDA_TRY(cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking));
    const int nbytes = SpShape<SP_CAP_PER_ROW>::smem_bytes, wbytes = SpShape<SP_CAPR_WIDE>::smem_bytes;
    PC_CUDA_TRY(cudaFuncSetAttribute(batched_pcg_kernel<true, SP_CAP_PER_ROW>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, nbytes));
    PC_CUDA_TRY(cudaFuncSetAttribute(batched_pcg_kernel<false, SP_CAP_PER_ROW>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, nbytes));
    PC_CUDA_TRY(cudaFuncSetAttribute(batched_pcg_kernel<true, SP_CAPR_WIDE>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, wbytes));
    PC_CUDA_TRY(cudaFuncSetAttribute(batched_pcg_kernel<false, SP_CAPR_WIDE>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, wbytes));
    return PC_OK;
}

void pc_batched_free(pc_ctx *c)
{
    pc_batched_state *B = bt_state(c);
    if (!B) return;
    if (B->graph_exec) cudaGraphExecDestroy(B->graph_exec);
    if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
    cudaFree(B->row_inst);
    cudaFree(B->part);
    cudaFree(B->part_pq);
    cudaFree(B->inst);
    cudaFree(B->g);
    cudaFree(B->inst_rows);
    delete B;
    c->batched = nullptr;
}
