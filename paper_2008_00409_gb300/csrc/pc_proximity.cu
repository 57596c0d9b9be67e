// Proximity query feeding the one-sided thickness contact model: every (vertex p,
// triangle t) pair whose distance at the current positions is below the contact
// thickness delta, t touching neither p nor a mesh-edge neighbour of p, with the
// barycentric weights of the point of t closest to p. It is the proximity step in front
// of the implicit integrator (Sec. 2.5, Eq. 3); the paper's own collision handling
// (spatial hashing, continuous collision detection, Sec. 4) is not reproduced.
//
// Uniform grid, rebuilt per call: the cell size is the largest triangle bounding box
// grown by delta (so every grown box covers at most 2 x 2 x 2 cells); each triangle is
// listed under every cell its grown box overlaps (key = packed cell coordinates), the
// list is put in key order by the stable radix sort (triangles of a cell stay in index
// order), and each vertex tests the triangles listed under its own cell: a vertex within
// delta of a triangle lies in that triangle's grown box, hence in one of its cells. Two
// passes over the vertices (count, scan, write) give the pairs ordered by vertex, then
// by triangle, without atomics.
//
// The region of the closest point (Voronoi classification of a point against a
// triangle, Ericson 2005, Sec. 5.1.5) and the test d^2 < delta^2 are decided in FP32
// with one rounding per operation in a fixed order (the _rn intrinsics keep the compiler
// from contracting into fused multiply-adds), so the pairs are reproducible bit for bit.
#include <cstring>

#include "pc_internal.cuh"

#define PX_CELLS_PER_TRI 8
#define PX_COORD_BIAS (1 << 20)  // cell coordinates must lie in [-2^20, 2^20)

__device__ __forceinline__ float3 px_ld(const float *x, int i)
{
    return make_float3(x[3ll * i], x[3ll * i + 1], x[3ll * i + 2]);
}
__device__ __forceinline__ float3 px_sub(float3 a, float3 b)
{
    return make_float3(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z));
}
__device__ __forceinline__ float px_dot(float3 u, float3 v)
{
    return __fadd_rn(__fadd_rn(__fmul_rn(u.x, v.x), __fmul_rn(u.y, v.y)), __fmul_rn(u.z, v.z));
}

// Weights (wa, wb, wc) of the point of (a, b, c) closest to p; returns the squared
// distance. Regions in priority order: vertex a, vertex b, edge ab, vertex c, edge ac,
// edge bc, a degenerate triangle (treated as vertex a), the face.
__device__ float px_closest(float3 p, float3 a, float3 b, float3 c, float &wa, float &wb, float &wc)
{
    const float3 ab = px_sub(b, a), ac = px_sub(c, a), ap = px_sub(p, a);
    const float d1 = px_dot(ab, ap), d2 = px_dot(ac, ap);
    const float3 bp = px_sub(p, b);
    const float d3 = px_dot(ab, bp), d4 = px_dot(ac, bp);
    const float3 cp = px_sub(p, c);
    const float d5 = px_dot(ab, cp), d6 = px_dot(ac, cp);
    const float vc = __fsub_rn(__fmul_rn(d1, d4), __fmul_rn(d3, d2));
    const float vb = __fsub_rn(__fmul_rn(d5, d2), __fmul_rn(d1, d6));
    const float va = __fsub_rn(__fmul_rn(d3, d6), __fmul_rn(d5, d4));
    const float e43 = __fsub_rn(d4, d3), e56 = __fsub_rn(d5, d6);
    const float s = __fadd_rn(__fadd_rn(va, vb), vc);
    if (d1 <= 0.f && d2 <= 0.f) { wb = 0.f; wc = 0.f; }
    else if (d3 >= 0.f && d4 <= d3) { wb = 1.f; wc = 0.f; }
    else if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) { wb = __fdiv_rn(d1, __fsub_rn(d1, d3)); wc = 0.f; }
    else if (d6 >= 0.f && d5 <= d6) { wb = 0.f; wc = 1.f; }
    else if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) { wb = 0.f; wc = __fdiv_rn(d2, __fsub_rn(d2, d6)); }
    else if (va <= 0.f && e43 >= 0.f && e56 >= 0.f) {
        const float t = __fdiv_rn(e43, __fadd_rn(e43, e56));
        wb = __fsub_rn(1.f, t);
        wc = t;
    } else if (!(s > 0.f)) { wb = 0.f; wc = 0.f; }
    else { wb = __fdiv_rn(vb, s); wc = __fdiv_rn(vc, s); }
    wa = __fsub_rn(__fsub_rn(1.f, wb), wc);
    const float3 q = make_float3(__fadd_rn(__fadd_rn(a.x, __fmul_rn(ab.x, wb)), __fmul_rn(ac.x, wc)),
                                 __fadd_rn(__fadd_rn(a.y, __fmul_rn(ab.y, wb)), __fmul_rn(ac.y, wc)),
                                 __fadd_rn(__fadd_rn(a.z, __fmul_rn(ab.z, wb)), __fmul_rn(ac.z, wc)));
    const float3 r = px_sub(p, q);
    return px_dot(r, r);
}

// Grown bounding box of triangle t.
__device__ __forceinline__ void px_box(const float *x, const int32_t *tri, int t, float pad, float3 &lo, float3 &hi)
{
    const float3 a = px_ld(x, tri[3ll * t]), b = px_ld(x, tri[3ll * t + 1]), c = px_ld(x, tri[3ll * t + 2]);
    lo = make_float3(fminf(fminf(a.x, b.x), c.x) - pad, fminf(fminf(a.y, b.y), c.y) - pad,
                     fminf(fminf(a.z, b.z), c.z) - pad);
    hi = make_float3(fmaxf(fmaxf(a.x, b.x), c.x) + pad, fmaxf(fmaxf(a.y, b.y), c.y) + pad,
                     fmaxf(fmaxf(a.z, b.z), c.z) + pad);
}

// Cell coordinate along one axis; false when outside the packable range.
__device__ __forceinline__ bool px_cell(float v, float inv, int &i)
{
    const float f = floorf(v * inv);
    if (!(f >= -(float)PX_COORD_BIAS && f < (float)PX_COORD_BIAS)) return false;
    i = (int)f;
    return true;
}
__device__ __forceinline__ uint64_t px_key(int ix, int iy, int iz)
{
    return ((uint64_t)(ix + PX_COORD_BIAS) << 42) | ((uint64_t)(iy + PX_COORD_BIAS) << 21) |
           (uint64_t)(iz + PX_COORD_BIAS);
}

// Largest edge of the grown boxes (non-negative floats order like their bit patterns).
__global__ void px_extent_kernel(int T, const float *x, const int32_t *tri, float pad, uint32_t *max_bits)
{
    float m = 0.f;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        float3 lo, hi;
        px_box(x, tri, t, pad, lo, hi);
        m = fmaxf(m, fmaxf(fmaxf(hi.x - lo.x, hi.y - lo.y), hi.z - lo.z));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(max_bits, __float_as_uint(m));
}

// Cells per triangle (0 and an error bit when a box leaves the grid).
__global__ void px_count_cells_kernel(int T, const float *x, const int32_t *tri, float pad, float inv,
                                      int32_t *cnt, uint32_t *err)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > T) return;
    if (t == T) {
        cnt[T] = 0;
        return;
    }
    float3 lo, hi;
    px_box(x, tri, t, pad, lo, hi);
    int i0, i1, j0, j1, k0, k1;
    if (!(px_cell(lo.x, inv, i0) && px_cell(hi.x, inv, i1) && px_cell(lo.y, inv, j0) && px_cell(hi.y, inv, j1) &&
          px_cell(lo.z, inv, k0) && px_cell(hi.z, inv, k1))) {
        cnt[t] = 0;
        pc_set_err(err, PC_DERR_INDEX);
        return;
    }
    cnt[t] = (i1 - i0 + 1) * (j1 - j0 + 1) * (k1 - k0 + 1);
}

__global__ void px_emit_cells_kernel(int T, const float *x, const int32_t *tri, float pad, float inv,
                                     const int32_t *off, int64_t cap, uint64_t *keys, uint32_t *vals)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    float3 lo, hi;
    px_box(x, tri, t, pad, lo, hi);
    int i0, i1, j0, j1, k0, k1;
    if (!(px_cell(lo.x, inv, i0) && px_cell(hi.x, inv, i1) && px_cell(lo.y, inv, j0) && px_cell(hi.y, inv, j1) &&
          px_cell(lo.z, inv, k0) && px_cell(hi.z, inv, k1)))
        return;
    int64_t o = off[t];
    for (int k = k0; k <= k1; ++k)
        for (int j = j0; j <= j1; ++j)
            for (int i = i0; i <= i1; ++i) {
                if (o < cap) {
                    keys[o] = px_key(i, j, k);
                    vals[o] = (uint32_t)t;
                }
                ++o;
            }
}

// true when v is among ecol[lo .. hi) (sorted)
__device__ __forceinline__ bool px_ring_has(const int32_t *ecol, int lo, int hi, int v)
{
    const int end = hi;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ecol[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo < end && ecol[lo] == v;
}

// One thread per vertex: the triangles listed under its cell. COUNT: cnt[p] = pairs of p;
// WRITE: the pairs at off[p] ...
template <bool WRITE>
__global__ void px_pairs_kernel(int V, const float *x, const int32_t *tri, const uint64_t *keys, const uint32_t *vals,
                                int64_t K, float inv, float delta, const int32_t *erp, const int32_t *ecol,
                                int32_t *cnt, const int32_t *off, int32_t *pairs, float *w, uint32_t *err)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > V) return;
    if (p == V) {
        if (!WRITE) cnt[V] = 0;
        return;
    }
    const float3 xp = px_ld(x, p);
    int ix, iy, iz;
    if (!(px_cell(xp.x, inv, ix) && px_cell(xp.y, inv, iy) && px_cell(xp.z, inv, iz))) {
        if (!WRITE) cnt[p] = 0;
        pc_set_err(err, PC_DERR_INDEX);
        return;
    }
    const uint64_t key = px_key(ix, iy, iz);
    int64_t lo = 0, hi = K;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    const float d2max = __fmul_rn(delta, delta);
    const int r0 = erp[p], r1 = erp[p + 1];
    int n = 0;
    const int64_t o0 = WRITE ? off[p] : 0;
    for (int64_t i = lo; i < K && keys[i] == key; ++i) {
        const int t = (int)vals[i];
        const int a = tri[3ll * t], b = tri[3ll * t + 1], c = tri[3ll * t + 2];
        if (a == p || b == p || c == p) continue;
        if (px_ring_has(ecol, r0, r1, a) || px_ring_has(ecol, r0, r1, b) || px_ring_has(ecol, r0, r1, c)) continue;
        float wa, wb, wc;
        const float d2 = px_closest(xp, px_ld(x, a), px_ld(x, b), px_ld(x, c), wa, wb, wc);
        if (!(d2 < d2max)) continue;
        if (WRITE) {
            const int64_t o = o0 + n;
            pairs[4 * o] = p;
            pairs[4 * o + 1] = a;
            pairs[4 * o + 2] = b;
            pairs[4 * o + 3] = c;
            w[3 * o] = wa;
            w[3 * o + 1] = wb;
            w[3 * o + 2] = wc;
        }
        ++n;
    }
    if (!WRITE) cnt[p] = n;
}

extern "C" pc_status pc_proximity_query(pc_ctx *ctx, const float *x, float delta, int32_t cap, int32_t *pairs,
                                        float *w, int32_t *n_out, void *stream)
{
    if (!ctx || !x || !n_out || cap < 0 || (cap > 0 && (!pairs || !w))) return PC_ERR_ARG;
    if (!(delta > 0.f) || !(delta < 1e30f)) return PC_ERR_ARG;
    *n_out = 0;
    cudaStream_t st = (cudaStream_t)stream;
    const int V = ctx->V, T = ctx->T;
    if (T == 0) return PC_OK;
    if (!ctx->px_keys) return PC_ERR_ARG;
    const float pad = delta * 1.01f;
    // cell size: the largest grown box (at least delta)
    PC_CUDA_TRY(cudaMemsetAsync(ctx->px_max, 0, sizeof(uint32_t), st));
    const unsigned ext_grid = pc_blocks(T, 256) < (unsigned)(ctx->num_sms * 8) ? pc_blocks(T, 256) : ctx->num_sms * 8;
    PC_LAUNCH(ctx, px_extent_kernel, ext_grid, 256, 0, st, T, x, ctx->tri, pad, ctx->px_max);
    PC_CUDA_TRY(cudaMemcpyAsync(ctx->h_count, ctx->px_max, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    uint32_t bits_ext = *reinterpret_cast<uint32_t *>(ctx->h_count);
    float cs;
    memcpy(&cs, &bits_ext, sizeof(float));
    if (!(cs < 1e30f)) return PC_ERR_NONFINITE;
    cs = fmaxf(cs, delta) * 1.001f;
    const int64_t cap_k = ctx->px_cap;
    int64_t K = 0;
    for (int attempt = 0;; ++attempt) {
        const float inv = 1.0f / cs;
        PC_CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), st));
        PC_LAUNCH(ctx, px_count_cells_kernel, pc_blocks(T + 1ll, 256), 256, 0, st, T, x, ctx->tri, pad, inv,
                  ctx->px_cnt, ctx->d_err);
        PC_TRY(pc_exclusive_scan(ctx, ctx->px_cnt, ctx->px_off, T, st));
        PC_CUDA_TRY(cudaMemcpyAsync(ctx->h_count, ctx->px_off + T, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        uint32_t bits = 0;
        PC_TRY(pc_read_errors(ctx, st, &bits));
        if (bits) return PC_ERR_ARG;  // positions too far out for the cell grid
        K = *reinterpret_cast<int32_t *>(ctx->h_count);
        if (K <= cap_k) {
            PC_LAUNCH(ctx, px_emit_cells_kernel, pc_blocks(T, 256), 256, 0, st, T, x, ctx->tri, pad, inv,
                      ctx->px_off, cap_k, ctx->px_keys, ctx->px_vals);
            PC_TRY(pc_radix_sort(ctx, ctx->px_keys, ctx->px_vals, K, 63, st));
            break;
        }
        if (attempt >= 4) return PC_ERR_CAPACITY;
        cs *= 2.0f;  // rounding put some boxes across three cells: coarser grid
    }
    const float inv = 1.0f / cs;
    PC_LAUNCH(ctx, px_pairs_kernel<false>, pc_blocks(V + 1ll, 128), 128, 0, st, V, x, ctx->tri, ctx->px_keys,
              ctx->px_vals, K, inv, delta, ctx->erp, ctx->ecol, ctx->px_vcnt, nullptr, nullptr, nullptr, ctx->d_err);
    PC_TRY(pc_exclusive_scan(ctx, ctx->px_vcnt, ctx->px_voff, V, st));
    PC_CUDA_TRY(cudaMemcpyAsync(ctx->h_count, ctx->px_voff + V, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    uint32_t bits = 0;
    PC_TRY(pc_read_errors(ctx, st, &bits));
    if (bits) return PC_ERR_ARG;
    const int32_t P = *reinterpret_cast<int32_t *>(ctx->h_count);
    *n_out = P;
    if (P > cap) return PC_ERR_CAPACITY;
    if (P > 0)
        PC_LAUNCH(ctx, px_pairs_kernel<true>, pc_blocks(V + 1ll, 128), 128, 0, st, V, x, ctx->tri, ctx->px_keys,
                  ctx->px_vals, K, inv, delta, ctx->erp, ctx->ecol, nullptr, ctx->px_voff, pairs, w, ctx->d_err);
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    return PC_OK;
}

// Query buffers (called at context creation): 8 cell entries per triangle, per-triangle
// and per-vertex counts and offsets.
pc_status pc_proximity_alloc(pc_ctx *c)
{
    c->px_cap = (int64_t)PX_CELLS_PER_TRI * c->T + 1;
    PC_CUDA_TRY(cudaMalloc(&c->px_keys, sizeof(uint64_t) * (size_t)c->px_cap));
    PC_CUDA_TRY(cudaMalloc(&c->px_vals, sizeof(uint32_t) * (size_t)c->px_cap));
    PC_CUDA_TRY(cudaMalloc(&c->px_cnt, sizeof(int32_t) * (c->T + 1ll)));
    PC_CUDA_TRY(cudaMalloc(&c->px_off, sizeof(int32_t) * (c->T + 1ll)));
    PC_CUDA_TRY(cudaMalloc(&c->px_vcnt, sizeof(int32_t) * (c->V + 1ll)));
    PC_CUDA_TRY(cudaMalloc(&c->px_voff, sizeof(int32_t) * (c->V + 1ll)));
    PC_CUDA_TRY(cudaMalloc(&c->px_max, sizeof(uint32_t)));
    return PC_OK;
}
