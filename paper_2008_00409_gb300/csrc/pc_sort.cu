// Key sort and prefix scan used by pattern construction (Sec. 3.2.2 redesigned: the
// paper fills an index table with atomics and sorts each row; here every key is placed
// by a stable LSD radix sort whose ranks come from warp match/popc, so no atomics are
// involved and the output order is fully determined by the input).
#include "pc_internal.cuh"

#define RS_THREADS 256
#define RS_WARPS (RS_THREADS / 32)
#define RS_WARP_KEYS 512
#define RS_TILE (RS_WARPS * RS_WARP_KEYS)  // 4096 keys per tile

// Per-warp digit histograms of one tile, combined in warp order.
__device__ __forceinline__ void rs_warp_hist(const uint64_t *keys, int64_t n, int shift, int64_t base,
                                             uint32_t (*wh)[256], int warp, int lane)
{
    for (int r = 0; r < RS_WARP_KEYS / 32; ++r) {
        int64_t i = base + r * 32 + lane;
        unsigned d = (i < n) ? (unsigned)((keys[i] >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int leader = __ffs(peers) - 1;
        if (lane == leader && d < 256u) wh[warp][d] += __popc(peers);
        __syncwarp();
    }
}

__global__ void rs_hist_kernel(const uint64_t *keys, int64_t n, int shift, uint32_t *hist, int tiles)
{
    __shared__ uint32_t wh[RS_WARPS][256];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += blockDim.x) (&wh[0][0])[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * RS_WARP_KEYS;
    rs_warp_hist(keys, n, shift, base, wh, warp, lane);
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        uint32_t s = 0;
        for (int w = 0; w < RS_WARPS; ++w) s += wh[w][d];
        hist[(int64_t)d * tiles + blockIdx.x] = s;
    }
}

// offs = exclusive scan of hist (digit-major): offs[d * tiles + tile] is where the first
// key of digit d from this tile goes.
__global__ void rs_scatter_kernel(const uint64_t *keys, const uint32_t *vals, int64_t n, int shift,
                                  const int32_t *offs, int tiles, uint64_t *okeys, uint32_t *ovals)
{
    __shared__ uint32_t wh[RS_WARPS][256];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += blockDim.x) (&wh[0][0])[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * RS_WARP_KEYS;
    rs_warp_hist(keys, n, shift, base, wh, warp, lane);
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) {
        uint32_t b = (uint32_t)offs[(int64_t)d * tiles + blockIdx.x];
        for (int w = 0; w < RS_WARPS; ++w) {
            uint32_t c = wh[w][d];
            wh[w][d] = b;
            b += c;
        }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < RS_WARP_KEYS / 32; ++r) {
        int64_t i = base + r * 32 + lane;
        bool valid = i < n;
        uint64_t k = valid ? keys[i] : 0ull;
        unsigned d = valid ? (unsigned)((k >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t pos = 0;
        if (valid) pos = wh[warp][d] + __popc(peers & lt);
        __syncwarp();
        int leader = __ffs(peers) - 1;
        if (lane == leader && valid) wh[warp][d] += __popc(peers);
        __syncwarp();
        if (valid) {
            okeys[pos] = k;
            if (vals) ovals[pos] = vals[i];
        }
    }
}

// ------------------------------------------------------------------------- exclusive scan

#define SCAN_THREADS 256
#define SCAN_ITEMS 8
#define SCAN_TILE (SCAN_THREADS * SCAN_ITEMS)

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t *total)
{
    __shared__ int32_t warp_sums[SCAN_THREADS / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t s = lane < SCAN_THREADS / 32 ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SCAN_THREADS / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    int32_t before = warp > 0 ? warp_sums[warp - 1] : 0;
    *total = warp_sums[SCAN_THREADS / 32 - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void scan_tile_kernel(const int32_t *in, int32_t *out, int64_t n, int32_t *tile_sums)
{
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int32_t total;
    int32_t ex = block_exclusive_scan(s, &total);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// One block scans the tile sums in place (any count) and writes the grand total.
__global__ void scan_sums_kernel(int32_t *tile_sums, int64_t tiles, int32_t *grand_total)
{
    int64_t per = (tiles + SCAN_THREADS - 1) / SCAN_THREADS;
    int64_t b = (int64_t)threadIdx.x * per;
    int32_t s = 0;
    for (int64_t i = b; i < b + per && i < tiles; ++i) s += tile_sums[i];
    int32_t total;
    int32_t ex = block_exclusive_scan(s, &total);
    for (int64_t i = b; i < b + per && i < tiles; ++i) {
        int32_t t = tile_sums[i];
        tile_sums[i] = ex;
        ex += t;
    }
    if (threadIdx.x == 0) *grand_total = total;
}

__global__ void scan_add_kernel(int32_t *out, int64_t n, const int32_t *tile_sums)
{
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int32_t add = tile_sums[blockIdx.x];
    for (int k = threadIdx.x; k < SCAN_TILE; k += SCAN_THREADS) {
        int64_t i = base + k;
        if (i < n) out[i] += add;
    }
}

// out[0..n-1] = exclusive scan of in, out[n] = total. `in` and `out` may alias.
pc_status pc_exclusive_scan(pc_ctx *ctx, const int32_t *in, int32_t *out, int64_t n, cudaStream_t st)
{
    if (n <= 0) {
        PC_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int32_t), st));
        return PC_OK;
    }
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles > ctx->scan_tmp_cap) return PC_ERR_ARG;
    PC_LAUNCH(ctx, scan_tile_kernel, (unsigned)tiles, SCAN_THREADS, 0, st, in, out, n, ctx->scan_tmp);
    PC_LAUNCH(ctx, scan_sums_kernel, 1, SCAN_THREADS, 0, st, ctx->scan_tmp, tiles, out + n);
    PC_LAUNCH(ctx, scan_add_kernel, (unsigned)tiles, SCAN_THREADS, 0, st, out, n, ctx->scan_tmp);
    return PC_OK;
}

// Grow the sort scratch to hold n keys (called only at context creation).
pc_status pc_sort_reserve(pc_ctx *ctx, int64_t n)
{
    if (n < 1) n = 1;
    pc_sort_scratch &s = ctx->sort;
    if (n > s.cap) {
        cudaFree(s.keys_alt);
        cudaFree(s.vals_alt);
        s.keys_alt = nullptr;
        s.vals_alt = nullptr;
        PC_CUDA_TRY(cudaMalloc(&s.keys_alt, sizeof(uint64_t) * n));
        PC_CUDA_TRY(cudaMalloc(&s.vals_alt, sizeof(uint32_t) * n));
        s.cap = n;
    }
    int64_t tiles = (n + RS_TILE - 1) / RS_TILE;
    if (256 * tiles + 1 > s.hist_cap) {
        cudaFree(s.hist);
        s.hist = nullptr;
        PC_CUDA_TRY(cudaMalloc(&s.hist, sizeof(uint32_t) * (256 * tiles + 1)));
        s.hist_cap = 256 * tiles + 1;
    }
    int64_t scan_tiles = (256 * tiles + 1 + SCAN_TILE - 1) / SCAN_TILE + (n + SCAN_TILE) / SCAN_TILE + 1;
    if (scan_tiles > ctx->scan_tmp_cap) {
        cudaFree(ctx->scan_tmp);
        ctx->scan_tmp = nullptr;
        PC_CUDA_TRY(cudaMalloc(&ctx->scan_tmp, sizeof(int32_t) * scan_tiles));
        ctx->scan_tmp_cap = scan_tiles;
    }
    return PC_OK;
}

// Stable LSD radix sort of n keys (and optional values) on their low `bits` bits, in
// place. n must not exceed the reserved scratch and must be below 2^31.
pc_status pc_radix_sort(pc_ctx *ctx, uint64_t *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t st)
{
    if (n <= 1) return PC_OK;
    if (n > ctx->sort.cap || n >= (1ll << 31)) return PC_ERR_ARG;
    int tiles = (int)((n + RS_TILE - 1) / RS_TILE);
    uint64_t *k_in = keys, *k_out = ctx->sort.keys_alt;
    uint32_t *v_in = vals, *v_out = vals ? ctx->sort.vals_alt : nullptr;
    int32_t *offs = reinterpret_cast<int32_t *>(ctx->sort.hist);
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        PC_LAUNCH(ctx, rs_hist_kernel, tiles, RS_THREADS, 0, st, k_in, n, shift, ctx->sort.hist, tiles);
        PC_TRY(pc_exclusive_scan(ctx, offs, offs, (int64_t)256 * tiles, st));
        PC_LAUNCH(ctx, rs_scatter_kernel, tiles, RS_THREADS, 0, st, k_in, v_in, n, shift, offs, tiles, k_out, v_out);
        uint64_t *tk = k_in; k_in = k_out; k_out = tk;
        uint32_t *tv = v_in; v_in = v_out; v_out = tv;
    }
    if (k_in != keys) {
        PC_CUDA_TRY(cudaMemcpyAsync(keys, k_in, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st));
        if (vals) PC_CUDA_TRY(cudaMemcpyAsync(vals, v_in, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
    }
    return PC_OK;
}
