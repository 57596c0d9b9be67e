// Learned warm start: a per-vertex MLP (12 -> 64 -> 64 -> 3, ReLU) that predicts the
// initial guess of the Eq. 3 solve, its training (forward, back-propagation, Adam) and
// the step's initial guess combining the learned and previous-step guesses.
// The paper has no learned component; this is an extension built on its integrator.
//
// Features of vertex i (12): v_i, dv_prev_i, l_i (b_i / h - m_i g) / m_i (the internal
// force per unit mass at the first-order end-of-step position, from the assembled
// right-hand side b = h (f(x_t) - h K v_t) + h M g, times the vertex's mean rest edge
// length l_i), and the mean of dv_prev over the edge one-ring.
// Inputs and targets are standardised with training-set statistics; the network predicts
// the change dv - dv_prev, so the guess is dv0 = dv_prev + sd_y * y + mu_y (0 at pins).
//
// Every matrix product, in inference and in training, runs on the 5th-generation tensor
// cores (tcgen05.mma, BF16 operands in shared memory, FP32 accumulators in tensor memory).
// Training forms the weight gradients dW = dZ^T H as products over a tile's rows,
// accumulated in tensor memory; per-CTA partial gradients are summed in a fixed order
// (deterministic) by the kernel that applies Adam to the FP32 master weights.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <cmath>

#include "pc_internal.cuh"
#include "pc_tc.cuh"
#include "pc_tma.cuh"

#define MLP_IN 12
#define MLP_HID 64
#define MLP_OUT 3
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + MLP_HID * MLP_IN)
#define OFF_W2 (OFF_B1 + MLP_HID)
#define OFF_B2 (OFF_W2 + MLP_HID * MLP_HID)
#define OFF_W3 (OFF_B2 + MLP_HID)
#define OFF_B3 (OFF_W3 + MLP_OUT * MLP_HID)
static_assert(OFF_B3 + MLP_OUT == PC_MLP_NPARAMS, "parameter layout");
static_assert(2 * MLP_IN + 2 * MLP_OUT == PC_MLP_NSTATS, "statistics layout");


// ------------------------------------------------------------------------- tensor-core helpers

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (low half) = lo
    return *reinterpret_cast<uint32_t *>(&v);
}

// ------------------------------------------------------------------------- inference (tcgen05)

// One CTA of four warps per 128-row tile (persistent over tiles): the three layers are
// tcgen05 MMAs (M = 128, K = 16 per instruction, BF16 operands from shared memory, FP32
// accumulators in tensor memory), issued by one thread and committed to an mbarrier;
// warp w reads tensor-memory lanes 32w.. (its 32 rows), adds the bias, applies the ReLU
// and writes the BF16 activations back to shared memory as the next layer's A operand.
#define TC_ROWS 128
#define TC_THREADS 128
#define TC_TMEM_COLS 128  // D1 at column 0, D2 at 64, D3 at 0 again
#define TC_OFF_W1 0       // 64 x 16 BF16 (2 KB)
#define TC_OFF_W2 2048    // 64 x 64 (8 KB)
#define TC_OFF_W3 10240   // 16 x 64, outputs 3..15 zero (2 KB)
#define TC_OFF_X 12288    // 128 x 16 (4 KB)
#define TC_OFF_H 16384    // 128 x 64 (16 KB)
// padded so that at most two CTAs share an SM: their 2 x 128 tensor-memory columns
// always fit in the SM's 512, so an allocation never waits
#define TC_SMEM_BYTES (100 * 1024)
#define TC_WAIT_BUDGET (1ll << 31)  // cycles (about a second) before an MMA wait gives up

// byte offset of element (row, k) of a K-major operand with K columns (no swizzle)
__device__ __forceinline__ uint32_t tc_off(int row, int k, int K)
{
    return (uint32_t)((row >> 3) * (K * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void tc_put(unsigned char *base, int row, int k, int K, float v)
{
    *reinterpret_cast<__nv_bfloat16 *>(base + tc_off(row, k, K)) = __float2bfloat16_rn(v);
}

// Bias + ReLU of 64 accumulator columns (tensor memory, this thread's row) into the BF16
// A operand (row t, K = 64).
__device__ __forceinline__ void tc_hidden(uint32_t taddr, const float *bias, unsigned char *H, int t)
{
#pragma unroll
    for (int c = 0; c < 64; c += 16) {
        float v[16];
        tc_ld16(taddr + c, v);
        uint32_t q[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            q[i] = pack_bf16(fmaxf(v[2 * i] + bias[c + 2 * i], 0.f), fmaxf(v[2 * i + 1] + bias[c + 2 * i + 1], 0.f));
        *reinterpret_cast<uint4 *>(H + tc_off(t, c, 64)) = make_uint4(q[0], q[1], q[2], q[3]);
        *reinterpret_cast<uint4 *>(H + tc_off(t, c + 8, 64)) = make_uint4(q[4], q[5], q[6], q[7]);
    }
}

// dv0 = dv_prev + sd_y * net(standardised feat) + mu_y; rows with fixed[r] != 0 get 0.
__global__ void __launch_bounds__(TC_THREADS) mlp_infer_kernel(int64_t n, const float *params, const float *stats,
                                                               const float *feat, const float *dv_prev,
                                                               const uint8_t *fixed, float *dv0, uint32_t *err)
{
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail;
    __shared__ float b1[MLP_HID], b2[MLP_HID], b3[4], mx[MLP_IN], sx[MLP_IN], my[4], sy[4];
    const int t = threadIdx.x, warp = t >> 5;
    // weights as BF16 operands (B = W, N x K, K-major)
    for (int i = t; i < MLP_HID * 16; i += TC_THREADS) {
        const int r = i >> 4, k = i & 15;
        tc_put(tsm + TC_OFF_W1, r, k, 16, k < MLP_IN ? params[OFF_W1 + r * MLP_IN + k] : 0.f);
    }
    for (int i = t; i < MLP_HID * MLP_HID; i += TC_THREADS) {
        const int r = i >> 6, k = i & 63;
        tc_put(tsm + TC_OFF_W2, r, k, 64, params[OFF_W2 + r * MLP_HID + k]);
    }
    for (int i = t; i < 16 * MLP_HID; i += TC_THREADS) {
        const int r = i >> 6, k = i & 63;
        tc_put(tsm + TC_OFF_W3, r, k, 64, r < MLP_OUT ? params[OFF_W3 + r * MLP_HID + k] : 0.f);
    }
    if (t < MLP_HID) {
        b1[t] = params[OFF_B1 + t];
        b2[t] = params[OFF_B2 + t];
    }
    if (t < MLP_IN) {
        mx[t] = stats[t];
        sx[t] = stats[MLP_IN + t];
    }
    if (t < 4) {
        b3[t] = t < MLP_OUT ? params[OFF_B3 + t] : 0.f;
        my[t] = t < MLP_OUT ? stats[2 * MLP_IN + t] : 0.f;
        sy[t] = t < MLP_OUT ? stats[2 * MLP_IN + MLP_OUT + t] : 1.f;
    }
    if (t == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
        s_fail = 0;
    }
    if (warp == 0) tc_alloc(&tmem_slot, TC_TMEM_COLS);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t lanes = (uint32_t)(32 * warp) << 16;
    const uint32_t idesc64 = tc_idesc_bf16(TC_ROWS, 64), idesc16 = tc_idesc_bf16(TC_ROWS, 16);
    unsigned char *X = tsm + TC_OFF_X, *H = tsm + TC_OFF_H;
    uint32_t phase = 0;
    const int64_t ntiles = (n + TC_ROWS - 1) / TC_ROWS;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r = tile * TC_ROWS + t;
        // ---- standardised inputs of row t as the BF16 A operand (K = 16, inputs 12..15 zero)
        {
            float v[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = 0.f;
            if (r < n) {
                const float *x = feat + MLP_IN * r;
#pragma unroll
                for (int k = 0; k < MLP_IN; ++k) v[k] = (x[k] - mx[k]) / sx[k];
            }
            uint32_t q[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) q[i] = pack_bf16(v[2 * i], v[2 * i + 1]);
            *reinterpret_cast<uint4 *>(X + tc_off(t, 0, 16)) = make_uint4(q[0], q[1], q[2], q[3]);
            *reinterpret_cast<uint4 *>(X + tc_off(t, 8, 16)) = make_uint4(q[4], q[5], q[6], q[7]);
        }
        // three layers: MMA(s) by thread 0, wait on the commit, epilogue by every thread
        for (int layer = 0; layer < 3; ++layer) {
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (t == 0) {
                if (layer == 0) {
                    tc_mma_bf16(tmem, tc_smem_desc(X, 128, 256), tc_smem_desc(tsm + TC_OFF_W1, 128, 256), idesc64,
                                false);
                } else {
                    const unsigned char *W = tsm + (layer == 1 ? TC_OFF_W2 : TC_OFF_W3);
                    const uint32_t d = tmem + (layer == 1 ? 64u : 0u);
                    for (int kk = 0; kk < 4; ++kk)
                        tc_mma_bf16(d, tc_smem_desc(H + 256 * kk, 128, 1024), tc_smem_desc(W + 256 * kk, 128, 1024),
                                    layer == 1 ? idesc64 : idesc16, kk > 0);
                }
                tc_commit(&bar);
            }
            const bool ok = mbar_wait_bounded(&bar, phase, TC_WAIT_BUDGET);
            phase ^= 1u;
            if (!ok) s_fail = 1;
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (s_fail) break;
            if (layer == 0) {
                tc_hidden(tmem + lanes, b1, H, t);
            } else if (layer == 1) {
                tc_hidden(tmem + lanes + 64, b2, H, t);
            } else {
                float y[16];
                tc_ld16(tmem + lanes, y);
                if (r < n) {
                    const bool fx = fixed && fixed[r];
#pragma unroll
                    for (int o = 0; o < MLP_OUT; ++o) {
                        const float d = dv_prev ? dv_prev[3 * r + o] : 0.f;
                        dv0[3 * r + o] = fx ? 0.f : fmaf(y[o] + b3[o], sy[o], my[o]) + d;
                    }
                }
            }
        }
        if (s_fail) break;
    }
    // every tensor-memory read of this CTA is complete before the columns are released
    tc_fence_before();
    __syncthreads();
    if (s_fail && t == 0) pc_set_err(err, PC_DERR_TIMEOUT);
    if (warp == 0) tc_dealloc(tmem, TC_TMEM_COLS);
}

// ------------------------------------------------------------------------- training (tcgen05)
//
// One CTA of four warps per SM (persistent over 128-row tiles; its shared memory keeps a
// second CTA off the SM, so the CTA owns all 512 tensor-memory columns). Per tile, one
// thread issues the tensor-core products and every thread handles its own row in the
// epilogues (warp w reads tensor-memory lanes 32w.., the tile's rows 32w..):
//   forward   D1 = X W1^T, D2 = H1 W2^T, D3 = H2 W3^T                  (M = 128 rows)
//   backward  dH2 = dY W3, dH1 = dZ2 W2                                (M = 128 rows)
//   gradients [dZ2^T ; dZ1^T] [H1^T ; X^T]^T   (M = 128: dW2 and dW1 are its diagonal
//             blocks, 64 x 64 and 64 x 16), H2^T dY (dW3^T): products over the tile's rows
//             (K = 128), accumulated in tensor memory across the CTA's tiles.
// Every operand is a K-major BF16 array in shared memory (the layout the inference kernel
// uses): the epilogues write each row's activations and back-propagated signals both as a
// row of the next product's A operand and, transposed, as a column of the gradient
// products' operands. BF16 rounding happens where the oracle's bfloat16 mode rounds
// (standardised inputs, weights, hidden activations, dY, dZ2, dZ1); the bias gradients and
// the loss are summed on the CUDA cores from the unrounded FP32 signals, per warp in a
// fixed order, so training stays bit-reproducible.
#define TT_ROWS 128
#define TT_THREADS 128
#define TT_TMEM_COLS 512  // D1 / dH2 at 0, D2 / dH1 at 64, D3 at 128, gradients at 256 and 352
#define TT_GW12 256       // 80 columns: [dW2 | dW1] blocks
#define TT_GW3 352        // 16 columns: dW3^T
#define TT_W1 0           // 64 x 16 (forward B: W1[n][k])
#define TT_W2 2048        // 64 x 64
#define TT_W3 10240       // 16 x 64 (outputs 3..15 zero)
#define TT_W3T 12288      // 64 x 16: W3T[n][k] = W3[k][n] (k < 3)
#define TT_W2T 14336      // 64 x 64: W2T[n][k] = W2[k][n]
#define TT_X 22528        // 128 x 16: standardised inputs (A of layer 1)
#define TT_H1 26624       // 128 x 64
#define TT_H2 43008       // 128 x 64
#define TT_DY 59392       // 128 x 16: dY (outputs 3..15 zero)
#define TT_DZ2 63488      // 128 x 64
#define TT_TH2 79872      // 64 x 128: H2^T; its M = 128 operand runs on into TT_TZ (rows never read)
#define TT_TZ 96256       // 128 x 128: dZ2^T (rows 0..63), dZ1^T (rows 64..127)
#define TT_TB 129024      // 80 x 128: H1^T (rows 0..63), X^T (rows 64..79; inputs 12..15 zero)
#define TT_TDY 149504     // 16 x 128: dY^T (rows 3..15 zero)
#define TT_SMEM 153600    // 150 KB: one CTA per SM

// Sum over the warp's 32 rows (lane 0 holds the total).
__device__ __forceinline__ float tt_warp_sum(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Thread 0 issues `nk` K-steps of an M = 128 product into tensor memory and commits; every
// thread waits (bounded). A and B are K-major with K extents ka, kb (bytes per 8-row group:
// 16 K). A thread whose wait gives up records it in *fail before the block barrier, so the
// return value (no failure) is the same in every thread.
__device__ __forceinline__ bool tt_mma(uint32_t d, const unsigned char *A, int ka, const unsigned char *B, int kb,
                                       int nk, uint32_t idesc, bool acc_first, uint64_t *bar, uint32_t &phase,
                                       volatile int *fail)
{
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0) {
        for (int kk = 0; kk < nk; ++kk)
            tc_mma_bf16(d, tc_smem_desc(A + 256 * kk, 128, 16 * ka), tc_smem_desc(B + 256 * kk, 128, 16 * kb), idesc,
                        acc_first || kk > 0);
        tc_commit(bar);
    }
    const bool ok = mbar_wait_bounded(bar, phase, TC_WAIT_BUDGET);
    phase ^= 1u;
    if (!ok) *fail = 1;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *fail == 0;
}

__global__ void __launch_bounds__(TT_THREADS, 1) mlp_train_kernel(int64_t n, const int32_t *rows, const float *params,
                                                                  const float *stats, const float *feat,
                                                                  const float *target, float *part, double *loss_part,
                                                                  uint32_t *err)
{
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail;
    __shared__ float b1[MLP_HID], b2[MLP_HID], b3[4], mx[MLP_IN], sx[MLP_IN], my[4], sy[4];
    __shared__ float sdb[4][2 * MLP_HID + 4];  // per-warp bias-gradient sums: db1, db2, db3
    __shared__ double sloss[4];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    // weights in the four layouts the products read; every other buffer starts at zero
    // (the padding columns of X, dY, their transposes and of W3 are never written again)
    for (int i = t; i < (TT_SMEM - TT_X) / 16; i += TT_THREADS)
        reinterpret_cast<uint4 *>(tsm + TT_X)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = t; i < MLP_HID * 16; i += TT_THREADS) {
        const int r = i >> 4, k = i & 15;
        tc_put(tsm + TT_W1, r, k, 16, k < MLP_IN ? params[OFF_W1 + r * MLP_IN + k] : 0.f);
        tc_put(tsm + TT_W3T, r, k, 16, k < MLP_OUT ? params[OFF_W3 + k * MLP_HID + r] : 0.f);
    }
    for (int i = t; i < MLP_HID * MLP_HID; i += TT_THREADS) {
        const int r = i >> 6, k = i & 63;
        tc_put(tsm + TT_W2, r, k, 64, params[OFF_W2 + r * MLP_HID + k]);
        tc_put(tsm + TT_W2T, r, k, 64, params[OFF_W2 + k * MLP_HID + r]);
    }
    for (int i = t; i < 16 * MLP_HID; i += TT_THREADS) {
        const int r = i >> 6, k = i & 63;
        tc_put(tsm + TT_W3, r, k, 64, r < MLP_OUT ? params[OFF_W3 + r * MLP_HID + k] : 0.f);
    }
    if (t < MLP_HID) {
        b1[t] = params[OFF_B1 + t];
        b2[t] = params[OFF_B2 + t];
    }
    if (t < MLP_IN) {
        mx[t] = stats[t];
        sx[t] = stats[MLP_IN + t];
    }
    if (t < 4) {
        b3[t] = t < MLP_OUT ? params[OFF_B3 + t] : 0.f;
        my[t] = t < MLP_OUT ? stats[2 * MLP_IN + t] : 0.f;
        sy[t] = t < MLP_OUT ? stats[2 * MLP_IN + MLP_OUT + t] : 1.f;
    }
    for (int i = t; i < 4 * (2 * MLP_HID + 4); i += TT_THREADS) (&sdb[0][0])[i] = 0.f;
    if (t == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
        s_fail = 0;
    }
    if (warp == 0) tc_alloc(&tmem_slot, TT_TMEM_COLS);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot, lanes = (uint32_t)(32 * warp) << 16;
    const uint32_t id64 = tc_idesc_bf16(TT_ROWS, 64), id16 = tc_idesc_bf16(TT_ROWS, 16);
    const uint32_t id80 = tc_idesc_bf16(TT_ROWS, 80);
    unsigned char *X = tsm + TT_X, *H1 = tsm + TT_H1, *H2 = tsm + TT_H2, *DY = tsm + TT_DY, *DZ2 = tsm + TT_DZ2;
    unsigned char *TH2 = tsm + TT_TH2, *TZ = tsm + TT_TZ, *TB = tsm + TT_TB, *TDY = tsm + TT_TDY;
    const float inv_n = 1.f / (float)n;
    double loss = 0.0;
    uint32_t phase = 0;
    bool first = true;
    const int64_t ntiles = (n + TT_ROWS - 1) / TT_ROWS;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r = tile * TT_ROWS + t;
        const int64_t R = r < n ? (rows ? (int64_t)rows[r] : r) : 0;
        // ---- standardised inputs: row t of X and column t of X^T (rows past n are zero)
        {
            float v[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = 0.f;
            if (r < n) {
                const float *x = feat + (int64_t)MLP_IN * R;
#pragma unroll
                for (int k = 0; k < MLP_IN; ++k) v[k] = (x[k] - mx[k]) / sx[k];
            }
            uint32_t q[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) q[i] = pack_bf16(v[2 * i], v[2 * i + 1]);
            *reinterpret_cast<uint4 *>(X + tc_off(t, 0, 16)) = make_uint4(q[0], q[1], q[2], q[3]);
            *reinterpret_cast<uint4 *>(X + tc_off(t, 8, 16)) = make_uint4(q[4], q[5], q[6], q[7]);
#pragma unroll
            for (int k = 0; k < MLP_IN; ++k) tc_put(TB, 64 + k, t, 128, v[k]);
        }
        // ---- forward: layer 1 (K = 16), bias + ReLU into H1 and H1^T
        uint64_t m1 = 0, m2 = 0;
        if (!tt_mma(tmem, X, 16, tsm + TT_W1, 16, 1, id64, false, &bar, phase, &s_fail)) break;
#pragma unroll
        for (int c = 0; c < 64; c += 16) {
            float v[16];
            tc_ld16(tmem + lanes + c, v);
            uint32_t q[8];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float z = v[i] + b1[c + i];
                m1 |= (uint64_t)(z > 0.f) << (c + i);
                v[i] = fmaxf(z, 0.f);
                tc_put(TB, c + i, t, 128, v[i]);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) q[i] = pack_bf16(v[2 * i], v[2 * i + 1]);
            *reinterpret_cast<uint4 *>(H1 + tc_off(t, c, 64)) = make_uint4(q[0], q[1], q[2], q[3]);
            *reinterpret_cast<uint4 *>(H1 + tc_off(t, c + 8, 64)) = make_uint4(q[4], q[5], q[6], q[7]);
        }
        // ---- layer 2 (K = 64): H2 and H2^T
        if (!tt_mma(tmem + 64, H1, 64, tsm + TT_W2, 64, 4, id64, false, &bar, phase, &s_fail)) break;
#pragma unroll
        for (int c = 0; c < 64; c += 16) {
            float v[16];
            tc_ld16(tmem + lanes + 64 + c, v);
            uint32_t q[8];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const float z = v[i] + b2[c + i];
                m2 |= (uint64_t)(z > 0.f) << (c + i);
                v[i] = fmaxf(z, 0.f);
                tc_put(TH2, c + i, t, 128, v[i]);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) q[i] = pack_bf16(v[2 * i], v[2 * i + 1]);
            *reinterpret_cast<uint4 *>(H2 + tc_off(t, c, 64)) = make_uint4(q[0], q[1], q[2], q[3]);
            *reinterpret_cast<uint4 *>(H2 + tc_off(t, c + 8, 64)) = make_uint4(q[4], q[5], q[6], q[7]);
        }
        // ---- layer 3 (K = 64, N = 16): output error dY = (y - t) / n into dY and dY^T
        if (!tt_mma(tmem + 128, H2, 64, tsm + TT_W3, 64, 4, id16, false, &bar, phase, &s_fail)) break;
        {
            float v[16];
            tc_ld16(tmem + lanes + 128, v);
            float dy[MLP_OUT] = {0.f, 0.f, 0.f};
            if (r < n) {
#pragma unroll
                for (int o = 0; o < MLP_OUT; ++o) {
                    const float raw = target[3 * R + o] - feat[(int64_t)MLP_IN * R + 3 + o];  // dv - dv_prev
                    const float tn = (raw - my[o]) / sy[o];
                    const float e = (v[o] + b3[o]) - tn;
                    loss += (double)e * (double)e;
                    dy[o] = e * inv_n;
                }
            }
            *reinterpret_cast<uint4 *>(DY + tc_off(t, 0, 16)) =
                make_uint4(pack_bf16(dy[0], dy[1]), pack_bf16(dy[2], 0.f), 0u, 0u);
#pragma unroll
            for (int o = 0; o < MLP_OUT; ++o) {
                tc_put(TDY, o, t, 128, dy[o]);
                const float s_ = tt_warp_sum(dy[o]);
                if (lane == 0) sdb[warp][2 * MLP_HID + o] += s_;
            }
        }
        // ---- dH2 = dY W3 (K = 16): dZ2 = dH2 [Z2 > 0] into dZ2 and dZ2^T (TZ rows 0..63)
        if (!tt_mma(tmem, DY, 16, tsm + TT_W3T, 16, 1, id64, false, &bar, phase, &s_fail)) break;
#pragma unroll
        for (int c = 0; c < 64; c += 16) {
            float v[16];
            tc_ld16(tmem + lanes + c, v);
            uint32_t q[8];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                v[i] = ((m2 >> (c + i)) & 1u) ? v[i] : 0.f;
                tc_put(TZ, c + i, t, 128, v[i]);
                const float s_ = tt_warp_sum(v[i]);
                if (lane == 0) sdb[warp][MLP_HID + c + i] += s_;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) q[i] = pack_bf16(v[2 * i], v[2 * i + 1]);
            *reinterpret_cast<uint4 *>(DZ2 + tc_off(t, c, 64)) = make_uint4(q[0], q[1], q[2], q[3]);
            *reinterpret_cast<uint4 *>(DZ2 + tc_off(t, c + 8, 64)) = make_uint4(q[4], q[5], q[6], q[7]);
        }
        // ---- dH1 = dZ2 W2 (K = 64): dZ1 = dH1 [Z1 > 0] into dZ1^T (TZ rows 64..127)
        if (!tt_mma(tmem + 64, DZ2, 64, tsm + TT_W2T, 64, 4, id64, false, &bar, phase, &s_fail)) break;
#pragma unroll
        for (int c = 0; c < 64; c += 16) {
            float v[16];
            tc_ld16(tmem + lanes + 64 + c, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                v[i] = ((m1 >> (c + i)) & 1u) ? v[i] : 0.f;
                tc_put(TZ, 64 + c + i, t, 128, v[i]);
                const float s_ = tt_warp_sum(v[i]);
                if (lane == 0) sdb[warp][c + i] += s_;
            }
        }
        // ---- weight gradients over the tile's rows (K = 128), accumulated in tensor memory
        if (!tt_mma(tmem + TT_GW12, TZ, 128, TB, 128, 8, id80, !first, &bar, phase, &s_fail)) break;
        if (!tt_mma(tmem + TT_GW3, TH2, 128, TDY, 128, 8, id16, !first, &bar, phase, &s_fail)) break;
        first = false;
    }
    // ---- this CTA's partials: dW2 (rows 0..63, columns 0..63 of the first gradient),
    // dW1 (rows 64..127, columns 64..75), dW3^T (rows 0..63 of the second)
    float *out = part + (int64_t)blockIdx.x * PC_MLP_NPARAMS;
    if (!s_fail) {
        if (warp < 2) {
            const int i = 32 * warp + lane;  // dW2 row (output unit) / dW3^T row (hidden unit)
#pragma unroll
            for (int c = 0; c < 64; c += 16) {
                float v[16];
                tc_ld16(tmem + lanes + TT_GW12 + c, v);
#pragma unroll
                for (int k = 0; k < 16; ++k) out[OFF_W2 + i * MLP_HID + c + k] = first ? 0.f : v[k];
            }
            float w[16];
            tc_ld16(tmem + lanes + TT_GW3, w);
#pragma unroll
            for (int o = 0; o < MLP_OUT; ++o) out[OFF_W3 + o * MLP_HID + i] = first ? 0.f : w[o];
        } else {
            const int o = 32 * (warp - 2) + lane;  // dW1 row (hidden unit)
            float v[16];
            tc_ld16(tmem + lanes + TT_GW12 + 64, v);
#pragma unroll
            for (int k = 0; k < MLP_IN; ++k) out[OFF_W1 + o * MLP_IN + k] = first ? 0.f : v[k];
        }
    }
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if (lane == 0) sloss[warp] = loss;
    // every tensor-memory read of this CTA is complete before the columns are released
    tc_fence_before();
    __syncthreads();
    for (int j = t; j < 2 * MLP_HID + MLP_OUT; j += TT_THREADS) {
        float s_ = 0.f;
        for (int w = 0; w < 4; ++w) s_ += sdb[w][j];
        const int dst = j < MLP_HID ? OFF_B1 + j : j < 2 * MLP_HID ? OFF_B2 + (j - MLP_HID) : OFF_B3 + (j - 2 * MLP_HID);
        out[dst] = s_;
    }
    if (t == 0) {
        loss_part[blockIdx.x] = sloss[0] + sloss[1] + sloss[2] + sloss[3];
        if (s_fail) pc_set_err(err, PC_DERR_TIMEOUT);
    }
    if (warp == 0) tc_dealloc(tmem, TT_TMEM_COLS);
}

// grad = sum of the CTA partials in CTA order (FP64 accumulation); with adam != 0 also the
// Adam update of the FP32 master weights: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr (m / bc1) / (sqrt(v / bc2) + eps) with bc = 1 - beta^t.
__global__ void mlp_reduce_adam_kernel(int nparts, const float *part, float *grad, int adam, float *params, float *m,
                                       float *v, float lr, float beta1, float beta2, float eps, float bc1, float bc2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= PC_MLP_NPARAMS) return;
    double acc = 0.0;
    for (int c = 0; c < nparts; ++c) acc += (double)part[(int64_t)c * PC_MLP_NPARAMS + p];
    const float gr = (float)acc;
    if (grad) grad[p] = gr;
    if (adam) {
        const float mm = beta1 * m[p] + (1.f - beta1) * gr;
        const float vv = beta2 * v[p] + (1.f - beta2) * gr * gr;
        m[p] = mm;
        v[p] = vv;
        params[p] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
    }
}

__global__ void mlp_loss_sum_kernel(int nparts, const double *loss_part, double *loss)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double t = 0.0;
    for (int c = 0; c < nparts; ++c) t += loss_part[c];
    *loss = t;
}

// ------------------------------------------------------------------------- statistics

#define ST_COLS (MLP_IN + MLP_OUT)

// per-block FP64 sums of each column and of its square (rows grid-strided, fixed order)
__global__ void __launch_bounds__(256) mlp_stats_partial_kernel(int64_t n, const float *feat, const float *target,
                                                                double *part)
{
    __shared__ double s[2 * ST_COLS][8];
    double acc[2 * ST_COLS];
#pragma unroll
    for (int j = 0; j < 2 * ST_COLS; ++j) acc[j] = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int j = 0; j < ST_COLS; ++j) {
            const double x = j < MLP_IN ? (double)feat[MLP_IN * r + j]
                                        : (double)target[MLP_OUT * r + j - MLP_IN] - (double)feat[MLP_IN * r + 3 + j - MLP_IN];
            acc[j] += x;
            acc[ST_COLS + j] += x * x;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 2 * ST_COLS; ++j) {
        double w = acc[j];
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (lane == 0) s[j][warp] = w;
    }
    __syncthreads();
    if (threadIdx.x < 2 * ST_COLS) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[threadIdx.x][w];
        part[(int64_t)blockIdx.x * 2 * ST_COLS + threadIdx.x] = t;
    }
}

__global__ void mlp_stats_final_kernel(int nparts, int64_t n, const double *part, float *stats)
{
    const int j = threadIdx.x;
    if (j >= ST_COLS) return;
    double s1 = 0.0, s2 = 0.0;
    for (int b = 0; b < nparts; ++b) {
        s1 += part[(int64_t)b * 2 * ST_COLS + j];
        s2 += part[(int64_t)b * 2 * ST_COLS + ST_COLS + j];
    }
    const double mean = s1 / (double)n;
    const double var = fmax(s2 / (double)n - mean * mean, 0.0);
    const double sd = fmax(sqrt(var), 1e-12);
    if (j < MLP_IN) {
        stats[j] = (float)mean;
        stats[MLP_IN + j] = (float)sd;
    } else {
        stats[2 * MLP_IN + (j - MLP_IN)] = (float)mean;
        stats[2 * MLP_IN + MLP_OUT + (j - MLP_IN)] = (float)sd;
    }
}

// ------------------------------------------------------------------------- features

__global__ void mlp_features_kernel(int V, const float *v, const float *dv_prev, const float *b, const float *mass,
                                    const float *rest_len, float inv_h, float g0, float g1, float g2,
                                    const int32_t *erp, const int32_t *ecol, float *feat)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V) return;
    float *f = feat + (int64_t)MLP_IN * i;
    const float m = mass[i];
    // force per unit mass times the vertex's rest edge length: the membrane's share does
    // not change with the grid spacing (force ~ stress x edge, mass ~ edge^2)
    const float inv_m = m > 0.f ? rest_len[i] / m : 0.f;
    const float g[3] = {g0, g1, g2};
    float ring[3] = {0.f, 0.f, 0.f};
    const int e0 = erp[i], e1 = erp[i + 1];
    for (int e = e0; e < e1; ++e) {
        const int j = ecol[e];
        for (int d = 0; d < 3; ++d) ring[d] += dv_prev[3ll * j + d];
    }
    const float inv_deg = e1 > e0 ? 1.f / (float)(e1 - e0) : 0.f;
    for (int d = 0; d < 3; ++d) {
        f[d] = v[3ll * i + d];
        f[3 + d] = dv_prev[3ll * i + d];
        f[6 + d] = (b[3ll * i + d] * inv_h - m * g[d]) * inv_m;
        f[9 + d] = ring[d] * inv_deg;
    }
}

// ------------------------------------------------------------------------- host side

struct pc_mlp {
    int device = 0;
    int num_sms = 0;
    int max_parts = 0;
    float *part = nullptr;     // [max_parts][NPARAMS]
    double *loss_part = nullptr;
    double *loss = nullptr;    // device scalar
    double *h_loss = nullptr;  // pinned mirror
    double *stat_part = nullptr;
    float *m = nullptr, *v = nullptr;  // Adam moments
    int64_t t = 0;                     // Adam steps taken
    uint32_t *err = nullptr;           // timeout flag of the training products
    uint32_t *h_err = nullptr;         // pinned mirror
};

extern "C" pc_status pc_mlp_create(pc_mlp **out)
{
    if (!out) return PC_ERR_ARG;
    *out = nullptr;
    pc_mlp *M = new pc_mlp();
    auto fail = [&](cudaError_t e, const char *what) {
        pc_note_cuda_error(e, what, __FILE__, __LINE__);
        pc_mlp_destroy(M);
        return PC_ERR_CUDA;
    };
    cudaError_t e;
    if ((e = cudaGetDevice(&M->device)) != cudaSuccess) return fail(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&M->num_sms, cudaDevAttrMultiProcessorCount, M->device)) != cudaSuccess)
        return fail(e, "cudaDeviceGetAttribute");
    M->max_parts = 2 * M->num_sms;
    if ((e = cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TT_SMEM)) !=
        cudaSuccess)
        return fail(e, "cudaFuncSetAttribute");
    if ((e = cudaMalloc(&M->err, sizeof(uint32_t))) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMemset(M->err, 0, sizeof(uint32_t))) != cudaSuccess) return fail(e, "cudaMemset");
    if ((e = cudaMallocHost(&M->h_err, sizeof(uint32_t))) != cudaSuccess) return fail(e, "cudaMallocHost");
    if ((e = cudaMalloc(&M->part, sizeof(float) * PC_MLP_NPARAMS * (size_t)M->max_parts)) != cudaSuccess)
        return fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&M->loss_part, sizeof(double) * (size_t)M->max_parts)) != cudaSuccess)
        return fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&M->loss, sizeof(double))) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMallocHost(&M->h_loss, sizeof(double))) != cudaSuccess) return fail(e, "cudaMallocHost");
    if ((e = cudaMalloc(&M->stat_part, sizeof(double) * 2 * ST_COLS * (size_t)M->max_parts)) != cudaSuccess)
        return fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&M->m, sizeof(float) * PC_MLP_NPARAMS)) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMalloc(&M->v, sizeof(float) * PC_MLP_NPARAMS)) != cudaSuccess) return fail(e, "cudaMalloc");
    if ((e = cudaMemset(M->m, 0, sizeof(float) * PC_MLP_NPARAMS)) != cudaSuccess) return fail(e, "cudaMemset");
    if ((e = cudaMemset(M->v, 0, sizeof(float) * PC_MLP_NPARAMS)) != cudaSuccess) return fail(e, "cudaMemset");
    *out = M;
    return PC_OK;
}

extern "C" pc_status pc_mlp_destroy(pc_mlp *M)
{
    if (!M) return PC_OK;
    cudaFree(M->part);
    cudaFree(M->loss_part);
    cudaFree(M->loss);
    if (M->h_loss) cudaFreeHost(M->h_loss);
    cudaFree(M->stat_part);
    cudaFree(M->m);
    cudaFree(M->v);
    cudaFree(M->err);
    if (M->h_err) cudaFreeHost(M->h_err);
    delete M;
    return PC_OK;
}

extern "C" pc_status pc_mlp_reset(pc_mlp *M, void *stream)
{
    if (!M) return PC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    PC_CUDA_TRY(cudaMemsetAsync(M->m, 0, sizeof(float) * PC_MLP_NPARAMS, st));
    PC_CUDA_TRY(cudaMemsetAsync(M->v, 0, sizeof(float) * PC_MLP_NPARAMS, st));
    M->t = 0;
    return PC_OK;
}

#define MLP_LAUNCH(kernel, grid, block, smem, stream, ...)                           \
    do {                                                                           \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                \
        cudaError_t _le = cudaGetLastError();                                      \
        if (_le != cudaSuccess) {                                                  \
            pc_note_cuda_error(_le, #kernel, __FILE__, __LINE__);                  \
            return PC_ERR_CUDA;                                                    \
        }                                                                          \
    } while (0)

extern "C" pc_status pc_mlp_stats(pc_mlp *M, int64_t n, const float *feat, const float *target, float *stats,
                                  void *stream)
{
    if (!M || n <= 0 || !feat || !target || !stats) return PC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = (int)std::min<int64_t>(M->max_parts, (n + 255) / 256);
    MLP_LAUNCH(mlp_stats_partial_kernel, grid, 256, 0, st, n, feat, target, M->stat_part);
    MLP_LAUNCH(mlp_stats_final_kernel, 1, 32, 0, st, grid, n, M->stat_part, stats);
    return PC_OK;
}

extern "C" pc_status pc_mlp_infer(int64_t n, const float *params, const float *stats, const float *feat,
                                  const float *dv_prev, const uint8_t *fixed, float *dv0, void *stream)
{
    if (n < 0 || !params || !stats || !feat || !dv0) return PC_ERR_ARG;
    if (n == 0) return PC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    PC_CUDA_TRY(cudaGetDevice(&dev));
    PC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PC_CUDA_TRY(cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_BYTES));
    static thread_local uint32_t *d_err = nullptr;  // timeout flag of this host thread's launches
    static thread_local int err_dev = -1;
    if (!d_err || err_dev != dev) {
        PC_CUDA_TRY(cudaMalloc(&d_err, sizeof(uint32_t)));
        err_dev = dev;
    }
    PC_CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(uint32_t), st));
    const int64_t tiles = (n + TC_ROWS - 1) / TC_ROWS;
    const int grid = (int)std::min<int64_t>(tiles, 2ll * sms);
    MLP_LAUNCH(mlp_infer_kernel, grid, TC_THREADS, TC_SMEM_BYTES, st, n, params, stats, feat, dv_prev, fixed, dv0,
               d_err);
    uint32_t h_err = 0;
    PC_CUDA_TRY(cudaMemcpyAsync(&h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    return h_err ? PC_ERR_TIMEOUT : PC_OK;
}

static pc_status mlp_grad_impl(pc_mlp *M, int64_t n, const int32_t *rows, const float *params, const float *stats,
                               const float *feat, const float *target, float *grad, bool adam,
                               const pc_adam_opts *o, double *loss, cudaStream_t st)
{
    if (!M || n <= 0 || !params || !stats || !feat || !target) return PC_ERR_ARG;
    const int64_t tiles = (n + TT_ROWS - 1) / TT_ROWS;
    // one CTA per SM at most: each holds all of its SM's tensor-memory columns
    const int grid = (int)std::min<int64_t>(tiles, M->num_sms);
    MLP_LAUNCH(mlp_train_kernel, grid, TT_THREADS, TT_SMEM, st, n, rows, params, stats, feat, target, M->part,
               M->loss_part, M->err);
    float lr = 0.f, b1 = 0.f, b2 = 0.f, eps = 0.f, bc1 = 1.f, bc2 = 1.f;
    if (adam) {
        M->t += 1;
        lr = o->lr;
        b1 = o->beta1;
        b2 = o->beta2;
        eps = o->eps;
        bc1 = (float)(1.0 - pow((double)b1, (double)M->t));
        bc2 = (float)(1.0 - pow((double)b2, (double)M->t));
    }
    MLP_LAUNCH(mlp_reduce_adam_kernel, (PC_MLP_NPARAMS + 255) / 256, 256, 0, st, grid, M->part, grad, adam ? 1 : 0,
               (float *)params, M->m, M->v, lr, b1, b2, eps, bc1, bc2);
    if (loss) {
        MLP_LAUNCH(mlp_loss_sum_kernel, 1, 32, 0, st, grid, M->loss_part, M->loss);
        PC_CUDA_TRY(cudaMemcpyAsync(M->h_loss, M->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        PC_CUDA_TRY(cudaMemcpyAsync(M->h_err, M->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        PC_CUDA_TRY(cudaStreamSynchronize(st));
        *loss = 0.5 * *M->h_loss / (double)n;
        if (*M->h_err) {  // a product wait gave up (in this or an earlier unsynchronised call)
            PC_CUDA_TRY(cudaMemsetAsync(M->err, 0, sizeof(uint32_t), st));
            return PC_ERR_TIMEOUT;
        }
    }
    return PC_OK;
}

extern "C" pc_status pc_mlp_grad(pc_mlp *M, int64_t n, const int32_t *rows, const float *params, const float *stats,
                                 const float *feat, const float *target, float *grad, double *loss, void *stream)
{
    if (!grad) return PC_ERR_ARG;
    return mlp_grad_impl(M, n, rows, params, stats, feat, target, grad, false, nullptr, loss, (cudaStream_t)stream);
}

extern "C" pc_status pc_mlp_train_step(pc_mlp *M, int64_t n, const int32_t *rows, float *params, const float *stats,
                                       const float *feat, const float *target, const pc_adam_opts *o, double *loss,
                                       void *stream)
{
    if (!o || !(o->lr > 0.f) || !(o->beta1 >= 0.f && o->beta1 < 1.f) || !(o->beta2 >= 0.f && o->beta2 < 1.f) ||
        !(o->eps > 0.f))
        return PC_ERR_ARG;
    return mlp_grad_impl(M, n, rows, params, stats, feat, target, nullptr, true, o, loss, (cudaStream_t)stream);
}

extern "C" pc_status pc_mlp_adam_apply(pc_mlp *M, float *params, const float *grad, const pc_adam_opts *o,
                                       void *stream)
{
    if (!M || !params || !grad || !o) return PC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // the gradient goes through the partial-sum path as a single "CTA"
    PC_CUDA_TRY(cudaMemcpyAsync(M->part, grad, sizeof(float) * PC_MLP_NPARAMS, cudaMemcpyDeviceToDevice, st));
    M->t += 1;
    const float bc1 = (float)(1.0 - pow((double)o->beta1, (double)M->t));
    const float bc2 = (float)(1.0 - pow((double)o->beta2, (double)M->t));
    MLP_LAUNCH(mlp_reduce_adam_kernel, (PC_MLP_NPARAMS + 255) / 256, 256, 0, st, 1, M->part, (float *)nullptr, 1,
               params, M->m, M->v, o->lr, o->beta1, o->beta2, o->eps, bc1, bc2);
    return PC_OK;
}

extern "C" pc_status pc_mlp_features(pc_ctx *ctx, const float *v, const float *dv_prev, const float *b, float h,
                                     float *feat, void *stream)
{
    if (!ctx || !v || !dv_prev || !b || !feat || !(h > 0.f)) return PC_ERR_ARG;
    PC_LAUNCH(ctx, mlp_features_kernel, pc_blocks(ctx->V, 256), 256, 0, (cudaStream_t)stream, ctx->V, v, dv_prev, b,
              ctx->mass, ctx->rest_len, 1.f / h, ctx->mat.gravity[0], ctx->mat.gravity[1], ctx->mat.gravity[2],
              ctx->erp, ctx->ecol, feat);
    return PC_OK;
}

extern "C" pc_status pc_set_warm_mlp(pc_ctx *ctx, const float *params, const float *stats)
{
    if (!ctx || (params == nullptr) != (stats == nullptr)) return PC_ERR_ARG;
    if (params && !ctx->mlp_feat) {
        PC_CUDA_TRY(cudaMalloc(&ctx->mlp_feat, sizeof(float) * MLP_IN * (size_t)ctx->V));
        PC_CUDA_TRY(cudaMalloc(&ctx->mlp_dv, sizeof(float) * 3 * (size_t)ctx->V));
    }
    ctx->mlp_params = params;
    ctx->mlp_stats = stats;
    return PC_OK;
}

void pc_mlp_ctx_free(pc_ctx *c)
{
    cudaFree(c->mlp_feat);
    cudaFree(c->mlp_dv);
    c->mlp_feat = nullptr;
    c->mlp_dv = nullptr;
}

// The step's initial guess (ctx->A_dv holds the previous step's dv, or zeros). Features
// are written to feat_out when given. PC_WARM_MLP combines the previous-step guess g_p
// and the learned guess g_l: the combination c_p g_p + c_l g_l with the lowest CG energy
// phi(g) = 1/2 g.A g - b.g (phi(g) - phi(dv*) is half the squared A-norm of the guess's
// error, the measure CG's convergence is bounded by) solves the 2x2 Galerkin system
//   [g_p.A g_p  g_p.A g_l] [c_p]   [b.g_p]
//   [g_l.A g_p  g_l.A g_l] [c_l] = [b.g_l],
// formed in FP64 from the matrix the solve uses. The zero, previous and learned guesses
// are points of the same plane, so the optimum is never worse than any of them; the
// energy of the FP32 combination actually formed is evaluated again and compared with
// theirs, and the best of the four starts the solve. Residuals |b - A g| / |b| of the
// single guesses are reported too.
pc_status pc_warm_guess(pc_ctx *c, const pc_bsr *A, const float *v, float h, int32_t mode, float *feat_out,
                        int32_t *guess, double *guess_res, double *guess_energy, double *guess_coef,
                        double *combo_energy, cudaStream_t st)
{
    const size_t vb = sizeof(float) * 3 * (size_t)c->V;
    for (int k = 0; k < 3; ++k) {
        guess_res[k] = -1.0;
        guess_energy[k] = 0.0;
    }
    guess_coef[0] = guess_coef[1] = 0.0;
    *combo_energy = 0.0;
    float *feat = feat_out ? feat_out : c->mlp_feat;
    if (mode == PC_WARM_MLP && (!c->mlp_params || !c->mlp_feat)) return PC_ERR_ARG;
    if (feat) PC_TRY(pc_mlp_features(c, v, c->A_dv, c->A_b, h, feat, st));
    if (mode == PC_WARM_PREV) {
        *guess = c->has_prev_dv ? PC_WARM_PREV : PC_WARM_ZERO;
        return PC_OK;
    }
    if (mode != PC_WARM_MLP) {
        *guess = PC_WARM_ZERO;
        PC_CUDA_TRY(cudaMemsetAsync(c->A_dv, 0, vb, st));
        return PC_OK;
    }
    PC_TRY(pc_mlp_infer(c->V, c->mlp_params, c->mlp_stats, feat, c->A_dv, c->pinned, c->mlp_dv, st));
    double rr_prev = 0.0, rr_mlp = 0.0, bb = 0.0, e_prev = 0.0, e_mlp = 0.0;
    PC_TRY(pc_guess_eval(c, A, c->A_vals, c->A_dres, c->A_b, c->A_dv, &rr_prev, &bb, &e_prev, st));
    const double gAg_p = c->sc_host->pq, bg_p = c->sc_host->rz;
    PC_TRY(pc_guess_eval(c, A, c->A_vals, c->A_dres, c->A_b, c->mlp_dv, &rr_mlp, &bb, &e_mlp, st));
    const double gAg_l = c->sc_host->pq, bg_l = c->sc_host->rz;
    const double nb = sqrt(bb);
    guess_res[0] = bb > 0 ? 1.0 : 0.0;
    guess_res[1] = bb > 0 ? sqrt(rr_prev) / nb : 0.0;
    guess_res[2] = bb > 0 ? sqrt(rr_mlp) / nb : 0.0;
    guess_energy[1] = e_prev;
    guess_energy[2] = e_mlp;
    // the best single guess, the fallback
    int best = 0;
    double e_best = 0.0;
    if (c->has_prev_dv && e_prev < e_best) { best = 1; e_best = e_prev; }
    if (std::isfinite(e_mlp) && e_mlp < e_best) { best = 2; e_best = e_mlp; }
    // the Galerkin combination (one-dimensional on the learned guess before the first step)
    double cp = 0.0, cl = 0.0;
    bool combo = false;
    if (std::isfinite(e_mlp) && gAg_l > 0.0) {
        if (c->has_prev_dv && gAg_p > 0.0) {
            double g_pl = 0.0;
            PC_TRY(pc_guess_cross(c, A, c->A_vals, c->A_dres, c->A_dv, c->mlp_dv, &g_pl, st));
            const double det = gAg_p * gAg_l - g_pl * g_pl;
            if (std::isfinite(g_pl) && det > 1e-12 * gAg_p * gAg_l) {
                cp = (bg_p * gAg_l - bg_l * g_pl) / det;
                cl = (bg_l * gAg_p - bg_p * g_pl) / det;
                combo = true;
            }
        } else {
            cl = bg_l / gAg_l;
            combo = true;
        }
    }
    if (combo && std::isfinite(cp) && std::isfinite(cl)) {
        // form it in scratch (rhs32 is free until the solve) and measure what was formed
        float *g = c->rhs32;
        PC_TRY(pc_guess_combine(c, g, c->A_dv, c->mlp_dv, c->has_prev_dv ? cp : 0.0, cl, st));
        double rr_c = 0.0, e_c = 0.0;
        PC_TRY(pc_guess_eval(c, A, c->A_vals, c->A_dres, c->A_b, g, &rr_c, &bb, &e_c, st));
        if (std::isfinite(e_c) && e_c <= e_best) {
            *guess = PC_WARM_COMBINED;
            guess_coef[0] = c->has_prev_dv ? cp : 0.0;
            guess_coef[1] = cl;
            *combo_energy = e_c;
            PC_CUDA_TRY(cudaMemcpyAsync(c->A_dv, g, vb, cudaMemcpyDeviceToDevice, st));
            return PC_OK;
        }
    }
    *combo_energy = e_best;
    if (best == 0) {
        *guess = PC_WARM_ZERO;
        PC_CUDA_TRY(cudaMemsetAsync(c->A_dv, 0, vb, st));
    } else if (best == 1) {
        *guess = PC_WARM_PREV;
    } else {
        *guess = PC_WARM_MLP;
        PC_CUDA_TRY(cudaMemcpyAsync(c->A_dv, c->mlp_dv, vb, cudaMemcpyDeviceToDevice, st));
    }
    return PC_OK;
}

extern "C" pc_status pc_mlp_get_state(pc_mlp *m, float *m1, float *m2, int64_t *t, void *stream)
{
    if (!m || !m1 || !m2 || !t) return PC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    PC_CUDA_TRY(cudaMemcpyAsync(m1, m->m, sizeof(float) * PC_MLP_NPARAMS, cudaMemcpyDeviceToDevice, st));
    PC_CUDA_TRY(cudaMemcpyAsync(m2, m->v, sizeof(float) * PC_MLP_NPARAMS, cudaMemcpyDeviceToDevice, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    *t = m->t;
    return PC_OK;
}

extern "C" pc_status pc_mlp_set_state(pc_mlp *m, const float *m1, const float *m2, int64_t t, void *stream)
{
    if (!m || !m1 || !m2 || t < 0) return PC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    PC_CUDA_TRY(cudaMemcpyAsync(m->m, m1, sizeof(float) * PC_MLP_NPARAMS, cudaMemcpyDeviceToDevice, st));
    PC_CUDA_TRY(cudaMemcpyAsync(m->v, m2, sizeof(float) * PC_MLP_NPARAMS, cudaMemcpyDeviceToDevice, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    m->t = t;
    return PC_OK;
}
