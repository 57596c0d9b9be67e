// Row-partitioned PCG across ranks (Sec. 3.1, Eq. 4-5): the system's rows are split into
// contiguous blocks, one per rank (one GPU each). A rank stores its rows of A, of every
// PCG vector and of the right-hand side; vector operations need no communication, and
// the product A p needs, besides the rank's own entries of p, the "halo": the entries of
// p owned by other ranks that its rows' blocks reference.
//
// GB300-first reading of the paper's pipelined SpMV. The paper splits each rank's rows
// into column blocks A_ij and multiplies each as soon as the peer's whole sub-vector v_j
// has arrived (Eq. 5). Here a rank receives only the halo entries it needs (cloth rows
// touch few remote rows: the partition boundary and cross-rank contact pairs), and the
// product runs in two parts, which is Eq. 5 with the peers' column blocks merged:
//   q = A_own p_own                 (the bulk-copy SpMV kernel, launched first)
//     + A_halo p_halo               (the halo blocks, accumulated once the halo arrived)
// The halo is packed on the main stream, exchanged on a second stream while the own-part
// product runs on the main stream, and the halo part waits only for the exchange: the
// overlap of transfers and multiplication the paper's pipeline is built for.
//
// The caller supplies the communication (pc_comm: NCCL, MPI, gloo ...): one all-reduce of
// a few doubles and one exchange of device buffers between peers. Per iteration: one
// halo exchange of p and two all-reduces (p.q for alpha; r.z and r.r for beta and the
// stop test). Every rank reduces to the same global scalars, so all ranks take the same
// decisions and make the same number of calls.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "pc_internal.cuh"

#define RED_SLOTS 4

__device__ __forceinline__ double ds_warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// block sum of n <= RED_SLOTS doubles in a fixed tree (thread 0 gets the totals)
__device__ __forceinline__ void block_sum_d(double *v, int n)
{
    __shared__ double s[RED_SLOTS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < n; ++k) {
        double w = ds_warp_sum(v[k]);
        if (lane == 0) s[k][warp] = w;
    }
    __syncthreads();
    if (warp == 0) {
        for (int k = 0; k < n; ++k) {
            double w = lane < nw ? s[k][lane] : 0.0;
            v[k] = ds_warp_sum(w);
        }
    }
    __syncthreads();
}
#include "pc_spmv.cuh"

#define DS_THREADS 256
#define DS_MAX_BLOCKS 2048

struct pc_dist {
    int device = 0, rank = 0, nranks = 1, num_sms = 0;
    int32_t V_global = 0, row0 = 0, row1 = 0, n_own = 0;
    std::vector<int32_t> row_starts;
    int64_t cap = 0;        // local block capacity
    int64_t halo_cap = 0;   // halo entries and send entries capacity
    // pattern of the last plan
    int planned = 0;
    int64_t off0 = 0, nnzb = 0, nnzb_own = 0, nnzb_halo = 0, n_halo = 0, n_send = 0;
    std::vector<int64_t> recv_cnt, recv_start, send_cnt, send_start;  // entries per peer
    int32_t *own_rp = nullptr, *own_ci = nullptr, *halo_rp = nullptr, *halo_ci = nullptr;
    int32_t *own_cnt = nullptr, *halo_cnt = nullptr;
    int32_t *blk_dst = nullptr;     // per local block: own position, or -(halo position) - 1
    int32_t *halo_cols = nullptr;   // [halo_cap] global columns of the halo, sorted
    int32_t *remote = nullptr;      // [cap] remote columns as found (any order)
    int32_t *req = nullptr;         // [halo_cap] requested global rows received from the peers
    int32_t *send_idx = nullptr;    // [halo_cap] local rows to send, grouped by peer
    int64_t *cnt_send = nullptr, *cnt_recv = nullptr;  // [nranks] request counts (exchange)
    uint32_t *counter = nullptr;    // remote-column counter
    float *own_vals = nullptr, *halo_vals = nullptr;
    // vectors
    float4 *p_ext = nullptr;        // [n_own + halo_cap]: own p, then the halo
    float4 *q4 = nullptr, *z4 = nullptr, *send4 = nullptr;
    float *x = nullptr, *r = nullptr, *dinv = nullptr;  // packed float[n_own][3]
    double *x64 = nullptr;          // [n_own + halo_cap][3]: own accumulator, then the halo
    double *send64 = nullptr;       // [halo_cap][3]
    double *partials = nullptr;     // [DS_MAX_BLOCKS][RED_SLOTS]
    double *hpart = nullptr;        // [DS_MAX_BLOCKS] halo-part p.q partials
    double *red = nullptr;          // [8] local sums, all-reduced in place
    pc_scalars *sc = nullptr;
    pc_scalars *sc_host = nullptr;
    uint32_t *err = nullptr, *h_err = nullptr;
    int64_t *h_tmp = nullptr;       // pinned host scratch
    cudaStream_t s1 = nullptr;
    cudaEvent_t ev_pack = nullptr, ev_halo = nullptr;
    int64_t launches = 0;
};

#define DS_LAUNCH(d, kernel, grid, block, smem, stream, ...)                          \
    do {                                                                          \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);               \
        (d)->launches++;                                                          \
        cudaError_t _le = cudaGetLastError();                                     \
        if (_le != cudaSuccess) {                                                 \
            pc_note_cuda_error(_le, #kernel, __FILE__, __LINE__);                 \
            return PC_ERR_CUDA;                                                   \
        }                                                                         \
    } while (0)

static unsigned ds_grid(const pc_dist *d, int64_t n)
{
    int64_t b = (n + DS_THREADS - 1) / DS_THREADS;
    int64_t g = (int64_t)d->num_sms * 4;
    if (b < 1) b = 1;
    if (b > g) b = g;
    if (b > DS_MAX_BLOCKS) b = DS_MAX_BLOCKS;
    return (unsigned)b;
}

// ------------------------------------------------------------------------- partition (host)

// Balanced contiguous row blocks, boundaries on multiples of 32 rows (the product's tile):
// by block count when row_ptr (host, V+1 entries) is given, else by rows.
extern "C" pc_status pc_dist_partition(int32_t V, const int32_t *row_ptr, int32_t nranks, int32_t *row_starts)
{
    if (V < 1 || nranks < 1 || !row_starts) return PC_ERR_ARG;
    const int64_t total = row_ptr ? (int64_t)row_ptr[V] - row_ptr[0] : (int64_t)V;
    row_starts[0] = 0;
    int32_t prev = 0;
    for (int k = 1; k < nranks; ++k) {
        const int64_t target = total * k / nranks;
        int32_t r;
        if (row_ptr) {
            r = (int32_t)(std::lower_bound(row_ptr, row_ptr + V + 1, (int32_t)(row_ptr[0] + target)) - row_ptr);
        } else {
            r = (int32_t)target;
        }
        r = (r + 16) / 32 * 32;  // nearest tile boundary
        if (r < prev) r = prev;
        if (r > V) r = V;
        row_starts[k] = r;
        prev = r;
    }
    row_starts[nranks] = V;
    return PC_OK;
}

// The halo of a rank from the remote columns its rows reference (host arrays, any order,
// repeats allowed): the sorted distinct columns, and how many of them each rank owns.
// PC_ERR_ARG when a column is outside [0, V) or owned by `rank` itself.
extern "C" pc_status pc_dist_halo(int32_t nranks, const int32_t *row_starts, int32_t rank, int64_t n_remote,
                                  const int32_t *remote, int32_t *halo, int64_t *n_halo, int64_t *counts)
{
    if (nranks < 1 || !row_starts || rank < 0 || rank >= nranks || n_remote < 0 || (n_remote > 0 && !remote) ||
        !n_halo || !counts || (n_remote > 0 && !halo))
        return PC_ERR_ARG;
    const int32_t V = row_starts[nranks];
    std::vector<int32_t> h(remote, remote + n_remote);
    std::sort(h.begin(), h.end());
    h.erase(std::unique(h.begin(), h.end()), h.end());
    for (int k = 0; k < nranks; ++k) counts[k] = 0;
    for (int32_t c : h) {
        if (c < 0 || c >= V || (c >= row_starts[rank] && c < row_starts[rank + 1])) return PC_ERR_ARG;
        const int owner = (int)(std::upper_bound(row_starts, row_starts + nranks + 1, c) - row_starts) - 1;
        counts[owner] += 1;
    }
    for (size_t i = 0; i < h.size(); ++i) halo[i] = h[i];
    *n_halo = (int64_t)h.size();
    return PC_OK;
}

// ------------------------------------------------------------------------- plan kernels

// Per local row: own and halo block counts; remote columns appended to `remote` (order
// irrelevant: they are sorted on the host). Column range errors set PC_DERR_INDEX.
__global__ void ds_classify_kernel(int n_own, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                   int32_t b0, int32_t b1, int32_t V, int32_t row0, int32_t row1, int32_t *own_cnt,
                                   int32_t *halo_cnt, int32_t *remote, int64_t remote_cap, uint32_t *counter,
                                   uint32_t *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_own) return;
    const int k0 = rp[i], k1 = rp[i + 1];
    int no = 0, nh = 0;
    if (k0 < b0 || k1 < k0 || k1 > b1) {  // a row outside the rank's block range: not read
        pc_set_err(err, PC_DERR_INDEX);
    } else {
        for (int k = k0; k < k1; ++k) {
            const int c = ci[k];
            if (c < 0 || c >= V) {
                pc_set_err(err, PC_DERR_INDEX);
            } else if (c >= row0 && c < row1) {
                ++no;
            } else {
                ++nh;
                const uint32_t pos = atomicAdd(counter, 1u);
                if ((int64_t)pos < remote_cap) remote[pos] = c;
                else pc_set_err(err, PC_DERR_CAPACITY);
            }
        }
    }
    own_cnt[i] = no;
    halo_cnt[i] = nh;
}

// Exclusive scan of n counts into out[0..n] by one block (plan time only).
__global__ void ds_scan_kernel(int n, const int32_t *__restrict__ cnt, int32_t *out)
{
    __shared__ int64_t s_part[1024];
    const int T = blockDim.x, t = threadIdx.x;
    const int per = (n + T - 1) / T;
    const int a = min(n, t * per), b = min(n, a + per);
    int64_t sum = 0;
    for (int i = a; i < b; ++i) sum += cnt[i];
    s_part[t] = sum;
    __syncthreads();
    if (t == 0) {
        int64_t acc = 0;
        for (int k = 0; k < T; ++k) {
            const int64_t v = s_part[k];
            s_part[k] = acc;
            acc += v;
        }
        out[n] = (int32_t)acc;
    }
    __syncthreads();
    int64_t acc = s_part[t];
    for (int i = a; i < b; ++i) {
        out[i] = (int32_t)acc;
        acc += cnt[i];
    }
}

// Split the rank's rows into the own part (columns renumbered to local rows) and the halo
// part (columns renumbered to n_own + position in the sorted halo list), and record where
// each local block goes (values are split the same way at every solve).
__global__ void ds_split_kernel(int n_own, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                int32_t row0, int32_t row1, const int32_t *__restrict__ own_rp,
                                const int32_t *__restrict__ halo_rp, const int32_t *__restrict__ halo_cols,
                                int32_t n_halo, int32_t *own_ci, int32_t *halo_ci, int32_t *blk_dst, uint32_t *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_own) return;
    const int base = rp[0];
    int po = own_rp[i], ph = halo_rp[i];
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        const int c = ci[k];
        if (c >= row0 && c < row1) {
            own_ci[po] = c - row0;
            blk_dst[k - base] = po;
            ++po;
        } else {
            int lo = 0, hi = n_halo;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (halo_cols[mid] < c) lo = mid + 1;
                else hi = mid;
            }
            if (lo >= n_halo || halo_cols[lo] != c) {
                pc_set_err(err, PC_DERR_INDEX);
                lo = 0;
            }
            halo_ci[ph] = n_own + lo;
            blk_dst[k - base] = -ph - 1;
            ++ph;
        }
    }
}

// Requested global rows -> local rows to send (range checked).
__global__ void ds_requests_kernel(int64_t n, const int32_t *__restrict__ req, int32_t row0, int32_t row1,
                                   int32_t *send_idx, uint32_t *err)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = req[i];
    if (c < row0 || c >= row1) {
        pc_set_err(err, PC_DERR_INDEX);
        send_idx[i] = 0;
    } else {
        send_idx[i] = c - row0;
    }
}

// ------------------------------------------------------------------------- solve kernels

__global__ void ds_split_vals_kernel(int64_t nnzb, const float *__restrict__ vals, const int32_t *__restrict__ dst,
                                     float *own_vals, float *halo_vals)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nnzb) return;
    const int d = dst[k];
    float *o = d >= 0 ? own_vals + 9ll * d : halo_vals + 9ll * (-d - 1);
#pragma unroll
    for (int e = 0; e < 9; ++e) o[e] = vals[9 * k + e];
}

// Scalar Jacobi inverse of the rank's rows (the diagonal block is an own block).
__global__ void ds_dinv_kernel(int n_own, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                               const float *__restrict__ vals, float *dinv, uint32_t *err)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_own) return;
    int s = -1;
    for (int k = rp[i]; k < rp[i + 1]; ++k)
        if (ci[k] == i) { s = k; break; }
    bool ok = s >= 0;
    for (int a = 0; a < 3; ++a) {
        const double d = ok ? (double)vals[9ll * s + 4 * a] : 0.0;
        ok = ok && d > 0.0 && isfinite(d);
        dinv[3ll * i + a] = ok ? (float)(1.0 / d) : 1.f;
    }
    if (!ok) pc_set_err(err, PC_DERR_NONFINITE);
}

__global__ void ds_pack4_kernel(int64_t n, const int32_t *__restrict__ idx, const float4 *__restrict__ p4,
                                float4 *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = p4[idx[i]];
}
__global__ void ds_pack64_kernel(int64_t n, const int32_t *__restrict__ idx, const double *__restrict__ x,
                                 double *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = idx[i];
    out[3 * i] = x[3ll * r];
    out[3 * i + 1] = x[3ll * r + 1];
    out[3 * i + 2] = x[3ll * r + 2];
}

// Block-reduce n values and store the block's sums at part[blockIdx * stride + k].
__device__ __forceinline__ void ds_store_partials(double *v, int n, double *part, int stride)
{
    block_sum_d(v, n);
    if (threadIdx.x == 0)
        for (int k = 0; k < n; ++k) part[(int64_t)blockIdx.x * stride + k] = v[k];
}

// q_i += sum over the halo blocks of row i of A_ij (p_j - p_i) (difference form) or
// A_ij p_j; partial p.(delta q) per block.
template <bool DIFF>
__global__ void __launch_bounds__(DS_THREADS) ds_halo_kernel(int n_own, const int32_t *__restrict__ hrp,
                                                             const int32_t *__restrict__ hci,
                                                             const float *__restrict__ hvals,
                                                             const float4 *__restrict__ p_ext, float4 *q4,
                                                             double *hpart, const pc_scalars *sc)
{
    if (sc->done) return;
    double pq = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_own; i += gridDim.x * blockDim.x) {
        const int k0 = hrp[i], k1 = hrp[i + 1];
        if (k0 == k1) continue;
        const float4 pi = p_ext[i];
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        for (int k = k0; k < k1; ++k) {
            float4 u = p_ext[hci[k]];
            if (DIFF) { u.x -= pi.x; u.y -= pi.y; u.z -= pi.z; }
            spmv_fma(hvals + 9ll * k, u, a0, a1, a2);
        }
        float4 q = q4[i];
        q.x += a0;
        q.y += a1;
        q.z += a2;
        q4[i] = q;
        pq += (double)fmaf(pi.x, a0, fmaf(pi.y, a1, pi.z * a2));
    }
    double v[1] = {pq};
    ds_store_partials(v, 1, hpart, 1);
}

// red[slot] = sum of n partials (stride apart) + sum of m extra partials, in a fixed order.
// With `pair` the n partials are double-float pairs (float2 in the 8-byte slot; the
// product kernel's p.q partials), else doubles.
__global__ void ds_sum_kernel(int n, const double *__restrict__ part, int stride, int m,
                              const double *__restrict__ extra, double *red, int slot, int pair)
{
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (pair) {
            const float2 w = reinterpret_cast<const float2 *>(part)[(int64_t)i * stride];
            v[0] += pc_df_value(w.x, w.y);
        } else {
            v[0] += part[(int64_t)i * stride];
        }
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) v[0] += extra[i];
    block_sum_d(v, 1);
    if (threadIdx.x == 0) red[slot] = v[0];
}

// p = z + beta p (beta from the scalars; p = z after a start, where beta = 0).
__global__ void ds_direction_kernel(int n_own, const float4 *__restrict__ z4, float4 *p4, const pc_scalars *sc)
{
    if (sc->done) return;
    const float beta = (float)sc->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_own; i += gridDim.x * blockDim.x) {
        const float4 z = z4[i], p = p4[i];
        p4[i] = make_float4(fmaf(beta, p.x, z.x), fmaf(beta, p.y, z.y), fmaf(beta, p.z, z.z), 0.f);
    }
}

// alpha = r.z / p.q with p.q the all-reduced red[0]; x += alpha p, r -= alpha q,
// z = D^-1 r; partial (r.z, r.r) per block.
__global__ void __launch_bounds__(DS_THREADS) ds_update_kernel(int n_own, float *x, const float4 *__restrict__ p4,
                                                               float *r, const float4 *__restrict__ q4,
                                                               const float *__restrict__ dinv, float4 *z4,
                                                               const double *red, double *part, pc_scalars *sc)
{
    if (sc->done) return;
    const double pq = red[0];
    double al = sc->rz / pq;
    if (!(pq > 0.0) || !isfinite(al)) al = 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->pq = pq;
        sc->alpha = al;
    }
    const float alpha = (float)al;
    double rz = 0.0, rr = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_own; i += gridDim.x * blockDim.x) {
        const float4 p = p4[i], q = q4[i];
        float *xi = x + 3ll * i, *ri = r + 3ll * i;
        const float *di = dinv + 3ll * i;
        const float r0 = fmaf(-alpha, q.x, ri[0]), r1 = fmaf(-alpha, q.y, ri[1]), r2 = fmaf(-alpha, q.z, ri[2]);
        xi[0] = fmaf(alpha, p.x, xi[0]);
        xi[1] = fmaf(alpha, p.y, xi[1]);
        xi[2] = fmaf(alpha, p.z, xi[2]);
        ri[0] = r0;
        ri[1] = r1;
        ri[2] = r2;
        const float4 z = make_float4(di[0] * r0, di[1] * r1, di[2] * r2, 0.f);
        z4[i] = z;
        rz += (double)fmaf(r0, z.x, fmaf(r1, z.y, r2 * z.z));
        rr += (double)fmaf(r0, r0, fmaf(r1, r1, r2 * r2));
    }
    double v[2] = {rz, rr};
    ds_store_partials(v, 2, part, RED_SLOTS);
}

// After the all-reduce of (r.z, r.r) into red[1], red[2]: beta, the iteration count and
// the stop tests (one thread).
__global__ void ds_finish_kernel(const double *red, pc_scalars *sc)
{
    if (sc->done) return;
    const double rz_new = red[1], rr = red[2];
    const double beta = rz_new / sc->rz;
    sc->beta = beta;
    sc->rz = rz_new;
    sc->rr = rr;
    sc->iter += 1;
    if (!(sc->pq > 0.0) || !isfinite(sc->alpha) || !isfinite(rr) || !isfinite(beta)) {
        sc->status = PC_ERR_NONFINITE;
        sc->done = 1;
    } else if (rr <= sc->tol2) {
        sc->status = PC_OK;
        sc->done = 1;
    } else if (sc->iter >= sc->max_iter) {
        sc->status = PC_ERR_NOT_CONVERGED;
        sc->done = 1;
    }
}

// FP64 residual r64 = b - A x64 of the rank's rows (x64 holds the own rows then the
// halo); r = (float) r64, z = D^-1 r; partial (r.z, r64.r64, b.b) per block. With
// `replace` the FP32 vectors are overwritten (residual replacement / start).
template <bool DIFF>
__global__ void __launch_bounds__(DS_THREADS) ds_residual64_kernel(
    int n_own, const int32_t *__restrict__ orp, const int32_t *__restrict__ oci, const float *__restrict__ ovals,
    const int32_t *__restrict__ hrp, const int32_t *__restrict__ hci, const float *__restrict__ hvals,
    const float *__restrict__ dres, const float *__restrict__ b, const double *__restrict__ x64,
    const float *__restrict__ dinv, float *r, float4 *z4, int replace, double *part)
{
    double rz = 0.0, rr = 0.0, bb = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_own; i += gridDim.x * blockDim.x) {
        const double xi[3] = {x64[3ll * i], x64[3ll * i + 1], x64[3ll * i + 2]};
        double acc[3] = {0.0, 0.0, 0.0};
        for (int part_k = 0; part_k < 2; ++part_k) {
            const int32_t *rp = part_k ? hrp : orp;
            const int32_t *ci = part_k ? hci : oci;
            const float *vals = part_k ? hvals : ovals;
            for (int k = rp[i]; k < rp[i + 1]; ++k) {
                const int c = ci[k];
                double xc[3] = {x64[3ll * c], x64[3ll * c + 1], x64[3ll * c + 2]};
                if (DIFF) {
                    if (c == i) continue;
                    for (int d = 0; d < 3; ++d) xc[d] -= xi[d];
                }
                const float *B = vals + 9ll * k;
                for (int a = 0; a < 3; ++a)
                    acc[a] += (double)B[3 * a] * xc[0] + (double)B[3 * a + 1] * xc[1] + (double)B[3 * a + 2] * xc[2];
            }
        }
        if (DIFF) {
            const float *D = dres + 9ll * i;
            for (int a = 0; a < 3; ++a)
                acc[a] += (double)D[3 * a] * xi[0] + (double)D[3 * a + 1] * xi[1] + (double)D[3 * a + 2] * xi[2];
        }
        float rf[3];
        for (int a = 0; a < 3; ++a) {
            const double bv = (double)b[3ll * i + a], rv = bv - acc[a];
            rr += rv * rv;
            bb += bv * bv;
            rf[a] = (float)rv;
        }
        if (replace) {
            const float *di = dinv + 3ll * i;
            const float4 z = make_float4(di[0] * rf[0], di[1] * rf[1], di[2] * rf[2], 0.f);
            r[3ll * i] = rf[0];
            r[3ll * i + 1] = rf[1];
            r[3ll * i + 2] = rf[2];
            z4[i] = z;
            rz += (double)fmaf(rf[0], z.x, fmaf(rf[1], z.y, rf[2] * z.z));
        }
    }
    double v[3] = {rz, rr, bb};
    ds_store_partials(v, 3, part, RED_SLOTS);
}

// Install the all-reduced (r.z, r.r, b.b) of a start or residual replacement (red[1..3]).
__global__ void ds_install_kernel(const double *red, pc_scalars *sc, int first, double tol, int max_iter)
{
    sc->rz = red[1];
    sc->rr = red[2];
    if (first) {
        sc->bb = red[3];
        sc->tol2 = tol * tol * red[3];
        sc->alpha = sc->beta = sc->pq = 0.0;
        sc->iter = 0;
        sc->max_iter = max_iter;
    }
    sc->status = PC_OK;
    sc->done = 0;
    if (!isfinite(red[2]) || !isfinite(red[3])) {
        sc->status = PC_ERR_NONFINITE;
        sc->done = 1;
    } else if (red[2] <= sc->tol2) {
        sc->done = 1;
    } else if (sc->iter >= sc->max_iter) {
        sc->status = PC_ERR_NOT_CONVERGED;
        sc->done = 1;
    }
}

// x64 (own rows) += x; x = 0. With `to_dv`, dv = (float) x64 as well.
__global__ void ds_fold_kernel(int n_own, float *x, double *x64, float *dv, int to_dv)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n_own; i += gridDim.x * blockDim.x) {
        x64[i] += (double)x[i];
        x[i] = 0.f;
        if (to_dv) dv[i] = (float)x64[i];
    }
}
__global__ void ds_load_kernel(int n, const float *dv, double *x64, float *x)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += gridDim.x * blockDim.x) {
        x64[i] = (double)dv[i];
        x[i] = 0.f;
    }
}
__global__ void ds_zero4_kernel(int n, float4 *a)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        a[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ------------------------------------------------------------------------- host side

extern "C" pc_status pc_dist_destroy(pc_dist *d)
{
    if (!d) return PC_OK;
    cudaFree(d->own_rp); cudaFree(d->own_ci); cudaFree(d->halo_rp); cudaFree(d->halo_ci);
    cudaFree(d->own_cnt); cudaFree(d->halo_cnt); cudaFree(d->blk_dst); cudaFree(d->halo_cols);
    cudaFree(d->remote); cudaFree(d->req); cudaFree(d->send_idx); cudaFree(d->cnt_send); cudaFree(d->cnt_recv);
    cudaFree(d->counter); cudaFree(d->own_vals); cudaFree(d->halo_vals); cudaFree(d->p_ext); cudaFree(d->q4);
    cudaFree(d->z4); cudaFree(d->send4); cudaFree(d->x); cudaFree(d->r); cudaFree(d->dinv); cudaFree(d->x64);
    cudaFree(d->send64); cudaFree(d->partials); cudaFree(d->hpart); cudaFree(d->red); cudaFree(d->sc);
    cudaFree(d->err);
    cudaFreeHost(d->sc_host); cudaFreeHost(d->h_err); cudaFreeHost(d->h_tmp);
    if (d->ev_pack) cudaEventDestroy(d->ev_pack);
    if (d->ev_halo) cudaEventDestroy(d->ev_halo);
    if (d->s1) cudaStreamDestroy(d->s1);
    delete d;
    return PC_OK;
}

static pc_status ds_alloc(pc_dist *d)
{
    const int64_t n = d->n_own, H = d->halo_cap, C = d->cap;
    PC_CUDA_TRY(cudaMalloc(&d->own_rp, sizeof(int32_t) * (n + 1)));
    PC_CUDA_TRY(cudaMalloc(&d->halo_rp, sizeof(int32_t) * (n + 1)));
    PC_CUDA_TRY(cudaMalloc(&d->own_cnt, sizeof(int32_t) * (n + 1)));
    PC_CUDA_TRY(cudaMalloc(&d->halo_cnt, sizeof(int32_t) * (n + 1)));
    PC_CUDA_TRY(cudaMalloc(&d->own_ci, sizeof(int32_t) * (C + 4)));
    PC_CUDA_TRY(cudaMalloc(&d->halo_ci, sizeof(int32_t) * (C + 4)));
    PC_CUDA_TRY(cudaMemset(d->own_ci, 0, sizeof(int32_t) * (C + 4)));
    PC_CUDA_TRY(cudaMalloc(&d->blk_dst, sizeof(int32_t) * (C + 4)));
    PC_CUDA_TRY(cudaMalloc(&d->remote, sizeof(int32_t) * (C + 4)));
    PC_CUDA_TRY(cudaMalloc(&d->halo_cols, sizeof(int32_t) * (H + 4)));
    PC_CUDA_TRY(cudaMalloc(&d->req, sizeof(int32_t) * (H + 4)));
    PC_CUDA_TRY(cudaMalloc(&d->send_idx, sizeof(int32_t) * (H + 4)));
    PC_CUDA_TRY(cudaMalloc(&d->cnt_send, sizeof(int64_t) * d->nranks));
    PC_CUDA_TRY(cudaMalloc(&d->cnt_recv, sizeof(int64_t) * d->nranks));
    PC_CUDA_TRY(cudaMalloc(&d->counter, sizeof(uint32_t)));
    PC_CUDA_TRY(cudaMalloc(&d->own_vals, sizeof(float) * (9 * C + 16)));
    PC_CUDA_TRY(cudaMemset(d->own_vals, 0, sizeof(float) * (9 * C + 16)));
    PC_CUDA_TRY(cudaMalloc(&d->halo_vals, sizeof(float) * (9 * C + 16)));
    PC_CUDA_TRY(cudaMalloc(&d->p_ext, sizeof(float4) * (n + H + 1)));
    PC_CUDA_TRY(cudaMemset(d->p_ext, 0, sizeof(float4) * (n + H + 1)));
    PC_CUDA_TRY(cudaMalloc(&d->q4, sizeof(float4) * (n + 1)));
    PC_CUDA_TRY(cudaMalloc(&d->z4, sizeof(float4) * (n + 1)));
    PC_CUDA_TRY(cudaMalloc(&d->send4, sizeof(float4) * (H + 1)));
    PC_CUDA_TRY(cudaMalloc(&d->x, sizeof(float) * 3 * (n + 1)));
    PC_CUDA_TRY(cudaMalloc(&d->r, sizeof(float) * 3 * (n + 1)));
    PC_CUDA_TRY(cudaMalloc(&d->dinv, sizeof(float) * 3 * (n + 1)));
    PC_CUDA_TRY(cudaMalloc(&d->x64, sizeof(double) * 3 * (n + H + 1)));
    PC_CUDA_TRY(cudaMalloc(&d->send64, sizeof(double) * 3 * (H + 1)));
    PC_CUDA_TRY(cudaMalloc(&d->partials, sizeof(double) * RED_SLOTS * DS_MAX_BLOCKS));
    PC_CUDA_TRY(cudaMalloc(&d->hpart, sizeof(double) * DS_MAX_BLOCKS));
    PC_CUDA_TRY(cudaMalloc(&d->red, sizeof(double) * 8));
    PC_CUDA_TRY(cudaMalloc(&d->sc, sizeof(pc_scalars)));
    PC_CUDA_TRY(cudaMemset(d->sc, 0, sizeof(pc_scalars)));
    PC_CUDA_TRY(cudaMalloc(&d->err, sizeof(uint32_t)));
    PC_CUDA_TRY(cudaMallocHost(&d->sc_host, sizeof(pc_scalars)));
    PC_CUDA_TRY(cudaMallocHost(&d->h_err, sizeof(uint32_t)));
    PC_CUDA_TRY(cudaMallocHost(&d->h_tmp, sizeof(int64_t) * 4));
    PC_CUDA_TRY(cudaStreamCreateWithFlags(&d->s1, cudaStreamNonBlocking));
    PC_CUDA_TRY(cudaEventCreateWithFlags(&d->ev_pack, cudaEventDisableTiming));
    PC_CUDA_TRY(cudaEventCreateWithFlags(&d->ev_halo, cudaEventDisableTiming));
    const int w = SpShape<SP_CAPR_WIDE>::smem_bytes;
    PC_CUDA_TRY(cudaFuncSetAttribute(spmv_kernel<true, true, SP_CAPR_WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, w));
    PC_CUDA_TRY(cudaFuncSetAttribute(spmv_kernel<false, true, SP_CAPR_WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, w));
    return PC_OK;
}

extern "C" pc_status pc_dist_create(pc_dist **out, int32_t rank, int32_t nranks, const int32_t *row_starts,
                                    int64_t max_blocks, int64_t max_halo)
{
    if (!out) return PC_ERR_ARG;
    *out = nullptr;
    if (nranks < 1 || rank < 0 || rank >= nranks || !row_starts || row_starts[0] != 0 || max_blocks < 1 ||
        max_halo < 0)
        return PC_ERR_ARG;
    for (int k = 0; k < nranks; ++k)
        if (row_starts[k + 1] < row_starts[k]) return PC_ERR_ARG;
    if (row_starts[rank + 1] - row_starts[rank] < 1) return PC_ERR_ARG;
    pc_dist *d = new pc_dist();
    d->rank = rank;
    d->nranks = nranks;
    d->row_starts.assign(row_starts, row_starts + nranks + 1);
    d->V_global = row_starts[nranks];
    d->row0 = row_starts[rank];
    d->row1 = row_starts[rank + 1];
    d->n_own = d->row1 - d->row0;
    d->cap = (max_blocks + 3) / 4 * 4;
    d->halo_cap = max_halo > 0 ? max_halo : (int64_t)d->V_global - d->n_own + 1;
    d->recv_cnt.assign(nranks, 0);
    d->recv_start.assign(nranks + 1, 0);
    d->send_cnt.assign(nranks, 0);
    d->send_start.assign(nranks + 1, 0);
    pc_status s = PC_OK;
    if (cudaGetDevice(&d->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&d->num_sms, cudaDevAttrMultiProcessorCount, d->device) != cudaSuccess)
        s = PC_ERR_CUDA;
    if (s == PC_OK) s = ds_alloc(d);
    if (s != PC_OK) {
        pc_dist_destroy(d);
        return s;
    }
    *out = d;
    return PC_OK;
}

static pc_status ds_read_err(pc_dist *d, cudaStream_t st, uint32_t *bits)
{
    PC_CUDA_TRY(cudaMemcpyAsync(d->h_err, d->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    *bits = *d->h_err;
    return PC_OK;
}

static pc_status ds_exchange(const pc_comm *comm, const void *send, const std::vector<int64_t> &send_start,
                             const std::vector<int64_t> &send_cnt, void *recv, const std::vector<int64_t> &recv_start,
                             const std::vector<int64_t> &recv_cnt, int64_t elem, int nranks, cudaStream_t st)
{
    std::vector<int64_t> so(nranks), sb(nranks), ro(nranks), rb(nranks);
    for (int j = 0; j < nranks; ++j) {
        so[j] = send_start[j] * elem;
        sb[j] = send_cnt[j] * elem;
        ro[j] = recv_start[j] * elem;
        rb[j] = recv_cnt[j] * elem;
    }
    const int32_t s = comm->exchange(comm->user, send, so.data(), sb.data(), recv, ro.data(), rb.data(), (void *)st);
    return s == 0 ? PC_OK : PC_ERR_CUDA;
}

extern "C" pc_status pc_dist_plan(pc_dist *d, const pc_bsr *A, const pc_comm *comm, void *stream)
{
    if (!d || !A || !A->row_ptr || !A->col_idx || !comm || !comm->exchange || !comm->allreduce_sum) return PC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int n = d->n_own;
    d->planned = 0;
    // the rank's block range [row_ptr[0], row_ptr[n_own])
    PC_CUDA_TRY(cudaMemcpyAsync(d->h_tmp, A->row_ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaMemcpyAsync(reinterpret_cast<int32_t *>(d->h_tmp) + 1, A->row_ptr + n, sizeof(int32_t),
                                cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    const int32_t b0 = reinterpret_cast<int32_t *>(d->h_tmp)[0], b1 = reinterpret_cast<int32_t *>(d->h_tmp)[1];
    if (b0 < 0 || b1 < b0 || (A->nnzb > 0 && b1 > A->nnzb)) return PC_ERR_ARG;
    if ((int64_t)(b1 - b0) > d->cap) return PC_ERR_CAPACITY;
    d->off0 = b0;
    d->nnzb = b1 - b0;
    PC_CUDA_TRY(cudaMemsetAsync(d->err, 0, sizeof(uint32_t), st));
    PC_CUDA_TRY(cudaMemsetAsync(d->counter, 0, sizeof(uint32_t), st));
    DS_LAUNCH(d, ds_classify_kernel, pc_blocks(n, 256), 256, 0, st, n, A->row_ptr, A->col_idx, b0, b1, d->V_global,
              d->row0, d->row1, d->own_cnt, d->halo_cnt, d->remote, d->cap, d->counter, d->err);
    DS_LAUNCH(d, ds_scan_kernel, 1, 1024, 0, st, n, d->own_cnt, d->own_rp);
    DS_LAUNCH(d, ds_scan_kernel, 1, 1024, 0, st, n, d->halo_cnt, d->halo_rp);
    uint32_t bits = 0;
    PC_TRY(ds_read_err(d, st, &bits));
    if (bits & PC_DERR_INDEX) return PC_ERR_ARG;
    if (bits) return PC_ERR_CAPACITY;
    uint32_t n_remote = 0;
    PC_CUDA_TRY(cudaMemcpy(&n_remote, d->counter, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    // the halo: sorted distinct remote columns, grouped by owner
    std::vector<int32_t> remote(n_remote), halo(n_remote + 1);
    if (n_remote)
        PC_CUDA_TRY(cudaMemcpy(remote.data(), d->remote, sizeof(int32_t) * n_remote, cudaMemcpyDeviceToHost));
    int64_t n_halo = 0;
    std::vector<int64_t> cnt(d->nranks, 0);
    PC_TRY(pc_dist_halo(d->nranks, d->row_starts.data(), d->rank, n_remote, remote.data(), halo.data(), &n_halo,
                        cnt.data()));
    if (n_halo > d->halo_cap) return PC_ERR_CAPACITY;
    d->n_halo = n_halo;
    for (int j = 0; j < d->nranks; ++j) {
        d->recv_cnt[j] = cnt[j];
        d->recv_start[j + 1] = d->recv_start[j] + cnt[j];
    }
    if (n_halo) PC_CUDA_TRY(cudaMemcpy(d->halo_cols, halo.data(), sizeof(int32_t) * n_halo, cudaMemcpyHostToDevice));
    // tell each owner how many of its rows this rank needs, then which
    std::vector<int64_t> one(d->nranks), idx(d->nranks + 1);
    for (int j = 0; j <= d->nranks; ++j) idx[j] = j;
    for (int j = 0; j < d->nranks; ++j) one[j] = j == d->rank ? 0 : 1;
    PC_CUDA_TRY(cudaMemcpy(d->cnt_send, d->recv_cnt.data(), sizeof(int64_t) * d->nranks, cudaMemcpyHostToDevice));
    PC_CUDA_TRY(cudaMemset(d->cnt_recv, 0, sizeof(int64_t) * d->nranks));
    PC_TRY(ds_exchange(comm, d->cnt_send, idx, one, d->cnt_recv, idx, one, sizeof(int64_t), d->nranks, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int64_t> want(d->nranks);
    PC_CUDA_TRY(cudaMemcpy(want.data(), d->cnt_recv, sizeof(int64_t) * d->nranks, cudaMemcpyDeviceToHost));
    int64_t n_send = 0;
    for (int j = 0; j < d->nranks; ++j) {
        if (j == d->rank) want[j] = 0;
        if (want[j] < 0) return PC_ERR_ARG;
        d->send_cnt[j] = want[j];
        d->send_start[j] = n_send;
        n_send += want[j];
    }
    d->send_start[d->nranks] = n_send;
    if (n_send > d->halo_cap) return PC_ERR_CAPACITY;
    d->n_send = n_send;
    // requests: this rank sends its halo segment for owner j to j and receives the rows j wants
    PC_TRY(ds_exchange(comm, d->halo_cols, d->recv_start, d->recv_cnt, d->req, d->send_start, d->send_cnt,
                       sizeof(int32_t), d->nranks, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    if (n_send)
        DS_LAUNCH(d, ds_requests_kernel, pc_blocks(n_send, 256), 256, 0, st, n_send, d->req, d->row0, d->row1,
                  d->send_idx, d->err);
    DS_LAUNCH(d, ds_split_kernel, pc_blocks(n, 256), 256, 0, st, n, A->row_ptr, A->col_idx, d->row0, d->row1,
              d->own_rp, d->halo_rp, d->halo_cols, (int32_t)n_halo, d->own_ci, d->halo_ci, d->blk_dst, d->err);
    PC_TRY(ds_read_err(d, st, &bits));
    if (bits) return PC_ERR_ARG;
    PC_CUDA_TRY(cudaMemcpy(d->h_tmp, d->own_rp + n, sizeof(int32_t), cudaMemcpyDeviceToHost));
    d->nnzb_own = reinterpret_cast<int32_t *>(d->h_tmp)[0];
    d->nnzb_halo = d->nnzb - d->nnzb_own;
    d->planned = 1;
    return PC_OK;
}

extern "C" pc_status pc_dist_sizes(const pc_dist *d, int32_t *row0, int32_t *row1, int64_t *n_halo, int64_t *n_send,
                                   int64_t *nnzb_own, int64_t *nnzb_halo)
{
    if (!d) return PC_ERR_ARG;
    if (row0) *row0 = d->row0;
    if (row1) *row1 = d->row1;
    if (n_halo) *n_halo = d->n_halo;
    if (n_send) *n_send = d->n_send;
    if (nnzb_own) *nnzb_own = d->nnzb_own;
    if (nnzb_halo) *nnzb_halo = d->nnzb_halo;
    return PC_OK;
}

// All-reduce `n` doubles of d->red starting at `slot` through the caller's communicator.
static pc_status ds_allreduce(pc_dist *d, const pc_comm *comm, int slot, int n, cudaStream_t st)
{
    return comm->allreduce_sum(comm->user, d->red + slot, n, (void *)st) == 0 ? PC_OK : PC_ERR_CUDA;
}

// The FP64 residual of the accumulated solution: fold, exchange the FP64 halo, residual
// kernel, all-reduce (r.z, r.r, b.b) into red[1..3].
static pc_status ds_residual(pc_dist *d, const pc_comm *comm, const float *dres, const float *b, int replace,
                             cudaStream_t st)
{
    const int n = d->n_own;
    if (d->n_send)
        DS_LAUNCH(d, ds_pack64_kernel, pc_blocks(d->n_send, 256), 256, 0, st, d->n_send, d->send_idx, d->x64,
                  d->send64);
    PC_TRY(ds_exchange(comm, d->send64, d->send_start, d->send_cnt, d->x64 + 3ll * n, d->recv_start, d->recv_cnt,
                       3 * sizeof(double), d->nranks, st));
    const unsigned g = ds_grid(d, n);
    if (dres)
        DS_LAUNCH(d, ds_residual64_kernel<true>, g, DS_THREADS, 0, st, n, d->own_rp, d->own_ci, d->own_vals,
                  d->halo_rp, d->halo_ci, d->halo_vals, dres, b, d->x64, d->dinv, d->r, d->z4, replace, d->partials);
    else
        DS_LAUNCH(d, ds_residual64_kernel<false>, g, DS_THREADS, 0, st, n, d->own_rp, d->own_ci, d->own_vals,
                  d->halo_rp, d->halo_ci, d->halo_vals, dres, b, d->x64, d->dinv, d->r, d->z4, replace, d->partials);
    for (int k = 0; k < 3; ++k)
        DS_LAUNCH(d, ds_sum_kernel, 1, 256, 0, st, (int)g, d->partials + k, RED_SLOTS, 0, (const double *)nullptr,
                  d->red, 1 + k, 0);
    return ds_allreduce(d, comm, 1, 3, st);
}

static pc_status ds_read_scalars(pc_dist *d, cudaStream_t st)
{
    PC_CUDA_TRY(cudaMemcpyAsync(d->sc_host, d->sc, sizeof(pc_scalars), cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    return PC_OK;
}

// One PCG iteration of the rank (direction, halo exchange overlapped with the own-part
// product, halo part, alpha, update, beta and the stop tests).
static pc_status ds_iteration(pc_dist *d, const pc_comm *comm, const float *dres, cudaStream_t st)
{
    const int n = d->n_own;
    const unsigned g = ds_grid(d, n);
    DS_LAUNCH(d, ds_direction_kernel, g, DS_THREADS, 0, st, n, (const float4 *)d->z4, d->p_ext, (const pc_scalars *)d->sc);
    if (d->n_send)
        DS_LAUNCH(d, ds_pack4_kernel, pc_blocks(d->n_send, 256), 256, 0, st, d->n_send, d->send_idx,
                  (const float4 *)d->p_ext, d->send4);
    PC_CUDA_TRY(cudaEventRecord(d->ev_pack, st));
    // own part first: it runs while the halo travels on the second stream
    SpmvArgs a{};
    a.V = n;
    a.rp = d->own_rp;
    a.ci = d->own_ci;
    a.vals = d->own_vals;
    a.dres = dres;
    a.dsc = nullptr;
    a.x4 = d->p_ext;
    a.y4 = d->q4;
    a.partials = d->partials;
    a.sc = d->sc;
    a.err = d->err;
    const int tiles = (n + SP_ROWS - 1) / SP_ROWS;
    const int gs = std::max(1, std::min(tiles, d->num_sms * SpShape<SP_CAPR_WIDE>::ctas_per_sm));
    const int w = SpShape<SP_CAPR_WIDE>::smem_bytes;
    if (dres) DS_LAUNCH(d, (spmv_kernel<true, true, SP_CAPR_WIDE>), gs, SP_THREADS, w, st, a);
    else DS_LAUNCH(d, (spmv_kernel<false, true, SP_CAPR_WIDE>), gs, SP_THREADS, w, st, a);
    PC_CUDA_TRY(cudaStreamWaitEvent(d->s1, d->ev_pack, 0));
    PC_TRY(ds_exchange(comm, d->send4, d->send_start, d->send_cnt, d->p_ext + n, d->recv_start, d->recv_cnt,
                       sizeof(float4), d->nranks, d->s1));
    PC_CUDA_TRY(cudaEventRecord(d->ev_halo, d->s1));
    PC_CUDA_TRY(cudaStreamWaitEvent(st, d->ev_halo, 0));
    if (dres)
        DS_LAUNCH(d, ds_halo_kernel<true>, g, DS_THREADS, 0, st, n, d->halo_rp, d->halo_ci, d->halo_vals,
                  (const float4 *)d->p_ext, d->q4, d->hpart, (const pc_scalars *)d->sc);
    else
        DS_LAUNCH(d, ds_halo_kernel<false>, g, DS_THREADS, 0, st, n, d->halo_rp, d->halo_ci, d->halo_vals,
                  (const float4 *)d->p_ext, d->q4, d->hpart, (const pc_scalars *)d->sc);
    DS_LAUNCH(d, ds_sum_kernel, 1, 256, 0, st, gs, d->partials + 3, RED_SLOTS, (int)g, (const double *)d->hpart,
              d->red, 0, 1);
    PC_TRY(ds_allreduce(d, comm, 0, 1, st));
    DS_LAUNCH(d, ds_update_kernel, g, DS_THREADS, 0, st, n, d->x, (const float4 *)d->p_ext, d->r,
              (const float4 *)d->q4, d->dinv, d->z4, (const double *)d->red, d->partials, d->sc);
    DS_LAUNCH(d, ds_sum_kernel, 1, 256, 0, st, (int)g, d->partials, RED_SLOTS, 0, (const double *)nullptr, d->red, 1,
              0);
    DS_LAUNCH(d, ds_sum_kernel, 1, 256, 0, st, (int)g, d->partials + 1, RED_SLOTS, 0, (const double *)nullptr, d->red,
              2, 0);
    PC_TRY(ds_allreduce(d, comm, 1, 2, st));
    DS_LAUNCH(d, ds_finish_kernel, 1, 1, 0, st, (const double *)d->red, d->sc);
    return PC_OK;
}

extern "C" pc_status pc_dist_pcg_solve(pc_dist *d, const float *vals, const float *dres, const float *b, float *dv,
                                       const pc_solve_opts *opts, const pc_comm *comm, pc_solve_info *info,
                                       void *stream)
{
    if (!d || !vals || !b || !dv || !comm || !comm->exchange || !comm->allreduce_sum) return PC_ERR_ARG;
    if (!d->planned) return PC_ERR_ARG;
    pc_solve_opts o;
    pc_default_solve_opts(&o);
    if (opts) o = *opts;
    if (!(o.tol > 0.0) || o.max_iter < 0 || (o.precision != PC_PREC_FP32 && o.precision != PC_PREC_MIXED) ||
        o.precond != PC_PRECOND_JACOBI || !(o.refresh > 0.0 && o.refresh < 1.0))
        return PC_ERR_ARG;
    if (o.check_every < 1) o.check_every = 32;
    if (o.refresh_every < 1) o.refresh_every = 1000;
    const bool mixed = o.precision == PC_PREC_MIXED;
    cudaStream_t st = (cudaStream_t)stream;
    const int n = d->n_own;
    const unsigned g = ds_grid(d, n);
    PC_CUDA_TRY(cudaMemsetAsync(d->err, 0, sizeof(uint32_t), st));
    PC_CUDA_TRY(cudaMemsetAsync(d->sc, 0, sizeof(pc_scalars), st));
    if (d->nnzb)
        DS_LAUNCH(d, ds_split_vals_kernel, pc_blocks(d->nnzb, 256), 256, 0, st, d->nnzb, vals + 9 * d->off0,
                  d->blk_dst, d->own_vals, d->halo_vals);
    DS_LAUNCH(d, ds_dinv_kernel, pc_blocks(n, 256), 256, 0, st, n, d->own_rp, d->own_ci, d->own_vals, d->dinv,
              d->err);
    uint32_t bits = 0;
    PC_TRY(ds_read_err(d, st, &bits));
    // a singular diagonal on any rank stops every rank: agree through the all-reduce
    {
        double flag = bits ? 1.0 : 0.0;
        PC_CUDA_TRY(cudaMemcpyAsync(d->red + 4, &flag, sizeof(double), cudaMemcpyHostToDevice, st));
        PC_TRY(ds_allreduce(d, comm, 4, 1, st));
        PC_CUDA_TRY(cudaMemcpyAsync(&flag, d->red + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
        PC_CUDA_TRY(cudaStreamSynchronize(st));
        if (flag != 0.0) return PC_ERR_NONFINITE;
    }
    // start: x64 = dv, x = 0, FP64 residual, p = 0 (the first direction is z)
    DS_LAUNCH(d, ds_load_kernel, g, DS_THREADS, 0, st, n, dv, d->x64, d->x);
    DS_LAUNCH(d, ds_zero4_kernel, g, DS_THREADS, 0, st, n, d->p_ext);
    PC_TRY(ds_residual(d, comm, dres, b, 1, st));
    DS_LAUNCH(d, ds_install_kernel, 1, 1, 0, st, (const double *)d->red, d->sc, 1, o.tol, o.max_iter);
    PC_TRY(ds_read_scalars(d, st));
    double rr_last = d->sc_host->rr;
    int iter_last = 0, replacements = 0, launched = 0;
    for (;;) {
        const pc_scalars h = *d->sc_host;
        if (h.done) {
            // mixed: a converged recurrence residual is confirmed by an FP64 replacement
            if (mixed && h.status == PC_OK && h.iter > iter_last) {
                DS_LAUNCH(d, ds_fold_kernel, g, DS_THREADS, 0, st, n, d->x, d->x64, dv, 0);
                PC_TRY(ds_residual(d, comm, dres, b, 1, st));
                DS_LAUNCH(d, ds_install_kernel, 1, 1, 0, st, (const double *)d->red, d->sc, 0, o.tol, o.max_iter);
                ++replacements;
                PC_TRY(ds_read_scalars(d, st));
                rr_last = d->sc_host->rr;
                iter_last = d->sc_host->iter;
                continue;
            }
            break;
        }
        if (launched >= o.max_iter + o.check_every) break;
        if (mixed && h.iter > iter_last &&
            (h.rr <= rr_last * o.refresh * o.refresh || h.iter - iter_last >= o.refresh_every)) {
            DS_LAUNCH(d, ds_fold_kernel, g, DS_THREADS, 0, st, n, d->x, d->x64, dv, 0);
            PC_TRY(ds_residual(d, comm, dres, b, 1, st));
            DS_LAUNCH(d, ds_install_kernel, 1, 1, 0, st, (const double *)d->red, d->sc, 0, o.tol, o.max_iter);
            ++replacements;
            PC_TRY(ds_read_scalars(d, st));
            rr_last = d->sc_host->rr;
            iter_last = d->sc_host->iter;
            continue;
        }
        // mixed: the FP32 increment goes into the FP64 accumulator at every check (its
        // rounding stays far below what a residual replacement measures)
        if (mixed && launched > 0) DS_LAUNCH(d, ds_fold_kernel, g, DS_THREADS, 0, st, n, d->x, d->x64, dv, 0);
        for (int k = 0; k < o.check_every; ++k) PC_TRY(ds_iteration(d, comm, dres, st));
        launched += o.check_every;
        PC_TRY(ds_read_scalars(d, st));
        // a failure only this rank saw (a timed-out wait) stops every rank: the ranks must
        // keep making the same collective calls
        double flag = d->sc_host->status == PC_ERR_TIMEOUT ? 1.0 : 0.0;
        PC_CUDA_TRY(cudaMemcpyAsync(d->red + 4, &flag, sizeof(double), cudaMemcpyHostToDevice, st));
        PC_TRY(ds_allreduce(d, comm, 4, 1, st));
        PC_CUDA_TRY(cudaMemcpyAsync(&flag, d->red + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
        PC_CUDA_TRY(cudaStreamSynchronize(st));
        if (flag != 0.0) return PC_ERR_TIMEOUT;
    }
    const pc_scalars fin = *d->sc_host;
    // the solution: fold what the iterations built, then its FP64 residual (reported)
    DS_LAUNCH(d, ds_fold_kernel, g, DS_THREADS, 0, st, n, d->x, d->x64, dv, 1);
    PC_TRY(ds_residual(d, comm, dres, b, 0, st));
    double sums[4];
    PC_CUDA_TRY(cudaMemcpyAsync(sums, d->red, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    PC_TRY(ds_read_err(d, st, &bits));
    if (bits & PC_DERR_TIMEOUT) return PC_ERR_TIMEOUT;
    if (info) {
        info->iters = fin.iter;
        info->outer = mixed ? replacements : 0;
        info->bnorm = sqrt(sums[3]);
        info->rel_res = sums[3] > 0 ? sqrt(sums[2] / sums[3]) : 0.0;
    }
    return (pc_status)fin.status;
}
