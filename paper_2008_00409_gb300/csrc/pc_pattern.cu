// Context creation (rest state, hinges, static pattern, element incidence) and the
// per-step dynamic pattern (Sec. 3.2.2: index table of the step's sparse matrix).
//
// The paper fills a per-row index table with atomics, then sorts and compacts each row
// (Sec. 3.2.2 steps 2-3). Here the static mesh pattern is built once by sorting all
// element keys; each step only the contact keys are sorted, deduplicated and merged into
// the static pattern by ranking, so row pointers and column indices are bit-exact.
#include <stdlib.h>
#include <string.h>

#include "pc_internal.cuh"

// ------------------------------------------------------------------------- error plumbing

static char g_last_error[512];

void pc_note_cuda_error(cudaError_t e, const char *what, const char *file, int line)
{
    snprintf(g_last_error, sizeof(g_last_error), "%s:%d %s: %s", file, line, what, cudaGetErrorString(e));
    if (getenv("PCLOTH_VERBOSE")) fprintf(stderr, "pcloth: %s\n", g_last_error);
}

extern "C" PC_API const char *pc_last_cuda_error(void) { return g_last_error; }

pc_status pc_read_errors(pc_ctx *ctx, cudaStream_t st, uint32_t *bits)
{
    PC_CUDA_TRY(cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    *bits = *ctx->h_err;
    return PC_OK;
}

static pc_status errors_to_status(uint32_t bits)
{
    if (bits & PC_DERR_MESH) return PC_ERR_MESH;
    if (bits & (PC_DERR_INDEX | PC_DERR_PAIR)) return PC_ERR_ARG;
    if (bits & PC_DERR_CAPACITY) return PC_ERR_CAPACITY;
    if (bits & PC_DERR_NONFINITE) return PC_ERR_NONFINITE;
    return PC_OK;
}

// ------------------------------------------------------------------------- rest kernels

__global__ void check_tris_kernel(int T, int V, const int32_t *tri, uint32_t *err)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    int a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
    if (a < 0 || a >= V || b < 0 || b >= V || c < 0 || c >= V) pc_set_err(err, PC_DERR_INDEX);
    else if (a == b || b == c || a == c) pc_set_err(err, PC_DERR_MESH);
}

// Rest edge matrix in the triangle's own plane, its inverse, area and the rest Gram
// matrix of the two edges (as float pairs, computed in FP64 from the FP32 positions).
__global__ void rest_tri_kernel(int T, const int32_t *tri, const float *X, float *dmi, float *area, float *rgram,
                                uint32_t *err)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int32_t *v = tri + 3 * t;
    double e1[3], e2[3];
    for (int a = 0; a < 3; ++a) {
        e1[a] = (double)X[3 * v[1] + a] - (double)X[3 * v[0] + a];
        e2[a] = (double)X[3 * v[2] + a] - (double)X[3 * v[0] + a];
    }
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double ln = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    if (!(ln > 0.0) || !(l1 > 0.0)) {
        pc_set_err(err, PC_DERR_MESH);
        return;
    }
    double u[3], w[3], vv[3];
    for (int a = 0; a < 3; ++a) { u[a] = e1[a] / l1; w[a] = n[a] / ln; }
    vv[0] = w[1] * u[2] - w[2] * u[1];
    vv[1] = w[2] * u[0] - w[0] * u[2];
    vv[2] = w[0] * u[1] - w[1] * u[0];
    double d00 = l1, d01 = e2[0] * u[0] + e2[1] * u[1] + e2[2] * u[2];
    double d11 = e2[0] * vv[0] + e2[1] * vv[1] + e2[2] * vv[2];
    double det = d00 * d11;
    dmi[4 * t + 0] = (float)(d11 / det);
    dmi[4 * t + 1] = (float)(-d01 / det);
    dmi[4 * t + 2] = 0.0f;
    dmi[4 * t + 3] = (float)(d00 / det);
    area[t] = (float)(0.5 * ln);
    double g[3] = {e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2], e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2],
                   e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2]};
    for (int k = 0; k < 3; ++k) {
        float hi = (float)g[k];
        rgram[6 * t + 2 * k] = hi;
        rgram[6 * t + 2 * k + 1] = (float)(g[k] - (double)hi);
    }
}

// half-edge keys: min*V + max, value = 3t + k (edge k runs from vertex k to k+1)
__global__ void half_edge_kernel(int T, int V, const int32_t *tri, uint64_t *keys, uint32_t *vals)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3ll * T) return;
    int t = (int)(i / 3), k = (int)(i % 3);
    uint32_t a = (uint32_t)tri[3 * t + k], b = (uint32_t)tri[3 * t + (k + 1) % 3];
    uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
    keys[i] = (uint64_t)lo * (uint64_t)V + hi;
    vals[i] = (uint32_t)i;
}

__global__ void hinge_flag_kernel(int64_t n, const uint64_t *keys, int32_t *flag, uint32_t *err)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool start = (i == 0) || keys[i] != keys[i - 1];
    int f = 0;
    if (start && i + 1 < n && keys[i + 1] == keys[i]) {
        f = 1;
        if (i + 2 < n && keys[i + 2] == keys[i]) pc_set_err(err, PC_DERR_MESH);
    }
    flag[i] = f;
}

__host__ __device__ inline double hinge_angle_d(const double *x1, const double *x2, const double *x3, const double *x4)
{
    double a[3], b[3], N1[3], N2[3], E[3];
    for (int k = 0; k < 3; ++k) { a[k] = x1[k] - x3[k]; b[k] = x1[k] - x4[k]; }
    N1[0] = a[1] * b[2] - a[2] * b[1]; N1[1] = a[2] * b[0] - a[0] * b[2]; N1[2] = a[0] * b[1] - a[1] * b[0];
    for (int k = 0; k < 3; ++k) { a[k] = x2[k] - x4[k]; b[k] = x2[k] - x3[k]; }
    N2[0] = a[1] * b[2] - a[2] * b[1]; N2[1] = a[2] * b[0] - a[0] * b[2]; N2[2] = a[0] * b[1] - a[1] * b[0];
    for (int k = 0; k < 3; ++k) E[k] = x4[k] - x3[k];
    double ln1 = sqrt(N1[0] * N1[0] + N1[1] * N1[1] + N1[2] * N1[2]);
    double ln2 = sqrt(N2[0] * N2[0] + N2[1] * N2[1] + N2[2] * N2[2]);
    double lE = sqrt(E[0] * E[0] + E[1] * E[1] + E[2] * E[2]);
    double c[3] = {N1[1] * N2[2] - N1[2] * N2[1], N1[2] * N2[0] - N1[0] * N2[2], N1[0] * N2[1] - N1[1] * N2[0]};
    double s = (c[0] * E[0] + c[1] * E[1] + c[2] * E[2]) / (ln1 * ln2 * lE);
    double co = (N1[0] * N2[0] + N1[1] * N2[1] + N1[2] * N2[2]) / (ln1 * ln2);
    return atan2(s, co);
}

// Emit hinge h from the half-edge pair starting at sorted index i. The edge is oriented
// as in the lower-indexed triangle; wing0 is that triangle's third vertex.
__global__ void hinge_emit_kernel(int64_t n, const uint32_t *he_vals, const int32_t *flag, const int32_t *pos,
                                  const int32_t *tri, const float *X, const float *area, float kb, int32_t *hinge,
                                  float *hcoef, float *hrest)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag[i]) return;
    int h = pos[i];
    uint32_t a = he_vals[i], b = he_vals[i + 1];
    int t0 = (int)(a / 3), k0 = (int)(a % 3), t1 = (int)(b / 3), k1 = (int)(b % 3);
    int e0 = tri[3 * t0 + k0], e1 = tri[3 * t0 + (k0 + 1) % 3];
    int w0 = tri[3 * t0 + (k0 + 2) % 3], w1 = tri[3 * t1 + (k1 + 2) % 3];
    hinge[4 * h + 0] = w0;
    hinge[4 * h + 1] = w1;
    hinge[4 * h + 2] = e0;
    hinge[4 * h + 3] = e1;
    double p[4][3];
    int vid[4] = {w0, w1, e0, e1};
    for (int k = 0; k < 4; ++k)
        for (int c = 0; c < 3; ++c) p[k][c] = (double)X[3 * vid[k] + c];
    double el2 = 0.0;
    for (int c = 0; c < 3; ++c) el2 += (p[3][c] - p[2][c]) * (p[3][c] - p[2][c]);
    double ch = 3.0 * el2 / ((double)area[t0] + (double)area[t1]);
    hcoef[h] = (float)(2.0 * (double)kb * ch);
    hrest[h] = (float)hinge_angle_d(p[0], p[1], p[2], p[3]);
}

// incidence keys: vertex of each (element, local vertex); values = element refs
__global__ void incidence_kernel(int T, int H, const int32_t *tri, const int32_t *hinge, uint64_t *keys,
                                 uint32_t *vals)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t nt = 3ll * T;
    if (i < nt) {
        int t = (int)(i / 3), k = (int)(i % 3);
        keys[i] = (uint64_t)tri[3 * t + k];
        vals[i] = pc_ref(PC_REF_TRI, k, t);
    } else if (i < nt + 4ll * H) {
        int64_t j = i - nt;
        int h = (int)(j / 4), k = (int)(j % 4);
        keys[i] = (uint64_t)hinge[4 * h + k];
        vals[i] = pc_ref(PC_REF_HINGE, k, h);
    }
}

// ptr[r] = first index of sorted keys with key >= r (r = 0..V)
__global__ void segment_ptr_kernel(int V, const uint64_t *keys, int64_t n, int32_t *ptr)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > V) return;
    ptr[r] = (int32_t)pc_lower_bound_u64(keys, n, (uint64_t)r);
}

__global__ void mass_kernel(int V, const int32_t *vinc_ptr, const uint32_t *vinc, const float *area, float rho,
                            float *mass)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= V) return;
    double m = 0.0;
    for (int i = vinc_ptr[r]; i < vinc_ptr[r + 1]; ++i) {
        uint32_t ref = vinc[i];
        if (pc_ref_type(ref) == PC_REF_TRI) m += (double)rho * (double)area[pc_ref_id(ref)] / 3.0;
    }
    mass[r] = (float)m;
}

__global__ void pins_kernel(int n, int V, const int32_t *pins, uint8_t *pinned, uint32_t *err)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p = pins[i];
    if (p < 0 || p >= V) pc_set_err(err, PC_DERR_INDEX);
    else pinned[p] = 1;
}

// static pattern keys: diagonal, 3x3 per triangle, the two wing pairs of each hinge
__global__ void static_keys_kernel(int V, int T, int H, const int32_t *tri, const int32_t *hinge, uint64_t *keys)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t VV = (uint64_t)V;
    if (i < V) {
        keys[i] = (uint64_t)i * VV + (uint64_t)i;
        return;
    }
    i -= V;
    if (i < 9ll * T) {
        int t = (int)(i / 9), kl = (int)(i % 9);
        keys[V + 9ll * t + kl] = (uint64_t)tri[3 * t + kl / 3] * VV + (uint64_t)tri[3 * t + kl % 3];
        return;
    }
    i -= 9ll * T;
    if (i < 2ll * H) {
        int h = (int)(i / 2), k = (int)(i % 2);
        uint64_t a = (uint64_t)hinge[4 * h + k], b = (uint64_t)hinge[4 * h + 1 - k];
        keys[V + 9ll * T + i] = a * VV + b;
    }
}

// ordered vertex pairs (a, b), a != b, of every triangle: key a * V + b (6 per triangle)
__global__ void edge_keys_kernel(int T, int V, const int32_t *tri, uint64_t *keys)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6ll * T) return;
    const int t = (int)(i / 6), k = (int)(i % 6);
    const int a = k >> 1, b = (a + 1 + (k & 1)) % 3;  // (0,1) (0,2) (1,2) (1,0) (2,0) (2,1)
    keys[i] = (uint64_t)tri[3 * t + a] * (uint64_t)V + (uint64_t)tri[3 * t + b];
}

__global__ void unique_flag_kernel(int64_t n, const uint64_t *keys, int32_t *flag)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void compact_cols_kernel(int64_t n, const uint64_t *keys, const int32_t *flag, const int32_t *pos, int V,
                                    int32_t *cols, uint64_t *ukeys)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag[i]) return;
    int32_t p = pos[i];
    if (cols) cols[p] = (int32_t)(keys[i] % (uint64_t)V);
    if (ukeys) ukeys[p] = keys[i];
}

// row_ptr[r] = first unique key with row >= r
__global__ void rowptr_from_keys_kernel(int V, const uint64_t *ukeys, int64_t n, int32_t *rp)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > V) return;
    rp[r] = (int32_t)pc_lower_bound_u64(ukeys, n, (uint64_t)r * (uint64_t)V);
}

// Mean rest length of each vertex's mesh edges (0 for an isolated vertex), in FP64.
__global__ void rest_len_kernel(int V, const int32_t *__restrict__ erp, const int32_t *__restrict__ ecol,
                                const float *__restrict__ rest, float *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= V) return;
    double s = 0.0;
    const int e0 = erp[i], e1 = erp[i + 1];
    for (int e = e0; e < e1; ++e) {
        const int j = ecol[e];
        double d2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double d = (double)rest[3ll * j + a] - (double)rest[3ll * i + a];
            d2 += d * d;
        }
        s += sqrt(d2);
    }
    out[i] = e1 > e0 ? (float)(s / (double)(e1 - e0)) : 0.f;
}

// ------------------------------------------------------------------------- context

static void free_ctx(pc_ctx *c)
{
    if (!c) return;
    pc_batched_free(c);
    pc_mlp_ctx_free(c);
    void *ptrs[] = {c->tri, c->rest, c->tri_dmi, c->tri_area, c->tri_rgram, c->mass, c->pinned, c->hinge, c->hcoef,
                    c->hrest, c->srp, c->scol, c->erp, c->ecol, c->rest_len, c->vinc_ptr, c->vinc, c->dkeys, c->dnew, c->dflag, c->dscan, c->ckeys,
                    c->cinc, c->cinc_ptr, c->tri_buf, c->hinge_buf, c->cont_buf, c->r, c->z, c->p0, c->p1, c->q,
                    c->dinv, c->dtmp, c->rhs32, c->x64, c->r64, c->partials, c->sc, c->A_rp, c->A_ci, c->A_vals, c->A_dres,
                    c->A_b, c->A_dv, c->h_state, c->h_pairs, c->h_w, c->sort.keys_alt, c->sort.vals_alt, c->sort.hist,
                    c->d_err, c->d_count, c->scan_tmp, c->sym_urp, c->sym_lrp, c->sym_dpos, c->sym_ucnt, c->sym_lcnt,
                    c->sym_uci, c->sym_lcol, c->sym_lsrc, c->sym_uvals, c->sell_perm, c->sell_width,
                    c->sell_base, c->sell_dpos, c->sell_data, c->sell_diag, c->od_rp, c->od_cnt, c->od_dpos,
                    c->od_ci, c->od_vals, c->px_keys, c->px_vals, c->px_cnt, c->px_off, c->px_vcnt, c->px_voff,
                    c->px_max, c->dsc, c->fbar};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->sc_host) cudaFreeHost(c->sc_host);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->h_count) cudaFreeHost(c->h_count);
    for (int i = 0; i < c->ev_used; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    delete c;
}

template <typename T>
static pc_status dalloc(T **p, int64_t n)
{
    if (n < 1) n = 1;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (size_t)n);
    if (e != cudaSuccess) {
        pc_note_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
        *p = nullptr;
        return PC_ERR_CUDA;
    }
    return PC_OK;
}

static pc_status create_impl(pc_ctx *c, const int32_t *tris, const float *rest, const int32_t *pins, cudaStream_t st)
{
    const int V = c->V, T = c->T;
    PC_CUDA_TRY(cudaGetDevice(&c->device));
    PC_CUDA_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
    PC_TRY(dalloc(&c->d_err, 1));
    PC_TRY(dalloc(&c->d_count, 4));
    PC_CUDA_TRY(cudaMallocHost(&c->h_err, sizeof(uint32_t)));
    PC_CUDA_TRY(cudaMallocHost(&c->h_count, 4 * sizeof(int64_t)));
    PC_CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(uint32_t), st));
    PC_TRY(dalloc(&c->tri, 3ll * T));
    PC_TRY(dalloc(&c->rest, 3ll * V));
    PC_TRY(dalloc(&c->tri_dmi, 4ll * T));
    PC_TRY(dalloc(&c->tri_area, T));
    PC_TRY(dalloc(&c->tri_rgram, 6ll * T));
    PC_TRY(dalloc(&c->mass, V));
    PC_TRY(dalloc(&c->pinned, V));
    if (T > 0) PC_CUDA_TRY(cudaMemcpyAsync(c->tri, tris, sizeof(int32_t) * 3 * (size_t)T, cudaMemcpyDeviceToDevice, st));
    PC_CUDA_TRY(cudaMemcpyAsync(c->rest, rest, sizeof(float) * 3 * (size_t)V, cudaMemcpyDeviceToDevice, st));
    PC_CUDA_TRY(cudaMemsetAsync(c->pinned, 0, V, st));

    // sort scratch for the largest static sort: pattern keys V + 9T + 2H (H <= 1.5T)
    int64_t n_static_keys = (int64_t)V + 9ll * T + 3ll * T;
    int64_t n_inc = 3ll * T + 6ll * T;
    int64_t n_sort = n_static_keys > n_inc ? n_static_keys : n_inc;
    int64_t n_dyn = 6ll * c->max_contacts;
    if (n_dyn > n_sort) n_sort = n_dyn;
    PC_TRY(pc_sort_reserve(c, n_sort + 1));

    uint64_t *keys = nullptr;
    uint32_t *vals = nullptr;
    int32_t *flag = nullptr, *pos = nullptr;
    PC_TRY(dalloc(&keys, n_sort + 1));
    pc_status s = PC_OK;
    do {
        if ((s = dalloc(&vals, n_sort + 1)) != PC_OK) break;
        if ((s = dalloc(&flag, n_sort + 1)) != PC_OK) break;
        if ((s = dalloc(&pos, n_sort + 2)) != PC_OK) break;

        if (T > 0) {
            check_tris_kernel<<<pc_blocks(T, 256), 256, 0, st>>>(T, V, c->tri, c->d_err);
            c->launches++;
        }
        uint32_t bits = 0;
        if ((s = pc_read_errors(c, st, &bits)) != PC_OK) break;
        if (bits) { s = errors_to_status(bits); break; }
        if (T > 0) {
            rest_tri_kernel<<<pc_blocks(T, 128), 128, 0, st>>>(T, c->tri, c->rest, c->tri_dmi, c->tri_area,
                                                               c->tri_rgram, c->d_err);
            c->launches++;
        }
        if (c->n_pins > 0) {
            pins_kernel<<<pc_blocks(c->n_pins, 256), 256, 0, st>>>(c->n_pins, V, pins, c->pinned, c->d_err);
            c->launches++;
        }
        // hinges
        int64_t nhe = 3ll * T;
        int vbits = pc_bits_for((int64_t)V);
        if (nhe > 0) {
            half_edge_kernel<<<pc_blocks(nhe, 256), 256, 0, st>>>(T, V, c->tri, keys, vals);
            c->launches++;
            if ((s = pc_radix_sort(c, keys, vals, nhe, 2 * vbits, st)) != PC_OK) break;
            hinge_flag_kernel<<<pc_blocks(nhe, 256), 256, 0, st>>>(nhe, keys, flag, c->d_err);
            c->launches++;
            if ((s = pc_exclusive_scan(c, flag, pos, nhe, st)) != PC_OK) break;
            PC_CUDA_TRY(cudaMemcpyAsync(c->h_count, pos + nhe, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            PC_CUDA_TRY(cudaStreamSynchronize(st));
            c->H = *(int32_t *)c->h_count;
        } else {
            c->H = 0;
        }
        if ((s = pc_read_errors(c, st, &bits)) != PC_OK) break;
        if (bits) { s = errors_to_status(bits); break; }
        const int H = c->H;
        if ((s = dalloc(&c->hinge, 4ll * H)) != PC_OK) break;
        if ((s = dalloc(&c->hcoef, H)) != PC_OK) break;
        if ((s = dalloc(&c->hrest, H)) != PC_OK) break;
        if (H > 0) {
            hinge_emit_kernel<<<pc_blocks(nhe, 256), 256, 0, st>>>(nhe, vals, flag, pos, c->tri, c->rest, c->tri_area,
                                                                   c->mat.k_bend, c->hinge, c->hcoef, c->hrest);
            c->launches++;
        }
        // element incidence, grouped by vertex (triangles by id, then hinges by id)
        int64_t ninc = 3ll * T + 4ll * H;
        if ((s = dalloc(&c->vinc, ninc)) != PC_OK) break;
        if ((s = dalloc(&c->vinc_ptr, V + 1ll)) != PC_OK) break;
        if (ninc > 0) {
            incidence_kernel<<<pc_blocks(ninc, 256), 256, 0, st>>>(T, H, c->tri, c->hinge, keys, vals);
            c->launches++;
            if ((s = pc_radix_sort(c, keys, vals, ninc, vbits, st)) != PC_OK) break;
            PC_CUDA_TRY(cudaMemcpyAsync(c->vinc, vals, sizeof(uint32_t) * ninc, cudaMemcpyDeviceToDevice, st));
        }
        segment_ptr_kernel<<<pc_blocks(V + 1ll, 256), 256, 0, st>>>(V, keys, ninc, c->vinc_ptr);
        c->launches++;
        mass_kernel<<<pc_blocks(V, 256), 256, 0, st>>>(V, c->vinc_ptr, c->vinc, c->tri_area, c->mat.rho, c->mass);
        c->launches++;
        // static pattern
        int64_t nkeys = (int64_t)V + 9ll * T + 2ll * H;
        static_keys_kernel<<<pc_blocks(nkeys, 256), 256, 0, st>>>(V, T, H, c->tri, c->hinge, keys);
        c->launches++;
        int kbits = pc_bits_for((int64_t)V * (int64_t)V);
        if ((s = pc_radix_sort(c, keys, nullptr, nkeys, kbits, st)) != PC_OK) break;
        unique_flag_kernel<<<pc_blocks(nkeys, 256), 256, 0, st>>>(nkeys, keys, flag);
        c->launches++;
        if ((s = pc_exclusive_scan(c, flag, pos, nkeys, st)) != PC_OK) break;
        PC_CUDA_TRY(cudaMemcpyAsync(c->h_count, pos + nkeys, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        PC_CUDA_TRY(cudaStreamSynchronize(st));
        c->snnz = *(int32_t *)c->h_count;
        if ((s = dalloc(&c->scol, c->snnz)) != PC_OK) break;
        if ((s = dalloc(&c->srp, V + 1ll)) != PC_OK) break;
        uint64_t *ukeys = c->sort.keys_alt;  // free after the sort
        compact_cols_kernel<<<pc_blocks(nkeys, 256), 256, 0, st>>>(nkeys, keys, flag, pos, V, c->scol, ukeys);
        c->launches++;
        rowptr_from_keys_kernel<<<pc_blocks(V + 1ll, 256), 256, 0, st>>>(V, ukeys, c->snnz, c->srp);
        c->launches++;
        // edge one-rings (mesh edge neighbours of each vertex, sorted): the neighbourhood
        // of the learned warm start's features
        const int64_t nek = 6ll * T;
        if ((s = dalloc(&c->erp, V + 1ll)) != PC_OK) break;
        if (nek > 0) {
            edge_keys_kernel<<<pc_blocks(nek, 256), 256, 0, st>>>(T, V, c->tri, keys);
            c->launches++;
            if ((s = pc_radix_sort(c, keys, nullptr, nek, kbits, st)) != PC_OK) break;
            unique_flag_kernel<<<pc_blocks(nek, 256), 256, 0, st>>>(nek, keys, flag);
            c->launches++;
            if ((s = pc_exclusive_scan(c, flag, pos, nek, st)) != PC_OK) break;
            PC_CUDA_TRY(cudaMemcpyAsync(c->h_count, pos + nek, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            PC_CUDA_TRY(cudaStreamSynchronize(st));
            c->enn = *(int32_t *)c->h_count;
        } else {
            c->enn = 0;
        }
        if ((s = dalloc(&c->ecol, c->enn)) != PC_OK) break;
        if (nek > 0) {
            compact_cols_kernel<<<pc_blocks(nek, 256), 256, 0, st>>>(nek, keys, flag, pos, V, c->ecol, ukeys);
            c->launches++;
        }
        rowptr_from_keys_kernel<<<pc_blocks(V + 1ll, 256), 256, 0, st>>>(V, ukeys, c->enn, c->erp);
        c->launches++;
        // each vertex's mean rest edge length (the learned warm start's length scale)
        if ((s = dalloc(&c->rest_len, V)) != PC_OK) break;
        rest_len_kernel<<<pc_blocks(V, 256), 256, 0, st>>>(V, c->erp, c->ecol, c->rest, c->rest_len);
        c->launches++;
        if ((s = pc_read_errors(c, st, &bits)) != PC_OK) break;
        if (bits) { s = errors_to_status(bits); break; }
    } while (0);
    cudaFree(keys);
    cudaFree(vals);
    cudaFree(flag);
    cudaFree(pos);
    if (s != PC_OK) return s;

    // per-step buffers
    const int64_t P = c->max_contacts;
    PC_TRY(dalloc(&c->dkeys, 6 * P + 1));
    PC_TRY(dalloc(&c->dnew, 6 * P + 1));
    PC_TRY(dalloc(&c->dflag, 6 * P + 2));
    PC_TRY(dalloc(&c->dscan, 6 * P + 2));
    PC_TRY(dalloc(&c->ckeys, 4 * P + 1));
    PC_TRY(dalloc(&c->cinc, 4 * P + 1));
    PC_TRY(dalloc(&c->cinc_ptr, V + 1ll));
    PC_TRY(dalloc(&c->tri_buf, (int64_t)PC_TRI_STRIDE * T));
    PC_TRY(dalloc(&c->hinge_buf, (int64_t)PC_HINGE_STRIDE * c->H));
    PC_TRY(dalloc(&c->cont_buf, (int64_t)PC_CONTACT_STRIDE * P));
    PC_TRY(dalloc(&c->h_pairs, 4 * P));
    PC_TRY(dalloc(&c->h_w, 3 * P));
    PC_TRY(dalloc(&c->h_state, 6ll * V));
    // context-owned step system
    c->A_cap = ((c->snnz + 6 * P) + 3) / 4 * 4;
    PC_TRY(dalloc(&c->A_rp, V + 1ll));
    PC_TRY(dalloc(&c->A_ci, c->A_cap));
    PC_TRY(dalloc(&c->A_vals, 9 * c->A_cap));
    PC_TRY(dalloc(&c->A_dres, 9ll * V));
    PC_TRY(dalloc(&c->A_b, 3ll * V));
    PC_TRY(dalloc(&c->A_dv, 3ll * V));
    PC_CUDA_TRY(cudaMemsetAsync(c->A_dv, 0, sizeof(float) * 3 * (size_t)V, st));
    PC_TRY(pc_solver_alloc(c));
    PC_TRY(pc_batched_alloc(c));
    PC_TRY(pc_proximity_alloc(c));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    return PC_OK;
}

extern "C" pc_status pc_create(pc_ctx **out, int32_t V, int32_t T, const int32_t *tris, const float *rest,
                               const int32_t *pins, int32_t n_pins, const pc_material *mat, int32_t max_contacts,
                               void *stream)
{
    if (!out) return PC_ERR_ARG;
    *out = nullptr;
    if (V < 1 || T < 0 || n_pins < 0 || max_contacts < 0 || !mat || !rest || (T > 0 && !tris) ||
        (n_pins > 0 && !pins))
        return PC_ERR_ARG;
    if (3ll * T >= (1ll << 28) || (int64_t)V * (int64_t)V >= (1ll << 62) || 6ll * max_contacts >= (1ll << 30))
        return PC_ERR_ARG;
    if (!(mat->rho > 0.0f) || !(mat->young > 0.0f) || !(mat->poisson > -1.0f && mat->poisson < 0.5f) ||
        mat->k_bend < 0.0f || mat->k_contact < 0.0f || !(mat->damp_mass >= 0.0f && mat->damp_mass < 1e30f) ||
        !(mat->damp_stiff >= 0.0f && mat->damp_stiff < 1e30f) ||
        !(mat->contact_thickness >= 0.0f && mat->contact_thickness < 1e30f))
        return PC_ERR_ARG;
    pc_ctx *c = new pc_ctx();
    c->V = V;
    c->T = T;
    c->n_pins = n_pins;
    c->max_contacts = max_contacts;
    c->mat = *mat;
    c->mu = mat->young / (2.0f * (1.0f + mat->poisson));
    c->lam = mat->young * mat->poisson / (1.0f - mat->poisson * mat->poisson);
    cudaStream_t st = (cudaStream_t)stream;
    pc_status s = create_impl(c, tris, rest, pins, st);
    if (s != PC_OK) {
        cudaStreamSynchronize(st);
        free_ctx(c);
        return s;
    }
    *out = c;
    return PC_OK;
}

extern "C" pc_status pc_destroy(pc_ctx *ctx)
{
    if (!ctx) return PC_OK;
    cudaDeviceSynchronize();
    free_ctx(ctx);
    return PC_OK;
}

extern "C" pc_status pc_get_sizes(const pc_ctx *ctx, int32_t *V, int32_t *T, int32_t *H, int64_t *static_nnzb)
{
    if (!ctx) return PC_ERR_ARG;
    if (V) *V = ctx->V;
    if (T) *T = ctx->T;
    if (H) *H = ctx->H;
    if (static_nnzb) *static_nnzb = ctx->snnz;
    return PC_OK;
}

extern "C" pc_status pc_get_rest(const pc_ctx *ctx, int32_t *hinges, float *mass, void *stream)
{
    if (!ctx) return PC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (hinges && ctx->H > 0)
        PC_CUDA_TRY(cudaMemcpyAsync(hinges, ctx->hinge, sizeof(int32_t) * 4 * (size_t)ctx->H, cudaMemcpyDeviceToDevice, st));
    if (mass) PC_CUDA_TRY(cudaMemcpyAsync(mass, ctx->mass, sizeof(float) * (size_t)ctx->V, cudaMemcpyDeviceToDevice, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    return PC_OK;
}

// ------------------------------------------------------------------------- per-step pattern

// 6 dynamic pattern keys and 4 incidence entries per contact pair; validates the pair.
__global__ void contact_keys_kernel(int P, int V, const int32_t *pairs, uint64_t *dkeys, uint64_t *ckeys,
                                    uint32_t *cinc, uint32_t *err)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    int v[4];
    bool bad = false;
    for (int k = 0; k < 4; ++k) {
        v[k] = pairs[4 * i + k];
        if (v[k] < 0 || v[k] >= V) bad = true;
    }
    if (bad) {
        pc_set_err(err, PC_DERR_INDEX);
        for (int k = 0; k < 4; ++k) v[k] = 0;
    } else if (v[0] == v[1] || v[0] == v[2] || v[0] == v[3] || v[1] == v[2] || v[1] == v[3] || v[2] == v[3]) {
        pc_set_err(err, PC_DERR_PAIR);
    }
    uint64_t VV = (uint64_t)V, p = (uint64_t)v[0];
    for (int k = 1; k < 4; ++k) {
        uint64_t a = (uint64_t)v[k];
        dkeys[6ll * i + 2 * (k - 1)] = p * VV + a;
        dkeys[6ll * i + 2 * (k - 1) + 1] = a * VV + p;
    }
    for (int k = 0; k < 4; ++k) {
        ckeys[4ll * i + k] = (uint64_t)v[k];
        cinc[4ll * i + k] = pc_ref(PC_REF_CONTACT, k, i);
    }
}

// flag sorted dynamic keys that are first of their run and absent from the static pattern
__global__ void dyn_new_flag_kernel(int64_t n, const uint64_t *keys, int V, const int32_t *srp, const int32_t *scol,
                                    int32_t *flag)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = keys[i];
    int f = 0;
    if (i == 0 || keys[i - 1] != k) {
        int r = (int)(k / (uint64_t)V), c = (int)(k % (uint64_t)V);
        int lo = srp[r], hi = srp[r + 1];
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            if (scol[mid] < c) lo = mid + 1; else hi = mid;
        }
        f = (lo < srp[r + 1] && scol[lo] == c) ? 0 : 1;
    }
    flag[i] = f;
}

__global__ void dyn_compact_kernel(int64_t n, const uint64_t *keys, const int32_t *flag, const int32_t *pos,
                                   uint64_t *dnew)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag[i]) return;
    dnew[pos[i]] = keys[i];
}

// row_ptr[r] = static row_ptr[r] + number of new keys in rows < r
__global__ void dyn_rowptr_kernel(int V, const int32_t *srp, const uint64_t *dnew, const int32_t *n_new_ptr,
                                  int32_t *rp)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > V) return;
    int64_t nn = *n_new_ptr;
    rp[r] = srp[r] + (int32_t)pc_lower_bound_u64(dnew, nn, (uint64_t)r * (uint64_t)V);
}

// merge each row's static columns with its new columns (both ascending)
__global__ void dyn_cols_kernel(int V, const int32_t *srp, const int32_t *scol, const uint64_t *dnew,
                                const int32_t *rp, int64_t cap, int32_t *col, uint32_t *err)
{
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= V) return;
    int s = srp[r], se = srp[r + 1];
    int o = rp[r];
    int nn_row = rp[r + 1] - o - (se - s);
    int d = rp[r] - srp[r];  // new keys in rows < r = index of this row's first new key
    int de = d + nn_row;
    if ((int64_t)rp[r + 1] > cap) {
        pc_set_err(err, PC_DERR_CAPACITY);
        return;
    }
    uint64_t VV = (uint64_t)V;
    while (s < se || d < de) {
        int cs = s < se ? scol[s] : 0x7FFFFFFF;
        int cd = d < de ? (int)(dnew[d] % VV) : 0x7FFFFFFF;
        if (cs < cd) { col[o++] = cs; ++s; } else { col[o++] = cd; ++d; }
    }
}

extern "C" pc_status pc_assemble_pattern(pc_ctx *ctx, const pc_contacts *contacts, pc_bsr *A, void *stream)
{
    if (!ctx || !A || !A->row_ptr || !A->col_idx) return PC_ERR_ARG;
    if ((A->cap & 3) != 0 || !pc_aligned16(A->col_idx)) return PC_ERR_ARG;
    int32_t P = contacts ? contacts->n : 0;
    if (P < 0 || P > ctx->max_contacts || (P > 0 && (!contacts->pairs || !contacts->w))) return PC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int V = ctx->V;
    PC_CUDA_TRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), st));
    int64_t nd = 6ll * P, nc = 4ll * P;
    if (P > 0) {
        PC_LAUNCH(ctx, contact_keys_kernel, pc_blocks(P, 256), 256, 0, st, P, V, contacts->pairs, ctx->dkeys,
                  ctx->ckeys, ctx->cinc, ctx->d_err);
        PC_TRY(pc_radix_sort(ctx, ctx->dkeys, nullptr, nd, pc_bits_for((int64_t)V * V), st));
        PC_TRY(pc_radix_sort(ctx, ctx->ckeys, ctx->cinc, nc, pc_bits_for(V), st));
        PC_LAUNCH(ctx, dyn_new_flag_kernel, pc_blocks(nd, 256), 256, 0, st, nd, ctx->dkeys, V, ctx->srp, ctx->scol,
                  ctx->dflag);
        PC_TRY(pc_exclusive_scan(ctx, ctx->dflag, ctx->dscan, nd, st));
        PC_LAUNCH(ctx, dyn_compact_kernel, pc_blocks(nd, 256), 256, 0, st, nd, ctx->dkeys, ctx->dflag, ctx->dscan,
                  ctx->dnew);
    } else {
        PC_CUDA_TRY(cudaMemsetAsync(ctx->dscan, 0, sizeof(int32_t), st));
    }
    PC_LAUNCH(ctx, dyn_rowptr_kernel, pc_blocks(V + 1ll, 256), 256, 0, st, V, ctx->srp, ctx->dnew, ctx->dscan + nd,
              A->row_ptr);
    PC_LAUNCH(ctx, segment_ptr_kernel, pc_blocks(V + 1ll, 256), 256, 0, st, V, ctx->ckeys, nc, ctx->cinc_ptr);
    PC_LAUNCH(ctx, dyn_cols_kernel, pc_blocks(V, 128), 128, 0, st, V, ctx->srp, ctx->scol, ctx->dnew, A->row_ptr,
              A->cap, A->col_idx, ctx->d_err);
    PC_CUDA_TRY(cudaMemcpyAsync(ctx->h_count, ctx->dscan + nd, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    uint32_t bits = 0;
    PC_TRY(pc_read_errors(ctx, st, &bits));
    ctx->n_new = *(int32_t *)ctx->h_count;
    A->nnzb = ctx->snnz + ctx->n_new;
    ctx->n_contacts = P;
    ctx->last_pairs = P > 0 ? contacts->pairs : nullptr;
    if (bits & (PC_DERR_INDEX | PC_DERR_PAIR)) return PC_ERR_ARG;
    if (A->nnzb > A->cap) return PC_ERR_CAPACITY;
    return errors_to_status(bits);
}
