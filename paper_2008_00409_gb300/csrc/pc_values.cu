// Value assembly (Sec. 3.2.2 "value filling", Eq. 2-3): element kernels evaluate every
// assembly element once (force and Hessian at x_t) into per-element records, and the
// right-hand side is Eq. 3's h f(x_t + h v_t) to first order, b = h (f(x_t) - h K v_t);
// a warp per matrix row then gathers the records of the elements incident to that row
// and reduces them into the row's blocks in a fixed order. No atomics: the result is
// deterministic and the matrix is bitwise symmetric.
//
// Precision: the membrane strain G = (F^T F - I)/2 cancels catastrophically in FP32 at
// cloth strains (1e-5..1e-3). It is formed instead as Dm^-T (Ds^T Ds - Dm^T Dm) Dm^-1 with
// the Gram difference of the current and rest edges evaluated in double-float (pairs of
// FP32 values, exact TwoSum / fma-based TwoProduct), so the strain keeps FP32 relative
// accuracy; everything else is plain FP32.
#include "pc_internal.cuh"

// ------------------------------------------------------------------------- double-float

struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ dfl quick_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b)
{
    dfl s = two_sum(a.hi, b.hi);
    float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return quick_two_sum(s.hi, lo);
}
__device__ __forceinline__ dfl df_mul(dfl a, dfl b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}
__device__ __forceinline__ dfl df_dot3(const dfl *a, const dfl *b)
{
    return df_add(df_add(df_mul(a[0], b[0]), df_mul(a[1], b[1])), df_mul(a[2], b[2]));
}

// ------------------------------------------------------------------------- small helpers

__device__ __forceinline__ float3 ld3(const float *p, int i) { return make_float3(p[3 * i], p[3 * i + 1], p[3 * i + 2]); }
__device__ __forceinline__ float3 sub(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 add(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 mul(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b)
{
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// upper-triangular block index of (k, l), k <= l, in a 3-vertex element
__device__ __forceinline__ int tri_blk(int k, int l) { return k == 0 ? l : (k == 1 ? 2 + l : 5); }

// Positive part of a symmetric 2x2 matrix [a b; b c].
__device__ __forceinline__ void sym2_positive(float a, float b, float c, float &pa, float &pb, float &pc)
{
    float m = 0.5f * (a + c);
    float r = sqrtf(0.25f * (a - c) * (a - c) + b * b);
    float l1 = m + r, l2 = m - r;
    if (l2 >= 0.0f) { pa = a; pb = b; pc = c; return; }
    if (l1 <= 0.0f) { pa = pb = pc = 0.0f; return; }
    float v0, v1;
    if (fabsf(b) > 0.0f) {
        if (fabsf(l1 - a) > fabsf(l1 - c)) { v0 = b; v1 = l1 - a; } else { v0 = l1 - c; v1 = b; }
    } else if (a >= c) { v0 = 1.0f; v1 = 0.0f; } else { v0 = 0.0f; v1 = 1.0f; }
    float inv = rsqrtf(v0 * v0 + v1 * v1);
    v0 *= inv;
    v1 *= inv;
    pa = l1 * v0 * v0;
    pb = l1 * v0 * v1;
    pc = l1 * v1 * v1;
}

// ------------------------------------------------------------------------- membrane triangles

// Green strain G = Dm^-T (Gram(edges) - Gram(rest)) Dm^-1 / 2 from exact edge pairs.
__device__ __forceinline__ void strain_from_edges(const dfl *e1, const dfl *e2, const float *rg, const float *dmi,
                                                  float &G00, float &G01, float &G11)
{
    dfl g11 = df_dot3(e1, e1), g22 = df_dot3(e2, e2), g12 = df_dot3(e1, e2);
    float D11 = df_add(g11, {-rg[0], -rg[1]}).hi;
    float D22 = df_add(g22, {-rg[2], -rg[3]}).hi;
    float D12 = df_add(g12, {-rg[4], -rg[5]}).hi;
    // G = 1/2 Dm^-T D Dm^-1 with Dm^-1 = [[d0 d1] [d2 d3]]
    float d0 = dmi[0], d1 = dmi[1], d2 = dmi[2], d3 = dmi[3];
    // M = D Dm^-1
    float m00 = D11 * d0 + D12 * d2, m01 = D11 * d1 + D12 * d3;
    float m10 = D12 * d0 + D22 * d2, m11 = D12 * d1 + D22 * d3;
    G00 = 0.5f * (d0 * m00 + d2 * m10);
    G01 = 0.5f * (d0 * m01 + d2 * m11);
    G11 = 0.5f * (d1 * m01 + d3 * m11);
}

// One thread per triangle, everything at x_t. Record: right-hand-side contributions
// c_k = h f_k - sum_l (h^2 H_kl) v_l for k = 0, 1, 2 (the element's share of
// b = h (f - h K v), the first-order form of h f(x_t + h v_t), Eq. 2-3), then the h^2
// Hessian blocks (0,0) (0,1) (0,2) (1,1) (1,2) (2,2), each 3x3 row-major. Since each
// Hessian row sums to zero, sum_l H_kl v_l is formed as sum_l H_kl (v_l - v_k).
__global__ void __launch_bounds__(128) tri_eval_kernel(int T, const int32_t *__restrict__ tri,
                                                       const float *__restrict__ x, const float *__restrict__ v,
                                                       const float *__restrict__ dmi_all,
                                                       const float *__restrict__ area, const float *__restrict__ rgram,
                                                       float mu, float lam, float h, float hk,
                                                       float *__restrict__ out)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    int i0 = tri[3 * t], i1 = tri[3 * t + 1], i2 = tri[3 * t + 2];
    float dmi[4] = {dmi_all[4 * t], dmi_all[4 * t + 1], dmi_all[4 * t + 2], dmi_all[4 * t + 3]};
    float rg[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) rg[k] = rgram[6 * t + k];
    const float A0 = area[t];
    float x0[3], x1[3], x2[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        x0[a] = x[3 * i0 + a]; x1[a] = x[3 * i1 + a]; x2[a] = x[3 * i2 + a];
    }
    dfl e1[3], e2[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        e1[a] = two_sum(x1[a], -x0[a]);
        e2[a] = two_sum(x2[a], -x0[a]);
    }
    // shape-function gradients: g1 = row 0 of Dm^-1, g2 = row 1, g0 = -g1 - g2
    float g[3][2] = {{-dmi[0] - dmi[2], -dmi[1] - dmi[3]}, {dmi[0], dmi[1]}, {dmi[2], dmi[3]}};
    float G00, G01, G11;
    strain_from_edges(e1, e2, rg, dmi, G00, G01, G11);
    const float tr = G00 + G11;
    const float S00 = 2.0f * mu * G00 + lam * tr, S01 = 2.0f * mu * G01, S11 = 2.0f * mu * G11 + lam * tr;
    float F[3][2];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        F[a][0] = e1[a].hi * dmi[0] + e2[a].hi * dmi[2];
        F[a][1] = e1[a].hi * dmi[1] + e2[a].hi * dmi[3];
    }
    float f[3][3];  // forces at x_t
    {
        float P[3][2];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            P[a][0] = F[a][0] * S00 + F[a][1] * S01;
            P[a][1] = F[a][0] * S01 + F[a][1] * S11;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            f[1][a] = -A0 * (P[a][0] * g[1][0] + P[a][1] * g[1][1]);
            f[2][a] = -A0 * (P[a][0] * g[2][0] + P[a][1] * g[2][1]);
            f[0][a] = -(f[1][a] + f[2][a]);
        }
    }
    // ---- Hessian at x_t (stress clamped to its positive part in the geometric term)
    {
        float Sp00, Sp01, Sp11;
        sym2_positive(S00, S01, S11, Sp00, Sp01, Sp11);
        float Fg[3][3], FFt[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int a = 0; a < 3; ++a) Fg[k][a] = F[a][0] * g[k][0] + F[a][1] * g[k][1];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = a; b < 3; ++b) FFt[a][b] = F[a][0] * F[b][0] + F[a][1] * F[b][1];
        const float c = hk * A0;
        float *o = out + (int64_t)PC_TRI_STRIDE * t + 9;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int l = k; l < 3; ++l) {
                float gg = g[k][0] * g[l][0] + g[k][1] * g[l][1];
                float gSg = g[k][0] * (Sp00 * g[l][0] + Sp01 * g[l][1]) + g[k][1] * (Sp01 * g[l][0] + Sp11 * g[l][1]);
                float *B = o + 9 * tri_blk(k, l);
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        if (k == l && b < a) continue;
                        float ffab = a <= b ? FFt[a][b] : FFt[b][a];
                        float val = mu * Fg[l][a] * Fg[k][b] + mu * gg * ffab + lam * Fg[k][a] * Fg[l][b];
                        if (a == b) val += gSg;
                        B[3 * a + b] = c * val;
                        if (k == l && a != b) B[3 * b + a] = c * val;
                    }
            }
    }
    // ---- right-hand-side contributions c_k = h f_k - sum_{l != k} Hs_kl (v_l - v_k)
    {
        const float *Bs = out + (int64_t)PC_TRI_STRIDE * t + 9;
        const int vid[3] = {i0, i1, i2};
        float vv[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int a = 0; a < 3; ++a) vv[k][a] = v[3 * vid[k] + a];
        float *o = out + (int64_t)PC_TRI_STRIDE * t;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float ck[3] = {h * f[k][0], h * f[k][1], h * f[k][2]};
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                if (l == k) continue;
                float dv0 = vv[l][0] - vv[k][0], dv1 = vv[l][1] - vv[k][1], dv2 = vv[l][2] - vv[k][2];
                const float *B = Bs + 9 * tri_blk(k < l ? k : l, k < l ? l : k);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    // row a of block (k, l): B[a][*] if k < l, else column a of block (l, k)
                    float b0 = k < l ? B[3 * a] : B[a], b1 = k < l ? B[3 * a + 1] : B[3 + a],
                          b2 = k < l ? B[3 * a + 2] : B[6 + a];
                    ck[a] -= b0 * dv0 + b1 * dv1 + b2 * dv2;
                }
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) o[3 * k + a] = ck[a];
        }
        o[63] = 0.0f;
    }
}

// ------------------------------------------------------------------------- bending hinges

// theta = atan2((n1 x n2).e, n1.n2) of a hinge given relative vectors a1 = x1-x3,
// a2 = x2-x3, a4 = x4-x3 (x1, x2 wings; x3, x4 edge) and its gradient
// (Bridson, Marino and Fedkiw 2003).
__device__ __forceinline__ float hinge_angle_grad(float3 a1, float3 a2, float3 a4, float3 *grad)
{
    float3 E = a4;
    float3 N1 = cross(a1, sub(a1, a4));            // (x1-x3) x (x1-x4)
    float3 N2 = cross(sub(a2, a4), a2);            // (x2-x4) x (x2-x3)
    float lE = sqrtf(dot(E, E));
    float n1sq = dot(N1, N1), n2sq = dot(N2, N2);
    float in1 = rsqrtf(n1sq), in2 = rsqrtf(n2sq);
    float3 c = cross(N1, N2);
    float s = dot(c, E) * (in1 * in2 / lE);
    float co = dot(N1, N2) * (in1 * in2);
    float theta = atan2f(s, co);
    float3 u1 = mul(lE / n1sq, N1), u2 = mul(lE / n2sq, N2);
    float s13 = dot(sub(a1, a4), E) / lE, s23 = dot(sub(a2, a4), E) / lE;
    float s14 = dot(a1, E) / lE, s24 = dot(a2, E) / lE;
    float3 u3 = add(mul(s13 / n1sq, N1), mul(s23 / n2sq, N2));
    float3 u4 = add(mul(-s14 / n1sq, N1), mul(-s24 / n2sq, N2));
    grad[0] = mul(-1.0f, u1);
    grad[1] = mul(-1.0f, u2);
    grad[2] = mul(-1.0f, u3);
    grad[3] = mul(-1.0f, u4);
    return theta;
}

// One thread per hinge, at x_t. Record: right-hand-side contributions on (wing0, wing1,
// edge0, edge1), c_k = h f_k - q_k (q . v), then the scaled angle gradient
// q = h sqrt(2 kb c_h) grad(theta), so the Gauss-Newton Hessian block (k, l) is q_k q_l^T.
// The gradient sums to zero over the four vertices, so q . v uses velocities relative
// to edge0.
__global__ void __launch_bounds__(128) hinge_eval_kernel(int H, const int32_t *__restrict__ hinge,
                                                         const float *__restrict__ x, const float *__restrict__ v,
                                                         const float *__restrict__ hcoef,
                                                         const float *__restrict__ hrest, float h, float hk,
                                                         float *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= H) return;
    int vid[4] = {hinge[4 * i], hinge[4 * i + 1], hinge[4 * i + 2], hinge[4 * i + 3]};
    float3 X[4], W[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) { X[k] = ld3(x, vid[k]); W[k] = ld3(v, vid[k]); }
    const float kc = hcoef[i];
    float *o = out + (int64_t)PC_HINGE_STRIDE * i;
    float3 grad[4];
    // positions relative to edge0
    float3 a1 = sub(X[0], X[2]), a2 = sub(X[1], X[2]), a4 = sub(X[3], X[2]);
    float th = hinge_angle_grad(a1, a2, a4, grad);
    float s = -kc * (th - hrest[i]);  // f_k = s grad_k
    float sc = sqrtf(hk * kc);
    float3 q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = mul(sc, grad[k]);
    float qv = dot(q[0], sub(W[0], W[2])) + dot(q[1], sub(W[1], W[2])) + dot(q[3], sub(W[3], W[2]));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        o[3 * k] = h * s * grad[k].x - q[k].x * qv;
        o[3 * k + 1] = h * s * grad[k].y - q[k].y * qv;
        o[3 * k + 2] = h * s * grad[k].z - q[k].z * qv;
        o[12 + 3 * k] = q[k].x;
        o[12 + 3 * k + 1] = q[k].y;
        o[12 + 3 * k + 2] = q[k].z;
    }
}

// ------------------------------------------------------------------------- contacts

// One thread per pair (p; a, b, c). Record: right-hand-side contributions (12), unit
// normal n of (a, b, c) at x (3), weights (3), h^2 kc (1) (h (h + beta) kc with Rayleigh
// damping; 0 for an inactive thickness contact). With s = (1, -w_a, -w_b, -w_c) the
// Hessian block (k, l) is h^2 kc s_k s_l n n^T. The hold penalty is zero at x_t (d = d0)
// and linear in x, so its contribution h (f - h K v) is -h^2 kc (n . sum_l s_l v_l) s_k n;
// the thickness penalty adds its force at x_t, h kc (delta - d) s_k n.
__global__ void contact_eval_kernel(int P, const int32_t *__restrict__ pairs, const float *__restrict__ wts,
                                    const float *__restrict__ x, const float *__restrict__ v, float kc, float h,
                                    float hk, float thick, float *__restrict__ out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    int vid[4] = {pairs[4 * i], pairs[4 * i + 1], pairs[4 * i + 2], pairs[4 * i + 3]};
    float w[3] = {wts[3 * i], wts[3 * i + 1], wts[3 * i + 2]};
    float3 xa = ld3(x, vid[1]);
    float3 n = cross(sub(ld3(x, vid[2]), xa), sub(ld3(x, vid[3]), xa));
    n = mul(rsqrtf(dot(n, n)), n);
    float s[4] = {1.0f, -w[0], -w[1], -w[2]};
    // one-sided thickness model: n turned towards p at x_t, force h kc (delta - d) at x_t
    // while d < delta, no stiffness otherwise; hold penalty (delta = 0): no force at x_t
    float kc_eff = kc, fd = 0.f;
    if (thick > 0.f) {
        float3 r = make_float3(0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 4; ++k) r = add(r, mul(s[k], ld3(x, vid[k])));
        float dt = dot(n, r);
        if (dt < 0.f) {
            n = mul(-1.0f, n);
            dt = -dt;
        }
        if (dt < thick) fd = h * kc * (thick - dt);
        else kc_eff = 0.f;
    }
    float3 rv = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 4; ++k) rv = add(rv, mul(s[k], ld3(v, vid[k])));
    float dd = dot(n, rv);  // n . sum_l s_l v_l
    float *o = out + (int64_t)PC_CONTACT_STRIDE * i;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float fk = (fd - hk * kc_eff * dd) * s[k];
        o[3 * k] = fk * n.x;
        o[3 * k + 1] = fk * n.y;
        o[3 * k + 2] = fk * n.z;
    }
    o[12] = n.x; o[13] = n.y; o[14] = n.z;
    o[15] = w[0]; o[16] = w[1]; o[17] = w[2];
    o[18] = hk * kc_eff;
    o[19] = 0.0f;
}

// ------------------------------------------------------------------------- row reduction

#define RR_WARPS 4
#define RR_ENTRIES 128  // 32 references x up to 4 blocks

// Fetch element reference `ref`'s contribution to its local vertex's row: the
// right-hand-side share (3 floats) and one block per element vertex (3 or 4), with the
// column of each.
__device__ __forceinline__ int fetch_contribution(uint32_t ref, const int32_t *__restrict__ tri,
                                                  const int32_t *__restrict__ hinge,
                                                  const int32_t *__restrict__ pairs,
                                                  const float *__restrict__ tri_buf,
                                                  const float *__restrict__ hinge_buf,
                                                  const float *__restrict__ cont_buf, float *blk /*[4][9]*/,
                                                  int *cols /*[4]*/, float *f /*[3]*/)
{
    uint32_t type = pc_ref_type(ref), k = pc_ref_local(ref), id = pc_ref_id(ref);
    if (type == PC_REF_TRI) {
        const float *o = tri_buf + (int64_t)PC_TRI_STRIDE * id;
        f[0] = o[3 * k]; f[1] = o[3 * k + 1]; f[2] = o[3 * k + 2];
        for (int l = 0; l < 3; ++l) {
            cols[l] = tri[3 * id + l];
            const float *B = o + 9 + 9 * tri_blk(k < l ? k : l, k < l ? l : k);
            if (k <= (uint32_t)l) {
                for (int e = 0; e < 9; ++e) blk[9 * l + e] = B[e];
            } else {
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) blk[9 * l + 3 * a + b] = B[3 * b + a];
            }
        }
        return 3;
    }
    if (type == PC_REF_HINGE) {
        const float *o = hinge_buf + (int64_t)PC_HINGE_STRIDE * id;
        f[0] = o[3 * k]; f[1] = o[3 * k + 1]; f[2] = o[3 * k + 2];
        float qk[3] = {o[12 + 3 * k], o[12 + 3 * k + 1], o[12 + 3 * k + 2]};
        for (int l = 0; l < 4; ++l) {
            cols[l] = hinge[4 * id + l];
            const float *ql = o + 12 + 3 * l;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) blk[9 * l + 3 * a + b] = qk[a] * ql[b];
        }
        return 4;
    }
    const float *o = cont_buf + (int64_t)PC_CONTACT_STRIDE * id;
    f[0] = o[3 * k]; f[1] = o[3 * k + 1]; f[2] = o[3 * k + 2];
    float n[3] = {o[12], o[13], o[14]};
    float s[4] = {1.0f, -o[15], -o[16], -o[17]};
    float c = o[18];
    for (int l = 0; l < 4; ++l) {
        cols[l] = pairs[4 * id + l];
        float cs = c * (s[k] * s[l]);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) blk[9 * l + 3 * a + b] = cs * (n[a] * n[b]);
    }
    return 4;
}

// One warp per row. Lane s owns slot s of the row (in chunks of 32 slots); lanes stage
// the contributions of up to 32 incident elements at a time in shared memory, and each
// slot owner adds the staged blocks whose column matches its own, in staging order
// (static incidence order, then contact order). Then mass, pins and the right-hand side.
__global__ void __launch_bounds__(32 * RR_WARPS) row_reduce_kernel(
    int V, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const int32_t *__restrict__ vinc_ptr,
    const uint32_t *__restrict__ vinc, const int32_t *__restrict__ cinc_ptr, const uint32_t *__restrict__ cinc,
    const int32_t *__restrict__ tri, const int32_t *__restrict__ hinge, const int32_t *__restrict__ pairs,
    const float *__restrict__ tri_buf, const float *__restrict__ hinge_buf, const float *__restrict__ cont_buf,
    const float *__restrict__ mass, const uint8_t *__restrict__ pinned, float gx, float gy, float gz, float h,
    float md, float ha, const float *__restrict__ v, float *__restrict__ vals, float *__restrict__ b,
    float *__restrict__ dres)
{
    __shared__ float s_blk[RR_WARPS][RR_ENTRIES][9];
    __shared__ int s_col[RR_WARPS][RR_ENTRIES];
    __shared__ float s_f[RR_WARPS][32][3];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * RR_WARPS + warp;
    if (row >= V) return;
    const int s0 = rp[row], nslots = rp[row + 1] - s0;
    const int i0 = vinc_ptr[row], ni = vinc_ptr[row + 1] - i0;
    const int c0 = cinc_ptr[row], nc = cinc_ptr[row + 1] - c0;
    const int nref = ni + nc;
    const float m = mass[row];
    const float mA = md * m;  // diagonal mass term (1 + h alpha) m of an unpinned row
    const bool prow = pinned[row] != 0;
    float fsum[3] = {0.f, 0.f, 0.f};
    float dsum[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) dsum[e] = 0.f;

    for (int sc = 0; sc < nslots; sc += 32) {
        const bool has = sc + lane < nslots;
        const int slot = s0 + sc + lane;
        const int col = has ? ci[slot] : -1;
        float acc[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) acc[e] = 0.f;
        for (int rc = 0; rc < nref; rc += 32) {
            const int k = rc + lane;
            float blk[36];
            int cols[4] = {-1, -1, -1, -1};
            float f[3] = {0.f, 0.f, 0.f};
            if (k < nref) {
                uint32_t ref = k < ni ? vinc[i0 + k] : cinc[c0 + (k - ni)];
                fetch_contribution(ref, tri, hinge, pairs, tri_buf, hinge_buf, cont_buf, blk, cols, f);
            }
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                s_col[warp][4 * lane + l] = cols[l];
                if (cols[l] >= 0)
#pragma unroll
                    for (int e = 0; e < 9; ++e) s_blk[warp][4 * lane + l][e] = blk[9 * l + e];
            }
            s_f[warp][lane][0] = f[0];
            s_f[warp][lane][1] = f[1];
            s_f[warp][lane][2] = f[2];
            __syncwarp();
            const int cnt = min(32, nref - rc);
            for (int e = 0; e < 4 * cnt; ++e) {
                if (s_col[warp][e] == col) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) acc[q] += s_blk[warp][e][q];
                }
            }
            if (sc == 0 && lane == 0) {
                for (int e = 0; e < cnt; ++e) {
                    fsum[0] += s_f[warp][e][0];
                    fsum[1] += s_f[warp][e][1];
                    fsum[2] += s_f[warp][e][2];
                }
            }
            __syncwarp();
        }
        if (has) {
            const bool pcol = pinned[col] != 0;
            float outv[9];
            if (prow || pcol) {
#pragma unroll
                for (int q = 0; q < 9; ++q) outv[q] = 0.f;
                if (col == row) outv[0] = outv[4] = outv[8] = m;
                if (pcol && !prow && col != row) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) dsum[q] += acc[q];
                }
            } else {
#pragma unroll
                for (int q = 0; q < 9; ++q) outv[q] = acc[q];
                if (col == row) {
                    outv[0] += mA;
                    outv[4] += mA;
                    outv[8] += mA;
                }
            }
            float *dst = vals + 9ll * slot;
#pragma unroll
            for (int q = 0; q < 9; ++q) dst[q] = outv[q];
        }
    }
    // difference-form diagonal: m I minus the unzeroed blocks toward pinned neighbours
#pragma unroll
    for (int q = 0; q < 9; ++q)
        for (int o = 16; o > 0; o >>= 1) dsum[q] += __shfl_xor_sync(0xffffffffu, dsum[q], o);
    if (lane == 0) {
        if (dres) {
            float *d = dres + 9ll * row;
#pragma unroll
            for (int q = 0; q < 9; ++q) d[q] = prow ? 0.f : -dsum[q];
            const float md_row = prow ? m : mA;
            d[0] += md_row;
            d[4] += md_row;
            d[8] += md_row;
        }
        float *bb = b + 3ll * row;
        if (prow) {
            bb[0] = bb[1] = bb[2] = 0.f;
        } else {
            // gravity and the mass-damping force at v_t, both times h
            const float hm = h * m, ham = ha * m;
            bb[0] = fsum[0] + hm * gx - ham * v[3ll * row];
            bb[1] = fsum[1] + hm * gy - ham * v[3ll * row + 1];
            bb[2] = fsum[2] + hm * gz - ham * v[3ll * row + 2];
        }
    }
}

extern "C" pc_status pc_assemble_values(pc_ctx *ctx, const pc_bsr *A, const float *x, const float *v,
                                        const pc_contacts *contacts, float h, float *vals, float *b, float *dres,
                                        void *stream)
{
    if (!ctx || !A || !A->row_ptr || !A->col_idx || !x || !v || !vals || !b) return PC_ERR_ARG;
    int32_t P = contacts ? contacts->n : 0;
    if (P < 0 || P > ctx->max_contacts || (P > 0 && (!contacts->pairs || !contacts->w))) return PC_ERR_ARG;
    if (P != ctx->n_contacts) return PC_ERR_ARG;  // pattern was built for another contact set
    if (!(h > 0.0f)) return PC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int V = ctx->V, T = ctx->T, H = ctx->H;
    // Rayleigh damping: element Hessians enter A as h (h + beta) K, the mass as
    // (1 + h alpha) M (beta = alpha = 0: h^2 K and M)
    const float hk = h * (h + ctx->mat.damp_stiff);
    const float md = 1.0f + h * ctx->mat.damp_mass, ha = h * ctx->mat.damp_mass;
    if (T > 0)
        PC_LAUNCH(ctx, tri_eval_kernel, pc_blocks(T, 128), 128, 0, st, T, ctx->tri, x, v, ctx->tri_dmi, ctx->tri_area,
                  ctx->tri_rgram, ctx->mu, ctx->lam, h, hk, ctx->tri_buf);
    if (H > 0)
        PC_LAUNCH(ctx, hinge_eval_kernel, pc_blocks(H, 128), 128, 0, st, H, ctx->hinge, x, v, ctx->hcoef, ctx->hrest, h,
                  hk, ctx->hinge_buf);
    if (P > 0)
        PC_LAUNCH(ctx, contact_eval_kernel, pc_blocks(P, 128), 128, 0, st, P, contacts->pairs, contacts->w, x, v,
                  ctx->mat.k_contact, h, hk, ctx->mat.contact_thickness, ctx->cont_buf);
    PC_LAUNCH(ctx, row_reduce_kernel, pc_blocks(V, RR_WARPS), 32 * RR_WARPS, 0, st, V, A->row_ptr, A->col_idx,
              ctx->vinc_ptr, ctx->vinc, ctx->cinc_ptr, ctx->cinc, ctx->tri, ctx->hinge,
              P > 0 ? contacts->pairs : nullptr, ctx->tri_buf, ctx->hinge_buf, ctx->cont_buf, ctx->mass, ctx->pinned,
              ctx->mat.gravity[0], ctx->mat.gravity[1], ctx->mat.gravity[2], h, md, ha, v, vals, b, dres);
    return PC_OK;
}
