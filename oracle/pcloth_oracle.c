/*
 * pcloth_oracle.c -- plain FP64 CPU oracle for the implicit-integrator hot path of
 * P-Cloth (Li, Tang, Manocha et al., "P-Cloth: Interactive Complex Cloth Simulation
 * on Multi-GPU Systems using Dynamic Matrix Assembly and Pipelined Implicit
 * Integrators", SIGGRAPH Asia 2020).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load this file's library. The product path (the CUDA library) never
 * calls it, shares no code with it, and fails loudly when its own extension is missing.
 *
 * What it computes, each piece written out from its definition, in double precision,
 * with no blocking, fusion or reordering:
 *
 *  - Sec. 2.5, Eq. 1: M u'' = f on a p-vertex triangle mesh, M lumped (m_i = sum over
 *    incident triangles of rho * A0 / 3).
 *  - Sec. 2.5, Eq. 2-3: backward Euler with a first-order Taylor expansion of f,
 *      (M - h^2 J) dv = h f(x_t + h v_t),   J = df/dx at x_t,
 *    with J replaced by minus the sum of positive-semidefinite element Hessians K, and
 *    the right-hand side read to first order as Eq. 2 prescribes:
 *      f(x_t + h v_t) ~= f(x_t) + h J v_t,  so  b = h (f(x_t) - h K v_t).
 *    (Evaluating the force at x_t + h v_t without linearising is unstable for the stiff
 *    membranes of the workloads: it extrapolates rotations into spurious stretch.)
 *  - Sec. 3.2: "assembly elements" forming f and J. The paper names the forces
 *    (stretching, bending, contact, gravity; it cites Bridson et al. 2002 and Otaduy
 *    et al. 2009) but gives no formulas, so this file uses:
 *      membrane: St. Venant-Kirchhoff, plane stress, W = A0 (mu |G|^2 + lam/2 tr(G)^2),
 *                G = (F^T F - I)/2, F = [x1-x0, x2-x0] Dm^-1; Hessian with the second
 *                Piola-Kirchhoff stress clamped to its positive part in the geometric term;
 *      bending:  dihedral hinge E = kb c_h (theta - theta_rest)^2,
 *                c_h = 3 |e|^2 / (A1 + A2) at rest, angle gradient of Bridson, Marino
 *                and Fedkiw 2003, Gauss-Newton Hessian 2 kb c_h grad(theta) grad(theta)^T;
 *      contact:  hold penalty E = kc/2 (d - d0)^2, d = n . (x_p - sum w_k x_k), n the
 *                unit normal of the partner triangle at x_t (frozen), d0 = d(x_t); or,
 *                with a contact thickness delta > 0 (an extension), the one-sided
 *                penalty E = kc/2 (delta - d)^2 while d(x_t) < delta, n turned towards
 *                the vertex's side at x_t;
 *      gravity:  f_i = m_i g.
 *  - Sec. 3.2.2: the matrix pattern is the set of (row, col) vertex pairs coupled by some
 *    element, duplicates removed, stored as block compressed rows of 3x3 blocks with
 *    columns ascending and the diagonal always present.
 *  - Rayleigh damping (an extension; the paper's Eq. 3 has no velocity derivative):
 *    f_d = -(alpha M + beta K) v. Backward Euler keeps the -h df/dv term of the
 *    linearisation (Baraff and Witkin 1998), so
 *      A = (1 + h alpha) M + h (h + beta) K,
 *      b = h (f(x_t) - alpha M v_t - (h + beta) K v_t);
 *    alpha = beta = 0 gives the system above.
 *  - Pinned vertices keep their pattern entries; their rows and columns are zero except
 *    A_ii = m_i I, and b_i = 0, so dv_i = 0.
 *  - Sec. 2.5: the system is solved with preconditioned conjugate gradients (Jacobi:
 *    the scalar diagonal of A), stopping on the unpreconditioned relative residual.
 *
 * The row loops of the matrix-vector product and the vector loops of the solver carry
 * OpenMP work-sharing pragmas, so the oracle uses every host core at the benchmark sizes;
 * they split independent rows (or independent terms of a sum) across threads and change
 * nothing else. Without OpenMP the file compiles to the same single-threaded program.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OM_OK 0
#define OM_ERR_ARG -1
#define OM_ERR_PATTERN -2
#define OM_ERR_CAPACITY -3
#define OM_ERR_NOT_CONVERGED -4

typedef struct {
    int V, T, H, npin;
    int *tri;            /* [T][3] */
    double *Dminv;       /* [T][4] inverse of the 2x2 rest edge matrix, row-major */
    double *area;        /* [T] rest area A0 */
    double *mass;        /* [V] lumped mass */
    int *hinge;          /* [H][4]: wing0, wing1, edge0, edge1 */
    double *hcoef;       /* [H] c_h */
    double *hrest;       /* [H] rest dihedral angle */
    unsigned char *pinned; /* [V] */
    double rho, E, nu, kb, kc, g[3];
    double alpha, beta;  /* Rayleigh damping: mass (1/s) and stiffness (s) coefficients */
    double thick;        /* contact thickness delta (m): 0 = hold penalty, > 0 = one-sided */
    double mu, lam;
} om_mesh;

void om_spmv(int V, const int *row_ptr, const int *col_idx, const double *vals, const double *x, double *y);

/* ------------------------------------------------------------------ small vector helpers */

static void sub3(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* ------------------------------------------------------------------ rest state */

/* Rest edge matrix of one triangle in its own plane: Dm = [[|e1|, e2.u], [0, e2.v]],
 * u = e1/|e1|, v = n x u. Returns 0 for a degenerate triangle. */
static int tri_rest(const double *X0, const double *X1, const double *X2, double *Dminv, double *A0)
{
    double e1[3], e2[3], n[3], u[3], w[3], v[3];
    sub3(X1, X0, e1);
    sub3(X2, X0, e2);
    cross3(e1, e2, n);
    double ln = norm3(n), l1 = norm3(e1);
    if (!(ln > 0.0) || !(l1 > 0.0)) return 0;
    for (int a = 0; a < 3; ++a) { u[a] = e1[a] / l1; w[a] = n[a] / ln; }
    cross3(w, u, v);
    double d00 = l1, d01 = dot3(e2, u), d10 = 0.0, d11 = dot3(e2, v);
    double det = d00 * d11 - d01 * d10;
    Dminv[0] = d11 / det;
    Dminv[1] = -d01 / det;
    Dminv[2] = -d10 / det;
    Dminv[3] = d00 / det;
    *A0 = 0.5 * ln;
    return 1;
}

/* Dihedral angle of hinge (x1, x2 wings; x3, x4 edge): theta = atan2((n1 x n2).e, n1.n2)
 * with N1 = (x1-x3) x (x1-x4), N2 = (x2-x4) x (x2-x3), e = (x4-x3)/|x4-x3|. Also returns
 * its gradient (Bridson, Marino and Fedkiw 2003): grad = -(u1, u2, u3, u4) with
 * u1 = |E| N1/|N1|^2, u2 = |E| N2/|N2|^2,
 * u3 = (x1-x4).E/|E| N1/|N1|^2 + (x2-x4).E/|E| N2/|N2|^2,
 * u4 = -(x1-x3).E/|E| N1/|N1|^2 - (x2-x3).E/|E| N2/|N2|^2. */
static double hinge_angle(const double *x1, const double *x2, const double *x3, const double *x4, double grad[12])
{
    double a[3], b[3], N1[3], N2[3], E[3];
    sub3(x1, x3, a);
    sub3(x1, x4, b);
    cross3(a, b, N1);
    sub3(x2, x4, a);
    sub3(x2, x3, b);
    cross3(a, b, N2);
    sub3(x4, x3, E);
    double lE = norm3(E), n1sq = dot3(N1, N1), n2sq = dot3(N2, N2);
    double n1[3], n2[3], c[3], e[3];
    for (int k = 0; k < 3; ++k) { n1[k] = N1[k] / sqrt(n1sq); n2[k] = N2[k] / sqrt(n2sq); e[k] = E[k] / lE; }
    cross3(n1, n2, c);
    double theta = atan2(dot3(c, e), dot3(n1, n2));
    if (grad) {
        double d;
        for (int k = 0; k < 3; ++k) {
            grad[0 + k] = -lE * N1[k] / n1sq;
            grad[3 + k] = -lE * N2[k] / n2sq;
        }
        double t1[3], t2[3];
        sub3(x1, x4, t1);
        sub3(x2, x4, t2);
        double s13 = dot3(t1, E) / lE, s23 = dot3(t2, E) / lE;
        sub3(x1, x3, t1);
        sub3(x2, x3, t2);
        double s14 = dot3(t1, E) / lE, s24 = dot3(t2, E) / lE;
        for (int k = 0; k < 3; ++k) {
            d = s13 * N1[k] / n1sq + s23 * N2[k] / n2sq;
            grad[6 + k] = -d;
            d = -s14 * N1[k] / n1sq - s24 * N2[k] / n2sq;
            grad[9 + k] = -d;
        }
    }
    return theta;
}

/* ------------------------------------------------------------------ elements */

/* Positive part of a symmetric 2x2 matrix (negative eigenvalues set to zero). */
static void sym2_positive(const double S[2][2], double P[2][2])
{
    double a = S[0][0], b = S[0][1], c = S[1][1];
    double m = 0.5 * (a + c), r = sqrt(0.25 * (a - c) * (a - c) + b * b);
    double l1 = m + r, l2 = m - r;
    if (l2 >= 0.0) { memcpy(P, S, sizeof(double) * 4); return; }
    if (l1 <= 0.0) { memset(P, 0, sizeof(double) * 4); return; }
    double v0, v1;
    if (fabs(b) > 0.0) {
        if (fabs(l1 - a) > fabs(l1 - c)) { v0 = b; v1 = l1 - a; } else { v0 = l1 - c; v1 = b; }
    } else if (a >= c) { v0 = 1.0; v1 = 0.0; } else { v0 = 0.0; v1 = 1.0; }
    double nv = sqrt(v0 * v0 + v1 * v1);
    v0 /= nv;
    v1 /= nv;
    P[0][0] = l1 * v0 * v0;
    P[0][1] = P[1][0] = l1 * v0 * v1;
    P[1][1] = l1 * v1 * v1;
}

/* StVK membrane triangle at positions (x0, x1, x2). Any output may be NULL.
 * f[k*3+a]: force on vertex k; H[(k*3+l)*9 + a*3+b] = d2W / dx_{k,a} dx_{l,b}
 * with the stress clamped to its positive part in the geometric term. */
static void membrane(const double *x0, const double *x1, const double *x2, const double *Dmi, double A0,
                     double mu, double lam, double *W, double *f, double *H)
{
    double g[3][2];
    g[1][0] = Dmi[0]; g[1][1] = Dmi[1];
    g[2][0] = Dmi[2]; g[2][1] = Dmi[3];
    g[0][0] = -g[1][0] - g[2][0];
    g[0][1] = -g[1][1] - g[2][1];
    const double *xs[3] = {x0, x1, x2};
    double F[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 2; ++c) F[a][c] += xs[k][a] * g[k][c];
    double C[2][2];
    for (int c = 0; c < 2; ++c)
        for (int d = 0; d < 2; ++d) C[c][d] = F[0][c] * F[0][d] + F[1][c] * F[1][d] + F[2][c] * F[2][d];
    double G[2][2] = {{0.5 * (C[0][0] - 1.0), 0.5 * C[0][1]}, {0.5 * C[1][0], 0.5 * (C[1][1] - 1.0)}};
    double tr = G[0][0] + G[1][1];
    double S[2][2] = {{2.0 * mu * G[0][0] + lam * tr, 2.0 * mu * G[0][1]},
                      {2.0 * mu * G[1][0], 2.0 * mu * G[1][1] + lam * tr}};
    if (W) *W = A0 * (mu * (G[0][0] * G[0][0] + G[0][1] * G[0][1] + G[1][0] * G[1][0] + G[1][1] * G[1][1]) +
                      0.5 * lam * tr * tr);
    if (f) {
        double P[3][2];
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 2; ++c) P[a][c] = F[a][0] * S[0][c] + F[a][1] * S[1][c];
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) f[k * 3 + a] = -A0 * (P[a][0] * g[k][0] + P[a][1] * g[k][1]);
    }
    if (H) {
        double Sp[2][2];
        sym2_positive(S, Sp);
        double Fg[3][3], FFt[3][3];
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) Fg[k][a] = F[a][0] * g[k][0] + F[a][1] * g[k][1];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) FFt[a][b] = F[a][0] * F[b][0] + F[a][1] * F[b][1];
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) {
                double gg = g[k][0] * g[l][0] + g[k][1] * g[l][1];
                double gSg = 0.0;
                for (int c = 0; c < 2; ++c)
                    for (int d = 0; d < 2; ++d) gSg += g[k][c] * Sp[c][d] * g[l][d];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        H[(k * 3 + l) * 9 + a * 3 + b] =
                            A0 * ((a == b ? gSg : 0.0) + mu * Fg[l][a] * Fg[k][b] + mu * gg * FFt[a][b] +
                                  lam * Fg[k][a] * Fg[l][b]);
            }
    }
}

/* Dihedral hinge (x1, x2 wings; x3, x4 edge). f[k*3+a], H[(k*4+l)*9+a*3+b], k,l in 0..3. */
static void bending(const double *x1, const double *x2, const double *x3, const double *x4, double kb, double ch,
                    double theta0, double *E, double *f, double *H)
{
    double grad[12];
    double theta = hinge_angle(x1, x2, x3, x4, grad);
    double dth = theta - theta0;
    if (E) *E = kb * ch * dth * dth;
    if (f)
        for (int i = 0; i < 12; ++i) f[i] = -2.0 * kb * ch * dth * grad[i];
    if (H)
        for (int k = 0; k < 4; ++k)
            for (int l = 0; l < 4; ++l)
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        H[(k * 4 + l) * 9 + a * 3 + b] = 2.0 * kb * ch * grad[k * 3 + a] * grad[l * 3 + b];
}

/* Contact frame at x_t: unit normal n of (a, b, c) and d0 = n . (x_p - sum w x). */
static void contact_frame(const double *xt, const int *pr, const double *w, double n[3], double *d0)
{
    double e1[3], e2[3], c[3];
    sub3(xt + 3 * pr[2], xt + 3 * pr[1], e1);
    sub3(xt + 3 * pr[3], xt + 3 * pr[1], e2);
    cross3(e1, e2, c);
    double lc = norm3(c);
    for (int k = 0; k < 3; ++k) n[k] = c[k] / lc;
    double r[3];
    for (int k = 0; k < 3; ++k)
        r[k] = xt[3 * pr[0] + k] - w[0] * xt[3 * pr[1] + k] - w[1] * xt[3 * pr[2] + k] - w[2] * xt[3 * pr[3] + k];
    *d0 = dot3(n, r);
}

/* The frame of contact c for the mesh's contact model, from the state x_t:
 *  - hold penalty (thickness 0): n the unit normal of (a, b, c), d0 = n . (x_p - sum w x)
 *    at x_t, so E = kc/2 (d - d0)^2 is zero with zero force at x_t;
 *  - one-sided thickness delta > 0: n oriented towards p's side (d(x_t) >= 0) and
 *    E = kc/2 (delta - d)^2, active when d(x_t) < delta and zero otherwise; the active set
 *    and n are frozen over the step, so E is the hold penalty with d0 = delta.
 * Returns the stiffness of the contact (kc, or 0 when inactive). */
static double contact_setup(const om_mesh *M, const double *xt, const int *pr, const double *w, double n[3],
                            double *d0)
{
    double dt;
    contact_frame(xt, pr, w, n, &dt);
    if (M->thick <= 0.0) {
        *d0 = dt;
        return M->kc;
    }
    if (dt < 0.0) {
        for (int k = 0; k < 3; ++k) n[k] = -n[k];
        dt = -dt;
    }
    *d0 = M->thick;
    return dt < M->thick ? M->kc : 0.0;
}

/* Hold-penalty contact (p; a, b, c) with frozen n, d0. Vertex order p, a, b, c. */
static void contact(const double *x, const int *pr, const double *w, const double *n, double d0, double kc,
                    double *E, double *f, double *H)
{
    double s[4] = {1.0, -w[0], -w[1], -w[2]};
    double r[3] = {0, 0, 0};
    for (int k = 0; k < 4; ++k)
        for (int a = 0; a < 3; ++a) r[a] += s[k] * x[3 * pr[k] + a];
    double d = dot3(n, r) - d0;
    if (E) *E = 0.5 * kc * d * d;
    if (f)
        for (int k = 0; k < 4; ++k)
            for (int a = 0; a < 3; ++a) f[k * 3 + a] = -kc * d * s[k] * n[a];
    if (H)
        for (int k = 0; k < 4; ++k)
            for (int l = 0; l < 4; ++l)
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) H[(k * 4 + l) * 9 + a * 3 + b] = kc * s[k] * s[l] * n[a] * n[b];
}

/* ------------------------------------------------------------------ mesh set-up */

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

typedef struct { uint64_t key; int tri, opp; } half_edge;

static int cmp_half_edge(const void *a, const void *b)
{
    const half_edge *x = a, *y = b;
    if (x->key != y->key) return (x->key > y->key) - (x->key < y->key);
    return (x->tri > y->tri) - (x->tri < y->tri);
}

void om_mesh_destroy(om_mesh *M)
{
    if (!M) return;
    free(M->tri); free(M->Dminv); free(M->area); free(M->mass);
    free(M->hinge); free(M->hcoef); free(M->hrest); free(M->pinned);
    free(M);
}

/* mat = {rho, E, nu, kb, kc, gx, gy, gz, alpha, beta, delta}. Returns NULL on invalid input (index out of
 * range, degenerate triangle, an edge shared by more than two triangles). */
om_mesh *om_mesh_create(int V, int T, const int *tri, const double *rest, const double *mat, int npin, const int *pins)
{
    if (V <= 0 || T < 0) return NULL;
    om_mesh *M = calloc(1, sizeof(om_mesh));
    M->V = V; M->T = T; M->npin = npin;
    M->rho = mat[0]; M->E = mat[1]; M->nu = mat[2]; M->kb = mat[3]; M->kc = mat[4];
    M->g[0] = mat[5]; M->g[1] = mat[6]; M->g[2] = mat[7];
    M->alpha = mat[8]; M->beta = mat[9]; M->thick = mat[10];
    M->mu = M->E / (2.0 * (1.0 + M->nu));
    M->lam = M->E * M->nu / (1.0 - M->nu * M->nu);
    M->tri = malloc(sizeof(int) * 3 * (size_t)(T > 0 ? T : 1));
    M->Dminv = malloc(sizeof(double) * 4 * (size_t)(T > 0 ? T : 1));
    M->area = malloc(sizeof(double) * (size_t)(T > 0 ? T : 1));
    M->mass = calloc((size_t)V, sizeof(double));
    M->pinned = calloc((size_t)V, 1);
    for (int t = 0; t < T; ++t) {
        for (int k = 0; k < 3; ++k) {
            int v = tri[3 * t + k];
            if (v < 0 || v >= V) { om_mesh_destroy(M); return NULL; }
            M->tri[3 * t + k] = v;
        }
        const int *tv = M->tri + 3 * t;
        if (tv[0] == tv[1] || tv[1] == tv[2] || tv[0] == tv[2]) { om_mesh_destroy(M); return NULL; }
        if (!tri_rest(rest + 3 * tv[0], rest + 3 * tv[1], rest + 3 * tv[2], M->Dminv + 4 * t, M->area + t)) {
            om_mesh_destroy(M);
            return NULL;
        }
        for (int k = 0; k < 3; ++k) M->mass[tv[k]] += M->rho * M->area[t] / 3.0;
    }
    for (int i = 0; i < npin; ++i) {
        if (pins[i] < 0 || pins[i] >= V) { om_mesh_destroy(M); return NULL; }
        M->pinned[pins[i]] = 1;
    }
    /* hinges: interior edges shared by exactly two triangles */
    half_edge *he = malloc(sizeof(half_edge) * 3 * (size_t)(T > 0 ? T : 1));
    for (int t = 0; t < T; ++t)
        for (int k = 0; k < 3; ++k) {
            int a = M->tri[3 * t + k], b = M->tri[3 * t + (k + 1) % 3], o = M->tri[3 * t + (k + 2) % 3];
            int lo = a < b ? a : b, hi = a < b ? b : a;
            he[3 * t + k].key = (uint64_t)lo * (uint64_t)V + (uint64_t)hi;
            he[3 * t + k].tri = t;
            he[3 * t + k].opp = o;
            (void)hi;
        }
    qsort(he, 3 * (size_t)T, sizeof(half_edge), cmp_half_edge);
    int cap = 3 * T / 2 + 1;
    M->hinge = malloc(sizeof(int) * 4 * (size_t)cap);
    M->hcoef = malloc(sizeof(double) * (size_t)cap);
    M->hrest = malloc(sizeof(double) * (size_t)cap);
    int H = 0;
    for (int i = 0; i < 3 * T;) {
        int j = i;
        while (j < 3 * T && he[j].key == he[i].key) ++j;
        if (j - i > 2) { free(he); om_mesh_destroy(M); return NULL; }
        if (j - i == 2) {
            /* edge vertices in the order they appear in the first triangle */
            int t0 = he[i].tri, o0 = he[i].opp, o1 = he[i + 1].opp;
            int e0 = -1, e1 = -1;
            for (int k = 0; k < 3; ++k) {
                int a = M->tri[3 * t0 + k], b = M->tri[3 * t0 + (k + 1) % 3];
                if (M->tri[3 * t0 + (k + 2) % 3] == o0) { e0 = a; e1 = b; }
            }
            int *hv = M->hinge + 4 * H;
            hv[0] = o0; hv[1] = o1; hv[2] = e0; hv[3] = e1;
            double el[3];
            sub3(rest + 3 * e1, rest + 3 * e0, el);
            M->hcoef[H] = 3.0 * dot3(el, el) / (M->area[he[i].tri] + M->area[he[i + 1].tri]);
            M->hrest[H] = hinge_angle(rest + 3 * o0, rest + 3 * o1, rest + 3 * e0, rest + 3 * e1, NULL);
            ++H;
        }
        i = j;
    }
    free(he);
    M->H = H;
    return M;
}

int om_mesh_num_hinges(const om_mesh *M) { return M->H; }

void om_mesh_get(const om_mesh *M, double *mass, double *Dminv, double *area, int *hinge, double *hcoef, double *hrest)
{
    if (mass) memcpy(mass, M->mass, sizeof(double) * (size_t)M->V);
    if (Dminv) memcpy(Dminv, M->Dminv, sizeof(double) * 4 * (size_t)M->T);
    if (area) memcpy(area, M->area, sizeof(double) * (size_t)M->T);
    if (hinge) memcpy(hinge, M->hinge, sizeof(int) * 4 * (size_t)M->H);
    if (hcoef) memcpy(hcoef, M->hcoef, sizeof(double) * (size_t)M->H);
    if (hrest) memcpy(hrest, M->hrest, sizeof(double) * (size_t)M->H);
}

static int check_pairs(const om_mesh *M, int P, const int *pairs)
{
    for (int i = 0; i < P; ++i) {
        const int *p = pairs + 4 * i;
        for (int k = 0; k < 4; ++k)
            if (p[k] < 0 || p[k] >= M->V) return 0;
        for (int k = 0; k < 4; ++k)
            for (int l = k + 1; l < 4; ++l)
                if (p[k] == p[l]) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------------ energy and forces */

/* Total potential energy at x: membrane + bending + contact (frame from xt) - sum m g.x */
double om_energy(const om_mesh *M, const double *x, int P, const int *pairs, const double *w, const double *xt)
{
    double E = 0.0, e;
    for (int t = 0; t < M->T; ++t) {
        const int *v = M->tri + 3 * t;
        membrane(x + 3 * v[0], x + 3 * v[1], x + 3 * v[2], M->Dminv + 4 * t, M->area[t], M->mu, M->lam, &e, NULL, NULL);
        E += e;
    }
    for (int h = 0; h < M->H; ++h) {
        const int *v = M->hinge + 4 * h;
        bending(x + 3 * v[0], x + 3 * v[1], x + 3 * v[2], x + 3 * v[3], M->kb, M->hcoef[h], M->hrest[h], &e, NULL, NULL);
        E += e;
    }
    for (int c = 0; c < P; ++c) {
        double n[3], d0;
        const double kc = contact_setup(M, xt, pairs + 4 * c, w + 3 * c, n, &d0);
        contact(x, pairs + 4 * c, w + 3 * c, n, d0, kc, &e, NULL, NULL);
        E += e;
    }
    for (int i = 0; i < M->V; ++i) E -= M->mass[i] * dot3(M->g, x + 3 * i);
    return E;
}

/* f = -dE/dx at x (contact frame from xt). */
int om_forces(const om_mesh *M, const double *x, int P, const int *pairs, const double *w, const double *xt, double *f)
{
    if (!check_pairs(M, P, pairs)) return OM_ERR_ARG;
    for (int i = 0; i < M->V; ++i)
        for (int a = 0; a < 3; ++a) f[3 * i + a] = M->mass[i] * M->g[a];
    double fe[12];
    for (int t = 0; t < M->T; ++t) {
        const int *v = M->tri + 3 * t;
        membrane(x + 3 * v[0], x + 3 * v[1], x + 3 * v[2], M->Dminv + 4 * t, M->area[t], M->mu, M->lam, NULL, fe, NULL);
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) f[3 * v[k] + a] += fe[3 * k + a];
    }
    for (int h = 0; h < M->H; ++h) {
        const int *v = M->hinge + 4 * h;
        bending(x + 3 * v[0], x + 3 * v[1], x + 3 * v[2], x + 3 * v[3], M->kb, M->hcoef[h], M->hrest[h], NULL, fe, NULL);
        for (int k = 0; k < 4; ++k)
            for (int a = 0; a < 3; ++a) f[3 * v[k] + a] += fe[3 * k + a];
    }
    for (int c = 0; c < P; ++c) {
        double n[3], d0;
        const int *v = pairs + 4 * c;
        const double kc = contact_setup(M, xt, v, w + 3 * c, n, &d0);
        contact(x, v, w + 3 * c, n, d0, kc, NULL, fe, NULL);
        for (int k = 0; k < 4; ++k)
            for (int a = 0; a < 3; ++a) f[3 * v[k] + a] += fe[3 * k + a];
    }
    return OM_OK;
}

/* ------------------------------------------------------------------ pattern */

/* Sorted, duplicate-free (row, col) set of all element couplings plus the diagonal.
 * Writes row_ptr[V+1] and col_idx[nnzb] when nnzb <= cap; returns nnzb, or a negative
 * error code. */
long om_pattern(const om_mesh *M, int P, const int *pairs, int *row_ptr, int *col_idx, long cap)
{
    if (!check_pairs(M, P, pairs)) return OM_ERR_ARG;
    size_t n = (size_t)M->V + 9 * (size_t)M->T + 16 * (size_t)M->H + 16 * (size_t)P;
    uint64_t *keys = malloc(sizeof(uint64_t) * n);
    size_t m = 0;
    uint64_t V = (uint64_t)M->V;
    for (int i = 0; i < M->V; ++i) keys[m++] = (uint64_t)i * V + (uint64_t)i;
    for (int t = 0; t < M->T; ++t)
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) keys[m++] = (uint64_t)M->tri[3 * t + k] * V + (uint64_t)M->tri[3 * t + l];
    for (int h = 0; h < M->H; ++h)
        for (int k = 0; k < 4; ++k)
            for (int l = 0; l < 4; ++l) keys[m++] = (uint64_t)M->hinge[4 * h + k] * V + (uint64_t)M->hinge[4 * h + l];
    for (int c = 0; c < P; ++c)
        for (int k = 0; k < 4; ++k)
            for (int l = 0; l < 4; ++l) keys[m++] = (uint64_t)pairs[4 * c + k] * V + (uint64_t)pairs[4 * c + l];
    qsort(keys, m, sizeof(uint64_t), cmp_u64);
    size_t u = 0;
    for (size_t i = 0; i < m; ++i)
        if (i == 0 || keys[i] != keys[i - 1]) keys[u++] = keys[i];
    if ((long)u > cap) { free(keys); return (long)u; }
    size_t j = 0;
    for (int r = 0; r <= M->V; ++r) {
        while (j < u && keys[j] / V < (uint64_t)r) ++j;
        row_ptr[r] = (int)j;
    }
    for (size_t i = 0; i < u; ++i) col_idx[i] = (int)(keys[i] % V);
    free(keys);
    return (long)u;
}

static long find_slot(const int *row_ptr, const int *col_idx, int r, int c)
{
    int lo = row_ptr[r], hi = row_ptr[r + 1];
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (col_idx[mid] < c) lo = mid + 1; else hi = mid;
    }
    if (lo < row_ptr[r + 1] && col_idx[lo] == c) return lo;
    return -1;
}

static int add_blocks(const int *row_ptr, const int *col_idx, double *vals, const int *v, int nv, const double *H,
                      double scale)
{
    for (int k = 0; k < nv; ++k)
        for (int l = 0; l < nv; ++l) {
            long s = find_slot(row_ptr, col_idx, v[k], v[l]);
            if (s < 0) return 0;
            for (int e = 0; e < 9; ++e) vals[9 * s + e] += scale * H[(k * nv + l) * 9 + e];
        }
    return 1;
}

/* K = sum of element Hessians (clamped membrane, Gauss-Newton bending, contact) at x,
 * contact frame from xt, into the given pattern. No mass, no h^2, no pins. */
int om_hessian(const om_mesh *M, const double *x, int P, const int *pairs, const double *w, const double *xt,
               const int *row_ptr, const int *col_idx, double *vals)
{
    if (!check_pairs(M, P, pairs)) return OM_ERR_ARG;
    memset(vals, 0, sizeof(double) * 9 * (size_t)row_ptr[M->V]);
    double He[144];
    for (int t = 0; t < M->T; ++t) {
        const int *v = M->tri + 3 * t;
        membrane(x + 3 * v[0], x + 3 * v[1], x + 3 * v[2], M->Dminv + 4 * t, M->area[t], M->mu, M->lam, NULL, NULL, He);
        if (!add_blocks(row_ptr, col_idx, vals, v, 3, He, 1.0)) return OM_ERR_PATTERN;
    }
    for (int h = 0; h < M->H; ++h) {
        const int *v = M->hinge + 4 * h;
        bending(x + 3 * v[0], x + 3 * v[1], x + 3 * v[2], x + 3 * v[3], M->kb, M->hcoef[h], M->hrest[h], NULL, NULL, He);
        if (!add_blocks(row_ptr, col_idx, vals, v, 4, He, 1.0)) return OM_ERR_PATTERN;
    }
    for (int c = 0; c < P; ++c) {
        double n[3], d0;
        const double kc = contact_setup(M, xt, pairs + 4 * c, w + 3 * c, n, &d0);
        contact(x, pairs + 4 * c, w + 3 * c, n, d0, kc, NULL, NULL, He);
        if (!add_blocks(row_ptr, col_idx, vals, pairs + 4 * c, 4, He, 1.0)) return OM_ERR_PATTERN;
    }
    return OM_OK;
}

/* Eq. 3 with its right-hand side taken to first order, as Eq. 2 prescribes:
 *   f(x_t + h v_t) ~= f(x_t) + J h v_t,  J = -K(x_t),
 * so A = M + h^2 K(x_t) and b = h (f(x_t) - h K(x_t) v_t), K the same sum of element
 * Hessians in both. With Rayleigh damping f_d = -(alpha M + beta K) v the velocity
 * derivative adds h (alpha M + beta K) to A and the damping force at v_t to the
 * right-hand side: A = (1 + h alpha) M + h (h + beta) K,
 * b = h (f(x_t) - alpha M v_t - (h + beta) K v_t). Then the pin rule if `apply_pins` is
 * nonzero (pinned rows/cols zero, A_ii = m_i I, b_i = 0). */
int om_assemble(const om_mesh *M, const double *x, const double *v, int P, const int *pairs, const double *w,
                double h, int apply_pins, const int *row_ptr, const int *col_idx, double *vals, double *b)
{
    int V = M->V;
    int st = om_hessian(M, x, P, pairs, w, x, row_ptr, col_idx, vals);
    if (st != OM_OK) return st;
    double *Kv = malloc(sizeof(double) * 3 * (size_t)V);
    om_spmv(V, row_ptr, col_idx, vals, v, Kv);
    st = om_forces(M, x, P, pairs, w, x, b);
    if (st != OM_OK) { free(Kv); return st; }
    for (int i = 0; i < V; ++i)
        for (int a = 0; a < 3; ++a) {
            long k = 3L * i + a;
            b[k] = h * (b[k] - M->alpha * M->mass[i] * v[k] - (h + M->beta) * Kv[k]);
        }
    free(Kv);
    long nnzb = row_ptr[V];
    for (long s = 0; s < 9 * nnzb; ++s) vals[s] *= h * (h + M->beta);
    for (int i = 0; i < V; ++i) {
        long s = find_slot(row_ptr, col_idx, i, i);
        if (s < 0) return OM_ERR_PATTERN;
        for (int a = 0; a < 3; ++a) vals[9 * s + 4 * a] += (1.0 + h * M->alpha) * M->mass[i];
    }
    if (apply_pins) {
        for (int r = 0; r < V; ++r)
            for (int s = row_ptr[r]; s < row_ptr[r + 1]; ++s) {
                int c = col_idx[s];
                if (!M->pinned[r] && !M->pinned[c]) continue;
                for (int e = 0; e < 9; ++e) vals[9 * (long)s + e] = 0.0;
                if (r == c)
                    for (int a = 0; a < 3; ++a) vals[9 * (long)s + 4 * a] = M->mass[r];
            }
        for (int r = 0; r < V; ++r)
            if (M->pinned[r]) b[3 * r] = b[3 * r + 1] = b[3 * r + 2] = 0.0;
    }
    return OM_OK;
}

/* y = (1 + h alpha) M p + h (h + beta) sum_e H_e p_e, element by element with no
 * matrix (no pins). */
int om_matfree_apply(const om_mesh *M, const double *x, int P, const int *pairs, const double *w, double h,
                     const double *p, double *y)
{
    if (!check_pairs(M, P, pairs)) return OM_ERR_ARG;
    double He[144];
    for (int i = 0; i < M->V; ++i)
        for (int a = 0; a < 3; ++a) y[3 * i + a] = (1.0 + h * M->alpha) * M->mass[i] * p[3 * i + a];
    for (int t = 0; t < M->T + M->H + P; ++t) {
        const int *v;
        int nv;
        if (t < M->T) {
            v = M->tri + 3 * t;
            nv = 3;
            membrane(x + 3 * v[0], x + 3 * v[1], x + 3 * v[2], M->Dminv + 4 * t, M->area[t], M->mu, M->lam, NULL, NULL, He);
        } else if (t < M->T + M->H) {
            int hh = t - M->T;
            v = M->hinge + 4 * hh;
            nv = 4;
            bending(x + 3 * v[0], x + 3 * v[1], x + 3 * v[2], x + 3 * v[3], M->kb, M->hcoef[hh], M->hrest[hh], NULL, NULL, He);
        } else {
            int c = t - M->T - M->H;
            double n[3], d0;
            v = pairs + 4 * c;
            nv = 4;
            const double kc = contact_setup(M, x, v, w + 3 * c, n, &d0);
            contact(x, v, w + 3 * c, n, d0, kc, NULL, NULL, He);
        }
        for (int k = 0; k < nv; ++k)
            for (int l = 0; l < nv; ++l)
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        y[3 * v[k] + a] += h * (h + M->beta) * He[(k * nv + l) * 9 + a * 3 + b] * p[3 * v[l] + b];
    }
    return OM_OK;
}

/* Single-element evaluations for tests: kind 0 membrane (x: 3 vertices, aux: Dminv[4],
 * area), 1 bending (x: 4 vertices, aux: c_h, theta_rest), 2 contact (x: 4 vertices,
 * xt: 4 vertices of the frame state, aux: w[3]). Vertex indices are local 0..n-1. */
double om_element(const om_mesh *M, int kind, const double *x, const double *xt, const double *aux, double *f, double *H)
{
    double E = 0.0;
    if (kind == 0) {
        membrane(x, x + 3, x + 6, aux, aux[4], M->mu, M->lam, &E, f, H);
    } else if (kind == 1) {
        bending(x, x + 3, x + 6, x + 9, M->kb, aux[0], aux[1], &E, f, H);
    } else {
        int pr[4] = {0, 1, 2, 3};
        double n[3], d0;
        const double kc = contact_setup(M, xt, pr, aux, n, &d0);
        contact(x, pr, aux, n, d0, kc, &E, f, H);
    }
    return E;
}

double om_hinge_angle(const double *x1, const double *x2, const double *x3, const double *x4, double *grad)
{
    return hinge_angle(x1, x2, x3, x4, grad);
}

/* ------------------------------------------------------------------ linear algebra */

void om_spmv(int V, const int *row_ptr, const int *col_idx, const double *vals, const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int r = 0; r < V; ++r) {
        double acc[3] = {0, 0, 0};
        for (int s = row_ptr[r]; s < row_ptr[r + 1]; ++s) {
            const double *B = vals + 9 * (long)s;
            const double *xc = x + 3 * (long)col_idx[s];
            for (int a = 0; a < 3; ++a) acc[a] += B[3 * a] * xc[0] + B[3 * a + 1] * xc[1] + B[3 * a + 2] * xc[2];
        }
        y[3 * r] = acc[0]; y[3 * r + 1] = acc[1]; y[3 * r + 2] = acc[2];
    }
}

static double vdot(long n, const double *a, const double *b)
{
    double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Number of threads the oracle's parallel loops use (1 without OpenMP). */
int om_num_threads(void)
{
#ifdef _OPENMP
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        n = omp_get_num_threads();
    }
    return n;
#else
    return 1;
#endif
}

/* Jacobi-preconditioned conjugate gradients on A x = b (A symmetric positive definite),
 * x holds the initial guess on entry and the iterate on exit. Stops when
 * |b - A x| / |b| <= tol (recurrence residual, confirmed by a true residual at exit);
 * info = {iterations, true relative residual}. */
int om_pcg(int V, const int *row_ptr, const int *col_idx, const double *vals, const double *b, double *x,
           double tol, int max_iter, double *info)
{
    long n = 3L * V;
    double *r = malloc(sizeof(double) * n), *z = malloc(sizeof(double) * n), *p = malloc(sizeof(double) * n);
    double *q = malloc(sizeof(double) * n), *dinv = malloc(sizeof(double) * n);
    for (int i = 0; i < V; ++i) {
        long s = find_slot(row_ptr, col_idx, i, i);
        for (int a = 0; a < 3; ++a) dinv[3 * i + a] = 1.0 / vals[9 * s + 4 * a];
    }
    double bnorm = sqrt(vdot(n, b, b));
    int status = OM_OK, it = 0;
    if (bnorm == 0.0) {
        memset(x, 0, sizeof(double) * n);
        info[0] = 0; info[1] = 0.0;
        free(r); free(z); free(p); free(q); free(dinv);
        return OM_OK;
    }
    om_spmv(V, row_ptr, col_idx, vals, x, q);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) { r[i] = b[i] - q[i]; z[i] = dinv[i] * r[i]; p[i] = z[i]; }
    double rz = vdot(n, r, z);
    double rn = sqrt(vdot(n, r, r));
    while (rn > tol * bnorm) {
        if (it >= max_iter) { status = OM_ERR_NOT_CONVERGED; break; }
        om_spmv(V, row_ptr, col_idx, vals, p, q);
        double alpha = rz / vdot(n, p, q);
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        ++it;
        rn = sqrt(vdot(n, r, r));
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
        double rz_new = vdot(n, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    om_spmv(V, row_ptr, col_idx, vals, x, q);
    for (long i = 0; i < n; ++i) r[i] = b[i] - q[i];
    info[0] = it;
    info[1] = sqrt(vdot(n, r, r)) / bnorm;
    free(r); free(z); free(p); free(q); free(dinv);
    return status;
}
