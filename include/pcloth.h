/*
 * pcloth.h -- C ABI of the GB300 (sm_103a) implicit-integrator hot path of P-Cloth
 * (Li, Tang, Manocha et al., SIGGRAPH Asia 2020).
 *
 * One time step of the method (Sec. 2.5, Eq. 2-3) solves
 *
 *     (M - h^2 J) dv = h (f(x_t) + h J v_t),     J = df/dx at x_t = -K,
 *
 * for the velocity increment dv: Eq. 3's right-hand side h f(x_t + h v_t) taken to first
 * order around x_t, as Eq. 2 linearises f (the same J as in the matrix; K is the sum of
 * the positive-semidefinite element Hessians). The matrix is assembled anew each step from the
 * mesh's assembly elements (Sec. 3.2: membrane triangles, bending hinges, contact pairs,
 * gravity) and its sparsity pattern changes with the step's contact pairs (Sec. 3, first
 * paragraph). The system is solved with preconditioned conjugate gradients, whose cost
 * is the block-sparse matrix-vector product (Sec. 3.1).
 *
 * Conventions (every entry point):
 *  - Returns a pc_status; nothing throws or exits across the ABI and device code never
 *    traps. pc_status_string() turns a code into text.
 *  - Array arguments are DEVICE pointers owned by the caller, contiguous, 16-byte
 *    aligned, unless a parameter says "host". Indices are int32, values float32 unless
 *    stated. Vectors are float[V][3] (x, y, z per vertex).
 *  - Block matrices are block-CSR with 3x3 blocks ("BSR"): row_ptr[V+1], col_idx[nnzb]
 *    with columns ascending within a row and the diagonal block always present,
 *    vals[nnzb][9] row-major blocks. Block capacities must be multiples of 4.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). Work is
 *    stream-ordered; calls that return host-visible results (counts, solve info)
 *    synchronize the stream before returning.
 *  - A context (pc_ctx) holds one mesh's rest state and all scratch memory of the
 *    assembly and solve calls, allocated once by pc_create. The calls that allocate
 *    device memory are: pc_create; pc_mlp_create (training state); pc_set_warm_mlp
 *    (the context's feature and guess buffers, on the first attach); pc_mlp_infer (a
 *    4-byte timeout flag, on its first call in each host thread on each device, kept
 *    until the process exits); pc_step_batched (the CUDA graph it instantiates on its
 *    first call for a system shape). pc_pcg_solve_static allocates nothing at all.
 */
#ifndef PCLOTH_H
#define PCLOTH_H

#include <stdint.h>

#if defined(__GNUC__)
#define PC_API __attribute__((visibility("default")))
#else
#define PC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pc_status;
#define PC_OK 0
#define PC_ERR_ARG 1            /* invalid argument (null, size, alignment, index out of range) */
#define PC_ERR_CAPACITY 2       /* output buffer too small; the required size is reported */
#define PC_ERR_NOT_CONVERGED 3  /* PCG hit max_iter; outputs hold the last iterate and its residual */
#define PC_ERR_NONFINITE 4      /* NaN/Inf met in the right-hand side or a PCG scalar */
#define PC_ERR_TIMEOUT 5        /* a bounded device wait gave up */
#define PC_ERR_CUDA 6           /* a CUDA runtime call failed */
#define PC_ERR_MESH 7           /* degenerate triangle or an edge shared by more than two triangles */

#define PC_PREC_FP32 0   /* FP32 PCG (FP64 dot products) */
#define PC_PREC_MIXED 1  /* FP32 PCG with FP64 residual recomputation and refinement */

#define PC_WARM_ZERO 0   /* initial guess dv = 0 */
#define PC_WARM_PREV 1   /* initial guess = previous step's dv */
#define PC_WARM_GIVEN 2  /* initial guess = the dv buffer passed in */
#define PC_WARM_MLP 3    /* learned guess (pc_set_warm_mlp), combined with the previous-step guess:
                            the solve starts from the combination c_p g_prev + c_l g_learned with the
                            lowest CG energy 1/2 g.A g - b.g (the smallest A-norm error), found by a
                            2x2 Galerkin solve in FP64; the zero, previous and learned guesses are
                            its special cases, so it is never worse than any of them */
#define PC_WARM_COMBINED 4 /* pc_step_info.guess only: the solve started from that combination */

typedef struct pc_ctx pc_ctx;

/* Contact models (k = k_contact; pair (p; a, b, c) with weights w, s = (1, -w), n the unit
 * normal of (a, b, c) at x_t, d = n . (x_p - sum w_k x_k)):
 *  - contact_thickness = 0: hold penalty E = k/2 (d - d(x_t))^2, zero force at x_t;
 *  - contact_thickness = delta > 0 (an extension: one-sided thickness contact): n turned
 *    towards p's side at x_t and E = k/2 (delta - d)^2 while d(x_t) < delta, zero (and no
 *    stiffness) otherwise; the active set and n are frozen over the step.
 * Material of the cloth (SI units). Membrane: St. Venant-Kirchhoff, plane stress,
 * Young's modulus x thickness `young` (N/m) and `poisson`. Bending: dihedral hinges with
 * stiffness `k_bend` (N m). Contact: hold penalty `k_contact` (N/m). Optional Rayleigh
 * damping f_d = -(damp_mass M + damp_stiff K) v (an extension; the paper's Eq. 3 has no
 * velocity derivative): backward Euler then assembles
 *   A = (1 + h damp_mass) M + h (h + damp_stiff) K,
 *   b = h (f(x_t) - damp_mass M v_t - (h + damp_stiff) K v_t),
 * and both zero give Eq. 3 exactly. Pinned rows keep A_ii = m_i I. */
typedef struct {
    float rho;         /* area density, kg/m^2 */
    float young;       /* N/m */
    float poisson;
    float k_bend;      /* N m */
    float k_contact;   /* N/m */
    float gravity[3];  /* m/s^2 */
    float damp_mass;   /* Rayleigh alpha, 1/s (>= 0) */
    float damp_stiff;  /* Rayleigh beta, s (>= 0) */
    float contact_thickness; /* m (>= 0): 0 = hold penalty; > 0 = one-sided thickness penalty */
} pc_material;

/* Contact pairs of one step (Sec. 4: proximity forces inside the implicit integrator;
 * here they arrive as input). Pair i couples vertex p = pairs[4i] with triangle
 * (a, b, c) = pairs[4i+1..4i+3] through barycentric weights w[3i..3i+2] (sum 1). All
 * four vertices must be distinct and in range. Device pointers; n may be 0. */
typedef struct {
    int32_t n;
    const int32_t *pairs;  /* device [n][4] */
    const float *w;        /* device [n][3] */
} pc_contacts;

/* Caller-owned BSR pattern buffers. */
typedef struct {
    int32_t *row_ptr;  /* device [V+1] */
    int32_t *col_idx;  /* device [cap] */
    int64_t cap;       /* capacity in blocks, multiple of 4 */
    int64_t nnzb;      /* out: number of blocks */
} pc_bsr;

#define PC_PRECOND_JACOBI 0  /* inverse of the scalar diagonal of A */
#define PC_PRECOND_BLOCK 1   /* inverse of each 3x3 diagonal block of A */

typedef struct {
    double tol;          /* stop when |b - A dv|_2 / |b|_2 <= tol (default 1e-6) */
    int32_t max_iter;    /* total PCG iterations (default 20000) */
    int32_t precision;   /* PC_PREC_FP32 or PC_PREC_MIXED */
    double refresh;      /* PC_PREC_MIXED: recompute the residual in FP64 whenever |r| has
                            dropped by this factor since the last recomputation (default 1e-2) */
    int32_t refresh_every; /* PC_PREC_MIXED: ... or after this many iterations (default 1000) */
    int32_t check_every; /* iterations between convergence checks on the host (default 32) */
    int32_t precond;     /* PC_PRECOND_JACOBI (default) or PC_PRECOND_BLOCK */
    int32_t storage;     /* PC_STORAGE_OFFDIAG (default), PC_STORAGE_FULL, PC_STORAGE_SYM or
                            PC_STORAGE_SELL: matrix layout the PCG products read (the
                            result is the same up to summation order) */
    int32_t fuse;        /* 1 (default): each iteration's update and direction step run as one
                            kernel with a grid-wide barrier (z stays in registers; used when
                            every thread can carry its rows, up to about 0.9M rows on GB300);
                            0: two kernels. Same method, same stop tests. */
    int32_t schedule;    /* PC_SCHED_AUTO (default), PC_SCHED_GRID or PC_SCHED_CLUSTER */
} pc_solve_opts;

/* How pc_pcg_solve (and pc_step, pc_pcg_solve_static) runs the iterations.
 * PC_SCHED_CLUSTER: the whole solve is one launch of one thread-block cluster (16 CTAs,
 * one per SM, else 8 where 16 cannot be co-scheduled). Each CTA keeps a contiguous range
 * of rows -- their 3x3 blocks, diagonal data and vectors, and copies of the rows of other
 * CTAs that its rows reference -- in shared memory for the length of the solve. The
 * iteration is the single-reduction (Chronopoulos-Gear) form of the same preconditioned
 * CG: per iteration one product, one reduction and two cluster barriers, no kernel
 * boundary. Same preconditioners, stop tests and mixed precision as the grid schedule
 * (FP64 residual replacement in PC_PREC_MIXED, the FP64 iterate folded every check_every
 * iterations); the first residual is formed in FP64 in both precisions, and storage and
 * fuse do not apply. At a relative residual of 1e-6 it takes the grid schedule's
 * iteration count; near FP32's attainable accuracy (PC_PREC_MIXED at 1e-9) up to about a
 * third more. It takes systems up to about 6,000 rows at cloth density (at most 512 rows
 * per CTA, and every CTA's blocks and copied rows within its shared memory); larger ones
 * return PC_ERR_CAPACITY.
 * PC_SCHED_GRID: kernels over the whole GPU, iterations launched from the host (the
 * storage and fuse options apply).
 * PC_SCHED_AUTO: the cluster schedule when the system fits it, else the grid schedule. */
#define PC_SCHED_AUTO 0
#define PC_SCHED_GRID 1
#define PC_SCHED_CLUSTER 2

/* PC_STORAGE_FULL: the products read the full BSR matrix.
 * PC_STORAGE_SYM: at the start of each pc_pcg_solve / pc_step the (bitwise symmetric)
 * matrix is rewritten into its upper blocks plus, per row, the list of lower blocks as
 * references to the transposed upper blocks, and the products read that: a third less
 * DRAM traffic per product, but the gathered lower blocks put a second round of
 * dependent loads on each row's critical path, and on GB300 the product is slower
 * (about 1.7x at 512^2). It falls back to the full matrix when the system is larger than
 * the context's step-system capacity or its pattern is not symmetric. */
/* PC_STORAGE_SELL: at the start of each solve the off-diagonal blocks are rewritten into
 * sliced ELL (the ELL family of Sec. 3.2): slices of 32 rows, rows sorted by length inside
 * windows of 1024 rows, each 3x3 block stored as 10 words (column, 9 values) in structure
 * of arrays so that a warp reads every word with coalesced loads; the diagonal blocks are
 * not in the stream (the difference form does not need them). It falls back to the full
 * matrix when the layout exceeds the context's capacity. */
/* PC_STORAGE_OFFDIAG: with the difference-form diagonal given (dres), the products read a
 * copy of the BSR matrix without its diagonal blocks, made at the start of each solve (in
 * the difference form the diagonal block multiplies p_i - p_i = 0, so the copy gives the
 * same product with one block per row fewer to stream). Without dres, or when the copy
 * exceeds the context's capacity, the products read the matrix itself. */
#define PC_STORAGE_SYM 0
#define PC_STORAGE_FULL 1
#define PC_STORAGE_SELL 2
#define PC_STORAGE_OFFDIAG 3

typedef struct {
    int32_t iters;      /* PCG iterations (all inner solves) */
    int32_t outer;      /* FP64 residual recomputations (PC_PREC_MIXED), 0 for FP32 */
    double rel_res;     /* |b - A dv| / |b| recomputed in FP64 at exit */
    double bnorm;       /* |b|_2 */
} pc_solve_info;

typedef struct {
    float h;              /* time step, s */
    pc_solve_opts solve;
    int32_t warm_start;   /* PC_WARM_ZERO, PC_WARM_PREV or PC_WARM_MLP */
    float *feat_out;      /* device float[V][PC_MLP_IN] or NULL: receives this step's warm-start
                             features (computed after assembly, before the solve) */
} pc_step_opts;

typedef struct {
    int64_t nnzb;
    pc_solve_info solve;
    int32_t guess;         /* initial guess used: PC_WARM_ZERO, PC_WARM_PREV, PC_WARM_MLP or
                              PC_WARM_COMBINED */
    int32_t pad;
    double guess_res[3];   /* PC_WARM_MLP: |b - A g| / |b| of the zero, previous and learned
                              guesses (FP64); -1 when not evaluated */
    double guess_energy[3]; /* PC_WARM_MLP: 1/2 g.A g - b.g of the same guesses (0 for zero) */
    double guess_coef[2];  /* PC_WARM_MLP: the combination's coefficients (c_p, c_l) */
    double combo_energy;   /* PC_WARM_MLP: the CG energy of the guess the solve started from */
} pc_step_info;

/* Text for a status code (static storage). */
PC_API const char *pc_status_string(pc_status s);

/* Text of the most recent CUDA runtime failure seen by the library (static storage,
 * empty if none); PC_ERR_CUDA results point here. */
PC_API const char *pc_last_cuda_error(void);

/* Fill *o with the defaults named in pc_solve_opts. */
PC_API void pc_default_solve_opts(pc_solve_opts *o);

/* Create a context for a triangle mesh and precompute its rest state on the GPU:
 * per-triangle rest edge matrices and areas, lumped masses (rho * area / 3 per incident
 * triangle), the interior-edge hinges (two triangles per edge) with their rest angle and
 * coefficient 3|e|^2/(A1 + A2), the static block pattern of the mesh elements, and the
 * vertex-to-element incidence (Sec. 3.2.1: elements grouped by the rows they touch).
 *   V, T        vertex and triangle counts (V >= 1, T >= 0, 3T < 2^28)
 *   tris        device int32[T][3]
 *   rest        device float[V][3] rest positions (each triangle non-degenerate)
 *   pins        device int32[n_pins] pinned vertices (their dv is 0), may be NULL if n_pins = 0
 *   mat         host pointer to the material
 *   max_contacts  largest contact count any later call will pass
 * On failure *out is NULL and nothing is leaked. PC_ERR_MESH reports degenerate
 * triangles and edges shared by three or more triangles. Synchronizes `stream`. */
PC_API pc_status pc_create(pc_ctx **out, int32_t V, int32_t T, const int32_t *tris, const float *rest, const int32_t *pins,
                    int32_t n_pins, const pc_material *mat, int32_t max_contacts, void *stream);

/* Release a context and everything it owns (NULL is a no-op). */
PC_API pc_status pc_destroy(pc_ctx *ctx);

/* Sizes known to the context: V, T, hinge count H and the static (contact-free)
 * pattern's block count. Host pointers, each may be NULL. */
PC_API pc_status pc_get_sizes(const pc_ctx *ctx, int32_t *V, int32_t *T, int32_t *H, int64_t *static_nnzb);

/* Copy the hinges found by pc_create: int32[H][4] = (wing0, wing1, edge0, edge1), edge
 * ordered as in the lower-indexed triangle, hinges sorted by edge key min*V+max; and the
 * lumped masses float[V]. Device pointers, either may be NULL. */
PC_API pc_status pc_get_rest(const pc_ctx *ctx, int32_t *hinges, float *mass, void *stream);

/* Sec. 3.2.2, dynamic matrix assembly, pattern half: the step's block pattern is the set
 * of (row, col) vertex pairs coupled by any triangle, hinge or contact pair of this step,
 * plus the diagonal, sorted by (row, col) with duplicates removed. The contact keys are
 * sorted with a key sort and merged into the static pattern (no atomics), so row_ptr and
 * col_idx are bit-exact and deterministic.
 * On return A->nnzb holds the block count. If it exceeds A->cap the call returns
 * PC_ERR_CAPACITY with A->nnzb = required size and col_idx untouched beyond cap.
 * Synchronizes `stream`. */
PC_API pc_status pc_assemble_pattern(pc_ctx *ctx, const pc_contacts *contacts, pc_bsr *A, void *stream);

/* Sec. 3.2.2, value half, and Eq. 2-3: writes
 *   vals[nnzb][9]  A = M + h^2 K,  K = sum_e H_e(x_t)   (element Hessians: membrane with its
 *                  stress clamped to the positive part, Gauss-Newton bending, contact penalty)
 *   b[V][3]        b = h (f(x_t) - h K v_t)     (f includes gravity; the first-order
 *                  expansion of Eq. 3's h f(x_t + h v_t), with the same K as the matrix)
 * on the pattern that pc_assemble_pattern produced for the same contacts. Pinned vertex
 * i: row and column blocks zero except A_ii = m_i I, b_i = 0.
 * dres (optional, float[V][9], may be NULL) receives the "difference-form" diagonal
 * D_i = m_i I - sum over pinned neighbours j of the unzeroed block A_ij, with which
 * (A p)_i = D_i p_i + sum_{j != i} A_ij (p_j - p_i) holds exactly for this model (every
 * element's Hessian rows sum to zero). Element contributions are combined per row by a
 * warp-level reduction in a fixed order (no atomics): results are deterministic and
 * A is bitwise symmetric. x, v: device float[V][3]. Does not synchronize. */
PC_API pc_status pc_assemble_values(pc_ctx *ctx, const pc_bsr *A, const float *x, const float *v,
                             const pc_contacts *contacts, float h, float *vals, float *b, float *dres,
                             void *stream);

/* y = A x for a BSR matrix (V rows). With dres != NULL the product is formed in the
 * difference form above (the diagonal blocks in vals are not used). */
PC_API pc_status pc_bsr_spmv(pc_ctx *ctx, const pc_bsr *A, const float *vals, const float *dres, const float *x,
                      float *y, void *stream);

/* Sec. 2.5: solve A dv = b by preconditioned conjugate gradients (Jacobi: the scalar
 * diagonal of A, or its 3x3 diagonal blocks). dv holds the initial guess on entry and the
 * solution on exit. opts == NULL uses the defaults. With dres != NULL the matrix
 * products use the difference form (more accurate for stiff systems whose rows sum to
 * the mass).
 * PC_PREC_FP32: FP32 vectors and products, FP64 dot-product accumulation; stops on the
 * recurrence residual. The FP64 residual of the FP32 iterate is reported in info.
 * PC_PREC_MIXED: the matrix and the PCG vectors stay FP32, but the solution is kept as
 * an FP64 accumulator plus an FP32 increment. Whenever the recurrence residual has
 * dropped by `refresh` (or every `refresh_every` iterations, and whenever it meets tol),
 * the increment is added into the accumulator in FP64 and the residual r = b - A dv is
 * recomputed in FP64 and replaces the recurrence residual, without restarting the search
 * direction (iterative refinement by residual replacement). The solve stops when the
 * FP64 residual meets tol.
 * info (host, may be NULL) receives iterations and the FP64 true relative residual.
 * Returns PC_ERR_NOT_CONVERGED (dv = last iterate) or PC_ERR_NONFINITE when those occur,
 * and PC_ERR_ARG, before any product runs, when the pattern is malformed (row pointers
 * decreasing or outside [0, A->nnzb], a column index outside [0, V)).
 * Synchronizes `stream`. */
PC_API pc_status pc_pcg_solve(pc_ctx *ctx, const pc_bsr *A, const float *vals, const float *dres, const float *b,
                       float *dv, const pc_solve_opts *opts, pc_solve_info *info, void *stream);

/* After a PC_PREC_MIXED pc_pcg_solve or pc_step on this context: copy the solve's FP64
 * solution accumulator -- the iterate whose FP64 residual the stop test measured; the
 * returned dv is its rounding to FP32 -- into dv64 (device double[V][3]). On stiff
 * systems (|A| |dv| much larger than |b|) the FP32 rounding alone can raise the relative
 * residual far above tol, so this is the solution to check a tolerance against.
 * Does not synchronize. */
PC_API pc_status pc_get_solution64(pc_ctx *ctx, double *dv64, void *stream);

/* Batched solve of many independent systems (garments) in ONE persistent PCG launch.
 * The context holds the union of the garments' meshes; instance k owns the contiguous
 * rows inst_rows[k] .. inst_rows[k+1]-1 (host array of n_inst + 1 entries, first 0, last
 * V, every instance at least 32 rows, n_inst <= 1024) and no matrix block may couple two
 * instances (checked: PC_ERR_ARG). Each instance runs Jacobi-PCG with its own scalars
 * and stop test |b_k - A_k dv_k| / |b_k| <= tol, with FP64 residual replacement as in
 * PC_PREC_MIXED (refresh, refresh_every); finished instances drop out while the others
 * continue. The launch is cooperative (all CTAs co-resident) with bounded grid-wide
 * waits (PC_ERR_TIMEOUT instead of a hang). On the first call for a matrix shape an
 * autotuner times short solves for each tile and schedule (the SpMV phase's stage width
 * x its entry order x the grid: 16, 32, 64 CTAs or 2..5 per SM) and keeps the fastest
 * (pc_batched_config reports the choice). info: host array of n_inst results, may be
 * NULL. Returns the first non-OK instance status. Synchronizes `stream`.
 * (The paper solves one garment system per step; batching is this library's extension.) */
PC_API pc_status pc_pcg_solve_batched(pc_ctx *ctx, const pc_bsr *A, const float *vals, const float *dres,
                                      const float *b, float *dv, int32_t n_inst, const int32_t *inst_rows,
                                      const pc_solve_opts *opts, pc_solve_info *info, void *stream);

/* Tile and schedule chosen by the batched autotuner: the grid in CTAs (0 if not tuned
 * yet), the SpMV entry order (0: strided, CTA b takes entries b, b+G, ...; 1: contiguous
 * chunks), the SpMV phase's stage width in blocks per row of a 32-row tile (14 or 18), the
 * seven candidate grid sizes (grid_sizes[7]: 16, 32 and 64 CTAs where that is below one
 * per SM, else 0; then 2..5 CTAs per SM) and the timings (ms) of every candidate,
 * tune_ms[14 * (width == 18) + 7 * order + grid index] (0 where not tried: a grid that
 * does not fit). Host pointers, may be NULL. */
PC_API pc_status pc_batched_config(pc_ctx *ctx, int32_t *grid, int32_t *spmv_order, int32_t *stage_blocks,
                                   int32_t *grid_sizes, float *tune_ms);

/* Cycle budget of each grid-barrier wait in the persistent batched solver and in the
 * fused PCG update of pc_pcg_solve / pc_step (software barriers polling an arrival
 * counter). A wait longer than the budget aborts: in the batched solver every CTA leaves at
 * its next barrier, no result is written back and dv keeps its initial guess; in the
 * single-system solve the iteration stops; the calls return PC_ERR_TIMEOUT with the
 * context still usable. cycles <= 0 restores the default of 2^31 SM cycles (about
 * a second at 2 GHz). A budget of a few cycles makes every solve time out: that is how the
 * timeout path is exercised without a hang. Host-only; takes effect at the next launch. */
PC_API pc_status pc_set_barrier_wait(pc_ctx *ctx, int64_t cycles);

/* Proximity query for the one-sided thickness contact model: every pair of a vertex p
 * and a triangle t = (a, b, c) of the context's mesh whose distance at positions x (device
 * float[V][3]) is below delta, t touching neither p nor a mesh-edge neighbour of p,
 * written as pairs (device int32[cap][4]: p, a, b, c) and the barycentric weights of the
 * point of t closest to p (device float[cap][3]), ordered by p, then by triangle index.
 * The closest point and the test d^2 < delta^2 are evaluated in FP32 with one rounding
 * per operation in a fixed order, so the result is reproducible bit for bit. *n_out
 * (host) receives the pair count; PC_ERR_CAPACITY when it exceeds cap (nothing written),
 * PC_ERR_ARG when delta <= 0 or a position is too far from the origin for the cell grid
 * (|x| / cell size >= 2^20). Synchronizes `stream`. Feed the result to pc_step /
 * pc_assemble_pattern as the step's contacts (at most the context's max_contacts). */
PC_API pc_status pc_proximity_query(pc_ctx *ctx, const float *x, float delta, int32_t cap, int32_t *pairs, float *w,
                                    int32_t *n_out, void *stream);

/* One batched time step: the dynamic pattern of the whole union (synchronous), then a
 * CUDA graph holding value assembly, the persistent batched solve and v += dv,
 * x += h v, replayed (updated in place) from step to step. Instances as for
 * pc_pcg_solve_batched; info receives one result per instance. The update applies to
 * the instances whose solve ended PC_OK or PC_ERR_NOT_CONVERGED; an instance that failed
 * (PC_ERR_NONFINITE) keeps its x and v, and after PC_ERR_TIMEOUT no instance moves. */
PC_API pc_status pc_step_batched(pc_ctx *ctx, float *x, float *v, const pc_contacts *contacts, int32_t n_inst,
                                 const int32_t *inst_rows, const pc_step_opts *opts, pc_solve_info *info,
                                 void *stream);

/* Allocation-free variant of pc_pcg_solve (the paper has no counterpart): the same
 * solver, for callers that cannot allocate device memory and so cannot hold a context --
 * for example a plug-in inside a host application that owns and pre-reserves all GPU
 * memory itself, or a real-time loop that must never call cudaMalloc because an
 * allocation can synchronize the device and stall the frame.
 * All scratch (PCG vectors, FP64 accumulator, reduction partials and scalars) lives in
 * one static device array inside the library sized for PC_STATIC_MAX_ROWS rows (about
 * 2.7 MB, held by every GPU that loads the library until the process exits); nothing is
 * allocated. The caller passes the system (V rows, as for pc_pcg_solve) and the output.
 * V > PC_STATIC_MAX_ROWS returns PC_ERR_CAPACITY before any device work; a pattern whose
 * row pointers or column indices do not fit V rows and A->nnzb blocks returns PC_ERR_ARG
 * before any product runs. Options, stop tests and results are those of pc_pcg_solve,
 * except opts->storage: there is no room for a second layout of the matrix, so every
 * storage choice (including the default PC_STORAGE_OFFDIAG) is read as PC_STORAGE_FULL
 * -- the products stream the caller's matrix; the solution is the same up to summation
 * order. The stage shape of the product is chosen per solve as in pc_pcg_solve, and so is
 * opts->schedule: the cluster schedule keeps its working set in the cluster's shared
 * memory and needs no scratch beyond the scalars, so small systems solve there as with a
 * context (its cluster-size query and shared-memory set-up are host-side, no allocation).
 * Each call looks up the array's device address on the current device and sets the
 * kernels' shared-memory limit (host-side set-up, no allocation); make the first call on
 * a device before any stream capture. Every call on a device shares the array, which
 * keeps the last call's contents; each call clears what must start at zero (scalars,
 * reduction ticket, barrier word, error bits) on entry. Calls that overlap on the GPU
 * (concurrent streams, or several host threads on one device) race and must be
 * serialized by the caller. Synchronizes `stream`. */
#define PC_STATIC_MAX_ROWS 16384
PC_API pc_status pc_pcg_solve_static(int32_t V, const pc_bsr *A, const float *vals, const float *dres,
                                     const float *b, float *dv, const pc_solve_opts *opts, pc_solve_info *info,
                                     void *stream);

/* ---------------------------------------------------------------- row-partitioned solve
 * Sec. 3.1, Eq. 4-5: the system's rows are split into contiguous blocks, one per rank
 * (one process and GPU each). Each rank holds its rows of A, of the vectors and of b;
 * vector operations need no communication, and the product needs the "halo": the entries
 * of the direction owned by other ranks that the rank's blocks reference. The product
 * runs as an own-column part (started before the halo arrives) plus a halo part, so the
 * exchange overlaps the multiplication (the paper's pipelined SpMV, with each peer's
 * column block reduced to the entries actually referenced).
 * Communication is the caller's: pc_comm holds two callbacks, implemented with NCCL,
 * MPI, gloo or anything else, that every rank calls in the same order with the same
 * sizes. Both must leave their results visible to work enqueued later on `stream`
 * (either enqueue on it, or synchronize it, transfer and return), and return 0 on
 * success (anything else makes the library call return PC_ERR_CUDA). */
typedef struct {
    void *user;
    /* Sum n doubles over all ranks, in place. vals: DEVICE pointer. */
    int32_t (*allreduce_sum)(void *user, double *vals, int32_t n, void *stream);
    /* Point-to-point exchange among all ranks: to every rank j this rank sends
     * send_bytes[j] bytes starting at send + send_off[j] and receives recv_bytes[j] bytes
     * from rank j into recv + recv_off[j]. send, recv: DEVICE pointers; the four arrays
     * are HOST arrays of nranks entries (the rank's own entries are 0). */
    int32_t (*exchange)(void *user, const void *send, const int64_t *send_off, const int64_t *send_bytes,
                        void *recv, const int64_t *recv_off, const int64_t *recv_bytes, void *stream);
} pc_comm;

typedef struct pc_dist pc_dist;

/* Rows per rank: contiguous blocks with boundaries on multiples of 32 rows, balanced by
 * block count when row_ptr (HOST, V+1 entries) is given, else by rows. row_starts: HOST
 * int32[nranks + 1] (0 .. V). Host-only; needs no GPU. */
PC_API pc_status pc_dist_partition(int32_t V, const int32_t *row_ptr, int32_t nranks, int32_t *row_starts);

/* The halo a rank needs, from the remote columns its rows reference (HOST arrays, any
 * order, repeats allowed): halo (HOST int32[n_remote]) receives the distinct columns in
 * ascending order, *n_halo their count, counts (HOST int64[nranks]) how many each rank
 * owns. PC_ERR_ARG when a column is outside [0, V) or is one of the rank's own rows.
 * Host-only; needs no GPU. */
PC_API pc_status pc_dist_halo(int32_t nranks, const int32_t *row_starts, int32_t rank, int64_t n_remote,
                              const int32_t *remote, int32_t *halo, int64_t *n_halo, int64_t *counts);

/* Create rank `rank` of `nranks` on the current device: it owns global rows
 * [row_starts[rank], row_starts[rank+1]) (HOST int32[nranks+1], from pc_dist_partition or
 * any non-decreasing split with every rank non-empty). max_blocks: capacity for the rank's
 * blocks; max_halo: capacity for halo and send entries (0: every remote row).
 * Allocates the rank's scratch and a second stream for the exchange. */
PC_API pc_status pc_dist_create(pc_dist **out, int32_t rank, int32_t nranks, const int32_t *row_starts,
                                int64_t max_blocks, int64_t max_halo);
PC_API pc_status pc_dist_destroy(pc_dist *d);

/* Plan the rank's part of a new pattern (once per step, as the pattern changes): A->row_ptr
 * points at the rank's n_own + 1 row pointers (DEVICE; global block positions, e.g. the
 * full system's row_ptr + row0), A->col_idx at the column indices those positions index
 * (DEVICE, global columns), A->nnzb the total block count they index. Finds the remote
 * columns, the halo and its owners, exchanges the requests with the peers (two calls of
 * comm->exchange), and splits the rows into the own part (local columns) and the halo
 * part. PC_ERR_ARG for indices out of range, PC_ERR_CAPACITY when the rank's blocks or
 * halo exceed the capacities. Synchronizes `stream`; collective (every rank calls it). */
PC_API pc_status pc_dist_plan(pc_dist *d, const pc_bsr *A, const pc_comm *comm, void *stream);

/* Sizes of the last plan (HOST pointers, each may be NULL). */
PC_API pc_status pc_dist_sizes(const pc_dist *d, int32_t *row0, int32_t *row1, int64_t *n_halo, int64_t *n_send,
                               int64_t *nnzb_own, int64_t *nnzb_halo);

/* Jacobi-PCG (Sec. 2.5) on the partitioned system, every rank on its rows: vals (DEVICE)
 * is indexed like the col_idx array the plan was given (the rank reads its own range);
 * dres (DEVICE float[n_own][9], may be NULL) the difference-form diagonal of its rows;
 * b and dv (DEVICE float[n_own][3]) its rows of the right-hand side and of the solution
 * (guess in, solution out). Options as pc_pcg_solve (PC_PREC_FP32 or PC_PREC_MIXED, scalar
 * Jacobi; storage and fuse are not used). The global dot products are the all-reduced
 * sums of the ranks' partial sums, so every rank gets the same scalars, iterations and
 * stop decision; info (HOST, may be NULL) receives the global iteration count and the
 * FP64 relative residual of the whole system. Collective; synchronizes `stream`. */
PC_API pc_status pc_dist_pcg_solve(pc_dist *d, const float *vals, const float *dres, const float *b, float *dv,
                                   const pc_solve_opts *opts, const pc_comm *comm, pc_solve_info *info, void *stream);

/* One time step on device state: pattern, values (with the difference-form diagonal),
 * PCG solve, then v += dv, x += h v. Uses buffers owned by the context. dv_out (device
 * float[V][3], may be NULL) receives dv. Synchronizes `stream`. */
PC_API pc_status pc_step(pc_ctx *ctx, float *x, float *v, const pc_contacts *contacts, const pc_step_opts *opts,
                  float *dv_out, pc_step_info *info, void *stream);

/* The previous step's dv that PC_WARM_PREV starts from (and the learned guess reads):
 * get copies it to dv (device float[V][3]; zeros and *valid = 0 before the first step),
 * set restores it (NULL: forget it, as before the first step). With positions,
 * velocities and the step index this is the integrator state a checkpoint needs.
 * Synchronize `stream`. */
PC_API pc_status pc_get_prev_dv(pc_ctx *ctx, float *dv, int32_t *valid, void *stream);
PC_API pc_status pc_set_prev_dv(pc_ctx *ctx, const float *dv, void *stream);

/* pc_step on HOST buffers: copies x, v (host float[V][3]) and the contacts (host
 * int32[n][4], float[n][3]) to the device, runs pc_step, and copies x and v back. Host
 * buffers may be pageable or pinned. */
PC_API pc_status pc_step_host(pc_ctx *ctx, float *x_host, float *v_host, int32_t n_contacts, const int32_t *pairs_host,
                       const float *w_host, const pc_step_opts *opts, pc_step_info *info, void *stream);

/* ---------------------------------------------------------------- learned warm start
 * The paper has no learned component; this is an extension built on its integrator. A
 * per-vertex MLP predicts the initial guess of the Eq. 3 solve:
 *   features (PC_MLP_IN = 12 per vertex): v_i; the previous step's dv_i; the internal
 *     force per unit mass at the first-order end-of-step position times the vertex's mean
 *     rest edge length l_i, l_i (b_i / h - m_i g) / m_i with b the assembled right-hand
 *     side (the length scale makes the membrane's share independent of the grid spacing,
 *     so a network trained on one resolution sees the same inputs on another); the mean
 *     of the previous dv over the vertex's mesh-edge neighbours;
 *   network: 12 -> 64 -> 64 -> 3 with ReLU, on inputs standardised by stats
 *     (mu_x[12], sd_x[12], mu_y[3], sd_y[3]); it predicts the change of dv from the
 *     previous step: dv0 = dv_prev + sd_y * y + mu_y;
 *   params: float[PC_MLP_NPARAMS] = W1[64][12], b1[64], W2[64][64], b2[64], W3[3][64],
 *     b3[3] (row-major [out][in]).
 * Every matrix product runs on the tensor cores with BF16 operands (weights, standardised
 * inputs, activations and back-propagated signals rounded to BF16) and FP32
 * accumulation; the FP32 params are the master weights. Training minimises
 * L = 1/(2n) sum over rows and outputs of (y - t)^2, t the standardised target
 * dv - dv_prev, with Adam. All pointers are device pointers unless stated. */
#define PC_MLP_IN 12
#define PC_MLP_HIDDEN 64
#define PC_MLP_OUT 3
#define PC_MLP_NPARAMS 5187
#define PC_MLP_NSTATS 30

typedef struct pc_mlp pc_mlp;  /* training state: Adam moments, step count, reduction scratch */

typedef struct {
    float lr, beta1, beta2, eps;
} pc_adam_opts;

/* The 12 raw features of every vertex of a cloth state: v, dv_prev (float[V][3]), b the
 * right-hand side assembled for this state (pc_assemble_values), h the time step (the
 * rest edge lengths come from the context).
 * feat: float[V][12]. Does not synchronize. */
PC_API pc_status pc_mlp_features(pc_ctx *ctx, const float *v, const float *dv_prev, const float *b, float h,
                                 float *feat, void *stream);

/* Create / destroy training state (on the current device). */
PC_API pc_status pc_mlp_create(pc_mlp **out);
PC_API pc_status pc_mlp_destroy(pc_mlp *m);
/* Zero the Adam moments and the step count. */
PC_API pc_status pc_mlp_reset(pc_mlp *m, void *stream);
/* Adam state for checkpoints: the first and second moments (device float[PC_MLP_NPARAMS]
 * each) and the step count (host). Get copies out, set copies in. Synchronize `stream`. */
PC_API pc_status pc_mlp_get_state(pc_mlp *m, float *m1, float *m2, int64_t *t, void *stream);
PC_API pc_status pc_mlp_set_state(pc_mlp *m, const float *m1, const float *m2, int64_t t, void *stream);

/* Training rows: feat float[*][12] as pc_mlp_features writes it and target float[*][3]
 * the solution dv of the same step (pc_step's dv_out); the network's target is
 * dv - dv_prev, dv_prev being features 3..5 of the row.
 * Standardisation statistics of n training rows: per-column mean and population standard
 * deviation (FP64 sums, floor 1e-12) of the 12 features and of the 3 target components,
 * written to stats float[PC_MLP_NSTATS]. Deterministic. Does not synchronize. */
PC_API pc_status pc_mlp_stats(pc_mlp *m, int64_t n, const float *feat, const float *target, float *stats,
                              void *stream);

/* Inference: dv0[r] = dv_prev[r] + sd_y * net((feat[r] - mu_x) / sd_x) + mu_y for n rows
 * (dv_prev may be NULL = 0); rows with fixed[r] != 0 (uint8[n], may be NULL) get 0.
 * Does not synchronize. */
PC_API pc_status pc_mlp_infer(int64_t n, const float *params, const float *stats, const float *feat,
                              const float *dv_prev, const uint8_t *fixed, float *dv0, void *stream);

/* Gradient of L over a batch of n rows: rows (int32[n], may be NULL = rows 0..n-1) index
 * feat and target (training rows as above). grad: float[NPARAMS]
 * (partials summed in a fixed order: deterministic). loss (host, may be NULL) receives L
 * and then the call synchronizes `stream`. */
PC_API pc_status pc_mlp_grad(pc_mlp *m, int64_t n, const int32_t *rows, const float *params, const float *stats,
                             const float *feat, const float *target, float *grad, double *loss, void *stream);

/* One Adam step on params (in place) with the gradient of that batch. */
PC_API pc_status pc_mlp_train_step(pc_mlp *m, int64_t n, const int32_t *rows, float *params, const float *stats,
                                   const float *feat, const float *target, const pc_adam_opts *o, double *loss,
                                   void *stream);

/* One Adam step on params with a given gradient (float[NPARAMS]). */
PC_API pc_status pc_mlp_adam_apply(pc_mlp *m, float *params, const float *grad, const pc_adam_opts *o,
                                   void *stream);

/* Attach a trained network to a context for PC_WARM_MLP steps (the pointers are kept,
 * not copied; NULL, NULL detaches). Allocates the context's feature and guess scratch
 * on first use. */
PC_API pc_status pc_set_warm_mlp(pc_ctx *ctx, const float *params, const float *stats);

/* Kernel launches issued by this context since creation (all entry points). */
PC_API int64_t pc_launch_count(const pc_ctx *ctx);

/* When enabled, the PCG loop brackets two SpMV launches of each chunk of iterations
 * (check_every) with CUDA events on its stream: the chunk's first launch, which follows
 * the host's convergence check, and its middle one, which stands for the chunk's other
 * launches (weighted by the iterations the chunk ran); pc_step brackets its assembly the
 * same way. pc_spmv_stats returns (launches represented, their total ms, block count of
 * the last matrix) and resets the counters. */
PC_API pc_status pc_set_profiling(pc_ctx *ctx, int32_t enable);
PC_API pc_status pc_spmv_stats(pc_ctx *ctx, int64_t *launches, double *total_ms, int64_t *nnzb);
/* Likewise for pc_step's assembly (pattern and values, Sec. 3.2.2): (steps timed, total
 * ms), then reset. */
PC_API pc_status pc_assembly_stats(pc_ctx *ctx, int64_t *steps, double *total_ms);
/* Likewise for solves run on the cluster schedule (PC_SCHED_CLUSTER): (solves timed,
 * their PCG iterations, total ms of the solve kernel), then reset. */
PC_API pc_status pc_cluster_stats(pc_ctx *ctx, int64_t *solves, int64_t *iters, double *total_ms);

#ifdef __cplusplus
}
#endif

#endif /* PCLOTH_H */
