// Time step driver (Sec. 2.5: each step assembles Eq. 3 anew and solves it) and small
// ABI utilities.
#include "pc_internal.cuh"

extern "C" const char *pc_status_string(pc_status s)
{
    switch (s) {
    case PC_OK: return "ok";
    case PC_ERR_ARG: return "invalid argument";
    case PC_ERR_CAPACITY: return "output capacity too small";
    case PC_ERR_NOT_CONVERGED: return "PCG did not converge within max_iter";
    case PC_ERR_NONFINITE: return "non-finite value in the system or a PCG scalar";
    case PC_ERR_TIMEOUT: return "bounded device wait timed out";
    case PC_ERR_CUDA: return "CUDA runtime error";
    case PC_ERR_MESH: return "invalid mesh (degenerate triangle or non-manifold edge)";
    default: return "unknown status";
    }
}

extern "C" int64_t pc_launch_count(const pc_ctx *ctx) { return ctx ? ctx->launches : 0; }

extern "C" pc_status pc_set_profiling(pc_ctx *ctx, int32_t enable)
{
    if (!ctx) return PC_ERR_ARG;
    ctx->profiling = enable ? 1 : 0;
    return PC_OK;
}

extern "C" pc_status pc_spmv_stats(pc_ctx *ctx, int64_t *launches, double *total_ms, int64_t *nnzb)
{
    if (!ctx) return PC_ERR_ARG;
    if (launches) *launches = ctx->spmv_launches;
    if (total_ms) *total_ms = ctx->spmv_ms;
    if (nnzb) *nnzb = ctx->spmv_nnzb;
    ctx->spmv_launches = 0;
    ctx->spmv_ms = 0.0;
    return PC_OK;
}

extern "C" pc_status pc_assembly_stats(pc_ctx *ctx, int64_t *steps, double *total_ms)
{
    if (!ctx) return PC_ERR_ARG;
    if (steps) *steps = ctx->asm_steps;
    if (total_ms) *total_ms = ctx->asm_ms;
    ctx->asm_steps = 0;
    ctx->asm_ms = 0.0;
    return PC_OK;
}

extern "C" pc_status pc_cluster_stats(pc_ctx *ctx, int64_t *solves, int64_t *iters, double *total_ms)
{
    if (!ctx) return PC_ERR_ARG;
    if (solves) *solves = ctx->cl_solves;
    if (iters) *iters = ctx->cl_iters;
    if (total_ms) *total_ms = ctx->cl_ms;
    ctx->cl_solves = 0;
    ctx->cl_iters = 0;
    ctx->cl_ms = 0.0;
    return PC_OK;
}

extern "C" pc_status pc_step(pc_ctx *ctx, float *x, float *v, const pc_contacts *contacts, const pc_step_opts *opts,
                             float *dv_out, pc_step_info *info, void *stream)
{
    if (!ctx || !x || !v || !opts) return PC_ERR_ARG;
    if (!(opts->h > 0.0f)) return PC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    pc_bsr A{ctx->A_rp, ctx->A_ci, ctx->A_cap, 0};
    if (ctx->profiling) PC_CUDA_TRY(cudaEventRecord(ctx->ev[2], st));
    PC_TRY(pc_assemble_pattern(ctx, contacts, &A, stream));
    PC_TRY(pc_assemble_values(ctx, &A, x, v, contacts, opts->h, ctx->A_vals, ctx->A_b, ctx->A_dres, stream));
    if (ctx->profiling) {
        PC_CUDA_TRY(cudaEventRecord(ctx->ev[3], st));
        PC_CUDA_TRY(cudaEventSynchronize(ctx->ev[3]));
        float ms = 0.f;
        PC_CUDA_TRY(cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]));
        ctx->asm_ms += ms;
        ctx->asm_steps += 1;
    }
    // A_dv holds the previous step's dv (zeros before the first step); choose the guess
    if (!ctx->has_prev_dv) PC_CUDA_TRY(cudaMemsetAsync(ctx->A_dv, 0, sizeof(float) * 3 * (size_t)ctx->V, st));
    int32_t guess = PC_WARM_ZERO;
    double guess_res[3], guess_energy[3], guess_coef[2] = {0.0, 0.0}, combo_energy = 0.0;
    PC_TRY(pc_warm_guess(ctx, &A, v, opts->h, opts->warm_start, opts->feat_out, &guess, guess_res, guess_energy,
                         guess_coef, &combo_energy, st));
    pc_solve_info si{};
    pc_status s = pc_pcg_solve(ctx, &A, ctx->A_vals, ctx->A_dres, ctx->A_b, ctx->A_dv, &opts->solve, &si, stream);
    if (info) {
        info->nnzb = A.nnzb;
        info->solve = si;
        info->guess = guess;
        info->pad = 0;
        for (int k = 0; k < 3; ++k) {
            info->guess_res[k] = guess_res[k];
            info->guess_energy[k] = guess_energy[k];
        }
        info->guess_coef[0] = guess_coef[0];
        info->guess_coef[1] = guess_coef[1];
        info->combo_energy = combo_energy;
    }
    if (s != PC_OK && s != PC_ERR_NOT_CONVERGED) return s;
    ctx->has_prev_dv = 1;
    PC_TRY(pc_update_state(ctx, x, v, ctx->A_dv, opts->h, st));
    if (dv_out)
        PC_CUDA_TRY(cudaMemcpyAsync(dv_out, ctx->A_dv, sizeof(float) * 3 * (size_t)ctx->V, cudaMemcpyDeviceToDevice, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    return s;
}

extern "C" pc_status pc_step_host(pc_ctx *ctx, float *x_host, float *v_host, int32_t n_contacts,
                                  const int32_t *pairs_host, const float *w_host, const pc_step_opts *opts,
                                  pc_step_info *info, void *stream)
{
    if (!ctx || !x_host || !v_host || !opts) return PC_ERR_ARG;
    if (n_contacts < 0 || n_contacts > ctx->max_contacts || (n_contacts > 0 && (!pairs_host || !w_host)))
        return PC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t vb = sizeof(float) * 3 * (size_t)ctx->V;
    float *dx = ctx->h_state, *dvel = ctx->h_state + 3ll * ctx->V;
    PC_CUDA_TRY(cudaMemcpyAsync(dx, x_host, vb, cudaMemcpyHostToDevice, st));
    PC_CUDA_TRY(cudaMemcpyAsync(dvel, v_host, vb, cudaMemcpyHostToDevice, st));
    if (n_contacts > 0) {
        PC_CUDA_TRY(cudaMemcpyAsync(ctx->h_pairs, pairs_host, sizeof(int32_t) * 4 * (size_t)n_contacts,
                                    cudaMemcpyHostToDevice, st));
        PC_CUDA_TRY(cudaMemcpyAsync(ctx->h_w, w_host, sizeof(float) * 3 * (size_t)n_contacts, cudaMemcpyHostToDevice, st));
    }
    pc_contacts c{n_contacts, ctx->h_pairs, ctx->h_w};
    pc_status s = pc_step(ctx, dx, dvel, &c, opts, nullptr, info, stream);
    if (s != PC_OK && s != PC_ERR_NOT_CONVERGED) return s;
    PC_CUDA_TRY(cudaMemcpyAsync(x_host, dx, vb, cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaMemcpyAsync(v_host, dvel, vb, cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    return s;
}

extern "C" pc_status pc_get_prev_dv(pc_ctx *ctx, float *dv, int32_t *valid, void *stream)
{
    if (!ctx || !dv || !valid) return PC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    *valid = ctx->has_prev_dv;
    if (ctx->has_prev_dv)
        PC_CUDA_TRY(cudaMemcpyAsync(dv, ctx->A_dv, sizeof(float) * 3 * (size_t)ctx->V, cudaMemcpyDeviceToDevice, st));
    else
        PC_CUDA_TRY(cudaMemsetAsync(dv, 0, sizeof(float) * 3 * (size_t)ctx->V, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    return PC_OK;
}

extern "C" pc_status pc_set_prev_dv(pc_ctx *ctx, const float *dv, void *stream)
{
    if (!ctx) return PC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (dv) {
        PC_CUDA_TRY(cudaMemcpyAsync(ctx->A_dv, dv, sizeof(float) * 3 * (size_t)ctx->V, cudaMemcpyDeviceToDevice, st));
        ctx->has_prev_dv = 1;
    } else {
        PC_CUDA_TRY(cudaMemsetAsync(ctx->A_dv, 0, sizeof(float) * 3 * (size_t)ctx->V, st));
        ctx->has_prev_dv = 0;
    }
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    return PC_OK;
}
