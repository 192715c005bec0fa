// C ABI of libawg (include/awg.h): argument checks, handle lifetime, setup
// orchestration and the apply / PCG entry points.

#include "awg_common.cuh"
#include "ops.cuh"
#include "block.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <new>

namespace awg {

awg_status dalloc(Handle* h, DevBuf& b, size_t bytes) {
    if (b.p) dfree(h, b);
    bytes = std::max<size_t>(bytes, 8);
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return e == cudaErrorMemoryAllocation ? AWG_ERR_OOM : AWG_ERR_CUDA;
    }
    b.bytes = bytes;
    h->device_bytes += bytes;
    return AWG_OK;
}

void dfree(Handle* h, DevBuf& b) {
    if (b.p) {
        cudaFree(b.p);
        h->device_bytes -= b.bytes;
    }
    b.p = nullptr;
    b.bytes = 0;
}

awg_status upload(Handle* h, DevBuf& b, const void* src, size_t bytes) {
    AWG_TRY(dalloc(h, b, bytes));
    AWG_CUDA(cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, h->stream));
    AWG_CUDA(cudaStreamSynchronize(h->stream));
    return AWG_OK;
}

awg_status read_flag(Handle* h, int* out) {
    AWG_CUDA(cudaMemcpyAsync(h->h_flag, h->flag.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    AWG_CUDA(cudaStreamSynchronize(h->stream));
    *out = *h->h_flag;
    return AWG_OK;
}

awg_status pcg1(Handle* h, int prec, int stage, const double* b, double* x, double rtol, int* iters,
                double* relres, cudaStream_t s);

void free_all(Handle* h) {
    DevBuf* bufs[] = {&h->rowptr, &h->colidx, &h->val, &h->ns, &h->sub_ptr, &h->sub_idx,
                      &h->inc_ptr, &h->inc_pos, &h->inc_sub, &h->pos_sub, &h->dvec, &h->mmu,
                      &h->bval, &h->dense_off, &h->g32_off, &h->nm, &h->nstrict, &h->nm_ptr, &h->vm_off,
                      &h->Vm, &h->lam_m, &h->sigma, &h->modes, &h->mode_ptr, &h->z_off, &h->Z,
                      &h->E, &h->Einv, &h->wcol_ptr, &h->Wcm, &h->F64, &h->ws, &h->flag,
                      &h->bws, &h->bval32, &h->bvm32, &h->blam32, &h->blam64, &h->bz32,
                      &h->ul_gt, &h->ul_gtoff, &h->ul_kcpre, &h->ul_tsub, &h->ul_trt, &h->g1buf, &h->g1cnt,
                      &h->bws2};
    for (DevBuf* b : bufs) dfree(h, *b);
    for (int k = 0; k < 9; k++) {
        dfree(h, h->oz_q[k]);
        dfree(h, h->oz_ex[k]);
        h->oz_dim[k] = 0;
    }
    for (auto& P : h->prec) {
        dfree(h, P.G);
        dfree(h, P.W);
        dfree(h, P.Finv);
        dfree(h, P.inexInv);
        dfree(h, P.rscale);
        dfree(h, P.cscale);
        for (DevBuf* b : {&P.corr_rowptr, &P.corr_col, &P.corr_val, &P.corr_colptr, &P.corr_row, &P.corr_cval,
                          &P.sp_rowptr, &P.sp_col, &P.sp_val, &P.sp_colptr, &P.sp_row, &P.sp_cval})
            dfree(h, *b);
    }
    for (int g = 0; g < 4; g++) {
        if (h->g1_exec[g]) cudaGraphExecDestroy(h->g1_exec[g]);
        if (h->g1_graph[g]) cudaGraphDestroy(h->g1_graph[g]);
        h->g1_exec[g] = nullptr;
        h->g1_graph[g] = nullptr;
    }
    for (int g = 0; g < 12; g++) {
        if (h->bg2_exec[g]) cudaGraphExecDestroy(h->bg2_exec[g]);
        if (h->bg2_graph[g]) cudaGraphDestroy(h->bg2_graph[g]);
        h->bg2_exec[g] = nullptr;
        h->bg2_graph[g] = nullptr;
    }
    for (cudaEvent_t* e : {&h->ev2_fork, &h->ev2_mid, &h->ev2_join, &h->ev2_in, &h->ev2_out}) {
        if (*e) cudaEventDestroy(*e);
        *e = nullptr;
    }
    if (h->side2) cudaStreamDestroy(h->side2);
    if (h->hp2) cudaStreamDestroy(h->hp2);
    h->side2 = h->hp2 = nullptr;
    for (int g = 0; g < 12; g++) {
        if (h->bg_exec[g]) cudaGraphExecDestroy(h->bg_exec[g]);
        if (h->bg_graph[g]) cudaGraphDestroy(h->bg_graph[g]);
        h->bg_exec[g] = nullptr;
        h->bg_graph[g] = nullptr;
    }
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    h->ev_pool.clear();
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_mid) cudaEventDestroy(h->ev_mid);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->hp) cudaStreamDestroy(h->hp);
    h->ev_fork = h->ev_join = h->ev_mid = h->ev_in = h->ev_out = nullptr;
    h->side = h->hp = nullptr;
    if (h->h_flag) cudaFreeHost(h->h_flag);
    if (h->h_scal) cudaFreeHost(h->h_scal);
    h->h_flag = nullptr;
    h->h_scal = nullptr;
}

// Streams, events, pinned host words and the status flag of a handle (the
// runtime part of a handle, shared by awg_setup and awg_load).
awg_status runtime_init(Handle* h) {
    AWG_CUDA(cudaMallocHost(&h->h_flag, sizeof(int)));
    AWG_CUDA(cudaMallocHost(&h->h_scal, 16 * sizeof(double)));
    int prio_least = 0, prio_greatest = 0;
    AWG_CUDA(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
    AWG_CUDA(cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, prio_least));
    AWG_CUDA(cudaStreamCreateWithPriority(&h->hp, cudaStreamNonBlocking, prio_greatest));
    AWG_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    AWG_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    AWG_CUDA(cudaEventCreateWithFlags(&h->ev_mid, cudaEventDisableTiming));
    AWG_CUDA(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    AWG_CUDA(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
    AWG_TRY(dalloc(h, h->flag, sizeof(int)));
    return AWG_OK;
}

static double now_ms() {
    return std::chrono::duration<double, std::milli>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

}  // namespace awg

using namespace awg;

extern "C" {

void awg_default_options(awg_options* opt) {
    if (!opt) return;
    opt->variant = AWG_H3_AD;
    opt->h2 = AWG_H2_NN_HYB;
    opt->tau_flat = 10.0;
    opt->precisions = 1 << AWG_FP64;
    opt->zero_rtol = 1e-12;
    opt->w_rtol = 1e-13;
    opt->w_maxit = 500;
    opt->maxit = 1000;
    opt->verbose = 0;
    opt->w_precision = AWG_MIXED_FP32;
    opt->geneo_solver = 0;
    opt->geneo_block = 8;
    opt->geneo_maxit = 60;
    opt->learned_params = nullptr;
    opt->autotune = 1;
    opt->w16_keep = 0.1;
    opt->block_tensor_cores = 1;
    opt->coarse_tensor_cores = 1;
    opt->w_drop_tol = 0.0;
}

const char* awg_status_string(awg_status s) {
    switch (s) {
        case AWG_OK: return "AWG_OK";
        case AWG_ERR_INVALID_ARG: return "AWG_ERR_INVALID_ARG";
        case AWG_ERR_MIN_OVERLAP: return "AWG_ERR_MIN_OVERLAP";
        case AWG_ERR_NOT_SPD: return "AWG_ERR_NOT_SPD";
        case AWG_ERR_EIG: return "AWG_ERR_EIG";
        case AWG_ERR_BREAKDOWN: return "AWG_ERR_BREAKDOWN";
        case AWG_ERR_MAXIT: return "AWG_ERR_MAXIT";
        case AWG_ERR_OOM: return "AWG_ERR_OOM";
        case AWG_ERR_CUDA: return "AWG_ERR_CUDA";
        case AWG_ERR_NOT_SYMMETRIC: return "AWG_ERR_NOT_SYMMETRIC";
        case AWG_ERR_STATE: return "AWG_ERR_STATE";
        case AWG_ERR_IO: return "AWG_ERR_IO";
    }
    return "AWG_ERR_UNKNOWN";
}

static awg_status setup_impl(Handle* h, const int* d_rowptr, const int* d_colidx,
                             const double* d_val, const int* d_part) {
    cudaStream_t s = h->stream;
    const double t0 = now_ms();
    {
        NvtxRange nv_("awg_setup: structure");  // the numeric stages have ranges of their own
        AWG_TRY(runtime_init(h));
        AWG_TRY(dalloc(h, h->rowptr, (size_t)(h->n + 1) * sizeof(int)));
        AWG_TRY(dalloc(h, h->colidx, (size_t)h->nnz * sizeof(int)));
        AWG_TRY(dalloc(h, h->val, (size_t)h->nnz * sizeof(double)));
        AWG_CUDA(cudaMemcpyAsync(h->rowptr.p, d_rowptr, (size_t)(h->n + 1) * sizeof(int), cudaMemcpyDefault, s));
        AWG_CUDA(cudaMemcpyAsync(h->colidx.p, d_colidx, (size_t)h->nnz * sizeof(int), cudaMemcpyDefault, s));
        AWG_CUDA(cudaMemcpyAsync(h->val.p, d_val, (size_t)h->nnz * sizeof(double), cudaMemcpyDefault, s));
        AWG_CUDA(cudaStreamSynchronize(s));
        AWG_TRY(setup_structure(h, d_part));
        AWG_CUDA(cudaStreamSynchronize(s));
    }
    h->setup_ms[0] = now_ms() - t0;
    if (h->opt.verbose)
        fprintf(stderr, "libawg: structure %.1f ms (N=%d, sum n^s=%lld, max n^s=%d)\n", h->setup_ms[0],
                h->N, (long long)h->sum_ns, h->max_ns);
    if (h->max_ns * 8 > 200 * 1024) return AWG_ERR_INVALID_ARG;  // shared-memory staging limit
    AWG_TRY(build_setup_numeric(h));
    h->setup_ms[7] = now_ms() - t0;
    if (h->opt.verbose)
        fprintf(stderr,
                "libawg: split %.1f, local %.1f, geneo %.1f, E %.1f, W %.1f, F %.1f, total %.1f ms; "
                "n0=%d n_minus=%d (all %d), W its %d relres %.2e\n",
                h->setup_ms[1], h->setup_ms[2], h->setup_ms[3], h->setup_ms[4], h->setup_ms[5],
                h->setup_ms[6], h->setup_ms[7], h->n0, h->n_minus, h->n_minus_all, h->w_iters,
                h->w_relres);
    if (h->opt.verbose && h->opt.geneo_solver)
        fprintf(stderr, "libawg: GenEO block solver: steps max %d, sum %lld; dense fallback %d of %d\n",
                h->geneo_its_max, (long long)h->geneo_its_sum, h->geneo_dense, h->N);
    return AWG_OK;
}

awg_status awg_setup(int n, int nnz, const int* d_rowptr, const int* d_colidx, const double* d_val,
                     const int* d_partition, int nparts, int overlap, double tau,
                     const awg_options* opt, void* stream, awg_handle* out) {
    if (!out) return AWG_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || nnz < n || nparts < 1 || nparts > n || overlap < 0 || !(tau > 0.0) || !d_rowptr ||
        !d_colidx || !d_val || !d_partition)
        return AWG_ERR_INVALID_ARG;
    awg_options o;
    awg_default_options(&o);
    if (opt) o = *opt;
    if (o.variant < 0 || o.variant > 2 || !(o.zero_rtol >= 0.0) || !(o.w_rtol > 0.0) ||
        o.w_maxit < 1 || o.maxit < 1 || (o.w_precision != AWG_FP64 && o.w_precision != AWG_MIXED_FP32) ||
        o.geneo_solver < 0 || o.geneo_solver > 2 || o.geneo_block < 2 || o.geneo_block > 16 ||
        o.geneo_maxit < 1 || (o.geneo_solver == 2 && !o.learned_params) || !(o.w16_keep >= 0.0) ||
        o.w16_keep > 1.0 || o.h2 < AWG_H2_NN_HYB || o.h2 > AWG_H2_AS_HYB || !(o.tau_flat > 0.0) ||
        o.coarse_tensor_cores < 0 || o.coarse_tensor_cores > 1 || !(o.w_drop_tol >= 0.0) || o.w_drop_tol >= 1.0 ||
        (o.w_drop_tol > 0.0 && o.variant == AWG_H3_INEX))
        return AWG_ERR_INVALID_ARG;
    o.precisions |= 1 << AWG_FP64;
    Handle* h = new (std::nothrow) Handle();
    if (!h) return AWG_ERR_OOM;
    h->n = n;
    h->nnz = nnz;
    h->N = nparts;
    h->overlap = overlap;
    // GenEO threshold: tau_sharp (Thms. 4, 5) or 1 / tau_flat (Thm. 3)
    h->tau = (o.h2 == AWG_H2_ASP_HYB || o.h2 == AWG_H2_ASP_AD) ? 1.0 / o.tau_flat : tau;
    h->opt = o;
    if (o.geneo_solver == 2) h->h_learned.assign(o.learned_params, o.learned_params + AWG_LEARNED_NPARAM);
    h->opt.learned_params = nullptr;  // the caller's array is read during setup only
    h->stream = (cudaStream_t)stream;
    awg_status st = setup_impl(h, d_rowptr, d_colidx, d_val, d_partition);
    if (st != AWG_OK) {
        cudaStreamSynchronize(h->stream);
        free_all(h);
        delete h;
        return st;
    }
    *out = reinterpret_cast<awg_handle>(h);
    return AWG_OK;
}

void awg_destroy(awg_handle hh) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

awg_status awg_get_info(awg_handle hh, awg_info* info) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !info) return AWG_ERR_INVALID_ARG;
    info->n = h->n;
    info->nnz = h->nnz;
    info->nparts = h->N;
    info->sum_ns = h->sum_ns;
    info->max_ns = h->max_ns;
    info->n0 = h->n0;
    info->n_minus = h->n_minus;
    info->n_minus_all = h->n_minus_all;
    info->w_iters = h->w_iters;
    info->w_relres = h->w_relres;
    for (int i = 0; i < 8; i++) info->setup_ms[i] = h->setup_ms[i];
    info->device_bytes = h->device_bytes;
    info->geneo_its_max = h->geneo_its_max;
    info->geneo_its_sum = h->geneo_its_sum;
    info->geneo_dense = h->geneo_dense;
    for (int p = 0; p < 4; p++) {
        info->wt_blocks[p] = h->prec[p].built ? h->prec[p].wt_blocks : 0;
        info->wd_blocks[p] = h->prec[p].built ? h->prec[p].wd_blocks : 0;
    }
    for (int k = 0; k < 3; k++) {
        info->block_wt_ctas[k] = h->bt_wt[k];
        info->block_dense_bps[k] = h->bt_dense[k];
    }
    info->w_kept = h->prec[AWG_FP64].sp_nnz;
    return AWG_OK;
}

static int variant_stage(const Handle* h) { return 4 + h->opt.variant; }

awg_status awg_apply(awg_handle hh, int precision, const double* d_r, double* d_z, int nrhs, int ld,
                     void* stream) {
    NvtxRange nv_("awg_apply");
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !d_r || !d_z || nrhs < 0 || ld < h->n || precision < 0 || precision >= AWG_NPREC)
        return AWG_ERR_INVALID_ARG;
    if (!h->prec[precision].built) return AWG_ERR_STATE;
    cudaStream_t us = (cudaStream_t)stream;
    AWG_CUDA(cudaEventRecord(h->ev_in, us));
    AWG_CUDA(cudaStreamWaitEvent(h->hp, h->ev_in, 0));
    awg_status st = AWG_OK;
    for (int c = 0; c < nrhs && st == AWG_OK; c++)
        st = apply_stage(h, variant_stage(h), precision, d_r + (size_t)c * ld, d_z + (size_t)c * ld, h->hp);
    AWG_CUDA(cudaEventRecord(h->ev_out, h->hp));
    AWG_CUDA(cudaStreamWaitEvent(us, h->ev_out, 0));
    return st;
}

awg_status awg_apply_stage(awg_handle hh, int which, int precision, const double* d_x, double* d_y,
                           void* stream) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !d_x || !d_y || which < 0 || which > 6 || precision < 0 || precision >= AWG_NPREC)
        return AWG_ERR_INVALID_ARG;
    if (!h->prec[precision].built) return AWG_ERR_STATE;
    if (which == 6 && h->n_minus > 0 && !h->prec[precision].inexInv.p) return AWG_ERR_STATE;
    return apply_stage(h, which, precision, d_x, d_y, (cudaStream_t)stream);
}

awg_status awg_pcg(awg_handle hh, int precision, const double* d_b, double* d_x, int nrhs, int ld,
                   double rtol, int* h_iters, double* h_relres, void* stream) {
    NvtxRange nv_("awg_pcg");
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !d_b || !d_x || nrhs < 0 || ld < h->n || !(rtol > 0.0) || precision < 0 || precision >= AWG_NPREC)
        return AWG_ERR_INVALID_ARG;
    if (!h->prec[precision].built) return AWG_ERR_STATE;
    awg_status worst = AWG_OK;
    cudaStream_t us = (cudaStream_t)stream;
    AWG_CUDA(cudaEventRecord(h->ev_in, us));
    AWG_CUDA(cudaStreamWaitEvent(h->hp, h->ev_in, 0));
    for (int c = 0; c < nrhs; c++) {
        int it = 0;
        double rr = 0.0;
        awg_status st = pcg1(h, precision, variant_stage(h), d_b + (size_t)c * ld, d_x + (size_t)c * ld,
                             rtol, &it, &rr, h->hp);
        if (h_iters) h_iters[c] = it;
        if (h_relres) h_relres[c] = rr;
        if (st != AWG_OK && (worst == AWG_OK || st == AWG_ERR_CUDA)) worst = st;
        if (st == AWG_ERR_CUDA) break;
    }
    AWG_CUDA(cudaEventRecord(h->ev_out, h->hp));
    AWG_CUDA(cudaStreamWaitEvent(us, h->ev_out, 0));
    return worst;
}

awg_status awg_apply_block(awg_handle hh, int which, int precision, const double* d_x, double* d_y, int nrhs,
                           int ld, void* stream) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !d_x || !d_y || which < 0 || which > 6 || nrhs < 1 || nrhs > 64 || ld < h->n || precision < 0 ||
        precision >= AWG_NPREC)
        return AWG_ERR_INVALID_ARG;
    // the mixed block forms apply the float32 local pseudo-inverses
    if (!h->prec[precision].built || (precision != AWG_FP64 && !h->prec[AWG_MIXED_FP32].G.p)) return AWG_ERR_STATE;
    if (precision == AWG_FP64 && h->n_minus > 0 && !h->prec[AWG_FP64].W.p) return AWG_ERR_STATE;  // truncated W
    if (which == 6 && h->n_minus > 0 && !h->prec[precision].inexInv.p) return AWG_ERR_STATE;
    cudaStream_t us = (cudaStream_t)stream;
    AWG_CUDA(cudaEventRecord(h->ev_in, us));
    AWG_CUDA(cudaStreamWaitEvent(h->hp, h->ev_in, 0));
    const awg_status st = block_apply(h, which, precision, d_x, d_y, nrhs, ld, h->hp);
    AWG_CUDA(cudaEventRecord(h->ev_out, h->hp));
    AWG_CUDA(cudaStreamWaitEvent(us, h->ev_out, 0));
    return st;
}

awg_status awg_coarse_apply_block(awg_handle hh, int which, int precision, int engine, const double* d_x,
                                  double* d_y, int nrhs, void* stream) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !d_x || !d_y || which < 0 || which > 2 || engine < 0 || engine > 2 || nrhs < 1 || nrhs > 64 ||
        precision < 0 || precision >= AWG_NPREC)
        return AWG_ERR_INVALID_ARG;
    if (!h->prec[precision].built) return AWG_ERR_STATE;
    cudaStream_t us = (cudaStream_t)stream;
    AWG_CUDA(cudaEventRecord(h->ev_in, us));
    AWG_CUDA(cudaStreamWaitEvent(h->hp, h->ev_in, 0));
    const awg_status st = block_coarse_apply(h, which, precision, engine, d_x, d_y, nrhs, h->hp);
    AWG_CUDA(cudaEventRecord(h->ev_out, h->hp));
    AWG_CUDA(cudaStreamWaitEvent(us, h->ev_out, 0));
    AWG_CUDA(cudaStreamSynchronize(us));
    return st;
}

awg_status awg_pcg_block(awg_handle hh, int precision, const double* d_b, double* d_x, int nrhs, int ld,
                         double rtol, int* h_iters, double* h_relres, void* stream) {
    NvtxRange nv_("awg_pcg_block");
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !d_b || !d_x || nrhs < 0 || ld < h->n || !(rtol > 0.0) || precision < 0 || precision >= AWG_NPREC)
        return AWG_ERR_INVALID_ARG;
    // the mixed block forms apply the float32 local pseudo-inverses
    if (!h->prec[precision].built || (precision != AWG_FP64 && !h->prec[AWG_MIXED_FP32].G.p)) return AWG_ERR_STATE;
    if (precision == AWG_FP64 && h->n_minus > 0 && !h->prec[AWG_FP64].W.p) return AWG_ERR_STATE;  // truncated W
    if (nrhs == 0) return AWG_OK;
    cudaStream_t us = (cudaStream_t)stream;
    AWG_CUDA(cudaEventRecord(h->ev_in, us));
    AWG_CUDA(cudaStreamWaitEvent(h->hp, h->ev_in, 0));
    const awg_status st = block_pcg(h, precision, d_b, d_x, nrhs, ld, rtol, h_iters, h_relres, h->hp);
    AWG_CUDA(cudaEventRecord(h->ev_out, h->hp));
    AWG_CUDA(cudaStreamWaitEvent(us, h->ev_out, 0));
    AWG_CUDA(cudaStreamSynchronize(us));
    return st;
}

awg_status awg_pcg_block_async(awg_handle hh, int precision, const double* d_b, double* d_x, int nrhs, int ld,
                               double rtol, int* d_iters, double* d_relres, int* d_status, void* stream) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !d_b || !d_x || nrhs < 1 || nrhs > 128 || ld < h->n || !(rtol > 0.0) || precision < 0 ||
        precision >= AWG_NPREC)
        return AWG_ERR_INVALID_ARG;
    if (!h->prec[precision].built || (precision != AWG_FP64 && !h->prec[AWG_MIXED_FP32].G.p)) return AWG_ERR_STATE;
    if (nrhs > 1 && precision == AWG_FP64 && h->n_minus > 0 && !h->prec[AWG_FP64].W.p) return AWG_ERR_STATE;  // truncated W
    cudaStream_t us = (cudaStream_t)stream;
    AWG_CUDA(cudaEventRecord(h->ev_in, us));
    AWG_CUDA(cudaStreamWaitEvent(h->hp, h->ev_in, 0));
    // one right-hand side: the single-RHS apply (GEMV passes) in the loop graph
    const awg_status st =
        nrhs == 1 ? pcg1_async(h, precision, variant_stage(h), d_b, d_x, rtol, d_iters, d_relres, d_status, h->hp)
                  : block_pcg_async(h, precision, d_b, d_x, nrhs, ld, rtol, d_iters, d_relres, d_status, h->hp);
    AWG_CUDA(cudaEventRecord(h->ev_out, h->hp));
    AWG_CUDA(cudaStreamWaitEvent(us, h->ev_out, 0));
    return st;
}

awg_status awg_get_array(awg_handle hh, int what, void* h_out, size_t count) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !h_out) return AWG_ERR_INVALID_ARG;
    const void* src = nullptr;
    size_t len = 0, esz = 4;
    bool host = false;
    switch (what) {
        case 0: src = h->h_ns.data(); len = h->N; host = true; break;
        case 1: src = h->sub_idx.p; len = (size_t)h->sum_ns; break;
        case 2: src = h->h_nm.data(); len = h->N; host = true; break;
        case 3: src = h->h_nstrict.data(); len = h->N; host = true; break;
        case 4: src = h->h_modes.data(); len = h->N; host = true; break;
        case 5: src = h->lam_m.p; len = h->n_minus_all; esz = 8; break;
        case 6: src = h->mmu.p; len = h->nnz; esz = 8; break;
        case 7: src = h->dvec.p; len = h->n; esz = 8; break;
        case 8: src = h->E.p; len = (size_t)h->n0 * h->n0; esz = 8; break;
        case 9: src = h->F64.p; len = (size_t)h->n_minus * h->n_minus; esz = 8; break;
        case 10: src = h->Wcm.p; len = (size_t)h->n * h->n_minus; esz = 8; break;
        case 12: src = h->Z.p; len = (size_t)h->h_z_off[h->N]; esz = 8; break;
        case 11: {
            // dense Z, column-major n x n0, assembled on the host from the blocks
            if (count < (size_t)h->n * h->n0) return AWG_ERR_INVALID_ARG;
            std::vector<double> zb(std::max<int64_t>(1, h->h_z_off[h->N]));
            std::vector<int> idx(h->sum_ns);
            AWG_CUDA(cudaMemcpy(zb.data(), h->Z.p, zb.size() * 8, cudaMemcpyDeviceToHost));
            AWG_CUDA(cudaMemcpy(idx.data(), h->sub_idx.p, idx.size() * 4, cudaMemcpyDeviceToHost));
            double* out = (double*)h_out;
            std::fill(out, out + (size_t)h->n * h->n0, 0.0);
            for (int t = 0; t < h->N; t++) {
                const int m = h->h_ns[t];
                for (int j = 0; j < h->h_modes[t]; j++)
                    for (int p = 0; p < m; p++)
                        out[(size_t)(h->h_mode_ptr[t] + j) * h->n + idx[h->h_sub_ptr[t] + p]] =
                            zb[h->h_z_off[t] + (size_t)j * m + p];
            }
            return AWG_OK;
        }
        default: return AWG_ERR_INVALID_ARG;
    }
    if (count < len) return AWG_ERR_INVALID_ARG;
    if (len == 0) return AWG_OK;
    if (host) {
        memcpy(h_out, src, len * esz);
        return AWG_OK;
    }
    if (!src) return AWG_ERR_STATE;
    AWG_CUDA(cudaStreamSynchronize(h->stream));
    AWG_CUDA(cudaMemcpy(h_out, src, len * esz, cudaMemcpyDeviceToHost));
    return AWG_OK;
}

awg_status awg_profile(awg_handle hh, int enable) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return AWG_ERR_INVALID_ARG;
    if (enable) {
        AWG_CUDA(cudaStreamSynchronize(h->stream));
        if (h->ev_pool.empty()) {
            h->ev_pool.resize(65536);
            for (auto& e : h->ev_pool) AWG_CUDA(cudaEventCreate(&e));
        }
        h->ev_used = 0;
        h->ev_kernel.clear();
        h->launches = 0;
        AWG_CUDA(cudaStreamSynchronize(h->hp));
        block_graph_launches(h);  // drop the graph-loop kernels counted so far
        pcg1_graph_launches(h);
        for (int i = 0; i < AWG_NPROF; i++) { h->prof_ms[i] = 0.0; h->prof_cnt[i] = 0; }
    }
    h->prof = enable;
    return AWG_OK;
}

awg_status awg_profile_trace(awg_handle hh, int cap, int* h_class, double* h_t0, double* h_t1,
                             int* h_count) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || cap < 0 || !h_count || (cap > 0 && (!h_class || !h_t0 || !h_t1))) return AWG_ERR_INVALID_ARG;
    const int k = (int)std::min<size_t>((size_t)cap, h->ev_kernel.size());
    for (int i = 0; i < k; i++) {
        AWG_CUDA(cudaEventSynchronize(h->ev_pool[2 * i + 1]));
        float a = 0.f, b = 0.f;
        AWG_CUDA(cudaEventElapsedTime(&a, h->ev_pool[0], h->ev_pool[2 * i]));
        AWG_CUDA(cudaEventElapsedTime(&b, h->ev_pool[0], h->ev_pool[2 * i + 1]));
        h_class[i] = h->ev_kernel[i];
        h_t0[i] = a;
        h_t1[i] = b;
    }
    *h_count = k;
    return AWG_OK;
}

awg_status awg_profile_read(awg_handle hh, int64_t* h_launches, double* h_ms, int64_t* h_count) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return AWG_ERR_INVALID_ARG;
    // resolve the recorded event pairs
    for (size_t k = 0; k < h->ev_kernel.size(); k++) {
        AWG_CUDA(cudaEventSynchronize(h->ev_pool[2 * k + 1]));
        float ms = 0.f;
        AWG_CUDA(cudaEventElapsedTime(&ms, h->ev_pool[2 * k], h->ev_pool[2 * k + 1]));
        h->prof_ms[h->ev_kernel[k]] += ms;
        h->prof_cnt[h->ev_kernel[k]] += 1;
    }
    h->ev_kernel.clear();
    h->ev_used = 0;
    AWG_CUDA(cudaStreamSynchronize(h->hp));
    h->launches += block_graph_launches(h) + pcg1_graph_launches(h);  // kernels run inside graph loops
    if (h_launches) *h_launches = h->launches;
    for (int i = 0; i < AWG_NPROF; i++) {
        if (h_ms) h_ms[i] = h->prof_ms[i];
        if (h_count) h_count[i] = h->prof_cnt[i];
    }
    return AWG_OK;
}

}  // extern "C"
