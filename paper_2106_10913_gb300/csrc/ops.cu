// Block (multi-right-hand-side) operators of the AWG preconditioner, used by
// the setup (E = Z^T A_+ Z, the multi-RHS PCG that builds W) and by the
// multi-RHS apply.  Local work is batched GEMM over the per-subdomain slabs;
// every sum over subdomains is an owner-computes gather (deterministic).

#include "ops.cuh"

#include <algorithm>

namespace awg {

// Y = A X, one thread per (row, column)
__global__ void k_spmm(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                       const double* __restrict__ a, const double* __restrict__ X,
                       double* __restrict__ Y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const size_t c = blockIdx.y;
    const double* x = X + c * n;
    double acc = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; k++) acc = fma(a[k], x[ci[k]], acc);
    Y[c * n + i] = acc;
}

awg_status blk_spmm(Handle* h, const double* X, double* Y, int k, cudaStream_t s) {
    if (k == 0) return AWG_OK;
    dim3 g((h->n + 255) / 256, k);
    k_spmm<<<g, 256, 0, s>>>(h->n, (int*)h->rowptr.p, (int*)h->colidx.p, (double*)h->val.p, X, Y);
    AWG_LAUNCH();
    return AWG_OK;
}

// loc_s(p, c) = X(idx_s(p), c)
__global__ void k_gather(int n, int64_t sum_ns, int k, const int* __restrict__ sub_ptr,
                         const int* __restrict__ ns, const int* __restrict__ sub_idx,
                         const int* __restrict__ pos_sub, const double* __restrict__ X,
                         double* __restrict__ loc) {
    const int64_t P = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= sum_ns) return;
    const int c = blockIdx.y;
    const int s = pos_sub[P];
    const int64_t base = (int64_t)sub_ptr[s];
    loc[base * k + (P - base) + (int64_t)c * ns[s]] = X[(size_t)c * n + sub_idx[P]];
}

awg_status blk_gather(Handle* h, const double* X, double* loc, int k, cudaStream_t s) {
    if (k == 0) return AWG_OK;
    dim3 g((unsigned)((h->sum_ns + 255) / 256), k);
    k_gather<<<g, 256, 0, s>>>(h->n, h->sum_ns, k, (int*)h->sub_ptr.p, (int*)h->ns.p,
                               (int*)h->sub_idx.p, (int*)h->pos_sub.p, X, loc);
    AWG_LAUNCH();
    return AWG_OK;
}

// Y(i, c) = beta Y(i, c) + alpha sum over copies of i of loc
__global__ void k_prolong(int n, int k, const int* __restrict__ inc_ptr,
                          const int* __restrict__ inc_pos, const int* __restrict__ inc_sub,
                          const int* __restrict__ sub_ptr, const int* __restrict__ ns,
                          const double* __restrict__ loc, double* __restrict__ Y, double alpha,
                          double beta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = blockIdx.y;
    double acc = 0.0;
    for (int e = inc_ptr[i]; e < inc_ptr[i + 1]; e++) {
        const int s = inc_sub[e];
        const int64_t base = sub_ptr[s];
        acc += loc[base * k + (inc_pos[e] - base) + (int64_t)c * ns[s]];
    }
    double* y = Y + (size_t)c * n + i;
    *y = (beta == 0.0) ? alpha * acc : fma(beta, *y, alpha * acc);
}

awg_status blk_prolong(Handle* h, const double* loc, double* Y, int k, double alpha, double beta,
                       cudaStream_t s) {
    if (k == 0) return AWG_OK;
    dim3 g((h->n + 255) / 256, k);
    k_prolong<<<g, 256, 0, s>>>(h->n, k, (int*)h->inc_ptr.p, (int*)h->inc_pos.p, (int*)h->inc_sub.p,
                                (int*)h->sub_ptr.p, (int*)h->ns.p, loc, Y, alpha, beta);
    AWG_LAUNCH();
    return AWG_OK;
}

// T_s(r, c) *= w_r (row weights of each subdomain's block)
__global__ void k_scale_rows(int k, const int* __restrict__ cnt_ptr, const double* __restrict__ w,
                             double* T) {
    const int s = blockIdx.x;
    const int r0 = cnt_ptr[s], nr = cnt_ptr[s + 1] - r0;
    double* Ts = T + (int64_t)r0 * k;
    for (int e = threadIdx.x; e < nr * k; e += blockDim.x) Ts[e] *= w[r0 + (e % nr)];
}

__global__ void k_neg(int len, const double* __restrict__ x, double* y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) y[i] = -x[i];
}

awg_status blk_aminus(Handle* h, const double* X, double* Y, int k, bool add, cudaStream_t s) {
    const int N = h->N;
    if (h->n_minus_all == 0) {
        if (!add) AWG_CUDA(cudaMemsetAsync(Y, 0, (size_t)h->n * k * 8, s));
        return AWG_OK;
    }
    double *loc = nullptr, *T = nullptr, *w = nullptr;
    AWG_CUDA(cudaMallocAsync(&loc, (size_t)h->sum_ns * k * 8, s));
    AWG_CUDA(cudaMallocAsync(&T, (size_t)h->n_minus_all * k * 8, s));
    AWG_CUDA(cudaMallocAsync(&w, (size_t)h->n_minus_all * 8, s));
    k_neg<<<(h->n_minus_all + 255) / 256, 256, 0, s>>>(h->n_minus_all, (double*)h->lam_m.p, w);
    AWG_LAUNCH();
    AWG_TRY(blk_gather(h, X, loc, k, s));
    std::vector<GemmDesc> d1, d2;
    const double* V = (const double*)h->Vm.p;
    for (int t = 0; t < N; t++) {
        const int m = h->h_ns[t], nu = h->h_nm[t];
        if (nu == 0) continue;
        const double* Vt = V + h->h_vm_off[t];
        double* Tt = T + (int64_t)h->h_nm_ptr[t] * k;
        double* Lt = loc + (int64_t)h->h_sub_ptr[t] * k;
        d1.push_back({Vt, Lt, Tt, nu, k, m, m, m, nu, 1, 0, 1.0, 0.0});
        d2.push_back({Vt, Tt, Lt, m, k, nu, m, nu, m, 0, 0, 1.0, 0.0});
    }
    AWG_TRY(gemm_batched(h, d1, s));
    k_scale_rows<<<N, 256, 0, s>>>(k, (int*)h->nm_ptr.p, w, T);
    AWG_LAUNCH();
    // subdomains without V^s_- keep their gathered values: zero them first
    for (int t = 0; t < N; t++)
        if (h->h_nm[t] == 0)
            AWG_CUDA(cudaMemsetAsync(loc + (int64_t)h->h_sub_ptr[t] * k, 0,
                                     (size_t)h->h_ns[t] * k * 8, s));
    AWG_TRY(gemm_batched(h, d2, s));
    AWG_TRY(blk_prolong(h, loc, Y, k, 1.0, add ? 1.0 : 0.0, s));
    AWG_CUDA(cudaFreeAsync(loc, s));
    AWG_CUDA(cudaFreeAsync(T, s));
    AWG_CUDA(cudaFreeAsync(w, s));
    return AWG_OK;
}

awg_status blk_aplus(Handle* h, const double* X, double* Y, int k, cudaStream_t s) {
    AWG_TRY(blk_spmm(h, X, Y, k, s));
    return blk_aminus(h, X, Y, k, true, s);
}

awg_status blk_zt(Handle* h, const double* X, double* C, int k, cudaStream_t s) {
    if (h->n0 == 0 || k == 0) return AWG_OK;
    double* loc = nullptr;
    AWG_CUDA(cudaMallocAsync(&loc, (size_t)h->sum_ns * k * 8, s));
    AWG_TRY(blk_gather(h, X, loc, k, s));
    std::vector<GemmDesc> d;
    const double* Z = (const double*)h->Z.p;
    for (int t = 0; t < h->N; t++) {
        const int m = h->h_ns[t], mt = h->h_modes[t];
        if (mt == 0) continue;
        d.push_back({Z + h->h_z_off[t], loc + (int64_t)h->h_sub_ptr[t] * k, C + h->h_mode_ptr[t],
                     mt, k, m, m, m, h->n0, 1, 0, 1.0, 0.0});
    }
    AWG_TRY(gemm_batched(h, d, s));
    AWG_CUDA(cudaFreeAsync(loc, s));
    return AWG_OK;
}

awg_status blk_z(Handle* h, const double* C, double* Y, int k, double alpha, double beta,
                 cudaStream_t s) {
    if (k == 0) return AWG_OK;
    double* loc = nullptr;
    AWG_CUDA(cudaMallocAsync(&loc, (size_t)h->sum_ns * k * 8, s));
    AWG_CUDA(cudaMemsetAsync(loc, 0, (size_t)h->sum_ns * k * 8, s));
    std::vector<GemmDesc> d;
    const double* Z = (const double*)h->Z.p;
    for (int t = 0; t < h->N; t++) {
        const int m = h->h_ns[t], mt = h->h_modes[t];
        if (mt == 0) continue;
        d.push_back({Z + h->h_z_off[t], C + h->h_mode_ptr[t], loc + (int64_t)h->h_sub_ptr[t] * k,
                     m, k, mt, m, h->n0, m, 0, 0, 1.0, 0.0});
    }
    AWG_TRY(gemm_batched(h, d, s));
    AWG_TRY(blk_prolong(h, loc, Y, k, alpha, beta, s));
    AWG_CUDA(cudaFreeAsync(loc, s));
    return AWG_OK;
}

awg_status blk_hnn(Handle* h, const double* X, double* Y, int k, cudaStream_t s, int prec) {
    double *loc = nullptr, *out = nullptr;
    AWG_CUDA(cudaMallocAsync(&loc, (size_t)h->sum_ns * k * 8, s));
    AWG_CUDA(cudaMallocAsync(&out, (size_t)h->sum_ns * k * 8, s));
    AWG_TRY(blk_gather(h, X, loc, k, s));
    if (prec == AWG_MIXED_FP32) {
        std::vector<GemmDescF> d;
        const float* G = (const float*)h->prec[AWG_MIXED_FP32].G.p;
        if (!G) return AWG_ERR_STATE;
        for (int t = 0; t < h->N; t++) {
            const int m = h->h_ns[t], ld = (m + 3) & ~3;  // padded float32 layout
            d.push_back({G + h->h_g32_off[t], loc + (int64_t)h->h_sub_ptr[t] * k,
                         out + (int64_t)h->h_sub_ptr[t] * k, m, k, m, ld, m, m, 0, 1.0, 0.0});
        }
        AWG_TRY(gemm_batched_f32(h, d, s));
    } else {
        std::vector<GemmDesc> d;
        const double* G = (const double*)h->prec[AWG_FP64].G.p;
        for (int t = 0; t < h->N; t++) {
            const int m = h->h_ns[t];
            d.push_back({G + h->h_dense_off[t], loc + (int64_t)h->h_sub_ptr[t] * k,
                         out + (int64_t)h->h_sub_ptr[t] * k, m, k, m, m, m, m, 0, 0, 1.0, 0.0});
        }
        AWG_TRY(gemm_batched(h, d, s));
    }
    AWG_TRY(blk_prolong(h, out, Y, k, 1.0, 0.0, s));
    AWG_CUDA(cudaFreeAsync(loc, s));
    AWG_CUDA(cudaFreeAsync(out, s));
    return AWG_OK;
}

__global__ void k_axpby(size_t len, double a, const double* __restrict__ x, double b,
                        double* __restrict__ y) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < len) y[i] = fma(a, x[i], b * y[i]);
}

static awg_status axpby(size_t len, double a, const double* x, double b, double* y, cudaStream_t s) {
    if (len == 0) return AWG_OK;
    k_axpby<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(len, a, x, b, y);
    AWG_LAUNCH();
    return AWG_OK;
}

awg_status blk_h2(Handle* h, const double* X, double* Y, int k, cudaStream_t s, int prec) {
    const size_t nk = (size_t)h->n * k;
    const int n0 = h->n0;
    if (n0 == 0) return blk_hnn(h, X, Y, k, s, prec);
    double *C0, *C1, *X1, *T, *U;
    AWG_CUDA(cudaMallocAsync(&C0, (size_t)n0 * k * 8, s));
    AWG_CUDA(cudaMallocAsync(&C1, (size_t)n0 * k * 8, s));
    AWG_CUDA(cudaMallocAsync(&X1, nk * 8, s));
    AWG_CUDA(cudaMallocAsync(&T, nk * 8, s));
    AWG_CUDA(cudaMallocAsync(&U, nk * 8, s));
    const double* Einv = (const double*)h->Einv.p;
    // C1 = E^-1 Z^T X
    AWG_TRY(blk_zt(h, X, C0, k, s));
    AWG_TRY(gemm_batched(h, {{Einv, C0, C1, n0, k, n0, n0, n0, n0, 0, 0, 1.0, 0.0}}, s));
    if (h->opt.h2 == AWG_H2_ASP_AD) {  // H^AS_+,ad (Thm. 3): Y = H_1 X + Z C1
        AWG_TRY(blk_hnn(h, X, Y, k, s, prec));
        AWG_TRY(blk_z(h, C1, Y, k, 1.0, 1.0, s));
        for (double* p : {C0, C1, X1, T, U}) AWG_CUDA(cudaFreeAsync(p, s));
        return AWG_OK;
    }
    // T = X - A_+ Z C1   (Pi^T X)
    AWG_TRY(blk_z(h, C1, X1, k, 1.0, 0.0, s));
    AWG_TRY(blk_aplus(h, X1, T, k, s));
    AWG_TRY(axpby(nk, 1.0, X, -1.0, T, s));
    // U = H^NN T
    AWG_TRY(blk_hnn(h, T, U, k, s, prec));
    // C0 = E^-1 Z^T A_+ U ; Y = U - Z C0 + Z C1
    AWG_TRY(blk_aplus(h, U, T, k, s));
    AWG_TRY(blk_zt(h, T, X1, k, s));  // X1 reused as n0 x k scratch
    AWG_TRY(gemm_batched(h, {{Einv, X1, C0, n0, k, n0, n0, n0, n0, 0, 0, 1.0, 0.0}}, s));
    AWG_TRY(axpby((size_t)n0 * k, -1.0, C0, 1.0, C1, s));  // C1 = C1 - C0
    AWG_CUDA(cudaMemcpyAsync(Y, U, nk * 8, cudaMemcpyDeviceToDevice, s));
    AWG_TRY(blk_z(h, C1, Y, k, 1.0, 1.0, s));
    for (double* p : {C0, C1, X1, T, U}) AWG_CUDA(cudaFreeAsync(p, s));
    return AWG_OK;
}

// out[c] = sum_i X(i, c) Y(i, c), one block per column (fixed order)
__global__ void k_coldot(int n, const double* __restrict__ X, const double* __restrict__ Y,
                         double* out) {
    __shared__ double red[32];
    const size_t c = blockIdx.x;
    const double* x = X + c * n;
    const double* y = Y + c * n;
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc = fma(x[i], y[i], acc);
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) out[c] = acc;
}

awg_status col_dot(Handle* h, const double* X, const double* Y, double* out, int k, cudaStream_t s) {
    if (k == 0) return AWG_OK;
    k_coldot<<<k, 512, 0, s>>>(h->n, X, Y, out);
    AWG_LAUNCH();
    return AWG_OK;
}

}  // namespace awg
