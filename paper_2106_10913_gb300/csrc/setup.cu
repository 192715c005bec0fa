// Numeric setup of the AWG preconditioner on the device (Sections 3-4):
//   1. eigen-split of every B^s (Def. 6): selected eigenpairs lambda <= 0;
//   2. local factors: K^s = B^s + V^s_-(sigma I - L^s_-)V^s_-^T = A^s_+ + sigma
//      V^s_- V^s_-^T is SPD; (A^s_+)^+ = P K^s^-1 P with P = I - V^s_- V^s_-^T
//      (Section 4.4 item 3) from the Cholesky factor of K^s, stored as the
//      explicit symmetric D^s (A^s_+)^+ D^s;
//   3. GenEO pencil (M_A, M_B) = (D^s^-1 A^s_+ D^s^-1, R^s A_+ R^sT) with M_B
//      from Section 4.4 item 4; reduced by the Cholesky factor of M_B to a
//      standard symmetric problem; eigenvectors with lambda < tau (Def. 9)
//      (H^AS_hyb: two pencils, Thm. 5); with an AS choice of H_2, the local
//      solvers (R^s A_+ R^sT)^-1 or (R^s A R^sT)^-1 (Thms. 3, 5);
//   4. E = Z^T A_+ Z (Thm. 4), Cholesky, explicit inverse;
//   5. W = A_+^-1 [R^sT V^s_-] (strictly negative eigenvalues, Section 4.4
//      items 1-2) by PCG preconditioned with H_2 on all columns at once;
//   6. F = W^T A W (Def. 10), Cholesky, explicit inverse; the reduced-
//      precision copies of W and of the local operators, each with its own F.

#include "awg_common.cuh"
#include "ops.cuh"
#include "block.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>

namespace awg {

size_t ws_bytes(const Handle* h);
awg_status set_smem_limits(Handle* h);

// K = B + V diag(sigma - lambda) V^T with sigma = mean of diag(B)
__global__ void k_form_K(const int* __restrict__ ns, const int64_t* __restrict__ off,
                         const int* __restrict__ nm_ptr, const int64_t* __restrict__ vm_off,
                         const double* __restrict__ V, const double* __restrict__ lam, double* arena,
                         double* sigma) {
    __shared__ double red[32];
    __shared__ double wsh[256];
    const int s = blockIdx.x;
    const int m = ns[s];
    double* K = arena + off[s];
    double tr = 0.0;
    for (int p = threadIdx.x; p < m; p += blockDim.x) tr += K[p + (size_t)p * m];
    tr = block_sum(tr, red);
    const double sg = tr / m;
    if (threadIdx.x == 0) sigma[s] = sg;
    const int l0 = nm_ptr[s], nu = nm_ptr[s + 1] - l0;
    const double* Vs = V + vm_off[s];
    for (int k0 = 0; k0 < nu; k0 += 256) {
        const int kk = min(256, nu - k0);
        __syncthreads();
        for (int k = threadIdx.x; k < kk; k += blockDim.x) wsh[k] = sg - lam[l0 + k0 + k];
        __syncthreads();
        for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
            const int p = (int)(e % m), q = (int)(e / m);
            double acc = 0.0;
            for (int k = 0; k < kk; k++)
                acc = fma(Vs[p + (size_t)(k0 + k) * m] * wsh[k], Vs[q + (size_t)(k0 + k) * m], acc);
            K[e] += acc;
        }
    }
}

// G = D (Kinv - V T^T - T V^T + U V^T) D, T = Kinv V, U = V (V^T T)
__global__ void k_form_G(const int* __restrict__ ns, const int64_t* __restrict__ off,
                         const int* __restrict__ sub_ptr, const int* __restrict__ sub_idx,
                         const double* __restrict__ dvec, const int* __restrict__ nm_ptr,
                         const int64_t* __restrict__ vm_off, const double* __restrict__ V,
                         const double* __restrict__ T, const double* __restrict__ U, double* arena) {
    const int s = blockIdx.x;
    const int m = ns[s];
    double* G = arena + off[s];
    const int nu = nm_ptr[s + 1] - nm_ptr[s];
    const double* Vs = V + vm_off[s];
    const double* Ts = T + vm_off[s];
    const double* Us = U + vm_off[s];
    const int* idx = sub_idx + sub_ptr[s];
    for (int64_t e = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * m;
         e += (int64_t)gridDim.y * blockDim.x) {
        const int p = (int)(e % m), q = (int)(e / m);
        double acc = G[e];
        for (int k = 0; k < nu; k++) {
            const double vp = Vs[p + (size_t)k * m], vq = Vs[q + (size_t)k * m];
            acc -= vp * Ts[q + (size_t)k * m] + Ts[p + (size_t)k * m] * vq;
            acc = fma(Us[p + (size_t)k * m], vq, acc);
        }
        G[e] = acc * dvec[idx[p]] * dvec[idx[q]];
    }
}

// M_A = D^-1 (B + V |L| V^T) D^-1 in place over B
__global__ void k_form_MA(const int* __restrict__ ns, const int64_t* __restrict__ off,
                          const int* __restrict__ sub_ptr, const int* __restrict__ sub_idx,
                          const double* __restrict__ dvec, const int* __restrict__ nm_ptr,
                          const int64_t* __restrict__ vm_off, const double* __restrict__ V,
                          const double* __restrict__ lam, double* arena) {
    const int s = blockIdx.x;
    const int m = ns[s];
    double* M = arena + off[s];
    const int l0 = nm_ptr[s], nu = nm_ptr[s + 1] - l0;
    const double* Vs = V + vm_off[s];
    const int* idx = sub_idx + sub_ptr[s];
    for (int64_t e = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * m;
         e += (int64_t)gridDim.y * blockDim.x) {
        const int p = (int)(e % m), q = (int)(e / m);
        double acc = M[e];
        for (int k = 0; k < nu; k++)
            acc = fma(Vs[p + (size_t)k * m] * (-lam[l0 + k]), Vs[q + (size_t)k * m], acc);
        M[e] = acc / (dvec[idx[p]] * dvec[idx[q]]);
    }
}

// M_B += sum_t R^s R^tT V^t_- |L^t_-| V^t_-^T R^t R^sT  (Section 4.4 item 4)
__global__ void k_add_nbr_MB(const int* __restrict__ ns, const int64_t* __restrict__ off,
                             const int* __restrict__ sub_ptr, const int* __restrict__ sub_idx,
                             const int* __restrict__ inc_ptr, const int* __restrict__ inc_pos,
                             const int* __restrict__ inc_sub, const int* __restrict__ nm_ptr,
                             const int64_t* __restrict__ vm_off, const double* __restrict__ V,
                             const double* __restrict__ lam, double* arena) {
    const int s = blockIdx.x;
    const int m = ns[s];
    double* M = arena + off[s];
    const int* idx = sub_idx + sub_ptr[s];
    for (int64_t e = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * m;
         e += (int64_t)gridDim.y * blockDim.x) {
        const int p = (int)(e % m), q = (int)(e / m);
        const int ip = idx[p], iq = idx[q];
        double acc = 0.0;
        for (int e1 = inc_ptr[ip]; e1 < inc_ptr[ip + 1]; e1++) {
            const int t = inc_sub[e1];
            const int nu = nm_ptr[t + 1] - nm_ptr[t];
            if (nu == 0) continue;
            for (int e2 = inc_ptr[iq]; e2 < inc_ptr[iq + 1]; e2++) {
                if (inc_sub[e2] != t) continue;
                const int mt = ns[t];
                const int pt = inc_pos[e1] - sub_ptr[t], qt = inc_pos[e2] - sub_ptr[t];
                const double* Vt = V + vm_off[t];
                const double* lt = lam + nm_ptr[t];
                for (int k = 0; k < nu; k++)
                    acc = fma(Vt[pt + (size_t)k * mt] * (-lt[k]), Vt[qt + (size_t)k * mt], acc);
            }
        }
        M[e] += acc;
    }
}

__global__ void k_symmetrize(const int* __restrict__ ns, const int64_t* __restrict__ off,
                             double* arena) {
    const int s = blockIdx.x;
    const int m = ns[s];
    double* C = arena + off[s];
    for (int64_t e = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * m;
         e += (int64_t)gridDim.y * blockDim.x) {
        const int p = (int)(e % m), q = (int)(e / m);
        if (p > q) {
            const double v = 0.5 * (C[e] + C[q + (size_t)p * m]);
            C[e] = v;
            C[q + (size_t)p * m] = v;
        }
    }
}

// Y (n x k, column-major) gets, for every global column g = colptr[s] + j in
// [c0, c0 + k), column g - c0 = R^sT B_s(:, j); other rows untouched.
__global__ void k_scatter_cols(int n, const int* __restrict__ sub_ptr,
                               const int* __restrict__ sub_idx, const int* __restrict__ colptr,
                               const int64_t* __restrict__ boff, const double* __restrict__ B,
                               double* Y, int c0, int k) {
    const int s = blockIdx.x;
    const int p0 = sub_ptr[s], m = sub_ptr[s + 1] - p0;
    const int g0 = colptr[s], nc = colptr[s + 1] - g0;
    const int ja = max(0, c0 - g0), jb = min(nc, c0 + k - g0);
    if (ja >= jb) return;
    const double* Bs = B + boff[s];
    for (int64_t e = (int64_t)ja * m + threadIdx.x; e < (int64_t)jb * m; e += blockDim.x) {
        const int p = (int)(e % m), j = (int)(e / m);
        Y[(size_t)(g0 + j - c0) * n + sub_idx[p0 + p]] = Bs[e];
    }
}

// row-major copy of a column-major n x k block into ld columns, in TS
template <typename TS>
__global__ void k_to_rowmajor(int n, int k, int ld, const double* __restrict__ X, TS* Y) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * ld) return;
    const int i = (int)(e / ld), c = (int)(e % ld);
    const double v = (c < k) ? X[(size_t)c * n + i] : 0.0;
    Y[e] = (TS)v;
}
template <>
__global__ void k_to_rowmajor<__nv_bfloat16>(int n, int k, int ld, const double* __restrict__ X,
                                             __nv_bfloat16* Y) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * ld) return;
    const int i = (int)(e / ld), c = (int)(e % ld);
    Y[e] = __double2bfloat16((c < k) ? X[(size_t)c * n + i] : 0.0);
}

// FP64 copy of a rounded column-major block (rounding through TS)
__global__ void k_round_f32(size_t len, const double* __restrict__ X, double* Y) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < len) Y[e] = (double)(float)X[e];
}
__global__ void k_round_bf16(size_t len, const double* __restrict__ X, double* Y) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < len) Y[e] = (double)__bfloat162float(__double2bfloat16(X[e]));
}
// ---- float16 W with power-of-two row and column scales: W = S_r What S_c
// 2^e with |x| < 2^e <= 2|x| (1 for x = 0), within the normal float32 range;
// built from the exponent bits, so the scaling itself is exact
__device__ __forceinline__ float pow2_above(double x) {
    if (!(x > 0.0)) return 1.f;
    int e;
    (void)frexp(x, &e);  // x = f 2^e, f in [1/2, 1)
    e = max(-126, min(127, e));
    return __int_as_float((e + 127) << 23);
}
__global__ void k_w16_cscale(int n, const double* __restrict__ W, float* cs, double* cmax) {
    __shared__ double red[32];
    const int j = blockIdx.x;
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(W[(size_t)j * n + i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t = fmax(t, red[w]);
        cs[j] = pow2_above(t);
        cmax[j] = t;
    }
}
// entries kept exact: |W_ij| >= keep * max_i |W_ij| (and nonzero)
__device__ __forceinline__ bool w16_kept(double v, double cmax, double keep) {
    return keep > 0.0 && v != 0.0 && fabs(v) >= keep * cmax;
}
__global__ void k_w16_corr_count(int n, int nm, const double* __restrict__ W, const double* __restrict__ cmax,
                                 double keep, int* cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0;
    for (int j = 0; j < nm; j++) c += w16_kept(W[(size_t)j * n + i], cmax[j], keep);
    cnt[i] = c;
}
// CSR of the correction (scaled units): What_ij exact minus its float16 rounding
__global__ void k_w16_corr_fill(int n, int nm, const double* __restrict__ W, const double* __restrict__ cmax,
                                double keep, const float* __restrict__ rs, const float* __restrict__ cs,
                                const int* __restrict__ rowptr, int* col, float* val) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = rowptr[i];
    for (int j = 0; j < nm; j++) {
        const double v = W[(size_t)j * n + i];
        if (!w16_kept(v, cmax[j], keep)) continue;
        const double sv = v / ((double)rs[i] * (double)cs[j]);
        col[k] = j;
        val[k] = (float)(sv - (double)__half2float(__double2half(sv)));
        k++;
    }
}
__global__ void k_w16_rscale(int n, int nm, const double* __restrict__ W, const float* __restrict__ cs,
                             float* rs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double m = 0.0;
    for (int j = 0; j < nm; j++) m = fmax(m, fabs(W[(size_t)j * n + i]) / (double)cs[j]);
    rs[i] = pow2_above(m);
}
// float64 copy of the rounded W (column-major), for F
// float64 copy of the stored W (float16 value plus the float32 correction
// where kept), column-major, for F
__global__ void k_round_fp16(int n, size_t len, const double* __restrict__ X, const float* __restrict__ rs,
                             const float* __restrict__ cs, const double* __restrict__ cmax, double keep,
                             double* Y) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= len) return;
    const double sc = (double)rs[e % n] * (double)cs[e / n];
    const double sv = X[e] / sc;
    const double h = (double)__half2float(__double2half(sv));
    Y[e] = w16_kept(X[e], cmax[e / n], keep) ? sc * (h + (double)(float)(sv - h)) : sc * h;
}
__global__ void k_to_rowmajor_fp16(int n, int k, int ld, const double* __restrict__ X,
                                   const float* __restrict__ rs, const float* __restrict__ cs, __half* Y) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * ld) return;
    const int i = (int)(e / ld), c = (int)(e % ld);
    Y[e] = __double2half((c < k) ? X[(size_t)c * n + i] / ((double)rs[i] * (double)cs[c]) : 0.0);
}

__global__ void k_conv_f32(size_t len, const double* __restrict__ X, float* Y) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < len) Y[e] = (float)X[e];
}

// float32 copy of the per-subdomain blocks with the leading dimension
// rounded up to 4 (padding rows zero)
__global__ void k_conv_f32_padded(const int* __restrict__ ns, const int64_t* __restrict__ off,
                                  const int64_t* __restrict__ off32, const double* __restrict__ X,
                                  float* Y) {
    const int s = blockIdx.x;
    const int m = ns[s], ld = (m + 3) & ~3;
    const double* Xs = X + off[s];
    float* Ys = Y + off32[s];
    for (int64_t e = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)ld * m;
         e += (int64_t)gridDim.y * blockDim.x) {
        const int q = (int)(e % ld), p = (int)(e / ld);
        Ys[e] = (q < m) ? (float)Xs[q + (size_t)p * m] : 0.f;
    }
}

// per-column PCG updates
__global__ void k_col_axpy(int n, const double* __restrict__ alpha, const double* __restrict__ X,
                           double* Y) {
    const size_t c = blockIdx.y;
    const double a = alpha[c];
    if (a == 0.0) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        Y[c * n + i] = fma(a, X[c * n + i], Y[c * n + i]);
}
__global__ void k_col_xpby(int n, const double* __restrict__ beta, const double* __restrict__ Zb,
                           double* P) {
    const size_t c = blockIdx.y;
    const double b = beta[c];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        P[c * n + i] = fma(b, P[c * n + i], Zb[c * n + i]);
}

__global__ void k_diag_minus(int dim, const double* __restrict__ dgl, double* M) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < dim) M[i + (size_t)i * dim] = dgl[i] - M[i + (size_t)i * dim];
}
__global__ void k_neg_offdiag(int dim, double* M) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)dim * dim) return;
    const int i = (int)(e % dim), j = (int)(e / dim);
    if (i != j) M[e] = -M[e];
}

static double now_ms() {
    return std::chrono::duration<double, std::milli>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

static awg_status check_flag(Handle* h, int mask, awg_status err) {
    int f = 0;
    AWG_TRY(read_flag(h, &f));
    return (f & mask) ? err : AWG_OK;
}

// Cholesky + explicit inverse of one dense SPD matrix M (dim x dim) into Minv.
static awg_status atb_sym(Handle* h, int n, int m, const double* A, const double* B, double* C, cudaStream_t s);

// Minv = M^-1 for an SPD coarse matrix (E or F): blocked Cholesky M = L L^T
// over the whole GPU, L^-1 by block rows, then M^-1 = L^-T L^-1 by the
// symmetric A^T B kernel (float64 throughout).
static awg_status spd_inverse(Handle* h, DevBuf& M, DevBuf& Minv, int dim) {
    cudaStream_t s = h->stream;
    if (dim == 0) return AWG_OK;
    DevBuf L, Li;
    AWG_TRY(dalloc(h, L, (size_t)dim * dim * 8));
    AWG_TRY(dalloc(h, Li, (size_t)dim * dim * 8));
    AWG_CUDA(cudaMemcpyAsync(L.p, M.p, (size_t)dim * dim * 8, cudaMemcpyDeviceToDevice, s));
    AWG_CUDA(cudaMemsetAsync(h->flag.p, 0, sizeof(int), s));
    AWG_TRY(chol_blocked(h, (double*)L.p, dim, (int*)h->flag.p, s));
    AWG_TRY(check_flag(h, FLAG_NOT_SPD, AWG_ERR_NOT_SPD));
    AWG_TRY(trtri_blocked(h, (double*)L.p, (double*)Li.p, dim, s));
    if (!Minv.p) AWG_TRY(dalloc(h, Minv, (size_t)dim * dim * 8));
    AWG_TRY(atb_sym(h, dim, dim, (double*)Li.p, (double*)Li.p, (double*)Minv.p, s));
    AWG_CUDA(cudaStreamSynchronize(s));
    dfree(h, L);
    dfree(h, Li);
    return AWG_OK;
}

// ------------------------------------------------------------ W by PCG
static awg_status build_W(Handle* h) {
    cudaStream_t s = h->stream;
    const int n = h->n, N = h->N, nm = h->n_minus;
    // right-hand sides Vhat = [R^sT V^s_-(strict)]
    AWG_TRY(dalloc(h, h->Wcm, (size_t)n * nm * 8));
    double* Vhat = nullptr;
    AWG_CUDA(cudaMallocAsync(&Vhat, (size_t)n * nm * 8, s));
    AWG_CUDA(cudaMemsetAsync(Vhat, 0, (size_t)n * nm * 8, s));
    k_scatter_cols<<<N, 256, 0, s>>>(n, (int*)h->sub_ptr.p, (int*)h->sub_idx.p, (int*)h->wcol_ptr.p,
                                     (int64_t*)h->vm_off.p, (double*)h->Vm.p, Vhat, 0, nm);
    AWG_LAUNCH();
    // the block path: groups of 64 columns through the block kernels (local
    // solves on the tensor cores for the float32 preconditioner)
    if (h->opt.block_tensor_cores) {
        int its = 0;
        double worst = 0.0;
        AWG_TRY(block_solve_w(h, h->opt.w_precision, Vhat, (double*)h->Wcm.p, nm, h->opt.w_rtol, h->opt.w_maxit,
                              &its, &worst, s));
        h->w_iters = its;
        h->w_relres = worst;
        AWG_CUDA(cudaFreeAsync(Vhat, s));
        AWG_CUDA(cudaStreamSynchronize(s));
        return AWG_OK;
    }
    // columns per chunk: about 10 n-vectors per column live at once
    const size_t budget = (size_t)24 << 30;
    int chunk = (int)std::max<size_t>(1, std::min<size_t>(nm, budget / ((size_t)n * 8 * 13)));
    const int wp = h->opt.w_precision;
    double *R, *Zb, *Zo, *P, *Q, *dots;
    AWG_CUDA(cudaMallocAsync(&Zo, (size_t)n * chunk * 8, s));
    AWG_CUDA(cudaMallocAsync(&R, (size_t)n * chunk * 8, s));
    AWG_CUDA(cudaMallocAsync(&Zb, (size_t)n * chunk * 8, s));
    AWG_CUDA(cudaMallocAsync(&P, (size_t)n * chunk * 8, s));
    AWG_CUDA(cudaMallocAsync(&Q, (size_t)n * chunk * 8, s));
    AWG_CUDA(cudaMallocAsync(&dots, (size_t)chunk * 5 * 8, s));
    std::vector<double> hb(chunk), hrz(chunk), hpq(chunk), hrr(chunk), hrzn(chunk), ha(chunk), hbeta(chunk);
    int max_it = 0;
    double worst = 0.0;
    for (int c0 = 0; c0 < nm; c0 += chunk) {
        const int k = std::min(chunk, nm - c0);
        const size_t nk = (size_t)n * k;
        double* X = (double*)h->Wcm.p + (size_t)c0 * n;
        const double* Bc = Vhat + (size_t)c0 * n;
        AWG_CUDA(cudaMemsetAsync(X, 0, nk * 8, s));
        AWG_CUDA(cudaMemcpyAsync(R, Bc, nk * 8, cudaMemcpyDeviceToDevice, s));
        AWG_TRY(col_dot(h, Bc, Bc, dots, k, s));
        AWG_TRY(blk_h2(h, R, Zb, k, s, wp));
        AWG_TRY(col_dot(h, R, Zb, dots + chunk, k, s));
        AWG_CUDA(cudaMemcpyAsync(P, Zb, nk * 8, cudaMemcpyDeviceToDevice, s));
        AWG_CUDA(cudaMemcpyAsync(hb.data(), dots, k * 8, cudaMemcpyDeviceToHost, s));
        AWG_CUDA(cudaMemcpyAsync(hrz.data(), dots + chunk, k * 8, cudaMemcpyDeviceToHost, s));
        AWG_CUDA(cudaStreamSynchronize(s));
        std::vector<char> active(k, 1);
        int it = 0;
        dim3 gcol((unsigned)std::min((n + 255) / 256, 64), (unsigned)k);
        for (;;) {
            AWG_TRY(blk_aplus(h, P, Q, k, s));
            AWG_TRY(col_dot(h, P, Q, dots, k, s));
            AWG_CUDA(cudaMemcpyAsync(hpq.data(), dots, k * 8, cudaMemcpyDeviceToHost, s));
            AWG_CUDA(cudaStreamSynchronize(s));
            for (int c = 0; c < k; c++) {
                ha[c] = (active[c] && hpq[c] > 0.0) ? hrz[c] / hpq[c] : 0.0;
                if (active[c] && !(hpq[c] > 0.0)) active[c] = 0;  // exact solution reached
            }
            AWG_CUDA(cudaMemcpyAsync(dots + 2 * chunk, ha.data(), k * 8, cudaMemcpyHostToDevice, s));
            k_col_axpy<<<gcol, 256, 0, s>>>(n, dots + 2 * chunk, P, X);
            AWG_LAUNCH();
            for (int c = 0; c < k; c++) ha[c] = -ha[c];
            AWG_CUDA(cudaMemcpyAsync(dots + 3 * chunk, ha.data(), k * 8, cudaMemcpyHostToDevice, s));
            k_col_axpy<<<gcol, 256, 0, s>>>(n, dots + 3 * chunk, Q, R);
            AWG_LAUNCH();
            AWG_TRY(col_dot(h, R, R, dots, k, s));
            AWG_CUDA(cudaMemcpyAsync(hrr.data(), dots, k * 8, cudaMemcpyDeviceToHost, s));
            AWG_CUDA(cudaStreamSynchronize(s));
            it++;
            int nact = 0;
            double wst = 0.0;
            for (int c = 0; c < k; c++) {
                const double rel = sqrt(hrr[c] / hb[c]);
                if (rel <= h->opt.w_rtol) active[c] = 0;
                if (active[c]) nact++;
                wst = std::max(wst, rel);
            }
            if (nact == 0 || it >= h->opt.w_maxit) { worst = std::max(worst, wst); break; }
            // flexible (Polak-Ribiere) beta = r^T (z - z_old) / r_old^T z_old: the
            // preconditioner may apply its local operators in float32
            std::swap(Zb, Zo);
            AWG_TRY(blk_h2(h, R, Zb, k, s, wp));
            AWG_TRY(col_dot(h, R, Zb, dots, k, s));
            AWG_TRY(col_dot(h, R, Zo, dots + chunk, k, s));
            AWG_CUDA(cudaMemcpyAsync(hrzn.data(), dots, k * 8, cudaMemcpyDeviceToHost, s));
            AWG_CUDA(cudaMemcpyAsync(hpq.data(), dots + chunk, k * 8, cudaMemcpyDeviceToHost, s));
            AWG_CUDA(cudaStreamSynchronize(s));
            for (int c = 0; c < k; c++) {
                hbeta[c] = (hrz[c] != 0.0) ? (hrzn[c] - hpq[c]) / hrz[c] : 0.0;
                hrz[c] = hrzn[c];
            }
            AWG_CUDA(cudaMemcpyAsync(dots + 4 * chunk, hbeta.data(), k * 8, cudaMemcpyHostToDevice, s));
            k_col_xpby<<<gcol, 256, 0, s>>>(n, dots + 4 * chunk, Zb, P);
            AWG_LAUNCH();
        }
        max_it = std::max(max_it, it);
        if (h->opt.verbose)
            fprintf(stderr, "libawg: W columns %d..%d: %d iterations, max relres %.3e\n", c0,
                    c0 + k, it, worst);
    }
    h->w_iters = max_it;
    h->w_relres = worst;
    for (double* p : {Vhat, R, Zb, Zo, P, Q, dots}) AWG_CUDA(cudaFreeAsync(p, s));
    AWG_CUDA(cudaStreamSynchronize(s));
    return AWG_OK;
}

// C = A^T B for A, B n x m column-major (ld n), C m x m symmetric: the
// float64 contraction of F = W^T (A W) (Def. 10).  Only the tiles on and
// above the diagonal are formed (64 x 64 per block, each thread 4 x 4, the
// reduction over n in 16-row chunks staged in shared memory, split over
// blockIdx.y into part[sp]); k_atb_sum adds the splits in order and mirrors
// the upper triangle, so C is exactly symmetric.
constexpr int AT_T = 64, AT_KC = 16;
__global__ void __launch_bounds__(256) k_atb_part(int n, int m, int klen, const double* __restrict__ A,
                                                  const double* __restrict__ B, double* __restrict__ part) {
    __shared__ double as[AT_KC][AT_T + 1];
    __shared__ double bs[AT_KC][AT_T + 1];
    __shared__ int tij[2];
    const int nt = (m + AT_T - 1) / AT_T;
    if (threadIdx.x == 0) {  // blockIdx.x -> (ti, tj), ti <= tj, row by row
        int t = blockIdx.x, ti = 0;
        while (t >= nt - ti) { t -= nt - ti; ti++; }
        tij[0] = ti;
        tij[1] = ti + t;
    }
    __syncthreads();
    const int i0 = tij[0] * AT_T, j0 = tij[1] * AT_T;
    const int k0s = blockIdx.y * klen, k1s = min(n, k0s + klen);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int k0 = k0s; k0 < k1s; k0 += AT_KC) {
        __syncthreads();
        for (int e = threadIdx.x; e < AT_KC * AT_T; e += 256) {
            const int c = e / AT_KC, kk = e % AT_KC, k = k0 + kk;
            const bool kin = k < k1s;
            as[kk][c] = (kin && i0 + c < m) ? A[(size_t)(i0 + c) * n + k] : 0.0;
            bs[kk][c] = (kin && j0 + c < m) ? B[(size_t)(j0 + c) * n + k] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < AT_KC; kk++) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; u++) { a[u] = as[kk][ty * 4 + u]; b[u] = bs[kk][tx * 4 + u]; }
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int v = 0; v < 4; v++) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
    }
    double* P = part + (size_t)blockIdx.y * m * m;
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
        for (int v = 0; v < 4; v++) {
            const int i = i0 + ty * 4 + u, j = j0 + tx * 4 + v;
            if (i < m && j < m) P[(size_t)j * m + i] = acc[u][v];
        }
}

__global__ void k_atb_sum(int m, int S, const double* __restrict__ part, double* __restrict__ C) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)m * m) return;
    const int i = (int)(e % m), j = (int)(e / m);
    const size_t src = (i <= j) ? e : (size_t)i * m + j;  // (j, i) above the diagonal
    double v = 0.0;
    for (int sp = 0; sp < S; sp++) v += part[(size_t)sp * m * m + src];
    C[e] = v;
}

static awg_status atb_sym(Handle* h, int n, int m, const double* A, const double* B, double* C, cudaStream_t s) {
    if (m == 0) return AWG_OK;
    const int nt = (m + AT_T - 1) / AT_T;
    const int tiles = nt * (nt + 1) / 2;
    const int S = std::max(1, std::min(16, (8 * 152 + tiles - 1) / tiles));
    const int klen = ((n + S - 1) / S + AT_KC - 1) / AT_KC * AT_KC;
    double* part = nullptr;
    AWG_CUDA(cudaMallocAsync(&part, (size_t)S * m * m * 8, s));
    k_atb_part<<<dim3(tiles, S), 256, 0, s>>>(n, m, klen, A, B, part);
    AWG_LAUNCH();
    const size_t len = (size_t)m * m;
    k_atb_sum<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(m, S, part, C);
    AWG_LAUNCH();
    AWG_CUDA(cudaFreeAsync(part, s));
    return AWG_OK;
}

// ------------------------------------------------------------ truncated W
// Wt(:, j) = W(:, j) with the entries below tol * max_i |W(i, j)| set to 0
// (column-major n x nm); cnt[j] = entries kept.  One block per column.
__global__ void __launch_bounds__(256) k_w_truncate(int n, const double* __restrict__ W, double tol,
                                                    double* __restrict__ Wt, int64_t* __restrict__ cnt) {
    __shared__ double red[32];
    __shared__ unsigned long long kept;
    const int j = blockIdx.x;
    const double* w = W + (size_t)j * n;
    double mx = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, fabs(w[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    if (threadIdx.x == 0) kept = 0ull;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    const double thr = tol * red[0];
    unsigned c = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = w[i];
        const bool keep = fabs(v) >= thr;
        Wt[(size_t)j * n + i] = keep ? v : 0.0;
        c += keep;
    }
    atomicAdd(&kept, (unsigned long long)c);
    __syncthreads();
    if (threadIdx.x == 0) cnt[j] = (int64_t)kept;
}

// CSC of the truncated W: column j's nonzeros in row order at colptr[j]
// (order-preserving compaction: warp ballots, then the warps' counts in
// order).  One block of 256 threads per column.
__global__ void __launch_bounds__(256) k_w_csc(int n, const double* __restrict__ Wt,
                                               const int64_t* __restrict__ colptr, int* __restrict__ row,
                                               double* __restrict__ val) {
    __shared__ int wc[8];
    const int j = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double* w = Wt + (size_t)j * n;
    int64_t base = colptr[j];
    for (int i0 = 0; i0 < n; i0 += 256) {
        const int i = i0 + threadIdx.x;
        const double v = i < n ? w[i] : 0.0;
        const bool nz = v != 0.0;
        const unsigned m = __ballot_sync(0xffffffffu, nz);
        if (lane == 0) wc[warp] = __popc(m);
        __syncthreads();
        int off = 0;
        for (int q = 0; q < warp; q++) off += wc[q];
        int tot = 0;
        for (int q = 0; q < 8; q++) tot += wc[q];
        if (nz) {
            const int64_t k = base + off + __popc(m & ((1u << lane) - 1u));
            row[k] = i;
            val[k] = v;
        }
        base += tot;
        __syncthreads();
    }
}

// CSR of the truncated W: row i's nonzeros in column order.  rcnt: a
// thread per row counts its kept entries; rfill: the same thread writes
// them from rowptr[i].
__global__ void k_w_rcnt(int n, int nm, const double* __restrict__ Wt, int64_t* __restrict__ rcnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t c = 0;
    for (int j = 0; j < nm; j++) c += Wt[(size_t)j * n + i] != 0.0;
    rcnt[i] = c;
}
__global__ void k_w_rfill(int n, int nm, const double* __restrict__ Wt, const int64_t* __restrict__ rowptr,
                          int* __restrict__ col, double* __restrict__ val) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t k = rowptr[i];
    for (int j = 0; j < nm; j++) {
        const double v = Wt[(size_t)j * n + i];
        if (v != 0.0) {
            col[k] = j;
            val[k] = v;
            k++;
        }
    }
}

// The truncated W of the float64 form (w_drop_tol > 0): the dense truncated
// copy (column-major, caller frees it) and its CSR / CSC in P
static awg_status build_truncated_W(Handle* h, const double* W64, double** Wt_out, PrecOps& P) {
    cudaStream_t s = h->stream;
    const int n = h->n, nm = h->n_minus;
    double* Wt = nullptr;
    int64_t* dcnt = nullptr;
    AWG_CUDA(cudaMallocAsync(&Wt, (size_t)n * nm * 8, s));
    AWG_CUDA(cudaMallocAsync(&dcnt, (size_t)std::max(n, nm) * 8, s));
    k_w_truncate<<<nm, 256, 0, s>>>(n, W64, h->opt.w_drop_tol, Wt, dcnt);
    AWG_LAUNCH();
    std::vector<int64_t> cnt(nm), ptr(std::max(n, nm) + 1, 0);
    AWG_CUDA(cudaMemcpyAsync(cnt.data(), dcnt, (size_t)nm * 8, cudaMemcpyDeviceToHost, s));
    AWG_CUDA(cudaStreamSynchronize(s));
    for (int j = 0; j < nm; j++) ptr[j + 1] = ptr[j] + cnt[j];
    const int64_t nnz = ptr[nm];
    P.sp_nnz = nnz;
    AWG_TRY(upload(h, P.sp_colptr, ptr.data(), (size_t)(nm + 1) * 8));
    AWG_TRY(dalloc(h, P.sp_row, (size_t)std::max<int64_t>(nnz, 1) * 4));
    AWG_TRY(dalloc(h, P.sp_cval, (size_t)std::max<int64_t>(nnz, 1) * 8));
    k_w_csc<<<nm, 256, 0, s>>>(n, Wt, (const int64_t*)P.sp_colptr.p, (int*)P.sp_row.p, (double*)P.sp_cval.p);
    AWG_LAUNCH();
    k_w_rcnt<<<(n + 255) / 256, 256, 0, s>>>(n, nm, Wt, dcnt);
    AWG_LAUNCH();
    std::vector<int64_t> rc(n);
    AWG_CUDA(cudaMemcpyAsync(rc.data(), dcnt, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    AWG_CUDA(cudaStreamSynchronize(s));
    ptr.assign(n + 1, 0);
    for (int i = 0; i < n; i++) ptr[i + 1] = ptr[i] + rc[i];
    AWG_TRY(upload(h, P.sp_rowptr, ptr.data(), (size_t)(n + 1) * 8));
    AWG_TRY(dalloc(h, P.sp_col, (size_t)std::max<int64_t>(nnz, 1) * 4));
    AWG_TRY(dalloc(h, P.sp_val, (size_t)std::max<int64_t>(nnz, 1) * 8));
    k_w_rfill<<<(n + 255) / 256, 256, 0, s>>>(n, nm, Wt, (const int64_t*)P.sp_rowptr.p, (int*)P.sp_col.p,
                                              (double*)P.sp_val.p);
    AWG_LAUNCH();
    AWG_CUDA(cudaFreeAsync(dcnt, s));
    if (h->opt.verbose)
        fprintf(stderr, "libawg: truncated W: %lld of %lld entries kept (tol %.1e)\n", (long long)nnz,
                (long long)n * nm, h->opt.w_drop_tol);
    *Wt_out = Wt;
    return AWG_OK;
}

// F = Wt^T A Wt for a column-major (rounded) W, its inverse into Finv
static awg_status build_F(Handle* h, const double* Wt, DevBuf& Finv, DevBuf* keepF) {
    cudaStream_t s = h->stream;
    const int n = h->n, nm = h->n_minus;
    double* AW = nullptr;
    AWG_CUDA(cudaMallocAsync(&AW, (size_t)n * nm * 8, s));
    AWG_TRY(blk_spmm(h, Wt, AW, nm, s));
    DevBuf F;
    AWG_TRY(dalloc(h, F, (size_t)nm * nm * 8));
    const double t0 = now_ms();
    AWG_TRY(atb_sym(h, n, nm, Wt, AW, (double*)F.p, s));  // F = W^T (A W), exactly symmetric
    AWG_CUDA(cudaFreeAsync(AW, s));
    AWG_CUDA(cudaStreamSynchronize(s));
    const double t1 = now_ms();
    AWG_TRY(spd_inverse(h, F, Finv, nm));
    if (h->opt.verbose)
        fprintf(stderr, "libawg: F (%d x %d): W^T A W %.1f ms, Cholesky inverse %.1f ms\n", nm, nm, t1 - t0,
                now_ms() - t1);
    if (keepF) { dfree(h, *keepF); *keepF = F; } else dfree(h, F);
    return AWG_OK;
}

// (C^-1 - Vhat^T Wt)^-1 for H_3,inex (Thm. 7), C = diag|L^s_-| (strict)
static awg_status build_inex(Handle* h, const double* Wt, DevBuf& out) {
    cudaStream_t s = h->stream;
    const int n = h->n, nm = h->n_minus, N = h->N;
    double *Vhat = nullptr, *loc = nullptr;
    AWG_CUDA(cudaMallocAsync(&loc, (size_t)h->sum_ns * nm * 8, s));
    AWG_TRY(blk_gather(h, Wt, loc, nm, s));
    DevBuf M;
    AWG_TRY(dalloc(h, M, (size_t)nm * nm * 8));
    std::vector<GemmDesc> d;
    const double* V = (const double*)h->Vm.p;
    for (int t = 0; t < N; t++) {
        const int m = h->h_ns[t], k = h->h_nstrict[t];
        if (k == 0) continue;
        d.push_back({V + h->h_vm_off[t], loc + (int64_t)h->h_sub_ptr[t] * nm, (double*)M.p + h->h_wcol_ptr[t],
                     k, nm, m, m, m, nm, 1, 0, 1.0, 0.0});
    }
    AWG_TRY(gemm_batched(h, d, s));
    // diag of C^-1 in wcol order
    std::vector<double> lam(h->n_minus_all);
    AWG_CUDA(cudaMemcpyAsync(lam.data(), h->lam_m.p, lam.size() * 8, cudaMemcpyDeviceToHost, s));
    AWG_CUDA(cudaStreamSynchronize(s));
    std::vector<double> cinv(nm);
    for (int t = 0; t < N; t++)
        for (int j = 0; j < h->h_nstrict[t]; j++) cinv[h->h_wcol_ptr[t] + j] = -1.0 / lam[h->h_nm_ptr[t] + j];
    double* dcinv = nullptr;
    AWG_CUDA(cudaMallocAsync(&dcinv, (size_t)nm * 8, s));
    AWG_CUDA(cudaMemcpyAsync(dcinv, cinv.data(), nm * 8, cudaMemcpyHostToDevice, s));
    // M = C^-1 - Vhat^T W
    k_neg_offdiag<<<(unsigned)(((size_t)nm * nm + 255) / 256), 256, 0, s>>>(nm, (double*)M.p);
    AWG_LAUNCH();
    k_diag_minus<<<(nm + 255) / 256, 256, 0, s>>>(nm, dcinv, (double*)M.p);
    AWG_LAUNCH();
    int64_t zero = 0;
    DevBuf dm, doff;
    AWG_TRY(upload(h, dm, &nm, sizeof(int)));
    AWG_TRY(upload(h, doff, &zero, sizeof(int64_t)));
    k_symmetrize<<<dim3(1, 64), 256, 0, s>>>((int*)dm.p, (int64_t*)doff.p, (double*)M.p);
    AWG_LAUNCH();
    AWG_TRY(spd_inverse(h, M, out, nm));
    dfree(h, M);
    dfree(h, dm);
    dfree(h, doff);
    AWG_CUDA(cudaFreeAsync(loc, s));
    AWG_CUDA(cudaFreeAsync(dcinv, s));
    (void)Vhat;
    return AWG_OK;
}

// Sparse correction of the float16 W (rows on the device, columns by a
// stable transpose on the host: setup-time only)
static awg_status build_w16_correction(Handle* h, PrecOps& P, const double* W64, const double* cmax,
                                       double keep) {
    cudaStream_t s = h->stream;
    const int n = h->n, nm = h->n_minus;
    AWG_TRY(dalloc(h, P.corr_rowptr, (size_t)(n + 1) * 4));
    AWG_TRY(dalloc(h, P.corr_colptr, (size_t)(nm + 1) * 4));
    std::vector<int> cnt(n), rp(n + 1, 0);
    if (keep > 0.0) {
        k_w16_corr_count<<<(n + 255) / 256, 256, 0, s>>>(n, nm, W64, cmax, keep, (int*)P.corr_rowptr.p);
        AWG_LAUNCH();
        AWG_CUDA(cudaMemcpyAsync(cnt.data(), P.corr_rowptr.p, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
        AWG_CUDA(cudaStreamSynchronize(s));
        int64_t tot = 0;
        for (int i = 0; i < n; i++) tot += cnt[i];
        if (tot > INT32_MAX) return AWG_ERR_INVALID_ARG;
        for (int i = 0; i < n; i++) rp[i + 1] = rp[i] + cnt[i];
    }
    const int64_t nnz = rp[n];
    P.corr_nnz = nnz;
    AWG_CUDA(cudaMemcpyAsync(P.corr_rowptr.p, rp.data(), (size_t)(n + 1) * 4, cudaMemcpyHostToDevice, s));
    for (DevBuf* b : {&P.corr_col, &P.corr_row}) AWG_TRY(dalloc(h, *b, (size_t)std::max<int64_t>(1, nnz) * 4));
    for (DevBuf* b : {&P.corr_val, &P.corr_cval}) AWG_TRY(dalloc(h, *b, (size_t)std::max<int64_t>(1, nnz) * 4));
    std::vector<int> cp(nm + 1, 0);
    if (nnz > 0) {
        k_w16_corr_fill<<<(n + 255) / 256, 256, 0, s>>>(n, nm, W64, cmax, keep, (float*)P.rscale.p,
                                                         (float*)P.cscale.p, (int*)P.corr_rowptr.p,
                                                         (int*)P.corr_col.p, (float*)P.corr_val.p);
        AWG_LAUNCH();
        std::vector<int> col(nnz), row(nnz);
        std::vector<float> val(nnz), cval(nnz);
        AWG_CUDA(cudaMemcpyAsync(col.data(), P.corr_col.p, (size_t)nnz * 4, cudaMemcpyDeviceToHost, s));
        AWG_CUDA(cudaMemcpyAsync(val.data(), P.corr_val.p, (size_t)nnz * 4, cudaMemcpyDeviceToHost, s));
        AWG_CUDA(cudaStreamSynchronize(s));
        for (int64_t k = 0; k < nnz; k++) cp[col[k] + 1]++;
        for (int j = 0; j < nm; j++) cp[j + 1] += cp[j];
        std::vector<int> next(cp.begin(), cp.end() - 1);
        for (int i = 0; i < n; i++)  // rows ascending within each column
            for (int k = rp[i]; k < rp[i + 1]; k++) {
                const int t = next[col[k]]++;
                row[t] = i;
                cval[t] = val[k];
            }
        AWG_CUDA(cudaMemcpyAsync(P.corr_row.p, row.data(), (size_t)nnz * 4, cudaMemcpyHostToDevice, s));
        AWG_CUDA(cudaMemcpyAsync(P.corr_cval.p, cval.data(), (size_t)nnz * 4, cudaMemcpyHostToDevice, s));
    }
    AWG_CUDA(cudaMemcpyAsync(P.corr_colptr.p, cp.data(), (size_t)(nm + 1) * 4, cudaMemcpyHostToDevice, s));
    AWG_CUDA(cudaStreamSynchronize(s));
    return AWG_OK;
}

// G^s = (R^s A_+ R^sT)^-1 (plus: H^AS_+) or (R^s A R^sT)^-1 (H^AS) for
// every subdomain (Def. 8), over the float64 local operators of H^NN: the
// dense block R^s A R^sT (plus the neighbour terms of A_-, Section 4.4 item
// 4), Cholesky, triangular inverse, L^-T L^-1.  `work` holds dense_total
// doubles.
static awg_status build_local_as(Handle* h, double* work, bool plus) {
    cudaStream_t s = h->stream;
    const int N = h->N;
    AWG_TRY(assemble_local(h, (double*)h->val.p, work));
    if (plus && h->n_minus_all > 0) {
        k_add_nbr_MB<<<dim3(N, 16), 256, 0, s>>>((int*)h->ns.p, (int64_t*)h->dense_off.p, (int*)h->sub_ptr.p,
                                                 (int*)h->sub_idx.p, (int*)h->inc_ptr.p, (int*)h->inc_pos.p,
                                                 (int*)h->inc_sub.p, (int*)h->nm_ptr.p, (int64_t*)h->vm_off.p,
                                                 (double*)h->Vm.p, (double*)h->lam_m.p, work);
        AWG_LAUNCH();
    }
    AWG_CUDA(cudaMemsetAsync(h->flag.p, 0, sizeof(int), s));
    AWG_TRY(potrf_batched(h, work, (int*)h->ns.p, (int64_t*)h->dense_off.p, N, h->max_ns, (int*)h->flag.p, s));
    AWG_TRY(check_flag(h, FLAG_NOT_SPD, AWG_ERR_NOT_SPD));
    AWG_TRY(trtri_batched(h, work, (int*)h->ns.p, (int64_t*)h->dense_off.p, N, h->max_ns, s));
    std::vector<GemmDesc> d;
    double* G = (double*)h->prec[AWG_FP64].G.p;
    for (int t = 0; t < N; t++) {
        const int m = h->h_ns[t];
        const int64_t o = h->h_dense_off[t];
        d.push_back({work + o, work + o, G + o, m, m, m, m, m, m, 1, 0, 1.0, 0.0});
    }
    AWG_TRY(gemm_batched(h, d, s));  // L^-T L^-1
    AWG_CUDA(cudaStreamSynchronize(s));
    return AWG_OK;
}

// Y_L(thr, M_A, M_B) of every subdomain (Def. 9) by the dense route: M_B =
// L L^T, eigenpairs of L^-1 M_A L^-T below thr, Y = L^-T Q (M_B-orthonormal
// columns).  MA, MB and work are dense arenas (destroyed); Y gets the
// column-major n^s x cnt[s] blocks at yoff[s].
static awg_status dense_pencil(Handle* h, double* MA, double* MB, double* work, double thr, std::vector<int>& cnt,
                               DevBuf& Y, std::vector<int64_t>& yoff) {
    cudaStream_t s = h->stream;
    const int N = h->N;
    AWG_CUDA(cudaMemsetAsync(h->flag.p, 0, sizeof(int), s));
    AWG_TRY(potrf_batched(h, MB, (int*)h->ns.p, (int64_t*)h->dense_off.p, N, h->max_ns, (int*)h->flag.p, s));
    AWG_TRY(check_flag(h, FLAG_NOT_SPD, AWG_ERR_NOT_SPD));
    AWG_TRY(trtri_batched(h, MB, (int*)h->ns.p, (int64_t*)h->dense_off.p, N, h->max_ns, s));
    {
        std::vector<GemmDesc> d1, d2;
        for (int t = 0; t < N; t++) {
            const int m = h->h_ns[t];
            const int64_t o = h->h_dense_off[t];
            d1.push_back({MB + o, MA + o, work + o, m, m, m, m, m, m, 0, 0, 1.0, 0.0});
            d2.push_back({work + o, MB + o, MA + o, m, m, m, m, m, m, 0, 1, 1.0, 0.0});
        }
        AWG_TRY(gemm_batched(h, d1, s));  // work = L^-1 M_A
        AWG_TRY(gemm_batched(h, d2, s));  // M_A <- work L^-T
    }
    k_symmetrize<<<dim3(N, 16), 256, 0, s>>>((int*)h->ns.p, (int64_t*)h->dense_off.p, MA);
    AWG_LAUNCH();
    std::vector<int> strict, vptr;
    std::vector<int64_t> qoff;
    DevBuf Q, qvals;
    AWG_CUDA(cudaMemsetAsync(h->flag.p, 0, sizeof(int), s));
    AWG_TRY(eig_select_batched(h, MA, (int*)h->ns.p, (int64_t*)h->dense_off.p, h->h_ns, N, h->max_ns, 1, thr, cnt,
                               strict, Q, qoff, qvals, vptr, s));
    AWG_TRY(check_flag(h, FLAG_EIG, AWG_ERR_EIG));
    yoff = qoff;
    AWG_TRY(dalloc(h, Y, std::max<size_t>(8, (size_t)qoff[N] * 8)));
    std::vector<GemmDesc> d;
    for (int t = 0; t < N; t++) {
        const int m = h->h_ns[t], c = cnt[t];
        if (c == 0) continue;
        d.push_back({MB + h->h_dense_off[t], (double*)Q.p + qoff[t], (double*)Y.p + qoff[t], m, c, m, m, m, m, 1, 0,
                     1.0, 0.0});  // Y = L^-T Q
    }
    AWG_TRY(gemm_batched(h, d, s));
    AWG_CUDA(cudaStreamSynchronize(s));
    dfree(h, Q);
    dfree(h, qvals);
    return AWG_OK;
}

// V^0_AS(tau_sharp, tau_flat) (Thm. 5): per subdomain the columns of
// Y_L(1/tau_flat, D^s^-1 A^s_+ D^s^-1, R^s A R^sT) followed by those of
// Y_L(tau_sharp, R^s A R^sT, R^s A_+ R^sT), both by the dense route, packed
// into Z.  A1 holds dense_total doubles.
static awg_status geneo_as_dense(Handle* h, double* A1) {
    cudaStream_t s = h->stream;
    const int N = h->N;
    const dim3 gblk(N, 16);
    DevBuf A2, A3, Y1, Y2;
    AWG_TRY(dalloc(h, A2, (size_t)h->dense_total * 8));
    AWG_TRY(dalloc(h, A3, (size_t)h->dense_total * 8));
    std::vector<int> k1, k2;
    std::vector<int64_t> o1, o2;
    // pencil 1: M_A against R^s A R^sT, below 1 / tau_flat
    AWG_TRY(assemble_local(h, (double*)h->val.p, A1));
    AWG_TRY(assemble_local(h, (double*)h->bval.p, (double*)A2.p));
    k_form_MA<<<gblk, 256, 0, s>>>((int*)h->ns.p, (int64_t*)h->dense_off.p, (int*)h->sub_ptr.p, (int*)h->sub_idx.p,
                                   (double*)h->dvec.p, (int*)h->nm_ptr.p, (int64_t*)h->vm_off.p, (double*)h->Vm.p,
                                   (double*)h->lam_m.p, (double*)A2.p);
    AWG_LAUNCH();
    AWG_TRY(dense_pencil(h, (double*)A2.p, A1, (double*)A3.p, 1.0 / h->opt.tau_flat, k1, Y1, o1));
    // pencil 2: R^s A R^sT against R^s A_+ R^sT, below tau_sharp
    AWG_TRY(assemble_local(h, (double*)h->val.p, (double*)A2.p));
    AWG_TRY(assemble_local(h, (double*)h->val.p, A1));
    if (h->n_minus_all > 0) {
        k_add_nbr_MB<<<gblk, 256, 0, s>>>((int*)h->ns.p, (int64_t*)h->dense_off.p, (int*)h->sub_ptr.p,
                                          (int*)h->sub_idx.p, (int*)h->inc_ptr.p, (int*)h->inc_pos.p,
                                          (int*)h->inc_sub.p, (int*)h->nm_ptr.p, (int64_t*)h->vm_off.p,
                                          (double*)h->Vm.p, (double*)h->lam_m.p, A1);
        AWG_LAUNCH();
    }
    AWG_TRY(dense_pencil(h, (double*)A2.p, A1, (double*)A3.p, h->tau, k2, Y2, o2));
    dfree(h, A2);
    dfree(h, A3);
    std::vector<int> mc(N);
    for (int t = 0; t < N; t++) mc[t] = k1[t] + k2[t];
    h->h_modes = mc;
    h->h_mode_ptr.assign(N + 1, 0);
    h->h_z_off.assign(N + 1, 0);
    for (int t = 0; t < N; t++) {
        h->h_mode_ptr[t + 1] = h->h_mode_ptr[t] + mc[t];
        h->h_z_off[t + 1] = h->h_z_off[t] + (int64_t)h->h_ns[t] * mc[t];
    }
    h->n0 = h->h_mode_ptr[N];
    AWG_TRY(upload(h, h->modes, mc.data(), N * sizeof(int)));
    AWG_TRY(upload(h, h->mode_ptr, h->h_mode_ptr.data(), (N + 1) * sizeof(int)));
    AWG_TRY(upload(h, h->z_off, h->h_z_off.data(), (N + 1) * sizeof(int64_t)));
    AWG_TRY(dalloc(h, h->Z, std::max<size_t>(8, (size_t)h->h_z_off[N] * 8)));
    for (int t = 0; t < N; t++) {  // Z^s = [Y1^s Y2^s], column-major n^s x (k1 + k2)
        double* z = (double*)h->Z.p + h->h_z_off[t];
        const size_t b1 = (size_t)h->h_ns[t] * k1[t] * 8, b2 = (size_t)h->h_ns[t] * k2[t] * 8;
        if (b1) AWG_CUDA(cudaMemcpyAsync(z, (double*)Y1.p + o1[t], b1, cudaMemcpyDeviceToDevice, s));
        if (b2) AWG_CUDA(cudaMemcpyAsync((char*)z + b1, (double*)Y2.p + o2[t], b2, cudaMemcpyDeviceToDevice, s));
    }
    AWG_CUDA(cudaStreamSynchronize(s));
    dfree(h, Y1);
    dfree(h, Y2);
    h->geneo_dense = N;
    h->geneo_its_max = 0;
    h->geneo_its_sum = 0;
    return AWG_OK;
}

awg_status build_setup_numeric(Handle* h) {
    cudaStream_t s = h->stream;
    const int N = h->N, n = h->n;
    const int maxm = h->max_ns;
    double t0 = now_ms();
    const dim3 gblk(N, 16);
    // ---------------------------------------------- 1. eigen-split of B^s
    NvtxRange nv_("awg_setup: eigen-split of B^s");
    DevBuf A1;
    AWG_TRY(dalloc(h, A1, (size_t)h->dense_total * 8));
    AWG_TRY(assemble_local(h, (double*)h->bval.p, (double*)A1.p));
    std::vector<int> cnt, strict, vptr;
    std::vector<int64_t> voff;
    AWG_CUDA(cudaMemsetAsync(h->flag.p, 0, sizeof(int), s));
    AWG_TRY(eig_select_batched(h, (double*)A1.p, (int*)h->ns.p, (int64_t*)h->dense_off.p, h->h_ns, N,
                               maxm, 0, h->opt.zero_rtol, cnt, strict, h->Vm, voff, h->lam_m, vptr, s));
    AWG_TRY(check_flag(h, FLAG_EIG, AWG_ERR_EIG));
    h->h_nm = cnt;
    h->h_nstrict = strict;
    h->h_nm_ptr = vptr;
    h->h_vm_off = voff;
    h->n_minus_all = vptr[N];
    h->h_wcol_ptr.assign(N + 1, 0);
    for (int t = 0; t < N; t++) h->h_wcol_ptr[t + 1] = h->h_wcol_ptr[t] + strict[t];
    h->n_minus = h->h_wcol_ptr[N];
    h->ldw = (h->n_minus + 7) / 8 * 8;  // W rows 16-byte aligned for vector loads
    AWG_TRY(upload(h, h->nm, cnt.data(), N * sizeof(int)));
    AWG_TRY(upload(h, h->nstrict, strict.data(), N * sizeof(int)));
    AWG_TRY(upload(h, h->nm_ptr, vptr.data(), (N + 1) * sizeof(int)));
    AWG_TRY(upload(h, h->vm_off, voff.data(), (N + 1) * sizeof(int64_t)));
    AWG_TRY(upload(h, h->wcol_ptr, h->h_wcol_ptr.data(), (N + 1) * sizeof(int)));
    AWG_CUDA(cudaStreamSynchronize(s));
    double t1 = now_ms();
    h->setup_ms[1] = t1 - t0;

    // ---------------------------------------------- 2. local factors
    nv_.next("awg_setup: local factors");
    AWG_TRY(assemble_local(h, (double*)h->bval.p, (double*)A1.p));
    AWG_TRY(dalloc(h, h->sigma, N * 8));
    k_form_K<<<N, 256, 0, s>>>((int*)h->ns.p, (int64_t*)h->dense_off.p, (int*)h->nm_ptr.p,
                               (int64_t*)h->vm_off.p, (double*)h->Vm.p, (double*)h->lam_m.p,
                               (double*)A1.p, (double*)h->sigma.p);
    AWG_LAUNCH();
    AWG_CUDA(cudaMemsetAsync(h->flag.p, 0, sizeof(int), s));
    AWG_TRY(potrf_batched(h, (double*)A1.p, (int*)h->ns.p, (int64_t*)h->dense_off.p, N, maxm,
                          (int*)h->flag.p, s));
    AWG_TRY(check_flag(h, FLAG_NOT_SPD, AWG_ERR_NOT_SPD));
    AWG_TRY(trtri_batched(h, (double*)A1.p, (int*)h->ns.p, (int64_t*)h->dense_off.p, N, maxm, s));
    DevBuf& G = h->prec[AWG_FP64].G;
    AWG_TRY(dalloc(h, G, (size_t)h->dense_total * 8));
    {
        std::vector<GemmDesc> d;
        const double* L = (const double*)A1.p;
        for (int t = 0; t < N; t++) {
            const int m = h->h_ns[t];
            d.push_back({L + h->h_dense_off[t], L + h->h_dense_off[t], (double*)G.p + h->h_dense_off[t],
                         m, m, m, m, m, m, 1, 0, 1.0, 0.0});
        }
        AWG_TRY(gemm_batched(h, d, s));  // K^-1 = L^-T L^-1
    }
    if (h->n_minus_all > 0) {
        const size_t vlen = (size_t)voff[N];
        double *T = nullptr, *S = nullptr, *U = nullptr;
        AWG_CUDA(cudaMallocAsync(&T, vlen * 8, s));
        AWG_CUDA(cudaMallocAsync(&U, vlen * 8, s));
        size_t slen = 0;
        std::vector<size_t> soff(N + 1, 0);
        for (int t = 0; t < N; t++) soff[t + 1] = soff[t] + (size_t)cnt[t] * cnt[t];
        slen = soff[N];
        AWG_CUDA(cudaMallocAsync(&S, std::max<size_t>(slen, 1) * 8, s));
        std::vector<GemmDesc> d1, d2, d3;
        const double* V = (const double*)h->Vm.p;
        for (int t = 0; t < N; t++) {
            const int m = h->h_ns[t], nu = cnt[t];
            if (nu == 0) continue;
            const double* Kinv = (const double*)G.p + h->h_dense_off[t];
            d1.push_back({Kinv, V + voff[t], T + voff[t], m, nu, m, m, m, m, 0, 0, 1.0, 0.0});
            d2.push_back({V + voff[t], T + voff[t], S + soff[t], nu, nu, m, m, m, nu, 1, 0, 1.0, 0.0});
            d3.push_back({V + voff[t], S + soff[t], U + voff[t], m, nu, nu, m, nu, m, 0, 0, 1.0, 0.0});
        }
        AWG_TRY(gemm_batched(h, d1, s));
        AWG_TRY(gemm_batched(h, d2, s));
        AWG_TRY(gemm_batched(h, d3, s));
        k_form_G<<<gblk, 256, 0, s>>>((int*)h->ns.p, (int64_t*)h->dense_off.p, (int*)h->sub_ptr.p,
                                      (int*)h->sub_idx.p, (double*)h->dvec.p, (int*)h->nm_ptr.p,
                                      (int64_t*)h->vm_off.p, V, T, U, (double*)G.p);
        AWG_LAUNCH();
        for (double* p : {T, S, U}) AWG_CUDA(cudaFreeAsync(p, s));
    } else {
        k_form_G<<<gblk, 256, 0, s>>>((int*)h->ns.p, (int64_t*)h->dense_off.p, (int*)h->sub_ptr.p,
                                      (int*)h->sub_idx.p, (double*)h->dvec.p, (int*)h->nm_ptr.p,
                                      (int64_t*)h->vm_off.p, (double*)h->Vm.p, nullptr, nullptr,
                                      (double*)G.p);
        AWG_LAUNCH();
    }
    h->prec[AWG_FP64].built = true;
    AWG_CUDA(cudaStreamSynchronize(s));
    double t2 = now_ms();
    h->setup_ms[2] = t2 - t1;

    // ---------------------------------------------- 3. GenEO
    nv_.next("awg_setup: GenEO");
    if (h->opt.h2 == AWG_H2_AS_HYB) {  // two pencils, dense route (Thm. 5)
        AWG_TRY(geneo_as_dense(h, (double*)A1.p));
    } else {
        // A1 <- M_B = R^s A R^sT + neighbour terms; A2 <- M_A
        DevBuf A2, A3;
        AWG_TRY(assemble_local(h, (double*)h->val.p, (double*)A1.p));
        if (h->n_minus_all > 0) {
            k_add_nbr_MB<<<gblk, 256, 0, s>>>((int*)h->ns.p, (int64_t*)h->dense_off.p, (int*)h->sub_ptr.p,
                                              (int*)h->sub_idx.p, (int*)h->inc_ptr.p, (int*)h->inc_pos.p,
                                              (int*)h->inc_sub.p, (int*)h->nm_ptr.p, (int64_t*)h->vm_off.p,
                                              (double*)h->Vm.p, (double*)h->lam_m.p, (double*)A1.p);
            AWG_LAUNCH();
        }
        AWG_TRY(dalloc(h, A2, (size_t)h->dense_total * 8));
        AWG_TRY(assemble_local(h, (double*)h->bval.p, (double*)A2.p));
        k_form_MA<<<gblk, 256, 0, s>>>((int*)h->ns.p, (int64_t*)h->dense_off.p, (int*)h->sub_ptr.p,
                                       (int*)h->sub_idx.p, (double*)h->dvec.p, (int*)h->nm_ptr.p,
                                       (int64_t*)h->vm_off.p, (double*)h->Vm.p, (double*)h->lam_m.p,
                                       (double*)A2.p);
        AWG_LAUNCH();
        // Block eigensolver first (it reads M_A and M_B and keeps them); the
        // pencils it does not certify go to the dense eigensolver below.
        GeneoIter gi;
        std::vector<int> sel;
        h->geneo_its_max = 0;
        h->geneo_its_sum = 0;
        if (h->opt.geneo_solver != 0) {
            DevBuf prm;
            if (h->opt.geneo_solver == 2)
                AWG_TRY(upload(h, prm, h->h_learned.data(), LEARNED_NPARAM * sizeof(double)));
            AWG_TRY(geneo_block_solve(h, (double*)A2.p, (double*)A1.p, (double*)prm.p, h->opt.geneo_block,
                                      h->opt.geneo_maxit, 1e-13, gi));
            dfree(h, prm);
            for (int t = 0; t < N; t++) {
                if (gi.ecount[t] < 0) sel.push_back(t);
                h->geneo_its_max = std::max(h->geneo_its_max, gi.its[t]);
                h->geneo_its_sum += gi.its[t];
            }
        } else {
            for (int t = 0; t < N; t++) sel.push_back(t);
        }
        h->geneo_dense = (int)sel.size();
        // dense eigensolver on that subset: M_B = L L^T, eigenpairs of
        // L^-1 M_A L^-T below tau, Y = L^-T Q
        const int nsel = (int)sel.size();
        std::vector<int> mc_sel;
        std::vector<int64_t> qoff;
        DevBuf Q, qvals, dms, dos;
        if (nsel > 0) {
            std::vector<int> hms(nsel);
            std::vector<int64_t> hos(nsel);
            int maxsel = 1;
            for (int k = 0; k < nsel; k++) {
                hms[k] = h->h_ns[sel[k]];
                hos[k] = h->h_dense_off[sel[k]];
                maxsel = std::max(maxsel, hms[k]);
            }
            AWG_TRY(upload(h, dms, hms.data(), nsel * sizeof(int)));
            AWG_TRY(upload(h, dos, hos.data(), nsel * sizeof(int64_t)));
            AWG_CUDA(cudaMemsetAsync(h->flag.p, 0, sizeof(int), s));
            AWG_TRY(potrf_batched(h, (double*)A1.p, (int*)dms.p, (int64_t*)dos.p, nsel, maxsel, (int*)h->flag.p, s));
            AWG_TRY(check_flag(h, FLAG_NOT_SPD, AWG_ERR_NOT_SPD));
            AWG_TRY(trtri_batched(h, (double*)A1.p, (int*)dms.p, (int64_t*)dos.p, nsel, maxsel, s));
            AWG_TRY(dalloc(h, A3, (size_t)h->dense_total * 8));
            {
                std::vector<GemmDesc> d1, d2;
                const double* Li = (const double*)A1.p;
                for (int t : sel) {
                    const int m = h->h_ns[t];
                    const int64_t o = h->h_dense_off[t];
                    d1.push_back({Li + o, (double*)A2.p + o, (double*)A3.p + o, m, m, m, m, m, m, 0, 0, 1.0, 0.0});
                    d2.push_back({(double*)A3.p + o, Li + o, (double*)A2.p + o, m, m, m, m, m, m, 0, 1, 1.0, 0.0});
                }
                AWG_TRY(gemm_batched(h, d1, s));  // A3 = L^-1 M_A
                AWG_TRY(gemm_batched(h, d2, s));  // A2 = A3 L^-T
            }
            dfree(h, A3);
            k_symmetrize<<<dim3(nsel, 16), 256, 0, s>>>((int*)dms.p, (int64_t*)dos.p, (double*)A2.p);
            AWG_LAUNCH();
            std::vector<int> mcs, mptr;
            AWG_CUDA(cudaMemsetAsync(h->flag.p, 0, sizeof(int), s));
            AWG_TRY(eig_select_batched(h, (double*)A2.p, (int*)dms.p, (int64_t*)dos.p, hms, nsel, maxsel, 1,
                                       h->tau, mc_sel, mcs, Q, qoff, qvals, mptr, s));
            AWG_TRY(check_flag(h, FLAG_EIG, AWG_ERR_EIG));
        }
        {
            std::vector<int> mc(N, 0);
            for (int t = 0; t < N; t++)
                if (h->opt.geneo_solver != 0 && gi.ecount[t] >= 0) mc[t] = h->h_nm[t] + gi.ecount[t];
            for (int k = 0; k < nsel; k++) mc[sel[k]] = mc_sel[k];
            h->h_modes = mc;
            h->h_mode_ptr.assign(N + 1, 0);
            h->h_z_off.assign(N + 1, 0);
            for (int t = 0; t < N; t++) {
                h->h_mode_ptr[t + 1] = h->h_mode_ptr[t] + mc[t];
                h->h_z_off[t + 1] = h->h_z_off[t] + (int64_t)h->h_ns[t] * mc[t];
            }
            h->n0 = h->h_mode_ptr[N];
            AWG_TRY(upload(h, h->modes, mc.data(), N * sizeof(int)));
            AWG_TRY(upload(h, h->mode_ptr, h->h_mode_ptr.data(), (N + 1) * sizeof(int)));
            AWG_TRY(upload(h, h->z_off, h->h_z_off.data(), (N + 1) * sizeof(int64_t)));
            AWG_TRY(dalloc(h, h->Z, std::max<size_t>(8, (size_t)h->h_z_off[N] * 8)));
            if (h->opt.geneo_solver != 0) {
                AWG_TRY(geneo_block_pack(h, gi, (int64_t*)h->z_off.p, (double*)h->Z.p));
                geneo_block_free(h, gi);
            }
            std::vector<GemmDesc> d;
            const double* Li = (const double*)A1.p;
            for (int k = 0; k < nsel; k++) {
                const int t = sel[k], m = h->h_ns[t], c = mc_sel[k];
                if (c == 0) continue;
                d.push_back({Li + h->h_dense_off[t], (double*)Q.p + qoff[k], (double*)h->Z.p + h->h_z_off[t], m, c, m,
                             m, m, m, 1, 0, 1.0, 0.0});  // Y = L^-T Q
            }
            AWG_TRY(gemm_batched(h, d, s));
            AWG_CUDA(cudaStreamSynchronize(s));
            for (DevBuf* bb : {&Q, &qvals, &dms, &dos}) dfree(h, *bb);
        }
        dfree(h, A2);
    }
    // H^AS_+ (Thm. 3) / H^AS (Thm. 5): the local solvers become
    // (R^s A_+ R^sT)^-1 / (R^s A R^sT)^-1, after the GenEO solve (whose block
    // solver applies the H^NN local operators)
    if (h->opt.h2 != AWG_H2_NN_HYB) AWG_TRY(build_local_as(h, (double*)A1.p, h->opt.h2 != AWG_H2_AS_HYB));
    dfree(h, A1);
    double t3 = now_ms();
    h->setup_ms[3] = t3 - t2;

    // ---------------------------------------------- 4. E = Z^T A_+ Z
    nv_.next("awg_setup: E");
    const int n0 = h->n0;
    if (n0 > 0) {
        AWG_TRY(dalloc(h, h->E, (size_t)n0 * n0 * 8));
        const size_t budget = (size_t)16 << 30;
        const int chunk = (int)std::max<size_t>(1, std::min<size_t>(n0, budget / ((size_t)n * 8 * 4)));
        double *Zc = nullptr, *Qc = nullptr;
        AWG_CUDA(cudaMallocAsync(&Zc, (size_t)n * chunk * 8, s));
        AWG_CUDA(cudaMallocAsync(&Qc, (size_t)n * chunk * 8, s));
        for (int c0 = 0; c0 < n0; c0 += chunk) {
            const int k = std::min(chunk, n0 - c0);
            AWG_CUDA(cudaMemsetAsync(Zc, 0, (size_t)n * k * 8, s));
            k_scatter_cols<<<N, 256, 0, s>>>(n, (int*)h->sub_ptr.p, (int*)h->sub_idx.p,
                                             (int*)h->mode_ptr.p, (int64_t*)h->z_off.p,
                                             (double*)h->Z.p, Zc, c0, k);
            AWG_LAUNCH();
            AWG_TRY(blk_aplus(h, Zc, Qc, k, s));
            AWG_TRY(blk_zt(h, Qc, (double*)h->E.p + (size_t)c0 * n0, k, s));
        }
        AWG_CUDA(cudaFreeAsync(Zc, s));
        AWG_CUDA(cudaFreeAsync(Qc, s));
        int64_t zero = 0;
        DevBuf dm, doff;
        AWG_TRY(upload(h, dm, &n0, sizeof(int)));
        AWG_TRY(upload(h, doff, &zero, sizeof(int64_t)));
        k_symmetrize<<<dim3(1, 64), 256, 0, s>>>((int*)dm.p, (int64_t*)doff.p, (double*)h->E.p);
        AWG_LAUNCH();
        dfree(h, dm);
        dfree(h, doff);
        AWG_CUDA(cudaStreamSynchronize(s));
        const double te = now_ms();
        AWG_TRY(spd_inverse(h, h->E, h->Einv, n0));
        if (h->opt.verbose)
            fprintf(stderr, "libawg: E (%d x %d): Z^T A_+ Z %.1f ms, Cholesky inverse %.1f ms\n", n0, n0,
                    te - t3, now_ms() - te);
    }
    // workspace of the single-RHS apply
    h->red_blocks = std::min(1216, std::max(1, (n + 127) / 128));
    AWG_TRY(dalloc(h, h->ws, ws_bytes(h)));
    AWG_CUDA(cudaMemsetAsync(h->ws.p, 0, ws_bytes(h), s));  // ticket counters start at zero
    AWG_TRY(set_smem_limits(h));
    AWG_CUDA(cudaStreamSynchronize(s));
    double t4 = now_ms();
    h->setup_ms[4] = t4 - t3;

    // float32 local operators: used by the float32 and bfloat16 apply forms
    // (the bfloat16 form rounds only W) and by the W solve's preconditioner
    if ((h->opt.precisions & 14) || h->opt.w_precision == AWG_MIXED_FP32) {
        PrecOps& P = h->prec[AWG_MIXED_FP32];
        h->h_g32_off.assign(N + 1, 0);
        for (int t = 0; t < N; t++)
            h->h_g32_off[t + 1] = h->h_g32_off[t] + (int64_t)h->h_ns[t] * ((h->h_ns[t] + 3) & ~3);
        AWG_TRY(upload(h, h->g32_off, h->h_g32_off.data(), (N + 1) * sizeof(int64_t)));
        AWG_TRY(dalloc(h, P.G, (size_t)h->h_g32_off[N] * 4));
        k_conv_f32_padded<<<gblk, 256, 0, s>>>((int*)h->ns.p, (int64_t*)h->dense_off.p,
                                               (int64_t*)h->g32_off.p, (double*)G.p, (float*)P.G.p);
        AWG_LAUNCH();
    }
    // ---------------------------------------------- 5. W, 6. F
    nv_.next("awg_setup: W and F");
    const int nm = h->n_minus;
    if (nm > 0) {
        AWG_TRY(build_W(h));
        double t5 = now_ms();
        h->setup_ms[5] = t5 - t4;
        const double* W64 = (const double*)h->Wcm.p;
        PrecOps& P64 = h->prec[AWG_FP64];
        const bool inex = (h->opt.variant == AWG_H3_INEX) || (n <= 200000 && nm <= 4096);
        const unsigned gw = (unsigned)(((size_t)n * h->ldw + 255) / 256);
        if (h->opt.w_drop_tol > 0.0) {
            // the float64 form on the truncated W: F (and the H_3,inex
            // matrix) from the truncated copy, the apply from its CSR / CSC
            double* Wt = nullptr;
            AWG_TRY(build_truncated_W(h, W64, &Wt, P64));
            // (no H_3,inex matrix: Thm. 7's inner matrix C^-1 - Vhat^T W
            // needs W = A_+^-1 Vhat, which the truncated W no longer is)
            AWG_TRY(build_F(h, Wt, P64.Finv, &h->F64));
            AWG_CUDA(cudaFreeAsync(Wt, s));
        } else {
            AWG_TRY(build_F(h, W64, P64.Finv, &h->F64));
            if (inex) AWG_TRY(build_inex(h, W64, P64.inexInv));
            AWG_TRY(dalloc(h, P64.W, (size_t)n * h->ldw * 8));
            k_to_rowmajor<double><<<gw, 256, 0, s>>>(n, nm, h->ldw, W64, (double*)P64.W.p);
            AWG_LAUNCH();
        }
        for (int p = 1; p < AWG_NPREC; p++) {
            if (!(h->opt.precisions & (1 << p))) continue;
            PrecOps& P = h->prec[p];
            double* Wr = nullptr;
            AWG_CUDA(cudaMallocAsync(&Wr, (size_t)n * nm * 8, s));
            const size_t len = (size_t)n * nm;
            const unsigned gl = (unsigned)((len + 255) / 256);
            if (p == AWG_MIXED_FP16) {
                AWG_TRY(dalloc(h, P.rscale, (size_t)n * 4));
                AWG_TRY(dalloc(h, P.cscale, (size_t)h->ldw * 4));
                AWG_CUDA(cudaMemsetAsync(P.cscale.p, 0, (size_t)h->ldw * 4, s));
                DevBuf cmax;
                AWG_TRY(dalloc(h, cmax, (size_t)nm * 8));
                k_w16_cscale<<<nm, 256, 0, s>>>(n, W64, (float*)P.cscale.p, (double*)cmax.p);
                AWG_LAUNCH();
                k_w16_rscale<<<(n + 255) / 256, 256, 0, s>>>(n, nm, W64, (float*)P.cscale.p, (float*)P.rscale.p);
                AWG_LAUNCH();
                const double keep = h->opt.w16_keep;
                AWG_TRY(build_w16_correction(h, P, W64, (double*)cmax.p, keep));
                k_round_fp16<<<gl, 256, 0, s>>>(n, len, W64, (float*)P.rscale.p, (float*)P.cscale.p,
                                                (double*)cmax.p, keep, Wr);
                AWG_LAUNCH();
                AWG_CUDA(cudaStreamSynchronize(s));
                dfree(h, cmax);
            } else if (p == AWG_MIXED_FP32) {
                k_round_f32<<<gl, 256, 0, s>>>(len, W64, Wr);
            } else {
                k_round_bf16<<<gl, 256, 0, s>>>(len, W64, Wr);
            }
            AWG_LAUNCH();
            AWG_TRY(build_F(h, Wr, P.Finv, nullptr));
            if (inex) AWG_TRY(build_inex(h, Wr, P.inexInv));
            AWG_TRY(dalloc(h, P.W, (size_t)n * h->ldw * (p == AWG_MIXED_FP32 ? 4 : 2)));
            if (p == AWG_MIXED_FP32)
                k_to_rowmajor<float><<<gw, 256, 0, s>>>(n, nm, h->ldw, Wr, (float*)P.W.p);
            else if (p == AWG_MIXED_FP16)  // from the float64 W: the scaled values round once
                k_to_rowmajor_fp16<<<gw, 256, 0, s>>>(n, nm, h->ldw, W64, (float*)P.rscale.p,
                                                     (float*)P.cscale.p, (__half*)P.W.p);
            else
                k_to_rowmajor<__nv_bfloat16><<<gw, 256, 0, s>>>(n, nm, h->ldw, Wr, (__nv_bfloat16*)P.W.p);
            AWG_LAUNCH();
            AWG_CUDA(cudaFreeAsync(Wr, s));
        }
        AWG_CUDA(cudaStreamSynchronize(s));
        h->setup_ms[6] = now_ms() - t5;
    }
    for (int p = 1; p < AWG_NPREC; p++)
        if (h->opt.precisions & (1 << p)) h->prec[p].built = true;
    AWG_CUDA(cudaStreamSynchronize(s));
    if (h->opt.autotune) AWG_TRY(autotune_apply(h));
    return AWG_OK;
}

}  // namespace awg
