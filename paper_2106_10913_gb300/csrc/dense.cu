// Batched dense FP64 kernels over uneven per-subdomain blocks.
//
// Every block s is an m_s x m_s column-major matrix (ld = m_s) at offset
// off[s] of an arena.  One CTA works on one block for the factorisations; the
// GEMM kernel tiles every product of a batch over the whole GPU.
//
// On GB300 the FP64 FMA rate (about 0.6 TFMA/s) rather than HBM bounds these
// kernels, so they are written to keep the FP64 pipes fed (register-blocked
// GEMM, coalesced column sweeps) rather than to minimise bytes.

#include "awg_common.cuh"

#include <cmath>
#include <algorithm>

namespace awg {

// =============================================================== batched GEMM
// C = alpha op(A) op(B) + beta C for every descriptor of the batch.
constexpr int GBM = 64, GBN = 64, GBK = 16;

__global__ void __launch_bounds__(256) k_gemm(const GemmDesc* __restrict__ descs, int tilesM) {
    const GemmDesc d = descs[blockIdx.y];
    const int tm = blockIdx.x % tilesM, tn = blockIdx.x / tilesM;
    const int m0 = tm * GBM, n0 = tn * GBN;
    if (m0 >= d.M || n0 >= d.N) return;
    __shared__ double As[GBK][GBM + 1];
    __shared__ double Bs[GBK][GBN + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[r][c] = 0.0;
    for (int k0 = 0; k0 < d.K; k0 += GBK) {
        for (int e = threadIdx.x; e < GBM * GBK; e += 256) {
            int i, k;
            if (!d.transA) { i = e % GBM; k = e / GBM; } else { k = e % GBK; i = e / GBK; }
            const int gi = m0 + i, gk = k0 + k;
            double v = 0.0;
            if (gi < d.M && gk < d.K)
                v = d.transA ? d.A[gk + (size_t)gi * d.lda] : d.A[gi + (size_t)gk * d.lda];
            As[k][i] = v;
        }
        for (int e = threadIdx.x; e < GBN * GBK; e += 256) {
            int j, k;
            if (!d.transB) { k = e % GBK; j = e / GBK; } else { j = e % GBN; k = e / GBN; }
            const int gj = n0 + j, gk = k0 + k;
            double v = 0.0;
            if (gj < d.N && gk < d.K)
                v = d.transB ? d.B[gj + (size_t)gk * d.ldb] : d.B[gk + (size_t)gj * d.ldb];
            Bs[k][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GBK; k++) {
            double a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; r++) a[r] = As[k][tx + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; c++) b[c] = Bs[k][ty + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[r][c] = fma(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const int gj = n0 + ty + 16 * c;
        if (gj >= d.N) continue;
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int gi = m0 + tx + 16 * r;
            if (gi >= d.M) continue;
            double* cp = d.C + gi + (size_t)gj * d.ldc;
            const double v = d.alpha * acc[r][c];
            *cp = (d.beta == 0.0) ? v : fma(d.beta, *cp, v);
        }
    }
}

awg_status gemm_batched(Handle* h, const std::vector<GemmDesc>& descs, cudaStream_t s) {
    if (descs.empty()) return AWG_OK;
    int maxM = 0, maxN = 0;
    for (auto& d : descs) { maxM = std::max(maxM, d.M); maxN = std::max(maxN, d.N); }
    if (maxM == 0 || maxN == 0) return AWG_OK;
    const int tilesM = (maxM + GBM - 1) / GBM, tilesN = (maxN + GBN - 1) / GBN;
    // descriptors travel through a temporary device buffer (a copy from
    // pageable memory returns once the host data is staged), in chunks that
    // respect the grid's y limit
    const size_t chunk = 65535;
    for (size_t b0 = 0; b0 < descs.size(); b0 += chunk) {
        const size_t nb = std::min(chunk, descs.size() - b0);
        GemmDesc* d_desc = nullptr;
        AWG_CUDA(cudaMallocAsync(&d_desc, nb * sizeof(GemmDesc), s));
        AWG_CUDA(cudaMemcpyAsync(d_desc, descs.data() + b0, nb * sizeof(GemmDesc),
                                 cudaMemcpyHostToDevice, s));
        dim3 grid((unsigned)(tilesM * tilesN), (unsigned)nb);
        k_gemm<<<grid, 256, 0, s>>>(d_desc, tilesM);
        AWG_LAUNCH();
        AWG_CUDA(cudaFreeAsync(d_desc, s));
    }
    (void)h;
    return AWG_OK;
}

// ------------------------------------------- batched GEMM, FP32 operands
// C (float64) = alpha op(A) B + beta C with A float32, B float64 rounded to
// float32 on load, float32 products and accumulation (the reduced-precision
// local operators inside the multi-RHS solves).
__global__ void __launch_bounds__(256) k_gemm_f32(const GemmDescF* __restrict__ descs, int tilesM) {
    const GemmDescF d = descs[blockIdx.y];
    const int tm = blockIdx.x % tilesM, tn = blockIdx.x / tilesM;
    const int m0 = tm * GBM, n0 = tn * GBN;
    if (m0 >= d.M || n0 >= d.N) return;
    __shared__ float As[GBK][GBM + 4];
    __shared__ float Bs[GBK][GBN + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[r][c] = 0.f;
    for (int k0 = 0; k0 < d.K; k0 += GBK) {
        for (int e = threadIdx.x; e < GBM * GBK; e += 256) {
            int i, k;
            if (!d.transA) { i = e % GBM; k = e / GBM; } else { k = e % GBK; i = e / GBK; }
            const int gi = m0 + i, gk = k0 + k;
            float v = 0.f;
            if (gi < d.M && gk < d.K)
                v = d.transA ? d.A[gk + (size_t)gi * d.lda] : d.A[gi + (size_t)gk * d.lda];
            As[k][i] = v;
        }
        for (int e = threadIdx.x; e < GBN * GBK; e += 256) {
            const int k = e % GBK, j = e / GBK;
            const int gj = n0 + j, gk = k0 + k;
            Bs[k][j] = (gj < d.N && gk < d.K) ? (float)d.B[gk + (size_t)gj * d.ldb] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GBK; k++) {
            float a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; r++) a[r] = As[k][tx + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; c++) b[c] = Bs[k][ty + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; r++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const int gj = n0 + ty + 16 * c;
        if (gj >= d.N) continue;
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int gi = m0 + tx + 16 * r;
            if (gi >= d.M) continue;
            double* cp = d.C + gi + (size_t)gj * d.ldc;
            const double v = d.alpha * (double)acc[r][c];
            *cp = (d.beta == 0.0) ? v : fma(d.beta, *cp, v);
        }
    }
}

awg_status gemm_batched_f32(Handle* h, const std::vector<GemmDescF>& descs, cudaStream_t s) {
    if (descs.empty()) return AWG_OK;
    int maxM = 0, maxN = 0;
    for (auto& d : descs) { maxM = std::max(maxM, d.M); maxN = std::max(maxN, d.N); }
    if (maxM == 0 || maxN == 0) return AWG_OK;
    const int tilesM = (maxM + GBM - 1) / GBM, tilesN = (maxN + GBN - 1) / GBN;
    const size_t chunk = 65535;
    for (size_t b0 = 0; b0 < descs.size(); b0 += chunk) {
        const size_t nb = std::min(chunk, descs.size() - b0);
        GemmDescF* d_desc = nullptr;
        AWG_CUDA(cudaMallocAsync(&d_desc, nb * sizeof(GemmDescF), s));
        AWG_CUDA(cudaMemcpyAsync(d_desc, descs.data() + b0, nb * sizeof(GemmDescF),
                                 cudaMemcpyHostToDevice, s));
        dim3 grid((unsigned)(tilesM * tilesN), (unsigned)nb);
        k_gemm_f32<<<grid, 256, 0, s>>>(d_desc, tilesM);
        AWG_LAUNCH();
        AWG_CUDA(cudaFreeAsync(d_desc, s));
    }
    (void)h;
    return AWG_OK;
}

// ========================================================= batched Cholesky
// Lower Cholesky factor in place (right-looking).  A pivot that is not
// positive (or not finite) raises FLAG_NOT_SPD and stops that block.
__global__ void __launch_bounds__(512) k_potrf(double* arena, const int* __restrict__ ms,
                                               const int64_t* __restrict__ offs, int* flag,
                                               int* status) {
    extern __shared__ double col[];
    __shared__ int bad;
    const int s = blockIdx.x;
    const int m = ms[s];
    double* A = arena + offs[s];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < m; j++) {
        if (threadIdx.x == 0) {
            const double a = A[j + (size_t)j * m];
            if (!(a > 0.0) || !isfinite(a)) {
                bad = 1;
            } else {
                A[j + (size_t)j * m] = sqrt(a);
            }
        }
        __syncthreads();
        if (bad) break;
        const double inv = 1.0 / A[j + (size_t)j * m];
        for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) {
            const double v = A[i + (size_t)j * m] * inv;
            A[i + (size_t)j * m] = v;
            col[i] = v;
        }
        __syncthreads();
        for (int c = j + 1 + wid; c < m; c += nw) {
            const double lc = col[c];
            double* Ac = A + (size_t)c * m;
            for (int i = c + lane; i < m; i += 32) Ac[i] = fma(-col[i], lc, Ac[i]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && bad && flag) atomicOr(flag, FLAG_NOT_SPD);
    if (threadIdx.x == 0 && status) status[s] = bad;
    // zero the strict upper triangle so that the block is a plain lower matrix
    if (!bad) {
        for (int c = 1 + wid; c < m; c += nw) {
            double* Ac = A + (size_t)c * m;
            for (int i = lane; i < c; i += 32) Ac[i] = 0.0;
        }
    }
}

awg_status potrf_batched(Handle* h, double* arena, const int* d_m, const int64_t* d_off, int nb,
                         int max_m, int* d_flag, cudaStream_t s, int* d_status) {
    if (nb == 0) return AWG_OK;
    const size_t smem = (size_t)max_m * sizeof(double);
    if (smem > 48 * 1024)
        AWG_CUDA(cudaFuncSetAttribute(k_potrf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    k_potrf<<<nb, 512, smem, s>>>(arena, d_m, d_off, d_flag, d_status);
    AWG_LAUNCH();
    (void)h;
    return AWG_OK;
}

// ================================================= batched triangular inverse
// In-place inverse of a lower triangular block (columns from last to first):
// column j of L^-1 is -L^-1_jj * T x with T the already inverted trailing
// block and x the original column below the diagonal.
__global__ void __launch_bounds__(512) k_trtri(double* arena, const int* __restrict__ ms,
                                               const int64_t* __restrict__ offs) {
    extern __shared__ double x[];
    const int s = blockIdx.x;
    const int m = ms[s];
    double* A = arena + offs[s];
    for (int j = m - 1; j >= 0; j--) {
        const double ajj = 1.0 / A[j + (size_t)j * m];
        for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) x[i] = A[i + (size_t)j * m];
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) {
            double acc = 0.0;
            for (int k = j + 1; k <= i; k++) acc = fma(A[i + (size_t)k * m], x[k], acc);
            A[i + (size_t)j * m] = -ajj * acc;
        }
        if (threadIdx.x == 0) A[j + (size_t)j * m] = ajj;
        __syncthreads();
    }
}

awg_status trtri_batched(Handle* h, double* arena, const int* d_m, const int64_t* d_off, int nb,
                         int max_m, cudaStream_t s) {
    if (nb == 0) return AWG_OK;
    const size_t smem = (size_t)max_m * sizeof(double);
    if (smem > 48 * 1024)
        AWG_CUDA(cudaFuncSetAttribute(k_trtri, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    k_trtri<<<nb, 512, smem, s>>>(arena, d_m, d_off);
    AWG_LAUNCH();
    (void)h;
    return AWG_OK;
}

// ===================================================== tridiagonalisation
// Householder reduction A = Q T Q^T of a full symmetric block (both triangles
// kept up to date), LAPACK convention H_k = I - tau_k v_k v_k^T with
// v_k(0) = 1.  v_k(1:) overwrites A(k+2:, k); diag/offdiag/tau go to the
// per-row arrays at ptr[s].
__global__ void __launch_bounds__(1024) k_tridiag(double* arena, const int* __restrict__ ms,
                                                  const int64_t* __restrict__ offs,
                                                  const int* __restrict__ ptr, double* dg,
                                                  double* eo, double* tv) {
    extern __shared__ double sh[];
    __shared__ double red[32];
    __shared__ double sc[4];
    const int s = blockIdx.x;
    const int m = ms[s];
    double* A = arena + offs[s];
    double* dd = dg + ptr[s];
    double* ee = eo + ptr[s];
    double* tt = tv + ptr[s];
    double* v = sh;          // length m
    double* w = sh + m;      // length m
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k + 2 < m; k++) {
        const int len = m - k - 1;
        double* xk = A + (k + 1) + (size_t)k * m;  // x = A(k+1:, k), length len
        double part = 0.0;
        for (int i = 1 + threadIdx.x; i < len; i += blockDim.x) part = fma(xk[i], xk[i], part);
        const double sig = block_sum(part, red);
        if (threadIdx.x == 0) {
            const double alpha = xk[0];
            double beta, tau, scal;
            if (sig == 0.0) {
                beta = alpha; tau = 0.0; scal = 0.0;
            } else {
                const double mu = sqrt(alpha * alpha + sig);
                beta = (alpha <= 0.0) ? mu : -mu;
                tau = (beta - alpha) / beta;
                scal = 1.0 / (alpha - beta);
            }
            sc[0] = tau; sc[1] = scal;
            dd[k] = A[k + (size_t)k * m];
            ee[k] = beta;
            tt[k] = tau;
        }
        __syncthreads();
        const double tau = sc[0], scal = sc[1];
        if (tau == 0.0) {
            __syncthreads();
            continue;
        }
        for (int i = threadIdx.x; i < len; i += blockDim.x) {
            const double vi = (i == 0) ? 1.0 : xk[i] * scal;
            v[i] = vi;
            if (i > 0) xk[i] = vi;  // store v(1:) below the subdiagonal
        }
        __syncthreads();
        // w = tau * A22 v  (A22 = A(k+1:, k+1:))
        double* A22 = A + (k + 1) + (size_t)(k + 1) * m;
        for (int i = threadIdx.x; i < len; i += blockDim.x) {
            double acc0 = 0.0, acc1 = 0.0;
            int j = 0;
            for (; j + 1 < len; j += 2) {
                acc0 = fma(A22[i + (size_t)j * m], v[j], acc0);
                acc1 = fma(A22[i + (size_t)(j + 1) * m], v[j + 1], acc1);
            }
            if (j < len) acc0 = fma(A22[i + (size_t)j * m], v[j], acc0);
            w[i] = tau * (acc0 + acc1);
        }
        __syncthreads();
        double pv = 0.0;
        for (int i = threadIdx.x; i < len; i += blockDim.x) pv = fma(w[i], v[i], pv);
        const double K = -0.5 * tau * block_sum(pv, red);
        for (int i = threadIdx.x; i < len; i += blockDim.x) w[i] = fma(K, v[i], w[i]);
        __syncthreads();
        // A22 -= v w^T + w v^T
        for (int j = wid; j < len; j += nw) {
            const double vj = v[j], wj = w[j];
            double* col = A22 + (size_t)j * m;
            for (int i = lane; i < len; i += 32) col[i] -= fma(v[i], wj, w[i] * vj);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (m >= 2) {
            dd[m - 2] = A[(m - 2) + (size_t)(m - 2) * m];
            ee[m - 2] = A[(m - 1) + (size_t)(m - 2) * m];
            tt[m - 2] = 0.0;
        }
        dd[m - 1] = A[(m - 1) + (size_t)(m - 1) * m];
        ee[m - 1] = 0.0;
        tt[m - 1] = 0.0;
    }
}

// Number of eigenvalues of the tridiagonal (d, e) strictly below x
// (negative pivots of the LDL^T of T - xI, pivots smaller than pivmin in
// magnitude replaced by -pivmin).
__device__ int sturm_count(const double* d, const double* e2, int m, double x, double pivmin) {
    int cnt = 0;
    double q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) cnt++;
    for (int i = 1; i < m; i++) {
        q = (d[i] - x) - e2[i - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        if (q < 0.0) cnt++;
    }
    return cnt;
}

// j-th smallest eigenvalue (0-based) by bisection on [lo, hi].
__device__ double bisect_index(const double* d, const double* e2, int m, int j, double lo, double hi,
                               double pivmin) {
    const double eps = 2.220446049250313e-16;
    for (int it = 0; it < 200; it++) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (hi - lo <= 2.0 * eps * fmax(fabs(lo), fabs(hi)) + 2.0 * pivmin) break;
        if (sturm_count(d, e2, m, mid, pivmin) > j) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Per block: Gershgorin interval, pivmin, thresholds and eigenvalue counts.
// mode 0: thr = param * max|lambda|; count = #(lambda <= thr), strict = #(lambda < -thr)
// mode 1: count = strict = #(lambda < param)
__global__ void k_eig_count(const int* __restrict__ ms, const int* __restrict__ ptr,
                            const double* __restrict__ dg, const double* __restrict__ eo,
                            double* e2o, double* info, int* cnt, int* strict, int mode,
                            double param) {
    __shared__ double wl[32], wu[32], we[32];
    __shared__ double ext[2];
    const int s = blockIdx.x;
    const int m = ms[s];
    const double* d = dg + ptr[s];
    const double* e = eo + ptr[s];
    double* e2 = e2o + ptr[s];
    double l = INFINITY, u = -INFINITY, em2 = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double ei = (i + 1 < m) ? fabs(e[i]) : 0.0;
        const double emm = (i > 0) ? fabs(e[i - 1]) : 0.0;
        l = fmin(l, d[i] - ei - emm);
        u = fmax(u, d[i] + ei + emm);
        if (i + 1 < m) {
            e2[i] = e[i] * e[i];
            em2 = fmax(em2, e2[i]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        l = fmin(l, __shfl_xor_sync(0xffffffffu, l, o));
        u = fmax(u, __shfl_xor_sync(0xffffffffu, u, o));
        em2 = fmax(em2, __shfl_xor_sync(0xffffffffu, em2, o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { wl[wid] = l; wu[wid] = u; we[wid] = em2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int k = 1; k < nw; k++) { l = fmin(l, wl[k]); u = fmax(u, wu[k]); em2 = fmax(em2, we[k]); }
        const double span = fmax(fabs(l), fabs(u));
        l -= 8.0 * 2.220446049250313e-16 * span + 1e-300;
        u += 8.0 * 2.220446049250313e-16 * span + 1e-300;
        info[4 * s + 0] = l;
        info[4 * s + 1] = u;
        info[4 * s + 2] = 2.2250738585072014e-308 * fmax(1.0, em2);
    }
    __syncthreads();
    const double lo = info[4 * s + 0], hi = info[4 * s + 1], pivmin = info[4 * s + 2];
    if (mode == 0) {
        if (threadIdx.x < 2) {
            const int j = (threadIdx.x == 0) ? 0 : m - 1;
            ext[threadIdx.x] = bisect_index(d, e2, m, j, lo, hi, pivmin);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const double thr = param * fmax(fabs(ext[0]), fabs(ext[1]));
            info[4 * s + 3] = thr;
            // #(lambda <= thr) = #(lambda < next double above thr)
            // thr >= 0: adding one to the bit pattern gives the next double above it
            cnt[s] = sturm_count(d, e2, m, __longlong_as_double(__double_as_longlong(thr) + 1), pivmin);
            strict[s] = sturm_count(d, e2, m, -thr, pivmin);
        }
    } else if (threadIdx.x == 0) {
        info[4 * s + 3] = param;
        const int c = sturm_count(d, e2, m, param, pivmin);
        cnt[s] = c;
        strict[s] = c;
    }
}

// Eigenvalues 0..cnt-1 of each block by bisection (one thread per value).
__global__ void k_bisect(const int* __restrict__ ms, const int* __restrict__ ptr,
                         const double* __restrict__ dg, const double* __restrict__ e2o,
                         const double* __restrict__ info, const int* __restrict__ cnt,
                         const int* __restrict__ vptr, double* vals) {
    const int s = blockIdx.x;
    const int m = ms[s];
    const double* d = dg + ptr[s];
    const double* e2 = e2o + ptr[s];
    for (int j = threadIdx.x; j < cnt[s]; j += blockDim.x)
        vals[vptr[s] + j] = bisect_index(d, e2, m, j, info[4 * s], info[4 * s + 1], info[4 * s + 2]);
}

// Inverse iteration for the selected eigenvalues of each tridiagonal, with
// modified Gram-Schmidt inside clusters (eigenvalues closer than 1e-3 ||T||),
// following the structure of LAPACK's dstein: LU of T - lambda I with
// partial pivoting, solves with tiny pivots perturbed, four iterations.
__global__ void __launch_bounds__(256) k_inviter(const int* __restrict__ ms,
                                                 const int* __restrict__ ptr,
                                                 const double* __restrict__ dg,
                                                 const double* __restrict__ eo,
                                                 const int* __restrict__ cnt,
                                                 const int* __restrict__ vptr,
                                                 const double* __restrict__ vals,
                                                 const int64_t* __restrict__ voff, double* vecs,
                                                 int* flag) {
    extern __shared__ double sh[];
    __shared__ double red[32];
    __shared__ double scal[2];
    const int s = blockIdx.x;
    const int m = ms[s];
    const int c = cnt[s];
    if (c == 0) return;
    const double* d = dg + ptr[s];
    const double* e = eo + ptr[s];
    const double* lam = vals + vptr[s];
    double* X = vecs + voff[s];
    double* a = sh;            // U diagonal
    double* b = sh + m;        // U first superdiagonal
    double* u2 = sh + 2 * m;   // U second superdiagonal
    double* l = sh + 3 * m;    // multipliers
    double* y = sh + 4 * m;    // iterate
    int* piv = reinterpret_cast<int*>(sh + 5 * m);
    // ||T||_1
    double nrm = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double r = fabs(d[i]);
        if (i + 1 < m) r += fabs(e[i]);
        if (i > 0) r += fabs(e[i - 1]);
        nrm = fmax(nrm, r);
    }
    for (int o = 16; o > 0; o >>= 1) nrm = fmax(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t = fmax(t, red[k]);
        scal[0] = t;
    }
    __syncthreads();
    const double onenrm = fmax(scal[0], 1e-300);
    const double eps = 2.220446049250313e-16;
    const double ortol = 1e-3 * onenrm;
    int jblk = 0;  // first index of the current cluster
    double xjm = 0.0;
    for (int j = 0; j < c; j++) {
        double xj = lam[j];
        if (j > 0) {
            if (xj - xjm > ortol) jblk = j;
            else {
                const double pertol = 10.0 * fabs(eps * xj);
                if (xj - xjm < pertol) xj = xjm + pertol;
            }
        }
        xjm = xj;
        // LU with partial pivoting of T - xj I (thread 0, sequential)
        if (threadIdx.x == 0) {
            for (int i = 0; i < m; i++) {
                a[i] = d[i] - xj;
                b[i] = (i + 1 < m) ? e[i] : 0.0;
                l[i] = (i + 1 < m) ? e[i] : 0.0;  // subdiagonal, becomes multipliers
                u2[i] = 0.0;
                piv[i] = 0;
            }
            const double tol = fmax(fabs(xj), onenrm) * eps;
            for (int k = 0; k + 1 < m; k++) {
                const double ck = l[k];
                if (fabs(a[k]) >= fabs(ck)) {
                    if (a[k] == 0.0) a[k] = tol;
                    const double mult = ck / a[k];
                    l[k] = mult;
                    a[k + 1] -= mult * b[k];
                    piv[k] = 0;
                } else {
                    const double mult = a[k] / ck;
                    a[k] = ck;
                    const double temp = a[k + 1];
                    a[k + 1] = b[k] - mult * temp;
                    if (k + 2 < m) {
                        u2[k] = b[k + 1];
                        b[k + 1] = -mult * u2[k];
                    }
                    b[k] = temp;
                    l[k] = mult;
                    piv[k] = 1;
                }
            }
            scal[1] = tol;
        }
        // deterministic pseudo-random start vector
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            uint32_t hsh = (uint32_t)(i * 2654435761u) ^ (uint32_t)((j + 1) * 40503u) ^ 0x9e3779b9u;
            hsh ^= hsh >> 13; hsh *= 0x5bd1e995u; hsh ^= hsh >> 15;
            y[i] = ((double)(hsh & 0xffffff) / 16777216.0) * 2.0 - 1.0;
        }
        __syncthreads();
        const double tol = scal[1];
        for (int it = 0; it < 4; it++) {
            if (threadIdx.x == 0) {
                // apply L^-1 (with the row interchanges), then U^-1
                for (int k = 0; k + 1 < m; k++) {
                    if (piv[k] == 0) {
                        y[k + 1] -= l[k] * y[k];
                    } else {
                        const double t = y[k];
                        y[k] = y[k + 1];
                        y[k + 1] = t - l[k] * y[k];
                    }
                }
                auto pv = [&](double x) { return (fabs(x) < tol) ? (x < 0.0 ? -tol : tol) : x; };
                y[m - 1] = y[m - 1] / pv(a[m - 1]);
                if (m >= 2) y[m - 2] = (y[m - 2] - b[m - 2] * y[m - 1]) / pv(a[m - 2]);
                for (int k = m - 3; k >= 0; k--)
                    y[k] = (y[k] - b[k] * y[k + 1] - u2[k] * y[k + 2]) / pv(a[k]);
                // rescale to avoid overflow in later iterations
                double mx = 0.0;
                for (int k = 0; k < m; k++) mx = fmax(mx, fabs(y[k]));
                scal[0] = (mx > 0.0 && isfinite(mx)) ? 1.0 / mx : 0.0;
            }
            __syncthreads();
            const double sc = scal[0];
            for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] *= sc;
            __syncthreads();
            // orthogonalise against the earlier vectors of the cluster
            for (int q = jblk; q < j; q++) {
                const double* xq = X + (size_t)q * m;
                double part = 0.0;
                for (int i = threadIdx.x; i < m; i += blockDim.x) part = fma(xq[i], y[i], part);
                const double dotv = block_sum(part, red);
                for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] = fma(-dotv, xq[i], y[i]);
                __syncthreads();
            }
            double part = 0.0;
            for (int i = threadIdx.x; i < m; i += blockDim.x) part = fma(y[i], y[i], part);
            const double nn = block_sum(part, red);
            const double inv = (nn > 0.0 && isfinite(nn)) ? 1.0 / sqrt(nn) : 0.0;
            if (inv == 0.0 && threadIdx.x == 0) atomicOr(flag, FLAG_EIG);
            for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] *= inv;
            __syncthreads();
        }
        // fix the sign (largest component positive) and store
        if (threadIdx.x == 0) {
            int im = 0;
            double mx = -1.0;
            for (int k = 0; k < m; k++) if (fabs(y[k]) > mx) { mx = fabs(y[k]); im = k; }
            scal[0] = (y[im] < 0.0) ? -1.0 : 1.0;
        }
        __syncthreads();
        const double sg = scal[0];
        double* xj_out = X + (size_t)j * m;
        for (int i = threadIdx.x; i < m; i += blockDim.x) xj_out[i] = sg * y[i];
        __syncthreads();
    }
}

// Back-transformation X <- Q X with Q = H_0 ... H_{m-3}; one warp per vector.
__global__ void __launch_bounds__(256) k_backtransform(const double* __restrict__ arena,
                                                       const int* __restrict__ ms,
                                                       const int64_t* __restrict__ offs,
                                                       const int* __restrict__ ptr,
                                                       const double* __restrict__ tv,
                                                       const int* __restrict__ cnt,
                                                       const int64_t* __restrict__ voff,
                                                       double* vecs) {
    const int s = blockIdx.x;
    const int m = ms[s];
    const int c = cnt[s];
    const double* A = arena + offs[s];
    const double* tt = tv + ptr[s];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = wid; q < c; q += nw) {
        double* y = vecs + voff[s] + (size_t)q * m;
        for (int k = m - 3; k >= 0; k--) {
            const double tau = tt[k];
            if (tau == 0.0) continue;
            const double* vk = A + (size_t)k * m;  // v(0) = 1 at row k+1, v(i) at row k+1+i
            double part = 0.0;
            for (int i = k + 1 + lane; i < m; i += 32) {
                const double vi = (i == k + 1) ? 1.0 : vk[i];
                part = fma(vi, y[i], part);
            }
            const double dotv = warp_sum(part) * tau;
            for (int i = k + 1 + lane; i < m; i += 32) {
                const double vi = (i == k + 1) ? 1.0 : vk[i];
                y[i] = fma(-dotv, vi, y[i]);
            }
            __syncwarp();
        }
    }
}

awg_status eig_select_batched(Handle* h, double* arena, const int* d_m, const int64_t* d_off,
                              const std::vector<int>& h_m, int nb, int max_m, int mode,
                              double param, std::vector<int>& h_count,
                              std::vector<int>& h_strict, DevBuf& vecs,
                              std::vector<int64_t>& h_vec_off, DevBuf& vals,
                              std::vector<int>& h_val_ptr, cudaStream_t s) {
    // per-row arrays (prefix of m)
    std::vector<int> h_ptr(nb + 1, 0);
    for (int b = 0; b < nb; b++) h_ptr[b + 1] = h_ptr[b] + h_m[b];
    const int tot = h_ptr[nb];
    DevBuf dptr, dg, eo, e2, tv, info, dcnt, dstrict;
    AWG_TRY(dalloc(h, dptr, (nb + 1) * sizeof(int)));
    AWG_TRY(dalloc(h, dg, (size_t)tot * 8));
    AWG_TRY(dalloc(h, eo, (size_t)tot * 8));
    AWG_TRY(dalloc(h, e2, (size_t)tot * 8));
    AWG_TRY(dalloc(h, tv, (size_t)tot * 8));
    AWG_TRY(dalloc(h, info, (size_t)nb * 4 * 8));
    AWG_TRY(dalloc(h, dcnt, nb * sizeof(int)));
    AWG_TRY(dalloc(h, dstrict, nb * sizeof(int)));
    AWG_CUDA(cudaMemcpyAsync(dptr.p, h_ptr.data(), (nb + 1) * sizeof(int), cudaMemcpyHostToDevice, s));

    size_t smem = (size_t)2 * max_m * sizeof(double);
    AWG_CUDA(cudaFuncSetAttribute(k_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 1)));
    k_tridiag<<<nb, 1024, smem, s>>>(arena, d_m, d_off, (int*)dptr.p, (double*)dg.p, (double*)eo.p,
                                     (double*)tv.p);
    AWG_LAUNCH();
    k_eig_count<<<nb, 256, 0, s>>>(d_m, (int*)dptr.p, (double*)dg.p, (double*)eo.p, (double*)e2.p,
                                   (double*)info.p, (int*)dcnt.p, (int*)dstrict.p, mode, param);
    AWG_LAUNCH();
    h_count.assign(nb, 0);
    h_strict.assign(nb, 0);
    AWG_CUDA(cudaMemcpyAsync(h_count.data(), dcnt.p, nb * sizeof(int), cudaMemcpyDeviceToHost, s));
    AWG_CUDA(cudaMemcpyAsync(h_strict.data(), dstrict.p, nb * sizeof(int), cudaMemcpyDeviceToHost, s));
    AWG_CUDA(cudaStreamSynchronize(s));
    h_val_ptr.assign(nb + 1, 0);
    h_vec_off.assign(nb + 1, 0);
    for (int b = 0; b < nb; b++) {
        h_val_ptr[b + 1] = h_val_ptr[b] + h_count[b];
        h_vec_off[b + 1] = h_vec_off[b] + (int64_t)h_count[b] * h_m[b];
    }
    DevBuf dvptr, dvoff;
    AWG_TRY(dalloc(h, dvptr, (nb + 1) * sizeof(int)));
    AWG_TRY(dalloc(h, dvoff, (nb + 1) * sizeof(int64_t)));
    AWG_CUDA(cudaMemcpyAsync(dvptr.p, h_val_ptr.data(), (nb + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
    AWG_CUDA(cudaMemcpyAsync(dvoff.p, h_vec_off.data(), (nb + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    AWG_TRY(dalloc(h, vals, std::max<size_t>(8, (size_t)h_val_ptr[nb] * 8)));
    AWG_TRY(dalloc(h, vecs, std::max<size_t>(8, (size_t)h_vec_off[nb] * 8)));
    if (h_val_ptr[nb] > 0) {
        k_bisect<<<nb, 128, 0, s>>>(d_m, (int*)dptr.p, (double*)dg.p, (double*)e2.p, (double*)info.p,
                                    (int*)dcnt.p, (int*)dvptr.p, (double*)vals.p);
        AWG_LAUNCH();
        size_t smi = (size_t)6 * max_m * sizeof(double);
        AWG_CUDA(cudaFuncSetAttribute(k_inviter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smi));
        k_inviter<<<nb, 256, smi, s>>>(d_m, (int*)dptr.p, (double*)dg.p, (double*)eo.p, (int*)dcnt.p,
                                       (int*)dvptr.p, (double*)vals.p, (int64_t*)dvoff.p,
                                       (double*)vecs.p, (int*)h->flag.p);
        AWG_LAUNCH();
        k_backtransform<<<nb, 256, 0, s>>>(arena, d_m, d_off, (int*)dptr.p, (double*)tv.p,
                                           (int*)dcnt.p, (int64_t*)dvoff.p, (double*)vecs.p);
        AWG_LAUNCH();
    }
    AWG_CUDA(cudaStreamSynchronize(s));
    for (DevBuf* b : {&dptr, &dg, &eo, &e2, &tv, &info, &dcnt, &dstrict, &dvptr, &dvoff}) dfree(h, *b);
    return AWG_OK;
}

}  // namespace awg
