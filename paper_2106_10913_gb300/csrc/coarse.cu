// Dense float64 factorisation of the coarse matrices E = Z^T A_+ Z (Thm. 4)
// and F = W^T A W (Def. 10): a blocked right-looking Cholesky spread over
// the whole GPU, the inverse of the triangular factor by block columns, and
// M^-1 = L^-T L^-1 through the symmetric A^T B kernel of setup.cu.
//
// Matrices are column-major dim x dim (ld = dim), 64 x 64 blocks.  Per block
// column j: k_chol_diag factors the diagonal block in one CTA, k_chol_trsm
// solves the panel below it (one thread per row), k_chol_update subtracts
// L_ij L_kj^T from every trailing block on or below the diagonal (one CTA
// per block, 4 x 4 per thread).  A non-positive pivot raises FLAG_NOT_SPD.

#include "awg_common.cuh"

#include <algorithm>

namespace awg {

namespace {

constexpr int CB = 64;

__global__ void __launch_bounds__(256) k_chol_diag(double* A, int ld, int j0, int bs, int* flag) {
    __shared__ double a[CB][CB + 1];
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
        const int r = e % bs, c = e / bs;
        a[r][c] = A[(size_t)(j0 + c) * ld + j0 + r];
    }
    __syncthreads();
    for (int k = 0; k < bs; k++) {
        if (threadIdx.x == 0) {
            double d = a[k][k];
            if (!(d > 0.0) || !isfinite(d)) {
                atomicOr(flag, FLAG_NOT_SPD);
                d = 1.0;
            }
            a[k][k] = sqrt(d);
        }
        __syncthreads();
        const double dk = a[k][k];
        for (int r = k + 1 + threadIdx.x; r < bs; r += blockDim.x) a[r][k] /= dk;
        __syncthreads();
        const int m = bs - k - 1;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int r = k + 1 + e % m, c = k + 1 + e / m;
            if (r >= c) a[r][c] -= a[r][k] * a[c][k];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
        const int r = e % bs, c = e / bs;
        A[(size_t)(j0 + c) * ld + j0 + r] = (r >= c) ? a[r][c] : 0.0;
    }
}

// rows r >= j0 + bs: A(r, j0 .. j0+bs) <- A(r, .) L_jj^-T (forward substitution per row)
__global__ void __launch_bounds__(128) k_chol_trsm(double* A, int ld, int dim, int j0, int bs) {
    __shared__ double l[CB][CB + 1];
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
        const int r = e % bs, c = e / bs;
        l[r][c] = A[(size_t)(j0 + c) * ld + j0 + r];
    }
    __syncthreads();
    const int r = j0 + bs + blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= dim) return;
    double x[CB];
#pragma unroll
    for (int c = 0; c < CB; c++) {
        if (c < bs) {
            double v = A[(size_t)(j0 + c) * ld + r];
#pragma unroll
            for (int k = 0; k < CB; k++)
                if (k < c) v -= x[k] * l[c][k];
            x[c] = v / l[c][c];
        }
    }
#pragma unroll
    for (int c = 0; c < CB; c++)
        if (c < bs) A[(size_t)(j0 + c) * ld + r] = x[c];
}

// blocks (bi, bk), j < bk <= bi, of the trailing matrix: A_ik -= L_ij L_kj^T
constexpr int CU_KC = 16;
__global__ void __launch_bounds__(256) k_chol_update(double* A, int ld, int dim, int jb) {
    __shared__ double li[CU_KC][CB + 1];
    __shared__ double lk[CU_KC][CB + 1];
    __shared__ int bik[2];
    const int nb = (dim + CB - 1) / CB;
    const int m = nb - jb - 1;  // trailing block rows
    if (threadIdx.x == 0) {     // blockIdx.x -> (bi, bk), bk <= bi, column by column
        int t = blockIdx.x, c = 0;
        while (t >= m - c) { t -= m - c; c++; }
        bik[0] = jb + 1 + c + t;
        bik[1] = jb + 1 + c;
    }
    __syncthreads();
    const int i0 = bik[0] * CB, k0 = bik[1] * CB, j0 = jb * CB;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int q0 = 0; q0 < CB; q0 += CU_KC) {
        __syncthreads();
        for (int e = threadIdx.x; e < CU_KC * CB; e += 256) {
            const int r = e % CB, q = e / CB;
            li[q][r] = (i0 + r < dim) ? A[(size_t)(j0 + q0 + q) * ld + i0 + r] : 0.0;
            lk[q][r] = (k0 + r < dim) ? A[(size_t)(j0 + q0 + q) * ld + k0 + r] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < CU_KC; q++) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; u++) { a[u] = li[q][ty * 4 + u]; b[u] = lk[q][tx * 4 + u]; }
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int v = 0; v < 4; v++) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
    }
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
        for (int v = 0; v < 4; v++) {
            const int r = i0 + ty * 4 + u, c = k0 + tx * 4 + v;
            if (r < dim && c < dim) A[(size_t)c * ld + r] -= acc[u][v];
        }
}

// inverses of the lower-triangular diagonal blocks of L into Li (one CTA per
// block, one thread per column: forward substitution on e_c)
__global__ void __launch_bounds__(64) k_trtri_diag(const double* L, double* Li, int ld, int dim) {
    __shared__ double l[CB][CB + 1];
    const int j0 = blockIdx.x * CB, bs = min(CB, dim - j0);
    for (int e = threadIdx.x; e < bs * bs; e += blockDim.x) {
        const int r = e % bs, c = e / bs;
        l[r][c] = L[(size_t)(j0 + c) * ld + j0 + r];
    }
    __syncthreads();
    const int c = threadIdx.x;
    if (c >= bs) return;
    double x[CB];
#pragma unroll
    for (int r = 0; r < CB; r++) {
        if (r < bs) {
            double v = (r == c) ? 1.0 : 0.0;
#pragma unroll
            for (int k = 0; k < CB; k++)
                if (k < r && k >= c) v -= l[r][k] * x[k];
            x[r] = (r < c) ? 0.0 : v / l[r][r];
        }
    }
#pragma unroll
    for (int r = 0; r < CB; r++)
        if (r < bs) Li[(size_t)(j0 + c) * ld + j0 + r] = x[r];
}

// block row i of L^-1 below the diagonal: for every j < i,
// Li_ij = -Li_ii (sum over k = j .. i-1 of L_ik Li_kj)  (one CTA per j)
constexpr int TR_KC = 8;  // 8-deep chunks: S (33 KB) and both chunks fit 48 KB
__global__ void __launch_bounds__(256) k_trtri_row(const double* L, double* Li, int ld, int dim, int ib) {
    __shared__ double sa[TR_KC][CB + 1];
    __shared__ double sb[TR_KC][CB + 1];
    __shared__ double S[CB][CB + 1];
    const int jb = blockIdx.x;  // < ib
    const int i0 = ib * CB, j0 = jb * CB;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    // S = sum_k L_ik Li_kj: rows of block i, columns of block j, reduction over k0 in [j0, i0)
    for (int q0 = j0; q0 < i0; q0 += TR_KC) {
        __syncthreads();
        for (int e = threadIdx.x; e < TR_KC * CB; e += 256) {
            const int r = e % CB, q = e / CB;
            sa[q][r] = (i0 + r < dim) ? L[(size_t)(q0 + q) * ld + i0 + r] : 0.0;   // L(i0 + r, q0 + q)
            sb[q][r] = Li[(size_t)(j0 + r) * ld + q0 + q];                         // Li(q0 + q, j0 + r)
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < TR_KC; q++) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; u++) { a[u] = sa[q][ty * 4 + u]; b[u] = sb[q][tx * 4 + u]; }
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int v = 0; v < 4; v++) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
        for (int v = 0; v < 4; v++) S[ty * 4 + u][tx * 4 + v] = acc[u][v];
    // Li_ij = -Li_ii S
    double out[4][4] = {};
    const int bsi = min(CB, dim - i0);
    for (int q0 = 0; q0 < CB; q0 += TR_KC) {
        __syncthreads();
        for (int e = threadIdx.x; e < TR_KC * CB; e += 256) {
            const int r = e % CB, q = e / CB;
            sa[q][r] = (r < bsi && q0 + q < bsi) ? Li[(size_t)(i0 + q0 + q) * ld + i0 + r] : 0.0;  // Li_ii(r, q)
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < TR_KC; q++) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; u++) { a[u] = sa[q][ty * 4 + u]; b[u] = S[q0 + q][tx * 4 + u]; }
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int v = 0; v < 4; v++) out[u][v] = fma(a[u], b[v], out[u][v]);
        }
    }
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
        for (int v = 0; v < 4; v++) {
            const int r = i0 + ty * 4 + u, c = j0 + tx * 4 + v;
            if (r < dim) Li[(size_t)c * ld + r] = -out[u][v];
        }
}

}  // namespace

awg_status chol_blocked(Handle* h, double* A, int dim, int* d_flag, cudaStream_t s) {
    const int nb = (dim + CB - 1) / CB;
    for (int jb = 0; jb < nb; jb++) {
        const int j0 = jb * CB, bs = std::min(CB, dim - j0);
        k_chol_diag<<<1, 256, 0, s>>>(A, dim, j0, bs, d_flag);
        AWG_LAUNCH();
        const int below = dim - j0 - bs;
        if (below <= 0) break;
        k_chol_trsm<<<(below + 127) / 128, 128, 0, s>>>(A, dim, dim, j0, bs);
        AWG_LAUNCH();
        const int m = nb - jb - 1;
        k_chol_update<<<m * (m + 1) / 2, 256, 0, s>>>(A, dim, dim, jb);
        AWG_LAUNCH();
    }
    (void)h;
    return AWG_OK;
}

awg_status trtri_blocked(Handle* h, const double* L, double* Li, int dim, cudaStream_t s) {
    const int nb = (dim + CB - 1) / CB;
    AWG_CUDA(cudaMemsetAsync(Li, 0, (size_t)dim * dim * 8, s));
    k_trtri_diag<<<nb, 64, 0, s>>>(L, Li, dim, dim);
    AWG_LAUNCH();
    for (int ib = 1; ib < nb; ib++) {
        k_trtri_row<<<ib, 256, 0, s>>>(L, Li, dim, dim, ib);
        AWG_LAUNCH();
    }
    (void)h;
    return AWG_OK;
}

}  // namespace awg
