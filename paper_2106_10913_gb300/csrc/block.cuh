// Multi-right-hand-side ("block") hot path: declarations shared by block.cu
// (CUDA-core kernels, block apply and block PCG) and umma.cu (tensor-core
// passes over W).  Not part of the C ABI.
//
// A block vector holds K columns (K = 16, 32 or 64; the caller's nrhs
// columns padded with zero columns) stored row by row: X[i * K + c].  Every
// warp then reads whole rows, so the gathers through index lists (CSR
// columns, subdomain index lists, incidence lists) move K contiguous values
// per index instead of one.
#pragma once

#include "awg_common.cuh"

namespace awg {

constexpr int BLK_KMAX = 64;

// Block apply of one stage (0 A, 1 A_+, 2 H^NN, 3 H_2, 4 H_3,ad) to nrhs <=
// 64 columns (column-major, ld), and block PCG with H_3,ad (groups of up to
// 64 columns), on stream s.
awg_status block_apply(Handle* h, int which, int prec, const double* x, double* y, int nrhs, int ld,
                       cudaStream_t s);
awg_status block_pcg(Handle* h, int prec, const double* b, double* x, int nrhs, int ld, double rtol, int* iters,
                     double* relres, cudaStream_t s);

// Y = M X with a dense coarse inverse (which 0 E^-1, 1 F^-1, 2 H_3,inex
// inner inverse of form prec) through the block coarse product (engine 0
// float64 CUDA cores, 1 tensor-core slices, 2 the same with short reduction
// splits); X, Y column-major dim x nrhs; synchronises s
awg_status block_coarse_apply(Handle* h, int which, int prec, int engine, const double* x, double* y, int nrhs,
                              cudaStream_t s);
// Block PCG whose iterations run as one CUDA graph launch (conditional
// while node, device-side stopping test); asynchronous on s.
awg_status block_pcg_async(Handle* h, int prec, const double* b, double* x, int nrhs, int ld, double rtol,
                           int* d_iters, double* d_relres, int* d_status, cudaStream_t s);
// kernels launched by graph loop bodies since the last call (reset)
int64_t block_graph_launches(Handle* h);
// W = A_+^-1 Vhat (n x nm column-major, ld = n) by flexible block PCG with
// H_2 in precision wprec, groups of 64 columns
awg_status block_solve_w(Handle* h, int wprec, const double* Vhat, double* W, int nm, double rtol, int maxit,
                         int* its_max, double* worst, cudaStream_t s);

// Tensor-core passes over a 16-bit W (float16 or bfloat16), row-major
// n x ldw.  All pointers are device pointers.
struct UmmaW {
    const void* W = nullptr;      // n x ldw, 16-bit
    int n = 0, ldw = 0, nm = 0;   // rows, stride (multiple of 8), used columns
    int bf16 = 0;                 // 1: bfloat16 storage, 0: float16
};

// part[split][c * K + j] = sum over rows i of split of W(i, c) * Bt(j, i) (hi + lo)
// Bt: 2K x n 16-bit with row stride ldb (a multiple of 8), row j (< K) the
// high part of column j of the scaled right-hand side, row K + j its low
// part.  Returns AWG_ERR_INVALID_ARG for unsupported sizes.
awg_status umma_wt(const UmmaW& u, int K, const void* Bt, int ldb, float* part, int splits, int* d_err,
                   cudaStream_t s);
// out(i, j) = sum_c W(i, c) * Dt(j, c) (hi + lo), fp32 n x K row-major;
// Dt: 2K x ldw 16-bit (row stride ldw)
awg_status umma_wd(const UmmaW& u, int K, const void* Dt, float* out, int* d_err, cudaStream_t s);
// Tensor-core local solves with the float32 local pseudo-inverses (TF32,
// three products of high and low parts): tables built once per handle.
struct UmmaLocal {
    int N = 0, ntiles = 0, max_kc = 0, max_tiles_sub = 0;
    const int* sub_ptr = nullptr;     // int32[N+1]
    const int* sub_idx = nullptr;     // int32[sum_ns]
    const float* Gt = nullptr;        // 16 KB G images, sum over s of RT_s * KC_s
    const int64_t* gt_off = nullptr;  // int64[N]: first image of subdomain s
    const int64_t* kc_prefix = nullptr;  // int64[N+1]: prefix of KC_s = ceil(n^s / 32)
    const int* tile_sub = nullptr;    // int32[ntiles]: subdomain of CTA tile t
    const int* tile_rt = nullptr;     // int32[ntiles]: 128-row tile of CTA tile t
};
// Gt from the float32 local pseudo-inverses (column-major, ld = n^s rounded up to 4)
awg_status umma_local_tiles(const UmmaLocal& u, const int64_t* g32off, const float* G, cudaStream_t s);
// out(P, :) (row-major sum_ns x K) = G_s X_s for every subdomain, X row-major
// n x K; lt: scratch of kc_prefix[N] * 2 * K * 32 floats
awg_status umma_local(const UmmaLocal& u, int K, const float* X, float* lt, float* out, int* d_err,
                      cudaStream_t s);

// Float64-accurate products with a dense coarse inverse on the tensor cores
// (ozaki.cu): the matrix is cut once into OZ_SLICES bfloat16 slices of
// OZ_BITS-bit integer digits with power-of-two row scales, the right-hand
// sides per call, and the exact slice products are summed in float64.
constexpr int OZ_BITS = 7;
constexpr int OZ_SLICES = 8;
struct OzMat {
    const void* q = nullptr;   // bfloat16 slices, OZ_SLICES x dimp x ldk
    const int* ex = nullptr;   // row exponents, int32[dimp]
    int dim = 0, dimp = 0, ldk = 0;
};
// bytes of the slices of a dim x dim matrix; doubles of the partial sums and
// bytes of the right-hand-side slices (with the column exponents) of one
// product with K columns
size_t oz_slices_bytes(int dim);
constexpr int OZ_CHUNKS_MAX = 63;  // 64-deep stages per reduction split: sums of <= 4032 products stay exact
size_t oz_part_elems(int dim, int K, int chunks_per_split = OZ_CHUNKS_MAX);
size_t oz_xs_bytes(int dim, int K);
// slices of M (dim x dim row-major float64) into q / ex (allocated in the
// handle when empty); fills *out
awg_status oz_slice_matrix(const double* M, int dim, DevBuf& q, DevBuf& ex, Handle* h, cudaStream_t s,
                           OzMat* out);
// Y = alpha M X + beta Sub (Sub may be NULL), X and Y row-major dim x K
// float64 (K = 16, 32, 64); xs: oz_xs_bytes(dim, K) bytes, part:
// oz_part_elems(dim, K, chunks_per_split) doubles of scratch; the reduction
// is split every chunks_per_split x 64 (<= OZ_CHUNKS_MAX) terms
awg_status oz_gemm(const OzMat& m, int K, const double* X, double* Y, double alpha, const double* Sub, double beta,
                   void* xs, double* part, int* d_err, cudaStream_t s, int chunks_per_split = OZ_CHUNKS_MAX);

// Whether the tensor-core passes are available (driver entry point found).
bool umma_available();
// Number of row splits umma_wt uses when asked for `want` (no empty split).
int umma_wt_splits(int n, int want);

}  // namespace awg
