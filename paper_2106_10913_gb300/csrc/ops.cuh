// Operators of the AWG preconditioner shared by setup and solve.
#pragma once

#include "awg_common.cuh"

namespace awg {

// ---------------------------------------------------------------- block ops
// X, Y: n x k column-major (ld = n).  The local arena of a block has, for
// subdomain s, an n^s x k column-major slab at offset sub_ptr[s] * k.

awg_status blk_spmm(Handle* h, const double* X, double* Y, int k, cudaStream_t s);
awg_status blk_gather(Handle* h, const double* X, double* loc, int k, cudaStream_t s);
// Y = beta Y + alpha sum_s R^sT loc_s
awg_status blk_prolong(Handle* h, const double* loc, double* Y, int k, double alpha, double beta,
                       cudaStream_t s);
// Y (+)= A_- X   (add: Y += A_- X, else Y = A_- X)
awg_status blk_aminus(Handle* h, const double* X, double* Y, int k, bool add, cudaStream_t s);
// Y = A_+ X
awg_status blk_aplus(Handle* h, const double* X, double* Y, int k, cudaStream_t s);
// C (n0 x k) = Z^T X
awg_status blk_zt(Handle* h, const double* X, double* C, int k, cudaStream_t s);
// Y = beta Y + alpha Z C
awg_status blk_z(Handle* h, const double* C, double* Y, int k, double alpha, double beta,
                 cudaStream_t s);
// Y = H^NN X with the local pseudo-inverses of precision `prec`
// (AWG_FP64: float64 GEMM; AWG_MIXED_FP32: float32 operands and accumulation)
awg_status blk_hnn(Handle* h, const double* X, double* Y, int k, cudaStream_t s,
                   int prec = AWG_FP64);
// Y = H_2 X = Pi H^NN Pi^T X + Z E^-1 Z^T X
awg_status blk_h2(Handle* h, const double* X, double* Y, int k, cudaStream_t s,
                  int prec = AWG_FP64);

// column-wise helpers (k columns of length n, ld = n)
awg_status col_dot(Handle* h, const double* X, const double* Y, double* out, int k, cudaStream_t s);

}  // namespace awg
