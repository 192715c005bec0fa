// Single-right-hand-side hot path: CSR SpMV, the AWG apply (H_3,ad, H_3,hyb,
// H_3,inex over H_2 = H^NN_hyb(tau)) and PCG.
//
// Per apply of H_3,ad (Def. 10 with Thm. 4):
//   y0 = Z^T r, w0 = W^T r             block-sparse gather-dot, tall-skinny pass 1
//   c1 = E^-1 y0, d = F^-1 w0          dense coarse solves (explicit inverses)
//   t  = r - A_+ Z c1                  Pi^T r  (A_+ x = A x + A_- x)
//   u  = H^NN t                        batched local pseudo-inverse GEMVs
//   c2 = E^-1 Z^T A_+ u
//   z  = u + Z (c1 - c2) + W d         Pi H^NN Pi^T r + Z E^-1 Z^T r + W F^-1 W^T r
// Every sum over subdomains is an owner-computes gather over the incidence
// lists, every reduction a fixed-order tree: results are bitwise repeatable.

#include "awg_common.cuh"
#include "ops.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace awg {

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}

// Finish of a grid-wide sum in one launch: every block stores its block sum
// v in part[blockIdx.x]; the last block to arrive (ticket counter) adds the
// partials in block order, exactly as a separate one-block kernel would, writes
// *out and resets the counter.  The result does not depend on scheduling.
__device__ __forceinline__ void grid_sum_finish(double v, double* part, unsigned* counter, double* out,
                                                double* red) {
    __shared__ unsigned ticket;
    if (threadIdx.x == 0) {
        part[blockIdx.x] = v;
        __threadfence();
        ticket = atomicAdd(counter, 1u);
    }
    __syncthreads();
    if (ticket != gridDim.x - 1) return;
    __threadfence();
    double acc = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) acc += __ldcg(part + b);
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) {
        *out = acc;
        *counter = 0u;
    }
}

// ------------------------------------------------------------------ SpMV
// y = A x; if pdot, also the sum x^T y into *dot (grid_sum_finish).
__global__ void __launch_bounds__(256) k_spmv(int n, const int* __restrict__ rp,
                                              const int* __restrict__ ci,
                                              const double* __restrict__ a,
                                              const double* __restrict__ x, double* __restrict__ y,
                                              double* pdot, unsigned* counter, double* dot) {
    __shared__ double red[32];
    double part = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double acc = 0.0;
        const int e = rp[i + 1];
        for (int k = rp[i]; k < e; k++) acc = fma(a[k], x[ci[k]], acc);
        y[i] = acc;
        part = fma(acc, x[i], part);
    }
    if (pdot) {
        part = block_sum(part, red);
        grid_sum_finish(part, pdot, counter, dot, red);
    }
}

// -------------------------------------------------------- block-sparse ops
// c[colptr[s] + j] = wsign w_j sum_p B_s(p, j) x(idx_s(p))  (w optional):
// every thread takes rows p = t, t + blockDim, ... and keeps one accumulator
// per column (all loads independent and coalesced along p), then the
// per-warp sums meet in shared memory in a fixed order.
constexpr int TG_MAXC = 16;
__global__ void __launch_bounds__(256) k_blk_tgemv2(const int* __restrict__ sub_ptr,
                                                    const int* __restrict__ sub_idx,
                                                    const int* __restrict__ colptr,
                                                    const int64_t* __restrict__ boff,
                                                    const double* __restrict__ B,
                                                    const double* __restrict__ x,
                                                    const double* __restrict__ w, double wsign,
                                                    double* c) {
    __shared__ double red[8][TG_MAXC];
    const int s = blockIdx.x;
    const int p0 = sub_ptr[s], m = sub_ptr[s + 1] - p0;
    const int c0 = colptr[s], nc = colptr[s + 1] - c0;
    const double* Bs = B + boff[s];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int cb = 0; cb < nc; cb += TG_MAXC) {
        const int k = min(TG_MAXC, nc - cb);
        double acc[TG_MAXC];
#pragma unroll
        for (int j = 0; j < TG_MAXC; j++) acc[j] = 0.0;
        for (int q = threadIdx.x; q < m; q += blockDim.x) {
            const double xv = x[sub_idx[p0 + q]];
            const double* col = Bs + (size_t)cb * m + q;
#pragma unroll
            for (int j = 0; j < TG_MAXC; j++)
                if (j < k) acc[j] = fma(col[(size_t)j * m], xv, acc[j]);
        }
#pragma unroll
        for (int j = 0; j < TG_MAXC; j++) {
            if (j >= k) break;
            const double v = warp_sum(acc[j]);
            if (lane == 0) red[wid][j] = v;
        }
        __syncthreads();
        if (threadIdx.x < k) {
            double v = 0.0;
#pragma unroll
            for (int q = 0; q < 8; q++) v += red[q][threadIdx.x];
            const int cj = c0 + cb + threadIdx.x;
            c[cj] = w ? wsign * w[cj] * v : v;
        }
        __syncthreads();
    }
}

// Same product with the rows of a subdomain split over blockIdx.y (256 rows
// per block, one per thread, so every load of a block is in flight at once):
// block (s, y) leaves its column sums in part[(s * gridDim.y + y) * TG_MAXC],
// and the last block of subdomain s to finish (ticket counter cnt[s]) adds
// them in block order and resets the counter.  At most TG_MAXC columns per
// subdomain.
__global__ void __launch_bounds__(256) k_blk_tgemv3(const int* __restrict__ sub_ptr,
                                                    const int* __restrict__ sub_idx,
                                                    const int* __restrict__ colptr,
                                                    const int64_t* __restrict__ boff,
                                                    const double* __restrict__ B,
                                                    const double* __restrict__ x,
                                                    const double* __restrict__ w, double wsign,
                                                    double* part, unsigned* cnt, double* c) {
    __shared__ double red[8][TG_MAXC];
    __shared__ unsigned ticket;
    const int s = blockIdx.x, yb = blockIdx.y;
    const int p0 = sub_ptr[s], m = sub_ptr[s + 1] - p0;
    const int nsplit = (m + 255) >> 8;
    if (yb >= nsplit) return;
    const int c0 = colptr[s], nc = colptr[s + 1] - c0;
    if (nc == 0) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int q = (yb << 8) + threadIdx.x;
    double acc[TG_MAXC];
    if (q < m) {
        const double xv = x[sub_idx[p0 + q]];
        const double* col = B + boff[s] + q;
        double bv[TG_MAXC];
#pragma unroll
        for (int j = 0; j < TG_MAXC; j++) bv[j] = (j < nc) ? col[(size_t)j * m] : 0.0;
#pragma unroll
        for (int j = 0; j < TG_MAXC; j++) acc[j] = bv[j] * xv;
    } else {
#pragma unroll
        for (int j = 0; j < TG_MAXC; j++) acc[j] = 0.0;
    }
#pragma unroll
    for (int j = 0; j < TG_MAXC; j++) {
        if (j >= nc) break;
        const double v = warp_sum(acc[j]);
        if (lane == 0) red[wid][j] = v;
    }
    __syncthreads();
    double* ps = part + (size_t)s * gridDim.y * TG_MAXC;
    if (threadIdx.x < nc) {
        double v = 0.0;
#pragma unroll
        for (int k = 0; k < 8; k++) v += red[k][threadIdx.x];
        ps[yb * TG_MAXC + threadIdx.x] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) ticket = atomicAdd(cnt + s, 1u);
    __syncthreads();
    if (ticket != (unsigned)(nsplit - 1)) return;
    __threadfence();
    if (threadIdx.x < nc) {
        double v = 0.0;
        for (int k = 0; k < nsplit; k++) v += __ldcg(ps + k * TG_MAXC + threadIdx.x);
        const int cj = c0 + threadIdx.x;
        c[cj] = w ? wsign * w[cj] * v : v;
    }
    if (threadIdx.x == 0) cnt[s] = 0u;
}

// y(i) = beta y(i) + alpha sum over the copies (s, p) of i of
// sum_j B_s(p, j) c[colptr[s] + j] + gamma z(i): block-sparse GEMV and
// prolongation in one owner-computes pass (copies in subdomain order)
__global__ void k_blk_prolong(int n, const int* __restrict__ inc_ptr, const int* __restrict__ inc_pos,
                              const int* __restrict__ inc_sub, const int* __restrict__ sub_ptr,
                              const int* __restrict__ colptr, const int64_t* __restrict__ boff,
                              const double* __restrict__ B, const double* __restrict__ c, double* y,
                              double alpha, double beta, const double* z, double gamma,
                              const double* __restrict__ z2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int e = inc_ptr[i]; e < inc_ptr[i + 1]; e++) {
        const int s = inc_sub[e];
        const int ps = sub_ptr[s], m = sub_ptr[s + 1] - ps;
        const int c0 = colptr[s], nc = colptr[s + 1] - c0;
        const double* b = B + boff[s] + (inc_pos[e] - ps);
        int j = 0;
        for (; j + 8 <= nc; j += 8) {  // eight loads in flight, then the FMAs
            double bv[8], cv[8];
#pragma unroll
            for (int k = 0; k < 8; k++) { bv[k] = b[(size_t)(j + k) * m]; cv[k] = c[c0 + j + k]; }
#pragma unroll
            for (int k = 0; k < 8; k++) acc = fma(bv[k], cv[k], acc);
        }
        for (; j < nc; j++) acc = fma(b[(size_t)j * m], c[c0 + j], acc);
    }
    double v = alpha * acc;
    if (beta != 0.0) v = fma(beta, y[i], v);
    if (z) v = fma(gamma, z[i], v);
    if (z2) v += z2[i];
    y[i] = v;
}

__global__ void k_add(int n, const double* __restrict__ a, double* y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += a[i];
}

// y(i) = yin(i) + sign (A x + A_- x)(i), with cm = |Lambda_-| V_-^T R x per
// subdomain from k_blk_tgemv2: one row of A and the copies of i in one pass
__global__ void k_aplus_row(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                            const double* __restrict__ a, const double* __restrict__ x,
                            const int* __restrict__ inc_ptr, const int* __restrict__ inc_pos,
                            const int* __restrict__ inc_sub, const int* __restrict__ sub_ptr,
                            const int* __restrict__ colptr, const int64_t* __restrict__ boff,
                            const double* __restrict__ V, const double* __restrict__ cm,
                            const double* yin, double sign, double* y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; k++) acc = fma(a[k], x[ci[k]], acc);
    if (cm) {
        for (int e = inc_ptr[i]; e < inc_ptr[i + 1]; e++) {
            const int s = inc_sub[e];
            const int ps = sub_ptr[s], m = sub_ptr[s + 1] - ps;
            const int c0 = colptr[s], nc = colptr[s + 1] - c0;
            const double* b = V + boff[s] + (inc_pos[e] - ps);
            int j = 0;
            for (; j + 8 <= nc; j += 8) {
                double bv[8], cv[8];
#pragma unroll
                for (int k = 0; k < 8; k++) { bv[k] = b[(size_t)(j + k) * m]; cv[k] = cm[c0 + j + k]; }
#pragma unroll
                for (int k = 0; k < 8; k++) acc = fma(bv[k], cv[k], acc);
            }
            for (; j < nc; j++) acc = fma(b[(size_t)j * m], cm[c0 + j], acc);
        }
    }
    y[i] = yin ? fma(sign, acc, yin[i]) : sign * acc;
}

// y = beta y + alpha sum_copies loc + gamma z
__global__ void k_prolong1(int n, const int* __restrict__ inc_ptr, const int* __restrict__ inc_pos,
                           const double* __restrict__ loc, double* y, double alpha, double beta,
                           const double* z, double gamma) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int e = inc_ptr[i]; e < inc_ptr[i + 1]; e++) acc += loc[inc_pos[e]];
    double v = alpha * acc;
    if (beta != 0.0) v = fma(beta, y[i], v);
    if (z) v = fma(gamma, z[i], v);
    y[i] = v;
}

// ------------------------------------------------------ local pseudo-inverse
// loc[sub_ptr[s] + p] = sum_q G_s(p, q) x(idx_s(q)), G_s symmetric, full
// column-major storage: row p is read as column p (contiguous).
constexpr int LG_ROWS = 32;

__global__ void __launch_bounds__(256) k_local_gemv64(const int* __restrict__ sub_ptr,
                                                      const int* __restrict__ sub_idx,
                                                      const int64_t* __restrict__ goff,
                                                      const double* __restrict__ G,
                                                      const double* __restrict__ x, double* loc) {
    extern __shared__ double xs[];
    const int s = blockIdx.x;
    const int p0 = sub_ptr[s], m = sub_ptr[s + 1] - p0;
    const int r0 = blockIdx.y * LG_ROWS;
    if (r0 >= m) return;
    for (int q = threadIdx.x; q < m; q += blockDim.x) xs[q] = x[sub_idx[p0 + q]];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double* Gs = G + goff[s];
    const int r1 = min(m, r0 + LG_ROWS);
    for (int p = r0 + wid; p < r1; p += nw) {
        const double* col = Gs + (size_t)p * m;
        double a0 = 0.0, a1 = 0.0;
        int q = lane;
        for (; q + 32 < m; q += 64) {
            a0 = fma(col[q], xs[q], a0);
            a1 = fma(col[q + 32], xs[q + 32], a1);
        }
        if (q < m) a0 = fma(col[q], xs[q], a0);
        const double acc = warp_sum(a0 + a1);
        if (lane == 0) loc[p0 + p] = acc;
    }
}

// float32 local operators: column-major with a leading dimension padded to a
// multiple of 4 (columns 16-byte aligned, padding zero) at offsets g32off.
// The gathered x comes in float32 from k_gather_f32 (one conversion per
// local position per apply), rows are read with 16-byte streaming loads and
// the results of a block's rows leave through one conversion instruction:
// no float64 operation sits in the inner loop, because the float64 pipe is
// about 58 times narrower than the float32 one on this GPU.
__global__ void k_gather_f32(int64_t sum_ns, const int* __restrict__ sub_idx,
                             const double* __restrict__ x, float* xloc) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < sum_ns) xloc[p] = (float)x[sub_idx[p]];
}

__global__ void __launch_bounds__(256) k_local_gemv_f32(const int* __restrict__ sub_ptr,
                                                        const int64_t* __restrict__ g32off,
                                                        const float* __restrict__ G,
                                                        const float* __restrict__ xloc,
                                                        double* loc) {
    extern __shared__ __align__(16) float xs32[];
    float* xs = xs32;
    __shared__ float outr[LG_ROWS];
    const int s = blockIdx.x;
    const int p0 = sub_ptr[s], m = sub_ptr[s + 1] - p0;
    const int ld = (m + 3) & ~3;
    const int r0 = blockIdx.y * LG_ROWS;
    if (r0 >= m) return;
    for (int q = threadIdx.x; q < ld; q += blockDim.x) xs[q] = (q < m) ? xloc[p0 + q] : 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float* Gs = G + g32off[s];
    const float4* x4 = reinterpret_cast<const float4*>(xs);
    const int nq = ld >> 2;
    const int r1 = min(m, r0 + LG_ROWS);
    for (int p = r0 + wid; p < r1; p += nw) {
        const float4* col = reinterpret_cast<const float4*>(Gs + (size_t)p * ld);
        float a0 = 0.f, a1 = 0.f;
        int q = lane;
        for (; q + 32 < nq; q += 64) {
            const float4 g0 = __ldcs(col + q), g1 = __ldcs(col + q + 32);
            const float4 u0 = x4[q], u1 = x4[q + 32];
            a0 = fmaf(g0.x, u0.x, fmaf(g0.y, u0.y, fmaf(g0.z, u0.z, fmaf(g0.w, u0.w, a0))));
            a1 = fmaf(g1.x, u1.x, fmaf(g1.y, u1.y, fmaf(g1.z, u1.z, fmaf(g1.w, u1.w, a1))));
        }
        if (q < nq) {
            const float4 g0 = __ldcs(col + q);
            const float4 u0 = x4[q];
            a0 = fmaf(g0.x, u0.x, fmaf(g0.y, u0.y, fmaf(g0.z, u0.z, fmaf(g0.w, u0.w, a0))));
        }
        const float acc = warp_sumf(a0 + a1);
        if (lane == 0) outr[p - r0] = acc;
    }
    __syncthreads();
    if (threadIdx.x < r1 - r0) loc[p0 + r0 + threadIdx.x] = (double)outr[threadIdx.x];
}

// ------------------------------------------------------------ dense coarse
// y = M x, M symmetric dim x dim (row p = column p), warp per row
// y = alpha M x + beta sub  (sub optional; y must not alias x)
__global__ void __launch_bounds__(256) k_dense_gemv(int dim, const double* __restrict__ M,
                                                    const double* __restrict__ x, double* y,
                                                    double alpha, const double* sub, double beta) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= dim) return;
    const double* col = M + (size_t)row * dim;
    double acc = 0.0;
    for (int q = lane; q < dim; q += 32) acc = fma(col[q], x[q], acc);
    acc = warp_sum(acc);
    if (lane == 0) y[row] = sub ? fma(beta, sub[row], alpha * acc) : alpha * acc;
}

// ------------------------------------------------- tall-skinny W (row-major)
// W is stored row-major with ldw a multiple of 8 (rows 16-byte aligned, the
// padding columns zero).  Each thread moves 16 bytes per load (2 float64,
// 4 float32 or 8 bfloat16) with the streaming cache hint (W is read once per
// pass and is far larger than L2) and accumulates in the compute type of the
// storage (float64 for float64; float32 for float32 and bfloat16), never
// converting element by element through float64, whose pipe is narrow on
// this GPU.
template <typename TS> struct Vec;
template <> struct Vec<double> {
    static constexpr int V = 2;
    using A = double;
    __device__ __forceinline__ static void load(const double* p, double* o) {
        const double2 t = __ldcs(reinterpret_cast<const double2*>(p));
        o[0] = t.x; o[1] = t.y;
    }
};
template <> struct Vec<float> {
    static constexpr int V = 4;
    using A = float;
    __device__ __forceinline__ static void load(const float* p, float* o) {
        const float4 t = __ldcs(reinterpret_cast<const float4*>(p));
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    }
};
template <> struct Vec<__nv_bfloat16> {
    static constexpr int V = 8;
    using A = float;
    __device__ __forceinline__ static void load(const __nv_bfloat16* p, float* o) {
        const uint4 t = __ldcs(reinterpret_cast<const uint4*>(p));
        const unsigned w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            o[2 * k] = __uint_as_float(w[k] << 16);          // low half: element 2k
            o[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
        }
    }
};

template <> struct Vec<__half> {
    static constexpr int V = 8;
    using A = float;
    __device__ __forceinline__ static void load(const __half* p, float* o) {
        const uint4 t = __ldcs(reinterpret_cast<const uint4*>(p));
        const __half2* hv = reinterpret_cast<const __half2*>(&t);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float2 f = __half22float2(hv[k]);  // .x: element 2k
            o[2 * k] = f.x;
            o[2 * k + 1] = f.y;
        }
    }
};

// V consecutive values of a 16-byte aligned shared array, 16 bytes per load
template <typename A, int V>
__device__ __forceinline__ void lds_vec(const A* p, A* o) {
    static_assert((V * sizeof(A)) % 16 == 0, "vector width");
#pragma unroll
    for (int k = 0; k < (int)(V * sizeof(A) / 16); k++) {
        const float4 t = reinterpret_cast<const float4*>(p)[k];
        reinterpret_cast<float4*>(o)[k] = t;
    }
}

constexpr int WT_THREADS = 256;  // 8 warps
constexpr int WT_CW = 256;       // columns of W per block (blockIdx.y)

// part[b*ldw + c] = sum over the rows of row block b of W(i, c) r(i), for the
// 256 columns of column chunk blockIdx.y.  The block's r values are staged
// once in shared memory in the compute type (times the row scale of a scaled
// float16 W); the 8 warps take every 8th row and the 8 partial sums meet in
// shared memory in a fixed order.
template <typename TS>
__global__ void __launch_bounds__(WT_THREADS) k_wt_partial(int n, int ldw, int rows,
                                                           const TS* __restrict__ W,
                                                           const double* __restrict__ r,
                                                           const float* __restrict__ rscale,
                                                           double* part, float* rf) {
    using A = typename Vec<TS>::A;
    constexpr int V = Vec<TS>::V;
    constexpr int UNR = WT_CW / (32 * V);
    extern __shared__ __align__(16) unsigned char wt_smem[];
    A* red = reinterpret_cast<A*>(wt_smem);  // [8][WT_CW]
    A* rs = red + 8 * WT_CW;                 // [rows]
    const int i0 = blockIdx.x * rows;
    const int nr = min(n, i0 + rows) - i0;
    const int c0 = blockIdx.y * WT_CW;
    if (rscale) {
        for (int t = threadIdx.x; t < nr; t += WT_THREADS) rs[t] = (A)r[i0 + t] * rscale[i0 + t];
        if (rf && blockIdx.y == 0)  // S_r r in float32 for the sparse correction
            for (int t = threadIdx.x; t < nr; t += WT_THREADS) rf[i0 + t] = (float)rs[t];
    } else
        for (int t = threadIdx.x; t < nr; t += WT_THREADS) rs[t] = (A)r[i0 + t];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    A acc[UNR][V];
#pragma unroll
    for (int u = 0; u < UNR; u++)
#pragma unroll
        for (int j = 0; j < V; j++) acc[u][j] = 0;
    // four rows per step: their loads are issued before the first FMA
    int i = wid;
    for (; i + 24 < nr; i += 32) {
        A wv[4][UNR][V];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const TS* row = W + (size_t)(i0 + i + 8 * k) * ldw;
#pragma unroll
            for (int u = 0; u < UNR; u++) {
                const int c = c0 + (u * 32 + lane) * V;
                if (c < ldw) Vec<TS>::load(row + c, wv[k][u]);
                else
#pragma unroll
                    for (int j = 0; j < V; j++) wv[k][u][j] = 0;
            }
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const A ri = rs[i + 8 * k];
#pragma unroll
            for (int u = 0; u < UNR; u++)
#pragma unroll
                for (int j = 0; j < V; j++) acc[u][j] = fma(wv[k][u][j], ri, acc[u][j]);
        }
    }
    for (; i < nr; i += 8) {
        const A ri = rs[i];
        const TS* row = W + (size_t)(i0 + i) * ldw;
#pragma unroll
        for (int u = 0; u < UNR; u++) {
            const int c = c0 + (u * 32 + lane) * V;
            if (c < ldw) {
                A w[V];
                Vec<TS>::load(row + c, w);
#pragma unroll
                for (int j = 0; j < V; j++) acc[u][j] = fma(w[j], ri, acc[u][j]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < UNR; u++)
#pragma unroll
        for (int j = 0; j < V; j++) red[wid * WT_CW + (u * 32 + lane) * V + j] = acc[u][j];
    __syncthreads();
    const int c = c0 + threadIdx.x;
    if (c < ldw) {
        A sum = 0;
#pragma unroll
        for (int w = 0; w < 8; w++) sum += red[w * WT_CW + threadIdx.x];
        part[(size_t)blockIdx.x * ldw + c] = (double)sum;
    }
}

// out[c] = sum over the row blocks of part[b*ldp + c]  (fixed order), times
// the column scale of a scaled float16 W
__global__ void k_reduce_cols(int nb, int nm, int ldp, const double* __restrict__ part,
                              const float* __restrict__ cscale, double* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nm) return;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int b = 0;
    for (; b + 3 < nb; b += 4) {
        a0 += part[(size_t)b * ldp + c];
        a1 += part[(size_t)(b + 1) * ldp + c];
        a2 += part[(size_t)(b + 2) * ldp + c];
        a3 += part[(size_t)(b + 3) * ldp + c];
    }
    for (; b < nb; b++) a0 += part[(size_t)b * ldp + c];
    const double v = (a0 + a1) + (a2 + a3);
    out[c] = cscale ? v * (double)cscale[c] : v;
}

// out[c] = cscale[c] (sum of the partials + sum_i C_ic (S_r r)_i): the
// float16 form's column sums plus its sparse correction (CSC, one block per
// column; fixed order)
__global__ void __launch_bounds__(256) k_reduce_cols_corr(int nb, int ldp, const double* __restrict__ part,
                                                          const float* __restrict__ cscale,
                                                          const int* __restrict__ ccp,
                                                          const int* __restrict__ crow,
                                                          const float* __restrict__ cval,
                                                          const float* __restrict__ rf, double* out) {
    __shared__ double red[32];
    const int c = blockIdx.x;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += part[(size_t)b * ldp + c];
    float fc = 0.f;
    for (int k = ccp[c] + threadIdx.x; k < ccp[c + 1]; k += blockDim.x) fc = fmaf(cval[k], rf[crow[k]], fc);
    acc = block_sum(acc + (double)fc, red);
    if (threadIdx.x == 0) out[c] = acc * (double)cscale[c];
}

template <typename A>
__device__ __forceinline__ A warp_sum_t(A v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// d in the compute type of W's storage (one conversion per element per
// apply), times the column scale of a scaled float16 W
__global__ void k_d_to_f32(int nm, int ldw, const double* __restrict__ d, const float* __restrict__ cscale,
                           float* d32) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ldw) d32[c] = (c < nm) ? (cscale ? (float)(d[c] * (double)cscale[c]) : (float)d[c]) : 0.f;
}

// z(i) = v(i) + sum_c W(i, c) d(c).  One warp per row (grid-stride, many
// warps in flight), the row sum reduced in the compute type; only lane 0
// touches float64 (one conversion and one add per row, next to a row read of
// ldw elements).  d (compute type, zero-padded to ldw) is staged in shared
// memory: d itself for float64 storage, the float32 copy from k_d_to_f32
// otherwise.
template <typename TS>
__global__ void __launch_bounds__(256) k_w_d(int n, int ldw, const TS* __restrict__ W,
                                             const typename Vec<TS>::A* __restrict__ dA,
                                             const float* __restrict__ rscale, const int* __restrict__ crp,
                                             const int* __restrict__ ccol, const float* __restrict__ cval,
                                             const double* v, double* z) {
    using A = typename Vec<TS>::A;
    constexpr int V = Vec<TS>::V;
    extern __shared__ __align__(16) unsigned char wd_smem[];
    A* ds = reinterpret_cast<A*>(wd_smem);
    for (int c = threadIdx.x; c < ldw; c += blockDim.x) ds[c] = dA[c];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const TS* row = W + (size_t)i * ldw;
        // four 16-byte loads in flight per lane: a grid of a few blocks per
        // SM still covers the memory latency (the pass shares the GPU with
        // the H_2 chain)
        A acc[4] = {0, 0, 0, 0};
        int c = lane * V;
        for (; c + 96 * V < ldw; c += 128 * V) {
            A wv[4][V];
#pragma unroll
            for (int u = 0; u < 4; u++) Vec<TS>::load(row + c + u * 32 * V, wv[u]);
#pragma unroll
            for (int u = 0; u < 4; u++) {
                A dv[V];
                lds_vec<A, V>(ds + c + u * 32 * V, dv);
#pragma unroll
                for (int j = 0; j < V; j++) acc[u] = fma(wv[u][j], dv[j], acc[u]);
            }
        }
        for (; c < ldw; c += 32 * V) {
            A w0[V], d0[V];
            Vec<TS>::load(row + c, w0);
            lds_vec<A, V>(ds + c, d0);
#pragma unroll
            for (int j = 0; j < V; j++) acc[0] = fma(w0[j], d0[j], acc[0]);
        }
        if (crp)  // sparse correction of the row (scaled units, d staged scaled)
            for (int k = crp[i] + lane; k < crp[i + 1]; k += 32) acc[1] = fma((A)cval[k], ds[ccol[k]], acc[1]);
        A s = warp_sum_t<A>((acc[0] + acc[1]) + (acc[2] + acc[3]));
        if (lane == 0) {
            if (rscale) s *= rscale[i];
            z[i] = (v ? v[i] : 0.0) + (double)s;
        }
    }
}

// -------------------------------------------------------------- vector ops
__global__ void k_sub(int n, const double* a, const double* b, double* c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) c[i] = a[i] - b[i];
}

// *out = x^T y (nothing when *gate is 0)
__global__ void k_dot(int n, const double* __restrict__ x, const double* __restrict__ y, double* part,
                      unsigned* counter, double* out, const double* gate = nullptr) {
    if (gate && *gate == 0.0) return;
    __shared__ double red[32];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        acc = fma(x[i], y[i], acc);
    acc = block_sum(acc, red);
    grid_sum_finish(acc, part, counter, out, red);
}

// PCG scalars (device): 0 rz, 1 pq, 2 rr, 3 rz_new, 5 b.b, 6 true residual
enum { S_RZ = 0, S_PQ = 1, S_RR = 2, S_RZN = 3, S_BB = 5, S_TR = 6 };

// x += alpha p, r -= alpha q with alpha = rz / pq; scal[S_RR] = r.r
__global__ void k_pcg_xr(int n, double* scal, const double* __restrict__ p, const double* __restrict__ q,
                         double* x, double* r, double* part, unsigned* counter) {
    __shared__ double red[32];
    const double pq = scal[S_PQ];
    const double alpha = (pq > 0.0) ? scal[S_RZ] / pq : 0.0;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
    }
    acc = block_sum(acc, red);
    grid_sum_finish(acc, part, counter, scal + S_RR, red);
}

// p = z + beta p with beta = rz_new / rz; the last block then moves rz_new
// into rz (every block has read both by then)
__global__ void k_pcg_p(int n, double* scal, const double* __restrict__ z, double* p, unsigned* counter) {
    __shared__ unsigned ticket;
    const double rz = scal[S_RZ], rzn = scal[S_RZN];
    const double beta = (rz != 0.0) ? rzn / rz : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], z[i]);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        ticket = atomicAdd(counter, 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0 && ticket == gridDim.x - 1) {
        scal[S_RZ] = rzn;
        *counter = 0u;
    }
}

// ===================================================================== host
struct Ws {
    double *y0, *y2, *c1, *c2, *w0, *w1, *dd, *x1, *t, *u, *q, *loc, *loc2, *cm, *part, *wpart, *tmp, *tmp2;
    unsigned* cnt;    // ticket counters of the one-launch grid sums (zero between launches)
    double* tgpart;   // k_blk_tgemv3 partial column sums, N x splits x TG_MAXC
    unsigned* tgcnt;  // k_blk_tgemv3 ticket counter per subdomain (zero between launches)
    float *xf, *d32;  // float32 gathered local vector, float32 copy of d
    float* rf;        // S_r r in float32 (sparse correction of the float16 W)
    double* dpad;     // d zero-padded to ldw (float64 W)
};

// Carving of the single-RHS workspace; `dry` only measures it.
static size_t carve(const Handle* h, double* base, Ws* w) {
    double* p = base;
    const size_t n = h->n, n0 = std::max(1, h->n0), nm = std::max(1, h->n_minus);
    auto take = [&](size_t len) { double* r = p; p += (len + 31) / 32 * 32; return r; };
    Ws t;
    t.y0 = take(n0); t.y2 = take(n0); t.c1 = take(n0); t.c2 = take(n0);
    t.w0 = take(nm); t.w1 = take(nm); t.dd = take(nm);
    t.x1 = take(n); t.t = take(n); t.u = take(n); t.q = take(n); t.tmp = take(n); t.tmp2 = take(n);
    t.loc = take(h->sum_ns); t.loc2 = take(h->sum_ns);
    t.cm = take(std::max(1, h->n_minus_all));
    t.part = take(4096);
    t.cnt = reinterpret_cast<unsigned*>(t.part + 4064);
    t.tgpart = take((size_t)h->N * ((h->max_ns + 255) / 256) * TG_MAXC);
    t.tgcnt = reinterpret_cast<unsigned*>(take(((size_t)h->N + 1) / 2));
    t.wpart = take((size_t)h->red_blocks * std::max(8, h->ldw));
    t.xf = reinterpret_cast<float*>(take((h->sum_ns + 1) / 2 + 4));
    t.d32 = reinterpret_cast<float*>(take((std::max(8, h->ldw) + 1) / 2 + 4));
    t.rf = reinterpret_cast<float*>(take((n + 1) / 2 + 4));
    t.dpad = take(std::max(8, h->ldw));
    if (w) *w = t;
    return (size_t)(p - base) * sizeof(double);
}

static Ws ws_of(Handle* h) {
    Ws w;
    carve(h, (double*)h->ws.p, &w);
    return w;
}

size_t ws_bytes(const Handle* h) { return carve(h, nullptr, nullptr); }

static int grid_n(int n) { return std::min((n + 255) / 256, 152 * 8); }

awg_status spmv1(Handle* h, const double* x, double* y, double* pdot, cudaStream_t s) {
    // pdot: x^T y into *pdot (scratch and ticket counter in the workspace)
    Ws w = ws_of(h);
    {
        ProfScope ps_(h, AWG_PROF_SPMV, s);
        k_spmv<<<grid_n(h->n), 256, 0, s>>>(h->n, (int*)h->rowptr.p, (int*)h->colidx.p,
                                            (double*)h->val.p, x, y, pdot ? w.part : nullptr,
                                            w.cnt, pdot);
    }
    AWG_LAUNCH();
    return AWG_OK;
}

static awg_status prolong1(Handle* h, const double* loc, double* y, double alpha, double beta,
                           const double* z, double gamma, cudaStream_t s) {
    {
        ProfScope ps_(h, AWG_PROF_PROLONG, s);
        k_prolong1<<<(h->n + 255) / 256, 256, 0, s>>>(h->n, (int*)h->inc_ptr.p, (int*)h->inc_pos.p, loc,
                                                      y, alpha, beta, z, gamma);
    }
    AWG_LAUNCH();
    return AWG_OK;
}

// cm = |Lambda_-| V_-^T R x per subdomain (the middle of A_- x, Thm. 2)
// c_s = wsign w .* (B_s^T x|Omega^s) for every subdomain: the split-row
// kernel when every block has at most TG_MAXC columns, else one block per
// subdomain
static awg_status blk_tgemv(Handle* h, const int* colptr, const int64_t* boff, const double* B,
                            int maxc, const double* x, const double* wv, double wsign, double* c,
                            cudaStream_t s) {
    ProfScope ps_(h, AWG_PROF_SUBDOMAIN, s);
    if (maxc <= TG_MAXC) {
        Ws w = ws_of(h);
        const dim3 g(h->N, (h->max_ns + 255) / 256);
        k_blk_tgemv3<<<g, 256, 0, s>>>((int*)h->sub_ptr.p, (int*)h->sub_idx.p, colptr, boff, B, x, wv, wsign,
                                       w.tgpart, w.tgcnt, c);
    } else {
        k_blk_tgemv2<<<h->N, 256, 0, s>>>((int*)h->sub_ptr.p, (int*)h->sub_idx.p, colptr, boff, B, x, wv,
                                          wsign, c);
    }
    AWG_LAUNCH();
    return AWG_OK;
}

static awg_status vmt1(Handle* h, const double* x, double* cm, cudaStream_t s) {
    const int maxc = *std::max_element(h->h_nm.begin(), h->h_nm.end());
    return blk_tgemv(h, (int*)h->nm_ptr.p, (int64_t*)h->vm_off.p, (double*)h->Vm.p, maxc, x,
                     (double*)h->lam_m.p, -1.0, cm, s);
}

// y = yin + sign * A_+ x  (A_+ = A + A_-, Thm. 2)
static awg_status aplus1(Handle* h, const double* x, double* y, const double* yin, double sign,
                         Ws& w, cudaStream_t s) {
    const bool vm = h->n_minus_all > 0;
    if (vm) AWG_TRY(vmt1(h, x, w.cm, s));
    {
        ProfScope ps_(h, AWG_PROF_SPMV, s);
        k_aplus_row<<<(h->n + 255) / 256, 256, 0, s>>>(
            h->n, (int*)h->rowptr.p, (int*)h->colidx.p, (double*)h->val.p, x, (int*)h->inc_ptr.p,
            (int*)h->inc_pos.p, (int*)h->inc_sub.p, (int*)h->sub_ptr.p, (int*)h->nm_ptr.p,
            (int64_t*)h->vm_off.p, (double*)h->Vm.p, vm ? w.cm : nullptr, yin, sign, y);
    }
    AWG_LAUNCH();
    return AWG_OK;
}

// c = Z^T x (block-sparse, Thm. 4)
static awg_status zt1(Handle* h, const double* x, double* c, cudaStream_t s) {
    if (h->n0 == 0) return AWG_OK;
    const int maxc = *std::max_element(h->h_modes.begin(), h->h_modes.end());
    return blk_tgemv(h, (int*)h->mode_ptr.p, (int64_t*)h->z_off.p, (double*)h->Z.p, maxc, x, nullptr, 1.0,
                     c, s);
}

// y = beta y + alpha Z c + gamma v (+ v2)
static awg_status zc1(Handle* h, const double* c, double* y, double alpha, double beta, const double* v,
                      double gamma, cudaStream_t s, const double* v2 = nullptr) {
    {
        ProfScope ps_(h, AWG_PROF_PROLONG, s);
        k_blk_prolong<<<(h->n + 255) / 256, 256, 0, s>>>(h->n, (int*)h->inc_ptr.p, (int*)h->inc_pos.p,
                                                         (int*)h->inc_sub.p, (int*)h->sub_ptr.p,
                                                         (int*)h->mode_ptr.p, (int64_t*)h->z_off.p,
                                                         (double*)h->Z.p, c, y, alpha, beta, v, gamma, v2);
    }
    AWG_LAUNCH();
    return AWG_OK;
}

static awg_status dense_gemv(Handle* h, int dim, const double* M, const double* x, double* y,
                             double alpha, const double* sub, double beta, cudaStream_t s) {
    if (dim == 0) return AWG_OK;
    ProfScope ps(h, AWG_PROF_COARSE, s);
    k_dense_gemv<<<(dim + 7) / 8, 256, 0, s>>>(dim, M, x, y, alpha, sub, beta);
    AWG_LAUNCH();
    return AWG_OK;
}

static awg_status hnn1(Handle* h, int prec, const double* x, double* y, Ws& w, cudaStream_t s) {
    dim3 g(h->N, (h->max_ns + LG_ROWS - 1) / LG_ROWS);
    // the bfloat16 and float16 forms keep float32 local operators: the
    // explicit local pseudo-inverses carry cond(A^s_+), which 8 or 11
    // significant bits cannot hold on high-contrast problems; only W (whose
    // accuracy PCG tolerates) is rounded further
    const int gp = (prec == AWG_MIXED_BF16 || prec == AWG_MIXED_FP16) ? AWG_MIXED_FP32 : prec;
    const PrecOps& P = h->prec[gp];
    if (gp == AWG_FP64) {
        {
            ProfScope ps_(h, AWG_PROF_LOCAL, s);
            k_local_gemv64<<<g, 256, (size_t)h->max_ns * 8, s>>>((int*)h->sub_ptr.p, (int*)h->sub_idx.p,
                                                                 (int64_t*)h->dense_off.p,
                                                                 (double*)P.G.p, x, w.loc);
        }
    } else {
        {
            ProfScope ps_(h, AWG_PROF_PROLONG, s);
            k_gather_f32<<<(unsigned)((h->sum_ns + 255) / 256), 256, 0, s>>>(h->sum_ns, (int*)h->sub_idx.p,
                                                                            x, w.xf);
        }
        AWG_LAUNCH();
        {
            ProfScope ps_(h, AWG_PROF_LOCAL, s);
            k_local_gemv_f32<<<g, 256, (size_t)((h->max_ns + 3) & ~3) * 4, s>>>(
                (int*)h->sub_ptr.p, (int64_t*)h->g32_off.p, (float*)P.G.p, w.xf, w.loc);
        }
    }
    AWG_LAUNCH();
    return prolong1(h, w.loc, y, 1.0, 0.0, nullptr, 0.0, s);
}

// c = E^-1 Z^T x
static awg_status coarse_e(Handle* h, const double* x, double* y0, double* c, cudaStream_t s) {
    AWG_TRY(zt1(h, x, y0, s));
    return dense_gemv(h, h->n0, (double*)h->Einv.p, y0, c, 1.0, nullptr, 0.0, s);
}

// H_2 x = Pi H_1 Pi^T x + Z E^-1 Z^T x  (Thm. 4 with H_1 = H^NN; Thm. 3 with
// H_1 = H^AS_+), or H_1 x + Z E^-1 Z^T x (H^AS_+,ad, Thm. 3); H_1 is the
// local solvers the setup built
// z = H_2 r (+ add, once the event `wait` has completed)
static awg_status h2_1(Handle* h, int prec, const double* r, double* z, Ws& w, cudaStream_t s,
                       const double* add = nullptr, cudaEvent_t wait = nullptr) {
    if (h->n0 > 0 && h->opt.h2 == AWG_H2_ASP_AD) {
        AWG_TRY(coarse_e(h, r, w.y0, w.c1, s));  // c1 = E^-1 Z^T r
        AWG_TRY(hnn1(h, prec, r, w.u, w, s));    // u = H_1 r
        if (wait) AWG_CUDA(cudaStreamWaitEvent(s, wait, 0));
        return zc1(h, w.c1, z, 1.0, 0.0, w.u, 1.0, s, add);  // z = u + Z c1 (+ add)
    }
    if (h->n0 == 0) {
        AWG_TRY(hnn1(h, prec, r, z, w, s));
        if (add) {
            if (wait) AWG_CUDA(cudaStreamWaitEvent(s, wait, 0));
            ProfScope ps_(h, AWG_PROF_VECTOR, s);
            k_add<<<(h->n + 255) / 256, 256, 0, s>>>(h->n, add, z);
            AWG_LAUNCH();
        }
        return AWG_OK;
    }
    AWG_TRY(coarse_e(h, r, w.y0, w.c1, s));                 // c1 = E^-1 Z^T r
    AWG_TRY(zc1(h, w.c1, w.x1, 1.0, 0.0, nullptr, 0.0, s));  // x1 = Z c1
    AWG_TRY(aplus1(h, w.x1, w.t, r, -1.0, w, s));           // t = r - A_+ x1
    AWG_TRY(hnn1(h, prec, w.t, w.u, w, s));                 // u = H^NN t
    AWG_TRY(aplus1(h, w.u, w.q, nullptr, 1.0, w, s));        // q = A_+ u
    AWG_TRY(zt1(h, w.q, w.y2, s));
    AWG_TRY(dense_gemv(h, h->n0, (double*)h->Einv.p, w.y2, w.c2, 1.0, w.c1, -1.0, s));  // c2 = E^-1 y2 - c1
    if (wait) AWG_CUDA(cudaStreamWaitEvent(s, wait, 0));
    return zc1(h, w.c2, z, -1.0, 0.0, w.u, 1.0, s, add);    // z = u - Z (c2 - c1) (+ add)
}

// Row blocks of the W^T r pass: about 3 blocks per SM in total over the
// 256-column chunks (the pass shares the GPU with the H_2 chain), at most
// 8192 rows per block (its r values sit in shared memory), never more blocks
// than the partial buffer holds.
static int wt_row_blocks(const Handle* h, const PrecOps& P) {
    const int chunks = (h->ldw + WT_CW - 1) / WT_CW;
    int rb = std::max(1, (P.wt_blocks > 0 ? P.wt_blocks : 152 * 3) / std::max(1, chunks));
    rb = std::max(rb, (h->n + 8191) / 8192);
    rb = std::min(rb, std::max(1, (h->n + 31) / 32));
    return std::min(rb, h->red_blocks);
}

// Truncated W (float64 form with w_drop_tol > 0): out[j] = sum over the
// kept entries of column j of W(i, j) r(i) (CSC; one warp per column, lanes
// over the entries, a fixed-order warp sum)
__global__ void __launch_bounds__(256) k_wt_csc(int nm, const int64_t* __restrict__ colptr,
                                                const int* __restrict__ row, const double* __restrict__ val,
                                                const double* __restrict__ r, double* __restrict__ out) {
    const int j = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= nm) return;
    double a = 0.0;
    for (int64_t k = colptr[j] + lane; k < colptr[j + 1]; k += 32) a = fma(val[k], r[row[k]], a);
    a = warp_sum(a);
    if (lane == 0) out[j] = a;
}

// z(i) = v(i) + sum over the kept entries of row i of W(i, j) d(j) (CSR; one
// warp per row)
__global__ void __launch_bounds__(256) k_wd_csr(int n, const int64_t* __restrict__ rowptr,
                                                const int* __restrict__ col, const double* __restrict__ val,
                                                const double* __restrict__ d, const double* __restrict__ v,
                                                double* __restrict__ z) {
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= n) return;
    double a = 0.0;
    for (int64_t k = rowptr[i] + lane; k < rowptr[i + 1]; k += 32) a = fma(val[k], d[col[k]], a);
    a = warp_sum(a);
    if (lane == 0) z[i] = (v ? v[i] : 0.0) + a;
}

template <typename TS>
static awg_status wt_r_t(Handle* h, const PrecOps& P, const double* r, double* out, Ws& w,
                         cudaStream_t s) {
    const void* W = P.W.p;
    const float* rsc = (const float*)P.rscale.p;
    const float* csc = (const float*)P.cscale.p;
    using A = typename Vec<TS>::A;
    const int rb = wt_row_blocks(h, P);
    const int rows = (h->n + rb - 1) / rb;
    const dim3 grid(rb, (h->ldw + WT_CW - 1) / WT_CW);
    const size_t smem = (size_t)(8 * WT_CW + rows) * sizeof(A);
    {
        ProfScope ps_(h, AWG_PROF_WT, s);
        k_wt_partial<TS><<<grid, WT_THREADS, smem, s>>>(h->n, h->ldw, rows, (const TS*)W, r, rsc, w.wpart,
                                                        P.corr_nnz > 0 ? w.rf : nullptr);
    }
    AWG_LAUNCH();
    {
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        if (P.corr_nnz > 0)
            k_reduce_cols_corr<<<h->n_minus, 256, 0, s>>>(rb, h->ldw, w.wpart, csc, (int*)P.corr_colptr.p,
                                                          (int*)P.corr_row.p, (float*)P.corr_cval.p, w.rf, out);
        else
            k_reduce_cols<<<(h->n_minus + 255) / 256, 256, 0, s>>>(rb, h->n_minus, h->ldw, w.wpart, csc, out);
    }
    AWG_LAUNCH();
    return AWG_OK;
}

static awg_status wt_r(Handle* h, int prec, const double* r, double* out, Ws& w, cudaStream_t s) {
    const PrecOps& P = h->prec[prec];
    if (prec == AWG_FP64 && !P.W.p && P.sp_colptr.p) {  // truncated W
        ProfScope ps_(h, AWG_PROF_WT, s);
        k_wt_csc<<<(h->n_minus + 7) / 8, 256, 0, s>>>(h->n_minus, (const int64_t*)P.sp_colptr.p, (const int*)P.sp_row.p,
                                                      (const double*)P.sp_cval.p, r, out);
        AWG_LAUNCH();
        return AWG_OK;
    }
    if (prec == AWG_FP64) return wt_r_t<double>(h, P, r, out, w, s);
    if (prec == AWG_MIXED_FP32) return wt_r_t<float>(h, P, r, out, w, s);
    if (prec == AWG_MIXED_FP16) return wt_r_t<__half>(h, P, r, out, w, s);
    return wt_r_t<__nv_bfloat16>(h, P, r, out, w, s);
}

// d zero-padded to ldw in the compute type of W's storage
__global__ void k_d_pad64(int nm, int ldw, const double* __restrict__ d, double* dp) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ldw) dp[c] = (c < nm) ? d[c] : 0.0;
}

static awg_status w_d(Handle* h, int prec, const double* d, const double* v, double* z, Ws& w,
                      cudaStream_t s) {
    const PrecOps& P = h->prec[prec];
    const void* W = P.W.p;
    // 8 rows (warps) per block, grid-stride; the pass runs after H_2 has
    // issued its bandwidth-heavy part, so it takes the whole GPU
    const int grid = std::max(1, std::min((h->n + 7) / 8, P.wd_blocks > 0 ? P.wd_blocks : 152 * 16));
    const int gd = (h->ldw + 255) / 256;
    if (prec == AWG_FP64 && !W && P.sp_rowptr.p) {  // truncated W
        ProfScope ps_(h, AWG_PROF_WD, s);
        k_wd_csr<<<(h->n + 7) / 8, 256, 0, s>>>(h->n, (const int64_t*)P.sp_rowptr.p, (const int*)P.sp_col.p,
                                                (const double*)P.sp_val.p, d, v, z);
        AWG_LAUNCH();
        return AWG_OK;
    }
    if (prec == AWG_FP64) {
        double* dp = w.dpad;
        {
            ProfScope ps_(h, AWG_PROF_VECTOR, s);
            k_d_pad64<<<gd, 256, 0, s>>>(h->n_minus, h->ldw, d, dp);
        }
        AWG_LAUNCH();
        ProfScope ps_(h, AWG_PROF_WD, s);
        k_w_d<double><<<grid, 256, (size_t)h->ldw * 8, s>>>(h->n, h->ldw, (const double*)W, dp, nullptr, nullptr,
                                                            nullptr, nullptr, v, z);
    } else {
        const float* rsc = (const float*)P.rscale.p;
        {
            ProfScope ps_(h, AWG_PROF_VECTOR, s);
            k_d_to_f32<<<gd, 256, 0, s>>>(h->n_minus, h->ldw, d, (const float*)P.cscale.p, w.d32);
        }
        AWG_LAUNCH();
        ProfScope ps_(h, AWG_PROF_WD, s);
        const size_t sm = (size_t)h->ldw * 4;
        const bool cor = P.corr_nnz > 0;
        const int* crp = cor ? (const int*)P.corr_rowptr.p : nullptr;
        const int* ccol = cor ? (const int*)P.corr_col.p : nullptr;
        const float* cval = cor ? (const float*)P.corr_val.p : nullptr;
        if (prec == AWG_MIXED_FP32)
            k_w_d<float><<<grid, 256, sm, s>>>(h->n, h->ldw, (const float*)W, w.d32, rsc, crp, ccol, cval, v, z);
        else if (prec == AWG_MIXED_FP16)
            k_w_d<__half><<<grid, 256, sm, s>>>(h->n, h->ldw, (const __half*)W, w.d32, rsc, crp, ccol, cval, v, z);
        else
            k_w_d<__nv_bfloat16><<<grid, 256, sm, s>>>(h->n, h->ldw, (const __nv_bfloat16*)W, w.d32, rsc, crp,
                                                       ccol, cval, v, z);
    }
    AWG_LAUNCH();
    return AWG_OK;
}

awg_status set_smem_limits(Handle* h) {
    const int mx = (int)std::max<size_t>((size_t)h->max_ns * 8, (size_t)std::max(1, h->ldw) * 8);
    if (mx > 48 * 1024) {
        if (mx > 227 * 1024) return AWG_ERR_INVALID_ARG;
        AWG_CUDA(cudaFuncSetAttribute(k_local_gemv64, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        AWG_CUDA(cudaFuncSetAttribute(k_local_gemv_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        AWG_CUDA(cudaFuncSetAttribute(k_w_d<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        AWG_CUDA(cudaFuncSetAttribute(k_w_d<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        AWG_CUDA(cudaFuncSetAttribute(k_w_d<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        AWG_CUDA(cudaFuncSetAttribute(k_w_d<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    }
    // W^T r stages up to 8192 values of r plus 8 x 256 partial sums
    const int wt = (8 * WT_CW + 8192) * 8;
    AWG_CUDA(cudaFuncSetAttribute(k_wt_partial<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, wt));
    AWG_CUDA(cudaFuncSetAttribute(k_wt_partial<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, wt / 2));
    AWG_CUDA(cudaFuncSetAttribute(k_wt_partial<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, wt / 2));
    AWG_CUDA(cudaFuncSetAttribute(k_wt_partial<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, wt / 2));
    return AWG_OK;
}

// One single-RHS apply of the selected stage (see awg_apply_stage).
awg_status apply_stage(Handle* h, int which, int prec, const double* x, double* y, cudaStream_t s) {
    if (prec < 0 || prec >= AWG_NPREC || !h->prec[prec].built) return AWG_ERR_INVALID_ARG;
    Ws w = ws_of(h);
    switch (which) {
        case 0: return spmv1(h, x, y, nullptr, s);
        case 1: return aplus1(h, x, y, nullptr, 1.0, w, s);
        case 2: return hnn1(h, prec, x, y, w, s);
        case 3: return h2_1(h, prec, x, y, w, s);
        case 4: {  // H_3,ad = H_2 + W F^-1 W^T  (Def. 10)
            if (h->n_minus == 0) return h2_1(h, prec, x, y, w, s);
            // W F^-1 W^T x on the side stream while H_2 x runs on s; the two
            // meet in the last kernel of H_2
            const cudaStream_t side = side_stream(h, h->side, s);
            AWG_CUDA(cudaEventRecord(h->ev_fork, s));
            AWG_CUDA(cudaStreamWaitEvent(side, h->ev_fork, 0));
            AWG_TRY(wt_r(h, prec, x, w.w0, w, side));
            AWG_TRY(dense_gemv(h, h->n_minus, (double*)h->prec[prec].Finv.p, w.w0, w.dd, 1.0, nullptr, 0,
                               side));
            AWG_TRY(w_d(h, prec, w.dd, nullptr, w.tmp2, w, side));
            AWG_CUDA(cudaEventRecord(h->ev_join, side));
            return h2_1(h, prec, x, y, w, s, w.tmp2, h->ev_join);
        }
        case 5: {  // H_3,hyb = Pi_3 H_2 Pi_3^T + W F^-1 W^T  (Def. 10)
            if (h->n_minus == 0) return h2_1(h, prec, x, y, w, s);
            const double* Finv = (double*)h->prec[prec].Finv.p;
            AWG_TRY(wt_r(h, prec, x, w.w0, w, s));
            AWG_TRY(dense_gemv(h, h->n_minus, Finv, w.w0, w.dd, 1.0, nullptr, 0, s));  // d = F^-1 W^T x
            AWG_TRY(w_d(h, prec, w.dd, nullptr, w.tmp, w, s));                        // tmp = W d
            AWG_TRY(spmv1(h, w.tmp, w.q, nullptr, s));
            {
                ProfScope ps_(h, AWG_PROF_VECTOR, s);
                k_sub<<<(h->n + 255) / 256, 256, 0, s>>>(h->n, x, w.q, w.tmp);
            }        // tmp = Pi_3^T x
            AWG_LAUNCH();
            AWG_TRY(h2_1(h, prec, w.tmp, y, w, s));                                // y = v = H_2 Pi_3^T x
            AWG_TRY(spmv1(h, y, w.q, nullptr, s));                                 // q = A v
            AWG_TRY(wt_r(h, prec, w.q, w.w0, w, s));
            AWG_TRY(dense_gemv(h, h->n_minus, Finv, w.w0, w.w1, -1.0, w.dd, 1.0, s)); // w1 = d - F^-1 W^T A v
            return w_d(h, prec, w.w1, y, y, w, s);                                     // z = v + W w1
        }
        case 6: {  // H_3,inex = H_2 + W (C^-1 - Vhat^T W)^-1 W^T  (Thm. 7)
            if (h->n_minus == 0) return h2_1(h, prec, x, y, w, s);
            const cudaStream_t side = side_stream(h, h->side, s);
            AWG_CUDA(cudaEventRecord(h->ev_fork, s));
            AWG_CUDA(cudaStreamWaitEvent(side, h->ev_fork, 0));
            AWG_TRY(wt_r(h, prec, x, w.w0, w, side));
            AWG_TRY(dense_gemv(h, h->n_minus, (double*)h->prec[prec].inexInv.p, w.w0, w.dd, 1.0, nullptr,
                               0, side));
            AWG_TRY(w_d(h, prec, w.dd, nullptr, w.tmp2, w, side));
            AWG_CUDA(cudaEventRecord(h->ev_join, side));
            return h2_1(h, prec, x, y, w, s, w.tmp2, h->ev_join);
        }
        default: return AWG_ERR_INVALID_ARG;
    }
}

// ------------------------------------------------------------- autotuner
__global__ void k_fill_unit(int n, double* x) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t v = (uint32_t)i * 0x9e3779b1u + 0x7f4a7c15u;
    v ^= v >> 15; v *= 0x2c1b3c6du; v ^= v >> 12; v *= 0x297a2d39u; v ^= v >> 15;
    x[i] = (double)(v & 0xffffff) / 16777216.0 - 0.5;
}

awg_status autotune_apply(Handle* h) {
    if (h->n_minus == 0) return AWG_OK;
    cudaStream_t s = h->hp;
    double *x = nullptr, *y = nullptr;
    AWG_CUDA(cudaMallocAsync(&x, (size_t)h->n * 8, s));
    AWG_CUDA(cudaMallocAsync(&y, (size_t)h->n * 8, s));
    k_fill_unit<<<(h->n + 255) / 256, 256, 0, s>>>(h->n, x);
    AWG_LAUNCH();
    cudaEvent_t e0, e1;
    AWG_CUDA(cudaEventCreate(&e0));
    AWG_CUDA(cudaEventCreate(&e1));
    const int stage = 4 + h->opt.variant;
    auto timed = [&](int p, float* ms) -> awg_status {
        AWG_TRY(apply_stage(h, stage, p, x, y, s));
        AWG_CUDA(cudaEventRecord(e0, s));
        for (int k = 0; k < 3; k++) AWG_TRY(apply_stage(h, stage, p, x, y, s));
        AWG_CUDA(cudaEventRecord(e1, s));
        AWG_CUDA(cudaEventSynchronize(e1));
        AWG_CUDA(cudaEventElapsedTime(ms, e0, e1));
        return AWG_OK;
    };
    awg_status st = AWG_OK;
    for (int p = 0; p < AWG_NPREC && st == AWG_OK; p++) {
        PrecOps& P = h->prec[p];
        if (!P.built) continue;
        const int wt_c[] = {2, 3, 4, 6, 8}, wd_c[] = {4, 8, 16};
        float best = 1e30f;
        int bwt = 152 * 3, bwd = 152 * 16;
        P.wd_blocks = bwd;
        for (int c : wt_c) {
            P.wt_blocks = 152 * c;
            float ms = 0.f;
            if ((st = timed(p, &ms)) != AWG_OK) break;
            if (ms < best) { best = ms; bwt = P.wt_blocks; }
        }
        P.wt_blocks = bwt;
        for (int c : wd_c) {
            if (st != AWG_OK) break;
            P.wd_blocks = 152 * c;
            float ms = 0.f;
            if ((st = timed(p, &ms)) != AWG_OK) break;
            if (ms < best) { best = ms; bwd = P.wd_blocks; }
        }
        P.wd_blocks = bwd;
        if (h->opt.verbose)
            fprintf(stderr, "libawg: autotune form %d: W^T r %d blocks, W d %d blocks, apply %.3f ms\n", p,
                    P.wt_blocks, P.wd_blocks, best / 3.0f);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    AWG_CUDA(cudaFreeAsync(x, s));
    AWG_CUDA(cudaFreeAsync(y, s));
    AWG_CUDA(cudaStreamSynchronize(s));
    return st;
}

// ------------------------------------------------------------------- PCG
static awg_status dot1(Handle* h, const double* x, const double* y, double* out, Ws& w,
                       cudaStream_t s) {
    ProfScope ps_(h, AWG_PROF_VECTOR, s);
    k_dot<<<grid_n(h->n), 256, 0, s>>>(h->n, x, y, w.part, w.cnt, out);
    AWG_LAUNCH();
    return AWG_OK;
}

// q = b - A x
static awg_status resid1(Handle* h, const double* b, const double* x, double* q, cudaStream_t s) {
    ProfScope ps_(h, AWG_PROF_SPMV, s);
    k_aplus_row<<<(h->n + 255) / 256, 256, 0, s>>>(h->n, (int*)h->rowptr.p, (int*)h->colidx.p,
                                                   (double*)h->val.p, x, nullptr, nullptr, nullptr, nullptr,
                                                   nullptr, nullptr, nullptr, nullptr, b, -1.0, q);
    AWG_LAUNCH();
    return AWG_OK;
}

awg_status pcg1(Handle* h, int prec, int variant_stage, const double* b, double* x, double rtol,
                int* iters, double* relres, cudaStream_t s) {
    Ws w = ws_of(h);
    const int n = h->n, nb = grid_n(n);
    // partial buffer (4096 doubles): [0, 1216) holds per-block partials
    // (grid_n <= 1216 blocks), the device scalars live at [4000, 4016), the
    // ticket counters at [4064, 4068)
    double* scal = w.part + 4000;
    double *r, *p, *q, *z;
    AWG_CUDA(cudaMallocAsync(&r, (size_t)n * 8, s));
    AWG_CUDA(cudaMallocAsync(&p, (size_t)n * 8, s));
    AWG_CUDA(cudaMallocAsync(&q, (size_t)n * 8, s));
    AWG_CUDA(cudaMallocAsync(&z, (size_t)n * 8, s));
    AWG_CUDA(cudaMemsetAsync(x, 0, (size_t)n * 8, s));
    AWG_CUDA(cudaMemcpyAsync(r, b, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
    AWG_TRY(dot1(h, b, b, scal + S_BB, w, s));
    AWG_TRY(apply_stage(h, variant_stage, prec, r, z, s));
    AWG_TRY(dot1(h, r, z, scal + S_RZ, w, s));
    AWG_CUDA(cudaMemcpyAsync(p, z, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
    AWG_CUDA(cudaMemcpyAsync(h->h_scal, scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    AWG_CUDA(cudaStreamSynchronize(s));
    const double bnorm = sqrt(h->h_scal[S_BB]);
    awg_status st = AWG_OK;
    int it = 0;
    double rel = (bnorm > 0) ? 1.0 : 0.0, true_rel = rel;
    if (bnorm == 0.0) {
        it = 0;
    } else {
        const int maxit = h->opt.maxit;
        bool done = false;
        while (!done) {
            if (it >= maxit) { st = AWG_ERR_MAXIT; break; }
            AWG_TRY(spmv1(h, p, q, scal + S_PQ, s));                  // q = A p, p.q
            {
                ProfScope ps_(h, AWG_PROF_VECTOR, s);
                k_pcg_xr<<<nb, 256, 0, s>>>(n, scal, p, q, x, r, w.part, w.cnt);  // x, r, r.r
            }
            AWG_LAUNCH();
            it++;
            AWG_CUDA(cudaMemcpyAsync(h->h_scal, scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
            AWG_CUDA(cudaStreamSynchronize(s));
            const double pq = h->h_scal[S_PQ];
            if (!(pq > 0.0) || !std::isfinite(pq)) { st = AWG_ERR_BREAKDOWN; break; }
            rel = sqrt(h->h_scal[S_RR]) / bnorm;
            if (rel <= rtol) {
                // confirm on the true residual b - A x
                AWG_TRY(resid1(h, b, x, q, s));
                AWG_TRY(dot1(h, q, q, scal + S_TR, w, s));
                AWG_CUDA(cudaMemcpyAsync(h->h_scal, scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
                AWG_CUDA(cudaStreamSynchronize(s));
                true_rel = sqrt(h->h_scal[S_TR]) / bnorm;
                if (true_rel <= rtol || rel <= 1e-6 * rtol) {
                    if (true_rel > rtol) st = AWG_ERR_MAXIT;
                    break;
                }
            }
            AWG_TRY(apply_stage(h, variant_stage, prec, r, z, s));
            AWG_TRY(dot1(h, r, z, scal + S_RZN, w, s));
            {
                ProfScope ps_(h, AWG_PROF_VECTOR, s);
                k_pcg_p<<<nb, 256, 0, s>>>(n, scal, z, p, w.cnt);  // beta, p, rz <- rz_new
            }
            AWG_LAUNCH();
        }
    }
    if (st != AWG_OK || true_rel == rel) {
        AWG_TRY(resid1(h, b, x, q, s));
        AWG_TRY(dot1(h, q, q, scal + S_TR, w, s));
        AWG_CUDA(cudaMemcpyAsync(h->h_scal, scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
        AWG_CUDA(cudaStreamSynchronize(s));
        true_rel = bnorm > 0 ? sqrt(h->h_scal[S_TR]) / bnorm : 0.0;
    }
    for (double* ptr : {r, p, q, z}) AWG_CUDA(cudaFreeAsync(ptr, s));
    AWG_CUDA(cudaStreamSynchronize(s));
    if (iters) *iters = it;
    if (relres) *relres = true_rel;
    return st;
}

// ------------------------------------------------- graph-driven PCG, one RHS
// Control words next to the PCG scalars: [8] iterations done, [9] rtol,
// [10] maxit, [11] status, [12] active (1/0), [13] relative residual and
// [14] iterations at exit, [15] candidate (recurrence residual at rtol, true
// residual to be confirmed in this iteration).
enum { C_IT = 8, C_RTOL = 9, C_MAXIT = 10, C_ST = 11, C_ACT = 12, C_REL = 13, C_ITS = 14, C_CAND = 15 };

// q = b - A x, only when *gate is not 0
__global__ void __launch_bounds__(256) k_resid1(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                const double* __restrict__ a, const double* __restrict__ b,
                                                const double* __restrict__ x, double* __restrict__ q,
                                                const double* gate) {
    if (*gate == 0.0) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double acc = 0.0;
        const int e = rp[i + 1];
        for (int k = rp[i]; k < e; k++) acc = fma(a[k], x[ci[k]], acc);
        q[i] = b[i] - acc;
    }
}

__global__ void k_pcg1_init(double* scal, double rtol, double maxit) {
    if (threadIdx.x == 0) {
        scal[C_IT] = 0.0;
        scal[C_RTOL] = rtol;
        scal[C_MAXIT] = maxit;
        scal[C_ST] = 0.0;
        scal[C_ACT] = scal[S_BB] > 0.0 ? 1.0 : 0.0;
        scal[C_REL] = 0.0;
        scal[C_ITS] = 0.0;
        scal[C_CAND] = 0.0;
    }
}

// after an x, r update: stop on breakdown or the iteration cap; a
// recurrence residual <= rtol ||b|| makes the iteration a candidate, whose
// true residual (k_resid1, k_dot gated by C_CAND) k_pcg1_confirm checks
__global__ void k_pcg1_cond(double* scal) {
    if (threadIdx.x != 0) return;
    scal[C_CAND] = 0.0;
    if (scal[C_ACT] != 0.0) {
        const int it = (int)scal[C_IT] + 1;
        scal[C_IT] = it;
        const double pq = scal[S_PQ];
        const double rel = sqrt(scal[S_RR] / scal[S_BB]);
        scal[C_REL] = rel;
        scal[C_ITS] = it;
        if (!(pq > 0.0) || !isfinite(pq)) {
            scal[C_ST] = AWG_ERR_BREAKDOWN;
            scal[C_ACT] = 0.0;
        } else if (rel <= scal[C_RTOL]) {
            scal[C_CAND] = 1.0;
        } else if (it >= (int)scal[C_MAXIT]) {
            scal[C_ST] = AWG_ERR_MAXIT;
            scal[C_ACT] = 0.0;
        }
    }
}

// a candidate stops once its true relative residual is <= rtol (reported
// as the residual at exit), or its recurrence residual fell below 1e-6 rtol
// (stagnation: AWG_ERR_MAXIT); with `set`, the loop condition
__global__ void k_pcg1_confirm(double* scal, cudaGraphConditionalHandle hc, int set, unsigned long long* launches,
                               int add) {
    if (threadIdx.x != 0) return;
    if (scal[C_ACT] != 0.0 && scal[C_CAND] != 0.0) {
        const double rtol = scal[C_RTOL];
        const double tr = sqrt(scal[S_TR] / scal[S_BB]);
        if (tr <= rtol || scal[C_REL] <= 1e-6 * rtol) {
            if (tr > rtol) scal[C_ST] = AWG_ERR_MAXIT;
            scal[C_ACT] = 0.0;
            scal[C_REL] = tr;
        } else if ((int)scal[C_IT] >= (int)scal[C_MAXIT]) {
            scal[C_ST] = AWG_ERR_MAXIT;
            scal[C_ACT] = 0.0;
            scal[C_REL] = tr;
        }
        scal[C_CAND] = 0.0;
    }
    if (set) cudaGraphSetConditional(hc, scal[C_ACT] != 0.0 ? 1u : 0u);
    if (launches && add) atomicAdd(launches, (unsigned long long)add);
}

__global__ void k_pcg1_fini(const double* scal, int* d_it, double* d_rel, int* d_st) {
    if (threadIdx.x != 0) return;
    if (d_it) *d_it = (int)scal[C_ITS];
    if (d_rel) *d_rel = scal[C_REL];
    if (d_st) *d_st = (int)scal[C_ST];
}

namespace {
struct G1 {
    double *b, *x, *r, *p, *q, *z;
};
G1 g1_of(Handle* h) {
    double* base = (double*)h->g1buf.p;
    const size_t n = (size_t)h->n;
    return {base, base + n, base + 2 * n, base + 3 * n, base + 4 * n, base + 5 * n};
}

// stopping test after an x, r update: candidate, then (gated on it) the
// true residual q = b - A x and its norm, then the confirmation
awg_status pcg1_stop(Handle* h, const G1& g, double* scal, Ws& w, cudaStream_t s, cudaGraphConditionalHandle hc,
                     int set, unsigned long long* launches, int add) {
    const int n = h->n;
    {
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        k_pcg1_cond<<<1, 32, 0, s>>>(scal);
        AWG_LAUNCH();
    }
    {
        ProfScope ps_(h, AWG_PROF_SPMV, s);
        k_resid1<<<(n + 255) / 256, 256, 0, s>>>(n, (int*)h->rowptr.p, (int*)h->colidx.p, (double*)h->val.p, g.b,
                                                 g.x, g.q, scal + C_CAND);
        AWG_LAUNCH();
    }
    {
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        k_dot<<<grid_n(n), 256, 0, s>>>(n, g.q, g.q, w.part, w.cnt, scal + S_TR, scal + C_CAND);
        AWG_LAUNCH();
    }
    ProfScope ps_(h, AWG_PROF_VECTOR, s);
    k_pcg1_confirm<<<1, 32, 0, s>>>(scal, hc, set, launches, add);
    AWG_LAUNCH();
    return AWG_OK;
}

// one iteration: z = H r, rz_new, p = z + beta p, q = A p (p.q), x, r (r.r), stop test
awg_status pcg1_body(Handle* h, int prec, int stage, const G1& g, double* scal, Ws& w, cudaStream_t s,
                     cudaGraphConditionalHandle hc, int set, unsigned long long* launches, int add) {
    const int n = h->n, nb = grid_n(n);
    AWG_TRY(apply_stage(h, stage, prec, g.r, g.z, s));
    AWG_TRY(dot1(h, g.r, g.z, scal + S_RZN, w, s));
    {
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        k_pcg_p<<<nb, 256, 0, s>>>(n, scal, g.z, g.p, w.cnt);
    }
    AWG_LAUNCH();
    AWG_TRY(spmv1(h, g.p, g.q, scal + S_PQ, s));
    {
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        k_pcg_xr<<<nb, 256, 0, s>>>(n, scal, g.p, g.q, g.x, g.r, w.part, w.cnt);
    }
    AWG_LAUNCH();
    return pcg1_stop(h, g, scal, w, s, hc, set, launches, add);
}
}  // namespace

awg_status pcg1_async(Handle* h, int prec, int stage, const double* b, double* x, double rtol, int* d_it,
                      double* d_rel, int* d_st, cudaStream_t s) {
    Ws w = ws_of(h);
    const int n = h->n, nb = grid_n(n);
    if (!h->g1buf.p) AWG_TRY(dalloc(h, h->g1buf, (size_t)n * 6 * 8));
    if (!h->g1cnt.p) {
        AWG_TRY(dalloc(h, h->g1cnt, 8));
        AWG_CUDA(cudaMemset(h->g1cnt.p, 0, 8));
    }
    const G1 g = g1_of(h);
    double* scal = w.part + 4000;
    unsigned long long* gl = (unsigned long long*)h->g1cnt.p;
    AWG_CUDA(cudaMemcpyAsync(g.b, b, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
    AWG_CUDA(cudaMemsetAsync(g.x, 0, (size_t)n * 8, s));
    AWG_CUDA(cudaMemcpyAsync(g.r, g.b, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
    AWG_TRY(dot1(h, g.b, g.b, scal + S_BB, w, s));
    {
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        k_pcg1_init<<<1, 32, 0, s>>>(scal, rtol, (double)h->opt.maxit);
    }
    AWG_LAUNCH();
    // first iteration: z = H r, rz, p = z, q = A p, x, r
    AWG_TRY(apply_stage(h, stage, prec, g.r, g.z, s));
    AWG_TRY(dot1(h, g.r, g.z, scal + S_RZ, w, s));
    AWG_CUDA(cudaMemcpyAsync(g.p, g.z, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
    AWG_TRY(spmv1(h, g.p, g.q, scal + S_PQ, s));
    {
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        k_pcg_xr<<<nb, 256, 0, s>>>(n, scal, g.p, g.q, g.x, g.r, w.part, w.cnt);
    }
    AWG_LAUNCH();
    AWG_TRY(pcg1_stop(h, g, scal, w, s, 0, 0, nullptr, 0));
    // the loop graph of this precision (captured once, after the first
    // iteration has been issued)
    if (!h->g1_exec[prec]) {
        cudaGraph_t gr = nullptr;
        AWG_CUDA(cudaGraphCreate(&gr, 0));
        cudaGraphConditionalHandle hc;
        AWG_CUDA(cudaGraphConditionalHandleCreate(&hc, gr, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = hc;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        AWG_CUDA(cudaGraphAddNode(&node, gr, nullptr, nullptr, 0, &np));
        cudaGraph_t body = np.conditional.phGraph_out[0];
        const int prof = h->prof;
        const int64_t l0 = h->launches;
        h->prof = 1 << 30;  // count, do not time, while capturing
        // one body to count its kernels, then the captured one with that count
        AWG_CUDA(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        awg_status st = pcg1_body(h, prec, stage, g, scal, w, s, hc, 1, gl, 0);
        cudaGraph_t cap = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(s, &cap);
        const int add = (int)(h->launches - l0);
        h->prof = prof;
        h->launches = l0;
        if (st != AWG_OK || ce != cudaSuccess) {
            cudaGetLastError();
            cudaGraphDestroy(gr);
            return st != AWG_OK ? st : AWG_ERR_CUDA;
        }
        size_t nn = 0;
        AWG_CUDA(cudaGraphGetNodes(body, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        AWG_CUDA(cudaGraphGetNodes(body, nodes.data(), &nn));
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType t;
            AWG_CUDA(cudaGraphNodeGetType(nd, &t));
            if (t != cudaGraphNodeTypeKernel) continue;
            cudaKernelNodeParams kp;
            AWG_CUDA(cudaGraphKernelNodeGetParams(nd, &kp));
            if (kp.func != (void*)k_pcg1_confirm) continue;
            *(int*)kp.kernelParams[4] = add;
            AWG_CUDA(cudaGraphKernelNodeSetParams(nd, &kp));
        }
        cudaGraphExec_t ex = nullptr;
        AWG_CUDA(cudaGraphInstantiate(&ex, gr, cudaGraphInstantiateFlagUseNodePriority));
        h->g1_graph[prec] = gr;
        h->g1_exec[prec] = ex;
    }
    AWG_CUDA(cudaGraphLaunch(h->g1_exec[prec], s));
    AWG_CUDA(cudaMemcpyAsync(x, g.x, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
    ProfScope ps_(h, AWG_PROF_VECTOR, s);
    k_pcg1_fini<<<1, 32, 0, s>>>(scal, d_it, d_rel, d_st);
    AWG_LAUNCH();
    return AWG_OK;
}

// kernels launched by single-RHS graph loop bodies since the last call (reset)
int64_t pcg1_graph_launches(Handle* h) {
    if (!h->g1cnt.p) return 0;
    unsigned long long c = 0;
    if (cudaMemcpy(&c, h->g1cnt.p, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return 0;
    cudaMemset(h->g1cnt.p, 0, 8);
    return (int64_t)c;
}

}  // namespace awg
