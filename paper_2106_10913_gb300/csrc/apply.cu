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

namespace awg {

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}

// ------------------------------------------------------------------ SpMV
// y = A x; if pdot, also writes per-block partials of x^T y (fixed order).
__global__ void __launch_bounds__(256) k_spmv(int n, const int* __restrict__ rp,
                                              const int* __restrict__ ci,
                                              const double* __restrict__ a,
                                              const double* __restrict__ x, double* __restrict__ y,
                                              double* pdot) {
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
        if (threadIdx.x == 0) pdot[blockIdx.x] = part;
    }
}

// -------------------------------------------------------- block-sparse ops
// c[colptr[s] + j] = sum_p B_s(p, j) x(idx_s(p)),  B_s column-major n^s x cols
__global__ void __launch_bounds__(256) k_blk_tgemv(const int* __restrict__ sub_ptr,
                                                   const int* __restrict__ sub_idx,
                                                   const int* __restrict__ colptr,
                                                   const int64_t* __restrict__ boff,
                                                   const double* __restrict__ B,
                                                   const double* __restrict__ x, double* c) {
    extern __shared__ double xs[];
    const int s = blockIdx.x;
    const int p0 = sub_ptr[s], m = sub_ptr[s + 1] - p0;
    const int c0 = colptr[s], nc = colptr[s + 1] - c0;
    if (nc == 0) return;
    for (int p = threadIdx.x; p < m; p += blockDim.x) xs[p] = x[sub_idx[p0 + p]];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double* Bs = B + boff[s];
    for (int j = wid; j < nc; j += nw) {
        const double* col = Bs + (size_t)j * m;
        double acc = 0.0;
        for (int p = lane; p < m; p += 32) acc = fma(col[p], xs[p], acc);
        acc = warp_sum(acc);
        if (lane == 0) c[c0 + j] = acc;
    }
}

// loc[sub_ptr[s] + p] = sum_j B_s(p, j) w_j c_j   (w optional)
__global__ void __launch_bounds__(256) k_blk_gemv(const int* __restrict__ sub_ptr,
                                                  const int* __restrict__ colptr,
                                                  const int64_t* __restrict__ boff,
                                                  const double* __restrict__ B,
                                                  const double* __restrict__ c,
                                                  const double* __restrict__ w, double wsign,
                                                  double* loc) {
    extern __shared__ double cs[];
    const int s = blockIdx.x;
    const int p0 = sub_ptr[s], m = sub_ptr[s + 1] - p0;
    const int c0 = colptr[s], nc = colptr[s + 1] - c0;
    for (int j = threadIdx.x; j < nc; j += blockDim.x) cs[j] = w ? wsign * w[c0 + j] * c[c0 + j] : c[c0 + j];
    __syncthreads();
    const double* Bs = B + boff[s];
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < nc; j++) acc = fma(Bs[p + (size_t)j * m], cs[j], acc);
        loc[p0 + p] = acc;
    }
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
                                                           double* part) {
    using A = typename Vec<TS>::A;
    constexpr int V = Vec<TS>::V;
    constexpr int UNR = WT_CW / (32 * V);
    extern __shared__ __align__(16) unsigned char wt_smem[];
    A* red = reinterpret_cast<A*>(wt_smem);  // [8][WT_CW]
    A* rs = red + 8 * WT_CW;                 // [rows]
    const int i0 = blockIdx.x * rows;
    const int nr = min(n, i0 + rows) - i0;
    const int c0 = blockIdx.y * WT_CW;
    if (rscale)
        for (int t = threadIdx.x; t < nr; t += WT_THREADS) rs[t] = (A)r[i0 + t] * rscale[i0 + t];
    else
        for (int t = threadIdx.x; t < nr; t += WT_THREADS) rs[t] = (A)r[i0 + t];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    A acc[UNR][V];
#pragma unroll
    for (int u = 0; u < UNR; u++)
#pragma unroll
        for (int j = 0; j < V; j++) acc[u][j] = 0;
#pragma unroll 2
    for (int i = wid; i < nr; i += 8) {
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
                                             const float* __restrict__ rscale, const double* v,
                                             double* z) {
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
        A acc0 = 0, acc1 = 0;
        int c = lane * V;
        for (; c + 32 * V < ldw; c += 64 * V) {
            A w0[V], w1[V], d0[V], d1[V];
            Vec<TS>::load(row + c, w0);
            Vec<TS>::load(row + c + 32 * V, w1);
            lds_vec<A, V>(ds + c, d0);
            lds_vec<A, V>(ds + c + 32 * V, d1);
#pragma unroll
            for (int j = 0; j < V; j++) {
                acc0 = fma(w0[j], d0[j], acc0);
                acc1 = fma(w1[j], d1[j], acc1);
            }
        }
        if (c < ldw) {
            A w0[V], d0[V];
            Vec<TS>::load(row + c, w0);
            lds_vec<A, V>(ds + c, d0);
#pragma unroll
            for (int j = 0; j < V; j++) acc0 = fma(w0[j], d0[j], acc0);
        }
        A s = warp_sum_t<A>(acc0 + acc1);
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

__global__ void k_dot_partial(int n, const double* __restrict__ x, const double* __restrict__ y,
                              double* part) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        acc = fma(x[i], y[i], acc);
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_final_sum(int nb, const double* __restrict__ part, double* out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += part[b];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) *out = acc;
}

// PCG scalars (device): 0 rz, 1 pq, 2 rr, 3 rz_new, 4 beta
enum { S_RZ = 0, S_PQ = 1, S_RR = 2, S_RZN = 3, S_BETA = 4, S_BB = 5, S_TR = 6 };

// x += alpha p, r -= alpha q with alpha = rz / pq; partials of r.r
__global__ void k_pcg_xr(int n, const double* __restrict__ scal, const double* __restrict__ p,
                         const double* __restrict__ q, double* x, double* r, double* part) {
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
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_pcg_beta(double* scal) {
    const double rz = scal[S_RZ], rzn = scal[S_RZN];
    scal[S_BETA] = (rz != 0.0) ? rzn / rz : 0.0;
    scal[S_RZ] = rzn;
}

__global__ void k_pcg_p(int n, const double* __restrict__ scal, const double* __restrict__ z,
                        double* p) {
    const double beta = scal[S_BETA];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], z[i]);
}

// ===================================================================== host
struct Ws {
    double *y0, *y2, *c1, *c2, *w0, *w1, *dd, *x1, *t, *u, *q, *loc, *loc2, *cm, *part, *wpart, *tmp, *tmp2;
    float *xf, *d32;  // float32 gathered local vector, float32 copy of d
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
    t.wpart = take((size_t)h->red_blocks * std::max(8, h->ldw));
    t.xf = reinterpret_cast<float*>(take((h->sum_ns + 1) / 2 + 4));
    t.d32 = reinterpret_cast<float*>(take((std::max(8, h->ldw) + 1) / 2 + 4));
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
    {
        ProfScope ps_(h, AWG_PROF_SPMV, s);
        k_spmv<<<grid_n(h->n), 256, 0, s>>>(h->n, (int*)h->rowptr.p, (int*)h->colidx.p,
                                            (double*)h->val.p, x, y, pdot);
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

// y = A_- x, or y = yin + sign * A_- x
static awg_status aminus1(Handle* h, const double* x, double* y, const double* yin, double sign,
                          Ws& w, cudaStream_t s) {
    if (h->n_minus_all == 0) {
        if (yin) { if (yin != y) AWG_CUDA(cudaMemcpyAsync(y, yin, h->n * 8, cudaMemcpyDeviceToDevice, s)); }
        else AWG_CUDA(cudaMemsetAsync(y, 0, h->n * 8, s));
        return AWG_OK;
    }
    const size_t sm = (size_t)h->max_ns * 8;
    {
        ProfScope ps_(h, AWG_PROF_SUBDOMAIN, s);
        k_blk_tgemv<<<h->N, 256, sm, s>>>((int*)h->sub_ptr.p, (int*)h->sub_idx.p, (int*)h->nm_ptr.p,
                                          (int64_t*)h->vm_off.p, (double*)h->Vm.p, x, w.cm);
    }
    AWG_LAUNCH();
    {
        ProfScope ps_(h, AWG_PROF_SUBDOMAIN, s);
        k_blk_gemv<<<h->N, 256, (size_t)std::max(1, *std::max_element(h->h_nm.begin(), h->h_nm.end())) * 8, s>>>(
            (int*)h->sub_ptr.p, (int*)h->nm_ptr.p, (int64_t*)h->vm_off.p, (double*)h->Vm.p, w.cm,
            (double*)h->lam_m.p, -1.0, w.loc2);
    }
    AWG_LAUNCH();
    return prolong1(h, w.loc2, y, sign, 0.0, yin, 1.0, s);
}

// y = yin + sign * A_+ x
static awg_status aplus1(Handle* h, const double* x, double* y, const double* yin, double sign,
                         Ws& w, cudaStream_t s) {
    AWG_TRY(spmv1(h, x, w.tmp2, nullptr, s));
    // tmp2 = A x ; y = yin + sign*(A x + A_- x)
    if (yin) {
        {
            ProfScope ps_(h, AWG_PROF_VECTOR, s);
            k_sub<<<(h->n + 255) / 256, 256, 0, s>>>(h->n, yin, w.tmp2, w.tmp2);
        }  // yin - A x
        AWG_LAUNCH();
        if (sign != -1.0) return AWG_ERR_INVALID_ARG;
        return aminus1(h, x, y, w.tmp2, -1.0, w, s);
    }
    return aminus1(h, x, y, w.tmp2, sign, w, s);
}

static awg_status zt1(Handle* h, const double* x, double* c, cudaStream_t s) {
    if (h->n0 == 0) return AWG_OK;
    {
        ProfScope ps_(h, AWG_PROF_SUBDOMAIN, s);
        k_blk_tgemv<<<h->N, 256, (size_t)h->max_ns * 8, s>>>((int*)h->sub_ptr.p, (int*)h->sub_idx.p,
                                                            (int*)h->mode_ptr.p, (int64_t*)h->z_off.p,
                                                            (double*)h->Z.p, x, c);
    }
    AWG_LAUNCH();
    return AWG_OK;
}

// loc = Z c (local slabs)
static awg_status zloc1(Handle* h, const double* c, double* loc, cudaStream_t s) {
    const int mx = std::max(1, *std::max_element(h->h_modes.begin(), h->h_modes.end()));
    {
        ProfScope ps_(h, AWG_PROF_SUBDOMAIN, s);
        k_blk_gemv<<<h->N, 256, (size_t)mx * 8, s>>>((int*)h->sub_ptr.p, (int*)h->mode_ptr.p,
                                                     (int64_t*)h->z_off.p, (double*)h->Z.p, c,
                                                     nullptr, 1.0, loc);
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

// H_2 x = Pi H^NN Pi^T x + Z E^-1 Z^T x  (Thm. 4)
static awg_status h2_1(Handle* h, int prec, const double* r, double* z, Ws& w, cudaStream_t s) {
    if (h->n0 == 0) return hnn1(h, prec, r, z, w, s);
    AWG_TRY(coarse_e(h, r, w.y0, w.c1, s));                 // c1 = E^-1 Z^T r
    AWG_TRY(zloc1(h, w.c1, w.loc, s));
    AWG_TRY(prolong1(h, w.loc, w.x1, 1.0, 0.0, nullptr, 0.0, s));  // x1 = Z c1
    AWG_TRY(aplus1(h, w.x1, w.t, r, -1.0, w, s));           // t = r - A_+ x1
    AWG_TRY(hnn1(h, prec, w.t, w.u, w, s));                 // u = H^NN t
    AWG_TRY(aplus1(h, w.u, w.q, nullptr, 1.0, w, s));        // q = A_+ u
    AWG_TRY(zt1(h, w.q, w.y2, s));
    AWG_TRY(dense_gemv(h, h->n0, (double*)h->Einv.p, w.y2, w.c2, 1.0, w.c1, -1.0, s));  // c2 = E^-1 y2 - c1
    AWG_TRY(zloc1(h, w.c2, w.loc, s));
    return prolong1(h, w.loc, z, -1.0, 0.0, w.u, 1.0, s);   // z = u - Z (c2 - c1)
}

// Row blocks of the W^T r pass: about 8 blocks per SM in total over the
// 256-column chunks, at most 8192 rows per block (its r values sit in
// shared memory), never more blocks than the partial buffer holds.
static int wt_row_blocks(const Handle* h) {
    const int chunks = (h->ldw + WT_CW - 1) / WT_CW;
    int rb = std::max(1, 152 * 8 / std::max(1, chunks));
    rb = std::max(rb, (h->n + 8191) / 8192);
    rb = std::min(rb, std::max(1, (h->n + 31) / 32));
    return std::min(rb, h->red_blocks);
}

template <typename TS>
static awg_status wt_r_t(Handle* h, const PrecOps& P, const double* r, double* out, Ws& w,
                         cudaStream_t s) {
    const void* W = P.W.p;
    const float* rsc = (const float*)P.rscale.p;
    const float* csc = (const float*)P.cscale.p;
    using A = typename Vec<TS>::A;
    const int rb = wt_row_blocks(h);
    const int rows = (h->n + rb - 1) / rb;
    const dim3 grid(rb, (h->ldw + WT_CW - 1) / WT_CW);
    const size_t smem = (size_t)(8 * WT_CW + rows) * sizeof(A);
    {
        ProfScope ps_(h, AWG_PROF_WT, s);
        k_wt_partial<TS><<<grid, WT_THREADS, smem, s>>>(h->n, h->ldw, rows, (const TS*)W, r, rsc, w.wpart);
    }
    AWG_LAUNCH();
    {
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        k_reduce_cols<<<(h->n_minus + 255) / 256, 256, 0, s>>>(rb, h->n_minus, h->ldw, w.wpart, csc, out);
    }
    AWG_LAUNCH();
    return AWG_OK;
}

static awg_status wt_r(Handle* h, int prec, const double* r, double* out, Ws& w, cudaStream_t s) {
    const PrecOps& P = h->prec[prec];
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
    const int grid = std::max(1, std::min((h->n + 7) / 8, 152 * 16));  // 8 rows (warps) per block
    const int gd = (h->ldw + 255) / 256;
    if (prec == AWG_FP64) {
        double* dp = w.dpad;
        {
            ProfScope ps_(h, AWG_PROF_VECTOR, s);
            k_d_pad64<<<gd, 256, 0, s>>>(h->n_minus, h->ldw, d, dp);
        }
        AWG_LAUNCH();
        ProfScope ps_(h, AWG_PROF_WD, s);
        k_w_d<double><<<grid, 256, (size_t)h->ldw * 8, s>>>(h->n, h->ldw, (const double*)W, dp, nullptr, v, z);
    } else {
        const float* rsc = (const float*)P.rscale.p;
        {
            ProfScope ps_(h, AWG_PROF_VECTOR, s);
            k_d_to_f32<<<gd, 256, 0, s>>>(h->n_minus, h->ldw, d, (const float*)P.cscale.p, w.d32);
        }
        AWG_LAUNCH();
        ProfScope ps_(h, AWG_PROF_WD, s);
        const size_t sm = (size_t)h->ldw * 4;
        if (prec == AWG_MIXED_FP32)
            k_w_d<float><<<grid, 256, sm, s>>>(h->n, h->ldw, (const float*)W, w.d32, rsc, v, z);
        else if (prec == AWG_MIXED_FP16)
            k_w_d<__half><<<grid, 256, sm, s>>>(h->n, h->ldw, (const __half*)W, w.d32, rsc, v, z);
        else
            k_w_d<__nv_bfloat16><<<grid, 256, sm, s>>>(h->n, h->ldw, (const __nv_bfloat16*)W, w.d32, rsc, v, z);
    }
    AWG_LAUNCH();
    return AWG_OK;
}

awg_status set_smem_limits(Handle* h) {
    const int mx = (int)std::max<size_t>((size_t)h->max_ns * 8, (size_t)std::max(1, h->ldw) * 8);
    if (mx > 48 * 1024) {
        if (mx > 227 * 1024) return AWG_ERR_INVALID_ARG;
        AWG_CUDA(cudaFuncSetAttribute(k_blk_tgemv, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        AWG_CUDA(cudaFuncSetAttribute(k_blk_gemv, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
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
            // d = F^-1 W^T x on the side stream while H_2 x runs on s
            AWG_CUDA(cudaEventRecord(h->ev_fork, s));
            AWG_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
            AWG_TRY(wt_r(h, prec, x, w.w0, w, h->side));
            AWG_TRY(dense_gemv(h, h->n_minus, (double*)h->prec[prec].Finv.p, w.w0, w.dd, 1.0, nullptr, 0,
                               h->side));
            AWG_CUDA(cudaEventRecord(h->ev_join, h->side));
            AWG_TRY(h2_1(h, prec, x, w.tmp, w, s));
            AWG_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
            return w_d(h, prec, w.dd, w.tmp, y, w, s);
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
            AWG_CUDA(cudaEventRecord(h->ev_fork, s));
            AWG_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
            AWG_TRY(wt_r(h, prec, x, w.w0, w, h->side));
            AWG_TRY(dense_gemv(h, h->n_minus, (double*)h->prec[prec].inexInv.p, w.w0, w.dd, 1.0, nullptr,
                               0, h->side));
            AWG_CUDA(cudaEventRecord(h->ev_join, h->side));
            AWG_TRY(h2_1(h, prec, x, w.tmp, w, s));
            AWG_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
            return w_d(h, prec, w.dd, w.tmp, y, w, s);
        }
        default: return AWG_ERR_INVALID_ARG;
    }
}

// ------------------------------------------------------------------- PCG
static awg_status dot1(Handle* h, const double* x, const double* y, double* out, Ws& w,
                       cudaStream_t s) {
    const int nb = grid_n(h->n);
    {
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        k_dot_partial<<<nb, 256, 0, s>>>(h->n, x, y, w.part);
    }
    AWG_LAUNCH();
    {
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        k_final_sum<<<1, 256, 0, s>>>(nb, w.part, out);
    }
    AWG_LAUNCH();
    return AWG_OK;
}

awg_status pcg1(Handle* h, int prec, int variant_stage, const double* b, double* x, double rtol,
                int* iters, double* relres, cudaStream_t s) {
    Ws w = ws_of(h);
    const int n = h->n, nb = grid_n(n);
    // partial buffer (4096 doubles): [0, 1216) and [1536, 2752) hold per-block
    // partials (grid_n <= 1216 blocks), the device scalars live at [4000, 4016)
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
            AWG_TRY(spmv1(h, p, q, w.part, s));                       // q = A p, partial p.q
            {
                ProfScope ps_(h, AWG_PROF_VECTOR, s);
                k_final_sum<<<1, 256, 0, s>>>(nb, w.part, scal + S_PQ);
            }
            AWG_LAUNCH();
            {
                ProfScope ps_(h, AWG_PROF_VECTOR, s);
                k_pcg_xr<<<nb, 256, 0, s>>>(n, scal, p, q, x, r, w.part + 1536);
            }
            AWG_LAUNCH();
            {
                ProfScope ps_(h, AWG_PROF_VECTOR, s);
                k_final_sum<<<1, 256, 0, s>>>(nb, w.part + 1536, scal + S_RR);
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
                AWG_TRY(spmv1(h, x, q, nullptr, s));
                {
                    ProfScope ps_(h, AWG_PROF_VECTOR, s);
                    k_sub<<<(n + 255) / 256, 256, 0, s>>>(n, b, q, q);
                }
                AWG_LAUNCH();
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
                k_pcg_beta<<<1, 1, 0, s>>>(scal);
            }
            AWG_LAUNCH();
            {
                ProfScope ps_(h, AWG_PROF_VECTOR, s);
                k_pcg_p<<<nb, 256, 0, s>>>(n, scal, z, p);
            }
            AWG_LAUNCH();
        }
    }
    if (st != AWG_OK || true_rel == rel) {
        AWG_TRY(spmv1(h, x, q, nullptr, s));
        {
            ProfScope ps_(h, AWG_PROF_VECTOR, s);
            k_sub<<<(n + 255) / 256, 256, 0, s>>>(n, b, q, q);
        }
        AWG_LAUNCH();
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

}  // namespace awg
