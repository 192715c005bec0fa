// Multi-right-hand-side hot path: the AWG apply and PCG for K columns at
// once (K = 16, 32 or 64; nrhs <= 64 columns padded with zero columns).
//
// Every column runs its own PCG recurrence (its own alpha, beta and stopping
// test, Section 1 PCG), so each column's iterates are those of a
// single-right-hand-side solve; what the columns share is one pass over each
// operator per iteration.  The local pseudo-inverses, W and the GenEO / V_-
// blocks are then read once for K right-hand sides instead of K times, which
// turns the bandwidth-bound GEMVs of the single-RHS path into GEMMs.
//
// Precision of a block apply (awg_precision):
//   FP64        every step in float64 (the parity form);
//   MIXED_*     the preconditioner's internal block vectors and arithmetic
//               in float32 (local pseudo-inverses float32; W float32, or
//               float16 / bfloat16 on the tensor cores, umma.cu), the two
//               coarse solves E^-1, F^-1 in float64; the PCG recurrences
//               (dot products, x, r, p updates, stopping test) always float64.
// Layout: block vectors row-major X[i * K + c]; local arenas row-major per
// local position loc[P * K + c], P in the concatenated subdomain lists.

#include "block.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <unordered_map>

namespace awg {

// Thread-to-(row, column) map of the row kernels: every thread moves 16
// bytes of a row (V = 4 float32 or 2 float64 consecutive columns, from
// column c0), TPR = K / V threads cover a row, RPW rows per warp.
template <typename T, int K>
struct RM {
    static constexpr int V = 16 / sizeof(T);
    static constexpr int TPR = K / V;
    static constexpr int RPW = 32 / TPR;
    static constexpr int RPB = 8 * RPW;  // rows per 256-thread block
};

template <typename T> struct Acc { using type = float; };
template <> struct Acc<double> { using type = double; };

__device__ __forceinline__ void ldv(const float* p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ldv(const double* p, double (&v)[2]) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    v[0] = t.x; v[1] = t.y;
}
// float32 <-> float64 conversions on the integer pipes.  On this GPU a
// conversion to or from float64 issues on the float64 pipes (about two
// per clock per SM), which bound the PCG vector kernels of the mixed forms;
// for normal numbers the conversion is a rearrangement of the IEEE 754
// fields (sign; exponent rebiased by 1023 - 127 = 896; significand shifted
// by 52 - 23 = 29 bits, rounded to nearest even on the way down), done here
// with integer operations.  Zeros keep their sign; subnormals, infinities,
// NaNs and float64 values outside the float32 normal range take the
// hardware conversion.
__device__ __forceinline__ double f2d(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xFFu;
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    if ((u & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)sign);
    if (e == 0u || e == 0xFFu) return (double)f;
    return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 896u) << 52) |
                                            ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}
__device__ __forceinline__ float d2f(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    if ((b << 1) == 0ull) return __uint_as_float(sign);
    const int e = (int)((b >> 52) & 0x7FF) - 896;
    if (e < 1 || e > 254) return (float)d;
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull, rem = m & 0x1FFFFFFFull;
    unsigned r = ((unsigned)e << 23) | (unsigned)(m >> 29);
    r += (rem > 0x10000000ull || (rem == 0x10000000ull && (r & 1u))) ? 1u : 0u;  // may carry into inf
    return __uint_as_float(r | sign);
}
template <typename TO, typename TI> __device__ __forceinline__ TO cvt(TI a) { return (TO)a; }
template <> __device__ __forceinline__ double cvt<double, float>(float a) { return f2d(a); }
template <> __device__ __forceinline__ float cvt<float, double>(double a) { return d2f(a); }

// two consecutive values of a float64 row kernel's columns, from float64 or
// float32 storage
__device__ __forceinline__ void ld2(const double* p, double (&v)[2]) { ldv(p, v); }
__device__ __forceinline__ void ld2(const float* p, double (&v)[2]) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = f2d(t.x); v[1] = f2d(t.y);
}
__device__ __forceinline__ void stv(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void stv(double* p, const double (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
}

// Column sums of `count` partial rows src[b * K + c] (b in order, read
// through L2) into dst[c], by all 256 threads of the block: thread t takes
// column t % K and every Q-th row from t / K (Q = 256 / K) with eight
// independent sums (the loads stay in flight), then the Q sums of a column
// meet in a fixed order
template <int K>
__device__ __forceinline__ void sum_partials(const double* src, int count, double* dst) {
    constexpr int Q = 256 / K;
    __shared__ double qs[Q][K];
    __syncthreads();
    {
        const int c = threadIdx.x % K, q = threadIdx.x / K;
        double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        int b = q;
        for (; b + 7 * Q < count; b += 8 * Q) {
#pragma unroll
            for (int u = 0; u < 8; u++) a[u] += __ldcg(src + (size_t)(b + u * Q) * K + c);
        }
        for (; b < count; b += Q) a[0] += __ldcg(src + (size_t)b * K + c);
        qs[q][c] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double v = 0.0;
#pragma unroll
        for (int q = 0; q < Q; q++) v += qs[q][threadIdx.x];
        dst[threadIdx.x] = v;
    }
}

// Per-column sums of a 256-thread block of float64 row kernels (thread
// partials acc[j] belong to column c0 + j), then over the grid in two
// levels: block partials go to part[b * K + c]; the last block to arrive
// of each group of CS_G blocks (ticket cnt[1 + g]) adds the group's
// partials in block order into part[(CS_PMAX + g) * K + c], and the last
// group to finish (ticket cnt[0]) adds the group sums in group order.  Two
// short rounds of L2 loads instead of one block reading every partial;
// deterministic for a given grid (at most CS_PMAX blocks).  The counters
// return to zero.
constexpr int CS_G = 128, CS_PMAX = 1216;
template <int K>
__device__ __forceinline__ void colsum_grid(const double (&acc)[2], double* part, unsigned* cnt, double* out) {
    using M = RM<double, K>;
    __shared__ double red[8 * M::RPW][K];
    __shared__ unsigned ticket;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int rw = lane / M::TPR, c0 = (lane % M::TPR) * 2;
    red[w * M::RPW + rw][c0] = acc[0];
    red[w * M::RPW + rw][c0 + 1] = acc[1];
    __syncthreads();
    if (threadIdx.x < K) {
        double v = 0.0;
        for (int r = 0; r < 8 * M::RPW; r++) v += red[r][threadIdx.x];
        part[(size_t)blockIdx.x * K + threadIdx.x] = v;
    }
    __threadfence();
    __syncthreads();
    const int g = blockIdx.x / CS_G, g0 = g * CS_G;
    const int gn = min(CS_G, (int)gridDim.x - g0), ng = ((int)gridDim.x + CS_G - 1) / CS_G;
    if (threadIdx.x == 0) ticket = atomicAdd(cnt + 1 + g, 1u);
    __syncthreads();
    if (ticket != (unsigned)gn - 1u) return;
    __threadfence();
    double* gp = part + (size_t)CS_PMAX * K;
    sum_partials<K>(part + (size_t)g0 * K, gn, ng == 1 ? out : gp + (size_t)g * K);
    if (threadIdx.x == 0) cnt[1 + g] = 0u;
    if (ng == 1) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) ticket = atomicAdd(cnt, 1u);
    __syncthreads();
    if (ticket != (unsigned)ng - 1u) return;
    __threadfence();
    sum_partials<K>(gp, ng, out);
    if (threadIdx.x == 0) cnt[0] = 0u;
}

// (unrolled by 4: the loads of four rows are in flight together)
#define ROW_LOOP(T_, K_)                                                                 \
    using M = RM<T_, K_>;                                                                \
    const int lane_ = threadIdx.x & 31, w_ = threadIdx.x >> 5;                           \
    const int rw_ = lane_ / M::TPR, c0 = (lane_ % M::TPR) * M::V;                        \
    _Pragma("unroll 4")                                                                  \
    for (int i = blockIdx.x * M::RPB + w_ * M::RPW + rw_; i < n; i += gridDim.x * M::RPB)

// ------------------------------------------------------------- PCG (float64)
// PCG scalars of a block solve, K values each: rz, pq, rr, rz_new, b.b,
// true residual, active flag (1.0 / 0.0), candidate flag of the graph-driven
// loop (recurrence residual at rtol, true residual not yet confirmed)
enum { B_RZ = 0, B_PQ = 1, B_RR = 2, B_RZN = 3, B_BB = 4, B_TR = 5, B_ACT = 6, B_CAND = 7, B_NSC = 8 };

// Y = A X and, if dot, the column sums of X .* Y
template <int K>
__global__ void __launch_bounds__(256) kb_spmv_dot(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                   const double* __restrict__ a, const double* __restrict__ X,
                                                   double* __restrict__ Y, double* part, unsigned* cnt,
                                                   double* dot) {
    double acc[2] = {0.0, 0.0};
    ROW_LOOP(double, K) {
        double y[2] = {0.0, 0.0};
        const int e1 = rp[i + 1];
        for (int k = rp[i]; k < e1; k++) {
            double xv[2];
            ldv(X + (size_t)ci[k] * K + c0, xv);
            const double av = a[k];
            y[0] = fma(av, xv[0], y[0]);
            y[1] = fma(av, xv[1], y[1]);
        }
        stv(Y + (size_t)i * K + c0, y);
        double xi[2];
        ldv(X + (size_t)i * K + c0, xi);
        acc[0] = fma(y[0], xi[0], acc[0]);
        acc[1] = fma(y[1], xi[1], acc[1]);
    }
    if (dot) colsum_grid<K>(acc, part, cnt, dot);
}

// Q = B - A X (nothing when *gate is 0: the graph-driven loop computes the
// true residual only in iterations where some column is a candidate)
template <int K>
__global__ void __launch_bounds__(256) kb_resid(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                const double* __restrict__ a, const double* __restrict__ B,
                                                const double* __restrict__ X, double* __restrict__ Q,
                                                const double* gate = nullptr) {
    if (gate && *gate == 0.0) return;
    ROW_LOOP(double, K) {
        double y[2] = {0.0, 0.0};
        for (int k = rp[i]; k < rp[i + 1]; k++) {
            double xv[2];
            ldv(X + (size_t)ci[k] * K + c0, xv);
            y[0] = fma(a[k], xv[0], y[0]);
            y[1] = fma(a[k], xv[1], y[1]);
        }
        double b[2];
        ldv(B + (size_t)i * K + c0, b);
        const double q[2] = {b[0] - y[0], b[1] - y[1]};
        stv(Q + (size_t)i * K + c0, q);
    }
}

// out[c] = sum_i X(i, c) Y(i, c) in float64 (Y float64, or the float32
// output of a mixed-precision apply); nothing when *gate is 0, as kb_resid
template <int K, typename TY = double>
__global__ void __launch_bounds__(256) kb_coldot(int n, const double* __restrict__ X, const TY* __restrict__ Y,
                                                 double* part, unsigned* cnt, double* out,
                                                 const double* gate = nullptr) {
    if (gate && *gate == 0.0) return;
    double acc[2] = {0.0, 0.0};
    ROW_LOOP(double, K) {
        double x[2], y[2];
        ldv(X + (size_t)i * K + c0, x);
        ld2(Y + (size_t)i * K + c0, y);
        acc[0] = fma(x[0], y[0], acc[0]);
        acc[1] = fma(x[1], y[1], acc[1]);
    }
    colsum_grid<K>(acc, part, cnt, out);
}

// per column c: alpha = rz / pq (0 for inactive columns or pq <= 0);
// X += alpha P, R -= alpha Q, rr = R . R
// (R32, if given: R rounded to float32, the input of the next mixed-precision apply)
template <int K>
__global__ void __launch_bounds__(256) kb_pcg_xr(int n, double* sc, const double* __restrict__ P,
                                                 const double* __restrict__ Q, double* X, double* R,
                                                 double* part, unsigned* cnt, float* R32 = nullptr) {
    double alpha[2], acc[2] = {0.0, 0.0};
    {
        const int cc = ((threadIdx.x & 31) % RM<double, K>::TPR) * 2;
#pragma unroll
        for (int j = 0; j < 2; j++) {
            const int c = cc + j;
            const double pq = sc[B_PQ * K + c];
            alpha[j] = (sc[B_ACT * K + c] != 0.0 && pq > 0.0) ? sc[B_RZ * K + c] / pq : 0.0;
        }
    }
    ROW_LOOP(double, K) {
        const size_t e = (size_t)i * K + c0;
        double p[2], q[2], x[2], r[2];
        ldv(P + e, p);
        ldv(Q + e, q);
        ldv(X + e, x);
        ldv(R + e, r);
#pragma unroll
        for (int j = 0; j < 2; j++) {
            x[j] = fma(alpha[j], p[j], x[j]);
            r[j] = fma(-alpha[j], q[j], r[j]);
            acc[j] = fma(r[j], r[j], acc[j]);
        }
        stv(X + e, x);
        stv(R + e, r);
        if (R32) *reinterpret_cast<float2*>(R32 + e) = make_float2(d2f(r[0]), d2f(r[1]));
    }
    colsum_grid<K>(acc, part, cnt, sc + B_RR * K);
}

// per active column: beta = rz_new / rz, P = Z + beta P; the last block
// then moves rz_new into rz
template <int K, typename TZ = double>
__global__ void __launch_bounds__(256) kb_pcg_p(int n, double* sc, const TZ* __restrict__ Z, double* P,
                                                unsigned* cnt) {
    __shared__ unsigned ticket;
    double beta[2];
    {
        const int cc = ((threadIdx.x & 31) % RM<double, K>::TPR) * 2;
#pragma unroll
        for (int j = 0; j < 2; j++) {
            const int c = cc + j;
            const double rz = sc[B_RZ * K + c];
            // inactive columns keep P: beta = 1 and Z replaced by 0 below
            beta[j] = (sc[B_ACT * K + c] == 0.0) ? 1.0 : ((rz != 0.0) ? sc[B_RZN * K + c] / rz : 0.0);
        }
    }
    const int cc = ((threadIdx.x & 31) % RM<double, K>::TPR) * 2;
    const bool a0 = sc[B_ACT * K + cc] != 0.0, a1 = sc[B_ACT * K + cc + 1] != 0.0;
    ROW_LOOP(double, K) {
        const size_t e = (size_t)i * K + c0;
        double z[2], pv[2];
        ld2(Z + e, z);
        ldv(P + e, pv);
        pv[0] = a0 ? fma(beta[0], pv[0], z[0]) : pv[0];
        pv[1] = a1 ? fma(beta[1], pv[1], z[1]) : pv[1];
        stv(P + e, pv);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        ticket = atomicAdd(cnt, 1u);
    }
    __syncthreads();
    if (ticket == gridDim.x - 1) {
        if (threadIdx.x < K && sc[B_ACT * K + threadIdx.x] != 0.0)
            sc[B_RZ * K + threadIdx.x] = sc[B_RZN * K + threadIdx.x];
        if (threadIdx.x == 0) *cnt = 0u;
    }
}

// flexible (Polak-Ribiere) update for a preconditioner applied in lower
// precision: per active column beta = (r.z - r.z_old) / rz_old with r.z in
// B_RZN and r.z_old in B_TR, P = Z + beta P; the last block moves rz_new
// into rz
template <int K>
__global__ void __launch_bounds__(256) kb_pcg_p_flex(int n, double* sc, const double* __restrict__ Z, double* P,
                                                     unsigned* cnt) {
    __shared__ unsigned ticket;
    const int cc = ((threadIdx.x & 31) % RM<double, K>::TPR) * 2;
    double beta[2];
    bool act[2];
#pragma unroll
    for (int j = 0; j < 2; j++) {
        const int c = cc + j;
        const double rz = sc[B_RZ * K + c];
        act[j] = sc[B_ACT * K + c] != 0.0;
        beta[j] = (rz != 0.0) ? (sc[B_RZN * K + c] - sc[B_TR * K + c]) / rz : 0.0;
    }
    ROW_LOOP(double, K) {
        const size_t e = (size_t)i * K + c0;
        double z[2], pv[2];
        ldv(Z + e, z);
        ldv(P + e, pv);
        pv[0] = act[0] ? fma(beta[0], pv[0], z[0]) : pv[0];
        pv[1] = act[1] ? fma(beta[1], pv[1], z[1]) : pv[1];
        stv(P + e, pv);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        ticket = atomicAdd(cnt, 1u);
    }
    __syncthreads();
    if (ticket == gridDim.x - 1) {
        if (threadIdx.x < K && sc[B_ACT * K + threadIdx.x] != 0.0)
            sc[B_RZ * K + threadIdx.x] = sc[B_RZN * K + threadIdx.x];
        if (threadIdx.x == 0) *cnt = 0u;
    }
}

// --------------------------------------------------------- layout / types
// dst (n x K row-major) from nrhs columns of src (column-major, ld), zero
// columns beyond nrhs; 32 x 32 tiles through shared memory
template <typename TD>
__global__ void kb_from_cols(int n, int nrhs, int ld, int K, const double* __restrict__ src, TD* __restrict__ dst) {
    __shared__ double t[32][33];
    const int i0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int c = c0 + r, i = i0 + threadIdx.x;
        t[r][threadIdx.x] = (c < nrhs && i < n) ? src[(size_t)c * ld + i] : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r, c = c0 + threadIdx.x;
        if (i < n && c < K) dst[(size_t)i * K + c] = (TD)t[threadIdx.x][r];
    }
}

// nrhs columns of dst (column-major, ld) from src (n x K row-major)
template <typename TS>
__global__ void kb_to_cols(int n, int nrhs, int ld, int K, const TS* __restrict__ src, double* __restrict__ dst) {
    __shared__ double t[32][33];
    const int i0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r, c = c0 + threadIdx.x;
        t[r][threadIdx.x] = (i < n && c < K) ? (double)src[(size_t)i * K + c] : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int c = c0 + r, i = i0 + threadIdx.x;
        if (c < nrhs && i < n) dst[(size_t)c * ld + i] = t[threadIdx.x][r];
    }
}

template <typename T>
__global__ void kb_sub(size_t len, const T* __restrict__ a, const T* __restrict__ b, T* c) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < len) c[e] = a[e] - b[e];
}

template <typename T>
__global__ void kb_add(size_t len, const T* __restrict__ a, T* y) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < len) y[e] += a[e];
}

template <typename TI, typename TO>
__global__ void kb_cvt(size_t len, const TI* __restrict__ a, TO* __restrict__ b) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < len) b[e] = cvt<TO>(a[e]);
}

// ------------------------------------------------------ preconditioner ops
// Y = Yin + sign (A X + sum over the copies (s, q) of i of V_s(q, :) cm_s)
// (A_+ = A + A_-, Thm. 2), cm_s = |Lambda^s_-| V^s_-^T R^s X from kb_tgemv2
template <typename T, int K>
__global__ void __launch_bounds__(256) kb_aplus(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                const T* __restrict__ a, const T* __restrict__ X,
                                                const int* __restrict__ inc_ptr, const int* __restrict__ inc_pos,
                                                const int* __restrict__ inc_sub, const int* __restrict__ sub_ptr,
                                                const int* __restrict__ colptr, const int64_t* __restrict__ boff,
                                                const T* __restrict__ V, const T* __restrict__ cm,
                                                const T* Yin, T sign, T* Y) {
    ROW_LOOP(T, K) {
        T y[M::V] = {};
        const int k1 = rp[i + 1];
        for (int k = rp[i]; k < k1; k++) {
            T xv[M::V];
            ldv(X + (size_t)ci[k] * K + c0, xv);
            const T av = a[k];
#pragma unroll
            for (int j = 0; j < M::V; j++) y[j] = fma(av, xv[j], y[j]);
        }
        if (cm) {
            for (int e = inc_ptr[i]; e < inc_ptr[i + 1]; e++) {
                const int s = inc_sub[e];
                const int ps = sub_ptr[s], m = sub_ptr[s + 1] - ps;
                const int cq = colptr[s], nc = colptr[s + 1] - cq;
                const T* b = V + boff[s] + (inc_pos[e] - ps);
#pragma unroll 4
                for (int q = 0; q < nc; q++) {
                    T cv[M::V];
                    ldv(cm + (size_t)(cq + q) * K + c0, cv);
                    const T bv = b[(size_t)q * m];
#pragma unroll
                    for (int j = 0; j < M::V; j++) y[j] = fma(bv, cv[j], y[j]);
                }
            }
        }
        const size_t e = (size_t)i * K + c0;
        T o[M::V];
        if (Yin) {
            ldv(Yin + e, o);
#pragma unroll
            for (int j = 0; j < M::V; j++) o[j] = fma(sign, y[j], o[j]);
        } else {
#pragma unroll
            for (int j = 0; j < M::V; j++) o[j] = sign * y[j];
        }
        stv(Y + e, o);
    }
}

// C_s(q, :) = wsign w_q sum_p B_s(p, q) X(idx_s(p), :) for every subdomain s
// (B_s n^s x nc_s column-major; block-sparse Z^T X and V_-^T X).  Block
// (s, ps) of kb_tgemv2 takes the local positions of split ps and the columns
// of B_s in passes of 16 or 32: each chunk of rows of X is gathered once
// into shared memory (16-byte loads of whole rows) and serves all columns of
// the pass; thread t owns column c = t % K of X and TJ / (256 / K)
// consecutive columns of B_s, read from shared memory as 16-byte vectors
// (one shared load per FMA left the kernel bound by its load/store pipe).
// Partial sums go to part[ps][colptr[s] + q][c]; kb_tg_sum adds the TG_PS
// splits in order.
constexpr int TG_PS = 8;
template <typename T> struct V16;
template <> struct V16<float> {
    using type = float4;
    static __device__ __forceinline__ float get(const float4& v, int i) {
        return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
    }
};
template <> struct V16<double> {
    using type = double2;
    static __device__ __forceinline__ double get(const double2& v, int i) { return i == 0 ? v.x : v.y; }
};
constexpr int TG2_TJ = 32;  // columns q per pass (at most)
template <typename T> struct TG2 {
    static constexpr int ROWS = sizeof(T) == 8 ? 32 : 64;      // rows per chunk (about 24 KB of shared memory)
    static constexpr int BP = TG2_TJ + 16 / (int)sizeof(T);    // padded row of bs (16-byte multiple)
};
// One block's work with TJ columns q per pass: TJ = 16 for subdomains with
// at most 16 columns (half the shared loads and FMAs of a 32-column pass,
// most of which would multiply padding), 32 otherwise
template <typename T, int K, int TJ>
__device__ __forceinline__ void tgemv2_body(T (*xs)[K], T (*bs)[TG2<T>::BP], const int* __restrict__ sub_idx,
                                            const T* __restrict__ Bs, const T* __restrict__ X, int p0, int m,
                                            int c0, int nc, int pa, int pb, int rs, int ncol_total,
                                            T* __restrict__ part) {
    constexpr int ROWS = TG2<T>::ROWS;
    constexpr int JG = 256 / K, JU = TJ / JG;
    constexpr int V4 = K * (int)sizeof(T) / 16;
    constexpr int BV16 = 16 / (int)sizeof(T);            // values per 16-byte load
    constexpr int BV = JU % BV16 == 0 ? BV16 : 1;         // (scalar loads for narrow column blocks)
    const int c = threadIdx.x % K, jb = (threadIdx.x / K) * JU;
    for (int j0 = 0; j0 < nc; j0 += TJ) {
        const int jn = min(TJ, nc - j0);
        T acc[JU];
#pragma unroll
        for (int u = 0; u < JU; u++) acc[u] = 0;
        for (int q0 = pa; q0 < pb; q0 += ROWS) {
            const int pn = min(ROWS, pb - q0);
            __syncthreads();
            for (int e = threadIdx.x; e < TJ * ROWS; e += 256) {
                const int jj = e / ROWS, pp = e % ROWS;
                bs[pp][jj] = (jj < jn && pp < pn) ? Bs[(size_t)(j0 + jj) * m + q0 + pp] : (T)0;
            }
            for (int e = threadIdx.x; e < ROWS * V4; e += 256) {
                const int pp = e / V4, cc = e % V4;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (pp < pn) v = reinterpret_cast<const float4*>(X + (size_t)sub_idx[p0 + q0 + pp] * K)[cc];
                reinterpret_cast<float4*>(&xs[pp][0])[cc] = v;
            }
            __syncthreads();
#pragma unroll 4
            for (int pp = 0; pp < ROWS; pp++) {
                const T x = xs[pp][c];
                if constexpr (BV == BV16) {
                    using V = typename V16<T>::type;
#pragma unroll
                    for (int u0 = 0; u0 < JU; u0 += BV) {
                        const V bv = *reinterpret_cast<const V*>(&bs[pp][jb + u0]);
#pragma unroll
                        for (int u = 0; u < BV; u++) acc[u0 + u] = fma(V16<T>::get(bv, u), x, acc[u0 + u]);
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < JU; u++) acc[u] = fma(bs[pp][jb + u], x, acc[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < JU; u++) {
            const int jj = jb + u;
            if (jj < jn) part[((size_t)rs * ncol_total + c0 + j0 + jj) * K + c] = acc[u];
        }
    }
}

template <typename T, int K>
__global__ void __launch_bounds__(256) kb_tgemv2(const int* __restrict__ sub_ptr, const int* __restrict__ sub_idx,
                                                 const int* __restrict__ colptr, const int64_t* __restrict__ boff,
                                                 const T* __restrict__ B, const T* __restrict__ X, int ncol_total,
                                                 T* __restrict__ part) {
    __shared__ __align__(16) T xs[TG2<T>::ROWS][K];
    __shared__ __align__(16) T bs[TG2<T>::ROWS][TG2<T>::BP];
    const int s = blockIdx.x, rs = blockIdx.y;
    const int p0 = sub_ptr[s], m = sub_ptr[s + 1] - p0;
    const int c0 = colptr[s], nc = colptr[s + 1] - c0;
    if (nc == 0) return;
    const int plen = (m + gridDim.y - 1) / gridDim.y;
    const int pa = rs * plen, pb = min(m, pa + plen);
    const T* Bs = B + boff[s];
    if (nc <= 16)
        tgemv2_body<T, K, 16>(xs, bs, sub_idx, Bs, X, p0, m, c0, nc, pa, pb, rs, ncol_total, part);
    else
        tgemv2_body<T, K, TG2_TJ>(xs, bs, sub_idx, Bs, X, p0, m, c0, nc, pa, pb, rs, ncol_total, part);
}

template <typename T, int K>
__global__ void kb_tg_sum(int ncol_total, const T* __restrict__ part, const T* __restrict__ w, T wsign, T* C) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t len = (size_t)ncol_total * K;
    if (e >= len) return;
    T v = 0;
#pragma unroll
    for (int ps = 0; ps < TG_PS; ps++) v += part[(size_t)ps * len + e];
    C[e] = w ? wsign * w[e / K] * v : v;
}

// Y(i, :) = beta Y(i, :) + alpha sum over the copies (s, p) of i of
// sum_q B_s(p, q) C(colptr[s] + q, :) + gamma V(i, :) (+ V2(i, :))
template <typename T, int K>
__global__ void __launch_bounds__(256) kb_blk_prolong(int n, const int* __restrict__ inc_ptr,
                                                      const int* __restrict__ inc_pos,
                                                      const int* __restrict__ inc_sub,
                                                      const int* __restrict__ sub_ptr,
                                                      const int* __restrict__ colptr,
                                                      const int64_t* __restrict__ boff, const T* __restrict__ B,
                                                      const T* __restrict__ C, T* Y, T alpha, T beta,
                                                      const T* V, T gamma, const T* V2) {
    ROW_LOOP(T, K) {
        T y[M::V] = {};
        for (int e = inc_ptr[i]; e < inc_ptr[i + 1]; e++) {
            const int s = inc_sub[e];
            const int ps = sub_ptr[s], m = sub_ptr[s + 1] - ps;
            const int cq = colptr[s], nc = colptr[s + 1] - cq;
            const T* b = B + boff[s] + (inc_pos[e] - ps);
#pragma unroll 4
            for (int q = 0; q < nc; q++) {
                T cv[M::V];
                ldv(C + (size_t)(cq + q) * K + c0, cv);
                const T bv = b[(size_t)q * m];
#pragma unroll
                for (int j = 0; j < M::V; j++) y[j] = fma(bv, cv[j], y[j]);
            }
        }
        const size_t e = (size_t)i * K + c0;
        T o[M::V], t[M::V];
#pragma unroll
        for (int j = 0; j < M::V; j++) o[j] = alpha * y[j];
        if (beta != (T)0) {
            ldv(Y + e, t);
#pragma unroll
            for (int j = 0; j < M::V; j++) o[j] = fma(beta, t[j], o[j]);
        }
        if (V) {
            ldv(V + e, t);
#pragma unroll
            for (int j = 0; j < M::V; j++) o[j] = fma(gamma, t[j], o[j]);
        }
        if (V2) {
            ldv(V2 + e, t);
#pragma unroll
            for (int j = 0; j < M::V; j++) o[j] += t[j];
        }
        stv(Y + e, o);
    }
}

// Y(i, :) = beta Y(i, :) + alpha sum over the copies of i of loc(pos, :) + gamma V(i, :)
template <typename T, int K>
__global__ void __launch_bounds__(256) kb_prolong(int n, const int* __restrict__ inc_ptr,
                                                  const int* __restrict__ inc_pos, const T* __restrict__ loc,
                                                  T* Y, T alpha, T beta, const T* V, T gamma) {
    ROW_LOOP(T, K) {
        T y[M::V] = {};
        for (int e = inc_ptr[i]; e < inc_ptr[i + 1]; e++) {
            T lv[M::V];
            ldv(loc + (size_t)inc_pos[e] * K + c0, lv);
#pragma unroll
            for (int j = 0; j < M::V; j++) y[j] += lv[j];
        }
        const size_t e = (size_t)i * K + c0;
        T o[M::V], t[M::V];
#pragma unroll
        for (int j = 0; j < M::V; j++) o[j] = alpha * y[j];
        if (beta != (T)0) {
            ldv(Y + e, t);
#pragma unroll
            for (int j = 0; j < M::V; j++) o[j] = fma(beta, t[j], o[j]);
        }
        if (V) {
            ldv(V + e, t);
#pragma unroll
            for (int j = 0; j < M::V; j++) o[j] = fma(gamma, t[j], o[j]);
        }
        stv(Y + e, o);
    }
}

// loc(P, :) = X(sub_idx[P], :)
template <typename T, int K>
__global__ void kb_gather(int64_t sum_ns, const int* __restrict__ sub_idx, const T* __restrict__ X,
                          T* __restrict__ loc) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= sum_ns * K) return;
    const int64_t P = e / K;
    const int c = (int)(e % K);
    loc[e] = X[(size_t)sub_idx[P] * K + c];
}

// out_s = G_s loc_s for every subdomain s: G_s symmetric n^s x n^s stored
// column-major with leading dimension ld_s (n^s for float64; n^s rounded up
// to 4, zero padded, for float32), so row r of G_s is read as column r.
// Each thread owns RT consecutive rows and all K columns (RT * K = 64
// accumulators): per step q one load of RT values of column q of G_s, the
// K values of loc_s(q, :) from shared memory (broadcast), RT * K FMAs.
template <typename T, int K>
struct LG {
    static constexpr int RT = 64 / K;            // rows per thread: 4, 2, 1
    static constexpr int ROWS = 128 * RT;        // rows per 128-thread block
    static constexpr int JC = 64;                // staged local positions
};

template <typename T, int RT> struct LoadRT;
template <> struct LoadRT<float, 1> {
    __device__ static void ld(const float* p, float* o) { o[0] = __ldcs(p); }
};
template <> struct LoadRT<float, 2> {
    __device__ static void ld(const float* p, float* o) {
        const float2 v = __ldcs(reinterpret_cast<const float2*>(p));
        o[0] = v.x; o[1] = v.y;
    }
};
template <> struct LoadRT<float, 4> {
    __device__ static void ld(const float* p, float* o) {
        const float4 v = __ldcs(reinterpret_cast<const float4*>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
};
template <int RT> struct LoadRT<double, RT> {
    __device__ static void ld(const double* p, double* o) {
#pragma unroll
        for (int r = 0; r < RT; r++) o[r] = __ldcs(p + r);
    }
};

// 16 bytes of a 16-byte aligned shared array in one load
template <typename T>
__device__ __forceinline__ void lds16(const T* p, T* o) {
    *reinterpret_cast<float4*>(o) = *reinterpret_cast<const float4*>(p);
}

template <typename T, int K>
__global__ void __launch_bounds__(128) kb_local_gemm(const int* __restrict__ sub_ptr, const int64_t* __restrict__ goff,
                                                     const T* __restrict__ G, int pad4,
                                                     const T* __restrict__ loc, T* __restrict__ out) {
    using L = LG<T, K>;
    constexpr int RT = L::RT;
    constexpr int QG = sizeof(T) == 4 ? 8 : 4;     // columns of G per step
    constexpr int V = 16 / sizeof(T);              // values per 16-byte shared load
    __shared__ __align__(16) T xs[L::JC][K];
    const int s = blockIdx.x;
    const int p0 = sub_ptr[s], m = sub_ptr[s + 1] - p0;
    const int ld = pad4 ? ((m + 3) & ~3) : m;
    const int r0 = blockIdx.y * L::ROWS;
    if (r0 >= m) return;
    const int rb = r0 + threadIdx.x * RT;          // first row of this thread
    const bool live = rb < m;
    const bool vec = pad4 || rb + RT <= m;         // whole RT rows inside the column
    const T* Gs = G + goff[s] + rb;
    T acc[RT][K];
#pragma unroll
    for (int r = 0; r < RT; r++)
#pragma unroll
        for (int c = 0; c < K; c++) acc[r][c] = 0;
    // the RT values of columns q .. q + QG - 1 (zero past column m - 1)
    auto load_group = [&](int q, T (&g)[QG][RT]) {
#pragma unroll
        for (int u = 0; u < QG; u++) {
            if (live && q + u < m) {
                if (vec) LoadRT<T, RT>::ld(Gs + (size_t)(q + u) * ld, g[u]);
                else
#pragma unroll
                    for (int r = 0; r < RT; r++) g[u][r] = (rb + r < m) ? Gs[(size_t)(q + u) * ld + r] : (T)0;
            } else {
#pragma unroll
                for (int r = 0; r < RT; r++) g[u][r] = (T)0;
            }
        }
    };
    // software pipeline: the loads of the next QG columns are in flight
    // while the current ones are multiplied
    T gc[QG][RT], gn[QG][RT];
    load_group(0, gc);
    const T* ls = loc + (size_t)p0 * K;
    for (int q0 = 0; q0 < m; q0 += L::JC) {
        const int qn = min(L::JC, m - q0);
        __syncthreads();
        for (int e = threadIdx.x; e < L::JC * K; e += blockDim.x)
            (&xs[0][0])[e] = (e / K < qn) ? ls[(size_t)q0 * K + e] : (T)0;
        __syncthreads();
        for (int q = 0; q < qn; q += QG) {
            load_group(q0 + q + QG, gn);
#pragma unroll
            for (int u = 0; u < QG; u++)
#pragma unroll
                for (int c = 0; c < K; c += V) {
                    T xv[V];
                    lds16(&xs[q + u][c], xv);
#pragma unroll
                    for (int cc = 0; cc < V; cc++)
#pragma unroll
                        for (int r = 0; r < RT; r++) acc[r][c + cc] = fma(gc[u][r], xv[cc], acc[r][c + cc]);
                }
#pragma unroll
            for (int u = 0; u < QG; u++)
#pragma unroll
                for (int r = 0; r < RT; r++) gc[u][r] = gn[u][r];
        }
    }
    if (!live) return;
#pragma unroll
    for (int r = 0; r < RT; r++) {
        if (rb + r >= m) break;
        T* o = out + (size_t)(p0 + rb + r) * K;
#pragma unroll
        for (int c = 0; c < K; c += V) {
            if constexpr (sizeof(T) == 4)
                *reinterpret_cast<float4*>(o + c) = make_float4(acc[r][c], acc[r][c + 1], acc[r][c + 2], acc[r][c + 3]);
            else
                *reinterpret_cast<double2*>(o + c) = make_double2(acc[r][c], acc[r][c + 1]);
        }
    }
}

// Y = alpha M X + beta Sub in float64, M symmetric dim x dim (row p read as
// column p), X, Y, Sub dim x K row-major.  The float64 pipes of this GPU
// are its narrowest unit, so the product is spread over about four blocks
// per SM: block (t, sp) multiplies rows 32 t .. 32 t + 31 of M by the rows
// jlen sp .. jlen (sp + 1) - 1 of X into part[sp] (each thread 2 rows x 4
// columns, chunks of 32 staged in shared memory); kb_dense_sum adds the
// splits in order.
constexpr int DG_RB = 32, DG_JC = 32, DG_SMAX = 16;
template <int K>
__global__ void __launch_bounds__(4 * K) kb_dense_part(int dim, int jlen, const double* __restrict__ Mx,
                                                       const double* __restrict__ X, double* __restrict__ part) {
    __shared__ double ms[DG_RB][DG_JC + 1];
    __shared__ __align__(16) double xs[DG_JC][K];
    const int r0 = blockIdx.x * DG_RB;
    const int j0s = blockIdx.y * jlen, j1s = min(dim, j0s + jlen);
    const int cg = threadIdx.x % (K / 4), rp = threadIdx.x / (K / 4);  // rp < 16
    double acc[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    for (int j0 = j0s; j0 < j1s; j0 += DG_JC) {
        const int jn = min(DG_JC, j1s - j0);
        __syncthreads();
        for (int e = threadIdx.x; e < DG_RB * DG_JC; e += blockDim.x) {
            const int rr = e / DG_JC, jj = e % DG_JC;
            ms[rr][jj] = (r0 + rr < dim && jj < jn) ? Mx[(size_t)(r0 + rr) * dim + j0 + jj] : 0.0;
        }
        for (int e = threadIdx.x; e < DG_JC * K; e += blockDim.x)
            (&xs[0][0])[e] = (e / K < jn) ? X[(size_t)j0 * K + e] : 0.0;
        __syncthreads();
#pragma unroll 8
        for (int jj = 0; jj < DG_JC; jj++) {
            const double m0 = ms[2 * rp][jj], m1 = ms[2 * rp + 1][jj];
            const double2 x01 = *reinterpret_cast<const double2*>(&xs[jj][cg * 4]);
            const double2 x23 = *reinterpret_cast<const double2*>(&xs[jj][cg * 4 + 2]);
            acc[0][0] = fma(m0, x01.x, acc[0][0]);
            acc[0][1] = fma(m0, x01.y, acc[0][1]);
            acc[0][2] = fma(m0, x23.x, acc[0][2]);
            acc[0][3] = fma(m0, x23.y, acc[0][3]);
            acc[1][0] = fma(m1, x01.x, acc[1][0]);
            acc[1][1] = fma(m1, x01.y, acc[1][1]);
            acc[1][2] = fma(m1, x23.x, acc[1][2]);
            acc[1][3] = fma(m1, x23.y, acc[1][3]);
        }
    }
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const int row = r0 + 2 * rp + u;
        if (row >= dim) continue;
        double* o = part + ((size_t)blockIdx.y * dim + row) * K + cg * 4;
        *reinterpret_cast<double2*>(o) = make_double2(acc[u][0], acc[u][1]);
        *reinterpret_cast<double2*>(o + 2) = make_double2(acc[u][2], acc[u][3]);
    }
}

template <int K>
__global__ void kb_dense_sum(int dim, int S, const double* __restrict__ part, double* Y, double alpha,
                             const double* Sub, double beta) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t len = (size_t)dim * K;
    if (e >= len) return;
    double v = 0.0;
    for (int sp = 0; sp < S; sp++) v += part[(size_t)sp * len + e];
    Y[e] = Sub ? fma(beta, Sub[e], alpha * v) : alpha * v;
}

// ------------------------------------------- W passes on the CUDA cores
template <typename TS> __device__ __forceinline__ typename Acc<TS>::type wval(TS v) {
    return (typename Acc<TS>::type)v;
}
template <> __device__ __forceinline__ float wval<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float wval<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// part[b][c * K + j] = sum over the rows i of row block b of W(i, c) Xs(i, j),
// Xs = S_r X (rscale) or X; one column of W per thread, 32-row chunks of Xs
// in shared memory.  Block (b, 0) also stores Xs (for the sparse correction).
template <typename TS, typename A, int K>
__global__ void __launch_bounds__(256) kb_wt_partial(int n, int ldw, int rows, const TS* __restrict__ W,
                                                     const A* __restrict__ X, const float* __restrict__ rscale,
                                                     A* part, A* xs_out) {
    __shared__ __align__(16) A xs[32][K];
    const int i0 = blockIdx.x * rows, i1 = min(n, i0 + rows);
    const int c = blockIdx.y * 256 + threadIdx.x;
    A acc[K];
#pragma unroll
    for (int j = 0; j < K; j++) acc[j] = 0;
    for (int ib = i0; ib < i1; ib += 32) {
        const int nr = min(32, i1 - ib);
        __syncthreads();
        for (int e = threadIdx.x; e < nr * K; e += 256) {
            const int r = e / K;
            A v = X[(size_t)(ib + r) * K + (e % K)];
            if (rscale) v *= (A)rscale[ib + r];
            (&xs[0][0])[e] = v;
            if (xs_out && blockIdx.y == 0) xs_out[(size_t)ib * K + e] = v;
        }
        __syncthreads();
        if (c < ldw) {
            for (int r = 0; r < nr; r++) {
                const A wv = wval<TS>(W[(size_t)(ib + r) * ldw + c]);
#pragma unroll
                for (int j = 0; j < K; j++) acc[j] = fma(wv, xs[r][j], acc[j]);
            }
        }
    }
    if (c < ldw) {
        A* o = part + ((size_t)blockIdx.x * ldw + c) * K;
#pragma unroll
        for (int j = 0; j < K; j++) o[j] = acc[j];
    }
}

// out(c, j) = cscale_c (sum_b part[b][c * K + j] + sum_k C_kc Xs(k, j)) in
// float64 (the input of the F^-1 solve); C is the sparse float32 correction
// of a float16 W (CSC)
template <typename A, int K>
__global__ void kb_wt_reduce(int nb, int ldw, int nm, const A* __restrict__ part, const float* __restrict__ cscale,
                             const int* __restrict__ ccp, const int* __restrict__ crow,
                             const float* __restrict__ cval, const A* __restrict__ xs, double* out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nm * K) return;
    const int c = e / K, j = e % K;
    A v = 0;
    for (int b = 0; b < nb; b++) v += part[((size_t)b * ldw + c) * K + j];
    if (ccp)
        for (int k = ccp[c]; k < ccp[c + 1]; k++) v = fma((A)cval[k], xs[(size_t)crow[k] * K + j], v);
    out[e] = cscale ? (double)v * (double)cscale[c] : (double)v;
}

// Ds(c, j) = cscale_c D(c, j) in the compute type, zero on the padding
// columns c >= nm (c < ldw)
template <typename A, int K>
__global__ void kb_d_scaled(int nm, int ldw, const double* __restrict__ D, const float* __restrict__ cscale, A* Ds) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ldw * K) return;
    const int c = e / K;
    Ds[e] = (c < nm) ? (A)(cscale ? D[e] * (double)cscale[c] : D[e]) : (A)0;
}

// out(i, :) = (V(i, :)) + rscale_i (sum_c W(i, c) Ds(c, :) + sum_k C_ik Ds(col_k, :)):
// 32 rows of W and 32-column chunks staged in shared memory; thread (r, g)
// computes row r, columns g*K/8 .. g*K/8 + K/8 - 1.
template <typename TS, typename A, int K>
__global__ void __launch_bounds__(256) kb_w_d(int n, int ldw, const TS* __restrict__ W, const A* __restrict__ Ds,
                                              const float* __restrict__ rscale, const int* __restrict__ crp,
                                              const int* __restrict__ ccol, const float* __restrict__ cval,
                                              const A* V, A* out) {
    constexpr int CG = K / 8, CC = 32;
    __shared__ A ws[32][CC + 1];
    __shared__ __align__(16) A dsm[CC][K];
    const int i0 = blockIdx.x * 32;
    const int r = threadIdx.x / 8, g = threadIdx.x % 8;
    A acc[CG];
#pragma unroll
    for (int q = 0; q < CG; q++) acc[q] = 0;
    for (int c0 = 0; c0 < ldw; c0 += CC) {
        const int cn = min(CC, ldw - c0);
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * CC; e += 256) {
            const int rr = e / CC, cc = e % CC;
            ws[rr][cc] = (i0 + rr < n && cc < cn) ? wval<TS>(W[(size_t)(i0 + rr) * ldw + c0 + cc]) : (A)0;
        }
        for (int e = threadIdx.x; e < CC * K; e += 256)
            (&dsm[0][0])[e] = (e / K < cn) ? Ds[(size_t)c0 * K + e] : (A)0;
        __syncthreads();
#pragma unroll 4
        for (int cc = 0; cc < CC; cc++) {
            const A wv = ws[r][cc];
#pragma unroll
            for (int q = 0; q < CG; q++) acc[q] = fma(wv, dsm[cc][g * CG + q], acc[q]);
        }
    }
    const int i = i0 + r;
    if (i >= n) return;
    if (crp)
        for (int k = crp[i]; k < crp[i + 1]; k++) {
            const A cv = (A)cval[k];
            const A* dr = Ds + (size_t)ccol[k] * K + g * CG;
#pragma unroll
            for (int q = 0; q < CG; q++) acc[q] = fma(cv, dr[q], acc[q]);
        }
    const A sc = rscale ? (A)rscale[i] : (A)1;
#pragma unroll
    for (int q = 0; q < CG; q++) {
        const size_t e = (size_t)i * K + g * CG + q;
        out[e] = (V ? V[e] : (A)0) + sc * acc[q];
    }
}

// ---------------------------------------------- tensor-core operand prep
// Bt (2K x n, 16-bit, n contiguous, row stride ldb): rows j < K the high part, rows K + j
// the low part of Xs(:, j) = S_r X(:, j) 2^-e_j, where 2^e_j >= max_i
// |Xs(i, j)| (a power of two from the column maxima colmax, so the scaled
// values lie in [-1, 1] and the low parts stay in the normal range of
// float16 down to 2^-14 of the column maximum)
__device__ __forceinline__ float pow2_ceil_inv(float mx) {
    if (!(mx > 0.f)) return 1.f;
    int e;
    frexpf(mx, &e);        // mx = f 2^e, f in [0.5, 1)
    return ldexpf(1.f, -e);
}

// max |S_r X(:, j)| per column as float bits (non-negative floats order
// like their bit patterns): block maxima in shared memory, one atomic per
// block and column
template <int K>
__global__ void __launch_bounds__(256) kb_colmax(int n, const float* __restrict__ X, const float* __restrict__ rscale,
                                                 unsigned* mx) {
    __shared__ unsigned bm[K];
    if (threadIdx.x < K) bm[threadIdx.x] = 0u;
    __syncthreads();
    float tm[4] = {0.f, 0.f, 0.f, 0.f};
    int cc = 0;
    ROW_LOOP(float, K) {
        float v[4];
        ldv(X + (size_t)i * K + c0, v);
        const float sc = rscale ? rscale[i] : 1.f;
#pragma unroll
        for (int j = 0; j < 4; j++) tm[j] = fmaxf(tm[j], fabsf(v[j]) * sc);
        cc = c0;
    }
    {
        const int cl = ((threadIdx.x & 31) % RM<float, K>::TPR) * 4;
        (void)cc;
#pragma unroll
        for (int j = 0; j < 4; j++) atomicMax(bm + cl + j, __float_as_uint(tm[j]));
    }
    __syncthreads();
    if (threadIdx.x < K) atomicMax(mx + threadIdx.x, bm[threadIdx.x]);
}

template <typename H, int K>
__global__ void kb_split16(int n, int ldb, const float* __restrict__ X, const float* __restrict__ rscale,
                           const unsigned* __restrict__ mx, H* __restrict__ Bt) {
    __shared__ float t[32][K + 1];
    const int i0 = blockIdx.x * 32;
    for (int e = threadIdx.x; e < 32 * K; e += blockDim.x) {
        const int r = e / K, c = e % K, i = i0 + r;
        float v = 0.f;
        if (i < n) {
            v = X[(size_t)i * K + c] * pow2_ceil_inv(__uint_as_float(mx[c]));
            if (rscale) v *= rscale[i];
        }
        t[r][c] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * K; e += blockDim.x) {
        const int c = e / 32, r = e % 32, i = i0 + r;
        if (i >= n) continue;
        const float v = t[r][c];
        H hi, lo;
        if constexpr (std::is_same<H, __half>::value) {
            hi = __float2half_rn(v);
            lo = __float2half_rn(v - __half2float(hi));
        } else {
            hi = __float2bfloat16_rn(v);
            lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        }
        Bt[(size_t)c * ldb + i] = hi;
        Bt[(size_t)(K + c) * ldb + i] = lo;
    }
}

// Dt (2K x ldw) from Ds (ldw x K float32, cscale applied, zero padding
// columns): Ds 2^-f_j split in two 16-bit parts, 2^f_j >= max_c |Ds(c, j)|
// from the column maxima mx (kb_colmax over Ds); also stores 2^f_j.
template <typename H, int K>
__global__ void kb_split16_d(int ldw, const float* __restrict__ Ds, const unsigned* __restrict__ mx,
                             H* __restrict__ Dt, float* __restrict__ dscale) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ldw * K) return;
    const int j = e / ldw, c = e % ldw;
    const float inv = pow2_ceil_inv(__uint_as_float(mx[j]));
    const float v = Ds[(size_t)c * K + j] * inv;
    H hi, lo;
    if constexpr (std::is_same<H, __half>::value) {
        hi = __float2half_rn(v);
        lo = __float2half_rn(v - __half2float(hi));
    } else {
        hi = __float2bfloat16_rn(v);
        lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
    Dt[(size_t)j * ldw + c] = hi;
    Dt[(size_t)(K + j) * ldw + c] = lo;
    if (c == 0) dscale[j] = 1.f / inv;
}

// out(c, j) = cscale_c (2^e_j sum_b part[b][c * K + j] + sum_k C_kc S_r X(k, j)),
// float64: one block per column c; the column's correction entries are
// spread over the block (K / 4 threads per entry, 16 bytes of X each) and
// their sums meet in shared memory in a fixed order
template <int K>
__global__ void __launch_bounds__(256) kb_wt_reduce_umma(int nb, int ldw, int nm, const float* __restrict__ part,
                                                         const unsigned* __restrict__ mx,
                                                         const float* __restrict__ cscale,
                                                         const int* __restrict__ ccp, const int* __restrict__ crow,
                                                         const float* __restrict__ cval, const float* __restrict__ X,
                                                         const float* __restrict__ rscale, double* out) {
    constexpr int TPE = K / 4, EPB = 256 / TPE;
    __shared__ float red[EPB][K];
    const int c = blockIdx.x;
    const int slot = threadIdx.x / TPE, j0 = (threadIdx.x % TPE) * 4;
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    if (ccp) {
        const int k1 = ccp[c + 1];
#pragma unroll 4
        for (int k = ccp[c] + slot; k < k1; k += EPB) {
            const int i = crow[k];
            const float cv = cval[k] * (rscale ? rscale[i] : 1.f);
            float xv[4];
            ldv(X + (size_t)i * K + j0, xv);
#pragma unroll
            for (int j = 0; j < 4; j++) a[j] = fmaf(cv, xv[j], a[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < 4; j++) red[slot][j0 + j] = a[j];
    __syncthreads();
    if (threadIdx.x < K) {
        const int j = threadIdx.x;
        float v = 0.f;
        for (int b = 0; b < nb; b++) v += part[((size_t)b * ldw + c) * K + j];
        v *= 1.f / pow2_ceil_inv(__uint_as_float(mx[j]));
        float corr = 0.f;
        for (int t = 0; t < EPB; t++) corr += red[t][j];
        v += corr;
        out[(size_t)c * K + j] = cscale ? (double)v * (double)cscale[c] : (double)v;
    }
}

// out(i, :) = V(i, :) + rscale_i (2^f_j acc(i, j) + sum_k C_ik Ds(col_k, j))
template <int K>
__global__ void __launch_bounds__(256) kb_wd_finish_umma(int n, const float* __restrict__ acc,
                                                         const float* __restrict__ dscale,
                                                         const float* __restrict__ rscale, const int* __restrict__ crp,
                                                         const int* __restrict__ ccol, const float* __restrict__ cval,
                                                         const float* __restrict__ Ds, const float* V, float* out) {
    ROW_LOOP(float, K) {
        const size_t e = (size_t)i * K + c0;
        float v[4], d[4];
        ldv(acc + e, v);
        ldv(dscale + c0, d);
#pragma unroll
        for (int j = 0; j < 4; j++) v[j] *= d[j];
        if (crp)
            for (int k = crp[i]; k < crp[i + 1]; k++) {
                float dv[4];
                ldv(Ds + (size_t)ccol[k] * K + c0, dv);
                const float cv = cval[k];
#pragma unroll
                for (int j = 0; j < 4; j++) v[j] = fmaf(cv, dv[j], v[j]);
            }
        if (rscale) {
            const float r = rscale[i];
#pragma unroll
            for (int j = 0; j < 4; j++) v[j] *= r;
        }
        if (V) {
            float t[4];
            ldv(V + e, t);
#pragma unroll
            for (int j = 0; j < 4; j++) v[j] += t[j];
        }
        stv(out + e, v);
    }
}

// ------------------------------------------------ device-driven PCG control
// Control words of a graph-driven block PCG: ctl[0] iterations done,
// ctl[1] rtol, ctl[2] maxit, ctl[3] status (0, AWG_ERR_BREAKDOWN,
// AWG_ERR_MAXIT), ctl[4] 1 when some column is a candidate in this
// iteration; its[c] / rel[c] the iteration at which column c stopped and its
// relative residual (the true one where it stopped converged).
template <int K>
__global__ void kb_pcg_init(int nrhs, double* sc, double* ctl, double rtol, double maxit, int* its, double* rel) {
    const int c = threadIdx.x;
    if (c < K) {
        const double bb = sc[B_BB * K + c];
        const bool a = c < nrhs && bb > 0.0;
        sc[B_ACT * K + c] = a ? 1.0 : 0.0;
        sc[B_CAND * K + c] = 0.0;
        its[c] = 0;
        rel[c] = 0.0;
    }
    if (c == 0) {
        ctl[0] = 0.0;
        ctl[1] = rtol;
        ctl[2] = maxit;
        ctl[3] = 0.0;
        ctl[4] = 0.0;
    }
}

// After an x, r update: one more iteration; an active column whose p^T A p
// is not positive (breakdown) stops; one whose recurrence residual reached
// rtol becomes a candidate (ctl[4] = 1), to be confirmed on its true
// residual b - A x (kb_resid, kb_coldot gated by ctl[4], then
// kb_pcg_confirm), as the host-driven solve does (Section 1; the recurrence
// residual can drift below the true one).
template <int K>
__global__ void kb_pcg_cond(double* sc, double* ctl, int* its, double* rel) {
    const int c = threadIdx.x;
    const int it = (int)ctl[0] + 1;
    const double rtol = ctl[1];
    const int maxit = (int)ctl[2];
    bool cand = false;
    int status = 0;
    if (c < K && sc[B_ACT * K + c] != 0.0) {
        const double pq = sc[B_PQ * K + c];
        const double r = sqrt(sc[B_RR * K + c] / sc[B_BB * K + c]);
        if (!(pq > 0.0) || !isfinite(pq)) {
            sc[B_ACT * K + c] = 0.0;
            its[c] = it;
            rel[c] = r;
            status = AWG_ERR_BREAKDOWN;
        } else if (r <= rtol) {
            sc[B_CAND * K + c] = 1.0;
            cand = true;
        } else if (it >= maxit) {
            its[c] = it;
            rel[c] = r;
            status = AWG_ERR_MAXIT;
        }
    }
    const int anyc = __syncthreads_or(cand);
    const int st = __syncthreads_or(status == AWG_ERR_BREAKDOWN) ? AWG_ERR_BREAKDOWN
                   : (__syncthreads_or(status == AWG_ERR_MAXIT) ? AWG_ERR_MAXIT : 0);
    if (c == 0) {
        ctl[0] = (double)it;
        ctl[4] = anyc ? 1.0 : 0.0;
        if (st && ctl[3] == 0.0) ctl[3] = (double)st;
    }
}

// Candidates whose true relative residual (sc[B_TR], when ctl[4] is set)
// is <= rtol stop, with that residual; so does one whose recurrence
// residual fell below 1e-6 rtol (stagnation: status AWG_ERR_MAXIT); the
// others go on.  With `set`, the loop condition of the enclosing graph
// becomes "some column active and iterations < maxit"; `add` kernels per
// loop body go to *launches (profiling).
template <int K>
__global__ void kb_pcg_confirm(double* sc, double* ctl, int* its, double* rel, cudaGraphConditionalHandle hc,
                               int set, unsigned long long* launches, int add) {
    const int c = threadIdx.x;
    const int it = (int)ctl[0];
    const double rtol = ctl[1];
    const int maxit = (int)ctl[2];
    bool active = false;
    int status = 0;
    if (c < K && sc[B_ACT * K + c] != 0.0) {
        active = true;
        if (ctl[4] != 0.0 && sc[B_CAND * K + c] != 0.0) {
            sc[B_CAND * K + c] = 0.0;
            const double r = sqrt(sc[B_RR * K + c] / sc[B_BB * K + c]);
            const double tr = sqrt(sc[B_TR * K + c] / sc[B_BB * K + c]);
            if (tr <= rtol || r <= 1e-6 * rtol) {
                sc[B_ACT * K + c] = 0.0;
                its[c] = it;
                rel[c] = tr;
                active = false;
                if (tr > rtol) status = AWG_ERR_MAXIT;
            } else if (it >= maxit) {
                its[c] = it;
                rel[c] = tr;
                status = AWG_ERR_MAXIT;
            }
        }
    }
    const int any = __syncthreads_or(active && it < maxit);
    const int st = __syncthreads_or(status == AWG_ERR_MAXIT);
    if (c == 0) {
        if (st && ctl[3] == 0.0) ctl[3] = (double)AWG_ERR_MAXIT;
        ctl[4] = 0.0;
        if (set) cudaGraphSetConditional(hc, any ? 1u : 0u);
        if (launches && add) atomicAdd(launches, (unsigned long long)add);
    }
}

// iterations and residuals of the nrhs columns and the status to the
// caller's arrays
__global__ void kb_pcg_fini(int nrhs, const int* __restrict__ its, const double* __restrict__ rel,
                            const double* __restrict__ ctl, int* d_its, double* d_rel, int* d_status) {
    const int c = threadIdx.x;
    if (c < nrhs) {
        if (d_its) d_its[c] = its[c];
        if (d_rel) d_rel[c] = rel[c];
    }
    if (c == 0 && d_status) *d_status = (int)ctl[3];
}

// ===================================================================== host
namespace {

template <typename T>
struct BView {
    // preconditioner block vectors (n x K), local arenas (sum_ns x K)
    T *rin, *x1, *t, *u, *q, *out, *tmpw, *loc, *loc2, *cm, *cf;
    // coarse vectors, float64 (n0 x K, n_- x K)
    double *y0, *y2, *c1, *c2, *w0, *dd, *w1, *y0d;
    double *dpm, *dps;  // split partials of the float64 coarse GEMMs (main, side stream)
    void *ozxm, *ozxs;  // right-hand-side slices of the tensor-core coarse products (main, side)
    T* tgp;             // p-split partials of the block-sparse transposed products
    // W passes
    void* part;    // row-block partials (compute type)
    void* xs;      // S_r X (compute type), n x K
    void* ds;      // S_c D (compute type), ldw x K
    void* bt;      // 16-bit split operands: 2K x n
    void* dt;      //                        2K x ldw
    float* wacc;   // tensor-core W d accumulators, n x K
    float* lt;     // tensor-core local solves: TF32 hi / lo right-hand-side images
    float* dscale;
    unsigned* mx;  // column maxima (float bits) of S_r X
    unsigned* mx2; //                             of S_c D
    int* err;
    // PCG (float64, n x K)
    double *pb, *px, *pr, *pp, *pq, *pz;
    double *sc, *red;
    unsigned* cnt;
    // graph-driven PCG: iteration, rtol, maxit, status; per-column iterations
    // and residuals; kernels launched by graph loop bodies (profiling)
    double* ctl;
    int* gits;
    double* grel;
    unsigned long long* glaunch;
};

constexpr int WT_SPLITS_MAX = 64;

size_t carve_block(const Handle* h, char* base, BView<double>* vd, BView<float>* vf) {
    // one layout serves both element types: every region is sized for the
    // float64 form (the float32 form uses the first half of each)
    char* p = base;
    auto take = [&](size_t bytes) { char* r = p; p += (bytes + 255) / 256 * 256; return r; };
    const size_t K = BLK_KMAX;
    const size_t n = h->n, n0 = std::max(1, h->n0), nm = std::max(1, h->n_minus);
    const size_t ldw = std::max(8, h->ldw);
    BView<double> d{};
    d.rin = (double*)take(n * K * 8); d.x1 = (double*)take(n * K * 8); d.t = (double*)take(n * K * 8);
    d.u = (double*)take(n * K * 8); d.q = (double*)take(n * K * 8); d.out = (double*)take(n * K * 8);
    d.tmpw = (double*)take(n * K * 8);
    d.loc = (double*)take((size_t)h->sum_ns * K * 8); d.loc2 = (double*)take((size_t)h->sum_ns * K * 8);
    d.cm = (double*)take((size_t)std::max(1, h->n_minus_all) * K * 8);
    d.cf = (double*)take(std::max(n0, nm) * K * 8);
    d.y0 = (double*)take(n0 * K * 8); d.y2 = (double*)take(n0 * K * 8); d.c1 = (double*)take(n0 * K * 8);
    d.c2 = (double*)take(n0 * K * 8); d.y0d = (double*)take(std::max(n0, nm) * K * 8);
    d.w0 = (double*)take(nm * K * 8); d.dd = (double*)take(nm * K * 8); d.w1 = (double*)take(nm * K * 8);
    // both streams' partials hold a product with E^-1 or with F^-1 (H_3,hyb
    // runs its F^-1 products on the main stream)
    const size_t dpart = std::max((size_t)DG_SMAX * std::max(n0, nm) * K,
                                  oz_part_elems((int)std::max(n0, nm), (int)K));
    d.dpm = (double*)take(dpart * 8);
    d.dps = (double*)take(dpart * 8);
    d.ozxm = take(oz_xs_bytes((int)std::max(n0, nm), (int)K));
    d.ozxs = take(oz_xs_bytes((int)std::max(n0, nm), (int)K));
    d.tgp = (double*)take((size_t)TG_PS * std::max<size_t>(n0, std::max(1, h->n_minus_all)) * K * 8);
    d.part = take((size_t)WT_SPLITS_MAX * ldw * K * 8);
    d.xs = take(n * K * 8);
    d.ds = take(ldw * K * 8);
    d.bt = take(2 * K * ((n + 63) / 64 * 64) * 2);
    d.dt = take(2 * K * ldw * 2);
    d.wacc = (float*)take(n * K * 4);
    d.dscale = (float*)take(K * 4);
    d.mx = (unsigned*)take(K * 4);
    d.mx2 = (unsigned*)take(K * 4);
    d.err = (int*)take(64);
    {
        int64_t kcs = 0;
        for (int t = 0; t < h->N; t++) kcs += (h->h_ns[t] + 31) / 32;
        d.lt = (float*)take((size_t)kcs * 2 * K * 32 * 4);
    }
    d.pb = (double*)take(n * K * 8); d.px = (double*)take(n * K * 8); d.pr = (double*)take(n * K * 8);
    d.pp = (double*)take(n * K * 8); d.pq = (double*)take(n * K * 8); d.pz = (double*)take(n * K * 8);
    d.sc = (double*)take(B_NSC * K * 8);
    d.red = (double*)take((size_t)(CS_PMAX + 64) * K * 8);  // block partials, then group sums
    d.cnt = (unsigned*)take(256);                              // colsum_grid tickets (global, per group)
    d.ctl = (double*)take(8 * 8);
    d.gits = (int*)take(K * 4);
    d.grel = (double*)take(K * 8);
    d.glaunch = (unsigned long long*)take(64);
    if (vd) *vd = d;
    if (vf) {
        BView<float> f{};
        f.rin = (float*)d.rin; f.x1 = (float*)d.x1; f.t = (float*)d.t; f.u = (float*)d.u; f.q = (float*)d.q;
        f.out = (float*)d.out; f.tmpw = (float*)d.tmpw; f.loc = (float*)d.loc; f.loc2 = (float*)d.loc2;
        f.cm = (float*)d.cm; f.cf = (float*)d.cf;
        f.y0 = d.y0; f.y2 = d.y2; f.c1 = d.c1; f.c2 = d.c2; f.y0d = d.y0d; f.w0 = d.w0; f.dd = d.dd; f.w1 = d.w1;
        f.dpm = d.dpm; f.dps = d.dps; f.ozxm = d.ozxm; f.ozxs = d.ozxs; f.tgp = (float*)d.tgp;
        f.part = d.part; f.xs = d.xs; f.ds = d.ds; f.bt = d.bt; f.dt = d.dt; f.wacc = d.wacc; f.lt = d.lt;
        f.dscale = d.dscale; f.mx = d.mx; f.mx2 = d.mx2; f.err = d.err;
        f.pb = d.pb; f.px = d.px; f.pr = d.pr; f.pp = d.pp; f.pq = d.pq; f.pz = d.pz;
        f.sc = d.sc; f.red = d.red; f.cnt = d.cnt;
        f.ctl = d.ctl; f.gits = d.gits; f.grel = d.grel; f.glaunch = d.glaunch;
        *vf = f;
    }
    return (size_t)(p - base);
}

template <typename T> T* fl(const DevBuf& d64, const DevBuf& d32);
template <> double* fl<double>(const DevBuf& d64, const DevBuf&) { return (double*)d64.p; }
template <> float* fl<float>(const DevBuf&, const DevBuf& d32) { return (float*)d32.p; }

int grid_rows(int n, int rpb) { return std::max(1, std::min((n + rpb - 1) / rpb, 152 * 8)); }

// Blocks of 256 threads per SM that the kernel `kern` keeps resident (its
// registers and shared memory decide; at most 8), looked up once per kernel.
int resident_blocks(const void* kern) {
    static std::mutex mu;
    static std::unordered_map<const void*, int> cache;
    std::lock_guard<std::mutex> lock(mu);
    const auto it = cache.find(kern);
    if (it != cache.end()) return it->second;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 256, 0) != cudaSuccess) {
        cudaGetLastError();
        b = 8;
    }
    b = std::max(1, std::min(8, b));
    cache[kern] = b;
    return b;
}

// Grid of a grid-stride row kernel: one wave of resident blocks (a grid of
// 8 blocks per SM for a kernel that keeps 6 resident would run 1.33 waves)
unsigned grid_for(const void* kern, int n, int rpb) {
    return (unsigned)std::max(1, std::min((n + rpb - 1) / rpb, 152 * resident_blocks(kern)));
}

}  // namespace

// A block slot: workspace, the side stream and events of its apply, and
// its cache of loop graphs.  Slot 0 is the handle's main set; slot 1 the
// second set used by wide graph-driven solves.
struct Slot {
    char* ws;
    cudaStream_t main, side;
    cudaEvent_t fork, mid, join;
    cudaGraph_t* graph;
    cudaGraphExec_t* exec;
};
Slot slot0(Handle* h) {
    return {(char*)h->bws.p, h->hp, h->side, h->ev_fork, h->ev_mid, h->ev_join, h->bg_graph, h->bg_exec};
}
Slot slot1(Handle* h) {
    return {(char*)h->bws2.p, h->hp2, h->side2, h->ev2_fork, h->ev2_mid, h->ev2_join, h->bg2_graph, h->bg2_exec};
}

UmmaLocal ul_of(const Handle* h) {
    UmmaLocal u;
    u.N = h->N;
    u.ntiles = h->ul_ntiles;
    u.max_kc = h->ul_maxkc;
    u.max_tiles_sub = h->ul_maxtiles;
    u.sub_ptr = (const int*)h->sub_ptr.p;
    u.sub_idx = (const int*)h->sub_idx.p;
    u.Gt = (const float*)h->ul_gt.p;
    u.gt_off = (const int64_t*)h->ul_gtoff.p;
    u.kc_prefix = (const int64_t*)h->ul_kcpre.p;
    u.tile_sub = (const int*)h->ul_tsub.p;
    u.tile_rt = (const int*)h->ul_trt.p;
    return u;
}

// Float32 copies of the small operators the float32 block apply reads (A's
// values, V^s_-, |Lambda^s_-|, Z), the workspace, and the side stream's
// error word: built on the first block call of a handle.
awg_status block_prepare(Handle* h) {
    if (h->bws.p) return AWG_OK;
    cudaStream_t s = h->stream;
    auto cvt = [&](DevBuf& dst, const DevBuf& src, size_t len, bool neg) -> awg_status {
        AWG_TRY(dalloc(h, dst, std::max<size_t>(len, 1) * 4));
        if (len == 0) return AWG_OK;
        std::vector<double> hv(len);
        std::vector<float> fv(len);
        AWG_CUDA(cudaMemcpy(hv.data(), src.p, len * 8, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < len; i++) fv[i] = (float)(neg ? -hv[i] : hv[i]);
        AWG_CUDA(cudaMemcpy(dst.p, fv.data(), len * 4, cudaMemcpyHostToDevice));
        return AWG_OK;
    };
    AWG_TRY(cvt(h->bval32, h->val, (size_t)h->nnz, false));
    AWG_TRY(cvt(h->bvm32, h->Vm, (size_t)(h->h_vm_off.empty() ? 0 : h->h_vm_off[h->N]), false));
    AWG_TRY(cvt(h->blam32, h->lam_m, (size_t)h->n_minus_all, true));   // |Lambda_-| = -Lambda_-
    AWG_TRY(dalloc(h, h->blam64, (size_t)std::max(1, h->n_minus_all) * 8));
    if (h->n_minus_all > 0) {
        std::vector<double> hv(h->n_minus_all);
        AWG_CUDA(cudaMemcpy(hv.data(), h->lam_m.p, hv.size() * 8, cudaMemcpyDeviceToHost));
        for (double& v : hv) v = -v;
        AWG_CUDA(cudaMemcpy(h->blam64.p, hv.data(), hv.size() * 8, cudaMemcpyHostToDevice));
    }
    AWG_TRY(cvt(h->bz32, h->Z, (size_t)(h->h_z_off.empty() ? 0 : h->h_z_off[h->N]), false));
    if (h->prec[AWG_MIXED_FP32].G.p && h->opt.block_tensor_cores && umma_available()) {
        // 16 KB images of G_s, 128-row tiles by 32-column chunks
        const int N = h->N;
        std::vector<int64_t> gtoff(N), kcpre(N + 1, 0);
        std::vector<int> tsub, trt;
        int64_t tiles = 0;
        int maxkc = 0, maxtiles = 0;
        for (int t = 0; t < N; t++) {
            const int m = h->h_ns[t], RT = (m + 127) / 128, KC = (m + 31) / 32;
            gtoff[t] = tiles;
            tiles += (int64_t)RT * KC;
            kcpre[t + 1] = kcpre[t] + KC;
            maxkc = std::max(maxkc, KC);
            maxtiles = std::max(maxtiles, RT * KC);
            for (int r = 0; r < RT; r++) { tsub.push_back(t); trt.push_back(r); }
        }
        AWG_TRY(dalloc(h, h->ul_gt, (size_t)tiles * 16384));
        AWG_TRY(upload(h, h->ul_gtoff, gtoff.data(), N * 8));
        AWG_TRY(upload(h, h->ul_kcpre, kcpre.data(), (N + 1) * 8));
        AWG_TRY(upload(h, h->ul_tsub, tsub.data(), tsub.size() * 4));
        AWG_TRY(upload(h, h->ul_trt, trt.data(), trt.size() * 4));
        h->ul_ntiles = (int)tsub.size();
        h->ul_maxkc = maxkc;
        h->ul_maxtiles = maxtiles;
        AWG_TRY(umma_local_tiles(ul_of(h), (int64_t*)h->g32_off.p, (float*)h->prec[AWG_MIXED_FP32].G.p, s));
        AWG_CUDA(cudaStreamSynchronize(s));
    }
    const size_t bytes = carve_block(h, nullptr, nullptr, nullptr);
    AWG_TRY(dalloc(h, h->bws, bytes));
    AWG_CUDA(cudaMemset(h->bws.p, 0, bytes));
    return AWG_OK;
}

// bfloat16 slices of every dense coarse inverse built so far (E^-1 during
// setup, for the W solve; F^-1 and the H_3,inex inner inverses once they
// exist) for the float64-accurate tensor-core products (ozaki.cu); a no-op
// once all are built or with coarse_tensor_cores = 0.  Not inside a stream
// capture (allocates and synchronises).
awg_status oz_prepare(Handle* h) {
    if (!h->opt.coarse_tensor_cores || !umma_available()) return AWG_OK;
    cudaStream_t s = h->stream;
    bool any = false;
    auto slice = [&](int k, const DevBuf& M, int dim) -> awg_status {
        if (!M.p || dim < 1 || h->oz_dim[k]) return AWG_OK;
        OzMat m;
        AWG_TRY(oz_slice_matrix((const double*)M.p, dim, h->oz_q[k], h->oz_ex[k], h, s, &m));
        h->oz_dim[k] = dim;
        any = true;
        return AWG_OK;
    };
    AWG_TRY(slice(0, h->Einv, h->n0));
    for (int p = 0; p < AWG_NPREC; p++) {
        AWG_TRY(slice(1 + p, h->prec[p].Finv, h->n_minus));
        AWG_TRY(slice(5 + p, h->prec[p].inexInv, h->n_minus));
    }
    if (any) AWG_CUDA(cudaStreamSynchronize(s));
    return AWG_OK;
}

// The tensor-core slices of the dense coarse inverse at Mx, if built.
static bool oz_of(const Handle* h, const double* Mx, OzMat* out) {
    int k = -1;
    if (Mx == (const double*)h->Einv.p) k = 0;
    for (int p = 0; p < AWG_NPREC && k < 0; p++) {
        if (Mx == (const double*)h->prec[p].Finv.p) k = 1 + p;
        else if (Mx == (const double*)h->prec[p].inexInv.p) k = 5 + p;
    }
    if (k < 0 || !h->oz_dim[k] || !Mx) return false;
    const int dim = h->oz_dim[k];
    out->q = h->oz_q[k].p;
    out->ex = (const int*)h->oz_ex[k].p;
    out->dim = dim;
    out->dimp = (dim + 127) / 128 * 128;
    out->ldk = (dim + 63) / 64 * 64;
    return true;
}

namespace {

template <typename T, int K>
struct BlockApply {
    Handle* h;
    BView<T> v;
    Slot sl;
    using A = T;

    static dim3 rows_grid(const void* kern, int n) { return dim3(grid_for(kern, n, RM<T, K>::RPB)); }

    const T* aval() const { return fl<T>(h->val, h->bval32); }
    const T* vm() const { return fl<T>(h->Vm, h->bvm32); }
    const T* lam() const { return fl<T>(h->blam64, h->blam32); }
    const T* zb() const { return fl<T>(h->Z, h->bz32); }

    awg_status cvt_d2t(const double* a, T* b, size_t len, cudaStream_t s) {
        if (len == 0) return AWG_OK;
        kb_cvt<double, T><<<(unsigned)((len + 255) / 256), 256, 0, s>>>(len, a, b);
        AWG_LAUNCH();
        return AWG_OK;
    }
    awg_status cvt_t2d(const T* a, double* b, size_t len, cudaStream_t s) {
        if (len == 0) return AWG_OK;
        kb_cvt<T, double><<<(unsigned)((len + 255) / 256), 256, 0, s>>>(len, a, b);
        AWG_LAUNCH();
        return AWG_OK;
    }

    // C = wsign w .* (B^T X) per subdomain (ncol_total columns in all)
    awg_status tgemv(const int* colptr, const int64_t* boff, const T* B, int maxc, int ncol_total, const T* X,
                     const T* w, T wsign, T* C, cudaStream_t s) {
        if (maxc == 0 || ncol_total == 0) return AWG_OK;
        ProfScope ps_(h, AWG_PROF_SUBDOMAIN, s);
        kb_tgemv2<T, K><<<dim3(h->N, TG_PS), 256, 0, s>>>((int*)h->sub_ptr.p, (int*)h->sub_idx.p, colptr, boff, B, X,
                                                          ncol_total, v.tgp);
        AWG_LAUNCH();
        const size_t len = (size_t)ncol_total * K;
        kb_tg_sum<T, K><<<(unsigned)((len + 255) / 256), 256, 0, s>>>(ncol_total, v.tgp, w, wsign, C);
        AWG_LAUNCH();
        extra_launches(h, 1);
        return AWG_OK;
    }

    // Y = Yin + sign A_+ X
    awg_status aplus(const T* X, T* Y, const T* Yin, T sign, cudaStream_t s) {
        const bool vmb = h->n_minus_all > 0;
        if (vmb) {
            const int maxc = *std::max_element(h->h_nm.begin(), h->h_nm.end());
            AWG_TRY(tgemv((int*)h->nm_ptr.p, (int64_t*)h->vm_off.p, vm(), maxc, h->n_minus_all, X, lam(), (T)1,
                          v.cm, s));
        }
        ProfScope ps_(h, AWG_PROF_SPMV, s);
        kb_aplus<T, K><<<rows_grid((const void*)kb_aplus<T, K>, h->n), 256, 0, s>>>(
            h->n, (int*)h->rowptr.p, (int*)h->colidx.p, aval(), X, (int*)h->inc_ptr.p, (int*)h->inc_pos.p,
            (int*)h->inc_sub.p, (int*)h->sub_ptr.p, (int*)h->nm_ptr.p, (int64_t*)h->vm_off.p, vm(),
            vmb ? v.cm : nullptr, Yin, sign, Y);
        AWG_LAUNCH();
        return AWG_OK;
    }

    // c (float64, n0 x K) = Z^T X
    awg_status zt(const T* X, double* c, cudaStream_t s) {
        const int maxc = *std::max_element(h->h_modes.begin(), h->h_modes.end());
        if constexpr (std::is_same<T, double>::value) {
            return tgemv((int*)h->mode_ptr.p, (int64_t*)h->z_off.p, zb(), maxc, h->n0, X, nullptr, (T)1, c, s);
        } else {
            AWG_TRY(tgemv((int*)h->mode_ptr.p, (int64_t*)h->z_off.p, zb(), maxc, h->n0, X, nullptr, (T)1, v.cf, s));
            ProfScope ps_(h, AWG_PROF_VECTOR, s);
            return cvt_t2d(v.cf, c, (size_t)h->n0 * K, s);
        }
    }

    // Y = beta Y + alpha Z c + gamma V (+ V2), c float64
    awg_status zc(const double* c, T* Y, T alpha, T beta, const T* V, T gamma, const T* V2, cudaStream_t s) {
        const T* cc;
        if constexpr (std::is_same<T, double>::value) {
            cc = c;
        } else {
            ProfScope pc_(h, AWG_PROF_VECTOR, s);
            AWG_TRY(cvt_d2t(c, v.cf, (size_t)h->n0 * K, s));
            cc = v.cf;
        }
        ProfScope ps_(h, AWG_PROF_PROLONG, s);
        kb_blk_prolong<T, K><<<rows_grid((const void*)kb_blk_prolong<T, K>, h->n), 256, 0, s>>>(
            h->n, (int*)h->inc_ptr.p, (int*)h->inc_pos.p, (int*)h->inc_sub.p, (int*)h->sub_ptr.p,
            (int*)h->mode_ptr.p, (int64_t*)h->z_off.p, zb(), cc, Y, alpha, beta, V, gamma, V2);
        AWG_LAUNCH();
        return AWG_OK;
    }

    // Y = alpha M X + beta Sub (float64); part: the partial buffer of the
    // stream s (the main and side streams each own one)
    awg_status dense(int dim, const double* Mx, const double* X, double* Y, double alpha, const double* Sub,
                     double beta, double* part, cudaStream_t s) {
        if (dim == 0) return AWG_OK;
        ProfScope ps_(h, AWG_PROF_COARSE, s);
        OzMat om;
        if (oz_of(h, Mx, &om) && om.dim == dim) {
            // float64-accurate slice products on the tensor cores (ozaki.cu)
            AWG_TRY(oz_gemm(om, K, X, Y, alpha, Sub, beta, part == v.dpm ? v.ozxm : v.ozxs, part, v.err, s));
            extra_launches(h, 2);
            return AWG_OK;
        }
        const int tiles = (dim + DG_RB - 1) / DG_RB;
        const int bps = h->bt_dense[kidx] > 0 ? h->bt_dense[kidx] : 4;  // (autotuned) blocks per SM
        int S = std::max(1, std::min(DG_SMAX, (bps * 152 + tiles - 1) / tiles));
        int jlen = (dim + S - 1) / S;
        jlen = (jlen + DG_JC - 1) / DG_JC * DG_JC;
        S = (dim + jlen - 1) / jlen;
        kb_dense_part<K><<<dim3(tiles, S), 4 * K, 0, s>>>(dim, jlen, Mx, X, part);
        AWG_LAUNCH();
        const size_t len = (size_t)dim * K;
        kb_dense_sum<K><<<(unsigned)((len + 255) / 256), 256, 0, s>>>(dim, S, part, Y, alpha, Sub, beta);
        AWG_LAUNCH();
        extra_launches(h, 1);
        return AWG_OK;
    }

    // Y = H^NN X
    awg_status hnn(int prec, const T* X, T* Y, cudaStream_t s) {
        if constexpr (std::is_same<T, float>::value) {
            if (h->ul_ntiles > 0) {  // tensor cores: gather + TF32 split, then the tile GEMMs
                {
                    ProfScope ps_(h, AWG_PROF_LOCAL, s);
                    AWG_TRY(umma_local(ul_of(h), K, X, v.lt, v.loc2, v.err, s));
                    extra_launches(h, 1);
                }
                ProfScope ps_(h, AWG_PROF_PROLONG, s);
                kb_prolong<T, K><<<rows_grid((const void*)kb_prolong<T, K>, h->n), 256, 0, s>>>(h->n, (int*)h->inc_ptr.p, (int*)h->inc_pos.p, v.loc2,
                                                                Y, (T)1, (T)0, nullptr, (T)0);
                AWG_LAUNCH();
                return AWG_OK;
            }
        }
        {
            ProfScope ps_(h, AWG_PROF_PROLONG, s);
            const int64_t len = h->sum_ns * K;
            kb_gather<T, K><<<(unsigned)((len + 255) / 256), 256, 0, s>>>(h->sum_ns, (int*)h->sub_idx.p, X, v.loc);
        }
        AWG_LAUNCH();
        {
            ProfScope ps_(h, AWG_PROF_LOCAL, s);
            const dim3 g(h->N, (h->max_ns + LG<T, K>::ROWS - 1) / LG<T, K>::ROWS);
            if constexpr (std::is_same<T, double>::value) {
                kb_local_gemm<double, K><<<g, 128, 0, s>>>((int*)h->sub_ptr.p, (int64_t*)h->dense_off.p,
                                                           (double*)h->prec[AWG_FP64].G.p, 0, v.loc, v.loc2);
            } else {
                (void)prec;
                kb_local_gemm<float, K><<<g, 128, 0, s>>>((int*)h->sub_ptr.p, (int64_t*)h->g32_off.p,
                                                          (float*)h->prec[AWG_MIXED_FP32].G.p, 1, v.loc, v.loc2);
            }
        }
        AWG_LAUNCH();
        ProfScope ps_(h, AWG_PROF_PROLONG, s);
        kb_prolong<T, K><<<rows_grid((const void*)kb_prolong<T, K>, h->n), 256, 0, s>>>(h->n, (int*)h->inc_ptr.p, (int*)h->inc_pos.p, v.loc2, Y,
                                                        (T)1, (T)0, nullptr, (T)0);
        AWG_LAUNCH();
        return AWG_OK;
    }

    // H_2 X = Pi H_1 Pi^T X + Z E^-1 Z^T X (Thms. 3, 4; H_1 = H^NN or
    // H^AS_+), or H_1 X + Z E^-1 Z^T X (H^AS_+,ad), in two parts, so that
    // another stream's work can be issued between them: h2a computes
    // c1 = E^-1 Z^T X, h2b the rest (+ V2 once the event `wait` completed)
    awg_status h2a(const T* X, cudaStream_t s) {
        if (h->n0 == 0) return AWG_OK;
        AWG_TRY(zt(X, v.y0, s));                                                          // y0 = Z^T X
        return dense(h->n0, (double*)h->Einv.p, v.y0, v.c1, 1.0, nullptr, 0.0, v.dpm, s);  // c1 = E^-1 y0
    }
    awg_status h2b(int prec, const T* X, T* Y, cudaStream_t s, const T* V2 = nullptr, cudaEvent_t wait = nullptr) {
        if (h->n0 == 0) {
            AWG_TRY(hnn(prec, X, Y, s));
            if (V2) {
                if (wait) AWG_CUDA(cudaStreamWaitEvent(s, wait, 0));
                ProfScope ps_(h, AWG_PROF_VECTOR, s);
                const size_t len = (size_t)h->n * K;
                kb_add<T><<<(unsigned)((len + 255) / 256), 256, 0, s>>>(len, V2, Y);
                AWG_LAUNCH();
            }
            return AWG_OK;
        }
        const int n0 = h->n0;
        if (h->opt.h2 == AWG_H2_ASP_AD) {  // H^AS_+,ad (Thm. 3): Y = H_1 X + Z c1 (+ V2)
            AWG_TRY(hnn(prec, X, v.u, s));
            if (wait) AWG_CUDA(cudaStreamWaitEvent(s, wait, 0));
            return zc(v.c1, Y, (T)1, (T)0, v.u, (T)1, V2, s);
        }
        AWG_TRY(zc(v.c1, v.x1, (T)1, (T)0, nullptr, (T)0, nullptr, s));            // x1 = Z c1
        AWG_TRY(aplus(v.x1, v.t, X, (T)-1, s));                                    // t = X - A_+ x1
        AWG_TRY(hnn(prec, v.t, v.u, s));                                           // u = H^NN t
        AWG_TRY(aplus(v.u, v.q, nullptr, (T)1, s));                                // q = A_+ u
        AWG_TRY(zt(v.q, v.y2, s));
        AWG_TRY(dense(n0, (double*)h->Einv.p, v.y2, v.c2, 1.0, v.c1, -1.0, v.dpm, s));  // c2 = E^-1 y2 - c1
        if (wait) AWG_CUDA(cudaStreamWaitEvent(s, wait, 0));
        return zc(v.c2, Y, (T)-1, (T)0, v.u, (T)1, V2, s);                         // Y = u - Z c2 (+ V2)
    }
    awg_status h2(int prec, const T* X, T* Y, cudaStream_t s) {
        AWG_TRY(h2a(X, s));
        return h2b(prec, X, Y, s);
    }

    // w0 (float64, n_- x K) = W^T X
    awg_status wt(int prec, const T* X, double* w0, cudaStream_t s) {
        const PrecOps& P = h->prec[prec];
        const int n = h->n, ldw = h->ldw, nm = h->n_minus;
        const bool cor = P.corr_nnz > 0;
        const float* rsc = (const float*)P.rscale.p;
        const float* csc = (const float*)P.cscale.p;
        if constexpr (std::is_same<T, float>::value) {
            if ((prec == AWG_MIXED_FP16 || prec == AWG_MIXED_BF16) && h->opt.block_tensor_cores &&
                umma_available()) {
                const unsigned gr = grid_rows(n, RM<float, K>::RPB);
                {
                    ProfScope ps_(h, AWG_PROF_VECTOR, s);
                    AWG_CUDA(cudaMemsetAsync(v.mx, 0, K * 4, s));
                    kb_colmax<K><<<gr, 256, 0, s>>>(n, X, rsc, v.mx);
                    AWG_LAUNCH();
                    if (prec == AWG_MIXED_FP16)
                        kb_split16<__half, K><<<(n + 31) / 32, 256, 0, s>>>(n, ldb(), X, rsc, v.mx, (__half*)v.bt);
                    else
                        kb_split16<__nv_bfloat16, K><<<(n + 31) / 32, 256, 0, s>>>(n, ldb(), X, rsc, v.mx,
                                                                                  (__nv_bfloat16*)v.bt);
                    AWG_LAUNCH();
                    extra_launches(h, 1);
                }
                UmmaW u;
                u.W = P.W.p; u.n = n; u.ldw = ldw; u.nm = nm; u.bf16 = (prec == AWG_MIXED_BF16);
                const int splits = wt_splits();
                {
                    ProfScope ps_(h, AWG_PROF_WT, s);
                    AWG_TRY(umma_wt(u, K, v.bt, ldb(), (float*)v.part, splits, v.err, s));
                }
                ProfScope ps_(h, AWG_PROF_VECTOR, s);
                kb_wt_reduce_umma<K><<<nm, 256, 0, s>>>(
                    splits, ldw, nm, (float*)v.part, v.mx, csc, cor ? (int*)P.corr_colptr.p : nullptr,
                    cor ? (int*)P.corr_row.p : nullptr, cor ? (float*)P.corr_cval.p : nullptr, X, rsc, w0);
                AWG_LAUNCH();
                return AWG_OK;
            }
        }
        const int rb = std::max(1, std::min(WT_SPLITS_MAX, (n + 2047) / 2048));
        const int rows = (n + rb - 1) / rb;
        const dim3 g(rb, (ldw + 255) / 256);
        {
            ProfScope ps_(h, AWG_PROF_WT, s);
            if constexpr (std::is_same<T, double>::value) {
                kb_wt_partial<double, double, K><<<g, 256, 0, s>>>(n, ldw, rows, (const double*)P.W.p, X, nullptr,
                                                                  (double*)v.part, nullptr);
            } else {
                float* xo = cor ? (float*)v.xs : nullptr;
                if (prec == AWG_MIXED_FP32)
                    kb_wt_partial<float, float, K><<<g, 256, 0, s>>>(n, ldw, rows, (const float*)P.W.p, X, rsc,
                                                                    (float*)v.part, xo);
                else if (prec == AWG_MIXED_FP16)
                    kb_wt_partial<__half, float, K><<<g, 256, 0, s>>>(n, ldw, rows, (const __half*)P.W.p, X, rsc,
                                                                     (float*)v.part, xo);
                else
                    kb_wt_partial<__nv_bfloat16, float, K><<<g, 256, 0, s>>>(
                        n, ldw, rows, (const __nv_bfloat16*)P.W.p, X, rsc, (float*)v.part, xo);
            }
        }
        AWG_LAUNCH();
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        kb_wt_reduce<A, K><<<(nm * K + 255) / 256, 256, 0, s>>>(
            rb, ldw, nm, (const A*)v.part, csc, cor ? (int*)P.corr_colptr.p : nullptr,
            cor ? (int*)P.corr_row.p : nullptr, cor ? (float*)P.corr_cval.p : nullptr, (const A*)v.xs, w0);
        AWG_LAUNCH();
        return AWG_OK;
    }

    int ldb() const { return (h->n + 63) / 64 * 64; }

    static constexpr int kidx = K == 16 ? 0 : (K == 32 ? 1 : 2);

    int wt_splits() const {
        // (autotuned) CTAs per SM over the 256-column tiles of W; default 2
        const int per_sm = h->bt_wt[kidx] > 0 ? h->bt_wt[kidx] : 2;
        const int tiles = (h->ldw + 255) / 256;
        return umma_wt_splits(h->n, std::max(1, std::min(WT_SPLITS_MAX, (per_sm * 152 + tiles - 1) / tiles)));
    }

    // out = W d (+ V), d float64 n_- x K
    awg_status wd(int prec, const double* d, T* out, const T* V, cudaStream_t s) {
        const PrecOps& P = h->prec[prec];
        const int n = h->n, ldw = h->ldw, nm = h->n_minus;
        const bool cor = P.corr_nnz > 0;
        const float* rsc = (const float*)P.rscale.p;
        const float* csc = (const float*)P.cscale.p;
        if constexpr (std::is_same<T, float>::value) {
            if ((prec == AWG_MIXED_FP16 || prec == AWG_MIXED_BF16) && h->opt.block_tensor_cores &&
                umma_available()) {
                {
                    ProfScope ps_(h, AWG_PROF_VECTOR, s);
                    kb_d_scaled<float, K><<<(ldw * K + 255) / 256, 256, 0, s>>>(nm, ldw, d, csc, (float*)v.ds);
                    AWG_LAUNCH();
                    AWG_CUDA(cudaMemsetAsync(v.mx2, 0, K * 4, s));
                    kb_colmax<K><<<grid_rows(ldw, RM<float, K>::RPB), 256, 0, s>>>(ldw, (float*)v.ds, nullptr, v.mx2);
                    AWG_LAUNCH();
                    const unsigned gs = (ldw * K + 255) / 256;
                    if (prec == AWG_MIXED_FP16)
                        kb_split16_d<__half, K><<<gs, 256, 0, s>>>(ldw, (float*)v.ds, v.mx2, (__half*)v.dt, v.dscale);
                    else
                        kb_split16_d<__nv_bfloat16, K><<<gs, 256, 0, s>>>(ldw, (float*)v.ds, v.mx2,
                                                                         (__nv_bfloat16*)v.dt, v.dscale);
                    extra_launches(h, 2);
                    AWG_LAUNCH();
                }
                UmmaW u;
                u.W = P.W.p; u.n = n; u.ldw = ldw; u.nm = nm; u.bf16 = (prec == AWG_MIXED_BF16);
                {
                    ProfScope ps_(h, AWG_PROF_WD, s);
                    AWG_TRY(umma_wd(u, K, v.dt, v.wacc, v.err, s));
                }
                ProfScope ps_(h, AWG_PROF_VECTOR, s);
                kb_wd_finish_umma<K><<<grid_rows(n, RM<float, K>::RPB), 256, 0, s>>>(
                    n, v.wacc, v.dscale, rsc, cor ? (int*)P.corr_rowptr.p : nullptr,
                    cor ? (int*)P.corr_col.p : nullptr, cor ? (float*)P.corr_val.p : nullptr, (float*)v.ds, V, out);
                AWG_LAUNCH();
                return AWG_OK;
            }
        }
        {
            ProfScope ps_(h, AWG_PROF_VECTOR, s);
            kb_d_scaled<A, K><<<(ldw * K + 255) / 256, 256, 0, s>>>(nm, ldw, d, csc, (A*)v.ds);
            AWG_LAUNCH();
        }
        ProfScope ps_(h, AWG_PROF_WD, s);
        const unsigned g = (n + 31) / 32;
        const int* crp = cor ? (int*)P.corr_rowptr.p : nullptr;
        const int* ccol = cor ? (int*)P.corr_col.p : nullptr;
        const float* cval = cor ? (float*)P.corr_val.p : nullptr;
        if constexpr (std::is_same<T, double>::value) {
            kb_w_d<double, double, K><<<g, 256, 0, s>>>(n, ldw, (const double*)P.W.p, (const double*)v.ds, nullptr,
                                                        nullptr, nullptr, nullptr, V, out);
        } else {
            if (prec == AWG_MIXED_FP32)
                kb_w_d<float, float, K><<<g, 256, 0, s>>>(n, ldw, (const float*)P.W.p, (const float*)v.ds, rsc, crp,
                                                          ccol, cval, V, out);
            else if (prec == AWG_MIXED_FP16)
                kb_w_d<__half, float, K><<<g, 256, 0, s>>>(n, ldw, (const __half*)P.W.p, (const float*)v.ds, rsc,
                                                           crp, ccol, cval, V, out);
            else
                kb_w_d<__nv_bfloat16, float, K><<<g, 256, 0, s>>>(n, ldw, (const __nv_bfloat16*)P.W.p,
                                                                  (const float*)v.ds, rsc, crp, ccol, cval, V, out);
        }
        AWG_LAUNCH();
        return AWG_OK;
    }

    // Y = stage(X) on preconditioner block vectors (X may be v.rin)
    awg_status stage(int which, int prec, const T* X, T* Y, cudaStream_t s) {
        switch (which) {
            case 0: {
                ProfScope ps_(h, AWG_PROF_SPMV, s);
                kb_aplus<T, K><<<rows_grid((const void*)kb_aplus<T, K>, h->n), 256, 0, s>>>(
                    h->n, (int*)h->rowptr.p, (int*)h->colidx.p, aval(), X, nullptr, nullptr, nullptr, nullptr,
                    nullptr, nullptr, nullptr, nullptr, nullptr, (T)1, Y);
                AWG_LAUNCH();
                return AWG_OK;
            }
            case 1: return aplus(X, Y, nullptr, (T)1, s);
            case 2: return hnn(prec, X, Y, s);
            case 3: return h2(prec, X, Y, s);
            case 4:    // H_3,ad = H_2 + W F^-1 W^T (Def. 10)
            case 6: {  // H_3,inex = H_2 + W (C^-1 - Vhat^T W)^-1 W^T (Thm. 7)
                if (h->n_minus == 0) return h2(prec, X, Y, s);
                const double* coarse = (double*)(which == 4 ? h->prec[prec].Finv.p : h->prec[prec].inexInv.p);
                const cudaStream_t side = side_stream(h, sl.side, s);
                AWG_CUDA(cudaEventRecord(sl.fork, s));
                AWG_CUDA(cudaStreamWaitEvent(side, sl.fork, 0));
                // side stream: W^T X (HBM) beside the first E^-1 (FP64 pipes),
                // then the second coarse solve (FP64) after it, beside the
                // local solves (FP32), and W d beside the second E^-1
                AWG_TRY(wt(prec, X, v.w0, side));
                AWG_TRY(h2a(X, s));
                AWG_CUDA(cudaEventRecord(sl.mid, s));
                AWG_CUDA(cudaStreamWaitEvent(side, sl.mid, 0));
                AWG_TRY(dense(h->n_minus, coarse, v.w0, v.dd, 1.0, nullptr, 0.0, v.dps, side));
                AWG_TRY(wd(prec, v.dd, v.tmpw, nullptr, side));
                AWG_CUDA(cudaEventRecord(sl.join, side));
                return h2b(prec, X, Y, s, v.tmpw, sl.join);
            }
            case 5: {  // H_3,hyb = Pi_3 H_2 Pi_3^T + W F^-1 W^T (Def. 10), in order on s
                if (h->n_minus == 0) return h2(prec, X, Y, s);
                const double* Finv = (double*)h->prec[prec].Finv.p;
                const size_t len = (size_t)h->n * K;
                AWG_TRY(wt(prec, X, v.w0, s));
                AWG_TRY(dense(h->n_minus, Finv, v.w0, v.dd, 1.0, nullptr, 0.0, v.dpm, s));  // d = F^-1 W^T X
                AWG_TRY(wd(prec, v.dd, v.tmpw, nullptr, s));                                   // W d
                AWG_TRY(stage(0, prec, v.tmpw, v.q, s));                                       // A W d
                {
                    ProfScope ps_(h, AWG_PROF_VECTOR, s);
                    kb_sub<T><<<(unsigned)((len + 255) / 256), 256, 0, s>>>(len, X, v.q, v.tmpw);  // Pi_3^T X
                    AWG_LAUNCH();
                }
                AWG_TRY(h2(prec, v.tmpw, Y, s));                                                // y = H_2 Pi_3^T X
                AWG_TRY(stage(0, prec, Y, v.q, s));                                             // A y
                AWG_TRY(wt(prec, v.q, v.w0, s));
                AWG_TRY(dense(h->n_minus, Finv, v.w0, v.w1, -1.0, v.dd, 1.0, v.dpm, s));      // d - F^-1 W^T A y
                return wd(prec, v.w1, Y, Y, s);                                                 // Y = y + W w1
            }
            default: return AWG_ERR_INVALID_ARG;
        }
    }

    // float64 in, float64 out (row-major n x K): conversions around the
    // float32 internal vectors of the mixed forms
    awg_status apply64(int which, int prec, const double* X, double* Y, cudaStream_t s) {
        if constexpr (std::is_same<T, double>::value) {
            return stage(which, prec, X, Y, s);
        } else {
            const size_t len = (size_t)h->n * K;
            {
                ProfScope ps_(h, AWG_PROF_VECTOR, s);
                AWG_TRY(cvt_d2t(X, v.rin, len, s));
            }
            AWG_TRY(stage(which, prec, v.rin, v.out, s));
            ProfScope ps_(h, AWG_PROF_VECTOR, s);
            return cvt_t2d(v.out, Y, len, s);
        }
    }
};

template <int K>
awg_status tune_k(Handle* h, int prec, const double* X, double* Y, cudaStream_t s, const Slot& sl);

template <int K>
awg_status apply64_k(Handle* h, int which, int prec, const double* X, double* Y, cudaStream_t s, const Slot& sl) {
    constexpr int kidx = K == 16 ? 0 : (K == 32 ? 1 : 2);
    if (which >= 4 && h->opt.autotune && h->bt_wt[kidx] == 0 && h->n_minus > 0) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        AWG_CUDA(cudaStreamIsCapturing(s, &cs));
        if (cs == cudaStreamCaptureStatusNone) AWG_TRY(tune_k<K>(h, prec, X, Y, s, sl));
    }
    if (prec == AWG_FP64) {
        BlockApply<double, K> b{h, {}, sl};
        carve_block(h, sl.ws, &b.v, nullptr);
        return b.apply64(which, prec, X, Y, s);
    }
    BlockApply<float, K> b{h, {}, sl};
    carve_block(h, sl.ws, nullptr, &b.v);
    return b.apply64(which, prec, X, Y, s);
}

awg_status apply64_any(Handle* h, int K, int which, int prec, const double* X, double* Y, cudaStream_t s,
                       const Slot& sl) {
    if (K == 16) return apply64_k<16>(h, which, prec, X, Y, s, sl);
    if (K == 32) return apply64_k<32>(h, which, prec, X, Y, s, sl);
    return apply64_k<64>(h, which, prec, X, Y, s, sl);
}

// A mixed-precision form on float32 block vectors, without the float64
// conversions around it: the PCG kernels write r in float32 beside its
// float64 copy (kb_pcg_xr) and read z in float32 (kb_coldot, kb_pcg_p), so
// the preconditioner's input and output need no separate passes.
// (the block autotuner is not run from here: it uses the float32 input
// vector as scratch, so the PCG drivers call tune_first before they write r)
template <int K>
awg_status apply32_k(Handle* h, int which, int prec, const float* X, float* Y, cudaStream_t s, const Slot& sl) {
    BlockApply<float, K> b{h, {}, sl};
    carve_block(h, sl.ws, nullptr, &b.v);
    return b.stage(which, prec, X, Y, s);
}

// The block autotuner on the first H_3 apply of width K, before a PCG
// driver fills the apply's float32 input (X, Y float64 n x K scratch)
template <int K>
awg_status tune_first(Handle* h, int which, int prec, const double* X, double* Y, cudaStream_t s, const Slot& sl) {
    constexpr int kidx = K == 16 ? 0 : (K == 32 ? 1 : 2);
    if (which >= 4 && h->opt.autotune && h->bt_wt[kidx] == 0 && h->n_minus > 0) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        AWG_CUDA(cudaStreamIsCapturing(s, &cs));
        if (cs == cudaStreamCaptureStatusNone) AWG_TRY(tune_k<K>(h, prec, X, Y, s, sl));
    }
    return AWG_OK;
}

awg_status apply32_any(Handle* h, int K, int which, int prec, const float* X, float* Y, cudaStream_t s,
                       const Slot& sl) {
    if (K == 16) return apply32_k<16>(h, which, prec, X, Y, s, sl);
    if (K == 32) return apply32_k<32>(h, which, prec, X, Y, s, sl);
    return apply32_k<64>(h, which, prec, X, Y, s, sl);
}

// Block autotuner: on the first H_3 apply of width K, time the apply (on
// the caller's X, Y) for CTAs per SM of the W^T B pass in {1, 2, 4} and
// blocks per SM of the float64 coarse GEMM in {2, 4, 8}, keep the fastest
// pair (two timed applies each, after one warm-up).
template <int K>
awg_status tune_k(Handle* h, int prec, const double* X, double* Y, cudaStream_t s, const Slot& sl) {
    constexpr int kidx = K == 16 ? 0 : (K == 32 ? 1 : 2);
    const int prof = h->prof;
    const int64_t l0 = h->launches;
    h->prof = 0;
    cudaEvent_t e0, e1;
    AWG_CUDA(cudaEventCreate(&e0));
    AWG_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int bw = 2, bd = 4;
    awg_status st = AWG_OK;
    for (int w : {1, 2, 4}) {
        for (int d : {2, 4, 8}) {
            h->bt_wt[kidx] = w;
            h->bt_dense[kidx] = d;
            float ms = 0.f;
            for (int rep = 0; rep < 3 && st == AWG_OK; rep++) {
                if (rep == 1) cudaEventRecord(e0, s);
                if (prec == AWG_FP64) {
                    BlockApply<double, K> b{h, {}, sl};
                    carve_block(h, sl.ws, &b.v, nullptr);
                    st = b.apply64(4 + h->opt.variant, prec, X, Y, s);
                } else {
                    BlockApply<float, K> b{h, {}, sl};
                    carve_block(h, sl.ws, nullptr, &b.v);
                    st = b.apply64(4 + h->opt.variant, prec, X, Y, s);
                }
            }
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            if (st == AWG_OK && ms < best) { best = ms; bw = w; bd = d; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->bt_wt[kidx] = bw;
    h->bt_dense[kidx] = bd;
    h->prof = prof;
    h->launches = l0;
    if (h->opt.verbose)
        fprintf(stderr, "libawg: block autotune K=%d: W^T B %d CTAs/SM, coarse GEMM %d blocks/SM (%.3f ms/apply)\n",
                K, bw, bd, best / 2);
    return st;
}

int pick_k(int nrhs) { return nrhs <= 16 ? 16 : (nrhs <= 32 ? 32 : 64); }

// PCG steps shared by the host-driven and graph-driven block solves.  The
// float64 form applies the preconditioner to the float64 r (v.pr) into the
// float64 z (v.pz); the mixed forms apply it to the float32 copy of r that
// the last x, r update wrote (v.rin) into a float32 z (v.out), which the dot
// products and the p update read directly (z is computed in float32 there,
// so nothing is lost), and the recurrences stay float64.
template <int K>
struct PcgSteps {
    Handle* h;
    const BView<double>& v;
    int prec;
    cudaStream_t s;
    const Slot& sl;

    unsigned g(const void* kern) const { return grid_for(kern, h->n, RM<double, K>::RPB); }
    float* r32() const { return (float*)v.rin; }
    float* z32() const { return (float*)v.out; }

    // first use of the autotuner, then the float32 copy of r = b
    awg_status start() {
        AWG_TRY(tune_first<K>(h, 4 + h->opt.variant, prec, v.pb, v.pz, s, sl));
        if (prec == AWG_FP64) return AWG_OK;
        const size_t len = (size_t)h->n * K;
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        kb_cvt<double, float><<<(unsigned)((len + 255) / 256), 256, 0, s>>>(len, v.pr, r32());
        AWG_LAUNCH();
        return AWG_OK;
    }
    // z = H r, *rz = r . z (per column)
    awg_status precond(double* rz) {
        const int n = h->n;
        if (prec == AWG_FP64) {
            AWG_TRY(apply64_any(h, K, 4 + h->opt.variant, prec, v.pr, v.pz, s, sl));
            ProfScope ps_(h, AWG_PROF_VECTOR, s);
            kb_coldot<K><<<g((const void*)kb_coldot<K>), 256, 0, s>>>(n, v.pr, v.pz, v.red, v.cnt, rz);
            AWG_LAUNCH();
            return AWG_OK;
        }
        AWG_TRY(apply32_any(h, K, 4 + h->opt.variant, prec, r32(), z32(), s, sl));
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        kb_coldot<K, float><<<g((const void*)kb_coldot<K, float>), 256, 0, s>>>(n, v.pr, z32(), v.red, v.cnt, rz);
        AWG_LAUNCH();
        return AWG_OK;
    }
    // p = z (first iteration)
    awg_status p_first() {
        const size_t len = (size_t)h->n * K;
        if (prec == AWG_FP64) {
            AWG_CUDA(cudaMemcpyAsync(v.pp, v.pz, len * 8, cudaMemcpyDeviceToDevice, s));
            return AWG_OK;
        }
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        kb_cvt<float, double><<<(unsigned)((len + 255) / 256), 256, 0, s>>>(len, z32(), v.pp);
        AWG_LAUNCH();
        return AWG_OK;
    }
    // p = z + beta p
    awg_status p_update() {
        const int n = h->n;
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        if (prec == AWG_FP64)
            kb_pcg_p<K><<<g((const void*)kb_pcg_p<K>), 256, 0, s>>>(n, v.sc, v.pz, v.pp, v.cnt);
        else
            kb_pcg_p<K, float><<<g((const void*)kb_pcg_p<K, float>), 256, 0, s>>>(n, v.sc, z32(), v.pp, v.cnt);
        AWG_LAUNCH();
        return AWG_OK;
    }
    // q = A p with p . q, then x, r (and the float32 r) updates with r . r
    awg_status spmv_xr() {
        const int n = h->n;
        {
            ProfScope ps_(h, AWG_PROF_SPMV, s);
            kb_spmv_dot<K><<<g((const void*)kb_spmv_dot<K>), 256, 0, s>>>(n, (int*)h->rowptr.p, (int*)h->colidx.p,
                                                                        (double*)h->val.p, v.pp, v.pq, v.red,
                                                                        v.cnt, v.sc + B_PQ * K);
            AWG_LAUNCH();
        }
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        kb_pcg_xr<K><<<g((const void*)kb_pcg_xr<K>), 256, 0, s>>>(n, v.sc, v.pp, v.pq, v.px, v.pr, v.red, v.cnt,
                                                                  prec == AWG_FP64 ? nullptr : r32());
        AWG_LAUNCH();
        return AWG_OK;
    }
};

template <int K>
awg_status pcg_k(Handle* h, int prec, const double* b, double* x, int nrhs, int ld, double rtol, int* iters,
                 double* relres, cudaStream_t s) {
    BView<double> v;
    carve_block(h, (char*)h->bws.p, &v, nullptr);
    const int n = h->n;
    const dim3 tg((n + 31) / 32, (K + 31) / 32), tb(32, 8);
    const unsigned gr = grid_rows(n, RM<double, K>::RPB);
    double* sc = v.sc;
    const size_t len = (size_t)n * K;
    auto prof_vec = [&](auto&& f) -> awg_status {
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        f();
        AWG_LAUNCH();
        return AWG_OK;
    };
    AWG_TRY(prof_vec([&] { kb_from_cols<double><<<tg, tb, 0, s>>>(n, nrhs, ld, K, b, v.pb); }));
    AWG_CUDA(cudaMemsetAsync(v.px, 0, len * 8, s));
    AWG_CUDA(cudaMemcpyAsync(v.pr, v.pb, len * 8, cudaMemcpyDeviceToDevice, s));
    AWG_TRY(prof_vec([&] { kb_coldot<K><<<grid_for((const void*)kb_coldot<K>, n, RM<double, K>::RPB), 256, 0, s>>>(n, v.pb, v.pb, v.red, v.cnt, sc + B_BB * K); }));
    const Slot sl0 = slot0(h);
    PcgSteps<K> ps{h, v, prec, s, sl0};
    AWG_TRY(ps.start());
    AWG_TRY(ps.precond(sc + B_RZ * K));
    AWG_TRY(ps.p_first());
    std::vector<double> hs(B_NSC * K);
    AWG_CUDA(cudaMemcpyAsync(hs.data(), sc, B_NSC * K * 8, cudaMemcpyDeviceToHost, s));
    AWG_CUDA(cudaStreamSynchronize(s));
    std::vector<double> bnorm(K), act(K, 0.0), rel(K, 1.0), trel(K, -1.0);
    std::vector<int> its(K, 0);
    int nact = 0;
    for (int c = 0; c < K; c++) {
        bnorm[c] = sqrt(hs[B_BB * K + c]);
        if (c < nrhs && bnorm[c] > 0.0) { act[c] = 1.0; nact++; }
        else trel[c] = 0.0;
    }
    awg_status st = AWG_OK;
    int it = 0;
    auto upload_act = [&]() -> awg_status {
        AWG_CUDA(cudaMemcpyAsync(sc + B_ACT * K, act.data(), K * 8, cudaMemcpyHostToDevice, s));
        return AWG_OK;
    };
    AWG_TRY(upload_act());
    auto true_resid = [&]() -> awg_status {
        AWG_TRY(prof_vec([&] {
            kb_resid<K><<<grid_for((const void*)kb_resid<K>, n, RM<double, K>::RPB), 256, 0, s>>>(n, (int*)h->rowptr.p, (int*)h->colidx.p, (double*)h->val.p, v.pb, v.px,
                                           v.pq);
        }));
        AWG_TRY(prof_vec([&] { kb_coldot<K><<<grid_for((const void*)kb_coldot<K>, n, RM<double, K>::RPB), 256, 0, s>>>(n, v.pq, v.pq, v.red, v.cnt, sc + B_TR * K); }));
        AWG_CUDA(cudaMemcpyAsync(hs.data() + B_TR * K, sc + B_TR * K, K * 8, cudaMemcpyDeviceToHost, s));
        AWG_CUDA(cudaStreamSynchronize(s));
        return AWG_OK;
    };
    while (nact > 0) {
        if (it >= h->opt.maxit) { st = AWG_ERR_MAXIT; break; }
        AWG_TRY(ps.spmv_xr());
        it++;
        AWG_CUDA(cudaMemcpyAsync(hs.data(), sc, 3 * K * 8, cudaMemcpyDeviceToHost, s));
        AWG_CUDA(cudaStreamSynchronize(s));
        bool cand = false, changed = false;
        for (int c = 0; c < K; c++) {
            if (act[c] == 0.0) continue;
            const double pq = hs[B_PQ * K + c];
            if (!(pq > 0.0) || !std::isfinite(pq)) {
                act[c] = 0.0; nact--; changed = true; its[c] = it; st = AWG_ERR_BREAKDOWN;
                continue;
            }
            rel[c] = sqrt(hs[B_RR * K + c]) / bnorm[c];
            if (rel[c] <= rtol) cand = true;
        }
        if (cand) {
            AWG_TRY(true_resid());
            for (int c = 0; c < K; c++) {
                if (act[c] == 0.0 || rel[c] > rtol) continue;
                const double tr = sqrt(hs[B_TR * K + c]) / bnorm[c];
                if (tr <= rtol || rel[c] <= 1e-6 * rtol) {
                    if (tr > rtol) st = AWG_ERR_MAXIT;
                    act[c] = 0.0; nact--; changed = true; its[c] = it; trel[c] = tr;
                }
            }
        }
        if (nact == 0) break;
        if (changed) AWG_TRY(upload_act());
        AWG_TRY(ps.precond(sc + B_RZN * K));
        AWG_TRY(ps.p_update());
    }
    bool need = false;
    for (int c = 0; c < nrhs; c++)
        if (trel[c] < 0.0) { need = true; its[c] = it; }
    if (need) {
        AWG_TRY(true_resid());
        for (int c = 0; c < nrhs; c++)
            if (trel[c] < 0.0) trel[c] = sqrt(hs[B_TR * K + c]) / bnorm[c];
    }
    AWG_TRY(prof_vec([&] { kb_to_cols<double><<<tg, tb, 0, s>>>(n, nrhs, ld, K, v.px, x); }));
    AWG_CUDA(cudaStreamSynchronize(s));
    int herr = 0;
    AWG_CUDA(cudaMemcpy(&herr, v.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) {
        fprintf(stderr, "libawg: tensor-core W pass reported error %d\n", herr);
        AWG_CUDA(cudaMemset(v.err, 0, sizeof(int)));
        return AWG_ERR_CUDA;
    }
    for (int c = 0; c < nrhs; c++) {
        if (iters) iters[c] = its[c];
        if (relres) relres[c] = trel[c];
    }
    return st;
}

}  // namespace

// Device-side stopping test after an x, r update: candidates (recurrence
// residual <= rtol), then, only in iterations that have one, the true
// residual B - A X of every column (into v.pq, free until the next q = A p)
// and its column norms, then the confirmation that stops or continues each
// candidate and sets the loop condition.
template <int K>
awg_status stop_test_k(Handle* h, const BView<double>& v, cudaStream_t s, cudaGraphConditionalHandle hc, int set,
                       int add) {
    const int n = h->n;
    const unsigned gr = grid_rows(n, RM<double, K>::RPB);
    {
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        kb_pcg_cond<K><<<1, K, 0, s>>>(v.sc, v.ctl, v.gits, v.grel);
        AWG_LAUNCH();
    }
    {
        ProfScope ps_(h, AWG_PROF_SPMV, s);
        kb_resid<K><<<grid_for((const void*)kb_resid<K>, n, RM<double, K>::RPB), 256, 0, s>>>(n, (int*)h->rowptr.p, (int*)h->colidx.p, (double*)h->val.p, v.pb, v.px,
                                       v.pq, v.ctl + 4);
        AWG_LAUNCH();
    }
    {
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        kb_coldot<K><<<grid_for((const void*)kb_coldot<K>, n, RM<double, K>::RPB), 256, 0, s>>>(n, v.pq, v.pq, v.red, v.cnt, v.sc + B_TR * K, v.ctl + 4);
        AWG_LAUNCH();
    }
    ProfScope ps_(h, AWG_PROF_VECTOR, s);
    kb_pcg_confirm<K><<<1, K, 0, s>>>(v.sc, v.ctl, v.gits, v.grel, hc, set, v.glaunch, add);
    AWG_LAUNCH();
    return AWG_OK;
}

// One PCG iteration of K columns issued on the handle's streams (the body of
// the graph loop): z = H r, rz_new, p update, q = A p, x and r update, stop test.
template <int K>
awg_status pcg_body_k(Handle* h, int prec, const BView<double>& v, cudaStream_t s, cudaGraphConditionalHandle hc,
                      int set, int add, const Slot& sl) {
    PcgSteps<K> ps{h, v, prec, s, sl};
    AWG_TRY(ps.precond(v.sc + B_RZN * K));
    AWG_TRY(ps.p_update());
    AWG_TRY(ps.spmv_xr());
    return stop_test_k<K>(h, v, s, hc, set, add);
}

// The loop graph of (prec, K): a conditional while node whose body is one
// PCG iteration captured from the handle's streams; built on first use.
template <int K>
awg_status pcg_graph_k(Handle* h, int prec, const BView<double>& v, cudaGraphExec_t* out, const Slot& sl) {
    const int slot = prec * 3 + (K == 16 ? 0 : (K == 32 ? 1 : 2));
    if (sl.exec[slot]) {
        *out = sl.exec[slot];
        return AWG_OK;
    }
    cudaGraph_t g = nullptr;
    AWG_CUDA(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle hc;
    AWG_CUDA(cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hc;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    AWG_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    // capture one iteration; kernels are counted (not timed) while capturing
    const int prof = h->prof;
    const int64_t l0 = h->launches;
    h->prof = 1 << 30;
    AWG_CUDA(cudaStreamBeginCaptureToGraph(sl.main, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    awg_status st = pcg_body_k<K>(h, prec, v, sl.main, hc, 1, 0, sl);
    cudaGraph_t cap = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(sl.main, &cap);
    const int body_launches = (int)(h->launches - l0);
    h->prof = prof;
    h->launches = l0;
    if (st != AWG_OK || ce != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        return st != AWG_OK ? st : AWG_ERR_CUDA;
    }
    // the counting argument of the body's last kernel: patch it now that the
    // number of kernels per body is known
    {
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
            if (kp.func != (void*)kb_pcg_confirm<K>) continue;
            int* addp = (int*)kp.kernelParams[7];
            *addp = body_launches;
            AWG_CUDA(cudaGraphKernelNodeSetParams(nd, &kp));
        }
    }
    cudaGraphExec_t exec = nullptr;
    // keep the capture-time stream priorities (H_2 chain ahead of the W passes)
    AWG_CUDA(cudaGraphInstantiate(&exec, g, cudaGraphInstantiateFlagUseNodePriority));
    sl.graph[slot] = g;
    sl.exec[slot] = exec;
    *out = exec;
    return AWG_OK;
}

template <int K>
awg_status pcg_async_k(Handle* h, int prec, const double* b, double* x, int nrhs, int ld, double rtol, int* d_iters,
                       double* d_relres, int* d_status, const Slot& sl) {
    const cudaStream_t s = sl.main;
    BView<double> v;
    carve_block(h, sl.ws, &v, nullptr);
    const int n = h->n;
    const dim3 tg((n + 31) / 32, (K + 31) / 32), tb(32, 8);
    const unsigned gr = grid_rows(n, RM<double, K>::RPB);
    const size_t len = (size_t)n * K;
    {
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        kb_from_cols<double><<<tg, tb, 0, s>>>(n, nrhs, ld, K, b, v.pb);
        AWG_LAUNCH();
    }
    AWG_CUDA(cudaMemsetAsync(v.px, 0, len * 8, s));
    AWG_CUDA(cudaMemcpyAsync(v.pr, v.pb, len * 8, cudaMemcpyDeviceToDevice, s));
    {
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        kb_coldot<K><<<grid_for((const void*)kb_coldot<K>, n, RM<double, K>::RPB), 256, 0, s>>>(n, v.pb, v.pb, v.red, v.cnt, v.sc + B_BB * K);
        AWG_LAUNCH();
    }
    {
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        kb_pcg_init<K><<<1, K, 0, s>>>(nrhs, v.sc, v.ctl, rtol, (double)h->opt.maxit, v.gits, v.grel);
        AWG_LAUNCH();
    }
    // first iteration with z = H r, p = z (then the loop's iterations)
    PcgSteps<K> ps{h, v, prec, s, sl};
    AWG_TRY(ps.start());
    AWG_TRY(ps.precond(v.sc + B_RZ * K));
    AWG_TRY(ps.p_first());
    AWG_TRY(ps.spmv_xr());
    AWG_TRY(stop_test_k<K>(h, v, s, 0, 0, 0));
    // the loop graph is captured after the first iteration has been issued
    // (every kernel attribute and tensor-map entry point is set up by then)
    cudaGraphExec_t exec;
    AWG_TRY(pcg_graph_k<K>(h, prec, v, &exec, sl));
    AWG_CUDA(cudaGraphLaunch(exec, s));
    {
        ProfScope ps_(h, AWG_PROF_VECTOR, s);
        kb_to_cols<double><<<tg, tb, 0, s>>>(n, nrhs, ld, K, v.px, x);
        AWG_LAUNCH();
    }
    ProfScope ps_(h, AWG_PROF_VECTOR, s);
    kb_pcg_fini<<<1, 64, 0, s>>>(nrhs, v.gits, v.grel, v.ctl, d_iters, d_relres, d_status);
    AWG_LAUNCH();
    return AWG_OK;
}

awg_status pcg_async_group(Handle* h, int prec, const double* b, double* x, int nrhs, int ld, double rtol,
                           int* d_iters, double* d_relres, int* d_status, const Slot& sl) {
    const int K = pick_k(nrhs);
    if (K == 16) return pcg_async_k<16>(h, prec, b, x, nrhs, ld, rtol, d_iters, d_relres, d_status, sl);
    if (K == 32) return pcg_async_k<32>(h, prec, b, x, nrhs, ld, rtol, d_iters, d_relres, d_status, sl);
    return pcg_async_k<64>(h, prec, b, x, nrhs, ld, rtol, d_iters, d_relres, d_status, sl);
}

// the second slot: its workspace, streams (the priorities of the first) and events
awg_status slot1_prepare(Handle* h) {
    if (h->bws2.p) return AWG_OK;
    int lo = 0, hi = 0;
    AWG_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    AWG_CUDA(cudaStreamCreateWithPriority(&h->hp2, cudaStreamNonBlocking, hi));
    AWG_CUDA(cudaStreamCreateWithPriority(&h->side2, cudaStreamNonBlocking, lo));
    for (cudaEvent_t* e : {&h->ev2_fork, &h->ev2_mid, &h->ev2_join, &h->ev2_in, &h->ev2_out})
        AWG_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    const size_t bytes = carve_block(h, nullptr, nullptr, nullptr);
    AWG_TRY(dalloc(h, h->bws2, bytes));
    AWG_CUDA(cudaMemset(h->bws2.p, 0, bytes));
    return AWG_OK;
}

// status of two groups into *d_status: breakdown before maxit before ok
__global__ void kb_status_merge(const double* ctl_a, const double* ctl_b, int* d_status) {
    if (threadIdx.x != 0 || !d_status) return;
    const int a = (int)ctl_a[3], b = (int)ctl_b[3];
    *d_status = (a == AWG_ERR_BREAKDOWN || b == AWG_ERR_BREAKDOWN) ? AWG_ERR_BREAKDOWN : (a ? a : b);
}

awg_status block_pcg_async(Handle* h, int prec, const double* b, double* x, int nrhs, int ld, double rtol,
                           int* d_iters, double* d_relres, int* d_status, cudaStream_t s) {
    if (nrhs < 1 || nrhs > 2 * BLK_KMAX) return AWG_ERR_INVALID_ARG;
    AWG_TRY(block_prepare(h));
    AWG_TRY(oz_prepare(h));
    if (nrhs <= BLK_KMAX)
        return pcg_async_group(h, prec, b, x, nrhs, ld, rtol, d_iters, d_relres, d_status, slot0(h));
    // two groups side by side: columns [0, 64) on slot 0, the rest on slot 1
    AWG_TRY(slot1_prepare(h));
    const int ka = BLK_KMAX, kb = nrhs - BLK_KMAX;
    AWG_CUDA(cudaEventRecord(h->ev2_in, s));
    AWG_CUDA(cudaStreamWaitEvent(h->hp2, h->ev2_in, 0));
    AWG_TRY(pcg_async_group(h, prec, b, x, ka, ld, rtol, d_iters, d_relres, nullptr, slot0(h)));
    AWG_TRY(pcg_async_group(h, prec, b + (size_t)ka * ld, x + (size_t)ka * ld, kb, ld, rtol,
                            d_iters ? d_iters + ka : nullptr, d_relres ? d_relres + ka : nullptr, nullptr, slot1(h)));
    AWG_CUDA(cudaEventRecord(h->ev2_out, h->hp2));
    AWG_CUDA(cudaStreamWaitEvent(s, h->ev2_out, 0));
    BView<double> va, vb;
    carve_block(h, (char*)h->bws.p, &va, nullptr);
    carve_block(h, (char*)h->bws2.p, &vb, nullptr);
    kb_status_merge<<<1, 32, 0, s>>>(va.ctl, vb.ctl, d_status);
    AWG_LAUNCH();
    extra_launches(h, 1);
    return AWG_OK;
}

// kernels launched by graph loop bodies since the last call (reset)
int64_t block_graph_launches(Handle* h) {
    int64_t total = 0;
    for (DevBuf* ws : {&h->bws, &h->bws2}) {
        if (!ws->p) continue;
        BView<double> v;
        carve_block(h, (char*)ws->p, &v, nullptr);
        unsigned long long c = 0;
        if (cudaMemcpy(&c, v.glaunch, 8, cudaMemcpyDeviceToHost) != cudaSuccess) continue;
        cudaMemset(v.glaunch, 0, 8);
        total += (int64_t)c;
    }
    return total;
}

// W columns c0 .. c0 + k - 1: A_+ X = B by flexible block PCG (K = 64
// columns per group) with H_2 in the precision wprec (Section 4.4 items 1-2):
// the A_+ products and every recurrence in float64, the preconditioner in
// float32 for the mixed forms (its local solves on the tensor cores).
// Columns stop at ||b - A_+ x|| <= rtol ||b|| (recurrence residual) or
// breakdown; *its and *worst report the group's iterations and largest
// final relative residual.
template <int K>
awg_status wsolve_k(Handle* h, int wprec, const double* B, double* X, int k, double rtol, int maxit, int* its,
                    double* worst, cudaStream_t s) {
    BView<double> v;
    carve_block(h, (char*)h->bws.p, &v, nullptr);
    BlockApply<double, K> bd{h, v, slot0(h)};
    const int n = h->n;
    const dim3 tg((n + 31) / 32, (K + 31) / 32), tb(32, 8);
    const unsigned gr = grid_rows(n, RM<double, K>::RPB);
    const size_t len = (size_t)n * K;
    double* sc = v.sc;
    double* z = v.pz;
    double* zo = v.tmpw;  // previous z (float64 view of the W-pass output, unused by H_2)
    kb_from_cols<double><<<tg, tb, 0, s>>>(n, k, n, K, B, v.pb);
    AWG_LAUNCH();
    AWG_CUDA(cudaMemsetAsync(v.px, 0, len * 8, s));
    AWG_CUDA(cudaMemcpyAsync(v.pr, v.pb, len * 8, cudaMemcpyDeviceToDevice, s));
    kb_coldot<K><<<grid_for((const void*)kb_coldot<K>, n, RM<double, K>::RPB), 256, 0, s>>>(n, v.pb, v.pb, v.red, v.cnt, sc + B_BB * K);
    AWG_LAUNCH();
    AWG_TRY(apply64_any(h, K, 3, wprec, v.pr, z, s, slot0(h)));
    kb_coldot<K><<<grid_for((const void*)kb_coldot<K>, n, RM<double, K>::RPB), 256, 0, s>>>(n, v.pr, z, v.red, v.cnt, sc + B_RZ * K);
    AWG_LAUNCH();
    AWG_CUDA(cudaMemcpyAsync(v.pp, z, len * 8, cudaMemcpyDeviceToDevice, s));
    std::vector<double> hs(B_NSC * K), act(K, 0.0);
    AWG_CUDA(cudaMemcpyAsync(hs.data(), sc, B_NSC * K * 8, cudaMemcpyDeviceToHost, s));
    AWG_CUDA(cudaStreamSynchronize(s));
    int nact = 0;
    for (int c = 0; c < k; c++)
        if (hs[B_BB * K + c] > 0.0) { act[c] = 1.0; nact++; }
    AWG_CUDA(cudaMemcpyAsync(sc + B_ACT * K, act.data(), K * 8, cudaMemcpyHostToDevice, s));
    int it = 0;
    double wst = 0.0;
    while (nact > 0) {
        AWG_TRY(bd.aplus(v.pp, v.pq, nullptr, 1.0, s));  // q = A_+ p
        kb_coldot<K><<<grid_for((const void*)kb_coldot<K>, n, RM<double, K>::RPB), 256, 0, s>>>(n, v.pp, v.pq, v.red, v.cnt, sc + B_PQ * K);
        AWG_LAUNCH();
        kb_pcg_xr<K><<<grid_for((const void*)kb_pcg_xr<K>, n, RM<double, K>::RPB), 256, 0, s>>>(n, sc, v.pp, v.pq, v.px, v.pr, v.red, v.cnt);
        AWG_LAUNCH();
        AWG_CUDA(cudaMemcpyAsync(hs.data(), sc, 3 * K * 8, cudaMemcpyDeviceToHost, s));
        AWG_CUDA(cudaStreamSynchronize(s));
        it++;
        bool changed = false;
        wst = 0.0;
        for (int c = 0; c < k; c++) {
            const double rel = sqrt(hs[B_RR * K + c] / hs[B_BB * K + c]);
            if (hs[B_BB * K + c] > 0.0) wst = std::max(wst, rel);
            if (act[c] == 0.0) continue;
            if (!(hs[B_PQ * K + c] > 0.0) || rel <= rtol) {  // exact solution reached, or converged
                act[c] = 0.0;
                nact--;
                changed = true;
            }
        }
        if (nact == 0 || it >= maxit) break;
        if (changed) AWG_CUDA(cudaMemcpyAsync(sc + B_ACT * K, act.data(), K * 8, cudaMemcpyHostToDevice, s));
        std::swap(z, zo);
        AWG_TRY(apply64_any(h, K, 3, wprec, v.pr, z, s, slot0(h)));  // z = H_2 r
        kb_coldot<K><<<grid_for((const void*)kb_coldot<K>, n, RM<double, K>::RPB), 256, 0, s>>>(n, v.pr, z, v.red, v.cnt, sc + B_RZN * K);
        AWG_LAUNCH();
        kb_coldot<K><<<grid_for((const void*)kb_coldot<K>, n, RM<double, K>::RPB), 256, 0, s>>>(n, v.pr, zo, v.red, v.cnt, sc + B_TR * K);
        AWG_LAUNCH();
        kb_pcg_p_flex<K><<<grid_for((const void*)kb_pcg_p_flex<K>, n, RM<double, K>::RPB), 256, 0, s>>>(n, sc, z, v.pp, v.cnt);
        AWG_LAUNCH();
    }
    kb_to_cols<double><<<tg, tb, 0, s>>>(n, k, n, K, v.px, X);
    AWG_LAUNCH();
    AWG_CUDA(cudaStreamSynchronize(s));
    *its = it;
    *worst = wst;
    return AWG_OK;
}

awg_status block_solve_w(Handle* h, int wprec, const double* Vhat, double* W, int nm, double rtol, int maxit,
                         int* its_max, double* worst, cudaStream_t s) {
    AWG_TRY(block_prepare(h));
    AWG_TRY(oz_prepare(h));
    *its_max = 0;
    *worst = 0.0;
    for (int c0 = 0; c0 < nm; c0 += BLK_KMAX) {
        const int k = std::min(BLK_KMAX, nm - c0);
        int it = 0;
        double w = 0.0;
        const double* Bc = Vhat + (size_t)c0 * h->n;
        double* Xc = W + (size_t)c0 * h->n;
        const int K = pick_k(k);
        awg_status st;
        if (K == 16) st = wsolve_k<16>(h, wprec, Bc, Xc, k, rtol, maxit, &it, &w, s);
        else if (K == 32) st = wsolve_k<32>(h, wprec, Bc, Xc, k, rtol, maxit, &it, &w, s);
        else st = wsolve_k<64>(h, wprec, Bc, Xc, k, rtol, maxit, &it, &w, s);
        AWG_TRY(st);
        *its_max = std::max(*its_max, it);
        *worst = std::max(*worst, w);
        if (h->opt.verbose)
            fprintf(stderr, "libawg: W columns %d..%d: %d iterations, max relres %.3e\n", c0, c0 + k, it, w);
    }
    return AWG_OK;
}

awg_status block_apply(Handle* h, int which, int prec, const double* x, double* y, int nrhs, int ld,
                       cudaStream_t s) {
    if (nrhs < 1 || nrhs > BLK_KMAX) return AWG_ERR_INVALID_ARG;
    AWG_TRY(block_prepare(h));
    AWG_TRY(oz_prepare(h));
    const int K = pick_k(nrhs);
    BView<double> v;
    carve_block(h, (char*)h->bws.p, &v, nullptr);
    const int n = h->n;
    const dim3 tg((n + 31) / 32, (K + 31) / 32), tb(32, 8);
    kb_from_cols<double><<<tg, tb, 0, s>>>(n, nrhs, ld, K, x, v.pb);
    AWG_LAUNCH();
    AWG_TRY(apply64_any(h, K, which, prec, v.pb, v.pz, s, slot0(h)));
    kb_to_cols<double><<<tg, tb, 0, s>>>(n, nrhs, ld, K, v.pz, y);
    AWG_LAUNCH();
    return AWG_OK;
}

// Y = M X for a dense coarse inverse M of the handle (which: 0 E^-1, 1 F^-1
// of form prec, 2 the H_3,inex inner inverse of form prec), X and Y
// column-major dim x nrhs (ld = dim), through the block path's coarse
// product: engine 0 the float64 CUDA-core GEMM, 1 the tensor-core slice
// products, 2 the same with reduction splits of 256 terms (exercises the
// split path on small coarse spaces).
awg_status block_coarse_apply(Handle* h, int which, int prec, int engine, const double* x, double* y, int nrhs,
                              cudaStream_t s) {
    if (nrhs < 1 || nrhs > BLK_KMAX || which < 0 || which > 2 || engine < 0 || engine > 2) return AWG_ERR_INVALID_ARG;
    const DevBuf& M = which == 0 ? h->Einv : (which == 1 ? h->prec[prec].Finv : h->prec[prec].inexInv);
    const int dim = which == 0 ? h->n0 : h->n_minus;
    if (!M.p || dim < 1) return AWG_ERR_STATE;
    AWG_TRY(block_prepare(h));
    AWG_TRY(oz_prepare(h));
    const int K = pick_k(nrhs);
    OzMat om;
    const bool have = oz_of(h, (const double*)M.p, &om);
    if (engine > 0 && !have) return AWG_ERR_STATE;
    const int cps = engine == 2 ? 4 : OZ_CHUNKS_MAX;
    const size_t len = (size_t)dim * K;
    const size_t part_elems = std::max((size_t)DG_SMAX * len, oz_part_elems(dim, K, cps));
    double *xr = nullptr, *yr = nullptr, *part = nullptr;
    void* xs = nullptr;
    int* err = nullptr;
    AWG_CUDA(cudaMallocAsync(&xr, len * 8, s));
    AWG_CUDA(cudaMallocAsync(&yr, len * 8, s));
    AWG_CUDA(cudaMallocAsync(&part, part_elems * 8, s));
    AWG_CUDA(cudaMallocAsync(&xs, oz_xs_bytes(dim, K), s));
    AWG_CUDA(cudaMallocAsync(&err, 4, s));
    AWG_CUDA(cudaMemsetAsync(err, 0, 4, s));
    const dim3 tg((dim + 31) / 32, (K + 31) / 32), tb(32, 8);
    kb_from_cols<double><<<tg, tb, 0, s>>>(dim, nrhs, dim, K, x, xr);
    AWG_LAUNCH();
    awg_status st = AWG_OK;
    if (engine > 0) {
        st = oz_gemm(om, K, xr, yr, 1.0, nullptr, 0.0, xs, part, err, s, cps);
    } else {
        const int tiles = (dim + DG_RB - 1) / DG_RB;
        int S = std::max(1, std::min(DG_SMAX, (4 * 152 + tiles - 1) / tiles));
        int jlen = (dim + S - 1) / S;
        jlen = (jlen + DG_JC - 1) / DG_JC * DG_JC;
        S = (dim + jlen - 1) / jlen;
        if (K == 16) kb_dense_part<16><<<dim3(tiles, S), 64, 0, s>>>(dim, jlen, (const double*)M.p, xr, part);
        else if (K == 32) kb_dense_part<32><<<dim3(tiles, S), 128, 0, s>>>(dim, jlen, (const double*)M.p, xr, part);
        else kb_dense_part<64><<<dim3(tiles, S), 256, 0, s>>>(dim, jlen, (const double*)M.p, xr, part);
        AWG_LAUNCH();
        const unsigned g = (unsigned)((len + 255) / 256);
        if (K == 16) kb_dense_sum<16><<<g, 256, 0, s>>>(dim, S, part, yr, 1.0, nullptr, 0.0);
        else if (K == 32) kb_dense_sum<32><<<g, 256, 0, s>>>(dim, S, part, yr, 1.0, nullptr, 0.0);
        else kb_dense_sum<64><<<g, 256, 0, s>>>(dim, S, part, yr, 1.0, nullptr, 0.0);
        AWG_LAUNCH();
    }
    if (st == AWG_OK) {
        kb_to_cols<double><<<tg, tb, 0, s>>>(dim, nrhs, dim, K, yr, y);
        AWG_LAUNCH();
    }
    int herr = 0;
    AWG_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s));
    for (void* ptr : {(void*)xr, (void*)yr, (void*)part, xs, (void*)err}) AWG_CUDA(cudaFreeAsync(ptr, s));
    AWG_CUDA(cudaStreamSynchronize(s));
    if (herr) {
        fprintf(stderr, "libawg: tensor-core coarse product reported error %d\n", herr);
        return AWG_ERR_CUDA;
    }
    return st;
}

awg_status block_pcg(Handle* h, int prec, const double* b, double* x, int nrhs, int ld, double rtol, int* iters,
                     double* relres, cudaStream_t s) {
    AWG_TRY(block_prepare(h));
    AWG_TRY(oz_prepare(h));
    awg_status worst = AWG_OK;
    for (int c0 = 0; c0 < nrhs; c0 += BLK_KMAX) {
        const int k = std::min(BLK_KMAX, nrhs - c0);
        const int K = pick_k(k);
        awg_status st;
        const double* bc = b + (size_t)c0 * ld;
        double* xc = x + (size_t)c0 * ld;
        int* ic = iters ? iters + c0 : nullptr;
        double* rc = relres ? relres + c0 : nullptr;
        if (K == 16) st = pcg_k<16>(h, prec, bc, xc, k, ld, rtol, ic, rc, s);
        else if (K == 32) st = pcg_k<32>(h, prec, bc, xc, k, ld, rtol, ic, rc, s);
        else st = pcg_k<64>(h, prec, bc, xc, k, ld, rtol, ic, rc, s);
        if (st != AWG_OK && (worst == AWG_OK || st == AWG_ERR_CUDA)) worst = st;
        if (st == AWG_ERR_CUDA) break;
    }
    return worst;
}

}  // namespace awg
