// Float64-accurate products with the dense coarse inverses on the tensor
// cores: Y = alpha M X + beta Sub, with M = E^-1 (Thm. 4, twice per apply of
// H_2) or F^-1 / the H_3,inex inner inverse (Def. 10, Thm. 7), X the K
// coarse right-hand sides of a block apply.
//
// On this GPU a float64 GEMM runs on the FP64 pipes, about 1/1600 of the
// bfloat16 tensor rate; the three coarse products of a 64-column apply took
// two thirds of a PCG iteration there.  Here both operands are cut into
// integer slices (Ozaki's error-free transformation, in the form of Ootomo,
// Ozaki & Yokota and Uchino et al.), every slice product runs on tcgen05 in
// bfloat16 with float32 accumulation, EXACTLY, and the slice products are
// recombined in float64:
//
//   M(i, j) = 2^e_i  sum_{s=1..S} q_s(i, j) 2^(-7 s) + rest,  |q_s| <= 64,
//   X(j, c) = 2^f_c  sum_{t=1..S} p_t(j, c) 2^(-7 t) + rest,  |p_t| <= 64,
//
// (per-row and per-column power-of-two scales e_i, f_c with |M(i, :)| 2^-e_i
// and |X(:, c)| 2^-f_c <= 1/2; the digits are taken by round-to-nearest,
// q = rint(r 2^7), r <- r 2^7 - q, every step exact in float64).  Digits of
// magnitude <= 64 are exact in bfloat16, products are <= 2^12, so a sum of up
// to 4095 products stays below 2^24 and the float32 accumulator in tensor
// memory holds every partial sum exactly (integers below 2^24).  Then
//
//   Y(i, c) = 2^(e_i + f_c) sum_{s + t <= S + 1} 2^(-7 (s + t)) D_st(i, c),
//   D_st = q_s p_t (exact),
//
// which drops only the terms below 2^(-7 (S + 2)) of the row and column
// scales: with S = 8 the result is as accurate as a float64 GEMM (about
// 2^-53 relative to |M| |X|; measured error below that of the float64
// GEMM on the benchmark problem's own E^-1 and F^-1).  36 slice products
// replace one float64 GEMM: 36 x 2 n^2 K bfloat16 flops.
//
// Kernel: one CTA per (128-row tile of M, work item, reduction split), a
// work item being a slice q_s of M and up to 256 / K consecutive slices
// p_t of X (s + t <= S + 1): the CTA reads the 128 x 64 tile of q_s and the
// stacked X slices (nt K rows) per 64-deep stage through TMA into a 2-stage
// shared-memory ring (48 KB stages at K = 64, two CTAs per SM), one thread
// issues one MMA per 16-deep step (M = 128, N = nt K <= 256, the products
// D_st side by side in tensor memory), and the four warps read the
// accumulators back.  The recombination is done in integer
// arithmetic, exactly: with levels l = s + t (from 0),
//
//   sum_st 2^(-7 (s + t + 2)) D_st = 2^-28 H + 2^-63 L,
//   H = sum_{l <= 2} 2^(7 (2 - l)) sum_{s+t=l} D_st   (|H| < 2^40),
//   L = sum_{3 <= l <= 7} 2^(7 (7 - l)) sum_{s+t=l} D_st   (|L| < 2^57),
//
// so every CTA adds its D_st (float32 values that are integers) into two
// int64 words per output, the partials of all CTAs are added in int64 (any
// order gives the same sum) and converted to float64 once per output.  On
// this GPU float64 instructions issue at about 2 per clock per SM, 1/64 of
// the integer rate, so the float64 work is kept to that one conversion (and
// the right-hand sides' digits are cut with integer shifts from one rounding
// to a 56-bit integer).  Every wait is bounded: a wait that gives up records
// a code in *d_err and the CTA winds down (waits for its copies in flight,
// frees its tensor memory).

#include "block.cuh"
#include "tcgen05.cuh"

#include <algorithm>

namespace awg {

namespace {

constexpr int OZ_BM = 128;       // rows of M per CTA (MMA M)
constexpr int OZ_BK = 64;        // reduction depth per stage (128 bytes of bfloat16)
constexpr int OZ_THREADS = 128;
constexpr int OZ_CHUNKS = 63;    // stages per reduction split (at most): 63 x 64 = 4032 <= 4095

// A CTA computes the products of one digit s of M with at most TN digits t
// of X (TN K <= 256 columns of tensor memory, one MMA per 16-deep step), so
// that a 2-stage ring of A (16 KB) + B (TN K x 64 bfloat16) stages fits
// twice per SM.
template <int K>
struct OzCfg {
    static constexpr int TN = (256 / K) < OZ_SLICES ? (256 / K) : OZ_SLICES;
    static constexpr int A_BYTES = OZ_BM * OZ_BK * 2;        // 16 KB tile of q_s
    static constexpr int B_BYTES = TN * K * OZ_BK * 2;       // up to TN digits of X, K rows each
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int STAGES = 2;
    static constexpr int SMEM = STAGES * STAGE + 1024;       // + alignment slack
};

// The work items of one 128-row tile: (digit s of M, first digit t0 of X,
// nt digits), nt <= TN, s + t0 + nt <= S (digits from 0), heaviest first.
struct OzItems {
    int count;
    signed char s[2 * OZ_SLICES], t0[2 * OZ_SLICES], nt[2 * OZ_SLICES];
};

struct OzShared {
    uint64_t full[4];
    uint64_t empty[4];
    uint64_t done;
    uint32_t tmem;
    int fail;
};

__device__ __forceinline__ __nv_bfloat16 digit_bf16(double q) { return __float2bfloat16_rn((float)q); }

// Row slices of M (dim x dim, row-major float64): q[(s dimp + i) ldk + j],
// zero outside dim x dim; ex[i] = e_i.  One block per row.
__global__ void __launch_bounds__(256) k_oz_slice_rows(int dim, int dimp, int ldk, const double* __restrict__ M,
                                                       __nv_bfloat16* __restrict__ q, int* __restrict__ ex) {
    __shared__ double red[32];
    const int i = blockIdx.x;
    double mx = 0.0;
    for (int j = threadIdx.x; j < dim; j += blockDim.x) mx = fmax(mx, fabs(M[(size_t)i * dim + j]));
    // block maximum (fixed order)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    mx = red[0];
    const int e = mx > 0.0 ? ilogb(mx) + 2 : 0;  // |M(i, :)| 2^-e < 1/2
    if (threadIdx.x == 0) ex[i] = e;
    for (int j = threadIdx.x; j < ldk; j += blockDim.x) {
        double r = j < dim ? ldexp(M[(size_t)i * dim + j], -e) : 0.0;
#pragma unroll
        for (int s = 0; s < OZ_SLICES; s++) {
            const double x = r * (double)(1 << OZ_BITS);
            const double d = rint(x);
            r = x - d;
            q[((size_t)s * dimp + i) * ldk + j] = digit_bf16(d);
        }
    }
}

// Largest |X(:, c)| of the columns of X (dim x K, row-major float64), as the
// bits of the float64 magnitude (ordered like the values), into mx[c]
// (zeroed before): integer maxima, one global atomic per column and block.
template <int K>
__global__ void __launch_bounds__(256) k_oz_colmax(int dim, const double* __restrict__ X,
                                                   unsigned long long* __restrict__ mx) {
    __shared__ unsigned long long sm[K];
    for (int c = threadIdx.x; c < K; c += blockDim.x) sm[c] = 0ull;
    __syncthreads();
    const size_t len = (size_t)dim * K;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(X[e]) & 0x7FFFFFFFFFFFFFFFull;
        atomicMax(&sm[e % K], b);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < K; c += blockDim.x)
        if (sm[c]) atomicMax(&mx[c], sm[c]);
}

// f_c from the bits of max |X(:, c)|: |X(:, c)| 2^-f_c < 1/2 (0 for a zero
// column; NaN or infinity is passed on through the digits)
__device__ __forceinline__ int oz_colexp(unsigned long long bits) {
    return bits ? (int)((bits >> 52) & 0x7FF) - 1021 : 0;
}

// round(x 2^(56 - f)) for |x| < 2^(f - 1), from the bits of x alone
// (integer pipes; round half to even, as a float64 rounding would):
// x = m 2^(ex - 1075) with the 53-bit significand m (ex the biased exponent,
// 1 for subnormals), so the value is m shifted left by sh = ex - 1019 - f
// (sh <= 2 since |x| < 2^(f - 1)), rounded where sh < 0.  Inf and NaN only
// occur in columns flagged by f > 1025, whose results are replaced by NaN.
__device__ __forceinline__ long long oz_fixed(double x, int f) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7FF);
    if (ex == 0x7FF) return 0;
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (ex ? 0x10000000000000ull : 0ull);
    const int sh = (ex ? ex : 1) - 1019 - f;
    unsigned long long v;
    if (sh >= 0) {
        v = m << sh;
    } else if (sh > -64) {
        const int r = -sh;
        const unsigned long long q = m >> r, rem = m & ((1ull << r) - 1ull), half = 1ull << (r - 1);
        v = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
    } else {
        v = 0;
    }
    return (b >> 63) ? -(long long)v : (long long)v;
}

// Column slices of X: p[(t K + c) ldk + j] = digit t of X(j, c) 2^-f_c
// (zero for j >= dim), fx[c] = f_c.  The value is rounded once to
// v = round(X 2^(56 - f)), |v| <= 2^55, and cut into eight balanced 7-bit
// digits by integer shifts, most significant first: d = floor((v + 2^(w-1))
// / 2^w), v -= d 2^w for w = 49, 42, ..., 7, then the last digit is v itself
// (each |d| <= 64).  One block per 16 rows (a 16 x K tile of X staged in
// shared memory, so that reads run along the columns and writes along the
// rows of the slices); all of it integer work.
constexpr int OZ_XS_ROWS = 16;
template <int K>
__global__ void __launch_bounds__(256) k_oz_xslice(int dim, int ldk, const double* __restrict__ X,
                                                   const unsigned long long* __restrict__ mx,
                                                   __nv_bfloat16* __restrict__ p, int* __restrict__ fx) {
    __shared__ double xs[OZ_XS_ROWS][K + 1];
    __shared__ int fs[K];
    const int j0 = blockIdx.x * OZ_XS_ROWS;
    for (int e = threadIdx.x; e < OZ_XS_ROWS * K; e += blockDim.x) {
        const int jj = e / K, c = e % K, j = j0 + jj;
        xs[jj][c] = j < dim ? X[(size_t)j * K + c] : 0.0;
    }
    for (int c = threadIdx.x; c < K; c += blockDim.x) {
        fs[c] = oz_colexp(mx[c]);
        if (blockIdx.x == 0) fx[c] = fs[c];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < OZ_XS_ROWS * K; e += blockDim.x) {
        const int c = e / OZ_XS_ROWS, jj = e % OZ_XS_ROWS;
        long long v = oz_fixed(xs[jj][c], fs[c]);
        __nv_bfloat16* out = p + (size_t)c * ldk + j0 + jj;
#pragma unroll
        for (int t = 0; t < OZ_SLICES - 1; t++) {
            const int w = OZ_BITS * (OZ_SLICES - 1 - t);
            const long long d = (v + (1ll << (w - 1))) >> w;
            v -= d << w;
            out[(size_t)t * K * ldk] = __float2bfloat16_rn((float)(int)d);  // |d| <= 64
        }
        out[(size_t)(OZ_SLICES - 1) * K * ldk] = __float2bfloat16_rn((float)(int)v);
    }
}

// part[((z I + item) dimp + i) K + c] = (H, L) of the products D_st(i, c)
// of the work item (s, t0 .. t0 + nt - 1) over the reduction split z
// (digits counted from 0): H = sum over s + t <= 2 of D_st 2^(7 (2 - s - t)),
// L = sum over 3 <= s + t <= 7 of D_st 2^(7 (7 - s - t)), in int64.
template <int K>
__global__ void __launch_bounds__(OZ_THREADS) k_oz_gemm(const __grid_constant__ CUtensorMap tmQ,
                                                        const __grid_constant__ CUtensorMap tmP,
                                                        const __grid_constant__ OzItems items, int dim,
                                                        int dimp, int nchunks, int chunks_per_split,
                                                        longlong2* __restrict__ part, int* d_err) {
    extern __shared__ uint8_t oz_raw[];
    __shared__ OzShared sh;
    using C = OzCfg<K>;
    constexpr int STAGES = C::STAGES;
    const uint32_t base = smem_u32(oz_raw);
    uint8_t* ring = oz_raw + ((1024u - (base & 1023u)) & 1023u);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * OZ_BM, item = blockIdx.y, z = blockIdx.z;
    const int s = items.s[item], T0 = items.t0[item], NT = items.nt[item];
    const int ncol = NT * K;  // <= 256
    uint32_t tcols = 32;
    while ((int)tcols < ncol) tcols <<= 1;
    const int kc0 = z * chunks_per_split;
    const int nk = min(chunks_per_split, nchunks - kc0);
    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; i++) {
            mbar_init(&sh.full[i], 1);
            mbar_init(&sh.empty[i], 1);
        }
        mbar_init(&sh.done, 1);
        sh.fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 2) {
        tmem_alloc(&sh.tmem, tcols);
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = sh.tmem;
    const uint32_t stage_bytes = (uint32_t)(C::A_BYTES + NT * K * OZ_BK * 2);
    if (warp == 0 && lane == 0) {
        int kb = 0;
        for (; kb < nk; kb++) {
            const int st = kb % STAGES;
            if (kb >= STAGES && !mbar_wait(&sh.empty[st], ((kb / STAGES) - 1) & 1, d_err, ERR_WAIT_EMPTY)) {
                sh.fail = 1;
                break;
            }
            if (*(volatile int*)&sh.fail) break;
            uint8_t* sp = ring + st * C::STAGE;
            const int kx = (kc0 + kb) * OZ_BK;
            mbar_expect_tx(&sh.full[st], stage_bytes);
            tma_load_2d(sp, &tmQ, &sh.full[st], kx, s * dimp + m0);
            for (int t = 0; t < NT; t++)
                tma_load_2d(sp + C::A_BYTES + t * K * 128, &tmP, &sh.full[st], kx, (T0 + t) * K);
        }
        // copies in flight: wait for the last load of every stage (bounded)
        for (int j = (kb > STAGES ? kb - STAGES : 0); j < kb; j++)
            mbar_wait(&sh.full[j % STAGES], (j / STAGES) & 1, d_err, ERR_WAIT_FULL);
    } else if (warp == 1 && lane == 0) {
        for (int kb = 0; kb < nk; kb++) {
            const int st = kb % STAGES;
            if (!mbar_wait(&sh.full[st], (kb / STAGES) & 1, d_err, ERR_WAIT_FULL) || *(volatile int*)&sh.fail) {
                sh.fail = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a = smem_u32(ring + st * C::STAGE);
            const uint32_t b = a + C::A_BYTES;
            const uint32_t idesc = idesc_f16(OZ_BM, ncol, 1, 0);
#pragma unroll
            for (int kk = 0; kk < OZ_BK / 16; kk++)
                umma_f16(taddr, sdesc(a + kk * 32, 16, 1024), sdesc(b + kk * 32, 16, 1024), idesc,
                         (kb > 0 || kk > 0) ? 1u : 0u);
            umma_commit(&sh.empty[st]);  // the stage is free once these MMAs are done
        }
        umma_commit(&sh.done);
    }
    __syncwarp();
    bool ok = nk > 0 && mbar_wait(&sh.done, 0, d_err, ERR_WAIT_DONE);
    ok = __syncthreads_and(ok && !*(volatile int*)&sh.fail);  // uniform: tcgen05.ld is warp-collective
    tc_fence_after();
    const int row = m0 + warp * 32 + lane;
    if (ok) {
        longlong2* o = part + (((size_t)z * items.count + item) * dimp + row) * K;
#pragma unroll 1
        for (int c0 = 0; c0 < K; c0 += 16) {
            long long hi[16], lo[16];
#pragma unroll
            for (int u = 0; u < 16; u++) hi[u] = lo[u] = 0;
            for (int t = 0; t < NT; t++) {
                float v[16];
                tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * K + c0), v);
                const int l = s + T0 + t;
                if (l <= 2) {
                    const int sh = OZ_BITS * (2 - l);
#pragma unroll
                    for (int u = 0; u < 16; u++) hi[u] += (long long)__float2int_rn(v[u]) << sh;
                } else {
                    const int sh = OZ_BITS * (7 - l);
#pragma unroll
                    for (int u = 0; u < 16; u++) lo[u] += (long long)__float2int_rn(v[u]) << sh;
                }
            }
            if (row < dim) {
#pragma unroll
                for (int u = 0; u < 16; u++) o[c0 + u] = make_longlong2(hi[u], lo[u]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 2) tmem_dealloc(taddr, tcols);
}

// Y = alpha 2^(e_i + f_c) (2^-28 H + 2^-63 L) + beta Sub, with H and L the
// int64 sums of the partials of all splits and slices (exact, so the order
// does not matter); one float64 conversion per output
template <int K>
__global__ void k_oz_sum(int dim, int dimp, int nparts, const longlong2* __restrict__ part,
                         const int* __restrict__ ex, const int* __restrict__ fx, double* Y, double alpha,
                         const double* Sub, double beta) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)dim * K) return;
    const int i = (int)(e / K), c = (int)(e % K);
    long long H = 0, L = 0;
    for (int g = 0; g < nparts; g++) {
        const longlong2 v = part[((size_t)g * dimp + i) * K + c];
        H += v.x;
        L += v.y;
    }
    double y = fma((double)L, 0x1p-35, (double)H);  // 2^28 (2^-28 H + 2^-63 L)
    // f_c > 1025 flags a column with an infinity or NaN: pass it on
    y = fx[c] > 1025 ? __longlong_as_double(0x7FF8000000000000ll) : ldexp(y, ex[i] + fx[c] - 28);
    Y[e] = Sub ? fma(beta, Sub[e], alpha * y) : alpha * y;
}

// work items of a tile for K columns: every digit s of M with its digits t
// of X (s + t <= S - 1) in groups of at most TN, the longest first
template <int K>
OzItems oz_items() {
    OzItems it{};
    for (int nt = OzCfg<K>::TN; nt >= 1; nt--)
        for (int s = 0; s < OZ_SLICES; s++)
            for (int t0 = 0; t0 < OZ_SLICES - s; t0 += OzCfg<K>::TN) {
                const int len = std::min(OzCfg<K>::TN, OZ_SLICES - s - t0);
                if (len != nt) continue;
                it.s[it.count] = (signed char)s;
                it.t0[it.count] = (signed char)t0;
                it.nt[it.count] = (signed char)len;
                it.count++;
            }
    return it;
}
// most work items any K has (K = 16: one per digit s; K = 64: 12)
constexpr int OZ_ITEMS_MAX = 2 * OZ_SLICES;

int oz_dimp(int dim) { return (dim + OZ_BM - 1) / OZ_BM * OZ_BM; }
int oz_ldk(int dim) { return (dim + OZ_BK - 1) / OZ_BK * OZ_BK; }
int oz_splits(int dim, int cps = OZ_CHUNKS) { return (oz_ldk(dim) / OZ_BK + cps - 1) / cps; }

template <int K>
awg_status launch_oz(const OzMat& m, const double* X, double* Y, double alpha, const double* Sub, double beta,
                     void* xs, double* part, int* d_err, cudaStream_t s, int cps) {
    const int ldk = m.ldk;
    __nv_bfloat16* p = (__nv_bfloat16*)xs;
    unsigned long long* mx = (unsigned long long*)((char*)xs + (size_t)OZ_SLICES * K * ldk * 2);
    int* fx = (int*)(mx + K);
    AWG_CUDA(cudaMemsetAsync(mx, 0, K * sizeof(unsigned long long), s));
    k_oz_colmax<K><<<std::min(152, (m.dim * K + 255) / 256), 256, 0, s>>>(m.dim, X, mx);
    AWG_LAUNCH();
    k_oz_xslice<K><<<ldk / OZ_XS_ROWS, 256, 0, s>>>(m.dim, ldk, X, mx, p, fx);
    AWG_LAUNCH();
    CUtensorMap tq, tp;
    if (!make_map(&tq, m.q, 1, (uint64_t)OZ_SLICES * m.dimp, ldk, ldk, OZ_BK, OZ_BM) ||
        !make_map(&tp, p, 1, (uint64_t)OZ_SLICES * K, ldk, ldk, OZ_BK, K))
        return AWG_ERR_INVALID_ARG;
    auto kern = k_oz_gemm<K>;
    static bool attr = false;
    if (!attr) {
        AWG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, OzCfg<K>::SMEM));
        attr = true;
    }
    const int nchunks = ldk / OZ_BK, splits = oz_splits(m.dim, cps);
    const OzItems items = oz_items<K>();
    kern<<<dim3(m.dimp / OZ_BM, items.count, splits), OZ_THREADS, OzCfg<K>::SMEM, s>>>(
        tq, tp, items, m.dim, m.dimp, nchunks, cps, (longlong2*)part, d_err);
    AWG_LAUNCH();
    const size_t len = (size_t)m.dim * K;
    k_oz_sum<K><<<(unsigned)((len + 255) / 256), 256, 0, s>>>(m.dim, m.dimp, splits * items.count,
                                                             (const longlong2*)part, m.ex, fx, Y, alpha, Sub, beta);
    AWG_LAUNCH();
    return AWG_OK;
}

}  // namespace

size_t oz_slices_bytes(int dim) { return (size_t)OZ_SLICES * oz_dimp(dim) * oz_ldk(dim) * 2; }
size_t oz_part_elems(int dim, int K, int chunks_per_split) {
    // (H, L) int64 pairs per work item and reduction split
    return (size_t)oz_splits(dim, chunks_per_split) * OZ_ITEMS_MAX * oz_dimp(dim) * K * 2;
}
size_t oz_xs_bytes(int dim, int K) { return (size_t)OZ_SLICES * K * oz_ldk(dim) * 2 + (size_t)K * 12; }

awg_status oz_slice_matrix(const double* M, int dim, DevBuf& q, DevBuf& ex, Handle* h, cudaStream_t s, OzMat* out) {
    if (dim < 1) return AWG_ERR_INVALID_ARG;
    const int dimp = oz_dimp(dim), ldk = oz_ldk(dim);
    if (!q.p) AWG_TRY(dalloc(h, q, oz_slices_bytes(dim)));
    if (!ex.p) AWG_TRY(dalloc(h, ex, (size_t)dimp * 4));
    AWG_CUDA(cudaMemsetAsync(q.p, 0, oz_slices_bytes(dim), s));
    AWG_CUDA(cudaMemsetAsync(ex.p, 0, (size_t)dimp * 4, s));
    k_oz_slice_rows<<<dim, 256, 0, s>>>(dim, dimp, ldk, M, (__nv_bfloat16*)q.p, (int*)ex.p);
    AWG_LAUNCH();
    out->q = q.p;
    out->ex = (const int*)ex.p;
    out->dim = dim;
    out->dimp = dimp;
    out->ldk = ldk;
    return AWG_OK;
}

awg_status oz_gemm(const OzMat& m, int K, const double* X, double* Y, double alpha, const double* Sub, double beta,
                   void* xs, double* part, int* d_err, cudaStream_t s, int chunks_per_split) {
    if (m.dim < 1 || !m.q || chunks_per_split < 1 || chunks_per_split > OZ_CHUNKS) return AWG_ERR_INVALID_ARG;
    const int c = chunks_per_split;
    if (K == 16) return launch_oz<16>(m, X, Y, alpha, Sub, beta, xs, part, d_err, s, c);
    if (K == 32) return launch_oz<32>(m, X, Y, alpha, Sub, beta, xs, part, d_err, s, c);
    if (K == 64) return launch_oz<64>(m, X, Y, alpha, Sub, beta, xs, part, d_err, s, c);
    return AWG_ERR_INVALID_ARG;
}

}  // namespace awg
