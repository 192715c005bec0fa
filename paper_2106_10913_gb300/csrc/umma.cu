// Tensor-core passes over the 16-bit second coarse basis W (float16 with
// power-of-two row and column scales, or bfloat16) for K right-hand sides at
// once: W^T B (first projection of Def. 10) and W D (prolongation of the
// second coarse correction).  With K columns the two passes are GEMMs of
// shape (ldw x n) x (n x K) and (n x ldw) x (ldw x K), bound by the bytes of
// W; on the CUDA cores their K FMAs per element of W would bound them
// instead.
//
// Both kernels: one CTA per 256-row tile of the product (two M = 128
// accumulators), the K right-hand sides as N, the reduction in 64-deep
// chunks.  W tiles and the right-hand-side tiles come through TMA
// (cp.async.bulk.tensor, 128-byte swizzle) into a shared-memory ring
// guarded by mbarriers; one
// thread issues tcgen05.mma (kind::f16, float32 accumulation in tensor
// memory); the four warps read the accumulator back with tcgen05.ld.  The
// right-hand sides enter as two 16-bit parts (high and low: about 22
// significant bits for float16), accumulated into the same tensor-memory
// tile, so the products carry the rounding of W alone.
//
// Every wait is bounded (about two seconds): a wait that gives up records a
// code in *d_err and the CTA winds down (waits for its copies in flight,
// frees its tensor memory) instead of hanging.

#include "block.cuh"
#include "tcgen05.cuh"

#include <cuda.h>

#include <algorithm>
#include <cstdint>

namespace awg {

namespace {

constexpr int UM_BM = 128;     // rows of the product per CTA (MMA M)
constexpr int UM_BK = 64;      // reduction depth per stage (128 bytes of 16-bit)
constexpr int UM_STAGES = 4;
constexpr int UM_THREADS = 128;

template <int K>
struct UmCfg {
    static constexpr int A_BYTES = 2 * UM_BM * UM_BK * 2;        // 32 KB: 256 rows (or columns) of W
    static constexpr int B_BYTES = 2 * K * UM_BK * 2;            // hi + lo parts
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int STAGES = 2;
    static constexpr int SMEM = STAGES * STAGE + 1024;
    static constexpr int TMEM_COLS = 2 * K < 32 ? 32 : 2 * K;
};

struct UmShared {
    uint64_t full[UM_STAGES];
    uint64_t empty[UM_STAGES];
    uint64_t done;
    uint32_t tmem;
    int fail;
};

// Shared prologue: 1024-aligned stage ring, barriers, tensor memory.
template <int K, typename C = UmCfg<K>>
__device__ __forceinline__ uint8_t* um_setup(uint8_t* raw, UmShared& sh) {
    const uint32_t base = smem_u32(raw);
    uint8_t* ring = raw + ((1024u - (base & 1023u)) & 1023u);
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < UM_STAGES; s++) {
            mbar_init(&sh.full[s], 1);
            mbar_init(&sh.empty[s], 1);
        }
        mbar_init(&sh.done, 1);
        sh.fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 2) {
        tmem_alloc(&sh.tmem, C::TMEM_COLS);
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    return ring;
}

// Producer / MMA issue over nk chunks; the two callbacks issue one stage's
// TMA loads and return its shared-memory descriptors' bases.
// LoadF(stage_ptr, bar, kb); MmaF(a_base, b_base, first)
template <int K, typename C = UmCfg<K>, typename LoadF, typename MmaF>
__device__ __forceinline__ void um_mainloop(uint8_t* ring, UmShared& sh, int nk, int* d_err, LoadF load,
                                            MmaF mma) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0 && lane == 0) {
        int kb = 0;
        for (; kb < nk; kb++) {
            const int st = kb % C::STAGES;
            if (kb >= C::STAGES && !mbar_wait(&sh.empty[st], ((kb / C::STAGES) - 1) & 1, d_err, ERR_WAIT_EMPTY)) {
                sh.fail = 1;
                break;
            }
            if (*(volatile int*)&sh.fail) break;
            uint8_t* sp = ring + st * C::STAGE;
            mbar_expect_tx(&sh.full[st], C::STAGE);
            load(sp, &sh.full[st], kb);
        }
        // copies in flight: wait for the last load of every stage (bounded)
        for (int j = (kb > C::STAGES ? kb - C::STAGES : 0); j < kb; j++)
            mbar_wait(&sh.full[j % C::STAGES], (j / C::STAGES) & 1, d_err, ERR_WAIT_FULL);
    } else if (warp == 1 && lane == 0) {
        bool ok = true;
        for (int kb = 0; kb < nk; kb++) {
            const int st = kb % C::STAGES;
            if (!mbar_wait(&sh.full[st], (kb / C::STAGES) & 1, d_err, ERR_WAIT_FULL) || *(volatile int*)&sh.fail) {
                sh.fail = 1;
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t sp = smem_u32(ring + st * C::STAGE);
            mma(sp, sp + C::A_BYTES, kb == 0);
            umma_commit(&sh.empty[st]);  // the stage is free once these MMAs are done
        }
        (void)ok;
        umma_commit(&sh.done);
    }
    __syncwarp();
}

// Both W passes take two 128-row tiles of the product per CTA (M = 256 in
// two MMAs that share the right-hand-side tile of each stage), so that the
// right-hand side, which every CTA reads whole (2K x ldw for W D, 2K x
// rows of its split for W^T B), costs half a byte per byte of W.  Stages
// of 32 KB of W + 2K x 64 16-bit right-hand sides, two stages (two CTAs
// per SM at K = 64); the two accumulators side by side in tensor memory
// (2K columns).

// W D: out(i, :) = sum_c W(i, c) (Dt_hi(:, c) + Dt_lo(:, c)) for the 256
// rows of this CTA.  A = W tile (K-major: rows of W, 64 columns per stage,
// one 64 x 256 box: rows 0-127, then 128-255), B = Dt tile (K-major: 2K
// rows, 64 columns of W per stage).
template <int K, int BF16>
__global__ void __launch_bounds__(UM_THREADS) k_umma_wd2(const __grid_constant__ CUtensorMap tmW,
                                                         const __grid_constant__ CUtensorMap tmD, int n, int ldw,
                                                         float* __restrict__ out, int* d_err) {
    extern __shared__ uint8_t um_raw[];
    __shared__ UmShared sh;
    using C = UmCfg<K>;
    uint8_t* ring = um_setup<K, C>(um_raw, sh);
    const uint32_t taddr = sh.tmem;
    const int m0 = blockIdx.x * 2 * UM_BM;
    const int nk = (ldw + UM_BK - 1) / UM_BK;
    constexpr uint32_t idesc = idesc_f16(UM_BM, K, BF16, 0);
    um_mainloop<K, C>(
        ring, sh, nk, d_err,
        [&](uint8_t* sp, uint64_t* bar, int kb) {
            tma_load_2d(sp, &tmW, bar, kb * UM_BK, m0);
            tma_load_2d(sp + C::A_BYTES, &tmD, bar, kb * UM_BK, 0);
        },
        [&](uint32_t a, uint32_t b, bool first) {
#pragma unroll
            for (int kk = 0; kk < UM_BK / 16; kk++) {
                const uint64_t bh = sdesc(b + kk * 32, 16, 1024);
                const uint64_t bl = sdesc(b + K * 128 + kk * 32, 16, 1024);
#pragma unroll
                for (int t = 0; t < 2; t++) {
                    const uint64_t ad = sdesc(a + t * (UM_BM * 128) + kk * 32, 16, 1024);
                    const uint32_t d = taddr + (uint32_t)(t * K);
                    umma_f16(d, ad, bh, idesc, (first && kk == 0) ? 0u : 1u);
                    umma_f16(d, ad, bl, idesc, 1u);
                }
            }
        });
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    bool ok = mbar_wait(&sh.done, 0, d_err, ERR_WAIT_DONE);
    ok = __syncthreads_and(ok && !*(volatile int*)&sh.fail);  // uniform: tcgen05.ld is warp-collective
    tc_fence_after();
    if (ok) {
#pragma unroll
        for (int t = 0; t < 2; t++) {
            const int row = m0 + t * UM_BM + warp * 32 + lane;
#pragma unroll
            for (int c0 = 0; c0 < K; c0 += 16) {
                float v[16];
                tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * K + c0), v);
                if (row < n) {
                    float4* o = reinterpret_cast<float4*>(out + (size_t)row * K + c0);
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 2) tmem_dealloc(taddr, C::TMEM_COLS);
}

// W^T B: part(split, c, :) = sum over the rows i of this split of W(i, c)
// (Bt_hi(:, i) + Bt_lo(:, i)) for the 256 columns c of this CTA.  A = W^T
// tiles (MN-major: four 64-column boxes of W side by side, 64 rows per
// stage; columns 0-127 in boxes 0 and 1, 128-255 in boxes 2 and 3), B = Bt
// tile (K-major: 2K rows, 64 rows of W per stage).
template <int K, int BF16>
__global__ void __launch_bounds__(UM_THREADS) k_umma_wt2(const __grid_constant__ CUtensorMap tmW,
                                                         const __grid_constant__ CUtensorMap tmB, int n, int ldw,
                                                         int rows_per_split, float* __restrict__ part, int* d_err) {
    extern __shared__ uint8_t um_raw[];
    __shared__ UmShared sh;
    using C = UmCfg<K>;
    constexpr int BOX = UM_BK * 64 * 2;  // one 64-column x 64-row box, 8 KB
    uint8_t* ring = um_setup<K, C>(um_raw, sh);
    const uint32_t taddr = sh.tmem;
    const int c0 = blockIdx.x * 2 * UM_BM;
    const int i0 = blockIdx.y * rows_per_split;
    const int i1 = min(n, i0 + rows_per_split);
    const int nk = i1 > i0 ? (i1 - i0 + UM_BK - 1) / UM_BK : 0;
    constexpr uint32_t idesc = idesc_f16(UM_BM, K, BF16, 1);
    um_mainloop<K, C>(
        ring, sh, nk, d_err,
        [&](uint8_t* sp, uint64_t* bar, int kb) {
            const int i = i0 + kb * UM_BK;
#pragma unroll
            for (int q = 0; q < 4; q++) tma_load_2d(sp + q * BOX, &tmW, bar, c0 + 64 * q, i);
            tma_load_2d(sp + C::A_BYTES, &tmB, bar, i, 0);
        },
        [&](uint32_t a, uint32_t b, bool first) {
#pragma unroll
            for (int kk = 0; kk < UM_BK / 16; kk++) {
                const uint64_t bh = sdesc(b + kk * 32, 16, 1024);
                const uint64_t bl = sdesc(b + K * 128 + kk * 32, 16, 1024);
#pragma unroll
                for (int t = 0; t < 2; t++) {
                    // 16 rows of W per MMA: two 8-row groups, 2048 bytes further
                    const uint64_t ad = sdesc(a + t * 2 * BOX + kk * 2048, BOX, 1024);
                    const uint32_t d = taddr + (uint32_t)(t * K);
                    umma_f16(d, ad, bh, idesc, (first && kk == 0) ? 0u : 1u);
                    umma_f16(d, ad, bl, idesc, 1u);
                }
            }
        });
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    bool ok = nk > 0 && mbar_wait(&sh.done, 0, d_err, ERR_WAIT_DONE);
    ok = __syncthreads_and(ok && !*(volatile int*)&sh.fail);  // uniform: tcgen05.ld is warp-collective
    tc_fence_after();
#pragma unroll
    for (int t = 0; t < 2; t++) {
        const int c = c0 + t * UM_BM + warp * 32 + lane;
        float* o = part + ((size_t)blockIdx.y * ldw + c) * K;
#pragma unroll
        for (int j0 = 0; j0 < K; j0 += 16) {
            float v[16];
            if (ok) tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(t * K + j0), v);
            else
#pragma unroll
                for (int q = 0; q < 16; q++) v[q] = 0.f;
            if (c < ldw) {
                float4* o4 = reinterpret_cast<float4*>(o + j0);
#pragma unroll
                for (int q = 0; q < 4; q++) o4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 2) tmem_dealloc(taddr, C::TMEM_COLS);
}

// D[tmem] (+)= A[smem] * B[smem]^T, kind::tf32 (float32 operands read as
// TF32, float32 accumulation)
__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Instruction descriptor of kind::tf32: float32 accumulator, A and B TF32,
// both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Position (float index) of element (r, q), q < 32, of a 128-byte-row tile in
// the 128-byte swizzled layout: 16-byte chunk q / 4 of row r is stored at
// chunk (q / 4) ^ (r % 8).
__device__ __forceinline__ int sw128_f32(int r, int q) { return r * 32 + ((((q >> 2) ^ (r & 7))) << 2) + (q & 3); }

// Tiles of the float32 local pseudo-inverses G_s for the tensor cores: tile
// (rt, kc) of subdomain s holds G_s(rt*128 + r, kc*32 + q), r < 128, q < 32
// (zero outside n^s x n^s), as a 16 KB image in the 128-byte swizzled
// K-major layout.  G_s is symmetric, so its rows are read as its columns.
__global__ void __launch_bounds__(256) k_tile_g(const int* __restrict__ sub_ptr, const int64_t* __restrict__ g32off,
                                                const float* __restrict__ G, const int64_t* __restrict__ gt_off,
                                                float* __restrict__ Gt) {
    const int s = blockIdx.y;
    const int m = sub_ptr[s + 1] - sub_ptr[s];
    const int ld = (m + 3) & ~3;
    const int RT = (m + 127) / 128, KC = (m + 31) / 32;
    const int t = blockIdx.x;
    if (t >= RT * KC) return;
    const int rt = t / KC, kc = t % KC;
    const float* Gs = G + g32off[s];
    float* img = Gt + (size_t)(gt_off[s] + t) * 4096;
    for (int e = threadIdx.x; e < 4096; e += 256) {
        const int r = e / 32, q = e % 32;
        const int i = rt * 128 + r, j = kc * 32 + q;
        img[sw128_f32(r, q)] = (i < m && j < m) ? Gs[(size_t)i * ld + j] : 0.f;
    }
}

// Right-hand-side images of the tensor-core local solves: for subdomain s
// and chunk kc, the TF32 high and low parts (round to nearest: hi =
// tf32(x), lo = tf32(x - hi)) of X(idx_s(kc*32 + jj), c) as two K x 32
// images (row c) in the 128-byte swizzled layout, at
// lt + (kc_prefix[s] + kc) * 2 * K * 32 floats.
template <int K>
__global__ void __launch_bounds__(256) k_local_bimg(const int* __restrict__ sub_ptr, const int* __restrict__ sub_idx,
                                                    const int64_t* __restrict__ kc_prefix,
                                                    const float* __restrict__ X, float* __restrict__ lt) {
    __shared__ float xs[32][K + 1];
    const int s = blockIdx.y, kc = blockIdx.x;
    const int p0 = sub_ptr[s], m = sub_ptr[s + 1] - p0;
    if (kc * 32 >= m) return;
    for (int e = threadIdx.x; e < 32 * K; e += 256) {
        const int jj = e / K, c = e % K, p = kc * 32 + jj;
        xs[jj][c] = (p < m) ? X[(size_t)sub_idx[p0 + p] * K + c] : 0.f;
    }
    __syncthreads();
    float* hi = lt + (size_t)(kc_prefix[s] + kc) * 2 * K * 32;
    float* lo = hi + K * 32;
    for (int e = threadIdx.x; e < 32 * K; e += 256) {
        const int c = e / 32, q = e % 32;
        const float x = xs[q][c];
        const float h = tf32_rna(x);
        hi[sw128_f32(c, q)] = h;
        lo[sw128_f32(c, q)] = tf32_rna(x - h);
    }
}

// U_s(rt*128 + r, :) = sum over kc of G_s tile (rt, kc) times X_s chunk kc,
// with G = G_hi + G_lo and X = X_hi + X_lo split in TF32 and the three
// products hi*hi + hi*lo + lo*hi accumulated in float32 in tensor memory
// (two MMAs per step: G_hi against the stacked [X_hi; X_lo], G_lo against X_hi)
// (error about 2^-22 of each product, the float32 level).  One CTA per
// 128-row tile (flattened list tile_sub / tile_rt); 6 warps: warp 0 issues
// the bulk copies of the two right-hand-side images of each stage, warp 1
// the MMAs, and warps 2-5 load the 16 KB G images straight into registers,
// UL_PF images ahead of the stage they go to (G is read from HBM once, and
// its loads are in flight while earlier stages are split and multiplied),
// split them there and write hi and lo into the stage; they also read the
// accumulator back.
constexpr int UL_STAGES = 2;  // split G stages (hi + lo): two CTAs share an SM
constexpr int UL_BMAX = 4;    // right-hand-side stages (at most)
constexpr int UL_PF = 3;      // G images held in registers ahead of the stage they go to
constexpr int UL_THREADS = 192;
// The right-hand-side images have a ring of their own, deeper than the
// split G stages where shared memory allows (four stages up to 32 columns),
// so that their copies from L2 are issued further ahead of the MMAs that
// read them; at 64 columns two CTAs per SM leave room for two (two split
// G stages of 32 KB and three right-hand-side stages of 16 KB exceed half
// of the SM's 228 KB by the alignment slack).
template <int K>
struct UlCfg {
    static constexpr int A_BYTES = 128 * 32 * 4;          // 16 KB G image
    static constexpr int B_BYTES = 2 * K * 32 * 4;        // hi + lo right-hand-side images
    static constexpr int A_STAGE = 2 * A_BYTES;           // G hi, G lo
    static constexpr int B_STAGES = K == 64 ? 2 : UL_BMAX;
    static constexpr int SMEM = UL_STAGES * A_STAGE + B_STAGES * B_BYTES + 1024;
    static constexpr int TMEM_COLS = 2 * K < 32 ? 32 : 2 * K;  // [hi*hi + lo*hi | hi*lo]
};

struct UlShared {
    uint64_t full[UL_BMAX];      // right-hand-side stage landed
    uint64_t bempty[UL_BMAX];    // right-hand-side stage read by the MMAs
    uint64_t ready[UL_STAGES];   // split G stage written
    uint64_t empty[UL_STAGES];   // split G stage read by the MMAs
    uint64_t done;
    uint32_t tmem;
    int fail;
};

template <int K>
__global__ void __launch_bounds__(UL_THREADS) k_umma_local(const int* __restrict__ sub_ptr,
                                                           const int* __restrict__ tile_sub,
                                                           const int* __restrict__ tile_rt,
                                                           const int64_t* __restrict__ gt_off,
                                                           const int64_t* __restrict__ kc_prefix,
                                                           const float* __restrict__ Gt, const float* __restrict__ lt,
                                                           float* __restrict__ out, int* d_err) {
    extern __shared__ uint8_t ul_raw[];
    __shared__ UlShared sh;
    using C = UlCfg<K>;
    const uint32_t base = smem_u32(ul_raw);
    uint8_t* ring = ul_raw + ((1024u - (base & 1023u)) & 1023u);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = tile_sub[blockIdx.x], rt = tile_rt[blockIdx.x];
    const int p0 = sub_ptr[s], m = sub_ptr[s + 1] - p0;
    const int KC = (m + 31) / 32;
    constexpr int BS = C::B_STAGES;
    uint8_t* bring = ring + UL_STAGES * C::A_STAGE;
    if (threadIdx.x == 0) {
        for (int i = 0; i < UL_STAGES; i++) {
            mbar_init(&sh.ready[i], 128);
            mbar_init(&sh.empty[i], 1);
        }
        for (int i = 0; i < BS; i++) {
            mbar_init(&sh.full[i], 1);
            mbar_init(&sh.bempty[i], 1);
        }
        mbar_init(&sh.done, 1);
        sh.fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 2) {
        tmem_alloc(&sh.tmem, C::TMEM_COLS);
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = sh.tmem;
    const float* gsrc = Gt + (size_t)(gt_off[s] + (int64_t)rt * KC) * 4096;
    const float* bsrc = lt + (size_t)kc_prefix[s] * 2 * K * 32;
    if (warp == 0) {
        if (lane == 0) {
            // right-hand-side images through the bulk copy engine
            int kc = 0;
            for (; kc < KC; kc++) {
                const int bt = kc % BS;
                if (kc >= BS && !mbar_wait(&sh.bempty[bt], ((kc / BS) - 1) & 1, d_err, ERR_WAIT_EMPTY)) {
                    sh.fail = 1;
                    break;
                }
                if (*(volatile int*)&sh.fail) break;
                mbar_expect_tx(&sh.full[bt], C::B_BYTES);
                bulk_load(bring + bt * C::B_BYTES, bsrc + (size_t)kc * 2 * K * 32, C::B_BYTES, &sh.full[bt]);
            }
            for (int j = (kc > BS ? kc - BS : 0); j < kc; j++)
                mbar_wait(&sh.full[j % BS], (j / BS) & 1, d_err, ERR_WAIT_FULL);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // columns [0, K): G_hi X_hi + G_lo X_hi; [K, 2K): G_hi X_lo (one
            // MMA over the hi and lo right-hand-side images stacked as 2K rows)
            constexpr uint32_t idesc2 = idesc_tf32(128, 2 * K);
            constexpr uint32_t idesc1 = idesc_tf32(128, K);
            for (int kc = 0; kc < KC; kc++) {
                const int st = kc % UL_STAGES, bt = kc % BS;
                if (!mbar_wait(&sh.full[bt], (kc / BS) & 1, d_err, ERR_WAIT_FULL) ||
                    !mbar_wait(&sh.ready[st], (kc / UL_STAGES) & 1, d_err, ERR_WAIT_FULL) ||
                    *(volatile int*)&sh.fail) {
                    sh.fail = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t a = smem_u32(ring + st * C::A_STAGE);
                const uint32_t al = a + C::A_BYTES, b = smem_u32(bring + bt * C::B_BYTES);
#pragma unroll
                for (int kk = 0; kk < 4; kk++) {  // 8 TF32 values (32 bytes) per MMA
                    const uint64_t ah = sdesc(a + kk * 32, 16, 1024), alo = sdesc(al + kk * 32, 16, 1024);
                    const uint64_t bb = sdesc(b + kk * 32, 16, 1024);
                    umma_tf32(taddr, ah, bb, idesc2, (kc == 0 && kk == 0) ? 0u : 1u);
                    umma_tf32(taddr, alo, bb, idesc1, 1u);
                }
                umma_commit(&sh.empty[st]);   // the split G stage is free once these MMAs are done,
                umma_commit(&sh.bempty[bt]);  // and so is the right-hand-side stage
            }
            umma_commit(&sh.done);
        }
    } else {
        // the G images come straight into registers, UL_PF stages ahead
        // (thread t holds 16-byte chunks t + 128 u of an image, coalesced),
        // and are split there: hi = tf32(g) and lo = tf32(g - hi) are
        // written into the stage once the tensor cores are done with it
        const int t = threadIdx.x - 64;
        const float4* g4 = reinterpret_cast<const float4*>(gsrc);
        float4 g[UL_PF][8];
#pragma unroll
        for (int j = 0; j < UL_PF; j++)
            if (j < KC)
#pragma unroll
                for (int u = 0; u < 8; u++) g[j][u] = __ldcs(g4 + (size_t)j * 1024 + t + 128 * u);
        bool stop = false;
        for (int kb = 0; kb < KC && !stop; kb += UL_PF) {
#pragma unroll
            for (int j = 0; j < UL_PF; j++) {
                const int kc = kb + j;
                if (kc >= KC || stop) break;
                const int st = kc % UL_STAGES;
                if (kc >= UL_STAGES && !mbar_wait(&sh.empty[st], ((kc / UL_STAGES) - 1) & 1, d_err, ERR_WAIT_EMPTY)) {
                    sh.fail = 1;
                    stop = true;
                    break;
                }
                float4* a4 = reinterpret_cast<float4*>(ring + st * C::A_STAGE);
                float4* l4 = reinterpret_cast<float4*>(ring + st * C::A_STAGE + C::A_BYTES);
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    const float4 v = g[j][u];
                    float4 h, l;
                    h.x = tf32_rna(v.x); l.x = tf32_rna(v.x - h.x);
                    h.y = tf32_rna(v.y); l.y = tf32_rna(v.y - h.y);
                    h.z = tf32_rna(v.z); l.z = tf32_rna(v.z - h.z);
                    h.w = tf32_rna(v.w); l.w = tf32_rna(v.w - h.w);
                    a4[t + 128 * u] = h;
                    l4[t + 128 * u] = l;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
                mbar_arrive(&sh.ready[st]);
                if (kc + UL_PF < KC)
#pragma unroll
                    for (int u = 0; u < 8; u++) g[j][u] = __ldcs(g4 + (size_t)(kc + UL_PF) * 1024 + t + 128 * u);
            }
        }
    }
    __syncwarp();
    bool ok = mbar_wait(&sh.done, 0, d_err, ERR_WAIT_DONE);
    ok = __syncthreads_and(ok && !*(volatile int*)&sh.fail);
    tc_fence_after();
    if (warp >= 2 && ok) {
        const int q = warp & 3;  // tensor-memory lanes 32 q .. 32 q + 31
        const int row = rt * 128 + q * 32 + lane;
#pragma unroll
        for (int c0 = 0; c0 < K; c0 += 16) {
            float v[16], w[16];
            tmem_ld16(taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
            tmem_ld16(taddr + ((uint32_t)(q * 32) << 16) + (uint32_t)(K + c0), w);
#pragma unroll
            for (int u = 0; u < 16; u++) v[u] += w[u];
            if (row < m) {
                float4* o = reinterpret_cast<float4*>(out + (size_t)(p0 + row) * K + c0);
#pragma unroll
                for (int u = 0; u < 4; u++) o[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 2) tmem_dealloc(taddr, C::TMEM_COLS);
}

// ----------------------------------------------------------------- host
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    }
    return fn;
}

// rows per split of W^T B: a multiple of the 64-row stage
int split_rows(int n, int splits) {
    const int rps = (n + splits - 1) / splits;
    return (rps + UM_BK - 1) / UM_BK * UM_BK;
}

template <int K, int BF16>
awg_status launch_wd2(const UmmaW& u, const void* Dt, float* out, int* d_err, cudaStream_t s) {
    CUtensorMap mW, mD;
    if (!make_map(&mW, u.W, BF16, u.n, u.ldw, u.ldw, UM_BK, 2 * UM_BM) ||
        !make_map(&mD, Dt, BF16, 2 * K, u.ldw, u.ldw, UM_BK, 2 * K))
        return AWG_ERR_INVALID_ARG;
    auto kern = k_umma_wd2<K, BF16>;
    static bool attr = false;
    if (!attr) {
        AWG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, UmCfg<K>::SMEM));
        attr = true;
    }
    kern<<<(u.n + 2 * UM_BM - 1) / (2 * UM_BM), UM_THREADS, UmCfg<K>::SMEM, s>>>(mW, mD, u.n, u.ldw, out, d_err);
    AWG_LAUNCH();
    return AWG_OK;
}

template <int K, int BF16>
awg_status launch_wt2(const UmmaW& u, const void* Bt, int ldb, float* part, int splits, int* d_err,
                      cudaStream_t s) {
    CUtensorMap mW, mB;
    if (!make_map(&mW, u.W, BF16, u.n, u.ldw, u.ldw, 64, UM_BK) ||
        !make_map(&mB, Bt, BF16, 2 * K, u.n, ldb, UM_BK, 2 * K))
        return AWG_ERR_INVALID_ARG;
    auto kern = k_umma_wt2<K, BF16>;
    static bool attr = false;
    if (!attr) {
        AWG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, UmCfg<K>::SMEM));
        attr = true;
    }
    const int rps = split_rows(u.n, splits);
    const dim3 grid((u.ldw + 2 * UM_BM - 1) / (2 * UM_BM), (u.n + rps - 1) / rps);
    kern<<<grid, UM_THREADS, UmCfg<K>::SMEM, s>>>(mW, mB, u.n, u.ldw, rps, part, d_err);
    AWG_LAUNCH();
    return AWG_OK;
}

template <int K>
awg_status launch_local(const UmmaLocal& u, const float* X, float* lt, float* out, int* d_err, cudaStream_t s) {
    k_local_bimg<K><<<dim3(u.max_kc, u.N), 256, 0, s>>>(u.sub_ptr, u.sub_idx, u.kc_prefix, X, lt);
    AWG_LAUNCH();
    auto kern = k_umma_local<K>;
    static bool attr = false;
    if (!attr) {
        AWG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, UlCfg<K>::SMEM));
        attr = true;
    }
    kern<<<u.ntiles, UL_THREADS, UlCfg<K>::SMEM, s>>>(u.sub_ptr, u.tile_sub, u.tile_rt, u.gt_off, u.kc_prefix, u.Gt,
                                                       lt, out, d_err);
    AWG_LAUNCH();
    return AWG_OK;
}

}  // namespace

// 2D tensor map of a row-major 16-bit matrix (rows x cols, row stride ld
// elements, a multiple of 8), box of box_cols x box_rows, 128-byte swizzle,
// zero fill outside
bool make_map(CUtensorMap* m, const void* ptr, int bf16, uint64_t rows, uint64_t cols, uint64_t ld,
              uint32_t box_cols, uint32_t box_rows) {
    EncodeTiledFn enc = encoder();
    if (!enc || ((uintptr_t)ptr & 15) || (ld % 8)) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {ld * 2};
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t es[2] = {1, 1};
    const CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                           const_cast<void*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

awg_status umma_local_tiles(const UmmaLocal& u, const int64_t* g32off, const float* G, cudaStream_t s) {
    k_tile_g<<<dim3(u.max_tiles_sub, u.N), 256, 0, s>>>(u.sub_ptr, g32off, G, u.gt_off, const_cast<float*>(u.Gt));
    AWG_LAUNCH();
    return AWG_OK;
}

awg_status umma_local(const UmmaLocal& u, int K, const float* X, float* lt, float* out, int* d_err,
                      cudaStream_t s) {
    if (K == 16) return launch_local<16>(u, X, lt, out, d_err, s);
    if (K == 32) return launch_local<32>(u, X, lt, out, d_err, s);
    if (K == 64) return launch_local<64>(u, X, lt, out, d_err, s);
    return AWG_ERR_INVALID_ARG;
}

bool umma_available() { return encoder() != nullptr; }

int umma_wt_splits(int n, int want) {
    const int rps = split_rows(n, std::max(1, want));
    return (n + rps - 1) / rps;
}

awg_status umma_wd(const UmmaW& u, int K, const void* Dt, float* out, int* d_err, cudaStream_t s) {
    if (u.n < 1 || u.ldw < 8 || (u.ldw % 8)) return AWG_ERR_INVALID_ARG;
    if (K == 16) return u.bf16 ? launch_wd2<16, 1>(u, Dt, out, d_err, s) : launch_wd2<16, 0>(u, Dt, out, d_err, s);
    if (K == 32) return u.bf16 ? launch_wd2<32, 1>(u, Dt, out, d_err, s) : launch_wd2<32, 0>(u, Dt, out, d_err, s);
    if (K == 64) return u.bf16 ? launch_wd2<64, 1>(u, Dt, out, d_err, s) : launch_wd2<64, 0>(u, Dt, out, d_err, s);
    return AWG_ERR_INVALID_ARG;
}

awg_status umma_wt(const UmmaW& u, int K, const void* Bt, int ldb, float* part, int splits, int* d_err,
                   cudaStream_t s) {
    if (u.n < 1 || u.ldw < 8 || (u.ldw % 8) || (ldb % 8) || splits < 1) return AWG_ERR_INVALID_ARG;
    if (K == 16)
        return u.bf16 ? launch_wt2<16, 1>(u, Bt, ldb, part, splits, d_err, s)
                      : launch_wt2<16, 0>(u, Bt, ldb, part, splits, d_err, s);
    if (K == 32)
        return u.bf16 ? launch_wt2<32, 1>(u, Bt, ldb, part, splits, d_err, s)
                      : launch_wt2<32, 0>(u, Bt, ldb, part, splits, d_err, s);
    if (K == 64)
        return u.bf16 ? launch_wt2<64, 1>(u, Bt, ldb, part, splits, d_err, s)
                      : launch_wt2<64, 0>(u, Bt, ldb, part, splits, d_err, s);
    return AWG_ERR_INVALID_ARG;
}

}  // namespace awg
