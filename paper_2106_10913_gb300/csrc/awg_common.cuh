// Shared declarations of libawg's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/awg.h"

namespace awg {

#define AWG_CUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t err__ = (call);                                                       \
        if (err__ != cudaSuccess) {                                                       \
            if (err__ == cudaErrorMemoryAllocation) {                                     \
                cudaGetLastError();                                                       \
                return AWG_ERR_OOM;                                                       \
            }                                                                             \
            fprintf(stderr, "libawg: %s failed at %s:%d: %s\n", #call, __FILE__, __LINE__, \
                    cudaGetErrorString(err__));                                           \
            return AWG_ERR_CUDA;                                                          \
        }                                                                                 \
    } while (0)

#define AWG_TRY(expr)                         \
    do {                                      \
        awg_status st__ = (expr);             \
        if (st__ != AWG_OK) return st__;      \
    } while (0)

#define AWG_LAUNCH() AWG_CUDA(cudaGetLastError())

// Bits of the device status word that kernels raise.
enum : int {
    FLAG_MIN_OVERLAP = 1,
    FLAG_NOT_SPD = 2,
    FLAG_EIG = 4,
    FLAG_NOT_SYM = 8,
    FLAG_BAD_CSR = 16,
};

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Storage of the apply for one precision (awg_precision).
struct PrecOps {
    bool built = false;
    DevBuf G;         // local D^s (A^s_+)^+ D^s: float64 full n^s x n^s, or packed tiles
    DevBuf W;         // second coarse basis, row-major n x ldw (float64/float32/bf16)
    DevBuf Finv;      // (W^T A W)^-1 for this W, float64 n_- x n_-
    DevBuf inexInv;   // (C^-1 - Vhat^T W)^-1 (H_3,inex), float64 n_- x n_-
    DevBuf rscale;    // float16 W: power-of-two row scales, float32[n]
    DevBuf cscale;    // float16 W: power-of-two column scales, float32[ldw] (0 on padding)
    // float16 W: sparse float32 correction of the largest entries (|W_ij| >=
    // w16_keep * max_i |W_ij|), in the scaled units of What: the exact value
    // minus its float16 rounding.  Rows (CSR, for W d) and columns (CSC, for
    // W^T r), indices ascending.
    int64_t corr_nnz = 0;
    DevBuf corr_rowptr, corr_col, corr_val;   // int32[n+1], int32[nnz], float32[nnz]
    DevBuf corr_colptr, corr_row, corr_cval;  // int32[n_-+1], int32[nnz], float32[nnz]
    // truncated W of the float64 form (awg_options.w_drop_tol > 0): the
    // entries with |W_ij| >= w_drop_tol * max_i |W_ij|, float64, by rows (CSR,
    // for W d) and by columns (CSC, for W^T r), indices ascending; W stays
    // empty then
    int64_t sp_nnz = 0;
    DevBuf sp_rowptr, sp_col, sp_val;     // int64[n+1], int32[nnz], float64[nnz]
    DevBuf sp_colptr, sp_row, sp_cval;    // int64[n_-+1], int32[nnz], float64[nnz]
    // grid sizes of the W^T r and W d passes (0: defaults), set by the
    // autotuner at the end of setup
    int wt_blocks = 0, wd_blocks = 0;
};
constexpr int AWG_NPREC = 4;

struct Handle {
    int n = 0, nnz = 0, N = 0, overlap = 0;
    double tau = 0.1;
    awg_options opt{};
    cudaStream_t stream = nullptr;

    DevBuf rowptr, colidx, val;          // A

    // subdomains Omega^s (Def. 1), sizes n^s
    std::vector<int> h_ns, h_sub_ptr;
    int64_t sum_ns = 0;
    int max_ns = 0;
    DevBuf ns, sub_ptr, sub_idx;         // int32[N], int32[N+1], int32[sum_ns]
    DevBuf inc_ptr, inc_pos, inc_sub;    // per dof i: positions (in the local arena)
                                         // of its copies and their subdomain,
                                         // ordered by subdomain
    DevBuf pos_sub;                      // subdomain of each local-arena position
    DevBuf dvec;                         // D (Def. 3): 1/multiplicity, float64[n]
    DevBuf mmu, bval;                    // M_mu and B = A/M_mu per stored entry

    // per-subdomain dense n^s x n^s blocks, column-major, ld = n^s
    std::vector<int64_t> h_dense_off;
    DevBuf dense_off;                    // int64[N+1]
    int64_t dense_total = 0;
    // float32 local operators: ld = n^s rounded up to 4 (16-byte columns)
    std::vector<int64_t> h_g32_off;
    DevBuf g32_off;                      // int64[N+1]

    // eigen-split of B^s (Def. 6)
    std::vector<int> h_nm, h_nstrict, h_nm_ptr;
    std::vector<int64_t> h_vm_off;
    DevBuf nm, nstrict, nm_ptr, vm_off;  // int32[N], int32[N], int32[N+1], int64[N+1]
    DevBuf Vm, lam_m;                    // V^s_- (n^s x n^s_-), eigenvalues
    DevBuf sigma;                        // shift of K^s per subdomain
    int n_minus_all = 0;

    // GenEO coarse space (Def. 9, Thm. 4)
    std::vector<int> h_modes, h_mode_ptr;
    std::vector<int64_t> h_z_off;
    DevBuf modes, mode_ptr, z_off, Z;    // Z^s column-major n^s x m^s (M_B-normalised)
    int n0 = 0;
    DevBuf E, Einv;                      // n0 x n0, float64

    // second coarse space (Def. 10)
    int n_minus = 0, ldw = 0;
    std::vector<int> h_wcol_ptr;         // prefix of the strict counts (N+1)
    DevBuf wcol_ptr;
    DevBuf Wcm;                          // W float64 column-major n x n_- (kept for checks)
    DevBuf F64;                          // W^T A W of the float64 W
    PrecOps prec[AWG_NPREC];

    // GenEO block solver (awg_options.geneo_solver): network parameters of
    // the learned start and per-setup iteration figures
    std::vector<double> h_learned;
    int geneo_its_max = 0;
    int64_t geneo_its_sum = 0;
    int geneo_dense = 0;

    // info
    int w_iters = 0;
    double w_relres = 0.0;
    double setup_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    size_t device_bytes = 0;

    // single right-hand-side workspace of the apply
    DevBuf ws;
    // multi-right-hand-side (block) path: workspace and float32 copies of
    // A's values, V^s_-, |Lambda^s_-| and Z (built on the first block call),
    // |Lambda^s_-| in float64
    DevBuf bws, bval32, bvm32, blam32, blam64, bz32;
    // tensor-core local solves of the block path: 16 KB images of the
    // float32 local pseudo-inverses and their tables (ul_ntiles = 0: not built)
    DevBuf ul_gt, ul_gtoff, ul_kcpre, ul_tsub, ul_trt;
    int ul_ntiles = 0, ul_maxkc = 0, ul_maxtiles = 0;
    // float64-accurate tensor-core coarse products of the block path:
    // bfloat16 slices and row exponents of the dense coarse inverses (slot 0
    // E^-1, 1 + p F^-1 of storage form p, 5 + p the H_3,inex inner inverse
    // of form p), built on the first block call; oz_dim[k] = 0: not built
    DevBuf oz_q[9], oz_ex[9];
    int oz_dim[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    // graph-driven block PCG: loop graph per (precision, K in 16/32/64)
    cudaGraph_t bg_graph[12] = {};
    cudaGraphExec_t bg_exec[12] = {};
    // a second block slot (workspace, stream pair, events, loop graphs): the
    // two column groups of a wide graph-driven solve run side by side, so
    // one group's float64 coarse GEMMs overlap the other's bandwidth-bound
    // passes
    DevBuf bws2;
    // block-path tunables per width (16, 32, 64), set by the block
    // autotuner on the first H_3 apply of that width: CTAs per SM of the
    // tensor-core W^T B pass (split-K) and blocks per SM of the float64
    // coarse GEMM (split-j); 0 = not tuned yet (defaults 2 and 4)
    int bt_wt[3] = {0, 0, 0};
    int bt_dense[3] = {0, 0, 0};
    cudaStream_t hp2 = nullptr, side2 = nullptr;
    cudaEvent_t ev2_fork = nullptr, ev2_mid = nullptr, ev2_join = nullptr, ev2_in = nullptr, ev2_out = nullptr;
    cudaGraph_t bg2_graph[12] = {};
    cudaGraphExec_t bg2_exec[12] = {};
    // graph-driven single-RHS PCG: loop graph per precision, its vectors
    // (b, x, r, p, q, z) and the graph-loop kernel counter
    cudaGraph_t g1_graph[4] = {};
    cudaGraphExec_t g1_exec[4] = {};
    DevBuf g1buf, g1cnt;
    DevBuf flag;                         // int status word
    int red_blocks = 0;
    int* h_flag = nullptr;               // pinned host mirror
    double* h_scal = nullptr;            // pinned host scalars
    // the second-coarse-space pass W^T r runs on `side`, concurrently with
    // H_2 on the caller's stream (fork and join through the two events)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // block path: recorded after the first E^-1 of H_2 on the main stream;
    // the side stream's F^-1 waits for it, so the two float64 GEMMs do not
    // share the FP64 pipes
    cudaEvent_t ev_mid = nullptr;
    // awg_pcg and awg_apply run on `hp`, created with the highest stream
    // priority (`side` has the lowest): blocks of the H_2 chain, the critical
    // path, are dispatched ahead of the bandwidth-bound W^T r pass, which
    // fills the SMs they leave free.  Fork and join with the caller's stream
    // through ev_in / ev_out.
    cudaStream_t hp = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;

    // profiling (awg_profile): launch count of the apply/PCG path and CUDA
    // event times of its heaviest kernels
    int prof = 0;
    int64_t launches = 0;
    double prof_ms[AWG_NPROF] = {0};
    int64_t prof_cnt[AWG_NPROF] = {0};
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_kernel;          // kernel id of each recorded pair
    size_t ev_used = 0;
};

// Brackets one launch with CUDA events on its stream when profiling is on.
// NVTX range of a host-side phase (setup stages, entry points), for
// profilers that filter by range; next() closes the current range and opens
// the following one, the destructor closes the last (also on early return).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    void next(const char* name) {
        nvtxRangePop();
        nvtxRangePushA(name);
    }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// The stream of an apply's side branch: `side`, or the main stream `s`
// while a serialising profile (AWG_PROF_SERIAL) runs
inline cudaStream_t side_stream(const Handle* h, cudaStream_t side, cudaStream_t s) {
    return (h->prof & AWG_PROF_SERIAL) ? s : side;
}

struct ProfScope {
    Handle* h;
    int id;
    cudaStream_t s;
    bool on;
    ProfScope(Handle* hh, int kid, cudaStream_t ss) : h(hh), id(kid), s(ss), on(false) {
        h->launches += (h->prof != 0);
        if ((h->prof >> id) & 1 && h->ev_used + 2 <= h->ev_pool.size()) {
            cudaEventRecord(h->ev_pool[h->ev_used], s);
            on = true;
        }
    }
    ~ProfScope() {
        if (on) {
            cudaEventRecord(h->ev_pool[h->ev_used + 1], s);
            h->ev_kernel.push_back(id);
            h->ev_used += 2;
        }
    }
};

// Kernels launched inside one ProfScope beyond its first (launch count).
inline void extra_launches(Handle* h, int k) { h->launches += (h->prof != 0) * k; }

awg_status dalloc(Handle* h, DevBuf& b, size_t bytes);
void dfree(Handle* h, DevBuf& b);
awg_status read_flag(Handle* h, int* out);
// api.cu: streams, events, pinned words and the flag of a new handle; release
// of everything a handle holds
awg_status runtime_init(Handle* h);
void free_all(Handle* h);
awg_status upload(Handle* h, DevBuf& b, const void* src, size_t bytes);

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum in a fixed order (deterministic).  `sh` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0) t = warp_sum(t);
    if (threadIdx.x == 0) sh[0] = t;
    __syncthreads();
    double r = sh[0];
    __syncthreads();
    return r;
}

// First position of `key` in the sorted int array a[0..len), or -1.
__device__ __forceinline__ int bsearch_idx(const int* a, int len, int key) {
    int lo = 0, hi = len - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int v = a[mid];
        if (v == key) return mid;
        if (v < key) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// ------------------------------------------------------------------ cross-unit API
// structure.cu
awg_status setup_structure(Handle* h, const int* d_part);
awg_status assemble_local(Handle* h, const double* d_vals, double* arena);

// dense.cu : batched dense FP64 kernels over the per-subdomain blocks
struct GemmDesc {
    const double* A;
    const double* B;
    double* C;
    int M, N, K, lda, ldb, ldc;
    int transA, transB;
    double alpha, beta;
};
awg_status gemm_batched(Handle* h, const std::vector<GemmDesc>& descs, cudaStream_t s);
struct GemmDescF {
    const float* A;
    const double* B;
    double* C;
    int M, N, K, lda, ldb, ldc;
    int transA;
    double alpha, beta;
};
awg_status gemm_batched_f32(Handle* h, const std::vector<GemmDescF>& descs, cudaStream_t s);
// Lower Cholesky factor in place of every block; a non-positive pivot raises
// FLAG_NOT_SPD in *d_flag (if given) and sets d_status[block] = 1 (if given).
awg_status potrf_batched(Handle* h, double* arena, const int* d_m, const int64_t* d_off, int nb,
                         int max_m, int* d_flag, cudaStream_t s, int* d_status = nullptr);
awg_status trtri_batched(Handle* h, double* arena, const int* d_m, const int64_t* d_off, int nb,
                         int max_m, cudaStream_t s);
// Selected eigenpairs of symmetric blocks (destroys the blocks).  mode 0: all
// eigenvalues <= zero_rtol * max|lambda| (counts strictly negative ones too);
// mode 1: all eigenvalues < tau.  Returns host counts and device arenas of the
// eigenvectors (column-major n^s x count) and eigenvalues.
awg_status eig_select_batched(Handle* h, double* arena, const int* d_m, const int64_t* d_off,
                              const std::vector<int>& h_m, int nb, int max_m, int mode,
                              double param, std::vector<int>& h_count,
                              std::vector<int>& h_strict, DevBuf& vecs,
                              std::vector<int64_t>& h_vec_off, DevBuf& vals,
                              std::vector<int>& h_val_ptr, cudaStream_t s);

// coarse.cu : blocked float64 Cholesky (lower factor in place; the strict
// upper blocks keep their input) and inverse of its triangular factor
awg_status chol_blocked(Handle* h, double* A, int dim, int* d_flag, cudaStream_t s);
awg_status trtri_blocked(Handle* h, const double* L, double* Li, int dim, cudaStream_t s);

// apply.cu
awg_status apply_stage(Handle* h, int which, int prec, const double* x, double* y, cudaStream_t s);
// times the apply of every built form over a few grid sizes of the two W
// passes (which share the GPU with the H_2 chain) and keeps the fastest
awg_status autotune_apply(Handle* h);
awg_status build_setup_numeric(Handle* h);
// PCG of one right-hand side as one CUDA graph launch (device-side loop)
awg_status pcg1_async(Handle* h, int prec, int stage, const double* b, double* x, double rtol, int* d_it,
                      double* d_rel, int* d_st, cudaStream_t s);
int64_t pcg1_graph_launches(Handle* h);

// learned.cu : features, network and start block of the GenEO block solver
constexpr int LEARNED_NF = 5;
constexpr int LEARNED_NPARAM = 385;
awg_status learned_features(Handle* h, double* d_F, cudaStream_t s);
awg_status learned_forward(int P, const double* d_F, const double* d_params, double* d_out, int prec,
                           cudaStream_t s);
// gradient (LEARNED_NPARAM values) then the loss into d_g; d_part holds
// nblocks x (LEARNED_NPARAM + 1) partial sums
awg_status learned_grad(int P, const double* d_F, const double* d_t, const double* d_params,
                        double* d_g, double* d_part, int nblocks, int prec, cudaStream_t s);
awg_status learned_adam(int t, double lr, const double* d_g, double* d_th, double* d_m, double* d_v,
                        cudaStream_t s);
awg_status learned_targets(Handle* h, double* d_t, cudaStream_t s);
awg_status learned_start_block(Handle* h, const int64_t* d_xoff, int b, const double* d_g, double* d_X0,
                               cudaStream_t s);

// geneo_iter.cu : certified block eigensolver of the GenEO pencils
struct GeneoIter {
    int b = 0;
    std::vector<int> ecount;   // extra modes per subdomain, -1: not certified
    std::vector<int> its;      // iterations per subdomain
    std::vector<int64_t> hx;   // offsets of the m x b blocks
    DevBuf xoff, X, BX, Kq, MBKq;
};
awg_status geneo_block_solve(Handle* h, const double* MA, const double* MB, const double* d_params,
                             int b, int maxit, double tol, GeneoIter& r);
// writes [Kq_s | X_s(:, 0..e_s)] of every certified subdomain at Z + zoff[s]
awg_status geneo_block_pack(Handle* h, GeneoIter& r, const int64_t* d_zoff, double* Z);
void geneo_block_free(Handle* h, GeneoIter& r);

}  // namespace awg
