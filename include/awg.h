/*
 * awg.h — C ABI of libawg, a GB300 (sm_103a) implementation of the AWG
 * (Algebraic-Woodbury-GenEO) preconditioned conjugate gradient method of
 * Gouarin & Spillane, "Fully algebraic domain decomposition preconditioners
 * with adaptive spectral bounds" (arXiv 2106.10913).
 *
 * The solver knows only a sparse SPD matrix A (Section 1, eq. (Ax=b)), a
 * non-overlapping owner of every degree of freedom, an overlap width and the
 * GenEO threshold tau (Thm. 4).  From those it builds, on the device:
 *   - overlapping subdomains Omega^s (Def. 1, Assumption 1),
 *   - the partition of unity D^s (Def. 3),
 *   - the splitting B^s by pair multiplicity (Def. 5, Thm. 1),
 *   - the eigen-split B^s = A^s_+ - A^s_- (Def. 6) and A_+ (Def. 7, Thm. 2),
 *   - the one-level H^NN (Def. 8) through a Cholesky factorisation of
 *     K^s = A^s_+ + sigma V^s_- V^s_-^T (Section 4.4 item 3),
 *   - the GenEO coarse space and H_2 = H^NN_hyb(tau) (Def. 9, Thm. 4), or
 *     H^AS_+,hyb / H^AS_+,ad(tau_flat) with local solvers (R^s A_+ R^sT)^-1
 *     (Def. 8, Thm. 3), or H^AS_hyb(tau, tau_flat) with local solvers
 *     (R^s A R^sT)^-1 (Thm. 5) (awg_options.h2),
 *   - the second coarse space W = A_+^-1 [R^sT V^s_-] by multi-right-hand-
 *     side PCG with H_2 (Section 4.4 items 1-2) and F = W^T A W (Def. 10),
 * and applies H_3,ad (default), H_3,hyb (Def. 10) or H_3,inex (Thm. 7)
 * inside PCG.
 *
 * Conventions shared by every entry point:
 *   - Pointers named d_* are DEVICE pointers, h_* are HOST pointers.
 *   - Dense vectors are float64 arrays of length n; several right-hand sides
 *     are stored column by column with a leading dimension ld >= n.
 *   - A is CSR with int32 row pointers (length n+1, rowptr[0] = 0) and int32
 *     column indices (length nnz, sorted in each row, no duplicates, pattern
 *     structurally symmetric), float64 values.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is ordered on that stream.  awg_setup and awg_pcg*
 *     synchronise the stream before they return; awg_apply* and awg_spmv do
 *     not (their status reports argument and launch errors only).
 *   - Ownership: the caller owns every array it passes and may free it once
 *     the call returns; the handle owns everything it allocates and frees it
 *     in awg_destroy.  A handle must not be used from two host threads or on
 *     two streams at the same time.
 *   - Errors are returned as awg_status; no call aborts the process.  After
 *     AWG_ERR_CUDA the handle should be destroyed.
 */
#ifndef AWG_H
#define AWG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct awg_handle_s* awg_handle;

typedef enum {
    AWG_OK = 0,
    AWG_ERR_INVALID_ARG = 1,   /* bad size, pointer or option */
    AWG_ERR_MIN_OVERLAP = 2,   /* Assumption 1 fails: some A_ij in no Omega^s */
    AWG_ERR_NOT_SPD = 3,       /* a Cholesky pivot <= 0 (A, K^s, M_B^s, E or F) */
    AWG_ERR_EIG = 4,           /* a tridiagonal eigensolve did not converge */
    AWG_ERR_BREAKDOWN = 5,     /* PCG p^T A p <= 0 or not finite */
    AWG_ERR_MAXIT = 6,         /* PCG stopped at the iteration cap */
    AWG_ERR_OOM = 7,           /* device allocation failed */
    AWG_ERR_CUDA = 8,          /* any other CUDA runtime error */
    AWG_ERR_NOT_SYMMETRIC = 9, /* the CSR pattern is not structurally symmetric */
    AWG_ERR_STATE = 10,        /* call not valid for this handle (e.g. no W) */
    AWG_ERR_IO = 11            /* file not written or read, or not a handle file */
} awg_status;

/* Variant of the AWG preconditioner (Def. 10, Thm. 7). */
typedef enum { AWG_H3_AD = 0, AWG_H3_HYB = 1, AWG_H3_INEX = 2 } awg_variant;

/* Two-level preconditioner H_2 for A_+ inside H_3 (Section 3.4):
 * NN_HYB   H^NN_hyb(tau) of Thm. 4: local solvers D^s (A^s_+)^+ D^s, GenEO
 *          space of the pencil (D^s^-1 A^s_+ D^s^-1, R^s A_+ R^sT) below tau;
 * ASP_HYB  H^AS_+,hyb(tau_flat) of Thm. 3: local solvers (R^s A_+ R^sT)^-1
 *          (each the Cholesky inverse of the dense principal block of A_+,
 *          assembled as in Section 4.4 item 4), coarse space of the same
 *          pencil below 1 / tau_flat, combined as Pi H^AS_+ Pi^T + Z E^-1 Z^T;
 * ASP_AD   H^AS_+,ad(tau_flat) of Thm. 3: the same pieces combined additively,
 *          H^AS_+ + Z E^-1 Z^T;
 * AS_HYB   H^AS_hyb(tau, tau_flat) of Thm. 5: local solvers (R^s A R^sT)^-1,
 *          coarse space of two pencils per subdomain, the eigenvectors of
 *          (D^s^-1 A^s_+ D^s^-1, R^s A R^sT) below 1 / tau_flat followed by
 *          those of (R^s A R^sT, R^s A_+ R^sT) below tau (both by the dense
 *          route; awg_options.geneo_solver is not used); a union that is not
 *          linearly independent leaves E singular (AWG_ERR_NOT_SPD).
 * E = Z^T A_+ Z and Pi = I - Z E^-1 Z^T A_+ in every case. */
typedef enum { AWG_H2_NN_HYB = 0, AWG_H2_ASP_HYB = 1, AWG_H2_ASP_AD = 2, AWG_H2_AS_HYB = 3 } awg_h2;

/* Storage/arithmetic of the two largest operators of the apply: the local
 * pseudo-inverses D^s (A^s_+)^+ D^s and the second coarse basis W.  FP64
 * keeps everything in float64.  MIXED_FP32 stores both in float32 with
 * float32 accumulation; MIXED_BF16 stores W in bfloat16 and the local
 * operators in float32 (the explicit local pseudo-inverses carry
 * cond(A^s_+), far beyond 8 mantissa bits on high-contrast problems);
 * MIXED_FP16 stores W as float16 values times power-of-two row and column
 * scales (W = S_r What S_c, every row of What with largest magnitude in
 * [1/2, 1); 11 significant bits, 3 more than bfloat16) plus a sparse
 * float32 correction of its largest entries (awg_options.w16_keep), and the
 * local operators in float32.  All keep the PCG recurrences, both coarse
 * factorisations and solves and the GenEO selection test in float64, and
 * assemble F from the same rounded W (so H_3 stays SPD). */
typedef enum { AWG_FP64 = 0, AWG_MIXED_FP32 = 1, AWG_MIXED_BF16 = 2, AWG_MIXED_FP16 = 3 } awg_precision;

typedef struct {
    int variant;            /* awg_variant, default AWG_H3_AD                  */
    int precisions;         /* bit mask of awg_precision values to build
                               (bit p = 1 << p); FP64 is always built          */
    double zero_rtol;       /* |lambda| <= zero_rtol * max|lambda(B^s)| is a
                               zero eigenvalue (in V^s_-, not in W); 1e-12     */
    double w_rtol;          /* relative residual of the A_+ solves for W;
                               default 1e-13                                   */
    int w_maxit;            /* iteration cap of those solves; default 500      */
    int maxit;              /* iteration cap of awg_pcg; default 1000          */
    int verbose;            /* 1: print setup stage timings to stderr          */
    int w_precision;        /* local operators of H_2 inside the W solve:
                               AWG_MIXED_FP32 (default; the outer PCG, its
                               residuals and A_+ products stay float64, so W
                               still converges to w_rtol) or AWG_FP64          */
    int geneo_solver;       /* eigensolver of the GenEO pencils (Def. 9):
                               0 (default) dense: Cholesky of M_B, Householder
                               tridiagonalisation, bisection, inverse iteration;
                               1 block inverse iteration with Rayleigh-Ritz from
                               a pseudo-random start block, each subdomain
                               accepted only under an inertia certificate
                               (Sylvester's law) that no eigenvalue below tau
                               was missed; pencils it cannot certify within
                               geneo_maxit steps go to the dense solver;
                               2 as 1, start block from the learned network
                               (learned_params)                                 */
    int geneo_block;        /* block width b of solvers 1-2, 2..16; default 8.
                               A subdomain with b or more extra modes (beyond
                               the kernel D^s V^s_-) goes to the dense solver  */
    int geneo_maxit;        /* step cap of solvers 1-2; default 60             */
    const double* learned_params; /* host float64[AWG_LEARNED_NPARAM], read
                               during awg_setup only (solver 2)                */
    int autotune;           /* 1 (default): at the end of setup, time the apply
                               of every built form over a few grid sizes of the
                               two W passes (they run beside the H_2 chain on
                               a second stream) and keep the fastest; 0: fixed
                               defaults                                         */
    double w16_keep;        /* MIXED_FP16: entries with |W_ij| >= w16_keep *
                               max_i |W_ij| also keep a float32 correction of
                               their float16 rounding (a sparse term added in
                               both W passes; the largest ~1 % of W carry most
                               of each column, so this restores nearly the
                               float32 iteration count); 0 disables; 0.1       */
    int block_tensor_cores; /* awg_apply_block / awg_pcg_block with
                               AWG_MIXED_FP16 or AWG_MIXED_BF16: 1 (default)
                               the two passes over W on the tensor cores
                               (tcgen05.mma fed by TMA); 0 on the CUDA cores   */
    int h2;                 /* awg_h2, default AWG_H2_NN_HYB                   */
    double tau_flat;        /* tau_flat > 0 of the AS choices of H_2 (the
                               AS_+ ones select below 1 / tau_flat and leave
                               the tau of awg_setup unused); default 10        */
    int coarse_tensor_cores; /* block path (awg_apply_block, awg_pcg_block*):
                               1 (default) the float64 products with the dense
                               coarse inverses E^-1, F^-1 (Thm. 4, Def. 10) on
                               the tensor cores, both operands cut into eight
                               7-bit integer slices whose bfloat16 products are
                               exact in float32 and summed in float64 (as
                               accurate as a float64 GEMM); 0 on the float64
                               CUDA cores                                      */
    double w_drop_tol;      /* > 0: the float64 form keeps a truncated second
                               coarse basis, the entries of W with |W_ij| >=
                               w_drop_tol * max_i |W_ij| of their column,
                               stored sparse by rows and by columns, and
                               F = W^T A W rebuilt from it (so H_3 stays SPD;
                               the conclusion, Section 6, leaves sparser
                               second coarse spaces open).  The single-RHS
                               applies and PCG of that form use it (H_3,ad,
                               H_3,hyb; not H_3,inex, whose inner matrix of
                               Thm. 7 assumes W = A_+^-1 Vhat: variant
                               AWG_H3_INEX is refused and stage 6 returns
                               AWG_ERR_STATE); its block forms return
                               AWG_ERR_STATE.  The mixed forms keep the full
                               W.  0 (default): full W                      */
} awg_options;

/* Per-handle figures reported after setup (cf. Table 1 of the paper). */
typedef struct {
    int n, nnz, nparts;
    int64_t sum_ns;         /* sum of subdomain sizes n^s                       */
    int max_ns;             /* largest n^s                                      */
    int n0;                 /* GenEO coarse dimension #V_0                      */
    int n_minus;            /* second coarse dimension (strictly negative
                               eigenvalues of all B^s)                          */
    int n_minus_all;        /* columns of all V^s_- (zeros included)            */
    int w_iters;            /* iterations of the multi-RHS PCG that built W     */
    double w_relres;        /* its largest final relative residual              */
    double setup_ms[8];     /* stage times: subdomains, split, local factors,
                               GenEO, E, W, F, total                            */
    size_t device_bytes;    /* device memory held by the handle                 */
    int geneo_its_max;      /* block solver: most steps taken by a subdomain    */
    int64_t geneo_its_sum;  /* block solver: steps summed over subdomains       */
    int geneo_dense;        /* subdomains whose pencil went through the dense
                               eigensolver (all of them with geneo_solver 0)    */
    int wt_blocks[4];       /* per awg_precision form: blocks of the W^T r and  */
    int wd_blocks[4];       /* W d passes (autotuned; 0 if the form is unbuilt) */
    int block_wt_ctas[3];   /* block path, widths 16 / 32 / 64: CTAs per SM of
                               the tensor-core W^T B pass and blocks per SM of  */
    int block_dense_bps[3]; /* the float64 coarse GEMM (autotuned on the first
                               H_3 apply of that width; 0 before)              */
    int64_t w_kept;         /* entries kept in the float64 form's truncated W
                               (awg_options.w_drop_tol > 0), else 0           */
} awg_info;

/* Fill *opt with the defaults above. */
void awg_default_options(awg_options* opt);

/* Human-readable name of a status. */
const char* awg_status_string(awg_status s);

/*
 * Build the AWG preconditioner for A (Sections 2-4 of the paper).
 *   n, nnz          order and stored entries of A (n >= 1)
 *   d_rowptr        device int32[n+1]
 *   d_colidx        device int32[nnz]
 *   d_val           device float64[nnz]
 *   d_partition     device int32[n], owner subdomain of each dof, values in
 *                   [0, nparts); every part non-empty
 *   nparts          number of subdomains N (>= 1)
 *   overlap         layers of graph neighbours added to each part (>= 0);
 *                   Assumption 1 must hold afterwards (overlap >= 1 suffices)
 *   tau             GenEO threshold tau_sharp of Thm. 4 (> 0)
 *   opt             NULL for defaults
 *   out             receives the handle (NULL on error)
 * Errors: AWG_ERR_INVALID_ARG, AWG_ERR_NOT_SYMMETRIC, AWG_ERR_MIN_OVERLAP,
 * AWG_ERR_NOT_SPD, AWG_ERR_EIG, AWG_ERR_OOM, AWG_ERR_CUDA.
 */
awg_status awg_setup(int n, int nnz, const int* d_rowptr, const int* d_colidx,
                     const double* d_val, const int* d_partition, int nparts,
                     int overlap, double tau, const awg_options* opt,
                     void* stream, awg_handle* out);

/* Release everything the handle owns.  NULL is accepted. */
void awg_destroy(awg_handle h);

/* Copy the setup figures into *info (host struct). */
awg_status awg_get_info(awg_handle h, awg_info* info);

/*
 * z = H r for nrhs right-hand sides (columns of length n, leading dimension
 * ld), with H the variant chosen at setup (H_3,ad: Def. 10) and the storage
 * precision `precision` (must have been built).  d_r and d_z are device
 * float64 arrays and must not overlap.
 */
awg_status awg_apply(awg_handle h, int precision, const double* d_r, double* d_z,
                     int nrhs, int ld, void* stream);

/*
 * Apply one building block of the preconditioner (for stage-by-stage
 * checks).  `which`:
 *   0  y = A x                           (CSR SpMV)
 *   1  y = A_+ x = A x + A_- x           (Thm. 2, Section 4.4 item 4)
 *   2  y = H^NN x                        (Def. 8)
 *   3  y = H^NN_hyb(tau) x = H_2 x       (Thm. 4)
 *   4  y = H_3,ad x                      (Def. 10)
 *   5  y = H_3,hyb x                     (Def. 10)
 *   6  y = H_3,inex x                    (Thm. 7)
 * Single right-hand side; d_x, d_y device float64[n].
 */
awg_status awg_apply_stage(awg_handle h, int which, int precision, const double* d_x,
                           double* d_y, void* stream);

/*
 * Solve A x = b by PCG preconditioned with H (x_0 = 0), for nrhs columns
 * (leading dimension ld) at once; each column stops when its recurrence
 * residual satisfies ||b - A x|| <= rtol ||b|| and the true residual is
 * confirmed.  h_iters (int[nrhs]) and h_relres (double[nrhs], true relative
 * residual) are HOST arrays and may be NULL.
 * Errors: AWG_ERR_MAXIT (some column hit opt.maxit), AWG_ERR_BREAKDOWN.
 */
awg_status awg_pcg(awg_handle h, int precision, const double* d_b, double* d_x,
                   int nrhs, int ld, double rtol, int* h_iters, double* h_relres,
                   void* stream);

/*
 * Copy setup results to HOST arrays, for checks.  `what`:
 *   0  subdomain sizes n^s                      int32[nparts]
 *   1  subdomain index lists, concatenated      int32[sum_ns]
 *   2  n^s_- (zeros included)                   int32[nparts]
 *   3  strictly negative counts                 int32[nparts]
 *   4  GenEO mode counts m^s                    int32[nparts]
 *   5  eigenvalues of B^s in V^s_-, concatenated float64[n_minus_all]
 *   6  pair multiplicity M_mu per stored entry  float64[nnz]
 *   7  partition of unity diagonal D            float64[n]
 *   8  E = Z^T A_+ Z                            float64[n0*n0]
 *   9  F = W^T A W                              float64[n_minus^2]
 *  10  W (column-major n x n_minus)             float64[n*n_minus]
 *  11  Z (column-major n x n0)                  float64[n*n0]
 *  12  the blocks of Z: per subdomain s, Y^s    float64[sum_s n^s m^s]
 *      column-major n^s x m^s (rows in the order of Omega^s), one after
 *      the other
 * `count` is the capacity of h_out in elements; AWG_ERR_INVALID_ARG if it
 * is too small.
 */
awg_status awg_get_array(awg_handle h, int what, void* h_out, size_t count);

/*
 * Checkpoint of a set-up handle: awg_save writes to the file `path` what
 * awg_setup computed (A, the subdomains and their incidence lists, D, M_mu,
 * B, the eigen-splits V^s_- and Lambda^s_-, the local operators of every
 * built storage form, the GenEO basis Z with E and E^-1, W in every built
 * form with F^-1 (and the H_3,inex matrix where built), the options and the
 * tuned grid sizes); awg_load makes a new handle from such a file on the
 * current device, ordered on `stream`, without repeating the setup (the
 * setup is the expensive part: eigenproblems and the n_- solves for W).
 * Loaded handles apply and solve exactly as the saved one (the same bytes
 * in every operator); what is built on first use (block-path copies,
 * tensor-core tiles, loop graphs, the block autotuner) is built again then.
 * The file is in the byte order and type sizes of the machine that wrote it
 * (little-endian, LP64) and carries a format tag and version.
 *   awg_save: synchronises the handle's streams; AWG_ERR_INVALID_ARG for a
 *     NULL argument, AWG_ERR_IO if the file cannot be written (a partial
 *     file may be left), AWG_ERR_CUDA on a copy error.
 *   awg_load: *out = NULL on any error; AWG_ERR_INVALID_ARG for a NULL
 *     argument; AWG_ERR_IO if the file cannot be read, has another format
 *     tag, version or options layout, or is truncated (checked before any
 *     device work for the header); AWG_ERR_OOM, AWG_ERR_CUDA.  Free the
 *     handle with awg_destroy.
 */
awg_status awg_save(awg_handle h, const char* path);
awg_status awg_load(const char* path, void* stream, awg_handle* out);

/* Kernel classes timed by awg_profile (index into the arrays it returns). */
enum {
    AWG_PROF_SPMV = 0,       /* CSR SpMV                                  */
    AWG_PROF_LOCAL = 1,      /* batched local pseudo-inverse GEMV         */
    AWG_PROF_WT = 2,         /* W^T r, first pass over W                  */
    AWG_PROF_WD = 3,         /* W d, second pass over W                   */
    AWG_PROF_COARSE = 4,     /* dense E^-1 / F^-1 GEMVs                   */
    AWG_PROF_SUBDOMAIN = 5,  /* block-sparse Z / V^s_- products           */
    AWG_PROF_PROLONG = 6,    /* prolongation gathers                      */
    AWG_PROF_VECTOR = 7,     /* PCG vector updates and dot products       */
    AWG_NPROF = 8
};
/* Further awg_profile mask bits: AWG_PROF_SERIAL runs the apply's side-stream
 * work (the W F^-1 W^T branch of H_3,ad / H_3,inex) in order on the main
 * stream, so that event times are kernel times rather than times shared with
 * concurrent kernels; AWG_PROF_COUNT (alone) counts launches, no events. */
enum { AWG_PROF_SERIAL = 1 << 8, AWG_PROF_COUNT = 1 << 9 };

/*
 * Profiling of the apply / PCG path, for benchmarks.  awg_profile(h, mask)
 * with mask != 0 resets and starts: every kernel the apply and PCG launch
 * is counted, and each launch of a kernel class k with bit (1 << k) set in
 * mask is bracketed by two CUDA events recorded on its own stream (up to a
 * pool of 65536 events); with AWG_PROF_SERIAL in mask the apply's two
 * streams are serialised while profiling (see above).  awg_profile(h, 0)
 * stops.
 * awg_profile_read synchronises the handle's last stream, and writes the
 * launch count to *h_launches and, per kernel class, the summed event time
 * (ms) and the number of timed launches to the HOST arrays h_ms[AWG_NPROF]
 * and h_count[AWG_NPROF] (either may be NULL).
 */
awg_status awg_profile(awg_handle h, int enable);
awg_status awg_profile_read(awg_handle h, int64_t* h_launches, double* h_ms, int64_t* h_count);

/*
 * Trace of the launches timed since awg_profile started (call before
 * awg_profile_read, which clears them): for up to `cap` launches in the
 * order they were issued, the kernel class (h_class, int32), and the start
 * and end (h_t0, h_t1, ms) relative to the first timed launch's start, on
 * the device clock shared by all streams; launches on the side stream
 * overlap those on the main stream where the GPU ran them concurrently.
 * Returns the number of launches written in *h_count.  Synchronises.
 */
awg_status awg_profile_trace(awg_handle h, int cap, int* h_class, double* h_t0, double* h_t1,
                             int* h_count);

/*
 * Multi-right-hand-side ("block") forms of awg_apply_stage and awg_pcg: the
 * nrhs columns are processed together, so every pass over an operator (the
 * local pseudo-inverses, W, Z, V^s_-, E^-1, F^-1, A) serves all of them; the
 * GEMV-shaped steps of the single-RHS path become GEMMs.  Each column keeps
 * its own PCG recurrence (Section 1: alpha, beta and the stopping test per
 * column), so column c of a block solve follows the single-RHS solve of
 * column c.  `precision`: AWG_FP64 computes every step in float64; the
 * mixed forms keep the preconditioner's internal vectors and arithmetic in
 * float32 (with their stored W: float32 on the CUDA cores, float16 or
 * bfloat16 on the tensor cores, see awg_options.block_tensor_cores) and the
 * coarse solves E^-1, F^-1 and all PCG recurrences in float64.
 *   d_x, d_y / d_b, d_x   device float64, nrhs columns of length n with
 *                         leading dimension ld >= n (column-major)
 * awg_apply_block: which = 0 (A), 1 (A_+), 2 (H^NN), 3 (H_2), 4 (H_3,ad),
 * 5 (H_3,hyb), 6 (H_3,inex: AWG_ERR_STATE unless its matrix was built, as
 * for awg_apply_stage); 1 <= nrhs <= 64; asynchronous on `stream`
 * (allocates its workspace on the handle's first block call).
 * awg_pcg_block: the handle's variant (H_3,ad, H_3,hyb or H_3,inex), any
 * nrhs >= 1 (groups of up to 64 columns), x_0 = 0; synchronises `stream`;
 * h_iters / h_relres as awg_pcg.  Errors: AWG_ERR_INVALID_ARG,
 * AWG_ERR_STATE, AWG_ERR_MAXIT, AWG_ERR_BREAKDOWN, AWG_ERR_OOM,
 * AWG_ERR_CUDA (also when a tensor-core pass reports a timed-out wait).
 */
awg_status awg_apply_block(awg_handle h, int which, int precision, const double* d_x, double* d_y, int nrhs,
                           int ld, void* stream);
awg_status awg_pcg_block(awg_handle h, int precision, const double* d_b, double* d_x, int nrhs, int ld,
                         double rtol, int* h_iters, double* h_relres, void* stream);

/*
 * Y = M X with one of the handle's dense coarse inverses, through the block
 * path's coarse product (for checks of that product): which = 0 E^-1 of the
 * GenEO coarse problem E = Z^T A_+ Z (Thm. 4), 1 F^-1 of the second coarse
 * problem F = W^T A W of the storage form `precision` (Def. 10), 2 the
 * H_3,inex inner inverse (C^-1 - Vhat^T W)^-1 of that form (Thm. 7).
 *   engine   0: float64 GEMM on the CUDA cores; 1: the tensor-core slice
 *            products of awg_options.coarse_tensor_cores (AWG_ERR_STATE if
 *            they are not built); 2: as 1 with the reduction split every
 *            256 terms (the split that dimensions above 4032 take)
 *   d_x, d_y device float64, nrhs (1..64) columns of length dim (n0 or n_-),
 *            column-major with ld = dim, must not overlap
 * Synchronises `stream`.  Errors: AWG_ERR_INVALID_ARG, AWG_ERR_STATE (matrix
 * not built), AWG_ERR_OOM, AWG_ERR_CUDA.
 */
awg_status awg_coarse_apply_block(awg_handle h, int which, int precision, int engine, const double* d_x,
                                  double* d_y, int nrhs, void* stream);

/*
 * Asynchronous block PCG (the handle's variant, 1 <= nrhs <= 128 columns,
 * x_0 = 0): the
 * iterations run as one CUDA graph launch, a conditional while node whose
 * body is one iteration captured from the handle's two streams, with the
 * stopping test (per column, recurrence residual <= rtol ||b||, Section 1)
 * evaluated on the device: a column whose recurrence residual reaches rtol
 * ||b|| is confirmed on its true residual b - A x (computed in that
 * iteration only) and goes on iterating while the true residual exceeds
 * rtol ||b||, as in awg_pcg.  No host synchronisation: the call returns once
 * the work is enqueued on `stream`, so one host thread can keep several
 * handles (independent problems) solving at the same time.  The loop graph
 * of each (precision, nrhs width 16/32/64) is captured on first use (make
 * that first call outside any stream capture).  DEVICE outputs, written
 * when the work completes: d_iters int32[nrhs] (iterations per column),
 * d_relres float64[nrhs] (relative residual at exit: the true one for a
 * column that stopped converged, the recurrence one after a breakdown or at
 * the iteration cap), d_status int32[1] (AWG_OK, AWG_ERR_BREAKDOWN or
 * AWG_ERR_MAXIT, the latter also for a column whose recurrence residual
 * fell below 1e-6 rtol without the true one reaching rtol); any may be NULL.
 * With nrhs = 1 the loop body is the single-right-hand-side apply (the
 * GEMV-shaped passes of awg_pcg), otherwise the block apply of
 * awg_pcg_block; more than 64 columns run as two groups (64 and the rest)
 * side by side on the handle's two block slots (own workspace, stream pair
 * and loop graphs), so one group's float64 coarse GEMMs overlap the other's
 * bandwidth-bound passes.
 * Errors returned: AWG_ERR_INVALID_ARG, AWG_ERR_STATE, AWG_ERR_OOM,
 * AWG_ERR_CUDA.
 */
awg_status awg_pcg_block_async(awg_handle h, int precision, const double* d_b, double* d_x, int nrhs, int ld,
                               double rtol, int* d_iters, double* d_relres, int* d_status, void* stream);

/* Capacity, in float64 values, of the static scratch of awg_apply_hnn_noalloc. */
#define AWG_NOALLOC_MAX_LOCAL (1 << 20)

/*
 * y = H^NN x (the batched local pseudo-inverses and the prolongation sum,
 * as awg_apply_stage with which = 2) WITHOUT ANY DEVICE ALLOCATION.  The
 * paper has no counterpart: this entry point serves callers that may not
 * call cudaMalloc while they apply the preconditioner: frameworks that hand
 * out all device memory from their own pool and forbid libraries to
 * allocate, and real-time loops that cannot afford cudaMalloc / cudaFree
 * (which may synchronise the device).  Its scratch (sum of n^s float64 values) is a static
 * device array of AWG_NOALLOC_MAX_LOCAL doubles (8 MiB) that every GPU
 * loading the library keeps until the process exits; a handle whose
 * subdomains hold more values is rejected with AWG_ERR_INVALID_ARG (and a
 * message on stderr).
 *   h          a handle built by awg_setup on the current device
 *   precision  AWG_FP64 or AWG_MIXED_FP32 (the latter must have been built)
 *   d_x, d_y   device float64[n], caller-owned, must not overlap
 * The first call on a device looks up the scratch's device address (no
 * allocation) and caches it: make that first call before any stream
 * capture.  Every call shares the scratch and finds the previous call's
 * values there (each value read is written earlier in the same call, so
 * nothing needs clearing); calls that overlap on the GPU (two streams or
 * two host threads at once) race on it and must be serialised by the
 * caller.  Asynchronous on `stream`; errors: AWG_ERR_INVALID_ARG,
 * AWG_ERR_STATE, AWG_ERR_CUDA.
 */
awg_status awg_apply_hnn_noalloc(awg_handle h, int precision, const double* d_x, double* d_y,
                                 void* stream);

/* ------------------------------------------------------------------------
 * Learned start block of the GenEO block solver.  The paper has no
 * counterpart: it names iterative eigensolvers for the GenEO pencils
 * (remark after Def. 9) without fixing their start.  A 5-16-16-1 network
 * (tanh, tanh, sigmoid) maps per-node features of a subdomain, computed
 * from A, to the predicted normalised leverage of the subdomain's extra
 * modes (GenEO eigenvectors with eigenvalue in (0, tau)).  Parameters are
 * float64[AWG_LEARNED_NPARAM]: W1[16x5] row-major, b1[16], W2[16x16]
 * row-major, b2[16], w3[16], b3.  Features are float64[P x 5], row-major:
 *   f0 = (log10 A_pp - mean over the subdomain of log10 A_qq) / 6
 *   f1 = (multiplicity of p - 1) / 3
 *   f2 = mean of f0 over the neighbours of p inside the subdomain (0 if none)
 *   f3 = largest f0 over those neighbours (f0_p if none)
 *   f4 = (sum of the stored row of A) / A_pp
 * The functions below are asynchronous on `stream` except awg_learned_train,
 * which returns after the last step.
 */
#define AWG_LEARNED_NPARAM 385
#define AWG_LEARNED_NFEAT 5

/* Features (d_features, device float64[sum_ns x 5], row k = k-th entry of
 * the concatenated subdomain index lists) and training targets (d_targets,
 * device float64[sum_ns]: per subdomain, the diagonal of the orthogonal
 * projector onto the span of its extra modes, divided by its maximum; zero
 * where a subdomain has none; at most 16 extra modes enter) of a built
 * handle.  Either pointer may be NULL.  Errors: AWG_ERR_INVALID_ARG,
 * AWG_ERR_CUDA. */
awg_status awg_learned_data(awg_handle h, double* d_features, double* d_targets, void* stream);

/* d_out[p] = network(d_features row p), p < P, in float64 (precision
 * AWG_FP64) or float32 (AWG_MIXED_FP32) arithmetic.  d_params is device
 * float64[AWG_LEARNED_NPARAM].  Errors: AWG_ERR_INVALID_ARG, AWG_ERR_CUDA. */
awg_status awg_learned_forward(int P, const double* d_features, const double* d_params, double* d_out,
                               int precision, void* stream);

/* Gradient of the mean squared error L = (1/P) sum_p (out_p - t_p)^2 with
 * respect to the parameters: d_grad (device float64[AWG_LEARNED_NPARAM + 1])
 * receives the gradient, then L.  Sums are taken in a fixed order (the
 * result does not depend on scheduling).  Allocates scratch on `stream`.
 * Errors: AWG_ERR_INVALID_ARG, AWG_ERR_OOM, AWG_ERR_CUDA. */
awg_status awg_learned_grad(int P, const double* d_features, const double* d_targets,
                            const double* d_params, double* d_grad, int precision, void* stream);

/* `steps` full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, step
 * size lr) on L, all on the device.  h_params (host float64[NPARAM]) holds
 * the start on entry and the result on return; h_loss (host float64[steps]
 * or NULL) receives L before each step.  Synchronous.  Errors:
 * AWG_ERR_INVALID_ARG, AWG_ERR_OOM, AWG_ERR_CUDA. */
awg_status awg_learned_train(int P, const double* d_features, const double* d_targets, double* h_params,
                             int steps, double lr, int precision, double* h_loss, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* AWG_H */
