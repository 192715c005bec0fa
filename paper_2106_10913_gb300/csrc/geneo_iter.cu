// Block eigensolver for the GenEO pencils (Def. 9, Thm. 4), judged by an
// inertia certificate.
//
// Per subdomain the pencil is (M_A, M_B) = (D^-1 A^s_+ D^-1, R^s A_+ R^sT);
// its kernel K = D^s V^s_- is known exactly (Remark after Thm. 5) and is
// always selected.  The remaining modes with eigenvalue below tau are found
// by block inverse iteration with Rayleigh-Ritz in the M_B-orthogonal
// complement of K, with T = D (A^s_+)^+ D (the local operator of H^NN, a
// generalised inverse of M_A) as the inverse:
//     Y = (I - K (K^T M_B K)^-1 K^T M_B) T M_B X,   Rayleigh-Ritz on span(Y).
// A subdomain is finished when every Ritz pair below tau has a norm-wise
// backward error ||M_A x - th M_B x|| / ((|M_A|_F + |th| |M_B|_F) |x|) <=
// tol and the certificate holds: M_A - mu M_B + sigma (M_B U)(M_B U)^T with
// U = [M_B-orthonormal K, those Ritz vectors], mu = tau (1 - 1e-6),
// sigma = 2, has a Cholesky factor.  By Sylvester's law of inertia that is
// the case exactly when no eigenvalue below mu is missing from U.
// Subdomains that do not finish within maxit are reported so that the
// caller falls back to the exact eigensolve.
//
// All m x m x b products use the symmetry of M_A, M_B and T: row p is read
// as column p, contiguous (one warp per row, the b columns of the right-hand
// block in shared memory).

#include "awg_common.cuh"

#include <algorithm>
#include <cmath>

namespace awg {

constexpr int GI_MAXB = 16;
constexpr int GI_ROWS = 32;

// C_s = alpha A_s B_s + beta C_s, A_s symmetric m x m (arena off), B_s and
// C_s m x b column-major (arena xoff); only subdomains with act[s] != 0.
__global__ void __launch_bounds__(256) k_symm_skinny(const int* __restrict__ ns,
                                                     const int64_t* __restrict__ off,
                                                     const double* __restrict__ A,
                                                     const int64_t* __restrict__ xoff,
                                                     const double* __restrict__ B, double* C, int b,
                                                     double alpha, double beta,
                                                     const int* __restrict__ act) {
    extern __shared__ double Bs[];
    const int s = blockIdx.x;
    if (!act[s]) return;
    const int m = ns[s];
    const int r0 = blockIdx.y * GI_ROWS;
    if (r0 >= m) return;
    const double* Bg = B + xoff[s];
    for (int e = threadIdx.x; e < m * b; e += blockDim.x) Bs[e] = Bg[e];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double* As = A + off[s];
    double* Cg = C + xoff[s];
    const int r1 = min(m, r0 + GI_ROWS);
    for (int p = r0 + wid; p < r1; p += nw) {
        const double* col = As + (size_t)p * m;
        double acc[GI_MAXB];
#pragma unroll
        for (int j = 0; j < GI_MAXB; j++) acc[j] = 0.0;
        for (int q = lane; q < m; q += 32) {
            const double a = col[q];
#pragma unroll
            for (int j = 0; j < GI_MAXB; j++)
                if (j < b) acc[j] = fma(a, Bs[q + j * m], acc[j]);
        }
#pragma unroll
        for (int j = 0; j < GI_MAXB; j++) {
            if (j >= b) break;
            const double v = warp_sum(acc[j]);
            if (lane == 0) {
                double* c = Cg + p + (size_t)j * m;
                *c = (beta == 0.0) ? alpha * v : fma(beta, *c, alpha * v);
            }
        }
    }
}

// G_s (b1 x b2) = X_s^T Y_s over the m rows (X_s m x b1 at xo, Y_s m x b2 at yo)
__global__ void k_gram(const int* __restrict__ ns, const int64_t* __restrict__ xo, const double* X,
                       int b1, const int64_t* __restrict__ yo, const double* Y, int b2, double* G,
                       const int* __restrict__ act) {
    __shared__ double red[32];
    const int s = blockIdx.x;
    if (!act[s]) return;
    const int m = ns[s];
    const double* Xs = X + xo[s];
    const double* Ys = Y + yo[s];
    for (int i = 0; i < b1; i++)
        for (int j = 0; j < b2; j++) {
            double part = 0.0;
            for (int p = threadIdx.x; p < m; p += blockDim.x) part = fma(Xs[p + (size_t)i * m], Ys[p + (size_t)j * m], part);
            const double v = block_sum(part, red);
            if (threadIdx.x == 0) G[(size_t)s * GI_MAXB * GI_MAXB + i + j * b1] = v;
        }
}

// Y_s (m x b2) = X_s (m x b1) S_s (b1 x b2, from k_small_geig's layout)
__global__ void k_small_mul(const int* __restrict__ ns, const int64_t* __restrict__ xoff,
                            const double* X, int b1, const double* S, int b2, double* Y,
                            const int* __restrict__ act) {
    const int s = blockIdx.x;
    if (!act[s]) return;
    const int m = ns[s];
    const double* Xs = X + xoff[s];
    const double* Ss = S + (size_t)s * GI_MAXB * GI_MAXB;
    double* Ys = Y + xoff[s];
    for (int e = threadIdx.x; e < m * b2; e += blockDim.x) {
        const int p = e % m, j = e / m;
        double acc = 0.0;
        for (int k = 0; k < b1; k++) acc = fma(Xs[p + (size_t)k * m], Ss[k + j * b1], acc);
        Ys[e] = acc;
    }
}

// Generalised symmetric-definite b x b eigenproblem At c = theta Bt c per
// subdomain (one thread).  The columns of the block are first scaled to unit
// M_B-norm (S = diag(Bt)^-1/2: inverse iteration scales them by the inverse
// eigenvalues, which can span many decades), then Cholesky of S Bt S,
// cyclic Jacobi on L^-1 S At S L^-T, eigenvalues ascending,
// C = S L^-T V (Bt-orthonormal columns).
__global__ void k_small_geig(int N, int b, const double* __restrict__ At, const double* __restrict__ Bt,
                             double* theta, double* C, int* bad, const int* __restrict__ act) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N || !act[s]) return;
    double L[GI_MAXB][GI_MAXB], M[GI_MAXB][GI_MAXB], V[GI_MAXB][GI_MAXB];
    const double* a = At + (size_t)s * GI_MAXB * GI_MAXB;
    const double* bb = Bt + (size_t)s * GI_MAXB * GI_MAXB;
    int fail = 0;
    double sc[GI_MAXB];
    for (int j = 0; j < b; j++) {
        const double d = bb[j + j * b];
        if (!(d > 0.0)) fail = 1;
        sc[j] = (d > 0.0) ? 1.0 / sqrt(d) : 1.0;
    }
    for (int j = 0; j < b; j++) {
        for (int i = 0; i < b; i++) L[i][j] = 0.0;
        double d = bb[j + j * b] * sc[j] * sc[j];
        for (int k = 0; k < j; k++) d -= L[j][k] * L[j][k];
        if (!(d > 0.0)) { fail = 1; d = 1e-300; }
        d = sqrt(d);
        L[j][j] = d;
        for (int i = j + 1; i < b; i++) {
            double v = 0.5 * (bb[i + j * b] + bb[j + i * b]) * sc[i] * sc[j];
            for (int k = 0; k < j; k++) v -= L[i][k] * L[j][k];
            L[i][j] = v / d;
        }
    }
    // M = L^-1 At L^-T: first solve L Y = At (columns), then L M^T = Y^T
    double Y[GI_MAXB][GI_MAXB];
    for (int c = 0; c < b; c++)
        for (int i = 0; i < b; i++) {
            double v = 0.5 * (a[i + c * b] + a[c + i * b]) * sc[i] * sc[c];
            for (int k = 0; k < i; k++) v -= L[i][k] * Y[k][c];
            Y[i][c] = v / L[i][i];
        }
    for (int r = 0; r < b; r++)
        for (int i = 0; i < b; i++) {
            double v = Y[r][i];
            for (int k = 0; k < i; k++) v -= L[i][k] * M[r][k];
            M[r][i] = v / L[i][i];
        }
    for (int i = 0; i < b; i++)
        for (int j = 0; j < b; j++) {
            const double v = 0.5 * (M[i][j] + M[j][i]);
            M[i][j] = v;
            V[i][j] = (i == j) ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < b; i++)
            for (int j = 0; j < b; j++) {
                if (i != j) off += M[i][j] * M[i][j];
                else diag += M[i][i] * M[i][i];
            }
        if (off <= 1e-32 * diag || off == 0.0) break;
        for (int p = 0; p < b; p++)
            for (int q = p + 1; q < b; q++) {
                if (M[p][q] == 0.0) continue;
                const double tau = (M[q][q] - M[p][p]) / (2.0 * M[p][q]);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
                for (int k = 0; k < b; k++) {  // M <- J^T M J
                    const double mkp = M[k][p], mkq = M[k][q];
                    M[k][p] = c * mkp - sn * mkq;
                    M[k][q] = sn * mkp + c * mkq;
                }
                for (int k = 0; k < b; k++) {
                    const double mpk = M[p][k], mqk = M[q][k];
                    M[p][k] = c * mpk - sn * mqk;
                    M[q][k] = sn * mpk + c * mqk;
                }
                for (int k = 0; k < b; k++) {
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - sn * vkq;
                    V[k][q] = sn * vkp + c * vkq;
                }
            }
    }
    // sort ascending (selection sort on the columns)
    int ord[GI_MAXB];
    for (int i = 0; i < b; i++) ord[i] = i;
    for (int i = 0; i < b; i++)
        for (int j = i + 1; j < b; j++)
            if (M[ord[j]][ord[j]] < M[ord[i]][ord[i]]) { const int t = ord[i]; ord[i] = ord[j]; ord[j] = t; }
    double* th = theta + (size_t)s * GI_MAXB;
    double* Cs = C + (size_t)s * GI_MAXB * GI_MAXB;
    for (int jj = 0; jj < b; jj++) {
        const int j = ord[jj];
        th[jj] = M[j][j];
        // column = L^-T v_j
        double x[GI_MAXB];
        for (int i = b - 1; i >= 0; i--) {
            double v = V[i][j];
            for (int k = i + 1; k < b; k++) v -= L[k][i] * x[k];
            x[i] = v / L[i][i];
        }
        for (int i = 0; i < b; i++) Cs[i + jj * b] = sc[i] * x[i];
    }
    bad[s] = fail;
}

// backward error of each Ritz pair: |AX_j - th_j BX_j| / ((nA + |th_j| nB) |X_j|)
__global__ void k_ritz_err(const int* __restrict__ ns, const int64_t* __restrict__ xoff,
                           const double* AX, const double* BX, const double* X, int b,
                           const double* __restrict__ theta, const double* __restrict__ nrm,
                           double* err, const int* __restrict__ act) {
    __shared__ double red[32];
    const int s = blockIdx.x;
    if (!act[s]) return;
    const int m = ns[s];
    for (int j = 0; j < b; j++) {
        const double th = theta[(size_t)s * GI_MAXB + j];
        const double* ax = AX + xoff[s] + (size_t)j * m;
        const double* bx = BX + xoff[s] + (size_t)j * m;
        const double* x = X + xoff[s] + (size_t)j * m;
        double r2 = 0.0, x2 = 0.0;
        for (int p = threadIdx.x; p < m; p += blockDim.x) {
            const double r = ax[p] - th * bx[p];
            r2 += r * r;
            x2 += x[p] * x[p];
        }
        r2 = block_sum(r2, red);
        x2 = block_sum(x2, red);
        if (threadIdx.x == 0)
            err[(size_t)s * GI_MAXB + j] = sqrt(r2) / ((nrm[2 * s] + fabs(th) * nrm[2 * s + 1]) * sqrt(x2) + 1e-300);
    }
}

// Frobenius norms of M_A and M_B per subdomain
__global__ void k_fro2(const int* __restrict__ ns, const int64_t* __restrict__ off, const double* A,
                       const double* B, double* nrm) {
    __shared__ double red[32];
    const int s = blockIdx.x;
    const int64_t mm = (int64_t)ns[s] * ns[s];
    double pa = 0.0, pb = 0.0;
    for (int64_t e = threadIdx.x; e < mm; e += blockDim.x) {
        const double a = A[off[s] + e], b = B[off[s] + e];
        pa += a * a;
        pb += b * b;
    }
    pa = block_sum(pa, red);
    pb = block_sum(pb, red);
    if (threadIdx.x == 0) { nrm[2 * s] = sqrt(pa); nrm[2 * s + 1] = sqrt(pb); }
}

// K_s = D_s V^s_- (rows scaled by the partition of unity)
__global__ void k_kernel_basis(const int* __restrict__ ns, const int* __restrict__ sub_ptr,
                               const int* __restrict__ sub_idx, const double* __restrict__ dvec,
                               const int* __restrict__ nm_ptr, const int64_t* __restrict__ vm_off,
                               const double* __restrict__ V, double* K) {
    const int s = blockIdx.x;
    const int m = ns[s], nu = nm_ptr[s + 1] - nm_ptr[s];
    const int* idx = sub_idx + sub_ptr[s];
    for (int e = threadIdx.x; e < m * nu; e += blockDim.x) {
        const int p = e % m;
        K[vm_off[s] + e] = dvec[idx[p]] * V[vm_off[s] + e];
    }
}

// S_s = M_A - mu M_B (dense), certificate matrix before the low-rank term
__global__ void k_cert_base(const int* __restrict__ ns, const int64_t* __restrict__ off,
                            const double* MA, const double* MB, double mu, double* S,
                            const int* __restrict__ act) {
    const int s = blockIdx.x;
    if (!act[s]) return;
    const int64_t mm = (int64_t)ns[s] * ns[s];
    for (int64_t e = blockIdx.y * (int64_t)blockDim.x + threadIdx.x; e < mm; e += (int64_t)gridDim.y * blockDim.x)
        S[off[s] + e] = MA[off[s] + e] - mu * MB[off[s] + e];
}

// U_s = [Kq_s | X_s(:, 0..e_s)] and (if BU is given) BU_s = [MBKq_s | BX_s(:, 0..e_s)],
// m x (nu+e)
__global__ void k_pack_u(const int* __restrict__ ns, const int* __restrict__ nm_ptr,
                         const int64_t* __restrict__ vm_off, const double* Kq, const double* MBKq,
                         const int64_t* __restrict__ xoff, const double* X, const double* BX,
                         const int* __restrict__ ecount, const int64_t* __restrict__ uoff, double* U,
                         double* BU, const int* __restrict__ act) {
    const int s = blockIdx.x;
    if (!act[s]) return;
    const int m = ns[s], nu = nm_ptr[s + 1] - nm_ptr[s], e = ecount[s];
    for (int t = threadIdx.x; t < m * (nu + e); t += blockDim.x) {
        const int p = t % m, c = t / m;
        double u, bu;
        if (c < nu) { u = Kq[vm_off[s] + t]; bu = MBKq[vm_off[s] + t]; }
        else {
            const size_t o = xoff[s] + (size_t)(c - nu) * m + p;
            u = X[o];
            bu = BX[o];
        }
        U[uoff[s] + t] = u;
        if (BU) BU[uoff[s] + t] = bu;
    }
}

awg_status geneo_block_solve(Handle* h, const double* MA, const double* MB, const double* d_params,
                             int b, int maxit, double tol, GeneoIter& r) {
    cudaStream_t s = h->stream;
    const int N = h->N;
    b = std::max(2, std::min(b, GI_MAXB));
    r.b = b;
    r.ecount.assign(N, -1);
    r.its.assign(N, 0);
    const std::vector<int>& hm = h->h_ns;
    const std::vector<int>& hnu = h->h_nm;
    const int maxm = h->max_ns;
    const size_t smem = (size_t)maxm * b * 8;
    if (smem > 227 * 1024) return AWG_OK;  // every subdomain goes to the dense eigensolver
    // arenas of m x b blocks
    r.hx.assign(N + 1, 0);
    for (int t = 0; t < N; t++) r.hx[t + 1] = r.hx[t] + (int64_t)hm[t] * b;
    const std::vector<int64_t>& hx = r.hx;
    DevBuf Y, T1, AY, BY, AX, small, act, bad, Kb, MBK, KMK, nrm, err, theta, dkoff;
    AWG_TRY(upload(h, r.xoff, hx.data(), (N + 1) * sizeof(int64_t)));
    const size_t xb = (size_t)hx[N] * 8;
    for (DevBuf* buf : {&r.X, &r.BX, &Y, &T1, &AY, &BY, &AX}) AWG_TRY(dalloc(h, *buf, xb));
    AWG_TRY(dalloc(h, small, (size_t)N * GI_MAXB * GI_MAXB * 8 * 3));
    AWG_TRY(dalloc(h, theta, (size_t)N * GI_MAXB * 8));
    AWG_TRY(dalloc(h, err, (size_t)N * GI_MAXB * 8));
    AWG_TRY(dalloc(h, nrm, (size_t)N * 2 * 8));
    AWG_TRY(dalloc(h, act, N * sizeof(int)));
    AWG_TRY(dalloc(h, bad, N * sizeof(int)));
    double* At = (double*)small.p;
    double* Bt = At + (size_t)N * GI_MAXB * GI_MAXB;
    double* Cs = Bt + (size_t)N * GI_MAXB * GI_MAXB;
    int* dact = (int*)act.p;
    const int64_t* dxoff = (const int64_t*)r.xoff.p;
    // a subdomain whose complement of the kernel is narrower than the block
    // goes to the dense eigensolver
    std::vector<int> hact(N, 1);
    int n_active = N;
    for (int t = 0; t < N; t++)
        if (hm[t] - hnu[t] < b) { hact[t] = 0; n_active--; }
    AWG_CUDA(cudaMemcpyAsync(dact, hact.data(), N * sizeof(int), cudaMemcpyHostToDevice, s));
    k_fro2<<<N, 256, 0, s>>>((int*)h->ns.p, (int64_t*)h->dense_off.p, MA, MB, (double*)nrm.p);
    AWG_LAUNCH();

    // kernel basis K, M_B K, K^T M_B K = L L^T, Kq = K L^-T, M_B Kq
    const int64_t vlen = std::max<int64_t>(1, h->h_vm_off[N]);
    for (DevBuf* buf : {&Kb, &MBK, &r.Kq, &r.MBKq}) AWG_TRY(dalloc(h, *buf, vlen * 8));
    std::vector<int64_t> hk(N + 1, 0);
    for (int t = 0; t < N; t++) hk[t + 1] = hk[t] + (int64_t)hnu[t] * hnu[t];
    AWG_TRY(dalloc(h, KMK, std::max<int64_t>(1, hk[N]) * 8));
    AWG_TRY(upload(h, dkoff, hk.data(), (N + 1) * sizeof(int64_t)));
    auto release = [&]() {
        for (DevBuf* bb : {&Y, &T1, &AY, &BY, &AX, &small, &act, &bad, &Kb, &MBK, &KMK, &nrm, &err, &theta,
                           &dkoff})
            dfree(h, *bb);
    };
    if (h->h_vm_off[N] > 0) {
        k_kernel_basis<<<N, 256, 0, s>>>((int*)h->ns.p, (int*)h->sub_ptr.p, (int*)h->sub_idx.p,
                                         (double*)h->dvec.p, (int*)h->nm_ptr.p, (int64_t*)h->vm_off.p,
                                         (double*)h->Vm.p, (double*)Kb.p);
        AWG_LAUNCH();
        std::vector<GemmDesc> d1, d2;
        for (int t = 0; t < N; t++) {
            const int m = hm[t], nu = hnu[t];
            if (!nu) continue;
            const int64_t o = h->h_vm_off[t];
            d1.push_back({MB + h->h_dense_off[t], (double*)Kb.p + o, (double*)MBK.p + o, m, nu, m, m, m, m, 0, 0, 1.0, 0.0});
            d2.push_back({(double*)Kb.p + o, (double*)MBK.p + o, (double*)KMK.p + hk[t], nu, nu, m, m, m, nu, 1, 0, 1.0, 0.0});
        }
        AWG_TRY(gemm_batched(h, d1, s));
        AWG_TRY(gemm_batched(h, d2, s));
        const int maxnu = *std::max_element(hnu.begin(), hnu.end());
        AWG_CUDA(cudaMemsetAsync(h->flag.p, 0, sizeof(int), s));
        AWG_TRY(potrf_batched(h, (double*)KMK.p, (int*)h->nm.p, (int64_t*)dkoff.p, N, std::max(1, maxnu),
                              (int*)h->flag.p, s));
        int fl = 0;
        AWG_TRY(read_flag(h, &fl));
        if (fl & FLAG_NOT_SPD) {  // K^T M_B K not SPD: leave the pencils to the dense eigensolver
            release();
            return AWG_OK;
        }
        AWG_TRY(trtri_batched(h, (double*)KMK.p, (int*)h->nm.p, (int64_t*)dkoff.p, N, std::max(1, maxnu), s));
        std::vector<GemmDesc> d3, d4;
        for (int t = 0; t < N; t++) {
            const int m = hm[t], nu = hnu[t];
            if (!nu) continue;
            const int64_t o = h->h_vm_off[t];
            d3.push_back({(double*)Kb.p + o, (double*)KMK.p + hk[t], (double*)r.Kq.p + o, m, nu, nu, m, nu, m, 0, 1, 1.0, 0.0});
            d4.push_back({(double*)MBK.p + o, (double*)KMK.p + hk[t], (double*)r.MBKq.p + o, m, nu, nu, m, nu, m, 0, 1, 1.0, 0.0});
        }
        AWG_TRY(gemm_batched(h, d3, s));
        AWG_TRY(gemm_batched(h, d4, s));
    }

    // start block: predicted leverage profile (learned) or plain random
    double *dX = (double*)r.X.p, *dBX = (double*)r.BX.p, *dY = (double*)Y.p, *dT1 = (double*)T1.p,
           *dAY = (double*)AY.p, *dBY = (double*)BY.p, *dAX = (double*)AX.p;
    {
        DevBuf F, g;
        const double* dg = nullptr;
        if (d_params) {
            AWG_TRY(dalloc(h, F, (size_t)h->sum_ns * 5 * 8));
            AWG_TRY(dalloc(h, g, (size_t)h->sum_ns * 8));
            AWG_TRY(learned_features(h, (double*)F.p, s));
            AWG_TRY(learned_forward((int)h->sum_ns, (double*)F.p, d_params, (double*)g.p, AWG_MIXED_FP32, s));
            dg = (double*)g.p;
        }
        AWG_TRY(learned_start_block(h, dxoff, b, dg, dX, s));
        AWG_CUDA(cudaStreamSynchronize(s));
        dfree(h, F);
        dfree(h, g);
    }
    // X0 <- P X0 happens through the first step (P is applied after T)

    if (smem > 48 * 1024)
        AWG_CUDA(cudaFuncSetAttribute(k_symm_skinny, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const dim3 gsk(N, (maxm + GI_ROWS - 1) / GI_ROWS);
    const double* G = (const double*)h->prec[AWG_FP64].G.p;  // T = D (A^s_+)^+ D
    const int* dns = (const int*)h->ns.p;
    const int64_t* doff = (const int64_t*)h->dense_off.p;
    std::vector<double> hth((size_t)N * GI_MAXB), herr((size_t)N * GI_MAXB);
    std::vector<int> hbad(N);
    const double mu = h->tau * (1.0 - 1e-6);
    std::vector<int64_t> hpc(N + 1, 0);
    for (int t = 0; t < N; t++) hpc[t + 1] = hpc[t] + (int64_t)hnu[t] * b;
    DevBuf PC1, Sarena;
    AWG_TRY(dalloc(h, PC1, std::max<int64_t>(1, hpc[N]) * 8));
    AWG_TRY(dalloc(h, Sarena, (size_t)h->dense_total * 8));
    std::vector<int> cand(N, 0), ec(N, 0);
    for (int it = 1; it <= maxit && n_active > 0; it++) {
        // Y = P T M_B X
        k_symm_skinny<<<gsk, 256, smem, s>>>(dns, doff, MB, dxoff, dX, dT1, b, 1.0, 0.0, dact);
        AWG_LAUNCH();
        k_symm_skinny<<<gsk, 256, smem, s>>>(dns, doff, G, dxoff, dT1, dY, b, 1.0, 0.0, dact);
        AWG_LAUNCH();
        {
            std::vector<GemmDesc> d1, d2;
            for (int t = 0; t < N; t++) {
                const int m = hm[t], nu = hnu[t];
                if (!nu || !hact[t]) continue;
                const int64_t o = h->h_vm_off[t];
                d1.push_back({(double*)r.MBKq.p + o, dY + hx[t], (double*)PC1.p + hpc[t], nu, b, m, m, m, nu, 1, 0, 1.0, 0.0});
                d2.push_back({(double*)r.Kq.p + o, (double*)PC1.p + hpc[t], dY + hx[t], m, b, nu, m, nu, m, 0, 0, -1.0, 1.0});
            }
            AWG_TRY(gemm_batched(h, d1, s));
            AWG_TRY(gemm_batched(h, d2, s));
        }
        // Rayleigh-Ritz on span(Y)
        k_symm_skinny<<<gsk, 256, smem, s>>>(dns, doff, MA, dxoff, dY, dAY, b, 1.0, 0.0, dact);
        AWG_LAUNCH();
        k_symm_skinny<<<gsk, 256, smem, s>>>(dns, doff, MB, dxoff, dY, dBY, b, 1.0, 0.0, dact);
        AWG_LAUNCH();
        k_gram<<<N, 256, 0, s>>>(dns, dxoff, dY, b, dxoff, dAY, b, At, dact);
        AWG_LAUNCH();
        k_gram<<<N, 256, 0, s>>>(dns, dxoff, dY, b, dxoff, dBY, b, Bt, dact);
        AWG_LAUNCH();
        k_small_geig<<<(N + 63) / 64, 64, 0, s>>>(N, b, At, Bt, (double*)theta.p, Cs, (int*)bad.p, dact);
        AWG_LAUNCH();
        k_small_mul<<<N, 256, 0, s>>>(dns, dxoff, dY, b, Cs, b, dX, dact);
        AWG_LAUNCH();
        k_small_mul<<<N, 256, 0, s>>>(dns, dxoff, dAY, b, Cs, b, dAX, dact);
        AWG_LAUNCH();
        k_small_mul<<<N, 256, 0, s>>>(dns, dxoff, dBY, b, Cs, b, dBX, dact);
        AWG_LAUNCH();
        k_ritz_err<<<N, 256, 0, s>>>(dns, dxoff, dAX, dBX, dX, b, (double*)theta.p, (double*)nrm.p,
                                     (double*)err.p, dact);
        AWG_LAUNCH();
        AWG_CUDA(cudaMemcpyAsync(hth.data(), theta.p, hth.size() * 8, cudaMemcpyDeviceToHost, s));
        AWG_CUDA(cudaMemcpyAsync(herr.data(), err.p, herr.size() * 8, cudaMemcpyDeviceToHost, s));
        AWG_CUDA(cudaMemcpyAsync(hbad.data(), bad.p, N * sizeof(int), cudaMemcpyDeviceToHost, s));
        AWG_CUDA(cudaStreamSynchronize(s));
        // candidates: every Ritz pair below tau has converged
        int nc = 0;
        for (int t = 0; t < N; t++) {
            cand[t] = 0;
            if (!hact[t]) continue;
            int e = 0;
            bool ok = !hbad[t];
            for (int j = 0; j < b; j++)
                if (hth[(size_t)t * GI_MAXB + j] < h->tau) {
                    e++;
                    if (!(herr[(size_t)t * GI_MAXB + j] <= tol)) ok = false;
                }
            if (e == b) {  // the block cannot hold the extra modes: dense eigensolver
                hact[t] = 0;
                r.its[t] = it;
                n_active--;
                continue;
            }
            if (ok) { cand[t] = 1; ec[t] = e; nc++; }
        }
        // certificates are dense Cholesky factorisations: batch them
        const bool attempt = nc > 0 && (2 * nc >= n_active || it % 4 == 0 || it == maxit);
        if (attempt) {
            std::vector<int64_t> hu(N + 1, 0);
            for (int t = 0; t < N; t++) hu[t + 1] = hu[t] + (cand[t] ? (int64_t)hm[t] * (hnu[t] + ec[t]) : 0);
            DevBuf dcand, duoff, decount, U, BU, cst, dcm, dco;
            AWG_TRY(upload(h, dcand, cand.data(), N * sizeof(int)));
            AWG_TRY(upload(h, duoff, hu.data(), (N + 1) * sizeof(int64_t)));
            AWG_TRY(upload(h, decount, ec.data(), N * sizeof(int)));
            AWG_TRY(dalloc(h, U, std::max<int64_t>(1, hu[N]) * 8));
            AWG_TRY(dalloc(h, BU, std::max<int64_t>(1, hu[N]) * 8));
            k_pack_u<<<N, 256, 0, s>>>(dns, (int*)h->nm_ptr.p, (int64_t*)h->vm_off.p, (double*)r.Kq.p,
                                       (double*)r.MBKq.p, dxoff, dX, dBX, (int*)decount.p, (int64_t*)duoff.p,
                                       (double*)U.p, (double*)BU.p, (int*)dcand.p);
            AWG_LAUNCH();
            k_cert_base<<<dim3(N, 16), 256, 0, s>>>(dns, doff, MA, MB, mu, (double*)Sarena.p, (int*)dcand.p);
            AWG_LAUNCH();
            std::vector<GemmDesc> dc;
            std::vector<int> cm, sel;
            std::vector<int64_t> coff;
            for (int t = 0; t < N; t++) {
                if (!cand[t]) continue;
                const int m = hm[t], k = hnu[t] + ec[t];
                if (k > 0)
                    dc.push_back({(double*)BU.p + hu[t], (double*)BU.p + hu[t],
                                  (double*)Sarena.p + h->h_dense_off[t], m, m, k, m, m, m, 0, 1, 2.0, 1.0});
                cm.push_back(m);
                coff.push_back(h->h_dense_off[t]);
                sel.push_back(t);
            }
            AWG_TRY(gemm_batched(h, dc, s));
            AWG_TRY(upload(h, dcm, cm.data(), cm.size() * sizeof(int)));
            AWG_TRY(upload(h, dco, coff.data(), coff.size() * sizeof(int64_t)));
            AWG_TRY(dalloc(h, cst, cm.size() * sizeof(int)));
            AWG_TRY(potrf_batched(h, (double*)Sarena.p, (int*)dcm.p, (int64_t*)dco.p, (int)cm.size(), maxm,
                                  nullptr, s, (int*)cst.p));
            std::vector<int> hst(cm.size());
            AWG_CUDA(cudaMemcpyAsync(hst.data(), cst.p, cm.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
            AWG_CUDA(cudaStreamSynchronize(s));
            for (size_t k = 0; k < sel.size(); k++) {
                const int t = sel[k];
                if (hst[k] == 0) {
                    hact[t] = 0;
                    r.its[t] = it;
                    r.ecount[t] = ec[t];
                    n_active--;
                }
            }
            for (DevBuf* bb : {&dcand, &duoff, &decount, &U, &BU, &cst, &dcm, &dco}) dfree(h, *bb);
        }
        AWG_CUDA(cudaMemcpyAsync(dact, hact.data(), N * sizeof(int), cudaMemcpyHostToDevice, s));
    }
    for (int t = 0; t < N; t++)
        if (hact[t]) r.its[t] = maxit;  // not certified within maxit
    AWG_CUDA(cudaStreamSynchronize(s));
    dfree(h, PC1);
    dfree(h, Sarena);
    release();
    return AWG_OK;
}

awg_status geneo_block_pack(Handle* h, GeneoIter& r, const int64_t* d_zoff, double* Z) {
    cudaStream_t s = h->stream;
    const int N = h->N;
    std::vector<int> ok(N), ec(N);
    for (int t = 0; t < N; t++) {
        ok[t] = r.ecount[t] >= 0;
        ec[t] = std::max(0, r.ecount[t]);
    }
    DevBuf dok, dec;
    AWG_TRY(upload(h, dok, ok.data(), N * sizeof(int)));
    AWG_TRY(upload(h, dec, ec.data(), N * sizeof(int)));
    k_pack_u<<<N, 256, 0, s>>>((int*)h->ns.p, (int*)h->nm_ptr.p, (int64_t*)h->vm_off.p, (double*)r.Kq.p,
                               (double*)r.MBKq.p, (int64_t*)r.xoff.p, (double*)r.X.p, (double*)r.BX.p,
                               (int*)dec.p, d_zoff, Z, nullptr, (int*)dok.p);
    AWG_LAUNCH();
    AWG_CUDA(cudaStreamSynchronize(s));
    dfree(h, dok);
    dfree(h, dec);
    return AWG_OK;
}

void geneo_block_free(Handle* h, GeneoIter& r) {
    for (DevBuf* bb : {&r.xoff, &r.X, &r.BX, &r.Kq, &r.MBKq}) dfree(h, *bb);
}

}  // namespace awg
