// Subdomain structure on the device (Sections 2.1-2.2 and 3.1 of the paper):
// overlapping sets Omega^s (Def. 1) grown from the owner of every dof,
// the partition of unity D (Def. 3), the incidence lists used by every
// prolongation sum_s R^sT (.), the pair multiplicity M_mu and the splitting
// B = A / M_mu (Def. 5), with the minimal-overlap check of Assumption 1.

#include "awg_common.cuh"

#include <algorithm>
#include <numeric>

namespace awg {

// CSR sanity: rowptr non-decreasing, column indices in range and strictly
// increasing inside each row.
__global__ void k_check_csr(int n, const int* __restrict__ rp, const int* __restrict__ ci, int nnz,
                            int* flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int a = rp[i], b = rp[i + 1];
    if (a < 0 || b < a || b > nnz) { atomicOr(flag, FLAG_BAD_CSR); return; }
    int prev = -1;
    bool diag = false;
    for (int k = a; k < b; k++) {
        const int j = ci[k];
        if (j < 0 || j >= n || j <= prev) { atomicOr(flag, FLAG_BAD_CSR); return; }
        if (j == i) diag = true;
        prev = j;
    }
    if (!diag) atomicOr(flag, FLAG_NOT_SPD);  // an SPD matrix stores its diagonal
}

// Structural symmetry: every stored (i, j) has a stored (j, i).
__global__ void k_check_sym(int n, const int* __restrict__ rp, const int* __restrict__ ci, int* flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = rp[i]; k < rp[i + 1]; k++) {
        const int j = ci[k];
        if (bsearch_idx(ci + rp[j], rp[j + 1] - rp[j], i) < 0) { atomicOr(flag, FLAG_NOT_SYM); return; }
    }
}

__global__ void k_mask_init(int n, int N, const int* __restrict__ part, uint8_t* mask, int* flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = part[i];
    if (p < 0 || p >= N) { atomicOr(flag, FLAG_BAD_CSR); return; }
    mask[(size_t)p * n + i] = 1;
}

// One layer of growth: i joins Omega^s if a stored neighbour is in it.
__global__ void k_grow(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                       const uint8_t* __restrict__ in, uint8_t* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const size_t base = (size_t)blockIdx.y * n;
    uint8_t v = in[base + i];
    for (int k = rp[i]; k < rp[i + 1] && !v; k++) v = in[base + ci[k]];
    out[base + i] = v;
}

__global__ void k_mask_count(int n, const uint8_t* __restrict__ mask, int* cnt) {
    __shared__ double red[32];
    const size_t base = (size_t)blockIdx.x * n;
    double c = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) c += mask[base + i];
    c = block_sum(c, red);
    if (threadIdx.x == 0) cnt[blockIdx.x] = (int)c;
}

// Ordered compaction of mask row s into sub_idx[sub_ptr[s] ...].
__global__ void __launch_bounds__(1024) k_compact(int n, const uint8_t* __restrict__ mask,
                                                  const int* __restrict__ sub_ptr, int* sub_idx) {
    __shared__ int warp_tot[32];
    __shared__ int base_sh;
    const int s = blockIdx.x;
    const size_t mb = (size_t)s * n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) base_sh = sub_ptr[s];
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        const int f = (i < n) ? mask[mb + i] : 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        const int before = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[wid] = __popc(bal);
        __syncthreads();
        int woff = 0;
        for (int w = 0; w < wid; w++) woff += warp_tot[w];
        const int base = base_sh;
        if (f) sub_idx[base + woff + before] = i;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int w = 0; w < nw; w++) t += warp_tot[w];
            base_sh = base + t;
        }
        __syncthreads();
    }
}

__global__ void k_mult(int n, int N, const uint8_t* __restrict__ mask, int* mult, double* dvec,
                       int* flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0;
    for (int s = 0; s < N; s++) c += mask[(size_t)s * n + i];
    mult[i] = c;
    if (c == 0) atomicOr(flag, FLAG_MIN_OVERLAP);
    dvec[i] = (c > 0) ? 1.0 / (double)c : 0.0;
}

// Incidence: the copies of dof i, in subdomain order, as positions in the
// concatenated local arena (sub_ptr[s] + local index) and their subdomain.
__global__ void k_incidence(int n, int N, const uint8_t* __restrict__ mask,
                            const int* __restrict__ sub_ptr, const int* __restrict__ sub_idx,
                            const int* __restrict__ inc_ptr, int* inc_pos, int* inc_sub) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = inc_ptr[i];
    for (int s = 0; s < N; s++) {
        if (!mask[(size_t)s * n + i]) continue;
        const int a = sub_ptr[s];
        const int p = bsearch_idx(sub_idx + a, sub_ptr[s + 1] - a, i);
        inc_pos[c] = a + p;
        inc_sub[c] = s;
        c++;
    }
}

// M_mu(i, j) = #{s : i, j in Omega^s} for stored (i, j) and B = A / M_mu.
__global__ void k_pair_mult(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                            const double* __restrict__ a, const int* __restrict__ inc_ptr,
                            const int* __restrict__ inc_sub, const uint8_t* __restrict__ mask,
                            double* mmu, double* b, int* flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = rp[i]; k < rp[i + 1]; k++) {
        const int j = ci[k];
        int c = 0;
        for (int e = inc_ptr[i]; e < inc_ptr[i + 1]; e++) c += mask[(size_t)inc_sub[e] * n + j];
        mmu[k] = (double)c;
        if (c == 0) {
            atomicOr(flag, FLAG_MIN_OVERLAP);
            b[k] = 0.0;
        } else {
            b[k] = a[k] / (double)c;
        }
    }
}

__global__ void k_pos_sub(int N, const int* __restrict__ sub_ptr, int* pos_sub) {
    const int s = blockIdx.x;
    for (int p = sub_ptr[s] + threadIdx.x; p < sub_ptr[s + 1]; p += blockDim.x) pos_sub[p] = s;
}

// Dense R^s X R^sT of a CSR value array X (same pattern as A) into the
// per-subdomain blocks (arena zeroed beforehand).
__global__ void k_assemble_local(const int* __restrict__ rp, const int* __restrict__ ci,
                                 const double* __restrict__ x, const int* __restrict__ sub_ptr,
                                 const int* __restrict__ sub_idx, const int64_t* __restrict__ off,
                                 double* arena) {
    const int s = blockIdx.x;
    const int a0 = sub_ptr[s], m = sub_ptr[s + 1] - a0;
    const int* idx = sub_idx + a0;
    double* blk = arena + off[s];
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        const int i = idx[p];
        for (int k = rp[i]; k < rp[i + 1]; k++) {
            const int q = bsearch_idx(idx, m, ci[k]);
            if (q >= 0) blk[p + (size_t)q * m] = x[k];
        }
    }
}

awg_status assemble_local(Handle* h, const double* d_vals, double* arena) {
    AWG_CUDA(cudaMemsetAsync(arena, 0, (size_t)h->dense_total * sizeof(double), h->stream));
    k_assemble_local<<<h->N, 256, 0, h->stream>>>((int*)h->rowptr.p, (int*)h->colidx.p, d_vals,
                                                  (int*)h->sub_ptr.p, (int*)h->sub_idx.p,
                                                  (int64_t*)h->dense_off.p, arena);
    AWG_LAUNCH();
    return AWG_OK;
}

awg_status setup_structure(Handle* h, const int* d_part) {
    const int n = h->n, N = h->N;
    cudaStream_t s = h->stream;
    const int tb = 256, gb = (n + tb - 1) / tb;
    int* flag = (int*)h->flag.p;
    AWG_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
    k_check_csr<<<gb, tb, 0, s>>>(n, (int*)h->rowptr.p, (int*)h->colidx.p, h->nnz, flag);
    AWG_LAUNCH();
    int f = 0;
    AWG_TRY(read_flag(h, &f));
    if (f & FLAG_BAD_CSR) return AWG_ERR_INVALID_ARG;
    if (f & FLAG_NOT_SPD) return AWG_ERR_NOT_SPD;
    k_check_sym<<<gb, tb, 0, s>>>(n, (int*)h->rowptr.p, (int*)h->colidx.p, flag);
    AWG_LAUNCH();
    AWG_TRY(read_flag(h, &f));
    if (f & FLAG_NOT_SYM) return AWG_ERR_NOT_SYMMETRIC;

    // masks of Omega^s, N x n bytes, grown layer by layer
    DevBuf m0, m1;
    const size_t mbytes = (size_t)N * n;
    AWG_TRY(dalloc(h, m0, mbytes));
    AWG_TRY(dalloc(h, m1, mbytes));
    AWG_CUDA(cudaMemsetAsync(m0.p, 0, mbytes, s));
    k_mask_init<<<gb, tb, 0, s>>>(n, N, d_part, (uint8_t*)m0.p, flag);
    AWG_LAUNCH();
    AWG_TRY(read_flag(h, &f));
    if (f & FLAG_BAD_CSR) { dfree(h, m0); dfree(h, m1); return AWG_ERR_INVALID_ARG; }
    for (int l = 0; l < h->overlap; l++) {
        dim3 g(gb, N);
        k_grow<<<g, tb, 0, s>>>(n, (int*)h->rowptr.p, (int*)h->colidx.p, (uint8_t*)m0.p,
                                (uint8_t*)m1.p);
        AWG_LAUNCH();
        std::swap(m0, m1);
    }
    uint8_t* mask = (uint8_t*)m0.p;
    dfree(h, m1);

    // sizes, offsets, sorted index lists
    DevBuf cnt;
    AWG_TRY(dalloc(h, cnt, N * sizeof(int)));
    k_mask_count<<<N, 256, 0, s>>>(n, mask, (int*)cnt.p);
    AWG_LAUNCH();
    h->h_ns.assign(N, 0);
    AWG_CUDA(cudaMemcpyAsync(h->h_ns.data(), cnt.p, N * sizeof(int), cudaMemcpyDeviceToHost, s));
    AWG_CUDA(cudaStreamSynchronize(s));
    dfree(h, cnt);
    h->h_sub_ptr.assign(N + 1, 0);
    h->h_dense_off.assign(N + 1, 0);
    h->max_ns = 0;
    for (int i = 0; i < N; i++) {
        if (h->h_ns[i] == 0) { dfree(h, m0); return AWG_ERR_INVALID_ARG; }  // empty part
        h->h_sub_ptr[i + 1] = h->h_sub_ptr[i] + h->h_ns[i];
        h->h_dense_off[i + 1] = h->h_dense_off[i] + (int64_t)h->h_ns[i] * h->h_ns[i];
        h->max_ns = std::max(h->max_ns, h->h_ns[i]);
    }
    h->sum_ns = h->h_sub_ptr[N];
    h->dense_total = h->h_dense_off[N];
    AWG_TRY(upload(h, h->ns, h->h_ns.data(), N * sizeof(int)));
    AWG_TRY(upload(h, h->sub_ptr, h->h_sub_ptr.data(), (N + 1) * sizeof(int)));
    AWG_TRY(upload(h, h->dense_off, h->h_dense_off.data(), (N + 1) * sizeof(int64_t)));
    AWG_TRY(dalloc(h, h->sub_idx, (size_t)h->sum_ns * sizeof(int)));
    k_compact<<<N, 1024, 0, s>>>(n, mask, (int*)h->sub_ptr.p, (int*)h->sub_idx.p);
    AWG_LAUNCH();
    AWG_TRY(dalloc(h, h->pos_sub, (size_t)h->sum_ns * sizeof(int)));
    k_pos_sub<<<N, 256, 0, s>>>(N, (int*)h->sub_ptr.p, (int*)h->pos_sub.p);
    AWG_LAUNCH();

    // multiplicity, D, incidence
    DevBuf mult;
    DevBuf& inc_sub = h->inc_sub;
    AWG_TRY(dalloc(h, mult, n * sizeof(int)));
    AWG_TRY(dalloc(h, h->dvec, n * sizeof(double)));
    k_mult<<<gb, tb, 0, s>>>(n, N, mask, (int*)mult.p, (double*)h->dvec.p, flag);
    AWG_LAUNCH();
    std::vector<int> hm(n), hptr(n + 1, 0);
    AWG_CUDA(cudaMemcpyAsync(hm.data(), mult.p, n * sizeof(int), cudaMemcpyDeviceToHost, s));
    AWG_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < n; i++) hptr[i + 1] = hptr[i] + hm[i];
    AWG_TRY(upload(h, h->inc_ptr, hptr.data(), (n + 1) * sizeof(int)));
    AWG_TRY(dalloc(h, h->inc_pos, (size_t)hptr[n] * sizeof(int)));
    AWG_TRY(dalloc(h, inc_sub, (size_t)hptr[n] * sizeof(int)));
    k_incidence<<<gb, tb, 0, s>>>(n, N, mask, (int*)h->sub_ptr.p, (int*)h->sub_idx.p,
                                  (int*)h->inc_ptr.p, (int*)h->inc_pos.p, (int*)inc_sub.p);
    AWG_LAUNCH();

    // M_mu and B
    AWG_TRY(dalloc(h, h->mmu, (size_t)h->nnz * sizeof(double)));
    AWG_TRY(dalloc(h, h->bval, (size_t)h->nnz * sizeof(double)));
    k_pair_mult<<<gb, tb, 0, s>>>(n, (int*)h->rowptr.p, (int*)h->colidx.p, (double*)h->val.p,
                                  (int*)h->inc_ptr.p, (int*)inc_sub.p, mask, (double*)h->mmu.p,
                                  (double*)h->bval.p, flag);
    AWG_LAUNCH();
    AWG_TRY(read_flag(h, &f));
    dfree(h, mult);
    dfree(h, m0);
    if (f & FLAG_MIN_OVERLAP) return AWG_ERR_MIN_OVERLAP;
    return AWG_OK;
}

}  // namespace awg
