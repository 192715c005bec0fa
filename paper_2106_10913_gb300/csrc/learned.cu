// Learned start block for the GenEO block eigensolver (setup of Thm. 4).
//
// A 5-16-16-1 network (tanh, tanh, sigmoid) maps per-node features of a
// subdomain, computed from A alone, to the predicted normalised leverage of
// the subdomain's extra GenEO modes (eigenvalue in (0, tau); the kernel part
// D^s V^s_- is known exactly).  The start block of the block eigensolver is
// built from the square root of that profile.  Training data come from the
// exact eigensolve of the setup itself; training (forward, backward, Adam)
// and inference are the kernels below, in float32 or float64.
//
// Parameter layout (385 values): W1[16x5] row-major, b1[16], W2[16x16]
// row-major, b2[16], w3[16], b3.

#include "awg_common.cuh"

#include <algorithm>
#include <cmath>

namespace awg {

constexpr int LN_F = 5, LN_H1 = 16, LN_H2 = 16;
constexpr int LN_P = LN_H1 * LN_F + LN_H1 + LN_H2 * LN_H1 + LN_H2 + LN_H2 + 1;  // 385
static_assert(LN_P == LEARNED_NPARAM && LN_F == LEARNED_NF, "network layout");

// ---------------------------------------------------------------- features
// One block per subdomain; features row-major (sum_ns x 5) at sub_ptr[s]:
//   f0 = (log10 A_pp - mean_subdomain log10 A_qq) / 6
//   f1 = (multiplicity - 1) / 3
//   f2 = mean of f0 over the neighbours inside the subdomain (0 if none)
//   f3 = max of f0 over those neighbours (f0 if none)
//   f4 = (sum over the whole stored row of A) / A_pp
__global__ void k_node_features(const int* __restrict__ rp, const int* __restrict__ ci,
                                const double* __restrict__ a, const int* __restrict__ sub_ptr,
                                const int* __restrict__ sub_idx, const double* __restrict__ dvec,
                                double* F) {
    __shared__ double red[32];
    const int s = blockIdx.x;
    const int p0 = sub_ptr[s], m = sub_ptr[s + 1] - p0;
    const int* idx = sub_idx + p0;
    double part = 0.0;
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        const int i = idx[p];
        double dg = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; k++)
            if (ci[k] == i) dg = a[k];
        part += log10(dg);
    }
    const double mean = block_sum(part, red) / m;
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        const int i = idx[p];
        double dg = 0.0, rs = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; k++) {
            if (ci[k] == i) dg = a[k];
            rs += a[k];
        }
        double* f = F + (size_t)(p0 + p) * LN_F;
        f[0] = (log10(dg) - mean) / 6.0;
        f[1] = (1.0 / dvec[i] - 1.0) / 3.0;
        f[4] = rs / dg;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        const int i = idx[p];
        double sum = 0.0, mx = -INFINITY;
        int cnt = 0;
        for (int k = rp[i]; k < rp[i + 1]; k++) {
            const int j = ci[k];
            if (j == i) continue;
            const int q = bsearch_idx(idx, m, j);
            if (q < 0) continue;
            const double fq = F[(size_t)(p0 + q) * LN_F];
            sum += fq;
            mx = fmax(mx, fq);
            cnt++;
        }
        double* f = F + (size_t)(p0 + p) * LN_F;
        f[2] = cnt ? sum / cnt : 0.0;
        f[3] = cnt ? mx : f[0];
    }
}

// ----------------------------------------------------------------- network
template <typename T> __device__ __forceinline__ T act_tanh(T x);
template <> __device__ __forceinline__ float act_tanh<float>(float x) { return tanhf(x); }
template <> __device__ __forceinline__ double act_tanh<double>(double x) { return tanh(x); }
template <typename T> __device__ __forceinline__ T act_sigmoid(T x);
template <> __device__ __forceinline__ float act_sigmoid<float>(float x) { return 1.f / (1.f + expf(-x)); }
template <> __device__ __forceinline__ double act_sigmoid<double>(double x) { return 1.0 / (1.0 + exp(-x)); }

template <typename T>
struct Acts {
    T f[LN_F], a1[LN_H1], a2[LN_H2], out;
};

template <typename T>
__device__ __forceinline__ void mlp_fwd(const T* th, const double* frow, Acts<T>& z) {
    const T* W1 = th;
    const T* b1 = W1 + LN_H1 * LN_F;
    const T* W2 = b1 + LN_H1;
    const T* b2 = W2 + LN_H2 * LN_H1;
    const T* w3 = b2 + LN_H2;
    const T b3 = w3[LN_H2];
#pragma unroll
    for (int k = 0; k < LN_F; k++) z.f[k] = (T)frow[k];
#pragma unroll
    for (int j = 0; j < LN_H1; j++) {
        T s = b1[j];
#pragma unroll
        for (int k = 0; k < LN_F; k++) s += W1[j * LN_F + k] * z.f[k];
        z.a1[j] = act_tanh<T>(s);
    }
#pragma unroll
    for (int j = 0; j < LN_H2; j++) {
        T s = b2[j];
#pragma unroll
        for (int k = 0; k < LN_H1; k++) s += W2[j * LN_H1 + k] * z.a1[k];
        z.a2[j] = act_tanh<T>(s);
    }
    T s = b3;
#pragma unroll
    for (int k = 0; k < LN_H2; k++) s += w3[k] * z.a2[k];
    z.out = act_sigmoid<T>(s);
}

template <typename T>
__global__ void __launch_bounds__(256) k_mlp_forward(int P, const double* __restrict__ F,
                                                     const double* __restrict__ params, double* out) {
    __shared__ T th[LN_P];
    for (int k = threadIdx.x; k < LN_P; k += blockDim.x) th[k] = (T)params[k];
    __syncthreads();
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        Acts<T> z;
        mlp_fwd<T>(th, F + (size_t)p * LN_F, z);
        out[p] = (double)z.out;
    }
}

// Per-block partial gradient (and loss) of L = mean_p (out_p - t_p)^2:
// part[b * (LN_P + 1) + k], k < LN_P the gradient, k = LN_P the loss.
// Nodes are taken in tiles of LN_TILE: each thread runs forward and backward
// for one node and leaves its activations and deltas in shared memory; then
// each thread owns a few parameters and adds up their terms over the tile
// (every parameter's gradient is an outer-product sum over nodes) in a
// fixed order.
constexpr int LN_TILE = 128;
constexpr int LN_ROW = LN_F + LN_H1 + LN_H2 + LN_H1 + LN_H2 + 2;  // f, a1, a2, dz1, dz2, dz3, loss

template <typename T>
__global__ void __launch_bounds__(LN_TILE) k_mlp_grad(int P, const double* __restrict__ F,
                                                      const double* __restrict__ tgt,
                                                      const double* __restrict__ params,
                                                      double* part) {
    __shared__ T th[LN_P];
    extern __shared__ __align__(16) unsigned char ln_smem[];
    T* tile = reinterpret_cast<T*>(ln_smem);  // [LN_TILE][LN_ROW]
    for (int k = threadIdx.x; k < LN_P; k += blockDim.x) th[k] = (T)params[k];
    __syncthreads();
    const T* W2 = th + LN_H1 * LN_F + LN_H1;
    const T* w3 = W2 + LN_H2 * LN_H1 + LN_H2;
    constexpr int oF = 0, oA1 = LN_F, oA2 = oA1 + LN_H1, oD1 = oA2 + LN_H2, oD2 = oD1 + LN_H1,
                  oD3 = oD2 + LN_H2, oL = oD3 + 1;
    constexpr int PER = (LN_P + LN_TILE - 1) / LN_TILE;  // parameters per thread
    T acc[PER + 1];
#pragma unroll
    for (int u = 0; u <= PER; u++) acc[u] = 0;
    const T invP = (T)1 / (T)P;
    for (int base = blockIdx.x * LN_TILE; base < P; base += gridDim.x * LN_TILE) {
        T* row = tile + threadIdx.x * LN_ROW;
        const int p = base + threadIdx.x;
        if (p < P) {
            Acts<T> z;
            mlp_fwd<T>(th, F + (size_t)p * LN_F, z);
            const T err = z.out - (T)tgt[p];
            const T dz3 = (T)2 * err * invP * z.out * ((T)1 - z.out);
            T da1[LN_H1];
#pragma unroll
            for (int k = 0; k < LN_H1; k++) da1[k] = 0;
#pragma unroll
            for (int j = 0; j < LN_H2; j++) {
                const T dz2 = dz3 * w3[j] * ((T)1 - z.a2[j] * z.a2[j]);
                row[oD2 + j] = dz2;
#pragma unroll
                for (int k = 0; k < LN_H1; k++) da1[k] += dz2 * W2[j * LN_H1 + k];
            }
#pragma unroll
            for (int j = 0; j < LN_H1; j++) row[oD1 + j] = da1[j] * ((T)1 - z.a1[j] * z.a1[j]);
#pragma unroll
            for (int k = 0; k < LN_F; k++) row[oF + k] = z.f[k];
#pragma unroll
            for (int k = 0; k < LN_H1; k++) row[oA1 + k] = z.a1[k];
#pragma unroll
            for (int k = 0; k < LN_H2; k++) row[oA2 + k] = z.a2[k];
            row[oD3] = dz3;
            row[oL] = err * err * invP;
        } else {
            for (int k = 0; k < LN_ROW; k++) row[k] = 0;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PER; u++) {
            const int k = threadIdx.x + u * LN_TILE;
            if (k >= LN_P) continue;
            // parameter k: d(loss)/d(theta_k) = sum over the tile of delta * input
            int di, ii;  // offsets of the delta and of the input (-1: bias)
            if (k < LN_H1 * LN_F) { di = oD1 + k / LN_F; ii = oF + k % LN_F; }
            else if (k < LN_H1 * LN_F + LN_H1) { di = oD1 + (k - LN_H1 * LN_F); ii = -1; }
            else if (k < LN_H1 * LN_F + LN_H1 + LN_H2 * LN_H1) {
                const int q = k - LN_H1 * LN_F - LN_H1;
                di = oD2 + q / LN_H1; ii = oA1 + q % LN_H1;
            } else if (k < LN_H1 * LN_F + LN_H1 + LN_H2 * LN_H1 + LN_H2) {
                di = oD2 + (k - LN_H1 * LN_F - LN_H1 - LN_H2 * LN_H1); ii = -1;
            } else if (k < LN_P - 1) {
                di = oD3; ii = oA2 + (k - (LN_P - 1 - LN_H2));
            } else { di = oD3; ii = -1; }
            T s = 0;
            for (int nn = 0; nn < LN_TILE; nn++) {
                const T* r = tile + nn * LN_ROW;
                s += (ii >= 0) ? r[di] * r[ii] : r[di];
            }
            acc[u] += s;
        }
        if (threadIdx.x == 0) {
            T s = 0;
            for (int nn = 0; nn < LN_TILE; nn++) s += tile[nn * LN_ROW + oL];
            acc[PER] += s;
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < PER; u++) {
        const int k = threadIdx.x + u * LN_TILE;
        if (k < LN_P) part[(size_t)blockIdx.x * (LN_P + 1) + k] = (double)acc[u];
    }
    if (threadIdx.x == 0) part[(size_t)blockIdx.x * (LN_P + 1) + LN_P] = (double)acc[PER];
}

__global__ void k_grad_reduce(int nb, const double* __restrict__ part, double* g) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > LN_P) return;
    double v = 0.0;
    for (int b = 0; b < nb; b++) v += part[(size_t)b * (LN_P + 1) + k];
    g[k] = v;
}

// Adam (Kingma & Ba) on the float64 master parameters
__global__ void k_adam(int t, double lr, const double* __restrict__ g, double* th, double* m, double* v) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= LN_P) return;
    const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
    m[k] = b1 * m[k] + (1 - b1) * g[k];
    v[k] = b2 * v[k] + (1 - b2) * g[k] * g[k];
    const double mh = m[k] / (1 - pow(b1, (double)t)), vh = v[k] / (1 - pow(b2, (double)t));
    th[k] -= lr * mh / (sqrt(vh) + eps);
}

// -------------------------------------------------------------- targets
// Normalised leverage of the extra modes Y = Z_s(:, nu_s:m_s): g_p = ||Q_p||^2
// with Q = Y L^-T, L L^T = Y^T Y (Euclidean orthonormalisation), divided by
// its maximum; zero when the subdomain has no extra mode.  At most 16 extra
// modes per subdomain are used.
__global__ void k_leverage(const int* __restrict__ sub_ptr, const int* __restrict__ modes,
                           const int* __restrict__ nker, const int64_t* __restrict__ zoff,
                           const double* __restrict__ Z, double* tgt) {
    __shared__ double Gm[16][16];
    __shared__ double red[32];
    const int s = blockIdx.x;
    const int p0 = sub_ptr[s], m = sub_ptr[s + 1] - p0;
    const int nu = nker[s];
    const int e = min(16, modes[s] - nu);
    if (e <= 0) {
        for (int p = threadIdx.x; p < m; p += blockDim.x) tgt[p0 + p] = 0.0;
        return;
    }
    const double* Y = Z + zoff[s] + (size_t)nu * m;
    for (int a = 0; a < e; a++)
        for (int b = 0; b <= a; b++) {
            double part = 0.0;
            for (int p = threadIdx.x; p < m; p += blockDim.x) part += Y[p + (size_t)a * m] * Y[p + (size_t)b * m];
            const double v = block_sum(part, red);
            if (threadIdx.x == 0) Gm[a][b] = v;
        }
    __syncthreads();
    if (threadIdx.x == 0) {  // Cholesky then inverse of L, in place (lower)
        for (int j = 0; j < e; j++) {
            double d = Gm[j][j];
            for (int k = 0; k < j; k++) d -= Gm[j][k] * Gm[j][k];
            d = sqrt(fmax(d, 1e-300));
            Gm[j][j] = d;
            for (int i = j + 1; i < e; i++) {
                double v = Gm[i][j];
                for (int k = 0; k < j; k++) v -= Gm[i][k] * Gm[j][k];
                Gm[i][j] = v / d;
            }
        }
        for (int j = e - 1; j >= 0; j--) {  // L^-1, columns from last to first
            const double ljj = 1.0 / Gm[j][j];
            for (int i = e - 1; i > j; i--) {
                double v = 0.0;
                for (int k = j + 1; k <= i; k++) v += Gm[i][k] * Gm[k][j];
                Gm[i][j] = -ljj * v;
            }
            Gm[j][j] = ljj;
        }
    }
    __syncthreads();
    double mx = 0.0;
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        double g = 0.0;
        for (int c = 0; c < e; c++) {  // Q(p, c) = sum_k Y(p, k) Linv(c, k)
            double q = 0.0;
            for (int k = 0; k <= c; k++) q += Y[p + (size_t)k * m] * Gm[c][k];
            g += q * q;
        }
        tgt[p0 + p] = g;
        mx = fmax(mx, g);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t = fmax(t, red[w]);
        red[0] = t;
    }
    __syncthreads();
    const double inv = red[0] > 0.0 ? 1.0 / red[0] : 0.0;
    for (int p = threadIdx.x; p < m; p += blockDim.x) tgt[p0 + p] *= inv;
}

// ----------------------------------------------------------- start block
__device__ __forceinline__ double hash_unit(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t h = a * 0x9e3779b1u ^ (b + 0x7f4a7c15u) * 0x85ebca77u ^ (c + 0x165667b1u) * 0xc2b2ae3du;
    h ^= h >> 15; h *= 0x2c1b3c6du; h ^= h >> 12; h *= 0x297a2d39u; h ^= h >> 15;
    return ((double)(h & 0xffffff) / 16777216.0) * 2.0 - 1.0;
}

// X0_s (m x b, column-major at xoff[s]).  Without a prediction: uniform
// pseudo-random entries.  With one (g = predicted leverage in [0, 1]):
// column 0 = sqrt(g) + 1e-3 r, columns 1..b-2 = (sqrt(g) + 0.05) r, column
// b-1 = r (a plain random direction keeps the block general).
__global__ void k_start_block(const int* __restrict__ sub_ptr, const int64_t* __restrict__ xoff,
                              int b, const double* __restrict__ g, double* X0) {
    const int s = blockIdx.x;
    const int p0 = sub_ptr[s], m = sub_ptr[s + 1] - p0;
    double* X = X0 + xoff[s];
    for (int e = threadIdx.x; e < m * b; e += blockDim.x) {
        const int p = e % m, c = e / m;
        const double r = hash_unit((uint32_t)s, (uint32_t)p, (uint32_t)c);
        double v = r;
        if (g) {
            const double sg = sqrt(fmax(0.0, g[p0 + p]));
            if (c == 0) v = sg + 1e-3 * r;
            else if (c < b - 1) v = (sg + 0.05) * r;
        }
        X[e] = v;
    }
}

// ------------------------------------------------------------- host side
awg_status learned_features(Handle* h, double* d_F, cudaStream_t s) {
    k_node_features<<<h->N, 256, 0, s>>>((int*)h->rowptr.p, (int*)h->colidx.p, (double*)h->val.p,
                                         (int*)h->sub_ptr.p, (int*)h->sub_idx.p, (double*)h->dvec.p,
                                         d_F);
    AWG_LAUNCH();
    return AWG_OK;
}

awg_status learned_forward(int P, const double* d_F, const double* d_params, double* d_out, int prec,
                           cudaStream_t s) {
    const int grid = std::max(1, std::min((P + 255) / 256, 152 * 8));
    if (prec == AWG_FP64) k_mlp_forward<double><<<grid, 256, 0, s>>>(P, d_F, d_params, d_out);
    else k_mlp_forward<float><<<grid, 256, 0, s>>>(P, d_F, d_params, d_out);
    AWG_LAUNCH();
    return AWG_OK;
}

// grad (LN_P) and loss into d_g[0..LN_P]
awg_status learned_grad(int P, const double* d_F, const double* d_t, const double* d_params,
                        double* d_g, double* d_part, int nblocks, int prec, cudaStream_t s) {
    if (prec == AWG_FP64) {
        const int sm = LN_TILE * LN_ROW * 8;
        AWG_CUDA(cudaFuncSetAttribute(k_mlp_grad<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
        k_mlp_grad<double><<<nblocks, LN_TILE, sm, s>>>(P, d_F, d_t, d_params, d_part);
    } else {
        const int sm = LN_TILE * LN_ROW * 4;
        k_mlp_grad<float><<<nblocks, LN_TILE, sm, s>>>(P, d_F, d_t, d_params, d_part);
    }
    AWG_LAUNCH();
    k_grad_reduce<<<(LN_P + 1 + 255) / 256, 256, 0, s>>>(nblocks, d_part, d_g);
    AWG_LAUNCH();
    return AWG_OK;
}

awg_status learned_adam(int t, double lr, const double* d_g, double* d_th, double* d_m, double* d_v,
                        cudaStream_t s) {
    k_adam<<<(LN_P + 255) / 256, 256, 0, s>>>(t, lr, d_g, d_th, d_m, d_v);
    AWG_LAUNCH();
    return AWG_OK;
}

awg_status learned_targets(Handle* h, double* d_t, cudaStream_t s) {
    k_leverage<<<h->N, 256, 0, s>>>((int*)h->sub_ptr.p, (int*)h->modes.p, (int*)h->nm.p,
                                    (int64_t*)h->z_off.p, (double*)h->Z.p, d_t);
    AWG_LAUNCH();
    return AWG_OK;
}

awg_status learned_start_block(Handle* h, const int64_t* d_xoff, int b, const double* d_g, double* d_X0,
                               cudaStream_t s) {
    k_start_block<<<h->N, 256, 0, s>>>((int*)h->sub_ptr.p, d_xoff, b, d_g, d_X0);
    AWG_LAUNCH();
    return AWG_OK;
}

}  // namespace awg

// ------------------------------------------------------------------ C ABI
using namespace awg;

namespace {
int grad_blocks(int P) { return std::max(1, std::min((P + LN_TILE - 1) / LN_TILE, 152 * 4)); }
bool prec_ok(int p) { return p == AWG_FP64 || p == AWG_MIXED_FP32; }
}  // namespace

extern "C" {

awg_status awg_learned_data(awg_handle hh, double* d_features, double* d_targets, void* stream) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return AWG_ERR_INVALID_ARG;
    if (!h->Z.p) return AWG_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    if (d_features) AWG_TRY(learned_features(h, d_features, s));
    if (d_targets) AWG_TRY(learned_targets(h, d_targets, s));
    return AWG_OK;
}

awg_status awg_learned_forward(int P, const double* d_features, const double* d_params, double* d_out,
                               int precision, void* stream) {
    if (P < 0 || (P > 0 && (!d_features || !d_params || !d_out)) || !prec_ok(precision))
        return AWG_ERR_INVALID_ARG;
    if (P == 0) return AWG_OK;
    return learned_forward(P, d_features, d_params, d_out, precision, (cudaStream_t)stream);
}

awg_status awg_learned_grad(int P, const double* d_features, const double* d_targets,
                            const double* d_params, double* d_grad, int precision, void* stream) {
    if (P < 1 || !d_features || !d_targets || !d_params || !d_grad || !prec_ok(precision))
        return AWG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = grad_blocks(P);
    double* part = nullptr;
    AWG_CUDA(cudaMallocAsync(&part, (size_t)nb * (LN_P + 1) * 8, s));
    const awg_status st = learned_grad(P, d_features, d_targets, d_params, d_grad, part, nb, precision, s);
    AWG_CUDA(cudaFreeAsync(part, s));
    return st;
}

awg_status awg_learned_train(int P, const double* d_features, const double* d_targets, double* h_params,
                             int steps, double lr, int precision, double* h_loss, void* stream) {
    if (P < 1 || !d_features || !d_targets || !h_params || steps < 0 || !(lr > 0.0) || !prec_ok(precision))
        return AWG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = grad_blocks(P);
    // th | m | v | g (P+1) | loss[steps] | partial sums
    const size_t nbuf = 3 * LN_P + (LN_P + 1) + (size_t)std::max(steps, 1) + (size_t)nb * (LN_P + 1);
    double* buf = nullptr;
    AWG_CUDA(cudaMallocAsync(&buf, nbuf * 8, s));
    double *th = buf, *m = th + LN_P, *v = m + LN_P, *g = v + LN_P, *loss = g + LN_P + 1,
           *part = loss + std::max(steps, 1);
    awg_status st = AWG_OK;
    do {
        if (cudaMemcpyAsync(th, h_params, LN_P * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(m, 0, 2 * LN_P * 8, s) != cudaSuccess) {
            st = AWG_ERR_CUDA;
            break;
        }
        for (int t = 0; t < steps && st == AWG_OK; t++) {
            st = learned_grad(P, d_features, d_targets, th, g, part, nb, precision, s);
            if (st != AWG_OK) break;
            if (cudaMemcpyAsync(loss + t, g + LN_P, 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
                st = AWG_ERR_CUDA;
                break;
            }
            st = learned_adam(t + 1, lr, g, th, m, v, s);
        }
        if (st != AWG_OK) break;
        if (cudaMemcpyAsync(h_params, th, LN_P * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            (h_loss && steps > 0 &&
             cudaMemcpyAsync(h_loss, loss, (size_t)steps * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = AWG_ERR_CUDA;
    } while (0);
    cudaFreeAsync(buf, s);
    cudaStreamSynchronize(s);
    return st;
}

}  // extern "C"
