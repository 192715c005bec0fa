// awg_apply_hnn_noalloc: the one-level apply y = H^NN x (batched local
// pseudo-inverse GEMVs, then the prolongation sum) without any device
// allocation.
//
// Who needs it: callers that may not call cudaMalloc while they run the
// preconditioner.  A host framework that hands all device memory out of its
// own pool forbids libraries to allocate behind its back; a real-time or
// latency-bound loop cannot afford cudaMalloc / cudaFree, which may
// synchronise the device and take unbounded time.  The regular entry points
// keep their scratch in the handle's workspace, allocated by the handle;
// this variant keeps its scratch (the per-subdomain local results, sum of
// n^s float64 values) in a fixed array that the library defines at file
// scope instead, and calls no allocating routine at all.
//
// The array is a static __device__ buffer of AWG_NOALLOC_MAX_LOCAL doubles
// (8 MiB): every GPU on which the library is loaded holds it until the
// process exits.  Host code must not use its name as a device address (on
// the host the name only stands in for the symbol); the first call on each
// device looks the address up with cudaGetSymbolAddress, with that device
// current, and caches it.  That first call should therefore come before any
// stream capture.  All calls share the array and it keeps the last call's
// contents: every element a call reads has been written earlier in the same
// call, so nothing needs clearing, but two calls that overlap on the GPU
// (different streams, or different host threads) race on it.

#include "awg_common.cuh"

#include <mutex>

namespace awg {

static constexpr int64_t NOALLOC_MAX_LOCAL = AWG_NOALLOC_MAX_LOCAL;
static __device__ __align__(256) double g_noalloc_local[NOALLOC_MAX_LOCAL];

static std::mutex g_noalloc_mutex;
static double* g_noalloc_ptr[256] = {nullptr};

// loc[sub_ptr[s] + p] = sum_q G_s(p, q) x(idx_s(q)) for the rows of this
// block (G_s symmetric, full column-major, stored as TS; float32 blocks have
// their leading dimension rounded up to 4)
template <typename TS, typename TA>
__global__ void __launch_bounds__(256) k_hnn_local_noalloc(const int* __restrict__ sub_ptr,
                                                           const int* __restrict__ sub_idx,
                                                           const int64_t* __restrict__ goff,
                                                           const TS* __restrict__ G,
                                                           const double* __restrict__ x,
                                                           double* loc, int rows_per_block) {
    extern __shared__ __align__(16) unsigned char na_smem[];
    TA* xs = reinterpret_cast<TA*>(na_smem);
    const int s = blockIdx.x;
    const int p0 = sub_ptr[s], m = sub_ptr[s + 1] - p0;
    const int r0 = blockIdx.y * rows_per_block;
    if (r0 >= m) return;
    for (int q = threadIdx.x; q < m; q += blockDim.x) xs[q] = (TA)x[sub_idx[p0 + q]];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const TS* Gs = G + goff[s];
    const int ld = (sizeof(TS) == 4) ? ((m + 3) & ~3) : m;
    const int r1 = min(m, r0 + rows_per_block);
    for (int p = r0 + wid; p < r1; p += nw) {
        const TS* col = Gs + (size_t)p * ld;
        TA acc = 0;
        for (int q = lane; q < m; q += 32) acc = fma((TA)col[q], xs[q], acc);
        double a = (double)acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) loc[p0 + p] = a;
    }
}

// y(i) = sum over the copies of dof i of loc
__global__ void k_hnn_prolong_noalloc(int n, const int* __restrict__ inc_ptr,
                                      const int* __restrict__ inc_pos,
                                      const double* __restrict__ loc, double* y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int e = inc_ptr[i]; e < inc_ptr[i + 1]; e++) acc += loc[inc_pos[e]];
    y[i] = acc;
}

// Device address of the static scratch for the current device (looked up
// once per device, with that device current).
static awg_status noalloc_scratch(double** out) {
    int dev = 0;
    AWG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return AWG_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        AWG_CUDA(cudaGetSymbolAddress(&p, g_noalloc_local));
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return AWG_OK;
}

}  // namespace awg

using namespace awg;

extern "C" awg_status awg_apply_hnn_noalloc(awg_handle hh, int precision, const double* d_x,
                                            double* d_y, void* stream) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !d_x || !d_y || (precision != AWG_FP64 && precision != AWG_MIXED_FP32))
        return AWG_ERR_INVALID_ARG;
    if (h->sum_ns > NOALLOC_MAX_LOCAL) {
        fprintf(stderr,
                "libawg: awg_apply_hnn_noalloc: the subdomains hold %lld values, more than the "
                "%lld of the static scratch\n",
                (long long)h->sum_ns, (long long)NOALLOC_MAX_LOCAL);
        return AWG_ERR_INVALID_ARG;
    }
    const PrecOps& P = h->prec[precision];
    if (!P.G.p) return AWG_ERR_STATE;
    // the handle's arrays must live on the current device
    cudaPointerAttributes attr;
    AWG_CUDA(cudaPointerGetAttributes(&attr, h->val.p));
    int dev = 0;
    AWG_CUDA(cudaGetDevice(&dev));
    if (attr.device != dev) return AWG_ERR_INVALID_ARG;
    double* loc = nullptr;
    AWG_TRY(noalloc_scratch(&loc));
    cudaStream_t s = (cudaStream_t)stream;
    const int rows = 32;
    dim3 g(h->N, (h->max_ns + rows - 1) / rows);
    if (precision == AWG_FP64) {
        const size_t sm = (size_t)h->max_ns * 8;
        if (sm > 48 * 1024)
            AWG_CUDA(cudaFuncSetAttribute(k_hnn_local_noalloc<double, double>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_hnn_local_noalloc<double, double><<<g, 256, sm, s>>>(
            (int*)h->sub_ptr.p, (int*)h->sub_idx.p, (int64_t*)h->dense_off.p, (const double*)P.G.p,
            d_x, loc, rows);
    } else {
        const size_t sm = (size_t)h->max_ns * 4;
        if (sm > 48 * 1024)
            AWG_CUDA(cudaFuncSetAttribute(k_hnn_local_noalloc<float, float>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_hnn_local_noalloc<float, float><<<g, 256, sm, s>>>(
            (int*)h->sub_ptr.p, (int*)h->sub_idx.p, (int64_t*)h->g32_off.p, (const float*)P.G.p,
            d_x, loc, rows);
    }
    AWG_LAUNCH();
    k_hnn_prolong_noalloc<<<(h->n + 255) / 256, 256, 0, s>>>(h->n, (int*)h->inc_ptr.p,
                                                            (int*)h->inc_pos.p, loc, d_y);
    AWG_LAUNCH();
    return AWG_OK;
}
