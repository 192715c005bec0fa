// Checkpoint of a set-up handle (awg_save / awg_load): what the setup
// computed is written to a file and read back into a new handle, so that a
// later process skips the setup (its eigenproblems and the n_- solves of W
// are the expensive part).  Host code only: file I/O and plain copies.
//
// File: an 8-byte tag, the format version and sizeof(awg_options), then the
// scalar fields, the host tables (element count + elements) and the device
// buffers (byte count + bytes), each in the fixed order of the visitors
// below.  What the handle builds on first use (block-path copies, tensor-core
// tiles, loop graphs, workspaces) is not stored.

#include "awg_common.cuh"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

namespace awg {

size_t ws_bytes(const Handle* h);
awg_status set_smem_limits(Handle* h);

namespace {

constexpr char kTag[8] = {'A', 'W', 'G', 'H', 'N', 'D', 'L', '\n'};
constexpr uint32_t kVersion = 2;
constexpr size_t kChunk = (size_t)64 << 20;  // host staging of the device copies

struct Out {
    FILE* f;
    bool ok = true;
    void bytes(const void* p, size_t n) {
        if (ok && n && std::fwrite(p, 1, n, f) != n) ok = false;
    }
    template <class T>
    void pod(const T& v) { bytes(&v, sizeof(T)); }
    template <class T>
    void vec(const std::vector<T>& v) {
        const uint64_t c = v.size();
        pod(c);
        bytes(v.data(), c * sizeof(T));
    }
};

struct In {
    FILE* f;
    bool ok = true;
    void bytes(void* p, size_t n) {
        if (ok && n && std::fread(p, 1, n, f) != n) ok = false;
    }
    template <class T>
    void pod(T& v) { bytes(&v, sizeof(T)); }
    template <class T>
    void vec(std::vector<T>& v) {
        uint64_t c = 0;
        pod(c);
        if (!ok || c > ((uint64_t)1 << 36) / sizeof(T)) {
            ok = false;
            return;
        }
        v.resize(c);
        bytes(v.data(), c * sizeof(T));
    }
};

// scalar fields, in file order (IO = Out or In)
template <class IO>
void scalars(IO& io, Handle& h) {
    io.pod(h.n);
    io.pod(h.nnz);
    io.pod(h.N);
    io.pod(h.overlap);
    io.pod(h.tau);
    io.pod(h.opt);
    io.pod(h.sum_ns);
    io.pod(h.max_ns);
    io.pod(h.dense_total);
    io.pod(h.n_minus_all);
    io.pod(h.n0);
    io.pod(h.n_minus);
    io.pod(h.ldw);
    io.pod(h.geneo_its_max);
    io.pod(h.geneo_its_sum);
    io.pod(h.geneo_dense);
    io.pod(h.w_iters);
    io.pod(h.w_relres);
    io.pod(h.setup_ms);
    io.pod(h.red_blocks);
    io.pod(h.bt_wt);
    io.pod(h.bt_dense);
    for (PrecOps& P : h.prec) {
        io.pod(P.built);
        io.pod(P.corr_nnz);
        io.pod(P.wt_blocks);
        io.pod(P.wd_blocks);
        io.pod(P.sp_nnz);
    }
}

// host copies of the per-subdomain tables, in file order
template <class IO>
void tables(IO& io, Handle& h) {
    io.vec(h.h_ns);
    io.vec(h.h_sub_ptr);
    io.vec(h.h_dense_off);
    io.vec(h.h_g32_off);
    io.vec(h.h_nm);
    io.vec(h.h_nstrict);
    io.vec(h.h_nm_ptr);
    io.vec(h.h_vm_off);
    io.vec(h.h_modes);
    io.vec(h.h_mode_ptr);
    io.vec(h.h_z_off);
    io.vec(h.h_wcol_ptr);
}

// device buffers that hold setup results, in file order
std::vector<DevBuf*> buffers(Handle& h) {
    std::vector<DevBuf*> b = {&h.rowptr,  &h.colidx,   &h.val,    &h.ns,     &h.sub_ptr, &h.sub_idx, &h.inc_ptr,
                              &h.inc_pos, &h.inc_sub,  &h.pos_sub, &h.dvec,  &h.mmu,     &h.bval,    &h.dense_off,
                              &h.g32_off, &h.nm,       &h.nstrict, &h.nm_ptr, &h.vm_off, &h.Vm,      &h.lam_m,
                              &h.sigma,   &h.modes,    &h.mode_ptr, &h.z_off, &h.Z,      &h.E,       &h.Einv,
                              &h.wcol_ptr, &h.Wcm,     &h.F64};
    for (PrecOps& P : h.prec)
        for (DevBuf* d : {&P.G, &P.W, &P.Finv, &P.inexInv, &P.rscale, &P.cscale, &P.corr_rowptr, &P.corr_col,
                          &P.corr_val, &P.corr_colptr, &P.corr_row, &P.corr_cval, &P.sp_rowptr, &P.sp_col,
                          &P.sp_val, &P.sp_colptr, &P.sp_row, &P.sp_cval})
            b.push_back(d);
    return b;
}

template <class T>
bool nondecreasing(const std::vector<T>& v) {
    if (v.empty() || v[0] != 0) return false;
    for (size_t i = 1; i < v.size(); i++)
        if (v[i] < v[i - 1]) return false;
    return true;
}

// the tables agree with the scalars and with each other (a file from another
// build or a damaged one is refused before any device work): every prefix
// table starts at 0 and never decreases, its steps are the per-subdomain
// sizes it is built from, and every n^s lies in [1, max_ns]
bool consistent(const Handle& h) {
    const size_t N = (size_t)h.N;
    if (!(h.n >= 1 && h.nnz >= h.n && h.N >= 1 && h.N <= h.n && h.n0 >= 0 && h.n_minus >= 0 &&
          h.n_minus_all >= h.n_minus && h.ldw >= h.n_minus && h.ldw % 8 == 0 && h.max_ns >= 1 &&
          h.max_ns <= h.n && h.h_ns.size() == N && h.h_sub_ptr.size() == N + 1 && h.h_dense_off.size() == N + 1 &&
          h.h_nm.size() == N && h.h_nstrict.size() == N && h.h_nm_ptr.size() == N + 1 &&
          h.h_vm_off.size() == N + 1 && h.h_modes.size() == N && h.h_mode_ptr.size() == N + 1 &&
          h.h_z_off.size() == N + 1 && h.h_wcol_ptr.size() == N + 1 &&
          (h.h_g32_off.empty() || h.h_g32_off.size() == N + 1)))
        return false;
    for (const auto* v : {&h.h_sub_ptr, &h.h_nm_ptr, &h.h_mode_ptr, &h.h_wcol_ptr})
        if (!nondecreasing(*v)) return false;
    for (const auto* v : {&h.h_dense_off, &h.h_vm_off, &h.h_z_off})
        if (!nondecreasing(*v)) return false;
    if (!h.h_g32_off.empty() && !nondecreasing(h.h_g32_off)) return false;
    int mx = 0;
    for (size_t t = 0; t < N; t++) {
        const int64_t m = h.h_ns[t];
        if (m < 1 || m > h.max_ns || h.h_sub_ptr[t + 1] - h.h_sub_ptr[t] != m) return false;
        if (h.h_dense_off[t + 1] - h.h_dense_off[t] != m * m) return false;
        if (!h.h_g32_off.empty() && h.h_g32_off[t + 1] - h.h_g32_off[t] != m * ((m + 3) & ~3)) return false;
        if (h.h_nm[t] < 0 || h.h_nm[t] > m || h.h_nm_ptr[t + 1] - h.h_nm_ptr[t] != h.h_nm[t]) return false;
        if (h.h_vm_off[t + 1] - h.h_vm_off[t] != m * h.h_nm[t]) return false;
        if (h.h_nstrict[t] < 0 || h.h_nstrict[t] > h.h_nm[t] ||
            h.h_wcol_ptr[t + 1] - h.h_wcol_ptr[t] != h.h_nstrict[t])
            return false;
        if (h.h_modes[t] < 0 || h.h_mode_ptr[t + 1] - h.h_mode_ptr[t] != h.h_modes[t]) return false;
        if (h.h_z_off[t + 1] - h.h_z_off[t] != m * h.h_modes[t]) return false;
        mx = std::max(mx, (int)m);
    }
    return mx == h.max_ns && h.h_mode_ptr[N] == h.n0 && h.h_wcol_ptr[N] == h.n_minus &&
           h.h_nm_ptr[N] == h.n_minus_all && h.h_sub_ptr[N] == h.sum_ns && h.h_dense_off[N] == h.dense_total;
}

// Smallest byte count of each device buffer (in the order of buffers()) that
// the kernels can index given the scalars and tables: `need` bytes, or, for
// a buffer that may be absent (a storage form not built, the H_3,inex
// matrix), 0 or at least `need`.
struct Need {
    uint64_t need;
    bool optional;
};
std::vector<Need> needs(const Handle& h) {
    const uint64_t n = h.n, nnz = h.nnz, N = h.N, S = (uint64_t)h.sum_ns, n0 = h.n0, nm = h.n_minus;
    const uint64_t ldw = h.ldw, N1 = N + 1;
    std::vector<Need> r = {
        {(n + 1) * 4, false}, {nnz * 4, false}, {nnz * 8, false}, {N * 4, false}, {N1 * 4, false},
        {S * 4, false}, {(n + 1) * 4, false}, {S * 4, false}, {S * 4, false}, {S * 4, false},
        {n * 8, false}, {nnz * 8, false}, {nnz * 8, false}, {N1 * 8, false},
        {h.h_g32_off.empty() ? 0 : N1 * 8, h.h_g32_off.empty()}, {N * 4, false}, {N * 4, false}, {N1 * 4, false},
        {N1 * 8, false}, {(uint64_t)h.h_vm_off[N] * 8, h.h_vm_off[N] == 0}, {(uint64_t)h.n_minus_all * 8, h.n_minus_all == 0},
        {N * 8, false}, {N * 4, false}, {N1 * 4, false}, {N1 * 8, false}, {(uint64_t)h.h_z_off[N] * 8, h.h_z_off[N] == 0},
        {n0 * n0 * 8, n0 == 0}, {n0 * n0 * 8, n0 == 0}, {N1 * 4, false}, {n * nm * 8, true},
        {nm * nm * 8, nm == 0}};
    for (int p = 0; p < AWG_NPREC; p++) {
        const PrecOps& P = h.prec[p];
        const bool b = P.built;
        const uint64_t w = p == AWG_FP64 ? 8 : (p == AWG_MIXED_FP32 ? 4 : 2);
        const uint64_t g = p == AWG_FP64 ? (uint64_t)h.dense_total * 8
                                         : (p == AWG_MIXED_FP32 && !h.h_g32_off.empty() ? (uint64_t)h.h_g32_off[N] * 4
                                                                                        : 0);
        const uint64_t cn = (uint64_t)std::max<int64_t>(0, P.corr_nnz);
        const uint64_t sn = (uint64_t)std::max<int64_t>(0, P.sp_nnz);
        const bool sparse = p == AWG_FP64 && sn > 0;
        r.push_back({g, !(b && p == AWG_FP64)});                          // G
        r.push_back({n * ldw * w, !(b && nm > 0 && !sparse)});           // W (absent when truncated)
        r.push_back({nm * nm * 8, !(b && nm > 0)});                      // Finv
        r.push_back({nm * nm * 8, true});                                // inexInv
        r.push_back({p == AWG_MIXED_FP16 ? n * 4 : 0, !(b && p == AWG_MIXED_FP16 && nm > 0)});    // rscale
        r.push_back({p == AWG_MIXED_FP16 ? ldw * 4 : 0, !(b && p == AWG_MIXED_FP16 && nm > 0)});  // cscale
        r.push_back({cn ? (n + 1) * 4 : 0, cn == 0});                   // corr_rowptr
        r.push_back({cn * 4, cn == 0});                                  // corr_col
        r.push_back({cn * 4, cn == 0});                                  // corr_val
        r.push_back({cn ? (nm + 1) * 4 : 0, cn == 0});                  // corr_colptr
        r.push_back({cn * 4, cn == 0});                                  // corr_row
        r.push_back({cn * 4, cn == 0});                                  // corr_cval
        r.push_back({sparse ? (n + 1) * 8 : 0, !sparse});                // sp_rowptr
        r.push_back({sn * 4, !sparse});                                  // sp_col
        r.push_back({sn * 8, !sparse});                                  // sp_val
        r.push_back({sparse ? (nm + 1) * 8 : 0, !sparse});               // sp_colptr
        r.push_back({sn * 4, !sparse});                                  // sp_row
        r.push_back({sn * 8, !sparse});                                  // sp_cval
    }
    return r;
}

awg_status save_buffer(Out& o, const DevBuf& b, std::vector<char>& stage) {
    const uint64_t n = b.p ? b.bytes : 0;
    o.pod(n);
    for (uint64_t off = 0; off < n && o.ok; off += kChunk) {
        const size_t len = (size_t)std::min<uint64_t>(kChunk, n - off);
        AWG_CUDA(cudaMemcpy(stage.data(), (const char*)b.p + off, len, cudaMemcpyDeviceToHost));
        o.bytes(stage.data(), len);
    }
    return AWG_OK;
}

awg_status load_buffer(In& in, Handle* h, DevBuf& b, const Need& need, std::vector<char>& stage) {
    uint64_t n = 0;
    in.pod(n);
    if (!in.ok || n > ((uint64_t)1 << 42)) return AWG_ERR_IO;
    // fewer bytes than the tables imply would let the kernels read past the buffer
    if (n == 0 ? !need.optional && need.need > 0 : n < need.need) return AWG_ERR_IO;
    if (n == 0) return AWG_OK;
    AWG_TRY(dalloc(h, b, (size_t)n));
    if (stage.size() < std::min<uint64_t>(kChunk, n)) stage.resize((size_t)std::min<uint64_t>(kChunk, n));
    for (uint64_t off = 0; off < n; off += kChunk) {
        const size_t len = (size_t)std::min<uint64_t>(kChunk, n - off);
        in.bytes(stage.data(), len);
        if (!in.ok) return AWG_ERR_IO;
        AWG_CUDA(cudaMemcpy((char*)b.p + off, stage.data(), len, cudaMemcpyHostToDevice));
    }
    return AWG_OK;
}

awg_status load_into(In& in, Handle* h, void* stream) {
    scalars(in, *h);
    h->opt.learned_params = nullptr;  // a pointer of the writing process
    tables(in, *h);
    if (!in.ok || !consistent(*h)) return AWG_ERR_IO;
    if (h->opt.coarse_tensor_cores < 0 || h->opt.coarse_tensor_cores > 1) return AWG_ERR_IO;
    h->stream = (cudaStream_t)stream;
    AWG_TRY(runtime_init(h));
    std::vector<char> stage;
    const std::vector<DevBuf*> bufs = buffers(*h);
    const std::vector<Need> need = needs(*h);
    if (bufs.size() != need.size()) return AWG_ERR_IO;
    for (size_t i = 0; i < bufs.size(); i++) AWG_TRY(load_buffer(in, h, *bufs[i], need[i], stage));
    // single right-hand-side workspace (its ticket counters start at zero)
    AWG_TRY(dalloc(h, h->ws, ws_bytes(h)));
    AWG_CUDA(cudaMemsetAsync(h->ws.p, 0, ws_bytes(h), h->stream));
    AWG_TRY(set_smem_limits(h));
    AWG_CUDA(cudaStreamSynchronize(h->stream));
    return AWG_OK;
}

}  // namespace

}  // namespace awg

using namespace awg;

extern "C" {

awg_status awg_save(awg_handle hh, const char* path) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h || !path) return AWG_ERR_INVALID_ARG;
    AWG_CUDA(cudaStreamSynchronize(h->stream));
    for (cudaStream_t s : {h->hp, h->side, h->hp2, h->side2})
        if (s) AWG_CUDA(cudaStreamSynchronize(s));
    FILE* f = std::fopen(path, "wb");
    if (!f) return AWG_ERR_IO;
    Out o{f};
    o.bytes(kTag, sizeof(kTag));
    o.pod(kVersion);
    const uint32_t osz = sizeof(awg_options);
    o.pod(osz);
    scalars(o, *h);
    tables(o, *h);
    size_t largest = 0;
    for (DevBuf* b : buffers(*h)) largest = std::max(largest, b->p ? b->bytes : 0);
    std::vector<char> stage(std::min(kChunk, std::max<size_t>(largest, 1)));
    awg_status st = AWG_OK;
    for (DevBuf* b : buffers(*h)) {
        st = save_buffer(o, *b, stage);
        if (st != AWG_OK || !o.ok) break;
    }
    if (std::fclose(f) != 0) o.ok = false;
    if (st != AWG_OK) return st;
    return o.ok ? AWG_OK : AWG_ERR_IO;
}

awg_status awg_load(const char* path, void* stream, awg_handle* out) {
    if (!out) return AWG_ERR_INVALID_ARG;
    *out = nullptr;
    if (!path) return AWG_ERR_INVALID_ARG;
    FILE* f = std::fopen(path, "rb");
    if (!f) return AWG_ERR_IO;
    In in{f};
    char tag[sizeof(kTag)] = {};
    uint32_t ver = 0, osz = 0;
    in.bytes(tag, sizeof(tag));
    in.pod(ver);
    in.pod(osz);
    if (!in.ok || std::memcmp(tag, kTag, sizeof(kTag)) != 0 || ver != kVersion || osz != sizeof(awg_options)) {
        std::fclose(f);
        return AWG_ERR_IO;
    }
    Handle* h = new (std::nothrow) Handle();
    if (!h) {
        std::fclose(f);
        return AWG_ERR_OOM;
    }
    const awg_status st = load_into(in, h, stream);
    std::fclose(f);
    if (st != AWG_OK) {
        if (h->hp) cudaStreamSynchronize(h->stream);
        free_all(h);
        delete h;
        return st;
    }
    *out = reinterpret_cast<awg_handle>(h);
    return AWG_OK;
}

}  // extern "C"
