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
constexpr uint32_t kVersion = 1;
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
                          &P.corr_val, &P.corr_colptr, &P.corr_row, &P.corr_cval})
            b.push_back(d);
    return b;
}

// the tables agree with the scalars (a file from another build or a
// damaged one is refused before any device work)
bool consistent(const Handle& h) {
    const size_t N = (size_t)h.N;
    return h.n >= 1 && h.nnz >= h.n && h.N >= 1 && h.N <= h.n && h.n0 >= 0 && h.n_minus >= 0 &&
           h.ldw >= h.n_minus && h.max_ns >= 1 && h.h_ns.size() == N && h.h_sub_ptr.size() == N + 1 &&
           h.h_dense_off.size() == N + 1 && h.h_nm.size() == N && h.h_nstrict.size() == N &&
           h.h_nm_ptr.size() == N + 1 && h.h_vm_off.size() == N + 1 && h.h_modes.size() == N &&
           h.h_mode_ptr.size() == N + 1 && h.h_z_off.size() == N + 1 && h.h_wcol_ptr.size() == N + 1 &&
           (h.h_g32_off.empty() || h.h_g32_off.size() == N + 1) && h.h_mode_ptr[N] == h.n0 &&
           h.h_wcol_ptr[N] == h.n_minus && h.h_sub_ptr[N] == h.sum_ns && h.h_dense_off[N] == h.dense_total;
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

awg_status load_buffer(In& in, Handle* h, DevBuf& b, std::vector<char>& stage) {
    uint64_t n = 0;
    in.pod(n);
    if (!in.ok || n > ((uint64_t)1 << 42)) return AWG_ERR_IO;
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
    h->stream = (cudaStream_t)stream;
    AWG_TRY(runtime_init(h));
    std::vector<char> stage;
    for (DevBuf* b : buffers(*h)) AWG_TRY(load_buffer(in, h, *b, stage));
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
