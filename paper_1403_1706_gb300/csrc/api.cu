// The C ABI (include/peanut.h): argument checks, object lifetimes, errors, device memory.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "internal.cuh"

namespace pn {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

static std::atomic<unsigned long long> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static peanut_alloc_fn g_alloc = nullptr;
static peanut_release_fn g_release = nullptr;
static void* g_ctx = nullptr;

// Threads that allocate from CUDA's stream-ordered pool whatever provider is installed (an
// engine's executors and I/O thread: a provider may call back into an interpreter, which would
// serialize them).
static thread_local bool t_pool_only = false;
void use_pool_on_this_thread() { t_pool_only = true; }
bool pool_on_this_thread() { return t_pool_only; }

// Threads whose map calls run their sync-free stretches as CUDA graphs (engine executors whose
// engine was created with graphs = 1; they allocate from the stream-ordered pool).
static thread_local bool t_graphs = false;
void use_graphs_on_this_thread(bool on) { t_graphs = on; }
bool graphs_on_this_thread() { return t_graphs && t_pool_only; }

Allocator current_allocator() {
    return t_pool_only ? Allocator{} : Allocator{g_alloc, g_release, g_ctx};
}

// Keep memory freed to the process's default CUDA memory pool cached for reuse (release threshold
// raised once per device), so per-batch temporaries are not returned to the driver and re-mapped
// at every stream synchronization.
static void retain_pool_memory() {
    static std::atomic<bool> done[256];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256 || done[dev].load()) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done[dev].store(true);
}

void* dalloc(size_t bytes, cudaStream_t s, Allocator* used) {
    void* p = nullptr;
    if (bytes == 0) bytes = 1;
    if (used) *used = current_allocator();
    if (g_alloc && !t_pool_only) {
        p = g_alloc(bytes, (void*)s, g_ctx);
        if (!p) {
            set_error("device allocation of %zu bytes failed (external allocator)", bytes);
            throw Fail{PEANUT_NO_MEMORY};
        }
        return p;
    }
    retain_pool_memory();
    const cudaError_t e = cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        throw Fail{PEANUT_NO_MEMORY};
    }
    return p;
}

void dfree(void* p, cudaStream_t s, const Allocator& a) {
    if (!p) return;
    if (a.release) {
        a.release(p, (void*)s, a.ctx);
        return;
    }
    if (cudaFreeAsync(p, s) != cudaSuccess) cudaGetLastError();  // never leave a stale error behind
}

int sm_count() {  // of the current device, looked up once per device (any thread)
    static std::atomic<int> cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n <= 0) {
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cudaGetLastError();
        if (n <= 0) n = 1;
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

void free_device_hits(DeviceHits* H);

// Result arrays live in page-locked host blocks so the device-to-host copy runs at link speed.
// Freed blocks are kept (up to kPinnedKeep bytes) and reused by later calls of similar size.
static std::mutex g_pin_mu;
static std::multimap<size_t, void*> g_pin_free;
static size_t g_pin_kept = 0;
static std::atomic<uint64_t> g_pageable_blocks{0};  // result blocks that could not be page-locked
constexpr size_t kPinnedKeep = 8ull << 30;

void* host_block_alloc(size_t bytes, size_t* got, bool* pinned) {
    if (bytes == 0) bytes = 1;
    {
        std::lock_guard<std::mutex> lock(g_pin_mu);
        auto it = g_pin_free.lower_bound(bytes);
        if (it != g_pin_free.end() && it->first <= 2 * bytes + (64u << 20)) {
            void* p = it->second;
            *got = it->first;
            g_pin_kept -= it->first;
            g_pin_free.erase(it);
            *pinned = true;
            return p;
        }
    }
    const size_t want = ((bytes + (1u << 20) - 1) >> 20) << 20;
    void* p = nullptr;
    if (cudaHostAlloc(&p, want, cudaHostAllocDefault) == cudaSuccess) {
        *got = want;
        *pinned = true;
        return p;
    }
    cudaGetLastError();
    g_pageable_blocks.fetch_add(1, std::memory_order_relaxed);
    p = malloc(bytes);
    *got = bytes;
    *pinned = false;
    return p;
}

uint64_t pageable_blocks() { return g_pageable_blocks.load(); }

void host_block_free(void* p, size_t bytes, bool pinned) {
    if (!p) return;
    if (!pinned) {
        free(p);
        return;
    }
    std::lock_guard<std::mutex> lock(g_pin_mu);
    if (g_pin_kept + bytes <= kPinnedKeep) {
        g_pin_free.emplace(bytes, p);
        g_pin_kept += bytes;
    } else {
        cudaFreeHost(p);
    }
}

HostHits* download_hits(const peanut_device_hits& dh, cudaStream_t s) {
    HostHits* H = new HostHits();
    const uint64_t n = dh.n;
    H->h.n = n;
    const uint64_t c = n ? n : 1;
    // one block: end_pos (8-byte aligned first), read_id, strand, dist
    const size_t bytes = c * (sizeof(uint64_t) + sizeof(uint32_t) + 2);
    H->block = host_block_alloc(bytes, &H->block_bytes, &H->pinned);
    if (!H->block) {
        delete H;
        set_error("host allocation failed");
        throw Fail{PEANUT_NO_MEMORY};
    }
    char* b = static_cast<char*>(H->block);
    H->h.end_pos = reinterpret_cast<uint64_t*>(b);
    H->h.read_id = reinterpret_cast<uint32_t*>(b + c * sizeof(uint64_t));
    H->h.strand = reinterpret_cast<uint8_t*>(b + c * (sizeof(uint64_t) + sizeof(uint32_t)));
    H->h.dist = H->h.strand + c;
    try {
        if (n) {
            PN_CUDA(cudaMemcpyAsync(H->h.read_id, dh.read_id, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            PN_CUDA(cudaMemcpyAsync(H->h.strand, dh.strand, n, cudaMemcpyDeviceToHost, s));
            PN_CUDA(cudaMemcpyAsync(H->h.end_pos, dh.end_pos, n * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
            PN_CUDA(cudaMemcpyAsync(H->h.dist, dh.dist, n, cudaMemcpyDeviceToHost, s));
        }
        PN_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        free_host_hits(H);
        throw;
    }
    return H;
}

void free_host_hits(HostHits* H) {
    if (!H) return;
    host_block_free(H->block, H->block_bytes, H->pinned);
    H->magic = 0;
    delete H;
}

}  // namespace pn

using namespace pn;

template <class F>
static peanut_status guarded(F&& f) {
    clear_error();
    cudaGetLastError();  // an earlier, unrelated failure must not be reported by this call
    try {
        f();
        return PEANUT_OK;
    } catch (const Fail& e) {
        return e.st;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return PEANUT_NO_MEMORY;
    } catch (...) {
        set_error("unexpected internal error");
        return PEANUT_CUDA_ERROR;
    }
}

extern "C" {

const char* peanut_last_error(void) { return g_err; }

uint64_t peanut_kernel_launches(void) { return g_launches.load(); }

peanut_status peanut_set_allocator(peanut_alloc_fn alloc, peanut_release_fn release, void* ctx) {
    return guarded([&] {
        PN_REQUIRE((alloc == nullptr) == (release == nullptr), PEANUT_INVALID_ARG,
                   "allocator and release must both be set or both be NULL");
        g_alloc = alloc;
        g_release = release;
        g_ctx = ctx;
    });
}

peanut_status peanut_pack_reference_contigs(const char* seq, uint64_t len, const uint64_t* contig_starts,
                                            uint32_t n_contigs, uint32_t gap_min, uint64_t n_seed, void* stream,
                                            peanut_ref** out) {
    return guarded([&] {
        PN_REQUIRE(seq && out, PEANUT_INVALID_ARG, "NULL argument");
        PN_REQUIRE(len >= 1 && len < kMaxRefLen, PEANUT_INVALID_ARG, "reference length %llu outside 1..2^39",
                   (unsigned long long)len);
        *out = nullptr;
        peanut_ref* ref = new peanut_ref();
        ref->stream = (cudaStream_t)stream;
        try {
            pack_reference(ref, seq, len, contig_starts, n_contigs, gap_min, n_seed, ref->stream);
        } catch (...) {
            delete ref;
            throw;
        }
        *out = ref;
    });
}

peanut_status peanut_pack_reference(const char* seq, uint64_t len, void* stream, peanut_ref** out) {
    return peanut_pack_reference_contigs(seq, len, nullptr, 0, PEANUT_DEFAULT_GAP_MIN, 0, stream, out);
}

peanut_status peanut_ref_segments(const peanut_ref* ref, uint64_t* count, uint64_t* starts, uint64_t* ends) {
    return guarded([&] {
        PN_REQUIRE(ref && ref->magic == kMagicRef && count, PEANUT_INVALID_ARG, "bad reference or NULL count");
        *count = ref->n_seg;
        for (uint32_t x = 0; x < ref->n_seg; ++x) {
            if (starts) starts[x] = ref->hseg[2 * x];
            if (ends) ends[x] = ref->hseg[2 * x + 1];
        }
    });
}

uint64_t peanut_ref_length(const peanut_ref* ref) {
    return ref && ref->magic == kMagicRef ? ref->n : 0;
}


}  // extern "C"

namespace pn {

static void check_params(const peanut_params* p) {
    PN_REQUIRE(p, PEANUT_INVALID_ARG, "NULL params");
    PN_REQUIRE(p->q >= 1 && p->q <= 16, PEANUT_UNSUPPORTED, "q = %u outside 1..16", p->q);
    PN_REQUIRE(p->k_fixed != 0xFFFFFFFFu || p->k_permille <= 1000, PEANUT_INVALID_ARG, "k_permille > 1000");
    PN_REQUIRE(p->stride <= 64, PEANUT_INVALID_ARG, "stride = %u outside 0..64", p->stride);
    PN_REQUIRE(p->ref_index <= 1, PEANUT_INVALID_ARG, "ref_index = %u outside 0..1", p->ref_index);
    PN_REQUIRE(p->index_layout <= 2, PEANUT_INVALID_ARG, "index_layout = %u outside 0..2", p->index_layout);
}

peanut_reads* index_batch(const peanut_ref* ref, const char* d_seqs, const uint64_t* d_offsets, uint32_t n_reads,
                          uint64_t total, const peanut_params* p) {
    PN_REQUIRE(ref && ref->magic == kMagicRef, PEANUT_INVALID_ARG, "bad reference");
    check_params(p);
    PN_REQUIRE(n_reads >= 1 && n_reads <= kMaxReads, PEANUT_INVALID_ARG, "n_reads = %u outside 1..2^23", n_reads);
    cudaStream_t s = (cudaStream_t)p->stream;
    const uint32_t cap = p->freq_cap ? p->freq_cap : default_freq_cap(ref->n, p->q);
    peanut_ref* mref = const_cast<peanut_ref*>(ref);
    std::shared_ptr<RefPrep> prep;
    {
        std::lock_guard<std::mutex> lock(mref->prep_mu);
        if (!mref->prep[p->q] || mref->prep[p->q]->cap != cap) {
            std::shared_ptr<RefPrep> P(prepare_reference(ref, p->q, cap, s), free_prep);
            PN_CUDA(cudaStreamSynchronize(s));
            P->rehome();
            mref->prep[p->q] = P;
        }
        prep = mref->prep[p->q];
    }
    std::shared_ptr<const RefIndex> rindex;
    if (p->ref_index) {
        std::lock_guard<std::mutex> lock(mref->prep_mu);
        PN_REQUIRE(mref->rindex[p->q], PEANUT_INVALID_ARG,
                   "ref_index = 1 needs the reference's q-group index at q = %u (peanut_index_reference)", p->q);
        rindex = mref->rindex[p->q];
    }
    peanut_reads* R = new peanut_reads();
    try {
        R->rindex = rindex;
        R->layout = p->index_layout;
        R->prep = prep;
        R->ref = ref;
        R->stream = s;
        R->q = p->q;
        R->n_reads = n_reads;
        R->freq_cap = cap;
        R->total_bases = total;
        index_reads(R, d_seqs, d_offsets, p->k_fixed, p->k_permille, p->stride ? p->stride : 1);
    } catch (...) {
        delete R;
        throw;
    }
    return R;
}

}  // namespace pn

extern "C" {

static peanut_status index_common(const peanut_ref* ref, const char* d_seqs, const uint64_t* d_offsets,
                                  uint32_t n_reads, uint64_t total, const peanut_params* p, peanut_reads** out,
                                  bool host_input, const char* h_seqs, const uint64_t* h_offsets) {
    return guarded([&] {
        PN_REQUIRE(ref && ref->magic == kMagicRef && out, PEANUT_INVALID_ARG, "bad reference or NULL out");
        check_params(p);
        PN_REQUIRE(n_reads >= 1 && n_reads <= kMaxReads, PEANUT_INVALID_ARG, "n_reads = %u outside 1..2^23", n_reads);
        *out = nullptr;
        if (host_input) {
            cudaStream_t s = (cudaStream_t)p->stream;
            DBuf<char> ds(total ? total : 1, s);
            DBuf<uint64_t> doff((uint64_t)n_reads + 1, s);
            if (total) PN_CUDA(cudaMemcpyAsync(ds.p, h_seqs, total, cudaMemcpyHostToDevice, s));
            PN_CUDA(cudaMemcpyAsync(doff.p, h_offsets, ((uint64_t)n_reads + 1) * sizeof(uint64_t),
                                    cudaMemcpyHostToDevice, s));
            *out = index_batch(ref, ds.p, doff.p, n_reads, total, p);
        } else {
            *out = index_batch(ref, d_seqs, d_offsets, n_reads, total, p);
        }
    });
}

peanut_status peanut_index_reads(const peanut_ref* ref, const char* seqs, const uint64_t* offsets,
                                 uint32_t n_reads, const peanut_params* p, peanut_reads** out) {
    if (!seqs || !offsets) {
        set_error("NULL argument");
        return PEANUT_INVALID_ARG;
    }
    if (n_reads >= 1 && n_reads <= kMaxReads) {
        for (uint32_t i = 0; i < n_reads; ++i)
            if (offsets[i + 1] < offsets[i]) {
                set_error("read offsets must ascend");
                return PEANUT_INVALID_ARG;
            }
        if (offsets[0] != 0) {
            // rebase: the device copy starts at offsets[0]
            uint64_t* o = (uint64_t*)malloc(((uint64_t)n_reads + 1) * sizeof(uint64_t));
            if (!o) return PEANUT_NO_MEMORY;
            for (uint32_t i = 0; i <= n_reads; ++i) o[i] = offsets[i] - offsets[0];
            const peanut_status st =
                index_common(ref, nullptr, nullptr, n_reads, o[n_reads], p, out, true, seqs + offsets[0], o);
            free(o);
            return st;
        }
    }
    const uint64_t total = (n_reads >= 1 && n_reads <= kMaxReads) ? offsets[n_reads] : 0;
    return index_common(ref, nullptr, nullptr, n_reads, total, p, out, true, seqs, offsets);
}

peanut_status peanut_index_reads_device(const peanut_ref* ref, const char* d_seqs, const uint64_t* d_offsets,
                                        uint32_t n_reads, uint64_t total_bases, const peanut_params* p,
                                        peanut_reads** out) {
    if (!d_seqs || !d_offsets) {
        set_error("NULL argument");
        return PEANUT_INVALID_ARG;
    }
    return index_common(ref, d_seqs, d_offsets, n_reads, total_bases, p, out, false, nullptr, nullptr);
}

peanut_status peanut_map_device(const peanut_ref* ref, peanut_reads* reads, int mode, peanut_device_hits** out) {
    return guarded([&] {
        PN_REQUIRE(ref && ref->magic == kMagicRef && reads && reads->magic == kMagicReads && out, PEANUT_INVALID_ARG,
                   "bad reference, batch or NULL out");
        PN_REQUIRE(reads->ref == ref, PEANUT_INVALID_ARG, "batch was indexed against another reference");
        PN_REQUIRE(mode == 0 || mode == 1, PEANUT_INVALID_ARG, "mode must be 0 (all) or 1 (best stratum)");
        *out = nullptr;
        DeviceHits* H = map_batch(ref, reads, mode);
        *out = &H->h;
    });
}

static DeviceHits* dh_of(const peanut_device_hits* h) {
    return reinterpret_cast<DeviceHits*>(reinterpret_cast<char*>(const_cast<peanut_device_hits*>(h)) -
                                         offsetof(DeviceHits, h));
}

static HostHits* hh_of(peanut_hits* h) {
    return reinterpret_cast<HostHits*>(reinterpret_cast<char*>(h) - offsetof(HostHits, h));
}

peanut_status peanut_download_hits(const peanut_device_hits* dh, void* stream, peanut_hits** out) {
    return guarded([&] {
        PN_REQUIRE(dh && out && dh_of(dh)->magic == kMagicDHits, PEANUT_INVALID_ARG, "bad device hits");
        *out = nullptr;
        *out = &download_hits(*dh, (cudaStream_t)stream)->h;
    });
}

peanut_status peanut_map(const peanut_ref* ref, peanut_reads* reads, int mode, peanut_hits** out) {
    peanut_device_hits* dh = nullptr;
    peanut_status st = peanut_map_device(ref, reads, mode, &dh);
    if (st != PEANUT_OK) return st;
    st = peanut_download_hits(dh, (void*)reads->stream, out);
    peanut_free(dh);
    return st;
}

peanut_status peanut_get_map_stats(const peanut_reads* reads, peanut_map_stats* out) {
    return guarded([&] {
        PN_REQUIRE(reads && reads->magic == kMagicReads && out, PEANUT_INVALID_ARG, "bad batch");
        *out = reads->stats;
    });
}

void peanut_free(void* obj) {
    if (!obj) return;
    const uint32_t magic = *static_cast<const uint32_t*>(obj);
    if (magic == kMagicRef) {
        peanut_ref* r = static_cast<peanut_ref*>(obj);
        cudaStreamSynchronize(r->stream);
        for (auto& p : r->prep) p.reset();
        r->magic = 0;
        delete r;
        return;
    }
    if (magic == kMagicEngine) {
        destroy_engine(static_cast<peanut_engine*>(obj));
        return;
    }
    if (magic == kMagicReads) {
        peanut_reads* R = static_cast<peanut_reads*>(obj);
        cudaStreamSynchronize(R->stream);
        R->magic = 0;
        delete R;
        return;
    }
    // hit lists are passed by their public struct; their headers sit just before it
    HostHits* hh = hh_of(static_cast<peanut_hits*>(obj));
    if (hh->magic == kMagicHits) {
        free_host_hits(hh);
        return;
    }
    DeviceHits* dh = dh_of(static_cast<peanut_device_hits*>(obj));
    if (dh->magic == kMagicDHits) {
        free_device_hits(dh);
        dh->magic = 0;
        delete dh;
        return;
    }
    DevicePairs* dp = reinterpret_cast<DevicePairs*>(static_cast<char*>(obj) - offsetof(DevicePairs, p));
    if (dp->magic == kMagicDPairs) {
        cudaStreamSynchronize(dp->stream);
        dp->magic = 0;
        delete dp;
        return;
    }
}

peanut_status peanut_index_sizes(const peanut_reads* R, uint64_t* n_groups, uint64_t* n_distinct,
                                 uint64_t* n_indexed) {
    return guarded([&] {
        PN_REQUIRE(R && R->magic == kMagicReads, PEANUT_INVALID_ARG, "bad batch");
        if (n_groups) *n_groups = R->n_groups;
        if (n_distinct) *n_distinct = R->n_distinct;
        if (n_indexed) *n_indexed = R->n_indexed;
    });
}

peanut_status peanut_export_index(const peanut_reads* R, uint32_t* I, uint32_t* S, uint32_t* Sp, uint32_t* O) {
    return guarded([&] {
        PN_REQUIRE(R && R->magic == kMagicReads, PEANUT_INVALID_ARG, "bad batch");
        cudaStream_t s = R->stream;
        if (I || S) {
            // the w = 32 form: I word and S of every group of 32 codes
            std::vector<uint32_t> wi(R->n_groups + 1), ws(R->n_groups + 1);
            cudaError_t e = cudaSuccess;
            if (R->layout == 0) {
                std::vector<uint2> tmp(R->n_groups);
                e = cudaMemcpyAsync(tmp.data(), R->IS.p, R->n_groups * sizeof(uint2), cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                for (uint64_t g = 0; g < R->n_groups; ++g) {
                    wi[g] = tmp[g].x;
                    ws[g] = tmp[g].y;
                }
            } else if (R->layout == 1) {
                const uint64_t pairs = (R->n_groups + 1) / 2;
                std::vector<uint32_t> s2(pairs);
                e = cudaMemcpyAsync(wi.data(), R->I32.p, R->n_groups * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaMemcpyAsync(s2.data(), R->S2.p, pairs * 4, cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                for (uint64_t g = 0; g < R->n_groups; ++g)
                    ws[g] = s2[g >> 1] + ((g & 1) ? (uint32_t)__builtin_popcount(wi[g - 1]) : 0u);
            } else {
                const uint64_t g64 = (R->n_groups + 1) / 2;
                std::vector<unsigned long long> i64(g64);
                std::vector<uint32_t> s64(g64);
                e = cudaMemcpyAsync(i64.data(), R->I64.p, g64 * 8, cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaMemcpyAsync(s64.data(), R->S64.p, g64 * 4, cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                for (uint64_t g = 0; g < R->n_groups; ++g) {
                    const unsigned long long w = i64[g >> 1];
                    wi[g] = (g & 1) ? (uint32_t)(w >> 32) : (uint32_t)w;
                    ws[g] = s64[g >> 1] + ((g & 1) ? (uint32_t)__builtin_popcount((uint32_t)w) : 0u);
                }
            }
            PN_REQUIRE(e == cudaSuccess, PEANUT_CUDA_ERROR, "copy of the index failed: %s", cudaGetErrorString(e));
            for (uint64_t g = 0; g < R->n_groups; ++g) {
                if (I) I[g] = wi[g];
                if (S) S[g] = ws[g];
            }
        }
        if (Sp) PN_CUDA(cudaMemcpyAsync(Sp, R->Sp.p, (R->n_distinct + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        if (O && R->n_indexed)
            PN_CUDA(cudaMemcpyAsync(O, R->O.p, R->n_indexed * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        PN_CUDA(cudaStreamSynchronize(s));
    });
}

peanut_status peanut_export_read_params(const peanut_reads* R, uint16_t* thr, uint8_t* lowcx) {
    return guarded([&] {
        PN_REQUIRE(R && R->magic == kMagicReads, PEANUT_INVALID_ARG, "bad batch");
        cudaStream_t s = R->stream;
        if (thr) PN_CUDA(cudaMemcpyAsync(thr, R->thr.p, R->n_reads * sizeof(uint16_t), cudaMemcpyDeviceToHost, s));
        if (lowcx) PN_CUDA(cudaMemcpyAsync(lowcx, R->lowcx.p, R->n_reads, cudaMemcpyDeviceToHost, s));
        PN_CUDA(cudaStreamSynchronize(s));
    });
}

peanut_status peanut_export_candidates(const peanut_reads* R, uint64_t* n, uint32_t* read, uint8_t* strand,
                                       uint64_t* lo, uint64_t* hi) {
    return guarded([&] {
        PN_REQUIRE(R && R->magic == kMagicReads && n, PEANUT_INVALID_ARG, "bad batch or NULL n");
        const uint64_t nc = R->n_cand, nl = R->n_live;
        if (!read && !strand && !lo && !hi) {
            *n = nl;
            return;
        }
        PN_REQUIRE(*n >= nl, PEANUT_INVALID_ARG, "buffers hold %llu entries, %llu needed", (unsigned long long)*n,
                   (unsigned long long)nl);
        *n = nl;
        if (!nc) return;
        uint64_t* k = (uint64_t*)malloc(nc * 8);
        uint64_t* h = (uint64_t*)malloc(nc * 8);
        PN_REQUIRE(k && h, PEANUT_NO_MEMORY, "host allocation failed");
        cudaStream_t s = R->stream;
        cudaMemcpyAsync(k, R->cand_key.p, nc * 8, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(h, R->cand_hi.p, nc * 8, cudaMemcpyDeviceToHost, s);
        const cudaError_t e = cudaStreamSynchronize(s);
        uint64_t o = 0;
        for (uint64_t x = 0; x < nc && e == cudaSuccess; ++x) {
            if (h[x] == ~0ull) continue;  // removed by the q'-gram filter
            if (o < nl) {
                if (read) read[o] = (uint32_t)(k[x] >> 41);
                if (strand) strand[o] = (uint8_t)((k[x] >> 40) & 1);
                if (lo) lo[o] = k[x] & ((1ull << 40) - 1);
                if (hi) hi[o] = h[x];
            }
            ++o;
        }
        free(k);
        free(h);
        PN_REQUIRE(e == cudaSuccess, PEANUT_CUDA_ERROR, "candidate copy failed: %s", cudaGetErrorString(e));
    });
}

peanut_status peanut_debug_bitvector_columns(const char* pat, const uint64_t* pat_off, uint32_t n_pat, const char* txt,
                                             const uint64_t* txt_off, int32_t* out, void* stream) {
    return guarded([&] {
        PN_REQUIRE(pat && pat_off && txt && txt_off && out && n_pat >= 1, PEANUT_INVALID_ARG, "bad arguments");
        bitvector_columns(pat, pat_off, n_pat, txt, txt_off, out, (cudaStream_t)stream);
    });
}

peanut_status peanut_bitvector_columns_noalloc(const char* d_pat, const uint64_t* d_pat_off, uint32_t n_pat,
                                               const char* d_txt, const uint64_t* d_txt_off, int32_t* d_out,
                                               void* stream) {
    return guarded([&] {
        PN_REQUIRE(d_pat && d_pat_off && d_txt && d_txt_off && d_out, PEANUT_INVALID_ARG, "NULL argument");
        bitvector_columns_noalloc(d_pat, d_pat_off, n_pat, d_txt, d_txt_off, d_out, (cudaStream_t)stream);
    });
}

peanut_status peanut_index_reference(peanut_ref* ref, uint32_t q, void* stream) {
    return guarded([&] {
        PN_REQUIRE(ref && ref->magic == kMagicRef, PEANUT_INVALID_ARG, "bad reference");
        PN_REQUIRE(q >= 1 && q <= 16, PEANUT_UNSUPPORTED, "q = %u outside 1..16", q);
        {
            std::lock_guard<std::mutex> lock(ref->prep_mu);
            if (ref->rindex[q]) return;
        }
        std::shared_ptr<RefIndex> X(build_ref_index(ref, q, (cudaStream_t)stream));
        X->rehome();
        std::lock_guard<std::mutex> lock(ref->prep_mu);
        if (!ref->rindex[q]) ref->rindex[q] = X;
    });
}

peanut_status peanut_annotate_hits(const peanut_ref* ref, const peanut_reads* reads, const peanut_device_hits* hits,
                                   uint64_t* d_start, uint32_t* d_rank, uint8_t* d_mapq) {
    return guarded([&] {
        PN_REQUIRE(ref && ref->magic == kMagicRef && reads && reads->magic == kMagicReads && hits, PEANUT_INVALID_ARG,
                   "bad reference, batch or hit list");
        PN_REQUIRE(reads->ref == ref, PEANUT_INVALID_ARG, "the batch was indexed against another reference");
        PN_REQUIRE(hits->n == 0 || (hits->read_id && hits->strand && hits->end_pos && hits->dist && d_start && d_rank &&
                                    d_mapq), PEANUT_INVALID_ARG, "NULL array");
        annotate_hits(ref, reads, *hits, d_start, d_rank, d_mapq);
    });
}

uint32_t peanut_batch_max_k(const peanut_reads* reads) {
    return reads && reads->magic == kMagicReads ? reads->max_k : 0;
}

peanut_status peanut_hit_alignments(const peanut_ref* ref, const peanut_reads* reads, const peanut_device_hits* hits,
                                    const uint64_t* d_start, uint32_t ops_per_hit, uint32_t* d_ops, uint16_t* d_nops) {
    return guarded([&] {
        PN_REQUIRE(ref && ref->magic == kMagicRef && reads && reads->magic == kMagicReads && hits, PEANUT_INVALID_ARG,
                   "bad reference, batch or hit list");
        PN_REQUIRE(reads->ref == ref, PEANUT_INVALID_ARG, "the batch was indexed against another reference");
        PN_REQUIRE(ops_per_hit >= 1, PEANUT_INVALID_ARG, "ops_per_hit must be at least 1");
        PN_REQUIRE(hits->n == 0 || (hits->read_id && hits->strand && hits->end_pos && hits->dist && d_start && d_ops &&
                                    d_nops), PEANUT_INVALID_ARG, "NULL array");
        hit_alignments(ref, reads, *hits, d_start, ops_per_hit, d_ops, d_nops);
    });
}

static DevicePairs* dp_of(const peanut_device_pairs* p) {
    return reinterpret_cast<DevicePairs*>(reinterpret_cast<char*>(const_cast<peanut_device_pairs*>(p)) -
                                          offsetof(DevicePairs, p));
}

peanut_status peanut_pair_hits(const peanut_ref* ref, const peanut_reads* reads, const peanut_device_hits* hits,
                               const uint64_t* d_start, uint32_t min_insert, uint32_t max_insert, int mode,
                               peanut_device_pairs** out) {
    return guarded([&] {
        PN_REQUIRE(ref && ref->magic == kMagicRef && reads && reads->magic == kMagicReads && hits && out,
                   PEANUT_INVALID_ARG, "bad reference, batch, hit list or NULL out");
        PN_REQUIRE(reads->ref == ref, PEANUT_INVALID_ARG, "the batch was indexed against another reference");
        PN_REQUIRE(hits->n == 0 || (hits->read_id && hits->strand && hits->end_pos && hits->dist && d_start),
                   PEANUT_INVALID_ARG, "NULL array");
        PN_REQUIRE(mode == 0 || mode == 1, PEANUT_INVALID_ARG, "mode must be 0 (all) or 1 (best stratum)");
        *out = nullptr;
        *out = &pair_hits(ref, reads, *hits, d_start, min_insert, max_insert, mode)->p;
    });
}

peanut_status peanut_download_pairs(const peanut_device_pairs* pairs, void* stream, uint64_t* i1, uint64_t* i2,
                                    uint32_t* score, uint32_t* rank, uint8_t* mapq) {
    return guarded([&] {
        PN_REQUIRE(pairs && dp_of(pairs)->magic == kMagicDPairs, PEANUT_INVALID_ARG, "bad pairs object");
        const uint64_t n = pairs->n;
        cudaStream_t s = (cudaStream_t)stream;
        if (n && i1) PN_CUDA(cudaMemcpyAsync(i1, pairs->i1, n * 8, cudaMemcpyDeviceToHost, s));
        if (n && i2) PN_CUDA(cudaMemcpyAsync(i2, pairs->i2, n * 8, cudaMemcpyDeviceToHost, s));
        if (n && score) PN_CUDA(cudaMemcpyAsync(score, pairs->score, n * 4, cudaMemcpyDeviceToHost, s));
        if (n && rank) PN_CUDA(cudaMemcpyAsync(rank, pairs->rank, n * 4, cudaMemcpyDeviceToHost, s));
        if (n && mapq) PN_CUDA(cudaMemcpyAsync(mapq, pairs->mapq, n, cudaMemcpyDeviceToHost, s));
        PN_CUDA(cudaStreamSynchronize(s));
    });
}

peanut_status peanut_int_peak(uint32_t kind, uint32_t iters, void* stream, double* ms, uint64_t* ops,
                              uint32_t* grid, uint32_t* block) {
    return guarded([&] {
        PN_REQUIRE(ms && ops && grid && block && iters >= 1, PEANUT_INVALID_ARG, "bad arguments");
        int_peak(kind, iters, (cudaStream_t)stream, ms, ops, grid, block);
    });
}

}  // extern "C"
