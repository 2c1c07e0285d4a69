// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <mutex>
#include <vector>
#include <string>

#include "peanut.h"

namespace pn {

constexpr int kMaxReadLen = 255;
constexpr int kMaxWords = 4;                 // 64-bit words per bit-vector column (m <= 256)
constexpr uint32_t kMaxReads = 1u << 23;     // read id fits 23 bits of a hit key
constexpr uint64_t kMaxRefLen = 1ull << 39;  // biased diagonal fits 40 bits of a hit key
constexpr int64_t kDiagBias = 256;           // diagonal d >= -254; key stores d + kDiagBias
constexpr uint32_t kSentinel = 0xFFFFFFFFu;  // "not indexed" code (no canonical q-gram is all ones)
constexpr uint32_t kDefaultFreqCap = 256;
constexpr uint64_t kClusterGap = 64;         // occurrences closer than this share a cluster
constexpr int kFilterBits = 24;              // frequent-q-gram prefilter: 2^24 bits

constexpr uint32_t kMagicRef = 0x50524546u;    // 'PREF'
constexpr uint32_t kMagicReads = 0x50524453u;  // 'PRDS'
constexpr uint32_t kMagicHits = 0x50484954u;   // 'PHIT'
constexpr uint32_t kMagicDHits = 0x50444854u;  // 'PDHT'
constexpr uint32_t kMagicEngine = 0x50454E47u; // 'PENG'
constexpr uint32_t kMagicDPairs = 0x50445052u; // 'PDPR'

// device status bits (written by kernels, read at synchronization points)
enum : uint32_t {
    kStBadBase = 1u,
    kStBadLength = 2u,
    kStBadThreshold = 4u,
    kStOverflow = 8u,
    kStHasN = 16u,  // an unknown base (N) was seen; its replacement runs afterwards
};

// ---- errors -------------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

struct Fail {
    peanut_status st;
};

#define PN_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            ::pn::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                            __LINE__);                                                      \
            throw ::pn::Fail{PEANUT_CUDA_ERROR};                                            \
        }                                                                                   \
    } while (0)

void note_launch();  // counts kernel launches (peanut_kernel_launches)
#define PN_CHECK_LAUNCH()                \
    do {                                 \
        ::pn::note_launch();             \
        PN_CUDA(cudaGetLastError());     \
    } while (0)

#define PN_REQUIRE(cond, status, ...)        \
    do {                                     \
        if (!(cond)) {                       \
            ::pn::set_error(__VA_ARGS__);    \
            throw ::pn::Fail{status};        \
        }                                    \
    } while (0)

// ---- device memory ----------------------------------------------------------------------
// The provider that made an allocation releases it, even if another was installed since.
struct Allocator {
    peanut_alloc_fn alloc = nullptr;      // nullptr: cudaMallocAsync / cudaFreeAsync
    peanut_release_fn release = nullptr;
    void* ctx = nullptr;
};
Allocator current_allocator();
void use_pool_on_this_thread();  // this thread allocates from the stream-ordered pool
bool pool_on_this_thread();
void use_graphs_on_this_thread(bool on);
bool graphs_on_this_thread();

// Records ev on s; inside a stream capture as an event-record node of the graph (a plain record
// there only orders the capture), so that the event is recorded when the graph runs.
inline cudaError_t record_event(cudaEvent_t ev, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        return cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
    return cudaEventRecord(ev, s);
}

// A sync-free stretch of work on stream s captured as a CUDA graph and launched once (when
// enabled: an engine created with graphs = 1, whose threads allocate from the stream-ordered
// pool; its allocations and frees become graph memory nodes).  run() ends the capture and launches the graph; the graph is released when
// the segment is destroyed (after the caller's next synchronization).  An exception inside the
// captured stretch ends the capture and discards it.
struct GraphSegment {
    cudaStream_t s = nullptr;
    bool on = false, capturing = false;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    GraphSegment(cudaStream_t st, bool enable) : s(st), on(enable) {
        if (on) {
            PN_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            capturing = true;
        }
    }
    GraphSegment(const GraphSegment&) = delete;
    GraphSegment& operator=(const GraphSegment&) = delete;
    bool run() {
        if (!on) return false;
        capturing = false;
        PN_CUDA(cudaStreamEndCapture(s, &g));
        PN_CUDA(cudaGraphInstantiate(&x, g, 0));
        PN_CUDA(cudaGraphLaunch(x, s));
        return true;
    }
    ~GraphSegment() {
        if (capturing) {
            cudaGraph_t t = nullptr;
            cudaStreamEndCapture(s, &t);
            if (t) cudaGraphDestroy(t);
            cudaGetLastError();
        }
        if (x) cudaGraphExecDestroy(x);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
    }
};
void* dalloc(size_t bytes, cudaStream_t s, Allocator* used = nullptr);  // throws Fail{NO_MEMORY}
void dfree(void* p, cudaStream_t s, const Allocator& a);

template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    Allocator a;
    DBuf() = default;
    DBuf(size_t count, cudaStream_t st) { alloc(count, st); }
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), n(o.n), s(o.s), a(o.a) { o.p = nullptr; o.n = 0; }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) { reset(); p = o.p; n = o.n; s = o.s; a = o.a; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DBuf() { reset(); }
    void alloc(size_t count, cudaStream_t st) {
        reset();
        s = st;
        n = count;
        p = count ? static_cast<T*>(dalloc(count * sizeof(T), st, &a)) : nullptr;
    }
    void zero() {
        if (n) PN_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
    }
    void reset() {
        if (p) dfree(p, s, a);
        p = nullptr;
        n = 0;
    }
    T* release() { T* q = p; p = nullptr; n = 0; return q; }
    size_t bytes() const { return n * sizeof(T); }
};

template <class T>
T to_host(const T* d, cudaStream_t s) {
    T h;
    PN_CUDA(cudaMemcpyAsync(&h, d, sizeof(T), cudaMemcpyDeviceToHost, s));
    PN_CUDA(cudaStreamSynchronize(s));
    return h;
}

inline unsigned grid_for(uint64_t n, unsigned block, unsigned cap = 1u << 30) {
    uint64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

int sm_count();

// ---- frequent q-grams of a reference (per q) --------------------------------------------
struct RefPrep {
    uint32_t q = 0, cap = 0;
    uint32_t n_phi = 0;          // number of frequent canonical q-grams
    uint64_t n_clusters = 0;
    uint64_t n_occ = 0;          // their total occurrences
    DBuf<uint32_t> phi_codes;    // sorted canonical codes, n_phi
    DBuf<uint32_t> filter;       // 2^kFilterBits bit prefilter over code >> filter_shift
    uint32_t filter_shift = 0;
    DBuf<uint64_t> grp_off;      // 2*n_phi + 1: cluster range of (phi, orientation)
    DBuf<uint64_t> cl_lo, cl_hi; // first / last occurrence position of each cluster
    // The table outlives the stream it was built on (batches of any stream share it): once its
    // work is complete its buffers are released on the legacy default stream.
    void rehome() {
        phi_codes.s = filter.s = nullptr;
        grp_off.s = cl_lo.s = cl_hi.s = nullptr;
    }
};

// ---- the batch's q-group index as the device sees it (one of three layouts) ---------------
struct IndexView {
    uint32_t layout;
    const uint2* IS;
    const uint32_t* I32;
    const uint32_t* S2;
    const unsigned long long* I64;
    const uint32_t* S64;
};

// ---- the reference's own q-group index (Algorithm 1 over the reference's q-grams) -----------
struct RefIndex {
    uint32_t q = 0;
    uint64_t n_groups = 0, n_distinct = 0, n_pos = 0;
    DBuf<uint2> IS;         // (I word, S) per group of 32 canonical codes
    DBuf<uint32_t> Sp;      // n_distinct + 1 starts into O (positions < 2^32)
    DBuf<uint32_t> O;       // reference positions grouped by canonical code
    DBuf<uint32_t> orient;  // bit x: occurrence O[x] holds the reverse complement of its code
    void rehome() { IS.s = Sp.s = O.s = orient.s = nullptr; }
};

}  // namespace pn

struct peanut_ref {
    uint32_t magic = pn::kMagicRef;
    uint64_t n = 0;             // bases
    uint64_t n_words = 0;       // packed 32-bit words (16 bases each), plus padding
    pn::DBuf<uint32_t> packed;  // base p at bits 30 - 2 (p % 16) of word p / 16
    cudaStream_t stream = nullptr;
    std::shared_ptr<pn::RefPrep> prep[17];  // per q; batches share the table they were indexed with
    std::shared_ptr<pn::RefIndex> rindex[17];  // per q, built on request (peanut_index_reference)
    std::mutex prep_mu;
    // Segments: the stretches of each contig between gaps (runs of >= gap_min unknown bases).
    // No alignment leaves its segment; seg holds [start, end) pairs, ascending.
    uint64_t n_seed = 0;                 // seeds the replacement of unknown bases (reference and reads)
    uint32_t n_contigs = 1;
    pn::DBuf<uint64_t> contig;           // contig starts on the device (the first 0)
    uint64_t n_gaps = 0;
    std::vector<uint64_t> hseg;          // host copy, 2 per segment
    pn::DBuf<uint64_t> seg;              // device copy
    uint32_t n_seg = 0;
};

struct peanut_reads {
    uint32_t magic = pn::kMagicReads;
    const peanut_ref* ref = nullptr;
    cudaStream_t stream = nullptr;
    uint32_t q = 0, n_reads = 0, max_len = 0, max_k = 0, freq_cap = 0, stride = 1;
    std::shared_ptr<const pn::RefIndex> rindex;  // set: hits come from the reference's index
    uint64_t total_bases = 0;
    std::shared_ptr<const pn::RefPrep> prep;  // frequent q-grams of the reference at this q and cap
    // per read
    pn::DBuf<uint64_t> base_off;  // n+1 offsets into codes
    pn::DBuf<uint8_t> codes;      // 2-bit codes, one per byte
    pn::DBuf<uint8_t> len;        // read length (1..255)
    pn::DBuf<uint8_t> kk;         // error budget
    pn::DBuf<uint16_t> thr;       // q-gram count threshold used by the filter
    pn::DBuf<uint8_t> lowcx;      // 1 = verified around frequent-q-gram clusters
    pn::DBuf<uint64_t> peq;       // [n][2 strands][4 bases][kMaxWords] match bit masks
    // q-group index
    uint64_t n_groups = 0, n_distinct = 0, n_indexed = 0, n_qgrams = 0;
    uint32_t layout = 0;          // 0: (I, S) interleaved per group of 32 codes; 1: I per 32 codes,
                                  // S sampled at every second group; 2: I per 64 codes (w = 64)
    pn::DBuf<uint2> IS;           // layout 0: (I word, S) per group of 32 canonical codes
    pn::DBuf<uint32_t> I32, S2;   // layout 1: I per group of 32; S of the even groups
    pn::DBuf<unsigned long long> I64;  // layout 2: I per group of 64
    pn::DBuf<uint32_t> S64;       // layout 2: S per group of 64
    pn::DBuf<uint32_t> Sp;        // n_qgrams + 1 (first n_distinct + 1 meaningful)
    pn::DBuf<uint32_t> O;         // n_indexed entries (read << 9 | orientation << 8 | offset)
    pn::DBuf<uint64_t> bloom;     // blocked Bloom filter of the indexed canonical codes (L2-sized)
    uint64_t bloom_mask = 0;      // words - 1
    // frequent q-grams of each read (only meaningful for reads with fcnt > 0)
    pn::DBuf<uint64_t> qoff;      // n+1: q-gram slot offsets
    pn::DBuf<uint32_t> fcnt;      // frequent q-grams per read
    pn::DBuf<uint64_t> fent;      // phi << 32 | palindrome << 9 | orientation << 8 | offset
    pn::DBuf<uint32_t> lowcx_list;
    uint32_t n_lowcx = 0;
    // results of the last map call kept for introspection
    pn::DBuf<uint64_t> cand_key;  // lo (40 bits) | strand << 40 | read << 41
    pn::DBuf<uint64_t> cand_hi;
    uint64_t n_cand = 0;
    uint64_t n_live = 0;          // of those, ranges the q'-gram filter kept (cand_hi != ~0)
    peanut_map_stats stats = {};
};

struct HostHits {
    uint32_t magic = pn::kMagicHits;
    peanut_hits h = {};
    void* block = nullptr;  // one host block holding the four arrays
    size_t block_bytes = 0;
    bool pinned = false;
};

struct DeviceHits {
    uint32_t magic = pn::kMagicDHits;
    peanut_device_hits h = {};
    cudaStream_t stream = nullptr;
    pn::Allocator a;  // made the four arrays
};

struct DevicePairs {
    uint32_t magic = pn::kMagicDPairs;
    peanut_device_pairs p = {};
    cudaStream_t stream = nullptr;
    pn::DBuf<uint64_t> i1, i2;
    pn::DBuf<uint32_t> score, rank;
    pn::DBuf<uint8_t> mapq;
};

namespace pn {
// api.cu: page-locked host blocks for results, kept for reuse after they are freed
void* host_block_alloc(size_t bytes, size_t* got, bool* pinned);
void host_block_free(void* p, size_t bytes, bool pinned);
HostHits* download_hits(const peanut_device_hits& dh, cudaStream_t s);  // synchronizes s
uint64_t pageable_blocks();  // result blocks so far that fell back to pageable memory
void free_host_hits(HostHits* H);
// index.cu
// True when the reference is more than one segment [0, n) (several contigs, or gaps).
inline bool segmented(const peanut_ref* ref) {
    return !(ref->n_seg == 1 && ref->hseg[0] == 0 && ref->hseg[1] == ref->n);
}

void pack_reference(peanut_ref* ref, const char* host_seq, uint64_t len, const uint64_t* contig_starts,
                    uint32_t n_contigs, uint32_t gap_min, uint64_t seed, cudaStream_t s);
RefPrep* prepare_reference(const peanut_ref* ref, uint32_t q, uint32_t cap, cudaStream_t s);
void free_prep(RefPrep* p);
void index_reads(peanut_reads* R, const char* d_seqs, const uint64_t* d_offsets, uint32_t k_fixed,
                 uint32_t k_permille, uint32_t stride);
uint32_t default_freq_cap(uint64_t ref_len, uint32_t q);
RefIndex* build_ref_index(const peanut_ref* ref, uint32_t q, cudaStream_t s);
// engine.cu: joins the executor threads and releases everything the engine holds
void destroy_engine(peanut_engine* E);
// api.cu: a new batch indexed from reads in device memory (throws Fail on error)
peanut_reads* index_batch(const peanut_ref* ref, const char* d_seqs, const uint64_t* d_offsets, uint32_t n_reads,
                          uint64_t total, const peanut_params* p);
inline IndexView index_view(const peanut_reads* R) {
    return IndexView{R->layout, R->IS.p, R->I32.p, R->S2.p, R->I64.p, R->S64.p};
}
// map.cu
DeviceHits* map_batch(const peanut_ref* ref, peanut_reads* R, int mode);
// keeps, per read, the results at the read's smallest distance over both strands (in: sorted)
void best_stratum(const peanut_device_hits& in, uint32_t n_reads, DeviceHits* out, cudaStream_t s);
void alloc_device_hits(DeviceHits* H, uint64_t n, cudaStream_t s);
void free_device_hits(DeviceHits* H);
void bitvector_columns(const char* pat, const uint64_t* pat_off, uint32_t n_pat, const char* txt,
                       const uint64_t* txt_off, int32_t* out, cudaStream_t s);
// post.cu: start, hit-rank and mapping quality of a batch's hits (device arrays of H.n entries)
void hit_alignments(const peanut_ref* ref, const peanut_reads* R, const peanut_device_hits& H, const uint64_t* d_start,
                    uint32_t cap, uint32_t* d_ops, uint16_t* d_nops);
DevicePairs* pair_hits(const peanut_ref* ref, const peanut_reads* R, const peanut_device_hits& H, const uint64_t* d_start,
                       uint32_t min_insert, uint32_t max_insert, int mode);
void annotate_hits(const peanut_ref* ref, const peanut_reads* R, const peanut_device_hits& H, uint64_t* d_start,
                   uint32_t* d_rank, uint8_t* d_mapq);
// peak.cu: integer issue-rate microbenchmark (timed with CUDA events on s)
void int_peak(uint32_t kind, uint32_t iters, cudaStream_t s, double* ms, uint64_t* ops, uint32_t* grid,
              uint32_t* block);
void bitvector_columns_noalloc(const char* d_pat, const uint64_t* d_pat_off, uint32_t n_pat, const char* d_txt,
                               const uint64_t* d_txt_off, int32_t* d_out, cudaStream_t s);
}  // namespace pn
