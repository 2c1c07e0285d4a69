// Batched and served mapping: the runtime behind peanut_engine_* (include/peanut.h).
//
// Submissions are admitted against a device-memory budget, their reads classified by the largest
// q each admits (the q-gram lemma threshold, Section "The q-group index"), and the reads of a
// class coalesced across submissions into launches of the per-batch path (index_batch +
// map_batch).  Executor threads, each with its own non-blocking stream, take launches from the
// class queues, so launches overlap on the device.  A submission's results are collected from
// every launch that held some of its reads, renumbered and sorted on the device, and returned
// as one host hit list.  An autotuner maps the first launch of each class under several
// (q, stride) settings and keeps the one with the lowest predicted time per read.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <system_error>
#include <thread>
#include <unordered_map>
#include <vector>

#include "prims.cuh"

namespace pn {

constexpr uint32_t kEngineMaxReads = 1u << 24;  // per submission: read id fits 24 bits of a sort key
constexpr uint32_t kTuneReads = 1u << 17;       // reads of a class's first (timed) launch
constexpr uint32_t kMinLaunch = 1u << 12;       // smallest launch formed while others are in flight
constexpr double kMaxLaunchHits = 2147483648.0; // expected q-gram hits of one launch at most
constexpr int kMaxExecutors = 4;
constexpr int kQSlots = 17;                     // classes are indexed by q (1..16)

// ---- device helpers ------------------------------------------------------------------------

// Per read of a submission: its length, budget and the largest q (<= qcap) with
// m + 1 - q(k + 1) >= 1 (0 = none); the lengths seen per class go into a 256-bit mask.
__global__ void classify_k(const uint64_t* __restrict__ off, uint32_t n, uint64_t span, uint32_t k_fixed,
                           uint32_t k_permille, uint32_t qcap, uint32_t fixed_q, uint8_t* cls, uint32_t* counts,
                           uint32_t* lenmask, uint32_t* status) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const uint64_t o0 = off[0], a = off[r], b = off[r + 1];
    if (b < a || a < o0 || b - o0 > span || b - a < 1 || b - a > (uint64_t)kMaxReadLen) {
        atomicOr(status, kStBadLength);
        cls[r] = 0;
        return;
    }
    const uint32_t m = (uint32_t)(b - a);
    const uint64_t k = k_fixed != 0xFFFFFFFFu ? k_fixed : ((uint64_t)m * k_permille + 999) / 1000;
    uint32_t q = 0;
    if (k <= 255) {
        q = (uint32_t)((uint64_t)m / (k + 1));  // largest q with q(k + 1) <= m
        if (q > qcap) q = qcap;
        if (fixed_q) q = ((uint64_t)fixed_q * (k + 1) <= m) ? fixed_q : 0;
    }
    if (q == 0) {
        atomicOr(status, kStBadThreshold);
        cls[r] = 0;
        return;
    }
    cls[r] = (uint8_t)q;
    atomicAdd(&counts[q], 1u);
    atomicOr(&lenmask[q * 8 + (m >> 5)], 1u << (m & 31));
}

__global__ void check_bases_k(const uint8_t* __restrict__ s, uint64_t n, uint32_t* status) {
    bool bad = false;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint8_t c = s[x];
        const uint8_t u = (c >= 'a' && c <= 'z') ? (uint8_t)(c - 32) : c;  // either case
        bad |= !(u == 'A' || u == 'C' || u == 'G' || u == 'T' || u == 'N');
    }
    if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStBadBase);
}

// Stable compaction of the reads of class c: list[rank] = read id.
struct ClassFlag {
    const uint8_t* cls;
    uint8_t c;
    __device__ __forceinline__ uint64_t operator()(uint64_t i) const { return cls[i] == c ? 1 : 0; }
};
struct ClassScatter {
    const uint8_t* cls;
    uint8_t c;
    uint32_t* list;
    __device__ __forceinline__ void operator()(uint64_t i, uint64_t v) const {
        if (cls[i] == c) list[v] = (uint32_t)i;
    }
};

// A launch is a list of segments: reads list[x0 .. x0 + n) of one submission, at launch-local
// ids base .. base + n.
struct SegDev {
    const char* seq;
    const uint64_t* off;
    const uint32_t* list;
    uint64_t off0;
    uint32_t x0, n, base, pad;
};

__device__ __forceinline__ uint32_t seg_of(const SegDev* seg, uint32_t nseg, uint32_t j) {
    uint32_t lo = 0, hi = nseg;  // last segment with base <= j
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (seg[mid].base <= j) lo = mid;
        else hi = mid;
    }
    return lo;
}

struct GatherLen {
    const SegDev* seg;
    uint32_t nseg;
    __device__ uint64_t operator()(uint64_t j) const {
        const SegDev& s = seg[seg_of(seg, nseg, (uint32_t)j)];
        const uint32_t r = s.list[s.x0 + ((uint32_t)j - s.base)];
        return s.off[r + 1] - s.off[r];
    }
};

// One warp per launch-local read: copy its bases into the launch's contiguous buffer.
__global__ void gather_copy_k(const SegDev* __restrict__ seg, uint32_t nseg, uint32_t n, const uint64_t* __restrict__ noff,
                              char* __restrict__ dst) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < n; j += warps) {
        const SegDev& s = seg[seg_of(seg, nseg, j)];
        const uint32_t r = s.list[s.x0 + (j - s.base)];
        const char* src = s.seq + (s.off[r] - s.off0);
        const uint32_t m = (uint32_t)(s.off[r + 1] - s.off[r]);
        char* d = dst + noff[j];
        for (uint32_t x = lane; x < m; x += 32) d[x] = src[x];
    }
}

// First result row of every segment boundary (results are sorted by launch-local read).
__global__ void seg_bounds_k(const uint32_t* __restrict__ rd, uint64_t nt, const uint32_t* __restrict__ bases,
                             uint32_t nb, uint64_t* out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    const uint32_t key = bases[i];
    uint64_t lo = 0, hi = nt;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (rd[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    out[i] = lo;
}

// Result rows of one part -> sort keys in the submission's read ids:
// key = read << 40 | strand << 39 | end (end < 2^39), value = distance.
__global__ void renumber_k(const uint32_t* __restrict__ rd, const uint8_t* __restrict__ st,
                           const uint64_t* __restrict__ en, const uint8_t* __restrict__ di, uint64_t lo, uint64_t hi,
                           uint32_t base, const uint32_t* __restrict__ list, uint64_t* key, uint64_t* val) {
    for (uint64_t x = lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < hi;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = list[rd[x] - base];
        key[x - lo] = (r << 40) | ((uint64_t)st[x] << 39) | en[x];
        val[x - lo] = di[x];
    }
}

__global__ void unpack_k(const uint64_t* __restrict__ key, const uint64_t* __restrict__ val, uint64_t n,
                         peanut_device_hits h) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t k = key[x];
        h.read_id[x] = (uint32_t)(k >> 40);
        h.strand[x] = (uint8_t)((k >> 39) & 1u);
        h.end_pos[x] = k & ((1ull << 39) - 1);
        h.dist[x] = (uint8_t)val[x];
    }
}

__host__ __device__ inline int64_t sampled_threshold_host(uint32_t nq, uint32_t q, uint32_t k, uint32_t s) {
    const int64_t na = (nq + s - 1) / s;
    const int64_t cover = (int64_t)k * ((q + s - 1) / s);
    return na - (cover < na ? cover : na);
}

// ---- host structures -----------------------------------------------------------------------

struct Launch {  // one mapped batch; parts of several submissions share its result arrays
    DeviceHits* out = nullptr;
    ~Launch() {
        if (out) {
            free_device_hits(out);
            delete out;
        }
    }
};

struct Part {
    std::shared_ptr<Launch> launch;
    uint64_t lo = 0, hi = 0;  // result rows
    uint32_t base = 0;        // launch-local id of the segment's first read
    uint32_t cls = 0, x0 = 0; // class and first position in the submission's class list
};

struct Submission {
    uint64_t ticket = 0;
    int mode = 0;
    uint32_t n_reads = 0;
    uint64_t span = 0;                     // bytes from offsets[0] to offsets[n]
    const char* h_seq = nullptr;           // host input (caller-owned), or
    const uint64_t* h_off = nullptr;
    const char* u_seq = nullptr;           // device input (caller-owned)
    const uint64_t* u_off = nullptr;
    DBuf<char> d_seq;                      // device copies of host input
    DBuf<uint64_t> d_off;
    const char* seq = nullptr;             // device view: read i at seq + off[i] - off0
    const uint64_t* off = nullptr;
    uint64_t off0 = 0;
    DBuf<uint32_t> list[kQSlots];          // read ids of each class, ascending
    uint32_t cnt[kQSlots] = {}, next[kQSlots] = {};
    uint32_t lenmask[kQSlots][8] = {};
    uint32_t remaining = 0, classes = 0, inflight = 0;
    uint64_t reserved = 0, order = 0;
    std::vector<Part> parts;
    peanut_status status = PEANUT_OK;
    std::string err;
    HostHits* result = nullptr;      // host result, or
    DeviceHits* dresult = nullptr;   // device result (PEANUT_RESULT_ON_DEVICE)
    bool on_device = false;
    bool done = false, queued = false;
};

struct ClassState {
    uint32_t q = 0, stride = 1, cap = 0;
    bool tuned = false, tuning = false;
    std::deque<Submission*> queue;  // submissions with unconsumed reads of this class
    uint64_t waiting = 0;
    uint32_t lenmask[8] = {};
    double bytes_per_read = 0;      // measured (largest seen), 0 = not yet
    double hits_per_read = 0;       // q-gram hits per read, measured (largest seen), 0 = not yet
    uint64_t launches = 0, reads = 0;
    float tuned_ms_per_mread = 0;
    uint32_t tune_candidates = 0;
};

struct Segment {
    Submission* sub;
    uint32_t cls, x0, n, base;
};

struct Download {  // an assembled result on its way to the host
    Submission* sub = nullptr;
    DeviceHits* fin = nullptr;
    cudaEvent_t ready = nullptr;  // recorded after the assembly on the executor's stream
};

static double wall_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace pn

struct peanut_engine {
    uint32_t magic = pn::kMagicEngine;
    const peanut_ref* ref = nullptr;
    peanut_engine_params p = {};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<pn::Submission*> pending;
    std::unordered_map<uint64_t, pn::Submission*> subs;
    pn::ClassState cls[pn::kQSlots];
    uint64_t budget = 0, reserved = 0, reserved_peak = 0;
    uint64_t next_ticket = 1, next_order = 0;
    int running = 0;  // admissions and launches in progress
    int tuning_active = 0;  // tuning runs in progress (they run alone)
    int launching = 0, admitting = 0;  // launches / admissions in progress
    bool stop = false;
    std::vector<std::thread> threads;
    std::vector<cudaStream_t> streams;
    cudaStream_t io_stream = nullptr;
    std::deque<pn::Download> downloads;  // results waiting for the I/O thread
    uint64_t n_submitted = 0, n_completed = 0, n_reads = 0, n_launches = 0, n_tuning = 0;
    struct {
        uint64_t hits = 0, candidates = 0, word_columns = 0, present_probes = 0, results = 0;
        uint64_t bases_scanned = 0, runs = 0, columns = 0, useful_columns = 0, filter_positions = 0;
        uint64_t graph_segments = 0;
        double ms_filter = 0;
        double ms_verify = 0, ms_scan = 0, ms_probe = 0;
        double ms_admit = 0, ms_launch = 0, ms_assemble = 0, ms_download = 0;  // wall time per phase
    } sum;
};

namespace pn {

static uint32_t k_of(const peanut_engine_params& p, uint32_t m) {
    return p.k_fixed != 0xFFFFFFFFu ? p.k_fixed : (uint32_t)(((uint64_t)m * p.k_permille + 999) / 1000);
}

// Device bytes of a launch of n reads of class c before any measurement: the index tables plus a
// generous per-read allowance that grows with the expected random q-gram hits.
// Expected q-gram hits per read of a class: measured, else the random hits of its longest reads
// in a uniform reference (twice, for repeats) plus their own q-grams.
static double hits_per_read(const peanut_engine* E, const ClassState& C, uint32_t q) {
    if (C.hits_per_read > 0) return C.hits_per_read;
    uint32_t mmax = 0;
    for (uint32_t m = 1; m <= (uint32_t)kMaxReadLen; ++m)
        if ((C.lenmask[m >> 5] >> (m & 31)) & 1u) mmax = m;
    const double nq = mmax >= q ? (double)(mmax - q + 1) : 1.0;
    return nq / C.stride * (2.0 * 2.0 * (double)E->ref->n / (double)(1ull << (2 * q))) + nq;
}

// Device bytes per result row held from its launch until its submission is assembled: the row
// itself (read, strand, end, distance: 14 B) and the assembly's sort keys, values and final
// arrays (about 48 B).
constexpr uint64_t kResultHoldBytes = 14 + 48;

static double launch_bytes(const peanut_engine* E, const ClassState& C, uint32_t q, uint64_t n) {
    const double fixed = (double)(((1ull << (2 * q)) + 31) / 32) * 8.0 + (80u << 20);
    double per = C.bytes_per_read;
    if (per <= 0) {
        const double nq = 256.0;
        const double rand = nq / C.stride * (2.0 * (double)E->ref->n / (double)(1ull << (2 * q)));
        per = 16384.0 + 64.0 * rand;
    }
    return fixed + per * (double)n;
}

// Whether every length in the mask admits (q, stride): the lemma threshold and the sampled
// threshold both at least 1.
static bool setting_ok(const peanut_engine* E, const uint32_t* lenmask, uint32_t q, uint32_t stride) {
    for (uint32_t m = 1; m <= (uint32_t)kMaxReadLen; ++m) {
        if (!((lenmask[m >> 5] >> (m & 31)) & 1u)) continue;
        const uint32_t k = k_of(E->p, m);
        if (m < q || (int64_t)m + 1 - (int64_t)q * (k + 1) < 1 || sampled_threshold_host(m - q + 1, q, k, stride) < 1)
            return false;
    }
    return true;
}

static uint64_t admission_bytes(const Submission* S) {
    const uint64_t copies = S->h_seq ? S->span + 8ull * (S->n_reads + 1) : 0;
    return copies + 5ull * S->n_reads + 64ull * S->n_reads + (16u << 20);  // classes, lists, result slack
}

static void set_failed(Submission* S, peanut_status st, const char* msg) {
    if (S->status == PEANUT_OK) {
        S->status = st;
        S->err = msg && *msg ? msg : "mapping failed";
    }
}

// Copies, validates and classifies a submission on stream s (no engine lock held).
static void admit(peanut_engine* E, Submission* S, cudaStream_t s) {
    if (S->h_seq) {
        S->d_seq.alloc(S->span ? S->span : 1, s);
        S->d_off.alloc((uint64_t)S->n_reads + 1, s);
        if (S->span)
            PN_CUDA(cudaMemcpyAsync(S->d_seq.p, S->h_seq + S->h_off[0], S->span, cudaMemcpyHostToDevice, s));
        PN_CUDA(cudaMemcpyAsync(S->d_off.p, S->h_off, ((uint64_t)S->n_reads + 1) * 8, cudaMemcpyHostToDevice, s));
        S->seq = S->d_seq.p;
        S->off = S->d_off.p;
        S->off0 = S->h_off[0];
    } else {
        S->seq = S->u_seq;
        S->off = S->u_off;
        PN_CUDA(cudaMemcpyAsync(&S->off0, S->u_off, 8, cudaMemcpyDeviceToHost, s));
        PN_CUDA(cudaStreamSynchronize(s));
    }
    const uint32_t n = S->n_reads;
    DBuf<uint8_t> cls(n, s);
    DBuf<uint32_t> meta(1 + kQSlots + kQSlots * 8, s);  // status, counts, length masks
    meta.zero();
    uint32_t* d_status = meta.p;
    uint32_t* d_counts = meta.p + 1;
    uint32_t* d_mask = meta.p + 1 + kQSlots;
    classify_k<<<grid_for(n, 256), 256, 0, s>>>(S->off, n, S->span, E->p.k_fixed, E->p.k_permille, 16,
                                                E->p.fixed_q, cls.p, d_counts, d_mask, d_status);
    PN_CHECK_LAUNCH();
    if (S->span) {
        check_bases_k<<<grid_for(S->span, 256, (unsigned)sm_count() * 8), 256, 0, s>>>(
            (const uint8_t*)S->seq, S->span, d_status);
        PN_CHECK_LAUNCH();
    }
    std::vector<uint32_t> h(meta.n);
    PN_CUDA(cudaMemcpyAsync(h.data(), meta.p, meta.n * 4, cudaMemcpyDeviceToHost, s));
    PN_CUDA(cudaStreamSynchronize(s));
    PN_REQUIRE(!(h[0] & kStBadLength), PEANUT_INVALID_ARG,
               "read offsets must ascend within the submission and give lengths 1..%d", kMaxReadLen);
    PN_REQUIRE(!(h[0] & kStBadBase), PEANUT_INVALID_ARG, "a read contains a byte other than A/C/G/T/N (either case)");
    PN_REQUIRE(!(h[0] & kStBadThreshold), PEANUT_INVALID_ARG,
               "a read admits no q with m + 1 - q(k + 1) >= 1%s", E->p.fixed_q ? " at the engine's fixed q" : "");
    for (int c = 1; c < kQSlots; ++c) {
        S->cnt[c] = h[1 + c];
        for (int w = 0; w < 8; ++w) S->lenmask[c][w] = h[1 + kQSlots + c * 8 + w];
        if (!S->cnt[c]) continue;
        S->classes++;
        S->list[c].alloc(S->cnt[c], s);
        exclusive_scan(ClassFlag{cls.p, (uint8_t)c}, ClassScatter{cls.p, (uint8_t)c, S->list[c].p}, n, nullptr, s);
    }
    PN_CUDA(cudaStreamSynchronize(s));
    S->remaining = n;
}

// Renumbers and sorts a submission's results into its own read ids and applies the best stratum
// if asked (no engine lock held); returns them in device memory, complete when s is.
static DeviceHits* assemble(peanut_engine* E, Submission* S, cudaStream_t s) {
    std::sort(S->parts.begin(), S->parts.end(), [](const Part& a, const Part& b) {
        return a.cls != b.cls ? a.cls < b.cls : a.x0 < b.x0;
    });
    uint64_t total = 0;
    for (const Part& P : S->parts) total += P.hi - P.lo;
    DeviceHits all;
    {
        DBuf<uint64_t> key(total ? total : 1, s), val(total ? total : 1, s);
        uint64_t at = 0;
        for (const Part& P : S->parts) {
            if (P.hi == P.lo) continue;
            const peanut_device_hits& h = P.launch->out->h;
            renumber_k<<<grid_for(P.hi - P.lo, 256, (unsigned)sm_count() * 16), 256, 0, s>>>(
                h.read_id, h.strand, h.end_pos, h.dist, P.lo, P.hi, P.base, S->list[P.cls].p + P.x0, key.p + at,
                val.p + at);
            PN_CHECK_LAUNCH();
            at += P.hi - P.lo;
        }
        if (S->classes > 1 && total > 1) {
            DBuf<uint64_t> kt(total, s), vt(total, s);
            int bits = 40;
            while ((1ull << (bits - 40)) < S->n_reads) ++bits;
            radix_sort_pairs(key.p, val.p, kt.p, vt.p, total, bits, s);
        }
        alloc_device_hits(&all, total, s);
        if (total) {
            unpack_k<<<grid_for(total, 256, (unsigned)sm_count() * 16), 256, 0, s>>>(key.p, val.p, total, all.h);
            PN_CHECK_LAUNCH();
        }
    }
    // every row is read: the launches' arrays may go
    PN_CUDA(cudaStreamSynchronize(s));
    S->parts.clear();
    DeviceHits* fin = new DeviceHits();
    try {
        if (S->mode == 1) {
            best_stratum(all.h, S->n_reads, fin, s);
            free_device_hits(&all);
        } else {
            fin->stream = s;
            fin->a = all.a;
            fin->h = all.h;
            all.h = peanut_device_hits{};
        }
    } catch (...) {
        free_device_hits(&all);
        free_device_hits(fin);
        delete fin;
        throw;
    }
    return fin;
}

struct LaunchOut {
    std::shared_ptr<Launch> launch;
    std::vector<uint64_t> bounds;  // result row of each segment start, plus the total
    peanut_map_stats st = {};
    std::vector<peanut_map_stats> runs;  // every mapping run of the launch (several when tuning)
    peanut_map_stats st_model = {};      // the run of the setting used from now on (memory model)
    uint64_t nqg_model = 0;
    uint64_t n_qgrams = 0, total = 0;
};

// Index + map of gathered reads with one setting; returns the results and timing.
static std::shared_ptr<Launch> map_setting(peanut_engine* E, const char* d_seq, const uint64_t* d_off, uint32_t n,
                                           uint64_t total, uint32_t q, uint32_t stride, cudaStream_t s,
                                           peanut_map_stats* st, uint64_t* nqg, float* ms) {
    peanut_params P = {};
    P.q = q;
    P.k_fixed = E->p.k_fixed;
    P.k_permille = E->p.k_permille;
    P.freq_cap = 0;
    P.stride = stride;
    P.stream = (void*)s;
    cudaEvent_t e0, e1;
    PN_CUDA(cudaEventCreate(&e0));
    PN_CUDA(cudaEventCreate(&e1));
    std::unique_ptr<peanut_reads, void (*)(peanut_reads*)> R(nullptr, [](peanut_reads* r) { delete r; });
    auto L = std::make_shared<Launch>();
    try {
        PN_CUDA(cudaEventRecord(e0, s));
        R.reset(index_batch(E->ref, d_seq, d_off, n, total, &P));
        L->out = map_batch(E->ref, R.get(), 0);
        PN_CUDA(cudaEventRecord(e1, s));
        PN_CUDA(cudaEventSynchronize(e1));
        cudaEventElapsedTime(ms, e0, e1);
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *st = R->stats;
    *nqg = R->n_qgrams;
    return L;
}

static double launch_measured_bytes(const peanut_map_stats& st, uint32_t n, uint64_t total, uint64_t nqg) {
    return 48.0 * st.hits + 12.0 * st.present_probes + 48.0 * st.candidates +
           (32.0 + (double)kResultHoldBytes) * st.results +
           40.0 * st.lowcx_ranges + 3.0 * total + 330.0 * n + 28.0 * nqg;
}

static LaunchOut run_launch(peanut_engine* E, int c, const std::vector<Segment>& segs, uint32_t n, bool tune,
                            uint32_t q_use, uint32_t stride_use, cudaStream_t s,
                            std::vector<std::pair<uint32_t, uint32_t>>* tried, uint32_t* best_q,
                            uint32_t* best_stride, float* best_pred) {
    // gather the reads into one batch
    std::vector<SegDev> hseg(segs.size());
    std::vector<uint32_t> hb(segs.size() + 1);
    for (size_t i = 0; i < segs.size(); ++i) {
        const Segment& g = segs[i];
        hseg[i] = SegDev{g.sub->seq, g.sub->off, g.sub->list[g.cls].p, g.sub->off0, g.x0, g.n, g.base, 0};
        hb[i] = g.base;
    }
    hb[segs.size()] = n;
    const uint32_t nseg = (uint32_t)segs.size();
    DBuf<SegDev> dseg(nseg, s);
    DBuf<uint32_t> dbase(nseg + 1, s);
    PN_CUDA(cudaMemcpyAsync(dseg.p, hseg.data(), nseg * sizeof(SegDev), cudaMemcpyHostToDevice, s));
    PN_CUDA(cudaMemcpyAsync(dbase.p, hb.data(), (nseg + 1) * 4, cudaMemcpyHostToDevice, s));
    DBuf<uint64_t> noff((uint64_t)n + 1, s), tot(1, s);
    exclusive_scan(GatherLen{dseg.p, nseg}, ArrayOut<uint64_t>{noff.p}, n, tot.p, s);
    PN_CUDA(cudaMemcpyAsync(noff.p + n, tot.p, 8, cudaMemcpyDeviceToDevice, s));
    const uint64_t total = to_host(tot.p, s);
    DBuf<char> buf(total ? total : 1, s);
    gather_copy_k<<<grid_for((uint64_t)n * 32, 256, (unsigned)sm_count() * 16), 256, 0, s>>>(dseg.p, nseg, n, noff.p,
                                                                                             buf.p);
    PN_CHECK_LAUNCH();

    LaunchOut out;
    out.total = total;
    if (!tune) {
        float ms = 0;
        out.launch = map_setting(E, buf.p, noff.p, n, total, q_use, stride_use, s, &out.st, &out.n_qgrams, &ms);
        out.runs.push_back(out.st);
        out.st_model = out.st;
        out.nqg_model = out.n_qgrams;
    } else {
        // candidate settings: q and q - 1 (if its random hits stay moderate), strides 1..4 that
        // every length of the class admits; the first (q, 1) is the plain setting and its
        // results are the ones kept
        std::vector<std::pair<uint32_t, uint32_t>> cand;
        uint32_t mask[8];
        for (int w = 0; w < 8; ++w) mask[w] = 0;
        for (const Segment& g : segs)
            for (int w = 0; w < 8; ++w) mask[w] |= g.sub->lenmask[c][w];
        for (uint32_t q = (uint32_t)c; q + 1 >= (uint32_t)c && q >= 1; --q) {
            const double rand_per_qgram = 2.0 * (double)E->ref->n / (double)(1ull << (2 * q));
            if (q != (uint32_t)c && (E->p.fixed_q || rand_per_qgram * 200.0 > 2.0e4)) break;
            // strides up to q (disjoint q-grams, the pigeonhole case) for the class's own q
            static const uint32_t kStrides[] = {1, 2, 3, 4, 6, 8, 12, 16};
            for (uint32_t st : kStrides)
                if (st <= (q == (uint32_t)c ? q : 4u) && setting_ok(E, mask, q, st)) cand.push_back({q, st});
            if (q == 1) break;
        }
        float best = 1e30f;
        for (size_t i = 0; i < cand.size(); ++i) {
            peanut_map_stats st = {};
            uint64_t nqg = 0;
            float ms = 0;
            std::shared_ptr<Launch> L =
                map_setting(E, buf.p, noff.p, n, total, cand[i].first, cand[i].second, s, &st, &nqg, &ms);
            // the launch size this setting would run at: max_reads, or fewer where its hits per
            // read or device bytes per read (as measured here, with the model's margin) cap it
            const double hpr = 1.25 * (double)st.hits / n + 1.0;
            const double bpr = 1.25 * launch_measured_bytes(st, n, total, nqg) / n + 1.0;
            const double plan = std::max((double)n, std::min({(double)E->p.max_reads, kMaxLaunchHits / hpr,
                                                             0.5 * (double)E->budget / bpr}));
            // the probe pass costs the same for any batch size; the rest grows with the reads
            const double fixed = st.ms_probe_kernel;
            const double pred = (fixed + ((double)ms - fixed) * plan / (double)n) / plan * 1e6;
            tried->push_back(cand[i]);
            out.runs.push_back(st);
            if (pred < best) {
                best = (float)pred;
                *best_q = cand[i].first;
                *best_stride = cand[i].second;
                out.st_model = st;
                out.nqg_model = nqg;
            }
            if (i == 0) {
                out.launch = L;
                out.st = st;
                out.n_qgrams = nqg;
            }
        }
        *best_pred = best;
    }
    // result rows of each segment
    const peanut_device_hits& h = out.launch->out->h;
    DBuf<uint64_t> bnd(nseg + 1, s);
    seg_bounds_k<<<grid_for(nseg + 1, 128), 128, 0, s>>>(h.read_id, h.n, dbase.p, nseg + 1, bnd.p);
    PN_CHECK_LAUNCH();
    out.bounds.resize(nseg + 1);
    PN_CUDA(cudaMemcpyAsync(out.bounds.data(), bnd.p, (nseg + 1) * 8, cudaMemcpyDeviceToHost, s));
    PN_CUDA(cudaStreamSynchronize(s));
    return out;
}

// Removes a submission's unconsumed reads from the class queues (engine lock held).
static void unqueue(peanut_engine* E, Submission* S) {
    for (int c = 1; c < kQSlots; ++c) {
        if (S->next[c] >= S->cnt[c]) continue;
        ClassState& C = E->cls[c];
        C.waiting -= S->cnt[c] - S->next[c];
        S->next[c] = S->cnt[c];
        auto it = std::find(C.queue.begin(), C.queue.end(), S);
        if (it != C.queue.end()) C.queue.erase(it);
    }
}

static void finish(peanut_engine* E, Submission* S) {  // engine lock held
    unqueue(E, S);
    E->reserved -= S->reserved;
    S->reserved = 0;
    for (auto& l : S->list) l.reset();
    S->d_seq.reset();
    S->d_off.reset();
    S->parts.clear();
    S->done = true;
    E->n_completed++;
    E->cv_done.notify_all();
    E->cv_work.notify_all();
}

static void fail_and_maybe_finish(peanut_engine* E, Submission* S, peanut_status st, const char* msg) {
    set_failed(S, st, msg);
    if (S->inflight == 0 && !S->done) finish(E, S);
}

static int pick_class(peanut_engine* E) {
    int best = -1, best_untuned = -1;
    uint64_t order = UINT64_MAX, order_untuned = UINT64_MAX;
    for (int c = 1; c < kQSlots; ++c) {
        ClassState& C = E->cls[c];
        while (!C.queue.empty() && C.queue.front()->status != PEANUT_OK) {  // drop failed submissions
            Submission* S = C.queue.front();
            C.waiting -= S->cnt[c] - S->next[c];
            S->remaining -= S->cnt[c] - S->next[c];
            S->next[c] = S->cnt[c];
            C.queue.pop_front();
            if (S->inflight == 0 && !S->done) finish(E, S);
        }
        if (C.queue.empty() || C.tuning) continue;
        if (C.queue.front()->order < order) {
            order = C.queue.front()->order;
            best = c;
        }
        if (E->p.autotune && !C.tuned && C.queue.front()->order < order_untuned) {
            order_untuned = C.queue.front()->order;
            best_untuned = c;
        }
    }
    return best_untuned >= 0 ? best_untuned : best;  // classes still to be tuned go first
}

static void executor(peanut_engine* E, int idx) {
    cudaSetDevice(E->device);
    use_pool_on_this_thread();
    use_graphs_on_this_thread(E->p.graphs != 0);
    cudaStream_t s = E->streams[idx];
    std::unique_lock<std::mutex> lk(E->mu);
    while (!E->stop) {
        // a tuning run has the GPU to itself: nothing else starts meanwhile
        if (E->tuning_active) {
            E->cv_work.wait(lk);
            continue;
        }
        // a launch from the class with the oldest waiting reads
        const int c = pick_class(E);
        if (c < 0) {
            E->cv_work.wait(lk);
            continue;
        }
        ClassState& C = E->cls[c];
        if (!C.q) {
            C.q = (uint32_t)c;
            C.stride = 1;
        }
        const bool tune = E->p.autotune && !C.tuned;
        if (tune && E->running > 0) {  // wait for the work in flight to drain first
            E->cv_work.wait(lk);
            continue;
        }
        // the largest launch of this class: max_reads, and at most kMaxLaunchHits expected q-gram
        // hits (the sorts of one launch index 32 bits)
        const double hpr = hits_per_read(E, C, C.q);
        uint64_t cap = tune ? std::min(kTuneReads, E->p.max_reads) : E->p.max_reads;
        if ((double)cap * hpr > kMaxLaunchHits) cap = std::max<uint64_t>(1, (uint64_t)(kMaxLaunchHits / hpr));
        // while another launch keeps the GPU busy and submissions are still being admitted, let
        // the class fill up to half a launch instead of starting a small one
        if (!tune && E->launching > 0 && C.waiting < cap / 2 && (!E->pending.empty() || E->admitting > 0)) {
            E->cv_work.wait(lk);
            continue;
        }
        uint64_t n = std::min<uint64_t>(C.waiting, cap);
        const double avail = (double)E->budget - (double)E->reserved;
        while (n > kMinLaunch && launch_bytes(E, C, C.q, n) > avail) n >>= 1;
        if (launch_bytes(E, C, C.q, n) > avail && E->running > 0) {
            E->cv_work.wait(lk);  // memory frees up when a launch or submission finishes
            continue;
        }
        const uint64_t need = (uint64_t)launch_bytes(E, C, C.q, n);
        std::vector<Segment> segs;
        uint32_t mask[8] = {};
        uint32_t taken = 0;
        while (taken < n && !C.queue.empty()) {
            Submission* S = C.queue.front();
            const uint32_t t = (uint32_t)std::min<uint64_t>(S->cnt[c] - S->next[c], n - taken);
            segs.push_back(Segment{S, (uint32_t)c, S->next[c], t, taken});
            for (int w = 0; w < 8; ++w) mask[w] |= S->lenmask[c][w];
            S->next[c] += t;
            S->inflight++;
            taken += t;
            if (S->next[c] == S->cnt[c]) C.queue.pop_front();
        }
        C.waiting -= taken;
        if (tune) {
            C.tuning = true;
            E->tuning_active++;
        }
        // the class's setting, unless a length in this launch does not admit it
        const bool keep = setting_ok(E, mask, C.q, C.stride);
        const uint32_t q_use = keep ? C.q : (uint32_t)c, stride_use = keep ? C.stride : 1;
        E->reserved += need;
        E->reserved_peak = std::max(E->reserved_peak, E->reserved);
        E->running++;
        E->launching++;
        lk.unlock();

        peanut_status st = PEANUT_OK;
        std::string msg;
        LaunchOut L;
        std::vector<std::pair<uint32_t, uint32_t>> tried;
        uint32_t bq = q_use, bs = stride_use;  // (read under the lock above)
        float bpred = 0;
        const double t_launch = wall_ms();
        try {
            L = run_launch(E, c, segs, taken, tune, q_use, stride_use, s, &tried, &bq, &bs, &bpred);
        } catch (const Fail& f) {
            st = f.st;
            msg = peanut_last_error();
        } catch (...) {
            st = PEANUT_CUDA_ERROR;
            msg = "launch failed";
        }

        lk.lock();
        E->sum.ms_launch += wall_ms() - t_launch;
        E->running--;
        E->launching--;
        E->reserved -= need;
        if (tune) {
            C.tuning = false;
            E->tuning_active--;
            if (st == PEANUT_OK) {
                C.tuned = true;
                C.q = bq;
                C.stride = bs;
                C.tuned_ms_per_mread = bpred;
                C.tune_candidates = (uint32_t)tried.size();
                E->n_tuning += tried.size() > 0 ? tried.size() - 1 : 0;
            }
        }
        std::vector<Submission*> ready;
        if (st == PEANUT_OK) {
            C.launches++;
            C.reads += taken;
            E->n_launches++;
            E->n_reads += taken;
            C.cap = default_freq_cap(E->ref->n, q_use);
            // the class's memory model, from the setting it uses: set by the tuning launch, raised by
            // any later launch that needed more
            const double nr = (double)std::max<uint32_t>(taken, 1);
            const double per = launch_measured_bytes(L.st_model, taken, L.total, L.nqg_model) / nr;
            const double hpr = (double)L.st_model.hits / nr;
            C.bytes_per_read = tune ? 1.25 * per : std::max(C.bytes_per_read, 1.25 * per);
            C.hits_per_read = tune ? 1.25 * hpr : std::max(C.hits_per_read, 1.25 * hpr);
            for (const peanut_map_stats& m : L.runs) {
                E->sum.hits += m.hits;
                E->sum.candidates += m.candidates;
                E->sum.word_columns += m.candidate_word_columns;
                E->sum.columns += m.candidate_columns;
                E->sum.useful_columns += m.useful_columns;
                E->sum.filter_positions += m.filter_positions;
                E->sum.graph_segments += m.graph_segments;
                E->sum.ms_filter += m.ms_filter_kernel;
                E->sum.present_probes += m.present_probes;
                E->sum.results += m.results;
                E->sum.ms_verify += m.ms_verify_kernel;
                E->sum.ms_scan += m.ms_scan_kernel;
                E->sum.ms_probe += m.ms_probe_kernel;
                E->sum.bases_scanned += E->ref->n;
                E->sum.runs += 1;
            }
        }
        for (size_t i = 0; i < segs.size(); ++i) {
            Submission* S = segs[i].sub;
            S->inflight--;
            if (st == PEANUT_OK && S->status == PEANUT_OK) {
                Part P;
                P.launch = L.launch;
                P.lo = L.bounds[i];
                P.hi = L.bounds[i + 1];
                // the part's rows stay in device memory until the submission is assembled, and the
                // assembly needs its own arrays for them: both are held against the budget until
                // the submission finishes
                const uint64_t hold = (P.hi - P.lo) * kResultHoldBytes;
                S->reserved += hold;
                E->reserved += hold;
                E->reserved_peak = std::max(E->reserved_peak, E->reserved);
                P.base = segs[i].base;
                P.cls = (uint32_t)c;
                P.x0 = segs[i].x0;
                S->parts.push_back(std::move(P));
                S->remaining -= segs[i].n;
                if (S->remaining == 0) ready.push_back(S);
            } else {
                S->remaining -= segs[i].n;
                fail_and_maybe_finish(E, S, st == PEANUT_OK ? S->status : st, msg.c_str());
            }
        }
        L.launch.reset();
        if (!ready.empty()) {
            E->running++;
            lk.unlock();
            std::vector<std::pair<peanut_status, std::string>> res(ready.size());
            std::vector<Download> outs(ready.size());
            const double t_asm = wall_ms();
            for (size_t i = 0; i < ready.size(); ++i) {
                try {
                    DeviceHits* fin = assemble(E, ready[i], s);
                    outs[i].fin = fin;
                    if (ready[i]->on_device) {
                        PN_CUDA(cudaStreamSynchronize(s));
                        fin->stream = nullptr;  // the caller may free it after the engine is gone
                    } else {
                        PN_CUDA(cudaEventCreateWithFlags(&outs[i].ready, cudaEventDisableTiming));
                        PN_CUDA(cudaEventRecord(outs[i].ready, s));
                    }
                } catch (const Fail& f) {
                    res[i] = {f.st, peanut_last_error()};
                } catch (...) {
                    res[i] = {PEANUT_CUDA_ERROR, "assembly failed"};
                }
            }
            lk.lock();
            E->sum.ms_assemble += wall_ms() - t_asm;
            E->running--;
            for (size_t i = 0; i < ready.size(); ++i) {
                Submission* S = ready[i];
                if (res[i].first != PEANUT_OK) {
                    if (outs[i].fin) {
                        free_device_hits(outs[i].fin);
                        delete outs[i].fin;
                    }
                    if (outs[i].ready) cudaEventDestroy(outs[i].ready);
                    set_failed(S, res[i].first, res[i].second.c_str());
                    finish(E, S);
                } else if (S->on_device) {
                    S->dresult = outs[i].fin;
                    finish(E, S);
                } else {
                    outs[i].sub = S;  // the copy to the host runs on the I/O thread
                    E->downloads.push_back(outs[i]);
                }
            }
        }
        E->cv_work.notify_all();
    }
}

// The I/O thread: every host<->device copy of the engine, so that executors only launch work.
// Results waiting to go to the host come first (they hold device memory), then admissions in
// submission order while their footprint fits (none while a tuning run has the GPU).
static void io_loop(peanut_engine* E) {
    cudaSetDevice(E->device);
    use_pool_on_this_thread();
    cudaStream_t s = E->io_stream;
    std::unique_lock<std::mutex> lk(E->mu);
    while (!E->stop) {
        if (!E->downloads.empty()) {
            Download D = E->downloads.front();
            E->downloads.pop_front();
            lk.unlock();
            peanut_status st = PEANUT_OK;
            std::string msg;
            HostHits* h = nullptr;
            const double t0 = wall_ms();
            try {
                PN_CUDA(cudaStreamWaitEvent(s, D.ready, 0));
                h = download_hits(D.fin->h, s);
            } catch (const Fail& f) {
                st = f.st;
                msg = peanut_last_error();
            } catch (...) {
                st = PEANUT_CUDA_ERROR;
                msg = "copy of the results failed";
            }
            D.fin->stream = s;  // copied (or failed) on this stream: release it here
            free_device_hits(D.fin);
            delete D.fin;
            cudaEventDestroy(D.ready);
            lk.lock();
            E->sum.ms_download += wall_ms() - t0;
            if (st != PEANUT_OK) set_failed(D.sub, st, msg.c_str());
            else D.sub->result = h;
            finish(E, D.sub);
            continue;
        }
        if (!E->pending.empty() && !E->tuning_active) {
            Submission* S = E->pending.front();
            const uint64_t need = admission_bytes(S);
            if (need > E->budget) {
                E->pending.pop_front();
                set_failed(S, PEANUT_NO_MEMORY, "submission does not fit the engine's device-memory budget");
                finish(E, S);
                continue;
            }
            if (E->reserved + need <= E->budget || E->running == 0) {
                E->pending.pop_front();
                E->reserved += need;
                E->reserved_peak = std::max(E->reserved_peak, E->reserved);
                S->reserved = need;
                E->running++;
                E->admitting++;
                lk.unlock();
                peanut_status st = PEANUT_OK;
                std::string msg;
                const double t0 = wall_ms();
                try {
                    admit(E, S, s);
                } catch (const Fail& f) {
                    st = f.st;
                    msg = peanut_last_error();
                } catch (...) {
                    st = PEANUT_CUDA_ERROR;
                    msg = "admission failed";
                }
                lk.lock();
                E->sum.ms_admit += wall_ms() - t0;
                E->running--;
                E->admitting--;
                if (st != PEANUT_OK) {
                    set_failed(S, st, msg.c_str());
                    finish(E, S);
                } else {
                    S->order = E->next_order++;
                    for (int c = 1; c < kQSlots; ++c) {
                        if (!S->cnt[c]) continue;
                        ClassState& C = E->cls[c];
                        C.queue.push_back(S);
                        C.waiting += S->cnt[c];
                        for (int w = 0; w < 8; ++w) C.lenmask[w] |= S->lenmask[c][w];
                    }
                }
                E->cv_work.notify_all();
                continue;
            }
        }
        E->cv_work.wait(lk);
    }
}

static void destroy_engine_impl(peanut_engine* E) {
    {
        std::lock_guard<std::mutex> lk(E->mu);
        E->stop = true;
    }
    E->cv_work.notify_all();
    for (auto& t : E->threads)
        if (t.joinable()) t.join();
    for (Download& D : E->downloads) {
        free_device_hits(D.fin);
        delete D.fin;
        cudaEventDestroy(D.ready);
    }
    for (auto& kv : E->subs) {
        Submission* S = kv.second;
        if (S->result) free_host_hits(S->result);
        if (S->dresult) {
            free_device_hits(S->dresult);
            delete S->dresult;
        }
        delete S;
    }
    for (auto& s : E->streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    if (E->io_stream) {
        cudaStreamSynchronize(E->io_stream);
        cudaStreamDestroy(E->io_stream);
    }
    E->magic = 0;
    delete E;
}

void destroy_engine(peanut_engine* E) { destroy_engine_impl(E); }

static uint64_t free_device_bytes() {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool;
    uint64_t cached = 0;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t resv = 0, used = 0;
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &resv);
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
        cached = resv > used ? resv - used : 0;
    }
    cudaGetLastError();
    return (uint64_t)fr + cached;
}

}  // namespace pn

using namespace pn;

template <class F>
static peanut_status eguard(F&& f) {
    clear_error();
    cudaGetLastError();
    try {
        f();
        return PEANUT_OK;
    } catch (const Fail& e) {
        return e.st;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return PEANUT_NO_MEMORY;
    } catch (const std::system_error&) {
        set_error("could not start an executor thread");
        return PEANUT_CUDA_ERROR;
    } catch (...) {
        set_error("unexpected internal error");
        return PEANUT_CUDA_ERROR;
    }
}

static peanut_engine* engine_of(peanut_engine* e) {
    PN_REQUIRE(e && e->magic == kMagicEngine, PEANUT_INVALID_ARG, "bad engine");
    return e;
}

extern "C" {

peanut_status peanut_engine_create(const peanut_ref* ref, const peanut_engine_params* p, peanut_engine** out) {
    return eguard([&] {
        PN_REQUIRE(ref && ref->magic == kMagicRef && p && out, PEANUT_INVALID_ARG, "bad reference or NULL argument");
        PN_REQUIRE(p->k_fixed != 0xFFFFFFFFu || p->k_permille <= 1000, PEANUT_INVALID_ARG, "k_permille > 1000");
        PN_REQUIRE(p->executors <= (uint32_t)kMaxExecutors, PEANUT_INVALID_ARG, "executors = %u outside 0..%d",
                   p->executors, kMaxExecutors);
        PN_REQUIRE(p->max_reads <= kMaxReads, PEANUT_INVALID_ARG, "max_reads above 2^23");
        PN_REQUIRE(p->fixed_q <= 16, PEANUT_UNSUPPORTED, "fixed_q = %u outside 0..16", p->fixed_q);
        *out = nullptr;
        peanut_engine* E = new peanut_engine();
        E->ref = ref;
        E->p = *p;
        if (!E->p.executors) E->p.executors = 2;
        if (!E->p.max_reads) E->p.max_reads = 1u << 22;
        cudaGetDevice(&E->device);
        if (p->hbm_budget) {
            E->budget = p->hbm_budget;
        } else {
            const double fr = (double)free_device_bytes();
            E->budget = (uint64_t)std::max(0.0, 0.9 * fr - (double)(4ull << 30));
        }
        try {
            for (uint32_t i = 0; i < E->p.executors; ++i) {
                cudaStream_t s;
                PN_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
                E->streams.push_back(s);
            }
            PN_CUDA(cudaStreamCreateWithFlags(&E->io_stream, cudaStreamNonBlocking));
            for (uint32_t i = 0; i < E->p.executors; ++i) E->threads.emplace_back(executor, E, (int)i);
            E->threads.emplace_back(io_loop, E);
        } catch (...) {
            destroy_engine_impl(E);
            throw;
        }
        *out = E;
    });
}

static peanut_status submit_common(peanut_engine* e, const char* hs, const uint64_t* ho, const char* ds,
                                   const uint64_t* dof, uint32_t n_reads, uint64_t span, int mode, uint64_t* ticket) {
    return eguard([&] {
        peanut_engine* E = engine_of(e);
        PN_REQUIRE(ticket, PEANUT_INVALID_ARG, "NULL ticket");
        PN_REQUIRE((mode & 0xFF) <= 1 && (mode & ~0x1FF) == 0, PEANUT_INVALID_ARG,
                   "mode must be 0 (all) or 1 (best stratum), optionally | PEANUT_RESULT_ON_DEVICE");
        PN_REQUIRE(n_reads >= 1 && n_reads <= kEngineMaxReads, PEANUT_INVALID_ARG, "n_reads = %u outside 1..2^24",
                   n_reads);
        Submission* S = new Submission();
        S->mode = mode & 0xFF;
        S->on_device = (mode & PEANUT_RESULT_ON_DEVICE) != 0;
        S->n_reads = n_reads;
        S->h_seq = hs;
        S->h_off = ho;
        S->u_seq = ds;
        S->u_off = dof;
        S->span = span;
        std::lock_guard<std::mutex> lk(E->mu);
        S->ticket = E->next_ticket++;
        E->subs[S->ticket] = S;
        E->pending.push_back(S);
        E->n_submitted++;
        *ticket = S->ticket;
        E->cv_work.notify_all();
    });
}

peanut_status peanut_engine_submit(peanut_engine* e, const char* seqs, const uint64_t* offsets, uint32_t n_reads,
                                   int mode, uint64_t* ticket) {
    if (!seqs || !offsets) {
        set_error("NULL argument");
        return PEANUT_INVALID_ARG;
    }
    if (n_reads >= 1 && n_reads <= kEngineMaxReads) {
        for (uint32_t i = 0; i < n_reads; ++i)
            if (offsets[i + 1] < offsets[i]) {
                set_error("read offsets must ascend");
                return PEANUT_INVALID_ARG;
            }
    }
    const uint64_t span = (n_reads >= 1 && n_reads <= kEngineMaxReads) ? offsets[n_reads] - offsets[0] : 0;
    return submit_common(e, seqs, offsets, nullptr, nullptr, n_reads, span, mode, ticket);
}

peanut_status peanut_engine_submit_device(peanut_engine* e, const char* d_seqs, const uint64_t* d_offsets,
                                          uint32_t n_reads, uint64_t total_bases, int mode, uint64_t* ticket) {
    if (!d_seqs || !d_offsets) {
        set_error("NULL argument");
        return PEANUT_INVALID_ARG;
    }
    return submit_common(e, nullptr, nullptr, d_seqs, d_offsets, n_reads, total_bases, mode, ticket);
}

// Waits for a submission and takes it out of the engine (engine lock taken here).
static std::unique_ptr<Submission> take(peanut_engine* E, uint64_t ticket, int64_t timeout_ms, int want_device) {
    std::unique_lock<std::mutex> lk(E->mu);
    auto it = E->subs.find(ticket);
    PN_REQUIRE(it != E->subs.end(), PEANUT_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    Submission* S = it->second;
    PN_REQUIRE(!(want_device && !S->on_device), PEANUT_INVALID_ARG,
               "submission %llu was not made with PEANUT_RESULT_ON_DEVICE", (unsigned long long)ticket);
    auto ready = [&] { return S->done; };
    if (timeout_ms < 0) {
        E->cv_done.wait(lk, ready);
    } else if (!E->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
        set_error("submission %llu still running", (unsigned long long)ticket);
        throw Fail{PEANUT_TIMEOUT};
    }
    E->subs.erase(it);
    std::unique_ptr<Submission> own(S);
    if (S->status != PEANUT_OK) {
        set_error("%s", S->err.c_str());
        throw Fail{S->status};
    }
    return own;
}

peanut_status peanut_engine_wait(peanut_engine* e, uint64_t ticket, int64_t timeout_ms, peanut_hits** out) {
    return eguard([&] {
        peanut_engine* E = engine_of(e);
        PN_REQUIRE(out, PEANUT_INVALID_ARG, "NULL out");
        *out = nullptr;
        std::unique_ptr<Submission> S = take(E, ticket, timeout_ms, 0);
        if (S->dresult) {  // a device result asked for on the host: copy it down on the legacy stream
            HostHits* h = nullptr;
            try {
                h = download_hits(S->dresult->h, nullptr);
            } catch (...) {
                free_device_hits(S->dresult);
                delete S->dresult;
                S->dresult = nullptr;
                throw;
            }
            free_device_hits(S->dresult);
            delete S->dresult;
            S->dresult = nullptr;
            *out = &h->h;
            return;
        }
        *out = &S->result->h;
        S->result = nullptr;
    });
}

peanut_status peanut_engine_wait_device(peanut_engine* e, uint64_t ticket, int64_t timeout_ms,
                                        peanut_device_hits** out) {
    return eguard([&] {
        peanut_engine* E = engine_of(e);
        PN_REQUIRE(out, PEANUT_INVALID_ARG, "NULL out");
        *out = nullptr;
        std::unique_ptr<Submission> S = take(E, ticket, timeout_ms, 1);
        *out = &S->dresult->h;
        S->dresult = nullptr;
    });
}

peanut_status peanut_engine_get_stats(peanut_engine* e, peanut_engine_stats* out) {
    return eguard([&] {
        peanut_engine* E = engine_of(e);
        PN_REQUIRE(out, PEANUT_INVALID_ARG, "NULL out");
        std::lock_guard<std::mutex> lk(E->mu);
        *out = peanut_engine_stats{};
        out->submissions = E->n_submitted;
        out->completed = E->n_completed;
        out->reads = E->n_reads;
        out->launches = E->n_launches;
        out->tuning_launches = E->n_tuning;
        out->hbm_budget = E->budget;
        out->hbm_reserved_peak = E->reserved_peak;
        out->map_runs = E->sum.runs;
        out->hits = E->sum.hits;
        out->candidates = E->sum.candidates;
        out->candidate_word_columns = E->sum.word_columns;
        out->present_probes = E->sum.present_probes;
        out->results = E->sum.results;
        out->bases_scanned = E->sum.bases_scanned;
        out->ms_verify_kernel = E->sum.ms_verify;
        out->ms_scan_kernel = E->sum.ms_scan;
        out->ms_probe_kernel = E->sum.ms_probe;
        out->ms_admit = E->sum.ms_admit;
        out->ms_launch = E->sum.ms_launch;
        out->ms_assemble = E->sum.ms_assemble;
        out->ms_download = E->sum.ms_download;
        out->pageable_result_blocks = pageable_blocks();
        out->candidate_columns = E->sum.columns;
        out->useful_columns = E->sum.useful_columns;
        out->filter_positions = E->sum.filter_positions;
        out->ms_filter_kernel = E->sum.ms_filter;
        out->graph_segments = E->sum.graph_segments;
        for (int c = 1; c < kQSlots && out->n_classes < 16; ++c) {
            const ClassState& C = E->cls[c];
            if (!C.launches && !C.waiting && C.queue.empty()) continue;
            peanut_engine_class& o = out->cls[out->n_classes++];
            o.q_class = (uint32_t)c;
            o.q = C.q;
            o.stride = C.stride;
            o.freq_cap = C.cap;
            o.launches = C.launches;
            o.reads = C.reads;
            o.bytes_per_read = (uint64_t)C.bytes_per_read;
            o.tuned_ms_per_mread = C.tuned_ms_per_mread;
            o.tune_candidates = C.tune_candidates;
        }
    });
}

}  // extern "C"
