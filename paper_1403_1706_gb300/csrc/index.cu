// Reference packing, the reference's frequent-q-gram clusters, and the q-group index over reads.
//
// Encoding (Section "The q-group index"): A=00 C=01 G=10 T=11, a q-gram is the 2q-bit number
// with its first base most significant.  The index is Algorithm 1 run over the CANONICAL code
// c = min(g, revcomp(g)) of every read q-gram, so one index serves both strands; each
// occurrence records whether the read holds c itself or its reverse complement.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <mutex>

#include "prims.cuh"

namespace pn {

__constant__ uint8_t kCodeLut[256];  // A/C/G/T (either case) -> 0..3, N/n -> 4, else 0xFF

static void init_lut() {
    static std::mutex mu;
    static std::atomic<bool> done{false};
    if (done.load()) return;
    std::lock_guard<std::mutex> lock(mu);
    if (done.load()) return;
    uint8_t lut[256];
    for (int i = 0; i < 256; ++i) lut[i] = 0xFF;
    const char* up = "ACGT";
    const char* lo = "acgt";
    for (int c = 0; c < 4; ++c) {
        lut[(uint8_t)up[c]] = (uint8_t)c;
        lut[(uint8_t)lo[c]] = (uint8_t)c;
    }
    lut['N'] = 4;
    lut['n'] = 4;
    PN_CUDA(cudaMemcpyToSymbol(kCodeLut, lut, sizeof(lut)));
    done = true;
}

// ---- unknown bases -----------------------------------------------------------------------
//
// Section "The q-group index" (encoding paragraph) turns an unknown base N into a random base.
// Here the draw is reproducible: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014: the state steps by
// the odd constant 0x9E3779B97F4A7C15, each output is the state through the generator's
// finalizer).  Reference position p takes the top two bits of output p + 1 of the generator
// seeded with the reference's seed; offset i of a read takes those of output i + 1 of the one
// seeded with (seed XOR the FNV-1a 64 hash of the read's upper-cased bytes), so a read's bases
// do not depend on the batch it arrives in.

__host__ __device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + i * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ---- reference packing --------------------------------------------------------------------

// One packed word (16 bases) per thread; bytes at or beyond len pack as A (never read as data).
// An N takes its seeded base and sets its bit in nmask (bit t of word w = base 16 w + t), from
// which the gaps are found.
__global__ void pack_reference_k(const uint8_t* __restrict__ ascii, uint64_t len, uint64_t base0, uint64_t seed,
                                 uint32_t* __restrict__ words, uint16_t* __restrict__ nmask, uint32_t* status) {
    const uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t b0 = w * 16;
    if (b0 >= len) return;
    uint8_t buf[16];
    if (b0 + 16 <= len) {
        const uint4 v = *reinterpret_cast<const uint4*>(ascii + b0);
        *reinterpret_cast<uint4*>(buf) = v;
    } else {
        for (int t = 0; t < 16; ++t) buf[t] = b0 + t < len ? ascii[b0 + t] : 'A';
    }
    uint32_t word = 0, nm = 0;
    bool bad = false;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        uint32_t c = kCodeLut[buf[t]];
        bad |= c > 4;
        if (c == 4) {
            c = (uint32_t)(splitmix64_at(seed, base0 + b0 + t + 1) >> 62);
            nm |= 1u << t;
        }
        word |= (c & 3u) << (30 - 2 * t);
    }
    words[w] = word;
    nmask[w] = (uint16_t)nm;
    if (bad) atomicOr(status, kStBadBase);
    if (nm) atomicOr(status, kStHasN);
}

// Boundaries of the runs of N: positions p where N-ness changes (p is N and p - 1 is not, or the
// reverse), from the mask read as 32-bit words (bit b of word i = base 32 i + b; the mask's zero
// padding ends a run that reaches the end).  Pass 0 counts them, pass 1 lists them (unordered).
template <bool kList>
__global__ void n_edges_k(const uint32_t* __restrict__ m32, uint64_t nw, unsigned long long* count,
                          uint64_t* __restrict__ edges, uint64_t cap) {
    uint32_t local = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t cur = m32[i], prev = i ? m32[i - 1] : 0u;
        uint32_t t = cur ^ ((cur << 1) | (prev >> 31));
        if (!kList) {
            local += __popc(t);
            continue;
        }
        while (t) {
            const uint32_t b = __ffs(t) - 1;
            t &= t - 1;
            const unsigned long long x = atomicAdd(count, 1ull);
            if (x < cap) edges[x] = i * 32 + b;
        }
    }
    if (!kList && local) atomicAdd(count, (unsigned long long)local);
}

constexpr uint64_t kMaxNEdges = 1ull << 27;  // run boundaries of N the packing lists (2^26 runs)

void pack_reference(peanut_ref* ref, const char* host_seq, uint64_t len, const uint64_t* contig_starts,
                    uint32_t n_contigs, uint32_t gap_min, uint64_t seed, cudaStream_t s) {
    init_lut();
    std::vector<uint64_t> cs;
    if (contig_starts && n_contigs)
        cs.assign(contig_starts, contig_starts + n_contigs);
    else
        cs.push_back(0);
    PN_REQUIRE(cs[0] == 0, PEANUT_INVALID_ARG, "the first contig must start at 0");
    for (size_t c = 1; c < cs.size(); ++c)
        PN_REQUIRE(cs[c] > cs[c - 1] && cs[c] < len, PEANUT_INVALID_ARG,
                   "contig starts must ascend strictly and lie inside the reference (contig %zu)", c);
    PN_REQUIRE(gap_min >= 1, PEANUT_INVALID_ARG, "gap_min must be at least 1");
    ref->n = len;
    ref->n_seed = seed;
    ref->n_contigs = (uint32_t)cs.size();
    ref->n_words = (len + 15) / 16 + 8;  // lookahead padding for the scan's 64-bit windows
    ref->packed.alloc(ref->n_words, s);
    ref->packed.zero();
    // N mask: one 16-bit word per packed word, an even count and one zero 32-bit word past the end
    const uint64_t nw16 = (((len + 15) / 16) + 3) & ~1ull;
    DBuf<uint16_t> nmask(nw16, s);
    nmask.zero();
    DBuf<uint32_t> status(1, s);
    status.zero();
    const uint64_t chunk = 1ull << 30;  // bases per upload (multiple of 16)
    DBuf<uint8_t> tmp(len < chunk ? ((len + 15) / 16) * 16 : chunk, s);
    for (uint64_t b = 0; b < len; b += chunk) {
        const uint64_t nb = len - b < chunk ? len - b : chunk;
        PN_CUDA(cudaMemcpyAsync(tmp.p, host_seq + b, nb, cudaMemcpyHostToDevice, s));
        const uint64_t nw = (nb + 15) / 16;
        pack_reference_k<<<grid_for(nw, 256), 256, 0, s>>>(tmp.p, nb, b, seed, ref->packed.p + b / 16,
                                                            nmask.p + b / 16, status.p);
        PN_CHECK_LAUNCH();
    }
    tmp.reset();
    const uint32_t st = to_host(status.p, s);
    PN_REQUIRE(!(st & kStBadBase), PEANUT_INVALID_ARG, "reference contains a byte other than A/C/G/T/N (either case)");
    // runs of N as [start, end) pairs, ascending
    std::vector<uint64_t> runs;
    if (st & kStHasN) {
        const uint64_t nw32 = nw16 / 2;
        const unsigned g = grid_for(nw32, 256, (unsigned)sm_count() * 16);
        DBuf<unsigned long long> cnt(1, s);
        cnt.zero();
        n_edges_k<false><<<g, 256, 0, s>>>(reinterpret_cast<const uint32_t*>(nmask.p), nw32, cnt.p, nullptr, 0);
        PN_CHECK_LAUNCH();
        const uint64_t E = to_host(cnt.p, s);
        PN_REQUIRE(E <= kMaxNEdges, PEANUT_UNSUPPORTED, "more than %llu runs of N",
                   (unsigned long long)(kMaxNEdges / 2));
        PN_REQUIRE(E % 2 == 0, PEANUT_CUDA_ERROR, "unpaired run boundary of N");
        DBuf<uint64_t> edges(E ? E : 1, s);
        cnt.zero();
        n_edges_k<true><<<g, 256, 0, s>>>(reinterpret_cast<const uint32_t*>(nmask.p), nw32, cnt.p, edges.p, E);
        PN_CHECK_LAUNCH();
        runs.resize(E);
        if (E) PN_CUDA(cudaMemcpyAsync(runs.data(), edges.p, E * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        PN_CUDA(cudaStreamSynchronize(s));
        std::sort(runs.begin(), runs.end());
    }
    nmask.reset();
    // segments: each contig cut by the pieces of runs of at least gap_min Ns inside it
    std::vector<uint64_t> seg;
    uint64_t gaps = 0;
    size_t ri = 0;
    for (size_t c = 0; c < cs.size(); ++c) {
        const uint64_t a = cs[c], b = c + 1 < cs.size() ? cs[c + 1] : len;
        uint64_t open = a;
        while (ri < runs.size() / 2 && runs[2 * ri + 1] <= a) ++ri;
        for (size_t x = ri; x < runs.size() / 2 && runs[2 * x] < b; ++x) {
            const uint64_t ga = runs[2 * x] > a ? runs[2 * x] : a;
            const uint64_t gb = runs[2 * x + 1] < b ? runs[2 * x + 1] : b;
            if (gb - ga < gap_min) continue;
            if (ga > open) {
                seg.push_back(open);
                seg.push_back(ga);
            }
            open = gb;
            ++gaps;
        }
        if (b > open) {
            seg.push_back(open);
            seg.push_back(b);
        }
    }
    ref->contig.alloc(cs.size(), s);
    PN_CUDA(cudaMemcpyAsync(ref->contig.p, cs.data(), cs.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    ref->n_gaps = gaps;
    ref->n_seg = (uint32_t)(seg.size() / 2);
    PN_REQUIRE(seg.size() / 2 < (1ull << 31), PEANUT_UNSUPPORTED, "too many segments");
    ref->hseg = seg;
    ref->seg.alloc(seg.size() ? seg.size() : 2, s);
    ref->seg.zero();
    if (!seg.empty())
        PN_CUDA(cudaMemcpyAsync(ref->seg.p, ref->hseg.data(), seg.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    PN_CUDA(cudaStreamSynchronize(s));
}

// ---- frequent q-grams of the reference ------------------------------------------------------

// 2q-bit code of the q-gram starting at chunk offset o (0..31) of a 32-base chunk whose packed
// words are w[0..2] (w[0] holds the chunk's first 16 bases).
__device__ __forceinline__ uint32_t chunk_code(const uint32_t w[3], int o, uint32_t q) {
    const uint64_t win = ((uint64_t)w[o >> 4] << 32) | w[(o >> 4) + 1];
    const uint64_t g = win >> (64 - 2 * q - 2 * (o & 15));
    return q == 16 ? (uint32_t)g : (uint32_t)g & ((1u << (2 * q)) - 1u);
}

// tab[c - c0] += 1 for the canonical code c of every reference position p <= n - q with
// c in [c0, c0 + span) (the table is built one range of codes at a time).
__global__ void ref_count_k(const uint32_t* __restrict__ packed, uint64_t n, uint32_t q, uint32_t* tab, uint64_t c0,
                            uint64_t span) {
    const uint64_t nchunks = (n + 31) / 32;
    for (uint64_t ch = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < nchunks;
         ch += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t p0 = ch * 32;
        const uint32_t w[3] = {packed[p0 / 16], packed[p0 / 16 + 1], packed[p0 / 16 + 2]};
        for (int o = 0; o < 32; ++o) {
            const uint64_t p = p0 + o;
            if (p + q > n) break;
            const uint32_t g = chunk_code(w, o, q);
            const uint32_t h = revcomp_code(g, q);
            const uint64_t c = (uint64_t)(g < h ? g : h) - c0;  // wraps above span when below c0
            if (c < span) atomicAdd(&tab[c], 1u);
        }
    }
}

// Codes of the range (c0 + index) occurring more than cap times, as code << 32 | count; at most
// max_out are written (the count keeps growing past it).
__global__ void phi_collect_k(const uint32_t* tab, uint64_t span, uint64_t c0, uint32_t cap, uint64_t* out,
                              uint64_t max_out, unsigned long long* n_out) {
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < span;
         c += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = tab[c];
        if (v > cap) {
            const unsigned long long i = atomicAdd(n_out, 1ull);
            if (i < max_out) out[i] = ((c0 + c) << 32) | v;
        }
    }
}

__global__ void phi_mark_k(const uint64_t* keys, uint32_t n_phi, uint32_t* codes, uint64_t* counts, uint32_t* filter,
                           uint32_t shift) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_phi) return;
    const uint32_t c = (uint32_t)(keys[i] >> 32);
    codes[i] = c;
    counts[i] = keys[i] & 0xFFFFFFFFull;
    const uint32_t b = c >> shift;
    atomicOr(&filter[b >> 5], 1u << (b & 31));
}

// Index of code c in the sorted frequent codes, or -1 (the prefilter bit is tested first).
__device__ __forceinline__ int64_t phi_index(uint32_t c, const uint32_t* __restrict__ codes, uint32_t n_phi,
                                             const uint32_t* __restrict__ filter, uint32_t shift) {
    const uint32_t b = c >> shift;
    if (!((__ldg(filter + (b >> 5)) >> (b & 31)) & 1u)) return -1;
    uint32_t lo = 0, hi = n_phi;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(codes + mid) < c) lo = mid + 1;
        else hi = mid;
    }
    return lo < n_phi && __ldg(codes + lo) == c ? (int64_t)lo : -1;
}

// For each position whose canonical q-gram is frequent: key = phi << 41 | orientation << 40 | p.
__global__ void ref_occ_k(const uint32_t* __restrict__ packed, uint64_t n, uint32_t q,
                          const uint32_t* __restrict__ codes, uint32_t n_phi, const uint32_t* __restrict__ filter,
                          uint32_t shift, uint64_t* occ, unsigned long long* n_occ) {
    const uint64_t nchunks = (n + 31) / 32;
    for (uint64_t ch = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < nchunks;
         ch += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t p0 = ch * 32;
        const uint32_t w[3] = {packed[p0 / 16], packed[p0 / 16 + 1], packed[p0 / 16 + 2]};
        for (int o = 0; o < 32; ++o) {
            const uint64_t p = p0 + o;
            if (p + q > n) break;
            const uint32_t g = chunk_code(w, o, q);
            const uint32_t h = revcomp_code(g, q);
            const int64_t x = phi_index(g < h ? g : h, codes, n_phi, filter, shift);
            if (x >= 0) {
                const uint64_t phi = (uint64_t)x;
                const unsigned long long i = atomicAdd(n_occ, 1ull);
                occ[i] = (phi << 41) | ((uint64_t)(g > h) << 40) | p;
            }
        }
    }
}

__global__ void cluster_start_k(const uint64_t* occ, uint64_t n, uint32_t* start) {
    const uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const uint64_t mask = (1ull << 40) - 1;
    bool s = x == 0;
    if (!s) {
        const uint64_t a = occ[x - 1], b = occ[x];
        s = (a >> 40) != (b >> 40) || (b & mask) - (a & mask) > kClusterGap;
    }
    start[x] = s;
}

__global__ void cluster_write_k(const uint64_t* occ, uint64_t n, const uint32_t* start,
                                const uint64_t* sid, uint64_t* lo, uint64_t* hi, uint64_t* gcnt) {
    const uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const uint64_t mask = (1ull << 40) - 1;
    const uint64_t p = occ[x] & mask;
    const bool s = start[x];
    const uint64_t cid = s ? sid[x] : sid[x] - 1;
    if (s) {
        lo[cid] = p;
        atomicAdd((unsigned long long*)&gcnt[occ[x] >> 40], 1ull);
    }
    if (x + 1 == n || start[x + 1]) hi[cid] = p;
}

void free_prep(RefPrep* p) { delete p; }

// Default frequency cap: eight times the expected occurrences of a canonical q-gram in a uniform
// reference of this length (both strands), and at least 256, so that short q-grams on long
// references are not all declared frequent.
uint32_t default_freq_cap(uint64_t ref_len, uint32_t q) {
    const double expect = 2.0 * (double)ref_len / (double)(1ull << (2 * q));
    const double cap = 8.0 * expect;
    return cap > (double)kDefaultFreqCap ? (cap < 4e9 ? (uint32_t)cap : 4000000000u) : kDefaultFreqCap;
}

constexpr uint64_t kCountSpan = 1ull << 29;  // codes counted per pass over the reference
constexpr uint64_t kMaxPhi = 1ull << 23;     // frequent q-grams at most (their index fits 23 bits)

RefPrep* prepare_reference(const peanut_ref* ref, uint32_t q, uint32_t cap, cudaStream_t s) {
    RefPrep* P = new RefPrep();
    try {
        P->q = q;
        P->cap = cap;
        const uint64_t size = 1ull << (2 * q);
        P->filter_shift = 2 * q > (uint32_t)kFilterBits ? 2 * q - kFilterBits : 0;
        P->filter.alloc((1ull << kFilterBits) / 32, s);
        P->filter.zero();
        const uint64_t n = ref->n;
        if (n < q) {
            P->grp_off.alloc(1, s);
            P->grp_off.zero();
            return P;
        }
        // occurrence counts of every canonical code, one range of at most 2^29 codes (a 2 GiB
        // table) at a time, so that the transient memory stays bounded at q = 16 (4^16 codes)
        const uint64_t span = size < kCountSpan ? size : kCountSpan;
        DBuf<uint32_t> tab(span, s);
        const uint64_t nchunks = (n + 31) / 32;
        const unsigned g = grid_for(nchunks, 256, (unsigned)sm_count() * 32);
        const unsigned gt = grid_for(span, 256, (unsigned)sm_count() * 64);
        DBuf<unsigned long long> cnt(1, s);
        cnt.zero();
        DBuf<uint64_t> keys(kMaxPhi, s);
        for (uint64_t c0 = 0; c0 < size; c0 += span) {
            tab.zero();
            ref_count_k<<<g, 256, 0, s>>>(ref->packed.p, n, q, tab.p, c0, span);
            PN_CHECK_LAUNCH();
            phi_collect_k<<<gt, 256, 0, s>>>(tab.p, span, c0, cap, keys.p, kMaxPhi, cnt.p);
            PN_CHECK_LAUNCH();
        }
        tab.reset();
        const uint64_t n_phi = to_host(cnt.p, s);
        PN_REQUIRE(n_phi < kMaxPhi, PEANUT_UNSUPPORTED, "too many frequent q-grams (%llu)", (unsigned long long)n_phi);
        P->n_phi = (uint32_t)n_phi;
        if (n_phi == 0) {
            P->grp_off.alloc(1, s);
            P->grp_off.zero();
            return P;
        }
        DBuf<uint64_t> tmpk(n_phi, s);
        radix_sort_u64(keys.p, tmpk.p, n_phi, 64, s);
        P->phi_codes.alloc(n_phi, s);
        DBuf<uint64_t> counts(n_phi, s);
        phi_mark_k<<<grid_for(n_phi, 256), 256, 0, s>>>(keys.p, (uint32_t)n_phi, P->phi_codes.p, counts.p,
                                                        P->filter.p, P->filter_shift);
        PN_CHECK_LAUNCH();
        keys.reset();
        tmpk.reset();
        // every occurrence of a frequent q-gram, sorted by (phi, orientation, position)
        DBuf<uint64_t> tot(1, s);
        DBuf<uint64_t> scratch(n_phi, s);
        exclusive_scan(ArrayIn<uint64_t>{counts.p}, ArrayOut<uint64_t>{scratch.p}, n_phi, tot.p, s);
        const uint64_t n_occ = to_host(tot.p, s);
        P->n_occ = n_occ;
        DBuf<uint64_t> occ(n_occ, s), occ_tmp(n_occ, s);
        cnt.zero();
        ref_occ_k<<<g, 256, 0, s>>>(ref->packed.p, n, q, P->phi_codes.p, (uint32_t)n_phi, P->filter.p,
                                    P->filter_shift, occ.p, cnt.p);
        PN_CHECK_LAUNCH();
        int phi_bits = 0;
        while ((1ull << phi_bits) < n_phi) ++phi_bits;
        radix_sort_u64(occ.p, occ_tmp.p, n_occ, 41 + phi_bits, s);
        occ_tmp.reset();
        // clusters: maximal runs of one (phi, orientation) with gaps <= kClusterGap
        DBuf<uint32_t> start(n_occ, s);
        DBuf<uint64_t> sid(n_occ, s);
        cluster_start_k<<<grid_for(n_occ, 256), 256, 0, s>>>(occ.p, n_occ, start.p);
        PN_CHECK_LAUNCH();
        exclusive_scan(ArrayIn<uint32_t>{start.p}, ArrayOut<uint64_t>{sid.p}, n_occ, tot.p, s);
        const uint64_t ncl = to_host(tot.p, s);
        P->n_clusters = ncl;
        P->cl_lo.alloc(ncl, s);
        P->cl_hi.alloc(ncl, s);
        DBuf<uint64_t> gcnt(2 * n_phi + 1, s);
        gcnt.zero();
        cluster_write_k<<<grid_for(n_occ, 256), 256, 0, s>>>(occ.p, n_occ, start.p, sid.p, P->cl_lo.p,
                                                             P->cl_hi.p, gcnt.p);
        PN_CHECK_LAUNCH();
        P->grp_off.alloc(2 * n_phi + 1, s);
        exclusive_scan(ArrayIn<uint64_t>{gcnt.p}, ArrayOut<uint64_t>{P->grp_off.p}, 2 * n_phi + 1, nullptr, s);
        PN_CUDA(cudaStreamSynchronize(s));
        return P;
    } catch (...) {
        delete P;
        throw;
    }
}

// ---- the read batch ---------------------------------------------------------------------

__device__ __forceinline__ int phi_lookup(uint32_t c, const uint32_t* __restrict__ filter, uint32_t shift,
                                          const uint32_t* __restrict__ codes, uint32_t n) {
    if (n == 0) return -1;
    const uint32_t b = c >> shift;
    if (!((filter[b >> 5] >> (b & 31)) & 1u)) return -1;
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (codes[mid] < c) lo = mid + 1; else hi = mid;
    }
    return lo < n && codes[lo] == c ? (int)lo : -1;
}

// Sampled offsets 0, s, 2s, ... below nq; an edit touches at most ceil(q / s) of their q-grams,
// and k windows of q offsets can hold at most k ceil(q / s) of them (packed from offset 0), so at
// least the returned number stay intact (the q-gram lemma for s = 1).
__host__ __device__ __forceinline__ int64_t sampled_threshold(uint32_t nq, uint32_t q, uint32_t k, uint32_t s) {
    const int64_t na = (nq + s - 1) / s;
    const int64_t cover = (int64_t)k * ((q + s - 1) / s);
    return na - (cover < na ? cover : na);
}

__global__ void read_meta_k(const uint64_t* __restrict__ off, uint32_t n_reads, uint64_t total,
                            uint32_t q, uint32_t stride, uint32_t k_fixed, uint32_t k_permille, uint8_t* len,
                            uint8_t* kk, uint64_t* nq, uint32_t* status, uint32_t* maxes) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_reads) return;
    const uint64_t a = off[r], b = off[r + 1];
    if (b < a || b > total || b - a < 1 || b - a > (uint64_t)kMaxReadLen) {
        atomicOr(status, kStBadLength);
        len[r] = 0;
        kk[r] = 0;
        nq[r] = 0;
        return;
    }
    const uint32_t m = (uint32_t)(b - a);
    uint64_t k = k_fixed != 0xFFFFFFFFu ? k_fixed : ((uint64_t)m * k_permille + 999) / 1000;
    const int64_t t = (int64_t)m + 1 - (int64_t)q * (int64_t)(k + 1);
    if (t < 1 || k > 255 || (stride > 1 && sampled_threshold(m - q + 1, q, (uint32_t)k, stride) < 1)) {
        atomicOr(status, kStBadThreshold);
        k = 0;
    }
    len[r] = (uint8_t)m;
    kk[r] = (uint8_t)k;
    nq[r] = m >= q ? m - q + 1 : 0;
    atomicMax(&maxes[0], m);
    atomicMax(&maxes[1], (uint32_t)k);
}

// Base codes of the batch; an N keeps code 4 until read_fix_n_k replaces it.
__global__ void read_codes_k(const uint8_t* __restrict__ ascii, uint64_t total, uint8_t* codes, uint32_t* status) {
    bool bad = false, has_n = false;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint8_t c = kCodeLut[ascii[x]];
        bad |= c > 4;
        has_n |= c == 4;
        codes[x] = c > 4 ? 0 : c;
    }
    if (bad) atomicOr(status, kStBadBase);
    if (has_n) atomicOr(status, kStHasN);
}

// One thread per read holding an N: FNV-1a 64 (Fowler, Noll & Vo: offset basis
// 0xcbf29ce484222325, per byte xor then multiply by 0x100000001b3) of its upper-cased bytes, then
// every N at offset i takes the top two bits of output i + 1 of SplitMix64 seeded with
// (seed XOR that hash).
__global__ void read_fix_n_k(const uint8_t* __restrict__ ascii, const uint64_t* __restrict__ off, uint32_t n,
                             uint64_t seed, uint8_t* __restrict__ codes) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const uint64_t a = off[r], b = off[r + 1];  // offsets index the batch's bytes and codes alike
    bool any = false;
    for (uint64_t x = a; x < b; ++x) any |= codes[x] == 4;
    if (!any) return;
    uint64_t h = 0xcbf29ce484222325ull;
    for (uint64_t x = a; x < b; ++x) {
        uint8_t c = ascii[x];
        if (c >= 'a' && c <= 'z') c = (uint8_t)(c - 32);
        h = (h ^ c) * 0x100000001b3ull;
    }
    for (uint64_t x = a; x < b; ++x)
        if (codes[x] == 4) codes[x] = (uint8_t)(splitmix64_at(seed ^ h, x - a + 1) >> 62);
}

// Classifies every read q-gram (one warp per read): canonical code, orientation, whether it is
// frequent in the reference.  Indexed q-grams go to (tcode, tpay); frequent ones to fent.  Then
// chooses the read's filter threshold: t* = (#non-frequent offsets) - (most non-frequent offsets
// that k windows of q consecutive offsets can cover) is the q-gram lemma bound restricted to the
// indexed q-grams (each edit destroys the q-grams of at most q consecutive offsets).  If t* >= 1
// the read is filtered with t* on indexed q-grams alone; otherwise it keeps the full lemma
// threshold t and is also verified around every cluster of its frequent q-grams.
__global__ void __launch_bounds__(256)
    read_qgrams_k(const uint8_t* __restrict__ codes, const uint64_t* __restrict__ off,
                  const uint8_t* __restrict__ len, const uint8_t* __restrict__ kk,
                  const uint64_t* __restrict__ qoff, uint32_t n_reads, uint32_t q, uint32_t stride,
                  const uint32_t* __restrict__ filter, uint32_t shift, const uint32_t* __restrict__ phi,
                  uint32_t n_phi, uint32_t* tcode, uint32_t* tpay, uint64_t* fent, uint32_t* fcnt,
                  uint16_t* thr, uint8_t* lowcx, uint32_t* lowcx_list, uint32_t* n_lowcx) {
    const int lane = threadIdx.x & 31;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_reads; r += warps) {
        const uint32_t m = len[r], k = kk[r];
        const uint32_t nq = m >= q ? m - q + 1 : 0;
        const uint8_t* rd = codes + off[r];
        const uint64_t qb = qoff[r];
        uint32_t nf = 0;
        uint32_t imask[8];  // offsets whose q-gram is indexed (sampled and not frequent)
#pragma unroll
        for (int t = 0; t < 8; ++t) imask[t] = 0;
#pragma unroll 1
        for (uint32_t t = 0; t * 32 < nq; ++t) {
            const uint32_t i = t * 32 + lane;
            bool freq = false, indexed = false;
            uint64_t fe = 0;
            if (i < nq && i % stride != 0) {
                tcode[qb + i] = kSentinel;
            } else if (i < nq) {
                uint32_t g = 0;
                for (uint32_t x = 0; x < q; ++x) g = (g << 2) | rd[i + x];
                const uint32_t h = revcomp_code(g, q);
                const uint32_t c = g < h ? g : h;
                const uint32_t f = g > h ? 1u : 0u;
                const int ph = phi_lookup(c, filter, shift, phi, n_phi);
                if (ph < 0) {
                    tcode[qb + i] = c;
                    tpay[qb + i] = (r << 9) | (f << 8) | i;
                    indexed = true;
                } else {
                    tcode[qb + i] = kSentinel;
                    freq = true;
                    fe = ((uint64_t)ph << 32) | ((uint64_t)(g == h) << 9) | (f << 8) | i;
                }
            }
            const unsigned bal = __ballot_sync(kFull, freq);
            if (freq) fent[qb + nf + __popc(bal & lanemask_lt())] = fe;
            nf += __popc(bal);
            const unsigned ibal = __ballot_sync(kFull, indexed);
            if (t < 8) imask[t] = ibal;
        }
        if (lane == 0) {
            // intact sampled q-grams guaranteed by the lemma (all offsets when stride = 1)
            const int32_t tsampled = (int32_t)sampled_threshold(nq, q, k, stride);
            fcnt[r] = nf;
            if (nf == 0) {
                thr[r] = (uint16_t)tsampled;
                lowcx[r] = 0;
            } else {
                // maximum coverage of the indexed offsets by k windows of q offsets
                uint16_t pre[257], f0[257], f1[257];
                pre[0] = 0;
                for (uint32_t x = 0; x < nq; ++x) pre[x + 1] = pre[x] + ((imask[x >> 5] >> (x & 31)) & 1u);
                for (uint32_t x = 0; x <= nq; ++x) f0[x] = 0;
                uint16_t* prev = f0;
                uint16_t* cur = f1;
                for (uint32_t j = 1; j <= k; ++j) {
                    cur[nq] = 0;
                    for (int x = (int)nq - 1; x >= 0; --x) {
                        const uint32_t e = (uint32_t)x + q < nq ? (uint32_t)x + q : nq;
                        const uint16_t v = (uint16_t)(pre[e] - pre[x] + prev[e]);
                        cur[x] = v > cur[x + 1] ? v : cur[x + 1];
                    }
                    uint16_t* tt = prev;
                    prev = cur;
                    cur = tt;
                }
                const int32_t tstar = (int32_t)pre[nq] - (int32_t)prev[0];
                if (tstar >= 1) {
                    thr[r] = (uint16_t)tstar;
                    lowcx[r] = 0;
                } else {
                    thr[r] = (uint16_t)tsampled;
                    lowcx[r] = 1;
                    lowcx_list[atomicAdd(n_lowcx, 1u)] = r;
                }
            }
        }
    }
}

__global__ void set_bits_k(const uint32_t* __restrict__ tcode, uint64_t n, uint2* IS) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = tcode[x];
        if (c != kSentinel) atomicOr(&IS[c >> 5].x, 1u << (c & 31));
    }
}

// GROUPBIT for the other layouts: I words of 32 codes (layout 1) or of 64 codes (layout 2).
__global__ void set_bits_alt_k(const uint32_t* __restrict__ tcode, uint64_t n, uint32_t* I32, unsigned long long* I64) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = tcode[x];
        if (c == kSentinel) continue;
        if (I32) atomicOr(&I32[c >> 5], 1u << (c & 31));
        else atomicOr(&I64[c >> 6], 1ull << (c & 63));
    }
}

// Population counts per stored S entry: two 32-code words (layout 1) or one 64-code word (layout 2).
struct PopcPairIn {
    const uint32_t* I32;
    __device__ __forceinline__ uint64_t operator()(uint64_t t) const { return __popc(I32[2 * t]) + __popc(I32[2 * t + 1]); }
};
struct Popc64In {
    const unsigned long long* I64;
    __device__ __forceinline__ uint64_t operator()(uint64_t t) const { return __popcll(I64[t]); }
};

struct PopcIn {
    const uint2* IS;
    __device__ __forceinline__ uint64_t operator()(uint64_t i) const { return __popc(IS[i].x); }
};
struct SOut {
    uint2* IS;
    __device__ __forceinline__ void operator()(uint64_t i, uint64_t v) const { IS[i].y = (uint32_t)v; }
};

// GROUPBIT + GROUPRANK: the slot of code c in S' (S[i] + popcount(I[i] & (2^j - 1))).
__device__ __forceinline__ uint32_t qgram_slot(const uint2* __restrict__ IS, uint32_t c) {
    const uint2 v = IS[c >> 5];
    return v.y + __popc(v.x & ((1u << (c & 31)) - 1u));
}

template <int L>
__device__ __forceinline__ uint32_t view_slot(const IndexView& V, uint32_t c) {
    const uint2 v = index_group<L>(V, c);
    return v.y + __popc(v.x & ((1u << (c & 31)) - 1u));
}

template <int L>
__global__ void count_qgrams_k(const uint32_t* __restrict__ tcode, uint64_t n, IndexView V, uint32_t* cnt) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = tcode[x];
        if (c != kSentinel) atomicAdd(&cnt[view_slot<L>(V, c)], 1u);
    }
}

template <int L>
__global__ void scatter_qgrams_k(const uint32_t* __restrict__ tcode, const uint32_t* __restrict__ tpay,
                                 uint64_t n, IndexView V, const uint32_t* __restrict__ Sp, uint32_t* cur,
                                 uint32_t* O) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = tcode[x];
        if (c == kSentinel) continue;
        const uint32_t slot = view_slot<L>(V, c);
        O[Sp[slot] + atomicAdd(&cur[slot], 1u)] = tpay[x];
    }
}

__global__ void bloom_set_k(const uint32_t* __restrict__ tcode, uint64_t n, uint64_t* bloom, uint64_t mask) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = tcode[x];
        if (c == kSentinel) continue;
        const BloomKey bk = bloom_key(c, (uint32_t)(mask + 1));
        atomicOr((unsigned long long*)(bloom + bk.word), ((unsigned long long)bk.hi << 32) | bk.lo);
    }
}

// Match masks of Myers' algorithm (Section "Validation"): bit i of peq[r][s][c][w] is set when
// position 64 w + i of the pattern (the read for s = 0, its reverse complement for s = 1) is c.
__global__ void peq_k(const uint8_t* __restrict__ codes, const uint64_t* __restrict__ off,
                      const uint8_t* __restrict__ len, uint32_t n_reads, uint64_t* peq) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_reads) return;
    const uint32_t m = len[r];
    const uint8_t* rd = codes + off[r];
    uint64_t* out = peq + (uint64_t)r * 2 * 4 * kMaxWords;
    for (int s = 0; s < 2; ++s) {
        uint64_t w[4][kMaxWords] = {};
        for (uint32_t i = 0; i < m; ++i) {
            const uint32_t c = s == 0 ? rd[i] : 3u - rd[m - 1 - i];
            w[c][i >> 6] |= 1ull << (i & 63);
        }
        for (int c = 0; c < 4; ++c)
            for (int x = 0; x < kMaxWords; ++x) out[(s * 4 + c) * kMaxWords + x] = w[c][x];
    }
}

// ---- the reference's own q-group index ---------------------------------------------------
//
// Algorithm 1 run over the reference instead of the reads (the reference-side index of Section
// "Filtration", without repeat masking): every position p <= n - q contributes its canonical
// code; I / S as for the reads (interleaved per group of 32 codes), S' by an exclusive scan of the
// per-code counts, O the positions grouped by code, one orientation bit per O entry.

__global__ void ref_set_bits_k(const uint32_t* __restrict__ packed, uint64_t n, uint32_t q, uint2* IS) {
    const uint64_t nchunks = (n + 31) / 32;
    for (uint64_t ch = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < nchunks;
         ch += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t p0 = ch * 32;
        const uint32_t w[3] = {packed[p0 / 16], packed[p0 / 16 + 1], packed[p0 / 16 + 2]};
        for (int o = 0; o < 32; ++o) {
            if (p0 + o + q > n) break;
            const uint32_t g = chunk_code(w, o, q), h = revcomp_code(g, q);
            const uint32_t c = g < h ? g : h;
            atomicOr(&IS[c >> 5].x, 1u << (c & 31));
        }
    }
}

template <bool kScatter>
__global__ void ref_slots_k(const uint32_t* __restrict__ packed, uint64_t n, uint32_t q,
                            const uint2* __restrict__ IS, uint32_t* cnt, const uint32_t* __restrict__ Sp,
                            uint32_t* O, uint32_t* orient) {
    const uint64_t nchunks = (n + 31) / 32;
    for (uint64_t ch = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; ch < nchunks;
         ch += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t p0 = ch * 32;
        const uint32_t w[3] = {packed[p0 / 16], packed[p0 / 16 + 1], packed[p0 / 16 + 2]};
        for (int o = 0; o < 32; ++o) {
            if (p0 + o + q > n) break;
            const uint32_t g = chunk_code(w, o, q), h = revcomp_code(g, q);
            const uint32_t c = g < h ? g : h;
            const uint32_t slot = qgram_slot(IS, c);
            if (!kScatter) {
                atomicAdd(&cnt[slot], 1u);
            } else {
                const uint32_t x = Sp[slot] + atomicAdd(&cnt[slot], 1u);
                O[x] = (uint32_t)(p0 + o);
                if (g > h) atomicOr(&orient[x >> 5], 1u << (x & 31));
            }
        }
    }
}

RefIndex* build_ref_index(const peanut_ref* ref, uint32_t q, cudaStream_t s) {
    PN_REQUIRE(q >= 1 && q <= 16, PEANUT_UNSUPPORTED, "q = %u outside 1..16", q);
    PN_REQUIRE(ref->n < (1ull << 32), PEANUT_UNSUPPORTED,
               "the reference index stores 32-bit positions (the reference has %llu bases)",
               (unsigned long long)ref->n);
    RefIndex* X = new RefIndex();
    try {
        X->q = q;
        const uint64_t n = ref->n;
        X->n_pos = n >= q ? n - q + 1 : 0;
        X->n_groups = ((1ull << (2 * q)) + 31) / 32;
        X->IS.alloc(X->n_groups, s);
        X->IS.zero();
        const unsigned g = grid_for((n + 31) / 32, 256, (unsigned)sm_count() * 32);
        ref_set_bits_k<<<g, 256, 0, s>>>(ref->packed.p, n, q, X->IS.p);
        PN_CHECK_LAUNCH();
        DBuf<uint64_t> tot(1, s);
        exclusive_scan(PopcIn{X->IS.p}, SOut{X->IS.p}, X->n_groups, tot.p, s);
        X->n_distinct = to_host(tot.p, s);
        DBuf<uint32_t> cnt(X->n_distinct + 1, s);
        cnt.zero();
        ref_slots_k<false><<<g, 256, 0, s>>>(ref->packed.p, n, q, X->IS.p, cnt.p, nullptr, nullptr, nullptr);
        PN_CHECK_LAUNCH();
        X->Sp.alloc(X->n_distinct + 1, s);
        exclusive_scan(ArrayIn<uint32_t>{cnt.p}, ArrayOut<uint32_t>{X->Sp.p}, X->n_distinct + 1, nullptr, s);
        cnt.zero();
        X->O.alloc(X->n_pos ? X->n_pos : 1, s);
        X->orient.alloc((X->n_pos + 31) / 32 + 1, s);
        X->orient.zero();
        ref_slots_k<true><<<g, 256, 0, s>>>(ref->packed.p, n, q, X->IS.p, cnt.p, X->Sp.p, X->O.p, X->orient.p);
        PN_CHECK_LAUNCH();
        PN_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        delete X;
        throw;
    }
    return X;
}

void index_reads(peanut_reads* R, const char* d_seqs, const uint64_t* d_offsets, uint32_t k_fixed,
                 uint32_t k_permille, uint32_t stride) {
    init_lut();
    cudaStream_t s = R->stream;
    const uint32_t n = R->n_reads, q = R->q;
    const uint64_t total = R->total_bases;
    R->base_off.alloc((uint64_t)n + 1, s);
    PN_CUDA(cudaMemcpyAsync(R->base_off.p, d_offsets, ((uint64_t)n + 1) * sizeof(uint64_t),
                            cudaMemcpyDeviceToDevice, s));
    R->len.alloc(n, s);
    R->kk.alloc(n, s);
    DBuf<uint64_t> nq(n, s);
    DBuf<uint32_t> status(3, s);  // [0] status, [1] max len, [2] max k
    status.zero();
    R->stride = stride;
    read_meta_k<<<grid_for(n, 256), 256, 0, s>>>(R->base_off.p, n, total, q, stride, k_fixed, k_permille,
                                                  R->len.p, R->kk.p, nq.p, status.p, status.p + 1);
    PN_CHECK_LAUNCH();
    R->codes.alloc(total ? total : 1, s);
    read_codes_k<<<grid_for(total, 256, (unsigned)sm_count() * 16), 256, 0, s>>>(
        (const uint8_t*)d_seqs, total, R->codes.p, status.p);
    PN_CHECK_LAUNCH();
    uint32_t st[3];
    PN_CUDA(cudaMemcpyAsync(st, status.p, sizeof(st), cudaMemcpyDeviceToHost, s));
    PN_CUDA(cudaStreamSynchronize(s));
    PN_REQUIRE(!(st[0] & kStBadLength), PEANUT_INVALID_ARG,
               "read offsets must ascend within the sequence buffer and give lengths 1..%d", kMaxReadLen);
    PN_REQUIRE(!(st[0] & kStBadBase), PEANUT_INVALID_ARG, "a read contains a byte other than A/C/G/T/N (either case)");
    if (st[0] & kStHasN) {
        read_fix_n_k<<<grid_for(n, 128), 128, 0, s>>>((const uint8_t*)d_seqs, R->base_off.p, n, R->ref->n_seed,
                                                       R->codes.p);
        PN_CHECK_LAUNCH();
    }
    PN_REQUIRE(!(st[0] & kStBadThreshold), PEANUT_INVALID_ARG,
               "a read violates the q-gram lemma threshold m + 1 - q(k + 1) >= 1 (q = %u), or keeps no "
               "guaranteed intact q-gram at sampling stride %u", q, stride);
    R->max_len = st[1];
    R->max_k = st[2];

    // q-gram slots per read
    R->qoff.alloc((uint64_t)n + 1, s);
    DBuf<uint64_t> tot(1, s);
    exclusive_scan(ArrayIn<uint64_t>{nq.p}, ArrayOut<uint64_t>{R->qoff.p}, n, tot.p, s);
    PN_CUDA(cudaMemcpyAsync(R->qoff.p + n, tot.p, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    const uint64_t nqg = to_host(tot.p, s);
    R->n_qgrams = nqg;
    nq.reset();

    const RefPrep* P = R->prep.get();
    DBuf<uint32_t> tcode(nqg ? nqg : 1, s), tpay(nqg ? nqg : 1, s);
    R->fent.alloc(nqg ? nqg : 1, s);
    R->fcnt.alloc(n, s);
    R->thr.alloc(n, s);
    R->lowcx.alloc(n, s);
    R->lowcx_list.alloc(n, s);
    DBuf<uint32_t> nlc(1, s);
    nlc.zero();
    read_qgrams_k<<<grid_for((uint64_t)n * 32, 256, (unsigned)sm_count() * 8), 256, 0, s>>>(
        R->codes.p, R->base_off.p, R->len.p, R->kk.p, R->qoff.p, n, q, stride, P->filter.p, P->filter_shift,
        P->phi_codes.p, P->n_phi, tcode.p, tpay.p, R->fent.p, R->fcnt.p, R->thr.p, R->lowcx.p,
        R->lowcx_list.p, nlc.p);
    PN_CHECK_LAUNCH();

    // Algorithm 1 over the indexed canonical codes, in the batch's layout of I and S
    R->n_groups = ((1ull << (2 * q)) + 31) / 32;
    const unsigned gq = grid_for(nqg, 256, (unsigned)sm_count() * 16);
    DBuf<uint64_t> tot2(1, s);
    if (R->layout == 0) {
        R->IS.alloc(R->n_groups, s);
        R->IS.zero();
        set_bits_k<<<gq, 256, 0, s>>>(tcode.p, nqg, R->IS.p);
        PN_CHECK_LAUNCH();
        exclusive_scan(PopcIn{R->IS.p}, SOut{R->IS.p}, R->n_groups, tot2.p, s);
    } else if (R->layout == 1) {
        const uint64_t pairs = (R->n_groups + 1) / 2;
        R->I32.alloc(2 * pairs, s);
        R->I32.zero();
        R->S2.alloc(pairs, s);
        set_bits_alt_k<<<gq, 256, 0, s>>>(tcode.p, nqg, R->I32.p, nullptr);
        PN_CHECK_LAUNCH();
        exclusive_scan(PopcPairIn{R->I32.p}, ArrayOut<uint32_t>{R->S2.p}, pairs, tot2.p, s);
    } else {
        const uint64_t g64 = ((1ull << (2 * q)) + 63) / 64;
        R->I64.alloc(g64, s);
        R->I64.zero();
        R->S64.alloc(g64, s);
        set_bits_alt_k<<<gq, 256, 0, s>>>(tcode.p, nqg, nullptr, R->I64.p);
        PN_CHECK_LAUNCH();
        exclusive_scan(Popc64In{R->I64.p}, ArrayOut<uint32_t>{R->S64.p}, g64, tot2.p, s);
    }
    const IndexView IV = index_view(R);
    DBuf<uint32_t> cnt(nqg + 1, s);
    cnt.zero();
    switch (R->layout) {
        case 0: count_qgrams_k<0><<<gq, 256, 0, s>>>(tcode.p, nqg, IV, cnt.p); break;
        case 1: count_qgrams_k<1><<<gq, 256, 0, s>>>(tcode.p, nqg, IV, cnt.p); break;
        default: count_qgrams_k<2><<<gq, 256, 0, s>>>(tcode.p, nqg, IV, cnt.p); break;
    }
    PN_CHECK_LAUNCH();
    R->Sp.alloc(nqg + 1, s);
    exclusive_scan(ArrayIn<uint32_t>{cnt.p}, ArrayOut<uint32_t>{R->Sp.p}, nqg + 1, tot.p, s);
    cnt.zero();
    uint64_t sizes[2];
    PN_CUDA(cudaMemcpyAsync(&sizes[0], tot2.p, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    PN_CUDA(cudaMemcpyAsync(&sizes[1], tot.p, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    PN_CUDA(cudaStreamSynchronize(s));
    R->n_distinct = sizes[0];
    R->n_indexed = sizes[1];
    R->O.alloc(R->n_indexed ? R->n_indexed : 1, s);
    switch (R->layout) {
        case 0: scatter_qgrams_k<0><<<gq, 256, 0, s>>>(tcode.p, tpay.p, nqg, IV, R->Sp.p, cnt.p, R->O.p); break;
        case 1: scatter_qgrams_k<1><<<gq, 256, 0, s>>>(tcode.p, tpay.p, nqg, IV, R->Sp.p, cnt.p, R->O.p); break;
        default: scatter_qgrams_k<2><<<gq, 256, 0, s>>>(tcode.p, tpay.p, nqg, IV, R->Sp.p, cnt.p, R->O.p); break;
    }
    PN_CHECK_LAUNCH();
    // prefilter for the reference scan: 16 to 32 bits per distinct code (four bits of a 64-bit
    // word each, so that few absent codes pass on to an 8-byte probe of the index in HBM), at
    // most 64 MB so that it stays resident in the 129 MB L2 while the index is probed in HBM
    uint64_t words = 1024;
    while (words < (1ull << 23) && words * 64 < R->n_distinct * 16) words <<= 1;
    R->bloom.alloc(words, s);
    R->bloom.zero();
    R->bloom_mask = words - 1;
    bloom_set_k<<<gq, 256, 0, s>>>(tcode.p, nqg, R->bloom.p, R->bloom_mask);
    PN_CHECK_LAUNCH();

    R->peq.alloc((uint64_t)n * 2 * 4 * kMaxWords, s);
    peq_k<<<grid_for(n, 128), 128, 0, s>>>(R->codes.p, R->base_off.p, R->len.p, n, R->peq.p);
    PN_CHECK_LAUNCH();
    R->n_lowcx = to_host(nlc.p, s);
}

}  // namespace pn
