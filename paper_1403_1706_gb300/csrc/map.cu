// Mapping a read batch: reference scan (Algorithm 2), candidate windows, bit-vector verification
// (Section "Validation") and the per-read stratum reduction (Section "Postprocessing").
//
// Hit key layout (64 bits): read << 41 | strand << 40 | (diagonal + kDiagBias).
// The diagonal of a hit is the putative read start d = p - i (Section "Filtration"); for the
// reverse-complement strand the offset i is taken in the reverse-complemented read.
//
// Candidate windows (the q-gram lemma, Section "The q-group index"): an alignment with e <= k
// edits keeps at least t of the read's q-grams intact, all on diagonals spanning at most e + 1
// values; with d0 the smallest of them, the alignment ends in [d0 + m - 1 - k, d0 + m - 1 + k].
// So it suffices to verify, for every window of k + 1 consecutive diagonals holding at least t
// hits, the end range [d0 + m - 1 - k, d0 + m - 1 + k]; with sorted hit diagonals d_x this is
// the union over x with d_{x+t-1} - d_x <= k of [d_{x+t-1} + m - 1 - 2k, d_x + m - 1 + k].
// Overlapping or touching ranges are merged so every maximal run of end positions lies in one;
// ranges less than m + k apart are joined too (the gap holds no end within k edits, and verifying
// it costs fewer columns than the m + k warm-up columns a separate range needs).
#include <cstdio>
#include <mutex>

#include "prims.cuh"

namespace pn {

constexpr int kScanBlock = 256;
constexpr int kStageCap = 256;  // staged hits per warp before one global append
constexpr int kWinWarps = 4;
constexpr int kWinCap = 1024;   // hits per read sorted in shared memory by one warp
constexpr uint32_t kMedCap = 12288;  // hits per read sorted in shared memory by one block
constexpr int kMedThreads = 1024;
constexpr int kMedWarps = kMedThreads / 32;
constexpr int kMedRounds = kMedCap / (kMedWarps * 32);  // 32-key rounds per warp
constexpr size_t kMedSmem = 2 * kMedCap * sizeof(uint64_t) + kMedWarps * 256 * sizeof(uint16_t);
constexpr uint64_t kKeyMask41 = (1ull << 41) - 1;
constexpr uint64_t kPosMask40 = (1ull << 40) - 1;

// ---- reference scan ------------------------------------------------------------------------

// L2 cache policies: the Bloom filter is read by every position and should stay resident; index
// probes touch each line about once.
__device__ __forceinline__ uint64_t l2_policy_keep() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_stream() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t ld_u64_policy(const uint64_t* ptr, uint64_t pol) {
    uint64_t v;
    asm volatile("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ uint2 ld_u32x2_policy(const uint2* ptr, uint64_t pol) {
    uint2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(ptr), "l"(pol));
    return v;
}

__device__ __forceinline__ void stage_flush(uint64_t* st, uint32_t cnt, uint64_t* hits, uint64_t cap,
                                            unsigned long long* n_hits) {
    __syncwarp();
    unsigned long long base = 0;
    if ((threadIdx.x & 31) == 0 && cnt) base = atomicAdd(n_hits, (unsigned long long)cnt);
    base = __shfl_sync(kFull, base, 0);
    for (uint32_t j = threadIdx.x & 31; j < cnt; j += 32)
        if (base + j < cap) __stcs(hits + base + j, st[j]);
    __syncwarp();
}

// Algorithm 2 in two stages.
//
// probe_ref_k, one pass over reference positions p in [0, n - q]: each lane takes 32 consecutive
// positions of a chunk, forms the canonical code of each, tests it against the L2-resident Bloom
// word and, if it passes, probes the index word (I, S).  Positions whose code is indexed are
// appended as (p << 2 | palindrome << 1 | orientation, S' slot), staged per warp in shared
// memory and written with one atomic per stage.
//
// expand_k, one present position per lane: reads its S' pair, turns every occurrence in O into a
// hit key (two for a palindromic q-gram), and appends the keys through the same per-warp staging;
// rcount[r] counts each read's hits.  Splitting the stages keeps many independent loads in flight
// in both kernels instead of one chain of dependent DRAM loads per position.

__device__ __forceinline__ void stage_flush2(uint64_t* sk, uint32_t* ss, uint32_t cnt, uint64_t* okey,
                                             uint32_t* oslot, uint64_t cap, unsigned long long* n_out) {
    __syncwarp();
    unsigned long long base = 0;
    if ((threadIdx.x & 31) == 0 && cnt) base = atomicAdd(n_out, (unsigned long long)cnt);
    base = __shfl_sync(kFull, base, 0);
    for (uint32_t j = threadIdx.x & 31; j < cnt; j += 32)
        if (base + j < cap) {
            __stcs(okey + base + j, sk[j]);
            __stcs(oslot + base + j, ss[j]);
        }
    __syncwarp();
}

// kQ16: q = 16 known at compile time (the common case): constant shifts, no masks.
template <int L, bool kQ16>
__global__ void __launch_bounds__(kScanBlock, 4)
    probe_ref_k(const uint32_t* __restrict__ packed, uint64_t n, uint32_t q_arg, IndexView V,
                const uint64_t* __restrict__ bloom, uint64_t bloom_mask, uint64_t* __restrict__ okey,
                uint32_t* __restrict__ oslot, uint64_t cap, unsigned long long* n_out) {
    __shared__ uint64_t sk[kScanBlock / 32][kStageCap];
    __shared__ uint32_t ss[kScanBlock / 32][kStageCap];
    const uint32_t q = kQ16 ? 16u : q_arg;
    const uint32_t bloom_words = (uint32_t)(bloom_mask + 1);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t scnt = 0;
    const uint64_t npos = n >= q ? n - q + 1 : 0;
    const uint64_t nchunks = (npos + 31) / 32;
    const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t qm = q == 16 ? 0xFFFFFFFFu : (1u << (2 * q)) - 1u;
    const uint64_t keep = l2_policy_keep(), stream = l2_policy_stream();
    for (uint64_t ch0 = gwarp * 32; ch0 < nchunks; ch0 += nwarps * 32) {
        const uint64_t ch = ch0 + lane;
        const bool active = ch < nchunks;
        const uint64_t p0 = ch * 32;
        uint32_t w0 = 0, w1 = 0, w2 = 0;
        if (active) {
            w0 = __ldcs(packed + p0 / 16);
            w1 = __ldcs(packed + p0 / 16 + 1);
            w2 = __ldcs(packed + p0 / 16 + 2);
        }
        // q = 16: the reverse complement of the chunk's 48 bases as three words (r0 first), so
        // that both the code and its reverse complement are one funnel shift per position
        const uint32_t r0 = kQ16 ? revcomp_code(w2, 16) : 0u, r1 = kQ16 ? revcomp_code(w1, 16) : 0u,
                       r2 = kQ16 ? revcomp_code(w0, 16) : 0u;
#pragma unroll 1
        for (int o0 = 0; o0 < 32; o0 += 8) {
            uint32_t cc[8];
            uint32_t meta[8];  // bit 0: valid, bit 1: orientation, bit 2: palindrome
            uint64_t fw[8];
            uint32_t flo[8], fhi[8];
            // bases o .. o + 15 (o = o0 + u) lie in (hiw, low) from bit 2 (o mod 16) on; their
            // reverse complement starts at base 32 - o of the reversed chunk
            const uint32_t hiw = o0 < 16 ? w0 : w1, low = o0 < 16 ? w1 : w2;
            const uint32_t hir = o0 < 16 ? r1 : r0, lor = o0 < 16 ? r2 : r1;
            const uint32_t sh0 = 2u * (uint32_t)(o0 & 15);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int o = o0 + u;
                uint32_t g, h;
                if constexpr (kQ16) {
                    g = __funnelshift_l(low, hiw, sh0 + 2u * u);
                    h = __funnelshift_lc(lor, hir, 32u - sh0 - 2u * u);
                } else {
                    const uint64_t win = o < 16 ? (((uint64_t)w0 << 32) | w1) : (((uint64_t)w1 << 32) | w2);
                    g = (uint32_t)(win >> (64 - 2 * q - 2 * (o & 15))) & qm;
                    h = revcomp_code(g, q);
                }
                const uint32_t c = g < h ? g : h;
                const bool valid = active && p0 + o < npos;
                cc[u] = c;
                meta[u] = (valid ? 1u : 0u) | (g > h ? 2u : 0u) | (g == h ? 4u : 0u);
                const BloomKey bk = bloom_key(c, bloom_words);
                flo[u] = bk.lo;
                fhi[u] = bk.hi;
                fw[u] = valid ? ld_u64_policy(bloom + bk.word, keep) : 0;
            }
            uint2 vv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const bool pass = (meta[u] & 1u) && ((uint32_t)fw[u] & flo[u]) == flo[u] &&
                                  ((uint32_t)(fw[u] >> 32) & fhi[u]) == fhi[u];
                if constexpr (L == 0) {
                    vv[u] = pass ? ld_u32x2_policy(V.IS + (cc[u] >> 5), stream) : make_uint2(0, 0);
                } else {
                    vv[u] = pass ? index_group<L>(V, cc[u]) : make_uint2(0, 0);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t c = cc[u];
                const bool present = (vv[u].x >> (c & 31)) & 1u;
                const unsigned bal = __ballot_sync(kFull, present);
                if (bal) {
                    if (scnt + 32 > kStageCap) {
                        stage_flush2(sk[wid], ss[wid], scnt, okey, oslot, cap, n_out);
                        scnt = 0;
                    }
                    if (present) {
                        const uint32_t pos = scnt + __popc(bal & lanemask_lt());
                        sk[wid][pos] = ((p0 + o0 + u) << 2) | ((meta[u] >> 1) & 3u);
                        ss[wid][pos] = vv[u].y + __popc(vv[u].x & ((1u << (c & 31)) - 1u));
                    }
                    scnt += __popc(bal);
                }
            }
            __syncwarp();
        }
    }
    stage_flush2(sk[wid], ss[wid], scnt, okey, oslot, cap, n_out);
}

__global__ void __launch_bounds__(kScanBlock)
    expand_k(const uint64_t* __restrict__ pkey, const uint32_t* __restrict__ pslot,
             const unsigned long long* __restrict__ d_npres, uint64_t pcap, uint32_t q,
             const uint32_t* __restrict__ Sp, const uint32_t* __restrict__ O, const uint8_t* __restrict__ len,
             uint64_t* __restrict__ hits, uint64_t cap, unsigned long long* n_hits, uint32_t* __restrict__ rcount) {
    __shared__ uint64_t stage[kScanBlock / 32][kStageCap];
    const uint64_t npres = *d_npres < pcap ? *d_npres : pcap;  // present positions (counted on the device)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t* st = stage[wid];
    uint32_t scnt = 0;
    const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t b0 = gwarp * 32; b0 < npres; b0 += nwarps * 32) {
        const uint64_t x = b0 + lane;
        uint32_t kb = 0, ke = 0;
        uint64_t key = 0;
        if (x < npres) {
            key = __ldcs(pkey + x);
            const uint32_t slot = __ldcs(pslot + x);
            kb = __ldg(Sp + slot);
            ke = __ldg(Sp + slot + 1);
        }
        const int64_t p = (int64_t)(key >> 2);
        const uint32_t fref = key & 1u;
        const bool pal = (key >> 1) & 1u;
        while (true) {
            const bool has = kb < ke;
            if (!__any_sync(kFull, has)) break;
            uint64_t key0 = 0, key1 = 0;
            int nk = 0;
            if (has) {
                const uint32_t e = __ldg(O + kb);
                ++kb;
                const uint32_t r = e >> 9, fr = (e >> 8) & 1u, i = e & 255u;
                const int64_t m = __ldg(len + r);
                const int64_t dp = p - (int64_t)i + kDiagBias;
                const int64_t dm = p - (m - (int64_t)q - (int64_t)i) + kDiagBias;
                const uint64_t rk = (uint64_t)r << 41;
                if (pal) {
                    key0 = rk | (uint64_t)dp;
                    key1 = rk | (1ull << 40) | (uint64_t)dm;
                    nk = 2;
                } else if (fr == fref) {
                    key0 = rk | (uint64_t)dp;
                    nk = 1;
                } else {
                    key0 = rk | (1ull << 40) | (uint64_t)dm;
                    nk = 1;
                }
                atomicAdd(rcount + r, (uint32_t)nk);
            }
            const unsigned b1 = __ballot_sync(kFull, nk >= 1), b2 = __ballot_sync(kFull, nk == 2);
            const uint32_t tot = __popc(b1) + __popc(b2);
            if (scnt + tot > kStageCap) {
                stage_flush(st, scnt, hits, cap, n_hits);
                scnt = 0;
            }
            const uint32_t pos = scnt + __popc(b1 & lanemask_lt()) + __popc(b2 & lanemask_lt());
            if (nk >= 1) st[pos] = key0;
            if (nk == 2) st[pos + 1] = key1;
            scnt += tot;
            __syncwarp();
        }
    }
    stage_flush(st, scnt, hits, cap, n_hits);
}

// Algorithm 2 against the reference's own q-group index instead of a pass over the reference
// (the reference-side index of Section "Filtration", kept whole: no repeat masking).  One entry of
// the batch's O per lane (an indexed read q-gram: read, orientation, offset): its canonical code
// from the read's bases, the code's occurrences in the reference index, and for each occurrence the
// hit key(s) expand_k makes for the same (read q-gram, reference position) pair.  The hits are the
// same multiset as the streaming scan's, so everything downstream and the output are unchanged.
__global__ void __launch_bounds__(kScanBlock)
    refprobe_k(const uint32_t* __restrict__ O, uint64_t n_entries, uint32_t q, const uint8_t* __restrict__ codes,
               const uint64_t* __restrict__ base_off, const uint8_t* __restrict__ len, const uint2* __restrict__ RIS,
               const uint32_t* __restrict__ RSp, const uint32_t* __restrict__ RO,
               const uint32_t* __restrict__ Rorient, uint64_t* __restrict__ hits, uint64_t cap,
               unsigned long long* n_hits, uint32_t* __restrict__ rcount) {
    __shared__ uint64_t stage[kScanBlock / 32][kStageCap];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t* st = stage[wid];
    uint32_t scnt = 0;
    const uint64_t gwarp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t b0 = gwarp * 32; b0 < n_entries; b0 += nwarps * 32) {
        const uint64_t x = b0 + lane;
        uint32_t kb = 0, ke = 0, r = 0, fr = 0, i = 0;
        bool pal = false;
        if (x < n_entries) {
            const uint32_t e = __ldg(O + x);
            r = e >> 9;
            fr = (e >> 8) & 1u;
            i = e & 255u;
            const uint8_t* rd = codes + base_off[r] + i;
            uint32_t g = 0;
            for (uint32_t t = 0; t < q; ++t) g = (g << 2) | rd[t];
            const uint32_t h = revcomp_code(g, q);
            const uint32_t c = g < h ? g : h;
            pal = g == h;
            const uint2 v = __ldg(RIS + (c >> 5));
            if ((v.x >> (c & 31)) & 1u) {
                const uint32_t slot = v.y + __popc(v.x & ((1u << (c & 31)) - 1u));
                kb = __ldg(RSp + slot);
                ke = __ldg(RSp + slot + 1);
            }
        }
        const int64_t m = x < n_entries ? (int64_t)len[r] : 0;
        while (true) {
            const bool has = kb < ke;
            if (!__any_sync(kFull, has)) break;
            uint64_t key0 = 0, key1 = 0;
            int nk = 0;
            if (has) {
                const int64_t p = (int64_t)__ldg(RO + kb);
                const uint32_t fref = (__ldg(Rorient + (kb >> 5)) >> (kb & 31)) & 1u;
                ++kb;
                const int64_t dp = p - (int64_t)i + kDiagBias;
                const int64_t dm = p - (m - (int64_t)q - (int64_t)i) + kDiagBias;
                const uint64_t rk = (uint64_t)r << 41;
                if (pal) {
                    key0 = rk | (uint64_t)dp;
                    key1 = rk | (1ull << 40) | (uint64_t)dm;
                    nk = 2;
                } else if (fr == fref) {
                    key0 = rk | (uint64_t)dp;
                    nk = 1;
                } else {
                    key0 = rk | (1ull << 40) | (uint64_t)dm;
                    nk = 1;
                }
                atomicAdd(rcount + r, (uint32_t)nk);
            }
            const unsigned b1 = __ballot_sync(kFull, nk >= 1), b2 = __ballot_sync(kFull, nk == 2);
            const uint32_t tot = __popc(b1) + __popc(b2);
            if (scnt + tot > kStageCap) {
                stage_flush(st, scnt, hits, cap, n_hits);
                scnt = 0;
            }
            const uint32_t pos = scnt + __popc(b1 & lanemask_lt()) + __popc(b2 & lanemask_lt());
            if (nk >= 1) st[pos] = key0;
            if (nk == 2) st[pos + 1] = key1;
            scnt += tot;
            __syncwarp();
        }
    }
    stage_flush(st, scnt, hits, cap, n_hits);
}

// ---- binning hits by read ---------------------------------------------------------------

__global__ void bin_hits_k(const uint64_t* __restrict__ hits, uint64_t nh, const uint64_t* __restrict__ roff,
                           uint32_t* cur, uint64_t* __restrict__ binned) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nh;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t key = hits[x];
        const uint32_t r = (uint32_t)(key >> 41);
        binned[roff[r] + atomicAdd(cur + r, 1u)] = key & kKeyMask41;
    }
}

// ---- windows ----------------------------------------------------------------------------

struct WinParams {
    const uint64_t* roff;
    const uint8_t* len;
    const uint8_t* kk;
    const uint16_t* thr;
    uint64_t n;           // reference length
    uint64_t* wlo;        // interval lo | strand << 40, at roff[r] + x
    uint64_t* whi;
    uint32_t* wcnt;       // [2 * r + s]
};

__device__ __forceinline__ int64_t key_diag(uint64_t key) {
    return (int64_t)(key & kPosMask40) - kDiagBias;
}

// Lane 0 accumulates merged end ranges of one (read, strand) in increasing order.
struct RangeMerger {
    int64_t lo = 0, hi = -1;
    bool open = false;
    uint32_t cnt = 0;
    __device__ __forceinline__ void flush(uint64_t* wlo, uint64_t* whi, uint64_t base, uint32_t s, uint64_t n) {
        if (!open) return;
        const int64_t a = lo < 0 ? 0 : lo;
        const int64_t b = hi > (int64_t)n - 1 ? (int64_t)n - 1 : hi;
        if (a <= b) {
            wlo[base + cnt] = (uint64_t)a | ((uint64_t)s << 40);
            whi[base + cnt] = (uint64_t)b;
            ++cnt;
        }
        open = false;
    }
    int64_t join = 1;  // ranges closer than this are verified as one
    __device__ __forceinline__ void add(int64_t l, int64_t h, uint64_t* wlo, uint64_t* whi, uint64_t base,
                                        uint32_t s, uint64_t n) {
        if (open && l <= hi + join) {
            if (h > hi) hi = h;
            return;
        }
        flush(wlo, whi, base, s, n);
        lo = l;
        hi = h;
        open = true;
    }
};

// Sweep of one read's sorted hit keys (both strands) by one warp; writes the merged end ranges.
// Window j (T hits within k + 1 diagonals) covers ends [lo_j, hi_j]; both bounds grow with j, so
// a window opens a new range exactly when its lo lies beyond the previous window's hi by more
// than the join distance, and a range's hi is its last window's hi.  Each chunk of 32 windows
// decides this with one ballot and one shuffle.  Windows entirely outside the reference are
// dropped first (they cannot hold an end, and every range stays non-empty after clamping).
__device__ void window_sweep(const uint64_t* keys, uint32_t h, uint32_t r, const WinParams& P) {
    const int lane = threadIdx.x & 31;
    const int64_t m = P.len[r], k = P.kk[r];
    const uint32_t T = P.thr[r];
    const uint64_t base = P.roff[r];
    const int64_t n = (int64_t)P.n;
    const int64_t join = m + k;  // ranges closer than this are verified as one
    // number of strand-0 keys
    uint32_t h0 = 0;
    for (uint32_t x = lane; x < h; x += 32) h0 += (keys[x] & kKeyMask41) < (1ull << 40) ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h0 += __shfl_xor_sync(kFull, h0, o);
    uint32_t total = 0;
    for (uint32_t s = 0; s < 2; ++s) {
        const uint32_t b = s == 0 ? 0 : h0, e = s == 0 ? h0 : h;
        uint32_t cnt = total;   // ranges written so far (uniform)
        bool have = false;      // a range is open (uniform)
        int64_t open_hi = 0;    // hi of the last valid window (uniform)
        for (uint32_t j0 = b; j0 + T - 1 < e; j0 += 32) {
            const uint32_t j = j0 + lane;
            bool valid = false;
            int64_t lo = 0, hi = 0;
            if (j + T - 1 < e) {
                const int64_t dj = key_diag(keys[j]), dl = key_diag(keys[j + T - 1]);
                if (dl - dj <= k) {
                    lo = dl + m - 1 - 2 * k;
                    hi = dj + m - 1 + k;
                    valid = hi >= 0 && lo <= n - 1;
                }
            }
            const unsigned bal = __ballot_sync(kFull, valid);
            if (!bal) continue;
            const unsigned below = bal & lanemask_lt();
            const int64_t hin = __shfl_sync(kFull, hi, below ? 31 - __clz(below) : lane);
            const bool has_prev = below != 0 || have;
            const int64_t hprev = below ? hin : open_hi;
            const bool start = valid && (!has_prev || lo > hprev + join);
            const unsigned sb = __ballot_sync(kFull, start);
            if (start) {
                const uint32_t idx = cnt + __popc(sb & lanemask_lt());
                P.wlo[base + idx] = (uint64_t)(lo < 0 ? 0 : lo) | ((uint64_t)s << 40);
                if (has_prev) P.whi[base + idx - 1] = (uint64_t)(hprev > n - 1 ? n - 1 : hprev);
            }
            cnt += __popc(sb);
            have = true;
            open_hi = __shfl_sync(kFull, hi, 31 - __clz(bal));
        }
        if (have && lane == 0) P.whi[base + cnt - 1] = (uint64_t)(open_hi > n - 1 ? n - 1 : open_hi);
        if (lane == 0) P.wcnt[2 * r + s] = cnt - total;
        total = cnt;
    }
}

// One warp per read: sort its hits in shared memory (bitonic), then sweep.  Reads with more
// than kWinCap hits go to the block path (up to kMedCap) or the global-memory path.
__global__ void __launch_bounds__(kWinWarps * 32)
    windows_k(const uint64_t* __restrict__ binned, uint32_t n_reads, WinParams P, uint32_t* big_list,
              uint32_t* n_big, uint32_t* med_list) {
    __shared__ uint64_t sk[kWinWarps][kWinCap];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t* s = sk[wid];
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_reads; r += nw) {
        const uint64_t b = P.roff[r];
        const uint32_t h = (uint32_t)(P.roff[r + 1] - b);
        if (h < P.thr[r]) {
            if (lane == 0) P.wcnt[2 * r] = P.wcnt[2 * r + 1] = 0;
            continue;
        }
        if (h > (uint32_t)kWinCap) {
            if (lane == 0) {
                if (h <= kMedCap) med_list[atomicAdd(n_big + 1, 1u)] = r;
                else big_list[atomicAdd(n_big, 1u)] = r;
            }
            continue;
        }
        uint32_t np = 32;
        while (np < h) np <<= 1;
        for (uint32_t x = lane; x < np; x += 32) s[x] = x < h ? binned[b + x] : ~0ull;
        __syncwarp();
        for (uint32_t size = 2; size <= np; size <<= 1) {
            for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
                for (uint32_t t = lane; t < np / 2; t += 32) {
                    const uint32_t i = 2 * stride * (t / stride) + (t % stride);
                    const uint32_t j = i + stride;
                    const bool up = (i & size) == 0;
                    const uint64_t a = s[i], c = s[j];
                    if ((a > c) == up) {
                        s[i] = c;
                        s[j] = a;
                    }
                }
                __syncwarp();
            }
        }
        window_sweep(s, h, r, P);
        __syncwarp();
    }
}

// Block-wide exclusive scans over one value per thread (kMedThreads threads; sc: 32 ints).
__device__ __forceinline__ int32_t block_excl_max(int32_t v, int32_t* sc) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl = max(incl, t);
    }
    if (lane == 31) sc[w] = incl;
    __syncthreads();
    if (w == 0) {
        int32_t x = sc[lane], y = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(kFull, y, o);
            if (lane >= o) y = max(y, t);
        }
        sc[lane] = y;  // inclusive over warps
        (void)x;
    }
    __syncthreads();
    int32_t before = __shfl_up_sync(kFull, incl, 1);
    if (lane == 0) before = -1;
    const int32_t r = max(before, w ? sc[w - 1] : -1);
    __syncthreads();
    return r;
}

__device__ __forceinline__ uint32_t block_excl_sum(uint32_t v, uint32_t* sc, uint32_t* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sc[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint32_t y = sc[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, y, o);
            if (lane >= o) y += t;
        }
        sc[lane] = y;
    }
    __syncthreads();
    const uint32_t r = incl - v + (w ? sc[w - 1] : 0u);
    *total = sc[31];
    __syncthreads();
    return r;
}

// The sweep of window_sweep by a whole block over one read's sorted keys in shared memory: each
// thread takes a run of consecutive windows; the previous valid window of every window comes from
// an exclusive max-scan, range indices from an exclusive sum-scan of the range starts.
__device__ void block_sweep(const uint64_t* keys, uint32_t h, uint32_t r, const WinParams& P, int32_t* sci,
                            uint32_t* scu, uint32_t* s_h0) {
    const int64_t m = P.len[r], k = P.kk[r];
    const uint32_t T = P.thr[r];
    const uint64_t base = P.roff[r];
    const int64_t n = (int64_t)P.n, join = m + k;
    if (threadIdx.x == 0) *s_h0 = h;
    __syncthreads();
    const uint32_t E = (h + kMedThreads - 1) / kMedThreads;  // windows per thread (<= kMedRounds)
    const uint32_t j0 = threadIdx.x * E;
    for (uint32_t e = 0; e < E; ++e) {
        const uint32_t j = j0 + e;
        if (j < h && (keys[j] >> 40) & 1ull && (j == 0 || !((keys[j - 1] >> 40) & 1ull))) *s_h0 = j;
    }
    __syncthreads();
    const uint32_t h0 = *s_h0;
    auto seg = [&](uint32_t j) { return j < h0 ? 0u : 1u; };
    auto hi_of = [&](uint32_t j) { return key_diag(keys[j]) + m - 1 + k; };
    auto lo_of = [&](uint32_t j) { return key_diag(keys[j + T - 1]) + m - 1 - 2 * k; };
    auto valid = [&](uint32_t j) {
        const uint32_t e = j < h0 ? h0 : h;
        if (j + T - 1 >= e) return false;
        if (key_diag(keys[j + T - 1]) - key_diag(keys[j]) > k) return false;
        return hi_of(j) >= 0 && lo_of(j) <= n - 1;
    };
    // valid windows of this thread, and its last one
    uint32_t vmask = 0;
    int32_t last = -1;
    for (uint32_t e = 0; e < E; ++e) {
        const uint32_t j = j0 + e;
        if (j < h && valid(j)) {
            vmask |= 1u << e;
            last = (int32_t)j;
        }
    }
    const int32_t pre = block_excl_max(last, sci);
    // range starts
    uint32_t smask = 0, ns = 0, ns0 = 0;
    int32_t cur = pre;
    for (uint32_t e = 0; e < E; ++e) {
        if (!((vmask >> e) & 1u)) continue;
        const uint32_t j = j0 + e;
        const bool start = cur < 0 || seg((uint32_t)cur) != seg(j) || lo_of(j) > hi_of((uint32_t)cur) + join;
        if (start) {
            smask |= 1u << e;
            ++ns;
            ns0 += seg(j) == 0 ? 1u : 0u;
        }
        cur = (int32_t)j;
    }
    uint32_t total = 0, total0 = 0;
    uint32_t idx = block_excl_sum(ns, scu, &total);
    block_excl_sum(ns0, scu, &total0);
    // the last valid window of each strand closes its strand's last range
    int32_t last0 = -1, last1 = -1;
    if (last >= 0) {
        for (uint32_t e = 0; e < E; ++e)
            if ((vmask >> e) & 1u) {
                if (seg(j0 + e) == 0) last0 = (int32_t)(j0 + e);
                else last1 = (int32_t)(j0 + e);
            }
    }
    // block-wide max of last0 / last1: an exclusive max-scan of the values shifted by one thread
    const int32_t m0 = block_excl_max(last0, sci), m1 = block_excl_max(last1, sci);
    __shared__ int32_t s_last[2];
    if (threadIdx.x == kMedThreads - 1) {
        s_last[0] = max(m0, last0);
        s_last[1] = max(m1, last1);
    }
    __syncthreads();
    const int32_t lastv0 = s_last[0], lastv1 = s_last[1];
    cur = pre;
    for (uint32_t e = 0; e < E; ++e) {
        if (!((vmask >> e) & 1u)) continue;
        const uint32_t j = j0 + e;
        if ((smask >> e) & 1u) {
            const int64_t lo = lo_of(j);
            P.wlo[base + idx] = (uint64_t)(lo < 0 ? 0 : lo) | ((uint64_t)seg(j) << 40);
            if (cur >= 0 && seg((uint32_t)cur) == seg(j)) {
                const int64_t hp = hi_of((uint32_t)cur);
                P.whi[base + idx - 1] = (uint64_t)(hp > n - 1 ? n - 1 : hp);
            }
            ++idx;
        }
        if ((int32_t)j == lastv0 || (int32_t)j == lastv1) {
            const int64_t hp = hi_of(j);
            P.whi[base + idx - 1] = (uint64_t)(hp > n - 1 ? n - 1 : hp);
        }
        cur = (int32_t)j;
    }
    if (threadIdx.x == 0) {
        P.wcnt[2 * r] = total0;
        P.wcnt[2 * r + 1] = total - total0;
    }
    __syncthreads();
}

// Stable LSD radix sort of h <= kMedCap keys in shared memory (bufA) by bits [lo_bit, hi_bit),
// 8-bit digits: every warp ranks a contiguous chunk of keys in 32-key rounds (eight ballots find
// the lanes with equal digits, a per-warp counter per digit carries over rounds), the counters
// become digit-major, warp-minor offsets, and the keys are scattered to the other buffer.  All
// threads of the block call it; returns the buffer that holds the sorted keys.
__device__ uint64_t* block_radix_sort(uint64_t* bufA, uint64_t* bufB, uint16_t* cnt, uint32_t* s_tot,
                                      uint32_t* s_part, uint32_t h, int lo_bit, int hi_bit) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t chunk = ((h + kMedWarps * 32 - 1) / (kMedWarps * 32)) * 32;  // keys per warp
    const uint32_t w0 = (uint32_t)w * chunk, w1 = min(h, w0 + chunk);
    uint64_t* src = bufA;
    uint64_t* dst = bufB;
    for (int shift = lo_bit; shift < hi_bit; shift += 8) {
        for (int i = threadIdx.x; i < kMedWarps * 256; i += blockDim.x) cnt[i] = 0;
        __syncthreads();
        uint32_t lr[kMedRounds];
        const int nrounds = (int)((w1 > w0 ? w1 - w0 : 0) + 31) / 32;
#pragma unroll
        for (int i = 0; i < kMedRounds; ++i) {
            if (i >= nrounds) break;  // warp-uniform
            const uint32_t idx = w0 + 32 * i + lane;
            const bool valid = idx < w1;
            const uint32_t dig = valid ? (uint32_t)(src[idx] >> shift) & 255u : 0u;
            // lanes with the same digit: intersect the eight bit-ballots
            unsigned peers = __ballot_sync(kFull, valid);
#pragma unroll
            for (int bb = 0; bb < 8; ++bb) {
                const unsigned bal = __ballot_sync(kFull, (dig >> bb) & 1u);
                peers &= ((dig >> bb) & 1u) ? bal : ~bal;
            }
            const uint32_t base = valid ? cnt[w * 256 + dig] : 0u;
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) cnt[w * 256 + dig] = (uint16_t)(base + __popc(peers));
            __syncwarp();
            lr[i] = base + __popc(peers & lanemask_lt());
        }
        __syncthreads();
        {  // per digit: exclusive prefix over the warps, four groups of eight warps in parallel
            const int d = threadIdx.x & 255, g = threadIdx.x >> 8;
            uint32_t run = 0;
#pragma unroll
            for (int ww = 8 * g; ww < 8 * g + 8; ++ww) {
                const uint32_t c = cnt[ww * 256 + d];
                cnt[ww * 256 + d] = (uint16_t)run;
                run += c;
            }
            s_part[g * 256 + d] = run;
        }
        __syncthreads();
        if (threadIdx.x < 256) {
            const int d = threadIdx.x;
            uint32_t run = 0;
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const uint32_t c = s_part[g * 256 + d];
                s_part[g * 256 + d] = run;
                run += c;
            }
            s_tot[d] = run;
        }
        __syncthreads();
        if (threadIdx.x < 32) {  // exclusive prefix over the digits, 8 per lane
            uint32_t v[8], sum = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                v[j] = s_tot[lane * 8 + j];
                sum += v[j];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            uint32_t run = incl - sum;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                s_tot[lane * 8 + j] = run;
                run += v[j];
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kMedWarps * 256; i += blockDim.x)
            cnt[i] = (uint16_t)(cnt[i] + s_tot[i & 255] + s_part[(i >> 11) * 256 + (i & 255)]);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kMedRounds; ++i) {
            if (i >= nrounds) break;
            const uint32_t idx = w0 + 32 * i + lane;
            if (idx < w1) {
                const uint64_t key = src[idx];
                dst[cnt[w * 256 + ((uint32_t)(key >> shift) & 255u)] + lr[i]] = key;
            }
        }
        __syncthreads();
        uint64_t* t = src;
        src = dst;
        dst = t;
    }
    return src;
}

// Reads with kWinCap < hits <= kMedCap: one block each sorts them in shared memory, then the
// block sweeps them; the sort key is strand << sbit | biased diagonal.
__global__ void __launch_bounds__(kMedThreads, 1)
    windows_med_k(const uint64_t* __restrict__ binned, const uint32_t* __restrict__ list, uint32_t n_list,
                  WinParams P, uint32_t* cursor, int sbit) {
    extern __shared__ uint64_t sm[];
    uint64_t* bufA = sm;
    uint64_t* bufB = sm + kMedCap;
    uint16_t* cnt = reinterpret_cast<uint16_t*>(sm + 2 * kMedCap);  // [warp][256]
    __shared__ uint32_t s_next, s_h0;
    __shared__ uint32_t s_tot[256];
    __shared__ uint32_t s_part[4 * 256];
    __shared__ int32_t s_sci[32];
    const uint64_t low = (1ull << sbit) - 1;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(cursor, 1u);  // reads of uneven size: dynamic order
        __syncthreads();
        const uint32_t x = s_next;
        if (x >= n_list) break;
        const uint32_t r = list[x];
        const uint64_t b = P.roff[r];
        const uint32_t h = (uint32_t)(P.roff[r + 1] - b);
        for (uint32_t i = threadIdx.x; i < h; i += blockDim.x) {
            const uint64_t k0 = binned[b + i];
            bufA[i] = (((k0 >> 40) & 1ull) << sbit) | (k0 & kPosMask40);
        }
        uint64_t* src = block_radix_sort(bufA, bufB, cnt, s_tot, s_part, h, 0, sbit + 1);
        for (uint32_t i = threadIdx.x; i < h; i += blockDim.x) {  // back to strand << 40
            const uint64_t k1 = src[i];
            src[i] = ((k1 >> sbit) << 40) | (k1 & low);
        }
        __syncthreads();
        block_sweep(src, h, r, P, s_sci, s_tot, &s_h0);
    }
}

// Deferred reads: their hits, tagged with the list index, sorted globally; one warp each.
__global__ void big_gather_k(const uint64_t* __restrict__ binned, const uint32_t* big_list, uint32_t n_big,
                             const uint64_t* roff, const uint64_t* goff, uint64_t* out) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n_big; x += nw) {
        const uint32_t r = big_list[x];
        const uint64_t b = roff[r], h = roff[r + 1] - b;
        for (uint64_t j = lane; j < h; j += 32) out[goff[x] + j] = ((uint64_t)x << 41) | binned[b + j];
    }
}

struct BigSize {
    const uint32_t* list;
    const uint64_t* roff;
    __device__ uint64_t operator()(uint64_t x) const { return roff[list[x] + 1] - roff[list[x]]; }
};

__global__ void big_sweep_k(const uint64_t* sorted, const uint32_t* big_list, uint32_t n_big,
                            const uint64_t* goff, WinParams P) {
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n_big; x += nw) {
        const uint32_t r = big_list[x];
        window_sweep(sorted + goff[x], (uint32_t)(goff[x + 1] - goff[x]), r, P);
    }
}

// ---- reads verified around frequent-q-gram clusters -------------------------------------

struct LcParams {
    const uint32_t* list;   // lowcx reads
    uint32_t n_list;
    const uint64_t* qoff;
    const uint32_t* fcnt;
    uint64_t* fent;         // sorted in place per read by lc_sort_k
    const uint8_t* len;
    const uint8_t* kk;
    uint32_t q;
    uint64_t n;
    const uint64_t* grp_off;
    const uint64_t* cl_lo;
    const uint64_t* cl_hi;
    const uint64_t* roff;   // W_n ranges of the read at roff[r]
    const uint64_t* wlo;
    const uint64_t* whi;
    const uint32_t* wcnt;
    const uint8_t* codes;   // read bases (2-bit codes, one per byte)
    const uint64_t* base_off;
    const uint32_t* packed; // reference
};

// Sort each listed read's frequent entries by (phi, orientation, offset) (insertion sort; <= 252).
__global__ void lc_sort_k(LcParams L) {
    const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= L.n_list) return;
    const uint32_t r = L.list[x];
    uint64_t* a = L.fent + L.qoff[r];
    const uint32_t n = L.fcnt[r];
    for (uint32_t i = 1; i < n; ++i) {
        const uint64_t v = a[i];
        int j = (int)i - 1;
        while (j >= 0 && a[j] > v) {
            a[j + 1] = a[j];
            --j;
        }
        a[j + 1] = v;
    }
}

// Visits, for (read r, strand s), every list of clusters to verify: the clusters of (phi, f_ref)
// with the smallest and largest offset i' of the read's q-grams on that strand.  For strand 0 a
// read q-gram of orientation f meets reference occurrences of orientation f at diagonal p - i;
// for strand 1 those of orientation 1 - f at diagonal p - (m - q - i).  A palindromic q-gram
// meets its (single-orientation) occurrences on both strands.
template <class F>
__device__ void lc_lists(const LcParams& L, uint32_t r, uint32_t s, F&& visit) {
    const uint64_t* a = L.fent + L.qoff[r];
    const uint32_t n = L.fcnt[r];
    const int64_t m = L.len[r], q = L.q;
    uint32_t x = 0;
    while (x < n) {
        const uint32_t phi = (uint32_t)(a[x] >> 32);
        int64_t mn[2] = {INT64_MAX, INT64_MAX}, mx[2] = {INT64_MIN, INT64_MIN};
        while (x < n && (uint32_t)(a[x] >> 32) == phi) {
            const uint32_t f = (a[x] >> 8) & 1u, pal = (a[x] >> 9) & 1u, i = a[x] & 255u;
            const uint32_t fref = pal ? 0u : (s == 0 ? f : 1u - f);
            const int64_t ip = s == 0 ? (int64_t)i : m - q - (int64_t)i;
            if (ip < mn[fref]) mn[fref] = ip;
            if (ip > mx[fref]) mx[fref] = ip;
            ++x;
        }
        for (uint32_t fr = 0; fr < 2; ++fr)
            if (mn[fr] != INT64_MAX) visit(L.grp_off[2 * phi + fr], L.grp_off[2 * phi + fr + 1], mn[fr], mx[fr]);
    }
}

// One list of clusters to verify for a (read, strand): clusters [cb, ce) of one (q-gram,
// orientation) with the smallest / largest offset i' of the read's q-grams on that strand; lo / hi
// is the (clipped) range of cluster cb, the list's next range.
struct LcDesc {
    uint64_t cb, ce;
    int64_t imin, imax;
    int64_t lo, hi;
};

// The range to verify around cluster c (Section "Filtration" diagonals p - i'), clipped to the
// reference: [cl_lo - i'max + m - 1 - 2k, cl_hi - i'min + m - 1 + k].
__device__ __forceinline__ void cluster_range(const LcParams& L, uint64_t c, int64_t imin, int64_t imax, int64_t m,
                                              int64_t k, int64_t* lo, int64_t* hi) {
    const int64_t n = (int64_t)L.n;
    const int64_t a = (int64_t)L.cl_lo[c] - imax + m - 1 - 2 * k;
    const int64_t b = (int64_t)L.cl_hi[c] - imin + m - 1 + k;
    *lo = a < 0 ? 0 : a;
    *hi = b > n - 1 ? n - 1 : b;
}

// Per segment y = 2 * list index + strand: its number of cluster lists and an upper bound on its
// merged ranges (counting-filter ranges plus one per cluster).
__global__ void lc_count_k(LcParams L, uint64_t* ndesc, uint64_t* cap) {
    const uint32_t y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= 2 * L.n_list) return;
    const uint32_t r = L.list[y >> 1], s = y & 1;
    uint64_t nd = 0, c = L.wcnt[2 * r + s];
    lc_lists(L, r, s, [&](uint64_t cb, uint64_t ce, int64_t, int64_t) {
        ++nd;
        c += ce - cb;
    });
    ndesc[y] = nd;
    cap[y] = c;
}

__global__ void lc_desc_k(LcParams L, const uint64_t* doff, LcDesc* desc) {
    const uint32_t y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= 2 * L.n_list) return;
    const uint32_t r = L.list[y >> 1], s = y & 1;
    const int64_t m = L.len[r], k = L.kk[r];
    uint64_t o = doff[y];
    lc_lists(L, r, s, [&](uint64_t cb, uint64_t ce, int64_t imin, int64_t imax) {
        LcDesc d{cb, ce, imin, imax, 0, 0};
        cluster_range(L, cb, imin, imax, m, k, &d.lo, &d.hi);
        desc[o++] = d;
    });
}

// Merged ranges of one segment are written to olo / ohi at off[y] + cnt.
struct MergeOut {
    int64_t cur_lo = 0, cur_hi = -2;
    bool open = false;
    uint32_t cnt = 0;
    int64_t join = 1;  // ranges closer than this are verified as one
    // Consumes the next range in increasing start; returns true when a finished range must be
    // written as (wlo, whi).
    __device__ __forceinline__ bool add(int64_t lo, int64_t hi, int64_t* wlo, int64_t* whi) {
        if (lo > hi) return false;  // clipped away
        if (open && lo <= cur_hi + join) {
            if (hi > cur_hi) cur_hi = hi;
            return false;
        }
        const bool flush = open;
        *wlo = cur_lo;
        *whi = cur_hi;
        cur_lo = lo;
        cur_hi = hi;
        open = true;
        return flush;
    }
};

// Slow path (a segment with 32 or more cluster lists): one lane merges sequentially.
__device__ void lc_kmerge_serial(const LcParams& L, uint32_t r, uint32_t s, uint64_t d0, uint64_t d1, LcDesc* desc,
                                 uint64_t o, uint64_t* olo, uint64_t* ohi, uint32_t* ocnt_y) {
    const int64_t m = L.len[r], k = L.kk[r];
    uint64_t w = L.roff[r] + (s == 0 ? 0 : L.wcnt[2 * r]);
    const uint64_t we = w + L.wcnt[2 * r + s];
    MergeOut M;
    M.join = m + k;
    int64_t a, b;
    while (true) {
        int64_t lo = INT64_MAX, hi = 0;
        int64_t src = -2;
        if (w < we) {
            lo = (int64_t)(L.wlo[w] & kPosMask40);
            hi = (int64_t)L.whi[w];
            src = -1;
        }
        for (uint64_t j = d0; j < d1; ++j)
            if (desc[j].cb < desc[j].ce && desc[j].lo < lo) {
                lo = desc[j].lo;
                hi = desc[j].hi;
                src = (int64_t)j;
            }
        if (src == -2) break;
        if (src == -1) {
            ++w;
        } else {
            LcDesc& d = desc[src];
            if (++d.cb < d.ce) cluster_range(L, d.cb, d.imin, d.imax, m, k, &d.lo, &d.hi);
        }
        if (M.add(lo, hi, &a, &b)) {
            olo[o + M.cnt] = (uint64_t)a;
            ohi[o + M.cnt] = (uint64_t)b;
            ++M.cnt;
        }
    }
    if (M.open) {
        olo[o + M.cnt] = (uint64_t)M.cur_lo;
        ohi[o + M.cnt] = (uint64_t)M.cur_hi;
        ++M.cnt;
    }
    *ocnt_y = M.cnt;
}

// Sort keys of the large segments: (2^40 - 1 - ranges) ascending = ranges descending.
__global__ void rest_order_k(const uint32_t* list, uint32_t n, const uint64_t* off, uint64_t* key, uint64_t* y) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t s = list[i];
    const uint64_t sz = off[s + 1] - off[s];
    key[i] = ((1ull << 40) - 1) - (sz < (1ull << 40) - 1 ? sz : (1ull << 40) - 1);
    y[i] = s;
}

constexpr int kMergeWarps = 4;  // warps per block of the k-way merge
constexpr int kMergeBuf = 16;   // ranges buffered per source (8 KB per warp)

// k-way merge, one warp per segment: the counting-filter ranges of the strand and every cluster
// list are each sorted by start.  Lane j < (number of lists) owns list j, the next lane owns the
// counting-filter ranges.  Each source's next 32 ranges sit in a shared-memory buffer that the
// warp refills with one coalesced load; every step the warp takes the smallest start (shuffle
// reduction over the owners' buffer heads), the owner advances, and overlapping or touching
// ranges are merged, so every maximal run of end positions lies in one output range.
__global__ void __launch_bounds__(kMergeWarps * 32)
    lc_kmerge_k(LcParams L, const uint64_t* doff, LcDesc* desc, const uint64_t* off, uint64_t* olo, uint64_t* ohi,
                uint32_t* ocnt, const uint64_t* ylist, uint32_t ny, uint32_t* cursor, uint32_t* n_serial) {
    __shared__ int64_t blo[kMergeWarps][32][kMergeBuf], bhi[kMergeWarps][32][kMergeBuf];
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (;;) {
        uint32_t yi = 0;
        if (lane == 0) yi = atomicAdd(cursor, 1u);  // largest segments first, then whoever is free
        yi = __shfl_sync(kFull, yi, 0);
        if (yi >= ny) break;
        const uint32_t y = (uint32_t)ylist[yi];
        const uint32_t r = L.list[y >> 1], s = y & 1;
        const int64_t m = L.len[r], k = L.kk[r];
        const uint64_t d0 = doff[y], d1 = doff[y + 1];
        const uint32_t nd = (uint32_t)(d1 - d0);
        const uint64_t o = off[y];
        if (nd >= 32) {
            if (lane == 0) {
                atomicAdd(n_serial, 1u);
                lc_kmerge_serial(L, r, s, d0, d1, desc, o, olo, ohi, ocnt + y);
            }
            __syncwarp();
            continue;
        }
        const uint32_t S = nd + 1;  // sources: nd cluster lists and the counting-filter ranges
        uint64_t cur = 0, end = 0;
        int64_t imin = 0, imax = 0;
        uint32_t cnt = 0, rd = 0;
        if (lane < nd) {
            cur = desc[d0 + lane].cb;
            end = desc[d0 + lane].ce;
            imin = desc[d0 + lane].imin;
            imax = desc[d0 + lane].imax;
        } else if (lane == nd) {
            cur = L.roff[r] + (s == 0 ? 0 : L.wcnt[2 * r]);
            end = cur + L.wcnt[2 * r + s];
        }
        // the first kMergeBuf lanes load the next (up to) kMergeBuf ranges of source j into its buffer
        auto refill = [&](uint32_t j) {
            const uint64_t c0 = __shfl_sync(kFull, cur, j), e0 = __shfl_sync(kFull, end, j);
            const int64_t mn = __shfl_sync(kFull, imin, j), mx = __shfl_sync(kFull, imax, j);
            const uint64_t e = c0 + lane;
            if (lane < kMergeBuf && e < e0) {
                int64_t lo, hi;
                if (j < nd) {
                    cluster_range(L, e, mn, mx, m, k, &lo, &hi);
                } else {
                    lo = (int64_t)(L.wlo[e] & kPosMask40);
                    hi = (int64_t)L.whi[e];
                }
                blo[wid][j][lane] = lo;
                bhi[wid][j][lane] = hi;
            }
            const uint32_t got = (uint32_t)(e0 - c0 < kMergeBuf ? e0 - c0 : kMergeBuf);
            if (lane == j) {
                cnt = got;
                rd = 0;
                cur += got;
            }
            __syncwarp();
        };
        for (uint32_t j = 0; j < S; ++j) refill(j);
        MergeOut M;
        M.join = m + k;
        while (true) {
            unsigned need = __ballot_sync(kFull, lane < S && rd == cnt && cur < end);
            while (need) {
                const uint32_t j = __ffs(need) - 1;
                need &= need - 1;
                refill(j);
            }
            uint64_t key = ~0ull;
            if (lane < S && rd < cnt) key = ((uint64_t)blo[wid][lane][rd] << 5) | lane;
            // warp minimum of the 64-bit keys: high halves first, then low halves among the ties
            const uint32_t kh = (uint32_t)(key >> 32);
            const uint32_t mh = __reduce_min_sync(kFull, kh);
            const uint32_t ml = __reduce_min_sync(kFull, kh == mh ? (uint32_t)key : 0xFFFFFFFFu);
            key = ((uint64_t)mh << 32) | ml;
            if (key == ~0ull) break;
            const uint32_t wl = (uint32_t)(key & 31);
            const int64_t lo = (int64_t)(key >> 5);
            const int64_t hi = bhi[wid][wl][__shfl_sync(kFull, rd, wl)];
            if (lane == wl) ++rd;
            int64_t a, b;
            if (M.add(lo, hi, &a, &b)) {
                if (lane == 0) {
                    olo[o + M.cnt] = (uint64_t)a;
                    ohi[o + M.cnt] = (uint64_t)b;
                }
                ++M.cnt;
            }
            __syncwarp();
        }
        if (lane == 0) {
            if (M.open) {
                olo[o + M.cnt] = (uint64_t)M.cur_lo;
                ohi[o + M.cnt] = (uint64_t)M.cur_hi;
            }
            ocnt[y] = M.cnt + (M.open ? 1 : 0);
        }
        __syncwarp();
    }
}

// ---- low-complexity merge, block path -------------------------------------------------------
//
// Most segments hold at most kMedCap ranges.  Their ranges (counting-filter ranges and every
// cluster range) are written as keys lo << 24 | (hi - lo), sorted by lo in shared memory by one
// block, and merged with a block-wide max-scan of hi: range j opens a merged range exactly when
// its lo lies beyond the largest hi before it by more than m + k, and that largest hi closes the
// previous merged range.  Segments with more ranges, or with a range of 2^24 bases or more, keep
// the k-way merge.

constexpr uint64_t kLcWide = (1ull << 24) - 1;  // widths from here on do not fit the key
constexpr uint64_t kLcDrop = ~0ull;             // a range clipped away (sorts last, skipped)

__device__ __forceinline__ int64_t block_excl_max64(int64_t v, int64_t* sc) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl = max(incl, t);
    }
    if (lane == 31) sc[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t y = sc[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(kFull, y, o);
            if (lane >= o) y = max(y, t);
        }
        sc[lane] = y;
    }
    __syncthreads();
    int64_t before = __shfl_up_sync(kFull, incl, 1);
    if (lane == 0) before = INT64_MIN;
    const int64_t r = max(before, w ? sc[w - 1] : INT64_MIN);
    __syncthreads();
    return r;
}

// One warp per segment: its ranges as sort keys at off[y]; wide[y] = 1 if a range does not fit.
__global__ void lc_gather_k(LcParams L, const uint64_t* __restrict__ doff, const LcDesc* __restrict__ desc,
                            const uint64_t* __restrict__ off, uint64_t* keys, uint32_t* wide) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t y = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; y < 2 * L.n_list; y += nw) {
        const uint32_t r = L.list[y >> 1], s = y & 1;
        const int64_t m = L.len[r], k = L.kk[r];
        uint64_t at = off[y];
        bool wd = false;
        auto put = [&](int64_t lo, int64_t hi, uint64_t pos) {
            uint64_t key = kLcDrop;
            if (lo <= hi) {
                const uint64_t width = (uint64_t)(hi - lo);
                if (width >= kLcWide) wd = true;
                key = ((uint64_t)lo << 24) | (width < kLcWide ? width : kLcWide);
            }
            keys[pos] = key;
        };
        const uint64_t w0 = L.roff[r] + (s == 0 ? 0 : L.wcnt[2 * r]), nwr = L.wcnt[2 * r + s];
        for (uint64_t e = lane; e < nwr; e += 32)
            put((int64_t)(L.wlo[w0 + e] & kPosMask40), (int64_t)L.whi[w0 + e], at + e);
        at += nwr;
        for (uint64_t d = doff[y]; d < doff[y + 1]; ++d) {
            const LcDesc D = desc[d];
            for (uint64_t c = D.cb + lane; c < D.ce; c += 32) {
                int64_t lo, hi;
                cluster_range(L, c, D.imin, D.imax, m, k, &lo, &hi);
                put(lo, hi, at + (c - D.cb));
            }
            at += D.ce - D.cb;
        }
        if (__any_sync(kFull, wd) && lane == 0) wide[y] = 1;
    }
}

// One block per segment (dynamic order): sort its keys by lo, merge, write the merged ranges to
// olo / ohi at off[y] and their number to ocnt[y].  Segments left for the k-way merge go to
// rest_list (count in rest[0]); cursor is rest[1].
__global__ void __launch_bounds__(kMedThreads, 1)
    lc_merge_med_k(LcParams L, const uint64_t* __restrict__ off, const uint64_t* __restrict__ keys,
                   const uint32_t* __restrict__ wide, int hi_bit, uint64_t* olo, uint64_t* ohi, uint32_t* ocnt,
                   uint32_t* rest_list, uint32_t* rest) {
    extern __shared__ uint64_t sm[];
    uint64_t* bufA = sm;
    uint64_t* bufB = sm + kMedCap;
    uint16_t* cnt = reinterpret_cast<uint16_t*>(sm + 2 * kMedCap);
    __shared__ uint32_t s_next, s_nv;
    __shared__ uint32_t s_tot[256];
    __shared__ uint32_t s_part[4 * 256];
    __shared__ int64_t s_sc64[32];
    __shared__ int64_t s_top;
    const uint32_t nseg = 2 * L.n_list;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(rest + 1, 1u);
        __syncthreads();
        const uint32_t y = s_next;
        if (y >= nseg) break;
        const uint64_t base = off[y];
        const uint64_t hall = off[y + 1] - base;
        const uint32_t h = hall > kMedCap ? kMedCap + 1 : (uint32_t)hall;
        if (h > kMedCap || wide[y]) {
            if (threadIdx.x == 0) rest_list[atomicAdd(rest, 1u)] = y;
            __syncthreads();
            continue;
        }
        const uint32_t r = L.list[y >> 1];
        const int64_t join = (int64_t)L.len[r] + L.kk[r];
        if (threadIdx.x == 0) s_nv = 0;
        __syncthreads();
        uint32_t nv = 0;
        for (uint32_t i = threadIdx.x; i < h; i += blockDim.x) {
            const uint64_t key = keys[base + i];
            bufA[i] = key;
            nv += key != kLcDrop ? 1u : 0u;
        }
        atomicAdd(&s_nv, nv);
        uint64_t* src = block_radix_sort(bufA, bufB, cnt, s_tot, s_part, h, 24, hi_bit);
        const uint32_t hv = s_nv;  // valid ranges, sorted by lo ahead of the dropped ones
        const uint32_t E = (hv + kMedThreads - 1) / kMedThreads;
        const uint32_t j0 = threadIdx.x * E;
        int64_t tmax = INT64_MIN;
        for (uint32_t e = 0; e < E; ++e) {
            const uint32_t j = j0 + e;
            if (j < hv) {
                const uint64_t key = src[j];
                tmax = max(tmax, (int64_t)(key >> 24) + (int64_t)(key & kLcWide));
            }
        }
        const int64_t pre = block_excl_max64(tmax, s_sc64);
        uint32_t ns = 0;
        int64_t run = pre;
        for (uint32_t e = 0; e < E; ++e) {
            const uint32_t j = j0 + e;
            if (j >= hv) break;
            const uint64_t key = src[j];
            const int64_t lo = (int64_t)(key >> 24), hi = lo + (int64_t)(key & kLcWide);
            if (j == 0 || lo > run + join) ++ns;
            run = max(run, hi);
        }
        uint32_t total = 0;
        uint32_t idx = block_excl_sum(ns, s_tot, &total);
        run = pre;
        for (uint32_t e = 0; e < E; ++e) {
            const uint32_t j = j0 + e;
            if (j >= hv) break;
            const uint64_t key = src[j];
            const int64_t lo = (int64_t)(key >> 24), hi = lo + (int64_t)(key & kLcWide);
            if (j == 0 || lo > run + join) {
                olo[base + idx] = (uint64_t)lo;
                if (idx > 0) ohi[base + idx - 1] = (uint64_t)run;
                ++idx;
            }
            run = max(run, hi);
        }
        if (threadIdx.x == kMedThreads - 1) s_top = max(pre, tmax);  // the largest hi of all
        __syncthreads();
        if (threadIdx.x == 0) {
            if (total) ohi[base + total - 1] = (uint64_t)s_top;
            ocnt[y] = total;
        }
        __syncthreads();
    }
}

// ---- candidate compaction ---------------------------------------------------------------

struct CandCount {
    const uint32_t* wcnt;
    const uint8_t* lowcx;
    const uint32_t* lcpos;
    const uint32_t* lcnt;
    __device__ uint64_t operator()(uint64_t r) const {
        if (lowcx && lowcx[r]) {
            const uint32_t x = lcpos[r];
            return (uint64_t)lcnt[2 * x] + lcnt[2 * x + 1];
        }
        return (uint64_t)wcnt[2 * r] + wcnt[2 * r + 1];
    }
};

__global__ void lcpos_k(const uint32_t* list, uint32_t n, uint32_t* lcpos) {
    const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n) lcpos[list[x]] = x;
}

// One warp per read copies its ranges (strand 0 first) into the candidate arrays.
__global__ void compact_k(uint32_t n_reads, CandCount cc, const uint64_t* __restrict__ coff,
                          const uint64_t* __restrict__ roff, const uint64_t* __restrict__ wlo,
                          const uint64_t* __restrict__ whi, const uint64_t* __restrict__ lc_off,
                          const uint64_t* __restrict__ lc_keys, const uint64_t* __restrict__ lc_vals,
                          uint64_t* __restrict__ cand_key, uint64_t* __restrict__ cand_hi) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_reads; r += nw) {
        const uint64_t o = coff[r];
        const uint64_t rk = (uint64_t)r << 41;
        if (cc.lowcx && cc.lowcx[r]) {
            const uint32_t x = cc.lcpos[r];
            const uint32_t c0 = cc.lcnt[2 * x], c1 = cc.lcnt[2 * x + 1];
#pragma unroll 4
            for (uint32_t j = lane; j < c0 + c1; j += 32) {
                const uint32_t s = j < c0 ? 0 : 1;
                const uint64_t src = lc_off[2 * x + s] + (s ? j - c0 : j);
                cand_key[o + j] = rk | ((uint64_t)s << 40) | lc_keys[src];
                cand_hi[o + j] = lc_vals[src];
            }
        } else {
            const uint32_t c = cc.wcnt[2 * r] + cc.wcnt[2 * r + 1];
#pragma unroll 4
            for (uint32_t j = lane; j < c; j += 32) {
                cand_key[o + j] = rk | wlo[roff[r] + j];
                cand_hi[o + j] = whi[roff[r] + j];
            }
        }
    }
}

// ---- candidate ranges cut at the reference's segment edges -----------------------------------
//
// Section "Overview": every step runs per chromosome, and long runs of N stay out of the index
// (Section "The q-group index").  A reference of several contigs, or with gaps, is a list of
// segments; a candidate range of end positions is cut into its pieces inside each segment it
// meets (a piece in no segment, i.e. in a gap, is dropped), so that verification can start the
// matrix at the segment start and no reported run crosses a segment edge.

// The first segment whose end lies after p (n_seg when none).
__device__ __forceinline__ uint32_t first_segment_after(const uint64_t* __restrict__ seg, uint32_t n_seg, uint64_t p) {
    uint32_t l = 0, h = n_seg;
    while (l < h) {
        const uint32_t mid = (l + h) >> 1;
        if (seg[2 * mid + 1] <= p)
            l = mid + 1;
        else
            h = mid;
    }
    return l;
}

// Number of pieces of candidate x: the segments that meet [lo, hi].
struct PieceCount {
    const uint64_t* key;
    const uint64_t* hi;
    const uint64_t* seg;
    uint32_t n_seg;
    __device__ uint64_t operator()(uint64_t x) const {
        const uint64_t lo = key[x] & kPosMask40, h = hi[x];
        uint64_t c = 0;
        for (uint32_t i = first_segment_after(seg, n_seg, lo); i < n_seg && seg[2 * i] <= h; ++i) ++c;
        return c;
    }
};

__global__ void seg_split_k(PieceCount pc, uint64_t n, const uint64_t* __restrict__ off, uint64_t* __restrict__ okey,
                            uint64_t* __restrict__ ohi) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t key = pc.key[x], lo = key & kPosMask40, h = pc.hi[x];
        uint64_t o = off[x];
        for (uint32_t i = first_segment_after(pc.seg, pc.n_seg, lo); i < pc.n_seg && pc.seg[2 * i] <= h; ++i) {
            const uint64_t sa = pc.seg[2 * i], sb = pc.seg[2 * i + 1];
            okey[o] = (key & ~kPosMask40) | (lo > sa ? lo : sa);
            ohi[o] = h < sb - 1 ? h : sb - 1;
            ++o;
        }
    }
}

// ---- bit-vector verification (Myers 1999 / Hyyro 2003; Section "Validation") ------------------
//
// Column j of the semiglobal matrix is held as vertical delta vectors Pv (+1) and Mv (-1), one
// bit per pattern row, as one W x 64-bit integer (word 0 = rows 1..64).  One column step is Myers'
// single-word recurrence on that wide integer: Xv = Eq | Mv; Xh = (((Eq & Pv) + Pv) ^ Pv) | Eq with
// the addition carried across words; Ph = Mv | ~(Xh | Pv); Mh = Pv & Xh; the horizontal delta at
// row m is bit m-1 of Ph minus that of Mh; Ph and Mh shift up one row with 0 shifted in (row 0
// has E[0][j] = 0 for every j); Pv = Mh | ~(Xv | Ph); Mv = Ph & Xv.  Initial column (j = a - 1):
// E[i][a-1] = i, all Pv set, score m.

// s = a + b over W 64-bit words, carries chained.
template <int W>
__device__ __forceinline__ void wide_add(const uint64_t (&a)[W], const uint64_t (&b)[W], uint64_t (&s)[W]) {
    if constexpr (W == 1) {
        s[0] = a[0] + b[0];
    } else if constexpr (W == 2) {
        asm("add.cc.u64 %0, %2, %4;\n\t"
            "addc.u64 %1, %3, %5;"
            : "=l"(s[0]), "=l"(s[1])
            : "l"(a[0]), "l"(a[1]), "l"(b[0]), "l"(b[1]));
    } else if constexpr (W == 3) {
        asm("add.cc.u64 %0, %3, %6;\n\t"
            "addc.cc.u64 %1, %4, %7;\n\t"
            "addc.u64 %2, %5, %8;"
            : "=l"(s[0]), "=l"(s[1]), "=l"(s[2])
            : "l"(a[0]), "l"(a[1]), "l"(a[2]), "l"(b[0]), "l"(b[1]), "l"(b[2]));
    } else {
        asm("add.cc.u64 %0, %4, %8;\n\t"
            "addc.cc.u64 %1, %5, %9;\n\t"
            "addc.cc.u64 %2, %6, %10;\n\t"
            "addc.u64 %3, %7, %11;"
            : "=l"(s[0]), "=l"(s[1]), "=l"(s[2]), "=l"(s[3])
            : "l"(a[0]), "l"(a[1]), "l"(a[2]), "l"(a[3]), "l"(b[0]), "l"(b[1]), "l"(b[2]), "l"(b[3]));
    }
}

// One column step on the wide vectors; returns the change of E[m][j] (lastbit = (m - 1) % 64,
// row m lives in word W - 1).
template <int W>
__device__ __forceinline__ int wide_step(uint64_t (&Pv)[W], uint64_t (&Mv)[W], const uint64_t (&e)[W], int lastbit) {
    uint64_t t[W], sum[W];
#pragma unroll
    for (int w = 0; w < W; ++w) t[w] = e[w] & Pv[w];
    wide_add<W>(t, Pv, sum);
    uint64_t ph[W], mh[W], xv[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const uint64_t xh = (sum[w] ^ Pv[w]) | e[w];
        xv[w] = e[w] | Mv[w];
        ph[w] = Mv[w] | ~(xh | Pv[w]);
        mh[w] = Pv[w] & xh;
    }
    const int delta = (int)((ph[W - 1] >> lastbit) & 1ull) - (int)((mh[W - 1] >> lastbit) & 1ull);
#pragma unroll
    for (int w = W - 1; w >= 0; --w) {
        const uint64_t p = (ph[w] << 1) | (w ? ph[w - 1] >> 63 : 0ull);
        const uint64_t q = (mh[w] << 1) | (w ? mh[w - 1] >> 63 : 0ull);
        Pv[w] = q | ~(xv[w] | p);
        Mv[w] = p & xv[w];
    }
    return delta;
}

template <int W>
struct Myers {
    uint64_t Pv[W], Mv[W];
    uint64_t eq[4][W];
    int32_t score;
    int lastbit;

    __device__ __forceinline__ void init(const uint64_t* __restrict__ peq, uint32_t m) {
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int w = 0; w < W; ++w) eq[c][w] = __ldg(peq + c * kMaxWords + w);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            Pv[w] = ~0ull;
            Mv[w] = 0;
        }
        score = (int32_t)m;
        lastbit = (int)((m - 1) & 63);
    }

    // Advances one text column with base code c; returns E[m][j].
    __device__ __forceinline__ int32_t step(uint32_t c) {
        uint64_t e[W];
#pragma unroll
        for (int w = 0; w < W; ++w) e[w] = c == 0 ? eq[0][w] : c == 1 ? eq[1][w] : c == 2 ? eq[2][w] : eq[3][w];
        score += wide_step<W>(Pv, Mv, e, lastbit);
        return score;
    }
};

struct VerifyParams {
    const uint64_t* cand_key;
    const uint64_t* cand_hi;
    uint64_t n_cand;
    const uint32_t* packed;
    const uint8_t* len;
    const uint8_t* kk;
    const uint64_t* peq;
    uint32_t* cnt;          // tuples per candidate
    uint64_t* inl;          // 2 inline tuples per candidate: end << 8 | dist
    unsigned long long* columns;  // [0] columns, [1] columns x words, [2] columns with D <= k
    // phase 2
    const uint64_t* toff;
    uint32_t* out_read;
    uint8_t* out_strand;
    uint64_t* out_end;
    uint8_t* out_dist;
};

constexpr int kVerifyThreads = 128;

// The same recurrence as Myers<W> with the match masks of the current pattern in shared memory,
// one slot per thread: eq(c, w) is read from seq[(c * kMaxWords + w) * blockDim].
template <int W>
struct MyersShared {
    uint64_t Pv[W], Mv[W];
    const uint64_t* seq;
    int32_t score;
    int lastbit;

    __device__ __forceinline__ int32_t step(uint32_t c) {
        uint64_t e[W];
#pragma unroll
        for (int w = 0; w < W; ++w) e[w] = seq[(c * kMaxWords + w) * kVerifyThreads];
        score += wide_step<W>(Pv, Mv, e, lastbit);
        return score;
    }
    // The recurrence alone, without tracking E[m][j] (warm-up columns).
    __device__ __forceinline__ void advance(uint32_t c) {
        uint64_t e[W];
#pragma unroll
        for (int w = 0; w < W; ++w) e[w] = seq[(c * kMaxWords + w) * kVerifyThreads];
        (void)wide_step<W>(Pv, Mv, e, lastbit);
    }
    // E[m][j] from the vertical deltas: E[0][j] = 0 and rows 1..m add +1 (Pv) or -1 (Mv).
    __device__ __forceinline__ void rescore() {
        int32_t v = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint64_t rows = (w < W - 1 || lastbit == 63) ? ~0ull : ((1ull << (lastbit + 1)) - 1);
            v += __popcll(Pv[w] & rows) - __popcll(Mv[w] & rows);
        }
        score = v;
    }
};

// Start of the reference segment holding position p (n_seg >= 1 segments as [start, end) pairs,
// ascending; p inside one of them).
__device__ __forceinline__ int64_t segment_start(const uint64_t* __restrict__ seg, uint32_t n_seg, int64_t p) {
    uint32_t l = 0, h = n_seg;
    while (l < h) {
        const uint32_t mid = (l + h) >> 1;
        if ((int64_t)__ldg(seg + 2 * mid + 1) <= p)
            l = mid + 1;
        else
            h = mid;
    }
    return (int64_t)__ldg(seg + 2 * (l < n_seg ? l : n_seg - 1));
}

// Verifies one candidate range: columns a .. hi of the pattern's semiglobal matrix, runs of ends
// with distance <= k, leftmost minimum of each run.  Returns the number of columns.  Columns
// before lo only warm the recurrence up; whole packed words (16 bases) are stepped unrolled.  The
// range lies inside one segment of the reference (contig, or stretch between runs of N): the
// matrix starts at that segment's start at the earliest, so no alignment leaves it.
template <int W, bool kWrite>
__device__ uint64_t verify_one(const VerifyParams& V, uint64_t x, uint64_t* seq, unsigned long long& useful,
                               const uint64_t* __restrict__ seg, uint32_t n_seg) {
    const uint64_t key = V.cand_key[x];
    const uint32_t r = (uint32_t)(key >> 41), s = (uint32_t)(key >> 40) & 1u;
    const int64_t lo = (int64_t)(key & kPosMask40), hi = (int64_t)V.cand_hi[x];
    const uint32_t m = V.len[r];
    const int32_t k = V.kk[r];
    // the first column: m + k before lo, but not before the start of lo's segment (ranges were
    // cut at segment edges, so the whole range lies in that segment)
    int64_t a = lo - ((int64_t)m + k) + 1;
    if (a < 0) a = 0;
    if (seg) {
        const int64_t sa = segment_start(seg, n_seg, lo);
        if (a < sa) a = sa;
    }
    const uint64_t* pq = V.peq + ((uint64_t)r * 2 + s) * 4 * kMaxWords;
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int w = 0; w < W; ++w) seq[(c * kMaxWords + w) * kVerifyThreads] = __ldg(pq + c * kMaxWords + w);
    MyersShared<W> M;
    M.seq = seq;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        M.Pv[w] = ~0ull;
        M.Mv[w] = 0;
    }
    M.score = (int32_t)m;
    M.lastbit = (int)((m - 1) & 63);
    uint32_t nt = 0;
    uint64_t o = kWrite ? V.toff[x] : 0;
    bool in = false;
    int32_t best = 0;
    int64_t bestj = 0;
    auto emit = [&]() {
        if (kWrite) {
            V.out_read[o] = r;
            V.out_strand[o] = (uint8_t)s;
            V.out_end[o] = (uint64_t)bestj;
            V.out_dist[o] = (uint8_t)best;
            ++o;
        } else if (nt < 2) {
            V.inl[2 * x + nt] = ((uint64_t)bestj << 8) | (uint64_t)best;
        }
        ++nt;
    };
    auto column = [&](uint32_t c, int64_t jj) {
        const int32_t d = M.step(c);
        if (d <= k) {
            if (!kWrite) ++useful;
            if (!in || d < best) {
                best = d;
                bestj = jj;
            }
            in = true;
        } else if (in) {
            emit();
            in = false;
        }
    };
    int64_t j = a;
    // warm-up: head of the first word, then whole words, then the tail; the score is recovered
    // from the bit vectors at the end
    if (j < lo) {
        uint32_t word = __ldg(V.packed + (j >> 4)) << (2 * (uint32_t)(j & 15));
        while (j < lo && (j & 15)) {
            M.advance(word >> 30);
            word <<= 2;
            ++j;
        }
#pragma unroll 1
        while (j + 16 <= lo) {
            uint32_t wd = __ldg(V.packed + (j >> 4));
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                M.advance(wd >> 30);
                wd <<= 2;
            }
            j += 16;
        }
        if (j < lo) {
            word = __ldg(V.packed + (j >> 4));
            while (j < lo) {
                M.advance(word >> 30);
                word <<= 2;
                ++j;
            }
        }
        M.rescore();
    }
    // reported columns lo .. hi
    while (j <= hi && (j & 15)) {
        column((__ldg(V.packed + (j >> 4)) >> (30 - 2 * (uint32_t)(j & 15))) & 3u, j);
        ++j;
    }
#pragma unroll 1
    while (j + 16 <= hi + 1) {
        uint32_t wd = __ldg(V.packed + (j >> 4));
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            column(wd >> 30, j + u);
            wd <<= 2;
        }
        j += 16;
    }
    if (j <= hi) {
        uint32_t word = __ldg(V.packed + (j >> 4));
        while (j <= hi) {
            column(word >> 30, j);
            word <<= 2;
            ++j;
        }
    }
    if (in) emit();
    if (!kWrite) V.cnt[x] = nt;
    return (uint64_t)(hi - a + 1);
}

// ---- q'-gram counting filter on candidate ranges (the q-gram lemma per end position) ---------
//
// An alignment of a read of length m with e <= k edits ending at reference position j keeps at
// least m - q' + 1 - q' e of the read's q'-grams intact (each edit touches at most q' of them;
// Section "The q-group index", q-gram lemma), and every intact one occurs in the reference at a
// distinct start position p in [j - m - k + 1, j - q' + 1] (the alignment spans at most m + k
// bases).  So an end j can have distance <= k only if at least T' = m - q' + 1 - q' k reference
// positions of that window start a q'-gram that occurs in the read.  The filter counts such
// positions per 16-base block of the reference (one packed word) and, for every block of end
// positions, sums the counts of the blocks its windows can reach: ends in blocks whose sum is
// below T' cannot hold a hit.  The intact q'-grams are moreover a sub-multiset of the read's, so
// a q'-gram that the window repeats more often than the read holds it counts only as often as
// the read holds it: the count less that excess for the read's most frequent q'-grams is a
// tighter bound, and on tandem-run text (where the low-complexity reads' candidates lie) it
// removes most of what the plain count keeps.  A candidate range shrinks to its first .. last
// surviving block (or is dropped), and the bit-vector verification runs only there, with its
// usual m + k warm-up columns before the new start.  q' = 4: the read's 4-gram set is a 256-bit
// table per (read, strand).  The result is unchanged: no end with distance <= k is removed.
constexpr int kQf = 4;                  // q'
constexpr int kFilterThreads = 128;
constexpr uint64_t kDeadRange = ~0ull;  // cand_hi of a range the filter removed

__device__ __forceinline__ uint32_t rc4(uint32_t g) {
    return (3u - (g & 3u)) << 6 | (3u - ((g >> 2) & 3u)) << 4 | (3u - ((g >> 4) & 3u)) << 2 | (3u - (g >> 6));
}

// 4-gram sets of every read: qset[(r * 2 + s) * 8 + w] bit b = 4-gram 32 w + b occurs in the
// read (s = 0) or in its reverse complement (s = 1); qtop[r * 2 + s] = the four 4-grams occurring
// most often there (x: one code per byte, y: their counts per byte, 0xFF for an unused slot;
// ties go to the smaller code).  One warp per read.
__global__ void __launch_bounds__(256)
    qset_k(const uint8_t* __restrict__ codes, const uint64_t* __restrict__ base_off, uint32_t n_reads,
           uint32_t* __restrict__ qset, uint2* __restrict__ qtop) {
    __shared__ uint32_t s_hist[8][256];
    const uint32_t lane = threadIdx.x & 31;
    uint32_t* hist = s_hist[threadIdx.x >> 5];
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_reads; r += nw) {
        const uint64_t b = base_off[r], m = base_off[r + 1] - b;
#pragma unroll
        for (int e = 0; e < 8; ++e) hist[lane * 8 + e] = 0;
        __syncwarp();
        uint32_t f[8] = {}, rc[8] = {};
        for (uint64_t i = lane; i + kQf <= m; i += 32) {
            const uint32_t g = (uint32_t)codes[b + i] << 6 | (uint32_t)codes[b + i + 1] << 4 |
                               (uint32_t)codes[b + i + 2] << 2 | (uint32_t)codes[b + i + 3];
            // reverse complement: complement every base (3 - c) and reverse their order
            const uint32_t h = rc4(g);
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                f[w] |= (g >> 5) == (uint32_t)w ? 1u << (g & 31) : 0u;
                rc[w] |= (h >> 5) == (uint32_t)w ? 1u << (h & 31) : 0u;
            }
            atomicAdd(&hist[g], 1u);
        }
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const uint32_t a = __reduce_or_sync(kFull, f[w]), c = __reduce_or_sync(kFull, rc[w]);
            if (lane == 0) {
                qset[(uint64_t)r * 16 + w] = a;
                qset[(uint64_t)r * 16 + 8 + w] = c;
            }
        }
        __syncwarp();
        // the four most frequent codes: four rounds of a warp-wide maximum over (count, -code)
        uint32_t tc = 0, tn = 0, rtc = 0;
#pragma unroll 1
        for (int t = 0; t < 4; ++t) {
            uint32_t best = 0;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint32_t g = lane * 8 + e, v = (hist[g] << 8) | (255u - g);
                best = v > best ? v : best;
            }
            best = __reduce_max_sync(kFull, best);
            const uint32_t cnt = best >> 8, g = 255u - (best & 255u);
            __syncwarp();
            if (lane == 0) hist[g] = 0;
            __syncwarp();
            tc |= g << (8 * t);
            rtc |= rc4(g) << (8 * t);
            tn |= (cnt ? cnt : 0xFFu) << (8 * t);  // an unused slot never limits the count
        }
        if (lane == 0) {
            qtop[(uint64_t)r * 2] = make_uint2(tc, tn);
            qtop[(uint64_t)r * 2 + 1] = make_uint2(rtc, tn);
        }
        __syncwarp();
    }
}

// One thread per candidate range, in verification order (similar lengths share a warp).  Writes
// the narrowed range in place (cand_hi = kDeadRange if nothing survives); fstats[0] += reference
// positions scanned, fstats[1] += surviving ranges, fstats[2] += columns the verification would
// have run without the filter.
//
// The bound per block J of end positions, over the union U of the blocks J - D .. J that its
// windows reach: the intact q'-grams of an alignment are a sub-multiset of both the read's and
// the window's q'-grams, so their number is at most sum over g of min(cnt_read(g), cnt_U(g)) <=
// (positions of U holding a q'-gram of the read) - sum over the tracked g of
// max(0, cnt_U(g) - cnt_read(g)), for any set of tracked q'-grams; the read's four most frequent
// ones are tracked (on tandem-run text the window repeats a few q'-grams far more often than the
// read holds them).  Their per-block counts are kept four to a word (one byte each, at most 16).
__global__ void __launch_bounds__(kFilterThreads)
    qfilter_k(uint64_t* __restrict__ cand_key, uint64_t* __restrict__ cand_hi, const uint64_t* __restrict__ order,
              uint64_t n, const uint32_t* __restrict__ packed, const uint8_t* __restrict__ len,
              const uint8_t* __restrict__ kk, const uint32_t* __restrict__ qset, const uint2* __restrict__ qtop,
              unsigned long long* fstats) {
    __shared__ uint32_t s_set[8 * kFilterThreads];
    __shared__ uint8_t s_ring[32 * kFilterThreads];
    __shared__ uint32_t s_ring4[32 * kFilterThreads];
    uint32_t* set = s_set + threadIdx.x;
    uint8_t* ring = s_ring + threadIdx.x;
    uint32_t* ring4 = s_ring4 + threadIdx.x;
    unsigned long long scanned = 0, live = 0, before = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = order[i];
        const uint64_t key = cand_key[x];
        const uint32_t r = (uint32_t)(key >> 41), s = (uint32_t)(key >> 40) & 1u;
        const int64_t lo = (int64_t)(key & kPosMask40), hi = (int64_t)cand_hi[x];
        const int64_t m = len[r], k = kk[r];
        const int64_t a = lo - (m + k) + 1 < 0 ? 0 : lo - (m + k) + 1;
        before += (unsigned long long)(hi - a + 1);
        const int64_t T = m - kQf + 1 - (int64_t)kQf * k;  // T'
        if (T <= 0) {  // nothing can be excluded
            ++live;
            continue;
        }
#pragma unroll
        for (int w = 0; w < 8; ++w) set[w * kFilterThreads] = __ldg(qset + ((uint64_t)r * 2 + s) * 8 + w);
        const uint2 top = __ldg(qtop + (uint64_t)r * 2 + s);
        const uint32_t G4 = top.x;  // tracked codes, one per byte
        int32_t cr[4];              // their counts in the read (an unused slot never limits)
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const uint32_t c = (top.y >> (8 * h)) & 0xFFu;
            cr[h] = c == 0xFFu ? 0x7FFFFFFF : (int32_t)c;
        }
        const int64_t D = (m + k - 1 + 15) >> 4;  // blocks a window reaches before its own
        const int64_t B0 = a >> 4, J0 = lo >> 4, J1 = hi >> 4;
        int32_t sum = 0;
        uint32_t u02 = 0, u13 = 0;  // union counts of tracked codes 0 / 2 and 1 / 3 (16 bits each)
        int64_t first = -1, last = -1;
        uint32_t wc = __ldg(packed + B0);
#pragma unroll 1
        for (int64_t w = B0; w <= J1; ++w) {
            const uint32_t wn = __ldg(packed + w + 1);
            int32_t cnt = 0;
            uint32_t pc = 0;  // per-byte counts of the tracked codes in this block
            // the word shifted by 0, 1, 2 and 3 bases: the 4-gram at base 4 j + q is byte 3 - j of
            // the q-th shift
            const uint32_t sh[4] = {wc, __funnelshift_l(wn, wc, 2), __funnelshift_l(wn, wc, 4),
                                    __funnelshift_l(wn, wc, 6)};
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t g = __byte_perm(sh[q], 0u, 0x4440u | (uint32_t)(3 - j));
                    const uint32_t sw = set[(g >> 5) * kFilterThreads];
                    cnt += (int32_t)(__funnelshift_r(sw, sw, g) & 1u);  // bit g mod 32 (a rotation)
                    const uint32_t xq = G4 ^ (g * 0x01010101u);  // zero bytes: tracked codes equal to g
                    const uint32_t zb = ~(((xq & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | xq) & 0x80808080u;
                    pc += zb >> 7;
                }
            ring[(w & 31) * kFilterThreads] = (uint8_t)cnt;
            ring4[(w & 31) * kFilterThreads] = pc;
            sum += cnt;
            u02 += pc & 0x00FF00FFu;
            u13 += (pc >> 8) & 0x00FF00FFu;
            if (w - D - 1 >= B0) {
                const uint32_t slot = (uint32_t)((w - D - 1) & 31) * kFilterThreads;
                sum -= ring[slot];
                const uint32_t old = ring4[slot];
                u02 -= old & 0x00FF00FFu;
                u13 -= (old >> 8) & 0x00FF00FFu;
            }
            if (w >= J0) {
                const int32_t ex = max(0, (int32_t)(u02 & 0xFFFFu) - cr[0]) + max(0, (int32_t)(u13 & 0xFFFFu) - cr[1]) +
                                   max(0, (int32_t)(u02 >> 16) - cr[2]) + max(0, (int32_t)(u13 >> 16) - cr[3]);
                if (sum - ex >= T) {
                    if (first < 0) first = w;
                    last = w;
                }
            }
            wc = wn;
        }
        scanned += (unsigned long long)(J1 - B0 + 1) * 16;
        if (first < 0) {
            cand_hi[x] = kDeadRange;
        } else {
            const int64_t nlo = first * 16 > lo ? first * 16 : lo;
            const int64_t nhi = last * 16 + 15 < hi ? last * 16 + 15 : hi;
            cand_key[x] = (key & ~kPosMask40) | (uint64_t)nlo;
            cand_hi[x] = (uint64_t)nhi;
            ++live;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        scanned += __shfl_xor_sync(kFull, scanned, o);
        live += __shfl_xor_sync(kFull, live, o);
        before += __shfl_xor_sync(kFull, before, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(fstats, scanned);
        atomicAdd(fstats + 1, live);
        atomicAdd(fstats + 2, before);
    }
}

// Work order of the verification: candidates grouped by words per column and by length (8-column
// steps up to 384 columns, 64-column steps up to 1344, longer ones together), so that the 32
// ranges of a warp take about the same number of steps; one 8-bit key, one radix pass.  Ranges
// the q'-gram filter removed sort last.
constexpr int kOrderBits = 8;
__global__ void order_key_k(const uint64_t* __restrict__ cand_key, const uint64_t* __restrict__ cand_hi, uint64_t n,
                            const uint8_t* __restrict__ len, const uint8_t* __restrict__ kk, uint64_t* keys,
                            uint64_t* vals) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
        vals[x] = x;
        if (cand_hi[x] == kDeadRange) {
            keys[x] = 255;
            continue;
        }
        const uint64_t key = cand_key[x];
        const uint32_t r = (uint32_t)(key >> 41);
        const int64_t lo = (int64_t)(key & kPosMask40), hi = (int64_t)cand_hi[x];
        const uint32_t m = len[r];
        int64_t a = lo - ((int64_t)m + kk[r]) + 1;
        if (a < 0) a = 0;
        const uint64_t c8 = (uint64_t)(hi - a + 1) >> 3;
        const uint64_t b = c8 < 48 ? c8 : 48 + ((c8 - 48) >> 3);
        const uint64_t w = (m + 63) >> 6;
        keys[x] = ((w - 1) << 6) | (b < 62 ? b : 62);  // at most 254
    }
}

template <bool kWrite>
__global__ void __launch_bounds__(kVerifyThreads, 8)
    verify_k(VerifyParams V, const uint64_t* __restrict__ order, const unsigned long long* __restrict__ n_live,
             const uint64_t* __restrict__ seg, uint32_t n_seg) {
    __shared__ uint64_t s_eq[4 * kMaxWords * kVerifyThreads];
    uint64_t* seq = s_eq + threadIdx.x;
    unsigned long long cols = 0, wcols = 0, useful = 0;
    const uint64_t nl = *n_live;  // surviving ranges come first in `order`
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nl;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = order[i];
        if (kWrite && V.cnt[x] <= 2) continue;
        const uint32_t r = (uint32_t)(V.cand_key[x] >> 41);
        const uint32_t W = (V.len[r] + 63) >> 6;
        uint64_t c = 0;
        switch (W) {
            case 1: c = verify_one<1, kWrite>(V, x, seq, useful, seg, n_seg); break;
            case 2: c = verify_one<2, kWrite>(V, x, seq, useful, seg, n_seg); break;
            case 3: c = verify_one<3, kWrite>(V, x, seq, useful, seg, n_seg); break;
            default: c = verify_one<4, kWrite>(V, x, seq, useful, seg, n_seg); break;
        }
        cols += c;
        wcols += c * W;
    }
    if (!kWrite) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cols += __shfl_xor_sync(kFull, cols, o);
            wcols += __shfl_xor_sync(kFull, wcols, o);
            useful += __shfl_xor_sync(kFull, useful, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(V.columns, cols);
            atomicAdd(V.columns + 1, wcols);
            atomicAdd(V.columns + 2, useful);
        }
    }
}

__global__ void inline_out_k(VerifyParams V) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < V.n_cand;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = V.cnt[x];
        if (c == 0 || c > 2) continue;
        const uint64_t key = V.cand_key[x];
        const uint32_t r = (uint32_t)(key >> 41), s = (uint32_t)(key >> 40) & 1u;
        const uint64_t o = V.toff[x];
        for (uint32_t t = 0; t < c; ++t) {
            const uint64_t v = V.inl[2 * x + t];
            V.out_read[o + t] = r;
            V.out_strand[o + t] = (uint8_t)s;
            V.out_end[o + t] = v >> 8;
            V.out_dist[o + t] = (uint8_t)(v & 255u);
        }
    }
}

// ---- best stratum ------------------------------------------------------------------------

__global__ void min_dist_k(const uint32_t* rd, const uint8_t* dist, uint64_t n, uint32_t* mind) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (uint64_t)gridDim.x * blockDim.x)
        atomicMin(mind + rd[x], (uint32_t)dist[x]);
}

struct KeepBest {
    const uint32_t* rd;
    const uint8_t* dist;
    const uint32_t* mind;
    __device__ uint64_t operator()(uint64_t x) const { return dist[x] == mind[rd[x]] ? 1 : 0; }
};

__global__ void keep_best_k(KeepBest kb, uint64_t n, const uint64_t* pos, const uint32_t* rd, const uint8_t* st,
                            const uint64_t* en, const uint8_t* di, uint32_t* ord, uint8_t* ost, uint64_t* oen,
                            uint8_t* odi) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (uint64_t)gridDim.x * blockDim.x) {
        if (!kb(x)) continue;
        const uint64_t o = pos[x];
        ord[o] = rd[x];
        ost[o] = st[x];
        oen[o] = en[x];
        odi[o] = di[x];
    }
}

// ---- driver -------------------------------------------------------------------------------

static void alloc_hits(DeviceHits* H, uint64_t n, cudaStream_t s);

void best_stratum(const peanut_device_hits& in, uint32_t n_reads, DeviceHits* out, cudaStream_t s) {
    const uint64_t NT = in.n;
    if (!NT) {
        alloc_hits(out, 0, s);
        return;
    }
    DBuf<uint32_t> mind(n_reads ? n_reads : 1, s);
    PN_CUDA(cudaMemsetAsync(mind.p, 0xFF, (uint64_t)mind.n * sizeof(uint32_t), s));
    DBuf<uint64_t> tot(1, s);
    min_dist_k<<<grid_for(NT, 256, (unsigned)sm_count() * 16), 256, 0, s>>>(in.read_id, in.dist, NT, mind.p);
    PN_CHECK_LAUNCH();
    KeepBest kb{in.read_id, in.dist, mind.p};
    DBuf<uint64_t> pos(NT, s);
    exclusive_scan(kb, ArrayOut<uint64_t>{pos.p}, NT, tot.p, s);
    alloc_hits(out, to_host(tot.p, s), s);
    keep_best_k<<<grid_for(NT, 256, (unsigned)sm_count() * 16), 256, 0, s>>>(
        kb, NT, pos.p, in.read_id, in.strand, in.end_pos, in.dist, out->h.read_id, out->h.strand, out->h.end_pos,
        out->h.dist);
    PN_CHECK_LAUNCH();
}

// Milliseconds between two recorded events (0, and no error left behind, if either was not
// recorded).
static float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float t = 0;
    if (cudaEventElapsedTime(&t, a, b) != cudaSuccess) {
        cudaGetLastError();
        t = 0;
    }
    return t;
}

struct Timer {
    cudaEvent_t ev[12];
    int n = 0;
    cudaStream_t s;
    explicit Timer(cudaStream_t st) : s(st) {
        for (auto& e : ev) PN_CUDA(cudaEventCreate(&e));
    }
    ~Timer() {
        for (auto& e : ev) cudaEventDestroy(e);
    }
    void mark() { PN_CUDA(record_event(ev[n++], s)); }
    void mark_at(int i) { PN_CUDA(record_event(ev[i], s)); }
    float ms(int a, int b) { return elapsed(ev[a], ev[b]); }
};

static void alloc_hits(DeviceHits* H, uint64_t n, cudaStream_t s) {
    H->stream = s;
    H->h.n = n;
    H->a = current_allocator();
    const uint64_t c = n ? n : 1;
    H->h.read_id = static_cast<uint32_t*>(dalloc(c * sizeof(uint32_t), s));
    H->h.strand = static_cast<uint8_t*>(dalloc(c, s));
    H->h.end_pos = static_cast<uint64_t*>(dalloc(c * sizeof(uint64_t), s));
    H->h.dist = static_cast<uint8_t*>(dalloc(c, s));
}

void alloc_device_hits(DeviceHits* H, uint64_t n, cudaStream_t s) { alloc_hits(H, n, s); }

static void free_hits_arrays(DeviceHits* H) {
    if (H->h.read_id) dfree(H->h.read_id, H->stream, H->a);
    if (H->h.strand) dfree(H->h.strand, H->stream, H->a);
    if (H->h.end_pos) dfree(H->h.end_pos, H->stream, H->a);
    if (H->h.dist) dfree(H->h.dist, H->stream, H->a);
    H->h = peanut_device_hits{};
}

DeviceHits* map_batch(const peanut_ref* ref, peanut_reads* R, int mode) {
    cudaStream_t s = R->stream;
    const uint32_t n_reads = R->n_reads, q = R->q;
    const uint64_t n = ref->n;
    PN_REQUIRE(R->max_k < 64, PEANUT_UNSUPPORTED, "error budgets above 63 are not supported (max k = %u)", R->max_k);
    Timer tm(s);
    Timer ktm(s);
    cudaEvent_t* kev = ktm.ev;
    peanut_map_stats st = {};
    tm.mark();  // 0

    // 1. reference scan: present positions, then their hits
    DBuf<uint32_t> rcount((uint64_t)n_reads + 1, s);
    DBuf<unsigned long long> nh(2, s);  // [0] present positions, [1] hits
    const double rand_hits = 2.0 * (double)n * (double)R->n_indexed / (double)(1ull << (2 * q));
    const double rand_present = 2.0 * (double)n * (double)R->n_distinct / (double)(1ull << (2 * q));
    uint64_t pcap = (uint64_t)(1.5 * rand_present) + 2 * R->n_indexed + (1u << 20);
    uint64_t cap = (uint64_t)(1.5 * rand_hits) + 2 * R->n_indexed + (1u << 20);
    int per_sm = 0;
    PN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, probe_ref_k<0, true>, kScanBlock, 0));
    const unsigned gscan = (unsigned)sm_count() * (unsigned)(per_sm > 0 ? per_sm : 1);  // one resident wave
    const unsigned gexp = (unsigned)sm_count() * 8;  // persistent: the count of present positions is on the device
    // Sync-free stretches run as CUDA graphs on the executors of an engine created with graphs = 1;
    // elsewhere the same launches run one by one.
    const bool graphs = graphs_on_this_thread();
    DBuf<uint64_t> pkey;
    DBuf<uint32_t> pslot;
    DBuf<uint64_t> hits;
    uint64_t NP = 0, H = 0;
    const RefIndex* RX = R->rindex.get();
    for (int attempt = 0;; ++attempt) {
        // capacity-sized buffers; the kernels count past the capacity, so an overflow is seen once
        // afterwards and the scan runs again with the exact sizes
        if (!RX) {
            pkey.alloc(pcap, s);
            pslot.alloc(pcap, s);
        }
        hits.alloc(cap, s);
        GraphSegment seg(s, graphs);
        PN_CUDA(record_event(kev[0], s));
        nh.zero();
        rcount.zero();
        if (!RX) {
            const IndexView IV = index_view(R);
            auto launch = [&](auto k16, auto kq) {
                (q == 16 ? k16 : kq)<<<gscan, kScanBlock, 0, s>>>(ref->packed.p, n, q, IV, R->bloom.p,
                                                                  R->bloom_mask, pkey.p, pslot.p, pcap, nh.p);
            };
            switch (R->layout) {
                case 0: launch(probe_ref_k<0, true>, probe_ref_k<0, false>); break;
                case 1: launch(probe_ref_k<1, true>, probe_ref_k<1, false>); break;
                default: launch(probe_ref_k<2, true>, probe_ref_k<2, false>); break;
            }
            PN_CHECK_LAUNCH();
        }
        PN_CUDA(record_event(kev[7], s));
        if (RX) {
            refprobe_k<<<grid_for(R->n_indexed, kScanBlock, (unsigned)sm_count() * 8), kScanBlock, 0, s>>>(
                R->O.p, R->n_indexed, q, R->codes.p, R->base_off.p, R->len.p, RX->IS.p, RX->Sp.p, RX->O.p,
                RX->orient.p, hits.p, cap, nh.p + 1, rcount.p);
        } else {
            expand_k<<<gexp, kScanBlock, 0, s>>>(pkey.p, pslot.p, nh.p, pcap, q, R->Sp.p, R->O.p, R->len.p, hits.p,
                                                  cap, nh.p + 1, rcount.p);
        }
        PN_CHECK_LAUNCH();
        PN_CUDA(record_event(kev[1], s));
        st.graph_segments += seg.run() ? 1 : 0;
        unsigned long long c[2];
        PN_CUDA(cudaMemcpyAsync(c, nh.p, sizeof(c), cudaMemcpyDeviceToHost, s));
        PN_CUDA(cudaStreamSynchronize(s));
        NP = c[0];
        H = c[1];
        if ((RX || NP <= pcap) && H <= cap) break;
        st.scan_retries++;
        if (!RX && NP > pcap) pcap = NP + (NP >> 4) + 1024;
        if (H > cap) cap = H + (H >> 4) + 1024;
        PN_REQUIRE(attempt < 3, PEANUT_NO_MEMORY, "present-position or hit buffer kept overflowing");
    }
    st.present_probes = RX ? R->n_indexed : NP;
    pkey.reset();
    pslot.reset();
    st.hits = H;
    tm.mark();  // 1

    // 2. bin by read, 3. windows of reads with few hits (one graph)
    DBuf<uint64_t> roff((uint64_t)n_reads + 1, s), tot(1, s);
    DBuf<uint64_t> binned(H ? H : 1, s);
    DBuf<uint64_t> wlo(H ? H : 1, s), whi(H ? H : 1, s);
    DBuf<uint32_t> wcnt(2 * (uint64_t)n_reads, s);
    DBuf<uint32_t> big_list(n_reads, s), med_list(n_reads, s), nbig(3, s);  // big, medium, cursor
    WinParams WP{roff.p, R->len.p, R->kk.p, R->thr.p, n, wlo.p, whi.p, wcnt.p};
    uint32_t nbm[2];
    {
        GraphSegment seg(s, graphs);
        exclusive_scan(ArrayIn<uint32_t>{rcount.p}, ArrayOut<uint64_t>{roff.p}, n_reads, tot.p, s);
        PN_CUDA(cudaMemcpyAsync(roff.p + n_reads, tot.p, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        rcount.zero();
        bin_hits_k<<<grid_for(H, 256, (unsigned)sm_count() * 16), 256, 0, s>>>(hits.p, H, roff.p, rcount.p,
                                                                                binned.p);
        PN_CHECK_LAUNCH();
        tm.mark();  // 2
        nbig.zero();
        windows_k<<<grid_for((uint64_t)n_reads * 32, kWinWarps * 32, (unsigned)sm_count() * 16), kWinWarps * 32, 0,
                    s>>>(binned.p, n_reads, WP, big_list.p, nbig.p, med_list.p);
        PN_CHECK_LAUNCH();
        st.graph_segments += seg.run() ? 1 : 0;
        PN_CUDA(cudaMemcpyAsync(nbm, nbig.p, sizeof(nbm), cudaMemcpyDeviceToHost, s));
        PN_CUDA(cudaStreamSynchronize(s));
    }
    hits.reset();
    const uint32_t n_big = nbm[0], n_med = nbm[1];
    st.med_reads = n_med;
    st.big_reads = n_big;
    PN_CUDA(record_event(kev[8], s));
    if (n_med) {
        // opt in to the block path's shared memory (a per-device function attribute; cheap to repeat)
        PN_CUDA(cudaFuncSetAttribute(windows_med_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMedSmem));
        // keys as strand << sbit | biased diagonal: 33 bits when the reference allows
        const int sbit = (n + (uint64_t)kDiagBias + 1) < (1ull << 32) ? 32 : 40;
        windows_med_k<<<grid_for(n_med, 1, (unsigned)sm_count()), kMedThreads, kMedSmem, s>>>(
            binned.p, med_list.p, n_med, WP, nbig.p + 2, sbit);
        PN_CHECK_LAUNCH();
    }
    PN_CUDA(record_event(kev[9], s));
    if (n_big) {
        DBuf<uint64_t> goff((uint64_t)n_big + 1, s);
        exclusive_scan(BigSize{big_list.p, roff.p}, ArrayOut<uint64_t>{goff.p}, n_big, tot.p, s);
        PN_CUDA(cudaMemcpyAsync(goff.p + n_big, tot.p, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        const uint64_t nbk = to_host(tot.p, s);
        DBuf<uint64_t> bk(nbk, s), btmp(nbk, s);
        big_gather_k<<<grid_for((uint64_t)n_big * 32, 256), 256, 0, s>>>(binned.p, big_list.p, n_big, roff.p,
                                                                          goff.p, bk.p);
        PN_CHECK_LAUNCH();
        int bits = 0;
        while ((1ull << bits) < n_big) ++bits;
        radix_sort_u64(bk.p, btmp.p, nbk, 41 + bits, s);
        big_sweep_k<<<grid_for((uint64_t)n_big * 32, 256), 256, 0, s>>>(bk.p, big_list.p, n_big, goff.p, WP);
        PN_CHECK_LAUNCH();
    }
    binned.reset();
    ktm.mark_at(4);

    // 3b. low-complexity reads: their counting-filter ranges and a range around every cluster of
    // their frequent q-grams, merged per (read, strand)
    const RefPrep* P = R->prep.get();
    const uint32_t nl = R->n_lowcx;
    DBuf<uint32_t> lcpos, lcnt;
    DBuf<uint64_t> lc_off, lc_keys, lc_vals;
    if (nl) {
        const uint64_t nseg = 2 * (uint64_t)nl;
        LcParams L{R->lowcx_list.p, nl, R->qoff.p, R->fcnt.p, R->fent.p, R->len.p, R->kk.p, q, n,
                   P->grp_off.p, P->cl_lo.p, P->cl_hi.p, roff.p, wlo.p, whi.p, wcnt.p, R->codes.p,
                   R->base_off.p, ref->packed.p};
        lc_sort_k<<<grid_for(nl, 128), 128, 0, s>>>(L);
        PN_CHECK_LAUNCH();
        DBuf<uint64_t> nd(nseg, s), cap(nseg, s), doff(nseg + 1, s);
        lc_count_k<<<grid_for(nseg, 128), 128, 0, s>>>(L, nd.p, cap.p);
        PN_CHECK_LAUNCH();
        exclusive_scan(ArrayIn<uint64_t>{nd.p}, ArrayOut<uint64_t>{doff.p}, nseg, tot.p, s);
        PN_CUDA(cudaMemcpyAsync(doff.p + nseg, tot.p, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        const uint64_t ndesc = to_host(tot.p, s);
        lc_off.alloc(nseg + 1, s);
        exclusive_scan(ArrayIn<uint64_t>{cap.p}, ArrayOut<uint64_t>{lc_off.p}, nseg, tot.p, s);
        PN_CUDA(cudaMemcpyAsync(lc_off.p + nseg, tot.p, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        const uint64_t ncap = to_host(tot.p, s);
        st.lowcx_ranges = ncap;
        DBuf<LcDesc> desc(ndesc ? ndesc : 1, s);
        lc_desc_k<<<grid_for(nseg, 128), 128, 0, s>>>(L, doff.p, desc.p);
        PN_CHECK_LAUNCH();
        lc_keys.alloc(ncap ? ncap : 1, s);
        lc_vals.alloc(ncap ? ncap : 1, s);
        lcnt.alloc(nseg, s);
        // block path for segments of up to kMedCap ranges, the k-way merge for the rest
        {
            DBuf<uint64_t> gk(ncap ? ncap : 1, s);
            DBuf<uint32_t> wide(nseg, s), rest_list(nseg, s), rest(3, s);  // count, cursor, serial merges
            wide.zero();
            rest.zero();
            lc_gather_k<<<grid_for(nseg * 32, 256, (unsigned)sm_count() * 16), 256, 0, s>>>(L, doff.p, desc.p,
                                                                                          lc_off.p, gk.p, wide.p);
            PN_CHECK_LAUNCH();
            PN_CUDA(cudaFuncSetAttribute(lc_merge_med_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMedSmem));
            int top = 24;  // key bits: lo << 24 with lo < n < 2^(top - 24), so lo never reads all ones
            while (top < 64 && (1ull << (top - 24)) <= n) ++top;
            lc_merge_med_k<<<grid_for(nseg, 1, (unsigned)sm_count()), kMedThreads, kMedSmem, s>>>(
                L, lc_off.p, gk.p, wide.p, top, lc_keys.p, lc_vals.p, lcnt.p, rest_list.p, rest.p);
            PN_CHECK_LAUNCH();
            const uint32_t n_rest = to_host(rest.p, s);
            st.lowcx_rest_segments = n_rest;
            if (n_rest) {
                // largest first, so that the biggest segments do not start last
                DBuf<uint64_t> sk(n_rest, s), sy(n_rest, s), t1(n_rest, s), t2(n_rest, s);
                rest_order_k<<<grid_for(n_rest, 256), 256, 0, s>>>(rest_list.p, n_rest, lc_off.p, sk.p, sy.p);
                PN_CHECK_LAUNCH();
                radix_sort_pairs(sk.p, sy.p, t1.p, t2.p, n_rest, 40, s);
                PN_CUDA(cudaMemsetAsync(rest.p + 1, 0, sizeof(uint32_t), s));
                lc_kmerge_k<<<grid_for((uint64_t)n_rest * 32, kMergeWarps * 32, (unsigned)sm_count() * 32),
                              kMergeWarps * 32, 0, s>>>(L, doff.p, desc.p, lc_off.p, lc_keys.p, lc_vals.p, lcnt.p,
                                                        sy.p, n_rest, rest.p + 1, rest.p + 2);
                PN_CHECK_LAUNCH();
                st.lowcx_serial_segments = to_host(rest.p + 2, s);
            }
        }
        lcpos.alloc(n_reads, s);
        lcpos_k<<<grid_for(nl, 256), 256, 0, s>>>(R->lowcx_list.p, nl, lcpos.p);
        PN_CHECK_LAUNCH();
    }
    st.lowcx_reads = nl;
    ktm.mark_at(5);

    // 3c. candidate compaction in (read, strand, lo) order
    CandCount cc{wcnt.p, nl ? R->lowcx.p : nullptr, lcpos.p, lcnt.p};
    DBuf<uint64_t> coff((uint64_t)n_reads + 1, s);
    exclusive_scan(cc, ArrayOut<uint64_t>{coff.p}, n_reads, tot.p, s);
    uint64_t NC = to_host(tot.p, s);
    R->cand_key.alloc(NC ? NC : 1, s);
    R->cand_hi.alloc(NC ? NC : 1, s);
    compact_k<<<grid_for((uint64_t)n_reads * 32, 256, (unsigned)sm_count() * 16), 256, 0, s>>>(
        n_reads, cc, coff.p, roff.p, wlo.p, whi.p, lc_off.p, lc_keys.p, lc_vals.p, R->cand_key.p, R->cand_hi.p);
    PN_CHECK_LAUNCH();
    wlo.reset();
    whi.reset();
    if (segmented(ref) && NC) {  // cut the ranges at segment edges (order kept)
        const PieceCount pc{R->cand_key.p, R->cand_hi.p, ref->seg.p, ref->n_seg};
        DBuf<uint64_t> poff(NC, s);
        exclusive_scan(pc, ArrayOut<uint64_t>{poff.p}, NC, tot.p, s);
        const uint64_t NP = to_host(tot.p, s);
        DBuf<uint64_t> pkey(NP ? NP : 1, s), phi(NP ? NP : 1, s);
        seg_split_k<<<grid_for(NC, 256, (unsigned)sm_count() * 16), 256, 0, s>>>(pc, NC, poff.p, pkey.p, phi.p);
        PN_CHECK_LAUNCH();
        R->cand_key = std::move(pkey);
        R->cand_hi = std::move(phi);
        NC = NP;
    }
    R->n_cand = NC;
    ktm.mark_at(6);
    st.candidates = NC;
    tm.mark();  // 3

    // 4. verification: q'-gram filter, count + inline pass, offsets (one graph), write pass (one graph)
    DBuf<uint32_t> vcnt(NC ? NC : 1, s);
    DBuf<uint64_t> inl(2 * (NC ? NC : 1), s), toff(NC ? NC : 1, s);
    DBuf<unsigned long long> cols(3, s), fst(3, s);  // fst: filter positions, surviving ranges, columns before
    VerifyParams V{R->cand_key.p, R->cand_hi.p, NC, ref->packed.p, R->len.p, R->kk.p, R->peq.p, vcnt.p, inl.p,
                   cols.p, toff.p, nullptr, nullptr, nullptr, nullptr};
    // the reference's segments ([start, end) pairs), or none when it is one segment [0, n)
    const uint64_t* vseg = segmented(ref) ? ref->seg.p : nullptr;
    const uint32_t vnseg = segmented(ref) ? ref->n_seg : 0u;
    const unsigned gv = grid_for(NC, kVerifyThreads, (unsigned)sm_count() * 32);
    DBuf<uint64_t> okey(NC ? NC : 1, s), order(NC ? NC : 1, s);
    uint64_t NT = 0;
    {
        GraphSegment seg(s, graphs);
        vcnt.zero();  // ranges the filter removes report no tuples
        cols.zero();
        fst.zero();
        PN_CUDA(record_event(kev[10], s));
        PN_CUDA(record_event(kev[11], s));
        if (NC) {
            DBuf<uint64_t> t1(NC, s), t2(NC, s);
            order_key_k<<<grid_for(NC, 256, (unsigned)sm_count() * 16), 256, 0, s>>>(
                R->cand_key.p, R->cand_hi.p, NC, R->len.p, R->kk.p, okey.p, order.p);
            PN_CHECK_LAUNCH();
            radix_sort_pairs(okey.p, order.p, t1.p, t2.p, NC, kOrderBits, s);
            DBuf<uint32_t> qset((uint64_t)n_reads * 16, s);
            DBuf<uint2> qtop((uint64_t)n_reads * 2, s);
            qset_k<<<grid_for((uint64_t)n_reads * 32, 256, (unsigned)sm_count() * 16), 256, 0, s>>>(
                R->codes.p, R->base_off.p, n_reads, qset.p, qtop.p);
            PN_CHECK_LAUNCH();
            PN_CUDA(record_event(kev[10], s));
            qfilter_k<<<grid_for(NC, kFilterThreads, (unsigned)sm_count() * 32), kFilterThreads, 0, s>>>(
                R->cand_key.p, R->cand_hi.p, order.p, NC, ref->packed.p, R->len.p, R->kk.p, qset.p, qtop.p, fst.p);
            PN_CHECK_LAUNCH();
            PN_CUDA(record_event(kev[11], s));
            // verification order over the narrowed ranges; removed ones last
            order_key_k<<<grid_for(NC, 256, (unsigned)sm_count() * 16), 256, 0, s>>>(
                R->cand_key.p, R->cand_hi.p, NC, R->len.p, R->kk.p, okey.p, order.p);
            PN_CHECK_LAUNCH();
            radix_sort_pairs(okey.p, order.p, t1.p, t2.p, NC, kOrderBits, s);
        }
        PN_CUDA(record_event(kev[2], s));
        if (NC) {
            verify_k<false><<<gv, kVerifyThreads, 0, s>>>(V, order.p, fst.p + 1, vseg, vnseg);
            PN_CHECK_LAUNCH();
        }
        PN_CUDA(record_event(kev[3], s));
        exclusive_scan(ArrayIn<uint32_t>{vcnt.p}, ArrayOut<uint64_t>{toff.p}, NC, tot.p, s);
        st.graph_segments += seg.run() ? 1 : 0;
        unsigned long long cv[3], fv[3];
        PN_CUDA(cudaMemcpyAsync(&NT, tot.p, sizeof(NT), cudaMemcpyDeviceToHost, s));
        PN_CUDA(cudaMemcpyAsync(cv, cols.p, sizeof(cv), cudaMemcpyDeviceToHost, s));
        PN_CUDA(cudaMemcpyAsync(fv, fst.p, sizeof(fv), cudaMemcpyDeviceToHost, s));
        PN_CUDA(cudaStreamSynchronize(s));
        st.candidate_columns = cv[0];
        st.candidate_word_columns = cv[1];
        st.useful_columns = cv[2];
        st.filter_positions = fv[0];
        st.filter_live = fv[1];
        st.prefilter_columns = fv[2];
        R->n_live = fv[1];
    }
    okey.reset();
    DeviceHits* out = new DeviceHits();
    try {
        DeviceHits all;
        alloc_hits(&all, NT, s);
        V.out_read = all.h.read_id;
        V.out_strand = all.h.strand;
        V.out_end = all.h.end_pos;
        V.out_dist = all.h.dist;
        GraphSegment seg(s, graphs && NC);
        if (NC) {
            inline_out_k<<<grid_for(NC, 256, (unsigned)sm_count() * 16), 256, 0, s>>>(V);
            PN_CHECK_LAUNCH();
            verify_k<true><<<gv, kVerifyThreads, 0, s>>>(V, order.p, fst.p + 1, vseg, vnseg);
            PN_CHECK_LAUNCH();
        }
        st.graph_segments += seg.run() ? 1 : 0;
        tm.mark();  // 4
        // 5. best stratum
        if (mode == 1 && NT) {
            best_stratum(all.h, n_reads, out, s);
            free_hits_arrays(&all);
        } else {
            out->stream = s;
            out->a = all.a;
            out->h = all.h;
            all.h = peanut_device_hits{};
        }
        tm.mark();  // 5
        PN_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
        free_hits_arrays(out);
        delete out;
        throw;
    }
    st.results = out->h.n;
    st.ms_scan = tm.ms(0, 1);
    st.ms_bin = tm.ms(1, 2);
    st.ms_windows = tm.ms(2, 3);
    st.ms_verify = tm.ms(3, 4);
    st.ms_output = tm.ms(4, 5);
    st.ms_scan_kernel = elapsed(kev[0], kev[1]);
    st.ms_verify_kernel = elapsed(kev[2], kev[3]);
    st.ms_probe_kernel = elapsed(kev[0], kev[7]);
    st.ms_windows_med = elapsed(kev[8], kev[9]);
    st.ms_windows_big = elapsed(kev[9], kev[4]);
    st.ms_windows_sweep = elapsed(tm.ev[2], kev[4]);
    st.ms_lowcx = elapsed(kev[4], kev[5]);
    st.ms_compact = elapsed(kev[5], kev[6]);
    st.ms_filter_kernel = elapsed(kev[10], kev[11]);
    R->stats = st;
    return out;
}

void free_device_hits(DeviceHits* H) {
    free_hits_arrays(H);
}

// ---- test hook: bit-vector columns of explicit (pattern, text) pairs ------------------------

__global__ void bv_columns_k(const uint8_t* pat, const uint64_t* pat_off, uint32_t n_pat, const uint8_t* txt,
                             const uint64_t* txt_off, const uint64_t* peq, int32_t* out) {
    const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n_pat) return;
    const uint32_t m = (uint32_t)(pat_off[x + 1] - pat_off[x]);
    const uint32_t W = (m + 63) >> 6;
    const uint64_t* pq = peq + (uint64_t)x * 2 * 4 * kMaxWords;
    const uint64_t b = txt_off[x], e = txt_off[x + 1];
    auto run = [&](auto M) {
        M.init(pq, m);
        for (uint64_t j = b; j < e; ++j) out[j] = M.step(txt[j]);
    };
    switch (W) {
        case 1: run(Myers<1>{}); break;
        case 2: run(Myers<2>{}); break;
        case 3: run(Myers<3>{}); break;
        default: run(Myers<4>{}); break;
    }
}

__global__ void ascii_codes_k(uint8_t* a, uint64_t n, uint32_t* bad) {
    const uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const uint8_t c = a[x];
    uint8_t v = c == 'A' ? 0 : c == 'C' ? 1 : c == 'G' ? 2 : c == 'T' ? 3 : 255;
    if (v == 255) {
        atomicOr(bad, 1u);
        v = 0;
    }
    a[x] = v;
}

__global__ void pattern_peq_k(const uint8_t* pat, const uint64_t* off, const uint8_t* len, uint32_t n, uint64_t* peq);

void bitvector_columns(const char* pat, const uint64_t* pat_off, uint32_t n_pat, const char* txt,
                       const uint64_t* txt_off, int32_t* out, cudaStream_t s) {
    const uint64_t np = pat_off[n_pat], nt = txt_off[n_pat];
    for (uint32_t i = 0; i < n_pat; ++i) {
        const uint64_t m = pat_off[i + 1] - pat_off[i];
        PN_REQUIRE(m >= 1 && m <= (uint64_t)kMaxReadLen, PEANUT_INVALID_ARG, "pattern length out of range");
        PN_REQUIRE(txt_off[i + 1] >= txt_off[i], PEANUT_INVALID_ARG, "text offsets must ascend");
    }
    DBuf<uint8_t> dp(np ? np : 1, s), dt(nt ? nt : 1, s), lens(n_pat, s);
    DBuf<uint64_t> dpo((uint64_t)n_pat + 1, s), dto((uint64_t)n_pat + 1, s), peq((uint64_t)n_pat * 2 * 4 * kMaxWords, s);
    DBuf<int32_t> dout(nt ? nt : 1, s);
    DBuf<uint32_t> bad(1, s);
    bad.zero();
    PN_CUDA(cudaMemcpyAsync(dp.p, pat, np, cudaMemcpyHostToDevice, s));
    PN_CUDA(cudaMemcpyAsync(dt.p, txt, nt, cudaMemcpyHostToDevice, s));
    PN_CUDA(cudaMemcpyAsync(dpo.p, pat_off, ((uint64_t)n_pat + 1) * 8, cudaMemcpyHostToDevice, s));
    PN_CUDA(cudaMemcpyAsync(dto.p, txt_off, ((uint64_t)n_pat + 1) * 8, cudaMemcpyHostToDevice, s));
    if (np) ascii_codes_k<<<grid_for(np, 256), 256, 0, s>>>(dp.p, np, bad.p);
    if (nt) ascii_codes_k<<<grid_for(nt, 256), 256, 0, s>>>(dt.p, nt, bad.p);
    PN_CHECK_LAUNCH();
    pattern_peq_k<<<grid_for(n_pat, 128), 128, 0, s>>>(dp.p, dpo.p, nullptr, n_pat, peq.p);
    PN_CHECK_LAUNCH();
    bv_columns_k<<<grid_for(n_pat, 64), 64, 0, s>>>(dp.p, dpo.p, n_pat, dt.p, dto.p, peq.p, dout.p);
    PN_CHECK_LAUNCH();
    PN_REQUIRE(to_host(bad.p, s) == 0, PEANUT_INVALID_ARG, "non-ACGT byte");
    PN_CUDA(cudaMemcpyAsync(out, dout.p, nt * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PN_CUDA(cudaStreamSynchronize(s));
}

__global__ void pattern_peq_k(const uint8_t* pat, const uint64_t* off, const uint8_t*, uint32_t n, uint64_t* peq) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const uint32_t m = (uint32_t)(off[r + 1] - off[r]);
    uint64_t w[4][kMaxWords] = {};
    for (uint32_t i = 0; i < m; ++i) w[pat[off[r] + i]][i >> 6] |= 1ull << (i & 63);
    for (int c = 0; c < 4; ++c)
        for (int x = 0; x < kMaxWords; ++x) peq[((uint64_t)r * 2 * 4 + c) * kMaxWords + x] = w[c][x];
}

}  // namespace pn

// ---- bit-vector columns without any allocation ----------------------------------------------
//
// peanut_bitvector_columns_noalloc runs the same Myers kernel as the test hook above, for callers
// that must not allocate device memory.  Its scratch (the match masks of every pattern and one
// status word) lives in this file-scope device array, which every GPU that loads the library
// holds until the process exits.  All calls share it: a call overwrites the masks of the
// patterns it runs and clears the status word first, and two calls whose work overlaps on the
// GPU (different streams, or different host threads) race on it.

namespace pn {

constexpr uint32_t kNoAllocMaxPatterns = 8192;  // 1 MiB of match masks
constexpr size_t kNoAllocPeqWords = (size_t)kNoAllocMaxPatterns * 4 * kMaxWords;
static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocPeqWords + 32];

enum : uint32_t { kNaBadPatLen = 1u, kNaBadBase = 2u, kNaBadTxtOff = 4u };

__device__ __forceinline__ uint32_t na_code(uint8_t ch, uint32_t* status) {
    switch (ch) {
        case 'A': return 0;
        case 'C': return 1;
        case 'G': return 2;
        case 'T': return 3;
        default: atomicOr(status, kNaBadBase); return 0;
    }
}

__global__ void noalloc_peq_k(const uint8_t* __restrict__ pat, const uint64_t* __restrict__ pat_off, uint32_t n,
                              uint64_t* scratch) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    uint32_t* status = reinterpret_cast<uint32_t*>(scratch + kNoAllocPeqWords);
    const uint64_t a = pat_off[r], b = pat_off[r + 1];
    uint64_t w[4][kMaxWords] = {};
    if (b < a || b - a < 1 || b - a > (uint64_t)kMaxReadLen) {
        atomicOr(status, kNaBadPatLen);
    } else {
        for (uint64_t i = 0; i < b - a; ++i) w[na_code(pat[a + i], status)][i >> 6] |= 1ull << (i & 63);
    }
    for (int c = 0; c < 4; ++c)
        for (int x = 0; x < kMaxWords; ++x) scratch[((uint64_t)r * 4 + c) * kMaxWords + x] = w[c][x];
}

__global__ void noalloc_columns_k(const uint64_t* __restrict__ pat_off, uint32_t n, const uint8_t* __restrict__ txt,
                                  const uint64_t* __restrict__ txt_off, int32_t* __restrict__ out,
                                  const uint64_t* scratch) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    uint32_t* status = reinterpret_cast<uint32_t*>(const_cast<uint64_t*>(scratch) + kNoAllocPeqWords);
    const uint64_t a = pat_off[r], b = pat_off[r + 1];
    if (b < a || b - a < 1 || b - a > (uint64_t)kMaxReadLen) return;
    const uint64_t tb = txt_off[r], te = txt_off[r + 1];
    if (te < tb) {
        atomicOr(status, kNaBadTxtOff);
        return;
    }
    const uint32_t m = (uint32_t)(b - a);
    const uint64_t* pq = scratch + (uint64_t)r * 4 * kMaxWords;
    auto run = [&](auto M) {
        M.init(pq, m);
        for (uint64_t j = tb; j < te; ++j) out[j] = M.step(na_code(txt[j], status));
    };
    switch ((m + 63) >> 6) {
        case 1: run(Myers<1>{}); break;
        case 2: run(Myers<2>{}); break;
        case 3: run(Myers<3>{}); break;
        default: run(Myers<4>{}); break;
    }
}

// Device address of the scratch array on the current device, looked up once per device with
// that device current.
static uint64_t* noalloc_scratch() {
    static std::mutex mu;
    static uint64_t* ptrs[256] = {};
    int dev = 0;
    PN_CUDA(cudaGetDevice(&dev));
    PN_REQUIRE(dev >= 0 && dev < 256, PEANUT_UNSUPPORTED, "device ordinal %d", dev);
    std::lock_guard<std::mutex> lock(mu);
    if (!ptrs[dev]) {
        void* p = nullptr;
        PN_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        ptrs[dev] = static_cast<uint64_t*>(p);
    }
    return ptrs[dev];
}

void bitvector_columns_noalloc(const char* d_pat, const uint64_t* d_pat_off, uint32_t n_pat, const char* d_txt,
                               const uint64_t* d_txt_off, int32_t* d_out, cudaStream_t s) {
    PN_REQUIRE(n_pat >= 1 && n_pat <= kNoAllocMaxPatterns, PEANUT_INVALID_ARG,
               "n_pat = %u outside 1..%u (the fixed scratch holds the masks of %u patterns)", n_pat,
               kNoAllocMaxPatterns, kNoAllocMaxPatterns);
    uint64_t* scratch = noalloc_scratch();
    PN_CUDA(cudaMemsetAsync(scratch + kNoAllocPeqWords, 0, sizeof(uint64_t), s));
    noalloc_peq_k<<<grid_for(n_pat, 128), 128, 0, s>>>((const uint8_t*)d_pat, d_pat_off, n_pat, scratch);
    PN_CHECK_LAUNCH();
    noalloc_columns_k<<<grid_for(n_pat, 64), 64, 0, s>>>(d_pat_off, n_pat, (const uint8_t*)d_txt, d_txt_off, d_out,
                                                         scratch);
    PN_CHECK_LAUNCH();
    uint32_t st = 0;
    PN_CUDA(cudaMemcpyAsync(&st, scratch + kNoAllocPeqWords, sizeof(st), cudaMemcpyDeviceToHost, s));
    PN_CUDA(cudaStreamSynchronize(s));
    PN_REQUIRE(!(st & kNaBadPatLen), PEANUT_INVALID_ARG, "a pattern length is outside 1..%d", kMaxReadLen);
    PN_REQUIRE(!(st & kNaBadTxtOff), PEANUT_INVALID_ARG, "text offsets must ascend");
    PN_REQUIRE(!(st & kNaBadBase), PEANUT_INVALID_ARG, "a pattern or text contains a byte other than A/C/G/T");
}

}  // namespace pn
