// Device-wide parallel primitives: exclusive prefix sum and LSD radix sort.
//
// Section "GPU architecture" of the paper builds every cumulative sum and stream compaction on
// parallel prefix scans (Blelloch 1990).  These are this library's own: a three-phase scan
// (tile reduce, scan of tile sums, tile scan with offset) using warp shuffles, and a stable
// 8-bit-digit LSD radix sort whose per-tile ranking uses warp match masks.
#pragma once

#include "internal.cuh"

namespace pn {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
struct ArrayIn {
    const T* a;
    __device__ __forceinline__ uint64_t operator()(uint64_t i) const { return (uint64_t)a[i]; }
};

template <class T>
struct ArrayOut {
    T* a;
    __device__ __forceinline__ void operator()(uint64_t i, uint64_t v) const { a[i] = (T)v; }
};

// Exclusive sum over the block of one value per thread; *total receives the block total.
__device__ __forceinline__ uint64_t block_exclusive_sum(uint64_t v, uint64_t* total) {
    __shared__ uint64_t ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint64_t w = lane < nw ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        ws[lane] = w;
    }
    __syncthreads();
    const uint64_t before = wid ? ws[wid - 1] : 0;
    *total = ws[nw - 1];
    __syncthreads();
    return before + x - v;
}

template <class In>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_k(In in, uint64_t n, uint64_t* partial) {
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    uint64_t s = 0;
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
        uint64_t i = base + (uint64_t)it * kScanThreads + threadIdx.x;
        if (i < n) s += in(i);
    }
    uint64_t tot;
    block_exclusive_sum(s, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <class In, class Out>
__global__ void __launch_bounds__(kScanThreads)
    scan_down_k(In in, Out out, uint64_t n, const uint64_t* offs, uint64_t* total) {
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    uint64_t v[kScanItems];
    uint64_t s = 0;
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
        uint64_t i = base + it;
        v[it] = i < n ? in(i) : 0;
        s += v[it];
    }
    uint64_t tot;
    uint64_t run = block_exclusive_sum(s, &tot) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int it = 0; it < kScanItems; ++it) {
        uint64_t i = base + it;
        if (i < n) out(i, run);
        run += v[it];
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
        *total = (offs ? offs[blockIdx.x] : 0) + tot;
}

// out(i, sum_{j < i} in(j)) for i < n; *d_total (device, optional) = sum of all.
template <class In, class Out>
void exclusive_scan(In in, Out out, uint64_t n, uint64_t* d_total, cudaStream_t s) {
    if (n == 0) {
        if (d_total) PN_CUDA(cudaMemsetAsync(d_total, 0, sizeof(uint64_t), s));
        return;
    }
    const uint64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        scan_down_k<<<1, kScanThreads, 0, s>>>(in, out, n, (const uint64_t*)nullptr, d_total);
        PN_CHECK_LAUNCH();
        return;
    }
    DBuf<uint64_t> partial(nb, s), pscan(nb, s);
    scan_reduce_k<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, partial.p);
    PN_CHECK_LAUNCH();
    exclusive_scan(ArrayIn<uint64_t>{partial.p}, ArrayOut<uint64_t>{pscan.p}, nb, nullptr, s);
    scan_down_k<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, pscan.p, d_total);
    PN_CHECK_LAUNCH();
}

// ---- LSD radix sort of uint64 keys --------------------------------------------------------

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;

static __global__ void __launch_bounds__(kSortThreads)
    radix_hist_k(const uint64_t* keys, uint64_t n, int shift, uint32_t* hist, uint32_t nb) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int it = 0; it < kSortItems; ++it) {
        uint64_t i = base + (uint64_t)it * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(uint64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

template <bool kVals>
__global__ void __launch_bounds__(kSortThreads)
    radix_scatter_k(const uint64_t* in, uint64_t* out, const uint64_t* vin, uint64_t* vout, uint64_t n,
                    int shift, const uint32_t* offs, uint32_t nb) {
    __shared__ uint32_t cnt[kSortThreads / 32][256];
    __shared__ uint32_t running[256];
    __shared__ uint32_t basev[256];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    running[threadIdx.x] = offs[(uint64_t)threadIdx.x * nb + blockIdx.x];
    const uint64_t base = (uint64_t)blockIdx.x * kSortTile;
    const unsigned lt = (1u << lane) - 1u;
    for (int it = 0; it < kSortItems; ++it) {
        const uint64_t i = base + (uint64_t)it * kSortThreads + threadIdx.x;
        const bool valid = i < n;
        const uint64_t key = valid ? in[i] : 0;
        const unsigned digit = valid ? (unsigned)((key >> shift) & 255u) : 256u;
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; ++w) cnt[w][threadIdx.x] = 0;
        __syncthreads();
        const unsigned peers = __match_any_sync(kFull, digit);
        const unsigned rank = __popc(peers & lt);
        if (valid && rank == 0) cnt[wid][digit] = __popc(peers);
        __syncthreads();
        {
            uint32_t acc = 0;
#pragma unroll
            for (int w = 0; w < kSortThreads / 32; ++w) {
                uint32_t c = cnt[w][threadIdx.x];
                cnt[w][threadIdx.x] = acc;
                acc += c;
            }
            basev[threadIdx.x] = running[threadIdx.x];
            running[threadIdx.x] += acc;
        }
        __syncthreads();
        if (valid) {
            const uint32_t dst = basev[digit] + cnt[wid][digit] + rank;
            out[dst] = key;
            if (kVals) vout[dst] = vin[i];
        }
        __syncthreads();
    }
}

// Stable sort of keys[0..n) ascending by bits [0, bits), carrying vals (may be null) along.
// tmp / vtmp hold n entries each.  n < 2^32.
inline void radix_sort_pairs(uint64_t* keys, uint64_t* vals, uint64_t* tmp, uint64_t* vtmp, uint64_t n, int bits,
                             cudaStream_t s) {
    if (n <= 1 || bits <= 0) return;
    PN_REQUIRE(n < (1ull << 32), PEANUT_UNSUPPORTED,
               "radix sort of %llu keys (2^32 at most): too many q-gram hits in one batch; map fewer reads "
               "per batch or use a larger q", (unsigned long long)n);
    const uint32_t nb = (uint32_t)((n + kSortTile - 1) / kSortTile);
    DBuf<uint32_t> hist((uint64_t)256 * nb, s), offs((uint64_t)256 * nb, s);
    uint64_t *a = keys, *b = tmp, *va = vals, *vb = vtmp;
    for (int shift = 0; shift < bits; shift += 8) {
        radix_hist_k<<<nb, kSortThreads, 0, s>>>(a, n, shift, hist.p, nb);
        PN_CHECK_LAUNCH();
        exclusive_scan(ArrayIn<uint32_t>{hist.p}, ArrayOut<uint32_t>{offs.p}, (uint64_t)256 * nb, nullptr, s);
        if (vals)
            radix_scatter_k<true><<<nb, kSortThreads, 0, s>>>(a, b, va, vb, n, shift, offs.p, nb);
        else
            radix_scatter_k<false><<<nb, kSortThreads, 0, s>>>(a, b, nullptr, nullptr, n, shift, offs.p, nb);
        PN_CHECK_LAUNCH();
        uint64_t* t = a;
        a = b;
        b = t;
        t = va;
        va = vb;
        vb = t;
    }
    if (a != keys) {
        PN_CUDA(cudaMemcpyAsync(keys, a, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        if (vals) PN_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    }
}

inline void radix_sort_u64(uint64_t* keys, uint64_t* tmp, uint64_t n, int bits, cudaStream_t s) {
    radix_sort_pairs(keys, nullptr, tmp, nullptr, n, bits, s);
}

// ---- small helpers ----------------------------------------------------------------------

__device__ __forceinline__ unsigned lanemask_lt() {
    return (1u << (threadIdx.x & 31)) - 1u;
}

// The 32-code group of canonical code c as (I word, S: the number of distinct codes before the
// group) for any layout of the batch's q-group index: interleaved; I per 32 codes with S kept for
// the even groups only (an odd group adds the population count of the even one before it, the
// sampling of S of Section "The q-group index"); or I per 64 codes (w = 64) with S per 64 codes.
template <int L>
__device__ __forceinline__ uint2 index_group(const IndexView& V, uint32_t c) {
    if constexpr (L == 0) {
        return V.IS[c >> 5];
    } else if constexpr (L == 1) {
        const uint32_t g = c >> 5;
        const uint2 pair = *reinterpret_cast<const uint2*>(V.I32 + (g & ~1u));
        const uint32_t base = V.S2[g >> 1];
        return (g & 1u) ? make_uint2(pair.y, base + __popc(pair.x)) : make_uint2(pair.x, base);
    } else {
        const unsigned long long w = V.I64[c >> 6];
        const uint32_t base = V.S64[c >> 6];
        return (c & 32u) ? make_uint2((uint32_t)(w >> 32), base + __popc((uint32_t)w)) : make_uint2((uint32_t)w, base);
    }
}

// 2-bit base code at position p of the packed reference (first base most significant).
__device__ __forceinline__ uint32_t ref_base(const uint32_t* packed, uint64_t p) {
    return (packed[p >> 4] >> (30 - 2 * (uint32_t)(p & 15))) & 3u;
}

// Reverse complement of a q-gram code (complement = 3 - c, then reverse the 2-bit groups).
__device__ __forceinline__ uint32_t revcomp_code(uint32_t g, uint32_t q) {
    uint32_t x = ~g;
    x = __brev(x);
    x = ((x >> 1) & 0x55555555u) | ((x & 0x55555555u) << 1);
    return q == 16 ? x : (x >> (32 - 2 * q)) & ((1u << (2 * q)) - 1u);
}

// Blocked Bloom filter over canonical q-gram codes: one 64-bit word per key, two bits in each of
// its 32-bit halves.  All 32-bit arithmetic: the code is mixed by the "lowbias32" multiply /
// xor-shift sequence (C. Wellons' hash search); the high bits of the mix pick the word (its
// product with the number of words, high half), and the top 20 bits of one more odd multiple of
// the mix pick the four bit positions.  Keys that share a word differ in the low bits of the mix,
// which reach every top bit of the multiple, so their bit positions are independent of the word.
struct BloomKey {
    uint32_t word;    // word index, < the number of words
    uint32_t lo, hi;  // the key's bits in the low and high half of the word
};

__device__ __forceinline__ BloomKey bloom_key(uint32_t c, uint32_t words) {
    uint32_t h = c;
    h ^= h >> 16;
    h *= 0x7FEB352Du;
    h ^= h >> 15;
    h *= 0x846CA68Bu;
    h ^= h >> 16;
    const uint32_t g = h * 0x9E3779B1u;
    BloomKey k;
    k.word = __umulhi(h, words);
    k.lo = (1u << (g >> 27)) | (1u << ((g >> 22) & 31u));
    k.hi = (1u << ((g >> 17) & 31u)) | (1u << ((g >> 12) & 31u));
    return k;
}

}  // namespace pn
