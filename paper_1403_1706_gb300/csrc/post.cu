// Postprocessing of a batch's hit list on the device: the alignment start of every hit (the
// backward pass of Section "Validation"), its hit-rank and its mapping quality (Section
// "Postprocessing").
//
// Start.  For a hit of pattern P (the read, or its reverse complement for strand 1; length m)
// ending at j with distance d, G[c] = the edit distance between P and the c reference bases ending
// at j.  Reading P and the reference backwards from j turns this into the edit matrix of the
// reversed pattern against the reversed text with the top row E[0][c] = c (the alignment must end
// exactly at j): Myers' recurrence with a horizontal delta of +1 entering at row 0, i.e. Ph
// shifted up with a 1 instead of a 0.  min over c of G[c] is d (the definition of D[j]); the
// start is j - c + 1 for the largest c with G[c] = d (the leftmost start; an alignment of cost d
// spans at most m + d bases, and stays inside the segment of the reference that holds j, so c
// never reaches past that segment's start).
//
// Hit-rank and quality.  R = the number of the read's hits (both strands) whose percent identity
// (m - d') / m is at least the hit's, i.e. d' <= d; quality = min(-10 log10((R - 1) / n), 255)
// for a reference of n positions, 255 when R = 1, the integer part taken after adding 1e-9 (so
// that ratios at exact powers of ten give their integer), clamped at 0.
#include "prims.cuh"

namespace pn {

constexpr int kPostThreads = 128;

// One column of the anchored matrix on W 64-bit words; returns the change of E[m][c].
template <int W>
__device__ __forceinline__ int anchored_step(uint64_t (&Pv)[W], uint64_t (&Mv)[W], const uint64_t (&e)[W],
                                             int lastbit) {
    uint64_t t[W], sum[W], ph[W], mh[W], xv[W];
#pragma unroll
    for (int w = 0; w < W; ++w) t[w] = e[w] & Pv[w];
    uint64_t carry = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {  // sum = t + Pv over W words
        const uint64_t a = t[w] + Pv[w];
        const uint64_t c1 = a < t[w] ? 1ull : 0ull;
        sum[w] = a + carry;
        carry = c1 | (sum[w] < a ? 1ull : 0ull);
    }
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
        const uint64_t p = (ph[w] << 1) | (w ? ph[w - 1] >> 63 : 1ull);  // row 0: E[0][c] - E[0][c-1] = +1
        const uint64_t q = (mh[w] << 1) | (w ? mh[w - 1] >> 63 : 0ull);
        Pv[w] = q | ~(xv[w] | p);
        Mv[w] = p & xv[w];
    }
    return delta;
}

template <int W>
__device__ uint64_t hit_start(const uint64_t* __restrict__ pq, uint32_t m, int64_t sa, int64_t j, int32_t d,
                              const uint32_t* __restrict__ packed, bool* ok) {
    // match masks of the reversed pattern: bit i of rev = bit m - 1 - i of the forward mask
    uint64_t eq[4][W];
    const int sh = 64 * W - (int)m;  // 0..63
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint64_t r[W];
#pragma unroll
        for (int w = 0; w < W; ++w) r[w] = __brevll(__ldg(pq + c * kMaxWords + (W - 1 - w)));
#pragma unroll
        for (int w = 0; w < W; ++w)
            eq[c][w] = sh ? (r[w] >> sh) | (w + 1 < W ? r[w + 1] << (64 - sh) : 0ull) : r[w];
    }
    uint64_t Pv[W], Mv[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        Pv[w] = ~0ull;  // column c = 0: E[i][0] = i
        Mv[w] = 0;
    }
    const int lastbit = (int)((m - 1) & 63);
    int32_t score = (int32_t)m;
    int64_t best = score == d ? 0 : -1;
    const int64_t C = (int64_t)m + d < j + 1 - sa ? (int64_t)m + d : j + 1 - sa;
    for (int64_t c = 1; c <= C; ++c) {
        const int64_t t = j - c + 1;
        const uint32_t b = (__ldg(packed + (t >> 4)) >> (30 - 2 * (uint32_t)(t & 15))) & 3u;
        uint64_t e[W];
#pragma unroll
        for (int w = 0; w < W; ++w) e[w] = b == 0 ? eq[0][w] : b == 1 ? eq[1][w] : b == 2 ? eq[2][w] : eq[3][w];
        score += anchored_step<W>(Pv, Mv, e, lastbit);
        if (score == d) best = c;
        if (score < d) *ok = false;  // d is not the minimum: not a hit of this pattern
    }
    if (best < 0) *ok = false;
    return best < 0 ? ~0ull : (uint64_t)(j - best + 1);
}

__global__ void __launch_bounds__(kPostThreads)
    start_k(peanut_device_hits H, const uint8_t* __restrict__ len, const uint64_t* __restrict__ peq,
            const uint32_t* __restrict__ packed, uint64_t n_ref, const uint64_t* __restrict__ seg, uint32_t n_seg,
            uint32_t n_reads, uint64_t* __restrict__ start, uint32_t* status) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < H.n; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = H.read_id[x], s = H.strand[x];
        const uint64_t j = H.end_pos[x];
        if (r >= n_reads || s > 1 || j >= n_ref) {
            atomicOr(status, 1u);
            start[x] = ~0ull;
            continue;
        }
        // the segment holding j: the first one ending after j
        uint32_t l = 0, h = n_seg;
        while (l < h) {
            const uint32_t mid = (l + h) >> 1;
            if (seg[2 * mid + 1] <= j)
                l = mid + 1;
            else
                h = mid;
        }
        if (l == n_seg || seg[2 * l] > j) {  // an end in a gap
            atomicOr(status, 1u);
            start[x] = ~0ull;
            continue;
        }
        const int64_t sa = (int64_t)seg[2 * l];
        const uint32_t m = len[r];
        const uint64_t* pq = peq + ((uint64_t)r * 2 + s) * 4 * kMaxWords;
        bool ok = true;
        uint64_t st = 0;
        switch ((m + 63) >> 6) {
            case 1: st = hit_start<1>(pq, m, sa, (int64_t)j, H.dist[x], packed, &ok); break;
            case 2: st = hit_start<2>(pq, m, sa, (int64_t)j, H.dist[x], packed, &ok); break;
            case 3: st = hit_start<3>(pq, m, sa, (int64_t)j, H.dist[x], packed, &ok); break;
            default: st = hit_start<4>(pq, m, sa, (int64_t)j, H.dist[x], packed, &ok); break;
        }
        if (!ok) atomicOr(status, 2u);
        start[x] = st;
    }
}

// Hits grouped by read (ascending): the half-open range of each read's hits.
__global__ void read_ranges_k(const uint32_t* __restrict__ rd, uint64_t n, uint64_t* rb, uint64_t* re,
                              uint32_t* status) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = rd[x];
        if (x > 0 && rd[x - 1] > r) atomicOr(status, 4u);
        if (x == 0 || rd[x - 1] != r) rb[r] = x;
        if (x + 1 == n || rd[x + 1] != r) re[r] = x + 1;
    }
}

// One warp per read: a histogram of its hits' distances, its prefix sums, then every hit's rank
// and quality.
__global__ void __launch_bounds__(kPostThreads)
    rank_k(const uint8_t* __restrict__ dist, const uint64_t* __restrict__ rb, const uint64_t* __restrict__ re,
           uint32_t n_reads, double n_ref, uint32_t* __restrict__ rank, uint8_t* __restrict__ mapq) {
    __shared__ uint32_t hist[kPostThreads / 32][64];
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    uint32_t* h = hist[wid];
    for (uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_reads; r += nw) {
        const uint64_t a = rb[r], b = re[r];
        if (b <= a) continue;
        h[lane] = 0;
        h[lane + 32] = 0;
        __syncwarp();
        for (uint64_t x = a + lane; x < b; x += 32) atomicAdd(&h[dist[x] & 63], 1u);
        __syncwarp();
        // inclusive prefix over the 64 bins (two per lane)
        const uint32_t v0 = h[2 * lane], v1 = h[2 * lane + 1];
        uint32_t incl = v0 + v1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= (uint32_t)o) incl += t;
        }
        __syncwarp();
        h[2 * lane] = incl - v1;
        h[2 * lane + 1] = incl;
        __syncwarp();
        for (uint64_t x = a + lane; x < b; x += 32) {
            const uint32_t R = h[dist[x] & 63];
            rank[x] = R;
            uint8_t q = 255;
            if (R > 1) {
                const double v = floor(-10.0 * log10((double)(R - 1) / n_ref) + 1e-9);
                q = (uint8_t)(v < 0.0 ? 0.0 : v > 255.0 ? 255.0 : v);
            }
            mapq[x] = q;
        }
        __syncwarp();
    }
}

void annotate_hits(const peanut_ref* ref, const peanut_reads* R, const peanut_device_hits& H, uint64_t* d_start,
                   uint32_t* d_rank, uint8_t* d_mapq) {
    cudaStream_t s = R->stream;
    const uint64_t n = H.n;
    if (!n) return;
    DBuf<uint32_t> status(1, s);
    status.zero();
    start_k<<<grid_for(n, kPostThreads, (unsigned)sm_count() * 16), kPostThreads, 0, s>>>(
        H, R->len.p, R->peq.p, ref->packed.p, ref->n, ref->seg.p, ref->n_seg, R->n_reads, d_start, status.p);
    PN_CHECK_LAUNCH();
    // read ids index rb / re below: refuse the list before that if any is out of range
    PN_REQUIRE(!(to_host(status.p, s) & 1u), PEANUT_INVALID_ARG,
               "a hit names a read, strand or end outside the batch / reference, or an end in a gap");
    DBuf<uint64_t> rb(R->n_reads, s), re(R->n_reads, s);
    rb.zero();
    re.zero();
    read_ranges_k<<<grid_for(n, 256, (unsigned)sm_count() * 16), 256, 0, s>>>(H.read_id, n, rb.p, re.p, status.p);
    PN_CHECK_LAUNCH();
    rank_k<<<grid_for((uint64_t)R->n_reads * 32, kPostThreads, (unsigned)sm_count() * 16), kPostThreads, 0, s>>>(
        H.dist, rb.p, re.p, R->n_reads, (double)ref->n, d_rank, d_mapq);
    PN_CHECK_LAUNCH();
    const uint32_t st = to_host(status.p, s);
    PN_REQUIRE(!(st & 1u), PEANUT_INVALID_ARG, "a hit names a read, strand or end outside the batch / reference");
    PN_REQUIRE(!(st & 2u), PEANUT_INVALID_ARG, "a hit's distance is not the pattern's distance at its end");
    PN_REQUIRE(!(st & 4u), PEANUT_INVALID_ARG, "hits are not grouped by ascending read");
}

}  // namespace pn
