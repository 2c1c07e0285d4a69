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
#include <algorithm>

namespace pn {

constexpr int kPostThreads = 128;

// The quality of rank R for a reference of n positions: the integer part of
// -10 log10((R - 1) / n) + 1e-9, clamped to 0..255, and 255 for R <= 1.  It is first taken in single
// precision from l10n = 10 log10(n): log10f's error (2 ulp) and the roundings keep that value
// within 1e-4 of the exact one, so when it lies more than 1e-3 from an integer its integer part is
// the exact one; otherwise the double-precision expression decides.  (GB300's FP64 rate is a
// small fraction of its FP32 rate, so a double log10 per hit would bound the ranking kernels.)
__device__ __forceinline__ uint8_t hit_quality(uint32_t R, double n_ref, float l10n) {
    if (R <= 1) return 255;
    const float vf = l10n - 10.0f * log10f((float)(R - 1));
    const float fl = floorf(vf), fr = vf - fl;
    float v = fl;
    if (!(fr > 1e-3f && fr < 1.0f - 1e-3f)) v = (float)floor(-10.0 * log10((double)(R - 1) / n_ref) + 1e-9);
    return (uint8_t)(v < 0.0f ? 0.0f : v > 255.0f ? 255.0f : v);
}

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

// The same start for a hit of distance d <= 7, on the 2d + 1 diagonals |c - i| <= d of the reversed
// pattern (rows i) against the reference read leftwards from j (columns c): every path of cost <= d
// to E(m, c), c in [m - d, m + d] (the only columns that can score d), stays in them.  Cell k of
// column c is row c - d + k, held as a 2-bit field of one word (the lower bit the cell's flag, the
// upper bit a spacer through which the carry below crosses into the next cell).  Cells above row 0 take
// the virtual value c - i (as row 0 takes c), which satisfies the recurrence whatever the bases.
// Per column, the cells that exceed their diagonal neighbour (D) are those whose bases differ while
// neither the left neighbour nor the cell above is below that neighbour; "the cell above is not
// below" chains down the column, Z(k) = G(k) | (P(k) & Z(k - 1)) for Z = not D, and one addition
// gives all of it: Z is the carry vector of (G | P) + G.  The column's vertical differences (UP,
// UN: +1, -1) follow from the previous column's and D; row m's value from the top cell's (tracked)
// and the differences above row m.
__device__ uint64_t hit_start_band(const uint8_t* __restrict__ rd, uint32_t s, int32_t m, int64_t sa, int64_t j,
                                   int32_t d, const uint32_t* __restrict__ packed, bool* ok) {
    const int32_t W = 2 * d + 1;
    const uint32_t E = 0x55555555u & ((1u << (2 * W)) - 1u), ODD = E << 1;
    const uint32_t upper = E & ~((1u << (2 * (d + 1))) - 1u);
    uint32_t UP = upper, UN = E & ~upper & ~1u;  // column 0: E(i, 0) = |i|
    int32_t v0 = d;                               // the top cell's value
    // row i's base of the reversed pattern (any base outside 1..m)
    auto base = [&](int32_t i) -> uint32_t {
        if (i < 1 || i > m) return 0u;
        return s == 0 ? rd[m - i] : 3u - rd[i - 1];
    };
    uint32_t pw = 0;  // the band's pattern bases, cell k at bits 2k
    for (int32_t r = 1; r <= d && r <= m; ++r) pw |= base(r) << (2 * (r + d));
    const int64_t C = (int64_t)m + d < j + 1 - sa ? (int64_t)m + d : j + 1 - sa;
    int64_t best = m == d ? 0 : -1;
    // the text base of column c sits at position p = j - c + 1: the packed word holding p and the
    // one before it (loaded 16 columns ahead)
    int64_t p = j;
    uint64_t wq = (uint64_t)p >> 4;
    uint32_t wc = __ldg(packed + wq), wn = wq ? __ldg(packed + wq - 1) : 0u;
    uint32_t b_next = base(1 + d);
    for (int64_t c = 1; c <= C; ++c) {
        pw = (pw >> 2) | (b_next << (2 * (W - 1)));
        b_next = base((int32_t)c + 1 + d);
        const uint32_t t = (wc >> (30 - 2 * (uint32_t)(p & 15))) & 3u;
        if ((p & 15) == 0 && wq > 0) {  // position 0 ends the loop: no word before it is read
            wc = wn;
            --wq;
            wn = wq ? __ldg(packed + wq - 1) : 0u;
        }
        --p;
        const uint32_t x = pw ^ (t * 0x55555555u);
        const uint32_t mis = (x | (x >> 1)) & E;
        const uint32_t G = (~mis & E) | ((UN >> 2) & E);
        const uint32_t X = G | UP | ODD;
        const uint32_t Z = (((X + G) ^ X ^ G) >> 2) & E;
        const uint32_t D = ~Z & E;
        const uint32_t D1 = (D << 2) & E;  // D of the cell above, at each cell
        const uint32_t same = ~(D ^ D1) & E, U0 = ~(UP | UN) & E;
        const uint32_t up = ((UP & same) | (U0 & D & ~D1)) & E & ~1u;
        UN = ((UN & same) | (U0 & ~D & D1)) & E & ~1u;
        UP = up;
        v0 += (int32_t)(D & 1u);
        const int32_t k = m - (int32_t)c + d;  // row m's cell
        if ((uint32_t)k < (uint32_t)W) {
            const uint32_t low = ((1u << (2 * k + 1)) - 1u) & E;
            const int32_t val = v0 + __popc(UP & low) - __popc(UN & low);
            if (val == d) best = c;
            if (val < d) *ok = false;  // d is not the minimum: not a hit of this pattern
        }
    }
    if (best < 0) *ok = false;
    return best < 0 ? ~0ull : (uint64_t)(j - best + 1);
}

// kBand: the hits of distance <= 7 (the band above); otherwise the others (Myers' columns), so that
// the common case keeps the band's register count.
template <bool kBand>
__global__ void __launch_bounds__(kPostThreads)
    start_k(peanut_device_hits H, const uint8_t* __restrict__ len, const uint64_t* __restrict__ peq,
            const uint8_t* __restrict__ codes, const uint64_t* __restrict__ base_off,
            const uint32_t* __restrict__ packed, uint64_t n_ref, const uint64_t* __restrict__ seg, uint32_t n_seg,
            uint32_t n_reads, uint64_t* __restrict__ start, uint32_t* status) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < H.n; x += (uint64_t)gridDim.x * blockDim.x) {
        const int32_t d = H.dist[x];
        if (kBand != (d <= 7)) continue;
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
        if (kBand) {
            st = hit_start_band(codes + base_off[r], s, (int32_t)m, sa, (int64_t)j, d, packed, &ok);
        } else switch ((m + 63) >> 6) {
            case 1: st = hit_start<1>(pq, m, sa, (int64_t)j, d, packed, &ok); break;
            case 2: st = hit_start<2>(pq, m, sa, (int64_t)j, d, packed, &ok); break;
            case 3: st = hit_start<3>(pq, m, sa, (int64_t)j, d, packed, &ok); break;
            default: st = hit_start<4>(pq, m, sa, (int64_t)j, d, packed, &ok); break;
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
           uint32_t n_reads, double n_ref, float l10n, uint32_t* __restrict__ rank, uint8_t* __restrict__ mapq) {
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
            mapq[x] = hit_quality(R, n_ref, l10n);
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
    // every hit goes to exactly one instance; the second reads only the distances when none is 8
    // or more
    start_k<true><<<grid_for(n, kPostThreads, (unsigned)sm_count() * 16), kPostThreads, 0, s>>>(
        H, R->len.p, R->peq.p, R->codes.p, R->base_off.p, ref->packed.p, ref->n, ref->seg.p, ref->n_seg, R->n_reads,
        d_start, status.p);
    PN_CHECK_LAUNCH();
    start_k<false><<<grid_for(n, kPostThreads, (unsigned)sm_count() * 16), kPostThreads, 0, s>>>(
        H, R->len.p, R->peq.p, R->codes.p, R->base_off.p, ref->packed.p, ref->n, ref->seg.p, ref->n_seg, R->n_reads,
        d_start, status.p);
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
        H.dist, rb.p, re.p, R->n_reads, (double)ref->n, (float)(10.0 * log10((double)ref->n)), d_rank, d_mapq);
    PN_CHECK_LAUNCH();
    const uint32_t st = to_host(status.p, s);
    PN_REQUIRE(!(st & 1u), PEANUT_INVALID_ARG, "a hit names a read, strand or end outside the batch / reference");
    PN_REQUIRE(!(st & 2u), PEANUT_INVALID_ARG, "a hit's distance is not the pattern's distance at its end");
    PN_REQUIRE(!(st & 4u), PEANUT_INVALID_ARG, "hits are not grouped by ascending read");
}

// ---- paired-end mates (Section "Postprocessing") ------------------------------------------
//
// In paired-end mode the paper pairs mates and sums the percent identities of properly paired
// hits when it forms strata.  Here reads 2p and 2p + 1 of a batch are the mates of fragment p,
// read from its two ends (forward-reverse).  Hits u of mate 1 and x of mate 2 are properly paired
// when they lie on opposite strands, in the same contig, and the fragment from the strand-0 hit's
// start to the strand-1 hit's end is min_insert .. max_insert bases long.  A pair's score is the
// numerator (m1 - d1) m2 + (m2 - d2) m1 of its summed identity over the fragment's common
// denominator m1 m2 (exact comparison); its rank is the number of the fragment's pairs scoring at
// least as high, its quality the hit quality formula with that rank.  Best-stratum mode keeps
// each fragment's top-scoring pairs.  Pairs are listed in (mate-1 hit, mate-2 hit) order.

constexpr int kScoreBits = 17;  // scores < 2 * 255 * 255 < 2^17

struct PairIn {
    peanut_device_hits H;
    const uint64_t* start;
    const uint64_t* rb;  // per read: its hits [rb, re)
    const uint64_t* re;
    const uint8_t* len;
    const uint8_t* kk;
    const uint64_t* contig;  // contig starts, ascending, the first 0
    uint32_t n_contig;
    uint32_t n_reads;
    int64_t min_ins, max_ins;
};

// Index of the contig holding position p.
__device__ __forceinline__ uint32_t contig_index(const uint64_t* __restrict__ cs, uint32_t nc, uint64_t p) {
    uint32_t l = 0, h = nc;
    while (h - l > 1) {
        const uint32_t mid = (l + h) >> 1;
        if (cs[mid] <= p)
            l = mid;
        else
            h = mid;
    }
    return l;
}

// The proper pairs of mate-1 hit u (none for a mate-2 hit): counted, or written from slot o on.
template <bool kWrite>
__device__ uint32_t pairs_of(const PairIn& P, uint64_t u, uint64_t o, uint64_t* o1, uint64_t* o2, uint32_t* osc) {
    const uint32_t r = P.H.read_id[u];
    if ((r & 1u) || r + 1 >= P.n_reads) return 0;
    const uint64_t a = P.rb[r + 1], b = P.re[r + 1];
    if (b <= a) return 0;
    const uint32_t su = P.H.strand[u];
    // mate 2's hits: its strand-0 hits, then its strand-1 hits, each by end
    uint64_t l = a, h = b;
    while (l < h) {
        const uint64_t mid = (l + h) >> 1;
        if (P.H.strand[mid] < 1)
            l = mid + 1;
        else
            h = mid;
    }
    const uint64_t va = su ? a : l, vb = su ? l : b;
    const int64_t m1 = P.len[r], m2 = P.len[r + 1], k2 = P.kk[r + 1];
    const int64_t eu = (int64_t)P.H.end_pos[u], stu = (int64_t)P.start[u];
    // ends that can close a fragment of allowed length: u forward, the mate's end lies in
    // [start + min - 1, start + max - 1]; u reverse, the mate's start lies in
    // [end - max + 1, end - min + 1] and its end at most m2 + k2 - 1 after its start
    const int64_t lo_end = su == 0 ? stu + P.min_ins - 1 : eu - P.max_ins + 1;
    const int64_t hi_end = su == 0 ? stu + P.max_ins - 1 : eu - P.min_ins + m2 + k2;
    l = va;
    h = vb;
    while (l < h) {
        const uint64_t mid = (l + h) >> 1;
        if ((int64_t)P.H.end_pos[mid] < lo_end)
            l = mid + 1;
        else
            h = mid;
    }
    const uint32_t cu = contig_index(P.contig, P.n_contig, (uint64_t)eu);
    const int64_t d1 = P.H.dist[u];
    uint32_t c = 0;
    for (uint64_t x = l; x < vb && (int64_t)P.H.end_pos[x] <= hi_end; ++x) {
        const int64_t ev = (int64_t)P.H.end_pos[x];
        const int64_t ins = su == 0 ? ev - stu + 1 : eu - (int64_t)P.start[x] + 1;
        if (ins < P.min_ins || ins > P.max_ins) continue;
        if (contig_index(P.contig, P.n_contig, (uint64_t)ev) != cu) continue;
        if (kWrite) {
            o1[o + c] = u;
            o2[o + c] = x;
            osc[o + c] = (uint32_t)((m1 - d1) * m2 + (m2 - (int64_t)P.H.dist[x]) * m1);
        }
        ++c;
    }
    return c;
}

struct PairCount {
    PairIn P;
    __device__ uint64_t operator()(uint64_t u) const { return pairs_of<false>(P, u, 0, nullptr, nullptr, nullptr); }
};

__global__ void pair_write_k(PairIn P, const uint64_t* __restrict__ off, uint64_t* o1, uint64_t* o2, uint32_t* osc) {
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < P.H.n; u += (uint64_t)gridDim.x * blockDim.x)
        (void)pairs_of<true>(P, u, off[u], o1, o2, osc);
}

// The hit list must be grouped by read, each read's hits in (strand, end) order, every start at
// or before its end (status bit 8 otherwise).
__global__ void pair_check_k(peanut_device_hits H, const uint64_t* __restrict__ start, uint32_t* status) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < H.n; x += (uint64_t)gridDim.x * blockDim.x) {
        bool bad = start[x] > H.end_pos[x];
        if (x > 0 && H.read_id[x - 1] == H.read_id[x])
            bad |= !(H.strand[x - 1] < H.strand[x] || (H.strand[x - 1] == H.strand[x] && H.end_pos[x - 1] < H.end_pos[x]));
        if (bad) atomicOr(status, 8u);
    }
}

// Sort keys: fragment, then score descending.
__global__ void pair_keys_k(const uint32_t* __restrict__ read_id, const uint64_t* __restrict__ i1,
                            const uint32_t* __restrict__ score, uint64_t n, uint64_t* key, uint64_t* val) {
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
        key[t] = ((uint64_t)(read_id[i1[t]] >> 1) << kScoreBits) | (uint64_t)((1u << kScoreBits) - 1u - score[t]);
        val[t] = t;
    }
}

// Over the sorted keys: rank = pairs of the fragment up to the last one of equal score; keep =
// the pair has the fragment's best score.
__global__ void pair_rank_k(const uint64_t* __restrict__ key, const uint64_t* __restrict__ val, uint64_t n,
                            double n_ref, float l10n, uint32_t* rank, uint8_t* mapq, uint8_t* keep) {
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t k = key[t], f = k >> kScoreBits << kScoreBits;
        uint64_t l = 0, h = t;  // first key of the fragment
        while (l < h) {
            const uint64_t mid = (l + h) >> 1;
            if (key[mid] < f)
                l = mid + 1;
            else
                h = mid;
        }
        const uint64_t f0 = l;
        l = t + 1;
        h = n;  // one past the last equal key
        while (l < h) {
            const uint64_t mid = (l + h) >> 1;
            if (key[mid] <= k)
                l = mid + 1;
            else
                h = mid;
        }
        const uint32_t R = (uint32_t)(l - f0);
        const uint64_t x = val[t];
        rank[x] = R;
        mapq[x] = hit_quality(R, n_ref, l10n);
        keep[x] = key[f0] == k;
    }
}

struct PairOut {
    uint64_t *i1, *i2;
    uint32_t *score, *rank;
    uint8_t* mapq;
};

__global__ void pair_keep_k(PairOut in, const uint8_t* __restrict__ keep, const uint64_t* __restrict__ off, uint64_t n,
                            PairOut out) {
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
        if (!keep[t]) continue;
        const uint64_t o = off[t];
        out.i1[o] = in.i1[t];
        out.i2[o] = in.i2[t];
        out.score[o] = in.score[t];
        out.rank[o] = in.rank[t];
        out.mapq[o] = in.mapq[t];
    }
}

DevicePairs* pair_hits(const peanut_ref* ref, const peanut_reads* R, const peanut_device_hits& H, const uint64_t* d_start,
                       uint32_t min_insert, uint32_t max_insert, int mode) {
    cudaStream_t s = R->stream;
    PN_REQUIRE(R->n_reads % 2 == 0, PEANUT_INVALID_ARG, "a paired batch holds an even number of reads (%u)",
               R->n_reads);
    PN_REQUIRE(min_insert >= 1 && max_insert >= min_insert, PEANUT_INVALID_ARG, "insert range %u..%u", min_insert,
               max_insert);
    std::unique_ptr<DevicePairs> out(new DevicePairs());
    out->stream = s;
    const uint64_t n = H.n;
    const unsigned g = grid_for(n, 256, (unsigned)sm_count() * 16);
    DBuf<uint32_t> status(1, s);
    status.zero();
    DBuf<uint64_t> rb(R->n_reads, s), re(R->n_reads, s);
    rb.zero();
    re.zero();
    if (n) {
        read_ranges_k<<<g, 256, 0, s>>>(H.read_id, n, rb.p, re.p, status.p);
        PN_CHECK_LAUNCH();
        pair_check_k<<<g, 256, 0, s>>>(H, d_start, status.p);
        PN_CHECK_LAUNCH();
    }
    const uint32_t st = to_host(status.p, s);
    PN_REQUIRE(!(st & 4u), PEANUT_INVALID_ARG, "hits are not grouped by ascending read");
    PN_REQUIRE(!(st & 8u), PEANUT_INVALID_ARG, "a read's hits are not in (strand, end) order, or a start lies after its end");
    const PairIn P{H, d_start, rb.p, re.p, R->len.p, R->kk.p, ref->contig.p, ref->n_contigs, R->n_reads,
                   (int64_t)min_insert, (int64_t)max_insert};
    DBuf<uint64_t> off(n ? n : 1, s), tot(1, s);
    exclusive_scan(PairCount{P}, ArrayOut<uint64_t>{off.p}, n, tot.p, s);
    const uint64_t np = to_host(tot.p, s);
    PairOut a{};
    DBuf<uint64_t> i1(np ? np : 1, s), i2(np ? np : 1, s);
    DBuf<uint32_t> sc(np ? np : 1, s), rk(np ? np : 1, s);
    DBuf<uint8_t> mq(np ? np : 1, s), keep(np ? np : 1, s);
    a = PairOut{i1.p, i2.p, sc.p, rk.p, mq.p};
    if (np) {
        pair_write_k<<<g, 256, 0, s>>>(P, off.p, i1.p, i2.p, sc.p);
        PN_CHECK_LAUNCH();
        DBuf<uint64_t> key(np, s), val(np, s), kt(np, s), vt(np, s);
        const unsigned gp = grid_for(np, 256, (unsigned)sm_count() * 16);
        pair_keys_k<<<gp, 256, 0, s>>>(H.read_id, i1.p, sc.p, np, key.p, val.p);
        PN_CHECK_LAUNCH();
        radix_sort_pairs(key.p, val.p, kt.p, vt.p, np, kScoreBits + 23, s);
        pair_rank_k<<<gp, 256, 0, s>>>(key.p, val.p, np, (double)ref->n, (float)(10.0 * log10((double)ref->n)), rk.p,
                                       mq.p, keep.p);
        PN_CHECK_LAUNCH();
    }
    uint64_t nk = np;
    if (mode == 1 && np) {
        DBuf<uint64_t> koff(np, s);
        exclusive_scan(ArrayIn<uint8_t>{keep.p}, ArrayOut<uint64_t>{koff.p}, np, tot.p, s);
        nk = to_host(tot.p, s);
        out->i1.alloc(nk ? nk : 1, s);
        out->i2.alloc(nk ? nk : 1, s);
        out->score.alloc(nk ? nk : 1, s);
        out->rank.alloc(nk ? nk : 1, s);
        out->mapq.alloc(nk ? nk : 1, s);
        pair_keep_k<<<grid_for(np, 256, (unsigned)sm_count() * 16), 256, 0, s>>>(
            a, keep.p, koff.p, np, PairOut{out->i1.p, out->i2.p, out->score.p, out->rank.p, out->mapq.p});
        PN_CHECK_LAUNCH();
    } else {
        out->i1 = std::move(i1);
        out->i2 = std::move(i2);
        out->score = std::move(sc);
        out->rank = std::move(rk);
        out->mapq = std::move(mq);
    }
    PN_CUDA(cudaStreamSynchronize(s));
    out->p = peanut_device_pairs{nk, out->i1.p, out->i2.p, out->score.p, out->rank.p, out->mapq.p};
    return out.release();
}

// ---- the actual alignment of each hit (Section "Postprocessing") ----------------------------
//
// The pattern P (the read, or its reverse complement for strand 1; length m) against the n
// reference bases T = R[start..end], both ends fixed, at the hit's cost d: E[i][c] = the edit
// distance of P[0..i) and T[0..c).  Every path of cost at most d stays within |c - i| <= d of the
// main diagonal, so a DP over that band (2d + 1 cells per row) holds the full matrix's value at
// every cell a traceback of the optimal alignment compares.  The traceback runs from (m, n) and
// takes, at every cell, the diagonal step when it is optimal ('=' or 'X'), else a reference-only
// step ('D'), else a read-only step ('I'); runs of equal operations are written in forward order
// as len << 2 | code (0 '=', 1 'X', 2 'I', 3 'D').  The band lives in a per-thread scratch area of
// the caller's call (cells interleaved across threads: cell e of thread t at e * T + t).
constexpr int kCigarThreads = 128;

__global__ void __launch_bounds__(kCigarThreads)
    cigar_k(peanut_device_hits H, const uint64_t* __restrict__ start, const uint8_t* __restrict__ codes,
            const uint64_t* __restrict__ base_off, const uint8_t* __restrict__ len,
            const uint32_t* __restrict__ packed, uint32_t n_reads, uint64_t n_ref, uint16_t* __restrict__ band,
            uint32_t band_cells, const uint32_t* __restrict__ list, const unsigned long long* __restrict__ count,
            uint32_t* __restrict__ ops, uint32_t cap, uint16_t* __restrict__ nops, uint32_t* status) {
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x, t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint16_t* B = band + t;
    const uint64_t nl = *count;
    for (uint64_t li = t; li < nl; li += T) {
        const uint64_t x = list[li];
        nops[x] = 0;
        const uint32_t r = H.read_id[x], s = H.strand[x];
        const int64_t j = (int64_t)H.end_pos[x], st = (int64_t)start[x];
        const int32_t d = H.dist[x];
        if (r >= n_reads || s > 1 || (uint64_t)j >= n_ref || st < 0 || st > j) {
            atomicOr(status, 1u);
            continue;
        }
        const int32_t m = len[r], n = (int32_t)(j - st + 1), W = 2 * d + 1;
        if (n - m > d || m - n > d || (uint64_t)(m + 1) * W > band_cells) {
            atomicOr(status, 2u);
            continue;
        }
        const uint8_t* rd = codes + base_off[r];
        auto pat = [&](int32_t i) -> uint32_t { return s == 0 ? rd[i] : 3u - rd[m - 1 - i]; };
        auto txt = [&](int32_t c) -> uint32_t { return ref_base(packed, (uint64_t)(st + c)); };
        // E(i, c) for |c - i| <= d at cell i * W + (c - i + d)
        auto at = [&](int32_t i, int32_t c) -> uint16_t& { return B[((uint64_t)i * W + (c - i + d)) * T]; };
        for (int32_t i = 0; i <= m; ++i) {
            const int32_t c0 = i - d > 0 ? i - d : 0, c1 = i + d < n ? i + d : n;
            const uint32_t p = i > 0 ? pat(i - 1) : 0u;
            for (int32_t c = c0; c <= c1; ++c) {
                uint32_t v;
                if (i == 0) {
                    v = (uint32_t)c;
                } else if (c == 0) {
                    v = (uint32_t)i;
                } else {
                    v = at(i - 1, c - 1) + (p != txt(c - 1) ? 1u : 0u);
                    if (c - 1 - i >= -d) v = min(v, at(i, c - 1) + 1u);
                    if (c - i + 1 <= d) v = min(v, at(i - 1, c) + 1u);
                }
                at(i, c) = (uint16_t)v;
            }
        }
        if (at(m, n) != d) {
            atomicOr(status, 2u);
            continue;
        }
        uint32_t* out = ops + x * cap;
        uint32_t runs = 0, last = 4;
        bool full = false;
        int32_t i = m, c = n;
        while (i > 0 || c > 0) {
            const uint32_t e = at(i, c);
            uint32_t code;
            if (i > 0 && c > 0 && at(i - 1, c - 1) + (pat(i - 1) != txt(c - 1) ? 1u : 0u) == e) {
                code = pat(i - 1) == txt(c - 1) ? 0u : 1u;
                --i;
                --c;
            } else if (c > 0 && c - 1 - i >= -d && at(i, c - 1) + 1u == e) {
                code = 3u;
                --c;
            } else {
                code = 2u;
                --i;
            }
            if (code == last) {
                out[runs - 1] += 4u;
            } else if (runs == cap) {
                full = true;
                break;
            } else {
                out[runs++] = 4u | code;
                last = code;
            }
        }
        if (full) {
            atomicOr(status, 4u);
            continue;
        }
        for (uint32_t a = 0, b = runs ? runs - 1 : 0; a < b; ++a, --b) {  // forward order
            const uint32_t tmp = out[a];
            out[a] = out[b];
            out[b] = tmp;
        }
        nops[x] = (uint16_t)runs;
    }
}

// Hits by distance class (d = 0 .. 7 each a class, 8 and more the last), one list per class in
// hit order, so that the lanes of a warp all run the same band and neighbouring lanes mostly align
// the same read.  Block b owns the hits [b * chunk, (b + 1) * chunk): a count pass writes its
// count of every class (cnt[class * blocks + b]), the host turns them into offsets in class-major
// order, and a fill pass writes every block's hits of each class from its offset on, tile by tile,
// in hit order.
constexpr int kCigarClasses = 9;
constexpr int kClassifyThreads = 256;

__device__ __forceinline__ uint32_t cigar_class(uint8_t d) {
    return d < kCigarClasses - 1 ? d : kCigarClasses - 1;
}

__global__ void __launch_bounds__(kClassifyThreads)
    cigar_count_k(const uint8_t* __restrict__ dist, uint64_t n, uint64_t chunk, uint32_t* __restrict__ cnt) {
    const uint64_t lo = (uint64_t)blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
    uint32_t c[kCigarClasses];
#pragma unroll
    for (int z = 0; z < kCigarClasses; ++z) c[z] = 0;
    for (uint64_t x = lo + threadIdx.x; x < hi; x += kClassifyThreads) {
        const uint32_t k = cigar_class(dist[x]);
#pragma unroll
        for (int z = 0; z < kCigarClasses; ++z) c[z] += k == (uint32_t)z ? 1u : 0u;
    }
    __shared__ uint32_t part[kClassifyThreads / 32][kCigarClasses];
#pragma unroll
    for (int z = 0; z < kCigarClasses; ++z) {
        const uint32_t t = __reduce_add_sync(kFull, c[z]);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5][z] = t;
    }
    __syncthreads();
    if (threadIdx.x < kCigarClasses) {
        uint32_t t = 0;
        for (int w = 0; w < kClassifyThreads / 32; ++w) t += part[w][threadIdx.x];
        cnt[(uint64_t)threadIdx.x * gridDim.x + blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(kClassifyThreads)
    cigar_fill_k(const uint8_t* __restrict__ dist, uint64_t n, uint64_t chunk, const uint32_t* __restrict__ off,
                 uint32_t* __restrict__ list) {
    const uint64_t lo = (uint64_t)blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
    __shared__ uint32_t base[kCigarClasses];
    __shared__ uint32_t wcnt[kClassifyThreads / 32][kCigarClasses];
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x < kCigarClasses) base[threadIdx.x] = off[(uint64_t)threadIdx.x * gridDim.x + blockIdx.x];
    for (uint64_t t0 = lo; t0 < hi; t0 += kClassifyThreads) {
        const uint64_t x = t0 + threadIdx.x;
        const uint32_t k = x < hi ? cigar_class(dist[x]) : (uint32_t)kCigarClasses;
        uint32_t rank = 0;
#pragma unroll
        for (int z = 0; z < kCigarClasses; ++z) {
            const unsigned bal = __ballot_sync(kFull, k == (uint32_t)z);
            if (lane == 0) wcnt[w][z] = __popc(bal);
            if (k == (uint32_t)z) rank = __popc(bal & ((1u << lane) - 1u));
        }
        __syncthreads();
        if (k < kCigarClasses) {
            uint32_t at = base[k] + rank;
            for (uint32_t v = 0; v < w; ++v) at += wcnt[v][k];
            list[at] = (uint32_t)x;
        }
        __syncthreads();
        if (threadIdx.x < kCigarClasses) {
            uint32_t t = 0;
            for (int v = 0; v < kClassifyThreads / 32; ++v) t += wcnt[v][threadIdx.x];
            base[threadIdx.x] += t;
        }
        __syncthreads();
    }
}

// The same alignment for hits of distance D (0 to 7, one instance each), on a narrower band: with
// Delta = n - m, a path of cost d that visits diagonal offset delta = c - i pays at least
// |delta| + |Delta - delta| for its gaps, so every path of cost d stays within
// lo = ceil((Delta - d) / 2) <= delta <= floor((Delta + d) / 2), at most d + 1 diagonals; any cell a
// traceback of an optimal path compares and could step to lies on a path of cost d, so the band's
// values decide every step as the full matrix does (the others compare as not optimal either way).
// The band's row lives in registers (D + 1 cells, one per o = delta - lo), and only the traceback
// direction of every cell is kept, two bits per cell, one 16-bit word per row: 0 the diagonal step
// on a match, 3 on a mismatch, 1 the reference-only step, 2 the read-only step, chosen by the
// traceback's own preference from the final values, so the walk back reads the same decisions (and
// needs no bases).  The direction words live in a scratch area of the call, interleaved across
// threads (row i of thread t at i * T + t), which leaves the occupancy to the registers.  Hits of
// other distances are left to the other kernels.
constexpr int kBandThreads = 64;

template <int D>
__global__ void __launch_bounds__(kBandThreads)
    cigar_band_k(peanut_device_hits H, const uint64_t* __restrict__ start, const uint8_t* __restrict__ codes,
                 const uint64_t* __restrict__ base_off, const uint8_t* __restrict__ len,
                 const uint32_t* __restrict__ packed, uint32_t n_reads, uint64_t n_ref,
                 const uint32_t* __restrict__ list, const unsigned long long* __restrict__ count,
                 uint16_t* __restrict__ dirs_all, uint32_t* __restrict__ ops, uint32_t cap, uint16_t* __restrict__ nops,
                 uint32_t* status) {
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    uint16_t* dirs = dirs_all + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nl = *count;
    constexpr int WB = D + 1;
    constexpr int32_t d = D;
    static_assert(2 * WB <= 16, "a row's directions fill one 16-bit word");
    for (uint64_t li = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; li < nl; li += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = list[li];
        nops[x] = 0;
        const uint32_t r = H.read_id[x], s = H.strand[x];
        const int64_t j = (int64_t)H.end_pos[x], st = (int64_t)start[x];
        if (r >= n_reads || s > 1 || (uint64_t)j >= n_ref || st < 0 || st > j) {
            atomicOr(status, 1u);
            continue;
        }
        const int32_t m = len[r], n = (int32_t)(j - st + 1);
        if (n - m > d || m - n > d) {
            atomicOr(status, 2u);
            continue;
        }
        const int32_t lo = -((d - (n - m)) / 2);  // ceil((Delta - d) / 2), Delta - d <= 0
        const uint8_t* rd = codes + base_off[r];
        auto pat = [&](int32_t i) -> uint32_t { return s == 0 ? rd[i] : 3u - rd[m - 1 - i]; };
        // 16 reference bases starting at position p, first base most significant (a window that
        // starts before position 0 is shifted so that its bases keep their places; those before
        // 0, and those past the hit's end, are never used)
        auto bases16 = [&](int64_t p) -> uint32_t {
            const uint64_t q = p < 0 ? 0 : (uint64_t)p;
            const uint32_t w0 = __ldg(packed + (q >> 4)), w1 = __ldg(packed + (q >> 4) + 1);
            const uint32_t w = __funnelshift_l(w1, w0, 2u * (uint32_t)(q & 15));
            return p < 0 ? w >> (2 * (uint32_t)(-p)) : w;
        };
        constexpr uint32_t kInf = 0xFFFFu;
        // the band's row, updated in place: before cell o of row i is written, row[o] and
        // row[o + 1] still hold row i - 1 (the diagonal and the up neighbours) and row[o - 1]
        // already holds row i (the left neighbour)
        uint32_t row[WB];
        // row 0: E(0, c) = c for c = lo + o >= 0
        uint32_t wdir = 0;
#pragma unroll
        for (int o = 0; o < WB; ++o) {
            const int32_t c = lo + o;
            row[o] = (c >= 0 && c <= n) ? (uint32_t)c : kInf;
            wdir |= 1u << (2 * o);  // reference-only steps along row 0
        }
        dirs[0] = (uint16_t)wdir;
        // row i needs read base i - 1 and the d + 1 text bases from position st + i - 1 + lo on
        // (first base most significant).  Rows whose window starts at or after position 0 take
        // it from a sliding pair of packed words (w0, w1) with the next word (w2) loaded 16 rows
        // ahead; the first rows of a band that starts before position 0 load a shifted window.
        int64_t q = st + lo;  // the window start of row i (row 1 first)
        uint32_t w0 = 0, w1 = 0, w2 = 0;
        bool slid = false;
        uint32_t p_next = m > 0 ? pat(0) : 0u;
        for (int32_t i = 1; i <= m; ++i, ++q) {
            const uint32_t p = p_next;
            if (i < m) p_next = pat(i);
            uint32_t tw;
            if (q < 0) {
                tw = bases16(q);
            } else {
                const uint32_t sh = (uint32_t)q & 15u;
                if (!slid || sh == 0) {
                    if (!slid) {
                        const uint32_t* pw = packed + (q >> 4);
                        w0 = __ldg(pw);
                        w1 = __ldg(pw + 1);
                        w2 = __ldg(pw + 2);
                        slid = true;
                    } else {
                        w0 = w1;
                        w1 = w2;
                        w2 = __ldg(packed + (q >> 4) + 2);
                    }
                }
                tw = __funnelshift_l(w1, w0, 2u * sh);
            }
            wdir = 0;
            if (i + lo >= 1 && i + lo + WB - 1 <= n) {
                // every cell of the row lies inside the rectangle (1 <= c <= n), so its value is
                // its diagonal neighbour a or a + 1: a + 1 exactly when the bases differ and
                // neither the left nor the up neighbour is below a.  The direction follows the
                // traceback's preference: the diagonal when it is optimal (a match, or a
                // mismatch with value a + 1), else the reference-only step when the left
                // neighbour is a - 1, else the read-only step.
                const uint32_t x = tw ^ (p * 0x55555555u);
                const uint32_t mm = (x | (x >> 1)) & 0x55555555u;  // bit 30 - 2o: cell o's bases differ
#pragma unroll
                for (int o = 0; o < WB; ++o) {
                    const uint32_t av = row[o];
                    const uint32_t lf = o > 0 ? row[o - 1] : kInf;
                    const uint32_t up = o + 1 < WB ? row[o + 1] : kInf;
                    const bool mis = (mm >> (30 - 2 * o)) & 1u;
                    const bool ge = lf >= av && up >= av;
                    const uint32_t dir = !mis ? 0u : (ge ? 3u : (lf < av ? 1u : 2u));
                    row[o] = av + (mis && ge ? 1u : 0u);
                    wdir |= dir << (2 * o);
                }
            } else {
#pragma unroll
                for (int o = 0; o < WB; ++o) {
                    const int32_t c = i + lo + o;
                    uint32_t v = kInf, dir = 0;
                    if (c >= 0 && c <= n) {
                        if (c == 0) {
                            v = (uint32_t)i;
                            dir = 2;
                        } else {
                            const uint32_t mis = p != ((tw >> (30 - 2 * o)) & 3u) ? 1u : 0u;
                            const uint32_t dg = row[o] + mis;
                            const uint32_t lf = o > 0 ? row[o - 1] + 1u : kInf;
                            const uint32_t up = o + 1 < WB ? row[o + 1] + 1u : kInf;
                            v = min(dg, min(lf, up));
                            dir = dg == v ? 3u * mis : (lf == v ? 1u : 2u);
                        }
                    }
                    row[o] = v;
                    wdir |= dir << (2 * o);
                }
            }
            dirs[(uint64_t)i * T] = (uint16_t)wdir;
        }
        // E(m, n) sits at offset n - m - lo of the last row
        uint32_t em = kInf;
#pragma unroll
        for (int o = 0; o < WB; ++o)
            if (o == n - m - lo) em = row[o];
        if (em != (uint32_t)d) {
            atomicOr(status, 2u);
            continue;
        }
        uint32_t* out = ops + x * cap;
        uint32_t runs = 0, last = 4;
        uint32_t fail = 0;
        int32_t i = m, c = n;
        while (i > 0 || c > 0) {
            const int32_t o = c - i - lo;
            if (o < 0 || o >= WB) {  // an optimal path never leaves the band
                fail = 2u;
                break;
            }
            const uint32_t dir = ((uint32_t)dirs[(uint64_t)i * T] >> (2 * o)) & 3u;
            uint32_t code;
            if (dir == 0 || dir == 3) {  // the diagonal step: 0 a match, 3 a mismatch
                code = dir == 0 ? 0u : 1u;
                --i;
                --c;
            } else if (dir == 1) {
                code = 3u;
                --c;
            } else {
                code = 2u;
                --i;
            }
            if (code == last) {
                out[runs - 1] += 4u;
            } else if (runs == cap) {
                fail = 4u;
                break;
            } else {
                out[runs++] = 4u | code;
                last = code;
            }
        }
        if (fail) {
            atomicOr(status, fail);
            continue;
        }
        for (uint32_t a = 0, b = runs ? runs - 1 : 0; a < b; ++a, --b) {
            const uint32_t tmp = out[a];
            out[a] = out[b];
            out[b] = tmp;
        }
        nops[x] = (uint16_t)runs;
    }
}

void hit_alignments(const peanut_ref* ref, const peanut_reads* R, const peanut_device_hits& H, const uint64_t* d_start,
                    uint32_t cap, uint32_t* d_ops, uint16_t* d_nops) {
    cudaStream_t s = R->stream;
    const uint64_t n = H.n;
    if (!n) return;
    DBuf<uint32_t> status(1, s);
    status.zero();
    // distances 0..7: the register band of exactly 2 d + 1 diagonals; 8 and more: the scratch band
    PN_REQUIRE(n < (1ull << 32), PEANUT_UNSUPPORTED, "more than 2^32 - 1 hits in one call");
    const uint32_t nb = (uint32_t)std::min<uint64_t>((n + 4095) / 4096, (uint64_t)sm_count() * 8);
    const uint64_t chunk = (n + nb - 1) / nb;
    DBuf<uint32_t> bcnt((uint64_t)kCigarClasses * nb, s);
    cigar_count_k<<<nb, kClassifyThreads, 0, s>>>(H.dist, n, chunk, bcnt.p);
    PN_CHECK_LAUNCH();
    std::vector<uint32_t> hoff((size_t)kCigarClasses * nb);
    PN_CUDA(cudaMemcpyAsync(hoff.data(), bcnt.p, hoff.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    PN_CUDA(cudaStreamSynchronize(s));
    unsigned long long nc[kCigarClasses], off[kCigarClasses];
    uint32_t run = 0;
    for (int c = 0; c < kCigarClasses; ++c) {
        off[c] = run;
        for (uint32_t b = 0; b < nb; ++b) {
            const uint32_t t = hoff[(size_t)c * nb + b];
            hoff[(size_t)c * nb + b] = run;
            run += t;
        }
        nc[c] = run - off[c];
        PN_REQUIRE(nc[c] == 0 || (uint32_t)c <= R->max_k, PEANUT_INVALID_ARG,
                   "a hit's distance exceeds the batch's largest k (%u)", R->max_k);
    }
    DBuf<unsigned long long> len_d(kCigarClasses, s);
    PN_CUDA(cudaMemcpyAsync(bcnt.p, hoff.data(), hoff.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    PN_CUDA(cudaMemcpyAsync(len_d.p, nc, sizeof(nc), cudaMemcpyHostToDevice, s));
    DBuf<uint32_t> list(n, s);
    cigar_fill_k<<<nb, kClassifyThreads, 0, s>>>(H.dist, n, chunk, bcnt.p, list.p);
    PN_CHECK_LAUNCH();
    // one grid per band width, as many blocks as its registers let stay resident (and no more
    // than its hits need); the direction scratch is sized for the largest
    using BandKernel = decltype(&cigar_band_k<0>);
    const BandKernel kern[kCigarClasses - 1] = {cigar_band_k<0>, cigar_band_k<1>, cigar_band_k<2>, cigar_band_k<3>,
                                               cigar_band_k<4>, cigar_band_k<5>, cigar_band_k<6>, cigar_band_k<7>};
    unsigned grid[kCigarClasses - 1] = {};
    unsigned gmax = 0;
    for (int c = 0; c < kCigarClasses - 1; ++c) {
        if (!nc[c]) continue;
        int per_sm = 0;
        PN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern[c], kBandThreads, 0));
        grid[c] = grid_for(nc[c], kBandThreads, (unsigned)sm_count() * (unsigned)std::max(per_sm, 1));
        gmax = std::max(gmax, grid[c]);
    }
    DBuf<uint16_t> dirs((uint64_t)(R->max_len + 1) * std::max(gmax, 1u) * kBandThreads, s);
    for (int c = 0; c < kCigarClasses - 1; ++c) {
        if (!nc[c]) continue;
        kern[c]<<<grid[c], kBandThreads, 0, s>>>(H, d_start, R->codes.p, R->base_off.p, R->len.p, ref->packed.p,
                                                 R->n_reads, ref->n, list.p + off[c], len_d.p + c, dirs.p, d_ops,
                                                 cap, d_nops, status.p);
        PN_CHECK_LAUNCH();
    }
    if (nc[kCigarClasses - 1]) {
        const uint32_t W = 2 * R->max_k + 1;
        const uint32_t cells = (R->max_len + 1) * W;
        const unsigned g = grid_for(n, kCigarThreads, (unsigned)sm_count() * 4);
        DBuf<uint16_t> bandbuf((uint64_t)cells * g * kCigarThreads, s);
        cigar_k<<<g, kCigarThreads, 0, s>>>(H, d_start, R->codes.p, R->base_off.p, R->len.p, ref->packed.p, R->n_reads,
                                            ref->n, bandbuf.p, cells, list.p + off[kCigarClasses - 1],
                                            len_d.p + kCigarClasses - 1, d_ops, cap, d_nops, status.p);
        PN_CHECK_LAUNCH();
    }
    const uint32_t st = to_host(status.p, s);
    PN_REQUIRE(!(st & 1u), PEANUT_INVALID_ARG, "a hit names a read, strand or end outside the batch / reference, "
               "or a start after its end");
    PN_REQUIRE(!(st & 2u), PEANUT_INVALID_ARG, "a hit's distance is not the edit distance of its pattern and "
               "reference bases from its start");
    PN_REQUIRE(!(st & 4u), PEANUT_INVALID_ARG, "a hit's alignment has more than %u runs of operations", cap);
}

}  // namespace pn
