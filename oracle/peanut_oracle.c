/* PEANUT read-mapping oracle: TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, __graft_entry__.smoke() and bench.py's CPU-baseline / reference arm may load,
 * call or link this file.  The CUDA library never does, and this file includes nothing of it.
 *
 * A plain, slow, single-threaded CPU restatement of what the filter-and-verify hot path of
 * Köster & Rahmann, "Massively parallel read mapping on GPUs with PEANUT", computes:
 *
 *   Section "Validation": E[i][j] is the smallest edit distance (unit costs) between the read
 *   prefix of length i and any reference substring ending at j.  Boundary: E[0][j] = 0 (the
 *   alignment may start anywhere), E[i][-1] = i.  Recurrence:
 *       E[i][j] = min(E[i-1][j-1] + [P[i-1] != R[j]], E[i-1][j] + 1, E[i][j-1] + 1).
 *   D[j] = E[m][j] for j in [0, n).  A reference of several contigs, or with long runs of N, is
 *   a list of segments (below, "unknown bases and contigs"); the matrix then restarts at every
 *   segment start (E[i][a-1] = i for segment [a, b)) and only ends inside a segment count.
 *
 *   Hit set (the reading adopted for the paper's "duplicate removal" and strata, Section
 *   "Postprocessing"): for read r, strand s (s = 1 aligns the reverse complement of the read to
 *   the forward reference, in forward coordinates) and every maximal run of consecutive end
 *   positions j with D[j] <= k, one tuple (r, s, j*, D[j*]) where j* is the leftmost position of
 *   the run's minimum.  "all" mode keeps every tuple; "best-stratum" keeps, per read, the tuples
 *   whose D equals the read's minimum over both strands.
 *
 * Two routes to the same set:
 *   oracle_map_bruteforce: the definition above, the full DP over the whole reference;
 *   oracle_map_filter:     the q-gram filter of Section "Filtration" (hash-map q-gram index of the
 *                          reads and of their reverse complements; every reference q-gram looked
 *                          up; hits counted per (read, strand, diagonal d = p - i)), the q-gram
 *                          lemma threshold t = m + 1 - q(k + 1) of Section "The q-group index"
 *                          applied to every window of k+1 consecutive diagonals, and the DP of
 *                          Section "Validation" run only over the end range
 *                          [d0 + m - 1 - 2k, d0 + m - 1 + 3k] of each window that passes.
 *   oracle_qgroup_build:   Algorithm 1 (q-group index I, S, S', O) over a text of q-gram codes,
 *                          with GROUPBIT / GROUPRANK / INDEXPAIR as defined in Section
 *                          "The q-group index" and Section "Filtration".
 *   oracle_annotate:       per hit, the alignment start from the backward DP (Section
 *                          "Validation"), the hit-rank and the mapping quality (Section
 *                          "Postprocessing").
 *
 * Readings where the paper is silent: 0-based inclusive end positions in forward coordinates;
 * exclusive cumulative sums in Algorithm 1, S' with one sentinel entry holding |T|; only
 * q-grams lying fully inside one read are indexed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- encoding (Section "The q-group index": A=00, C=01, G=10, T=11) ---- */

static int base_code(char c) {
    switch (c) {
        case 'A': return 0;
        case 'C': return 1;
        case 'G': return 2;
        case 'T': return 3;
        default: return -1;
    }
}

static char complement(char c) {
    switch (c) {
        case 'A': return 'T';
        case 'C': return 'G';
        case 'G': return 'C';
        default: return 'A';
    }
}

static int check_acgt(const char* s, int64_t n) {
    for (int64_t i = 0; i < n; i++)
        if (base_code(s[i]) < 0) return -1;
    return 0;
}

/* ---- unknown bases and contigs ----
 *
 * Section "The q-group index" (encoding paragraph): an unknown base N becomes a random base, and
 * long runs of N stay out of the index.  Section "Overview": every step runs per chromosome, so
 * no hit spans two contigs.  Readings:
 *   - the random base is drawn from a counter-based generator, so that a run is reproducible:
 *     reference position p takes the top two bits of output p + 1 of SplitMix64 started at the
 *     reference's seed; offset i of a read takes the top two bits of output i + 1 of SplitMix64
 *     started at (seed XOR the FNV-1a 64 hash of the read's bytes, upper-cased), so a read's
 *     bases do not depend on the batch it arrives in;
 *   - a run of at least gap_min Ns inside one contig is a gap: like a contig boundary, no
 *     alignment enters it and none spans it.  The reference is then a list of segments (the
 *     stretches of each contig between gaps), and the semiglobal matrix restarts at every
 *     segment start: D[j] for j in segment [a, b) is computed over R[a..j] only;
 *   - lower-case a, c, g, t, n mean their upper-case bases (soft-masked input). */

/* SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the state advances by the odd constant 0x9E3779B97F4A7C15 and each
 * output is the state passed through the generator's finalizer (xor-shift 30, multiply
 * 0xBF58476D1CE4E5B9, xor-shift 27, multiply 0x94D049BB133111EB, xor-shift 31).  Returns output
 * number i (i >= 1) of the generator seeded with `seed`. */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + i * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* FNV-1a, 64 bits (G. Fowler, L. C. Noll, K.-P. Vo): start from the offset basis
 * 0xcbf29ce484222325; per byte, xor it in, then multiply by the prime 0x100000001b3. */
uint64_t oracle_fnv1a64(const char* s, int64_t n) {
    uint64_t h = 0xcbf29ce484222325ULL;
    for (int64_t i = 0; i < n; i++) {
        h ^= (uint8_t)s[i];
        h *= 0x100000001b3ULL;
    }
    return h;
}

static char upper_base(char c) {
    switch (c) {
        case 'a': return 'A';
        case 'c': return 'C';
        case 'g': return 'G';
        case 't': return 'T';
        case 'n': return 'N';
        default: return c;
    }
}

/* Replaces the unknown bases of a reference and lists its segments.
 *   seq[0..n): A/C/G/T/N in either case.  contig_starts[0..ncontig): 0 first, strictly
 *   ascending, each < n (contig c spans [contig_starts[c], contig_starts[c + 1]) and the last
 *   ends at n).  gap_min >= 1.
 *   text[0..n) receives the reference with every N replaced (gap bases too, although no
 *   alignment uses them).  seg[2 s], seg[2 s + 1] receive segment s as [start, end).
 * Returns the number of segments, -1 on a bad byte or contig list, -2 if more than seg_cap. */
int64_t oracle_prepare_reference(const char* seq, int64_t n, const int64_t* contig_starts, int64_t ncontig,
                                 int64_t gap_min, uint64_t seed, char* text, int64_t* seg, int64_t seg_cap) {
    if (ncontig < 1 || contig_starts[0] != 0 || gap_min < 1) return -1;
    for (int64_t c = 1; c < ncontig; c++)
        if (contig_starts[c] <= contig_starts[c - 1] || contig_starts[c] >= n) return -1;
    for (int64_t p = 0; p < n; p++) {
        char u = upper_base(seq[p]);
        if (u == 'N') {
            text[p] = "ACGT"[oracle_splitmix64(seed, (uint64_t)p + 1) >> 62];
        } else if (base_code(u) >= 0) {
            text[p] = u;
        } else {
            return -1;
        }
    }
    int64_t ns = 0;
    for (int64_t c = 0; c < ncontig; c++) {
        const int64_t a = contig_starts[c], b = c + 1 < ncontig ? contig_starts[c + 1] : n;
        int64_t open = a; /* start of the current segment */
        int64_t p = a;
        while (p < b) {
            if (upper_base(seq[p]) != 'N') {
                p++;
                continue;
            }
            int64_t e = p;
            while (e < b && upper_base(seq[e]) == 'N') e++;
            if (e - p >= gap_min) { /* a gap: close the segment before it */
                if (p > open) {
                    if (ns == seg_cap) return -2;
                    seg[2 * ns] = open;
                    seg[2 * ns + 1] = p;
                    ns++;
                }
                open = e;
            }
            p = e;
        }
        if (b > open) {
            if (ns == seg_cap) return -2;
            seg[2 * ns] = open;
            seg[2 * ns + 1] = b;
            ns++;
        }
    }
    return ns;
}

/* Replaces the unknown bases of a batch of reads (bytes A/C/G/T/N in either case) into out,
 * upper-cased.  Returns 0, or -1 on a bad byte. */
int oracle_prepare_reads(const char* reads, const int64_t* offs, int64_t nreads, uint64_t seed, char* out) {
    for (int64_t r = 0; r < nreads; r++) {
        const int64_t a = offs[r], m = offs[r + 1] - offs[r];
        for (int64_t i = 0; i < m; i++) {
            out[a + i] = upper_base(reads[a + i]);
            if (out[a + i] != 'N' && base_code(out[a + i]) < 0) return -1;
        }
        const uint64_t h = oracle_fnv1a64(out + a, m);
        for (int64_t i = 0; i < m; i++)
            if (out[a + i] == 'N') out[a + i] = "ACGT"[oracle_splitmix64(seed ^ h, (uint64_t)i + 1) >> 62];
    }
    return 0;
}

/* The segments a call maps against: seg[0..2 nseg) when given, else one segment [0, n). */
typedef struct {
    const int64_t* v;
    int64_t n;
    int64_t whole[2];
} segs_t;

static void segs_init(segs_t* S, const int64_t* seg, int64_t nseg, int64_t n) {
    S->whole[0] = 0;
    S->whole[1] = n;
    if (seg && nseg > 0) {
        S->v = seg;
        S->n = nseg;
    } else {
        S->v = S->whole;
        S->n = n > 0 ? 1 : 0;
    }
}

/* Segments must be non-empty, ascending, disjoint and inside [0, n). */
static int segs_valid(const segs_t* S, int64_t n) {
    for (int64_t x = 0; x < S->n; x++) {
        if (S->v[2 * x] < 0 || S->v[2 * x] >= S->v[2 * x + 1] || S->v[2 * x + 1] > n) return 0;
        if (x > 0 && S->v[2 * x] < S->v[2 * x - 1]) return 0;
    }
    return 1;
}

/* ---- semiglobal DP (Section "Validation") ---- */

/* One DP column sweep over R[a..b] (inclusive) with boundary E[i][a-1] = i; D[j - a] = E[m][j]. */
static void dp_columns(const char* P, int64_t m, const char* R, int64_t a, int64_t b, int32_t* col,
                       int32_t* D) {
    for (int64_t i = 0; i <= m; i++) col[i] = (int32_t)i;
    for (int64_t j = a; j <= b; j++) {
        int32_t diag = col[0]; /* E[0][j-1] */
        col[0] = 0;            /* E[0][j] */
        for (int64_t i = 1; i <= m; i++) {
            int32_t up = col[i]; /* E[i][j-1] */
            int32_t v = diag + (P[i - 1] != R[j] ? 1 : 0);
            if (up + 1 < v) v = up + 1;
            if (col[i - 1] + 1 < v) v = col[i - 1] + 1;
            col[i] = v;
            diag = up;
        }
        D[j - a] = col[m];
    }
}

/* D[j] = E[m][j] for all j in [0, n).  Returns 0, or -1 on a non-ACGT character. */
int oracle_semiglobal_column(const char* P, int64_t m, const char* R, int64_t n, int32_t* D) {
    if (check_acgt(P, m) || check_acgt(R, n)) return -1;
    if (n <= 0) return 0;
    int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    dp_columns(P, m, R, 0, n - 1, col, D);
    free(col);
    return 0;
}

/* ---- result list ---- */

typedef struct {
    int64_t n, cap;
    uint32_t* read;
    uint8_t* strand;
    int64_t* end;
    int32_t* dist;
} oracle_hits;

static void hits_push(oracle_hits* h, uint32_t r, uint8_t s, int64_t j, int32_t d) {
    if (h->n == h->cap) {
        h->cap = h->cap ? 2 * h->cap : 1024;
        h->read = (uint32_t*)realloc(h->read, sizeof(uint32_t) * (size_t)h->cap);
        h->strand = (uint8_t*)realloc(h->strand, (size_t)h->cap);
        h->end = (int64_t*)realloc(h->end, sizeof(int64_t) * (size_t)h->cap);
        h->dist = (int32_t*)realloc(h->dist, sizeof(int32_t) * (size_t)h->cap);
    }
    h->read[h->n] = r;
    h->strand[h->n] = s;
    h->end[h->n] = j;
    h->dist[h->n] = d;
    h->n++;
}

int64_t oracle_hits_count(const oracle_hits* h) { return h ? h->n : -1; }

void oracle_hits_copy(const oracle_hits* h, uint32_t* read, uint8_t* strand, int64_t* end, int32_t* dist) {
    memcpy(read, h->read, sizeof(uint32_t) * (size_t)h->n);
    memcpy(strand, h->strand, (size_t)h->n);
    memcpy(end, h->end, sizeof(int64_t) * (size_t)h->n);
    memcpy(dist, h->dist, sizeof(int32_t) * (size_t)h->n);
}

void oracle_hits_free(oracle_hits* h) {
    if (!h) return;
    free(h->read);
    free(h->strand);
    free(h->end);
    free(h->dist);
    free(h);
}

/* mode: 0 = all (canonical tuple per maximal run), 1 = best stratum, 2 = every end with D <= k */
enum { MODE_ALL = 0, MODE_BEST = 1, MODE_ENDS = 2 };

/* Ends js[0..cnt) strictly increasing with values ds (all <= k): emit one tuple per maximal run
 * of consecutive positions (leftmost minimum), or every end in MODE_ENDS. */
static void emit_runs(oracle_hits* h, uint32_t r, uint8_t s, const int64_t* js, const int32_t* ds,
                      int64_t cnt, int mode) {
    int64_t x = 0;
    while (x < cnt) {
        if (mode == MODE_ENDS) {
            hits_push(h, r, s, js[x], ds[x]);
            x++;
            continue;
        }
        int64_t y = x, best = x;
        while (y + 1 < cnt && js[y + 1] == js[y] + 1) {
            y++;
            if (ds[y] < ds[best]) best = y;
        }
        hits_push(h, r, s, js[best], ds[best]);
        x = y + 1;
    }
}

/* Best stratum: keep, for every read, the tuples whose distance equals that read's minimum.
 * Tuples of one read are contiguous in h (both strands). */
static void best_stratum(oracle_hits* h) {
    int64_t w = 0, x = 0;
    while (x < h->n) {
        int64_t y = x;
        int32_t mn = h->dist[x];
        while (y < h->n && h->read[y] == h->read[x]) {
            if (h->dist[y] < mn) mn = h->dist[y];
            y++;
        }
        for (int64_t z = x; z < y; z++) {
            if (h->dist[z] == mn) {
                h->read[w] = h->read[z];
                h->strand[w] = h->strand[z];
                h->end[w] = h->end[z];
                h->dist[w] = h->dist[z];
                w++;
            }
        }
        x = y;
    }
    h->n = w;
}

static char* revcomp_copy(const char* s, int64_t m) {
    char* o = (char*)malloc((size_t)m + 1);
    for (int64_t i = 0; i < m; i++) o[i] = complement(s[m - 1 - i]);
    o[m] = 0;
    return o;
}

/* ---- brute force: the definition over the whole reference ---- */

oracle_hits* oracle_map_bruteforce(const char* R, int64_t n, const char* reads, const int64_t* offs,
                                   int64_t nreads, const int32_t* k, int mode, const int64_t* seg, int64_t nseg) {
    if (check_acgt(R, n) || check_acgt(reads, offs[nreads] - offs[0])) return NULL;
    segs_t S;
    segs_init(&S, seg, nseg, n);
    if (!segs_valid(&S, n)) return NULL;
    oracle_hits* h = (oracle_hits*)calloc(1, sizeof(oracle_hits));
    int32_t* D = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t* js = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t* ds = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t r = 0; r < nreads; r++) {
        int64_t m = offs[r + 1] - offs[r];
        int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
        for (int s = 0; s < 2; s++) {
            char* P = s == 0 ? NULL : revcomp_copy(reads + offs[r], m);
            const char* pat = s == 0 ? reads + offs[r] : P;
            for (int64_t x = 0; x < S.n; x++) { /* the matrix restarts at every segment start */
                const int64_t a = S.v[2 * x], b = S.v[2 * x + 1];
                dp_columns(pat, m, R, a, b - 1, col, D);
                int64_t cnt = 0;
                for (int64_t j = a; j < b; j++)
                    if (D[j - a] <= k[r]) {
                        js[cnt] = j;
                        ds[cnt] = D[j - a];
                        cnt++;
                    }
                emit_runs(h, (uint32_t)r, (uint8_t)s, js, ds, cnt, mode);
            }
            free(P);
        }
        free(col);
    }
    free(D);
    free(js);
    free(ds);
    if (mode == MODE_BEST) best_stratum(h);
    return h;
}

/* ---- q-gram filter (Section "Filtration") + windowed DP ---- */

typedef struct { uint64_t key; int64_t head; } slot_t;
typedef struct { int32_t r; int8_t s; int16_t i; int64_t next; } occ_t;

typedef struct { int64_t* v; int64_t n, cap; } vec64;

static void vec_push(vec64* a, int64_t x) {
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 16;
        a->v = (int64_t*)realloc(a->v, sizeof(int64_t) * (size_t)a->cap);
    }
    a->v[a->n++] = x;
}

static int cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return x < y ? -1 : x > y;
}

typedef struct { int64_t lo, hi; } ival;

static int cmp_ival(const void* a, const void* b) {
    const ival* x = (const ival*)a;
    const ival* y = (const ival*)b;
    if (x->lo != y->lo) return x->lo < y->lo ? -1 : 1;
    return x->hi < y->hi ? -1 : x->hi > y->hi;
}

/* first index in sorted v[0..n) with v[idx] >= x */
static int64_t lower_bound(const int64_t* v, int64_t n, int64_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (v[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

static uint64_t hash64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    return x;
}

/* q-gram code, first base most significant (numeric order = lexicographic order) */
static uint64_t qgram_code(const char* s, int q) {
    uint64_t g = 0;
    for (int t = 0; t < q; t++) g = (g << 2) | (uint64_t)base_code(s[t]);
    return g;
}

/* Returns NULL if q is out of range [1, 31], a character is not ACGT, or some read has a
 * lemma threshold t = m + 1 - q(k + 1) below 1 (the filter would not be lossless). */
oracle_hits* oracle_map_filter(const char* R, int64_t n, const char* reads, const int64_t* offs,
                               int64_t nreads, const int32_t* k, int q, int mode, const int64_t* seg, int64_t nseg) {
    if (q < 1 || q > 31) return NULL;
    if (check_acgt(R, n) || check_acgt(reads, offs[nreads] - offs[0])) return NULL;
    segs_t S;
    segs_init(&S, seg, nseg, n);
    if (!segs_valid(&S, n)) return NULL;
    for (int64_t r = 0; r < nreads; r++) {
        int64_t m = offs[r + 1] - offs[r];
        if (m + 1 - (int64_t)q * (k[r] + 1) < 1) return NULL;
    }
    /* 1. index: q-gram code -> list of (read, strand, offset), reads and reverse complements */
    int64_t total = 0;
    for (int64_t r = 0; r < nreads; r++) total += 2 * (offs[r + 1] - offs[r] - q + 1);
    uint64_t cap = 16;
    while (cap < (uint64_t)(2 * total + 16)) cap <<= 1;
    slot_t* tab = (slot_t*)malloc(sizeof(slot_t) * cap);
    for (uint64_t x = 0; x < cap; x++) { tab[x].key = UINT64_MAX; tab[x].head = -1; }
    occ_t* occ = (occ_t*)malloc(sizeof(occ_t) * (size_t)(total > 0 ? total : 1));
    int64_t nocc = 0;
    char** pats = (char**)malloc(sizeof(char*) * (size_t)(2 * nreads + 1));
    for (int64_t r = 0; r < nreads; r++) {
        int64_t m = offs[r + 1] - offs[r];
        pats[2 * r] = (char*)malloc((size_t)m + 1);
        memcpy(pats[2 * r], reads + offs[r], (size_t)m);
        pats[2 * r + 1] = revcomp_copy(reads + offs[r], m);
        for (int s = 0; s < 2; s++) {
            const char* P = pats[2 * r + s];
            for (int64_t i = 0; i + q <= m; i++) {
                uint64_t g = qgram_code(P + i, q);
                uint64_t x = hash64(g) & (cap - 1);
                while (tab[x].key != UINT64_MAX && tab[x].key != g) x = (x + 1) & (cap - 1);
                tab[x].key = g;
                occ[nocc].r = (int32_t)r;
                occ[nocc].s = (int8_t)s;
                occ[nocc].i = (int16_t)i;
                occ[nocc].next = tab[x].head;
                tab[x].head = nocc++;
            }
        }
    }
    /* 2. scan: every reference q-gram, hits on diagonal d = p - i.  The code of the q-gram at p
     * is that of p - 1 shifted by one base (drop the first, append R[p + q - 1]). */
    vec64* dg = (vec64*)calloc((size_t)(2 * nreads + 1), sizeof(vec64));
    const uint64_t qmask = (q == 32) ? ~0ULL : ((1ULL << (2 * q)) - 1);
    uint64_t g = n >= q ? qgram_code(R, q) : 0;
    for (int64_t p = 0; p + q <= n; p++) {
        if (p > 0) g = ((g << 2) | (uint64_t)base_code(R[p + q - 1])) & qmask;
        uint64_t x = hash64(g) & (cap - 1);
        while (tab[x].key != UINT64_MAX && tab[x].key != g) x = (x + 1) & (cap - 1);
        if (tab[x].key != g) continue;
        for (int64_t e = tab[x].head; e >= 0; e = occ[e].next)
            vec_push(&dg[2 * occ[e].r + occ[e].s], p - occ[e].i);
    }
    /* 3.-5. windows of k+1 diagonals with >= t hits, end ranges, windowed DP */
    oracle_hits* h = (oracle_hits*)calloc(1, sizeof(oracle_hits));
    for (int64_t r = 0; r < nreads; r++) {
        int64_t m = offs[r + 1] - offs[r];
        int64_t kk = k[r];
        int64_t t = m + 1 - (int64_t)q * (kk + 1);
        int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
        for (int s = 0; s < 2; s++) {
            vec64* v = &dg[2 * r + s];
            if (v->n == 0) continue;
            qsort(v->v, (size_t)v->n, sizeof(int64_t), cmp_i64);
            ival* iv = NULL;
            int64_t niv = 0, civ = 0;
            for (int64_t x = 0; x < v->n; x++) {
                if (x > 0 && v->v[x] == v->v[x - 1]) continue;
                for (int64_t d0 = v->v[x] - kk; d0 <= v->v[x]; d0++) {
                    int64_t c = lower_bound(v->v, v->n, d0 + kk + 1) - lower_bound(v->v, v->n, d0);
                    if (c < t) continue;
                    if (niv == civ) {
                        civ = civ ? 2 * civ : 64;
                        iv = (ival*)realloc(iv, sizeof(ival) * (size_t)civ);
                    }
                    iv[niv].lo = d0 + m - 1 - 2 * kk;
                    iv[niv].hi = d0 + m - 1 + 3 * kk;
                    niv++;
                }
            }
            if (niv == 0) { free(iv); continue; }
            qsort(iv, (size_t)niv, sizeof(ival), cmp_ival);
            /* union of end ranges, clipped to the reference; DP over each merged range */
            int64_t* js = NULL;
            int32_t* ds = NULL;
            int64_t cnt = 0, cj = 0;
            int64_t x = 0;
            while (x < niv) {
                int64_t lo = iv[x].lo, hi = iv[x].hi;
                x++;
                while (x < niv && iv[x].lo <= hi + 1) {
                    if (iv[x].hi > hi) hi = iv[x].hi;
                    x++;
                }
                if (lo < 0) lo = 0;
                if (hi > n - 1) hi = n - 1;
                /* the range's piece in each segment; the matrix restarts at the segment start */
                for (int64_t y = 0; y < S.n; y++) {
                    const int64_t sa = S.v[2 * y], sb = S.v[2 * y + 1];
                    const int64_t plo = lo > sa ? lo : sa, phi = hi < sb - 1 ? hi : sb - 1;
                    if (plo > phi) continue;
                    int64_t a = plo - (m + kk) + 1;
                    if (a < sa) a = sa;
                    int32_t* D = (int32_t*)malloc(sizeof(int32_t) * (size_t)(phi - a + 1));
                    dp_columns(pats[2 * r + s], m, R, a, phi, col, D);
                    cnt = 0;
                    for (int64_t j = plo; j <= phi; j++) {
                        if (D[j - a] > kk) continue;
                        if (cnt == cj) {
                            cj = cj ? 2 * cj : 64;
                            js = (int64_t*)realloc(js, sizeof(int64_t) * (size_t)cj);
                            ds = (int32_t*)realloc(ds, sizeof(int32_t) * (size_t)cj);
                        }
                        js[cnt] = j;
                        ds[cnt] = D[j - a];
                        cnt++;
                    }
                    free(D);
                    /* 6. canonical tuple per maximal run (a run ends at its piece's edges) */
                    emit_runs(h, (uint32_t)r, (uint8_t)s, js, ds, cnt, mode);
                }
            }
            free(js);
            free(ds);
            free(iv);
        }
        free(col);
    }
    if (mode == MODE_BEST) best_stratum(h);
    for (int64_t x = 0; x < 2 * nreads; x++) free(dg[x].v);
    free(dg);
    for (int64_t x = 0; x < 2 * nreads; x++) free(pats[x]);
    free(pats);
    free(occ);
    free(tab);
    return h;
}

/* ---- Algorithm 1: the q-group index over a text of q-gram codes ---- */

/* GROUPBIT(g) = (g div w, g mod w) */
static void groupbit(uint64_t g, int w, uint64_t* i, int* j) {
    *i = g / (uint64_t)w;
    *j = (int)(g % (uint64_t)w);
}

static int popcount64(uint64_t x) {
    int c = 0;
    while (x) { c += (int)(x & 1); x >>= 1; }
    return c;
}

/* GROUPRANK(I, i, j) = popcount(I[i] & (2^j - 1)) */
static uint64_t grouprank(const uint64_t* I, uint64_t i, int j) {
    uint64_t mask = j == 0 ? 0 : (j >= 64 ? ~0ULL : ((1ULL << j) - 1));
    return (uint64_t)popcount64(I[i] & mask);
}

/* Builds (I, S, S', O) of Algorithm 1 for the text positions 0..T-1 whose q-gram codes are
 * codes[p]; O stores payload[p] instead of p so the caller can attach (read, offset) labels.
 * Sizes: I and S have ceil(4^q / w) entries (I holds w-bit words in uint64), S' has T + 1
 * entries (only the first distinct + 1 are used; the last of those is the sentinel |T|), O has
 * T entries.  Returns the number of distinct q-grams, or -1 on bad arguments. */
int64_t oracle_qgroup_build(const uint64_t* codes, const uint64_t* payload, int64_t T, int q, int w,
                            uint64_t* I, uint64_t* S, uint64_t* Sp, uint64_t* O) {
    if (q < 1 || q > 31 || w < 1 || w > 64) return -1;
    uint64_t ngroups = ((1ULL << (2 * q)) + (uint64_t)w - 1) / (uint64_t)w;
    /* step 1: presence bits */
    memset(I, 0, sizeof(uint64_t) * ngroups);
    for (int64_t p = 0; p < T; p++) {
        uint64_t i;
        int j;
        groupbit(codes[p], w, &i, &j);
        I[i] |= 1ULL << j;
    }
    /* steps 2-3: S = exclusive cumulative sum of popcount(I) */
    uint64_t run = 0;
    for (uint64_t i = 0; i < ngroups; i++) {
        uint64_t c = (uint64_t)popcount64(I[i]);
        S[i] = run;
        run += c;
    }
    uint64_t distinct = run;
    /* steps 4-5: occurrences per q-gram, then exclusive cumulative sum with sentinel */
    memset(Sp, 0, sizeof(uint64_t) * (size_t)(T + 1));
    for (int64_t p = 0; p < T; p++) {
        uint64_t i;
        int j;
        groupbit(codes[p], w, &i, &j);
        Sp[S[i] + grouprank(I, i, j)] += 1;
    }
    run = 0;
    for (uint64_t x = 0; x <= distinct; x++) {
        uint64_t c = x < distinct ? Sp[x] : 0;
        Sp[x] = run;
        run += c;
    }
    /* step 6: every position into the next free entry of its q-gram's interval of O */
    uint64_t* used = (uint64_t*)calloc((size_t)(distinct + 1), sizeof(uint64_t));
    for (int64_t p = 0; p < T; p++) {
        uint64_t i;
        int j;
        groupbit(codes[p], w, &i, &j);
        uint64_t x = S[i] + grouprank(I, i, j);
        O[Sp[x] + used[x]++] = payload[p];
    }
    free(used);
    return (int64_t)distinct;
}

/* INDEXPAIR(g) = (S'[S[i] + j'], S'[S[i] + j' + 1]) if bit j of I[i] is set, else (0, 0). */
void oracle_indexpair(const uint64_t* I, const uint64_t* S, const uint64_t* Sp, int w, uint64_t g,
                      uint64_t* kstart, uint64_t* kend) {
    uint64_t i;
    int j;
    groupbit(g, w, &i, &j);
    if (!((I[i] >> j) & 1)) {
        *kstart = 0;
        *kend = 0;
        return;
    }
    uint64_t x = S[i] + grouprank(I, i, j);
    *kstart = Sp[x];
    *kend = Sp[x + 1];
}

/* ---- the canonical q-gram text the GPU index is built over ---- */

/* For every read r and offset i in [0, m - q]: g = code of read[i..i+q), h = code of the same
 * window of the reverse complement read (positions m-q-i .. m-i-1 of revcomp), c = min(g, h),
 * f = (g != c).  Writes codes[x] = c and payload[x] = (r << 9) | (f << 8) | i in read order, and
 * returns the count.  Returns -1 on a non-ACGT character or q outside [1, 31]. */
int64_t oracle_canonical_text(const char* reads, const int64_t* offs, int64_t nreads, int q,
                              uint64_t* codes, uint64_t* payload) {
    if (q < 1 || q > 31) return -1;
    if (check_acgt(reads, offs[nreads] - offs[0])) return -1;
    int64_t x = 0;
    for (int64_t r = 0; r < nreads; r++) {
        int64_t m = offs[r + 1] - offs[r];
        char* rc = revcomp_copy(reads + offs[r], m);
        for (int64_t i = 0; i + q <= m; i++) {
            uint64_t g = qgram_code(reads + offs[r] + i, q);
            uint64_t h = qgram_code(rc + (m - q - i), q);
            uint64_t c = g < h ? g : h;
            codes[x] = c;
            payload[x] = ((uint64_t)r << 9) | ((uint64_t)(g != c) << 8) | (uint64_t)i;
            x++;
        }
        free(rc);
    }
    return x;
}

/* Occurrence count of every canonical q-gram of the reference whose count exceeds cap:
 * writes up to max_out (code, count) pairs sorted by code and returns how many exist.
 * The canonical code of position p is min(code(R[p..p+q)), code(revcomp(R[p..p+q)))). */
int64_t oracle_frequent_qgrams(const char* R, int64_t n, int q, int64_t cap, uint64_t* out_codes,
                               int64_t* out_counts, int64_t max_out) {
    if (q < 1 || q > 31 || check_acgt(R, n)) return -1;
    int64_t np = n - q + 1;
    if (np <= 0) return 0;
    uint64_t* cs = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)np);
    char* win = (char*)malloc((size_t)q);
    for (int64_t p = 0; p < np; p++) {
        for (int t = 0; t < q; t++) win[t] = complement(R[p + q - 1 - t]);
        uint64_t g = qgram_code(R + p, q), h = qgram_code(win, q);
        cs[p] = g < h ? g : h;
    }
    free(win);
    qsort(cs, (size_t)np, sizeof(uint64_t), cmp_i64); /* codes < 2^62: signed order = unsigned */
    int64_t nout = 0, x = 0;
    while (x < np) {
        int64_t y = x;
        while (y < np && cs[y] == cs[x]) y++;
        if (y - x > cap) {
            if (nout < max_out) { out_codes[nout] = cs[x]; out_counts[nout] = y - x; }
            nout++;
        }
        x = y;
    }
    free(cs);
    return nout;
}

/* ---- postprocessing: alignment start, hit-rank, mapping quality ---- */

/* Start of a hit (Section "Validation", last paragraph: the distance of the semi-global
 * alignment recomputed in backward direction gives the alignment's start).  For a hit of
 * pattern P (the read, or its reverse complement for strand 1; length m) ending at j with
 * distance d: G[c] = edit distance between P and R[j-c+1 .. j] for c = 0, 1, ..., the edit matrix
 * of the reversed pattern against the reference read leftwards from j, with E[0][c] = c (the
 * alignment must end exactly at j) and E[i][0] = i.  min_c G[c] = d by the definition of D[j].
 * Reading (the paper does not say which start when several give d): the leftmost one,
 * start = j - c + 1 for the largest c with G[c] = d; an alignment of cost d spans at most m + d
 * reference bases, so c <= min(j + 1, m + d).  Returns -1 if no c reaches d (not a hit). */
static int64_t hit_start(const char* P, int64_t m, const char* R, int64_t seg_start, int64_t j, int32_t d) {
    int64_t C = m + d;
    if (C > j + 1 - seg_start) C = j + 1 - seg_start; /* the alignment stays in j's segment */
    int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    for (int64_t i = 0; i <= m; i++) col[i] = (int32_t)i; /* c = 0: the whole pattern deleted */
    int64_t best = (col[m] == d) ? 0 : -1;
    for (int64_t c = 1; c <= C; c++) {
        const char t = R[j - c + 1];  /* c-th reference base going left */
        int32_t diag = col[0];
        col[0] = (int32_t)c;
        for (int64_t i = 1; i <= m; i++) {
            int32_t up = col[i];
            int32_t v = diag + (P[m - i] != t ? 1 : 0); /* i-th pattern base from the right */
            if (up + 1 < v) v = up + 1;
            if (col[i - 1] + 1 < v) v = col[i - 1] + 1;
            col[i] = v;
            diag = up;
        }
        if (col[m] == d) best = c;
    }
    free(col);
    return best < 0 ? -1 : j - best + 1;
}

/* Section "Postprocessing": for the hits of a read (all of them, both strands), the hit-rank of a
 * hit is the number of the read's hits whose percent identity (m - d) / m is at least its own,
 * i.e. whose distance is at most its own; the mapping quality is
 * min(-10 log10(Pr), 255) with Pr = (rank - 1) / |P|, |P| = n reference positions.  Readings:
 * rank 1 gives Pr = 0 and quality 255; the quality is the integer part of -10 log10(Pr) computed
 * in double precision plus 1e-9 (so that ratios at exact powers of ten land on their integer on
 * any machine), clamped to 0..255.
 * Hits must be grouped by read.  start[], rank[] and mapq[] receive one value per hit.
 * Returns 0, or -1 on bad input (non-ACGT base, a hit whose start cannot be found). */
int oracle_annotate(const char* R, int64_t n, const char* reads, const int64_t* offs, int64_t nreads,
                    const uint32_t* hr, const uint8_t* hs, const int64_t* he, const int32_t* hd, int64_t nh,
                    int64_t* start, uint32_t* rank, int32_t* mapq, const int64_t* seg, int64_t nseg) {
    if (check_acgt(R, n) || check_acgt(reads, offs[nreads] - offs[0])) return -1;
    segs_t S;
    segs_init(&S, seg, nseg, n);
    if (!segs_valid(&S, n)) return -1;
    int64_t x = 0;
    while (x < nh) {
        int64_t y = x;
        while (y < nh && hr[y] == hr[x]) y++;
        const uint32_t r = hr[x];
        if ((int64_t)r >= nreads) return -1;
        const int64_t m = offs[r + 1] - offs[r];
        char* fw = (char*)malloc((size_t)m + 1);
        memcpy(fw, reads + offs[r], (size_t)m);
        char* rc = revcomp_copy(reads + offs[r], m);
        for (int64_t z = x; z < y; z++) {
            if (he[z] < 0 || he[z] >= n) return -1;
            int64_t sx = 0; /* the segment holding the end */
            while (sx < S.n && S.v[2 * sx + 1] <= he[z]) sx++;
            if (sx == S.n || S.v[2 * sx] > he[z]) return -1; /* an end in a gap */
            start[z] = hit_start(hs[z] ? rc : fw, m, R, S.v[2 * sx], he[z], hd[z]);
            if (start[z] < 0) return -1;
            uint32_t c = 0;
            for (int64_t u = x; u < y; u++) c += hd[u] <= hd[z] ? 1u : 0u;
            rank[z] = c;
            if (c <= 1) {
                mapq[z] = 255;
            } else {
                double q = -10.0 * log10((double)(c - 1) / (double)n);
                int64_t qi = (int64_t)floor(q + 1e-9);
                mapq[z] = (int32_t)(qi < 0 ? 0 : qi > 255 ? 255 : qi);
            }
        }
        free(fw);
        free(rc);
        x = y;
    }
    return 0;
}

/* ---- paired-end mates (Section "Postprocessing") ----
 *
 * The paper pairs mates during postprocessing and, in paired-end mode, sums the percent
 * identities of properly paired hits when it forms strata.  Readings (the paper does not define
 * a proper pair): reads 2p and 2p + 1 of a batch are the two mates of fragment p, sequenced from
 * its two ends (forward-reverse); hits x of mate 1 and y of mate 2 are properly paired when they
 * lie on opposite strands, in the same contig, and the fragment they span, from the start of
 * the strand-0 hit to the end of the strand-1 hit, is min_insert .. max_insert bases long.  The
 * pair's score is its summed percent identity (m1 - d1) / m1 + (m2 - d2) / m2, compared exactly
 * through the numerator (m1 - d1) m2 + (m2 - d2) m1 over the common denominator m1 m2.  Its rank
 * is the number of proper pairs of the fragment scoring at least as high, and its quality the
 * formula of oracle_annotate with that rank.  mode 0 keeps every proper pair, 1 the fragment's
 * best-scoring ones.
 *
 * Hits (grouped by read, ascending) with their starts; contig_starts[0..ncontig) as in
 * oracle_prepare_reference; n = reference length.  Pairs go to the out arrays in (fragment,
 * mate-1 hit, mate-2 hit) order.  Returns the number of pairs (filling at most cap), or -1 on
 * bad input. */
static int64_t contig_of(const int64_t* cs, int64_t nc, int64_t p) {
    int64_t c = 0;
    while (c + 1 < nc && cs[c + 1] <= p) c++;
    return c;
}

int64_t oracle_pair_hits(const uint32_t* hr, const uint8_t* hs, const int64_t* he, const int64_t* hst,
                         const int32_t* hd, int64_t nh, const int64_t* offs, int64_t nreads, const int64_t* cs,
                         int64_t ncontig, int64_t n, int64_t min_insert, int64_t max_insert, int mode, int64_t* o1,
                         int64_t* o2, int64_t* oscore, uint32_t* orank, int32_t* omapq, int64_t cap) {
    if (nreads % 2 || min_insert < 1 || max_insert < min_insert || ncontig < 1) return -1;
    for (int64_t x = 1; x < nh; x++)
        if (hr[x] < hr[x - 1]) return -1;
    int64_t np = 0, x = 0;
    while (x < nh) {
        const int64_t p = hr[x] / 2;
        int64_t a1 = x, b1 = x; /* mate-1 hits [a1, b1), mate-2 hits [b1, b2) */
        while (b1 < nh && hr[b1] == 2 * p) b1++;
        int64_t b2 = b1;
        while (b2 < nh && hr[b2] == 2 * p + 1) b2++;
        if (hr[x] == 2 * p + 1) { /* no mate-1 hits */
            a1 = b1 = x;
        }
        const int64_t m1 = offs[2 * p + 1] - offs[2 * p], m2 = offs[2 * p + 2] - offs[2 * p + 1];
        const int64_t first = np;
        int64_t best = -1;
        for (int64_t u = a1; u < b1; u++)
            for (int64_t v = b1; v < b2; v++) {
                if (hs[u] == hs[v]) continue;
                if (contig_of(cs, ncontig, he[u]) != contig_of(cs, ncontig, he[v])) continue;
                const int64_t fwd = hs[u] == 0 ? u : v, rev = hs[u] == 0 ? v : u;
                const int64_t ins = he[rev] - hst[fwd] + 1;
                if (ins < min_insert || ins > max_insert) continue;
                const int64_t sc = (m1 - hd[u]) * m2 + (m2 - hd[v]) * m1;
                if (np < cap) {
                    o1[np] = u;
                    o2[np] = v;
                    oscore[np] = sc;
                }
                if (sc > best) best = sc;
                np++;
            }
        if (np <= cap) {
            /* ranks and qualities over the fragment's pairs, then the best stratum */
            int64_t w = first;
            for (int64_t z = first; z < np; z++) {
                uint32_t c = 0;
                for (int64_t t = first; t < np; t++) c += oscore[t] >= oscore[z] ? 1u : 0u;
                orank[z] = c;
                if (c <= 1) {
                    omapq[z] = 255;
                } else {
                    double qv = -10.0 * log10((double)(c - 1) / (double)n);
                    int64_t qi = (int64_t)floor(qv + 1e-9);
                    omapq[z] = (int32_t)(qi < 0 ? 0 : qi > 255 ? 255 : qi);
                }
            }
            if (mode == 1) {
                for (int64_t z = first; z < np; z++)
                    if (oscore[z] == best) {
                        o1[w] = o1[z];
                        o2[w] = o2[z];
                        oscore[w] = oscore[z];
                        orank[w] = orank[z];
                        omapq[w] = omapq[z];
                        w++;
                    }
                np = w;
            }
        }
        x = b2 > b1 ? b2 : b1;
        if (x == a1) x++; /* defensive: always advance */
    }
    return np;
}

/* ---- the actual alignment of a hit (Section "Postprocessing") ----
 *
 * The paper's postprocessing "calculates the actual alignment of each hit".  Reading: the
 * alignment of the pattern P (the read, or its reverse complement for strand 1; length m) with
 * the n reference bases T = R[start..end] of the hit, both ends fixed, of cost dist = the hit's
 * distance: E[i][c] = the edit distance between P[0..i) and T[0..c), E[i][0] = i, E[0][c] = c.
 * Among the optimal alignments it takes the one traced back from (m, n) preferring, at every
 * cell, the diagonal step (a match '=' or a mismatch 'X') when it is optimal, else a reference
 * base against no read base ('D'), else a read base against no reference base ('I').  Output:
 * the runs of equal operations in forward order, op codes '=', 'X', 'I', 'D' in ops[] and their
 * lengths in lens[].  Returns the number of runs, -1 if E[m][n] != dist, -2 if more than cap. */
int64_t oracle_cigar(const char* P, int64_t m, const char* T, int64_t n, int32_t d, char* ops, int32_t* lens,
                     int64_t cap) {
    if (m < 0 || n < 0 || m > (1 << 20) || n > (1 << 20)) return -1;
    int32_t* E = (int32_t*)malloc(sizeof(int32_t) * (size_t)((m + 1) * (n + 1)));
#define EE(i, c) E[(i) * (n + 1) + (c)]
    for (int64_t i = 0; i <= m; i++) EE(i, 0) = (int32_t)i;
    for (int64_t c = 0; c <= n; c++) EE(0, c) = (int32_t)c;
    for (int64_t i = 1; i <= m; i++)
        for (int64_t c = 1; c <= n; c++) {
            int32_t v = EE(i - 1, c - 1) + (P[i - 1] != T[c - 1] ? 1 : 0);
            if (EE(i, c - 1) + 1 < v) v = EE(i, c - 1) + 1;
            if (EE(i - 1, c) + 1 < v) v = EE(i - 1, c) + 1;
            EE(i, c) = v;
        }
    if (EE(m, n) != d) {
        free(E);
        return -1;
    }
    /* trace back, one operation per step, then run-length encode in forward order */
    char* rev = (char*)malloc((size_t)(m + n + 1));
    int64_t nr = 0, i = m, c = n;
    while (i > 0 || c > 0) {
        const int32_t e = EE(i, c);
        if (i > 0 && c > 0 && EE(i - 1, c - 1) + (P[i - 1] != T[c - 1] ? 1 : 0) == e) {
            rev[nr++] = P[i - 1] == T[c - 1] ? '=' : 'X';
            i--;
            c--;
        } else if (c > 0 && EE(i, c - 1) + 1 == e) {
            rev[nr++] = 'D';
            c--;
        } else {
            rev[nr++] = 'I';
            i--;
        }
    }
#undef EE
    int64_t runs = 0;
    for (int64_t x = nr - 1; x >= 0; x--) {
        if (runs > 0 && ops[runs - 1] == rev[x]) {
            lens[runs - 1]++;
            continue;
        }
        if (runs == cap) {
            free(rev);
            free(E);
            return -2;
        }
        ops[runs] = rev[x];
        lens[runs] = 1;
        runs++;
    }
    free(rev);
    free(E);
    return runs;
}
