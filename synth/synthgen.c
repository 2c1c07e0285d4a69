/* Seeded synthetic references and reads (input generation only; no read-mapping arithmetic).
 *
 * Random numbers: one counter-based generator, splitmix64 (Steele, Lea & Flood, OOPSLA 2014).
 * Draw i of stream s under seed S is mix64(key(S, s) + (i + 1) * GOLDEN), where
 * key(S, s) = mix64(S * 0x100000001B3 + s * 0x632BE59BD9B4E019 + GOLDEN).  Every draw is
 * addressed by (stream, counter), so results do not depend on thread count or chunking.
 *
 * Shapes follow the workloads of Köster & Rahmann (PEANUT), Section "Results": uniform
 * background, interspersed repeat families, low-complexity tandem runs, and reads with
 * substitutions and single-base insertions/deletions sampled on a uniform strand.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

enum {
    S_BACKGROUND = 1, S_REPEAT_FAMILY = 2, S_REPEAT_BASES = 3, S_TANDEM = 4, S_TANDEM_UNIT = 5,
    S_REPEAT_MUT = 1003, S_REPEAT_POS = 1002,
    S_READ_START = 10, S_READ_STRAND = 11, S_READ_EVENTS = 12, S_READ_RANDOM = 13,
    S_READ_RATE = 14, S_READ_LEN = 15, S_READ_KIND = 16
};

static const uint8_t ASCII[4] = {'A', 'C', 'G', 'T'};

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t synth_key(uint64_t seed, uint64_t stream) {
    return mix64(seed * 0x100000001B3ULL + stream * 0x632BE59BD9B4E019ULL + GOLDEN);
}

static inline uint64_t draw(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * GOLDEN); }

static inline double unif(uint64_t key, uint64_t i) { return (double)(draw(key, i) >> 11) * 0x1.0p-53; }

/* draws [start, start+count) of a stream, for cross-checking the generator itself */
void synth_draws(uint64_t seed, uint64_t stream, uint64_t start, uint64_t count, uint64_t* out) {
    uint64_t key = synth_key(seed, stream);
    for (uint64_t i = 0; i < count; i++) out[i] = draw(key, start + i);
}

/* base b of a uniform stream: bits 2*(b%32) .. of draw b/32 */
static inline uint8_t stream_base(uint64_t key, uint64_t b) {
    return (uint8_t)((draw(key, b >> 5) >> (2 * (b & 31))) & 3);
}

/* Reference of n bases into out (ASCII).  Background uniform; then repeat families until
 * repeat_frac*n bases are placed (consensus length log-uniform in [300, 6000], 2..50 copies,
 * per-copy substitution divergence uniform in [0.10, 0.20], copies at uniform positions);
 * then tandem runs until tandem_frac*n bases are placed (period 1..6, length 20..200). */
void synth_reference(uint8_t* out, uint64_t n, uint64_t seed, double repeat_frac, double tandem_frac) {
    uint64_t kb = synth_key(seed, S_BACKGROUND);
    #pragma omp parallel for schedule(static)
    for (int64_t w = 0; w < (int64_t)((n + 31) / 32); w++) {
        uint64_t r = draw(kb, (uint64_t)w);
        uint64_t b0 = (uint64_t)w * 32;
        for (int j = 0; j < 32 && b0 + j < n; j++) out[b0 + j] = ASCII[(r >> (2 * j)) & 3];
    }
    if (repeat_frac > 0 && n > 6000) {
        uint64_t target = (uint64_t)(repeat_frac * (double)n), placed = 0;
        uint64_t kf = synth_key(seed, S_REPEAT_FAMILY), kc = synth_key(seed, S_REPEAT_BASES);
        uint64_t km = synth_key(seed, S_REPEAT_MUT), kp = synth_key(seed, S_REPEAT_POS);
        uint64_t cons_ctr = 0, mut_ctr = 0;
        double lo = log(300.0), hi = log(6000.0);
        uint8_t* cons = (uint8_t*)malloc(6001);
        for (uint64_t fam = 0; placed < target; fam++) {
            uint64_t len = (uint64_t)llround(exp(lo + (hi - lo) * unif(kf, fam * 4)));
            uint64_t copies = 2 + (uint64_t)(unif(kf, fam * 4 + 1) * 49.0);
            double div = 0.10 + 0.10 * unif(kf, fam * 4 + 2);
            uint32_t thr = (uint32_t)(div * 4096.0);
            for (uint64_t j = 0; j < len; j++) cons[j] = stream_base(kc, cons_ctr + j);
            cons_ctr += len;
            for (uint64_t c = 0; c < copies; c++) {
                uint64_t p = draw(kp, fam * 64 + c) % (n - len);
                for (uint64_t j = 0; j < len; j++) {
                    uint64_t lane = mut_ctr + c * len + j;
                    uint16_t v = (uint16_t)(draw(km, lane >> 2) >> (16 * (lane & 3)));
                    uint8_t b = cons[j];
                    if ((uint32_t)(v & 0xFFF) < thr) b = (uint8_t)((b + 1 + ((v >> 12) % 3)) & 3);
                    out[p + j] = ASCII[b];
                }
            }
            mut_ctr += copies * len;
            placed += copies * len;
        }
        free(cons);
    }
    if (tandem_frac > 0 && n > 400) {
        uint64_t target = (uint64_t)(tandem_frac * (double)n), placed = 0;
        uint64_t kt = synth_key(seed, S_TANDEM), ku = synth_key(seed, S_TANDEM_UNIT);
        for (uint64_t r = 0; placed < target; r++) {
            uint64_t period = 1 + (uint64_t)(unif(kt, r * 3) * 6.0);
            uint64_t len = 20 + (uint64_t)(unif(kt, r * 3 + 1) * 181.0);
            uint64_t p = (uint64_t)(unif(kt, r * 3 + 2) * (double)(n - len));
            uint8_t unit[6];
            for (uint64_t j = 0; j < period; j++) unit[j] = ASCII[stream_base(ku, r * 6 + j)];
            for (uint64_t j = 0; j < len; j++) out[p + j] = unit[j % period];
            placed += len;
        }
    }
}

/* Read lengths only (so the caller can size buffers): lens[i] for i < n_reads. */
void synth_read_lengths(uint64_t n_reads, uint64_t seed, const int32_t* lengths, int n_lengths, int32_t* lens) {
    uint64_t kl = synth_key(seed, S_READ_LEN);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n_reads; i++)
        lens[i] = n_lengths == 1 ? lengths[0] : lengths[draw(kl, (uint64_t)i) % (uint64_t)n_lengths];
}

static inline uint8_t comp_ascii(uint8_t c) {
    switch (c) { case 'A': return 'T'; case 'C': return 'G'; case 'G': return 'C'; default: return 'A'; }
}

/* Reads sampled from ref (ASCII, length n).  Read i has length lens[i] (from synth_read_lengths)
 * and is written at seq + offsets[i].  Error model per source base: substitution with
 * probability p_sub, insertion p_indel/2, deletion p_indel/2; when rate_hi > 0 the per-read total
 * rate e ~ U[rate_lo, rate_hi] replaces them (p_sub = e*sub_share, p_indel = e*(1-sub_share)).
 * A fraction random_frac of reads are uniform random (truth_end = -1, truth_edits = -1).
 * Truth: forward-coordinate inclusive end of the planted alignment, its strand, and its edit
 * count (an upper bound on its cost: a leading deletion is counted although it is free).
 * Returns 0, or -1 if some read's source window ran out (more deletions than the slack). */
int synth_reads(const uint8_t* ref, uint64_t n, uint64_t n_reads, uint64_t seed,
                const int32_t* lens, const uint64_t* offsets, int32_t lmax,
                double p_sub, double p_indel, double rate_lo, double rate_hi, double sub_share,
                double random_frac, uint8_t* seq, int64_t* truth_end, uint8_t* truth_strand,
                int32_t* truth_edits) {
    const uint64_t src_len = (uint64_t)lmax + 32;
    if (n <= src_len) return -1;
    uint64_t ks = synth_key(seed, S_READ_START), kd = synth_key(seed, S_READ_STRAND);
    uint64_t ke = synth_key(seed, S_READ_EVENTS), kr = synth_key(seed, S_READ_RANDOM);
    uint64_t kt = synth_key(seed, S_READ_RATE), kk = synth_key(seed, S_READ_KIND);
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 4096) reduction(|:bad)
    for (int64_t ii = 0; ii < (int64_t)n_reads; ii++) {
        uint64_t i = (uint64_t)ii;
        int32_t L = lens[i];
        uint8_t* out = seq + offsets[i];
        int random_read = unif(kk, i) < random_frac;
        if (random_read) {
            for (int32_t j = 0; j < L; j++) out[j] = ASCII[stream_base(kr, i * (uint64_t)lmax + (uint64_t)j)];
            truth_end[i] = -1; truth_strand[i] = 0; truth_edits[i] = -1;
            continue;
        }
        uint64_t start = draw(ks, i) % (n - src_len);
        int strand = (int)(draw(kd, i) & 1);
        double ps = p_sub, pi = p_indel / 2, pd = p_indel / 2;
        if (rate_hi > 0) {
            double e = rate_lo + (rate_hi - rate_lo) * unif(kt, i);
            ps = e * sub_share; pi = e * (1 - sub_share) / 2; pd = pi;
        }
        int32_t o = 0, edits = 0;
        int64_t end = -1;
        for (uint64_t x = 0; x < src_len && o < L; x++) {
            uint64_t r = draw(ke, i * src_len + x);
            double u = (double)(r >> 11) * 0x1.0p-53;
            uint32_t pick = (uint32_t)(r & 0x7FF);
            uint8_t b = ref[start + x];
            if (u < ps) {                      /* substitution */
                uint8_t code = b == 'A' ? 0 : b == 'C' ? 1 : b == 'G' ? 2 : 3;
                out[o++] = ASCII[(code + 1 + pick % 3) & 3];
                edits++; end = (int64_t)(start + x);
            } else if (u < ps + pi) {          /* insertion of a random base before source base x */
                out[o++] = ASCII[(pick >> 2) & 3];
                edits++; end = (int64_t)(start + x) - 1;
                if (o < L) { out[o++] = b; end = (int64_t)(start + x); }
            } else if (u < ps + pi + pd) {     /* deletion of source base x */
                edits++;
            } else {
                out[o++] = b; end = (int64_t)(start + x);
            }
        }
        if (o < L) { bad = 1; continue; }
        if (strand) {
            for (int32_t j = 0; j < L / 2; j++) {
                uint8_t a = out[j], c = out[L - 1 - j];
                out[j] = comp_ascii(c); out[L - 1 - j] = comp_ascii(a);
            }
            if (L & 1) out[L / 2] = comp_ascii(out[L / 2]);
        }
        truth_end[i] = end; truth_strand[i] = (uint8_t)strand; truth_edits[i] = edits;
    }
    return bad ? -1 : 0;
}
