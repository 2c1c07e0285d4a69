/* peanut.h: C ABI of the GB300 (sm_103a) filter-and-verify read-mapping library.
 *
 * The library maps DNA reads to a reference with at most k unit-cost edits, following Köster &
 * Rahmann, "Massively parallel read mapping on GPUs with PEANUT":
 *   - a q-group index (Section "The q-group index", Algorithm 1) is built over a batch of reads
 *     on the device;
 *   - the 2-bit packed reference is streamed past it and q-gram hits are counted per
 *     (read, strand, diagonal) (Section "Filtration", Algorithm 2);
 *   - every candidate region is verified with bit-parallel semiglobal edit distance (Section
 *     "Validation", Myers' algorithm) and reduced to one hit per maximal run of end positions
 *     within k edits, in all-hits or best-stratum mode (Section "Postprocessing").
 *
 * Output definition (exact, no heuristics): for read r of length m with error budget k and
 * strand s (0 = the read, 1 = its reverse complement, both aligned to the FORWARD reference),
 * D[j] = min edit distance between the pattern and any reference substring ending at j.  For
 * every maximal run of consecutive j with D[j] <= k the library reports one hit
 * (r, s, j*, D[j*]), j* = the leftmost position of the run's minimum.  End positions are 0-based
 * and inclusive.  Best-stratum mode keeps, per read, only the hits whose D equals the read's
 * minimum over both strands.  Hits are sorted by (read, strand, end).
 *
 * Conventions for every call:
 *   - Return value: peanut_status; PEANUT_OK = 0.  On failure peanut_last_error() returns a
 *     message (thread-local, valid until the next call on the same thread).  No call aborts.
 *   - "host" pointers are CPU memory, "device" pointers are CUDA device memory of the current
 *     device.  Inputs are caller-owned and only read during the call (device inputs until the
 *     work queued on the given stream completes).  Outputs are library-owned objects released
 *     with peanut_free().
 *   - stream: a cudaStream_t passed as void* (NULL = the legacy default stream).  All device
 *     work of a call is queued on that stream; calls that return host results synchronize it.
 *   - Objects may be used from one host thread at a time.
 *   - Sequences are ASCII 'A','C','G','T' (upper case).  Any other byte (including 'N') makes
 *     the call fail with PEANUT_INVALID_ARG.
 */
#ifndef PEANUT_H
#define PEANUT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PEANUT_OK = 0,
    PEANUT_INVALID_ARG = 1,  /* bad argument, bad base, read too long, threshold below 1 */
    PEANUT_NO_MEMORY = 2,    /* a device or host allocation failed */
    PEANUT_CUDA_ERROR = 3,   /* a CUDA runtime call or kernel failed */
    PEANUT_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    PEANUT_UNSUPPORTED = 5   /* valid but not supported by this build (e.g. q > 16) */
} peanut_status;

typedef struct peanut_ref peanut_ref;     /* resident packed reference (device) */
typedef struct peanut_reads peanut_reads; /* a read batch and its q-group index (device) */

/* Host-side hit list (struct of arrays, n entries each), sorted by (read_id, strand, end_pos). */
typedef struct {
    uint64_t n;
    uint32_t* read_id; /* index of the read within its batch */
    uint8_t* strand;   /* 0 = read, 1 = reverse complement of the read */
    uint64_t* end_pos; /* 0-based inclusive end on the forward reference */
    uint8_t* dist;     /* edit distance, <= the read's k */
} peanut_hits;

/* Device-side hit list: same layout, pointers are device memory owned by the object. */
typedef struct {
    uint64_t n;
    uint32_t* read_id;
    uint8_t* strand;
    uint64_t* end_pos;
    uint8_t* dist;
} peanut_device_hits;

/* Proper pairs of a paired-end batch (peanut_pair_hits), in device memory owned by the object;
 * release with peanut_free. */
typedef struct {
    uint64_t n;
    uint64_t* i1;     /* index in the hit list of the mate-1 hit */
    uint64_t* i2;     /* index in the hit list of the mate-2 hit */
    uint32_t* score;  /* summed identity (m1 - d1) / m1 + (m2 - d2) / m2 as its numerator over m1 m2:
                         (m1 - d1) m2 + (m2 - d2) m1 */
    uint32_t* rank;   /* proper pairs of the fragment scoring at least as high (>= 1) */
    uint8_t* mapq;    /* min(floor(-10 log10((rank - 1) / n) + 1e-9), 255), 255 at rank 1 */
} peanut_device_pairs;

/* Per-batch parameters. */
typedef struct {
    uint32_t q;          /* q-gram length, 1..16 (Section "The q-group index"; the paper uses 16) */
    uint32_t k_fixed;    /* error budget of every read; UINT32_MAX = derive from k_permille */
    uint32_t k_permille; /* k = ceil(length * k_permille / 1000) when k_fixed == UINT32_MAX */
    uint32_t freq_cap;   /* a canonical q-gram occurring more than freq_cap times in the
                            reference is not indexed; reads containing such q-grams are verified
                            around every occurrence cluster instead (exact either way).
                            0 = default: max(256, 8 x the expected count 2 n / 4^q of a
                            canonical q-gram in a uniform reference of n bases) */
    uint32_t stride;     /* index only the q-grams at read offsets 0, stride, 2 stride, ...;
                            the count threshold becomes the number of them an alignment with k
                            edits keeps intact (Section "The q-group index", q-gram lemma, with
                            at most ceil(q / stride) sampled q-grams touched per edit).  Exact
                            for any stride the reads admit; 0 or 1 = every offset, 1..64 */
    void* stream;        /* cudaStream_t for all device work of the batch */
    uint32_t ref_index;  /* 0 = stream the packed reference past the batch's index (Algorithm 2);
                            1 = look the batch's indexed q-grams up in the reference's own q-group
                            index instead (built beforehand with peanut_index_reference at this q).
                            Same hits, same output; a comparison of the two scans */
    uint32_t index_layout; /* storage of the batch index's I and S (Algorithm 1; the output is the
                            same for every layout): 0 = (I, S) interleaved per group of w = 32
                            codes, one 8-byte probe (8 B per 32 codes); 1 = I per 32 codes and S
                            kept for every second group only, an odd group adding the population
                            count of the even one (the sampling of S of Section "The q-group
                            index", 6 B per 32 codes); 2 = w = 64: a 64-bit I word and S per 64
                            codes (6 B per 32 codes) */
} peanut_params;

/* Counters of the last peanut_map() on a batch (diagnostics; all device-computed). */
typedef struct {
    uint64_t hits;             /* q-gram hits emitted by the reference scan */
    uint64_t candidates;       /* candidate end ranges verified */
    uint64_t candidate_columns;/* reference columns run through the bit-vector verification */
    uint64_t results;          /* hits returned */
    uint64_t lowcx_reads;      /* reads verified around frequent q-gram clusters */
    uint64_t lowcx_ranges;     /* cluster and counting ranges of those reads, before merging */
    uint64_t scan_retries;     /* present-position or hit buffer regrowths */
    uint64_t present_probes;   /* reference positions whose canonical q-gram is indexed */
    uint64_t candidate_word_columns; /* columns x 64-bit words of the verification */
    float ms_scan, ms_bin, ms_windows, ms_verify, ms_output; /* device time per stage */
    float ms_scan_kernel;      /* the reference-scan kernels alone (probe and expand; CUDA events on
                                  their stream) */
    float ms_verify_kernel;    /* the verification count pass alone (CUDA events on its stream) */
    float ms_windows_sweep, ms_lowcx, ms_compact; /* parts of ms_windows */
    float ms_probe_kernel;     /* the probe half of the reference scan (present positions) */
    float ms_windows_med, ms_windows_big; /* window paths of reads with many hits (block / global) */
    uint64_t med_reads, big_reads;        /* reads taking those paths */
    uint64_t lowcx_rest_segments; /* (read, strand) segments of low-complexity reads too large for
                                     the block merge (merged by the warp k-way merge) */
    uint64_t lowcx_serial_segments; /* of those, segments with 32 or more cluster lists (merged by
                                       one lane) */
    uint64_t useful_columns;   /* verified columns whose distance is within the read's k (the
                                  columns that lie in reported runs) */
    uint64_t prefilter_columns;/* columns the verification would have run without the q'-gram
                                  filter on candidate ranges */
    uint64_t filter_positions; /* reference positions scanned by that filter */
    uint64_t filter_live;      /* candidate ranges it kept (narrowed); the rest hold no end
                                  within k edits */
    float ms_filter_kernel;    /* the filter kernel (CUDA events on its stream) */
    uint64_t graph_segments;   /* stretches of the call's work launched as CUDA graphs (an engine's
                                  launches: the scan, the binning and short-read windows, the
                                  filter and verification count pass, the write pass) */
} peanut_map_stats;

/* Packs an ASCII reference into 2 bits per base on the device (A=00, C=01, G=10, T=11, first
 * base most significant; Section "The q-group index", encoding paragraph) and keeps it resident.
 * One contig; the same as peanut_pack_reference_contigs with contig_starts = {0}, gap_min =
 * PEANUT_DEFAULT_GAP_MIN and n_seed = 0.
 *   seq: host, len bytes of A/C/G/T/N in either case.  len: 1 .. 2^39.  stream: see conventions.
 *   out: receives the new reference object.
 * Errors: INVALID_ARG (NULL pointer, len out of range, another byte), NO_MEMORY, CUDA_ERROR. */
peanut_status peanut_pack_reference(const char* seq, uint64_t len, void* stream, peanut_ref** out);

#define PEANUT_DEFAULT_GAP_MIN 16u

/* Packs a reference made of one or more contigs (chromosomes) laid end to end.
 * Section "Overview": every step runs per chromosome, so no hit spans two contigs.  Section "The
 * q-group index" (encoding paragraph): an unknown base N becomes a random base, and long runs of
 * N stay out of the index.  Here:
 *   - N at reference position p becomes base (SplitMix64 output number p + 1 of the generator
 *     seeded with n_seed) >> 62 (Steele, Lea & Flood 2014), so packing is reproducible; N in a
 *     read at offset i becomes (output i + 1 of SplitMix64 seeded with n_seed XOR the FNV-1a 64
 *     hash of the read's upper-cased bytes) >> 62, in every batch indexed against this reference;
 *   - a run of at least gap_min Ns inside one contig is a gap.  Contig boundaries and gaps cut the
 *     reference into segments: every alignment lies inside one segment (the semiglobal matrix
 *     restarts at each segment start), so no hit ends in a gap or spans a boundary;
 *   - lower-case a, c, g, t, n are read as their upper-case bases (soft-masked input).
 * Hits keep global coordinates (positions in the concatenated sequence, gaps included); the
 * caller maps them to (contig, offset) with its own contig_starts.
 *   seq: host, len bytes.  len: 1 .. 2^39.
 *   contig_starts: host, n_contigs ascending start positions, the first 0, each < len (contig c
 *     spans [contig_starts[c], contig_starts[c + 1]), the last ends at len); NULL or
 *     n_contigs = 0 means one contig.
 *   gap_min: 1 .. 2^32 - 1 (PEANUT_DEFAULT_GAP_MIN = the paper's q, a run long enough to hold a
 *     whole q-gram of Ns).  n_seed: any value.  stream: see conventions.
 * Errors: INVALID_ARG (NULL pointer, len out of range, a byte other than A/C/G/T/N, a bad contig
 *         list, gap_min = 0), UNSUPPORTED (more than 2^26 runs of N), NO_MEMORY, CUDA_ERROR. */
peanut_status peanut_pack_reference_contigs(const char* seq, uint64_t len, const uint64_t* contig_starts,
                                            uint32_t n_contigs, uint32_t gap_min, uint64_t n_seed, void* stream,
                                            peanut_ref** out);

/* The reference's segments (see peanut_pack_reference_contigs): count, then the [start, end)
 * pairs into caller-owned host arrays of that many entries each (either may be NULL).
 * peanut_ref_segments returns INVALID_ARG for a bad reference or a NULL count. */
peanut_status peanut_ref_segments(const peanut_ref* ref, uint64_t* count, uint64_t* starts, uint64_t* ends);

/* Reference length in bases. */
uint64_t peanut_ref_length(const peanut_ref* ref);

/* Builds the reference's own q-group index (Algorithm 1 run over the reference's canonical
 * q-grams: the reference-side index of Section "Filtration", without repeat masking) and keeps
 * it with the reference; batches indexed with peanut_params.ref_index = 1 at this q then find
 * their hits by looking their q-grams up in it instead of streaming the reference.  Device
 * memory: 4^q / 4 bytes for I and S, at most 8.2 bytes per reference position for S' and the
 * occurrences (26 GB at q = 16 for 3.1 Gbp), and 4 bytes per distinct q-gram more while it is
 * built; building again at the same q is a no-op.
 *   ref: a packed reference of fewer than 2^32 bases; q: 1..16; stream: see conventions
 *   (synchronized).
 * Errors: INVALID_ARG (bad reference), UNSUPPORTED (q outside 1..16, reference of 2^32 bases or
 *         more), NO_MEMORY, CUDA_ERROR. */
peanut_status peanut_index_reference(peanut_ref* ref, uint32_t q, void* stream);

/* Builds the q-group index (I, S, S', O of Algorithm 1, with the canonical q-gram of every read
 * position, Section "The q-group index") over a batch of reads, on the device.
 *   ref: the reference the batch will be mapped against (it must outlive the batch; its
 *        frequent-q-gram table for this q is computed and cached on first use).
 *   seqs: host, the concatenated reads; offsets: host, n_reads + 1 ascending byte offsets
 *        into seqs (read i = seqs[offsets[i] .. offsets[i+1])).
 *   n_reads: 1 .. 2^23.  Every read length must be 1..255 and every read must satisfy the
 *        q-gram lemma threshold t = m + 1 - q(k + 1) >= 1 (Section "The q-group index").
 *   p: parameters (q, k rule, stream).
 *   out: receives the batch object.
 * Errors: INVALID_ARG (argument out of range, non-ACGT byte, length or threshold violation),
 *         UNSUPPORTED (q outside 1..16), NO_MEMORY, CUDA_ERROR. */
peanut_status peanut_index_reads(const peanut_ref* ref, const char* seqs, const uint64_t* offsets,
                                 uint32_t n_reads, const peanut_params* p, peanut_reads** out);

/* Same as peanut_index_reads with the reads already in device memory:
 *   d_seqs: device, total_bases bytes; d_offsets: device, n_reads + 1 uint64 offsets. */
peanut_status peanut_index_reads_device(const peanut_ref* ref, const char* d_seqs,
                                        const uint64_t* d_offsets, uint32_t n_reads,
                                        uint64_t total_bases, const peanut_params* p,
                                        peanut_reads** out);

/* Maps a batch: reference scan and hit counting (Algorithm 2), candidate compaction, bit-vector
 * verification (Section "Validation") and per-read stratum reduction (Section "Postprocessing").
 *   mode: 0 = all hits, 1 = best stratum.
 *   out: receives a host hit list (see peanut_hits), sorted by (read_id, strand, end_pos).
 * Synchronizes the batch's stream.
 * Errors: INVALID_ARG, NO_MEMORY, CUDA_ERROR, TIMEOUT. */
peanut_status peanut_map(const peanut_ref* ref, peanut_reads* reads, int mode, peanut_hits** out);

/* Same as peanut_map with the result left in device memory (peanut_device_hits). */
peanut_status peanut_map_device(const peanut_ref* ref, peanut_reads* reads, int mode,
                                peanut_device_hits** out);

/* Copies a device hit list to a new host hit list. */
peanut_status peanut_download_hits(const peanut_device_hits* dh, void* stream, peanut_hits** out);

/* Counters and stage times of the last map call on this batch. */
peanut_status peanut_get_map_stats(const peanut_reads* reads, peanut_map_stats* out);

/* Frees any object returned by this library (peanut_ref, peanut_reads, peanut_hits,
 * peanut_device_hits, peanut_engine).  NULL is a no-op.  Device memory is released on the
 * object's stream. */
void peanut_free(void* obj);

/* Message describing the last failure on this thread ("" if none). */
const char* peanut_last_error(void);

/* Number of CUDA kernels this library has launched in this process (diagnostics). */
uint64_t peanut_kernel_launches(void);

/* Device memory provider for all later allocations made on the caller's threads (e.g. the
 * caching allocator of the host framework; the Python binding installs PyTorch's when a GPU is
 * present).  alloc(bytes, stream, ctx) returns device memory or NULL; release(ptr, stream, ctx)
 * frees it.  Passing NULL functions restores the default (cudaMallocAsync / cudaFreeAsync on the
 * stream, CUDA's stream-ordered pool).  Not thread-safe with concurrent calls.  An engine's own
 * threads (executors, I/O) always allocate from the stream-ordered pool, so a provider that calls
 * back into an interpreter never serializes them.  An object is released by the provider that
 * allocated it, even after another was installed. */
typedef void* (*peanut_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*peanut_release_fn)(void* ptr, void* stream, void* ctx);
peanut_status peanut_set_allocator(peanut_alloc_fn alloc, peanut_release_fn release, void* ctx);

/* ---- introspection used by the parity tests ---- */

/* Sizes of a batch's q-group index: n_groups = ceil(4^q / 32) (entries of I and S),
 * n_distinct = distinct indexed q-grams (S' has n_distinct + 1 entries, the last = n_indexed),
 * n_indexed = indexed q-gram positions (entries of O). */
peanut_status peanut_index_sizes(const peanut_reads* reads, uint64_t* n_groups, uint64_t* n_distinct,
                                 uint64_t* n_indexed);

/* Copies the index arrays to host buffers sized by peanut_index_sizes (any pointer may be NULL),
 * in the w = 32 form whatever the batch's layout (S of a group not stored is recomputed from I):
 * I[n_groups] (bit j of I[i] = canonical q-gram 32 i + j occurs), S[n_groups] (exclusive
 * cumulative popcount of I), Sp[n_distinct + 1], O[n_indexed] (entries
 * (read << 9) | (orientation << 8) | offset; orientation 1 = the read holds the reverse
 * complement of the canonical q-gram at that offset). */
peanut_status peanut_export_index(const peanut_reads* reads, uint32_t* I, uint32_t* S, uint32_t* Sp,
                                  uint32_t* O);

/* Per-read filter parameters chosen at indexing: thr[i] = q-gram count threshold used for read i,
 * lowcx[i] = 1 if read i is verified around frequent-q-gram clusters (host arrays of n_reads). */
peanut_status peanut_export_read_params(const peanut_reads* reads, uint16_t* thr, uint8_t* lowcx);

/* Candidate end ranges the last map call verified (host arrays of *n entries, or NULL to query
 * n): read, strand, lo, hi (inclusive, clipped to the reference), in (read, strand, lo) order:
 * the compacted windows after the q'-gram filter narrowed them (ranges it removed are left out). */
peanut_status peanut_export_candidates(const peanut_reads* reads, uint64_t* n, uint32_t* read,
                                       uint8_t* strand, uint64_t* lo, uint64_t* hi);

/* Runs the bit-vector verification kernel alone: for pattern i (ASCII, lengths 1..255, host
 * arrays pat / pat_off[n_pat + 1]) against text i (ASCII, host arrays txt / txt_off[n_pat + 1]),
 * writes D[j] (semiglobal distance of the whole pattern ending at text position j, boundary
 * E[i][-1] = i) to out (host, txt_off[n_pat] int32 entries).  Test hook for the kernel that
 * peanut_map uses. */
peanut_status peanut_debug_bitvector_columns(const char* pat, const uint64_t* pat_off, uint32_t n_pat,
                                             const char* txt, const uint64_t* txt_off, int32_t* out,
                                             void* stream);

/* Same computation as peanut_debug_bitvector_columns, for callers that cannot allocate device
 * memory (the paper has no counterpart): a process whose device memory is all reserved by another
 * allocator's pool, where a cudaMalloc fails or takes memory the pool counts on, or a
 * latency-critical path that must not pay an allocation's implicit synchronization.  This call
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *   d_pat / d_pat_off[n_pat + 1]: device, ASCII patterns (lengths 1..255) and their offsets.
 *   d_txt / d_txt_off[n_pat + 1]: device, ASCII texts and their offsets.
 *   d_out: device, txt_off[n_pat] int32 entries, D[j] for every text position (as above).
 *   n_pat: 1 .. 8192 (more is rejected with PEANUT_INVALID_ARG).
 * Scratch: the match masks of up to 8192 patterns and a status word sit in one fixed array of
 * about 1 MiB of device memory inside the library, held by every GPU that loads it until the
 * process exits.  The first call on a device looks up that array's device address (once per
 * device, with the device current); make that first call before any stream capture.  Every call
 * shares the array and leaves its contents behind; calls whose work overlaps on the GPU (other
 * streams, other host threads) race on it and must be serialized by the caller.  The call
 * synchronizes the stream to read the status word.
 * Errors: INVALID_ARG (NULL pointer, n_pat out of range, bad length or offsets, non-ACGT byte),
 *         CUDA_ERROR. */
peanut_status peanut_bitvector_columns_noalloc(const char* d_pat, const uint64_t* d_pat_off, uint32_t n_pat,
                                               const char* d_txt, const uint64_t* d_txt_off, int32_t* d_out,
                                               void* stream);

/* ---- postprocessing ------------------------------------------------------------------------
 *
 * Annotates a batch's hit list (from peanut_map_device on that batch, either mode, or any list of
 * its hits grouped by ascending read) on the device:
 *   start: the alignment start, from the edit distance recomputed backwards from the hit's end
 *          (Section "Validation", last paragraph): the leftmost reference position i such that
 *          the edit distance between the pattern (the read, or its reverse complement for
 *          strand 1) and reference[i .. end] equals the hit's distance;
 *   rank:  the hit-rank of Section "Postprocessing": the number of the read's hits in the list
 *          (both strands) whose distance is at most this hit's (percent identity at least as
 *          high);
 *   mapq:  the mapping quality of Section "Postprocessing", min(-10 log10((rank - 1) / n), 255)
 *          for a reference of n bases; 255 for rank 1; the integer part of the double-precision
 *          value plus 1e-9, clamped to 0..255.
 *   hits: device hit list (peanut_device_hits); d_start / d_rank / d_mapq: caller-owned device
 *   arrays of hits->n entries.  Work runs on the batch's stream; the call synchronizes it.
 * Errors: INVALID_ARG (bad objects, the batch indexed against another reference, a hit naming a
 *         read / strand / end outside the batch or reference, a distance that is not the
 *         pattern's distance at that end, hits not grouped by ascending read), NO_MEMORY,
 *         CUDA_ERROR. */
peanut_status peanut_annotate_hits(const peanut_ref* ref, const peanut_reads* reads, const peanut_device_hits* hits,
                                   uint64_t* d_start, uint32_t* d_rank, uint8_t* d_mapq);

/* ---- measurement ---------------------------------------------------------------------------
 *
 * Integer issue-rate microbenchmark: the measured ceiling against which the bit-vector
 * verification kernel (Section "Validation") is reported.  Runs one kernel of the given kind on
 * 8 x 256-thread blocks per SM of the current device, every thread twelve independent chains of
 * one instruction form (no two foldable, operands in registers, no memory traffic), after one
 * shorter warm-up launch, and times it with CUDA events on `stream` (synchronized).
 *   kind: 0 = 3-input logic (lop3.b32), 1 = funnel shift (shf.l.wrap.b32), 2 = 32-bit add
 *         (add.u32), 3 = integer multiply-add (mad.lo.u32), 4 = population count (popc.b32);
 *         5 / 6 = Myers' column step on 1 / 2 64-bit words with the match masks in shared memory,
 *         one column stream per thread (the verification kernel's recurrence without its
 *         global-memory accesses, run bookkeeping or lane divergence);
 *         7 / 8 = random 8-byte loads (eight in flight per thread) from an 8 MiB table (held in
 *         L2) / a 2 GiB table (HBM): the access pattern of the reference scan's filter and index
 *         probes (Section "Filtration").
 *   iters: loop trips per thread (48 instructions, 16 columns, or 8 loads per trip).
 *   ms: kernel time; ops: instructions executed (kinds 0-4), 64-bit word-columns (5, 6) or loads
 *   (7, 8), over all threads; grid / block: the launch shape.
 * Errors: INVALID_ARG (NULL pointer, iters = 0, unknown kind), NO_MEMORY, CUDA_ERROR. */
/* The actual alignment of every hit (Section "Postprocessing": the postprocessing calculates the
 * actual alignment of each hit).  The pattern (the read, or its reverse complement for strand 1)
 * is aligned with the reference bases start .. end of the hit, both ends fixed, at the hit's
 * distance; among the optimal alignments the one traced back from the last cell preferring the
 * diagonal step, then a reference-only step, then a read-only step.  Output per hit: up to
 * ops_per_hit runs of equal operations in forward order, each encoded as length << 2 | code
 * (0 '=' match, 1 'X' mismatch, 2 'I' read base only, 3 'D' reference base only: an extended
 * CIGAR), and their number.  A hit of distance d has at most 2 d + 1 runs, so
 * ops_per_hit = 2 k + 1 for the batch's largest k always suffices.
 *   hits: a device hit list of this batch; d_start: device, hits->n alignment starts
 *   (peanut_annotate_hits).  d_ops: device, hits->n * ops_per_hit words, caller-owned;
 *   d_nops: device, hits->n entries.  Uses the batch's stream (synchronized); allocates transient
 *   device memory: the hits' indices listed by distance (4 bytes per hit), nine 32-bit counts
 *   per classifying block, one 16-bit word of traceback directions per read base (plus one) and
 *   thread of the widest launch, and, when a hit has distance 8 or more, a band of
 *   (2 k + 1)(m + 1) 16-bit cells per thread for those.  A hit whose distance exceeds the
 *   batch's largest k is refused (INVALID_ARG).
 * Errors: INVALID_ARG (bad object, NULL pointer, a hit outside the batch or reference, a start
 *         after its end, a distance that is not the pattern's distance to those bases, more runs
 *         than ops_per_hit), NO_MEMORY, CUDA_ERROR. */
/* The largest error budget k among the batch's reads (0 for a bad batch). */
uint32_t peanut_batch_max_k(const peanut_reads* batch);

peanut_status peanut_hit_alignments(const peanut_ref* ref, const peanut_reads* batch, const peanut_device_hits* hits,
                                    const uint64_t* d_start, uint32_t ops_per_hit, uint32_t* d_ops, uint16_t* d_nops);

/* Pairs the mates of a paired-end batch (Section "Postprocessing": mates are paired, and in
 * paired-end mode the percent identities of properly paired hits are summed to form strata).
 * Reads 2p and 2p + 1 of the batch are the two mates of fragment p, read from its two ends
 * (forward-reverse).  Hit u of mate 1 and hit x of mate 2 are a proper pair when they lie on
 * opposite strands, in the same contig, and the fragment from the strand-0 hit's start to the
 * strand-1 hit's end is min_insert .. max_insert bases long.  Pairs are listed in (mate-1 hit,
 * mate-2 hit) order with their score, rank and quality (peanut_device_pairs); mode 1 keeps each
 * fragment's best-scoring pairs (the paired best stratum), mode 0 all of them.
 *   hits: a device hit list of this batch in the order peanut_map_device gives (grouped by read,
 *     each read's hits by strand, then end); d_start: device, hits->n alignment starts
 *     (peanut_annotate_hits).  The batch's stream is used and synchronized.
 *   out: receives a new pairs object.
 * Errors: INVALID_ARG (bad object, NULL pointer, odd number of reads, min_insert = 0 or
 *         max_insert < min_insert, hits out of order, a start after its end), NO_MEMORY,
 *         CUDA_ERROR. */
peanut_status peanut_pair_hits(const peanut_ref* ref, const peanut_reads* batch, const peanut_device_hits* hits,
                               const uint64_t* d_start, uint32_t min_insert, uint32_t max_insert, int mode,
                               peanut_device_pairs** out);

/* Copies a pairs object to caller-owned host arrays of pairs->n entries each (any may be NULL).
 * Synchronizes stream.  Errors: INVALID_ARG (bad object), CUDA_ERROR. */
peanut_status peanut_download_pairs(const peanut_device_pairs* pairs, void* stream, uint64_t* i1, uint64_t* i2,
                                    uint32_t* score, uint32_t* rank, uint8_t* mapq);

peanut_status peanut_int_peak(uint32_t kind, uint32_t iters, void* stream, double* ms, uint64_t* ops,
                              uint32_t* grid, uint32_t* block);

/* ---- batched and served mapping ------------------------------------------------------------
 *
 * An engine maps many read sets ("submissions") against one resident reference.  The paper
 * fixes one q and one batch per kernel sequence, with reads strided by a common length; the
 * engine runs the same per-batch path (index, scan, windows, verification, strata) over
 * launches it forms itself:
 *   - every read belongs to the class of the largest q its length and budget admit (the q-gram
 *     lemma threshold m + 1 - q(k + 1) >= 1, Section "The q-group index"), so reads of uneven
 *     length share launches only with reads that admit the same q;
 *   - reads of a class are coalesced across submissions, in submission order, into launches of
 *     up to max_reads reads, sized so that the engine's device memory stays within its budget;
 *   - up to `executors` launches are in flight at once, each on its own CUDA stream and host
 *     thread, so one launch's memory-bound reference scan overlaps another's ALU-bound
 *     verification; a submission is admitted (its reads copied to the device) when its
 *     footprint fits next to the work in flight ("admission by free HBM");
 *   - with autotune, the first launch of each class is mapped once per candidate setting
 *     (its q with sampling strides 1, 2, 3, 4, 6, 8, 12, 16 up to q, and q - 1 with strides 1..4,
 *     as far as every length of the class admits them) and the setting with the lowest predicted
 *     time per read at full launch size is used from then on;
 *   - each submission's hits are renumbered to its own read ids and sorted on the device,
 *     reduced to the best stratum if asked, and returned in one host hit list.
 * A read's hits depend only on the read, its budget and the reference, so a submission's
 * result is the same whether it is mapped alone, with peanut_map, or in any mix. */
typedef struct peanut_engine peanut_engine;

typedef struct {
    uint32_t k_fixed;     /* error budget of every read; UINT32_MAX = derive from k_permille */
    uint32_t k_permille;  /* k = ceil(length * k_permille / 1000) when k_fixed == UINT32_MAX */
    uint32_t executors;   /* launches in flight at once, 1..4 (0 = 2) */
    uint32_t max_reads;   /* reads per launch at most, 1 .. 2^23 (0 = 2^22) */
    uint32_t autotune;    /* 1 = pick (q, stride) per class by timing its first launch */
    uint32_t fixed_q;     /* 0 = per class; else every read is mapped with this q (1..16) */
    uint64_t hbm_budget;  /* device bytes the engine may hold (0 = 90 % of the free memory at
                             creation, less 4 GiB; give explicit budgets when several engines
                             share a device) */
    uint32_t graphs;      /* 1 = each launch runs its sync-free stretches (the scan; binning and
                             the windows of reads with few hits; the candidate filter and the
                             verification count pass; the write pass) as CUDA graphs, one readback
                             between stretches.  While such an engine has work in flight the
                             process must not synchronize the whole device (cudaDeviceSynchronize,
                             torch.cuda.synchronize()): a stream being captured makes that call
                             fail.  Synchronize streams or events instead.  0 = plain launches */
} peanut_engine_params;

/* Per-class record of an engine (peanut_engine_get_stats). */
typedef struct {
    uint32_t q_class;     /* the largest q the class's reads admit */
    uint32_t q, stride;   /* the setting in use */
    uint32_t freq_cap;
    uint64_t launches, reads;
    uint64_t bytes_per_read; /* measured device footprint per read of a launch */
    float tuned_ms_per_mread; /* autotune: predicted ms per 10^6 reads at full launch size */
    uint32_t tune_candidates; /* settings timed by the autotuner */
} peanut_engine_class;

typedef struct {
    uint64_t submissions, completed, reads, launches, tuning_launches;
    uint64_t hbm_budget, hbm_reserved_peak;
    uint32_t n_classes;
    peanut_engine_class cls[16];
    /* totals over every mapping run (tuning runs included), as in peanut_map_stats */
    uint64_t map_runs, hits, candidates, candidate_word_columns, present_probes, results;
    uint64_t bases_scanned;   /* reference bases streamed by the scans */
    double ms_verify_kernel, ms_scan_kernel, ms_probe_kernel; /* CUDA-event sums per kernel */
    /* wall time (ms): the I/O thread admitting submissions (copy in, classify) and copying
       results to the host; the executors (summed) running launches (gather, index, map) and
       assembling results (renumber, sort, strata) */
    double ms_admit, ms_launch, ms_assemble, ms_download;
    uint64_t pageable_result_blocks; /* host result blocks (process-wide) that could not be
                                        page-locked and fell back to pageable memory */
    uint64_t candidate_columns;       /* columns run through the bit-vector verification */
    uint64_t useful_columns;          /* of those, columns whose distance is within k */
    uint64_t filter_positions;        /* reference positions scanned by the q'-gram filter */
    double ms_filter_kernel;          /* CUDA-event sum of the q'-gram filter kernel */
    uint64_t graph_segments;          /* stretches of the launches' work run as CUDA graphs */
} peanut_engine_stats;

/* Mode flag of engine submissions: keep the result in device memory (take it with
 * peanut_engine_wait_device; peanut_engine_wait copies it to the host instead). */
#define PEANUT_RESULT_ON_DEVICE 0x100

/* Creates an engine over a resident reference (which must outlive it) and starts its executor
 * threads and its I/O thread (every host<->device copy: admissions and results).  Errors: INVALID_ARG (bad reference or parameters), NO_MEMORY, CUDA_ERROR. */
peanut_status peanut_engine_create(const peanut_ref* ref, const peanut_engine_params* p, peanut_engine** out);

/* Queues a submission of host reads (layout as in peanut_index_reads; n_reads 1 .. 2^24) in
 * mode 0 (all hits) or 1 (best stratum), optionally | PEANUT_RESULT_ON_DEVICE, and returns its
 * ticket at once.  seqs and offsets are
 * read when the submission is admitted: they must stay valid and unchanged until
 * peanut_engine_wait has returned its result.  Lengths, bases and thresholds are checked at
 * admission; a bad submission fails alone (its wait returns the error).
 * Errors: INVALID_ARG (bad engine, NULL pointer, n_reads or mode out of range). */
peanut_status peanut_engine_submit(peanut_engine* e, const char* seqs, const uint64_t* offsets,
                                   uint32_t n_reads, int mode, uint64_t* ticket);

/* As peanut_engine_submit with the reads already in device memory (d_offsets: n_reads + 1
 * uint64 offsets into d_seqs, total_bases bytes).  The caller's writes to them must be complete
 * (stream synchronized) before the call, and the buffers stay valid until the wait returns. */
peanut_status peanut_engine_submit_device(peanut_engine* e, const char* d_seqs, const uint64_t* d_offsets,
                                          uint32_t n_reads, uint64_t total_bases, int mode, uint64_t* ticket);

/* Waits up to timeout_ms (negative = without limit) for a submission.  On success *out is its
 * host hit list (read ids are the submission's own, sorted by (read, strand, end)), released
 * with peanut_free, and the ticket is consumed.  Returns TIMEOUT (ticket kept, *out NULL) if the
 * submission is still running, or the submission's own error (ticket consumed).
 * Errors: INVALID_ARG (bad engine or unknown ticket), TIMEOUT, and any error of the mapping. */
peanut_status peanut_engine_wait(peanut_engine* e, uint64_t ticket, int64_t timeout_ms, peanut_hits** out);

/* As peanut_engine_wait for a submission made with PEANUT_RESULT_ON_DEVICE: *out is its hit list
 * in device memory (read ids are the submission's own, sorted by (read, strand, end)), released
 * with peanut_free; it stays valid after the engine is released.
 * Errors: INVALID_ARG (bad engine, unknown ticket, or a submission without the flag), TIMEOUT,
 * and any error of the mapping. */
peanut_status peanut_engine_wait_device(peanut_engine* e, uint64_t ticket, int64_t timeout_ms,
                                        peanut_device_hits** out);

/* Counters and per-class settings of an engine. */
peanut_status peanut_engine_get_stats(peanut_engine* e, peanut_engine_stats* out);

/* An engine is released with peanut_free (from a thread not waiting on it): the launches in
 * flight complete, submissions not yet returned by peanut_engine_wait are discarded, and its
 * threads and streams end. */

#ifdef __cplusplus
}
#endif

#endif /* PEANUT_H */
