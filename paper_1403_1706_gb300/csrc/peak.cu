// Microbenchmarks for the rooflines: the integer issue rate (the ceiling of the bit-vector
// verification kernel) and the random-probe rate of L2 and HBM (the ceiling of the reference scan).
//
// The verification kernel (Section "Validation", Myers' bit-parallel recurrence) is bound by the
// integer ALU: 32-bit logic (LOP3), funnel shifts (SHF) and carried adds.  These kernels measure,
// on the device they run on, how many such instructions the SMs retire per second when nothing
// else limits them: every thread runs twelve independent chains (no dependent-issue stalls), each
// instruction takes three values produced by other chains (no two can be folded into one), all
// operands live in registers, no memory traffic, all 32 lanes active, full occupancy.  The Myers
// kernels run the verification's own column step (match masks in shared memory, one column
// stream per thread, as in the verification kernel), so their rate is the ceiling for that
// exact instruction mix.
#include "internal.cuh"

namespace pn {

constexpr int kPeakChains = 12;

template <int KIND>
__device__ __forceinline__ void peak_op(uint32_t (&r)[kPeakChains], int u) {
    uint32_t& d = r[u];
    const uint32_t a = r[(u + 1) % kPeakChains], b = r[(u + 5) % kPeakChains];
    if constexpr (KIND == 0) {  // 3-input logic
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(d) : "r"(a), "r"(b));
    } else if constexpr (KIND == 1) {  // funnel shift by a register amount
        asm volatile("shf.l.wrap.b32 %0, %1, %0, %2;" : "+r"(d) : "r"(a), "r"(b));
    } else if constexpr (KIND == 2) {  // 32-bit add
        asm volatile("add.u32 %0, %0, %1;" : "+r"(d) : "r"(a));
    } else if constexpr (KIND == 3) {  // integer multiply-add
        asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(d) : "r"(a), "r"(b));
    } else {  // population count
        asm volatile("popc.b32 %0, %1;" : "=r"(d) : "r"(a));
    }
}

template <int KIND>
__global__ void __launch_bounds__(256) int_peak_k(uint32_t seed, uint32_t iters, uint32_t* sink) {
    uint32_t r[kPeakChains];
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
    for (int u = 0; u < kPeakChains; ++u) r[u] = seed ^ (tid * 0x9E3779B9u + (uint32_t)u * 0x85EBCA6Bu);
#pragma unroll 1
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int rep = 0; rep < 4; ++rep)
#pragma unroll
            for (int u = 0; u < kPeakChains; ++u) peak_op<KIND>(r, u);
    }
    uint32_t x = 0;
#pragma unroll
    for (int u = 0; u < kPeakChains; ++u) x ^= r[u];
    if (x == seed) sink[tid & 1023] = x;  // keeps the chains live; practically never taken
}

// Myers' column step on W 64-bit words with the match masks in registers: the verification
// kernel's recurrence (Pv, Mv, carried add, shifted horizontal deltas, score) without its
// global-memory accesses, run bookkeeping or lane divergence.
template <int W>
__device__ __forceinline__ int myers_step_reg(uint64_t (&Pv)[W], uint64_t (&Mv)[W], const uint64_t (&e)[W],
                                              int lastbit) {
    uint64_t t[W], sum[W];
#pragma unroll
    for (int w = 0; w < W; ++w) t[w] = e[w] & Pv[w];
    if constexpr (W == 1) {
        sum[0] = t[0] + Pv[0];
    } else {
        asm("add.cc.u64 %0, %2, %4;\n\taddc.u64 %1, %3, %5;"
            : "=l"(sum[0]), "=l"(sum[1]) : "l"(t[0]), "l"(t[1]), "l"(Pv[0]), "l"(Pv[1]));
    }
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
__global__ void __launch_bounds__(256) myers_peak_k(uint32_t seed, uint32_t iters, uint32_t* sink) {
    // match masks in shared memory, one slot per thread, as the verification kernel keeps them
    __shared__ uint64_t s_eq[4 * W * 256];
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t* seq = s_eq + threadIdx.x;
    uint64_t h = 0x9E3779B97F4A7C15ull * (tid + 1) ^ seed;
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int w = 0; w < W; ++w) {
            h ^= h >> 29;
            h *= 0xBF58476D1CE4E5B9ull;
            seq[(c * W + w) * 256] = h;
        }
    uint64_t Pv[W], Mv[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        Pv[w] = ~0ull;
        Mv[w] = 0;
    }
    int score = 0;
    uint32_t t = (uint32_t)h;
    const int lastbit = 35;
#pragma unroll 1
    for (uint32_t it = 0; it < iters; ++it) {
        uint32_t a = t;
#pragma unroll
        for (int u = 0; u < 16; ++u) {  // one packed word of 16 text bases
            const uint32_t c = a >> 30;
            a <<= 2;
            uint64_t e[W];
#pragma unroll
            for (int w = 0; w < W; ++w) e[w] = seq[(c * W + w) * 256];
            score += myers_step_reg<W>(Pv, Mv, e, lastbit);
        }
        t = t * 1664525u + 1013904223u;  // the next text word
    }
    uint64_t x = (uint64_t)score;
#pragma unroll
    for (int w = 0; w < W; ++w) x ^= Pv[w] ^ Mv[w];
    if ((uint32_t)x == seed) sink[tid & 1023] = (uint32_t)x;
}

// Random 8-byte loads from a table of mask + 1 words (eight independent loads in flight per
// thread, addresses from a counter-based hash): the access pattern of the reference scan's filter
// and index probes.  The table's size decides whether they hit in L2 or go to HBM.
__global__ void __launch_bounds__(256) probe_peak_k(const uint64_t* __restrict__ tab, uint64_t mask, uint32_t iters,
                                                    uint32_t* sink) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t acc = 0;
    uint64_t h = 0x9E3779B97F4A7C15ull * (tid + 1);
#pragma unroll 1
    for (uint32_t it = 0; it < iters; ++it) {
        uint64_t v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            h ^= h >> 31;
            h *= 0xBF58476D1CE4E5B9ull;
            v[u] = __ldcg(tab + ((h >> 11) & mask));
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += v[u];
    }
    if ((uint32_t)acc == 0x12345u) sink[tid & 1023] = (uint32_t)acc;
}

void int_peak(uint32_t kind, uint32_t iters, cudaStream_t s, double* ms, uint64_t* ops, uint32_t* grid,
              uint32_t* block) {
    const unsigned threads = 256;
    unsigned per_sm = 8;  // 2,048 threads per SM
    const unsigned g = (unsigned)sm_count() * per_sm;
    DBuf<uint32_t> sink(1024, s);
    // probe tables: 8 MiB (resident in the 129 MB L2) or 2 GiB (HBM)
    const uint64_t words = kind == 7 ? (1ull << 20) : kind == 8 ? (1ull << 28) : 0;
    DBuf<uint64_t> tab(words, s);
    if (words) PN_CUDA(cudaMemsetAsync(tab.p, 1, words * 8, s));
    auto launch = [&](uint32_t n_it) {
        switch (kind) {
            case 0: int_peak_k<0><<<g, threads, 0, s>>>(0x1234567u, n_it, sink.p); break;
            case 1: int_peak_k<1><<<g, threads, 0, s>>>(0x1234567u, n_it, sink.p); break;
            case 2: int_peak_k<2><<<g, threads, 0, s>>>(0x1234567u, n_it, sink.p); break;
            case 3: int_peak_k<3><<<g, threads, 0, s>>>(0x1234567u, n_it, sink.p); break;
            case 4: int_peak_k<4><<<g, threads, 0, s>>>(0x1234567u, n_it, sink.p); break;
            case 5: myers_peak_k<1><<<g, threads, 0, s>>>(0x1234567u, n_it, sink.p); break;
            case 6: myers_peak_k<2><<<g, threads, 0, s>>>(0x1234567u, n_it, sink.p); break;
            case 7:
            case 8: probe_peak_k<<<g, threads, 0, s>>>(tab.p, words - 1, n_it, sink.p); break;
            default: PN_REQUIRE(false, PEANUT_INVALID_ARG, "unknown microbenchmark kind %u", kind);
        }
        PN_CHECK_LAUNCH();
    };
    launch(iters / 16 + 1);  // warm-up (clocks, instruction cache)
    cudaEvent_t e0, e1;
    PN_CUDA(cudaEventCreate(&e0));
    PN_CUDA(cudaEventCreate(&e1));
    PN_CUDA(cudaEventRecord(e0, s));
    launch(iters);
    PN_CUDA(cudaEventRecord(e1, s));
    PN_CUDA(cudaEventSynchronize(e1));
    float t = 0;
    PN_CUDA(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const uint64_t nthreads = (uint64_t)g * threads;
    // instructions (kinds 0-4), word-columns (Myers kinds: 16 columns x W words) or loads (probes)
    const uint64_t per_it = kind <= 4 ? 4ull * kPeakChains : kind <= 6 ? 16ull * (kind == 5 ? 1 : 2) : 8ull;
    *ms = t;
    *ops = nthreads * (uint64_t)iters * per_it;
    *grid = g;
    *block = threads;
}

}  // namespace pn
