// percolation.cu -- the site-percolation model of Sec. 2.3 on the GPU: the
// porosity field, the invasion cluster grown by synchronous passes, and its
// spanning (C ABI of include/percolation.h).
//
// Layout: bit-packed rows.  A medium has rows = L^(dims-1) rows (r = y + L z)
// of nq = ceil(L/32) uint32 words; bit b of word (r, q) is site x = 32 q + b
// (canonical i = x + L r), valid for x < L; padding bits are 0 in every
// bitmap.  Four bitmaps: pores, cluster, and two growth fronts (the sites
// that joined in the last pass, and the next pass's).
//
// A growth pass over a word: the neighbours of the last front are the front
// shifted by one bit either way (with the carry bit from the neighbouring
// word of the row), and the same word of the rows above and below (and of
// the neighbouring planes); the pass adds pore & ~cluster & that.  Only
// sites next to the last front can join (every other cluster site's pore
// neighbours joined already), so this is the synchronous pass of the paper's
// spreading, and the count of passes that add sites is exact.
//
// Draws: site i is a pore iff word (i & 3) of Philox4x32-10(seed; i >> 2, 0,
// 0, 3) is <= floor(P 2^32) (capped at 2^32 - 1).
//
// A single medium's passes touch only a band of rows: each pass records the
// lowest and highest row of the front it writes (Band), and the next pass
// visits the rows next to that front plus the rows of the front before it
// (which it must clear from the buffer it overwrites).  Two ways to run the
// passes, with the same results (the graph is the default: measured faster):
//   - one cooperative persistent launch: every CTA resident, the passes
//     separated by a grid barrier (an arrival counter and a generation word;
//     every wait on it bounded by %globaltimer, a CTA that gives up raises
//     the error flag and leaves, and the others then give up at their next
//     wait), the stop decided on the device from the pass's added count;
//   - a replayed CUDA graph of kPassesPerGraph chained launches (each pass
//     is placed on the SMs while the previous one drains, and waits for it
//     before touching memory); after each replay the host reads the per-pass
//     counts and stops at the first pass that added nothing (the rest of that
//     replay are no-ops on an empty front).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "engine_internal.h"
#include "ising_device.cuh"
#include "percolation.h"

namespace ising {

namespace {

constexpr uint32_t kTagPore = 3u;

struct PercGeom {
    uint32_t L, rows, nq;
    int dims;
};

// The pore bits of the nb <= 32 sites starting at canonical index i0.
__device__ __forceinline__ uint32_t pore_word(uint64_t i0, uint32_t nb, uint32_t key0,
                                              uint32_t key1, uint32_t thr) {
    uint32_t w = 0u;
    const uint32_t g0 = (uint32_t)(i0 >> 2);
    const int m = (int)(i0 & 3u);
    if (m == 0) {  // the bits are whole Philox groups: eight at most, four at a time
        const uint32_t groups = (nb + 3u) >> 2;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            Philox4 u[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t gi = 4u * half + k;
                u[k] = gi < groups ? philox4x32_10(g0 + gi, 0u, 0u, kTagPore, key0, key1)
                                   : Philox4{0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu};
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t v[4] = {u[k].w0, u[k].w1, u[k].w2, u[k].w3};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t b = 16u * half + 4u * k + j;
                    w |= (v[j] <= thr && b < nb ? 1u : 0u) << b;
                }
            }
        }
        return w;
    }
#pragma unroll 1
    for (int g = 0; g < 9; ++g) {  // a row that starts inside a group spans nine
        const int lo = 4 * g - m;
        if (lo >= (int)nb) break;
        const Philox4 u = philox4x32_10(g0 + (uint32_t)g, 0u, 0u, kTagPore, key0, key1);
        const uint32_t v[4] = {u.w0, u.w1, u.w2, u.w3};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int b = lo + j;
            if (b >= 0 && b < (int)nb && v[j] <= thr) w |= 1u << b;
        }
    }
    return w;
}

__device__ __forceinline__ uint32_t valid_bits(uint32_t L, uint32_t q) {
    const uint32_t nb = L - 32u * q < 32u ? L - 32u * q : 32u;
    return nb;
}

__device__ __forceinline__ bool in_first_face(const PercGeom& g, uint32_t r) {
    return g.dims == 2 ? r == 0u : r < g.L;
}
__device__ __forceinline__ bool in_last_face(const PercGeom& g, uint32_t r) {
    return g.dims == 2 ? r == g.L - 1u : r >= g.rows - g.L;
}

// The sites one growth pass adds to word w (front fo of the last pass).
__device__ __forceinline__ uint32_t grow_word(const uint32_t* pore, const uint32_t* C,
                                              const uint32_t* F, const PercGeom& g, uint32_t w) {
    const uint32_t r = w / g.nq, q = w - r * g.nq;
    const uint32_t fo = F[w];
    const uint32_t left = q > 0u ? F[w - 1u] : 0u;
    const uint32_t right = q + 1u < g.nq ? F[w + 1u] : 0u;
    uint32_t nb = (fo << 1) | (left >> 31) | (fo >> 1) | (right << 31);
    uint32_t y = r, z = 0u;
    if (g.dims == 3) {
        z = r / g.L;
        y = r - z * g.L;
    }
    if (y > 0u) nb |= F[w - g.nq];
    if (y + 1u < g.L) nb |= F[w + g.nq];
    if (g.dims == 3) {
        if (z > 0u) nb |= F[w - g.L * g.nq];
        if (z + 1u < g.L) nb |= F[w + g.L * g.nq];
    }
    return pore[w] & ~C[w] & nb;
}

__device__ __forceinline__ void block_sum_u64(unsigned long long v, unsigned long long* out) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __shared__ unsigned long long red[32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        unsigned long long s = lane < nw ? red[lane] : 0ull;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0 && s) atomicAdd(out, s);
    }
}

__global__ void perc_pores_kernel(uint32_t* pore, PercGeom g, uint32_t key0, uint32_t key1,
                                  uint32_t thr) {
    const uint64_t words = (uint64_t)g.rows * g.nq;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += stride) {
        const uint32_t r = (uint32_t)(w / g.nq), q = (uint32_t)(w - (uint64_t)r * g.nq);
        const uint64_t i0 = (uint64_t)g.L * r + 32u * q;
        pore[w] = pore_word(i0, valid_bits(g.L, q), key0, key1, thr);
    }
}

struct Band {
    unsigned int lo, hi;  // rows of a front (lo > hi: empty)
};
constexpr int kBandSlots = 4;  // pass k writes slot k % 4, reads k-1 and k-2, resets k+1
constexpr int kPassesPerGraph = 64;
constexpr size_t kCoopBytes = 128;  // 4 counters, barrier, steps, error flag

__device__ __forceinline__ void band_add(Band* b, unsigned int lo, unsigned int hi) {
    // block-wide min / max of the rows that got front bits, then one atomic each
    __shared__ unsigned int s_lo, s_hi;
    if (threadIdx.x == 0) {
        s_lo = 0xFFFFFFFFu;
        s_hi = 0u;
    }
    __syncthreads();
    if (lo <= hi) {
        atomicMin(&s_lo, lo);
        atomicMax(&s_hi, hi);
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_lo <= s_hi) {
        atomicMin(&b->lo, s_lo);
        atomicMax(&b->hi, s_hi);
    }
}

// Cluster and front start as the invasion sites; the other front buffer is
// cleared.
__global__ void perc_seed_kernel(const uint32_t* pore, uint32_t* C, uint32_t* F, uint32_t* F1,
                                 PercGeom g, int source, uint64_t site, Band* bands) {
    const uint64_t words = (uint64_t)g.rows * g.nq;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t site_r = site / g.L, site_x = site - site_r * g.L;
    const uint64_t site_w = site_r * g.nq + (site_x >> 5);
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += stride) {
        const uint32_t r = (uint32_t)(w / g.nq);
        uint32_t v;
        if (source == PERC_FACE)
            v = in_first_face(g, r) ? pore[w] : 0u;
        else
            v = w == site_w ? pore[w] & (1u << (site_x & 31u)) : 0u;
        C[w] = v;
        F[w] = v;
        F1[w] = 0u;
    }
    if (blockIdx.x == 0 && threadIdx.x < kBandSlots) {
        // the seed front is "pass -1" (slot 3): every row that may hold a seed;
        // "pass -2" (slot 2) is empty; slots 0 and 1 are reset for passes 0, 1
        Band b;
        if (source == PERC_FACE) {
            b.lo = 0u;
            b.hi = g.dims == 2 ? 0u : g.L - 1u;
        } else {
            b.lo = b.hi = (unsigned int)(site / g.L);
        }
        bands[threadIdx.x] = threadIdx.x == 3 ? b : Band{0xFFFFFFFFu, 0u};
    }
}

// The rows the banded pass k visits (empty when lo > hi).
__device__ __forceinline__ void pass_rows(const Band* bands, int k, const PercGeom& g,
                                          unsigned int& lo, unsigned int& hi) {
    const Band last = bands[(k + 3) % kBandSlots];   // rows of the front Fo
    const Band older = bands[(k + 2) % kBandSlots];  // rows of the stale front in Fn
    const unsigned int reach = g.dims == 2 ? 1u : g.L;  // rows a front row touches
    lo = 0xFFFFFFFFu;
    hi = 0u;
    if (last.lo <= last.hi) {
        lo = last.lo > reach ? last.lo - reach : 0u;
        hi = last.hi + reach < g.rows ? last.hi + reach : g.rows - 1u;
    }
    if (older.lo <= older.hi) {
        lo = older.lo < lo ? older.lo : lo;
        hi = older.hi > hi ? older.hi : hi;
    }
}

// One banded growth pass (pass index k within the graph, k % 4 picks slots).
__global__ void __launch_bounds__(256) perc_band_kernel(const uint32_t* pore, uint32_t* C,
                                                        const uint32_t* Fo, uint32_t* Fn,
                                                        PercGeom g, Band* bands, int k,
                                                        unsigned long long* added) {
    grid_dependency_wait();  // the previous pass has completed (chained launches)
    launch_dependents();
    if (blockIdx.x == 0 && threadIdx.x == 0) bands[(k + 1) % kBandSlots] = Band{0xFFFFFFFFu, 0u};
    unsigned int lo, hi;
    pass_rows(bands, k, g, lo, hi);
    const uint32_t w0 = lo <= hi ? lo * g.nq : 0u, w1 = lo <= hi ? (hi + 1u) * g.nq : 0u;
    // the grid covers the whole medium; CTAs past the band leave at once
    // (a whole CTA at a time, before any barrier)
    if (w0 + blockIdx.x * blockDim.x >= w1) return;
    unsigned long long cnt = 0ull;
    unsigned int got_lo = 0xFFFFFFFFu, got_hi = 0u;
    {
        const uint32_t stride = gridDim.x * blockDim.x;
        for (uint32_t w = w0 + blockIdx.x * blockDim.x + threadIdx.x; w < w1; w += stride) {
            const uint32_t add = grow_word(pore, C, Fo, g, w);
            Fn[w] = add;
            if (add) {
                C[w] |= add;
                cnt += (unsigned long long)__popc(add);
                const unsigned int r = w / g.nq;
                got_lo = r < got_lo ? r : got_lo;
                got_hi = r > got_hi ? r : got_hi;
            }
        }
    }
    if (!__syncthreads_or(cnt != 0ull)) return;  // nothing joined in this CTA's words
    band_add(&bands[k % kBandSlots], got_lo, got_hi);
    block_sum_u64(cnt, added);
}

struct GridBar {
    unsigned int count;  // CTAs arrived at the current barrier
    unsigned int gen;    // barriers completed
};
constexpr uint64_t kBarrierLimitNs = 1000000000ull;  // give up a barrier wait after ~1 s

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch; false if this CTA's wait ran out.
__device__ __forceinline__ bool grid_barrier(GridBar* gb, unsigned int nblocks) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int* vgen = &gb->gen;
        const unsigned int g0 = *vgen;  // read before arriving: the release comes after
        __threadfence();
        if (atomicAdd(&gb->count, 1u) == nblocks - 1u) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicAdd(&gb->gen, 1u);
        } else {
            const uint64_t t0 = now_ns();
            while (*vgen == g0) {
                if (now_ns() - t0 > kBarrierLimitNs) {
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// All growth passes in one cooperative launch (see the header comment).
// cnt: four per-pass added counters (zero at launch); out_steps: passes that
// added sites; err: raised when a barrier wait ran out.
__global__ void __launch_bounds__(256) perc_persistent_kernel(const uint32_t* pore, uint32_t* C,
                                                              uint32_t* F0, uint32_t* F1,
                                                              PercGeom g, Band* bands,
                                                              unsigned long long* cnt,
                                                              GridBar* gb,
                                                              unsigned long long* out_steps,
                                                              int* err, int drop_last_block) {
    // test hook: the last CTA leaves before the first barrier, so every other
    // CTA's wait there runs out (nothing else ever makes a CTA leave early)
    if (drop_last_block && blockIdx.x == gridDim.x - 1u) return;
    unsigned long long steps = 0ull;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (int k = 0;; ++k) {
        const uint32_t* Fo = (k & 1) ? F1 : F0;
        uint32_t* Fn = (k & 1) ? F0 : F1;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            bands[(k + 1) % kBandSlots] = Band{0xFFFFFFFFu, 0u};  // for pass k + 1
            cnt[(k + 1) % kBandSlots] = 0ull;
        }
        unsigned int lo, hi;
        pass_rows(bands, k, g, lo, hi);
        const uint32_t w0 = lo <= hi ? lo * g.nq : 0u, w1 = lo <= hi ? (hi + 1u) * g.nq : 0u;
        unsigned long long c = 0ull;
        unsigned int got_lo = 0xFFFFFFFFu, got_hi = 0u;
        for (uint32_t w = w0 + blockIdx.x * blockDim.x + threadIdx.x; w < w1; w += stride) {
            const uint32_t add = grow_word(pore, C, Fo, g, w);
            Fn[w] = add;
            if (add) {
                C[w] |= add;
                c += (unsigned long long)__popc(add);
                const unsigned int r = w / g.nq;
                got_lo = r < got_lo ? r : got_lo;
                got_hi = r > got_hi ? r : got_hi;
            }
        }
        if (__syncthreads_or(c != 0ull)) {
            band_add(&bands[k % kBandSlots], got_lo, got_hi);
            block_sum_u64(c, &cnt[k % kBandSlots]);
        }
        if (!grid_barrier(gb, gridDim.x)) {
            if (threadIdx.x == 0) *reinterpret_cast<volatile int*>(err) = 1;
            return;
        }
        if (*reinterpret_cast<volatile unsigned long long*>(&cnt[k % kBandSlots]) == 0ull) break;
        ++steps;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *out_steps = steps;
}

// out[0] = cluster size, out[1] = touches the first face, out[2] = the last.
__global__ void perc_measure_kernel(const uint32_t* C, PercGeom g, unsigned long long* out) {
    const uint32_t words = g.rows * g.nq;
    const uint32_t stride = gridDim.x * blockDim.x;
    unsigned long long cnt = 0ull;
    bool first = false, last = false;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < words; w += stride) {
        const uint32_t c = C[w];
        if (!c) continue;
        cnt += (unsigned long long)__popc(c);
        const uint32_t r = w / g.nq;
        first |= in_first_face(g, r);
        last |= in_last_face(g, r);
    }
    if (__syncthreads_or(first) && threadIdx.x == 0) atomicOr(&out[1], 1ull);
    if (__syncthreads_or(last) && threadIdx.x == 0) atomicOr(&out[2], 1ull);
    block_sum_u64(cnt, &out[0]);
}

__global__ void perc_export_kernel(const uint32_t* bits, PercGeom g, uint8_t* out,
                                   uint64_t sites) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < sites; i += stride) {
        const uint64_t r = i / g.L, x = i - r * g.L;
        out[i] = (uint8_t)((bits[r * g.nq + (x >> 5)] >> (x & 31u)) & 1u);
    }
}

// One CTA per medium, everything in shared memory: pores, cluster, fronts.
__global__ void __launch_bounds__(512) perc_batch_kernel(PercGeom g, uint32_t thr,
                                                         const uint64_t* seeds, int source,
                                                         uint64_t site, perc_result* res,
                                                         uint8_t* clusters) {
    extern __shared__ uint32_t sm[];
    const uint32_t words = g.rows * g.nq;
    uint32_t* P = sm;
    uint32_t* C = P + words;
    uint32_t* F[2] = {C + words, C + 2 * words};
    const uint64_t seed = seeds[blockIdx.x];
    const uint32_t key0 = (uint32_t)(seed & 0xFFFFFFFFu), key1 = (uint32_t)(seed >> 32);
    const uint64_t site_r = site / g.L, site_x = site - site_r * g.L;
    const uint32_t site_w = (uint32_t)(site_r * g.nq + (site_x >> 5));
    for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) {
        const uint32_t r = w / g.nq, q = w - r * g.nq;
        const uint32_t p = pore_word((uint64_t)g.L * r + 32u * q, valid_bits(g.L, q), key0, key1,
                                     thr);
        uint32_t v;
        if (source == PERC_FACE)
            v = in_first_face(g, r) ? p : 0u;
        else
            v = w == site_w ? p & (1u << (site_x & 31u)) : 0u;
        P[w] = p;
        C[w] = v;
        F[0][w] = v;
    }
    __syncthreads();
    // growth passes until one adds nothing (each pass that continues adds at
    // least one of the medium's finitely many sites)
    int cur = 0;
    int64_t steps = 0;
    while (true) {
        int any = 0;
        for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) {
            const uint32_t add = grow_word(P, C, F[cur], g, w);
            F[cur ^ 1][w] = add;
            if (add) {
                C[w] |= add;
                any = 1;
            }
        }
        if (!__syncthreads_or(any)) break;
        ++steps;
        cur ^= 1;
    }
    unsigned long long cnt = 0ull;
    int first = 0, last = 0;
    for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) {
        const uint32_t c = C[w];
        cnt += (unsigned long long)__popc(c);
        const uint32_t r = w / g.nq;
        if (c && in_first_face(g, r)) first = 1;
        if (c && in_last_face(g, r)) last = 1;
    }
    first = __syncthreads_or(first);
    last = __syncthreads_or(last);
    __shared__ unsigned long long total;
    if (threadIdx.x == 0) total = 0ull;
    __syncthreads();
    block_sum_u64(cnt, &total);
    __syncthreads();
    if (threadIdx.x == 0) {
        perc_result o;
        o.size = (int64_t)total;
        o.spans = first && last ? 1 : 0;
        o.reserved = 0;
        o.steps = steps;
        res[blockIdx.x] = o;
    }
    if (clusters) {
        const uint32_t sites = g.rows * g.L;
        uint8_t* out = clusters + (uint64_t)blockIdx.x * sites;
        for (uint32_t i = threadIdx.x; i < sites; i += blockDim.x) {
            const uint32_t r = i / g.L, x = i - r * g.L;
            out[i] = (uint8_t)((C[r * g.nq + (x >> 5)] >> (x & 31u)) & 1u);
        }
    }
}

unsigned grid_for(uint64_t n, int sm_count) {
    uint64_t b = (n + 255) / 256;
    const uint64_t cap = (uint64_t)sm_count * 16;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

int porosity_threshold(double P, uint32_t* thr) {
    if (!(P >= 0.0 && P <= 1.0)) return ISING_EINVAL;
    const double v = std::floor(std::ldexp(P, 32));  // exact: P times a power of two
    *thr = v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v;
    return ISING_OK;
}

}  // namespace

}  // namespace ising

using namespace ising;

struct perc_medium {
    PercGeom g{};
    uint64_t seed = 0;
    uint64_t sites = 0;
    size_t map_bytes = 0;
    uint32_t* pore = nullptr;
    uint32_t* C = nullptr;
    uint32_t* F[2] = {nullptr, nullptr};
    unsigned long long* counts = nullptr;  // per-pass additions of one graph replay
    unsigned long long* meas = nullptr;    // size, first face, last face
    Band* bands = nullptr;
    cudaGraphExec_t passes = nullptr;      // kPassesPerGraph banded passes
    int mode = PERC_PASSES_AUTO;
    int coop_grid = 0;                     // resident CTAs of the persistent kernel (0: none)
    void* coop = nullptr;                  // counters, barrier, steps, error flag
    cudaStream_t stream = nullptr;
    int sm_count = 0;
};

namespace {

void free_medium(perc_medium* m) {
    for (uint32_t* p : {m->pore, m->C, m->F[0], m->F[1]})
        if (p) cudaFree(p);
    if (m->counts) cudaFree(m->counts);
    if (m->meas) cudaFree(m->meas);
    if (m->bands) cudaFree(m->bands);
    if (m->coop) cudaFree(m->coop);
    if (m->passes) cudaGraphExecDestroy(m->passes);
    delete m;
}

bool geometry(int dims, int L, PercGeom* g, uint64_t* sites) {
    if ((dims != 2 && dims != 3) || L < 1 || L > (1 << 20)) return false;
    const uint64_t n = dims == 3 ? (uint64_t)L * L * L : (uint64_t)L * L;
    if (n > (1ull << 32)) return false;
    g->dims = dims;
    g->L = (uint32_t)L;
    g->rows = dims == 3 ? (uint32_t)L * (uint32_t)L : (uint32_t)L;
    g->nq = ((uint32_t)L + 31u) / 32u;
    if ((uint64_t)g->rows * g->nq > 0xFFFFFFFFull) return false;
    *sites = n;
    return true;
}

}  // namespace

#define PERC_CHECK(call)                                    \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return ising::cuda_fail(e_); \
    } while (0)

extern "C" {

int perc_create(perc_medium** out, int dims, int L, uint64_t seed) {
    if (!out) return ISING_EINVAL;
    *out = nullptr;
    PercGeom g;
    uint64_t sites = 0;
    if (!geometry(dims, L, &g, &sites)) return ISING_EINVAL;
    const DeviceProps* dp = nullptr;
    int rc = device_props(&dp);
    if (rc != ISING_OK) return rc;
    perc_medium* m = new (std::nothrow) perc_medium();
    if (!m) return ISING_ENOMEM;
    m->g = g;
    m->seed = seed;
    m->sites = sites;
    m->sm_count = dp->sm_count;
    m->map_bytes = (size_t)g.rows * g.nq * sizeof(uint32_t);
    cudaError_t e = cudaSuccess;
    for (uint32_t** p : {&m->pore, &m->C, &m->F[0], &m->F[1]}) {
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(p), m->map_bytes);
        if (e == cudaSuccess) e = cudaMemset(*p, 0, m->map_bytes);
    }
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&m->meas), 3 * 8);
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void**>(&m->counts), kPassesPerGraph * 8);
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void**>(&m->bands), kBandSlots * sizeof(Band));
    if (e == cudaSuccess) e = cudaMalloc(&m->coop, kCoopBytes);
    if (e == cudaSuccess) {
        int dev = 0, coop = 0, per_sm = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, perc_persistent_kernel,
                                                              256, 0);
        if (e == cudaSuccess && coop && per_sm > 0) {
            const uint64_t need = ((uint64_t)g.rows * g.nq + 255) / 256;
            const uint64_t resident = (uint64_t)(per_sm < 2 ? per_sm : 2) * dp->sm_count;
            m->coop_grid = (int)(need < resident ? (need < 1 ? 1 : need) : resident);
        }
    }
    if (e != cudaSuccess) {
        free_medium(m);
        return cuda_fail(e);
    }
    *out = m;
    return ISING_OK;
}

int perc_generate(perc_medium* m, double porosity) {
    if (!m) return ISING_EINVAL;
    uint32_t thr = 0;
    const int rc = porosity_threshold(porosity, &thr);
    if (rc != ISING_OK) return rc;
    perc_pores_kernel<<<grid_for((uint64_t)m->g.rows * m->g.nq, m->sm_count), 256, 0,
                        m->stream>>>(m->pore, m->g, (uint32_t)(m->seed & 0xFFFFFFFFu),
                                     (uint32_t)(m->seed >> 32), thr);
    PERC_CHECK(cudaGetLastError());
    PERC_CHECK(cudaMemsetAsync(m->C, 0, m->map_bytes, m->stream));
    return ISING_OK;
}

int perc_set_passes(perc_medium* m, int mode) {
    if (!m) return ISING_EINVAL;
    if (mode != PERC_PASSES_AUTO && mode != PERC_PASSES_GRAPH && mode != PERC_PASSES_PERSISTENT)
        return ISING_EINVAL;
    if (mode == PERC_PASSES_PERSISTENT && m->coop_grid == 0) return ISING_EINVAL;
    m->mode = mode;
    return ISING_OK;
}

int perc_invade(perc_medium* m, int source, int64_t site, perc_result* out) {
    if (!m || !out) return ISING_EINVAL;
    if (source != PERC_POINT && source != PERC_FACE) return ISING_EINVAL;
    if (source == PERC_POINT && (site < 0 || (uint64_t)site >= m->sites)) return ISING_EINVAL;
    const uint64_t words = (uint64_t)m->g.rows * m->g.nq;
    const unsigned grid = grid_for(words, m->sm_count);
    perc_seed_kernel<<<grid, 256, 0, m->stream>>>(m->pore, m->C, m->F[0], m->F[1], m->g, source,
                                                  source == PERC_POINT ? (uint64_t)site : 0ull,
                                                  m->bands);
    PERC_CHECK(cudaGetLastError());
    int64_t steps = 0;
    // AUTO takes the graph: on GB300 it measured 4.6 us per pass at L = 16384
    // (chained launches, eight CTAs per SM) against 8.5 us for the persistent
    // launch (2 - 4 CTAs per SM; 12 us with one, 14 us with all that fit): the
    // pass's own work needs the wide grid, and the grid barrier costs more than
    // a chained graph node
    if (m->mode == PERC_PASSES_PERSISTENT && m->coop_grid > 0) {
        unsigned char* cb = static_cast<unsigned char*>(m->coop);
        unsigned long long* cnt = reinterpret_cast<unsigned long long*>(cb);
        GridBar* gb = reinterpret_cast<GridBar*>(cb + kBandSlots * 8);
        unsigned long long* d_steps = reinterpret_cast<unsigned long long*>(cb + 64);
        int* d_err = reinterpret_cast<int*>(cb + 72);
        PERC_CHECK(cudaMemsetAsync(m->coop, 0, kCoopBytes, m->stream));
        const uint32_t* pore = m->pore;
        PercGeom g = m->g;
        int drop = ising::injecting_timeout() && m->coop_grid > 1 ? 1 : 0;
        void* args[] = {(void*)&pore, (void*)&m->C, (void*)&m->F[0], (void*)&m->F[1], (void*)&g,
                        (void*)&m->bands, (void*)&cnt, (void*)&gb, (void*)&d_steps,
                        (void*)&d_err, (void*)&drop};
        PERC_CHECK(cudaLaunchCooperativeKernel((const void*)perc_persistent_kernel,
                                               dim3((unsigned)m->coop_grid), dim3(256), args, 0,
                                               m->stream));
        struct {
            unsigned long long steps;
            int err;
        } host_out;
        PERC_CHECK(cudaMemcpyAsync(&host_out.steps, d_steps, 8, cudaMemcpyDeviceToHost,
                                   m->stream));
        PERC_CHECK(cudaMemcpyAsync(&host_out.err, d_err, 4, cudaMemcpyDeviceToHost, m->stream));
        PERC_CHECK(cudaStreamSynchronize(m->stream));
        if (host_out.err) return ISING_ETIMEOUT;
        steps = (int64_t)host_out.steps;
    } else {
    if (!m->passes) {
        // eight CTAs per SM walk the band (grid-stride): at L = 16384 on GB300
        // 4.6 us per pass, against 4.8 us with four, 6.4 us with two and 6.1 us
        // with sixteen (most of whose CTAs find no band words and leave)
        const unsigned cap8 = (unsigned)m->sm_count * 8u;
        const unsigned pass_grid = grid < cap8 ? grid : cap8;
        // capture [zero the counts, kPassesPerGraph banded passes] once; the
        // buffers and slots it uses belong to the medium, so replays continue
        cudaStream_t cap = nullptr;
        PERC_CHECK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = cudaMemsetAsync(m->counts, 0, kPassesPerGraph * 8, cap);
            for (int k = 0; k < kPassesPerGraph && le == cudaSuccess; ++k) {
                // chained: a pass is placed on the SMs while the previous one drains
                le = launch_chained(perc_band_kernel, pass_grid, 256u, 0, cap,
                                    static_cast<const uint32_t*>(m->pore), m->C,
                                    static_cast<const uint32_t*>(m->F[k & 1]),
                                    m->F[(k & 1) ^ 1], m->g, m->bands, k, m->counts + k);
            }
            e = cudaStreamEndCapture(cap, &graph);
            if (e == cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&m->passes, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    // replay until a pass adds nothing (each replay that continues added at
    // least kPassesPerGraph sites, so this ends)
    unsigned long long host[kPassesPerGraph];
    while (true) {
        PERC_CHECK(cudaGraphLaunch(m->passes, m->stream));
        PERC_CHECK(cudaMemcpyAsync(host, m->counts, sizeof(host), cudaMemcpyDeviceToHost,
                                   m->stream));
        PERC_CHECK(cudaStreamSynchronize(m->stream));
        int k = 0;
        while (k < kPassesPerGraph && host[k] != 0ull) ++k;
        steps += k;
        if (k < kPassesPerGraph) break;
    }
    }
    PERC_CHECK(cudaMemsetAsync(m->meas, 0, 3 * 8, m->stream));
    perc_measure_kernel<<<grid, 256, 0, m->stream>>>(m->C, m->g, m->meas);
    PERC_CHECK(cudaGetLastError());
    unsigned long long meas[3];
    PERC_CHECK(cudaMemcpyAsync(meas, m->meas, sizeof(meas), cudaMemcpyDeviceToHost, m->stream));
    PERC_CHECK(cudaStreamSynchronize(m->stream));
    out->size = (int64_t)meas[0];
    out->spans = meas[1] && meas[2] ? 1 : 0;
    out->reserved = 0;
    out->steps = steps;
    return ISING_OK;
}

static int export_bits(perc_medium* m, const uint32_t* bits, uint8_t* host_out) {
    if (!m || !host_out) return ISING_EINVAL;
    uint8_t* tmp = nullptr;
    PERC_CHECK(cudaMallocAsync(reinterpret_cast<void**>(&tmp), (size_t)m->sites, m->stream));
    perc_export_kernel<<<grid_for(m->sites, m->sm_count), 256, 0, m->stream>>>(bits, m->g, tmp,
                                                                             m->sites);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_out, tmp, (size_t)m->sites, cudaMemcpyDeviceToHost, m->stream);
    cudaFreeAsync(tmp, m->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    PERC_CHECK(cudaStreamSynchronize(m->stream));
    return ISING_OK;
}

int perc_get_pores(perc_medium* m, uint8_t* host_out) {
    return m ? export_bits(m, m->pore, host_out) : ISING_EINVAL;
}

int perc_get_cluster(perc_medium* m, uint8_t* host_out) {
    return m ? export_bits(m, m->C, host_out) : ISING_EINVAL;
}

int perc_set_stream(perc_medium* m, void* stream) {
    if (!m) return ISING_EINVAL;
    if (m->stream != static_cast<cudaStream_t>(stream))
        PERC_CHECK(cudaStreamSynchronize(m->stream));
    m->stream = static_cast<cudaStream_t>(stream);
    return ISING_OK;
}

void perc_destroy(perc_medium* m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    free_medium(m);
}

int perc_batch(int dims, int L, double porosity, const uint64_t* seeds, int n, int source,
               int64_t site, perc_result* results, uint8_t* clusters_dev, void* stream) {
    if (!seeds || !results || n < 1) return ISING_EINVAL;
    if (source != PERC_POINT && source != PERC_FACE) return ISING_EINVAL;
    PercGeom g;
    uint64_t sites = 0;
    if (!geometry(dims, L, &g, &sites)) return ISING_EINVAL;
    if ((dims == 2 && L > 512) || (dims == 3 && L > 64)) return ISING_EINVAL;
    if (source == PERC_POINT && (site < 0 || (uint64_t)site >= sites)) return ISING_EINVAL;
    uint32_t thr = 0;
    int rc = porosity_threshold(porosity, &thr);
    if (rc != ISING_OK) return rc;
    const size_t smem = (size_t)4 * g.rows * g.nq * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(perc_batch_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(smem > 48 * 1024 ? smem : 48 * 1024));
    if (e != cudaSuccess) return cuda_fail(e);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint64_t* d_seeds = nullptr;
    perc_result* d_res = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void**>(&d_seeds), sizeof(uint64_t) * (size_t)n, st);
    if (e == cudaSuccess)
        e = cudaMallocAsync(reinterpret_cast<void**>(&d_res), sizeof(perc_result) * (size_t)n, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_seeds, seeds, sizeof(uint64_t) * (size_t)n, cudaMemcpyHostToDevice,
                            st);
    if (e == cudaSuccess) {
        const int threads = g.rows * g.nq >= 2048 ? 512 : 256;
        perc_batch_kernel<<<(unsigned)n, threads, smem, st>>>(
            g, thr, d_seeds, source, source == PERC_POINT ? (uint64_t)site : 0ull, d_res,
            clusters_dev);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(results, d_res, sizeof(perc_result) * (size_t)n,
                            cudaMemcpyDeviceToHost, st);
    if (d_seeds) cudaFreeAsync(d_seeds, st);
    if (d_res) cudaFreeAsync(d_res, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? ISING_OK : cuda_fail(e);
}

}  // extern "C"
