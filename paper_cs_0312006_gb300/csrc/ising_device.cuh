// ising_device.cuh -- device building blocks shared by the sweep kernels:
// the counter-based Philox4x32-10 generator, the per-sweep kernel arguments
// and the exact integer reductions of E and M.
//
// Philox4x32-10 follows Salmon, Moraes, Dror and Shaw, "Parallel Random
// Numbers: As Easy as 1, 2, 3" (SC'11): ten rounds, each multiplying counter
// words 0 and 2 by two fixed odd 32-bit constants, exchanging the high halves
// of the products into words 0 and 2 (xored with the neighbouring word and a
// round key) and keeping the low halves in words 1 and 3; the two key words
// advance by Weyl increments between rounds.  It replaces the paper's linear
// congruential generator (Sec. 2.1) so that each site's draw is a pure
// function of (seed, sweep, colour, site group), independent of layout and
// launch shape.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ising {

constexpr uint32_t kPhiloxMulA = 0xD2511F53u;
constexpr uint32_t kPhiloxMulB = 0xCD9E8D57u;
constexpr uint32_t kPhiloxWeylA = 0x9E3779B9u;
constexpr uint32_t kPhiloxWeylB = 0xBB67AE85u;

// Local update rules (the values of ISING_RULE_* in ising.h).
constexpr int kRuleMetropolis = 0;
constexpr int kRuleHeatBath = 1;
constexpr int kRuleDemon = 2;
constexpr int kRuleMultiHit = 3;

// Counter word 3 ("tag") separates the uses of the stream.
constexpr uint32_t kTagSweep = 0u;
constexpr uint32_t kTagInit = 1u;

struct Philox4 {
    uint32_t w0, w1, w2, w3;
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                 uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        // one 32x32 -> 64-bit product per multiplier: high half mixes, low half carries over
        const uint64_t pa = (uint64_t)c0 * kPhiloxMulA;
        const uint64_t pb = (uint64_t)c2 * kPhiloxMulB;
        c0 = (uint32_t)(pb >> 32) ^ c1 ^ k0;
        c1 = (uint32_t)pb;
        c2 = (uint32_t)(pa >> 32) ^ c3 ^ k1;
        c3 = (uint32_t)pa;
        k0 += kPhiloxWeylA;
        k1 += kPhiloxWeylB;
    }
    return Philox4{c0, c1, c2, c3};
}

// The same function with each 32x32 -> 64-bit product taken as a separate
// low-half and high-half 32-bit multiply (mul.lo / mul.hi) instead of one
// widening multiply; identical results.  Kept for measuring which form the
// multiply pipe retires faster (ising_philox_probe).
__device__ __forceinline__ Philox4 philox4x32_10_split(uint32_t c0, uint32_t c1, uint32_t c2,
                                                       uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t pa_hi = __umulhi(c0, kPhiloxMulA), pa_lo = c0 * kPhiloxMulA;
        const uint32_t pb_hi = __umulhi(c2, kPhiloxMulB), pb_lo = c2 * kPhiloxMulB;
        c0 = pb_hi ^ c1 ^ k0;
        c1 = pb_lo;
        c2 = pa_hi ^ c3 ^ k1;
        c3 = pa_lo;
        k0 += kPhiloxWeylA;
        k1 += kPhiloxWeylB;
    }
    return Philox4{c0, c1, c2, c3};
}

// 4 * RUNS calls whose counter word 0 runs over RUNS sets of four
// consecutive values (base[r] .. base[r] + 3, no 32-bit wrap), the other
// counter words and the key shared, advanced one round at a time so that a
// caller can place other work between the rounds.  In the first round the
// product of base + i is the product of base plus i times the multiplier (a
// 64-bit add instead of a multiply).  result(w) equals philox4x32_10 of call
// w's counter (base[w / 4] + w % 4, ctr1, ctr2, ctr3) under the same key.
template <int RUNS>
struct PhiloxRuns {
    static constexpr int N = 4 * RUNS;
    uint32_t c0[N], c1[N], c2[N], c3[N];
    uint32_t k0, k1;

    __device__ __forceinline__ void first_round(const uint32_t (&base)[RUNS], uint32_t ctr1,
                                                uint32_t ctr2, uint32_t ctr3, uint32_t key0,
                                                uint32_t key1) {
        const uint64_t pb = (uint64_t)ctr2 * kPhiloxMulB;
#pragma unroll
        for (int r = 0; r < RUNS; ++r) {
            const uint64_t pa0 = (uint64_t)base[r] * kPhiloxMulA;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int w = 4 * r + i;
                const uint64_t pa = pa0 + (uint64_t)i * kPhiloxMulA;
                c0[w] = (uint32_t)(pb >> 32) ^ ctr1 ^ key0;
                c1[w] = (uint32_t)pb;
                c2[w] = (uint32_t)(pa >> 32) ^ ctr3 ^ key1;
                c3[w] = (uint32_t)pa;
            }
        }
        k0 = key0 + kPhiloxWeylA;
        k1 = key1 + kPhiloxWeylB;
    }

    __device__ __forceinline__ void next_round() {
#pragma unroll
        for (int w = 0; w < N; ++w) {
            const uint64_t pa = (uint64_t)c0[w] * kPhiloxMulA;
            const uint64_t pb = (uint64_t)c2[w] * kPhiloxMulB;
            c0[w] = (uint32_t)(pb >> 32) ^ c1[w] ^ k0;
            c1[w] = (uint32_t)pb;
            c2[w] = (uint32_t)(pa >> 32) ^ c3[w] ^ k1;
            c3[w] = (uint32_t)pa;
        }
        k0 += kPhiloxWeylA;
        k1 += kPhiloxWeylB;
    }

    __device__ __forceinline__ Philox4 result(int w) const {
        return Philox4{c0[w], c1[w], c2[w], c3[w]};
    }
};

// Programmatic dependent launch (griddepcontrol, sm_90 and later).  The
// per-lattice pass kernels are launched with programmatic stream
// serialisation (launch_chained), so the next kernel in the stream can be
// scheduled onto SMs while this one finishes.  Every such kernel calls
// grid_dependency_wait() before its first global memory access: it returns
// once all earlier kernels of the stream have completed and their writes are
// visible (a pass reads the colour the previous pass wrote and writes the
// colour it read), and it is a no-op for a kernel launched without the
// attribute.  launch_dependents() then lets the next pass's CTAs be placed as
// SMs free up; they in turn wait before touching memory.
__device__ __forceinline__ void grid_dependency_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Arguments of one colour pass.  The colour-c array is updated in place; it
// reads only the colour-(1-c) array, so no site reads a value written by the
// same pass (Sec. 2.2: a pass through all sites of one colour).
struct PassArgs {
    void* own;              // colour-c spins (int8 +-1, or packed words)
    const void* other;      // colour-(1-c) spins
    unsigned long long* obs; // (E, M) int64 slot of this sweep, or nullptr
    int64_t rows;           // half rows per colour: L^(dims-1)
    int L;                  // linear size
    int W;                  // sites of one colour per row: L / 2
    // acceptance thresholds of the pass's rule:
    //   kRuleMetropolis: thr[j] = floor(exp(-2 beta k) 2^32), k = 2j + 2 (j < dims)
    //   kRuleHeatBath:   thr[d] = floor(2^32 / (1 + exp(4 beta (dims - d)))),
    //                    d = 0..2*dims disagreeing neighbours
    uint32_t thr[7];
    uint32_t key0, key1;    // seed (low, high)
    uint32_t t;             // sweep index
    int c;                  // colour of this pass: 0 black, 1 white
    int nv;                 // 16-byte vectors per half row (W / 16), vector kernels only
    int strips;             // row strips per column, vector kernels only
    // demon dynamics only: the own colour's demons (one byte per site, half
    // rows; half row r's demons in storage row (r - rot) mod rows) and their cap
    void* dem;
    int qmax;
    uint32_t rot;
    int hits;  // multi-hit Metropolis: trials per visit (hit m draws with word 2 = c + 2m)
};

// Block-wide sum of two ints followed by one 64-bit atomic each into the
// sweep's slot.  Integer addition is exact, so the order of the atomics does
// not matter and the totals are bit-reproducible.
__device__ __forceinline__ void block_reduce_add(int e, int m, unsigned long long* slot,
                                                 bool with_e) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, off);
        m += __shfl_xor_sync(0xffffffffu, m, off);
    }
    __shared__ long long red_e[32], red_m[32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red_e[warp] = e;
        red_m[warp] = m;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        long long se = lane < nw ? red_e[lane] : 0;
        long long sm = lane < nw ? red_m[lane] : 0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            se += __shfl_xor_sync(0xffffffffu, se, off);
            sm += __shfl_xor_sync(0xffffffffu, sm, off);
        }
        if (lane == 0) {
            if (with_e && se != 0) atomicAdd(&slot[0], (unsigned long long)se);
            if (sm != 0) atomicAdd(&slot[1], (unsigned long long)sm);
        }
    }
}

}  // namespace ising
