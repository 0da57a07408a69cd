// sweep_bitpack.cu -- colour pass of the checkerboard Metropolis sweep on the
// bit-packed ("multispin") layout, with the E and M reductions fused in.
//
// Layout: each half row r of colour c (its W = L/2 sites, half column
// xh = 0..W-1, half index h = r*W + xh) takes nq = ceil(W/32) uint32 words;
// site xh is bit (xh mod 32) of word r*nq + xh/32, bit 1 meaning spin +1.  The
// bits past W in a row's last word are padding: zero, never read as spins,
// never flipped.  Row r's word q of the other colour lines up with the site
// word bit for bit (same half column), the second x-neighbour is one bit to
// the right (p = 0: xh - 1) or left (p = 1: xh + 1), p = (c + y + z) & 1, and
// the y- and z-neighbour words are the same word of the neighbouring rows.
//
// The Metropolis rule (Sec. 2.2) is evaluated for 32 sites at once: the
// per-site count d of disagreeing neighbours is formed by bit-sliced adders
// over the xor of the site word with its 2*dims neighbour words, which yields
// the mask of sites with dE <= 0 (d >= dims; they flip) and, for the others,
// the mask of sites with each d < dims, selecting the threshold
// floor(exp(-2 beta k) 2^32), k = 2(dims - d).  Draws are identical to the
// int8 layout: site h uses word h & 3 of Philox(seed; h >> 2, t, c, 0).
#include <cstdint>

#include "engine_internal.h"
#include "ising_device.cuh"
#include "pass_bodies.cuh"

namespace ising {

namespace {

// One item = one 32-site word of the colour array (see packed_word()).
// Rows that start inside a Philox group are visited grouped by their offset
// (rgroups, see packed_word).
// FULL instances serve lattices whose words are all full (W % 32 == 0) and
// whose word count per half row nq = 2^nq_shift is a power of two (then so is
// L = 64 nq; in 3D l_shift = log2 L): an item's row, word and neighbours come
// from shifts and masks, every row starts on a Philox group, and a thread
// loads its next item's six words (eight in 3D) before it updates the current
// one, so that their latency hides behind the current item's draws (at most
// 64 registers for four CTAs per SM measured slower: 2D L = 8192 29.2 ->
// 29.4 us per pass, 3D L = 256 9.0e11 -> 8.0e11 site updates/s).
template <int DIMS, bool MEASURE, int RULE, bool FULL>
__global__ void __launch_bounds__(256, 3) pass_packed(PassArgs a, uint32_t rgroups,
                                                      uint32_t nq_shift, uint32_t l_shift) {
    const uint32_t items = (uint32_t)a.rows * (((uint32_t)a.W + 31u) >> 5);
    const uint32_t stride = gridDim.x * blockDim.x;
    int e_acc = 0, m_acc = 0;
    grid_dependency_wait();
    launch_dependents();
    if constexpr (!FULL) {
        for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < items; g += stride)
            packed_word<DIMS, MEASURE, 1, RULE, RULE != kRuleMultiHit>(a, g, e_acc, m_acc,
                                                                       rgroups);
    } else {
        const uint32_t nq = 1u << nq_shift, L = (uint32_t)a.L, W = (uint32_t)a.W;
        uint32_t* own = static_cast<uint32_t*>(a.own);
        const uint32_t* other = static_cast<const uint32_t*>(a.other);
        struct Words {
            uint32_t o, x, ym, yp, zm, zp, s;
        };
        // the loads only: nothing here waits for them
        auto load = [&](uint32_t item, Words& w) {
            const uint32_t r = item >> nq_shift, q = item & (nq - 1u);
            const uint32_t z = DIMS == 3 ? r >> l_shift : 0u, y = r & (L - 1u);
            const uint32_t row = r * nq, plane = z * L;
            const int p = (a.c + (int)y + (int)z) & 1;
            // x-neighbour word: the one before (p = 0) or after (p = 1), wrapping in the row
            const uint32_t xq = (p == 0 ? q - 1u : q + 1u) & (nq - 1u);
            w.o = __ldg(other + row + q);
            w.x = __ldg(other + row + xq);
            w.ym = __ldg(other + (plane + ((y - 1u) & (L - 1u))) * nq + q);
            w.yp = __ldg(other + (plane + ((y + 1u) & (L - 1u))) * nq + q);
            if (DIMS == 3) {
                w.zm = __ldg(other + ((((z - 1u) & (L - 1u)) * L + y) * nq + q));
                w.zp = __ldg(other + ((((z + 1u) & (L - 1u)) * L + y) * nq + q));
            } else {
                w.zm = w.zp = 0u;
            }
            w.s = own[row + q];
        };
        uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
        if (g < items) {
            Words cur;
            load(g, cur);
            for (;;) {
                const uint32_t gn = g + stride;
                const bool more = gn < items;
                Words nxt = cur;
                if (more) load(gn, nxt);
                const uint32_t r = g >> nq_shift, q = g & (nq - 1u);
                const uint32_t z = DIMS == 3 ? r >> l_shift : 0u, y = r & (L - 1u);
                const int p = (a.c + (int)y + (int)z) & 1;
                // bit b <- neighbour xh - 1 (p = 0) or xh + 1 (p = 1)
                const uint32_t sh = p == 0 ? __funnelshift_l(cur.x, cur.o, 1)
                                           : __funnelshift_r(cur.o, cur.x, 1);
                packed_update<DIMS, MEASURE, RULE, RULE != kRuleMultiHit, true>(
                    a, own + r * nq + q, cur.s, cur.o, sh, cur.ym, cur.yp, cur.zm, cur.zp,
                    0xFFFFFFFFu, 32u, r * W + 32u * q, e_acc, m_acc);
                if (!more) break;
                cur = nxt;
                g = gn;
            }
        }
    }
    if (MEASURE) block_reduce_add(e_acc, m_acc, a.obs, a.c == 1);
}

// Initial state written straight into the packed layout: one thread per word
// of one colour; bit b of word (r, q) is half column xh = 32q + b, i.e. the
// canonical site i = L*r + 2*xh + p.
__global__ void init_packed(uint32_t* col0, uint32_t* col1, int L, int dims, int64_t rows,
                            int start, uint32_t key0, uint32_t key1) {
    const int W = L / 2, nq = (W + 31) / 32;
    const int64_t words = rows * nq;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w2 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w2 < 2 * words;
         w2 += stride) {
        const int c = (int)(w2 / words);
        const int64_t w = w2 - (int64_t)c * words;
        const int64_t r = w / nq;
        const int q = (int)(w - r * nq);
        const int nb = W - 32 * q < 32 ? W - 32 * q : 32;
        uint32_t bits = 0u;
        if (start == 0) {
            const int64_t y = r % L, z = dims == 3 ? r / L : 0;
            const int p = (int)((c + y + z) & 1);
            for (int b = 0; b < nb; ++b) {
                const int64_t i = (int64_t)L * r + 2 * (32 * q + b) + p;
                const Philox4 u = philox4x32_10((uint32_t)(i >> 2), 0u, 0u, kTagInit, key0, key1);
                const uint32_t wd[4] = {u.w0, u.w1, u.w2, u.w3};
                if (wd[i & 3] < 0x80000000u) bits |= 1u << b;
            }
        } else if (start == 1) {
            bits = nb == 32 ? 0xFFFFFFFFu : ((1u << nb) - 1u);
        }
        (c == 0 ? col0 : col1)[w] = bits;
    }
}

__global__ void export_packed(const uint32_t* col0, const uint32_t* col1, int8_t* out, int L,
                              int dims, int64_t sites) {
    const int nq = (L / 2 + 31) / 32;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < sites; i += stride) {
        const int64_t x = i % L, r = i / L;
        const int64_t y = r % L, z = dims == 3 ? r / L : 0;
        const int64_t xh = x >> 1;
        const uint32_t word = (((x + y + z) & 1) == 0 ? col0 : col1)[r * nq + (xh >> 5)];
        out[i] = ((word >> (xh & 31)) & 1u) ? (int8_t)1 : (int8_t)-1;
    }
}

// One thread per packed word: gather its canonical bytes.
__global__ void import_packed(uint32_t* col0, uint32_t* col1, const int8_t* in, int L, int dims,
                              int64_t rows) {
    const int W = L / 2, nq = (W + 31) / 32;
    const int64_t words = rows * nq;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w2 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w2 < 2 * words;
         w2 += stride) {
        const int c = (int)(w2 / words);
        const int64_t w = w2 - (int64_t)c * words;
        const int64_t r = w / nq;
        const int q = (int)(w - r * nq);
        const int64_t y = r % L, z = dims == 3 ? r / L : 0;
        const int p = (int)((c + y + z) & 1);
        const int nb = W - 32 * q < 32 ? W - 32 * q : 32;
        uint32_t bits = 0u;
        for (int b = 0; b < nb; ++b)
            if (in[(int64_t)L * r + 2 * (32 * q + b) + p] > 0) bits |= 1u << b;
        (c == 0 ? col0 : col1)[w] = bits;
    }
}

unsigned grid_for(int64_t n, const DeviceProps& dp) {
    int64_t b = (n + 255) / 256;
    const int64_t cap = (int64_t)dp.sm_count * 16;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

template <int DIMS, bool MEASURE, int RULE>
cudaError_t launch_packed_t(const PassArgs& a, const DeviceProps& dp, cudaStream_t st) {
    const int nq = (a.W + 31) >> 5;
    const int64_t items = a.rows * nq;
    // (multi-hit keeps the general loop: its trials need the registers)
    const bool full = RULE != kRuleMultiHit && a.W % 32 == 0 && is_pow2(nq);
    int64_t blocks = (items + 255) / 256;
    const int64_t cap =
        (int64_t)dp.sm_count * dp.blocks_per_sm_packed[RULE][DIMS - 2][MEASURE][full ? 1 : 0];
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    // odd W: a row's offset in its Philox group is r W mod 4, set by r mod 4;
    // W = 2 mod 4: by r mod 2
    const uint32_t rgroups = packed_row_groups((uint32_t)a.W);
    if constexpr (RULE != kRuleMultiHit) {
        if (full) {
            const uint32_t nq_shift = (uint32_t)__builtin_ctz((unsigned)nq);
            const uint32_t l_shift = DIMS == 3 ? (uint32_t)__builtin_ctz((unsigned)a.L) : 0u;
            return launch_chained(pass_packed<DIMS, MEASURE, RULE, true>, (unsigned)blocks, 256u,
                                  0, st, a, rgroups, nq_shift, l_shift);
        }
    }
    return launch_chained(pass_packed<DIMS, MEASURE, RULE, false>, (unsigned)blocks, 256u, 0, st,
                          a, rgroups, 0u, 0u);
}

}  // namespace

cudaError_t packed_query_occupancy(DeviceProps& dp) {
    cudaError_t e;
#define ISING_OCC1(R, D, M, F)                                                                \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&dp.blocks_per_sm_packed[R][D - 2][M][F],\
                                                      pass_packed<D, M, R, F>, 256, 0);       \
    if (e != cudaSuccess) return e;
#define ISING_OCC(R, D, M) ISING_OCC1(R, D, M, false) ISING_OCC1(R, D, M, true)
#define ISING_OCC_MH(R, D, M) ISING_OCC1(R, D, M, false)
    ISING_OCC(kRuleMetropolis, 2, false)
    ISING_OCC(kRuleMetropolis, 2, true)
    ISING_OCC(kRuleMetropolis, 3, false)
    ISING_OCC(kRuleMetropolis, 3, true)
    ISING_OCC(kRuleHeatBath, 2, false)
    ISING_OCC(kRuleHeatBath, 2, true)
    ISING_OCC(kRuleHeatBath, 3, false)
    ISING_OCC(kRuleHeatBath, 3, true)
    ISING_OCC_MH(kRuleMultiHit, 2, false)
    ISING_OCC_MH(kRuleMultiHit, 2, true)
    ISING_OCC_MH(kRuleMultiHit, 3, false)
    ISING_OCC_MH(kRuleMultiHit, 3, true)
#undef ISING_OCC_MH
#undef ISING_OCC
#undef ISING_OCC1
    return cudaSuccess;
}

template <int RULE>
static cudaError_t packed_pass_rule(const PassArgs& a, int dims, bool measure,
                                    const DeviceProps& dp, cudaStream_t st) {
    if (dims == 2)
        return measure ? launch_packed_t<2, true, RULE>(a, dp, st)
                       : launch_packed_t<2, false, RULE>(a, dp, st);
    return measure ? launch_packed_t<3, true, RULE>(a, dp, st)
                   : launch_packed_t<3, false, RULE>(a, dp, st);
}

cudaError_t packed_pass(const PassArgs& a, int dims, bool measure, int rule,
                        const DeviceProps& dp, cudaStream_t st) {
    if (rule == kRuleHeatBath) return packed_pass_rule<kRuleHeatBath>(a, dims, measure, dp, st);
    if (rule == kRuleMultiHit) return packed_pass_rule<kRuleMultiHit>(a, dims, measure, dp, st);
    return packed_pass_rule<kRuleMetropolis>(a, dims, measure, dp, st);
}

cudaError_t packed_init(uint32_t* col0, uint32_t* col1, int L, int dims, int64_t rows, int start,
                        uint32_t key0, uint32_t key1, const DeviceProps& dp, cudaStream_t st) {
    init_packed<<<grid_for(2 * rows * ((L / 2 + 31) / 32), dp), 256, 0, st>>>(
        col0, col1, L, dims, rows, start, key0, key1);
    return cudaGetLastError();
}

cudaError_t packed_export(const uint32_t* col0, const uint32_t* col1, int8_t* out, int L,
                          int dims, int64_t sites, const DeviceProps& dp, cudaStream_t st) {
    export_packed<<<grid_for(sites, dp), 256, 0, st>>>(col0, col1, out, L, dims, sites);
    return cudaGetLastError();
}

cudaError_t packed_import(uint32_t* col0, uint32_t* col1, const int8_t* in, int L, int dims,
                          int64_t rows, const DeviceProps& dp, cudaStream_t st) {
    import_packed<<<grid_for(2 * rows * ((L / 2 + 31) / 32), dp), 256, 0, st>>>(col0, col1, in,
                                                                                 L, dims, rows);
    return cudaGetLastError();
}

}  // namespace ising
