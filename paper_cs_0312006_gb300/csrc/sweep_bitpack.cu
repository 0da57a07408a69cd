// sweep_bitpack.cu -- colour pass of the checkerboard Metropolis sweep on the
// bit-packed ("multispin") layout, with the E and M reductions fused in.
//
// Layout: colour c's sites in half index order h = i >> 1 (canonical site
// i = x + L*y (+ L*L*z)), 32 sites per uint32 word, site h at bit (h mod 32) of
// word h / 32; bit 1 means spin +1.  With L % 64 == 0 every half row of W = L/2
// sites is a whole number nq = W/32 of words, so word q of half row r holds the
// sites h = r*W + 32q + b, b = 0..31, and row r's x-neighbour word of the other
// colour lines up bit for bit (h' = h), with the second x-neighbour one bit to
// the right (p = 0: h' - 1) or left (p = 1: h' + 1), p = (c + y + z) & 1.
//
// The Metropolis rule (Sec. 2.2) is evaluated for 32 sites at once: the
// per-site count d of disagreeing neighbours is formed by bit-sliced adders
// over the xor of the site word with its 2*dims neighbour words, which yields
// the mask of sites with dE <= 0 (d >= dims; they flip) and, for the others,
// the mask of sites with each d < dims, selecting the threshold
// floor(exp(-2 beta k) 2^32), k = 2(dims - d).  Draws are identical to the
// int8 layout: site h uses word h & 3 of Philox(seed; h >> 2, t, c, 0), so the
// eight Philox groups of a word are g0 .. g0 + 7 with g0 = (r*W + 32q) / 4.
#include <cstdint>

#include "engine_internal.h"
#include "ising_device.cuh"
#include "pass_bodies.cuh"

namespace ising {

namespace {

// One item = one 32-site word of the colour array (see packed_word()).
template <int DIMS, bool MEASURE>
__global__ void __launch_bounds__(256, 3) pass_packed(PassArgs a) {
    const uint32_t items = (uint32_t)a.rows * ((uint32_t)a.W >> 5);
    const uint32_t stride = gridDim.x * blockDim.x;
    int e_acc = 0, m_acc = 0;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < items; g += stride)
        packed_word<DIMS, MEASURE, 1>(a, g, e_acc, m_acc);
    if (MEASURE) block_reduce_add(e_acc, m_acc, a.obs, a.c == 1);
}

// Initial state written straight into the packed layout: one thread per word
// of one colour; bit b of word (r, q) is canonical site i = L*r + 64q + 2b + p.
__global__ void init_packed(uint32_t* col0, uint32_t* col1, int L, int dims, int64_t rows,
                            int start, uint32_t key0, uint32_t key1) {
    const int nq = L / 64;
    const int64_t words = rows * nq;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w2 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w2 < 2 * words;
         w2 += stride) {
        const int c = (int)(w2 / words);
        const int64_t w = w2 - (int64_t)c * words;
        const int64_t r = w / nq;
        const int q = (int)(w - r * nq);
        uint32_t bits;
        if (start == 0) {
            const int64_t y = r % L, z = dims == 3 ? r / L : 0;
            const int p = (int)((c + y + z) & 1);
            bits = 0u;
            for (int m = 0; m < 16; ++m) {  // sites b = 2m, 2m+1 share Philox group i >> 2
                const int64_t i0 = (int64_t)L * r + 64 * q + 4 * m;  // canonical group base
                const Philox4 u = philox4x32_10((uint32_t)(i0 >> 2), 0u, 0u, kTagInit, key0, key1);
                const uint32_t wd[4] = {u.w0, u.w1, u.w2, u.w3};
                // canonical word (2b + p) & 3 = 2*(b & 1) + p
                if (wd[p] < 0x80000000u) bits |= 1u << (2 * m);
                if (wd[2 + p] < 0x80000000u) bits |= 1u << (2 * m + 1);
            }
        } else {
            bits = start == 1 ? 0xFFFFFFFFu : 0u;
        }
        (c == 0 ? col0 : col1)[w] = bits;
    }
}

__global__ void export_packed(const uint32_t* col0, const uint32_t* col1, int8_t* out, int L,
                              int dims, int64_t sites) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < sites; i += stride) {
        const int64_t x = i % L, rest = i / L;
        const int64_t y = rest % L, z = dims == 3 ? rest / L : 0;
        const int64_t h = i >> 1;
        const uint32_t word = (((x + y + z) & 1) == 0 ? col0 : col1)[h >> 5];
        out[i] = ((word >> (h & 31)) & 1u) ? (int8_t)1 : (int8_t)-1;
    }
}

// One thread per packed word: gather its 32 canonical bytes.
__global__ void import_packed(uint32_t* col0, uint32_t* col1, const int8_t* in, int L, int dims,
                              int64_t rows) {
    const int nq = L / 64;
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
        uint32_t bits = 0u;
        for (int b = 0; b < 32; ++b)
            if (in[(int64_t)L * r + 64 * q + 2 * b + p] > 0) bits |= 1u << b;
        (c == 0 ? col0 : col1)[w] = bits;
    }
}

unsigned grid_for(int64_t n, const DeviceProps& dp) {
    int64_t b = (n + 255) / 256;
    const int64_t cap = (int64_t)dp.sm_count * 16;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

template <int DIMS, bool MEASURE>
cudaError_t launch_packed_t(const PassArgs& a, const DeviceProps& dp, cudaStream_t st) {
    const int64_t items = a.rows * (a.W >> 5);
    int64_t blocks = (items + 255) / 256;
    const int64_t cap = (int64_t)dp.sm_count * dp.blocks_per_sm_packed[DIMS - 2][MEASURE];
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    pass_packed<DIMS, MEASURE><<<(unsigned)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t packed_query_occupancy(DeviceProps& dp) {
    cudaError_t e;
#define ISING_OCC(D, M)                                                                       \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&dp.blocks_per_sm_packed[D - 2][M],      \
                                                      pass_packed<D, M>, 256, 0);              \
    if (e != cudaSuccess) return e;
    ISING_OCC(2, false)
    ISING_OCC(2, true)
    ISING_OCC(3, false)
    ISING_OCC(3, true)
#undef ISING_OCC
    return cudaSuccess;
}

cudaError_t packed_pass(const PassArgs& a, int dims, bool measure, const DeviceProps& dp,
                        cudaStream_t st) {
    if (dims == 2)
        return measure ? launch_packed_t<2, true>(a, dp, st) : launch_packed_t<2, false>(a, dp, st);
    return measure ? launch_packed_t<3, true>(a, dp, st) : launch_packed_t<3, false>(a, dp, st);
}

cudaError_t packed_init(uint32_t* col0, uint32_t* col1, int L, int dims, int64_t rows, int start,
                        uint32_t key0, uint32_t key1, const DeviceProps& dp, cudaStream_t st) {
    init_packed<<<grid_for(2 * rows * (L / 64), dp), 256, 0, st>>>(col0, col1, L, dims, rows,
                                                                    start, key0, key1);
    return cudaGetLastError();
}

cudaError_t packed_export(const uint32_t* col0, const uint32_t* col1, int8_t* out, int L,
                          int dims, int64_t sites, const DeviceProps& dp, cudaStream_t st) {
    export_packed<<<grid_for(sites, dp), 256, 0, st>>>(col0, col1, out, L, dims, sites);
    return cudaGetLastError();
}

cudaError_t packed_import(uint32_t* col0, uint32_t* col1, const int8_t* in, int L, int dims,
                          int64_t rows, const DeviceProps& dp, cudaStream_t st) {
    import_packed<<<grid_for(2 * rows * (L / 64), dp), 256, 0, st>>>(col0, col1, in, L, dims,
                                                                      rows);
    return cudaGetLastError();
}

}  // namespace ising
