// convert.cu -- canonical int8 spins <-> the two device layouts, and the
// initial states, for lattices whose half rows are whole 16-byte vectors
// (int8: L % 32 == 0) or whole 32-bit words (bit-packed: L % 64 == 0).
//
// A canonical row r (y = r mod L, z = r div L) of L bytes holds the sites
// x = 0..L-1; site x has colour (x + y + z) & 1 and half column x >> 1, so the
// even-x sites of the row are colour c_even = (y + z) & 1 and the odd-x sites
// the other colour, both at half row r.  One item moves 32 canonical bytes
// (int8: 16 bytes of each colour, split and merged with byte permutes) or 64
// canonical bytes (bit-packed: one 32-site word of each colour).  The
// canonical side may be host memory the device can reach (pinned, mapped):
// the kernels then read or write it directly over the host link.
//
// The hot start of Sec. 2.2 (spin up with probability p = 1/2) draws word
// i & 3 of Philox(seed; i >> 2, 0, 0, 1) for canonical site i; an item's sites
// are whole Philox groups, so every call serves four sites.
#include <cstdint>

#include "engine_internal.h"
#include "ising_device.cuh"

namespace ising {

namespace {

// Bytes of w made valid spins: negative -> 0xFF (-1), anything else -> 0x01
// (+1).  *bad collects the bits where w differed from that.
__device__ __forceinline__ uint32_t normalise_spins(uint32_t w, uint32_t& bad) {
    const uint32_t neg = w & 0x80808080u;
    const uint32_t v = neg | (neg - (neg >> 7)) | 0x01010101u;
    bad |= w ^ v;
    return v;
}

__device__ __forceinline__ void raise_flag(int* flag) {
    *reinterpret_cast<volatile int*>(flag) = 1;
}

struct RowGeom {
    uint32_t per_row;  // items per canonical row
    uint32_t L, W;
    uint32_t items;
};

__device__ __forceinline__ void item_pos(const RowGeom& g, uint32_t it, uint32_t& r, uint32_t& k,
                                         int& c_even) {
    r = it / g.per_row;
    k = it - r * g.per_row;
    const uint32_t z = r / g.L, y = r - z * g.L;  // 2D: z = 0 (r < L)
    c_even = (int)((y + z) & 1u);
}

// ---- int8 layout: 32 canonical bytes <-> 16 bytes of each colour ----------

template <bool CHECK>
__global__ void import_rows_int8(int8_t* col0, int8_t* col1, const int8_t* in, RowGeom g,
                                 int* bad_flag) {
    uint32_t bad = 0u;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < g.items; it += stride) {
        uint32_t r, k;
        int ce;
        item_pos(g, it, r, k, ce);
        const uint4* src = reinterpret_cast<const uint4*>(in + (size_t)r * g.L + 32u * k);
        const uint4 a = src[0], b = src[1];
        uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        if (CHECK) {
#pragma unroll
            for (int i = 0; i < 8; ++i) w[i] = normalise_spins(w[i], bad);
        }
        const uint4 ev = make_uint4(__byte_perm(w[0], w[1], 0x6420), __byte_perm(w[2], w[3], 0x6420),
                                    __byte_perm(w[4], w[5], 0x6420), __byte_perm(w[6], w[7], 0x6420));
        const uint4 od = make_uint4(__byte_perm(w[0], w[1], 0x7531), __byte_perm(w[2], w[3], 0x7531),
                                    __byte_perm(w[4], w[5], 0x7531), __byte_perm(w[6], w[7], 0x7531));
        const size_t h = (size_t)r * g.W + 16u * k;
        *reinterpret_cast<uint4*>((ce == 0 ? col0 : col1) + h) = ev;
        *reinterpret_cast<uint4*>((ce == 0 ? col1 : col0) + h) = od;
    }
    if (CHECK && bad != 0u) raise_flag(bad_flag);
}

__global__ void export_rows_int8(const int8_t* col0, const int8_t* col1, int8_t* out, RowGeom g) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < g.items; it += stride) {
        uint32_t r, k;
        int ce;
        item_pos(g, it, r, k, ce);
        const size_t h = (size_t)r * g.W + 16u * k;
        const uint4 ev = *reinterpret_cast<const uint4*>((ce == 0 ? col0 : col1) + h);
        const uint4 od = *reinterpret_cast<const uint4*>((ce == 0 ? col1 : col0) + h);
        uint4* dst = reinterpret_cast<uint4*>(out + (size_t)r * g.L + 32u * k);
        dst[0] = make_uint4(__byte_perm(ev.x, od.x, 0x5140), __byte_perm(ev.x, od.x, 0x7362),
                            __byte_perm(ev.y, od.y, 0x5140), __byte_perm(ev.y, od.y, 0x7362));
        dst[1] = make_uint4(__byte_perm(ev.z, od.z, 0x5140), __byte_perm(ev.z, od.z, 0x7362),
                            __byte_perm(ev.w, od.w, 0x5140), __byte_perm(ev.w, od.w, 0x7362));
    }
}

// Hot start: the item's 32 sites are Philox groups g0 .. g0 + 7.
__global__ void init_rows_int8_hot(int8_t* col0, int8_t* col1, RowGeom g, uint32_t key0,
                                   uint32_t key1) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < g.items; it += stride) {
        uint32_t r, k;
        int ce;
        item_pos(g, it, r, k, ce);
        const uint32_t g0 = (uint32_t)(((size_t)r * g.L + 32u * k) >> 2);
        uint32_t w[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const Philox4 u = philox4x32_10(g0 + (uint32_t)m, 0u, 0u, kTagInit, key0, key1);
            // byte j = +1 iff word j < 2^31, else -1
            const uint32_t d[4] = {u.w0, u.w1, u.w2, u.w3};
            uint32_t v = 0u;
#pragma unroll
            for (int j = 0; j < 4; ++j) v |= (d[j] < 0x80000000u ? 0x01u : 0xFFu) << (8 * j);
            w[m] = v;
        }
        const uint4 ev = make_uint4(__byte_perm(w[0], w[1], 0x6420), __byte_perm(w[2], w[3], 0x6420),
                                    __byte_perm(w[4], w[5], 0x6420), __byte_perm(w[6], w[7], 0x6420));
        const uint4 od = make_uint4(__byte_perm(w[0], w[1], 0x7531), __byte_perm(w[2], w[3], 0x7531),
                                    __byte_perm(w[4], w[5], 0x7531), __byte_perm(w[6], w[7], 0x7531));
        const size_t h = (size_t)r * g.W + 16u * k;
        *reinterpret_cast<uint4*>((ce == 0 ? col0 : col1) + h) = ev;
        *reinterpret_cast<uint4*>((ce == 0 ? col1 : col0) + h) = od;
    }
}

// ---- bit-packed layout: 64 canonical bytes <-> one word of each colour -----

// Bits of the even (byte 0, 2) and odd (byte 1, 3) bytes of w that hold +1
// (sign clear), as two 2-bit fields.
__device__ __forceinline__ void spin_bits(uint32_t w, uint32_t& ev2, uint32_t& od2) {
    const uint32_t pos = ~w & 0x80808080u;
    ev2 = ((pos >> 7) & 1u) | ((pos >> 22) & 2u);
    od2 = ((pos >> 15) & 1u) | ((pos >> 30) & 2u);
}

template <bool CHECK>
__global__ void import_rows_packed(uint32_t* col0, uint32_t* col1, const int8_t* in, RowGeom g,
                                   int* bad_flag) {
    uint32_t bad = 0u;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < g.items; it += stride) {
        uint32_t r, q;
        int ce;
        item_pos(g, it, r, q, ce);
        const uint4* src = reinterpret_cast<const uint4*>(in + (size_t)r * g.L + 64u * q);
        uint32_t ev = 0u, od = 0u;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const uint4 a = src[v];
            const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint32_t x = w[i];
                if (CHECK) x = normalise_spins(x, bad);
                uint32_t e2, o2;
                spin_bits(x, e2, o2);
                // canonical word 4v + i holds half columns 2(4v + i), +1
                ev |= e2 << (2 * (4 * v + i));
                od |= o2 << (2 * (4 * v + i));
            }
        }
        const size_t word = (size_t)r * (g.W >> 5) + q;
        (ce == 0 ? col0 : col1)[word] = ev;
        (ce == 0 ? col1 : col0)[word] = od;
    }
    if (CHECK && bad != 0u) raise_flag(bad_flag);
}

// Four sites as bytes from two bits of each colour word: canonical bytes
// (even b, odd b, even b+1, odd b+1) = +1 where the bit is set, else -1.
__device__ __forceinline__ uint32_t spin_bytes(uint32_t ev, uint32_t od, int b) {
    const uint32_t e = (ev >> b) & 3u, o = (od >> b) & 3u;
    const uint32_t ones = (e & 1u) | ((o & 1u) << 8) | ((e & 2u) << 15) | ((o & 2u) << 23);
    return 0xFFFFFFFFu - 0xFEu * ones;  // per byte: 1 -> 0x01, 0 -> 0xFF (no borrow)
}

__global__ void export_rows_packed(const uint32_t* col0, const uint32_t* col1, int8_t* out,
                                   RowGeom g) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < g.items; it += stride) {
        uint32_t r, q;
        int ce;
        item_pos(g, it, r, q, ce);
        const size_t word = (size_t)r * (g.W >> 5) + q;
        const uint32_t ev = (ce == 0 ? col0 : col1)[word];
        const uint32_t od = (ce == 0 ? col1 : col0)[word];
        uint4* dst = reinterpret_cast<uint4*>(out + (size_t)r * g.L + 64u * q);
#pragma unroll
        for (int v = 0; v < 4; ++v)
            dst[v] = make_uint4(spin_bytes(ev, od, 8 * v), spin_bytes(ev, od, 8 * v + 2),
                                spin_bytes(ev, od, 8 * v + 4), spin_bytes(ev, od, 8 * v + 6));
    }
}

// Hot start: the item's 64 canonical sites are Philox groups g0 .. g0 + 15;
// group m covers half columns 2m, 2m + 1 of both colours (word j of the call:
// x = 4m + j, even j -> the even-x colour).
__global__ void init_rows_packed_hot(uint32_t* col0, uint32_t* col1, RowGeom g, uint32_t key0,
                                     uint32_t key1) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < g.items; it += stride) {
        uint32_t r, q;
        int ce;
        item_pos(g, it, r, q, ce);
        const uint32_t g0 = (uint32_t)(((size_t)r * g.L + 64u * q) >> 2);
        uint32_t ev = 0u, od = 0u;
#pragma unroll 4
        for (int m = 0; m < 16; ++m) {
            const Philox4 u = philox4x32_10(g0 + (uint32_t)m, 0u, 0u, kTagInit, key0, key1);
            ev |= ((u.w0 < 0x80000000u ? 1u : 0u) | (u.w2 < 0x80000000u ? 2u : 0u)) << (2 * m);
            od |= ((u.w1 < 0x80000000u ? 1u : 0u) | (u.w3 < 0x80000000u ? 2u : 0u)) << (2 * m);
        }
        const size_t word = (size_t)r * (g.W >> 5) + q;
        (ce == 0 ? col0 : col1)[word] = ev;
        (ce == 0 ? col1 : col0)[word] = od;
    }
}

// Any length, any alignment: raise the flag if a byte is not +1 or -1.
__global__ void check_spins_kernel(const int8_t* in, int64_t n, int* bad_flag) {
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        bad |= in[i] != 1 && in[i] != -1;
    if (bad) raise_flag(bad_flag);
}

RowGeom row_geom(int L, int64_t rows, uint32_t bytes_per_item) {
    RowGeom g;
    g.L = (uint32_t)L;
    g.W = (uint32_t)(L / 2);
    g.per_row = (uint32_t)L / bytes_per_item;
    g.items = (uint32_t)((uint64_t)rows * g.per_row);
    return g;
}

unsigned grid_items(uint32_t items, const DeviceProps& dp) {
    uint64_t b = ((uint64_t)items + 255) / 256;
    const uint64_t cap = (uint64_t)dp.sm_count * 16;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

bool rows_ok(int layout, int L) {
    return layout == ISING_BITPACK ? L % 64 == 0 : L % 32 == 0;
}

cudaError_t rows_init(void* col0, void* col1, size_t col_data_bytes, int layout, int L,
                      int64_t rows, int start, uint32_t key0, uint32_t key1,
                      const DeviceProps& dp, cudaStream_t st) {
    if (start != 0) {
        // cold starts are one value everywhere: int8 0x01 / 0xFF bytes, packed
        // all-ones / all-zero words (every word holds 32 valid sites here)
        const int byte = layout == ISING_BITPACK ? (start == 1 ? 0xFF : 0x00)
                                                 : (start == 1 ? 0x01 : 0xFF);
        cudaError_t e = cudaMemsetAsync(col0, byte, col_data_bytes, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(col1, byte, col_data_bytes, st);
        return e;
    }
    if (layout == ISING_BITPACK) {
        const RowGeom g = row_geom(L, rows, 64u);
        init_rows_packed_hot<<<grid_items(g.items, dp), 256, 0, st>>>(
            static_cast<uint32_t*>(col0), static_cast<uint32_t*>(col1), g, key0, key1);
    } else {
        const RowGeom g = row_geom(L, rows, 32u);
        init_rows_int8_hot<<<grid_items(g.items, dp), 256, 0, st>>>(
            static_cast<int8_t*>(col0), static_cast<int8_t*>(col1), g, key0, key1);
    }
    return cudaGetLastError();
}

cudaError_t rows_import(void* col0, void* col1, const int8_t* in, int layout, int L, int64_t rows,
                        int* bad_flag, const DeviceProps& dp, cudaStream_t st) {
    if (layout == ISING_BITPACK) {
        const RowGeom g = row_geom(L, rows, 64u);
        if (bad_flag)
            import_rows_packed<true><<<grid_items(g.items, dp), 256, 0, st>>>(
                static_cast<uint32_t*>(col0), static_cast<uint32_t*>(col1), in, g, bad_flag);
        else
            import_rows_packed<false><<<grid_items(g.items, dp), 256, 0, st>>>(
                static_cast<uint32_t*>(col0), static_cast<uint32_t*>(col1), in, g, nullptr);
    } else {
        const RowGeom g = row_geom(L, rows, 32u);
        if (bad_flag)
            import_rows_int8<true><<<grid_items(g.items, dp), 256, 0, st>>>(
                static_cast<int8_t*>(col0), static_cast<int8_t*>(col1), in, g, bad_flag);
        else
            import_rows_int8<false><<<grid_items(g.items, dp), 256, 0, st>>>(
                static_cast<int8_t*>(col0), static_cast<int8_t*>(col1), in, g, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t rows_export(const void* col0, const void* col1, int8_t* out, int layout, int L,
                        int64_t rows, const DeviceProps& dp, cudaStream_t st) {
    if (layout == ISING_BITPACK) {
        const RowGeom g = row_geom(L, rows, 64u);
        export_rows_packed<<<grid_items(g.items, dp), 256, 0, st>>>(
            static_cast<const uint32_t*>(col0), static_cast<const uint32_t*>(col1), out, g);
    } else {
        const RowGeom g = row_geom(L, rows, 32u);
        export_rows_int8<<<grid_items(g.items, dp), 256, 0, st>>>(
            static_cast<const int8_t*>(col0), static_cast<const int8_t*>(col1), out, g);
    }
    return cudaGetLastError();
}

cudaError_t check_spins(const int8_t* in, int64_t n, int* bad_flag, const DeviceProps& dp,
                        cudaStream_t st) {
    uint64_t b = ((uint64_t)n + 255) / 256;
    const uint64_t cap = (uint64_t)dp.sm_count * 16;
    if (b > cap) b = cap;
    check_spins_kernel<<<(unsigned)(b < 1 ? 1 : b), 256, 0, st>>>(in, n, bad_flag);
    return cudaGetLastError();
}

}  // namespace ising
