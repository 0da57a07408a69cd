// sweep_int8.cu -- colour pass of the checkerboard Metropolis sweep on the
// int8 layout, with the per-sweep E and M reductions fused in.
//
// Layout (the "two lattices, one per colour" checkerboard of Sec. 5): colour
// c's sites are stored as int8 +1 / -1 in their own array, indexed by the
// half index h = i >> 1 of canonical site i = x + L*y (+ L*L*z).  Because L is
// even, h = r*W + (x >> 1) with half-row r = y (+ L*z) and W = L/2, so each
// array is `rows` half rows of W bytes.  A colour-c site in half row r sits at
// x = 2*(h mod W) + p with p = (c + y + z) & 1, so its x-neighbours in the
// other colour's row are at h' - 1, h' (p = 0) or h', h' + 1 (p = 1); its y-
// and z-neighbours are at the same column in half rows r +- 1 (mod L within
// the plane) and r +- L (mod L*L).
//
// Site update (Sec. 2.2, Metropolis steps 1-4, integer form): with d the
// number of neighbours that disagree with s_i, k = s_i h_i = 2*(dims - d) and
// dE = 2k.  d >= dims (dE <= 0) always flips; otherwise the site flips iff its
// draw u = Philox(seed; h >> 2, t, c, 0)[h & 3] is below
// floor(exp(-2 beta k) 2^32).  Four consecutive half indices share one Philox
// call, which is exactly one 32-bit word of the colour array.
//
// Byte-sliced arithmetic: with s = 0x01 (+1) or 0xFF (-1), (s ^ n) & 0x02 is 2
// when s and n differ, so a 32-bit add of four masked xors counts 2d for four
// sites at once without carries between bytes.
#include <cstdint>

#include "engine_internal.h"
#include "ising_device.cuh"

namespace ising {

namespace {

constexpr uint32_t kBit1 = 0x02020202u;
constexpr uint32_t kBit7 = 0x80808080u;
constexpr uint32_t kOnes = 0x01010101u;

// Update four sites held in one 32-bit word (one Philox group).  n0..n5 are
// the words of the other colour that line up with the four sites' neighbours.
// Returns the new word; accumulates M (and E in the white pass).
template <int DIMS, bool MEASURE>
__device__ __forceinline__ uint32_t update_word(uint32_t s, uint32_t n0, uint32_t n1,
                                                uint32_t n2, uint32_t n3, uint32_t n4,
                                                uint32_t n5, uint32_t group,
                                                const PassArgs& a, int& e_acc, int& m_acc) {
    uint32_t D = ((s ^ n0) & kBit1) + ((s ^ n1) & kBit1) + ((s ^ n2) & kBit1) +
                 ((s ^ n3) & kBit1);
    if (DIMS == 3) D += ((s ^ n4) & kBit1) + ((s ^ n5) & kBit1);
    // byte j of D is 2*d_j; bias so that bit 7 is set iff 2*(count + d) >= 2*dims
    constexpr uint32_t bias = (0x80u - 2u * DIMS) * kOnes;
    uint32_t F = (D + bias) & kBit7;  // sites that flip without a draw
    if (F != kBit7) {
        const Philox4 u = philox4x32_10(group, a.t, (uint32_t)a.c, kTagSweep, a.key0, a.key1);
        const uint32_t cnt = below_count<DIMS>(u.w0, a) | (below_count<DIMS>(u.w1, a) << 8) |
                             (below_count<DIMS>(u.w2, a) << 16) |
                             (below_count<DIMS>(u.w3, a) << 24);
        F = (D + 2u * cnt + bias) & kBit7;
    }
    const uint32_t snew = s ^ ((F >> 7) * 0xFEu);  // 0x01 <-> 0xFF where flipped
    if (MEASURE) {
        m_acc += 4 - 2 * __popc(snew & kBit7);
        if (a.c == 1) {
            // white pass: E = -sum_white s_i h_i = sum (2 d_new - 2 dims)
            const uint32_t fmask = (F >> 7) * 0xFFu;
            constexpr uint32_t q2 = 4u * DIMS * kOnes;  // 2 * (2 dims) per byte
            const uint32_t Dn = (D & ~fmask) | ((q2 - D) & fmask);
            e_acc += (int)((Dn * kOnes) >> 24) - 8 * DIMS;
        }
    }
    return snew;
}

__device__ __forceinline__ int wrap_prev(int v, int n) { return v == 0 ? n - 1 : v - 1; }
__device__ __forceinline__ int wrap_next(int v, int n) { return v == n - 1 ? 0 : v + 1; }

// Vector kernel: W % 16 == 0.  One item = 16 sites (one uint4) of one half
// row; consecutive lanes take consecutive items, so the byte that crosses an
// item boundary in the x-shift comes from the neighbouring lane.
template <int DIMS, bool MEASURE>
__global__ void __launch_bounds__(256) pass_int8_vec(PassArgs a) {
    const int nv = a.W >> 4;
    const int64_t items = (int64_t)nv * a.rows;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int L = a.L;
    int8_t* own = static_cast<int8_t*>(a.own);
    const int8_t* other = static_cast<const int8_t*>(a.other);
    int e_acc = 0, m_acc = 0;

    // items and stride are multiples of 32, so whole warps enter each trip
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < items; g += stride) {
        const int64_t r = g / nv;
        const int v = (int)(g - r * nv);
        int y, z;
        if (DIMS == 2) {
            y = (int)r;
            z = 0;
        } else {
            z = (int)(r / L);
            y = (int)(r - (int64_t)z * L);
        }
        const int p = (a.c + y + z) & 1;
        const int64_t plane = (int64_t)z * L;
        const int64_t r_ym = plane + wrap_prev(y, L), r_yp = plane + wrap_next(y, L);

        const uint4* orow = reinterpret_cast<const uint4*>(other + r * a.W);
        const uint4 o = __ldg(orow + v);
        const uint4 oym = __ldg(reinterpret_cast<const uint4*>(other + r_ym * a.W) + v);
        const uint4 oyp = __ldg(reinterpret_cast<const uint4*>(other + r_yp * a.W) + v);
        uint4 ozm = make_uint4(0, 0, 0, 0), ozp = make_uint4(0, 0, 0, 0);
        if (DIMS == 3) {
            const int64_t r_zm = (int64_t)wrap_prev(z, L) * L + y;
            const int64_t r_zp = (int64_t)wrap_next(z, L) * L + y;
            ozm = __ldg(reinterpret_cast<const uint4*>(other + r_zm * a.W) + v);
            ozp = __ldg(reinterpret_cast<const uint4*>(other + r_zp * a.W) + v);
        }
        uint4* srow = reinterpret_cast<uint4*>(own + r * a.W);
        uint4 s = srow[v];

        // x-neighbour bytes shifted by one site
        uint32_t prev_w = __shfl_up_sync(0xffffffffu, o.w, 1);
        uint32_t next_x = __shfl_down_sync(0xffffffffu, o.x, 1);
        uint4 sh;
        if (p == 0) {
            if (lane == 0 || v == 0) prev_w = __ldg(orow + wrap_prev(v, nv)).w;
            sh.x = __funnelshift_l(prev_w, o.x, 8);
            sh.y = __funnelshift_l(o.x, o.y, 8);
            sh.z = __funnelshift_l(o.y, o.z, 8);
            sh.w = __funnelshift_l(o.z, o.w, 8);
        } else {
            if (lane == 31 || v == nv - 1) next_x = __ldg(orow + wrap_next(v, nv)).x;
            sh.x = __funnelshift_r(o.x, o.y, 8);
            sh.y = __funnelshift_r(o.y, o.z, 8);
            sh.z = __funnelshift_r(o.z, o.w, 8);
            sh.w = __funnelshift_r(o.w, next_x, 8);
        }

        const uint32_t group0 = (uint32_t)((r * a.W + 16 * v) >> 2);
        s.x = update_word<DIMS, MEASURE>(s.x, o.x, sh.x, oym.x, oyp.x, ozm.x, ozp.x, group0,
                                         a, e_acc, m_acc);
        s.y = update_word<DIMS, MEASURE>(s.y, o.y, sh.y, oym.y, oyp.y, ozm.y, ozp.y, group0 + 1,
                                         a, e_acc, m_acc);
        s.z = update_word<DIMS, MEASURE>(s.z, o.z, sh.z, oym.z, oyp.z, ozm.z, ozp.z, group0 + 2,
                                         a, e_acc, m_acc);
        s.w = update_word<DIMS, MEASURE>(s.w, o.w, sh.w, oym.w, oyp.w, ozm.w, ozp.w, group0 + 3,
                                         a, e_acc, m_acc);
        srow[v] = s;
    }
    if (MEASURE) block_reduce_add(e_acc, m_acc, a.obs, a.c == 1);
}

// General kernel: any even L.  One item = one 32-bit word (four consecutive
// half indices, one Philox group); each site finds its neighbours from its
// coordinates, so half rows need not align with words.
template <int DIMS, bool MEASURE>
__global__ void __launch_bounds__(256) pass_int8_any(PassArgs a, int64_t half_sites) {
    const int64_t words = (half_sites + 3) >> 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int L = a.L, W = a.W;
    int8_t* own = static_cast<int8_t*>(a.own);
    const int8_t* other = static_cast<const int8_t*>(a.other);
    int e_acc = 0, m_acc = 0;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += stride) {
        int s_val[4], d_val[4];
        bool valid[4], need_draw = false;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t h = 4 * w + j;
            valid[j] = h < half_sites;
            s_val[j] = 1;
            d_val[j] = DIMS;
            if (!valid[j]) continue;
            const int64_t r = h / W;
            const int xh = (int)(h - r * W);
            int y, z;
            if (DIMS == 2) {
                y = (int)r;
                z = 0;
            } else {
                z = (int)(r / L);
                y = (int)(r - (int64_t)z * L);
            }
            const int p = (a.c + y + z) & 1;
            const int x = 2 * xh + p;
            const int xm = (x == 0 ? L - 1 : x - 1) >> 1, xp = (x == L - 1 ? 0 : x + 1) >> 1;
            const int64_t plane = (int64_t)z * L;
            const int64_t rym = plane + (y == 0 ? L - 1 : y - 1);
            const int64_t ryp = plane + (y == L - 1 ? 0 : y + 1);
            const int s = own[h];
            int hsum = other[r * W + xm] + other[r * W + xp] + other[rym * W + xh] +
                       other[ryp * W + xh];
            if (DIMS == 3) {
                const int64_t rzm = (int64_t)(z == 0 ? L - 1 : z - 1) * L + y;
                const int64_t rzp = (int64_t)(z == L - 1 ? 0 : z + 1) * L + y;
                hsum += other[rzm * W + xh] + other[rzp * W + xh];
            }
            s_val[j] = s;
            d_val[j] = (2 * DIMS - s * hsum) >> 1;  // k = s*h = 2*(dims - d)
            if (d_val[j] < DIMS) need_draw = true;
        }
        uint32_t u[4] = {0u, 0u, 0u, 0u};
        if (need_draw) {
            const Philox4 q = philox4x32_10((uint32_t)w, a.t, (uint32_t)a.c, kTagSweep, a.key0,
                                            a.key1);
            u[0] = q.w0;
            u[1] = q.w1;
            u[2] = q.w2;
            u[3] = q.w3;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!valid[j]) continue;
            const bool flip = (int)below_count<DIMS>(u[j], a) + d_val[j] >= DIMS;
            const int sn = flip ? -s_val[j] : s_val[j];
            if (flip) own[4 * w + j] = (int8_t)sn;
            if (MEASURE) {
                m_acc += sn;
                if (a.c == 1) {
                    const int dn = flip ? 2 * DIMS - d_val[j] : d_val[j];
                    e_acc += 2 * dn - 2 * DIMS;
                }
            }
        }
    }
    if (MEASURE) block_reduce_add(e_acc, m_acc, a.obs, a.c == 1);
}

// Canonical <-> layout conversion and initial states.  Item = one canonical
// site; its colour array and half index follow from the coordinates.
__global__ void init_int8(int8_t* col0, int8_t* col1, int L, int dims, int64_t sites,
                          int start, uint32_t key0, uint32_t key1) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < sites; i += stride) {
        int8_t s;
        if (start == 0) {
            const Philox4 q = philox4x32_10((uint32_t)(i >> 2), 0u, 0u, kTagInit, key0, key1);
            const uint32_t words[4] = {q.w0, q.w1, q.w2, q.w3};
            s = words[i & 3] < 0x80000000u ? 1 : -1;
        } else {
            s = start == 1 ? 1 : -1;
        }
        const int64_t x = i % L, rest = i / L;
        const int64_t y = rest % L, z = dims == 3 ? rest / L : 0;
        const int c = (int)((x + y + z) & 1);
        (c == 0 ? col0 : col1)[i >> 1] = s;
    }
}

__global__ void export_int8(const int8_t* col0, const int8_t* col1, int8_t* out, int L,
                            int dims, int64_t sites) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < sites; i += stride) {
        const int64_t x = i % L, rest = i / L;
        const int64_t y = rest % L, z = dims == 3 ? rest / L : 0;
        out[i] = (((x + y + z) & 1) == 0 ? col0 : col1)[i >> 1];
    }
}

__global__ void import_int8(int8_t* col0, int8_t* col1, const int8_t* in, int L, int dims,
                            int64_t sites) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < sites; i += stride) {
        const int64_t x = i % L, rest = i / L;
        const int64_t y = rest % L, z = dims == 3 ? rest / L : 0;
        (((x + y + z) & 1) == 0 ? col0 : col1)[i >> 1] = in[i];
    }
}

template <int DIMS, bool MEASURE>
cudaError_t launch_pass_t(const PassArgs& a, int64_t half_sites, bool vec, const DeviceProps& dp,
                          cudaStream_t st) {
    const int threads = 256;
    if (vec) {
        const int64_t items = (int64_t)(a.W >> 4) * a.rows;
        int64_t blocks = (items + threads - 1) / threads;
        const int64_t cap = (int64_t)dp.sm_count * dp.blocks_per_sm_vec[DIMS - 2][MEASURE];
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        pass_int8_vec<DIMS, MEASURE><<<(unsigned)blocks, threads, 0, st>>>(a);
    } else {
        const int64_t words = (half_sites + 3) >> 2;
        int64_t blocks = (words + threads - 1) / threads;
        const int64_t cap = (int64_t)dp.sm_count * 8;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        pass_int8_any<DIMS, MEASURE><<<(unsigned)blocks, threads, 0, st>>>(a, half_sites);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t int8_query_occupancy(DeviceProps& dp) {
    cudaError_t e;
#define ISING_OCC(D, M)                                                                      \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&dp.blocks_per_sm_vec[D - 2][M],        \
                                                      pass_int8_vec<D, M>, 256, 0);           \
    if (e != cudaSuccess) return e;
    ISING_OCC(2, false)
    ISING_OCC(2, true)
    ISING_OCC(3, false)
    ISING_OCC(3, true)
#undef ISING_OCC
    return cudaSuccess;
}

bool int8_vec_ok(int L) { return (L / 2) % 16 == 0; }

cudaError_t int8_pass(const PassArgs& a, int dims, int64_t half_sites, bool measure,
                      const DeviceProps& dp, cudaStream_t st) {
    const bool vec = (a.W % 16) == 0;
    if (dims == 2)
        return measure ? launch_pass_t<2, true>(a, half_sites, vec, dp, st)
                       : launch_pass_t<2, false>(a, half_sites, vec, dp, st);
    return measure ? launch_pass_t<3, true>(a, half_sites, vec, dp, st)
                   : launch_pass_t<3, false>(a, half_sites, vec, dp, st);
}

static unsigned grid_for(int64_t n, const DeviceProps& dp) {
    int64_t b = (n + 255) / 256;
    const int64_t cap = (int64_t)dp.sm_count * 16;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t int8_init(int8_t* col0, int8_t* col1, int L, int dims, int64_t sites, int start,
                      uint32_t key0, uint32_t key1, const DeviceProps& dp, cudaStream_t st) {
    init_int8<<<grid_for(sites, dp), 256, 0, st>>>(col0, col1, L, dims, sites, start, key0,
                                                    key1);
    return cudaGetLastError();
}

cudaError_t int8_export(const int8_t* col0, const int8_t* col1, int8_t* out, int L, int dims,
                        int64_t sites, const DeviceProps& dp, cudaStream_t st) {
    export_int8<<<grid_for(sites, dp), 256, 0, st>>>(col0, col1, out, L, dims, sites);
    return cudaGetLastError();
}

cudaError_t int8_import(int8_t* col0, int8_t* col1, const int8_t* in, int L, int dims,
                        int64_t sites, const DeviceProps& dp, cudaStream_t st) {
    import_int8<<<grid_for(sites, dp), 256, 0, st>>>(col0, col1, in, L, dims, sites);
    return cudaGetLastError();
}

}  // namespace ising
