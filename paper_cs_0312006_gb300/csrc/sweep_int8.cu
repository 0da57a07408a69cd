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
#include "pass_bodies.cuh"

namespace ising {

namespace {

__device__ __forceinline__ int wrap_prev(int v, int n) { return v == 0 ? n - 1 : v - 1; }
__device__ __forceinline__ int wrap_next(int v, int n) { return v == n - 1 ? 0 : v + 1; }

// Strip kernel: W % 16 == 0.  Each thread owns one 16-byte column v of the
// colour arrays and walks a strip of consecutive half rows, keeping the other
// colour's rows y-1, y, y+1 of its column in registers (a sliding window) and
// prefetching the next row's data before computing the current one.  Lanes
// hold consecutive columns, so the byte that crosses a column boundary in the
// x-shift comes from the neighbouring lane.  Strips are as balanced as the
// row count allows; a strip that reaches the end of a plane reloads its
// window for the next plane.
template <int DIMS, bool MEASURE, int RULE>
__global__ void __launch_bounds__(256, DIMS == 2 ? 4 : 2) pass_int8_strip(PassArgs a) {
    const int nv = a.nv, S = a.strips, L = a.L;
    const int rows = (int)a.rows;
    const int lane = threadIdx.x & 31;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = tid < S * nv;
    const int sidx = active ? tid / nv : 0;
    const int v = active ? tid - sidx * nv : 0;
    const int r_begin = (int)(((int64_t)sidx * rows) / S);
    const int len = active ? (int)(((int64_t)(sidx + 1) * rows) / S) - r_begin : 0;
    const int max_len = (rows + S - 1) / S;
    const uint4* __restrict__ O = reinterpret_cast<const uint4*>(a.other) + v;
    uint4* __restrict__ Sv = reinterpret_cast<uint4*>(a.own) + v;
    const uint32_t* __restrict__ Ow = reinterpret_cast<const uint32_t*>(a.other);
    const uint32_t vm_word = 4u * (uint32_t)wrap_prev(v, nv) + 3u;  // last word of column v-1
    const uint32_t vp_word = 4u * (uint32_t)wrap_next(v, nv);       // first word of column v+1

    int z = DIMS == 3 ? r_begin / L : 0;
    int y = r_begin - z * L;
    int plane = z * L, plane_m = 0, plane_p = 0;
    if (DIMS == 3) {
        plane_m = wrap_prev(z, L) * L;
        plane_p = wrap_next(z, L) * L;
    }
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    uint4 om = zero, oc = zero, op = zero, sc = zero, zm = zero, zp = zero;
    bool reload = true;
    int e_acc = 0, m_neg = 0, n_rows = 0;
    grid_dependency_wait();
    launch_dependents();

    for (int i = 0; i < max_len; ++i) {
        const bool valid = i < len;
        const int r = r_begin + i;
        if (valid && reload) {
            om = __ldg(O + (uint32_t)(plane + wrap_prev(y, L)) * nv);
            oc = __ldg(O + (uint32_t)r * nv);
            op = __ldg(O + (uint32_t)(plane + wrap_next(y, L)) * nv);
            sc = Sv[(uint32_t)r * nv];
            if (DIMS == 3) {
                zm = __ldg(O + (uint32_t)(plane_m + y) * nv);
                zp = __ldg(O + (uint32_t)(plane_p + y) * nv);
            }
        }
        // prefetch row r + 1 while it stays in this plane
        const bool pf = (i + 1 < len) && (y + 1 < L);
        uint4 op_n = zero, sc_n = zero, zm_n = zero, zp_n = zero;
        if (pf) {
            op_n = __ldg(O + (uint32_t)(plane + (y + 2 < L ? y + 2 : y + 2 - L)) * nv);
            sc_n = Sv[(uint32_t)(r + 1) * nv];
            if (DIMS == 3) {
                zm_n = __ldg(O + (uint32_t)(plane_m + y + 1) * nv);
                zp_n = __ldg(O + (uint32_t)(plane_p + y + 1) * nv);
            }
        }
        // x-neighbour bytes shifted by one site (all lanes take part in the shuffles)
        uint32_t prev_w = __shfl_up_sync(0xffffffffu, oc.w, 1);
        uint32_t next_x = __shfl_down_sync(0xffffffffu, oc.x, 1);
        if (valid) {
            const int p = (a.c + y + z) & 1;
            uint4 sh;
            if (p == 0) {
                if (lane == 0 || v == 0) prev_w = __ldg(Ow + (uint32_t)r * nv * 4u + vm_word);
                sh.x = __funnelshift_l(prev_w, oc.x, 8);
                sh.y = __funnelshift_l(oc.x, oc.y, 8);
                sh.z = __funnelshift_l(oc.y, oc.z, 8);
                sh.w = __funnelshift_l(oc.z, oc.w, 8);
            } else {
                if (lane == 31 || v == nv - 1) next_x = __ldg(Ow + (uint32_t)r * nv * 4u + vp_word);
                sh.x = __funnelshift_r(oc.x, oc.y, 8);
                sh.y = __funnelshift_r(oc.y, oc.z, 8);
                sh.z = __funnelshift_r(oc.z, oc.w, 8);
                sh.w = __funnelshift_r(oc.w, next_x, 8);
            }
            const uint32_t g0 = ((uint32_t)r * nv + (uint32_t)v) * 4u;  // Philox group of word 0
            const uint4 s = update_vec<DIMS, MEASURE, RULE>(sc, oc, sh, om, op, zm, zp, g0, a,
                                                            e_acc, m_neg);
            Sv[(uint32_t)r * nv] = s;
            ++n_rows;
        }
        // slide the window
        if (pf) {
            om = oc;
            oc = op;
            op = op_n;
            sc = sc_n;
            zm = zm_n;
            zp = zp_n;
        }
        reload = !pf;
        if (++y == L) {
            y = 0;
            ++z;
            plane += L;
            if (DIMS == 3) {
                plane_m = wrap_prev(z, L) * L;
                plane_p = wrap_next(z, L) * L;
            }
        }
    }
    if (MEASURE) {
        e_acc -= n_rows * 16 * 2 * DIMS;          // E_white = sum_j (2 d_new_j - 2 dims)
        const int m_acc = n_rows * 16 - 2 * m_neg;  // sum of the new spins
        block_reduce_add(e_acc, m_acc, a.obs, a.c == 1);
    }
}

// General kernel: any even L.  One item = one 16-byte vector of the colour
// array (16 consecutive half indices, four Philox groups); see int8_vec().
template <int DIMS, bool MEASURE, int RULE>
__global__ void __launch_bounds__(256) pass_int8_vecs(PassArgs a, WordGeom g) {
    const uint32_t vecs = (g.half + 15u) >> 4;
    const uint32_t stride = gridDim.x * blockDim.x;
    int e_acc = 0, m_neg = 0, n_sites = 0;
    grid_dependency_wait();
    launch_dependents();
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < vecs; v += stride)
        int8_vec<DIMS, MEASURE, 1, RULE>(a, g, v, e_acc, m_neg, n_sites);
    if (MEASURE) block_reduce_add(e_acc, n_sites - 2 * m_neg, a.obs, a.c == 1);
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

template <int DIMS, bool MEASURE, int RULE>
cudaError_t launch_pass_t(const PassArgs& a0, int64_t half_sites, bool vec, const DeviceProps& dp,
                          cudaStream_t st) {
    const int threads = 256;
    if (vec) {
        PassArgs a = a0;
        a.nv = a.W >> 4;
        // one wave of resident threads, each walking a strip of rows of one column
        const int64_t resident =
            (int64_t)dp.sm_count * dp.blocks_per_sm_vec[RULE][DIMS - 2][MEASURE] * threads;
        int64_t strips = resident / a.nv;
        if (strips > a.rows) strips = a.rows;
        if (strips < 1) strips = 1;
        a.strips = (int)strips;
        const int64_t blocks = (strips * a.nv + threads - 1) / threads;
        return launch_chained(pass_int8_strip<DIMS, MEASURE, RULE>, (unsigned)blocks,
                              (unsigned)threads, 0, st, a);
    } else {
        const int64_t vecs = (half_sites + 15) >> 4;
        int64_t blocks = (vecs + threads - 1) / threads;
        const int64_t cap = (int64_t)dp.sm_count * 8;
        if (blocks > cap) blocks = cap;
        if (blocks < 1) blocks = 1;
        WordGeom g;
        g.W = (uint32_t)a0.W;
        g.L = (uint32_t)a0.L;
        g.rows = (uint32_t)a0.rows;
        g.half = (uint32_t)half_sites;
        return launch_chained(pass_int8_vecs<DIMS, MEASURE, RULE>, (unsigned)blocks,
                              (unsigned)threads, 0, st, a0, g);
    }
}

}  // namespace

// Philox4x32-10 blocks for counters (c0, c1, c2, c3), c0 = 0..n-1 under key
// (key0, key1): out[4 c0 + j] = word j.  Used to pin the device generator and
// to measure its throughput.
__global__ void philox_fill_kernel(uint4* out, uint32_t n, uint32_t c1, uint32_t c2, uint32_t c3,
                                   uint32_t key0, uint32_t key1) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const Philox4 u = philox4x32_10(i, c1, c2, c3, key0, key1);
        out[i] = make_uint4(u.w0, u.w1, u.w2, u.w3);
    }
}

// Throughput probe of the generator: each thread runs `iters` rounds of CHAINS
// independent calls (counters gid * iters * CHAINS + k, the sweep-like words
// c1 = t, c2 = c = 0, c3 = 0), folds all four output words of every call into
// a register and stores one word at the end, so stores and launch overhead
// vanish against the arithmetic.  VARIANT 0 is the engine's form, 1 the
// split-multiply form.
template <int VARIANT, int CHAINS>
__global__ void __launch_bounds__(256) philox_probe_kernel(uint32_t* out, uint32_t iters,
                                                           uint32_t c1, uint32_t key0,
                                                           uint32_t key1) {
    const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) acc[k] = 0u;
    uint32_t ctr = gid * iters * (uint32_t)CHAINS;
#pragma unroll 1
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) {
            const Philox4 u =
                VARIANT == 0 ? philox4x32_10(ctr + (uint32_t)k, c1, 0u, kTagSweep, key0, key1)
                             : philox4x32_10_split(ctr + (uint32_t)k, c1, 0u, kTagSweep, key0,
                                                   key1);
            acc[k] ^= u.w0 ^ u.w1 ^ u.w2 ^ u.w3;
        }
        ctr += (uint32_t)CHAINS;
    }
    uint32_t r = 0u;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) r ^= acc[k];
    out[gid] = r;
}

cudaError_t philox_probe(uint32_t* out, int blocks, int threads, uint32_t iters, int variant,
                         int chains, uint32_t c1, uint32_t key0, uint32_t key1, cudaStream_t st) {
#define ISING_PROBE(V, C)                                                                  \
    if (variant == V && chains == C) {                                                     \
        philox_probe_kernel<V, C><<<(unsigned)blocks, (unsigned)threads, 0, st>>>(out, iters, \
                                                                                  c1, key0, key1); \
        return cudaGetLastError();                                                         \
    }
    ISING_PROBE(0, 4)
    ISING_PROBE(0, 8)
    ISING_PROBE(1, 4)
    ISING_PROBE(1, 8)
#undef ISING_PROBE
    return cudaErrorInvalidValue;
}

cudaError_t int8_query_occupancy(DeviceProps& dp) {
    cudaError_t e;
#define ISING_OCC(R, D, M)                                                                   \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&dp.blocks_per_sm_vec[R][D - 2][M],     \
                                                      pass_int8_strip<D, M, R>, 256, 0);        \
    if (e != cudaSuccess) return e;
    ISING_OCC(kRuleMetropolis, 2, false)
    ISING_OCC(kRuleMetropolis, 2, true)
    ISING_OCC(kRuleMetropolis, 3, false)
    ISING_OCC(kRuleMetropolis, 3, true)
    ISING_OCC(kRuleHeatBath, 2, false)
    ISING_OCC(kRuleHeatBath, 2, true)
    ISING_OCC(kRuleHeatBath, 3, false)
    ISING_OCC(kRuleHeatBath, 3, true)
    ISING_OCC(kRuleMultiHit, 2, false)
    ISING_OCC(kRuleMultiHit, 2, true)
    ISING_OCC(kRuleMultiHit, 3, false)
    ISING_OCC(kRuleMultiHit, 3, true)
#undef ISING_OCC
    return cudaSuccess;
}

bool int8_vec_ok(int L) { return (L / 2) % 16 == 0; }

cudaError_t philox_fill(uint32_t* out, uint32_t n, uint32_t c1, uint32_t c2, uint32_t c3,
                        uint32_t key0, uint32_t key1, const DeviceProps& dp, cudaStream_t st) {
    int64_t blocks = ((int64_t)n + 255) / 256;
    const int64_t cap = (int64_t)dp.sm_count * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    philox_fill_kernel<<<(unsigned)blocks, 256, 0, st>>>(reinterpret_cast<uint4*>(out), n, c1, c2,
                                                          c3, key0, key1);
    return cudaGetLastError();
}

template <int RULE>
cudaError_t int8_pass_rule(const PassArgs& a, int dims, int64_t half_sites, bool measure,
                           const DeviceProps& dp, cudaStream_t st) {
    const bool vec = (a.W % 16) == 0;
    if (dims == 2)
        return measure ? launch_pass_t<2, true, RULE>(a, half_sites, vec, dp, st)
                       : launch_pass_t<2, false, RULE>(a, half_sites, vec, dp, st);
    return measure ? launch_pass_t<3, true, RULE>(a, half_sites, vec, dp, st)
                   : launch_pass_t<3, false, RULE>(a, half_sites, vec, dp, st);
}

cudaError_t int8_pass(const PassArgs& a, int dims, int64_t half_sites, bool measure, int rule,
                      const DeviceProps& dp, cudaStream_t st) {
    if (rule == kRuleHeatBath)
        return int8_pass_rule<kRuleHeatBath>(a, dims, half_sites, measure, dp, st);
    if (rule == kRuleMultiHit)
        return int8_pass_rule<kRuleMultiHit>(a, dims, half_sites, measure, dp, st);
    return int8_pass_rule<kRuleMetropolis>(a, dims, half_sites, measure, dp, st);
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
