// sweep_demon.cu -- colour pass of Creutz's deterministic demon dynamics on
// the int8 layout, with the E and M reductions fused in.
//
// Sec. 2.2 cites Creutz's checkerboard simulation with a fully deterministic
// flip rule that needs no random numbers.  Here every site carries a demon
// holding energy 4q, q = 0..qmax, stored as one byte per site in two arrays
// laid out like the spins (one per colour, half rows of W = L/2 bytes).  A
// site with d disagreeing neighbours (flip cost dE = 4 (dims - d)) flips iff
// 0 <= q - (dims - d) <= qmax, and its demon then keeps q - (dims - d), so
// E + 4 sum q is conserved.  After each sweep every demon moves one half row
// on within its colour (half row r, half column xh -> half row r + 1, same
// xh).  Nothing is moved in memory: the demon of half row r sits in storage
// row (r - rot) mod rows, and rot grows by one per sweep.
//
// With no draw the pass is a pure stream: it reads the own spins, the own
// demons and the other colour and writes the own spins and demons, 5 bytes
// per site update.
//
// Byte-sliced arithmetic (four sites per 32-bit word, no carries between
// bytes): D = 2d per byte as in the Metropolis pass; v = q + d per byte; the
// flip condition dims <= v <= dims + qmax is bit 7 of v + (0x80 - dims) and
// not bit 7 of v + (0x80 - dims - qmax - 1); the new demon is v - dims.
//
// Bit-packed layout (multispin coding, as Creutz's own code): qmax = 3, the
// demons held as two bit planes (q = q0 + 2 q1) laid out like the spin words;
// d comes as three bit planes from the bit-sliced neighbour count, v = q + d
// by a bit-sliced adder, and the range test and v - dims are fixed logic on
// the bits of v.  Per site update a pass moves 7 bits: own spin, other
// colour's spin and two demon bits read, own spin and two demon bits written.
#include <cstdint>

#include "engine_internal.h"
#include "ising_device.cuh"
#include "pass_bodies.cuh"

namespace ising {

namespace {

__device__ __forceinline__ int wrap_prev(int v, int n) { return v == 0 ? n - 1 : v - 1; }
__device__ __forceinline__ int wrap_next(int v, int n) { return v == n - 1 ? 0 : v + 1; }

// Update four sites (one word): spins s, demons q, byte-sliced D = 2d.
// Returns the flip mask (0xFE per flipped byte) and updates q in place.
template <int DIMS>
__device__ __forceinline__ uint32_t demon_word(uint32_t D, uint32_t& q, uint32_t lo_bias,
                                               uint32_t hi_bias) {
    const uint32_t v = q + (D >> 1);  // q + d per byte (D's bytes are even)
    const uint32_t F = (v + lo_bias) & ~(v + hi_bias) & kByteBit7;
    const uint32_t keep = F | (F - (F >> 7));  // 0xFF per flipped byte
    // v - dims per byte, without borrows between bytes (every byte of v is < 0x80)
    const uint32_t vn = ((v | kByteBit7) - (uint32_t)DIMS * kByteOnes) & 0x7F7F7F7Fu;
    q = (q & ~keep) | (vn & keep);
    return F | (F - (F >> 6));  // 0xFE per flipped byte
}

// The 16 sites of one vector; accumulates -1 spins written (m_neg) and, in the
// white pass, sum 2 d_new (e_acc).
template <int DIMS, bool MEASURE>
__device__ __forceinline__ uint4 demon_vec(const uint4& s, uint4& qv, const uint4& x,
                                           const uint4& xs, const uint4& ym, const uint4& yp,
                                           const uint4& zm, const uint4& zp, uint32_t lo_bias,
                                           uint32_t hi_bias, int c, int& e_acc, int& m_neg) {
    const uint32_t sv[4] = {s.x, s.y, s.z, s.w};
    uint32_t D[4], X[4], q[4] = {qv.x, qv.y, qv.z, qv.w};
    D[0] = disagreements<DIMS>(s.x, x.x, xs.x, ym.x, yp.x, zm.x, zp.x);
    D[1] = disagreements<DIMS>(s.y, x.y, xs.y, ym.y, yp.y, zm.y, zp.y);
    D[2] = disagreements<DIMS>(s.z, x.z, xs.z, ym.z, yp.z, zm.z, zp.z);
    D[3] = disagreements<DIMS>(s.w, x.w, xs.w, ym.w, yp.w, zm.w, zp.w);
    uint32_t out[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        X[w] = demon_word<DIMS>(D[w], q[w], lo_bias, hi_bias);
        out[w] = sv[w] ^ X[w];
        if (MEASURE) {
            m_neg += __popc(out[w] & kByteBit7);
            if (c == 1) {
                constexpr uint32_t q2 = 4u * DIMS * kByteOnes;
                const uint32_t Dn = (D[w] & ~X[w]) | ((q2 - D[w]) & X[w]);
                e_acc = __dp4a((int)Dn, (int)kByteOnes, e_acc);
            }
        }
    }
    qv = make_uint4(q[0], q[1], q[2], q[3]);
    return make_uint4(out[0], out[1], out[2], out[3]);
}

// W % 16 == 0: the register-window strip walk of the Metropolis strip kernel,
// with the own demons streamed beside the own spins.  The pass is a memory
// stream, so occupancy is what keeps loads in flight: in 2D at most 64
// registers (four CTAs per SM) measured 0.869 of the copy bandwidth at
// L = 32768 against 0.828 with 73 registers and three CTAs; 3D keeps three
// CTAs (at 64 registers it would spill).
template <int DIMS, bool MEASURE>
__global__ void __launch_bounds__(256, DIMS == 2 ? 4 : 3) pass_demon_strip(PassArgs a) {
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
    uint4* __restrict__ Q = reinterpret_cast<uint4*>(a.dem) + v;
    const uint32_t* __restrict__ Ow = reinterpret_cast<const uint32_t*>(a.other);
    const uint32_t vm_word = 4u * (uint32_t)wrap_prev(v, nv) + 3u;
    const uint32_t vp_word = 4u * (uint32_t)wrap_next(v, nv);
    const uint32_t lo_bias = (0x80u - (uint32_t)DIMS) * kByteOnes;
    const uint32_t hi_bias = (0x80u - (uint32_t)DIMS - (uint32_t)a.qmax - 1u) * kByteOnes;

    int z = DIMS == 3 ? r_begin / L : 0;
    int y = r_begin - z * L;
    int plane = z * L, plane_m = 0, plane_p = 0;
    if (DIMS == 3) {
        plane_m = wrap_prev(z, L) * L;
        plane_p = wrap_next(z, L) * L;
    }
    // storage row of half row r's demons
    int rd = r_begin - (int)a.rot;
    if (rd < 0) rd += rows;
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    uint4 om = zero, oc = zero, op = zero, sc = zero, qc = zero, zm = zero, zp = zero;
    bool reload = true;
    int e_acc = 0, m_neg = 0, n_rows = 0;
    grid_dependency_wait();
    launch_dependents();

    for (int i = 0; i < max_len; ++i) {
        const bool valid = i < len;
        const int r = r_begin + i;
        const int rd_next = rd + 1 == rows ? 0 : rd + 1;
        if (valid && reload) {
            om = __ldg(O + (uint32_t)(plane + wrap_prev(y, L)) * nv);
            oc = __ldg(O + (uint32_t)r * nv);
            op = __ldg(O + (uint32_t)(plane + wrap_next(y, L)) * nv);
            sc = Sv[(uint32_t)r * nv];
            qc = Q[(uint32_t)rd * nv];
            if (DIMS == 3) {
                zm = __ldg(O + (uint32_t)(plane_m + y) * nv);
                zp = __ldg(O + (uint32_t)(plane_p + y) * nv);
            }
        }
        // prefetch row r + 1 while it stays in this plane
        const bool pf = (i + 1 < len) && (y + 1 < L);
        uint4 op_n = zero, sc_n = zero, qc_n = zero, zm_n = zero, zp_n = zero;
        if (pf) {
            op_n = __ldg(O + (uint32_t)(plane + (y + 2 < L ? y + 2 : y + 2 - L)) * nv);
            sc_n = Sv[(uint32_t)(r + 1) * nv];
            qc_n = Q[(uint32_t)rd_next * nv];
            if (DIMS == 3) {
                zm_n = __ldg(O + (uint32_t)(plane_m + y + 1) * nv);
                zp_n = __ldg(O + (uint32_t)(plane_p + y + 1) * nv);
            }
        }
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
            const uint4 s = demon_vec<DIMS, MEASURE>(sc, qc, oc, sh, om, op, zm, zp, lo_bias,
                                                     hi_bias, a.c, e_acc, m_neg);
            Sv[(uint32_t)r * nv] = s;
            Q[(uint32_t)rd * nv] = qc;
            ++n_rows;
        }
        if (pf) {
            om = oc;
            oc = op;
            op = op_n;
            sc = sc_n;
            qc = qc_n;
            zm = zm_n;
            zp = zp_n;
        }
        reload = !pf;
        rd = rd_next;
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
        e_acc -= n_rows * 16 * 2 * DIMS;
        const int m_acc = n_rows * 16 - 2 * m_neg;
        block_reduce_add(e_acc, m_acc, a.obs, a.c == 1);
    }
}

// Any even L: one site per item, neighbours found from the coordinates.
template <int DIMS, bool MEASURE>
__global__ void __launch_bounds__(256) pass_demon_sites(PassArgs a, uint32_t half) {
    const int8_t* other = static_cast<const int8_t*>(a.other);
    int8_t* own = static_cast<int8_t*>(a.own);
    uint8_t* dem = static_cast<uint8_t*>(a.dem);
    const uint32_t W = (uint32_t)a.W, L = (uint32_t)a.L, rows = (uint32_t)a.rows;
    const uint32_t stride = gridDim.x * blockDim.x;
    int e_acc = 0, m_acc = 0;
    grid_dependency_wait();
    launch_dependents();
    for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < half; h += stride) {
        const uint32_t r = h / W, xh = h - r * W;
        uint32_t y = r, z = 0;
        if (DIMS == 3) {
            z = r / L;
            y = r - z * L;
        }
        const uint32_t p = ((uint32_t)a.c + y + z) & 1u;
        const uint32_t x = 2u * xh + p;
        const uint32_t xm = (x == 0u ? L - 1u : x - 1u) >> 1;
        const uint32_t xp = (x + 1u == L ? 0u : x + 1u) >> 1;
        const uint32_t plane = z * L;
        const uint32_t rym = plane + (y == 0u ? L - 1u : y - 1u);
        const uint32_t ryp = plane + (y + 1u == L ? 0u : y + 1u);
        int hs = other[r * W + xm] + other[r * W + xp] + other[rym * W + xh] + other[ryp * W + xh];
        if (DIMS == 3) {
            const uint32_t rzm = (z == 0u ? L - 1u : z - 1u) * L + y;
            const uint32_t rzp = (z + 1u == L ? 0u : z + 1u) * L + y;
            hs += other[rzm * W + xh] + other[rzp * W + xh];
        }
        const int s = own[h];
        const int delta = (s * hs) / 2;  // dims - d
        const uint32_t rd = r >= a.rot ? r - a.rot : r + rows - a.rot;
        const uint32_t qi = rd * W + xh;
        const int qn = (int)dem[qi] - delta;
        int sn = s;
        if (qn >= 0 && qn <= a.qmax) {
            sn = -s;
            own[h] = (int8_t)sn;
            dem[qi] = (uint8_t)qn;
        }
        if (MEASURE) {
            m_acc += sn;
            if (a.c == 1) e_acc -= sn * hs;  // the white pass sums every bond once
        }
    }
    if (MEASURE) block_reduce_add(e_acc, m_acc, a.obs, a.c == 1);
}

// Demons in canonical order <-> the two storage arrays (storage row of half
// row r is (r - rot) mod rows).
__global__ void export_demons_kernel(const uint8_t* d0, const uint8_t* d1, uint8_t* out, int L,
                                     int dims, int64_t sites, int64_t rows, int64_t rot) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t W = L / 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < sites; i += stride) {
        const int64_t x = i % L, r = i / L;  // r = y + L z
        const int64_t y = r % L, z = dims == 3 ? r / L : 0;
        int64_t rd = r - rot;
        if (rd < 0) rd += rows;
        out[i] = (((x + y + z) & 1) == 0 ? d0 : d1)[rd * W + (x >> 1)];
    }
}

__global__ void import_demons_kernel(uint8_t* d0, uint8_t* d1, const uint8_t* in, int L, int dims,
                                     int64_t sites) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < sites; i += stride) {
        const int64_t x = i % L, rest = i / L;
        const int64_t y = rest % L, z = dims == 3 ? rest / L : 0;
        (((x + y + z) & 1) == 0 ? d0 : d1)[i >> 1] = in[i];
    }
}

// The demon rule on one packed word: spins s, neighbour words, demon planes
// q0 / q1 (updated in place); returns the flip mask (within `valid`).
template <int DIMS>
__device__ __forceinline__ uint32_t demon_packed_bits(uint32_t s, uint32_t o, uint32_t sh,
                                                      uint32_t oym, uint32_t oyp, uint32_t ozm,
                                                      uint32_t ozp, uint32_t valid, uint32_t& q0,
                                                      uint32_t& q1) {
    const Digits d = DIMS == 2 ? digits2(s ^ o, s ^ sh, s ^ oym, s ^ oyp)
                               : digits3(s ^ o, s ^ sh, s ^ oym, s ^ oyp, s ^ ozm, s ^ ozp);
    // v = q + d, bit-sliced
    const uint32_t v0 = q0 ^ d.d0, c0 = q0 & d.d0;
    const uint32_t v1 = q1 ^ d.d1 ^ c0, c1 = (q1 & d.d1) | (c0 & (q1 ^ d.d1));
    const uint32_t v2 = d.d2 ^ c1, v3 = d.d2 & c1;
    uint32_t flip, n0, n1;
    if (DIMS == 2) {  // 2 <= v <= 5 (v <= 7 here: v3 = 0); q' = v - 2
        flip = (v1 | v2) & ~(v1 & v2);
        n0 = v0;
        n1 = v2;
    } else {          // 3 <= v <= 6; q' = v - 3
        flip = (v3 | v2 | (v1 & v0)) & ~(v3 | (v2 & v1 & v0));
        n0 = ~v0;
        n1 = v2 & (v0 | v1);
    }
    flip &= valid;
    q0 = (q0 & ~flip) | (n0 & flip);
    q1 = (q1 & ~flip) | (n1 & flip);
    return flip;
}

template <int DIMS>
__device__ __forceinline__ void demon_packed_measure(uint32_t snew, uint32_t o, uint32_t sh,
                                                     uint32_t oym, uint32_t oyp, uint32_t ozm,
                                                     uint32_t ozp, uint32_t valid, uint32_t nb,
                                                     int c, int& e_acc, int& m_acc) {
    m_acc += 2 * __popc(snew & valid) - (int)nb;
    if (c == 1) {
        int dsum = __popc((snew ^ o) & valid) + __popc((snew ^ sh) & valid) +
                   __popc((snew ^ oym) & valid) + __popc((snew ^ oyp) & valid);
        if (DIMS == 3) dsum += __popc((snew ^ ozm) & valid) + __popc((snew ^ ozp) & valid);
        e_acc += 2 * dsum - (int)nb * 2 * DIMS;
    }
}

// Rows of whole 16-byte groups (W % 128 == 0): four consecutive words per
// item, every stream read and written as 16-byte vectors.
template <int DIMS, bool MEASURE>
__global__ void __launch_bounds__(256) pass_demon_packed4(PassArgs a) {
    const uint32_t W = (uint32_t)a.W, L = (uint32_t)a.L, rows = (uint32_t)a.rows;
    const uint32_t nq = W >> 5, n4 = nq >> 2;
    const uint32_t items = rows * n4, words = rows * nq;
    uint4* own = static_cast<uint4*>(a.own);
    const uint4* other = static_cast<const uint4*>(a.other);
    const uint32_t* other_w = static_cast<const uint32_t*>(a.other);
    uint4* Q0 = static_cast<uint4*>(a.dem);
    uint4* Q1 = reinterpret_cast<uint4*>(static_cast<uint32_t*>(a.dem) + words);
    const uint32_t stride = gridDim.x * blockDim.x;
    int e_acc = 0, m_acc = 0;
    grid_dependency_wait();
    launch_dependents();
    for (uint32_t item = blockIdx.x * blockDim.x + threadIdx.x; item < items; item += stride) {
        const uint32_t r = item / n4, g = item - r * n4;
        uint32_t y = r, z = 0u;
        if (DIMS == 3) {
            z = r / L;
            y = r - z * L;
        }
        const uint32_t plane = z * L;
        const uint4 o = __ldg(other + r * n4 + g);
        const uint4 oym = __ldg(other + (plane + (y == 0u ? L - 1u : y - 1u)) * n4 + g);
        const uint4 oyp = __ldg(other + (plane + (y + 1u == L ? 0u : y + 1u)) * n4 + g);
        uint4 ozm = make_uint4(0u, 0u, 0u, 0u), ozp = ozm;
        if (DIMS == 3) {
            ozm = __ldg(other + ((z == 0u ? L - 1u : z - 1u) * L + y) * n4 + g);
            ozp = __ldg(other + ((z + 1u == L ? 0u : z + 1u) * L + y) * n4 + g);
        }
        const uint4 sv = own[r * n4 + g];
        const uint32_t rd = r >= a.rot ? r - a.rot : r + rows - a.rot;  // storage row
        uint4 qa = Q0[rd * n4 + g], qb = Q1[rd * n4 + g];
        const int p = (a.c + (int)y + (int)z) & 1;
        const uint32_t row = r * nq;
        uint4 sh;
        if (p == 0) {  // bit b <- neighbour xh - 1; word 0 takes the previous word's bit 31
            const uint32_t prev = g == 0u ? __ldg(other_w + row + nq - 1u)
                                          : __ldg(other_w + row + 4u * g - 1u);
            sh = make_uint4(__funnelshift_l(prev, o.x, 1), __funnelshift_l(o.x, o.y, 1),
                            __funnelshift_l(o.y, o.z, 1), __funnelshift_l(o.z, o.w, 1));
        } else {       // bit b <- neighbour xh + 1
            const uint32_t next = g + 1u == n4 ? __ldg(other_w + row) : __ldg(other_w + row + 4u * g + 4u);
            sh = make_uint4(__funnelshift_r(o.x, o.y, 1), __funnelshift_r(o.y, o.z, 1),
                            __funnelshift_r(o.z, o.w, 1), __funnelshift_r(o.w, next, 1));
        }
        const uint32_t fx = demon_packed_bits<DIMS>(sv.x, o.x, sh.x, oym.x, oyp.x, ozm.x, ozp.x,
                                                    0xFFFFFFFFu, qa.x, qb.x);
        const uint32_t fy = demon_packed_bits<DIMS>(sv.y, o.y, sh.y, oym.y, oyp.y, ozm.y, ozp.y,
                                                    0xFFFFFFFFu, qa.y, qb.y);
        const uint32_t fz = demon_packed_bits<DIMS>(sv.z, o.z, sh.z, oym.z, oyp.z, ozm.z, ozp.z,
                                                    0xFFFFFFFFu, qa.z, qb.z);
        const uint32_t fw = demon_packed_bits<DIMS>(sv.w, o.w, sh.w, oym.w, oyp.w, ozm.w, ozp.w,
                                                    0xFFFFFFFFu, qa.w, qb.w);
        const uint4 sn = make_uint4(sv.x ^ fx, sv.y ^ fy, sv.z ^ fz, sv.w ^ fw);
        own[r * n4 + g] = sn;
        if (fx | fy | fz | fw) {
            Q0[rd * n4 + g] = qa;
            Q1[rd * n4 + g] = qb;
        }
        if (MEASURE) {
            demon_packed_measure<DIMS>(sn.x, o.x, sh.x, oym.x, oyp.x, ozm.x, ozp.x, 0xFFFFFFFFu,
                                       32u, a.c, e_acc, m_acc);
            demon_packed_measure<DIMS>(sn.y, o.y, sh.y, oym.y, oyp.y, ozm.y, ozp.y, 0xFFFFFFFFu,
                                       32u, a.c, e_acc, m_acc);
            demon_packed_measure<DIMS>(sn.z, o.z, sh.z, oym.z, oyp.z, ozm.z, ozp.z, 0xFFFFFFFFu,
                                       32u, a.c, e_acc, m_acc);
            demon_packed_measure<DIMS>(sn.w, o.w, sh.w, oym.w, oyp.w, ozm.w, ozp.w, 0xFFFFFFFFu,
                                       32u, a.c, e_acc, m_acc);
        }
    }
    if (MEASURE) block_reduce_add(e_acc, m_acc, a.obs, a.c == 1);
}

// Bit-packed demon pass: one 32-site word per item (the neighbour words as in
// packed_word of pass_bodies.cuh).  a.dem is the own colour's two demon
// planes, plane 1 at a word offset of rows * nq.
template <int DIMS, bool MEASURE>
__global__ void __launch_bounds__(256) pass_demon_packed(PassArgs a) {
    const uint32_t W = (uint32_t)a.W, L = (uint32_t)a.L, rows = (uint32_t)a.rows;
    const uint32_t nq = (W + 31u) >> 5;
    const uint32_t items = rows * nq;
    uint32_t* own = static_cast<uint32_t*>(a.own);
    const uint32_t* other = static_cast<const uint32_t*>(a.other);
    uint32_t* Q0 = static_cast<uint32_t*>(a.dem);
    uint32_t* Q1 = Q0 + items;
    const uint32_t stride = gridDim.x * blockDim.x;
    int e_acc = 0, m_acc = 0;
    grid_dependency_wait();
    launch_dependents();
    for (uint32_t item = blockIdx.x * blockDim.x + threadIdx.x; item < items; item += stride) {
        const uint32_t r = item / nq, q = item - r * nq;
        uint32_t y = r, z = 0u;
        if (DIMS == 3) {
            z = r / L;
            y = r - z * L;
        }
        const uint32_t nb = W - 32u * q < 32u ? W - 32u * q : 32u;
        const uint32_t valid = nb == 32u ? 0xFFFFFFFFu : ((1u << nb) - 1u);
        const uint32_t plane = z * L, row = r * nq;
        const uint32_t o = __ldg(other + row + q);
        const uint32_t oym = __ldg(other + (plane + (y == 0u ? L - 1u : y - 1u)) * nq + q);
        const uint32_t oyp = __ldg(other + (plane + (y + 1u == L ? 0u : y + 1u)) * nq + q);
        uint32_t ozm = 0u, ozp = 0u;
        if (DIMS == 3) {
            ozm = __ldg(other + ((z == 0u ? L - 1u : z - 1u) * L + y) * nq + q);
            ozp = __ldg(other + ((z + 1u == L ? 0u : z + 1u) * L + y) * nq + q);
        }
        const uint32_t s = own[row + q];
        const int p = (a.c + (int)y + (int)z) & 1;
        uint32_t sh;
        if (p == 0) {  // bit b <- neighbour xh - 1
            const uint32_t prev = q == 0u ? __ldg(other + row + nq - 1u) << (31u - ((W - 1u) & 31u))
                                          : __ldg(other + row + q - 1u);
            sh = __funnelshift_l(prev, o, 1);
        } else {       // bit b <- neighbour xh + 1
            if (q + 1u == nq) {
                const uint32_t first = q == 0u ? o : __ldg(other + row);
                const uint32_t top = 1u << (nb - 1u);
                sh = ((o >> 1) & ~top) | ((first & 1u) ? top : 0u);
            } else {
                sh = __funnelshift_r(o, __ldg(other + row + q + 1u), 1);
            }
        }
        const Digits d = DIMS == 2 ? digits2(s ^ o, s ^ sh, s ^ oym, s ^ oyp)
                                   : digits3(s ^ o, s ^ sh, s ^ oym, s ^ oyp, s ^ ozm, s ^ ozp);
        const uint32_t rd = r >= a.rot ? r - a.rot : r + rows - a.rot;  // storage row
        const uint32_t qw = rd * nq + q;
        const uint32_t q0 = Q0[qw], q1 = Q1[qw];
        // v = q + d, bit-sliced
        const uint32_t v0 = q0 ^ d.d0, c0 = q0 & d.d0;
        const uint32_t v1 = q1 ^ d.d1 ^ c0, c1 = (q1 & d.d1) | (c0 & (q1 ^ d.d1));
        const uint32_t v2 = d.d2 ^ c1, v3 = d.d2 & c1;
        uint32_t flip, n0, n1;
        if (DIMS == 2) {  // 2 <= v <= 5 (v <= 7 here: v3 = 0); q' = v - 2
            flip = (v1 | v2) & ~(v1 & v2);
            n0 = v0;
            n1 = v2;
        } else {          // 3 <= v <= 6; q' = v - 3
            flip = (v3 | v2 | (v1 & v0)) & ~(v3 | (v2 & v1 & v0));
            n0 = ~v0;
            n1 = v2 & (v0 | v1);
        }
        flip &= valid;
        const uint32_t snew = s ^ flip;
        own[row + q] = snew;
        if (flip) {
            Q0[qw] = (q0 & ~flip) | (n0 & flip);
            Q1[qw] = (q1 & ~flip) | (n1 & flip);
        }
        if (MEASURE) {
            m_acc += 2 * __popc(snew & valid) - (int)nb;
            if (a.c == 1) {
                int dsum = __popc((snew ^ o) & valid) + __popc((snew ^ sh) & valid) +
                           __popc((snew ^ oym) & valid) + __popc((snew ^ oyp) & valid);
                if (DIMS == 3) dsum += __popc((snew ^ ozm) & valid) + __popc((snew ^ ozp) & valid);
                e_acc += 2 * dsum - (int)nb * 2 * DIMS;
            }
        }
    }
    if (MEASURE) block_reduce_add(e_acc, m_acc, a.obs, a.c == 1);
}

// Packed demons: canonical q (0..3) <-> two planes per colour, storage row
// of half row r = (r - rot) mod rows (rot = 0 when loading).
__global__ void import_demons_packed(uint32_t* d0, uint32_t* d1, const uint8_t* in, int L,
                                     int dims, int64_t rows) {
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
        uint32_t b0 = 0u, b1 = 0u;
        for (int b = 0; b < nb; ++b) {
            const uint8_t v = in[(int64_t)L * r + 2 * (32 * q + b) + p];
            b0 |= (uint32_t)(v & 1u) << b;
            b1 |= (uint32_t)((v >> 1) & 1u) << b;
        }
        uint32_t* dst = c == 0 ? d0 : d1;
        dst[w] = b0;
        dst[words + w] = b1;
    }
}

__global__ void export_demons_packed(const uint32_t* d0, const uint32_t* d1, uint8_t* out, int L,
                                     int dims, int64_t sites, int64_t rows, int64_t rot) {
    const int64_t nq = (L / 2 + 31) / 32, words = rows * nq;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < sites; i += stride) {
        const int64_t x = i % L, r = i / L;
        const int64_t y = r % L, z = dims == 3 ? r / L : 0;
        int64_t rd = r - rot;
        if (rd < 0) rd += rows;
        const int64_t xh = x >> 1, w = rd * nq + (xh >> 5);
        const uint32_t* src = ((x + y + z) & 1) == 0 ? d0 : d1;
        out[i] = (uint8_t)(((src[w] >> (xh & 31)) & 1u) | (((src[words + w] >> (xh & 31)) & 1u) << 1));
    }
}

unsigned grid_for(int64_t n, const DeviceProps& dp) {
    int64_t b = (n + 255) / 256;
    const int64_t cap = (int64_t)dp.sm_count * 16;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

template <int DIMS, bool MEASURE>
cudaError_t launch_demon_t(const PassArgs& a0, int64_t half_sites, const DeviceProps& dp,
                           cudaStream_t st) {
    const int threads = 256;
    if (a0.W % 16 == 0) {
        PassArgs a = a0;
        a.nv = a.W >> 4;
        const int64_t resident =
            (int64_t)dp.sm_count * dp.blocks_per_sm_demon[DIMS - 2][MEASURE] * threads;
        int64_t strips = resident / a.nv;
        if (strips > a.rows) strips = a.rows;
        if (strips < 1) strips = 1;
        a.strips = (int)strips;
        const int64_t blocks = (strips * a.nv + threads - 1) / threads;
        return launch_chained(pass_demon_strip<DIMS, MEASURE>, (unsigned)blocks,
                              (unsigned)threads, 0, st, a);
    }
    return launch_chained(pass_demon_sites<DIMS, MEASURE>, grid_for(half_sites, dp),
                          (unsigned)threads, 0, st, a0, (uint32_t)half_sites);
}

}  // namespace

cudaError_t demon_query_occupancy(DeviceProps& dp) {
    cudaError_t e;
#define ISING_OCC(D, M)                                                                      \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&dp.blocks_per_sm_demon[D - 2][M],      \
                                                      pass_demon_strip<D, M>, 256, 0);          \
    if (e != cudaSuccess) return e;
    ISING_OCC(2, false)
    ISING_OCC(2, true)
    ISING_OCC(3, false)
    ISING_OCC(3, true)
#undef ISING_OCC
    return cudaSuccess;
}

cudaError_t demon_pass(const PassArgs& a, int dims, int64_t half_sites, bool measure,
                       const DeviceProps& dp, cudaStream_t st) {
    if (dims == 2)
        return measure ? launch_demon_t<2, true>(a, half_sites, dp, st)
                       : launch_demon_t<2, false>(a, half_sites, dp, st);
    return measure ? launch_demon_t<3, true>(a, half_sites, dp, st)
                   : launch_demon_t<3, false>(a, half_sites, dp, st);
}

cudaError_t demon_packed_pass(const PassArgs& a, int dims, bool measure, const DeviceProps& dp,
                              cudaStream_t st) {
    const bool vec = a.W % 128 == 0;
    const int64_t items = a.rows * (int64_t)((a.W + 31) >> 5) / (vec ? 4 : 1);
    int64_t blocks = (items + 255) / 256;
    const int64_t cap = (int64_t)dp.sm_count * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    const unsigned g = (unsigned)blocks;
    if (vec) {
        if (dims == 2)
            return measure ? launch_chained(pass_demon_packed4<2, true>, g, 256u, 0, st, a)
                           : launch_chained(pass_demon_packed4<2, false>, g, 256u, 0, st, a);
        return measure ? launch_chained(pass_demon_packed4<3, true>, g, 256u, 0, st, a)
                       : launch_chained(pass_demon_packed4<3, false>, g, 256u, 0, st, a);
    }
    if (dims == 2)
        return measure ? launch_chained(pass_demon_packed<2, true>, g, 256u, 0, st, a)
                       : launch_chained(pass_demon_packed<2, false>, g, 256u, 0, st, a);
    return measure ? launch_chained(pass_demon_packed<3, true>, g, 256u, 0, st, a)
                   : launch_chained(pass_demon_packed<3, false>, g, 256u, 0, st, a);
}

cudaError_t demon_packed_import(uint32_t* d0, uint32_t* d1, const uint8_t* in, int L, int dims,
                                int64_t rows, const DeviceProps& dp, cudaStream_t st) {
    import_demons_packed<<<grid_for(2 * rows * ((L / 2 + 31) / 32), dp), 256, 0, st>>>(
        d0, d1, in, L, dims, rows);
    return cudaGetLastError();
}

cudaError_t demon_packed_export(const uint32_t* d0, const uint32_t* d1, uint8_t* out, int L,
                                int dims, int64_t sites, int64_t rows, int64_t rot,
                                const DeviceProps& dp, cudaStream_t st) {
    export_demons_packed<<<grid_for(sites, dp), 256, 0, st>>>(d0, d1, out, L, dims, sites, rows,
                                                              rot);
    return cudaGetLastError();
}

cudaError_t demon_export(const uint8_t* d0, const uint8_t* d1, uint8_t* out, int L, int dims,
                         int64_t sites, int64_t rows, int64_t rot, const DeviceProps& dp,
                         cudaStream_t st) {
    export_demons_kernel<<<grid_for(sites, dp), 256, 0, st>>>(d0, d1, out, L, dims, sites, rows,
                                                              rot);
    return cudaGetLastError();
}

cudaError_t demon_import(uint8_t* d0, uint8_t* d1, const uint8_t* in, int L, int dims,
                         int64_t sites, const DeviceProps& dp, cudaStream_t st) {
    import_demons_kernel<<<grid_for(sites, dp), 256, 0, st>>>(d0, d1, in, L, dims, sites);
    return cudaGetLastError();
}

}  // namespace ising
