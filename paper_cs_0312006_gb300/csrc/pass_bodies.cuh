// pass_bodies.cuh -- per-word bodies of a colour pass, shared by the
// per-lattice kernels (sweep_int8.cu, sweep_bitpack.cu) and the batched
// persistent kernel (batch.cu).
//
// The int8 body works for any even L: a word of the colour array holds the
// four half indices h = 4w..4w+3 (one Philox group), whatever rows they fall
// in.  A word that lies inside one half row, away from the x-wrap and from
// the first and last row (and plane) of the lattice, takes the byte-sliced
// path: its neighbour words are 4-byte windows of the other colour at byte
// offsets h - 1 / h + 1 (x), h -+ W (y) and h -+ L*W (z), read as two aligned
// words and a funnel shift.  Every other word (rows shorter than a word, row
// ends, wrap rows and planes, the ragged tail) takes the per-site path, which
// finds each neighbour from the site's coordinates.  Both paths apply the
// same rule and the same draw (word h & 3 of Philox(seed; h >> 2, t, c, 0)).
//
// NC selects how the other colour is read (see load_other): the per-lattice
// pass kernels use the read-only path; the batched kernel, which runs both
// colour passes of many sweeps in one launch, uses coherent loads.
#pragma once

#include <cstdint>

#include "ising_device.cuh"

namespace ising {

constexpr uint32_t kByteBit1 = 0x02020202u;
constexpr uint32_t kByteBit7 = 0x80808080u;
constexpr uint32_t kByteOnes = 0x01010101u;

// Load modes for the other colour: 1 = read-only path (ld.global.nc, only when
// nothing writes the array during the kernel), 2 = L2 only (ld.global.cg, for
// data written by other CTAs of a cluster earlier in the same kernel), 0 = a
// plain coherent load.
template <int NC, typename T>
__device__ __forceinline__ T load_other(const T* p) {
    if (NC == 1) return __ldg(p);
    if (NC == 2) return __ldcg(p);
    return *p;
}

// Byte mask 0xFE of each site whose flip is decided without a draw: byte j of
// D is 2*d_j, and bit 7 of D + bias is set iff d_j >= dims (dE <= 0).
template <int DIMS>
__device__ __forceinline__ uint32_t downhill_mask(uint32_t D) {
    constexpr uint32_t bias = (0x80u - 2u * DIMS) * kByteOnes;
    const uint32_t F = (D + bias) & kByteBit7;
    return F | (F - (F >> 6));  // 0x80 -> 0xFE per byte, borrow-free
}

// Metropolis test of site j (d_j < dims): u_j < thr[k], k = 2(dims - d_j).
template <int DIMS>
__device__ __forceinline__ uint32_t uphill_accept(uint32_t D, uint32_t u, int j,
                                                  const PassArgs& a) {
    const uint32_t dj = D & (0x0Eu << (8 * j));  // 2*d_j in place
    uint32_t t;
    if (DIMS == 2) {
        t = dj == 0u ? a.thr[1] : a.thr[0];
    } else {
        t = dj == 0u ? a.thr[2] : (dj == (0x02u << (8 * j)) ? a.thr[1] : a.thr[0]);
    }
    return u < t ? (0xFEu << (8 * j)) : 0u;
}

// The same test for four sites by counting: byte j gains 2 for every threshold
// u_j lies below; since the thresholds fall with k, site j (d_j < dims) flips
// iff 2*(count_j + d_j) >= 2*dims, read off bit 7 after the bias.  A site with
// d_j >= dims has bit 7 set by D + bias alone, and no byte carries (at most
// 0x80 + 4 dims < 0x100), so the mask already holds every downhill
// flip: where all four draws are made it is the whole flip mask.
template <int DIMS>
__device__ __forceinline__ uint32_t uphill_count(uint32_t D, const Philox4& u, const PassArgs& a) {
    constexpr uint32_t bias = (0x80u - 2u * DIMS) * kByteOnes;
    uint32_t acc = D + bias;
    acc += (u.w0 < a.thr[0] ? 0x00000002u : 0u) + (u.w0 < a.thr[1] ? 0x00000002u : 0u);
    acc += (u.w1 < a.thr[0] ? 0x00000200u : 0u) + (u.w1 < a.thr[1] ? 0x00000200u : 0u);
    acc += (u.w2 < a.thr[0] ? 0x00020000u : 0u) + (u.w2 < a.thr[1] ? 0x00020000u : 0u);
    acc += (u.w3 < a.thr[0] ? 0x02000000u : 0u) + (u.w3 < a.thr[1] ? 0x02000000u : 0u);
    if (DIMS == 3) {
        acc += (u.w0 < a.thr[2] ? 0x00000002u : 0u) + (u.w1 < a.thr[2] ? 0x00000200u : 0u);
        acc += (u.w2 < a.thr[2] ? 0x00020000u : 0u) + (u.w3 < a.thr[2] ? 0x02000000u : 0u);
    }
    const uint32_t F = acc & kByteBit7;
    return F | (F - (F >> 6));
}

// Heat-bath rule (every site draws; it flips iff u < thr[d], the thresholds
// rising with d): with cnt = #{m = 0..2 dims : u < thr[m]}, u < thr[d] iff
// cnt + d >= 2 dims + 1.  Byte j of D is 2 d_j, so byte j of D + bias + 2 cnt_j
// reaches bit 7 exactly then (at most 4*(2 dims) + 2 + bias < 256: no carry).
template <int DIMS>
__device__ __forceinline__ uint32_t heatbath_count(uint32_t D, const Philox4& u,
                                                   const PassArgs& a) {
    constexpr uint32_t bias = (0x80u - 2u * (2u * DIMS + 1u)) * kByteOnes;
    const uint32_t w[4] = {u.w0, u.w1, u.w2, u.w3};
    uint32_t acc = D + bias;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t cnt = 0u;
#pragma unroll
        for (int m = 0; m <= 2 * DIMS; ++m) cnt += w[j] < a.thr[m] ? 2u : 0u;
        acc += cnt << (8 * j);
    }
    const uint32_t F = acc & kByteBit7;
    return F | (F - (F >> 6));
}

// thr[d] by selects (d = 0..2*dims), for code that holds PassArgs in registers.
template <int DIMS>
__device__ __forceinline__ uint32_t heatbath_threshold(int d, const PassArgs& a) {
    uint32_t t = a.thr[0];
#pragma unroll
    for (int m = 1; m <= 2 * DIMS; ++m) t = d == m ? a.thr[m] : t;
    return t;
}

// Multi-hit Metropolis on one 4-site word: a.hits successive trials, the
// neighbours fixed; after a trial the flipped sites' D becomes 2(2 dims - d).
// Trial m draws Philox(seed; group, t, c + 2m, 0).  Returns the net flip mask.
template <int DIMS>
__device__ __forceinline__ uint32_t multihit_word(uint32_t D, uint32_t group, const PassArgs& a) {
    constexpr uint32_t q2 = 4u * DIMS * kByteOnes;
    uint32_t net = 0u;
#pragma unroll 1
    for (int m = 0; m < a.hits; ++m) {
        uint32_t X = downhill_mask<DIMS>(D);
        if (X != 0xFEFEFEFEu) {
            const Philox4 u = philox4x32_10(group, a.t, (uint32_t)a.c + 2u * (uint32_t)m,
                                            kTagSweep, a.key0, a.key1);
            X |= uphill_count<DIMS>(D, u, a);
        }
        D = (D & ~X) | ((q2 - D) & X);
        net ^= X;
    }
    return net;
}

template <int DIMS>
__device__ __forceinline__ uint32_t disagreements(uint32_t s, uint32_t n0, uint32_t n1,
                                                  uint32_t n2, uint32_t n3, uint32_t n4,
                                                  uint32_t n5) {
    uint32_t D = ((s ^ n0) & kByteBit1) + ((s ^ n1) & kByteBit1) + ((s ^ n2) & kByteBit1) +
                 ((s ^ n3) & kByteBit1);
    if (DIMS == 3) D += ((s ^ n4) & kByteBit1) + ((s ^ n5) & kByteBit1);
    return D;
}

// Four bytes of the other colour starting at byte offset o (o >= 0; the array
// is padded so that the word after the last one may be read).
template <int NC>
__device__ __forceinline__ uint32_t window4(const uint32_t* other, uint32_t o) {
    const uint32_t lo = load_other<NC>(other + (o >> 2));
    if ((o & 3u) == 0u) return lo;
    const uint32_t hi = load_other<NC>(other + (o >> 2) + 1);
    return __funnelshift_r(lo, hi, 8u * (o & 3u));
}

struct WordGeom {
    uint32_t W;       // sites per half row
    uint32_t L;
    uint32_t rows;    // L^(dims-1)
    uint32_t half;    // sites per colour
};

// Update word w of the int8 colour array `own` (colour a.c).  Accumulates the
// number of -1 spins written (m_neg), the number of sites written (n_sites)
// and, in the white pass, sum (2 d_new - 2 dims) over them (e_acc).
template <int DIMS, bool MEASURE, int NC, int RULE = kRuleMetropolis>
__device__ __forceinline__ void int8_word(const PassArgs& a, const WordGeom& g, uint32_t w,
                                          int& e_acc, int& m_neg, int& n_sites) {
    uint32_t* own = static_cast<uint32_t*>(a.own);
    const uint32_t* other = static_cast<const uint32_t*>(a.other);
    const int8_t* other_b = static_cast<const int8_t*>(a.other);
    const uint32_t h0 = 4u * w;
    const uint32_t r0 = h0 / g.W;
    const uint32_t xh0 = h0 - r0 * g.W;
    uint32_t y0 = r0, z0 = 0;
    if (DIMS == 3) {
        z0 = r0 / g.L;
        y0 = r0 - z0 * g.L;
    }
    const int p = (a.c + (int)y0 + (int)z0) & 1;
    bool fast = (xh0 + 3u < g.W) && (h0 + 3u < g.half) && y0 != 0u && y0 + 1u != g.L;
    if (DIMS == 3) fast = fast && z0 != 0u && z0 + 1u != g.L;
    fast = fast && (p == 0 ? xh0 != 0u : xh0 + 4u != g.W);
    if (fast) {
        const uint32_t s = own[w];
        const uint32_t nx = load_other<NC>(other + w);
        const uint32_t nxs = p == 0 ? window4<NC>(other, h0 - 1u) : window4<NC>(other, h0 + 1u);
        const uint32_t nym = window4<NC>(other, h0 - g.W);
        const uint32_t nyp = window4<NC>(other, h0 + g.W);
        uint32_t nzm = 0u, nzp = 0u;
        if (DIMS == 3) {
            nzm = window4<NC>(other, h0 - g.L * g.W);
            nzp = window4<NC>(other, h0 + g.L * g.W);
        }
        const uint32_t D = disagreements<DIMS>(s, nx, nxs, nym, nyp, nzm, nzp);
        uint32_t X;
        if (RULE == kRuleHeatBath) {
            const Philox4 u = philox4x32_10(w, a.t, (uint32_t)a.c, kTagSweep, a.key0, a.key1);
            X = heatbath_count<DIMS>(D, u, a);
        } else if (RULE == kRuleMultiHit) {
            X = multihit_word<DIMS>(D, w, a);
        } else {
            X = downhill_mask<DIMS>(D);
            if (X != 0xFEFEFEFEu) {
                const Philox4 u = philox4x32_10(w, a.t, (uint32_t)a.c, kTagSweep, a.key0, a.key1);
                X |= uphill_accept<DIMS>(D, u.w0, 0, a) | uphill_accept<DIMS>(D, u.w1, 1, a) |
                     uphill_accept<DIMS>(D, u.w2, 2, a) | uphill_accept<DIMS>(D, u.w3, 3, a);
            }
        }
        const uint32_t snew = s ^ X;
        own[w] = snew;
        if (MEASURE) {
            m_neg += __popc(snew & kByteBit7);
            n_sites += 4;
            if (a.c == 1) {
                constexpr uint32_t q2 = 4u * DIMS * kByteOnes;
                const uint32_t Dn = (D & ~X) | ((q2 - D) & X);
                e_acc += __dp4a((int)Dn, (int)kByteOnes, 0) - 4 * 2 * DIMS;
            }
        }
        return;
    }
    // per-site path
    int8_t* own_b = static_cast<int8_t*>(a.own);
    int s_val[4], d_val[4];
    bool valid[4], need = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t h = h0 + (uint32_t)j;
        valid[j] = h < g.half;
        s_val[j] = 1;
        d_val[j] = DIMS;
        if (!valid[j]) continue;
        const uint32_t r = h / g.W;
        const uint32_t xh = h - r * g.W;
        uint32_t y = r, z = 0;
        if (DIMS == 3) {
            z = r / g.L;
            y = r - z * g.L;
        }
        const int pp = (a.c + (int)y + (int)z) & 1;
        const uint32_t x = 2u * xh + (uint32_t)pp;
        const uint32_t xm = (x == 0u ? g.L - 1u : x - 1u) >> 1;
        const uint32_t xp = (x + 1u == g.L ? 0u : x + 1u) >> 1;
        const uint32_t plane = z * g.L;
        const uint32_t rym = plane + (y == 0u ? g.L - 1u : y - 1u);
        const uint32_t ryp = plane + (y + 1u == g.L ? 0u : y + 1u);
        const int s = own_b[h];
        int hsum = load_other<NC>(other_b + r * g.W + xm) + load_other<NC>(other_b + r * g.W + xp) +
                   load_other<NC>(other_b + rym * g.W + xh) +
                   load_other<NC>(other_b + ryp * g.W + xh);
        if (DIMS == 3) {
            const uint32_t rzm = (z == 0u ? g.L - 1u : z - 1u) * g.L + y;
            const uint32_t rzp = (z + 1u == g.L ? 0u : z + 1u) * g.L + y;
            hsum += load_other<NC>(other_b + rzm * g.W + xh) +
                    load_other<NC>(other_b + rzp * g.W + xh);
        }
        s_val[j] = s;
        d_val[j] = (2 * DIMS - s * hsum) >> 1;  // k = s*h = 2*(dims - d)
        if (d_val[j] < DIMS || RULE == kRuleHeatBath) need = true;
    }
    if (RULE == kRuleMultiHit) {
        int d_cur[4], flips[4] = {0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < 4; ++j) d_cur[j] = d_val[j];
#pragma unroll 1
        for (int m = 0; m < a.hits; ++m) {
            bool any = false;
#pragma unroll
            for (int j = 0; j < 4; ++j) any |= valid[j] && d_cur[j] < DIMS;
            uint32_t uu[4] = {0u, 0u, 0u, 0u};
            if (any) {
                const Philox4 q = philox4x32_10(w, a.t, (uint32_t)a.c + 2u * (uint32_t)m,
                                                kTagSweep, a.key0, a.key1);
                uu[0] = q.w0;
                uu[1] = q.w1;
                uu[2] = q.w2;
                uu[3] = q.w3;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                bool f = d_cur[j] >= DIMS;
                if (!f) {
                    const int dj = d_cur[j];
                    const uint32_t t = DIMS == 2 ? (dj == 0 ? a.thr[1] : a.thr[0])
                                                 : (dj == 0 ? a.thr[2] : (dj == 1 ? a.thr[1] : a.thr[0]));
                    f = uu[j] < t;
                }
                if (f) {
                    d_cur[j] = 2 * DIMS - d_cur[j];
                    flips[j] ^= 1;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!valid[j]) continue;
            const int sn = flips[j] ? -s_val[j] : s_val[j];
            if (flips[j]) own_b[h0 + j] = (int8_t)sn;
            if (MEASURE) {
                m_neg += sn < 0;
                n_sites += 1;
                if (a.c == 1) e_acc += 2 * d_cur[j] - 2 * DIMS;
            }
        }
        return;
    }
    uint32_t u[4] = {0u, 0u, 0u, 0u};
    if (need) {
        const Philox4 q = philox4x32_10(w, a.t, (uint32_t)a.c, kTagSweep, a.key0, a.key1);
        u[0] = q.w0;
        u[1] = q.w1;
        u[2] = q.w2;
        u[3] = q.w3;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (!valid[j]) continue;
        bool flip;
        if (RULE == kRuleHeatBath) {
            flip = u[j] < heatbath_threshold<DIMS>(d_val[j], a);
        } else {
            flip = d_val[j] >= DIMS;
            if (!flip) {
                const uint32_t t = DIMS == 2 ? (d_val[j] == 0 ? a.thr[1] : a.thr[0])
                                             : (d_val[j] == 0 ? a.thr[2] : (d_val[j] == 1 ? a.thr[1] : a.thr[0]));
                flip = u[j] < t;
            }
        }
        const int sn = flip ? -s_val[j] : s_val[j];
        if (flip) own_b[h0 + j] = (int8_t)sn;
        if (MEASURE) {
            m_neg += sn < 0;
            n_sites += 1;
            if (a.c == 1) {
                const int dn = flip ? 2 * DIMS - d_val[j] : d_val[j];
                e_acc += 2 * dn - 2 * DIMS;
            }
        }
    }
}

// Update the 16 sites of one 16-byte vector (four Philox groups g0..g0+3).
// The four Philox calls are independent and computed together when any of
// the 16 sites needs its draw (always, under the heat-bath rule).  Accumulates the number of -1 spins (m_neg)
// and, in the white pass, sum_j 2*d_new_j (e_acc).
template <int DIMS, bool MEASURE, int RULE = kRuleMetropolis>
__device__ __forceinline__ uint4 update_vec(const uint4& s, const uint4& x, const uint4& xs,
                                            const uint4& ym, const uint4& yp, const uint4& zm,
                                            const uint4& zp, uint32_t g0, const PassArgs& a,
                                            int& e_acc, int& m_neg) {
    const uint32_t sv[4] = {s.x, s.y, s.z, s.w};
    uint32_t D[4], X[4];
    D[0] = disagreements<DIMS>(s.x, x.x, xs.x, ym.x, yp.x, zm.x, zp.x);
    D[1] = disagreements<DIMS>(s.y, x.y, xs.y, ym.y, yp.y, zm.y, zp.y);
    D[2] = disagreements<DIMS>(s.z, x.z, xs.z, ym.z, yp.z, zm.z, zp.z);
    D[3] = disagreements<DIMS>(s.w, x.w, xs.w, ym.w, yp.w, zm.w, zp.w);
    if (RULE == kRuleMultiHit) {
        constexpr uint32_t q2 = 4u * DIMS * kByteOnes;
        uint32_t Dc[4] = {D[0], D[1], D[2], D[3]};
#pragma unroll
        for (int w = 0; w < 4; ++w) X[w] = 0u;
#pragma unroll 1
        for (int m = 0; m < a.hits; ++m) {
            uint32_t Y[4];
            bool need = false;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                Y[w] = downhill_mask<DIMS>(Dc[w]);
                need |= Y[w] != 0xFEFEFEFEu;
            }
            if (need) {
                Philox4 u[4];
#pragma unroll
                for (int w = 0; w < 4; ++w)
                    u[w] = philox4x32_10(g0 + (uint32_t)w, a.t, (uint32_t)a.c + 2u * (uint32_t)m,
                                         kTagSweep, a.key0, a.key1);
#pragma unroll
                for (int w = 0; w < 4; ++w) Y[w] |= uphill_count<DIMS>(Dc[w], u[w], a);
            }
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                Dc[w] = (Dc[w] & ~Y[w]) | ((q2 - Dc[w]) & Y[w]);
                X[w] ^= Y[w];
            }
        }
    } else if (RULE == kRuleHeatBath) {  // every site draws
        Philox4 u[4];
#pragma unroll
        for (int w = 0; w < 4; ++w)
            u[w] = philox4x32_10(g0 + (uint32_t)w, a.t, (uint32_t)a.c, kTagSweep, a.key0, a.key1);
#pragma unroll
        for (int w = 0; w < 4; ++w) X[w] = heatbath_count<DIMS>(D[w], u[w], a);
    } else {
        bool need = false;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            X[w] = downhill_mask<DIMS>(D[w]);
            need |= X[w] != 0xFEFEFEFEu;
        }
        if (need) {
            Philox4 u[4];
#pragma unroll
            for (int w = 0; w < 4; ++w)
                u[w] = philox4x32_10(g0 + (uint32_t)w, a.t, (uint32_t)a.c, kTagSweep, a.key0,
                                     a.key1);
            // counting thresholds below each draw measured a little faster here
            // than selecting one threshold per site (uphill_accept): it spreads
            // the work over the integer ALU and the multiply-add pipe
#pragma unroll
            for (int w = 0; w < 4; ++w) X[w] |= uphill_count<DIMS>(D[w], u[w], a);
        }
    }
    uint32_t out[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        out[w] = sv[w] ^ X[w];  // 0x01 <-> 0xFF where flipped
        if (MEASURE) {
            m_neg += __popc(out[w] & kByteBit7);
            if (a.c == 1) {
                // 2*d_new = 2*(2 dims) - 2*d where flipped; X covers bits 1..7 there
                constexpr uint32_t q2 = 4u * DIMS * kByteOnes;
                const uint32_t Dn = (D[w] & ~X[w]) | ((q2 - D[w]) & X[w]);
                e_acc = __dp4a((int)Dn, (int)kByteOnes, e_acc);
            }
        }
    }
    return make_uint4(out[0], out[1], out[2], out[3]);
}


// 16 bytes of the other colour at byte offset o (any alignment): two aligned
// 16-byte loads and a byte shift.  The shift r = o mod 16 is the same for a
// whole lattice and direction (it depends only on W, L and the direction), so
// the switch does not diverge.
template <int NC>
__device__ __forceinline__ uint4 window16(const uint4* other16, uint32_t o) {
    const uint32_t r = o & 15u;
    const uint4 lo = load_other<NC>(other16 + (o >> 4));
    if (r == 0u) return lo;
    const uint4 hi = load_other<NC>(other16 + (o >> 4) + 1);
    const uint32_t b = 8u * (r & 3u);
    uint32_t w0, w1, w2, w3, w4;
    switch (r >> 2) {
        case 0: w0 = lo.x; w1 = lo.y; w2 = lo.z; w3 = lo.w; w4 = hi.x; break;
        case 1: w0 = lo.y; w1 = lo.z; w2 = lo.w; w3 = hi.x; w4 = hi.y; break;
        case 2: w0 = lo.z; w1 = lo.w; w2 = hi.x; w3 = hi.y; w4 = hi.z; break;
        default: w0 = lo.w; w1 = hi.x; w2 = hi.y; w3 = hi.z; w4 = hi.w; break;
    }
    return make_uint4(__funnelshift_r(w0, w1, b), __funnelshift_r(w1, w2, b),
                      __funnelshift_r(w2, w3, b), __funnelshift_r(w3, w4, b));
}

// Update the 16 sites of vector v (half indices 16v..16v+15, Philox groups
// 4v..4v+3) of the int8 colour array.  A vector inside one half row, away from
// the x-wrap and the first/last row and plane, is updated as a whole from
// 16-byte neighbour windows; any other vector word by word (int8_word).
// Accumulates m_neg, n_sites and, in the white pass, e_acc as int8_word does.
template <int DIMS, bool MEASURE, int NC, int RULE = kRuleMetropolis>
__device__ __forceinline__ void int8_vec(const PassArgs& a, const WordGeom& g, uint32_t v,
                                         int& e_acc, int& m_neg, int& n_sites) {
    const uint32_t h0 = 16u * v;
    const uint32_t r0 = h0 / g.W;
    const uint32_t xh0 = h0 - r0 * g.W;
    uint32_t y0 = r0, z0 = 0;
    if (DIMS == 3) {
        z0 = r0 / g.L;
        y0 = r0 - z0 * g.L;
    }
    const int p = (a.c + (int)y0 + (int)z0) & 1;
    bool fast = (xh0 + 15u < g.W) && (h0 + 15u < g.half) && y0 != 0u && y0 + 1u != g.L;
    if (DIMS == 3) fast = fast && z0 != 0u && z0 + 1u != g.L;
    fast = fast && (p == 0 ? xh0 != 0u : xh0 + 16u != g.W);
    if (!fast) {
#pragma unroll 1
        for (uint32_t w = 4u * v; w < 4u * v + 4u; ++w)
            if (4u * w < g.half) int8_word<DIMS, MEASURE, NC, RULE>(a, g, w, e_acc, m_neg, n_sites);
        return;
    }
    const uint4* other16 = static_cast<const uint4*>(a.other);
    uint4* own16 = static_cast<uint4*>(a.own);
    const uint4 s = own16[v];
    const uint4 nx = load_other<NC>(other16 + v);
    uint4 nxs;
    if (p == 0) {  // neighbour h' - 1: byte j <- byte j - 1
        const uint32_t prev = load_other<NC>(static_cast<const uint32_t*>(a.other) + 4u * v - 1u);
        nxs = make_uint4(__funnelshift_l(prev, nx.x, 8), __funnelshift_l(nx.x, nx.y, 8),
                         __funnelshift_l(nx.y, nx.z, 8), __funnelshift_l(nx.z, nx.w, 8));
    } else {       // neighbour h' + 1: byte j <- byte j + 1
        const uint32_t next = load_other<NC>(static_cast<const uint32_t*>(a.other) + 4u * v + 4u);
        nxs = make_uint4(__funnelshift_r(nx.x, nx.y, 8), __funnelshift_r(nx.y, nx.z, 8),
                         __funnelshift_r(nx.z, nx.w, 8), __funnelshift_r(nx.w, next, 8));
    }
    const uint4 nym = window16<NC>(other16, h0 - g.W);
    const uint4 nyp = window16<NC>(other16, h0 + g.W);
    uint4 nzm = make_uint4(0u, 0u, 0u, 0u), nzp = nzm;
    if (DIMS == 3) {
        nzm = window16<NC>(other16, h0 - g.L * g.W);
        nzp = window16<NC>(other16, h0 + g.L * g.W);
    }
    int e_vec = 0;
    own16[v] = update_vec<DIMS, MEASURE, RULE>(s, nx, nxs, nym, nyp, nzm, nzp, 4u * v, a, e_vec,
                                               m_neg);
    if (MEASURE) {
        n_sites += 16;
        if (a.c == 1) e_acc += e_vec - 16 * 2 * DIMS;
    }
}

// ----------------------------------------------------------------------------
// Bit-packed body: one 32-site word per call; see sweep_bitpack.cu for the
// layout.
// ----------------------------------------------------------------------------
struct Counts {
    uint32_t always, eq0, eq1, eq2;
};

__device__ __forceinline__ Counts count2(uint32_t a, uint32_t b, uint32_t c, uint32_t e) {
    const uint32_t s1 = a ^ b, c1 = a & b;
    const uint32_t s2 = c ^ e, c2 = c & e;
    const uint32_t b0 = s1 ^ s2, c3 = s1 & s2;
    const uint32_t always = c1 | c2 | c3;  // d = b0 + 2 (c1 + c2 + c3) >= 2
    return Counts{always, ~(b0 | always), b0 & ~always, 0u};
}

__device__ __forceinline__ Counts count3(uint32_t a, uint32_t b, uint32_t c, uint32_t d,
                                         uint32_t e, uint32_t f) {
    const uint32_t s1 = a ^ b ^ c, k1 = (a & b) | (c & (a ^ b));
    const uint32_t s2 = d ^ e ^ f, k2 = (d & e) | (f & (d ^ e));
    const uint32_t bit0 = s1 ^ s2, k0 = s1 & s2;
    const uint32_t bit1 = k1 ^ k2 ^ k0, bit2 = (k1 & k2) | (k0 & (k1 ^ k2));
    const uint32_t always = bit2 | (bit1 & bit0);  // d = bit0 + 2 bit1 + 4 bit2 >= 3
    const uint32_t low = ~(bit2 | bit1);
    return Counts{always, low & ~bit0, low & bit0, bit1 & ~bit0 & ~bit2};
}

// Bit-sliced number of disagreeing neighbours d = d0 + 2 d1 + 4 d2 of each
// of the 32 sites (the heat-bath rule needs every value of d).
struct Digits {
    uint32_t d0, d1, d2;
};

__device__ __forceinline__ Digits digits2(uint32_t a, uint32_t b, uint32_t c, uint32_t e) {
    const uint32_t s1 = a ^ b, c1 = a & b;
    const uint32_t s2 = c ^ e, c2 = c & e;
    const uint32_t c3 = s1 & s2;  // d = (s1 ^ s2) + 2 (c1 + c2 + c3)
    return Digits{s1 ^ s2, c1 ^ c2 ^ c3, (c1 & c2) | (c3 & (c1 ^ c2))};
}

__device__ __forceinline__ Digits digits3(uint32_t a, uint32_t b, uint32_t c, uint32_t d,
                                          uint32_t e, uint32_t f) {
    const uint32_t s1 = a ^ b ^ c, k1 = (a & b) | (c & (a ^ b));
    const uint32_t s2 = d ^ e ^ f, k2 = (d & e) | (f & (d ^ e));
    const uint32_t k0 = s1 & s2;  // d = (s1 ^ s2) + 2 (k1 + k2 + k0)
    return Digits{s1 ^ s2, k1 ^ k2 ^ k0, (k1 & k2) | (k0 & (k1 ^ k2))};
}

// Threshold of bit b: Metropolis, for a site with dE > 0 (d < dims) ...
template <int DIMS>
__device__ __forceinline__ uint32_t site_threshold(const Counts& k, int b, const PassArgs& a) {
    if (DIMS == 2) return (k.eq0 >> b) & 1u ? a.thr[1] : a.thr[0];
    return (k.eq0 >> b) & 1u ? a.thr[2] : ((k.eq1 >> b) & 1u ? a.thr[1] : a.thr[0]);
}

// ... and heat bath, thr[d] for any d.
template <int DIMS>
__device__ __forceinline__ uint32_t site_threshold(const Digits& k, int b, const PassArgs& a) {
    const bool d0 = (k.d0 >> b) & 1u, d1 = (k.d1 >> b) & 1u, d2 = (k.d2 >> b) & 1u;
    const uint32_t lo = d1 ? (d0 ? a.thr[3] : a.thr[2]) : (d0 ? a.thr[1] : a.thr[0]);
    const uint32_t hi = DIMS == 2 ? a.thr[4] : (d1 ? a.thr[6] : (d0 ? a.thr[5] : a.thr[4]));
    return d2 ? hi : lo;
}

template <int DIMS, typename K>
__device__ __forceinline__ uint32_t group_accept(const K& k, const Philox4& u, int i,
                                                 const PassArgs& a) {
    const uint32_t w[4] = {u.w0, u.w1, u.w2, u.w3};
    uint32_t acc = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int b = 4 * i + j;
        acc |= (w[j] < site_threshold<DIMS>(k, b, a) ? 1u : 0u) << b;
    }
    return acc;
}

// Accept mask of a 16-site half of a packed word whose first bit is half
// index g0 * 4 + M + 16 * HALF (M = 1..3: the row starts inside a Philox
// group).  Its sites draw from the five groups g0 + 4 HALF .. g0 + 4 HALF + 4
// (bit b takes word (M + b) & 3 of group g0 + ((M + b) >> 2)); the five calls
// are made together, and every index is a compile-time constant.
template <int DIMS, int M, int HALF, typename K>
__device__ __forceinline__ uint32_t packed_accept_half_shifted(const K& k, uint32_t g0,
                                                               const PassArgs& a, uint32_t c2) {
    Philox4 u[5];
#pragma unroll
    for (int i = 0; i < 5; ++i)
        u[i] = philox4x32_10(g0 + (uint32_t)(4 * HALF + i), a.t, c2, kTagSweep, a.key0, a.key1);
    uint32_t acc = 0u;
#pragma unroll
    for (int b = 16 * HALF; b < 16 * HALF + 16; ++b) {
        const int q = M + b - 16 * HALF;  // draw index within the five calls
        const Philox4& g = u[q >> 2];
        const uint32_t w = (q & 3) == 0 ? g.w0 : (q & 3) == 1 ? g.w1 : (q & 3) == 2 ? g.w2 : g.w3;
        acc |= (w < site_threshold<DIMS>(k, b, a) ? 1u : 0u) << b;
    }
    return acc;
}

template <int DIMS, int M, typename K>
__device__ __forceinline__ uint32_t packed_accept_shifted(const K& k, uint32_t need, uint32_t g0,
                                                          const PassArgs& a, uint32_t c2) {
    uint32_t acc = 0u;
    if (need & 0xFFFFu) acc |= packed_accept_half_shifted<DIMS, M, 0>(k, g0, a, c2);
    if (need >> 16) acc |= packed_accept_half_shifted<DIMS, M, 1>(k, g0, a, c2);
    return acc;
}

// Accept mask of the `need` bits of a packed word (Metropolis: the sites with
// dE > 0; heat bath: every valid site) whose 32 bits are the half indices
// hb = hbase + b (b = 0..31).  Bit b's draw
// is word (hb & 3) of Philox group hb >> 2.  When hbase is a multiple of 4 the
// eight groups are the word's nibbles and are computed four at a time; when a
// row starts inside a group (W not a multiple of 4) the word spans nine
// groups.  With ILP9 (the per-lattice pass), when the lanes of the warp share
// the row offset, each half takes its five groups together
// (packed_accept_shifted); otherwise, and in the batched kernel (which runs at
// a fixed register budget), the nine are taken one at a time.
// ALIGNED: the caller knows hbase % 4 == 0 (rows of a multiple of 32 sites),
// so only the eight-group path is compiled.
template <int DIMS, typename K, bool ILP9 = false, bool ALIGNED = false>
__device__ __forceinline__ uint32_t packed_accept(const K& k, uint32_t need, uint32_t hbase,
                                                  const PassArgs& a, uint32_t c2) {
    uint32_t acc = 0u;
    const uint32_t m = ALIGNED ? 0u : hbase & 3u, g0 = hbase >> 2;
    if (!ALIGNED && ILP9 && m != 0u) {
        // the compile-time offset paths only when the warp agrees on it
        const uint32_t lanes = __activemask();
        const uint32_t m0 = __shfl_sync(lanes, m, __ffs(lanes) - 1);
        if (__all_sync(lanes, m == m0)) {
            if (m == 1u) return packed_accept_shifted<DIMS, 1>(k, need, g0, a, c2);
            if (m == 2u) return packed_accept_shifted<DIMS, 2>(k, need, g0, a, c2);
            return packed_accept_shifted<DIMS, 3>(k, need, g0, a, c2);
        }
    }
    if (m == 0u) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            if (!((need >> (16 * half)) & 0xFFFFu)) continue;
            // four consecutive groups: one first-round product for the four
            PhiloxRuns<1> ps;
            const uint32_t base[1] = {g0 + (uint32_t)(4 * half)};
            ps.first_round(base, a.t, c2, kTagSweep, a.key0, a.key1);
#pragma unroll
            for (int r = 1; r < 10; ++r) ps.next_round();
#pragma unroll
            for (int i = 0; i < 4; ++i) acc |= group_accept<DIMS>(k, ps.result(i), 4 * half + i, a);
        }
        return acc;
    }
    if constexpr (!ALIGNED) {
#pragma unroll 1
        for (int g = 0; g < 9; ++g) {
            const int lo = 4 * g - (int)m;  // bit of the group's word 0 (may be < 0)
            const uint32_t gmask = lo >= 0 ? (0xFu << lo) : (0xFu >> (-lo));
            if (!(need & gmask)) continue;
            const Philox4 u = philox4x32_10(g0 + (uint32_t)g, a.t, c2, kTagSweep, a.key0,
                                            a.key1);
            const uint32_t w[4] = {u.w0, u.w1, u.w2, u.w3};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int b = lo + j;
                if (b < 0 || b > 31) continue;
                acc |= (w[j] < site_threshold<DIMS>(k, b, a) ? 1u : 0u) << b;
            }
        }
    }
    return acc;
}

// Update word (r, q) of the packed colour array.  A half row of W sites takes
// nq = ceil(W / 32) words; bit b of word q is half column xh = 32q + b (valid
// when xh < W; the other bits of a row's last word stay 0 and never flip).
// The x-neighbour wrap at the row ends comes from the row's last valid bit
// (p = 0, first word) or first bit (p = 1, last word).
//
// With rgroups > 1 the items visit the rows grouped by r mod rgroups: every
// row of a group starts at the same offset inside a Philox group (r W mod 4
// depends only on r mod 4 for odd W, on r mod 2 for W = 2 mod 4), so the lanes
// of a warp share it and take the five-call path together instead of
// diverging over all four offsets.  Group c holds rows c, c + rgroups, ...
// (the first rows mod rgroups groups one row more).
__host__ __device__ __forceinline__ uint32_t packed_row_groups(uint32_t W) {
    return (W & 1u) ? 4u : ((W & 3u) == 2u ? 2u : 1u);
}

__device__ __forceinline__ uint32_t grouped_row(uint32_t j, uint32_t rows, uint32_t rgroups) {
    const uint32_t G = rows / rgroups, rem = rows - G * rgroups;
    const uint32_t head = rem * (G + 1u);  // rows in the longer groups
    uint32_t c, k;
    if (j < head) {
        c = j / (G + 1u);
        k = j - c * (G + 1u);
    } else {
        const uint32_t jj = j - head;
        c = G ? jj / G : 0u;
        k = jj - c * G;
        c += rem;
    }
    return k * rgroups + c;
}

// The rule applied to one packed word, given the word s and its neighbour
// words (sh: the x-neighbour across the colour, shifted into place), then the
// store and the word's share of E and M.  valid: the word's sites (nb bits);
// hbase: the half index of bit 0 (its Philox draw is word hbase & 3 of group
// hbase >> 2).  ALIGNED: hbase % 4 == 0 is known (packed_accept).
template <int DIMS, bool MEASURE, int RULE, bool ILP9, bool ALIGNED>
__device__ __forceinline__ void packed_update(const PassArgs& a, uint32_t* own_word, uint32_t s,
                                              uint32_t o, uint32_t sh, uint32_t oym,
                                              uint32_t oyp, uint32_t ozm, uint32_t ozp,
                                              uint32_t valid, uint32_t nb, uint32_t hbase,
                                              int& e_acc, int& m_acc) {
    uint32_t flip;
    if constexpr (RULE == kRuleHeatBath) {  // every valid site draws
        const Digits k = DIMS == 2 ? digits2(s ^ o, s ^ sh, s ^ oym, s ^ oyp)
                                   : digits3(s ^ o, s ^ sh, s ^ oym, s ^ oyp, s ^ ozm, s ^ ozp);
        flip = packed_accept<DIMS, Digits, ILP9, ALIGNED>(k, valid, hbase, a, (uint32_t)a.c);
    } else if constexpr (RULE == kRuleMultiHit) {  // a.hits trials, neighbours fixed
        uint32_t cur = s;
#pragma unroll 1
        for (int m = 0; m < a.hits; ++m) {
            Counts k;
            if (DIMS == 2) {
                k = count2(cur ^ o, cur ^ sh, cur ^ oym, cur ^ oyp);
            } else {
                k = count3(cur ^ o, cur ^ sh, cur ^ oym, cur ^ oyp, cur ^ ozm, cur ^ ozp);
            }
            uint32_t f = k.always;
            const uint32_t need = ~k.always & valid;
            if (need)
                f |= packed_accept<DIMS, Counts, ILP9, ALIGNED>(k, need, hbase, a,
                                                               (uint32_t)a.c + 2u * (uint32_t)m);
            cur ^= f & valid;
        }
        flip = cur ^ s;
    } else {
        Counts k;
        if (DIMS == 2) {
            k = count2(s ^ o, s ^ sh, s ^ oym, s ^ oyp);
        } else {
            k = count3(s ^ o, s ^ sh, s ^ oym, s ^ oyp, s ^ ozm, s ^ ozp);
        }
        flip = k.always;
        const uint32_t need = ~k.always & valid;
        if (need) flip |= packed_accept<DIMS, Counts, ILP9, ALIGNED>(k, need, hbase, a, (uint32_t)a.c);
    }
    const uint32_t snew = s ^ (flip & valid);
    *own_word = snew;
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

template <int DIMS, bool MEASURE, int NC, int RULE = kRuleMetropolis, bool ILP9 = false>
__device__ __forceinline__ void packed_word(const PassArgs& a, uint32_t item, int& e_acc,
                                            int& m_acc, uint32_t rgroups = 1u) {
    const uint32_t W = (uint32_t)a.W;
    const uint32_t nq = (W + 31u) >> 5;
    const uint32_t L = (uint32_t)a.L;
    uint32_t* own = static_cast<uint32_t*>(a.own);
    const uint32_t* other = static_cast<const uint32_t*>(a.other);
    const uint32_t j = item / nq, q = item - j * nq;
    const uint32_t r = rgroups > 1u ? grouped_row(j, (uint32_t)a.rows, rgroups) : j;
    uint32_t y = r, z = 0;
    if (DIMS == 3) {
        z = r / L;
        y = r - z * L;
    }
    const uint32_t nb = W - 32u * q < 32u ? W - 32u * q : 32u;  // valid bits
    const uint32_t valid = nb == 32u ? 0xFFFFFFFFu : ((1u << nb) - 1u);
    const uint32_t plane = z * L;
    const uint32_t row = r * nq;
    const uint32_t o = load_other<NC>(other + row + q);
    const uint32_t oym = load_other<NC>(other + (plane + (y == 0u ? L - 1u : y - 1u)) * nq + q);
    const uint32_t oyp = load_other<NC>(other + (plane + (y + 1u == L ? 0u : y + 1u)) * nq + q);
    uint32_t ozm = 0u, ozp = 0u;
    if (DIMS == 3) {
        ozm = load_other<NC>(other + ((z == 0u ? L - 1u : z - 1u) * L + y) * nq + q);
        ozp = load_other<NC>(other + ((z + 1u == L ? 0u : z + 1u) * L + y) * nq + q);
    }
    const uint32_t s = own[row + q];
    const int p = (a.c + (int)y + (int)z) & 1;
    uint32_t sh;
    if (p == 0) {  // bit b <- neighbour xh - 1
        uint32_t prev;
        if (q == 0u) {  // wrap: the row's last site, moved to bit 31
            const uint32_t last = load_other<NC>(other + row + nq - 1u);
            prev = last << (31u - ((W - 1u) & 31u));
        } else {
            prev = load_other<NC>(other + row + q - 1u);
        }
        sh = __funnelshift_l(prev, o, 1);
    } else {       // bit b <- neighbour xh + 1
        if (q + 1u == nq) {  // wrap: bit nb - 1 takes the row's first site
            const uint32_t first = q == 0u ? o : load_other<NC>(other + row);
            const uint32_t top = 1u << (nb - 1u);
            sh = ((o >> 1) & ~top) | ((first & 1u) ? top : 0u);
        } else {
            sh = __funnelshift_r(o, load_other<NC>(other + row + q + 1u), 1);
        }
    }
    packed_update<DIMS, MEASURE, RULE, ILP9, false>(a, own + row + q, s, o, sh, oym, oyp, ozm,
                                                     ozp, valid, nb, r * W + 32u * q, e_acc,
                                                     m_acc);
}

}  // namespace ising
