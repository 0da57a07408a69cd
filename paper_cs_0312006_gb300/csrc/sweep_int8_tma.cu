// sweep_int8_tma.cu -- the int8 colour pass with its inputs staged in shared
// memory by the Tensor Memory Accelerator (bulk asynchronous copies).
//
// Same rule and draws as the register-window strip kernel (sweep_int8.cu,
// update_vec in pass_bodies.cuh); the data movement and the order of the work
// differ.  A tile is a band of R consecutive half rows of one plane (full
// width W = L/2 bytes, W % 16 == 0).  For each tile one thread issues
// cp.async.bulk copies of
//   - the tile's own-colour rows (R*W contiguous bytes),
//   - the other colour's rows y0-1 .. y0+R (the band plus one halo row on
//     each side; the halo rows wrap around the plane, so they are separate
//     copies),
//   - for 3D, the other colour's bands in planes z-1 and z+1,
// into one of S pipeline stages, completing on that stage's mbarrier.
// Persistent CTAs walk their tiles while the copies for the next S-1 tiles
// are in flight.  A tile's work items are (row pair, 16-byte column); a
// thread takes its items two at a time, reads each item's own and neighbour
// rows from shared memory (x-neighbour edge bytes from the adjacent column,
// so no shuffles), and writes the updated vectors straight to global memory.
// Its Philox calls run from counters alone: the first item's while the
// tile's copies land, the second item's round by round between the first
// item's word updates.
//
// Waits on an mbarrier are bounded: if a phase does not complete within the
// limit the kernel raises the error flag, waits (bounded again) for its own
// copies still in flight, and returns; the host reports ISING_ETIMEOUT.
#include <cstdint>
#include <type_traits>

#include "engine_internal.h"
#include "ising_device.cuh"
#include "pass_bodies.cuh"

namespace ising {

namespace {

constexpr int kStages = 2;

// Rows per tile: about 8 KiB of own-colour rows (two rows of a 2D L = 8192
// lattice, which measured best there against 1, 4 and 8), at least 2 and at
// most 64 rows, a power of two that divides L.
__host__ __device__ inline int tile_rows(int L) {
    const int W = L / 2;
    int R = 2;
    while (R < 64 && 2 * R * W <= 8192 && L % (2 * R) == 0) R *= 2;
    while (R > 1 && L % R != 0) R >>= 1;
    return R;
}
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // give up on a phase after ~1 s

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t done;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return done != 0u;
}

// Bounded wait for `phase` of `bar`: false once ~1 s of wall time has passed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
    if (mbar_try_wait(bar, phase)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, phase)) return true;
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
}

// One bulk copy global -> shared, completing `bytes` on `bar`.  Both addresses
// are 16-byte aligned and bytes is a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

struct TmaGeom {
    int R;          // rows per tile
    int tiles;      // tiles in the lattice
    int bands;      // tiles per plane: L / R
    int nv_shift;   // log2 of the 16-byte vectors per half row, or -1
    uint32_t stage_bytes;
    uint32_t extra_tx;  // test hook: bytes expected on the first tile that never arrive
};

// Offsets inside one stage: own rows [0, R*W), other rows y0-1..y0+R at
// [R*W, (2R+2)*W), 3D: other band of plane z-1, then z+1.
template <int DIMS>
__device__ __forceinline__ void issue_tile(const PassArgs& a, const TmaGeom& tg, int tile,
                                           unsigned char* stage, uint64_t* bar,
                                           uint32_t extra_tx) {
    const uint32_t W = (uint32_t)a.W, L = (uint32_t)a.L, R = (uint32_t)tg.R;
    const uint32_t z = DIMS == 3 ? (uint32_t)tile / (uint32_t)tg.bands : 0u;
    const uint32_t y0 = ((uint32_t)tile - z * (uint32_t)tg.bands) * R;
    const uint32_t plane = z * L;
    const unsigned char* own = static_cast<const unsigned char*>(a.own);
    const unsigned char* oth = static_cast<const unsigned char*>(a.other);
    mbar_expect_tx(bar, tg.stage_bytes + extra_tx);
    bulk_g2s(stage, own + (size_t)(plane + y0) * W, R * W, bar);
    unsigned char* o = stage + R * W;
    const uint32_t ym = y0 == 0u ? L - 1u : y0 - 1u;
    const uint32_t yp = y0 + R == L ? 0u : y0 + R;
    bulk_g2s(o, oth + (size_t)(plane + ym) * W, W, bar);
    bulk_g2s(o + W, oth + (size_t)(plane + y0) * W, R * W, bar);
    bulk_g2s(o + (R + 1u) * W, oth + (size_t)(plane + yp) * W, W, bar);
    if (DIMS == 3) {
        const uint32_t zm = z == 0u ? L - 1u : z - 1u, zp = z + 1u == L ? 0u : z + 1u;
        unsigned char* zb = o + (R + 2u) * W;
        bulk_g2s(zb, oth + (size_t)(zm * L + y0) * W, R * W, bar);
        bulk_g2s(zb + R * W, oth + (size_t)(zp * L + y0) * W, R * W, bar);
    }
}


// One item of the pair walk: two 16-byte vectors (the same column of a row
// pair), as their 8 words and byte-sliced disagreement counts D (byte j of D
// is 2 d_j), taken from shared memory when the item is loaded; step(w) then
// applies the rule to word w with its draw u (word w & 3 of call w: vector
// w >> 2).  Metropolis takes the counting mask (uphill_count, which holds the
// downhill flips too); the heat bath reads thr[d] per site from a shared
// table.  en sums 2 d_new per byte (at most 12 per word: eight words fit a
// byte), mn sums 2 per spin -1 (at most 16 per byte).
template <int DIMS, bool MEASURE, int RULE>
struct PairUpdate {
    uint32_t sv[8], D[8], rowg[2];
    uint32_t en, mn;

    __device__ __forceinline__ void set(int q, const uint4& S, const uint4& x, const uint4& xs,
                                        const uint4& ym, const uint4& yp, const uint4& zm,
                                        const uint4& zp, uint32_t row) {
        sv[4 * q + 0] = S.x;
        sv[4 * q + 1] = S.y;
        sv[4 * q + 2] = S.z;
        sv[4 * q + 3] = S.w;
        D[4 * q + 0] = disagreements<DIMS>(S.x, x.x, xs.x, ym.x, yp.x, zm.x, zp.x);
        D[4 * q + 1] = disagreements<DIMS>(S.y, x.y, xs.y, ym.y, yp.y, zm.y, zp.y);
        D[4 * q + 2] = disagreements<DIMS>(S.z, x.z, xs.z, ym.z, yp.z, zm.z, zp.z);
        D[4 * q + 3] = disagreements<DIMS>(S.w, x.w, xs.w, ym.w, yp.w, zm.w, zp.w);
        rowg[q] = row;
        if (q == 0) en = mn = 0u;
    }

    __device__ __forceinline__ void step(int w, const Philox4& u, const PassArgs& a,
                                         const uint32_t* s_thb) {
        uint32_t X;
        if constexpr (RULE == kRuleHeatBath) {
            const uint32_t uw[4] = {u.w0, u.w1, u.w2, u.w3};
            X = 0u;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t t = s_thb[(D[w] >> (8 * j + 1)) & 7u];
                X |= uw[j] < t ? (0xFEu << (8 * j)) : 0u;
            }
        } else {
            X = uphill_count<DIMS>(D[w], u, a);
        }
        const uint32_t out = sv[w] ^ X;
        if (MEASURE) {
            mn += out & kByteBit1;
            if (a.c == 1) {
                constexpr uint32_t q2 = 4u * DIMS * kByteOnes;
                en += (D[w] & ~X) | ((q2 - D[w]) & X);
            }
        }
        sv[w] = out;
    }

    __device__ __forceinline__ void store(uint4* own_g, const PassArgs& a, int& e_acc,
                                          int& m_neg) const {
        own_g[rowg[0]] = make_uint4(sv[0], sv[1], sv[2], sv[3]);
        own_g[rowg[1]] = make_uint4(sv[4], sv[5], sv[6], sv[7]);
        if (MEASURE) {
            m_neg += __dp4a((int)mn, (int)kByteOnes, 0) >> 1;
            if (a.c == 1) e_acc = __dp4a((int)en, (int)kByteOnes, e_acc);
        }
    }
};

// WALK: kWalkTwo when every thread has exactly two (row pair, column) items
// per tile (R / 2 * W / 16 == 2 * 128), kWalkOne when it has at most one,
// kWalkLoop otherwise.  The first two instances hold no loop over items and no
// guard, which keeps them clear of the register cap; the one-item instance
// runs six CTAs per SM (at most 85 registers; 3D L = 256 with 32-row tiles:
// 6.7e11 at four, 7.0e11 at five, 7.2e11 site updates/s at six).
constexpr int kWalkLoop = 0, kWalkTwo = 1, kWalkOne = 2;

template <int DIMS, bool MEASURE, int RULE, int WALK>
__global__ void __launch_bounds__(128, WALK == kWalkOne ? 6 : 4) pass_int8_tma(PassArgs a, TmaGeom tg, int* err) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bars[kStages];
    __shared__ uint32_t s_thb[8];  // heat bath: thr[d] by d, read per site
    const uint32_t W = (uint32_t)a.W, R = (uint32_t)tg.R;
    const uint32_t nv = W >> 4;
    // this CTA's tiles: blockIdx.x, blockIdx.x + gridDim.x, ...
    const int first = blockIdx.x;
    const int my_tiles = first < tg.tiles ? (tg.tiles - 1 - first) / (int)gridDim.x + 1 : 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    grid_dependency_wait();  // the previous pass has completed (no global access before)
    if (RULE == kRuleHeatBath && threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < 7; ++i) s_thb[i] = a.thr[i];
        s_thb[7] = 0u;
    }
    __syncthreads();
    launch_dependents();
    if (threadIdx.x == 0)
        for (int k = 0; k < kStages && k < my_tiles; ++k)
            issue_tile<DIMS>(a, tg, first + k * gridDim.x, smem + k * tg.stage_bytes, &bars[k],
                             k == 0 ? tg.extra_tx : 0u);

    int e_acc = 0, m_neg = 0, n_vec = 0;
    uint4* own_g = static_cast<uint4*>(a.own);
    // (row pair, column) item -> pair index and column
    auto split = [&](uint32_t item, uint32_t& pr, uint32_t& v) {
        if (tg.nv_shift >= 0) {
            pr = item >> tg.nv_shift;
            v = item & (nv - 1u);
        } else {
            pr = item / nv;
            v = item - pr * nv;
        }
    };
    for (int k = 0; k < my_tiles; ++k) {
        const int s = k % kStages;
        const uint32_t phase = (uint32_t)(k / kStages) & 1u;
        const int tile = first + k * gridDim.x;
        const uint32_t z = DIMS == 3 ? (uint32_t)tile / (uint32_t)tg.bands : 0u;
        const uint32_t y0 = ((uint32_t)tile - z * (uint32_t)tg.bands) * R;
        // a thread's first eight Philox calls depend only on counters: they
        // run while the tile's copies land.  An item's calls are two runs of
        // four consecutive groups (its two rows), so they go through
        // PhiloxRuns<2>; `start` makes the first round, and the caller runs
        // the other nine, alone (draw) or between other work (walk).
        Philox4 u0[8];
        using Runs = PhiloxRuns<2>;
        auto start = [&](auto single, uint32_t item, Runs& ps) {
            uint32_t pr = 0u, v = item;
            if constexpr (!decltype(single)::value) split(item, pr, v);
            const uint32_t rg = (z * (uint32_t)a.L + y0 + 2u * pr) * nv + v;
            const uint32_t base[2] = {rg * 4u, (rg + nv) * 4u};
            ps.first_round(base, a.t, (uint32_t)a.c, kTagSweep, a.key0, a.key1);
        };
        auto draw = [&](auto single, uint32_t item, Philox4 (&u)[8]) {
            Runs ps;
            start(single, item, ps);
#pragma unroll
            for (int r = 1; r < 10; ++r) ps.next_round();
#pragma unroll
            for (int w = 0; w < 8; ++w) u[w] = ps.result(w);
        };
        if (RULE == kRuleMetropolis || RULE == kRuleHeatBath) {
            if (R == 2u)  // one pair of rows per tile: an item is a column
                draw(std::true_type{}, threadIdx.x, u0);
            else
                draw(std::false_type{}, threadIdx.x, u0);
        }
        const bool ok = mbar_wait(&bars[s], phase);
        if (__syncthreads_or(!ok)) {
            // a phase never completed: raise the flag, let this CTA's copies in
            // flight land (bounded), and leave without a reduction
            if (threadIdx.x == 0) {
                *reinterpret_cast<volatile int*>(err) = 1;  // host-mapped flag: a plain store
                for (int k2 = k; k2 < my_tiles && k2 < k + kStages; ++k2)
                    (void)mbar_wait(&bars[k2 % kStages], (uint32_t)(k2 / kStages) & 1u);
            }
            return;
        }
        const unsigned char* st = smem + s * tg.stage_bytes;
        const uint4* own_s = reinterpret_cast<const uint4*>(st);
        const unsigned char* oth = st + R * W;  // row slot j holds y0 - 1 + j
        const uint4* oth16 = reinterpret_cast<const uint4*>(oth);
        const uint4* zm16 = reinterpret_cast<const uint4*>(oth + (R + 2u) * W);
        const uint4* zp16 = zm16 + R * nv;
        uint32_t i0 = 0;
        if (RULE == kRuleMetropolis || RULE == kRuleHeatBath) {
            // two rows per step: eight Philox calls in flight per thread (the
            // heat bath reads each site's threshold from s_thb: 8.07e11 site
            // updates/s per pass at L = 8192 against 6.59e11 one row at a time
            // with the counting test).  The calls need only counters, so they
            // are issued before the loads of the spins (3 % faster at L = 8192
            // than drawing after the neighbour counts).
            // items are (row pair, column) of the tile, columns fastest, so that
            // short rows (3D) still give every thread work.  A thread takes its
            // items two at a time: the second item's calls are issued between
            // the first item's loads and its update, so that the generator's
            // multiplies overlap the update's logic (39.6 -> 37.4 us per pass
            // at L = 8192 with 128-thread CTAs, two items per thread per tile).
            const uint32_t pairs = R >> 1, n_items = pairs * nv;
            using Pair = PairUpdate<DIMS, MEASURE, RULE>;
            // with one pair of rows per tile (pairs == 1, the 2D default) an item
            // is a column and every row index below is a constant
            auto load = [&](auto single, uint32_t item, Pair& d) {
                uint32_t pr = 0u, v = item;
                if constexpr (!decltype(single)::value) split(item, pr, v);
                const uint32_t ip = 2u * pr;  // the pair's first row in the tile
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const uint32_t i = ip + (uint32_t)q;
                    const uint32_t y = y0 + i;
                    const int p = (a.c + (int)y + (int)z) & 1;
                    const uint32_t* row32 = reinterpret_cast<const uint32_t*>(oth + (i + 1u) * W);
                    const uint4 oc = oth16[(i + 1u) * nv + v];
                    uint4 zm = make_uint4(0u, 0u, 0u, 0u), zp = zm;
                    if (DIMS == 3) {
                        zm = zm16[i * nv + v];
                        zp = zp16[i * nv + v];
                    }
                    uint4 xs;
                    if (p == 0) {
                        const uint32_t prev = row32[(v == 0u ? nv - 1u : v - 1u) * 4u + 3u];
                        xs = make_uint4(__funnelshift_l(prev, oc.x, 8), __funnelshift_l(oc.x, oc.y, 8),
                                        __funnelshift_l(oc.y, oc.z, 8), __funnelshift_l(oc.z, oc.w, 8));
                    } else {
                        const uint32_t next = row32[(v + 1u == nv ? 0u : v + 1u) * 4u];
                        xs = make_uint4(__funnelshift_r(oc.x, oc.y, 8), __funnelshift_r(oc.y, oc.z, 8),
                                        __funnelshift_r(oc.z, oc.w, 8), __funnelshift_r(oc.w, next, 8));
                    }
                    d.set(q, own_s[i * nv + v], oc, xs, oth16[i * nv + v], oth16[(i + 2u) * nv + v],
                          zm, zp, (z * (uint32_t)a.L + y) * nv + v);
                }
            };
            auto finish = [&](const Pair& d) {
                d.store(own_g, a, e_acc, m_neg);
                n_vec += 2;
            };
            auto update = [&](Pair& d, const Philox4 (&u)[8]) {
#pragma unroll
                for (int w = 0; w < 8; ++w) d.step(w, u[w], a, s_thb);
                finish(d);
            };
            // the first item's update with the second item's calls: round r of
            // the calls, then word r of the update (r < 8); the generator's
            // multiplies and the update's logic interleave in the instruction
            // stream (36.1 -> 35.2 us per pass at L = 8192, with the
            // first-round shortcut)
            auto update_drawing = [&](auto single, Pair& d, uint32_t next_item,
                                      Philox4 (&u)[8]) {
                Runs ps;
                start(single, next_item, ps);
                d.step(0, u0[0], a, s_thb);
#pragma unroll
                for (int r = 1; r < 10; ++r) {
                    ps.next_round();
                    if (r < 8) d.step(r, u0[r], a, s_thb);
                }
                finish(d);
#pragma unroll
                for (int w = 0; w < 8; ++w) u[w] = ps.result(w);
            };
            // order: the first item's loads, then its update with the second
            // item's calls, then the second item (the calls placed between
            // the loads and the update measured 7 % faster than ahead of the
            // loads)
            auto walk = [&](auto single) {
                for (uint32_t base = threadIdx.x; base < n_items; base += 2u * blockDim.x) {
                    const uint32_t second = base + blockDim.x;
                    Pair d0;
                    load(single, base, d0);
                    Philox4 u1[8];
                    // counters only: harmless past the last item
                    update_drawing(single, d0, second, u1);
                    if (second < n_items) {
                        Pair d1;
                        load(single, second, d1);
                        update(d1, u1);
                    }
                    if (base + 2u * blockDim.x < n_items)
                        draw(single, base + 2u * blockDim.x, u0);
                }
            };
            // the same order when every thread has exactly two items (no loop,
            // no guard: 39.3 -> 38.0 us per pass at L = 8192, as the guards and
            // the loop-carried draws had held the kernel at its register cap)
            auto walk_two = [&](auto single) {
                const uint32_t second = threadIdx.x + blockDim.x;
                Pair d0;
                load(single, threadIdx.x, d0);
                Philox4 u1[8];
                update_drawing(single, d0, second, u1);
                Pair d1;
                load(single, second, d1);
                update(d1, u1);
            };
            // at most one item per thread: nothing more to draw
            auto walk_one = [&](auto single) {
                if (threadIdx.x < n_items) {
                    Pair d0;
                    load(single, threadIdx.x, d0);
                    update(d0, u0);
                }
            };
            if constexpr (WALK == kWalkTwo) {
                if (pairs == 1u) walk_two(std::true_type{});
                else walk_two(std::false_type{});
            } else if constexpr (WALK == kWalkOne) {
                if (pairs == 1u) walk_one(std::true_type{});
                else walk_one(std::false_type{});
            } else {
                if (pairs == 1u) walk(std::true_type{});
                else walk(std::false_type{});
            }
            i0 = 2u * pairs;
        }
        for (uint32_t i = i0; i < R; ++i) {
            const uint32_t y = y0 + i;
            const int p = (a.c + (int)y + (int)z) & 1;
            const uint32_t* row32 = reinterpret_cast<const uint32_t*>(oth + (i + 1u) * W);
            // columns fastest across the threads: a warp reads contiguous shared memory
            for (uint32_t v = threadIdx.x; v < nv; v += blockDim.x) {
                const uint4 oc = oth16[(i + 1u) * nv + v];
                const uint4 om = oth16[i * nv + v];
                const uint4 op = oth16[(i + 2u) * nv + v];
                uint4 zm = make_uint4(0u, 0u, 0u, 0u), zp = zm;
                if (DIMS == 3) {
                    zm = zm16[i * nv + v];
                    zp = zp16[i * nv + v];
                }
                uint4 sh;
                if (p == 0) {  // byte j <- byte j - 1 (wrapping to the row's last byte)
                    const uint32_t prev = row32[(v == 0u ? nv - 1u : v - 1u) * 4u + 3u];
                    sh = make_uint4(__funnelshift_l(prev, oc.x, 8), __funnelshift_l(oc.x, oc.y, 8),
                                    __funnelshift_l(oc.y, oc.z, 8), __funnelshift_l(oc.z, oc.w, 8));
                } else {       // byte j <- byte j + 1 (wrapping to the row's first byte)
                    const uint32_t next = row32[(v + 1u == nv ? 0u : v + 1u) * 4u];
                    sh = make_uint4(__funnelshift_r(oc.x, oc.y, 8), __funnelshift_r(oc.y, oc.z, 8),
                                    __funnelshift_r(oc.z, oc.w, 8), __funnelshift_r(oc.w, next, 8));
                }
                const uint32_t row = (z * (uint32_t)a.L + y) * nv + v;  // global vector index
                int e_vec = 0;
                own_g[row] = update_vec<DIMS, MEASURE, RULE>(own_s[i * nv + v], oc, sh, om, op,
                                                             zm, zp, row * 4u, a, e_vec, m_neg);
                e_acc += e_vec;
                ++n_vec;
            }
        }
        __syncthreads();  // every thread is done with stage s
        if (threadIdx.x == 0 && k + kStages < my_tiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_tile<DIMS>(a, tg, first + (k + kStages) * gridDim.x, smem + s * tg.stage_bytes,
                             &bars[s], 0u);
        }
    }
    if (MEASURE) {
        if (a.c == 1) e_acc -= n_vec * 16 * 2 * DIMS;  // E_white = sum (2 d_new - 2 dims)
        block_reduce_add(e_acc, n_vec * 16 - 2 * m_neg, a.obs, a.c == 1);
    }
}

template <int DIMS, bool MEASURE, int RULE, int WALK>
cudaError_t launch_tma_t(const PassArgs& a, const DeviceProps& dp, int* err, uint32_t extra_tx,
                         cudaStream_t st, int rows_per_tile, int ctas_per_sm) {
    TmaGeom tg;
    tg.extra_tx = extra_tx;
    const int planes = DIMS == 3 ? a.L : 1;
    // default: tile_rows() (2D L = 8192: two rows, measured best against 1, 4
    // and 8) and 128 threads, each taking its (row pair, column) items two at
    // a time; a tuned configuration may ask for other rows per tile
    const int R = rows_per_tile > 0 ? rows_per_tile : tile_rows(a.L);
    const int threads = 128;  // two items per thread per 2-row tile at L = 8192
    tg.R = R;
    tg.bands = a.L / R;
    const int nv = a.W >> 4;
    tg.nv_shift = (nv & (nv - 1)) == 0 ? __builtin_ctz((unsigned)nv) : -1;
    tg.tiles = tg.bands * planes;
    const uint32_t W = (uint32_t)a.W;
    tg.stage_bytes = (uint32_t)(2 * R + 2) * W + (DIMS == 3 ? 2u * R * W : 0u);
    const size_t smem = (size_t)kStages * tg.stage_bytes;
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    static int attr_set = 0;  // largest dynamic shared memory opted into so far
    cudaError_t e = cudaSuccess;
    if ((int)smem > attr_set) {
        e = cudaFuncSetAttribute(pass_int8_tma<DIMS, MEASURE, RULE, WALK>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set = 200 * 1024;
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pass_int8_tma<DIMS, MEASURE, RULE, WALK>,
                                                      threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    int grid = dp.sm_count * per_sm;
    if (grid > tg.tiles) grid = tg.tiles;
    return launch_chained(pass_int8_tma<DIMS, MEASURE, RULE, WALK>, (unsigned)grid, (unsigned)threads,
                          smem, st, a, tg, err);
}

}  // namespace

// The staged kernel needs W % 16 == 0, R rows per tile dividing L (R = 0:
// the default tile_rows) and its stages (2 x (2R+2) half rows, plus 2 x 2R
// for 3D) to fit in shared memory.
bool int8_tma_ok(int dims, int L, int rows_per_tile) {
    const int W = L / 2;
    if (W % 16 != 0) return false;
    const int R = rows_per_tile > 0 ? rows_per_tile : tile_rows(L);
    if (R < 1 || L % R != 0) return false;
    const size_t stage = (size_t)(2 * R + 2) * W + (dims == 3 ? 2u * R * W : 0u);
    return (size_t)kStages * stage <= 200 * 1024;
}

template <int RULE, int WALK>
static cudaError_t int8_pass_tma_walk(const PassArgs& a, int dims, bool measure,
                                      const DeviceProps& dp, int* err, uint32_t extra_tx,
                                      cudaStream_t st, int R, int ctas) {
    if (dims == 2)
        return measure ? launch_tma_t<2, true, RULE, WALK>(a, dp, err, extra_tx, st, R, ctas)
                       : launch_tma_t<2, false, RULE, WALK>(a, dp, err, extra_tx, st, R, ctas);
    return measure ? launch_tma_t<3, true, RULE, WALK>(a, dp, err, extra_tx, st, R, ctas)
                   : launch_tma_t<3, false, RULE, WALK>(a, dp, err, extra_tx, st, R, ctas);
}

template <int RULE>
static cudaError_t int8_pass_tma_rule(const PassArgs& a, int dims, bool measure,
                                      const DeviceProps& dp, int* err, uint32_t extra_tx,
                                      cudaStream_t st, int R, int ctas) {
    if constexpr (RULE == kRuleMultiHit) {  // takes the row-at-a-time loop only
        return int8_pass_tma_walk<RULE, kWalkLoop>(a, dims, measure, dp, err, extra_tx, st, R,
                                                   ctas);
    } else {
        const int rows = R > 0 ? R : tile_rows(a.L);
        const int items = (rows / 2) * (a.W / 16);  // (row pair, column) items per tile
        if (items == 2 * 128)                        // 128 threads per CTA
            return int8_pass_tma_walk<RULE, kWalkTwo>(a, dims, measure, dp, err, extra_tx, st, R,
                                                      ctas);
        if (items <= 128)
            return int8_pass_tma_walk<RULE, kWalkOne>(a, dims, measure, dp, err, extra_tx, st, R,
                                                      ctas);
        return int8_pass_tma_walk<RULE, kWalkLoop>(a, dims, measure, dp, err, extra_tx, st, R,
                                                   ctas);
    }
}

// Where the staged kernel measured faster than the strip kernel on GB300: 2D
// with long rows (L >= 4096) while two CTAs' stages fit in one SM's shared
// memory (L <= 16384: 8.38e11 against 7.76e11 site updates/s per pass at
// L = 16384; at L = 32768 one CTA per SM gives 7.24e11 against the strip
// kernel's 8.02e11).  With short rows (3D, small 2D) a tile holds about one
// vector per thread and its barriers dominate.
bool int8_tma_preferred(int dims, int L) {
    if (dims != 2 || L < 4096 || !int8_tma_ok(dims, L, 0)) return false;
    const int W = L / 2, R = tile_rows(L);
    return 2 * (size_t)kStages * (size_t)(2 * R + 2) * W <= 200 * 1024;
}

cudaError_t int8_pass_tma(const PassArgs& a, int dims, bool measure, int rule,
                          const DeviceProps& dp, int* err, uint32_t extra_tx, cudaStream_t st,
                          int rows_per_tile, int ctas_per_sm) {
    if (rule == kRuleHeatBath)
        return int8_pass_tma_rule<kRuleHeatBath>(a, dims, measure, dp, err, extra_tx, st,
                                                 rows_per_tile, ctas_per_sm);
    if (rule == kRuleMultiHit)
        return int8_pass_tma_rule<kRuleMultiHit>(a, dims, measure, dp, err, extra_tx, st,
                                                 rows_per_tile, ctas_per_sm);
    return int8_pass_tma_rule<kRuleMetropolis>(a, dims, measure, dp, err, extra_tx, st,
                                               rows_per_tile, ctas_per_sm);
}

}  // namespace ising
