// engine.cu -- host side of the C ABI declared in include/ising.h: lattice
// handles, acceptance thresholds, the per-sweep launch sequence and the E/M
// record buffer.  All simulation arithmetic runs in the kernels of
// sweep_int8.cu / sweep_bitpack.cu.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "engine_internal.h"
#include "ising.h"
#include "ising_device.cuh"

using ising::DeviceProps;
using ising::PassArgs;

static_assert(ising::kRuleMetropolis == ISING_RULE_METROPOLIS, "rule values");
static_assert(ising::kRuleHeatBath == ISING_RULE_HEATBATH, "rule values");
static_assert(ising::kRuleDemon == ISING_RULE_DEMON, "rule values");
static_assert(ising::kRuleMultiHit == ISING_RULE_MULTIHIT, "rule values");

namespace {

constexpr uint64_t kMaxSites = 1ull << 32;  // 32-bit half indices in the kernels

std::mutex g_props_mu;
DeviceProps g_props[64];

}  // namespace

namespace ising {

int cuda_fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? ISING_ENOMEM : ISING_ECUDA; }

#define ISING_CHECK(call)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return ising::cuda_fail(e_); \
    } while (0)

int device_props(const DeviceProps** out) {
    int dev = 0;
    ISING_CHECK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return ISING_ECUDA;
    std::lock_guard<std::mutex> lk(g_props_mu);
    DeviceProps& p = g_props[dev];
    if (p.device != dev) {
        DeviceProps q;
        q.device = dev;
        ISING_CHECK(cudaDeviceGetAttribute(&q.sm_count, cudaDevAttrMultiProcessorCount, dev));
        ISING_CHECK(ising::int8_query_occupancy(q));
        ISING_CHECK(ising::packed_query_occupancy(q));
        ISING_CHECK(ising::demon_query_occupancy(q));
        void* flag = nullptr;
        ISING_CHECK(cudaHostAlloc(&flag, sizeof(int), cudaHostAllocMapped));
        q.h_err = static_cast<volatile int*>(flag);
        *q.h_err = 0;
        ISING_CHECK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&q.d_err), flag, 0));
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        ISING_CHECK(cudaMemPoolCreate(&q.pool, &props));
        uint64_t keep = UINT64_MAX;  // never hand freed blocks back on a synchronisation
        ISING_CHECK(cudaMemPoolSetAttribute(q.pool, cudaMemPoolAttrReleaseThreshold, &keep));
        p = q;
    }
    *out = &p;
    return ISING_OK;
}

cudaError_t pool_alloc(void** p, size_t bytes, const DeviceProps& dp, cudaStream_t st) {
    return cudaMallocFromPoolAsync(p, bytes, dp.pool, st);
}

// floor(exp(-x) * 2^32) for x = 2 beta k > 0, decided exactly.  The double
// result is accepted when a relative bracket of 2^-40 around it (far wider than
// the error of exp() and of forming x) holds no integer; otherwise the value
// is recomputed in long double with a 2^-56 bracket; if even that straddles an
// integer the input is refused rather than rounded either way.
int floor_exp_scaled(double beta, int k, uint32_t* out) {
    const double x = 2.0 * beta * (double)k;
    if (std::isinf(x)) {
        *out = 0u;
        return ISING_OK;
    }
    if (x < 0x1p-33) {  // 2^32 (1 - x) <= value < 2^32, so the floor is 2^32 - 1
        *out = 0xFFFFFFFFu;
        return ISING_OK;
    }
    const double v = std::ldexp(std::exp(-x), 32);
    const double lo = v * (1.0 - 0x1p-40), hi = v * (1.0 + 0x1p-40);
    if (hi < 1.0) {
        *out = 0u;
        return ISING_OK;
    }
    if (std::floor(lo) == std::floor(hi)) {
        *out = (uint32_t)std::floor(v);
        return ISING_OK;
    }
    const long double xl = 2.0L * (long double)beta * (long double)k;
    const long double vl = std::ldexp(std::exp(-xl), 32);
    const long double lol = vl * (1.0L - 0x1p-56L), hil = vl * (1.0L + 0x1p-56L);
    if (std::floor(lol) != std::floor(hil)) return ISING_EINVAL;
    *out = (uint32_t)std::floor(vl);
    return ISING_OK;
}

int build_thresholds(int dims, double beta, uint32_t thr[3]) {
    if (!(beta > 0.0)) return ISING_EINVAL;  // also rejects NaN
    thr[0] = thr[1] = thr[2] = 0u;
    for (int j = 0; j < dims; ++j) {
        const int rc = floor_exp_scaled(beta, 2 * (j + 1), &thr[j]);
        if (rc != ISING_OK) return rc;
    }
    return ISING_OK;
}

// floor(2^32 / (1 + e^x)) for the heat-bath flip probability, x = 4 beta m,
// m = dims - d.  s = 2^32 / (1 + e^|x|) is the less likely outcome's share; the
// threshold is floor(s) for m > 0 and floor(2^32 - s) = 2^32 - 1 - floor(s) for
// m < 0 (s is never an integer there: the bracket test below excludes it).  s is
// decided with the same relative brackets as floor_exp_scaled; near x = 0 the
// answer is fixed by 0 < 2^31 - s = 2^31 tanh(|x| / 2) < 2^31 |x| / 2 < 1.
int floor_logistic_scaled(double beta, int m, uint32_t* out) {
    if (m == 0) {
        *out = 0x80000000u;
        return ISING_OK;
    }
    const int am = m < 0 ? -m : m;
    const double x = 4.0 * beta * (double)am;
    uint32_t fs;
    if (std::isinf(x) || x > 64.0) {
        fs = 0u;  // 0 < s < 2^32 e^-64 < 1
    } else if (x < 0x1p-32) {
        fs = 0x7FFFFFFFu;
    } else {
        const double v = std::ldexp(1.0 / (1.0 + std::exp(x)), 32);
        const double lo = v * (1.0 - 0x1p-40), hi = v * (1.0 + 0x1p-40);
        if (std::floor(lo) == std::floor(hi)) {
            fs = (uint32_t)std::floor(v);
        } else {
            const long double xl = 4.0L * (long double)beta * (long double)am;
            const long double vl = std::ldexp(1.0L / (1.0L + std::exp(xl)), 32);
            const long double lol = vl * (1.0L - 0x1p-56L), hil = vl * (1.0L + 0x1p-56L);
            if (std::floor(lol) != std::floor(hil)) return ISING_EINVAL;
            fs = (uint32_t)std::floor(vl);
        }
    }
    *out = m > 0 ? fs : 0xFFFFFFFFu - fs;
    return ISING_OK;
}

int build_thresholds_heatbath(int dims, double beta, uint32_t thb[7]) {
    if (!(beta > 0.0)) return ISING_EINVAL;
    for (int d = 0; d < 7; ++d) thb[d] = 0u;
    for (int d = 0; d <= 2 * dims; ++d) {
        const int rc = floor_logistic_scaled(beta, dims - d, &thb[d]);
        if (rc != ISING_OK) return rc;
    }
    return ISING_OK;
}

void rule_thresholds(const ising_lattice* h, uint32_t out[7]) {
    for (int i = 0; i < 7; ++i) out[i] = 0u;
    if (h->rule == ISING_RULE_HEATBATH)
        std::memcpy(out, h->thb, sizeof(h->thb));
    else
        std::memcpy(out, h->thr, sizeof(h->thr));
}

// Device buffers go back to the pool in the handle's stream order (after the
// work already queued there), so nothing waits here.
void free_device(ising_lattice* h) {
    for (void*& p : h->col) {
        if (p) cudaFreeAsync(p, h->stream);
        p = nullptr;
    }
    for (void*& p : h->dem) {
        if (p) cudaFreeAsync(p, h->stream);
        p = nullptr;
    }
    if (h->obs) cudaFreeAsync(h->obs, h->stream);
    h->obs = nullptr;
    if (h->host_obs) cudaFreeHost(h->host_obs);
    h->host_obs = nullptr;
    h->host_obs_cap = 0;
    h->obs_cap = 0;
    if (h->bad_host) cudaFreeHost(const_cast<int*>(h->bad_host));
    h->bad_host = nullptr;
    h->bad_dev = nullptr;

}

// Record slots at index >= n_rec are kept zero, so a sweep call never needs
// its own memset: the fused kernels add into already-zeroed slots.
int ensure_records(ising_lattice* h, int64_t need) {
    if (need <= h->obs_cap) return ISING_OK;
    int64_t cap = h->obs_cap * 2;
    if (cap < need) cap = need;
    if (cap < 64) cap = 64;
    unsigned long long* nb = nullptr;
    ISING_CHECK(pool_alloc(reinterpret_cast<void**>(&nb), (size_t)cap * 16, *h->dp, h->stream));
    ISING_CHECK(cudaMemsetAsync(nb, 0, (size_t)cap * 16, h->stream));
    if (h->n_rec > 0)
        ISING_CHECK(cudaMemcpyAsync(nb, h->obs, (size_t)h->n_rec * 16, cudaMemcpyDeviceToDevice,
                                    h->stream));
    if (h->obs) ISING_CHECK(cudaFreeAsync(h->obs, h->stream));
    h->obs = nb;
    h->obs_cap = cap;
    return ISING_OK;
}

// Drop pending records and restore the zero invariant of their slots.
int clear_records(ising_lattice* h) {
    if (h->n_rec > 0)
        ISING_CHECK(cudaMemsetAsync(h->obs, 0, (size_t)h->n_rec * 16, h->stream));
    h->n_rec = 0;
    return ISING_OK;
}

std::atomic<int> g_inject_timeout{0};

bool injecting_timeout() { return g_inject_timeout.load() != 0; }

// Read and clear the device's bounded-wait flag and the handle's invalid-input
// flag (after a synchronisation).
int check_bad_input(ising_lattice* h) {
    if (!h->bad_host || *h->bad_host == 0) return ISING_OK;
    *h->bad_host = 0;
    return ISING_EINVAL;
}

int check_timeout(ising_lattice* h) {
    const int rc = check_bad_input(h);
    if (rc != ISING_OK) return rc;
    if (*h->dp->h_err == 0) return ISING_OK;
    *h->dp->h_err = 0;
    return ISING_ETIMEOUT;
}

// Bytes of one colour array that hold sites (without the spare tail).
size_t col_data_bytes(const ising_lattice* h) {
    return h->layout == ISING_BITPACK
               ? (size_t)h->rows * (size_t)((h->L / 2 + 31) / 32) * sizeof(uint32_t)
               : (size_t)h->half_sites;
}

// Canonical spins out of the layout into `dst` (device-writable; may be mapped
// host memory), on the handle's stream.
cudaError_t export_spins(ising_lattice* h, int8_t* dst) {
    if (rows_ok(h->layout, h->L) && ((uintptr_t)dst & 15u) == 0)
        return rows_export(h->col[0], h->col[1], dst, h->layout, h->L, h->rows, *h->dp,
                           h->stream);
    if (h->layout == ISING_BITPACK)
        return packed_export(static_cast<const uint32_t*>(h->col[0]),
                             static_cast<const uint32_t*>(h->col[1]), dst, h->L, h->dims,
                             h->sites, *h->dp, h->stream);
    return int8_export(static_cast<const int8_t*>(h->col[0]),
                       static_cast<const int8_t*>(h->col[1]), dst, h->L, h->dims, h->sites,
                       *h->dp, h->stream);
}

// Canonical spins from `src` (device-readable) into the layout; with `bad`
// every byte is checked on the device and the flag raised if one is not +-1.
cudaError_t import_spins(ising_lattice* h, const int8_t* src, int* bad) {
    if (rows_ok(h->layout, h->L) && ((uintptr_t)src & 15u) == 0)
        return rows_import(h->col[0], h->col[1], src, h->layout, h->L, h->rows, bad, *h->dp,
                           h->stream);
    if (bad) {
        const cudaError_t e = check_spins(src, h->sites, bad, *h->dp, h->stream);
        if (e != cudaSuccess) return e;
    }
    if (h->layout == ISING_BITPACK)
        return packed_import(static_cast<uint32_t*>(h->col[0]), static_cast<uint32_t*>(h->col[1]),
                             src, h->L, h->dims, h->rows, *h->dp, h->stream);
    return int8_import(static_cast<int8_t*>(h->col[0]), static_cast<int8_t*>(h->col[1]), src,
                       h->L, h->dims, h->sites, *h->dp, h->stream);
}

// Records of several lattices in one launch (ising_observables_gather): one
// CTA walks the chunk's lattices, copies each one's pending (E, M) pairs to
// `out` (mapped pinned host memory) at its offset and zeroes them, restoring
// the zero invariant of the slots; then, if `flag` is set, it stores `value`
// there (mapped pinned host memory too) after a system-scope fence, so a host
// that sees the value also sees the records.
constexpr int kGatherChunk = 64;
struct GatherChunk {
    unsigned long long* src[kGatherChunk];
    int64_t n[kGatherChunk];
    int64_t off[kGatherChunk];
    int count;
};

__global__ void gather_records_kernel(GatherChunk c, long long* out, long long* flag,
                                      long long value) {
    grid_dependency_wait();  // the sweeps that wrote the records have completed
    launch_dependents();
    for (int i = 0; i < c.count; ++i) {
        unsigned long long* src = c.src[i];
        long long* dst = out + 2 * c.off[i];
        for (int64_t j = threadIdx.x; j < 2 * c.n[i]; j += blockDim.x) {
            dst[j] = (long long)src[j];
            src[j] = 0ull;
        }
    }
    if (flag) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence_system();
            *reinterpret_cast<volatile long long*>(flag) = value;
        }
    }
}

// Tuned int8 pass configurations (ising_set_int8_config): for lattices of
// dims and L_min <= L <= L_max, ISING_KERNEL_AUTO runs `cfg`; the latest
// matching entry wins.
struct Int8Policy {
    int dims, L_min, L_max;
    ising_int8_config cfg;
};
std::mutex g_policy_mu;
std::vector<Int8Policy> g_policy;

bool find_policy(int dims, int L, ising_int8_config* out) {
    std::lock_guard<std::mutex> lk(g_policy_mu);
    for (auto it = g_policy.rbegin(); it != g_policy.rend(); ++it)
        if (it->dims == dims && it->L_min <= L && L <= it->L_max) {
            *out = it->cfg;
            return true;
        }
    return false;
}

// The int8 pass a lattice runs: the kernel, and for the staged kernel its
// rows per tile and CTAs per SM (0: defaults).
ising_int8_config resolve_int8(const ising_lattice* h) {
    ising_int8_config c = {ISING_KERNEL_STRIP, 0, 0};
    if (h->layout == ISING_BITPACK) return c;
    ising_int8_config tuned;
    const bool have = find_policy(h->dims, h->L, &tuned);
    if (h->kernel == ISING_KERNEL_TMA) {
        c.kernel = ISING_KERNEL_TMA;
        if (have && tuned.kernel == ISING_KERNEL_TMA) {
            c.tile_rows = tuned.tile_rows;
            c.ctas_per_sm = tuned.ctas_per_sm;
        }
    } else if (h->kernel == ISING_KERNEL_AUTO) {
        if (have)
            c = tuned;
        else if (ising::int8_tma_preferred(h->dims, h->L))
            c.kernel = ISING_KERNEL_TMA;
    }
    if (c.kernel == ISING_KERNEL_TMA && !ising::int8_tma_ok(h->dims, h->L, c.tile_rows)) {
        // the staged kernel cannot take this shape: the general kernels run
        c.kernel = ISING_KERNEL_STRIP;
        c.tile_rows = c.ctas_per_sm = 0;
    }
    if (c.kernel != ISING_KERNEL_TMA) c.tile_rows = c.ctas_per_sm = 0;
    return c;
}

bool uses_tma(const ising_lattice* h) { return resolve_int8(h).kernel == ISING_KERNEL_TMA; }

int run_pass(ising_lattice* h, int c, uint32_t t, unsigned long long* slot) {
    PassArgs a;
    a.own = h->col[c];
    a.other = h->col[1 - c];
    a.obs = slot;
    a.rows = h->rows;
    a.L = h->L;
    a.W = h->W;
    rule_thresholds(h, a.thr);
    a.key0 = (uint32_t)(h->seed & 0xFFFFFFFFu);
    a.key1 = (uint32_t)(h->seed >> 32);
    a.t = t;
    a.c = c;
    a.dem = nullptr;
    a.qmax = 0;
    a.rot = 0;
    a.hits = h->hits;
    if (h->rule == ISING_RULE_DEMON) {
        a.dem = h->dem[c];
        a.qmax = h->qmax;
        a.rot = (uint32_t)h->dem_rot;
        if (h->layout == ISING_BITPACK)
            ISING_CHECK(ising::demon_packed_pass(a, h->dims, slot != nullptr, *h->dp, h->stream));
        else
            ISING_CHECK(ising::demon_pass(a, h->dims, h->half_sites, slot != nullptr, *h->dp,
                                          h->stream));
        if (c == 1) h->dem_rot = h->dem_rot + 1 == h->rows ? 0 : h->dem_rot + 1;
        return ISING_OK;
    }
    if (h->layout == ISING_BITPACK)
        ISING_CHECK(ising::packed_pass(a, h->dims, slot != nullptr, h->rule, *h->dp, h->stream));
    else if (const ising_int8_config c = resolve_int8(h); c.kernel == ISING_KERNEL_TMA)
        ISING_CHECK(ising::int8_pass_tma(a, h->dims, slot != nullptr, h->rule, *h->dp,
                                         h->dp->d_err, g_inject_timeout.load() ? 16u : 0u,
                                         h->stream, c.tile_rows, c.ctas_per_sm));
    else
        ISING_CHECK(ising::int8_pass(a, h->dims, h->half_sites, slot != nullptr, h->rule,
                                     *h->dp, h->stream));
    return ISING_OK;
}

}  // namespace ising

using namespace ising;

extern "C" {

const char* ising_version(void) { return "paper_cs_0312006_gb300 1.0 (sm_103a)"; }

const char* ising_strerror(int code) {
    switch (code) {
        case ISING_OK: return "ok";
        case ISING_EINVAL: return "invalid argument";
        case ISING_ENOMEM: return "out of memory";
        case ISING_ECUDA: return "CUDA error";
        case ISING_ETIMEOUT: return "bounded device wait timed out";
        case ISING_EBUDGET: return "memory budget exceeded";
        case ISING_ERANGE: return "counter or capacity out of range";
        default: return "unknown status";
    }
}

int ising_create(ising_lattice** out, int dims, int L, double beta, uint64_t seed, int layout) {
    if (!out) return ISING_EINVAL;
    *out = nullptr;
    if (dims != 2 && dims != 3) return ISING_EINVAL;
    if (L < 2 || (L & 1)) return ISING_EINVAL;
    if (layout != ISING_INT8 && layout != ISING_BITPACK && layout != ISING_AUTO)
        return ISING_EINVAL;
    const uint64_t sites = dims == 2 ? (uint64_t)L * L : (uint64_t)L * L * L;
    if ((uint64_t)L > (1u << 20) || sites > kMaxSites) return ISING_EINVAL;
    // ISING_AUTO: the bit-packed layout, the faster of the two on this GPU
    // (results are identical in both layouts)
    const int use_layout = layout == ISING_AUTO ? ISING_BITPACK : layout;
    uint32_t thr[3], thb[7];
    int rc = build_thresholds(dims, beta, thr);
    if (rc == ISING_OK) rc = build_thresholds_heatbath(dims, beta, thb);
    if (rc != ISING_OK) return rc;
    const DeviceProps* dp = nullptr;
    rc = device_props(&dp);
    if (rc != ISING_OK) return rc;

    ising_lattice* h = new (std::nothrow) ising_lattice();
    if (!h) return ISING_ENOMEM;
    h->dims = dims;
    h->L = L;
    h->layout = use_layout;
    h->beta = beta;
    h->seed = seed;
    std::memcpy(h->thr, thr, sizeof(thr));
    std::memcpy(h->thb, thb, sizeof(thb));
    h->sites = (int64_t)sites;
    h->half_sites = (int64_t)(sites / 2);
    h->W = L / 2;
    h->rows = dims == 2 ? L : (int64_t)L * L;
    h->dp = dp;
    // 16 spare bytes: the word kernels may read one word past the last one
    if (use_layout == ISING_BITPACK)
        h->col_bytes = (size_t)h->rows * (size_t)((L / 2 + 31) / 32) * sizeof(uint32_t) + 16;
    else
        h->col_bytes = (((size_t)h->half_sites + 15) & ~(size_t)15) + 16;
    for (int c = 0; c < 2; ++c) {
        cudaError_t e = ising::pool_alloc(&h->col[c], h->col_bytes, *dp, h->stream);
        if (e != cudaSuccess) {
            free_device(h);
            delete h;
            return cuda_fail(e);
        }
    }
    rc = ising_init(h, ISING_HOT);
    if (rc != ISING_OK) {
        free_device(h);
        delete h;
        return rc;
    }
    *out = h;
    return ISING_OK;
}

int ising_init(ising_lattice* h, int start) {
    if (!h) return ISING_EINVAL;
    if (start != ISING_HOT && start != ISING_COLD_UP && start != ISING_COLD_DOWN)
        return ISING_EINVAL;
    const uint32_t k0 = (uint32_t)(h->seed & 0xFFFFFFFFu), k1 = (uint32_t)(h->seed >> 32);
    if (ising::rows_ok(h->layout, h->L))
        ISING_CHECK(ising::rows_init(h->col[0], h->col[1], ising::col_data_bytes(h), h->layout,
                                     h->L, h->rows, start, k0, k1, *h->dp, h->stream));
    else if (h->layout == ISING_BITPACK)
        ISING_CHECK(ising::packed_init(static_cast<uint32_t*>(h->col[0]),
                                       static_cast<uint32_t*>(h->col[1]), h->L, h->dims, h->rows,
                                       start, k0, k1, *h->dp, h->stream));
    else
        ISING_CHECK(ising::int8_init(static_cast<int8_t*>(h->col[0]),
                                     static_cast<int8_t*>(h->col[1]), h->L, h->dims, h->sites,
                                     start, k0, k1, *h->dp, h->stream));
    h->t = 0;
    return clear_records(h);
}

int ising_sweep(ising_lattice* h, int64_t n, int measure_every) {
    if (!h || n < 0 || measure_every < 1) return ISING_EINVAL;
    if (n == 0) return ISING_OK;
    if (h->t + (uint64_t)n - 1 > kMaxSweep) return ISING_ERANGE;
    const uint64_t every = (uint64_t)measure_every;
    const int64_t new_rec = (int64_t)((h->t + (uint64_t)n) / every - h->t / every);
    if (new_rec > 0) {
        int rc = ensure_records(h, h->n_rec + new_rec);
        if (rc != ISING_OK) return rc;
    }
    int64_t rec = h->n_rec;
    if (h->sites <= kSmallSites && n >= 2 && n <= 0x7FFFFFFF &&
        (h->rule == ISING_RULE_METROPOLIS || h->rule == ISING_RULE_HEATBATH)) {
        const int rc = small_sweep(h, n, measure_every, h->obs ? h->obs + 2 * rec : nullptr);
        if (rc != ISING_OK) return rc;
        h->t += (uint64_t)n;
        h->n_rec = rec + new_rec;
        return ISING_OK;
    }
    for (int64_t s = 0; s < n; ++s) {
        const uint64_t t = h->t + (uint64_t)s;
        unsigned long long* slot = nullptr;
        if ((t + 1) % every == 0) slot = h->obs + 2 * (rec++);
        int rc = run_pass(h, 0, (uint32_t)t, slot);
        if (rc == ISING_OK) rc = run_pass(h, 1, (uint32_t)t, slot);
        if (rc != ISING_OK) return rc;
    }
    h->t += (uint64_t)n;
    h->n_rec = rec;
    return ISING_OK;
}

int ising_observables(ising_lattice* h, int64_t* E, int64_t* M, int64_t cap, int64_t* count) {
    if (!h) return ISING_EINVAL;
    const int64_t n = h->n_rec;
    // the copy into pinned staging and the clearing memset go ahead of the one
    // synchronisation, so a read costs a single round trip
    const bool copy = E && M && n > 0 && cap >= n;
    if (copy) {
        if (h->host_obs_cap < n) {
            if (h->host_obs) ISING_CHECK(cudaFreeHost(h->host_obs));
            h->host_obs = nullptr;
            h->host_obs_cap = 0;
            int64_t c = n < 64 ? 64 : n;
            ISING_CHECK(cudaMallocHost(reinterpret_cast<void**>(&h->host_obs), (size_t)c * 16));
            h->host_obs_cap = c;
        }
        ISING_CHECK(cudaMemcpyAsync(h->host_obs, h->obs, (size_t)n * 16, cudaMemcpyDeviceToHost,
                                    h->stream));
        ISING_CHECK(cudaMemsetAsync(h->obs, 0, (size_t)n * 16, h->stream));
    }
    ISING_CHECK(cudaStreamSynchronize(h->stream));
    if (copy) h->n_rec = 0;  // the slots are zero again
    const int trc = check_timeout(h);
    if (trc != ISING_OK) return trc;
    if (count) *count = n;
    if (!E || !M) return ISING_OK;
    if (cap < n) return ISING_ERANGE;
    for (int64_t r = 0; r < n; ++r) {
        E[r] = h->host_obs[2 * r];
        M[r] = h->host_obs[2 * r + 1];
    }
    return ISING_OK;
}

int ising_observables_async(ising_lattice* h, int64_t* pairs, int64_t cap, int64_t* count) {
    if (!h || !count || (!pairs && h->n_rec > 0)) return ISING_EINVAL;
    const int64_t n = h->n_rec;
    *count = n;
    if (n == 0) return ISING_OK;
    if (cap < n) return ISING_ERANGE;
    ISING_CHECK(cudaMemcpyAsync(pairs, h->obs, (size_t)n * 16, cudaMemcpyDeviceToHost,
                                h->stream));
    ISING_CHECK(cudaMemsetAsync(h->obs, 0, (size_t)n * 16, h->stream));
    h->n_rec = 0;
    return ISING_OK;
}

// The device pointer of mapped pinned host memory, or nullptr if `p` is not
// device-writable host memory.
static long long* mapped_host(void* p) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (attr.type != cudaMemoryTypeHost || !attr.devicePointer) return nullptr;
    return static_cast<long long*>(attr.devicePointer);
}

int ising_observables_gather_signal(ising_lattice* const* lats, int n, int64_t* pairs,
                                    int64_t cap, int64_t* counts, int64_t* flag,
                                    int64_t value) {
    if (!lats || n < 1 || !counts) return ISING_EINVAL;
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        if (!lats[i] || lats[i]->stream != lats[0]->stream) return ISING_EINVAL;
        total += lats[i]->n_rec;
    }
    if (total > 0 && !pairs) return ISING_EINVAL;
    if (total > cap) return ISING_ERANGE;
    // the kernel writes the host buffers directly: they must be pinned (mapped)
    long long* out = nullptr;
    if (total > 0 && !(out = mapped_host(pairs))) return ISING_EINVAL;
    long long* dflag = nullptr;
    if (flag && !(dflag = mapped_host(flag))) return ISING_EINVAL;
    if (total == 0 && !dflag) {
        for (int i = 0; i < n; ++i) counts[i] = 0;
        return ISING_OK;
    }
    // every count is known before anything is queued (a handle listed twice
    // reports its records at its first entry and 0 at the others)
    for (int i = 0; i < n; ++i) {
        counts[i] = lats[i]->n_rec;
        lats[i]->n_rec = 0;  // a later entry of the same handle reads 0
    }
    for (int i = 0; i < n; ++i)
        if (counts[i] > 0) lats[i]->n_rec = counts[i];  // restored until queued
    GatherChunk chunk;
    chunk.count = 0;
    int64_t off = 0;
    int chunk_begin = 0;
    for (int i = 0; i < n; ++i) {
        ising_lattice* h = lats[i];
        if (counts[i] > 0) {
            chunk.src[chunk.count] = h->obs;
            chunk.n[chunk.count] = counts[i];
            chunk.off[chunk.count] = off;
            ++chunk.count;
            off += counts[i];
        }
        // the last launch (possibly with no records) carries the flag
        const bool last = i == n - 1;
        if (chunk.count == kGatherChunk || last) {
            if (chunk.count > 0 || (last && dflag))
                ISING_CHECK(launch_chained(gather_records_kernel, 1u, 256u, 0, lats[0]->stream,
                                           chunk, out, last ? dflag : nullptr,
                                           (long long)value));
            // queued: this chunk's records now belong to the caller's buffer
            for (int k = chunk_begin; k <= i; ++k)
                if (counts[k] > 0) lats[k]->n_rec = 0;
            chunk_begin = i + 1;
            chunk.count = 0;
        }
    }
    return ISING_OK;
}

int ising_observables_gather(ising_lattice* const* lats, int n, int64_t* pairs, int64_t cap,
                             int64_t* counts) {
    return ising_observables_gather_signal(lats, n, pairs, cap, counts, nullptr, 0);
}

// The device address of `p` if kernels can read and write it directly (device
// or managed memory, or pinned host memory mapped into the device's address
// space), else nullptr.
static void* device_reachable(const void* p) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged)
        return const_cast<void*>(p);
    if (attr.type == cudaMemoryTypeHost && attr.devicePointer) return attr.devicePointer;
    return nullptr;
}

// The handle's invalid-input flag (mapped pinned host memory), made on first use.
static int ensure_bad_flag(ising_lattice* h) {
    if (h->bad_dev) return ISING_OK;
    int* p = nullptr;
    ISING_CHECK(cudaHostAlloc(reinterpret_cast<void**>(&p), sizeof(int), cudaHostAllocMapped));
    *p = 0;
    void* d = nullptr;
    const cudaError_t e = cudaHostGetDevicePointer(&d, p, 0);
    if (e != cudaSuccess) {
        cudaFreeHost(p);
        return cuda_fail(e);
    }
    h->bad_host = p;
    h->bad_dev = static_cast<int*>(d);
    return ISING_OK;
}

int ising_export_device(ising_lattice* h, int8_t* dev_out) {
    if (!h || !dev_out) return ISING_EINVAL;
    ISING_CHECK(ising::export_spins(h, dev_out));
    return ISING_OK;
}

int ising_get_spins_async(ising_lattice* h, int8_t* out) {
    if (!h || !out) return ISING_EINVAL;
    void* d = device_reachable(out);
    if (!d) return ISING_EINVAL;
    ISING_CHECK(ising::export_spins(h, static_cast<int8_t*>(d)));
    return ISING_OK;
}

int ising_get_spins(ising_lattice* h, int8_t* host_out) {
    if (!h || !host_out) return ISING_EINVAL;
    if (void* d = device_reachable(host_out)) {
        // pinned host (or device) memory: the export kernel writes it directly
        ISING_CHECK(ising::export_spins(h, static_cast<int8_t*>(d)));
    } else {
        int8_t* tmp = nullptr;
        ISING_CHECK(ising::pool_alloc(reinterpret_cast<void**>(&tmp), (size_t)h->sites, *h->dp, h->stream));
        cudaError_t e = ising::export_spins(h, tmp);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(host_out, tmp, (size_t)h->sites, cudaMemcpyDeviceToHost,
                                h->stream);
        cudaFreeAsync(tmp, h->stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    ISING_CHECK(cudaStreamSynchronize(h->stream));
    return check_bad_input(h);
}

int ising_set_spins_async(ising_lattice* h, const int8_t* in, uint64_t t) {
    if (!h || !in) return ISING_EINVAL;
    if (t > kMaxSweep + 1) return ISING_ERANGE;
    void* d = device_reachable(in);
    if (!d) return ISING_EINVAL;
    int rc = ensure_bad_flag(h);
    if (rc != ISING_OK) return rc;
    ISING_CHECK(ising::import_spins(h, static_cast<const int8_t*>(d), h->bad_dev));
    h->t = t;
    return clear_records(h);
}

int ising_set_spins(ising_lattice* h, const int8_t* host_in, uint64_t t) {
    if (!h || !host_in) return ISING_EINVAL;
    if (t > kMaxSweep + 1) return ISING_ERANGE;
    // every value must be +1 or -1; checked in chunks without early exits inside
    // a chunk, so the compiler can vectorise the test
    for (int64_t i0 = 0; i0 < h->sites; i0 += 65536) {
        const int64_t i1 = i0 + 65536 < h->sites ? i0 + 65536 : h->sites;
        int bad = 0;
        for (int64_t i = i0; i < i1; ++i) bad |= (host_in[i] != 1) & (host_in[i] != -1);
        if (bad) return ISING_EINVAL;
    }
    if (void* d = device_reachable(host_in)) {
        // pinned host (or device) memory: the import kernel reads it directly
        ISING_CHECK(ising::import_spins(h, static_cast<const int8_t*>(d), nullptr));
    } else {
        int8_t* tmp = nullptr;
        ISING_CHECK(ising::pool_alloc(reinterpret_cast<void**>(&tmp), (size_t)h->sites, *h->dp, h->stream));
        cudaError_t e = cudaMemcpyAsync(tmp, host_in, (size_t)h->sites, cudaMemcpyHostToDevice,
                                        h->stream);
        if (e == cudaSuccess) e = ising::import_spins(h, tmp, nullptr);
        cudaFreeAsync(tmp, h->stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    h->t = t;
    int rc = clear_records(h);
    if (rc != ISING_OK) return rc;
    ISING_CHECK(cudaStreamSynchronize(h->stream));
    return ISING_OK;
}

int ising_set_stream(ising_lattice* h, void* stream) {
    if (!h) return ISING_EINVAL;
    if (h->stream != static_cast<cudaStream_t>(stream)) {
        // order the new stream after everything already issued on the old one
        ISING_CHECK(cudaStreamSynchronize(h->stream));
    }
    h->stream = static_cast<cudaStream_t>(stream);
    return ISING_OK;
}

int ising_thresholds(const ising_lattice* h, uint32_t out[3]) {
    if (!h || !out) return ISING_EINVAL;
    std::memcpy(out, h->thr, sizeof(h->thr));
    return ISING_OK;
}

int ising_compute_thresholds(int dims, double beta, uint32_t out[3]) {
    if (!out || (dims != 2 && dims != 3)) return ISING_EINVAL;
    return build_thresholds(dims, beta, out);
}

int ising_compute_thresholds_heatbath(int dims, double beta, uint32_t out[7]) {
    if (!out || (dims != 2 && dims != 3)) return ISING_EINVAL;
    return build_thresholds_heatbath(dims, beta, out);
}

int ising_set_rule(ising_lattice* h, int rule) {
    if (!h) return ISING_EINVAL;
    if (rule != ISING_RULE_METROPOLIS && rule != ISING_RULE_HEATBATH && rule != ISING_RULE_DEMON &&
        rule != ISING_RULE_MULTIHIT)
        return ISING_EINVAL;
    if (rule == ISING_RULE_DEMON && !h->dem[0]) return ISING_EINVAL;  // ising_set_demons first
    h->rule = rule;
    return ISING_OK;
}

int ising_set_hits(ising_lattice* h, int hits) {
    if (!h || hits < 1 || hits > 64) return ISING_EINVAL;
    h->hits = hits;
    return ISING_OK;
}

int ising_set_demons(ising_lattice* h, const uint8_t* host_q, int fill, int qmax) {
    if (!h) return ISING_EINVAL;
    if (qmax < 1 || qmax > 63) return ISING_EINVAL;
    const bool packed = h->layout == ISING_BITPACK;
    if (packed && qmax != 3) return ISING_EINVAL;  // two demon bit planes
    if (host_q) {
        for (int64_t i = 0; i < h->sites; ++i)
            if (host_q[i] > qmax) return ISING_EINVAL;
    } else if (fill < 0 || fill > qmax) {
        return ISING_EINVAL;
    }
    // int8: one byte per site like the spins; packed: two planes of spin words
    const size_t dem_bytes = packed ? 2 * h->col_bytes : h->col_bytes;
    for (int c = 0; c < 2; ++c) {
        if (h->dem[c]) continue;
        ISING_CHECK(ising::pool_alloc(&h->dem[c], dem_bytes, *h->dp, h->stream));
        ISING_CHECK(cudaMemsetAsync(h->dem[c], 0, dem_bytes, h->stream));
    }
    if (!host_q && packed && fill != 0) {
        // a uniform fill of the planes: bits set in every valid position
        std::vector<uint8_t> tmp((size_t)h->sites, (uint8_t)fill);
        return ising_set_demons(h, tmp.data(), 0, qmax);
    }
    if (host_q) {
        uint8_t* tmp = nullptr;
        ISING_CHECK(ising::pool_alloc(reinterpret_cast<void**>(&tmp), (size_t)h->sites, *h->dp, h->stream));
        cudaError_t e = cudaMemcpyAsync(tmp, host_q, (size_t)h->sites, cudaMemcpyHostToDevice,
                                        h->stream);
        if (e == cudaSuccess)
            e = packed ? ising::demon_packed_import(static_cast<uint32_t*>(h->dem[0]),
                                                    static_cast<uint32_t*>(h->dem[1]), tmp, h->L,
                                                    h->dims, h->rows, *h->dp, h->stream)
                       : ising::demon_import(static_cast<uint8_t*>(h->dem[0]),
                                             static_cast<uint8_t*>(h->dem[1]), tmp, h->L,
                                             h->dims, h->sites, *h->dp, h->stream);
        cudaFreeAsync(tmp, h->stream);
        if (e != cudaSuccess) return cuda_fail(e);
    } else if (packed) {
        for (int c = 0; c < 2; ++c)  // fill == 0 here
            ISING_CHECK(cudaMemsetAsync(h->dem[c], 0, dem_bytes, h->stream));
    } else {
        for (int c = 0; c < 2; ++c)
            ISING_CHECK(cudaMemsetAsync(h->dem[c], fill, (size_t)h->half_sites, h->stream));
    }
    h->qmax = qmax;
    h->dem_rot = 0;
    ISING_CHECK(cudaStreamSynchronize(h->stream));
    return ISING_OK;
}

int ising_get_demons(ising_lattice* h, uint8_t* host_out) {
    if (!h || !host_out || !h->dem[0]) return ISING_EINVAL;
    uint8_t* tmp = nullptr;
    ISING_CHECK(ising::pool_alloc(reinterpret_cast<void**>(&tmp), (size_t)h->sites, *h->dp, h->stream));
    cudaError_t e =
        h->layout == ISING_BITPACK
            ? ising::demon_packed_export(static_cast<const uint32_t*>(h->dem[0]),
                                         static_cast<const uint32_t*>(h->dem[1]), tmp, h->L,
                                         h->dims, h->sites, h->rows, h->dem_rot, *h->dp,
                                         h->stream)
            : ising::demon_export(static_cast<const uint8_t*>(h->dem[0]),
                                  static_cast<const uint8_t*>(h->dem[1]), tmp, h->L, h->dims,
                                  h->sites, h->rows, h->dem_rot, *h->dp, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_out, tmp, (size_t)h->sites, cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(tmp, h->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    ISING_CHECK(cudaStreamSynchronize(h->stream));
    return ISING_OK;
}

int ising_get_info(const ising_lattice* h, ising_info_t* out) {
    if (!h || !out) return ISING_EINVAL;
    std::memset(out, 0, sizeof(*out));
    out->dims = h->dims;
    out->L = h->L;
    out->layout = h->layout;
    out->rule = h->rule;
    out->beta = h->beta;
    out->seed = h->seed;
    out->sweeps_done = h->t;
    out->sites = (uint64_t)h->sites;
    out->device_bytes = (uint64_t)(
        (h->dem[0] ? (h->layout == ISING_BITPACK ? 6 : 4) : 2) * h->col_bytes);
    out->pending_records = h->n_rec;
    return ISING_OK;
}

int ising_synchronize(ising_lattice* h) {
    if (!h) return ISING_EINVAL;
    ISING_CHECK(cudaStreamSynchronize(h->stream));
    return check_timeout(h);
}

int ising_set_kernel(ising_lattice* h, int kernel) {
    if (!h) return ISING_EINVAL;
    if (kernel != ISING_KERNEL_AUTO && kernel != ISING_KERNEL_STRIP && kernel != ISING_KERNEL_TMA)
        return ISING_EINVAL;
    h->kernel = kernel;
    return ISING_OK;
}

int ising_get_kernel(const ising_lattice* h, int* kernel) {
    if (!h || !kernel) return ISING_EINVAL;
    *kernel = h->layout == ISING_BITPACK ? -1
                                         : (uses_tma(h) ? ISING_KERNEL_TMA : ISING_KERNEL_STRIP);
    return ISING_OK;
}

int ising_set_int8_config(int dims, int L_min, int L_max, const ising_int8_config* cfg) {
    if (!cfg || (dims != 2 && dims != 3) || L_min < 2 || L_max < L_min) return ISING_EINVAL;
    if (cfg->kernel != ISING_KERNEL_STRIP && cfg->kernel != ISING_KERNEL_TMA) return ISING_EINVAL;
    const int R = cfg->tile_rows;
    if (R < 0 || R > 64 || (R & (R - 1)) != 0) return ISING_EINVAL;  // 0 or a power of two <= 64
    if (cfg->ctas_per_sm < 0 || cfg->ctas_per_sm > 8) return ISING_EINVAL;
    std::lock_guard<std::mutex> lk(g_policy_mu);
    g_policy.push_back(Int8Policy{dims, L_min, L_max, *cfg});
    return ISING_OK;
}

int ising_clear_int8_configs(void) {
    std::lock_guard<std::mutex> lk(g_policy_mu);
    g_policy.clear();
    return ISING_OK;
}

int ising_get_int8_config(const ising_lattice* h, ising_int8_config* out) {
    if (!h || !out) return ISING_EINVAL;
    if (h->layout == ISING_BITPACK) {
        *out = ising_int8_config{-1, 0, 0};
        return ISING_OK;
    }
    *out = resolve_int8(h);
    return ISING_OK;
}

int ising_philox_fill(uint32_t* dev_out, uint32_t n, uint32_t c1, uint32_t c2, uint32_t c3,
                      uint64_t seed, void* stream) {
    if (!dev_out && n > 0) return ISING_EINVAL;
    if (n == 0) return ISING_OK;
    const DeviceProps* dp = nullptr;
    const int rc = device_props(&dp);
    if (rc != ISING_OK) return rc;
    ISING_CHECK(ising::philox_fill(dev_out, n, c1, c2, c3, (uint32_t)(seed & 0xFFFFFFFFu),
                                   (uint32_t)(seed >> 32), *dp, static_cast<cudaStream_t>(stream)));
    return ISING_OK;
}

int ising_philox_probe(uint32_t* dev_out, int blocks, int threads, uint32_t iters, int variant,
                       int chains, uint64_t seed, void* stream) {
    if (!dev_out || blocks < 1 || (threads != 128 && threads != 256) || iters < 1 ||
        (variant != 0 && variant != 1) || (chains != 4 && chains != 8))
        return ISING_EINVAL;
    // every counter word 0 must be distinct: gid * iters * chains + k < 2^32
    if ((uint64_t)blocks * (uint64_t)threads * iters * (uint64_t)chains > 0xFFFFFFFFull)
        return ISING_ERANGE;
    ISING_CHECK(ising::philox_probe(dev_out, blocks, threads, iters, variant, chains, 5u,
                                    (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32),
                                    static_cast<cudaStream_t>(stream)));
    return ISING_OK;
}

int ising_test_inject_timeout(int on) {
    g_inject_timeout.store(on ? 1 : 0);
    return ISING_OK;
}

void ising_destroy(ising_lattice* h) {
    if (!h) return;
    // pinned host buffers that queued work may still touch are freed only
    // after that work; device memory returns to the pool in stream order
    if (h->host_obs || h->bad_host) cudaStreamSynchronize(h->stream);
    free_device(h);
    delete h;
}

int ising_release_cached_memory(void) {
    const DeviceProps* dp = nullptr;
    const int rc = device_props(&dp);
    if (rc != ISING_OK) return rc;
    ISING_CHECK(cudaDeviceSynchronize());
    ISING_CHECK(cudaMemPoolTrimTo(dp->pool, 0));
    return ISING_OK;
}

}  // extern "C"
