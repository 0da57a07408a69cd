// engine_internal.h -- declarations shared between the host engine and the
// kernel translation units (not part of the public C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "ising.h"

namespace ising {

struct PassArgs;
struct DeviceProps;

}  // namespace ising

// A lattice handle (the opaque type of the C ABI).
struct ising_lattice {
    int dims = 0, L = 0, layout = ISING_INT8;
    double beta = 0.0;
    uint64_t seed = 0;
    uint32_t thr[3] = {0, 0, 0};        // Metropolis: floor(exp(-2 beta k) 2^32), k = 2, 4, 6
    uint32_t thb[7] = {0, 0, 0, 0, 0, 0, 0}; // heat bath: floor(2^32 / (1 + exp(4 beta (dims - d))))
    int rule = ISING_RULE_METROPOLIS;
    int64_t sites = 0, half_sites = 0, rows = 0;
    int W = 0;
    void* col[2] = {nullptr, nullptr};  // colour 0 (black) and colour 1 (white) arrays
    size_t col_bytes = 0;
    uint64_t t = 0;                     // index of the next sweep
    cudaStream_t stream = nullptr;
    unsigned long long* obs = nullptr;  // (E, M) int64 pairs; slots >= n_rec are zero
    int64_t obs_cap = 0, n_rec = 0;
    const ising::DeviceProps* dp = nullptr;
    int kernel = ISING_KERNEL_AUTO;     // int8 pass kernel choice
    void* dem[2] = {nullptr, nullptr};  // demons per colour (int8 layout), or null
    int qmax = 0;                       // demon capacity: q = 0..qmax
    int64_t dem_rot = 0;                // half rows the demons have moved on, mod rows
    int hits = 2;                       // multi-hit Metropolis: trials per visit
    long long* host_obs = nullptr;      // pinned staging for ising_observables
    int64_t host_obs_cap = 0;           // in records
    // raised by an import kernel of ising_set_spins_async that met a value
    // other than +-1 (mapped pinned int: device view, host view)
    int* bad_dev = nullptr;
    volatile int* bad_host = nullptr;
};

namespace ising {

struct DeviceProps {
    int device = -1;
    int sm_count = 0;
    // resident CTAs per SM of the int8 strip pass and the bit-packed pass
    int blocks_per_sm_vec[4][2][2] = {};     // [rule][dims - 2][measure]; rule 2 unused
    int blocks_per_sm_packed[4][2][2][2] = {};  // ... [full words, power-of-two counts]
    int blocks_per_sm_demon[2][2] = {{1, 1}, {1, 1}};  // demon strip pass [dims-2][measure]
    // raised by a kernel whose bounded wait ran out: one int of mapped pinned
    // host memory (device view d_err, host view h_err), read without a copy
    int* d_err = nullptr;
    volatile int* h_err = nullptr;
    // the library's stream-ordered pool for lattice memory (spin, demon and
    // record buffers): freed blocks stay reserved for the next lattice, so
    // creating and destroying lattices never synchronises the device
    cudaMemPool_t pool = nullptr;
};

// Launch `kernel` on `st` with programmatic stream serialisation: it may be
// scheduled before the previous kernel of the stream completes, and must call
// grid_dependency_wait() (ising_device.cuh) before touching global memory.
template <typename... KArgs, typename... Args>
cudaError_t launch_chained(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                           cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// engine.cu helpers shared with batch.cu
int cuda_fail(cudaError_t e);
// the test hook of ising_test_inject_timeout is on
bool injecting_timeout();
// the threshold table of the lattice's rule, as the kernels take it (PassArgs::thr)
void rule_thresholds(const ising_lattice* h, uint32_t out[7]);
int device_props(const DeviceProps** out);
// stream-ordered allocation from the device's lattice pool
cudaError_t pool_alloc(void** p, size_t bytes, const DeviceProps& dp, cudaStream_t st);
int ensure_records(ising_lattice* h, int64_t need);
// n sweeps of a small lattice in one persistent single-CTA launch (batch.cu)
int small_sweep(ising_lattice* h, int64_t n, int every, unsigned long long* slots);
constexpr int64_t kSmallSites = 16384;  // at or below: the single-launch path
constexpr uint64_t kMaxSweep = 0xFFFFFFFFull;  // the sweep index is a 32-bit counter word

// int8 layout (sweep_int8.cu)
cudaError_t int8_query_occupancy(DeviceProps& dp);
bool int8_vec_ok(int L);
cudaError_t philox_fill(uint32_t* out, uint32_t n, uint32_t c1, uint32_t c2, uint32_t c3,
                        uint32_t key0, uint32_t key1, const DeviceProps& dp, cudaStream_t st);
cudaError_t philox_probe(uint32_t* out, int blocks, int threads, uint32_t iters, int variant,
                         int chains, uint32_t c1, uint32_t key0, uint32_t key1, cudaStream_t st);
cudaError_t int8_pass(const PassArgs& a, int dims, int64_t half_sites, bool measure, int rule,
                      const DeviceProps& dp, cudaStream_t st);
cudaError_t int8_init(int8_t* col0, int8_t* col1, int L, int dims, int64_t sites, int start,
                      uint32_t key0, uint32_t key1, const DeviceProps& dp, cudaStream_t st);
cudaError_t int8_export(const int8_t* col0, const int8_t* col1, int8_t* out, int L, int dims,
                        int64_t sites, const DeviceProps& dp, cudaStream_t st);
cudaError_t int8_import(int8_t* col0, int8_t* col1, const int8_t* in, int L, int dims,
                        int64_t sites, const DeviceProps& dp, cudaStream_t st);

// int8 layout, inputs staged by bulk copies (sweep_int8_tma.cu)
bool int8_tma_ok(int dims, int L, int rows_per_tile);
// ISING_KERNEL_AUTO's choice of the staged kernel without a tuned
// configuration (measured; see the definition)
bool int8_tma_preferred(int dims, int L);
cudaError_t int8_pass_tma(const PassArgs& a, int dims, bool measure, int rule,
                          const DeviceProps& dp, int* err, uint32_t extra_tx, cudaStream_t st,
                          int rows_per_tile, int ctas_per_sm);

// canonical <-> layout conversion and initial states for half rows of whole
// 16-byte vectors (int8, L % 32 == 0) or whole words (bit-packed, L % 64 == 0)
// (convert.cu)
bool rows_ok(int layout, int L);
cudaError_t rows_init(void* col0, void* col1, size_t col_data_bytes, int layout, int L,
                      int64_t rows, int start, uint32_t key0, uint32_t key1,
                      const DeviceProps& dp, cudaStream_t st);
cudaError_t rows_import(void* col0, void* col1, const int8_t* in, int layout, int L, int64_t rows,
                        int* bad_flag, const DeviceProps& dp, cudaStream_t st);
cudaError_t rows_export(const void* col0, const void* col1, int8_t* out, int layout, int L,
                        int64_t rows, const DeviceProps& dp, cudaStream_t st);
cudaError_t check_spins(const int8_t* in, int64_t n, int* bad_flag, const DeviceProps& dp,
                        cudaStream_t st);

// demon dynamics, int8 layout (sweep_demon.cu)
cudaError_t demon_query_occupancy(DeviceProps& dp);
cudaError_t demon_pass(const PassArgs& a, int dims, int64_t half_sites, bool measure,
                       const DeviceProps& dp, cudaStream_t st);
cudaError_t demon_export(const uint8_t* d0, const uint8_t* d1, uint8_t* out, int L, int dims,
                         int64_t sites, int64_t rows, int64_t rot, const DeviceProps& dp,
                         cudaStream_t st);
cudaError_t demon_import(uint8_t* d0, uint8_t* d1, const uint8_t* in, int L, int dims,
                         int64_t sites, const DeviceProps& dp, cudaStream_t st);
// bit-packed layout, qmax = 3: two demon planes per colour (plane 1 after plane 0)
cudaError_t demon_packed_pass(const PassArgs& a, int dims, bool measure, const DeviceProps& dp,
                              cudaStream_t st);
cudaError_t demon_packed_import(uint32_t* d0, uint32_t* d1, const uint8_t* in, int L, int dims,
                                int64_t rows, const DeviceProps& dp, cudaStream_t st);
cudaError_t demon_packed_export(const uint32_t* d0, const uint32_t* d1, uint8_t* out, int L,
                                int dims, int64_t sites, int64_t rows, int64_t rot,
                                const DeviceProps& dp, cudaStream_t st);

// bit-packed layout (sweep_bitpack.cu)
cudaError_t packed_query_occupancy(DeviceProps& dp);
cudaError_t packed_pass(const PassArgs& a, int dims, bool measure, int rule,
                        const DeviceProps& dp, cudaStream_t st);
cudaError_t packed_init(uint32_t* col0, uint32_t* col1, int L, int dims, int64_t rows, int start,
                        uint32_t key0, uint32_t key1, const DeviceProps& dp, cudaStream_t st);
cudaError_t packed_export(const uint32_t* col0, const uint32_t* col1, int8_t* out, int L,
                          int dims, int64_t sites, const DeviceProps& dp, cudaStream_t st);
cudaError_t packed_import(uint32_t* col0, uint32_t* col1, const int8_t* in, int L, int dims,
                          int64_t rows, const DeviceProps& dp, cudaStream_t st);

}  // namespace ising
