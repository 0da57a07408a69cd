// engine_internal.h -- declarations shared between the host engine and the
// kernel translation units (not part of the public C ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ising {

struct PassArgs;

struct DeviceProps {
    int device = -1;
    int sm_count = 0;
    int blocks_per_sm_vec[2][2] = {{1, 1}, {1, 1}};    // int8 vector pass [dims-2][measure]
    int blocks_per_sm_packed[2][2] = {{1, 1}, {1, 1}}; // bit-packed pass [dims-2][measure]
};

// int8 layout (sweep_int8.cu)
cudaError_t int8_query_occupancy(DeviceProps& dp);
bool int8_vec_ok(int L);
cudaError_t int8_pass(const PassArgs& a, int dims, int64_t half_sites, bool measure,
                      const DeviceProps& dp, cudaStream_t st);
cudaError_t int8_init(int8_t* col0, int8_t* col1, int L, int dims, int64_t sites, int start,
                      uint32_t key0, uint32_t key1, const DeviceProps& dp, cudaStream_t st);
cudaError_t int8_export(const int8_t* col0, const int8_t* col1, int8_t* out, int L, int dims,
                        int64_t sites, const DeviceProps& dp, cudaStream_t st);
cudaError_t int8_import(int8_t* col0, int8_t* col1, const int8_t* in, int L, int dims,
                        int64_t sites, const DeviceProps& dp, cudaStream_t st);

// bit-packed layout (sweep_bitpack.cu)
cudaError_t packed_query_occupancy(DeviceProps& dp);
cudaError_t packed_pass(const PassArgs& a, int dims, bool measure, const DeviceProps& dp,
                        cudaStream_t st);
cudaError_t packed_init(uint32_t* col0, uint32_t* col1, int L, int dims, int64_t rows, int start,
                        uint32_t key0, uint32_t key1, const DeviceProps& dp, cudaStream_t st);
cudaError_t packed_export(const uint32_t* col0, const uint32_t* col1, int8_t* out, int L,
                          int dims, int64_t sites, const DeviceProps& dp, cudaStream_t st);
cudaError_t packed_import(uint32_t* col0, uint32_t* col1, const int8_t* in, int L, int dims,
                          int64_t rows, const DeviceProps& dp, cudaStream_t st);

}  // namespace ising
