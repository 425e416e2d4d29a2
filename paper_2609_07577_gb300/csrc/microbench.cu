// On-chip ceiling of the neighbour histogram (snnmap_hist_ceiling in
// include/snnmap.h): the block tier's shared-memory table insert (hash
// probe, key claim, integer adds of score and shared count) run on keys
// made in registers, with the block tier's table size, block size and
// blocks per SM, so no global memory is touched while timing. Its rate is
// the most element updates per second the histogram stages could reach.
#include "histo.cuh"
#include "internal.cuh"

namespace snn {

__global__ void __launch_bounds__(HT_BTHREADS)
    k_hist_ceiling(int32_t keys, int32_t rounds, uint32_t seed, unsigned long long* sink)
{
    extern __shared__ __align__(16) unsigned char ht_dyn[];
    Table<uint32_t> t = carve_table<uint32_t>(ht_dyn, HT_BCAP);
    clear_slots(t, threadIdx.x, HT_BCAP, HT_BTHREADS);
    __syncthreads();
    uint32_t x = hash32(seed ^ (blockIdx.x * HT_BTHREADS + threadIdx.x));
    unsigned long long acc = 0;
    for (int32_t r = 0; r < rounds; r++) {
        // one vertex's worth of updates: 32 elements per thread into a table
        // of `keys` distinct neighbours, then the scan that reads and resets it
#pragma unroll 4
        for (int e = 0; e < 32; e++) {
            x = x * 1664525u + 1013904223u;
            int32_t m = (int32_t)((x >> 8) % (uint32_t)keys);
            if (!t.add(m, 1u + (x & 7u), (x >> 3) & 1u)) acc++;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < HT_BCAP; i += HT_BTHREADS) {
            if (t.key[i] >= 0) acc += t.sc[i] + t.ov[i];
            t.key[i] = -1;
            t.sc[i] = 0;
            t.ov[i] = 0;
        }
        __syncthreads();
    }
    if (acc == 0x7fffffffffffffffull) atomicAdd(sink, acc);   // keeps the work live
}

}  // namespace snn

extern "C" int snnmap_hist_ceiling(int32_t distinct_keys, int32_t rounds, void* stream,
                                   double* updates_per_s)
{
    using namespace snn;
    if (!updates_per_s || distinct_keys < 1 || distinct_keys > HT_BCAP * 3 / 4 || rounds < 1) {
        set_last_error("updates_per_s must be set, 1 <= distinct_keys <= 1536, rounds >= 1");
        return SNNMAP_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    size_t smem = (size_t)HT_BCAP * slot_bytes<uint32_t>();
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hist_ceiling, HT_BTHREADS, smem);
    int grid = sms * (per_sm > 0 ? per_sm : 1);
    unsigned long long* sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMallocAsync(&sink, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float ms = 0;
    if (e == cudaSuccess) {
        note_launch();
        k_hist_ceiling<<<grid, HT_BTHREADS, smem, s>>>(distinct_keys, rounds, 1u, sink);   // warm-up
        cudaEventRecord(a, s);
        note_launch();
        k_hist_ceiling<<<grid, HT_BTHREADS, smem, s>>>(distinct_keys, rounds, 2u, sink);
        cudaEventRecord(b, s);
        e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (sink) cudaFreeAsync(sink, s);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return SNNMAP_ERR_CUDA;
    }
    double updates = (double)grid * HT_BTHREADS * 32.0 * rounds;
    *updates_per_s = ms > 0 ? updates / (ms / 1e3) : 0.0;
    set_last_error("");
    return SNNMAP_OK;
}
