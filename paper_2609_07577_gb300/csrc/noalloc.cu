// Connectivity of a partition for callers that cannot allocate device memory
// (snnmap_connectivity_noalloc in include/snnmap.h).
//
// The scratch this computation needs (one distinct-partition count per
// hyperedge, an error word and a 64-bit accumulator) lives in a file-scope
// device array instead of memory from cudaMalloc or the handle's arena. The
// array exists once per device that loads the library and stays allocated
// until the process exits. Host code may not use its name as an address; the
// device address is looked up once per device with cudaGetSymbolAddress
// (the first call on a device does that, with that device current).
//
// Every call shares the array, and it keeps the previous call's contents:
// each call clears the accumulator and the error word before its kernels
// run. Two calls whose work overlaps on the GPU (different streams, or
// different host threads on one device) race on the array and may return
// wrong results; callers must order them.
#include "internal.cuh"

#include <mutex>

namespace {

constexpr int64_t kMaxHedges = (int64_t)1 << 22;   // 4,194,304 hyperedges (16 MiB of counts)
constexpr size_t kHeader = 256;                     // accumulator and error word
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kHeader + kMaxHedges * sizeof(int32_t)];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// device address of the scratch array on the current device
cudaError_t scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

bool device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// every neuron's partition id must lie in [0, n_parts)
__global__ void k_na_check_rho(int32_t V, const int32_t* __restrict__ rho, int32_t K, int32_t* err)
{
    int bad = 0;
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < V;
         n += (int64_t)gridDim.x * blockDim.x)
        if (rho[n] < 0 || rho[n] >= K) bad = 1;
    if (__any_sync(snn::FULL, bad) && (threadIdx.x & 31) == 0) atomicOr(err, 1);
}

// lambda(e): pins whose partition differs from every earlier pin's in the
// same hyperedge, counted by one warp per hyperedge (quadratic in |e|,
// 32 comparisons per shuffle round)
__global__ void k_na_lambda(const int64_t* __restrict__ off, const int32_t* __restrict__ pins,
                            int32_t E, int32_t V, const int32_t* __restrict__ rho, int32_t* lam,
                            int32_t* err)
{
    int lane = threadIdx.x & 31;
    int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (gw == 0 && lane == 0 && off[0] != 0) atomicOr(err, 1);
    for (int64_t a = gw; a < E; a += nw) {
        int64_t b = off[a], e = off[a + 1];
        if (e <= b) {
            if (lane == 0) atomicOr(err, 1);
            if (lane == 0) lam[a] = 1;
            continue;
        }
        int count = 0, bad = 0;
        for (int64_t cj = b; cj < e; cj += 32) {
            int64_t j = cj + lane;
            int32_t pj = -1;
            if (j < e) {
                int32_t q = pins[j];
                if (q < 0 || q >= V) bad = 1;
                else pj = rho[q];
            }
            bool first = pj >= 0;
            for (int64_t ci = b; ci <= cj; ci += 32) {
                int64_t i = ci + lane;
                int32_t pi = -1;
                if (i < e) {
                    int32_t q = pins[i];
                    if (q >= 0 && q < V) pi = rho[q];
                }
                for (int t = 0; t < 32; t++) {
                    int32_t o = __shfl_sync(snn::FULL, pi, t);
                    if (ci + t < j && o >= 0 && o == pj) first = false;
                }
            }
            count += __popc(__ballot_sync(snn::FULL, first));
        }
        if (__any_sync(snn::FULL, bad) && lane == 0) atomicOr(err, 1);
        if (lane == 0) lam[a] = count;
    }
}

__global__ void k_na_reduce(const int32_t* __restrict__ w, const int32_t* __restrict__ lam,
                            int32_t E, unsigned long long* acc, int32_t* err)
{
    int64_t s = 0;
    int bad = 0;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < E;
         a += (int64_t)gridDim.x * blockDim.x) {
        if (w[a] < 0) bad = 1;
        if (lam[a] > 1) s += (int64_t)w[a] * (lam[a] - 1);
    }
    s = snn::warp_sum(s);
    if ((threadIdx.x & 31) == 0) {
        if (s) atomicAdd(acc, (unsigned long long)s);
    }
    if (__any_sync(snn::FULL, bad) && (threadIdx.x & 31) == 0) atomicOr(err, 1);
}

__global__ void k_na_store(const unsigned long long* acc, int64_t* out) { *out = (int64_t)*acc; }

}  // namespace

extern "C" {

int snnmap_connectivity_noalloc(int32_t n_vertices, int32_t n_hedges, const int64_t* d_offsets,
                                const int32_t* d_pins, const int32_t* d_w, const int32_t* d_rho,
                                int32_t n_parts, int64_t* d_cost_out, void* stream)
{
    if (n_vertices < 0 || n_hedges < 0 || n_parts < 1) {
        snn::set_last_error("negative sizes or n_parts < 1");
        return SNNMAP_ERR_INVALID;
    }
    if (n_hedges > kMaxHedges) {
        snn::set_last_error("n_hedges exceeds 4194304, the capacity of the allocation-free scratch array");
        return SNNMAP_ERR_INVALID;
    }
    if (!device_ptr(d_offsets) || !device_ptr(d_cost_out) ||
        (n_vertices > 0 && !device_ptr(d_rho)) ||
        (n_hedges > 0 && (!device_ptr(d_pins) || !device_ptr(d_w)))) {
        snn::set_last_error("buffers must be device memory");
        return SNNMAP_ERR_INVALID;
    }
    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        snn::set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return SNNMAP_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* acc = (unsigned long long*)base;
    int32_t* err = (int32_t*)((char*)base + 8);
    int32_t* lam = (int32_t*)((char*)base + kHeader);
    e = cudaMemsetAsync(base, 0, kHeader, s);
    if (e == cudaSuccess && n_vertices > 0) {
        SNN_L k_na_check_rho<<<snn::grid_for(n_vertices, 256), 256, 0, s>>>(n_vertices, d_rho,
                                                                             n_parts, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && n_hedges > 0) {
        SNN_L k_na_lambda<<<snn::grid_for((int64_t)n_hedges * 32, 256), 256, 0, s>>>(
            d_offsets, d_pins, n_hedges, n_vertices, d_rho, lam, err);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            SNN_L k_na_reduce<<<snn::grid_for(n_hedges, 256), 256, 0, s>>>(d_w, lam, n_hedges, acc,
                                                                         err);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        SNN_L k_na_store<<<1, 1, 0, s>>>(acc, d_cost_out);
        e = cudaGetLastError();
    }
    int32_t herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        snn::set_last_error(cudaGetErrorString(e));
        return SNNMAP_ERR_CUDA;
    }
    if (herr) {
        snn::set_last_error("invalid input: offsets, pin id, weight or partition id out of range");
        return SNNMAP_ERR_INVALID;
    }
    snn::set_last_error("");
    return SNNMAP_OK;
}

}  // extern "C"
