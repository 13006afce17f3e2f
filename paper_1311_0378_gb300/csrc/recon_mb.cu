// GB300 versions of the paper's two device micro-benchmarks, which explain the
// irregular operations' performance (Sec. V-C):
//   Table III -- bandwidth of random 32-bit reads / writes in a 4K x 4K matrix
//                of integers (10 million operations);
//   Table IV  -- throughput of atomic adds, (1) every thread on one variable,
//                (2) every thread on its own array element.
// Both are added here in the two memories the wavefront phase actually uses:
// global memory (HBM / L2) and shared memory (the per-block J the wavefront
// updates with compare-and-swap).
//
// Random indices: SplitMix64 (Steele, Lea & Flood 2014; the constants of its
// published reference implementation) evaluated at counter k, top log2(n) bits.
// Written values depend only on the index, so colliding writes are benign.
#include <climits>
#include <cuda_runtime.h>
#include <stdint.h>

#include "recon.h"

namespace mb {

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint32_t written_value(uint64_t idx) { return (uint32_t)(idx * 0x9E3779B1ull) ^ 0x5A5A5A5Au; }

constexpr int UNROLL = 4;

// op k (k = 0 .. ops-1) touches M[splitmix64_at(seed, k + 1) >> (64 - log2n)].
// read: the sum of the values read (mod 2^64) goes to *sum.
__global__ void __launch_bounds__(256) random_access(uint32_t *M, int log2n, unsigned long long ops, int write,
                                                     uint64_t seed, unsigned long long *sum)
{
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned long long acc = 0;
    const int sh = 64 - log2n;
    for (unsigned long long k0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k0 < ops;
         k0 += stride * UNROLL) {
        uint64_t idx[UNROLL];
        bool ok[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const unsigned long long k = k0 + (unsigned long long)u * stride;
            ok[u] = k < ops;
            idx[u] = splitmix64_at(seed, k + 1) >> sh;
        }
        if (write) {
#pragma unroll
            for (int u = 0; u < UNROLL; ++u)
                if (ok[u]) M[idx[u]] = written_value(idx[u]);
        } else {
            uint32_t v[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) v[u] = ok[u] ? __ldcg(M + idx[u]) : 0u;   // all issued, then used
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) acc += v[u];
        }
    }
    if (!write) {
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if ((threadIdx.x & 31) == 0 && acc) atomicAdd(sum, acc);
    }
}

// mode 0: every thread adds 1 to C[0] `iters` times (global);
// mode 1: thread t adds 1 to C[t] (global);
// mode 2: every thread of a CTA adds 1 to one shared word, written to C[cta] at the end;
// mode 3: every thread adds 1 to its own shared word, written to C[t] at the end.
__global__ void __launch_bounds__(256) atomic_add(unsigned *C, int mode, int iters)
{
    __shared__ unsigned sw[256];
    const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
    sw[threadIdx.x] = 0;
    __syncthreads();
    if (mode == 0) {
        for (int i = 0; i < iters; ++i) atomicAdd(&C[0], 1u);
    } else if (mode == 1) {
        for (int i = 0; i < iters; ++i) atomicAdd(&C[t], 1u);
    } else if (mode == 2) {
        for (int i = 0; i < iters; ++i) atomicAdd(&sw[0], 1u);
    } else {
        for (int i = 0; i < iters; ++i) atomicAdd(&sw[threadIdx.x], 1u);
    }
    __syncthreads();
    if (mode == 2 && threadIdx.x == 0) C[blockIdx.x] = sw[0];
    if (mode == 3) C[t] = sw[threadIdx.x];
}

}  // namespace mb

namespace {
constexpr int MB_THREADS = 256;

int mb_grid(int dev)
{
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 0;
    return sms * 8;   // 8 resident CTAs of 256 threads per SM
}
}  // namespace

extern "C" int recon_mb_threads(int device)
{
    const int g = mb_grid(device);
    return g > 0 ? g * MB_THREADS : -RECON_ECUDA;
}

extern "C" int recon_mb_random(const void *matrix, int log2n, uint64_t ops, int write, uint64_t seed,
                               uint64_t *checksum, float *ms)
{
    if (!matrix || log2n < 1 || log2n > 34 || ops < 1 || (write != 0 && write != 1) || !ms) return RECON_EINVAL;
    if (!write && !checksum) return RECON_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RECON_ECUDA;
    const int grid = mb_grid(dev);
    if (!grid) return RECON_ECUDA;
    unsigned long long *dsum = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = RECON_OK;
    if (cudaMalloc(&dsum, sizeof(*dsum)) != cudaSuccess) return RECON_ENOMEM;
    if (cudaMemset(dsum, 0, sizeof(*dsum)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) rc = RECON_ECUDA;
    if (rc == RECON_OK) {
        cudaEventRecord(e0);
        mb::random_access<<<grid, MB_THREADS>>>((uint32_t *)matrix, log2n, ops, write, seed, dsum);
        cudaEventRecord(e1);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) rc = RECON_ECUDA;
    }
    if (rc == RECON_OK && !write) {
        unsigned long long h = 0;
        if (cudaMemcpy(&h, dsum, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) rc = RECON_ECUDA;
        else *checksum = h;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(dsum);
    return rc;
}

extern "C" int recon_mb_atomic(unsigned *counters, int mode, int iters, float *ms)
{
    if (!counters || mode < 0 || mode > 3 || iters < 1 || !ms) return RECON_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RECON_ECUDA;
    const int grid = mb_grid(dev);
    if (!grid) return RECON_ECUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = RECON_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = RECON_ECUDA;
    if (rc == RECON_OK) {
        cudaEventRecord(e0);
        mb::atomic_add<<<grid, MB_THREADS>>>(counters, mode, iters);
        cudaEventRecord(e1);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) rc = RECON_ECUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}
