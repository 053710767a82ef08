// Measurement of the device's 64-bit L2 reduction rate: the secondary bound
// of the transport's scoring, which adds every condensed-history step's
// fixed-point deposit to a voxel with one 64-bit atomic add (a reduction
// resolved in L2).
//
// The kernel adds 1 to pseudo-random entries of a buffer small enough to
// stay in L2, with the result unused (a fire-and-forget reduction, as in the
// scoring).  Entries follow a multiplicative hash of (thread, iteration), so
// a warp's 32 adds hit 32 different lines, as the lanes of a transport warp
// carry unrelated histories.  The rate is adds per second between two CUDA
// events; the buffer's sum afterwards must equal the number of adds.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/vpmc.h"
#include "context.h"

namespace vpmc {
namespace {

__global__ void k_l2_red(unsigned long long* __restrict__ buf, unsigned long long mask, int iters)
{
    const unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    unsigned long long h = (t + 1ull) * 0x9E3779B97F4A7C15ull;
    for (int i = 0; i < iters; ++i) {
        h = h * 6364136223846793005ull + 1442695040888963407ull;    // 64-bit LCG (Knuth)
        atomicAdd(buf + ((h >> 17) & mask), 1ull);
    }
}

__global__ void k_sum(const unsigned long long* __restrict__ buf, long long n, unsigned long long* out)
{
    unsigned long long s = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += buf[i];
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

}  // namespace
}  // namespace vpmc

extern "C" vpmc_status vpmc_measure_l2_atomics(int64_t n_entries, int iters, double* adds_per_s, int64_t* adds_out,
                                               int64_t* sum_out, void* stream)
{
    using namespace vpmc;
    clear_error();
    (void)cudaGetLastError();
    if (n_entries < 32 || (n_entries & (n_entries - 1)) || n_entries > (1ll << 26) || iters < 1 || iters > 4096 ||
        !adds_per_s)
        return report_error(VPMC_ERR_ARG, "n_entries must be a power of two in [32, 2^26], iters in [1, 4096]");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return report_error(VPMC_ERR_CUDA, "no CUDA device");
    unsigned long long* buf = nullptr;
    unsigned long long* sum = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    vpmc_status st = VPMC_OK;
    const int block = 1024, grid = 4 * sms;
    const long long adds = (long long)grid * block * iters;
    float ms = 0.0f;
    unsigned long long h_sum = 0;
    do {
        if (cudaMalloc(&buf, n_entries * sizeof(unsigned long long)) != cudaSuccess ||
            cudaMalloc(&sum, sizeof(unsigned long long)) != cudaSuccess) {
            st = report_error(VPMC_ERR_OOM, "buffer allocation failed");
            break;
        }
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
            cudaMemsetAsync(buf, 0, n_entries * sizeof(unsigned long long), s) != cudaSuccess ||
            cudaMemsetAsync(sum, 0, sizeof(unsigned long long), s) != cudaSuccess) {
            st = report_error(VPMC_ERR_CUDA, "set-up failed");
            break;
        }
        // one untimed pass brings the buffer into L2, then the timed one
        k_l2_red<<<grid, block, 0, s>>>(buf, (unsigned long long)(n_entries - 1), iters);
        cudaEventRecord(e0, s);
        k_l2_red<<<grid, block, 0, s>>>(buf, (unsigned long long)(n_entries - 1), iters);
        cudaEventRecord(e1, s);
        k_sum<<<sms, 256, 0, s>>>(buf, n_entries, sum);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            cudaMemcpyAsync(&h_sum, sum, sizeof h_sum, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = report_error(VPMC_ERR_CUDA, "measurement launch failed");
            break;
        }
    } while (false);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(sum);
    if (st != VPMC_OK) return st;
    *adds_per_s = (double)adds / (ms * 1e-3);
    if (adds_out) *adds_out = adds;
    if (sum_out) *sum_out = (int64_t)h_sum;
    return VPMC_OK;
}
