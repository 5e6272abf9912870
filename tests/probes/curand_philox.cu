// Test probe (not part of the library): the Philox4x32-10 words of CUDA's
// curand device API for given counters and keys, so that the oracle's own
// implementation of the generator can be checked against an independent one.
#include <cstdint>
#include <curand_kernel.h>

namespace {

__global__ void k_curand_philox(const uint4 *__restrict__ ctr, const uint2 *__restrict__ key, uint4 *__restrict__ out,
                                int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

}  // namespace

// ctr: device uint32[4 n], key: device uint32[2 n], out: device uint32[4 n];
// returns the launch's cudaError_t.
extern "C" int curand_philox_words(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int n, void *stream)
{
    if (n <= 0)
        return 0;
    k_curand_philox<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const uint4 *>(ctr), reinterpret_cast<const uint2 *>(key), reinterpret_cast<uint4 *>(out), n);
    return (int)cudaGetLastError();
}
