// Test helper (not part of the library): cuRAND's device-side
// Philox4x32-10 (NVIDIA's implementation of Salmon et al. 2011) applied to
// given counters under one key, for a known-answer comparison with the
// library's generator on arbitrary counters.  Built by the test that uses it.
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void curand_philox_kernel(const uint4 *ctr, int n, uint2 key, uint4 *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key);
}

// out[4 i ..] = Philox(ctr[4 i ..], key) for i < n; host arrays.  Returns a
// cudaError_t (0 on success).
extern "C" int curand_philox_ref(const unsigned *ctr, int n, unsigned long long key, unsigned *out)
{
    if (n <= 0) return 0;
    uint4 *d_in = nullptr, *d_out = nullptr;
    const size_t bytes = sizeof(uint4) * (size_t)n;
    cudaError_t e = cudaMalloc(&d_in, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&d_out, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(d_in, ctr, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        curand_philox_kernel<<<(n + 255) / 256, 256>>>(d_in, n, make_uint2((unsigned)key, (unsigned)(key >> 32)),
                                                        d_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, d_out, bytes, cudaMemcpyDeviceToHost);
    cudaFree(d_in);
    cudaFree(d_out);
    return (int)e;
}
