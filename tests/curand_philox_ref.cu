// Test helper (not part of the library): first 128-bit draw of the CUDA library's
// Philox4_32_10 device generator for subsequences 0..n-1 of one seed, copied to the host.
#include <cstdint>
#include <curand_kernel.h>

__global__ void k_draw(unsigned long long seed, int n, uint4* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed, (unsigned long long)i, 0ull, &st);
    out[i] = curand4(&st);
}

extern "C" int ref_curand_philox(unsigned long long seed, int n, uint32_t* host_out) {
    uint4* d = nullptr;
    if (cudaMalloc(&d, sizeof(uint4) * (size_t)n) != cudaSuccess) return 1;
    k_draw<<<(n + 127) / 128, 128>>>(seed, n, d);
    const cudaError_t e = cudaMemcpy(host_out, d, sizeof(uint4) * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? 0 : 2;
}
