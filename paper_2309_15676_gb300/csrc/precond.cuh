// Texture-gradient preconditioning: g <- (I + lambda L)^{-1} g per channel of an HWC texture.
#pragma once

#include "mer_internal.cuh"

namespace mer {

// Tables of one axis of length N: a power of two >= 4 uses the FFT route (log2n > 0, radix-2
// twiddles exp(-2 pi i j / N) for j < N/2 and exp(-i pi k / (2N)) for k < N); any other N the
// direct sum over cos(pi m / (2N)), m < 4N.
struct PcAxis {
    int N = 0, log2n = 0;
    float2* fft_tw = nullptr;
    float2* dct_tw = nullptr;
    float* cos4 = nullptr;
};

// per-problem transform tables and scratch (device)
struct Precond {
    int C = 0, H = 0, W = 0;
    float lambda = 0.0f;
    PcAxis ax_w, ax_h;
    float* St = nullptr;   // W x H: 1 / (1 + lambda * eigenvalue of L), frequency (k, l) at k * H + l
    float* T1 = nullptr;   // C x H x W scratch
    float* T2 = nullptr;
};

cudaError_t precond_init(Precond& pc, int C, int H, int W, float lambda);
void precond_free(Precond& pc);
// dynamic shared memory the row and column kernels need for a C x H x W texture
size_t precond_max_smem(int C, int H, int W);
// in place on the HWC gradient g (device), on stream st; returns the library's own launches (5)
int precond_apply(const Precond& pc, float* g, cudaStream_t st);

}  // namespace mer
