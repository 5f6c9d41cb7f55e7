// Texture-gradient preconditioning: g <- (I + lambda L)^{-1} g per channel of an HWC texture.
#pragma once

#include <cublas_v2.h>

#include "mer_internal.cuh"

namespace mer {

// per-problem transform tables and scratch (device)
struct Precond {
    int C = 0, H = 0, W = 0;
    float lambda = 0.0f;
    float* DW = nullptr;   // W x W orthonormal DCT-II (row k = frequency)
    float* DH = nullptr;   // H x H
    float* S = nullptr;    // H x W: 1 / (1 + lambda * eigenvalue of L)
    float* T1 = nullptr;   // C x H x W scratch
    float* T2 = nullptr;
};

cudaError_t precond_init(Precond& pc, int C, int H, int W, float lambda);
void precond_free(Precond& pc);
// in place on the HWC gradient g (device), on stream st; returns the library's own launches
int precond_apply(cublasHandle_t h, const Precond& pc, float* g, cudaStream_t st);

}  // namespace mer
