// Texture-gradient preconditioning (the experiments' setup of Sec. 6 preconditions texture
// gradients after Nicolet et al. 2021): g <- (I + lambda L)^{-1} g per channel on the texel grid,
// L the graph Laplacian of the W x H grid with Neumann boundary ((L x)_p = sum over the grid
// neighbours q of x_p - x_q). L is diagonal in the orthonormal DCT-II basis
//   d_k(x) = a_k cos(pi k (x + 1/2) / N),  a_0 = sqrt(1/N), a_k = sqrt(2/N),
// with eigenvalues (2 - 2 cos(pi k / W)) + (2 - 2 cos(pi l / H)), so the solve is exact: the two
// separable transforms, one scale per frequency and the two inverse transforms. The transforms
// are plain matrix products (cuBLAS SGEMM in FP32); the layout changes and the scale are the
// small kernels below.
#include "precond.cuh"

#include <cmath>
#include <vector>

namespace mer {

__global__ void k_hwc_to_chw(const float* __restrict__ g, float* __restrict__ t, int C, int64_t HW) {
    const int64_t n = HW * C, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t p = i / C;
        const int c = (int)(i - p * C);
        t[(int64_t)c * HW + p] = g[i];
    }
}

__global__ void k_chw_to_hwc(const float* __restrict__ t, float* __restrict__ g, int C, int64_t HW) {
    const int64_t n = HW * C, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t p = i / C;
        const int c = (int)(i - p * C);
        g[i] = t[(int64_t)c * HW + p];
    }
}

__global__ void k_scale_planes(float* __restrict__ t, const float* __restrict__ S, int C, int64_t HW) {
    const int64_t n = HW * C, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) t[i] *= S[i % HW];
}

static void dct_matrix(int N, std::vector<float>& D) {
    D.resize((size_t)N * N);
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < N; ++k) {
        const double a = k == 0 ? std::sqrt(1.0 / N) : std::sqrt(2.0 / N);
        for (int x = 0; x < N; ++x) D[(size_t)k * N + x] = (float)(a * std::cos(pi * k * (x + 0.5) / N));
    }
}

cudaError_t precond_init(Precond& pc, int C, int H, int W, float lambda) {
    pc.C = C;
    pc.H = H;
    pc.W = W;
    pc.lambda = lambda;
    std::vector<float> DW, DH, S((size_t)H * W);
    dct_matrix(W, DW);
    dct_matrix(H, DH);
    const double pi = 3.14159265358979323846;
    for (int l = 0; l < H; ++l)
        for (int k = 0; k < W; ++k) {
            const double mu = (2.0 - 2.0 * std::cos(pi * k / W)) + (2.0 - 2.0 * std::cos(pi * l / H));
            S[(size_t)l * W + k] = (float)(1.0 / (1.0 + (double)lambda * mu));
        }
    const size_t plane = (size_t)C * H * W;
    cudaError_t e = cudaMalloc(&pc.DW, sizeof(float) * DW.size());
    if (!e) e = cudaMalloc(&pc.DH, sizeof(float) * DH.size());
    if (!e) e = cudaMalloc(&pc.S, sizeof(float) * S.size());
    if (!e) e = cudaMalloc(&pc.T1, sizeof(float) * plane);
    if (!e) e = cudaMalloc(&pc.T2, sizeof(float) * plane);
    if (!e) e = cudaMemcpy(pc.DW, DW.data(), sizeof(float) * DW.size(), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(pc.DH, DH.data(), sizeof(float) * DH.size(), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(pc.S, S.data(), sizeof(float) * S.size(), cudaMemcpyHostToDevice);
    return e;
}

void precond_free(Precond& pc) {
    for (float* p : {pc.DW, pc.DH, pc.S, pc.T1, pc.T2})
        if (p) cudaFree(p);
    pc.DW = pc.DH = pc.S = pc.T1 = pc.T2 = nullptr;
}

// Row-major products through the column-major library: C(m x n) = op_a(A) op_b(B) is the
// column-major C^T = op_b(B)^T op_a(A)^T, i.e. the call with the operands swapped.
int precond_apply(cublasHandle_t h, const Precond& pc, float* g, cudaStream_t st) {
    const int C = pc.C, H = pc.H, W = pc.W;
    const int64_t HW = (int64_t)H * W, n = HW * C;
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
    const float one = 1.0f, zero = 0.0f;
    cublasSetStream(h, st);
    k_hwc_to_chw<<<blocks, 256, 0, st>>>(g, pc.T1, C, HW);
    // rows (along W): T2 = T1 . DW^T      (C*H rows)
    cublasSgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, W, C * H, W, &one, pc.DW, W, pc.T1, W, &zero, pc.T2, W);
    // columns (along H), per channel: T1_c = DH . T2_c
    cublasSgemmStridedBatched(h, CUBLAS_OP_N, CUBLAS_OP_N, W, H, H, &one, pc.T2, W, HW, pc.DH, H, 0, &zero, pc.T1, W,
                              HW, C);
    k_scale_planes<<<blocks, 256, 0, st>>>(pc.T1, pc.S, C, HW);
    // inverse columns: T2_c = DH^T . T1_c
    cublasSgemmStridedBatched(h, CUBLAS_OP_N, CUBLAS_OP_T, W, H, H, &one, pc.T1, W, HW, pc.DH, H, 0, &zero, pc.T2, W,
                              HW, C);
    // inverse rows: T1 = T2 . DW
    cublasSgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, W, C * H, W, &one, pc.DW, W, pc.T2, W, &zero, pc.T1, W);
    k_chw_to_hwc<<<blocks, 256, 0, st>>>(pc.T1, g, C, HW);
    return 3;   // own kernels (the four products are library launches)
}

}  // namespace mer
