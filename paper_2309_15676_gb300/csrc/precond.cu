// Texture-gradient preconditioning (the experiments' setup of Sec. 6 preconditions texture
// gradients after Nicolet et al. 2021): g <- (I + lambda L)^{-1} g per channel on the texel grid,
// L the graph Laplacian of the W x H grid with Neumann boundary ((L x)_p = sum over the grid
// neighbours q of x_p - x_q). L is diagonal in the DCT-II basis cos(pi k (2x + 1) / (2N)), with
// eigenvalues (2 - 2 cos(pi k / W)) + (2 - 2 cos(pi l / H)), so the solve is exact: the two
// separable forward transforms, one scale per frequency, the two inverse transforms. With the
// unnormalised transform C = Cos x and its inverse, (I + lambda L)^{-1} = Cos^{-1} S Cos for both
// axes (the orthonormal scale factors cancel), S = 1 / (1 + lambda mu).
//
// The 1-D transforms run in shared memory, several lines per block (the C channels of one texel
// row; about 2048 points of columns):
//  - N a power of two (every texture size of the workloads): Makhoul's reordering, an N-point
//    radix-2 complex FFT and one twiddle, so a transform costs O(N log N) and every pass is one
//    read and one write of the texture;
//  - any other N: the direct sum over a 4N-entry cosine table, O(N^2) per row.
// Five launches per gradient texture: row transforms (reading the HWC gradient), a transpose, the
// column transforms with the scale and the inverse column transforms, a transpose back, and the
// inverse row transforms (writing the HWC gradient). Twiddles and cosines are computed on the host
// in double precision.
#include "precond.cuh"

#include <cmath>
#include <vector>

namespace mer {

namespace {

constexpr int PC_THREADS = 256;
constexpr int kMaxTexSide = 4094;   // mer_scene_add's limit on a texture side

__host__ __device__ inline bool is_pow2(int n) { return n >= 4 && (n & (n - 1)) == 0; }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ unsigned bit_reverse(unsigned i, int bits) { return __brev(i) >> (32 - bits); }

// Complex scratch of a line is padded by one entry every 32, so that the bit-reversed scatter
// (consecutive n go to entries 2^k apart) and the butterflies spread over the shared-memory banks.
__host__ __device__ inline int zpad(int i) { return i + (i >> 5); }
__host__ __device__ inline int zline(int N) { return N + (N >> 5); }

// In-place radix-2 decimation-in-time FFTs of L lines (line l at z + l * zline(N), entry i at
// zpad(i); inputs already in bit-reversed order), all threads of the block; sign -1: forward
// (twiddles tw[j] = exp(-2 pi i j / N)), +1: inverse (conjugate twiddles, no 1/N).
__device__ void fft_lines(float2* z, int N, int L, int log2n, const float2* __restrict__ tw, float sign) {
    const int half_n = N >> 1, zs = zline(N);
    for (int s = 1; s <= log2n; ++s) {
        const int half = 1 << (s - 1);
        const int step = N >> s;   // twiddle index stride
        for (int t = threadIdx.x; t < L * half_n; t += blockDim.x) {
            const int l = t >> (log2n - 1), b = t & (half_n - 1);   // N and N / 2 are powers of two
            const int j = b & (half - 1);
            float2* zl = z + l * zs;
            const int i0 = ((b >> (s - 1)) << s) + j, i1 = i0 + half;
            float2 w = __ldg(tw + j * step);
            if (sign > 0.0f) w.y = -w.y;   // the inverse uses the conjugate twiddles
            const float2 v = cmul(w, zl[zpad(i1)]);
            const float2 u = zl[zpad(i0)];
            zl[zpad(i0)] = make_float2(u.x + v.x, u.y + v.y);
            zl[zpad(i1)] = make_float2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
}

// Forward unnormalised DCT-II of L lines at once: line l's input element n at
// x[l * xl + n * xe] (shared memory), output element k to out[l * ol + k * oe] (shared or
// global): out[k] = sum_n x[n] cos(pi k (2n + 1) / (2N)). z: L * N float2 of shared scratch
// (unused by the direct route).
__device__ void dct2_lines(const float* x, int xe, int xl, float* out, int oe, size_t ol, int L, const PcAxis& ax,
                           float2* z) {
    const int N = ax.N;
    if (ax.log2n > 0) {
        for (int t = threadIdx.x; t < L * N; t += blockDim.x) {
            const int l = t >> ax.log2n, n = t & (N - 1);
            // v[n] = x[2n] (n < N/2), v[N-1-n'] = x[2n'+1]
            const int src = n < N / 2 ? 2 * n : 2 * (N - 1 - n) + 1;
            z[l * zline(N) + zpad((int)bit_reverse((unsigned)n, ax.log2n))] = make_float2(x[l * xl + src * xe], 0.0f);
        }
        __syncthreads();
        fft_lines(z, N, L, ax.log2n, ax.fft_tw, -1.0f);
        for (int t = threadIdx.x; t < L * N; t += blockDim.x) {
            const int l = t >> ax.log2n, k = t & (N - 1);
            const float2 e = __ldg(ax.dct_tw + k);   // exp(-i pi k / (2N))
            const float2 v = z[l * zline(N) + zpad(k)];
            out[l * ol + (size_t)k * oe] = e.x * v.x - e.y * v.y;
        }
        __syncthreads();
    } else {
        for (int t = threadIdx.x; t < L * N; t += blockDim.x) {
            const int l = t / N, k = t - l * N;
            const float* xx = x + l * xl;
            float acc = 0.0f;
            int m = k;                       // k (2n + 1) mod 4N, stepping by 2k
            const int step = (2 * k) % (4 * N);
            for (int n = 0; n < N; ++n) {
                acc = fmaf(xx[n * xe], __ldg(ax.cos4 + m), acc);
                m += step;
                if (m >= 4 * N) m -= 4 * N;
            }
            out[l * ol + (size_t)k * oe] = acc;
        }
        __syncthreads();
    }
}

// Inverse of dct2_lines for L lines: line l's coefficients C[k] at c[l * cl + k * ce] (shared
// memory), the result element n to out[l * ol + n * oe].
__device__ void dct2_inv_lines(const float* c, int ce, int cl, float* out, int oe, size_t ol, int L,
                               const PcAxis& ax, float2* z) {
    const int N = ax.N;
    if (ax.log2n > 0) {
        // V[k] = exp(+i pi k / (2N)) (C[k] - i C[N-k]), C[N] = 0; v = IFFT(V) / N
        for (int t = threadIdx.x; t < L * N; t += blockDim.x) {
            const int l = t >> ax.log2n, k = t & (N - 1);
            const float* cc = c + l * cl;
            const float a = cc[k * ce], b = k == 0 ? 0.0f : cc[(N - k) * ce];
            const float2 e = __ldg(ax.dct_tw + k);
            const float2 w = make_float2(e.x, -e.y);   // exp(+i pi k / (2N))
            z[l * zline(N) + zpad((int)bit_reverse((unsigned)k, ax.log2n))] = cmul(w, make_float2(a, -b));
        }
        __syncthreads();
        fft_lines(z, N, L, ax.log2n, ax.fft_tw, 1.0f);
        const float inv = 1.0f / (float)N;
        for (int t = threadIdx.x; t < L * N; t += blockDim.x) {
            const int l = t >> ax.log2n, n = t & (N - 1);
            // x[2m] = Re v[m] (m < N/2), x[2m+1] = Re v[N-1-m]
            const int src = (n & 1) ? (N - 1 - (n >> 1)) : (n >> 1);
            out[l * ol + (size_t)n * oe] = z[l * zline(N) + zpad(src)].x * inv;
        }
        __syncthreads();
    } else {
        // x[n] = sum_k w_k C[k] cos(pi k (2n + 1) / (2N)), w_0 = 1/N, w_k = 2/N
        const float w0 = 1.0f / (float)N, w1 = 2.0f / (float)N;
        for (int t = threadIdx.x; t < L * N; t += blockDim.x) {
            const int l = t / N, n = t - l * N;
            const float* cc = c + l * cl;
            float acc = 0.0f;
            int m = 0;                       // k (2n + 1) mod 4N, stepping by 2n + 1
            const int step = (2 * n + 1) % (4 * N);
            for (int k = 0; k < N; ++k) {
                acc = fmaf((k == 0 ? w0 : w1) * cc[k * ce], __ldg(ax.cos4 + m), acc);
                m += step;
                if (m >= 4 * N) m -= 4 * N;
            }
            out[l * ol + (size_t)n * oe] = acc;
        }
        __syncthreads();
    }
}

__host__ __device__ inline size_t round4(size_t n) { return (n + 3) & ~(size_t)3; }

// rows of the HWC gradient, all C channels of one row at once: T[c][y][k] = forward transform
// along x of g[y][.][c]
__global__ void __launch_bounds__(PC_THREADS) k_pc_rows_fwd(const float* __restrict__ g, float* __restrict__ T, int C,
                                                            int H, PcAxis ax) {
    extern __shared__ float4 pc_smem[];
    const int W = ax.N, y = blockIdx.x;
    float* row = reinterpret_cast<float*>(pc_smem);                 // W x C (HWC order)
    float2* z = reinterpret_cast<float2*>(row + round4((size_t)W * C));
    const float* src = g + (size_t)y * W * C;
    for (int i = threadIdx.x; i < W * C; i += blockDim.x) row[i] = src[i];
    __syncthreads();
    dct2_lines(row, C, 1, T + (size_t)y * W, 1, (size_t)H * W, C, ax, z);
}

// inverse rows back into the HWC gradient, all channels of one row at once: g[y][.][c] = inverse
// transform of T[c][y][.]
__global__ void __launch_bounds__(PC_THREADS) k_pc_rows_inv(const float* __restrict__ T, float* __restrict__ g, int C,
                                                            int H, PcAxis ax) {
    extern __shared__ float4 pc_smem[];
    const int W = ax.N, y = blockIdx.x;
    float* row = reinterpret_cast<float*>(pc_smem);                 // C x W in
    float* res = row + round4((size_t)C * W);                       // W x C out (HWC order)
    float2* z = reinterpret_cast<float2*>(res + round4((size_t)W * C));
    for (int i = threadIdx.x; i < C * W; i += blockDim.x) {
        const int c = i / W, x = i - c * W;
        row[i] = T[((size_t)c * H + y) * W + x];
    }
    __syncthreads();
    dct2_inv_lines(row, 1, W, res, C, 1, C, ax, z);
    float* dst = g + (size_t)y * W * C;
    for (int i = threadIdx.x; i < W * C; i += blockDim.x) dst[i] = res[i];
}

// columns (as rows after the transpose), K of them per block:
// U[c][k][.] <- inverse_y( S^T[k][.] * forward_y(U[c][k][.]) )
__global__ void __launch_bounds__(PC_THREADS) k_pc_cols(float* __restrict__ U, const float* __restrict__ St, int W,
                                                        int K, PcAxis ax) {
    extern __shared__ float4 pc_smem[];
    const int H = ax.N;
    const int groups = (W + K - 1) / K;
    const int c = blockIdx.x / groups, k0 = (blockIdx.x - c * groups) * K;
    const int L = min(K, W - k0);
    float* col = reinterpret_cast<float*>(pc_smem);                 // L x H
    float* frq = col + round4((size_t)K * H);                       // L x H
    float2* z = reinterpret_cast<float2*>(frq + round4((size_t)K * H));
    float* lines = U + ((size_t)c * W + k0) * H;                    // L consecutive lines of H
    for (int i = threadIdx.x; i < L * H; i += blockDim.x) col[i] = lines[i];
    __syncthreads();
    dct2_lines(col, 1, H, frq, 1, H, L, ax, z);
    const float* s = St + (size_t)k0 * H;
    for (int i = threadIdx.x; i < L * H; i += blockDim.x) frq[i] *= __ldg(s + i);
    __syncthreads();
    dct2_inv_lines(frq, 1, H, lines, 1, H, L, ax, z);
}

// out[c][j][i] = in[c][i][j] for C planes of R x Q (32 x 32 tiles)
__global__ void k_pc_transpose(const float* __restrict__ in, float* __restrict__ out, int R, int Q) {
    __shared__ float tile[32][33];
    const int c = blockIdx.z;
    const int q0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const float* src = in + (size_t)c * R * Q;
    float* dst = out + (size_t)c * R * Q;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int r = r0 + dy, q = q0 + threadIdx.x;
        if (r < R && q < Q) tile[dy][threadIdx.x] = src[(size_t)r * Q + q];
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int q = q0 + dy, r = r0 + threadIdx.x;
        if (q < Q && r < R) dst[(size_t)q * R + r] = tile[threadIdx.x][dy];
    }
}

// complex scratch only for the FFT route
size_t fft_scratch(const PcAxis& ax, int lines) {
    return ax.log2n > 0 ? sizeof(float2) * (size_t)lines * zline(ax.N) : 0;
}
size_t rows_fwd_smem(const PcAxis& ax, int C) { return sizeof(float) * round4((size_t)ax.N * C) + fft_scratch(ax, C); }
size_t rows_inv_smem(const PcAxis& ax, int C) {
    return 2 * sizeof(float) * round4((size_t)ax.N * C) + fft_scratch(ax, C);
}
// columns per block: about 2048 points of work per block, at least one column
int cols_per_block(int H) { return H >= 2048 ? 1 : 2048 / H; }
size_t cols_smem(const PcAxis& ax, int K) {
    return 2 * sizeof(float) * round4((size_t)K * ax.N) + fft_scratch(ax, K);
}

cudaError_t axis_init(PcAxis& ax, int N) {
    ax.N = N;
    ax.log2n = 0;
    if (is_pow2(N))
        while ((1 << ax.log2n) < N) ++ax.log2n;
    const double pi = 3.14159265358979323846;
    cudaError_t e = cudaSuccess;
    if (ax.log2n > 0) {
        std::vector<float2> ft(N / 2), dt(N);
        for (int j = 0; j < N / 2; ++j) ft[j] = make_float2((float)std::cos(2 * pi * j / N), (float)-std::sin(2 * pi * j / N));
        for (int k = 0; k < N; ++k) dt[k] = make_float2((float)std::cos(pi * k / (2.0 * N)), (float)-std::sin(pi * k / (2.0 * N)));
        e = cudaMalloc(&ax.fft_tw, sizeof(float2) * ft.size());
        if (!e) e = cudaMalloc(&ax.dct_tw, sizeof(float2) * dt.size());
        if (!e) e = cudaMemcpy(ax.fft_tw, ft.data(), sizeof(float2) * ft.size(), cudaMemcpyHostToDevice);
        if (!e) e = cudaMemcpy(ax.dct_tw, dt.data(), sizeof(float2) * dt.size(), cudaMemcpyHostToDevice);
    } else {
        std::vector<float> ct(4 * (size_t)N);
        for (int m = 0; m < 4 * N; ++m) ct[m] = (float)std::cos(pi * m / (2.0 * N));
        e = cudaMalloc(&ax.cos4, sizeof(float) * ct.size());
        if (!e) e = cudaMemcpy(ax.cos4, ct.data(), sizeof(float) * ct.size(), cudaMemcpyHostToDevice);
    }
    return e;
}

void axis_free(PcAxis& ax) {
    for (void* p : {(void*)ax.fft_tw, (void*)ax.dct_tw, (void*)ax.cos4})
        if (p) cudaFree(p);
    ax.fft_tw = ax.dct_tw = nullptr;
    ax.cos4 = nullptr;
}

}  // namespace

size_t precond_max_smem(int C, int H, int W) {
    PcAxis aw, ah;   // sizes only (no tables)
    aw.N = W;
    ah.N = H;
    aw.log2n = is_pow2(W) ? 31 - __builtin_clz((unsigned)W) : 0;
    ah.log2n = is_pow2(H) ? 31 - __builtin_clz((unsigned)H) : 0;
    return std::max(std::max(rows_fwd_smem(aw, C), rows_inv_smem(aw, C)), cols_smem(ah, cols_per_block(H)));
}

cudaError_t precond_init(Precond& pc, int C, int H, int W, float lambda) {
    pc.C = C;
    pc.H = H;
    pc.W = W;
    pc.lambda = lambda;
    std::vector<float> St((size_t)H * W);
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < W; ++k)
        for (int l = 0; l < H; ++l) {
            const double mu = (2.0 - 2.0 * std::cos(pi * k / W)) + (2.0 - 2.0 * std::cos(pi * l / H));
            St[(size_t)k * H + l] = (float)(1.0 / (1.0 + (double)lambda * mu));
        }
    const size_t plane = (size_t)C * H * W;
    cudaError_t e = axis_init(pc.ax_w, W);
    if (!e) e = axis_init(pc.ax_h, H);
    if (!e) e = cudaMalloc(&pc.St, sizeof(float) * St.size());
    if (!e) e = cudaMalloc(&pc.T1, sizeof(float) * plane);
    if (!e) e = cudaMalloc(&pc.T2, sizeof(float) * plane);
    if (!e) e = cudaMemcpy(pc.St, St.data(), sizeof(float) * St.size(), cudaMemcpyHostToDevice);
    // the opt-in shared-memory limit of the three kernels, set for the largest texture the library
    // accepts (the largest power-of-two side, through the FFT route, and the largest side, through
    // the direct one), so that one problem's setting never lowers another's
    const int smem = (int)std::max(precond_max_smem(MER_MAX_CHANNELS, 2048, 2048),
                                   precond_max_smem(MER_MAX_CHANNELS, kMaxTexSide, kMaxTexSide));
    const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (!e) e = cudaFuncSetAttribute(k_pc_rows_fwd, at, smem);
    if (!e) e = cudaFuncSetAttribute(k_pc_rows_inv, at, smem);
    if (!e) e = cudaFuncSetAttribute(k_pc_cols, at, smem);
    return e;
}

void precond_free(Precond& pc) {
    axis_free(pc.ax_w);
    axis_free(pc.ax_h);
    for (float* p : {pc.St, pc.T1, pc.T2})
        if (p) cudaFree(p);
    pc.St = pc.T1 = pc.T2 = nullptr;
}

int precond_apply(const Precond& pc, float* g, cudaStream_t st) {
    const int C = pc.C, H = pc.H, W = pc.W;
    const dim3 tb(32, 8);
    // T1[c][y][k] <- row transforms of g
    k_pc_rows_fwd<<<H, PC_THREADS, rows_fwd_smem(pc.ax_w, C), st>>>(g, pc.T1, C, H, pc.ax_w);
    // T2[c][k][y] <- T1[c][y][k]
    k_pc_transpose<<<dim3((W + 31) / 32, (H + 31) / 32, C), tb, 0, st>>>(pc.T1, pc.T2, H, W);
    // columns: forward, scale, inverse (in place on T2)
    const int K = cols_per_block(H);
    k_pc_cols<<<C * ((W + K - 1) / K), PC_THREADS, cols_smem(pc.ax_h, K), st>>>(pc.T2, pc.St, W, K, pc.ax_h);
    // T1[c][y][k] <- T2[c][k][y]
    k_pc_transpose<<<dim3((H + 31) / 32, (W + 31) / 32, C), tb, 0, st>>>(pc.T2, pc.T1, W, H);
    // g <- inverse row transforms of T1
    k_pc_rows_inv<<<H, PC_THREADS, rows_inv_smem(pc.ax_w, C), st>>>(pc.T1, g, C, H, pc.ax_w);
    return 5;
}

}  // namespace mer
