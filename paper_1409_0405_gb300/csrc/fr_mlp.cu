// The per-element multilayer perceptron of the learned closure: forward,
// backward and Adam, with BF16 GEMM inputs (features, weights, hidden
// activations rounded to bfloat16, round-to-nearest-even) and FP32
// accumulation; biases, pre-activations, gradients and the FP32 master
// parameters stay in FP32.
//
// Network: in -> nh -> nh -> out, GELU (erf form) after the two hidden
// layers.  Parameter vector (FP32): W1[nh][in], b1[nh], W2[nh][nh], b2[nh],
// W3[out][nh], b3[out].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "../../include/fr.h"
#include "fr_mlp.h"

namespace fr {
namespace {

constexpr int TM = 64, TN = 64, TK = 16, NT = 256;

__device__ __forceinline__ float q_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// C[M x N] = alpha * op(A) op(B) + beta * C, FP32 out; op(A) is M x K, op(B)
// is K x N.  TA: A stored K x M (lda = M stride); TB: B stored N x K.
// qa/qb: round A/B elements to BF16 on load.
template <bool TA, bool TB>
__global__ void __launch_bounds__(NT) k_sgemm(int M, int N, int K, const float *__restrict__ A, int lda,
                                              const float *__restrict__ B, int ldb, float *__restrict__ C, int ldc,
                                              float beta, int qa, int qb, int kchunk) {
    __shared__ float sA[TK][TM + 1];
    __shared__ float sB[TK][TN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;  // row tiles on x (no 65535 limit)
    // split-K: slice z covers [z kchunk, (z+1) kchunk) and writes its own
    // M x N partial (C + z M ldc)
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    C += (size_t)blockIdx.z * M * ldc;
    float acc[4][4] = {};
    for (int k0 = kbeg; k0 < kend; k0 += TK) {
        for (int i = threadIdx.x; i < TK * TM; i += NT) {
            const int kk = i / TM, mm = i % TM;
            const int gm = m0 + mm, gk = k0 + kk;
            float v = 0.f;
            if (gm < M && gk < kend) v = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
            sA[kk][mm] = qa ? q_bf16(v) : v;
        }
        for (int i = threadIdx.x; i < TK * TN; i += NT) {
            const int kk = i / TN, nn = i % TN;
            const int gn = n0 + nn, gk = k0 + kk;
            float v = 0.f;
            if (gn < N && gk < kend) v = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
            sB[kk][nn] = qb ? q_bf16(v) : v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sA[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = sB[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
            if (gm < M && gn < N) {
                float *c = C + (size_t)gm * ldc + gn;
                *c = beta == 0.f ? acc[i][j] : acc[i][j] + beta * *c;
            }
        }
}

// C[i] = sum over z < nsplit of part[z][i], fixed order
__global__ void k_sum_splits(int64_t count, int nsplit, const float *part, float *C) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float s = 0.f;
    for (int z = 0; z < nsplit; ++z) s += part[(size_t)z * count + i];
    C[i] = s;
}

constexpr int kMaxSplit = 32;
// K slices of a weight-gradient GEMM (K = number of samples)
inline int splits_for(int64_t K) { return (int)std::min<int64_t>(kMaxSplit, std::max<int64_t>(1, K / 2048)); }

// C = op(A) op(B) (beta = 0) or + beta C; with split > 1 (beta must be 0)
// the K range is cut into `split` slices whose partials go to `part`
// (split x M x N floats) and are summed into C (ldc = N).
template <bool TA, bool TB>
cudaError_t sgemm(int M, int N, int K, const float *A, int lda, const float *B, int ldb, float *C, int ldc, float beta,
                  int qa, int qb, cudaStream_t s, int split = 1, float *part = nullptr) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (split > 1 && (!part || beta != 0.f || ldc != N)) return cudaErrorInvalidValue;
    const int kchunk = split > 1 ? ((K + split - 1) / split + TK - 1) / TK * TK : std::max(K, 1);
    const int nz = split > 1 ? (K + kchunk - 1) / kchunk : 1;
    dim3 grid((M + TM - 1) / TM, (N + TN - 1) / TN, nz);
    k_sgemm<TA, TB><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, nz > 1 ? part : C, ldc, beta, qa, qb, kchunk);
    if (nz > 1) {
        const int64_t cnt = (int64_t)M * N;
        k_sum_splits<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(cnt, nz, part, C);
    }
    return cudaGetLastError();
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x) {
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// Z[b][n] += bias[n]; H = gelu(Z) (act) or H = Z
__global__ void k_bias_act(int64_t rows, int n, float *Z, const float *bias, float *H, int act) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * n) return;
    const float z = Z[i] + bias[i % n];
    Z[i] = z;
    H[i] = act ? gelu(z) : z;
}

// loss = mean (Y - T)^2 (accumulated into loss[0]), dY = 2 (Y - T) / count
__global__ void k_mse(int64_t count, const float *Y, const float *T, float *dY, float *loss) {
    __shared__ float sh[8];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (i < count) {
        const float d = Y[i] - T[i];
        dY[i] = 2.f * d / (float)count;
        l = d * d / (float)count;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        atomicAdd(loss, t);
    }
}

// dZ = dH * gelu'(Z)
__global__ void k_gelu_back(int64_t count, const float *Z, float *dH) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dH[i] *= gelu_d(Z[i]);
}

// column sums db[c] = sum_r dZ[r][c] in two fixed-order stages: block
// (cx, y) sums rows y, y + gridDim.y, ... of 32 columns into part[y][c]
constexpr int kColRows = 64;
__global__ void k_colsum_part(int64_t rows, int n, const float *dZ, float *part) {
    __shared__ float sh[8][33];
    const int c = blockIdx.x * 32 + (threadIdx.x & 31), ty = threadIdx.x >> 5;
    float s = 0.f;
    if (c < n)
        for (int64_t r = (int64_t)blockIdx.y * 8 + ty; r < rows; r += (int64_t)gridDim.y * 8) s += dZ[r * n + c];
    sh[ty][threadIdx.x & 31] = s;
    __syncthreads();
    if (ty == 0 && c < n) {
        float t = 0.f;
        for (int k = 0; k < 8; ++k) t += sh[k][threadIdx.x];
        part[(size_t)blockIdx.y * n + c] = t;
    }
}

cudaError_t colsum(int64_t rows, int n, const float *dZ, float *db, float *part, cudaStream_t s) {
    dim3 grid((n + 31) / 32, kColRows);
    k_colsum_part<<<grid, 256, 0, s>>>(rows, n, dZ, part);
    k_sum_splits<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, kColRows, part, db);
    return cudaGetLastError();
}

// Adam; omb1 = 1 - beta1 and omb2 = 1 - beta2 are formed in double on the
// host (1.f - 0.999f would carry a 1.3e-5 relative error into v)
__global__ void k_adam(int64_t n, float *p, const float *g, float *m, float *v, float lr, float b1, float b2,
                       float omb1, float omb2, float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mm = b1 * m[i] + omb1 * g[i];
    const float vv = b2 * v[i] + omb2 * g[i] * g[i];
    m[i] = mm;
    v[i] = vv;
    p[i] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

inline unsigned nb(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

MlpLayout mlp_layout(int nin, int nh, int nout) {
    MlpLayout L;
    L.W1 = 0;
    L.b1 = L.W1 + (int64_t)nh * nin;
    L.W2 = L.b1 + nh;
    L.b2 = L.W2 + (int64_t)nh * nh;
    L.W3 = L.b2 + nh;
    L.b3 = L.W3 + (int64_t)nout * nh;
    L.n = L.b3 + nout;
    return L;
}

int64_t mlp_workspace_floats(int nin, int nh, int nout, int64_t n) {
    // Z1, H1, Z2, H2, dZ2, dZ1 (n x nh each), Y, dY (n x nout each), then
    // the split-K / column-sum partials
    const int64_t wmax = (int64_t)nh * std::max(std::max(nin, nh), nout);
    const int64_t part = std::max<int64_t>((int64_t)kMaxSplit * wmax, (int64_t)kColRows * std::max(nh, nout));
    return n * (6 * (int64_t)nh + 2 * (int64_t)nout) + part;
}

cudaError_t mlp_forward(int nin, int nh, int nout, int64_t n, const float *X, const float *P, float *Y, float *ws,
                        cudaStream_t s) {
    const MlpLayout L = mlp_layout(nin, nh, nout);
    float *Z1 = ws, *H1 = Z1 + n * nh, *Z2 = H1 + n * nh, *H2 = Z2 + n * nh;
    cudaError_t e;
    // Z1 = bf16(X) bf16(W1)^T + b1, H1 = gelu(Z1)
    if ((e = sgemm<false, true>((int)n, nh, nin, X, nin, P + L.W1, nin, Z1, nh, 0.f, 1, 1, s)) != cudaSuccess) return e;
    k_bias_act<<<nb(n * nh, 256), 256, 0, s>>>(n, nh, Z1, P + L.b1, H1, 1);
    // Z2 = bf16(H1) bf16(W2)^T + b2, H2 = gelu(Z2)
    if ((e = sgemm<false, true>((int)n, nh, nh, H1, nh, P + L.W2, nh, Z2, nh, 0.f, 1, 1, s)) != cudaSuccess) return e;
    k_bias_act<<<nb(n * nh, 256), 256, 0, s>>>(n, nh, Z2, P + L.b2, H2, 1);
    // Y = bf16(H2) bf16(W3)^T + b3
    if ((e = sgemm<false, true>((int)n, nout, nh, H2, nh, P + L.W3, nh, Y, nout, 0.f, 1, 1, s)) != cudaSuccess)
        return e;
    k_bias_act<<<nb(n * nout, 256), 256, 0, s>>>(n, nout, Y, P + L.b3, Y, 0);
    return cudaGetLastError();
}

cudaError_t mlp_grad(int nin, int nh, int nout, int64_t n, const float *X, const float *T, const float *P, float *G,
                     float *loss, float *ws, cudaStream_t s) {
    const MlpLayout L = mlp_layout(nin, nh, nout);
    float *Z1 = ws, *H1 = Z1 + n * nh, *Z2 = H1 + n * nh, *H2 = Z2 + n * nh;
    float *dZ2 = H2 + n * nh, *dZ1 = dZ2 + n * nh, *Y = dZ1 + n * nh, *dY = Y + n * nout, *part = dY + n * nout;
    const int sp = splits_for(n);
    cudaError_t e;
    if ((e = mlp_forward(nin, nh, nout, n, X, P, Y, ws, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(loss, 0, sizeof(float), s)) != cudaSuccess) return e;
    k_mse<<<nb(n * nout, 256), 256, 0, s>>>(n * nout, Y, T, dY, loss);
    // layer 3: dW3 = dY^T bf16(H2), db3 = sum dY, dZ2 = (dY bf16(W3)) gelu'(Z2)
    if ((e = sgemm<true, false>(nout, nh, (int)n, dY, nout, H2, nh, G + L.W3, nh, 0.f, 0, 1, s, sp, part)))
        return e;
    if ((e = colsum(n, nout, dY, G + L.b3, part, s))) return e;
    if ((e = sgemm<false, false>((int)n, nh, nout, dY, nout, P + L.W3, nh, dZ2, nh, 0.f, 0, 1, s))) return e;
    k_gelu_back<<<nb(n * nh, 256), 256, 0, s>>>(n * nh, Z2, dZ2);
    // layer 2: dW2 = dZ2^T bf16(H1), db2, dZ1 = (dZ2 bf16(W2)) gelu'(Z1)
    if ((e = sgemm<true, false>(nh, nh, (int)n, dZ2, nh, H1, nh, G + L.W2, nh, 0.f, 0, 1, s, sp, part))) return e;
    if ((e = colsum(n, nh, dZ2, G + L.b2, part, s))) return e;
    if ((e = sgemm<false, false>((int)n, nh, nh, dZ2, nh, P + L.W2, nh, dZ1, nh, 0.f, 0, 1, s))) return e;
    k_gelu_back<<<nb(n * nh, 256), 256, 0, s>>>(n * nh, Z1, dZ1);
    // layer 1: dW1 = dZ1^T bf16(X), db1
    if ((e = sgemm<true, false>(nh, nin, (int)n, dZ1, nh, X, nin, G + L.W1, nin, 0.f, 0, 1, s, sp, part)))
        return e;
    if ((e = colsum(n, nh, dZ1, G + L.b1, part, s))) return e;
    return cudaGetLastError();
}

cudaError_t mlp_adam(int64_t n, float *P, const float *G, float *m, float *v, int step, float lr, cudaStream_t s) {
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - std::pow(b1, step)), c2 = (float)(1.0 - std::pow(b2, step));
    k_adam<<<nb(n, 256), 256, 0, s>>>(n, P, G, m, v, lr, (float)b1, (float)b2, (float)(1.0 - b1), (float)(1.0 - b2),
                                      1e-8f, c1, c2);
    return cudaGetLastError();
}

}  // namespace fr
