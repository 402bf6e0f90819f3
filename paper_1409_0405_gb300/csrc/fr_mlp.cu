// The per-element multilayer perceptron of the learned closure: forward,
// backward and Adam, with BF16 GEMM inputs (features, weights, hidden
// activations rounded to bfloat16, round-to-nearest-even) and FP32
// accumulation; biases, pre-activations, gradients and the FP32 master
// parameters stay in FP32.
//
// Network: in -> nh -> nh -> out, GELU (erf form) after the two hidden
// layers.  Parameter vector (FP32): W1[nh][in], b1[nh], W2[nh][nh], b2[nh],
// W3[out][nh], b3[out].
//
// The layers run on the tcgen05 tensor cores through the operator kernel
// (fr_gemm_tc.cu): with the activations stored feature-major ([feature]
// [sample], samples fastest, the FR state layout), a layer H = act(W X + b)
// is an operator application with W as the resident operator, packed to
// bf16 on the device.  Forward: one product per K step, bf16(W) bf16(X),
// FP32 accumulation, bias and GELU in the epilogue.  Backward data
// gradients dZ = (W^T dY) * gelu'(Z): the same kernel on W^T, dY carried
// as bf16 hi + lo (two products), gelu' in the epilogue.  The weight
// gradients, reductions over the samples (dW = dZ bf16(H)^T), run on the
// split-K FP32 kernel below, summed in a fixed order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "../../include/fr.h"
#include "fr_kernels.h"
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

// out[c][r] = in[r][c] for r < rows, c < cols; in rows have stride ldi,
// out rows stride ldo, columns rows..ldo-1 of out are zero (32 x 32 tiles)
__global__ void k_transpose(int64_t rows, int cols, const float *__restrict__ in, int64_t ldi, int64_t ldo,
                            float *__restrict__ out) {
    __shared__ float tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int k = ty; k < 32; k += 8) {
        const int64_t r = r0 + k;
        const int c = c0 + tx;
        tile[k][tx] = (r < rows && c < cols) ? in[r * ldi + c] : 0.f;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int c = c0 + k;
        const int64_t r = r0 + tx;
        if (c < cols && r < ldo) out[(int64_t)c * ldo + r] = tile[tx][k];
    }
}

// feature-major loss: over rows x n samples (row stride ld), loss +=
// mean (Y - T)^2, dY = 2 (Y - T) / count; padding columns get dY = 0
__global__ void k_mse_fm(int rows, int64_t n, int64_t ld, const float *Y, const float *T, float *dY, float *loss) {
    __shared__ float sh[8];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const float count = (float)((double)rows * (double)n);
    float l = 0.f;
    if (i < (int64_t)rows * ld) {
        const int64_t c = i % ld;
        float d = 0.f;
        if (c < n) {
            d = Y[i] - T[i];
            l = d * d / count;
        }
        dY[i] = 2.f * d / count;
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

// row sums db[r] = sum_{c < n} dZ[r][c] (row stride ld), one block per row,
// a fixed order: strided partial sums, then a tree over the block
__global__ void k_rowsum(int64_t n, int64_t ld, const float *__restrict__ dZ, float *__restrict__ db) {
    __shared__ float sh[256];
    const float *row = dZ + (int64_t)blockIdx.x * ld;
    float s = 0.f;
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) s += row[c];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[blockIdx.x] = sh[0];
}

}  // namespace

// one network layer on the tensor cores: C[M][np] = epi(op . B[K][np])
static cudaError_t tc_layer(const TcOperator &op, int M, int K, int64_t np, const float *B, float *C, int mode,
                            const float *bias, float *Z, const float *Zin, int act, int *err, cudaStream_t s) {
    GemmArgsT<float> g;
    g.M = M;
    g.N = np;
    g.K1 = K;
    g.B1 = B;
    g.ldb1 = np;
    g.C = C;
    g.ldc = np;
    g.mode = mode;
    g.np = np;
    g.bias = bias;
    g.Z = Z;
    g.Zin = Zin;
    g.act = act;
    return launch_gemm_tc(g, op, err, s);
}

MlpWs mlp_ws(int nin, int nh, int nout, int64_t n, float *ws) {
    MlpWs w;
    w.npad = (n + 3) / 4 * 4;
    const int64_t np = w.npad;
    float *p = ws;
    w.err = reinterpret_cast<int *>(p);
    p += 4;
    w.X = p;
    p += (int64_t)nin * np;
    w.Z1 = p;
    w.H1 = w.Z1 + (int64_t)nh * np;
    w.Z2 = w.H1 + (int64_t)nh * np;
    w.H2 = w.Z2 + (int64_t)nh * np;
    w.dZ2 = w.H2 + (int64_t)nh * np;
    w.dZ1 = w.dZ2 + (int64_t)nh * np;
    w.Y = w.dZ1 + (int64_t)nh * np;
    w.dY = w.Y + (int64_t)nout * np;
    w.T = w.dY + (int64_t)nout * np;
    uint8_t *img = reinterpret_cast<uint8_t *>(w.T + (int64_t)nout * np);
    const size_t bi[5] = {tc_hi_image_bytes(nh, nin), tc_hi_image_bytes(nh, nh), tc_hi_image_bytes(nout, nh),
                          tc_hi_image_bytes(nh, nout), tc_hi_image_bytes(nh, nh)};
    for (int k = 0; k < 5; ++k) {
        w.img[k] = img;
        img += bi[k];
    }
    w.part = reinterpret_cast<float *>(img);
    return w;
}

cudaError_t mlp_pack_forward(int nin, int nh, int nout, const float *P, MlpWs &w, cudaStream_t s) {
    const MlpLayout L = mlp_layout(nin, nh, nout);
    cudaError_t e;
    if ((e = tc_pack_hi(P + L.W1, nh, nin, nin, 0, w.img[0], w.op[0], s)) != cudaSuccess) return e;
    if ((e = tc_pack_hi(P + L.W2, nh, nh, nh, 0, w.img[1], w.op[1], s)) != cudaSuccess) return e;
    return tc_pack_hi(P + L.W3, nout, nh, nh, 0, w.img[2], w.op[2], s);
}

cudaError_t mlp_forward_fm(int nin, int nh, int nout, int64_t np, const float *X, const float *P, float *Y,
                           const MlpWs &w, bool keep_z, int *err, cudaStream_t s, const ClosureOut *cl) {
    const MlpLayout L = mlp_layout(nin, nh, nout);
    cudaError_t e;
    if ((e = tc_layer(w.op[0], nh, nin, np, X, w.H1, GEMM_BIAS_ACT, P + L.b1, keep_z ? w.Z1 : nullptr, nullptr, 1,
                      err, s)) != cudaSuccess)
        return e;
    if ((e = tc_layer(w.op[1], nh, nh, np, w.H1, w.H2, GEMM_BIAS_ACT, P + L.b2, keep_z ? w.Z2 : nullptr, nullptr, 1,
                      err, s)) != cudaSuccess)
        return e;
    if (!cl) return tc_layer(w.op[2], nout, nh, np, w.H2, Y, GEMM_BIAS_ACT, P + L.b3, nullptr, nullptr, 0, err, s);
    // the output layer writes the RHS correction directly
    GemmArgsT<float> g;
    g.M = nout;
    g.N = np;
    g.K1 = nh;
    g.B1 = w.H2;
    g.ldb1 = np;
    g.ldc = np;
    g.mode = GEMM_BIAS_ACT;
    g.np = np;
    g.bias = P + L.b3;
    g.rfs = cl->rfs;
    g.cl_add = cl->add;
    g.cl_nu = cl->nu;
    g.cl_ne = cl->ne;
    for (int v = 0; v < 5; ++v) g.cl_scale[v] = cl->scale[v];
    return launch_gemm_tc(g, w.op[2], err, s);
}

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
    // the status word, X, Z1, H1, Z2, H2, dZ2, dZ1, Y, dY, T (feature-major,
    // npad samples each), the five bf16 weight images, then the split-K
    // partials of the weight gradients
    const int64_t np = (n + 3) / 4 * 4;
    const int64_t wmax = (int64_t)nh * std::max(std::max(nin, nh), nout);
    const size_t img = tc_hi_image_bytes(nh, nin) + 2 * tc_hi_image_bytes(nh, nh) + tc_hi_image_bytes(nout, nh) +
                       tc_hi_image_bytes(nh, nout);
    return 4 + np * ((int64_t)nin + 6 * (int64_t)nh + 3 * (int64_t)nout) + (int64_t)(img / 4) +
           (int64_t)kMaxSplit * wmax;
}

cudaError_t mlp_forward(int nin, int nh, int nout, int64_t n, const float *X, const float *P, float *Y, float *ws,
                        cudaStream_t s) {
    MlpWs w = mlp_ws(nin, nh, nout, n, ws);
    const int64_t np = w.npad;
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.err, 0, sizeof(int), s)) != cudaSuccess) return e;
    // samples to feature-major, the three layers, back to [n][nout]
    k_transpose<<<dim3(nb(np, 32), nb(nin, 32)), 256, 0, s>>>(n, nin, X, nin, np, w.X);
    if ((e = mlp_pack_forward(nin, nh, nout, P, w, s)) != cudaSuccess) return e;
    if ((e = mlp_forward_fm(nin, nh, nout, np, w.X, P, w.Y, w, true, w.err, s)) != cudaSuccess) return e;
    k_transpose<<<dim3(nb(nout, 32), nb(n, 32)), 256, 0, s>>>(nout, (int)n, w.Y, np, nout, Y);
    return cudaGetLastError();
}

cudaError_t mlp_grad(int nin, int nh, int nout, int64_t n, const float *X, const float *T, const float *P, float *G,
                     float *loss, float *ws, cudaStream_t s) {
    const MlpLayout L = mlp_layout(nin, nh, nout);
    MlpWs w = mlp_ws(nin, nh, nout, n, ws);
    const int64_t np = w.npad;
    const int sp = splits_for(n);
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.err, 0, sizeof(int), s)) != cudaSuccess) return e;
    k_transpose<<<dim3(nb(np, 32), nb(nin, 32)), 256, 0, s>>>(n, nin, X, nin, np, w.X);
    k_transpose<<<dim3(nb(np, 32), nb(nout, 32)), 256, 0, s>>>(n, nout, T, nout, np, w.T);
    if ((e = mlp_pack_forward(nin, nh, nout, P, w, s)) != cudaSuccess) return e;
    if ((e = mlp_forward_fm(nin, nh, nout, np, w.X, P, w.Y, w, true, w.err, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(loss, 0, sizeof(float), s)) != cudaSuccess) return e;
    k_mse_fm<<<nb(nout * np, 256), 256, 0, s>>>(nout, n, np, w.Y, w.T, w.dY, loss);
    // transposed weights for the data gradients
    if ((e = tc_pack_hi(P + L.W3, nout, nh, nh, 1, w.img[3], w.op[3], s)) != cudaSuccess) return e;
    if ((e = tc_pack_hi(P + L.W2, nh, nh, nh, 1, w.img[4], w.op[4], s)) != cudaSuccess) return e;
    // layer 3: dW3 = dY bf16(H2)^T, db3 = row sums of dY, dZ2 = (W3^T dY) gelu'(Z2)
    if ((e = sgemm<false, true>(nout, nh, (int)n, w.dY, (int)np, w.H2, (int)np, G + L.W3, nh, 0.f, 0, 1, s, sp,
                                w.part)))
        return e;
    k_rowsum<<<nout, 256, 0, s>>>(n, np, w.dY, G + L.b3);
    if ((e = tc_layer(w.op[3], nh, nout, np, w.dY, w.dZ2, GEMM_ACT_BACK, nullptr, nullptr, w.Z2, 0, w.err, s)))
        return e;
    // layer 2: dW2 = dZ2 bf16(H1)^T, db2, dZ1 = (W2^T dZ2) gelu'(Z1)
    if ((e = sgemm<false, true>(nh, nh, (int)n, w.dZ2, (int)np, w.H1, (int)np, G + L.W2, nh, 0.f, 0, 1, s, sp,
                                w.part)))
        return e;
    k_rowsum<<<nh, 256, 0, s>>>(n, np, w.dZ2, G + L.b2);
    if ((e = tc_layer(w.op[4], nh, nh, np, w.dZ2, w.dZ1, GEMM_ACT_BACK, nullptr, nullptr, w.Z1, 0, w.err, s)))
        return e;
    // layer 1: dW1 = dZ1 bf16(X)^T, db1
    if ((e = sgemm<false, true>(nh, nin, (int)n, w.dZ1, (int)np, w.X, (int)np, G + L.W1, nin, 0.f, 0, 1, s, sp,
                                w.part)))
        return e;
    k_rowsum<<<nh, 256, 0, s>>>(n, np, w.dZ1, G + L.b1);
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
