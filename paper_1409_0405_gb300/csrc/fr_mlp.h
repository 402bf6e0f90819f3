// Internal interface of the learned-closure MLP kernels (see fr_mlp.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fr_kernels.h"

namespace fr {

struct MlpLayout {
    int64_t W1, b1, W2, b2, W3, b3, n;  // offsets into the FP32 parameter vector
};
MlpLayout mlp_layout(int nin, int nh, int nout);
// floats of scratch a call on n samples needs
int64_t mlp_workspace_floats(int nin, int nh, int nout, int64_t n);
// The workspace of n samples (npad = n rounded up to 4): a status word (an
// int, non-zero if a tensor-core wait gave up), then feature-major arrays of
// npad columns: X [nin], Z1, H1, Z2, H2, dZ2, dZ1 [nh], Y, dY, T [nout]; the
// bf16 images of W1, W2, W3, W3^T, W2^T; the split-K partials.
struct MlpWs {
    int64_t npad = 0;
    int *err = nullptr;
    float *X = nullptr, *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
    float *Y = nullptr, *dY = nullptr, *T = nullptr, *part = nullptr;
    uint8_t *img[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    TcOperator op[5];
};
MlpWs mlp_ws(int nin, int nh, int nout, int64_t n, float *ws);
// packs W1, W2, W3 of the parameter vector P into the workspace's images
cudaError_t mlp_pack_forward(int nin, int nh, int nout, const float *P, MlpWs &w, cudaStream_t s);
// the closure's use of the output: add = rfs + scale_var * y in the FR
// layout [point][var][element] (nu points, ne elements, np columns)
struct ClosureOut {
    double *add = nullptr;
    const double *rfs = nullptr;
    int nu = 0;
    int64_t ne = 0;
    double scale[5] = {0, 0, 0, 0, 0};
};
// the forward pass on feature-major X [nin][np] into Y [nout][np] (or, with
// cl, straight into the RHS correction) with the packed images of w (H1, H2
// and, with keep_z, Z1, Z2 in w); *err (device) is set if a bounded wait of
// the tensor-core kernel gave up
cudaError_t mlp_forward_fm(int nin, int nh, int nout, int64_t np, const float *X, const float *P, float *Y,
                           const MlpWs &w, bool keep_z, int *err, cudaStream_t s, const ClosureOut *cl = nullptr);
// Y (n x nout) = MLP(X (n x nin)); ws holds the activations afterwards
cudaError_t mlp_forward(int nin, int nh, int nout, int64_t n, const float *X, const float *P, float *Y, float *ws,
                        cudaStream_t s);
// G = dL/dP of L = mean (MLP(X) - T)^2; loss[0] = L (device)
cudaError_t mlp_grad(int nin, int nh, int nout, int64_t n, const float *X, const float *T, const float *P, float *G,
                     float *loss, float *ws, cudaStream_t s);
// one Adam step (beta 0.9/0.999, eps 1e-8) on the FP32 master parameters
cudaError_t mlp_adam(int64_t n, float *P, const float *G, float *m, float *v, int step, float lr, cudaStream_t s);

}  // namespace fr
