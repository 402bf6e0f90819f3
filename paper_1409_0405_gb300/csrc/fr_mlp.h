// Internal interface of the learned-closure MLP kernels (see fr_mlp.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fr {

struct MlpLayout {
    int64_t W1, b1, W2, b2, W3, b3, n;  // offsets into the FP32 parameter vector
};
MlpLayout mlp_layout(int nin, int nh, int nout);
// floats of scratch a call on n samples needs
int64_t mlp_workspace_floats(int nin, int nh, int nout, int64_t n);
// Y (n x nout) = MLP(X (n x nin)); ws holds the activations afterwards
cudaError_t mlp_forward(int nin, int nh, int nout, int64_t n, const float *X, const float *P, float *Y, float *ws,
                        cudaStream_t s);
// G = dL/dP of L = mean (MLP(X) - T)^2; loss[0] = L (device)
cudaError_t mlp_grad(int nin, int nh, int nout, int64_t n, const float *X, const float *T, const float *P, float *G,
                     float *loss, float *ws, cudaStream_t s);
// one Adam step (beta 0.9/0.999, eps 1e-8) on the FP32 master parameters
cudaError_t mlp_adam(int64_t n, float *P, const float *G, float *m, float *v, int step, float lr, cudaStream_t s);

}  // namespace fr
