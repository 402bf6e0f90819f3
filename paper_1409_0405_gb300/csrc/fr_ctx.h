// Internal definition of the FR context (shared by the C ABI and the
// batched engine).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/fr.h"
#include "fr_kernels.h"

namespace fr {
constexpr int NVV = FR_NVARS;
}

struct DevType {
    int present = 0;
    int64_t ne = 0, np = 0;
    int nu = 0, nf = 0;
    // FP64 in every mode: RK registers, quadrature weights, the reference-flux
    // divergence, and the geometry/operators the set-up evaluates with
    double *U = nullptr, *Uacc = nullptr;   // [nu][V][np]
    double *wJ = nullptr;                   // [nu][np]
    double *Rfs = nullptr;                  // [nu][V][np]
    double *S = nullptr, *invJ = nullptr;   // [nu][9][np], [nu][np]
    double *M0 = nullptr, *AGRAD = nullptr, *ADIV = nullptr;
    // buffers in the arithmetic type of the right-hand side (double for
    // FR_FP64, float for FR_FP32; the geometry/operator views alias the
    // double arrays in FR_FP64)
    void *Us = nullptr, *R = nullptr;        // [nu][V][np]
    void *UF = nullptr, *DUF = nullptr, *FC = nullptr;   // [nf][V][np]
    void *GU = nullptr, *FT = nullptr;       // [nu][3][V][np]
    void *GUF = nullptr;                     // [nf][3][V][np]
    void *S_t = nullptr, *invJ_t = nullptr, *M0_t = nullptr, *AGRAD_t = nullptr, *ADIV_t = nullptr;
    std::vector<double> xu;  // host: ne x nu x 3 physical solution points
};

struct fr_ctx {
    fr_params prm{};
    int order = 0;
    int device = 0;
    DevType T[2];
    int64_t npairs = 0, nbnd = 0;
    int *ta = nullptr, *fa = nullptr, *ea = nullptr, *tb = nullptr, *fb = nullptr, *eb = nullptr;
    double *nrm = nullptr, *maga = nullptr, *magb = nullptr;
    int *bt = nullptr, *bf = nullptr, *be = nullptr, *btag = nullptr;
    double *bn = nullptr, *bmag = nullptr;
    double *red = nullptr;  // reduction partials + result
    int red_blocks[2] = {0, 0};
    std::vector<void *> allocs;
    // launch accounting: count of kernel launches, and (when profiling is
    // on) a CUDA event pair around every launch, tagged by kernel class
    int64_t launches = 0;
    int prof = 0;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_ev;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
};

namespace fr {
namespace api {

enum KClass { K_M0 = 0, K_COMMON_SOL, K_GRAD, K_M0_GRAD, K_FLUX, K_COMMON_FLUX, K_DIV, K_NCLASS };

struct RKStage {
    double c_acc, c_stage;
    int first, last;
};

int set_err(int code, const std::string &msg);
int cuda_check(cudaError_t e, const char *what);
Phys phys_of(const fr_ctx *c);
template <typename T>
FieldsT<T> fields_of(const fr_ctx *c);
Pairs pairs_of(const fr_ctx *c);
Bnd bnd_of(const fr_ctx *c);
// arguments of the operator applications of element type t (the same in
// the per-context and the grouped launches)
template <typename T>
GemmArgsT<T> args_m0(const fr_ctx *c, int t, const T *in);
template <typename T>
GemmArgsT<T> args_grad(const fr_ctx *c, int t, const T *in);
template <typename T>
GemmArgsT<T> args_m0grad(const fr_ctx *c, int t);
template <typename T>
GemmArgsT<T> args_div(const fr_ctx *c, int t, const RKStage *rk);
// nsteps RK4 steps on one context (its own launches)
template <typename T>
int step_impl(fr_ctx *c, double dt, int nsteps, cudaStream_t s);

}  // namespace api
}  // namespace fr
