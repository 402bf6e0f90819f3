// Internal definition of the FR context (shared by the C ABI and the
// batched engine).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/fr.h"
#include "fr_internal.h"
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
    // RK45[2R+]: the embedded error estimate, and the copy of U an adaptive
    // step restores on rejection (allocated by the first call that needs them)
    double *E = nullptr, *Ubak = nullptr;   // [nu][V][np]
    double *wJ = nullptr;                   // [nu][np]
    double *Rfs = nullptr;                  // [nu][V][np]
    double *S = nullptr, *invJ = nullptr;   // [nu][9][np], [nu][np]
    double *M0 = nullptr, *AGRAD = nullptr, *ADIV = nullptr;
    // buffers in the arithmetic type of the right-hand side (double for
    // FR_FP64, float for FR_FP32; the geometry/operator views alias the
    // double arrays in FR_FP64)
    void *Us = nullptr, *R = nullptr;        // [nu][V][np]
    void *Us0 = nullptr;                     // [nu][V][np], tensor-core modes: centred step start state
    void *UF = nullptr, *DUF = nullptr, *FC = nullptr;   // [nf][V][np]
    void *GU = nullptr, *FT = nullptr;       // [nu][3][V][np]
    void *GUF = nullptr;                     // [nf][3][V][np]
    void *S_t = nullptr, *invJ_t = nullptr, *M0_t = nullptr, *AGRAD_t = nullptr, *ADIV_t = nullptr;
    // tensor-core modes: S_t and invJ_t hold one value per element ([9][np],
    // [np]) when every element's float geometry factors are the same at all
    // of its solution points (straight-sided affine elements)
    int geo_elem = 0;
    std::vector<double> xu;  // host: ne x nu x 3 physical solution points
    // learned closure (off unless cl_on): FP32 parameters of the network
    // (20 nu -> cl_nh -> cl_nh -> 5 nu), its features/outputs/activations,
    // and the FP64 field the divergence epilogue adds (Rfs + correction)
    int cl_on = 0, cl_nh = 0;
    double cl_scale[5] = {0, 0, 0, 0, 0};  // per conserved variable
    float *cl_P = nullptr, *cl_X = nullptr, *cl_Y = nullptr, *cl_ws = nullptr;
    double *cl_add = nullptr;
    int64_t cl_cap_nh = 0;  // hidden width the buffers were sized for
    fr::TcOperator cl_op[3];  // the layers' bf16 weight images (in cl_ws)
    // FR_BF16X3 / FR_TF32X3: the packed operators M0, AGRAD, ADIV for the
    // tensor cores
    fr::TcOperator tc[3];
    // an operator with more rows than one tensor-core tile takes (the p=4
    // hex gradient): rows [0, tc_split) in tc[w], the rest in tc2[w]
    fr::TcOperator tc2[3];
    // FR_FP32: M0, AGRAD (rows ordered direction-major, so that a 4-row
    // block shares the zeros of n_d M3), ADIV for the streamed FP32 kernel
    fr::F32Operator f32op[3];
    int tc_split[3] = {0, 0, 0};
    // FR_FP64S: M0, AGRAD, ADIV for the exact-split tensor-core kernel
    // (img null: that operator stays on the FP64 FMA kernel)
    fr::X64Operator x64[3];
    // FR_FP64 / FR_FP32: chunk-compressed M0, AGRAD, ADIV (sp_rc 0: dense)
    int sp_rc[3] = {0, 0, 0}, sp_lmax[3] = {0, 0, 0}, sp_masked[3] = {0, 0, 0};
    int *sp_off[3] = {nullptr, nullptr, nullptr}, *sp_cols[3] = {nullptr, nullptr, nullptr};
    void *sp_vals[3] = {nullptr, nullptr, nullptr};  // double or float
};

struct fr_ctx {
    fr_params prm{};
    int order = 0;
    int device = 0;
    DevType T[fr::NT];  // tets, prisms, hexes
    int64_t npairs = 0, nbnd = 0;
    uint32_t *pcode = nullptr;  // pair_code of each pair (types, flux points, LDG switch)
    int *ea = nullptr, *eb = nullptr;
    double *nrm = nullptr, *maga = nullptr, *magb = nullptr;
    int *bt = nullptr, *bf = nullptr, *be = nullptr, *btag = nullptr;
    double *bn = nullptr, *bmag = nullptr;
    float *nrm_f = nullptr, *maga_f = nullptr, *magb_f = nullptr, *bn_f = nullptr, *bmag_f = nullptr;
    // partition of a partitioned mesh: halo slots (other partitions' flux
    // points on cut interfaces), padded to nhalo_p, in the RHS arithmetic
    // type: UF_h [V][nhalo_p], GUF_h [3][V][nhalo_p] (received), DUF_h and
    // FC_h (scratch for the face kernels' writes to the remote side)
    int64_t nhalo = 0, nhalo_p = 0;
    void *UF_h = nullptr, *GUF_h = nullptr, *DUF_h = nullptr, *FC_h = nullptr;
    double *red = nullptr;  // reduction partials + result
    double *bw = nullptr;    // face weight of each boundary flux point
    double *diag = nullptr;  // diagnostics partials + result
    int *tc_err = nullptr;  // set by a tensor-core kernel whose bounded wait gave up
    // FR_FP64S: the column exponents of the state operand of the current
    // operator application (launch_colexp), 15 np of the largest type
    int *x64_E = nullptr;
    // set (to 1) by the state check that ends every fr_step call when the
    // solution has a non-finite value or a non-positive density/pressure:
    // mapped pinned host memory, so the next fr_step reads it without a
    // synchronisation (nf_dev is its device address)
    int *nf_host = nullptr, *nf_dev = nullptr;
    int red_blocks[fr::NT] = {};
    std::vector<void *> allocs;
    // launch accounting: count of kernel launches, and (when profiling is
    // on) a CUDA event pair around every launch, tagged by kernel class
    int64_t launches = 0;
    int prof = 0;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_ev;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    // order-transfer matrices (nu_self x nu_from, FP64, device) for one
    // source order, and the scratch of the closure sample generator
    int tr_from = 0;
    double *tr[fr::NT] = {};
    double *smp_u = nullptr, *smp_r = nullptr, *smp_rr = nullptr, *smp_rhi = nullptr;
    int64_t smp_rhi_cap = 0;
};

namespace fr {
namespace api {

enum KClass { K_M0 = 0, K_COMMON_SOL, K_GRAD, K_M0_GRAD, K_FLUX, K_COMMON_FLUX, K_DIV, K_CLOSURE, K_CHECK, K_NCLASS };
// profile tag of a launch that works on one element type t: its class, and
// t in the blocks above the untyped tags (fr_profile_read_types)
inline int ktag(int kclass, int t) { return kclass + K_NCLASS * (t + 1); }

struct RKStage {
    double c_acc, c_stage;
    int first, last;
};

int set_err(int code, const std::string &msg);
// the engine's device allocations (counted; see fr_debug_fail_alloc)
cudaError_t dev_malloc(void **p, size_t bytes);
void dev_free(void *p);
int cuda_check(cudaError_t e, const char *what);
// cudaMalloc + zero fill; the context owns (and frees) the memory
int dev_alloc_bytes(fr_ctx *c, void **p, size_t bytes);
cudaEvent_t next_event(fr_ctx *c);
// Launch through `fn` (which issues `nk` kernels), counting the launches
// and, when profiling, timing them with an event pair on the stream.
template <class F>
cudaError_t launch(fr_ctx *c, int kclass, cudaStream_t s, F fn, int nk = 1) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (c->prof) {
        a = next_event(c);
        b = next_event(c);
        if (a && b) cudaEventRecord(a, s);
    }
    cudaError_t e = fn();
    c->launches += nk;
    if (c->prof && a && b) {
        cudaEventRecord(b, s);
        c->prof_ev.push_back({kclass, {a, b}});
    }
    return e;
}
int64_t ndof_of(const fr_ctx *c);
// multiprocessors of the context's device (cudaDevAttrMultiProcessorCount)
int num_sms(int device);
// FR_ERR_NONFINITE if an earlier step's state check found a bad state
int step_guard(const fr_ctx *c);
// the state check of the solution register (one launch per element type)
int step_check(fr_ctx *c, cudaStream_t s);
// FP32 storage (FR_FP32, FR_BF16X3, FR_TF32X3) rather than FP64 (FR_FP64,
// FR_FP64S)
inline bool f32_storage(int precision) { return precision != FR_FP64 && precision != FR_FP64S; }
inline bool is_f32(const fr_ctx *c) { return f32_storage(c->prm.precision); }
// FP64 with exact-split tensor-core operator products (FR_FP64S)
inline bool is_x64(const fr_ctx *c) { return c->prm.precision == FR_FP64S; }
// operator applications on the tensor cores (FR_BF16X3, FR_TF32X3)
inline bool is_tc(const fr_ctx *c) { return c->prm.precision == FR_BF16X3 || c->prm.precision == FR_TF32X3; }
// operator application `which` (0 M0, 1 AGRAD, 2 ADIV) of element type t:
// the tensor-core kernel in FR_BF16X3 / FR_TF32X3, else the FMA kernel
template <typename T>
cudaError_t op_gemm(fr_ctx *c, int t, int which, const GemmArgsT<T> &g, cudaStream_t s);
// the FP32-storage contexts keep every RHS buffer in float
template <typename T>
inline bool type_matches(const fr_ctx *c) { return is_f32(c) == (sizeof(T) == sizeof(float)); }
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
// one RHS on public-layout device arrays (FP64 in and out)
template <typename T>
int rhs_public(fr_ctx *c, const double *u_dev, double *r_dev, cudaStream_t s);
// the three phases of one RHS (see fr_api.cu): interpolation; common
// solution and gradients (Navier-Stokes; nothing for Euler); flux, common
// flux and divergence (with the fused RK4 update if rk is non-null)
template <typename T>
int phase_interp(fr_ctx *c, T *const in[NT], cudaStream_t s);
template <typename T>
int phase_grad(fr_ctx *c, T *const in[NT], cudaStream_t s);
template <typename T>
int phase_div(fr_ctx *c, T *const in[NT], const RKStage *rk, cudaStream_t s);
int check_params(int order, const fr_params *prm);
int host_setup(const fr_mesh *mesh, int order, HostSetup &h);
int device_setup(fr_ctx *c, int order, const fr_params *prm, const RefOps ops[NT], const TypeGeo geo[NT],
                 const Faces &faces, int64_t nhalo);
// stages 1-4 of the RHS (interpolation and, for Navier-Stokes, the
// corrected gradient at solution and flux points) on the stage input
template <typename T>
int front_stages(fr_ctx *c, T *const in[NT], cudaStream_t s);
// learned closure of type t: features of the stage input, the network,
// and cl_add = Rfs + scale * output in the internal layout
template <typename T>
int closure_apply(fr_ctx *c, int t, const T *in, cudaStream_t s);

}  // namespace api
}  // namespace fr
