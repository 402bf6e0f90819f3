// Launch interface of the FR engine's CUDA kernels (internal).
//
// Every kernel of the right-hand side is templated on its arithmetic type T
// (double for FR_FP64, float for FR_FP32: Table 1 lists single and double
// precision).  The RK registers, the reference-flux correction and the
// reductions are double in both modes.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include <vector>

#include "../../include/fr.h"

#ifndef FR_NT_DEFINED
#define FR_NT_DEFINED
namespace fr {
constexpr int NT = FR_NTYPES;  // element types: tet, prism, hex
}
#endif

namespace fr {

// Epilogues of the operator application C <- A [B1; B2] (Sec. 2.1, Eq. 1).
enum GemmMode {
    GEMM_STORE = 0,  // C = A B (+ uref[variable] with add_ref)
    GEMM_GRAD = 1,   // rows (j, d): C(j, m) = (1/J) sum_d S[d][m] (A B)(j, d)
    GEMM_DIV = 2,    // C(j) = -(1/J_j) (A B)(j) + rfs
    GEMM_DIV_RK = 3,  // r = -(1/J)(A B) + rfs; fused RK4 register update
    // the learned closure's network layers (tensor-core kernel only), on
    // feature-major activations [row][column = sample]:
    GEMM_BIAS_ACT = 4,  // Z = A B + bias[row] (stored if Z), C = act ? gelu(Z) : Z
    GEMM_ACT_BACK = 5   // C = (A B) * gelu'(Zin[row][column])
};

// The operator kernel's staged chunk of A keeps the RC values of one column k in a row padded
// to whole 16-byte vectors (rc_pad values), so that a thread loads them with
// vector loads (4 floats or 2 doubles each) instead of one load per value.
__host__ __device__ constexpr int rc_pad(int rc, int tsize) {
    return (rc * tsize + 15) / 16 * 16 / tsize;
}

// shared memory of one block: a dense chunk (rows padded, all K columns) or
// a compressed one (lmax listed columns and their column numbers)
inline size_t gemm_block_smem(int rc, int tsize, int K, int lmax) {
    const size_t row = (size_t)rc_pad(rc, tsize) * tsize;
    return lmax > 0 ? (size_t)lmax * (row + sizeof(int)) : (size_t)K * row;
}

template <typename T>
struct GemmArgsT {
    int M = 0;            // rows of A and C
    int64_t N = 0;        // columns of B and C
    int K1 = 0, K2 = 0;   // A = [A1 | A2], B = [B1; B2]
    const T *A = nullptr;  // M x (K1 + K2), row-major
    const T *B1 = nullptr;
    int64_t ldb1 = 0;
    const T *B2 = nullptr;
    int64_t ldb2 = 0;
    T *C = nullptr;
    int64_t ldc = 0;
    int mode = GEMM_STORE;
    int64_t np = 0;             // element stride: column n belongs to element n % np
    const T *invJ = nullptr;    // [nu][np] ([np] when geo_elem)
    int geo_elem = 0;           // the tensor-core GEMM_DIV epilogue: 1/J per element
    const T *S = nullptr;       // [nu][9][np]
    // GEMM_DIV_RK: with r the RHS,
    //   rk_first: Uacc = U + c_acc r,  else Uacc += c_acc r
    //   !rk_last: Us = U + c_stage r - uref;  rk_last: U = Uacc + c_acc r, Us = U - uref
    //   with Us0 (FP32 storage): stages 2-3's Us = Us0 + c_stage r in T, Us0
    //   the step's centred start state (copied from Us at the first stage)
    double *U = nullptr, *Uacc = nullptr;
    T *Us = nullptr, *Us0 = nullptr;
    double c_acc = 0, c_stage = 0;
    int rk_first = 0, rk_last = 0;
    // centring: the stage input Us holds u - uref (uref = the far-field
    // conserved state, one value per variable; column n has variable
    // n / np).  GEMM_STORE with add_ref adds uref back.
    int add_ref = 0;
    double uref[5] = {0, 0, 0, 0, 0};
    // GEMM_DIV(_RK): constant field added to r (the discrete divergence of
    // the subtracted reference flux, see Phys::fref); may be null
    const double *rfs = nullptr;
    // Optional chunk-compressed A (sp_rc > 0, used instead of A): the rows
    // in chunks of sp_rc; chunk c lists, in increasing order, the columns
    // in which any of its rows is non-zero: sp_cols[sp_off[2c] ..
    // sp_off[2c+2]), those below K1 first (up to sp_off[2c+1]); its values
    // are sp_vals[(i) * sp_rc + r] for list entry i (global index) and row
    // m0 + r (zero past M).  The other columns of the chunk are all zero, so
    // the result is that of the dense A.  sp_lmax bounds a chunk's list.
    int sp_rc = 0, sp_lmax = 0;
    const int *sp_off = nullptr, *sp_cols = nullptr;
    const T *sp_vals = nullptr;
    // sp_masked (with sp_rc == 3): each list entry is k | mask << 24, mask
    // bit r set when row m0 + r is non-zero in column k; only those FMAs run
    int sp_masked = 0;
    // GEMM_BIAS_ACT / GEMM_ACT_BACK (float): per-row bias, the stored
    // pre-activation Z (may be null) and its ldc-strided input Zin
    const float *bias = nullptr;
    float *Z = nullptr;
    const float *Zin = nullptr;
    int act = 0;
    // GEMM_BIAS_ACT, the closure's output layer inside the RHS: instead of
    // C, write the FP64 correction rfs + cl_scale[var] (A B + bias) to
    // cl_add in the FR layout [point][var][element] (output row
    // var * cl_nu + point; rfs may be null; elements >= cl_ne get rfs only)
    double *cl_add = nullptr;
    int cl_nu = 0;
    int64_t cl_ne = 0;
    double cl_scale[5] = {0, 0, 0, 0, 0};
};
using GemmArgs = GemmArgsT<double>;

template <typename T>
cudaError_t launch_gemm(const GemmArgsT<T> &g, cudaStream_t s);
// host: chunk-compressed form of a row-major M x (K1 + K2) operator for
// launch_gemm (see GemmArgsT::sp_*).  Picks the chunk size among the
// instantiated ones (a multiple of 3 if mult3; only only_rc if non-zero)
// that needs the fewest FMAs; returns 0 (use the dense operator) unless
// that saves at least 20%.
struct SparseOp {
    int rc = 0, lmax = 0;
    std::vector<int> off, cols;
    std::vector<double> vals;
};
int sparse_pack(const double *A, int M, int K1, int K2, bool mult3, SparseOp &out, int only_rc = 0);
// the masked form (chunks of 3 rows, a row mask per listed column): the
// FMAs executed are exactly the operator's non-zeros; 0 unless that saves
// at least 20% of the dense FMAs
int sparse_pack_masked(const double *A, int M, int K1, int K2, SparseOp &out);
inline cudaError_t launch_gemm_f64(const GemmArgs &g, cudaStream_t s) { return launch_gemm<double>(g, s); }

// Grouped persistent GEMM over ndesc device-resident descriptors; begin
// (device, ndesc) holds each descriptor's first block index, total the
// block count, for the row-chunk size rc (one of kGroupedRCs; GEMM_GRAD
// needs a multiple of 3); maxK bounds K1+K2; grid = persistent CTAs.
extern const int kGroupedRCs[6];
int64_t gemm_blocks(int M, int64_t N, int rc);
// sets the shared-memory attribute of every grouped instantiation (call
// before capturing grouped launches in a CUDA graph)
template <typename T>
cudaError_t configure_gemm_grouped();
template <typename T>
cudaError_t launch_gemm_grouped(const GemmArgsT<T> *descs, const int64_t *begin, int ndesc, int64_t total, int mode,
                                int rc, int maxK, int grid, cudaStream_t s);

// An operator packed for the tensor-core kernel: device image [hi | lo] of
// bf16 values in K-major core matrices (8 rows x 8 K values, 128 B; per
// 16-wide K step the Nmma/8 row groups x 2 K halves), rows padded to Nmma
// (a multiple of 16, <= 256) and each operand block's columns to a multiple
// of 16.
// The columns of the second operand block start at K1pad (a multiple of 16).
// tf32: split TF32 image, stage-major: per 16-wide K stage the slab
// [hi | lo], each Nmma/8 row groups x 4 K core matrices x 8 rows x 4 values.
// hi_only: BF16 operands (the network layers): the image holds only the hi
// half, the kernel rounds the state to bf16 (round to nearest even) and
// issues one MMA per K step, A_hi B_hi (FP32 accumulation).
struct TcOperator {
    const uint8_t *img = nullptr;
    int M = 0, K = 0, Nmma = 0, K1pad = 0, Kpad = 0, tf32 = 0, hi_only = 0;
};
// bytes of a hi-only image of an M x K operator (rows padded to 16, K to 16)
size_t tc_hi_image_bytes(int M, int K);
// device: packs the FP32 matrix W (rows x cols, row stride ldw) as the
// operator W, or W^T when trans (then the operator is cols x rows), into a
// hi-only image at img (tc_hi_image_bytes of the operator's shape) and fills
// op's sizes
cudaError_t tc_pack_hi(const float *W, int rows, int cols, int ldw, int trans, uint8_t *img, TcOperator &op,
                       cudaStream_t s);
// packs a row-major FP64 operator (M x (K1 + K2)) into the image layout (host)
void tc_pack(const double *A, int M, int K1, int K2, std::vector<uint16_t> &img, int &Nmma, int &K1pad, int &Kpad);
void tc_pack_tf32(const double *A, int M, int K1, int K2, std::vector<uint32_t> &img, int &Nmma, int &K1pad,
                  int &Kpad);
int tc_stages(const TcOperator &op);
size_t tc_smem_bytes(const TcOperator &op);
// C <- A [B1; B2] with g's epilogue on the tensor cores; *err (device) is set
// non-zero if a bounded wait of the kernel gave up.  no_producer (the
// bounded-wait self-test only): the state loads are never issued, so every
// wait runs out and the kernel takes its abort path
cudaError_t launch_gemm_tc(const GemmArgsT<float> &g, const TcOperator &op, int *err, cudaStream_t s,
                           int no_producer = 0);

// FP32 operator applications on the FP32 pipe (fr_gemm_f32.cu), the FR_FP32
// mode's operator kernel: the state streamed into shared memory by TMA
// boxes of 16 K rows x 128 columns, the operator beside it in one slab per
// 16-wide stage, and register tiles of 4 operator rows x 4 state columns
// per lane.  A 4-row block whose operator entries are all zero in a column
// of the stage skips that column (its FMAs would add exact zeros), so each
// output is the same FMA chain over k in increasing order as the
// chunk-staged kernel (fr_gemm.cu) computes: the results are bitwise equal.
// Up to 240 operator rows per pass (more rows: several passes).
constexpr int kF32RowsPerPass = 240;
struct F32Operator {
    const float *img = nullptr;      // [pass][stage][16][MP]: column 16 s + k of image row i
    const uint16_t *mask = nullptr;  // [pass][stage][MP / 4]: bit k set where the 4-row block is non-zero
    const int *rowmap = nullptr;     // [pass][MP]: output row of image row i, -1 for padding
    int M = 0, K1pad = 0, Kpad = 0, MP = 0, npass = 0;
};
// host: the image of A (M x (K1 + K2), row-major) with image row i of pass p
// holding operator row perm[p MP + i] (perm empty: the identity); fills op's
// sizes (the device pointers are the caller's to set)
void f32_pack(const double *A, int M, int K1, int K2, const std::vector<int> &perm, std::vector<float> &img,
              std::vector<uint16_t> &mask, std::vector<int> &rowmap, F32Operator &op);
// C <- A [B1; B2] (GEMM_STORE epilogue, with add_ref) on the FP32 pipe;
// *err (device) is set non-zero if a bounded wait of the kernel gave up.
// no_producer (the bounded-wait self-test only): the copies are never
// issued, so every wait runs out and the kernel takes its abort path
cudaError_t launch_gemm_f32(const GemmArgsT<float> &g, const F32Operator &op, int *err, cudaStream_t s,
                            int no_producer = 0);

// FP64 operator applications on the tensor cores by exact splitting
// (FR_FP64S, fr_gemm_x64.cu).  Every operand value x of a row (operator) or
// column (state) whose values all lie below 2^(E - 1022) in magnitude (E
// the largest biased FP64 exponent of the row or column) is held as the
// integer X = round(x 2^(56 - (E - 1022))), |X| < 2^56, written with eight
// signed base-128 digits, X = sum_p d_p 128^(7 - p), d_0 in [-128, 128] and
// d_1..d_7 in [-64, 63]: each digit is exact in bf16.  A digit product is an
// integer below 2^14, and the sum over K of the products of one level
// (p + q = L, L = 0..7) stays below 2^24 for K <= 409, so the tensor cores
// accumulate every level exactly in FP32; the levels are combined in
// integer arithmetic and rounded once to FP64.  Operators of more than 64
// rows run as row blocks (8 levels x 64 rows fill the 512 TMEM columns).
constexpr int kX64Digits = 8;
constexpr int kX64MaxRows = 64;
constexpr int kX64MaxK = 409;
struct X64Operator {
    // [row block][16-wide stage][digit q]: Nmma x 16 bf16 in K-major core
    // matrices (8 rows x 8 values; K halves 128 B apart, row groups 256 B)
    const uint8_t *img = nullptr;
    const int *rexp = nullptr;  // per operator row: largest biased exponent (0: the row is zero)
    int M = 0, K1 = 0, K2 = 0, K1pad = 0, Kpad = 0;
    int rows = 0;  // operator rows per row block (a multiple of 3 for GEMM_GRAD)
    int nrb = 0;   // row blocks
    int Nmma = 0;  // rows padded to 16 (the MMA's N)
    // bit L set: the level-L sums may reach 2^22 in magnitude (K 2^14 for
    // L = 0, K 2^12 (L + 3) above), past the float-to-integer shortcut
    uint32_t wide = 0;
};
// host: digits of a row-major M x (K1 + K2) FP64 operator in row blocks of
// at most kX64MaxRows rows (whole points, 3 rows each, if mult3); fills op's
// sizes (the device pointers are the caller's to set); false if K1 + K2
// exceeds kX64MaxK
bool x64_pack(const double *A, int M, int K1, int K2, bool mult3, std::vector<uint16_t> &img,
              std::vector<int> &rexp, X64Operator &op);
// the pre-pass: for every column n of [B1; B2] (N columns), the largest
// biased exponent of its values (0 if all are zero, 2047 if one is not finite)
cudaError_t launch_colexp(const double *B1, int64_t ldb1, int K1, const double *B2, int64_t ldb2, int K2, int64_t N,
                          int *E, cudaStream_t s);
// C <- A [B1; B2] with g's epilogue (GEMM_STORE with add_ref, GEMM_GRAD,
// GEMM_DIV, GEMM_DIV_RK; FP64 registers), E from launch_colexp of the same
// B; *err (device) is set non-zero if a bounded wait of the kernel gave up.
// no_producer (the bounded-wait self-test only): the copies are never
// issued, so every wait runs out and the kernel takes its abort path
cudaError_t launch_gemm_x64(const GemmArgsT<double> &g, const X64Operator &op, const int *E, int *err,
                            cudaStream_t s, int no_producer = 0);
// shared memory the kernel takes for op (0: the operator does not fit)
size_t x64_smem_bytes(const X64Operator &op);

struct Phys {
    double gamma, mu, prandtl, beta, tau;
    double rho_inf, vinf[3], p_inf, t_wall;
    int viscous;
    // inviscid flux of the far-field state, subtracted from every volume
    // and common flux before the divergence, which removes the cancellation
    // of the large constant pressure flux at low Mach number.  The discrete
    // divergence of this constant flux would vanish with exact geometry; with
    // the geometric factors rounded to double it is ~1e-11, so it is
    // evaluated once at set-up and added back (GemmArgs::rfs).
    double fref[5][3];
    // the far-field conserved state; the stage input is stored relative to it
    double uref[5];
};

// Index of the halo pseudo-type: in a partition of a partitioned mesh, an
// interface pair whose other side lies in another partition refers to that
// side as (HALO, flux point 0, halo slot).  The halo arrays hold the other
// partition's flux-point values ([V][np] and [3][V][np] with one "flux
// point"); what the face kernels write to the halo side lands in scratch.
constexpr int HALO = NT;

// Per-type field pointers (index 0 tet, 1 prism, 2 hex, HALO the halo);
// nullptr for an absent type.
template <typename T>
struct FieldsT {
    const T *UF[NT + 1];   // [nf][V][np]
    T *DUF[NT + 1];        // [nf][V][np]
    const T *GUF[NT + 1];  // [nf][3][V][np]
    T *FC[NT + 1];         // [nf][V][np]
    int64_t np[NT + 1];
};
using Fields = FieldsT<double>;

// Interface flux-point pairs: sides, side a's unit normal, both |S^T n^|,
// the LDG switch (+1 where side a is the left side), and (FP32-storage
// modes) float copies of the normal and magnitudes, rounded once on the host.
// The two sides' element types, flux-point numbers and the switch share one
// 32-bit word per pair (pair_code), the element numbers are ea, eb.
struct Pairs {
    int64_t n;
    const uint32_t *code;
    const int *ea, *eb;
    const double *nrm, *maga, *magb;
    const float *nrm_f, *maga_f, *magb_f;
};
// bits 0-1 type a, 2-3 type b (0..3: the element types and the halo),
// 4-12 flux point a, 13-21 flux point b (< 512), 22: the switch is +1
constexpr int kPairMaxFpt = 512;
__host__ __device__ inline uint32_t pair_code(int ta, int tb, int fa, int fb, int sgn) {
    return (uint32_t)ta | (uint32_t)tb << 2 | (uint32_t)fa << 4 | (uint32_t)fb << 13 | (uint32_t)(sgn > 0) << 22;
}
struct PairSides {
    int ta, tb, fa, fb, sgn;
};
__host__ __device__ inline PairSides pair_sides(uint32_t c) {
    return PairSides{(int)(c & 3u), (int)(c >> 2 & 3u), (int)(c >> 4 & 511u), (int)(c >> 13 & 511u),
                     (c >> 22 & 1u) ? 1 : -1};
}

struct Bnd {
    int64_t n;
    const int *bt, *bf, *be, *btag;
    const double *bn, *bmag;
    const float *bn_f, *bmag_f;
};

template <typename T>
cudaError_t launch_common_solution(const Pairs &P, const Bnd &B, const FieldsT<T> &F, const Phys &ph,
                                   cudaStream_t s);
template <typename T>
cudaError_t launch_common_flux(const Pairs &P, const Bnd &B, const FieldsT<T> &F, const Phys &ph,
                               cudaStream_t s);
// diagnostics: per-block partial sums (nblocks x 1, nblocks x 6) of the
// kinetic-energy rate sum w J (v.R_m - |v|^2/2 R_rho) over one type and of
// the wall force (inviscid xyz, viscous xyz) over the wall boundary points
// (bw: face weight of each boundary point); launch_sum_partials adds the
// nblocks rows of nq (<= 32) values into out
template <typename T>
cudaError_t launch_ke_rate(int nu, int64_t ne, int64_t np, const double *U, const T *R, const double *wJ,
                           double *partial, int nblocks, cudaStream_t s);
template <typename T>
cudaError_t launch_wall_force(const Bnd &B, const double *bw, const FieldsT<T> &F, const Phys &ph, double *partial,
                              int nblocks, cudaStream_t s);
cudaError_t launch_sum_partials(const double *partial, int nblocks, int nq, double *out, cudaStream_t s);
// transformed flux at the solution points of one type; U is the centred
// stage input (u - uref).  invJ non-null: GU holds the reference gradient
// (rows (j, d)) on entry and receives the physical gradient (rows (j, m)).
// gj = 1: S [nu][9][np] and invJ [nu][np] per point; gj = 0: per element
// ([9][np], [np]), for a type whose geometry factors are point-invariant
template <typename T>
cudaError_t launch_flux(int nu, int64_t ne, int64_t np, const T *U, T *GU, const T *S, const T *invJ, T *FT,
                        const Phys &ph, cudaStream_t s, int gj = 1);
// public [e][v][j] (double) -> internal [j][v][e]: `in` (double, may be
// null) receives the values, `centred` (T, may be null) u - uref
template <typename T>
cudaError_t launch_pub_to_int(int nu, int64_t ne, int64_t np, const double *pub, double *in, cudaStream_t s,
                              T *centred, const double *uref);
// internal [j][v][e] (T) -> public [e][v][j] (double)
template <typename T>
cudaError_t launch_int_to_pub(int nu, int64_t ne, int64_t np, const T *in, double *pub, cudaStream_t s);
// work items of the grouped point-wise launches
template <typename T>
struct FluxItem {
    int nu;
    int64_t ne, np;
    const T *U, *GU, *S;
    T *FT;
    const T *invJ;  // non-null: GU holds the reference gradient (see launch_flux)
};
template <typename T>
struct FaceItem {
    Pairs P;
    Bnd B;
    FieldsT<T> F;
};
template <typename T>
struct CenterItem {
    int64_t n, np;  // n = nu * V * np
    const double *U;
    T *Us;
    double uref[5];
};
// grouped launches over device-resident items; begin[i] = first global
// index of item i (prefix sums of nu*np, pairs+boundary points, n)
template <typename T>
cudaError_t launch_flux_grouped(const FluxItem<T> *items, const int64_t *begin, int n, int64_t total, const Phys &ph,
                                int grid, cudaStream_t s, bool xform = false);
// which = 0: common solution, 1: common flux
template <typename T>
cudaError_t launch_face_grouped(const FaceItem<T> *items, const int64_t *begin, int n, int64_t total, const Phys &ph,
                                int which, int grid, cudaStream_t s);
template <typename T>
cudaError_t launch_center_grouped(const CenterItem<T> *items, const int64_t *begin, int n, int64_t total, int grid,
                                  cudaStream_t s);
// One RK stage of a batch as one persistent cooperative launch: the phases
// run in order, separated by grid-wide barriers whose waits are bounded.
// A phase holds a grouped operator application (descriptor list as for
// launch_gemm_grouped, with its row-chunk size rc and mode) and/or
// point-wise work (flux items; face items with which = 0 common solution,
// 1 common flux) that does not depend on it.
template <typename T>
struct StagePhase {
    const GemmArgsT<T> *descs = nullptr;
    const int64_t *begin = nullptr;
    int ndesc = 0, mode = 0, rc = 0, maxK = 0;
    int64_t total = 0;
    const FluxItem<T> *fitems = nullptr;
    const int64_t *fbegin = nullptr;
    int fn = 0, xform = 0;
    int64_t ftotal = 0;
    const FaceItem<T> *citems = nullptr;
    const int64_t *cbegin = nullptr;
    int cn = 0, which = 0;
    int64_t ctotal = 0;
};
constexpr int kMaxStagePhases = 8;
// row-chunk sizes of the batched engine (both schedules): 6, 8 or 12; the
// persistent stage kernel is compiled for these only (register budget)
constexpr int kMaxBatchRC = 12;
template <typename T>
struct StagePlan {
    StagePhase<T> ph[kMaxStagePhases];
    int nph = 0;
};
// error code a barrier wait that ran out writes to *err
constexpr int kStageTimeout = 11;
// the largest co-resident grid of the stage kernel for this plan (viscous:
// the Navier-Stokes instantiation, else the Euler one)
template <typename T>
cudaError_t stage_grid(const StagePlan<T> &plan, int viscous, int *grid);
// bar: 2 device words (arrivals, generation), zero before the first launch;
// err: device int (0: fine; set to kStageTimeout when a wait runs out, after
// which every later stage launch returns at once).  skip_block >= 0 (the
// bounded-wait self-test only): that CTA takes no part, so the first
// barrier's waits run out and the kernel returns with the error set.
template <typename T>
cudaError_t launch_stage(const StagePlan<T> &plan, const Phys &ph, unsigned *bar, int *err, int skip_block, int grid,
                         cudaStream_t s);
// transformed reference flux at solution points, FT = S F_ref (padding 0)
cudaError_t launch_const_flux(int nu, int64_t ne, int64_t np, const double *S, double *FT, const Phys &ph,
                              cudaStream_t s);
// reference normal flux at every flux point, FC = F_ref.n |S^T n^|
cudaError_t launch_const_common(const Pairs &P, const Bnd &B, const Fields &F, const Phys &ph, cudaStream_t s);
// Us = U - uref over a whole [nu][V][np] register
template <typename T>
cudaError_t launch_center(int nu, int64_t np, const double *U, T *Us, const double *uref, cudaStream_t s);
// RK4 register update (the GEMM_DIV_RK epilogue) from a stored RHS R
// [nu][V][np]: see GemmArgsT for c_acc, c_stage, first, last.  invJ
// non-null: R is the raw product of the divergence operator, and the RHS
// is -(1/J) R (formed in T) plus rfs (FP64, may be null).  Us0 non-null
// (a T register): the stage inputs of stages 2-3 are formed in T from the
// step's centred start state, which the first stage copies from Us to Us0.
// gj as for launch_flux (invJ per point or per element)
template <typename T>
cudaError_t launch_rk_update(int nu, int64_t np, const T *R, double *U, double *Uacc, T *Us, const double *uref,
                             double c_acc, double c_stage, int first, int last, const T *invJ, const double *rfs,
                             T *Us0, cudaStream_t s, int gj = 1);
// low-storage (2N) RK stage: dU = a dU + dt R (dU unread when first),
// U += b dU, Us = U - uref; R [nu][V][np]
template <typename T>
cudaError_t launch_rk_2n_update(int nu, int64_t np, const T *R, double *U, double *dU, T *Us, const double *uref,
                                double a, double b, double dt, int first, cudaStream_t s);
// RK45[2R+] stage (two registers plus the error register E, which may be
// null): Us = (U - uref) + c_stage r (last: the new U - uref), U += c_acc r,
// E = (first ? 0 : E) + c_err r; R [nu][V][np]
template <typename T>
cudaError_t launch_rk_2r_update(int nu, int64_t np, const T *R, double *U, double *E, T *Us, const double *uref,
                                double c_stage, double c_acc, double c_err, int first, int last, cudaStream_t s);
// per-block partial sums (nblocks x 1) of (E / (atol + rtol |U|))^2 over one
// type's registers, element columns below ne only
cudaError_t launch_err_norm_partial(int nu, int64_t ne, int64_t np, const double *U, const double *E, double atol,
                                    double rtol, double *partial, int nblocks, cudaStream_t s);
// element-wise double -> float copy
cudaError_t launch_to_float(int64_t n, const double *src, float *dst, cudaStream_t s);
// per-block partial integrals (7 per block) of one type's register
cudaError_t launch_reduce_partial(int nu, int64_t ne, int64_t np, const double *U, const double *wJ,
                                  double gamma, double *partial, int nblocks, cudaStream_t s);
cudaError_t launch_reduce_final(const double *partial, int nblocks, double *out, cudaStream_t s);
// *flag = 1 if any solution value of the register (element columns below
// ne) is non-finite or has a non-positive density or pressure (one thread
// per point; gamma and nblocks are not needed: the pressure is positive iff
// 2 rho E > |rho v|^2 for any gamma > 1)
cudaError_t launch_state_check(int nu, int64_t ne, int64_t np, const double *U, double gamma, int *flag, int nblocks,
                               cudaStream_t s);
// measured FP64 FMA throughput (GFLOP/s) of the current device
cudaError_t probe_fp64(double *gflops, cudaStream_t s);

}  // namespace fr
