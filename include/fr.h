/*
 * fr.h - C ABI of the GB300 flux-reconstruction (FR) right-hand-side engine.
 *
 * The engine evaluates the FR semi-discretisation of the compressible Euler
 * and Navier-Stokes equations (constant viscosity, Sec. 3.4) on mixed
 * prism/tetrahedral meshes (Sec. 3.3) and on hexahedral meshes (Sec. 3.2;
 * Table 2 lists tets, prisms and hexes) and advances it with classic RK4
 * (Table 1 lists Euler, RK4 and RK45 steppers).  Every operator application
 * is a constant operator matrix times a row-major state matrix,
 * C <- c1 A B + c2 C (Sec. 2.1, Eq. 1); everything else is point-wise
 * (Sec. 2.1).  All device work runs in this library's CUDA kernels on the
 * current CUDA device; there is no CPU fallback.
 *
 * Conventions shared with callers
 * -------------------------------
 * Conserved variables per point: rho, rho*u, rho*v, rho*w, E (5 values);
 * ideal gas p = (gamma-1)(E - rho|v|^2/2).
 *
 * Public state layout ("public layout"): one float64 array, tetrahedra
 * first, then prisms, then hexahedra, each block
 * [element][variable][solution point]
 * (element slowest, point fastest).  Its length is fr_ndof().
 *
 * Element vertex order: tet vertices 0..3 map to reference vertices
 * (-1,-1,-1), (1,-1,-1), (-1,1,-1), (-1,-1,1).  Prism vertices 0..2 form the
 * zeta=-1 triangle (-1,-1), (1,-1), (-1,1); vertex a+3 lies above vertex a
 * at zeta=+1.  Hex vertices 0..3 are the zeta=-1 face (-1,-1), (1,-1),
 * (1,1), (-1,1); vertex a+4 lies above vertex a at zeta=+1.  Local faces:
 * tet (0,1,2), (0,1,3), (0,2,3), (1,2,3); prism (0,1,2), (3,4,5),
 * (0,1,4,3), (1,2,5,4), (2,0,3,5); hex (0,1,2,3), (0,1,5,4), (1,2,6,5),
 * (2,3,7,6), (3,0,4,7), (4,5,6,7).
 *
 * Solution points: the Blyth-Pozrikidis barycentric set built from the p+1
 * Gauss-Legendre nodes (tet: order k, j, i slowest to fastest; prism:
 * triangle set x Gauss-Legendre in zeta, zeta slowest); hex: the
 * Gauss-Legendre tensor points, zeta slowest, xi fastest.  The paper fixes only
 * their number (Table 2).
 *
 * Errors: every int-returning call returns FR_OK (0) or a negative FR_ERR_*
 * code; nothing throws or aborts across the ABI.  fr_strerror() describes a
 * code; fr_last_error() gives the detail of the most recent failure on the
 * calling thread.
 */
#ifndef FR_H
#define FR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FR_NVARS 5
#define FR_NTYPES 3 /* element types: FR_ETYPE_TET, FR_ETYPE_PRI, FR_ETYPE_HEX */

enum {
    FR_OK = 0,
    FR_ERR_ARG = -1,        /* invalid argument (null pointer, bad size, ...) */
    FR_ERR_MESH = -2,       /* J <= 0, unmatched or non-conforming face, bad tag */
    FR_ERR_CUDA = -3,       /* a CUDA runtime call failed */
    FR_ERR_NONFINITE = -4,  /* NaN/Inf or non-positive density/pressure found */
    FR_ERR_TIMEOUT = -5,    /* a bounded device wait gave up (tensor-core kernels) */
    FR_ERR_NOMEM = -6,      /* host or device allocation failed */
    FR_ERR_UNSUPPORTED = -7 /* valid request this build does not implement */
};

enum { FR_ETYPE_TET = 0, FR_ETYPE_PRI = 1, FR_ETYPE_HEX = 2 };
enum { FR_BC_WALL = 1, FR_BC_FARFIELD = 2 };
/* Arithmetic of the operator applications (Table 1: single and double;
 * FR_BF16X3 / FR_TF32X3: FP32 storage with the operator applications on the
 * tensor cores in split BF16 or split TF32, x = r(x) + r(x - r(x)), three
 * products per pair and FP32 accumulation; FR_FP64S: FP64 everywhere, the
 * operator products of element types with dense operators formed on the
 * tensor cores from exact integer digits, each output rounded once to
 * FP64). */
enum { FR_FP64 = 0, FR_FP32 = 1, FR_BF16X3 = 2, FR_TF32X3 = 3, FR_FP64S = 4 };

typedef struct fr_ctx fr_ctx; /* opaque; owned by the library */

/* Mesh description.  All arrays are caller-owned, read during fr_create only. */
typedef struct {
    int64_t n_nodes;
    const double *xyz;    /* [n_nodes][3] node coordinates */
    int64_t n_tet;
    const int64_t *tet;   /* [n_tet][4] node ids, vertex order above */
    int64_t n_pri;
    const int64_t *pri;   /* [n_pri][6] node ids, vertex order above */
    int64_t n_hex;
    const int64_t *hex;   /* [n_hex][8] node ids, vertex order above */
    int64_t n_bface;
    const int64_t *bface; /* [n_bface][4]: etype, element, local face, bc tag */
    double period[3];     /* periodic translation per axis; 0 = not periodic */
    /* Element geometry.  geom_order 1 (or 0): straight-sided elements, the
     * maps of the vertices above.  geom_order 2: quadratically curved
     * elements (the paper's cylinder mesh is quadratically curved, Sec.
     * 3.2): per element the physical coordinates of its quadratic nodes,
     * whose reference positions are, in order:
     *   tet (10): the 4 vertices, then the midpoints of edges (0,1), (0,2),
     *     (0,3), (1,2), (1,3), (2,3);
     *   prism (18): for zeta = -1, 0, +1 in turn, the six triangle nodes
     *     (-1,-1), (1,-1), (-1,1), (0,-1), (0,0), (-1,0);
     *   hex (27): the grid {-1,0,1}^3, xi fastest, zeta slowest.
     * The map is the Lagrange interpolant of the degree-2 space of the
     * element (P2; P2(triangle) x P2(zeta); Q2) through those nodes.  The
     * vertex ids above still define the topology (face matching); faces
     * shared by two elements must carry the same node coordinates. */
    int geom_order;
    const double *tet_nodes; /* geom_order 2: [n_tet][10][3] */
    const double *pri_nodes; /* geom_order 2: [n_pri][18][3] */
    const double *hex_nodes; /* geom_order 2: [n_hex][27][3] */
} fr_mesh;

/* Gas, viscous and boundary parameters. */
typedef struct {
    double gamma;     /* ratio of specific heats */
    double mu;        /* constant dynamic viscosity (Sec. 3.4) */
    double prandtl;   /* Prandtl number */
    double ldg_beta;  /* LDG common-solution bias, switch along a fixed direction;
                         with 0.5 the common solution is one side's value and
                         the common viscous flux the other side's, and the
                         face kernels read and form only those sides */
    double ldg_tau;   /* LDG penalty on the normal flux */
    int viscous;      /* 0: Euler, 1: Navier-Stokes */
    int precision;    /* FR_FP64, or FR_FP32: operator applications and point-wise
                         work in FP32; RK registers and the reductions stay
                         FP64 (the FP64 reference-flux correction, ~1e-11,
                         is below FP32 resolution and skipped); or
                         FR_BF16X3 / FR_TF32X3: as FR_FP32 with the operator
                         applications on the tensor cores (split BF16 or
                         split TF32, FP32 accumulate); or FR_FP64S: as
                         FR_FP64, with the operator products of the types
                         whose operators are mostly non-zero (tetrahedra)
                         on the tensor cores by exact splitting: every
                         operator row and state column scaled by its
                         largest power of two, its values cut into eight
                         signed 7-bit integer digits (exact in BF16), the
                         digit products of each of eight levels summed
                         exactly in FP32, the levels combined in integer
                         arithmetic and rounded once to FP64 (error about
                         2^-56 K max|A| max|B| per output, below the FP64
                         FMA chain's) */
    double rho_inf;   /* far-field density */
    double vel_inf[3];/* far-field velocity */
    double p_inf;     /* far-field pressure */
    double t_wall;    /* wall temperature p/rho (gas constant 1) */
} fr_params;

/*
 * fr_create: validate the mesh, build points, operators (M0 of Table 2 and
 * the gradient, divergence and DG-correction operators), geometry and face
 * connectivity on the host, and upload them to the current CUDA device.
 * order: polynomial order p in 1..4 (the paper exercises p = 1..4, Sec. 3.4).
 * On success *out receives a context the caller frees with fr_destroy.
 * Errors: FR_ERR_ARG, FR_ERR_MESH, FR_ERR_NOMEM, FR_ERR_CUDA;
 * FR_ERR_UNSUPPORTED for a precision outside FR_FP64..FR_FP64S, or a
 * split-BF16 context whose resident operator image leaves no room for two
 * ring slots (hexahedra at p = 4; split TF32 streams its operators and
 * takes them; operators of more than 256 rows run as two row blocks).
 */
int fr_create(const fr_mesh *mesh, int order, const fr_params *params, fr_ctx **out);

/* Free all host and device memory of the context.  NULL is ignored. */
void fr_destroy(fr_ctx *ctx);

/* Number of float64 values of the public state layout (5 x total points). */
int fr_ndof(const fr_ctx *ctx, int64_t *ndof);

/*
 * fr_info: sizes of the context.  out (caller-owned, 11 int64) receives
 * n_tet, n_pri, order, nupts(tet), nupts(pri), nfpts(tet), nfpts(pri),
 * number of interface flux-point pairs, n_hex, nupts(hex), nfpts(hex).
 */
int fr_info(const fr_ctx *ctx, int64_t *out);

/* Physical solution-point coordinates, public layout with the variable
 * axis replaced by x, y, z (3 values per point).  xyz: host array of
 * 3*fr_ndof()/5 doubles, caller-owned.  Synchronous. */
int fr_upts(const fr_ctx *ctx, double *xyz);

/* Copy a host state in the public layout into / out of the context's
 * internal solution register.  Host arrays are caller-owned, fr_ndof()
 * doubles.  A page-locked buffer mapped into the device's address space
 * (cudaHostAlloc / cudaHostRegister with unified addressing) is read or
 * written in place by the layout kernel over the CPU-GPU link; any other
 * host buffer is copied through device memory.  The results are the same.
 * Synchronous on the given stream (NULL = legacy default). */
int fr_set_state(fr_ctx *ctx, const double *u_host, void *cuda_stream);
int fr_get_state(fr_ctx *ctx, double *u_host, void *cuda_stream);

/*
 * fr_rhs: r = R(u), the FR right-hand side du/dt of the semi-discrete
 * system, for a state given in the public layout.  u_dev and r_dev are
 * caller-owned device pointers of fr_ndof() doubles (they may not alias).
 * Asynchronous on cuda_stream (a cudaStream_t; NULL = legacy default).
 * The context's scratch buffers are shared by all calls: calls on one
 * context must not overlap in time.
 */
int fr_rhs(fr_ctx *ctx, const double *u_dev, double *r_dev, void *cuda_stream);

/*
 * fr_step: nsteps classic RK4 steps of size dt on the internal solution
 * register (set by fr_set_state).  Four RHS evaluations per step; the
 * register update is fused into the divergence operator's epilogue.
 * Asynchronous on cuda_stream; contains no host synchronisation.
 */
int fr_step(fr_ctx *ctx, double dt, int nsteps, void *cuda_stream);

/*
 * Blow-up detection of the steppers.  Every fr_step, fr_step_ls and
 * fr_step_rk45 call with nsteps > 0 ends with a state check on the device
 * that sets a flag when any solution value is non-finite or any point has a
 * non-positive density or pressure.  The flag lives in mapped pinned host
 * memory: the next stepping call reads it on entry, without synchronising,
 * and returns FR_ERR_NONFINITE (doing nothing) once a completed earlier call
 * has set it.  fr_check synchronises cuda_stream and returns
 * FR_ERR_NONFINITE if the flag is set (FR_ERR_TIMEOUT if a tensor-core
 * kernel gave up a bounded wait, else FR_OK).  fr_set_state clears the flag.
 */
int fr_check(fr_ctx *ctx, void *cuda_stream);

/*
 * fr_step_ls: nsteps steps of the five-stage fourth-order low-storage
 * (2N) Runge-Kutta scheme of Carpenter & Kennedy (1994) on the internal
 * register: per stage dU <- A_i dU + dt R(U), U <- U + B_i dU (the paper
 * advances with a low-storage scheme of this family; fr_step is classic
 * RK4).  Same registers and stream semantics as fr_step; 5 RHS per step.
 * Errors: FR_ERR_ARG (nsteps < 0 or dt NaN), FR_ERR_CUDA.
 */
int fr_step_ls(fr_ctx *ctx, double dt, int nsteps, void *cuda_stream);

/*
 * fr_step_rk45: nsteps fixed steps of RK45[2R+], the scheme the paper's runs
 * used (Sec. 3.4: "RK45[2R+]"; Table 1 lists RK45): the five-stage
 * fourth-order scheme RK4(3)5[2R+]C of Kennedy, Carpenter & Lewis (2000),
 * in two registers.  Per stage i, with k_i = R(x) the RHS of the stage
 * input x:  x <- U + dt a_i k_i (formed before U moves),
 * U <- U + dt b_i k_i, and the error register E <- E + dt (b_i - bhat_i) k_i
 * (the difference between the fourth-order solution and the embedded
 * third-order one; E holds the last step's estimate afterwards).  The
 * first call allocates E (one state-sized FP64 array owned by the
 * context); make it before any stream capture.  5 RHS per step;
 * asynchronous on cuda_stream.
 * Errors: FR_ERR_ARG (nsteps < 0 or dt not finite), FR_ERR_NOMEM, FR_ERR_CUDA.
 */
int fr_step_rk45(fr_ctx *ctx, double dt, int nsteps, void *cuda_stream);

/*
 * fr_rk45_error: weighted RMS norm of the last RK45 step's error estimate,
 * *norm = sqrt(mean over every value of the state of
 * (E / (atol + rtol |u_{n+1}|))^2) (host double).  Synchronous.
 * Errors: FR_ERR_ARG (null norm, negative tolerances, atol + rtol == 0, or
 * no RK45 step taken yet), FR_ERR_CUDA.
 */
int fr_rk45_error(fr_ctx *ctx, double atol, double rtol, double *norm, void *cuda_stream);

/*
 * fr_rk45_get_error: copy the error register E (last RK45 step) into e
 * (host, caller-owned, public layout, fr_ndof doubles).  Synchronous.
 */
int fr_rk45_get_error(fr_ctx *ctx, double *e, void *cuda_stream);

/*
 * fr_step_rk45_adaptive: advance the internal solution by exactly t_span
 * with error-controlled RK45[2R+] steps.  Each attempted step of size h
 * (the last one shortened to end at t_span) is accepted when
 * fr_rk45_error(atol, rtol) <= 1 and rejected otherwise (the solution is
 * restored from a backup register); either way the next step size is
 * h * clamp(0.9 norm^(-1/4), 0.3, 2.5).  *dt (in: first step size, out:
 * the size proposed for the next step).  stats (host, may be null):
 * [accepted, rejected].  One host synchronisation per attempted step; the
 * first call allocates the error and backup registers.
 * Errors: FR_ERR_ARG (bad arguments, or max_steps attempts before t_span),
 * FR_ERR_NONFINITE (non-finite error estimate), FR_ERR_NOMEM, FR_ERR_CUDA.
 */
int fr_step_rk45_adaptive(fr_ctx *ctx, double t_span, double atol, double rtol, double *dt, int max_steps,
                          int64_t *stats, void *cuda_stream);

/*
 * fr_reduce: integrals of the internal solution register.  out (host,
 * caller-owned, 7 doubles) receives sum_e sum_j w_j J_j u_j for the 5
 * conserved variables, the kinetic energy integral, and the number of
 * points whose state is non-finite or has non-positive density/pressure.
 * Synchronous.  Returns FR_ERR_NONFINITE (with out filled) if that count
 * is non-zero.
 */
int fr_reduce(fr_ctx *ctx, double *out, void *cuda_stream);

/*
 * fr_diagnostics: flow diagnostics of the internal solution register u.
 * Evaluates R(u), the right-hand side (as the first stage of fr_step
 * does: the same kernels and precision), then reduces in FP64:
 *   out[0]    dKE/dt = sum_e sum_j w_j J_j (v_j . R_m,j - |v_j|^2/2 R_rho,j),
 *             the rate of change of the kinetic-energy integral under the
 *             semi-discrete system (chain rule of |m|^2 / (2 rho)); the
 *             kinetic-energy dissipation rate is -out[0];
 *   out[1..3] inviscid force of the fluid on the no-slip walls (tag
 *             FR_BC_WALL): the integral over the wall faces of the momentum
 *             components of the Rusanov flux against the wall ghost state,
 *             normal pointing out of the fluid;
 *   out[4..6] viscous force on the walls: the same integral of
 *             -F_v(C_b, grad u).n + tau (u - C_b), C_b the wall's common
 *             solution (zero for Euler).
 * The face integral is sum over the wall flux points of fw |S^T n^| times
 * the value, fw the integral of the flux point's face Lagrange polynomial
 * over the reference face (fr_operator FW).  out: host, caller-owned, 7
 * doubles.  Synchronous.  Overwrites the RHS scratch (and fr_rhs's input
 * buffer), not the solution registers.  Errors: FR_ERR_ARG,
 * FR_ERR_CUDA, FR_ERR_TIMEOUT (tensor-core modes).
 */
int fr_diagnostics(fr_ctx *ctx, double *out, void *cuda_stream);

/*
 * fr_selftest_wait_timeout: failure-detection self-test of the streaming
 * operator kernels: the tensor-core kernel (FR_BF16X3 / FR_TF32X3), the
 * streamed FP32 kernel (FR_FP32) or the exact-split FP64 kernel (FR_FP64S,
 * the first element type it serves).  Launches the kernel of an element
 * type's interpolation with its copies withheld, so every bounded wait
 * inside it runs out (about 2 s); the kernel then leaves all its loops
 * (the tensor-core kernel frees its tensor memory) and reports
 * FR_ERR_TIMEOUT through the context's status.  Returns FR_OK when exactly
 * that happened, after clearing the status, so the context stays usable;
 * no GPU fault, trap or unbounded wait is involved.  Overwrites the
 * interpolation scratch.  Errors: FR_ERR_ARG, FR_ERR_UNSUPPORTED
 * (FR_FP64; FR_FP64S without a type on the tensor cores), FR_ERR_TIMEOUT (a status left by earlier work), FR_ERR_CUDA.
 */
int fr_selftest_wait_timeout(fr_ctx *ctx, void *cuda_stream);

/*
 * fr_operator: host-only query (no GPU needed) of one operator matrix the
 * engine builds for (etype, order), row-major float64.  which:
 *   0 M0   (nf x nu)        interpolation to flux points (Table 2)
 *   1 D    (3*nu x nu)      reference gradient, row (j, d), d fastest
 *   2 M3   (nu x nf)        DG correction (lift) of flux-point jumps
 *   3 AGRAD (3*nu x (nu+nf)) [D | n^ (x) M3], corrected gradient operator
 *   4 ADIV (nu x (3*nu+nf)) [M1 - M3 M2 | M3] with the divergence
 *                           M1[j][(i,d)] = D[(j,d)][i] and the normal-flux
 *                           interpolation M2[f][(i,d)] = n^_d(f) M0[f][i]
 *   5 W    (nu x 1)         quadrature weights of the solution points
 *   6 UPTS (nu x 3)         reference solution points
 *   7 FPTS (nf x 3)         reference flux points
 *   8 FNORM (nf x 3)        outward unit reference normal per flux point
 *   9 FW    (nf x 1)        face weights: integral over its reference face of
 *                           each flux point's face Lagrange polynomial
 * With out == NULL only *rows and *cols are written.  Errors: FR_ERR_ARG.
 */
int fr_operator(int etype, int order, int which, double *out, int64_t *rows, int64_t *cols);

/*
 * Launch accounting.  fr_profile(ctx, enable) resets the counters; while
 * enabled, every kernel launch of fr_rhs/fr_step is bracketed by a CUDA
 * event pair on its stream.  fr_profile_read synchronises on those events
 * and writes, per kernel class (8 entries, caller-owned arrays), the summed
 * device milliseconds and the launch counts, plus the total number of
 * kernel launches since the last reset (counted with profiling on or off).
 * Classes: 0 M0 interpolation, 1 common solution, 2 corrected gradient,
 * 3 M0 on gradients, 4 point-wise flux, 5 common normal flux,
 * 6 divergence + correction (+ RK update), 7 learned closure (features,
 * network, correction; 8 launches per element type), 8 the state check
 * that ends every fr_step / fr_step_ls / fr_step_rk45 call (one launch per
 * element type).
 */
#define FR_NKCLASS 9
int fr_profile(fr_ctx *ctx, int enable);
int fr_profile_read(fr_ctx *ctx, double *ms, int64_t *count, int64_t *launches);
/*
 * fr_profile_read_types: the same events split by element type, for the
 * launches that work on one type (the operator applications of classes
 * 0, 2, 3, 6 and the point-wise flux of class 4): ms and count are
 * caller-owned arrays of (FR_NTYPES + 1) * FR_NKCLASS entries, entry
 * [b * FR_NKCLASS + k] for class k, with block b = 0 the launches that
 * span all types (face kernels, closure, state check, the streaming RK
 * update of the FP32-storage modes) and b = 1 + etype those of one type.
 * Summing the blocks gives fr_profile_read's values.  Synchronises like
 * fr_profile_read.  Errors: FR_ERR_ARG (null argument), FR_ERR_CUDA.
 */
int fr_profile_read_types(fr_ctx *ctx, double *ms, int64_t *count);

/*
 * fr_peak_fp64: measured FP64 FMA throughput of the current device, the
 * denominator of the FP64 roofline.  Runs a kernel of independent FMA
 * chains (no memory traffic) on cuda_stream, times it with CUDA events and
 * writes GFLOP/s (2 flop per FMA) to *gflops.  Synchronous.
 */
int fr_peak_fp64(double *gflops, void *cuda_stream);

/*
 * fr_gemm_fp64s: C = A B in FP64 through the exact-split tensor-core kernel
 * of FR_FP64S (the operator application of Sec. 2.1, Eq. 1, with the store
 * epilogue), on arbitrary operands, for testing and for callers with their
 * own constant operators.  A: host, row-major M x K, M >= 1, 1 <= K <= 409
 * (the exactness bound of the level sums), finite.  B: device, row-major
 * K x N (N >= 2 even, base 16-byte aligned).  C: device, row-major M x N,
 * written.  Each C[i][n] is sum_k A[i][k] B[k][n] with an error of about
 * 2^-56 K max_k|A[i][k]| max_k|B[k][n]| (operands rounded to 56 bits below
 * their row and column maxima; the digit products summed exactly); a
 * non-finite value in a column of B gives NaN in that column of C.  All
 * arguments caller-owned; device scratch (the packed operator, column
 * exponents, status) is allocated and freed by the call.  Synchronous.
 * Errors: FR_ERR_ARG, FR_ERR_NOMEM, FR_ERR_CUDA, FR_ERR_TIMEOUT (a bounded
 * wait of the kernel gave up).
 */
int fr_gemm_fp64s(int M, int K, const double *A, int64_t N, const double *B, double *C, void *cuda_stream);

/*
 * Batched engine: many independent problems (their own meshes, element
 * mixes and orders, the same fr_params) advanced together.  Every operator
 * application and point-wise pass of all problems and element types is a
 * device work list.  An RK stage of the whole batch runs either as ONE
 * persistent cooperative launch (the stage's phases in order, separated by
 * grid-wide barriers whose waits are bounded) or as one grouped launch per
 * operator class and point-wise kernel; one RK step is captured in a CUDA
 * graph.  The results are bit-identical to advancing each problem on its
 * own.
 *
 * fr_batch_create: builds nprob contexts (meshes[i], orders[i], *params) and
 *   the work lists.  Errors as fr_create.
 * fr_batch_problem: the context of problem i (owned by the batch: use it with
 *   fr_set_state / fr_get_state / fr_rhs / fr_reduce, never fr_destroy).
 * fr_batch_tune: times the candidate row-chunk sizes (the operator blocks'
 *   tile shapes, used by both schedules) and the grids of every grouped
 *   launch on this batch and keeps the fastest (leaves the solution
 *   registers untouched).  Synchronous.
 * fr_batch_step: nsteps RK4 steps, dt[i] for problem i (host array of
 *   nprob).  batched == 1: one persistent launch per RK stage (4 per step);
 *   batched == 2: the grouped launches per class; both replayed from a CUDA
 *   graph (captured on first use and after tuning, a change of dt or of the
 *   schedule); batched == 0: each problem's own launch sequence, one after
 *   another (the comparison).  Asynchronous on cuda_stream.
 * fr_batch_check: synchronises and returns FR_ERR_TIMEOUT if a barrier wait
 *   of the persistent stage kernel ran out (its status is then cleared and
 *   the batch stays usable; the steps since then did no work), else FR_OK.
 * fr_batch_selftest_wait_timeout: failure-detection self-test: one stage of
 *   the persistent kernel, without its register update, launched with one
 *   CTA withheld from the barriers, so every other CTA's bounded wait runs
 *   out (about 2 s).  FR_OK if that timeout was reported (and cleared).
 * fr_batch_info: out (14 int64): nprob, total DOF, launches per step of the
 *   last captured graph, launches per step of the per-problem sequence, the
 *   tuned row-chunk sizes (M0, gradient, M0 on gradients, divergence) and
 *   grids (GEMM, divergence, flux, face kernels), the persistent stage
 *   kernel's grid (0 before its first use), launches per step of the
 *   grouped schedule (0 before its first use).
 */
typedef struct fr_batch fr_batch;
int fr_batch_create(int nprob, const fr_mesh *meshes, const int *orders, const fr_params *params, fr_batch **out);
void fr_batch_destroy(fr_batch *b);
int fr_batch_problem(fr_batch *b, int i, fr_ctx **ctx);
int fr_batch_tune(fr_batch *b, void *cuda_stream);
int fr_batch_step(fr_batch *b, const double *dt, int nsteps, int batched, void *cuda_stream);
int fr_batch_check(fr_batch *b, void *cuda_stream);
int fr_batch_selftest_wait_timeout(fr_batch *b, void *cuda_stream);
int fr_batch_info(const fr_batch *b, int64_t *out);

/*
 * ---- Partitioned meshes ---------------------------------------------------
 * Sec. 2.5: multi-node runs split the mesh into partitions whose ranks
 * exchange interface data; Sec. 5.2: a mixed mesh is partitioned with
 * per-type weights hex : pri : tet = 3 : 2 : 1, avoiding partitions with
 * only a few (fewer than about a thousand) elements of a type.  Here the
 * partitions of one mesh live on the current device as partition
 * contexts; per RHS evaluation they exchange, through device-local
 * buffers, the flux-point states of the cut faces after the interpolation
 * and (Navier-Stokes) the flux-point gradients after their interpolation.
 * Every cut interface pair keeps its global data, so the result equals the
 * unpartitioned mesh's (bit for bit in FP64; see the tests).
 */
typedef struct fr_part fr_part; /* opaque; owned by the library */

/*
 * fr_partition (host only, no GPU): weighted recursive coordinate bisection
 * of the element centroids into nparts parts.  weights (may be null:
 * tet 1, prism 2, hex 3, the paper's 1 : 2 : 3) gives the cost of a tet, a
 * prism and a hex.  part (host, caller-owned, n_tet + n_pri + n_hex
 * int32) receives each element's partition in public order (tets, then
 * prisms, then hexes).  Deterministic.
 * Errors: FR_ERR_ARG (null pointers, nparts < 1, more partitions than
 * elements, non-positive weights), FR_ERR_MESH (node id out of range).
 */
int fr_partition(const fr_mesh *mesh, int nparts, const double *weights, int32_t *part);

/*
 * fr_part_plan (host only, no GPU): the exchange plan of partition `rank`
 * for the partition array part (as fr_partition writes it).  A partition's
 * local element numbering is its elements of each type in increasing
 * global order.  counts (host, nparts int64): the number of flux points
 * rank sends to each partition, which equals the number it receives from
 * it.  send_pts (may be null; sum(counts) x 3 int32): rank's flux points
 * (etype, local element, flux point), grouped by destination in
 * increasing order, each group in the order of the mesh's interface pairs.
 * halo_pts (may be null; sum(counts) x 3 int32): for each of rank's halo
 * slots, the remote flux point (etype, global element, flux point),
 * grouped by source in increasing order: slot i of the group from q
 * receives entry i of q's send list to rank.
 * Errors: FR_ERR_ARG, FR_ERR_MESH, FR_ERR_NOMEM.
 */
int fr_part_plan(const fr_mesh *mesh, int order, int nparts, const int32_t *part, int rank, int64_t *counts,
                 int32_t *send_pts, int32_t *halo_pts);

/*
 * fr_part_create: a partitioned mesh on the current device.  part (host,
 * may be null: fr_partition with the default weights) assigns every
 * element (public order) to one of nparts partitions; every partition
 * must hold at least one element.  Other arguments as fr_create.
 * Errors: as fr_create, and FR_ERR_ARG for an invalid partition.
 */
int fr_part_create(const fr_mesh *mesh, int order, const fr_params *params, int nparts, const int32_t *part,
                   fr_part **out);
void fr_part_destroy(fr_part *pp);
/* fr_part_info: out (host, 4 * nparts int64): per partition its tet,
 * prism and hex counts and its number of halo slots. */
int fr_part_info(const fr_part *pp, int64_t *out);
/* fr_part_set_state / fr_part_get_state: host state in the mesh's public
 * layout (the unpartitioned order); synchronous. */
int fr_part_set_state(fr_part *pp, const double *u, void *cuda_stream);
int fr_part_get_state(fr_part *pp, double *u, void *cuda_stream);
/* fr_part_rhs: as fr_rhs, device arrays in the mesh's public layout; the
 * first call allocates two state-sized scratch arrays (make it before any
 * stream capture). */
int fr_part_rhs(fr_part *pp, const double *u_dev, double *r_dev, void *cuda_stream);
/* fr_part_step: nsteps classic RK4 steps of every partition, with the
 * halo exchanges inside each stage; asynchronous. */
int fr_part_step(fr_part *pp, double dt, int nsteps, void *cuda_stream);
/* fr_part_reduce: as fr_reduce, summed over the partitions. */
int fr_part_reduce(fr_part *pp, double *out, void *cuda_stream);
/* fr_part_launches: kernels launched by the partitioned mesh so far
 * (partitions' kernels and the halo pack kernels). */
int fr_part_launches(const fr_part *pp, int64_t *launches);

/*
 * ---- Allocation-failure injection (tests) ----------------------------------
 * Every device allocation the library makes is counted.
 * fr_debug_fail_alloc(k): the k-th device allocation after this call fails
 * as if the device were out of memory (k = 0: none fails), so a test can
 * drive each FR_ERR_NOMEM path of fr_create, fr_batch_create and
 * fr_part_create.  fr_debug_alloc_stats: out[0] = device allocations
 * attempted since the last fr_debug_fail_alloc, out[1] = the library's live
 * device allocations (which must return to their earlier value when a
 * failed creation has freed what it took).  Process-wide, not thread-safe
 * against concurrent creations.
 */
int fr_debug_fail_alloc(int64_t k);
int fr_debug_alloc_stats(int64_t *out);

/*
 * fr_reduce_noalloc: the integrals of fr_reduce for callers that cannot
 * allocate device memory.  The paper has no counterpart; this entry point
 * exists for code that may not call cudaMalloc (a device owned by another
 * allocator, or a path where an allocation and its implicit
 * synchronisation are not allowed).  It needs no context and allocates
 * nothing: its scratch (one partial per block) is a file-scope static
 * device array of FR_NOALLOC_MAX_BLOCKS x 7 doubles (229,376 bytes) that
 * every GPU loading this library keeps until the process exits.
 *
 * Input: one element block of the public layout, u_dev [ne][5][nu], and
 * the quadrature weights times Jacobians wJ_dev [ne][nu] (device pointers,
 * caller-owned).  Output: out_dev (device, caller-owned, 7 doubles) =
 * sum w J u for the 5 conserved variables, the kinetic-energy integral and
 * the number of points with a non-finite state or non-positive
 * density/pressure.  Asynchronous on cuda_stream.
 *
 * Limits and errors: ne*nu may not exceed FR_NOALLOC_MAX_POINTS (8,388,608
 * points, i.e. FR_NOALLOC_MAX_BLOCKS blocks of 2,048 points); larger sizes,
 * null pointers, nu <= 0 or gamma <= 1 return FR_ERR_ARG without touching
 * the GPU.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, so make it before any
 * stream capture.  All calls share the array and it keeps the last call's
 * contents (each call overwrites the slots it reads); calls that overlap on
 * the GPU race on it, so serialise them.
 */
#define FR_NOALLOC_MAX_BLOCKS 4096
#define FR_NOALLOC_MAX_POINTS (FR_NOALLOC_MAX_BLOCKS * 2048LL)
int fr_reduce_noalloc(int64_t ne, int nu, const double *u_dev, const double *wJ_dev, double gamma,
                      double *out_dev, void *cuda_stream);

/*
 * ---- Learned closure -----------------------------------------------------
 * The paper has no learned closure; these entry points add one to the FR
 * right-hand side of a low order p_lo: a per-element multilayer perceptron
 * (one network per element type) predicts, from the element's own p_lo
 * state and corrected gradient, the difference between the projection of
 * a higher-order (p_hi) right-hand side and the p_lo right-hand side,
 *     target_e = P(RHS_hi(u_hi))_e - RHS_lo(u_lo)_e,
 * P the element-wise L2 projection from order p_hi to p_lo, and u_lo
 * either P u_hi or a p_lo state at the same time (a p_lo solution that
 * started from the projection of the same initial state).
 *
 * Network (FP32 master parameters, BF16 GEMM inputs): nin -> nh -> nh ->
 * nout, GELU (erf form) after the two hidden layers.  The parameter vector
 * (FP32) is W1[nh][nin], b1[nh], W2[nh][nh], b2[nh], W3[nout][nh],
 * b3[nout].  Every GEMM rounds its inputs (features, weights, hidden
 * activations) to bfloat16, nearest-even, and accumulates in FP32; biases,
 * pre-activations, gradients and Adam moments are FP32.
 *
 * Features of one element (row of nin = 20 nu floats, nu the element's
 * solution points at p_lo): u - u_inf at the solution points, variable-major
 * (5 x nu; u_inf the far-field state of fr_params), then the corrected
 * physical gradient, direction-major (3 x 5 x nu).  Outputs (nout = 5 nu):
 * the correction at the solution points, variable-major, in units of the
 * per-variable scales passed to fr_closure_set.
 */

/*
 * fr_transfer: host-only query (no GPU needed) of the order-transfer matrix
 * of one element type, nu(p_to) x nu(p_from), row-major float64: the L2
 * projection, on the reference element, of the p_from solution-point
 * interpolant onto the p_to space, evaluated at the p_to solution points
 * (a restriction for p_to < p_from, an exact prolongation otherwise).
 * With out == NULL only *rows/*cols are written.  Errors: FR_ERR_ARG.
 */
int fr_transfer(int etype, int p_from, int p_to, double *out, int64_t *rows, int64_t *cols);

/*
 * fr_transfer_state: u_to_dev = the order transfer of u_from_dev, element
 * by element, from the order of ctx_from to that of ctx_to (public layouts,
 * device, caller-owned; both contexts on the same mesh).  The first call for
 * a source order uploads the matrices into ctx_to (allocates).
 * Asynchronous on cuda_stream.  Errors: FR_ERR_ARG (null pointer, element
 * counts that differ), FR_ERR_NOMEM, FR_ERR_CUDA.
 */
int fr_transfer_state(const fr_ctx *ctx_from, fr_ctx *ctx_to, const double *u_from_dev, double *u_to_dev,
                      void *cuda_stream);

/*
 * fr_closure_features: the features (see above) of every element of type
 * etype for the public state u_dev (device, FP64), written to x_dev (device,
 * caller-owned, ne x 20 nu floats, row-major).  Runs the interpolation and
 * gradient stages of the RHS.  Requires a Navier-Stokes context
 * (viscous != 0; FR_ERR_UNSUPPORTED otherwise).  Asynchronous.
 */
int fr_closure_features(fr_ctx *ctx, const double *u_dev, int etype, float *x_dev, void *cuda_stream);

/*
 * fr_closure_sample: one set of training samples.  With u_hi_dev the public
 * state of ctx_hi (device, FP64) it evaluates RHS_hi(u_hi) and projects it
 * to the order of ctx_lo, evaluates RHS_lo (without any closure) of u_lo_dev
 * (a public state of ctx_lo) or, when u_lo_dev is NULL, of the projected
 * u_hi, and writes for the elements of type etype: the features of that
 * low-order state to x_dev (ne x 20 nu floats), the target
 * inv_scale[v] * (P RHS_hi - RHS_lo) to t_dev (ne x 5 nu floats, v the
 * variable of each entry; inv_scale a host array of 5, NULL = 1), and adds
 * the per-variable sums of squares of the unscaled target to ss_dev[0..4]
 * (device, FP64).  Any of x_dev, t_dev, ss_dev may be NULL.  ctx_lo must be
 * Navier-Stokes; its scratch is allocated on the first call.  Asynchronous.
 * Errors as fr_transfer_state and fr_closure_features.
 */
int fr_closure_sample(fr_ctx *ctx_hi, fr_ctx *ctx_lo, const double *u_hi_dev, const double *u_lo_dev, int etype,
                      const double *inv_scale, float *x_dev, float *t_dev, double *ss_dev, void *cuda_stream);

/*
 * fr_closure_set: attach (params_dev != NULL) or detach (NULL) the network
 * of element type etype.  params_dev (device, FP32, fr_mlp_nparams(20 nu,
 * nh, 5 nu) floats) is copied into the context.  While attached, every
 * fr_rhs / fr_step adds out_scale[v] * network(features) (out_scale: host
 * array of 5, one per conserved variable) to the RHS of those elements,
 * inside the divergence epilogue.  Requires a Navier-Stokes context;
 * batched steps (fr_batch_step) reject problems with a closure.
 * Synchronous (allocates on the first call).  Errors: FR_ERR_ARG,
 * FR_ERR_UNSUPPORTED, FR_ERR_NOMEM, FR_ERR_CUDA.
 */
int fr_closure_set(fr_ctx *ctx, int etype, const float *params_dev, int nh, const double *out_scale);

/*
 * The network's kernels, usable on their own (all pointers device,
 * caller-owned; x, t, y row-major per sample; asynchronous on cuda_stream).
 * The layers run on the tcgen05 tensor cores (bf16 weights and inputs, FP32
 * accumulation; the backward data gradients keep dL/dz as bf16 hi + lo),
 * the weight gradients (sums over the samples) on an FP32 split-K kernel.
 * fr_mlp_nparams: length of the parameter vector (host, no GPU).
 * fr_mlp_workspace: floats of scratch one call on n samples needs (host).
 *   ws must be 16-byte aligned.  Its layout, with npad = n rounded up to a
 *   multiple of 4 and every array feature-major ([row][sample], npad
 *   columns): a status int (then 3 floats of padding; non-zero if a
 *   bounded wait of the tensor-core kernel gave up), X [nin], Z1, H1, Z2,
 *   H2, dZ2, dZ1 [nh], y, dL/dy, t [nout] rows, then internal scratch.
 * fr_mlp_forward: y (n x nout) = network(x (n x nin)); ws holds X, Z1, H1,
 *   Z2, H2, y afterwards (Z the pre-activations, H = GELU(Z) before
 *   rounding).
 * fr_mlp_grad: forward then backward of the loss L = mean over all n*nout
 *   entries of (y - t)^2; g (nparams floats) = dL/dparams, loss_dev[0] = L;
 *   ws as fr_mlp_forward, plus dZ2, dZ1, dL/dy and t.
 * fr_mlp_adam: params -= lr * mhat / (sqrt(vhat) + 1e-8) with m, v the
 *   first/second moments (beta 0.9 / 0.999, updated in place) and the bias
 *   corrections of step (counting from 1).
 * Errors: FR_ERR_ARG for non-positive sizes, null pointers, an unaligned
 * workspace or step < 1; FR_ERR_UNSUPPORTED for nh or nout above 256 or a
 * layer's bf16 weight image above 192 KB.
 */
int64_t fr_mlp_nparams(int nin, int nh, int nout);
int64_t fr_mlp_workspace(int nin, int nh, int nout, int64_t n);
int fr_mlp_forward(int nin, int nh, int nout, int64_t n, const float *x_dev, const float *params_dev, float *y_dev,
                   float *ws_dev, void *cuda_stream);
int fr_mlp_grad(int nin, int nh, int nout, int64_t n, const float *x_dev, const float *t_dev,
                const float *params_dev, float *g_dev, float *loss_dev, float *ws_dev, void *cuda_stream);
int fr_mlp_adam(int64_t nparams, float *params_dev, const float *g_dev, float *m_dev, float *v_dev, int step,
                float lr, void *cuda_stream);

/* Static description of an error code. */
const char *fr_strerror(int code);

/* Detail of the most recent error on the calling thread ("" if none). */
const char *fr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FR_H */
