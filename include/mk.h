/* mk — the fine-mesh correction step of the multilevel-correction adaptive finite element method for the
 * Kohn-Sham equation (Hu, Xie, Xu, "On accelerating a multilevel correction adaptive finite element method for
 * Kohn-Sham equation"), on one NVIDIA GB300 (sm_103a).
 *
 * One step, per occupied orbital i (Algorithm 1, steps 5-7, with the frozen potential V_Hxc(rho_H) on the
 * right-hand side):
 *   mk_prolongate         u_i = P psi_{H,i}                                   (V_H subset V_h, Sec. 2)
 *   mk_hartree_poisson    (grad w, grad v) = 4 pi (rho_H, v)                   (Eq. (W_h_equation), Sec. 2)
 *   mk_assemble_rhs       b_i(v) = (lambda_{H,i}+sigma)(u_i,v) - ((w+V_xc(rho_H)) u_i, v)
 *   mk_correction_solve   (1/2)(grad x,grad v) + (V_ext x,v) + sigma (x,v) = b_i(v)   (Eq. (Aux_Linear_Problem))
 *   mk_augmented_project  A_H, M_H, b_i, c_i, beta_i, gamma_i                   (Eqs. (Adef), (bdef), (betadef))
 *   mk_small_eigensolve   Eq. (Eigenvalue_H_h), selection of Algorithm 2 (a)
 *   mk_orbital_assemble   psi_i = P phi_{i,H} + theta_{2,i} psi^_i              (Algorithm 3, output)
 *
 * Conventions shared by every entry point
 *   - Return value: MK_OK (0) or a negative MK_ERR_* code; mk_last_error() gives a message (thread-local).
 *   - Device pointers are caller-owned (e.g. torch tensors).  Nothing is allocated per call except scratch held
 *     by the mk_ctx, which grows on demand and is reused; calls on one ctx must not overlap on different streams.
 *   - `stream` is a cudaStream_t passed as void* (NULL = default stream).  Calls are asynchronous on it, except
 *     where a report is filled: those synchronise the stream before returning.
 *   - Fine-mesh vectors are node-major with orbitals contiguous: X[node * ld + i], node over ALL fine nodes
 *     (boundary nodes included and held at 0 for orbitals), i < N <= ld.  Coarse vectors are over the coarse
 *     FREE DOF (interior nodes, in increasing node order): Y[k * ldc + i].
 *   - Node numbering (both levels): the mesh vertices first, then, for P2, one node per edge in order of first
 *     appearance when tetrahedra are scanned in index order with local edges (01,02,03,12,13,23).
 *   - All arithmetic that a report or an output depends on is FP64 unless mk_solve_opts.precision says MIXED.
 */
#ifndef MK_H
#define MK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MK_OK 0
#define MK_ERR_INVALID_ARG (-1)
#define MK_ERR_CUDA (-2)
#define MK_ERR_OOM (-3)
#define MK_ERR_NOT_CONVERGED (-4) /* outputs still written, report filled */
#define MK_ERR_BREAKDOWN (-5)     /* p^T A p <= 0 met: operator not positive definite (sigma too small) */
#define MK_ERR_TIMEOUT (-6)       /* a bounded device-side wait gave up */
#define MK_ERR_SINGULAR_AUG (-7)  /* per-orbital status: psi^ lies in V_H, coarse Ritz pair returned */
#define MK_ERR_UNSUPPORTED (-8)

#define MK_MAX_RHS 64

typedef struct mk_ctx mk_ctx;
typedef struct mk_mesh mk_mesh;

/* A conforming tetrahedral mesh (Sec. 2, T_h).  Host arrays, read during mk_mesh_upload only.
 * coords [n_vertices*3] (x,y,z), tets [n_elems*4] vertex indices with positive orientation (det J > 0). */
typedef struct {
  int order; /* 1 (P1) or 2 (P2); both levels of one mesh pair use the same order */
  int64_t n_vertices;
  const double* coords;
  int64_t n_elems;
  const int32_t* tets;
} mk_mesh_desc;

/* Nuclei of V_ext = -sum_k Z_k / |x - R_k| (Sec. 2).  Host arrays Z [n], R [n*3]. */
typedef struct {
  int n_nuclei;
  const double* Z;
  const double* R;
} mk_molecule;

/* Exchange-correlation (Sec. 4): Slater exchange V_x = -(3 rho/pi)^(1/3); X-alpha -(3/2) alpha (3 rho/pi)^(1/3);
 * LDA = Slater + Perdew-Zunger correlation with the constants printed in Sec. 4. */
enum { MK_XC_NONE = 0, MK_XC_SLATER = 1, MK_XC_XALPHA = 2, MK_XC_LDA_PZ = 3 };
typedef struct {
  int kind;
  double alpha; /* X-alpha only */
} mk_xc;

enum { MK_PREC_FP64 = 0, MK_PREC_MIXED = 1, MK_PREC_PAIRS = 2 };
/* Preconditioners: JACOBI (diagonal); CHEBYSHEV (FP64 only): z = p(D^-1 A) D^-1 r, the degree-4 Chebyshev
 * polynomial of the Chebyshev iteration (D the diagonal) on [a, 1.1 b] with a, b the extreme Ritz values of 16
 * Lanczos steps on D^-1/2 A D^-1/2, three operator applications per preconditioner call (a plain comparison for
 * the learned form); LEARNED (the element-patch network, FCG(1), mixed precision only). */
enum { MK_PRECOND_JACOBI = 0, MK_PRECOND_CHEBYSHEV = 1, MK_PRECOND_LEARNED = 2 };
enum { MK_BC_ZERO = 0, MK_BC_MULTIPOLE = 1 };

typedef struct mk_mlp mk_mlp;

typedef struct {
  int precision;     /* MK_PREC_FP64: plain FP64 PCG.  MK_PREC_MIXED: FP32 inner PCG + FP64 residual refinement */
  int precond;       /* MK_PRECOND_*.  LEARNED (MIXED only): FCG(1) inner solve with mk_learned_precond */
  double rtol;       /* stop when ||b_i - A x_i||_2 / ||b_i||_2 <= rtol for every column (FP64, free DOF) */
  int maxit;         /* cap on PCG iterations (inner iterations summed for MIXED) */
  double inner_rtol; /* MIXED: relative reduction asked of each FP32 inner solve */
  int max_refine;    /* MIXED: cap on FP64 refinement cycles */
  int check_every;   /* iterations between host convergence checks (>= 1) */
  const mk_mlp* mlp; /* LEARNED: the network (NULL otherwise) */
  int mlp_precision; /* LEARNED: MK_MLP_BF16 (tensor cores) or MK_MLP_FP32 */
  /* FP64 path only: every trace_every-th iterate x_k and recursive residual r_k (k = 0, trace_every, ...) is
   * copied to trace_x / trace_r, device double [trace_cap][n_nodes*ld], until trace_cap are taken (0 = off);
   * the report's n_traced says how many.  These pairs are the training data of the learned preconditioner. */
  int trace_every, trace_cap;
  double* trace_x;
  double* trace_r;
  /* MIXED only.  1: add the exact coarse-space correction P A_H^-1 P^T r to the preconditioner (two-level:
   * Jacobi or learned fine part plus the Galerkin coarse operator A_H = P^T A P on V_H, inverted densely once per
   * mesh for the Poisson operator and once per (molecule, sigma) for the correction operator; for the Poisson
   * solve the multiplicative form Jacobi sweep / coarse correction / Jacobi sweep).  2 (Hartree Poisson solve
   * only, on a mesh with mk_mesh_set_hierarchy): the multigrid V(1,1) cycle over the fine mesh, the intermediate
   * levels and V_H (damped Jacobi, w = 0.8, one sweep before and after each coarse-level correction; the dense
   * inverse on V_H) -- the multigrid solver the paper names for its boundary-value problems (Sec. 3.1). */
  int coarse;
} mk_solve_opts;

typedef struct {
  int status;        /* MK_OK, MK_ERR_NOT_CONVERGED or MK_ERR_BREAKDOWN */
  int iterations;    /* PCG iterations run (all columns advance together) */
  int refinements;   /* FP64 residual refinements (MIXED) */
  int n_rhs;
  double max_rel_residual;              /* max over columns of the final FP64 relative residual */
  int iters[MK_MAX_RHS];                /* per column: iterations until it met rtol */
  double rel_residual[MK_MAX_RHS];      /* per column: final FP64 ||b - A x|| / ||b|| */
  int n_traced;                         /* iterates copied to mk_solve_opts.trace_x / trace_r */
} mk_solve_report;

typedef struct {
  int order, nloc;
  int64_t n_nodes, n_free, n_elems, n_colours;            /* fine level */
  int64_t n_nodes_coarse, n_free_coarse, n_elems_coarse;  /* coarse level */
  int n_quad;                                             /* quadrature points per element */
} mk_mesh_info;

/* ---------------------------------------------------------------------------------------------- context */
/* Creates a context on CUDA device `device`.  Errors: MK_ERR_CUDA (no device / bad id). */
int mk_ctx_create(mk_ctx** ctx, int device);
int mk_ctx_destroy(mk_ctx* ctx);
/* Waits for the device, then returns in *fault the context's device fault word and clears it: 0, or
 * MK_FAULT_* bits set by kernels whose bounded waits for their own asynchronous copies or tensor-core operations
 * gave up (those kernels return early and their outputs are invalid; the solves that launched them return
 * MK_ERR_TIMEOUT).  A diagnostic with no counterpart in the paper. */
#define MK_FAULT_PATCH_WAIT 1
#define MK_FAULT_PATCH_RECORD 2
#define MK_FAULT_TC_WAIT 4
int mk_ctx_fault(mk_ctx* ctx, int* fault);
/* Context options (diagnostics and tests; no counterpart in the paper).  Errors: MK_ERR_INVALID_ARG.
 *   MK_OPT_GRAPHS (default 1): 0 runs the inner iterations of the mixed-precision solves eagerly instead of
 *     replaying them from a CUDA graph.
 *   MK_OPT_PATCH_PIPELINE (default 1): the kernel of the element-by-element operator.  1: for FP32 the
 *     register-staged kernel (one element per thread, its matrix loaded into registers, several patch CTAs per
 *     SM), for FP64 the persistent two-group pipelined kernel;
 *     2: the two-group pipelined kernel for FP32 as well; 0: the one-patch-per-CTA kernel (the fallback).  All
 *     three give bitwise equal results.
 *   MK_OPT_WAIT_LIMIT (default -1 = about a second): the number of polls (each suspending the thread up to about
 *     1 us) after which the persistent operator kernels' waits for their own copies give up; 0 makes the first wait
 *     give up at once.  A kernel that gives up sets MK_FAULT_PATCH_WAIT, then still waits, with the default limit,
 *     for every copy it issued before it ends; the call that launched it returns MK_ERR_TIMEOUT (solves) or leaves
 *     the bit for mk_ctx_fault (mk_operator_apply), and the outputs are invalid.
 *   MK_OPT_DECOMPOSE_CTAS (default 0 = one per SM): the number of CTAs of the cooperative block-Jacobi kernel of
 *     mk_coarse_decompose(_warm); clamped to the SM count, and at least one more than the block pairs of a round
 *     (else the decomposition returns MK_ERR_INVALID_ARG).  Fewer CTAs leave more of each SM to kernels running
 *     beside it on another stream.
 *   MK_OPT_PAIR_RESIDUAL (default 1): the FP64 residual b - A x of every refinement step of the mixed-precision
 *     solves computed on the FP32 units from FP32 pairs (each FP64 value as hi + lo, error-free products and sums,
 *     about 48 significant bits; see MK_PREC_PAIRS), FP64 node sums; 0: plain FP64 products. */
#define MK_OPT_GRAPHS 1
#define MK_OPT_PATCH_PIPELINE 2
#define MK_OPT_WAIT_LIMIT 3
#define MK_OPT_DECOMPOSE_CTAS 4
#define MK_OPT_PAIR_RESIDUAL 5
int mk_ctx_set_option(mk_ctx* ctx, int option, int value);
/* Copies the calling thread's last error message into buf (always NUL-terminated); returns its length. */
int mk_last_error(char* buf, size_t len);
/* Version string of the library build. */
const char* mk_version(void);
/* Number of CUDA kernels this library has launched in the process so far (all contexts); a diagnostic counter
 * with no counterpart in the paper, used to report launches per step. */
long long mk_launch_count(void);
/* Optional timing of the operator applications with CUDA events recorded on the launching stream (diagnostic, no
 * counterpart in the paper).  mk_profile_enable(ctx, 1) clears and starts recording; mk_profile_read waits for
 * the recorded events and returns the summed duration and the number of timed applications of kind
 * 0 = FP64 element-by-element apply, 1 = FP32 patch apply of the correction operator (the pipelined or the
 * one-patch-per-CTA kernel), 2 = FP32 halo sum, 3 = learned-preconditioner patch kernel (the network and the node
 * sums, without the halo pass), 4 = FP32 matrix-free stiffness operator of the Poisson solve, 5 = the FP64-accurate
 * operator on FP32 pairs (one launch per 4 columns, without the split of x and the halo pass).  Every application is
 * timed, including those inside the CUDA graphs of the inner iterations (each has its own event pair in the
 * graph, up to 128 pairs of a kind per captured chunk). */
#define MK_PROF_APPLY64 0
#define MK_PROF_APPLY32 1
#define MK_PROF_HALO 2
#define MK_PROF_LEARNED 3
#define MK_PROF_STIFF 4
#define MK_PROF_PAIRS 5
int mk_profile_enable(mk_ctx* ctx, int on);
int mk_profile_read(mk_ctx* ctx, int kind, double* total_ms, long long* count);

/* ---------------------------------------------------------------------------------------------- mesh (A0) */
/* Uploads a nested fine/coarse mesh pair (Sec. 2: V_H subset V_h needs T_h to refine T_H).  fine_parent [n_elems
 * of fine] gives, for each fine tetrahedron, the coarse tetrahedron containing it.  Computed here on the host:
 * P2 edge-node numbering, boundary nodes (nodes on faces that belong to one tetrahedron), greedy element
 * colouring (elements in index order, smallest colour not used by an earlier element sharing a vertex), the
 * coarse-to-fine interpolation P (coarse basis functions evaluated at fine nodes), the element patches used by
 * the FP32 operator.  Device copies are owned by the returned handle.  Errors: MK_ERR_INVALID_ARG (orders differ,
 * index out of range, det J <= 0, a fine element outside its parent), MK_ERR_OOM, MK_ERR_CUDA. */
int mk_mesh_upload(mk_ctx* ctx, const mk_mesh_desc* fine, const mk_mesh_desc* coarse, const int32_t* fine_parent,
                   mk_mesh** out);
int mk_mesh_destroy(mk_mesh* mesh);
/* Intermediate levels of a nested hierarchy between the coarse and the fine mesh of `mesh`, for the multigrid
 * preconditioner of the Hartree Poisson solve (mk_solve_opts.coarse = 2): levels[0..n_mid) from coarsest to
 * finest, levels[0] nested in the coarse mesh, each next one in the previous, the fine mesh in the last;
 * parents[k] [levels[k].n_elems] gives the element of the next coarser mesh that contains each element of
 * levels[k], and parents[n_mid] [fine n_elems] the element of levels[n_mid - 1] containing each fine element
 * (n_mid = 0: the fine mesh directly on V_H; parents may then be NULL).  Host arrays, read during the call.  Built
 * here on the host and kept by the handle: each level's numbering and boundary, its stiffness matrix on the
 * interior nodes (FP32 CSR) and inverse diagonal, the interpolation between consecutive levels (coarse basis
 * functions at the finer nodes, exact on nested meshes) and its transpose.  Replaces an earlier hierarchy;
 * synchronises the device.  Errors: MK_ERR_INVALID_ARG (orders differ, a level not nested in its parent),
 * MK_ERR_OOM. */
int mk_mesh_set_hierarchy(mk_mesh* mesh, int n_mid, const mk_mesh_desc* levels, const int32_t* const* parents);

int mk_mesh_get_info(const mk_mesh* mesh, mk_mesh_info* info);
/* Host copies of the A0 results, for checking: level 0 = fine, 1 = coarse.  Any pointer may be NULL.
 * nodes [n_nodes*3], boundary [n_nodes] (1 = boundary), elem [n_elems*nloc] node indices, colour [n_elems]. */
int mk_mesh_get_topology(const mk_mesh* mesh, int level, double* nodes, uint8_t* boundary, int32_t* elem,
                         int32_t* colour);

/* ---------------------------------------------------------------------------------------------- A1 */
/* u = P psi_H: psiH [N_H * ldc] (coarse free DOF) -> u [n_nodes * ld] fine, boundary rows 0 (Sec. 2, V_H subset
 * V_h: exact interpolation).  Errors: MK_ERR_INVALID_ARG (N < 1, N > ld, N > ldc). */
int mk_prolongate(mk_ctx* ctx, const mk_mesh* mesh, const double* psiH, int ldc, int N, double* u, int ld,
                  void* stream);

/* ---------------------------------------------------------------------------------------------- A2 */
/* Hartree potential (Sec. 2, -Delta V_Har = 4 pi rho; Eq. (W_h_equation)): solves (grad w, grad v) =
 * 4 pi (rho_H, v) for all free v with rho_H(x) = sum_i occ[i] u_i(x)^2 evaluated at the quadrature points.
 * bc = MK_BC_MULTIPOLE: boundary values from the multipole expansion of int rho(y)/|x-y| dy about the origin
 * through l = 2 (Remark after Algorithm 3); MK_BC_ZERO: w = 0 on the boundary.
 * u [n_nodes*ld] device, occ [N] host, w [n_nodes] device output (boundary values included).  rho_q: rho_H at
 * the quadrature points as mk_density writes it for the same u and occ, or NULL (computed here).  The report is
 * filled (stream synchronised).  Errors: MK_ERR_NOT_CONVERGED, MK_ERR_BREAKDOWN, MK_ERR_INVALID_ARG. */
int mk_hartree_poisson(mk_ctx* ctx, const mk_mesh* mesh, const double* u, int ld, const double* occ, int N,
                       const double* rho_q, int bc, double* w, const mk_solve_opts* opts, mk_solve_report* report,
                       void* stream);
/* rho_H = sum_i occ[i] u_i^2 at the quadrature points of every fine element, rho_q [n_elems * n_quad] device
 * (element order of the upload; n_quad from mk_mesh_info), FP64; u [n_nodes*ld] device, occ [N] host.  Computed
 * once per step, it serves mk_hartree_poisson and mk_frozen_potential (both evaluate the same rho_H). */
int mk_density(mk_ctx* ctx, const mk_mesh* mesh, const double* u, int ld, const double* occ, int N, double* rho_q,
               void* stream);

/* ---------------------------------------------------------------------------------------------- A3 */
/* Right-hand sides of the correction problems (Eq. (Aux_Linear_Problem) with V_Hxc(rho_H) moved to the right):
 * rhs_i(v) = (lambdaH[i] + sigma)(u_i, v) - ((w + V_xc(rho_H)) u_i, v), rho_H = sum_i occ[i] u_i^2, for all
 * fine nodes v (boundary rows written as 0).  Also writes the frozen potential w + V_xc(rho_H) at the quadrature
 * points, vq [n_elems * n_quad] (element order of the upload), which mk_augmented_project reuses.
 * u, rhs [n_nodes*ld] device; w [n_nodes] device or NULL (= 0); lambdaH, occ [N] host. */
int mk_assemble_rhs(mk_ctx* ctx, const mk_mesh* mesh, const double* u, int ld, const double* lambdaH,
                    const double* occ, int N, const double* w, double sigma, mk_xc xc, double* rhs, double* vq,
                    void* stream);
/* The two halves of mk_assemble_rhs, so that the coarse pencil (which needs vq, not rhs) can start on another
 * stream as soon as vq exists.  mk_frozen_potential: rho_H = sum_i occ[i] u_i^2 and vq = w + V_xc(rho_H) at the
 * quadrature points [n_elems * n_quad] (rho_q as for mk_hartree_poisson, or NULL).  mk_assemble_rhs_from_vq: rhs
 * from u and that vq (as mk_assemble_rhs). */
int mk_frozen_potential(mk_ctx* ctx, const mk_mesh* mesh, const double* u, int ld, const double* occ, int N,
                        const double* rho_q, const double* w, mk_xc xc, double* vq, void* stream);
int mk_assemble_rhs_from_vq(mk_ctx* ctx, const mk_mesh* mesh, const double* u, int ld, const double* lambdaH, int N,
                            const double* vq, double sigma, double* rhs, void* stream);

/* ---------------------------------------------------------------------------------------------- A4 */
/* Solves (K/2 + M_{V_ext} + sigma M) x_i = rhs_i on the free fine DOF for i < N at once (Eq. (Aux_Linear_Problem),
 * one boundary-value problem per orbital, Algorithm 1 step 5), matrix-free element by element.
 * x [n_nodes*ld] device: initial guess in, solution psi^ out (boundary rows 0).  opts->precision selects plain
 * FP64 PCG or FP32 inner PCG with FP64 residual refinement; either way convergence is judged on the FP64
 * residual.  The report is filled (stream synchronised).  Errors: MK_ERR_NOT_CONVERGED (x still written),
 * MK_ERR_BREAKDOWN (sigma too small), MK_ERR_INVALID_ARG (bad options, e.g. CHEBYSHEV with MIXED). */
int mk_correction_solve(mk_ctx* ctx, const mk_mesh* mesh, const mk_molecule* mol, double sigma, const double* rhs,
                        double* x, int ld, int N, const mk_solve_opts* opts, mk_solve_report* report, void* stream);

/* The paper's own form of step 5 (Eq. (Aux_Linear_Problem) as Algorithm 1 writes it): the frozen potential on the
 * left, (K/2 + M_{V_ext} + M_{vq} + sigma M) x_i = rhs_i, with vq [n_elems * n_quad] device (e.g. the previous
 * Hartree potential plus V_xc of the step's input orbitals, from mk_frozen_potential) and rhs_i = (lambda_i +
 * sigma) M u_i (mk_assemble_rhs_from_vq with a zero vq).  x, opts, report and errors as mk_correction_solve;
 * opts->coarse must be 0 (the cached coarse operators are those without vq). */
int mk_correction_solve_vq(mk_ctx* ctx, const mk_mesh* mesh, const mk_molecule* mol, const double* vq, double sigma,
                           const double* rhs, double* x, int ld, int N, const mk_solve_opts* opts,
                           mk_solve_report* report, void* stream);

/* The operator of the correction problems alone (Eq. (Aux_Linear_Problem) with the shift): y = (K/2 + M_{V_ext} +
 * sigma M) x on the free DOF (boundary rows of y written as 0), all ld columns, matrix-free element by element with
 * the patch scatter (owner-computes in shared memory, halo slots summed in patch order; bitwise reproducible).
 * precision MK_PREC_FP64: x, y are double [n_nodes*ld]; MK_PREC_MIXED: x, y are float [n_nodes*ld] (the FP32
 * operator of the mixed solve); MK_PREC_PAIRS: x, y are double, the products formed on the FP32 units from FP32
 * pairs (a value v as hi = fl32(v) plus lo = fl32(v - hi); exact products and two-sums; the error is a few units of
 * 2^-48 relative to sum_j |a_ij x_j|, against 2^-53 for FP64), the element and node sums rounded to FP64 (the
 * refinement residual of the mixed solves, MK_OPT_PAIR_RESIDUAL).  Element matrices are rebuilt on every call.  mol = NULL (with sigma = 0): the
 * stiffness operator K of the Hartree Poisson problem (Sec. 2, the Hartree equation) instead, in FP32 matrix-free
 * (per element |det J| J^-1 J^-T times the reference stiffness components), in FP64 from stored element matrices. */
int mk_operator_apply(mk_ctx* ctx, const mk_mesh* mesh, const mk_molecule* mol, double sigma, int precision,
                      const void* x, void* y, int ld, void* stream);

/* ---------------------------------------------------------------------------------------------- A6 */
/* Projection on the augmented spaces V_H + span{psi^_i} (Eqs. (Eigenvalue_H_h), (Adef), (bdef), (betadef)) with
 * H = K/2 + M_{V_ext} + M_{vq} the Hamiltonian at the frozen density (vq from mk_assemble_rhs):
 *   AH = P^T H P, MH = P^T M P           [N_H*N_H] row-major, coarse free DOF (shared by all orbitals)
 *   b[:,i] = P^T H psi^_i, c[:,i] = P^T M psi^_i      [N_H*N] (ld = N)
 *   beta[i] = psi^_i^T H psi^_i, gamma[i] = psi^_i^T M psi^_i                    [N]
 *   gramA = Psi^T H Psi, gramM = Psi^T M Psi   [N*N] (may be NULL)
 * All device FP64. */
int mk_augmented_project(mk_ctx* ctx, const mk_mesh* mesh, const mk_molecule* mol, const double* vq,
                         const double* psihat, int ld, int N, double* AH, double* MH, double* b, double* c,
                         double* beta, double* gamma, double* gramA, double* gramM, void* stream);

/* The coarse blocks alone: AH = P^T H P, MH = P^T M P [N_H*N_H] for the frozen potential vq (Eq. (Adef); the
 * coarse blocks are assembled on the fine mesh, ahead of the augmented solve).  They do not depend on psi^, so a
 * caller may compute them, and decompose them, on a second stream while mk_correction_solve runs.  vq may be NULL
 * (bare Hamiltonian K/2 + V_ext).  MH may be NULL: M_H does not depend on the density, and the decomposition uses
 * the factor of M_H kept by the mesh handle.  Uses its own scratch, separate from mk_correction_solve's. */
int mk_coarse_pencil(mk_ctx* ctx, const mk_mesh* mesh, const mk_molecule* mol, const double* vq, double* AH,
                     double* MH, void* stream);

/* ---------------------------------------------------------------------------------------------- A7 */
/* Shared part of the small eigenproblem of Eq. (Eigenvalue_H_h): all eigenpairs of the coarse pencil (AH, MH),
 * d [N_H] ascending and V [N_H*N_H] row-major (V[r*N_H + k] = component r of eigenvector k), M_H-orthonormal.
 * MH is the mesh's own P^T M P, whose Cholesky factor mk_mesh_upload computed (M_H is fixed for a mesh pair).
 * C = L^-1 AH L^-T by two FP64 GEMMs, then cyclic block Jacobi in two phases (cooperative launches): the sweeps
 * of the linear phase in FP32, its Q made orthogonal in FP64 and C projected onto it, then FP64 sweeps to
 * off(S) <= 1e-14 |S|; V = L^-T Q. */
int mk_coarse_decompose(mk_ctx* ctx, const mk_mesh* mesh, const double* AH, double* d, double* V, void* stream);
/* Report of the most recent decomposition on this context (mk_coarse_decompose, _warm, and the dense solves of
 * mk_joint_ritz / mk_joint_assemble): the sweeps of its FP32 and FP64 phases.  Synchronises the device.
 * Errors: MK_ERR_INVALID_ARG (null argument, or no decomposition yet). */
int mk_decompose_info(mk_ctx* ctx, int* sweeps32, int* sweeps64);
/* The same decomposition started from a known M_H-orthonormal basis V0 [N_H*N_H] (e.g. the eigenvectors of the
 * density-independent pencil (P^T (K/2 + M_Vext) P, M_H), which stays fixed for a molecule as the paper's static
 * blocks do): C = V0^T AH V0 is then close to diagonal and Jacobi needs fewer sweeps; V = V0 Q.  The result is
 * the eigen-decomposition of (AH, M_H) to FP64 accuracy whatever V0 is, as long as V0^T M_H V0 = I. */
int mk_coarse_decompose_warm(mk_ctx* ctx, int N_H, const double* AH, const double* V0, double* d, double* V,
                             void* stream);
/* Per-orbital part, given the shared decomposition (d, V) of (AH, MH): same outputs and selection rule as
 * mk_small_eigensolve below. */
int mk_small_eigensolve_shared(mk_ctx* ctx, int N_H, int N, const double* d, const double* V, const double* b,
                               const double* c, const double* beta, const double* gamma, double* lambda,
                               double* coef, int32_t* status, void* stream);
/* The same per-orbital solve as mk_small_eigensolve_shared, for callers that must not allocate device memory:
 * programs whose device memory is reserved up front by another allocator (a cudaMalloc would fail or break that
 * budget) and latency-sensitive loops that cannot afford cudaMalloc/cudaFree, which may synchronise the whole
 * device.  No counterpart in the paper.  Needs no mk_ctx and allocates nothing: its workspace is a fixed array
 * in the library (about 0.9 MB, held by every GPU that loads the library until the process exits), sized for
 * N_H <= 512 and N <= 16; larger sizes return MK_ERR_INVALID_ARG.  It runs on the current CUDA device.  The
 * first call on a device looks up the array's device address once (cudaGetSymbolAddress); make that first call
 * before any stream capture.  That address is kept for the life of the process: after cudaDeviceReset (or any other
 * teardown of the device's primary context) it is stale, so do not call this entry point again in that process.  All calls share the one array: calls that overlap on the GPU (other streams or
 * host threads) race, so serialise them.  Nothing in the array needs to start at zero. */
int mk_small_eigensolve_static(int N_H, int N, const double* d, const double* V, const double* b, const double* c,
                               const double* beta, const double* gamma, double* lambda, double* coef,
                               int32_t* status, void* stream);
/* For each orbital i < N, all eigenpairs of the (N_H+1) pencil of Eq. (Eigenvalue_H_h)
 *   [[AH, b_i], [b_i^T, beta_i]] x = lambda [[MH, c_i], [c_i^T, gamma_i]] x
 * and the one "with the largest component in span{psi^_i}" (Algorithm 2 (a)), read as the largest
 * |(x, psi^_i)_M| over M-normalised eigenvectors (ties within 1e-12 relative: lower eigenvalue).  Computed as one
 * shared FP64 eigen-decomposition of (AH, MH) plus, per orbital, the roots of the secular equation of the
 * bordered problem.  Outputs: lambda [N], coef [(N_H+1)*N] (column i = (phi_{i,H}, theta_{2,i}), M-normalised,
 * sign with (x, psi^_i)_M >= 0), status [N] (MK_OK or MK_ERR_SINGULAR_AUG when ||u||_M/||psi^||_M < 1e-7 with
 * u = psi^ - Pi_H psi^; then the coarse Ritz pair with the largest |(x, Pi_H psi^)_M| and theta = 0).
 * All device FP64 (status int32).  Errors: MK_ERR_INVALID_ARG, MK_ERR_CUDA. */
int mk_small_eigensolve(mk_ctx* ctx, int N_H, int N, const double* AH, const double* MH, const double* b,
                        const double* c, const double* beta, const double* gamma, double* lambda, double* coef,
                        int32_t* status, void* stream);

/* ---------------------------------------------------------------------------------------------- joint space */
/* Rayleigh-Ritz in the joint augmented space V_H + span{psi^_1, ..., psi^_N} (the multilevel-correction scheme
 * that augments the coarse space with all the corrections at once rather than one at a time; Sec. 2, the
 * original scheme the paper builds on): the lowest k eigenpairs of
 *   [[A_H, B], [B^T, G_A]] x = lambda [[M_H, C], [C^T, G_M]] x,
 * B = P^T H Psi^, C = P^T M Psi^, G_A = Psi^T H Psi^, G_M = Psi^T M Psi^ (mk_augmented_project's b, c, gramA,
 * gramM; the Grams are symmetrised), with (A_H, M_H) given by their shared decomposition d [N_H], V [N_H*N_H]
 * (mk_coarse_decompose).  The corrections are M-orthogonalised against V_H; directions whose mass in that basis is
 * at most 1e-12 max(1, largest) (a correction in V_H, two equal corrections) are dropped; *n_kept (host, may be
 * NULL) receives how many are kept.  The remaining problem is one dense symmetric FP64 eigensolve of size
 * N_H + n_kept (cyclic block Jacobi, as for the coarse decomposition; N_H + N below 2432).
 * Outputs (device FP64): lambda [k] ascending; X [(N_H + N) * k] row-major, column j = the coarse coefficients
 * (free DOF) then the coefficients of psi^_1..psi^_N of Ritz vector j, M-orthonormal, sign arbitrary.
 * Synchronises the stream once (the kept count decides the size of the dense problem).
 * Errors: MK_ERR_INVALID_ARG (k > N_H + n_kept, sizes), MK_ERR_CUDA. */
int mk_joint_ritz(mk_ctx* ctx, int N_H, int N, int k, const double* d, const double* V, const double* b,
                  const double* c, const double* gramA, const double* gramM, double* lambda, double* X, int* n_kept,
                  void* stream);
/* The joint Ritz vectors on the fine mesh: psi_j = P X[0:N_H, j] + sum_i X[N_H + i, j] psi^_i for j < k, sign chosen
 * so that (psi_j, u_j)_M >= 0 (u = P psi_H, the step's prolonged input orbitals).  psihat, u, psi [n_nodes*ld]. */
int mk_joint_assemble(mk_ctx* ctx, const mk_mesh* mesh, int k, int N, const double* X, const double* psihat,
                      const double* u, int ld, double* psi, void* stream);

/* ---------------------------------------------------------------------------------------------- A8 */
/* psi_i = P phi_{i,H} + theta_{2,i} psi^_i (Algorithm 3, output), sign chosen so that (psi_i, u_i)_M > 0.
 * coef [(N_H+1)*N] from mk_small_eigensolve, psihat/u/psi [n_nodes*ld] device. */
int mk_orbital_assemble(mk_ctx* ctx, const mk_mesh* mesh, const double* coef, const double* psihat,
                        const double* u, int ld, int N, double* psi, void* stream);

/* ---------------------------------------------------------------------------------------------- inner SCF */
/* The paper's step 7 (Eq. (Nonlinear_Eig_Hh_Full)) by the inner iteration of Algorithm 2 with the precomputations
 * of Algorithm 3: the orbitals in V_H + span{phi~_i}, the Hartree potential in w_b + V_H + span{w~0}, where
 * w~ = w_b + w~0 is the Hartree potential of the corrections' density (mk_hartree_poisson of phi~) split into its
 * boundary values w_b (zero inside) and the rest w~0 (zero on the boundary); the boundary values stay fixed.
 *
 * mk_inner_create (Algorithm 3, step 1): integrates on the fine mesh, once, everything an inner iteration needs,
 * so that an iteration costs O(N_H) coarse work: A1 = P^T H1 P, b1_i = P^T H1 phi~_i, beta1_i (H1 = K/2 + V_ext +
 * V_xc + w_b), A3 = P^T M_{w~0} P, b3_i, beta3_i (Eq. (FG)), c_i, gamma_i, the bordered Hartree system (P^T K P,
 * P^T K w~0, (K w~0, w~0)) with the lifts of w_b, and per coarse element the tensors (psi_a psi_b, psi_c),
 * (phi~_i psi_a, psi_b) (Eq. (Ah4def)), (phi~_i^2, psi_a) (Eq. (rhsdef)) and (w~0, phi~_i^2) on the fine
 * quadrature.  phit [n_nodes*ld] device (the corrections phi~, boundary rows 0), wt [n_nodes] device, vxc_q
 * [n_elems * n_quad] device (V_xc of the step's input orbitals at the quadrature points: mk_frozen_potential with
 * w = 0).  The handle owns its device memory (about (3 + 2N) N_H^2 + N n_elem_coarse n_loc^2 doubles) until
 * mk_inner_destroy.  Synchronises the stream.  MK_ERR_INVALID_ARG if P^T K P is not positive definite or
 * n_loc^3 + N (n_loc^2 + n_loc + 1) > 8192.  When w~0 already lies in V_H (Schur complement of the border at most
 * 1e-12 (K w~0, w~0)), the extra Hartree direction is dropped (theta_1 = 0); mk_inner_info reports it.
 *
 * mk_inner_run (Algorithm 2): from w = w~ (w_H = 0, theta_1 = 1), for s = 1 .. max_inner: (a) the per-orbital
 * eigenproblems in V_H + span{phi~_i} with the current Hartree potential and the selection of
 * mk_small_eigensolve_shared (lambda [N], coef [(N_H+1)*N] as there); (b) the Hartree potential of the density
 * sum_i occ_i (phi_{i,H} + theta_{2,i} phi~_i)^2 in W, mixed: (w_H, theta_1) <- (1 - mix) old + mix new; (c) stop
 * once s > 1 and the largest change of any coefficient is below tol.  occ [N] host.  Outputs: lambda, coef,
 * status [N] (or NULL), wH [N_H] (or NULL) device, from the last iteration (w_H and theta_1 after its update);
 * theta1, iters, delta (the last change) host or NULL.  Synchronises the stream after every iteration.
 * mk_inner_potential: w = w_b + P w_H + theta_1 w~0 [n_nodes] device, the inner Hartree potential after the last
 * mk_inner_run.  The output orbitals are mk_orbital_assemble(coef, phit, phit): P phi_H + theta_2 phi~. */
typedef struct mk_inner mk_inner;
int mk_inner_create(mk_ctx* ctx, const mk_mesh* mesh, const mk_molecule* mol, const double* phit, int ld, int N,
                    const double* wt, const double* vxc_q, mk_inner** out, void* stream);
int mk_inner_run(mk_ctx* ctx, mk_inner* inner, const double* occ, double tol, int max_inner, double mix,
                 double* lambda, double* coef, int32_t* status, double* wH, double* theta1, int* iters, double* delta,
                 void* stream);
int mk_inner_potential(mk_ctx* ctx, const mk_inner* inner, double* w, void* stream);
int mk_inner_info(const mk_inner* inner, int* w_in_VH, double* schur);
int mk_inner_destroy(mk_inner* inner);

/* ---------------------------------------------------------------------------------------------- AFEM */
/* The outer AFEM loop's Estimate and Mark steps (Sec. 2, the residual a posteriori error indicator and Dorfler's
 * marking strategy).  mk_error_indicators: for the orbitals psi [n_nodes*ld] device (columns < N) with eigenvalues
 * lambda [N] host, and vq [n_elems * n_quad] device = w + V_xc at the quadrature points (mk_frozen_potential of
 * psi's own density), per fine element T
 *   eta2[T] = h_T^2 sum_i ||H psi_i - lambda_i psi_i||_{0,T}^2
 *             + sum over the interior faces e of T of h_e sum_i ||1/2 grad psi_i|T+ . nu+ + 1/2 grad psi_i|T- . nu-||_{0,e}^2
 * with H = -1/2 Laplacian + V_ext(mol) + vq, h_T and h_e the longest edges of T and e; the element integral by
 * the 27-point rule, the face integral by the 3-point rule at the face's edge midpoints.  eta2 [n_elems] device.
 * The first call builds the mesh's face table (host, kept in the mesh handle).  Deterministic (no atomics).
 * mk_dorfler_mark: marked[T] = 1 for eta2[T] >= t*, with t* the largest t for which the indicators at or above t
 * sum to at least theta times their total (0 < theta <= 1; the paper's experiments use 0.4): without ties at the
 * cut, the smallest set in order of decreasing indicator; elements tied with the cut are all marked.  eta2 [n]
 * and marked [n] device; n_marked and threshold (t*) host, or NULL.  Synchronises the stream (about 64 fixed-order
 * reductions).  MK_ERR_INVALID_ARG if the indicators sum to zero. */
int mk_error_indicators(mk_ctx* ctx, const mk_mesh* mesh, const mk_molecule* mol, const double* psi, int ld, int N,
                        const double* lambda, const double* vq, double* eta2, void* stream);
int mk_dorfler_mark(mk_ctx* ctx, int64_t n, const double* eta2, double theta, uint8_t* marked, int64_t* n_marked,
                    double* threshold, void* stream);
/* The Refine step (Sec. 2: marked elements refined so that the mesh stays shape regular and conforming): newest-vertex
 * bisection in Maubach's form with conforming closure.  The mesh: coords [n_vertices*3] FP64, tets [n_elems*4] int32
 * with every tetrahedron's vertices in bisection order and tags [n_elems] int8 in {1,2,3} (the Kuhn tetrahedra of a
 * cube mesh in path order with tag 3 are such a mesh).  A tetrahedron (x0,x1,x2,x3) with tag k is cut at the midpoint
 * z of x0-xk into (x0,..,x_{k-1},z,x_{k+1},..,x3), which keeps its index, and (x1,..,xk,z,x_{k+1},..,x3), appended in
 * the order of the cut elements; both get tag k-1 (3 after 1).  The first round cuts the marked elements (marked
 * [n_elems] uint8), every later round the elements that hold an edge already cut, until none does.  A new midpoint
 * is numbered after the existing vertices in the order of the lowest-index element that cuts its edge in its round.
 * coords, tets, tags are refined in place (device buffers with room for max_vertices and max_elems); parent
 * [max_elems] device receives, per output element, the input element that contains it.  *n_vertices_out,
 * *n_elems_out and *rounds (or NULL) are host.  The output tetrahedra keep the bisection order, so their orientation
 * alternates; orient them (swap the last two vertices where the volume is negative) before mk_mesh_upload.
 * MK_ERR_INVALID_ARG if the result would exceed max_vertices or max_elems (the buffers' contents are then
 * unspecified).  Synchronises the stream twice per round. */
int mk_refine(mk_ctx* ctx, int64_t n_vertices, int64_t n_elems, double* coords, int32_t* tets, int8_t* tags,
              int32_t* parent, const uint8_t* marked, int64_t max_vertices, int64_t max_elems, int64_t* n_vertices_out,
              int64_t* n_elems_out, int* rounds, void* stream);

/* ---------------------------------------------------------------------------------------------- shift */
/* Lowest Ritz value of `steps` Lanczos steps on the pencil (K/2 + M_{V_ext}, M) over the free fine DOF, from the
 * start vector v0 [n_free] (host, free-DOF order); M^-1 applied by an inner CG.  Used for the shift rule
 * sigma = 1.05 max(0, -theta) + 0.5 that keeps the correction operator positive definite. */
int mk_lowest_ritz(mk_ctx* ctx, const mk_mesh* mesh, const mk_molecule* mol, const double* v0, int steps,
                   double* theta, void* stream);
/* The shift of the correction problems (the reading that keeps K/2 + M_{V_ext} + sigma M positive definite, since
 * the paper's operator a(.,.) + (V_ext .,.) is indefinite): theta from mk_lowest_ritz with the same arguments, then
 * sigma = 1.05 max(0, -theta) + 0.5 (Ha).  Both are written to the host doubles theta and sigma. */
int mk_correction_shift(mk_ctx* ctx, const mk_mesh* mesh, const mk_molecule* mol, const double* v0, int steps,
                        double* theta, double* sigma, void* stream);

/* ---------------------------------------------------------------------------------------------------------
 * Batching: many molecules (uneven meshes, uneven orbital counts) in shared launches, and autotuned patch sizes
 * --------------------------------------------------------------------------------------------------------- */
/* Solves the correction problems (Eq. (Aux_Linear_Problem)) of K molecules together: problem k is (meshes[k],
 * mols[k], sigmas[k]) with right-hand side rhs[k] and initial guess / result x[k] (device double
 * [n_nodes_k * ld[k]], columns < N[k]), as mk_correction_solve with *opts (MK_PREC_MIXED, Jacobi, no coarse
 * correction).  The FP64 residual refinement runs per problem; every inner FP32 PCG iteration runs as seven kernel
 * launches for the whole batch (one grid over the element patches of all meshes, the halo sums, the dot products
 * and updates of all problems), replayed from one CUDA graph per chunk of opts->check_every iterations; the operator
 * is the register-staged kernel of the single solve (every element matrix read once for all of a problem's
 * columns), or the one-patch-per-CTA kernel where the meshes have no patch records or MK_OPT_PATCH_PIPELINE is not
 * 1.  All meshes must use the same element order; ld[k] in {4, 8, 16, 32} (32 only with the register-staged
 * kernel); K <= MK_MAX_BATCH.  reports[k] (host) is filled for every
 * problem.  Each problem's result is bit-identical to mk_correction_solve's with the same options (same kernels,
 * same summation orders; a converged problem idles while others iterate).  Returns MK_ERR_NOT_CONVERGED or
 * MK_ERR_BREAKDOWN if any problem did (see the reports).  Synchronises the stream. */
#define MK_MAX_BATCH 256
int mk_batch_correction_solve(mk_ctx* ctx, int K, const mk_mesh* const* meshes, const mk_molecule* mols,
                              const double* sigmas, const double* const* rhs, double* const* x, const int* ld,
                              const int* N, const mk_solve_opts* opts, mk_solve_report* reports, void* stream);
/* Rebuilds the mesh's element patches with pe elements each (pe a multiple of 32 in [32, 512]; the patch
 * kernels' shared memory must fit).  Synchronises the device. */
int mk_mesh_set_patch_elems(mk_mesh* mesh, int pe);
/* Autotuner of the patch size: times the FP32 operator on this mesh for ld columns with each candidate (64, 96,
 * 128, 192 elements per patch for P2; 128, 192, 256, 384 for P1), leaves the mesh with the fastest and returns it
 * in *best_pe; ms (host, 4 entries, may be NULL) receives each candidate's time per application. */
int mk_autotune_patches(mk_ctx* ctx, mk_mesh* mesh, int ld, int* best_pe, double* ms);

/* ---------------------------------------------------------------------------------------------------------
 * Learned element-patch preconditioner (this library's addition; the paper solves its boundary-value problems
 * with standard solvers).  Definitions, for element e and orbital column j:
 *   input   x = [r_e / s, (v_k - centroid_e) / h_e (k = 0..3)]    r_e: residual at the element's n_loc nodes,
 *           s = ||r_e||_2 (x's first part 0 when s = 0), h_e = |det J_e|^(1/3); n_in = n_loc + 12
 *   network y = W3 relu(W2 relu(W1 x + b1) + b2) + b3, hidden width MK_MLP_HIDDEN, n_out = n_loc
 *   precond z(node) = r(node)/A(node,node) + (sum over the node's (element, slot) incidences of y[slot] s/h_e)
 *                     / (number of incidences); boundary rows 0
 *   training sample (x, u, e): u = s/h_e, e = (x* - x_k) at the element's nodes for an iterate x_k of a solve
 *            with residual r_k and converged solution x*; loss L = sum_s ||u_s y_s - e_s||^2 / sum_s u_s^2
 *            (the network predicts the error normalised like its input), Adam updates.
 * Parameters are FP32, flattened in the order W1 [H][n_in], b1 [H], W2 [H][H], b2 [H], W3 [n_out][H],
 * b3 [n_out], row-major.  Inference in BF16 (inputs, weights and the two ReLU outputs rounded to BF16, products
 * accumulated in FP32 on the tensor cores (tcgen05), biases kept to about 2^-16 relative as high + low BF16 parts)
 * or FP32; training in FP32 with deterministic (fixed-order) gradient sums.  A BF16 call whose bounded wait for
 * its tensor-core work gives up sets MK_FAULT_TC_WAIT in the context's fault word (outputs invalid).
 * --------------------------------------------------------------------------------------------------------- */
#define MK_MLP_HIDDEN 64
enum { MK_MLP_FP32 = 0, MK_MLP_BF16 = 1 };

typedef struct {
  double lr, beta1, beta2, eps; /* Adam (Kingma & Ba); lr = 0: gradient only, no update */
} mk_adam;

/* Number of parameters for elements with n_loc nodes (4 or 10). */
int64_t mk_mlp_param_count(int nloc);
/* Create a network for n_loc-node elements from `params` (host, mk_mlp_param_count(nloc) floats).  Adam moments
 * start at zero.  The handle owns its device memory (freed by mk_mlp_destroy). */
int mk_mlp_create(mk_ctx* ctx, int nloc, const float* params, mk_mlp** out);
int mk_mlp_destroy(mk_mlp* mlp);
/* Copy the FP32 parameters to host `params` (save) or from host `params` into the network (load; resets Adam). */
int mk_mlp_save(const mk_mlp* mlp, float* params);
int mk_mlp_load(mk_mlp* mlp, const float* params);
/* Y[s] = network(X[s]) for S rows: X device float [S][n_in], Y device float [S][n_out]; precision MK_MLP_*. */
int mk_mlp_forward(mk_ctx* ctx, const mk_mlp* mlp, const float* X, int64_t S, float* Y, int precision, void* stream);
/* One training step on S samples (rows idx[0..S) of X [.][n_in], U [.], E [.][n_out], all device float; idx
 * device int32 or NULL for rows 0..S-1): loss and gradient of L over the batch (FP32 products, FP64 sums over
 * blocks in fixed order), then an Adam update unless opt is NULL or opt->lr == 0.  *loss (host) and, if given,
 * grad (device float [param_count]) receive the values before the update.  Synchronises the stream. */
int mk_mlp_train_step(mk_ctx* ctx, mk_mlp* mlp, const float* X, const float* U, const float* E,
                      const int32_t* idx, int64_t S, const mk_adam* opt, double* loss, float* grad, void* stream);
/* Training samples from one iterate of a solve on the fine mesh: for every element e (original order) and
 * column j < N, row e*N + j of X [E*N][n_in], U [E*N], E [E*N][n_out] (device float).  Rk, Xk, Xstar: device
 * double [n_nodes*ld] (residual and iterate at step k, converged solution). */
int mk_mlp_harvest(mk_ctx* ctx, const mk_mesh* mesh, const double* Rk, const double* Xk, const double* Xstar, int ld,
                   int N, float* X, float* U, float* E, void* stream);
/* z = learned preconditioner applied to r for the operator K/2 + M_{V_ext} + sigma M of `mol` (its diagonal
 * gives the Jacobi part): r, z device float [n_nodes*ld], columns j < N (others of z untouched). */
int mk_learned_precond(mk_ctx* ctx, const mk_mesh* mesh, const mk_mlp* mlp, const mk_molecule* mol, double sigma,
                       const float* r, float* z, int ld, int N, int precision, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MK_H */
