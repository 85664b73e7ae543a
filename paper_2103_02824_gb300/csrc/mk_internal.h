// Internal declarations of the mk library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mk.h"

namespace mk {

// Every kernel launch of the library goes through MK_COUNT() so callers can read how many ran (mk_launch_count).
extern std::atomic<long long> g_launch_count;
#define MK_COUNT() (::mk::g_launch_count.fetch_add(1, std::memory_order_relaxed))

// ------------------------------------------------------------------------------------------------ errors
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
// MK_ERR_TIMEOUT if a kernel on stream s set the context's device fault word (synchronises s).
int check_fault(mk_ctx* c, cudaStream_t s);

#define MK_CUDA(call)                                                                          \
  do {                                                                                         \
    cudaError_t _e = (call);                                                                   \
    if (_e != cudaSuccess)                                                                     \
      return ::mk::fail(MK_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e));       \
  } while (0)

#define MK_TRY(call)           \
  do {                         \
    int _r = (call);           \
    if (_r != MK_OK) return _r; \
  } while (0)

#define MK_ARG(cond, msg)                                                     \
  do {                                                                        \
    if (!(cond)) return ::mk::fail(MK_ERR_INVALID_ARG, std::string(msg));      \
  } while (0)

constexpr int kProfKinds = 6;   // PROF_* kinds timed by mk_profile_*
constexpr int kCapPairs = 128;  // event pairs per kind available to one graph capture
constexpr int kWaitLimitDefault = 1 << 20;  // the patch kernel's kWaitLimit
constexpr int kQ = 27;          // quadrature points per element (3x3x3 conical product, exact to degree 5)
constexpr int kMaxLoc = 10;     // P2
constexpr int kMaxPacked = 55;  // packed symmetric 10x10

// Packed upper-triangular index of (a,b), a<=b, for an n x n symmetric matrix.
__host__ __device__ inline int sym_index(int a, int b, int n) {
  if (a > b) { int t = a; a = b; b = t; }
  return a * n - a * (a - 1) / 2 + (b - a);
}

// Reference-element tables for one order (device copy lives in the context).
struct RefTables {
  int order, nloc, npack;
  double qw[kQ];                     // weights on the reference tetrahedron (sum 1/6)
  double qx[kQ][3];                  // points
  double phi[kQ][kMaxLoc];           // basis values at the points
  double mass[kMaxPacked];           // int_ref phi_a phi_b (packed)
  double stiff[6][kMaxPacked];       // int_ref (d_i phi_a d_j phi_b + [i!=j] d_j phi_a d_i phi_b), (ij) = 00,11,22,01,02,12
  double node_bary[kMaxLoc][4];      // barycentrics of the local nodes
};

void build_ref_tables(int order, RefTables* t);           // host: Gauss-Jacobi by Newton iteration
void gauss_jacobi_newton(int n, double a, double b, double* x, double* w);

// Per-element geometry (FP64): x = x0 + J xi.
struct Geom {
  double J[9];     // row-major J[r][c] = (x_{c+1} - x_0)_r
  double Jinv[9];
  double det;
  double x0[3];
};

struct Level {
  int order = 0, nloc = 0;
  int64_t n_vertices = 0, n_nodes = 0, n_free = 0, n_elems = 0;
  int n_colours = 0;
  // host copies (A0 results)
  std::vector<double> nodes;          // [n_nodes*3]
  std::vector<uint8_t> boundary;      // [n_nodes]
  std::vector<int32_t> elem;          // [E*nloc]
  std::vector<int32_t> colour;        // [E]
  std::vector<int32_t> free_idx;      // [n_free] node of each free DOF
  std::vector<int32_t> node_to_free;  // [n_nodes] free index or -1
  std::vector<int64_t> colour_off;    // [n_colours+1] into colour_elems
  std::vector<Geom> geom;             // [E]
  // device copies
  int32_t* d_elem = nullptr;
  int32_t* d_colour_elems = nullptr;  // element ids sorted by colour (stable)
  uint8_t* d_boundary = nullptr;
  int32_t* d_free_idx = nullptr;
  int32_t* d_node_to_free = nullptr;
  Geom* d_geom = nullptr;
  double* d_nodes = nullptr;          // [n_nodes*3]
};

// Element patches for the FP32 operator (owner-computes scatter with a fixed-order halo sum).
struct Patches {
  int n_patches = 0, max_elems = 0, max_nodes = 0;
  int64_t n_halo_slots = 0, n_shared_nodes = 0;
  int32_t* d_patch_elem_off = nullptr;   // [P+1] patch p owns patch-ordered elements [off[p], off[p+1])
  int32_t* d_patch_node_off = nullptr;   // [P+1] its local nodes are [off[p], off[p+1]) of the node arrays
  int32_t* d_elem_id = nullptr;          // [E] original element id of each patch-ordered element
  int32_t* d_conn = nullptr;             // [E*nloc] global nodes of the patch-ordered elements
  int32_t* d_node_target = nullptr;      // [sum nodes] >= 0: global node written directly (bit 30 set for a boundary
                                         // node); < 0: -(halo slot)-1
  int32_t* d_inc_off = nullptr;          // [sum nodes + 1] start of each local node's incidences (global index)
  uint16_t* d_inc = nullptr;             // [E*nloc] incidence = local slot * max_elems + local element, fixed order
  int32_t* d_shared_node = nullptr;      // [n_shared] global node of each shared node
  int32_t* d_shared_off = nullptr;       // [n_shared+1] its halo slots (one per patch, in patch order)
  // learned preconditioner inputs: per patch-ordered element (h_e, (v_k - centroid)/h_e for k = 0..3, 0, 0, 0)
  // with h_e = |det J|^(1/3); per node 1 / (number of (element, slot) incidences)
  float* d_geomf = nullptr;              // [E*16]
  float* d_inv_mult = nullptr;           // [n_nodes]
  int32_t* d_node_gid = nullptr;         // [sum nodes] global node of each local node
  uint16_t* d_lconn = nullptr;           // [E*nloc] local node index of each (patch-ordered element, slot)
  // one record per patch for the pipelined operator kernel (bulk-copied into shared memory in one piece), at byte
  // offset rec_off[p] (a multiple of 16): int32 header {e0, ne, n0, nl, off_pos, off_ioff, off_tgt, off_gid}, then
  // the local connectivity (uint16 [ne*nloc], at byte 32), the place of each (element, slot) incidence in the
  // patch's node-sorted incidence list (uint16 [ne*nloc]), the start of each local node's run in that list
  // (uint16 [nl+1]), the node targets (int32 [nl]) and the global ids of the local nodes (int32 [nl]); every
  // section starts on a 16-byte boundary
  unsigned char* d_rec = nullptr;
  int64_t* d_rec_off = nullptr;          // [P+1]: p * max_rec_bytes (every record padded to the same stride)
  int max_rec_bytes = 0;
  // matrix-free stiffness operator: per patch-ordered element |det J| (J^-1 J^-T)_{ij}, ij = 00,11,22,01,02,12, and
  // two zeros (computed on first use)
  mutable float* d_stiff_fac = nullptr;  // [E*8]
};
constexpr int kRecHeader = 32;
int patch_elems(int nloc);

// A CSR matrix on the device (FP32 values): rows [n_rows], off [n_rows + 1].
struct Csr32 {
  int64_t n_rows = 0, nnz = 0;
  int32_t* d_off = nullptr;
  int32_t* d_col = nullptr;
  float* d_val = nullptr;
};
// An intermediate level of the multigrid hierarchy of the Hartree Poisson solve: its mesh, the stiffness matrix on
// its interior nodes (node indexing, boundary rows empty), the inverse diagonal (boundary 0), the interpolation P
// from the next coarser level (rows: this level's nodes; columns: the coarser level's interior nodes, or the free
// DOF of V_H for the coarsest intermediate level) and its transpose R.
struct MgLevel {
  Level L;
  Csr32 K, P, R;
  float* d_dinv = nullptr;
  mutable float omega = 0.f;  // damped-Jacobi weight of the level's smoother (0 until estimated)
};

}  // namespace mk

struct mk_ctx {
  int device = 0;
  int n_sms = 0;
  int* d_fault = nullptr;  // device word: MK_FAULT_* bits set by kernels whose bounded waits gave up
  mk::RefTables* d_ref[3] = {nullptr, nullptr, nullptr};  // by order (1, 2)
  mk::RefTables h_ref[3];
  // scratch: named slots grown on demand
  std::vector<void*> slot_ptr;
  std::vector<size_t> slot_size;
  void* pinned = nullptr;  // small pinned host buffer for reports
  size_t pinned_size = 0;
  // optional CUDA-event timing of operator applications (mk_profile_*): [kind][2*i], [2*i+1] start/stop
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev[mk::kProfKinds];
  int prof_used[mk::kProfKinds] = {};
  // inside a CUDA-graph capture every application of a kind records its own event pair from a pool made before the
  // capture (cap_ev); the graph re-records them on every replay and prof_harvest adds their durations after it
  bool capturing = false;
  std::vector<cudaEvent_t> cap_ev[mk::kProfKinds];
  int cap_n[mk::kProfKinds] = {};
  double acc_ms[mk::kProfKinds] = {};
  long long acc_n[mk::kProfKinds] = {};
  // options (mk_ctx_set_option)
  bool no_graphs = false;       // MK_OPT_GRAPHS = 0: the inner PCG iterations run eagerly instead of replayed
  // MK_OPT_PATCH_PIPELINE: 1 = register-staged kernel (FP32) and two-group pipelined kernel (FP64), 2 = the two-group
  // pipelined kernel for FP32 too, 0 = the one-patch-per-CTA kernel
  int patch_kernel = 1;
  int wait_limit = mk::kWaitLimitDefault;  // MK_OPT_WAIT_LIMIT: polls of the patch kernel's bounded copy waits
  int decompose_ctas = 0;  // MK_OPT_DECOMPOSE_CTAS: CTAs of the block-Jacobi kernel (0 = one per SM)
  bool pair_residual = true;  // MK_OPT_PAIR_RESIDUAL: the mixed solves' refinement residuals on FP32 pairs
  const int* last_decompose_info = nullptr;  // device {sweeps64, buffer, -, -, sweeps32} of the last decomposition
  // the inner PCG runs on this stream (graphs cannot be captured on the legacy default stream), ordered against
  // the caller's stream by two events
  cudaStream_t solve_stream = nullptr;
  cudaEvent_t solve_ev[2] = {nullptr, nullptr};
};

// Learned preconditioner network: FP32 master parameters (flattened W1,b1,W2,b2,W3,b3), Adam moments, and the
// BF16 copy in the padded layout of the tensor-core kernels (W1 [64][40], W2 [64][72], W3 [16][72] halves,
// zero padded) with FP32 biases [64 + 64 + 16].
struct mk_mlp {
  mk_ctx* ctx = nullptr;
  int device = 0;  // kept here so that the handle can be destroyed after its context
  int nloc = 0, nin = 0, nout = 0;
  int64_t count = 0;
  float* d_w = nullptr;
  float* d_m = nullptr;
  float* d_v = nullptr;
  void* d_wb = nullptr;  // BF16 copy of the parameters in the tensor-core (tcgen05) operand layout
  long long t = 0;  // Adam steps taken
};

namespace mk {
// Record a start (begin=true) or stop event for profiled operation `kind` on stream s (no-op unless enabled).
void prof_mark(mk_ctx* ctx, int kind, bool begin, cudaStream_t s);
void prof_capture(mk_ctx* ctx, bool on);
void prof_prepare_capture(mk_ctx* ctx);
void prof_harvest(mk_ctx* ctx);
enum ProfKind { PROF_APPLY64 = 0, PROF_APPLY32 = 1, PROF_HALO = 2, PROF_LEARNED = 3, PROF_STIFF = 4, PROF_PAIRS = 5 };
}  // namespace mk

struct mk_mesh {
  mk_ctx* ctx = nullptr;
  int device = 0;  // kept here so that the handle can be destroyed after its context
  mk::Level fine, coarse;
  std::vector<int32_t> parent;
  // prolongation P: fine node -> coarse free DOF (CSR over fine nodes)
  int32_t* d_P_off = nullptr;
  int32_t* d_P_col = nullptr;
  double* d_P_val = nullptr;
  // restriction P^T: coarse free DOF -> fine nodes (CSR over coarse free DOF, fine nodes increasing)
  int32_t* d_PT_off = nullptr;
  int32_t* d_PT_col = nullptr;
  double* d_PT_val = nullptr;
  int64_t PT_nnz = 0;
  // children of each coarse element (CSR, fine element ids increasing)
  int32_t* d_child_off = nullptr;
  int32_t* d_child = nullptr;
  mk::Patches patches;
  // M_H = P^T M P depends on the meshes only (it stays fixed, like the paper's M_H): its inverse Cholesky factor
  // Linv = L^-1 (M_H = L L^T), dense row-major [N_H*N_H], is computed once at upload.
  double* d_MH_Linv = nullptr;
  // K/2 + M_{V_ext} element matrices (FP64, element order) for the molecule in static_key (see static_matrices)
  mutable double* d_static = nullptr;
  mutable std::vector<double> static_key;
  mutable cudaEvent_t static_ev = nullptr;  // recorded after the set was written
  // M element matrices (FP64, element order), built on first use, and the event recorded after they were written
  mutable double* d_M64 = nullptr;
  mutable cudaEvent_t mass_ev = nullptr;
  // two-level preconditioner (built on first use): FP32 values of P and P^T, and FP32 dense inverses of the
  // Galerkin coarse operators P^T K P (Poisson) and P^T (K/2 + M_Vext + sigma M) P (the key: molecule, sigma)
  mutable float* d_P_val32 = nullptr;
  mutable float* d_PT_val32 = nullptr;
  mutable float* d_cinv_poisson = nullptr;
  // the Hartree Poisson operator: stiffness element matrices (FP64, element order) and K's diagonal, on first use
  mutable double* d_K64 = nullptr;
  mutable double* d_K64diag = nullptr;
  // face neighbours of the fine mesh for the error indicator (built on first use): for element e and face slot k
  // (the face opposite local vertex k), 4 e' + k' of the element across it, or -1 on the boundary
  mutable int32_t* d_face_nb = nullptr;
  mutable float* d_cinv_corr = nullptr;
  mutable std::vector<double> cinv_corr_key;
  // multigrid hierarchy (mk_mesh_set_hierarchy): intermediate levels coarsest first, and the interpolation from the
  // finest intermediate level (or from V_H when there is none) into the fine mesh with its transpose
  std::vector<mk::MgLevel> mg;
  mk::Csr32 mgP, mgR;
  bool has_mg = false;
  // damped-Jacobi weight of the fine-level smoother of the Poisson preconditioners (0 until estimated)
  mutable float poisson_omega = 0.f;
};

namespace mk {

// scratch slots
enum Slot : int {
  S_ELEM64 = 0,   // element matrices FP64 [E*55]
  S_ELEM64B,      // second FP64 element matrix set
  S_ELEM32,       // FP32 element matrices (patch order)
  S_DIAG64,       // Jacobi diagonal FP64 [n_nodes]
  S_DIAG32,
  S_R64, S_Z64, S_P64, S_Q64,   // PCG vectors FP64 [n_nodes*ld]
  S_R32, S_P32, S_Q32, S_X32,   // PCG vectors FP32
  S_HALO,         // halo partial sums
  S_RED,          // reduction partials
  S_SCAL,         // per-column scalars (device)
  S_RHO,          // rho at quadrature points
  S_VEC1, S_VEC2, S_VEC3,       // misc fine vectors
  S_EIG,          // eigensolver workspace
  S_COARSE,       // coarse element matrices
  S_NUC,          // nuclei (Z, R)
  S_OCC,          // occupations
  S_COEF,         // small per-column coefficient arrays
  S_VEC4, S_VEC5,
  S_GRAM,
  S_ELEM64C, S_ELEM64D,         // element matrices of the coarse-pencil path (may run on another stream)
  S_NUC2, S_COARSE2,
  S_EIG2,                       // workspace of the shared coarse decomposition
  S_EIG3, S_EIG4,               // general (unshared) eigensolve: factor + decomposition, Cholesky workspace
  S_HALO64,                     // halo partial sums of the FP64 patch operator
  S_OPA, S_OPB,                 // element matrices of mk_operator_apply (FP64 original order, patch order)
  S_Z32,                        // FCG preconditioned residual (FP32)
  S_LHALO,                      // halo partial sums of the learned preconditioner
  S_MLPPART, S_MLPGRAD,         // training: per-block gradient partials, reduced gradient
  S_LDINV,                      // mk_learned_precond: FP64 diagonal, FP32 inverse
  S_TLC, S_TLX, S_TLW,          // two-level setup: coarse element products, coarse matrices, Cholesky workspace
  S_TLT,                        // two-level apply: restricted residual and coarse solution (FP32)
  S_TLQ,                        // multiplicative two-level: the operator product A z (FP32)
  S_FINCTR,                     // arrival counter of the fused reductions of the mixed solve
  S_ELEMP64,                    // FP64 element matrices in patch order (apply64)
  S_BATCH,                      // batched solve: per-problem buffers
  S_JOINT, S_EIG5,              // joint augmented space: its matrices, its dense decompositions
  S_MG,                         // multigrid V-cycle: per-level right-hand sides, iterates, operator products
  S_AFEM,                       // error indicator: face values; Dorfler marking: reduction partials
  S_LMAX,                       // smoother weight estimate: the power iteration's two vectors (FP32)
  S_PAIRA,                      // FP32-pair parts of the mixed solve's element matrices (hi, lo; patch order)
  S_PAIRX,                      // FP32-pair parts of an FP64 operand (hi, lo)
  S_COUNT
};
void* scratch(mk_ctx* ctx, int slot, size_t bytes, int* err);
void free_csr(Csr32& c);
// element patches of the fine mesh (mk_patches.cpp): pe elements per patch, 0 = the default for the order
int build_patches(mk_mesh* m, int pe = 0);
void free_patches(Patches& p);

}  // namespace mk
