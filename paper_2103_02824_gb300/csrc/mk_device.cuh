// Device building blocks shared by the mk translation units.
#pragma once

#include <cuda_runtime.h>

#include "mk_internal.h"

namespace mk {

constexpr int kRedBlocksPerSM = 2;
constexpr int kRedThreads = 256;

inline int red_blocks(const mk_ctx* ctx) { return ctx->n_sms * kRedBlocksPerSM; }

// Small per-call arrays travel as kernel parameters (no device allocation, no host synchronisation).
constexpr int kMaxNuclei = 64;
struct NucParams {
  int n;
  double v[4 * kMaxNuclei];  // (Z, x, y, z) per nucleus
};
struct ColParams {
  double v[MK_MAX_RHS];
};

inline NucParams make_nuc(const mk_molecule* mol) {
  NucParams p{};
  p.n = mol ? mol->n_nuclei : 0;
  for (int k = 0; k < p.n && k < kMaxNuclei; ++k) {
    p.v[4 * k] = mol->Z[k];
    for (int c = 0; c < 3; ++c) p.v[4 * k + 1 + c] = mol->R[3 * k + c];
  }
  return p;
}

__device__ __forceinline__ double nuclear_potential(const NucParams& P, double x, double y, double z) {
  double v = 0.0;
  for (int k = 0; k < P.n; ++k) {
    double dx = x - P.v[4 * k + 1], dy = y - P.v[4 * k + 2], dz = z - P.v[4 * k + 3];
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    v -= P.v[4 * k] / fmax(r, 1e-8);
  }
  return v;
}

// y[node(e,a)][j] += sum_b A_e[a][b] x[node(e,b)][j] for the elements of one colour (no two share a node, so the
// read-modify-write scatter needs no atomics and the summation order is fixed: colour by colour).
template <int NLOC, typename T>
__global__ void k_apply_colour(const int32_t* __restrict__ celems, int count, const int32_t* __restrict__ elem,
                               const T* __restrict__ Ae, const T* __restrict__ x, T* __restrict__ y, int N, int ld) {
  constexpr int NP = NLOC * (NLOC + 1) / 2;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)count * N) return;
  const int i = (int)(t / N), j = (int)(t % N);
  const int e = celems[i];
  int nd[NLOC];
  T xv[NLOC];
#pragma unroll
  for (int a = 0; a < NLOC; ++a) {
    nd[a] = elem[(int64_t)e * NLOC + a];
    xv[a] = x[(int64_t)nd[a] * ld + j];
  }
  const T* A = Ae + (int64_t)e * NP;
#pragma unroll
  for (int a = 0; a < NLOC; ++a) {
    T s = 0;
#pragma unroll
    for (int b = 0; b < NLOC; ++b) s += A[sym_index(a, b, NLOC)] * xv[b];
    y[(int64_t)nd[a] * ld + j] += s;
  }
}

// Launches the colour sweep y += A x (y must hold its starting value).
template <typename T>
inline void apply_coloured(const Level& L, const T* Ae, const T* x, T* y, int N, int ld, cudaStream_t s) {
  const int th = 256;
  for (int c = 0; c < L.n_colours; ++c) {
    const int64_t off = L.colour_off[c], cnt = L.colour_off[c + 1] - off;
    const int64_t work = cnt * N;
    const int blocks = (int)((work + th - 1) / th);
    if (L.nloc == 4)
      MK_COUNT(), k_apply_colour<4, T><<<blocks, th, 0, s>>>(L.d_colour_elems + off, (int)cnt, L.d_elem, Ae, x, y, N, ld);
    else
      MK_COUNT(), k_apply_colour<10, T><<<blocks, th, 0, s>>>(L.d_colour_elems + off, (int)cnt, L.d_elem, Ae, x, y, N, ld);
  }
}

// Column-wise partial dot products over all nodes: part[blk*N + j] = sum_{nodes in blk's stride} a[n][j]*b[n][j].
// Deterministic: fixed grid, fixed node->thread map, fixed reduction tree.
template <typename T>
__global__ void k_dot_partial(int64_t n_nodes, const T* __restrict__ a, const T* __restrict__ b, int N, int ld,
                              double* __restrict__ part) {
  extern __shared__ double sh[];
  const int rows = blockDim.x / N;  // node rows handled per pass
  const int r = threadIdx.x / N, j = threadIdx.x % N;
  double acc = 0.0;
  if (r < rows) {
    for (int64_t nd = (int64_t)blockIdx.x * rows + r; nd < n_nodes; nd += (int64_t)gridDim.x * rows)
      acc += (double)a[nd * ld + j] * (double)b[nd * ld + j];
  }
  sh[threadIdx.x] = (r < rows) ? acc : 0.0;
  __syncthreads();
  int top = 1;
  while (top < rows) top <<= 1;
  for (int st = top >> 1; st > 0; st >>= 1) {  // fixed pairwise tree over the rows of each column
    if (r < st && r + st < rows) sh[threadIdx.x] += sh[threadIdx.x + st * N];
    __syncthreads();
  }
  if (threadIdx.x < N) part[(int64_t)blockIdx.x * N + threadIdx.x] = sh[threadIdx.x];
}

// Sums partials in block order: out[j] = sum_blk part[blk*N + j].
__global__ void k_sum_partials(const double* __restrict__ part, int nblk, int N, double* __restrict__ out);
void sum_partials(const double* part, int nblk, int N, double* out, cudaStream_t s);

int column_dots(mk_ctx* ctx, int64_t n_nodes, const double* a, const double* b, int N, int ld, double* out,
                cudaStream_t s);
int column_dots32(mk_ctx* ctx, int64_t n_nodes, const float* a, const float* b, int N, int ld, double* out,
                  cudaStream_t s);

// element matrices (packed, FP64) of half_k K + vext_scale M_{V_ext} + mass_shift M + M_{vq}
int element_matrices(mk_ctx* ctx, const Level& L, const mk_molecule* mol, double half_k, double vext_scale,
                     double mass_shift, const double* vq, double* out, cudaStream_t s,
                     const double* base = nullptr);
// cached M element matrices of the fine mesh (nullptr and *err set on failure)
const double* mass_matrices(mk_ctx* ctx, const mk_mesh* m, cudaStream_t s, int* err);
// cached K/2 + M_{V_ext} element matrices of the fine mesh for a molecule (nullptr and *err set on failure)
const double* static_matrices(mk_ctx* ctx, const mk_mesh* m, const mk_molecule* mol, cudaStream_t s, int* err);
// assembled diagonal of the packed element matrices, boundary rows set to 1
int assemble_diagonal(mk_ctx* ctx, const Level& L, const double* Ae, double* diag, cudaStream_t s);
// y = A x on the fine mesh (all ld columns) with the FP64 patch operator, from element matrices Ae in element
// order; boundary rows of y zeroed if mask_boundary
int apply64(mk_ctx* ctx, const mk_mesh* m, const double* Ae, const double* x, double* y, int N, int ld,
            bool mask_boundary, cudaStream_t s);
// the patch operator (mk_mixed.cu): element matrices packed in patch order, then y = A x
template <typename T>
int pack_elements(mk_ctx* ctx, const mk_mesh* m, const double* A64, T* A, cudaStream_t s);
template <typename T>
int apply_patch(mk_ctx* ctx, const mk_mesh* m, const T* Ae, const T* x, T* y, int ld, bool mask, cudaStream_t s);

// out = (float) (P^T A P)^-1, the dense inverse of the Galerkin coarse operator of the fine element matrices A64
// (synchronises s: the Cholesky factorisation reports a matrix that is not positive definite)
int coarse_inverse32(mk_ctx* ctx, const mk_mesh* m, const double* A64, float* out, cudaStream_t s);
// FP32 values of P and P^T for the two-level preconditioner (once per mesh)
int tl_prepare(const mk_mesh* m, cudaStream_t s);
// cached FP32 coarse inverse (P^T A P)^-1: key NULL = the mesh's Poisson operator, else (sigma, molecule)
const float* coarse_inverse_cached(mk_ctx* ctx, const mk_mesh* m, const double* A64, const std::vector<double>* key,
                                   cudaStream_t s, int* err);
// dinv = (float)(1 / diag)
int diag_inverse32(int64_t n, const double* diag, float* dinv, cudaStream_t s);
// z = learned preconditioner of r (FP32, columns < N); dinv: FP32 inverse diagonal of the operator
int learned_apply(mk_ctx* ctx, const mk_mesh* m, const mk_mlp* mlp, const float* dinv, const float* r, float* z,
                  int ld, int N, int precision, cudaStream_t s);

}  // namespace mk
