// The paper's own form of the correction step's last stage: the nonlinear eigenproblem in V_H + span{phi~_i}
// (Eq. (Nonlinear_Eig_Hh_Full)) solved by the inner SCF iteration of Algorithm 2, with the precomputations of
// Algorithm 3 so that an inner iteration touches coarse-sized data only.
//
// mk_inner_create (Algorithm 3, step 1) integrates, once, on the fine mesh:
//   A1 = P^T H1 P, b1_i = P^T H1 phi~_i, beta1_i = (H1 phi~_i, phi~_i)  with H1 = K/2 + V_ext + V_xc + w_b,
//   A3 = P^T M_{w~0} P (the paper's G), b3_i = P^T M_{w~0} phi~_i (its F_i), beta3_i, and c_i, gamma_i, M_H;
//   the Hartree system in W = V_H + span{w~0}: C_H = P^T K P, d = P^T K w~0, zeta = (K w~0, w~0) and the lifts of
//   the boundary values w_b; and per coarse element T the tensors of its basis functions psi_a on the fine
//   quadrature of its children: (psi_a psi_b, psi_c)_T, (phi~_i psi_a, psi_b)_T (the paper's A_h4), (phi~_i^2,
//   psi_a)_T (its rhs) and (w~0, phi~_i^2).
// mk_inner_run (Algorithm 2) then iterates, for s = 1, 2, ...:
//   (a) A_H = A1 + A_H2(w_H) + theta_1 A3 with A_H2 = (w_H psi_k, psi_j) from the tensor, b_i and beta_i likewise,
//       one coarse decomposition and the per-orbital secular solves (the eigenvector with the largest component
//       along phi~_i);
//   (b) the Hartree potential w_b + w_H + theta_1 w~0 of the new orbitals' density, from the coarse tensors and
//       one solve of the bordered system (C_H, d; d^T, zeta) through C_H^-1 and its Schur complement;
//   (c) stop when no orbital coefficient changed by more than tol.
// The inner Hartree coefficients are mixed, (w_H, theta_1) <- (1 - mix) old + mix new.  Every sum runs in a fixed
// order (children, quadrature points, coarse colours), so a run is bitwise reproducible.
#include <cmath>
#include <vector>

#include "mk_device.cuh"

namespace mk {

int coarse_matrices(mk_ctx*, const mk_mesh*, const double*, const double*, double*, double*, int, cudaStream_t);
int restrict_to_coarse(mk_ctx*, const mk_mesh*, const double*, int, int, double*, int, cudaStream_t);
int inverse_cholesky(mk_ctx* ctx, int n, const double* MH, double* Linv, int slot, cudaStream_t s);
int decompose(mk_ctx* ctx, int n, const double* X, bool w_is_x, const double* AH, double* d, double* V,
              cudaStream_t s, int slot);
int secular(mk_ctx* ctx, int n, int N, const double* d, const double* V, const double* b, const double* c,
            const double* beta, const double* gamma, double* lambda, double* coef, int32_t* status, cudaStream_t s);
int gram(mk_ctx* ctx, int64_t n, const double* X, const double* Y, int N, int ld, double* G, cudaStream_t s);

// scalars of the inner iteration kept on the device
enum InnerScalar { IS_THETA1 = 0, IS_THETA1_NEW, IS_DELTA, IS_ZETA, IS_DY, IS_LIFT0, IS_COUNT };

}  // namespace mk

struct mk_inner {
  mk_ctx* ctx = nullptr;
  const mk_mesh* mesh = nullptr;
  int device = 0;
  int NH = 0, N = 0, nl = 0;
  int64_t Ec = 0, n_nodes = 0;
  bool w_in_VH = false;      // w~0 lies in V_H: the extra Hartree direction is dropped (theta_1 = 0)
  double schur = 0.0, lift0 = 0.0;
  void* arena = nullptr;
  // fixed data (Algorithm 3, step 1)
  double *A1, *A3, *b1, *b3, *beta1, *beta3, *c, *gamma;
  double *Tc, *Ah4, *rvec, *g3, *CHinv, *y, *liftH, *wb, *w0;
  // state of the iteration
  double *AH, *b, *beta, *d, *V[2], *lam, *coef, *prev, *wH, *fH, *rH, *gpart, *sc;
  int32_t* status;
};

namespace mk {

constexpr int kInThreads = 256;
constexpr int kInChunks = 16;  // CTAs per coarse element in the tensor precomputation

__device__ __forceinline__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// out[e*Q+q] = (add ? add[e*Q+q] : 0) + w(x_q), w a nodal function of the fine mesh
template <int NLOC>
__global__ void k_in_at_quad(int64_t E, const RefTables* __restrict__ ref, const int32_t* __restrict__ elem,
                             const double* __restrict__ w, const double* __restrict__ add, double* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  double wa[NLOC];
#pragma unroll
  for (int a = 0; a < NLOC; ++a) wa[a] = w[elem[e * NLOC + a]];
  for (int q = 0; q < kQ; ++q) {
    double v = 0.0;
#pragma unroll
    for (int a = 0; a < NLOC; ++a) v += ref->phi[q][a] * wa[a];
    out[e * kQ + q] = (add ? add[e * kQ + q] : 0.0) + v;
  }
}

// w~ = w_b + w~0: the boundary values (zero inside) and the rest (zero on the boundary)
__global__ void k_in_split(int64_t n, const uint8_t* __restrict__ bnd, const double* __restrict__ wt,
                           double* __restrict__ wb, double* __restrict__ w0) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  wb[i] = bnd[i] ? wt[i] : 0.0;
  w0[i] = bnd[i] ? 0.0 : wt[i];
}

// Coarse basis function b of the parent (geometry cg) at the physical point x.
template <int NLOC>
__device__ __forceinline__ void coarse_basis_at(const Geom& cg, const double x[3], double* psi) {
  double s[3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
    s[r] = cg.Jinv[r * 3] * (x[0] - cg.x0[0]) + cg.Jinv[r * 3 + 1] * (x[1] - cg.x0[1]) +
           cg.Jinv[r * 3 + 2] * (x[2] - cg.x0[2]);
  const double l[4] = {1.0 - s[0] - s[1] - s[2], s[0], s[1], s[2]};
  if (NLOC == 4) {
#pragma unroll
    for (int b = 0; b < 4; ++b) psi[b] = l[b];
  } else {
#pragma unroll
    for (int b = 0; b < 4; ++b) psi[b] = l[b] * (2.0 * l[b] - 1.0);
    const int ea[6] = {0, 0, 0, 1, 1, 2}, eb[6] = {1, 2, 3, 2, 3, 3};
#pragma unroll
    for (int k = 0; k < 6; ++k) psi[4 + k] = 4.0 * l[ea[k]] * l[eb[k]];
  }
}

// One block per coarse element T: over its children (fixed order) and their quadrature points, the tensors
//   Tc[T][a][b][c] = (psi_a psi_b, psi_c),  Ah4[i][T][a][b] = (phi~_i psi_a, psi_b),  rc[i][T][a] = (phi~_i^2, psi_a),
//   g3p[T][i] = (w~0, phi~_i^2) restricted to T,
// psi the basis functions of T, phi~_i and w~0 fine nodal functions.  The accumulators (the concatenated outputs,
// in_tensor_count of them) live in dynamic shared memory; entry t belongs to thread t mod blockDim.
__host__ __device__ inline int in_tensor_count(int nl, int N) { return nl * nl * nl + N * (nl * nl + nl + 1); }
template <int NLOC>
__global__ void __launch_bounds__(kInThreads) k_in_tensors(const int32_t* __restrict__ child_off,
                                                           const int32_t* __restrict__ child,
                                                           const Geom* __restrict__ fgeom,
                                                           const int32_t* __restrict__ felem,
                                                           const Geom* __restrict__ cgeom,
                                                           const RefTables* __restrict__ ref,
                                                           const double* __restrict__ phit, int ld, int N,
                                                           const double* __restrict__ w0, int nchunk,
                                                           double* __restrict__ part) {
  constexpr int NL2 = NLOC * NLOC, NL3 = NL2 * NLOC;
  __shared__ double ps[kQ][NLOC];
  __shared__ double wd[kQ], wq[kQ];
  __shared__ double ph[kQ][MK_MAX_RHS];
  extern __shared__ double acc[];
  // block = (coarse element T, chunk ch of its children); the chunks' partial sums are added in chunk order later
  const int T = blockIdx.x / nchunk, ch = blockIdx.x % nchunk;
  const Geom cg = cgeom[T];
  const int K = in_tensor_count(NLOC, N);
  for (int t = threadIdx.x; t < K; t += blockDim.x) acc[t] = 0.0;
  const int c0 = child_off[T], len = child_off[T + 1] - c0;
  const int kb = c0 + (int)((int64_t)len * ch / nchunk), ke = c0 + (int)((int64_t)len * (ch + 1) / nchunk);
#pragma unroll 1
  for (int k = kb; k < ke; ++k) {
    const int64_t e = child[k];
    if ((int)threadIdx.x < kQ) {
      const Geom g = fgeom[e];
      const int q = threadIdx.x;
      const double xi = ref->qx[q][0], et = ref->qx[q][1], ze = ref->qx[q][2];
      double x[3];
      for (int r = 0; r < 3; ++r) x[r] = g.x0[r] + g.J[r * 3] * xi + g.J[r * 3 + 1] * et + g.J[r * 3 + 2] * ze;
      double psi[NLOC];
      coarse_basis_at<NLOC>(cg, x, psi);
      for (int a = 0; a < NLOC; ++a) ps[q][a] = psi[a];
      wd[q] = ref->qw[q] * fabs(g.det);
      double v = 0.0;
      for (int a = 0; a < NLOC; ++a) v += ref->phi[q][a] * w0[felem[e * NLOC + a]];
      wq[q] = v;
    }
    for (int t = threadIdx.x; t < kQ * N; t += blockDim.x) {
      const int q = t / N, i = t - q * N;
      double v = 0.0;
      for (int a = 0; a < NLOC; ++a) v += ref->phi[q][a] * phit[(int64_t)felem[e * NLOC + a] * ld + i];
      ph[q][i] = v;
    }
    __syncthreads();
#pragma unroll 1
    for (int t0 = threadIdx.x; t0 < K; t0 += blockDim.x) {
      int t = t0;
      double s = 0.0;
      if (t < NL3) {
        const int a = t / NL2, b = (t / NLOC) % NLOC, c = t % NLOC;
        for (int q = 0; q < kQ; ++q) s += wd[q] * ps[q][a] * ps[q][b] * ps[q][c];
      } else if ((t -= NL3) < N * NL2) {
        const int i = t / NL2, a = (t / NLOC) % NLOC, b = t % NLOC;
        for (int q = 0; q < kQ; ++q) s += wd[q] * ph[q][i] * ps[q][a] * ps[q][b];
      } else if ((t -= N * NL2) < N * NLOC) {
        const int i = t / NLOC, a = t % NLOC;
        for (int q = 0; q < kQ; ++q) s += wd[q] * ph[q][i] * ph[q][i] * ps[q][a];
      } else {
        const int i = t - N * NLOC;
        for (int q = 0; q < kQ; ++q) s += wd[q] * wq[q] * ph[q][i] * ph[q][i];
      }
      acc[t0] += s;
    }
    __syncthreads();
  }
  for (int t0 = threadIdx.x; t0 < K; t0 += blockDim.x) part[(int64_t)blockIdx.x * K + t0] = acc[t0];
}

// the chunks of every coarse element summed in chunk order, into the tensors' layouts:
//   Tc[T][a][b][c], Ah4[i][T][a][b], rc[i][T][a], g3p[T][i]
template <int NLOC>
__global__ void k_in_tensor_reduce(int64_t Ec, int N, int nchunk, const double* __restrict__ part,
                                   double* __restrict__ Tc, double* __restrict__ Ah4, double* __restrict__ rc,
                                   double* __restrict__ g3p) {
  constexpr int NL2 = NLOC * NLOC, NL3 = NL2 * NLOC;
  const int K = in_tensor_count(NLOC, N);
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Ec * K) return;
  const int64_t T = g / K;
  int t = (int)(g - T * K);
  double v = 0.0;
  for (int c = 0; c < nchunk; ++c) v += part[(T * nchunk + c) * K + t];
  if (t < NL3) {
    Tc[T * NL3 + t] = v;
  } else if ((t -= NL3) < N * NL2) {
    const int i = t / NL2;
    Ah4[((int64_t)i * Ec + T) * NL2 + (t - i * NL2)] = v;
  } else if ((t -= N * NL2) < N * NLOC) {
    const int i = t / NLOC;
    rc[((int64_t)i * Ec + T) * NLOC + (t - i * NLOC)] = v;
  } else {
    g3p[T * N + (t - N * NLOC)] = v;
  }
}

// rvec[f_a][i] += rc[i][T][a] over the coarse elements of one colour (no two share a node)
template <int NLOC>
__global__ void k_in_rc_scatter(const int32_t* __restrict__ celems, int count, const int32_t* __restrict__ elem,
                                const int32_t* __restrict__ n2f, int64_t Ec, int N, const double* __restrict__ rc,
                                double* __restrict__ rvec) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)count * NLOC * N) return;
  const int k = (int)(t / (NLOC * N)), r = (int)(t % (NLOC * N));
  const int a = r / N, i = r % N;
  const int T = celems[k];
  const int fa = n2f[elem[(int64_t)T * NLOC + a]];
  if (fa < 0) return;
  rvec[(int64_t)fa * N + i] += rc[((int64_t)i * Ec + T) * NLOC + a];
}

__global__ void k_in_g3(int64_t Ec, int N, const double* __restrict__ g3p, double* __restrict__ g3) {
  const int i = threadIdx.x;
  if (i >= N) return;
  double s = 0.0;
  for (int64_t T = 0; T < Ec; ++T) s += g3p[T * N + i];
  g3[i] = s;
}

// out = Li^T Li for the lower-triangular Li = L^-1 (so out = (L L^T)^-1)
__global__ void k_in_ltl(int n, const double* __restrict__ Li, double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  double s = 0.0;
  for (int k = i > j ? i : j; k < n; ++k) s += Li[(int64_t)k * n + i] * Li[(int64_t)k * n + j];
  out[t] = s;
}

// y = A x (n x n, row-major), one warp per row
__global__ void k_in_gemv(int n, const double* __restrict__ A, const double* __restrict__ x, double* __restrict__ y) {
  const int row = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32), lane = threadIdx.x % 32;
  if (row >= n) return;
  double s = 0.0;
  for (int k = lane; k < n; k += 32) s += A[(int64_t)row * n + k] * x[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = s;
}

// sc[IS_DY] = d^T y (one block)
__global__ void k_in_dot(int n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out) {
  __shared__ double sh[kInThreads];
  double v = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) v += a[k] * b[k];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) *out = v;
}

// (a) A_H = A1 + theta_1 A3, b = b1 + theta_1 b3 (the A_H2 terms are added per colour)
__global__ void k_in_init(int NH, int N, const double* __restrict__ A1, const double* __restrict__ A3,
                          const double* __restrict__ b1, const double* __restrict__ b3, const double* __restrict__ sc,
                          double* __restrict__ AH, double* __restrict__ b) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nA = (int64_t)NH * NH, nb = (int64_t)NH * N;
  const double th = sc[IS_THETA1];
  if (t < nA) AH[t] = A1[t] + th * A3[t];
  else if (t < nA + nb) b[t - nA] = b1[t - nA] + th * b3[t - nA];
}

// beta_i = beta1_i + theta_1 beta3_i + (phi~_i^2, w_H), one block per orbital
__global__ void k_in_beta(int NH, int N, const double* __restrict__ rvec, const double* __restrict__ wH,
                          const double* __restrict__ beta1, const double* __restrict__ beta3,
                          const double* __restrict__ sc, double* __restrict__ beta) {
  __shared__ double sh[kInThreads];
  const int i = blockIdx.x;
  double v = 0.0;
  for (int j = threadIdx.x; j < NH; j += blockDim.x) v += rvec[(int64_t)j * N + i] * wH[j];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) beta[i] = beta1[i] + sc[IS_THETA1] * beta3[i] + v;
}

// the coarse free index of local node a of coarse element T, or -1
__device__ __forceinline__ int free_of(const int32_t* elem, const int32_t* n2f, int T, int a, int nloc) {
  return n2f[elem[(int64_t)T * nloc + a]];
}

// (a) per colour: A_H[f_a][f_b] += sum_c Tc[T][a][b][c] w_H[f_c];  b[f_a][i] += sum_b Ah4[i][T][a][b] w_H[f_b]
template <int NLOC>
__global__ void k_in_scatter_ab(const int32_t* __restrict__ celems, int count, const int32_t* __restrict__ elem,
                                const int32_t* __restrict__ n2f, int64_t Ec, int NH, int N,
                                const double* __restrict__ Tc, const double* __restrict__ Ah4,
                                const double* __restrict__ wH, double* __restrict__ AH, double* __restrict__ b) {
  constexpr int NL2 = NLOC * NLOC;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nA = (int64_t)count * NL2;
  if (t >= nA + (int64_t)count * NLOC * N) return;
  double wl[NLOC];
  if (t < nA) {
    const int k = (int)(t / NL2), ab = (int)(t % NL2), a = ab / NLOC, bb = ab % NLOC;
    const int T = celems[k];
    const int fa = free_of(elem, n2f, T, a, NLOC), fb = free_of(elem, n2f, T, bb, NLOC);
    if (fa < 0 || fb < 0) return;
#pragma unroll
    for (int c = 0; c < NLOC; ++c) {
      const int fc = free_of(elem, n2f, T, c, NLOC);
      wl[c] = fc >= 0 ? wH[fc] : 0.0;
    }
    const double* tc = Tc + (int64_t)T * NL2 * NLOC + ab * NLOC;
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < NLOC; ++c) s += tc[c] * wl[c];
    AH[(int64_t)fa * NH + fb] += s;
  } else {
    const int64_t u = t - nA;
    const int k = (int)(u / (NLOC * N)), r = (int)(u % (NLOC * N)), a = r / N, i = r % N;
    const int T = celems[k];
    const int fa = free_of(elem, n2f, T, a, NLOC);
    if (fa < 0) return;
#pragma unroll
    for (int c = 0; c < NLOC; ++c) {
      const int fc = free_of(elem, n2f, T, c, NLOC);
      wl[c] = fc >= 0 ? wH[fc] : 0.0;
    }
    const double* h = Ah4 + ((int64_t)i * Ec + T) * NL2 + a * NLOC;
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < NLOC; ++c) s += h[c] * wl[c];
    b[(int64_t)fa * N + i] += s;
  }
}

// (b) fH[j] = sum_i f_i theta_2i^2 (phi~_i^2, psi_j)  (the coarse-coarse and mixed terms are added per colour)
__global__ void k_in_fh_init(int NH, int N, const double* __restrict__ rvec, const double* __restrict__ coef,
                             const ColParams occ, double* __restrict__ fH) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= NH) return;
  double s = 0.0;
  for (int i = 0; i < N; ++i) {
    const double t2 = coef[(int64_t)NH * N + i];
    s += occ.v[i] * t2 * t2 * rvec[(int64_t)j * N + i];
  }
  fH[j] = s;
}

// (b) per colour: fH[f_a] += sum_i f_i (sum_{b,c} Tc[T][a][b][c] p_ib p_ic + 2 theta_2i sum_b Ah4[i][T][a][b] p_ib),
// p_i = phi_{i,H} at the nodes of T
template <int NLOC>
__global__ void k_in_scatter_fh(const int32_t* __restrict__ celems, int count, const int32_t* __restrict__ elem,
                                const int32_t* __restrict__ n2f, int64_t Ec, int NH, int N,
                                const double* __restrict__ Tc, const double* __restrict__ Ah4,
                                const double* __restrict__ coef, const ColParams occ, double* __restrict__ fH) {
  constexpr int NL2 = NLOC * NLOC;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)count * NLOC) return;
  const int k = (int)(t / NLOC), a = (int)(t % NLOC);
  const int T = celems[k];
  const int fa = free_of(elem, n2f, T, a, NLOC);
  if (fa < 0) return;
  int fl[NLOC];
#pragma unroll
  for (int c = 0; c < NLOC; ++c) fl[c] = free_of(elem, n2f, T, c, NLOC);
  const double* tc = Tc + (int64_t)T * NL2 * NLOC + a * NL2;
  double s = 0.0;
  for (int i = 0; i < N; ++i) {
    double p[NLOC];
#pragma unroll
    for (int c = 0; c < NLOC; ++c) p[c] = fl[c] >= 0 ? coef[(int64_t)fl[c] * N + i] : 0.0;
    double q = 0.0;
#pragma unroll
    for (int bb = 0; bb < NLOC; ++bb) {
      double r = 0.0;
#pragma unroll
      for (int c = 0; c < NLOC; ++c) r += tc[bb * NLOC + c] * p[c];
      q += r * p[bb];
    }
    const double* h = Ah4 + ((int64_t)i * Ec + T) * NL2 + a * NLOC;
    double m = 0.0;
#pragma unroll
    for (int bb = 0; bb < NLOC; ++bb) m += h[bb] * p[bb];
    s += occ.v[i] * (q + 2.0 * coef[(int64_t)NH * N + i] * m);
  }
  fH[fa] += s;
}

// (b) gpart[i] = f_i (phi_iH^T A3 phi_iH + 2 theta_2i b3_i^T phi_iH + theta_2i^2 g3_i), one block per orbital
__global__ void k_in_g(int NH, int N, const double* __restrict__ A3, const double* __restrict__ b3,
                       const double* __restrict__ g3, const double* __restrict__ coef, const ColParams occ,
                       double* __restrict__ gpart) {
  __shared__ double sh[kInThreads];
  const int i = blockIdx.x;
  const double t2 = coef[(int64_t)NH * N + i];
  double v = 0.0;
  for (int j = threadIdx.x; j < NH; j += blockDim.x) {
    double r = 0.0;
    for (int k = 0; k < NH; ++k) r += A3[(int64_t)j * NH + k] * coef[(int64_t)k * N + i];
    const double pj = coef[(int64_t)j * N + i];
    v += pj * r + 2.0 * t2 * b3[(int64_t)j * N + i] * pj;
  }
  v = block_sum(v, sh);
  if (threadIdx.x == 0) gpart[i] = occ.v[i] * (v + t2 * t2 * g3[i]);
}

// (b) right-hand side of the bordered Hartree system and its border unknown:
//   r_H = 4 pi fH - lift_H,  theta_1' = (4 pi g - lift_0 - y^T r_H) / schur  (0 when w~0 lies in V_H), one block
__global__ void k_in_solve1(int NH, int N, const double* __restrict__ fH, const double* __restrict__ liftH,
                            const double* __restrict__ y, const double* __restrict__ gpart, double lift0,
                            double schur, int in_VH, double* __restrict__ rH, double* __restrict__ sc) {
  __shared__ double sh[kInThreads];
  const double fpi = 4.0 * M_PI;
  double v = 0.0;
  for (int j = threadIdx.x; j < NH; j += blockDim.x) {
    const double r = fpi * fH[j] - liftH[j];
    rH[j] = r;
    v += y[j] * r;
  }
  v = block_sum(v, sh);
  if (threadIdx.x == 0) {
    double g = 0.0;
    for (int i = 0; i < N; ++i) g += gpart[i];
    sc[IS_THETA1_NEW] = in_VH ? 0.0 : (fpi * g - lift0 - v) / schur;
  }
}

// (b) w_H' = C_H^-1 r_H - y theta_1', then mixing of (w_H, theta_1); one warp per row
__global__ void k_in_solve2(int NH, const double* __restrict__ CHinv, const double* __restrict__ rH,
                            const double* __restrict__ y, double mix, double* __restrict__ wH,
                            double* __restrict__ sc) {
  const int row = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32), lane = threadIdx.x % 32;
  const double th = sc[IS_THETA1_NEW];
  if (row < NH) {
    double s = 0.0;
    for (int k = lane; k < NH; k += 32) s += CHinv[(int64_t)row * NH + k] * rH[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) wH[row] = (1.0 - mix) * wH[row] + mix * (s - y[row] * th);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) sc[IS_THETA1] = (1.0 - mix) * sc[IS_THETA1] + mix * th;
}

// (c) sc[IS_DELTA] = max |coef - prev|, then prev = coef (one block)
__global__ void k_in_delta(int64_t n, const double* __restrict__ coef, double* __restrict__ prev,
                           double* __restrict__ sc) {
  __shared__ double sh[kInThreads];
  double m = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
    m = fmax(m, fabs(coef[k] - prev[k]));
    prev[k] = coef[k];
  }
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) sc[IS_DELTA] = sh[0];
}

// w = w_b + P w_H + theta_1 w~0 on the fine nodes
__global__ void k_in_potential(int64_t n, const int32_t* __restrict__ off, const int32_t* __restrict__ col,
                               const double* __restrict__ val, const uint8_t* __restrict__ bnd,
                               const double* __restrict__ wb, const double* __restrict__ w0,
                               const double* __restrict__ wH, const double* __restrict__ sc, double* __restrict__ w) {
  const int64_t nd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (nd >= n) return;
  double s = 0.0;
  if (!bnd[nd])
    for (int k = off[nd]; k < off[nd + 1]; ++k) s += val[k] * wH[col[k]];
  w[nd] = wb[nd] + s + sc[IS_THETA1] * w0[nd];
}

static int blocks_for(int64_t n, int th = 256) { return (int)((n + th - 1) / th); }

}  // namespace mk

using namespace mk;

extern "C" {

int mk_inner_create(mk_ctx* ctx, const mk_mesh* m, const mk_molecule* mol, const double* phit, int ld, int N,
                    const double* wt, const double* vxc_q, mk_inner** out, void* stream) {
  MK_ARG(ctx && m && mol && phit && wt && vxc_q && out, "mk_inner_create: null argument");
  MK_ARG(N >= 1 && N <= ld && N <= MK_MAX_RHS, "mk_inner_create: bad N/ld");
  MK_CUDA(cudaSetDevice(ctx->device));
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  const Level& F = m->fine;
  const Level& C = m->coarse;
  const int nl = F.nloc, NH = (int)C.n_free;
  const int64_t Ec = C.n_elems, n = F.n_nodes, E = F.n_elems;
  const size_t acc_bytes = (size_t)in_tensor_count(nl, N) * sizeof(double);
  MK_ARG(acc_bytes <= 160 * 1024, "mk_inner_create: too many orbitals");
  mk_inner* h = new mk_inner();
  h->ctx = ctx;
  h->mesh = m;
  h->device = ctx->device;
  h->NH = NH;
  h->N = N;
  h->nl = nl;
  h->Ec = Ec;
  h->n_nodes = n;
  // one arena for everything the handle keeps
  const size_t NH2 = (size_t)NH * NH, NHN = (size_t)NH * N, nl2 = (size_t)nl * nl;
  const size_t sizes[] = {NH2, NH2, NHN, NHN, (size_t)N, (size_t)N, NHN, (size_t)N,                  // A1..gamma
                          (size_t)Ec * nl2 * nl, (size_t)N * Ec * nl2, NHN, (size_t)N, NH2, (size_t)NH,  // Tc..y
                          (size_t)NH, (size_t)n, (size_t)n,                                           // liftH, wb, w0
                          NH2, NHN, (size_t)N, (size_t)NH, NH2, NH2, (size_t)N, (size_t)(NH + 1) * N,  // AH..coef
                          (size_t)(NH + 1) * N, (size_t)NH, (size_t)NH, (size_t)NH, (size_t)N, (size_t)IS_COUNT,
                          (size_t)N};  // prev, wH, fH, rH, gpart, sc, status (as doubles)
  constexpr int nbuf = sizeof(sizes) / sizeof(sizes[0]);
  size_t total = 0;
  for (int k = 0; k < nbuf; ++k) total += (sizes[k] * 8 + 255) / 256 * 256;
  if (cudaMalloc(&h->arena, total) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(MK_ERR_OOM, "mk_inner_create: device allocation failed");
  }
  double* ptr[nbuf];
  {
    char* p = (char*)h->arena;
    for (int k = 0; k < nbuf; ++k) {
      ptr[k] = (double*)p;
      p += (sizes[k] * 8 + 255) / 256 * 256;
    }
  }
  int k = 0;
  h->A1 = ptr[k++]; h->A3 = ptr[k++]; h->b1 = ptr[k++]; h->b3 = ptr[k++]; h->beta1 = ptr[k++];
  h->beta3 = ptr[k++]; h->c = ptr[k++]; h->gamma = ptr[k++];
  h->Tc = ptr[k++]; h->Ah4 = ptr[k++]; h->rvec = ptr[k++]; h->g3 = ptr[k++]; h->CHinv = ptr[k++]; h->y = ptr[k++];
  h->liftH = ptr[k++]; h->wb = ptr[k++]; h->w0 = ptr[k++];
  h->AH = ptr[k++]; h->b = ptr[k++]; h->beta = ptr[k++]; h->d = ptr[k++]; h->V[0] = ptr[k++]; h->V[1] = ptr[k++];
  h->lam = ptr[k++]; h->coef = ptr[k++]; h->prev = ptr[k++]; h->wH = ptr[k++]; h->fH = ptr[k++]; h->rH = ptr[k++];
  h->gpart = ptr[k++]; h->sc = ptr[k++]; h->status = (int32_t*)ptr[k++];
  auto bail = [&](int r) {
    mk_inner_destroy(h);
    return r;
  };
  int err = MK_OK;
  const size_t eb = (size_t)E * (nl * (nl + 1) / 2) * sizeof(double);
  double* H1e = (double*)scratch(ctx, S_ELEM64, eb, &err);
  double* M3e = (double*)scratch(ctx, S_ELEM64B, eb, &err);
  const double* Me = mass_matrices(ctx, m, s, &err);
  double* Ke = (double*)scratch(ctx, S_ELEM64D, eb, &err);
  double* Y = (double*)scratch(ctx, S_VEC1, (size_t)n * ld * sizeof(double), &err);
  double* V1 = (double*)scratch(ctx, S_VEC2, (size_t)n * sizeof(double), &err);
  double* V2 = (double*)scratch(ctx, S_VEC3, (size_t)n * sizeof(double), &err);
  double* vq = (double*)scratch(ctx, S_RHO, (size_t)E * kQ * sizeof(double), &err);
  double* wq0 = (double*)scratch(ctx, S_VEC4, (size_t)E * kQ * sizeof(double), &err);
  double* G = (double*)scratch(ctx, S_GRAM, (size_t)N * N * sizeof(double), &err);
  double* CH = (double*)scratch(ctx, S_JOINT, NH2 * 2 * sizeof(double), &err);
  double* rc = (double*)scratch(ctx, S_VEC5, ((size_t)N * Ec * nl + (size_t)Ec * N) * sizeof(double), &err);
  if (!H1e || !M3e || !Me || !Ke || !Y || !V1 || !V2 || !vq || !wq0 || !G || !CH || !rc) return bail(err);
  double* Li = CH + NH2;
  double* g3p = rc + (size_t)N * Ec * nl;
  const RefTables* ref = ctx->d_ref[nl == 4 ? 1 : 2];
  const int eblk = blocks_for(E, 128);
  // w~ = w_b + w~0; H1's potential V_xc + w_b and w~0 at the quadrature points
  MK_COUNT(), k_in_split<<<blocks_for(n), 256, 0, s>>>(n, F.d_boundary, wt, h->wb, h->w0);
  if (nl == 4) {
    MK_COUNT(), k_in_at_quad<4><<<eblk, 128, 0, s>>>(E, ref, F.d_elem, h->wb, vxc_q, vq);
    MK_COUNT(), k_in_at_quad<4><<<eblk, 128, 0, s>>>(E, ref, F.d_elem, h->w0, nullptr, wq0);
  } else {
    MK_COUNT(), k_in_at_quad<10><<<eblk, 128, 0, s>>>(E, ref, F.d_elem, h->wb, vxc_q, vq);
    MK_COUNT(), k_in_at_quad<10><<<eblk, 128, 0, s>>>(E, ref, F.d_elem, h->w0, nullptr, wq0);
  }
  const double* H0 = static_matrices(ctx, m, mol, s, &err);
  if (!H0) return bail(err);
  int r;
  if ((r = element_matrices(ctx, F, nullptr, 0.0, 0.0, 0.0, vq, H1e, s, H0)) != MK_OK) return bail(r);
  if ((r = element_matrices(ctx, F, nullptr, 0.0, 0.0, 0.0, wq0, M3e, s)) != MK_OK) return bail(r);
  if ((r = element_matrices(ctx, F, nullptr, 1.0, 0.0, 0.0, nullptr, Ke, s)) != MK_OK) return bail(r);
  // coarse blocks: A1 = P^T H1 P, A3 = P^T M_{w~0} P, C_H = P^T K P
  if ((r = coarse_matrices(ctx, m, H1e, M3e, h->A1, h->A3, S_COARSE, s)) != MK_OK) return bail(r);
  if ((r = coarse_matrices(ctx, m, Ke, nullptr, CH, nullptr, S_COARSE2, s)) != MK_OK) return bail(r);
  // restrictions and fine inner products of the corrections
  struct Proj { const double* Ae; double* bv; double* dg; };
  const Proj pj[3] = {{H1e, h->b1, h->beta1}, {M3e, h->b3, h->beta3}, {Me, h->c, h->gamma}};
  for (const Proj& q : pj) {
    if ((r = apply64(ctx, m, q.Ae, phit, Y, N, ld, true, s)) != MK_OK) return bail(r);
    if ((r = restrict_to_coarse(ctx, m, Y, ld, N, q.bv, N, s)) != MK_OK) return bail(r);
    if ((r = gram(ctx, n, phit, Y, N, ld, G, s)) != MK_OK) return bail(r);
    MK_CUDA(cudaMemcpy2DAsync(q.dg, sizeof(double), G, (N + 1) * sizeof(double), sizeof(double), N,
                              cudaMemcpyDeviceToDevice, s));
  }
  // Hartree system in W: d = P^T K w~0, zeta = (K w~0, w~0); lifts lift_H = P^T K_IB w_b, lift_0 = (K_IB w_b, w~0)
  double* dvec = h->rH;  // d lives in rH until y = C_H^-1 d is formed
  if ((r = apply64(ctx, m, Ke, h->w0, V1, 1, 1, true, s)) != MK_OK) return bail(r);
  if ((r = restrict_to_coarse(ctx, m, V1, 1, 1, dvec, 1, s)) != MK_OK) return bail(r);
  if ((r = gram(ctx, n, h->w0, V1, 1, 1, h->sc + IS_ZETA, s)) != MK_OK) return bail(r);
  if ((r = apply64(ctx, m, Ke, h->wb, V2, 1, 1, true, s)) != MK_OK) return bail(r);
  if ((r = restrict_to_coarse(ctx, m, V2, 1, 1, h->liftH, 1, s)) != MK_OK) return bail(r);
  if ((r = gram(ctx, n, h->w0, V2, 1, 1, h->sc + IS_LIFT0, s)) != MK_OK) return bail(r);
  // C_H^-1 = L^-T L^-1 and y = C_H^-1 d (synchronises: a C_H that is not positive definite is reported)
  if ((r = inverse_cholesky(ctx, NH, CH, Li, S_EIG4, s)) != MK_OK) return bail(r);
  MK_COUNT(), k_in_ltl<<<blocks_for((int64_t)NH * NH), 256, 0, s>>>(NH, Li, h->CHinv);
  MK_COUNT(), k_in_gemv<<<blocks_for((int64_t)NH * 32), 256, 0, s>>>(NH, h->CHinv, dvec, h->y);
  MK_COUNT(), k_in_dot<<<1, kInThreads, 0, s>>>(NH, dvec, h->y, h->sc + IS_DY);
  // the coarse-element tensors and their assembled parts: kInChunks CTAs per coarse element, then the chunks
  // summed in order
  const int K = in_tensor_count(nl, N);
  double* tpart = (double*)scratch(ctx, S_EIG5, (size_t)Ec * kInChunks * K * sizeof(double), &err);
  if (!tpart) return bail(err);
  const int tgrid = (int)(Ec * kInChunks);
  if (nl == 4) {
    MK_CUDA(cudaFuncSetAttribute(k_in_tensors<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)acc_bytes));
    MK_COUNT(), k_in_tensors<4><<<tgrid, kInThreads, acc_bytes, s>>>(m->d_child_off, m->d_child, F.d_geom, F.d_elem,
                                                                    C.d_geom, ref, phit, ld, N, h->w0, kInChunks,
                                                                    tpart);
    MK_COUNT(), k_in_tensor_reduce<4><<<blocks_for(Ec * K), 256, 0, s>>>(Ec, N, kInChunks, tpart, h->Tc, h->Ah4, rc,
                                                                         g3p);
  } else {
    MK_CUDA(cudaFuncSetAttribute(k_in_tensors<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)acc_bytes));
    MK_COUNT(), k_in_tensors<10><<<tgrid, kInThreads, acc_bytes, s>>>(m->d_child_off, m->d_child, F.d_geom, F.d_elem,
                                                                     C.d_geom, ref, phit, ld, N, h->w0, kInChunks,
                                                                     tpart);
    MK_COUNT(), k_in_tensor_reduce<10><<<blocks_for(Ec * K), 256, 0, s>>>(Ec, N, kInChunks, tpart, h->Tc, h->Ah4,
                                                                          rc, g3p);
  }
  MK_CUDA(cudaMemsetAsync(h->rvec, 0, NHN * sizeof(double), s));
  for (int col = 0; col < C.n_colours; ++col) {
    const int64_t off = C.colour_off[col], cnt = C.colour_off[col + 1] - off;
    if (nl == 4)
      MK_COUNT(), k_in_rc_scatter<4><<<blocks_for(cnt * 4 * N), 256, 0, s>>>(C.d_colour_elems + off, (int)cnt, C.d_elem,
                                                                            C.d_node_to_free, Ec, N, rc, h->rvec);
    else
      MK_COUNT(), k_in_rc_scatter<10><<<blocks_for(cnt * 10 * N), 256, 0, s>>>(C.d_colour_elems + off, (int)cnt,
                                                                              C.d_elem, C.d_node_to_free, Ec, N, rc,
                                                                              h->rvec);
  }
  MK_COUNT(), k_in_g3<<<1, MK_MAX_RHS, 0, s>>>(Ec, N, g3p, h->g3);
  MK_CUDA(cudaGetLastError());
  double hs[IS_COUNT];
  MK_CUDA(cudaMemcpyAsync(hs, h->sc, sizeof(hs), cudaMemcpyDeviceToHost, s));
  MK_CUDA(cudaStreamSynchronize(s));
  const double zeta = hs[IS_ZETA];
  h->schur = zeta - hs[IS_DY];
  h->w_in_VH = !(h->schur > 1e-12 * zeta);
  h->lift0 = hs[IS_LIFT0];
  *out = h;
  return MK_OK;
}

int mk_inner_run(mk_ctx* ctx, mk_inner* h, const double* occ, double tol, int max_inner, double mix, double* lambda,
                 double* coef, int32_t* status, double* wH, double* theta1, int* iters, double* delta,
                 void* stream) {
  MK_ARG(ctx && h && occ && lambda && coef, "mk_inner_run: null argument");
  MK_ARG(h->ctx == ctx, "mk_inner_run: handle of another context");
  MK_ARG(max_inner >= 1 && tol >= 0.0 && mix > 0.0 && mix <= 1.0, "mk_inner_run: bad tol/max_inner/mix");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const mk_mesh* m = h->mesh;
  const Level& C = m->coarse;
  const int NH = h->NH, N = h->N, nl = h->nl;
  const int64_t Ec = h->Ec;
  ColParams oc{};
  for (int i = 0; i < N; ++i) oc.v[i] = occ[i];
  // from w = w~: w_H = 0, theta_1 = 1
  const double one = 1.0;
  MK_CUDA(cudaMemsetAsync(h->wH, 0, (size_t)NH * sizeof(double), s));
  MK_CUDA(cudaMemcpyAsync(h->sc + IS_THETA1, &one, sizeof(double), cudaMemcpyHostToDevice, s));
  MK_CUDA(cudaMemsetAsync(h->prev, 0, (size_t)(NH + 1) * N * sizeof(double), s));
  double dl = 0.0;
  int it = 0;
  const int64_t nA = (int64_t)NH * NH + (int64_t)NH * N;
  for (it = 1; it <= max_inner; ++it) {
    // (a) the per-orbital augmented eigenproblems with the current Hartree potential
    MK_COUNT(), k_in_init<<<blocks_for(nA), 256, 0, s>>>(NH, N, h->A1, h->A3, h->b1, h->b3, h->sc, h->AH, h->b);
    MK_COUNT(), k_in_beta<<<N, kInThreads, 0, s>>>(NH, N, h->rvec, h->wH, h->beta1, h->beta3, h->sc, h->beta);
    for (int col = 0; col < C.n_colours; ++col) {
      const int64_t off = C.colour_off[col], cnt = C.colour_off[col + 1] - off;
      const int64_t work = cnt * nl * nl + cnt * nl * N;
      if (nl == 4)
        MK_COUNT(), k_in_scatter_ab<4><<<blocks_for(work), 256, 0, s>>>(C.d_colour_elems + off, (int)cnt, C.d_elem,
                                                                       C.d_node_to_free, Ec, NH, N, h->Tc, h->Ah4,
                                                                       h->wH, h->AH, h->b);
      else
        MK_COUNT(), k_in_scatter_ab<10><<<blocks_for(work), 256, 0, s>>>(C.d_colour_elems + off, (int)cnt, C.d_elem,
                                                                        C.d_node_to_free, Ec, NH, N, h->Tc, h->Ah4,
                                                                        h->wH, h->AH, h->b);
    }
    // warm start from the previous iteration's eigenbasis (the pencil changes little between iterations)
    double* Vn = h->V[it & 1];
    if (it == 1) MK_TRY(decompose(ctx, NH, m->d_MH_Linv, false, h->AH, h->d, Vn, s, S_EIG2));
    else MK_TRY(decompose(ctx, NH, h->V[(it - 1) & 1], true, h->AH, h->d, Vn, s, S_EIG2));
    MK_TRY(secular(ctx, NH, N, h->d, Vn, h->b, h->c, h->beta, h->gamma, h->lam, h->coef, h->status, s));
    // (b) the Hartree potential in W from the density of the new orbitals
    MK_COUNT(), k_in_fh_init<<<blocks_for(NH), 256, 0, s>>>(NH, N, h->rvec, h->coef, oc, h->fH);
    for (int col = 0; col < C.n_colours; ++col) {
      const int64_t off = C.colour_off[col], cnt = C.colour_off[col + 1] - off;
      if (nl == 4)
        MK_COUNT(), k_in_scatter_fh<4><<<blocks_for(cnt * 4), 256, 0, s>>>(C.d_colour_elems + off, (int)cnt, C.d_elem,
                                                                          C.d_node_to_free, Ec, NH, N, h->Tc, h->Ah4,
                                                                          h->coef, oc, h->fH);
      else
        MK_COUNT(), k_in_scatter_fh<10><<<blocks_for(cnt * 10), 256, 0, s>>>(C.d_colour_elems + off, (int)cnt,
                                                                            C.d_elem, C.d_node_to_free, Ec, NH, N,
                                                                            h->Tc, h->Ah4, h->coef, oc, h->fH);
    }
    MK_COUNT(), k_in_g<<<N, kInThreads, 0, s>>>(NH, N, h->A3, h->b3, h->g3, h->coef, oc, h->gpart);
    MK_COUNT(), k_in_solve1<<<1, kInThreads, 0, s>>>(NH, N, h->fH, h->liftH, h->y, h->gpart, h->lift0, h->schur,
                                                     h->w_in_VH ? 1 : 0, h->rH, h->sc);
    MK_COUNT(), k_in_solve2<<<blocks_for((int64_t)NH * 32), 256, 0, s>>>(NH, h->CHinv, h->rH, h->y, mix, h->wH, h->sc);
    // (c) the largest change of any orbital coefficient
    MK_COUNT(), k_in_delta<<<1, kInThreads, 0, s>>>((int64_t)(NH + 1) * N, h->coef, h->prev, h->sc);
    MK_CUDA(cudaGetLastError());
    MK_CUDA(cudaMemcpyAsync(&dl, h->sc + IS_DELTA, sizeof(double), cudaMemcpyDeviceToHost, s));
    MK_CUDA(cudaStreamSynchronize(s));
    if (it > 1 && dl < tol) break;
  }
  if (it > max_inner) it = max_inner;
  MK_CUDA(cudaMemcpyAsync(lambda, h->lam, (size_t)N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  MK_CUDA(cudaMemcpyAsync(coef, h->coef, (size_t)(NH + 1) * N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (status) MK_CUDA(cudaMemcpyAsync(status, h->status, (size_t)N * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  if (wH) MK_CUDA(cudaMemcpyAsync(wH, h->wH, (size_t)NH * sizeof(double), cudaMemcpyDeviceToDevice, s));
  double th = 0.0;
  MK_CUDA(cudaMemcpyAsync(&th, h->sc + IS_THETA1, sizeof(double), cudaMemcpyDeviceToHost, s));
  MK_CUDA(cudaStreamSynchronize(s));
  if (theta1) *theta1 = th;
  if (iters) *iters = it;
  if (delta) *delta = dl;
  return MK_OK;
}

int mk_inner_potential(mk_ctx* ctx, const mk_inner* h, double* w, void* stream) {
  MK_ARG(ctx && h && w, "mk_inner_potential: null argument");
  MK_ARG(h->ctx == ctx, "mk_inner_potential: handle of another context");
  MK_CUDA(cudaSetDevice(ctx->device));
  const mk_mesh* m = h->mesh;
  MK_COUNT(), k_in_potential<<<blocks_for(h->n_nodes), 256, 0, (cudaStream_t)stream>>>(
      h->n_nodes, m->d_P_off, m->d_P_col, m->d_P_val, m->fine.d_boundary, h->wb, h->w0, h->wH, h->sc, w);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

int mk_inner_info(const mk_inner* h, int* w_in_VH, double* schur) {
  MK_ARG(h, "mk_inner_info: null handle");
  if (w_in_VH) *w_in_VH = h->w_in_VH ? 1 : 0;
  if (schur) *schur = h->schur;
  return MK_OK;
}

int mk_inner_destroy(mk_inner* h) {
  if (!h) return MK_OK;
  cudaSetDevice(h->device);
  cudaFree(h->arena);
  delete h;
  return MK_OK;
}

}  // extern "C"
