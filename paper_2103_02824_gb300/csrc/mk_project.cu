// A6: projection of the frozen-density Hamiltonian on the augmented spaces V_H + span{psi^_i}
// (Eqs. (Eigenvalue_H_h), (Adef), (bdef), (betadef)).  Coarse blocks A_H = P^T H P and M_H = P^T M P are Galerkin
// products integrated on the fine mesh (the paper assembles them "in advance" on the fine mesh); b_i, c_i are
// restrictions P^T (H psi^_i), P^T (M psi^_i); beta, gamma and the Grams are fine-mesh inner products.
#include "mk_device.cuh"

namespace mk {

int restrict_to_coarse(mk_ctx*, const mk_mesh*, const double*, int, int, double*, int, cudaStream_t);

// Coarse element matrices sum_{children e} R_e^T A_e R_e, R_e[c][b] = coarse basis b of the parent at fine node c.
// One block per coarse element; children in increasing fine index (fixed order).
template <int NLOC>
__global__ void k_coarse_galerkin(const int32_t* __restrict__ child_off, const int32_t* __restrict__ child,
                                  const Geom* __restrict__ fgeom, const Geom* __restrict__ cgeom,
                                  const RefTables* __restrict__ ref, const double* __restrict__ A1,
                                  const double* __restrict__ A2, int nchunk, double* __restrict__ part1,
                                  double* __restrict__ part2) {
  constexpr int NP = NLOC * (NLOC + 1) / 2;
  __shared__ double R[NLOC][NLOC];
  __shared__ double S1[NLOC][NLOC], S2[NLOC][NLOC];
  __shared__ double T1[NLOC][NLOC], T2[NLOC][NLOC];
  // block = (coarse element T, chunk ch of its children): the children of one coarse element are spread over
  // nchunk CTAs, whose partial sums k_coarse_reduce adds in chunk order
  const int T = blockIdx.x / nchunk, ch = blockIdx.x % nchunk;
  const Geom cg = cgeom[T];
  const int tid = threadIdx.x;
  const int a = tid / NLOC, b = tid % NLOC;
  const bool two = A2 != nullptr;
  const int c0 = child_off[T], len = child_off[T + 1] - c0;
  const int kb = c0 + (int)((int64_t)len * ch / nchunk), ke = c0 + (int)((int64_t)len * (ch + 1) / nchunk);
  double acc1 = 0.0, acc2 = 0.0;
  for (int k = kb; k < ke; ++k) {
    const int e = child[k];
    if (tid < NLOC * NLOC) {
      const Geom g = fgeom[e];
      // fine local node a: reference coords from barycentrics, physical point, barycentrics in the parent
      const double* lb = ref->node_bary[a];
      const double xi[3] = {lb[1], lb[2], lb[3]};
      double x[3], sv[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) x[r] = g.x0[r] + g.J[r * 3] * xi[0] + g.J[r * 3 + 1] * xi[1] + g.J[r * 3 + 2] * xi[2];
#pragma unroll
      for (int r = 0; r < 3; ++r)
        sv[r] = cg.Jinv[r * 3] * (x[0] - cg.x0[0]) + cg.Jinv[r * 3 + 1] * (x[1] - cg.x0[1]) +
                cg.Jinv[r * 3 + 2] * (x[2] - cg.x0[2]);
      const double lam[4] = {1.0 - sv[0] - sv[1] - sv[2], sv[0], sv[1], sv[2]};
      double v;
      if (NLOC == 4) {
        v = lam[b];
      } else if (b < 4) {
        v = lam[b] * (2.0 * lam[b] - 1.0);
      } else {
        const int ea[6] = {0, 0, 0, 1, 1, 2}, eb[6] = {1, 2, 3, 2, 3, 3};
        v = 4.0 * lam[ea[b - 4]] * lam[eb[b - 4]];
      }
      R[a][b] = v;
      S1[a][b] = A1[(int64_t)e * NP + sym_index(a, b, NLOC)];
      if (two) S2[a][b] = A2[(int64_t)e * NP + sym_index(a, b, NLOC)];
    }
    __syncthreads();
    if (tid < NLOC * NLOC) {  // T = A R  (row a, col b)
      double t1 = 0.0, t2 = 0.0;
#pragma unroll
      for (int d = 0; d < NLOC; ++d) {
        t1 += S1[a][d] * R[d][b];
        if (two) t2 += S2[a][d] * R[d][b];
      }
      T1[a][b] = t1;
      if (two) T2[a][b] = t2;
    }
    __syncthreads();
    if (tid < NLOC * NLOC) {  // acc += (R^T T)[a][b]
#pragma unroll
      for (int c = 0; c < NLOC; ++c) {
        acc1 += R[c][a] * T1[c][b];
        if (two) acc2 += R[c][a] * T2[c][b];
      }
    }
    __syncthreads();
  }
  if (tid < NLOC * NLOC) {
    part1[(int64_t)blockIdx.x * NLOC * NLOC + tid] = acc1;
    if (two) part2[(int64_t)blockIdx.x * NLOC * NLOC + tid] = acc2;
  }
}

// out[T][i] = sum over chunks, in order, of part[T][chunk][i]
__global__ void k_coarse_reduce(int64_t ne, int nn, int nchunk, const double* __restrict__ part,
                                double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ne * nn) return;
  const int64_t T = t / nn;
  const int i = (int)(t - T * nn);
  double v = 0.0;
  for (int c = 0; c < nchunk; ++c) v += part[(T * nchunk + c) * nn + i];
  out[t] = v;
}

// Dense coarse matrices over the coarse free DOF, one colour of coarse elements at a time.
template <int NLOC>
__global__ void k_coarse_scatter(const int32_t* __restrict__ celems, int count, const int32_t* __restrict__ elem,
                                 const int32_t* __restrict__ node_to_free, const double* __restrict__ C1,
                                 const double* __restrict__ C2, double* __restrict__ AH, double* __restrict__ MH,
                                 int NH) {
  // one thread per (element, a, b): elements of one colour share no node, so every (f_a, f_b) is written once
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)count * NLOC * NLOC) return;
  const int i = (int)(t / (NLOC * NLOC)), ab = (int)(t % (NLOC * NLOC));
  const int a = ab / NLOC, b = ab % NLOC;
  const int T = celems[i];
  const int fa = node_to_free[elem[(int64_t)T * NLOC + a]], fb = node_to_free[elem[(int64_t)T * NLOC + b]];
  if (fa < 0 || fb < 0) return;
  AH[(int64_t)fa * NH + fb] += C1[(int64_t)T * NLOC * NLOC + ab];
  if (MH) MH[(int64_t)fa * NH + fb] += C2[(int64_t)T * NLOC * NLOC + ab];
}

// Gram partials: part[blk][j*N+k] = sum over nodes of X[n][j] Y[n][k]
__global__ void k_gram_partial(int64_t n, const double* __restrict__ X, const double* __restrict__ Y, int N, int ld,
                               double* __restrict__ part) {
  extern __shared__ double sh[];
  const int NN = N * N;
  const int rows = blockDim.x >= NN ? blockDim.x / NN : 1;
  const int pairs_per_thread = blockDim.x >= NN ? 1 : (NN + blockDim.x - 1) / blockDim.x;
  const int r = blockDim.x >= NN ? threadIdx.x / NN : 0;
  double acc[16];
  for (int k = 0; k < 16; ++k) acc[k] = 0.0;
  const bool live = blockDim.x >= NN ? (r < rows) : true;
  if (live) {
    for (int64_t nd = (int64_t)blockIdx.x * rows + r; nd < n; nd += (int64_t)gridDim.x * rows) {
      for (int k = 0; k < pairs_per_thread && k < 16; ++k) {
        const int p = blockDim.x >= NN ? threadIdx.x % NN : threadIdx.x + k * blockDim.x;
        if (p < NN) acc[k] += X[nd * ld + p / N] * Y[nd * ld + p % N];
      }
    }
  }
  if (blockDim.x >= NN) {
    sh[threadIdx.x] = live ? acc[0] : 0.0;
    __syncthreads();
    if (threadIdx.x < NN) {
      double s = 0.0;
      for (int k = 0; k < rows; ++k) s += sh[k * NN + threadIdx.x];
      part[(int64_t)blockIdx.x * NN + threadIdx.x] = s;
    }
  } else {
    for (int k = 0; k < pairs_per_thread && k < 16; ++k) {
      const int p = threadIdx.x + k * blockDim.x;
      if (p < NN) part[(int64_t)blockIdx.x * NN + p] = acc[k];
    }
  }
}

__global__ void k_diag_of(const double* __restrict__ G, int N, double* __restrict__ d) {
  const int j = threadIdx.x;
  if (j < N) d[j] = G[j * N + j];
}

int gram(mk_ctx* ctx, int64_t n, const double* X, const double* Y, int N, int ld, double* G, cudaStream_t s) {
  int err = MK_OK;
  const int nblk = red_blocks(ctx);
  double* part = (double*)scratch(ctx, S_RED, (size_t)nblk * N * N * sizeof(double), &err);
  if (!part) return err;
  MK_COUNT(), k_gram_partial<<<nblk, kRedThreads, kRedThreads * sizeof(double), s>>>(n, X, Y, N, ld, part);
  sum_partials(part, nblk, N * N, G, s);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

// Dense coarse Galerkin matrices X1 = P^T A1 P, X2 = P^T A2 P over the coarse free DOF from two sets of packed
// fine element matrices (children summed per coarse element in fixed order, then coarse colour by colour).
int coarse_matrices(mk_ctx* ctx, const mk_mesh* m, const double* A1, const double* A2, double* X1, double* X2,
                    int slot, cudaStream_t s) {
  // X1 = P^T A1 P and, when A2 and X2 are given, X2 = P^T A2 P (dense over the coarse free DOF)
  const Level& F = m->fine;
  const Level& C = m->coarse;
  const int NH = (int)C.n_free, nl = F.nloc;
  const bool two = A2 && X2;
  constexpr int kChunks = 16;
  int err = MK_OK;
  const size_t per = (size_t)C.n_elems * nl * nl;
  double* CE = (double*)scratch(ctx, slot, per * 2 * (kChunks + 1) * sizeof(double), &err);
  if (!CE) return err;
  double* C1 = CE;
  double* C2 = CE + per;
  double* P1 = CE + 2 * per;
  double* P2 = P1 + per * kChunks;
  const int blocks = (int)C.n_elems * kChunks;
  // the largest shared-memory carveout: room for the fine solve's CTAs (other stream) beside this kernel's
  if (nl == 4) {
    cudaFuncSetAttribute(k_coarse_galerkin<4>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    MK_COUNT(), k_coarse_galerkin<4><<<blocks, 128, 0, s>>>(m->d_child_off, m->d_child, F.d_geom, C.d_geom,
                                                           ctx->d_ref[1], A1, two ? A2 : nullptr, kChunks, P1, P2);
  } else {
    cudaFuncSetAttribute(k_coarse_galerkin<10>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    MK_COUNT(), k_coarse_galerkin<10><<<blocks, 128, 0, s>>>(m->d_child_off, m->d_child, F.d_geom, C.d_geom,
                                                            ctx->d_ref[2], A1, two ? A2 : nullptr, kChunks, P1, P2);
  }
  const int64_t work = (int64_t)per;
  MK_COUNT(), k_coarse_reduce<<<(int)((work + 255) / 256), 256, 0, s>>>(C.n_elems, nl * nl, kChunks, P1, C1);
  if (two) MK_COUNT(), k_coarse_reduce<<<(int)((work + 255) / 256), 256, 0, s>>>(C.n_elems, nl * nl, kChunks, P2, C2);
  MK_CUDA(cudaMemsetAsync(X1, 0, (size_t)NH * NH * sizeof(double), s));
  if (two) MK_CUDA(cudaMemsetAsync(X2, 0, (size_t)NH * NH * sizeof(double), s));
  for (int col = 0; col < C.n_colours; ++col) {
    const int64_t off = C.colour_off[col], cnt = C.colour_off[col + 1] - off;
    if (nl == 4)
      MK_COUNT(), k_coarse_scatter<4><<<(int)((cnt * 16 + 255) / 256), 256, 0, s>>>(C.d_colour_elems + off, (int)cnt, C.d_elem,
                                                                           C.d_node_to_free, C1, C2, X1, two ? X2 : nullptr, NH);
    else
      MK_COUNT(), k_coarse_scatter<10><<<(int)((cnt * 100 + 255) / 256), 256, 0, s>>>(C.d_colour_elems + off, (int)cnt,
                                                                            C.d_elem, C.d_node_to_free, C1, C2, X1,
                                                                            two ? X2 : nullptr, NH);
  }
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

}  // namespace mk

using namespace mk;

extern "C" int mk_coarse_pencil(mk_ctx* ctx, const mk_mesh* m, const mk_molecule* mol, const double* vq, double* AH,
                                double* MH, void* stream) {
  MK_ARG(ctx && m && mol && AH, "mk_coarse_pencil: null argument");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const Level& F = m->fine;
  const int nl = F.nloc;
  int err = MK_OK;
  const size_t eb = (size_t)F.n_elems * (nl * (nl + 1) / 2) * sizeof(double);
  double* He = (double*)scratch(ctx, S_ELEM64C, eb, &err);
  double* Me = MH ? (double*)scratch(ctx, S_ELEM64D, eb, &err) : nullptr;
  if (!He || (MH && !Me)) return err;
  const double* H0 = static_matrices(ctx, m, mol, s, &err);
  if (!H0) return err;
  MK_TRY(element_matrices(ctx, F, nullptr, 0.0, 0.0, 0.0, vq, He, s, H0));
  if (MH) MK_TRY(element_matrices(ctx, F, nullptr, 0.0, 0.0, 1.0, nullptr, Me, s));
  return coarse_matrices(ctx, m, He, Me, AH, MH, S_COARSE2, s);
}

extern "C" int mk_augmented_project(mk_ctx* ctx, const mk_mesh* m, const mk_molecule* mol, const double* vq,
                                    const double* psihat, int ld, int N, double* AH, double* MH, double* b, double* c,
                                    double* beta, double* gamma, double* gramA, double* gramM, void* stream) {
  MK_ARG(ctx && m && mol && vq && psihat && b && c && beta && gamma, "mk_augmented_project: null argument");
  MK_ARG((AH == nullptr) == (MH == nullptr), "mk_augmented_project: AH and MH must both be given or both NULL");
  MK_ARG(N >= 1 && N <= ld && N <= MK_MAX_RHS, "mk_augmented_project: bad N/ld");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const Level& F = m->fine;
  const int nl = F.nloc;
  int err = MK_OK;
  const size_t eb = (size_t)F.n_elems * (nl * (nl + 1) / 2) * sizeof(double);
  double* He = (double*)scratch(ctx, S_ELEM64, eb, &err);
  double* Y = (double*)scratch(ctx, S_VEC1, (size_t)F.n_nodes * ld * sizeof(double), &err);
  double* MY = (double*)scratch(ctx, S_VEC2, (size_t)F.n_nodes * ld * sizeof(double), &err);
  double* G = (double*)scratch(ctx, S_GRAM, (size_t)2 * N * N * sizeof(double), &err);
  if (!He || !Y || !MY || !G) return err;
  const double* Me = mass_matrices(ctx, m, s, &err);
  if (!Me) return err;
  const double* H0 = static_matrices(ctx, m, mol, s, &err);
  if (!H0) return err;
  MK_TRY(element_matrices(ctx, F, nullptr, 0.0, 0.0, 0.0, vq, He, s, H0));
  MK_TRY(apply64(ctx, m, He, psihat, Y, N, ld, true, s));
  MK_TRY(apply64(ctx, m, Me, psihat, MY, N, ld, true, s));
  MK_TRY(restrict_to_coarse(ctx, m, Y, ld, N, b, N, s));
  MK_TRY(restrict_to_coarse(ctx, m, MY, ld, N, c, N, s));
  double* GA = gramA ? gramA : G;
  double* GM = gramM ? gramM : G + N * N;
  MK_TRY(gram(ctx, F.n_nodes, psihat, Y, N, ld, GA, s));
  MK_TRY(gram(ctx, F.n_nodes, psihat, MY, N, ld, GM, s));
  MK_COUNT(), k_diag_of<<<1, MK_MAX_RHS, 0, s>>>(GA, N, beta);
  MK_COUNT(), k_diag_of<<<1, MK_MAX_RHS, 0, s>>>(GM, N, gamma);
  if (AH) MK_TRY(coarse_matrices(ctx, m, He, Me, AH, MH, S_COARSE, s));
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}
