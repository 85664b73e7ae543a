// Finite-element kernels on the fine mesh: element matrices by reference-element quadrature, coloured
// element-by-element operator application, reductions, prolongation/restriction, density and potentials.
#include <cmath>

#include "mk_device.cuh"
#include "mk_patch.cuh"

namespace mk {

// ------------------------------------------------------------------------------------------------ reductions
// One warp per output: lanes add the block partials lane-strided, then a fixed shuffle tree (deterministic).
__global__ void k_sum_partials(const double* __restrict__ part, int nblk, int N, double* __restrict__ out) {
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= N) return;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += part[(int64_t)b * N + j];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) out[j] = s;
}

void sum_partials(const double* part, int nblk, int N, double* out, cudaStream_t s) {
  MK_COUNT(), k_sum_partials<<<(N + 7) / 8, 256, 0, s>>>(part, nblk, N, out);
}

template <typename T>
static int column_dots_t(mk_ctx* ctx, int64_t n_nodes, const T* a, const T* b, int N, int ld, double* out,
                         cudaStream_t s) {
  int err = MK_OK;
  const int nblk = red_blocks(ctx);
  double* part = (double*)scratch(ctx, S_RED, (size_t)nblk * N * sizeof(double), &err);
  if (!part) return err;
  MK_COUNT(), k_dot_partial<T><<<nblk, kRedThreads, kRedThreads * sizeof(double), s>>>(n_nodes, a, b, N, ld, part);
  sum_partials(part, nblk, N, out, s);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

int column_dots(mk_ctx* ctx, int64_t n_nodes, const double* a, const double* b, int N, int ld, double* out,
                cudaStream_t s) {
  return column_dots_t<double>(ctx, n_nodes, a, b, N, ld, out, s);
}
int column_dots32(mk_ctx* ctx, int64_t n_nodes, const float* a, const float* b, int N, int ld, double* out,
                  cudaStream_t s) {
  return column_dots_t<float>(ctx, n_nodes, a, b, N, ld, out, s);
}

// ------------------------------------------------------------------------------------------------ element matrices
// out_e = base_e + half_k K_e + vext_scale M_{V_ext,e} + mass_shift M_e + M_{vq,e}, packed upper triangle, FP64
// (base optional: a precomputed set of element matrices in the same layout).
// K_e = |det J| sum_{i<=j} (J^-1 J^-T)_{ij} S^{ij} with the reference tensors S^{ij}; the mass-type terms by the
// 27-point rule at the physical points x_q = x0 + J xi_q (a constant coefficient uses the exact reference mass).
template <int NLOC>
__global__ void k_element_matrices(int64_t E, const RefTables* __restrict__ ref, const Geom* __restrict__ geom,
                                   const NucParams nucp, double half_k, double vext_scale, double mass_shift,
                                   const double* __restrict__ vq, const double* __restrict__ base,
                                   double* __restrict__ out) {
  constexpr int NP = NLOC * (NLOC + 1) / 2;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const Geom g = geom[e];
  const double det = fabs(g.det);
  double acc[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) acc[p] = base ? base[e * NP + p] : 0.0;
  const bool vext = vext_scale != 0.0 && nucp.n > 0;
  if (vext || vq != nullptr) {
    for (int q = 0; q < kQ; ++q) {
      const double xi = ref->qx[q][0], et = ref->qx[q][1], ze = ref->qx[q][2];
      double c = mass_shift;
      if (vext) {
        const double x = g.x0[0] + g.J[0] * xi + g.J[1] * et + g.J[2] * ze;
        const double y = g.x0[1] + g.J[3] * xi + g.J[4] * et + g.J[5] * ze;
        const double z = g.x0[2] + g.J[6] * xi + g.J[7] * et + g.J[8] * ze;
        c += vext_scale * nuclear_potential(nucp, x, y, z);
      }
      if (vq) c += vq[e * kQ + q];
      c *= ref->qw[q] * det;
      double ph[NLOC];
#pragma unroll
      for (int a = 0; a < NLOC; ++a) ph[a] = ref->phi[q][a];
#pragma unroll
      for (int a = 0; a < NLOC; ++a)
#pragma unroll
        for (int b = a; b < NLOC; ++b) acc[sym_index(a, b, NLOC)] += c * ph[a] * ph[b];
    }
  } else if (mass_shift != 0.0) {
    const double f = mass_shift * det;
#pragma unroll
    for (int p = 0; p < NP; ++p) acc[p] += f * ref->mass[p];
  }
  if (half_k != 0.0) {
    const double* Ji = g.Jinv;
    double G[6];  // (J^-1 J^-T)_{ij} for ij = 00,11,22,01,02,12
    const int I6[6] = {0, 1, 2, 0, 0, 1}, J6[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int c = 0; c < 6; ++c)
      G[c] = Ji[I6[c] * 3] * Ji[J6[c] * 3] + Ji[I6[c] * 3 + 1] * Ji[J6[c] * 3 + 1] + Ji[I6[c] * 3 + 2] * Ji[J6[c] * 3 + 2];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const double f = half_k * det * G[c];
#pragma unroll
      for (int p = 0; p < NP; ++p) acc[p] += f * ref->stiff[c][p];
    }
  }
#pragma unroll
  for (int p = 0; p < NP; ++p) out[e * NP + p] = acc[p];
}

int element_matrices(mk_ctx* ctx, const Level& L, const mk_molecule* mol, double half_k, double vext_scale,
                     double mass_shift, const double* vq, double* out, cudaStream_t s, const double* base) {
  MK_ARG(!mol || mol->n_nuclei <= kMaxNuclei, "at most 64 nuclei are supported");
  const NucParams nucp = make_nuc(mol);
  const int th = 128;
  const int blocks = (int)((L.n_elems + th - 1) / th);
  if (L.nloc == 4)
    MK_COUNT(), k_element_matrices<4><<<blocks, th, 0, s>>>(L.n_elems, ctx->d_ref[1], L.d_geom, nucp, half_k,
                                                            vext_scale, mass_shift, vq, base, out);
  else
    MK_COUNT(), k_element_matrices<10><<<blocks, th, 0, s>>>(L.n_elems, ctx->d_ref[2], L.d_geom, nucp, half_k,
                                                             vext_scale, mass_shift, vq, base, out);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

// K/2 + M_{V_ext} element matrices of the fine mesh for `mol`, computed once per (mesh, molecule) and kept in the
// mesh handle: they depend on neither the density nor the shift (the paper's static blocks, assembled in
// advance).  The molecule is compared by value; a different one replaces the cached set.
// M element matrices of the fine mesh (packed, FP64, element order), computed once per mesh and kept in the mesh
// handle (they depend on the geometry only).  Readers on another stream are ordered after the write by an event.
const double* mass_matrices(mk_ctx* ctx, const mk_mesh* m, cudaStream_t s, int* err) {
  const Level& L = m->fine;
  if (!m->mass_ev && cudaEventCreateWithFlags(&m->mass_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    m->mass_ev = nullptr;
    *err = fail(MK_ERR_CUDA, "mass element matrices: event creation failed");
    return nullptr;
  }
  if (m->d_M64) {
    if (cudaStreamWaitEvent(s, m->mass_ev, 0) != cudaSuccess) {
      *err = fail(MK_ERR_CUDA, "mass element matrices: cudaStreamWaitEvent failed");
      return nullptr;
    }
    return m->d_M64;
  }
  const size_t bytes = (size_t)L.n_elems * (L.nloc * (L.nloc + 1) / 2) * sizeof(double);
  if (cudaMalloc(&m->d_M64, bytes) != cudaSuccess) {
    cudaGetLastError();
    m->d_M64 = nullptr;
    *err = fail(MK_ERR_OOM, "mass element matrices: allocation failed");
    return nullptr;
  }
  const int r = element_matrices(ctx, L, nullptr, 0.0, 0.0, 1.0, nullptr, m->d_M64, s);
  if (r != MK_OK || cudaEventRecord(m->mass_ev, s) != cudaSuccess) {
    cudaFree(m->d_M64);
    m->d_M64 = nullptr;
    *err = r != MK_OK ? r : fail(MK_ERR_CUDA, "mass element matrices: cudaEventRecord failed");
    return nullptr;
  }
  return m->d_M64;
}

const double* static_matrices(mk_ctx* ctx, const mk_mesh* m, const mk_molecule* mol, cudaStream_t s, int* err) {
  const Level& L = m->fine;
  std::vector<double> key;
  const int n = mol ? mol->n_nuclei : 0;
  key.push_back(n);
  for (int k = 0; k < n; ++k) {
    key.push_back(mol->Z[k]);
    for (int c = 0; c < 3; ++c) key.push_back(mol->R[3 * k + c]);
  }
  if (!m->static_ev && cudaEventCreateWithFlags(&m->static_ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    m->static_ev = nullptr;
    *err = fail(MK_ERR_CUDA, "static element matrices: event creation failed");
    return nullptr;
  }
  if (m->d_static && m->static_key == key) {
    // the set may have been written on another stream: order this one after it
    if (cudaStreamWaitEvent(s, m->static_ev, 0) != cudaSuccess) {
      *err = fail(MK_ERR_CUDA, "static element matrices: cudaStreamWaitEvent failed");
      return nullptr;
    }
    return m->d_static;
  }
  if (m->d_static) {
    // another molecule: earlier readers of the old set, on any stream, finish first
    if (cudaDeviceSynchronize() != cudaSuccess) {
      *err = fail(MK_ERR_CUDA, "static element matrices: cudaDeviceSynchronize failed");
      return nullptr;
    }
  } else {
    const size_t bytes = (size_t)L.n_elems * (L.nloc * (L.nloc + 1) / 2) * sizeof(double);
    if (cudaMalloc(&m->d_static, bytes) != cudaSuccess) {
      cudaGetLastError();
      m->d_static = nullptr;
      *err = fail(MK_ERR_OOM, "static element matrices: allocation failed");
      return nullptr;
    }
  }
  const int r = element_matrices(ctx, L, mol, 0.5, 1.0, 0.0, nullptr, m->d_static, s);
  if (r != MK_OK) {
    *err = r;
    return nullptr;
  }
  if (cudaEventRecord(m->static_ev, s) != cudaSuccess) {
    *err = fail(MK_ERR_CUDA, "static element matrices: cudaEventRecord failed");
    return nullptr;
  }
  m->static_key = key;
  return m->d_static;
}

// ------------------------------------------------------------------------------------------------ diagonal
template <int NLOC>
__global__ void k_diag_colour(const int32_t* __restrict__ celems, int count, const int32_t* __restrict__ elem,
                              const double* __restrict__ Ae, double* __restrict__ diag) {
  constexpr int NP = NLOC * (NLOC + 1) / 2;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int e = celems[i];
#pragma unroll
  for (int a = 0; a < NLOC; ++a) diag[elem[(int64_t)e * NLOC + a]] += Ae[(int64_t)e * NP + sym_index(a, a, NLOC)];
}

__global__ void k_mask_rows(int64_t n, const uint8_t* __restrict__ bnd, double* __restrict__ v, int N, int ld,
                            double value) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * N) return;
  const int64_t nd = t / N;
  const int j = (int)(t % N);
  if (bnd[nd]) v[nd * ld + j] = value;
}

int assemble_diagonal(mk_ctx* ctx, const Level& L, const double* Ae, double* diag, cudaStream_t s) {
  (void)ctx;
  MK_CUDA(cudaMemsetAsync(diag, 0, L.n_nodes * sizeof(double), s));
  for (int c = 0; c < L.n_colours; ++c) {
    const int64_t off = L.colour_off[c], cnt = L.colour_off[c + 1] - off;
    const int blocks = (int)((cnt + 255) / 256);
    if (L.nloc == 4)
      MK_COUNT(), k_diag_colour<4><<<blocks, 256, 0, s>>>(L.d_colour_elems + off, (int)cnt, L.d_elem, Ae, diag);
    else
      MK_COUNT(), k_diag_colour<10><<<blocks, 256, 0, s>>>(L.d_colour_elems + off, (int)cnt, L.d_elem, Ae, diag);
  }
  MK_COUNT(), k_mask_rows<<<(int)((L.n_nodes + 255) / 256), 256, 0, s>>>(L.n_nodes, L.d_boundary, diag, 1, 1, 1.0);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

int apply64(mk_ctx* ctx, const mk_mesh* m, const double* Ae, const double* x, double* y, int N, int ld,
            bool mask_boundary, cudaStream_t s) {
  (void)N;  // the patch operator writes every row of all ld columns
  const Level& L = m->fine;
  int err = MK_OK;
  double* A = (double*)scratch(ctx, S_ELEMP64, (size_t)L.n_elems * padded_np(L.nloc, 8) * sizeof(double), &err);
  if (!A) return err;
  MK_TRY(pack_elements<double>(ctx, m, Ae, A, s));
  return apply_patch<double>(ctx, m, A, x, y, ld, mask_boundary, s);
}

// ------------------------------------------------------------------------------------------------ A1, restriction
__global__ void k_prolong(int64_t n_nodes, const int32_t* __restrict__ off, const int32_t* __restrict__ col,
                          const double* __restrict__ val, const uint8_t* __restrict__ bnd,
                          const double* __restrict__ psiH, int ldc, int N, double* __restrict__ u, int ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_nodes * ld) return;
  const int64_t nd = t / ld;
  const int j = (int)(t % ld);
  double s = 0.0;
  if (j < N && !bnd[nd])
    for (int k = off[nd]; k < off[nd + 1]; ++k) s += val[k] * psiH[(int64_t)col[k] * ldc + j];
  u[nd * ld + j] = s;
}

// out[k*ldo + j] = sum over fine nodes n of P[n,k] y[n*ld + j]  (one block per coarse free DOF, fixed tree)
__global__ void k_restrict(const int32_t* __restrict__ off, const int32_t* __restrict__ col,
                           const double* __restrict__ val, const double* __restrict__ y, int ld, int N,
                           double* __restrict__ out, int ldo) {
  extern __shared__ double sh[];
  const int k = blockIdx.x;
  const int b = off[k], e = off[k + 1];
  for (int j0 = 0; j0 < N; j0 += 8) {
    double acc[8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) acc[jj] = 0.0;
    for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
      const double w = val[i];
      const double* yr = y + (int64_t)col[i] * ld;
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
        if (j0 + jj < N) acc[jj] += w * yr[j0 + jj];
    }
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) sh[jj * blockDim.x + threadIdx.x] = acc[jj];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st)
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) sh[jj * blockDim.x + threadIdx.x] += sh[jj * blockDim.x + threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x < 8 && j0 + threadIdx.x < N) out[(int64_t)k * ldo + j0 + threadIdx.x] = sh[threadIdx.x * blockDim.x];
    __syncthreads();
  }
}

int restrict_to_coarse(mk_ctx* ctx, const mk_mesh* m, const double* y, int ld, int N, double* out, int ldo,
                       cudaStream_t s) {
  (void)ctx;
  const int th = 128;
  MK_COUNT(), k_restrict<<<(int)m->coarse.n_free, th, 8 * th * sizeof(double), s>>>(m->d_PT_off, m->d_PT_col, m->d_PT_val, y,
                                                                          ld, N, out, ldo);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

int prolongate(mk_ctx* ctx, const mk_mesh* m, const double* psiH, int ldc, int N, double* u, int ld,
               cudaStream_t s) {
  (void)ctx;
  const Level& F = m->fine;
  MK_COUNT(), k_prolong<<<(int)((F.n_nodes * ld + 255) / 256), 256, 0, s>>>(F.n_nodes, m->d_P_off, m->d_P_col, m->d_P_val,
                                                                 F.d_boundary, psiH, ldc, N, u, ld);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

// ------------------------------------------------------------------------------------------------ density, potentials
// rho[e*Q+q] = sum_j occ[j] u_j(x_q)^2
template <int NLOC>
__global__ void k_density(int64_t E, const RefTables* __restrict__ ref, const int32_t* __restrict__ elem,
                          const double* __restrict__ u, int ld, int N, const ColParams occ,
                          double* __restrict__ rho) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  int nd[NLOC];
#pragma unroll
  for (int a = 0; a < NLOC; ++a) nd[a] = elem[e * NLOC + a];
  double r[kQ];
#pragma unroll
  for (int q = 0; q < kQ; ++q) r[q] = 0.0;
  for (int j = 0; j < N; ++j) {
    double ua[NLOC];
#pragma unroll
    for (int a = 0; a < NLOC; ++a) ua[a] = u[(int64_t)nd[a] * ld + j];
    const double f = occ.v[j];
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      double v = 0.0;
#pragma unroll
      for (int a = 0; a < NLOC; ++a) v += ref->phi[q][a] * ua[a];
      r[q] += f * v * v;
    }
  }
#pragma unroll
  for (int q = 0; q < kQ; ++q) rho[e * kQ + q] = r[q];
}

// Exchange-correlation potential of Sec. 4 at density rho (rho < 1e-30 -> 0).
__device__ double vxc_of(double rho, int kind, double alpha) {
  if (kind == MK_XC_NONE || !(rho >= 1e-30)) return 0.0;
  const double vx = -cbrt(3.0 * rho / M_PI);
  if (kind == MK_XC_SLATER) return vx;
  if (kind == MK_XC_XALPHA) return 1.5 * alpha * vx;
  // Perdew-Zunger correlation: v_c = eps_c - (r_s/3) d eps_c / d r_s, branch split at r_s = 1
  const double rs = cbrt(3.0 / (4.0 * M_PI * rho));
  double ec, dec;
  if (rs < 1.0) {
    const double lr = log(rs);
    ec = 0.0311 * lr - 0.048 + 0.0020 * rs * lr - 0.0116 * rs;
    dec = 0.0311 / rs + 0.0020 * (lr + 1.0) - 0.0116;
  } else {
    const double sq = sqrt(rs);
    const double den = 1.0 + 1.0529 * sq + 0.3334 * rs;
    ec = -0.1423 / den;
    dec = 0.1423 * (0.5 * 1.0529 / sq + 0.3334) / (den * den);
  }
  return vx + ec - rs / 3.0 * dec;
}

// vq[e*Q+q] = w(x_q) + V_xc(rho[e*Q+q])
template <int NLOC>
__global__ void k_frozen_potential(int64_t E, const RefTables* __restrict__ ref, const int32_t* __restrict__ elem,
                                   const double* __restrict__ w, const double* __restrict__ rho, int kind,
                                   double alpha, double* __restrict__ vq) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  double wa[NLOC];
#pragma unroll
  for (int a = 0; a < NLOC; ++a) wa[a] = w ? w[elem[e * NLOC + a]] : 0.0;
  for (int q = 0; q < kQ; ++q) {
    double v = 0.0;
#pragma unroll
    for (int a = 0; a < NLOC; ++a) v += ref->phi[q][a] * wa[a];
    vq[e * kQ + q] = v + vxc_of(rho[e * kQ + q], kind, alpha);
  }
}

int density(mk_ctx* ctx, const Level& L, const double* u, int ld, int N, const double* occ_host, double* rho,
            cudaStream_t s) {
  ColParams occ{};
  for (int j = 0; j < N && j < MK_MAX_RHS; ++j) occ.v[j] = occ_host[j];
  const int th = 128, blocks = (int)((L.n_elems + th - 1) / th);
  if (L.nloc == 4)
    MK_COUNT(), k_density<4><<<blocks, th, 0, s>>>(L.n_elems, ctx->d_ref[1], L.d_elem, u, ld, N, occ, rho);
  else
    MK_COUNT(), k_density<10><<<blocks, th, 0, s>>>(L.n_elems, ctx->d_ref[2], L.d_elem, u, ld, N, occ, rho);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

int frozen_potential(mk_ctx* ctx, const Level& L, const double* w, const double* rho, mk_xc xc, double* vq,
                     cudaStream_t s) {
  const int th = 128, blocks = (int)((L.n_elems + th - 1) / th);
  if (L.nloc == 4)
    MK_COUNT(), k_frozen_potential<4><<<blocks, th, 0, s>>>(L.n_elems, ctx->d_ref[1], L.d_elem, w, rho, xc.kind, xc.alpha, vq);
  else
    MK_COUNT(), k_frozen_potential<10><<<blocks, th, 0, s>>>(L.n_elems, ctx->d_ref[2], L.d_elem, w, rho, xc.kind, xc.alpha, vq);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

// ------------------------------------------------------------------------------------------------ Poisson pieces
// F[node(e,a)] += sum_q w_q |det| rho_q phi_a(x_q), one colour at a time.  One warp per element: lane q forms
// c_q = w_q |det| rho_q (a coalesced read of the element's kQ values), lanes a < NLOC sum c_q phi_q[a] over q in
// order with c_q broadcast by shuffle (the same products and order as one thread per element), then scatter.
template <int NLOC>
__global__ void k_load_colour(const int32_t* __restrict__ celems, int count, const RefTables* __restrict__ ref,
                              const int32_t* __restrict__ elem, const Geom* __restrict__ geom,
                              const double* __restrict__ rho, double scale, double* __restrict__ F) {
  static_assert(kQ <= 32, "one quadrature point per lane");
  const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= count) return;  // the whole warp leaves together
  const int e = celems[i];
  const double det = fabs(geom[e].det);
  const double c = lane < kQ ? ref->qw[lane] * det * rho[(int64_t)e * kQ + lane] : 0.0;
  const int a = lane < NLOC ? lane : 0;
  double fa = 0.0;
  for (int q = 0; q < kQ; ++q) {
    const double cq = __shfl_sync(0xffffffffu, c, q);
    fa += cq * ref->phi[q][a];
  }
  if (lane < NLOC) F[elem[(int64_t)e * NLOC + lane]] += scale * fa;
}

int load_vector(mk_ctx* ctx, const Level& L, const double* rho, double scale, double* F, cudaStream_t s) {
  MK_CUDA(cudaMemsetAsync(F, 0, L.n_nodes * sizeof(double), s));
  for (int c = 0; c < L.n_colours; ++c) {
    const int64_t off = L.colour_off[c], cnt = L.colour_off[c + 1] - off;
    const int blocks = (int)((cnt * 32 + 127) / 128);  // four elements (warps) per block
    if (L.nloc == 4)
      MK_COUNT(), k_load_colour<4><<<blocks, 128, 0, s>>>(L.d_colour_elems + off, (int)cnt, ctx->d_ref[1], L.d_elem, L.d_geom,
                                             rho, scale, F);
    else
      MK_COUNT(), k_load_colour<10><<<blocks, 128, 0, s>>>(L.d_colour_elems + off, (int)cnt, ctx->d_ref[2], L.d_elem, L.d_geom,
                                              rho, scale, F);
  }
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

// moments: part[blk*10 + m] for m = (q0, px, py, pz, Qxx, Qyy, Qzz, Qxy, Qxz, Qyz) with Q_ij = int rho (3 x_i x_j - r^2 d_ij)
__global__ void k_moments(int64_t E, const RefTables* __restrict__ ref, const Geom* __restrict__ geom,
                          const double* __restrict__ rho, double* __restrict__ part) {
  __shared__ double sh[10][kRedThreads];
  double acc[10];
#pragma unroll
  for (int m = 0; m < 10; ++m) acc[m] = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const Geom g = geom[e];
    const double det = fabs(g.det);
    for (int q = 0; q < kQ; ++q) {
      const double xi = ref->qx[q][0], et = ref->qx[q][1], ze = ref->qx[q][2];
      const double x = g.x0[0] + g.J[0] * xi + g.J[1] * et + g.J[2] * ze;
      const double y = g.x0[1] + g.J[3] * xi + g.J[4] * et + g.J[5] * ze;
      const double z = g.x0[2] + g.J[6] * xi + g.J[7] * et + g.J[8] * ze;
      const double w = ref->qw[q] * det * rho[e * kQ + q];
      const double r2 = x * x + y * y + z * z;
      acc[0] += w;
      acc[1] += w * x; acc[2] += w * y; acc[3] += w * z;
      acc[4] += w * (3 * x * x - r2); acc[5] += w * (3 * y * y - r2); acc[6] += w * (3 * z * z - r2);
      acc[7] += w * 3 * x * y; acc[8] += w * 3 * x * z; acc[9] += w * 3 * y * z;
    }
  }
#pragma unroll
  for (int m = 0; m < 10; ++m) sh[m][threadIdx.x] = acc[m];
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
#pragma unroll
      for (int m = 0; m < 10; ++m) sh[m][threadIdx.x] += sh[m][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x < 10) part[blockIdx.x * 10 + threadIdx.x] = sh[threadIdx.x][0];
}

// w[node] = multipole value on boundary nodes, 0 elsewhere
__global__ void k_multipole_bc(int64_t n, const double* __restrict__ nodes, const uint8_t* __restrict__ bnd,
                               const double* __restrict__ mom, int use, double* __restrict__ w) {
  const int64_t nd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (nd >= n) return;
  double v = 0.0;
  if (bnd[nd] && use) {
    const double x = nodes[nd * 3], y = nodes[nd * 3 + 1], z = nodes[nd * 3 + 2];
    const double r2 = x * x + y * y + z * z, r = sqrt(r2);
    const double quad = mom[4] * x * x + mom[5] * y * y + mom[6] * z * z +
                        2.0 * (mom[7] * x * y + mom[8] * x * z + mom[9] * y * z);
    v = mom[0] / r + (mom[1] * x + mom[2] * y + mom[3] * z) / (r2 * r) + 0.5 * quad / (r2 * r2 * r);
  }
  w[nd] = v;
}

int multipole_boundary(mk_ctx* ctx, const Level& L, const double* rho, const double* d_nodes, int bc, double* w,
                       cudaStream_t s) {
  int err = MK_OK;
  const int nblk = red_blocks(ctx);
  double* part = (double*)scratch(ctx, S_RED, (size_t)nblk * 10 * sizeof(double), &err);
  double* mom = (double*)scratch(ctx, S_SCAL, 64 * sizeof(double), &err);
  if (!part || !mom) return err;
  MK_COUNT(), k_moments<<<nblk, kRedThreads, 0, s>>>(L.n_elems, ctx->d_ref[L.order], L.d_geom, rho, part);
  sum_partials(part, nblk, 10, mom, s);
  MK_COUNT(), k_multipole_bc<<<(int)((L.n_nodes + 255) / 256), 256, 0, s>>>(L.n_nodes, d_nodes, L.d_boundary, mom,
                                                                 bc == MK_BC_MULTIPOLE, w);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

}  // namespace mk
