// The outer AFEM loop's Estimate and Mark steps (Sec. 2): the residual a posteriori error indicator of the
// eigenpair approximation (Lambda_h, Phi_h) and Dorfler's marking.
//
//   eta^2(T) = h_T^2 sum_i ||H phi_i - lambda_i phi_i||_{0,T}^2 + sum over the interior faces e of T of
//              h_e sum_i ||1/2 grad phi_i|T+ . nu+ + 1/2 grad phi_i|T- . nu-||_{0,e}^2,
// H = -1/2 Laplacian + V_ext + vq (vq = w + V_xc at the quadrature points); h_T, h_e the longest edges; the element
// integral by the 27-point rule, the face integral by the 3-point rule at the face's edge midpoints (exact: the
// jump is linear on a face for P2).  Each interior face is evaluated once, by its lower-index element, which writes
// the value to the face slots of both elements; each element then adds its four slots in slot order: no atomics,
// the same result on every run.
// Dorfler: the marked set is {T : eta^2(T) >= t*} with t* the largest t for which the indicators at or above t sum
// to at least theta times the total, found by bisection on the bit patterns of t (indicators are >= 0, so the
// patterns order like the values): at most 64 fixed-order reductions.  Without ties at the cut this is the
// smallest set in order of decreasing eta^2; elements tied with the cut value are all marked.
#include <algorithm>
#include <array>
#include <cstring>
#include <vector>

#include "mk_device.cuh"

namespace mk {

namespace {

constexpr int kFaceVerts[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
// vertex j (0..2) of the face opposite local vertex k: the other three in increasing order
__host__ __device__ __forceinline__ int face_vertex(int k, int j) { return j + (j >= k ? 1 : 0); }

__device__ __forceinline__ void load_vertices(const double* __restrict__ nodes, const int32_t* __restrict__ elem,
                                              int64_t e, int nloc, double X[4][3]) {
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int64_t nd = elem[e * nloc + v];
#pragma unroll
    for (int r = 0; r < 3; ++r) X[v][r] = nodes[nd * 3 + r];
  }
}

// Physical gradients of the barycentric coordinates: grad lambda_k = row k-1 of J^-1, grad lambda_0 = -their sum.
__device__ __forceinline__ void bary_grads(const Geom& g, double G[4][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    G[1][c] = g.Jinv[c];
    G[2][c] = g.Jinv[3 + c];
    G[3][c] = g.Jinv[6 + c];
    G[0][c] = -(G[1][c] + G[2][c] + G[3][c]);
  }
}

// grad of the FE function with local nodal values u (stride ld, N columns) of element g at physical point x,
// accumulated with weight sgn into out[i][3]
template <int NLOC>
__device__ __forceinline__ void add_gradient(const Geom& g, const double x[3], const int32_t* __restrict__ nd,
                                             const double* __restrict__ psi, int ld, int N, double sgn,
                                             double (*out)[3]) {
  double s[3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
    s[r] = g.Jinv[r * 3] * (x[0] - g.x0[0]) + g.Jinv[r * 3 + 1] * (x[1] - g.x0[1]) + g.Jinv[r * 3 + 2] * (x[2] - g.x0[2]);
  const double l[4] = {1.0 - s[0] - s[1] - s[2], s[0], s[1], s[2]};
  double G[4][3];
  bary_grads(g, G);
  double dphi[NLOC][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) dphi[a][c] = (NLOC == 4 ? 1.0 : 4.0 * l[a] - 1.0) * G[a][c];
  if (NLOC == 10) {
    const int ea[6] = {0, 0, 0, 1, 1, 2}, eb[6] = {1, 2, 3, 2, 3, 3};
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) dphi[(4 + k) % NLOC][c] = 4.0 * (l[eb[k]] * G[ea[k]][c] + l[ea[k]] * G[eb[k]][c]);
  }
  for (int i = 0; i < N; ++i) {
    double gr[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < NLOC; ++a) {
      const double u = psi[(int64_t)nd[a] * ld + i];
#pragma unroll
      for (int c = 0; c < 3; ++c) gr[c] += u * dphi[a][c];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) out[i][c] += sgn * gr[c];
  }
}

__device__ __forceinline__ double dist3(const double* a, const double* b) {
  const double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
  return sqrt(dx * dx + dy * dy + dz * dz);
}

}  // namespace

// One thread per (element e, face slot k) whose neighbour has a higher index: h_e ||J||^2 over the face, written
// to both face slots.  Slots on the boundary get 0.
template <int NLOC>
__global__ void k_face_jump(int64_t E, const int32_t* __restrict__ nb, const Geom* __restrict__ geom,
                            const int32_t* __restrict__ elem, const double* __restrict__ nodes,
                            const double* __restrict__ psi, int ld, int N, double* __restrict__ faceval) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= E * 4) return;
  const int64_t e = t / 4;
  const int k = (int)(t % 4);
  const int32_t o = nb[t];
  if (o < 0) {
    faceval[t] = 0.0;
    return;
  }
  const int64_t n = o / 4;
  if (n < e) return;  // the lower-index element owns the face
  double X[4][3];
  load_vertices(nodes, elem, e, NLOC, X);
  const double* A = X[face_vertex(k, 0)];
  const double* B = X[face_vertex(k, 1)];
  const double* C = X[face_vertex(k, 2)];
  const double u1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]}, u2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
  double nu[3] = {u1[1] * u2[2] - u1[2] * u2[1], u1[2] * u2[0] - u1[0] * u2[2], u1[0] * u2[1] - u1[1] * u2[0]};
  const double nn = sqrt(nu[0] * nu[0] + nu[1] * nu[1] + nu[2] * nu[2]);
  const double area = 0.5 * nn;
#pragma unroll
  for (int c = 0; c < 3; ++c) nu[c] /= nn;
  const double* opp = X[k];
  if (nu[0] * (A[0] - opp[0]) + nu[1] * (A[1] - opp[1]) + nu[2] * (A[2] - opp[2]) < 0.0)
#pragma unroll
    for (int c = 0; c < 3; ++c) nu[c] = -nu[c];  // outward from e
  const double he = fmax(fmax(dist3(A, B), dist3(A, C)), dist3(B, C));
  int32_t nde[NLOC], ndn[NLOC];
#pragma unroll
  for (int a = 0; a < NLOC; ++a) {
    nde[a] = elem[e * NLOC + a];
    ndn[a] = elem[n * NLOC + a];
  }
  const Geom ge = geom[e], gn = geom[n];
  const double* P[3][2] = {{A, B}, {A, C}, {B, C}};
  double jj = 0.0;
  double d[MK_MAX_RHS][3];
  for (int m = 0; m < 3; ++m) {
    const double x[3] = {0.5 * (P[m][0][0] + P[m][1][0]), 0.5 * (P[m][0][1] + P[m][1][1]),
                         0.5 * (P[m][0][2] + P[m][1][2])};
    for (int i = 0; i < N; ++i) d[i][0] = d[i][1] = d[i][2] = 0.0;
    add_gradient<NLOC>(ge, x, nde, psi, ld, N, 1.0, d);
    add_gradient<NLOC>(gn, x, ndn, psi, ld, N, -1.0, d);
    double s = 0.0;
    for (int i = 0; i < N; ++i) {
      const double J = 0.5 * (nu[0] * d[i][0] + nu[1] * d[i][1] + nu[2] * d[i][2]);
      s += J * J;
    }
    jj += s * area / 3.0;
  }
  const double v = he * jj;
  faceval[t] = v;
  faceval[o] = v;
}

// One thread per element: h_T^2 ||R_T||^2 plus its four face slots.
template <int NLOC>
__global__ void k_elem_indicator(int64_t E, const RefTables* __restrict__ ref, const Geom* __restrict__ geom,
                                 const int32_t* __restrict__ elem, const double* __restrict__ nodes,
                                 const NucParams nucp, const double* __restrict__ psi, int ld, int N,
                                 const ColParams lam, const double* __restrict__ vq,
                                 const double* __restrict__ faceval, double* __restrict__ eta2) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const Geom g = geom[e];
  double X[4][3];
  load_vertices(nodes, elem, e, NLOC, X);
  double hT = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = a + 1; b < 4; ++b) hT = fmax(hT, dist3(X[a], X[b]));
  // Laplacians of the basis functions (constant per element): 4 |grad l_a|^2 and 8 grad l_a . grad l_b for P2
  double L[NLOC];
  if (NLOC == 4) {
#pragma unroll
    for (int a = 0; a < NLOC; ++a) L[a] = 0.0;
  } else {
    double G[4][3];
    bary_grads(g, G);
    auto dot = [&](int a, int b) { return G[a][0] * G[b][0] + G[a][1] * G[b][1] + G[a][2] * G[b][2]; };
#pragma unroll
    for (int a = 0; a < 4; ++a) L[a] = 4.0 * dot(a, a);
    const int ea[6] = {0, 0, 0, 1, 1, 2}, eb[6] = {1, 2, 3, 2, 3, 3};
#pragma unroll
    for (int k = 0; k < 6; ++k) L[(4 + k) % NLOC] = 8.0 * dot(ea[k], eb[k]);
  }
  double V[kQ], wq[kQ];
  const double det = fabs(g.det);
  for (int q = 0; q < kQ; ++q) {
    const double xi = ref->qx[q][0], et = ref->qx[q][1], ze = ref->qx[q][2];
    const double x = g.x0[0] + g.J[0] * xi + g.J[1] * et + g.J[2] * ze;
    const double y = g.x0[1] + g.J[3] * xi + g.J[4] * et + g.J[5] * ze;
    const double z = g.x0[2] + g.J[6] * xi + g.J[7] * et + g.J[8] * ze;
    V[q] = nuclear_potential(nucp, x, y, z) + vq[e * kQ + q];
    wq[q] = ref->qw[q] * det;
  }
  int32_t nd[NLOC];
#pragma unroll
  for (int a = 0; a < NLOC; ++a) nd[a] = elem[e * NLOC + a];
  double acc = 0.0;
  for (int i = 0; i < N; ++i) {
    double u[NLOC];
    double lap = 0.0;
#pragma unroll
    for (int a = 0; a < NLOC; ++a) {
      u[a] = psi[(int64_t)nd[a] * ld + i];
      lap += L[a] * u[a];
    }
    for (int q = 0; q < kQ; ++q) {
      double v = 0.0;
#pragma unroll
      for (int a = 0; a < NLOC; ++a) v += ref->phi[q][a] * u[a];
      const double R = -0.5 * lap + (V[q] - lam.v[i]) * v;
      acc += wq[q] * R * R;
    }
  }
  eta2[e] = hT * hT * acc + ((faceval[e * 4] + faceval[e * 4 + 1]) + faceval[e * 4 + 2]) + faceval[e * 4 + 3];
}

// part[blk] = sum of eta2 >= t over the block's grid-stride share (fixed order)
__global__ void k_df_partial(int64_t n, const double* __restrict__ eta2, double t, double* __restrict__ part) {
  __shared__ double sh[kRedThreads];
  double v = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    if (eta2[k] >= t) v += eta2[k];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_df_mark(int64_t n, const double* __restrict__ eta2, double t, uint8_t* __restrict__ marked,
                          double* __restrict__ part) {
  __shared__ double sh[kRedThreads];
  double c = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const bool m = eta2[k] >= t;
    marked[k] = m ? 1 : 0;
    c += m ? 1.0 : 0.0;
  }
  sh[threadIdx.x] = c;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// Face neighbours of the fine mesh on the host: faces keyed by their sorted vertex ids, equal keys paired.
static int build_face_neighbours(const mk_mesh* m) {
  const Level& F = m->fine;
  const int64_t E = F.n_elems;
  const int nl = F.nloc;
  struct Key {
    std::array<int32_t, 3> v;
    int64_t slot;
  };
  std::vector<Key> keys((size_t)E * 4);
  for (int64_t e = 0; e < E; ++e)
    for (int k = 0; k < 4; ++k) {
      std::array<int32_t, 3> v = {F.elem[e * nl + kFaceVerts[k][0]], F.elem[e * nl + kFaceVerts[k][1]],
                                  F.elem[e * nl + kFaceVerts[k][2]]};
      std::sort(v.begin(), v.end());
      keys[e * 4 + k] = Key{v, e * 4 + k};
    }
  std::sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
    return a.v != b.v ? a.v < b.v : a.slot < b.slot;
  });
  std::vector<int32_t> nb((size_t)E * 4, -1);
  for (size_t i = 0; i < keys.size();) {
    size_t j = i + 1;
    while (j < keys.size() && keys[j].v == keys[i].v) ++j;
    if (j - i > 2) return fail(MK_ERR_INVALID_ARG, "error indicator: a face shared by more than two elements");
    if (j - i == 2) {
      nb[keys[i].slot] = (int32_t)keys[i + 1].slot;
      nb[keys[i + 1].slot] = (int32_t)keys[i].slot;
    }
    i = j;
  }
  if (cudaMalloc(&m->d_face_nb, nb.size() * sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    m->d_face_nb = nullptr;
    return fail(MK_ERR_OOM, "error indicator: face table allocation failed");
  }
  MK_CUDA(cudaMemcpy(m->d_face_nb, nb.data(), nb.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  return MK_OK;
}

}  // namespace mk

using namespace mk;

extern "C" {

int mk_error_indicators(mk_ctx* ctx, const mk_mesh* m, const mk_molecule* mol, const double* psi, int ld, int N,
                        const double* lambda, const double* vq, double* eta2, void* stream) {
  MK_ARG(ctx && m && mol && psi && lambda && vq && eta2, "mk_error_indicators: null argument");
  MK_ARG(N >= 1 && N <= ld && N <= MK_MAX_RHS, "mk_error_indicators: bad N/ld");
  MK_ARG(mol->n_nuclei <= kMaxNuclei, "mk_error_indicators: at most 64 nuclei are supported");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const Level& F = m->fine;
  const int64_t E = F.n_elems;
  if (!m->d_face_nb) MK_TRY(build_face_neighbours(m));
  int err = MK_OK;
  double* fv = (double*)scratch(ctx, S_AFEM, (size_t)E * 4 * sizeof(double), &err);
  if (!fv) return err;
  ColParams lam{};
  for (int i = 0; i < N; ++i) lam.v[i] = lambda[i];
  const NucParams nucp = make_nuc(mol);
  const int fb = (int)((E * 4 + 127) / 128), eb = (int)((E + 127) / 128);
  if (F.nloc == 4) {
    MK_COUNT(), k_face_jump<4><<<fb, 128, 0, s>>>(E, m->d_face_nb, F.d_geom, F.d_elem, F.d_nodes, psi, ld, N, fv);
    MK_COUNT(), k_elem_indicator<4><<<eb, 128, 0, s>>>(E, ctx->d_ref[1], F.d_geom, F.d_elem, F.d_nodes, nucp, psi,
                                                        ld, N, lam, vq, fv, eta2);
  } else {
    MK_COUNT(), k_face_jump<10><<<fb, 128, 0, s>>>(E, m->d_face_nb, F.d_geom, F.d_elem, F.d_nodes, psi, ld, N, fv);
    MK_COUNT(), k_elem_indicator<10><<<eb, 128, 0, s>>>(E, ctx->d_ref[2], F.d_geom, F.d_elem, F.d_nodes, nucp, psi,
                                                         ld, N, lam, vq, fv, eta2);
  }
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

int mk_dorfler_mark(mk_ctx* ctx, int64_t n, const double* eta2, double theta, uint8_t* marked, int64_t* n_marked,
                    double* threshold, void* stream) {
  MK_ARG(ctx && eta2 && marked && n >= 1, "mk_dorfler_mark: bad argument");
  MK_ARG(theta > 0.0 && theta <= 1.0, "mk_dorfler_mark: theta must lie in (0, 1]");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int nblk = red_blocks(ctx);
  int err = MK_OK;
  double* part = (double*)scratch(ctx, S_RED, (size_t)nblk * sizeof(double) + 64, &err);
  double* sum = (double*)scratch(ctx, S_SCAL, 64, &err);
  if (!part || !sum) return err;
  auto S = [&](double t, double* out) -> int {
    MK_COUNT(), k_df_partial<<<nblk, kRedThreads, 0, s>>>(n, eta2, t, part);
    sum_partials(part, nblk, 1, sum, s);
    MK_CUDA(cudaMemcpyAsync(out, sum, sizeof(double), cudaMemcpyDeviceToHost, s));
    MK_CUDA(cudaStreamSynchronize(s));
    return MK_OK;
  };
  double total = 0.0;
  MK_TRY(S(0.0, &total));
  MK_ARG(total > 0.0, "mk_dorfler_mark: the indicators sum to zero");
  const double goal = theta * total;
  // lo: a valid threshold (S(lo) >= goal), hi: an invalid one; both as bit patterns of non-negative doubles
  uint64_t lo = 0, hi = 0x7FF0000000000000ull;  // +inf: nothing is at or above it
  while (hi - lo > 1) {
    const uint64_t mid = lo + (hi - lo) / 2;
    double v = 0.0;
    double tm;
    std::memcpy(&tm, &mid, sizeof(tm));
    MK_TRY(S(tm, &v));
    if (v >= goal) lo = mid; else hi = mid;
  }
  double t;
  std::memcpy(&t, &lo, sizeof(t));
  MK_COUNT(), k_df_mark<<<nblk, kRedThreads, 0, s>>>(n, eta2, t, marked, part);
  sum_partials(part, nblk, 1, sum, s);
  double cnt = 0.0;
  MK_CUDA(cudaMemcpyAsync(&cnt, sum, sizeof(double), cudaMemcpyDeviceToHost, s));
  MK_CUDA(cudaStreamSynchronize(s));
  if (n_marked) *n_marked = (int64_t)cnt;
  if (threshold) *threshold = t;
  return MK_OK;
}

}  // extern "C"
