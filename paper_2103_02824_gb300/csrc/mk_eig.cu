// A7: the small augmented eigenproblem of Eq. (Eigenvalue_H_h) for every orbital, and A8: the corrected orbitals.
//
// All orbitals share the coarse pencil (A_H, M_H).  It is decomposed once, in FP64: Cholesky M_H = L L^T,
// C = L^-1 A_H L^-T, cyclic Jacobi C = Q diag(d) Q^T (parallel round-robin ordering, cooperative grid),
// V = L^-T Q (M_H-orthonormal, A_H V = M_H V diag(d)).  For orbital i the extra direction psi^ is made
// M-orthogonal to V_H: with p = V^T c and ||u||^2 = gamma - |p|^2, the pencil becomes, in the orthonormal basis
// [V, u/||u||], the arrowhead matrix [[diag(d), z], [z^T, alpha]] with z = (V^T b - d .* p)/||u|| and
// alpha = (beta - 2 p.(V^T b) + p.(d .* p))/||u||^2.  Its eigenvalues are d_k for deflated k (z_k ~ 0, or d_k
// repeated) and the roots of the secular equation alpha - mu + sum_k z_k^2/(mu - d_k) = 0, one per interlacing
// interval, found by bisection in the offset from the nearer pole.  Every eigenvector's score |(x, psi^)_M| is
// formed and the largest kept (Algorithm 2 (a)); ties within 1e-12 go to the lower eigenvalue.
#include <cooperative_groups.h>

#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "mk_device.cuh"

namespace cg = cooperative_groups;

namespace mk {

// ------------------------------------------------------------------------------------------------ Cholesky
// Left-looking Cholesky of the n x n SPD matrix A (row-major); writes LT = L^T row-major (LT[k][i] = L[i][k]).
__global__ void k_cholesky(int n, const double* __restrict__ A, double* __restrict__ LT, int* __restrict__ flag) {
  __shared__ double red[1024];
  __shared__ double ljj;
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int k = threadIdx.x; k < j; k += blockDim.x) {
      const double v = LT[(int64_t)k * n + j];
      s += v * v;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double dd = A[(int64_t)j * n + j] - red[0];
      if (!(dd > 0.0)) *flag = 1;
      ljj = sqrt(fmax(dd, 1e-300));
      LT[(int64_t)j * n + j] = ljj;
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
      double t = A[(int64_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= LT[(int64_t)k * n + i] * LT[(int64_t)k * n + j];
      LT[(int64_t)j * n + i] = t / ljj;
    }
    for (int i = threadIdx.x; i < j; i += blockDim.x) LT[(int64_t)j * n + i] = 0.0;
    __syncthreads();
  }
}

// X = L^-1 B for each column of B (thread per column): forward substitution.
__global__ void k_forward(int n, const double* __restrict__ LT, const double* __restrict__ B, double* __restrict__ X) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int i = 0; i < n; ++i) {
    double t = B[(int64_t)i * n + j];
    for (int k = 0; k < i; ++k) t -= LT[(int64_t)k * n + i] * X[(int64_t)k * n + j];
    X[(int64_t)i * n + j] = t / LT[(int64_t)i * n + i];
  }
}

// X = L^-T B for each column (thread per column): back substitution with L^T.
__global__ void k_backward(int n, const double* __restrict__ LT, const double* __restrict__ B, double* __restrict__ X,
                           int ldb, int ldx) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int i = n - 1; i >= 0; --i) {
    double t = B[(int64_t)i * ldb + j];
    for (int k = i + 1; k < n; ++k) t -= LT[(int64_t)i * n + k] * X[(int64_t)k * ldx + j];
    X[(int64_t)i * ldx + j] = t / LT[(int64_t)i * n + i];
  }
}

__global__ void k_identity(int n, double* __restrict__ I) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < (int64_t)n * n) I[t] = (t / n == t % n) ? 1.0 : 0.0;
}

__global__ void k_transpose(int n, const double* __restrict__ A, double* __restrict__ B) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  B[(int64_t)j * n + i] = A[t];
}

// C (n x n) -> padded symmetric n2 x n2 (n2 even) with (C + C^T)/2; Q = I.
__global__ void k_pad_sym(int n, int n2, const double* __restrict__ C, double* __restrict__ S, double* __restrict__ Q,
                          double pad) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n2 * n2) return;
  const int i = (int)(t / n2), j = (int)(t % n2);
  double v = 0.0;
  if (i < n && j < n) v = 0.5 * (C[(int64_t)i * n + j] + C[(int64_t)j * n + i]);
  else if (i == j) v = pad;
  S[t] = v;
  Q[t] = (i == j) ? 1.0 : 0.0;
}

struct Rot {
  int p, q;
  double c, s;
};

__device__ __forceinline__ void pair_of(int r, int k, int n2, int* p, int* q) {
  int a, b;
  if (k == 0) {
    a = n2 - 1;
    b = r;
  } else {
    a = (r + k) % (n2 - 1);
    b = (r - k + (n2 - 1)) % (n2 - 1);
  }
  *p = min(a, b);
  *q = max(a, b);
}

// Rotation in the (p,q) plane that zeroes S[p][q]: J = [[c, s], [-s, c]], t = s/c the smaller root of
// t^2 + 2 theta t - 1 = 0, theta = (S_qq - S_pp) / (2 S_pq).
__device__ __forceinline__ Rot make_rot(const double* __restrict__ S, int n2, int r, int k) {
  int p, q;
  pair_of(r, k, n2, &p, &q);
  const double apq = S[(int64_t)p * n2 + q];
  double c = 1.0, s = 0.0;
  if (apq != 0.0) {
    const double app = S[(int64_t)p * n2 + p], aqq = S[(int64_t)q * n2 + q];
    const double theta = (aqq - app) / (2.0 * apq);
    const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
    c = 1.0 / sqrt(t * t + 1.0);
    s = t * c;
  }
  return Rot{p, q, c, s};
}

// Cyclic Jacobi on the symmetric n2 x n2 matrix (n2 even) in parallel round-robin order, accumulating Q <- Q J.
// Cooperative launch.  Round r reads S_in and writes S_out (ping-pong): every CTA first derives all n2/2
// rotations of the round from S_in into shared memory, then updates its share of the disjoint 2x2 blocks and
// of Q; one grid barrier per round.  *final_buf tells which buffer holds the result.
__global__ void k_jacobi(int n2, double* __restrict__ S0, double* __restrict__ S1, double* __restrict__ Q,
                         double* __restrict__ red, int max_sweeps, double tol, int* __restrict__ info) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ unsigned char smem_raw[];
  Rot* rot = reinterpret_cast<Rot*>(smem_raw);
  __shared__ double sh[256];
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  const int np = n2 / 2;
  const int64_t nblk2 = (int64_t)np * (np + 1) / 2;
  double* Sin = S0;
  double* Sout = S1;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int64_t t = tid; t < (int64_t)n2 * n2; t += nth) {
      const double v = Sin[t];
      tot += v * v;
      if (t / n2 != t % n2) off += v * v;
    }
    for (int pass = 0; pass < 2; ++pass) {
      sh[threadIdx.x] = pass == 0 ? off : tot;
      __syncthreads();
      for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
      }
      if (threadIdx.x == 0) red[2 * blockIdx.x + pass] = sh[0];
      __syncthreads();
    }
    grid.sync();
    double o = 0.0, f = 0.0;
    for (int bl = 0; bl < (int)gridDim.x; ++bl) {
      o += red[2 * bl];
      f += red[2 * bl + 1];
    }
    grid.sync();
    if (o <= tol * tol * f) break;
    for (int r = 0; r < n2 - 1; ++r) {
      for (int k = threadIdx.x; k < np; k += blockDim.x) rot[k] = make_rot(Sin, n2, r, k);
      __syncthreads();
      for (int64_t t = tid; t < nblk2; t += nth) {
        int k1 = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) / 2.0);
        while ((int64_t)(k1 + 1) * (k1 + 2) / 2 <= t) ++k1;
        while ((int64_t)k1 * (k1 + 1) / 2 > t) --k1;
        const int k2 = (int)(t - (int64_t)k1 * (k1 + 1) / 2);  // k2 <= k1
        const Rot A = rot[k2], B = rot[k1];                    // rows from pair k2, columns from pair k1
        const double b00 = Sin[(int64_t)A.p * n2 + B.p], b01 = Sin[(int64_t)A.p * n2 + B.q];
        const double b10 = Sin[(int64_t)A.q * n2 + B.p], b11 = Sin[(int64_t)A.q * n2 + B.q];
        const double r00 = A.c * b00 - A.s * b10, r01 = A.c * b01 - A.s * b11;
        const double r10 = A.s * b00 + A.c * b10, r11 = A.s * b01 + A.c * b11;
        double n00 = B.c * r00 - B.s * r01, n01 = B.s * r00 + B.c * r01;
        double n10 = B.c * r10 - B.s * r11, n11 = B.s * r10 + B.c * r11;
        if (k1 == k2) {
          n01 = 0.0;
          n10 = 0.0;
        }
        Sout[(int64_t)A.p * n2 + B.p] = n00;
        Sout[(int64_t)A.p * n2 + B.q] = n01;
        Sout[(int64_t)A.q * n2 + B.p] = n10;
        Sout[(int64_t)A.q * n2 + B.q] = n11;
        if (k1 != k2) {
          Sout[(int64_t)B.p * n2 + A.p] = n00;
          Sout[(int64_t)B.q * n2 + A.p] = n01;
          Sout[(int64_t)B.p * n2 + A.q] = n10;
          Sout[(int64_t)B.q * n2 + A.q] = n11;
        }
      }
      for (int64_t t = tid; t < (int64_t)n2 * np; t += nth) {
        const int row = (int)(t / np), k = (int)(t % np);
        const Rot R = rot[k];
        const double vp = Q[(int64_t)row * n2 + R.p], vq = Q[(int64_t)row * n2 + R.q];
        Q[(int64_t)row * n2 + R.p] = R.c * vp - R.s * vq;
        Q[(int64_t)row * n2 + R.q] = R.s * vp + R.c * vq;
      }
      grid.sync();
      double* tmp = Sin;
      Sin = Sout;
      Sout = tmp;
    }
  }
  if (tid == 0) {
    info[0] = sweep;
    info[1] = (Sin == S0) ? 0 : 1;
  }
}

// C[M x N] = op(A) op(B), op(X) = X or X^T (row-major storage), FP64, 32x32 tiles.
__global__ void k_gemm64(int M, int N, int K, const double* __restrict__ A, int lda, int ta,
                         const double* __restrict__ B, int ldb, int tb, double* __restrict__ C, int ldc) {
  __shared__ double As[32][33], Bs[32][33];
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8 threads
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int i = i0 + r, k = k0 + tx;
      As[r][tx] = (i < M && k < K) ? (ta ? A[(int64_t)k * lda + i] : A[(int64_t)i * lda + k]) : 0.0;
      const int kk = k0 + r, j = j0 + tx;
      Bs[r][tx] = (kk < K && j < N) ? (tb ? B[(int64_t)j * ldb + kk] : B[(int64_t)kk * ldb + j]) : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const double bv = Bs[k][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += As[ty + 8 * q][k] * bv;
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + ty + 8 * q, j = j0 + tx;
    if (i < M && j < N) C[(int64_t)i * ldc + j] = acc[q];
  }
}

static void gemm64(int M, int N, int K, const double* A, int lda, int ta, const double* B, int ldb, int tb, double* C,
                   int ldc, cudaStream_t s) {
  dim3 grid((N + 31) / 32, (M + 31) / 32);
  MK_COUNT(), k_gemm64<<<grid, 256, 0, s>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc);
}

// Sort the n eigenvalues (diag of S, first n of n2) ascending: perm[rank] = index (ties by index).
__global__ void k_rank(int n, int n2, const double* __restrict__ S, double* __restrict__ d, int* __restrict__ perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = S[(int64_t)i * n2 + i];
  int r = 0;
  for (int k = 0; k < n; ++k) {
    const double w = S[(int64_t)k * n2 + k];
    if (w < v || (w == v && k < i)) ++r;
  }
  d[r] = v;
  perm[r] = i;
}

// Qs[i][r] = Q[i][perm[r]] (n x n, columns sorted)
__global__ void k_gather_cols(int n, int n2, const double* __restrict__ Q, const int* __restrict__ perm,
                              double* __restrict__ Qs) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int i = (int)(t / n), r = (int)(t % n);
  Qs[t] = Q[(int64_t)i * n2 + perm[r]];
}

// G[k][col] = sum_i V[i][k] B[i][col]  (V^T [b|c]); B has 2N columns: b (ld N) then c (ld N)
__global__ void k_vt_bc(int n, int N, const double* __restrict__ V, const double* __restrict__ b,
                        const double* __restrict__ c, double* __restrict__ G) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * 2 * N) return;
  const int k = (int)(t / (2 * N)), col = (int)(t % (2 * N));
  const double* B = col < N ? b : c;
  const int j = col < N ? col : col - N;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += V[(int64_t)i * n + k] * B[(int64_t)i * N + j];
  G[(int64_t)k * 2 * N + col] = s;
}

// ------------------------------------------------------------------------------------------------ secular
__device__ __forceinline__ double secular_f(int m, const double* __restrict__ dd, const double* __restrict__ zz,
                                            double alpha, double origin, double delta) {
  double f = alpha - (origin + delta);
  for (int k = 0; k < m; ++k) {
    const double den = (origin - dd[k]) + delta;
    f += zz[k] * zz[k] / den;
  }
  return f;
}

constexpr int kEigThreads = 256;

// One block per orbital.  Work arrays in global memory: per orbital kWorkVecs*(n+1) doubles, 4*(n+1) ints.
constexpr int kWorkVecs = 10;

__global__ void k_secular_select(int n, int N, const double* __restrict__ d, const double* __restrict__ V,
                                 const double* __restrict__ G, const double* __restrict__ beta,
                                 const double* __restrict__ gamma, double* __restrict__ work, int* __restrict__ iwork,
                                 double* __restrict__ lambda, double* __restrict__ coef, int32_t* __restrict__ status,
                                 double sing_rtol, double tie_rtol) {
  const int i = blockIdx.x;
  if (i >= N) return;
  const int64_t n1 = n + 1;
  double* zs = work + (int64_t)i * kWorkVecs * n1;  // z in the (rotated) V basis
  double* ps = zs + n1;                             // p = V^T c in the (rotated) V basis
  double* dk = ps + n1;                             // poles kept in the secular equation
  double* zk = dk + n1;                             // their z
  double* score = zk + n1;                          // per candidate |(x, psi^)_M|
  double* eig = score + n1;                         // per candidate eigenvalue
  double* yv = eig + n1;                            // per root: offset delta; later the selected eigenvector
  double* rcos = yv + n1;                           // deflation rotation of index k with its partner
  double* rsin = rcos + n1;
  double* ytmp = rsin + n1;
  int* kind = iwork + (int64_t)i * 4 * n1;          // candidate t: >= 0 root index, < 0 deflated -(k+1)
  int* comp = kind + n1;                            // kept pole -> original index
  int* partner = comp + n1;                         // rotation partner of k (-1 none)
  int* origin_idx = partner + n1;                   // per root: kept pole used as origin
  __shared__ double s_alpha, s_un, s_norm, s_sign, s_ylast;
  __shared__ int s_m, s_ncand, s_sel, s_singular;
  __shared__ double s_red[kEigThreads];
  const int tid = threadIdx.x;
  // p = V^T c, g = V^T b;  ||u||^2 = gamma - |p|^2 (u = psi^ - Pi_H psi^, V is M_H-orthonormal)
  double pp = 0.0;
  for (int k = tid; k < n; k += blockDim.x) {
    const double pk = G[(int64_t)k * 2 * N + N + i];
    pp += pk * pk;
  }
  s_red[tid] = pp;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (tid < st) s_red[tid] += s_red[tid + st];
    __syncthreads();
  }
  if (tid == 0) {
    const double u2 = gamma[i] - s_red[0];
    s_singular = !(u2 > sing_rtol * sing_rtol * gamma[i]);
    s_un = s_singular ? 0.0 : sqrt(u2);
  }
  __syncthreads();
  if (s_singular) {  // psi^ in V_H: coarse Ritz pair with the largest |(v_k, Pi_H psi^)_M| = |p_k|
    if (tid == 0) {
      double best = -1.0;
      for (int k = 0; k < n; ++k) best = fmax(best, fabs(G[(int64_t)k * 2 * N + N + i]));
      int sel = 0;
      for (int k = 0; k < n; ++k)
        if (fabs(G[(int64_t)k * 2 * N + N + i]) >= best * (1.0 - tie_rtol)) { sel = k; break; }
      s_sel = sel;
      lambda[i] = d[sel];
      status[i] = MK_ERR_SINGULAR_AUG;
    }
    __syncthreads();
    const double sgn = G[(int64_t)s_sel * 2 * N + N + i] < 0 ? -1.0 : 1.0;
    for (int r = tid; r < n; r += blockDim.x) coef[(int64_t)r * N + i] = sgn * V[(int64_t)r * n + s_sel];
    if (tid == 0) coef[(int64_t)n * N + i] = 0.0;
    return;
  }
  // z = (V^T b - d .* p)/||u||, alpha = (beta - 2 p.(V^T b) + p.(d .* p))/||u||^2
  double a2 = 0.0;
  for (int k = tid; k < n; k += blockDim.x) {
    const double gk = G[(int64_t)k * 2 * N + i], pk = G[(int64_t)k * 2 * N + N + i];
    zs[k] = (gk - d[k] * pk) / s_un;
    ps[k] = pk;
    partner[k] = -1;
    a2 += -2.0 * pk * gk + pk * d[k] * pk;
  }
  s_red[tid] = a2;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (tid < st) s_red[tid] += s_red[tid + st];
    __syncthreads();
  }
  if (tid == 0) {
    s_alpha = (beta[i] + s_red[0]) / (s_un * s_un);
    // deflation (sequential, O(n)): negligible z_k, then (nearly) equal poles merged by Givens rotations
    double zn = 0.0, dmax = fabs(s_alpha);
    for (int k = 0; k < n; ++k) {
      zn += zs[k] * zs[k];
      dmax = fmax(dmax, fabs(d[k]));
    }
    zn = sqrt(zn);
    const double tol = 8.0 * 2.220446049250313e-16 * fmax(dmax, zn);
    int m = 0, nc = 0, last = -1;
    for (int k = 0; k < n; ++k) {
      if (fabs(zs[k]) <= tol) {
        kind[nc] = -(k + 1);
        eig[nc] = d[k];
        ++nc;
        continue;
      }
      if (last >= 0 && fabs(d[k] - d[last]) <= tol) {
        // v_last' = c v_last + s v_k, v_k' = -s v_last + c v_k with z_k' = 0
        const double r = hypot(zs[last], zs[k]);
        const double c = zs[last] / r, sn = zs[k] / r;
        const double pl = ps[last], pk = ps[k];
        ps[last] = c * pl + sn * pk;
        ps[k] = -sn * pl + c * pk;
        zs[last] = r;
        zs[k] = 0.0;
        partner[k] = last;
        rcos[k] = c;
        rsin[k] = sn;
        kind[nc] = -(k + 1);
        eig[nc] = d[k];
        ++nc;
        continue;
      }
      comp[m++] = k;
      last = k;
    }
    for (int t = 0; t < m; ++t) {
      dk[t] = d[comp[t]];
      zk[t] = zs[comp[t]];
    }
    for (int t = 0; t <= m; ++t) kind[nc + t] = t;
    s_m = m;
    s_ncand = nc + m + 1;
  }
  __syncthreads();
  const int m = s_m, nc0 = s_ncand - (m + 1);
  const double alpha = s_alpha;
  double zn2 = 0.0;
  for (int t = 0; t < m; ++t) zn2 += zk[t] * zk[t];
  const double zn = sqrt(zn2);
  // roots of alpha - mu + sum z_t^2/(mu - d_t): one in each of (-inf,d_0), (d_0,d_1), ..., (d_{m-1},inf)
  for (int r = tid; r <= m; r += blockDim.x) {
    double origin = alpha, lo = 0.0, hi = 0.0;
    int oi = -1;
    if (m > 0) {
      if (r == 0) {
        oi = 0; origin = dk[0];
        lo = fmin(dk[0], alpha) - zn - 1.0 - origin; hi = 0.0;
      } else if (r == m) {
        oi = m - 1; origin = dk[m - 1];
        lo = 0.0; hi = fmax(dk[m - 1], alpha) + zn + 1.0 - origin;
      } else {
        const double mid = 0.5 * (dk[r - 1] + dk[r]);
        if (secular_f(m, dk, zk, alpha, dk[r - 1], mid - dk[r - 1]) > 0) {
          oi = r; origin = dk[r]; lo = mid - dk[r]; hi = 0.0;   // root in (mid, d_r)
        } else {
          oi = r - 1; origin = dk[r - 1]; lo = 0.0; hi = mid - dk[r - 1];
        }
      }
    }
    double delta = 0.5 * (lo + hi);
    if (m > 0)
      for (int it = 0; it < 2100; ++it) {  // bisection to adjacent doubles (bounded)
        delta = 0.5 * (lo + hi);
        if (delta == lo || delta == hi) break;
        if (secular_f(m, dk, zk, alpha, origin, delta) > 0) lo = delta; else hi = delta;
      }
    origin_idx[r] = oi;
    yv[r] = delta;
    double yy = 1.0, yp = s_un;  // y_last = 1, p_last = ||u||
    for (int t = 0; t < m; ++t) {
      const double y = zk[t] / ((origin - dk[t]) + delta);
      yy += y * y;
      yp += y * ps[comp[t]];
    }
    score[nc0 + r] = fabs(yp) / sqrt(yy);
    eig[nc0 + r] = origin + delta;
  }
  for (int t = tid; t < nc0; t += blockDim.x) score[t] = fabs(ps[-kind[t] - 1]);
  __syncthreads();
  if (tid == 0) {  // largest score; ties within tie_rtol go to the lower eigenvalue
    double best = -1.0;
    for (int t = 0; t < s_ncand; ++t) best = fmax(best, score[t]);
    int sel = -1;
    for (int t = 0; t < s_ncand; ++t)
      if (score[t] >= best * (1.0 - tie_rtol) && (sel < 0 || eig[t] < eig[sel])) sel = t;
    s_sel = sel;
    lambda[i] = eig[sel];
    status[i] = MK_OK;
  }
  __syncthreads();
  const int sel = s_sel;
  // selected eigenvector in the rotated V basis (ytmp) and its last component
  for (int t = tid; t < n; t += blockDim.x) ytmp[t] = 0.0;
  __syncthreads();
  if (kind[sel] < 0) {
    if (tid == 0) {
      ytmp[-kind[sel] - 1] = 1.0;
      s_ylast = 0.0;
    }
  } else {
    const int r = kind[sel];
    const int oi = origin_idx[r];
    const double origin = oi >= 0 ? dk[oi] : alpha;
    const double delta = yv[r];
    for (int t = tid; t < m; t += blockDim.x) ytmp[comp[t]] = zk[t] / ((origin - dk[t]) + delta);
    if (tid == 0) s_ylast = 1.0;
  }
  __syncthreads();
  if (tid == 0) {
    double nn = s_ylast * s_ylast, sp = s_ylast * s_un;
    for (int t = 0; t < n; ++t) {
      nn += ytmp[t] * ytmp[t];
      sp += ytmp[t] * ps[t];
    }
    s_norm = sqrt(nn);
    s_sign = sp < 0 ? -1.0 : 1.0;
    // back to the original V basis: undo the rotations in reverse order of creation
    for (int k = n - 1; k >= 0; --k) {
      const int l = partner[k];
      if (l < 0) continue;
      const double a = ytmp[l], b = ytmp[k];
      ytmp[l] = a * rcos[k] - b * rsin[k];
      ytmp[k] = a * rsin[k] + b * rcos[k];
    }
  }
  __syncthreads();
  const double scale = s_sign / s_norm;
  const double yl = scale * s_ylast;
  // coarse part: phi_H = V (y - (y_last/||u||) p), theta_2 = y_last/||u||
  for (int k = tid; k < n; k += blockDim.x) yv[k] = scale * ytmp[k] - (yl / s_un) * G[(int64_t)k * 2 * N + N + i];
  __syncthreads();
  for (int r = tid; r < n; r += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += V[(int64_t)r * n + k] * yv[k];
    coef[(int64_t)r * N + i] = s;
  }
  if (tid == 0) coef[(int64_t)n * N + i] = yl / s_un;
}

// ------------------------------------------------------------------------------------------------ A8
__global__ void k_orbitals(int64_t n_nodes, const int32_t* __restrict__ off, const int32_t* __restrict__ col,
                           const double* __restrict__ val, const uint8_t* __restrict__ bnd,
                           const double* __restrict__ coef, int NH, const double* __restrict__ psihat, int N, int ld,
                           double* __restrict__ psi) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_nodes * ld) return;
  const int64_t nd = t / ld;
  const int j = (int)(t % ld);
  double s = 0.0;
  if (j < N && !bnd[nd]) {
    for (int k = off[nd]; k < off[nd + 1]; ++k) s += val[k] * coef[(int64_t)col[k] * N + j];
    s += coef[(int64_t)NH * N + j] * psihat[t];
  }
  psi[t] = s;
}

__global__ void k_flip(int64_t n_nodes, const double* __restrict__ dots, double* __restrict__ psi, int N, int ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_nodes * ld) return;
  const int j = (int)(t % ld);
  if (j < N && dots[j] < 0) psi[t] = -psi[t];
}



// Inverse Cholesky factor of the SPD n x n matrix MH: Linv = L^-1 (MH = L L^T), dense row-major.  Uses the
// workspace slot `slot` for L^T.  Returns MK_ERR_INVALID_ARG if MH is not positive definite.
int inverse_cholesky(mk_ctx* ctx, int n, const double* MH, double* Linv, int slot, cudaStream_t s) {
  int err = MK_OK;
  char* ws = (char*)scratch(ctx, slot, (size_t)n * n * 16 + 256, &err);
  if (!ws) return err;
  double* LT = (double*)ws;
  double* I = LT + (size_t)n * n;
  int* dflag = (int*)(I + (size_t)n * n);
  MK_CUDA(cudaMemsetAsync(dflag, 0, sizeof(int), s));
  MK_COUNT(), k_cholesky<<<1, 1024, 0, s>>>(n, MH, LT, dflag);
  MK_COUNT(), k_identity<<<(int)(((int64_t)n * n + 255) / 256), 256, 0, s>>>(n, I);
  MK_COUNT(), k_forward<<<(n + 127) / 128, 128, 0, s>>>(n, LT, I, Linv);
  int h = 0;
  MK_CUDA(cudaMemcpyAsync(&h, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
  MK_CUDA(cudaStreamSynchronize(s));
  if (h) return fail(MK_ERR_INVALID_ARG, "M_H is not positive definite");
  return MK_OK;
}

// Shared decomposition of the coarse pencil: C = Linv AH Linv^T, Jacobi C = Q diag Q^T, d ascending,
// V = Linv^T Q (columns sorted with d).  V row-major [n x n], V[i][k] = component i of eigenvector k.
int decompose(mk_ctx* ctx, int n, const double* Linv, const double* AH, double* d, double* V, cudaStream_t s) {
  const int n2 = (n + 1) / 2 * 2;
  int err = MK_OK;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  const size_t oT = take((size_t)n * n * 8), oC = take((size_t)n * n * 8), oS0 = take((size_t)n2 * n2 * 8);
  const size_t oS1 = take((size_t)n2 * n2 * 8), oQ = take((size_t)n2 * n2 * 8), oRed = take(8192 * 8);
  const size_t oPerm = take((size_t)n * 4), oInfo = take(64);
  char* ws = (char*)scratch(ctx, S_EIG2, off, &err);
  if (!ws) return err;
  double *T = (double*)(ws + oT), *C = (double*)(ws + oC), *S0 = (double*)(ws + oS0), *S1 = (double*)(ws + oS1);
  double *Q = (double*)(ws + oQ), *red = (double*)(ws + oRed);
  int *perm = (int*)(ws + oPerm), *info = (int*)(ws + oInfo);
  gemm64(n, n, n, Linv, n, 0, AH, n, 0, T, n, s);                   // T = Linv AH
  gemm64(n, n, n, T, n, 0, Linv, n, 1, C, n, s);                    // C = T Linv^T
  MK_COUNT(), k_pad_sym<<<(int)(((int64_t)n2 * n2 + 255) / 256), 256, 0, s>>>(n, n2, C, S0, Q, 0.0);
  const int np = n2 / 2;
  const size_t smem = (size_t)np * sizeof(Rot);
  if (smem > 48 * 1024) MK_CUDA(cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  MK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi, 256, smem));
  MK_ARG(per_sm >= 1, "mk: Jacobi kernel cannot be resident (coarse space too large)");
  int grid = std::min(ctx->n_sms, 4096);
  int max_sweeps = 60;
  double tol = 1e-15;
  int n2v = n2;
  void* args[] = {&n2v, &S0, &S1, &Q, &red, &max_sweeps, &tol, &info};
  MK_COUNT();
  MK_CUDA(cudaLaunchCooperativeKernel((void*)k_jacobi, grid, 256, args, smem, s));
  int hinfo[2];
  MK_CUDA(cudaMemcpyAsync(hinfo, info, sizeof(hinfo), cudaMemcpyDeviceToHost, s));
  MK_CUDA(cudaStreamSynchronize(s));
  const double* Sf = hinfo[1] ? S1 : S0;
  MK_COUNT(), k_rank<<<(n + 127) / 128, 128, 0, s>>>(n, n2, Sf, d, perm);
  MK_COUNT(), k_gather_cols<<<(int)(((int64_t)n * n + 255) / 256), 256, 0, s>>>(n, n2, Q, perm, C);  // C = Q sorted
  gemm64(n, n, n, Linv, n, 1, C, n, 0, V, n, s);                     // V = Linv^T Q
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

int secular(mk_ctx* ctx, int n, int N, const double* d, const double* V, const double* b, const double* c,
            const double* beta, const double* gamma, double* lambda, double* coef, int32_t* status, cudaStream_t s) {
  int err = MK_OK;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  const size_t oG = take((size_t)n * 2 * N * 8), oW = take((size_t)N * kWorkVecs * (n + 1) * 8);
  const size_t oIW = take((size_t)N * 4 * (n + 1) * 4);
  char* ws = (char*)scratch(ctx, S_EIG, off, &err);
  if (!ws) return err;
  double *G = (double*)(ws + oG), *W = (double*)(ws + oW);
  int* IW = (int*)(ws + oIW);
  MK_COUNT(), k_vt_bc<<<(int)(((int64_t)n * 2 * N + 127) / 128), 128, 0, s>>>(n, N, V, b, c, G);
  MK_COUNT(), k_secular_select<<<N, kEigThreads, 0, s>>>(n, N, d, V, G, beta, gamma, W, IW, lambda, coef, status,
                                                        1e-7, 1e-12);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

// At mesh upload: M_H = P^T M P and its inverse Cholesky factor, kept in the mesh handle.
int coarse_matrices(mk_ctx*, const mk_mesh*, const double*, const double*, double*, double*, int, cudaStream_t);

int mesh_mass_factor(mk_ctx* ctx, mk_mesh* m) {
  const Level& F = m->fine;
  const int n = (int)m->coarse.n_free;
  int err = MK_OK;
  const size_t eb = (size_t)F.n_elems * (F.nloc * (F.nloc + 1) / 2) * sizeof(double);
  double* Me = (double*)scratch(ctx, S_ELEM64D, eb, &err);
  double* MH = (double*)scratch(ctx, S_VEC5, (size_t)n * n * sizeof(double) * 2, &err);
  if (!Me || !MH) return err;
  cudaStream_t s = 0;
  MK_TRY(element_matrices(ctx, F, nullptr, 0.0, 0.0, 1.0, nullptr, Me, s, S_NUC2));
  MK_TRY(coarse_matrices(ctx, m, Me, Me, MH, MH + (size_t)n * n, S_COARSE2, s));
  if (cudaMalloc(&m->d_MH_Linv, (size_t)n * n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(MK_ERR_OOM, "mesh upload: M_H factor allocation failed");
  }
  MK_TRY(inverse_cholesky(ctx, n, MH, m->d_MH_Linv, S_EIG2, s));
  MK_CUDA(cudaStreamSynchronize(s));
  return MK_OK;
}

}  // namespace mk

using namespace mk;

extern "C" {

int mk_coarse_decompose(mk_ctx* ctx, const mk_mesh* m, const double* AH, double* d, double* V, void* stream) {
  MK_ARG(ctx && m && AH && d && V && m->d_MH_Linv, "mk_coarse_decompose: null argument");
  MK_CUDA(cudaSetDevice(ctx->device));
  return decompose(ctx, (int)m->coarse.n_free, m->d_MH_Linv, AH, d, V, (cudaStream_t)stream);
}

int mk_small_eigensolve_shared(mk_ctx* ctx, int NH, int N, const double* d, const double* V, const double* b,
                               const double* c, const double* beta, const double* gamma, double* lambda,
                               double* coef, int32_t* status, void* stream) {
  MK_ARG(ctx && d && V && b && c && beta && gamma && lambda && coef && status,
         "mk_small_eigensolve_shared: null argument");
  MK_ARG(NH >= 1 && N >= 1 && N <= MK_MAX_RHS, "mk_small_eigensolve_shared: bad sizes");
  MK_CUDA(cudaSetDevice(ctx->device));
  return secular(ctx, NH, N, d, V, b, c, beta, gamma, lambda, coef, status, (cudaStream_t)stream);
}

int mk_small_eigensolve(mk_ctx* ctx, int NH, int N, const double* AH, const double* MH, const double* b,
                        const double* c, const double* beta, const double* gamma, double* lambda, double* coef,
                        int32_t* status, void* stream) {
  MK_ARG(ctx && AH && MH && b && c && beta && gamma && lambda && coef && status, "mk_small_eigensolve: null argument");
  MK_ARG(NH >= 1 && N >= 1 && N <= MK_MAX_RHS, "mk_small_eigensolve: bad sizes");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  int err = MK_OK;
  double* buf = (double*)scratch(ctx, S_EIG3, (size_t)NH * NH * 2 * sizeof(double) + (size_t)NH * sizeof(double) + 256,
                                 &err);
  if (!buf) return err;
  double* Linv = buf;
  double* V = buf + (size_t)NH * NH;
  double* d = V + (size_t)NH * NH;
  MK_TRY(inverse_cholesky(ctx, NH, MH, Linv, S_EIG4, s));
  MK_TRY(decompose(ctx, NH, Linv, AH, d, V, s));
  return secular(ctx, NH, N, d, V, b, c, beta, gamma, lambda, coef, status, s);
}

int mk_orbital_assemble(mk_ctx* ctx, const mk_mesh* m, const double* coef, const double* psihat, const double* u,
                        int ld, int N, double* psi, void* stream) {
  MK_ARG(ctx && m && coef && psihat && u && psi, "mk_orbital_assemble: null argument");
  MK_ARG(N >= 1 && N <= ld && N <= MK_MAX_RHS, "mk_orbital_assemble: bad N/ld");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const Level& F = m->fine;
  int err = MK_OK;
  const size_t eb = (size_t)F.n_elems * (F.nloc * (F.nloc + 1) / 2) * sizeof(double);
  double* Me = (double*)scratch(ctx, S_ELEM64B, eb, &err);
  double* Mu = (double*)scratch(ctx, S_VEC1, (size_t)F.n_nodes * ld * sizeof(double), &err);
  double* dots = (double*)scratch(ctx, S_COEF, 64 * sizeof(double), &err);
  if (!Me || !Mu || !dots) return err;
  const int64_t work = F.n_nodes * ld;
  MK_COUNT(), k_orbitals<<<(int)((work + 255) / 256), 256, 0, s>>>(F.n_nodes, m->d_P_off, m->d_P_col, m->d_P_val, F.d_boundary,
                                                       coef, (int)m->coarse.n_free, psihat, N, ld, psi);
  MK_TRY(element_matrices(ctx, F, nullptr, 0.0, 0.0, 1.0, nullptr, Me, s));
  MK_TRY(apply64(ctx, F, Me, u, Mu, N, ld, true, s));
  MK_TRY(column_dots(ctx, F.n_nodes, psi, Mu, N, ld, dots, s));
  MK_COUNT(), k_flip<<<(int)((work + 255) / 256), 256, 0, s>>>(F.n_nodes, dots, psi, N, ld);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------ no allocation
// Per-orbital small eigensolve for callers that must not allocate device memory: programs whose device memory is
// reserved up front by another allocator (a cudaMalloc would fail or break that budget) and latency-sensitive
// loops that cannot afford cudaMalloc/cudaFree, which may synchronise the whole device.  Its workspace is the
// fixed array below, sized for N_H <= kStaticMaxNH and N <= kStaticMaxN (about 0.9 MB, held by every GPU that
// loads the library until the process exits).
namespace mk {
constexpr int kStaticMaxNH = 512;
constexpr int kStaticMaxN = 16;
constexpr size_t kStaticG = (size_t)kStaticMaxNH * 2 * kStaticMaxN;                   // doubles: V^T [b | c]
constexpr size_t kStaticW = (size_t)kStaticMaxN * kWorkVecs * (kStaticMaxNH + 1);     // doubles: per-orbital work
constexpr size_t kStaticIW = (size_t)kStaticMaxN * 4 * (kStaticMaxNH + 1);            // ints: per-orbital work
static __device__ __align__(256) double g_static_ws[kStaticG + kStaticW + (kStaticIW + 1) / 2];

static std::mutex g_static_mu;
static double* g_static_ptr[64] = {nullptr};

// Device address of g_static_ws on the current device, looked up once per device (host code cannot use the
// array's name as a device address).
static int static_workspace(double** out) {
  int dev = 0;
  MK_CUDA(cudaGetDevice(&dev));
  MK_ARG(dev >= 0 && dev < 64, "mk_small_eigensolve_static: device id out of range");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    MK_CUDA(cudaGetSymbolAddress(&p, g_static_ws));
    g_static_ptr[dev] = (double*)p;
  }
  *out = g_static_ptr[dev];
  return MK_OK;
}
}  // namespace mk

extern "C" int mk_small_eigensolve_static(int NH, int N, const double* d, const double* V, const double* b,
                                          const double* c, const double* beta, const double* gamma, double* lambda,
                                          double* coef, int32_t* status, void* stream) {
  MK_ARG(d && V && b && c && beta && gamma && lambda && coef && status, "mk_small_eigensolve_static: null argument");
  MK_ARG(NH >= 1 && N >= 1, "mk_small_eigensolve_static: sizes must be positive");
  MK_ARG(NH <= kStaticMaxNH, "mk_small_eigensolve_static: N_H = " + std::to_string(NH) + " exceeds the fixed maximum " +
                             std::to_string(kStaticMaxNH) + " (use mk_small_eigensolve_shared)");
  MK_ARG(N <= kStaticMaxN, "mk_small_eigensolve_static: N = " + std::to_string(N) + " exceeds the fixed maximum " +
                           std::to_string(kStaticMaxN) + " (use mk_small_eigensolve_shared)");
  double* ws = nullptr;
  MK_TRY(static_workspace(&ws));
  cudaStream_t s = (cudaStream_t)stream;
  double* G = ws;
  double* W = ws + kStaticG;
  int* IW = reinterpret_cast<int*>(ws + kStaticG + kStaticW);
  // Every workspace entry the kernels read is written first in the same call, so nothing needs clearing.
  MK_COUNT(), k_vt_bc<<<(int)(((int64_t)NH * 2 * N + 127) / 128), 128, 0, s>>>(NH, N, V, b, c, G);
  MK_COUNT(), k_secular_select<<<N, kEigThreads, 0, s>>>(NH, N, d, V, G, beta, gamma, W, IW, lambda, coef, status,
                                                        1e-7, 1e-12);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}
