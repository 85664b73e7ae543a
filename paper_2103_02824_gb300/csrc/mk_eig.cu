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
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>
#include <utility>
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

// ------------------------------------------------------------------------------------------------ block Jacobi
// Cyclic block Jacobi on the symmetric n2 x n2 matrix (n2 a multiple of 2 kBW), accumulating Q <- Q U.
// The indices are cut into blocks of kBW; a sweep pairs the blocks round-robin (nb - 1 rounds of nb / 2 disjoint
// block pairs).  In a round, each block pair's 2kBW x 2kBW diagonal sub-block is (nearly) diagonalised by an
// orthogonal U, and S <- U^T S U, Q <- Q U are applied with all the round's U at once in FP64.  The sub-problem runs
// one cyclic Jacobi sweep in FP32 (each angle from the FP64 difference of the two diagonal entries, rounded once, plus
// the FP32 changes of the diagonal since: nearly equal entries still give the right angle), then U is made
// orthogonal to FP64 precision by two Newton-Schulz steps U <- U (3I - U^T U) / 2.  So every applied transform is
// orthogonal in FP64 and the FP64 matrix stays similar to the input; an inexact angle only leaves a small residue
// that later sweeps remove.  GB300 executes FP64 at a small fraction of its FP32 rate, so FP64 is kept to the
// Newton-Schulz steps and the block application.
// Overlap: in round r, CTAs [0, nb/2) compute the U of round r + 1 — the sub-block they need, of S after round r,
// formed directly from S before round r and the round's U — while the other CTAs apply round r.  One grid barrier
// per round (kBW times fewer than the scalar cyclic Jacobi, whose barriers bound it on this GPU).
// *info = {sweeps, buffer holding the result}.
constexpr int kBW = 8;
constexpr int kBP = 2 * kBW;
constexpr int kBJThreads = 256;  // one thread per entry of a kBP x kBP block

__device__ __forceinline__ int bj_index(int I, int J, int k) { return k < kBW ? I * kBW + k : J * kBW + (k - kBW); }

struct BJSmem {
  double sa[kBP * kBP], sb[kBP * kBP], sc[kBP * kBP], sd[kBP * kBP];
  float fa[2][kBP * kBP], fu[2][kBP * kBP];
  double dg[kBP];
  float dd[kBP * kBP], dl[kBP];  // FP32 initial diagonal differences, changes of the diagonal since
  float rcs[kBP][2];             // per index: its coefficients (self, partner) in the current inner round
  int prt[kBP];                  // per index: its partner in the current inner round
  double sh[kBJThreads];
  double bb[3 * kBW * kBW];      // the three kBW x kBW blocks of the next round's sub-block
};

// The orthogonal U that nearly diagonalises the symmetric kBP x kBP block whose entry (ti, tj) = (tid / kBP,
// tid % kBP) this thread passes in v; written to Uout [kBP * kBP].  Called by all threads of the CTA.
__device__ void bj_pair_solve(BJSmem& S, double v, double* __restrict__ Uout) {
  const int tid = threadIdx.x, ti = tid / kBP, tj = tid % kBP;
  if (ti == tj) S.dg[ti] = v;
  S.fa[0][tid] = ti == tj ? 0.0f : (float)v;
  S.fu[0][tid] = ti == tj ? 1.0f : 0.0f;
  if (tid < kBP) S.dl[tid] = 0.0f;
  __syncthreads();
  S.dd[tid] = (float)(S.dg[tj] - S.dg[ti]);  // the FP64 difference of two diagonal entries, rounded once
  __syncthreads();
  int cur = 0;
  for (int k = 0; k < kBP - 1; ++k) {  // one inner sweep
    if (tid < kBP / 2) {                // rotation tid of inner round k, all in FP32
      int p, q;
      pair_of(k, tid, kBP, &p, &q);
      const float apq = S.fa[cur][p * kBP + q];
      float cc = 1.0f, ss = 0.0f;
      if (apq != 0.0f) {
        // a_qq - a_pp = (initial difference) + (the changes since), each part accurate in FP32
        const float theta = (S.dd[p * kBP + q] + (S.dl[q] - S.dl[p])) / (2.0f * apq);
        float t;
        if (!(fabsf(theta) <= 1e18f)) t = isfinite(theta) ? 0.5f / theta : 0.0f;
        else t = copysignf(1.0f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.0f));
        cc = rsqrtf(1.0f + t * t);
        ss = t * cc;
        S.dl[p] -= t * apq;
        S.dl[q] += t * apq;
      }
      // index p: row' = c row_p - s row_q; index q: row' = s row_p + c row_q (columns alike)
      S.rcs[p][0] = cc; S.rcs[p][1] = -ss; S.prt[p] = q;
      S.rcs[q][0] = cc; S.rcs[q][1] = ss; S.prt[q] = p;
    }
    __syncthreads();
    {  // A <- J^T A J and U <- U J with J = [[c, s], [-s, c]] in every (p, q) plane of the round
      const int yi = S.prt[ti], yj = S.prt[tj];
      const float ri = S.rcs[ti][0], ro = S.rcs[ti][1], cs_ = S.rcs[tj][0], co = S.rcs[tj][1];
      const float* A = S.fa[cur];
      float nv = 0.0f;  // the diagonal is tracked in dl; a pair's own entry is annihilated
      if (ti != tj && yi != tj) {
        const float row0 = ri * A[ti * kBP + tj] + ro * A[yi * kBP + tj];  // (J^T A)[ti][tj]
        const float row1 = ri * A[ti * kBP + yj] + ro * A[yi * kBP + yj];  // (J^T A)[ti][yj]
        nv = cs_ * row0 + co * row1;
      }
      S.fa[cur ^ 1][tid] = nv;
      const float* U = S.fu[cur];
      S.fu[cur ^ 1][tid] = cs_ * U[ti * kBP + tj] + co * U[ti * kBP + yj];
    }
    __syncthreads();
    cur ^= 1;
  }
  // U in FP64, two Newton-Schulz steps U <- U + U E / 2 with E = I - U^T U: E (symmetric) in FP64, the small
  // correction U E in FP32.  The FP32 U is orthogonal to ~1e-6; the steps take that to ~1e-12, then to FP64 rounding.
  S.sa[tid] = (double)S.fu[cur][tid];
  __syncthreads();
  for (int step = 0; step < 2; ++step) {
    if (ti <= tj) {
      double g = 0.0;
      for (int m = 0; m < kBP; ++m) g += S.sa[m * kBP + ti] * S.sa[m * kBP + tj];
      const float e = (float)((ti == tj ? 1.0 : 0.0) - g);
      S.fa[cur ^ 1][ti * kBP + tj] = e;
      S.fa[cur ^ 1][tj * kBP + ti] = e;
    }
    S.fu[cur][tid] = (float)S.sa[tid];
    __syncthreads();
    float corr = 0.0f;
    for (int m = 0; m < kBP; ++m) corr = fmaf(S.fu[cur][ti * kBP + m], S.fa[cur ^ 1][m * kBP + tj], corr);
    const double un = S.sa[tid] + 0.5 * (double)corr;
    __syncthreads();
    S.sa[tid] = un;
    __syncthreads();
  }
  Uout[tid] = S.sa[tid];
  __syncthreads();
}

// The round-r pair holding block K, and whether K is its second block.  Round r pairs block nb - 1 with r (pair 0)
// and every other block K with (2r - K) mod (nb - 1), in pair m = min((K - r) mod (nb - 1), (r - K) mod (nb - 1)).
__device__ __forceinline__ void bj_pair_of_block(int r, int K, int nb, int* pair, int* half) {
  int m = 0;
  if (K != nb - 1 && K != r) {
    const int d1 = ((K - r) % (nb - 1) + (nb - 1)) % (nb - 1);
    m = min(d1, (nb - 1) - d1);
  }
  int a, b;
  pair_of(r, m, nb, &a, &b);
  *pair = m;
  *half = (b == K) ? 1 : 0;
}

// This thread's entry (tid / kBP, tid % kBP) of the sub-block [I', J'] x [I', J'] of S after round r, i.e. of
// Ubar^T Sin Ubar with Ubar the round's block-diagonal transform (U of pair m at Ur + m kBP^2): for blocks K, L
// in round-r pairs x, y, S'[K, L] = U_x[:, half K]^T Sin[x, y] U_y[:, half L] (8 x 16 x 16 x 8 products).
__device__ double bj_next_block(BJSmem& S, const double* __restrict__ Sin, const double* __restrict__ Ur, int n2,
                                int nb, int r, int Ip, int Jp) {
  const int tid = threadIdx.x, ti = tid / kBP, tj = tid % kBP;
  int x, hx, y, hy;
  bj_pair_of_block(r, Ip, nb, &x, &hx);
  bj_pair_of_block(r, Jp, nb, &y, &hy);
  int Ix, Jx, Iy, Jy;
  pair_of(r, x, nb, &Ix, &Jx);
  pair_of(r, y, nb, &Iy, &Jy);
  // the three 16 x 16 blocks of Sin: [x, x], [x, y], [y, y]
  const double t1 = Sin[(int64_t)bj_index(Ix, Jx, ti) * n2 + bj_index(Ix, Jx, tj)];
  const double t2 = Sin[(int64_t)bj_index(Ix, Jx, ti) * n2 + bj_index(Iy, Jy, tj)];
  const double t3 = Sin[(int64_t)bj_index(Iy, Jy, ti) * n2 + bj_index(Iy, Jy, tj)];
  S.sb[tid] = Ur[(int64_t)x * kBP * kBP + tid];
  S.sc[tid] = Ur[(int64_t)y * kBP * kBP + tid];
  for (int part = 0; part < 3; ++part) {  // S'[I', I'], S'[I', J'], S'[J', J'] into bb
    S.sa[tid] = part == 0 ? t1 : part == 1 ? t2 : t3;
    const double* Ul = part == 2 ? S.sc : S.sb;   // left factor: U_x for [x, x] and [x, y], U_y for [y, y]
    const double* Urt = part == 0 ? S.sb : S.sc;  // right factor
    const int hl = part == 2 ? hy : hx, hr = part == 0 ? hx : hy;
    __syncthreads();
    if (tid < kBP * kBW) {  // W = T U_right[:, half] (16 x 8)
      const int i = tid / kBW, j = tid % kBW;
      double w = 0.0;
      for (int m = 0; m < kBP; ++m) w += S.sa[i * kBP + m] * Urt[m * kBP + hr * kBW + j];
      S.sd[tid] = w;
    }
    __syncthreads();
    if (tid < kBW * kBW) {  // B = U_left[:, half]^T W (8 x 8)
      const int i = tid / kBW, j = tid % kBW;
      double o = 0.0;
      for (int m = 0; m < kBP; ++m) o += Ul[m * kBP + hl * kBW + i] * S.sd[m * kBW + j];
      S.bb[part * kBW * kBW + tid] = o;
    }
    __syncthreads();
  }
  double v;
  if (ti < kBW && tj < kBW) v = S.bb[ti * kBW + tj];
  else if (ti < kBW) v = S.bb[kBW * kBW + ti * kBW + (tj - kBW)];
  else if (tj < kBW) v = S.bb[kBW * kBW + tj * kBW + (ti - kBW)];
  else v = S.bb[2 * kBW * kBW + (ti - kBW) * kBW + (tj - kBW)];
  __syncthreads();
  return v;
}

__global__ void __launch_bounds__(kBJThreads, 2) k_bjacobi(int n2, double* __restrict__ S0, double* __restrict__ S1,
                                                       double* __restrict__ Q, double* __restrict__ Ug,
                                                       double* __restrict__ red, int max_sweeps, double tol,
                                                       int* __restrict__ info) {
  cg::grid_group grid = cg::this_grid();
  __shared__ BJSmem S;
  const int tid = threadIdx.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + tid;
  const int64_t gnth = (int64_t)gridDim.x * blockDim.x;
  const int nb = n2 / kBW, npr = nb / 2;
  const int ti = tid / kBP, tj = tid % kBP;  // this thread's entry of a block
  const bool solver = (int)blockIdx.x < npr;  // computes the next round's U; the others apply the current round
  const int na = (int)gridDim.x - npr;       // applying CTAs
  double* Sin = S0;
  double* Sout = S1;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int64_t t = gtid; t < (int64_t)n2 * n2; t += gnth) {
      const double v = Sin[t];
      tot += v * v;
      if (t / n2 != t % n2) off += v * v;
    }
    for (int pass = 0; pass < 2; ++pass) {
      S.sh[tid] = pass == 0 ? off : tot;
      __syncthreads();
      for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (tid < st) S.sh[tid] += S.sh[tid + st];
        __syncthreads();
      }
      if (tid == 0) red[2 * blockIdx.x + pass] = S.sh[0];
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
    if (solver) {  // the U of round 0, from Sin itself
      int I, J;
      pair_of(0, blockIdx.x, nb, &I, &J);
      bj_pair_solve(S, Sin[(int64_t)bj_index(I, J, ti) * n2 + bj_index(I, J, tj)],
                    Ug + (int64_t)blockIdx.x * kBP * kBP);
    }
    grid.sync();
    for (int r = 0; r < nb - 1; ++r) {
      const double* Ur = Ug + (int64_t)(r & 1) * npr * kBP * kBP;
      if (solver) {
        if (r + 1 < nb - 1) {
          int Ip, Jp;
          pair_of(r + 1, blockIdx.x, nb, &Ip, &Jp);
          const double v = bj_next_block(S, Sin, Ur, n2, nb, r, Ip, Jp);
          bj_pair_solve(S, v, Ug + ((int64_t)((r + 1) & 1) * npr + blockIdx.x) * kBP * kBP);
        }
      } else {
        // S_out = U^T S_in U block by block (pairs a >= b, the transpose written too) and Q <- Q U in place; the
        // operands of a CTA's next item are loaded into registers while the current one is computed
        const int nS = npr * (npr + 1) / 2, nQ = (n2 / kBP) * npr;
        struct Item {
          int a, b;          // S item: row pair a, column pair b; Q item: a = -1 - row tile, b = column pair
          int64_t at, at2;   // this thread's entry (and its transposed place for S items)
          double x, ua, ub;  // S or Q entry, U_a entry, U_b entry
        };
        auto load_item = [&](int item, Item& it) {
          if (item < nS) {
            int a = (int)((sqrtf(8.0f * (float)item + 1.0f) - 1.0f) * 0.5f);  // item = a (a + 1) / 2 + b, b <= a
            while ((a + 1) * (a + 2) / 2 <= item) ++a;
            while (a * (a + 1) / 2 > item) --a;
            const int b = item - a * (a + 1) / 2;
            int Ia, Ja, Ib, Jb;
            pair_of(r, a, nb, &Ia, &Ja);
            pair_of(r, b, nb, &Ib, &Jb);
            const int row = bj_index(Ia, Ja, ti), col = bj_index(Ib, Jb, tj);
            it.a = a; it.b = b;
            it.at = (int64_t)row * n2 + col;
            it.at2 = (int64_t)col * n2 + row;
            it.x = Sin[it.at];
            it.ua = Ur[(int64_t)a * kBP * kBP + tid];
            it.ub = Ur[(int64_t)b * kBP * kBP + tid];
          } else {
            const int u = item - nS, rt = u / npr, b = u % npr;
            int Ib, Jb;
            pair_of(r, b, nb, &Ib, &Jb);
            it.a = -1 - rt; it.b = b;
            it.at = (int64_t)(rt * kBP + ti) * n2 + bj_index(Ib, Jb, tj);
            it.x = Q[it.at];
            it.ub = Ur[(int64_t)b * kBP * kBP + tid];
          }
        };
        const int first = (int)blockIdx.x - npr;
        Item cur{}, nxt{};
        if (first < nS + nQ) load_item(first, cur);
        for (int item = first; item < nS + nQ; item += na) {
          S.sa[tid] = cur.x;
          if (cur.a >= 0) S.sb[tid] = cur.ua;
          S.sc[tid] = cur.ub;
          __syncthreads();
          if (item + na < nS + nQ) load_item(item + na, nxt);
          if (cur.a >= 0) {
            double t = 0.0;  // (S U_b)[ti][tj]
            for (int m = 0; m < kBP; ++m) t += S.sa[ti * kBP + m] * S.sc[m * kBP + tj];
            S.sd[tid] = t;
            __syncthreads();
            double ov = 0.0;  // (U_a^T S U_b)[ti][tj]
            for (int m = 0; m < kBP; ++m) ov += S.sb[m * kBP + ti] * S.sd[m * kBP + tj];
            if (cur.a == cur.b) {  // the diagonal block stays exactly symmetric
              S.sa[tid] = ov;
              __syncthreads();
              ov = ti <= tj ? S.sa[tid] : S.sa[tj * kBP + ti];
            }
            Sout[cur.at] = ov;
            if (cur.a != cur.b) Sout[cur.at2] = ov;
          } else {
            double ov = 0.0;
            for (int m = 0; m < kBP; ++m) ov += S.sa[ti * kBP + m] * S.sc[m * kBP + tj];
            Q[cur.at] = ov;
          }
          __syncthreads();
          cur = nxt;
        }
      }
      grid.sync();
      double* tmp = Sin;
      Sin = Sout;
      Sout = tmp;
    }
  }
  if (gtid == 0) {
    info[0] = sweep;
    info[1] = (Sin == S0) ? 0 : 1;
  }
}

// ------------------------------------------------------------------------------------ block Jacobi, FP32 phase
// The same cyclic block Jacobi (rounds of nb / 2 disjoint block pairs, the next round's pair blocks formed by the
// solver CTAs while the others apply the current round, one grid barrier per round), all in FP32: S, Q and every
// transform.  The round's latency is what bounds it, so its two parts run at warp level: each pair solve in one
// warp (the block in registers, no block barrier), each 16 x 16 item of the application in one warp.  It takes the sweeps of the linear phase of the convergence, where most of the work lies, at the
// FP32 rate; it stops once off(S)^2 <= tol^2 |S|^2, or when a sweep no longer halves off(S)^2 (the FP32 floor),
// or after max_sweeps.  Its Q is orthogonal to FP32 precision only: the FP64 finish re-orthonormalises it and
// projects the FP64 matrix onto it before the FP64 sweeps.  *info = {sweeps, buffer holding the result}.
struct BJ32Smem {
  float a[1][kBP * kBP];  // the block a round's pair solve diagonalises
  float sa[kBP * kBP], sb[kBP * kBP], sc[kBP * kBP], sd[kBP * kBP];
  float bb[3 * kBW * kBW];
  double sh[kBJThreads];
  float wa[kBJThreads / 32][kBP * kBP], wb[kBJThreads / 32][kBP * kBP], wt[kBJThreads / 32][kBP * kBP];  // per warp
};

// The entry (tid / kBP, tid % kBP) of the next round's sub-block [I', J'] x [I', J'] of S after round r, from S
// before the round and the round's U (as bj_next_block, in FP32).
__device__ float bj32_next_block(BJ32Smem& S, const float* __restrict__ Sin, const float* __restrict__ Ur, int n2,
                                 int nb, int r, int Ip, int Jp) {
  const int tid = threadIdx.x, ti = tid / kBP, tj = tid % kBP;
  int x, hx, y, hy;
  bj_pair_of_block(r, Ip, nb, &x, &hx);
  bj_pair_of_block(r, Jp, nb, &y, &hy);
  int Ix, Jx, Iy, Jy;
  pair_of(r, x, nb, &Ix, &Jx);
  pair_of(r, y, nb, &Iy, &Jy);
  const float t1 = Sin[(int64_t)bj_index(Ix, Jx, ti) * n2 + bj_index(Ix, Jx, tj)];
  const float t2 = Sin[(int64_t)bj_index(Ix, Jx, ti) * n2 + bj_index(Iy, Jy, tj)];
  const float t3 = Sin[(int64_t)bj_index(Iy, Jy, ti) * n2 + bj_index(Iy, Jy, tj)];
  S.sb[tid] = Ur[(int64_t)x * kBP * kBP + tid];
  S.sc[tid] = Ur[(int64_t)y * kBP * kBP + tid];
  for (int part = 0; part < 3; ++part) {
    S.sa[tid] = part == 0 ? t1 : part == 1 ? t2 : t3;
    const float* Ul = part == 2 ? S.sc : S.sb;
    const float* Urt = part == 0 ? S.sb : S.sc;
    const int hl = part == 2 ? hy : hx, hr = part == 0 ? hx : hy;
    __syncthreads();
    if (tid < kBP * kBW) {
      const int i = tid / kBW, j = tid % kBW;
      float w = 0.0f;
      for (int m = 0; m < kBP; ++m) w = fmaf(S.sa[i * kBP + m], Urt[m * kBP + hr * kBW + j], w);
      S.sd[tid] = w;
    }
    __syncthreads();
    if (tid < kBW * kBW) {
      const int i = tid / kBW, j = tid % kBW;
      float o = 0.0f;
      for (int m = 0; m < kBP; ++m) o = fmaf(Ul[m * kBP + hl * kBW + i], S.sd[m * kBW + j], o);
      S.bb[part * kBW * kBW + tid] = o;
    }
    __syncthreads();
  }
  float v;
  if (ti < kBW && tj < kBW) v = S.bb[ti * kBW + tj];
  else if (ti < kBW) v = S.bb[kBW * kBW + ti * kBW + (tj - kBW)];
  else if (tj < kBW) v = S.bb[kBW * kBW + tj * kBW + (ti - kBW)];
  else v = S.bb[2 * kBW * kBW + (ti - kBW) * kBW + (tj - kBW)];
  __syncthreads();
  return v;
}

// Partner of index x in inner round k of the cyclic ordering of kBP = 16 indices used by pair_of (round k pairs
// 15 with k and every other x with (2k - x) mod 15).
__host__ __device__ constexpr int bj_partner(int k, int x) {
  return x == kBP - 1 ? k : (x == k ? kBP - 1 : ((2 * k - x) % (kBP - 1) + (kBP - 1)) % (kBP - 1));
}

__device__ __forceinline__ float bj_sel8(const float (&v)[8], int r) {
  float o = v[0];
#pragma unroll
  for (int q = 1; q < 8; ++q) o = (r == q) ? v[q] : o;
  return o;
}

// One warp's version of bj32_pair_solve: the same inner sweep, with the block in registers.  Lane l holds row
// i = l / 2, columns 8 (l % 2) .. 8 (l % 2) + 7 of A and of U; the inner rounds are unrolled, so every partner
// column has a fixed register; entries of other rows come by shuffles, with no block barrier.  Each rotation is
// computed from the diagonal entries and from a_pq as row p = min(p, q) holds it, the same values in the lanes of
// both rows.  Ab: the symmetric block [kBP * kBP] (row-major, shared memory); U to Uout.  Called by all 32 lanes.
__device__ void bj32_pair_solve_warp(const float* __restrict__ Ab, float* __restrict__ Uout) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, i = lane >> 1, h = lane & 1;
  float a[8], u[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    a[r] = Ab[i * kBP + 8 * h + r];
    u[r] = (8 * h + r == i) ? 1.0f : 0.0f;
  }
#pragma unroll
  for (int k = 0; k < kBP - 1; ++k) {
    const int y = bj_partner(k, i);
    const int p = min(i, y), q = max(i, y);
    const float dv = bj_sel8(a, i & 7);  // a_ii, in the lane of row i that holds column i
    const float ev = bj_sel8(a, y & 7);  // a_iy, in the lane of row i that holds column y
    const float app = __shfl_sync(FULL, dv, 2 * p + (p >> 3));
    const float aqq = __shfl_sync(FULL, dv, 2 * q + (q >> 3));
    const float apq = __shfl_sync(FULL, ev, 2 * p + (q >> 3));
    // t = sgn(theta) / (|theta| + sqrt(theta^2 + 1)), theta = (a_qq - a_pp) / (2 a_pq); t ~ 1 / (2 theta) where
    // theta^2 would overflow (equal diagonal entries give theta = 0 and t = +-1 however small a_pq is).  The
    // quotients and the root use the fast approximate forms (a few ulp): an angle off by that much only leaves a
    // residue of the same size, which the later sweeps remove, and c, s stay a rotation to FP32 rounding.
    float t = 0.0f;
    if (apq != 0.0f) {
      const float theta = __fdividef(aqq - app, 2.0f * apq);
      if (!(fabsf(theta) <= 1e18f)) t = isfinite(theta) ? __fdividef(0.5f, theta) : 0.0f;
      else {
        const float g = fmaf(theta, theta, 1.0f);
        t = copysignf(__fdividef(1.0f, fabsf(theta) + g * rsqrtf(g)), theta);
      }
    }
    const float c = rsqrtf(fmaf(t, t, 1.0f)), s = t * c;
    const float cs = c, co = (i == p) ? -s : s;  // index p: c row_p - s row_q; index q: s row_p + c row_q
    float cj[8], oj[8], ay[8], rm[8], rmo[8], uc[8], uo[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      cj[r] = __shfl_sync(FULL, cs, 2 * (8 * h + r));
      oj[r] = __shfl_sync(FULL, co, 2 * (8 * h + r));
      ay[r] = __shfl_sync(FULL, a[r], 2 * y + h);
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) rm[r] = cs * a[r] + co * ay[r];  // row i of J^T A
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      rmo[r] = __shfl_xor_sync(FULL, rm[r], 1);
      uc[r] = u[r];  // the row before this round (u is rewritten column by column below)
      uo[r] = __shfl_xor_sync(FULL, u[r], 1);
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int y0 = bj_partner(k, r), y1 = bj_partner(k, 8 + r);  // the partner of column 8h + r, for h = 0, 1
      const float r0 = (y0 < 8) ? rm[y0 & 7] : rmo[y0 & 7];         // row i at column y0 (h = 0: own half first)
      const float r1 = (y1 >= 8) ? rm[y1 & 7] : rmo[y1 & 7];        // row i at column y1 (h = 1)
      const float u0 = (y0 < 8) ? uc[y0 & 7] : uo[y0 & 7];
      const float u1 = (y1 >= 8) ? uc[y1 & 7] : uo[y1 & 7];
      const float rv = h ? r1 : r0, uv = h ? u1 : u0;
      const float na = cj[r] * rm[r] + oj[r] * rv;
      a[r] = (8 * h + r == y) ? 0.0f : na;  // a rotated pair's own entry is annihilated
      u[r] = cj[r] * uc[r] + oj[r] * uv;
    }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) Uout[i * kBP + 8 * h + r] = u[r];
}

__global__ void __launch_bounds__(kBJThreads, 2) k_bjacobi32(int n2, float* __restrict__ S0, float* __restrict__ S1,
                                                           float* __restrict__ Q, float* __restrict__ Ug,
                                                           double* __restrict__ red, int max_sweeps, double tol,
                                                           int* __restrict__ info) {
  cg::grid_group grid = cg::this_grid();
  __shared__ BJ32Smem S;
  const int tid = threadIdx.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + tid;
  const int64_t gnth = (int64_t)gridDim.x * blockDim.x;
  const int nb = n2 / kBW, npr = nb / 2;
  const int ti = tid / kBP, tj = tid % kBP;
  const bool solver = (int)blockIdx.x < npr;
  const int na = (int)gridDim.x - npr;
  float* Sin = S0;
  float* Sout = S1;
  double prev = -1.0;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int64_t t = gtid; t < (int64_t)n2 * n2; t += gnth) {
      const double v = Sin[t];
      tot += v * v;
      if (t / n2 != t % n2) off += v * v;
    }
    for (int pass = 0; pass < 2; ++pass) {
      S.sh[tid] = pass == 0 ? off : tot;
      __syncthreads();
      for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (tid < st) S.sh[tid] += S.sh[tid + st];
        __syncthreads();
      }
      if (tid == 0) red[2 * blockIdx.x + pass] = S.sh[0];
      __syncthreads();
    }
    grid.sync();
    double o = 0.0, f = 0.0;
    for (int bl = 0; bl < (int)gridDim.x; ++bl) {
      o += red[2 * bl];
      f += red[2 * bl + 1];
    }
    grid.sync();
    // converged, or at the FP32 floor (a sweep that does not halve off^2); the same decision in every CTA
    if (o <= tol * tol * f || (prev >= 0.0 && o > 0.5 * prev)) break;
    prev = o;
    if (solver) {
      int I, J;
      pair_of(0, blockIdx.x, nb, &I, &J);
      S.a[0][tid] = Sin[(int64_t)bj_index(I, J, ti) * n2 + bj_index(I, J, tj)];
      __syncthreads();
      if (tid < 32) bj32_pair_solve_warp(S.a[0], Ug + (int64_t)blockIdx.x * kBP * kBP);
    }
    grid.sync();
    for (int r = 0; r < nb - 1; ++r) {
      const float* Ur = Ug + (int64_t)(r & 1) * npr * kBP * kBP;
      if (solver) {
        if (r + 1 < nb - 1) {
          int Ip, Jp;
          pair_of(r + 1, blockIdx.x, nb, &Ip, &Jp);
          const float v = bj32_next_block(S, Sin, Ur, n2, nb, r, Ip, Jp);
          S.a[0][tid] = v;
          __syncthreads();
          if (tid < 32) bj32_pair_solve_warp(S.a[0], Ug + ((int64_t)((r + 1) & 1) * npr + blockIdx.x) * kBP * kBP);
          __syncthreads();  // S.a is rewritten by the next round's block
        }
      } else {
        // S_out = U^T S_in U by block pairs (a >= b, the transpose written too), Q <- Q U in place; one 16 x 16
        // item per warp (lane: row i = lane / 2, columns 8 (lane % 2) ..), every warp of the CTA on its own item
        const int nS = npr * (npr + 1) / 2, nQ = (n2 / kBP) * npr;
        const int wp = tid >> 5, lane = tid & 31, i = lane >> 1, h = lane & 1;
        float* Wa = S.wa[wp];
        float* Wb = S.wb[wp];
        float* Wt = S.wt[wp];
        const int nw = kBJThreads / 32;
        for (int item = ((int)blockIdx.x - npr) * nw + wp; item < nS + nQ; item += na * nw) {
          const bool sitem = item < nS;
          int a = 0, b, row, c0;
          if (sitem) {
            a = (int)((sqrtf(8.0f * (float)item + 1.0f) - 1.0f) * 0.5f);  // item = a (a + 1) / 2 + b, b <= a
            while ((a + 1) * (a + 2) / 2 <= item) ++a;
            while (a * (a + 1) / 2 > item) --a;
            b = item - a * (a + 1) / 2;
            int Ia, Ja, Ib, Jb;
            pair_of(r, a, nb, &Ia, &Ja);
            pair_of(r, b, nb, &Ib, &Jb);
            row = bj_index(Ia, Ja, i);
            c0 = h ? Jb * kBW : Ib * kBW;
          } else {
            const int u = item - nS, rt = u / npr;
            b = u % npr;
            int Ib, Jb;
            pair_of(r, b, nb, &Ib, &Jb);
            row = rt * kBP + i;
            c0 = h ? Jb * kBW : Ib * kBW;
          }
          const float* src = sitem ? Sin : Q;
          float x[8], xo[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            Wb[lane * 8 + q] = Ur[(int64_t)b * kBP * kBP + lane * 8 + q];
            if (sitem) Wa[lane * 8 + q] = Ur[(int64_t)a * kBP * kBP + lane * 8 + q];
            x[q] = src[(int64_t)row * n2 + c0 + q];
          }
#pragma unroll
          for (int q = 0; q < 8; ++q) xo[q] = __shfl_xor_sync(0xffffffffu, x[q], 1);
          __syncwarp();
          float t[8];  // (X U_b)[i][8h + q]
#pragma unroll
          for (int q = 0; q < 8; ++q) t[q] = 0.0f;
#pragma unroll
          for (int m = 0; m < kBP; ++m) {
            const float xm = (m < 8) == (h == 0) ? x[m & 7] : xo[m & 7];  // row i, column m of the item
#pragma unroll
            for (int q = 0; q < 8; ++q) t[q] = fmaf(xm, Wb[m * kBP + 8 * h + q], t[q]);
          }
          if (sitem) {
#pragma unroll
            for (int q = 0; q < 8; ++q) Wt[i * kBP + 8 * h + q] = t[q];
            __syncwarp();
            float o[8];  // (U_a^T X U_b)[i][8h + q]
#pragma unroll
            for (int q = 0; q < 8; ++q) o[q] = 0.0f;
#pragma unroll
            for (int m = 0; m < kBP; ++m) {
              const float um = Wa[m * kBP + i];
#pragma unroll
              for (int q = 0; q < 8; ++q) o[q] = fmaf(um, Wt[m * kBP + 8 * h + q], o[q]);
            }
            if (a == b) {  // the diagonal block stays exactly symmetric
              __syncwarp();
#pragma unroll
              for (int q = 0; q < 8; ++q) Wt[i * kBP + 8 * h + q] = o[q];
              __syncwarp();
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                const int j = 8 * h + q;
                o[q] = i <= j ? Wt[i * kBP + j] : Wt[j * kBP + i];
              }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              Sout[(int64_t)row * n2 + c0 + q] = o[q];
              if (a != b) Sout[(int64_t)(c0 + q) * n2 + row] = o[q];
            }
          } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) Q[(int64_t)row * n2 + c0 + q] = t[q];
          }
          __syncwarp();  // the next item rewrites this warp's staging
        }
      }
      grid.sync();
      float* tmp = Sin;
      Sin = Sout;
      Sout = tmp;
    }
  }
  if (gtid == 0) {
    info[0] = sweep;
    info[1] = (Sin == S0) ? 0 : 1;
  }
}

// FP64 n2 x n2 S -> FP32 copy, Q32 = I.
__global__ void k_bj_to32(int64_t nn, int n2, const double* __restrict__ S, float* __restrict__ S32,
                          float* __restrict__ Q32) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nn) return;
  S32[t] = (float)S[t];
  Q32[t] = (t / n2 == t % n2) ? 1.0f : 0.0f;
}

__global__ void k_f32_to_f64(int64_t nn, const float* __restrict__ a, double* __restrict__ b) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nn) b[t] = (double)a[t];
}

// One Newton-Schulz step X' = X + X E / 2 with E = I - G (G = X^T X, FP64): the correction X E in FP32 (E is
// small, so its FP32 rounding is far below the FP64 rounding of X'), X' in FP64.  n x n row-major, 32 x 32 tiles.
__global__ void k_ns_step(int n, const double* __restrict__ X, const double* __restrict__ G, double* __restrict__ Xo) {
  __shared__ float As[32][33], Bs[32][33];
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int k0 = 0; k0 < n; k0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int i = i0 + r, k = k0 + tx;
      As[r][tx] = (i < n && k < n) ? (float)X[(int64_t)i * n + k] : 0.0f;
      const int kk = k0 + r, j = j0 + tx;
      Bs[r][tx] = (kk < n && j < n) ? (float)((kk == j ? 1.0 : 0.0) - G[(int64_t)kk * n + j]) : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float bv = Bs[k][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(As[ty + 8 * q][k], bv, acc[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + ty + 8 * q, j = j0 + tx;
    if (i < n && j < n) Xo[(int64_t)i * n + j] = X[(int64_t)i * n + j] + 0.5 * (double)acc[q];
  }
}

// S = (T + T^T) / 2 for an n x n matrix T.
__global__ void k_symmetrize(int n, const double* __restrict__ T, double* __restrict__ S) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  S[t] = 0.5 * (T[t] + T[(int64_t)j * n + i]);
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
__global__ void k_rank(int n, int n2, const double* __restrict__ S0, const double* __restrict__ S1,
                       const int* __restrict__ info, double* __restrict__ d, int* __restrict__ perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* __restrict__ S = info[1] ? S1 : S0;  // buffer that holds the Jacobi result
  // strict total order on (key, index) with NaN keyed as +inf: the ranks always form a permutation
  auto key = [](double x) { return isnan(x) ? INFINITY : x; };
  const double v = S[(int64_t)i * n2 + i];
  const double kv = key(v);
  int r = 0;
  for (int k = 0; k < n; ++k) {
    const double kw = key(S[(int64_t)k * n2 + k]);
    if (kw < kv || (kw == kv && k < i)) ++r;
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
  const int c = perm[r];
  Qs[t] = (c >= 0 && c < n) ? Q[(int64_t)i * n2 + c] : NAN;
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

// Per-orbital workspace: kWorkVecs vectors of n+1 doubles, a 16-double header, and 4 int vectors of n+1.
constexpr int kWorkVecs = 10;
__host__ __device__ constexpr int64_t sec_stride(int n) { return (int64_t)kWorkVecs * (n + 1) + 16; }

struct SecWork {
  double *zs, *ps, *dk, *zk, *score, *eig, *yv, *rcos, *rsin, *ytmp, *hdr;
  int *kind, *comp, *partner, *origin_idx;
};

__device__ __forceinline__ SecWork sec_work(double* work, int* iwork, int n, int i) {
  const int64_t n1 = n + 1;
  SecWork w;
  w.zs = work + (int64_t)i * sec_stride(n);  // z in the (rotated) V basis
  w.ps = w.zs + n1;                          // p = V^T c in the (rotated) V basis
  w.dk = w.ps + n1;                          // poles kept in the secular equation
  w.zk = w.dk + n1;                          // their z
  w.score = w.zk + n1;                       // per candidate |(x, psi^)_M|
  w.eig = w.score + n1;                      // per candidate eigenvalue
  w.yv = w.eig + n1;                         // per root: offset delta from its origin pole
  w.rcos = w.yv + n1;                        // deflation rotation of index k with its partner
  w.rsin = w.rcos + n1;
  w.ytmp = w.rsin + n1;                      // selected eigenvector
  w.hdr = w.ytmp + n1;                       // alpha, ||u||, m, n_candidates, singular
  w.kind = iwork + (int64_t)i * 4 * n1;      // candidate t: >= 0 root index, < 0 deflated -(k+1)
  w.comp = w.kind + n1;                      // kept pole -> original index
  w.partner = w.comp + n1;                   // rotation partner of k (-1 none)
  w.origin_idx = w.partner + n1;             // per root: kept pole used as origin
  return w;
}

// Phase 1, one block per orbital: p = V^T c, ||u||, z, alpha, deflation; the singular case is finished here.
__global__ void k_sec_prepare(int n, int N, const double* __restrict__ d, const double* __restrict__ V,
                              const double* __restrict__ G, const double* __restrict__ beta,
                              const double* __restrict__ gamma, double* __restrict__ work, int* __restrict__ iwork,
                              double* __restrict__ lambda, double* __restrict__ coef, int32_t* __restrict__ status,
                              double sing_rtol, double tie_rtol) {
  const int i = blockIdx.x;
  if (i >= N) return;
  SecWork w = sec_work(work, iwork, n, i);
  __shared__ double s_red[kEigThreads];
  __shared__ double s_un;
  __shared__ int s_singular, s_sel;
  const int tid = threadIdx.x;
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
    w.hdr[1] = s_un;
    w.hdr[4] = s_singular;
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
      w.hdr[2] = -1.0;
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
    w.zs[k] = (gk - d[k] * pk) / s_un;
    w.ps[k] = pk;
    w.partner[k] = -1;
    a2 += -2.0 * pk * gk + pk * d[k] * pk;
  }
  s_red[tid] = a2;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (tid < st) s_red[tid] += s_red[tid + st];
    __syncthreads();
  }
  if (tid == 0) {
    const double alpha = (beta[i] + s_red[0]) / (s_un * s_un);
    // deflation (sequential, O(n)): negligible z_k, then (nearly) equal poles merged by Givens rotations
    double zn = 0.0, dmax = fabs(alpha);
    for (int k = 0; k < n; ++k) {
      zn += w.zs[k] * w.zs[k];
      dmax = fmax(dmax, fabs(d[k]));
    }
    zn = sqrt(zn);
    const double tol = 8.0 * 2.220446049250313e-16 * fmax(dmax, zn);
    int m = 0, nc = 0, last = -1;
    for (int k = 0; k < n; ++k) {
      if (fabs(w.zs[k]) <= tol) {
        w.kind[nc] = -(k + 1);
        w.eig[nc] = d[k];
        ++nc;
        continue;
      }
      if (last >= 0 && fabs(d[k] - d[last]) <= tol) {
        // v_last' = c v_last + s v_k, v_k' = -s v_last + c v_k with z_k' = 0
        const double r = hypot(w.zs[last], w.zs[k]);
        const double c = w.zs[last] / r, sn = w.zs[k] / r;
        const double pl = w.ps[last], pk = w.ps[k];
        w.ps[last] = c * pl + sn * pk;
        w.ps[k] = -sn * pl + c * pk;
        w.zs[last] = r;
        w.zs[k] = 0.0;
        w.partner[k] = last;
        w.rcos[k] = c;
        w.rsin[k] = sn;
        w.kind[nc] = -(k + 1);
        w.eig[nc] = d[k];
        ++nc;
        continue;
      }
      w.comp[m++] = k;
      last = k;
    }
    for (int t = 0; t < m; ++t) {
      w.dk[t] = d[w.comp[t]];
      w.zk[t] = w.zs[w.comp[t]];
    }
    for (int t = 0; t <= m; ++t) w.kind[nc + t] = t;
    for (int t = 0; t < nc; ++t) w.score[t] = fabs(w.ps[-w.kind[t] - 1]);
    w.hdr[0] = alpha;
    w.hdr[2] = m;
    w.hdr[3] = nc + m + 1;
  }
}

// Secular sum alpha - (origin + delta) + sum_t z_t^2 / ((origin - d_t) + delta), split over the 32 lanes and
// folded with a fixed tree; every lane returns lane 0's value.
__device__ __forceinline__ double warp_secular(int m, const double* __restrict__ dk, const double* __restrict__ zk,
                                              double alpha, double origin, double delta, int lane) {
  double f = 0.0;
  for (int t = lane; t < m; t += 32) f += zk[t] * zk[t] / ((origin - dk[t]) + delta);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) f += __shfl_down_sync(0xffffffffu, f, off);
  return __shfl_sync(0xffffffffu, f, 0) + (alpha - (origin + delta));
}

// The secular function and its derivative at origin + delta (warp-wide sums, the same values on every lane):
// f = sum_t z_t^2 / (mu - d_t) + alpha - mu,  f' = -sum_t z_t^2 / (mu - d_t)^2 - 1 < 0.
__device__ __forceinline__ void warp_secular_d(int m, const double* __restrict__ dk, const double* __restrict__ zk,
                                               double alpha, double origin, double delta, int lane, double* f,
                                               double* fp) {
  double a = 0.0, b = 0.0;
  for (int t = lane; t < m; t += 32) {
    const double q = zk[t] / ((origin - dk[t]) + delta);
    a += zk[t] * q;
    b += q * q;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, off);
    b += __shfl_down_sync(0xffffffffu, b, off);
  }
  *f = __shfl_sync(0xffffffffu, a, 0) + (alpha - (origin + delta));
  *fp = -__shfl_sync(0xffffffffu, b, 0) - 1.0;
}

// Phase 2, one warp per root: a pole-aware Newton-type iteration on the offset from the nearer pole, kept inside its
// bracket, then the root's score.
__global__ void k_sec_roots(int n, int N, double* __restrict__ work, int* __restrict__ iwork) {
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (gw >= (int64_t)N * (n + 1)) return;
  const int i = (int)(gw / (n + 1)), r = (int)(gw % (n + 1));
  SecWork w = sec_work(work, iwork, n, i);
  if (w.hdr[4] != 0.0) return;
  const int m = (int)w.hdr[2];
  if (r > m) return;
  const int nc0 = (int)w.hdr[3] - (m + 1);
  const double alpha = w.hdr[0], un = w.hdr[1];
  const double* dk = w.dk;
  const double* zk = w.zk;
  double zn2 = 0.0;
  for (int t = lane; t < m; t += 32) zn2 += zk[t] * zk[t];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) zn2 += __shfl_down_sync(0xffffffffu, zn2, off);
  const double zn = sqrt(__shfl_sync(0xffffffffu, zn2, 0));
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
      if (warp_secular(m, dk, zk, alpha, dk[r - 1], mid - dk[r - 1], lane) > 0) {
        oi = r; origin = dk[r]; lo = mid - dk[r]; hi = 0.0;   // root in (mid, d_r)
      } else {
        oi = r - 1; origin = dk[r - 1]; lo = 0.0; hi = mid - dk[r - 1];
      }
    }
  }
  // The bracket [lo, hi] has one end at 0 and never changes sign.  Its midpoint is taken in the ordering of the
  // doubles of that sign (the bit patterns of |delta|), so that halving reaches adjacent doubles in at most 64 steps
  // however close the root lies to its pole.
  auto bitmid = [](double l, double h) {
    const uint64_t a = (uint64_t)__double_as_longlong(fabs(l)), b = (uint64_t)__double_as_longlong(fabs(h));
    const uint64_t mb = a < b ? a + (b - a) / 2 : b + (a - b) / 2;
    const double dm = __longlong_as_double((long long)mb);
    return (l >= 0.0 && h >= 0.0) ? dm : -dm;
  };
  // Each step models f near the root as the pole term at the origin, s / delta with s = z_o^2, exactly, plus the rest
  // linearised at the current point (value and slope matched), and takes the root of that model on the bracket's side
  // (a quadratic); where the model gives no root inside the bracket, the bracket is halved instead.
  double delta = 0.5 * (lo + hi);
  if (m > 0) {
    const double sp = zk[oi] * zk[oi];
    for (int it = 0; it < 200; ++it) {  // bounded
      double f, fp;
      warp_secular_d(m, dk, zk, alpha, origin, delta, lane, &f, &fp);
      if (f > 0) lo = delta; else hi = delta;  // f decreases: the root lies above delta when f > 0
      if (f == 0.0) break;
      const double a = fp + sp / (delta * delta);       // slope of the rest (negative)
      const double b = (f - sp / delta) - a * delta;    // model: a x^2 + b x + sp = 0
      const double disc = b * b - 4.0 * a * sp;
      double nd = lo;                                   // outside the open bracket: halve instead
      if (a < 0.0 && disc >= 0.0) {
        const double q = -0.5 * (b + copysign(sqrt(disc), b));
        const double r1 = q / a, r2 = sp / q;            // the two roots have opposite signs
        nd = ((r1 > 0.0) == (hi > 0.0)) ? r1 : r2;
      }
      if (!(nd > lo && nd < hi)) nd = bitmid(lo, hi);
      if (nd == lo || nd == hi || nd == delta) break;
      delta = nd;
    }
  }
  // score of the eigenvector y_t = z_t/(mu - d_t), y_last = 1, against phi~ = (p, ||u||)
  double yy = 0.0, yp = 0.0;
  for (int t = lane; t < m; t += 32) {
    const double y = zk[t] / ((origin - dk[t]) + delta);
    yy += y * y;
    yp += y * w.ps[w.comp[t]];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    yy += __shfl_down_sync(0xffffffffu, yy, off);
    yp += __shfl_down_sync(0xffffffffu, yp, off);
  }
  if (lane == 0) {
    w.origin_idx[r] = oi;
    w.yv[r] = delta;
    w.score[nc0 + r] = fabs(yp + un) / sqrt(yy + 1.0);
    w.eig[nc0 + r] = origin + delta;
  }
}

// Phase 3, one block per orbital: selection (largest score; ties within tie_rtol to the lower eigenvalue), the
// eigenvector back in the V basis and the coarse coefficients.
__global__ void k_sec_select(int n, int N, const double* __restrict__ V, const double* __restrict__ G,
                             double* __restrict__ work, int* __restrict__ iwork, double* __restrict__ lambda,
                             double* __restrict__ coef, int32_t* __restrict__ status, double tie_rtol) {
  const int i = blockIdx.x;
  if (i >= N) return;
  SecWork w = sec_work(work, iwork, n, i);
  if (w.hdr[4] != 0.0) return;
  __shared__ double s_norm, s_sign, s_ylast;
  __shared__ int s_sel;
  const int tid = threadIdx.x;
  const int m = (int)w.hdr[2], ncand = (int)w.hdr[3];
  const double alpha = w.hdr[0], un = w.hdr[1];
  if (tid == 0) {
    double best = -1.0;
    for (int t = 0; t < ncand; ++t) best = fmax(best, w.score[t]);
    int sel = -1;
    for (int t = 0; t < ncand; ++t)
      if (w.score[t] >= best * (1.0 - tie_rtol) && (sel < 0 || w.eig[t] < w.eig[sel])) sel = t;
    s_sel = sel;
    if (sel >= 0) {
      lambda[i] = w.eig[sel];
      status[i] = MK_OK;
    } else {  // no finite score (non-finite input): report and write nothing else
      lambda[i] = NAN;
      status[i] = MK_ERR_NOT_CONVERGED;
    }
  }
  for (int t = tid; t < n; t += blockDim.x) w.ytmp[t] = 0.0;
  __syncthreads();
  if (s_sel < 0) {
    for (int r = tid; r <= n; r += blockDim.x) coef[(int64_t)r * N + i] = 0.0;
    return;
  }
  const int sel = s_sel;
  if (w.kind[sel] < 0) {
    if (tid == 0) {
      w.ytmp[-w.kind[sel] - 1] = 1.0;
      s_ylast = 0.0;
    }
  } else {
    const int r = w.kind[sel];
    const int oi = w.origin_idx[r];
    const double origin = oi >= 0 ? w.dk[oi] : alpha;
    const double delta = w.yv[r];
    for (int t = tid; t < m; t += blockDim.x) w.ytmp[w.comp[t]] = w.zk[t] / ((origin - w.dk[t]) + delta);
    if (tid == 0) s_ylast = 1.0;
  }
  __syncthreads();
  if (tid == 0) {
    double nn = s_ylast * s_ylast, sp = s_ylast * un;
    for (int t = 0; t < n; ++t) {
      nn += w.ytmp[t] * w.ytmp[t];
      sp += w.ytmp[t] * w.ps[t];
    }
    s_norm = sqrt(nn);
    s_sign = sp < 0 ? -1.0 : 1.0;
    // back to the original V basis: undo the rotations in reverse order of creation
    for (int k = n - 1; k >= 0; --k) {
      const int l = w.partner[k];
      if (l < 0) continue;
      const double a = w.ytmp[l], b = w.ytmp[k];
      w.ytmp[l] = a * w.rcos[k] - b * w.rsin[k];
      w.ytmp[k] = a * w.rsin[k] + b * w.rcos[k];
    }
  }
  __syncthreads();
  const double scale = s_sign / s_norm;
  const double yl = scale * s_ylast;
  // coarse part: phi_H = V (y - (y_last/||u||) p), theta_2 = y_last/||u||
  for (int k = tid; k < n; k += blockDim.x) w.yv[k] = scale * w.ytmp[k] - (yl / un) * G[(int64_t)k * 2 * N + N + i];
  __syncthreads();
  for (int r = tid; r < n; r += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += V[(int64_t)r * n + k] * w.yv[k];
    coef[(int64_t)r * N + i] = s;
  }
  if (tid == 0) coef[(int64_t)n * N + i] = yl / un;
}

// The three phases for all orbitals; work holds N * sec_stride(n) doubles, iwork N * 4 (n+1) ints.
static void secular_launch(int n, int N, const double* d, const double* V, const double* G, const double* beta,
                           const double* gamma, double* work, int* iwork, double* lambda, double* coef,
                           int32_t* status, cudaStream_t s) {
  const double sing_rtol = 1e-7, tie_rtol = 1e-12;
  MK_COUNT(), k_sec_prepare<<<N, kEigThreads, 0, s>>>(n, N, d, V, G, beta, gamma, work, iwork, lambda, coef, status,
                                                     sing_rtol, tie_rtol);
  const int64_t warps = (int64_t)N * (n + 1);
  MK_COUNT(), k_sec_roots<<<(int)((warps + 7) / 8), 256, 0, s>>>(n, N, work, iwork);
  MK_COUNT(), k_sec_select<<<N, kEigThreads, 0, s>>>(n, N, V, G, work, iwork, lambda, coef, status, tie_rtol);
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
  if (h) return fail(MK_ERR_INVALID_ARG, "coarse matrix is not positive definite");
  return MK_OK;
}

__global__ void k_to_float(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

int coarse_matrices(mk_ctx*, const mk_mesh*, const double*, const double*, double*, double*, int, cudaStream_t);

int coarse_inverse32(mk_ctx* ctx, const mk_mesh* m, const double* A64, float* out, cudaStream_t s) {
  const int n = (int)m->coarse.n_free;
  int err = MK_OK;
  double* X = (double*)scratch(ctx, S_TLX, (size_t)n * n * 3 * sizeof(double), &err);
  if (!X) return err;
  double* X2 = X + (size_t)n * n;
  double* Li = X2 + (size_t)n * n;
  MK_TRY(coarse_matrices(ctx, m, A64, nullptr, X, nullptr, S_TLC, s));  // A_H = P^T A P
  MK_TRY(inverse_cholesky(ctx, n, X, Li, S_TLW, s));                 // A_H = L L^T, Li = L^-1
  gemm64(n, n, n, Li, n, 1, Li, n, 0, X2, n, s);                     // A_H^-1 = L^-T L^-1
  MK_COUNT(), k_to_float<<<(int)(((int64_t)n * n + 255) / 256), 256, 0, s>>>((int64_t)n * n, X2, out);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

// Shared decomposition of the coarse pencil: C = Linv AH Linv^T, Jacobi C = Q diag Q^T, d ascending,
// V = Linv^T Q (columns sorted with d).  V row-major [n x n], V[i][k] = component i of eigenvector k.
// In a basis W with W^T M_H W = I the pencil (AH, M_H) is the symmetric matrix C = W^T AH W; its Jacobi
// eigenvectors Q give V = W Q (M_H-orthonormal), d ascending.  W = X when w_is_x (a previous eigenbasis: warm
// start, C is then nearly diagonal), W = X^T when X = L^-1 (M_H = L L^T).  V row-major, V[i][k] = component i
// of eigenvector k.
int decompose(mk_ctx* ctx, int n, const double* X, bool w_is_x, const double* AH, double* d, double* V,
              cudaStream_t s, int slot = S_EIG2) {
  // block Jacobi on n padded to a multiple of 2 kBW
  const int n2 = (n + kBP - 1) / kBP * kBP;
  int err = MK_OK;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  const size_t oT = take((size_t)n * n * 8), oC = take((size_t)n * n * 8), oS0 = take((size_t)n2 * n2 * 8);
  const size_t oS1 = take((size_t)n2 * n2 * 8), oQ = take((size_t)n2 * n2 * 8), oRed = take(8192 * 8);
  const size_t oPerm = take((size_t)n * 4), oInfo = take(64), oU = take((size_t)2 * (n2 / kBP) * kBP * kBP * 8);
  const size_t oG = take((size_t)n2 * n2 * 8), oX2 = take((size_t)n2 * n2 * 8);
  const size_t oS32a = take((size_t)n2 * n2 * 4), oS32b = take((size_t)n2 * n2 * 4), oQ32 = take((size_t)n2 * n2 * 4);
  char* ws = (char*)scratch(ctx, slot, off, &err);
  if (!ws) return err;
  double *T = (double*)(ws + oT), *C = (double*)(ws + oC), *S0 = (double*)(ws + oS0), *S1 = (double*)(ws + oS1);
  double *Q = (double*)(ws + oQ), *red = (double*)(ws + oRed);
  int *perm = (int*)(ws + oPerm), *info = (int*)(ws + oInfo);
  double* Ug = (double*)(ws + oU);
  double *G = (double*)(ws + oG), *X2 = (double*)(ws + oX2);
  float *S32a = (float*)(ws + oS32a), *S32b = (float*)(ws + oS32b), *Q32 = (float*)(ws + oQ32);
  float* Ug32 = (float*)(ws + oU);  // the FP32 phase's transforms, in the FP64 phase's (later) place
  const int tx = w_is_x ? 1 : 0;                                     // op for W^T
  gemm64(n, n, n, X, n, tx, AH, n, 0, T, n, s);                      // T = W^T AH
  gemm64(n, n, n, T, n, 0, X, n, 1 - tx, C, n, s);                   // C = T W
  const int64_t nn2 = (int64_t)n2 * n2;
  const int ew = (int)((nn2 + 255) / 256);
  MK_COUNT(), k_pad_sym<<<ew, 256, 0, s>>>(n, n2, C, S0, Q, 0.0);
  int n2v = n2;
  int per_sm = 0, per_sm32 = 0;
  MK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bjacobi, kBJThreads, 0));
  MK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm32, k_bjacobi32, kBJThreads, 0));
  MK_ARG(per_sm >= 1 && per_sm32 >= 1, "mk: block Jacobi kernel cannot be resident");
  // at most one CTA per SM (half its registers): the fine solve's kernels on the other stream run beside it
  int grid = std::min(ctx->n_sms, 4096);
  if (ctx->decompose_ctas > 0) grid = std::min(grid, ctx->decompose_ctas);
  MK_ARG(grid > n2 / kBP, "mk: block Jacobi needs more CTAs than block pairs (coarse space too large)");
  // the largest shared-memory carveout, so that an SM running this CTA can also take the fine solve's CTAs
  MK_CUDA(cudaFuncSetAttribute(k_bjacobi32, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared));
  MK_CUDA(cudaFuncSetAttribute(k_bjacobi, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared));
  // (1) the sweeps of the linear phase in FP32, to off(S) <= 1e-5 |S| or the FP32 floor
  {
    int max32 = 40;
    double tol32 = 1e-5;
    int* info32 = info + 4;
    MK_COUNT(), k_bj_to32<<<ew, 256, 0, s>>>(nn2, n2, S0, S32a, Q32);
    void* a32[] = {&n2v, &S32a, &S32b, &Q32, &Ug32, &red, &max32, &tol32, &info32};
    MK_COUNT();
    MK_CUDA(cudaLaunchCooperativeKernel((void*)k_bjacobi32, grid, kBJThreads, a32, 0, s));
  }
  // (2) its Q made orthogonal in FP64 (two Newton-Schulz steps: ~1e-6 -> ~1e-12 -> FP64 rounding) and the FP64
  // matrix projected onto it: S0 <- Q^T S0 Q, symmetrised; the FP64 sweeps then accumulate into this Q
  {
    MK_COUNT(), k_f32_to_f64<<<ew, 256, 0, s>>>(nn2, Q32, Q);
    const dim3 tg((n2 + 31) / 32, (n2 + 31) / 32);
    gemm64(n2, n2, n2, Q, n2, 1, Q, n2, 0, G, n2, s);                 // G = Q^T Q
    MK_COUNT(), k_ns_step<<<tg, 256, 0, s>>>(n2, Q, G, X2);
    gemm64(n2, n2, n2, X2, n2, 1, X2, n2, 0, G, n2, s);
    MK_COUNT(), k_ns_step<<<tg, 256, 0, s>>>(n2, X2, G, Q);
    gemm64(n2, n2, n2, S0, n2, 0, Q, n2, 0, G, n2, s);                // G = S0 Q
    gemm64(n2, n2, n2, Q, n2, 1, G, n2, 0, S1, n2, s);                // S1 = Q^T S0 Q
    MK_COUNT(), k_symmetrize<<<ew, 256, 0, s>>>(n2, S1, S0);
  }
  ctx->last_decompose_info = info;
  // (3) the FP64 sweeps to off(S) <= 1e-14 |S|
  int max_sweeps = 60;
  double tol = 1e-14;
  void* args[] = {&n2v, &S0, &S1, &Q, &Ug, &red, &max_sweeps, &tol, &info};
  MK_COUNT();
  MK_CUDA(cudaLaunchCooperativeKernel((void*)k_bjacobi, grid, kBJThreads, args, 0, s));
  MK_COUNT(), k_rank<<<(n + 127) / 128, 128, 0, s>>>(n, n2, S0, S1, info, d, perm);
  MK_COUNT(), k_gather_cols<<<(int)(((int64_t)n * n + 255) / 256), 256, 0, s>>>(n, n2, Q, perm, C);  // C = Q sorted
  gemm64(n, n, n, X, n, 1 - tx, C, n, 0, V, n, s);                   // V = W Q
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

int secular(mk_ctx* ctx, int n, int N, const double* d, const double* V, const double* b, const double* c,
            const double* beta, const double* gamma, double* lambda, double* coef, int32_t* status, cudaStream_t s) {
  int err = MK_OK;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  const size_t oG = take((size_t)n * 2 * N * 8), oW = take((size_t)N * sec_stride(n) * 8);
  const size_t oIW = take((size_t)N * 4 * (n + 1) * 4);
  char* ws = (char*)scratch(ctx, S_EIG, off, &err);
  if (!ws) return err;
  double *G = (double*)(ws + oG), *W = (double*)(ws + oW);
  int* IW = (int*)(ws + oIW);
  MK_COUNT(), k_vt_bc<<<(int)(((int64_t)n * 2 * N + 127) / 128), 128, 0, s>>>(n, N, V, b, c, G);
  secular_launch(n, N, d, V, G, beta, gamma, W, IW, lambda, coef, status, s);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

// At mesh upload: M_H = P^T M P and its inverse Cholesky factor, kept in the mesh handle.

// ------------------------------------------------------------------------------------------------ joint space
// Rayleigh-Ritz in V_H + span{psi^_1..psi^_N}.  With V the M_H-orthonormal eigenvectors of (A_H, M_H) (eigenvalues
// D), M_H^-1 = V V^T, so the corrections' parts M-orthogonal to V_H are U = Psi^ - P V (V^T C), with Gram
// S = G_M - (V^T C)^T (V^T C) and Hamiltonian block U^T H U = G_A - (V^T C)^T (V^T B) - (V^T B)^T (V^T C)
// + (V^T C)^T D (V^T C).  S = Y diag(s) Y^T; the columns with s_j above 1e-12 max(1, s_max) give an M-orthonormal
// basis U W of the corrections' new directions, W = Y_kept diag(s_kept)^-1/2 (linearly dependent ones dropped).  In
// the basis [P V, U W] the joint pencil is the standard symmetric problem
//   T = [[D, Z], [Z^T, W^T (U^T H U) W]],  Z = (V^T B - D V^T C) W,
// whose eigenvectors (y_top, y_bot) give the joint Ritz vectors P V (y_top - (V^T C) W y_bot) + Psi^ W y_bot.
// G = [V^T B | V^T C] [n][2N] as k_vt_bc writes it.
__global__ void k_joint_small(int n, int N, const double* __restrict__ G, const double* __restrict__ d,
                              const double* __restrict__ gA, const double* __restrict__ gM, double* __restrict__ S,
                              double* __restrict__ A0) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * N) return;
  const int i = t / N, j = t % N;
  double sm = 0.0, sa = 0.0;
  for (int r = 0; r < n; ++r) {
    const double* g = G + (int64_t)r * 2 * N;
    const double bi = g[i], bj = g[j], ci = g[N + i], cj = g[N + j];
    sm += ci * cj;
    sa += (ci * bj + bi * cj) - ci * d[r] * cj;
  }
  // the Grams symmetrised as the joint pencil is (each (i, j) and (j, i) sum the same terms in the same order)
  S[t] = 0.5 * (gM[i * N + j] + gM[j * N + i]) - sm;
  A0[t] = 0.5 * (gA[i * N + j] + gA[j * N + i]) - sa;
}
__global__ void k_joint_W(int N, int kp, int first, const double* __restrict__ s, const double* __restrict__ Y,
                          double* __restrict__ W) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * kp) return;
  const int i = t / kp, a = t % kp;
  W[t] = Y[(int64_t)i * N + first + a] / sqrt(s[first + a]);
}
// Z [n][kp] = (V^T B - D V^T C) W and At [kp][kp] = W^T A0 W
__global__ void k_joint_Z(int n, int N, int kp, const double* __restrict__ G, const double* __restrict__ d,
                          const double* __restrict__ W, double* __restrict__ Z) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * kp) return;
  const int r = (int)(t / kp), a = (int)(t % kp);
  const double* g = G + (int64_t)r * 2 * N;
  double z = 0.0;
  for (int i = 0; i < N; ++i) z += (g[i] - d[r] * g[N + i]) * W[i * kp + a];
  Z[t] = z;
}
__global__ void k_joint_At(int N, int kp, const double* __restrict__ A0, const double* __restrict__ W,
                           double* __restrict__ At) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kp * kp) return;
  const int a = t / kp, b = t % kp;
  double v = 0.0;
  for (int i = 0; i < N; ++i) {
    double w = 0.0;
    for (int j = 0; j < N; ++j) w += A0[i * N + j] * W[j * kp + b];
    v += W[i * kp + a] * w;
  }
  At[t] = v;
}
__global__ void k_joint_T(int n, int kp, const double* __restrict__ d, const double* __restrict__ Z,
                          const double* __restrict__ At, double* __restrict__ T) {
  const int nT = n + kp;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)nT * nT) return;
  const int r = (int)(t / nT), c = (int)(t % nT);
  double v;
  if (r < n && c < n) v = r == c ? d[r] : 0.0;
  else if (r < n) v = Z[(int64_t)r * kp + (c - n)];
  else if (c < n) v = Z[(int64_t)c * kp + (r - n)];
  else v = 0.5 * (At[(r - n) * kp + (c - n)] + At[(c - n) * kp + (r - n)]);
  T[t] = v;
}
// for Ritz vectors j < k: w = W y_bot (the corrections' coefficients, rows n.. of X) and
// tmp = y_top - (V^T C) w (coarse coefficients in the eigenbasis V)
__global__ void k_joint_coef(int n, int N, int kp, int k, const double* __restrict__ Yt, const double* __restrict__ W,
                             const double* __restrict__ G, double* __restrict__ X, double* __restrict__ tmp) {
  const int nT = n + kp;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)(n + N) * k) return;
  const int r = (int)(t / k), j = (int)(t % k);
  auto wcoef = [&](int i) {
    double w = 0.0;
    for (int a = 0; a < kp; ++a) w += W[i * kp + a] * Yt[(int64_t)(n + a) * nT + j];
    return w;
  };
  if (r >= n) {
    X[(int64_t)r * k + j] = wcoef(r - n);
  } else {
    double v = Yt[(int64_t)r * nT + j];
    const double* g = G + (int64_t)r * 2 * N;
    for (int i = 0; i < N; ++i) v -= g[N + i] * wcoef(i);
    tmp[(int64_t)r * k + j] = v;
  }
}
__global__ void k_joint_orbitals(int64_t n_nodes, const int32_t* __restrict__ off, const int32_t* __restrict__ col,
                                 const double* __restrict__ val, const uint8_t* __restrict__ bnd,
                                 const double* __restrict__ X, int n, int k, const double* __restrict__ psihat, int N,
                                 int ld, double* __restrict__ psi) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_nodes * ld) return;
  const int64_t nd = t / ld;
  const int j = (int)(t % ld);
  double v = 0.0;
  if (j < k && !bnd[nd]) {
    for (int q = off[nd]; q < off[nd + 1]; ++q) v += val[q] * X[(int64_t)col[q] * k + j];
    for (int i = 0; i < N; ++i) v += X[(int64_t)(n + i) * k + j] * psihat[nd * ld + i];
  }
  psi[t] = v;
}

int mesh_mass_factor(mk_ctx* ctx, mk_mesh* m) {
  const Level& F = m->fine;
  const int n = (int)m->coarse.n_free;
  int err = MK_OK;
  const size_t eb = (size_t)F.n_elems * (F.nloc * (F.nloc + 1) / 2) * sizeof(double);
  double* Me = (double*)scratch(ctx, S_ELEM64D, eb, &err);
  double* MH = (double*)scratch(ctx, S_VEC5, (size_t)n * n * sizeof(double) * 2, &err);
  if (!Me || !MH) return err;
  cudaStream_t s = 0;
  MK_TRY(element_matrices(ctx, F, nullptr, 0.0, 0.0, 1.0, nullptr, Me, s));
  MK_TRY(coarse_matrices(ctx, m, Me, nullptr, MH, nullptr, S_COARSE2, s));
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

int mk_decompose_info(mk_ctx* ctx, int* sweeps32, int* sweeps64) {
  MK_ARG(ctx && sweeps32 && sweeps64, "mk_decompose_info: null argument");
  MK_ARG(ctx->last_decompose_info, "mk_decompose_info: no decomposition on this context yet");
  MK_CUDA(cudaSetDevice(ctx->device));
  MK_CUDA(cudaDeviceSynchronize());
  int h[5];
  MK_CUDA(cudaMemcpy(h, ctx->last_decompose_info, sizeof(h), cudaMemcpyDeviceToHost));
  *sweeps64 = h[0];
  *sweeps32 = h[4];
  return MK_OK;
}

int mk_coarse_decompose(mk_ctx* ctx, const mk_mesh* m, const double* AH, double* d, double* V, void* stream) {
  MK_ARG(ctx && m && AH && d && V && m->d_MH_Linv, "mk_coarse_decompose: null argument");
  MK_CUDA(cudaSetDevice(ctx->device));
  return decompose(ctx, (int)m->coarse.n_free, m->d_MH_Linv, false, AH, d, V, (cudaStream_t)stream);
}

int mk_coarse_decompose_warm(mk_ctx* ctx, int NH, const double* AH, const double* V0, double* d, double* V,
                             void* stream) {
  MK_ARG(ctx && AH && V0 && d && V && NH >= 1, "mk_coarse_decompose_warm: bad argument");
  MK_ARG(V0 != V, "mk_coarse_decompose_warm: V0 and V must not alias");
  MK_CUDA(cudaSetDevice(ctx->device));
  return decompose(ctx, NH, V0, true, AH, d, V, (cudaStream_t)stream);
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
  MK_TRY(decompose(ctx, NH, Linv, false, AH, d, V, s));
  return secular(ctx, NH, N, d, V, b, c, beta, gamma, lambda, coef, status, s);
}

int mk_joint_ritz(mk_ctx* ctx, int NH, int N, int k, const double* d, const double* V, const double* b,
                  const double* c, const double* gramA, const double* gramM, double* lambda, double* X, int* n_kept,
                  void* stream) {
  MK_ARG(ctx && d && V && b && c && gramA && gramM && lambda && X, "mk_joint_ritz: null argument");
  MK_ARG(NH >= 1 && N >= 1 && N <= MK_MAX_RHS && k >= 1, "mk_joint_ritz: bad sizes");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  int err = MK_OK;
  const int nTmax = NH + N;
  size_t off = 0;
  auto take = [&](size_t doubles) { size_t o = off; off += (doubles + 31) / 32 * 32; return o; };
  const size_t oG = take((size_t)NH * 2 * N), oS = take((size_t)N * N), oA0 = take((size_t)N * N);
  const size_t oI = take((size_t)nTmax * nTmax), osv = take(N), oY = take((size_t)N * N), oW = take((size_t)N * N);
  const size_t oZ = take((size_t)NH * N), oAt = take((size_t)N * N), oT = take((size_t)nTmax * nTmax);
  const size_t omu = take(nTmax), oYt = take((size_t)nTmax * nTmax), otmp = take((size_t)NH * nTmax);
  double* ws = (double*)scratch(ctx, S_JOINT, off * sizeof(double), &err);
  if (!ws) return err;
  double *G = ws + oG, *S = ws + oS, *A0 = ws + oA0, *I = ws + oI, *sv = ws + osv, *Y = ws + oY, *W = ws + oW;
  double *Z = ws + oZ, *At = ws + oAt, *T = ws + oT, *mu = ws + omu, *Yt = ws + oYt, *tmp = ws + otmp;
  MK_COUNT(), k_vt_bc<<<(int)(((int64_t)NH * 2 * N + 127) / 128), 128, 0, s>>>(NH, N, V, b, c, G);
  MK_COUNT(), k_joint_small<<<(N * N + 127) / 128, 128, 0, s>>>(NH, N, G, d, gramA, gramM, S, A0);
  MK_COUNT(), k_identity<<<(N * N + 255) / 256, 256, 0, s>>>(N, I);
  MK_TRY(decompose(ctx, N, I, true, S, sv, Y, s, S_EIG5));
  std::vector<double> hs(N);
  MK_CUDA(cudaMemcpyAsync(hs.data(), sv, N * sizeof(double), cudaMemcpyDeviceToHost, s));
  MK_CUDA(cudaStreamSynchronize(s));
  const double smax = std::max(1.0, hs[N - 1]);
  int first = 0;
  while (first < N && !(hs[first] > 1e-12 * smax)) ++first;  // ascending: the dropped directions come first
  const int kp = N - first;
  const int nT = NH + kp;
  if (n_kept) *n_kept = kp;
  MK_ARG(k <= nT, "mk_joint_ritz: k exceeds the dimension of the joint space");
  if (kp > 0) {
    MK_COUNT(), k_joint_W<<<(N * kp + 127) / 128, 128, 0, s>>>(N, kp, first, sv, Y, W);
    MK_COUNT(), k_joint_Z<<<(int)(((int64_t)NH * kp + 127) / 128), 128, 0, s>>>(NH, N, kp, G, d, W, Z);
    MK_COUNT(), k_joint_At<<<(kp * kp + 127) / 128, 128, 0, s>>>(N, kp, A0, W, At);
  }
  MK_COUNT(), k_joint_T<<<(int)(((int64_t)nT * nT + 255) / 256), 256, 0, s>>>(NH, kp, d, Z, At, T);
  MK_COUNT(), k_identity<<<(int)(((int64_t)nT * nT + 255) / 256), 256, 0, s>>>(nT, I);
  MK_TRY(decompose(ctx, nT, I, true, T, mu, Yt, s, S_EIG5));
  MK_COUNT(), k_joint_coef<<<(int)(((int64_t)(NH + N) * k + 127) / 128), 128, 0, s>>>(NH, N, kp, k, Yt, W, G, X, tmp);
  gemm64(NH, k, NH, V, NH, 0, tmp, k, 0, X, k, s);  // coarse coefficients V tmp into rows [0, NH) of X
  MK_CUDA(cudaMemcpyAsync(lambda, mu, k * sizeof(double), cudaMemcpyDeviceToDevice, s));
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

int mk_joint_assemble(mk_ctx* ctx, const mk_mesh* m, int k, int N, const double* X, const double* psihat,
                      const double* u, int ld, double* psi, void* stream) {
  MK_ARG(ctx && m && X && psihat && u && psi, "mk_joint_assemble: null argument");
  MK_ARG(N >= 1 && k >= 1 && N <= ld && k <= ld && ld <= MK_MAX_RHS, "mk_joint_assemble: bad N/k/ld");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const Level& F = m->fine;
  int err = MK_OK;
  double* Mu = (double*)scratch(ctx, S_VEC1, (size_t)F.n_nodes * ld * sizeof(double), &err);
  double* dots = (double*)scratch(ctx, S_COEF, 64 * sizeof(double), &err);
  if (!Mu || !dots) return err;
  const double* Me = mass_matrices(ctx, m, s, &err);
  if (!Me) return err;
  const int64_t work = F.n_nodes * ld;
  MK_COUNT(), k_joint_orbitals<<<(int)((work + 255) / 256), 256, 0, s>>>(F.n_nodes, m->d_P_off, m->d_P_col, m->d_P_val,
                                                                         F.d_boundary, X, (int)m->coarse.n_free, k,
                                                                         psihat, N, ld, psi);
  MK_TRY(apply64(ctx, m, Me, u, Mu, k, ld, true, s));
  MK_TRY(column_dots(ctx, F.n_nodes, psi, Mu, k, ld, dots, s));
  MK_COUNT(), k_flip<<<(int)((work + 255) / 256), 256, 0, s>>>(F.n_nodes, dots, psi, k, ld);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

int mk_orbital_assemble(mk_ctx* ctx, const mk_mesh* m, const double* coef, const double* psihat, const double* u,
                        int ld, int N, double* psi, void* stream) {
  MK_ARG(ctx && m && coef && psihat && u && psi, "mk_orbital_assemble: null argument");
  MK_ARG(N >= 1 && N <= ld && N <= MK_MAX_RHS, "mk_orbital_assemble: bad N/ld");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const Level& F = m->fine;
  int err = MK_OK;
  double* Mu = (double*)scratch(ctx, S_VEC1, (size_t)F.n_nodes * ld * sizeof(double), &err);
  double* dots = (double*)scratch(ctx, S_COEF, 64 * sizeof(double), &err);
  if (!Mu || !dots) return err;
  const double* Me = mass_matrices(ctx, m, s, &err);
  if (!Me) return err;
  const int64_t work = F.n_nodes * ld;
  MK_COUNT(), k_orbitals<<<(int)((work + 255) / 256), 256, 0, s>>>(F.n_nodes, m->d_P_off, m->d_P_col, m->d_P_val, F.d_boundary,
                                                       coef, (int)m->coarse.n_free, psihat, N, ld, psi);
  MK_TRY(apply64(ctx, m, Me, u, Mu, N, ld, true, s));
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
constexpr size_t kStaticW = (size_t)kStaticMaxN * sec_stride(kStaticMaxNH);          // doubles: per-orbital work
constexpr size_t kStaticIW = (size_t)kStaticMaxN * 4 * (kStaticMaxNH + 1);            // ints: per-orbital work
static __device__ __align__(256) double g_static_ws[kStaticG + kStaticW + (kStaticIW + 1) / 2];

static std::mutex g_static_mu;
static double* g_static_ptr[64] = {nullptr};

// Device address of g_static_ws on the current device, looked up once per device (host code cannot use the
// array's name as a device address) and kept for the process: a device reset would make it stale, which the
// entry point's documentation rules out.
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
  secular_launch(NH, N, d, V, G, beta, gamma, W, IW, lambda, coef, status, s);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}
