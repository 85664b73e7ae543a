// Boundary-value problems on the fine mesh (Algorithm 1, steps 5 and 6): multi-RHS PCG on the matrix-free
// element-by-element operator, the Hartree Poisson solve, the right-hand sides, and the shift estimate.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "mk_device.cuh"
#include "mk_patch.cuh"

namespace mk {

int restrict_to_coarse(mk_ctx*, const mk_mesh*, const double*, int, int, double*, int, cudaStream_t);
int prolongate(mk_ctx*, const mk_mesh*, const double*, int, int, double*, int, cudaStream_t);
int density(mk_ctx*, const Level&, const double*, int, int, const double*, double*, cudaStream_t);
int frozen_potential(mk_ctx*, const Level&, const double*, const double*, mk_xc, double*, cudaStream_t);
int load_vector(mk_ctx*, const Level&, const double*, double, double*, cudaStream_t);
int multipole_boundary(mk_ctx*, const Level&, const double*, const double*, int, double*, cudaStream_t);
int solve_mixed(mk_ctx*, const mk_mesh*, const mk_molecule*, double, const double*, const double*, const double*,
                double*, int, int, const mk_solve_opts&, mk_solve_report*, cudaStream_t);
int pcg_mixed(mk_ctx*, const mk_mesh*, const double*, const double*, double*, int, int, const mk_solve_opts&,
              mk_solve_report*, cudaStream_t, const float* cinv = nullptr, bool stiff = false,
              const double* diag_pre = nullptr);

// Per-column PCG state on the device.
struct ColState {
  double rz, pq, rr, bn, alpha, beta, rz_new;
  int active, iters, breakdown, pad;
};

__global__ void k_residual(int64_t n, const uint8_t* __restrict__ bnd, const double* __restrict__ b,
                           const double* __restrict__ Ax, const double* __restrict__ diag, double* __restrict__ r,
                           double* __restrict__ z, double* __restrict__ p, int N, int ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ld) return;
  const int64_t nd = t / ld;
  const int j = (int)(t % ld);
  double rv = 0.0;
  if (j < N && !bnd[nd]) rv = b[t] - Ax[t];
  r[t] = rv;
  const double zv = rv / diag[nd];
  if (z) z[t] = zv;
  if (p) p[t] = zv;
}

__global__ void k_init_state(ColState* st, const double* bb, const double* rz, const double* rr, int N, double rtol) {
  const int j = threadIdx.x;
  if (j >= N) return;
  ColState c{};
  c.bn = bb[j] > 0 ? sqrt(bb[j]) : 1.0;
  c.rz = rz[j];
  c.rr = rr[j];
  c.active = sqrt(rr[j]) / c.bn > rtol;
  st[j] = c;
}

__global__ void k_alpha(ColState* st, const double* pq, int N) {
  const int j = threadIdx.x;
  if (j >= N) return;
  ColState c = st[j];
  c.pq = pq[j];
  if (c.active) {
    if (!(c.pq > 0.0)) {
      c.breakdown = 1;
      c.active = 0;
      c.alpha = 0.0;
    } else {
      c.alpha = c.rz / c.pq;
    }
  } else {
    c.alpha = 0.0;
  }
  st[j] = c;
}

__global__ void k_update(int64_t n, const ColState* __restrict__ st, const double* __restrict__ p,
                         const double* __restrict__ q, const double* __restrict__ diag, double* __restrict__ x,
                         double* __restrict__ r, double* __restrict__ z, int N, int ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ld) return;
  const int j = (int)(t % ld);
  if (j >= N) return;
  const double a = st[j].alpha;
  if (a == 0.0) return;
  x[t] += a * p[t];
  const double rv = r[t] - a * q[t];
  r[t] = rv;
  z[t] = rv / diag[t / ld];
}

__global__ void k_beta(ColState* st, const double* rz_new, const double* rr, int N, double rtol) {
  const int j = threadIdx.x;
  if (j >= N) return;
  ColState c = st[j];
  if (c.active) {
    c.beta = rz_new[j] / c.rz;
    c.rz = rz_new[j];
    c.rr = rr[j];
    c.iters += 1;
    c.active = sqrt(c.rr) / c.bn > rtol;
  } else {
    c.beta = 0.0;
  }
  st[j] = c;
}

__global__ void k_pupdate(int64_t n, const ColState* __restrict__ st, const double* __restrict__ z,
                          double* __restrict__ p, int N, int ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ld) return;
  const int j = (int)(t % ld);
  if (j >= N || !st[j].active) return;
  p[t] = z[t] + st[j].beta * p[t];
}

// Lowest (upper = false) or highest eigenvalue of a symmetric tridiagonal matrix (diagonal a, off-diagonal b) by
// Sturm-sequence bisection (host, tiny).
static double tridiag_extreme(const std::vector<double>& a, const std::vector<double>& b, bool upper) {
  const int n = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < n; ++i) {
    double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    int count = 0;  // eigenvalues below mid
    double d = 1.0;
    for (int i = 0; i < n; ++i) {
      d = a[i] - mid - (i > 0 ? b[i - 1] * b[i - 1] / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0) ++count;
    }
    if (upper ? count >= n : count >= 1) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

__global__ void k_scale(int64_t n, double* __restrict__ v, const double* __restrict__ num,
                        const double* __restrict__ den, int mode) {
  // mode 0: v *= 1/sqrt(num[0]);  used by Lanczos normalisation
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  (void)den;
  if (mode == 0) v[i] *= 1.0 / sqrt(num[0]);
}

__global__ void k_lanczos_w(int64_t n, const uint8_t* __restrict__ bnd, double* __restrict__ w,
                            const double* __restrict__ v, const double* __restrict__ vprev, double alpha,
                            double beta) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  w[i] = bnd[i] ? 0.0 : w[i] - alpha * v[i] - beta * vprev[i];
}

// ------------------------------------------------------------------------------------------------ Chebyshev
// Polynomial preconditioner z = p(D^-1 A) D^-1 r of degree kChebDegree: the Chebyshev iteration for A z = r with
// the diagonal D, started at z = 0, on an interval [a, b] of the spectrum of D^-1 A (Saad, Iterative Methods for
// Sparse Linear Systems, Sec. 12.3).  The same polynomial for every column and every call, so a fixed symmetric
// linear map; it is positive definite whenever b bounds the spectrum from above and a > 0 (the residual polynomial
// then stays below 1 on (0, b]).  b is 1.1 times, a once, the extreme Ritz values of kChebLanczos Lanczos steps
// on D^-1/2 A D^-1/2.
constexpr int kChebDegree = 4;
constexpr int kChebLanczos = 16;
struct ChebCoef {
  double theta, delta, sigma1;
};
// one step: res -= A d; d = c1 d + c2 D^-1 res; z += d (interior rows; columns < N)
__global__ void k_cheb_step(int64_t n, const uint8_t* __restrict__ bnd, const double* __restrict__ diag,
                            double* __restrict__ res, const double* __restrict__ Ad, double* __restrict__ d,
                            double* __restrict__ z, int N, int ld, double c1, double c2, int first) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ld) return;
  const int64_t nd = t / ld;
  const int j = (int)(t % ld);
  if (j >= N || bnd[nd]) {
    if (first) { d[t] = 0.0; z[t] = 0.0; }
    return;
  }
  double rv = res[t];
  if (!first) rv -= Ad[t];
  res[t] = rv;
  const double dv = (first ? 0.0 : c1 * d[t]) + c2 * rv / diag[nd];
  d[t] = dv;
  z[t] = first ? dv : z[t] + dv;
}
__global__ void k_copy_cols(int64_t n, const double* __restrict__ a, double* __restrict__ b, int ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n * ld) b[t] = a[t];
}
// u = D^-1/2 v (inverse) or D^1/2 v on the interior rows (the Lanczos steps on D^-1/2 A D^-1/2, one column)
__global__ void k_lz_scale(int64_t n, const uint8_t* __restrict__ bnd, const double* __restrict__ diag,
                           const double* v, double* u, int inverse) {  // u may be v
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  u[i] = bnd[i] ? 0.0 : (inverse ? v[i] / sqrt(diag[i]) : v[i] * sqrt(diag[i]));
}
__global__ void k_lz_start(int64_t n, const uint8_t* __restrict__ bnd, double* __restrict__ v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // a fixed start vector with no special symmetry: a hash of the node index in (0.5, 1.5)
  uint32_t h = (uint32_t)i * 2654435761u;
  h ^= h >> 16;
  v[i] = bnd[i] ? 0.0 : 0.5 + (double)(h & 0xffffu) / 65536.0;
}

// Plain FP64 PCG on all columns at once: Jacobi, or the Chebyshev polynomial preconditioner.  `Ae` packed element matrices of the SPD operator, `diag` its
// assembled diagonal (boundary rows 1).  x: initial guess in, solution out (boundary rows forced to 0).
int pcg64(mk_ctx* ctx, const mk_mesh* m, const double* Ae, const double* diag, const double* b, double* x, int N,
          int ld, const mk_solve_opts& o, mk_solve_report* rep, cudaStream_t s) {
  const Level& L = m->fine;
  int err = MK_OK;
  const int64_t n = L.n_nodes;
  // the FP64 patch operator: element matrices packed in patch order once per solve
  double* Ap = (double*)scratch(ctx, S_ELEMP64, (size_t)L.n_elems * padded_np(L.nloc, 8) * sizeof(double), &err);
  if (!Ap) return err;
  MK_TRY(pack_elements<double>(ctx, m, Ae, Ap, s));
  const size_t vb = (size_t)n * ld * sizeof(double);
  double* R = (double*)scratch(ctx, S_R64, vb, &err);
  double* Z = (double*)scratch(ctx, S_Z64, vb, &err);
  double* P = (double*)scratch(ctx, S_P64, vb, &err);
  double* Q = (double*)scratch(ctx, S_Q64, vb, &err);
  double* sc = (double*)scratch(ctx, S_SCAL, 8 * MK_MAX_RHS * sizeof(double) + MK_MAX_RHS * sizeof(ColState), &err);
  if (!R || !Z || !P || !Q || !sc) return err;
  double *d1 = sc, *d2 = sc + MK_MAX_RHS, *d3 = sc + 2 * MK_MAX_RHS;
  ColState* st = (ColState*)(sc + 8 * MK_MAX_RHS);
  const int th = 256;
  const int gb = (int)((n * ld + th - 1) / th);
  // host mirror of the column states
  if (ctx->pinned_size < sizeof(ColState) * MK_MAX_RHS) {
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    MK_CUDA(cudaMallocHost(&ctx->pinned, sizeof(ColState) * MK_MAX_RHS * 2));
    ctx->pinned_size = sizeof(ColState) * MK_MAX_RHS * 2;
  }
  ColState* hst = (ColState*)ctx->pinned;
  const bool cheb = o.precond == MK_PRECOND_CHEBYSHEV;
  double* CR = nullptr;   // Chebyshev: its residual, direction and operator product
  double* CD = nullptr;
  double* CQ = nullptr;
  ChebCoef cc{};
  if (cheb) {
    CR = (double*)scratch(ctx, S_VEC1, vb, &err);
    CD = (double*)scratch(ctx, S_VEC2, vb, &err);
    CQ = (double*)scratch(ctx, S_VEC3, vb, &err);
    if (!CR || !CD || !CQ) return err;
    // the interval from Lanczos on D^-1/2 A D^-1/2 (one column, in R, Z, P, Q)
    const int gn = (int)((n + 255) / 256);
    double* v = R;
    double* vp = Z;
    double* w = P;
    double* u = Q;
    MK_COUNT(), k_lz_start<<<gn, 256, 0, s>>>(n, L.d_boundary, v);
    MK_TRY(column_dots(ctx, n, v, v, 1, 1, d1, s));
    MK_COUNT(), k_scale<<<gn, 256, 0, s>>>(n, v, d1, nullptr, 0);
    MK_CUDA(cudaMemsetAsync(vp, 0, n * sizeof(double), s));
    std::vector<double> al, be;
    double beta = 0.0;
    for (int k = 0; k < kChebLanczos; ++k) {
      MK_COUNT(), k_lz_scale<<<gn, 256, 0, s>>>(n, L.d_boundary, diag, v, u, 1);   // u = D^-1/2 v
      MK_TRY(apply_patch<double>(ctx, m, Ap, u, w, 1, true, s));                      // w = A u
      MK_COUNT(), k_lz_scale<<<gn, 256, 0, s>>>(n, L.d_boundary, diag, w, w, 1);   // w = D^-1/2 A D^-1/2 v
      MK_TRY(column_dots(ctx, n, v, w, 1, 1, d2, s));
      double alpha;
      MK_CUDA(cudaMemcpyAsync(&alpha, d2, sizeof(double), cudaMemcpyDeviceToHost, s));
      MK_CUDA(cudaStreamSynchronize(s));
      MK_COUNT(), k_lanczos_w<<<gn, 256, 0, s>>>(n, L.d_boundary, w, v, vp, alpha, beta);
      MK_TRY(column_dots(ctx, n, w, w, 1, 1, d3, s));
      double bb;
      MK_CUDA(cudaMemcpyAsync(&bb, d3, sizeof(double), cudaMemcpyDeviceToHost, s));
      MK_CUDA(cudaStreamSynchronize(s));
      al.push_back(alpha);
      beta = std::sqrt(std::max(bb, 0.0));
      if (beta == 0.0 || k + 1 == kChebLanczos) break;
      be.push_back(beta);
      MK_CUDA(cudaMemcpyAsync(vp, v, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      MK_CUDA(cudaMemcpyAsync(v, w, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      MK_COUNT(), k_scale<<<gn, 256, 0, s>>>(n, v, d3, nullptr, 0);
    }
    be.resize(al.size() > 0 ? al.size() - 1 : 0);
    const double lo = tridiag_extreme(al, be, false), hi = 1.1 * tridiag_extreme(al, be, true);
    MK_ARG(lo > 0.0 && hi > lo, "Chebyshev preconditioner: the operator is not positive definite");
    cc.theta = 0.5 * (hi + lo);
    cc.delta = 0.5 * (hi - lo);
    cc.sigma1 = cc.theta / cc.delta;
  }
  // z = p(D^-1 A) D^-1 r for all columns (Chebyshev)
  auto cheb_apply = [&](const double* r, double* z) -> int {
    MK_COUNT(), k_copy_cols<<<gb, th, 0, s>>>(n, r, CR, ld);
    double rho = 1.0 / cc.sigma1;
    MK_COUNT(), k_cheb_step<<<gb, th, 0, s>>>(n, L.d_boundary, diag, CR, CQ, CD, z, N, ld, 0.0, 1.0 / cc.theta, 1);
    for (int k = 1; k < kChebDegree; ++k) {
      MK_TRY(apply_patch<double>(ctx, m, Ap, CD, CQ, ld, true, s));
      const double rho_new = 1.0 / (2.0 * cc.sigma1 - rho);
      MK_COUNT(), k_cheb_step<<<gb, th, 0, s>>>(n, L.d_boundary, diag, CR, CQ, CD, z, N, ld, rho_new * rho,
                                                2.0 * rho_new / cc.delta, 0);
      rho = rho_new;
    }
    return MK_OK;
  };

  MK_TRY(apply_patch<double>(ctx, m, Ap, x, Q, ld, true, s));
  MK_COUNT(), k_residual<<<gb, th, 0, s>>>(n, L.d_boundary, b, Q, diag, R, Z, P, N, ld);
  if (cheb) {
    MK_TRY(cheb_apply(R, Z));
    MK_COUNT(), k_copy_cols<<<gb, th, 0, s>>>(n, Z, P, ld);
  }
  // x boundary rows to 0 (Q := 0 then mask trick): write x = x - 0 on interior, 0 on boundary
  MK_TRY(column_dots(ctx, n, b, b, N, ld, d1, s));
  MK_TRY(column_dots(ctx, n, R, Z, N, ld, d2, s));
  MK_TRY(column_dots(ctx, n, R, R, N, ld, d3, s));
  MK_COUNT(), k_init_state<<<1, MK_MAX_RHS, 0, s>>>(st, d1, d2, d3, N, o.rtol);
  const int check = std::max(1, o.check_every);
  int it = 0, status = MK_OK;
  bool any_active = true;
  MK_CUDA(cudaMemcpyAsync(hst, st, sizeof(ColState) * N, cudaMemcpyDeviceToHost, s));
  MK_CUDA(cudaStreamSynchronize(s));
  any_active = false;
  for (int j = 0; j < N; ++j) any_active |= hst[j].active != 0;
  int ntr = 0;
  const bool trace = o.trace_cap > 0 && o.trace_every > 0 && o.trace_x && o.trace_r;
  while (any_active && it < o.maxit) {
    if (trace && it % o.trace_every == 0 && ntr < o.trace_cap) {  // training data of the learned preconditioner
      MK_CUDA(cudaMemcpyAsync(o.trace_x + (size_t)ntr * n * ld, x, vb, cudaMemcpyDeviceToDevice, s));
      MK_CUDA(cudaMemcpyAsync(o.trace_r + (size_t)ntr * n * ld, R, vb, cudaMemcpyDeviceToDevice, s));
      ++ntr;
    }
    MK_TRY(apply_patch<double>(ctx, m, Ap, P, Q, ld, true, s));
    MK_TRY(column_dots(ctx, n, P, Q, N, ld, d1, s));
    MK_COUNT(), k_alpha<<<1, MK_MAX_RHS, 0, s>>>(st, d1, N);
    MK_COUNT(), k_update<<<gb, th, 0, s>>>(n, st, P, Q, diag, x, R, Z, N, ld);
    if (cheb) MK_TRY(cheb_apply(R, Z));
    MK_TRY(column_dots(ctx, n, R, Z, N, ld, d2, s));
    MK_TRY(column_dots(ctx, n, R, R, N, ld, d3, s));
    MK_COUNT(), k_beta<<<1, MK_MAX_RHS, 0, s>>>(st, d2, d3, N, o.rtol);
    MK_COUNT(), k_pupdate<<<gb, th, 0, s>>>(n, st, Z, P, N, ld);
    ++it;
    if (it % check == 0 || it >= o.maxit) {
      MK_CUDA(cudaMemcpyAsync(hst, st, sizeof(ColState) * N, cudaMemcpyDeviceToHost, s));
      MK_CUDA(cudaStreamSynchronize(s));
      any_active = false;
      for (int j = 0; j < N; ++j) {
        any_active |= hst[j].active != 0;
        if (hst[j].breakdown) status = MK_ERR_BREAKDOWN;
      }
      if (status == MK_ERR_BREAKDOWN) break;
    }
  }
  MK_CUDA(cudaGetLastError());
  // final FP64 true residual
  MK_TRY(apply_patch<double>(ctx, m, Ap, x, Q, ld, true, s));
  MK_COUNT(), k_residual<<<gb, th, 0, s>>>(n, L.d_boundary, b, Q, diag, R, nullptr, nullptr, N, ld);
  MK_TRY(column_dots(ctx, n, R, R, N, ld, d3, s));
  MK_CUDA(cudaMemcpyAsync(hst, st, sizeof(ColState) * N, cudaMemcpyDeviceToHost, s));
  double rr[MK_MAX_RHS];
  MK_CUDA(cudaMemcpyAsync(rr, d3, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  MK_CUDA(cudaStreamSynchronize(s));
  MK_TRY(check_fault(ctx, s));
  if (rep) {
    std::memset(rep, 0, sizeof(*rep));
    rep->n_rhs = N;
    rep->iterations = it;
    double mx = 0.0;
    for (int j = 0; j < N; ++j) {
      rep->iters[j] = hst[j].iters;
      rep->rel_residual[j] = std::sqrt(rr[j]) / hst[j].bn;
      mx = std::max(mx, rep->rel_residual[j]);
    }
    rep->max_rel_residual = mx;
    rep->n_traced = ntr;
  }
  double mx = 0.0;
  for (int j = 0; j < N; ++j) mx = std::max(mx, std::sqrt(rr[j]) / hst[j].bn);
  if (status == MK_OK && !(mx <= o.rtol)) status = MK_ERR_NOT_CONVERGED;
  if (rep) rep->status = status;
  if (status == MK_ERR_BREAKDOWN) return fail(status, "PCG breakdown: p^T A p <= 0 (operator not positive definite)");
  if (status == MK_ERR_NOT_CONVERGED) return fail(status, "PCG did not reach rtol within maxit");
  return MK_OK;
}

static bool valid_opts(const mk_solve_opts* o) {
  if (!o || !(o->rtol > 0) || o->maxit <= 0 || o->coarse < 0 || o->coarse > 2) return false;
  if (o->coarse && o->precision != MK_PREC_MIXED) return false;
  if (o->precond == MK_PRECOND_LEARNED)
    return o->precision == MK_PREC_MIXED && o->mlp != nullptr &&
           (o->mlp_precision == MK_MLP_FP32 || o->mlp_precision == MK_MLP_BF16);
  if (o->precond == MK_PRECOND_CHEBYSHEV) return o->precision == MK_PREC_FP64;
  return o->precond == MK_PRECOND_JACOBI;
}

__global__ void k_combine_rhs(int64_t n, const uint8_t* __restrict__ bnd, const double* __restrict__ Mu,
                              const double* __restrict__ Vu, const ColParams coef, double* __restrict__ rhs,
                              int N, int ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ld) return;
  const int64_t nd = t / ld;
  const int j = (int)(t % ld);
  rhs[t] = (j < N && !bnd[nd]) ? coef.v[j] * Mu[t] - Vu[t] : 0.0;
}

__global__ void k_axpy_interior(int64_t n, const uint8_t* __restrict__ bnd, const double* __restrict__ d,
                                double* __restrict__ w) {
  const int64_t nd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (nd >= n || bnd[nd]) return;
  w[nd] += d[nd];
}

__global__ void k_scatter_free(int64_t nf, const int32_t* __restrict__ free_idx, const double* __restrict__ src,
                               double* __restrict__ dst) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nf) dst[free_idx[k]] = src[k];
}

}  // namespace mk

using namespace mk;

extern "C" {

int mk_prolongate(mk_ctx* ctx, const mk_mesh* m, const double* psiH, int ldc, int N, double* u, int ld,
                  void* stream) {
  MK_ARG(ctx && m && psiH && u, "mk_prolongate: null argument");
  MK_ARG(N >= 1 && N <= ld && N <= ldc && N <= MK_MAX_RHS, "mk_prolongate: bad N/ld");
  MK_CUDA(cudaSetDevice(ctx->device));
  return prolongate(ctx, m, psiH, ldc, N, u, ld, (cudaStream_t)stream);
}

int mk_density(mk_ctx* ctx, const mk_mesh* m, const double* u, int ld, const double* occ, int N, double* rho_q,
               void* stream) {
  MK_ARG(ctx && m && u && occ && rho_q, "mk_density: null argument");
  MK_ARG(N >= 1 && N <= ld && N <= MK_MAX_RHS, "mk_density: bad N/ld");
  MK_CUDA(cudaSetDevice(ctx->device));
  MK_TRY(density(ctx, m->fine, u, ld, N, occ, rho_q, (cudaStream_t)stream));
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

int mk_hartree_poisson(mk_ctx* ctx, const mk_mesh* m, const double* u, int ld, const double* occ, int N,
                       const double* rho_q, int bc, double* w, const mk_solve_opts* opts, mk_solve_report* report,
                       void* stream) {
  MK_ARG(ctx && m && u && occ && w, "mk_hartree_poisson: null argument");
  MK_ARG(N >= 1 && N <= ld && N <= MK_MAX_RHS, "mk_hartree_poisson: bad N/ld");
  MK_ARG(bc == MK_BC_ZERO || bc == MK_BC_MULTIPOLE, "mk_hartree_poisson: bad bc");
  MK_ARG(valid_opts(opts), "mk_hartree_poisson: bad opts");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const Level& L = m->fine;
  int err = MK_OK;
  double* rho_own = rho_q ? nullptr : (double*)scratch(ctx, S_RHO, (size_t)L.n_elems * kQ * sizeof(double), &err);
  const double* rho = rho_q ? rho_q : rho_own;
  double* F = (double*)scratch(ctx, S_VEC1, L.n_nodes * sizeof(double), &err);
  double* y = (double*)scratch(ctx, S_VEC2, L.n_nodes * sizeof(double), &err);
  double* d = (double*)scratch(ctx, S_VEC3, L.n_nodes * sizeof(double), &err);
  double* diag = (double*)scratch(ctx, S_DIAG64, L.n_nodes * sizeof(double), &err);
  if (!rho || !F || !y || !d || !diag) return err;
  // K and its diagonal depend on the mesh only: built on the first call, kept in the mesh handle
  if (!m->d_K64) {
    const size_t kb = (size_t)L.n_elems * (L.nloc * (L.nloc + 1) / 2) * sizeof(double);
    if (cudaMalloc(&m->d_K64, kb) != cudaSuccess || cudaMalloc(&m->d_K64diag, L.n_nodes * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(MK_ERR_OOM, "mk_hartree_poisson: stiffness allocation failed");
    }
    MK_TRY(element_matrices(ctx, L, nullptr, 1.0, 0.0, 0.0, nullptr, m->d_K64, s));
    MK_TRY(assemble_diagonal(ctx, L, m->d_K64, m->d_K64diag, s));
  }
  const double* Ke = m->d_K64;
  MK_CUDA(cudaMemcpyAsync(diag, m->d_K64diag, L.n_nodes * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (!rho_q) MK_TRY(density(ctx, L, u, ld, N, occ, rho_own, s));
  MK_TRY(load_vector(ctx, L, rho, 4.0 * M_PI, F, s));
  MK_TRY(multipole_boundary(ctx, L, rho, L.d_nodes, bc, w, s));
  MK_TRY(apply64(ctx, m, Ke, w, y, 1, 1, true, s));                     // K_IB g (interior rows)
  ColParams coef{};
  coef.v[0] = 1.0;
  MK_COUNT(), k_combine_rhs<<<(int)((L.n_nodes + 255) / 256), 256, 0, s>>>(L.n_nodes, L.d_boundary, F, y, coef, F, 1, 1);
  MK_CUDA(cudaMemsetAsync(d, 0, L.n_nodes * sizeof(double), s));
  const float* cinv = nullptr;
  MK_ARG(opts->coarse != 2 || m->has_mg, "mk_hartree_poisson: multigrid needs the mesh hierarchy (mk_mesh_set_hierarchy)");
  if (opts->precision == MK_PREC_MIXED && opts->coarse) {  // two-level or multigrid: the inverse of P^T K P on V_H
    MK_TRY(tl_prepare(m, s));
    cinv = coarse_inverse_cached(ctx, m, Ke, nullptr, s, &err);
    if (!cinv) return err;
  }
  int r = opts->precision == MK_PREC_MIXED ? pcg_mixed(ctx, m, Ke, F, d, 1, 1, *opts, report, s, cinv, true, diag)
                                           : pcg64(ctx, m, Ke, diag, F, d, 1, 1, *opts, report, s);
  MK_COUNT(), k_axpy_interior<<<(int)((L.n_nodes + 255) / 256), 256, 0, s>>>(L.n_nodes, L.d_boundary, d, w);
  MK_CUDA(cudaGetLastError());
  MK_CUDA(cudaStreamSynchronize(s));
  return r;
}

int mk_frozen_potential(mk_ctx* ctx, const mk_mesh* m, const double* u, int ld, const double* occ, int N,
                        const double* rho_q, const double* w, mk_xc xc, double* vq, void* stream) {
  MK_ARG(ctx && m && u && occ && w && vq, "mk_frozen_potential: null argument");
  MK_ARG(N >= 1 && N <= ld && N <= MK_MAX_RHS, "mk_frozen_potential: bad N/ld");
  MK_ARG(xc.kind >= MK_XC_NONE && xc.kind <= MK_XC_LDA_PZ, "mk_frozen_potential: bad xc");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const Level& L = m->fine;
  int err = MK_OK;
  const double* rho = rho_q;
  if (!rho) {
    double* own = (double*)scratch(ctx, S_RHO, (size_t)L.n_elems * kQ * sizeof(double), &err);
    if (!own) return err;
    MK_TRY(density(ctx, L, u, ld, N, occ, own, s));
    rho = own;
  }
  MK_TRY(frozen_potential(ctx, L, w, rho, xc, vq, s));
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

int mk_assemble_rhs_from_vq(mk_ctx* ctx, const mk_mesh* m, const double* u, int ld, const double* lambdaH, int N,
                            const double* vq, double sigma, double* rhs, void* stream) {
  MK_ARG(ctx && m && u && lambdaH && vq && rhs, "mk_assemble_rhs_from_vq: null argument");
  MK_ARG(N >= 1 && N <= ld && N <= MK_MAX_RHS, "mk_assemble_rhs_from_vq: bad N/ld");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const Level& L = m->fine;
  int err = MK_OK;
  const size_t eb = (size_t)L.n_elems * (L.nloc * (L.nloc + 1) / 2) * sizeof(double);
  double* Ve = (double*)scratch(ctx, S_ELEM64, eb, &err);
  double* Mu = (double*)scratch(ctx, S_VEC1, (size_t)L.n_nodes * ld * sizeof(double), &err);
  double* Vu = (double*)scratch(ctx, S_VEC2, (size_t)L.n_nodes * ld * sizeof(double), &err);
  if (!Ve || !Mu || !Vu) return err;
  const double* Me = mass_matrices(ctx, m, s, &err);
  if (!Me) return err;
  MK_TRY(element_matrices(ctx, L, nullptr, 0.0, 0.0, 0.0, vq, Ve, s));
  MK_TRY(apply64(ctx, m, Me, u, Mu, N, ld, true, s));
  MK_TRY(apply64(ctx, m, Ve, u, Vu, N, ld, true, s));
  ColParams coef{};
  for (int j = 0; j < N; ++j) coef.v[j] = lambdaH[j] + sigma;
  MK_COUNT(), k_combine_rhs<<<(int)((L.n_nodes * ld + 255) / 256), 256, 0, s>>>(L.n_nodes, L.d_boundary, Mu, Vu, coef, rhs, N, ld);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

int mk_assemble_rhs(mk_ctx* ctx, const mk_mesh* m, const double* u, int ld, const double* lambdaH,
                    const double* occ, int N, const double* w, double sigma, mk_xc xc, double* rhs, double* vq,
                    void* stream) {
  MK_ARG(ctx && m && u && lambdaH && occ && rhs && vq, "mk_assemble_rhs: null argument");
  MK_TRY(mk_frozen_potential(ctx, m, u, ld, occ, N, nullptr, w, xc, vq, stream));
  return mk_assemble_rhs_from_vq(ctx, m, u, ld, lambdaH, N, vq, sigma, rhs, stream);
}

int mk_correction_solve(mk_ctx* ctx, const mk_mesh* m, const mk_molecule* mol, double sigma, const double* rhs,
                        double* x, int ld, int N, const mk_solve_opts* opts, mk_solve_report* report,
                        void* stream) {
  MK_ARG(ctx && m && mol && rhs && x, "mk_correction_solve: null argument");
  MK_ARG(N >= 1 && N <= ld && N <= MK_MAX_RHS, "mk_correction_solve: bad N/ld");
  MK_ARG(valid_opts(opts), "mk_correction_solve: bad opts");
  MK_ARG(opts->coarse != 2, "mk_correction_solve: multigrid is for the Hartree Poisson solve");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const Level& L = m->fine;
  if (opts->precision == MK_PREC_MIXED) {
    return solve_mixed(ctx, m, mol, sigma, rhs, nullptr, nullptr, x, ld, N, *opts, report, s);
  }
  MK_ARG(opts->precision == MK_PREC_FP64, "mk_correction_solve: bad precision");

  int err = MK_OK;
  double* Ae = (double*)scratch(ctx, S_ELEM64, (size_t)L.n_elems * (L.nloc * (L.nloc + 1) / 2) * sizeof(double), &err);
  double* diag = (double*)scratch(ctx, S_DIAG64, L.n_nodes * sizeof(double), &err);
  if (!Ae || !diag) return err;
  const double* H0 = static_matrices(ctx, m, mol, s, &err);
  if (!H0) return err;
  MK_TRY(element_matrices(ctx, L, nullptr, 0.0, 0.0, sigma, nullptr, Ae, s, H0));
  MK_TRY(assemble_diagonal(ctx, L, Ae, diag, s));
  return pcg64(ctx, m, Ae, diag, rhs, x, N, ld, *opts, report, s);
}

int mk_correction_solve_vq(mk_ctx* ctx, const mk_mesh* m, const mk_molecule* mol, const double* vq, double sigma,
                           const double* rhs, double* x, int ld, int N, const mk_solve_opts* opts,
                           mk_solve_report* report, void* stream) {
  MK_ARG(ctx && m && mol && vq && rhs && x, "mk_correction_solve_vq: null argument");
  MK_ARG(N >= 1 && N <= ld && N <= MK_MAX_RHS, "mk_correction_solve_vq: bad N/ld");
  MK_ARG(valid_opts(opts), "mk_correction_solve_vq: bad opts");
  MK_ARG(opts->coarse == 0, "mk_correction_solve_vq: no coarse preconditioner with a potential in the operator");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const Level& L = m->fine;
  if (opts->precision == MK_PREC_MIXED)
    return solve_mixed(ctx, m, mol, sigma, rhs, vq, nullptr, x, ld, N, *opts, report, s);
  MK_ARG(opts->precision == MK_PREC_FP64, "mk_correction_solve_vq: bad precision");
  int err = MK_OK;
  double* Ae = (double*)scratch(ctx, S_ELEM64, (size_t)L.n_elems * (L.nloc * (L.nloc + 1) / 2) * sizeof(double), &err);
  double* diag = (double*)scratch(ctx, S_DIAG64, L.n_nodes * sizeof(double), &err);
  if (!Ae || !diag) return err;
  const double* H0 = static_matrices(ctx, m, mol, s, &err);
  if (!H0) return err;
  MK_TRY(element_matrices(ctx, L, nullptr, 0.0, 0.0, sigma, vq, Ae, s, H0));
  MK_TRY(assemble_diagonal(ctx, L, Ae, diag, s));
  return pcg64(ctx, m, Ae, diag, rhs, x, N, ld, *opts, report, s);
}

int mk_lowest_ritz(mk_ctx* ctx, const mk_mesh* m, const mk_molecule* mol, const double* v0, int steps,
                   double* theta, void* stream) {
  MK_ARG(ctx && m && mol && v0 && theta && steps >= 1, "mk_lowest_ritz: bad argument");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const Level& L = m->fine;
  const int64_t n = L.n_nodes;
  int err = MK_OK;
  const size_t eb = (size_t)L.n_elems * (L.nloc * (L.nloc + 1) / 2) * sizeof(double);
  double* He = (double*)scratch(ctx, S_ELEM64B, eb, &err);
  double* Me = (double*)scratch(ctx, S_ELEM64, eb, &err);
  double* diagM = (double*)scratch(ctx, S_DIAG64, n * sizeof(double), &err);
  double* v = (double*)scratch(ctx, S_VEC1, n * sizeof(double), &err);
  double* vp = (double*)scratch(ctx, S_VEC2, n * sizeof(double), &err);
  double* Hv = (double*)scratch(ctx, S_VEC3, n * sizeof(double), &err);
  double* w = (double*)scratch(ctx, S_VEC4, n * sizeof(double), &err);
  double* Mw = (double*)scratch(ctx, S_VEC5, n * sizeof(double), &err);
  double* dd = (double*)scratch(ctx, S_COEF, 64 * sizeof(double), &err);
  if (!He || !Me || !diagM || !v || !vp || !Hv || !w || !Mw || !dd) return err;
  MK_TRY(element_matrices(ctx, L, mol, 0.5, 1.0, 0.0, nullptr, He, s));
  MK_TRY(element_matrices(ctx, L, nullptr, 0.0, 0.0, 1.0, nullptr, Me, s));
  MK_TRY(assemble_diagonal(ctx, L, Me, diagM, s));
  MK_CUDA(cudaMemsetAsync(v, 0, n * sizeof(double), s));
  MK_CUDA(cudaMemsetAsync(vp, 0, n * sizeof(double), s));
  double* v0d = Mw;
  MK_CUDA(cudaMemcpyAsync(v0d, v0, L.n_free * sizeof(double), cudaMemcpyHostToDevice, s));
  MK_CUDA(cudaStreamSynchronize(s));
  MK_COUNT(), k_scatter_free<<<(int)((L.n_free + 255) / 256), 256, 0, s>>>(L.n_free, L.d_free_idx, v0d, v);
  MK_TRY(apply64(ctx, m, Me, v, Mw, 1, 1, true, s));
  MK_TRY(column_dots(ctx, n, v, Mw, 1, 1, dd, s));
  MK_COUNT(), k_scale<<<(int)((n + 255) / 256), 256, 0, s>>>(n, v, dd, nullptr, 0);
  mk_solve_opts mo{MK_PREC_FP64, MK_PRECOND_JACOBI, 1e-12, 5000, 0, 0, 25};
  std::vector<double> a, b;
  double beta = 0.0;
  for (int k = 0; k < steps; ++k) {
    MK_TRY(apply64(ctx, m, He, v, Hv, 1, 1, true, s));
    MK_TRY(column_dots(ctx, n, v, Hv, 1, 1, dd, s));
    double alpha;
    MK_CUDA(cudaMemcpyAsync(&alpha, dd, sizeof(double), cudaMemcpyDeviceToHost, s));
    MK_CUDA(cudaMemsetAsync(w, 0, n * sizeof(double), s));
    MK_CUDA(cudaStreamSynchronize(s));
    MK_TRY(pcg64(ctx, m, Me, diagM, Hv, w, 1, 1, mo, nullptr, s));   // w = M^-1 H v
    MK_COUNT(), k_lanczos_w<<<(int)((n + 255) / 256), 256, 0, s>>>(n, L.d_boundary, w, v, vp, alpha, beta);
    MK_TRY(apply64(ctx, m, Me, w, Mw, 1, 1, true, s));
    MK_TRY(column_dots(ctx, n, w, Mw, 1, 1, dd, s));
    double bb;
    MK_CUDA(cudaMemcpyAsync(&bb, dd, sizeof(double), cudaMemcpyDeviceToHost, s));
    MK_CUDA(cudaStreamSynchronize(s));
    a.push_back(alpha);
    beta = std::sqrt(std::max(bb, 0.0));
    if (beta == 0.0 || k + 1 == steps) break;
    b.push_back(beta);
    MK_CUDA(cudaMemcpyAsync(vp, v, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    MK_CUDA(cudaMemcpyAsync(v, w, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    MK_COUNT(), k_scale<<<(int)((n + 255) / 256), 256, 0, s>>>(n, v, dd, nullptr, 0);
  }
  b.resize(a.size() > 0 ? a.size() - 1 : 0);
  *theta = tridiag_extreme(a, b, false);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

int mk_correction_shift(mk_ctx* ctx, const mk_mesh* m, const mk_molecule* mol, const double* v0, int steps,
                        double* theta, double* sigma, void* stream) {
  MK_ARG(sigma, "mk_correction_shift: null sigma");
  double th = 0.0;
  MK_TRY(mk_lowest_ritz(ctx, m, mol, v0, steps, &th, stream));
  if (theta) *theta = th;
  *sigma = 1.05 * std::max(0.0, -th) + 0.5;
  return MK_OK;
}

}  // extern "C"
