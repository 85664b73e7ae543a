// Host side of the mk library: errors, context, scratch, reference-element tables and mesh preprocessing (A0).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>

#include "mk_internal.h"

namespace mk {

static thread_local std::string g_err;
std::atomic<long long> g_launch_count{0};

void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int check_fault(mk_ctx* c, cudaStream_t s) {
  int f = 0;
  MK_CUDA(cudaMemcpyAsync(&f, c->d_fault, sizeof(int), cudaMemcpyDeviceToHost, s));
  MK_CUDA(cudaStreamSynchronize(s));
  if (f) return fail(MK_ERR_TIMEOUT, "a bounded device-side wait gave up (fault word " + std::to_string(f) + ")");
  return MK_OK;
}

// ------------------------------------------------------------------------------------------------ quadrature
// Jacobi polynomial P_n^{(a,b)}(x) and its derivative by the three-term recurrence.
static void jacobi_eval(int n, double a, double b, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = 0.5 * (a - b + (a + b + 2.0) * x);
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  // derivative: d/dx P_n^{(a,b)} = (n+a+b+1)/2 P_{n-1}^{(a+1,b+1)}
  auto raw = [](int n, double a, double b, double x) {
    double q0 = 1.0, q1 = 0.5 * (a - b + (a + b + 2.0) * x);
    if (n == 0) return q0;
    for (int k = 2; k <= n; ++k) {
      double s = 2.0 * k + a + b;
      double c1 = 2.0 * k * (k + a + b) * (s - 2.0);
      double c2 = (s - 1.0) * (s * (s - 2.0) * x + a * a - b * b);
      double c3 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * s;
      double q2 = (c2 * q1 - c3 * q0) / c1;
      q0 = q1;
      q1 = q2;
    }
    return q1;
  };
  (void)p0; (void)p1;
  *p = raw(n, a, b, x);
  *dp = (n == 0) ? 0.0 : 0.5 * (n + a + b + 1.0) * raw(n - 1, a + 1.0, b + 1.0, x);
}

// n-point Gauss-Jacobi rule on [-1,1] for (1-x)^a (1+x)^b: Newton iteration on P_n with deflation of the roots
// already found, weights from w_i = C / ((1 - x_i^2) P_n'(x_i)^2).
void gauss_jacobi_newton(int n, double a, double b, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double r = -std::cos((2.0 * i + 1.0) * M_PI / (2.0 * n));  // Chebyshev guess, ascending
    if (i > 0 && r <= x[i - 1]) r = x[i - 1] + 1e-3;
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      jacobi_eval(n, a, b, r, &p, &dp);
      double s = 0.0;
      for (int j = 0; j < i; ++j) s += 1.0 / (r - x[j]);
      double delta = p / (dp - s * p);
      r -= delta;
      if (std::fabs(delta) < 1e-16 * std::max(1.0, std::fabs(r))) break;
    }
    x[i] = r;
  }
  double C = std::exp(std::lgamma(n + a + 1.0) + std::lgamma(n + b + 1.0) - std::lgamma(n + a + b + 1.0) -
                      std::lgamma(n + 1.0)) *
             std::pow(2.0, a + b + 1.0);
  for (int i = 0; i < n; ++i) {
    double p, dp;
    jacobi_eval(n, a, b, x[i], &p, &dp);
    w[i] = C / ((1.0 - x[i] * x[i]) * dp * dp);
  }
}

static const int kEdgeA[6] = {0, 0, 0, 1, 1, 2};
static const int kEdgeB[6] = {1, 2, 3, 2, 3, 3};

static void basis_host(int order, const double lam[4], double* phi, double (*dphi)[3]) {
  static const double G[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  if (order == 1) {
    for (int a = 0; a < 4; ++a) {
      phi[a] = lam[a];
      if (dphi) for (int k = 0; k < 3; ++k) dphi[a][k] = G[a][k];
    }
    return;
  }
  for (int a = 0; a < 4; ++a) {
    phi[a] = lam[a] * (2.0 * lam[a] - 1.0);
    if (dphi) for (int k = 0; k < 3; ++k) dphi[a][k] = (4.0 * lam[a] - 1.0) * G[a][k];
  }
  for (int e = 0; e < 6; ++e) {
    int a = kEdgeA[e], b = kEdgeB[e];
    phi[4 + e] = 4.0 * lam[a] * lam[b];
    if (dphi) for (int k = 0; k < 3; ++k) dphi[4 + e][k] = 4.0 * (lam[b] * G[a][k] + lam[a] * G[b][k]);
  }
}

void build_ref_tables(int order, RefTables* t) {
  std::memset(t, 0, sizeof(*t));
  t->order = order;
  t->nloc = order == 1 ? 4 : 10;
  t->npack = t->nloc * (t->nloc + 1) / 2;
  double u[3], wu[3], v[3], wv[3], s[3], ws[3];
  gauss_jacobi_newton(3, 2.0, 0.0, u, wu);
  gauss_jacobi_newton(3, 1.0, 0.0, v, wv);
  gauss_jacobi_newton(3, 0.0, 0.0, s, ws);
  for (int i = 0; i < 3; ++i) {  // map to [0,1] with weight (1-x)^a
    u[i] = 0.5 * (1.0 + u[i]); wu[i] *= std::pow(2.0, -3.0);
    v[i] = 0.5 * (1.0 + v[i]); wv[i] *= std::pow(2.0, -2.0);
    s[i] = 0.5 * (1.0 + s[i]); ws[i] *= 0.5;
  }
  int q = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k, ++q) {
        t->qx[q][0] = u[i];
        t->qx[q][1] = v[j] * (1.0 - u[i]);
        t->qx[q][2] = s[k] * (1.0 - u[i]) * (1.0 - v[j]);
        t->qw[q] = wu[i] * wv[j] * ws[k];
      }
  const int n = t->nloc;
  static const int I6[6] = {0, 1, 2, 0, 0, 1}, J6[6] = {0, 1, 2, 1, 2, 2};
  for (q = 0; q < kQ; ++q) {
    double lam[4] = {1.0 - t->qx[q][0] - t->qx[q][1] - t->qx[q][2], t->qx[q][0], t->qx[q][1], t->qx[q][2]};
    double phi[kMaxLoc], dphi[kMaxLoc][3];
    basis_host(order, lam, phi, dphi);
    for (int a = 0; a < n; ++a) t->phi[q][a] = phi[a];
    for (int a = 0; a < n; ++a)
      for (int b = a; b < n; ++b) {
        int p = sym_index(a, b, n);
        t->mass[p] += t->qw[q] * phi[a] * phi[b];
        for (int c = 0; c < 6; ++c) {
          int i = I6[c], j = J6[c];
          double v2 = dphi[a][i] * dphi[b][j];
          if (i != j) v2 += dphi[a][j] * dphi[b][i];
          t->stiff[c][p] += t->qw[q] * v2;
        }
      }
  }
  for (int a = 0; a < 4; ++a) t->node_bary[a][a] = 1.0;
  if (order == 2)
    for (int e = 0; e < 6; ++e) {
      t->node_bary[4 + e][kEdgeA[e]] = 0.5;
      t->node_bary[4 + e][kEdgeB[e]] = 0.5;
    }
}

// ------------------------------------------------------------------------------------------------ profiling
void prof_capture(mk_ctx* ctx, bool on) {
  ctx->capturing = on;
  if (on)
    for (int k = 0; k < kProfKinds; ++k) ctx->cap_n[k] = 0;
}

// The event pool of graph captures; made before any capture starts (nothing is created inside one).
void prof_prepare_capture(mk_ctx* ctx) {
  if (!ctx->prof_on) return;
  for (auto& pool : ctx->cap_ev)
    while (pool.size() < 2 * (size_t)kCapPairs) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return; }
      pool.push_back(e);
    }
}

// After a replay of the captured graph (its stream synchronised): adds every timed application of the replay.
void prof_harvest(mk_ctx* ctx) {
  if (!ctx->prof_on) return;
  for (int k = 0; k < kProfKinds; ++k)
    for (int i = 0; i < ctx->cap_n[k]; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ctx->cap_ev[k][2 * i], ctx->cap_ev[k][2 * i + 1]) == cudaSuccess) {
        ctx->acc_ms[k] += ms;
        ctx->acc_n[k] += 1;
      } else {
        cudaGetLastError();
      }
    }
}

void prof_mark(mk_ctx* ctx, int kind, bool begin, cudaStream_t s) {
  if (!ctx->prof_on) return;
  if (ctx->capturing) {
    int& n = ctx->cap_n[kind];
    const size_t idx = 2 * (size_t)n + (begin ? 0 : 1);
    if (idx >= ctx->cap_ev[kind].size()) return;  // pool exhausted: this application goes untimed
    // an external record node: the graph records the event again on every replay (a plain record during capture
    // only marks a position for cross-stream dependencies)
    cudaEventRecordWithFlags(ctx->cap_ev[kind][idx], s, cudaEventRecordExternal);
    if (!begin) ++n;
    return;
  }
  auto& ev = ctx->prof_ev[kind];
  int& used = ctx->prof_used[kind];
  const size_t idx = 2 * (size_t)used + (begin ? 0 : 1);
  if (idx >= ev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    ev.push_back(e);
  }
  cudaEventRecord(ev[idx], s);
  if (!begin) ++used;
}

// ------------------------------------------------------------------------------------------------ scratch
void* scratch(mk_ctx* ctx, int slot, size_t bytes, int* err) {
  if ((int)ctx->slot_ptr.size() < S_COUNT) {
    ctx->slot_ptr.assign(S_COUNT, nullptr);
    ctx->slot_size.assign(S_COUNT, 0);
  }
  if (bytes == 0) bytes = 16;
  if (ctx->slot_size[slot] >= bytes) return ctx->slot_ptr[slot];
  if (ctx->slot_ptr[slot]) {
    cudaDeviceSynchronize();  // growth is rare; make sure no in-flight work still uses the old buffer
    cudaFree(ctx->slot_ptr[slot]);
    ctx->slot_ptr[slot] = nullptr;
    ctx->slot_size[slot] = 0;
  }
  size_t want = (bytes + 255) / 256 * 256;
  void* p = nullptr;
  if (cudaMalloc(&p, want) != cudaSuccess) {
    cudaGetLastError();
    *err = fail(MK_ERR_OOM, "scratch allocation of " + std::to_string(want) + " bytes failed");
    return nullptr;
  }
  ctx->slot_ptr[slot] = p;
  ctx->slot_size[slot] = want;
  return p;
}

// ------------------------------------------------------------------------------------------------ mesh (A0)
static double det3(const double* J) {
  return J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) + J[2] * (J[3] * J[7] - J[4] * J[6]);
}

static void inv3(const double* J, double det, double* Ji) {
  Ji[0] = (J[4] * J[8] - J[5] * J[7]) / det;
  Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
  Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
  Ji[3] = (J[5] * J[6] - J[3] * J[8]) / det;
  Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det;
  Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
  Ji[6] = (J[3] * J[7] - J[4] * J[6]) / det;
  Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
  Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
}

static int build_level(const mk_mesh_desc* d, Level& L, const char* name) {
  MK_ARG(d && d->coords && d->tets, std::string(name) + ": null mesh arrays");
  MK_ARG(d->order == 1 || d->order == 2, std::string(name) + ": order must be 1 or 2");
  MK_ARG(d->n_vertices > 0 && d->n_elems > 0 && d->n_vertices < (1LL << 30) && d->n_elems < (1LL << 30),
         std::string(name) + ": bad sizes");
  const int64_t nv = d->n_vertices, E = d->n_elems;
  L.order = d->order;
  L.nloc = d->order == 1 ? 4 : 10;
  L.n_vertices = nv;
  L.n_elems = E;
  const int nloc = L.nloc;
  for (int64_t i = 0; i < 4 * E; ++i)
    MK_ARG(d->tets[i] >= 0 && d->tets[i] < nv, std::string(name) + ": vertex index out of range");
  L.elem.assign(E * nloc, 0);
  for (int64_t e = 0; e < E; ++e)
    for (int a = 0; a < 4; ++a) L.elem[e * nloc + a] = d->tets[e * 4 + a];
  std::vector<int64_t> edge_a, edge_b;
  std::vector<uint64_t> uniq_key;     // sorted edge keys
  std::vector<int32_t> uniq_number;   // edge number of each sorted key
  if (d->order == 2) {
    const int64_t ne = 6 * E;
    std::vector<uint64_t> key(ne);
    for (int64_t e = 0; e < E; ++e)
      for (int k = 0; k < 6; ++k) {
        uint64_t a = d->tets[e * 4 + kEdgeA[k]], b = d->tets[e * 4 + kEdgeB[k]];
        if (a > b) std::swap(a, b);
        key[e * 6 + k] = a * (uint64_t)nv + b;
      }
    std::vector<int64_t> idx(ne);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) { return key[x] < key[y]; });
    std::vector<int64_t> first;  // first occurrence of each unique key (sorted by key)
    for (int64_t i = 0; i < ne; ++i)
      if (i == 0 || key[idx[i]] != key[idx[i - 1]]) {
        uniq_key.push_back(key[idx[i]]);
        first.push_back(idx[i]);
      }
    const int64_t nu = (int64_t)uniq_key.size();
    std::vector<int64_t> ord(nu);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return first[x] < first[y]; });
    uniq_number.assign(nu, 0);
    edge_a.assign(nu, 0);
    edge_b.assign(nu, 0);
    for (int64_t r = 0; r < nu; ++r) {
      uniq_number[ord[r]] = (int32_t)r;
      edge_a[r] = uniq_key[ord[r]] / nv;
      edge_b[r] = uniq_key[ord[r]] % nv;
    }
    for (int64_t i = 0, u = -1; i < ne; ++i) {
      if (i == 0 || key[idx[i]] != key[idx[i - 1]]) ++u;
      int64_t e = idx[i] / 6, k = idx[i] % 6;
      L.elem[e * nloc + 4 + k] = (int32_t)(nv + uniq_number[u]);
    }
  }
  const int64_t n_nodes = nv + (int64_t)edge_a.size();
  L.n_nodes = n_nodes;
  L.nodes.assign(n_nodes * 3, 0.0);
  for (int64_t i = 0; i < nv * 3; ++i) L.nodes[i] = d->coords[i];
  for (size_t r = 0; r < edge_a.size(); ++r)
    for (int k = 0; k < 3; ++k)
      L.nodes[(nv + r) * 3 + k] = 0.5 * (d->coords[edge_a[r] * 3 + k] + d->coords[edge_b[r] * 3 + k]);
  // boundary: faces that belong to exactly one tetrahedron
  struct Face { int32_t v[3]; };
  std::vector<Face> faces(4 * E);
  static const int F[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
  for (int64_t e = 0; e < E; ++e)
    for (int f = 0; f < 4; ++f) {
      Face x{{d->tets[e * 4 + F[f][0]], d->tets[e * 4 + F[f][1]], d->tets[e * 4 + F[f][2]]}};
      std::sort(x.v, x.v + 3);
      faces[e * 4 + f] = x;
    }
  auto lessF = [](const Face& p, const Face& q) {
    return std::lexicographical_compare(p.v, p.v + 3, q.v, q.v + 3);
  };
  std::sort(faces.begin(), faces.end(), lessF);
  L.boundary.assign(n_nodes, 0);
  for (size_t i = 0; i < faces.size();) {
    size_t j = i + 1;
    while (j < faces.size() && !lessF(faces[i], faces[j]) && !lessF(faces[j], faces[i])) ++j;
    MK_ARG(j - i <= 2, std::string(name) + ": a face is shared by more than two tetrahedra");
    if (j - i == 1) {
      const Face& f = faces[i];
      for (int k = 0; k < 3; ++k) L.boundary[f.v[k]] = 1;
      if (d->order == 2) {
        static const int P[3][2] = {{0, 1}, {0, 2}, {1, 2}};
        for (auto& pr : P) {
          uint64_t k2 = (uint64_t)f.v[pr[0]] * nv + f.v[pr[1]];
          auto it = std::lower_bound(uniq_key.begin(), uniq_key.end(), k2);
          L.boundary[nv + uniq_number[it - uniq_key.begin()]] = 1;
        }
      }
    }
    i = j;
  }
  L.node_to_free.assign(n_nodes, -1);
  L.free_idx.clear();
  for (int64_t i = 0; i < n_nodes; ++i)
    if (!L.boundary[i]) {
      L.node_to_free[i] = (int32_t)L.free_idx.size();
      L.free_idx.push_back((int32_t)i);
    }
  L.n_free = (int64_t)L.free_idx.size();
  // greedy colouring: elements in index order, smallest colour unused by earlier vertex-sharing elements
  std::vector<int64_t> vcount(nv + 1, 0);
  for (int64_t i = 0; i < 4 * E; ++i) vcount[d->tets[i] + 1]++;
  for (int64_t v = 0; v < nv; ++v) vcount[v + 1] += vcount[v];
  std::vector<int32_t> v2e(4 * E);
  {
    std::vector<int64_t> pos(vcount.begin(), vcount.end() - 1);
    for (int64_t e = 0; e < E; ++e)
      for (int a = 0; a < 4; ++a) v2e[pos[d->tets[e * 4 + a]]++] = (int32_t)e;
  }
  L.colour.assign(E, -1);
  std::vector<int64_t> stamp(256, -1);
  int ncol = 0;
  for (int64_t e = 0; e < E; ++e) {
    for (int a = 0; a < 4; ++a) {
      int32_t v = d->tets[e * 4 + a];
      for (int64_t k = vcount[v]; k < vcount[v + 1]; ++k) {
        int c = L.colour[v2e[k]];
        if (c >= 0) {
          if (c >= (int)stamp.size()) stamp.resize(2 * c + 2, -1);
          stamp[c] = e;
        }
      }
    }
    int c = 0;
    while (c < (int)stamp.size() && stamp[c] == e) ++c;
    if (c >= (int)stamp.size()) stamp.resize(2 * c + 2, -1);
    L.colour[e] = c;
    ncol = std::max(ncol, c + 1);
  }
  L.n_colours = ncol;
  L.colour_off.assign(ncol + 1, 0);
  for (int64_t e = 0; e < E; ++e) L.colour_off[L.colour[e] + 1]++;
  for (int c = 0; c < ncol; ++c) L.colour_off[c + 1] += L.colour_off[c];
  // geometry
  L.geom.resize(E);
  for (int64_t e = 0; e < E; ++e) {
    Geom& g = L.geom[e];
    const double* x0 = &d->coords[d->tets[e * 4] * 3];
    for (int c = 0; c < 3; ++c) {
      const double* xc = &d->coords[d->tets[e * 4 + c + 1] * 3];
      for (int r = 0; r < 3; ++r) g.J[r * 3 + c] = xc[r] - x0[r];
    }
    for (int r = 0; r < 3; ++r) g.x0[r] = x0[r];
    g.det = det3(g.J);
    MK_ARG(g.det > 0.0, std::string(name) + ": element " + std::to_string(e) + " has det J <= 0");
    inv3(g.J, g.det, g.Jinv);
  }
  return MK_OK;
}

template <class T>
static int upload(T** dst, const T* src, size_t n) {
  if (n == 0) n = 1;
  if (cudaMalloc(dst, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return fail(MK_ERR_OOM, "device allocation failed in mesh upload");
  }
  if (src) MK_CUDA(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
  return MK_OK;
}

static int upload_level(Level& L) {
  MK_TRY(upload(&L.d_elem, L.elem.data(), L.elem.size()));
  std::vector<int32_t> ce(L.n_elems);
  std::vector<int64_t> pos(L.colour_off.begin(), L.colour_off.end() - 1);
  for (int64_t e = 0; e < L.n_elems; ++e) ce[pos[L.colour[e]]++] = (int32_t)e;
  MK_TRY(upload(&L.d_colour_elems, ce.data(), ce.size()));
  MK_TRY(upload(&L.d_boundary, L.boundary.data(), L.boundary.size()));
  MK_TRY(upload(&L.d_free_idx, L.free_idx.data(), L.free_idx.size()));
  MK_TRY(upload(&L.d_node_to_free, L.node_to_free.data(), L.node_to_free.size()));
  MK_TRY(upload(&L.d_geom, L.geom.data(), L.geom.size()));
  MK_TRY(upload(&L.d_nodes, L.nodes.data(), L.nodes.size()));
  return MK_OK;
}

static void free_level(Level& L) {
  cudaFree(L.d_elem); cudaFree(L.d_colour_elems); cudaFree(L.d_boundary); cudaFree(L.d_free_idx);
  cudaFree(L.d_node_to_free); cudaFree(L.d_geom); cudaFree(L.d_nodes);
  L.d_nodes = nullptr;
  L.d_elem = L.d_colour_elems = L.d_free_idx = L.d_node_to_free = nullptr;
  L.d_boundary = nullptr;
  L.d_geom = nullptr;
}


// ------------------------------------------------------------------------------------------------ nested levels
// Interpolation from the coarser level C into the finer level F of a nested pair (each fine element inside its
// parent): one row per fine node, the coarse basis functions of the parent evaluated at the node (exact: V_C is a
// subspace of V_F).  Columns: the free DOF of C (free_cols) or the nodes of C, boundary nodes of C left out either
// way; entries below 1e-12 dropped.  Errors: a fine node outside its element's parent, an unused fine node.
static int build_interp(const Level& F, const Level& C, const std::vector<int32_t>& parent, bool free_cols,
                        std::vector<int32_t>& P_off, std::vector<int32_t>& P_col, std::vector<double>& P_val) {
  const int nloc = F.nloc;
  std::vector<int64_t> first(F.n_nodes, -1);
  for (int64_t i = 0; i < F.n_elems * nloc; ++i)
    if (first[F.elem[i]] < 0) first[F.elem[i]] = i;
  P_off.assign(F.n_nodes + 1, 0);
  P_col.clear();
  P_val.clear();
  for (int64_t nd = 0; nd < F.n_nodes; ++nd) {
    if (first[nd] < 0) return fail(MK_ERR_INVALID_ARG, "nested levels: unused fine node");
    const int64_t e = first[nd] / nloc;
    const int32_t T = parent[e];
    const Geom& g = C.geom[T];
    const double dx[3] = {F.nodes[nd * 3] - g.x0[0], F.nodes[nd * 3 + 1] - g.x0[1], F.nodes[nd * 3 + 2] - g.x0[2]};
    double sref[3];
    for (int rr = 0; rr < 3; ++rr)
      sref[rr] = g.Jinv[rr * 3] * dx[0] + g.Jinv[rr * 3 + 1] * dx[1] + g.Jinv[rr * 3 + 2] * dx[2];
    const double lam[4] = {1.0 - sref[0] - sref[1] - sref[2], sref[0], sref[1], sref[2]};
    for (double l : lam)
      if (l < -1e-9 || l > 1.0 + 1e-9) return fail(MK_ERR_INVALID_ARG, "nested levels: fine element outside its parent");
    double phi[kMaxLoc];
    basis_host(C.order, lam, phi, nullptr);
    for (int b = 0; b < C.nloc; ++b) {
      const int32_t cn = C.elem[(int64_t)T * C.nloc + b];
      const int32_t cf = C.node_to_free[cn];
      if (cf >= 0 && std::fabs(phi[b]) > 1e-12) {
        P_col.push_back(free_cols ? cf : cn);
        P_val.push_back(phi[b]);
      }
    }
    P_off[nd + 1] = (int32_t)P_col.size();
  }
  return MK_OK;
}

// The transpose of a CSR matrix with n_cols columns (rows of the result in column order, entries in row order).
static void transpose_csr(int64_t n_cols, const std::vector<int32_t>& off, const std::vector<int32_t>& col,
                          const std::vector<double>& val, std::vector<int32_t>& toff, std::vector<int32_t>& tcol,
                          std::vector<double>& tval) {
  const int64_t n_rows = (int64_t)off.size() - 1;
  toff.assign(n_cols + 1, 0);
  for (int32_t c : col) toff[c + 1]++;
  for (int64_t k = 0; k < n_cols; ++k) toff[k + 1] += toff[k];
  tcol.assign(col.size(), 0);
  tval.assign(col.size(), 0.0);
  std::vector<int32_t> pos(toff.begin(), toff.end() - 1);
  for (int64_t r = 0; r < n_rows; ++r)
    for (int32_t k = off[r]; k < off[r + 1]; ++k) {
      const int32_t p = pos[col[k]]++;
      tcol[p] = (int32_t)r;
      tval[p] = val[k];
    }
}

// The stiffness matrix (grad phi_a, grad phi_b) of a level on its interior nodes (node indexing; boundary rows and
// columns left out), CSR with sorted columns, and its diagonal: per element |det J| (J^-1 J^-T)_ij times the
// reference components (Sec. 2, the bilinear form of the Hartree equation).
static void stiffness_csr(const Level& L, const RefTables& R, std::vector<int32_t>& off, std::vector<int32_t>& col,
                          std::vector<double>& val, std::vector<double>& diag) {
  const int nloc = L.nloc;
  std::vector<std::pair<int64_t, double>> trip;  // key row * n + col
  trip.reserve((size_t)L.n_elems * nloc * nloc);
  const int I6[6] = {0, 1, 2, 0, 0, 1}, J6[6] = {0, 1, 2, 1, 2, 2};
  for (int64_t e = 0; e < L.n_elems; ++e) {
    const Geom& g = L.geom[e];
    double fac[6];
    for (int c = 0; c < 6; ++c)
      fac[c] = std::fabs(g.det) * (g.Jinv[I6[c] * 3] * g.Jinv[J6[c] * 3] + g.Jinv[I6[c] * 3 + 1] * g.Jinv[J6[c] * 3 + 1] +
                                   g.Jinv[I6[c] * 3 + 2] * g.Jinv[J6[c] * 3 + 2]);
    for (int a = 0; a < nloc; ++a) {
      const int32_t na = L.elem[e * nloc + a];
      if (L.boundary[na]) continue;
      for (int b = 0; b < nloc; ++b) {
        const int32_t nb = L.elem[e * nloc + b];
        if (L.boundary[nb]) continue;
        double k = 0.0;
        for (int c = 0; c < 6; ++c) k += fac[c] * R.stiff[c][sym_index(a, b, nloc)];
        trip.emplace_back((int64_t)na * L.n_nodes + nb, k);
      }
    }
  }
  std::sort(trip.begin(), trip.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
  off.assign(L.n_nodes + 1, 0);
  col.clear();
  val.clear();
  diag.assign(L.n_nodes, 0.0);
  for (size_t i = 0; i < trip.size();) {
    const int64_t key = trip[i].first;
    double v = 0.0;
    for (; i < trip.size() && trip[i].first == key; ++i) v += trip[i].second;  // element order within the key
    const int64_t r = key / L.n_nodes, c = key % L.n_nodes;
    col.push_back((int32_t)c);
    val.push_back(v);
    off[r + 1]++;
    if (r == c) diag[r] = v;
  }
  for (int64_t k = 0; k < L.n_nodes; ++k) off[k + 1] += off[k];
}

static int upload_csr(Csr32& d, const std::vector<int32_t>& off, const std::vector<int32_t>& col,
                      const std::vector<double>& val) {
  d.n_rows = (int64_t)off.size() - 1;
  d.nnz = (int64_t)col.size();
  std::vector<float> v32(val.begin(), val.end());
  MK_TRY(upload(&d.d_off, off.data(), off.size()));
  MK_TRY(upload(&d.d_col, col.data(), std::max<size_t>(col.size(), 1)));
  MK_TRY(upload(&d.d_val, v32.data(), std::max<size_t>(v32.size(), 1)));
  return MK_OK;
}

void free_csr(Csr32& c) {
  cudaFree(c.d_off);
  cudaFree(c.d_col);
  cudaFree(c.d_val);
  c = Csr32{};
}

int mesh_mass_factor(mk_ctx* ctx, mk_mesh* m);  // mk_eig.cu

}  // namespace mk

using namespace mk;

extern "C" {

int mk_last_error(char* buf, size_t len) {
  if (!buf || len == 0) return (int)g_err.size();
  size_t n = std::min(len - 1, g_err.size());
  std::memcpy(buf, g_err.data(), n);
  buf[n] = 0;
  return (int)g_err.size();
}

const char* mk_version(void) { return "mk 0.1 (sm_103a)"; }

long long mk_launch_count(void) { return g_launch_count.load(std::memory_order_relaxed); }

int mk_profile_enable(mk_ctx* ctx, int on) {
  MK_ARG(ctx, "mk_profile_enable: null ctx");
  ctx->prof_on = on != 0;
  for (int k = 0; k < kProfKinds; ++k) {
    ctx->prof_used[k] = 0;
    ctx->acc_ms[k] = 0.0;
    ctx->acc_n[k] = 0;
  }
  return MK_OK;
}

int mk_profile_read(mk_ctx* ctx, int kind, double* total_ms, long long* count) {
  MK_ARG(ctx && total_ms && count && kind >= 0 && kind < kProfKinds, "mk_profile_read: bad argument");
  double t = 0.0;
  for (int i = 0; i < ctx->prof_used[kind]; ++i) {
    float ms = 0.f;
    MK_CUDA(cudaEventSynchronize(ctx->prof_ev[kind][2 * i + 1]));
    MK_CUDA(cudaEventElapsedTime(&ms, ctx->prof_ev[kind][2 * i], ctx->prof_ev[kind][2 * i + 1]));
    t += ms;
  }
  *total_ms = t + ctx->acc_ms[kind];
  *count = ctx->prof_used[kind] + ctx->acc_n[kind];
  return MK_OK;
}

int mk_ctx_create(mk_ctx** out, int device) {
  MK_ARG(out, "mk_ctx_create: null out");
  *out = nullptr;
  int n = 0;
  MK_CUDA(cudaGetDeviceCount(&n));
  MK_ARG(device >= 0 && device < n, "mk_ctx_create: bad device id");
  MK_CUDA(cudaSetDevice(device));
  mk_ctx* c = new mk_ctx();
  c->device = device;
  MK_CUDA(cudaDeviceGetAttribute(&c->n_sms, cudaDevAttrMultiProcessorCount, device));
  MK_CUDA(cudaMalloc(&c->d_fault, sizeof(int)));
  MK_CUDA(cudaMemset(c->d_fault, 0, sizeof(int)));
  MK_CUDA(cudaStreamCreateWithFlags(&c->solve_stream, cudaStreamNonBlocking));
  for (cudaEvent_t& e : c->solve_ev) MK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  for (int order = 1; order <= 2; ++order) {
    build_ref_tables(order, &c->h_ref[order]);
    MK_TRY(upload(&c->d_ref[order], &c->h_ref[order], 1));
  }
  *out = c;
  return MK_OK;
}

int mk_ctx_destroy(mk_ctx* c) {
  if (!c) return MK_OK;
  cudaSetDevice(c->device);
  for (void* p : c->slot_ptr) cudaFree(p);
  for (int o = 1; o <= 2; ++o) cudaFree(c->d_ref[o]);
  if (c->pinned) cudaFreeHost(c->pinned);
  for (auto& v : c->prof_ev)
    for (cudaEvent_t e : v) cudaEventDestroy(e);
  for (auto& v : c->cap_ev)
    for (cudaEvent_t e : v) cudaEventDestroy(e);
  for (cudaEvent_t e : c->solve_ev)
    if (e) cudaEventDestroy(e);
  if (c->solve_stream) cudaStreamDestroy(c->solve_stream);
  cudaFree(c->d_fault);
  delete c;
  return MK_OK;
}

int mk_ctx_set_option(mk_ctx* c, int option, int value) {
  MK_ARG(c, "mk_ctx_set_option: null ctx");
  switch (option) {
    case MK_OPT_GRAPHS: c->no_graphs = value == 0; return MK_OK;
    case MK_OPT_PATCH_PIPELINE:
      MK_ARG(value >= 0 && value <= 2, "mk_ctx_set_option: patch kernel must be 0, 1 or 2");
      c->patch_kernel = value;
      return MK_OK;
    case MK_OPT_WAIT_LIMIT:
      MK_ARG(value >= -1, "mk_ctx_set_option: wait limit must be >= 0, or -1 for the default");
      c->wait_limit = value < 0 ? kWaitLimitDefault : value;
      return MK_OK;
    case MK_OPT_DECOMPOSE_CTAS:
      MK_ARG(value >= 0, "mk_ctx_set_option: decomposition CTAs must be >= 0 (0 = one per SM)");
      c->decompose_ctas = value;
      return MK_OK;
    case MK_OPT_PAIR_RESIDUAL:
      MK_ARG(value == 0 || value == 1, "mk_ctx_set_option: pair residual must be 0 or 1");
      c->pair_residual = value == 1;
      return MK_OK;
    default: return fail(MK_ERR_INVALID_ARG, "mk_ctx_set_option: unknown option");
  }
}

int mk_ctx_fault(mk_ctx* c, int* fault) {
  MK_ARG(c && fault, "mk_ctx_fault: null argument");
  MK_CUDA(cudaSetDevice(c->device));
  MK_CUDA(cudaDeviceSynchronize());
  MK_CUDA(cudaMemcpy(fault, c->d_fault, sizeof(int), cudaMemcpyDeviceToHost));
  MK_CUDA(cudaMemset(c->d_fault, 0, sizeof(int)));
  return MK_OK;
}


int mk_mesh_upload(mk_ctx* ctx, const mk_mesh_desc* fine, const mk_mesh_desc* coarse, const int32_t* fine_parent,
                   mk_mesh** out) {
  MK_ARG(ctx && fine && coarse && fine_parent && out, "mk_mesh_upload: null argument");
  *out = nullptr;
  MK_ARG(fine->order == coarse->order, "mk_mesh_upload: fine and coarse orders differ");
  MK_CUDA(cudaSetDevice(ctx->device));
  mk_mesh* m = new mk_mesh();
  m->ctx = ctx;
  m->device = ctx->device;
  int r = build_level(fine, m->fine, "fine");
  if (r == MK_OK) r = build_level(coarse, m->coarse, "coarse");
  if (r != MK_OK) { delete m; return r; }
  const Level& F = m->fine;
  const Level& C = m->coarse;
  m->parent.assign(fine_parent, fine_parent + F.n_elems);
  for (int32_t p : m->parent)
    if (p < 0 || p >= C.n_elems) { delete m; return fail(MK_ERR_INVALID_ARG, "mk_mesh_upload: parent out of range"); }
  std::vector<int32_t> P_off, P_col;
  std::vector<double> P_val;
  r = build_interp(F, C, m->parent, true, P_off, P_col, P_val);
  if (r != MK_OK) { delete m; return r; }
  // transpose: coarse free DOF -> fine nodes (increasing)
  std::vector<int32_t> PT_off(C.n_free + 1, 0), PT_col(P_col.size());
  std::vector<double> PT_val(P_col.size());
  for (int32_t c : P_col) PT_off[c + 1]++;
  for (int64_t k = 0; k < C.n_free; ++k) PT_off[k + 1] += PT_off[k];
  {
    std::vector<int32_t> pos(PT_off.begin(), PT_off.end() - 1);
    for (int64_t nd = 0; nd < F.n_nodes; ++nd)
      for (int32_t k = P_off[nd]; k < P_off[nd + 1]; ++k) {
        int32_t p = pos[P_col[k]]++;
        PT_col[p] = (int32_t)nd;
        PT_val[p] = P_val[k];
      }
  }
  m->PT_nnz = (int64_t)PT_col.size();
  std::vector<int32_t> ch_off(C.n_elems + 1, 0), ch(F.n_elems);
  for (int32_t p : m->parent) ch_off[p + 1]++;
  for (int64_t k = 0; k < C.n_elems; ++k) ch_off[k + 1] += ch_off[k];
  {
    std::vector<int32_t> pos(ch_off.begin(), ch_off.end() - 1);
    for (int64_t e = 0; e < F.n_elems; ++e) ch[pos[m->parent[e]]++] = (int32_t)e;
  }
  r = upload_level(m->fine);
  if (r == MK_OK) r = upload_level(m->coarse);
  if (r == MK_OK) r = upload(&m->d_P_off, P_off.data(), P_off.size());
  if (r == MK_OK) r = upload(&m->d_P_col, P_col.data(), P_col.size());
  if (r == MK_OK) r = upload(&m->d_P_val, P_val.data(), P_val.size());
  if (r == MK_OK) r = upload(&m->d_PT_off, PT_off.data(), PT_off.size());
  if (r == MK_OK) r = upload(&m->d_PT_col, PT_col.data(), PT_col.size());
  if (r == MK_OK) r = upload(&m->d_PT_val, PT_val.data(), PT_val.size());
  if (r == MK_OK) r = upload(&m->d_child_off, ch_off.data(), ch_off.size());
  if (r == MK_OK) r = upload(&m->d_child, ch.data(), ch.size());
  if (r == MK_OK) r = build_patches(m);
  if (r == MK_OK) r = mesh_mass_factor(ctx, m);
  if (r != MK_OK) { mk_mesh_destroy(m); return r; }
  *out = m;
  return MK_OK;
}

int mk_mesh_destroy(mk_mesh* m) {
  if (!m) return MK_OK;
  cudaSetDevice(m->device);
  free_level(m->fine);
  free_level(m->coarse);
  cudaFree(m->d_P_off); cudaFree(m->d_P_col); cudaFree(m->d_P_val);
  cudaFree(m->d_PT_off); cudaFree(m->d_PT_col); cudaFree(m->d_PT_val);
  cudaFree(m->d_child_off); cudaFree(m->d_child);
  free_patches(m->patches);
  cudaFree(m->d_MH_Linv);
  cudaFree(m->d_static);
  cudaFree(m->d_M64);
  if (m->mass_ev) cudaEventDestroy(m->mass_ev);
  cudaFree(m->d_P_val32);
  cudaFree(m->d_PT_val32);
  cudaFree(m->d_cinv_poisson);
  cudaFree(m->d_K64);
  cudaFree(m->d_K64diag);
  cudaFree(m->d_face_nb);
  cudaFree(m->d_cinv_corr);
  if (m->static_ev) cudaEventDestroy(m->static_ev);
  for (MgLevel& g : m->mg) {
    free_level(g.L);
    free_csr(g.K); free_csr(g.P); free_csr(g.R);
    cudaFree(g.d_dinv);
  }
  free_csr(m->mgP);
  free_csr(m->mgR);
  delete m;
  return MK_OK;
}

int mk_mesh_get_info(const mk_mesh* m, mk_mesh_info* info) {
  MK_ARG(m && info, "mk_mesh_get_info: null argument");
  info->order = m->fine.order;
  info->nloc = m->fine.nloc;
  info->n_nodes = m->fine.n_nodes;
  info->n_free = m->fine.n_free;
  info->n_elems = m->fine.n_elems;
  info->n_colours = m->fine.n_colours;
  info->n_nodes_coarse = m->coarse.n_nodes;
  info->n_free_coarse = m->coarse.n_free;
  info->n_elems_coarse = m->coarse.n_elems;
  info->n_quad = kQ;
  return MK_OK;
}

int mk_mesh_get_topology(const mk_mesh* m, int level, double* nodes, uint8_t* boundary, int32_t* elem,
                         int32_t* colour) {
  MK_ARG(m && (level == 0 || level == 1), "mk_mesh_get_topology: bad argument");
  const Level& L = level == 0 ? m->fine : m->coarse;
  if (nodes) std::memcpy(nodes, L.nodes.data(), L.nodes.size() * sizeof(double));
  if (boundary) std::memcpy(boundary, L.boundary.data(), L.boundary.size());
  if (elem) std::memcpy(elem, L.elem.data(), L.elem.size() * sizeof(int32_t));
  if (colour) std::memcpy(colour, L.colour.data(), L.colour.size() * sizeof(int32_t));
  return MK_OK;
}


int mk_mesh_set_hierarchy(mk_mesh* m, int n_mid, const mk_mesh_desc* levels, const int32_t* const* parents) {
  MK_ARG(m && n_mid >= 0 && n_mid <= 16 && (n_mid == 0 || (levels && parents)), "mk_mesh_set_hierarchy: bad argument");
  MK_CUDA(cudaSetDevice(m->device));
  MK_CUDA(cudaDeviceSynchronize());
  const RefTables& R = m->ctx->h_ref[m->fine.order];
  std::vector<MgLevel> mg(n_mid);
  auto cleanup = [&]() {
    for (MgLevel& g : mg) {
      free_level(g.L);
      free_csr(g.K); free_csr(g.P); free_csr(g.R);
      cudaFree(g.d_dinv);
    }
  };
  int r = MK_OK;
  std::vector<int32_t> off, col, toff, tcol;
  std::vector<double> val, tval, diag;
  for (int k = 0; k < n_mid && r == MK_OK; ++k) {
    MgLevel& g = mg[k];
    r = build_level(&levels[k], g.L, "hierarchy level");
    if (r != MK_OK) break;
    if (g.L.order != m->fine.order) { r = fail(MK_ERR_INVALID_ARG, "mk_mesh_set_hierarchy: orders differ"); break; }
    const Level& C = k == 0 ? m->coarse : mg[k - 1].L;
    std::vector<int32_t> par(parents[k], parents[k] + g.L.n_elems);
    for (int32_t p : par)
      if (p < 0 || p >= C.n_elems) { r = fail(MK_ERR_INVALID_ARG, "mk_mesh_set_hierarchy: parent out of range"); break; }
    if (r != MK_OK) break;
    r = build_interp(g.L, C, par, k == 0, off, col, val);
    if (r != MK_OK) break;
    transpose_csr(k == 0 ? C.n_free : C.n_nodes, off, col, val, toff, tcol, tval);
    r = upload_csr(g.P, off, col, val);
    if (r == MK_OK) r = upload_csr(g.R, toff, tcol, tval);
    if (r != MK_OK) break;
    stiffness_csr(g.L, R, off, col, val, diag);
    r = upload_csr(g.K, off, col, val);
    if (r != MK_OK) break;
    std::vector<float> dinv(g.L.n_nodes, 0.f);
    for (int64_t i = 0; i < g.L.n_nodes; ++i)
      if (!g.L.boundary[i] && diag[i] > 0) dinv[i] = (float)(1.0 / diag[i]);
    r = upload(&g.d_dinv, dinv.data(), dinv.size());
    if (r == MK_OK) r = upload(&g.L.d_boundary, g.L.boundary.data(), g.L.boundary.size());
  }
  // the fine mesh from the finest intermediate level (or from V_H)
  Csr32 P, Rt;
  if (r == MK_OK) {
    if (n_mid > 0) {
      std::vector<int32_t> par(parents[n_mid], parents[n_mid] + m->fine.n_elems);
      for (int32_t p : par)
        if (p < 0 || p >= mg[n_mid - 1].L.n_elems) r = fail(MK_ERR_INVALID_ARG, "mk_mesh_set_hierarchy: parent out of range");
      if (r == MK_OK) r = build_interp(m->fine, mg[n_mid - 1].L, par, false, off, col, val);
      if (r == MK_OK) transpose_csr(mg[n_mid - 1].L.n_nodes, off, col, val, toff, tcol, tval);
    } else {
      r = build_interp(m->fine, m->coarse, m->parent, true, off, col, val);
      if (r == MK_OK) transpose_csr(m->coarse.n_free, off, col, val, toff, tcol, tval);
    }
    if (r == MK_OK) r = upload_csr(P, off, col, val);
    if (r == MK_OK) r = upload_csr(Rt, toff, tcol, tval);
  }
  if (r != MK_OK) {
    cleanup();
    free_csr(P);
    free_csr(Rt);
    return r;
  }
  // replace an earlier hierarchy
  for (MgLevel& g : m->mg) {
    free_level(g.L);
    free_csr(g.K); free_csr(g.P); free_csr(g.R);
    cudaFree(g.d_dinv);
  }
  free_csr(m->mgP);
  free_csr(m->mgR);
  m->mg = std::move(mg);
  m->mgP = P;
  m->mgR = Rt;
  m->has_mg = true;
  return MK_OK;
}

}  // extern "C"
