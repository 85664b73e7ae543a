// Element patches for the single-pass operator application (built once at mesh upload).
//
// Elements are ordered along a Morton curve of their centroids and cut into patches of at most kPatchElems(order)
// consecutive elements; one CTA applies one patch.  Inside the CTA the element products go to shared memory and
// each local node sums its incidences in a fixed order (owner computes).  A node used by one patch only is
// written directly; a node shared by several patches is written to one halo slot per patch, and a second kernel
// adds those slots in patch order.  Every sum has a fixed order, so results are bitwise reproducible, with no
// atomics and no colour-by-colour launches.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>

#include "mk_internal.h"

namespace mk {

// Elements per patch when a mesh is uploaded: 256 (P1) or 128 (P2); mk_mesh_set_patch_elems changes it later.
int patch_elems(int nloc) { return nloc == 4 ? 256 : 128; }

static uint32_t spread10(uint32_t v) {
  v &= 0x3ff;
  v = (v | (v << 16)) & 0x030000FF;
  v = (v | (v << 8)) & 0x0300F00F;
  v = (v | (v << 4)) & 0x030C30C3;
  v = (v | (v << 2)) & 0x09249249;
  return v;
}

template <class T>
static int up(T** dst, const std::vector<T>& src) {
  size_t n = std::max<size_t>(src.size(), 1);
  if (cudaMalloc(dst, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return fail(MK_ERR_OOM, "patch upload: allocation failed");
  }
  if (!src.empty() && cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(MK_ERR_CUDA, "patch upload: copy failed");
  return MK_OK;
}

// matches kOwnedBoundary of the patch kernels: an owned boundary node's target carries this bit
constexpr int32_t kOwnedBoundaryTarget = 1 << 30;

int build_patches(mk_mesh* m, int pe) {
  const Level& L = m->fine;
  Patches& P = m->patches;
  const int nloc = L.nloc;
  const int64_t E = L.n_elems, nn = L.n_nodes;
  if (nn >= kOwnedBoundaryTarget) return fail(MK_ERR_UNSUPPORTED, "patches: more than 2^30 fine nodes");
  const int PE = pe > 0 ? pe : patch_elems(nloc);
  // Morton order of element centroids
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t v = 0; v < L.n_vertices; ++v)
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], L.nodes[v * 3 + k]);
      hi[k] = std::max(hi[k], L.nodes[v * 3 + k]);
    }
  std::vector<uint32_t> code(E);
  for (int64_t e = 0; e < E; ++e) {
    uint32_t q[3];
    for (int k = 0; k < 3; ++k) {
      double c = 0.0;
      for (int a = 0; a < 4; ++a) c += L.nodes[(int64_t)L.elem[e * nloc + a] * 3 + k];
      c *= 0.25;
      const double t = (hi[k] > lo[k]) ? (c - lo[k]) / (hi[k] - lo[k]) : 0.0;
      q[k] = (uint32_t)std::min(1023.0, std::max(0.0, t * 1024.0));
    }
    code[e] = spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
  }
  std::vector<int32_t> order(E);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return code[a] < code[b]; });
  const int np = (int)((E + PE - 1) / PE);
  P.n_patches = np;
  P.max_elems = PE;
  std::vector<int32_t> elem_off(np + 1), node_off(np + 1, 0);
  for (int p = 0; p <= np; ++p) elem_off[p] = (int32_t)std::min<int64_t>((int64_t)p * PE, E);
  // local node lists (sorted unique global ids per patch)
  std::vector<int32_t> node_global;
  std::vector<int32_t> cnt(nn, 0);
  for (int p = 0; p < np; ++p) {
    std::vector<int32_t> ns;
    for (int32_t i = elem_off[p]; i < elem_off[p + 1]; ++i)
      for (int a = 0; a < nloc; ++a) ns.push_back(L.elem[(int64_t)order[i] * nloc + a]);
    std::sort(ns.begin(), ns.end());
    // incidences of each distinct node inside the patch; local nodes are numbered by decreasing count (ties by
    // global id) so that the threads of a warp, which take consecutive local nodes, sum lists of similar length
    std::vector<std::pair<int32_t, int32_t>> by_count;  // (-count, global id)
    for (size_t i = 0; i < ns.size();) {
      size_t j = i;
      while (j < ns.size() && ns[j] == ns[i]) ++j;
      by_count.push_back({-(int32_t)(j - i), ns[i]});
      i = j;
    }
    std::sort(by_count.begin(), by_count.end());
    ns.clear();
    for (const auto& bc : by_count) ns.push_back(bc.second);
    for (int32_t g : ns) cnt[g]++;
    node_off[p + 1] = node_off[p] + (int32_t)ns.size();
    P.max_nodes = std::max(P.max_nodes, (int)ns.size());
    node_global.insert(node_global.end(), ns.begin(), ns.end());
  }
  // halo slots of shared nodes: slots of one node are consecutive, in patch order
  std::vector<int64_t> hbase(nn, -1);
  std::vector<int32_t> shared_node, shared_off(1, 0);
  int64_t nslot = 0;
  for (int64_t g = 0; g < nn; ++g)
    if (cnt[g] >= 2) {
      hbase[g] = nslot;
      nslot += cnt[g];
      shared_node.push_back((int32_t)g);
      shared_off.push_back((int32_t)nslot);
    }
  P.n_halo_slots = nslot;
  P.n_shared_nodes = (int64_t)shared_node.size();
  std::vector<int32_t> seen(nn, 0);
  std::vector<int32_t> target(node_global.size());
  std::vector<int32_t> inc_off;
  std::vector<uint16_t> inc;
  inc_off.reserve(node_global.size() + np);
  std::vector<int32_t> conn((size_t)E * nloc);
  std::vector<uint16_t> lconn((size_t)E * nloc);
  std::vector<uint16_t> ypos((size_t)E * nloc);
  std::vector<int32_t> elem_id(E);
  for (int p = 0; p < np; ++p) {
    const int32_t nb = node_off[p], ne = node_off[p + 1];
    const int nl = ne - nb;
    for (int l = 0; l < nl; ++l) {
      const int32_t g = node_global[nb + l];
      target[nb + l] = (cnt[g] >= 2) ? -(int32_t)(hbase[g] + seen[g]++) - 1
                                     : (L.boundary[g] ? (g | kOwnedBoundaryTarget) : g);
    }
    // local index of each global node of the patch (node_global[nb, ne) is in count order, not sorted)
    std::vector<std::pair<int32_t, int32_t>> lookup(nl);  // (global id, local index), sorted by global id
    for (int l = 0; l < nl; ++l) lookup[l] = {node_global[nb + l], l};
    std::sort(lookup.begin(), lookup.end());
    // incidences per local node in (element, slot) order, CSR local to the patch
    std::vector<int32_t> c(nl + 1, 0);
    std::vector<int32_t> lidx((size_t)(elem_off[p + 1] - elem_off[p]) * nloc);
    for (int32_t i = elem_off[p]; i < elem_off[p + 1]; ++i) {
      elem_id[i] = order[i];
      for (int a = 0; a < nloc; ++a) {
        const int32_t g = L.elem[(int64_t)order[i] * nloc + a];
        conn[(size_t)i * nloc + a] = g;
        const int l = std::lower_bound(lookup.begin(), lookup.end(), std::make_pair(g, (int32_t)-1))->second;
        lidx[(size_t)(i - elem_off[p]) * nloc + a] = l;
        lconn[(size_t)i * nloc + a] = (uint16_t)l;
        c[l + 1]++;
      }
    }
    for (int l = 0; l < nl; ++l) c[l + 1] += c[l];
    std::vector<uint16_t> lst(c[nl]);
    std::vector<int32_t> pos(c.begin(), c.end() - 1);
    for (size_t k = 0; k < lidx.size(); ++k) {  // k = local element * nloc + slot; stored as slot * PE + element
      const int el = (int)(k / nloc), a = (int)(k % nloc);
      ypos[(size_t)elem_off[p] * nloc + k] = (uint16_t)pos[lidx[k]];  // its place in the node-sorted list
      lst[pos[lidx[k]]++] = (uint16_t)(a * PE + el);
    }
    const int32_t base = (int32_t)inc.size();
    for (int l = 0; l < nl; ++l) inc_off.push_back(base + c[l]);
    inc.insert(inc.end(), lst.begin(), lst.end());
  }
  inc_off.push_back((int32_t)inc.size());   // sentinel after the last patch
  // inc_off has one entry per local node of every patch (start) plus one final sentinel; the end of local node l
  // of patch p is the start of the next entry, which for the last node of a patch is the first node of the next
  // patch (or the sentinel): incidences of consecutive patches are contiguous, so starts alone suffice.
  // learned-preconditioner geometry (patch order) and node multiplicities
  std::vector<float> geomf((size_t)E * 16, 0.f);
  for (int64_t i = 0; i < E; ++i) {
    const Geom& G = L.geom[elem_id[i]];
    const double h = std::cbrt(std::fabs(G.det));
    double v[4][3];
    for (int c = 0; c < 3; ++c) {
      v[0][c] = G.x0[c];
      for (int k = 1; k < 4; ++k) v[k][c] = G.x0[c] + G.J[c * 3 + (k - 1)];
    }
    double cen[3];
    for (int c = 0; c < 3; ++c) cen[c] = 0.25 * (v[0][c] + v[1][c] + v[2][c] + v[3][c]);
    geomf[i * 16] = (float)h;
    for (int k = 0; k < 4; ++k)
      for (int c = 0; c < 3; ++c) geomf[i * 16 + 1 + 3 * k + c] = (float)((v[k][c] - cen[c]) / h);
  }
  // patch records (layout in Patches)
  auto a16 = [](int64_t b) { return (b + 15) / 16 * 16; };
  // every record takes the same stride (the largest record's size), so that a kernel finds patch p's record at
  // p * stride without first reading an offset
  std::vector<int64_t> rec_off(np + 1, 0);
  P.max_rec_bytes = 0;
  for (int p = 0; p < np; ++p) {
    const int64_t ne = elem_off[p + 1] - elem_off[p], nl = node_off[p + 1] - node_off[p];
    const int64_t bytes = kRecHeader + 2 * a16(ne * nloc * 2) + a16((nl + 1) * 2) + 2 * a16(nl * 4);
    P.max_rec_bytes = std::max<int>(P.max_rec_bytes, (int)bytes);
  }
  for (int p = 0; p < np; ++p) rec_off[p + 1] = rec_off[p] + P.max_rec_bytes;
  std::vector<unsigned char> rec((size_t)rec_off[np], 0);
  for (int p = 0; p < np; ++p) {
    const int32_t e0 = elem_off[p], ne = elem_off[p + 1] - e0, n0 = node_off[p], nl = node_off[p + 1] - n0;
    unsigned char* r = rec.data() + rec_off[p];
    const int32_t o_inc = kRecHeader + (int32_t)a16((int64_t)ne * nloc * 2);
    const int32_t o_io = o_inc + (int32_t)a16((int64_t)ne * nloc * 2);
    const int32_t o_tg = o_io + (int32_t)a16((int64_t)(nl + 1) * 2);
    const int32_t o_gd = o_tg + (int32_t)a16((int64_t)nl * 4);
    const int32_t hdr[8] = {e0, ne, n0, nl, o_inc, o_io, o_tg, o_gd};
    std::memcpy(r, hdr, sizeof(hdr));
    std::memcpy(r + kRecHeader, lconn.data() + (size_t)e0 * nloc, (size_t)ne * nloc * 2);
    std::memcpy(r + o_inc, ypos.data() + (size_t)e0 * nloc, (size_t)ne * nloc * 2);
    const int32_t ibase = e0 * nloc;
    for (int l = 0; l <= nl; ++l) {
      const int32_t v = inc_off[n0 + l] - ibase;  // the entry after a patch's last node starts the next patch
      const uint16_t u = (uint16_t)v;
      std::memcpy(r + o_io + 2 * l, &u, 2);
    }
    std::memcpy(r + o_tg, target.data() + n0, (size_t)nl * 4);
    std::memcpy(r + o_gd, node_global.data() + n0, (size_t)nl * 4);
    // the invariants the kernels index by, checked once here: local nodes, incidences and offsets in range
    for (int64_t k = 0; k < (int64_t)ne * nloc; ++k)
      if (lconn[(size_t)e0 * nloc + k] >= nl || ypos[(size_t)e0 * nloc + k] >= ne * nloc ||
          inc[(size_t)e0 * nloc + k] >= nloc * PE)
        return fail(MK_ERR_INVALID_ARG, "patches: local index out of range");
    for (int l = 0; l < nl; ++l)
      if (inc_off[n0 + l + 1] < inc_off[n0 + l] || inc_off[n0 + l + 1] - ibase > ne * nloc)
        return fail(MK_ERR_INVALID_ARG, "patches: incidence offsets out of range");
  }
  std::vector<int32_t> mult(nn, 0);
  for (int64_t i = 0; i < E * nloc; ++i) mult[L.elem[i]]++;
  std::vector<float> inv_mult(nn);
  for (int64_t g = 0; g < nn; ++g) inv_mult[g] = mult[g] > 0 ? (float)(1.0 / mult[g]) : 0.f;
  int r = up(&P.d_patch_elem_off, elem_off);
  if (r == MK_OK) r = up(&P.d_geomf, geomf);
  if (r == MK_OK) r = up(&P.d_inv_mult, inv_mult);
  if (r == MK_OK) r = up(&P.d_node_gid, node_global);
  if (r == MK_OK) r = up(&P.d_lconn, lconn);
  if (r == MK_OK) r = up(&P.d_patch_node_off, node_off);
  if (r == MK_OK) r = up(&P.d_elem_id, elem_id);
  if (r == MK_OK) r = up(&P.d_conn, conn);
  if (r == MK_OK) r = up(&P.d_node_target, target);
  if (r == MK_OK) r = up(&P.d_inc_off, inc_off);
  if (r == MK_OK) r = up(&P.d_inc, inc);
  if (r == MK_OK) r = up(&P.d_shared_node, shared_node);
  if (r == MK_OK) r = up(&P.d_shared_off, shared_off);
  if (r == MK_OK) r = up(&P.d_rec, rec);
  if (r == MK_OK) r = up(&P.d_rec_off, rec_off);
  return r;
}

void free_patches(Patches& p) {
  cudaFree(p.d_patch_elem_off); cudaFree(p.d_patch_node_off); cudaFree(p.d_elem_id); cudaFree(p.d_conn);
  cudaFree(p.d_node_target); cudaFree(p.d_inc_off); cudaFree(p.d_inc); cudaFree(p.d_shared_node);
  cudaFree(p.d_geomf); cudaFree(p.d_inv_mult); cudaFree(p.d_node_gid); cudaFree(p.d_lconn);
  cudaFree(p.d_shared_off); cudaFree(p.d_rec); cudaFree(p.d_rec_off); cudaFree(p.d_stiff_fac);
  p = Patches();
}

}  // namespace mk
