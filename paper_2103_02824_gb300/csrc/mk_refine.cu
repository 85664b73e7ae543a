// The outer AFEM loop's Refine step (Sec. 2: the marked elements are refined so that the mesh stays shape regular
// and conforming): newest-vertex bisection in Maubach's form with conforming closure, on the GPU.
//
// A tetrahedron (x0, x1, x2, x3) with tag k in {1, 2, 3} is cut at the midpoint z of its refinement edge x0-xk into
// (x0, .., x_{k-1}, z, x_{k+1}, .., x3), which keeps its index, and (x1, .., xk, z, x_{k+1}, .., x3), appended after
// the existing elements in the order of the cut ones; both take tag k - 1 (3 after 1).  One round bisects a set of
// elements; the first round takes the marked ones, and every later round the elements that hold an edge already
// cut (closure), until none does.  Cut edges live in an open-addressing hash table keyed by the sorted vertex pair
// (lo * 2^31 + hi); a new midpoint is numbered after the existing vertices in the order of the lowest-index element
// that cuts its edge in that round (the owner, found with atomicMin), so the numbering, like everything else here,
// does not depend on the order in which threads run.  Every probe loop is bounded by the table size; a full table
// is reported as an error.
#include <climits>
#include <vector>

#include "mk_device.cuh"

namespace mk {

namespace {

constexpr uint64_t kEmpty = ~0ull;
constexpr int kScanThreads = 1024;

struct EdgeTable {
  uint64_t* key;
  int32_t* owner;
  int32_t* mid;
  uint64_t mask;  // capacity - 1 (capacity a power of two)
};

__device__ __forceinline__ uint64_t edge_key(int32_t a, int32_t b) {
  const uint64_t lo = (uint64_t)min(a, b), hi = (uint64_t)max(a, b);
  return (lo << 31) | hi;
}

__device__ __forceinline__ uint64_t slot_of(uint64_t key, uint64_t mask) {
  uint64_t h = key * 0x9E3779B97F4A7C15ull;
  return (h ^ (h >> 29)) & mask;
}

// the slot of key, inserting it if absent; -1 if the table is full
__device__ __forceinline__ int64_t table_insert(EdgeTable t, uint64_t key) {
  uint64_t s = slot_of(key, t.mask);
  for (uint64_t probe = 0; probe <= t.mask; ++probe) {
    const unsigned long long prev =
        atomicCAS(reinterpret_cast<unsigned long long*>(t.key + s), (unsigned long long)kEmpty, (unsigned long long)key);
    if (prev == kEmpty || prev == key) return (int64_t)s;
    s = (s + 1) & t.mask;
  }
  return -1;
}

// the slot of key, or -1 if absent
__device__ __forceinline__ int64_t table_find(EdgeTable t, uint64_t key) {
  uint64_t s = slot_of(key, t.mask);
  for (uint64_t probe = 0; probe <= t.mask; ++probe) {
    const uint64_t k = t.key[s];
    if (k == key) return (int64_t)s;
    if (k == kEmpty) return -1;
    s = (s + 1) & t.mask;
  }
  return -1;
}

}  // namespace

// input check: every vertex id in [0, nv) and every tag in {1, 2, 3}, else *bad = 1
__global__ void k_rf_check(int64_t E, int64_t nv, const int32_t* __restrict__ T, const int8_t* __restrict__ K,
                           int* __restrict__ bad) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  bool ok = K[e] >= 1 && K[e] <= 3;
#pragma unroll
  for (int c = 0; c < 4; ++c) ok = ok && T[e * 4 + c] >= 0 && (int64_t)T[e * 4 + c] < nv;
  if (!ok) atomicOr(bad, 1);
}

__global__ void k_rf_table_init(uint64_t n, EdgeTable t) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > t.mask || i >= n) return;
  t.key[i] = kEmpty;
  t.owner[i] = INT_MAX;
  t.mid[i] = -1;
}

// round, step 1: the refinement edge of every flagged element into the table, its owner the lowest flagged index
__global__ void k_rf_claim(int64_t E, const int32_t* __restrict__ T, const int8_t* __restrict__ K,
                           const uint8_t* __restrict__ flag, EdgeTable t, int* __restrict__ full) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E || !flag[e]) return;
  const int k = K[e];
  const int64_t s = table_insert(t, edge_key(T[e * 4], T[e * 4 + k]));
  if (s < 0) {
    atomicOr(full, 1);
    return;
  }
  atomicMin(t.owner + s, (int32_t)e);
}

// round, step 2: own[e] = 1 if e owns a refinement edge that has no midpoint yet
__global__ void k_rf_own(int64_t E, const int32_t* __restrict__ T, const int8_t* __restrict__ K,
                         const uint8_t* __restrict__ flag, EdgeTable t, int32_t* __restrict__ own) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  int32_t o = 0;
  if (flag[e]) {
    const int64_t s = table_find(t, edge_key(T[e * 4], T[e * 4 + K[e]]));
    o = (s >= 0 && t.mid[s] < 0 && t.owner[s] == (int32_t)e) ? 1 : 0;
  }
  own[e] = o;
}

// round, step 3: the owners number their midpoints (nv + exclusive scan of own) and place them
__global__ void k_rf_midpoints(int64_t E, const int32_t* __restrict__ T, const int8_t* __restrict__ K,
                               const int32_t* __restrict__ own, const int32_t* __restrict__ rank, int64_t nv,
                               EdgeTable t, double* __restrict__ X) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E || !own[e]) return;
  const int32_t a = T[e * 4], b = T[e * 4 + K[e]];
  const int64_t s = table_find(t, edge_key(a, b));
  const int64_t z = nv + rank[e];
  t.mid[s] = (int32_t)z;
#pragma unroll
  for (int c = 0; c < 3; ++c) X[z * 3 + c] = 0.5 * (X[(int64_t)a * 3 + c] + X[(int64_t)b * 3 + c]);
}

// round, step 4: bisect every flagged element; the second child goes to E + pos[e]
__global__ void k_rf_bisect(int64_t E, int32_t* __restrict__ T, int8_t* __restrict__ K, int32_t* __restrict__ parent,
                            const uint8_t* __restrict__ flag, const int32_t* __restrict__ pos, EdgeTable t) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E || !flag[e]) return;
  int32_t v[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) v[c] = T[e * 4 + c];
  const int k = K[e];
  const int32_t z = t.mid[table_find(t, edge_key(v[0], v[k]))];
  const int8_t nk = (int8_t)(k > 1 ? k - 1 : 3);
  const int64_t f = E + pos[e];
  // second child (x1, .., xk, z, x_{k+1}, .., x3)
  int q = 0;
  for (int c = 1; c <= k; ++c) T[f * 4 + q++] = v[c];
  T[f * 4 + q++] = z;
  for (int c = k + 1; c < 4; ++c) T[f * 4 + q++] = v[c];
  K[f] = nk;
  parent[f] = parent[e];
  // first child: x_k replaced by z
  T[e * 4 + k] = z;
  K[e] = nk;
}

// closure: flag[e] = 1 if element e holds an edge that has a midpoint
__global__ void k_rf_hanging(int64_t E, const int32_t* __restrict__ T, EdgeTable t, uint8_t* __restrict__ flag,
                             int32_t* __restrict__ cnt) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {1, 2, 3, 2, 3, 3};
  uint8_t h = 0;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int64_t s = table_find(t, edge_key(T[e * 4 + pa[j]], T[e * 4 + pb[j]]));
    if (s >= 0 && t.mid[s] >= 0) h = 1;
  }
  flag[e] = h;
  cnt[e] = h;
}

// exclusive scan of int32 counts, three passes (block scans, the block totals by one block, the offsets)
__global__ void k_scan_blocks(int64_t n, const int32_t* __restrict__ in, int32_t* __restrict__ out,
                              int64_t* __restrict__ bsum) {
  __shared__ int32_t warp_tot[kScanThreads / 32];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int32_t v = i < n ? in[i] : 0;
  int32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int32_t s = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < (int)(blockDim.x >> 5)) warp_tot[lane] = s;  // inclusive prefix of the warp totals
  }
  __syncthreads();
  const int32_t before = w > 0 ? warp_tot[w - 1] : 0;
  if (i < n) out[i] = before + x - v;
  if (threadIdx.x == blockDim.x - 1) bsum[blockIdx.x] = (int64_t)warp_tot[(blockDim.x >> 5) - 1];
}

__global__ void k_scan_totals(int64_t nb, int64_t* __restrict__ bsum, int64_t* __restrict__ total) {
  if (threadIdx.x != 0) return;
  int64_t s = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const int64_t v = bsum[b];
    bsum[b] = s;
    s += v;
  }
  *total = s;
}

__global__ void k_scan_add(int64_t n, int32_t* __restrict__ out, const int64_t* __restrict__ boff) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += (int32_t)boff[i / kScanThreads];
}

__global__ void k_u8_to_i32(int64_t n, const uint8_t* __restrict__ a, int32_t* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = a[i];
}

__global__ void k_iota(int64_t n, int32_t* __restrict__ p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = (int32_t)i;
}

}  // namespace mk

using namespace mk;

extern "C" int mk_refine(mk_ctx* ctx, int64_t n_vertices, int64_t n_elems, double* coords, int32_t* tets, int8_t* tags,
                         int32_t* parent, const uint8_t* marked, int64_t max_vertices, int64_t max_elems,
                         int64_t* n_vertices_out, int64_t* n_elems_out, int* rounds, void* stream) {
  MK_ARG(ctx && coords && tets && tags && parent && marked && n_vertices_out && n_elems_out, "mk_refine: null argument");
  MK_ARG(n_vertices >= 4 && n_elems >= 1 && max_vertices >= n_vertices && max_elems >= n_elems,
         "mk_refine: bad sizes");
  MK_ARG(max_vertices < (1ll << 31) && max_elems < (1ll << 31), "mk_refine: at most 2^31 - 1 vertices and elements");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  // table: a power of two at least twice the new vertices there is room for
  uint64_t cap = 1024;
  while (cap < 2 * (uint64_t)(max_vertices - n_vertices) + 1024) cap <<= 1;
  const int64_t nbmax = (max_elems + kScanThreads - 1) / kScanThreads;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
  const size_t oKey = take(cap * 8), oOwn = take(cap * 4), oMid = take(cap * 4), oFlag = take((size_t)max_elems),
               oCnt = take((size_t)max_elems * 4), oScan = take((size_t)max_elems * 4),
               oPos = take((size_t)max_elems * 4), oB = take((size_t)(nbmax + 1) * 8), oTot = take(64);
  int err = MK_OK;
  char* ws = (char*)scratch(ctx, S_AFEM, off, &err);
  if (!ws) return err;
  EdgeTable t{(uint64_t*)(ws + oKey), (int32_t*)(ws + oOwn), (int32_t*)(ws + oMid), cap - 1};
  uint8_t* flag = (uint8_t*)(ws + oFlag);
  int32_t* cnt = (int32_t*)(ws + oCnt);
  int32_t* scn = (int32_t*)(ws + oScan);
  int32_t* pos = (int32_t*)(ws + oPos);
  int64_t* bsum = (int64_t*)(ws + oB);
  int64_t* tot = (int64_t*)(ws + oTot);
  int* full = (int*)(tot + 2);
  auto blocks = [](int64_t n) { return (int)((n + 255) / 256); };
  // exclusive scan of cnt[0..n) into scn; the total and the table-full flag to the host (synchronises)
  auto scan = [&](int64_t n, int64_t* total, int* hfull) -> int {
    const int64_t nb = (n + kScanThreads - 1) / kScanThreads;
    MK_COUNT(), k_scan_blocks<<<(int)nb, kScanThreads, 0, s>>>(n, cnt, scn, bsum);
    MK_COUNT(), k_scan_totals<<<1, 32, 0, s>>>(nb, bsum, tot);
    MK_COUNT(), k_scan_add<<<blocks(n), 256, 0, s>>>(n, scn, bsum);
    MK_CUDA(cudaMemcpyAsync(total, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    MK_CUDA(cudaMemcpyAsync(hfull, full, sizeof(int), cudaMemcpyDeviceToHost, s));
    MK_CUDA(cudaStreamSynchronize(s));
    MK_CUDA(cudaGetLastError());
    return MK_OK;
  };
  MK_CUDA(cudaMemsetAsync(full, 0, sizeof(int), s));
  MK_COUNT(), k_rf_check<<<blocks(n_elems), 256, 0, s>>>(n_elems, n_vertices, tets, tags, full);
  int bad = 0;
  MK_CUDA(cudaMemcpyAsync(&bad, full, sizeof(int), cudaMemcpyDeviceToHost, s));
  MK_CUDA(cudaStreamSynchronize(s));
  MK_ARG(!bad, "mk_refine: a vertex id out of range or a tag outside {1, 2, 3}");
  MK_COUNT(), k_rf_table_init<<<(int)((cap + 255) / 256), 256, 0, s>>>(cap, t);
  MK_COUNT(), k_iota<<<blocks(n_elems), 256, 0, s>>>(n_elems, parent);
  MK_CUDA(cudaMemcpyAsync(flag, marked, (size_t)n_elems, cudaMemcpyDeviceToDevice, s));
  int64_t E = n_elems, nv = n_vertices;
  int r = 0;
  for (;; ++r) {
    // the flagged elements and the places of their second children
    int64_t nflag = 0, nnew = 0;
    int hf = 0;
    MK_COUNT(), k_u8_to_i32<<<blocks(E), 256, 0, s>>>(E, flag, cnt);
    MK_TRY(scan(E, &nflag, &hf));
    if (nflag == 0) break;
    MK_ARG(r < 256, "mk_refine: closure did not end within 256 rounds");
    MK_ARG(E + nflag <= max_elems, "mk_refine: more elements than max_elems");
    MK_CUDA(cudaMemcpyAsync(pos, scn, (size_t)E * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    // their refinement edges, the owners of the new ones and the numbers of the new midpoints
    MK_COUNT(), k_rf_claim<<<blocks(E), 256, 0, s>>>(E, tets, tags, flag, t, full);
    MK_COUNT(), k_rf_own<<<blocks(E), 256, 0, s>>>(E, tets, tags, flag, t, cnt);
    MK_TRY(scan(E, &nnew, &hf));
    MK_ARG(!hf, "mk_refine: edge table full");
    MK_ARG(nv + nnew <= max_vertices, "mk_refine: more vertices than max_vertices");
    MK_COUNT(), k_rf_midpoints<<<blocks(E), 256, 0, s>>>(E, tets, tags, cnt, scn, nv, t, coords);
    MK_COUNT(), k_rf_bisect<<<blocks(E), 256, 0, s>>>(E, tets, tags, parent, flag, pos, t);
    E += nflag;
    nv += nnew;
    // closure: the elements that hold an edge already cut
    MK_COUNT(), k_rf_hanging<<<blocks(E), 256, 0, s>>>(E, tets, t, flag, cnt);
  }
  MK_CUDA(cudaGetLastError());
  *n_vertices_out = nv;
  *n_elems_out = E;
  if (rounds) *rounds = r;
  return MK_OK;
}
