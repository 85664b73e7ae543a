// Building blocks of the patch kernels (operator apply, learned preconditioner): vector loads, asynchronous
// staging of a patch into shared memory, and the shared-memory layout of one patch.
#pragma once

#include <cstdint>

#include "mk_device.cuh"

namespace mk {

// ------------------------------------------------------------------------------------------------ vectors
template <typename T, int VEC>
struct Vec {
  T v[VEC];
};

template <typename T, int VEC>
__device__ __forceinline__ Vec<T, VEC> ldv(const T* __restrict__ p) {
  Vec<T, VEC> r;
  if constexpr (VEC == 4 && sizeof(T) == 4) {
    const float4 f = *reinterpret_cast<const float4*>(p);
    r.v[0] = f.x; r.v[1] = f.y; r.v[2] = f.z; r.v[3] = f.w;
  } else if constexpr (VEC == 2 && sizeof(T) == 8) {
    const double2 f = *reinterpret_cast<const double2*>(p);
    r.v[0] = f.x; r.v[1] = f.y;
  } else {
#pragma unroll
    for (int c = 0; c < VEC; ++c) r.v[c] = p[c];
  }
  return r;
}

template <typename T, int VEC>
__device__ __forceinline__ void stv(T* __restrict__ p, const Vec<T, VEC>& r) {
  if constexpr (VEC == 4 && sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
  } else if constexpr (VEC == 2 && sizeof(T) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2(r.v[0], r.v[1]);
  } else {
#pragma unroll
    for (int c = 0; c < VEC; ++c) p[c] = r.v[c];
  }
}

// ------------------------------------------------------------------------------------------------ patch apply
// Asynchronous global -> shared copies (cp.async): every copy of a CTA is in flight at once, so staging a patch
// costs one memory latency instead of one per loop trip.
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Block-cooperative copy of nbytes (a multiple of 4) from the 4-byte aligned global address src into the 16-byte
// aligned shared region (nbytes + 16 bytes long).  The data land at region + (src mod 16), so the aligned body
// moves in 16-byte copies and only the head and tail in 4-byte ones; returns where src[0] landed.
template <typename U>
__device__ __forceinline__ const U* stage_async(unsigned char* region, const U* src, int nbytes) {
  const unsigned char* g = reinterpret_cast<const unsigned char*>(src);
  const int mis = (int)(reinterpret_cast<uintptr_t>(g) & 15);
  unsigned char* d = region + mis;
  const int head = min((16 - mis) & 15, nbytes);
  const int body = (nbytes - head) & ~15;
  const int tail = nbytes - head - body;
  for (int k = threadIdx.x; k < head / 4; k += blockDim.x) cp_async4(d + 4 * k, g + 4 * k);
  for (int k = threadIdx.x; k < body / 16; k += blockDim.x) cp_async16(d + head + 16 * k, g + head + 16 * k);
  for (int k = threadIdx.x; k < tail / 4; k += blockDim.x) cp_async4(d + head + body + 4 * k, g + head + body + 4 * k);
  return reinterpret_cast<const U*>(d);
}

// Row length of one packed element matrix of the patch operator, padded so that every row starts on a 16-byte
// boundary (55 -> 56 for P2 in FP32 or FP64, 10 -> 12 for P1 in FP32): rows load as whole 16-byte vectors.
__host__ __device__ constexpr int padded_np(int nloc, int tsize) {
  return (nloc * (nloc + 1) / 2 + 16 / tsize - 1) / (16 / tsize) * (16 / tsize);
}

// Shared-memory layout of one patch-apply CTA (byte offsets, each region 16-byte aligned).
struct PatchSmem {
  size_t ye, as, conn, inc, ioff, tgt, total;
};
__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }
__host__ __device__ inline PatchSmem patch_smem(int nloc, int pe, int max_nodes, int W, int tsize) {
  PatchSmem L;
  L.ye = 0;
  L.as = L.ye + align16((size_t)nloc * pe * W * tsize);
  L.conn = L.as + align16((size_t)pe * padded_np(nloc, tsize) * tsize + 16);
  L.inc = L.conn + align16((size_t)pe * nloc * 4 + 16);
  L.ioff = L.inc + align16((size_t)pe * nloc * 2 + 16);
  L.tgt = L.ioff + align16((size_t)(max_nodes + 1) * 4 + 16);
  L.total = L.tgt + align16((size_t)max_nodes * 4 + 16);
  return L;
}

// y = A x for one patch per CTA: owner-computes scatter, fixed summation order, no atomics.
// Staging: the patch's element matrices, connectivity, incidence lists and node targets are copied into shared
// memory asynchronously, all at once.  Phase 1: element products y_e = A_e x_e (x gathered from global, mostly L2
// hits) into shared memory laid out [slot][element][column]; one thread per element and group of VEC columns.
// Each element matrix is read from shared memory once (packed order), with all output rows held in registers.
// Phase 2: each local node sums its incidences in fixed order (shared memory only) and writes the global row
// (owned node) or its halo slot (shared node).  Columns [col0, col0 + W) with W = ncolg * VEC.
// Node targets of the patches: >= 0 a node written directly, with kOwnedBoundary set when it is a boundary node (its
// row is zeroed when the operator masks the boundary); < 0 a halo slot -(slot)-1.
constexpr int32_t kOwnedBoundary = 1 << 30;

template <int NLOC, typename T, int VEC, int NCG = 0>
__device__ __forceinline__ void patch_apply(int p, const int32_t* __restrict__ elem_off,
                                                     const int32_t* __restrict__ node_off,
                                                     const int32_t* __restrict__ conn, const T* __restrict__ Ae,
                                                     const int32_t* __restrict__ target,
                                                     const int32_t* __restrict__ inc_off,
                                                     const uint16_t* __restrict__ inc,
                                                     const uint8_t* __restrict__ bnd, int mask,
                                                     const T* __restrict__ x, T* __restrict__ y, T* __restrict__ halo,
                                                     int ncolg, int col0, int ld, int pe, int max_nodes,
                                                     unsigned char* smraw) {
  constexpr int NPS = padded_np(NLOC, (int)sizeof(T));
  const int ncg = NCG > 0 ? NCG : ncolg;  // column groups: a compile-time constant in the hot instances
  const int W = ncg * VEC;
  const PatchSmem lay = patch_smem(NLOC, pe, max_nodes, W, (int)sizeof(T));
  T* Ye = reinterpret_cast<T*>(smraw + lay.ye);  // [NLOC][pe][W]
  const int e0 = elem_off[p], ne = elem_off[p + 1] - e0;
  const int n0 = node_off[p], nl = node_off[p + 1] - n0;
  const int ibase = e0 * NLOC;  // the patch's incidences are inc[ibase, ibase + ne * NLOC)
  const T* As = stage_async(smraw + lay.as, Ae + (int64_t)e0 * NPS, ne * NPS * (int)sizeof(T));
  const int32_t* cs = stage_async(smraw + lay.conn, conn + ibase, ne * NLOC * 4);
  const uint16_t* is = stage_async(smraw + lay.inc, inc + ibase, ne * NLOC * 2);
  const int32_t* os = stage_async(smraw + lay.ioff, inc_off + n0, (nl + 1) * 4);
  const int32_t* ts = stage_async(smraw + lay.tgt, target + n0, nl * 4);
  cp_async_wait_all();
  __syncthreads();
  for (int it = threadIdx.x; it < ne * ncg; it += blockDim.x) {
    const int el = it / ncg, g = it - el * ncg;
    const T* xg = x + col0 + g * VEC;
    Vec<T, VEC> xv[NLOC];
#pragma unroll
    for (int a = 0; a < NLOC; ++a) xv[a] = ldv<T, VEC>(xg + cs[el * NLOC + a] * ld);
    // one pass over the packed upper triangle: each entry is read once and feeds rows a and b; nothing is
    // stored until every row is complete
    const T* A = As + el * NPS;
    Vec<T, VEC> acc[NLOC];
#pragma unroll
    for (int a = 0; a < NLOC; ++a)
#pragma unroll
      for (int c = 0; c < VEC; ++c) acc[a].v[c] = 0;
#pragma unroll
    for (int a = 0; a < NLOC; ++a)
#pragma unroll
      for (int b = a; b < NLOC; ++b) {
        const T w = A[sym_index(a, b, NLOC)];
#pragma unroll
        for (int c = 0; c < VEC; ++c) {
          acc[a].v[c] += w * xv[b].v[c];
          if (b != a) acc[b].v[c] += w * xv[a].v[c];
        }
      }
#pragma unroll
    for (int a = 0; a < NLOC; ++a) stv<T, VEC>(Ye + ((size_t)a * pe + el) * W + g * VEC, acc[a]);
  }
  __syncthreads();
  for (int it = threadIdx.x; it < nl * ncg; it += blockDim.x) {
    const int l = it / ncg, g = it - l * ncg;
    const int b = os[l] - ibase, e = os[l + 1] - ibase;
    Vec<T, VEC> acc;
#pragma unroll
    for (int c = 0; c < VEC; ++c) acc.v[c] = 0;
    auto ye = [&](int k) {  // product of incidence k (slot * pe + local element)
      return ldv<T, VEC>(Ye + (size_t)is[k] * W + g * VEC);
    };
    int k = b;
    for (; k + 4 <= e; k += 4) {  // four independent loads, then the sums in list order
      const Vec<T, VEC> v0 = ye(k), v1 = ye(k + 1), v2 = ye(k + 2), v3 = ye(k + 3);
#pragma unroll
      for (int c = 0; c < VEC; ++c) acc.v[c] = (((acc.v[c] + v0.v[c]) + v1.v[c]) + v2.v[c]) + v3.v[c];
    }
    for (; k < e; ++k) {
      const Vec<T, VEC> v = ye(k);
#pragma unroll
      for (int c = 0; c < VEC; ++c) acc.v[c] += v.v[c];
    }
    const int t = ts[l];
    if (t >= 0) {
      if (mask && (t & kOwnedBoundary))
#pragma unroll
        for (int c = 0; c < VEC; ++c) acc.v[c] = 0;
      stv<T, VEC>(y + (int64_t)(t & (kOwnedBoundary - 1)) * ld + col0 + g * VEC, acc);
    } else {
      stv<T, VEC>(halo + (int64_t)(-t - 1) * ld + col0 + g * VEC, acc);
    }
  }
}

// Shared nodes: y[node] = sum of the node's halo slots in patch order; item t = (shared node, column group).
template <typename T, int VEC>
__device__ __forceinline__ void halo_sum(int64_t t, int64_t nshared, const int32_t* __restrict__ node,
                                         const int32_t* __restrict__ off, const uint8_t* __restrict__ bnd, int mask,
                                         const T* __restrict__ halo, T* __restrict__ y, int ncolg, int col0, int ld) {
  if (t >= nshared * ncolg) return;
  const int64_t k = t / ncolg;
  const int g = (int)(t - k * ncolg);
  Vec<T, VEC> acc;
#pragma unroll
  for (int c = 0; c < VEC; ++c) acc.v[c] = 0;
  for (int s = off[k]; s < off[k + 1]; ++s) {
    const Vec<T, VEC> v = ldv<T, VEC>(halo + (int64_t)s * ld + col0 + g * VEC);
#pragma unroll
    for (int c = 0; c < VEC; ++c) acc.v[c] += v.v[c];
  }
  const int nd = node[k];
  if (mask && bnd[nd])
#pragma unroll
    for (int c = 0; c < VEC; ++c) acc.v[c] = 0;
  stv<T, VEC>(y + (int64_t)nd * ld + col0 + g * VEC, acc);
}

}  // namespace mk
