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

}  // namespace mk
