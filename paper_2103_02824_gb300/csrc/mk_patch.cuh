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
  } else if constexpr (VEC == 2 && sizeof(T) == 4) {
    const float2 f = *reinterpret_cast<const float2*>(p);
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
  } else if constexpr (VEC == 2 && sizeof(T) == 4) {
    *reinterpret_cast<float2*>(p) = make_float2(r.v[0], r.v[1]);
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

// ------------------------------------------------------------------------------------------------ FP32-pair apply
// y = A x to about 48 significant bits on the FP32 units: A and x split into pairs hi + lo of FP32 values
// (hi = fl32(v), lo = fl32(v - hi)), each product hi_a hi_x formed exactly (the rounded product and its error by an
// FMA), the cross terms hi_a lo_x + lo_a hi_x added to that error (lo_a lo_x, 2^-48 of the product, is dropped), and
// the sum kept as hi + lo by an exact two-sum of the leading parts.  The element sums are then rounded to FP64 and
// the node sums run in FP64 exactly as in patch_apply.  GB300 runs FP32 at 64 times its FP64 rate, so the dozen
// FP32 operations per product take a fraction of the time of one FP64 multiply-add; the result differs from the FP64
// operator by a few units of 2^-48 relative to sum |a_ij x_j|.  The _rn intrinsics keep the compiler from fusing
// the steps of the error-free transformations.
__device__ __forceinline__ void pair_madd(float& hi, float& lo, float wh, float wl, float xh, float xl) {
  const float p = __fmul_rn(wh, xh);
  float e = __fmaf_rn(wh, xh, -p);  // wh xh = p + e exactly
  e = __fmaf_rn(wh, xl, e);
  e = __fmaf_rn(wl, xh, e);
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));  // hi + p = s + t exactly
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(t, e));
}

// Shared-memory layout of one FP32-pair patch CTA: FP64 products [NLOC][pe][W], hi and lo element matrices (FP32,
// padded rows), connectivity, incidences, node runs and targets.
struct PairSmem {
  size_t ye, ah, al, conn, inc, ioff, tgt, total;
};
__host__ __device__ inline PairSmem pair_smem(int nloc, int pe, int max_nodes, int W) {
  PairSmem L;
  const size_t am = (size_t)pe * padded_np(nloc, 4) * 4 + 16;
  L.ye = 0;
  L.ah = L.ye + align16((size_t)nloc * pe * W * 8);
  L.al = L.ah + align16(am);
  L.conn = L.al + align16(am);
  L.inc = L.conn + align16((size_t)pe * nloc * 4 + 16);
  L.ioff = L.inc + align16((size_t)pe * nloc * 2 + 16);
  L.tgt = L.ioff + align16((size_t)(max_nodes + 1) * 4 + 16);
  L.total = L.tgt + align16((size_t)max_nodes * 4 + 16);
  return L;
}

// One patch per CTA, as patch_apply: Ah, Al the pair parts of the element matrices (patch order, padded rows),
// xh, xl the pair parts of x [n_nodes * ld]; y and the halo slots in FP64.
template <int NLOC, int VEC, int NCG = 0>
__device__ __forceinline__ void patch_apply_pair(int p, const int32_t* __restrict__ elem_off,
                                                 const int32_t* __restrict__ node_off,
                                                 const int32_t* __restrict__ conn, const float* __restrict__ Ah,
                                                 const float* __restrict__ Al, const int32_t* __restrict__ target,
                                                 const int32_t* __restrict__ inc_off,
                                                 const uint16_t* __restrict__ inc, int mask,
                                                 const float* __restrict__ xh, const float* __restrict__ xl,
                                                 double* __restrict__ y, double* __restrict__ halo, int ncolg,
                                                 int col0, int ld, int pe, int max_nodes, unsigned char* smraw) {
  constexpr int NPS = padded_np(NLOC, 4);
  const int ncg = NCG > 0 ? NCG : ncolg;
  const int W = ncg * VEC;
  const PairSmem lay = pair_smem(NLOC, pe, max_nodes, W);
  double* Ye = reinterpret_cast<double*>(smraw + lay.ye);  // [NLOC][pe][W]
  const int e0 = elem_off[p], ne = elem_off[p + 1] - e0;
  const int n0 = node_off[p], nl = node_off[p + 1] - n0;
  const int ibase = e0 * NLOC;
  const float* Ahs = stage_async(smraw + lay.ah, Ah + (int64_t)e0 * NPS, ne * NPS * 4);
  const float* Als = stage_async(smraw + lay.al, Al + (int64_t)e0 * NPS, ne * NPS * 4);
  const int32_t* cs = stage_async(smraw + lay.conn, conn + ibase, ne * NLOC * 4);
  const uint16_t* is = stage_async(smraw + lay.inc, inc + ibase, ne * NLOC * 2);
  const int32_t* os = stage_async(smraw + lay.ioff, inc_off + n0, (nl + 1) * 4);
  const int32_t* ts = stage_async(smraw + lay.tgt, target + n0, nl * 4);
  cp_async_wait_all();
  __syncthreads();
  for (int it = threadIdx.x; it < ne * ncg; it += blockDim.x) {
    const int el = it / ncg, g = it - el * ncg;
    Vec<float, VEC> xvh[NLOC], xvl[NLOC];
#pragma unroll
    for (int a = 0; a < NLOC; ++a) {
      const int64_t o = (int64_t)cs[el * NLOC + a] * ld + col0 + g * VEC;
      xvh[a] = ldv<float, VEC>(xh + o);
      xvl[a] = ldv<float, VEC>(xl + o);
    }
    const float* AH = Ahs + el * NPS;
    const float* AL = Als + el * NPS;
    float hi[NLOC][VEC], lo[NLOC][VEC];
#pragma unroll
    for (int a = 0; a < NLOC; ++a)
#pragma unroll
      for (int c = 0; c < VEC; ++c) hi[a][c] = lo[a][c] = 0.0f;
#pragma unroll
    for (int a = 0; a < NLOC; ++a)
#pragma unroll
      for (int b = a; b < NLOC; ++b) {
        const float wh = AH[sym_index(a, b, NLOC)], wl = AL[sym_index(a, b, NLOC)];
#pragma unroll
        for (int c = 0; c < VEC; ++c) {
          pair_madd(hi[a][c], lo[a][c], wh, wl, xvh[b].v[c], xvl[b].v[c]);
          if (b != a) pair_madd(hi[b][c], lo[b][c], wh, wl, xvh[a].v[c], xvl[a].v[c]);
        }
      }
#pragma unroll
    for (int a = 0; a < NLOC; ++a) {
      Vec<double, VEC> o;
#pragma unroll
      for (int c = 0; c < VEC; ++c) o.v[c] = (double)hi[a][c] + (double)lo[a][c];
      stv<double, VEC>(Ye + ((size_t)a * pe + el) * W + g * VEC, o);
    }
  }
  __syncthreads();
  for (int it = threadIdx.x; it < nl * ncg; it += blockDim.x) {  // the node sums of patch_apply, in FP64
    const int l = it / ncg, g = it - l * ncg;
    const int b = os[l] - ibase, e = os[l + 1] - ibase;
    Vec<double, VEC> acc;
#pragma unroll
    for (int c = 0; c < VEC; ++c) acc.v[c] = 0;
    auto ye = [&](int k) { return ldv<double, VEC>(Ye + (size_t)is[k] * W + g * VEC); };
    int k = b;
    for (; k + 4 <= e; k += 4) {
      const Vec<double, VEC> v0 = ye(k), v1 = ye(k + 1), v2 = ye(k + 2), v3 = ye(k + 3);
#pragma unroll
      for (int c = 0; c < VEC; ++c) acc.v[c] = (((acc.v[c] + v0.v[c]) + v1.v[c]) + v2.v[c]) + v3.v[c];
    }
    for (; k < e; ++k) {
      const Vec<double, VEC> v = ye(k);
#pragma unroll
      for (int c = 0; c < VEC; ++c) acc.v[c] += v.v[c];
    }
    const int t = ts[l];
    if (t >= 0) {
      if (mask && (t & kOwnedBoundary))
#pragma unroll
        for (int c = 0; c < VEC; ++c) acc.v[c] = 0;
      stv<double, VEC>(y + (int64_t)(t & (kOwnedBoundary - 1)) * ld + col0 + g * VEC, acc);
    } else {
      stv<double, VEC>(halo + (int64_t)(-t - 1) * ld + col0 + g * VEC, acc);
    }
  }
}

// ------------------------------------------------------------------------------------------------ pipelined apply
// ------------------------------------------------------------------------------------------------ bulk copies
// mbarrier and bulk (TMA, non-tensor) copy primitives.  Every wait is bounded: a limit of polls of
// mbarrier.try_wait (each suspending the thread for at most about kSuspendNs), then the caller is told.  kWaitLimit
// is the default limit (about a second); a context may lower it for the waits of the patch kernel
// (mk_ctx_set_option), but the drain after a wait gave up always uses kWaitLimit.
constexpr int kWaitLimit = kWaitLimitDefault;
constexpr unsigned kSuspendNs = 1000;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// one arrival that also announces `bytes` more bytes of transactions for the current phase
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// waits for the phase of the given parity, suspending up to about kSuspendNs per call
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}
// the barrier's current phase also waits for every cp.async this thread issued before (an arrival counted in
// the barrier's initial count)
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int limit = kWaitLimit) {
  for (int i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// global -> shared bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned), completing on bar
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Shared-memory layout of the pipelined patch kernel: mbarriers, kRecBufs patch-record buffers, kAStages buffers
// of element matrices, two of local-node x rows, and two product buffers Ye [incidence][W].
constexpr int kAStages = 2;   // element matrices are fetched kAStages - 1 steps ahead
constexpr int kRecAhead = 3;  // records are fetched kRecAhead steps ahead
constexpr int kRecBufs = kRecAhead + 2;
struct StreamSmem {
  size_t bar, rec, rec_stride, as, as_stride, xs, xs_stride, ye, ye_stride, total;
};
__host__ __device__ inline StreamSmem stream_smem(int nloc, int pe, int max_nodes, int max_rec, int W, int tsize) {
  StreamSmem L;
  L.bar = 0;
  L.rec = 256;
  L.rec_stride = align16((size_t)max_rec);
  L.as = L.rec + kRecBufs * L.rec_stride;
  L.as_stride = align16((size_t)pe * padded_np(nloc, tsize) * tsize);
  L.xs = L.as + kAStages * L.as_stride;
  L.xs_stride = align16((size_t)max_nodes * W * tsize);
  L.ye = L.xs + 2 * L.xs_stride;
  L.ye_stride = align16((size_t)nloc * pe * W * tsize);
  L.total = L.ye + 2 * L.ye_stride;
  return L;
}
// 8 warps: warps 0-3 compute element products, warps 4-7 sum and copy.  With at most 128 registers a thread the CTA
// takes half an SM's registers, so a CTA of the coarse decomposition (run on another stream) fits beside it.
constexpr int kStreamThreads = 256;
constexpr int kStreamP1 = 128;

// y = A x (columns [col0, col0 + W)) over the patches blockIdx.x, blockIdx.x + gridDim.x, ... of one CTA,
// pipelined across two warp groups.  In step t the product group (threads [0, kStreamP1)) computes the element
// products of patch t, while the sum group (the other threads) sums the incidences of patch t - 1 and starts the
// copies for later patches: the element matrices of patch t + 1 (one bulk copy; they depend on the patch index
// only), the x rows of the local nodes of patch t + 1 (cp.async; their ids come with the patch's record, which
// arrived kRecAhead - 1 steps of slack earlier) and the record of patch t + kRecAhead (one bulk copy).  One CTA
// barrier ends the step.  So the two phases of the method overlap, and no copy waits on another within a step.
// Products: one item per (element, group of VEC columns); product row a of element e goes to the place of
// incidence (e, a) in the patch's node-sorted incidence list, so that a local node's incidences are consecutive
// rows.  Sums: one item per (local node, V2 columns), the node's rows in list order, written to its row of y
// (owned node) or to its halo slot (shared node).  Every sum has the terms and order of patch_apply, so both
// kernels give bitwise identical results.  The lanes that read one element matrix are neighbours (NCG >= 2), so
// its 16-byte loads are conflict-free at the packed row stride.
// Requires blockDim.x == kStreamThreads; patches of pe consecutive elements (the last one shorter); Ae, x
// 16-byte aligned; ld and col0 multiples of 16 / sizeof(T).  A record whose header is out of range, or a wait
// that gives up (after wait_limit polls), sets a bit of *fault and ends the CTA after a bounded wait (the default
// limit) for every copy it has issued.
template <int NLOC, typename T, int VEC, int NCG>
__device__ __forceinline__ void patch_apply_pipelined(const unsigned char* __restrict__ rec,
                                                      const int64_t* __restrict__ rec_off, const T* __restrict__ Ae,
                                                      int mask, const T* __restrict__ x, T* __restrict__ y,
                                                      T* __restrict__ halo, int col0, int ld, int pe, int max_nodes,
                                                      int max_rec, int n_patches, int64_t n_nodes, int64_t n_elems,
                                                      int* __restrict__ fault, int wait_limit,
                                                      unsigned char* smraw) {
  constexpr int NPS = padded_np(NLOC, (int)sizeof(T));
  constexpr int V2 = 16 / (int)sizeof(T);  // columns per sum item (one 16-byte vector)
  constexpr int W = NCG * VEC;
  constexpr int XCH = W / V2;              // 16-byte chunks per x row
  constexpr int NG2 = W / V2;
  constexpr int NSUM = kStreamThreads - kStreamP1;
  const StreamSmem lay = stream_smem(NLOC, pe, max_nodes, max_rec, W, (int)sizeof(T));
  uint64_t* barR = reinterpret_cast<uint64_t*>(smraw + lay.bar);  // [kRecBufs] records
  uint64_t* barM = barR + kRecBufs;                                // [kAStages] element matrices
  uint64_t* barX = barM + kAStages;                                // [2] x rows
  const int tid = threadIdx.x;
  const bool prod = tid < kStreamP1;
  const int gt = prod ? tid : tid - kStreamP1;  // thread index within its group
  const bool elected = tid == kStreamP1;        // issues the bulk copies
  const int np_mine = n_patches > (int)blockIdx.x ? (n_patches - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (np_mine == 0) return;
  auto patch_of = [&](int i) { return (int)blockIdx.x + i * (int)gridDim.x; };
  auto recbuf = [&](int i) { return smraw + lay.rec + (size_t)(i % kRecBufs) * lay.rec_stride; };
  auto hdr = [&](int i) { return reinterpret_cast<const int32_t*>(recbuf(i)); };
  // phases issued, and record phases seen complete, by this thread (for the drain after a failure)
  int rec_issued = 0, rec_waited = 0, mat_issued = 0, x_issued = 0;
  bool ok = true;
  auto issue_rec = [&](int i) {  // elected thread: the record of patch i
    if (elected) {
      const int64_t o = rec_off[patch_of(i)];
      const int64_t bytes = rec_off[patch_of(i) + 1] - o;
      if (bytes <= 0 || bytes > max_rec || (bytes & 15) || (o & 15)) {
        atomicOr(fault, MK_FAULT_PATCH_RECORD);
        *reinterpret_cast<int32_t*>(recbuf(i) + 4) = 0;  // ne = 0: the header check rejects the record
        mbar_arrive_expect(&barR[i % kRecBufs], 0);      // completes the phase with nothing copied
      } else {
        fence_proxy_async();
        mbar_arrive_expect(&barR[i % kRecBufs], (unsigned)bytes);
        bulk_g2s(recbuf(i), rec + o, (unsigned)bytes, &barR[i % kRecBufs]);
      }
    }
    ++rec_issued;
  };
  auto issue_mat = [&](int i) {  // elected thread: the element matrices of patch i (elements [p*pe, p*pe + ne))
    if (elected) {
      const int64_t e0 = (int64_t)patch_of(i) * pe;
      const int ne = (int)(n_elems - e0 < (int64_t)pe ? n_elems - e0 : (int64_t)pe);
      uint64_t* bar = &barM[i % kAStages];
      fence_proxy_async();
      const unsigned bytes = (unsigned)(ne * NPS * (int)sizeof(T));
      mbar_arrive_expect(bar, bytes);
      bulk_g2s(smraw + lay.as + (size_t)(i % kAStages) * lay.as_stride, Ae + e0 * NPS, bytes, bar);
    }
    ++mat_issued;
  };
  // waits for the record of patch i and checks its header (sizes within the launch's bounds; the elements those
  // of the patch index); both groups wait on it themselves (its buffer is rewritten only after patch i's sums).
  // Once a wait has failed no later one runs, so rec_waited counts exactly the leading phases seen complete.
  auto wait_rec = [&](int i) {
    if (!ok) return;
    const bool w = mbar_wait(&barR[i % kRecBufs], (unsigned)((i / kRecBufs) & 1), wait_limit);
    rec_waited += w;
    ok = ok && w;
    if (ok) {
      const int32_t* h = hdr(i);
      const bool sane = h[1] >= 1 && h[1] <= pe && h[3] >= 1 && h[3] <= max_nodes &&
                        (int64_t)h[0] == (int64_t)patch_of(i) * pe && (int64_t)h[0] + h[1] <= n_elems &&
                        h[4] >= kRecHeader && h[5] > h[4] && h[6] > h[5] && h[7] > h[6] && h[7] + 4 * h[3] <= max_rec;
      if (!sane) {
        if (elected) atomicOr(fault, MK_FAULT_PATCH_RECORD);
        ok = false;
      }
    }
  };
  // sum group: x rows of patch i (cp.async; each thread then arrives once its own copies land).  After a failed
  // wait the copies are skipped but the arrivals still happen, so the phase completes and the step's barrier
  // reports the failure.
  auto issue_x = [&](int i) {
    uint64_t* bar = &barX[i & 1];
    if (ok) {
      const int32_t* h = hdr(i);
      const int nl = h[3];
      const int32_t* gid = reinterpret_cast<const int32_t*>(recbuf(i) + h[7]);
      unsigned char* xs = smraw + lay.xs + (size_t)(i & 1) * lay.xs_stride;
      for (int k = gt; k < nl * XCH; k += NSUM) {
        const int l = k / XCH, j = k - l * XCH;
        int64_t g = gid[l];
        if (g < 0 || g >= n_nodes) {  // a bad id: record it and copy row 0 instead
          atomicOr(fault, MK_FAULT_PATCH_RECORD);
          g = 0;
        }
        cp_async16(xs + ((size_t)l * W + j * V2) * sizeof(T), x + g * ld + col0 + j * V2);
      }
    }
    cp_async_arrive(bar);
    ++x_issued;
  };
  // after a failure detected at the end of step t: the sum group, which issued every copy, waits (bounded) for the
  // record phases it has not seen complete and for the element-matrix and x phases of patches t onwards
  auto drain = [&](int t) {
    if (tid == 0) atomicOr(fault, MK_FAULT_PATCH_WAIT);
    if (prod) return;
    for (int k = rec_waited; k < rec_issued; ++k) mbar_wait(&barR[k % kRecBufs], (unsigned)((k / kRecBufs) & 1));
    for (int k = t; k < mat_issued; ++k) mbar_wait(&barM[k % kAStages], (unsigned)((k / kAStages) & 1));
    for (int k = t; k < x_issued; ++k) mbar_wait(&barX[k & 1], (unsigned)((k >> 1) & 1));
  };
  if (tid == 0) {
    for (int k = 0; k < kRecBufs; ++k) mbar_init(&barR[k], 1);
    for (int k = 0; k < kAStages; ++k) mbar_init(&barM[k], 1);
    for (int k = 0; k < 2; ++k) mbar_init(&barX[k], (unsigned)NSUM);  // the sum group's cp.async arrivals
    mbar_fence_init();
  }
  __syncthreads();
  for (int k = 0; k < kAStages - 1 && k < np_mine; ++k) issue_mat(k);
  for (int k = 0; k < kRecAhead && k < np_mine; ++k) issue_rec(k);
  if (!prod) {
    wait_rec(0);
    issue_x(0);
  }
  for (int t = 0; t <= np_mine; ++t) {
    if (!prod) {
      if (t + 1 < np_mine) {
        wait_rec(t + 1);
        issue_x(t + 1);
      }
      if (t + kAStages - 1 < np_mine) issue_mat(t + kAStages - 1);  // into the buffer of patch t - 1
      if (t + kRecAhead < np_mine) issue_rec(t + kRecAhead);  // into the buffer of record t - 2, read in step t - 1
      if (t >= 1 && ok) {                     // sums of patch t - 1
        const int i = t - 1;
        const int32_t* h = hdr(i);
        const int nl = h[3];
        const unsigned char* rb = recbuf(i);
        const uint16_t* os = reinterpret_cast<const uint16_t*>(rb + h[5]);
        const int32_t* ts = reinterpret_cast<const int32_t*>(rb + h[6]);
        const T* Ye = reinterpret_cast<const T*>(smraw + lay.ye + (size_t)(i & 1) * lay.ye_stride);
        for (int it = gt; it < nl * NG2; it += NSUM) {
          const int l = it / NG2, g = it - l * NG2;
          const int e = os[l + 1];
          Vec<T, V2> acc;
#pragma unroll
          for (int c = 0; c < V2; ++c) acc.v[c] = 0;
          const T* yr = Ye + g * V2;
          int k = os[l];
          for (; k + 4 <= e; k += 4) {
            const Vec<T, V2> v0 = ldv<T, V2>(yr + (size_t)k * W), v1 = ldv<T, V2>(yr + (size_t)(k + 1) * W),
                             v2 = ldv<T, V2>(yr + (size_t)(k + 2) * W), v3 = ldv<T, V2>(yr + (size_t)(k + 3) * W);
#pragma unroll
            for (int c = 0; c < V2; ++c) acc.v[c] = (((acc.v[c] + v0.v[c]) + v1.v[c]) + v2.v[c]) + v3.v[c];
          }
          for (; k < e; ++k) {
            const Vec<T, V2> v = ldv<T, V2>(yr + (size_t)k * W);
#pragma unroll
            for (int c = 0; c < V2; ++c) acc.v[c] += v.v[c];
          }
          const int tg = ts[l];
          if (tg >= 0) {
            if (mask && (tg & kOwnedBoundary))
#pragma unroll
              for (int c = 0; c < V2; ++c) acc.v[c] = 0;
            stv<T, V2>(y + (int64_t)(tg & (kOwnedBoundary - 1)) * ld + col0 + g * V2, acc);
          } else {
            stv<T, V2>(halo + (int64_t)(-tg - 1) * ld + col0 + g * V2, acc);
          }
        }
      }
    } else if (t < np_mine) {  // products of patch t
      wait_rec(t);
      ok = ok && mbar_wait(&barM[t % kAStages], (unsigned)((t / kAStages) & 1), wait_limit);
      ok = ok && mbar_wait(&barX[t & 1], (unsigned)((t >> 1) & 1), wait_limit);
      const int32_t* h = hdr(t);
      const int ne = h[1];
      const unsigned char* rb = recbuf(t);
      const uint16_t* cs = reinterpret_cast<const uint16_t*>(rb + kRecHeader);
      const uint16_t* yp = reinterpret_cast<const uint16_t*>(rb + h[4]);
      const T* As = reinterpret_cast<const T*>(smraw + lay.as + (size_t)(t % kAStages) * lay.as_stride);
      const T* Xs = reinterpret_cast<const T*>(smraw + lay.xs + (size_t)(t & 1) * lay.xs_stride);
      T* Ye = reinterpret_cast<T*>(smraw + lay.ye + (size_t)(t & 1) * lay.ye_stride);
      for (int it = gt; ok && it < ne * NCG; it += kStreamP1) {
        const int el = it / NCG, g = it - el * NCG;
        Vec<T, VEC> xv[NLOC];
#pragma unroll
        for (int a = 0; a < NLOC; ++a) xv[a] = ldv<T, VEC>(Xs + (int)cs[el * NLOC + a] * W + g * VEC);
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
            const T wv = A[sym_index(a, b, NLOC)];
#pragma unroll
            for (int c = 0; c < VEC; ++c) {
              acc[a].v[c] += wv * xv[b].v[c];
              if (b != a) acc[b].v[c] += wv * xv[a].v[c];
            }
          }
#pragma unroll
        for (int a = 0; a < NLOC; ++a) stv<T, VEC>(Ye + (size_t)yp[el * NLOC + a] * W + g * VEC, acc[a]);
      }
    }
    if (__syncthreads_or(!ok)) { drain(t); return; }
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
