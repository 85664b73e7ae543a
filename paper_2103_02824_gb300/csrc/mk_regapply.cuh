// The FP32 element-by-element operator y = A x with the element matrices staged in registers.
//
// The operator streams one packed element matrix per element (55 values, padded to 56) and reads each only once,
// so the kernel is bound by how many of those bytes each SM keeps in flight, and by the shared-memory traffic of
// the element products.  Here each thread owns one element: it loads the element's matrix with 14 coalesced 16-byte
// loads straight into registers (a warp reads 32 consecutive matrices, 7 KB) while the CTA copies the patch's
// record into shared memory; then the x rows of the patch's nodes are staged (one cp.async per 16-byte chunk) and
// the element multiplies two columns at a time.  Several small CTAs per SM (one patch each) keep about 100 KB of
// matrices per SM in flight, and each CTA waits on memory only twice.  The products are placed in
// shared memory at their incidence in the patch's node-sorted incidence list, so that each local node then sums its
// rows in list order and writes its row of y (owned node) or its halo slot (shared node).  The arithmetic, and its order, is that of patch_apply,
// so the result is bitwise that of the other patch kernels.
#pragma once

#include "mk_patch.cuh"

namespace mk {

constexpr int kRegMaxThreads = 256;  // one element per thread: patches of at most this many elements

// Shared-memory layout of one patch CTA: the patch record, the x rows of its local nodes (W columns, rows padded
// to W + 4 floats), the products of one pass of 4 columns (16-byte rows).
struct RegSmem {
  size_t rec, xs, ye, total;
};
__host__ __device__ constexpr int reg_xs_stride(int W) { return W + 4; }
__host__ __device__ inline RegSmem reg_smem(int nloc, int pe, int max_nodes, int rec_stride, int W) {
  RegSmem L;
  L.rec = 0;
  L.xs = align16((size_t)rec_stride);
  L.ye = L.xs + align16((size_t)max_nodes * reg_xs_stride(W) * 4);
  L.total = L.ye + align16((size_t)nloc * pe * 4 * 4);
  return L;
}
// Physical row of product row r: the low three bits XOR the next three, a permutation within each aligned group of
// eight rows.  A node's products are consecutive rows and the nodes of a warp have runs of equal length (they are
// sorted by incidence count, and the counts are even on these meshes), so without it the lanes of a node-sum load
// would all hit one 16-byte bank group.
__device__ __forceinline__ int ye_row(int r) { return r ^ ((r >> 3) & 7); }

// Columns [col0, col0 + W) of y = A x for patch p (elements [p pe, p pe + ne), one per thread; W a multiple of 4,
// at most WMAX in {8, 32}: the element matrices are read once for all W columns).
// The record of patch p sits at rec + p * rec_stride (every record padded to that stride): the header {e0, ne, n0,
// nl, off_pos, off_ioff, off_tgt, off_gid}, the local connectivity (uint16, at byte kRecHeader), the incidence
// place of each (element, slot) (uint16), the start of each local node's run (uint16), the node targets (int32)
// and the local nodes' global ids (int32).  Two memory latencies per CTA: the record copy and the matrix loads go
// out together (neither needs an earlier load), then the x rows, whose ids come with the record.  Products and
// node sums then run in passes of 4 columns, from shared memory only.  A record whose header is out of range sets
// MK_FAULT_PATCH_RECORD and the CTA writes nothing.
template <int NLOC, int WMAX>
__device__ __forceinline__ void patch_apply_reg(int p, const unsigned char* __restrict__ rec, int rec_stride,
                                                const float* __restrict__ Ae, int mask, const float* __restrict__ x,
                                                float* __restrict__ y, float* __restrict__ halo, int col0, int W,
                                                int ld, int pe, int max_nodes, int64_t n_nodes, int64_t n_elems,
                                                int* __restrict__ fault, unsigned char* __restrict__ smraw) {
  constexpr int NPS = padded_np(NLOC, 4);
  constexpr int NV = NPS / 4;  // 16-byte vectors per element matrix
  static_assert(WMAX == 8 || WMAX == 32, "column block");
  const int XCH = W / 4;       // 16-byte chunks of an x row
  constexpr int XS = reg_xs_stride(WMAX);  // x row stride (floats): 48 bytes for WMAX = 8, so gathers spread over banks
  const RegSmem lay = reg_smem(NLOC, pe, max_nodes, rec_stride, WMAX);
  unsigned char* Rs = smraw + lay.rec;
  float* Xs = reinterpret_cast<float*>(smraw + lay.xs);
  float* Ye = reinterpret_cast<float*>(smraw + lay.ye);
  const int64_t e0 = (int64_t)p * pe;
  const int ne = (int)(n_elems - e0 < (int64_t)pe ? n_elems - e0 : (int64_t)pe);
  const int el = threadIdx.x;
  const bool mine = el < ne;
  // (1) the record into shared memory and the element's matrix into registers
  const unsigned char* rg = rec + (int64_t)p * rec_stride;
  for (int k = threadIdx.x; k < rec_stride / 16; k += blockDim.x) cp_async16(Rs + 16 * k, rg + 16 * k);
  float A[NPS];
  if (mine) {
    const float4* A4 = reinterpret_cast<const float4*>(Ae + (e0 + el) * NPS);
#pragma unroll
    for (int k = 0; k < NV; ++k) {  // read once: streaming loads that do not displace other data in L1
      const float4 v = __ldcs(A4 + k);
      A[4 * k] = v.x; A[4 * k + 1] = v.y; A[4 * k + 2] = v.z; A[4 * k + 3] = v.w;
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const int32_t* h = reinterpret_cast<const int32_t*>(Rs);
  const int nl = h[3];
  const bool sane = (int64_t)h[0] == e0 && h[1] == ne && ne >= 1 && ne <= (int)blockDim.x && nl >= 1 &&
                    nl <= max_nodes && h[4] >= kRecHeader && h[5] > h[4] && h[6] > h[5] && h[7] > h[6] &&
                    h[7] + 4 * nl <= rec_stride;
  if (!sane) {  // the same header for every thread: the whole CTA leaves
    if (threadIdx.x == 0) atomicOr(fault, MK_FAULT_PATCH_RECORD);
    return;
  }
  const uint16_t* cs = reinterpret_cast<const uint16_t*>(Rs + kRecHeader);
  const uint16_t* yp = reinterpret_cast<const uint16_t*>(Rs + h[4]);
  const uint16_t* os = reinterpret_cast<const uint16_t*>(Rs + h[5]);
  const int32_t* ts = reinterpret_cast<const int32_t*>(Rs + h[6]);
  const int32_t* gid = reinterpret_cast<const int32_t*>(Rs + h[7]);
  // (2) the x rows of the patch's local nodes, one 16-byte copy per chunk (a row is read once per patch)
  for (int k = threadIdx.x; k < nl * XCH; k += blockDim.x) {
    const int l = k / XCH, c = k - l * XCH;
    int64_t g = gid[l];
    if (g < 0 || g >= n_nodes) {  // a bad id: record it and copy row 0 instead
      atomicOr(fault, MK_FAULT_PATCH_RECORD);
      g = 0;
    }
    cp_async16(Xs + (size_t)l * XS + c * 4, x + g * ld + col0 + c * 4);
  }
  int lnd[NLOC];
  int pos[NLOC];
  if (mine)
#pragma unroll
    for (int a = 0; a < NLOC; ++a) {
      lnd[a] = cs[el * NLOC + a];
      pos[a] = ye_row(yp[el * NLOC + a]);
    }
  cp_async_wait_all();
  __syncthreads();
  // (3) per pass of 4 columns: element products (two columns at a time), then the node sums
  const int npass = W / 4;
#pragma unroll 2
  for (int pass = 0; pass < npass; ++pass) {
    if (mine) {
#pragma unroll
      for (int c = 0; c < 4; c += 2) {
        // two columns per instruction (packed FP32 FMA, each lane the fused multiply-add of the scalar form, in the
        // same order: bitwise the products of the other patch kernels)
        float2 xv[NLOC];
#pragma unroll
        for (int b = 0; b < NLOC; ++b)
          xv[b] = *reinterpret_cast<const float2*>(Xs + (size_t)lnd[b] * XS + pass * 4 + c);
        float2 acc[NLOC];
#pragma unroll
        for (int a = 0; a < NLOC; ++a) acc[a] = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int a = 0; a < NLOC; ++a)
#pragma unroll
          for (int b = a; b < NLOC; ++b) {
            const float wv = A[sym_index(a, b, NLOC)];
            const float2 w2 = make_float2(wv, wv);
            acc[a] = __ffma2_rn(w2, xv[b], acc[a]);
            if (b != a) acc[b] = __ffma2_rn(w2, xv[a], acc[b]);
          }
#pragma unroll
        for (int a = 0; a < NLOC; ++a) *reinterpret_cast<float2*>(Ye + (size_t)pos[a] * 4 + c) = acc[a];
      }
    }
    __syncthreads();
    for (int l = threadIdx.x; l < nl; l += blockDim.x) {
      const int e = os[l + 1];
      Vec<float, 4> acc;
#pragma unroll
      for (int q = 0; q < 4; ++q) acc.v[q] = 0;
      int k = os[l];
      for (; k + 4 <= e; k += 4) {
        const Vec<float, 4> v0 = ldv<float, 4>(Ye + (size_t)ye_row(k) * 4),
                            v1 = ldv<float, 4>(Ye + (size_t)ye_row(k + 1) * 4),
                            v2 = ldv<float, 4>(Ye + (size_t)ye_row(k + 2) * 4),
                            v3 = ldv<float, 4>(Ye + (size_t)ye_row(k + 3) * 4);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc.v[q] = (((acc.v[q] + v0.v[q]) + v1.v[q]) + v2.v[q]) + v3.v[q];
      }
      for (; k < e; ++k) {
        const Vec<float, 4> v = ldv<float, 4>(Ye + (size_t)ye_row(k) * 4);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc.v[q] += v.v[q];
      }
      const int tg = ts[l];
      const int cc = col0 + pass * 4;
      if (tg >= 0) {
        if (mask && (tg & kOwnedBoundary))
#pragma unroll
          for (int q = 0; q < 4; ++q) acc.v[q] = 0;
        stv<float, 4>(y + (int64_t)(tg & (kOwnedBoundary - 1)) * ld + cc, acc);
      } else {
        stv<float, 4>(halo + (int64_t)(-tg - 1) * ld + cc, acc);
      }
    }
    if (pass + 1 < npass) __syncthreads();  // the next pass rewrites the products
  }
}

}  // namespace mk
