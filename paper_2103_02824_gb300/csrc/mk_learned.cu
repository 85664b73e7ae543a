// Learned element-patch preconditioner: the network (FP32 master weights, Adam, BF16 inference copy), its
// forward pass on CUDA cores (FP32) and on the warp tensor cores (BF16 MMA, FP32 accumulation), the fused
// patch kernel that turns a residual into z = D^-1 r + (assembled network corrections) / multiplicity, the
// deterministic training gradient, Adam, and the harvest of training samples from solver iterates.
//
// Definitions (the library's own; the paper's boundary-value problems use standard solvers):
//   x   = [r_e / s, (v_k - centroid)/h_e],  s = ||r_e||_2, h_e = |det J_e|^(1/3)
//   y   = W3 relu(W2 relu(W1 x + b1) + b2) + b3
//   z   = r / diag(A) + (sum over incidences of y[slot] s / h_e) / multiplicity        (boundary rows 0)
//   L   = sum_s ||u_s y_s - e_s||^2 / sum_s u_s^2,  u = s / h_e, e = (x* - x_k) at the element's nodes
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mk_device.cuh"
#include "mk_patch.cuh"

namespace mk {

constexpr int kNH = MK_MLP_HIDDEN;  // hidden width (64)
constexpr int kK1 = 32;             // layer-1 input width of the tensor-core tile (n_in <= 22, zero padded)
constexpr int kS1 = 40;             // row stride in halves of the input tile and of W1 (conflict-free fragments)
constexpr int kS2 = 72;             // row stride in halves of W2 and W3
constexpr int kWbHalves = kNH * kS1 + kNH * kS2 + 16 * kS2;
constexpr int kBias = kNH + kNH + 16;
constexpr int kLW = 8;              // orbital columns per pass of the patch kernel

// Layer-1 input columns of the tensor-core tile (k = 0..31): the first half of the n_loc residual features at
// k = 0.., the second half at k = 8.., the 12 geometry features at k = 16..27, zeros elsewhere.  With this order
// the lane (g, t) of an m16n8k16 A fragment holds residual features 2t, 2t+1, H+2t, H+2t+1 (H = n_loc / 2) of rows
// g and g+8, so the patch kernel builds the residual half of the fragment in registers, and the geometry half is
// one ldmatrix from a per-element table.  Returns the network input index at column kt, or -1 for a zero column.
__host__ __device__ inline int tile_feature(int kt, int nloc) {
  const int H = nloc / 2;
  if (kt < 8) return kt < H ? kt : -1;
  if (kt < 16) return kt - 8 < nloc - H ? H + kt - 8 : -1;
  if (kt < 28) return nloc + kt - 16;
  return -1;
}

static inline int64_t mlp_count(int nin, int nout) {
  return (int64_t)kNH * nin + kNH + (int64_t)kNH * kNH + kNH + (int64_t)nout * kNH + nout;
}

// ------------------------------------------------------------------------------------------------ forward
// FP32 forward of one row on CUDA cores; w = flattened parameters (shared memory).
template <int NLOC>
__device__ __forceinline__ void mlp_row32(const float* __restrict__ w, const float (&x)[NLOC + 12],
                                          float (&y)[NLOC]) {
  constexpr int NIN = NLOC + 12;
  const float* W1 = w;
  const float* b1 = W1 + kNH * NIN;
  const float* W2 = b1 + kNH;
  const float* b2 = W2 + kNH * kNH;
  const float* W3 = b2 + kNH;
  const float* b3 = W3 + NLOC * kNH;
  float h1[kNH];
#pragma unroll
  for (int u = 0; u < kNH; ++u) {
    float z = b1[u];
#pragma unroll
    for (int k = 0; k < NIN; ++k) z = fmaf(W1[u * NIN + k], x[k], z);
    h1[u] = fmaxf(z, 0.f);
  }
#pragma unroll
  for (int o = 0; o < NLOC; ++o) y[o] = b3[o];
#pragma unroll 2
  for (int u = 0; u < kNH; ++u) {
    float z = b2[u];
#pragma unroll
    for (int k = 0; k < kNH; ++k) z = fmaf(W2[u * kNH + k], h1[k], z);
    const float h = fmaxf(z, 0.f);
#pragma unroll
    for (int o = 0; o < NLOC; ++o) y[o] = fmaf(W3[o * kNH + u], h, y[o]);
  }
}

// relu(lo), relu(hi) rounded to BF16 and packed (lo in the low half), one instruction
__device__ __forceinline__ uint32_t pack_relu_bf16(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;\n" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}


// D += A B for one m16n8k16 BF16 tile (FP32 accumulators), the warp-level tensor-core MMA.
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Four 8 x 8 BF16 matrices from shared memory (ldmatrix): lanes 8m .. 8m + 7 give the row addresses of matrix m,
// and register m of lane l receives row l / 4, columns 2 (l % 4) and + 1 of matrix m.
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const __nv_bfloat16* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

// The network on 16 rows by one warp.  Xs: 16 x kS1 BF16 inputs (columns >= n_in zero); W1b/W2b/W3b: BF16
// weights [out][in] with row strides kS1/kS2/kS2 halves (16-byte rows: every ldmatrix row address is aligned, and
// the strides put the eight rows of a matrix in distinct bank groups); bias: FP32 b1 | b2 | b3 (zero padded to 16).
// Fragment layout of m16n8k16 (g = lane / 4, t = lane % 4): A holds (row g | g+8, cols 2t, 2t+1 | 2t+8, 2t+9),
// B holds (k = 2t, 2t+1 | 2t+8, 2t+9; n = g), C holds (row g | g+8, cols 2t, 2t+1).  A comes from the input tile by
// ldmatrix (matrices: rows 0-7 / 8-15 x k 0-7 / 8-15 of a k-step), B from the weights by ldmatrix (rows n of an
// n-tile x consecutive 8-wide k blocks).  The accumulators start at the bias, and one cvt.relu turns two of them
// into a packed BF16 pair.  The C tiles of two neighbouring n-blocks are exactly the A fragment of the next
// layer's k-block, so hidden activations stay in registers.  out[nt][0..1]: row g, outputs
// nt*8 + 2t + {0,1}; out[nt][2..3]: row g + 8.
__device__ __forceinline__ void mlp_tile_bf16(const uint32_t (&a1)[2][4], const __nv_bfloat16* __restrict__ W1b,
                                              const __nv_bfloat16* __restrict__ W2b,
                                              const __nv_bfloat16* __restrict__ W3b,
                                              const float* __restrict__ bias, float (&out)[2][4]) {
  const int lane = threadIdx.x & 31, r8 = lane & 7, mm = lane >> 3, t = lane & 3;
  uint32_t h1[4][4], h2[4][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    uint32_t b[4];
    ldsm_x4(b, W1b + (nt * 8 + r8) * kS1 + 8 * mm);  // k blocks 0, 8, 16, 24
    const float b0 = bias[nt * 8 + 2 * t], b1 = bias[nt * 8 + 2 * t + 1];
    float c[4] = {b0, b1, b0, b1};  // the accumulators start at the bias
    mma_bf16(c, a1[0], b[0], b[1]);
    mma_bf16(c, a1[1], b[2], b[3]);
    h1[nt >> 1][(nt & 1) * 2 + 0] = pack_relu_bf16(c[0], c[1]);
    h1[nt >> 1][(nt & 1) * 2 + 1] = pack_relu_bf16(c[2], c[3]);
  }
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    uint32_t b[2][4];
    ldsm_x4(b[0], W2b + (nt * 8 + r8) * kS2 + 8 * mm);       // k blocks 0, 8, 16, 24
    ldsm_x4(b[1], W2b + (nt * 8 + r8) * kS2 + 32 + 8 * mm);  // k blocks 32, 40, 48, 56
    const float b0 = bias[kNH + nt * 8 + 2 * t], b1 = bias[kNH + nt * 8 + 2 * t + 1];
    float c[4] = {b0, b1, b0, b1};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) mma_bf16(c, h1[kk], b[kk >> 1][(kk & 1) * 2], b[kk >> 1][(kk & 1) * 2 + 1]);
    h2[nt >> 1][(nt & 1) * 2 + 0] = pack_relu_bf16(c[0], c[1]);
    h2[nt >> 1][(nt & 1) * 2 + 1] = pack_relu_bf16(c[2], c[3]);
  }
#pragma unroll
  for (int nt = 0; nt < 2; ++nt) {
    uint32_t b[2][4];
    ldsm_x4(b[0], W3b + (nt * 8 + r8) * kS2 + 8 * mm);
    ldsm_x4(b[1], W3b + (nt * 8 + r8) * kS2 + 32 + 8 * mm);
    const float b0 = bias[2 * kNH + nt * 8 + 2 * t], b1 = bias[2 * kNH + nt * 8 + 2 * t + 1];
    float c[4] = {b0, b1, b0, b1};
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) mma_bf16(c, h2[kk], b[kk >> 1][(kk & 1) * 2], b[kk >> 1][(kk & 1) * 2 + 1]);
#pragma unroll
    for (int i = 0; i < 4; ++i) out[nt][i] = c[i];
  }
}

// Y = network(X) on CUDA cores, one thread per row.
template <int NLOC>
__global__ void k_mlp_forward32(int64_t S, const float* __restrict__ w, int64_t count, const float* __restrict__ X,
                                float* __restrict__ Y) {
  extern __shared__ float wsm[];
  for (int64_t k = threadIdx.x; k < count; k += blockDim.x) wsm[k] = w[k];
  __syncthreads();
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  constexpr int NIN = NLOC + 12;
  float x[NIN], y[NLOC];
#pragma unroll
  for (int k = 0; k < NIN; ++k) x[k] = X[s * NIN + k];
  mlp_row32<NLOC>(wsm, x, y);
#pragma unroll
  for (int o = 0; o < NLOC; ++o) Y[s * NLOC + o] = y[o];
}

// The same with the layer-1 input fragments loaded from a 16-row tile Xs (row stride kS1 halves).
__device__ __forceinline__ void mlp_tile_bf16(const __nv_bfloat16* __restrict__ Xs,
                                              const __nv_bfloat16* __restrict__ W1b,
                                              const __nv_bfloat16* __restrict__ W2b,
                                              const __nv_bfloat16* __restrict__ W3b,
                                              const float* __restrict__ bias, float (&out)[2][4]) {
  const int lane = threadIdx.x & 31, r8 = lane & 7, mm = lane >> 3;
  uint32_t a1[2][4];
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) ldsm_x4(a1[ks], Xs + (r8 + 8 * (mm & 1)) * kS1 + 16 * ks + 8 * (mm >> 1));
  mlp_tile_bf16(a1, W1b, W2b, W3b, bias, out);
}

// Two floats as a packed BF16 pair (lo in the low half), round to nearest even.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Y = network(X) on the tensor cores (BF16), one warp per 16 rows.
template <int NLOC>
__global__ void __launch_bounds__(256) k_mlp_forward16(int64_t S, const __nv_bfloat16* __restrict__ wb,
                                                      const float* __restrict__ bias, const float* __restrict__ X,
                                                      float* __restrict__ Y) {
  constexpr int NIN = NLOC + 12;
  __shared__ __align__(16) __nv_bfloat16 wsm[kWbHalves];
  __shared__ float bsm[kBias];
  __shared__ __align__(16) __nv_bfloat16 xt[8][16 * kS1];
  for (int k = threadIdx.x; k < kWbHalves; k += blockDim.x) wsm[k] = wb[k];
  for (int k = threadIdx.x; k < kBias; k += blockDim.x) bsm[k] = bias[k];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tile = (int64_t)blockIdx.x * 8 + warp;
  if (tile * 16 >= S) return;
  __nv_bfloat16* Xs = xt[warp];
  {
    const int i = lane & 15, half = lane >> 4;
    const int64_t row = tile * 16 + i;
    for (int k = half * 16; k < half * 16 + 16; ++k) {
      const int f = tile_feature(k, NLOC);
      Xs[i * kS1 + k] = __float2bfloat16_rn((row < S && f >= 0) ? X[row * NIN + f] : 0.f);
    }
  }
  __syncwarp();
  float out[2][4];
  mlp_tile_bf16(Xs, wsm, wsm + kNH * kS1, wsm + kNH * kS1 + kNH * kS2, bsm, out);
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int hr = 0; hr < 2; ++hr) {
    const int64_t row = tile * 16 + g + 8 * hr;
    if (row >= S) continue;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int o = nt * 8 + 2 * t + q;
        if (o < NLOC) Y[row * NLOC + o] = out[nt][2 * hr + q];
      }
  }
}

// BF16 copy of the parameters in the padded tensor-core layout, FP32 biases.
__global__ void k_mlp_pack(const float* __restrict__ w, int nin, int nout, __nv_bfloat16* __restrict__ wb,
                           float* __restrict__ bias) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const float* W1 = w;
  const float* b1 = W1 + kNH * nin;
  const float* W2 = b1 + kNH;
  const float* b2 = W2 + kNH * kNH;
  const float* W3 = b2 + kNH;
  const float* b3 = W3 + nout * kNH;
  if (i < kNH * kS1) {
    const int u = i / kS1, k = i % kS1;
    const int f = k < kK1 ? tile_feature(k, nin - 12) : -1;
    wb[i] = __float2bfloat16_rn(f >= 0 ? W1[u * nin + f] : 0.f);
  } else if (i < kNH * kS1 + kNH * kS2) {
    const int j = i - kNH * kS1, u = j / kS2, k = j % kS2;
    wb[i] = __float2bfloat16_rn(k < kNH ? W2[u * kNH + k] : 0.f);
  } else if (i < kWbHalves) {
    const int j = i - kNH * kS1 - kNH * kS2, o = j / kS2, k = j % kS2;
    wb[i] = __float2bfloat16_rn((o < nout && k < kNH) ? W3[o * kNH + k] : 0.f);
  }
  if (i < kBias) bias[i] = i < kNH ? b1[i] : i < 2 * kNH ? b2[i - kNH] : (i - 2 * kNH < nout ? b3[i - 2 * kNH] : 0.f);
}

// ------------------------------------------------------------------------------------------------ preconditioner
struct LearnSmem {
  size_t ye, rs, conn, inc, ioff, tgt, geo, w, gb, total;
};
__host__ __device__ inline LearnSmem learn_smem(int nloc, int pe, int max_nodes, bool tc, int64_t count, int nwarps) {
  LearnSmem L;
  L.ye = 0;
  L.rs = L.ye + align16((size_t)nloc * pe * kLW * 4);                 // residual rows of the local nodes
  L.conn = L.rs + align16((size_t)max_nodes * kLW * 4);              // local node of each element slot (uint16)
  L.inc = L.conn + align16((size_t)pe * nloc * 2 + 16);
  L.ioff = L.inc + align16((size_t)pe * nloc * 2 + 16);
  L.tgt = L.ioff + align16((size_t)(max_nodes + 1) * 4 + 16);
  L.geo = L.tgt + align16((size_t)max_nodes * 4 + 16);
  L.w = L.geo + align16((size_t)pe * 16 * 4 + 16);
  const size_t wbytes = tc ? (size_t)kWbHalves * 2 + 16 + (size_t)kBias * 4 + 16 : (size_t)count * 4 + 16;
  L.gb = L.w + align16(wbytes);                                        // BF16 geometry table [element][16]
  L.total = L.gb + (tc ? align16((size_t)pe * 16 * 2) : 0);
  return L;
}

// One patch per CTA (the patches of the operator apply).  Phase 1: the network on every (element, column) row
// of the patch, scaled by s / h_e, into shared memory [slot][element][column]; on the tensor cores (TC) one
// warp takes 16 rows at a time (the layer-1 fragments built in registers, see tile_feature), otherwise one
// thread per row in FP32.  Phase 2: per local node the incidences
// in fixed order, then z = sum / multiplicity + r / diag (owned nodes) or the partial sum to the node's halo
// slot (shared nodes, finished by k_learned_halo).  Columns [col0, col0 + Nw), Nw = min(kLW, N - col0).
template <int NLOC, bool TC>
__global__ void __launch_bounds__(256, 2) k_learned_patch(
    const int32_t* __restrict__ elem_off, const int32_t* __restrict__ node_off, const uint16_t* __restrict__ lconn,
    const int32_t* __restrict__ node_gid, const int32_t* __restrict__ target, const int32_t* __restrict__ inc_off,
    const uint16_t* __restrict__ inc,
    const float* __restrict__ geomf, const void* __restrict__ wsrc, const float* __restrict__ bias, int64_t count,
    const float* __restrict__ dinv, const float* __restrict__ inv_mult, const uint8_t* __restrict__ bnd,
    const float* __restrict__ r, float* __restrict__ z, float* __restrict__ halo, int N, int col0, int ld, int pe,
    int max_nodes) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nwarps = blockDim.x >> 5;
  const LearnSmem lay = learn_smem(NLOC, pe, max_nodes, TC, count, nwarps);
  float* Ye = reinterpret_cast<float*>(smraw + lay.ye);
  const int p = blockIdx.x;
  const int e0 = elem_off[p], ne = elem_off[p + 1] - e0;
  const int n0 = node_off[p], nl = node_off[p + 1] - n0;
  const int ibase = e0 * NLOC;
  const int Nw = min(kLW, N - col0);
  const uint16_t* cs = stage_async(smraw + lay.conn, lconn + ibase, ne * NLOC * 2);
  // the residual rows of the patch's local nodes, columns [col0, col0 + 8) (16-byte copies; ld % 4 == 0)
  float* rs = reinterpret_cast<float*>(smraw + lay.rs);
  const int nvec = min(kLW, ld - col0) / 4;
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    const float* src = r + (int64_t)node_gid[n0 + l] * ld + col0;
    for (int v = 0; v < nvec; ++v) cp_async16(rs + l * kLW + 4 * v, src + 4 * v);
  }
  const uint16_t* is = stage_async(smraw + lay.inc, inc + ibase, ne * NLOC * 2);
  const int32_t* os = stage_async(smraw + lay.ioff, inc_off + n0, (nl + 1) * 4);
  const int32_t* ts = stage_async(smraw + lay.tgt, target + n0, nl * 4);
  const float* gs = stage_async(smraw + lay.geo, geomf + (int64_t)e0 * 16, ne * 16 * 4);
  const unsigned char* wsm;
  const float* bsm = nullptr;
  if constexpr (TC) {
    wsm = stage_async(smraw + lay.w, reinterpret_cast<const unsigned char*>(wsrc), kWbHalves * 2);
    bsm = stage_async(smraw + lay.w + align16((size_t)kWbHalves * 2 + 16), bias, kBias * 4);
  } else {
    wsm = stage_async(smraw + lay.w, reinterpret_cast<const unsigned char*>(wsrc), (int)(count * 4));
  }
  cp_async_wait_all();
  __syncthreads();
  const int nrows = ne * Nw;
  if constexpr (TC) {
    // the geometry features of the patch's elements in BF16, one 32-byte row per element (columns 12-15 zero)
    __nv_bfloat16* gbw = reinterpret_cast<__nv_bfloat16*>(smraw + lay.gb);
    for (int i = threadIdx.x; i < ne * 8; i += blockDim.x) {
      const int el = i >> 3, c = 2 * (i & 7);
      reinterpret_cast<uint32_t*>(gbw)[i] =
          pack_bf16(c < 12 ? gs[el * 16 + 1 + c] : 0.f, c + 1 < 12 ? gs[el * 16 + 2 + c] : 0.f);
    }
    __syncthreads();
    const __nv_bfloat16* gbt = gbw;
    const __nv_bfloat16* W1b = reinterpret_cast<const __nv_bfloat16*>(wsm);
    const __nv_bfloat16* W2b = W1b + kNH * kS1;
    const __nv_bfloat16* W3b = W2b + kNH * kS2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3, r8 = lane & 7, mm = lane >> 3;
    constexpr int H = NLOC / 2;
    const int fa = 2 * t, fb = 2 * t + 1;  // this lane's residual features fa, fb, H + fa, H + fb (those < H)
    // row / Nw as (row * ceil(2^16 / Nw)) >> 16: the ceiling adds less than row / 2^16, which stays below 1 / Nw
    // for row < 2^16 / Nw (8,192 for Nw = 8; a patch has at most 512 * 8 rows), so the quotient is exact
    const unsigned mnw = (65536u + (unsigned)Nw - 1u) / (unsigned)Nw;
    for (int tile = warp; tile * 16 < nrows; tile += nwarps) {
      uint32_t a1[2][4];
      int el[2], jj[2];
      float sc[2];
#pragma unroll
      for (int hr = 0; hr < 2; ++hr) {  // rows g and g + 8 of the tile
        const int row = tile * 16 + g + 8 * hr;
        const bool valid = row < nrows;
        const int e = valid ? (int)(((unsigned)row * mnw) >> 16) : 0;
        el[hr] = e;
        jj[hr] = valid ? row - e * Nw : 0;
        const uint16_t* ce = cs + e * NLOC;
        const float* rj = rs + jj[hr];
        const float v0 = (valid && fa < H) ? rj[ce[fa] * kLW] : 0.f;
        const float v1 = (valid && fb < H) ? rj[ce[fb] * kLW] : 0.f;
        const float v2 = (valid && fa < H) ? rj[ce[H + fa] * kLW] : 0.f;
        const float v3 = (valid && fb < H) ? rj[ce[H + fb] * kLW] : 0.f;
        float ss = fmaf(v3, v3, fmaf(v2, v2, fmaf(v1, v1, v0 * v0)));
        ss += __shfl_xor_sync(0xffffffffu, ss, 1);  // the row's four lanes hold all its features
        ss += __shfl_xor_sync(0xffffffffu, ss, 2);
        const float s = sqrtf(ss);
        const float inv = s > 0.f ? 1.f / s : 0.f;
        a1[0][hr] = pack_bf16(v0 * inv, v1 * inv);      // k = 2t, 2t+1
        a1[0][2 + hr] = pack_bf16(v2 * inv, v3 * inv);  // k = 8 + 2t, 8 + 2t + 1
        sc[hr] = valid ? s / gs[e * 16] : 0.f;
      }
      {  // geometry k-step: matrix mm holds rows (mm & 1) * 8 .. + 7, columns 16 + 8 * (mm >> 1) .. + 7
        const int row = tile * 16 + r8 + 8 * (mm & 1);
        const int e = row < nrows ? (int)(((unsigned)row * mnw) >> 16) : 0;
        ldsm_x4(a1[1], gbt + e * 16 + 8 * (mm >> 1));
      }
      float out[2][4];
      mlp_tile_bf16(a1, W1b, W2b, W3b, bsm, out);
#pragma unroll
      for (int hr = 0; hr < 2; ++hr) {
        if (tile * 16 + g + 8 * hr < nrows) {
#pragma unroll
          for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const int o = nt * 8 + 2 * t + q;
              if (o < NLOC) Ye[((size_t)o * pe + el[hr]) * kLW + jj[hr]] = out[nt][2 * hr + q] * sc[hr];
            }
        }
      }
    }
  } else {
    const float* wf = reinterpret_cast<const float*>(wsm);
    for (int row = threadIdx.x; row < nrows; row += blockDim.x) {
      const int el = row / Nw, jj = row - el * Nw;
      float x[NLOC + 12], y[NLOC], ss = 0.f;
#pragma unroll
      for (int a = 0; a < NLOC; ++a) {
        x[a] = rs[cs[el * NLOC + a] * kLW + jj];
        ss = fmaf(x[a], x[a], ss);
      }
      const float s = sqrtf(ss);
      const float inv = s > 0.f ? 1.f / s : 0.f;
#pragma unroll
      for (int a = 0; a < NLOC; ++a) x[a] *= inv;
#pragma unroll
      for (int k = 0; k < 12; ++k) x[NLOC + k] = gs[el * 16 + 1 + k];
      mlp_row32<NLOC>(wf, x, y);
      const float sc = s / gs[el * 16];
#pragma unroll
      for (int o = 0; o < NLOC; ++o) Ye[((size_t)o * pe + el) * kLW + jj] = y[o] * sc;
    }
  }
  __syncthreads();
  for (int it = threadIdx.x; it < nl * Nw; it += blockDim.x) {
    const int l = it / Nw, jj = it - l * Nw;
    const int b = os[l] - ibase, e = os[l + 1] - ibase;
    float acc = 0.f;
    for (int k = b; k < e; ++k) acc += Ye[(size_t)is[k] * kLW + jj];
    const int tg = ts[l];
    if (tg >= 0) {
      const int nd = tg & (kOwnedBoundary - 1);
      const int64_t t = (int64_t)nd * ld + col0 + jj;
      z[t] = (tg & kOwnedBoundary) ? 0.f : fmaf(acc, inv_mult[nd], dinv[nd] * r[t]);
    } else {
      halo[(int64_t)(-tg - 1) * ld + col0 + jj] = acc;
    }
  }
}

// Shared nodes: z = (sum of the node's halo slots in patch order) / multiplicity + r / diag.
__global__ void k_learned_halo(int64_t nshared, const int32_t* __restrict__ node, const int32_t* __restrict__ off,
                               const uint8_t* __restrict__ bnd, const float* __restrict__ halo,
                               const float* __restrict__ inv_mult, const float* __restrict__ dinv,
                               const float* __restrict__ r, float* __restrict__ z, int Nw, int col0, int ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nshared * Nw) return;
  const int64_t k = t / Nw;
  const int jj = (int)(t - k * Nw);
  float acc = 0.f;
  for (int s = off[k]; s < off[k + 1]; ++s) acc += halo[(int64_t)s * ld + col0 + jj];
  const int nd = node[k];
  const int64_t i = (int64_t)nd * ld + col0 + jj;
  z[i] = bnd[nd] ? 0.f : fmaf(acc, inv_mult[nd], dinv[nd] * r[i]);
}

int learned_apply(mk_ctx* ctx, const mk_mesh* m, const mk_mlp* mlp, const float* dinv, const float* r, float* z,
                  int ld, int N, int precision, cudaStream_t s) {
  const Patches& P = m->patches;
  const Level& L = m->fine;
  MK_ARG(mlp->nloc == L.nloc, "learned preconditioner: network built for another element order");
  MK_ARG(precision == MK_MLP_FP32 || precision == MK_MLP_BF16, "learned preconditioner: bad precision");
  MK_ARG(ld % 4 == 0, "learned preconditioner: ld must be a multiple of 4");
  int err = MK_OK;
  float* halo = (float*)scratch(ctx, S_LHALO, (size_t)std::max<int64_t>(P.n_halo_slots, 1) * ld * sizeof(float), &err);
  if (!halo) return err;
  const bool tc = precision == MK_MLP_BF16;
  const int th = 256;
  const LearnSmem lay = learn_smem(L.nloc, P.max_elems, P.max_nodes, tc, mlp->count, th / 32);
  MK_ARG(lay.total <= 227 * 1024, "learned preconditioner: patch too large for shared memory");
  const void* wsrc = tc ? mlp->d_wb : (const void*)mlp->d_w;
  for (int col0 = 0; col0 < N; col0 += kLW) {
    const int Nw = std::min(kLW, N - col0);
#define MK_LEARN_LAUNCH(NL, TCV)                                                                                   \
  do {                                                                                                            \
    auto kern = k_learned_patch<NL, TCV>;                                                                         \
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total);                     \
    MK_COUNT(), kern<<<P.n_patches, th, lay.total, s>>>(P.d_patch_elem_off, P.d_patch_node_off, P.d_lconn,        \
                                                        P.d_node_gid, P.d_node_target, P.d_inc_off, P.d_inc,      \
                                                        P.d_geomf, wsrc,                                          \
                                                        mlp->d_bias, mlp->count, dinv, P.d_inv_mult, L.d_boundary, \
                                                        r, z, halo, N, col0, ld, P.max_elems, P.max_nodes);       \
  } while (0)
    if (L.nloc == 4) {
      if (tc) MK_LEARN_LAUNCH(4, true); else MK_LEARN_LAUNCH(4, false);
    } else {
      if (tc) MK_LEARN_LAUNCH(10, true); else MK_LEARN_LAUNCH(10, false);
    }
#undef MK_LEARN_LAUNCH
    const int64_t work = P.n_shared_nodes * Nw;
    if (work > 0)
      MK_COUNT(), k_learned_halo<<<(int)((work + 255) / 256), 256, 0, s>>>(P.n_shared_nodes, P.d_shared_node,
                                                                          P.d_shared_off, L.d_boundary, halo,
                                                                          P.d_inv_mult, dinv, r, z, Nw, col0, ld);
  }
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

// ------------------------------------------------------------------------------------------------ training
constexpr int kCH = 64;  // samples per chunk of the gradient kernel

// Gradient of sum_s ||u_s y_s - e_s||^2 (and that sum, and sum_s u_s^2) over the batch, FP32 products.
// Block b takes chunks b, b + gridDim.x, ... of kCH samples and accumulates its own partial gradient in shared
// memory; every sum runs in a fixed order, so the result does not depend on scheduling.
template <int NLOC>
__global__ void __launch_bounds__(256) k_mlp_grad(const float* __restrict__ w, int64_t count,
                                                 const float* __restrict__ X, const float* __restrict__ U,
                                                 const float* __restrict__ Eg, const int32_t* __restrict__ idx,
                                                 int64_t S, float* __restrict__ part, double* __restrict__ part2) {
  constexpr int NIN = NLOC + 12, NOUT = NLOC;
  extern __shared__ float sm[];
  float* Wl = sm;
  float* G = Wl + count;
  float* Xc = G + count;
  float* Z1 = Xc + kCH * NIN;
  float* Z2 = Z1 + kCH * kNH;
  float* D3 = Z2 + kCH * kNH;
  float* Uc = D3 + kCH * NOUT;
  __shared__ double red[2][256];
  const float* W1 = Wl;
  const float* b1 = W1 + kNH * NIN;
  const float* W2 = b1 + kNH;
  const float* b2 = W2 + kNH * kNH;
  const float* W3 = b2 + kNH;
  const float* b3 = W3 + NOUT * kNH;
  const int64_t oW1 = 0, ob1 = kNH * NIN, oW2 = ob1 + kNH, ob2 = oW2 + kNH * kNH, oW3 = ob2 + kNH,
                ob3 = oW3 + NOUT * kNH;
  for (int64_t k = threadIdx.x; k < count; k += blockDim.x) {
    Wl[k] = w[k];
    G[k] = 0.f;
  }
  double lacc = 0.0, uacc = 0.0;
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int64_t c = blockIdx.x; c * kCH < S; c += gridDim.x) {
    const int ns = (int)min((int64_t)kCH, S - c * kCH);
    __syncthreads();
    for (int i = tid; i < kCH * NIN; i += nth) {
      const int s = i / NIN, k = i - s * NIN;
      const int64_t row = s < ns ? (idx ? idx[c * kCH + s] : c * kCH + s) : 0;
      Xc[i] = s < ns ? X[row * NIN + k] : 0.f;
    }
    for (int i = tid; i < kCH * NOUT; i += nth) {
      const int s = i / NOUT, o = i - s * NOUT;
      const int64_t row = s < ns ? (idx ? idx[c * kCH + s] : c * kCH + s) : 0;
      D3[i] = s < ns ? Eg[row * NOUT + o] : 0.f;
    }
    for (int s = tid; s < kCH; s += nth) {
      const int64_t row = s < ns ? (idx ? idx[c * kCH + s] : c * kCH + s) : 0;
      Uc[s] = s < ns ? U[row] : 0.f;
      if (s < ns) uacc += (double)Uc[s] * Uc[s];
    }
    __syncthreads();
    for (int i = tid; i < kCH * kNH; i += nth) {  // z1 = W1 x + b1
      const int s = i / kNH, u = i - s * kNH;
      float a = b1[u];
      for (int k = 0; k < NIN; ++k) a = fmaf(W1[u * NIN + k], Xc[s * NIN + k], a);
      Z1[i] = a;
    }
    __syncthreads();
    for (int i = tid; i < kCH * kNH; i += nth) {  // z2 = W2 relu(z1) + b2
      const int s = i / kNH, u = i - s * kNH;
      float a = b2[u];
      for (int k = 0; k < kNH; ++k) a = fmaf(W2[u * kNH + k], fmaxf(Z1[s * kNH + k], 0.f), a);
      Z2[i] = a;
    }
    __syncthreads();
    for (int i = tid; i < kCH * NOUT; i += nth) {  // y, residual u y - e, dL/dy = 2 u (u y - e)
      const int s = i / NOUT, o = i - s * NOUT;
      float a = b3[o];
      for (int k = 0; k < kNH; ++k) a = fmaf(W3[o * kNH + k], fmaxf(Z2[s * kNH + k], 0.f), a);
      const float res = Uc[s] * a - D3[i];
      if (s < ns) lacc += (double)res * res;
      D3[i] = s < ns ? 2.f * Uc[s] * res : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < NOUT * kNH + NOUT; i += nth) {  // layer 3 gradient
      if (i < NOUT * kNH) {
        const int o = i / kNH, k = i - o * kNH;
        float a = 0.f;
        for (int s = 0; s < kCH; ++s) a = fmaf(D3[s * NOUT + o], fmaxf(Z2[s * kNH + k], 0.f), a);
        G[oW3 + i] += a;
      } else {
        const int o = i - NOUT * kNH;
        float a = 0.f;
        for (int s = 0; s < kCH; ++s) a += D3[s * NOUT + o];
        G[ob3 + o] += a;
      }
    }
    __syncthreads();
    for (int i = tid; i < kCH * kNH; i += nth) {  // delta2 = (W3^T delta3) * [z2 > 0], in place of z2
      const int s = i / kNH, u = i - s * kNH;
      float a = 0.f;
      for (int o = 0; o < NOUT; ++o) a = fmaf(D3[s * NOUT + o], W3[o * kNH + u], a);
      Z2[i] = Z2[i] > 0.f ? a : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < kNH * kNH + kNH; i += nth) {  // layer 2 gradient
      if (i < kNH * kNH) {
        const int u = i / kNH, k = i - u * kNH;
        float a = 0.f;
        for (int s = 0; s < kCH; ++s) a = fmaf(Z2[s * kNH + u], fmaxf(Z1[s * kNH + k], 0.f), a);
        G[oW2 + i] += a;
      } else {
        const int u = i - kNH * kNH;
        float a = 0.f;
        for (int s = 0; s < kCH; ++s) a += Z2[s * kNH + u];
        G[ob2 + u] += a;
      }
    }
    __syncthreads();
    for (int i = tid; i < kCH * kNH; i += nth) {  // delta1 = (W2^T delta2) * [z1 > 0], in place of z1
      const int s = i / kNH, k = i - s * kNH;
      float a = 0.f;
      for (int u = 0; u < kNH; ++u) a = fmaf(Z2[s * kNH + u], W2[u * kNH + k], a);
      Z1[i] = Z1[i] > 0.f ? a : 0.f;
    }
    __syncthreads();
    for (int i = tid; i < kNH * NIN + kNH; i += nth) {  // layer 1 gradient
      if (i < kNH * NIN) {
        const int u = i / NIN, k = i - u * NIN;
        float a = 0.f;
        for (int s = 0; s < kCH; ++s) a = fmaf(Z1[s * kNH + u], Xc[s * NIN + k], a);
        G[oW1 + i] += a;
      } else {
        const int u = i - kNH * NIN;
        float a = 0.f;
        for (int s = 0; s < kCH; ++s) a += Z1[s * kNH + u];
        G[ob1 + u] += a;
      }
    }
  }
  __syncthreads();
  for (int64_t k = threadIdx.x; k < count; k += blockDim.x) part[(int64_t)blockIdx.x * count + k] = G[k];
  red[0][threadIdx.x] = lacc;
  red[1][threadIdx.x] = uacc;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      red[0][threadIdx.x] += red[0][threadIdx.x + st];
      red[1][threadIdx.x] += red[1][threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part2[2 * blockIdx.x] = red[0][0];
    part2[2 * blockIdx.x + 1] = red[1][0];
  }
}

// grad = (sum of the block partials in block order) / sum u^2; loss likewise; out[0] = loss.
__global__ void k_mlp_reduce(const float* __restrict__ part, const double* __restrict__ part2, int nblk,
                             int64_t count, float* __restrict__ grad, double* __restrict__ out) {
  double den = 0.0, num = 0.0;
  for (int b = 0; b < nblk; ++b) {
    num += part2[2 * b];
    den += part2[2 * b + 1];
  }
  const double inv = den > 0.0 ? 1.0 / den : 0.0;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) out[0] = num * inv;
  if (k >= count) return;
  double g = 0.0;
  for (int b = 0; b < nblk; ++b) g += part[(int64_t)b * count + k];
  grad[k] = (float)(g * inv);
}

// Adam with bias-corrected moments (FP32 state).
__global__ void k_adam(int64_t count, const float* __restrict__ grad, float* __restrict__ w, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const float g = grad[k];
  const float mk = b1 * m[k] + (1.f - b1) * g;
  const float vk = b2 * v[k] + (1.f - b2) * g * g;
  m[k] = mk;
  v[k] = vk;
  w[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// Training samples (original element order): features of r_k, u = s / h_e, e = x* - x_k at the nodes.
template <int NLOC>
__global__ void k_harvest(int64_t E, const Geom* __restrict__ geom, const int32_t* __restrict__ elem,
                          const double* __restrict__ Rk, const double* __restrict__ Xk,
                          const double* __restrict__ Xs, int ld, int N, float* __restrict__ X,
                          float* __restrict__ U, float* __restrict__ Eo) {
  constexpr int NIN = NLOC + 12;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= E * N) return;
  const int64_t e = t / N;
  const int j = (int)(t - e * N);
  const Geom G = geom[e];
  double rv[NLOC], ss = 0.0;
#pragma unroll
  for (int a = 0; a < NLOC; ++a) {
    const int64_t i = (int64_t)elem[e * NLOC + a] * ld + j;
    rv[a] = Rk[i];
    ss += rv[a] * rv[a];
    Eo[t * NLOC + a] = (float)(Xs[i] - Xk[i]);
  }
  const double s = sqrt(ss);
  const double h = cbrt(fabs(G.det));
#pragma unroll
  for (int a = 0; a < NLOC; ++a) X[t * NIN + a] = s > 0.0 ? (float)(rv[a] / s) : 0.f;
  double v[4][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    v[0][c] = G.x0[c];
#pragma unroll
    for (int k = 1; k < 4; ++k) v[k][c] = G.x0[c] + G.J[c * 3 + (k - 1)];
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double cen = 0.25 * (v[0][c] + v[1][c] + v[2][c] + v[3][c]);
#pragma unroll
    for (int k = 0; k < 4; ++k) X[t * NIN + NLOC + 3 * k + c] = (float)((v[k][c] - cen) / h);
  }
  U[t] = (float)(s / h);
}

static int mlp_pack(const mk_mlp* mlp, cudaStream_t s) {
  MK_COUNT(), k_mlp_pack<<<(kWbHalves + 255) / 256, 256, 0, s>>>(mlp->d_w, mlp->nin, mlp->nout,
                                                                   (__nv_bfloat16*)mlp->d_wb, mlp->d_bias);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

}  // namespace mk

using namespace mk;

extern "C" {

int64_t mk_mlp_param_count(int nloc) {
  if (nloc != 4 && nloc != 10) return -1;
  return mlp_count(nloc + 12, nloc);
}

int mk_mlp_create(mk_ctx* ctx, int nloc, const float* params, mk_mlp** out) {
  MK_ARG(ctx && params && out, "mk_mlp_create: null argument");
  MK_ARG(nloc == 4 || nloc == 10, "mk_mlp_create: nloc must be 4 or 10");
  MK_CUDA(cudaSetDevice(ctx->device));
  mk_mlp* m = new mk_mlp();
  m->ctx = ctx;
  m->device = ctx->device;
  m->nloc = nloc;
  m->nin = nloc + 12;
  m->nout = nloc;
  m->count = mlp_count(m->nin, m->nout);
  const size_t b = (size_t)m->count * sizeof(float);
  if (cudaMalloc(&m->d_w, b) != cudaSuccess || cudaMalloc(&m->d_m, b) != cudaSuccess ||
      cudaMalloc(&m->d_v, b) != cudaSuccess || cudaMalloc(&m->d_wb, (size_t)kWbHalves * 2) != cudaSuccess ||
      cudaMalloc(&m->d_bias, (size_t)kBias * 4) != cudaSuccess) {
    cudaGetLastError();
    mk_mlp_destroy(m);
    return fail(MK_ERR_OOM, "mk_mlp_create: allocation failed");
  }
  const int r = mk_mlp_load(m, params);
  if (r != MK_OK) {
    mk_mlp_destroy(m);
    return r;
  }
  *out = m;
  return MK_OK;
}

int mk_mlp_destroy(mk_mlp* m) {
  if (!m) return MK_OK;
  cudaSetDevice(m->device);
  cudaFree(m->d_w);
  cudaFree(m->d_m);
  cudaFree(m->d_v);
  cudaFree(m->d_wb);
  cudaFree(m->d_bias);
  delete m;
  return MK_OK;
}

int mk_mlp_save(const mk_mlp* m, float* params) {
  MK_ARG(m && params, "mk_mlp_save: null argument");
  MK_CUDA(cudaSetDevice(m->device));
  MK_CUDA(cudaDeviceSynchronize());
  MK_CUDA(cudaMemcpy(params, m->d_w, (size_t)m->count * sizeof(float), cudaMemcpyDeviceToHost));
  return MK_OK;
}

int mk_mlp_load(mk_mlp* m, const float* params) {
  MK_ARG(m && params, "mk_mlp_load: null argument");
  MK_CUDA(cudaSetDevice(m->device));
  MK_CUDA(cudaDeviceSynchronize());
  const size_t b = (size_t)m->count * sizeof(float);
  MK_CUDA(cudaMemcpy(m->d_w, params, b, cudaMemcpyHostToDevice));
  MK_CUDA(cudaMemset(m->d_m, 0, b));
  MK_CUDA(cudaMemset(m->d_v, 0, b));
  m->t = 0;
  MK_TRY(mlp_pack(m, 0));
  MK_CUDA(cudaDeviceSynchronize());
  return MK_OK;
}

int mk_mlp_forward(mk_ctx* ctx, const mk_mlp* m, const float* X, int64_t S, float* Y, int precision, void* stream) {
  MK_ARG(ctx && m && X && Y && S >= 0, "mk_mlp_forward: bad argument");
  MK_ARG(precision == MK_MLP_FP32 || precision == MK_MLP_BF16, "mk_mlp_forward: bad precision");
  MK_CUDA(cudaSetDevice(ctx->device));
  if (S == 0) return MK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == MK_MLP_FP32) {
    const size_t smem = (size_t)m->count * sizeof(float);
    const int blocks = (int)((S + 127) / 128);
    if (m->nloc == 4) {
      cudaFuncSetAttribute(k_mlp_forward32<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      MK_COUNT(), k_mlp_forward32<4><<<blocks, 128, smem, s>>>(S, m->d_w, m->count, X, Y);
    } else {
      cudaFuncSetAttribute(k_mlp_forward32<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      MK_COUNT(), k_mlp_forward32<10><<<blocks, 128, smem, s>>>(S, m->d_w, m->count, X, Y);
    }
  } else {
    const int blocks = (int)((S + 127) / 128);  // 8 warps x 16 rows
    if (m->nloc == 4)
      MK_COUNT(), k_mlp_forward16<4><<<blocks, 256, 0, s>>>(S, (const __nv_bfloat16*)m->d_wb, m->d_bias, X, Y);
    else
      MK_COUNT(), k_mlp_forward16<10><<<blocks, 256, 0, s>>>(S, (const __nv_bfloat16*)m->d_wb, m->d_bias, X, Y);
  }
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

int mk_mlp_train_step(mk_ctx* ctx, mk_mlp* m, const float* X, const float* U, const float* E, const int32_t* idx,
                      int64_t S, const mk_adam* opt, double* loss, float* grad, void* stream) {
  MK_ARG(ctx && m && X && U && E && loss && S >= 1, "mk_mlp_train_step: bad argument");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nchunks = (S + kCH - 1) / kCH;
  const int nblk = (int)std::min<int64_t>(nchunks, ctx->n_sms);
  int err = MK_OK;
  char* part = (char*)scratch(ctx, S_MLPPART, (size_t)nblk * m->count * sizeof(float) + (size_t)nblk * 2 * sizeof(double) + 64, &err);
  float* g = (float*)scratch(ctx, S_MLPGRAD, (size_t)m->count * sizeof(float) + 64, &err);
  if (!part || !g) return err;
  float* pf = (float*)part;
  double* p2 = (double*)(part + ((size_t)nblk * m->count * sizeof(float) + 15) / 16 * 16);
  double* dloss = (double*)((char*)g + ((size_t)m->count * sizeof(float) + 15) / 16 * 16);
  const size_t smem = ((size_t)2 * m->count + (size_t)kCH * m->nin + 2 * kCH * kNH + (size_t)kCH * m->nout + kCH) *
                      sizeof(float);
  MK_ARG(smem <= 200 * 1024, "mk_mlp_train_step: network too large");
  if (m->nloc == 4) {
    cudaFuncSetAttribute(k_mlp_grad<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    MK_COUNT(), k_mlp_grad<4><<<nblk, 256, smem, s>>>(m->d_w, m->count, X, U, E, idx, S, pf, p2);
  } else {
    cudaFuncSetAttribute(k_mlp_grad<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    MK_COUNT(), k_mlp_grad<10><<<nblk, 256, smem, s>>>(m->d_w, m->count, X, U, E, idx, S, pf, p2);
  }
  MK_COUNT(), k_mlp_reduce<<<(int)((m->count + 255) / 256), 256, 0, s>>>(pf, p2, nblk, m->count, g, dloss);
  if (grad) MK_CUDA(cudaMemcpyAsync(grad, g, (size_t)m->count * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (opt && opt->lr > 0.0) {
    m->t += 1;
    const float c1 = (float)(1.0 - std::pow(opt->beta1, (double)m->t));
    const float c2 = (float)(1.0 - std::pow(opt->beta2, (double)m->t));
    MK_COUNT(), k_adam<<<(int)((m->count + 255) / 256), 256, 0, s>>>(m->count, g, m->d_w, m->d_m, m->d_v,
                                                                      (float)opt->lr, (float)opt->beta1,
                                                                      (float)opt->beta2, (float)opt->eps, c1, c2);
    MK_TRY(mlp_pack(m, s));
  }
  MK_CUDA(cudaMemcpyAsync(loss, dloss, sizeof(double), cudaMemcpyDeviceToHost, s));
  MK_CUDA(cudaStreamSynchronize(s));
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

int mk_mlp_harvest(mk_ctx* ctx, const mk_mesh* mesh, const double* Rk, const double* Xk, const double* Xstar, int ld,
                   int N, float* X, float* U, float* E, void* stream) {
  MK_ARG(ctx && mesh && Rk && Xk && Xstar && X && U && E, "mk_mlp_harvest: null argument");
  MK_ARG(N >= 1 && N <= ld, "mk_mlp_harvest: bad N/ld");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const Level& L = mesh->fine;
  const int64_t work = L.n_elems * N;
  const int blocks = (int)((work + 255) / 256);
  if (L.nloc == 4)
    MK_COUNT(), k_harvest<4><<<blocks, 256, 0, s>>>(L.n_elems, L.d_geom, L.d_elem, Rk, Xk, Xstar, ld, N, X, U, E);
  else
    MK_COUNT(), k_harvest<10><<<blocks, 256, 0, s>>>(L.n_elems, L.d_geom, L.d_elem, Rk, Xk, Xstar, ld, N, X, U, E);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

int mk_learned_precond(mk_ctx* ctx, const mk_mesh* mesh, const mk_mlp* mlp, const mk_molecule* mol, double sigma,
                       const float* r, float* z, int ld, int N, int precision, void* stream) {
  MK_ARG(ctx && mesh && mlp && mol && r && z, "mk_learned_precond: null argument");
  MK_ARG(N >= 1 && N <= ld && ld <= 256, "mk_learned_precond: bad N/ld");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const Level& L = mesh->fine;
  const int np = L.nloc * (L.nloc + 1) / 2;
  int err = MK_OK;
  double* A64 = (double*)scratch(ctx, S_OPA, (size_t)L.n_elems * np * sizeof(double), &err);
  char* dd = (char*)scratch(ctx, S_LDINV, (size_t)L.n_nodes * (sizeof(double) + sizeof(float)) + 64, &err);
  if (!A64 || !dd) return err;
  double* diag = (double*)dd;
  float* dinv = (float*)(dd + ((size_t)L.n_nodes * sizeof(double) + 15) / 16 * 16);
  const double* H0 = static_matrices(ctx, mesh, mol, s, &err);
  if (!H0) return err;
  MK_TRY(element_matrices(ctx, L, nullptr, 0.0, 0.0, sigma, nullptr, A64, s, H0));
  MK_TRY(assemble_diagonal(ctx, L, A64, diag, s));
  MK_TRY(diag_inverse32(L.n_nodes, diag, dinv, s));
  return learned_apply(ctx, mesh, mlp, dinv, r, z, ld, N, precision, s);
}

}  // extern "C"
