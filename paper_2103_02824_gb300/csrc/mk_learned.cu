// Learned element-patch preconditioner: the network (FP32 master weights, Adam, BF16 inference copy), its
// forward pass on CUDA cores (FP32) and on the 5th-generation tensor cores (tcgen05: BF16 operands in shared
// memory, FP32 accumulation in tensor memory), the fused patch kernels that turn a residual into
// z = D^-1 r + (assembled network corrections) / multiplicity, the deterministic training gradient, Adam, and
// the harvest of training samples from solver iterates.
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
constexpr int kLW = 8;              // orbital columns per pass of the patch kernel

// ---- the BF16 network on the 5th-generation tensor cores (tcgen05)
// Operands live in shared memory in the K-major, unswizzled canonical layout of tcgen05.mma: an R x K BF16 matrix
// is a grid of core matrices of 8 rows x 8 columns, each 128 contiguous bytes (row r of a core matrix at byte
// 16 r); core matrices adjacent in K are 128 bytes apart (the descriptor's leading-dimension byte offset) and
// groups of 8 rows K * 16 bytes apart (its stride-dimension byte offset).
constexpr int kK1 = 32;       // layer-1 input width: the n_in <= 22 features, the two bias inputs, zeros
constexpr int kKOne = 28;     // input columns 28 and 29 hold 1.0 against the layer-1 bias (high, low BF16 parts)
constexpr int kTcRows = 128;  // rows per tile: the MMA's M, the TMEM lanes, the threads of a warpgroup
__host__ __device__ constexpr int umma_off(int row, int k, int K) {  // element (row, k) in halves
  return (row >> 3) * (K * 8) + (k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}
// Packed weights (halves, each matrix [out][in] in the layout above): W1 [64 x 32] with the layer-1 bias parts in
// columns kKOne, kKOne + 1; W2 [64 x 64]; W3 [16 x 64] (rows >= n_out zero); the layer-2 and layer-3 biases as
// [64 x 16] and [16 x 16] matrices whose columns 0 and 1 hold the high and low BF16 parts, multiplied by an
// all-ones input tile.  high + low carries the FP32 bias to about 2^-16 relative.
constexpr int kUW1 = 0;
constexpr int kUW2 = kUW1 + kNH * kK1;
constexpr int kUW3 = kUW2 + kNH * kNH;
constexpr int kUB2 = kUW3 + 16 * kNH;
constexpr int kUB3 = kUB2 + kNH * 16;
constexpr int kWuHalves = kUB3 + 16 * 16;
constexpr uint32_t kTmemCols = 64;  // per warpgroup: every layer's accumulator starts at its column 0 (layer 3: 16)

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


// Two floats as a packed BF16 pair (lo in the low half), round to nearest even.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// ---- tcgen05 primitives (inline PTX).  tcgen05.mma reads A and B from shared memory through 64-bit matrix
// descriptors and accumulates in tensor memory (TMEM: 128 lanes x 512 32-bit columns per SM); one thread issues
// it, tcgen05.commit makes an mbarrier track its completion, and each warp reads back its quarter of the lanes
// (warp w of the CTA: lanes 32 (w % 4) .. + 31) with tcgen05.ld.  For M = 128, row i of D is TMEM lane i and
// column n is TMEM column base + n.
// Shared-memory matrix descriptor: start address / 16 (bits 0-13), leading-dimension byte offset 128 / 16 (bits
// 16-29: the next core matrix along K), stride-dimension byte offset sbo / 16 (bits 32-45: the next 8-row
// group), the fixed 0b001 at bits 46-48, base offset 0, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}
// Instruction descriptor of kind::f16: dense, FP32 accumulator (bits 4-5 = 1), BF16 A and B (bits 7-9 and 10-12 =
// 1), neither negated, both K-major (bits 15, 16 = 0), N / 8 at bits 17-22, M / 16 at bits 24-28.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// D = A B^T (acc = 0) or D += A B^T (acc = 1), A [M x K], B [N x K], both K-major, one K = 16 step
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
// the mbarrier receives one arrival when every tcgen05.mma this thread issued before has completed
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// by one whole warp: ncols TMEM columns (a power of two >= 32), the address written to *slot
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
// 64 (16) consecutive 32-bit columns of this thread's TMEM lane, waited for inside the same statement so that no
// use of the registers can be scheduled before the load has completed
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&r)[64]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];\n"
               "tcgen05.wait::ld.sync.aligned;\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n"
               "tcgen05.wait::ld.sync.aligned;\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr)
               : "memory");
}

// Barrier of one warpgroup (128 threads): id 0 is the CTA barrier (CTAs of one warpgroup), ids 1.. named ones.
__device__ __forceinline__ void wg_barrier(int id) {
  if (id == 0) __syncthreads();
  else asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(kTcRows) : "memory");
}
// This thread's shared-memory writes become visible to the tensor cores, its TMEM reads are ordered before the
// barrier, and tcgen05 work after the barrier is ordered after it.
__device__ __forceinline__ void sync_for_mma(int barid) {
  fence_proxy_async();
  tc_fence_before();
  wg_barrier(barid);
  tc_fence_after();
}

// State of one warpgroup running the network on tcgen05 (kTcRows threads, one tile row each).  Pointers into the
// activation tile are deliberately not __restrict__: the tile is read by the tensor cores between the threads'
// stores, and a no-alias promise would let the compiler move those stores past the proxy fence and the barrier.
struct TcState {
  uint32_t tmem;         // TMEM address of this warpgroup's kTmemCols columns (lane 0)
  uint32_t xh, w, one;   // shared addresses: activation tile [128 x 64], packed weights, all-ones tile [128 x 16]
  uint64_t* bar;         // this warpgroup's MMA mbarrier
  int barid;             // its barrier id
  unsigned phase;        // parity of the mbarrier's next completion
  bool ok;               // false once a bounded wait of this thread gave up
};

// Allocates ncols TMEM columns for the CTA (warp 0), initialises nbar MMA mbarriers and writes the all-ones tile
// (threads 0-127, one row each).  The caller completes its staging and calls sync_for_mma(0) before reading *slot.
__device__ __forceinline__ void tc_setup(uint32_t* slot, uint32_t ncols, uint64_t* bars, int nbar,
                                         __nv_bfloat16* one) {
  if (threadIdx.x < 32) tmem_alloc(slot, ncols);
  if (threadIdx.x == 0) {
    for (int b = 0; b < nbar; ++b) mbar_init(bars + b, 1);
    mbar_fence_init();
  }
  const int r = threadIdx.x;
  if (r < kTcRows) {
    *reinterpret_cast<uint4*>(one + umma_off(r, 0, 16)) = make_uint4(pack_bf16(1.f, 1.f), 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(one + umma_off(r, 8, 16)) = make_uint4(0u, 0u, 0u, 0u);
  }
}
// Every tcgen05 operation of the CTA has completed (all waited for): warp 0 frees the TMEM.
__device__ __forceinline__ void tc_teardown(uint32_t tmem, uint32_t ncols) {
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    tmem_dealloc(tmem, ncols);
  }
}
__device__ __forceinline__ void mma_wait(TcState& S) {
  if (S.ok && !mbar_wait(S.bar, S.phase)) S.ok = false;
  S.phase ^= 1u;
  tc_fence_after();
}
// relu(acc) of this thread's row as the next layer's input row (K = 64)
__device__ __forceinline__ void store_hidden_row(__nv_bfloat16* xh, int row, const uint32_t (&a)[64]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    uint4 v;
    v.x = pack_relu_bf16(__uint_as_float(a[8 * c + 0]), __uint_as_float(a[8 * c + 1]));
    v.y = pack_relu_bf16(__uint_as_float(a[8 * c + 2]), __uint_as_float(a[8 * c + 3]));
    v.z = pack_relu_bf16(__uint_as_float(a[8 * c + 4]), __uint_as_float(a[8 * c + 5]));
    v.w = pack_relu_bf16(__uint_as_float(a[8 * c + 6]), __uint_as_float(a[8 * c + 7]));
    *reinterpret_cast<uint4*>(xh + umma_off(row, 8 * c, kNH)) = v;
  }
}
// This thread's layer-1 input row (kK1 values) into the activation tile.
__device__ __forceinline__ void store_input_row(__nv_bfloat16* xh, int row, const float (&f)[kK1]) {
#pragma unroll
  for (int c = 0; c < kK1 / 8; ++c)
    *reinterpret_cast<uint4*>(xh + umma_off(row, 8 * c, kK1)) =
        make_uint4(pack_bf16(f[8 * c + 0], f[8 * c + 1]), pack_bf16(f[8 * c + 2], f[8 * c + 3]),
                   pack_bf16(f[8 * c + 4], f[8 * c + 5]), pack_bf16(f[8 * c + 6], f[8 * c + 7]));
}

// The network on one tile of kTcRows rows whose layer-1 inputs the warpgroup's threads have just stored (row =
// thread index in the warpgroup); y receives this thread's row of the output layer (16 columns, those >= n_out
// zero).  Each layer: the warpgroup's first thread issues the MMAs (the bias first, against the all-ones tile, for
// layers 2 and 3; through the constant input columns for layer 1) and commits them to the mbarrier; every thread
// waits, reads its accumulator row from TMEM and writes relu of it, in BF16, over the activation tile (the MMAs
// reading that tile have completed by then).
__device__ __forceinline__ void umma_mlp_tile(TcState& S, __nv_bfloat16* xh, float (&y)[16]) {
  constexpr uint32_t i64 = umma_idesc_bf16(kTcRows, kNH), i16 = umma_idesc_bf16(kTcRows, 16);
  const int tid = threadIdx.x & (kTcRows - 1);
  const uint32_t lane = (uint32_t)(tid & ~31) << 16;  // this warp's TMEM lane quarter (warp index mod 4)
  uint32_t a[64];
  sync_for_mma(S.barid);
  if (tid == 0 && S.ok) {
#pragma unroll
    for (int ks = 0; ks < kK1 / 16; ++ks)
      umma_bf16(S.tmem, umma_desc(S.xh + 256 * ks, kK1 * 16), umma_desc(S.w + 2 * kUW1 + 256 * ks, kK1 * 16), i64,
                ks > 0);
    umma_commit(S.bar);
  }
  mma_wait(S);
  tmem_ld64(S.tmem + lane, a);
  store_hidden_row(xh, tid, a);
  sync_for_mma(S.barid);
  if (tid == 0 && S.ok) {
    umma_bf16(S.tmem, umma_desc(S.one, 256), umma_desc(S.w + 2 * kUB2, 256), i64, 0);
#pragma unroll
    for (int ks = 0; ks < kNH / 16; ++ks)
      umma_bf16(S.tmem, umma_desc(S.xh + 256 * ks, kNH * 16), umma_desc(S.w + 2 * kUW2 + 256 * ks, kNH * 16), i64, 1);
    umma_commit(S.bar);
  }
  mma_wait(S);
  tmem_ld64(S.tmem + lane, a);
  store_hidden_row(xh, tid, a);
  sync_for_mma(S.barid);
  if (tid == 0 && S.ok) {
    umma_bf16(S.tmem, umma_desc(S.one, 256), umma_desc(S.w + 2 * kUB3, 256), i16, 0);
#pragma unroll
    for (int ks = 0; ks < kNH / 16; ++ks)
      umma_bf16(S.tmem, umma_desc(S.xh + 256 * ks, kNH * 16), umma_desc(S.w + 2 * kUW3 + 256 * ks, kNH * 16), i16, 1);
    umma_commit(S.bar);
  }
  mma_wait(S);
  uint32_t o[16];
  tmem_ld16(S.tmem + lane, o);
#pragma unroll
  for (int k = 0; k < 16; ++k) y[k] = __uint_as_float(o[k]);
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

// Y = network(X) on the tensor cores (tcgen05, BF16 operands, FP32 accumulation), 128 rows per tile; the CTAs
// take tiles blockIdx.x, + gridDim.x, ...  A bounded wait that gave up sets MK_FAULT_TC_WAIT in *fault.
template <int NLOC>
__global__ void __launch_bounds__(kTcRows) k_mlp_forward_tc(int64_t S, const __nv_bfloat16* __restrict__ wu,
                                                           const float* __restrict__ X, float* __restrict__ Y,
                                                           int* __restrict__ fault) {
  constexpr int NIN = NLOC + 12;
  __shared__ __align__(128) __nv_bfloat16 wsm[kWuHalves];
  __shared__ __align__(128) __nv_bfloat16 xh[kTcRows * kNH];
  __shared__ __align__(128) __nv_bfloat16 one[kTcRows * 16];
  __shared__ uint64_t bar;
  __shared__ uint32_t slot;
  for (int k = threadIdx.x; k < kWuHalves / 8; k += blockDim.x) cp_async16(wsm + 8 * k, wu + 8 * k);
  tc_setup(&slot, kTmemCols, &bar, 1, one);
  cp_async_wait_all();
  sync_for_mma(0);
  TcState st{slot, smem_u32(xh), smem_u32(wsm), smem_u32(one), &bar, 0, 0u, true};
  const int64_t ntiles = (S + kTcRows - 1) / kTcRows;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t row = t * kTcRows + threadIdx.x;
    const bool valid = row < S;
    float f[kK1];
#pragma unroll
    for (int k = 0; k < kK1; ++k)
      f[k] = k < NIN ? (valid ? X[row * NIN + k] : 0.f) : (k == kKOne || k == kKOne + 1) ? 1.f : 0.f;
    store_input_row(xh, threadIdx.x, f);
    float y[16];
    umma_mlp_tile(st, xh, y);
    if (valid)
#pragma unroll
      for (int o = 0; o < NLOC; ++o) Y[row * NLOC + o] = y[o];
  }
  tc_teardown(slot, kTmemCols);
  if (!st.ok) atomicOr(fault, MK_FAULT_TC_WAIT);
}

// The BF16 copy of the parameters in the tcgen05 layout (kUW1 ... kUB3), one element per thread.
__global__ void k_mlp_pack_umma(const float* __restrict__ w, int nin, int nout, __nv_bfloat16* __restrict__ wu) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kWuHalves) return;
  const float* W1 = w;
  const float* b1 = W1 + kNH * nin;
  const float* W2 = b1 + kNH;
  const float* b2 = W2 + kNH * kNH;
  const float* W3 = b2 + kNH;
  const float* b3 = W3 + nout * kNH;
  // value v at (row, k) of a matrix with K columns starting at base; bias parts: high = bf16(b), low = bf16(b - high)
  auto bias_part = [](float b, int k) -> float {
    const float hi = __bfloat162float(__float2bfloat16_rn(b));
    return k == 0 ? hi : k == 1 ? b - hi : 0.f;
  };
  int base, row, k, K;
  float v;
  if (i < kUW2) {
    base = kUW1, K = kK1, row = (i - base) / K, k = (i - base) % K;
    v = k < nin ? W1[row * nin + k] : (k == kKOne || k == kKOne + 1) ? bias_part(b1[row], k - kKOne) : 0.f;
  } else if (i < kUW3) {
    base = kUW2, K = kNH, row = (i - base) / K, k = (i - base) % K;
    v = W2[row * kNH + k];
  } else if (i < kUB2) {
    base = kUW3, K = kNH, row = (i - base) / K, k = (i - base) % K;
    v = row < nout ? W3[row * kNH + k] : 0.f;
  } else if (i < kUB3) {
    base = kUB2, K = 16, row = (i - base) / K, k = (i - base) % K;
    v = bias_part(b2[row], k);
  } else {
    base = kUB3, K = 16, row = (i - base) / K, k = (i - base) % K;
    v = row < nout ? bias_part(b3[row], k) : 0.f;
  }
  wu[base + umma_off(row, k, K)] = __float2bfloat16_rn(v);
}

// ------------------------------------------------------------------------------------------------ preconditioner
struct LearnSmem {
  size_t ye, rs, conn, inc, ioff, tgt, geo, w, xh, one, total;
};
constexpr int kTcGroups = 2;  // warpgroups (tiles in flight) per CTA of the tensor-core patch kernel

// tc: the tensor-core kernel (network outputs in BF16, packed BF16 weights, one activation tile per warpgroup, the
// all-ones tile); otherwise FP32 outputs and the FP32 parameters (count floats)
__host__ __device__ inline LearnSmem learn_smem(int nloc, int pe, int max_nodes, bool tc, int64_t count) {
  LearnSmem L;
  L.ye = 0;
  L.rs = L.ye + align16((size_t)nloc * pe * kLW * (tc ? 2 : 4));      // residual rows of the local nodes
  L.conn = L.rs + align16((size_t)max_nodes * kLW * 4);              // local node of each element slot (uint16)
  L.inc = L.conn + align16((size_t)pe * nloc * 2 + 16);
  L.ioff = L.inc + align16((size_t)pe * nloc * 2 + 16);
  L.tgt = L.ioff + align16((size_t)(max_nodes + 1) * 4 + 16);
  L.geo = L.tgt + align16((size_t)max_nodes * 4 + 16);
  L.w = L.geo + align16((size_t)pe * 16 * 4 + 16);
  L.xh = L.w + align16(tc ? (size_t)kWuHalves * 2 + 16 : (size_t)count * 4 + 16);
  L.one = L.xh + (tc ? (size_t)kTcGroups * kTcRows * kNH * 2 : 0);
  L.total = L.one + (tc ? (size_t)kTcRows * 16 * 2 : 0);
  return L;
}

// The patch's data in shared memory (cp.async, not yet waited for).
struct LearnPatch {
  int e0, ne, n0, nl, ibase, Nw;
  const uint16_t *cs, *is;
  const int32_t *os, *ts;
  const float *gs, *rs;
  const unsigned char* wsm;
};
template <int NLOC>
__device__ __forceinline__ LearnPatch learn_stage(unsigned char* smraw, const LearnSmem& lay, int p,
                                                  const int32_t* __restrict__ elem_off,
                                                  const int32_t* __restrict__ node_off,
                                                  const uint16_t* __restrict__ lconn,
                                                  const int32_t* __restrict__ node_gid,
                                                  const int32_t* __restrict__ target,
                                                  const int32_t* __restrict__ inc_off,
                                                  const uint16_t* __restrict__ inc, const float* __restrict__ geomf,
                                                  const void* __restrict__ wsrc, int wbytes,
                                                  const float* __restrict__ r, int N, int col0, int ld) {
  LearnPatch P;
  P.e0 = elem_off[p];
  P.ne = elem_off[p + 1] - P.e0;
  P.n0 = node_off[p];
  P.nl = node_off[p + 1] - P.n0;
  P.ibase = P.e0 * NLOC;
  P.Nw = min(kLW, N - col0);
  P.cs = stage_async(smraw + lay.conn, lconn + P.ibase, P.ne * NLOC * 2);
  // the residual rows of the patch's local nodes, columns [col0, col0 + 8) (16-byte copies; ld % 4 == 0)
  float* rs = reinterpret_cast<float*>(smraw + lay.rs);
  const int nvec = min(kLW, ld - col0) / 4;
  for (int l = threadIdx.x; l < P.nl; l += blockDim.x) {
    const float* src = r + (int64_t)node_gid[P.n0 + l] * ld + col0;
    for (int v = 0; v < nvec; ++v) cp_async16(rs + l * kLW + 4 * v, src + 4 * v);
  }
  P.rs = rs;
  P.is = stage_async(smraw + lay.inc, inc + P.ibase, P.ne * NLOC * 2);
  P.os = stage_async(smraw + lay.ioff, inc_off + P.n0, (P.nl + 1) * 4);
  P.ts = stage_async(smraw + lay.tgt, target + P.n0, P.nl * 4);
  P.gs = stage_async(smraw + lay.geo, geomf + (int64_t)P.e0 * 16, P.ne * 16 * 4);
  P.wsm = stage_async(smraw + lay.w, reinterpret_cast<const unsigned char*>(wsrc), wbytes);
  return P;
}

// Phase 2 of the patch kernels: per local node the incidences in fixed order (FP32 sums), then z = sum /
// multiplicity + r / diag (owned nodes) or the partial sum to the node's halo slot (shared nodes, finished by
// k_learned_halo).
__device__ __forceinline__ float ye_value(float v) { return v; }
__device__ __forceinline__ float ye_value(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename YT>
__device__ __forceinline__ void learn_assemble(const LearnPatch& P, const YT* __restrict__ Ye,
                                               const float* __restrict__ dinv, const float* __restrict__ inv_mult,
                                               const float* __restrict__ r, float* __restrict__ z,
                                               float* __restrict__ halo, int col0, int ld) {
  const int Nw = P.Nw;
  for (int it = threadIdx.x; it < P.nl * Nw; it += blockDim.x) {
    const int l = it / Nw, jj = it - l * Nw;
    const int b = P.os[l] - P.ibase, e = P.os[l + 1] - P.ibase;
    float acc = 0.f;
    for (int k = b; k < e; ++k) acc += ye_value(Ye[(size_t)P.is[k] * kLW + jj]);
    const int tg = P.ts[l];
    if (tg >= 0) {
      const int nd = tg & (kOwnedBoundary - 1);
      const int64_t t = (int64_t)nd * ld + col0 + jj;
      z[t] = (tg & kOwnedBoundary) ? 0.f : fmaf(acc, inv_mult[nd], dinv[nd] * r[t]);
    } else {
      halo[(int64_t)(-tg - 1) * ld + col0 + jj] = acc;
    }
  }
}

// One patch per CTA (the patches of the operator apply), the network in FP32 on CUDA cores, one thread per
// (element, column) row: phase 1 writes network(x) * s / h_e into shared memory [slot][element][column], phase 2
// assembles.  Columns [col0, col0 + Nw), Nw = min(kLW, N - col0).
template <int NLOC>
__global__ void __launch_bounds__(256, 2) k_learned_patch(
    const int32_t* __restrict__ elem_off, const int32_t* __restrict__ node_off, const uint16_t* __restrict__ lconn,
    const int32_t* __restrict__ node_gid, const int32_t* __restrict__ target, const int32_t* __restrict__ inc_off,
    const uint16_t* __restrict__ inc, const float* __restrict__ geomf, const float* __restrict__ w, int64_t count,
    const float* __restrict__ dinv, const float* __restrict__ inv_mult, const float* __restrict__ r,
    float* __restrict__ z, float* __restrict__ halo, int N, int col0, int ld, int pe, int max_nodes) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const LearnSmem lay = learn_smem(NLOC, pe, max_nodes, false, count);
  float* Ye = reinterpret_cast<float*>(smraw + lay.ye);
  const LearnPatch P = learn_stage<NLOC>(smraw, lay, blockIdx.x, elem_off, node_off, lconn, node_gid, target, inc_off,
                                         inc, geomf, w, (int)(count * 4), r, N, col0, ld);
  cp_async_wait_all();
  __syncthreads();
  const int Nw = P.Nw, nrows = P.ne * Nw;
  const float* wf = reinterpret_cast<const float*>(P.wsm);
  for (int row = threadIdx.x; row < nrows; row += blockDim.x) {
    const int el = row / Nw, jj = row - el * Nw;
    float x[NLOC + 12], y[NLOC], ss = 0.f;
#pragma unroll
    for (int a = 0; a < NLOC; ++a) {
      x[a] = P.rs[P.cs[el * NLOC + a] * kLW + jj];
      ss = fmaf(x[a], x[a], ss);
    }
    const float s = sqrtf(ss);
    const float inv = s > 0.f ? 1.f / s : 0.f;
#pragma unroll
    for (int a = 0; a < NLOC; ++a) x[a] *= inv;
#pragma unroll
    for (int k = 0; k < 12; ++k) x[NLOC + k] = P.gs[el * 16 + 1 + k];
    mlp_row32<NLOC>(wf, x, y);
    const float sc = s / P.gs[el * 16];
#pragma unroll
    for (int o = 0; o < NLOC; ++o) Ye[((size_t)o * pe + el) * kLW + jj] = y[o] * sc;
  }
  __syncthreads();
  learn_assemble(P, Ye, dinv, inv_mult, r, z, halo, col0, ld);
}

// The same with the network on the tensor cores (tcgen05, BF16 operands, FP32 accumulation in TMEM): kTcGroups
// warpgroups, warpgroup g taking the tiles g, g + kTcGroups, ... of 128 (element, column) rows with its own
// activation tile, mbarrier, named barrier and kTmemCols TMEM columns, so that kTcGroups tiles are in flight per
// CTA.  One row per thread: it gathers and normalises its residual features, adds the element's geometry and the
// bias inputs, and scales its outputs, stored in BF16 (the precision of the network).  A bounded wait that gave up
// sets MK_FAULT_TC_WAIT in *fault (outputs invalid).
template <int NLOC>
__global__ void __launch_bounds__(kTcGroups * kTcRows, 2) k_learned_patch_tc(
    const int32_t* __restrict__ elem_off, const int32_t* __restrict__ node_off, const uint16_t* __restrict__ lconn,
    const int32_t* __restrict__ node_gid, const int32_t* __restrict__ target, const int32_t* __restrict__ inc_off,
    const uint16_t* __restrict__ inc, const float* __restrict__ geomf, const __nv_bfloat16* __restrict__ wu,
    const float* __restrict__ dinv, const float* __restrict__ inv_mult, const float* __restrict__ r,
    float* __restrict__ z, float* __restrict__ halo, int N, int col0, int ld, int pe, int max_nodes,
    int* __restrict__ fault) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ uint64_t bars[kTcGroups];
  __shared__ uint32_t slot;
  const LearnSmem lay = learn_smem(NLOC, pe, max_nodes, true, 0);
  __nv_bfloat16* Ye = reinterpret_cast<__nv_bfloat16*>(smraw + lay.ye);
  const int g = threadIdx.x / kTcRows, tid = threadIdx.x & (kTcRows - 1);
  __nv_bfloat16* xh = reinterpret_cast<__nv_bfloat16*>(smraw + lay.xh) + g * kTcRows * kNH;
  __nv_bfloat16* one = reinterpret_cast<__nv_bfloat16*>(smraw + lay.one);
  const LearnPatch P = learn_stage<NLOC>(smraw, lay, blockIdx.x, elem_off, node_off, lconn, node_gid, target, inc_off,
                                         inc, geomf, wu, kWuHalves * 2, r, N, col0, ld);
  tc_setup(&slot, kTcGroups * kTmemCols, bars, kTcGroups, one);
  cp_async_wait_all();
  sync_for_mma(0);
  TcState st{slot + g * kTmemCols, smem_u32(xh), smem_u32(P.wsm), smem_u32(one), bars + g, 1 + g, 0u, true};
  const int Nw = P.Nw, nrows = P.ne * Nw;
  // row / Nw as (row * ceil(2^16 / Nw)) >> 16: the ceiling adds less than row / 2^16, which stays below 1 / Nw
  // for row < 2^16 / Nw (8,192 for Nw = 8; a patch has at most 512 * 8 rows), so the quotient is exact
  const unsigned mnw = (65536u + (unsigned)Nw - 1u) / (unsigned)Nw;
  for (int tile = g; tile * kTcRows < nrows; tile += kTcGroups) {
    const int row = tile * kTcRows + tid;
    const bool valid = row < nrows;
    const int el = valid ? (int)(((unsigned)row * mnw) >> 16) : 0, jj = valid ? row - el * Nw : 0;
    float f[kK1], ss = 0.f;
#pragma unroll
    for (int a = 0; a < NLOC; ++a) {
      f[a] = valid ? P.rs[P.cs[el * NLOC + a] * kLW + jj] : 0.f;
      ss = fmaf(f[a], f[a], ss);
    }
    const float s = sqrtf(ss);
    const float inv = s > 0.f ? 1.f / s : 0.f;
#pragma unroll
    for (int a = 0; a < NLOC; ++a) f[a] *= inv;
#pragma unroll
    for (int k = 0; k < 12; ++k) f[NLOC + k] = P.gs[el * 16 + 1 + k];
#pragma unroll
    for (int k = NLOC + 12; k < kK1; ++k) f[k] = (k == kKOne || k == kKOne + 1) ? 1.f : 0.f;
    const float sc = valid ? s / P.gs[el * 16] : 0.f;
    store_input_row(xh, tid, f);
    float y[16];
    umma_mlp_tile(st, xh, y);
    if (valid)
#pragma unroll
      for (int o = 0; o < NLOC; ++o) Ye[((size_t)o * pe + el) * kLW + jj] = __float2bfloat16_rn(y[o] * sc);
  }
  tc_teardown(slot, kTcGroups * kTmemCols);  // its CTA barrier also completes Ye
  if (!st.ok) atomicOr(fault, MK_FAULT_TC_WAIT);
  learn_assemble(P, Ye, dinv, inv_mult, r, z, halo, col0, ld);
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
  const LearnSmem lay = learn_smem(L.nloc, P.max_elems, P.max_nodes, tc, mlp->count);
  MK_ARG(lay.total <= 227 * 1024 - 256, "learned preconditioner: patch too large for shared memory");
  MK_ARG(((uintptr_t)mlp->d_wb & 15) == 0, "learned preconditioner: packed weights not 16-byte aligned");
  for (int col0 = 0; col0 < N; col0 += kLW) {
    const int Nw = std::min(kLW, N - col0);
    const __nv_bfloat16* wu = (const __nv_bfloat16*)mlp->d_wb;
    auto launch_tc = [&](auto kern) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total);
      MK_COUNT(), kern<<<P.n_patches, kTcGroups * kTcRows, lay.total, s>>>(
          P.d_patch_elem_off, P.d_patch_node_off, P.d_lconn, P.d_node_gid, P.d_node_target, P.d_inc_off, P.d_inc,
          P.d_geomf, wu, dinv, P.d_inv_mult, r, z, halo, N, col0, ld, P.max_elems, P.max_nodes, ctx->d_fault);
    };
    auto launch_fp32 = [&](auto kern) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lay.total);
      MK_COUNT(), kern<<<P.n_patches, 256, lay.total, s>>>(
          P.d_patch_elem_off, P.d_patch_node_off, P.d_lconn, P.d_node_gid, P.d_node_target, P.d_inc_off, P.d_inc,
          P.d_geomf, mlp->d_w, mlp->count, dinv, P.d_inv_mult, r, z, halo, N, col0, ld, P.max_elems, P.max_nodes);
    };
    prof_mark(ctx, PROF_LEARNED, true, s);
    if (L.nloc == 4) {
      if (tc) launch_tc(k_learned_patch_tc<4>);
      else launch_fp32(k_learned_patch<4>);
    } else {
      if (tc) launch_tc(k_learned_patch_tc<10>);
      else launch_fp32(k_learned_patch<10>);
    }
    prof_mark(ctx, PROF_LEARNED, false, s);
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
  MK_COUNT(), k_mlp_pack_umma<<<(kWuHalves + 255) / 256, 256, 0, s>>>(mlp->d_w, mlp->nin, mlp->nout,
                                                                        (__nv_bfloat16*)mlp->d_wb);
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
      cudaMalloc(&m->d_v, b) != cudaSuccess || cudaMalloc(&m->d_wb, (size_t)kWuHalves * 2) != cudaSuccess) {
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
    // at most 2 CTAs per SM in the grid-stride loop; each holds kTmemCols of the SM's 512 TMEM columns
    const int blocks = (int)std::min<int64_t>((S + kTcRows - 1) / kTcRows, 2 * (int64_t)ctx->n_sms);
    const __nv_bfloat16* wu = (const __nv_bfloat16*)m->d_wb;
    if (m->nloc == 4)
      MK_COUNT(), k_mlp_forward_tc<4><<<blocks, kTcRows, 0, s>>>(S, wu, X, Y, ctx->d_fault);
    else
      MK_COUNT(), k_mlp_forward_tc<10><<<blocks, kTcRows, 0, s>>>(S, wu, X, Y, ctx->d_fault);
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
