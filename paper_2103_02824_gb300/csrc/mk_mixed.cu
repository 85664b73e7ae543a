// Mixed-precision correction solve: FP32 patch-based operator inside PCG, FP64 residuals and iterative refinement.
//
// The operator A = K/2 + M_{V_ext} + sigma M is applied element by element from FP32 element matrices stored in
// patch order; the FP64 residual b - A x is recomputed with the FP64 element matrices after every inner solve and
// decides convergence, so the answer is the FP64 answer to rtol whatever the inner precision.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "mk_device.cuh"
#include "mk_patch.cuh"
#include "mk_regapply.cuh"

namespace mk {

// y = A x for one patch per CTA (see patch_apply); NCG > 0: the number of column groups fixed at compile time.
template <int NLOC, typename T, int VEC, int NCG>
__global__ void __launch_bounds__(256) k_apply_patch(const int32_t* __restrict__ elem_off,
                                                     const int32_t* __restrict__ node_off,
                                                     const int32_t* __restrict__ conn, const T* __restrict__ Ae,
                                                     const int32_t* __restrict__ target,
                                                     const int32_t* __restrict__ inc_off,
                                                     const uint16_t* __restrict__ inc,
                                                     const uint8_t* __restrict__ bnd, int mask,
                                                     const T* __restrict__ x, T* __restrict__ y, T* __restrict__ halo,
                                                     int ncolg, int col0, int ld, int pe, int max_nodes) {
  extern __shared__ __align__(16) unsigned char smraw[];
  patch_apply<NLOC, T, VEC, NCG>(blockIdx.x, elem_off, node_off, conn, Ae, target, inc_off, inc, bnd, mask, x, y,
                                 halo, ncolg, col0, ld, pe, max_nodes, smraw);
}

// y = A x over a persistent grid of CTAs, each looping over its patches with the next patch's bulk copies in
// flight (see patch_apply_pipelined).
template <int NLOC, typename T, int VEC, int NCG>
__global__ void __launch_bounds__(kStreamThreads, 2) k_apply_stream(const unsigned char* __restrict__ rec,
                                                          const int64_t* __restrict__ rec_off,
                                                          const T* __restrict__ Ae, int mask,
                                                          const T* __restrict__ x, T* __restrict__ y,
                                                          T* __restrict__ halo, int col0, int ld, int pe,
                                                          int max_nodes, int max_rec, int n_patches, int64_t n_nodes,
                                                          int64_t n_elems, int* __restrict__ fault,
                                                          int wait_limit) {
  extern __shared__ __align__(16) unsigned char smraw[];
  patch_apply_pipelined<NLOC, T, VEC, NCG>(rec, rec_off, Ae, mask, x, y, halo, col0, ld, pe, max_nodes, max_rec,
                                           n_patches, n_nodes, n_elems, fault, wait_limit, smraw);
}

// y = A x (FP32), one CTA per patch, one element per thread, the element matrices staged in registers and the x
// rows in shared memory (see patch_apply_reg).  At most 128 registers a thread, so four 128-thread CTAs share an SM.
template <int NLOC, int WMAX>
__global__ void __launch_bounds__(kRegMaxThreads, 2) k_apply_reg(const unsigned char* __restrict__ rec, int rec_stride,
                                                                 const float* __restrict__ Ae, int mask,
                                                                 const float* __restrict__ x, float* __restrict__ y,
                                                                 float* __restrict__ halo, int col0, int W, int ld,
                                                                 int pe, int max_nodes, int64_t n_nodes,
                                                                 int64_t n_elems, int* __restrict__ fault) {
  extern __shared__ __align__(16) unsigned char smraw_reg[];
  patch_apply_reg<NLOC, WMAX>((int)blockIdx.x, rec, rec_stride, Ae, mask, x, y, halo, col0, W, ld, pe, max_nodes,
                              n_nodes, n_elems, fault, smraw_reg);
}

template <typename T, int VEC>
__global__ void k_halo(int64_t nshared, const int32_t* __restrict__ node, const int32_t* __restrict__ off,
                       const uint8_t* __restrict__ bnd, int mask, const T* __restrict__ halo, T* __restrict__ y,
                       int ncolg, int col0, int ld) {
  halo_sum<T, VEC>((int64_t)blockIdx.x * blockDim.x + threadIdx.x, nshared, node, off, bnd, mask, halo, y, ncolg,
                   col0, ld);
}

template <typename T>
__global__ void k_pack_elements(int64_t E, int np, int nps, const int32_t* __restrict__ elem_id,
                                const double* __restrict__ A64, T* __restrict__ A) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= E * nps) return;
  const int64_t i = t / nps;
  const int k = (int)(t - i * nps);
  A[t] = k < np ? (T)A64[(int64_t)elem_id[i] * np + k] : (T)0;
}

// The shared nodes' rows of y from their halo slots, columns [col0, col0 + ncolg * vec).
template <typename T>
static int halo_pass(mk_ctx* ctx, const mk_mesh* m, const T* halo, T* y, bool mask, int ncolg, int vec, int col0,
                     int ld, cudaStream_t s) {
  const Patches& P = m->patches;
  const Level& L = m->fine;
  constexpr int VEC = sizeof(T) == 4 ? 4 : 2;
  const int64_t work = P.n_shared_nodes * ncolg;
  if (work == 0) return MK_OK;
  prof_mark(ctx, PROF_HALO, true, s);
  if (vec == VEC)
    MK_COUNT(), k_halo<T, VEC><<<(int)((work + 255) / 256), 256, 0, s>>>(P.n_shared_nodes, P.d_shared_node,
                                                                       P.d_shared_off, L.d_boundary, mask, halo, y,
                                                                       ncolg, col0, ld);
  else
    MK_COUNT(), k_halo<T, 1><<<(int)((work + 255) / 256), 256, 0, s>>>(P.n_shared_nodes, P.d_shared_node,
                                                                     P.d_shared_off, L.d_boundary, mask, halo, y,
                                                                     ncolg, col0, ld);
  prof_mark(ctx, PROF_HALO, false, s);
  return MK_OK;
}

template <int NL, typename T, int PV, int G>
static int launch_stream_kernel(mk_ctx* ctx, const mk_mesh* m, const T* Ae, const T* x, T* y, T* halo, int col0,
                                int ld, bool mask, size_t ssm, int th, cudaStream_t s) {
  const Patches& P = m->patches;
  const Level& L = m->fine;
  auto kern = k_apply_stream<NL, T, PV, G>;
  MK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm));
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, th, ssm) != cudaSuccess || bps < 1) bps = 1;
  const int grid = (int)std::min<int64_t>(P.n_patches, (int64_t)ctx->n_sms * bps);
  MK_COUNT(), kern<<<grid, th, ssm, s>>>(P.d_rec, P.d_rec_off, Ae, mask, x, y, halo, col0, ld, P.max_elems,
                                         P.max_nodes, P.max_rec_bytes, P.n_patches, L.n_nodes, L.n_elems,
                                         ctx->d_fault, ctx->wait_limit);
  return MK_OK;
}

// The pipelined patch kernel for columns [col0, col0 + W), if its shared memory fits and an instance exists for
// this column width (*launched = 1); product items take 4 FP32 columns or 2 FP64 ones.
template <typename T>
static int launch_stream(mk_ctx* ctx, const mk_mesh* m, const T* Ae, const T* x, T* y, T* halo, int col0, int W,
                         int ld, bool mask, cudaStream_t s, int* launched) {
  const Patches& P = m->patches;
  const int nloc = m->fine.nloc;
  *launched = 0;
  const size_t ssm = stream_smem(nloc, P.max_elems, P.max_nodes, P.max_rec_bytes, W, (int)sizeof(T)).total;
  if (ssm > 227 * 1024) return MK_OK;
  constexpr int pv = sizeof(T) == 8 ? 2 : 4;
  if (W % pv) return MK_OK;
  const int th = kStreamThreads;
  const int kind = sizeof(T) == 4 ? PROF_APPLY32 : PROF_APPLY64;
  int r = MK_OK;
  prof_mark(ctx, kind, true, s);
#define MK_SL(NL, PVV, G) (r = launch_stream_kernel<NL, T, PVV, G>(ctx, m, Ae, x, y, halo, col0, ld, mask, ssm, th, s), *launched = 1)
#define MK_SD(NL)                                                        \
  do {                                                                   \
    if constexpr (sizeof(T) == 8) {                                      \
      if (W == 2) MK_SL(NL, 2, 1);                                       \
      else if (W == 4) MK_SL(NL, 2, 2);                                  \
    } else {                                                             \
      if (W == 4) MK_SL(NL, 4, 1);                                       \
      else if (W == 8) MK_SL(NL, 4, 2);                                  \
      else if (W == 12) MK_SL(NL, 4, 3);                                 \
      else if (W == 16) MK_SL(NL, 4, 4);                                 \
    }                                                                    \
  } while (0)
  if (nloc == 4) MK_SD(4);
  else MK_SD(10);
#undef MK_SD
#undef MK_SL
  prof_mark(ctx, kind, false, s);
  return r;
}

// The register-staged kernel for FP32 columns [col0, col0 + W), W in {4, 8} (*launched = 1 if it ran).
static int launch_reg(mk_ctx* ctx, const mk_mesh* m, const float* Ae, const float* x, float* y, float* halo,
                      int col0, int W, int ld, bool mask, cudaStream_t s, int* launched) {
  const Patches& P = m->patches;
  const Level& L = m->fine;
  *launched = 0;
  if (W < 4 || W > 32 || W % 4 != 0 || P.max_elems > kRegMaxThreads) return MK_OK;
  const int wmax = W <= 8 ? 8 : 32;
  const size_t ssm = reg_smem(L.nloc, P.max_elems, P.max_nodes, P.max_rec_bytes, wmax).total;
  if (ssm > 227 * 1024) return MK_OK;
  const int th = (P.max_elems + 31) / 32 * 32;
  prof_mark(ctx, PROF_APPLY32, true, s);
#define MK_RG(NL, WW)                                                                                           \
  do {                                                                                                          \
    auto kern = k_apply_reg<NL, WW>;                                                                            \
    if (ssm > 48 * 1024) MK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm)); \
    MK_COUNT(), kern<<<P.n_patches, th, ssm, s>>>(P.d_rec, P.max_rec_bytes, Ae, mask, x, y, halo, col0, W, ld,  \
                                                  P.max_elems, P.max_nodes, L.n_nodes, L.n_elems, ctx->d_fault); \
  } while (0)
  if (L.nloc == 4) {
    if (wmax == 8) MK_RG(4, 8); else MK_RG(4, 32);
  } else {
    if (wmax == 8) MK_RG(10, 8); else MK_RG(10, 32);
  }
#undef MK_RG
  prof_mark(ctx, PROF_APPLY32, false, s);
  *launched = 1;
  return MK_OK;
}

// y = A x with the patch operator (all ld columns), FP32 or FP64.
template <typename T>
int apply_patch(mk_ctx* ctx, const mk_mesh* m, const T* Ae, const T* x, T* y, int ld, bool mask, cudaStream_t s) {
  const Patches& P = m->patches;
  const Level& L = m->fine;
  int err = MK_OK;
  T* halo = (T*)scratch(ctx, sizeof(T) == 4 ? S_HALO : S_HALO64, (size_t)std::max<int64_t>(P.n_halo_slots, 1) * ld * sizeof(T), &err);
  if (!halo) return err;
  constexpr int VEC = sizeof(T) == 4 ? 4 : 2;
  const int vec = (ld % VEC == 0) ? VEC : 1;
  const int nloc = L.nloc;
  // the pipelined kernel stages x rows in 16-byte copies: x aligned, ld a multiple of 16 bytes
  const bool pipe_ok = ctx->patch_kernel != 0 && ld % (16 / (int)sizeof(T)) == 0 &&
                       (reinterpret_cast<uintptr_t>(x) & 15) == 0 && (reinterpret_cast<uintptr_t>(y) & 15) == 0 &&
                       (reinterpret_cast<uintptr_t>(halo) & 15) == 0 && (reinterpret_cast<uintptr_t>(Ae) & 15) == 0 &&
                       P.d_rec != nullptr;
  // columns per pass: the shared memory of one patch bounds them (16 FP32 / 4 FP64); the pipelined kernel, which
  // holds two patches' products, takes 8 FP32 columns per pass when 16 do not fit
  int wmax = sizeof(T) == 4 ? 16 : 4;
  if (pipe_ok && sizeof(T) == 4 && ld > 8 &&
      stream_smem(nloc, P.max_elems, P.max_nodes, P.max_rec_bytes, std::min(ld, 16), 4).total > 227 * 1024)
    wmax = 8;
  if constexpr (sizeof(T) == 4) {
    // FP32, default: the register-staged kernel, up to 32 columns per launch (every element matrix read once)
    if (pipe_ok && ctx->patch_kernel == 1 && P.max_elems <= kRegMaxThreads) {
      for (int col0 = 0; col0 < ld;) {
        int W = std::min(32, ld - col0);
        int launched = 0;
        MK_TRY(launch_reg(ctx, m, Ae, x, y, halo, col0, W, ld, mask, s, &launched));
        if (!launched && W > 8) {  // the wide block's x rows do not fit: 8 columns per launch
          W = 8;
          MK_TRY(launch_reg(ctx, m, Ae, x, y, halo, col0, W, ld, mask, s, &launched));
        }
        if (!launched) return fail(MK_ERR_UNSUPPORTED, "patch operator: register-staged kernel does not fit");
        MK_TRY(halo_pass<T>(ctx, m, halo, y, mask, W / 4, 4, col0, ld, s));
        col0 += W;
      }
      MK_CUDA(cudaGetLastError());
      return MK_OK;
    }
  }
  for (int col0 = 0; col0 < ld; col0 += wmax) {
    const int W = std::min(wmax, ld - col0);
    const int ncolg = W / vec;
    if (pipe_ok) {
      int launched = 0;
      MK_TRY(launch_stream<T>(ctx, m, Ae, x, y, halo, col0, W, ld, mask, s, &launched));
      if (launched) {
        MK_TRY(halo_pass<T>(ctx, m, halo, y, mask, W / (16 / (int)sizeof(T)), 16 / (int)sizeof(T), col0, ld, s));
        continue;
      }
    }
    const size_t smem = patch_smem(nloc, P.max_elems, P.max_nodes, W, (int)sizeof(T)).total;
    if (smem > 227 * 1024) return fail(MK_ERR_UNSUPPORTED, "patch operator: patch too large for shared memory");
    const int th = std::min(256, (P.max_elems * ncolg + 31) / 32 * 32);  // one phase-1 item per thread
    prof_mark(ctx, sizeof(T) == 4 ? PROF_APPLY32 : PROF_APPLY64, true, s);
#define MK_PATCH_LAUNCH(NL, V, G)                                                                                    \
  do {                                                                                                              \
    auto kern = k_apply_patch<NL, T, V, G>;                                                                         \
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);       \
    MK_COUNT(), kern<<<P.n_patches, th, smem, s>>>(P.d_patch_elem_off, P.d_patch_node_off, P.d_conn, Ae,            \
                                                    P.d_node_target, P.d_inc_off, P.d_inc, L.d_boundary, mask, x, y, \
                                                    halo, ncolg, col0, ld, P.max_elems, P.max_nodes);               \
  } while (0)
#define MK_PATCH_DISPATCH(NL)                                      \
  do {                                                             \
    if (vec == VEC) {                                              \
      if (ncolg == 1) MK_PATCH_LAUNCH(NL, VEC, 1);                 \
      else if (ncolg == 2) MK_PATCH_LAUNCH(NL, VEC, 2);            \
      else if (ncolg == 4) MK_PATCH_LAUNCH(NL, VEC, 4);            \
      else MK_PATCH_LAUNCH(NL, VEC, 0);                            \
    } else {                                                       \
      if (ncolg == 1) MK_PATCH_LAUNCH(NL, 1, 1);                   \
      else MK_PATCH_LAUNCH(NL, 1, 0);                              \
    }                                                              \
  } while (0)
    if (nloc == 4) MK_PATCH_DISPATCH(4);
    else MK_PATCH_DISPATCH(10);
#undef MK_PATCH_DISPATCH
#undef MK_PATCH_LAUNCH
    prof_mark(ctx, sizeof(T) == 4 ? PROF_APPLY32 : PROF_APPLY64, false, s);
    MK_TRY(halo_pass<T>(ctx, m, halo, y, mask, ncolg, vec, col0, ld, s));
  }
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

template int apply_patch<float>(mk_ctx*, const mk_mesh*, const float*, const float*, float*, int, bool, cudaStream_t);
template int apply_patch<double>(mk_ctx*, const mk_mesh*, const double*, const double*, double*, int, bool,
                                 cudaStream_t);

// ------------------------------------------------------------------------------------------------ FP32-pair apply
// The FP64-accurate operator on the FP32 units (patch_apply_pair): element matrices split into FP32 pairs once per
// solve, x split before each application, node sums and halo in FP64.
template <int NLOC, int VEC, int NCG>
__global__ void __launch_bounds__(256) k_apply_pair(const int32_t* __restrict__ elem_off,
                                                    const int32_t* __restrict__ node_off,
                                                    const int32_t* __restrict__ conn, const float* __restrict__ Ah,
                                                    const float* __restrict__ Al, const int32_t* __restrict__ target,
                                                    const int32_t* __restrict__ inc_off,
                                                    const uint16_t* __restrict__ inc, int mask,
                                                    const float* __restrict__ xh, const float* __restrict__ xl,
                                                    double* __restrict__ y, double* __restrict__ halo, int ncolg,
                                                    int col0, int ld, int pe, int max_nodes) {
  extern __shared__ __align__(16) unsigned char smraw[];
  patch_apply_pair<NLOC, VEC, NCG>(blockIdx.x, elem_off, node_off, conn, Ah, Al, target, inc_off, inc, mask, xh, xl,
                                   y, halo, ncolg, col0, ld, pe, max_nodes, smraw);
}

// v -> (hi, lo) = (fl32(v), fl32(v - hi)), for n values
__global__ void k_split_pairs(int64_t n, const double* __restrict__ v, float* __restrict__ hi, float* __restrict__ lo) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double a = v[t];
  const float h = (float)a;
  hi[t] = h;
  lo[t] = (float)(a - (double)h);
}

// The pair parts of the FP64 element matrices in patch order with padded rows (as pack_elements).
__global__ void k_pack_pairs(int64_t E, int np, int nps, const int32_t* __restrict__ elem_id,
                             const double* __restrict__ A64, float* __restrict__ Ah, float* __restrict__ Al) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= E * nps) return;
  const int64_t i = t / nps;
  const int k = (int)(t - i * nps);
  const double a = k < np ? A64[(int64_t)elem_id[i] * np + k] : 0.0;
  const float h = (float)a;
  Ah[t] = h;
  Al[t] = (float)(a - (double)h);
}

int pack_pairs(mk_ctx* ctx, const mk_mesh* m, const double* A64, float* Ah, float* Al, cudaStream_t s) {
  (void)ctx;
  const Level& L = m->fine;
  const int np = L.nloc * (L.nloc + 1) / 2;
  const int nps = padded_np(L.nloc, 4);
  const int64_t work = L.n_elems * nps;
  MK_COUNT(), k_pack_pairs<<<(int)((work + 255) / 256), 256, 0, s>>>(L.n_elems, np, nps, m->patches.d_elem_id, A64,
                                                                     Ah, Al);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

// y = A x (all ld columns, FP64 in and out) from the pair parts Ah, Al of the element matrices.
int apply_pair(mk_ctx* ctx, const mk_mesh* m, const float* Ah, const float* Al, const double* x, double* y, int ld,
               bool mask, cudaStream_t s) {
  const Patches& P = m->patches;
  const Level& L = m->fine;
  const int64_t n = L.n_nodes;
  int err = MK_OK;
  double* halo = (double*)scratch(ctx, S_HALO64, (size_t)std::max<int64_t>(P.n_halo_slots, 1) * ld * sizeof(double), &err);
  float* xh = (float*)scratch(ctx, S_PAIRX, (size_t)2 * n * ld * sizeof(float), &err);
  if (!halo || !xh) return err;
  float* xl = xh + (size_t)n * ld;
  MK_COUNT(), k_split_pairs<<<(int)((n * ld + 255) / 256), 256, 0, s>>>(n * ld, x, xh, xl);
  constexpr int VEC = 2;
  const int vec = (ld % VEC == 0) ? VEC : 1;
  const int nloc = L.nloc;
  const int wmax = 4;
  for (int col0 = 0; col0 < ld; col0 += wmax) {
    const int W = std::min(wmax, ld - col0);
    const int ncolg = W / vec;
    const size_t smem = pair_smem(nloc, P.max_elems, P.max_nodes, W).total;
    if (smem > 227 * 1024) return fail(MK_ERR_UNSUPPORTED, "pair operator: patch too large for shared memory");
    const int th = std::min(256, (P.max_elems * ncolg + 31) / 32 * 32);
    prof_mark(ctx, PROF_PAIRS, true, s);
#define MK_PAIR_LAUNCH(NL, V, G)                                                                                   \
  do {                                                                                                            \
    auto kern = k_apply_pair<NL, V, G>;                                                                           \
    if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);     \
    MK_COUNT(), kern<<<P.n_patches, th, smem, s>>>(P.d_patch_elem_off, P.d_patch_node_off, P.d_conn, Ah, Al,      \
                                                    P.d_node_target, P.d_inc_off, P.d_inc, mask, xh, xl, y, halo, \
                                                    ncolg, col0, ld, P.max_elems, P.max_nodes);                  \
  } while (0)
#define MK_PAIR_DISPATCH(NL)                                  \
  do {                                                        \
    if (vec == VEC) {                                         \
      if (ncolg == 1) MK_PAIR_LAUNCH(NL, VEC, 1);             \
      else if (ncolg == 2) MK_PAIR_LAUNCH(NL, VEC, 2);        \
      else MK_PAIR_LAUNCH(NL, VEC, 0);                        \
    } else {                                                  \
      if (ncolg == 1) MK_PAIR_LAUNCH(NL, 1, 1);               \
      else MK_PAIR_LAUNCH(NL, 1, 0);                          \
    }                                                         \
  } while (0)
    if (nloc == 4) MK_PAIR_DISPATCH(4);
    else MK_PAIR_DISPATCH(10);
#undef MK_PAIR_DISPATCH
#undef MK_PAIR_LAUNCH
    prof_mark(ctx, PROF_PAIRS, false, s);
    MK_TRY(halo_pass<double>(ctx, m, halo, y, mask, ncolg, vec, col0, ld, s));
  }
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

// y = A x on FP32 pairs from FP64 element matrices in their original order (packed on every call).
int apply64_pairs(mk_ctx* ctx, const mk_mesh* m, const double* A64, const double* x, double* y, int ld, bool mask,
                  cudaStream_t s) {
  const Level& L = m->fine;
  const size_t na = (size_t)L.n_elems * padded_np(L.nloc, 4);
  int err = MK_OK;
  float* Ah = (float*)scratch(ctx, S_PAIRA, 2 * na * sizeof(float), &err);
  if (!Ah) return err;
  MK_TRY(pack_pairs(ctx, m, A64, Ah, Ah + na, s));
  return apply_pair(ctx, m, Ah, Ah + na, x, y, ld, mask, s);
}

// Element matrices of the patch operator from FP64 originals (patch order).
template <typename T>
int pack_elements(mk_ctx* ctx, const mk_mesh* m, const double* A64, T* A, cudaStream_t s) {
  (void)ctx;
  const Level& L = m->fine;
  const int np = L.nloc * (L.nloc + 1) / 2;
  const int nps = padded_np(L.nloc, (int)sizeof(T));
  const int64_t work = L.n_elems * nps;
  MK_COUNT(), k_pack_elements<T><<<(int)((work + 255) / 256), 256, 0, s>>>(L.n_elems, np, nps, m->patches.d_elem_id,
                                                                           A64, A);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}
template int pack_elements<float>(mk_ctx*, const mk_mesh*, const double*, float*, cudaStream_t);
template int pack_elements<double>(mk_ctx*, const mk_mesh*, const double*, double*, cudaStream_t);

// ------------------------------------------------------------------------------------------------ stiffness operator
// Matrix-free FP32 stiffness operator y = K x (the Hartree Poisson operator).  Per element six factors
// f_c = |det J| (J^-1 J^-T)_{ij} (ij = 00, 11, 22, 01, 02, 12) and K_e = sum_c f_c Khat_c, with Khat_c the reference
// stiffness components (the tables the FP64 element matrices are built from), so an element streams 32 bytes of
// factors instead of 55 matrix values.  One CTA per patch, owner-computes sums in the fixed order of patch_apply.
struct StiffRef {
  float k[6][55];  // packed symmetric reference components (P1 uses the first 10 of each)
};

__global__ void k_stiff_factors(int64_t E, const int32_t* __restrict__ elem_id, const Geom* __restrict__ geom,
                                float* __restrict__ fac) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  const Geom g = geom[elem_id[i]];
  const double det = fabs(g.det);
  const int I6[6] = {0, 1, 2, 0, 0, 1}, J6[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const double G = g.Jinv[I6[c] * 3] * g.Jinv[J6[c] * 3] + g.Jinv[I6[c] * 3 + 1] * g.Jinv[J6[c] * 3 + 1] +
                     g.Jinv[I6[c] * 3 + 2] * g.Jinv[J6[c] * 3 + 2];
    fac[i * 8 + c] = (float)(det * G);
  }
  fac[i * 8 + 6] = 0.f;
  fac[i * 8 + 7] = 0.f;
}

// Shared memory of one stiffness-patch CTA: the layout of patch_apply with the element-matrix region holding the
// eight factors of each element instead.
__host__ __device__ inline PatchSmem stiff_smem(int nloc, int pe, int max_nodes, int W) {
  PatchSmem L;
  L.ye = 0;
  L.as = L.ye + align16((size_t)nloc * pe * W * 4);
  L.conn = L.as + align16((size_t)pe * 8 * 4 + 16);
  L.inc = L.conn + align16((size_t)pe * nloc * 4 + 16);
  L.ioff = L.inc + align16((size_t)pe * nloc * 2 + 16);
  L.tgt = L.ioff + align16((size_t)(max_nodes + 1) * 4 + 16);
  L.total = L.tgt + align16((size_t)max_nodes * 4 + 16);
  return L;
}

template <int NLOC>
__global__ void __launch_bounds__(128, 8) k_stiff_patch(const int32_t* __restrict__ elem_off,
                                                    const int32_t* __restrict__ node_off,
                                                    const int32_t* __restrict__ conn, const float* __restrict__ fac,
                                                    const int32_t* __restrict__ target,
                                                    const int32_t* __restrict__ inc_off,
                                                    const uint16_t* __restrict__ inc, int mask,
                                                    const float* __restrict__ x, float* __restrict__ y,
                                                    float* __restrict__ halo, int ncol, int ld, int pe, int max_nodes,
                                                    const StiffRef ref) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const PatchSmem lay = stiff_smem(NLOC, pe, max_nodes, ncol);
  float* Ye = reinterpret_cast<float*>(smraw + lay.ye);  // [NLOC][pe][ncol]
  const int p = blockIdx.x;
  const int e0 = elem_off[p], ne = elem_off[p + 1] - e0;
  const int n0 = node_off[p], nl = node_off[p + 1] - n0;
  const int ibase = e0 * NLOC;
  const float* fs = stage_async(smraw + lay.as, fac + (int64_t)e0 * 8, ne * 8 * 4);
  const int32_t* cs = stage_async(smraw + lay.conn, conn + ibase, ne * NLOC * 4);
  const uint16_t* is = stage_async(smraw + lay.inc, inc + ibase, ne * NLOC * 2);
  const int32_t* os = stage_async(smraw + lay.ioff, inc_off + n0, (nl + 1) * 4);
  const int32_t* ts = stage_async(smraw + lay.tgt, target + n0, nl * 4);
  cp_async_wait_all();
  __syncthreads();
  constexpr int NP = NLOC * (NLOC + 1) / 2;
  for (int it = threadIdx.x; it < ne * ncol; it += blockDim.x) {
    const int el = it / ncol, col = it - el * ncol;
    float xv[NLOC];
#pragma unroll
    for (int a = 0; a < NLOC; ++a) xv[a] = x[(int64_t)cs[el * NLOC + a] * ld + col];
    // y_e = sum_c f_c (Khat_c x_e): the reference components come from the constant bank, so a thread keeps only
    // x_e, y_e and one Khat_c x_e in registers (many CTAs per SM hide the gather latency)
    float acc[NLOC];
#pragma unroll
    for (int a = 0; a < NLOC; ++a) acc[a] = 0.f;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      float t[NLOC];
#pragma unroll
      for (int a = 0; a < NLOC; ++a) t[a] = 0.f;
#pragma unroll
      for (int a = 0; a < NLOC; ++a)
#pragma unroll
        for (int b = a; b < NLOC; ++b) {
          const float w = ref.k[c][sym_index(a, b, NLOC)];
          t[a] = fmaf(w, xv[b], t[a]);
          if (b != a) t[b] = fmaf(w, xv[a], t[b]);
        }
      const float fc = fs[el * 8 + c];
#pragma unroll
      for (int a = 0; a < NLOC; ++a) acc[a] = fmaf(fc, t[a], acc[a]);
    }
    (void)NP;
#pragma unroll
    for (int a = 0; a < NLOC; ++a) Ye[((size_t)a * pe + el) * ncol + col] = acc[a];
  }
  __syncthreads();
  for (int it = threadIdx.x; it < nl * ncol; it += blockDim.x) {
    const int l = it / ncol, col = it - l * ncol;
    const int b = os[l] - ibase, e = os[l + 1] - ibase;
    float acc = 0.f;
    int k = b;
    for (; k + 4 <= e; k += 4) {
      const float v0 = Ye[(size_t)is[k] * ncol + col], v1 = Ye[(size_t)is[k + 1] * ncol + col];
      const float v2 = Ye[(size_t)is[k + 2] * ncol + col], v3 = Ye[(size_t)is[k + 3] * ncol + col];
      acc = (((acc + v0) + v1) + v2) + v3;
    }
    for (; k < e; ++k) acc += Ye[(size_t)is[k] * ncol + col];
    const int t = ts[l];
    if (t >= 0) {
      if (mask && (t & kOwnedBoundary)) acc = 0.f;
      y[(int64_t)(t & (kOwnedBoundary - 1)) * ld + col] = acc;
    } else {
      halo[(int64_t)(-t - 1) * ld + col] = acc;
    }
  }
}

// The six patch-ordered stiffness factors per element of mesh m (computed on first use, kept in the mesh handle).
static const float* stiff_factors(const mk_mesh* m, cudaStream_t s, int* err) {
  const Patches& P = m->patches;
  if (P.d_stiff_fac) return P.d_stiff_fac;
  const Level& L = m->fine;
  if (cudaMalloc(&P.d_stiff_fac, (size_t)L.n_elems * 8 * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    *err = fail(MK_ERR_OOM, "stiffness factors: allocation failed");
    return nullptr;
  }
  MK_COUNT(), k_stiff_factors<<<(int)((L.n_elems + 255) / 256), 256, 0, s>>>(L.n_elems, P.d_elem_id, L.d_geom,
                                                                            P.d_stiff_fac);
  return P.d_stiff_fac;
}

// y = K x with the matrix-free stiffness operator (all ld columns, boundary rows zero when mask).
static int apply_stiff(mk_ctx* ctx, const mk_mesh* m, const float* x, float* y, int ld, bool mask, cudaStream_t s) {
  const Patches& P = m->patches;
  const Level& L = m->fine;
  int err = MK_OK;
  const float* fac = stiff_factors(m, s, &err);
  float* halo = (float*)scratch(ctx, S_HALO, (size_t)std::max<int64_t>(P.n_halo_slots, 1) * ld * sizeof(float), &err);
  if (!fac || !halo) return err;
  StiffRef ref;
  const RefTables& R = ctx->h_ref[L.order];
  for (int c = 0; c < 6; ++c)
    for (int q = 0; q < 55; ++q) ref.k[c][q] = q < R.npack ? (float)R.stiff[c][q] : 0.f;
  for (int col0 = 0; col0 < ld; col0 += 16) {
    const int W = std::min(16, ld - col0);
    const size_t smem = stiff_smem(L.nloc, P.max_elems, P.max_nodes, W).total;
    if (smem > 227 * 1024) return fail(MK_ERR_UNSUPPORTED, "stiffness operator: patch too large for shared memory");
    prof_mark(ctx, PROF_STIFF, true, s);
    if (L.nloc == 4) {
      if (smem > 48 * 1024) cudaFuncSetAttribute(k_stiff_patch<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      MK_COUNT(), k_stiff_patch<4><<<P.n_patches, 128, smem, s>>>(P.d_patch_elem_off, P.d_patch_node_off, P.d_conn,
                                                                  fac, P.d_node_target, P.d_inc_off, P.d_inc, mask,
                                                                  x + col0, y + col0, halo + col0, W, ld,
                                                                  P.max_elems, P.max_nodes, ref);
    } else {
      if (smem > 48 * 1024) cudaFuncSetAttribute(k_stiff_patch<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      MK_COUNT(), k_stiff_patch<10><<<P.n_patches, 128, smem, s>>>(P.d_patch_elem_off, P.d_patch_node_off, P.d_conn,
                                                                   fac, P.d_node_target, P.d_inc_off, P.d_inc, mask,
                                                                   x + col0, y + col0, halo + col0, W, ld,
                                                                   P.max_elems, P.max_nodes, ref);
    }
    prof_mark(ctx, PROF_STIFF, false, s);
    MK_TRY(halo_pass<float>(ctx, m, halo, y, mask, W, 1, col0, ld, s));
  }
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

// ------------------------------------------------------------------------------------------------ two-level
// Coarse-space correction of the preconditioner (two-level additive, the coarse space V_H of the method):
// t = P^T r restricted to the coarse free DOF, y = A_H^-1 t with the dense inverse of the Galerkin coarse operator
// A_H = P^T A P, then z = (Jacobi or learned part) + P y.  FP32; every sum has a fixed order.
constexpr int kTLC = 8;  // orbital columns per pass

constexpr int kTLS = 32;  // segments (warps) per coarse DOF in the restriction
constexpr int kTLW = 8;   // warps per CTA of the restriction
static_assert(kTLS % kTLW == 0, "a restriction CTA holds whole segments of one or more coarse DOF");

// tp[k][seg][j] = sum over segment seg of the support of coarse DOF k of P^T[k][i] v[i][j], v = r, or r - q when
// q is given (boundary rows of both are zero: masked residual, masked operator); one CTA of kTLS warps per coarse
// DOF, warp seg takes segment seg (lane-strided, then a fixed shuffle tree), so no CTA barrier is needed; a CTA
// holds kTLW consecutive (coarse DOF, segment) warps.
__global__ void __launch_bounds__(kTLW * 32) k_tl_restrict(const int32_t* __restrict__ off,
                                                          const int32_t* __restrict__ col,
                                                          const float* __restrict__ val, const float* __restrict__ r,
                                                          const float* __restrict__ q, int ld, int N,
                                                          float* __restrict__ tp) {
  const int gw = blockIdx.x * kTLW + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  const int k = gw / kTLS, seg = gw % kTLS;
  const int b0 = off[k], len = off[k + 1] - b0;
  const int b = b0 + (int)((int64_t)len * seg / kTLS), e = b0 + (int)((int64_t)len * (seg + 1) / kTLS);
  for (int c0 = 0; c0 < N; c0 += kTLC) {
    const int nc = min(kTLC, N - c0);
    float acc[kTLC];
#pragma unroll
    for (int c = 0; c < kTLC; ++c) acc[c] = 0.f;
#pragma unroll 4
    for (int i = b + lane; i < e; i += 32) {
      const float w = val[i];
      const int64_t o = (int64_t)col[i] * ld + c0;
#pragma unroll
      for (int c = 0; c < kTLC; ++c)
        if (c < nc) acc[c] = fmaf(w, q ? r[o + c] - q[o + c] : r[o + c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < kTLC; ++c)
      if (c < nc) {  // nc is uniform over the warp
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], o);
      }
    if (lane == 0)
#pragma unroll
      for (int c = 0; c < kTLC; ++c)
        if (c < nc) tp[((int64_t)k * kTLS + seg) * ld + c0 + c] = acc[c];
  }
}

// y[k][j] = sum_l Ainv[k][l] t[l][j] with t[l][j] = sum over segments of tp[l][seg][j] (in order); a CTA first
// forms t for its column chunk in shared memory, then each of its warps takes one coarse DOF k.
constexpr int kTLRows = 8;  // coarse DOF per CTA (one per warp)
__global__ void __launch_bounds__(kTLRows * 32) k_tl_coarse(int nH, const float* __restrict__ Ainv,
                                                           const float* __restrict__ tp, int ld, int N,
                                                           float* __restrict__ y) {
  extern __shared__ float tsh[];  // [nH][kTLC]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * kTLRows + warp;
  for (int c0 = 0; c0 < N; c0 += kTLC) {
    const int nc = min(kTLC, N - c0);
    for (int i = threadIdx.x; i < nH * nc; i += blockDim.x) {
      const int l = i / nc, c = i - l * nc;
      float t = 0.f;
#pragma unroll
      for (int sg = 0; sg < kTLS; ++sg) t += tp[((int64_t)l * kTLS + sg) * ld + c0 + c];
      tsh[l * kTLC + c] = t;
    }
    __syncthreads();
    if (k < nH) {
      float acc[kTLC];
#pragma unroll
      for (int c = 0; c < kTLC; ++c) acc[c] = 0.f;
      for (int l = lane; l < nH; l += 32) {
        const float a = Ainv[(int64_t)k * nH + l];
#pragma unroll
        for (int c = 0; c < kTLC; ++c)
          if (c < nc) acc[c] = fmaf(a, tsh[l * kTLC + c], acc[c]);
      }
#pragma unroll
      for (int c = 0; c < kTLC; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], o);
      }
      if (lane == 0)
#pragma unroll
        for (int c = 0; c < kTLC; ++c)
          if (c < nc) y[(int64_t)k * ld + c0 + c] = acc[c];
    }
    __syncthreads();
  }
}

__global__ void k_tl_prolong(int64_t n, const int32_t* __restrict__ off, const int32_t* __restrict__ col,
                             const float* __restrict__ val, const float* __restrict__ y,
                             const float* __restrict__ dinv, const uint8_t* __restrict__ bnd,
                             const float* __restrict__ r, float* __restrict__ z, int ld, int N, int add) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * N) return;
  const int64_t i = t / N;
  const int j = (int)(t - i * N);
  const int64_t idx = i * ld + j;
  if (bnd[i]) {
    z[idx] = 0.f;
    return;
  }
  float acc = add ? z[idx] : dinv[i] * r[idx];
  for (int q = off[i]; q < off[i + 1]; ++q) acc = fmaf(val[q], y[(int64_t)col[q] * ld + j], acc);
  z[idx] = acc;
}

__global__ void k_f64_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// FP32 copies of the values of P and P^T (built once per mesh, before any graph capture uses them).
int tl_prepare(const mk_mesh* m, cudaStream_t s) {
  if (m->d_P_val32) return MK_OK;
  const int64_t nP = m->PT_nnz;  // P and P^T hold the same entries
  float *a = nullptr, *b = nullptr;
  if (cudaMalloc(&a, (size_t)std::max<int64_t>(nP, 1) * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&b, (size_t)std::max<int64_t>(nP, 1) * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(a);
    return fail(MK_ERR_OOM, "two-level preconditioner: allocation failed");
  }
  MK_COUNT(), k_f64_to_f32<<<(int)((nP + 255) / 256), 256, 0, s>>>(nP, m->d_P_val, a);
  MK_COUNT(), k_f64_to_f32<<<(int)((nP + 255) / 256), 256, 0, s>>>(nP, m->d_PT_val, b);
  MK_CUDA(cudaGetLastError());
  m->d_P_val32 = a;
  m->d_PT_val32 = b;
  return MK_OK;
}

// Cached FP32 coarse inverse for the operator of A64: the mesh's Poisson operator (key empty) or the correction
// operator of a molecule and shift (key = Z, R, sigma).  Built on first use.
const float* coarse_inverse_cached(mk_ctx* ctx, const mk_mesh* m, const double* A64, const std::vector<double>* key,
                                   cudaStream_t s, int* err) {
  const int64_t nH = m->coarse.n_free;
  float** slot = key ? &m->d_cinv_corr : &m->d_cinv_poisson;
  if (*slot && (!key || m->cinv_corr_key == *key)) return *slot;
  if (*slot && key && cudaDeviceSynchronize() != cudaSuccess) {  // earlier users of the old inverse finish first
    *err = fail(MK_ERR_CUDA, "two-level preconditioner: cudaDeviceSynchronize failed");
    return nullptr;
  }
  if (!*slot && cudaMalloc(slot, (size_t)nH * nH * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    *slot = nullptr;
    *err = fail(MK_ERR_OOM, "two-level preconditioner: allocation failed");
    return nullptr;
  }
  const int r = coarse_inverse32(ctx, m, A64, *slot, s);
  if (r != MK_OK) {
    *err = r;
    if (key) m->cinv_corr_key.clear();
    return nullptr;
  }
  if (key) m->cinv_corr_key = *key;
  return *slot;
}

// z = (add ? z : D^-1 r) + P A_H^-1 P^T r for columns < N.
// Symmetric multiplicative two-level preconditioner (one damped Jacobi sweep, the coarse correction, one damped
// Jacobi sweep): z = w D^-1 r;  z += P A_H^-1 P^T (r - A z);  z += w D^-1 (r - A z).  The sweep is a smoother, and
// the preconditioner positive definite, while w lambda_max(D^-1 A) < 2.  On the uniform cube meshes lambda_max is
// about 2 for the P1/P2 stiffness matrices and w = kTLOmega = 0.8; on graded meshes it is larger (2.83 on the
// 874,510-tetrahedron graded mesh), so the Poisson preconditioners take w = min(0.8, 1.6 / lambda), lambda estimated
// per level by smoother_omega.  On the 250,047-DOF P2 Poisson problem the multiplicative form takes FCG to 1e-8 in
// 47 iterations against 85 for the additive form (CPU experiment with the same matrices).
constexpr float kTLOmega = 0.8f;
constexpr int kOmegaIts = 50;

// x[i] = a deterministic pseudo-random value in [0.5, 1.5), 0 on boundary rows (bnd may be NULL)
__global__ void k_om_start(int64_t n, const uint8_t* __restrict__ bnd, float* __restrict__ x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t h = (uint32_t)(i * 2654435761ull >> 7) & 1023u;
  x[i] = (bnd && bnd[i]) ? 0.f : 0.5f + (float)h / 1024.f;
}
// part[blk] = (sum x y, sum x^2 / dinv) over the block's grid-stride share (rows with dinv = 0 skipped)
__global__ void k_om_dots(int64_t n, const float* __restrict__ x, const float* __restrict__ y,
                          const float* __restrict__ dinv, double* __restrict__ part) {
  __shared__ double sa[kRedThreads], sb[kRedThreads];
  double a = 0.0, b = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    a += (double)x[i] * y[i];
    if (dinv[i] != 0.f) b += (double)x[i] * x[i] / dinv[i];
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sa[threadIdx.x] += sa[threadIdx.x + w];
      sb[threadIdx.x] += sb[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sa[0];
    part[2 * blockIdx.x + 1] = sb[0];
  }
}
__global__ void k_om_next(int64_t n, const float* __restrict__ dinv, const float* __restrict__ y, float scale,
                          float* __restrict__ x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = scale * dinv[i] * y[i];
}

// Smoother weight of one level: lambda = the Rayleigh quotient (x, A x) / (x, D x) after kOmegaIts steps of the power
// iteration on D^-1 A (a lower bound of lambda_max that rises with the steps), w = min(kTLOmega, 1.6 / lambda).
// apply(x, y): y = A x on the level's n rows (one column).  Synchronises s once per step; run once per level.
template <typename Apply>
static int smoother_omega(mk_ctx* ctx, int64_t n, Apply&& apply, const float* dinv, const uint8_t* bnd,
                          cudaStream_t s, float* omega) {
  int err = MK_OK;
  const int nblk = red_blocks(ctx);
  const size_t vb = ((size_t)n * 2 * sizeof(float) + 255) / 256 * 256;
  char* ws = (char*)scratch(ctx, S_LMAX, vb + (size_t)nblk * 2 * sizeof(double) + 64, &err);
  if (!ws) return err;
  float* x = (float*)ws;
  float* y = x + n;
  double* part = (double*)(ws + vb);
  double* sums = part + 2 * nblk;
  const int gb = (int)((n + 255) / 256);
  MK_COUNT(), k_om_start<<<gb, 256, 0, s>>>(n, bnd, x);
  double lam = 0.0;
  for (int it = 0; it < kOmegaIts; ++it) {
    MK_TRY(apply(x, y));
    MK_COUNT(), k_om_dots<<<nblk, kRedThreads, 0, s>>>(n, x, y, dinv, part);
    sum_partials(part, nblk, 2, sums, s);
    double h[2];
    MK_CUDA(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, s));
    MK_CUDA(cudaStreamSynchronize(s));
    MK_ARG(h[1] > 0.0 && h[0] > 0.0, "multigrid: the level's operator is not positive definite");
    lam = h[0] / h[1];
    MK_COUNT(), k_om_next<<<gb, 256, 0, s>>>(n, dinv, y, (float)(1.0 / lam), x);
  }
  *omega = (float)std::min((double)kTLOmega, 1.6 / lam);
  return MK_OK;
}

__global__ void k_tl_jacobi(int64_t n, const uint8_t* __restrict__ bnd, const float* __restrict__ dinv,
                            const float* __restrict__ r, float* __restrict__ z, int ld, int N, float w) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * N) return;
  const int64_t i = t / N;
  const int64_t idx = i * ld + (t - i * N);
  z[idx] = bnd[i] ? 0.f : w * dinv[i] * r[idx];
}
// mode 0: t = r - q;  mode 1: z += w D^-1 (r - q)
__global__ void k_tl_resid(int64_t n, const uint8_t* __restrict__ bnd, const float* __restrict__ dinv,
                           const float* __restrict__ r, const float* __restrict__ q, float* __restrict__ out, int ld,
                           int N, float w, int mode) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * N) return;
  const int64_t i = t / N;
  const int64_t idx = i * ld + (t - i * N);
  if (bnd[i]) {
    out[idx] = 0.f;
    return;
  }
  const float d = r[idx] - q[idx];
  out[idx] = mode == 0 ? d : fmaf(w * dinv[i], d, out[idx]);
}

// z0_ready: z already holds the first sweep w D^-1 r (written by the FCG update kernel); defer_final: the last
// sweep z += w D^-1 (r - q) is left to the caller's next kernel (q = the S_TLQ scratch, A z at that point).
// ------------------------------------------------------------------------------------------------ multigrid
// The V(1,1) cycle of the Hartree Poisson operator on the nested hierarchy fine mesh > intermediate levels > V_H
// (one column, FP32), the preconditioner of the multigrid FCG: on each level from the fine one down, x = w D^-1 b
// (one damped Jacobi sweep from zero), the residual b - A x restricted to the next level by P^T; on V_H the dense
// inverse of P^T K P; then on each level back up, x += P x_coarse and one more sweep x += w D^-1 (b - A x).  The
// same smoother before and after and restriction = transpose of interpolation: a symmetric positive definite
// preconditioner for w below 2 / lambda_max(D^-1 A) on every level.
__global__ void k_mg_jac0(int64_t n, const float* __restrict__ dinv, const float* __restrict__ b,
                          float* __restrict__ x, float w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = w * dinv[i] * b[i];
}
__global__ void k_mg_post(int64_t n, const float* __restrict__ dinv, const float* __restrict__ b,
                          const float* __restrict__ q, float* __restrict__ x, float w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = fmaf(w * dinv[i], b[i] - q[i], x[i]);
}
// y = K x (CSR, one warp per row)
__global__ void k_mg_spmv(int64_t n, const int32_t* __restrict__ off, const int32_t* __restrict__ col,
                          const float* __restrict__ val, const float* __restrict__ x, float* __restrict__ y) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  float acc = 0.f;
  for (int k = off[row] + lane; k < off[row + 1]; k += 32) acc = fmaf(val[k], x[col[k]], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) y[row] = acc;
}
// out = R (b - q) (R = P^T, one warp per coarse row)
__global__ void k_mg_restrict(int64_t n, const int32_t* __restrict__ off, const int32_t* __restrict__ col,
                              const float* __restrict__ val, const float* __restrict__ b,
                              const float* __restrict__ q, float* __restrict__ out) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  float acc = 0.f;
  for (int k = off[row] + lane; k < off[row + 1]; k += 32) acc = fmaf(val[k], b[col[k]] - q[col[k]], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) out[row] = acc;
}
// x += P xc on the rows with a nonzero inverse diagonal (interior rows)
__global__ void k_mg_prolong(int64_t n, const int32_t* __restrict__ off, const int32_t* __restrict__ col,
                             const float* __restrict__ val, const float* __restrict__ dinv,
                             const float* __restrict__ xc, float* __restrict__ x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || dinv[i] == 0.f) return;
  float acc = x[i];
  for (int k = off[i]; k < off[i + 1]; ++k) acc = fmaf(val[k], xc[col[k]], acc);
  x[i] = acc;
}
// y = Ainv t on V_H (dense, one warp per row)
__global__ void k_mg_dense(int n, const float* __restrict__ Ainv, const float* __restrict__ t, float* __restrict__ y) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  float acc = 0.f;
  for (int k = lane; k < n; k += 32) acc = fmaf(Ainv[(int64_t)row * n + k], t[k], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) y[row] = acc;
}

// z = V-cycle(r) on the fine level (one column); apply32 is the fine operator (matrix-free stiffness), dinv the
// fine inverse diagonal (0 on boundary rows), cinv the dense FP32 inverse of P^T K P on V_H.
template <typename Apply>
static int mg_apply(mk_ctx* ctx, const mk_mesh* m, Apply&& apply32, const float* dinv, const float* cinv,
                    const float* r, float* z, cudaStream_t s, float w) {
  const int nm = (int)m->mg.size();
  const int64_t nf = m->fine.n_nodes, nH = m->coarse.n_free;
  // scratch: the fine operator product, then per intermediate level b, x, q, then b and x on V_H
  size_t total = (size_t)nf;
  for (const MgLevel& g : m->mg) total += 3 * (size_t)g.L.n_nodes;
  total += 2 * (size_t)nH;
  int err = MK_OK;
  float* ws = (float*)scratch(ctx, S_MG, total * sizeof(float), &err);
  if (!ws) return err;
  float* qf = ws;
  std::vector<float*> b(nm), x(nm), q(nm);
  float* p = ws + nf;
  for (int k = 0; k < nm; ++k) {
    const int64_t n = m->mg[k].L.n_nodes;
    b[k] = p; x[k] = p + n; q[k] = p + 2 * n;
    p += 3 * n;
  }
  float* bH = p;
  float* xH = p + nH;
  auto blocks = [](int64_t n) { return (int)((n + 255) / 256); };
  auto wblocks = [](int64_t n) { return (int)((n * 32 + 255) / 256); };
  // down: fine level
  MK_COUNT(), k_mg_jac0<<<blocks(nf), 256, 0, s>>>(nf, dinv, r, z, w);
  MK_TRY(apply32(z, qf));
  float* bc = nm > 0 ? b[nm - 1] : bH;
  MK_COUNT(), k_mg_restrict<<<wblocks(m->mgR.n_rows), 256, 0, s>>>(m->mgR.n_rows, m->mgR.d_off, m->mgR.d_col,
                                                                   m->mgR.d_val, r, qf, bc);
  // down: intermediate levels, finest first
  for (int k = nm - 1; k >= 0; --k) {
    const MgLevel& g = m->mg[k];
    const int64_t n = g.L.n_nodes;
    MK_COUNT(), k_mg_jac0<<<blocks(n), 256, 0, s>>>(n, g.d_dinv, b[k], x[k], g.omega);
    MK_COUNT(), k_mg_spmv<<<wblocks(n), 256, 0, s>>>(n, g.K.d_off, g.K.d_col, g.K.d_val, x[k], q[k]);
    float* bnext = k > 0 ? b[k - 1] : bH;
    MK_COUNT(), k_mg_restrict<<<wblocks(g.R.n_rows), 256, 0, s>>>(g.R.n_rows, g.R.d_off, g.R.d_col, g.R.d_val, b[k],
                                                                  q[k], bnext);
  }
  // V_H
  MK_COUNT(), k_mg_dense<<<(int)((nH * 32 + 255) / 256), 256, 0, s>>>((int)nH, cinv, bH, xH);
  // up: intermediate levels, coarsest first
  for (int k = 0; k < nm; ++k) {
    const MgLevel& g = m->mg[k];
    const int64_t n = g.L.n_nodes;
    const float* xc = k > 0 ? x[k - 1] : xH;
    MK_COUNT(), k_mg_prolong<<<blocks(n), 256, 0, s>>>(n, g.P.d_off, g.P.d_col, g.P.d_val, g.d_dinv, xc, x[k]);
    MK_COUNT(), k_mg_spmv<<<wblocks(n), 256, 0, s>>>(n, g.K.d_off, g.K.d_col, g.K.d_val, x[k], q[k]);
    MK_COUNT(), k_mg_post<<<blocks(n), 256, 0, s>>>(n, g.d_dinv, b[k], q[k], x[k], g.omega);
  }
  // up: fine level
  MK_COUNT(), k_mg_prolong<<<blocks(nf), 256, 0, s>>>(nf, m->mgP.d_off, m->mgP.d_col, m->mgP.d_val, dinv,
                                                      nm > 0 ? x[nm - 1] : xH, z);
  MK_TRY(apply32(z, qf));
  MK_COUNT(), k_mg_post<<<blocks(nf), 256, 0, s>>>(nf, dinv, r, qf, z, w);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

template <typename Apply>
static int twolevel_mult_apply(mk_ctx* ctx, const mk_mesh* m, Apply&& apply32, const float* cinv, const float* dinv,
                               const float* r, float* z, int ld, int N, cudaStream_t s, float w,
                               bool z0_ready = false, bool defer_final = false) {
  const Level& L = m->fine;
  const int nH = (int)m->coarse.n_free;
  int err = MK_OK;
  float* t = (float*)scratch(ctx, S_TLT, (size_t)(kTLS + 1) * nH * ld * sizeof(float), &err);
  float* q = (float*)scratch(ctx, S_TLQ, (size_t)L.n_nodes * ld * sizeof(float), &err);
  if (!t || !q) return err;
  float* y = t + (size_t)kTLS * nH * ld;
  const int gb = (int)((L.n_nodes * N + 255) / 256);
  if (!z0_ready) MK_COUNT(), k_tl_jacobi<<<gb, 256, 0, s>>>(L.n_nodes, L.d_boundary, dinv, r, z, ld, N, w);
  MK_TRY(apply32(z, q));
  MK_COUNT(), k_tl_restrict<<<nH * kTLS / kTLW, kTLW * 32, 0, s>>>(m->d_PT_off, m->d_PT_col, m->d_PT_val32, r, q,
                                                                   ld, N, t);
  MK_COUNT(), k_tl_coarse<<<(nH + kTLRows - 1) / kTLRows, kTLRows * 32, (size_t)nH * kTLC * sizeof(float), s>>>(
      nH, cinv, t, ld, N, y);
  MK_COUNT(), k_tl_prolong<<<gb, 256, 0, s>>>(L.n_nodes, m->d_P_off, m->d_P_col, m->d_P_val32, y, dinv,
                                              L.d_boundary, r, z, ld, N, 1);
  MK_TRY(apply32(z, q));
  if (!defer_final)
    MK_COUNT(), k_tl_resid<<<gb, 256, 0, s>>>(L.n_nodes, L.d_boundary, dinv, r, q, z, ld, N, w, 1);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

static int twolevel_apply(mk_ctx* ctx, const mk_mesh* m, const float* cinv, const float* dinv, const float* r,
                          float* z, int ld, int N, bool add, cudaStream_t s) {
  const Level& L = m->fine;
  const int nH = (int)m->coarse.n_free;
  int err = MK_OK;
  float* t = (float*)scratch(ctx, S_TLT, (size_t)(kTLS + 1) * nH * ld * sizeof(float), &err);
  if (!t) return err;
  float* y = t + (size_t)kTLS * nH * ld;
  MK_COUNT(), k_tl_restrict<<<nH * kTLS / kTLW, kTLW * 32, 0, s>>>(m->d_PT_off, m->d_PT_col, m->d_PT_val32, r,
                                                                   nullptr, ld, N, t);
  MK_COUNT(), k_tl_coarse<<<(nH + kTLRows - 1) / kTLRows, kTLRows * 32, (size_t)nH * kTLC * sizeof(float), s>>>(
      nH, cinv, t, ld, N, y);
  MK_COUNT(), k_tl_prolong<<<(int)((L.n_nodes * N + 255) / 256), 256, 0, s>>>(
      L.n_nodes, m->d_P_off, m->d_P_col, m->d_P_val32, y, dinv, L.d_boundary, r, z, ld, N, add ? 1 : 0);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

// ------------------------------------------------------------------------------------------------ mixed PCG
struct MixState {
  double rz, pq, rr, rr0, alpha, beta, rr64, bn;
  int active, iters, breakdown, outer_active;
};

// Column partial sums with a fixed map: thread t of a block of ld*(256/ld) threads always handles column t % ld.
// part[blk][k*ld + j] for k < NS sums.
template <int NS>
__device__ __forceinline__ void block_partials(double (&acc)[NS], double* sh, int ld, double* part, int bx) {
  const int rows = blockDim.x / ld;
  const int r = threadIdx.x / ld;
  int top = 1;
  while (top < rows) top <<= 1;
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    sh[threadIdx.x] = acc[k];
    __syncthreads();
    for (int st = top >> 1; st > 0; st >>= 1) {  // fixed pairwise tree over the rows of each column
      if (r < st && r + st < rows) sh[threadIdx.x] += sh[threadIdx.x + st * ld];
      __syncthreads();
    }
    if (threadIdx.x < ld) part[(int64_t)bx * NS * ld + k * ld + threadIdx.x] = sh[threadIdx.x];
    __syncthreads();
  }
}

// Finalisers: one block of ld threads, sums partials in block order.
// mode 0: outer residual (bb, rr64) -> bn, rr64, outer_active
// mode 1: inner init (rz, rr) -> rz, rr0, rr, active (outer_active), iters=0
// mode 2: alpha from pq
// mode 3: beta from (rz_new, rr) and convergence of the inner solve
// FCG(1) (flexible CG, the learned preconditioner): mode 4: alpha = (p.r)/(p.q); mode 5: rr and convergence;
// mode 6: beta = -(z.q)/(p.q); mode 7: inner init from r.r
// Launched with kFinThreads threads: one warp per (sum, column) pair adds the block partials lane-strided and
// folds them with a fixed shuffle tree (deterministic), then one thread per column updates its state.
constexpr int kFinThreads = 1024;
__device__ __forceinline__ void finalize_body(int mode, const double* __restrict__ part, int nblk, int NS, int ld,
                                              int N, MixState* __restrict__ st, double rtol, double inner_rtol2) {
  __shared__ double sums[2 * 256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int pr = warp; pr < NS * ld; pr += nw) {
    const int k = pr / ld, jj = pr - k * ld;
    const double* pp = part + k * ld + jj;
    const int64_t bs = (int64_t)NS * ld;
    double v = 0.0;
    int b = lane;
    for (; b + 96 < nblk; b += 128) {  // four independent loads in flight, added in the same order as one by one
      const double x0 = __ldcg(pp + b * bs), x1 = __ldcg(pp + (b + 32) * bs), x2 = __ldcg(pp + (b + 64) * bs),
                   x3 = __ldcg(pp + (b + 96) * bs);
      v += x0;
      v += x1;
      v += x2;
      v += x3;
    }
    for (; b < nblk; b += 32) v += __ldcg(pp + b * bs);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) sums[k * ld + jj] = v;
  }
  __syncthreads();
  const int j = threadIdx.x;
  if (j >= ld) return;
  double s[2] = {sums[j], NS > 1 ? sums[ld + j] : 0.0};
  MixState c = st[j];
  if (mode == 0) {
    c.bn = s[0] > 0 ? sqrt(s[0]) : 1.0;
    c.rr64 = s[1];
    c.outer_active = (j < N) && (sqrt(s[1]) / c.bn > rtol);
  } else if (mode == 1) {
    c.rz = s[0];
    c.rr0 = s[1];
    c.rr = s[1];
    c.active = c.outer_active && s[1] > 0.0;
    c.alpha = 0.0;
    c.beta = 0.0;
  } else if (mode == 2) {
    c.pq = s[0];
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
  } else if (mode == 3) {
    if (c.active) {
      c.beta = s[0] / c.rz;
      c.rz = s[0];
      c.rr = s[1];
      c.iters += 1;
      c.active = c.rr > inner_rtol2 * c.rr0;
    } else {
      c.beta = 0.0;
    }
  } else if (mode == 4) {
    c.pq = s[0];
    if (c.active) {
      if (!(c.pq > 0.0)) {
        c.breakdown = 1;
        c.active = 0;
        c.alpha = 0.0;
      } else {
        c.alpha = s[1] / c.pq;
      }
    } else {
      c.alpha = 0.0;
    }
  } else if (mode == 5) {
    if (c.active) {
      c.rr = s[0];
      c.iters += 1;
      c.active = c.rr > inner_rtol2 * c.rr0;
    }
  } else if (mode == 6) {
    c.beta = c.active ? -s[0] / c.pq : 0.0;
  } else {
    c.rr0 = s[0];
    c.rr = s[0];
    c.active = c.outer_active && s[0] > 0.0;
    c.alpha = 0.0;
    c.beta = 0.0;
  }
  st[j] = c;
}
__global__ void __launch_bounds__(kFinThreads) k_mixed_finalize(int mode, const double* __restrict__ part, int nblk,
                                                               int NS, int ld, int N, MixState* __restrict__ st,
                                                               double rtol, double inner_rtol2) {
  finalize_body(mode, part, nblk, NS, ld, N, st, rtol, inner_rtol2);
}


// Finalisation fused into the kernel that produced the partials: each block publishes its partials, then the last
// block of the grid to arrive (an atomic counter) folds them in block order exactly as k_mixed_finalize would and
// resets the counter for the next launch.  ctr == nullptr: no finalisation here (a separate launch does it).
struct FinArgs {
  int* ctr;
  int mode, NS, N;
  MixState* st;
  double rtol, inner2;
};
__device__ __forceinline__ void finalize_if_last(const FinArgs& f, const double* __restrict__ part, int ld) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(f.ctr, 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x == 0) *f.ctr = 0;
  finalize_body(f.mode, part, (int)gridDim.x, f.NS, ld, f.N, f.st, f.rtol, f.inner2);
}

// r64 = b - Ax (interior rows), r32 = (float) r64, d32 = 0; partials of (b.b, r64.r64)
__global__ void k_mixed_residual(int64_t n, const uint8_t* __restrict__ bnd, const double* __restrict__ b,
                                 const double* __restrict__ Ax, float* __restrict__ r32, float* __restrict__ d32,
                                 int N, int ld, double* __restrict__ part, FinArgs fin) {
  __shared__ double sh[256];
  double acc[2] = {0.0, 0.0};
  const int rows = blockDim.x / ld;
  const int j = threadIdx.x % ld, r = threadIdx.x / ld;
  if (r < rows)
    for (int64_t nd = (int64_t)blockIdx.x * rows + r; nd < n; nd += (int64_t)gridDim.x * rows) {
      const int64_t t = nd * ld + j;
      double rv = 0.0, bv = 0.0;
      if (j < N && !bnd[nd]) {
        bv = b[t];
        rv = bv - Ax[t];
      }
      r32[t] = (float)rv;
      d32[t] = 0.f;
      acc[0] += bv * bv;
      acc[1] += rv * rv;
    }
  block_partials<2>(acc, sh, ld, part, blockIdx.x);
  if (fin.ctr) finalize_if_last(fin, part, ld);
}

// The FP32 vector kernels below visit the nodes of a thread in chunks of kChunk grid-stride steps: the chunk's
// loads are independent (issued together), its products are summed in FP32 in a fixed order, and each chunk sum
// is added to the thread's FP64 accumulator.  That keeps the FP64 units (about 2 operations per clock per SM) off
// the per-element path; the partials and their tree stay FP64 and the result stays independent of scheduling.
constexpr int kChunk = 4;

// p = Dinv r; partials of (r.z, r.r)
__global__ void k_mixed_init(int64_t n, const float* __restrict__ dinv, const float* __restrict__ r,
                             float* __restrict__ p, int ld, double* __restrict__ part, FinArgs fin) {
  __shared__ double sh[256];
  double acc[2] = {0.0, 0.0};
  const int rows = blockDim.x / ld;
  const int j = threadIdx.x % ld, rr = threadIdx.x / ld;
  const int64_t stride = (int64_t)gridDim.x * rows;
  if (rr < rows)
    for (int64_t nd0 = (int64_t)blockIdx.x * rows + rr; nd0 < n; nd0 += kChunk * stride) {
      float rv[kChunk], dv[kChunk];
#pragma unroll
      for (int u = 0; u < kChunk; ++u) {
        const int64_t nd = nd0 + u * stride;
        rv[u] = nd < n ? r[nd * ld + j] : 0.f;
        dv[u] = nd < n ? dinv[nd] : 0.f;
      }
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int u = 0; u < kChunk; ++u) {
        const int64_t nd = nd0 + u * stride;
        const float z = rv[u] * dv[u];
        if (nd < n) p[nd * ld + j] = z;
        s0 = fmaf(rv[u], z, s0);
        s1 = fmaf(rv[u], rv[u], s1);
      }
      acc[0] += (double)s0;
      acc[1] += (double)s1;
    }
  block_partials<2>(acc, sh, ld, part, blockIdx.x);
  if (fin.ctr) finalize_if_last(fin, part, ld);
}

// partial p.q (block bx of gx)
__device__ __forceinline__ void mixed_pq_body(int bx, int gx, int64_t n, const float* __restrict__ p,
                                              const float* __restrict__ q, int ld, double* __restrict__ part) {
  __shared__ double sh[256];
  double acc[1] = {0.0};
  const int rows = blockDim.x / ld;
  const int j = threadIdx.x % ld, rr = threadIdx.x / ld;
  const int64_t stride = (int64_t)gx * rows;
  if (rr < rows)
    for (int64_t nd0 = (int64_t)bx * rows + rr; nd0 < n; nd0 += kChunk * stride) {
      float pv[kChunk], qv[kChunk];
#pragma unroll
      for (int u = 0; u < kChunk; ++u) {
        const int64_t nd = nd0 + u * stride;
        pv[u] = nd < n ? p[nd * ld + j] : 0.f;
        qv[u] = nd < n ? q[nd * ld + j] : 0.f;
      }
      float s0 = 0.f;
#pragma unroll
      for (int u = 0; u < kChunk; ++u) s0 = fmaf(pv[u], qv[u], s0);
      acc[0] += (double)s0;
    }
  block_partials<1>(acc, sh, ld, part, bx);
}
__global__ void k_mixed_pq(int64_t n, const float* __restrict__ p, const float* __restrict__ q, int ld,
                           double* __restrict__ part, FinArgs fin) {
  mixed_pq_body(blockIdx.x, gridDim.x, n, p, q, ld, part);
  if (fin.ctr) finalize_if_last(fin, part, ld);
}

// d += alpha p; r -= alpha q; partials of (r.z, r.r) with z = Dinv r (block bx of gx)
__device__ __forceinline__ void mixed_update_body(int bx, int gx, int64_t n, const MixState* __restrict__ st,
                                                  const float* __restrict__ dinv, const float* __restrict__ p,
                                                  const float* __restrict__ q, float* __restrict__ d,
                                                  float* __restrict__ r, int ld, double* __restrict__ part) {
  __shared__ double sh[256];
  double acc[2] = {0.0, 0.0};
  const int rows = blockDim.x / ld;
  const int j = threadIdx.x % ld, rr = threadIdx.x / ld;
  const float a = rr < rows ? (float)st[j].alpha : 0.f;
  const int64_t stride = (int64_t)gx * rows;
  if (rr < rows)
    for (int64_t nd0 = (int64_t)bx * rows + rr; nd0 < n; nd0 += kChunk * stride) {
      float rv[kChunk], dv[kChunk];
#pragma unroll
      for (int u = 0; u < kChunk; ++u) {
        const int64_t nd = nd0 + u * stride;
        rv[u] = nd < n ? r[nd * ld + j] : 0.f;
        dv[u] = nd < n ? dinv[nd] : 0.f;
      }
      if (a != 0.f) {
        float pv[kChunk], qv[kChunk], dd[kChunk];
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
          const int64_t nd = nd0 + u * stride;
          pv[u] = nd < n ? p[nd * ld + j] : 0.f;
          qv[u] = nd < n ? q[nd * ld + j] : 0.f;
          dd[u] = nd < n ? d[nd * ld + j] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
          const int64_t nd = nd0 + u * stride;
          rv[u] -= a * qv[u];
          if (nd < n) {
            d[nd * ld + j] = dd[u] + a * pv[u];
            r[nd * ld + j] = rv[u];
          }
        }
      }
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int u = 0; u < kChunk; ++u) {
        s0 = fmaf(rv[u], rv[u] * dv[u], s0);
        s1 = fmaf(rv[u], rv[u], s1);
      }
      acc[0] += (double)s0;
      acc[1] += (double)s1;
    }
  block_partials<2>(acc, sh, ld, part, bx);
}
__global__ void k_mixed_update(int64_t n, const MixState* __restrict__ st, const float* __restrict__ dinv,
                               const float* __restrict__ p, const float* __restrict__ q, float* __restrict__ d,
                               float* __restrict__ r, int ld, double* __restrict__ part, FinArgs fin) {
  mixed_update_body(blockIdx.x, gridDim.x, n, st, dinv, p, q, d, r, ld, part);
  if (fin.ctr) finalize_if_last(fin, part, ld);
}

// p = Dinv r + beta p (active columns); item t = node * ld + column
__device__ __forceinline__ void mixed_p_body(int64_t t, int64_t n, const MixState* __restrict__ st,
                                             const float* __restrict__ dinv, const float* __restrict__ r,
                                             float* __restrict__ p, int ld) {
  if (t >= n * ld) return;
  const int j = (int)(t % ld);
  if (!st[j].active) return;
  const int64_t nd = t / ld;
  p[t] = r[t] * dinv[nd] + (float)st[j].beta * p[t];
}
__global__ void k_mixed_p(int64_t n, const MixState* __restrict__ st, const float* __restrict__ dinv,
                          const float* __restrict__ r, float* __restrict__ p, int ld) {
  mixed_p_body((int64_t)blockIdx.x * blockDim.x + threadIdx.x, n, st, dinv, r, p, ld);
}

// FCG(1): partials of (p.q, p.r)
__global__ void k_fcg_pq(int64_t n, const float* __restrict__ p, const float* __restrict__ q,
                         const float* __restrict__ r, int ld, double* __restrict__ part, FinArgs fin) {
  __shared__ double sh[256];
  double acc[2] = {0.0, 0.0};
  const int rows = blockDim.x / ld;
  const int j = threadIdx.x % ld, rr = threadIdx.x / ld;
  const int64_t stride = (int64_t)gridDim.x * rows;
  if (rr < rows)
    for (int64_t nd0 = (int64_t)blockIdx.x * rows + rr; nd0 < n; nd0 += kChunk * stride) {
      float pv[kChunk], qv[kChunk], rv[kChunk];
#pragma unroll
      for (int u = 0; u < kChunk; ++u) {
        const int64_t nd = nd0 + u * stride;
        pv[u] = nd < n ? p[nd * ld + j] : 0.f;
        qv[u] = nd < n ? q[nd * ld + j] : 0.f;
        rv[u] = nd < n ? r[nd * ld + j] : 0.f;
      }
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int u = 0; u < kChunk; ++u) {
        s0 = fmaf(pv[u], qv[u], s0);
        s1 = fmaf(pv[u], rv[u], s1);
      }
      acc[0] += (double)s0;
      acc[1] += (double)s1;
    }
  block_partials<2>(acc, sh, ld, part, blockIdx.x);
  if (fin.ctr) finalize_if_last(fin, part, ld);
}

// FCG(1): d += alpha p; r -= alpha q; partial r.r.  With z0 given, also the first sweep of the multiplicative
// two-level preconditioner on the new residual: z0 = w D^-1 r (columns < N, boundary rows 0).
__global__ void k_fcg_update(int64_t n, const MixState* __restrict__ st, const float* __restrict__ p,
                             const float* __restrict__ q, float* __restrict__ d, float* __restrict__ r, int ld,
                             double* __restrict__ part, FinArgs fin, float* __restrict__ z0,
                             const float* __restrict__ dinv, const uint8_t* __restrict__ bnd, int N, float w) {
  __shared__ double sh[256];
  double acc[1] = {0.0};
  const int rows = blockDim.x / ld;
  const int j = threadIdx.x % ld, rr = threadIdx.x / ld;
  const float a = rr < rows ? (float)st[j].alpha : 0.f;
  const int64_t stride = (int64_t)gridDim.x * rows;
  if (rr < rows)
    for (int64_t nd0 = (int64_t)blockIdx.x * rows + rr; nd0 < n; nd0 += kChunk * stride) {
      float rv[kChunk];
#pragma unroll
      for (int u = 0; u < kChunk; ++u) {
        const int64_t nd = nd0 + u * stride;
        rv[u] = nd < n ? r[nd * ld + j] : 0.f;
      }
      if (a != 0.f) {
        float pv[kChunk], qv[kChunk], dd[kChunk];
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
          const int64_t nd = nd0 + u * stride;
          pv[u] = nd < n ? p[nd * ld + j] : 0.f;
          qv[u] = nd < n ? q[nd * ld + j] : 0.f;
          dd[u] = nd < n ? d[nd * ld + j] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
          const int64_t nd = nd0 + u * stride;
          rv[u] -= a * qv[u];
          if (nd < n) {
            d[nd * ld + j] = dd[u] + a * pv[u];
            r[nd * ld + j] = rv[u];
          }
        }
      }
      if (z0 && j < N) {
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
          const int64_t nd = nd0 + u * stride;
          if (nd < n) z0[nd * ld + j] = bnd[nd] ? 0.f : w * dinv[nd] * rv[u];
        }
      }
      float s0 = 0.f;
#pragma unroll
      for (int u = 0; u < kChunk; ++u) s0 = fmaf(rv[u], rv[u], s0);
      acc[0] += (double)s0;
    }
  block_partials<1>(acc, sh, ld, part, blockIdx.x);
  if (fin.ctr) finalize_if_last(fin, part, ld);
}

// FCG(1): p = z + beta p (active columns)
__global__ void k_fcg_p(int64_t n, const MixState* __restrict__ st, const float* __restrict__ z,
                        float* __restrict__ p, int ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ld) return;
  const int j = (int)(t % ld);
  if (!st[j].active) return;
  p[t] = z[t] + (float)st[j].beta * p[t];
}

// The last sweep of the multiplicative two-level preconditioner, z += w D^-1 (r - t) (columns < N, boundary
// rows 0; t = A z from inside the preconditioner), fused with the FCG(1) partial z.q of the next beta.
__global__ void k_tl_final_pq(int64_t n, const uint8_t* __restrict__ bnd, const float* __restrict__ dinv,
                              const float* __restrict__ r, const float* __restrict__ t, float* __restrict__ z,
                              const float* __restrict__ q, int ld, int N, float w, double* __restrict__ part,
                              FinArgs fin) {
  __shared__ double sh[256];
  double acc[1] = {0.0};
  const int rows = blockDim.x / ld;
  const int j = threadIdx.x % ld, rr = threadIdx.x / ld;
  const int64_t stride = (int64_t)gridDim.x * rows;
  if (rr < rows)
    for (int64_t nd0 = (int64_t)blockIdx.x * rows + rr; nd0 < n; nd0 += kChunk * stride) {
      float zv[kChunk], qv[kChunk];
#pragma unroll
      for (int u = 0; u < kChunk; ++u) {
        const int64_t nd = nd0 + u * stride;
        zv[u] = nd < n ? z[nd * ld + j] : 0.f;
        qv[u] = nd < n ? q[nd * ld + j] : 0.f;
      }
      if (j < N) {
#pragma unroll
        for (int u = 0; u < kChunk; ++u) {
          const int64_t nd = nd0 + u * stride;
          if (nd < n) {
            const int64_t i = nd * ld + j;
            zv[u] = bnd[nd] ? 0.f : fmaf(w * dinv[nd], r[i] - t[i], zv[u]);
            z[i] = zv[u];
          }
        }
      }
      float s0 = 0.f;
#pragma unroll
      for (int u = 0; u < kChunk; ++u) s0 = fmaf(zv[u], qv[u], s0);
      acc[0] += (double)s0;
    }
  block_partials<1>(acc, sh, ld, part, blockIdx.x);
  if (fin.ctr) finalize_if_last(fin, part, ld);
}

__global__ void k_mixed_add(int64_t n, const float* __restrict__ d, double* __restrict__ x, int N, int ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ld) return;
  if ((int)(t % ld) < N) x[t] += (double)d[t];
}

__global__ void k_dinv32(int64_t n, const double* __restrict__ diag, float* __restrict__ dinv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dinv[i] = (float)(1.0 / diag[i]);
}

int diag_inverse32(int64_t n, const double* diag, float* dinv, cudaStream_t s) {
  MK_COUNT(), k_dinv32<<<(int)((n + 255) / 256), 256, 0, s>>>(n, diag, dinv);
  MK_CUDA(cudaGetLastError());
  return MK_OK;
}

__global__ void k_zero_boundary(int64_t n, const uint8_t* __restrict__ bnd, double* __restrict__ x, int ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n * ld && bnd[t / ld]) x[t] = 0.0;
}

int pcg_mixed(mk_ctx* ctx, const mk_mesh* m, const double* A64, const double* b, double* x, int ld, int N,
              const mk_solve_opts& o, mk_solve_report* rep, cudaStream_t s, const float* cinv, bool stiff,
              const double* diag_pre);

// vq: an optional potential at the quadrature points added to the operator (K/2 + M_Vext + M_vq + sigma M)
int solve_mixed(mk_ctx* ctx, const mk_mesh* m, const mk_molecule* mol, double sigma, const double* b,
                const double* vq, const double*, double* x, int ld, int N, const mk_solve_opts& o,
                mk_solve_report* rep, cudaStream_t s) {
  if (o.precond != MK_PRECOND_JACOBI && o.precond != MK_PRECOND_LEARNED)
    return fail(MK_ERR_UNSUPPORTED, "mixed path: Jacobi or learned preconditioner");
  if (o.precond == MK_PRECOND_LEARNED && !o.mlp) return fail(MK_ERR_INVALID_ARG, "learned preconditioner: no network");
  const Level& L = m->fine;
  const int np = L.nloc * (L.nloc + 1) / 2;
  int err = MK_OK;
  double* A64 = (double*)scratch(ctx, S_ELEM64, (size_t)L.n_elems * np * sizeof(double), &err);
  if (!A64) return err;
  const double* H0 = static_matrices(ctx, m, mol, s, &err);
  if (!H0) return err;
  MK_TRY(element_matrices(ctx, L, nullptr, 0.0, 0.0, sigma, vq, A64, s, H0));
  const float* cinv = nullptr;
  if (o.coarse) {  // two-level: the coarse inverse of this molecule's shifted operator (cached)
    if (vq) return fail(MK_ERR_UNSUPPORTED, "two-level preconditioner: not with a potential in the operator");
    std::vector<double> key;
    key.push_back(sigma);
    for (int k = 0; k < mol->n_nuclei; ++k) {
      key.push_back(mol->Z[k]);
      for (int c = 0; c < 3; ++c) key.push_back(mol->R[3 * k + c]);
    }
    MK_TRY(tl_prepare(m, s));
    cinv = coarse_inverse_cached(ctx, m, A64, &key, s, &err);
    if (!cinv) return err;
  }
  return pcg_mixed(ctx, m, A64, b, x, ld, N, o, rep, s, cinv, false, nullptr);
}

// FP32 inner Jacobi-PCG on the patch operator built from the FP64 element matrices A64 (element order), FP64
// residual b - A x and iterative refinement of x until every column meets o.rtol.  stiff: A64 is the stiffness
// matrix K itself, and the inner FP32 applications use the matrix-free stiffness operator.  diag_pre: the
// operator's diagonal if already known (else assembled here).
static int pcg_mixed_on(mk_ctx* ctx, const mk_mesh* m, const double* A64, const double* b, double* x, int ld, int N,
                        const mk_solve_opts& o, mk_solve_report* rep, cudaStream_t s, const float* cinv, bool stiff,
                        const double* diag_pre);

// Runs the solve on the context's own stream (CUDA graphs cannot be captured on the legacy default stream), after
// everything already queued on the caller's stream and before anything queued there afterwards.
int pcg_mixed(mk_ctx* ctx, const mk_mesh* m, const double* A64, const double* b, double* x, int ld, int N,
              const mk_solve_opts& o, mk_solve_report* rep, cudaStream_t caller, const float* cinv, bool stiff,
              const double* diag_pre) {
  MK_CUDA(cudaEventRecord(ctx->solve_ev[0], caller));
  MK_CUDA(cudaStreamWaitEvent(ctx->solve_stream, ctx->solve_ev[0], 0));
  const int r = pcg_mixed_on(ctx, m, A64, b, x, ld, N, o, rep, ctx->solve_stream, cinv, stiff, diag_pre);
  MK_CUDA(cudaEventRecord(ctx->solve_ev[1], ctx->solve_stream));
  MK_CUDA(cudaStreamWaitEvent(caller, ctx->solve_ev[1], 0));
  return r;
}

static int pcg_mixed_on(mk_ctx* ctx, const mk_mesh* m, const double* A64, const double* b, double* x, int ld, int N,
                        const mk_solve_opts& o, mk_solve_report* rep, cudaStream_t s, const float* cinv, bool stiff,
                        const double* diag_pre) {
  MK_ARG(ld <= 256, "mixed path: ld must be <= 256");
  const Level& L = m->fine;
  const int64_t n = L.n_nodes;
  int err = MK_OK;
  float* A32 = (float*)scratch(ctx, S_ELEM32, (size_t)L.n_elems * padded_np(L.nloc, 4) * sizeof(float), &err);
  double* diag = (double*)scratch(ctx, S_DIAG64, n * sizeof(double), &err);
  float* dinv = (float*)scratch(ctx, S_DIAG32, n * sizeof(float), &err);
  double* Ax = (double*)scratch(ctx, S_Q64, (size_t)n * ld * sizeof(double), &err);
  float* r = (float*)scratch(ctx, S_R32, (size_t)n * ld * sizeof(float), &err);
  float* p = (float*)scratch(ctx, S_P32, (size_t)n * ld * sizeof(float), &err);
  float* q = (float*)scratch(ctx, S_Q32, (size_t)n * ld * sizeof(float), &err);
  float* d = (float*)scratch(ctx, S_X32, (size_t)n * ld * sizeof(float), &err);
  const bool learned = o.precond == MK_PRECOND_LEARNED && o.mlp;
  // the multigrid V-cycle (Poisson operator on a mesh with a hierarchy) instead of the two-level form
  const bool mg = stiff && o.coarse == 2 && m->has_mg && cinv != nullptr;
  // an explicit preconditioned residual z (FCG(1), which is PCG for a fixed SPD preconditioner) whenever the
  // preconditioner is more than the diagonal: learned, two-level, multigrid
  const bool fcg = learned || cinv != nullptr;
  float* zb = fcg ? (float*)scratch(ctx, S_Z32, (size_t)n * ld * sizeof(float), &err) : nullptr;
  if (fcg && !zb) return err;
  const int nblk = red_blocks(ctx);
  double* part = (double*)scratch(ctx, S_RED, (size_t)nblk * 2 * ld * sizeof(double), &err);
  MixState* st = (MixState*)scratch(ctx, S_SCAL, 256 * sizeof(MixState), &err);
  if (!A32 || !diag || !dinv || !Ax || !r || !p || !q || !d || !part || !st) return err;
  if (ctx->pinned_size < 256 * sizeof(MixState)) {
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    MK_CUDA(cudaMallocHost(&ctx->pinned, 256 * sizeof(MixState)));
    ctx->pinned_size = 256 * sizeof(MixState);
  }
  MixState* hst = (MixState*)ctx->pinned;
  if (diag_pre) MK_CUDA(cudaMemcpyAsync(diag, diag_pre, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else MK_TRY(assemble_diagonal(ctx, L, A64, diag, s));
  if (!stiff) MK_TRY(pack_elements<float>(ctx, m, A64, A32, s));
  // the element matrices for every refinement residual of this solve, packed once in patch order: as FP32 pairs
  // (the products on the FP32 units, MK_OPT_PAIR_RESIDUAL) or in FP64
  const bool pairs = ctx->pair_residual;
  double* A64p = nullptr;
  float* Aph = nullptr;
  const size_t npa = (size_t)L.n_elems * padded_np(L.nloc, 4);
  if (pairs) {
    if (!(Aph = (float*)scratch(ctx, S_PAIRA, 2 * npa * sizeof(float), &err))) return err;
    MK_TRY(pack_pairs(ctx, m, A64, Aph, Aph + npa, s));
  } else {
    A64p = (double*)scratch(ctx, S_ELEMP64, (size_t)L.n_elems * padded_np(L.nloc, 8) * sizeof(double), &err);
    if (!A64p) return err;
    MK_TRY(pack_elements<double>(ctx, m, A64, A64p, s));
  }
  // the inner FP32 operator: the packed element matrices, or the matrix-free stiffness operator
  auto apply32 = [&](const float* xin, float* yout) -> int {
    return stiff ? apply_stiff(ctx, m, xin, yout, ld, true, s) : apply_patch<float>(ctx, m, A32, xin, yout, ld, true, s);
  };
  MK_COUNT(), k_dinv32<<<(int)((n + 255) / 256), 256, 0, s>>>(n, diag, dinv);
  // the smoother weight of the Poisson preconditioners, estimated once per mesh and per multigrid level
  float wsm = kTLOmega;
  if (stiff && cinv) {
    if (m->poisson_omega == 0.f)
      MK_TRY(smoother_omega(ctx, n, [&](const float* xi, float* yo) { return apply_stiff(ctx, m, xi, yo, 1, true, s); },
                            dinv, L.d_boundary, s, &m->poisson_omega));
    wsm = m->poisson_omega;
    if (mg)
      for (const MgLevel& g : m->mg)
        if (g.omega == 0.f) {
          const int64_t nl = g.L.n_nodes;
          auto spmv = [&](const float* xi, float* yo) -> int {
            MK_COUNT(), k_mg_spmv<<<(int)((nl * 32 + 255) / 256), 256, 0, s>>>(nl, g.K.d_off, g.K.d_col, g.K.d_val,
                                                                               xi, yo);
            MK_CUDA(cudaGetLastError());
            return MK_OK;
          };
          MK_TRY(smoother_omega(ctx, nl, spmv, g.d_dinv, nullptr, s, &g.omega));
        }
  }
  MK_COUNT(), k_zero_boundary<<<(int)((n * ld + 255) / 256), 256, 0, s>>>(n, L.d_boundary, x, ld);
  MK_CUDA(cudaMemsetAsync(st, 0, 256 * sizeof(MixState), s));
  const int th = ld * (256 / ld);
  const int gb = (int)((n * ld + 255) / 256);
  const int check = std::max(1, o.check_every);
  const double inner2 = o.inner_rtol * o.inner_rtol;
  // the finalisation of each reduction runs in the last block of the kernel that produced the partials
  int* fin_ctr = (int*)scratch(ctx, S_FINCTR, 64, &err);
  if (!fin_ctr) return err;
  MK_CUDA(cudaMemsetAsync(fin_ctr, 0, sizeof(int), s));
  auto fin = [&](int mode, int NS) { return FinArgs{fin_ctr, mode, NS, N, st, o.rtol, inner2}; };
  int total_it = 0, refine = 0, status = MK_OK;
  bool converged = false;
  const int max_refine = o.max_refine > 0 ? o.max_refine : 20;
  cudaGraphExec_t exec = nullptr;
  long long graph_kernels = 0;
  const bool use_graph = !ctx->no_graphs;
  // the operator's halo buffer must exist before a capture starts (nothing may allocate inside a capture)
  if (!scratch(ctx, S_HALO, (size_t)std::max<int64_t>(m->patches.n_halo_slots, 1) * ld * sizeof(float), &err))
    return err;
  if (cinv && !scratch(ctx, S_TLT, (size_t)(kTLS + 1) * m->coarse.n_free * ld * sizeof(float), &err)) return err;
  float* tlq = nullptr;  // A z inside the multiplicative two-level preconditioner
  if (cinv && !learned && !mg && !(tlq = (float*)scratch(ctx, S_TLQ, (size_t)n * ld * sizeof(float), &err))) return err;
  if (mg) {  // the V-cycle's scratch must exist before a capture starts
    size_t total = (size_t)n;
    for (const MgLevel& g : m->mg) total += 3 * (size_t)g.L.n_nodes;
    total += 2 * (size_t)m->coarse.n_free;
    if (!scratch(ctx, S_MG, total * sizeof(float), &err)) return err;
  }
  if (stiff && !stiff_factors(m, s, &err)) return err;  // allocated here: nothing may allocate inside a capture
  if (fcg) {
    if (!scratch(ctx, S_LHALO, (size_t)std::max<int64_t>(m->patches.n_halo_slots, 1) * ld * sizeof(float), &err))
      return err;
    MK_CUDA(cudaMemsetAsync(zb, 0, (size_t)n * ld * sizeof(float), s));  // columns >= N stay zero
  }
  for (;;) {
    if (pairs) MK_TRY(apply_pair(ctx, m, Aph, Aph + npa, x, Ax, ld, true, s));  // residual of the current x
    else MK_TRY(apply_patch<double>(ctx, m, A64p, x, Ax, ld, true, s));
    MK_COUNT(), k_mixed_residual<<<nblk, th, 0, s>>>(n, L.d_boundary, b, Ax, r, d, N, ld, part, fin(0, 2));
    MK_CUDA(cudaMemcpyAsync(hst, st, sizeof(MixState) * ld, cudaMemcpyDeviceToHost, s));
    MK_CUDA(cudaStreamSynchronize(s));
    bool any = false;
    for (int j = 0; j < N; ++j) any |= hst[j].outer_active != 0;
    if (!any) { converged = true; break; }
    if (refine >= max_refine || total_it >= o.maxit) break;
    ++refine;
    auto precond = [&]() -> int {  // zb = M(r)
      if (mg) return mg_apply(ctx, m, apply32, dinv, cinv, r, zb, s, wsm);
      if (learned) {
        MK_TRY(learned_apply(ctx, m, o.mlp, dinv, r, zb, ld, N, o.mlp_precision, s));
        if (cinv) MK_TRY(twolevel_apply(ctx, m, cinv, dinv, r, zb, ld, N, true, s));
        return MK_OK;
      }
      return twolevel_mult_apply(ctx, m, apply32, cinv, dinv, r, zb, ld, N, s, wsm);
    };
    if (fcg) {
      MK_TRY(precond());
      MK_CUDA(cudaMemcpyAsync(p, zb, (size_t)n * ld * sizeof(float), cudaMemcpyDeviceToDevice, s));
      MK_COUNT(), k_mixed_pq<<<nblk, th, 0, s>>>(n, r, r, ld, part, fin(7, 1));
    } else {
      MK_COUNT(), k_mixed_init<<<nblk, th, 0, s>>>(n, dinv, r, p, ld, part, fin(1, 2));
    }
    int it = 0;
    bool inner_active = true;
    // one PCG (or FCG(1)) iteration; every scalar it needs lives on the device, so `check` of them can be
    // replayed as a graph
    auto iteration = [&]() -> int {
      MK_TRY(apply32(p, q));
      if (fcg) {
        MK_COUNT(), k_fcg_pq<<<nblk, th, 0, s>>>(n, p, q, r, ld, part, fin(4, 2));
        if (tlq) {
          // multiplicative two-level: the first sweep rides on the update, the last on the z.q reduction
          MK_COUNT(), k_fcg_update<<<nblk, th, 0, s>>>(n, st, p, q, d, r, ld, part, fin(5, 1), zb, dinv,
                                                       L.d_boundary, N, wsm);
          MK_TRY(twolevel_mult_apply(ctx, m, apply32, cinv, dinv, r, zb, ld, N, s, wsm, true, true));
          MK_COUNT(), k_tl_final_pq<<<nblk, th, 0, s>>>(n, L.d_boundary, dinv, r, tlq, zb, q, ld, N, wsm, part,
                                                        fin(6, 1));
        } else {
          MK_COUNT(), k_fcg_update<<<nblk, th, 0, s>>>(n, st, p, q, d, r, ld, part, fin(5, 1), nullptr, nullptr,
                                                       nullptr, N, 0.f);
          MK_TRY(precond());
          MK_COUNT(), k_mixed_pq<<<nblk, th, 0, s>>>(n, zb, q, ld, part, fin(6, 1));
        }
        MK_COUNT(), k_fcg_p<<<gb, 256, 0, s>>>(n, st, zb, p, ld);
        return MK_OK;
      }
      MK_COUNT(), k_mixed_pq<<<nblk, th, 0, s>>>(n, p, q, ld, part, fin(2, 1));
      MK_COUNT(), k_mixed_update<<<nblk, th, 0, s>>>(n, st, dinv, p, q, d, r, ld, part, fin(3, 2));
      MK_COUNT(), k_mixed_p<<<gb, 256, 0, s>>>(n, st, dinv, r, p, ld);
      return MK_OK;
    };
    while (inner_active && total_it < o.maxit) {
      const int k = std::min(check, o.maxit - total_it);
      bool replayed = false;  // this chunk ran as a graph replay (its timed applications are harvested below)
      if (use_graph && k == check) {
        if (!exec) {
          const long long c0 = g_launch_count.load();
          prof_prepare_capture(ctx);
          MK_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
          prof_capture(ctx, true);
          int rc = MK_OK;
          for (int c = 0; c < check && rc == MK_OK; ++c) rc = iteration();
          prof_capture(ctx, false);
          cudaGraph_t graph = nullptr;
          const cudaError_t ce = cudaStreamEndCapture(s, &graph);
          if (rc != MK_OK) return rc;
          if (ce != cudaSuccess) return fail(MK_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
          MK_CUDA(cudaGraphInstantiate(&exec, graph, 0));
          cudaGraphDestroy(graph);
          graph_kernels = g_launch_count.load() - c0;
          g_launch_count.fetch_sub(graph_kernels);   // counted when replayed, below
        }
        MK_CUDA(cudaGraphLaunch(exec, s));
        g_launch_count.fetch_add(graph_kernels);
        replayed = true;
      } else {
        for (int c = 0; c < k; ++c) MK_TRY(iteration());
      }
      it += k;
      total_it += k;
      MK_CUDA(cudaMemcpyAsync(hst, st, sizeof(MixState) * ld, cudaMemcpyDeviceToHost, s));
      MK_CUDA(cudaStreamSynchronize(s));
      if (replayed) prof_harvest(ctx);
      inner_active = false;
      for (int j = 0; j < N; ++j) {
        inner_active |= hst[j].active != 0;
        if (hst[j].breakdown) status = MK_ERR_BREAKDOWN;
      }
      if (status == MK_ERR_BREAKDOWN) break;
    }
    MK_COUNT(), k_mixed_add<<<gb, 256, 0, s>>>(n, d, x, N, ld);
    if (status == MK_ERR_BREAKDOWN) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  MK_CUDA(cudaGetLastError());
  MK_CUDA(cudaMemcpyAsync(hst, st, sizeof(MixState) * ld, cudaMemcpyDeviceToHost, s));
  MK_CUDA(cudaStreamSynchronize(s));
  MK_TRY(check_fault(ctx, s));
  double mx = 0.0;
  for (int j = 0; j < N; ++j) mx = std::max(mx, std::sqrt(hst[j].rr64) / hst[j].bn);
  if (rep) {
    std::memset(rep, 0, sizeof(*rep));
    rep->n_rhs = N;
    rep->iterations = total_it;
    rep->refinements = refine;
    rep->max_rel_residual = mx;
    for (int j = 0; j < N; ++j) {
      rep->iters[j] = hst[j].iters;
      rep->rel_residual[j] = std::sqrt(hst[j].rr64) / hst[j].bn;
    }
  }
  if (status == MK_OK && !converged) status = MK_ERR_NOT_CONVERGED;
  if (rep) rep->status = status;
  if (status == MK_ERR_BREAKDOWN) return fail(status, "mixed PCG breakdown: p^T A p <= 0 (operator not SPD)");
  if (status == MK_ERR_NOT_CONVERGED) return fail(status, "mixed PCG did not reach rtol");
  return MK_OK;
}

}  // namespace mk

using namespace mk;

extern "C" int mk_operator_apply(mk_ctx* ctx, const mk_mesh* m, const mk_molecule* mol, double sigma, int precision,
                                 const void* x, void* y, int ld, void* stream) {
  MK_ARG(ctx && m && x && y && ld >= 1 && ld <= 256, "mk_operator_apply: bad argument");
  MK_ARG(mol || sigma == 0.0, "mk_operator_apply: the stiffness operator (no molecule) takes sigma = 0");
  MK_ARG(precision == MK_PREC_FP64 || precision == MK_PREC_MIXED || precision == MK_PREC_PAIRS,
         "mk_operator_apply: bad precision");
  MK_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const Level& L = m->fine;
  const int np = L.nloc * (L.nloc + 1) / 2;
  int err = MK_OK;
  if (!mol && precision == MK_PREC_MIXED)  // the Hartree Poisson operator K, matrix-free in FP32
    return apply_stiff(ctx, m, (const float*)x, (float*)y, ld, true, s);
  double* A64 = (double*)scratch(ctx, S_OPA, (size_t)L.n_elems * np * sizeof(double), &err);
  if (!A64) return err;
  if (mol) {
    const double* H0 = static_matrices(ctx, m, mol, s, &err);
    if (!H0) return err;
    MK_TRY(element_matrices(ctx, L, nullptr, 0.0, 0.0, sigma, nullptr, A64, s, H0));
  } else {
    MK_TRY(element_matrices(ctx, L, nullptr, 1.0, 0.0, 0.0, nullptr, A64, s));  // K
  }
  if (precision == MK_PREC_FP64) {
    double* A = (double*)scratch(ctx, S_OPB, (size_t)L.n_elems * padded_np(L.nloc, 8) * sizeof(double), &err);
    if (!A) return err;
    MK_TRY(pack_elements<double>(ctx, m, A64, A, s));
    return apply_patch<double>(ctx, m, A, (const double*)x, (double*)y, ld, true, s);
  }
  if (precision == MK_PREC_PAIRS) {
    const size_t na = (size_t)L.n_elems * padded_np(L.nloc, 4);
    float* Ah = (float*)scratch(ctx, S_OPB, 2 * na * sizeof(float), &err);
    if (!Ah) return err;
    MK_TRY(pack_pairs(ctx, m, A64, Ah, Ah + na, s));
    return apply_pair(ctx, m, Ah, Ah + na, (const double*)x, (double*)y, ld, true, s);
  }
  float* A = (float*)scratch(ctx, S_OPB, (size_t)L.n_elems * padded_np(L.nloc, 4) * sizeof(float), &err);
  if (!A) return err;
  MK_TRY(pack_elements<float>(ctx, m, A64, A, s));
  return apply_patch<float>(ctx, m, A, (const float*)x, (float*)y, ld, true, s);
}

// ------------------------------------------------------------------------------------------------ batched solve
// Many correction problems (different meshes, molecules, orbital counts) share every launch of the inner FP32
// PCG iteration.  A device table describes each problem; the operator grid spans the patches of all meshes (block
// -> problem through blk_prob), the other kernels take the problem from blockIdx.y or from item offsets.  Every
// kernel body is the single-problem one, so each problem's arithmetic is exactly that of its own solve.
namespace mk {

constexpr int kBatchCols = 32;  // columns a batched problem may have (its per-column scalars)

struct BatchProb {
  // patch operator
  const int32_t *elem_off, *node_off, *conn, *target, *inc_off, *shared_node, *shared_off;
  const uint16_t* inc;
  const uint8_t* bnd;
  const float* A32;
  float* halo;
  int64_t n_shared, n, n_elems;
  int pe, max_nodes, first_block, ld, N;
  const unsigned char* rec;  // patch records (the register-staged operator)
  int rec_stride;
  // PCG state
  const float* dinv;
  float *r, *p, *q, *d;
  MixState* st;
  double* part;
};

// whether any column of problem P is still iterating (the same value for every thread of a CTA)
__device__ __forceinline__ bool batch_active(const BatchProb& P) {
  bool any = false;
  for (int j = 0; j < P.N; ++j) any = any || P.st[j].active != 0;
  return any;
}

__device__ __forceinline__ int batch_find(const int64_t* __restrict__ off, int K, int64_t t) {
  int lo = 0, hi = K;  // largest k with off[k] <= t
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

template <int NLOC>
__global__ void __launch_bounds__(256) k_bapply(const BatchProb* __restrict__ probs, const int32_t* __restrict__ blk_prob) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int b = blk_prob[blockIdx.x];
  const BatchProb& P = probs[b];
  if (!batch_active(P)) return;  // a problem whose columns all converged: its q is not read again
  patch_apply<NLOC, float, 4>((int)blockIdx.x - P.first_block, P.elem_off, P.node_off, P.conn, P.A32, P.target,
                              P.inc_off, P.inc, P.bnd, 1, P.p, P.q, P.halo, P.ld / 4, 0, P.ld, P.pe, P.max_nodes, smraw);
}

// the register-staged operator body (the single solve's default operator) over the patches of all problems
template <int NLOC>
__global__ void __launch_bounds__(kRegMaxThreads, 2) k_bapply_reg(const BatchProb* __restrict__ probs,
                                                                  const int32_t* __restrict__ blk_prob,
                                                                  int* __restrict__ fault) {
  extern __shared__ __align__(16) unsigned char smraw_breg[];
  const int b = blk_prob[blockIdx.x];
  const BatchProb& P = probs[b];
  if (!batch_active(P)) return;  // a problem whose columns all converged: its q is not read again
  patch_apply_reg<NLOC, 32>((int)blockIdx.x - P.first_block, P.rec, P.rec_stride, P.A32, 1, P.p, P.q, P.halo, 0,
                            P.ld, P.ld, P.pe, P.max_nodes, P.n, P.n_elems, fault, smraw_breg);
}

__global__ void k_bhalo(const BatchProb* __restrict__ probs, int K, const int64_t* __restrict__ off) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= off[K]) return;
  const int b = batch_find(off, K, t);
  const BatchProb& P = probs[b];
  halo_sum<float, 4>(t - off[b], P.n_shared, P.shared_node, P.shared_off, P.bnd, 1, P.halo, P.q, P.ld / 4, 0, P.ld);
}

__global__ void k_bpq(const BatchProb* __restrict__ probs) {
  const BatchProb& P = probs[blockIdx.y];
  mixed_pq_body(blockIdx.x, gridDim.x, P.n, P.p, P.q, P.ld, P.part);
}

__global__ void k_bupdate(const BatchProb* __restrict__ probs) {
  const BatchProb& P = probs[blockIdx.y];
  mixed_update_body(blockIdx.x, gridDim.x, P.n, P.st, P.dinv, P.p, P.q, P.d, P.r, P.ld, P.part);
}

__global__ void k_bp(const BatchProb* __restrict__ probs, int K, const int64_t* __restrict__ off) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= off[K]) return;
  const int b = batch_find(off, K, t);
  const BatchProb& P = probs[b];
  mixed_p_body(t - off[b], P.n, P.st, P.dinv, P.r, P.p, P.ld);
}

__global__ void __launch_bounds__(kFinThreads) k_bfinalize(int mode, const BatchProb* __restrict__ probs, int nblk,
                                                          int NS, double rtol, double inner_rtol2) {
  const BatchProb& P = probs[blockIdx.x];
  finalize_body(mode, P.part, nblk, NS, P.ld, P.N, P.st, rtol, inner_rtol2);
}

}  // namespace mk

extern "C" int mk_batch_correction_solve(mk_ctx* ctx, int K, const mk_mesh* const* meshes, const mk_molecule* mols,
                                         const double* sigmas, const double* const* rhs, double* const* x,
                                         const int* ld, const int* N, const mk_solve_opts* opts,
                                         mk_solve_report* reports, void* stream) {
  MK_ARG(ctx && meshes && mols && sigmas && rhs && x && ld && N && opts && reports,
         "mk_batch_correction_solve: null argument");
  MK_ARG(K >= 1 && K <= MK_MAX_BATCH, "mk_batch_correction_solve: bad K");
  MK_ARG(opts->precision == MK_PREC_MIXED && opts->precond == MK_PRECOND_JACOBI && !opts->coarse &&
             opts->rtol > 0 && opts->maxit > 0,
         "mk_batch_correction_solve: mixed precision with Jacobi only");
  MK_ARG(meshes[0], "mk_batch_correction_solve: null mesh");
  const int nloc = meshes[0]->fine.nloc;
  for (int k = 0; k < K; ++k) {
    MK_ARG(meshes[k] && rhs[k] && x[k], "mk_batch_correction_solve: null problem");
    MK_ARG(meshes[k]->fine.nloc == nloc, "mk_batch_correction_solve: all meshes must use one element order");
    MK_ARG(ld[k] == 4 || ld[k] == 8 || ld[k] == 16 || ld[k] == 32,
           "mk_batch_correction_solve: ld must be 4, 8, 16 or 32");
    MK_ARG(N[k] >= 1 && N[k] <= ld[k], "mk_batch_correction_solve: bad N");
  }
  MK_CUDA(cudaSetDevice(ctx->device));
  const mk_solve_opts& o = *opts;
  cudaStream_t caller = (cudaStream_t)stream;
  MK_CUDA(cudaEventRecord(ctx->solve_ev[0], caller));
  MK_CUDA(cudaStreamWaitEvent(ctx->solve_stream, ctx->solve_ev[0], 0));
  cudaStream_t s = ctx->solve_stream;
  const int nblk = red_blocks(ctx);
  const int np = nloc * (nloc + 1) / 2, nps = padded_np(nloc, 4);
  // one scratch region: per-problem buffers, then the device tables
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o2 = off; off += (bytes + 255) / 256 * 256; return o2; };
  std::vector<size_t> oA64(K), oA32(K), oDiag(K), oDinv(K), oAx(K), oR(K), oP(K), oQ(K), oD(K), oH(K), oPart(K);
  int64_t nblocks = 0, hitems = 0, pitems = 0;
  size_t smem = 0, smem_reg = 0;
  int th_reg = 32;
  bool reg_ok = true, wide = false;
  for (int k = 0; k < K; ++k) {
    const Level& L = meshes[k]->fine;
    const Patches& P = meshes[k]->patches;
    const size_t n = (size_t)L.n_nodes, v32 = n * ld[k] * sizeof(float);
    oA64[k] = take((size_t)L.n_elems * np * 8);
    oA32[k] = take((size_t)L.n_elems * nps * 4);
    oDiag[k] = take(n * 8);
    oDinv[k] = take(n * 4);
    oAx[k] = take(n * ld[k] * 8);
    oR[k] = take(v32);
    oP[k] = take(v32);
    oQ[k] = take(v32);
    oD[k] = take(v32);
    oH[k] = take((size_t)std::max<int64_t>(P.n_halo_slots, 1) * ld[k] * 4);
    oPart[k] = take((size_t)nblk * 2 * ld[k] * 8);
    nblocks += P.n_patches;
    hitems += P.n_shared_nodes * (ld[k] / 4);
    pitems += (int64_t)n * ld[k];
    smem = std::max(smem, patch_smem(nloc, P.max_elems, P.max_nodes, std::min(ld[k], 16), 4).total);
    smem_reg = std::max(smem_reg, reg_smem(nloc, P.max_elems, P.max_nodes, P.max_rec_bytes, 32).total);
    th_reg = std::max(th_reg, (P.max_elems + 31) / 32 * 32);
    reg_ok = reg_ok && P.d_rec != nullptr && P.max_elems <= kRegMaxThreads;
    wide = wide || ld[k] > 16;
  }
  // the register-staged operator (one element per thread) when every mesh has patch records and it fits; the
  // one-patch-per-CTA operator otherwise, at most 16 columns
  const bool use_reg = reg_ok && ctx->patch_kernel == 1 && smem_reg <= 227 * 1024;
  MK_ARG(use_reg || !wide, "mk_batch_correction_solve: ld = 32 needs the register-staged operator");
  if (use_reg) smem = smem_reg;
  MK_ARG(smem <= 227 * 1024, "mk_batch_correction_solve: patch too large for shared memory");
  const size_t oSt = take((size_t)K * kBatchCols * sizeof(MixState)), oProbs = take((size_t)K * sizeof(BatchProb));
  const size_t oBlk = take((size_t)nblocks * 4), oHoff = take((size_t)(K + 1) * 8), oPoff = take((size_t)(K + 1) * 8);
  int err = MK_OK;
  char* ws = (char*)scratch(ctx, S_BATCH, off, &err);
  if (!ws) return err;
  if (ctx->pinned_size < (size_t)K * kBatchCols * sizeof(MixState)) {
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    ctx->pinned = nullptr;
    ctx->pinned_size = 0;
    MK_CUDA(cudaMallocHost(&ctx->pinned, (size_t)K * kBatchCols * sizeof(MixState)));
    ctx->pinned_size = (size_t)K * kBatchCols * sizeof(MixState);
  }
  MixState* hst = (MixState*)ctx->pinned;
  MixState* dst = (MixState*)(ws + oSt);
  std::vector<BatchProb> hp(K);
  std::vector<int32_t> blk(nblocks);
  std::vector<int64_t> hoff(K + 1, 0), poff(K + 1, 0);
  int64_t b0 = 0;
  for (int k = 0; k < K; ++k) {
    const mk_mesh* m = meshes[k];
    const Level& L = m->fine;
    const Patches& P = m->patches;
    BatchProb& B = hp[k];
    B.elem_off = P.d_patch_elem_off;
    B.node_off = P.d_patch_node_off;
    B.conn = P.d_conn;
    B.target = P.d_node_target;
    B.inc_off = P.d_inc_off;
    B.shared_node = P.d_shared_node;
    B.shared_off = P.d_shared_off;
    B.inc = P.d_inc;
    B.bnd = L.d_boundary;
    B.A32 = (const float*)(ws + oA32[k]);
    B.halo = (float*)(ws + oH[k]);
    B.n_shared = P.n_shared_nodes;
    B.n = L.n_nodes;
    B.pe = P.max_elems;
    B.max_nodes = P.max_nodes;
    B.n_elems = L.n_elems;
    B.rec = P.d_rec;
    B.rec_stride = P.max_rec_bytes;
    B.first_block = (int)b0;
    B.ld = ld[k];
    B.N = N[k];
    B.dinv = (const float*)(ws + oDinv[k]);
    B.r = (float*)(ws + oR[k]);
    B.p = (float*)(ws + oP[k]);
    B.q = (float*)(ws + oQ[k]);
    B.d = (float*)(ws + oD[k]);
    B.st = dst + (size_t)k * kBatchCols;
    B.part = (double*)(ws + oPart[k]);
    for (int i = 0; i < P.n_patches; ++i) blk[b0 + i] = k;
    b0 += P.n_patches;
    hoff[k + 1] = hoff[k] + P.n_shared_nodes * (ld[k] / 4);
    poff[k + 1] = poff[k] + L.n_nodes * ld[k];
  }
  BatchProb* dprobs = (BatchProb*)(ws + oProbs);
  int32_t* dblk = (int32_t*)(ws + oBlk);
  int64_t* dhoff = (int64_t*)(ws + oHoff);
  int64_t* dpoff = (int64_t*)(ws + oPoff);
  MK_CUDA(cudaMemcpyAsync(dprobs, hp.data(), (size_t)K * sizeof(BatchProb), cudaMemcpyHostToDevice, s));
  MK_CUDA(cudaMemcpyAsync(dblk, blk.data(), (size_t)nblocks * 4, cudaMemcpyHostToDevice, s));
  MK_CUDA(cudaMemcpyAsync(dhoff, hoff.data(), (size_t)(K + 1) * 8, cudaMemcpyHostToDevice, s));
  MK_CUDA(cudaMemcpyAsync(dpoff, poff.data(), (size_t)(K + 1) * 8, cudaMemcpyHostToDevice, s));
  MK_CUDA(cudaMemsetAsync(dst, 0, (size_t)K * kBatchCols * sizeof(MixState), s));
  MK_CUDA(cudaStreamSynchronize(s));  // the host tables above may go out of scope only after the copies
  // per problem: operator K/2 + M_Vext + sigma M (FP64 element matrices, FP32 patch copy), Jacobi diagonal
  for (int k = 0; k < K; ++k) {
    const mk_mesh* m = meshes[k];
    const Level& L = m->fine;
    double* A64 = (double*)(ws + oA64[k]);
    const double* H0 = static_matrices(ctx, m, &mols[k], s, &err);
    if (!H0) return err;
    MK_TRY(element_matrices(ctx, L, nullptr, 0.0, 0.0, sigmas[k], nullptr, A64, s, H0));
    MK_TRY(assemble_diagonal(ctx, L, A64, (double*)(ws + oDiag[k]), s));
    MK_TRY(pack_elements<float>(ctx, m, A64, (float*)(ws + oA32[k]), s));
    MK_COUNT(), k_dinv32<<<(int)((L.n_nodes + 255) / 256), 256, 0, s>>>(L.n_nodes, (const double*)(ws + oDiag[k]),
                                                                         (float*)(ws + oDinv[k]));
    MK_COUNT(), k_zero_boundary<<<(int)((L.n_nodes * ld[k] + 255) / 256), 256, 0, s>>>(L.n_nodes, L.d_boundary, x[k],
                                                                                         ld[k]);
  }
  if (use_reg) {
    if (nloc == 4) MK_CUDA(cudaFuncSetAttribute(k_bapply_reg<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    else MK_CUDA(cudaFuncSetAttribute(k_bapply_reg<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  } else {
    if (nloc == 4) MK_CUDA(cudaFuncSetAttribute(k_bapply<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    else MK_CUDA(cudaFuncSetAttribute(k_bapply<10>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  const int check = std::max(1, o.check_every);
  const double inner2 = o.inner_rtol * o.inner_rtol;
  const int max_refine = o.max_refine > 0 ? o.max_refine : 20;
  auto iteration = [&]() -> int {  // one inner PCG iteration of every problem
    if (use_reg) {
      if (nloc == 4) MK_COUNT(), k_bapply_reg<4><<<(int)nblocks, th_reg, smem, s>>>(dprobs, dblk, ctx->d_fault);
      else MK_COUNT(), k_bapply_reg<10><<<(int)nblocks, th_reg, smem, s>>>(dprobs, dblk, ctx->d_fault);
    } else {
      if (nloc == 4) MK_COUNT(), k_bapply<4><<<(int)nblocks, 256, smem, s>>>(dprobs, dblk);
      else MK_COUNT(), k_bapply<10><<<(int)nblocks, 256, smem, s>>>(dprobs, dblk);
    }
    if (hitems > 0) MK_COUNT(), k_bhalo<<<(int)((hitems + 255) / 256), 256, 0, s>>>(dprobs, K, dhoff);
    MK_COUNT(), k_bpq<<<dim3(nblk, K), 256, 0, s>>>(dprobs);
    MK_COUNT(), k_bfinalize<<<K, kFinThreads, 0, s>>>(2, dprobs, nblk, 1, o.rtol, inner2);
    MK_COUNT(), k_bupdate<<<dim3(nblk, K), 256, 0, s>>>(dprobs);
    MK_COUNT(), k_bfinalize<<<K, kFinThreads, 0, s>>>(3, dprobs, nblk, 2, o.rtol, inner2);
    MK_COUNT(), k_bp<<<(int)((pitems + 255) / 256), 256, 0, s>>>(dprobs, K, dpoff);
    return MK_OK;
  };
  std::vector<int> refines(K, 0);
  std::vector<char> conv(K, 0);
  int total_it = 0, status = MK_OK;
  cudaGraphExec_t exec = nullptr;
  long long graph_kernels = 0;
  for (int refine = 0;; ++refine) {
    for (int k = 0; k < K; ++k) {  // FP64 residual of every problem (on FP32 pairs, as the single solves)
      const BatchProb& B = hp[k];
      if (ctx->pair_residual)
        MK_TRY(apply64_pairs(ctx, meshes[k], (const double*)(ws + oA64[k]), x[k], (double*)(ws + oAx[k]), ld[k], true,
                             s));
      else
        MK_TRY(apply64(ctx, meshes[k], (const double*)(ws + oA64[k]), x[k], (double*)(ws + oAx[k]), ld[k], ld[k],
                       true, s));
      MK_COUNT(), k_mixed_residual<<<nblk, 256, 0, s>>>(B.n, B.bnd, rhs[k], (const double*)(ws + oAx[k]), B.r, B.d,
                                                         N[k], ld[k], B.part, FinArgs{});
      MK_COUNT(), k_mixed_finalize<<<1, kFinThreads, 0, s>>>(0, B.part, nblk, 2, ld[k], N[k], B.st, o.rtol, inner2);
    }
    MK_CUDA(cudaMemcpyAsync(hst, dst, (size_t)K * kBatchCols * sizeof(MixState), cudaMemcpyDeviceToHost, s));
    MK_CUDA(cudaStreamSynchronize(s));
    bool any = false;
    for (int k = 0; k < K; ++k) {
      bool a = false;
      for (int j = 0; j < N[k]; ++j) a |= hst[k * kBatchCols + j].outer_active != 0;
      conv[k] = !a;
      any |= a;
    }
    if (!any || refine >= max_refine || total_it >= o.maxit) break;
    for (int k = 0; k < K; ++k) {
      const BatchProb& B = hp[k];
      if (!conv[k]) refines[k] += 1;
      MK_COUNT(), k_mixed_init<<<nblk, 256, 0, s>>>(B.n, B.dinv, B.r, B.p, ld[k], B.part, FinArgs{});
      MK_COUNT(), k_mixed_finalize<<<1, kFinThreads, 0, s>>>(1, B.part, nblk, 2, ld[k], N[k], B.st, o.rtol, inner2);
    }
    bool inner_active = true;
    while (inner_active && total_it < o.maxit) {
      const int kk = std::min(check, o.maxit - total_it);
      if (!ctx->no_graphs && kk == check) {
        if (!exec) {  // one graph of `check` iterations of the whole batch, replayed for the rest of the solve
          const long long c0 = g_launch_count.load();
          MK_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
          int rc = MK_OK;
          for (int c = 0; c < check && rc == MK_OK; ++c) rc = iteration();
          cudaGraph_t graph = nullptr;
          const cudaError_t ce = cudaStreamEndCapture(s, &graph);
          if (rc != MK_OK) return rc;
          if (ce != cudaSuccess) return fail(MK_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(ce));
          MK_CUDA(cudaGraphInstantiate(&exec, graph, 0));
          cudaGraphDestroy(graph);
          graph_kernels = g_launch_count.load() - c0;
          g_launch_count.fetch_sub(graph_kernels);
        }
        MK_CUDA(cudaGraphLaunch(exec, s));
        g_launch_count.fetch_add(graph_kernels);
      } else {
        for (int c = 0; c < kk; ++c) MK_TRY(iteration());
      }
      total_it += kk;
      MK_CUDA(cudaMemcpyAsync(hst, dst, (size_t)K * kBatchCols * sizeof(MixState), cudaMemcpyDeviceToHost, s));
      MK_CUDA(cudaStreamSynchronize(s));
      inner_active = false;
      for (int k = 0; k < K; ++k)
        for (int j = 0; j < N[k]; ++j) {
          inner_active |= hst[k * kBatchCols + j].active != 0;
          if (hst[k * kBatchCols + j].breakdown) status = MK_ERR_BREAKDOWN;
        }
      if (status == MK_ERR_BREAKDOWN) break;
    }
    for (int k = 0; k < K; ++k) {
      const BatchProb& B = hp[k];
      MK_COUNT(), k_mixed_add<<<(int)((B.n * ld[k] + 255) / 256), 256, 0, s>>>(B.n, B.d, x[k], N[k], ld[k]);
    }
    if (status == MK_ERR_BREAKDOWN) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  MK_CUDA(cudaGetLastError());
  // reports from the last FP64 residual (taken at the top of the final pass of the refinement loop)
  int worst = status;
  for (int k = 0; k < K; ++k) {
    mk_solve_report& R = reports[k];
    std::memset(&R, 0, sizeof(R));
    R.n_rhs = N[k];
    R.refinements = refines[k];
    double mx = 0.0;
    int its = 0;
    for (int j = 0; j < N[k]; ++j) {
      const MixState& c = hst[k * kBatchCols + j];
      R.iters[j] = c.iters;
      R.rel_residual[j] = std::sqrt(c.rr64) / c.bn;
      mx = std::max(mx, R.rel_residual[j]);
      its = std::max(its, c.iters);
      if (c.breakdown) R.status = MK_ERR_BREAKDOWN;
    }
    R.iterations = its;
    R.max_rel_residual = mx;
    if (R.status == MK_OK && !conv[k]) R.status = MK_ERR_NOT_CONVERGED;
    if (R.status != MK_OK && worst == MK_OK) worst = R.status;
  }
  MK_CUDA(cudaEventRecord(ctx->solve_ev[1], s));
  MK_CUDA(cudaStreamWaitEvent(caller, ctx->solve_ev[1], 0));
  MK_TRY(check_fault(ctx, s));
  if (worst == MK_ERR_BREAKDOWN) return fail(worst, "batched PCG breakdown: p^T A p <= 0 in some problem");
  if (worst == MK_ERR_NOT_CONVERGED) return fail(worst, "batched PCG: some problem did not reach rtol");
  return MK_OK;
}

extern "C" int mk_mesh_set_patch_elems(mk_mesh* m, int pe) {
  MK_ARG(m, "mk_mesh_set_patch_elems: null mesh");
  MK_ARG(pe >= 32 && pe <= 512 && pe % 32 == 0, "mk_mesh_set_patch_elems: pe must be a multiple of 32 in [32, 512]");
  MK_CUDA(cudaSetDevice(m->device));
  MK_CUDA(cudaDeviceSynchronize());  // no kernel may still read the old patches
  free_patches(m->patches);
  return build_patches(m, pe);
}

extern "C" int mk_autotune_patches(mk_ctx* ctx, mk_mesh* m, int ld, int* best_pe, double* ms_out) {
  MK_ARG(ctx && m && best_pe, "mk_autotune_patches: null argument");
  MK_ARG(ld >= 1 && ld <= 256, "mk_autotune_patches: bad ld");
  MK_CUDA(cudaSetDevice(ctx->device));
  const Level& L = m->fine;
  const int cand2[4] = {64, 96, 128, 192}, cand1[4] = {128, 192, 256, 384};
  const int* cand = L.nloc == 10 ? cand2 : cand1;
  const int np = L.nloc * (L.nloc + 1) / 2;
  int err = MK_OK;
  double* A64 = (double*)scratch(ctx, S_OPA, (size_t)L.n_elems * np * sizeof(double), &err);
  float* A = (float*)scratch(ctx, S_OPB, (size_t)L.n_elems * padded_np(L.nloc, 4) * sizeof(float), &err);
  float* xy = (float*)scratch(ctx, S_VEC4, (size_t)L.n_nodes * ld * 2 * sizeof(float), &err);
  if (!A64 || !A || !xy) return err;
  cudaStream_t s = ctx->solve_stream;
  MK_TRY(element_matrices(ctx, L, nullptr, 0.5, 0.0, 1.0, nullptr, A64, s));  // K/2 + M: timing stand-in
  MK_CUDA(cudaMemsetAsync(xy, 0, (size_t)L.n_nodes * ld * 2 * sizeof(float), s));
  cudaEvent_t e0, e1;
  MK_CUDA(cudaEventCreate(&e0));
  MK_CUDA(cudaEventCreate(&e1));
  double best = 1e300;
  int bpe = cand[0];
  for (int c = 0; c < 4; ++c) {
    int r = mk_mesh_set_patch_elems(m, cand[c]);
    if (r == MK_OK) r = pack_elements<float>(ctx, m, A64, A, s);
    for (int w = 0; w < 3 && r == MK_OK; ++w) r = apply_patch<float>(ctx, m, A, xy, xy + L.n_nodes * ld, ld, true, s);
    double ms = 1e300;
    if (r == MK_OK) {
      cudaEventRecord(e0, s);
      for (int it = 0; it < 10 && r == MK_OK; ++it)
        r = apply_patch<float>(ctx, m, A, xy, xy + L.n_nodes * ld, ld, true, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      ms = t / 10.0;
    } else {
      cudaGetLastError();  // a candidate whose shared memory does not fit is skipped
    }
    if (ms_out) ms_out[c] = r == MK_OK ? ms : -1.0;
    if (r == MK_OK && ms < best) {
      best = ms;
      bpe = cand[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *best_pe = bpe;
  return mk_mesh_set_patch_elems(m, bpe);
}
