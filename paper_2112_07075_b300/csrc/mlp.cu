// Per-element MLP of the learned form: 586 -> 128 -> 128 -> 192, GELU (erf form)
// after both hidden layers, BF16 weights and activations on the tensor cores
// (tcgen05 MMA fed by TMA, FP32 accumulation in tensor memory), FP32 master
// weights, Adam.
// Used to predict the mass-CG initial guess (see learned.cu); this file holds
// the network itself: parameter init, forward, backward, optimiser step.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda.h>

#include "lh_device.cuh"
#include "lh_internal.h"
#include "lh_mlp.h"
#include "tc_sm100.cuh"

namespace lh {
namespace mlp {
namespace {

// ---------------------------------------------------------------------------
// BF16 GEMM on the 5th-generation tensor cores: C[m][n] = sum_k A(m,k) B(k,n)
// (+ bias[n]), FP32 accumulation in tensor memory. A is K-major (A[m*lda+k]) or
// MN-major (A[k*lda+m]); B is K-major (B[n*ldb+k], a row-major weight used as
// B = W^T) or MN-major (B[k*ldb+n]). A CTA owns a 128 x BN tile: one thread
// issues TMA tile loads (cp.async.bulk.tensor, 128-byte swizzle, zero fill past
// the extents) into a 4-stage ring, one thread issues tcgen05.mma (K = 16 per
// instruction) and releases stages by tcgen05.commit; the four warps then read
// the accumulator rows back with tcgen05.ld for the epilogue. With splits > 1
// the K range is cut into `splits` slices (grid z) whose FP32 partial tiles are
// summed afterwards in a fixed order (k_split_sum): deterministic.
// Epilogue: C32 (FP32) and/or C16 (BF16) with optional bias and GELU; when PRE
// is given the pre-activation is written there (FP32).
// ---------------------------------------------------------------------------
constexpr int kStages = 2;
constexpr int kBK = 64;   // K per stage: one 128-byte swizzle row of BF16
constexpr long long kSpin = 2000000000LL;   // bounded waits (~1 s)

enum { A_ROW = 0, A_COL = 1 };
enum { B_NMAJOR = 0, B_ROW = 1 };

struct GemmArgs {
  const __nv_bfloat16 *A, *B;
  int M, N, K, lda, ldb;
  const float *bias;
  float *C32;
  __nv_bfloat16 *C16;
  float *pre;
  int ldc, gelu, accumulate;
  int splits;       // K slices (grid z); > 1 writes partial tiles
  float *partial;   // [splits][M][N] FP32 when splits > 1
  int *status;      // LH_ERR_TIMEOUT latched here if a bounded wait gives up
};

template <int BN>
struct GemmCfg {
  static constexpr int A_BYTES = 128 * kBK * 2;
  static constexpr int B_BYTES = BN * kBK * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int SMEM = 1024 + kStages * STAGE;
  static constexpr int TCOLS = BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

// Sixteen consecutive outputs of one row: two 16-byte stores (BF16) or four
// (FP32) where the address allows, else element by element (the same values).
__device__ __forceinline__ void st16_f32(float *p, const float (&v)[16]) {
  if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
#pragma unroll
    for (int l = 0; l < 16; l += 4) *reinterpret_cast<float4 *>(p + l) = make_float4(v[l], v[l + 1], v[l + 2], v[l + 3]);
  } else {
#pragma unroll
    for (int l = 0; l < 16; ++l) p[l] = v[l];
  }
}
__device__ __forceinline__ void st16_bf16(__nv_bfloat16 *p, const float (&v)[16]) {
  if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
    uint32_t w[8];
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * l], v[2 * l + 1]);
      w[l] = *reinterpret_cast<const uint32_t *>(&h);
    }
    reinterpret_cast<uint4 *>(p)[0] = make_uint4(w[0], w[1], w[2], w[3]);
    reinterpret_cast<uint4 *>(p)[1] = make_uint4(w[4], w[5], w[6], w[7]);
  } else {
#pragma unroll
    for (int l = 0; l < 16; ++l) p[l] = __float2bfloat16(v[l]);
  }
}
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// TMA: 2D tile (x = inner coordinate, y = outer) into shared memory, counted on bar.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(tc::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(tc::smem_u32(bar))
      : "memory");
}

// Instruction descriptor of kind::f16, BF16 inputs, FP32 accumulator, with the
// A and B major-ness bits (15: A MN-major, 16: B MN-major).
__host__ __device__ constexpr uint32_t idesc_ab(int M, int N, bool a_mn, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int AL, int BL, int BN>
__global__ void __launch_bounds__(128, 1) k_gemm(const __grid_constant__ CUtensorMap tmA,
                                                 const __grid_constant__ CUtensorMap tmB, GemmArgs g) {
  using C = GemmCfg<BN>;
  extern __shared__ unsigned char gemm_smem_raw[];
  char *base = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(gemm_smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full[kStages], empty[kStages], done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int m0 = blockIdx.y * 128, n0 = blockIdx.x * BN;
  const int kblocks = (g.K + kBK - 1) / kBK;
  const int per = (kblocks + g.splits - 1) / g.splits;
  const int kb0 = blockIdx.z * per;
  const int nkb = max(0, min(kblocks, kb0 + per) - kb0);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(&done, 1);
    tc::fence_mbar_init();
    s_fail = 0;
  }
  if (threadIdx.x < 32) {
    tc::tmem_alloc(&s_tmem, C::TCOLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  constexpr uint32_t IDESC = idesc_ab(128, BN, AL == A_COL, BL == B_ROW);
  if (threadIdx.x == 0) {   // producer: TMA tile loads into the ring
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kStages, u = i / kStages;
      if (u > 0 && !tc::mbar_wait(&empty[s], (u - 1) & 1, kSpin)) { s_fail = 1; break; }
      char *sa = base + s * C::STAGE, *sb = sa + C::A_BYTES;
      tc::mbar_arrive_expect_tx(&full[s], C::STAGE);
      const int k0 = (kb0 + i) * kBK;
      if (AL == A_ROW) {
        tma_load_2d(sa, &tmA, k0, m0, &full[s]);
      } else {
        tma_load_2d(sa, &tmA, m0, k0, &full[s]);
        tma_load_2d(sa + 8192, &tmA, m0 + 64, k0, &full[s]);
      }
      if (BL == B_NMAJOR) {
        tma_load_2d(sb, &tmB, k0, n0, &full[s]);
      } else {
#pragma unroll
        for (int j = 0; j < BN / 64; ++j) tma_load_2d(sb + j * 8192, &tmB, n0 + 64 * j, k0, &full[s]);
      }
    }
  } else if (threadIdx.x == 32) {   // MMA issuer
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kStages, u = i / kStages;
      if (!tc::mbar_wait(&full[s], u & 1, kSpin)) { s_fail = 1; break; }
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(base + s * C::STAGE), b0 = a0 + C::A_BYTES;
#pragma unroll
      for (int ks = 0; ks < kBK / 16; ++ks) {
        // K-major: the 16-wide K step moves 32 bytes along the swizzled row;
        // MN-major: it moves two 8-row atoms (2 KB); 64-wide MN blocks are 8 KB apart
        const uint64_t ad = AL == A_ROW ? tc::sdesc(a0 + ks * 32, 16, 1024) : tc::sdesc(a0 + ks * 2048, 8192, 1024);
        const uint64_t bd = BL == B_NMAJOR ? tc::sdesc(b0 + ks * 32, 16, 1024) : tc::sdesc(b0 + ks * 2048, 8192, 1024);
        tc::mma_bf16(tmem, ad, bd, IDESC, (i > 0 || ks > 0) ? 1u : 0u);
      }
      tc::mma_commit(&empty[s]);
    }
    tc::mma_commit(&done);
  }
  __syncwarp();
  const bool ok = nkb == 0 || tc::mbar_wait(&done, 0, kSpin);
  const int all_ok = __syncthreads_and(ok ? 1 : 0) && !s_fail;
  if (!all_ok && threadIdx.x == 0 && g.status) atomicExch(g.status, 6);
  tc::fence_after_sync();
  if (all_ok) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = m0 + warp * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      if (nkb > 0) {
        tc::tmem_ld16(tl + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int l = 0; l < 16; ++l) v[l] = 0.0f;
      }
      const int n = n0 + c0;   // N is a multiple of 16: a chunk is all in or all out
      if (m >= g.M || n >= g.N) continue;
      if (g.splits > 1) {
        float *dst = g.partial + ((size_t)blockIdx.z * g.M + m) * g.N + n;
#pragma unroll
        for (int l = 0; l < 16; l += 4) *reinterpret_cast<float4 *>(dst + l) = make_float4(v[l], v[l + 1], v[l + 2], v[l + 3]);
        continue;
      }
      const size_t idx = (size_t)m * g.ldc + n;
      // each thread owns a row: its 16 outputs are contiguous, so they go out as
      // whole 16-byte stores (one thread per row makes the element-wise form 16
      // scattered stores per chunk and output)
      float z[16], o[16];
#pragma unroll
      for (int l = 0; l < 16; ++l) {
        z[l] = g.bias ? v[l] + g.bias[n + l] : v[l];
        o[l] = g.gelu ? gelu_f(z[l]) : z[l];
      }
      if (g.pre) st16_f32(g.pre + idx, z);
      if (g.C32) {
        if (g.accumulate) {
#pragma unroll
          for (int l = 0; l < 16; ++l) o[l] = g.C32[idx + l] + o[l];
        }
        st16_f32(g.C32 + idx, o);
      }
      if (g.C16) st16_bf16(g.C16 + idx, o);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x < 32) tc::tmem_dealloc(tmem, C::TCOLS);
}

// C32[m][n] (+)= sum over slices of partial[z][m][n], slices in order.
__global__ void k_split_sum(int splits, int M, int N, const float *__restrict__ partial, float *__restrict__ C,
                            int ldc, int accumulate) {
  const size_t total = (size_t)M * N;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int z = 0; z < splits; ++z) s += partial[(size_t)z * total + t];
    const size_t idx = (t / N) * (size_t)ldc + t % N;
    C[idx] = accumulate ? C[idx] + s : s;
  }
}

// Host: 2D BF16 tensor map (inner x outer elements, row pitch in bytes) with
// the 128-byte swizzle and a box of box_inner x box_outer.
using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn encode_fn() {
  static const EncodeFn fn = []() -> EncodeFn {   // resolved once (thread-safe static init)
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeFn>(p);
    return nullptr;
  }();
  return fn;
}
bool make_tmap(CUtensorMap *tm, const void *ptr, int inner, int outer, int pitch_elems, int box_inner, int box_outer) {
  EncodeFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch_elems * 2};
  const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
  const cuuint32_t es[2] = {1, 1};
  return fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Launch C = A B with the layouts AL/BL (see k_gemm); returns false if a tensor
// map cannot be built or the launch fails.
template <int AL, int BL, int BN>
bool gemm(GemmArgs g, cudaStream_t s) {
  CUtensorMap ta, tb;
  // A(m,k): K-major = [M rows][K cols]; MN-major = [K rows][M cols]
  const bool okA = AL == A_ROW ? make_tmap(&ta, g.A, g.K, g.M, g.lda, kBK, 128)
                               : make_tmap(&ta, g.A, g.M, g.K, g.lda, 64, kBK);
  // B(k,n): K-major = [N rows][K cols]; MN-major = [K rows][N cols]
  const bool okB = BL == B_NMAJOR ? make_tmap(&tb, g.B, g.K, g.N, g.ldb, kBK, BN)
                                  : make_tmap(&tb, g.B, g.N, g.K, g.ldb, 64, kBK);
  if (!okA || !okB) return false;
  // the shared-memory opt-in, once per instantiation (thread-safe static init)
  static const bool attr = cudaFuncSetAttribute((const void *)k_gemm<AL, BL, BN>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                GemmCfg<BN>::SMEM) == cudaSuccess;
  if (!attr) return false;
  if (g.splits < 1) g.splits = 1;
  dim3 grid((g.N + BN - 1) / BN, (g.M + 127) / 128, g.splits);
  k_gemm<AL, BL, BN><<<grid, 128, GemmCfg<BN>::SMEM, s>>>(ta, tb, g);
  if (g.splits > 1)
    k_split_sum<<<296, 256, 0, s>>>(g.splits, g.M, g.N, g.partial, g.C32, g.ldc, g.accumulate);
  return cudaGetLastError() == cudaSuccess;
}

// --- elementwise helpers -----------------------------------------------------
__global__ void k_pack_input(int n, const float *__restrict__ X, __nv_bfloat16 *__restrict__ Xh) {
  const size_t total = (size_t)n * kInPad;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const size_t r = t / kInPad;
    const int c = (int)(t % kInPad);
    Xh[t] = __float2bfloat16(c < kIn ? X[r * kIn + c] : 0.0f);
  }
}

// dY = 2 (Y - T) / (n * OUT) as BF16; per-block partial sums of (Y - T)^2.
__global__ void k_loss_grad(int n, const float *__restrict__ Y, const float *__restrict__ T,
                            __nv_bfloat16 *__restrict__ dY, double *__restrict__ part) {
  const size_t total = (size_t)n * kOut;
  const float sc = 2.0f / (float)total;
  double acc = 0.0;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const float d = Y[t] - T[t];
    acc += (double)d * d;
    if (dY) dY[t] = __float2bfloat16(sc * d);
  }
  double v[1] = {acc};
  __shared__ double red[32];
  block_sum<1>(v, red);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

__global__ void k_loss_final(int nblocks, const double *__restrict__ part, size_t total, float *loss) {
  if (threadIdx.x < 32) {
    double s = warp_sum_partials(part, nblocks);
    if (threadIdx.x == 0) *loss = (float)(s / (double)total);
  }
}

// dZ = dH * gelu'(Z) as BF16 (dH FP32 [n][cols], Z pre-activation FP32).
__global__ void k_gelu_back(size_t total, const float *__restrict__ dH, const float *__restrict__ Z,
                            __nv_bfloat16 *__restrict__ dZ) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x)
    dZ[t] = __float2bfloat16(dH[t] * gelu_grad(Z[t]));
}

// Column sums of a BF16 [n][cols] matrix (bias gradients), deterministic two-level.
__global__ void k_colsum_part(int n, int cols, const __nv_bfloat16 *__restrict__ G, float *__restrict__ part,
                              int rows_per_block) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  const int r0 = blockIdx.y * rows_per_block, r1 = min(n, r0 + rows_per_block);
  float s = 0.0f;
  for (int r = r0; r < r1; ++r) s += __bfloat162float(G[(size_t)r * cols + c]);
  part[(size_t)blockIdx.y * cols + c] = s;
}
__global__ void k_colsum_final(int nparts, int cols, const float *__restrict__ part, float *__restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.0f;
  for (int p = 0; p < nparts; ++p) s += part[(size_t)p * cols + c];
  out[c] = s;
}

// Adam on the FP32 master parameters, then refresh of the BF16 weight copies.
__global__ void k_adam(int n, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m1,
                       float *__restrict__ m2, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.0f - b1) * gi;
    const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    w[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
  }
}

__global__ void k_to_bf16(int n, const float *__restrict__ w, __nv_bfloat16 *__restrict__ h) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) h[i] = __float2bfloat16(w[i]);
}

// parameter offsets inside the flat parameter vectors
constexpr int oW1 = 0, oB1 = oW1 + kHid * kInPad, oW2 = oB1 + kHid, oB2 = oW2 + kHid * kHid, oW3 = oB2 + kHid,
              oB3 = oW3 + kOut * kHid, kNParam = oB3 + kOut;

// Initial parameters: weights uniform in (-a, a), a = sqrt(6 / fan_in), from a
// counter-based hash (splitmix64 finalizer) of (seed, index); biases and the
// padded input columns of W1 are zero.
__global__ void k_init(float *__restrict__ w, unsigned long long seed) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNParam; i += gridDim.x * blockDim.x) {
    int fan = 0;
    if (i < oB1) fan = (i - oW1) % kInPad < kIn ? kIn : 0;
    else if (i >= oW2 && i < oB2) fan = kHid;
    else if (i >= oW3 && i < oB3) fan = kHid;
    if (fan == 0) { w[i] = 0.0f; continue; }
    unsigned long long z = seed * 0xD1B54A32D192ED03ull + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    w[i] = (float)((2.0 * u - 1.0) * sqrt(6.0 / (double)fan));
  }
}

}  // namespace
}  // namespace mlp
}  // namespace lh

using namespace lh;
using namespace lh::mlp;

struct lh_mlp {
  int max_rows = 0;
  char *arena = nullptr;
  // FP32 parameter blocks (master, grad, Adam moments), one contiguous vector each
  float *w = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
  __nv_bfloat16 *wh = nullptr;           // BF16 copies of W1, W2, W3 (same offsets as w)
  // activations for up to max_rows rows
  __nv_bfloat16 *Xh = nullptr, *H1h = nullptr, *H2h = nullptr, *dY = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *Y = nullptr, *dH2 = nullptr, *dH1 = nullptr, *part = nullptr;
  float *split = nullptr;   // split-K partial tiles of the weight-gradient GEMMs
  int *status = nullptr;    // LH_ERR_TIMEOUT latched by a GEMM whose bounded wait gave up
  double *lpart = nullptr;
  int steps = 0;
  std::string err;
};

namespace {
constexpr int kColParts = 64;
constexpr int kMaxSplits = 32;

// K slices for a weight-gradient GEMM (K = rows): about one CTA per SM in total.
int splits_for(int M, int N, int BN, int K) {
  const int tiles = ((N + BN - 1) / BN) * ((M + 127) / 128);
  const int kb = (K + kBK - 1) / kBK;
  int sp = 148 / tiles;
  if (sp > kMaxSplits) sp = kMaxSplits;
  if (sp > kb) sp = kb;
  return sp < 1 ? 1 : sp;
}

lh_status mfail(lh_mlp *m, lh_status s, const std::string &msg) {
  if (m) m->err = msg;
  lh::set_global_error(msg);
  return s;
}

// forward pass for n rows already packed in m->Xh; Y (FP32) out. keep_pre: also
// store the layers' pre-activations (needed by the backward pass only)
bool forward(lh_mlp *m, int n, float *Y, cudaStream_t s, bool keep_pre) {
  bool ok = true;
  GemmArgs g{};
  g.A = m->Xh; g.B = m->wh + oW1; g.M = n; g.N = kHid; g.K = kInPad; g.lda = kInPad; g.ldb = kInPad;
  g.bias = m->w + oB1; g.C16 = m->H1h; g.pre = keep_pre ? m->Z1 : nullptr; g.ldc = kHid; g.gelu = 1; g.status = m->status;
  ok = ok && gemm<A_ROW, B_NMAJOR, kHid>(g, s);
  g = GemmArgs{};
  g.A = m->H1h; g.B = m->wh + oW2; g.M = n; g.N = kHid; g.K = kHid; g.lda = kHid; g.ldb = kHid;
  g.bias = m->w + oB2; g.C16 = m->H2h; g.pre = keep_pre ? m->Z2 : nullptr; g.ldc = kHid; g.gelu = 1; g.status = m->status;
  ok = ok && gemm<A_ROW, B_NMAJOR, kHid>(g, s);
  g = GemmArgs{};
  g.A = m->H2h; g.B = m->wh + oW3; g.M = n; g.N = kOut; g.K = kHid; g.lda = kHid; g.ldb = kHid;
  g.bias = m->w + oB3; g.C32 = Y; g.ldc = kOut; g.status = m->status;
  ok = ok && gemm<A_ROW, B_NMAJOR, kOut>(g, s);
  return ok;
}

void colsum(lh_mlp *m, int n, int cols, const __nv_bfloat16 *G, float *out, cudaStream_t s) {
  const int rpb = (n + kColParts - 1) / kColParts;
  dim3 grid((cols + 127) / 128, kColParts);
  k_colsum_part<<<grid, 128, 0, s>>>(n, cols, G, m->part, rpb);
  k_colsum_final<<<(cols + 127) / 128, 128, 0, s>>>(kColParts, cols, m->part, out);
}

// loss and gradients of the mean squared error for n rows (Xh packed, T targets)
bool backward(lh_mlp *m, int n, const float *T, float *loss, cudaStream_t s) {
  const int lb = 296;
  bool ok = true;
  k_loss_grad<<<lb, 256, 0, s>>>(n, m->Y, T, m->dY, m->lpart);
  k_loss_final<<<1, 32, 0, s>>>(lb, m->lpart, (size_t)n * kOut, loss);
  GemmArgs g{};
  // dW3[o][h] = sum_r dY[r][o] H2[r][h]
  g.A = m->dY; g.B = m->H2h; g.M = kOut; g.N = kHid; g.K = n; g.lda = kOut; g.ldb = kHid;
  g.C32 = m->g + oW3; g.ldc = kHid; g.status = m->status;
  g.splits = splits_for(kOut, kHid, kHid, n); g.partial = m->split;
  ok = ok && gemm<A_COL, B_ROW, kHid>(g, s);
  colsum(m, n, kOut, m->dY, m->g + oB3, s);
  // dH2[r][h] = sum_o dY[r][o] W3[o][h]
  g = GemmArgs{};
  g.A = m->dY; g.B = m->wh + oW3; g.M = n; g.N = kHid; g.K = kOut; g.lda = kOut; g.ldb = kHid;
  g.C32 = m->dH2; g.ldc = kHid; g.status = m->status;
  ok = ok && gemm<A_ROW, B_ROW, kHid>(g, s);
  k_gelu_back<<<1024, 256, 0, s>>>((size_t)n * kHid, m->dH2, m->Z2, m->dZ2);
  // dW2[h][k] = sum_r dZ2[r][h] H1[r][k]
  g = GemmArgs{};
  g.A = m->dZ2; g.B = m->H1h; g.M = kHid; g.N = kHid; g.K = n; g.lda = kHid; g.ldb = kHid;
  g.C32 = m->g + oW2; g.ldc = kHid; g.status = m->status;
  g.splits = splits_for(kHid, kHid, kHid, n); g.partial = m->split;
  ok = ok && gemm<A_COL, B_ROW, kHid>(g, s);
  colsum(m, n, kHid, m->dZ2, m->g + oB2, s);
  // dH1[r][k] = sum_h dZ2[r][h] W2[h][k]
  g = GemmArgs{};
  g.A = m->dZ2; g.B = m->wh + oW2; g.M = n; g.N = kHid; g.K = kHid; g.lda = kHid; g.ldb = kHid;
  g.C32 = m->dH1; g.ldc = kHid; g.status = m->status;
  ok = ok && gemm<A_ROW, B_ROW, kHid>(g, s);
  k_gelu_back<<<1024, 256, 0, s>>>((size_t)n * kHid, m->dH1, m->Z1, m->dZ1);
  // dW1[h][i] = sum_r dZ1[r][h] X[r][i]
  g = GemmArgs{};
  g.A = m->dZ1; g.B = m->Xh; g.M = kHid; g.N = kInPad; g.K = n; g.lda = kHid; g.ldb = kInPad;
  g.C32 = m->g + oW1; g.ldc = kInPad; g.status = m->status;
  g.splits = splits_for(kHid, kInPad, kHid, n); g.partial = m->split;
  ok = ok && gemm<A_COL, B_ROW, kHid>(g, s);
  colsum(m, n, kHid, m->dZ1, m->g + oB1, s);
  return ok;
}

void refresh_bf16(lh_mlp *m, cudaStream_t s) { k_to_bf16<<<512, 256, 0, s>>>(kNParam, m->w, m->wh); }
}  // namespace

extern "C" {

int lh_mlp_num_params(void) { return kNParam; }

void lh_mlp_destroy(lh_mlp *m) {
  if (!m) return;
  if (m->arena) cudaFree(m->arena);
  delete m;
}

const char *lh_mlp_last_error(const lh_mlp *m) { return m ? m->err.c_str() : "null mlp"; }

lh_status lh_mlp_sync_status(lh_mlp *m) {
  if (!m) return LH_ERR_ARG;
  int st = 0;
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(&st, m->status, sizeof(int), cudaMemcpyDeviceToHost) !=
                                                    cudaSuccess)
    return mfail(m, LH_ERR_CUDA, "MLP status read failed");
  if (st != 0) {
    cudaMemset(m->status, 0, sizeof(int));
    return mfail(m, LH_ERR_TIMEOUT, "an MLP GEMM gave up a bounded device wait");
  }
  return LH_OK;
}

lh_status lh_mlp_create(unsigned long long seed, int max_rows, lh_mlp **out) {
  if (!out || max_rows < 1) return mfail(nullptr, LH_ERR_ARG, "bad lh_mlp_create arguments");
  *out = nullptr;
  lh_mlp *m = new lh_mlp();
  m->max_rows = max_rows;
  const size_t R = (size_t)max_rows;
  struct Item { void **p; size_t bytes; };
  std::vector<Item> items = {
      {(void **)&m->w, kNParam * 4},   {(void **)&m->g, kNParam * 4},       {(void **)&m->m1, kNParam * 4},
      {(void **)&m->m2, kNParam * 4},  {(void **)&m->wh, kNParam * 2},      {(void **)&m->Xh, R * kInPad * 2},
      {(void **)&m->H1h, R * kHid * 2}, {(void **)&m->H2h, R * kHid * 2},   {(void **)&m->dY, R * kOut * 2},
      {(void **)&m->dZ2, R * kHid * 2}, {(void **)&m->dZ1, R * kHid * 2},   {(void **)&m->Z1, R * kHid * 4},
      {(void **)&m->Z2, R * kHid * 4}, {(void **)&m->Y, R * kOut * 4},      {(void **)&m->dH2, R * kHid * 4},
      {(void **)&m->dH1, R * kHid * 4}, {(void **)&m->part, (size_t)kColParts * kInPad * 4},
      {(void **)&m->lpart, 4096 * 8},   {(void **)&m->split, (size_t)kMaxSplits * kHid * kInPad * 4},
      {(void **)&m->status, 256}};
  size_t bytes = 0;
  for (auto &it : items) bytes += (it.bytes + 255) / 256 * 256;
  if (cudaMalloc(&m->arena, bytes) != cudaSuccess) {
    m->arena = nullptr;
    lh_mlp_destroy(m);
    return mfail(nullptr, LH_ERR_OOM, "MLP arena allocation failed");
  }
  size_t off = 0;
  for (auto &it : items) {
    *it.p = m->arena + off;
    off += (it.bytes + 255) / 256 * 256;
  }
  cudaMemset(m->arena, 0, bytes);
  k_init<<<512, 256>>>(m->w, seed);
  refresh_bf16(m, 0);
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    lh_mlp_destroy(m);
    return mfail(nullptr, LH_ERR_CUDA, std::string("MLP init: ") + cudaGetErrorString(e));
  }
  *out = m;
  return LH_OK;
}

lh_status lh_mlp_get_params(const lh_mlp *m, float *host_out) {
  if (!m || !host_out) return LH_ERR_ARG;
  return cudaMemcpy(host_out, m->w, kNParam * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? LH_OK : LH_ERR_CUDA;
}

lh_status lh_mlp_set_params(lh_mlp *m, const float *host_in) {
  if (!m || !host_in) return LH_ERR_ARG;
  if (cudaMemcpy(m->w, host_in, kNParam * 4, cudaMemcpyHostToDevice) != cudaSuccess) return LH_ERR_CUDA;
  refresh_bf16(m, 0);
  m->steps = 0;
  cudaMemset(m->m1, 0, kNParam * 4);
  cudaMemset(m->m2, 0, kNParam * 4);
  return cudaDeviceSynchronize() == cudaSuccess ? LH_OK : LH_ERR_CUDA;
}

lh_status lh_mlp_forward(lh_mlp *m, const float *X, int n, float *Y, lh_stream_t stream) {
  if (!m || !X || !Y || n < 1) return mfail(m, LH_ERR_ARG, "bad lh_mlp_forward arguments");
  if (n > m->max_rows) return mfail(m, LH_ERR_ARG, "more rows than the MLP was created for");
  cudaStream_t s = (cudaStream_t)stream;
  k_pack_input<<<1024, 256, 0, s>>>(n, X, m->Xh);
  if (!forward(m, n, Y, s, false)) return mfail(m, LH_ERR_CUDA, "MLP forward: tensor map or launch failed");
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LH_OK : mfail(m, LH_ERR_CUDA, cudaGetErrorString(e));
}

lh_status lh_mlp_gradients(lh_mlp *m, const float *X, const float *T, int n, float *grads, float *loss,
                           lh_stream_t stream) {
  if (!m || !X || !T || !loss || n < 1) return mfail(m, LH_ERR_ARG, "bad lh_mlp_gradients arguments");
  if (n > m->max_rows) return mfail(m, LH_ERR_ARG, "more rows than the MLP was created for");
  cudaStream_t s = (cudaStream_t)stream;
  k_pack_input<<<1024, 256, 0, s>>>(n, X, m->Xh);
  if (!forward(m, n, m->Y, s, true) || !backward(m, n, T, loss, s))
    return mfail(m, LH_ERR_CUDA, "MLP gradients: tensor map or launch failed");
  if (grads) cudaMemcpyAsync(grads, m->g, kNParam * 4, cudaMemcpyDeviceToDevice, s);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LH_OK : mfail(m, LH_ERR_CUDA, cudaGetErrorString(e));
}

lh_status lh_mlp_train_step(lh_mlp *m, const float *X, const float *T, int n, float lr, float *loss,
                            lh_stream_t stream) {
  if (lh_status st = lh_mlp_gradients(m, X, T, n, nullptr, loss, stream)) return st;
  cudaStream_t s = (cudaStream_t)stream;
  m->steps += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)m->steps), c2 = 1.0f - powf(b2, (float)m->steps);
  // padded input columns of W1 get zero gradients and therefore stay zero
  k_adam<<<512, 256, 0, s>>>(kNParam, m->w, m->g, m->m1, m->m2, lr, b1, b2, 1e-8f, c1, c2);
  refresh_bf16(m, s);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LH_OK : mfail(m, LH_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"

namespace lh {
// For the learned form, which writes its features straight into the network's
// packed BF16 input ([max_rows][kInPad], padding columns zero since creation and
// never written): the buffer and its row capacity, and the forward pass from it.
__nv_bfloat16 *mlp_packed_input(lh_mlp *m, int *max_rows) {
  if (max_rows) *max_rows = m ? m->max_rows : 0;
  return m ? m->Xh : nullptr;
}
lh_status mlp_forward_packed(lh_mlp *m, int n, float *Y, cudaStream_t s) {
  if (!m || !Y || n < 1) return mfail(m, LH_ERR_ARG, "bad MLP forward arguments");
  if (n > m->max_rows) return mfail(m, LH_ERR_ARG, "more rows than the MLP was created for");
  if (!forward(m, n, Y, s, false)) return mfail(m, LH_ERR_CUDA, "MLP forward: tensor map or launch failed");
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LH_OK : mfail(m, LH_ERR_CUDA, cudaGetErrorString(e));
}
}  // namespace lh
