// Per-element MLP of the learned form: 586 -> 128 -> 128 -> 192, GELU (erf form)
// after both hidden layers, BF16 weights and activations on the tensor cores
// (mma.sync m16n8k16, FP32 accumulation), FP32 master weights, Adam.
// Used to predict the mass-CG initial guess (see learned.cu); this file holds
// the network itself: parameter init, forward, backward, optimiser step.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "lh_device.cuh"
#include "lh_internal.h"
#include "lh_mlp.h"

namespace lh {
namespace mlp {
namespace {

// ---------------------------------------------------------------------------
// BF16 GEMM on the tensor cores: C[m][n] = sum_k A(m,k) B(k,n) (+ bias[n]),
// FP32 accumulation. A is row-major (A[m*lda+k]) or column-major (A[k*lda+m]);
// B is "n-major" (B[n*ldb+k], i.e. a row-major weight matrix used as B = W^T)
// or row-major (B[k*ldb+n]). Block tile 64x64x32, 4 warps (2x2), each warp 32x32
// with m16n8k16 MMAs. Out-of-range rows/cols/k read as zero.
// Epilogue: C32 (FP32) and/or C16 (BF16) with optional bias and GELU; when
// PRE is given the pre-activation is written there (FP32).
// ---------------------------------------------------------------------------
constexpr int BM = 64, BN = 64, BK = 32, PADK = BK + 8;

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
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int AL, int BL>
__global__ void __launch_bounds__(128) k_gemm(GemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 sA[BM][PADK];   // [m][k]
  __shared__ __align__(16) __nv_bfloat16 sB[BN][PADK];   // [n][k]
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int grp = lane >> 2, tig = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  for (int k0 = 0; k0 < g.K; k0 += BK) {
    for (int t = threadIdx.x; t < BM * BK; t += 128) {
      int mm, kk;
      if (AL == A_ROW) { mm = t / BK; kk = t % BK; } else { kk = t / BM; mm = t % BM; }
      const int m = m0 + mm, k = k0 + kk;
      __nv_bfloat16 v = zero;
      if (m < g.M && k < g.K) v = AL == A_ROW ? g.A[(size_t)m * g.lda + k] : g.A[(size_t)k * g.lda + m];
      sA[mm][kk] = v;
    }
    for (int t = threadIdx.x; t < BN * BK; t += 128) {
      int nn, kk;
      if (BL == B_NMAJOR) { nn = t / BK; kk = t % BK; } else { kk = t / BN; nn = t % BN; }
      const int n = n0 + nn, k = k0 + kk;
      __nv_bfloat16 v = zero;
      if (n < g.N && k < g.K) v = BL == B_NMAJOR ? g.B[(size_t)n * g.ldb + k] : g.B[(size_t)k * g.ldb + n];
      sB[nn][kk] = v;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
      unsigned af[2][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + i * 16 + grp;
        af[i][0] = *(const unsigned *)&sA[r][ks + tig * 2];
        af[i][1] = *(const unsigned *)&sA[r + 8][ks + tig * 2];
        af[i][2] = *(const unsigned *)&sA[r][ks + tig * 2 + 8];
        af[i][3] = *(const unsigned *)&sA[r + 8][ks + tig * 2 + 8];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + j * 8 + grp;
        bf[j][0] = *(const unsigned *)&sB[c][ks + tig * 2];
        bf[j][1] = *(const unsigned *)&sB[c][ks + tig * 2 + 8];
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + wm + i * 16 + grp + (r >= 2 ? 8 : 0);
        const int n = n0 + wn + j * 8 + tig * 2 + (r & 1);
        if (m >= g.M || n >= g.N) continue;
        float z = acc[i][j][r];
        if (g.bias) z += g.bias[n];
        const size_t idx = (size_t)m * g.ldc + n;
        if (g.pre) g.pre[idx] = z;
        const float o = g.gelu ? gelu_f(z) : z;
        if (g.C32) g.C32[idx] = g.accumulate ? g.C32[idx] + o : o;
        if (g.C16) g.C16[idx] = __float2bfloat16(o);
      }
}

template <int AL, int BL>
void gemm(const GemmArgs &g, cudaStream_t s) {
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM);
  k_gemm<AL, BL><<<grid, 128, 0, s>>>(g);
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
  double *lpart = nullptr;
  int steps = 0;
  std::string err;
};

namespace {
constexpr int kColParts = 64;

lh_status mfail(lh_mlp *m, lh_status s, const std::string &msg) {
  if (m) m->err = msg;
  lh::set_global_error(msg);
  return s;
}

// forward pass for n rows already packed in m->Xh; Y (FP32) out
void forward(lh_mlp *m, int n, float *Y, cudaStream_t s) {
  GemmArgs g{};
  g.A = m->Xh; g.B = m->wh + oW1; g.M = n; g.N = kHid; g.K = kInPad; g.lda = kInPad; g.ldb = kInPad;
  g.bias = m->w + oB1; g.C16 = m->H1h; g.pre = m->Z1; g.ldc = kHid; g.gelu = 1;
  gemm<A_ROW, B_NMAJOR>(g, s);
  g = GemmArgs{};
  g.A = m->H1h; g.B = m->wh + oW2; g.M = n; g.N = kHid; g.K = kHid; g.lda = kHid; g.ldb = kHid;
  g.bias = m->w + oB2; g.C16 = m->H2h; g.pre = m->Z2; g.ldc = kHid; g.gelu = 1;
  gemm<A_ROW, B_NMAJOR>(g, s);
  g = GemmArgs{};
  g.A = m->H2h; g.B = m->wh + oW3; g.M = n; g.N = kOut; g.K = kHid; g.lda = kHid; g.ldb = kHid;
  g.bias = m->w + oB3; g.C32 = Y; g.ldc = kOut;
  gemm<A_ROW, B_NMAJOR>(g, s);
}

void colsum(lh_mlp *m, int n, int cols, const __nv_bfloat16 *G, float *out, cudaStream_t s) {
  const int rpb = (n + kColParts - 1) / kColParts;
  dim3 grid((cols + 127) / 128, kColParts);
  k_colsum_part<<<grid, 128, 0, s>>>(n, cols, G, m->part, rpb);
  k_colsum_final<<<(cols + 127) / 128, 128, 0, s>>>(kColParts, cols, m->part, out);
}

// loss and gradients of the mean squared error for n rows (Xh packed, T targets)
void backward(lh_mlp *m, int n, const float *T, float *loss, cudaStream_t s) {
  const int lb = 296;
  k_loss_grad<<<lb, 256, 0, s>>>(n, m->Y, T, m->dY, m->lpart);
  k_loss_final<<<1, 32, 0, s>>>(lb, m->lpart, (size_t)n * kOut, loss);
  GemmArgs g{};
  // dW3[o][h] = sum_r dY[r][o] H2[r][h]
  g.A = m->dY; g.B = m->H2h; g.M = kOut; g.N = kHid; g.K = n; g.lda = kOut; g.ldb = kHid;
  g.C32 = m->g + oW3; g.ldc = kHid;
  gemm<A_COL, B_ROW>(g, s);
  colsum(m, n, kOut, m->dY, m->g + oB3, s);
  // dH2[r][h] = sum_o dY[r][o] W3[o][h]
  g = GemmArgs{};
  g.A = m->dY; g.B = m->wh + oW3; g.M = n; g.N = kHid; g.K = kOut; g.lda = kOut; g.ldb = kHid;
  g.C32 = m->dH2; g.ldc = kHid;
  gemm<A_ROW, B_ROW>(g, s);
  k_gelu_back<<<1024, 256, 0, s>>>((size_t)n * kHid, m->dH2, m->Z2, m->dZ2);
  // dW2[h][k] = sum_r dZ2[r][h] H1[r][k]
  g = GemmArgs{};
  g.A = m->dZ2; g.B = m->H1h; g.M = kHid; g.N = kHid; g.K = n; g.lda = kHid; g.ldb = kHid;
  g.C32 = m->g + oW2; g.ldc = kHid;
  gemm<A_COL, B_ROW>(g, s);
  colsum(m, n, kHid, m->dZ2, m->g + oB2, s);
  // dH1[r][k] = sum_h dZ2[r][h] W2[h][k]
  g = GemmArgs{};
  g.A = m->dZ2; g.B = m->wh + oW2; g.M = n; g.N = kHid; g.K = kHid; g.lda = kHid; g.ldb = kHid;
  g.C32 = m->dH1; g.ldc = kHid;
  gemm<A_ROW, B_ROW>(g, s);
  k_gelu_back<<<1024, 256, 0, s>>>((size_t)n * kHid, m->dH1, m->Z1, m->dZ1);
  // dW1[h][i] = sum_r dZ1[r][h] X[r][i]
  g = GemmArgs{};
  g.A = m->dZ1; g.B = m->Xh; g.M = kHid; g.N = kInPad; g.K = n; g.lda = kHid; g.ldb = kInPad;
  g.C32 = m->g + oW1; g.ldc = kInPad;
  gemm<A_COL, B_ROW>(g, s);
  colsum(m, n, kHid, m->dZ1, m->g + oB1, s);
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
      {(void **)&m->lpart, 4096 * 8}};
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
  forward(m, n, Y, s);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LH_OK : mfail(m, LH_ERR_CUDA, cudaGetErrorString(e));
}

lh_status lh_mlp_gradients(lh_mlp *m, const float *X, const float *T, int n, float *grads, float *loss,
                           lh_stream_t stream) {
  if (!m || !X || !T || !loss || n < 1) return mfail(m, LH_ERR_ARG, "bad lh_mlp_gradients arguments");
  if (n > m->max_rows) return mfail(m, LH_ERR_ARG, "more rows than the MLP was created for");
  cudaStream_t s = (cudaStream_t)stream;
  k_pack_input<<<1024, 256, 0, s>>>(n, X, m->Xh);
  forward(m, n, m->Y, s);
  backward(m, n, T, loss, s);
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
