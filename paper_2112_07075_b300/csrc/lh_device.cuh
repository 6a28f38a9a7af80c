// Device-side building blocks shared by every kernel of liblh:
//  * compile-time tensor contractions over shared memory (sum factorization,
//    arXiv 2112.07075 Section 3.2: B = B1d (x) B1d (x) B1d applied one axis at a time),
//  * warp / block reductions,
//  * a bounded grid-wide barrier for the persistent cooperative CG kernel.
#pragma once

#include <cuda/atomic>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lh {

// ---------------------------------------------------------------------------
// Integer powers.
// ---------------------------------------------------------------------------
template <int B, int E>
struct ipow { static constexpr int value = B * ipow<B, E - 1>::value; };
template <int B>
struct ipow<B, 0> { static constexpr int value = 1; };

// ---------------------------------------------------------------------------
// One-axis contraction over a block-resident tensor.
//   in  : [A][K][BS] (flattened, BS fastest)
//   out : [A][O][BS]
//   out[a][o][b] = sum_k M[o][k] * in[a][k][b],  M row-major [O][K].
// All threads of the block share the work; the caller synchronises.
// Every output costs K FP64 fused multiply-adds (the first one a multiply).
// ---------------------------------------------------------------------------
template <int A, int K, int O, int BS, typename T>
__device__ __forceinline__ void contract(const T *__restrict__ in, T *__restrict__ out, const T *__restrict__ M) {
  constexpr int N = A * O * BS;
  for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
    const int b = idx % BS;
    const int t = idx / BS;
    const int o = t % O;
    const int a = t / O;
    const T *ip = in + a * K * BS + b;
    const T *mp = M + o * K;
    T s = mp[0] * ip[0];
#pragma unroll
    for (int k = 1; k < K; ++k) s = fma(mp[k], ip[k * BS], s);
    out[idx] = s;
  }
}

// Same as contract but two inputs and two matrices summed:
//   out[a][o][b] = sum_k M1[o][k] in1[a][k][b] + M2[o][k] in2[a][k][b].
template <int A, int K, int O, int BS>
__device__ __forceinline__ void contract2(const double *__restrict__ in1, const double *__restrict__ M1,
                                          const double *__restrict__ in2, const double *__restrict__ M2,
                                          double *__restrict__ out) {
  constexpr int N = A * O * BS;
  for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
    const int b = idx % BS;
    const int t = idx / BS;
    const int o = t % O;
    const int a = t / O;
    const double *i1 = in1 + a * K * BS + b;
    const double *i2 = in2 + a * K * BS + b;
    const double *m1 = M1 + o * K;
    const double *m2 = M2 + o * K;
    double s = m1[0] * i1[0];
#pragma unroll
    for (int k = 1; k < K; ++k) s = fma(m1[k], i1[k * BS], s);
#pragma unroll
    for (int k = 0; k < K; ++k) s = fma(m2[k], i2[k * BS], s);
    out[idx] = s;
  }
}

// ---------------------------------------------------------------------------
// Pencil form of `contract`: one thread owns a whole pencil (a, b): it loads
// in[a][0..K-1][b] into registers once and writes out[a][0..O-1][b]. Matrix
// entries are read as warp-uniform shared-memory broadcasts. Fewer address and
// shared-memory instructions per multiply-add than one-output-per-step loops,
// which matters where the arithmetic itself is cheap (FP32); the O x K matrix
// is kept in registers.
// ---------------------------------------------------------------------------
template <int A, int K, int O, int BS, typename T>
__device__ __forceinline__ void contract_p(const T *__restrict__ in, T *__restrict__ out, const T *__restrict__ Ms) {
  constexpr int NP = A * BS;
  T M[O * K];   // the 1D matrix, held in registers for the whole stage
#pragma unroll
  for (int j = 0; j < O * K; ++j) M[j] = Ms[j];
  for (int idx = threadIdx.x; idx < NP; idx += blockDim.x) {
    const int b = idx % BS;
    const int a = idx / BS;
    const T *ip = in + a * K * BS + b;
    T v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = ip[k * BS];
    T *op = out + a * O * BS + b;
#pragma unroll
    for (int o = 0; o < O; ++o) {
      T s = M[o * K] * v[0];
#pragma unroll
      for (int k = 1; k < K; ++k) s = fma(M[o * K + k], v[k], s);
      op[o * BS] = s;
    }
  }
}

// Pencil-form tensor-product interpolation (same result layout as interp).
template <int DIM, int NI, int NO, int C, typename T>
__device__ __forceinline__ void interp_p(const T *__restrict__ in, T *__restrict__ out, T *__restrict__ S,
                                         const T *__restrict__ M) {
  if constexpr (DIM == 2) {
    contract_p<C * NI, NI, NO, 1>(in, S, M);
    __syncthreads();
    contract_p<C, NI, NO, NO>(S, out, M);
    __syncthreads();
  } else {
    T *t2 = S + C * NI * NI * NO;
    contract_p<C * NI * NI, NI, NO, 1>(in, S, M);
    __syncthreads();
    contract_p<C * NI, NI, NO, NO>(S, t2, M);
    __syncthreads();
    contract_p<C, NI, NO, NO * NO>(t2, out, M);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Scratch sizes (doubles) of the helpers below, for C tensors.
// ---------------------------------------------------------------------------
template <int DIM, int NI, int NO>
__host__ __device__ constexpr int interp_scratch(int C) {
  return DIM == 2 ? C * NI * NO : C * NI * NO * (NI + NO);
}
template <int DIM, int D, int Q>
__host__ __device__ constexpr int grad_scratch(int C) {
  return DIM == 2 ? 2 * C * D * Q : 2 * C * D * D * Q + 3 * C * D * Q * Q;
}

// ---------------------------------------------------------------------------
// Full tensor-product interpolation with one 1D matrix M [NO][NI] on every axis:
//   out[c][o_z][o_y][o_x] = sum M[o_x][i_x] M[o_y][i_y] M[o_z][i_z] in[c][i_z][i_y][i_x]
// for C independent tensors. S: interp_scratch(C) doubles. Ends with a __syncthreads.
// ---------------------------------------------------------------------------
template <int DIM, int NI, int NO, int C, typename T>
__device__ __forceinline__ void interp(const T *__restrict__ in, T *__restrict__ out, T *__restrict__ S,
                                       const T *__restrict__ M) {
  if constexpr (DIM == 2) {
    contract<C * NI, NI, NO, 1>(in, S, M);          // x: [C][iy][ox]
    __syncthreads();
    contract<C, NI, NO, NO>(S, out, M);             // y: [C][oy][ox]
    __syncthreads();
  } else {
    T *t2 = S + C * NI * NI * NO;
    contract<C * NI * NI, NI, NO, 1>(in, S, M);     // x: [C][iz][iy][ox]
    __syncthreads();
    contract<C * NI, NI, NO, NO>(S, t2, M);         // y: [C][iz][oy][ox]
    __syncthreads();
    contract<C, NI, NO, NO * NO>(t2, out, M);       // z: [C][oz][oy][ox]
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Reference gradient at quadrature points of C scalar H1 tensors:
//   g[l][c][q] = sum_i dw_i/dxi_l(q) u[c][i],  B, G: [Q][D].
// S: grad_scratch(C) doubles. Ends with a __syncthreads.
// FP64 cost per tensor (3D): 2QD^3 + 3Q^2D^2 + 3Q^3D fused multiply-adds.
// ---------------------------------------------------------------------------
template <int DIM, int D, int Q, int C>
__device__ __forceinline__ void grad_ref(const double *__restrict__ u, double *__restrict__ g,
                                         double *__restrict__ S, const double *__restrict__ B,
                                         const double *__restrict__ G) {
  constexpr int NQ = ipow<Q, DIM>::value;
  if constexpr (DIM == 2) {
    double *ta = S, *tb = S + C * D * Q;
    contract<C * D, D, Q, 1>(u, ta, B);       // [C][iy][qx] B_x
    contract<C * D, D, Q, 1>(u, tb, G);       // [C][iy][qx] G_x
    __syncthreads();
    contract<C, D, Q, Q>(tb, g, B);           // d/dx: G_x B_y
    contract<C, D, Q, Q>(ta, g + C * NQ, G);  // d/dy: B_x G_y
    __syncthreads();
  } else {
    double *ta = S, *tb = ta + C * D * D * Q, *tc = tb + C * D * D * Q;
    double *td = tc + C * D * Q * Q, *te = td + C * D * Q * Q;
    contract<C * D * D, D, Q, 1>(u, ta, B);   // [C][iz][iy][qx] B_x
    contract<C * D * D, D, Q, 1>(u, tb, G);   // G_x
    __syncthreads();
    contract<C * D, D, Q, Q>(tb, tc, B);      // [C][iz][qy][qx] G_x B_y
    contract<C * D, D, Q, Q>(ta, td, G);      // B_x G_y
    contract<C * D, D, Q, Q>(ta, te, B);      // B_x B_y
    __syncthreads();
    contract<C, D, Q, Q * Q>(tc, g, B);               // d/dx: G_x B_y B_z
    contract<C, D, Q, Q * Q>(td, g + C * NQ, B);      // d/dy: B_x G_y B_z
    contract<C, D, Q, Q * Q>(te, g + 2 * C * NQ, G);  // d/dz: B_x B_y G_z
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Transposed reference gradient: for C components,
//   y[c][i] = sum_q sum_l dw_i/dxi_l(q) f[l][c][q],   f: [DIM][C][Q^DIM]
// Bt, Gt: [D][Q] (transposed tables). S: grad_scratch(C) doubles.
// Ends with a __syncthreads. FP64 cost per component (3D): 3Q^3D + 3Q^2D^2 + 2QD^3.
// ---------------------------------------------------------------------------
template <int DIM, int D, int Q, int C>
__device__ __forceinline__ void grad_ref_t(const double *__restrict__ f, double *__restrict__ y,
                                           double *__restrict__ S, const double *__restrict__ Bt,
                                           const double *__restrict__ Gt) {
  constexpr int NQ = ipow<Q, DIM>::value;
  if constexpr (DIM == 2) {
    double *ta = S, *tb = S + C * D * Q;
    contract<C, Q, D, Q>(f, ta, Bt);            // [C][iy][qx]: B_y^T f_x
    contract<C, Q, D, Q>(f + C * NQ, tb, Gt);   // G_y^T f_y
    __syncthreads();
    contract2<C * D, Q, D, 1>(ta, Gt, tb, Bt, y);  // x: G_x^T (.) + B_x^T (.)
    __syncthreads();
  } else {
    double *ta = S, *tb = ta + C * D * Q * Q, *tc = tb + C * D * Q * Q;
    double *td = tc + C * D * Q * Q, *te = td + C * D * D * Q;
    contract<C, Q, D, Q * Q>(f, ta, Bt);               // [C][iz][qy][qx]: B_z^T f_x
    contract<C, Q, D, Q * Q>(f + C * NQ, tb, Bt);      // B_z^T f_y
    contract<C, Q, D, Q * Q>(f + 2 * C * NQ, tc, Gt);  // G_z^T f_z
    __syncthreads();
    contract<C * D, Q, D, Q>(ta, td, Bt);              // [C][iz][iy][qx]: B_y^T (x-term)
    contract2<C * D, Q, D, Q>(tb, Gt, tc, Bt, te);     // G_y^T (y-term) + B_y^T (z-term)
    __syncthreads();
    contract2<C * D * D, Q, D, 1>(td, Gt, te, Bt, y);  // G_x^T (x-term) + B_x^T (rest)
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Warp and block reductions (fixed order, hence deterministic).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block sum of NV values per thread; result valid in warp 0 (all lanes).
// red: >= 32*NV doubles of shared memory. Contains __syncthreads.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) red[k * 32 + warp] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = lane < nw ? red[k * 32 + lane] : 0.0;
      v[k] = warp_sum(s);
    }
  }
  __syncthreads();
}

// Block max; result valid in warp 0. Contains __syncthreads.
__device__ __forceinline__ double block_max(double v, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double s = lane < nw ? red[lane] : -INFINITY;
    v = warp_max(s);
  }
  __syncthreads();
  return v;
}

// Sum of n partials in a fixed order, computed by one warp (result in every lane):
// lane l adds p[l], p[l + 32], ... in turn, then the lanes are summed. The loads
// are issued eight at a time, ahead of the additions, which keep that order.
__device__ __forceinline__ double warp_sum_partials(const double *p, int n) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  if (n <= 10 * 32) {
    // the usual grid sizes (two CTAs per SM: 296 partials): every load of the lane
    // is issued before the first add, so the sum costs one memory round trip instead
    // of one per load after the first eight; the adds run in the same index order
    double v[10];
#pragma unroll
    for (int j = 0; j < 10; ++j) v[j] = lane + 32 * j < n ? p[lane + 32 * j] : 0.0;
#pragma unroll
    for (int j = 0; j < 10; ++j)
      if (lane + 32 * j < n) s += v[j];
    return warp_sum(s);
  }
  int i = lane;
  for (; i + 7 * 32 < n; i += 8 * 32) {
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = p[i + 32 * j];
#pragma unroll
    for (int j = 0; j < 8; ++j) s += v[j];
  }
  for (; i < n; i += 32) s += p[i];
  return warp_sum(s);
}

// This block's work items [k0, k1) when n items are split into gridDim.x
// contiguous chunks of equal size (+-1): every block, hence every SM, gets the
// same share (a grid-stride loop gives the first blocks one item more per thread).
__device__ __forceinline__ void block_chunk(int n, int &k0, int &k1) {
  const int G = gridDim.x, b = blockIdx.x, base = n / G, rem = n % G;
  k0 = b * base + (b < rem ? b : rem);
  k1 = k0 + base + (b < rem ? 1 : 0);
}

// FP32 twin of warp_sum_partials (same order: lane l adds p[l], p[l + 32], ...,
// then the lanes are summed by xor shuffles).
__device__ __forceinline__ float warp_sum_partials_f(const float *p, int n) {
  const int lane = threadIdx.x & 31;
  float s = 0.0f;
  if (n <= 10 * 32) {   // one round trip, as in warp_sum_partials
    float v[10];
#pragma unroll
    for (int j = 0; j < 10; ++j) v[j] = lane + 32 * j < n ? p[lane + 32 * j] : 0.0f;
#pragma unroll
    for (int j = 0; j < 10; ++j)
      if (lane + 32 * j < n) s += v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
  }
  int i = lane;
  for (; i + 7 * 32 < n; i += 8 * 32) {
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = p[i + 32 * j];
#pragma unroll
    for (int j = 0; j < 8; ++j) s += v[j];
  }
  for (; i < n; i += 32) s += p[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// ---------------------------------------------------------------------------
// Device status word: the first error wins.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void latch_status(int *status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------
// Bounded grid barrier for cooperative launches (all blocks co-resident).
// A monotonic 64-bit arrival counter, zeroed by the host before each launch:
// barrier number k (1, 2, ...) of a launch waits until the counter reaches
// k * gridDim.x. Arrival is a release add (no return value), waiting an acquire
// load, so the block's writes before the barrier are visible after it. Waiters
// give up after about one second (clock64), latch LH_ERR_TIMEOUT and report
// failure; callers then return.
// ---------------------------------------------------------------------------
struct GridBarrier {
  unsigned long long count;
};

constexpr long long kBarrierSpinCycles = 2000000000LL;  // ~1 s at 2 GHz
constexpr int kStatusTimeout = 6;                        // LH_ERR_TIMEOUT

__device__ __forceinline__ bool grid_sync(GridBarrier *gb, unsigned long long target, int *status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> cnt(gb->count);
    cnt.fetch_add(1ull, cuda::memory_order_release);
    int ok = 1;
    const long long t0 = clock64();
    while (cnt.load(cuda::memory_order_acquire) < target) {
      if (clock64() - t0 > kBarrierSpinCycles) {
        ok = 0;
        latch_status(status, kStatusTimeout);
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace lh
