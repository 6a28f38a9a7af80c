// Tensor-core (tcgen05) element operator of the precision form's inner solver,
// 3D, H1 order p >= 3 (the mass operator of Section 3.2 with its contractions
// on the tensor cores, BF16 inputs and FP32 accumulation).
//
// Per row = (element, velocity component) the interpolation to the quadrature
// points and its transpose are products with the Kronecker matrix
//   K = B (x) B (x) B,   K[q][i] = B[qx][ix] B[qy][iy] B[qz][iz],
//   q = qx + Q qy + Q^2 qz,   i = ix + D iy + D^2 iz,
// i.e. the sum-factorized B of Section 3.2 assembled per element. A tile of 128
// rows X[128][ND] (the search direction at the rows' element nodes) runs
//   GEMM1  Y = X K^T            (128 x N1, K = ND)   accumulator in tensor memory
//   scale  Z = Y .* mq          (omega rho0 detJ0 of the row's element, FP32)
//   GEMM2  W = Z K              (128 x N2, K = N1)   accumulator in tensor memory
// and W is the row's part of the E-vector (nodes summed afterwards by the same
// deterministic gather as every other sweep). Every operand is split as
// x = x_hi + x_lo in BF16 and each GEMM accumulates hi*hi + hi*lo + lo*hi in
// FP32: the dropped lo*lo term and the split residual are ~2^-17 relative, so
// the element operator is accurate to a few 1e-6, enough for inner solves of
// 1e-4 under the FP64 refinement of the precision form.
//
// K lives in shared memory once, as a 128B-swizzled BF16 image (hi, then lo):
// rows q (N1 of them), 64 node values per 128-byte row, 64-node blocks one after
// the other. GEMM1 reads it K-major (B[n=q][k=i]); GEMM2 reads the same bytes
// MN-major (B[k=q][n=i]: 8-row groups of q 1024 B apart, 64-node blocks one
// image block apart).
#pragma once

#include <cstdint>
#include <cstring>

#include "lh_kernels.cuh"
#include "tc_sm100.cuh"

namespace lh {

template <int P, int Q>
struct TcLayout {
  static constexpr int D = P + 1, ND = D * D * D, NQ = Q * Q * Q;
  static constexpr int ROWS = 128;                  // (element, component) rows per tile = MMA M
  static constexpr int NKB = (ND + 63) / 64;        // 64-wide blocks of the node index (GEMM1's K)
  static constexpr int N1 = (NQ + 31) / 32 * 32;    // GEMM1 N: quadrature points, padded
  static constexpr int NCH = (N1 + 63) / 64;        // 64-wide q chunks (GEMM2's K)
  static constexpr int N2 = NKB * 64;               // GEMM2 N: nodes, padded
  static constexpr bool supported = P >= 3 && N1 <= 256 && N2 <= 128 && NQ % 8 == 0;
  static constexpr int IMG_BLOCK = N1 * 128;        // one node block of the image: N1 rows x 128 B
  static constexpr int IMG_HALF = NKB * IMG_BLOCK;  // hi image; the lo image follows
  static constexpr int IMG = 2 * IMG_HALF;
  static constexpr int A_BLOCK = ROWS * 128;        // 128 rows x 64 BF16 values
  static constexpr int A1 = 2 * NKB * A_BLOCK;      // X tile, hi + lo
  static constexpr int A2 = 4 * A_BLOCK;            // two q-chunk buffers of Z, hi + lo each
  static constexpr int STG_LD = ND % 2 == 0 ? ND + 1 : ND;   // odd row stride: conflict-free writes
  static constexpr int STG = ROWS * STG_LD * 4;     // W staged for coalesced E-vector stores
  static constexpr int AREG0 = A1 > A2 ? (A1 > STG ? A1 : STG) : (A2 > STG ? A2 : STG);
  static constexpr int AREG = (AREG0 + 1023) / 1024 * 1024;
  static constexpr int MQ_E = ROWS / 3 + 2;         // elements a tile touches, at most
  static constexpr int MQB = (MQ_E * NQ * 4 + 1023) / 1024 * 1024;
  static constexpr int TMEM_COLS = 512, D1_COL = 0, D2_COL = 256;
  // Byte offset of (row, k) in a K-major operand block of 128-byte rows (64 BF16
  // values) with the 128-byte swizzle: 16-byte chunk index XOR (row mod 8).
  __host__ __device__ static constexpr int sw128(int row, int k) {
    return (row >> 3) * 1024 + (row & 7) * 128 + ((((k >> 3) ^ row) & 7) << 4) + (k & 7) * 2;
  }
};

template <int DIM, int P, int Q>
struct TcTraits {
  static constexpr bool on = DIM == 3 && TcLayout<P, Q>::supported;
};

template <int P, int Q>
struct TcMass {
  using L = TcLayout<P, Q>;
  using F = Family<3, P, Q>;
  static constexpr int THREADS = 512;   // the launcher table (lh_ops.cuh) assumes 512
  static constexpr int D = L::D, ND = L::ND, NQ = L::NQ;
  static constexpr uint32_t IDESC1 = tc::idesc_bf16(128, L::N1, false);
  static constexpr uint32_t IDESC2 = tc::idesc_bf16(128, L::N2, true);
  // dynamic shared memory: [alignment slack][image][A region][mq tile][reduction scratch]
  static constexpr size_t RED_BYTES = sizeof(double) * F::RED;
  static constexpr size_t SMEM = 1024 + L::IMG + L::AREG + L::MQB + RED_BYTES;
  // the FP64 refinement sweep (tables + one element batch) reuses A region + mq tile
  static constexpr size_t FP64_BYTES = sizeof(double) * (F::TAB + F::IR_D);
  static_assert(FP64_BYTES <= (size_t)(L::AREG + L::MQB), "FP64 sweep space does not fit");
  static_assert(SMEM + 1024 <= 232448, "shared memory of the tensor-core solver exceeds 227 KB");

  char *img, *areg, *mqs;
  uint64_t *bars;   // [0] MMA completion, [1] [2] q-chunk buffers, [3] bulk copies (image, mq tile)
  int *s_base;      // per element of the tile: its base H1 node
  uint32_t tmem;
  uint32_t n_mma, n_buf[2], n_copy;   // phases completed so far (the same in every thread)

  // Bounded wait on an mbarrier phase, made block-uniform; latches LH_ERR_TIMEOUT.
  __device__ bool wait(uint64_t *bar, uint32_t parity, int *status) {
    const bool ok = tc::mbar_wait(bar, parity, kBarrierSpinCycles);
    const int all = __syncthreads_and(ok ? 1 : 0);
    if (!all && threadIdx.x == 0) latch_status(status, kStatusTimeout);
    return all != 0;
  }

  // Sets up one block: barriers, tensor memory (512 columns), the image of K.
  // Block-uniform result; false after a bounded wait gave up.
  __device__ bool begin(const CgIrArgs &a, char *base, uint64_t *bar4, uint32_t *s_tmem, int *base_rows) {
    img = base;
    areg = base + L::IMG;
    mqs = areg + L::AREG;
    bars = bar4;
    s_base = base_rows;
    n_mma = 0;
    n_buf[0] = n_buf[1] = 0;
    n_copy = 0;
    if (threadIdx.x == 0) {
      for (int k = 0; k < 4; ++k) tc::mbar_init(&bars[k], 1);
      tc::fence_mbar_init();
    }
    if (threadIdx.x < 32) {
      tc::tmem_alloc(s_tmem, L::TMEM_COLS);
      tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    tmem = *s_tmem;
    if (threadIdx.x == 0) {   // the interpolation-matrix image, once per launch
      tc::mbar_arrive_expect_tx(&bars[3], L::IMG);
      tc::bulk_g2s(img, a.kimg, L::IMG, &bars[3]);
    }
    const bool ok = wait(&bars[3], 0, a.status);
    n_copy = 1;
    return ok;
  }
  // Releases the tensor memory once every MMA issued by this block has completed.
  __device__ void end(const CgIrArgs &a) {
    __syncthreads();
    if (threadIdx.x == 0) tc::mma_commit(&bars[0]);
    wait(&bars[0], n_mma & 1, a.status);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x < 32) tc::tmem_dealloc(tmem, L::TMEM_COLS);
  }

  // FP32 E-vector of M u for u = p_new = invdiag r + beta p (MODE 3, the inner
  // sweep) or u = d32 masked to the free DOFs (MODE 0).
  // pq: this thread's share of u . M u = sum_e sum_q mq (B u_e)_q^2, formed from the
  // interpolated values it scales (the GEMM1 output).
  template <int MODE>
  __device__ bool sweep(const CgIrArgs &a, float beta, float &pq) {
    const MeshDesc &m = a.mesh;
    const int rows_total = 3 * m.ne;
    const int ntiles = (rows_total + L::ROWS - 1) / L::ROWS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = warp & 3, cgrp = warp >> 2;   // tensor-memory lane quarter, column group 0..3
    const int r_own = quarter * 32 + lane;            // the tile row this thread reads back
    const uint32_t t_lane = (uint32_t)(quarter * 32) << 16;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int R0 = t * L::ROWS;
      const int e_lo = R0 / 3;
      const int e_hi = min(m.ne - 1, (R0 + L::ROWS - 1) / 3);
      if (threadIdx.x == 0) {   // this tile's mass data, by the bulk-copy engine
        const uint32_t bytes = (uint32_t)(e_hi - e_lo + 1) * (uint32_t)(NQ * 4);
        tc::fence_proxy_async();
        tc::mbar_arrive_expect_tx(&bars[3], bytes);
        tc::bulk_g2s(mqs, a.mq32 + (size_t)e_lo * NQ, bytes, &bars[3]);
      }
      const int ne_t = e_hi - e_lo + 1;   // elements of this tile (the first and last may be partial)
      if (threadIdx.x < ne_t) s_base[threadIdx.x] = h1_base<3, D>(m, e_lo + threadIdx.x);
      if (L::NKB * 64 > ND || R0 + L::ROWS > rows_total) {   // padding columns / rows must read as 0
        for (int k = threadIdx.x; k < L::A1 / 16; k += THREADS)
          reinterpret_cast<uint4 *>(areg)[k] = make_uint4(0u, 0u, 0u, 0u);
      }
      __syncthreads();
      // X = u at the tile's element nodes, gathered along mesh lines: a warp takes
      // one (component, iy, iz) line and its lanes walk the tile's elements and
      // their x-nodes, i.e. consecutive H1 nodes (one repeat per element face), so
      // the loads are coalesced; values go to the swizzled hi/lo blocks.
      {
        const int seg = ne_t * D;   // (element, ix) pairs of one line
        for (int line = warp; line < 3 * D * D; line += THREADS / 32) {
          const int c = line / (D * D), iy = line % D, iz = (line / D) % D;
          const int r_c = 3 * e_lo + c - R0;   // row of (e_lo, c); rows step by 3 per element
          const int goff = c * m.nh1 + m.n1x * (iy + m.n1y * iz);
          const int i_line = D * (iy + D * iz);
          constexpr int J = (L::MQ_E * D + 31) / 32;
          // every load is issued unconditionally (at a valid index) so that all of
          // a lane's loads are in flight together; invalid slots are zeroed after
          float v[J];
          {
            float ld0[J], ld1[J], ld2[J];
#pragma unroll
            for (int jj = 0; jj < J; ++jj) {
              const int k = lane + 32 * jj;
              const int el = k < seg ? k / D : 0, ix = k < seg ? k - (k / D) * D : 0;
              const int gi = goff + s_base[el] + ix;
              if constexpr (MODE == 0) {
                ld0[jj] = __ldg(a.invdiag32 + gi);
                ld1[jj] = a.d32[gi];
              } else {   // z = invdiag r is kept beside r by the node sweeps
                ld1[jj] = a.z32[gi];
                ld2[jj] = a.p32[gi];
              }
            }
#pragma unroll
            for (int jj = 0; jj < J; ++jj) {
              const int k = lane + 32 * jj;
              const int r = r_c + 3 * (k / D);
              float val;
              if constexpr (MODE == 0) val = ld0[jj] != 0.0f ? ld1[jj] : 0.0f;   // masked x
              else val = fmaf(beta, ld2[jj], ld1[jj]);                            // z + beta p
              v[jj] = (k < seg && r >= 0 && r < L::ROWS) ? val : 0.0f;
            }
          }
#pragma unroll
          for (int jj = 0; jj < J; ++jj) {
            const int k = lane + 32 * jj;
            const int el = k / D, ix = k - el * D;
            const int r = r_c + 3 * el;
            if (k < seg && r >= 0 && r < L::ROWS) {
              const int i = i_line + ix;
              const __nv_bfloat16 h = __float2bfloat16_rn(v[jj]);
              const __nv_bfloat16 l = __float2bfloat16_rn(v[jj] - __bfloat162float(h));
              const int off = (i >> 6) * L::A_BLOCK + L::sw128(r, i & 63);
              *reinterpret_cast<__nv_bfloat16 *>(areg + off) = h;
              *reinterpret_cast<__nv_bfloat16 *>(areg + L::NKB * L::A_BLOCK + off) = l;
            }
          }
        }
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();
      if (threadIdx.x == 0) {   // GEMM1: D1 = X K^T
        tc::fence_after_sync();
        const uint32_t a0 = tc::smem_u32(areg), b0 = tc::smem_u32(img);
#pragma unroll 1
        for (int ks = 0; ks < 4 * L::NKB; ++ks) {
          const uint32_t ao = (ks >> 2) * L::A_BLOCK + (ks & 3) * 32;
          const uint32_t bo = (ks >> 2) * L::IMG_BLOCK + (ks & 3) * 32;
          const uint64_t ah = tc::sdesc(a0 + ao, 16, 1024), al = tc::sdesc(a0 + L::NKB * L::A_BLOCK + ao, 16, 1024);
          const uint64_t bh = tc::sdesc(b0 + bo, 16, 1024), bl = tc::sdesc(b0 + L::IMG_HALF + bo, 16, 1024);
          const uint32_t d = tmem + L::D1_COL;
          tc::mma_bf16(d, ah, bh, IDESC1, ks > 0 ? 1u : 0u);
          tc::mma_bf16(d, ah, bl, IDESC1, 1u);
          tc::mma_bf16(d, al, bh, IDESC1, 1u);
        }
        tc::mma_commit(&bars[0]);
      }
      if (!wait(&bars[0], n_mma & 1, a.status)) return false;
      ++n_mma;
      if (!wait(&bars[3], n_copy & 1, a.status)) return false;
      ++n_copy;
      tc::fence_after_sync();
      // Z = Y .* mq per 64-wide q chunk into alternating buffers; GEMM2 of a
      // chunk runs while the next chunk is scaled
      const int R = R0 + r_own;
      const bool row_ok = R < rows_total;
      const float *mrow = reinterpret_cast<const float *>(mqs) + (size_t)(row_ok ? R / 3 - e_lo : 0) * NQ;
#pragma unroll 1
      for (int ch = 0; ch < L::NCH; ++ch) {
        const int q0 = ch * 64, W = min(64, L::N1 - q0), cw = W / 4;   // cw = 16 or 8 columns per warp
        const int b = ch & 1;
        if (ch >= 2 && !wait(&bars[1 + b], (n_buf[b] - 1) & 1, a.status)) return false;
        char *buf = areg + b * 2 * L::A_BLOCK;
        const int qc = q0 + cgrp * cw;   // first column (quadrature point) of this warp
        const uint32_t taddr = tmem + t_lane + (uint32_t)(L::D1_COL + qc);
        if (cw == 16) {
          float yv[16];
          tc::tmem_ld16(taddr, yv);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int q8 = qc + 8 * h;
            float z[8];
            if (row_ok && q8 < NQ) {
              const float4 m0 = *reinterpret_cast<const float4 *>(mrow + q8);
              const float4 m1 = *reinterpret_cast<const float4 *>(mrow + q8 + 4);
              z[0] = yv[8 * h + 0] * m0.x; z[1] = yv[8 * h + 1] * m0.y;
              z[2] = yv[8 * h + 2] * m0.z; z[3] = yv[8 * h + 3] * m0.w;
              z[4] = yv[8 * h + 4] * m1.x; z[5] = yv[8 * h + 5] * m1.y;
              z[6] = yv[8 * h + 6] * m1.z; z[7] = yv[8 * h + 7] * m1.w;
#pragma unroll
              for (int l = 0; l < 8; ++l) pq = fmaf(yv[8 * h + l], z[l], pq);
            } else {
#pragma unroll
              for (int l = 0; l < 8; ++l) z[l] = 0.0f;
            }
            uint4 hi, lo;
            tc::split8(z, hi, lo);
            const int off = L::sw128(r_own, cgrp * cw + 8 * h);
            *reinterpret_cast<uint4 *>(buf + off) = hi;
            *reinterpret_cast<uint4 *>(buf + L::A_BLOCK + off) = lo;
          }
        } else {
          float yv[8];
          tc::tmem_ld8(taddr, yv);
          float z[8];
          if (row_ok && qc < NQ) {
            const float4 m0 = *reinterpret_cast<const float4 *>(mrow + qc);
            const float4 m1 = *reinterpret_cast<const float4 *>(mrow + qc + 4);
            z[0] = yv[0] * m0.x; z[1] = yv[1] * m0.y; z[2] = yv[2] * m0.z; z[3] = yv[3] * m0.w;
            z[4] = yv[4] * m1.x; z[5] = yv[5] * m1.y; z[6] = yv[6] * m1.z; z[7] = yv[7] * m1.w;
#pragma unroll
            for (int l = 0; l < 8; ++l) pq = fmaf(yv[l], z[l], pq);
          } else {
#pragma unroll
            for (int l = 0; l < 8; ++l) z[l] = 0.0f;
          }
          uint4 hi, lo;
          tc::split8(z, hi, lo);
          const int off = L::sw128(r_own, cgrp * cw);
          *reinterpret_cast<uint4 *>(buf + off) = hi;
          *reinterpret_cast<uint4 *>(buf + L::A_BLOCK + off) = lo;
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (threadIdx.x == 0) {   // GEMM2 part: D2 += Z[:, chunk] K[chunk, :]
          tc::fence_after_sync();
          const uint32_t a0 = tc::smem_u32(buf), b0 = tc::smem_u32(img);
#pragma unroll 1
          for (int ks = 0; ks < W / 16; ++ks) {
            const int kq = ch * 4 + ks;   // 16-row group of q in the image
            const uint64_t ah = tc::sdesc(a0 + ks * 32, 16, 1024);
            const uint64_t al = tc::sdesc(a0 + L::A_BLOCK + ks * 32, 16, 1024);
            const uint64_t bh = tc::sdesc(b0 + kq * 2048, L::IMG_BLOCK, 1024);
            const uint64_t bl = tc::sdesc(b0 + L::IMG_HALF + kq * 2048, L::IMG_BLOCK, 1024);
            const uint32_t d = tmem + L::D2_COL;
            tc::mma_bf16(d, ah, bh, IDESC2, (ch > 0 || ks > 0) ? 1u : 0u);
            tc::mma_bf16(d, ah, bl, IDESC2, 1u);
            tc::mma_bf16(d, al, bh, IDESC2, 1u);
          }
          tc::mma_commit(&bars[1 + b]);
          if (ch == L::NCH - 1) tc::mma_commit(&bars[0]);
        }
        ++n_buf[b];
      }
      if (!wait(&bars[0], n_mma & 1, a.status)) return false;
      ++n_mma;
      tc::fence_after_sync();
      // W -> staging in shared memory (the operand buffers are free now) -> E-vector
      float *stg = reinterpret_cast<float *>(areg);
      constexpr int cw2 = L::N2 / 4;   // 32 or 16 columns per warp
#pragma unroll
      for (int h = 0; h < cw2 / 16; ++h) {
        const int i0 = cgrp * cw2 + 16 * h;
        float wv[16];
        tc::tmem_ld16(tmem + t_lane + (uint32_t)(L::D2_COL + i0), wv);
#pragma unroll
        for (int l = 0; l < 16; ++l)
          if (i0 + l < ND) stg[r_own * L::STG_LD + i0 + l] = wv[l];
      }
      __syncthreads();
      const int nrows = min(L::ROWS, rows_total - R0);
      float *dst = a.evec32 + (size_t)R0 * ND;
      for (int k = threadIdx.x; k < nrows * ND; k += THREADS) {
        const int rr = k / ND, ii = k - rr * ND;
        dst[k] = stg[rr * L::STG_LD + ii];
      }
      tc::fence_before_sync();
      __syncthreads();
    }
    return true;
  }
};

// Persistent cooperative solver of the precision form with the tensor-core
// inner sweep: one CTA per SM (shared memory), 512 threads.
template <int P, int Q>
__global__ void __launch_bounds__(512, 1) k_cg_tc(CgIrArgs a) {
  using L = TcLayout<P, Q>;
  using F = Family<3, P, Q>;
  extern __shared__ unsigned char tc_smem_raw[];
  char *base = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bars[4];
  __shared__ uint32_t s_tmem;
  __shared__ int s_base[L::ROWS];
  __shared__ int s_eb[F::NB_EB];
  TcMass<P, Q> tcm;
  const bool ok = tcm.begin(a, base, bars, &s_tmem, s_base);
  // FP64 refinement space: tables and one element batch over A region + mq tile
  double *st = reinterpret_cast<double *>(tcm.areg);
  double *u = st + F::TAB, *S = u + F::CXC * F::ND, *uq = S + F::MC_S, *y = uq + F::CXC * F::NQ;
  double *red = reinterpret_cast<double *>(tcm.mqs + L::MQB);
  if (ok)
    F::template cg_ir_core<true>(
        a, st, u, S, uq, y, red, s_eb, [&]() {}, [&](float beta, float &pq) { return tcm.template sweep<3>(a, beta, pq); });
  tcm.end(a);
}

// E-vector of M x with the tensor-core element operator, x = a.d32 masked to
// the free DOFs (a.invdiag32 != 0), into a.evec32; one CTA per SM, no grid sync.
template <int P, int Q>
__global__ void __launch_bounds__(512, 1) k_tc_apply(CgIrArgs a) {
  using L = TcLayout<P, Q>;
  extern __shared__ unsigned char tc_smem_raw[];
  char *base = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bars[4];
  __shared__ uint32_t s_tmem;
  __shared__ int s_base[L::ROWS];
  TcMass<P, Q> tcm;
  float unused = 0.0f;
  if (tcm.begin(a, base, bars, &s_tmem, s_base)) tcm.template sweep<0>(a, 0.0f, unused);
  tcm.end(a);
}

// FP32 node sum of a 3-component E-vector (the deterministic G^T).
template <int D>
__global__ void k_gather_f32(MeshDesc m, const float *__restrict__ evec, float *__restrict__ out) {
  const size_t n = (size_t)3 * m.nh1;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(k / m.nh1), g = (int)(k % m.nh1);
    out[k] = gather_node<3, D, float>(m, evec, 3, c, g);
  }
}

// Host: the shared-memory image of K (BF16 hi, then lo) from the 1D table
// B[q][i] (q1 x (p+1), row-major).
inline unsigned short host_bf16_rne(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return (unsigned short)(u >> 16);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (unsigned short)(u >> 16);
}
inline float host_bf16_to_float(unsigned short h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
template <int P, int Q>
void tc_build_image(const double *B, unsigned short *img) {
  using L = TcLayout<P, Q>;
  constexpr int D = L::D;
  std::memset(img, 0, L::IMG);
  for (int kb = 0; kb < L::NKB; ++kb)
    for (int q = 0; q < L::N1; ++q)
      for (int il = 0; il < 64; ++il) {
        const int i = kb * 64 + il;
        double v = 0.0;
        if (q < L::NQ && i < L::ND) {
          const int qx = q % Q, qy = (q / Q) % Q, qz = q / (Q * Q);
          const int ix = i % D, iy = (i / D) % D, iz = i / (D * D);
          v = B[qx * D + ix] * B[qy * D + iy] * B[qz * D + iz];
        }
        const unsigned short h = host_bf16_rne((float)v);
        const unsigned short l = host_bf16_rne((float)(v - (double)host_bf16_to_float(h)));
        const int off = kb * L::IMG_BLOCK + L::sw128(q, il);
        img[off / 2] = h;
        img[(L::IMG_HALF + off) / 2] = l;
      }
}

}  // namespace lh
