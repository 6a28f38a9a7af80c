// Learned form: a per-element MLP (mlp.cu) predicts the initial guess of the
// velocity mass solve from the three most recent mass-solve solutions and the
// element's Jacobian at its centroid. Supported for 3D Q3 (64 nodes x 3
// components = 192 outputs per element) with q1 = 6.
//
// Per solve of lh_rk2avg_step, with a_1, a_2, a_3 the three most recent solutions,
// s = RMS of a_1 and s_d = RMS of a_1 - a_2 over the free DOFs:
//   features  X_e = [a_1 / s, (a_1 - a_2) / s_d, (a_2 - a_3) / s_d at the element's
//             nodes] (576 values) ++ [J(centroid) / (h0 p), det J / (h0 p)^3] (10)
//   target    T_e = (a_new - a_1) / s_d at the element's nodes (recording mode)
//   guess     g = a_1 + s_d * (average over the elements sharing each node of the
//             MLP output), zero on constrained DOFs (prediction mode)
// Successive solutions differ by a small fraction of their size, so the history
// enters as normalised differences: raw solutions rounded to BF16 would lose it.
// In prediction mode the Jacobi-preconditioned residual norms (r, D^-1 r) of g and
// a_1 are compared and the smaller one's vector starts CG; the CG tolerance is
// unchanged, so the guess only changes the iteration count. The residual of g
// takes one FP32 mass action; that of a_1 needs none: the mass matrix does not
// change between solves (rho|J| = rho0|J0|) and a_1 solved the previous system to
// the CG tolerance, so b - M a_1 = (b - b_prev) + O(tol |b_prev|) with b_prev the
// previous right-hand side.
// Recording mode can keep every k-th element of each solve (a rotating subset:
// element e = o + j k with o = solve count mod k), so long runs on large meshes
// fit a bounded example buffer.
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "lh_kernels.cuh"
#include "lh_mlp.h"

using namespace lh;
using namespace lh::mlp;

namespace lh {
__nv_bfloat16 *mlp_packed_input(lh_mlp *m, int *max_rows);
lh_status mlp_forward_packed(lh_mlp *m, int n, float *Y, cudaStream_t s);
}  // namespace lh

namespace lh {
namespace learn {
namespace {

using F = Family<3, 3, 6>;
constexpr int D = 4, ND = 64;
constexpr int kBlocks = 592;

struct Cent { double v[4], d[4]; };   // 1D basis values / derivatives at the centre 0.5

__global__ void k_sumsq(size_t nv, const double *__restrict__ a1, const double *__restrict__ a2,
                        const double *__restrict__ idg, double *__restrict__ part) {
  double v[3] = {0.0, 0.0, 0.0};
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < nv; k += (size_t)gridDim.x * blockDim.x)
    if (idg[k] != 0.0) {
      const double d = a1[k] - a2[k];
      v[0] = fma(a1[k], a1[k], v[0]);
      v[1] = fma(d, d, v[1]);
      v[2] += 1.0;
    }
  __shared__ double red[96];
  block_sum<3>(v, red);
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) part[3 * blockIdx.x + q] = v[q];
}
// s[0] = RMS of a_1, s[1] = RMS of a_1 - a_2 (1 where zero)
__global__ void k_scale_final(int nb, const double *__restrict__ part, double *__restrict__ s) {
  if (threadIdx.x < 32) {
    double a = 0.0, d = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < nb; i += 32) { a += part[3 * i]; d += part[3 * i + 1]; c += part[3 * i + 2]; }
    a = warp_sum(a);
    d = warp_sum(d);
    c = warp_sum(c);
    if (threadIdx.x == 0) {
      const double ra = c > 0.0 ? sqrt(a / c) : 0.0, rd = c > 0.0 ? sqrt(d / c) : 0.0;
      s[0] = ra > 0.0 ? ra : 1.0;
      s[1] = rd > 0.0 ? rd : 1.0;
    }
  }
}

// History features: X[e][c*64 + i] = a_1 / s, X[e][192 + c*64 + i] = (a_1 - a_2) / s_d,
// X[e][384 + c*64 + i] = (a_2 - a_3) / s_d at node(e, i), component c.
// Row r of X holds element e = off + r * stride (stride 1, off 0: every element).
// One thread per (row, element node): the node's index is formed once and its three
// components of the three history vectors give nine features. OT = float: rows of
// kIn floats (recorded training data); OT = BF16: straight into the network's packed
// input, rows of ldx values (the value is the float feature rounded to nearest, the
// same as packing the float rows).
__device__ __forceinline__ void put_feature(float *p, float v) { *p = v; }
__device__ __forceinline__ void put_feature(__nv_bfloat16 *p, float v) { *p = __float2bfloat16(v); }

template <typename OT>
__global__ void k_hist_features(MeshDesc m, int rows, int stride, int off, const double *__restrict__ h0,
                                const double *__restrict__ h1, const double *__restrict__ h2,
                                const double *__restrict__ s, OT *__restrict__ X, int ldx) {
  const size_t total = (size_t)rows * ND;
  // the differences are formed in FP64 (consecutive solutions can agree to many
  // digits), the scalings in FP32: the features feed a BF16 network, and FP64
  // multiplies run at 1/64 of the FP32 rate on this part
  const float is = (float)(1.0 / s[0]), isd = (float)(1.0 / s[1]);
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / ND), i = (int)(t % ND);
    const int e = off + r * stride;
    const size_t g = (size_t)h1_base<3, D>(m, e) + h1_local<3, D>(m, i);
    OT *xr = X + (size_t)r * ldx;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t gi = (size_t)c * m.nh1 + g;
      const double a0 = h0[gi], a1 = h1[gi], a2 = h2[gi];
      put_feature(xr + c * ND + i, (float)a0 * is);
      put_feature(xr + 192 + c * ND + i, (float)(a0 - a1) * isd);
      put_feature(xr + 384 + c * ND + i, (float)(a1 - a2) * isd);
    }
  }
}

// Jacobian features at the element centroid: 9 entries of J / (h0 p) and det J / (h0 p)^3.
template <typename OT>
__global__ void k_jac_features(MeshDesc m, int rows, int stride, int off, const double *__restrict__ x, Cent cb,
                               double hs, OT *__restrict__ X, int ldx) {
  // FP32 arithmetic (the features feed a BF16 network); positions are taken relative
  // to the element's first node, which leaves J unchanged (the basis derivatives sum
  // to zero) and avoids cancellation between O(1) coordinates
  float cv[D], cd[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    cv[k] = (float)cb.v[k];
    cd[k] = (float)cb.d[k];
  }
  const float ihs = (float)(1.0 / hs);
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    const int e = off + r * stride;
    const int base = h1_base<3, D>(m, e);
    double x0[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) x0[c] = x[(size_t)c * m.nh1 + base];
    float J[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < ND; ++i) {
      const int ix = i % D, iy = (i / D) % D, iz = i / (D * D);
      const float gx = cd[ix] * cv[iy] * cv[iz];
      const float gy = cv[ix] * cd[iy] * cv[iz];
      const float gz = cv[ix] * cv[iy] * cd[iz];
      const int g = base + h1_local<3, D>(m, i);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float xc = (float)(x[(size_t)c * m.nh1 + g] - x0[c]) * ihs;
        J[c * 3 + 0] = fmaf(xc, gx, J[c * 3 + 0]);
        J[c * 3 + 1] = fmaf(xc, gy, J[c * 3 + 1]);
        J[c * 3 + 2] = fmaf(xc, gz, J[c * 3 + 2]);
      }
    }
    const float det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                      J[2] * (J[3] * J[7] - J[4] * J[6]);
    OT *out = X + (size_t)r * ldx + 576;
    for (int k = 0; k < 9; ++k) put_feature(out + k, J[k]);
    put_feature(out + 9, det);
  }
}

// Targets: T[e][c*64 + i] = (a_new - a_1)[c][node(e,i)] / s_d.
__global__ void k_targets(MeshDesc m, int rows, int stride, int off, const double *__restrict__ anew,
                          const double *__restrict__ a1, const double *__restrict__ s, float *__restrict__ T) {
  const size_t total = (size_t)rows * kOut;
  const double is = 1.0 / s[1];
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / kOut), f = (int)(t % kOut);
    const int e = off + r * stride;
    const int c = f / 64, i = f % 64;
    const size_t k = (size_t)c * m.nh1 + h1_base<3, D>(m, e) + h1_local<3, D>(m, i);
    T[t] = (float)((anew[k] - a1[k]) * is);
  }
}

// Guess at nodes: g = a_1 + s_d * mean over element copies of the MLP output; 0 on constrained DOFs.
__global__ void k_assemble(MeshDesc m, const float *__restrict__ Y, const double *__restrict__ a1,
                           const double *__restrict__ s, const double *__restrict__ idg, double *__restrict__ g) {
  const double sc = s[1];
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < m.nh1; n += gridDim.x * blockDim.x) {
    int off[8];
    const int cnt = node_copies<3, D>(m, n, 3, off);
    // cnt = 1, 2, 4 or 8 (one or two owners per axis): dividing by it is the exact
    // scaling by 2^-log2(cnt), done here without an FP64 division
    const double icnt = __hiloint2double((1023 - (__ffs(cnt) - 1)) << 20, 0);
    for (int c = 0; c < 3; ++c) {
      const size_t k = (size_t)c * m.nh1 + n;
      double sum = 0.0;
      for (int j = 0; j < cnt; ++j) sum += (double)Y[off[j] + c * ND];
      g[k] = idg[k] != 0.0 ? fma(sc, sum * icnt, a1[k]) : 0.0;
    }
  }
}

// FP32 E-vector of M g for the residual comparison: kResidNb elements per CTA (one
// element per CTA left most of each 224-thread block idle at 216 qpoints).
constexpr int kResidNb = 8, kResidCx = 3 * kResidNb, kResidThreads = 256;
constexpr int kResidS = interp_scratch<3, D, 6>(kResidCx) > interp_scratch<3, 6, D>(kResidCx)
                            ? interp_scratch<3, D, 6>(kResidCx) : interp_scratch<3, 6, D>(kResidCx);
constexpr size_t kResidSmem = sizeof(float) * (2 * 6 * D + kResidCx * ND + kResidS + kResidCx * 216 + kResidCx * ND);
__global__ void __launch_bounds__(kResidThreads) k_resid_elem(MeshDesc m, const double *__restrict__ tab,
                                                              const float *__restrict__ mq32,
                                                              const double *__restrict__ g, float *__restrict__ evA) {
  constexpr int CX = kResidCx, NQ = 216, Q = 6;
  extern __shared__ double smd[];
  float *tb = (float *)smd, *tbt = tb + Q * D, *u = tbt + Q * D, *S = u + CX * ND, *uq = S + kResidS, *y = uq + CX * NQ;
  for (int k = threadIdx.x; k < 2 * Q * D; k += blockDim.x) tb[k] = (float)tab[k < Q * D ? F::oB + k : F::oBt + k - Q * D];
  const int e0 = blockIdx.x * kResidNb, nb = min(kResidNb, m.ne - e0);
  for (int k = threadIdx.x; k < CX * ND; k += blockDim.x) {
    const int i = k % ND, bc = k / ND, c = bc % 3, b = bc / 3;
    float val = 0.0f;
    if (b < nb) {
      const size_t gi = (size_t)c * m.nh1 + h1_base<3, D>(m, e0 + b) + h1_local<3, D>(m, i);
      val = (float)g[gi];   // k_assemble leaves g = 0 on the constrained DOFs
    }
    u[k] = val;
  }
  __syncthreads();
  interp_p<3, D, Q, CX>(u, uq, S, tb);   // pencil form: FP32 work is cheap, smem traffic is not
  for (int k = threadIdx.x; k < CX * NQ; k += blockDim.x) {
    const int q = k % NQ, b = (k / NQ) / 3;
    uq[k] *= b < nb ? mq32[(size_t)(e0 + b) * NQ + q] : 0.0f;
  }
  __syncthreads();
  interp_p<3, Q, D, CX>(uq, y, S, tbt);
  for (int k = threadIdx.x; k < nb * 3 * ND; k += blockDim.x) evA[(size_t)e0 * 3 * ND + k] = y[k];
}

// Preconditioned residual norms (r, D^-1 r) -- the quantity Jacobi-PCG itself
// reduces -- of both candidates as per-block partials: r_g = b - M g (FP32 action,
// FP64 sums) and r_1 = b - b_prev for the previous solution a_1.
__global__ void k_resid_nodes(MeshDesc m, const double *__restrict__ b, const double *__restrict__ bprev,
                              const double *__restrict__ idg, const float *__restrict__ evA,
                              double *__restrict__ part) {
  double acc[2] = {0.0, 0.0};
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < m.nh1; n += gridDim.x * blockDim.x) {
    int off[8];
    const int cnt = node_copies<3, D>(m, n, 3, off);
    for (int c = 0; c < 3; ++c) {
      const size_t k = (size_t)c * m.nh1 + n;
      if (idg[k] == 0.0) continue;
      float ma = 0.0f;
      for (int j = 0; j < cnt; ++j) ma += evA[off[j] + c * ND];
      const double ra = b[k] - (double)ma, rb = b[k] - bprev[k];
      acc[0] = fma(ra * idg[k], ra, acc[0]);
      acc[1] = fma(rb * idg[k], rb, acc[1]);
    }
  }
  __shared__ double red[64];
  block_sum<2>(acc, red);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = acc[0]; part[2 * blockIdx.x + 1] = acc[1]; }
}

// Decide (one warp) and count: flag = (r_g, D^-1 r_g) < (r_1, D^-1 r_1).
__global__ void k_decide(int nb, const double *__restrict__ part, int *__restrict__ flag, int *__restrict__ used,
                         double *__restrict__ ratio_sum) {
  if (threadIdx.x < 32) {
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += 32) { a += part[2 * i]; b += part[2 * i + 1]; }
    a = warp_sum(a);
    b = warp_sum(b);
    if (threadIdx.x == 0) {
      const int f = a < b ? 1 : 0;
      *flag = f;
      *used += f;
      *ratio_sum += b > 0.0 ? sqrt(a / b) : 1.0;
    }
  }
}

__global__ void k_to_f32(size_t n, const double *__restrict__ a, float *__restrict__ b) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    b[k] = (float)a[k];
}

__global__ void k_apply(size_t nv, const int *__restrict__ flag, const double *__restrict__ g, double *__restrict__ a) {
  if (!*flag) return;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < nv; k += (size_t)gridDim.x * blockDim.x)
    a[k] = g[k];
}

}  // namespace
}  // namespace learn
}  // namespace lh

struct lh_learn {
  lh_mlp *mlp = nullptr;
  int mode = 0;              // 1 record, 2 predict
  char *arena = nullptr;
  double *hist[3] = {nullptr, nullptr, nullptr};
  int count = 0, head = 0;   // solutions stored, next ring slot
  float *Y = nullptr, *evA32 = nullptr;
  double *bprev = nullptr;   // right-hand side of the previous solve
  int stride = 1;            // recording: every stride-th element of a solve
  float *mq32 = nullptr;     // FP32 mass data for the residual check (own copy for FP64 contexts)
  double *guess = nullptr, *scale = nullptr, *part = nullptr, *ratio = nullptr;
  int *flag = nullptr, *used = nullptr;
  float *dX = nullptr, *dT = nullptr;
  int capacity = 0, rows = 0, solves = 0, predicted = 0;
  bool pending = false;      // features of the current solve were recorded
  int pend_rows = 0, pend_off = 0;
  size_t smem_resid = 0;
  learn::Cent cent{};
  double hs = 1.0;
};

namespace lh {

static const double *hist_at(lh_learn *L, int age) {   // age 0 = most recent
  return L->hist[(L->head + 2 - age + 3) % 3];
}

// Before a mass solve of lh_rk2avg_step (positions x of the stage, rhs in c->rhs).
lh_status learn_before_solve(lh_ctx *c, const double *x, cudaStream_t s) {
  lh_learn *L = c->learn;
  if (!L || L->mode == 0 || L->count < 3) return LH_OK;
  using namespace learn;
  const MeshDesc &m = c->mesh;
  const size_t nv = c->nv;
  const double *a1 = hist_at(L, 0);
  k_sumsq<<<kBlocks, 256, 0, s>>>(nv, a1, hist_at(L, 1), c->invdiag, L->part);
  k_scale_final<<<1, 32, 0, s>>>(kBlocks, L->part, L->scale);
  float *X = nullptr;   // recording: this solve's rows of the caller's buffer
  L->pending = false;
  int rows = m.ne, stride = 1, off = 0;
  if (L->mode == 1) {
    stride = L->stride;
    off = L->solves % stride;
    rows = off < m.ne ? (m.ne - off + stride - 1) / stride : 0;
    if (rows == 0 || L->rows + rows > L->capacity) return LH_OK;
    X = L->dX + (size_t)L->rows * kIn;
    L->pending = true;
    L->pend_rows = rows;
    L->pend_off = off;
  }
  if (L->mode == 1) {
    k_hist_features<<<4 * kBlocks, 256, 0, s>>>(m, rows, stride, off, a1, hist_at(L, 1), hist_at(L, 2), L->scale,
                                                X, kIn);
    k_jac_features<<<(rows + 255) / 256, 256, 0, s>>>(m, rows, stride, off, x, L->cent, L->hs, X, kIn);
  } else {
    // prediction: the features go straight into the network's packed BF16 input
    int cap = 0;
    __nv_bfloat16 *Xh = mlp_packed_input(L->mlp, &cap);
    if (!Xh || m.ne > cap) {
      c->err = "learned guess: the MLP was created for fewer rows than the mesh has elements";
      return LH_ERR_ARG;
    }
    k_hist_features<<<4 * kBlocks, 256, 0, s>>>(m, rows, stride, off, a1, hist_at(L, 1), hist_at(L, 2), L->scale,
                                                Xh, kInPad);
    k_jac_features<<<(rows + 255) / 256, 256, 0, s>>>(m, rows, stride, off, x, L->cent, L->hs, Xh, kInPad);
  }
  if (L->mode == 2) {
    if (lh_status st = mlp_forward_packed(L->mlp, m.ne, L->Y, s)) return st;
    k_assemble<<<2 * kBlocks, 256, 0, s>>>(m, L->Y, a1, L->scale, c->invdiag, L->guess);
    k_resid_elem<<<(m.ne + kResidNb - 1) / kResidNb, kResidThreads, L->smem_resid, s>>>(m, c->tab, L->mq32,
                                                                                         L->guess, L->evA32);
    k_resid_nodes<<<kBlocks, 256, 0, s>>>(m, c->rhs, L->bprev, c->invdiag, L->evA32, L->part);
    k_decide<<<1, 32, 0, s>>>(kBlocks, L->part, L->flag, L->used, L->ratio);
    k_apply<<<kBlocks, 256, 0, s>>>(nv, L->flag, L->guess, c->a_prev);
    L->predicted += 1;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    c->err = std::string("learned guess: ") + cudaGetErrorString(e);
    return LH_ERR_CUDA;
  }
  return LH_OK;
}

// After a mass solve: record the target (recording mode) and push the solution into the history.
lh_status learn_after_solve(lh_ctx *c, cudaStream_t s) {
  lh_learn *L = c->learn;
  if (!L || L->mode == 0) return LH_OK;
  using namespace learn;
  if (L->mode == 1 && L->pending) {
    k_targets<<<4 * kBlocks, 256, 0, s>>>(c->mesh, L->pend_rows, L->stride, L->pend_off, c->a_prev,
                                          hist_at(L, 0), L->scale, L->dT + (size_t)L->rows * kOut);
    L->rows += L->pend_rows;
    L->pending = false;
  }
  cudaMemcpyAsync(L->hist[L->head], c->a_prev, c->nv * sizeof(double), cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(L->bprev, c->rhs, c->nv * sizeof(double), cudaMemcpyDeviceToDevice, s);
  L->head = (L->head + 1) % 3;
  L->count = L->count < 3 ? L->count + 1 : 3;
  L->solves += 1;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    c->err = std::string("learned history: ") + cudaGetErrorString(e);
    return LH_ERR_CUDA;
  }
  return LH_OK;
}

void learn_free(lh_learn *L) {
  if (!L) return;
  if (L->arena) cudaFree(L->arena);
  delete L;
}

}  // namespace lh

extern "C" {

lh_status lh_learn_attach(lh_ctx *c, lh_mlp *mlp, int mode, float *X_buf, float *T_buf, int capacity_rows) {
  if (!c) return LH_ERR_ARG;
  if (mode == 0) {
    learn_free(c->learn);
    c->learn = nullptr;
    return LH_OK;
  }
  if (c->dim != 3 || c->p != 3 || c->q1 != 6) {
    c->err = "the learned guess is defined for 3D Q3 with q1 = 6";
    return LH_ERR_UNSUPPORTED;
  }
  if (mode == 1 && (!X_buf || !T_buf || capacity_rows < 1)) {
    c->err = "recording needs example buffers";
    return LH_ERR_ARG;
  }
  if (mode == 2 && !mlp) {
    c->err = "prediction needs an MLP";
    return LH_ERR_ARG;
  }
  if (mode != 1 && mode != 2) { c->err = "mode must be 0, 1 or 2"; return LH_ERR_ARG; }
  learn_free(c->learn);
  c->learn = nullptr;
  lh_learn *L = new lh_learn();
  L->mlp = mlp;
  L->mode = mode;
  L->dX = X_buf;
  L->dT = T_buf;
  L->capacity = capacity_rows;
  const size_t nv = c->nv, ne = c->mesh.ne;
  const bool own_mq32 = c->mq32 == nullptr;
  const size_t nq = ne * (size_t)c->nq;
  const size_t bytes_list[] = {3 * nv * 8, 0, ne * lh::mlp::kOut * 4, ne * 3 * 64 * 4,
                               nv * 8, nv * 8, 4 * 1184 * 8 + 1024, own_mq32 ? nq * 4 : 0};
  size_t bytes = 0;
  for (size_t b : bytes_list) bytes += (b + 255) / 256 * 256;
  if (cudaMalloc(&L->arena, bytes) != cudaSuccess) {
    delete L;
    c->err = "learned-form buffers could not be allocated";
    return LH_ERR_OOM;
  }
  cudaMemset(L->arena, 0, bytes);
  char *p = L->arena;
  auto take = [&](size_t b) { char *q = p; p += (b + 255) / 256 * 256; return q; };
  double *h = (double *)take(bytes_list[0]);
  for (int k = 0; k < 3; ++k) L->hist[k] = h + k * nv;
  L->Y = (float *)take(bytes_list[2]);
  L->evA32 = (float *)take(bytes_list[3]);
  L->bprev = (double *)take(bytes_list[4]);
  L->guess = (double *)take(bytes_list[5]);
  char *misc = take(bytes_list[6]);
  L->mq32 = own_mq32 ? (float *)take(bytes_list[7]) : c->mq32;
  L->part = (double *)misc;
  L->scale = (double *)(misc + 4 * 1184 * 8);
  L->ratio = L->scale + 2;
  L->flag = (int *)(L->scale + 3);
  L->used = L->flag + 1;
  lh::h1_basis_at(3, 0.5, L->cent.v, L->cent.d);
  L->hs = c->h0 * c->p;
  const size_t smem = lh::learn::kResidSmem + 16;
  cudaFuncSetAttribute((const void *)lh::learn::k_resid_elem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  L->smem_resid = smem;
  if (own_mq32) lh::learn::k_to_f32<<<1024, 256>>>(nq, c->mq, L->mq32);
  c->learn = L;
  return cudaDeviceSynchronize() == cudaSuccess ? LH_OK : LH_ERR_CUDA;
}

lh_status lh_learn_set_record_stride(lh_ctx *c, int stride) {
  if (!c || !c->learn || stride < 1) return LH_ERR_ARG;
  c->learn->stride = stride;
  return LH_OK;
}

lh_status lh_learn_stats(const lh_ctx *c, int *rows_recorded, int *solves, int *predictions, int *learned_used,
                         double *mean_ratio) {
  if (!c || !c->learn) return LH_ERR_ARG;
  const lh_learn *L = c->learn;
  if (rows_recorded) *rows_recorded = L->rows;
  if (solves) *solves = L->solves;
  if (predictions) *predictions = L->predicted;
  if (learned_used) {
    if (cudaMemcpy(learned_used, L->used, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LH_ERR_CUDA;
  }
  if (mean_ratio) {
    double sum = 0.0;
    if (cudaMemcpy(&sum, L->ratio, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return LH_ERR_CUDA;
    *mean_ratio = L->predicted > 0 ? sum / L->predicted : 0.0;
  }
  return LH_OK;
}

}  // extern "C"
