// Batching form: many independent 2D problems of uneven order (p = 1..4,
// q1 = 2p) and mesh size advanced together. Each stage of an RK2-average step
// is three persistent launches over all problems: (1) the element pass of the
// quadrature data fused with F.1 (both element-local), (2) one cooperative
// launch that gathers the right-hand side, runs every problem's mass solve with
// its own scalars and convergence test, and applies the stage's node update,
// (3) the element pass of F^T v with the energy update. Work items (problem,
// first element, batch count) are sorted by order and dispatch to the compiled
// kernel family of their order. The whole step (six launches) is captured once
// into a CUDA graph and replayed. The tile shapes -- element batches per work
// item for the element passes and for the solver, per order, and the threads
// per block of the element passes (threads sharing one element's quadrature
// slab) -- are picked by an autotuner that times whole steps. Each problem
// keeps its own lh_ctx for set-up and buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "lh_kernels.cuh"

namespace lh {
namespace {

template <int P>
using F2 = Family<2, P, 2 * P>;

struct ItemE {      // element work item
  int pid, e0, nbat, order;   // nbat consecutive batches of the family's NB (or NBC) elements
};
struct ItemN {      // node work item: scalar H1 nodes [g0, g1) of problem pid
  int pid, g0, g1, k;   // k = index of this item among the problem's node items
};

struct BProb {      // per-problem record used by node kernels and the batched solver
  MeshDesc m;
  int order, n_nitems, first_nitem, source;
  int n_eitems, first_eitem;             // the problem's solver element items (set with the tiles)
  const double *tab, *mq, *invdiag, *dt;
  const int *ncopy;                      // the problem's node-copy table [N_H1][4]
  double *evec, *r, *p, *ap, *a, *rhs;   // a = acceleration (CG solution, warm start)
  double *x, *v, *e, *xh, *vh, *vb;
  lh_step_info *info;
};

struct BScal {      // per-problem CG scalars (device)
  double bb, rr, rz, rz_old, alpha, beta;
  int it, active, status, pad;
  unsigned int cnt, pad2;
};

constexpr int kThreads = 256;        // element kernels of all 2D families
constexpr int kThreadsCG = 512;      // batched solver CTAs
constexpr int kNodeItem = 2048;      // nodes per node work item (four per solver thread)

static_assert(F2<1>::THREADS == kThreads && F2<2>::THREADS == kThreads && F2<3>::THREADS == kThreads &&
                  F2<4>::THREADS == kThreads, "2D families must share the element block size");
static_assert(F2<1>::TC == kThreadsCG && F2<4>::TC == kThreadsCG, "2D families must share the solver block size");

template <typename F>
__device__ __forceinline__ void dispatch_order(int order, F &&f) {
  switch (order) {
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    default: f(std::integral_constant<int, 4>{}); break;
  }
}

// ---- batched element kernels (one launch for all problems) ----------------
// The element bodies stride every loop by blockDim.x, so any block size gives
// the same per-value arithmetic: TPB only sets how many threads share the
// quadrature points of a tile (the autotuner's second axis).
template <int TPB>
__global__ void __launch_bounds__(TPB) k_b_qf(const QdataArgs *qa, const ForceArgs *fa, const ItemE *items,
                                              int nitems) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const ItemE w = items[it];
    dispatch_order(w.order, [&](auto P) {
      using F = F2<decltype(P)::value>;
      for (int b = 0; b < w.nbat; ++b) {
        F::body_qdata(qa[w.pid], w.e0 + b * F::NB);   // D of these elements ...
        __syncthreads();
        F::body_force(fa[w.pid], w.e0 + b * F::NB);   // ... is all F.1 of them needs
        __syncthreads();
      }
    });
  }
}

template <int TPB>
__global__ void __launch_bounds__(TPB) k_b_force_t(const ForceTArgs *args, const ItemE *items, int nitems) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const ItemE w = items[it];
    dispatch_order(w.order, [&](auto P) {
      using F = F2<decltype(P)::value>;
      for (int b = 0; b < w.nbat; ++b) {
        F::body_force_t(args[w.pid], w.e0 + b * F::NB);
        __syncthreads();
      }
    });
  }
}

// Copies of node g from the problem's node-copy table (the -1 padding comes last, so
// the first n entries are the copies in the fixed gather order); returns n.
__device__ __forceinline__ int table_copies(const int *__restrict__ tab, int g, int (&off)[4]) {
  const int4 t = __ldg(reinterpret_cast<const int4 *>(tab + (size_t)g * 4));
  off[0] = t.x; off[1] = t.y; off[2] = t.z; off[3] = t.w;
  return (t.x >= 0) + (t.y >= 0) + (t.z >= 0) + (t.w >= 0);
}

// ---- node phases of the batched solver launch (one thread per scalar node) --
// rhs = -(F.1) gathered from the E-vector, zero on constrained DOFs.
__device__ __forceinline__ void node_rhs(const BProb &pb, const ItemN &w) {
  dispatch_order(pb.order, [&](auto P) {
    constexpr int D = decltype(P)::value + 1, ND = D * D;
    for (int g = w.g0 + threadIdx.x; g < w.g1; g += blockDim.x) {
      int off[4];
      const int n = table_copies(pb.ncopy, g, off);
      for (int c = 0; c < 2; ++c) {
        const int k = c * pb.m.nh1 + g;
        double s = pb.evec[off[0] + c * ND];
        for (int j = 1; j < n; ++j) s += pb.evec[off[j] + c * ND];
        pb.rhs[k] = pb.invdiag[k] != 0.0 ? -s : 0.0;
      }
    }
  });
}

// Stage-1 update: vb0 = v + dt/2 a0, v_h = vb0, x_h = x + dt/2 vb0.
__device__ __forceinline__ void node_mid(const BProb &pb, const ItemN &w) {
  const double hdt = 0.5 * *pb.dt;
  for (int g = w.g0 + threadIdx.x; g < w.g1; g += blockDim.x) {
    for (int c = 0; c < 2; ++c) {
      const int k = c * pb.m.nh1 + g;
      const double vb = fma(hdt, pb.a[k], pb.v[k]);
      pb.vh[k] = vb;
      pb.xh[k] = fma(hdt, vb, pb.x[k]);
    }
  }
}

// Final update: vb = v + dt/2 a, x += dt vb, v += dt a; node item 0 of a problem
// also advances its step record.
__device__ __forceinline__ void node_final(const BProb &pb, const ItemN &w) {
  const double dt = *pb.dt, hdt = 0.5 * dt;
  for (int g = w.g0 + threadIdx.x; g < w.g1; g += blockDim.x) {
    for (int c = 0; c < 2; ++c) {
      const int k = c * pb.m.nh1 + g;
      const double ak = pb.a[k], vk = pb.v[k];
      const double vb = fma(hdt, ak, vk);
      pb.vb[k] = vb;
      pb.x[k] = fma(dt, vb, pb.x[k]);
      pb.v[k] = fma(dt, ak, vk);
    }
  }
  if (w.k == 0 && threadIdx.x == 0 && pb.info) {
    pb.info->dt = dt;
    pb.info->t += dt;
    pb.info->steps += 1;
  }
}

// ---- batched persistent Jacobi PCG -----------------------------------------
struct BCgArgs {
  const BProb *probs;
  BScal *scal;
  const ItemE *items_e;   // batches of the solver's NBC elements
  int nitems_e;
  const ItemN *items_n;
  int nitems_n, nprob;
  double *partials;       // [nitems_n][3]
  double *partials_e;     // [nitems_e]: per solver element item
  int *active;            // number of problems still iterating
  GridBarrier *bar;       // this launch's barrier (zero at launch)
  GridBarrier *bar_next;  // the next launch's barrier, zeroed at the end of this one
  int *status;
  int stage;              // 0 or 1: which cg_iters slot of the step records and which update
  double tol;
  int max_it;
};

template <int P>
// E-vector of M u for one batch of the problem's elements (mode 0: u = a masked to
// the free DOFs; mode 1: u = p_new = D^-1 r + beta p); returns this thread's share of
// u . M u summed element by element (the search direction's energy p_new^T M p_new).
__device__ __forceinline__ double b_cg_matvec(const BProb &pb, int e0, int mode, double beta, double *sm) {
  using F = F2<P>;
  constexpr int ND = F::ND, NQ = F::NQ, CXC = F::CXC;
  double *st = sm, *u = st + F::TAB, *S = u + CXC * ND, *uq = S + F::MC_S, *y = uq + CXC * NQ;
  __shared__ int s_eb[F2<1>::NBC];
  const MeshDesc &m = pb.m;
  const int nb = min(F::NBC, m.ne - e0);
  double mqr[F::MQT_C];   // mass data first: the loads overlap the gather below
  F::template load_mq<double>(pb.mq, e0, nb, mqr);
  for (int k = threadIdx.x; k < F::oZ + F::D; k += blockDim.x) st[k] = pb.tab[k];
  if (threadIdx.x < nb) s_eb[threadIdx.x] = h1_base<2, F::D>(m, e0 + threadIdx.x);
  __syncthreads();
  for (int k = threadIdx.x; k < CXC * ND; k += blockDim.x) {
    const int i = k % ND, bc = k / ND, c = bc % 2, b = bc / 2;
    double val = 0.0;
    if (b < nb) {
      const int gi = c * m.nh1 + s_eb[b] + h1_local<2, F::D>(m, i);
      const double idg = pb.invdiag[gi];
      val = mode == 0 ? (idg != 0.0 ? pb.a[gi] : 0.0) : fma(beta, pb.p[gi], idg * pb.r[gi]);
    }
    u[k] = val;
  }
  __syncthreads();
  F::template batch_matvec_r<double>(st + F::oB, st + F::oBt, u, S, uq, y, mqr);
  double d = 0.0;
  for (int k = threadIdx.x; k < nb * 2 * ND; k += blockDim.x) {
    const double yk = y[k];
    pb.evec[(size_t)e0 * 2 * ND + k] = yk;
    d = fma(u[k], yk, d);
  }
  __syncthreads();
  return d;
}

// Deterministic per-problem reduction of node-item partials: the last item of
// a problem to finish sums all of them in item order. Returns true in that block.
__device__ __forceinline__ bool last_item(BScal &sc, int nitems) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&sc.cnt, 1u) == (unsigned)(nitems - 1);
  }
  __syncthreads();
  return s_last != 0;
}

__device__ __forceinline__ void sum_item_partials(const double *partials, int first, int n, int nv, double *out) {
  if (threadIdx.x < 32) {
    __threadfence();
    for (int q = 0; q < nv; ++q) {
      double s = 0.0;
      for (int i = threadIdx.x; i < n; i += 32) s += ((volatile const double *)partials)[(size_t)(first + i) * 3 + q];
      s = warp_sum(s);
      if (threadIdx.x == 0) out[q] = s;
    }
  }
  __syncthreads();
}

// One stage's solver launch: right-hand sides, then per problem the standard
// Jacobi-PCG recurrences with two grid barriers per iteration (p_new^T M p_new is
// summed element by element in the element sweep, so alpha is known after the first
// barrier and one node sweep updates p, a, r and forms r.r, r.z), then the stage's
// node update.
__global__ void __launch_bounds__(kThreadsCG) k_b_cg(BCgArgs A) {
  extern __shared__ double sm[];
  __shared__ double red[32 * 3];
  __shared__ double s_v[3];
  const int G = gridDim.x;
  unsigned long long nbar = 0;
  auto sync = [&]() { ++nbar; return grid_sync(A.bar, nbar * (unsigned long long)G, A.status); };
  const double tol2 = A.tol * A.tol;

  // ---- right-hand side: rhs = -(F.1) from the force pass's E-vector (read
  // before the matvec below overwrites it); the solver count starts at zero
  if (blockIdx.x == 0 && threadIdx.x == 0) *A.active = 0;
  for (int it = blockIdx.x; it < A.nitems_n; it += G) {
    const ItemN w = A.items_n[it];
    node_rhs(A.probs[w.pid], w);
  }
  if (!sync()) return;
  // ---- init: E-vector of M a (a masked)
  for (int it = blockIdx.x; it < A.nitems_e; it += G) {
    const ItemE w = A.items_e[it];
    const BProb &pb = A.probs[w.pid];
    dispatch_order(w.order, [&](auto P) {
      for (int b = 0; b < w.nbat; ++b) b_cg_matvec<decltype(P)::value>(pb, w.e0 + b * F2<decltype(P)::value>::NBC, 0, 0.0, sm);
    });
  }
  if (!sync()) return;
  // r = b - A a, p = q = 0; partials b.b, r.r, r.z; per-problem reduction
  for (int it = blockIdx.x; it < A.nitems_n; it += G) {
    const ItemN w = A.items_n[it];
    const BProb &pb = A.probs[w.pid];
    double acc[3] = {0.0, 0.0, 0.0};
    dispatch_order(pb.order, [&](auto P) {
      constexpr int D = decltype(P)::value + 1, ND = D * D;
      for (int g = w.g0 + threadIdx.x; g < w.g1; g += blockDim.x) {
        int off[4];
        const int n = table_copies(pb.ncopy, g, off);
        for (int c = 0; c < 2; ++c) {
          const int k = c * pb.m.nh1 + g;
          const double idg = pb.invdiag[k];
          double rv = 0.0;
          if (idg != 0.0) {
            double ax = pb.evec[off[0] + c * ND];
            for (int j = 1; j < n; ++j) ax += pb.evec[off[j] + c * ND];
            const double bv = pb.rhs[k];
            rv = bv - ax;
            acc[0] = fma(bv, bv, acc[0]);
            acc[1] = fma(rv, rv, acc[1]);
            acc[2] = fma(rv * idg, rv, acc[2]);
          } else {
            pb.a[k] = 0.0;
          }
          pb.r[k] = rv;
          pb.p[k] = 0.0;
          pb.ap[k] = 0.0;
        }
      }
    });
    block_sum<3>(acc, red);
    if (threadIdx.x == 0)
      for (int q = 0; q < 3; ++q) A.partials[(size_t)it * 3 + q] = acc[q];
    BScal &sc = A.scal[w.pid];
    if (last_item(sc, pb.n_nitems)) {
      sum_item_partials(A.partials, pb.first_nitem, pb.n_nitems, 3, s_v);
      if (threadIdx.x == 0) {
        sc.cnt = 0;
        sc.bb = s_v[0];
        sc.rr = s_v[1];
        sc.rz = s_v[2];
        sc.rz_old = s_v[2];
        sc.beta = 0.0;
        sc.it = 0;
        sc.status = 0;
        sc.active = (s_v[0] > 0.0 && s_v[1] > tol2 * s_v[0]) ? 1 : 0;
        if (sc.active) atomicAdd(A.active, 1);
      }
    }
  }
  if (!sync()) return;

  for (int iter = 0;; ++iter) {
    const int nact = *(volatile int *)A.active;
    if (nact == 0 || iter >= A.max_it) break;
    // E: element matvec of p_new = invdiag r + beta p for active problems, with
    // p_new . M p_new summed element by element into one partial per item
    for (int it = blockIdx.x; it < A.nitems_e; it += G) {
      const ItemE w = A.items_e[it];
      BScal &sc = A.scal[w.pid];
      if (!sc.active) continue;
      const BProb &pb = A.probs[w.pid];
      const double beta = sc.beta;
      double acc[1] = {0.0};
      dispatch_order(w.order, [&](auto P) {
        for (int b = 0; b < w.nbat; ++b)
          acc[0] += b_cg_matvec<decltype(P)::value>(pb, w.e0 + b * F2<decltype(P)::value>::NBC, 1, beta, sm);
      });
      block_sum<1>(acc, red);
      if (threadIdx.x == 0) A.partials_e[it] = acc[0];
    }
    if (!sync()) return;
    // B: one node sweep: q = M p_new gathered, p = p_new, a += alpha p, r -= alpha q,
    // r.r and r.z; the last item of a problem forms beta and tests convergence.
    // alpha = r.z / p.Mp is formed by every node item of the problem from the element
    // items' partials, summed in item order (the same value in every block): there are
    // a few node items per block and many element items, so this costs less than an
    // atomic-counted last element item per problem
    for (int it = blockIdx.x; it < A.nitems_n; it += G) {
      const ItemN w = A.items_n[it];
      BScal &sc = A.scal[w.pid];
      if (!sc.active) continue;
      const BProb &pb = A.probs[w.pid];
      if (threadIdx.x < 32) {
        double t = 0.0;
        for (int i = threadIdx.x; i < pb.n_eitems; i += 32)
          t += ((volatile const double *)A.partials_e)[pb.first_eitem + i];
        t = warp_sum(t);
        if (threadIdx.x == 0) s_v[2] = sc.rz / t;
      }
      __syncthreads();
      const double alpha = s_v[2], beta = sc.beta;
      double acc[3] = {0.0, 0.0, 0.0};
      dispatch_order(pb.order, [&](auto P) {
        constexpr int D = decltype(P)::value + 1, ND = D * D;
        for (int g = w.g0 + threadIdx.x; g < w.g1; g += blockDim.x) {
          int off[4];
          const int n = table_copies(pb.ncopy, g, off);
          // every load of both components first (the problems live in DRAM), then
          // the arithmetic in the same order as one component at a time
          double idg[2], rv[2], pv[2], av[2], ev[2][4];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int k = c * pb.m.nh1 + g;
            idg[c] = pb.invdiag[k];
            rv[c] = pb.r[k];
            pv[c] = pb.p[k];
            av[c] = pb.a[k];
#pragma unroll
            for (int j = 0; j < 4; ++j) ev[c][j] = j < n ? pb.evec[off[j] + c * ND] : 0.0;
          }
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            if (idg[c] == 0.0) continue;
            const int k = c * pb.m.nh1 + g;
            double qv = ev[c][0];
#pragma unroll
            for (int j = 1; j < 4; ++j)
              if (j < n) qv += ev[c][j];
            const double pn = fma(beta, pv[c], idg[c] * rv[c]);
            const double r2 = fma(-alpha, qv, rv[c]);
            pb.p[k] = pn;
            pb.a[k] = fma(alpha, pn, av[c]);
            pb.r[k] = r2;
            acc[0] = fma(r2, r2, acc[0]);
            acc[1] = fma(r2 * idg[c], r2, acc[1]);
          }
        }
      });
      block_sum<3>(acc, red);
      if (threadIdx.x == 0) {
        A.partials[(size_t)it * 3] = acc[0];
        A.partials[(size_t)it * 3 + 1] = acc[1];
      }
      if (last_item(sc, pb.n_nitems)) {
        sum_item_partials(A.partials, pb.first_nitem, pb.n_nitems, 2, s_v);
        if (threadIdx.x == 0) {
          sc.cnt = 0;
          sc.it += 1;
          sc.rr = s_v[0];
          sc.rz_old = sc.rz;
          sc.rz = s_v[1];
          sc.beta = sc.rz / sc.rz_old;
          if (sc.rr <= tol2 * sc.bb) {
            sc.active = 0;
            atomicSub(A.active, 1);
          } else if (sc.it >= A.max_it) {
            sc.active = 0;
            sc.status = 5;
            atomicSub(A.active, 1);
            latch_status(A.status, 5);
          }
        }
      }
    }
    if (!sync()) return;
  }
  // report per problem; problems with b = 0 get a = 0
  for (int pid = blockIdx.x; pid < A.nprob; pid += G) {
    const BProb &pb = A.probs[pid];
    const BScal &sc = A.scal[pid];
    if (sc.bb == 0.0)
      for (int k = threadIdx.x; k < 2 * pb.m.nh1; k += blockDim.x) pb.a[k] = 0.0;
    if (threadIdx.x == 0 && pb.info) {
      pb.info->cg_iters[A.stage] = sc.it;
      pb.info->cg_rel_res[A.stage] = sc.bb > 0.0 ? sqrt(sc.rr / sc.bb) : 0.0;
      if (sc.status) pb.info->status = sc.status;
    }
  }
  if (!sync()) return;
  // ---- the stage's node update with the solved accelerations
  for (int it = blockIdx.x; it < A.nitems_n; it += G) {
    const ItemN w = A.items_n[it];
    if (A.stage == 0) node_mid(A.probs[w.pid], w);
    else node_final(A.probs[w.pid], w);
  }
  // nothing waits on bar_next during this launch: the next launch starts from zero
  if (blockIdx.x == 0 && threadIdx.x == 0) A.bar_next->count = 0ull;
}

}  // namespace
}  // namespace lh

using namespace lh;

struct lh_batch {
  int n = 0;
  std::vector<lh_ctx *> ctx;
  std::vector<int> order;
  // tile shapes (autotuned): element batches per work item of the element passes
  // and of the solver, per order, and the threads per block of the element passes
  int tiles[5] = {0, 1, 1, 1, 1};
  int tiles_cg[5] = {0, 1, 1, 1, 1};
  int tpb = 256;
  char *arena = nullptr;
  size_t arena_bytes = 0;
  // device arrays
  QdataArgs *q1 = nullptr, *q2 = nullptr;
  ForceArgs *fa = nullptr;
  ForceTArgs *t1 = nullptr, *t2 = nullptr;
  BProb *probs = nullptr;
  BScal *scal = nullptr;
  ItemE *items_e = nullptr, *items_cg = nullptr;
  ItemN *items_n = nullptr;
  int n_items_e = 0, n_items_cg = 0, n_items_n = 0, cap_items_e = 0, cap_items_cg = 0;
  double *partials = nullptr, *partials_e = nullptr, *dts = nullptr;
  std::vector<BProb> probs_host;   // host copy: the solver item ranges change with the tiles
  int *active = nullptr, *status = nullptr;
  GridBarrier *bar = nullptr;   // two: one per stage's solver launch
  int grid_e[3] = {0, 0, 0};    // per element block size 128, 256, 512
  int grid_cg = 0;
  size_t smem_e = 0, smem_cg = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double graph_tol = -1.0;
  int graph_max_it = -1;
  lh_step_info *infos = nullptr;
  std::vector<double *> xs, vs, es;
  std::string err;
};

static lh_status bfail(lh_batch *b, lh_status s, const std::string &msg) {
  if (b) b->err = msg;
  lh::set_global_error(msg);
  return s;
}

#define BCUDA(b, call)                                                                          \
  do {                                                                                          \
    cudaError_t _e = (call);                                                                    \
    if (_e != cudaSuccess) return bfail((b), LH_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
  } while (0)

static int nb_of(int order) {
  switch (order) {
    case 1: return F2<1>::NB;
    case 2: return F2<2>::NB;
    case 3: return F2<3>::NB;
    default: return F2<4>::NB;
  }
}
static int nbc_of(int order) {
  switch (order) {
    case 1: return F2<1>::NBC;
    case 2: return F2<2>::NBC;
    case 3: return F2<3>::NBC;
    default: return F2<4>::NBC;
  }
}

// Work items of all problems, sorted by order, `tiles[p]` batches of `nbf(p)` elements each.
template <typename NBF>
static std::vector<ItemE> make_items(const lh_batch *b, const int *tiles, NBF nbf) {
  std::vector<ItemE> items;
  for (int p = 1; p <= 4; ++p)
    for (int i = 0; i < b->n; ++i) {
      if (b->order[i] != p) continue;
      const int ne = b->ctx[i]->mesh.ne, nb = nbf(p), tile = std::max(1, tiles[p]);
      const int nbat = (ne + nb - 1) / nb;
      for (int bt = 0; bt < nbat; bt += tile) items.push_back({i, bt * nb, std::min(tile, nbat - bt), p});
    }
  return items;
}

// Each problem's solver element items are contiguous in the work list (sorted by
// order, then problem): record where they start and how many there are.
static void set_solver_ranges(std::vector<BProb> &pr, const std::vector<ItemE> &ic) {
  for (auto &p : pr) { p.first_eitem = 0; p.n_eitems = 0; }
  for (int k = 0; k < (int)ic.size(); ++k) {
    BProb &p = pr[ic[k].pid];
    if (p.n_eitems == 0) p.first_eitem = k;
    p.n_eitems += 1;
  }
}

static lh_status upload_items(lh_batch *b) {
  std::vector<ItemE> ie = make_items(b, b->tiles, nb_of);
  std::vector<ItemE> ic = make_items(b, b->tiles_cg, nbc_of);
  if ((int)ie.size() > b->cap_items_e || (int)ic.size() > b->cap_items_cg)
    return bfail(b, LH_ERR_ARG, "work list larger than at creation");
  BCUDA(b, cudaMemcpy(b->items_e, ie.data(), ie.size() * sizeof(ItemE), cudaMemcpyHostToDevice));
  BCUDA(b, cudaMemcpy(b->items_cg, ic.data(), ic.size() * sizeof(ItemE), cudaMemcpyHostToDevice));
  b->n_items_e = (int)ie.size();
  b->n_items_cg = (int)ic.size();
  set_solver_ranges(b->probs_host, ic);
  BCUDA(b, cudaMemcpy(b->probs, b->probs_host.data(), b->probs_host.size() * sizeof(BProb), cudaMemcpyHostToDevice));
  return LH_OK;
}

static int tpb_index(int tpb) { return tpb == 128 ? 0 : (tpb == 512 ? 2 : 1); }

static void drop_graph(lh_batch *b) {
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
}

extern "C" {

void lh_batch_destroy(lh_batch *b) {
  if (!b) return;
  drop_graph(b);
  if (b->arena) cudaFree(b->arena);
  delete b;
}

const char *lh_batch_last_error(const lh_batch *b) { return b ? b->err.c_str() : "null batch"; }

lh_status lh_batch_create(int n, lh_ctx *const *ctxs, double *const *x, double *const *v, double *const *e,
                          const double *dt, lh_step_info *infos, lh_batch **out) {
  if (!out) return bfail(nullptr, LH_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || !ctxs || !x || !v || !e || !dt) return bfail(nullptr, LH_ERR_ARG, "bad batch arguments");
  lh_batch *b = new lh_batch();
  b->n = n;
  for (int i = 0; i < n; ++i) {
    lh_ctx *c = ctxs[i];
    if (!c || !x[i] || !v[i] || !e[i]) { lh_batch_destroy(b); return bfail(nullptr, LH_ERR_ARG, "null problem"); }
    if (c->dim != 2 || c->q1 != 2 * c->p || c->prm.precision != LH_PRECISION_FP64) {
      lh_batch_destroy(b);
      return bfail(nullptr, LH_ERR_UNSUPPORTED, "batched problems must be 2D, q1 = 2p, FP64");
    }
    if (!(dt[i] > 0.0)) { lh_batch_destroy(b); return bfail(nullptr, LH_ERR_ARG, "dt must be > 0"); }
    b->ctx.push_back(c);
    b->order.push_back(c->p);
    b->xs.push_back(x[i]);
    b->vs.push_back(v[i]);
    b->es.push_back(e[i]);
  }
  b->infos = infos;
  // work lists (element items with the largest tile count used later must fit: size with tile 1)
  const int tiles1[5] = {0, 1, 1, 1, 1};
  std::vector<ItemE> ie = make_items(b, tiles1, nb_of);
  std::vector<ItemE> ic = make_items(b, tiles1, nbc_of);
  std::vector<ItemN> in;
  std::vector<BProb> pr(n);
  for (int i = 0; i < n; ++i) {
    lh_ctx *c = b->ctx[i];
    const int first = (int)in.size(), nh1 = c->mesh.nh1;
    int k = 0;
    for (int g0 = 0; g0 < nh1; g0 += kNodeItem, ++k) in.push_back({i, g0, std::min(nh1, g0 + kNodeItem), k});
    BProb &p = pr[i];
    p.m = c->mesh;
    p.order = c->p;
    p.n_nitems = (int)in.size() - first;
    p.first_nitem = first;
    p.source = c->prm.source;
    p.tab = c->tab;
    p.mq = c->mq;
    p.invdiag = c->invdiag;
    p.ncopy = c->ncopy;
    p.evec = c->evec;
    p.r = c->r;
    p.p = c->pv;
    p.ap = c->ap;
    p.a = c->a_prev;
    p.rhs = c->rhs;
    p.x = x[i];
    p.v = v[i];
    p.e = e[i];
    p.xh = c->xh;
    p.vh = c->vh;
    p.vb = c->vb;
    p.info = infos ? infos + i : nullptr;
  }
  // arena
  struct Item { void **ptr; size_t bytes; };
  const size_t nie = ie.size(), nic = ic.size(), nin = in.size();
  std::vector<Item> items = {
      {(void **)&b->q1, n * sizeof(QdataArgs)},   {(void **)&b->q2, n * sizeof(QdataArgs)},
      {(void **)&b->fa, n * sizeof(ForceArgs)},   {(void **)&b->t1, n * sizeof(ForceTArgs)},
      {(void **)&b->t2, n * sizeof(ForceTArgs)},  {(void **)&b->probs, n * sizeof(BProb)},
      {(void **)&b->scal, n * sizeof(BScal)},     {(void **)&b->items_e, nie * sizeof(ItemE)},
      {(void **)&b->items_cg, nic * sizeof(ItemE)}, {(void **)&b->items_n, nin * sizeof(ItemN)},
      {(void **)&b->partials, nin * 3 * sizeof(double)}, {(void **)&b->partials_e, nic * sizeof(double)},
      {(void **)&b->dts, n * sizeof(double)},
      {(void **)&b->active, 64}, {(void **)&b->status, 64}, {(void **)&b->bar, 2 * sizeof(GridBarrier)}};
  size_t bytes = 0;
  for (auto &it : items) bytes += (it.bytes + 255) / 256 * 256;
  if (cudaMalloc(&b->arena, bytes) != cudaSuccess) {
    b->arena = nullptr;
    lh_batch_destroy(b);
    return bfail(nullptr, LH_ERR_OOM, "batch arena allocation failed");
  }
  b->arena_bytes = bytes;
  size_t off = 0;
  for (auto &it : items) {
    *it.ptr = b->arena + off;
    off += (it.bytes + 255) / 256 * 256;
  }
  cudaMemset(b->arena, 0, bytes);
  for (int i = 0; i < n; ++i) pr[i].dt = b->dts + i;
  set_solver_ranges(pr, ic);
  b->probs_host = pr;
  // per-problem argument structs
  std::vector<QdataArgs> q1(n), q2(n);
  std::vector<ForceArgs> fa(n);
  std::vector<ForceTArgs> t1(n), t2(n);
  for (int i = 0; i < n; ++i) {
    lh_ctx *c = b->ctx[i];
    QdataArgs q{};
    q.mesh = c->mesh;
    q.tab = c->tab;
    q.mq = c->mq;
    q.jinv0 = c->jinv0;
    q.D = c->D;
    q.phys.gamma = c->prm.gamma;
    q.phys.h0 = c->h0;
    q.phys.order = (double)c->p;
    q.phys.use_viscosity = c->prm.use_viscosity;
    q.want_dt = 0;
    q.cfl = c->prm.cfl;
    q.status = c->dstatus;
    q.x = x[i];
    q.v = v[i];
    q.e = e[i];
    q1[i] = q;
    q.x = c->xh;
    q.v = c->vh;
    q.e = c->eh;
    q2[i] = q;
    fa[i] = ForceArgs{c->mesh, c->tab, c->D, nullptr, c->evec};
    const bool src = c->prm.source == LH_SOURCE_TAYLOR_GREEN_2D;
    ForceTArgs t{};
    t.mesh = c->mesh;
    t.tab = c->tab;
    t.D = c->D;
    t.mq = c->mq;
    t.me_inv = c->me_inv;
    t.dt = b->dts + i;
    t.v = c->vh;
    t.src_x = src ? x[i] : nullptr;
    t.e_base = e[i];
    t.coef = 0.5;
    t.out = c->eh;
    t1[i] = t;
    t.v = c->vb;
    t.src_x = src ? c->xh : nullptr;
    t.coef = 1.0;
    t.out = e[i];
    t2[i] = t;
  }
  BCUDA(b, cudaMemcpy(b->q1, q1.data(), n * sizeof(QdataArgs), cudaMemcpyHostToDevice));
  BCUDA(b, cudaMemcpy(b->q2, q2.data(), n * sizeof(QdataArgs), cudaMemcpyHostToDevice));
  BCUDA(b, cudaMemcpy(b->fa, fa.data(), n * sizeof(ForceArgs), cudaMemcpyHostToDevice));
  BCUDA(b, cudaMemcpy(b->t1, t1.data(), n * sizeof(ForceTArgs), cudaMemcpyHostToDevice));
  BCUDA(b, cudaMemcpy(b->t2, t2.data(), n * sizeof(ForceTArgs), cudaMemcpyHostToDevice));
  BCUDA(b, cudaMemcpy(b->probs, pr.data(), n * sizeof(BProb), cudaMemcpyHostToDevice));
  BCUDA(b, cudaMemcpy(b->dts, dt, n * sizeof(double), cudaMemcpyHostToDevice));
  BCUDA(b, cudaMemcpy(b->items_e, ie.data(), nie * sizeof(ItemE), cudaMemcpyHostToDevice));
  BCUDA(b, cudaMemcpy(b->items_cg, ic.data(), nic * sizeof(ItemE), cudaMemcpyHostToDevice));
  BCUDA(b, cudaMemcpy(b->items_n, in.data(), nin * sizeof(ItemN), cudaMemcpyHostToDevice));
  b->n_items_e = (int)nie;
  b->cap_items_e = (int)nie;
  b->n_items_cg = (int)nic;
  b->cap_items_cg = (int)nic;
  b->n_items_n = (int)nin;
  // launch shapes: shared memory = largest family's need
  b->smem_e = std::max({F2<1>::qdata_smem(), F2<2>::qdata_smem(), F2<3>::qdata_smem(), F2<4>::qdata_smem(),
                        F2<1>::force_smem(), F2<2>::force_smem(), F2<3>::force_smem(), F2<4>::force_smem(),
                        F2<1>::force_t_smem(), F2<2>::force_t_smem(), F2<3>::force_t_smem(),
                        F2<4>::force_t_smem()});
  b->smem_cg = std::max({F2<1>::cg_smem(), F2<2>::cg_smem(), F2<3>::cg_smem(), F2<4>::cg_smem()});
  int sms = 0, dev = 0, occ = 0;
  BCUDA(b, cudaGetDevice(&dev));
  BCUDA(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const void *ke[3][2] = {{(const void *)k_b_qf<128>, (const void *)k_b_force_t<128>},
                          {(const void *)k_b_qf<256>, (const void *)k_b_force_t<256>},
                          {(const void *)k_b_qf<512>, (const void *)k_b_force_t<512>}};
  const int tpbs[3] = {128, 256, 512};
  for (int t = 0; t < 3; ++t) {
    int occ_e = 1 << 30;
    for (const void *k : ke[t]) {
      BCUDA(b, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_e));
      BCUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, tpbs[t], b->smem_e));
      occ_e = std::min(occ_e, occ);
    }
    b->grid_e[t] = std::max(1, occ_e) * sms;
  }
  BCUDA(b, cudaFuncSetAttribute((const void *)k_b_cg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_cg));
  BCUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)k_b_cg, kThreadsCG, b->smem_cg));
  if (occ < 1) { lh_batch_destroy(b); return bfail(nullptr, LH_ERR_CUDA, "batched solver cannot be resident"); }
  b->grid_cg = std::min(occ, 2) * sms;
  BCUDA(b, cudaDeviceSynchronize());
  *out = b;
  return LH_OK;
}

static lh_status enqueue_step(lh_batch *b, double tol, int max_it, cudaStream_t s) {
  const int ti = tpb_index(b->tpb), ge = b->grid_e[ti];
  auto qf = [&](const QdataArgs *q) {
    switch (b->tpb) {
      case 128: k_b_qf<128><<<ge, 128, b->smem_e, s>>>(q, b->fa, b->items_e, b->n_items_e); break;
      case 512: k_b_qf<512><<<ge, 512, b->smem_e, s>>>(q, b->fa, b->items_e, b->n_items_e); break;
      default: k_b_qf<256><<<ge, 256, b->smem_e, s>>>(q, b->fa, b->items_e, b->n_items_e); break;
    }
  };
  auto ft = [&](const ForceTArgs *t) {
    switch (b->tpb) {
      case 128: k_b_force_t<128><<<ge, 128, b->smem_e, s>>>(t, b->items_e, b->n_items_e); break;
      case 512: k_b_force_t<512><<<ge, 512, b->smem_e, s>>>(t, b->items_e, b->n_items_e); break;
      default: k_b_force_t<256><<<ge, 256, b->smem_e, s>>>(t, b->items_e, b->n_items_e); break;
    }
  };
  auto cg = [&](int stage) -> lh_status {
    BCgArgs a{b->probs, b->scal, b->items_cg, b->n_items_cg, b->items_n, b->n_items_n, b->n,
              b->partials, b->partials_e, b->active, b->bar + stage, b->bar + (1 - stage), b->status, stage,
              tol, max_it};
    void *args[] = {&a};
    BCUDA(b, cudaLaunchCooperativeKernel((const void *)k_b_cg, dim3(b->grid_cg), dim3(kThreadsCG), args,
                                         b->smem_cg, s));
    return LH_OK;
  };
  // stage 1 at S_n: qdata + F.1, solve + rhs + mid update, F^T v + e update
  qf(b->q1);
  if (lh_status st = cg(0)) return st;
  ft(b->t1);
  // stage 2 at S_half
  qf(b->q2);
  if (lh_status st = cg(1)) return st;
  ft(b->t2);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bfail(b, LH_ERR_CUDA, std::string("batched step launch: ") + cudaGetErrorString(e));
  return LH_OK;
}

lh_status lh_batch_step(lh_batch *b, double rel_tol, int max_it, lh_stream_t stream) {
  if (!b) return LH_ERR_ARG;
  if (rel_tol <= 0.0) rel_tol = 1e-12;
  if (max_it <= 0) max_it = 1000;
  cudaStream_t s = (cudaStream_t)stream;
  if (!b->exec || b->graph_tol != rel_tol || b->graph_max_it != max_it) {
    drop_graph(b);
    cudaStream_t cap;
    BCUDA(b, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    BCUDA(b, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    lh_status st = enqueue_step(b, rel_tol, max_it, cap);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (st != LH_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (ec != cudaSuccess) return bfail(b, LH_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
    b->graph = g;
    BCUDA(b, cudaGraphInstantiate(&b->exec, g, 0));
    b->graph_tol = rel_tol;
    b->graph_max_it = max_it;
  }
  BCUDA(b, cudaGraphLaunch(b->exec, s));
  return LH_OK;
}

static void get_config(const lh_batch *b, int *cfg) {
  for (int p = 1; p <= 4; ++p) {
    cfg[p - 1] = b->tiles[p];
    cfg[3 + p] = b->tiles_cg[p];
  }
  cfg[8] = b->tpb;
}

lh_status lh_batch_set_config(lh_batch *b, const int *cfg) {
  if (!b || !cfg) return LH_ERR_ARG;
  for (int k = 0; k < 8; ++k)
    if (cfg[k] != 1 && cfg[k] != 2 && cfg[k] != 4) return bfail(b, LH_ERR_ARG, "tiles must be 1, 2 or 4");
  if (cfg[8] != 128 && cfg[8] != 256 && cfg[8] != 512)
    return bfail(b, LH_ERR_ARG, "threads per block must be 128, 256 or 512");
  for (int p = 1; p <= 4; ++p) {
    b->tiles[p] = cfg[p - 1];
    b->tiles_cg[p] = cfg[3 + p];
  }
  b->tpb = cfg[8];
  if (lh_status st = upload_items(b)) return st;
  drop_graph(b);   // the captured step holds the old work lists and launch shapes
  return LH_OK;
}

// Autotuner: times whole batched steps (both element passes and the solver) for
// candidate tile shapes and keeps, coordinate by coordinate, every change that
// makes the step at least 1 % faster: per order the element tile (1, 2, 4
// batches per work item) and the solver tile (1, 2, 4), then the element passes'
// threads per block (128, 256, 512). Every candidate starts from the same state
// (x, v, e, the accelerations that warm-start the solves and the step records
// are saved first and restored after each trial and at the end), so the
// problems are left exactly as they were. Synchronous; allocates and frees one
// snapshot buffer.
lh_status lh_batch_autotune(lh_batch *b, int *cfg_out) {
  if (!b) return LH_ERR_ARG;
  // snapshot of everything a step changes
  struct Seg { double *p; size_t n; };
  std::vector<Seg> segs;
  for (int i = 0; i < b->n; ++i) {
    const lh_ctx *c = b->ctx[i];
    const size_t nv = (size_t)2 * c->mesh.nh1, nl = (size_t)c->mesh.ne * c->p * c->p;
    segs.push_back({b->xs[i], nv});
    segs.push_back({b->vs[i], nv});
    segs.push_back({b->es[i], nl});
    segs.push_back({c->a_prev, nv});
  }
  size_t total = 0;
  for (auto &g : segs) total += g.n;
  const size_t info_bytes = b->infos ? (size_t)b->n * sizeof(lh_step_info) : 0;
  char *snap = nullptr;
  BCUDA(b, cudaMalloc(&snap, total * sizeof(double) + info_bytes));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  lh_status result = LH_OK;
  auto copy_all = [&](bool save) -> cudaError_t {
    size_t off = 0;
    for (auto &g : segs) {
      double *d = (double *)snap + off;
      const cudaError_t e = save ? cudaMemcpy(d, g.p, g.n * sizeof(double), cudaMemcpyDeviceToDevice)
                                 : cudaMemcpy(g.p, d, g.n * sizeof(double), cudaMemcpyDeviceToDevice);
      if (e != cudaSuccess) return e;
      off += g.n;
    }
    if (info_bytes) {
      char *d = snap + total * sizeof(double);
      return save ? cudaMemcpy(d, b->infos, info_bytes, cudaMemcpyDeviceToDevice)
                  : cudaMemcpy(b->infos, d, info_bytes, cudaMemcpyDeviceToDevice);
    }
    return cudaSuccess;
  };
  // one trial: restore, one warm-up step (captures the graph), three timed steps
  auto trial = [&](float *ms_out) -> lh_status {
    cudaError_t e = copy_all(false);
    if (e != cudaSuccess) return bfail(b, LH_ERR_CUDA, std::string("autotune restore: ") + cudaGetErrorString(e));
    if (lh_status st = lh_batch_step(b, 1e-12, 1000, nullptr)) return st;
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
      cudaEventRecord(e0);
      if (lh_status st = lh_batch_step(b, 1e-12, 1000, nullptr)) return st;
      cudaEventRecord(e1);
      e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) return bfail(b, LH_ERR_CUDA, std::string("autotune step: ") + cudaGetErrorString(e));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best = std::min(best, ms);
    }
    int st_host = 0;
    e = cudaMemcpy(&st_host, b->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bfail(b, LH_ERR_CUDA, std::string("autotune status: ") + cudaGetErrorString(e));
    if (st_host) return bfail(b, (lh_status)st_host, "autotune: a batched step latched a device error");
    *ms_out = best;
    return LH_OK;
  };
  int cfg[9];
  do {
    cudaError_t e = copy_all(true);
    if (e != cudaSuccess) { result = bfail(b, LH_ERR_CUDA, std::string("autotune snapshot: ") + cudaGetErrorString(e)); break; }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      result = bfail(b, LH_ERR_CUDA, "autotune: cudaEventCreate failed");
      break;
    }
    get_config(b, cfg);
    float best = 0.f;
    if ((result = trial(&best)) != LH_OK) break;
    auto try_cfg = [&](int k, int val) -> lh_status {
      int cand[9];
      std::memcpy(cand, cfg, sizeof(cand));
      if (cand[k] == val) return LH_OK;
      cand[k] = val;
      if (lh_status st = lh_batch_set_config(b, cand)) return st;
      float t = 0.f;
      if (lh_status st = trial(&t)) return st;
      if (t < 0.99f * best) {
        best = t;
        std::memcpy(cfg, cand, sizeof(cand));
      }
      return lh_batch_set_config(b, cfg);
    };
    for (int p = 1; p <= 4 && result == LH_OK; ++p) {
      bool present = false;
      for (int o : b->order) present |= o == p;
      if (!present) continue;
      // every listed value (try_cfg skips the current one), so a search that starts
      // from a shape set by lh_batch_set_config explores the same candidates
      for (int t : {1, 2, 4})
        if (result == LH_OK) result = try_cfg(p - 1, t);
      for (int t : {1, 2, 4})
        if (result == LH_OK) result = try_cfg(3 + p, t);
    }
    for (int t : {128, 256, 512})
      if (result == LH_OK) result = try_cfg(8, t);
  } while (false);
  const cudaError_t er = copy_all(false);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(snap);
  if (result != LH_OK) return result;
  if (er != cudaSuccess) return bfail(b, LH_ERR_CUDA, std::string("autotune restore: ") + cudaGetErrorString(er));
  if (cfg_out) get_config(b, cfg_out);
  return LH_OK;
}

}  // extern "C"
