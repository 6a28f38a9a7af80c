// Internal types of liblh shared by the host API and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/lh.h"

namespace lh {

struct MeshDesc {
  int nx, ny, nz;      // elements per direction (nz = 1 in 2D)
  int n1x, n1y, n1z;   // H1 nodes per direction
  int ne;              // elements
  int nh1;             // scalar H1 nodes
};

struct PhysParams {
  double gamma;
  double h0;           // (|Omega_0| / NE)^(1/dim) / p
  double order;        // p, for hmin = sigma_min(J) / p
  int use_viscosity;
};

struct QdataArgs {
  MeshDesc mesh;
  const double *tab, *x, *v, *e, *mq, *jinv0;
  double *D;
  PhysParams phys;
  int want_dt;
  double cfl, fixed_dt;
  double *partials;          // [gridDim] block maxima of 1/dt
  unsigned int *counter;     // last-block ticket (reset by the last block)
  double *dt_est_out;        // optional
  lh_step_info *step;        // optional: dt control of lh_rk2avg_step
  int ctl;                   // step control with rejection: 0 off, 1 stage 1 (choose dt), 2 stage 2 (decide)
  int *status;
};

struct ForceArgs {
  MeshDesc mesh;
  const double *tab, *D, *u;
  double *evec;              // [NE][DIM][ND]
};

struct ForceTArgs {
  MeshDesc mesh;
  const double *tab, *D, *v, *mq;
  const double *src_x;       // positions for the TG-2D energy source, or NULL
  const double *me_inv;      // NULL: out = F^T v; else out = e_base + coef*dt*Me^{-1}(F^T v + b)
  const double *e_base, *dt;
  double coef;
  double *out;
  double *partials;          // for the source sum
  unsigned int *counter;
  double *src_sum;           // optional: dt * sum_j b_j
  const int *skip;           // optional: nonzero -> the launch does nothing (rejected step)
};

struct MassArgs {
  MeshDesc mesh;
  const double *tab, *mq, *x;
  double *evec;
};

struct CgArgs {
  MeshDesc mesh;
  const double *tab, *mq, *invdiag, *b;
  double *x, *r, *p, *ap, *evec, *partials;
  double *z;                 // invdiag * r, kept with r
  const int *ncopy;          // [N_H1][2^DIM] E-vector offsets e*DIM*ND + i of each node's copies, -1 padded
  void *bar;                 // GridBarrier
  int *status;
  lh_cg_info *info;
  int *iters_out;
  double *relres_out;
  double tol;
  int max_it;
};

struct CgIrArgs {
  MeshDesc mesh;
  const double *tab, *mq, *invdiag, *b;
  const float *mq32, *invdiag32;
  double *x, *evec, *partials;
  float *r32, *p32, *ap32, *d32, *evec32;
  float *z32;         // invdiag32 * r32, kept beside r32 by the inner solver
  void *bar;
  int *status;
  lh_cg_info *info;
  int *iters_out;
  double *relres_out;
  double tol, inner_tol;
  int max_it, max_outer, max_inner;
  const void *kimg;   // tensor-core form: shared-memory image of the BF16 interpolation matrix
  const int *ncopy;   // as in CgArgs
};

struct GeomArgs {
  MeshDesc mesh;
  const double *tab, *x0, *rho0_in;
  double *rho0, *mq, *jinv0, *partials;
  int *status;
};

struct DiagArgs {
  MeshDesc mesh;
  const double *tab, *mq;
  double *evec;              // [NE][ND]
};

struct EmassArgs {
  const double *tab, *mq;
  double *me_inv;
};

// Remap phase (Section 3.5): one stage's element pass on the mesh x(tau) = x0 + tau u.
struct RemapArgs {
  MeshDesc mesh;
  const double *tab, *x0, *u;  // H1 [DIM][N_H1]: source positions, displacement x1 - x0
  const double *v, *k;         // stage input w = v + s k (k may be NULL: w = v)
  double s, tau;
  double *mq;                  // out [NE][NQ]: omega detJ(tau)
  double *evec;                // out [NE][DIM][ND]: element contributions of K(tau) w, or NULL
  double *dvec;                // out [NE][ND]: element diagonal of M(tau), or NULL
  int *status;
};

// Stiffness operator (Sections 2.1, 3.3): setup on a mesh and the PA action.
struct StiffArgs {
  MeshDesc mesh;
  const double *tab;
  const double *x;   // setup: H1 node positions [DIM][N_H1]
  double *G;         // [NE][DIM(DIM+1)/2][NQ] PA data (setup writes, action reads)
  double *mq;        // setup: out [NE][NQ] unit-density mass data omega det J
  double *dvec;      // setup: out [NE][ND] element diagonal of that mass matrix
  const double *u;   // action: input [DIM][N_H1]
  double *evec;      // action: out [NE][DIM][ND]
  int *status;
};

// Mesh optimisation (TMOP, Sections 2.2 and 3.4): one fully matrix-free element pass.
struct TmopArgs {
  MeshDesc mesh;
  const double *tab;
  const double *x;     // positions [DIM][N_H1]
  const double *x0;    // limiting reference positions (objective, gradient), or NULL
  const double *u;     // Hessian action: direction [DIM][N_H1]
  double h_inv, detW;  // target W = h I: 1/h, h^DIM
  double lim;          // gamma / d^2 (0: no limiting term)
  double *evec;        // gradient / Hessian action / diagonal: [NE][DIM][ND]
  double *pa;          // partially assembled Hessian data [NE][NH2][NQ] (setup writes, apply reads)
  double *partials;    // objective: block sums, last-block total into *out
  unsigned int *counter;
  double *out;
  int *status;
};

struct InitEArgs {
  MeshDesc mesh;
  const double *tab, *x0, *mq, *rho0, *me_inv;
  double *e;
  double gamma;
  int problem;
};

// Launchers of one compiled (dim, p, q1) family.
struct Ops {
  int dim, p, q1, nb, threads, nb_cg, threads_cg;
  size_t smem_qdata, smem_force, smem_force_t, smem_mass, smem_cg, smem_geom, smem_diag, smem_emass, smem_init_e,
      smem_cg_ir;
  void *k_qdata, *k_force, *k_force_t, *k_mass, *k_cg, *k_geom, *k_diag, *k_emass, *k_init_e, *k_cg_ir;
  void (*qdata)(const QdataArgs &, int grid, cudaStream_t);
  void (*force)(const ForceArgs &, int grid, cudaStream_t);
  void (*force_t)(const ForceTArgs &, int grid, cudaStream_t);
  void (*mass)(const MassArgs &, int grid, cudaStream_t);
  cudaError_t (*cg)(CgArgs &, int grid, cudaStream_t);
  cudaError_t (*cg_ir)(CgIrArgs &, int grid, cudaStream_t);
  void (*geom)(const GeomArgs &, int grid, cudaStream_t);
  void (*diag)(const DiagArgs &, int grid, cudaStream_t);
  void (*emass)(const EmassArgs &, int grid, cudaStream_t);
  void (*init_e)(const InitEArgs &, int grid, cudaStream_t);
  void (*gather)(const MeshDesc &, const double *evec, int C, double *out, double scale, const double *mask,
                 int grid, int threads, cudaStream_t);
  // tensor-core inner solver of the precision form (NULL where the family has none)
  void *k_cg_tc;
  size_t smem_cg_tc;
  int threads_cg_tc;
  size_t tc_img_bytes;
  cudaError_t (*cg_tc)(CgIrArgs &, int grid, cudaStream_t);
  void (*tc_image)(const double *B, unsigned short *img);   // host: B = 1D table [q1][p+1]
  void *k_tc_apply;
  // M x with the tensor-core element operator: x = a.d32 (free DOFs), E-vector in
  // a.evec32, node sums in a.ap32
  cudaError_t (*tc_apply)(CgIrArgs &, int grid, cudaStream_t);
  // remap phase: element pass and the node pass (K w gathered into rhs, Jacobi
  // inverse of the gathered diagonal into invdiag, 0 on constrained DOFs if asked)
  size_t smem_remap;
  void *k_remap;
  void (*remap)(const RemapArgs &, int grid, cudaStream_t);
  void (*remap_nodes)(const MeshDesc &, const double *evec, const double *dvec, int constrained, double *rhs,
                      double *invdiag, int grid, int threads, cudaStream_t);
  // stiffness operator: setup pass and action (element parts)
  size_t smem_stiff_setup, smem_stiff;
  void *k_stiff_setup, *k_stiff;
  void (*stiff_setup)(const StiffArgs &, int grid, cudaStream_t);
  void (*stiff)(const StiffArgs &, int grid, cudaStream_t);
  // TMOP element passes, mode 0 objective, 1 gradient, 2 Hessian action, 3 diagonal,
  // 4 partially assembled Hessian setup, 5 its action
  size_t smem_tmop[6];
  void *k_tmop[6];
  void (*tmop)(int mode, const TmopArgs &, int grid, cudaStream_t);
  // setup: the node-copy table of the solvers' node sweeps
  void (*node_table)(const MeshDesc &, int *ncopy, int grid, int threads, cudaStream_t);
};

const Ops *find_ops_2d(int p, int q1);
const Ops *find_ops_3d(int p, int q1);

// Host-side 1D tables (basis_host.cpp): fills tab in the layout the kernels expect.
void build_tables(int p, int q1, double *tab, int tab_len);
int table_length(int p, int q1);
void gll_nodes(int p, double *z);
// H1 (GLL-node) basis values and derivatives of order p at the reference point x.
void h1_basis_at(int p, double x, double *vals, double *ders);

// Sets the message lh_last_error(NULL) returns (calls without a context).
void set_global_error(const std::string &msg);

}  // namespace lh

struct lh_learn;
namespace lh {
// Learned-form hooks around each mass solve of lh_rk2avg_step (learned.cu).
lh_status learn_before_solve(lh_ctx *c, const double *x, cudaStream_t s);
lh_status learn_after_solve(lh_ctx *c, cudaStream_t s);
void learn_free(lh_learn *L);
}  // namespace lh

// The context behind the opaque lh_ctx handle (one problem: mesh, tables, arena).
struct lh_ctx {
  lh_params prm{};
  lh::MeshDesc mesh{};
  const lh::Ops *ops = nullptr;
  int dim = 0, p = 0, q1 = 0, nd = 0, nl = 0, nq = 0;
  size_t nv = 0;
  int grid_elem = 0, grid_cg = 0, grid_node = 0, sms = 0;
  double h0 = 0.0, volume = 0.0;
  char *arena = nullptr;
  size_t arena_bytes = 0;
  // sub-buffers
  double *tab = nullptr, *verts = nullptr, *x0 = nullptr, *rho0 = nullptr, *mq = nullptr, *jinv0 = nullptr,
         *D = nullptr, *me_inv = nullptr, *invdiag = nullptr, *evec = nullptr, *r = nullptr, *pv = nullptr,
         *ap = nullptr, *a_prev = nullptr, *rhs = nullptr, *xh = nullptr, *vh = nullptr, *vb = nullptr,
         *eh = nullptr, *partials = nullptr, *zv = nullptr;
  // stiffness operator on a mesh set by lh_stiffness_setup: PA data, unit-density mass
  // data and its Jacobi inverse (every DOF)
  double *stiff_G = nullptr, *stiff_mq = nullptr, *stiff_inv = nullptr;
  float *stiff_mq32 = nullptr, *stiff_inv32 = nullptr;   // precision form only
  bool stiff_ready = false;
  float *mq32 = nullptr, *invdiag32 = nullptr, *r32 = nullptr, *p32 = nullptr, *ap32 = nullptr, *d32 = nullptr,
        *evec32 = nullptr, *z32 = nullptr;
  int grid_cg_ir = 0, grid_cg_tc = 0;
  unsigned short *kimg = nullptr;   // tensor-core form: BF16 image of the interpolation matrix
  unsigned int *counter = nullptr;
  void *bar = nullptr;   // lh::GridBarrier
  int *dstatus = nullptr;
  int *ncopy = nullptr;   // [N_H1][2^dim] E-vector offsets of each node's copies (CgArgs::ncopy)
  lh_cg_info *remap_ci = nullptr;   // result of the remap's latest mass solve
  bool dt_control = false;          // lh_set_dt_control
  lh_learn *learn = nullptr;   // learned-form state (lh_learn_attach), or NULL
  // solver timing probe (lh_timing_enable): event pairs around solver launches
  static constexpr int kTimingPairs = 64;
  bool timing = false;
  int timing_n = 0;
  cudaEvent_t tev[2 * kTimingPairs] = {};
  std::string err = "no error";
};

