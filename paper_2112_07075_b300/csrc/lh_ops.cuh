// Builds the launcher table (Ops) of one compiled (DIM, P, Q) kernel family.
#pragma once

#include "lh_kernels.cuh"
#include "lh_tc.cuh"

namespace lh {

template <int DIM, int D>
__global__ void k_gather(MeshDesc m, const double *__restrict__ evec, int C, double *__restrict__ out, double scale,
                         const double *__restrict__ mask) {
  const size_t n = (size_t)C * m.nh1;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(k / m.nh1), g = (int)(k % m.nh1);
    double v = scale * gather_node<DIM, D>(m, evec, C, c, g);
    if (mask && mask[k] == 0.0) v = 0.0;
    out[k] = v;
  }
}

// Remap node pass: rhs = gathered K w (C = DIM), invdiag = 1 / gathered diagonal of
// M(tau) for every component (0 on constrained DOFs when constrained != 0).
template <int DIM, int D>
__global__ void k_remap_nodes(MeshDesc m, const double *__restrict__ evec, const double *__restrict__ dvec,
                              int constrained, double *__restrict__ rhs, double *__restrict__ invdiag) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < m.nh1; g += gridDim.x * blockDim.x) {
    if (rhs)
      for (int c = 0; c < DIM; ++c) rhs[(size_t)c * m.nh1 + g] = gather_node<DIM, D>(m, evec, DIM, c, g);
    if (invdiag) {
      const double inv = 1.0 / gather_node<DIM, D>(m, dvec, 1, 0, g);
      for (int c = 0; c < DIM; ++c)
        invdiag[(size_t)c * m.nh1 + g] = constrained && h1_constrained<DIM>(m, g, c) ? 0.0 : inv;
    }
  }
}

// Node-copy table: for node g, the offsets e*DIM*ND + i of its element-local
// copies in a DIM-component E-vector, in node_copies order, padded with -1.
template <int DIM, int D>
__global__ void k_node_table(MeshDesc m, int *__restrict__ tab) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < m.nh1; g += gridDim.x * blockDim.x) {
    int off[1 << DIM];
    const int n = node_copies<DIM, D>(m, g, DIM, off);
    for (int j = 0; j < (1 << DIM); ++j) tab[(size_t)g * (1 << DIM) + j] = j < n ? off[j] : -1;
  }
}

template <int DIM, int P, int Q>
struct OpsBuilder {
  using F = Family<DIM, P, Q>;
  static void qdata(const QdataArgs &a, int grid, cudaStream_t s) {
    k_qdata<DIM, P, Q><<<grid, F::THREADS, F::qdata_smem(), s>>>(a);
  }
  static void force(const ForceArgs &a, int grid, cudaStream_t s) {
    k_force<DIM, P, Q><<<grid, F::THREADS, F::force_smem(), s>>>(a);
  }
  static void force_t(const ForceTArgs &a, int grid, cudaStream_t s) {
    k_force_t<DIM, P, Q><<<grid, F::THREADS, F::force_t_smem(), s>>>(a);
  }
  static void mass(const MassArgs &a, int grid, cudaStream_t s) {
    k_mass<DIM, P, Q><<<grid, F::THREADS, F::mass_smem(), s>>>(a);
  }
  static cudaError_t cg(CgArgs &a, int grid, cudaStream_t s) {
    void *args[] = {&a};
    cudaError_t e = cudaMemsetAsync(a.bar, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel((const void *)k_cg<DIM, P, Q>, dim3(grid), dim3(F::TC), args, F::cg_smem(), s);
  }
  static cudaError_t cg_ir(CgIrArgs &a, int grid, cudaStream_t s) {
    void *args[] = {&a};
    cudaError_t e = cudaMemsetAsync(a.bar, 0, sizeof(GridBarrier), s);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel((const void *)k_cg_ir<DIM, P, Q>, dim3(grid), dim3(F::TC), args,
                                       F::cg_ir_smem(), s);
  }
  static constexpr bool kTc = TcTraits<DIM, P, Q>::on;
  static cudaError_t cg_tc(CgIrArgs &a, int grid, cudaStream_t s) {
    if constexpr (kTc) {
      void *args[] = {&a};
      cudaError_t e = cudaMemsetAsync(a.bar, 0, sizeof(GridBarrier), s);
      if (e != cudaSuccess) return e;
      return cudaLaunchCooperativeKernel((const void *)k_cg_tc<P, Q>, dim3(grid), dim3(TcMass<P, Q>::THREADS), args,
                                         TcMass<P, Q>::SMEM, s);
    } else {
      return cudaErrorNotSupported;
    }
  }
  static cudaError_t tc_apply(CgIrArgs &a, int grid, cudaStream_t s) {
    if constexpr (kTc) {
      k_tc_apply<P, Q><<<grid, TcMass<P, Q>::THREADS, TcMass<P, Q>::SMEM, s>>>(a);
      k_gather_f32<P + 1><<<grid * 4, 256, 0, s>>>(a.mesh, a.evec32, a.ap32);
      return cudaGetLastError();
    } else {
      return cudaErrorNotSupported;
    }
  }
  static void *tc_apply_kernel() {
    if constexpr (kTc) return (void *)k_tc_apply<P, Q>;
    else return nullptr;
  }
  static void *tc_kernel() {
    if constexpr (kTc) return (void *)k_cg_tc<P, Q>;
    else return nullptr;
  }
  static size_t tc_smem() {
    if constexpr (kTc) return TcMass<P, Q>::SMEM;
    else return 0;
  }
  static size_t tc_img_bytes() {
    if constexpr (kTc) return TcLayout<P, Q>::IMG;
    else return 0;
  }
  static void tc_image(const double *B, unsigned short *img) {
    if constexpr (kTc) tc_build_image<P, Q>(B, img);
  }
  static void geom(const GeomArgs &a, int grid, cudaStream_t s) {
    k_geom<DIM, P, Q><<<grid, F::THREADS, F::geom_smem(), s>>>(a);
  }
  static void diag(const DiagArgs &a, int grid, cudaStream_t s) {
    k_diag<DIM, P, Q><<<grid, F::THREADS, F::diag_smem(), s>>>(a);
  }
  static void emass(const EmassArgs &a, int grid, cudaStream_t s) {
    k_emass<DIM, P, Q><<<grid, 128, F::emass_smem(), s>>>(a);
  }
  static void init_e(const InitEArgs &a, int grid, cudaStream_t s) {
    k_init_e<DIM, P, Q><<<grid, F::THREADS, F::init_e_smem(), s>>>(a);
  }
  static void gather(const MeshDesc &m, const double *evec, int C, double *out, double scale, const double *mask,
                     int grid, int threads, cudaStream_t s) {
    k_gather<DIM, P + 1><<<grid, threads, 0, s>>>(m, evec, C, out, scale, mask);
  }
  static void remap(const RemapArgs &a, int grid, cudaStream_t s) {
    k_remap<DIM, P, Q><<<grid, F::THREADS, F::remap_smem(), s>>>(a);
  }
  static void remap_nodes(const MeshDesc &m, const double *evec, const double *dvec, int constrained, double *rhs,
                          double *invdiag, int grid, int threads, cudaStream_t s) {
    k_remap_nodes<DIM, P + 1><<<grid, threads, 0, s>>>(m, evec, dvec, constrained, rhs, invdiag);
  }
  static void stiff_setup(const StiffArgs &a, int grid, cudaStream_t s) {
    k_stiff_setup<DIM, P, Q><<<grid, F::THREADS, F::stiff_setup_smem(), s>>>(a);
  }
  static void stiff(const StiffArgs &a, int grid, cudaStream_t s) {
    k_stiff<DIM, P, Q><<<grid, F::THREADS, F::stiff_smem(), s>>>(a);
  }
  static void tmop(int mode, const TmopArgs &a, int grid, cudaStream_t s) {
    switch (mode) {
      case 0: k_tmop<DIM, P, Q, 0><<<grid, F::THREADS, F::tmop_smem(0), s>>>(a); break;
      case 1: k_tmop<DIM, P, Q, 1><<<grid, F::THREADS, F::tmop_smem(1), s>>>(a); break;
      case 2: k_tmop<DIM, P, Q, 2><<<grid, F::THREADS, F::tmop_smem(2), s>>>(a); break;
      case 3: k_tmop<DIM, P, Q, 3><<<grid, F::THREADS, F::tmop_smem(3), s>>>(a); break;
      case 4: k_tmop<DIM, P, Q, 4><<<grid, F::THREADS, F::tmop_smem(0), s>>>(a); break;
      default: k_tmop<DIM, P, Q, 5><<<grid, F::THREADS, F::tmop_smem(0), s>>>(a); break;
    }
  }
  static void node_table(const MeshDesc &m, int *tab, int grid, int threads, cudaStream_t s) {
    k_node_table<DIM, P + 1><<<grid, threads, 0, s>>>(m, tab);
  }
  static const Ops *get() {
    static const Ops ops = {DIM, P, Q, F::NB, F::THREADS, F::NBC, F::TC,
                            F::qdata_smem(), F::force_smem(), F::force_t_smem(), F::mass_smem(), F::cg_smem(),
                            F::geom_smem(), F::diag_smem(), F::emass_smem(), F::init_e_smem(), F::cg_ir_smem(),
                            (void *)k_qdata<DIM, P, Q>, (void *)k_force<DIM, P, Q>, (void *)k_force_t<DIM, P, Q>, (void *)k_mass<DIM, P, Q>,
                            (void *)k_cg<DIM, P, Q>, (void *)k_geom<DIM, P, Q>, (void *)k_diag<DIM, P, Q>, (void *)k_emass<DIM, P, Q>,
                            (void *)k_init_e<DIM, P, Q>, (void *)k_cg_ir<DIM, P, Q>,
                            &qdata, &force, &force_t, &mass, &cg, &cg_ir, &geom, &diag, &emass, &init_e,
                            &gather,
                            tc_kernel(), tc_smem(), kTc ? 512 : 0, tc_img_bytes(),
                            kTc ? &cg_tc : nullptr, kTc ? &tc_image : nullptr,
                            tc_apply_kernel(), kTc ? &tc_apply : nullptr,
                            F::remap_smem(), (void *)k_remap<DIM, P, Q>, &remap, &remap_nodes,
                            F::stiff_setup_smem(), F::stiff_smem(), (void *)k_stiff_setup<DIM, P, Q>,
                            (void *)k_stiff<DIM, P, Q>, &stiff_setup, &stiff,
                            {F::tmop_smem(0), F::tmop_smem(1), F::tmop_smem(2), F::tmop_smem(3), F::tmop_smem(0),
                             F::tmop_smem(0)},
                            {(void *)k_tmop<DIM, P, Q, 0>, (void *)k_tmop<DIM, P, Q, 1>, (void *)k_tmop<DIM, P, Q, 2>,
                             (void *)k_tmop<DIM, P, Q, 3>, (void *)k_tmop<DIM, P, Q, 4>, (void *)k_tmop<DIM, P, Q, 5>},
                            &tmop, &node_table};
    return &ops;
  }
};

}  // namespace lh
