// lh_mass_mult_noalloc: the PA mass action y = M_v x for callers that must not
// allocate device memory (see include/lh.h). The element vector that the
// regular path keeps in the context's arena lives here in a file-scope static
// device array of fixed size, so neither this call nor its set-up allocates.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "lh_internal.h"

namespace {

// Maximum scratch: 32 MiB of element-vector data (dim * NE * (p+1)^dim doubles).
constexpr size_t kScratchDoubles = (size_t(32) << 20) / sizeof(double);
// Basis tables of every compiled (order, q1) pair, one fixed slot each.
constexpr int kTabDoubles = 512;
constexpr int kFamilies[][2] = {{1, 2}, {2, 3}, {2, 4}, {3, 6}, {4, 6}, {4, 8}};
constexpr int kNumFamilies = sizeof(kFamilies) / sizeof(kFamilies[0]);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_scratch[kScratchDoubles];
static __device__ __align__(256) double g_tab[kNumFamilies * kTabDoubles];

// Device addresses of the two arrays, looked up once per device. In host code
// g_scratch / g_tab are only host-side stand-ins for the symbols and must never
// be passed to a kernel.
struct DevAddrs {
  double *scratch = nullptr;
  double *tab = nullptr;
};
std::mutex g_mu;
DevAddrs g_addrs[kMaxDevices];

lh_status fail(lh_status s, const std::string &msg) {
  lh::set_global_error(msg);
  return s;
}

int family_slot(int order, int q1) {
  for (int k = 0; k < kNumFamilies; ++k)
    if (kFamilies[k][0] == order && kFamilies[k][1] == q1) return k;
  return -1;
}

// One-time set-up of the current device (caller holds g_mu): resolve the arrays'
// device addresses, upload the basis tables of every family into their slots
// (synchronous copy, then a device synchronisation so that later calls on any
// stream see the tables), and raise the dynamic shared-memory limit of every
// compiled mass kernel. After this, calls only launch kernels.
lh_status setup_device(int dev) {
  void *ps = nullptr, *pt = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ps, g_scratch);
  if (e != cudaSuccess) return fail(LH_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
  e = cudaGetSymbolAddress(&pt, g_tab);
  if (e != cudaSuccess) return fail(LH_ERR_CUDA, std::string("cudaGetSymbolAddress(tab): ") + cudaGetErrorString(e));
  std::vector<double> tabs((size_t)kNumFamilies * kTabDoubles, 0.0);
  for (int k = 0; k < kNumFamilies; ++k) {
    if (lh::table_length(kFamilies[k][0], kFamilies[k][1]) > kTabDoubles)
      return fail(LH_ERR_ARG, "lh_mass_mult_noalloc: basis table too large");
    lh::build_tables(kFamilies[k][0], kFamilies[k][1], tabs.data() + (size_t)k * kTabDoubles, kTabDoubles);
  }
  e = cudaMemcpy(pt, tabs.data(), tabs.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(LH_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(LH_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));
  for (int k = 0; k < kNumFamilies; ++k) {
    for (int dim = 2; dim <= 3; ++dim) {
      const lh::Ops *ops = dim == 2 ? lh::find_ops_2d(kFamilies[k][0], kFamilies[k][1])
                                    : lh::find_ops_3d(kFamilies[k][0], kFamilies[k][1]);
      if (!ops) continue;
      e = cudaFuncSetAttribute(ops->k_mass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ops->smem_mass);
      if (e != cudaSuccess) return fail(LH_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    }
  }
  g_addrs[dev].scratch = (double *)ps;
  g_addrs[dev].tab = (double *)pt;
  return LH_OK;
}

}  // namespace

extern "C" lh_status lh_mass_mult_noalloc(int dim, int nx, int ny, int nz, int order, int q1, const double *mq,
                                          const double *x, double *y, lh_stream_t stream) {
  if (dim != 2 && dim != 3) return fail(LH_ERR_ARG, "lh_mass_mult_noalloc: dim must be 2 or 3");
  if (nx < 1 || ny < 1 || (dim == 3 && nz < 1))
    return fail(LH_ERR_ARG, "lh_mass_mult_noalloc: element counts must be >= 1");
  if (order < 1 || order > 4) return fail(LH_ERR_ARG, "lh_mass_mult_noalloc: order must be in 1..4");
  if (!mq || !x || !y) return fail(LH_ERR_ARG, "lh_mass_mult_noalloc: null pointer");
  if (x == y) return fail(LH_ERR_ARG, "lh_mass_mult_noalloc: x and y must not alias");
  const lh::Ops *ops = dim == 2 ? lh::find_ops_2d(order, q1) : lh::find_ops_3d(order, q1);
  const int slot = family_slot(order, q1);
  if (!ops || slot < 0)
    return fail(LH_ERR_UNSUPPORTED, "lh_mass_mult_noalloc: no compiled kernels for this (dim, order, q1)");
  if (dim == 2) nz = 1;
  const double ne_d = (double)nx * ny * nz;
  int nd = 1;
  for (int a = 0; a < dim; ++a) nd *= order + 1;
  const double need = ne_d * dim * nd;
  if (need > (double)kScratchDoubles) {
    return fail(LH_ERR_ARG, "lh_mass_mult_noalloc: the mesh needs " + std::to_string((long long)need * 8) +
                                " bytes of element-vector scratch; the static maximum is " +
                                std::to_string((long long)kScratchDoubles * 8) + " bytes (32 MiB)");
  }

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(LH_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(LH_ERR_ARG, "lh_mass_mult_noalloc: device index too large");
  DevAddrs addrs;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addrs[dev].scratch) {
      const lh_status st = setup_device(dev);
      if (st != LH_OK) return st;
    }
    addrs = g_addrs[dev];
  }

  lh::MeshDesc m;
  m.nx = nx;
  m.ny = ny;
  m.nz = nz;
  m.n1x = nx * order + 1;
  m.n1y = ny * order + 1;
  m.n1z = dim == 3 ? nz * order + 1 : 1;
  m.ne = nx * ny * nz;
  m.nh1 = m.n1x * m.n1y * m.n1z;
  cudaStream_t s = (cudaStream_t)stream;

  // Every element writes all of its scratch entries before the gather reads
  // them, so no part of the scratch has to start at zero.
  lh::MassArgs a{m, addrs.tab + (size_t)slot * kTabDoubles, mq, x, addrs.scratch};
  ops->mass(a, (m.ne + ops->nb - 1) / ops->nb, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LH_ERR_CUDA, std::string("mass kernel: ") + cudaGetErrorString(e));
  size_t nv = (size_t)dim * m.nh1;
  int grid = (int)std::min<size_t>((nv + 255) / 256, 65535);
  ops->gather(m, addrs.scratch, dim, y, 1.0, nullptr, grid, 256, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LH_ERR_CUDA, std::string("gather kernel: ") + cudaGetErrorString(e));
  return LH_OK;
}
