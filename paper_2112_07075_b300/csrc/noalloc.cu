// lh_mass_mult_noalloc: the PA mass action y = M_v x for callers that must not
// allocate device memory (see include/lh.h). The element vector that the
// regular path keeps in the context's arena lives here in a file-scope static
// device array of fixed size, so neither this call nor its set-up allocates.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "lh_internal.h"

namespace {

// Maximum scratch: 32 MiB of element-vector data (dim * NE * (p+1)^dim doubles).
constexpr size_t kScratchDoubles = (size_t(32) << 20) / sizeof(double);
constexpr int kTabDoubles = 512;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_scratch[kScratchDoubles];
static __device__ __align__(256) double g_tab[kTabDoubles];

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
  if (!ops) return fail(LH_ERR_UNSUPPORTED, "lh_mass_mult_noalloc: no compiled kernels for this (dim, order, q1)");
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
  const int tablen = lh::table_length(order, q1);
  if (tablen > kTabDoubles) return fail(LH_ERR_ARG, "lh_mass_mult_noalloc: basis table too large");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(LH_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(LH_ERR_ARG, "lh_mass_mult_noalloc: device index too large");
  DevAddrs addrs;
  {
    // One-time set-up per device (the current one): resolve the symbols' device addresses.
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addrs[dev].scratch) {
      void *ps = nullptr, *pt = nullptr;
      e = cudaGetSymbolAddress(&ps, g_scratch);
      if (e != cudaSuccess)
        return fail(LH_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      e = cudaGetSymbolAddress(&pt, g_tab);
      if (e != cudaSuccess)
        return fail(LH_ERR_CUDA, std::string("cudaGetSymbolAddress(tab): ") + cudaGetErrorString(e));
      g_addrs[dev].scratch = (double *)ps;
      g_addrs[dev].tab = (double *)pt;
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

  double tab[kTabDoubles];
  lh::build_tables(order, q1, tab, kTabDoubles);
  e = cudaMemcpyAsync(addrs.tab, tab, tablen * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(LH_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));
  e = cudaFuncSetAttribute(ops->k_mass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ops->smem_mass);
  if (e != cudaSuccess) return fail(LH_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));

  // Every element writes all of its scratch entries before the gather reads
  // them, so no part of the scratch has to start at zero.
  lh::MassArgs a{m, addrs.tab, mq, x, addrs.scratch};
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
