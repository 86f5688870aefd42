// Coarsest-level solve for callers that must not allocate device memory.
//
// cf_coarse_solve stages its input and output through two lattice-layout
// vectors that the problem handle allocated with cudaMalloc.  Some callers
// cannot have a call allocate: code that runs while a stream is being
// captured into a CUDA graph, services that reserve all device memory up
// front in their own arena, and real-time loops that forbid allocation on
// the hot path.  cf_coarse_solve_noalloc does the same work with its two
// staging vectors in one file-scope __device__ array of fixed size, so the
// call itself allocates nothing.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/cutmg.h"
#include "engine_api.hpp"
#include "kernels.cuh"

namespace {

// room for two coarsest-level lattice vectors of up to kMaxCoarseBox nodes
constexpr int64_t kMaxCoarseBox = 32768;
static __device__ __align__(256) double g_coarse_stage[2 * kMaxCoarseBox];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_stage_ptr[kMaxDevices] = {nullptr};

// device address of g_coarse_stage on the current device (looked up once per
// device: the host-side symbol is only a stand-in for the device array)
cudaError_t stage_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_stage_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_coarse_stage);
    if (e != cudaSuccess) return e;
    g_stage_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_stage_ptr[dev];
  return cudaSuccess;
}

}  // namespace

// defined in capi.cu
extern "C" cf_status cutmg_noalloc_engine(cf_problem* pb, cutmg::EngineBase** eng, int* device);
cf_status cutmg_set_error(cf_status s, const char* msg);

extern "C" cf_status cf_coarse_solve_noalloc(cf_problem* pb, const double* d_b0, double* d_x0,
                                             void* stream) {
  using namespace cutmg;
  if (!d_b0 || !d_x0) return cutmg_set_error(CF_EINVAL, "null argument");
  EngineBase* eng = nullptr;
  int pdev = -1;
  cf_status st = cutmg_noalloc_engine(pb, &eng, &pdev);
  if (st != CF_OK) return st;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != pdev)
    return cutmg_set_error(CF_EINVAL, "the current device is not the problem's device");
  if (dev < 0 || dev >= kMaxDevices) return cutmg_set_error(CF_EUNSUPPORTED, "device ordinal out of range");
  const double* inv = nullptr;
  const int* nodes = nullptr;
  const int64_t* dofs = nullptr;
  int64_t n0 = 0, nbox = 0;
  eng->coarse_data(&inv, &nodes, &dofs, &n0, &nbox);
  if (nbox > kMaxCoarseBox)
    return cutmg_set_error(CF_EINVAL, ("coarsest lattice has " + std::to_string(nbox) +
                                       " nodes; cf_coarse_solve_noalloc supports at most " +
                                       std::to_string(kMaxCoarseBox))
                                          .c_str());
  double* stage = nullptr;
  cudaError_t e = stage_address(dev, &stage);
  if (e != cudaSuccess)
    return cutmg_set_error(CF_ECUDA, (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
  double* box_b = stage;
  double* box_x = stage + kMaxCoarseBox;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // only the coarse DoF entries of the two staging vectors are written and
  // read, so nothing needs clearing between calls
  const int nb = (int)((n0 + 255) / 256);
  k_scatter<double, double><<<nb, 256, 0, s>>>(dofs, n0, d_b0, box_b);
  k_coarse<double><<<(int)((n0 + 7) / 8), 256, 0, s>>>(inv, nodes, (int)n0, box_b, box_x);
  k_gather<double, double><<<nb, 256, 0, s>>>(dofs, n0, box_x, d_x0);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return cutmg_set_error(CF_ECUDA, (std::string("coarse solve launch: ") + cudaGetErrorString(e)).c_str());
  return CF_OK;
}
