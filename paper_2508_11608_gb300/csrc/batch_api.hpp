// Host interface of a batch group (implemented in batch.cuh).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace cutmg {

struct BatchInfo {
  int iterations = 0;
  double rel = 0.0, true_rel = 0.0;
};

// one group of problems with the same (dimension, degree)
class BatchGroupBase {
 public:
  virtual ~BatchGroupBase() = default;
  virtual int size() const = 0;
  // CG on every problem of the group; b and x compact FP64 device vectors
  virtual void start(int prec, const double* const* b, cudaStream_t s) = 0;
  virtual void half_a(cudaStream_t s) = 0;                    // q = A p ... (r, r)
  virtual void read_rr(double* host_rr, cudaStream_t s) = 0;  // synchronises
  virtual void deactivate(const std::vector<int>& idx) = 0;   // converged problems
  virtual int active() const = 0;
  virtual void half_b(int prec, cudaStream_t s) = 0;          // z = B r ... p
  virtual void finish(double* const* x, BatchInfo* info, cudaStream_t s) = 0;
  virtual void bnorms(double* host_bn) = 0;
  virtual int64_t launches() const = 0;
  virtual void autotune(cudaStream_t s) = 0;
  virtual void get_tile(int* warps, int* blocks_per_sm) const = 0;
  virtual void set_tile(int warps, int blocks_per_sm) = 0;
};

}  // namespace cutmg
