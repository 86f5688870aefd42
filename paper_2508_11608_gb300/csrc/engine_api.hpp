// Type-erased interface between the C ABI and the (dim, degree)-specialised
// device engines.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

namespace cutmg {

struct Hierarchy;

struct CudaError : std::runtime_error {
  using std::runtime_error::runtime_error;
};
struct OomError : std::runtime_error {
  using std::runtime_error::runtime_error;
};
struct TimeoutError : std::runtime_error {
  using std::runtime_error::runtime_error;
};

class EngineBase {
 public:
  virtual ~EngineBase() = default;
  virtual int n_levels() const = 0;
  virtual int64_t n_dofs(int level) const = 0;
  virtual size_t device_bytes() const = 0;
  virtual void level_apply(int l, int prec, const double* x, double* y, cudaStream_t s) = 0;
  virtual void level_colour(int l, int prec, int cut, int colour, double* x, const double* b,
                            cudaStream_t s) = 0;
  virtual void level_smooth(int l, int prec, int post, double* x, const double* b, cudaStream_t s) = 0;
  virtual void level_restrict(int l, int prec, const double* rf, double* bc, cudaStream_t s) = 0;
  virtual void level_prolongate(int l, int prec, const double* xc, double* xf, cudaStream_t s) = 0;
  virtual void coarse_solve(int prec, const double* b0, double* x0, cudaStream_t s) = 0;
  virtual void apply_fine(const double* x, double* y, cudaStream_t s) = 0;
  virtual void rhs(double* b, cudaStream_t s) = 0;
  virtual void vcycle(int prec, const double* r, double* z, cudaStream_t s) = 0;
  virtual int solve(int prec, const double* b, double* x, double rtol, int maxit, double* rel,
                    double* true_rel, float* ms, cudaStream_t s) = 0;
  // the parts of a CG solve around its iterations: x = 0, r = b, z = B r,
  // p = z (returns ||b||); at the end the true residual norm and x gathered
  // The V-cycle as the solver: x += B (b - A x) from x = 0 (Sec. 2.2)
  virtual int solve_vcycle(int prec, const double* b, double* x, double rtol, int maxit, double* rel,
                           double* true_rel, float* ms, cudaStream_t s) = 0;
  // GMRES(restart) with the V-cycle as right preconditioner (Sec. 2.2)
  virtual int solve_gmres(int prec, const double* b, double* x, double rtol, int restart, int maxit, double* rel,
                          double* true_rel, float* ms, cudaStream_t s) = 0;
  virtual double cg_begin(int prec, const double* b, cudaStream_t s) = 0;
  virtual double cg_end(double* x, cudaStream_t s) = 0;
  // launch variant of a kernel family (0 = the automatic choice), and the
  // polls the cut-patch kernel waits for its TMA copy before it reports a
  // timeout; both drop the captured CUDA graphs
  virtual void set_variant(int family, int variant) = 0;
  virtual void set_wait_limit(int polls) = 0;
  // packed lower triangle of cut patch j's inverse on level l (FP64, from the
  // device records; synchronises)
  virtual void cut_inverse(int l, int64_t j, double* h_inv) = 0;  // m x m, row-major
  // kernel launches issued so far, and event timing of one kernel family
  virtual int64_t launches() const = 0;
  virtual void profile_start(int kind, int level) = 0;
  virtual void profile_read(double* ms, int64_t* n, double* flops, double* bytes) = 0;
  // device data of the coarsest level: FP64 explicit inverse (n0 x n0),
  // lattice index of each coarse DoF (int and int64), lattice size
  virtual void coarse_data(const double** inv, const int** nodes, const int64_t** dofs, int64_t* n0,
                           int64_t* nbox) const = 0;
};

// device engine of a built hierarchy; its uploads are ordered on `stream`,
// which the constructor synchronises before it returns
std::unique_ptr<EngineBase> make_engine_d2(int degree, const Hierarchy& H, cudaStream_t stream);
std::unique_ptr<EngineBase> make_engine_d3(int degree, const Hierarchy& H, cudaStream_t stream);

class BatchGroupBase;
std::unique_ptr<BatchGroupBase> make_batch_group_d2(int degree, const std::vector<EngineBase*>& inst, int n_c);
std::unique_ptr<BatchGroupBase> make_batch_group_d3(int degree, const std::vector<EngineBase*>& inst, int n_c);

}  // namespace cutmg
