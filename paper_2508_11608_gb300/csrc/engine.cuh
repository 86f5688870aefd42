// Device-resident hierarchy and the orchestration of the hot path: V-cycle
// (Sec. 2.2) with the partitioned multiplicative vertex-patch smoother
// (eq. "smoother-split") inside FP64 CG.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <array>
#include <map>
#include <memory>
#include <tuple>
#include <type_traits>
#include <stdexcept>
#include <string>
#include <vector>

#include "cutpipe.cuh"
#include "engine_api.hpp"
#include "sumfact.cuh"
#include "kernels.cuh"
#include "setup.hpp"

namespace cutmg {

#define CUTMG_CUDA(expr)                                                                   \
  do {                                                                                     \
    cudaError_t e__ = (expr);                                                              \
    if (e__ != cudaSuccess)                                                                \
      throw CudaError(std::string(#expr) + ": " + cudaGetErrorString(e__));               \
  } while (0)

inline void launch_check(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw CudaError(std::string(what) + ": " + cudaGetErrorString(e));
}

// FP32 -> TF32 (10 explicit mantissa bits), round to nearest even
inline float round_tf32(float v) {
  uint32_t u;
  std::memcpy(&u, &v, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) u += 0xfffu + ((u >> 13) & 1u);
  u &= 0xffffe000u;
  std::memcpy(&v, &u, 4);
  return v;
}

// One step of the Chebyshev smoother over a level's active box:
// x_new = x + c1 (x - xp) + c2 D^{-1} r, then xp <- x, x <- x_new
template <typename T>
__global__ void __launch_bounds__(256) k_chebyshev(Region R, T* __restrict__ x, T* __restrict__ xp,
                                                   const T* __restrict__ r, const T* __restrict__ dinv, T c1,
                                                   T c2) {
  R.for_each_node([&](int64_t o) {
    const T xo = x[o];
    x[o] = xo + c1 * (xo - xp[o]) + c2 * (dinv[o] * r[o]);
    xp[o] = xo;
  });
}

// w = D^{-1} v over a region (the power iteration of the Chebyshev bound)
template <typename T>
__global__ void __launch_bounds__(256) k_scale_diag(Region R, const T* __restrict__ dinv, const T* __restrict__ v,
                                                    T* __restrict__ w) {
  R.for_each_node([&](int64_t o) { w[o] = dinv[o] * v[o]; });
}

// FP64 vector updates of the Krylov solvers (finest level, box layout)
// y += a x over a region; a = sign * (*as) when as is given, else a = sign
static __global__ void __launch_bounds__(256) k_axpy(Region R, const double* __restrict__ as, double sign,
                                                     const double* __restrict__ x, double* __restrict__ y) {
  const double a = as ? sign * *as : sign;
  R.for_each_node([&](int64_t o) { y[o] += a * x[o]; });
}

// y = x / sqrt(*nn) over a region (normalisation by a squared norm on the device)
static __global__ void __launch_bounds__(256) k_scale_rsqrt(Region R, const double* __restrict__ nn,
                                                            const double* __restrict__ x, double* __restrict__ y) {
  const double a = 1.0 / sqrt(*nn);
  R.for_each_node([&](int64_t o) { y[o] = a * x[o]; });
}

// Owns every device allocation of a problem.  Zero fills and uploads are
// ordered on the stream given at set-up (uploads from pageable host memory
// return once the data has been staged).
class DevPool {
 public:
  ~DevPool() {
    for (void* p : ptrs_) cudaFree(p);
  }
  void set_stream(cudaStream_t s) { s_ = s; }
  template <typename T>
  T* alloc(size_t count, bool zero = true) {
    if (count == 0) count = 1;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) throw OomError("cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
    ptrs_.push_back(p);
    bytes_ += count * sizeof(T);
    if (zero) CUTMG_CUDA(cudaMemsetAsync(p, 0, count * sizeof(T), s_));
    return static_cast<T*>(p);
  }
  template <typename T, typename S, typename A>
  T* upload(const std::vector<S, A>& v) {
    T* p = alloc<T>(v.size(), false);
    if (v.empty()) return p;
    if constexpr (std::is_same<T, S>::value) {
      CUTMG_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s_));
    } else {
      std::vector<T> tmp(v.begin(), v.end());
      CUTMG_CUDA(cudaMemcpyAsync(p, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice, s_));
      CUTMG_CUDA(cudaStreamSynchronize(s_));  // tmp is released on return
    }
    return p;
  }
  size_t bytes() const { return bytes_; }

 private:
  std::vector<void*> ptrs_;
  size_t bytes_ = 0;
  cudaStream_t s_ = nullptr;
};

inline int blocks_for(int64_t n, int bs) { return (int)((n + bs - 1) / bs); }

template <int DIM, int P>
class BatchGroup;

template <int DIM, int P>
class Engine final : public EngineBase {
  friend class BatchGroup<DIM, P>;
  static constexpr int NB = Shape<DIM, P>::NB;
  static constexpr int C = 2 * P + 1, M = 2 * P - 1;
  static constexpr int WARPS = 4;

  struct Common {  // precision-independent level data
    int N, n;
    int64_t nbox, ndof;
    uint8_t* cflag;
    int* cut_id;
    uint8_t* nact;
    int64_t* dofs;
    int* bulk;
    int nbulk;
    int* bnd;
    int nbnd;
    double bnd_work[3] = {0.0, 0.0, 0.0};  // boundary-row launch: flops, scalars, index bytes
    int* sf_tiles = nullptr;     // sum-factorised operator: tiles of bulk positions
    uint32_t* sf_masks = nullptr;
    int nsf = 0;
    int* mnode;
    int* faces;
    int nfaces;
    int* face_id;
    int* fofs;
    int* fent;
    int* cfaces;
    std::vector<int> cf_start;
    int* cart;
    std::vector<int> cart_start;
    int* cutv;
    int* cutn;
    int* cutmo;
    int64_t* cutio;
    int* cutfo;
    int* cutcell;
    int* citoff;
    uint8_t* citems;
    uint16_t* members;
    std::vector<int> cut_start;
    std::vector<int> cut_maxm2;
    std::vector<int> cut_maxit;
    int64_t nmembers;
    // pipelined cut kernel (closures of more than 64 nodes)
    int* members32 = nullptr;
    int* pioff = nullptr;
    int* pnit = nullptr;
    uint32_t* pitems = nullptr;
    int* ppk = nullptr;
    uint64_t* pgmask = nullptr;
    int64_t* proff = nullptr;
    std::vector<int> cut_maxrec;
    int* gboff = nullptr;     // boundary-face moment slots per patch
    int* geoff = nullptr;     // ghost-entry lists per patch
    uint16_t* gent = nullptr;
    int* bf_face = nullptr;   // per colour: block-boundary ghost faces to compute
    int* bf_dst = nullptr;    // and their two destination slots
    std::vector<int> bf_start;
    int* pro_col;
    int* res_col;
    int* coarse_nodes;
    Region region;  // bbox of the active nodes
    int bb_lo[3], bb_hi[3];
  };
  template <typename T>
  struct Typed {  // per-precision level data and work vectors
    OpArgs<T> op;
    FdArgs<T, P> fd;
    SfArgs<T> sf;
    T* inv;
    T* pro_w;
    T* res_w;
    T* coarse_inv;
    float* dense_d;  // FP32 interior-patch map, transposed, rows padded to 4 (Wt[kc][r])
    float* tc_b = nullptr;  // the same map as the tensor-core B operand (TF32, core-matrix layout)
    T* rec = nullptr;       // cut-patch records of the pipelined kernel (packed inverse + cut rows)
    T* Gb = nullptr;        // moment slots of the block-boundary ghost faces
    T* kp = nullptr;        // uncut element matrix for h = 1, rows padded to NBP (record kernel)
    T ksc = T(1);           // h^(d-2): the uncut element matrix is ksc kp
    T* dinv = nullptr;  // Chebyshev smoother: 1 / diag(A_l) on the box (0 off the DoFs)
    T* xp = nullptr;    // Chebyshev smoother: previous iterate
    T *x, *b, *r;          // box vectors
    T *t1, *t2, *t3, *t4;  // transfer intermediates (restriction: t1,t2; prolongation: t3,t4)
  };

 public:
  Engine(const Hierarchy& H, cudaStream_t stream) : H_(H), setup_stream_(stream) {
    pool_.set_stream(stream);
    const int L = (int)H.levels.size();
    com_.resize(L);
    d64_.resize(L);
    d32_.resize(L);
    err_ = pool_.alloc<int>(1);
    for (int l = 0; l < L; ++l) upload_level(l);
    const auto& F = com_.back();
    xF_ = pool_.alloc<double>(F.nbox);
    rF_ = pool_.alloc<double>(F.nbox);
    pF_ = pool_.alloc<double>(F.nbox);
    qF_ = pool_.alloc<double>(F.nbox);
    zF_ = pool_.alloc<double>(F.nbox);
    bF_ = pool_.alloc<double>(F.nbox);
    tF_ = pool_.alloc<double>(F.nbox);
    aux_ = pool_.alloc<double>(F.nbox);
    aux2_ = pool_.alloc<double>(F.nbox);
    part_ = pool_.alloc<double>(kDotBlocks);
    sc_ = pool_.alloc<double>(16);
    CUTMG_CUDA(cudaFuncSetAttribute(k_smooth_tc<DIM, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    TcGeo<DIM, P>::SMEM));
    CUTMG_CUDA(cudaFuncSetAttribute(k_apply_sf<DIM, P, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    SfGeo<DIM, P>::ELEMS * (int)sizeof(double)));
    CUTMG_CUDA(cudaFuncSetAttribute(k_apply_sf<DIM, P, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    SfGeo<DIM, P>::ELEMS * (int)sizeof(float)));
    if (!kWarpCut) {
      CUTMG_CUDA(cudaFuncSetAttribute(k_cut_warp<DIM, P, float, kCutWarps>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kCutWarps * warp_stage_bytes<DIM, P, float>()));
      CUTMG_CUDA(cudaFuncSetAttribute(k_cut_warp<DIM, P, double, kCutWarps>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kCutWarps * warp_stage_bytes<DIM, P, double>()));
      CUTMG_CUDA(cudaFuncSetAttribute(k_cut_warp<DIM, P, float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      warp_stage_bytes<DIM, P, float>()));
      CUTMG_CUDA(cudaFuncSetAttribute(k_cut_warp<DIM, P, double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      warp_stage_bytes<DIM, P, double>()));
      CUTMG_CUDA(cudaFuncSetAttribute(k_cut_team<DIM, P, float, kCutTeam>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, warp_stage_bytes<DIM, P, float>()));
      CUTMG_CUDA(cudaFuncSetAttribute(k_cut_team<DIM, P, double, kCutTeam>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, warp_stage_bytes<DIM, P, double>()));
    }
    {
      int dev = 0;
      CUTMG_CUDA(cudaGetDevice(&dev));
      CUTMG_CUDA(cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, dev));
    }
    CUTMG_CUDA(cudaMallocHost(&host_sc_, 16 * sizeof(double)));
    CUTMG_CUDA(cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking));
    if (H.prm.smoother == 1) {
      lam_.assign(L, 0.0);
      for (int l = 1; l < L; ++l) lam_[l] = power_lambda_max(l);
    }
    const char* g = std::getenv("CUTMG_GRAPHS");
    use_graphs_ = !(g && g[0] == '0');
    CUTMG_CUDA(cudaStreamSynchronize(stream));
  }
  ~Engine() override {
    drop_graphs();
    if (cap_) cudaStreamDestroy(cap_);
    if (host_sc_) cudaFreeHost(host_sc_);
    for (auto& e : prof_.ev) cudaEventDestroy(e);
  }

  int64_t launches() const override { return launches_; }
  // family 1 = interior-patch step (FP32: 1 dense one patch per thread, 2 dense
  // two per thread, 3 dense split, 4 tensor cores; FP64: 1 two patches per
  // warp, 2 block per patch); family 2 = cut-patch step of the record kernel (1
  // records prefetched into L2 at issue, 2 no prefetch, 3 one patch ahead,
  // 4 eight warps per block at every size, 5 one warp per block for small
  // colours, 6 one patch per block at every size); family 3 = operator rows of
  // plain nodes (1 element matrices, 2 sum factorisation).  0 restores the
  // automatic choice.
  void set_variant(int family, int variant) override {
    if (family == 1) {
      if (variant < 0 || variant > 4) throw std::invalid_argument("interior variant must be 0..4");
      var_int_ = variant;
    } else if (family == 2) {
      if (variant < 0 || variant > 6) throw std::invalid_argument("cut variant must be 0..6");
      var_cut_ = variant;
    } else if (family == 3) {
      if (variant < 0 || variant > 2) throw std::invalid_argument("operator variant must be 0..2");
      var_op_ = variant;
    } else {
      throw std::invalid_argument("kernel family must be 1 (interior), 2 (cut) or 3 (operator)");
    }
    drop_graphs();
  }
  void cut_inverse(int l, int64_t j, double* h_inv) override {
    if (kWarpCut || l < 1 || l >= n_levels()) throw std::invalid_argument("no cut-patch records on this level");
    const HostLevel& h = H_.levels[l];
    const int m = h.cut_n[j], mp = (m + 3) / 4 * 4;
    std::vector<double> a((size_t)m * mp);
    CUTMG_CUDA(cudaMemcpy(a.data(), d64_[l].rec + h.cut_roff[j], sizeof(double) * a.size(), cudaMemcpyDeviceToHost));
    for (int i = 0; i < m; ++i)
      for (int c = 0; c < m; ++c) h_inv[(size_t)i * m + c] = a[(size_t)i * mp + c];
  }
  void set_wait_limit(int polls) override {
    if (polls < 0) throw std::invalid_argument("wait limit must be >= 0");
    spin_ = polls;
    drop_graphs();
  }
  void coarse_data(const double** inv, const int** nodes, const int64_t** dofs, int64_t* n0,
                   int64_t* nbox) const override {
    *inv = d64_[0].coarse_inv;
    *nodes = com_[0].coarse_nodes;
    *dofs = com_[0].dofs;
    *n0 = com_[0].ndof;
    *nbox = com_[0].nbox;
  }
  void profile_start(int kind, int level) override {
    prof_.kind = kind;
    prof_.level = level;
    prof_.used = 0;
    prof_.flops = prof_.bytes = 0.0;
    prof_.n = 0;
  }
  void profile_read(double* ms, int64_t* n, double* flops, double* bytes) override {
    double tot = 0.0;
    for (int i = 0; i + 1 < prof_.used; i += 2) {
      CUTMG_CUDA(cudaEventSynchronize(prof_.ev[i + 1]));
      float t = 0.f;
      CUTMG_CUDA(cudaEventElapsedTime(&t, prof_.ev[i], prof_.ev[i + 1]));
      tot += t;
    }
    *ms = tot;
    *n = prof_.n;
    *flops = prof_.flops;
    *bytes = prof_.bytes;
    prof_.kind = 0;
    prof_.used = 0;
  }

  int n_levels() const override { return (int)com_.size(); }
  int64_t n_dofs(int l) const override { return com_[l].ndof; }
  size_t device_bytes() const override { return pool_.bytes(); }

  // ---- single steps on compact FP64 vectors --------------------------------
  void level_apply(int l, int prec, const double* x, double* y, cudaStream_t s) override {
    if (prec == 1) {
      auto& D = d32_[l];
      to_box(l, x, D.x, s);
      apply<float>(l, D, D.x, nullptr, D.r, s);
      from_box(l, D.r, y, s);
    } else {
      auto& D = d64_[l];
      to_box(l, x, D.x, s);
      apply<double>(l, D, D.x, nullptr, D.r, s);
      from_box(l, D.r, y, s);
    }
  }
  void level_colour(int l, int prec, int cut, int colour, double* x, const double* b,
                    cudaStream_t s) override {
    check_smooth_level(l);
    if (prec == 1) {
      auto& D = d32_[l];
      to_box(l, x, D.x, s);
      to_box(l, b, D.b, s);
      colour_step<float>(l, D, cut, colour, D.x, D.b, s);
      from_box(l, D.x, x, s);
    } else {
      auto& D = d64_[l];
      to_box(l, x, D.x, s);
      to_box(l, b, D.b, s);
      colour_step<double>(l, D, cut, colour, D.x, D.b, s);
      from_box(l, D.x, x, s);
    }
  }
  void level_smooth(int l, int prec, int post, double* x, const double* b, cudaStream_t s) override {
    check_smooth_level(l);
    if (prec == 1) {
      auto& D = d32_[l];
      to_box(l, x, D.x, s);
      to_box(l, b, D.b, s);
      smooth<float>(l, D, post != 0, D.x, D.b, s);
      from_box(l, D.x, x, s);
    } else {
      auto& D = d64_[l];
      to_box(l, x, D.x, s);
      to_box(l, b, D.b, s);
      smooth<double>(l, D, post != 0, D.x, D.b, s);
      from_box(l, D.x, x, s);
    }
  }
  void level_restrict(int l, int prec, const double* rf, double* bc, cudaStream_t s) override {
    check_smooth_level(l);
    if (prec == 1) {
      to_box(l, rf, d32_[l].r, s);
      restrict_<float>(l, d32_, d32_[l].r, d32_[l - 1].b, s);
      from_box(l - 1, d32_[l - 1].b, bc, s);
    } else {
      to_box(l, rf, d64_[l].r, s);
      restrict_<double>(l, d64_, d64_[l].r, d64_[l - 1].b, s);
      from_box(l - 1, d64_[l - 1].b, bc, s);
    }
  }
  void level_prolongate(int l, int prec, const double* xc, double* xf, cudaStream_t s) override {
    check_smooth_level(l);
    if (prec == 1) {
      to_box(l - 1, xc, d32_[l - 1].x, s);
      to_box(l, xf, d32_[l].x, s);
      prolong<float>(l, d32_, d32_[l - 1].x, d32_[l].x, s);
      from_box(l, d32_[l].x, xf, s);
    } else {
      to_box(l - 1, xc, d64_[l - 1].x, s);
      to_box(l, xf, d64_[l].x, s);
      prolong<double>(l, d64_, d64_[l - 1].x, d64_[l].x, s);
      from_box(l, d64_[l].x, xf, s);
    }
  }
  void coarse_solve(int prec, const double* b0, double* x0, cudaStream_t s) override {
    if (prec == 1) {
      to_box(0, b0, d32_[0].b, s);
      coarse<float>(d32_[0], d32_[0].b, d32_[0].x, s);
      from_box(0, d32_[0].x, x0, s);
    } else {
      to_box(0, b0, d64_[0].b, s);
      coarse<double>(d64_[0], d64_[0].b, d64_[0].x, s);
      from_box(0, d64_[0].x, x0, s);
    }
  }

  // ---- finest-level operations ------------------------------------------------
  void apply_fine(const double* x, double* y, cudaStream_t s) override {
    level_apply(n_levels() - 1, 0, x, y, s);
  }
  void rhs(double* b, cudaStream_t s) override {
    CUTMG_CUDA(cudaMemcpyAsync(b, rhs_d_, sizeof(double) * com_.back().ndof,
                               cudaMemcpyDeviceToDevice, s));
  }
  void vcycle(int prec, const double* r, double* z, cudaStream_t s) override {
    const int L = n_levels() - 1;
    to_box(L, r, aux_, s);
    run_graph(GraphKey{300 + prec, aux_, aux2_}, s, [&](cudaStream_t cs) { precondition(prec, aux_, aux2_, cs); });
    from_box(L, aux2_, z, s);
  }

  double cg_begin(int prec, const double* b, cudaStream_t s) override {
    const int L = n_levels() - 1;
    const auto& F = com_[L];
    to_box(L, b, bF_, s);
    const size_t bytes = sizeof(double) * F.nbox;
    CUTMG_CUDA(cudaMemsetAsync(xF_, 0, bytes, s));
    CUTMG_CUDA(cudaMemcpyAsync(rF_, bF_, bytes, cudaMemcpyDeviceToDevice, s));
    dot(F.region, bF_, bF_, sc_ + 4, s);
    const double bn = std::sqrt(read_scalar(4, s));
    if (bn > 0.0) {
      run_graph(GraphKey{300 + prec, rF_, zF_}, s, [&](cudaStream_t cs) { precondition(prec, rF_, zF_, cs); });
      dot(F.region, rF_, zF_, sc_ + 0, s);
      CUTMG_CUDA(cudaMemcpyAsync(pF_, zF_, bytes, cudaMemcpyDeviceToDevice, s));
    }
    return bn;
  }
  double cg_end(double* x, cudaStream_t s) override {
    const int L = n_levels() - 1;
    const auto& F = com_[L];
    apply<double>(L, d64_[L], xF_, bF_, tF_, s);
    dot(F.region, tF_, tF_, sc_ + 5, s);
    const double tr = std::sqrt(read_scalar(5, s));
    from_box(L, xF_, x, s);
    return tr;
  }

  int solve(int prec, const double* b, double* x, double rtol, int maxit, double* rel,
            double* true_rel, float* ms, cudaStream_t s) override {
    const int L = n_levels() - 1;
    const auto& F = com_[L];
    cudaEvent_t e0, e1;
    CUTMG_CUDA(cudaEventCreate(&e0));
    CUTMG_CUDA(cudaEventCreate(&e1));
    CUTMG_CUDA(cudaEventRecord(e0, s));
    to_box(L, b, bF_, s);
    const size_t bytes = sizeof(double) * F.nbox;
    CUTMG_CUDA(cudaMemsetAsync(xF_, 0, bytes, s));
    CUTMG_CUDA(cudaMemcpyAsync(rF_, bF_, bytes, cudaMemcpyDeviceToDevice, s));
    dot(F.region, bF_, bF_, sc_ + 4, s);
    double bn2 = read_scalar(4, s);
    const double bn = std::sqrt(bn2);
    int it = 0;
    double rn = bn;
    if (bn > 0.0) {
      run_graph(GraphKey{300 + prec, rF_, zF_}, s, [&](cudaStream_t cs) { precondition(prec, rF_, zF_, cs); });
      dot(F.region, rF_, zF_, sc_ + 0, s);  // rz
      CUTMG_CUDA(cudaMemcpyAsync(pF_, zF_, bytes, cudaMemcpyDeviceToDevice, s));
      while (it < maxit) {
        // q = A p, alpha = rz / (p, q), x += alpha p, r -= alpha q, ||r||^2 to the host
        run_graph(GraphKey{100, pF_, xF_}, s, [&](cudaStream_t cs) {
          apply<double>(L, d64_[L], pF_, nullptr, qF_, cs);
          dot(F.region, pF_, qF_, sc_ + 1, cs);  // pq
          k_cg_update_xr<<<kVecBlocks, 256, 0, cs>>>(F.region, sc_, xF_, rF_, pF_, qF_);
          count_launch("cg update x r");
          dot(F.region, rF_, rF_, sc_ + 3, cs);  // rr
          CUTMG_CUDA(cudaMemcpyAsync(host_sc_ + 3, sc_ + 3, sizeof(double), cudaMemcpyDeviceToHost, cs));
        });
        CUTMG_CUDA(cudaStreamSynchronize(s));
        ++it;
        rn = std::sqrt(host_sc_[3]);
        if (!(rn > rtol * bn)) break;
        // z = B r, beta = (r, z)_new / (r, z), p = z + beta p
        run_graph(GraphKey{200 + prec, rF_, zF_}, s, [&](cudaStream_t cs) {
          precondition(prec, rF_, zF_, cs);
          dot(F.region, rF_, zF_, sc_ + 2, cs);  // rz_new
          k_cg_update_p<<<kVecBlocks, 256, 0, cs>>>(F.region, sc_, pF_, zF_);
          count_launch("cg update p");
          k_copy_scalar<<<1, 1, 0, cs>>>(sc_, 0, 2);
          count_launch("cg scalar");
        });
      }
    }
    CUTMG_CUDA(cudaEventRecord(e1, s));
    CUTMG_CUDA(cudaEventSynchronize(e1));
    CUTMG_CUDA(cudaEventElapsedTime(ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    check_err(s);
    // true residual
    apply<double>(L, d64_[L], xF_, bF_, tF_, s);
    dot(F.region, tF_, tF_, sc_ + 5, s);
    double tr = std::sqrt(read_scalar(5, s));
    from_box(L, xF_, x, s);
    *rel = bn > 0 ? rn / bn : 0.0;
    *true_rel = bn > 0 ? tr / bn : 0.0;
    return it;
  }

  // The V-cycle as the solver (Sec. 2.2): x_{k+1} = x_k + B (b - A x_k),
  // x_0 = 0, until ||b - A x_k|| <= rtol ||b||; one host read per iteration.
  int solve_vcycle(int prec, const double* b, double* x, double rtol, int maxit, double* rel, double* true_rel,
                   float* ms, cudaStream_t s) override {
    const int L = n_levels() - 1;
    const auto& F = com_[L];
    Timer tm(s);
    to_box(L, b, bF_, s);
    const size_t bytes = sizeof(double) * F.nbox;
    CUTMG_CUDA(cudaMemsetAsync(xF_, 0, bytes, s));
    CUTMG_CUDA(cudaMemcpyAsync(rF_, bF_, bytes, cudaMemcpyDeviceToDevice, s));
    dot(F.region, bF_, bF_, sc_ + 4, s);
    const double bn = std::sqrt(read_scalar(4, s));
    double rn = bn;
    int it = 0;
    while (rn > rtol * bn && it < maxit) {
      run_graph(GraphKey{300 + prec, rF_, zF_}, s, [&](cudaStream_t cs) { precondition(prec, rF_, zF_, cs); });
      run_graph(GraphKey{400, zF_, rF_}, s, [&](cudaStream_t cs) {
        k_axpy<<<kVecBlocks, 256, 0, cs>>>(F.region, nullptr, 1.0, zF_, xF_);
        count_launch("axpy");
        apply<double>(L, d64_[L], xF_, bF_, rF_, cs);
        dot(F.region, rF_, rF_, sc_ + 3, cs);
        CUTMG_CUDA(cudaMemcpyAsync(host_sc_ + 3, sc_ + 3, sizeof(double), cudaMemcpyDeviceToHost, cs));
      });
      CUTMG_CUDA(cudaStreamSynchronize(s));
      rn = std::sqrt(host_sc_[3]);
      ++it;
    }
    *ms = tm.stop();
    check_err(s);
    *true_rel = bn > 0 ? true_residual(s) / bn : 0.0;
    *rel = bn > 0 ? rn / bn : 0.0;
    from_box(L, xF_, x, s);
    return it;
  }

  // GMRES(restart) right-preconditioned by one V-cycle (Sec. 2.2): minimises
  // ||b - A x|| over x_0 + B K_k(A B, r_0), Arnoldi by modified Gram-Schmidt
  // with the Hessenberg entries on the device, Givens rotations of each new
  // column on the host; restarts from the true residual.
  int solve_gmres(int prec, const double* b, double* x, double rtol, int restart, int maxit, double* rel,
                  double* true_rel, float* ms, cudaStream_t s) override {
    const int L = n_levels() - 1;
    const auto& F = com_[L];
    const int m = restart;
    gmres_storage(m);
    Timer tm(s);
    to_box(L, b, bF_, s);
    const size_t bytes = sizeof(double) * F.nbox;
    CUTMG_CUDA(cudaMemsetAsync(xF_, 0, bytes, s));
    CUTMG_CUDA(cudaMemcpyAsync(rF_, bF_, bytes, cudaMemcpyDeviceToDevice, s));
    dot(F.region, bF_, bF_, sc_ + 4, s);
    const double bn = std::sqrt(read_scalar(4, s));
    dot(F.region, rF_, rF_, gsc_ + m + 1, s);
    double beta = bn, rn = bn;
    int total = 0;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), col(m + 2);
    while (beta > rtol * bn && total < maxit) {
      // v_0 = r / ||r||  (gsc_[m + 1] holds ||r||^2)
      for (auto& h : H) h = 0.0;
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      k_scale_rsqrt<<<kVecBlocks, 256, 0, s>>>(F.region, gsc_ + m + 1, rF_, gV_[0]);
      count_launch("gmres normalise");
      int k = 0;
      bool done = false;
      for (int j = 0; j < m; ++j) {
        // z_j = B v_j, w = A z_j, MGS against v_0..v_j, h_{j+1,j} = ||w||
        run_graph(GraphKey{300 + prec, gV_[j], gZ_[j]}, s,
                  [&](cudaStream_t c2) { precondition(prec, gV_[j], gZ_[j], c2); });
        apply<double>(L, d64_[L], gZ_[j], nullptr, gW_, s);
        for (int i = 0; i <= j; ++i) {
          dot(F.region, gW_, gV_[i], gsc_ + i, s);
          k_axpy<<<kVecBlocks, 256, 0, s>>>(F.region, gsc_ + i, -1.0, gV_[i], gW_);
          count_launch("gmres orthogonalise");
        }
        dot(F.region, gW_, gW_, gsc_ + j + 1, s);
        k_scale_rsqrt<<<kVecBlocks, 256, 0, s>>>(F.region, gsc_ + j + 1, gW_, gV_[j + 1]);
        count_launch("gmres normalise");
        CUTMG_CUDA(cudaMemcpyAsync(col.data(), gsc_, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, s));
        CUTMG_CUDA(cudaStreamSynchronize(s));
        col[j + 1] = std::sqrt(col[j + 1]);
        for (int i = 0; i <= j + 1; ++i) H[(size_t)i * m + j] = col[i];
        for (int i = 0; i < j; ++i) {
          const double t = cs[i] * H[(size_t)i * m + j] + sn[i] * H[(size_t)(i + 1) * m + j];
          H[(size_t)(i + 1) * m + j] = -sn[i] * H[(size_t)i * m + j] + cs[i] * H[(size_t)(i + 1) * m + j];
          H[(size_t)i * m + j] = t;
        }
        const double den = std::hypot(H[(size_t)j * m + j], H[(size_t)(j + 1) * m + j]);
        cs[j] = H[(size_t)j * m + j] / den;
        sn[j] = H[(size_t)(j + 1) * m + j] / den;
        H[(size_t)j * m + j] = den;
        H[(size_t)(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        k = j + 1;
        ++total;
        rn = std::fabs(g[j + 1]);
        if (rn <= rtol * bn || total >= maxit) {
          done = true;
          break;
        }
      }
      // x += Z_k y with H_k y = g_k (upper triangular, on the host)
      std::vector<double> y(k);
      for (int i = k - 1; i >= 0; --i) {
        double t = g[i];
        for (int q = i + 1; q < k; ++q) t -= H[(size_t)i * m + q] * y[q];
        y[i] = t / H[(size_t)i * m + i];
      }
      for (int i = 0; i < k; ++i) {
        k_axpy<<<kVecBlocks, 256, 0, s>>>(F.region, nullptr, y[i], gZ_[i], xF_);
        count_launch("gmres update");
      }
      apply<double>(L, d64_[L], xF_, bF_, rF_, s);
      dot(F.region, rF_, rF_, gsc_ + m + 1, s);
      CUTMG_CUDA(cudaMemcpyAsync(col.data(), gsc_ + m + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
      CUTMG_CUDA(cudaStreamSynchronize(s));
      beta = std::sqrt(col[0]);
      if (done) break;
    }
    *ms = tm.stop();
    check_err(s);
    *true_rel = bn > 0 ? true_residual(s) / bn : 0.0;
    *rel = bn > 0 ? rn / bn : 0.0;
    from_box(L, xF_, x, s);
    return total;
  }

  template <typename T>
  std::vector<Typed<T>>& typed();

  // descriptors of the separable transfer passes of level l (restriction
  // l -> l-1 and prolongation l-1 -> l), as run by restrict_ and prolong
  template <typename T, typename PD>
  void pass_descs(int l, std::vector<PD>* rp, std::vector<PD>* pp, int i) {
    auto& DD = typed<T>();
    const Common& F = com_[l];
    const Common& Cc = com_[l - 1];
    Typed<T>& D = DD[l];
    const int nf = F.n, nc = Cc.n, Wr = 4 * P + 1, Wp = P + 1;
    auto set = [](PD& q, const void* in, void* out, int in0, int in1, int out0, int out1, int axis,
                  const int* lo, const int* ext, const int* col, const void* wt, int W, const uint8_t* mask) {
      q.in = in;
      q.out = out;
      q.in0 = in0;
      q.in1 = in1;
      q.out0 = out0;
      q.out1 = out1;
      q.axis = axis;
      q.W = W;
      for (int k = 0; k < 3; ++k) {
        q.lo[k] = lo[k];
        q.ext[k] = ext[k];
      }
      q.col = col;
      q.wt = wt;
      q.mask = mask;
    };
    if (DIM == 3) {
      int lo1[3] = {Cc.bb_lo[0], F.bb_lo[1], F.bb_lo[2]};
      int ex1[3] = {Cc.bb_hi[0] - Cc.bb_lo[0] + 1, F.bb_hi[1] - F.bb_lo[1] + 1, F.bb_hi[2] - F.bb_lo[2] + 1};
      set(rp[0][i], D.r, D.t1, nf, nf, nc, nf, 0, lo1, ex1, F.res_col, D.res_w, Wr, nullptr);
      int lo2[3] = {Cc.bb_lo[0], Cc.bb_lo[1], F.bb_lo[2]};
      int ex2[3] = {ex1[0], Cc.bb_hi[1] - Cc.bb_lo[1] + 1, ex1[2]};
      set(rp[1][i], D.t1, D.t2, nc, nf, nc, nc, 1, lo2, ex2, F.res_col, D.res_w, Wr, nullptr);
      int lo3[3] = {Cc.bb_lo[0], Cc.bb_lo[1], Cc.bb_lo[2]};
      int ex3[3] = {ex1[0], ex2[1], Cc.bb_hi[2] - Cc.bb_lo[2] + 1};
      set(rp[2][i], D.t2, DD[l - 1].b, nc, nc, nc, nc, 2, lo3, ex3, F.res_col, D.res_w, Wr, Cc.nact);
      int plo1[3] = {F.bb_lo[0], Cc.bb_lo[1], Cc.bb_lo[2]};
      int pex1[3] = {F.bb_hi[0] - F.bb_lo[0] + 1, Cc.bb_hi[1] - Cc.bb_lo[1] + 1, Cc.bb_hi[2] - Cc.bb_lo[2] + 1};
      set(pp[0][i], DD[l - 1].x, D.t3, nc, nc, nf, nc, 0, plo1, pex1, F.pro_col, D.pro_w, Wp, nullptr);
      int plo2[3] = {F.bb_lo[0], F.bb_lo[1], Cc.bb_lo[2]};
      int pex2[3] = {pex1[0], F.bb_hi[1] - F.bb_lo[1] + 1, pex1[2]};
      set(pp[1][i], D.t3, D.t4, nf, nc, nf, nf, 1, plo2, pex2, F.pro_col, D.pro_w, Wp, nullptr);
      int plo3[3] = {F.bb_lo[0], F.bb_lo[1], F.bb_lo[2]};
      int pex3[3] = {pex1[0], pex2[1], F.bb_hi[2] - F.bb_lo[2] + 1};
      set(pp[2][i], D.t4, D.x, nf, nf, nf, nf, 2, plo3, pex3, F.pro_col, D.pro_w, Wp, F.nact);
    } else {
      int lo1[3] = {Cc.bb_lo[0], F.bb_lo[1], 0};
      int ex1[3] = {Cc.bb_hi[0] - Cc.bb_lo[0] + 1, F.bb_hi[1] - F.bb_lo[1] + 1, 1};
      set(rp[0][i], D.r, D.t1, nf, nf, nc, nf, 0, lo1, ex1, F.res_col, D.res_w, Wr, nullptr);
      int lo2[3] = {Cc.bb_lo[0], Cc.bb_lo[1], 0};
      int ex2[3] = {ex1[0], Cc.bb_hi[1] - Cc.bb_lo[1] + 1, 1};
      set(rp[1][i], D.t1, DD[l - 1].b, nc, nf, nc, nc, 1, lo2, ex2, F.res_col, D.res_w, Wr, Cc.nact);
      int plo1[3] = {F.bb_lo[0], Cc.bb_lo[1], 0};
      int pex1[3] = {F.bb_hi[0] - F.bb_lo[0] + 1, Cc.bb_hi[1] - Cc.bb_lo[1] + 1, 1};
      set(pp[0][i], DD[l - 1].x, D.t3, nc, nc, nf, nc, 0, plo1, pex1, F.pro_col, D.pro_w, Wp, nullptr);
      int plo2[3] = {F.bb_lo[0], F.bb_lo[1], 0};
      int pex2[3] = {pex1[0], F.bb_hi[1] - F.bb_lo[1] + 1, 1};
      set(pp[1][i], D.t3, D.x, nf, nc, nf, nf, 1, plo2, pex2, F.pro_col, D.pro_w, Wp, F.nact);
    }
  }

 private:
  static constexpr int kDotBlocks = 512;
 public:
  // when no patch can exceed 64 DoFs, (2p+1)^d <= 64 (2D Q1-Q3, 3D Q1), one
  // warp solves a patch, one or two rows per lane, from entry lists;
  // otherwise (3D Q2) the warp-per-patch record kernel (k_cut_warp) takes
  // the patches.  The choice depends on (d, p) only, so a problem solved
  // alone and inside a batch runs the same arithmetic.
  static constexpr bool kWarpCut = (DIM == 2 ? (2 * P + 1) * (2 * P + 1) : (2 * P + 1) * (2 * P + 1) * (2 * P + 1)) <= 64;
  // Record kernel: kCutWarps independent warps per block, each with its own
  // stage; the records are read from global memory, prefetched into L2 per
  // patch when its loads are issued (variant 1 of the cut family), one patch
  // ahead (variant 3), or not (variant 2); the same arithmetic.  The grid:
  // every block the occupancy calculator lets reside, at most one warp per
  // patch.  A colour of fewer than kCutWarps patches per SM (the coarse
  // levels, where a launch lasts about one patch's chain of dependent steps)
  // runs one patch per block at a time with the block's kCutTeam warps
  // working on it together (k_cut_team), which shortens that chain and
  // spreads the patches over the SMs (whose warps share one FP64 pipe);
  // variant 4 keeps kCutWarps warps per block, one patch each, at every
  // size, variant 5 runs such colours one warp per block.
  static constexpr int kCutWarps = 8;
  static constexpr int kCutTeam = 4;
  struct PipePlan {
    int grid = 0, smem = 0, prefetch = 1, wpb = kCutWarps;
    bool team = false;
  };
  template <typename T>
  PipePlan pipe_plan(const Common& c, int colour) const {
    PipePlan pl;
    const int cnt = c.cut_start[colour + 1] - c.cut_start[colour];
    pl.prefetch = var_cut_ == 1 ? 1 : var_cut_ == 2 ? 0 : var_cut_ == 3 ? 2 : kCutPrefetch;
    const bool small = (cnt < kCutWarps * sms_ && var_cut_ != 4) || var_cut_ == 6;
    pl.team = small && var_cut_ != 5;
    pl.wpb = small ? (pl.team ? kCutTeam : 1) : kCutWarps;
    pl.smem = (pl.team ? 1 : pl.wpb) * warp_stage_bytes<DIM, P, T>();
    int nb = 0;
    if (pl.team)
      CUTMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cut_team<DIM, P, T, kCutTeam>, 32 * kCutTeam,
                                                               pl.smem));
    else if (pl.wpb == 1)
      CUTMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cut_warp<DIM, P, T, 1>, 32, pl.smem));
    else
      CUTMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cut_warp<DIM, P, T, kCutWarps>, 32 * kCutWarps,
                                                               pl.smem));
    const int per_block = pl.team ? 1 : pl.wpb;
    pl.grid = std::max(1, std::min((cnt + per_block - 1) / per_block, std::max(1, nb) * sms_));
    return pl;
  }
  template <typename T>
  PipeLevel<T> pipe_level(const Common& c, Typed<T>& D, T* x, const T* b) const {
    PipeLevel<T> L;
    L.op = D.op;
    L.x = x;
    L.b = b;
    L.vert = c.cutv;
    L.cnt = c.cutn;
    L.moff = c.cutmo;
    L.members = c.members32;
    L.ioff = c.pioff;
    L.nit = c.pnit;
    L.items = c.pitems;
    L.pk = c.ppk;
    L.gmask = c.pgmask;
    L.roff = c.proff;
    L.rec = D.rec;
    L.kp = D.kp;
    L.ksc = D.ksc;
    L.gboff = c.gboff;
    L.Gb = D.Gb;
    L.geoff = c.geoff;
    L.gent = c.gent;
    return L;
  }
 private:
  static constexpr int kVecBlocks = 1024;
  int sms_ = 152;
  std::vector<double> lam_;        // Chebyshev smoother: lambda_max(D^{-1} A_l) estimates
  std::vector<double*> gV_, gZ_;  // GMRES basis (box vectors), allocated on first use
  double* gW_ = nullptr;
  double* gsc_ = nullptr;

  const Hierarchy& H_;
  cudaStream_t setup_stream_ = nullptr;  // the stream of cf_setup (uploads, power iteration)
  DevPool pool_;
  int64_t launches_ = 0;
  struct Prof {
    int kind = 0;  // 1 cut-patch solve, 2 interior-patch step, 3 apply (bulk), 4 apply (boundary),
                   // 5 ghost-face moments
    int level = -1;  // only launches on this level (-1: all levels)
    std::vector<cudaEvent_t> ev;
    int used = 0;
    int64_t n = 0;
    double flops = 0.0, bytes = 0.0;
  } prof_;

  // CUDA graphs: a fixed launch sequence is captured once on the internal
  // stream cap_ and replayed on the caller's stream (graph launches are legal
  // on every stream, capture is not legal on the legacy default stream).
  // Disabled while a kernel family is being event-timed.
  struct GraphEntry {
    cudaGraphExec_t exec;
    int64_t launches;
  };
  using GraphKey = std::tuple<int, const void*, const void*>;
  std::map<GraphKey, GraphEntry> graphs_;
  cudaStream_t cap_ = nullptr;
  bool use_graphs_ = true;

  int var_int_ = 0, var_cut_ = 0, var_op_ = 0;  // forced launch variants (0: automatic)
  // operator on bulk positions: 1 element-matrix form, 2 sum-factorised
  // (automatic: sum-factorised in FP64, where the flop count sets the time)
  template <typename T>
  bool use_sumfact() const {
    return var_op_ == 2 || (var_op_ == 0 && sizeof(T) == 8);
  }
  int spin_ = kTmaSpin;            // polls of the tensor-core interior kernel's wait on its MMA

  void drop_graphs() {
    for (auto& kv : graphs_) cudaGraphExecDestroy(kv.second.exec);
    graphs_.clear();
  }

  template <class F>
  void run_graph(const GraphKey& key, cudaStream_t s, F&& body) {
    if (!use_graphs_ || prof_.kind != 0) {
      body(s);
      return;
    }
    auto it = graphs_.find(key);
    if (it == graphs_.end()) {
      const int64_t l0 = launches_;
      cudaGraph_t g = nullptr;
      CUTMG_CUDA(cudaStreamBeginCapture(cap_, cudaStreamCaptureModeThreadLocal));
      try {
        body(cap_);
      } catch (...) {
        cudaStreamEndCapture(cap_, &g);
        if (g) cudaGraphDestroy(g);
        launches_ = l0;
        throw;
      }
      CUTMG_CUDA(cudaStreamEndCapture(cap_, &g));
      cudaGraphExec_t ex = nullptr;
      cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) throw CudaError(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
      it = graphs_.emplace(key, GraphEntry{ex, launches_ - l0}).first;
      launches_ = l0;
    }
    CUTMG_CUDA(cudaGraphLaunch(it->second.exec, s));
    launches_ += it->second.launches;
  }

  void count_launch(const char* what) {
    launch_check(what);
    ++launches_;
  }
  // event pair around a launch of the profiled family (on the launching stream)
  void prof_mark(int kind, int level, cudaStream_t s) {
    if (prof_.kind != kind || (prof_.level >= 0 && prof_.level != level)) return;
    if (prof_.used == (int)prof_.ev.size()) {
      cudaEvent_t e;
      CUTMG_CUDA(cudaEventCreate(&e));
      prof_.ev.push_back(e);
    }
    CUTMG_CUDA(cudaEventRecord(prof_.ev[prof_.used++], s));
  }
  void prof_work(int kind, int level, double flops, double bytes) {
    if (prof_.kind != kind || (prof_.level >= 0 && prof_.level != level)) return;
    prof_.n += 1;
    prof_.flops += flops;
    prof_.bytes += bytes;
  }
  std::vector<Common> com_;
  std::vector<Typed<double>> d64_;
  std::vector<Typed<float>> d32_;
  double *xF_, *rF_, *pF_, *qF_, *zF_, *bF_, *tF_, *aux_, *aux2_, *part_, *sc_;
  int* err_ = nullptr;  // set by kernels whose bounded waits ran out
  double* host_sc_ = nullptr;
  double* rhs_d_ = nullptr;
  float *bL32_ = nullptr, *xL32_ = nullptr;

  void check_smooth_level(int l) const {
    if (l < 1 || l >= n_levels()) throw std::invalid_argument("level must be in [1, n_levels)");
  }

  template <typename T>
  void fill_typed(const HostLevel& h, Typed<T>& D, const Common& c, int l) {
    D.op.N = h.N;
    D.op.n = h.n;
    D.op.cflag = c.cflag;
    D.op.cut_id = c.cut_id;
    D.op.cutmat = pool_.upload<T>(h.cutmat);
    D.op.face_id = c.face_id;
    D.op.G = pool_.alloc<T>((size_t)std::max<int64_t>(1, (int64_t)h.ghost_faces.size()) * P * (DIM == 2 ? P + 1 : (P + 1) * (P + 1)));
    D.op.Kref = pool_.upload<T>(h.Kref);
    if (!kWarpCut) {
      constexpr int NB = Shape<DIM, P>::NB, NBP = PipeGeo<DIM, P>::NBP;
      std::vector<T> kp((size_t)NB * NBP, T(0));
      for (int i = 0; i < NB; ++i)
        for (int j = 0; j < NB; ++j) kp[(size_t)i * NBP + j] = (T)h.Kunit[(size_t)i * NB + j];
      D.kp = pool_.upload<T>(kp);
      D.ksc = (T)h.kscale;
    }
    for (int m = 0; m < 4; ++m) {
      for (int i = 0; i < 9; ++i) D.op.dvec[m][i] = (T)h.dvec[m][i];
      D.op.coef[m] = (T)h.coef[m];
    }
    for (int a = 0; a < 5; ++a)
      for (int b2 = 0; b2 < 5; ++b2) D.op.Mhat[a][b2] = (T)h.Mhat[a][b2];
    for (int i = 0; i < M; ++i) {
      for (int j = 0; j < C; ++j) {
        D.fd.Mr[i][j] = (T)h.Mr[i * C + j];
        D.fd.Kr[i][j] = (T)h.Kr[i * C + j];
      }
      for (int j = 0; j < M; ++j) D.fd.S[i][j] = (T)h.S[i * M + j];
      D.fd.lam[i] = (T)h.lam[i];
    }
    // the eigenvalue sums of the fast-diagonalised solve, inverted once
    for (int c = 0; c < (DIM == 3 ? M : 1); ++c)
      for (int b2 = 0; b2 < M; ++b2)
        for (int a = 0; a < M; ++a) {
          const double den = h.lam[a] + h.lam[b2] + (DIM == 3 ? h.lam[c] : 0.0);
          D.fd.dinv[a + M * (b2 + M * c)] = (T)(1.0 / den);
        }
    // assembled 1D rows by residue (column i - p + s at tap s) from the
    // two-cell rows: residue 0 = the middle row, residue r = row r of cell 0
    for (int r = 0; r < 4; ++r)
      for (int t = 0; t < 9; ++t) D.sf.Mrow[r][t] = D.sf.Krow[r][t] = T(0);
    for (int r = 0; r < P; ++r) {
      const int row = r == 0 ? P - 1 : r - 1, sh = r == 0 ? 0 : P - r;
      for (int t = 0; t <= 2 * P; ++t) {
        if (t + sh > 2 * P) continue;
        D.sf.Mrow[r][t + sh] = (T)h.Mr[row * C + t];
        D.sf.Krow[r][t + sh] = (T)h.Kr[row * C + t];
      }
    }
    {
      using G = DenseGeo<DIM, P>;
      std::vector<float> wt((size_t)G::NC * G::NR4, 0.f);
      if (l > 0)
        for (int i = 0; i < G::NI; ++i)
          for (int k = 0; k < G::NC; ++k) wt[(size_t)k * G::NR4 + i] = (float)h.Wcart[(size_t)i * G::NC + k];
      D.dense_d = pool_.upload<float>(wt);
      if (std::is_same<T, float>::value && l > 0) {
        using TG = TcGeo<DIM, P>;
        std::vector<float> bo((size_t)TG::B_BYTES / 4, 0.f);
        for (int i = 0; i < G::NI; ++i)
          for (int k = 0; k < G::NC; ++k)
            bo[(size_t)umma_off<TG::NP>(i, k) / 4] = round_tf32((float)h.Wcart[(size_t)i * G::NC + k]);
        D.tc_b = pool_.upload<float>(bo);
      }
    }
    if (kWarpCut) {
      D.inv = pool_.upload<T>(h.inv);
    } else {
      if (!h.inv_on_device) {
        D.rec = pool_.upload<T>(h.rec);
      } else if (std::is_same<T, double>::value) {
        // A_j (rows padded to 4) in the records: inverted here, in FP64
        D.rec = pool_.upload<T>(h.rec);
        device_inverses(h, reinterpret_cast<double*>(D.rec));
      } else {
        // the mixed form's records: the FP64 device records rounded
        D.rec = pool_.alloc<T>((size_t)std::max<int64_t>(1, h.n_rec), false);
        k_to_float<<<1024, 256, 0, setup_stream_>>>(d64_[l].rec, reinterpret_cast<float*>(D.rec), h.n_rec);
        launch_check("record conversion");
      }
      D.Gb = pool_.alloc<T>((size_t)std::max(1, h.cut_gboff.empty() ? 0 : h.cut_gboff.back()) * P *
                            FaceGeo<DIM, P>::NT);
    }
    D.pro_w = l > 0 ? pool_.upload<T>(h.pro_w) : nullptr;
    D.res_w = l > 0 ? pool_.upload<T>(h.res_w) : nullptr;
    D.coarse_inv = l == 0 ? pool_.upload<T>(h.coarse_inv) : nullptr;
    D.x = pool_.alloc<T>(c.nbox);
    D.b = pool_.alloc<T>(c.nbox);
    D.r = pool_.alloc<T>(c.nbox);
    if (H_.prm.smoother == 1 && l > 0) {
      std::vector<T> dv((size_t)c.nbox, T(0));
      for (size_t i = 0; i < h.dofs.size(); ++i) dv[(size_t)h.dofs[i]] = (T)(1.0 / h.diag[i]);
      D.dinv = pool_.upload<T>(dv);
      D.xp = pool_.alloc<T>(c.nbox);
    }
    D.t1 = D.t2 = D.t3 = D.t4 = nullptr;
    if (l > 0) {
      const int64_t nf = h.n, nc = H_.levels[l - 1].n;
      if (DIM == 3) {
        D.t1 = pool_.alloc<T>(nc * nf * nf);
        D.t2 = pool_.alloc<T>(nc * nc * nf);
        D.t3 = pool_.alloc<T>(nf * nc * nc);
        D.t4 = pool_.alloc<T>(nf * nf * nc);
      } else {
        D.t1 = pool_.alloc<T>(nc * nf);
        D.t3 = pool_.alloc<T>(nf * nc);
      }
    }
  }

  // the cut-patch inverses of a level from the assembled A_j in the FP64
  // records (k_patch_inverse, in place)
  void device_inverses(const HostLevel& h, double* rec) {
    const int64_t ncp = (int64_t)h.cut_vert.size();
    if (ncp == 0) return;
    int mmax = 1;
    for (int m : h.cut_n) mmax = std::max(mmax, m);
    const int ld = mmax | 1;
    const size_t dyn = sizeof(double) * ((size_t)ld * ld + ld);
    CUTMG_CUDA(cudaFuncSetAttribute(k_patch_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int* cnt = pool_.upload<int>(h.cut_n);
    int64_t* roff = pool_.upload<int64_t>(h.cut_roff);
    k_patch_inverse<<<(int)std::min<int64_t>(ncp, 8 * sms_), 128, dyn, setup_stream_>>>(rec, roff, cnt, (int)ncp, ld,
                                                                                         err_);
    launch_check("cut-patch inverses");
    int e = 0;
    CUTMG_CUDA(cudaMemcpyAsync(&e, err_, sizeof(int), cudaMemcpyDeviceToHost, setup_stream_));
    CUTMG_CUDA(cudaStreamSynchronize(setup_stream_));
    if (e) throw std::runtime_error("a cut-patch matrix is not positive definite (device Cholesky, level N=" +
                                    std::to_string(h.N) + ")");
  }

  void upload_level(int l) {
    const HostLevel& h = H_.levels[l];
    Common& c = com_[l];
    c.N = h.N;
    c.n = h.n;
    c.nbox = (int64_t)h.nact.size();
    c.ndof = (int64_t)h.dofs.size();
    c.cflag = pool_.upload<uint8_t>(h.cflag);
    c.cut_id = pool_.upload<int>(h.cut_id);
    c.nact = pool_.upload<uint8_t>(h.nact);
    c.dofs = pool_.upload<int64_t>(h.dofs);
    c.bulk = pool_.upload<int>(h.bulk_pos);
    c.nbulk = (int)h.bulk_pos.size();
    {
      // boundary nodes grouped by the number of directions in which they lie
      // on a cell boundary (8, 4, 2 or 1 cells in 3D), lattice order within
      // a group: a warp's rows then loop over the same number of cells and
      // faces (each node's row is formed alone, so the order changes no
      // result)
      std::vector<int> bnd = h.bnd_node;
      auto on_planes = [&](int node) {
        int c = 0, u = node;
        for (int k = 0; k < DIM; ++k) {
          c += (u % h.n) % P == 0;
          u /= h.n;
        }
        return c;
      };
      std::stable_sort(bnd.begin(), bnd.end(), [&](int a, int b) { return on_planes(a) > on_planes(b); });
      c.bnd = pool_.upload<int>(bnd);
      c.nbnd = (int)bnd.size();
    }
    {
      // work model of one boundary-row launch (k_apply_bnd): per node its
      // active cells' rows (2 NB flops; NB values of x, plus the NB entries
      // of a cut cell's row) and its ghost faces (2 p flops, p moments);
      // b read and y written
      double fl = 0.0, sc = 0.0;
      const int N = h.N, n = h.n;
      for (int node : h.bnd_node) {
        int idx[3] = {0, 0, 0}, u = node;
        for (int k = 0; k < DIM; ++k) {
          idx[k] = u % n;
          u /= n;
        }
        int cc[3][2], nopt[3];
        for (int k = 0; k < DIM; ++k) {
          const int a = idx[k] / P, r = idx[k] - a * P;
          int m = 0;
          if (r == 0) {
            if (a - 1 >= 0) cc[k][m++] = a - 1;
            if (a < N) cc[k][m++] = a;
          } else {
            cc[k][m++] = a;
          }
          nopt[k] = m;
        }
        const int tot = DIM == 2 ? nopt[0] * nopt[1] : nopt[0] * nopt[1] * nopt[2];
        for (int t = 0; t < tot; ++t) {
          int q = t, cell = 0, st = 1;
          for (int k = 0; k < DIM; ++k) {
            cell += cc[k][q % nopt[k]] * st;
            q /= nopt[k];
            st *= N;
          }
          const uint8_t f = h.cflag[cell];
          if (!(f & kFlagActive)) continue;
          fl += 2.0 * NB;
          sc += NB + ((f & kFlagCut) ? NB : 0);
        }
        for (int k = 0; k < DIM; ++k) {
          const int a = idx[k] / P, r = idx[k] - a * P;
          const int Llo = std::max(0, r == 0 ? a - 2 : a - 1), Lhi = std::min(a, N - 2);
          int td[2] = {0, 0}, q2 = 0;
          for (int j = 0; j < DIM; ++j)
            if (j != k) td[q2++] = j;
          const int n0 = nopt[td[0]], n1 = DIM == 3 ? nopt[td[1]] : 1;
          for (int Lk = Llo; Lk <= Lhi; ++Lk)
            for (int u0 = 0; u0 < n0; ++u0)
              for (int u1 = 0; u1 < n1; ++u1) {
                int c[3] = {0, 0, 0};
                c[k] = Lk;
                c[td[0]] = cc[td[0]][u0];
                if (DIM == 3) c[td[1]] = cc[td[1]][u1];
                const int64_t cell = c[0] + (int64_t)N * (c[1] + (DIM == 3 ? (int64_t)N * c[2] : 0));
                if (h.face_id[(size_t)cell * DIM + k] < 0) continue;
                fl += 2.0 * P;
                sc += P;
              }
        }
        sc += 2.0;
      }
      c.bnd_work[0] = fl;
      c.bnd_work[1] = sc;
      c.bnd_work[2] = 4.0 * (double)h.bnd_node.size();
    }
    {
      // tiles of the sum-factorised operator: the bulk positions grouped by
      // the tile of SfGeo positions that contains them
      using SG = SfGeo<DIM, P>;
      const int np = h.N + 1;
      std::map<int64_t, std::array<uint32_t, SG::MASKW>> tm;
      for (int q : h.bulk_pos) {
        int a[3] = {0, 0, 0}, t = q;
        for (int k = 0; k < DIM; ++k) {
          a[k] = t % np;
          t /= np;
        }
        const int T3[3] = {SG::TX, SG::TY, SG::TZ};
        int ti[3] = {0, 0, 0}, loc[3] = {0, 0, 0};
        for (int k = 0; k < DIM; ++k) {
          ti[k] = (a[k] - 1) / T3[k];
          loc[k] = (a[k] - 1) - ti[k] * T3[k];
        }
        const int64_t key = (int64_t)(1 + ti[0] * SG::TX) +
                            (int64_t)np * ((1 + ti[1] * SG::TY) + (int64_t)np * (DIM == 3 ? 1 + ti[2] * SG::TZ : 0));
        const int bit = loc[0] + SG::TX * (loc[1] + SG::TY * loc[2]);
        auto it = tm.find(key);
        if (it == tm.end()) it = tm.emplace(key, std::array<uint32_t, SG::MASKW>{}).first;
        it->second[bit / 32] |= 1u << (bit % 32);
      }
      std::vector<int> tiles;
      std::vector<uint32_t> masks;
      for (auto& kv : tm) {
        tiles.push_back((int)kv.first);
        masks.insert(masks.end(), kv.second.begin(), kv.second.end());
      }
      c.nsf = (int)tiles.size();
      c.sf_tiles = pool_.upload<int>(tiles);
      c.sf_masks = pool_.upload<uint32_t>(masks);
    }
    c.faces = pool_.upload<int>(h.ghost_faces);
    c.nfaces = (int)h.ghost_faces.size();
    c.face_id = pool_.upload<int>(h.face_id);
    c.fofs = pool_.upload<int>(h.fofs);
    c.fent = pool_.upload<int>(h.fent);
    c.cfaces = pool_.upload<int>(h.cfaces);
    c.cf_start = h.cf_start;
    c.mnode = pool_.upload<int>(h.member_node);
    c.cart = pool_.upload<int>(h.cart_vert);
    c.cart_start = h.cart_start;
    c.cutv = pool_.upload<int>(h.cut_vert);
    c.cutn = pool_.upload<int>(h.cut_n);
    c.cutmo = pool_.upload<int>(h.cut_moff);
    c.cutio = pool_.upload<int64_t>(h.cut_ioff);
    c.cutfo = pool_.upload<int>(h.cut_fo);
    c.cutcell = pool_.upload<int>(h.cut_cell);
    c.citoff = pool_.upload<int>(h.cut_item_off);
    c.citems = pool_.upload<uint8_t>(h.cut_items);
    c.members = pool_.upload<uint16_t>(h.members);
    c.cut_start = h.cut_start;
    c.cut_maxm2 = h.cut_maxm2;
    c.cut_maxit = h.cut_maxit;
    c.nmembers = (int64_t)h.members.size();
    if (!kWarpCut) {
      std::vector<int> m32(h.members.begin(), h.members.end());
      c.members32 = pool_.upload<int>(m32);
      // row items in 4-byte aligned runs per patch
      const int64_t ncp = (int64_t)h.cut_vert.size();
      std::vector<int> io(ncp), ni(ncp);
      std::vector<uint32_t> words;
      for (int64_t j = 0; j < ncp; ++j) {
        const int i0 = h.cut_item_off[j], i1 = h.cut_item_off[j + 1];
        io[j] = (int)words.size();
        ni[j] = i1 - i0;
        for (int q = i0; q < i1; q += 4) {
          uint32_t w = 0;
          for (int b = 0; b < 4 && q + b < i1; ++b) w |= (uint32_t)h.cut_items[q + b] << (8 * b);
          words.push_back(w);
        }
      }
      c.pioff = pool_.upload<int>(io);
      c.pnit = pool_.upload<int>(ni);
      c.pitems = pool_.upload<uint32_t>(words);
      c.ppk = pool_.upload<int>(h.cut_pk);
      c.pgmask = pool_.upload<uint64_t>(h.cut_gmask);
      c.proff = pool_.upload<int64_t>(h.cut_roff);
      c.cut_maxrec = h.cut_maxrec;
      c.gboff = pool_.upload<int>(h.cut_gboff);
      c.geoff = pool_.upload<int>(h.cut_geoff);
      c.gent = pool_.upload<uint16_t>(h.cut_gent);
      c.bf_face = pool_.upload<int>(h.bf_face);
      c.bf_dst = pool_.upload<int>(h.bf_dst);
      c.bf_start = h.bf_start;
    }
    c.pro_col = l > 0 ? pool_.upload<int>(h.pro_col) : nullptr;
    c.res_col = l > 0 ? pool_.upload<int>(h.res_col) : nullptr;
    if (l == 0) {
      std::vector<int> nodes(h.dofs.begin(), h.dofs.end());
      c.coarse_nodes = pool_.upload<int>(nodes);
    } else {
      c.coarse_nodes = nullptr;
    }
    for (int k = 0; k < 3; ++k) {
      c.bb_lo[k] = h.bb_lo[k];
      c.bb_hi[k] = h.bb_hi[k];
    }
    c.region.n0 = h.n;
    c.region.n1 = DIM >= 2 ? h.n : 1;
    c.region.lo0 = h.bb_lo[0];
    c.region.lo1 = h.bb_lo[1];
    c.region.lo2 = DIM == 3 ? h.bb_lo[2] : 0;
    c.region.e0 = h.bb_hi[0] - h.bb_lo[0] + 1;
    c.region.e1 = h.bb_hi[1] - h.bb_lo[1] + 1;
    c.region.e2 = DIM == 3 ? h.bb_hi[2] - h.bb_lo[2] + 1 : 1;
    fill_typed<double>(h, d64_[l], c, l);
    fill_typed<float>(h, d32_[l], c, l);
    if (l == (int)H_.levels.size() - 1) rhs_d_ = pool_.upload<double>(H_.rhs);
  }

  // compact (FP64) <-> box (T): the box is zeroed first so that inactive
  // nodes are zero whatever the buffer held before
  template <typename T>
  void to_box(int l, const double* in, T* box, cudaStream_t s) {
    const Common& c = com_[l];
    CUTMG_CUDA(cudaMemsetAsync(box, 0, sizeof(T) * c.nbox, s));
    k_scatter<T, double><<<std::min(blocks_for(c.ndof, 256), 4096), 256, 0, s>>>(c.dofs, c.ndof, in, box);
    count_launch("scatter");
  }
  template <typename T>
  void from_box(int l, const T* box, double* out, cudaStream_t s) {
    const Common& c = com_[l];
    k_gather<double, T><<<std::min(blocks_for(c.ndof, 256), 4096), 256, 0, s>>>(c.dofs, c.ndof, box, out);
    count_launch("gather");
  }

  // a bounded wait inside a kernel ran out: report and clear the flag
  void check_err(cudaStream_t s) {
    int h = 0;
    CUTMG_CUDA(cudaMemcpyAsync(&h, err_, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUTMG_CUDA(cudaStreamSynchronize(s));
    if (h) {
      CUTMG_CUDA(cudaMemsetAsync(err_, 0, sizeof(int), s));
      throw TimeoutError("a bounded wait ran out in a kernel (TMA copy of a patch inverse or tensor-core MMA completion)");
    }
  }

  // CUDA-event timer on one stream
  struct Timer {
    cudaStream_t s;
    cudaEvent_t e0, e1;
    explicit Timer(cudaStream_t st) : s(st) {
      CUTMG_CUDA(cudaEventCreate(&e0));
      CUTMG_CUDA(cudaEventCreate(&e1));
      CUTMG_CUDA(cudaEventRecord(e0, s));
    }
    float stop() {
      float ms = 0.f;
      CUTMG_CUDA(cudaEventRecord(e1, s));
      CUTMG_CUDA(cudaEventSynchronize(e1));
      CUTMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      return ms;
    }
    ~Timer() {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
  };

  // ||b - A x|| of the finest-level iterate (FP64)
  double true_residual(cudaStream_t s) {
    const int L = n_levels() - 1;
    apply<double>(L, d64_[L], xF_, bF_, tF_, s);
    dot(com_[L].region, tF_, tF_, sc_ + 5, s);
    return std::sqrt(read_scalar(5, s));
  }

  // Krylov basis of GMRES(m): v_0..v_m, z_0..z_{m-1}, w and m + 2 scalars
  void gmres_storage(int m) {
    if ((int)gZ_.size() >= m) return;
    const int64_t nb = com_.back().nbox;
    while ((int)gV_.size() < m + 1) gV_.push_back(pool_.alloc<double>(nb));  // zeroed
    while ((int)gZ_.size() < m) gZ_.push_back(pool_.alloc<double>(nb));
    if (!gW_) gW_ = pool_.alloc<double>(nb);
    gsc_ = pool_.alloc<double>(m + 2);
  }

  double read_scalar(int i, cudaStream_t s) {
    CUTMG_CUDA(cudaMemcpyAsync(host_sc_ + i, sc_ + i, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUTMG_CUDA(cudaStreamSynchronize(s));
    return host_sc_[i];
  }

  void dot(const Region& R, const double* a, const double* b, double* out, cudaStream_t s) {
    k_dot_partial<<<kDotBlocks, 256, 0, s>>>(R, a, b, part_);
    count_launch("dot partial");
    k_dot_final<<<1, 256, 0, s>>>(part_, kDotBlocks, out);
    count_launch("dot final");
  }

  // y = A x or y = b - A x on level l (box layout, precision T)
  template <typename T>
  void apply(int l, Typed<T>& D, const T* x, const T* b, T* y, cudaStream_t s) {
    const Common& c = com_[l];
    if (c.nbulk > 0) {
      prof_mark(3, l, s);
      if (use_sumfact<T>()) {
        using SG = SfGeo<DIM, P>;
        int nb = 0;  // resident blocks per SM (shared memory bound)
        CUTMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_apply_sf<DIM, P, T>, 256,
                                                                 SG::ELEMS * sizeof(T)));
        k_apply_sf<DIM, P, T><<<std::min(c.nsf, std::max(1, nb) * sms_), 256, SG::ELEMS * sizeof(T), s>>>(
            D.sf, c.N, c.n, x, b, y, c.sf_tiles, c.sf_masks, c.nsf);
      } else {
        k_apply_bulk<DIM, P, T><<<blocks_for(c.nbulk, 128), 128, 0, s>>>(D.op, x, b, y, c.bulk, c.nbulk);
      }
      count_launch("apply bulk");
      prof_mark(3, l, s);
      // per position: the (cell, owned node) pairs that run are (p+1)^d (a
      // cell s contributes the owned nodes with alpha_k = 0 wherever s_k = 1),
      // NB terms each; x read and y written once per owned node (+ b)
      constexpr int NO = Shape<DIM, P>::NO;
      // flops: the element-matrix form's (p+1)^d (cell, node) pairs of NB
      // terms; the sum-factorised form per owned node 2 taps per product
      // of each pass (3D: 2 + 3 + 2 products, 2D: 2 + 2) and the combination
      constexpr int PAIRS = (DIM == 2) ? (P + 1) * (P + 1) : (P + 1) * (P + 1) * (P + 1);
      constexpr double TAPS = (2.0 * P + 1 + (P - 1) * (P + 1.0)) / P;
      const double fl = use_sumfact<T>() ? (double)NO * (2.0 * TAPS * (DIM == 3 ? 7 : 4) + 2.0) : 2.0 * PAIRS * NB;
      prof_work(3, l, fl * c.nbulk, (double)c.nbulk * (NO * (b ? 3 : 2) * sizeof(T) + 4));
    }
    if (c.nbnd > 0) {
      face_moments<T>(l, D, x, s);
      prof_mark(4, l, s);
      k_apply_bnd<DIM, P, T><<<blocks_for(c.nbnd, 128), 128, 0, s>>>(D.op, x, b, y, c.bnd, c.nbnd);
      count_launch("apply boundary");
      prof_mark(4, l, s);
      prof_work(4, l, c.bnd_work[0], c.bnd_work[1] * sizeof(T) + c.bnd_work[2]);
    }
  }

  // jump moments of every ghost face of level l for the vector x
  // (colour < 0: all of them; else only the faces the colour's cut patches need)
  template <typename T>
  void face_moments(int l, Typed<T>& D, const T* x, cudaStream_t s, int colour = -1) {
    const Common& c = com_[l];
    const int* ids = nullptr;
    int cnt = c.nfaces;
    if (colour >= 0) {
      ids = c.cfaces + c.cf_start[colour];
      cnt = c.cf_start[colour + 1] - c.cf_start[colour];
    }
    if (cnt <= 0) return;
    constexpr int PW = FaceGeo<DIM, P>::PER_WARP;
    prof_mark(5, l, s);
    k_face_moments<DIM, P, T><<<blocks_for(blocks_for(cnt, PW), 4), 128, 0, s>>>(D.op, x, c.faces, ids, cnt);
    count_launch("ghost face moments");
    prof_mark(5, l, s);
    {
      constexpr int NTF = FaceGeo<DIM, P>::NT;
      const double flf = 2.0 * (2 * P + 1) * P * NTF + 2.0 * P * (P + 1) * NTF * (DIM - 1) + (double)P * NTF;
      prof_work(5, l, cnt * flf, cnt * (((2.0 * P + 1) * NTF + (double)P * NTF) * sizeof(T) + 8.0));
    }
  }

  // moments of the block-boundary ghost faces of the cut patches of a colour,
  // from x before the colour step, into the patches' moment slots
  template <typename T>
  void boundary_face_moments(int l, Typed<T>& D, const T* x, cudaStream_t s, int colour) {
    const Common& c = com_[l];
    const int f0 = c.bf_start[colour], cnt = c.bf_start[colour + 1] - f0;
    if (cnt <= 0) return;
    constexpr int PW = FaceGeo<DIM, P>::PER_WARP;
    prof_mark(5, l, s);
    k_face_moments_to<DIM, P, T><<<blocks_for(blocks_for(cnt, PW), 4), 128, 0, s>>>(
        D.op, x, c.faces, c.bf_face + f0, c.bf_dst + 2 * f0, cnt, D.Gb);
    count_launch("boundary ghost face moments");
    prof_mark(5, l, s);
    const auto& w = H_.levels[l].work_face[colour];
    prof_work(5, l, w[0], w[1] * sizeof(T) + w[2]);
  }

  template <typename T>
  void colour_step(int l, Typed<T>& D, int cut, int colour, T* x, const T* b, cudaStream_t s) {
    const Common& c = com_[l];
    if (!cut) {
      const int a0 = c.cart_start[colour], cnt = c.cart_start[colour + 1] - a0;
      if (cnt <= 0) return;
      prof_mark(2, l, s);
      if constexpr (std::is_same<T, float>::value)
      {
        constexpr int PPB = 128 / DenseGeo<DIM, P>::NPART;
        int v = var_int_;
        if (v == 0) v = 4;  // tensor cores (TF32 products, FP32 accumulation)
        if (v == 4)
          k_smooth_tc<DIM, P><<<std::min(blocks_for(cnt, 128), 2 * sms_), 256, TcGeo<DIM, P>::SMEM, s>>>(
              D.tc_b, c.N, c.n, x, b, c.cart + a0, cnt, err_, spin_);
        else if (v == 2)
          k_smooth_dense<DIM, P, 2><<<blocks_for(cnt, 256), 128, 0, s>>>(D.dense_d, c.N, c.n, x, b, c.cart + a0, cnt);
        else if (v == 1)
          k_smooth_dense<DIM, P, 1><<<blocks_for(cnt, 128), 128, 0, s>>>(D.dense_d, c.N, c.n, x, b, c.cart + a0, cnt);
        else
          k_smooth_dense_split<DIM, P><<<blocks_for(cnt, PPB), 128, 0, s>>>(D.dense_d, c.N, c.n, x, b,
                                                                          c.cart + a0, cnt);
      }
      else if (var_int_ == 2 || (var_int_ != 1 && cnt <= 4 * sms_))
        k_smooth_cart_cta<DIM, P, T><<<std::min(cnt, 16 * sms_), 128, 0, s>>>(D.fd, c.N, c.n, x, b, c.cart + a0, cnt);
      else
        k_smooth_cart<DIM, P, T, WARPS><<<blocks_for(cnt, 2 * WARPS), 32 * WARPS, 0, s>>>(
            D.fd, c.N, c.n, x, b, c.cart + a0, cnt);
      count_launch("smooth interior patches");
      prof_mark(2, l, s);
      const auto& w = H_.levels[l].work_cart[colour];
      prof_work(2, l, w[0], w[1] * sizeof(T) + w[2]);
    } else {
      const int a0 = c.cut_start[colour], cnt = c.cut_start[colour + 1] - a0;
      if (cnt <= 0) return;
      if (kWarpCut) face_moments<T>(l, D, x, s, colour);
      else boundary_face_moments<T>(l, D, x, s, colour);
      prof_mark(1, l, s);
      if (!kWarpCut) {
        const PipePlan pl = pipe_plan<T>(c, colour);
        if (pl.team)
          k_cut_team<DIM, P, T, kCutTeam><<<pl.grid, 32 * kCutTeam, pl.smem, s>>>(pipe_level<T>(c, D, x, b), a0, cnt,
                                                                                  pl.prefetch);
        else if (pl.wpb == 1)
          k_cut_warp<DIM, P, T, 1><<<pl.grid, 32, pl.smem, s>>>(pipe_level<T>(c, D, x, b), a0, cnt, pl.prefetch);
        else
          k_cut_warp<DIM, P, T, kCutWarps><<<pl.grid, 32 * kCutWarps, pl.smem, s>>>(pipe_level<T>(c, D, x, b), a0,
                                                                                   cnt, pl.prefetch);
      } else {
        k_cut_solve<DIM, P, T, WARPS><<<blocks_for(cnt, WARPS), 32 * WARPS, 0, s>>>(
            D.op, x, b, c.cutv + a0, c.cutn + a0, c.cutmo + a0, c.cutio + a0, c.members, c.mnode, c.fofs,
            c.fent, D.inv, cnt);
      }
      count_launch("cut patch solve");
      prof_mark(1, l, s);
      const auto& w = H_.levels[l].work_cut[colour];
      prof_work(1, l, w[0], w[1] * sizeof(T) + w[2]);
    }
  }

  // Chebyshev smoothing of A_l x = b (the baseline smoother of Sec. 4):
  // point-Jacobi scaling on [lambda / 20, lambda], lambda = 1.2 lambda_max,
  // three-term recurrence, `cheb_degree` operator applications; the same
  // polynomial before and after the coarse correction
  template <typename T>
  void chebyshev(int l, Typed<T>& D, T* x, const T* b, cudaStream_t s) {
    const Common& c = com_[l];
    const double lmax = 1.2 * lam_[l], lmin = lmax / 20.0;
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
    double rho = 1.0 / sigma;
    for (int k = 0; k < H_.prm.cheb_degree; ++k) {
      apply<T>(l, D, x, b, D.r, s);  // r = b - A x
      double c1 = 0.0, c2 = 1.0 / theta;
      if (k > 0) {
        const double rho_new = 1.0 / (2.0 * sigma - rho);
        c1 = rho_new * rho;
        c2 = 2.0 * rho_new / delta;
        rho = rho_new;
      }
      k_chebyshev<T><<<kVecBlocks, 256, 0, s>>>(c.region, x, D.xp, D.r, D.dinv, (T)c1, (T)c2);
      count_launch("chebyshev step");
    }
  }

  // lambda_max(D^{-1} A_l) by 30 power iterations from the normalised
  // all-ones vector (FP64): v <- w / ||w||, w = D^{-1} A v; the last ||w||
  double power_lambda_max(int l) {
    Typed<double>& D = d64_[l];
    const Common& c = com_[l];
    cudaStream_t s = setup_stream_;
    std::vector<double> ones((size_t)c.nbox, 0.0);
    for (int64_t i = 0; i < c.ndof; ++i) ones[(size_t)H_.levels[l].dofs[i]] = 1.0 / std::sqrt((double)c.ndof);
    CUTMG_CUDA(cudaMemcpyAsync(D.x, ones.data(), sizeof(double) * c.nbox, cudaMemcpyHostToDevice, s));
    CUTMG_CUDA(cudaStreamSynchronize(s));
    for (int it = 0; it < 30; ++it) {
      apply<double>(l, D, D.x, nullptr, D.r, s);
      k_scale_diag<double><<<kVecBlocks, 256, 0, s>>>(c.region, D.dinv, D.r, D.r);
      dot(c.region, D.r, D.r, sc_ + 6, s);
      k_scale_rsqrt<<<kVecBlocks, 256, 0, s>>>(c.region, sc_ + 6, D.r, D.x);
    }
    const double lam = std::sqrt(read_scalar(6, s));
    CUTMG_CUDA(cudaMemsetAsync(D.x, 0, sizeof(double) * c.nbox, s));
    CUTMG_CUDA(cudaMemsetAsync(D.r, 0, sizeof(double) * c.nbox, s));
    CUTMG_CUDA(cudaStreamSynchronize(s));
    return lam;
  }

  // eq. "smoother-split": interior colours, then n_c sweeps of the cut
  // colours; the post-smoother runs the same steps in reverse order
  template <typename T>
  void smooth(int l, Typed<T>& D, bool post, T* x, const T* b, cudaStream_t s) {
    if (H_.prm.smoother == 1) {
      chebyshev<T>(l, D, x, b, s);
      return;
    }
    const int ncol = 1 << DIM, nc = H_.prm.n_c;
    std::vector<std::pair<int, int>> seq;
    for (int c = 0; c < ncol; ++c) seq.push_back({0, c});
    for (int r = 0; r < nc; ++r)
      for (int c = 0; c < ncol; ++c) seq.push_back({1, c});
    if (post)
      for (int i = (int)seq.size() - 1; i >= 0; --i) colour_step<T>(l, D, seq[i].first, seq[i].second, x, b, s);
    else
      for (auto& st : seq) colour_step<T>(l, D, st.first, st.second, x, b, s);
  }

  template <typename T, int MODE>
  void pass(const T* in, T* out, int in0, int in1, int out0, int out1, int axis, const int* lo,
            const int* ext, const int* col, const T* wt, int W, const uint8_t* mask, cudaStream_t s) {
    const int64_t tot = (int64_t)ext[0] * ext[1] * ext[2];
    if (tot <= 0) return;
    const int bs = ext[0] > 64 ? 128 : (ext[0] > 32 ? 64 : 32);
    const dim3 grid((unsigned)((ext[0] + bs - 1) / bs), (unsigned)ext[1], (unsigned)ext[2]);
    k_pass<T, MODE><<<grid, bs, 0, s>>>(in, out, in0, in1, out0, out1, axis, lo[0], lo[1],
                                                          lo[2], ext[0], ext[1], ext[2], col, wt, W, mask);
    count_launch("transfer pass");
  }

  // b_{l-1} = P^T r_l, separably (x, y, z passes) over the active boxes
  template <typename T>
  void restrict_(int l, std::vector<Typed<T>>& DD, const T* rf, T* bc, cudaStream_t s) {
    const Common& F = com_[l];
    const Common& Cc = com_[l - 1];
    Typed<T>& D = DD[l];
    const int nf = F.n, nc = Cc.n, W = 4 * P + 1;
    if (DIM == 3) {
      int lo1[3] = {Cc.bb_lo[0], F.bb_lo[1], F.bb_lo[2]};
      int ex1[3] = {Cc.bb_hi[0] - Cc.bb_lo[0] + 1, F.bb_hi[1] - F.bb_lo[1] + 1, F.bb_hi[2] - F.bb_lo[2] + 1};
      pass<T, 0>(rf, D.t1, nf, nf, nc, nf, 0, lo1, ex1, F.res_col, D.res_w, W, nullptr, s);
      int lo2[3] = {Cc.bb_lo[0], Cc.bb_lo[1], F.bb_lo[2]};
      int ex2[3] = {ex1[0], Cc.bb_hi[1] - Cc.bb_lo[1] + 1, ex1[2]};
      pass<T, 0>(D.t1, D.t2, nc, nf, nc, nc, 1, lo2, ex2, F.res_col, D.res_w, W, nullptr, s);
      int lo3[3] = {Cc.bb_lo[0], Cc.bb_lo[1], Cc.bb_lo[2]};
      int ex3[3] = {ex1[0], ex2[1], Cc.bb_hi[2] - Cc.bb_lo[2] + 1};
      CUTMG_CUDA(cudaMemsetAsync(bc, 0, sizeof(T) * Cc.nbox, s));
      pass<T, 1>(D.t2, bc, nc, nc, nc, nc, 2, lo3, ex3, F.res_col, D.res_w, W, Cc.nact, s);
    } else {
      int lo1[3] = {Cc.bb_lo[0], F.bb_lo[1], 0};
      int ex1[3] = {Cc.bb_hi[0] - Cc.bb_lo[0] + 1, F.bb_hi[1] - F.bb_lo[1] + 1, 1};
      pass<T, 0>(rf, D.t1, nf, nf, nc, nf, 0, lo1, ex1, F.res_col, D.res_w, W, nullptr, s);
      int lo2[3] = {Cc.bb_lo[0], Cc.bb_lo[1], 0};
      int ex2[3] = {ex1[0], Cc.bb_hi[1] - Cc.bb_lo[1] + 1, 1};
      CUTMG_CUDA(cudaMemsetAsync(bc, 0, sizeof(T) * Cc.nbox, s));
      pass<T, 1>(D.t1, bc, nc, nf, nc, nc, 1, lo2, ex2, F.res_col, D.res_w, W, Cc.nact, s);
    }
  }

  // x_l += P x_{l-1}
  template <typename T>
  void prolong(int l, std::vector<Typed<T>>& DD, const T* xc, T* xf, cudaStream_t s) {
    const Common& F = com_[l];
    const Common& Cc = com_[l - 1];
    Typed<T>& D = DD[l];
    const int nf = F.n, nc = Cc.n, W = P + 1;
    if (DIM == 3) {
      int lo1[3] = {F.bb_lo[0], Cc.bb_lo[1], Cc.bb_lo[2]};
      int ex1[3] = {F.bb_hi[0] - F.bb_lo[0] + 1, Cc.bb_hi[1] - Cc.bb_lo[1] + 1, Cc.bb_hi[2] - Cc.bb_lo[2] + 1};
      pass<T, 0>(xc, D.t3, nc, nc, nf, nc, 0, lo1, ex1, F.pro_col, D.pro_w, W, nullptr, s);
      int lo2[3] = {F.bb_lo[0], F.bb_lo[1], Cc.bb_lo[2]};
      int ex2[3] = {ex1[0], F.bb_hi[1] - F.bb_lo[1] + 1, ex1[2]};
      pass<T, 0>(D.t3, D.t4, nf, nc, nf, nf, 1, lo2, ex2, F.pro_col, D.pro_w, W, nullptr, s);
      int lo3[3] = {F.bb_lo[0], F.bb_lo[1], F.bb_lo[2]};
      int ex3[3] = {ex1[0], ex2[1], F.bb_hi[2] - F.bb_lo[2] + 1};
      pass<T, 2>(D.t4, xf, nf, nf, nf, nf, 2, lo3, ex3, F.pro_col, D.pro_w, W, F.nact, s);
    } else {
      int lo1[3] = {F.bb_lo[0], Cc.bb_lo[1], 0};
      int ex1[3] = {F.bb_hi[0] - F.bb_lo[0] + 1, Cc.bb_hi[1] - Cc.bb_lo[1] + 1, 1};
      pass<T, 0>(xc, D.t3, nc, nc, nf, nc, 0, lo1, ex1, F.pro_col, D.pro_w, W, nullptr, s);
      int lo2[3] = {F.bb_lo[0], F.bb_lo[1], 0};
      int ex2[3] = {ex1[0], F.bb_hi[1] - F.bb_lo[1] + 1, 1};
      pass<T, 2>(D.t3, xf, nf, nc, nf, nf, 1, lo2, ex2, F.pro_col, D.pro_w, W, F.nact, s);
    }
  }

  template <typename T>
  void coarse(Typed<T>& D, const T* b, T* x, cudaStream_t s) {
    const Common& c = com_[0];
    const int n0 = (int)c.ndof;
    k_coarse<T><<<blocks_for(n0, 8), 256, 0, s>>>(D.coarse_inv, c.coarse_nodes, n0, b, x);
    count_launch("coarse solve");
  }

  // V-cycle with zero initial guess on level l: x = B_l b (Sec. 2.2)
  template <typename T>
  void vcycle_level(int l, std::vector<Typed<T>>& DD, const T* b, T* x, cudaStream_t s) {
    if (l == 0) {
      coarse<T>(DD[0], b, x, s);
      return;
    }
    Typed<T>& D = DD[l];
    CUTMG_CUDA(cudaMemsetAsync(x, 0, sizeof(T) * com_[l].nbox, s));
    smooth<T>(l, D, false, x, b, s);
    apply<T>(l, D, x, b, D.r, s);
    restrict_<T>(l, DD, D.r, DD[l - 1].b, s);
    vcycle_level<T>(l - 1, DD, DD[l - 1].b, DD[l - 1].x, s);
    prolong<T>(l, DD, DD[l - 1].x, x, s);
    smooth<T>(l, D, true, x, b, s);
  }

  // z = B r on the finest level (box layout, FP64 in and out)
  void precondition(int prec, const double* r, double* z, cudaStream_t s) {
    const int L = n_levels() - 1;
    const auto& F = com_[L];
    if (prec == 1) {
      Typed<float>& D = d32_[L];
      k_convert<float, double><<<kVecBlocks, 256, 0, s>>>(F.region, r, D.b);
      count_launch("convert r");
      vcycle_level<float>(L, d32_, D.b, D.x, s);
      CUTMG_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * F.nbox, s));
      k_convert<double, float><<<kVecBlocks, 256, 0, s>>>(F.region, D.x, z);
      count_launch("convert z");
    } else {
      vcycle_level<double>(L, d64_, r, z, s);
    }
  }
};

template <int DIM, int P>
template <typename T>
std::vector<typename Engine<DIM, P>::template Typed<T>>& Engine<DIM, P>::typed() {
  if constexpr (std::is_same<T, double>::value) return d64_;
  else return d32_;
}

}  // namespace cutmg
