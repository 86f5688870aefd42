// Batched form: many independent problems of one (dimension, degree) solved
// together.  Every step of the hot path is one persistent, grid-stride launch
// over a work list of (instance, item) pairs (items = patches of one colour,
// ghost faces, owner positions, boundary nodes, lattice points, coarse rows),
// so uneven instances fill the GPU together and the launch count per CG
// iteration does not grow with the number of instances.  Each item runs the
// same device body as the single-problem kernels, and every reduction keeps
// the single-problem partition, so a batched solve of an instance performs
// the same floating-point operations as solving it alone.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <memory>
#include <vector>

#include "batch_api.hpp"
#include "engine.cuh"

namespace cutmg {

// ---------------------------------------------------------------------------
// device descriptors

template <int DIM, int P, typename T>
struct LvlDesc {
  OpArgs<T> op;
  FdArgs<T, P> fd;
  int N, n;
  T *x, *b, *r;
  const int* cart;
  const int* cutv;
  const int* cutn;
  const int* cutmo;
  const int64_t* cutio;
  const float* dense_d;  // FP32 interior-patch map of the level
  const uint16_t* members;
  const int* mnode;
  const int* fofs;
  const int* fent;
  const int* faces;
  const int* cfaces;
  const int* bulk;
  const int* bnd;
  const T* inv;
  int cart_start[9], cut_start[9], cf_start[9];
  int nfaces;
  const T* coarse_inv;
  const int* coarse_nodes;
  int n0;
  PipeLevel<T> pl;  // the level for the pipelined cut kernel (closures of more than 64 nodes)
  const int* bf_face;  // per colour: block-boundary ghost faces and their moment slots
  const int* bf_dst;
  int bf_start[9];
  const float* tc_b;  // FP32 interior-patch map as the tensor-core B operand
  SfArgs<T> sf;       // sum-factorised operator: 1D rows, tiles of bulk positions
  const int* sf_tiles;
  const uint32_t* sf_masks;
};

struct PassDesc {  // one separable transfer pass of one instance
  const void* in;
  void* out;
  int in0, in1, out0, out1, axis, W;
  int lo[3], ext[3];
  const int* col;
  const void* wt;
  const uint8_t* mask;
};

struct VecDesc {  // vectors of one instance over its active bounding box
  Region R;
  void* a;
  void* b;
  void* c;
  void* d;
};

__device__ __forceinline__ int find_inst(const int* __restrict__ off, int K, int w) {
  int lo = 0, hi = K;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= w)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// batched kernels

template <int DIM, int P, typename T, int WARPS>
__global__ void __launch_bounds__(32 * WARPS) kb_cart(const LvlDesc<DIM, P, T>* __restrict__ D,
                                                      const int* __restrict__ off, int K, int total,
                                                      int colour) {
  __shared__ CartScratch<DIM, P, T> sCS[WARPS];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int it = blockIdx.x * WARPS + w; it < total; it += gridDim.x * WARPS) {
    const int i = find_inst(off, K, it);
    const LvlDesc<DIM, P, T>& L = D[i];
    const int vert = L.cart[L.cart_start[colour] + it - off[i]];
    cart_body<DIM, P, T>(L.fd, L.N, L.n, L.x, L.b, vert, lane, sCS[w]);
    __syncwarp();
  }
}

// FP32 interior-patch step of the batched form: the dense map of
// k_smooth_dense with each instance's transposed W read from its level
// descriptor (the same products in the same order, so batched and solo
// agree bitwise)
template <int DIM, int P>
__global__ void __launch_bounds__(256) kb_cart_dense(const LvlDesc<DIM, P, float>* __restrict__ D,
                                                     const int* __restrict__ off, int K, int total, int colour) {
  using G = DenseGeo<DIM, P>;
  constexpr int C = G::C, NI = G::NI, NR4 = G::NR4;
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
    const int i = find_inst(off, K, it);
    const LvlDesc<DIM, P, float>& L = D[i];
    const int base = dense_base<DIM, P>(L.cart[L.cart_start[colour] + it - off[i]], L.N, L.n);
    float acc[NI];
#pragma unroll
    for (int r = 0; r < NI; ++r) acc[r] = 0.f;
    for (int row = 0; row < G::ROWS; ++row) {
      bool inner;
      const int ro = dense_row<DIM, P>(row, L.n, inner);
#pragma unroll
      for (int cx = 0; cx < C; ++cx) {
        const float* src = (inner && cx >= 1 && cx <= C - 2) ? L.b : L.x;
        dense_fma<NI, NR4>(L.dense_d + (row * C + cx) * NR4, src[base + ro + cx], acc);
      }
    }
#pragma unroll
    for (int r = 0; r < NI; ++r) L.x[base + dense_interior_offset<DIM, P>(r, L.n)] = acc[r];
  }
}

// FP32 interior-patch step of the batched form on the tensor cores: work
// items are tiles of 128 patches of one instance; the B operand is reloaded
// when the instance changes.  A patch gets the same products as in the solo
// kernel (k_smooth_tc): rows of an MMA do not interact.
template <int DIM, int P>
__global__ void __launch_bounds__(256, 2) kb_smooth_tc(const LvlDesc<DIM, P, float>* __restrict__ D,
                                                       const int* __restrict__ off, int K, int total, int colour,
                                                       int* err) {
  extern __shared__ __align__(128) unsigned char tsm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  TcBlock tb;
  tc_begin<DIM, P>(tb, tsm, &bar, &tmem_slot);
  int loaded = -1;
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const int i = find_inst(off, K, it);
    const LvlDesc<DIM, P, float>& L = D[i];
    if (i != loaded) {  // the previous tile's MMAs have completed (tc_tile waited)
      tc_load_b<DIM, P>(L.tc_b, tb.sB);
      loaded = i;
    }
    const int t0 = (it - off[i]) * 128, a0 = L.cart_start[colour];
    const int cnt = L.cart_start[colour + 1] - a0;
    tc_tile<DIM, P>(tb, L.N, L.n, L.x, L.b, L.cart + a0 + t0, min(128, cnt - t0), err, kTmaSpin);
  }
  tc_end<DIM, P>(tb);
}

// block-boundary ghost-face moments of a colour's cut patches, over the
// (instance, face) work list (the face list of k_face_moments_to)
template <int DIM, int P, typename T>
__global__ void __launch_bounds__(128) kb_face_moments_to(const LvlDesc<DIM, P, T>* __restrict__ D,
                                                          const int* __restrict__ off, int K, int total,
                                                          int colour) {
  constexpr int NT = FaceGeo<DIM, P>::NT, PW = FaceGeo<DIM, P>::PER_WARP;
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * PW < total; w += warps) {
    const int it = w * PW + lane / NT;
    const bool ok = lane / NT < PW && it < total;
    const int i = find_inst(off, K, ok ? it : w * PW);
    const LvlDesc<DIM, P, T>& L = D[i];
    const int e = L.bf_start[colour] + (ok ? it : w * PW) - off[i];
    const int d0 = ok ? L.bf_dst[2 * e] : -1, d1 = ok ? L.bf_dst[2 * e + 1] : -1;
    T* out = const_cast<T*>(L.pl.Gb);
    face_moment_lanes<DIM, P, T>(L.op, L.x, ok ? L.faces[L.bf_face[e]] : -1, lane,
                                 d0 >= 0 ? out + (size_t)d0 * P * NT : nullptr,
                                 d1 >= 0 ? out + (size_t)d1 * P * NT : nullptr);
  }
}

template <int DIM, int P, typename T>
__global__ void __launch_bounds__(128) kb_face_moments(const LvlDesc<DIM, P, T>* __restrict__ D,
                                                       const T* const* __restrict__ X,
                                                       const int* __restrict__ off, int K, int total,
                                                       int colour) {
  constexpr int NT = FaceGeo<DIM, P>::NT, PW = FaceGeo<DIM, P>::PER_WARP;
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  // warp-uniform loop over groups of PW faces; lanes of one warp may serve
  // faces of different instances
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * PW < total; w += warps) {
    const int it = w * PW + lane / NT;
    const bool ok = lane / NT < PW && it < total;
    const int i = find_inst(off, K, ok ? it : w * PW);
    const LvlDesc<DIM, P, T>& L = D[i];
    const int local = (ok ? it : w * PW) - off[i];
    const int f = colour >= 0 ? L.cfaces[L.cf_start[colour] + local] : local;
    face_moment_lanes<DIM, P, T>(L.op, X ? X[i] : L.x, ok ? L.faces[f] : -1, lane,
                                 L.op.G + (size_t)f * P * FaceGeo<DIM, P>::NT, nullptr);
  }
}

template <int DIM, int P, typename T, int WARPS>
__global__ void __launch_bounds__(32 * WARPS) kb_cut_solve(const LvlDesc<DIM, P, T>* __restrict__ D,
                                                           const int* __restrict__ off, int K, int total,
                                                           int colour) {
  __shared__ PatchScratch<DIM, P, T> sS[WARPS];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int it = blockIdx.x * WARPS + w; it < total; it += gridDim.x * WARPS) {
    const int i = find_inst(off, K, it);
    const LvlDesc<DIM, P, T>& L = D[i];
    const int j = L.cut_start[colour] + it - off[i];
    cut_body<DIM, P, T>(L.op, L.x, L.b, L.cutv[j], L.cutn[j], L.cutmo[j], L.cutio[j], L.members, L.mnode,
                        L.fofs, L.fent, L.inv, sS[w], L.op.Kref, lane);
    __syncwarp();
  }
}

// Cut-patch step over the (instance, patch) work list: the warp loop of
// k_cut_warp (same loads, same arithmetic), one warp per item, records
// prefetched into L2.
template <int DIM, int P, typename T, int WPB>
__global__ void __launch_bounds__(32 * WPB, cut_min_blocks<T>())
    kb_cut_warp(const LvlDesc<DIM, P, T>* __restrict__ D, const int* __restrict__ off, int K, int total, int colour) {
  extern __shared__ __align__(128) unsigned char wsm[];
  __shared__ CutTables<DIM, P> tb;
  cut_tables<DIM, P>(tb);
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  warp_loop<DIM, P, T>(
      blockIdx.x * WPB + warp, gridDim.x * WPB, total,
      [&](int it, const PipeLevel<T>*& lv, int& j) {
        const int i = find_inst(off, K, it);
        lv = &D[i].pl;
        j = D[i].cut_start[colour] + it - off[i];
      },
      *reinterpret_cast<WarpStage<DIM, P, T>*>(wsm + (size_t)warp * warp_stage_bytes<DIM, P, T>()), tb,
      kCutPrefetch);
}

// sum-factorised operator over the (instance, tile) work list: the tile body
// of k_apply_sf (the same arithmetic as the instance alone)
template <int DIM, int P, typename T>
__global__ void __launch_bounds__(256) kb_apply_sf(const LvlDesc<DIM, P, T>* __restrict__ D,
                                                   const T* const* __restrict__ X, const T* const* __restrict__ B,
                                                   T* const* __restrict__ Y, const int* __restrict__ off, int K,
                                                   int total) {
  extern __shared__ __align__(16) unsigned char sfm[];
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const int i = find_inst(off, K, it);
    const LvlDesc<DIM, P, T>& L = D[i];
    const int local = it - off[i];
    sf_tile<DIM, P, T>(L.sf, L.N, L.n, X[i], B ? B[i] : nullptr, Y[i], L.sf_tiles[local],
                       L.sf_masks + (size_t)local * SfGeo<DIM, P>::MASKW, reinterpret_cast<T*>(sfm));
  }
}

// apply: items are bulk positions (mode 0) or boundary nodes (mode 1)
template <int DIM, int P, typename T, int MODE>
__global__ void __launch_bounds__(128) kb_apply(const LvlDesc<DIM, P, T>* __restrict__ D,
                                                const T* const* __restrict__ X, const T* const* __restrict__ B,
                                                T* const* __restrict__ Y, const int* __restrict__ off, int K,
                                                int total) {
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
    const int i = find_inst(off, K, it);
    const LvlDesc<DIM, P, T>& L = D[i];
    const int local = it - off[i];
    const T* bb = B ? B[i] : nullptr;
    if (MODE == 0)
      bulk_body<DIM, P, T>(L.op, X[i], bb, Y[i], L.bulk[local], L.op.Kref);
    else
      bnd_body<DIM, P, T>(L.op, X[i], bb, Y[i], L.bnd[local], L.op.Kref);
  }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256) kb_pass(const PassDesc* __restrict__ PD, const int* __restrict__ off,
                                               int K, int total) {
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
    const int i = find_inst(off, K, it);
    const PassDesc& Q = PD[i];
    const int64_t t = it - off[i];
    const int i0 = Q.lo[0] + (int)(t % Q.ext[0]);
    const int i1 = Q.lo[1] + (int)((t / Q.ext[0]) % Q.ext[1]);
    const int i2 = Q.lo[2] + (int)(t / ((int64_t)Q.ext[0] * Q.ext[1]));
    const int io = (Q.axis == 0) ? i0 : (Q.axis == 1 ? i1 : i2);
    const T* in = static_cast<const T*>(Q.in);
    const T* wt = static_cast<const T*>(Q.wt);
    T acc = T(0);
    for (int e = 0; e < Q.W; ++e) {
      const int c = Q.col[io * Q.W + e];
      const int j0 = Q.axis == 0 ? c : i0, j1 = Q.axis == 1 ? c : i1, j2 = Q.axis == 2 ? c : i2;
      acc += wt[io * Q.W + e] * in[(int64_t)j0 + (int64_t)Q.in0 * (j1 + (int64_t)Q.in1 * j2)];
    }
    T* out = static_cast<T*>(Q.out);
    const int64_t o = (int64_t)i0 + (int64_t)Q.out0 * (i1 + (int64_t)Q.out1 * i2);
    if (MODE == 0) out[o] = acc;
    else if (MODE == 1) out[o] = Q.mask[o] ? acc : T(0);
    else if (Q.mask[o]) out[o] += acc;
  }
}

template <int DIM, int P, typename T>
__global__ void __launch_bounds__(256) kb_coarse(const LvlDesc<DIM, P, T>* __restrict__ D,
                                                 const int* __restrict__ off, int K, int total) {
  const int lane = threadIdx.x & 31;
  for (int it = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < total;
       it += gridDim.x * (blockDim.x >> 5)) {
    const int i = find_inst(off, K, it);
    const LvlDesc<DIM, P, T>& L = D[i];
    const int row = it - off[i], n0 = L.n0;
    T acc = T(0);
    for (int j = lane; j < n0; j += 32) acc += L.coarse_inv[(size_t)row * n0 + j] * L.b[L.coarse_nodes[j]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) L.x[L.coarse_nodes[row]] = acc;
  }
}

// a[o] = 0 over each instance's region
template <typename T>
__global__ void __launch_bounds__(256) kb_zero(const VecDesc* __restrict__ V, const int* __restrict__ off,
                                               int K, int total) {
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
    const int i = find_inst(off, K, it);
    static_cast<T*>(V[i].a)[V[i].R.at(it - off[i])] = T(0);
  }
}

// b[o] = (TO) a[o]
template <typename TO, typename TI>
__global__ void __launch_bounds__(256) kb_convert(const VecDesc* __restrict__ V, const int* __restrict__ off,
                                                  int K, int total) {
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
    const int i = find_inst(off, K, it);
    const int64_t o = V[i].R.at(it - off[i]);
    static_cast<TO*>(V[i].b)[o] = (TO) static_cast<const TI*>(V[i].a)[o];
  }
}

// per-instance dot products with the single-problem partition: block
// (i, bk) forms the same partial sum as block bk of k_dot_partial
constexpr int kBatchDotBlocks = 512;
static __global__ void __launch_bounds__(256) kb_dot_partial(const VecDesc* __restrict__ V, const int* __restrict__ list,
                                                      double* __restrict__ part) {
  __shared__ double s[256];
  const int i = list[blockIdx.x / kBatchDotBlocks], bk = blockIdx.x % kBatchDotBlocks;
  const VecDesc& Q = V[i];
  const double* a = static_cast<const double*>(Q.a);
  const double* b = static_cast<const double*>(Q.b);
  double acc = 0.0;
  Q.R.for_each_node_of(bk, kBatchDotBlocks, [&](int64_t o) { acc += a[o] * b[o]; });
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)i * kBatchDotBlocks + bk] = s[0];
}

static __global__ void __launch_bounds__(256) kb_dot_final(const double* __restrict__ part, const int* __restrict__ list,
                                                    double* const* __restrict__ sc, int slot) {
  __shared__ double s[256];
  const int i = list[blockIdx.x];
  double acc = 0.0;
  for (int k = threadIdx.x; k < kBatchDotBlocks; k += 256) acc += part[(size_t)i * kBatchDotBlocks + k];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) sc[i][slot] = s[0];
}

// CG updates of the listed instances: a = x, b = r, c = p, d = q (or z)
static __global__ void __launch_bounds__(256) kb_cg_xr(const VecDesc* __restrict__ V, double* const* __restrict__ sc,
                                                const int* __restrict__ off, int K, int total) {
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
    const int i = find_inst(off, K, it);
    const VecDesc& Q = V[i];
    const double alpha = sc[i][0] / sc[i][1];
    const int64_t o = Q.R.at(it - off[i]);
    static_cast<double*>(Q.a)[o] += alpha * static_cast<const double*>(Q.c)[o];
    static_cast<double*>(Q.b)[o] -= alpha * static_cast<const double*>(Q.d)[o];
  }
}

static __global__ void __launch_bounds__(256) kb_cg_p(const VecDesc* __restrict__ V, double* const* __restrict__ sc,
                                               const int* __restrict__ off, int K, int total) {
  for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
    const int i = find_inst(off, K, it);
    const VecDesc& Q = V[i];
    const double beta = sc[i][2] / sc[i][0];
    const int64_t o = Q.R.at(it - off[i]);
    double* p = static_cast<double*>(Q.c);
    p[o] = static_cast<const double*>(Q.d)[o] + beta * p[o];
  }
}

static __global__ void kb_gather_scalars(double* const* __restrict__ sc, int K, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < K * 16) out[t] = sc[t / 16][t % 16];
}

static __global__ void kb_copy_scalar(double* const* __restrict__ sc, const int* __restrict__ list, int n, int dst,
                                      int src) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) sc[list[t]][dst] = sc[list[t]][src];
}

// ---------------------------------------------------------------------------
// host side

template <int DIM, int P>
class BatchGroup final : public BatchGroupBase {
  using E = Engine<DIM, P>;
  static constexpr int NCOL = 1 << DIM;

 public:
  BatchGroup(std::vector<E*> inst, int n_c) : inst_(std::move(inst)), n_c_(n_c) {
    K_ = (int)inst_.size();
    depth_ = 0;
    for (E* e : inst_) depth_ = std::max(depth_, e->n_levels());
    act_.assign(K_, 1);
    CUTMG_CUDA(cudaGetDevice(&dev_));
    CUTMG_CUDA(cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, dev_));
    build_desc<double>(d64_);
    build_desc<float>(d32_);
    {
      std::vector<double*> sct(K_);
      for (int i = 0; i < K_; ++i) sct[i] = inst_[i]->sc_;
      sc_ = upload(sct);
    }
    part_ = pool_.alloc<double>((size_t)K_ * kBatchDotBlocks);
    scg_ = pool_.alloc<double>((size_t)K_ * 16);
    err_ = pool_.alloc<int>(1);
    CUTMG_CUDA(cudaFuncSetAttribute(kb_smooth_tc<DIM, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    TcGeo<DIM, P>::SMEM));
    CUTMG_CUDA(cudaFuncSetAttribute(kb_apply_sf<DIM, P, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    SfGeo<DIM, P>::ELEMS * (int)sizeof(double)));
    CUTMG_CUDA(cudaFuncSetAttribute(kb_apply_sf<DIM, P, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    SfGeo<DIM, P>::ELEMS * (int)sizeof(float)));
    if (!E::kWarpCut) {
      CUTMG_CUDA(cudaFuncSetAttribute(kb_cut_warp<DIM, P, double, E::kCutWarps>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      E::kCutWarps * warp_stage_bytes<DIM, P, double>()));
      CUTMG_CUDA(cudaFuncSetAttribute(kb_cut_warp<DIM, P, float, E::kCutWarps>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      E::kCutWarps * warp_stage_bytes<DIM, P, float>()));
    }
    CUTMG_CUDA(cudaMallocHost(&host_sc_, sizeof(double) * K_ * 16));
    rebuild_lists();
    // pointer tables of the level residuals, uploaded here: the first use is
    // inside a stream capture, where no allocation or copy may run
    res_tabs<double>(0);
    res_tabs<float>(0);
  }
  ~BatchGroup() override {
    for (auto& g : graphs_) if (g.exec) cudaGraphExecDestroy(g.exec);
    if (cap_) cudaStreamDestroy(cap_);
    if (host_sc_) cudaFreeHost(host_sc_);
  }

  int size() const override { return K_; }
  int active() const override {
    int a = 0;
    for (int v : act_) a += v;
    return a;
  }
  int64_t launches() const override { return launches_; }
  void get_tile(int* w, int* b) const override {
    *w = tile_w_;
    *b = tile_b_;
  }
  void set_tile(int w, int b) override {
    tile_w_ = (w == 2 || w == 8) ? w : 4;
    tile_b_ = b > 0 ? b : 4;
    ++version_;
  }

  void autotune(cudaStream_t s) override {
    // candidates for the two patch kernels: warps per block and blocks per
    // SM of the persistent grid; timed on the finest depth's colour 0
    const int cand_w[3] = {2, 4, 8};
    const int cand_b[3] = {2, 4, 8};
    float best = 1e30f;
    cudaEvent_t e0, e1;
    CUTMG_CUDA(cudaEventCreate(&e0));
    CUTMG_CUDA(cudaEventCreate(&e1));
    for (int wi = 0; wi < 3; ++wi)
      for (int bi = 0; bi < 3; ++bi) {
        tile_w_ = cand_w[wi];
        tile_b_ = cand_b[bi];
        // warm, then time one interior and one cut colour step in FP32
        for (int rep = 0; rep < 2; ++rep) {
          CUTMG_CUDA(cudaEventRecord(e0, s));
          colour_step<float>(d32_, 0, 0, 0, s);
          colour_step<float>(d32_, 0, 1, 0, s);
          CUTMG_CUDA(cudaEventRecord(e1, s));
        }
        CUTMG_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        CUTMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
          best = ms;
          best_w_ = cand_w[wi];
          best_b_ = cand_b[bi];
        }
      }
    tile_w_ = best_w_;
    tile_b_ = best_b_;
    ++version_;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }

  void bnorms(double* host_bn) override {
    for (int i = 0; i < K_; ++i) host_bn[i] = bn_[i];
  }

  void start(int prec, const double* const* b, cudaStream_t s) override {
    act_.assign(K_, 1);
    rebuild_lists();
    bn_.assign(K_, 0.0);
    for (int i = 0; i < K_; ++i) {
      E* e = inst_[i];
      const int L = e->n_levels() - 1;
      e->to_box(L, b[i], e->bF_, s);
      const size_t bytes = sizeof(double) * e->com_[L].nbox;
      CUTMG_CUDA(cudaMemsetAsync(e->xF_, 0, bytes, s));
      CUTMG_CUDA(cudaMemcpyAsync(e->rF_, e->bF_, bytes, cudaMemcpyDeviceToDevice, s));
    }
    dot_all(1, 4, s);  // ||b||^2 -> slot 4   (vec set 1: a = b, b = b)
    read_scalars(s);
    std::vector<int> zero;
    for (int i = 0; i < K_; ++i) {
      bn_[i] = std::sqrt(host_sc_[i * 16 + 4]);
      if (!(bn_[i] > 0.0)) zero.push_back(i);
    }
    its_.assign(K_, 0);
    rel_.assign(K_, 0.0);
    deactivate(zero);
    if (active() == 0) return;
    precondition(prec, s);
    dot_all(2, 0, s);  // rz = (r, z)
    for (int i = 0; i < K_; ++i)
      if (act_[i]) {
        E* e = inst_[i];
        const int L = e->n_levels() - 1;
        CUTMG_CUDA(cudaMemcpyAsync(e->pF_, e->zF_, sizeof(double) * e->com_[L].nbox, cudaMemcpyDeviceToDevice, s));
      }
  }

  void half_a(cudaStream_t s) override {
    run_graph(0, s, [&](cudaStream_t cs) {
      apply_fine(cs);
      dot_all(3, 1, cs);  // pq
      kb_cg_xr<<<grid(tot_vec_, 256), 256, 0, cs>>>(vec_cg_, sc_, off_vec_, K_, tot_vec_);
      count("batched cg update x r");
      dot_all(4, 3, cs);  // rr
    });
  }

  void read_rr(double* host_rr, cudaStream_t s) override {
    read_scalars(s);
    for (int i = 0; i < K_; ++i) host_rr[i] = host_sc_[i * 16 + 3];
    if ((int)its_.size() == K_)
      for (int i = 0; i < K_; ++i)
        if (act_[i]) {
          its_[i] += 1;
          rel_[i] = std::sqrt(host_rr[i]) / bn_[i];
        }
  }

  void deactivate(const std::vector<int>& idx) override {
    bool ch = false;
    for (int i : idx)
      if (act_[i]) {
        act_[i] = 0;
        ch = true;
      }
    if (ch) rebuild_lists();
  }

  void half_b(int prec, cudaStream_t s) override {
    run_graph(1 + prec, s, [&](cudaStream_t cs) {
      precondition(prec, cs);
      dot_all(2, 2, cs);  // rz_new
      kb_cg_p<<<grid(tot_vec_, 256), 256, 0, cs>>>(vec_cgz_, sc_, off_vec_, K_, tot_vec_);
      count("batched cg update p");
      kb_copy_scalar<<<(nact_ + 255) / 256, 256, 0, cs>>>(sc_, act_list_d_, nact_, 0, 2);
      count("batched cg scalar");
    });
  }

  void finish(double* const* x, BatchInfo* info, cudaStream_t s) override {
    // true residuals (all instances)
    std::vector<int> keep = act_;
    act_.assign(K_, 1);
    rebuild_lists();
    apply_true(s);
    dot_all(5, 5, s);
    read_scalars(s);
    for (int i = 0; i < K_; ++i) {
      E* e = inst_[i];
      e->from_box(e->n_levels() - 1, e->xF_, x[i], s);
      info[i].iterations = its_[i];
      info[i].rel = rel_[i];
      info[i].true_rel = bn_[i] > 0 ? std::sqrt(host_sc_[i * 16 + 5]) / bn_[i] : 0.0;
    }
    act_ = keep;
  }

 private:
  std::vector<E*> inst_;
  int K_ = 0, depth_ = 0, n_c_ = 2, dev_ = 0, sms_ = 152;
  DevPool pool_;
  int64_t launches_ = 0;
  // CUDA graphs of the two halves of a CG iteration (slot 0: q = A p .. (r, r);
  // 1 + precision: z = B r .. p), captured for one version of the work lists
  // (rebuild_lists starts a new version) and replayed while it holds
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    int version = -1;
    int64_t launches = 0;
  };
  Graph graphs_[3];
  int version_ = 0;
  cudaStream_t cap_ = nullptr;
  template <class F>
  void run_graph(int slot, cudaStream_t s, F&& body) {
    Graph& g = graphs_[slot];
    if (!g.exec || g.version != version_) {
      if (!cap_) CUTMG_CUDA(cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking));
      if (g.exec) {
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
      }
      const int64_t l0 = launches_;
      cudaGraph_t gr = nullptr;
      CUTMG_CUDA(cudaStreamBeginCapture(cap_, cudaStreamCaptureModeThreadLocal));
      try {
        body(cap_);
      } catch (...) {
        cudaStreamEndCapture(cap_, &gr);
        if (gr) cudaGraphDestroy(gr);
        launches_ = l0;
        throw;
      }
      CUTMG_CUDA(cudaStreamEndCapture(cap_, &gr));
      cudaError_t e = cudaGraphInstantiate(&g.exec, gr, 0);
      cudaGraphDestroy(gr);
      if (e != cudaSuccess) throw CudaError(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
      g.version = version_;
      g.launches = launches_ - l0;
      launches_ = l0;
    }
    CUTMG_CUDA(cudaGraphLaunch(g.exec, s));
    launches_ += g.launches;
  }
  int tile_w_ = 4, tile_b_ = 4, best_w_ = 4, best_b_ = 4;
  std::vector<int> act_, its_;
  std::vector<double> bn_, rel_;
  double** sc_ = nullptr;  // each problem's own CG scalars (Engine::sc_), so CG state survives regrouping
  double* part_ = nullptr;
  double* scg_ = nullptr;
  int* err_ = nullptr;
  double* host_sc_ = nullptr;

  template <typename T>
  struct Depth {  // descriptors of every instance at one depth below the finest
    LvlDesc<DIM, P, T>* desc = nullptr;  // device, K entries
    std::vector<LvlDesc<DIM, P, T>> host;
    std::vector<int> level;              // level of each instance (-1: none)
    PassDesc* rpass[3] = {nullptr, nullptr, nullptr};
    PassDesc* ppass[3] = {nullptr, nullptr, nullptr};
    std::vector<PassDesc> rpass_h[3], ppass_h[3];
    VecDesc* xzero = nullptr;
    std::vector<VecDesc> xzero_h;
  };
  std::vector<Depth<double>> d64_;
  std::vector<Depth<float>> d32_;

  // work lists (prefix offsets over instances), rebuilt when the active set changes
  struct Work {
    int* off = nullptr;  // device, K + 1
    int total = 0;
  };
  std::vector<std::vector<Work>> w_cart_, w_tile_, w_cut_, w_cf_, w_bf_;  // [depth][colour]
  std::vector<Work> w_bulk_, w_sft_, w_bnd_, w_faces_, w_coarse_, w_xzero_;
  std::vector<std::array<Work, 3>> w_rpass_, w_ppass_;
  Work w_vecF_;
  int* off_vec_ = nullptr;
  int tot_vec_ = 0;
  VecDesc *vec_cg_ = nullptr, *vec_cgz_ = nullptr, *vec_dot_[6] = {nullptr};
  VecDesc *vec_conv_r_ = nullptr, *vec_conv_z_ = nullptr, *vec_copy_r_ = nullptr, *vec_copy_z_ = nullptr;
  int* act_list_d_ = nullptr;
  int nact_ = 0;
  // fine-level operator descriptors (FP64) and vector pointer tables
  const double** Xp_ = nullptr;  // p per instance
  double** Yq_ = nullptr;        // q
  const double** Xx_ = nullptr;  // x
  const double** Bb_ = nullptr;  // b
  double** Yt_ = nullptr;        // t (true residual)
  std::vector<void*> scratch_;

  void count(const char* what) {
    launch_check(what);
    ++launches_;
  }
  // host copy of every problem's 16 CG scalars (gathered into one buffer)
  void read_scalars(cudaStream_t s) {
    kb_gather_scalars<<<(K_ * 16 + 255) / 256, 256, 0, s>>>(sc_, K_, scg_);
    count("batched gather scalars");
    CUTMG_CUDA(cudaMemcpyAsync(host_sc_, scg_, sizeof(double) * K_ * 16, cudaMemcpyDeviceToHost, s));
    CUTMG_CUDA(cudaStreamSynchronize(s));
  }
  int grid(int total, int per_block) const {
    int g = (total + per_block - 1) / per_block;
    return std::max(1, std::min(g, sms_ * 8));
  }

  template <typename T>
  std::vector<Depth<T>>& depths();

  template <typename T>
  void build_desc(std::vector<Depth<T>>& DV) {
    DV.resize(depth_);
    for (int t = 0; t < depth_; ++t) {
      Depth<T>& Dt = DV[t];
      Dt.host.resize(K_);
      Dt.level.assign(K_, -1);
      for (int r = 0; r < 3; ++r) {
        Dt.rpass_h[r].assign(K_, PassDesc{});
        Dt.ppass_h[r].assign(K_, PassDesc{});
      }
      Dt.xzero_h.assign(K_, VecDesc{});
      for (int i = 0; i < K_; ++i) {
        E* e = inst_[i];
        const int l = e->n_levels() - 1 - t;
        Dt.level[i] = l;
        LvlDesc<DIM, P, T>& L = Dt.host[i];
        std::memset(&L, 0, sizeof(L));
        if (l < 0) continue;
        auto& C = e->com_[l];
        auto& Ty = e->template typed<T>()[l];
        L.op = Ty.op;
        L.fd = Ty.fd;
        L.N = C.N;
        L.n = C.n;
        L.x = Ty.x;
        L.b = Ty.b;
        L.r = Ty.r;
        L.cart = C.cart;
        L.cutv = C.cutv;
        L.cutn = C.cutn;
        L.cutmo = C.cutmo;
        L.cutio = C.cutio;
        L.dense_d = e->template typed<float>()[l].dense_d;
        L.members = C.members;
        L.mnode = C.mnode;
        L.fofs = C.fofs;
        L.fent = C.fent;
        L.faces = C.faces;
        L.cfaces = C.cfaces;
        L.bulk = C.bulk;
        L.bnd = C.bnd;
        L.inv = Ty.inv;
        if (!E::kWarpCut) {
          L.pl = e->template pipe_level<T>(C, Ty, Ty.x, Ty.b);
          L.bf_face = C.bf_face;
          L.bf_dst = C.bf_dst;
          for (int c = 0; c <= NCOL; ++c) L.bf_start[c] = C.bf_start[c];
        }
        L.tc_b = e->template typed<float>()[l].tc_b;
        L.sf = Ty.sf;
        L.sf_tiles = C.sf_tiles;
        L.sf_masks = C.sf_masks;
        for (int c = 0; c <= NCOL; ++c) {
          L.cart_start[c] = C.cart_start[c];
          L.cut_start[c] = C.cut_start[c];
          L.cf_start[c] = C.cf_start[c];
        }
        L.nfaces = C.nfaces;
        L.coarse_inv = Ty.coarse_inv;
        L.coarse_nodes = C.coarse_nodes;
        L.n0 = (int)C.ndof;
        Dt.xzero_h[i].R = C.region;
        Dt.xzero_h[i].a = Ty.x;
        if (l >= 1) e->template pass_descs<T, PassDesc>(l, Dt.rpass_h, Dt.ppass_h, i);
      }
      Dt.desc = upload(Dt.host);
      for (int r = 0; r < 3; ++r) {
        Dt.rpass[r] = upload(Dt.rpass_h[r]);
        Dt.ppass[r] = upload(Dt.ppass_h[r]);
      }
      Dt.xzero = upload(Dt.xzero_h);
    }
  }

  template <typename V>
  V* upload(const std::vector<V>& h) {
    V* d = pool_.alloc<V>(std::max<size_t>(1, h.size()), false);
    if (!h.empty()) CUTMG_CUDA(cudaMemcpy(d, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice));
    return d;
  }

  Work make_work(const std::vector<int>& counts) {
    Work w;
    std::vector<int> off(K_ + 1, 0);
    for (int i = 0; i < K_; ++i) off[i + 1] = off[i] + (act_[i] ? counts[i] : 0);
    w.total = off[K_];
    w.off = upload(off);
    return w;
  }

  void rebuild_lists() {
    ++version_;  // captured graphs refer to the old lists
    // (device memory of old lists is kept in the pool; rebuilds are rare)
    w_cart_.assign(depth_, std::vector<Work>(NCOL));
    w_tile_.assign(depth_, std::vector<Work>(NCOL));
    w_bf_.assign(depth_, std::vector<Work>(NCOL));
    w_cut_.assign(depth_, std::vector<Work>(NCOL));
    w_cf_.assign(depth_, std::vector<Work>(NCOL));
    w_bulk_.assign(depth_, Work{});
    w_sft_.assign(depth_, Work{});
    w_bnd_.assign(depth_, Work{});
    w_faces_.assign(depth_, Work{});
    w_coarse_.assign(depth_, Work{});
    w_xzero_.assign(depth_, Work{});
    w_rpass_.assign(depth_, std::array<Work, 3>{});
    w_ppass_.assign(depth_, std::array<Work, 3>{});
    for (int t = 0; t < depth_; ++t) {
      const auto& lv = d64_[t].level;
      std::vector<int> cnt(K_, 0);
      auto fill = [&](auto f) {
        for (int i = 0; i < K_; ++i) cnt[i] = f(i);
        return make_work(cnt);
      };
      for (int c = 0; c < NCOL; ++c) {
        w_cart_[t][c] = fill([&](int i) {
          const int l = lv[i];
          if (l < 1) return 0;
          auto& C = inst_[i]->com_[l];
          return C.cart_start[c + 1] - C.cart_start[c];
        });
        w_tile_[t][c] = fill([&](int i) {
          const int l = lv[i];
          if (l < 1) return 0;
          auto& C = inst_[i]->com_[l];
          return (C.cart_start[c + 1] - C.cart_start[c] + 127) / 128;
        });
        w_bf_[t][c] = fill([&](int i) {
          const int l = lv[i];
          if (l < 1 || E::kWarpCut) return 0;
          auto& C = inst_[i]->com_[l];
          return C.bf_start[c + 1] - C.bf_start[c];
        });
        w_cut_[t][c] = fill([&](int i) {
          const int l = lv[i];
          if (l < 1) return 0;
          auto& C = inst_[i]->com_[l];
          return C.cut_start[c + 1] - C.cut_start[c];
        });
        w_cf_[t][c] = fill([&](int i) {
          const int l = lv[i];
          if (l < 1) return 0;
          auto& C = inst_[i]->com_[l];
          return C.cf_start[c + 1] - C.cf_start[c];
        });
      }
      w_bulk_[t] = fill([&](int i) { return lv[i] >= 1 || t == 0 ? (lv[i] >= 0 ? inst_[i]->com_[lv[i]].nbulk : 0) : 0; });
      w_sft_[t] = fill([&](int i) {
        return lv[i] >= 1 || t == 0 ? (lv[i] >= 0 && inst_[i]->com_[lv[i]].nbulk > 0 ? inst_[i]->com_[lv[i]].nsf : 0) : 0;
      });
      w_bnd_[t] = fill([&](int i) { return lv[i] >= 1 || t == 0 ? (lv[i] >= 0 ? inst_[i]->com_[lv[i]].nbnd : 0) : 0; });
      w_faces_[t] = fill([&](int i) { return lv[i] >= 1 || t == 0 ? (lv[i] >= 0 ? inst_[i]->com_[lv[i]].nfaces : 0) : 0; });
      w_coarse_[t] = fill([&](int i) { return lv[i] == 0 ? (int)inst_[i]->com_[0].ndof : 0; });
      w_xzero_[t] = fill([&](int i) { return lv[i] >= 1 ? (int)inst_[i]->com_[lv[i]].region.size() : 0; });
      for (int r = 0; r < 3; ++r) {
        w_rpass_[t][r] = fill([&](int i) {
          if (lv[i] < 1) return 0;
          const auto& q = d64_[t].rpass_h[r][i];
          return q.ext[0] * q.ext[1] * q.ext[2];
        });
        w_ppass_[t][r] = fill([&](int i) {
          if (lv[i] < 1) return 0;
          const auto& q = d64_[t].ppass_h[r][i];
          return q.ext[0] * q.ext[1] * q.ext[2];
        });
      }
    }
    // finest-level vector descriptors
    std::vector<int> vc(K_, 0);
    std::vector<VecDesc> cg(K_), cgz(K_), dots[6], conv_r(K_), conv_z(K_), copy_r(K_), copy_z(K_);
    for (int k = 0; k < 6; ++k) dots[k].assign(K_, VecDesc{});
    std::vector<const double*> xp(K_), xx(K_), bb(K_);
    std::vector<double*> yq(K_), yt(K_);
    std::vector<int> alist;
    for (int i = 0; i < K_; ++i) {
      E* e = inst_[i];
      const int L = e->n_levels() - 1;
      const Region R = e->com_[L].region;
      vc[i] = (int)R.size();
      cg[i] = VecDesc{R, e->xF_, e->rF_, e->pF_, e->qF_};
      cgz[i] = VecDesc{R, nullptr, nullptr, e->pF_, e->zF_};
      dots[1][i] = VecDesc{R, e->bF_, e->bF_, nullptr, nullptr};
      dots[2][i] = VecDesc{R, e->rF_, e->zF_, nullptr, nullptr};
      dots[3][i] = VecDesc{R, e->pF_, e->qF_, nullptr, nullptr};
      dots[4][i] = VecDesc{R, e->rF_, e->rF_, nullptr, nullptr};
      dots[5][i] = VecDesc{R, e->tF_, e->tF_, nullptr, nullptr};
      conv_r[i] = VecDesc{R, e->rF_, e->d32_[L].b, nullptr, nullptr};
      conv_z[i] = VecDesc{R, e->d32_[L].x, e->zF_, nullptr, nullptr};
      copy_r[i] = VecDesc{R, e->rF_, e->d64_[L].b, nullptr, nullptr};
      copy_z[i] = VecDesc{R, e->d64_[L].x, e->zF_, nullptr, nullptr};
      xp[i] = e->pF_;
      yq[i] = e->qF_;
      xx[i] = e->xF_;
      bb[i] = e->bF_;
      yt[i] = e->tF_;
      if (act_[i]) alist.push_back(i);
    }
    w_vecF_ = make_work(vc);
    off_vec_ = w_vecF_.off;
    tot_vec_ = w_vecF_.total;
    vec_cg_ = upload(cg);
    vec_cgz_ = upload(cgz);
    for (int k = 1; k < 6; ++k) vec_dot_[k] = upload(dots[k]);
    vec_conv_r_ = upload(conv_r);
    vec_conv_z_ = upload(conv_z);
    vec_copy_r_ = upload(copy_r);
    vec_copy_z_ = upload(copy_z);
    Xp_ = upload(xp);
    Yq_ = upload(yq);
    Xx_ = upload(xx);
    Bb_ = upload(bb);
    Yt_ = upload(yt);
    nact_ = (int)alist.size();
    act_list_d_ = upload(alist);
  }

  // per-instance dot products of vector set `set` into scalar slot `slot`
  void dot_all(int set, int slot, cudaStream_t s) {
    if (nact_ == 0) return;
    kb_dot_partial<<<nact_ * kBatchDotBlocks, 256, 0, s>>>(vec_dot_[set], act_list_d_, part_);
    count("batched dot partial");
    kb_dot_final<<<nact_, 256, 0, s>>>(part_, act_list_d_, sc_, slot);
    count("batched dot final");
  }

  template <typename T>
  void colour_step(std::vector<Depth<T>>& DV, int t, int cut, int colour, cudaStream_t s) {
    const auto* D = DV[t].desc;
    if (!cut) {
      const Work& w = w_cart_[t][colour];
      if (w.total == 0) return;
      if constexpr (std::is_same<T, float>::value) {
        // the tensor-core form, as the solo engine's automatic choice
        const Work& wt = w_tile_[t][colour];
        kb_smooth_tc<DIM, P><<<std::max(1, std::min(wt.total, 2 * sms_)), 256, TcGeo<DIM, P>::SMEM, s>>>(
            D, wt.off, K_, wt.total, colour, err_);
        count("batched interior patches");
        return;
      }
      launch_cart<T>(D, w, colour, s);
    } else {
      const Work& w = w_cut_[t][colour];
      if (w.total == 0) return;
      const Work& wf = w_cf_[t][colour];
      if (E::kWarpCut && wf.total > 0) {
        kb_face_moments<DIM, P, T><<<grid(wf.total, 4 * FaceGeo<DIM, P>::PER_WARP), 128, 0, s>>>(D, nullptr, wf.off, K_,
                                                                                             wf.total, colour);
        count("batched face moments");
      }
      if (E::kWarpCut) {
        launch_cut<T>(D, w, colour, s);
      } else {
        const Work& wb = w_bf_[t][colour];
        if (wb.total > 0) {
          kb_face_moments_to<DIM, P, T><<<grid(wb.total, 4 * FaceGeo<DIM, P>::PER_WARP), 128, 0, s>>>(
              D, wb.off, K_, wb.total, colour);
          count("batched boundary face moments");
        }
        constexpr int WPB = E::kCutWarps;
        const int smem = WPB * warp_stage_bytes<DIM, P, T>();
        int nb = 0;
        CUTMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kb_cut_warp<DIM, P, T, WPB>, 32 * WPB, smem));
        const int gridc = std::max(1, std::min((w.total + WPB - 1) / WPB, std::max(1, nb) * sms_));
        kb_cut_warp<DIM, P, T, WPB><<<gridc, 32 * WPB, smem, s>>>(D, w.off, K_, w.total, colour);
        count("batched cut patches");
      }
    }
  }

  template <typename T>
  void launch_cart(const LvlDesc<DIM, P, T>* D, const Work& w, int colour, cudaStream_t s) {
    const int gridw = std::max(1, std::min((w.total + tile_w_ - 1) / tile_w_, sms_ * tile_b_));
    if constexpr (std::is_same<T, float>::value) {
      const int bs = 32 * tile_w_;
      const int gridd = std::max(1, std::min((w.total + bs - 1) / bs, sms_ * tile_b_));
      kb_cart_dense<DIM, P><<<gridd, bs, 0, s>>>(D, w.off, K_, w.total, colour);
    } else if (tile_w_ == 2) {
      kb_cart<DIM, P, T, 2><<<gridw, 64, 0, s>>>(D, w.off, K_, w.total, colour);
    } else if (tile_w_ == 8) {
      kb_cart<DIM, P, T, 8><<<gridw, 256, 0, s>>>(D, w.off, K_, w.total, colour);
    } else {
      kb_cart<DIM, P, T, 4><<<gridw, 128, 0, s>>>(D, w.off, K_, w.total, colour);
    }
    count("batched interior patches");
  }
  template <typename T>
  void launch_cut(const LvlDesc<DIM, P, T>* D, const Work& w, int colour, cudaStream_t s) {
    const int gridw = std::max(1, std::min((w.total + tile_w_ - 1) / tile_w_, sms_ * tile_b_));
    if (tile_w_ == 2) kb_cut_solve<DIM, P, T, 2><<<gridw, 64, 0, s>>>(D, w.off, K_, w.total, colour);
    else if (tile_w_ == 8) kb_cut_solve<DIM, P, T, 8><<<gridw, 256, 0, s>>>(D, w.off, K_, w.total, colour);
    else kb_cut_solve<DIM, P, T, 4><<<gridw, 128, 0, s>>>(D, w.off, K_, w.total, colour);
    count("batched cut patches");
  }

  template <typename T>
  void smooth(std::vector<Depth<T>>& DV, int t, bool post, cudaStream_t s) {
    std::vector<std::pair<int, int>> seq;
    for (int c = 0; c < NCOL; ++c) seq.push_back({0, c});
    for (int r = 0; r < n_c_; ++r)
      for (int c = 0; c < NCOL; ++c) seq.push_back({1, c});
    if (post)
      for (int i = (int)seq.size() - 1; i >= 0; --i) colour_step<T>(DV, t, seq[i].first, seq[i].second, s);
    else
      for (auto& st : seq) colour_step<T>(DV, t, st.first, st.second, s);
  }

  // level residual r = b - A x of the smoothing instances at depth t
  template <typename T>
  void residual(std::vector<Depth<T>>& DV, int t, cudaStream_t s) {
    auto* D = DV[t].desc;
    const Work& wf = w_faces_[t];
    if (wf.total > 0) {
      kb_face_moments<DIM, P, T><<<grid(wf.total, 4 * FaceGeo<DIM, P>::PER_WARP), 128, 0, s>>>(D, nullptr, wf.off, K_,
                                                                                             wf.total, -1);
      count("batched face moments");
    }
    // X = x, B = b, Y = r from the descriptors: pointer tables built here once
    auto& tabs = res_tabs<T>(t);
    if (w_bulk_[t].total > 0) {
      if (inst_[0]->template use_sumfact<T>())
        kb_apply_sf<DIM, P, T><<<std::max(1, std::min(w_sft_[t].total, 3 * sms_)), 256,
                                 SfGeo<DIM, P>::ELEMS * sizeof(T), s>>>(D, tabs.X, tabs.B, tabs.Y, w_sft_[t].off, K_,
                                                                       w_sft_[t].total);
      else
        kb_apply<DIM, P, T, 0><<<grid(w_bulk_[t].total, 128), 128, 0, s>>>(D, tabs.X, tabs.B, tabs.Y,
                                                                           w_bulk_[t].off, K_, w_bulk_[t].total);
      count("batched apply bulk");
    }
    if (w_bnd_[t].total > 0) {
      kb_apply<DIM, P, T, 1><<<grid(w_bnd_[t].total, 128), 128, 0, s>>>(D, tabs.X, tabs.B, tabs.Y,
                                                                        w_bnd_[t].off, K_, w_bnd_[t].total);
      count("batched apply boundary");
    }
  }

  template <typename T>
  struct Tabs {
    const T** X = nullptr;
    const T** B = nullptr;
    T** Y = nullptr;
  };
  std::vector<Tabs<double>> tabs64_;
  std::vector<Tabs<float>> tabs32_;
  template <typename T>
  Tabs<T>& res_tabs(int t) {
    auto& TT = tabs_vec<T>();
    if ((int)TT.size() != depth_) {
      TT.resize(depth_);
      auto& DV = depth_vec<T>();
      for (int d = 0; d < depth_; ++d) {
        std::vector<const T*> X(K_), B(K_);
        std::vector<T*> Y(K_);
        for (int i = 0; i < K_; ++i) {
          X[i] = DV[d].host[i].x;
          B[i] = DV[d].host[i].b;
          Y[i] = DV[d].host[i].r;
        }
        TT[d].X = upload(X);
        TT[d].B = upload(B);
        TT[d].Y = upload(Y);
      }
    }
    return TT[t];
  }
  template <typename T>
  std::vector<Tabs<T>>& tabs_vec();
  template <typename T>
  std::vector<Depth<T>>& depth_vec();

  template <typename T>
  void transfer(std::vector<Depth<T>>& DV, int t, bool restrict_, cudaStream_t s) {
    auto& Dt = DV[t];
    for (int r = 0; r < (DIM == 3 ? 3 : 2); ++r) {
      const Work& w = restrict_ ? w_rpass_[t][r] : w_ppass_[t][r];
      if (w.total == 0) continue;
      const PassDesc* PD = restrict_ ? Dt.rpass[r] : Dt.ppass[r];
      const bool last = r == (DIM == 3 ? 2 : 1);
      if (!last)
        kb_pass<T, 0><<<grid(w.total, 256), 256, 0, s>>>(PD, w.off, K_, w.total);
      else if (restrict_)
        kb_pass<T, 1><<<grid(w.total, 256), 256, 0, s>>>(PD, w.off, K_, w.total);
      else
        kb_pass<T, 2><<<grid(w.total, 256), 256, 0, s>>>(PD, w.off, K_, w.total);
      count("batched transfer pass");
    }
  }

  template <typename T>
  void vcycle_depth(std::vector<Depth<T>>& DV, int t, cudaStream_t s) {
    if (t >= depth_) return;
    if (w_coarse_[t].total > 0) {
      kb_coarse<DIM, P, T><<<grid(w_coarse_[t].total, 8), 256, 0, s>>>(DV[t].desc, w_coarse_[t].off, K_,
                                                                       w_coarse_[t].total);
      count("batched coarse solve");
    }
    if (w_xzero_[t].total == 0) return;  // nobody smooths at this depth
    kb_zero<T><<<grid(w_xzero_[t].total, 256), 256, 0, s>>>(DV[t].xzero, w_xzero_[t].off, K_, w_xzero_[t].total);
    count("batched zero");
    smooth<T>(DV, t, false, s);
    residual<T>(DV, t, s);
    transfer<T>(DV, t, true, s);
    vcycle_depth<T>(DV, t + 1, s);
    transfer<T>(DV, t, false, s);
    smooth<T>(DV, t, true, s);
  }

  void precondition(int prec, cudaStream_t s) {
    if (prec == 1) {
      // r (FP64) -> b of the finest FP32 level; x (FP32) -> z (FP64)
      kb_convert<float, double><<<grid(tot_vec_, 256), 256, 0, s>>>(vec_conv_r_, off_vec_, K_, tot_vec_);
      count("batched convert r");
      vcycle_depth<float>(d32_, 0, s);
      kb_convert<double, float><<<grid(tot_vec_, 256), 256, 0, s>>>(vec_conv_z_, off_vec_, K_, tot_vec_);
      count("batched convert z");
    } else {
      // the FP64 V-cycle works in the finest level's own buffers: b <- r, z <- x
      copy_fine_b_from_r(s);
      vcycle_depth<double>(d64_, 0, s);
      copy_fine_z_from_x(s);
    }
  }

  void copy_fine_b_from_r(cudaStream_t s) {
    kb_convert<double, double><<<grid(tot_vec_, 256), 256, 0, s>>>(vec_copy_r_, off_vec_, K_, tot_vec_);
    count("batched copy r");
  }
  void copy_fine_z_from_x(cudaStream_t s) {
    kb_convert<double, double><<<grid(tot_vec_, 256), 256, 0, s>>>(vec_copy_z_, off_vec_, K_, tot_vec_);
    count("batched copy z");
  }

  // q = A p on the finest level of every active instance (FP64)
  void apply_fine(cudaStream_t s) { apply_fp64(Xp_, nullptr, Yq_, s); }
  void apply_true(cudaStream_t s) { apply_fp64(Xx_, Bb_, Yt_, s); }
  void apply_fp64(const double** X, const double** B, double** Y, cudaStream_t s) {
    auto* D = d64_[0].desc;
    const Work& wf = w_faces_[0];
    if (wf.total > 0) {
      kb_face_moments<DIM, P, double><<<grid(wf.total, 4 * FaceGeo<DIM, P>::PER_WARP), 128, 0, s>>>(D, X, wf.off, K_,
                                                                                                  wf.total, -1);
      count("batched face moments");
    }
    if (w_bulk_[0].total > 0) {
      if (inst_[0]->template use_sumfact<double>())
        kb_apply_sf<DIM, P, double><<<std::max(1, std::min(w_sft_[0].total, 3 * sms_)), 256,
                                      SfGeo<DIM, P>::ELEMS * sizeof(double), s>>>(D, X, B, Y, w_sft_[0].off, K_,
                                                                                  w_sft_[0].total);
      else
        kb_apply<DIM, P, double, 0><<<grid(w_bulk_[0].total, 128), 128, 0, s>>>(D, X, B, Y, w_bulk_[0].off, K_,
                                                                                w_bulk_[0].total);
      count("batched apply bulk");
    }
    if (w_bnd_[0].total > 0) {
      kb_apply<DIM, P, double, 1><<<grid(w_bnd_[0].total, 128), 128, 0, s>>>(D, X, B, Y, w_bnd_[0].off, K_,
                                                                             w_bnd_[0].total);
      count("batched apply boundary");
    }
  }
};

template <int DIM, int P>
template <typename T>
std::vector<typename BatchGroup<DIM, P>::template Tabs<T>>& BatchGroup<DIM, P>::tabs_vec() {
  if constexpr (std::is_same<T, double>::value) return tabs64_;
  else return tabs32_;
}
template <int DIM, int P>
template <typename T>
std::vector<typename BatchGroup<DIM, P>::template Depth<T>>& BatchGroup<DIM, P>::depth_vec() {
  if constexpr (std::is_same<T, double>::value) return d64_;
  else return d32_;
}

}  // namespace cutmg
