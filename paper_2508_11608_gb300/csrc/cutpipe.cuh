// Cut-patch colour step (Sec. 3: dense local solver on cut patches) for
// patch closures of more than 64 nodes (3D Q2), as one persistent kernel per
// colour step with a two-stage pipeline per block: while a block computes
// one patch, the data of its next patch are already in flight to the other
// stage.
//
// Per patch j the block needs
//   * the closure of x and b (cp.async, one element per thread),
//   * the DoF list, the row items and the cell kinds (cp.async),
//   * its record: the explicit inverse packed by rows of its lower triangle
//     and the rows of the cut-cell matrices its items use, one contiguous
//     run, and its ghost-entry list; both by TMA bulk copies (cp.async.bulk)
//     completing on one mbarrier,
//   * the moments of the ghost faces on the boundary planes of its block
//     (cp.async from its moment slots).
// Every ghost face in the row of a patch DoF is a face of an active cell that
// contains the DoF, hence of a patch cell, so it lies on one of the 3 planes
// per direction of the 2 x .. x 2 block (eq. "cutfem-ghost").  The faces on
// the middle plane are formed inside the block from the staged closure
// (G_m = coef_m (Mhat x Mhat) J_m, J_m[t] = sum_i dvec_m[i] x(i, t) over the
// 2p + 1 nodes across the face): all their nodes belong to active patch
// cells, so no other patch of the colour writes them.  The faces on the two
// boundary planes reach into the neighbouring block, whose cut patch of the
// same colour may update those nodes in the same launch; their moments are
// therefore computed before the colour step by a separate launch
// (k_face_moments_to), like every moment of the additive-within-a-colour
// step (Sec. 2.3): the patch sees the x from before the colour step only.
//
// The ghost-entry list of a patch (built at setup) holds, for each DoF row,
// the (face, node along the normal, tangential node) triples of the ghost
// faces whose stencil contains the DoF; the rows and the local solve split
// each DoF over 4 lanes, combined by shuffles in a fixed order.
#pragma once

#include "kernels.cuh"

namespace cutmg {

template <int DIM, int P>
struct PipeGeo {
  static constexpr int C = 2 * P + 1;
  static constexpr int NB = Shape<DIM, P>::NB;
  static constexpr int NCL = PatchGeo<DIM, P>::NCL;
  static constexpr int NCELL = 1 << DIM;
  static constexpr int NT = FaceGeo<DIM, P>::NT;  // nodes of a face, (p+1)^(d-1)
  static constexpr int HALF = 1 << (DIM - 1);     // cells per block plane
  static constexpr int NFACE = DIM * 3 * HALF;    // faces on the block's planes
  static constexpr int NIF = DIM * HALF;          // faces on its middle planes
  static constexpr int NBF = DIM * 2 * HALF;      // faces on its boundary planes
  static constexpr int HALO = NBF * P * NT;       // the moments of those
  static constexpr int ITEMW = (NCELL * NB + 3) / 4;  // 32-bit words of the item list
  static constexpr int GCAP = 1024;               // ghost-entry list entries staged (longer: global)
  static constexpr int LANES = 4;                 // threads per DoF row in rows and solve
};

// ghost entry: bit of the face in the block mask (6 bits), node along the
// normal (3 bits), tangential node (7 bits)
__host__ __device__ constexpr uint16_t ghost_entry(int bit, int i, int t) {
  return (uint16_t)(bit | (i << 6) | (t << 9));
}

// device arrays of one level for the pipelined cut kernel
template <typename T>
struct PipeLevel {
  OpArgs<T> op;             // N, n, dvec, coef, Mhat (Kref: the uncut element matrix)
  T* x;
  const T* b;
  const int* vert;          // packed patch vertex
  const int* cnt;           // DoFs m
  const int* moff;          // first DoF in members
  const int* members;       // closure-local index of each DoF (32-bit)
  const int* ioff;          // first 32-bit word of the patch's row items (4-byte aligned lists)
  const int* nit;           // row items of the patch
  const uint32_t* items;    // s * NB + i per item, four per word
  const int* pk;            // [patch][2^d] cell kind / first pack row and item
  const uint64_t* gmask;    // ghost faces of the block planes
  const int64_t* roff;      // record offsets (entries); roff[j + 1] - roff[j] = length
  const T* rec;             // records
  const int* gboff;         // first boundary-face moment slot of each patch
  const T* Gb;              // boundary-face moment slots, P (p+1)^(d-1) values each
  const int* geoff;         // ghost-entry lists: [geoff[j], geoff[j + 1]) in gent (16-byte aligned)
  const uint16_t* gent;     // per patch: m + 1 row offsets, then the entries
};

// bits of the block-boundary planes (0 and 2) in a ghost-face mask
template <int DIM, int P>
__host__ __device__ constexpr uint64_t pipe_bnd_bits() {
  constexpr int HALF = 1 << (DIM - 1);
  uint64_t m = 0;
  for (int k = 0; k < DIM; ++k)
    for (int u = 0; u < HALF; ++u) m |= (1ull << ((k * 3 + 0) * HALF + u)) | (1ull << ((k * 3 + 2) * HALF + u));
  return m;
}

template <int DIM, int P, typename T>
struct PipeStage {
  using G = PipeGeo<DIM, P>;
  T x[G::NCL];
  T b[G::NCL];
  T halo[G::HALO];
  int mem[G::NCL];
  uint32_t item[G::ITEMW];
  int pk[G::NCELL];
  __align__(16) uint16_t gl[G::GCAP];
  uint64_t gmask;
  const T* recp;         // the record: the stage's slot or global memory
  const uint16_t* glp;   // the ghost-entry list: gl or global memory
  int vert, m, nit;
};

template <int DIM, int P, typename T>
struct PipeShared {
  using G = PipeGeo<DIM, P>;
  T part[G::NCELL][G::NB];
  T r[G::NCL];
  T J[G::NIF][P][G::NT];
  T Gm[G::NIF][P][G::NT];
  int flist[G::NIF];
};

struct PipeMeta {
  int vert, m, mo, io, nit, gb, g0, g1;
  int64_t r0, r1;
  uint64_t gmask;
};

template <typename T>
__device__ __forceinline__ PipeMeta pipe_meta(const PipeLevel<T>& L, int j) {
  PipeMeta t;
  t.vert = L.vert[j];
  t.m = L.cnt[j];
  t.mo = L.moff[j];
  t.io = L.ioff[j];
  t.nit = L.nit[j];
  t.r0 = L.roff[j];
  t.r1 = L.roff[j + 1];
  t.gmask = L.gmask[j];
  t.gb = L.gboff[j];
  t.g0 = L.geoff[j];
  t.g1 = L.geoff[j + 1];
  return t;
}

// whether patch M's record goes through a shared-memory slot of slot_bytes,
// and whether its ghost-entry list goes into the stage
template <typename T>
__device__ __forceinline__ bool pipe_tma(const PipeMeta& M, int slot_bytes) {
  const int64_t len = M.r1 - M.r0;
  return len > 0 && (size_t)len * sizeof(T) <= (size_t)slot_bytes;
}
template <int DIM, int P>
__device__ __forceinline__ bool pipe_gl_tma(const PipeMeta& M) {
  return M.g1 - M.g0 <= PipeGeo<DIM, P>::GCAP;
}

// one expected-bytes arrival on the mbarrier (always made, also for zero
// bytes, so that every stage's phase completes once per prefetch), then the
// bulk copies that complete it
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Issue every load of patch j into stage `st` (cp.async, one group per call;
// the record when it fits `slot_bytes` and the ghost-entry list when it
// fits the stage, by TMA on `bar`).  All threads call it.
template <int DIM, int P, typename T, int NT>
__device__ __forceinline__ void pipe_prefetch(const PipeLevel<T>& L, const PipeMeta& M, int j,
                                              PipeStage<DIM, P, T>& st, T* slot, int slot_bytes, uint64_t* bar) {
  using G = PipeGeo<DIM, P>;
  constexpr int C = G::C;
  const int tid = threadIdx.x, n = L.op.n, np = L.op.N + 1;
  int v[3] = {0, 0, 0};
  {
    int q = M.vert;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      v[k] = q % np;
      q /= np;
    }
  }
  const bool tma = pipe_tma<T>(M, slot_bytes), gtma = pipe_gl_tma<DIM, P>(M);
  if (tid == 0) {
    st.vert = M.vert;
    st.m = M.m;
    st.nit = M.nit;
    st.gmask = M.gmask;
    st.recp = tma ? slot : L.rec + M.r0;
    st.glp = gtma ? st.gl : L.gent + M.g0;
    const uint32_t rb = tma ? (uint32_t)((M.r1 - M.r0) * sizeof(T)) : 0u;
    const uint32_t gb = gtma ? (uint32_t)((M.g1 - M.g0) * sizeof(uint16_t)) : 0u;
    mbar_expect(bar, rb + gb);
    if (rb) bulk_copy(slot, L.rec + M.r0, rb, bar);
    if (gb) bulk_copy(st.gl, L.gent + M.g0, gb, bar);
  }
  for (int e = tid; e < G::NCL; e += NT) {
    int u = e, c[3] = {0, 0, 0};
    bool in = true;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      c[k] = P * (v[k] - 1) + u % C;
      u /= C;
      if (c[k] < 0 || c[k] >= n) in = false;
    }
    if (in) {
      const int o = lat_index<DIM>(c, n);
      cp_async_elem(&st.x[e], L.x + o);
      cp_async_elem(&st.b[e], L.b + o);
    } else {
      st.x[e] = T(0);
      st.b[e] = T(0);
    }
    if (e < M.m) cp_async_elem(&st.mem[e], L.members + M.mo + e);
  }
  for (int w = tid; w < (M.nit + 3) / 4; w += NT) cp_async_elem(&st.item[w], L.items + M.io + w);
  if (tid < G::NCELL) cp_async_elem(&st.pk[tid], L.pk + (size_t)j * G::NCELL + tid);
  // moments of the block-boundary ghost faces (one slot per set bit)
  const int nbv = __popcll(M.gmask & pipe_bnd_bits<DIM, P>()) * P * G::NT;
  for (int w = tid; w < nbv; w += NT) cp_async_elem(&st.halo[w], L.Gb + (size_t)M.gb * P * G::NT + w);
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// x at closure coordinate ck along k and tangential cell u, node t, for a
// face of the middle plane
template <int DIM, int P, typename T>
__device__ __forceinline__ T pipe_x(const PipeStage<DIM, P, T>& st, int k, int u, int ck, int t) {
  constexpr int C = 2 * P + 1;
  int o = 0, st_ = 1, q = 0, tt = t;
#pragma unroll
  for (int kk = 0; kk < DIM; ++kk) {
    int c;
    if (kk == k) {
      c = ck;
    } else {
      c = P * ((u >> q) & 1) + tt % (P + 1);
      tt /= P + 1;
      ++q;
    }
    o += c * st_;
    st_ *= C;
  }
  return st.x[o];
}

// sum over the 4 lanes of a DoF row (lanes 4k .. 4k+3 of a warp), the same
// order on every lane
template <typename T>
__device__ __forceinline__ T lane4_sum(T v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  return v;
}

// One patch from a filled stage: ghost-face moments, residual rows, local
// solve, x updated in place.  Kref: the level's uncut element matrix.
template <int DIM, int P, typename T, int NT>
__device__ __forceinline__ void pipe_compute(const PipeLevel<T>& L, const PipeStage<DIM, P, T>& st,
                                             PipeShared<DIM, P, T>& sh, const T* __restrict__ Kref) {
  using G = PipeGeo<DIM, P>;
  constexpr int C = G::C, NB = G::NB, NTF = G::NT, LN = G::LANES, ROWS = NT / LN;
  const int tid = threadIdx.x, m = st.m, n = L.op.n, np = L.op.N + 1;
  constexpr uint64_t bnd = pipe_bnd_bits<DIM, P>();
  const uint64_t gm = st.gmask, gint = gm & ~bnd, gbnd = gm & bnd;
  const int nf = __popcll(gint);
  if (tid < G::NFACE && ((gint >> tid) & 1ull)) sh.flist[__popcll(gint & ((1ull << tid) - 1ull))] = tid;
  __syncthreads();
  // J_m[t] of the ghost faces of the middle planes, and the cell rows of the items
  for (int w = tid; w < nf * P * NTF; w += NT) {
    const int fi = w / (P * NTF), rem = w - fi * (P * NTF), mm = rem / NTF, t = rem - mm * NTF;
    const int f = sh.flist[fi], u = f % G::HALF, k = f / G::HALF / 3;
    T acc = T(0);
#pragma unroll
    for (int i = 0; i <= 2 * P; ++i) acc += L.op.dvec[mm][i] * pipe_x<DIM, P, T>(st, k, u, i, t);
    sh.J[fi][mm][t] = acc;
  }
  const T* rows = st.recp + ((m * (m + 1) / 2 + 3) / 4 * 4);
  const uint8_t* item = reinterpret_cast<const uint8_t*>(st.item);
  for (int q = tid; q < st.nit; q += NT) {
    const int it = item[q], sc = it / NB, jj = it - sc * NB;
    const int pkv = st.pk[sc];
    const T* row = pkv == -1 ? Kref + jj * NB : rows + (size_t)((pkv >> 8) + q - (pkv & 255)) * NB;
    int base = 0, ost = 1;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      base += P * ((sc >> k) & 1) * ost;
      ost *= C;
    }
    T acc = T(0);
    if (DIM == 2) {
#pragma unroll
      for (int q1 = 0; q1 <= P; ++q1)
#pragma unroll
        for (int q0 = 0; q0 <= P; ++q0) acc += row[q0 + (P + 1) * q1] * st.x[base + q0 + C * q1];
    } else {
#pragma unroll
      for (int q2 = 0; q2 <= P; ++q2)
#pragma unroll
        for (int q1 = 0; q1 <= P; ++q1)
#pragma unroll
          for (int q0 = 0; q0 <= P; ++q0)
            acc += row[q0 + (P + 1) * (q1 + (P + 1) * q2)] * st.x[base + q0 + C * (q1 + C * q2)];
    }
    sh.part[sc][jj] = acc;
  }
  __syncthreads();
  // G_m[t] = coef_m sum_t' (Mhat x Mhat)[t][t'] J_m[t']
  for (int w = tid; w < nf * P * NTF; w += NT) {
    const int fi = w / (P * NTF), rem = w - fi * (P * NTF), mm = rem / NTF, t = rem - mm * NTF;
    const int t0 = t % (P + 1), t1 = t / (P + 1);
    T acc = T(0);
#pragma unroll
    for (int s = 0; s < NTF; ++s) {
      const T wgt = (DIM == 2) ? L.op.Mhat[t0][s] : L.op.Mhat[t0][s % (P + 1)] * L.op.Mhat[t1][s / (P + 1)];
      acc += wgt * sh.J[fi][mm][s];
    }
    sh.Gm[fi][mm][t] = L.op.coef[mm] * acc;
  }
  __syncthreads();
  // residual of the own rows, LN lanes per DoF: lane 0 the cell parts in
  // cell order, every lane a strided share of the row's ghost entries
  const uint16_t* gl = st.glp;
  const int lane = tid % LN;
  for (int e0 = 0; e0 < m; e0 += ROWS) {
    const int e = e0 + tid / LN;
    T acc = T(0);
    if (e < m) {
      if (lane == 0) {
        int o[3] = {0, 0, 0}, u = st.mem[e];
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
          o[k] = u % C;
          u /= C;
        }
#pragma unroll
        for (int sc = 0; sc < G::NCELL; ++sc) {
          int jj = 0, jst = 1;
          bool in = st.pk[sc] != -2;
#pragma unroll
          for (int k = 0; k < DIM; ++k) {
            const int a = o[k] - P * ((sc >> k) & 1);
            if (a < 0 || a > P) in = false;
            jj += a * jst;
            jst *= (P + 1);
          }
          if (in) acc += sh.part[sc][jj];
        }
      }
      for (int q = gl[e] + lane; q < gl[e + 1]; q += LN) {
        const int en = gl[m + 1 + q], bit = en & 63, i = (en >> 6) & 7, t = en >> 9;
        const uint64_t below = (1ull << bit) - 1ull;
        const T* g = ((bnd >> bit) & 1ull) ? &st.halo[__popcll(gbnd & below) * P * NTF]
                                            : &sh.Gm[__popcll(gint & below)][0][0];
#pragma unroll
        for (int mm = 0; mm < P; ++mm) acc += L.op.dvec[mm][i] * g[mm * NTF + t];
      }
    }
    acc = lane4_sum(acc);
    if (e < m && lane == 0) sh.r[e] = st.b[st.mem[e]] - acc;
  }
  __syncthreads();
  // delta = A_j^{-1} r from the packed lower triangle, LN lanes per row; the
  // new value from the staged closure value (no other patch of the colour
  // writes this DoF)
  const T* Ai = st.recp;
  int v[3] = {0, 0, 0};
  {
    int q = st.vert;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      v[k] = q % np;
      q /= np;
    }
  }
  for (int e0 = 0; e0 < m; e0 += ROWS) {
    const int e = e0 + tid / LN;
    T acc = T(0);
    if (e < m) {
      const T* Re = Ai + e * (e + 1) / 2;
      int c = lane;
      for (; c <= e; c += LN) acc += Re[c] * sh.r[c];
      for (; c < m; c += LN) acc += Ai[c * (c + 1) / 2 + e] * sh.r[c];
    }
    acc = lane4_sum(acc);
    if (e < m && lane == 0) {
      int u = st.mem[e], lc[3] = {0, 0, 0};
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        lc[k] = P * (v[k] - 1) + u % C;
        u /= C;
      }
      L.x[lat_index<DIM>(lc, n)] = st.x[st.mem[e]] + acc;
    }
  }
  __syncthreads();
}

// waits for stage s's loads (the newer group of cp.asyncs may stay in flight)
// and for its mbarrier (ph bit s: the parity of stage s's next phase, flipped
// here); false when the bounded wait ran out (the copies are then drained
// within kTmaSpin polls)
template <bool NEWER_PENDING>
__device__ __forceinline__ bool pipe_wait(uint64_t* bar, uint32_t& ph, int s, int spin, int* err) {
  if (NEWER_PENDING)
    asm volatile("cp.async.wait_group 1;" ::: "memory");
  else
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  const uint32_t parity = (ph >> s) & 1u;
  bool ok = mbar_wait(bar, parity, spin);
  if (!ok) {
    atomicExch(err, 1);
    mbar_wait(bar, parity, kTmaSpin);
  }
  ph ^= 1u << s;
  __syncthreads();
  return ok;
}

// The pipelined loop of one block over the work items it, it + step, ..
// below total.  locate(item, level, patch) gives an item's level descriptor
// and patch; kref(level) its uncut element matrix.  Metadata run two items
// ahead, data one item ahead.
template <int DIM, int P, typename T, int NT, class Locate, class Kref>
__device__ __forceinline__ void pipe_loop(int it, int step, int total, Locate&& locate, Kref&& kref,
                                          unsigned char* psm, int slot_bytes, PipeStage<DIM, P, T>* stage,
                                          PipeShared<DIM, P, T>& sh, uint64_t* bar, int spin, int* err) {
  if (threadIdx.x == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
  }
  __syncthreads();
  uint32_t ph = 0;
  int s = 0;
  const PipeLevel<T>* Lc;
  int jc;
  locate(it, Lc, jc);
  PipeMeta cur = pipe_meta(*Lc, jc);
  const PipeLevel<T>* Ln = Lc;
  int jn = jc;
  PipeMeta nxt = cur;
  if (it + step < total) {
    locate(it + step, Ln, jn);
    nxt = pipe_meta(*Ln, jn);
  }
  pipe_prefetch<DIM, P, T, NT>(*Lc, cur, jc, stage[0], reinterpret_cast<T*>(psm), slot_bytes, &bar[0]);
  for (; it < total; it += step, s ^= 1) {
    const bool more = it + step < total;
    // metadata of the item after next
    const PipeLevel<T>* L2 = Ln;
    int j2 = jn;
    PipeMeta nn = nxt;
    if (it + 2 * step < total) {
      locate(it + 2 * step, L2, j2);
      nn = pipe_meta(*L2, j2);
    }
    if (more)
      pipe_prefetch<DIM, P, T, NT>(*Ln, nxt, jn, stage[s ^ 1], reinterpret_cast<T*>(psm + (s ^ 1) * slot_bytes),
                                   slot_bytes, &bar[s ^ 1]);
    bool ok;
    if (more)
      ok = pipe_wait<true>(&bar[s], ph, s, spin, err);
    else
      ok = pipe_wait<false>(&bar[s], ph, s, spin, err);
    if (__syncthreads_and(ok)) pipe_compute<DIM, P, T, NT>(*Lc, stage[s], sh, kref(Lc));
    Lc = Ln;
    jc = jn;
    cur = nxt;
    Ln = L2;
    jn = j2;
    nxt = nn;
  }
}

// One colour step: patches j0 .. j0 + npatch - 1, block b takes b, b + grid,
// ..; records of up to slot_bytes go through shared memory.
template <int DIM, int P, typename T>
__global__ void __launch_bounds__(128) k_cut_pipe(PipeLevel<T> L, int j0, int npatch, int slot_bytes, int* err,
                                                  int spin) {
  using G = PipeGeo<DIM, P>;
  constexpr int NT = 128;
  extern __shared__ __align__(16) unsigned char psm[];
  __shared__ __align__(16) PipeStage<DIM, P, T> stage[2];
  __shared__ PipeShared<DIM, P, T> sh;
  __shared__ __align__(16) T sK[G::NB * G::NB];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ PipeLevel<T> sL;
  if ((int)blockIdx.x >= npatch) return;
  for (int i = threadIdx.x; i < G::NB * G::NB; i += NT) sK[i] = L.op.Kref[i];
  if (threadIdx.x == 0) sL = L;  // the level's arrays and tables, read by every thread
  const PipeLevel<T>* Lp = &sL;
  pipe_loop<DIM, P, T, NT>(
      blockIdx.x, gridDim.x, npatch,
      [&](int it, const PipeLevel<T>*& lv, int& j) {
        lv = Lp;
        j = j0 + it;
      },
      [&](const PipeLevel<T>*) -> const T* { return sK; }, psm, slot_bytes, stage, sh, bar, spin, err);
}

}  // namespace cutmg

namespace cutmg {

// Cut-patch inverses on the device, FP64 (the local solver's setup, Sec. 3):
// for patch j, rec[roff[j] ..] holds the lower triangle of A_j by rows on
// entry and that of A_j^{-1} on exit.  One block per patch (block-stride),
// the matrix in shared memory with row stride ld >= m (dynamic, ld (ld + 1)
// doubles): Cholesky A = L L^T (right-looking, L in the lower triangle),
// W = L^{-1} by forward substitution, one column per thread (W's strictly
// lower part stored transposed in the strictly upper triangle, its diagonal
// apart), then A^{-1} = W^T W, entry (i, c) summed over k = i .. m-1 in
// increasing order.  A pivot that is not positive records *err = 2 (the
// patch matrix is not SPD) and the patch is skipped.
__device__ __forceinline__ int tri_row(int e) {
  int i = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
  while (i * (i + 1) / 2 > e) --i;
  while ((i + 1) * (i + 2) / 2 <= e) ++i;
  return i;
}

static __global__ void __launch_bounds__(128) k_patch_inverse(double* __restrict__ rec, const int64_t* __restrict__ roff,
                                                       const int* __restrict__ cnt, int npatch, int ld,
                                                       int* __restrict__ err) {
  extern __shared__ __align__(16) double S[];
  double* Wd = S + (size_t)ld * ld;
  __shared__ int bad;
  const int tid = threadIdx.x, NT = blockDim.x;
  for (int j = blockIdx.x; j < npatch; j += gridDim.x) {
    const int m = cnt[j];
    double* a = rec + roff[j];
    const int ne = m * (m + 1) / 2;
    if (tid == 0) bad = 0;
    for (int e = tid; e < ne; e += NT) {
      const int i = tri_row(e), c = e - i * (i + 1) / 2;
      S[i * ld + c] = a[e];
    }
    __syncthreads();
    for (int k = 0; k < m; ++k) {
      if (tid == 0) {
        const double d = S[k * ld + k];
        if (!(d > 0.0)) bad = 1;
        S[k * ld + k] = d > 0.0 ? sqrt(d) : 1.0;
      }
      __syncthreads();
      const double piv = S[k * ld + k];
      for (int i = k + 1 + tid; i < m; i += NT) S[i * ld + k] /= piv;
      __syncthreads();
      for (int i = k + 1 + tid; i < m; i += NT) {
        const double lik = S[i * ld + k];
        for (int c = k + 1; c <= i; ++c) S[i * ld + c] -= lik * S[c * ld + k];
      }
      __syncthreads();
    }
    for (int c = tid; c < m; c += NT) {
      const double wcc = 1.0 / S[c * ld + c];
      Wd[c] = wcc;
      for (int i = c + 1; i < m; ++i) {
        double s = S[i * ld + c] * wcc;
        for (int k = c + 1; k < i; ++k) s += S[i * ld + k] * S[c * ld + k];
        S[c * ld + i] = -s / S[i * ld + i];
      }
    }
    __syncthreads();
    if (bad) {
      if (tid == 0) atomicExch(err, 2);
    } else {
      for (int e = tid; e < ne; e += NT) {
        const int i = tri_row(e), c = e - i * (i + 1) / 2;
        double s = (i == c ? Wd[i] : S[c * ld + i]) * Wd[i];
        for (int k = i + 1; k < m; ++k) s += S[i * ld + k] * S[c * ld + k];
        a[e] = s;
      }
    }
    __syncthreads();
  }
}

// FP64 -> FP32 copy of a whole array (the mixed form's records)
static __global__ void __launch_bounds__(256) k_to_float(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

}  // namespace cutmg
