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
//     run brought into shared memory by one TMA bulk copy (cp.async.bulk,
//     completion on an mbarrier),
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
};

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
  uint64_t gmask;
  const T* recp;  // the record: the stage's slot or global memory
  int vert, m, nit, tma;
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
  int vert, m, mo, io, nit, gb;
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
  return t;
}

// whether patch M's record goes through a shared-memory slot of slot_bytes
template <typename T>
__device__ __forceinline__ bool pipe_tma(const PipeMeta& M, int slot_bytes) {
  const int64_t len = M.r1 - M.r0;
  return len > 0 && (size_t)len * sizeof(T) <= (size_t)slot_bytes;
}

// Issue every load of patch j into stage `st` (cp.async, one group per call;
// the record by TMA on `bar` when it fits `slot_bytes`).  All threads call it.
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
  const bool tma = pipe_tma<T>(M, slot_bytes);
  if (tid == 0) {
    st.vert = M.vert;
    st.m = M.m;
    st.nit = M.nit;
    st.tma = tma;
    st.gmask = M.gmask;
    st.recp = tma ? slot : L.rec + M.r0;
    if (tma) tma_load_1d(slot, L.rec + M.r0, (uint32_t)((M.r1 - M.r0) * sizeof(T)), bar);
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

// One patch from a filled stage: ghost-face moments, residual rows, local
// solve, x updated in place.  Kref: the level's uncut element matrix.
template <int DIM, int P, typename T, int NT>
__device__ __forceinline__ void pipe_compute(const PipeLevel<T>& L, const PipeStage<DIM, P, T>& st,
                                             PipeShared<DIM, P, T>& sh, const T* __restrict__ Kref) {
  using G = PipeGeo<DIM, P>;
  constexpr int C = G::C, NB = G::NB, NTF = G::NT;
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
  // residual of the own rows: cell parts in cell order, then the ghost faces
  for (int e = tid; e < m; e += NT) {
    int o[3] = {0, 0, 0}, u = st.mem[e];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      o[k] = u % C;
      u /= C;
    }
    T acc = T(0);
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
    T fac = T(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      // planes of the faces of the node's cell layers along k
      const int ok = o[k], lay = ok / P, onp = ok - lay * P == 0;
      const int Llo = onp ? lay - 1 : lay, Lhi = lay + 1;
      for (int Lp = Llo < 0 ? 0 : Llo; Lp <= (Lhi > 2 ? 2 : Lhi); ++Lp) {
        const int i = ok - P * (Lp - 1);
        // tangential cells of the block plane containing the node
        int ulo[2] = {0, 0}, uhi[2] = {0, 0}, tj[2] = {0, 0}, q = 0;
#pragma unroll
        for (int kk = 0; kk < DIM; ++kk) {
          if (kk == k) continue;
          const int oj = o[kk], cj = oj / P, on = oj - cj * P == 0;
          ulo[q] = on ? cj - 1 : cj;
          uhi[q] = cj;
          if (ulo[q] < 0) ulo[q] = 0;
          if (uhi[q] > 1) uhi[q] = 1;
          tj[q] = oj;
          ++q;
        }
        for (int u1 = (DIM == 3 ? ulo[1] : 0); u1 <= (DIM == 3 ? uhi[1] : 0); ++u1)
          for (int u0 = ulo[0]; u0 <= uhi[0]; ++u0) {
            const int uu = u0 + 2 * u1;
            const int bit = (k * 3 + Lp) * G::HALF + uu;
            if (!((gm >> bit) & 1ull)) continue;
            const uint64_t below = (1ull << bit) - 1ull;
            const int t = (tj[0] - P * u0) + (DIM == 3 ? (P + 1) * (tj[1] - P * u1) : 0);
            const T* g = Lp == 1 ? &sh.Gm[__popcll(gint & below)][0][0]
                                 : &st.halo[__popcll(gbnd & below) * P * NTF];
#pragma unroll
            for (int mm = 0; mm < P; ++mm) fac += L.op.dvec[mm][i] * g[mm * NTF + t];
          }
      }
    }
    sh.r[e] = st.b[st.mem[e]] - (acc + fac);
  }
  __syncthreads();
  // delta = A_j^{-1} r from the packed lower triangle; the new value from
  // the staged closure value (no other patch of the colour writes this DoF)
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
  for (int e = tid; e < m; e += NT) {
    const T* Re = Ai + e * (e + 1) / 2;
    T a0 = T(0), a1 = T(0);
    int c = 0;
    for (; c + 1 <= e; c += 2) {
      a0 += Re[c] * sh.r[c];
      a1 += Re[c + 1] * sh.r[c + 1];
    }
    if (c <= e) {
      a0 += Re[c] * sh.r[c];
      ++c;
    }
    for (; c < m; ++c) a1 += Ai[c * (c + 1) / 2 + e] * sh.r[c];
    int u = st.mem[e], lc[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      lc[k] = P * (v[k] - 1) + u % C;
      u /= C;
    }
    L.x[lat_index<DIM>(lc, n)] = st.x[st.mem[e]] + (a0 + a1);
  }
  __syncthreads();
}

// waits for stage `st`'s loads (the newer group of cp.asyncs may stay in
// flight) and, if its record came by TMA, for the mbarrier; false when the
// bounded wait ran out (the copy is then drained within kTmaSpin polls)
// (ph bit s: the parity of stage s's next mbarrier phase, flipped here)
template <bool NEWER_PENDING>
__device__ __forceinline__ bool pipe_wait(bool tma, uint64_t* bar, uint32_t& ph, int s, int spin, int* err) {
  if (NEWER_PENDING)
    asm volatile("cp.async.wait_group 1;" ::: "memory");
  else
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  bool ok = true;
  if (tma) {
    const uint32_t parity = (ph >> s) & 1u;
    ok = mbar_wait(bar, parity, spin);
    if (!ok) {
      atomicExch(err, 1);
      mbar_wait(bar, parity, kTmaSpin);
    }
    ph ^= 1u << s;
  }
  __syncthreads();
  return ok;
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
  if ((int)blockIdx.x >= npatch) return;
  for (int i = threadIdx.x; i < G::NB * G::NB; i += NT) sK[i] = L.op.Kref[i];
  if (threadIdx.x == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
  }
  __syncthreads();
  uint32_t ph = 0;
  int j = blockIdx.x, s = 0;
  PipeMeta cur = pipe_meta(L, j0 + j);
  pipe_prefetch<DIM, P, T, NT>(L, cur, j0 + j, stage[0], reinterpret_cast<T*>(psm), slot_bytes, &bar[0]);
  for (; j < npatch; j += gridDim.x, s ^= 1) {
    const int jn = j + (int)gridDim.x;
    const bool more = jn < npatch;
    if (more) {
      const PipeMeta nxt = pipe_meta(L, j0 + jn);
      pipe_prefetch<DIM, P, T, NT>(L, nxt, j0 + jn, stage[s ^ 1], reinterpret_cast<T*>(psm + (s ^ 1) * slot_bytes),
                                   slot_bytes, &bar[s ^ 1]);
    }
    const bool tma = pipe_tma<T>(cur, slot_bytes);
    bool ok;
    if (more)
      ok = pipe_wait<true>(tma, &bar[s], ph, s, spin, err);
    else
      ok = pipe_wait<false>(tma, &bar[s], ph, s, spin, err);
    if (__syncthreads_and(ok)) pipe_compute<DIM, P, T, NT>(L, stage[s], sh, sK);
    if (more) cur = pipe_meta(L, j0 + jn);
  }
}

}  // namespace cutmg
