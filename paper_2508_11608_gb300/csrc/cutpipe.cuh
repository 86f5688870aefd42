// Cut-patch colour step (Sec. 3: dense local solver on cut patches) for
// patch closures of more than 64 nodes (3D Q2): one warp per patch, several
// independent warps per block, each with its own stage in shared memory, so
// that no barrier of one patch holds back another and the loads of one
// warp's patch overlap the arithmetic of the others.
//
// Per patch j the warp stages (cp.async, one group)
//   * the closure of x and b, one element per lane,
//   * the DoF list, the row items, the cell kinds and its ghost-entry list,
//   * the moments of the ghost faces on the boundary planes of its block
//     (from its moment slots),
// and reads its record from global memory: the explicit inverse (m x m)
// and the rows of the cut-cell matrices its items use, stored by columns,
// so that the lanes of a warp always read consecutive addresses.  The
// record is prefetched into L2 by one bulk prefetch when the patch's loads
// are issued.
// Every ghost face in the row of a patch DoF is a face of an active cell that
// contains the DoF, hence of a patch cell, so it lies on one of the 3 planes
// per direction of the 2 x .. x 2 block (eq. "cutfem-ghost").  The faces on
// the middle plane are formed by the warp from the staged closure
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
// faces whose stencil contains the DoF.
#pragma once

#include "kernels.cuh"

namespace cutmg {

template <int DIM, int P>
struct PipeGeo {
  static constexpr int C = 2 * P + 1;
  static constexpr int NB = Shape<DIM, P>::NB;
  static constexpr int NBP = (NB + 3) / 4 * 4;  // padded row of a cell vector (16-byte rows)
  static constexpr int NCL = PatchGeo<DIM, P>::NCL;
  static constexpr int NCELL = 1 << DIM;
  static constexpr int NT = FaceGeo<DIM, P>::NT;  // nodes of a face, (p+1)^(d-1)
  static constexpr int HALF = 1 << (DIM - 1);     // cells per block plane
  static constexpr int NFACE = DIM * 3 * HALF;    // faces on the block's planes
  static constexpr int NIF = DIM * HALF;          // faces on its middle planes
  static constexpr int NBF = DIM * 2 * HALF;      // faces on its boundary planes
  static constexpr int HALO = NBF * P * NT;       // the moments of those
  static constexpr int ITEMW = (NCELL * NB + 3) / 4;  // 32-bit words of the item list
  static constexpr int GCAP = 512;                // ghost-entry list entries staged (longer: global)
};

// ghost entry: moment slot of the face in the patch (6 bits: the boundary-
// plane faces first, then the middle-plane faces, each in mask-bit order),
// node along the normal (4 bits, 0 .. 2p), tangential node (6 bits); the
// host setup writes the same packing
__host__ __device__ constexpr uint16_t ghost_entry(int slot, int i, int t) {
  return (uint16_t)(slot | (i << 6) | (t << 10));
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
  const T* kp;              // [NB][NBP] uncut element matrix for h = 1, rows padded to NBP
  T ksc;                    // h^(d-2): the level's uncut element matrix is ksc kp
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

// One warp's stage: the patch's closure and lists, and the scratch of its
// residual.  The record stays in global memory (read with coalesced loads).
template <int DIM, int P, typename T>
struct WarpStage {
  using G = PipeGeo<DIM, P>;
  T x[G::NCL];
  T b[G::NCL];
  __align__(16) T xc[G::NCELL][G::NBP];  // x on the nodes of each patch cell (cell order)
  // face moments G_m[t]: the block-boundary faces first (the staged slots),
  // then the middle-plane faces (formed here), each in mask-bit order
  __align__(16) T U[G::NFACE][P][G::NT];
  T part[G::NCELL][G::NB];               // cell row products of the items
  __align__(16) T r[(G::NCL + 3) / 4 * 4];  // residual of the patch rows (zero-padded to 4)
  T dv[P][2 * P + 1];                    // dvec of the level being worked on
  int mem[G::NCL];
  uint32_t item[G::ITEMW];
  int pk[G::NCELL];
  int flist[G::NIF];
  __align__(16) uint16_t gl[G::GCAP];
};

// bytes of one warp's stage, a multiple of 128
template <int DIM, int P, typename T>
__host__ __device__ constexpr int warp_stage_bytes() {
  return (int)((sizeof(WarpStage<DIM, P, T>) + 127) / 128 * 128);
}

// Per-lane constants of the record kernel, per level (reloaded when a warp
// moves to another level): the face-mass rows of the lane's tangential node,
// the penalty coefficients, the scale of the uncut element matrix and the
// lattice sizes.
template <int DIM, int P, typename T>
struct WarpLane {
  T mh0[P + 1], mh1[P + 1];
  T cf[P];
  T ksc;           // h^(d-2), the scale of the uncut element matrix
  int n, np;       // lattice nodes and vertices per direction
  float rnp;       // 1 / np, for the vertex decode
  bool fdiv;       // whether every packed vertex is below 2^24 (exact in FP32)
  const void* lv;  // the level descriptor the constants came from
};

// Level-independent tables of a block, in shared memory: per closure node o
// the cell-local index of o in each patch cell (byte sc; 0xff: not in that
// cell) and its closure coordinates (4 bits per direction); per entry of
// the cell vectors the closure index | (cell-vector index << 16).
template <int DIM, int P>
struct CutTables {
  using G = PipeGeo<DIM, P>;
  uint64_t cpt[G::NCL];
  int uc[G::NCL];
  int xcm[G::NCELL * G::NB];
};

// The closure's first lattice node c0 = p (v - 1) of the patch at packed
// vertex q = v_0 + np (v_1 + np v_2), its lattice index, and whether the
// closure lies inside the lattice.  The divisions by np go through a float
// reciprocal when q < 2^24 (q exact in FP32, the quotient off by at most
// one and corrected from the remainder).
struct PatchPos {
  int c0[3];
  int base;
  bool inside;
};
__device__ __forceinline__ int div_np(int q, int np, float rnp, bool fast) {
  if (!fast) return q / np;
  int t = (int)((float)q * rnp);
  const int r = q - t * np;
  if (r < 0) --t;
  else if (r >= np) ++t;
  return t;
}
template <int DIM, int P, typename T>
__device__ __forceinline__ PatchPos patch_pos(int vert, const WarpLane<DIM, P, T>& wl) {
  PatchPos pp;
  pp.base = 0;
  pp.inside = true;
  pp.c0[0] = pp.c0[1] = pp.c0[2] = 0;
  int q = vert, stn = 1;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const int qn = k + 1 < DIM ? div_np(q, wl.np, wl.rnp, wl.fdiv) : 0;
    const int v = k + 1 < DIM ? q - qn * wl.np : q;
    q = qn;
    pp.c0[k] = P * (v - 1);
    pp.base += pp.c0[k] * stn;
    stn *= wl.n;
    if (pp.c0[k] < 0 || pp.c0[k] + 2 * P >= wl.n) pp.inside = false;
  }
  return pp;
}

// A patch is worked on by a team of GW warps: one warp (GW = 1, several
// teams per block) or the whole block (GW = warps of the block).
template <int GW>
__device__ __forceinline__ void team_sync() {
  if constexpr (GW == 1) __syncwarp();
  else __syncthreads();
}

// the per-level constants of level op (all threads of the team; tid: index
// in the team; ends with a team barrier)
template <int DIM, int P, typename T, int GW = 1>
__device__ __forceinline__ void warp_lane_level(WarpLane<DIM, P, T>& wl, WarpStage<DIM, P, T>& st,
                                                const OpArgs<T>& op, T ksc, const void* lv, int lane, int tid) {
  using G = PipeGeo<DIM, P>;
#pragma unroll
  for (int mm = 0; mm < P; ++mm) wl.cf[mm] = op.coef[mm];
  const int t = lane % G::NT, t0 = t % (P + 1), t1 = t / (P + 1) % (P + 1);
#pragma unroll
  for (int s = 0; s <= P; ++s) {
    wl.mh0[s] = op.Mhat[t0][s];
    wl.mh1[s] = op.Mhat[t1][s];
  }
  for (int e = tid; e < P * (2 * P + 1); e += 32 * GW) st.dv[e / (2 * P + 1)][e % (2 * P + 1)] = op.dvec[e / (2 * P + 1)][e % (2 * P + 1)];
  wl.ksc = ksc;
  wl.n = op.n;
  wl.np = op.N + 1;
  wl.rnp = 1.0f / (float)wl.np;
  {
    int64_t nv = 1;
    for (int k = 0; k < DIM; ++k) nv *= wl.np;
    wl.fdiv = nv <= (int64_t(1) << 24);
  }
  wl.lv = lv;
  team_sync<GW>();
}

// the block's tables (all threads; the caller synchronises)
template <int DIM, int P>
__device__ __forceinline__ void cut_tables(CutTables<DIM, P>& tb) {
  using G = PipeGeo<DIM, P>;
  constexpr int C = G::C;
  for (int o = threadIdx.x; o < G::NCL; o += blockDim.x) {
    int oc[3] = {0, 0, 0}, u = o, code = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      oc[k] = u % C;
      u /= C;
      code |= oc[k] << (4 * k);
    }
    uint64_t tab = ~0ull;
#pragma unroll
    for (int sc = 0; sc < G::NCELL; ++sc) {
      int jj = 0, jst = 1;
      bool in = true;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const int a = oc[k] - P * ((sc >> k) & 1);
        if (a < 0 || a > P) in = false;
        jj += a * jst;
        jst *= P + 1;
      }
      if (in) tab = (tab & ~(0xffull << (8 * sc))) | ((uint64_t)jj << (8 * sc));
    }
    tb.cpt[o] = tab;
    tb.uc[o] = code;
  }
  for (int idx = threadIdx.x; idx < G::NCELL * G::NB; idx += blockDim.x) {
    const int sc = idx / G::NB, q = idx - sc * G::NB;
    int o = 0, st = 1, qq = q;
#pragma unroll
    for (int kk = 0; kk < DIM; ++kk) {
      o += (P * ((sc >> kk) & 1) + qq % (P + 1)) * st;
      qq /= P + 1;
      st *= C;
    }
    tb.xcm[idx] = o | ((sc * G::NBP + q) << 16);
  }
}

struct PipeMeta {
  int vert, m, mo, io, nit, gb, g0, g1;
  int64_t r0, r1;
  uint64_t gmask;
};

// The metadata of a patch spread over the lanes of a warp: lane f < 11
// loads field f (PipeMeta's fields in declaration order, r0 = roff[j],
// r1 = roff[j + 1], g1 = geoff[j + 1]); pipe_meta_gather rebuilds PipeMeta
// in every lane by shuffles.  A warp that reads the next patch's metadata
// while it works on the current one holds one 64-bit register per lane.
constexpr int kMetaFields = 11;
template <typename T>
__device__ __forceinline__ uint64_t pipe_meta_field(const PipeLevel<T>& L, int j, int f) {
  switch (f) {
    case 0: return (uint32_t)L.vert[j];
    case 1: return (uint32_t)L.cnt[j];
    case 2: return (uint32_t)L.moff[j];
    case 3: return (uint32_t)L.ioff[j];
    case 4: return (uint32_t)L.nit[j];
    case 5: return (uint32_t)L.gboff[j];
    case 6: return (uint32_t)L.geoff[j];
    case 7: return (uint32_t)L.geoff[j + 1];
    case 8: return (uint64_t)L.roff[j];
    case 9: return (uint64_t)L.roff[j + 1];
    case 10: return L.gmask[j];
    default: return 0;
  }
}
__device__ __forceinline__ PipeMeta pipe_meta_gather(uint64_t v) {
  PipeMeta t;
  const unsigned full = 0xffffffffu;
  const uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
  t.vert = (int)__shfl_sync(full, lo, 0);
  t.m = (int)__shfl_sync(full, lo, 1);
  t.mo = (int)__shfl_sync(full, lo, 2);
  t.io = (int)__shfl_sync(full, lo, 3);
  t.nit = (int)__shfl_sync(full, lo, 4);
  t.gb = (int)__shfl_sync(full, lo, 5);
  t.g0 = (int)__shfl_sync(full, lo, 6);
  t.g1 = (int)__shfl_sync(full, lo, 7);
  t.r0 = (int64_t)(((uint64_t)__shfl_sync(full, hi, 8) << 32) | __shfl_sync(full, lo, 8));
  t.r1 = (int64_t)(((uint64_t)__shfl_sync(full, hi, 9) << 32) | __shfl_sync(full, lo, 9));
  t.gmask = ((uint64_t)__shfl_sync(full, hi, 10) << 32) | __shfl_sync(full, lo, 10);
  return t;
}

// whether patch M's ghost-entry list goes into the stage
template <int DIM, int P>
__device__ __forceinline__ bool pipe_gl_staged(const PipeMeta& M) {
  return M.g1 - M.g0 <= PipeGeo<DIM, P>::GCAP;
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// bulk prefetch of bytes (a multiple of 16) at a 16-byte aligned address into L2
__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// lane 0: bulk prefetch of patch M's record into L2
template <typename T>
__device__ __forceinline__ void prefetch_record(const PipeLevel<T>& L, const PipeMeta& M, int tid) {
  if (tid == 0 && M.r1 > M.r0) prefetch_l2(L.rec + M.r0, (uint32_t)((M.r1 - M.r0) * sizeof(T)));
}

// Issue every load of patch j into the team's stage by cp.async (one
// group per thread): the closure of x and b, the DoF list, items, cell
// kinds, the boundary-face moments and (when it fits the stage) the
// ghost-entry list; with `prefetch`, thread 0 also starts a bulk prefetch of
// the patch's record into L2, read later by the row products and the solve.
// All threads of the team call it (tid: index in the team), after the team
// is done with the previous patch.
template <int DIM, int P, typename T, int GW = 1>
__device__ __forceinline__ void warp_issue(const PipeLevel<T>& L, const PipeMeta& M, const PatchPos& pp, int j,
                                           WarpStage<DIM, P, T>& st, const WarpLane<DIM, P, T>& wl,
                                           const CutTables<DIM, P>& tb, bool prefetch, int tid) {
  using G = PipeGeo<DIM, P>;
  constexpr int TS = 32 * GW;
  const int n = wl.n;
  if (prefetch) prefetch_record(L, M, tid);
  if (pipe_gl_staged<DIM, P>(M)) {
    // lists are 16-byte aligned runs of a multiple of 8 entries
    const int nch = (M.g1 - M.g0) / 8;
    for (int w = tid; w < nch; w += TS) cp_async16(&st.gl[8 * w], L.gent + M.g0 + 8 * w);
  }
  // a closure inside the lattice needs no per-node test
  const int* c0 = pp.c0;
  const int base = pp.base;
  const bool inside = pp.inside;
  for (int e = tid; e < G::NCL; e += TS) {
    const int code = tb.uc[e];
    int rel = 0, stn = 1;
    bool in = true;
#pragma unroll
    for (int kk = 0; kk < DIM; ++kk) {
      const int u = (code >> (4 * kk)) & 15;
      rel += u * stn;
      stn *= n;
      if (!inside) {
        const int c = c0[kk] + u;
        if (c < 0 || c >= n) in = false;
      }
    }
    if (in) {
      const int o = base + rel;
      cp_async_elem(&st.x[e], L.x + o);
      cp_async_elem(&st.b[e], L.b + o);
    } else {
      st.x[e] = T(0);
      st.b[e] = T(0);
    }
    if (e < M.m) cp_async_elem(&st.mem[e], L.members + M.mo + e);
  }
  for (int w = tid; w < (M.nit + 3) / 4; w += TS) cp_async_elem(&st.item[w], L.items + M.io + w);
  if (tid < G::NCELL) cp_async_elem(&st.pk[tid], L.pk + (size_t)j * G::NCELL + tid);
  // moments of the block-boundary ghost faces (one slot per set bit), in
  // 8-byte pieces (a slot holds an even number of FP32 values)
  const int nbv = __popcll(M.gmask & pipe_bnd_bits<DIM, P>()) * P * G::NT;
  const int nch = nbv * (int)sizeof(T) / 8;
  const char* src = reinterpret_cast<const char*>(L.Gb + (size_t)M.gb * P * G::NT);
  char* dst = reinterpret_cast<char*>(&st.U[0][0][0]);
  for (int w = tid; w < nch; w += TS) cp_async8(dst + 8 * w, src + 8 * (size_t)w);
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// four consecutive read-only values from a 16-byte aligned global address
__device__ __forceinline__ void ldg4(const float* p, float (&v)[4]) {
  const float4 t = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ __forceinline__ void ldg4(const double* p, double (&v)[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

// four consecutive values from a 16-byte aligned address (shared or global)
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

// lattice offset of closure node o (first coordinate fastest) from the
// closure's first node, on a lattice of n nodes per direction
template <int DIM, int P>
__device__ __forceinline__ int closure_offset(int o, int n) {
  constexpr int C = 2 * P + 1;
  int off = 0, stn = 1;
#pragma unroll
  for (int kk = 0; kk < DIM; ++kk) {
    off += (o % C) * stn;
    o /= C;
    stn *= n;
  }
  return off;
}

// One patch from a filled stage, by one team of GW warps (tid: index in the
// team; lane: index in the warp):
//   1. x on the nodes of each patch cell (cell vectors, padded to NBP);
//   2. G_m of the middle-plane ghost faces, NT lanes per face: lane t forms
//      J_m[t] = sum_i dvec_m[i] x(i, t) across the face, then the face mass
//      Mhat x Mhat in 1D passes by shuffles inside the lane group, times
//      coef_m;  and one lane per item: the cell row (record, or the uncut
//      element matrix for h = 1 times h^(d-2); 16-byte loads through the
//      read-only path) times the cell vector;
//   3. residual of the patch rows, one thread per row: b - (cell parts in
//      cell order, then the row's ghost entries in list order);
//   4. delta = A_j^{-1} r, one thread per row, reading its row of the
//      inverse and r four entries at a time; x updated in place.
// Every row and every face is formed by one thread or one lane group with
// the same operations whatever GW is, so the result does not depend on it.
// kp: the uncut element matrix for h = 1 (rows padded, global); tb: the
// block's tables; rec: the record (global); gl: the ghost-entry list.
// Products and solve rows run in independent partial sums (fixed split,
// fixed order).
template <int DIM, int P, typename T, int GW = 1>
__device__ __forceinline__ void warp_compute(const T* __restrict__ kp, T* __restrict__ xg, int base,
                                             WarpStage<DIM, P, T>& st, const WarpLane<DIM, P, T>& wl,
                                             const CutTables<DIM, P>& tb, const T* __restrict__ rec,
                                             const uint16_t* gl, const PipeMeta& M, int lane, int tid) {
  using G = PipeGeo<DIM, P>;
  constexpr int C = G::C, NB = G::NB, NBP = G::NBP, NTF = G::NT;
  constexpr int TS = 32 * GW;
  constexpr int KR = (G::NCL + TS - 1) / TS;  // rows per thread
  constexpr uint64_t bnd = pipe_bnd_bits<DIM, P>();
  const uint64_t gint = M.gmask & ~bnd;
  const int nbf = __popcll(M.gmask & bnd), nf = __popcll(gint);
  for (int f = tid; f < G::NFACE; f += TS)
    if ((gint >> f) & 1ull) st.flist[__popcll(gint & ((1ull << f) - 1ull))] = f;
  const int pkl = lane < G::NCELL ? st.pk[lane] : -2;
  const uint32_t amask = __ballot_sync(0xffffffffu, pkl != -2);  // active patch cells
  T* xc = &st.xc[0][0];
  for (int idx = tid; idx < G::NCELL * G::NB; idx += TS) {
    const int v = tb.xcm[idx];
    xc[v >> 16] = st.x[v & 0xffff];
  }
  team_sync<GW>();
  // 2a. middle-plane face moments
  {
    constexpr int FPR = 32 / NTF;
    const int grp = lane / NTF, t = lane - grp * NTF, t0 = t % (P + 1), t1 = t / (P + 1) % (P + 1);
    const int g0 = grp * NTF;
    for (int f0 = (tid >> 5) * FPR; f0 < nf; f0 += FPR * GW) {
      const int fi = f0 + grp;
      const bool act = grp < FPR && fi < nf;
      T J[P];
#pragma unroll
      for (int mm = 0; mm < P; ++mm) J[mm] = T(0);
      if (act) {
        const int f = st.flist[fi], u = f % G::HALF, k = f / G::HALF / 3;
        int o = 0, stc = 1, q = 0, tt = t, sk = 1;
#pragma unroll
        for (int kk = 0; kk < DIM; ++kk) {
          if (kk == k) {
            sk = stc;
          } else {
            o += (P * ((u >> q) & 1) + tt % (P + 1)) * stc;
            tt /= P + 1;
            ++q;
          }
          stc *= C;
        }
#pragma unroll
        for (int i = 0; i <= 2 * P; ++i) {
          const T xv = st.x[o + i * sk];
#pragma unroll
          for (int mm = 0; mm < P; ++mm) J[mm] += st.dv[mm][i] * xv;
        }
      }
#pragma unroll
      for (int mm = 0; mm < P; ++mm) {
        T a = T(0);
#pragma unroll
        for (int s0 = 0; s0 <= P; ++s0) a += wl.mh0[s0] * __shfl_sync(0xffffffffu, J[mm], g0 + s0 + (P + 1) * t1);
        T g = a;
        if (DIM == 3) {
          g = T(0);
#pragma unroll
          for (int s1 = 0; s1 <= P; ++s1) g += wl.mh1[s1] * __shfl_sync(0xffffffffu, a, g0 + t0 + (P + 1) * s1);
        }
        if (act) st.U[nbf + fi][mm][t] = wl.cf[mm] * g;
      }
    }
  }
  // 2b. cell rows of the items
  const int m = M.m, MP = (m + 3) / 4 * 4;
  {
    // one item per lane: its row (16-byte loads) times the cell vector
    const T* rows = rec + (size_t)m * MP;
    const uint8_t* item = reinterpret_cast<const uint8_t*>(st.item);
    for (int q = tid; q < M.nit; q += TS) {
      const int it = item[q], sc = it / NB, jj = it - sc * NB;
      const int pkv = st.pk[sc];
      const bool unc = pkv == -1;
      const T* row = unc ? kp + jj * NBP : rows + (size_t)((pkv >> 8) + q - (pkv & 255)) * NBP;
      const T* xv = &st.xc[sc][0];
      T acc[2] = {T(0), T(0)};  // entries of 4-groups 0, 2, 4, .. and 1, 3, 5, ..
#pragma unroll
      for (int c0 = 0; c0 < NBP; c0 += 4) {
        T a4[4], x4[4];
        ldg4(row + c0, a4);
        ld4(xv + c0, x4);
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (c0 + c < NB) acc[(c0 / 4) & 1] += a4[c] * x4[c];
      }
      const T sum = acc[0] + acc[1];
      st.part[sc][jj] = unc ? wl.ksc * sum : sum;
    }
  }
  team_sync<GW>();
  // 3. residual of the patch rows (tid + TS k)
#pragma unroll 1
  for (int k = 0; k < KR; ++k) {
    const int e = tid + TS * k;
    if (e >= m) {
      if (e < MP) st.r[e] = T(0);
      continue;
    }
    const int o = st.mem[e];
    const uint64_t tab = tb.cpt[o];
    T acc = T(0);
#pragma unroll
    for (int sc = 0; sc < G::NCELL; ++sc) {
      const int jj = (int)((tab >> (8 * sc)) & 0xffu);
      if (jj != 0xff && ((amask >> sc) & 1u)) acc += st.part[sc][jj];
    }
    const int q1 = gl[e + 1];
    for (int q = gl[e]; q < q1; ++q) {
      const int en = gl[m + 1 + q], slot = en & 63, i = (en >> 6) & 15, t = en >> 10;
      const T* g = &st.U[slot][0][t];
#pragma unroll
      for (int mm = 0; mm < P; ++mm) acc += st.dv[mm][i] * g[mm * NTF];
    }
    st.r[e] = st.b[o] - acc;
  }
  team_sync<GW>();
  // 4. local solve delta = A^{-1} r, x updated in place: one lane per row
  //    e, reading row e of the inverse (4 entries per load; zeros in the
  //    padding), columns in 4 partial sums by c mod 4, in increasing c; the
  //    loads of 4 groups of 4 columns issued before their products
  const int n = wl.n;
#pragma unroll 1
  for (int k = 0; k < KR; ++k) {
    const int e = tid + TS * k;
    if (e >= m) break;
    const T* Ae = rec + (size_t)e * MP;
    T a[4] = {T(0), T(0), T(0), T(0)};
    for (int c0 = 0; c0 < MP; c0 += 16) {
      T a4[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (c0 + 4 * u < MP) ldg4(Ae + c0 + 4 * u, a4[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (c0 + 4 * u >= MP) break;
        T r4[4];
        ld4(&st.r[c0 + 4 * u], r4);
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) a[qq] += a4[u][qq] * r4[qq];
      }
    }
    const T acc = (a[0] + a[1]) + (a[2] + a[3]);
    const int o = st.mem[e];
    xg[base + closure_offset<DIM, P>(o, n)] = st.x[o] + acc;
  }
  team_sync<GW>();
}

// The loop of one team (GW warps: one warp, or the whole block) over the
// work items it, it + step, .. below total; every warp of the team reads the
// metadata itself.
// locate(item, level, patch) gives an item's level descriptor and patch.
// st: the warp's stage; tb: the block's tables.  Per item: issue the
// loads, read the next item's metadata while they fly, wait for the
// cp.async group, compute.  prefetch: 0 no record prefetch; 1 each record
// prefetched into L2 when its patch's loads are issued; 2 the next item's
// record prefetched as soon as its metadata is read, one patch ahead of its
// use (the first item's at its issue).
template <int DIM, int P, typename T, int GW = 1, class Locate>
__device__ __forceinline__ void warp_loop(int it, int step, int total, Locate&& locate, WarpStage<DIM, P, T>& st,
                                          const CutTables<DIM, P>& tb, int prefetch) {
  if (it >= total) return;
  const int lane = threadIdx.x & 31, tid = threadIdx.x % (32 * GW);
  WarpLane<DIM, P, T> wl;
  wl.lv = nullptr;
  const PipeLevel<T>* Lc;
  int jc;
  locate(it, Lc, jc);
  PipeMeta cur = pipe_meta_gather(lane < kMetaFields ? pipe_meta_field(*Lc, jc, lane) : 0);
  bool first = true;
  for (; it < total; it += step) {
    if (wl.lv != Lc) warp_lane_level<DIM, P, T, GW>(wl, st, Lc->op, Lc->ksc, Lc, lane, tid);
    const PatchPos pp = patch_pos<DIM, P, T>(cur.vert, wl);
    warp_issue<DIM, P, T, GW>(*Lc, cur, pp, jc, st, wl, tb, prefetch == 1 || (prefetch == 2 && first), tid);
    first = false;
    const PipeLevel<T>* Ln = Lc;
    int jn = jc;
    const bool more = it + step < total;
    uint64_t nv = 0;  // this lane's field of the next patch's metadata
    if (more) {
      locate(it + step, Ln, jn);
      if (lane < kMetaFields) nv = pipe_meta_field(*Ln, jn, lane);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    team_sync<GW>();
    if (more && prefetch == 2) {
      const uint64_t r1 = __shfl_sync(0xffffffffu, nv, 9);
      if (tid == 8 && r1 > nv) prefetch_l2(Ln->rec + nv, (uint32_t)((r1 - nv) * sizeof(T)));
    }
    const uint16_t* gl = pipe_gl_staged<DIM, P>(cur) ? st.gl : Lc->gent + cur.g0;
    warp_compute<DIM, P, T, GW>(Lc->kp, Lc->x, pp.base, st, wl, tb, Lc->rec + cur.r0, gl, cur, lane, tid);
    team_sync<GW>();
    if (more) cur = pipe_meta_gather(nv);
    Lc = Ln;
    jc = jn;
  }
}

// record prefetch mode of the automatic launch choice (warp_loop)
constexpr int kCutPrefetch = 1;

// resident blocks per SM the kernel is compiled for (registers): two blocks
// of eight warps leave 128 registers per thread, which this kernel uses
// without spilling (with three blocks the FP32 form spills; measured no
// faster)
template <typename T>
constexpr int cut_min_blocks() {
  return 2;
}

// One colour step: patches j0 .. j0 + npatch - 1, warp w of the grid takes
// w, w + (warps of the grid), ..; `prefetch` as in warp_loop.  The level
// descriptor is copied to shared memory once.
template <int DIM, int P, typename T, int WPB>
__global__ void __launch_bounds__(32 * WPB, cut_min_blocks<T>())
    k_cut_warp(PipeLevel<T> L, int j0, int npatch, int prefetch) {
  extern __shared__ __align__(128) unsigned char wsm[];
  __shared__ PipeLevel<T> sL;
  __shared__ CutTables<DIM, P> tb;
  if (threadIdx.x == 0) sL = L;
  cut_tables<DIM, P>(tb);
  __syncthreads();
  const PipeLevel<T>* Lp = &sL;
  const int warp = threadIdx.x >> 5;
  warp_loop<DIM, P, T>(
      blockIdx.x * WPB + warp, gridDim.x * WPB, npatch,
      [&](int it, const PipeLevel<T>*& lv, int& j) {
        lv = Lp;
        j = j0 + it;
      },
      *reinterpret_cast<WarpStage<DIM, P, T>*>(wsm + (size_t)warp * warp_stage_bytes<DIM, P, T>()), tb,
      prefetch);
}

// The same colour step with one patch per block at a time, worked on by the
// block's GW warps together (colours of few patches: shorter chains of
// dependent steps per patch, the same arithmetic per row and face).
template <int DIM, int P, typename T, int GW>
__global__ void __launch_bounds__(32 * GW) k_cut_team(PipeLevel<T> L, int j0, int npatch, int prefetch) {
  extern __shared__ __align__(128) unsigned char wsm[];
  __shared__ PipeLevel<T> sL;
  __shared__ CutTables<DIM, P> tb;
  if (threadIdx.x == 0) sL = L;
  cut_tables<DIM, P>(tb);
  __syncthreads();
  const PipeLevel<T>* Lp = &sL;
  warp_loop<DIM, P, T, GW>(
      blockIdx.x, gridDim.x, npatch,
      [&](int it, const PipeLevel<T>*& lv, int& j) {
        lv = Lp;
        j = j0 + it;
      },
      *reinterpret_cast<WarpStage<DIM, P, T>*>(wsm), tb, prefetch);
}

}  // namespace cutmg

namespace cutmg {

// Cut-patch inverses on the device, FP64 (the local solver's setup, Sec. 3):
// for patch j, rec[roff[j] ..] holds A_j by rows with row stride
// MP = 4 ceil(m / 4) (symmetric; its lower triangle is read) on entry and
// A_j^{-1} (both triangles, the same layout) on exit.  One block per patch (block-stride),
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
    const int m = cnt[j], mp = (m + 3) / 4 * 4;
    double* a = rec + roff[j];
    const int ne = m * (m + 1) / 2;
    if (tid == 0) bad = 0;
    for (int e = tid; e < ne; e += NT) {
      const int i = tri_row(e), c = e - i * (i + 1) / 2;
      S[i * ld + c] = a[(size_t)i * mp + c];
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
        a[(size_t)i * mp + c] = s;
        a[(size_t)c * mp + i] = s;
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
