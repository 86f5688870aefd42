// Device kernels of the CutFEM multigrid hot path (sm_103a), templated on the
// dimension, the polynomial degree and the arithmetic type (double for the
// plain form, float for the mixed form's V-cycle).
//
// Layout: every level vector lives on the full (pN+1)^DIM lattice ("box"),
// first coordinate fastest; inactive nodes hold zero and are never written.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace cutmg {

constexpr uint8_t kActive = 1;
constexpr uint8_t kCutCell = 2;

template <int DIM, int P>
struct Shape {
  static constexpr int NB = (DIM == 2) ? (P + 1) * (P + 1) : (P + 1) * (P + 1) * (P + 1);
  static constexpr int C = 2 * P + 1;  // closure nodes per direction of a patch
  static constexpr int M = 2 * P - 1;  // interior nodes per direction of a patch
  static constexpr int NO = (DIM == 2) ? P * P : P * P * P;  // nodes owned by a position
};

// Everything the matrix-free operator needs on one level.
template <typename T>
struct OpArgs {
  int N, n;               // cells and nodes per direction
  const uint8_t* cflag;   // N^DIM cell flags
  const int* cut_id;      // N^DIM index of the cut-cell matrix, -1 if none
  const T* cutmat;        // [n_cut][NB][NB] volume + Nitsche terms of cut cells
  const T* Kref;          // [NB][NB] stiffness of an uncut cell
  T dvec[4][9];           // jump weights of the m-th normal derivative across a face (m <= p <= 4)
  T coef[4];              // gamma_m h^(2m-1)/(m!)^2 h^(DIM-1)
  T Mhat[5][5];           // 1D reference mass matrix
  const int* face_id;     // [N^DIM][DIM] index of the ghost face (c, c + e_k), -1 if none
  T* G;                   // [n_ghost][P][(P+1)^(DIM-1)] face moments of the current x
};

// ---------------------------------------------------------------------------
// Ghost faces.  For the face F between cells L and L + e_k the penalty
// couples the (2P+1) x (P+1)^(DIM-1) nodes of the two cells:
//   (G_F x)(i, t) = sum_m dvec_m[i] G_m[t],
//   G_m[t] = coef_m sum_t' prod_j Mhat[t_j][t'_j] sum_i' dvec_m[i'] x(i', t').
// k_face_moments evaluates G_m[t] once per ghost face for the current x; the
// rows then only look them up.
template <int DIM, int P>
struct FaceGeo {
  static constexpr int NT = (DIM == 2) ? P + 1 : (P + 1) * (P + 1);
  static constexpr int PER_WARP = 32 / NT;  // faces one warp evaluates together
};

// One face on NT lanes of a warp: lane t = (t0, t1) forms the jumps J_m[t]
// of its node column; the face mass Mhat x Mhat is applied in two 1D passes
// across the group by shuffles, and lane t writes G_m[t].  All 32 lanes must
// call this (packed < 0: padding lane).
template <int DIM, int P, typename T>
__device__ __forceinline__ void face_moment_lanes(const OpArgs<T>& A, const T* __restrict__ x, int packed, int lane,
                                                  T* out0, T* out1) {
  constexpr int NT = FaceGeo<DIM, P>::NT;
  const int grp = lane / NT, t = lane - grp * NT;
  T J[P];
#pragma unroll
  for (int m = 0; m < P; ++m) J[m] = T(0);
  if (packed >= 0) {
    const int k = packed % DIM;
    int c = packed / DIM, lc[3] = {0, 0, 0};
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      lc[j] = c % A.N;
      c /= A.N;
    }
    const int n = A.n;
    const int sk = (k == 0) ? 1 : (k == 1 ? n : n * n);
    int tdim[2] = {0, 0}, q = 0;
#pragma unroll
    for (int j = 0; j < DIM; ++j)
      if (j != k) tdim[q++] = j;
    const int s0 = (tdim[0] == 0) ? 1 : (tdim[0] == 1 ? n : n * n);
    const int s1 = (DIM == 3) ? ((tdim[1] == 0) ? 1 : (tdim[1] == 1 ? n : n * n)) : 0;
    const int base = P * (lc[0] + n * (lc[1] + (DIM == 3 ? n * lc[2] : 0)));
    const int off = base + (t % (P + 1)) * s0 + (DIM == 3 ? (t / (P + 1)) * s1 : 0);
    T xv[2 * P + 1];
#pragma unroll
    for (int ip = 0; ip <= 2 * P; ++ip) xv[ip] = x[off + ip * sk];
#pragma unroll
    for (int ip = 0; ip <= 2 * P; ++ip)
#pragma unroll
      for (int m = 0; m < P; ++m) J[m] += A.dvec[m][ip] * xv[ip];
  }
  const int src = (grp * NT < 32 - NT) ? grp * NT : 32 - NT;
  const int t0 = t % (P + 1), t1 = t / (P + 1);
  // face mass by sum factorisation: one 1D pass per face direction
  T acc[P];
#pragma unroll
  for (int m = 0; m < P; ++m) acc[m] = T(0);
#pragma unroll
  for (int q = 0; q <= P; ++q) {
    const T w = A.Mhat[t0][q];
#pragma unroll
    for (int m = 0; m < P; ++m) acc[m] += w * __shfl_sync(0xffffffffu, J[m], src + q + (P + 1) * t1);
  }
  if (DIM == 3) {
    T h[P];
#pragma unroll
    for (int m = 0; m < P; ++m) {
      h[m] = acc[m];
      acc[m] = T(0);
    }
#pragma unroll
    for (int q = 0; q <= P; ++q) {
      const T w = A.Mhat[t1][q];
#pragma unroll
      for (int m = 0; m < P; ++m) acc[m] += w * __shfl_sync(0xffffffffu, h[m], src + t0 + (P + 1) * q);
    }
  }
  if (packed >= 0) {
#pragma unroll
    for (int m = 0; m < P; ++m) {
      const T g = A.coef[m] * acc[m];
      if (out0) out0[m * NT + t] = g;
      if (out1) out1[m * NT + t] = g;
    }
  }
}

template <int DIM, int P, typename T>
__global__ void __launch_bounds__(128) k_face_moments(OpArgs<T> A, const T* __restrict__ x,
                                                      const int* __restrict__ faces,
                                                      const int* __restrict__ ids, int nfaces) {
  constexpr int NT = FaceGeo<DIM, P>::NT, PW = FaceGeo<DIM, P>::PER_WARP;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp * PW >= nfaces) return;  // whole warp
  const int i = warp * PW + lane / NT;
  const bool ok = lane / NT < PW && i < nfaces;
  const int f = ok ? (ids ? ids[i] : i) : 0;
  face_moment_lanes<DIM, P, T>(A, x, ok ? faces[f] : -1, lane, A.G + (size_t)f * P * NT, nullptr);
}

// The moments of listed ghost faces written to one or two destinations
// (offsets in units of P (p+1)^(d-1) values into `out`, -1: none): the
// block-boundary faces of the cut patches of a colour, each copied into the
// moment slots of the (at most two) patches whose rows read it.
template <int DIM, int P, typename T>
__global__ void __launch_bounds__(128) k_face_moments_to(OpArgs<T> A, const T* __restrict__ x,
                                                         const int* __restrict__ faces, const int* __restrict__ ids,
                                                         const int* __restrict__ dst, int nfaces, T* __restrict__ out) {
  constexpr int NT = FaceGeo<DIM, P>::NT, PW = FaceGeo<DIM, P>::PER_WARP;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp * PW >= nfaces) return;  // whole warp
  const int i = warp * PW + lane / NT;
  const bool ok = lane / NT < PW && i < nfaces;
  const int d0 = ok ? dst[2 * i] : -1, d1 = ok ? dst[2 * i + 1] : -1;
  face_moment_lanes<DIM, P, T>(A, x, ok ? faces[ids[i]] : -1, lane, d0 >= 0 ? out + (size_t)d0 * P * NT : nullptr,
                               d1 >= 0 ? out + (size_t)d1 * P * NT : nullptr);
}

// sum over the ghost faces whose two cells contain node idx of (G_F x)(node)
template <int DIM, int P, typename T>
__device__ __forceinline__ T node_faces(const OpArgs<T>& A, const int* idx) {
  constexpr int NT = FaceGeo<DIM, P>::NT;
  const int N = A.N;
  int cc[DIM][2], nopt[DIM];
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const int i = idx[k], a = i / P, r = i - a * P;
    int m = 0;
    if (r == 0) {
      if (a - 1 >= 0) cc[k][m++] = a - 1;
      if (a < N) cc[k][m++] = a;
    } else {
      cc[k][m++] = a;
    }
    nopt[k] = m;
  }
  T acc = T(0);
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const int i = idx[k], a = i / P, r = i - a * P;
    int Llo = (r == 0) ? a - 2 : a - 1, Lhi = a;
    if (Llo < 0) Llo = 0;
    if (Lhi > N - 2) Lhi = N - 2;
    int tdim[2] = {0, 0}, q = 0;
#pragma unroll
    for (int j = 0; j < DIM; ++j)
      if (j != k) tdim[q++] = j;
    const int n0 = nopt[tdim[0]], n1 = (DIM == 3) ? nopt[tdim[1]] : 1;
    for (int Lk = Llo; Lk <= Lhi; ++Lk)
      for (int u0 = 0; u0 < n0; ++u0)
        for (int u1 = 0; u1 < n1; ++u1) {
          int c[3] = {0, 0, 0};
          c[k] = Lk;
          c[tdim[0]] = cc[tdim[0]][u0];
          if (DIM == 3) c[tdim[1]] = cc[tdim[1]][u1];
          const int cell = (DIM == 2) ? c[0] + N * c[1] : c[0] + N * (c[1] + N * c[2]);
          const int id = A.face_id[cell * DIM + k];
          if (id < 0) continue;
          const int il = i - P * Lk;
          int t = idx[tdim[0]] - P * c[tdim[0]];
          if (DIM == 3) t += (P + 1) * (idx[tdim[1]] - P * c[tdim[1]]);
          const T* g = A.G + (size_t)id * P * NT;
#pragma unroll
          for (int m = 0; m < P; ++m) acc += A.dvec[m][il] * g[m * NT + t];
        }
  }
  return acc;
}

// (A x)_i for one lattice node: its active cells (cut-cell or uncut element
// matrix rows) plus its ghost faces (moments looked up).
template <int DIM, int P, typename T>
__device__ __forceinline__ T node_row(const OpArgs<T>& A, const T* __restrict__ x, const int* idx,
                                      const T* __restrict__ sK) {
  constexpr int NB = Shape<DIM, P>::NB;
  const int N = A.N, n = A.n;
  int cc[DIM][2], lc[DIM][2], nopt[DIM];
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const int i = idx[k], a = i / P, r = i - a * P;
    int m = 0;
    if (r == 0) {
      if (a - 1 >= 0) { cc[k][m] = a - 1; lc[k][m] = P; ++m; }
      if (a < N) { cc[k][m] = a; lc[k][m] = 0; ++m; }
    } else {
      cc[k][m] = a; lc[k][m] = r; ++m;
    }
    nopt[k] = m;
  }
  T acc = T(0);
  const int tot = (DIM == 2) ? nopt[0] * nopt[1] : nopt[0] * nopt[1] * nopt[2];
  for (int s = 0; s < tot; ++s) {
    int t = s, cell = 0, row = 0, base = 0, cst = 1, rst = 1, nst = 1;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const int o = t % nopt[k];
      t /= nopt[k];
      cell += cc[k][o] * cst;
      cst *= N;
      row += lc[k][o] * rst;
      rst *= (P + 1);
      base += P * cc[k][o] * nst;
      nst *= n;
    }
    const uint8_t f = A.cflag[cell];
    if (!(f & kActive)) continue;
    const T* Mrow = (f & kCutCell) ? (A.cutmat + (size_t)A.cut_id[cell] * NB * NB + row * NB)
                                   : (sK + row * NB);
    if (DIM == 2) {
#pragma unroll
      for (int j1 = 0; j1 <= P; ++j1)
#pragma unroll
        for (int j0 = 0; j0 <= P; ++j0) acc += Mrow[j0 + (P + 1) * j1] * x[base + j0 + n * j1];
    } else {
#pragma unroll
      for (int j2 = 0; j2 <= P; ++j2)
#pragma unroll
        for (int j1 = 0; j1 <= P; ++j1)
#pragma unroll
          for (int j0 = 0; j0 <= P; ++j0)
            acc += Mrow[j0 + (P + 1) * (j1 + (P + 1) * j2)] * x[base + j0 + n * (j1 + n * j2)];
    }
  }
  return acc + node_faces<DIM, P, T>(A, idx);
}

// ---------------------------------------------------------------------------
// Rows (A x)_i of the DoFs of a cut patch (vertex v, 2^DIM cells v-1+s) by
// one warp: the (2P+1)^DIM closure of x is staged in shared memory, every
// (patch cell, local node) pair whose node is a DoF of the patch gets its
// cell row times x once, then each DoF sums its cells in a fixed order and
// adds its ghost faces.  Every active cell containing a patch DoF is a patch
// cell (the support rule that defines the DoFs).
template <int DIM, int P>
struct PatchGeo {
  static constexpr int C = 2 * P + 1;
  static constexpr int NCL = (DIM == 2) ? C * C : C * C * C;
  static constexpr int NB = Shape<DIM, P>::NB;
  static constexpr int NCELL = 1 << DIM;
};

template <int DIM, int P, typename T>
struct PatchScratch {
  using G = PatchGeo<DIM, P>;
  T x[G::NCL];
  T part[G::NCELL][G::NB];
  T r[G::NCL];
  const T* rowbase[G::NCELL];  // element matrix of each patch cell, nullptr if inactive
  short mem[G::NCL];
};

template <int DIM>
__device__ __forceinline__ int lat_index(const int* c, int n) {
  return (DIM == 2) ? c[0] + n * c[1] : c[0] + n * (c[1] + n * c[2]);
}

// synchronisation of the threads that work on one patch
template <int NT>
__device__ __forceinline__ void psync() {
  if (NT <= 32)
    __syncwarp();
  else
    __syncthreads();
}

template <int DIM, int P, typename T, int NT = 32>
__device__ __forceinline__ void patch_rows(const OpArgs<T>& A, const T* __restrict__ x, const int* v,
                                           const uint16_t* __restrict__ tgt, int m,
                                           const int* __restrict__ fofs, const int* __restrict__ fent,
                                           PatchScratch<DIM, P, T>& S, const T* __restrict__ sK,
                                           int lane) {
  using G = PatchGeo<DIM, P>;
  constexpr int C = G::C, NB = G::NB, NTF = FaceGeo<DIM, P>::NT;
  const int N = A.N, n = A.n;
  constexpr int NROUND = (G::NCL + NT - 1) / NT;
#pragma unroll
  for (int rr = 0; rr < NROUND; ++rr) {
    const int e = lane + NT * rr;
    if (e < G::NCL) {
      int u = e, c[3] = {0, 0, 0};
      bool in = true;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        c[k] = P * (v[k] - 1) + u % C;
        u /= C;
        if (c[k] < 0 || c[k] >= n) in = false;
      }
      S.x[e] = in ? x[lat_index<DIM>(c, n)] : T(0);
      S.mem[e] = -1;
    }
  }
  if (lane < G::NCELL) {
    int c[3] = {0, 0, 0};
    bool ok = true;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      c[k] = v[k] - 1 + ((lane >> k) & 1);
      if (c[k] < 0 || c[k] >= N) ok = false;
    }
    const T* rb = nullptr;
    if (ok) {
      const int cell = (DIM == 2) ? c[0] + N * c[1] : c[0] + N * (c[1] + N * c[2]);
      const uint8_t fl = A.cflag[cell];
      if (fl & kActive) rb = (fl & kCutCell) ? A.cutmat + (size_t)A.cut_id[cell] * NB * NB : sK;
    }
    S.rowbase[lane] = rb;
  }
  psync<NT>();
  for (int e = lane; e < m; e += NT) S.mem[tgt[e]] = (short)e;
  psync<NT>();
  for (int it = lane; it < G::NCELL * NB; it += NT) {
    const int s = it / NB, j = it - s * NB;
    int c[3] = {0, 0, 0}, o = 0, ost = 1, u = j, base = 0;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const int sk = (s >> k) & 1, a = u % (P + 1);
      u /= (P + 1);
      c[k] = v[k] - 1 + sk;
      if (c[k] < 0 || c[k] >= N) ok = false;
      o += (P * sk + a) * ost;
      base += P * sk * ost;
      ost *= C;
    }
    if (!ok || S.mem[o] < 0 || !S.rowbase[s]) continue;
    const T* row = S.rowbase[s] + j * NB;
    T acc = T(0);
    if (DIM == 2) {
#pragma unroll
      for (int q1 = 0; q1 <= P; ++q1)
#pragma unroll
        for (int q0 = 0; q0 <= P; ++q0) acc += row[q0 + (P + 1) * q1] * S.x[base + q0 + C * q1];
    } else {
#pragma unroll
      for (int q2 = 0; q2 <= P; ++q2)
#pragma unroll
        for (int q1 = 0; q1 <= P; ++q1)
#pragma unroll
          for (int q0 = 0; q0 <= P; ++q0)
            acc += row[q0 + (P + 1) * (q1 + (P + 1) * q2)] * S.x[base + q0 + C * (q1 + C * q2)];
    }
    S.part[s][j] = acc;
  }
  psync<NT>();
  for (int e = lane; e < m; e += NT) {
    int o[3] = {0, 0, 0}, u = tgt[e];
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      o[k] = u % C;
      u /= C;
    }
    T acc = T(0);
#pragma unroll
    for (int s = 0; s < G::NCELL; ++s) {
      int j = 0, jst = 1;
      bool in = S.rowbase[s] != nullptr;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const int sk = (s >> k) & 1, a = o[k] - P * sk;
        if (a < 0 || a > P) in = false;
        j += a * jst;
        jst *= (P + 1);
      }
      if (in) acc += S.part[s][j];
    }
    const int f0 = fofs[e], f1 = fofs[e + 1];
    for (int q0 = f0; q0 < f1; q0 += 8) {
      int ent[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) ent[u] = (q0 + u < f1) ? fent[q0 + u] : -1;
      T gv[8][P];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (ent[u] < 0) continue;
        const T* g = A.G + (size_t)(ent[u] >> 4) / NTF * (P * NTF) + (ent[u] >> 4) % NTF;
#pragma unroll
        for (int mm = 0; mm < P; ++mm) gv[u][mm] = g[mm * NTF];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (ent[u] < 0) continue;
        const int il = ent[u] & 15;
#pragma unroll
        for (int mm = 0; mm < P; ++mm) acc += A.dvec[mm][il] * gv[u][mm];
      }
    }
    S.r[e] = acc;
  }
  psync<NT>();
}

template <int NB, typename T>
__device__ __forceinline__ void stage_kref(const T* __restrict__ g, T* s) {
  for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) s[i] = g[i];
  __syncthreads();
}

// y = A x (b == nullptr) or y = b - A x, at the active nodes of positions whose
// 2^DIM surrounding cells are all plain interior cells: each thread owns the
// P^DIM nodes P a + alpha, alpha in [0, P)^DIM, and sums their rows over the
// 2^DIM cells with the uncut element matrix.
template <int DIM, int P, typename T>
__device__ __forceinline__ void bulk_body(const OpArgs<T>& A, const T* __restrict__ x,
                                          const T* __restrict__ b, T* __restrict__ y, int q,
                                          const T* __restrict__ sK) {
  constexpr int NB = Shape<DIM, P>::NB;
  constexpr int NO = Shape<DIM, P>::NO;
  const int np = A.N + 1, n = A.n;
  int a[3] = {0, 0, 0};
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    a[k] = q % np;
    q /= np;
  }
  T out[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) out[o] = T(0);
#pragma unroll
  for (int s = 0; s < (1 << DIM); ++s) {
    int base = 0, st = 1;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      base += P * (a[k] - ((s >> k) & 1)) * st;
      st *= n;
    }
    T xv[NB];
    if (DIM == 2) {
#pragma unroll
      for (int j1 = 0; j1 <= P; ++j1)
#pragma unroll
        for (int j0 = 0; j0 <= P; ++j0) xv[j0 + (P + 1) * j1] = x[base + j0 + n * j1];
    } else {
#pragma unroll
      for (int j2 = 0; j2 <= P; ++j2)
#pragma unroll
        for (int j1 = 0; j1 <= P; ++j1)
#pragma unroll
          for (int j0 = 0; j0 <= P; ++j0)
            xv[j0 + (P + 1) * (j1 + (P + 1) * j2)] = x[base + j0 + n * (j1 + n * j2)];
    }
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      int al[3] = {0, 0, 0}, u = o;
      bool in = true;
      int row = 0, rst = 1;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        al[k] = u % P;
        u /= P;
        const int sk = (s >> k) & 1;
        if (sk && al[k] != 0) in = false;
        row += (sk ? P : al[k]) * rst;
        rst *= (P + 1);
      }
      if (!in) continue;
      T acc = T(0);
#pragma unroll
      for (int j = 0; j < NB; ++j) acc += sK[row * NB + j] * xv[j];
      out[o] += acc;
    }
  }
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    int u = o, node = 0, st = 1;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      node += (P * a[k] + u % P) * st;
      u /= P;
      st *= n;
    }
    y[node] = b ? b[node] - out[o] : out[o];
  }
}

template <int DIM, int P, typename T>
__global__ void __launch_bounds__(128) k_apply_bulk(OpArgs<T> A, const T* __restrict__ x,
                                                    const T* __restrict__ b, T* __restrict__ y,
                                                    const int* __restrict__ pos, int npos) {
  constexpr int NB = Shape<DIM, P>::NB;
  __shared__ T sK[NB * NB];
  stage_kref<NB>(A.Kref, sK);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npos) return;
  bulk_body<DIM, P, T>(A, x, b, y, pos[t], sK);
}

// Same output for the remaining active nodes (near the boundary), one thread
// per node: its cells' rows and its ghost faces (moments precomputed).
template <int DIM, int P, typename T>
__device__ __forceinline__ void bnd_body(const OpArgs<T>& A, const T* __restrict__ x,
                                         const T* __restrict__ b, T* __restrict__ y, int node,
                                         const T* __restrict__ sK) {
  int idx[3] = {0, 0, 0}, u = node;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    idx[k] = u % A.n;
    u /= A.n;
  }
  const T v = node_row<DIM, P, T>(A, x, idx, sK);
  y[node] = b ? b[node] - v : v;
}

template <int DIM, int P, typename T>
__global__ void __launch_bounds__(128) k_apply_bnd(OpArgs<T> A, const T* __restrict__ x,
                                                   const T* __restrict__ b, T* __restrict__ y,
                                                   const int* __restrict__ nodes, int nn) {
  constexpr int NB = Shape<DIM, P>::NB;
  __shared__ T sK[NB * NB];
  stage_kref<NB>(A.Kref, sK);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nn) return;
  bnd_body<DIM, P, T>(A, x, b, y, nodes[t], sK);
}

// ---------------------------------------------------------------------------
// Interior-patch colour step (Sec. 3, fast diagonalisation): one warp per
// patch.  r_I = b_I - (sum_k (x)_k Kbar/Mbar)[I, closure] x_closure by sum
// factorisation over the 2p+1 closure lattice; delta = (S x..x S)
// diag(1/sum lam) (S^T x..x S^T) r_I; x_I += delta.  Patches of one colour
// have disjoint closures' interiors and no ghost coupling, so every warp
// reads only values no other warp of the launch writes.
template <typename T, int P>
struct FdArgs {
  static constexpr int C = 2 * P + 1, M = 2 * P - 1;
  T Mr[M][C], Kr[M][C];  // interior rows of the two-cell 1D mass / stiffness
  T S[M][M];             // K_I S = M_I S diag(lam), S^T M_I S = I
  T lam[M];
  T dinv[M * M * M];     // 1 / (lam_a + lam_b (+ lam_c)), index a + M (b + M c), formed in FP64
};

template <int DIM, int P>
struct CartGeo {
  static constexpr int C = 2 * P + 1, M = 2 * P - 1;
  static constexpr int NC = (DIM == 2) ? C * C : C * C * C;
  static constexpr int NI = (DIM == 2) ? M * M : M * M * M;
  static constexpr int NU = (DIM == 2) ? M * C : M * C * C;  // after the first contraction
  static constexpr int NV = (DIM == 2) ? 1 : M * M * C;       // after the second (3D)
};

template <int DIM, int P, typename T>
struct CartScratch {
  using G = CartGeo<DIM, P>;
  T x[G::NC];
  T u[2][G::NU];
  T v[3][G::NV];
  T r[G::NI];
  T t[G::NI];
};

// NT threads (a half-warp, a warp, or a block for latency-bound launches)
// per patch; with live == false the patch is worked on but x is not written
// (the idle half of a warp keeps its synchronisations)
template <int DIM, int P, typename T, int NT = 32>
__device__ __forceinline__ void cart_body(const FdArgs<T, P>& F, int N, int n, T* __restrict__ x,
                                          const T* __restrict__ b, int vert, int lane,
                                          CartScratch<DIM, P, T>& CS, bool live = true) {
  constexpr int C = 2 * P + 1, M = 2 * P - 1;
  constexpr int NC = CartGeo<DIM, P>::NC;
  constexpr int NI = CartGeo<DIM, P>::NI;
  const int np = N + 1;
  int q = vert, v[3] = {0, 0, 0};
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    v[k] = q % np;
    q /= np;
  }
  int base = 0;
  {
    int s = 1;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      base += P * (v[k] - 1) * s;
      s *= n;
    }
  }
  T* X = CS.x;
  for (int e = lane; e < NC; e += NT) {
    int o0 = e % C, r = e / C;
    int off = (DIM == 2) ? o0 + n * r : o0 + n * (r % C + n * (r / C));
    X[e] = x[base + off];
  }
  psync<NT>();
  T* U1 = CS.u[0];
  T* U2 = CS.u[1];
  T* R = CS.r;
  if (DIM == 2) {
    // u1[yi][x] = sum_y Mr[yi][y] X[y][x]; u2 with Kr
    for (int e = lane; e < M * C; e += NT) {
      int xx = e % C, yi = e / C;
      T a1 = T(0), a2 = T(0);
#pragma unroll
      for (int y = 0; y < C; ++y) {
        T xv = X[y * C + xx];
        a1 += F.Mr[yi][y] * xv;
        a2 += F.Kr[yi][y] * xv;
      }
      U1[e] = a1;
      U2[e] = a2;
    }
    psync<NT>();
    // r = b - (Kx u1 + Mx u2)
    for (int e = lane; e < NI; e += NT) {
      int xi = e % M, yi = e / M;
      T acc = T(0);
#pragma unroll
      for (int xx = 0; xx < C; ++xx) acc += F.Kr[xi][xx] * U1[yi * C + xx] + F.Mr[xi][xx] * U2[yi * C + xx];
      int node = base + (xi + 1) + n * (yi + 1);
      R[e] = b[node] - acc;
    }
  } else {
    T* V1 = CS.v[0];
    T* V2 = CS.v[1];
    T* V3 = CS.v[2];
    // along z: u1 = Mz X, u2 = Kz X   (zi, y, x)
    for (int e = lane; e < M * C * C; e += NT) {
      int yx = e % (C * C), zi = e / (C * C);
      T a1 = T(0), a2 = T(0);
#pragma unroll
      for (int z = 0; z < C; ++z) {
        T xv = X[z * C * C + yx];
        a1 += F.Mr[zi][z] * xv;
        a2 += F.Kr[zi][z] * xv;
      }
      U1[e] = a1;
      U2[e] = a2;
    }
    psync<NT>();
    // along y: v1 = My u1, v2 = Ky u1, v3 = My u2   (zi, yi, x)
    for (int e = lane; e < M * M * C; e += NT) {
      int xx = e % C, r = e / C, yi = r % M, zi = r / M;
      T a1 = T(0), a2 = T(0), a3 = T(0);
#pragma unroll
      for (int y = 0; y < C; ++y) {
        T u1 = U1[(zi * C + y) * C + xx], u2 = U2[(zi * C + y) * C + xx];
        a1 += F.Mr[yi][y] * u1;
        a2 += F.Kr[yi][y] * u1;
        a3 += F.Mr[yi][y] * u2;
      }
      V1[e] = a1;
      V2[e] = a2;
      V3[e] = a3;
    }
    psync<NT>();
    // along x: r = b - (Kx v1 + Mx (v2 + v3))
    for (int e = lane; e < NI; e += NT) {
      int xi = e % M, r = e / M, yi = r % M, zi = r / M;
      T acc = T(0);
#pragma unroll
      for (int xx = 0; xx < C; ++xx) {
        int o = (zi * M + yi) * C + xx;
        acc += F.Kr[xi][xx] * V1[o] + F.Mr[xi][xx] * (V2[o] + V3[o]);
      }
      int node = base + (xi + 1) + n * ((yi + 1) + n * (zi + 1));
      R[e] = b[node] - acc;
    }
  }
  psync<NT>();
  // fast diagonalisation: t = (S^T)^{(x) DIM} r, scale, delta = S^{(x) DIM} t
  T* Tt = CS.t;
  // S^T along x
  for (int e = lane; e < NI; e += NT) {
    int a = e % M, rest = e / M;
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < M; ++i) acc += F.S[i][a] * R[rest * M + i];
    Tt[e] = acc;
  }
  psync<NT>();
  // S^T along y
  for (int e = lane; e < NI; e += NT) {
    int xx = e % M, r = e / M, bb = r % M, zi = r / M;
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < M; ++i) acc += F.S[i][bb] * Tt[(zi * M + i) * M + xx];
    R[e] = acc;
  }
  psync<NT>();
  if (DIM == 3) {
    // S^T along z, then scale
    for (int e = lane; e < NI; e += NT) {
      int yx = e % (M * M), cz = e / (M * M);
      T acc = T(0);
#pragma unroll
      for (int i = 0; i < M; ++i) acc += F.S[i][cz] * R[i * M * M + yx];
      int a = e % M, bb = (e / M) % M;
      Tt[e] = acc * F.dinv[e];
    }
    psync<NT>();
    // S along z
    for (int e = lane; e < NI; e += NT) {
      int yx = e % (M * M), zi = e / (M * M);
      T acc = T(0);
#pragma unroll
      for (int c = 0; c < M; ++c) acc += F.S[zi][c] * Tt[c * M * M + yx];
      R[e] = acc;
    }
  } else {
    for (int e = lane; e < NI; e += NT) {
      int a = e % M, bb = e / M;
      R[e] = R[e] * F.dinv[e];
    }
  }
  psync<NT>();
  // S along y
  for (int e = lane; e < NI; e += NT) {
    int xx = e % M, r = e / M, yi = r % M, zi = r / M;
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < M; ++c) acc += F.S[yi][c] * R[(zi * M + c) * M + xx];
    Tt[e] = acc;
  }
  psync<NT>();
  // S along x, update x
  for (int e = lane; e < NI; e += NT) {
    int xi = e % M, rest = e / M;
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < M; ++c) acc += F.S[xi][c] * Tt[rest * M + c];
    int yi = rest % M, zi = rest / M;
    int node = (DIM == 2) ? base + (xi + 1) + n * (yi + 1)
                          : base + (xi + 1) + n * ((yi + 1) + n * (zi + 1));
    if (live) x[node] += acc;
  }
}

// the 1D tables of the interior step copied from the kernel parameters into
// shared memory (all threads; a barrier follows): the lanes of a warp index
// them with different rows, which the parameter space serves one address at
// a time
template <typename T, int P>
__device__ __forceinline__ void stage_fd(const FdArgs<T, P>& F, FdArgs<T, P>& sF) {
  constexpr int NV = (int)(sizeof(FdArgs<T, P>) / sizeof(T));
  static_assert(sizeof(FdArgs<T, P>) % sizeof(T) == 0, "FdArgs holds T only");
  for (int i = threadIdx.x; i < NV; i += blockDim.x) reinterpret_cast<T*>(&sF)[i] = reinterpret_cast<const T*>(&F)[i];
}

// Two patches per warp, one per half-warp: the element loops of a patch
// (75, 45 and 27 entries for 3D Q2) fill 16 lanes better than 32, which the
// FP64 pipe, busy with every issued warp instruction, rewards; each entry
// is formed by one thread with the same operations as with a warp per patch.
template <int DIM, int P, typename T, int WARPS>
__global__ void __launch_bounds__(32 * WARPS) k_smooth_cart(FdArgs<T, P> F, int N, int n,
                                                            T* __restrict__ x, const T* __restrict__ b,
                                                            const int* __restrict__ verts, int nv) {
  __shared__ CartScratch<DIM, P, T> sCS[2 * WARPS];
  __shared__ FdArgs<T, P> sF;
  stage_fd<T, P>(F, sF);
  __syncthreads();
  const int w = threadIdx.x >> 5, half = (threadIdx.x >> 4) & 1, hl = threadIdx.x & 15;
  const int p0 = 2 * (blockIdx.x * WARPS + w);
  if (p0 >= nv) return;  // whole warp
  const bool live = p0 + half < nv;  // the idle half repeats the first patch without writing
  cart_body<DIM, P, T, 16>(sF, N, n, x, b, verts[live ? p0 + half : p0], hl, sCS[2 * w + half], live);
}

// FP32 interior-patch step as one dense map per level (the mixed form):
// every interior patch of a level has the same local matrices, so its exact
// local solve is x_I <- W [b_I ; x_B] with the fixed (2p-1)^d x (2p+1)^d
// matrix W = [A_I^{-1} | -A_I^{-1} A_{I,B}] over the closure (interior
// columns read b, boundary columns read x): a dense contraction of W with
// the gathered closures of all patches of a colour.  W is stored transposed
// with rows padded to a multiple of 4 (Wt[kc][r]).  Patches of one colour
// write interior nodes that no other patch of the colour reads.
template <int DIM, int P>
struct DenseGeo {
  static constexpr int C = 2 * P + 1, M = 2 * P - 1;
  static constexpr int NI = (DIM == 2) ? M * M : M * M * M;
  static constexpr int NC = (DIM == 2) ? C * C : C * C * C;
  static constexpr int NPART = (NI + 7) / 8;  // 8-row parts of W (split form)
  static constexpr int NR4 = NPART * 8;        // padded row count of Wt
  static constexpr int ROWS = NC / C;          // closure lines along x
};

template <int DIM, int P>
__device__ __forceinline__ int dense_base(int vert, int N, int n) {
  int base = 0, s = 1, q = vert;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    base += P * (q % (N + 1) - 1) * s;
    q /= N + 1;
    s *= n;
  }
  return base;
}

template <int DIM, int P>
__device__ __forceinline__ int dense_interior_offset(int r, int n) {
  constexpr int M = 2 * P - 1;
  const int ix = r % M + 1, iy = (r / M) % M + 1, iz = (DIM == 3) ? r / (M * M) + 1 : 0;
  return (DIM == 2) ? ix + n * iy : ix + n * (iy + n * iz);
}

// closure line `row` (the (cy, cz) pair): its lattice offset and whether
// its nodes with 1 <= cx <= C-2 are interior
template <int DIM, int P>
__device__ __forceinline__ int dense_row(int row, int n, bool& inner) {
  constexpr int C = 2 * P + 1;
  const int cy = row % C, cz = (DIM == 3) ? row / C : 0;
  inner = cy >= 1 && cy <= C - 2 && (DIM == 2 || (cz >= 1 && cz <= C - 2));
  return (DIM == 2) ? n * cy : n * (cy + n * cz);
}

// acc[r] += W[r][kc] g, rows in order, 4 rows of Wt per (broadcast) load
template <int NI, int NR4>
__device__ __forceinline__ void dense_fma(const float* __restrict__ wt, float g, float* acc) {
#pragma unroll
  for (int r4 = 0; r4 < NR4; r4 += 4) {
    const float4 w = *reinterpret_cast<const float4*>(wt + r4);
    if (r4 + 0 < NI) acc[r4 + 0] = fmaf(w.x, g, acc[r4 + 0]);
    if (r4 + 1 < NI) acc[r4 + 1] = fmaf(w.y, g, acc[r4 + 1]);
    if (r4 + 2 < NI) acc[r4 + 2] = fmaf(w.z, g, acc[r4 + 2]);
    if (r4 + 3 < NI) acc[r4 + 3] = fmaf(w.w, g, acc[r4 + 3]);
  }
}

// 128 threads and 128 * PPT patches per block: thread t takes patches t,
// t + 128, ..; Wt staged in shared memory once per block.  PPT = 2 reuses each
// W load for two patches (colours with enough patches to fill the GPU),
// PPT = 1 puts twice the threads on smaller colours.
template <int DIM, int P, int PPT>
__global__ void __launch_bounds__(128, PPT == 2 ? 6 : 8) k_smooth_dense(const float* __restrict__ Wt, int N,
                                                                        int n, float* __restrict__ x,
                                                                        const float* __restrict__ b,
                                                                        const int* __restrict__ verts, int nv) {
  using G = DenseGeo<DIM, P>;
  constexpr int C = G::C, NI = G::NI, NR4 = G::NR4;
  __shared__ __align__(16) float Ws[G::NC * NR4];
  for (int i = threadIdx.x; i < G::NC * NR4; i += blockDim.x) Ws[i] = Wt[i];
  __syncthreads();
  const int p0 = blockIdx.x * (128 * PPT) + threadIdx.x;
  if (p0 >= nv) return;
  int base[PPT];
  bool has[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    has[q] = p0 + 128 * q < nv;
    base[q] = has[q] ? dense_base<DIM, P>(verts[p0 + 128 * q], N, n) : base[0];
  }
  float acc[PPT][NI];
#pragma unroll
  for (int q = 0; q < PPT; ++q)
#pragma unroll
    for (int r = 0; r < NI; ++r) acc[q][r] = 0.f;
  for (int row = 0; row < G::ROWS; ++row) {
    bool inner;
    const int ro = dense_row<DIM, P>(row, n, inner);
#pragma unroll
    for (int cx = 0; cx < C; ++cx) {
      const float* src = (inner && cx >= 1 && cx <= C - 2) ? b : x;
      float g[PPT];
#pragma unroll
      for (int q = 0; q < PPT; ++q) g[q] = src[base[q] + ro + cx];
      const float* wt = Ws + (row * C + cx) * NR4;
#pragma unroll
      for (int q = 0; q < PPT; ++q) dense_fma<NI, NR4>(wt, g[q], acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    if (!has[q]) continue;
#pragma unroll
    for (int r = 0; r < NI; ++r) x[base[q] + dense_interior_offset<DIM, P>(r, n)] = acc[q][r];
  }
}

// Split form for colours too small to fill the GPU with one thread per patch:
// the closures of the block's 128 / NPART patches are first gathered into
// shared memory with every load in flight at once, then NPART threads per
// patch each form 8 rows of W [b_I ; x_B] (the same products in the same
// order as above, so the launch shape never changes a result).
template <int DIM, int P>
__global__ void __launch_bounds__(128) k_smooth_dense_split(const float* __restrict__ Wt, int N, int n,
                                                           float* __restrict__ x, const float* __restrict__ b,
                                                           const int* __restrict__ verts, int nv) {
  using G = DenseGeo<DIM, P>;
  constexpr int C = G::C, NC = G::NC, NI = G::NI, NR = G::NR4, NPART = G::NPART, PPB = 128 / NPART;
  __shared__ __align__(16) float Ws[NC * NR];
  __shared__ float Gs[PPB][NC + 1];
  __shared__ int Bs[PPB];
  for (int i = threadIdx.x; i < NC * NR; i += blockDim.x) Ws[i] = Wt[i];
  const int p0 = blockIdx.x * PPB;
  const int np = min(PPB, nv - p0);
  if (threadIdx.x < np) Bs[threadIdx.x] = dense_base<DIM, P>(verts[p0 + threadIdx.x], N, n);
  __syncthreads();
  for (int i = threadIdx.x; i < np * NC; i += blockDim.x) {
    const int q = i / NC, kc = i - q * NC;
    const int row = kc / C, cx = kc - row * C;
    bool inner;
    const int ro = dense_row<DIM, P>(row, n, inner);
    const float* src = (inner && cx >= 1 && cx <= C - 2) ? b : x;
    Gs[q][kc] = src[Bs[q] + ro + cx];
  }
  __syncthreads();
  const int part = threadIdx.x % NPART, slot = threadIdx.x / NPART;
  if (slot >= np) return;
  float acc[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) acc[r] = 0.f;
  for (int kc = 0; kc < NC; ++kc) {
    const float g = Gs[slot][kc];
    const float* wt = Ws + kc * NR + part * 8;
    const float4 w0 = *reinterpret_cast<const float4*>(wt);
    const float4 w1 = *reinterpret_cast<const float4*>(wt + 4);
    acc[0] = fmaf(w0.x, g, acc[0]);
    acc[1] = fmaf(w0.y, g, acc[1]);
    acc[2] = fmaf(w0.z, g, acc[2]);
    acc[3] = fmaf(w0.w, g, acc[3]);
    acc[4] = fmaf(w1.x, g, acc[4]);
    acc[5] = fmaf(w1.y, g, acc[5]);
    acc[6] = fmaf(w1.z, g, acc[6]);
    acc[7] = fmaf(w1.w, g, acc[7]);
  }
  const int base = Bs[slot];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int rr = part * 8 + r;
    if (rr < NI) x[base + dense_interior_offset<DIM, P>(rr, n)] = acc[r];
  }
}

// One 128-thread block per interior patch: for launches with few patches per
// SM, where one warp's chain of dependent FP64 steps sets the launch time.
template <int DIM, int P, typename T>
__global__ void __launch_bounds__(128) k_smooth_cart_cta(FdArgs<T, P> F, int N, int n, T* __restrict__ x,
                                                          const T* __restrict__ b,
                                                          const int* __restrict__ verts, int nv) {
  __shared__ CartScratch<DIM, P, T> CS;
  __shared__ FdArgs<T, P> sF;
  stage_fd<T, P>(F, sF);
  __syncthreads();
  for (int pidx = blockIdx.x; pidx < nv; pidx += gridDim.x) {
    cart_body<DIM, P, T, 128>(sF, N, n, x, b, verts[pidx], threadIdx.x, CS);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Cut-patch colour step (Sec. 3: dense local solver on cut patches), one warp
// per patch: r_I = b_I - (A x)_I by patch_rows, delta = A_j^{-1} r_I with the
// explicit inverse (symmetric, read by columns so that lanes load consecutive
// entries), x_I += delta.
//
// Additive within a colour (the paper's inconsistent treatment of the ghost
// coupling between patches, Sec. 2.3) without a second pass: the DoF sets of
// one colour's patches are disjoint, a DoF of patch A has all its active
// cells in A, so no cell row of another patch of the colour reads it, and the
// ghost-face terms read moments computed before the colour step.  Every patch
// therefore sees the x from before the colour step and writes its own DoFs.
template <int DIM, int P, typename T>
__device__ __forceinline__ void cut_body(const OpArgs<T>& A, T* __restrict__ x,
                                         const T* __restrict__ b, int vert, int m, int mo, int64_t io,
                                         const uint16_t* __restrict__ members,
                                         const int* __restrict__ mnode, const int* __restrict__ fofs,
                                         const int* __restrict__ fent, const T* __restrict__ inv,
                                         PatchScratch<DIM, P, T>& S, const T* __restrict__ sK, int lane) {
  const int np = A.N + 1;
  int q = vert, v[3] = {0, 0, 0};
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    v[k] = q % np;
    q /= np;
  }
  patch_rows<DIM, P, T>(A, x, v, members + mo, m, fofs + mo, fent, S, sK, lane);
  for (int e = lane; e < m; e += 32) S.r[e] = b[mnode[mo + e]] - S.r[e];
  __syncwarp();
  // delta = A_j^{-1} r with eight independent loads in flight per lane
  const T* Ai = inv + io;
  for (int e = lane; e < m; e += 32) {
    T acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = T(0);
    int j = 0;
    for (; j + 8 <= m; j += 8) {
      T a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = __ldg(Ai + (size_t)(j + u) * m + e);
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] += a[u] * S.r[j + u];
    }
    for (; j < m; ++j) acc[0] += __ldg(Ai + (size_t)j * m + e) * S.r[j];
    x[mnode[mo + e]] += ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  }
}

template <int DIM, int P, typename T, int WARPS>
__global__ void __launch_bounds__(32 * WARPS) k_cut_solve(OpArgs<T> A, T* __restrict__ x,
                                                          const T* __restrict__ b,
                                                          const int* __restrict__ verts,
                                                          const int* __restrict__ cnt,
                                                          const int* __restrict__ moff,
                                                          const int64_t* __restrict__ ioff,
                                                          const uint16_t* __restrict__ members,
                                                          const int* __restrict__ mnode,
                                                          const int* __restrict__ fofs,
                                                          const int* __restrict__ fent,
                                                          const T* __restrict__ inv, int npatch) {
  constexpr int NB = Shape<DIM, P>::NB;
  __shared__ T sK[NB * NB];
  __shared__ PatchScratch<DIM, P, T> sS[WARPS];
  stage_kref<NB>(A.Kref, sK);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pidx = blockIdx.x * WARPS + w;
  if (pidx >= npatch) return;
  cut_body<DIM, P, T>(A, x, b, verts[pidx], cnt[pidx], moff[pidx], ioff[pidx], members, mnode, fofs, fent,
                      inv, sS[w], sK, lane);
}

// ---------------------------------------------------------------------------
// Asynchronous copies into shared memory: TMA bulk copies (cp.async.bulk)
// completing on an mbarrier, and per-element cp.async.  Every wait on an
// mbarrier is bounded: past `limit` polls the caller records an error and
// drains its own copy (at most kTmaSpin polls) before it moves on, so that no
// copy is left in flight into shared memory.
constexpr int kTmaSpin = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// true once phase `parity` of the barrier has completed (at most `limit` polls)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit) {
  for (int it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Asynchronous copy of one element global -> shared (cp.async, 4 or 8 bytes).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(sizeof(T))
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------
// The same FP32 interior-patch step on the 5th-generation tensor cores: for a
// tile of 128 patches of one colour, D[128 x NP] = G[128 x KP] W^T[KP x NP]
// with G the gathered closures (rows = patches, K = closure nodes) and W the
// level's dense map (rows = interior nodes), one tcgen05.mma kind::tf32 per 8
// closure nodes (TF32 products, FP32 accumulation in tensor memory).  Both
// operands sit in shared memory in the canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices, each 128 contiguous bytes, ordered
// by 4-column K block, then by 8-row group.  One thread issues the MMAs and
// commits them to an mbarrier; the block's warps then read D back with
// tcgen05.ld (warp w: lanes 32 (w mod 4) .., half w / 4 of the columns) and
// write the new interior values.  256 threads per block: thread t gathers
// patch t mod 128, half t / 128 of its closure, with all its loads in flight
// at once; two blocks per SM overlap one block's gather with the other's
// MMA and write-back.  Persistent over the tiles of the colour.
template <int DIM, int P>
struct TcGeo {
  static constexpr int NI = DenseGeo<DIM, P>::NI, NC = DenseGeo<DIM, P>::NC;
  static constexpr int KP = (NC + 7) / 8 * 8;                       // K padded to the MMA's step
  static constexpr int NP = NI <= 16 ? 16 : (NI + 15) / 16 * 16;    // N padded (M = 128: N % 16 == 0)
  static constexpr int KH = KP / 2, NH = NP / 2;                    // per-thread halves
  static constexpr int COLS = NP <= 32 ? 32 : (NP <= 64 ? 64 : 128);  // tensor-memory columns
  static constexpr int A_BYTES = 128 * KP * 4, B_BYTES = NP * KP * 4;
  // The MMAs read [start, start + 2 (R / 8) 128) of an R-row operand per
  // K step.  The allocation also covers the reach the same descriptors would
  // have with the two byte offsets exchanged ((R / 8 - 1) (R / 8) 128 + 256
  // past the last step's start), so that no descriptor can address shared
  // memory outside the block.
  static constexpr int reach(int R, int start) { return start + (R / 8 - 1) * (R / 8) * 128 + 256; }
  static constexpr int cmax(int a, int b) { return a > b ? a : b; }
  static constexpr int SMEM =
      (cmax(cmax(A_BYTES + B_BYTES, reach(128, (KP / 8 - 1) * 2 * 16 * 128)),
            A_BYTES + reach(NP, (KP / 8 - 1) * 2 * (NP / 8) * 128)) + 127) / 128 * 128;
  static_assert(KH % 4 == 0, "each gathering thread stores whole 16-byte core-matrix rows");
};

// byte offset of element (row r, column k) of an R-row operand in the
// K-major, unswizzled core-matrix layout
template <int R>
__host__ __device__ constexpr int umma_off(int r, int k) {
  return ((k >> 2) * (R >> 3) + (r >> 3)) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

// shared-memory matrix descriptor: start address, leading-dimension byte
// offset (between K-adjacent core matrices), stride-dimension byte offset
// (between 8-row groups), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major,
// M = 128, N = np
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int np) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(np >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// columns of tensor memory for this block (one warp, converged); the
// address is written to *slot
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

// 32 lanes x NH consecutive 32-bit columns of tensor memory, one lane per thread
template <int NH>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float* v);
template <>
__device__ __forceinline__ void tmem_ld<8>(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t taddr, float* v) {
  tmem_ld<16>(taddr, v);
  tmem_ld<16>(taddr + 16u, v + 16);
}

__device__ __forceinline__ float to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

// closure values [H KH, H KH + KH) of the patch at lattice offset `base`
// (interior nodes read b, boundary nodes x), rounded to TF32, stored as
// row `p` of the A operand
template <int DIM, int P, int H>
__device__ __forceinline__ void tc_gather(const float* __restrict__ x, const float* __restrict__ b, int base, int n,
                                          bool has, int p, unsigned char* sA) {
  using G = TcGeo<DIM, P>;
  constexpr int C = 2 * P + 1;
  float g[G::KH];
#pragma unroll
  for (int q = 0; q < G::KH; ++q) {
    const int kc = H * G::KH + q;
    g[q] = 0.f;
    if (kc < G::NC && has) {
      const int cx = kc % C, cy = (kc / C) % C, cz = (DIM == 3) ? kc / (C * C) : 0;
      const bool inner = cx >= 1 && cx <= C - 2 && cy >= 1 && cy <= C - 2 && (DIM == 2 || (cz >= 1 && cz <= C - 2));
      const int off = (DIM == 2) ? cx + n * cy : cx + n * (cy + n * cz);
      g[q] = (inner ? b : x)[base + off];
    }
  }
#pragma unroll
  for (int q = 0; q < G::KH; q += 4) {
    const float4 v = make_float4(to_tf32(g[q]), to_tf32(g[q + 1]), to_tf32(g[q + 2]), to_tf32(g[q + 3]));
    *reinterpret_cast<float4*>(sA + umma_off<128>(p, H * G::KH + q)) = v;
  }
}

// Shared state of a tensor-core block: the A tile and B operand in dynamic
// shared memory (TcGeo::SMEM bytes), the MMA mbarrier, the tensor-memory
// columns.  tc_begin: all threads; tc_end releases the columns.
struct TcBlock {
  unsigned char* sA;
  unsigned char* sB;
  uint64_t* bar;
  uint32_t tmem;
  uint32_t phase;
};

// B operand (NP x KP, TF32-rounded, core-matrix layout, zero padding) into
// shared memory; every thread calls it, a barrier must follow before an MMA
template <int DIM, int P>
__device__ __forceinline__ void tc_load_b(const float* __restrict__ Bop, unsigned char* sB) {
  using G = TcGeo<DIM, P>;
  for (int i = threadIdx.x; i < G::B_BYTES / 16; i += blockDim.x)
    reinterpret_cast<float4*>(sB)[i] = reinterpret_cast<const float4*>(Bop)[i];
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One tile of up to 128 patches (verts[0 .. cnt)) of one level: gather,
// MMAs, write-back.  The per-patch result does not depend on the tile's other
// rows.  A bounded wait on the MMAs' mbarrier (`spin` polls) records a
// timeout in *err.
template <int DIM, int P>
__device__ __forceinline__ void tc_tile(TcBlock& tb, int N, int n, float* __restrict__ x,
                                        const float* __restrict__ b, const int* __restrict__ verts, int cnt,
                                        int* err, int spin) {
  using G = TcGeo<DIM, P>;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int p = tid & 127, half = tid >> 7;
  constexpr uint32_t idesc = umma_idesc_tf32(G::NP);
  const bool has = p < cnt;
  const int base = has ? dense_base<DIM, P>(verts[p], N, n) : 0;
  if (half == 0)
    tc_gather<DIM, P, 0>(x, b, base, n, has, p, tb.sA);
  else
    tc_gather<DIM, P, 1>(x, b, base, n, has, p, tb.sA);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid == 0) {
    const uint32_t a0 = smem_u32(tb.sA), b0 = smem_u32(tb.sB);
    tc_fence_after();
#pragma unroll
    for (int i = 0; i < G::KP / 8; ++i)
      umma_tf32(tb.tmem, umma_desc(a0 + i * 2 * 16 * 128, 16 * 128, 128),
                umma_desc(b0 + i * 2 * (G::NP / 8) * 128, (G::NP / 8) * 128, 128), idesc, i > 0 ? 1u : 0u);
    umma_commit(tb.bar);
  }
  if (!mbar_wait(tb.bar, tb.phase & 1u, spin)) {
    atomicExch(err, 1);
    mbar_wait(tb.bar, tb.phase & 1u, kTmaSpin);
  }
  tb.phase += 1;
  tc_fence_after();
  float d[G::NH];
  tmem_ld<G::NH>(tb.tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(G::NH * half), d);
  if (has) {
#pragma unroll
    for (int r = 0; r < G::NH; ++r) {
      const int rr = G::NH * half + r;
      if (rr < G::NI) x[base + dense_interior_offset<DIM, P>(rr, n)] = d[r];
    }
  }
  tc_fence_before();
  __syncthreads();
}

template <int DIM, int P>
__device__ __forceinline__ void tc_begin(TcBlock& tb, unsigned char* tsm, uint64_t* bar, uint32_t* tmem_slot) {
  using G = TcGeo<DIM, P>;
  tb.sA = tsm;
  tb.sB = tsm + G::A_BYTES;
  tb.bar = bar;
  tb.phase = 0;
  if ((threadIdx.x >> 5) == 0) tmem_alloc(tmem_slot, G::COLS);
  if (threadIdx.x == 0) mbar_init(bar);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  tb.tmem = *tmem_slot;
}

template <int DIM, int P>
__device__ __forceinline__ void tc_end(const TcBlock& tb) {
  tc_fence_after();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tb.tmem, TcGeo<DIM, P>::COLS);
}

// Bop: the level's W as the B operand.  Persistent over the colour's tiles.
template <int DIM, int P>
__global__ void __launch_bounds__(256, 2) k_smooth_tc(const float* __restrict__ Bop, int N, int n,
                                                      float* __restrict__ x, const float* __restrict__ b,
                                                      const int* __restrict__ verts, int nv, int* err, int spin) {
  extern __shared__ __align__(128) unsigned char tsm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  TcBlock tb;
  tc_load_b<DIM, P>(Bop, tsm + TcGeo<DIM, P>::A_BYTES);
  tc_begin<DIM, P>(tb, tsm, &bar, &tmem_slot);
  const int ntiles = (nv + 127) / 128;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
    tc_tile<DIM, P>(tb, N, n, x, b, verts + tile * 128, min(128, nv - tile * 128), err, spin);
  tc_end<DIM, P>(tb);
}

// ---------------------------------------------------------------------------
// Transfer: one direction of a tensor-product sparse 1D matrix with W entries
// per output index, over a box region of the output.  MODE 0: out = sum;
// MODE 1: out = mask ? sum : 0; MODE 2: out += mask ? sum : 0.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_pass(const T* __restrict__ in, T* __restrict__ out,
                                              int in0, int in1, int out0, int out1, int axis,
                                              int lo0, int lo1, int lo2, int ext0, int ext1,
                                              int ext2, const int* __restrict__ col,
                                              const T* __restrict__ wt, int W,
                                              const uint8_t* __restrict__ mask) {
  // grid (ceil(ext0 / blockDim.x), ext1, ext2): one thread per output node
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (t0 >= ext0) return;
  const int i0 = lo0 + t0, i1 = lo1 + (int)blockIdx.y, i2 = lo2 + (int)blockIdx.z;
  const int io = (axis == 0) ? i0 : (axis == 1 ? i1 : i2);
  T acc = T(0);
  for (int e = 0; e < W; ++e) {
    const int c = col[io * W + e];
    const T wv = wt[io * W + e];
    const int j0 = axis == 0 ? c : i0, j1 = axis == 1 ? c : i1, j2 = axis == 2 ? c : i2;
    acc += wv * in[(int64_t)j0 + (int64_t)in0 * (j1 + (int64_t)in1 * j2)];
  }
  const int64_t o = (int64_t)i0 + (int64_t)out0 * (i1 + (int64_t)out1 * i2);
  if (MODE == 0) out[o] = acc;
  else if (MODE == 1) out[o] = mask[o] ? acc : T(0);
  else if (mask[o]) out[o] += acc;
}

// Coarsest level: x0[node_i] = sum_j Ainv[i][j] b0[node_j], one warp per row.
template <typename T>
__global__ void __launch_bounds__(256) k_coarse(const T* __restrict__ Ainv, const int* __restrict__ nodes,
                                                int n0, const T* __restrict__ b, T* __restrict__ x) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n0) return;
  T acc = T(0);
  for (int j = lane; j < n0; j += 32) acc += Ainv[(size_t)row * n0 + j] * b[nodes[j]];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) x[nodes[row]] = acc;
}

// ---------------------------------------------------------------------------
// Vector kernels over a box region (bbox of the active nodes).
struct Region {
  int n0, n1;             // lattice strides (nodes per direction)
  int lo0, lo1, lo2;      // region origin
  int e0, e1, e2;         // region extents
  // lattice index of the t-th node of the region (first coordinate fastest);
  // 32-bit divisions while the region has fewer than 2^32 nodes
  __device__ __forceinline__ int64_t at(int64_t t) const {
    int i0, i1, i2;
    if (t < (int64_t(1) << 32)) {
      const uint32_t u = (uint32_t)t, q = u / (uint32_t)e0, q2 = q / (uint32_t)e1;
      i0 = lo0 + (int)(u - q * (uint32_t)e0);
      i1 = lo1 + (int)(q - q2 * (uint32_t)e1);
      i2 = lo2 + (int)q2;
    } else {
      i0 = lo0 + (int)(t % e0);
      i1 = lo1 + (int)((t / e0) % e1);
      i2 = lo2 + (int)(t / ((int64_t)e0 * e1));
    }
    return (int64_t)i0 + (int64_t)n0 * (i1 + (int64_t)n1 * i2);
  }
  __host__ __device__ int64_t size() const { return (int64_t)e0 * e1 * e2; }
  // f(o) for every node o of the region: each warp of the grid takes whole
  // rows (fixed i1, i2), row r = (i1 - lo1) + e1 (i2 - lo2) going to warp
  // r mod (warps of the grid), its lanes the row's consecutive nodes
  template <class F>
  __device__ __forceinline__ void for_each_node(F&& f) const {
    for_each_node_of(blockIdx.x, gridDim.x, f);
  }
  // the same partition with this block taking the place of block blk of
  // nblk (the batched kernels reproduce the single-problem partition)
  template <class F>
  __device__ __forceinline__ void for_each_node_of(int blk, int nblk, F&& f) const {
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int rows = e1 * e2;
    for (int r = blk * wpb + (threadIdx.x >> 5); r < rows; r += nblk * wpb) {
      const int q = r / e1;
      const int64_t base = (int64_t)lo0 + (int64_t)n0 * (lo1 + (r - q * e1) + (int64_t)n1 * (lo2 + q));
#pragma unroll 4
      for (int i = lane; i < e0; i += 32) f(base + i);
    }
  }
};

// partial sums of a.b, one per block, fixed assignment (deterministic)
static __global__ void __launch_bounds__(256) k_dot_partial(Region R, const double* __restrict__ a,
                                                     const double* __restrict__ b,
                                                     double* __restrict__ part) {
  __shared__ double s[256];
  double acc = 0.0;
  R.for_each_node([&](int64_t o) { acc += a[o] * b[o]; });
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

static __global__ void __launch_bounds__(256) k_dot_final(const double* __restrict__ part, int np,
                                                   double* __restrict__ out) {
  __shared__ double s[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += 256) acc += part[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// CG scalars: sc[0] = rz, sc[1] = pq, sc[2] = rz_new
// x += alpha p, r -= alpha q with alpha = rz / pq
static __global__ void __launch_bounds__(256) k_cg_update_xr(Region R, const double* __restrict__ sc,
                                                      double* __restrict__ x, double* __restrict__ r,
                                                      const double* __restrict__ p,
                                                      const double* __restrict__ q) {
  const double alpha = sc[0] / sc[1];
  R.for_each_node([&](int64_t o) {
    x[o] += alpha * p[o];
    r[o] -= alpha * q[o];
  });
}

// p = z + beta p, beta = rz_new / rz; then rz = rz_new (single writer after the grid)
static __global__ void __launch_bounds__(256) k_cg_update_p(Region R, const double* __restrict__ sc,
                                                     double* __restrict__ p, const double* __restrict__ z) {
  const double beta = sc[2] / sc[0];
  R.for_each_node([&](int64_t o) { p[o] = z[o] + beta * p[o]; });
}

static __global__ void k_copy_scalar(double* __restrict__ sc, int dst, int src) { sc[dst] = sc[src]; }

template <typename TO, typename TI>
__global__ void __launch_bounds__(256) k_convert(Region R, const TI* __restrict__ in, TO* __restrict__ out) {
  R.for_each_node([&](int64_t o) { out[o] = (TO)in[o]; });
}

// compact (DoF order) <-> box
template <typename TO, typename TI>
__global__ void __launch_bounds__(256) k_scatter(const int64_t* __restrict__ dofs, int64_t nd,
                                                 const TI* __restrict__ in, TO* __restrict__ box) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nd;
       i += (int64_t)gridDim.x * blockDim.x)
    box[dofs[i]] = (TO)in[i];
}

template <typename TO, typename TI>
__global__ void __launch_bounds__(256) k_gather(const int64_t* __restrict__ dofs, int64_t nd,
                                                const TI* __restrict__ box, TO* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nd;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (TO)box[dofs[i]];
}

}  // namespace cutmg
