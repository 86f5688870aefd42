// Operator on uncut cells by sum factorisation (Sec. 3: the uncut cells'
// integrals by tensor-product quadrature, here in its exact Kronecker form).
//
// Around a "bulk" owner position every cell is plain (active, uncut, no
// ghost face), so the rows of the nodes it owns are rows of the lattice-wide
// operator  A = sum_k M x .. x K x .. x M  (K on the k-th factor), with M and
// K the assembled 1D physical mass and stiffness on the node lattice: banded,
// 2p+1 entries on vertex rows (index = 0 mod p) and p+1 inside a cell.  A
// block takes a tile of owner positions, stages x on the tile's nodes plus p
// nodes of halo per side, and applies A by one 1D pass per direction
// (3D: z gives M x and K x, y gives three products, x combines), writing the
// owned nodes of the tile's bulk positions.  Per node about 2 (2p+1) flops
// per pass instead of 2 (p+1)^d per cell row: for 3D Q2 ~70 instead of 182.
#pragma once

#include <type_traits>

#include "kernels.cuh"

namespace cutmg {

template <int DIM, int P>
struct SfGeo {
  static constexpr int TX = DIM == 3 ? 8 : 16, TY = DIM == 3 ? 4 : 8, TZ = DIM == 3 ? 4 : 1;  // positions
  static constexpr int NX = P * TX, NY = P * TY, NZ = DIM == 3 ? P * TZ : 1;  // owned nodes
  static constexpr int EX = NX + 2 * P, EY = NY + 2 * P, EZ = DIM == 3 ? NZ + 2 * P : 1;  // with halo
  static constexpr int NPOS = TX * TY * TZ;
  static constexpr int MASKW = (NPOS + 31) / 32;
  static constexpr int W = 2 * P + 1;  // taps of a row (column offsets -p .. p)
  // shared memory (elements): X, then the pass outputs
  static constexpr int XS = EX * EY * EZ;
  static constexpr int US = DIM == 3 ? 2 * EX * EY * NZ : 2 * EX * NY;
  static constexpr int VS = DIM == 3 ? 3 * EX * NY * NZ : 0;
  // V (3D) reuses X's space: X is read only by the first pass, V written by
  // the second
  static constexpr int XV = XS > VS ? XS : VS;
  static constexpr int ELEMS = XV + US;
};

// rows of the assembled 1D physical mass / stiffness by residue r = i mod p,
// column i - p + s at tap s (zero outside the row's support)
template <typename T>
struct SfArgs {
  T Mrow[4][9], Krow[4][9];  // p <= 4
};

// taps [s0, s1] of residue r: vertex rows span both cells, others one cell
template <int P, int R>
struct SfTaps {
  static constexpr int S0 = R == 0 ? 0 : P - R;
  static constexpr int S1 = R == 0 ? 2 * P : 2 * P - R;
};

// out[o] for the P outputs o = P q + r (r = 0..P-1) of one line: a1 = M in,
// a2 = K in, with in[o + s] the input at column offset s - p
template <int P, int R, typename T>
__device__ __forceinline__ void sf_pair(const SfArgs<T>& A, const T* __restrict__ in, int stride, T& a1, T& a2) {
  a1 = T(0);
  a2 = T(0);
#pragma unroll
  for (int s = SfTaps<P, R>::S0; s <= SfTaps<P, R>::S1; ++s) {
    const T v = in[s * stride];
    a1 += A.Mrow[R][s] * v;
    a2 += A.Krow[R][s] * v;
  }
}

template <int P, int R, typename T>
__device__ __forceinline__ T sf_one(const T (&w)[4][9], const T* __restrict__ in, int stride) {
  T a = T(0);
#pragma unroll
  for (int s = SfTaps<P, R>::S0; s <= SfTaps<P, R>::S1; ++s) a += w[R][s] * in[s * stride];
  return a;
}

// Apply helpers unrolled over the residues of a group of P outputs
template <int P, typename T, typename F>
__device__ __forceinline__ void sf_residues(F&& f) {
  if constexpr (P >= 1) f(std::integral_constant<int, 0>());
  if constexpr (P >= 2) f(std::integral_constant<int, 1>());
  if constexpr (P >= 3) f(std::integral_constant<int, 2>());
  if constexpr (P >= 4) f(std::integral_constant<int, 3>());
  static_assert(P <= 4, "residues of degrees up to 4");
}

// y = A x (b == nullptr) or y = b - A x at the owned nodes of the bulk
// positions of one tile.  tile_pos: the tile's first position (packed
// a_0 + (N+1)(a_1 + (N+1) a_2)); mask: its bulk positions, bit
// ax + TX (ay + TY az).  smem: SfGeo::ELEMS elements.  All threads of the
// block call it; it ends with a barrier.
template <int DIM, int P, typename T>
__device__ __forceinline__ void sf_tile(const SfArgs<T>& A, int N, int n, const T* __restrict__ x,
                                        const T* __restrict__ b, T* __restrict__ y, int tile_pos,
                                        const uint32_t* __restrict__ mask, T* smem) {
  using G = SfGeo<DIM, P>;
  T* X = smem;
  T* U = X + G::XV;
  T* V = smem;  // over X (3D): written after the z pass, which is X's only reader
  const int tid = threadIdx.x, NT = blockDim.x, np = N + 1;
  {
    int a0[3] = {0, 0, 0};
    {
      int q = tile_pos;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        a0[k] = q % np;
        q /= np;
      }
    }
    // x on the tile's nodes and halo (outside the lattice: 0, used only by
    // rows that are not written)
    const int o0 = P * a0[0] - P, o1 = P * a0[1] - P, o2 = DIM == 3 ? P * a0[2] - P : 0;
    for (int e = tid; e < G::XS; e += NT) {
      const int ix = e % G::EX, r = e / G::EX, iy = r % G::EY, iz = r / G::EY;
      const int gx = o0 + ix, gy = o1 + iy, gz = o2 + iz;
      const bool in = gx >= 0 && gx < n && gy >= 0 && gy < n && (DIM == 2 || (gz >= 0 && gz < n));
      X[e] = in ? x[(DIM == 2) ? gx + (int64_t)n * gy : gx + (int64_t)n * (gy + (int64_t)n * gz)] : T(0);
    }
    __syncthreads();
    if (DIM == 3) {
      // z: U0 = Mz X, U1 = Kz X  on (EX, EY, NZ)
      constexpr int PL = G::EX * G::EY;
      for (int w = tid; w < PL * (G::NZ / P); w += NT) {
        const int xy = w % PL, q = w / PL;
        sf_residues<P, T>([&](auto rc) {
          constexpr int R = decltype(rc)::value;
          const int zo = P * q + R;
          T a1, a2;
          sf_pair<P, R>(A, X + xy + (size_t)zo * PL, PL, a1, a2);
          U[xy + (size_t)zo * PL] = a1;
          U[G::EX * G::EY * G::NZ + xy + (size_t)zo * PL] = a2;
        });
      }
      __syncthreads();
      // y: V0 = My U0, V1 = Ky U0, V2 = My U1  on (EX, NY, NZ)
      constexpr int VL = G::EX * G::NY * G::NZ;
      for (int w = tid; w < G::EX * (G::NY / P) * G::NZ; w += NT) {
        const int ix = w % G::EX, r = w / G::EX, q = r % (G::NY / P), zo = r / (G::NY / P);
        sf_residues<P, T>([&](auto rc) {
          constexpr int R = decltype(rc)::value;
          const int yo = P * q + R;
          const T* u0 = U + ix + G::EX * ((size_t)yo + G::EY * zo);
          const T* u1 = u0 + G::EX * G::EY * G::NZ;
          T m0, k0;
          sf_pair<P, R>(A, u0, G::EX, m0, k0);
          const T m1 = sf_one<P, R>(A.Mrow, u1, G::EX);
          const size_t o = ix + G::EX * ((size_t)yo + G::NY * zo);
          V[o] = m0;
          V[VL + o] = k0;
          V[2 * VL + o] = m1;
        });
      }
      __syncthreads();
      // x: y = Kx V0 + Mx (V1 + V2), owned nodes of bulk positions
      for (int w = tid; w < (G::NX / P) * G::NY * G::NZ; w += NT) {
        const int q = w % (G::NX / P), r = w / (G::NX / P), yo = r % G::NY, zo = r / G::NY;
        const int pos = q + G::TX * (yo / P + G::TY * (zo / P));
        if (!((mask[pos / 32] >> (pos % 32)) & 1u)) continue;
        sf_residues<P, T>([&](auto rc) {
          constexpr int R = decltype(rc)::value;
          const int xo = P * q + R;
          const size_t o = xo + G::EX * ((size_t)yo + G::NY * zo);
          T acc = sf_one<P, R>(A.Krow, V + o, 1);
          T s2 = T(0);
#pragma unroll
          for (int s = SfTaps<P, R>::S0; s <= SfTaps<P, R>::S1; ++s) s2 += A.Mrow[R][s] * (V[VL + o + s] + V[2 * VL + o + s]);
          acc += s2;
          const int64_t node = (P * a0[0] + xo) + (int64_t)n * ((P * a0[1] + yo) + (int64_t)n * (P * a0[2] + zo));
          y[node] = b ? b[node] - acc : acc;
        });
      }
    } else {
      // y: U0 = My X, U1 = Ky X  on (EX, NY)
      for (int w = tid; w < G::EX * (G::NY / P); w += NT) {
        const int ix = w % G::EX, q = w / G::EX;
        sf_residues<P, T>([&](auto rc) {
          constexpr int R = decltype(rc)::value;
          const int yo = P * q + R;
          T a1, a2;
          sf_pair<P, R>(A, X + ix + (size_t)G::EX * yo, G::EX, a1, a2);
          U[ix + G::EX * yo] = a1;
          U[G::EX * G::NY + ix + G::EX * yo] = a2;
        });
      }
      __syncthreads();
      // x: y = Kx U0 + Mx U1
      for (int w = tid; w < (G::NX / P) * G::NY; w += NT) {
        const int q = w % (G::NX / P), yo = w / (G::NX / P);
        const int pos = q + G::TX * (yo / P);
        if (!((mask[pos / 32] >> (pos % 32)) & 1u)) continue;
        sf_residues<P, T>([&](auto rc) {
          constexpr int R = decltype(rc)::value;
          const int xo = P * q + R;
          const size_t o = xo + G::EX * (size_t)yo;
          const T acc = sf_one<P, R>(A.Krow, U + o, 1) + sf_one<P, R>(A.Mrow, U + G::EX * G::NY + o, 1);
          const int64_t node = (P * a0[0] + xo) + (int64_t)n * (P * a0[1] + yo);
          y[node] = b ? b[node] - acc : acc;
        });
      }
    }
    __syncthreads();
  }
}

// The tiles of one level, block-stride over the tile list
template <int DIM, int P, typename T>
__global__ void __launch_bounds__(256) k_apply_sf(SfArgs<T> A, int N, int n, const T* __restrict__ x,
                                                  const T* __restrict__ b, T* __restrict__ y,
                                                  const int* __restrict__ tiles, const uint32_t* __restrict__ masks,
                                                  int ntiles) {
  extern __shared__ __align__(16) unsigned char sfm[];
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x)
    sf_tile<DIM, P, T>(A, N, n, x, b, y, tiles[tile], masks + (size_t)tile * SfGeo<DIM, P>::MASKW,
                       reinterpret_cast<T*>(sfm));
}

}  // namespace cutmg
