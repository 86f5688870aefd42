// Host construction of the CutFEM multigrid hierarchy (FP64, OpenMP over
// cells and patches).  See setup.hpp for the data layout.
//
// Operator (Sec. 2.1, eqs. "cutfem_nitsche", "cutfem-ghost"):
//   uncut cells       standard Q_p stiffness, Kronecker form of 1D matrices
//   cut cells         volume + Nitsche terms by the cut-cell rules
//   ghost faces       sum_m gamma_m h^(2m-1)/(m!)^2 ([d_n^m u], [d_n^m v])_F
//                     (the face scaling of the ghost penalty the paper cites; the
//                     printed h^(2m+1) loses coercivity under refinement)
// Patches (Sec. 2.3, Sec. 3): one per vertex of an active cell (the patches
// cover Omega_l); DoFs whose support lies in the patch; interior patches
// (2^d uncut cells, no ghost face on any patch cell) use fast
// diagonalisation, all others an explicit FP64 inverse of A[I_j, I_j].
#include "setup.hpp"

#include <algorithm>
#include <array>
#include <functional>

#include <omp.h>

#include <cmath>
#include <cstring>
#include <stdexcept>
#include <string>

namespace cutmg {
namespace {

int ipow(int b, int e) {
  int r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// SPD matrix (row-major, n x n) -> its inverse, in three passes of
// contiguous row updates (axpy form, so the inner loops vectorise without
// reassociating any sum):
//   1. A = U^T U, U upper triangular, right-looking Cholesky in place; the
//      trailing rows take the updates of a block of BS factor rows at once;
//   2. W = U^{-1} by rows, row c from the forward solve U^T w_c = e_c, for a
//      block of BS rows per pass over U;
//   3. A^{-1} = W W^T, row i accumulated over k = i..n-1 as rank-one updates
//      with column k of W, then mirrored.
// Each pass applies four consecutive updates per sweep over a row where it
// can.  Every entry's sum runs in ascending index order, whatever the thread
// count; large matrices (the coarsest-level operator) are split over threads.
void spd_inverse(int n, double* A) {
  constexpr int BS = 16;
  const bool par = n > 256;
  for (int jb = 0; jb < n; jb += BS) {
    const int je = std::min(n, jb + BS);
    for (int j = jb; j < je; ++j) {
      double* Aj = A + (size_t)j * n;
      for (int jj = jb; jj < j; ++jj) {
        const double* Ujj = A + (size_t)jj * n;
        const double a = Ujj[j];
        for (int k = j; k < n; ++k) Aj[k] -= a * Ujj[k];
      }
      const double s = Aj[j];
      if (!(s > 0.0))
        throw std::runtime_error("matrix is not positive definite (pivot " + std::to_string(j) + " of " +
                                 std::to_string(n) + ": " + std::to_string(s) + ")");
      const double d = std::sqrt(s);
      Aj[j] = d;
      for (int k = j + 1; k < n; ++k) Aj[k] /= d;
    }
    // rows i and i + 1 together (one load of each factor entry for both);
    // entry k = i belongs to row i only
#pragma omp parallel for schedule(dynamic, 2) if (par)
    for (int i = je; i < n; i += 2) {
      double* __restrict__ Ai = A + (size_t)i * n;
      double* __restrict__ Bi = Ai + n;
      const bool two = i + 1 < n;
      int j = jb;
      // four factor rows per sweep, subtracted in row order
      for (; j + 4 <= je; j += 4) {
        const double* __restrict__ U0 = A + (size_t)j * n;
        const double* __restrict__ U1 = U0 + n;
        const double* __restrict__ U2 = U1 + n;
        const double* __restrict__ U3 = U2 + n;
        const double a0 = U0[i], a1 = U1[i], a2 = U2[i], a3 = U3[i];
        Ai[i] = (((Ai[i] - a0 * U0[i]) - a1 * U1[i]) - a2 * U2[i]) - a3 * U3[i];
        if (two) {
          const double b0 = U0[i + 1], b1 = U1[i + 1], b2 = U2[i + 1], b3 = U3[i + 1];
          for (int k = i + 1; k < n; ++k) {
            const double u0 = U0[k], u1 = U1[k], u2 = U2[k], u3 = U3[k];
            Ai[k] = (((Ai[k] - a0 * u0) - a1 * u1) - a2 * u2) - a3 * u3;
            Bi[k] = (((Bi[k] - b0 * u0) - b1 * u1) - b2 * u2) - b3 * u3;
          }
        } else {
          for (int k = i + 1; k < n; ++k) Ai[k] = (((Ai[k] - a0 * U0[k]) - a1 * U1[k]) - a2 * U2[k]) - a3 * U3[k];
        }
      }
      for (; j < je; ++j) {
        const double* Uj = A + (size_t)j * n;
        const double a = Uj[i];
        Ai[i] -= a * Uj[i];
        if (two) {
          const double bb = Uj[i + 1];
          for (int k = i + 1; k < n; ++k) {
            Ai[k] -= a * Uj[k];
            Bi[k] -= bb * Uj[k];
          }
        } else {
          for (int k = i + 1; k < n; ++k) Ai[k] -= a * Uj[k];
        }
      }
    }
  }
  // W = U^{-1}: row c solves U^T w = e_c (w[k] = 0 for k < c); t carries the
  // right-hand side minus the terms already known
  std::vector<double> W((size_t)n * n, 0.0);
  const int nblk = (n + BS - 1) / BS;
#pragma omp parallel for schedule(dynamic, 1) if (par)
  for (int bi = 0; bi < nblk; ++bi) {
    const int c0 = bi * BS, c1 = std::min(n, c0 + BS);
    for (int c = c0; c < c1; ++c) W[(size_t)c * n + c] = 1.0;
    int k = c0;
    for (; k < n && k < c1 - 1; ++k) {  // rows c > k of the block start later
      const double* Uk = A + (size_t)k * n;
      const double dk = Uk[k];
      for (int c = c0; c < c1 && c <= k; ++c) {
        double* Wc = &W[(size_t)c * n];
        const double wk = Wc[k] / dk;
        Wc[k] = wk;
        for (int q = k + 1; q < n; ++q) Wc[q] -= wk * Uk[q];
      }
    }
    // four steps k..k+3 per sweep once every row of the block has started:
    // the four multipliers first (entries k+1..k+3 take the earlier steps'
    // updates in order), then one fused pass over q >= k + 4
    for (; k + 4 <= n; k += 4) {
      const double* U0 = A + (size_t)k * n;
      const double* U1 = U0 + n;
      const double* U2 = U1 + n;
      const double* U3 = U2 + n;
      // the four multipliers of a row (entries k+1..k+3 take the earlier
      // steps' updates in order)
      auto mult = [&](double* Wc, double* w) {
        w[0] = Wc[k] / U0[k];
        Wc[k] = w[0];
        Wc[k + 1] -= w[0] * U0[k + 1];
        Wc[k + 2] -= w[0] * U0[k + 2];
        Wc[k + 3] -= w[0] * U0[k + 3];
        w[1] = Wc[k + 1] / U1[k + 1];
        Wc[k + 1] = w[1];
        Wc[k + 2] -= w[1] * U1[k + 2];
        Wc[k + 3] -= w[1] * U1[k + 3];
        w[2] = Wc[k + 2] / U2[k + 2];
        Wc[k + 2] = w[2];
        Wc[k + 3] -= w[2] * U2[k + 3];
        w[3] = Wc[k + 3] / U3[k + 3];
        Wc[k + 3] = w[3];
      };
      int c = c0;
      for (; c + 2 <= c1; c += 2) {  // two rows per pass over q
        double* __restrict__ Wc = &W[(size_t)c * n];
        double* __restrict__ Vc = Wc + n;
        double w[4], v[4];
        mult(Wc, w);
        mult(Vc, v);
        for (int q = k + 4; q < n; ++q) {
          const double u0 = U0[q], u1 = U1[q], u2 = U2[q], u3 = U3[q];
          Wc[q] = (((Wc[q] - w[0] * u0) - w[1] * u1) - w[2] * u2) - w[3] * u3;
          Vc[q] = (((Vc[q] - v[0] * u0) - v[1] * u1) - v[2] * u2) - v[3] * u3;
        }
      }
      for (; c < c1; ++c) {
        double* __restrict__ Wc = &W[(size_t)c * n];
        double w[4];
        mult(Wc, w);
        for (int q = k + 4; q < n; ++q) Wc[q] = (((Wc[q] - w[0] * U0[q]) - w[1] * U1[q]) - w[2] * U2[q]) - w[3] * U3[q];
      }
    }
    for (; k < n; ++k) {
      const double* Uk = A + (size_t)k * n;
      const double dk = Uk[k];
      for (int c = c0; c < c1 && c <= k; ++c) {
        double* Wc = &W[(size_t)c * n];
        const double wk = Wc[k] / dk;
        Wc[k] = wk;
        for (int q = k + 1; q < n; ++q) Wc[q] -= wk * Uk[q];
      }
    }
  }
  // Z = W^T (row k of Z = column k of W), then A^{-1}[i][0..i] = sum over
  // k >= i of W[i][k] Z[k][0..i]
  std::vector<double> Z((size_t)n * n, 0.0);
#pragma omp parallel for schedule(static) if (par)
  for (int k = 0; k < n; ++k)
    for (int i = 0; i <= k; ++i) Z[(size_t)k * n + i] = W[(size_t)i * n + k];
#pragma omp parallel for schedule(dynamic, 1) if (par)
  for (int bi = 0; bi < nblk; ++bi) {
    const int i0 = bi * BS, i1 = std::min(n, i0 + BS);
    for (int i = i0; i < i1; ++i)
      for (int j = 0; j <= i; ++j) A[(size_t)i * n + j] = 0.0;
    int k = i0;
    for (; k < n && k < i1 - 1; ++k) {
      const double* Zk = &Z[(size_t)k * n];
      for (int i = i0; i < i1 && i <= k; ++i) {
        const double a = Zk[i];
        double* Ai = A + (size_t)i * n;
        for (int j = 0; j <= i; ++j) Ai[j] += a * Zk[j];
      }
    }
    // every row of the block takes every k from here: four k per sweep
    for (; k + 4 <= n; k += 4) {
      const double* Z0 = &Z[(size_t)k * n];
      const double* Z1 = Z0 + n;
      const double* Z2 = Z1 + n;
      const double* Z3 = Z2 + n;
      int i = i0;
      for (; i + 2 <= i1; i += 2) {  // rows i, i + 1; entry j = i + 1 is row i + 1's only
        const double a0 = Z0[i], a1 = Z1[i], a2 = Z2[i], a3 = Z3[i];
        const double b0 = Z0[i + 1], b1 = Z1[i + 1], b2 = Z2[i + 1], b3 = Z3[i + 1];
        double* __restrict__ Ai = A + (size_t)i * n;
        double* __restrict__ Bi = Ai + n;
        for (int j = 0; j <= i; ++j) {
          const double z0 = Z0[j], z1 = Z1[j], z2 = Z2[j], z3 = Z3[j];
          Ai[j] = (((Ai[j] + a0 * z0) + a1 * z1) + a2 * z2) + a3 * z3;
          Bi[j] = (((Bi[j] + b0 * z0) + b1 * z1) + b2 * z2) + b3 * z3;
        }
        Bi[i + 1] = (((Bi[i + 1] + b0 * Z0[i + 1]) + b1 * Z1[i + 1]) + b2 * Z2[i + 1]) + b3 * Z3[i + 1];
      }
      for (; i < i1; ++i) {
        const double a0 = Z0[i], a1 = Z1[i], a2 = Z2[i], a3 = Z3[i];
        double* __restrict__ Ai = A + (size_t)i * n;
        for (int j = 0; j <= i; ++j) Ai[j] = (((Ai[j] + a0 * Z0[j]) + a1 * Z1[j]) + a2 * Z2[j]) + a3 * Z3[j];
      }
    }
    for (; k < n; ++k) {
      const double* Zk = &Z[(size_t)k * n];
      for (int i = i0; i < i1 && i <= k; ++i) {
        const double a = Zk[i];
        double* Ai = A + (size_t)i * n;
        for (int j = 0; j <= i; ++j) Ai[j] += a * Zk[j];
      }
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) A[(size_t)j * n + i] = A[(size_t)i * n + j];
}

// Symmetric eigen-decomposition by cyclic Jacobi rotations: A = Q diag(lam) Q^T.
void jacobi_eigen(int n, std::vector<double> A, std::vector<double>& Q, std::vector<double>& lam) {
  Q.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
    if (off < 1e-60) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        double theta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double qkp = Q[(size_t)k * n + p], qkq = Q[(size_t)k * n + q];
          Q[(size_t)k * n + p] = c * qkp - s * qkq;
          Q[(size_t)k * n + q] = s * qkp + c * qkq;
        }
      }
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = A[(size_t)i * n + i];
}

struct RefTables {
  int p, d, NB;
  Poly1D b;
  std::vector<double> M1, K1;  // (p+1)^2 reference mass / stiffness on [0, 1]
  std::vector<std::array<int, 3>> mi;  // multi-index of local basis function j
  explicit RefTables(int p_, int d_) : p(p_), d(d_), NB(ipow(p_ + 1, d_)), b(p_), mi(NB) {
    for (int j = 0; j < NB; ++j) {
      int a[3] = {0, 0, 0};
      split(j, a);
      mi[j] = {a[0], a[1], a[2]};
    }
    GaussRule g = gauss_legendre01(p + 1);
    M1.assign((p + 1) * (p + 1), 0.0);
    K1.assign((p + 1) * (p + 1), 0.0);
    for (int a = 0; a <= p; ++a)
      for (int c = 0; c <= p; ++c)
        for (int i = 0; i <= p; ++i) {
          double xi = g.x[i];
          M1[a * (p + 1) + c] += g.w[i] * b.eval(a, xi) * b.eval(c, xi);
          K1[a * (p + 1) + c] += g.w[i] * b.eval(a, xi, 1) * b.eval(c, xi, 1);
        }
  }
  // local index j -> multi-index, first coordinate fastest
  void split(int j, int* a) const {
    for (int k = 0; k < d; ++k) {
      a[k] = j % (p + 1);
      j /= p + 1;
    }
  }
  // tensor basis values at reference point xi
  void values(const double* xi, double* v) const {
    double l[3][5];
    for (int k = 0; k < d; ++k)
      for (int a = 0; a <= p; ++a) l[k][a] = b.eval(a, xi[k]);
    for (int j = 0; j < NB; ++j) {
      const int* a = mi[j].data();
      double val = 1.0;
      for (int k = 0; k < d; ++k) val *= l[k][a[k]];
      v[j] = val;
    }
  }
  // tensor basis values and physical gradients at reference point xi
  void eval(const double* xi, double h, double* v, double* g /* NB x d */) const {
    double l[3][5], dl[3][5];
    for (int k = 0; k < d; ++k)
      for (int a = 0; a <= p; ++a) {
        l[k][a] = b.eval(a, xi[k]);
        dl[k][a] = b.eval(a, xi[k], 1) / h;
      }
    for (int j = 0; j < NB; ++j) {
      const int* a = mi[j].data();
      double val = 1.0;
      for (int k = 0; k < d; ++k) val *= l[k][a[k]];
      v[j] = val;
      for (int k = 0; k < d; ++k) {
        double t = 1.0;
        for (int kk = 0; kk < d; ++kk) t *= (kk == k) ? dl[kk][a[kk]] : l[kk][a[kk]];
        g[j * d + k] = t;
      }
    }
  }
};

// a_T(phi_j, phi_i) of a cut cell: volume + Nitsche terms.  Every term is
// symmetric in (i, j), so each quadrature point adds rank-one updates to the
// upper triangle (contiguous inner loops over j), mirrored at the end.
void cut_cell_matrix(const RefTables& R, const CutRule& rule, const double* lo, double h,
                     double gamma_D, double* K) {
  const int NB = R.NB, d = R.d;
  std::vector<double> v(NB), g(NB * d), dn(NB);
  std::fill(K, K + NB * NB, 0.0);
  double xi[3];
  // volume: w grad(phi_i) . grad(phi_j), one update per (point, direction)
  // row r, in point order; a batch of QB points is applied to each entry
  // with the entry held in a register (four entries of a row at a time)
  constexpr int QB = 8;
  std::vector<double> Wg((size_t)QB * d * NB), Gg((size_t)QB * d * NB);  // w dphi_j/dx_k, dphi_j/dx_k
  const size_t nv = rule.vol.size();
  for (size_t q0 = 0; q0 < nv; q0 += QB) {
    const int nb = (int)std::min<size_t>(QB, nv - q0);
    for (int bq = 0; bq < nb; ++bq) {
      const auto& nd = rule.vol[q0 + bq];
      for (int k = 0; k < d; ++k) xi[k] = (nd.x[k] - lo[k]) / h;
      R.eval(xi, h, v.data(), g.data());
      for (int k = 0; k < d; ++k)
        for (int j = 0; j < NB; ++j) {
          const size_t r = (size_t)(bq * d + k) * NB + j;
          Gg[r] = g[j * d + k];
          Wg[r] = nd.w * g[j * d + k];
        }
    }
    const int nr = nb * d;
    for (int i = 0; i < NB; ++i) {
      double* Ki = K + (size_t)i * NB;
      int j = i;
      for (; j + 4 <= NB; j += 4) {
        double a0 = Ki[j], a1 = Ki[j + 1], a2 = Ki[j + 2], a3 = Ki[j + 3];
        for (int r = 0; r < nr; ++r) {
          const double a = Wg[(size_t)r * NB + i];
          const double* gr = &Gg[(size_t)r * NB + j];
          a0 += a * gr[0];
          a1 += a * gr[1];
          a2 += a * gr[2];
          a3 += a * gr[3];
        }
        Ki[j] = a0;
        Ki[j + 1] = a1;
        Ki[j + 2] = a2;
        Ki[j + 3] = a3;
      }
      for (; j < NB; ++j) {
        double a0 = Ki[j];
        for (int r = 0; r < nr; ++r) a0 += Wg[(size_t)r * NB + i] * Gg[(size_t)r * NB + j];
        Ki[j] = a0;
      }
    }
  }
  // Nitsche: w (-(dn_i v_j + v_i dn_j) + gamma_D / h v_i v_j)
  //        = w (gamma_D / h v_i - dn_i) v_j - w v_i dn_j
  const double pen = gamma_D / h;
  for (size_t q = 0; q < rule.surf.size(); ++q) {
    const auto& nd = rule.surf[q];
    for (int k = 0; k < d; ++k) xi[k] = (nd.x[k] - lo[k]) / h;
    R.eval(xi, h, v.data(), g.data());
    for (int i = 0; i < NB; ++i) {
      double s = 0.0;
      for (int k = 0; k < d; ++k) s += rule.normal[q][k] * g[i * d + k];
      dn[i] = s;
    }
    for (int i = 0; i < NB; ++i) {
      double* Ki = K + (size_t)i * NB;
      const double a = nd.w * (pen * v[i] - dn[i]), c = -nd.w * v[i];
      for (int j = i; j < NB; ++j) Ki[j] += a * v[j] + c * dn[j];
    }
  }
  for (int i = 1; i < NB; ++i)
    for (int j = 0; j < i; ++j) K[(size_t)i * NB + j] = K[(size_t)j * NB + i];
}

// right-hand side terms of one cut cell from its quadrature rule (volume:
// f phi_j; Nitsche data: g (gamma_D / h phi_j - dphi_j/dn)), accumulated into
// loc (zeroed here) point by point in rule order
void cut_cell_rhs(const RefTables& R, const CutRule& rule, const double* lo, double h, double gamma_D,
                  const std::function<double(const double*)>& fsrc,
                  const std::function<double(const double*)>& gdir, double* loc) {
  const int NB = R.NB, d = R.d;
  std::vector<double> v(NB), gr(NB * d);
  for (int j = 0; j < NB; ++j) loc[j] = 0.0;
  for (const auto& nd : rule.vol) {
    double xi[3] = {0, 0, 0};
    for (int k = 0; k < d; ++k) xi[k] = (nd.x[k] - lo[k]) / h;
    R.values(xi, v.data());
    double fx = fsrc(nd.x) * nd.w;
    for (int j = 0; j < NB; ++j) loc[j] += v[j] * fx;
  }
  for (size_t s2 = 0; s2 < rule.surf.size(); ++s2) {
    const auto& nd = rule.surf[s2];
    double xi[3] = {0, 0, 0};
    for (int k = 0; k < d; ++k) xi[k] = (nd.x[k] - lo[k]) / h;
    R.eval(xi, h, v.data(), gr.data());
    double gx = gdir(nd.x) * nd.w;
    for (int j = 0; j < NB; ++j) {
      double dn = 0.0;
      for (int k = 0; k < d; ++k) dn += rule.normal[s2][k] * gr[j * d + k];
      loc[j] += gx * (gamma_D / h * v[j] - dn);
    }
  }
}

// cells containing lattice coordinate i along one direction
int cells_of(int i, int p, int N, int* c, int* loc) {
  int a = i / p, r = i - a * p, m = 0;
  if (r == 0) {
    if (a - 1 >= 0) { c[m] = a - 1; loc[m] = p; ++m; }
    if (a < N) { c[m] = a; loc[m] = 0; ++m; }
  } else {
    c[m] = a; loc[m] = r; ++m;
  }
  return m;
}

// flag of cell c (cell coordinates) of a level; 0 outside the mesh
uint8_t cell_flag(const HostLevel& L, const int* c) {
  int64_t f = 0, st = 1;
  for (int k = 0; k < L.d; ++k) {
    if (c[k] < 0 || c[k] >= L.N) return 0;
    f += (int64_t)c[k] * st;
    st *= L.N;
  }
  return L.cflag[f];
}

// Runs f(i, out) for i in [0, n) over contiguous blocks of i shared out to
// the threads, and appends what the calls pushed to `out` in increasing i:
// the result is the serial loop's, whatever the thread count.
template <class T, class Alloc, class F>
void ordered_collect(int64_t n, std::vector<T, Alloc>& out, F&& f) {
  const int64_t nblk = std::max<int64_t>(1, std::min<int64_t>(n, 16 * std::max(1, omp_get_max_threads())));
  std::vector<std::vector<T>> part(nblk);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t b = 0; b < nblk; ++b)
    for (int64_t i = n * b / nblk; i < n * (b + 1) / nblk; ++i) f(i, part[b]);
  size_t tot = out.size();
  for (const auto& q : part) tot += q.size();
  out.reserve(tot);
  for (const auto& q : part) out.insert(out.end(), q.begin(), q.end());
}

// "plain" cell: active, uncut, no cut face-neighbour (no ghost face)
bool plain_cell(const HostLevel& L, const int* c) {
  uint8_t f = cell_flag(L, c);
  if (!(f & kFlagActive) || (f & kFlagCut)) return false;
  for (int k = 0; k < L.d; ++k)
    for (int s = -1; s <= 1; s += 2) {
      int cj[3] = {c[0], c[1], c[2]};
      cj[k] += s;
      if (cell_flag(L, cj) & kFlagCut) return false;
    }
  return true;
}

// plain_cell of every cell of the level (cell order)
std::vector<uint8_t> plain_flags(const HostLevel& L) {
  const int d = L.d, N = L.N;
  const int64_t ncell = ipow(N, d);
  std::vector<uint8_t> pl(ncell);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < ncell; ++c) {
    int ci[3] = {0, 0, 0};
    int64_t t = c;
    for (int k = 0; k < d; ++k) {
      ci[k] = (int)(t % N);
      t /= N;
    }
    pl[c] = plain_cell(L, ci) ? 1 : 0;
  }
  return pl;
}

// Interior patches (every cell of the patch plain): the two-cell 1D mass and
// stiffness rows, the fast-diagonalisation eigenpairs and the level's dense
// interior-patch map.
void interior_patch_tables(const RefTables& R, HostLevel& L) {
  const int d = L.d, p = L.p;
  const double h = L.h;
  const int C = 2 * p + 1, M = 2 * p - 1;
  std::vector<double> Mb(C * C, 0.0), Kb(C * C, 0.0);
  for (int s = 0; s < 2; ++s)
    for (int a = 0; a <= p; ++a)
      for (int b = 0; b <= p; ++b) {
        Mb[(s * p + a) * C + s * p + b] += R.M1[a * (p + 1) + b] * h;
        Kb[(s * p + a) * C + s * p + b] += R.K1[a * (p + 1) + b] / h;
      }
  L.Mr.assign(M * C, 0.0);
  L.Kr.assign(M * C, 0.0);
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < C; ++j) {
      L.Mr[i * C + j] = Mb[(i + 1) * C + j];
      L.Kr[i * C + j] = Kb[(i + 1) * C + j];
    }
  // K_I s = lam M_I s with S^T M_I S = I: M_I = G G^T, Jacobi on G^-1 K_I G^-T
  std::vector<double> MI(M * M), KI(M * M), G(M * M, 0.0), Gi(M * M, 0.0);
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) {
      MI[i * M + j] = L.Mr[i * C + j + 1];
      KI[i * M + j] = L.Kr[i * C + j + 1];
    }
  for (int j = 0; j < M; ++j) {
    double s = MI[j * M + j];
    for (int k = 0; k < j; ++k) s -= G[j * M + k] * G[j * M + k];
    G[j * M + j] = std::sqrt(s);
    for (int i = j + 1; i < M; ++i) {
      double t = MI[i * M + j];
      for (int k = 0; k < j; ++k) t -= G[i * M + k] * G[j * M + k];
      G[i * M + j] = t / G[j * M + j];
    }
  }
  for (int c = 0; c < M; ++c)
    for (int i = c; i < M; ++i) {
      double t = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) t -= G[i * M + k] * Gi[k * M + c];
      Gi[i * M + c] = t / G[i * M + i];
    }
  std::vector<double> Cm(M * M, 0.0), Qv, lam;
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) {
      double t = 0.0;
      for (int a = 0; a < M; ++a)
        for (int b = 0; b < M; ++b) t += Gi[i * M + a] * KI[a * M + b] * Gi[j * M + b];
      Cm[i * M + j] = t;
    }
  jacobi_eigen(M, Cm, Qv, lam);
  L.S.assign(M * M, 0.0);
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) {
      double t = 0.0;
      for (int a = 0; a < M; ++a) t += Gi[a * M + i] * Qv[a * M + j];  // G^-T Q
      L.S[i * M + j] = t;
    }
  L.lam = lam;
  // The exact local solve of an interior patch as one dense map per level:
  // x_I <- A_I^{-1} b_I - A_I^{-1} A_{I,B} x_B over the closure; columns in
  // closure order (first coordinate fastest), b at interior columns and x
  // at boundary columns; rows in interior order.
  {
    const int NI = ipow(M, d), NC = ipow(C, d);
    std::vector<double> AIcl((size_t)NI * NC, 0.0);
    for (int i = 0; i < NI; ++i) {
      int ii[3] = {0, 0, 0}, t = i;
      for (int k = 0; k < d; ++k) {
        ii[k] = t % M;
        t /= M;
      }
      for (int kc = 0; kc < NC; ++kc) {
        int cc[3] = {0, 0, 0}, u = kc;
        for (int k = 0; k < d; ++k) {
          cc[k] = u % C;
          u /= C;
        }
        double v = 0.0;
        for (int a = 0; a < d; ++a) {  // stiffness along a, mass along the others
          double f = 1.0;
          for (int k = 0; k < d; ++k) f *= (k == a ? L.Kr[ii[k] * C + cc[k]] : L.Mr[ii[k] * C + cc[k]]);
          v += f;
        }
        AIcl[(size_t)i * NC + kc] = v;
      }
    }
    auto closure_of = [&](int i) {
      int kc = 0, st = 1, t = i;
      for (int k = 0; k < d; ++k) {
        kc += (t % M + 1) * st;
        t /= M;
        st *= C;
      }
      return kc;
    };
    std::vector<double> AIi((size_t)NI * NI);
    for (int i = 0; i < NI; ++i)
      for (int j = 0; j < NI; ++j) AIi[(size_t)i * NI + j] = AIcl[(size_t)i * NC + closure_of(j)];
    spd_inverse(NI, AIi.data());
    std::vector<int> interior_index(NC, -1);
    for (int j = 0; j < NI; ++j) interior_index[closure_of(j)] = j;
    L.Wcart.assign((size_t)NI * NC, 0.0);
    for (int i = 0; i < NI; ++i)
      for (int kc = 0; kc < NC; ++kc) {
        double w;
        if (interior_index[kc] >= 0) {
          w = AIi[(size_t)i * NI + interior_index[kc]];
        } else {
          w = 0.0;
          for (int j = 0; j < NI; ++j) w -= AIi[(size_t)i * NI + j] * AIcl[(size_t)j * NC + kc];
        }
        L.Wcart[(size_t)i * NC + kc] = w;
      }
  }
}

// Patch vertices of a level by colour: Cartesian (every patch cell plain)
// and cut patches, each list in vertex order.
void patch_vertex_sets(HostLevel& L) {
  const int d = L.d, N = L.N, np = N + 1, ncol = 1 << d;
  auto cflag_at = [&](const int* c) { return cell_flag(L, c); };
  const int64_t nvert = (int64_t)ipow(np, d);
  std::vector<std::vector<int>> cart(ncol), cutv(ncol);
  // per vertex: -1 (no active cell around it), else colour + 8 if Cartesian
  std::vector<int8_t> vkind(nvert);
  const std::vector<uint8_t> pl = plain_flags(L);
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < nvert; ++q) {
    int v[3] = {0, 0, 0};
    int64_t t = q;
    for (int k = 0; k < d; ++k) {
      v[k] = (int)(t % np);
      t /= np;
    }
    bool any = false, cartesian = true;
    for (int s = 0; s < (1 << d); ++s) {
      int c[3] = {0, 0, 0};
      bool in = true;
      int64_t ci = 0, st = 1;
      for (int k = 0; k < d; ++k) {
        c[k] = v[k] - 1 + ((s >> k) & 1);
        in = in && c[k] >= 0 && c[k] < N;
        ci += (int64_t)c[k] * st;
        st *= N;
      }
      if (cflag_at(c) & kFlagActive) any = true;
      if (!in || !pl[ci]) cartesian = false;  // plain_cell is false outside the mesh
    }
    int col = 0;
    for (int k = 0; k < d; ++k) col |= (v[k] & 1) << k;
    vkind[q] = any ? (int8_t)(col + (cartesian ? 8 : 0)) : (int8_t)-1;
  }
  for (int col = 0; col < ncol; ++col) {
    ordered_collect(nvert, cart[col], [&](int64_t q, std::vector<int>& o) {
      if (vkind[q] == col + 8) o.push_back((int)q);
    });
    ordered_collect(nvert, cutv[col], [&](int64_t q, std::vector<int>& o) {
      if (vkind[q] == col) o.push_back((int)q);
    });
  }
  L.cart_start.assign(ncol + 1, 0);
  L.cut_start.assign(ncol + 1, 0);
  for (int c = 0; c < ncol; ++c) {
    L.cart_vert.insert(L.cart_vert.end(), cart[c].begin(), cart[c].end());
    L.cut_vert.insert(L.cut_vert.end(), cutv[c].begin(), cutv[c].end());
    L.cart_start[c + 1] = (int)L.cart_vert.size();
    L.cut_start[c + 1] = (int)L.cut_vert.size();
  }
}

// Cut patches: their DoFs (closure nodes all of whose active cells are patch
// cells), member and inverse offsets, and the inverse storage.
void cut_patch_members(HostLevel& L, bool dry) {
  const int d = L.d, p = L.p, N = L.N, n = L.n;
  const int np = N + 1, C = 2 * p + 1, ncol = 1 << d, NCL = ipow(C, d);
  const int64_t ncp = (int64_t)L.cut_vert.size();
  auto cflag_at = [&](const int* c) { return cell_flag(L, c); };
  // members: closure nodes all of whose active cells are patch cells
  // closure node o: its coordinates in the (2p+1)^d closure and, along each
  // direction, the cells containing it as offsets from the patch's first
  // cell v - 1 (two where the node lies on a cell boundary)
  struct ClosureNode {
    int oc[3], rc[3][2], nrc[3];
  };
  std::vector<ClosureNode> cnode(NCL);
  for (int o = 0; o < NCL; ++o) {
    ClosureNode& q = cnode[o];
    int u = o;
    for (int k = 0; k < 3; ++k) {
      q.oc[k] = 0;
      q.rc[k][0] = q.rc[k][1] = 0;
      q.nrc[k] = 1;
    }
    for (int k = 0; k < d; ++k) {
      const int ok = u % C;
      u /= C;
      q.oc[k] = ok;
      q.rc[k][0] = (ok % p == 0) ? ok / p - 1 : ok / p;
      q.rc[k][1] = ok / p;
      q.nrc[k] = (ok % p == 0) ? 2 : 1;
    }
  }
  std::vector<std::vector<uint16_t>> mem(ncp);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t j = 0; j < ncp; ++j) {
    int v[3] = {0, 0, 0};
    int64_t t = L.cut_vert[j];
    for (int k = 0; k < d; ++k) {
      v[k] = (int)(t % np);
      t /= np;
    }
    for (int o = 0; o < NCL; ++o) {
      const ClosureNode& q = cnode[o];
      bool valid = true;
      for (int k = 0; k < d; ++k) {
        const int li = p * (v[k] - 1) + q.oc[k];
        if (li < 0 || li >= n) valid = false;
      }
      if (!valid) continue;
      bool inside = false, outside = false;
      for (int s2 = 0; s2 < q.nrc[2]; ++s2)
        for (int s1 = 0; s1 < q.nrc[1]; ++s1)
          for (int s0 = 0; s0 < q.nrc[0]; ++s0) {
            const int r[3] = {q.rc[0][s0], q.rc[1][s1], q.rc[2][s2]};
            int c[3] = {0, 0, 0};
            bool in_mesh = true, in_patch = true;
            for (int k = 0; k < d; ++k) {
              c[k] = v[k] - 1 + r[k];
              if (c[k] < 0 || c[k] >= N) in_mesh = false;
              if (r[k] != 0 && r[k] != 1) in_patch = false;
            }
            if (in_mesh && (cflag_at(c) & kFlagActive)) (in_patch ? inside : outside) = true;
          }
      if (inside && !outside) mem[j].push_back((uint16_t)o);
    }
  }
  L.cut_n.resize(ncp);
  L.cut_moff.resize(ncp);
  L.cut_ioff.resize(ncp);
  int64_t moff = 0, ioff = 0;
  L.cut_maxm2.assign(ncol, 0);
  for (int64_t j = 0; j < ncp; ++j) {
    int m = (int)mem[j].size();
    L.cut_n[j] = m;
    L.cut_moff[j] = (int)moff;
    L.cut_ioff[j] = ioff;
    moff += m;
    // every inverse starts on a 16-byte boundary in FP64 and FP32 (TMA bulk copies)
    ioff += ((int64_t)m * m + 3) / 4 * 4;
  }
  for (int col = 0; col < ncol; ++col)
    for (int j = L.cut_start[col]; j < L.cut_start[col + 1]; ++j)
      L.cut_maxm2[col] = std::max(L.cut_maxm2[col], L.cut_n[j] * L.cut_n[j]);
  L.members.resize((size_t)moff);
  L.member_node.resize((size_t)moff);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t j = 0; j < ncp; ++j) {
    const int m = L.cut_n[j];
    std::copy(mem[j].begin(), mem[j].end(), L.members.begin() + L.cut_moff[j]);
    int v[3] = {0, 0, 0};
    int64_t t = L.cut_vert[j];
    for (int k = 0; k < d; ++k) {
      v[k] = (int)(t % np);
      t /= np;
    }
    for (int e = 0; e < m; ++e) {
      int o = mem[j][e];
      int64_t node = 0, st = 1;
      for (int k = 0; k < d; ++k) {
        node += (int64_t)(p * (v[k] - 1) + o % C) * st;
        o /= C;
        st *= n;
      }
      L.member_node[(size_t)L.cut_moff[j] + e] = (int)node;
    }
  }
  L.n_inv = ioff;
  if (!dry) L.inv.resize(ioff);  // every slot zeroed and filled by its patch below
}

// Ghost-face entries of every cut-patch DoF (the faces whose two cells
// contain the node), and per colour the faces these rows need.  Entries
// are counted, then written at their offsets, member by member in
// parallel (the lists are the same for every thread count).
void cut_patch_face_entries(HostLevel& L) {
  const int d = L.d, p = L.p, N = L.N, n = L.n, ncol = 1 << d;
  const int NTf = ipow(p + 1, d - 1);
  const int64_t nmem = (int64_t)L.member_node.size();
  // entry = ((face id * NTf) + tangential node) * 16 + node along the normal (0 .. 2p)
  auto entries = [&](int64_t gm, auto&& emit) {
    int64_t t = L.member_node[gm];
    int idx[3] = {0, 0, 0};
    for (int k = 0; k < d; ++k) {
      idx[k] = (int)(t % n);
      t /= n;
    }
    int cc[3][2], lcl[3][2], nopt[3] = {1, 1, 1};
    for (int k = 0; k < d; ++k) nopt[k] = cells_of(idx[k], p, N, cc[k], lcl[k]);
    for (int k = 0; k < d; ++k) {
      const int a = idx[k] / p, r = idx[k] - a * p;
      int Llo = (r == 0) ? a - 2 : a - 1, Lhi = a;
      Llo = std::max(Llo, 0);
      Lhi = std::min(Lhi, N - 2);
      int td[2] = {0, 0}, q = 0;
      for (int jj = 0; jj < d; ++jj)
        if (jj != k) td[q++] = jj;
      const int n0 = nopt[td[0]], n1 = (d == 3) ? nopt[td[1]] : 1;
      for (int Lk = Llo; Lk <= Lhi; ++Lk)
        for (int u0 = 0; u0 < n0; ++u0)
          for (int u1 = 0; u1 < n1; ++u1) {
            int c[3] = {0, 0, 0};
            c[k] = Lk;
            c[td[0]] = cc[td[0]][u0];
            if (d == 3) c[td[1]] = cc[td[1]][u1];
            int64_t cell = c[0] + (int64_t)N * (c[1] + (d == 3 ? (int64_t)N * c[2] : 0));
            const int id = L.face_id[(size_t)cell * d + k];
            if (id < 0) continue;
            int tt = idx[td[0]] - p * c[td[0]];
            if (d == 3) tt += (p + 1) * (idx[td[1]] - p * c[td[1]]);
            emit(((id * NTf) + tt) * 16 + (idx[k] - p * Lk), id);
          }
    }
  };
  std::vector<int> cnt(nmem, 0);
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t gm = 0; gm < nmem; ++gm) {
    int c = 0;
    entries(gm, [&](int, int) { ++c; });
    cnt[gm] = c;
  }
  L.fofs.assign(nmem + 1, 0);
  for (int64_t gm = 0; gm < nmem; ++gm) L.fofs[gm + 1] = L.fofs[gm] + cnt[gm];
  L.fent.assign((size_t)L.fofs[nmem], 0);
  // colour of every member (the colour of its patch)
  std::vector<uint8_t> mcol(nmem);
  for (int col = 0; col < ncol; ++col)
    for (int j = L.cut_start[col]; j < L.cut_start[col + 1]; ++j)
      std::fill(mcol.begin() + L.cut_moff[j], mcol.begin() + L.cut_moff[j] + L.cut_n[j], (uint8_t)col);
  // need[col][face]: a row of the colour reads the face's moments
  const size_t nf = L.ghost_faces.size();
  std::vector<uint8_t> need((size_t)ncol * nf, 0);
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t gm = 0; gm < nmem; ++gm) {
    int o = L.fofs[gm];
    uint8_t* nc = &need[(size_t)mcol[gm] * nf];
    entries(gm, [&](int v, int id) {
      L.fent[o++] = v;
#pragma omp atomic write
      nc[id] = 1;
    });
  }
  L.cf_start.assign(ncol + 1, 0);
  for (int col = 0; col < ncol; ++col) {
    const uint8_t* nc = &need[(size_t)col * nf];
    for (size_t f = 0; f < nf; ++f)
      if (nc[f]) L.cfaces.push_back((int)f);
    L.cf_start[col + 1] = (int)L.cfaces.size();
  }
}

// Per cut patch, what its block loads up front: the range of its
// ghost-face entries, the element matrix of each patch cell and the
// (cell, local node) pairs whose rows it forms (node a patch DoF)
void cut_patch_rows(HostLevel& L) {
  const int d = L.d, p = L.p, N = L.N, NB = ipow(p + 1, d);
  const int np = N + 1, C = 2 * p + 1, ncol = 1 << d, NCL = ipow(C, d);
  const int64_t ncp = (int64_t)L.cut_vert.size();
  auto cflag_at = [&](const int* c) { return cell_flag(L, c); };
  const int NCELL = 1 << d;
  L.cut_fo.resize(ncp + 1);
  L.cut_cell.assign((size_t)ncp * NCELL, -2);
  L.cut_item_off.assign(ncp + 1, 0);
  L.cut_items.clear();
  // closure offset of local node jj of patch cell sc
  std::vector<int> cell_node((size_t)NCELL * NB);
  for (int sc = 0; sc < NCELL; ++sc)
    for (int jj = 0; jj < NB; ++jj) {
      int o = 0, ost = 1, u = jj;
      for (int k = 0; k < d; ++k) {
        o += (p * ((sc >> k) & 1) + u % (p + 1)) * ost;
        u /= (p + 1);
        ost *= C;
      }
      cell_node[(size_t)sc * NB + jj] = o;
    }
  // per patch (in parallel): its cells, then its items counted and written
  // at their offsets
  auto patch_items = [&](int64_t j, std::vector<char>& is_mem, auto&& emit) {
    int v[3] = {0, 0, 0};
    int64_t t = L.cut_vert[j];
    for (int k = 0; k < d; ++k) {
      v[k] = (int)(t % np);
      t /= np;
    }
    std::fill(is_mem.begin(), is_mem.end(), 0);
    for (int e = 0; e < L.cut_n[j]; ++e) is_mem[L.members[L.cut_moff[j] + e]] = 1;
    for (int sc = 0; sc < NCELL; ++sc) {
      int c[3] = {0, 0, 0};
      for (int k = 0; k < d; ++k) c[k] = v[k] - 1 + ((sc >> k) & 1);
      const uint8_t f = cflag_at(c);
      if (!(f & kFlagActive)) continue;
      const int64_t cell = c[0] + (int64_t)N * (c[1] + (d == 3 ? (int64_t)N * c[2] : 0));
      L.cut_cell[(size_t)j * NCELL + sc] = (f & kFlagCut) ? L.cut_id[cell] : -1;
      for (int jj = 0; jj < NB; ++jj)
        if (is_mem[cell_node[(size_t)sc * NB + jj]]) emit((uint8_t)(sc * NB + jj));
    }
  };
#pragma omp parallel
  {
    std::vector<char> is_mem(NCL);
#pragma omp for schedule(dynamic, 64)
    for (int64_t j = 0; j < ncp; ++j) {
      L.cut_fo[j] = L.fofs[L.cut_moff[j]];
      int c = 0;
      patch_items(j, is_mem, [&](uint8_t) { ++c; });
      L.cut_item_off[j + 1] = c;
    }
  }
  for (int64_t j = 0; j < ncp; ++j) L.cut_item_off[j + 1] += L.cut_item_off[j];
  L.cut_items.assign((size_t)L.cut_item_off[ncp], 0);
#pragma omp parallel
  {
    std::vector<char> is_mem(NCL);
#pragma omp for schedule(dynamic, 64)
    for (int64_t j = 0; j < ncp; ++j) {
      int o = L.cut_item_off[j];
      patch_items(j, is_mem, [&](uint8_t it) { L.cut_items[o++] = it; });
    }
  }
  L.cut_fo[ncp] = L.fofs[L.member_node.size()];
  L.cut_maxit.assign(ncol, 0);
  for (int col = 0; col < ncol; ++col)
    for (int j = L.cut_start[col]; j < L.cut_start[col + 1]; ++j)
      L.cut_maxit[col] = std::max(L.cut_maxit[col], L.cut_item_off[j + 1] - L.cut_item_off[j]);
}

// Work model of the cut-patch solve (what the kernel computes per patch):
// 2 NB flops per (active patch cell, patch DoF in it) for the cell rows,
// 2p per ghost-face entry of a patch row, 2 m^2 for the local inverse.
// Moved scalars: the inverse, the rows of cut-cell matrices used, the
// closure of x, b and delta of the DoFs, p moments per ghost-face entry;
// index bytes: the DoF lists, metadata, cell ids, row items and entries.
// Face moments (computed once per colour step for the faces its patches
// need): per face 2 (2p+1) p NT for the jumps, 2 p (p+1) NT per face
// direction for the face mass, p NT for the coefficients; x of the two
// cells read, p NT moments written.
void patch_work_model(HostLevel& L) {
  const int d = L.d, p = L.p, NB = ipow(p + 1, d);
  const int C = 2 * p + 1, ncol = 1 << d, NCL = ipow(C, d);
  const int NT = ipow(p + 1, d - 1);
  L.work_cut.assign(ncol, {0.0, 0.0, 0.0});
  L.work_face.assign(ncol, {0.0, 0.0, 0.0});
  for (int col = 0; col < ncol; ++col) {
    for (int j = L.cut_start[col]; j < L.cut_start[col + 1]; ++j) {
      const int m = L.cut_n[j];
      const double nent = L.cut_fo[j + 1] - L.cut_fo[j];
      const double nit = L.cut_item_off[j + 1] - L.cut_item_off[j];
      double fl = 2.0 * m * m + 2.0 * NB * nit + 2.0 * p * nent;
      double sc = (double)m * m + NCL + 2.0 * m + p * nent;
      for (int q = L.cut_item_off[j]; q < L.cut_item_off[j + 1]; ++q)
        if (L.cut_cell[(size_t)j * (1 << d) + L.cut_items[q] / NB] >= 0) sc += NB;
      L.work_cut[col][0] += fl;
      L.work_cut[col][1] += sc;
      L.work_cut[col][2] += 10.0 * m + 72.0 + nit + 4.0 * nent;
    }
    const double nf = L.cf_start[col + 1] - L.cf_start[col];
    const double flf = 2.0 * (2 * p + 1) * p * NT + 2.0 * p * (p + 1) * NT * (d - 1) + (double)p * NT;
    L.work_face[col] = {nf * flf, nf * ((2.0 * p + 1) * NT + (double)p * NT), nf * 8.0};
  }
  // interior patches: sum factorisation and fast diagonalisation
  const int M = 2 * p - 1;
  double flc, scc;
  if (d == 3) {
    flc = 2.0 * (2.0 * M * C * C * C + 3.0 * M * M * C * C + 2.0 * M * M * M * C + 6.0 * M * M * M * M + M * M * M);
    scc = (double)C * C * C + 2.0 * M * M * M;
  } else {
    flc = 2.0 * (2.0 * M * C * C + 2.0 * M * M * C + 4.0 * M * M * M + M * M);
    scc = (double)C * C + 2.0 * M * M;
  }
  L.work_cart.assign(ncol, {0.0, 0.0, 0.0});
  for (int col = 0; col < ncol; ++col) {
    double np_ = L.cart_start[col + 1] - L.cart_start[col];
    L.work_cart[col] = {np_ * flc, np_ * scc, np_ * 4.0};
  }
}

// Cut-patch matrices A_j = A[I_j, I_j] from their cell and ghost-face pieces,
// inverted in place (explicit FP64 inverse per patch).
void cut_patch_inverses(const RefTables& R, HostLevel& L, bool invert) {
  const int d = L.d, p = L.p, N = L.N, NB = R.NB;
  const int np = N + 1, C = 2 * p + 1, NCL = ipow(C, d);
  const int64_t ncp = (int64_t)L.cut_vert.size();
  auto cflag_at = [&](const int* c) { return cell_flag(L, c); };
  // ghost-face block of one face (block nodes e = i + (2p+1) u: i along the
  // normal over both cells, u tangential): the same for every face and
  // direction of the level
  const int tn = ipow(p + 1, d - 1), nbk = (2 * p + 1) * tn;
  std::vector<int> fb_i(nbk), fb_t((size_t)nbk * 2, 0);
  for (int e = 0; e < nbk; ++e) {
    int u = e / (2 * p + 1);
    fb_i[e] = e % (2 * p + 1);
    for (int q = 0; q < d - 1; ++q) {
      fb_t[e * 2 + q] = u % (p + 1);
      u /= p + 1;
    }
  }
  std::vector<double> fblk((size_t)nbk * nbk);
  for (int e1 = 0; e1 < nbk; ++e1)
    for (int e2 = 0; e2 < nbk; ++e2) {
      double tm = 1.0;
      for (int q = 0; q < d - 1; ++q) tm *= L.Mhat[fb_t[e1 * 2 + q]][fb_t[e2 * 2 + q]];
      double s = 0.0;
      for (int mm = 0; mm < p; ++mm) s += L.coef[mm] * L.dvec[mm][fb_i[e1]] * L.dvec[mm][fb_i[e2]];
      fblk[(size_t)e1 * nbk + e2] = s * tm;
    }
  // A_j = A[I_j, I_j] from cell and ghost-face pieces, then inverted
  std::vector<int> err(ncp, 0);
  std::string first_err;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t j = 0; j < ncp; ++j) {
    int v[3] = {0, 0, 0};
    int64_t t = L.cut_vert[j];
    for (int k = 0; k < d; ++k) {
      v[k] = (int)(t % np);
      t /= np;
    }
    const int m = L.cut_n[j];
    std::vector<int> pos(NCL, -1);
    for (int a = 0; a < m; ++a) pos[L.members[L.cut_moff[j] + a]] = a;
    double* A = &L.inv[L.cut_ioff[j]];
    std::fill(A, L.inv.data() + (j + 1 < ncp ? L.cut_ioff[j + 1] : (int64_t)L.inv.size()), 0.0);
    auto closure_of = [&](const int* lat) -> int {  // lattice coords -> member or -1
      int o = 0, st = 1;
      for (int k = 0; k < d; ++k) {
        int ok = lat[k] - p * (v[k] - 1);
        if (ok < 0 || ok >= C) return -1;
        o += ok * st;
        st *= C;
      }
      return pos[o];
    };
    // cells of the patch
    for (int s = 0; s < (1 << d); ++s) {
      int c[3] = {0, 0, 0};
      for (int k = 0; k < d; ++k) c[k] = v[k] - 1 + ((s >> k) & 1);
      uint8_t f = cflag_at(c);
      if (!(f & kFlagActive)) continue;
      int64_t cf = 0, st = 1;
      for (int k = 0; k < d; ++k) {
        cf += (int64_t)c[k] * st;
        st *= N;
      }
      const double* K = (f & kFlagCut) ? &L.cutmat[(size_t)L.cut_id[cf] * NB * NB] : L.Kref.data();
      // the cell's nodes that are patch DoFs (va, in node order) and their rows
      int mi[64], va[64], nv = 0;
      for (int jl = 0; jl < NB; ++jl) {
        int a[3] = {0, 0, 0}, lat[3] = {0, 0, 0};
        R.split(jl, a);
        for (int k = 0; k < d; ++k) lat[k] = p * c[k] + a[k];
        mi[jl] = closure_of(lat);
        if (mi[jl] >= 0) va[nv++] = jl;
      }
      for (int x = 0; x < nv; ++x) {
        const int a = va[x];
        double* Ar = A + (size_t)mi[a] * m;
        const double* Ka = K + a * NB;
        for (int y = 0; y < nv; ++y) Ar[mi[va[y]]] += Ka[va[y]];
      }
    }
    // ghost faces touching a patch cell: lower cell Lc, upper Lc + e_k
    for (int k = 0; k < d; ++k) {
      int rng_lo[3], rng_hi[3];
      for (int kk = 0; kk < d; ++kk) {
        rng_lo[kk] = v[kk] - 1;
        rng_hi[kk] = v[kk];
      }
      rng_lo[k] = v[k] - 2;
      for (int c2 = (d > 2 ? rng_lo[2] : 0); c2 <= (d > 2 ? rng_hi[2] : 0); ++c2)
        for (int c1 = rng_lo[1]; c1 <= rng_hi[1]; ++c1)
          for (int c0 = rng_lo[0]; c0 <= rng_hi[0]; ++c0) {
            int lc[3] = {c0, c1, c2}, uc[3] = {c0, c1, c2};
            uc[k] += 1;
            uint8_t f1 = cflag_at(lc), f2 = cflag_at(uc);
            if (!((f1 & kFlagActive) && (f2 & kFlagActive) && ((f1 | f2) & kFlagCut))) continue;
            // block nodes: i in [0, 2p] along k, t in [0, p] tangential
            int mi[7 * 16], ve[7 * 16], nv = 0;
            for (int e = 0; e < nbk; ++e) {
              int lat[3] = {0, 0, 0}, q = 0;
              for (int kk = 0; kk < d; ++kk)
                lat[kk] = p * lc[kk] + (kk == k ? fb_i[e] : fb_t[e * 2 + q++]);
              mi[e] = closure_of(lat);
              if (mi[e] >= 0) ve[nv++] = e;
            }
            for (int x = 0; x < nv; ++x) {
              const int e1 = ve[x];
              const double* fr = &fblk[(size_t)e1 * nbk];
              double* Ar = A + (size_t)mi[e1] * m;
              for (int y = 0; y < nv; ++y) Ar[mi[ve[y]]] += fr[ve[y]];
            }
          }
    }
    try {
      if (invert) spd_inverse(m, A);
    } catch (const std::exception& e) {
      err[j] = 1;
#pragma omp critical
      if (first_err.empty())
        first_err = "cut patch at vertex (" + std::to_string(v[0]) + "," + std::to_string(v[1]) + "," +
                    std::to_string(v[2]) + ") with " + std::to_string(m) + " DoFs on level N=" +
                    std::to_string(N) + ": " + e.what();
    }
  }
  for (int64_t j = 0; j < ncp; ++j)
    if (err[j]) throw std::runtime_error(first_err);
}

// Records of the block cut kernel: ghost-face masks, per-cell pack offsets,
// and (unless dry) the packed inverses and cut-cell row packs.
// row stride of a record's inverse: m rounded up to 4 (16-byte rows)
static inline int cut_n_pad(int m) { return (m + 3) / 4 * 4; }

void cut_patch_records(HostLevel& L, bool dry) {
  const int d = L.d, p = L.p, N = L.N, NB = ipow(p + 1, d), NCELL = 1 << d;
  const int NBP = (NB + 3) / 4 * 4;  // row stride of the cut rows (16-byte rows)
  if (ipow(2 * p + 1, d) <= 64) return;  // one warp per patch: the entry-list kernel
  const int64_t ncp = (int64_t)L.cut_vert.size();
  const int np = N + 1, ncol = 1 << d, half = 1 << (d - 1);
  auto cflag_at = [&](const int* c) { return cell_flag(L, c); };
  L.cut_roff.assign(ncp + 1, 0);
  L.cut_pk.assign((size_t)ncp * NCELL, -2);
  L.cut_gmask.assign(ncp, 0);
  std::vector<int> rows(ncp, 0);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t j = 0; j < ncp; ++j) {
    int v[3] = {0, 0, 0};
    int64_t t = L.cut_vert[j];
    for (int k = 0; k < d; ++k) {
      v[k] = (int)(t % np);
      t /= np;
    }
    // pack offsets: the items of one cell are consecutive (emitted cell by cell)
    const int i0 = L.cut_item_off[j], i1 = L.cut_item_off[j + 1];
    int r = 0;
    for (int sc = 0; sc < NCELL; ++sc) {
      const int id = L.cut_cell[(size_t)j * NCELL + sc];
      int q0 = i1 - i0, cnt = 0;
      for (int q = i0; q < i1; ++q)
        if (L.cut_items[q] / NB == sc) {
          if (cnt == 0) q0 = q - i0;
          ++cnt;
        }
      if (id == -2) continue;
      if (id == -1) {
        L.cut_pk[(size_t)j * NCELL + sc] = -1;
        continue;
      }
      L.cut_pk[(size_t)j * NCELL + sc] = (r << 8) | q0;
      r += cnt;
    }
    rows[j] = r;
    // ghost faces of the block: plane L of direction k between cell layers
    // L - 1 and L (block layers 0, 1; -1 and 2 outside)
    uint64_t mask = 0;
    for (int k = 0; k < d; ++k)
      for (int Lp = 0; Lp < 3; ++Lp)
        for (int u = 0; u < half; ++u) {
          int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, q = 0;
          for (int kk = 0; kk < d; ++kk) {
            if (kk == k) {
              lo[kk] = v[kk] - 1 + Lp - 1;
              hi[kk] = v[kk] - 1 + Lp;
            } else {
              lo[kk] = hi[kk] = v[kk] - 1 + ((u >> q) & 1);
              ++q;
            }
          }
          const uint8_t f1 = cflag_at(lo), f2 = cflag_at(hi);
          if ((f1 & kFlagActive) && (f2 & kFlagActive) && ((f1 | f2) & kFlagCut))
            mask |= 1ull << ((k * 3 + Lp) * half + u);
        }
    L.cut_gmask[j] = mask;
  }
  for (int64_t j = 0; j < ncp; ++j) {
    const int64_t m = L.cut_n[j];
    const int64_t len = m * ((m + 3) / 4 * 4) + (int64_t)rows[j] * NBP;
    L.cut_roff[j + 1] = L.cut_roff[j] + len;
  }
  L.n_rec = L.cut_roff[ncp];
  // moment slots of the block-boundary ghost faces, and per colour the faces
  // with their destination slots
  uint64_t bnd_bits = 0;
  for (int k = 0; k < d; ++k)
    for (int u = 0; u < half; ++u) bnd_bits |= (1ull << ((k * 3 + 0) * half + u)) | (1ull << ((k * 3 + 2) * half + u));
  L.cut_gboff.assign(ncp + 1, 0);
  for (int64_t j = 0; j < ncp; ++j) L.cut_gboff[j + 1] = L.cut_gboff[j] + __builtin_popcountll(L.cut_gmask[j] & bnd_bits);
  L.bf_start.assign(ncol + 1, 0);
  L.bf_face.clear();
  L.bf_dst.clear();
  // the colours side by side, each into its own lists, joined in colour order
  std::vector<std::vector<int>> bff(ncol), bfd(ncol);
  std::vector<std::string> bf_err(ncol);
#pragma omp parallel for schedule(dynamic, 1)
  for (int col = 0; col < ncol; ++col) try {
    std::vector<std::pair<int, int>> fd;  // (face id, slot)
    for (int j = L.cut_start[col]; j < L.cut_start[col + 1]; ++j) {
      int v[3] = {0, 0, 0};
      int64_t t = L.cut_vert[j];
      for (int k = 0; k < d; ++k) {
        v[k] = (int)(t % np);
        t /= np;
      }
      int rank = 0;
      for (int bit = 0; bit < 3 * d * half; ++bit) {
        if (!((L.cut_gmask[j] >> bit) & 1ull) || !((bnd_bits >> bit) & 1ull)) continue;
        const int u = bit % half, k = bit / half / 3, Lp = bit / half % 3;
        int lo[3] = {0, 0, 0}, q = 0;
        for (int kk = 0; kk < d; ++kk)
          lo[kk] = (kk == k) ? v[kk] - 1 + Lp - 1 : v[kk] - 1 + ((u >> q++) & 1);
        const int64_t cell = lo[0] + (int64_t)N * (lo[1] + (d == 3 ? (int64_t)N * lo[2] : 0));
        const int fid = L.face_id[(size_t)cell * d + k];
        if (fid < 0) throw std::logic_error("block-boundary ghost face without a face id");
        fd.push_back({fid, L.cut_gboff[j] + rank});
        ++rank;
      }
    }
    std::sort(fd.begin(), fd.end());
    std::vector<int>&face = bff[col], &dst = bfd[col];
    for (size_t i = 0; i < fd.size();) {
      face.push_back(fd[i].first);
      dst.push_back(fd[i].second);
      if (i + 1 < fd.size() && fd[i + 1].first == fd[i].first) {
        if (i + 2 < fd.size() && fd[i + 2].first == fd[i].first)
          throw std::logic_error("a ghost face read by three patches of one colour");
        dst.push_back(fd[i + 1].second);
        i += 2;
      } else {
        dst.push_back(-1);
        i += 1;
      }
    }
  } catch (const std::exception& e) {
    bf_err[col] = e.what();
  }
  for (int col = 0; col < ncol; ++col) {
    if (!bf_err[col].empty()) throw std::logic_error(bf_err[col]);
    L.bf_face.insert(L.bf_face.end(), bff[col].begin(), bff[col].end());
    L.bf_dst.insert(L.bf_dst.end(), bfd[col].begin(), bfd[col].end());
    L.bf_start[col + 1] = (int)L.bf_face.size();
  }
  // ghost-entry lists (the faces on the block planes whose stencil contains
  // each DoF: along every direction k the planes of the faces of the DoF's
  // cell layers, and the tangential cells of the plane containing it)
  {
    const int C = 2 * p + 1, NTf = ipow(p + 1, d - 1);
    (void)NTf;
    std::vector<std::vector<uint16_t>> lists(ncp);
    // closure-local digits of every closure node, and per digit its cell
    // layer and whether it lies on a layer boundary
    const int NCLc = ipow(C, d), nbits = 3 * d * half;
    std::vector<std::array<int, 3>> digits(NCLc);
    for (int o = 0; o < NCLc; ++o) {
      int u = o;
      digits[o] = {0, 0, 0};
      for (int k = 0; k < d; ++k) {
        digits[o][k] = u % C;
        u /= C;
      }
    }
    int lay_of[16], on_of[16];
    for (int ok = 0; ok < C; ++ok) {
      lay_of[ok] = ok / p;
      on_of[ok] = ok % p == 0;
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < ncp; ++j) {
      const int m = L.cut_n[j];
      const uint64_t gm = L.cut_gmask[j];
      // moment slot of every set face bit: the block-boundary faces first
      // (bit order), then the middle-plane faces (bit order)
      int slot_of[64];
      for (int bit = 0; bit < nbits; ++bit) {
        const uint64_t below = (1ull << bit) - 1ull;
        slot_of[bit] = ((bnd_bits >> bit) & 1ull)
                           ? __builtin_popcountll(gm & bnd_bits & below)
                           : __builtin_popcountll(gm & bnd_bits) + __builtin_popcountll(gm & ~bnd_bits & below);
      }
      std::vector<uint16_t> offs(m + 1, 0), ent;
      for (int e = 0; e < m; ++e) {
        const std::array<int, 3>& o = digits[L.members[L.cut_moff[j] + e]];
        for (int k = 0; k < d; ++k) {
          const int ok = o[k], lay = lay_of[ok], onp = on_of[ok];
          const int Llo = std::max(0, onp ? lay - 1 : lay), Lhi = std::min(2, lay + 1);
          for (int Lp = Llo; Lp <= Lhi; ++Lp) {
            const int i = ok - p * (Lp - 1);
            int ulo[2] = {0, 0}, uhi[2] = {0, 0}, tj[2] = {0, 0}, q = 0;
            for (int kk = 0; kk < d; ++kk) {
              if (kk == k) continue;
              const int oj = o[kk], cj = lay_of[oj], on = on_of[oj];
              ulo[q] = std::max(0, on ? cj - 1 : cj);
              uhi[q] = std::min(1, cj);
              tj[q] = oj;
              ++q;
            }
            for (int u1 = (d == 3 ? ulo[1] : 0); u1 <= (d == 3 ? uhi[1] : 0); ++u1)
              for (int u0 = ulo[0]; u0 <= uhi[0]; ++u0) {
                const int bit = (k * 3 + Lp) * half + u0 + 2 * u1;
                if (!((gm >> bit) & 1ull)) continue;
                const int t = (tj[0] - p * u0) + (d == 3 ? (p + 1) * (tj[1] - p * u1) : 0);
                ent.push_back((uint16_t)(slot_of[bit] | (i << 6) | (t << 10)));
              }
          }
        }
        offs[e + 1] = (uint16_t)ent.size();
      }
      std::vector<uint16_t>& out = lists[j];
      out = offs;
      out.insert(out.end(), ent.begin(), ent.end());
      out.resize((out.size() + 7) / 8 * 8, 0);
    }
    L.cut_geoff.assign(ncp + 1, 0);
    for (int64_t j = 0; j < ncp; ++j) L.cut_geoff[j + 1] = L.cut_geoff[j] + (int)lists[j].size();
    L.cut_gent.resize(L.cut_geoff[ncp]);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < ncp; ++j) std::copy(lists[j].begin(), lists[j].end(), L.cut_gent.begin() + L.cut_geoff[j]);
  }
  // work model of the record kernel (replaces the entry-list kernel's):
  // flops 2 m^2 (solve) + 2 NB per row item + per middle-plane ghost face
  // p NT (2 (2p+1) + 2 NT) for its moments + 2p per ghost entry of a row;
  // scalars, the algorithmic minimum: the inverse's m (m + 1) / 2 distinct
  // entries (the stored record holds all m^2, rows padded) and the cut rows'
  // NB entries each, the closures of x and b, the halo of the boundary ghost
  // faces, x of the DoFs written; index bytes: DoF list, items, cell kinds,
  // ghost-entry list, metadata.  The boundary-plane face moments are a
  // separate launch (work_face).
  {
    const int NTf = ipow(p + 1, d - 1), NCL = ipow(2 * p + 1, d);
    uint64_t bnd_mask = 0;
    for (int k = 0; k < d; ++k)
      for (int u = 0; u < half; ++u) bnd_mask |= (1ull << ((k * 3 + 0) * half + u)) | (1ull << ((k * 3 + 2) * half + u));
    L.work_cut.assign(ncol, {0.0, 0.0, 0.0});
    L.work_face.assign(ncol, {0.0, 0.0, 0.0});
    for (int col = 0; col < ncol; ++col)
      for (int j = L.cut_start[col]; j < L.cut_start[col + 1]; ++j) {
        const double m = L.cut_n[j], nit = L.cut_item_off[j + 1] - L.cut_item_off[j];
        const double nent = L.cut_gent[L.cut_geoff[j] + L.cut_n[j]];  // ghost entries of the patch rows
        const double nbf = __builtin_popcountll(L.cut_gmask[j] & bnd_mask);
        const double nf = __builtin_popcountll(L.cut_gmask[j]) - nbf;  // internal faces, formed in the block
        L.work_cut[col][0] += 2.0 * m * m + 2.0 * NB * nit + nf * p * NTf * (2.0 * (2 * p + 1) + 2.0 * NTf) +
                              2.0 * p * nent;
        L.work_cut[col][1] += m * (m + 1) / 2 + (double)rows[j] * NB + 2.0 * NCL + nbf * p * NTf + m;
        L.work_cut[col][2] += 4.0 * m + nit + 4.0 * NCELL + 56.0 + 2.0 * (L.cut_geoff[j + 1] - L.cut_geoff[j]);
      }
    // the boundary-face moment launch of each colour: per face the jumps,
    // the face mass and the coefficients; x of the two cells read, the
    // moments written to each destination slot
    for (int col = 0; col < ncol; ++col) {
      const double flf = 2.0 * (2 * p + 1) * p * NTf + 2.0 * p * (p + 1) * NTf * (d - 1) + (double)p * NTf;
      double fl = 0.0, sc = 0.0, ib = 0.0;
      for (int i = L.bf_start[col]; i < L.bf_start[col + 1]; ++i) {
        const int nd = (L.bf_dst[2 * i] >= 0) + (L.bf_dst[2 * i + 1] >= 0);
        fl += flf;
        sc += (2.0 * p + 1) * NTf + (double)p * NTf * nd;
        ib += 16.0;
      }
      L.work_face[col] = {fl, sc, ib};
    }
  }
  L.cut_maxrec.assign(ncol, 0);
  for (int col = 0; col < ncol; ++col)
    for (int j = L.cut_start[col]; j < L.cut_start[col + 1]; ++j)
      L.cut_maxrec[col] = std::max(L.cut_maxrec[col], (int)(L.cut_roff[j + 1] - L.cut_roff[j]));
  if (dry) return;
  L.rec.resize((size_t)L.n_rec);
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t j = 0; j < ncp; ++j) {
    // every entry written once: rows, their zero padding, and zeros after
    // the last row
    double* out = &L.rec[(size_t)L.cut_roff[j]];
    double* const end = L.rec.data() + L.cut_roff[j + 1];
    const int m = L.cut_n[j];
    const double* A = &L.inv[(size_t)L.cut_ioff[j]];
    const int MP = cut_n_pad(m);
    for (int i = 0; i < m; ++i) {
      std::copy(A + (size_t)i * m, A + (size_t)(i + 1) * m, out + (size_t)i * MP);
      std::fill(out + (size_t)i * MP + m, out + (size_t)(i + 1) * MP, 0.0);
    }
    double* rp = out + (size_t)m * MP;
    const int i0 = L.cut_item_off[j], i1 = L.cut_item_off[j + 1];
    for (int q = i0; q < i1; ++q) {
      const int sc = L.cut_items[q] / NB, jj = L.cut_items[q] % NB;
      const int id = L.cut_cell[(size_t)j * NCELL + sc];
      if (id < 0) continue;
      const double* K = &L.cutmat[((size_t)id * NB + jj) * NB];
      std::copy(K, K + NB, rp);
      std::fill(rp + NB, rp + NBP, 0.0);
      rp += NBP;
    }
    std::fill(rp, end, 0.0);
  }
}

// Patches (Sec. 2.3, Sec. 3) of a level: vertex sets by colour, and for the
// cut patches their DoF lists, ghost-face entries, row items, work model and
// explicit inverses.
void build_patches(const RefTables& R, HostLevel& L, bool dry, bool device_inverse) {
  patch_vertex_sets(L);
  cut_patch_members(L, dry);
  cut_patch_face_entries(L);
  cut_patch_rows(L);
  patch_work_model(L);
  L.inv_on_device = device_inverse && ipow(2 * L.p + 1, L.d) > 64;
  if (!dry) cut_patch_inverses(R, L, !L.inv_on_device);
  cut_patch_records(L, dry);
}

// Optional: with cut_rhs, the cut cells' right-hand side terms for source
// fsrc and Dirichlet data gdir are formed from the same quadrature rules
// (n_cut x NB, in cut-cell order).
using PointFn = std::function<double(const double*)>;
void build_level(const SetupParams& prm, const RefTables& R, int N, HostLevel& L, const PointFn* fsrc = nullptr,
                 const PointFn* gdir = nullptr, std::vector<double>* cut_rhs = nullptr) {
  const int d = prm.dim, p = prm.degree, NB = R.NB;
  L.d = d;
  L.p = p;
  L.N = N;
  L.n = p * N + 1;
  L.lo = prm.lo;
  L.h = (prm.hi - prm.lo) / N;
  const double h = L.h;
  const int n = L.n;
  const int64_t ncell = (int64_t)ipow(N, d), nnode = (int64_t)ipow(n, d);
  L.cflag.assign(ncell, 0);
  L.cut_id.assign(ncell, -1);
  // classification (Sec. 2.1: active = meets Omega, cut = meets Gamma), and
  // the range of the active cells' coordinates
  int cmin[3] = {N, N, N}, cmax[3] = {-1, -1, -1};
#pragma omp parallel for schedule(static) reduction(min : cmin[:3]) reduction(max : cmax[:3])
  for (int64_t c = 0; c < ncell; ++c) {
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    int ci[3] = {0, 0, 0};
    int64_t t = c;
    for (int k = 0; k < d; ++k) {
      ci[k] = (int)(t % N);
      t /= N;
      lo[k] = prm.lo + h * ci[k];
      hi[k] = prm.lo + h * (ci[k] + 1);
    }
    double mn, mx;
    prm.ls.box_minmax(lo, hi, mn, mx);
    uint8_t f = 0;
    if (mn < 0.0) f |= kFlagActive;
    if (mn < 0.0 && mx > 0.0) f |= kFlagCut;
    L.cflag[c] = f;
    if (f & kFlagActive)
      for (int k = 0; k < d; ++k) {
        cmin[k] = std::min(cmin[k], ci[k]);
        cmax[k] = std::max(cmax[k], ci[k]);
      }
  }
  std::vector<int64_t> cut_cells;
  ordered_collect(ncell, cut_cells, [&](int64_t c, std::vector<int64_t>& o) {
    if (L.cflag[c] & kFlagCut) o.push_back(c);
  });
  L.n_cut = (int64_t)cut_cells.size();
  int64_t n_active = 0;
#pragma omp parallel for schedule(static) reduction(+ : n_active)
  for (int64_t c = 0; c < ncell; ++c) n_active += (L.cflag[c] & kFlagActive) ? 1 : 0;
  L.n_active = n_active;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < L.n_cut; ++i) L.cut_id[cut_cells[i]] = (int)i;
  if (!prm.dry) L.cutmat.resize((size_t)L.n_cut * NB * NB);  // every block written below
  if (cut_rhs) cut_rhs->assign((size_t)L.n_cut * NB, 0.0);
  CutQuadrature Q(prm.ls, prm.quad_q);
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t i = 0; i < (prm.dry ? 0 : L.n_cut); ++i) {
    int64_t c = cut_cells[i], t = c;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int k = 0; k < d; ++k) {
      lo[k] = prm.lo + h * (int)(t % N);
      t /= N;
    }
    for (int k = 0; k < d; ++k) hi[k] = lo[k] + h;
    CutRule rule = Q.cell(lo, hi);
    cut_cell_matrix(R, rule, lo, h, prm.gamma_D, &L.cutmat[(size_t)i * NB * NB]);
    if (cut_rhs) cut_cell_rhs(R, rule, lo, h, prm.gamma_D, *fsrc, *gdir, &(*cut_rhs)[(size_t)i * NB]);
  }
  // uncut stiffness, Kronecker form of 1D reference matrices
  L.Kref.assign(NB * NB, 0.0);
  L.Kunit.assign(NB * NB, 0.0);
  L.kscale = std::pow(h, d - 2);
  for (int i = 0; i < NB; ++i)
    for (int j = 0; j < NB; ++j) {
      int a[3], b[3];
      R.split(i, a);
      R.split(j, b);
      double s = 0.0;
      for (int k = 0; k < d; ++k) {
        double t = 1.0;
        for (int kk = 0; kk < d; ++kk)
          t *= (kk == k ? R.K1 : R.M1)[a[kk] * (p + 1) + b[kk]];
        s += t;
      }
      L.Kunit[i * NB + j] = s;
      L.Kref[i * NB + j] = s * std::pow(h, d - 2);
    }
  // ghost-face tables
  for (int m = 1; m <= p; ++m) {
    double hm = std::pow(h, m), fact = 1.0;
    for (int j = 2; j <= m; ++j) fact *= j;
    for (int i = 0; i <= 2 * p; ++i) {
      double v = 0.0;
      if (i <= p) v += R.b.eval(i, 1.0, m) / hm;
      if (i >= p) v -= R.b.eval(i - p, 0.0, m) / hm;
      L.dvec[m - 1][i] = v;
    }
    L.coef[m - 1] = prm.gamma_ghost[m - 1] * std::pow(h, 2 * m - 1) / (fact * fact) * std::pow(h, d - 1);
  }
  for (int a = 0; a <= p; ++a)
    for (int b = 0; b <= p; ++b) L.Mhat[a][b] = R.M1[a * (p + 1) + b];
  // nodes
  // the nodes of the active cells, cell layers (outermost coordinate) in two
  // passes, even then odd: the layers of one pass share no node
  L.nact.assign(nnode, 0);
  const int64_t layer = ncell / N;
  for (int par = 0; par < 2; ++par) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int cl = par; cl < N; cl += 2)
      for (int64_t c = cl * layer; c < (cl + 1) * layer; ++c) {
        if (!(L.cflag[c] & kFlagActive)) continue;
        int ci[3] = {0, 0, 0};
        int64_t t = c;
        for (int k = 0; k < d; ++k) {
          ci[k] = (int)(t % N);
          t /= N;
        }
        for (int j = 0; j < NB; ++j) {
          int a[3] = {0, 0, 0};
          R.split(j, a);
          int64_t node = 0, st = 1;
          for (int k = 0; k < d; ++k) {
            node += (int64_t)(p * ci[k] + a[k]) * st;
            st *= n;
          }
          L.nact[node] = 1;
        }
      }
  }
  ordered_collect(nnode, L.dofs, [&](int64_t i, std::vector<int64_t>& o) {
    if (L.nact[i]) o.push_back(i);
  });
  // the active nodes span p cmin_k .. p (cmax_k + 1) along every direction
  for (int k = 0; k < 3; ++k) {
    L.bb_lo[k] = (k < d) ? (cmax[k] < 0 ? n : p * cmin[k]) : 0;
    L.bb_hi[k] = (k < d) ? (cmax[k] < 0 ? -1 : p * (cmax[k] + 1)) : 0;
  }
  auto cflag_at = [&](const int* c) -> uint8_t {
    int64_t f = 0, st = 1;
    for (int k = 0; k < d; ++k) {
      if (c[k] < 0 || c[k] >= N) return 0;
      f += (int64_t)c[k] * st;
      st *= N;
    }
    return L.cflag[f];
  };
  // ghost faces: list and per-cell ids
  L.face_id.assign((size_t)ncell * d, -1);
  ordered_collect(ncell, L.ghost_faces, [&](int64_t c, std::vector<int>& o) {
    const uint8_t f1 = L.cflag[c];
    if (!(f1 & kFlagActive)) return;
    int ci[3] = {0, 0, 0};
    int64_t t = c;
    for (int k = 0; k < d; ++k) {
      ci[k] = (int)(t % N);
      t /= N;
    }
    for (int k = 0; k < d; ++k) {
      int cj[3] = {ci[0], ci[1], ci[2]};
      cj[k] += 1;
      const uint8_t f2 = cflag_at(cj);
      if ((f2 & kFlagActive) && ((f1 | f2) & kFlagCut)) o.push_back((int)(c * d + k));
    }
  });
  L.n_ghost = (int64_t)L.ghost_faces.size();
#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < L.n_ghost; ++g) L.face_id[L.ghost_faces[g]] = (int)g;
  // apply: bulk positions (2^d plain cells around them) and boundary nodes
  {
    const int np = N + 1;
    const int64_t npos = (int64_t)ipow(np, d);
    const std::vector<uint8_t> pl = plain_flags(L);
    std::vector<uint8_t> bulk(npos, 0);
    ordered_collect(npos, L.bulk_pos, [&](int64_t q, std::vector<int>& o) {
      int a[3] = {0, 0, 0};
      int64_t t = q;
      for (int k = 0; k < d; ++k) {
        a[k] = (int)(t % np);
        t /= np;
        if (a[k] < 1 || a[k] > N - 1) return;
      }
      for (int s = 0; s < (1 << d); ++s) {
        int64_t c = 0, st = 1;
        for (int k = 0; k < d; ++k) {
          c += (int64_t)(a[k] - ((s >> k) & 1)) * st;
          st *= N;
        }
        if (!pl[c]) return;
      }
      bulk[q] = 1;
      o.push_back((int)q);
    });
    // the owner position of node i is (i_k / p)_k
    ordered_collect((int64_t)L.dofs.size(), L.bnd_node, [&](int64_t e, std::vector<int>& o) {
      const int64_t i = L.dofs[e];
      int64_t t = i, q = 0, st = 1;
      for (int k = 0; k < d; ++k) {
        const int ik = (int)(t % n);
        t /= n;
        q += (int64_t)(ik / p) * st;
        st *= np;
      }
      if (!bulk[q]) o.push_back((int)i);
    });
  }
  interior_patch_tables(R, L);
  build_patches(R, L, prm.dry, prm.device_inverse);
}

// 1D transfer tables between a coarse level (Nc cells) and its refinement
void build_transfer(const RefTables& R, int Nc, HostLevel& F) {
  const int p = R.p, Nf = 2 * Nc, nf = p * Nf + 1, nc = p * Nc + 1;
  F.pro_col.assign((size_t)nf * (p + 1), 0);
  F.pro_w.assign((size_t)nf * (p + 1), 0.0);
  std::vector<std::vector<std::pair<int, double>>> cols(nc);
  for (int I = 0; I < nf; ++I) {
    int cf = std::min(I / p, Nf - 1), af = I - p * cf, cc = cf / 2;
    double xi = ((cf % 2) + R.b.nodes[af]) * 0.5;
    for (int a = 0; a <= p; ++a) {
      double w = R.b.eval(a, xi);
      F.pro_col[(size_t)I * (p + 1) + a] = p * cc + a;
      F.pro_w[(size_t)I * (p + 1) + a] = w;
      if (w != 0.0) cols[p * cc + a].push_back({I, w});
    }
  }
  const int W = 4 * p + 1;
  F.res_col.assign((size_t)nc * W, 0);
  F.res_w.assign((size_t)nc * W, 0.0);
  for (int J = 0; J < nc; ++J) {
    if ((int)cols[J].size() > W) throw std::runtime_error("transfer stencil wider than expected");
    for (size_t e = 0; e < cols[J].size(); ++e) {
      F.res_col[(size_t)J * W + e] = cols[J][e].first;
      F.res_w[(size_t)J * W + e] = cols[J][e].second;
    }
    for (size_t e = cols[J].size(); e < (size_t)W; ++e) F.res_col[(size_t)J * W + e] = cols[J].empty() ? 0 : cols[J][0].first;
  }
}

// dense A_0 over the coarsest DoFs, explicit inverse
// Every contribution A_l[i][j] += v of a level (active cells' element
// matrices, then the ghost faces of each cell), in a fixed order, with i, j
// DoF indices: the coarse matrix and the Jacobi diagonal are built from it.
template <class Add>
void visit_level_entries(const RefTables& R, const HostLevel& L, Add&& add) {
  const int d = L.d, p = L.p, N = L.N, n = L.n, NB = R.NB;
  const int64_t nd = (int64_t)L.dofs.size();
  std::vector<int64_t> map((size_t)ipow(n, d), -1);
  for (int64_t i = 0; i < nd; ++i) map[L.dofs[i]] = i;
  auto node_of = [&](const int* lat) -> int64_t {
    int64_t f = 0, st = 1;
    for (int k = 0; k < d; ++k) {
      f += (int64_t)lat[k] * st;
      st *= n;
    }
    return map[f];
  };
  auto cflag_at = [&](const int* c) -> uint8_t {
    int64_t f = 0, st = 1;
    for (int k = 0; k < d; ++k) {
      if (c[k] < 0 || c[k] >= N) return 0;
      f += (int64_t)c[k] * st;
      st *= N;
    }
    return L.cflag[f];
  };
  const int64_t ncell = ipow(N, d);
  for (int64_t c = 0; c < ncell; ++c) {
    uint8_t f = L.cflag[c];
    if (!(f & kFlagActive)) continue;
    int ci[3] = {0, 0, 0};
    int64_t t = c;
    for (int k = 0; k < d; ++k) {
      ci[k] = (int)(t % N);
      t /= N;
    }
    const double* K = (f & kFlagCut) ? &L.cutmat[(size_t)L.cut_id[c] * NB * NB] : L.Kref.data();
    std::vector<int64_t> g(NB);
    for (int j = 0; j < NB; ++j) {
      int a[3] = {0, 0, 0}, lat[3] = {0, 0, 0};
      R.split(j, a);
      for (int k = 0; k < d; ++k) lat[k] = p * ci[k] + a[k];
      g[j] = node_of(lat);
    }
    for (int a = 0; a < NB; ++a)
      for (int b = 0; b < NB; ++b) add(g[a], g[b], K[a * NB + b]);
    for (int k = 0; k < d; ++k) {
      int uc[3] = {ci[0], ci[1], ci[2]};
      uc[k] += 1;
      uint8_t f2 = cflag_at(uc);
      if (!((f2 & kFlagActive) && ((f | f2) & kFlagCut))) continue;
      const int tn = ipow(p + 1, d - 1), nbk = (2 * p + 1) * tn;
      std::vector<int64_t> gi(nbk);
      std::vector<int> ii(nbk), tt(nbk * 2);
      for (int e = 0; e < nbk; ++e) {
        int i = e % (2 * p + 1), u = e / (2 * p + 1), q = 0;
        int lat[3] = {0, 0, 0};
        for (int kk = 0; kk < d; ++kk) {
          if (kk == k) {
            lat[kk] = p * ci[kk] + i;
          } else {
            int tv = u % (p + 1);
            u /= p + 1;
            lat[kk] = p * ci[kk] + tv;
            tt[e * 2 + q++] = tv;
          }
        }
        ii[e] = i;
        gi[e] = node_of(lat);
      }
      for (int e1 = 0; e1 < nbk; ++e1)
        for (int e2 = 0; e2 < nbk; ++e2) {
          double tm = 1.0;
          for (int q = 0; q < d - 1; ++q) tm *= L.Mhat[tt[e1 * 2 + q]][tt[e2 * 2 + q]];
          double s = 0.0;
          for (int mm = 0; mm < p; ++mm) s += L.coef[mm] * L.dvec[mm][ii[e1]] * L.dvec[mm][ii[e2]];
          add(gi[e1], gi[e2], s * tm);
        }
    }
  }
  (void)nd;
}

void build_coarse(const RefTables& R, HostLevel& L) {
  const int64_t nd = (int64_t)L.dofs.size();
  std::vector<double>& A = L.coarse_inv;
  A.assign((size_t)nd * nd, 0.0);
  visit_level_entries(R, L, [&](int64_t i, int64_t j, double v) { A[(size_t)i * nd + j] += v; });
  spd_inverse((int)nd, A.data());
}

// diagonal of A_l (point-Jacobi scaling of the Chebyshev smoother)
void build_diag(const RefTables& R, HostLevel& L) {
  L.diag.assign(L.dofs.size(), 0.0);
  visit_level_entries(R, L, [&](int64_t i, int64_t j, double v) {
    if (i == j) L.diag[i] += v;
  });
}

// b_i = (f, phi_i)_Omega + (g, gamma_D/h phi_i - d_n phi_i)_Gamma for
// u = prod sin(pi x_k), f = d pi^2 u, g = u
// loc[j] = sum over the q^d tensor points of F[point] times basis j there
// (Lt[a * q + i]: 1D basis a at Gauss point i), one 1D contraction per
// direction; points and basis indices both run first coordinate fastest.
// work holds 2 max(q, p + 1)^d values.
void tensor_contract(int d, int p, int q, const double* Lt, const double* F, double* loc, double* work) {
  const int half = ipow(std::max(q, p + 1), d);
  int sz[3] = {q, q, q};
  const double* cur = F;
  for (int k = 0; k < d; ++k) {
    double* out = (k == d - 1) ? loc : work + (k & 1) * half;
    int inner = 1, outer = 1;
    for (int kk = 0; kk < k; ++kk) inner *= sz[kk];
    for (int kk = k + 1; kk < d; ++kk) outer *= sz[kk];
    for (int o = 0; o < outer; ++o)
      for (int a = 0; a <= p; ++a)
        for (int i = 0; i < inner; ++i) {
          double acc = 0.0;
          for (int t = 0; t < q; ++t) acc += Lt[a * q + t] * cur[i + inner * (t + q * o)];
          out[i + inner * (a + (p + 1) * o)] = acc;
        }
    sz[k] = p + 1;
    cur = out;
  }
}

void build_rhs(const SetupParams& prm, const RefTables& R, const HostLevel& L, std::vector<double>& b,
               const std::function<double(const double*)>& fsrc, const std::function<double(const double*)>& gdir,
               bool parallel, const std::vector<double>* cut_rhs = nullptr, bool manufactured = false) {
  const int d = L.d, p = L.p, N = L.N, n = L.n, NB = R.NB, q = prm.quad_q;
  const double h = L.h;
  const int64_t nnode = ipow(n, d), ndof = (int64_t)L.dofs.size();
  std::vector<int64_t, DefaultInitAllocator<int64_t>> map((size_t)nnode);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nnode; ++i) map[i] = -1;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < ndof; ++e) map[L.dofs[e]] = e;
  b.assign(L.dofs.size(), 0.0);
  GaussRule g = gauss_legendre01(q);
  const int nq = ipow(q, d);
  std::vector<double> Lt((size_t)(p + 1) * q);
  for (int a = 0; a <= p; ++a)
    for (int t = 0; t < q; ++t) Lt[a * q + t] = R.b.eval(a, g.x[t]);
  const double hd = std::pow(h, d);
  CutQuadrature Q(prm.ls, q);
  const int64_t ncell = ipow(N, d);
  std::vector<int64_t> act;
  for (int64_t c = 0; c < ncell; ++c)
    if (L.cflag[c] & kFlagActive) act.push_back(c);
  // cell contributions in parallel, summed into b in cell order (the result
  // does not depend on the thread count)
  const int64_t nact = (int64_t)act.size(), CH = 1 << 16;
  std::vector<double> locs((size_t)std::min<int64_t>(CH, std::max<int64_t>(nact, 1)) * NB);
  for (int64_t c0 = 0; c0 < nact; c0 += CH) {
    const int64_t c1 = std::min(nact, c0 + CH);
#pragma omp parallel for schedule(dynamic, 64) if (parallel)
    for (int64_t ic = c0; ic < c1; ++ic) {
      const int64_t c = act[ic];
      const uint8_t f = L.cflag[c];
      int ci[3] = {0, 0, 0};
      double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
      int64_t t = c;
      for (int k = 0; k < d; ++k) {
        ci[k] = (int)(t % N);
        t /= N;
        lo[k] = prm.lo + h * ci[k];
        hi[k] = lo[k] + h;
      }
      std::vector<double> Fw((size_t)nq + 2 * ipow(std::max(q, p + 1), d));
      double* loc = &locs[(size_t)(ic - c0) * NB];
      for (int j = 0; j < NB; ++j) loc[j] = 0.0;
      if (!(f & kFlagCut)) {
        // tensor Gauss rule: f w at every point, then sum factorisation
        double* F = Fw.data();
        if (manufactured && q <= 16) {
          // fsrc is the manufactured source d pi^2 prod_k sin(pi x_k): each
          // direction's q sines once per cell, multiplied as fsrc does
          double sn[3][16];
          for (int k = 0; k < d; ++k)
            for (int a = 0; a < q; ++a) sn[k][a] = std::sin(M_PI * (lo[k] + h * g.x[a]));
          for (int iq = 0; iq < nq; ++iq) {
            double w = 1.0, uv = 1.0;
            int u = iq;
            for (int k = 0; k < d; ++k) {
              int a = u % q;
              u /= q;
              w *= g.w[a];
              uv *= sn[k][a];
            }
            const double fv = d * M_PI * M_PI * uv;
            F[iq] = fv * w * hd;
          }
        } else {
          for (int iq = 0; iq < nq; ++iq) {
            double x[3] = {0, 0, 0}, w = 1.0;
            int u = iq;
            for (int k = 0; k < d; ++k) {
              int a = u % q;
              u /= q;
              w *= g.w[a];
              x[k] = lo[k] + h * g.x[a];
            }
            F[iq] = fsrc(x) * w * hd;
          }
        }
        tensor_contract(d, p, q, Lt.data(), F, loc, F + nq);
      } else if (cut_rhs) {
        const double* src = &(*cut_rhs)[(size_t)L.cut_id[c] * NB];
        for (int j = 0; j < NB; ++j) loc[j] = src[j];
      } else {
        cut_cell_rhs(R, Q.cell(lo, hi), lo, h, prm.gamma_D, fsrc, gdir, loc);
      }
    }
    // the sums: node rows (all coordinates but the first, row = node / n)
    // split between the threads, each adding the terms of its rows cell by
    // cell in order, so that every entry takes its terms in cell order
    auto rows_of = [&](int64_t c, int* ci, int64_t& rlo, int64_t& rhi) {
      int64_t t = c, st = 1;
      rlo = rhi = 0;
      for (int k = 0; k < d; ++k) {
        ci[k] = (int)(t % N);
        t /= N;
        if (k > 0) {
          rlo += (int64_t)(p * ci[k]) * st;
          rhi += (int64_t)(p * ci[k] + p) * st;
          st *= n;
        }
      }
    };
    int cf[3], cl[3];
    int64_t R0, R1, dummy;
    rows_of(act[c0], cf, R0, dummy);
    rows_of(act[c1 - 1], cl, dummy, R1);
#pragma omp parallel if (parallel)
    {
      const int tid = omp_get_thread_num(), tn = omp_get_num_threads();
      const int64_t span = R1 - R0 + 1;
      const int64_t r0 = R0 + span * tid / tn, r1 = R0 + span * (tid + 1) / tn;
      for (int64_t ic = c0; ic < c1; ++ic) {
        int ci[3] = {0, 0, 0};
        int64_t rlo, rhi;
        rows_of(act[ic], ci, rlo, rhi);
        if (rhi < r0 || rlo >= r1) continue;
        const double* loc = &locs[(size_t)(ic - c0) * NB];
        for (int j = 0; j < NB; ++j) {
          int a[3] = {0, 0, 0};
          R.split(j, a);
          int64_t node = 0, st = 1;
          for (int k = 0; k < d; ++k) {
            node += (int64_t)(p * ci[k] + a[k]) * st;
            st *= n;
          }
          const int64_t row = node / n;
          if (row >= r0 && row < r1) b[map[node]] += loc[j];
        }
      }
    }
  }
}

}  // namespace

void build_hierarchy(const SetupParams& prm, Hierarchy& H) {
  if (prm.dim != 2 && prm.dim != 3) throw std::invalid_argument("dim must be 2 or 3");
  if (prm.degree < 1 || prm.degree > 4) throw std::invalid_argument("degree must be 1, 2, 3 or 4");
  if (prm.dim == 3 && prm.degree > 2) throw std::invalid_argument("dim 3 supports degree 1 and 2");
  if (prm.n_levels < 1 || prm.n_levels > 12) throw std::invalid_argument("n_levels out of range");
  if (prm.n_cells % (1 << (prm.n_levels - 1)) != 0)
    throw std::invalid_argument("n_cells must be divisible by 2^(n_levels-1)");
  if (prm.n_cells >> (prm.n_levels - 1) < 1) throw std::invalid_argument("coarsest level empty");
  if (!(prm.hi > prm.lo)) throw std::invalid_argument("empty box");
  H.prm = prm;
  H.levels.assign(prm.n_levels, HostLevel());
  RefTables R(prm.degree, prm.dim);
  // manufactured data of the workloads: u = prod sin(pi x_k), f = d pi^2 u, g = u
  const int d = prm.dim;
  auto uex = [d](const double* x) {
    double u = 1.0;
    for (int k = 0; k < d; ++k) u *= std::sin(M_PI * x[k]);
    return u;
  };
  const PointFn fman = [&](const double* x) { return d * M_PI * M_PI * uex(x); }, gman = uex;
  std::vector<double> cut_rhs;  // finest level: cut cells' terms, formed with their matrices
  for (int l = 0; l < prm.n_levels; ++l) {
    int Nl = prm.n_cells >> (prm.n_levels - 1 - l);
    if (l == prm.n_levels - 1 && !prm.dry)
      build_level(prm, R, Nl, H.levels[l], &fman, &gman, &cut_rhs);
    else
      build_level(prm, R, Nl, H.levels[l]);
    if (H.levels[l].dofs.empty()) throw std::invalid_argument("level without active cells");
    if (l > 0) {
      build_transfer(R, H.levels[l - 1].N, H.levels[l]);
      // nesting Omega_l within Omega_{l-1} (Sec. 2.2): every active fine cell has an active parent
      const HostLevel& F = H.levels[l];
      const HostLevel& Cc = H.levels[l - 1];
      const int64_t ncell = ipow(F.N, F.d);
      for (int64_t c = 0; c < ncell; ++c) {
        if (!(F.cflag[c] & kFlagActive)) continue;
        int64_t t = c, pc = 0, st = 1;
        for (int k = 0; k < F.d; ++k) {
          pc += (t % F.N) / 2 * st;
          t /= F.N;
          st *= Cc.N;
        }
        if (!(Cc.cflag[pc] & kFlagActive))
          throw std::invalid_argument("active domains are not nested across levels");
      }
    }
  }
  // without a cut cell there are no Nitsche terms: the operator is the pure
  // Neumann stiffness on the active cells (constants in its kernel)
  if (H.levels.back().n_cut == 0)
    throw std::invalid_argument("no cut cell on the finest level: the domain's boundary does not cross the mesh, "
                                "so the Nitsche-Dirichlet problem has no boundary condition");
  if (H.levels[0].dofs.size() > 12000)
    throw std::invalid_argument("the coarsest level has " + std::to_string(H.levels[0].dofs.size()) +
                                " DoFs (dense exact solve); use more levels");
  if (prm.dry) return;
  build_coarse(R, H.levels[0]);
  if (prm.smoother == 1)
    for (size_t l = 1; l < H.levels.size(); ++l) build_diag(R, H.levels[l]);
  build_rhs(prm, R, H.levels.back(), H.rhs, fman, gman, true, &cut_rhs, true);
}

void build_rhs_user(const Hierarchy& H, double (*f)(const double*, void*), double (*g)(const double*, void*),
                    void* user, std::vector<double>& b) {
  RefTables R(H.prm.degree, H.prm.dim);
  const int d = H.prm.dim;
  auto wrap = [d, user](double (*fn)(const double*, void*)) {
    return [d, user, fn](const double* x) {
      if (!fn) return 0.0;
      double y[3] = {x[0], d > 1 ? x[1] : 0.0, d > 2 ? x[2] : 0.0};
      return fn(y, user);
    };
  };
  build_rhs(H.prm, R, H.levels.back(), b, wrap(f), wrap(g), false);
}

}  // namespace cutmg
