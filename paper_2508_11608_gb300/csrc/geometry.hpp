// Host-side geometry for the setup phase: 1D polynomial bases, Gauss rules,
// level sets and the dimension-reduction cut-cell quadrature (Sec. 3: cut
// cells get non-tensor substitute rules computed upfront on the CPU, after
// Saye 2015).  Compiled with -ffp-contract=off so level-set values and
// bisection roots are reproducible bit for bit.
#pragma once

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <stdexcept>
#include <vector>

namespace cutmg {

// ---------------------------------------------------------------------------
// Gauss-Legendre rule on [0, 1] by Newton iteration on P_q (three-term
// recurrence), started from the Chebyshev-like guess cos(pi (i + 3/4)/(q + 1/2)).
struct GaussRule {
  std::vector<double> x, w;
};

inline GaussRule gauss_legendre01(int q) {
  GaussRule g;
  g.x.resize(q);
  g.w.resize(q);
  for (int i = 0; i < q; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (q + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= q; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      if (q == 1) { p1 = z; p0 = 1.0; }
      dp = q * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= q; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      if (q == 1) { p1 = z; p0 = 1.0; }
      dp = q * (z * p1 - p0) / (z * z - 1.0);
    }
    // node i of [-1,1] in decreasing order -> store increasing on [0,1]
    g.x[q - 1 - i] = 0.5 * (z + 1.0);
    g.w[q - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);  // 2/((1-z^2)P'^2) * 1/2
  }
  return g;
}

// ---------------------------------------------------------------------------
// Lagrange basis through the Gauss-Lobatto points of degree p on [0, 1],
// stored by monomial coefficients so derivatives of any order are exact.
struct Poly1D {
  int p = 0;
  std::vector<double> nodes;               // p + 1 GLL points
  std::vector<std::vector<double>> coef;   // coef[a][k] of xi^k

  explicit Poly1D(int deg) : p(deg) {
    nodes.assign(p + 1, 0.0);
    nodes[0] = 0.0;
    nodes[p] = 1.0;
    // interior GLL points: roots of P_p'(z) on (-1, 1), Newton on P_p' with
    // the derivative from the Legendre ODE: (1-z^2) P'' = 2 z P' - p(p+1) P
    for (int i = 1; i < p; ++i) {
      double z = -std::cos(M_PI * i / p);
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= p; ++k) {
          double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = pk;
        }
        double P = (p == 1) ? z : p1;
        double Pm1 = (p == 1) ? 1.0 : p0;
        double dP = p * (Pm1 - z * P) / (1.0 - z * z);
        double d2P = (2.0 * z * dP - p * (p + 1.0) * P) / (1.0 - z * z);
        double dz = dP / d2P;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      nodes[i] = 0.5 * (z + 1.0);
    }
    std::sort(nodes.begin(), nodes.end());
    coef.assign(p + 1, std::vector<double>(p + 1, 0.0));
    for (int a = 0; a <= p; ++a) {
      std::vector<double> c(1, 1.0);
      double den = 1.0;
      for (int b = 0; b <= p; ++b) {
        if (b == a) continue;
        std::vector<double> nc(c.size() + 1, 0.0);
        for (size_t k = 0; k < c.size(); ++k) {
          nc[k + 1] += c[k];
          nc[k] -= nodes[b] * c[k];
        }
        c.swap(nc);
        den *= nodes[a] - nodes[b];
      }
      for (int k = 0; k <= p; ++k) coef[a][k] = c[k] / den;
    }
  }

  // m-th derivative of l_a at xi
  double eval(int a, double xi, int m = 0) const {
    double s = 0.0;
    for (int k = p; k >= m; --k) {
      double f = 1.0;
      for (int j = 0; j < m; ++j) f *= (k - j);
      s = s * xi + coef[a][k] * f;
    }
    return s;
  }
};

// ---------------------------------------------------------------------------
// Level sets.  Omega = {phi < 0}.
struct LevelSet {
  int kind = 0;  // 0 sphere, 1 plane
  int d = 3;
  double c[3] = {0, 0, 0};
  double r = 0;
  double nrm[3] = {0, 0, 0};
  double off = 0;

  double phi(const double* x) const {
    if (kind == 0) {
      double s = 0.0;
      for (int k = 0; k < d; ++k) {
        double t = x[k] - c[k];
        s = (k == 0) ? t * t : s + t * t;
      }
      return std::sqrt(s) - r;
    }
    double s = 0.0;
    for (int k = 0; k < d; ++k) s = (k == 0) ? nrm[0] * x[0] : s + nrm[k] * x[k];
    return s - off;
  }

  void grad(const double* x, double* g) const {
    if (kind == 0) {
      double s = 0.0;
      for (int k = 0; k < d; ++k) {
        double t = x[k] - c[k];
        s = (k == 0) ? t * t : s + t * t;
      }
      double nr = std::sqrt(s);
      for (int k = 0; k < d; ++k) g[k] = (x[k] - c[k]) / nr;
      return;
    }
    for (int k = 0; k < d; ++k) g[k] = nrm[k];
  }

  // exact min / max of phi over a closed (possibly degenerate) box
  void box_minmax(const double* lo, const double* hi, double& mn, double& mx) const {
    if (kind == 0) {
      double s0 = 0.0, s1 = 0.0;
      for (int k = 0; k < d; ++k) {
        double a = lo[k] - c[k], b = hi[k] - c[k];
        double nearv = a > 0 ? a : (b < 0 ? -b : 0.0);
        double farv = std::max(std::fabs(a), std::fabs(b));
        s0 = s0 + nearv * nearv;
        s1 = s1 + farv * farv;
      }
      mn = std::sqrt(s0) - r;
      mx = std::sqrt(s1) - r;
      return;
    }
    mn = -off;
    mx = -off;
    for (int k = 0; k < d; ++k) {
      double u = nrm[k] * lo[k], v = nrm[k] * hi[k];
      mn += std::min(u, v);
      mx += std::max(u, v);
    }
  }

  // true when d phi / d x_k keeps one strict sign on the box
  bool monotone_in(int k, const double* lo, const double* hi) const {
    if (kind == 0) return c[k] < lo[k] || c[k] > hi[k];
    return nrm[k] != 0.0;
  }
};

// ---------------------------------------------------------------------------
// Cut-cell quadrature by dimension reduction.
//
// Fixed choices (one reading of a method whose parameters the paper leaves
// open): q Gauss points per sub-interval; height direction = free direction
// of largest |d phi/d x_k| at the box centre (ties to the lower k) among
// those where every current function is monotone; otherwise halve the box in
// all free directions, at most kMaxDepth times, after which the largest
// direction is used and roots are bracketed on 2q equal sub-intervals; a
// function without a zero on its box is dropped; roots by kBisect halvings.
constexpr int kMaxDepth = 4;
constexpr int kBisect = 64;

struct FixedCoords {  // a face restriction: coordinates pinned to values
  int n = 0;
  int dim[3];
  double val[3];
  void apply(double* x) const {
    for (int i = 0; i < n; ++i) x[dim[i]] = val[i];
  }
  FixedCoords with(int k, double v) const {
    FixedCoords f = *this;
    f.dim[f.n] = k;
    f.val[f.n] = v;
    f.n += 1;
    return f;
  }
};

struct Node {  // quadrature node in d <= 3 dimensions
  double x[3];
  double w;
};

struct CutRule {
  std::vector<Node> vol;
  std::vector<Node> surf;
  std::vector<std::array<double, 3>> normal;
};

class CutQuadrature {
 public:
  CutQuadrature(const LevelSet& ls, int q) : ls_(ls), q_(q), g_(gauss_legendre01(q)) {}

  CutRule cell(const double* lo, const double* hi) const {
    CutRule out;
    double L[3], H[3];
    for (int k = 0; k < 3; ++k) {
      L[k] = k < ls_.d ? lo[k] : 0.0;
      H[k] = k < ls_.d ? hi[k] : 0.0;
    }
    cell_rec(L, H, 0, out);
    return out;
  }

 private:
  const LevelSet& ls_;
  int q_;
  GaussRule g_;

  void fbox(const double* lo, const double* hi, const FixedCoords& f, double* blo,
            double* bhi) const {
    for (int k = 0; k < 3; ++k) {
      blo[k] = lo[k];
      bhi[k] = hi[k];
    }
    for (int i = 0; i < f.n; ++i) blo[f.dim[i]] = bhi[f.dim[i]] = f.val[i];
  }

  bool has_zero(const double* lo, const double* hi, const FixedCoords& f) const {
    double blo[3], bhi[3], mn, mx;
    fbox(lo, hi, f, blo, bhi);
    ls_.box_minmax(blo, bhi, mn, mx);
    return mn < 0.0 && 0.0 < mx;
  }

  // free directions ordered by |d phi/d x_k| at the centre of f's box
  std::vector<int> order(const double* lo, const double* hi, const std::vector<int>& freed,
                         const FixedCoords& f) const {
    double blo[3], bhi[3], ctr[3], g[3] = {0, 0, 0};
    fbox(lo, hi, f, blo, bhi);
    for (int k = 0; k < 3; ++k) ctr[k] = 0.5 * (blo[k] + bhi[k]);
    ls_.grad(ctr, g);
    std::vector<int> o = freed;
    std::stable_sort(o.begin(), o.end(), [&](int a, int b) {
      double ga = std::fabs(g[a]), gb = std::fabs(g[b]);
      if (ga != gb) return ga > gb;
      return a < b;
    });
    return o;
  }

  bool monotone_all(int k, const double* lo, const double* hi,
                    const std::vector<FixedCoords>& fs) const {
    for (const auto& f : fs) {
      double blo[3], bhi[3];
      fbox(lo, hi, f, blo, bhi);
      if (!ls_.monotone_in(k, blo, bhi)) return false;
    }
    return true;
  }

  double line_phi(const Node& base, const FixedCoords& f, int k, double t) const {
    double x[3] = {base.x[0], base.x[1], base.x[2]};
    f.apply(x);
    x[k] = t;
    return ls_.phi(x);
  }

  double bisect(const Node& base, const FixedCoords& f, int k, double a, double b,
                double ga) const {
    bool neg_a = ga < 0.0;
    for (int it = 0; it < kBisect; ++it) {
      double m = 0.5 * (a + b);
      double gm = line_phi(base, f, k, m);
      if (gm == 0.0) {
        a = m;
        b = m;
      } else if ((gm < 0.0) == neg_a) {
        a = m;
      } else {
        b = m;
      }
    }
    return 0.5 * (a + b);
  }

  // roots of t -> phi_f(base, t) in (a, b)
  void line_roots(const Node& base, const FixedCoords& f, int k, double a, double b,
                  bool monotone, std::vector<double>& roots) const {
    int nseg = monotone ? 1 : 2 * q_;
    for (int s = 0; s < nseg; ++s) {
      double ta = monotone ? a : a + ((b - a) * s) / (2 * q_);
      double tb = monotone ? b : (s + 1 == nseg ? b : a + ((b - a) * (s + 1)) / (2 * q_));
      double ga = line_phi(base, f, k, ta);
      double gb = line_phi(base, f, k, tb);
      if ((ga < 0.0 && gb > 0.0) || (ga > 0.0 && gb < 0.0))
        roots.push_back(bisect(base, f, k, ta, tb, ga));
    }
  }

  void tensor(const double* lo, const double* hi, const std::vector<int>& freed,
              std::vector<Node>& out) const {
    std::vector<Node> pts(1);
    pts[0] = Node{{0, 0, 0}, 1.0};
    for (int k : freed) {
      double len = hi[k] - lo[k];
      std::vector<Node> nxt;
      nxt.reserve(pts.size() * q_);
      for (const auto& P : pts)
        for (int i = 0; i < q_; ++i) {
          Node n = P;
          n.x[k] = lo[k] + len * g_.x[i];
          n.w = P.w * (g_.w[i] * len);
          nxt.push_back(n);
        }
      pts.swap(nxt);
    }
    out.insert(out.end(), pts.begin(), pts.end());
  }

  void children(const double* lo, const double* hi, const std::vector<int>& freed,
                std::vector<std::array<double, 6>>& kids) const {
    int nf = (int)freed.size();
    for (int bits = 0; bits < (1 << nf); ++bits) {
      std::array<double, 6> b;
      for (int k = 0; k < 3; ++k) {
        b[k] = lo[k];
        b[3 + k] = hi[k];
      }
      for (int i = 0; i < nf; ++i) {
        int k = freed[i];
        double mid = 0.5 * (lo[k] + hi[k]);
        if ((bits >> i) & 1)
          b[k] = mid;
        else
          b[3 + k] = mid;
      }
      kids.push_back(b);
    }
  }

  // rule over the free directions of the box, split at the zero sets of fs
  void base(const double* lo, const double* hi, const std::vector<int>& freed,
            const std::vector<FixedCoords>& fs, int depth, std::vector<Node>& out) const {
    std::vector<FixedCoords> kept;
    for (const auto& f : fs)
      if (has_zero(lo, hi, f)) kept.push_back(f);
    if (kept.empty()) {
      tensor(lo, hi, freed, out);
      return;
    }
    std::vector<int> ord = order(lo, hi, freed, kept[0]);
    int k = -1;
    for (int cand : ord)
      if (monotone_all(cand, lo, hi, kept)) {
        k = cand;
        break;
      }
    bool mono = k >= 0;
    if (!mono) {
      if (depth < kMaxDepth) {
        std::vector<std::array<double, 6>> kids;
        children(lo, hi, freed, kids);
        for (auto& b : kids) base(b.data(), b.data() + 3, freed, kept, depth + 1, out);
        return;
      }
      k = ord[0];
    }
    std::vector<int> sub;
    for (int j : freed)
      if (j != k) sub.push_back(j);
    std::vector<Node> bnodes;
    if (!sub.empty()) {
      std::vector<FixedCoords> sf;
      for (const auto& f : kept) {
        sf.push_back(f.with(k, lo[k]));
        sf.push_back(f.with(k, hi[k]));
      }
      base(lo, hi, sub, sf, depth, bnodes);
    } else {
      bnodes.push_back(Node{{0, 0, 0}, 1.0});
    }
    std::vector<double> roots;
    for (const auto& bn : bnodes) {
      roots.clear();
      for (const auto& f : kept) line_roots(bn, f, k, lo[k], hi[k], mono, roots);
      std::sort(roots.begin(), roots.end());
      double prev = lo[k];
      for (size_t i = 0; i <= roots.size(); ++i) {
        double nxt = i < roots.size() ? roots[i] : hi[k];
        double len = nxt - prev;
        for (int g = 0; g < q_; ++g) {
          Node n = bn;
          n.x[k] = prev + len * g_.x[g];
          n.w = bn.w * len * g_.w[g];
          out.push_back(n);
        }
        prev = nxt;
      }
    }
  }

  void cell_rec(const double* lo, const double* hi, int depth, CutRule& out) const {
    const int d = ls_.d;
    double mn, mx;
    ls_.box_minmax(lo, hi, mn, mx);
    if (mn >= 0.0) return;
    std::vector<int> all;
    for (int k = 0; k < d; ++k) all.push_back(k);
    if (mx <= 0.0) {
      tensor(lo, hi, all, out.vol);
      return;
    }
    FixedCoords none;
    std::vector<int> ord = order(lo, hi, all, none);
    int k = -1;
    for (int cand : ord)
      if (ls_.monotone_in(cand, lo, hi)) {
        k = cand;
        break;
      }
    bool mono = k >= 0;
    if (!mono) {
      if (depth < kMaxDepth) {
        std::vector<std::array<double, 6>> kids;
        children(lo, hi, all, kids);
        for (auto& b : kids) cell_rec(b.data(), b.data() + 3, depth + 1, out);
        return;
      }
      k = ord[0];
    }
    std::vector<int> sub;
    for (int j : all)
      if (j != k) sub.push_back(j);
    std::vector<FixedCoords> sf{none.with(k, lo[k]), none.with(k, hi[k])};
    std::vector<Node> bnodes;
    base(lo, hi, sub, sf, depth, bnodes);
    std::vector<double> roots;
    for (const auto& bn : bnodes) {
      roots.clear();
      line_roots(bn, none, k, lo[k], hi[k], mono, roots);
      std::sort(roots.begin(), roots.end());
      double prev = lo[k];
      for (size_t i = 0; i <= roots.size(); ++i) {
        double nxt = i < roots.size() ? roots[i] : hi[k];
        double mid[3] = {bn.x[0], bn.x[1], bn.x[2]};
        mid[k] = 0.5 * (prev + nxt);
        if (ls_.phi(mid) < 0.0) {
          double len = nxt - prev;
          for (int g = 0; g < q_; ++g) {
            Node n = bn;
            n.x[k] = prev + len * g_.x[g];
            n.w = bn.w * len * g_.w[g];
            out.vol.push_back(n);
          }
        }
        prev = nxt;
      }
      for (double t : roots) {
        Node s = bn;
        s.x[k] = t;
        double gr[3] = {0, 0, 0};
        ls_.grad(s.x, gr);
        double gn = 0.0;
        for (int j = 0; j < d; ++j) gn += gr[j] * gr[j];
        gn = std::sqrt(gn);
        s.w = bn.w * gn / std::fabs(gr[k]);
        out.surf.push_back(s);
        out.normal.push_back({gr[0] / gn, gr[1] / gn, d > 2 ? gr[2] / gn : 0.0});
      }
    }
  }
};

}  // namespace cutmg
