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
// Closed intervals for bounds of level sets over boxes (plain floating point,
// no outward rounding).
struct Iv {
  double lo, hi;
};
inline Iv iv_add(Iv a, Iv b) { return {a.lo + b.lo, a.hi + b.hi}; }
inline Iv iv_sub(Iv a, Iv b) { return {a.lo - b.hi, a.hi - b.lo}; }
inline Iv iv_scale(double s, Iv a) {
  double u = s * a.lo, v = s * a.hi;
  return {std::min(u, v), std::max(u, v)};
}
inline Iv iv_mul(Iv a, Iv b) {
  double p0 = a.lo * b.lo, p1 = a.lo * b.hi, p2 = a.hi * b.lo, p3 = a.hi * b.hi;
  return {std::min(std::min(p0, p1), std::min(p2, p3)), std::max(std::max(p0, p1), std::max(p2, p3))};
}
inline Iv iv_sqr(Iv a) {
  double u = a.lo * a.lo, v = a.hi * a.hi;
  if (a.lo <= 0.0 && 0.0 <= a.hi) return {0.0, std::max(u, v)};
  return {std::min(u, v), std::max(u, v)};
}
inline Iv iv_sqrt(Iv a) { return {std::sqrt(std::max(a.lo, 0.0)), std::sqrt(std::max(a.hi, 0.0))}; }
inline Iv iv_div(Iv a, Iv b) { return iv_mul(a, Iv{1.0 / b.hi, 1.0 / b.lo}); }
inline Iv iv_cos(Iv a) {
  const double tp = 2.0 * M_PI;
  if (a.hi - a.lo >= tp) return {-1.0, 1.0};
  double c0 = std::cos(a.lo), c1 = std::cos(a.hi);
  double mn = std::min(c0, c1), mx = std::max(c0, c1);
  if (tp * std::ceil(a.lo / tp) <= a.hi) mx = 1.0;
  if (M_PI + tp * std::ceil((a.lo - M_PI) / tp) <= a.hi) mn = -1.0;
  return {mn, mx};
}
inline Iv iv_sin(Iv a) { return iv_cos(Iv{a.lo - 0.5 * M_PI, a.hi - 0.5 * M_PI}); }

// ---------------------------------------------------------------------------
// Level sets.  Omega = {phi < 0}.  Sphere and plane have exact box bounds;
// ellipsoid, torus (3D) and the flower curve (2D) use interval enclosures,
// refined by halving the box in every non-degenerate direction while the sign
// is undecided, at most kBoxDepth times (dyadic, so that nested cells keep
// nested classifications).
constexpr int kBoxDepth = 2;

// A user level set is known only through point values and gradients, so its
// bounds on a box come from samples: the lattice of kSampleIntervals + 1
// points per free direction (one in a degenerate direction).  Every box point
// lies within delta (half the diagonal of a lattice cell) of a sample, so
//   [min phi - L delta, max phi + L delta], L = largest sampled |grad phi|,
// encloses phi whenever L bounds |grad phi| on the box (distance functions:
// L = 1).  d phi / d x_k counts as one-signed when every sample has the same
// strict sign and the smallest |d phi / d x_k| exceeds C delta, C the largest
// difference quotient of d phi / d x_k between neighbouring samples.
constexpr int kSampleIntervals = 4;
constexpr int kMaxSamples = (kSampleIntervals + 1) * (kSampleIntervals + 1) * (kSampleIntervals + 1);

struct LevelSet {
  enum Kind { kSphere = 0, kPlane = 1, kEllipsoid = 2, kTorus = 3, kFlower = 4, kCallback = 5 };
  int kind = kSphere;
  int d = 3;
  double c[3] = {0, 0, 0};
  double r = 0;                 // sphere radius / torus minor radius / flower base radius
  double nrm[3] = {0, 0, 0};    // plane normal
  double off = 0;               // plane offset
  double ax[3] = {1, 1, 1};     // ellipsoid semi-axes
  double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};  // rotation (rows = body axes)
  double major = 0;             // torus major radius
  int lobes = 0;                // flower
  double amp = 0, phase = 0;    // flower
  double (*uphi)(const double*, void*) = nullptr;          // user level set: value at a 3-component point
  void (*ugrad)(const double*, double*, void*) = nullptr;  // user level set: gradient (3 components)
  void* user = nullptr;
  uint64_t epoch = 0;  // user level set: unique per setup, keys the per-thread sample cache

  double user_phi(const double* x) const {
    double p[3] = {x[0], d > 1 ? x[1] : 0.0, d > 2 ? x[2] : 0.0};
    return uphi(p, user);
  }
  void user_grad(const double* x, double* g) const {
    double p[3] = {x[0], d > 1 ? x[1] : 0.0, d > 2 ? x[2] : 0.0}, q[3] = {0.0, 0.0, 0.0};
    ugrad(p, q, user);
    for (int k = 0; k < d; ++k) g[k] = q[k];
  }

  struct Samples {
    int cnt[3] = {1, 1, 1};
    int n = 0;
    double delta = 0.0;
    double v[kMaxSamples];
    double g[kMaxSamples][3];
  };
  // samples in lexicographic order, the first direction fastest
  void sample_box(const double* lo, const double* hi, Samples& S) const {
    for (int k = 0; k < d; ++k) S.cnt[k] = hi[k] > lo[k] ? kSampleIntervals + 1 : 1;
    S.n = S.cnt[0] * S.cnt[1] * S.cnt[2];
    for (int i = 0; i < S.n; ++i) {
      int t = i, ik[3];
      for (int k = 0; k < 3; ++k) {
        ik[k] = t % S.cnt[k];
        t /= S.cnt[k];
      }
      double x[3] = {0.0, 0.0, 0.0};
      for (int k = 0; k < d; ++k) x[k] = lo[k] + (hi[k] - lo[k]) * ik[k] / kSampleIntervals;
      S.v[i] = user_phi(x);
      user_grad(x, S.g[i]);
    }
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
      double t = (hi[k] - lo[k]) / kSampleIntervals;
      s = (k == 0) ? t * t : s + t * t;
    }
    S.delta = 0.5 * std::sqrt(s);
  }
  // The quadrature bounds a box and then tests each direction on it: keep
  // the last few boxes' samples per thread.
  const Samples& samples(const double* lo, const double* hi) const {
    constexpr int kSlots = 8;
    struct Slot {
      uint64_t epoch = 0;
      double lo[3], hi[3];
      Samples S;
    };
    thread_local Slot slot[kSlots];
    thread_local int next = 0;
    for (int i = 0; i < kSlots; ++i) {
      Slot& e = slot[i];
      bool same = e.epoch == epoch;
      for (int k = 0; same && k < d; ++k) same = e.lo[k] == lo[k] && e.hi[k] == hi[k];
      if (same) return e.S;
    }
    Slot& e = slot[next];
    next = (next + 1) % kSlots;
    e.epoch = 0;
    sample_box(lo, hi, e.S);
    for (int k = 0; k < d; ++k) {
      e.lo[k] = lo[k];
      e.hi[k] = hi[k];
    }
    e.epoch = epoch;
    return e.S;
  }
  void sampled_minmax(const double* lo, const double* hi, double& mn, double& mx) const {
    const Samples& S = samples(lo, hi);
    double vmin = S.v[0], vmax = S.v[0], lip = 0.0;
    for (int i = 0; i < S.n; ++i) {
      vmin = std::min(vmin, S.v[i]);
      vmax = std::max(vmax, S.v[i]);
      double q = S.g[i][0] * S.g[i][0];
      for (int k = 1; k < d; ++k) q = q + S.g[i][k] * S.g[i][k];
      lip = std::max(lip, std::sqrt(q));
    }
    mn = vmin - lip * S.delta;
    mx = vmax + lip * S.delta;
  }
  bool sampled_monotone(int k, const double* lo, const double* hi) const {
    const Samples& S = samples(lo, hi);
    bool pos = true, neg = true;
    double gmin = 1e300;
    for (int i = 0; i < S.n; ++i) {
      const double gk = S.g[i][k];
      if (!(gk > 0.0)) pos = false;
      if (!(gk < 0.0)) neg = false;
      gmin = std::min(gmin, std::fabs(gk));
    }
    if (!pos && !neg) return false;
    double curv = 0.0;
    int stride = 1;
    for (int j = 0; j < d; ++j) {
      if (S.cnt[j] > 1) {
        const double step = (hi[j] - lo[j]) / kSampleIntervals;
        for (int i = 0; i < S.n; ++i)
          if ((i / stride) % S.cnt[j] < S.cnt[j] - 1)
            curv = std::max(curv, std::fabs(S.g[i + stride][k] - S.g[i][k]) / step);
      }
      stride *= S.cnt[j];
    }
    return gmin > curv * S.delta;
  }

  // body coordinates y = R (x - c)
  void body(const double* x, double* y) const {
    double dd[3] = {x[0] - c[0], x[1] - c[1], d > 2 ? x[2] - c[2] : 0.0};
    for (int i = 0; i < 3; ++i) y[i] = R[3 * i + 0] * dd[0] + R[3 * i + 1] * dd[1] + R[3 * i + 2] * dd[2];
  }

  double phi(const double* x) const {
    switch (kind) {
      case kCallback: return user_phi(x);
      case kSphere: {
        double s = 0.0;
        for (int k = 0; k < d; ++k) {
          double t = x[k] - c[k];
          s = (k == 0) ? t * t : s + t * t;
        }
        return std::sqrt(s) - r;
      }
      case kPlane: {
        double s = 0.0;
        for (int k = 0; k < d; ++k) s = (k == 0) ? nrm[0] * x[0] : s + nrm[k] * x[k];
        return s - off;
      }
      case kEllipsoid: {
        double y[3];
        body(x, y);
        double s = 0.0;
        for (int i = 0; i < 3; ++i) {
          double t = y[i] / ax[i];
          s = (i == 0) ? t * t : s + t * t;
        }
        return std::sqrt(s) - 1.0;
      }
      case kTorus: {
        double y[3];
        body(x, y);
        double rho = std::sqrt(y[0] * y[0] + y[1] * y[1]);
        double t = rho - major;
        return std::sqrt(t * t + y[2] * y[2]) - r;
      }
      default: {
        double dx = x[0] - c[0], dy = x[1] - c[1];
        double rho = std::sqrt(dx * dx + dy * dy), th = std::atan2(dy, dx);
        return rho - (r + amp * std::cos(lobes * (th - phase)));
      }
    }
  }

  void grad(const double* x, double* g) const {
    switch (kind) {
      case kCallback: user_grad(x, g); return;
      case kSphere: {
        double s = 0.0;
        for (int k = 0; k < d; ++k) {
          double t = x[k] - c[k];
          s = (k == 0) ? t * t : s + t * t;
        }
        double nr = std::sqrt(s);
        for (int k = 0; k < d; ++k) g[k] = (x[k] - c[k]) / nr;
        return;
      }
      case kPlane:
        for (int k = 0; k < d; ++k) g[k] = nrm[k];
        return;
      case kEllipsoid: {
        double y[3];
        body(x, y);
        double s = 0.0;
        for (int i = 0; i < 3; ++i) {
          double t = y[i] / ax[i];
          s = (i == 0) ? t * t : s + t * t;
        }
        double q = std::sqrt(s), gy[3];
        for (int i = 0; i < 3; ++i) gy[i] = y[i] / (ax[i] * ax[i]) / q;
        for (int j = 0; j < 3; ++j) g[j] = R[j] * gy[0] + R[3 + j] * gy[1] + R[6 + j] * gy[2];
        return;
      }
      case kTorus: {
        double y[3];
        body(x, y);
        double rho = std::sqrt(y[0] * y[0] + y[1] * y[1]);
        double t = rho - major;
        double q = std::sqrt(t * t + y[2] * y[2]);
        double gy[3] = {t / q * y[0] / rho, t / q * y[1] / rho, y[2] / q};
        for (int j = 0; j < 3; ++j) g[j] = R[j] * gy[0] + R[3 + j] * gy[1] + R[6 + j] * gy[2];
        return;
      }
      default: {
        double dx = x[0] - c[0], dy = x[1] - c[1];
        double r2 = dx * dx + dy * dy, rho = std::sqrt(r2), th = std::atan2(dy, dx);
        double s = amp * lobes * std::sin(lobes * (th - phase));
        g[0] = dx / rho - s * dy / r2;
        g[1] = dy / rho + s * dx / r2;
        return;
      }
    }
  }

  // exact min / max of |x - c| over a box
  void box_dist(const double* lo, const double* hi, double& dmin, double& dmax) const {
    double s0 = 0.0, s1 = 0.0;
    for (int k = 0; k < d; ++k) {
      double a = lo[k] - c[k], b = hi[k] - c[k];
      double nearv = a > 0 ? a : (b < 0 ? -b : 0.0);
      double farv = std::max(std::fabs(a), std::fabs(b));
      s0 = s0 + nearv * nearv;
      s1 = s1 + farv * farv;
    }
    dmin = std::sqrt(s0);
    dmax = std::sqrt(s1);
  }

  void body_iv(const double* lo, const double* hi, Iv* y) const {
    Iv D[3] = {{lo[0] - c[0], hi[0] - c[0]}, {lo[1] - c[1], hi[1] - c[1]}, {lo[2] - c[2], hi[2] - c[2]}};
    for (int i = 0; i < 3; ++i) {
      Iv t = iv_scale(R[3 * i + 0], D[0]);
      t = iv_add(t, iv_scale(R[3 * i + 1], D[1]));
      t = iv_add(t, iv_scale(R[3 * i + 2], D[2]));
      y[i] = t;
    }
  }

  bool flower_contains_c(const double* lo, const double* hi) const {
    return lo[0] <= c[0] && c[0] <= hi[0] && lo[1] <= c[1] && c[1] <= hi[1];
  }
  // range of the polar angle over a box not containing c
  Iv flower_theta(const double* lo, const double* hi) const {
    double xs[2] = {lo[0] - c[0], hi[0] - c[0]}, ys[2] = {lo[1] - c[1], hi[1] - c[1]};
    bool wrap = xs[1] < 0.0 && ys[0] <= 0.0 && 0.0 <= ys[1];
    double mn = 1e300, mx = -1e300;
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        double a = std::atan2(ys[j], xs[i]);
        if (wrap && a < 0.0) a += 2.0 * M_PI;
        mn = std::min(mn, a);
        mx = std::max(mx, a);
      }
    return {mn, mx};
  }

  void natural(const double* lo, const double* hi, double& mn, double& mx) const {
    if (kind == kEllipsoid) {
      Iv y[3];
      body_iv(lo, hi, y);
      Iv s = iv_sqr(iv_scale(1.0 / ax[0], y[0]));
      s = iv_add(s, iv_sqr(iv_scale(1.0 / ax[1], y[1])));
      s = iv_add(s, iv_sqr(iv_scale(1.0 / ax[2], y[2])));
      Iv q = iv_sqrt(s);
      mn = q.lo - 1.0;
      mx = q.hi - 1.0;
    } else if (kind == kTorus) {
      Iv y[3];
      body_iv(lo, hi, y);
      Iv rho = iv_sqrt(iv_add(iv_sqr(y[0]), iv_sqr(y[1])));
      Iv t{rho.lo - major, rho.hi - major};
      Iv q = iv_sqrt(iv_add(iv_sqr(t), iv_sqr(y[2])));
      mn = q.lo - r;
      mx = q.hi - r;
    } else {  // flower
      double dmin, dmax;
      box_dist(lo, hi, dmin, dmax);
      Iv cw{-1.0, 1.0};
      if (!flower_contains_c(lo, hi)) {
        Iv th = flower_theta(lo, hi);
        cw = iv_cos(Iv{lobes * (th.lo - phase), lobes * (th.hi - phase)});
      }
      mn = dmin - (r + amp * cw.hi);
      mx = dmax - (r + amp * cw.lo);
    }
  }

  void refined(const double* lo, const double* hi, int depth, double& mn, double& mx) const {
    natural(lo, hi, mn, mx);
    if (!(mn < 0.0 && 0.0 < mx) || depth >= kBoxDepth) return;
    int freed[3], nf = 0;
    for (int k = 0; k < d; ++k)
      if (hi[k] > lo[k]) freed[nf++] = k;
    mn = 1e300;
    mx = -1e300;
    for (int bits = 0; bits < (1 << nf); ++bits) {
      double clo[3] = {lo[0], lo[1], lo[2]}, chi[3] = {hi[0], hi[1], hi[2]};
      for (int i = 0; i < nf; ++i) {
        int k = freed[i];
        double mid = 0.5 * (lo[k] + hi[k]);
        if ((bits >> i) & 1)
          clo[k] = mid;
        else
          chi[k] = mid;
      }
      double a, b;
      refined(clo, chi, depth + 1, a, b);
      mn = std::min(mn, a);
      mx = std::max(mx, b);
    }
  }

  // bounds of phi over a closed (possibly degenerate) box
  void box_minmax(const double* lo, const double* hi, double& mn, double& mx) const {
    if (kind == kSphere) {
      double dmin, dmax;
      box_dist(lo, hi, dmin, dmax);
      mn = dmin - r;
      mx = dmax - r;
      return;
    }
    if (kind == kPlane) {
      mn = -off;
      mx = -off;
      for (int k = 0; k < d; ++k) {
        double u = nrm[k] * lo[k], v = nrm[k] * hi[k];
        mn += std::min(u, v);
        mx += std::max(u, v);
      }
      return;
    }
    if (kind == kCallback) {
      sampled_minmax(lo, hi, mn, mx);
      return;
    }
    refined(lo, hi, 0, mn, mx);
  }

  // true when d phi / d x_k provably keeps one strict sign on the box
  bool monotone_in(int k, const double* lo, const double* hi) const {
    switch (kind) {
      case kCallback: return sampled_monotone(k, lo, hi);
      case kSphere: return c[k] < lo[k] || c[k] > hi[k];
      case kPlane: return nrm[k] != 0.0;
      case kEllipsoid: {
        Iv y[3];
        body_iv(lo, hi, y);
        Iv t = iv_scale(R[k] / (ax[0] * ax[0]), y[0]);
        t = iv_add(t, iv_scale(R[3 + k] / (ax[1] * ax[1]), y[1]));
        t = iv_add(t, iv_scale(R[6 + k] / (ax[2] * ax[2]), y[2]));
        return t.lo > 0.0 || t.hi < 0.0;
      }
      case kTorus: {
        Iv y[3];
        body_iv(lo, hi, y);
        Iv rho2 = iv_add(iv_sqr(y[0]), iv_sqr(y[1]));
        if (rho2.lo <= 0.0) return false;
        Iv rho = iv_sqrt(rho2);
        Iv t{rho.lo - major, rho.hi - major};
        Iv w = iv_add(iv_scale(R[k], y[0]), iv_scale(R[3 + k], y[1]));
        Iv a = iv_mul(iv_div(t, rho), w);
        Iv sm = iv_add(a, iv_scale(R[6 + k], y[2]));
        return sm.lo > 0.0 || sm.hi < 0.0;
      }
      default: {
        if (flower_contains_c(lo, hi)) return false;
        Iv dx{lo[0] - c[0], hi[0] - c[0]}, dy{lo[1] - c[1], hi[1] - c[1]};
        double dmin, dmax;
        box_dist(lo, hi, dmin, dmax);
        Iv th = flower_theta(lo, hi);
        Iv sw = iv_scale(amp * lobes, iv_sin(Iv{lobes * (th.lo - phase), lobes * (th.hi - phase)}));
        Iv rho{dmin, dmax};
        Iv v = (k == 0) ? iv_sub(iv_mul(dx, rho), iv_mul(sw, dy)) : iv_add(iv_mul(dy, rho), iv_mul(sw, dx));
        return v.lo > 0.0 || v.hi < 0.0;
      }
    }
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
