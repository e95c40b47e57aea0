// Built-in discrete direction sets (Sec. 3.2.1 of Weih et al. 2020).
//
// Every set is a list of unit vectors with weights summing to one.  The
// library keeps a canonical order so that populations can be exchanged
// index by index: 2D rings keep k = 0..N-1, 3D sets are sorted by the
// integer key (round(1e9 n_z), round(1e9 n_y), round(1e9 n_x)).  Components
// smaller than 1e-15 in magnitude are set to +0.0, so sgn(n) (with
// sgn(0) = +1) is exact.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <utility>

#include "lb_rt_internal.h"

namespace lbrt {
namespace {

using Vec = std::array<double, 3>;

double snap(double v) { return std::fabs(v) < 1e-15 ? 0.0 : v + 0.0; }

Vec unit(const Vec& v) {
  double r = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  return {v[0] / r, v[1] / r, v[2] / r};
}

void sort_canonical(std::vector<Vec>& pts, std::vector<double>& wts) {
  std::vector<size_t> idx(pts.size());
  for (size_t k = 0; k < idx.size(); ++k) idx[k] = k;
  auto key = [&](size_t k) {
    return std::array<long long, 3>{std::llround(pts[k][2] * 1e9), std::llround(pts[k][1] * 1e9),
                                    std::llround(pts[k][0] * 1e9)};
  };
  std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return key(a) < key(b); });
  std::vector<Vec> p2;
  std::vector<double> w2;
  for (size_t k : idx) {
    p2.push_back(pts[k]);
    w2.push_back(wts[k]);
  }
  pts.swap(p2);
  wts.swap(w2);
}

// N points on the unit circle at phi0 + 2 pi k / N.
void ring(int N, double phi0, std::vector<Vec>& pts, std::vector<double>& wts) {
  for (int k = 0; k < N; ++k) {
    double phi = phi0 + 2.0 * M_PI * k / N;
    pts.push_back({snap(std::cos(phi)), snap(std::sin(phi)), 0.0});
    wts.push_back(1.0 / N);
  }
}

// Icosahedron refined `level` times by 4-way splits at normalised edge midpoints.
void icosphere(int level, std::vector<Vec>& pts, std::vector<double>& wts) {
  const double p = 0.5 * (1.0 + std::sqrt(5.0));
  std::vector<Vec> v;
  // the 12 vertices are the cyclic permutations of (0, +-1, +-p)
  for (int s1 = -1; s1 <= 1; s1 += 2)
    for (int s2 = -1; s2 <= 1; s2 += 2) {
      v.push_back({0.0, (double)s1, s2 * p});
      v.push_back({(double)s1, s2 * p, 0.0});
      v.push_back({s2 * p, 0.0, (double)s1});
    }
  // faces: vertex triples pairwise at the edge length 2
  std::vector<std::array<int, 3>> faces;
  auto d2 = [&](int a, int b) {
    double s = 0;
    for (int c = 0; c < 3; ++c) s += (v[a][c] - v[b][c]) * (v[a][c] - v[b][c]);
    return s;
  };
  auto edge = [&](int a, int b) { double s = d2(a, b); return s > 3.5 && s < 4.5; };
  for (int a = 0; a < 12; ++a)
    for (int b = a + 1; b < 12; ++b)
      for (int c = b + 1; c < 12; ++c)
        if (edge(a, b) && edge(b, c) && edge(a, c)) faces.push_back({a, b, c});
  for (auto& q : v) q = unit(q);
  for (int l = 0; l < level; ++l) {
    std::map<std::pair<int, int>, int> mid;
    auto midpoint = [&](int a, int b) {
      auto key = std::make_pair(std::min(a, b), std::max(a, b));
      auto it = mid.find(key);
      if (it != mid.end()) return it->second;
      Vec m = unit({0.5 * (v[a][0] + v[b][0]), 0.5 * (v[a][1] + v[b][1]),
                    0.5 * (v[a][2] + v[b][2])});
      v.push_back(m);
      mid[key] = (int)v.size() - 1;
      return (int)v.size() - 1;
    };
    std::vector<std::array<int, 3>> nf;
    for (auto& f : faces) {
      int ab = midpoint(f[0], f[1]), bc = midpoint(f[1], f[2]), ca = midpoint(f[2], f[0]);
      nf.push_back({f[0], ab, ca});
      nf.push_back({f[1], bc, ab});
      nf.push_back({f[2], ca, bc});
      nf.push_back({ab, bc, ca});
    }
    faces.swap(nf);
  }
  for (auto& q : v) {
    pts.push_back({snap(q[0]), snap(q[1]), snap(q[2])});
    wts.push_back(1.0 / (double)v.size());
  }
  sort_canonical(pts, wts);
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int k = 0; k < n; ++k) {
    double z = std::cos(M_PI * (k + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      // p1 = P_n(z), p0 = P_{n-1}(z)
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        // recompute the derivative at the converged node
        p0 = 1.0;
        p1 = z;
        for (int j = 2; j <= n; ++j) {
          double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    x[k] = z;
    double p0 = 1.0, p1 = z;
    for (int j = 2; j <= n; ++j) {
      double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (z * p1 - p0) / (z * z - 1.0);
    w[k] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

void gl_product(int nt, int np, std::vector<Vec>& pts, std::vector<double>& wts) {
  std::vector<double> mu, wm;
  gauss_legendre(nt, mu, wm);
  for (int a = 0; a < nt; ++a) {
    double s = std::sqrt(std::max(0.0, 1.0 - mu[a] * mu[a]));
    for (int b = 0; b < np; ++b) {
      double phi = 2.0 * M_PI * (b + 0.5) / np;
      pts.push_back({snap(s * std::cos(phi)), snap(s * std::sin(phi)), snap(mu[a])});
      wts.push_back(wm[a] / 2.0 / np);
    }
  }
  sort_canonical(pts, wts);
}

}  // namespace

bool build_directions(const lb_rt_config& cfg, std::vector<double>& n, std::vector<double>& w,
                      std::string& err) {
  std::vector<Vec> pts;
  std::vector<double> wts;
  if (cfg.dirs) {
    if (cfg.ndir < 1 || cfg.ndir > LB_RT_MAX_DIRS) {
      err = "ndir out of range [1, LB_RT_MAX_DIRS]";
      return false;
    }
    for (int i = 0; i < cfg.ndir; ++i) {
      Vec q = {cfg.dirs[3 * i], cfg.dirs[3 * i + 1], cfg.dirs[3 * i + 2]};
      double r = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
      if (!(std::fabs(r - 1.0) < 1e-9)) {
        err = "custom direction is not a unit vector";
        return false;
      }
      pts.push_back({snap(q[0]), snap(q[1]), snap(q[2])});
      wts.push_back(cfg.weights ? cfg.weights[i] : 1.0 / cfg.ndir);
    }
  } else if (cfg.dirset == LB_RT_RING2D) {
    if (cfg.ndir < 3 || cfg.ndir > LB_RT_MAX_DIRS) {
      err = "ring: ndir must be in [3, LB_RT_MAX_DIRS]";
      return false;
    }
    ring(cfg.ndir, cfg.ring_offset, pts, wts);
  } else if (cfg.dirset == LB_RT_ICOSPHERE) {
    int level = cfg.dirset_param[0];
    if (level < 0 || level > 2) {
      err = "icosphere: level must be 0, 1 or 2";
      return false;
    }
    icosphere(level, pts, wts);
  } else if (cfg.dirset == LB_RT_GAUSS_LEGENDRE) {
    int nt = cfg.dirset_param[0], np = cfg.dirset_param[1];
    if (nt < 1 || np < 1 || nt * np > LB_RT_MAX_DIRS) {
      err = "gauss-legendre: need n_theta, n_phi >= 1 and n_theta*n_phi <= LB_RT_MAX_DIRS";
      return false;
    }
    gl_product(nt, np, pts, wts);
  } else {
    err = "unknown dirset";
    return false;
  }
  n.clear();
  w = wts;
  for (auto& q : pts) {
    n.push_back(q[0]);
    n.push_back(q[1]);
    n.push_back(q[2]);
  }
  return true;
}

}  // namespace lbrt
