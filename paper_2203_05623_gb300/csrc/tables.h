// Host-side tables of the plane-wave spheres and FFT plans (no device code).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "common.cuh"

namespace wgw {

// A plane-wave sphere 0.5|G|^2 <= ecut of a cubic cell, in canonical order
// (ascending h^2+k^2+l^2, then (h, k, l) lexicographically), with its
// real-basis pairing and the per-plane grid tables described in common.cuh.
// The real basis (internal to the library) numbers the pairs plane by plane: positive
// members in ascending (h, k, l), so that the points of one plane h are a contiguous range
// of real-basis elements and the plane kernels read and write them coalesced.
struct SphereHostTables {
  int n = 0;                 // plane waves
  int n_pairs = 0;           // positive members
  int i0 = -1;               // canonical index of G = 0
  int m = 0;                 // max |Miller component|
  int npt_max = 0;           // most entries of a plane h != 0
  std::vector<int> miller;   // 3 n, canonical order
  std::vector<int> pos, neg; // n_pairs + 1, [0] = i0
  std::vector<int> plane_off;
  std::vector<int2> ent;
  std::vector<double> g2;    // 0.5 |G|^2 per real-basis element
  std::vector<float> g2f;    // g2 rounded to FP32
  std::vector<double> vsqrt; // sqrt(4 pi)/|G| per canonical index (0 at G = 0)
  int nrb() const { return 2 * n_pairs + 1; }
};

inline bool positive_member(int h, int k, int l) {
  return h > 0 || (h == 0 && (k > 0 || (k == 0 && l > 0)));
}

inline void build_sphere(double L, double ecut, int N, SphereHostTables& s) {
  const double b = 2.0 * M_PI / L;
  const int M = (int)std::floor(std::sqrt(2.0 * ecut) / b) + 1;
  struct P { int n2, h, k, l; };
  std::vector<P> pts;
  for (int h = -M; h <= M; ++h)
    for (int k = -M; k <= M; ++k)
      for (int l = -M; l <= M; ++l) {
        const int n2 = h * h + k * k + l * l;
        if (0.5 * b * b * n2 <= ecut * (1.0 + 1e-12)) pts.push_back({n2, h, k, l});
      }
  std::sort(pts.begin(), pts.end(), [](const P& a, const P& c) {
    if (a.n2 != c.n2) return a.n2 < c.n2;
    if (a.h != c.h) return a.h < c.h;
    if (a.k != c.k) return a.k < c.k;
    return a.l < c.l;
  });
  s.n = (int)pts.size();
  s.miller.resize(3 * s.n);
  s.m = 0;
  for (int i = 0; i < s.n; ++i) {
    s.miller[3 * i] = pts[i].h; s.miller[3 * i + 1] = pts[i].k; s.miller[3 * i + 2] = pts[i].l;
    s.m = std::max(s.m, std::max(std::abs(pts[i].h), std::max(std::abs(pts[i].k), std::abs(pts[i].l))));
  }
  const int span = 2 * M + 1;
  std::vector<int> where((size_t)span * span * span, -1);
  auto key = [&](int h, int k, int l) { return ((size_t)(h + M) * span + (k + M)) * span + (l + M); };
  for (int i = 0; i < s.n; ++i) where[key(pts[i].h, pts[i].k, pts[i].l)] = i;
  s.pos.assign(1, 0);
  s.neg.assign(1, 0);
  std::vector<int> posi;
  for (int i = 0; i < s.n; ++i) {
    if (pts[i].n2 == 0) s.i0 = i;
    if (positive_member(pts[i].h, pts[i].k, pts[i].l)) posi.push_back(i);
  }
  std::sort(posi.begin(), posi.end(), [&](int a, int c) {
    if (pts[a].h != pts[c].h) return pts[a].h < pts[c].h;
    if (pts[a].k != pts[c].k) return pts[a].k < pts[c].k;
    return pts[a].l < pts[c].l;
  });
  for (int i : posi) {
    s.pos.push_back(i);
    s.neg.push_back(where[key(-pts[i].h, -pts[i].k, -pts[i].l)]);
  }
  s.pos[0] = s.neg[0] = s.i0;
  s.n_pairs = (int)s.pos.size() - 1;
  s.g2.assign(s.nrb(), 0.0);
  for (int j = 1; j <= s.n_pairs; ++j) s.g2[2 * j - 1] = s.g2[2 * j] = 0.5 * b * b * pts[s.pos[j]].n2;
  s.g2f.assign(s.g2.begin(), s.g2.end());
  s.vsqrt.assign(s.n, 0.0);
  for (int i = 0; i < s.n; ++i)
    if (pts[i].n2 > 0) s.vsqrt[i] = std::sqrt(4.0 * M_PI) / (b * std::sqrt((double)pts[i].n2));
  const int NP = 2 * s.m + 1;
  std::vector<std::vector<int2>> planes(NP);
  auto enc = [&](int k, int l, int ng) {
    return (int)(((k % N + N) % N) | (((l % N + N) % N) << 8) | (ng << 16));
  };
  planes[s.m].push_back(make_int2(enc(0, 0, 0), 0));
  std::vector<int2> mirrors0;
  for (int j = 1; j <= s.n_pairs; ++j) {
    const P& g = pts[s.pos[j]];
    if (g.h == 0) {
      planes[s.m].push_back(make_int2(enc(g.k, g.l, 0), j));
      mirrors0.push_back(make_int2(enc(-g.k, -g.l, 1), j));
    } else {
      planes[s.m + g.h].push_back(make_int2(enc(g.k, g.l, 0), j));
      planes[s.m - g.h].push_back(make_int2(enc(-g.k, -g.l, 1), j));
    }
  }
  for (const int2& e : mirrors0) planes[s.m].push_back(e);
  s.plane_off.assign(NP + 1, 0);
  s.ent.clear();
  s.npt_max = 0;
  for (int hi = 0; hi < NP; ++hi) {
    s.plane_off[hi] = (int)s.ent.size();
    for (const int2& e : planes[hi]) s.ent.push_back(e);
    if (hi != s.m) s.npt_max = std::max(s.npt_max, (int)planes[hi].size());
  }
  s.plane_off[NP] = (int)s.ent.size();
}

// Radices 8, 4, 2, 3, 5 (greedy, in that order of preference); false if n does not factor.
inline bool make_plan(int n, FftPlan& p) {
  p.n = n;
  p.nst = 0;
  int r = n;
  const int order[] = {8, 4, 2, 3, 5};
  while (r > 1) {
    bool found = false;
    for (int f : order) {
      if (r % f == 0) {
        if (p.nst >= 6) return false;
        p.radix[p.nst++] = f;
        r /= f;
        found = true;
        break;
      }
    }
    if (!found) return false;
  }
  return p.nst > 0;
}

}  // namespace wgw
