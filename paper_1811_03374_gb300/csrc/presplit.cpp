// presplit.cpp -- host-side (FP64) curve validation and pre-split for
// fiber_upload.
//
// Sec. 3.4: disjoint bounding volumes under recursive bisection need five
// inequalities on the control points (App. B.2 proves they suffice and are
// inherited by both halves); curves violating them "must be subdivided
// beforehand".  Thick fibers can still cross a partitioning plane; Sec. 3.4
// reduces the test to the two end planes of a fiber (Fig. 7).  Here a curve
// failing either test is halved at u = 1/2 recursively, left half first, up
// to a maximum level; pieces still failing at that level are kept and marked
// unsupported.  Each piece is stored as its (p, d, t0, t1) tuple (Sec. 3.1),
// differences formed in FP64 before rounding to FP32.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "presplit.h"

namespace fx {
namespace {

struct P4 {
  double v[4];  // x, y, z, r
};

inline double dot(const P4& a, const P4& b) { return a.v[0] * b.v[0] + a.v[1] * b.v[1] + a.v[2] * b.v[2]; }
inline P4 sub(const P4& a, const P4& b) {
  return P4{{a.v[0] - b.v[0], a.v[1] - b.v[1], a.v[2] - b.v[2], a.v[3] - b.v[3]}};
}
inline P4 axpy(double s, const P4& a, const P4& b) {  // s a + b
  return P4{{s * a.v[0] + b.v[0], s * a.v[1] + b.v[1], s * a.v[2] + b.v[2], s * a.v[3] + b.v[3]}};
}
inline double len(const P4& a) { return std::sqrt(dot(a, a)); }

using Curve = std::array<P4, 4>;

// The five inequalities of Sec. 3.4 (positions only).
bool constraints_hold(const Curve& c) {
  const P4 a = sub(c[2], c[0]), b = sub(c[1], c[0]), e = sub(c[3], c[1]), f = sub(c[3], c[2]);
  return dot(a, b) >= 0.0 && dot(e, b) >= 0.0 && dot(e, f) >= 0.0 && dot(a, f) >= 0.0 &&
         dot(a, e) >= 0.0;
}

P4 point_at(const Curve& c, double u) {
  const double s = 1.0 - u;
  const double w0 = s * s * s, w1 = 3.0 * u * s * s, w2 = 3.0 * u * u * s, w3 = u * u * u;
  P4 r;
  for (int k = 0; k < 4; ++k) r.v[k] = w0 * c[0].v[k] + w1 * c[1].v[k] + w2 * c[2].v[k] + w3 * c[3].v[k];
  return r;
}

// Tangent direction (c'(u) up to the factor 3).
P4 tangent_at(const Curve& c, double u) {
  const double s = 1.0 - u;
  P4 r;
  for (int k = 0; k < 4; ++k)
    r.v[k] = s * s * (c[1].v[k] - c[0].v[k]) + 2.0 * u * s * (c[2].v[k] - c[1].v[k]) +
             u * u * (c[3].v[k] - c[2].v[k]);
  return r;
}

// Curvature |c' x c''| / |c'|^3 at u.
double curvature_at(const Curve& c, double u) {
  const P4 t = tangent_at(c, u);
  double d1[3], d2[3];
  for (int k = 0; k < 3; ++k) {
    d1[k] = 3.0 * t.v[k];
    const double a = c[2].v[k] - 2.0 * c[1].v[k] + c[0].v[k];
    const double b = c[3].v[k] - 2.0 * c[2].v[k] + c[1].v[k];
    d2[k] = 6.0 * ((1.0 - u) * a + u * b);
  }
  const double cx = d1[1] * d2[2] - d1[2] * d2[1], cy = d1[2] * d2[0] - d1[0] * d2[2],
               cz = d1[0] * d2[1] - d1[1] * d2[0];
  const double l = std::sqrt(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2]);
  return std::sqrt(cx * cx + cy * cy + cz * cz) / (l * l * l);
}

// Sampled end-plane check (Sec. 3.4, Fig. 7): the surface point of the
// cross-section at u closest to an end plane sits rbar * |sin(angle between
// c'(u) and the plane normal)| beyond c(u) towards it; the plane crops the
// fiber if that exceeds the distance of c(u) from the plane.  Samples
// u = i / 32, plus rbar * curvature < 1 at both ends.
constexpr int kThickSamples = 32;

bool thick_ok(const Curve& c) {
  double rbar = 0.0;
  for (const P4& p : c) rbar = std::max(rbar, p.v[3]);
  const P4 ts = tangent_at(c, 0.0), te = tangent_at(c, 1.0);
  const double ls = len(ts), le = len(te);
  if (!(ls > 0.0) || !(le > 0.0)) return false;
  for (int i = 0; i <= kThickSamples; ++i) {
    const double u = double(i) / kThickSamples;
    const P4 tu = tangent_at(c, u);
    const double lu = len(tu);
    if (!(lu > 0.0)) return false;
    const P4 cu = point_at(c, u);
    if (i < kThickSamples) {
      // end plane through p3 with normal te / le
      const double ct = dot(te, tu) / (le * lu);
      P4 g = axpy(-ct, P4{{tu.v[0] / lu, tu.v[1] / lu, tu.v[2] / lu, 0}},
                  P4{{te.v[0] / le, te.v[1] / le, te.v[2] / le, 0}});
      const double dist = dot(sub(c[3], cu), te) / le;
      if (dist < rbar * len(g)) return false;
    }
    if (i > 0) {
      const double ct = dot(ts, tu) / (ls * lu);
      P4 g = axpy(-ct, P4{{tu.v[0] / lu, tu.v[1] / lu, tu.v[2] / lu, 0}},
                  P4{{ts.v[0] / ls, ts.v[1] / ls, ts.v[2] / ls, 0}});
      const double dist = dot(sub(cu, c[0]), ts) / ls;
      if (dist < rbar * len(g)) return false;
    }
  }
  return rbar * curvature_at(c, 0.0) < 1.0 && rbar * curvature_at(c, 1.0) < 1.0;
}

// De Casteljau at u = 1/2.
void halve(const Curve& c, Curve& L, Curve& R) {
  for (int k = 0; k < 4; ++k) {
    const double a = c[0].v[k], b = c[1].v[k], e = c[2].v[k], f = c[3].v[k];
    const double ab = 0.5 * (a + b), be = 0.5 * (b + e), ef = 0.5 * (e + f);
    const double abe = 0.5 * (ab + be), bef = 0.5 * (be + ef), m = 0.5 * (abe + bef);
    L[0].v[k] = a; L[1].v[k] = ab; L[2].v[k] = abe; L[3].v[k] = m;
    R[0].v[k] = m; R[1].v[k] = bef; R[2].v[k] = ef; R[3].v[k] = f;
  }
}

// Radius of a sphere about the chord midpoint p0 + d/2 that holds the root
// node's capped cylinder: the points within rc of the chord line between the
// start plane (through p0, normal t0) and the end plane (through p0 + d,
// normal t1).  Along the axis a point at distance q <= rc from it reaches at
// most rc |t_perp| / <d^, t> past an end plane's foot, so the region lies in
// the capsule a in [-e0, |d| + e1] x radius rc.  An end plane that does not
// face along the chord leaves the region unbounded: +inf.  Rounded up in
// FP32 with a relative margin for the kernel's FP32 evaluation.
float capped_bound(const P4& d, const P4& t0, const P4& t1, double rc) {
  const double L = std::sqrt(dot(d, d));
  if (!(L > 0.0)) return INFINITY;
  const double a0 = dot(d, t0) / L, a1 = dot(d, t1) / L;  // tangent components along the chord
  if (!(a0 > 0.0) || !(a1 > 0.0)) return INFINITY;
  const double p0 = std::sqrt(std::max(0.0, dot(t0, t0) - a0 * a0));
  const double p1 = std::sqrt(std::max(0.0, dot(t1, t1) - a1 * a1));
  const double e0 = rc * p0 / a0, e1 = rc * p1 / a1;
  const double h = 0.5 * L + std::max(e0, e1);
  const double R = std::sqrt(h * h + rc * rc) * (1.0 + 1e-6);
  const float f = (float)R;
  return (double)f >= R ? f : std::nextafter(f, INFINITY);
}

void emit(const Curve& c, int level, int off, bool ok, std::vector<PieceRec>& out) {
  PieceRec p;
  const P4 d = sub(c[3], c[0]), t0 = sub(c[1], c[0]), t1 = sub(c[3], c[2]);
  for (int k = 0; k < 4; ++k) {
    p.pdt[0 + k] = (float)c[0].v[k];
    p.pdt[4 + k] = (float)d.v[k];
    p.pdt[8 + k] = (float)t0.v[k];
    p.pdt[12 + k] = (float)t1.v[k];
  }
  // conservative radius of the whole piece: the inner control points'
  // distance from the chord plus the largest control radius (Sec. 3.3); a
  // rigid motion leaves it unchanged, so it is the same in every ray frame
  const double dd = dot(d, d);
  double m = 0.0;
  for (const P4* q : {&t0, &t1}) {
    double l2 = dot(*q, *q);
    if (dd > 0.0) {
      const double b = dot(*q, d) / dd;
      const P4 r = axpy(-b, d, *q);
      l2 = dot(r, r);
    }
    m = std::max(m, l2);
  }
  double rmax = 0.0;
  for (const P4& cpk : c) rmax = std::max(rmax, cpk.v[3]);
  const double rc = std::sqrt(m) + rmax;
  p.root_radius = (float)rc;
  p.bound_radius = capped_bound(d, t0, t1, rc * (1.0 + 1e-6));
  p.level = level;
  p.off = off;
  p.unsupported = !ok;
  out.push_back(p);
}

void split_rec(const Curve& c, int level, int off, int max_level, bool thick,
               std::vector<PieceRec>& out) {
  const bool ok = constraints_hold(c) && (!thick || thick_ok(c));
  if (ok || level >= max_level) {
    emit(c, level, off, ok, out);
    return;
  }
  Curve L, R;
  halve(c, L, R);
  split_rec(L, level + 1, 2 * off, max_level, thick, out);
  split_rec(R, level + 1, 2 * off + 1, max_level, thick, out);
}

}  // namespace

void presplit_all(const double* cps, int64_t n_seg, int max_level, bool thick, int n_threads,
                  std::vector<PieceRec>& pieces, std::vector<int32_t>& begin) {
  if (n_threads < 1) n_threads = 1;
  const int64_t per = (n_seg + n_threads - 1) / std::max(1, n_threads);
  std::vector<std::vector<PieceRec>> parts(n_threads);
  std::vector<std::vector<int32_t>> counts(n_threads);
  auto work = [&](int t) {
    const int64_t lo = t * per, hi = std::min(n_seg, lo + per);
    for (int64_t s = lo; s < hi; ++s) {
      Curve c;
      for (int k = 0; k < 4; ++k)
        for (int a = 0; a < 4; ++a) c[k].v[a] = cps[16 * s + 4 * k + a];
      const size_t before = parts[t].size();
      split_rec(c, 0, 0, max_level, thick, parts[t]);
      counts[t].push_back((int32_t)(parts[t].size() - before));
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < n_threads; ++t) th.emplace_back(work, t);
  work(0);
  for (auto& x : th) x.join();
  pieces.clear();
  begin.assign(1, 0);
  for (int t = 0; t < n_threads; ++t) {
    pieces.insert(pieces.end(), parts[t].begin(), parts[t].end());
    for (int32_t n : counts[t]) begin.push_back(begin.back() + n);
  }
}

}  // namespace fx
