// presplit.cpp -- host-side (FP64) curve validation and pre-split for
// fiber_upload.
//
// Sec. 3.4: disjoint bounding volumes under recursive bisection need five
// inequalities on the control points (App. B.2 proves they suffice and are
// inherited by both halves); a curve violating them has to be split before
// it is traversed.  Thick fibers can still cross a partitioning plane;
// Sec. 3.4 reduces the test to the two end planes of a fiber (Fig. 7),
// checked here exactly on polynomials in the Bernstein basis.  Here a curve
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

// Polynomials on [0, 1] in the Bernstein basis of their degree (at most 10).
struct Bern {
  int n = 0;
  double b[11] = {0};
};

double choose(int n, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// (f g)_k = sum_{i + j = k} C(m, i) C(n, j) / C(m + n, k) f_i g_j
Bern product(const Bern& f, const Bern& g) {
  Bern r;
  r.n = f.n + g.n;
  for (int i = 0; i <= f.n; ++i)
    for (int j = 0; j <= g.n; ++j)
      r.b[i + j] += choose(f.n, i) * choose(g.n, j) / choose(r.n, i + j) * f.b[i] * g.b[j];
  return r;
}

// degree elevation to n
Bern raise(Bern f, int n) {
  while (f.n < n) {
    Bern r;
    r.n = f.n + 1;
    for (int k = 0; k <= r.n; ++k) {
      const double a = k > 0 ? f.b[k - 1] * k / r.n : 0.0;
      const double c = k < r.n ? f.b[k] * (r.n - k) / r.n : 0.0;
      r.b[k] = a + c;
    }
    f = r;
  }
  return f;
}

Bern combine(const Bern& f, double sf, const Bern& g, double sg) {
  const int n = std::max(f.n, g.n);
  const Bern a = raise(f, n), c = raise(g, n);
  Bern r;
  r.n = n;
  for (int k = 0; k <= n; ++k) r.b[k] = sf * a.b[k] + sg * c.b[k];
  return r;
}

// f = (1 - u) h for f vanishing at u = 1: (1 - u) B^{n-1}_i = (n - i) / n B^n_i
Bern div_one_minus_u(const Bern& f) {
  Bern h;
  h.n = f.n - 1;
  for (int i = 0; i <= h.n; ++i) h.b[i] = f.b[i] * f.n / (f.n - i);
  return h;
}

// f = u h for f vanishing at u = 0: u B^{n-1}_i = (i + 1) / n B^n_{i+1}
Bern div_u(const Bern& f) {
  Bern h;
  h.n = f.n - 1;
  for (int i = 0; i <= h.n; ++i) h.b[i] = f.b[i + 1] * f.n / (i + 1);
  return h;
}

// f >= 0 on [0, 1]: all coefficients >= 0 proves it (convex hull), a
// negative end value (b_0 or b_n) disproves it, otherwise both halves
// (de Casteljau at 1/2) are checked.  Coefficients within tol of zero count
// as zero; an undecided 40th halving counts as a violation.
bool nonneg(const double* b, int n, double tol, int depth) {
  if (b[0] < -tol || b[n] < -tol) return false;
  bool all = true;
  for (int k = 0; k <= n; ++k) all = all && b[k] >= -tol;
  if (all) return true;
  if (depth >= 40) return false;
  double w[11], L[11], R[11];
  std::memcpy(w, b, sizeof(double) * (n + 1));
  for (int lvl = 0; lvl <= n; ++lvl) {
    L[lvl] = w[0];
    R[n - lvl] = w[n - lvl];
    for (int k = 0; k + lvl < n; ++k) w[k] = 0.5 * (w[k] + w[k + 1]);
  }
  return nonneg(L, n, tol, depth + 1) && nonneg(R, n, tol, depth + 1);
}

bool nonneg01(const Bern& f) {
  double m = 0.0;
  for (int k = 0; k <= f.n; ++k) m = std::max(m, std::fabs(f.b[k]));
  return nonneg(f.b, f.n, 1e-12 * m, 0);
}

// End-plane check for thick fibers (Sec. 3.4, Fig. 7).  The cross-section at
// u reaches rbar sin(theta(u)) beyond c(u) towards an end plane, theta the
// angle between c'(u) and the plane's normal n (Gram-Schmidt displacement);
// rbar is the largest control radius.  The fiber is not cropped by the end
// plane through p3, n = p3 - p2, if D = <p3 - c(u), n> >= 0 and
// D^2 |t|^2 >= rbar^2 |n x t|^2 (t = c' / 3) for all u in [0, 1]: degree 3
// and 10 with a simple and a double root at u = 1, where the fiber meets its
// own end plane, which are divided out before both are checked
// non-negative; at u = 1 the second becomes rbar * curvature <= 1.  The
// start plane through p0, n = p1 - p0, likewise with the roots at u = 0.
bool thick_ok(const Curve& c) {
  double rbar = 0.0;
  for (const P4& p : c) rbar = std::max(rbar, p.v[3]);
  Bern tj[3];  // t = c' / 3: Bernstein coefficients p1 - p0, p2 - p1, p3 - p2
  for (int j = 0; j < 3; ++j) {
    tj[j].n = 2;
    for (int k = 0; k < 3; ++k) tj[j].b[k] = c[k + 1].v[j] - c[k].v[j];
  }
  Bern T;
  T.n = 4;
  for (int j = 0; j < 3; ++j) T = combine(T, 1.0, product(tj[j], tj[j]), 1.0);
  for (int e = 0; e < 2; ++e) {
    const P4 n = e == 0 ? sub(c[1], c[0]) : sub(c[3], c[2]);
    const double nn = dot(n, n);
    if (!(nn > 0.0)) return false;
    Bern D, G;  // D = <c - p0, n> (start) or <p3 - c, n> (end); G = <n, t>
    D.n = 3;
    G.n = 2;
    for (int k = 0; k < 4; ++k) D.b[k] = e == 0 ? dot(sub(c[k], c[0]), n) : dot(sub(c[3], c[k]), n);
    for (int k = 0; k < 3; ++k) G.b[k] = n.v[0] * tj[0].b[k] + n.v[1] * tj[1].b[k] + n.v[2] * tj[2].b[k];
    const Bern X = combine(T, nn, product(G, G), -1.0);  // |n x t|^2
    const Bern P = combine(product(product(D, D), T), 1.0, X, -rbar * rbar);
    const Bern E = e == 0 ? div_u(D) : div_one_minus_u(D);
    const Bern Q = e == 0 ? div_u(div_u(P)) : div_one_minus_u(div_one_minus_u(P));
    if (!nonneg01(E) || !nonneg01(Q)) return false;
  }
  return true;
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
