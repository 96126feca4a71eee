// Device geometry for constrained Delaunay refinement on sm_103a.
//
// Exact predicates (the paper decides every geometric test exactly and breaks
// ties by simulation of simplicity, Sec. 7 set-up):
//   orient(a,b,c)      > 0  iff a,b,c counter-clockwise
//   incircle(a,b,c,d)  > 0  iff d strictly inside the circle of CCW a,b,c
//   dot(a,b;p) = (a-p).(b-p) < 0 iff p strictly inside the diametral circle of ab
//                            (p encroaches ab, Sec. 4.2, Ruppert's rule)
// Each predicate first evaluates a binary64 value with a forward error bound
// derived for that exact evaluation order (explicit _rn intrinsics: no
// contraction); only when the sign is not certain does it sum the
// determinant exactly as a floating-point expansion (error-free two-sum /
// two-product transformations and zero-eliminating expansion growth, after
// Shewchuk's published method).
//
// The FP64 geometry (bad-triangle test, circumcentre, midpoint, priority
// measure) follows a fixed evaluation order on a canonical vertex rotation
// so that every implementation of the same formulas agrees bit for bit.
#pragma once
#include <cstdint>

#define GDP_HD __host__ __device__ __forceinline__

namespace gdp {

constexpr double kU = 1.1102230246251565e-16;   // 2^-53
constexpr double kTiny = 1e-250;                // below: relative bounds unsafe -> exact

// ---------------------------------------------------------------- EFTs
__device__ __forceinline__ void two_sum(double a, double b, double& x, double& y) {
  x = __dadd_rn(a, b);
  double bv = __dsub_rn(x, a);
  double av = __dsub_rn(x, bv);
  y = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}
__device__ __forceinline__ void two_diff(double a, double b, double& x, double& y) {
  x = __dsub_rn(a, b);
  double bv = __dsub_rn(a, x);
  double av = __dadd_rn(x, bv);
  y = __dadd_rn(__dsub_rn(a, av), __dsub_rn(bv, b));
}
__device__ __forceinline__ void fast_two_sum(double a, double b, double& x, double& y) {
  x = __dadd_rn(a, b);
  y = __dsub_rn(b, __dsub_rn(x, a));
}
__device__ __forceinline__ void two_prod(double a, double b, double& x, double& y) {
  x = __dmul_rn(a, b);
  y = __fma_rn(a, b, -x);
}

// A nonoverlapping expansion with components in increasing magnitude.
template <int N>
struct Expansion {
  double e[N];
  int n = 0;
  __device__ __forceinline__ void grow(double b) {   // this += b, zero-eliminating
    if (b == 0.0) return;
    double q = b;
    int k = 0;
    for (int i = 0; i < n; ++i) {
      double h;
      two_sum(q, e[i], q, h);
      if (h != 0.0 && k < N - 1) e[k++] = h;   // k < N-1 keeps room for q (bounded range)
    }
    if (q != 0.0) e[k++] = q;
    n = k;
  }
  __device__ void compress() {                         // renormalise to few components
    if (n < 2) return;
    double g[N];
    int bottom = n - 1;
    double q = e[n - 1];
    for (int i = n - 2; i >= 0; --i) {
      double big, small;
      fast_two_sum(q, e[i], big, small);
      if (small != 0.0) {
        g[bottom--] = big;
        q = small;
      } else {
        q = big;
      }
    }
    g[bottom] = q;
    int top = 0;
    for (int i = bottom + 1; i < n; ++i) {
      double big, small;
      fast_two_sum(g[i], q, big, small);
      if (small != 0.0) e[top++] = small;
      q = big;
    }
    e[top++] = q;
    n = top;
    // drop zeros that compression can leave at the bottom
    int k = 0;
    for (int i = 0; i < n; ++i)
      if (e[i] != 0.0) e[k++] = e[i];
    n = k;
  }
  __device__ __forceinline__ int sign() const {
    if (n == 0) return 0;
    return e[n - 1] > 0.0 ? 1 : (e[n - 1] < 0.0 ? -1 : 0);
  }
};

// exact (a_h + a_l) * (b_h + b_l) added into X, times s (s = +-1 or +-2)
template <int N>
__device__ __forceinline__ void add_prod2(Expansion<N>& X, double ah, double al, double bh,
                                          double bl, double s) {
  double x, y;
  if (s != 1.0) { ah = __dmul_rn(ah, s); al = __dmul_rn(al, s); }   // exact: power of two
  two_prod(ah, bh, x, y); X.grow(y); X.grow(x);
  if (bl != 0.0) { two_prod(ah, bl, x, y); X.grow(y); X.grow(x); }
  if (al != 0.0) { two_prod(al, bh, x, y); X.grow(y); X.grow(x); }
  if (al != 0.0 && bl != 0.0) { two_prod(al, bl, x, y); X.grow(y); X.grow(x); }
}

// ---------------------------------------------------------------- orient
static __device__ __noinline__ int orient_exact(double ax, double ay, double bx, double by, double cx,
                                         double cy) {
  // (ax-cx)(by-cy) - (ay-cy)(bx-cx) with each difference as an exact pair
  double acxh, acxl, acyh, acyl, bcxh, bcxl, bcyh, bcyl;
  two_diff(ax, cx, acxh, acxl);
  two_diff(ay, cy, acyh, acyl);
  two_diff(bx, cx, bcxh, bcxl);
  two_diff(by, cy, bcyh, bcyl);
  Expansion<24> X;
  add_prod2(X, acxh, acxl, bcyh, bcyl, 1.0);
  add_prod2(X, acyh, acyl, bcxh, bcxl, -1.0);
  return X.sign();
}

__device__ __forceinline__ int orient(double ax, double ay, double bx, double by, double cx,
                                      double cy) {
  double l = __dmul_rn(__dsub_rn(ax, cx), __dsub_rn(by, cy));
  double r = __dmul_rn(__dsub_rn(ay, cy), __dsub_rn(bx, cx));
  double det = __dsub_rn(l, r);
  double perm = __dadd_rn(fabs(l), fabs(r));
  // three roundings in each product, one in the difference: |err| <= 4u perm + O(u^2)
  double bound = __dmul_rn(4.5 * kU, perm);
  if (perm > kTiny) {
    if (det > bound) return 1;
    if (-det > bound) return -1;
  }
  return orient_exact(ax, ay, bx, by, cx, cy);
}

__device__ __forceinline__ int orient(double2 a, double2 b, double2 c) {
  return orient(a.x, a.y, b.x, b.y, c.x, c.y);
}

// ---------------------------------------------------------------- incircle
// det = alift_a*(bdx*cdy - cdx*bdy) + alift_b*(cdx*ady - adx*cdy) + alift_c*(adx*bdy - bdx*ady)
// with every difference relative to d.
static __device__ __noinline__ int incircle_exact(double ax, double ay, double bx, double by, double cx,
                                           double cy, double dx, double dy) {
  double h[6], l[6];   // adx ady bdx bdy cdx cdy as exact pairs
  two_diff(ax, dx, h[0], l[0]);
  two_diff(ay, dy, h[1], l[1]);
  two_diff(bx, dx, h[2], l[2]);
  two_diff(by, dy, h[3], l[3]);
  two_diff(cx, dx, h[4], l[4]);
  two_diff(cy, dy, h[5], l[5]);
  Expansion<64> X;
  for (int t = 0; t < 3; ++t) {
    const int p = 2 * t, q = 2 * ((t + 1) % 3), r = 2 * ((t + 2) % 3);
    // lift of point t: x^2 + y^2 as monomials (h*h, 2 h*l, l*l) per coordinate
    double lf[6][2];
    double lc[6];
    int nl = 0;
    for (int c = 0; c < 2; ++c) {
      double hh = h[p + c], ll = l[p + c];
      lf[nl][0] = hh; lf[nl][1] = hh; lc[nl++] = 1.0;
      if (ll != 0.0) {
        lf[nl][0] = hh; lf[nl][1] = ll; lc[nl++] = 2.0;
        lf[nl][0] = ll; lf[nl][1] = ll; lc[nl++] = 1.0;
      }
    }
    // cross of the other two: q_x * r_y - r_x * q_y, as monomials
    double cf[8][2];
    double cs[8];
    int nc = 0;
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        double u = i ? l[q] : h[q], v = j ? l[r + 1] : h[r + 1];
        if (u != 0.0 && v != 0.0) { cf[nc][0] = u; cf[nc][1] = v; cs[nc++] = 1.0; }
        double u2 = i ? l[r] : h[r], v2 = j ? l[q + 1] : h[q + 1];
        if (u2 != 0.0 && v2 != 0.0) { cf[nc][0] = u2; cf[nc][1] = v2; cs[nc++] = -1.0; }
      }
    for (int i = 0; i < nl; ++i) {
      if (lf[i][0] == 0.0 || lf[i][1] == 0.0) continue;
      double lh, ll;
      two_prod(lf[i][0], lf[i][1], lh, ll);
      for (int j = 0; j < nc; ++j) {
        double ch, cl;
        two_prod(cf[j][0], cf[j][1], ch, cl);
        add_prod2(X, lh, ll, ch, cl, lc[i] * cs[j]);
        if (X.n > 48) X.compress();
      }
    }
  }
  return X.sign();
}

__device__ __forceinline__ int incircle_raw(double ax, double ay, double bx, double by, double cx,
                                            double cy, double dx, double dy) {
  double adx = __dsub_rn(ax, dx), ady = __dsub_rn(ay, dy);
  double bdx = __dsub_rn(bx, dx), bdy = __dsub_rn(by, dy);
  double cdx = __dsub_rn(cx, dx), cdy = __dsub_rn(cy, dy);
  double p1 = __dmul_rn(bdx, cdy), p2 = __dmul_rn(cdx, bdy);
  double p3 = __dmul_rn(cdx, ady), p4 = __dmul_rn(adx, cdy);
  double p5 = __dmul_rn(adx, bdy), p6 = __dmul_rn(bdx, ady);
  double al = __dadd_rn(__dmul_rn(adx, adx), __dmul_rn(ady, ady));
  double bl = __dadd_rn(__dmul_rn(bdx, bdx), __dmul_rn(bdy, bdy));
  double cl = __dadd_rn(__dmul_rn(cdx, cdx), __dmul_rn(cdy, cdy));
  double det = __dadd_rn(__dadd_rn(__dmul_rn(al, __dsub_rn(p1, p2)), __dmul_rn(bl, __dsub_rn(p3, p4))),
                         __dmul_rn(cl, __dsub_rn(p5, p6)));
  double perm = __dadd_rn(__dadd_rn(__dmul_rn(__dadd_rn(fabs(p1), fabs(p2)), al),
                                    __dmul_rn(__dadd_rn(fabs(p3), fabs(p4)), bl)),
                          __dmul_rn(__dadd_rn(fabs(p5), fabs(p6)), cl));
  // per term: lift 4 roundings, cross difference 4, product 1 -> 9u; two sums 2u:
  // |err| <= 11u perm + O(u^2)
  double bound = __dmul_rn(12.0 * kU, perm);
  if (perm > kTiny) {
    if (det > bound) return 1;
    if (-det > bound) return -1;
  }
  return incircle_exact(ax, ay, bx, by, cx, cy, dx, dy);
}

GDP_HD bool lex_less(double ax, double ay, double bx, double by) {
  return ax < bx || (ax == bx && ay < by);
}

// Simulation of simplicity: each lift x^2+y^2 is raised by eps_i, eps_i >> eps_j
// when point i is lexicographically (x, then y) larger than point j.  The
// perturbed determinant adds sum_i eps_i * C_i where C_i is the cofactor of
// row i's lift entry: C_a = +orient(b,c,d), C_b = -orient(a,c,d),
// C_c = +orient(a,b,d), C_d = -orient(a,b,c).  Ranking by coordinates (not by
// vertex number) makes the result independent of how vertices are numbered.
static __device__ __noinline__ int incircle_sos_tie(double2 a, double2 b, double2 c, double2 d) {
  double2 P[4] = {a, b, c, d};
  int ord[4] = {0, 1, 2, 3};
  for (int i = 1; i < 4; ++i) {       // decreasing lexicographic order
    int v = ord[i], j = i - 1;
    while (j >= 0 && lex_less(P[ord[j]].x, P[ord[j]].y, P[v].x, P[v].y)) {
      ord[j + 1] = ord[j];
      --j;
    }
    ord[j + 1] = v;
  }
  for (int r = 0; r < 4; ++r) {
    const int i = ord[r];
    double2 q[3];
    int k = 0;
    for (int j = 0; j < 4; ++j)
      if (j != i) q[k++] = P[j];
    int o = orient(q[0], q[1], q[2]);
    if (o != 0) return (i & 1) ? -o : o;
  }
  return 0;
}

__device__ __forceinline__ int incircle(double2 a, double2 b, double2 c, double2 d) {
  int s = incircle_raw(a.x, a.y, b.x, b.y, c.x, c.y, d.x, d.y);
  if (s != 0) return s;
  return incircle_sos_tie(a, b, c, d);
}

// ---------------------------------------------------------------- diametral circle
static __device__ __noinline__ int dot_exact(double ax, double ay, double bx, double by, double px,
                                      double py) {
  double axh, axl, ayh, ayl, bxh, bxl, byh, byl;
  two_diff(ax, px, axh, axl);
  two_diff(ay, py, ayh, ayl);
  two_diff(bx, px, bxh, bxl);
  two_diff(by, py, byh, byl);
  Expansion<24> X;
  add_prod2(X, axh, axl, bxh, bxl, 1.0);
  add_prod2(X, ayh, ayl, byh, byl, 1.0);
  return X.sign();
}

// sign of (a-p).(b-p)
__device__ __forceinline__ int dot_sign(double2 a, double2 b, double2 p) {
  double d1 = __dmul_rn(__dsub_rn(a.x, p.x), __dsub_rn(b.x, p.x));
  double d2 = __dmul_rn(__dsub_rn(a.y, p.y), __dsub_rn(b.y, p.y));
  double s = __dadd_rn(d1, d2);
  double perm = __dadd_rn(fabs(d1), fabs(d2));
  double bound = __dmul_rn(4.5 * kU, perm);
  if (perm > kTiny) {
    if (s > bound) return 1;
    if (-s > bound) return -1;
  }
  return dot_exact(a.x, a.y, b.x, b.y, p.x, p.y);
}

// ---------------------------------------------------------------- fixed-order FP64 geometry
// Canonical rotation: a = lexicographically smallest vertex, CCW order kept.
struct TriTerms {
  double ax, ay, dx, dy, ex, ey, la, lb, lc, cr;
};

__device__ __forceinline__ TriTerms tri_terms(double2 p0, double2 p1, double2 p2) {
  double2 a = p0, b = p1, c = p2;
  if (lex_less(p1.x, p1.y, a.x, a.y)) { a = p1; b = p2; c = p0; }
  if (lex_less(p2.x, p2.y, a.x, a.y)) { a = p2; b = p0; c = p1; }
  TriTerms t;
  t.ax = a.x;
  t.ay = a.y;
  t.dx = __dsub_rn(b.x, a.x);
  t.dy = __dsub_rn(b.y, a.y);
  t.ex = __dsub_rn(c.x, a.x);
  t.ey = __dsub_rn(c.y, a.y);
  double fx = __dsub_rn(c.x, b.x), fy = __dsub_rn(c.y, b.y);
  t.la = __dadd_rn(__dmul_rn(t.dx, t.dx), __dmul_rn(t.dy, t.dy));   // |ab|^2
  t.lb = __dadd_rn(__dmul_rn(t.ex, t.ex), __dmul_rn(t.ey, t.ey));   // |ac|^2
  t.lc = __dadd_rn(__dmul_rn(fx, fx), __dmul_rn(fy, fy));           // |bc|^2
  t.cr = __dsub_rn(__dmul_rn(t.dx, t.ey), __dmul_rn(t.dy, t.ex));   // 2 * signed area
  return t;
}

// R / l_min > B  <=>  la*lb*lc > 4 B^2 l_min^2 (2A)^2
__device__ __forceinline__ bool is_bad(const TriTerms& t, double B2) {
  double lmin = t.la;
  if (t.lb < lmin) lmin = t.lb;
  if (t.lc < lmin) lmin = t.lc;
  double lhs = __dmul_rn(__dmul_rn(t.la, t.lb), t.lc);
  double rhs = __dmul_rn(__dmul_rn(__dmul_rn(4.0, B2), lmin), __dmul_rn(t.cr, t.cr));
  return lhs > rhs;
}

__device__ __forceinline__ double2 circumcenter(const TriTerms& t) {
  double den = __dmul_rn(2.0, t.cr);
  double nx = __dsub_rn(__dmul_rn(t.ey, t.la), __dmul_rn(t.dy, t.lb));
  double ny = __dsub_rn(__dmul_rn(t.dx, t.lb), __dmul_rn(t.ex, t.la));
  return make_double2(__dadd_rn(t.ax, __ddiv_rn(nx, den)), __dadd_rn(t.ay, __ddiv_rn(ny, den)));
}

__device__ __forceinline__ double2 midpoint(double2 a, double2 b) {
  return make_double2(__dmul_rn(__dadd_rn(a.x, b.x), 0.5), __dmul_rn(__dadd_rn(a.y, b.y), 0.5));
}

// priority measure: float32 bits of a non-negative value (monotone in the value)
__device__ __forceinline__ uint32_t measure_bits(double v) {
  return __float_as_uint(__double2float_rn(v)) & 0x7fffffffu;
}

__device__ __forceinline__ double seg_measure(double2 a, double2 b) {
  if (lex_less(b.x, b.y, a.x, a.y)) { double2 t = a; a = b; b = t; }
  double dx = __dsub_rn(b.x, a.x), dy = __dsub_rn(b.y, a.y);
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

}  // namespace gdp
