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

// diagnostic counters (per translation unit), written only in a build with
// -DGDP_DIAG: exact-path calls and maxima
// 0 orient_exact, 1 incircle_exact, 2 incircle tie (simulation of simplicity),
// 3 dot_exact, 4 incircle_exact with inexact differences, 5 max walk steps,
// 6 max cycles in one grow, 7 max cycles in one walk, 8 max cycles of one exact incircle,
// 9/10/11 orient / incircle / dot calls, 12/13/14 of them past the FP32 filter
static __device__ unsigned long long g_diag[16];
#ifdef GDP_DIAG
#define GDP_DIAG_ADD(i) atomicAdd(&g_diag[i], 1ull)
#define GDP_DIAG_MAX(i, v) atomicMax(&g_diag[i], (unsigned long long)(v))
#define GDP_DIAG_CLOCK() clock64()
#else
#define GDP_DIAG_ADD(i) ((void)0)
#define GDP_DIAG_MAX(i, v) ((void)0)
#define GDP_DIAG_CLOCK() 0ll
#endif
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

// ---------------------------------------------------------------- exact sums in integers
// When every coordinate difference of a predicate is itself an exact double
// (two_diff leaves no tail -- the common case), the determinant is a signed
// sum of products of those doubles.  Each double is m * 2^e with an integer
// mantissa m < 2^53 (from its bit pattern, no floating-point operation), a
// product of k doubles is an integer of at most 53k bits times 2^(sum of e),
// and all products are summed exactly in a 576-bit two's-complement
// accumulator after aligning them to the smallest exponent.  Integer
// multiplies run at full rate on the SM, unlike FP64.
constexpr int IL = 9;   // accumulator limbs

struct Mono {
  unsigned long long m[4];   // |product|, little-endian limbs
  int nl;
  int e;
  bool neg;
};

__device__ __forceinline__ bool split_dbl(double x, unsigned long long& m, int& e, bool& neg) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0x7ff) return false;
  neg = (b >> 63) != 0;
  m = b & ((1ull << 52) - 1);
  if (ex == 0) {
    e = -1074;
  } else {
    m |= 1ull << 52;
    e = ex - 1075;
  }
  return true;
}

// product of k doubles (none zero) into mo
__device__ __forceinline__ bool mono_prod(const double* f, int k, double coef_sign, Mono& mo) {
  mo.m[0] = 1;
  mo.m[1] = mo.m[2] = mo.m[3] = 0;
  mo.nl = 1;
  mo.e = 0;
  mo.neg = coef_sign < 0;
  for (int j = 0; j < k; ++j) {
    unsigned long long m;
    int e;
    bool ng;
    if (!split_dbl(f[j], m, e, ng)) return false;
    mo.neg ^= ng;
    mo.e += e;
    unsigned long long carry = 0;
    for (int l = 0; l < mo.nl; ++l) {
      const unsigned long long lo = mo.m[l] * m;
      const unsigned long long hi = __umul64hi(mo.m[l], m);
      const unsigned long long s = lo + carry;
      carry = hi + (s < lo ? 1ull : 0ull);
      mo.m[l] = s;
    }
    if (carry) mo.m[mo.nl++] = carry;
  }
  return true;
}

// acc += (neg ? -1 : 1) * (m << sh); false if the shifted value does not fit
__device__ __forceinline__ bool acc_add(unsigned long long* acc, const Mono& mo, int sh) {
  const int w = sh >> 6, bsh = sh & 63;
  if (w + mo.nl + 1 > IL - 1) return false;
  unsigned long long t[IL];
  for (int l = 0; l < IL; ++l) t[l] = 0;
  for (int l = 0; l < mo.nl; ++l) {
    t[w + l] |= mo.m[l] << bsh;
    if (bsh) t[w + l + 1] |= mo.m[l] >> (64 - bsh);
  }
  if (!mo.neg) {
    unsigned long long c = 0;
    for (int l = 0; l < IL; ++l) {
      const unsigned long long s = acc[l] + t[l];
      const unsigned long long s2 = s + c;
      c = (s < acc[l] ? 1ull : 0ull) + (s2 < s ? 1ull : 0ull);
      acc[l] = s2;
    }
  } else {
    unsigned long long br = 0;
    for (int l = 0; l < IL; ++l) {
      const unsigned long long d = acc[l] - t[l];
      const unsigned long long d2 = d - br;
      br = (acc[l] < t[l] ? 1ull : 0ull) + (d < br ? 1ull : 0ull);
      acc[l] = d2;
    }
  }
  return true;
}

// exact sign of sum_i sign_i * prod_j f[i*k + j]; returns 2 when the integer
// range does not suffice (caller falls back to expansions)
static __device__ __noinline__ int int_sign(const double* f, const double* sg, int nmono, int k) {
  int emin = 1 << 30;
  for (int i = 0; i < nmono; ++i) {
    int e = 0;
    bool zero = false;
    for (int j = 0; j < k; ++j) {
      const double x = f[i * k + j];
      if (x == 0.0) { zero = true; break; }
      unsigned long long m;
      int ej;
      bool ng;
      if (!split_dbl(x, m, ej, ng)) return 2;
      e += ej;
    }
    if (!zero && e < emin) emin = e;
  }
  if (emin == (1 << 30)) return 0;
  unsigned long long acc[IL];
  for (int l = 0; l < IL; ++l) acc[l] = 0;
  for (int i = 0; i < nmono; ++i) {
    bool zero = false;
    for (int j = 0; j < k; ++j) zero |= f[i * k + j] == 0.0;
    if (zero) continue;
    Mono mo;
    if (!mono_prod(f + i * k, k, sg[i], mo)) return 2;
    if (!acc_add(acc, mo, mo.e - emin)) return 2;
  }
  if ((long long)acc[IL - 1] < 0) return -1;
  for (int l = 0; l < IL; ++l)
    if (acc[l]) return 1;
  return 0;
}

// ---------------------------------------------------------------- orient
static __device__ __noinline__ int orient_exact(double ax, double ay, double bx, double by, double cx,
                                         double cy) {
  // (ax-cx)(by-cy) - (ay-cy)(bx-cx) with each difference as an exact pair
  GDP_DIAG_ADD(0);
  double acxh, acxl, acyh, acyl, bcxh, bcxl, bcyh, bcyl;
  two_diff(ax, cx, acxh, acxl);
  two_diff(ay, cy, acyh, acyl);
  two_diff(bx, cx, bcxh, bcxl);
  two_diff(by, cy, bcyh, bcyl);
  if (acxl == 0.0 && acyl == 0.0 && bcxl == 0.0 && bcyl == 0.0) {
    const double f[4] = {acxh, bcyh, acyh, bcxh};
    const double sg[2] = {1.0, -1.0};
    const int r = int_sign(f, sg, 2, 2);
    if (r != 2) return r;
  }
  Expansion<24> X;
  add_prod2(X, acxh, acxl, bcyh, bcyl, 1.0);
  add_prod2(X, acyh, acyl, bcxh, bcxl, -1.0);
  return X.sign();
}

__device__ __forceinline__ int orient(double ax, double ay, double bx, double by, double cx,
                                      double cy) {
  const double d1 = __dsub_rn(ax, cx), d2 = __dsub_rn(by, cy);
  const double d3 = __dsub_rn(ay, cy), d4 = __dsub_rn(bx, cx);
  // a difference of two doubles rounds to zero only when they are equal, so a
  // zero factor on each side makes the determinant exactly zero
  if ((d1 == 0.0 || d2 == 0.0) && (d3 == 0.0 || d4 == 0.0)) return 0;
  double l = __dmul_rn(d1, d2);
  double r = __dmul_rn(d3, d4);
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
  const long long c0 = GDP_DIAG_CLOCK();
  GDP_DIAG_ADD(1);
  (void)c0;
  double h[6], l[6];   // adx ady bdx bdy cdx cdy as exact pairs
  two_diff(ax, dx, h[0], l[0]);
  two_diff(ay, dy, h[1], l[1]);
  two_diff(bx, dx, h[2], l[2]);
  two_diff(by, dy, h[3], l[3]);
  two_diff(cx, dx, h[4], l[4]);
  two_diff(cy, dy, h[5], l[5]);
  if (l[0] != 0.0 || l[1] != 0.0 || l[2] != 0.0 || l[3] != 0.0 || l[4] != 0.0 || l[5] != 0.0) {
    GDP_DIAG_ADD(4);
  } else {
    // sum over the three points t (q, r the other two) of
    // (x_t^2 + y_t^2) (x_q y_r - x_r y_q): 12 monomials of degree 4
    double f[48], sg[12];
    int n = 0;
    for (int t = 0; t < 3; ++t) {
      const int q = (t + 1) % 3, r = (t + 2) % 3;
      for (int c = 0; c < 2; ++c) {
        const double a = h[2 * t + c];
        f[4 * n] = a; f[4 * n + 1] = a; f[4 * n + 2] = h[2 * q]; f[4 * n + 3] = h[2 * r + 1];
        sg[n++] = 1.0;
        f[4 * n] = a; f[4 * n + 1] = a; f[4 * n + 2] = h[2 * r]; f[4 * n + 3] = h[2 * q + 1];
        sg[n++] = -1.0;
      }
    }
    const int rr = int_sign(f, sg, n, 4);
    if (rr != 2) {
      GDP_DIAG_MAX(8, GDP_DIAG_CLOCK() - c0);
      return rr;
    }
  }
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
  GDP_DIAG_MAX(8, GDP_DIAG_CLOCK() - c0);
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
  GDP_DIAG_ADD(2);
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
  GDP_DIAG_ADD(3);
  double axh, axl, ayh, ayl, bxh, bxl, byh, byl;
  two_diff(ax, px, axh, axl);
  two_diff(ay, py, ayh, ayl);
  two_diff(bx, px, bxh, bxl);
  two_diff(by, py, byh, byl);
  if (axl == 0.0 && ayl == 0.0 && bxl == 0.0 && byl == 0.0) {
    const double f[4] = {axh, bxh, ayh, byh};
    const double sg[2] = {1.0, 1.0};
    const int r = int_sign(f, sg, 2, 2);
    if (r != 2) return r;
  }
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

// ---------------------------------------------------------------- diametral lens
// p strictly inside the diametral lens of ab (Chew's rule, Sec. 4.2): the
// segment subtends more than 120 degrees at p.  With u = a - p, w = b - p,
// D = u.w and C = u x w, Lagrange's identity |u|^2 |w|^2 = D^2 + C^2 turns
// cos(angle) < -1/2 into D < 0 and Q = 3 D^2 - C^2 > 0, where
//   Q = 3 ux^2 wx^2 + 3 uy^2 wy^2 - ux^2 wy^2 - uy^2 wx^2 + 8 ux uy wx wy.
// Exact sign of Q: every difference as an exact pair (h + l); with no tails,
// the 16 degree-4 monomials (coefficients as repeated terms) go to the integer
// accumulator, otherwise the products of all h / l choices are summed as a
// floating-point expansion.
static __device__ __noinline__ int lens_q_exact(double ax, double ay, double bx, double by, double px,
                                                double py) {
  GDP_DIAG_ADD(3);
  double h[4], l[4];   // ux uy wx wy
  two_diff(ax, px, h[0], l[0]);
  two_diff(ay, py, h[1], l[1]);
  two_diff(bx, px, h[2], l[2]);
  two_diff(by, py, h[3], l[3]);
  // (coefficient, four factor indices)
  const int T[5][5] = {{3, 0, 0, 2, 2}, {3, 1, 1, 3, 3}, {-1, 0, 0, 3, 3}, {-1, 1, 1, 2, 2},
                       {8, 0, 1, 2, 3}};
  if (l[0] == 0.0 && l[1] == 0.0 && l[2] == 0.0 && l[3] == 0.0) {
    double f[64], sg[16];
    int n = 0;
    for (int t = 0; t < 5; ++t) {
      const int c = T[t][0] < 0 ? -T[t][0] : T[t][0];
      for (int r = 0; r < c; ++r) {
        for (int j = 0; j < 4; ++j) f[4 * n + j] = h[T[t][1 + j]];
        sg[n++] = T[t][0] < 0 ? -1.0 : 1.0;
      }
    }
    const int r = int_sign(f, sg, n, 4);
    if (r != 2) return r;
  }
  Expansion<64> X;
  for (int t = 0; t < 5; ++t) {
    for (int m = 0; m < 16; ++m) {   // bit j of m: the tail of factor j
      double f[4];
      bool zero = false;
      for (int j = 0; j < 4; ++j) {
        const int v = T[t][1 + j];
        f[j] = ((m >> j) & 1) ? l[v] : h[v];
        zero |= f[j] == 0.0;
      }
      if (zero) continue;
      double x, y, z, w;
      two_prod(f[0], f[1], x, y);
      two_prod(f[2], f[3], z, w);
      const int c = T[t][0];
      if (c == 3) {   // 3 = 2 + 1, each a power of two
        add_prod2(X, x, y, z, w, 2.0);
        add_prod2(X, x, y, z, w, 1.0);
      } else {
        add_prod2(X, x, y, z, w, (double)c);
      }
      if (X.n > 40) X.compress();
    }
  }
  return X.sign();
}

// FP64 filter for the sign of Q when D < 0 is known: D and C with forward
// error bounds (difference, product and sum roundings: 4.5 u of the sum of
// the absolute products), then Q over the intervals with the rounding of
// that last evaluation folded into the factors 1 -+ 8u.  0 when unsure.
__device__ __forceinline__ int lens_q_f64(double2 a, double2 b, double2 p) {
  const double ux = __dsub_rn(a.x, p.x), uy = __dsub_rn(a.y, p.y);
  const double wx = __dsub_rn(b.x, p.x), wy = __dsub_rn(b.y, p.y);
  const double t1 = __dmul_rn(ux, wx), t2 = __dmul_rn(uy, wy);
  const double t3 = __dmul_rn(ux, wy), t4 = __dmul_rn(uy, wx);
  const double aD = fabs(__dadd_rn(t1, t2)), aC = fabs(__dsub_rn(t3, t4));
  const double eD = __dmul_rn(4.5 * kU, __dadd_rn(fabs(t1), fabs(t2)));
  const double eC = __dmul_rn(4.5 * kU, __dadd_rn(fabs(t3), fabs(t4)));
  constexpr double kSmall = 1e-150;   // squares of larger values do not underflow
  if (!(aD > eD) || !(aD - eD > kSmall) || !(aD + eD < 1e150) || !(aC + eC < 1e150)) return 0;
  const double dlo = __dsub_rn(aD, eD), dhi = __dadd_rn(aD, eD);
  const double clo = (aC - eC > kSmall) ? __dsub_rn(aC, eC) : 0.0;
  const double chi = fmax(__dadd_rn(aC, eC), kSmall);
  const double lo = __dsub_rn(__dmul_rn(__dmul_rn(3.0 * (1.0 - 8.0 * kU), dlo), dlo),
                              __dmul_rn(__dmul_rn(1.0 + 8.0 * kU, chi), chi));
  const double hi = __dsub_rn(__dmul_rn(__dmul_rn(3.0 * (1.0 + 8.0 * kU), dhi), dhi),
                              __dmul_rn(__dmul_rn(1.0 - 8.0 * kU, clo), clo));
  return lo > 0.0 ? 1 : (hi < 0.0 ? -1 : 0);
}

// ---------------------------------------------------------------- FP32 filter stage
// GB300 executes FP64 at 1/64 of the FP32 rate, so every predicate first runs
// in FP32.  Each vertex keeps its coordinates translated to the mesh's
// bounding-box centre o as two floats: t = fl64(x - o), hi = fl32(t),
// lo = fl32(t - hi) (t - hi is exact in FP64), so hi + lo is within
// 2^-48 |t| of t and within 1.04 * 2^-48 M of x - o (M the largest |hi| of a
// test).  A coordinate difference is taken as s = fl32(fl32(hi_a - hi_b) +
// fl32(lo_a - lo_b)); working through the three roundings, s is within
//   delta(s) = 2.0001 v |s| + E3,   v = 2^-24,  E3 = 2^-44 M
// of the exact difference: relative to the difference itself, not to the
// coordinates, so small features far from the centre still filter well.
// Each filter adds the effect of delta on its products to the rounding error
// of its float evaluation; when the float value cannot decide, the FP64
// filter and then exact arithmetic do.
constexpr float kV = 5.9604645e-8f;   // 2^-24
constexpr float kE3 = 5.6843419e-14f;  // 2^-44

struct P2 {
  double2 d;   // exact (FP64) coordinates
  float4 f;    // translated copy as two floats: (hi.x, hi.y, lo.x, lo.y)
};

__device__ __forceinline__ float fmax6(float a, float b, float c, float d, float e, float g) {
  return fmaxf(fmaxf(fmaxf(a, b), fmaxf(c, d)), fmaxf(e, g));
}

// the two float differences a - b (x, y)
__device__ __forceinline__ float dfx(const float4& a, const float4& b) {
  return __fadd_rn(__fsub_rn(a.x, b.x), __fsub_rn(a.z, b.z));
}
__device__ __forceinline__ float dfy(const float4& a, const float4& b) {
  return __fadd_rn(__fsub_rn(a.y, b.y), __fsub_rn(a.w, b.w));
}
__device__ __forceinline__ float hmax3(const float4& a, const float4& b, const float4& c) {
  return fmax6(fabsf(a.x), fabsf(a.y), fabsf(b.x), fabsf(b.y), fabsf(c.x), fabsf(c.y));
}

// sign of s1 s2 - s3 s4 (sg = -1) or s1 s2 + s3 s4 (sg = +1) from four
// differences, when certain, else 0.  Input error: each product is off by at
// most 4.0003 v |s_i s_j| + E3 (|s_i| + |s_j|) + E3^2 from the differences;
// rounding of the two products and the sum: 2.0001 v (|p| + |q|).
__device__ __forceinline__ int sign2_f32(float s1, float s2, float s3, float s4, float sg, float M) {
  const float p = __fmul_rn(s1, s2), q = __fmul_rn(s3, s4);
  const float val = sg > 0.0f ? __fadd_rn(p, q) : __fsub_rn(p, q);
  const float E3 = kE3 * M;
  const float err = (6.0005f * kV * (fabsf(p) + fabsf(q)) +
                     E3 * (fabsf(s1) + fabsf(s2) + fabsf(s3) + fabsf(s4) + 2.0f * E3)) * 1.001f + 1e-37f;
  return val > err ? 1 : (-val > err ? -1 : 0);
}

// sign of (ax-cx)(by-cy) - (ay-cy)(bx-cx) when certain, else 0
__device__ __forceinline__ int orient_f32(float4 a, float4 b, float4 c) {
  const float M = hmax3(a, b, c);
  if (!(M < 1e8f) || M < 1e-15f) return 0;
  return sign2_f32(dfx(a, c), dfy(b, c), dfy(a, c), dfx(b, c), -1.0f, M);
}

// sign of the incircle determinant (same evaluation order as the FP64 filter).
// Input error: each of the 12 degree-4 monomials is off by at most
// ((1 + 2.0001 v)^4 - 1) |monomial| + 4 E3 (L' + E3)^3 (L' the largest |s|
// grown by 2.0001 v), in all 8.0013 v perm + 48 E3 (L' + E3)^3; rounding of
// the float evaluation: 12.5 v perm (11 v to first order).
__device__ __forceinline__ int incircle_f32(float4 a, float4 b, float4 c, float4 d) {
  const float M = fmaxf(hmax3(a, b, c), fmaxf(fabsf(d.x), fabsf(d.y)));
  if (!(M < 1e7f) || M < 1e-7f) return 0;
  const float adx = dfx(a, d), ady = dfy(a, d);
  const float bdx = dfx(b, d), bdy = dfy(b, d);
  const float cdx = dfx(c, d), cdy = dfy(c, d);
  const float p1 = __fmul_rn(bdx, cdy), p2 = __fmul_rn(cdx, bdy);
  const float p3 = __fmul_rn(cdx, ady), p4 = __fmul_rn(adx, cdy);
  const float p5 = __fmul_rn(adx, bdy), p6 = __fmul_rn(bdx, ady);
  const float al = __fadd_rn(__fmul_rn(adx, adx), __fmul_rn(ady, ady));
  const float bl = __fadd_rn(__fmul_rn(bdx, bdx), __fmul_rn(bdy, bdy));
  const float cl = __fadd_rn(__fmul_rn(cdx, cdx), __fmul_rn(cdy, cdy));
  const float det = __fadd_rn(__fadd_rn(__fmul_rn(al, __fsub_rn(p1, p2)), __fmul_rn(bl, __fsub_rn(p3, p4))),
                              __fmul_rn(cl, __fsub_rn(p5, p6)));
  const float perm = __fadd_rn(__fadd_rn(__fmul_rn(__fadd_rn(fabsf(p1), fabsf(p2)), al),
                                         __fmul_rn(__fadd_rn(fabsf(p3), fabsf(p4)), bl)),
                               __fmul_rn(__fadd_rn(fabsf(p5), fabsf(p6)), cl));
  const float L = fmax6(fabsf(adx), fabsf(ady), fabsf(bdx), fabsf(bdy), fabsf(cdx), fabsf(cdy)) * (1.0f + 2.0002f * kV);
  const float E3 = kE3 * M;
  const float LE = L + E3;
  const float err = (20.6f * kV * perm + 48.0f * E3 * LE * LE * LE) * 1.001f + 1e-37f;
  return det > err ? 1 : (-det > err ? -1 : 0);
}

// sign of (a-p).(b-p) when certain, else 0
__device__ __forceinline__ int dot_f32(float4 a, float4 b, float4 p) {
  const float M = hmax3(a, b, p);
  if (!(M < 1e8f) || M < 1e-15f) return 0;
  return sign2_f32(dfx(a, p), dfx(b, p), dfy(a, p), dfy(b, p), 1.0f, M);
}

// FP32 filter for the sign of Q = 3 D^2 - C^2 when D < 0 is known (see
// lens_q_exact): D and C from the float differences with the bound of
// sign2_f32, then Q over the intervals with the float rounding folded into
// the factors 1 -+ 8v.  0 when unsure.
__device__ __forceinline__ int lens_q_f32(float4 a, float4 b, float4 p) {
  const float M = hmax3(a, b, p);
  if (!(M < 1e8f) || M < 1e-15f) return 0;
  const float ux = dfx(a, p), uy = dfy(a, p);
  const float wx = dfx(b, p), wy = dfy(b, p);
  const float t1 = __fmul_rn(ux, wx), t2 = __fmul_rn(uy, wy);
  const float t3 = __fmul_rn(ux, wy), t4 = __fmul_rn(uy, wx);
  const float aD = fabsf(__fadd_rn(t1, t2)), aC = fabsf(__fsub_rn(t3, t4));
  const float E3 = kE3 * M;
  const float es = E3 * (fabsf(ux) + fabsf(uy) + fabsf(wx) + fabsf(wy) + 2.0f * E3);
  const float eD = (es + 6.0005f * kV * (fabsf(t1) + fabsf(t2))) * 1.001f + 1e-37f;
  const float eC = (es + 6.0005f * kV * (fabsf(t3) + fabsf(t4))) * 1.001f + 1e-37f;
  constexpr float kSmall = 1e-17f;   // squares of larger values stay normal
  if (!(aD - eD > kSmall) || !(aD + eD < 1e17f) || !(aC + eC < 1e17f)) return 0;
  const float dlo = aD - eD, dhi = aD + eD;
  const float clo = (aC - eC > kSmall) ? aC - eC : 0.0f;
  const float chi = fmaxf(aC + eC, kSmall);
  const float lo = __fsub_rn(__fmul_rn(__fmul_rn(3.0f * (1.0f - 8.0f * kV), dlo), dlo),
                             __fmul_rn(__fmul_rn(1.0f + 8.0f * kV, chi), chi));
  const float hi = __fsub_rn(__fmul_rn(__fmul_rn(3.0f * (1.0f + 8.0f * kV), dhi), dhi),
                             __fmul_rn(__fmul_rn(1.0f - 8.0f * kV, clo), clo));
  return lo > 0.0f ? 1 : (hi < 0.0f ? -1 : 0);
}

__device__ __forceinline__ int orient(const P2& a, const P2& b, const P2& c) {
  const int s = orient_f32(a.f, b.f, c.f);
  GDP_DIAG_ADD(9);
  if (!s) GDP_DIAG_ADD(12);
  return s ? s : orient(a.d, b.d, c.d);
}

__device__ __forceinline__ int dot_sign(const P2& a, const P2& b, const P2& p) {
  const int s = dot_f32(a.f, b.f, p.f);
  GDP_DIAG_ADD(11);
  if (!s) GDP_DIAG_ADD(14);
  return s ? s : dot_sign(a.d, b.d, p.d);
}

// -1: p strictly inside the diametral lens of ab (Chew's rule, Sec. 4.2),
// 0: p is a or b, or exactly on the lens boundary, +1: outside
__device__ __forceinline__ int lens_sign(const P2& a, const P2& b, const P2& p) {
  const int d = dot_sign(a, b, p);
  if (d > 0) return 1;
  if (d == 0) return ((p.d.x == a.d.x && p.d.y == a.d.y) || (p.d.x == b.d.x && p.d.y == b.d.y)) ? 0 : 1;
  int q = lens_q_f32(a.f, b.f, p.f);
  if (!q) q = lens_q_f64(a.d, b.d, p.d);
  if (!q) q = lens_q_exact(a.d.x, a.d.y, b.d.x, b.d.y, p.d.x, p.d.y);
  return q > 0 ? -1 : (q < 0 ? 1 : 0);
}

// p encroaches subsegment ab: strictly inside its diametral circle (Ruppert's
// rule) or, with lens, strictly inside its diametral lens (Chew's rule)
__device__ __forceinline__ bool encroaches(const P2& a, const P2& b, const P2& p, bool lens) {
  return lens ? lens_sign(a, b, p) < 0 : dot_sign(a, b, p) < 0;
}

__device__ __forceinline__ int incircle(const P2& a, const P2& b, const P2& c, const P2& d) {
  const int s = incircle_f32(a.f, b.f, c.f, d.f);
  GDP_DIAG_ADD(10);
  if (!s) GDP_DIAG_ADD(13);
  return s ? s : incircle(a.d, b.d, c.d, d.d);
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

// FP32 pre-check of is_bad: +1 when the FP64 formula above surely says bad,
// -1 when it surely says good, 0 when the float intervals overlap.  Interval
// bounds for the exact squared lengths and doubled area come from the float
// differences (error delta(s) each, as in the predicates): a squared length
// x^2 + y^2 is off by at most 6.01 v (x^2 + y^2) + 2.01 E3 (|x| + |y|) + 2 E3^2
// with its own rounding, the doubled area as in sign2_f32; the FP64 formula
// is within ~20 u of the exact quantities, far inside the float margins.
__device__ __forceinline__ int bad_f32(float4 a, float4 b, float4 c, float B2f) {
  const float M = hmax3(a, b, c);
  if (!(M < 1e7f) || M < 1e-6f) return 0;
  const float E3 = kE3 * M;
  const float x1 = dfx(b, a), y1 = dfy(b, a);
  const float x2 = dfx(c, a), y2 = dfy(c, a);
  const float x3 = dfx(c, b), y3 = dfy(c, b);
  const float la = __fadd_rn(__fmul_rn(x1, x1), __fmul_rn(y1, y1));
  const float lb = __fadd_rn(__fmul_rn(x2, x2), __fmul_rn(y2, y2));
  const float lc = __fadd_rn(__fmul_rn(x3, x3), __fmul_rn(y3, y3));
  const float ea = 6.01f * kV * la + 2.01f * E3 * (fabsf(x1) + fabsf(y1)) + 2.0f * E3 * E3;
  const float eb = 6.01f * kV * lb + 2.01f * E3 * (fabsf(x2) + fabsf(y2)) + 2.0f * E3 * E3;
  const float ec = 6.01f * kV * lc + 2.01f * E3 * (fabsf(x3) + fabsf(y3)) + 2.0f * E3 * E3;
  const float t1 = __fmul_rn(x1, y2), t2 = __fmul_rn(y1, x2);
  const float cr = fabsf(__fsub_rn(t1, t2));
  const float ecr = 6.0005f * kV * (fabsf(t1) + fabsf(t2)) +
                    E3 * (fabsf(x1) + fabsf(y2) + fabsf(y1) + fabsf(x2) + 2.0f * E3);
  if (!(la > ea && lb > eb && lc > ec && cr > ecr)) return 0;
  const float lo = 1.0f - 16.0f * kV, hi = 1.0f + 16.0f * kV;
  const float lhs_lo = (la - ea) * (lb - eb) * (lc - ec) * lo;
  const float lhs_hi = (la + ea) * (lb + eb) * (lc + ec) * hi;
  const float mn_lo = fminf(fminf(la - ea, lb - eb), lc - ec);
  const float mn_hi = fminf(fminf(la + ea, lb + eb), lc + ec);
  const float cl = cr - ecr, ch = cr + ecr;
  const float rhs_lo = 4.0f * B2f * mn_lo * cl * cl * lo;
  const float rhs_hi = 4.0f * B2f * mn_hi * ch * ch * hi;
  if (!(lhs_hi < 1e37f && rhs_hi < 1e37f && lhs_lo > 1e-36f && rhs_lo > 1e-36f)) return 0;
  if (lhs_lo > rhs_hi) return 1;
  if (lhs_hi < rhs_lo) return -1;
  return 0;
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
