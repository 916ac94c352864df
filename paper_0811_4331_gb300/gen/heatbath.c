/*
 * Seeded SU(3) Wilson-action heatbath (input generator, not part of the solver).
 *
 * Cabibbo-Marinari: every link is updated by the three SU(2) subgroups
 * (0,1), (1,2), (0,2) in turn, each drawn with the Kennedy-Pendleton
 * algorithm (Phys. Lett. B 156 (1985) 393) from the heatbath distribution
 * exp((beta/3) Re tr(R U A)) where A is the staple sum of the link.  One
 * sweep visits mu = 0..3 and, for each, the even then the odd sites in
 * lexicographic order (links of one direction and parity share no staple);
 * every link is reunitarised after each sweep.  Cold start.
 *
 * Bit reproducibility on every machine: the only floating-point operations
 * are +, -, *, / and sqrt (correctly rounded by IEEE 754) in a fixed order,
 * compiled with -ffp-contract=off (no fused multiply-add); the logarithm is a
 * fixed-length atanh series after an exact frexp; no trigonometric function
 * is used (Gaussian and spherical variates by rejection).  Random numbers:
 * one sequential SplitMix64 stream (Steele, Lea, Flood 2014) seeded with
 * `seed`; uniform u in (0, 1] = ((x >> 11) + 1) 2^-53.
 *
 * Layout: U is double complex [4][V][3][3] (mu = x, y, z, t; site
 * lexicographic x fastest), interleaved (re, im).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef struct {
  double re, im;
} cplx;

static inline cplx cadd(cplx a, cplx b) {
  cplx r = {a.re + b.re, a.im + b.im};
  return r;
}
static inline cplx csub(cplx a, cplx b) {
  cplx r = {a.re - b.re, a.im - b.im};
  return r;
}
static inline cplx cmul(cplx a, cplx b) {
  cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
  return r;
}
static inline cplx cconj(cplx a) {
  cplx r = {a.re, -a.im};
  return r;
}

typedef struct {
  cplx m[3][3];
} su3;

static su3 mm(const su3* a, const su3* b) {
  su3 c;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) {
      cplx s = cmul(a->m[i][0], b->m[0][k]);
      s = cadd(s, cmul(a->m[i][1], b->m[1][k]));
      s = cadd(s, cmul(a->m[i][2], b->m[2][k]));
      c.m[i][k] = s;
    }
  return c;
}
static su3 dag(const su3* a) {
  su3 c;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) c.m[i][k] = cconj(a->m[k][i]);
  return c;
}

/* ------------------------------------------------------------------ random numbers */
static inline uint64_t next64(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static inline double uniform(uint64_t* s) { return ((double)(next64(s) >> 11) + 1.0) * 0x1.0p-53; }

/* ln x for x > 0: x = m 2^e with m in [1/sqrt2, sqrt2), t = (m - 1)/(m + 1),
 * ln m = 2 (t + t^3/3 + ... + t^47/47). */
static double ln_series(double x) {
  int e;
  double m = frexp(x, &e); /* exact: m in [0.5, 1) */
  if (m < 0.70710678118654752) {
    m = m * 2.0;
    e = e - 1;
  }
  const double t = (m - 1.0) / (m + 1.0);
  const double t2 = t * t;
  double acc = 1.0 / 47.0;
  for (int k = 22; k >= 0; --k) acc = acc * t2 + 1.0 / (double)(2 * k + 1);
  return 2.0 * t * acc + (double)e * 0.6931471805599453;
}

/* Kennedy-Pendleton draw of x0 with density ~ sqrt(1 - x0^2) exp(alpha x0). */
static double kp_x0(uint64_t* s, double alpha) {
  for (;;) {
    const double r1 = uniform(s);
    double u, v, q;
    do {
      u = 2.0 * uniform(s) - 1.0;
      v = 2.0 * uniform(s) - 1.0;
      q = u * u + v * v;
    } while (!(q > 0.0 && q < 1.0));
    const double r4 = uniform(s);
    const double g = -(u * u) * ln_series(q) / q; /* Gamma(1/2) */
    const double delta = (-ln_series(r1) + g) / alpha;
    if (r4 * r4 <= 1.0 - 0.5 * delta) return 1.0 - delta;
  }
}

static void unit_vector(uint64_t* s, double d[3]) {
  for (;;) {
    const double a = 2.0 * uniform(s) - 1.0, b = 2.0 * uniform(s) - 1.0, c = 2.0 * uniform(s) - 1.0;
    const double r2 = (a * a + b * b) + c * c;
    if (r2 > 1e-6 && r2 <= 1.0) {
      const double r = sqrt(r2);
      d[0] = a / r;
      d[1] = b / r;
      d[2] = c / r;
      return;
    }
  }
}

/* ------------------------------------------------------------------ lattice */
typedef struct {
  int L[4];
  int V;
  cplx* U; /* [4][V][3][3] */
} lattice;

static inline su3 get(const lattice* g, int mu, int site) {
  su3 r;
  memcpy(&r, g->U + ((size_t)mu * g->V + site) * 9, sizeof(r));
  return r;
}
static inline void put(lattice* g, int mu, int site, const su3* r) {
  memcpy(g->U + ((size_t)mu * g->V + site) * 9, r, sizeof(*r));
}
static int shift(const lattice* g, int site, int mu, int step) {
  int c[4], q = site;
  c[0] = q % g->L[0];
  q /= g->L[0];
  c[1] = q % g->L[1];
  q /= g->L[1];
  c[2] = q % g->L[2];
  c[3] = q / g->L[2];
  c[mu] = (c[mu] + step + g->L[mu]) % g->L[mu];
  return c[0] + g->L[0] * (c[1] + g->L[1] * (c[2] + g->L[2] * c[3]));
}

static su3 staple_sum(const lattice* g, int mu, int n) {
  su3 A;
  memset(&A, 0, sizeof(A));
  const int np = shift(g, n, mu, +1);
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    /* up: U_nu(n+mu) U_mu(n+nu)^+ U_nu(n)^+ */
    su3 a = get(g, nu, np), b = get(g, mu, shift(g, n, nu, +1)), c = get(g, nu, n);
    su3 bd = dag(&b), cd = dag(&c);
    su3 t = mm(&a, &bd);
    su3 up = mm(&t, &cd);
    /* down: U_nu(n+mu-nu)^+ U_mu(n-nu)^+ U_nu(n-nu) */
    const int nm = shift(g, n, nu, -1);
    su3 d = get(g, nu, shift(g, np, nu, -1)), e = get(g, mu, nm), f = get(g, nu, nm);
    su3 dd = dag(&d), ed = dag(&e);
    su3 t2 = mm(&dd, &ed);
    su3 dn = mm(&t2, &f);
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k) A.m[i][k] = cadd(A.m[i][k], cadd(up.m[i][k], dn.m[i][k]));
  }
  return A;
}

/* R <- r embedded in (i, j), applied from the left: M <- R M. */
static void left_su2(su3* M, const cplx r[4], int i, int j) {
  for (int k = 0; k < 3; ++k) {
    const cplx a = M->m[i][k], b = M->m[j][k];
    M->m[i][k] = cadd(cmul(r[0], a), cmul(r[1], b));
    M->m[j][k] = cadd(cmul(r[2], a), cmul(r[3], b));
  }
}

static void su2_heatbath(uint64_t* s, const su3* W, int i, int j, double beta, cplx r[4]) {
  const cplx w00 = W->m[i][i], w01 = W->m[i][j], w10 = W->m[j][i], w11 = W->m[j][j];
  const double b0 = 0.5 * (w00.re + w11.re);
  const double b3 = 0.5 * (w00.im - w11.im);
  const double b1 = 0.5 * (w01.im + w10.im);
  const double b2 = 0.5 * (w01.re - w10.re);
  double k = sqrt((b0 * b0 + b1 * b1) + (b2 * b2 + b3 * b3));
  if (k < 1e-300) k = 1e-300;
  /* V = (b0 + i b.sigma) / k;  V^+ entries */
  const cplx vd00 = {b0 / k, -b3 / k}, vd01 = {-b2 / k, -b1 / k};
  const cplx vd10 = {b2 / k, -b1 / k}, vd11 = {b0 / k, b3 / k};
  const double x0 = kp_x0(s, 2.0 * beta * k / 3.0);
  double rad = 1.0 - x0 * x0;
  rad = rad > 0.0 ? sqrt(rad) : 0.0;
  double d[3];
  unit_vector(s, d);
  const double x1 = rad * d[0], x2 = rad * d[1], x3 = rad * d[2];
  /* X = [[x0 + i x3, x2 + i x1], [-x2 + i x1, x0 - i x3]];  r = X V^+ */
  const cplx X00 = {x0, x3}, X01 = {x2, x1}, X10 = {-x2, x1}, X11 = {x0, -x3};
  r[0] = cadd(cmul(X00, vd00), cmul(X01, vd10));
  r[1] = cadd(cmul(X00, vd01), cmul(X01, vd11));
  r[2] = cadd(cmul(X10, vd00), cmul(X11, vd10));
  r[3] = cadd(cmul(X10, vd01), cmul(X11, vd11));
}

static void reunitarize(su3* u) {
  cplx* r0 = u->m[0];
  cplx* r1 = u->m[1];
  double n0 = sqrt((r0[0].re * r0[0].re + r0[0].im * r0[0].im) + (r0[1].re * r0[1].re + r0[1].im * r0[1].im) +
                   (r0[2].re * r0[2].re + r0[2].im * r0[2].im));
  for (int c = 0; c < 3; ++c) {
    r0[c].re = r0[c].re / n0;
    r0[c].im = r0[c].im / n0;
  }
  cplx dt = cmul(cconj(r0[0]), r1[0]);
  dt = cadd(dt, cmul(cconj(r0[1]), r1[1]));
  dt = cadd(dt, cmul(cconj(r0[2]), r1[2]));
  for (int c = 0; c < 3; ++c) r1[c] = csub(r1[c], cmul(dt, r0[c]));
  double n1 = sqrt((r1[0].re * r1[0].re + r1[0].im * r1[0].im) + (r1[1].re * r1[1].re + r1[1].im * r1[1].im) +
                   (r1[2].re * r1[2].re + r1[2].im * r1[2].im));
  for (int c = 0; c < 3; ++c) {
    r1[c].re = r1[c].re / n1;
    r1[c].im = r1[c].im / n1;
  }
  u->m[2][0] = cconj(csub(cmul(r0[1], r1[2]), cmul(r0[2], r1[1])));
  u->m[2][1] = cconj(csub(cmul(r0[2], r1[0]), cmul(r0[0], r1[2])));
  u->m[2][2] = cconj(csub(cmul(r0[0], r1[1]), cmul(r0[1], r1[0])));
}

/* Fill U (caller-owned, 4 V 9 complex) with the field after `sweeps` sweeps.  Returns 0. */
int heatbath_su3(double* U, const int dims[4], double beta, int sweeps, uint64_t seed) {
  lattice g;
  for (int m = 0; m < 4; ++m) g.L[m] = dims[m];
  g.V = dims[0] * dims[1] * dims[2] * dims[3];
  g.U = (cplx*)U;
  su3 one;
  memset(&one, 0, sizeof(one));
  for (int a = 0; a < 3; ++a) one.m[a][a].re = 1.0;
  for (int mu = 0; mu < 4; ++mu)
    for (int n = 0; n < g.V; ++n) put(&g, mu, n, &one);
  uint64_t s = seed;
  static const int sub[3][2] = {{0, 1}, {1, 2}, {0, 2}};
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int mu = 0; mu < 4; ++mu)
      for (int par = 0; par < 2; ++par)
        for (int n = 0; n < g.V; ++n) {
          int q = n, c0 = q % g.L[0];
          q /= g.L[0];
          int c1 = q % g.L[1];
          q /= g.L[1];
          int c2 = q % g.L[2], c3 = q / g.L[2];
          if (((c0 + c1 + c2 + c3) & 1) != par) continue;
          su3 A = staple_sum(&g, mu, n);
          su3 M = get(&g, mu, n);
          su3 W = mm(&M, &A);
          for (int k = 0; k < 3; ++k) {
            cplx r[4];
            su2_heatbath(&s, &W, sub[k][0], sub[k][1], beta, r);
            left_su2(&M, r, sub[k][0], sub[k][1]);
            left_su2(&W, r, sub[k][0], sub[k][1]);
          }
          put(&g, mu, n, &M);
        }
    for (int mu = 0; mu < 4; ++mu)
      for (int n = 0; n < g.V; ++n) {
        su3 u = get(&g, mu, n);
        reunitarize(&u);
        put(&g, mu, n, &u);
      }
  }
  return 0;
}
