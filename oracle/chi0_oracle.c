/*
 * chi0_oracle.c -- plain, slow FP64 CPU oracle for the bare susceptibility chi0(q, w).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py (its
 * cpu_baseline leg and `--impl reference`) load this library.  It shares no code,
 * header, table or helper with the CUDA library; neither includes the other.
 *
 * What it computes (Heil, Sormann, Boeri, Aichhorn, von der Linden, "Accurate bare
 * susceptibilities from full-potential ab initio calculations", Sec. II):
 *
 *   Re chi0(q,w) = sum_{n,m} int_1BZ dk/(4 pi^3) Th(eF - e^m_k) Th(e^n_{k+q} - eF) |M_mn|^2
 *                     [ 1/(e^m_k - e^n_{k+q} + w) + 1/(e^m_k - e^n_{k+q} - w) ]      (Eq. 1)
 *   Im chi0(q,w) = -sum_{n,m} int dk/(4 pi^2) Th Th |M_mn|^2 delta(w + e^m_k - e^n_{k+q})  (Eq. 2)
 *   Im chi0(q,-w) = -Im chi0(q,w)                                                      (Eq. 3)
 *
 * with e^m_k, e^n_{k+q} and |M_mn|^2 all linearly interpolated inside every tetrahedron
 * of the k mesh (Sec. II: energies and matrix elements "on equal footing").  The steps
 * follow Sec. II in its order:
 *   1. first carving: keep the part of a tetrahedron with a = e^m - eF < 0 (Sec. II,
 *      Fig. 1a->b); empty tetrahedra vanish, full ones stay, cut ones are split into
 *      fully occupied sub-tetrahedra;
 *   2. second carving: the same cut for b = e^n_{k+q} - eF > 0 on every piece
 *      (Sec. II, Eq. 4, Fig. 1b->c), leaving at most 9 final tetrahedra on which
 *      Th*Th = 1;
 *   3. integration over the final tetrahedra.  The paper does not print its formulas
 *      ("a simpler set of integration formulas", Sec. II); this file uses the exact
 *      closed forms for linear integrands on a simplex (Hermite-Genocchi):
 *        (1/V) int_S lambda_j h(D) = g[d1, d2, d3, d4, d_j]   with g'''' = h,
 *      a fourth divided difference with the knot d_j repeated.  For h = 1/x,
 *      g(x) = x^3 ln|x| (PV for the real part); for h = delta(w - x) the divided
 *      difference is the cubic B-spline density M(w; d1..d4, d_j)/4.
 *
 * Output sign: sign=0 ("positive") returns -(Eq. 1) and -(Eq. 2), so the static chi0 is
 * positive and Im >= 0 for w > 0; sign=1 returns Eq. 1 and Eq. 2 as printed.
 * Normalisation: k is integrated in fractional coordinates (BZ volume 1), chi0 is per
 * cell and includes both spins: dk/(4 pi^3) over the BZ = 2 * d(fractional k).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_RHO 0.25              /* Taylor branch when knot spread <= RHO * |knot| */
#define ORC_TMAX 400              /* Taylor terms, hard cap */
#define ORC_FLOOR 9.313225746154785e-10 /* 2^-30: exact-zero knots with >= 3 zeros */

/* ============================================================================
 * divided differences of g(x) = x^3 ln|x|  (g(0) = 0)
 * ========================================================================== */
static double g0(double x) { return x == 0.0 ? 0.0 : x * x * x * log(fabs(x)); }

/* g^{(k)}(c) / k!  for c != 0 */
static double gtay(int k, double c) {
  double L = log(fabs(c));
  switch (k) {
  case 0: return c * c * c * L;
  case 1: return 3.0 * c * c * L + c * c;
  case 2: return (6.0 * c * L + 5.0 * c) / 2.0;
  case 3: return (6.0 * L + 11.0) / 6.0;
  default: {
    /* g^{(k)} = 6 (-1)^{k-4} (k-4)! / x^{k-3}  ->  / k! */
    double kk = (double)k;
    double v = 6.0 / (kk * (kk - 1.0) * (kk - 2.0) * (kk - 3.0)) / pow(c, (double)(k - 3));
    return ((k - 4) & 1) ? -v : v;
  }
  }
}

/* Divided difference over knots t[i..j] (one cluster away from 0) as the Taylor series
 * about their mean c:  g[t_i..t_j] = sum_{k>=n} g^{(k)}(c)/k! h_{k-n}(t_i-c, ..., t_j-c),
 * h_m the complete homogeneous symmetric polynomial of degree m. */
static double dd_taylor(const double *t, int i, int j) {
  int n = j - i, l, k;
  double c = 0.0, d[8], h[8], sum = 0.0, big = 0.0, prev = 0.0;
  for (l = i; l <= j; ++l) c += t[l];
  c /= (double)(n + 1);
  for (l = 0; l <= n; ++l) { d[l] = t[i + l] - c; h[l] = 1.0; }
  for (k = n; k < n + ORC_TMAX; ++k) {
    int m = k - n;
    double term;
    if (m > 0) {
      h[0] = d[0] * h[0];
      for (l = 1; l <= n; ++l) h[l] = h[l - 1] + d[l] * h[l];
    }
    term = gtay(k, c) * h[n];
    sum += term;
    if (fabs(term) > big) big = fabs(term);
    /* odd-degree h_m of mean-centred knots can vanish: stop on two small terms in a row */
    if (k >= 5 && m >= 2 &&
        fabs(term) + fabs(prev) <= 1e-18 * (fabs(sum) > big ? fabs(sum) : big)) break;
    prev = term;
  }
  return sum;
}

typedef struct {
  double t[5];
  double v[5][5];
  unsigned char have[5][5];
} ddtab;

/* g[t_i..t_j] for sorted knots: the recursion (g[t_{i+1}..t_j] - g[t_i..t_{j-1}])/(t_j - t_i)
 * where the end knots are far apart; the Taylor series where they cluster away from 0;
 * derivatives where knots coincide. */
static double dd_get(ddtab *T, int i, int j) {
  double r, ti, tj;
  if (T->have[i][j]) return T->v[i][j];
  ti = T->t[i];
  tj = T->t[j];
  if (i == j) {
    r = g0(ti);
  } else if (ti == tj) {
    /* all knots equal: g^{(n)}(t)/n!; at t = 0 this is 0 for n <= 2, divergent beyond */
    r = (ti == 0.0) ? ((j - i) <= 2 ? 0.0 : NAN) : gtay(j - i, ti);
  } else if ((ti > 0.0 && tj - ti <= ORC_RHO * ti) || (tj < 0.0 && tj - ti <= ORC_RHO * (-tj))) {
    r = dd_taylor(T->t, i, j);
  } else {
    r = (dd_get(T, i + 1, j) - dd_get(T, i, j - 1)) / (tj - ti);
  }
  T->v[i][j] = r;
  T->have[i][j] = 1;
  return r;
}

static void sort_small(double *x, int n) {
  int i, j;
  for (i = 1; i < n; ++i) {
    double v = x[i];
    for (j = i - 1; j >= 0 && x[j] > v; --j) x[j + 1] = x[j];
    x[j + 1] = v;
  }
}

/* (1/V) int_S lambda_j / X over a simplex S whose linear function X has vertex values
 * x[0..3] (principal value if X changes sign): = g[x0,x1,x2,x3,x_j], g = x^3 ln|x|.
 * Knots are scaled by s = max|x| (g[s u] = g[u]/s for a fourth difference). */
double oracle_inv_weight(const double x_in[4], int j) {
  double x[4], s = 0.0, t[5];
  int i, nz = 0;
  ddtab T;
  for (i = 0; i < 4; ++i) {
    x[i] = x_in[i];
    if (fabs(x[i]) > s) s = fabs(x[i]);
    if (x[i] == 0.0) ++nz;
  }
  if (s == 0.0) return 0.0;
  if (nz >= 3) /* face on X = 0: log-divergent, floored (measure-zero input) */
    for (i = 0; i < 4; ++i)
      if (x[i] == 0.0) x[i] = ORC_FLOOR * s;
  for (i = 0; i < 4; ++i) t[i] = x[i] / s;
  t[4] = x[j] / s;
  sort_small(t, 5);
  memset(&T, 0, sizeof(T));
  memcpy(T.t, t, sizeof(t));
  return dd_get(&T, 0, 4) / s;
}

/* Normalised B-spline density M(x; t_0..t_{nk-1}) of order nk-1 (integral 1), by the
 * de Boor-Cox recursion for M-splines; half-open support [t_0, t_{nk-1}). */
double oracle_mspline(const double *t_in, int nk, double x) {
  double t[8], M[8];
  int i, k;
  for (i = 0; i < nk; ++i) t[i] = t_in[i];
  sort_small(t, nk);
  for (i = 0; i < nk - 1; ++i) M[i] = (t[i] <= x && x < t[i + 1]) ? 1.0 / (t[i + 1] - t[i]) : 0.0;
  for (k = 2; k <= nk - 1; ++k)
    for (i = 0; i < nk - k; ++i) {
      double den = t[i + k] - t[i];
      M[i] = den > 0.0 ? (double)k * ((x - t[i]) * M[i] + (t[i + k] - x) * M[i + 1]) /
                             ((double)(k - 1) * den)
                       : 0.0;
    }
  return M[0];
}

/* (1/V) int_S lambda_j delta(w - D) = M(w; d0..d3, d_j) / 4 */
double oracle_delta_weight(const double d[4], int j, double w) {
  double t[5] = {d[0], d[1], d[2], d[3], d[j]};
  return 0.25 * oracle_mspline(t, 5, w);
}

/* ============================================================================
 * carving (Sec. II)
 * ========================================================================== */
/* vertex of a (carved) tetrahedron: a = e^m_k - eF, D = e^n_{k+q} - e^m_k (so that
 * b = e^n_{k+q} - eF = a + D), f = |M|^2, all linear; D is carried as its own attribute
 * so that it vanishes exactly wherever it vanishes at the corners */
typedef struct {
  double a, D, f;
  double l[4]; /* barycentric coordinates in the parent tetrahedron */
} vtx;

static void vmix(const vtx *P, const vtx *Q, double t, vtx *R) {
  int i;
  R->a = (1.0 - t) * P->a + t * Q->a;
  R->D = (1.0 - t) * P->D + t * Q->D;
  R->f = (1.0 - t) * P->f + t * Q->f;
  for (i = 0; i < 4; ++i) R->l[i] = (1.0 - t) * P->l[i] + t * Q->l[i];
}

static double vkey(const vtx *v, int which) { return which == 0 ? v->a : -(v->a + v->D); }

/* Point on edge P-Q where the cut function vanishes; key(P) < 0 <= key(Q). */
static void vcut(const vtx *P, const vtx *Q, int which, vtx *R) {
  double kp = vkey(P, which), kq = vkey(Q, which);
  double t = kp / (kp - kq);
  vmix(P, Q, t, R);
  if (which == 0) R->a = 0.0; /* on the first cut plane; the second cut is the last one */
}

/* Keep the part of tetrahedron T where key < 0 (which = 0: a < 0, first carving;
 * which = 1: b > 0, second carving).  Returns 0, 1 or 3 pieces. */
int oracle_cut(const void *Tv, int which, void *outv) {
  const vtx *T = (const vtx *)Tv;
  vtx(*out)[4] = (vtx(*)[4])outv;
  vtx S[4];
  int o[4] = {0, 1, 2, 3}, i, j, nneg = 0;
  /* order vertices by the cut function */
  for (i = 1; i < 4; ++i) {
    int v = o[i];
    for (j = i - 1; j >= 0 && vkey(&T[o[j]], which) > vkey(&T[v], which); --j) o[j + 1] = o[j];
    o[j + 1] = v;
  }
  for (i = 0; i < 4; ++i) {
    S[i] = T[o[i]];
    if (vkey(&S[i], which) < 0.0) ++nneg;
  }
  switch (nneg) {
  case 0: return 0;
  case 4:
    for (i = 0; i < 4; ++i) out[0][i] = S[i];
    return 1;
  case 1: /* corner tetrahedron at S0 */
    out[0][0] = S[0];
    vcut(&S[0], &S[1], which, &out[0][1]);
    vcut(&S[0], &S[2], which, &out[0][2]);
    vcut(&S[0], &S[3], which, &out[0][3]);
    return 1;
  case 2: { /* prism with triangles (S0,P02,P03) and (S1,P12,P13) */
    vtx P02, P03, P12, P13;
    vcut(&S[0], &S[2], which, &P02);
    vcut(&S[0], &S[3], which, &P03);
    vcut(&S[1], &S[2], which, &P12);
    vcut(&S[1], &S[3], which, &P13);
    out[0][0] = S[0]; out[0][1] = P02; out[0][2] = P03; out[0][3] = S[1];
    out[1][0] = P02;  out[1][1] = P03; out[1][2] = S[1]; out[1][3] = P12;
    out[2][0] = P03;  out[2][1] = S[1]; out[2][2] = P12; out[2][3] = P13;
    return 3;
  }
  case 3: { /* tetrahedron minus the corner at S3: prism (S0,S1,S2)-(P03,P13,P23) */
    vtx P03, P13, P23;
    vcut(&S[0], &S[3], which, &P03);
    vcut(&S[1], &S[3], which, &P13);
    vcut(&S[2], &S[3], which, &P23);
    out[0][0] = S[0]; out[0][1] = S[1]; out[0][2] = S[2]; out[0][3] = P03;
    out[1][0] = S[1]; out[1][1] = S[2]; out[1][2] = P03;  out[1][3] = P13;
    out[2][0] = S[2]; out[2][1] = P03;  out[2][2] = P13;  out[2][3] = P23;
    return 3;
  }
  }
  return 0;
}

/* volume of a piece relative to its parent tetrahedron: |det| of barycentric differences */
static double vfrac(const vtx *P) {
  double m[3][3];
  int r, c;
  for (r = 0; r < 3; ++r)
    for (c = 0; c < 3; ++c) m[r][c] = P[r + 1].l[c + 1] - P[0].l[c + 1];
  return fabs(m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
              m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
              m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]));
}

/* Final tetrahedra of one (tetrahedron, band pair): volumes (relative), D = b - a and f at
 * their vertices.  Returns the count (<= 9). */
int oracle_carve(const double a[4], const double b[4], const double f[4], double *vol,
                 double *dv, double *fv) {
  vtx T[4], P1[3][4], P2[3][4];
  int i, n1, p, n2, q, nout = 0;
  for (i = 0; i < 4; ++i) {
    T[i].a = a[i];
    T[i].D = b[i] - a[i];
    T[i].f = f[i];
    memset(T[i].l, 0, sizeof(T[i].l));
    T[i].l[i] = 1.0;
  }
  n1 = oracle_cut(T, 0, P1);
  for (p = 0; p < n1; ++p) {
    n2 = oracle_cut(P1[p], 1, P2);
    for (q = 0; q < n2; ++q) {
      vol[nout] = vfrac(P2[q]);
      for (i = 0; i < 4; ++i) {
        double d = P2[q][i].D;
        dv[4 * nout + i] = d > 0.0 ? d : 0.0;
        fv[4 * nout + i] = P2[q][i].f;
      }
      ++nout;
    }
  }
  return nout;
}

/* ============================================================================
 * one tetrahedron, one band pair
 * ========================================================================== */
/* Neumaier-compensated accumulator */
typedef struct { double s, c; } acc_t;
static void acc_add(acc_t *A, double x) {
  double t = A->s + x;
  if (fabs(A->s) >= fabs(x)) A->c += (A->s - t) + x;
  else A->c += (x - t) + A->s;
  A->s = t;
}
static double acc_val(const acc_t *A) { return A->s + A->c; }

/* Adds the POSITIVE-sign integrals over the tetrahedron (relative volume 1 times `vol`):
 *   nw == 0:  re[0] += vol * int f * 2/D           (static, w = 0)
 *   nw  > 0:  re[k] += vol * int f [1/(D-w_k) + 1/(D+w_k)]   (PV)
 *             im[k] += vol * pi * int f delta(|w_k| - D) * sgn(w_k)   (Eq. 3 for w < 0)
 * over the carved region a < 0 < b. */
static void tet_pair(const double a[4], const double b[4], const double f[4], double vol, int nw,
                     const double *w, acc_t *re, acc_t *im) {
  double V[9], D[36], F[36];
  int ns = oracle_carve(a, b, f, V, D, F), s, j, k;
  for (s = 0; s < ns; ++s) {
    const double *d = D + 4 * s, *ff = F + 4 * s;
    double vs = vol * V[s];
    if (vs == 0.0) continue;
    if (nw == 0) {
      double acc = 0.0;
      for (j = 0; j < 4; ++j) acc += ff[j] * 2.0 * oracle_inv_weight(d, j);
      acc_add(&re[0], vs * acc);
      continue;
    }
    for (k = 0; k < nw; ++k) {
      double wk = w[k], aw = fabs(wk), xm[4], xp[4], r = 0.0, m = 0.0;
      for (j = 0; j < 4; ++j) { xm[j] = d[j] - aw; xp[j] = d[j] + aw; }
      for (j = 0; j < 4; ++j) {
        r += ff[j] * (oracle_inv_weight(xm, j) + oracle_inv_weight(xp, j));
        if (aw > 0.0) m += ff[j] * oracle_delta_weight(d, j, aw);
      }
      acc_add(&re[k], vs * r);
      if (aw > 0.0) acc_add(&im[k], (wk < 0.0 ? -1.0 : 1.0) * vs * M_PI * m);
    }
  }
}

/* Tetrahedron DOS at eF for one band: (1/V) int delta(a) = M(0; a0..a3) (order 3). */
double oracle_tet_dos(const double a[4]) { return oracle_mspline(a, 4, 0.0); }

/* single-tetrahedron entry point for tests (relative volume 1) */
void oracle_tet_integrals(const double a[4], const double b[4], const double f[4], int nw,
                          const double *w, double *re, double *im) {
  int k, n = nw == 0 ? 1 : nw;
  acc_t *R = (acc_t *)calloc((size_t)n, sizeof(acc_t)), *I = (acc_t *)calloc((size_t)n, sizeof(acc_t));
  if (R && I) {
    tet_pair(a, b, f, 1.0, nw, w, R, I);
    for (k = 0; k < n; ++k) {
      re[k] = acc_val(&R[k]);
      if (im && nw > 0) im[k] = acc_val(&I[k]);
    }
  } else {
    for (k = 0; k < n; ++k) {
      re[k] = NAN;
      if (im && nw > 0) im[k] = NAN;
    }
  }
  free(R);
  free(I);
}

/* ============================================================================
 * full chi0 for one q
 * ========================================================================== */
typedef struct {
  int n[3];
  int periodic;
  int nb, norb;
  const double *E;  /* [Nc][nb] */
  const double *C;  /* [Nc][norb][nb][2] complex128, NULL for |M|^2 = 1 */
  const double *Eq; /* [Nc][nb] at k+q, NULL -> shift */
  const double *Cq; /* [Nc][norb][nb][2] at k+q, NULL -> shift */
  int shift[3];
  double ef;
  int lo, hi;       /* band window, both m and n */
  int cma;
  int gamma;        /* add the q -> 0 intraband limit N(eF) (static / w = 0 only) */
  int ntet;         /* 0 -> builtin 6 tetrahedra per cube */
  const int32_t *tet;   /* [ntet][4] corner indices */
  const double *tvol;   /* [ntet] fractional volumes */
  int nw;           /* 0 -> static */
  const double *omega;
  int sign;         /* 0 positive, 1 as printed in Eqs. 1-2 */
  int nthreads;
} oracle_input;

/* Builtin mesh: each cube (i0,i1,i2) splits into 6 tetrahedra around its (000)-(111)
 * diagonal, one per axis order (p0,p1,p2) in lexicographic order:
 * {000, e_p0, e_p0+e_p1, 111}. */
static const int PERM[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

static void corner_dims(const oracle_input *in, int N[3]) {
  int d;
  for (d = 0; d < 3; ++d) N[d] = in->periodic ? in->n[d] : in->n[d] + 1;
}

static int64_t corner_id(const oracle_input *in, const int N[3], int i0, int i1, int i2) {
  if (in->periodic) {
    i0 %= N[0]; i1 %= N[1]; i2 %= N[2];
  }
  return ((int64_t)i0 * N[1] + i1) * N[2] + i2;
}

static void builtin_tet(const oracle_input *in, const int N[3], int64_t t, int64_t c[4]) {
  int64_t cube = t / 6;
  int p = (int)(t % 6), i2 = (int)(cube % in->n[2]), i1 = (int)((cube / in->n[2]) % in->n[1]),
      i0 = (int)(cube / ((int64_t)in->n[2] * in->n[1]));
  int o[3] = {0, 0, 0};
  c[0] = corner_id(in, N, i0, i1, i2);
  o[PERM[p][0]] = 1;
  c[1] = corner_id(in, N, i0 + o[0], i1 + o[1], i2 + o[2]);
  o[PERM[p][1]] = 1;
  c[2] = corner_id(in, N, i0 + o[0], i1 + o[1], i2 + o[2]);
  c[3] = corner_id(in, N, i0 + 1, i1 + 1, i2 + 1);
}

static int64_t shifted(const oracle_input *in, const int N[3], int64_t c) {
  int i2 = (int)(c % N[2]), i1 = (int)((c / N[2]) % N[1]), i0 = (int)(c / ((int64_t)N[2] * N[1]));
  return corner_id(in, N, i0 + in->shift[0], i1 + in->shift[1], i2 + in->shift[2]);
}

/* |M_mn|^2 = |sum_o conj(C[k][o][m]) C[k+q][o][n]|^2 (Eq. 1; tight-binding form of the
 * matrix element with orbitals at the cell origin) */
static double msq(const oracle_input *in, int64_t ck, int64_t ckq, const double *Ck,
                  const double *Ckq, int m, int n) {
  double re = 0.0, im = 0.0;
  int o, nb = in->nb;
  for (o = 0; o < in->norb; ++o) {
    const double *x = Ck + 2 * (((int64_t)ck * in->norb + o) * nb + m);
    const double *y = Ckq + 2 * (((int64_t)ckq * in->norb + o) * nb + n);
    re += x[0] * y[0] + x[1] * y[1];
    im += x[0] * y[1] - x[1] * y[0];
  }
  return re * re + im * im;
}

/* Returns 0 on success.  re/im: [nw] (static: re[0] only). */
int oracle_chi0(const oracle_input *in, double *re_out, double *im_out) {
  int N[3], nw = in->nw, nout = in->nw == 0 ? 1 : in->nw, nth = 1;
  int64_t ntet, t;
  double vol_builtin;
  acc_t *accR, *accI;
  const double *Eq, *Cq;
  if (!in || !in->E || in->nb <= 0 || in->lo < 0 || in->hi > in->nb || in->lo >= in->hi) return -1;
  if (!in->cma && !in->C) return -1;
  if (!in->periodic && !in->Eq) return -1;
  corner_dims(in, N);
  ntet = in->ntet > 0 ? in->ntet : 6LL * in->n[0] * in->n[1] * in->n[2];
  vol_builtin = 1.0 / (6.0 * in->n[0] * in->n[1] * in->n[2]);
  Eq = in->Eq ? in->Eq : in->E;
  Cq = in->Eq ? in->Cq : in->C; /* explicit energies imply explicit vectors */
  if (!in->cma && !Cq) return -1;
#ifdef _OPENMP
  nth = in->nthreads > 0 ? in->nthreads : omp_get_max_threads();
#endif
  accR = (acc_t *)calloc((size_t)nth * nout, sizeof(acc_t));
  accI = (acc_t *)calloc((size_t)nth * nout, sizeof(acc_t));
  if (!accR || !accI) { free(accR); free(accI); return -2; }

#pragma omp parallel for schedule(dynamic, 256) num_threads(nth)
  for (t = 0; t < ntet; ++t) {
    int tid = 0, i, m, n;
    int64_t c[4], cq[4];
    double vol;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    if (in->ntet > 0) {
      for (i = 0; i < 4; ++i) c[i] = in->tet[4 * t + i];
      vol = in->tvol[t];
    } else {
      builtin_tet(in, N, t, c);
      vol = vol_builtin;
    }
    for (i = 0; i < 4; ++i) cq[i] = in->Eq ? c[i] : shifted(in, N, c[i]);
    for (m = in->lo; m < in->hi; ++m) {
      double a[4], amin = 1e300;
      for (i = 0; i < 4; ++i) {
        a[i] = in->E[c[i] * in->nb + m] - in->ef;
        if (a[i] < amin) amin = a[i];
      }
      if (!(amin < 0.0)) continue; /* no occupied part */
      for (n = in->lo; n < in->hi; ++n) {
        double b[4], f[4], bmax = -1e300;
        /* at Gamma the intraband region of Eq. 1 is empty; its q -> 0 limit is added below */
        if (in->gamma && n == m) continue;
        for (i = 0; i < 4; ++i) {
          b[i] = Eq[cq[i] * in->nb + n] - in->ef;
          if (b[i] > bmax) bmax = b[i];
        }
        if (!(bmax > 0.0)) continue; /* no empty part */
        for (i = 0; i < 4; ++i) f[i] = in->cma ? 1.0 : msq(in, c[i], cq[i], in->C, Cq, m, n);
        tet_pair(a, b, f, vol, nw, in->omega, accR + (size_t)tid * nout, accI + (size_t)tid * nout);
      }
    }
  }

  {
    int k, th;
    double sgn = in->sign ? -1.0 : 1.0;
    for (k = 0; k < nout; ++k) {
      acc_t R = {0, 0}, I = {0, 0};
      for (th = 0; th < nth; ++th) {
        acc_add(&R, acc_val(&accR[(size_t)th * nout + k]));
        acc_add(&I, acc_val(&accI[(size_t)th * nout + k]));
      }
      re_out[k] = sgn * 2.0 * acc_val(&R);
      if (im_out && nw > 0) im_out[k] = sgn * 2.0 * acc_val(&I);
    }
  }
  /* q -> 0 intraband limit: N(eF) = 2 sum_t sum_n V_t M(0; a) (Sec. III: chi0 must reach
   * the density of states at eF); added to the static value and to Re at w = 0 */
  if (in->gamma) {
    acc_t G = {0, 0};
    double sgn = in->sign ? -1.0 : 1.0;
    int k;
    for (t = 0; t < ntet; ++t) {
      int64_t c[4];
      double vol, a[4];
      int i, m;
      if (in->ntet > 0) {
        for (i = 0; i < 4; ++i) c[i] = in->tet[4 * t + i];
        vol = in->tvol[t];
      } else {
        builtin_tet(in, N, t, c);
        vol = vol_builtin;
      }
      for (m = in->lo; m < in->hi; ++m) {
        for (i = 0; i < 4; ++i) a[i] = in->E[c[i] * in->nb + m] - in->ef;
        acc_add(&G, vol * oracle_tet_dos(a));
      }
    }
    for (k = 0; k < nout; ++k)
      if (nw == 0 || in->omega[k] == 0.0) re_out[k] += sgn * 2.0 * acc_val(&G);
  }
  free(accR);
  free(accI);
  return 0;
}

/* Static chi0 resolved by band pair (Sec. III, Fig. 8: the contribution of the transitions
 * m -> n): pairs[(m - lo) * w + (n - lo)], w = hi - lo, the same sum as oracle_chi0 at w = 0
 * (same normalisation and sign) taken per (m, n); at Gamma the q -> 0 limit N(eF) of band m
 * goes to the pair (m, m).  Returns 0 on success. */
int oracle_chi0_pairs(const oracle_input *in, double *pairs) {
  int N[3], w, nth = 1;
  int64_t ntet, t;
  double vol_builtin, sgn;
  acc_t *P;
  const double *Eq, *Cq;
  if (!in || !pairs || in->nw != 0 || !in->E || in->nb <= 0 || in->lo < 0 || in->hi > in->nb ||
      in->lo >= in->hi)
    return -1;
  if (!in->cma && !in->C) return -1;
  if (!in->periodic && !in->Eq) return -1;
  corner_dims(in, N);
  w = in->hi - in->lo;
  ntet = in->ntet > 0 ? in->ntet : 6LL * in->n[0] * in->n[1] * in->n[2];
  vol_builtin = 1.0 / (6.0 * in->n[0] * in->n[1] * in->n[2]);
  Eq = in->Eq ? in->Eq : in->E;
  Cq = in->Eq ? in->Cq : in->C;
  if (!in->cma && !Cq) return -1;
#ifdef _OPENMP
  nth = in->nthreads > 0 ? in->nthreads : omp_get_max_threads();
#endif
  P = (acc_t *)calloc((size_t)nth * w * w, sizeof(acc_t));
  if (!P) return -2;

#pragma omp parallel for schedule(dynamic, 256) num_threads(nth)
  for (t = 0; t < ntet; ++t) {
    int tid = 0, i, m, n;
    int64_t c[4], cq[4];
    double vol;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    if (in->ntet > 0) {
      for (i = 0; i < 4; ++i) c[i] = in->tet[4 * t + i];
      vol = in->tvol[t];
    } else {
      builtin_tet(in, N, t, c);
      vol = vol_builtin;
    }
    for (i = 0; i < 4; ++i) cq[i] = in->Eq ? c[i] : shifted(in, N, c[i]);
    for (m = in->lo; m < in->hi; ++m) {
      double a[4], amin = 1e300;
      for (i = 0; i < 4; ++i) {
        a[i] = in->E[c[i] * in->nb + m] - in->ef;
        if (a[i] < amin) amin = a[i];
      }
      if (!(amin < 0.0)) continue;
      for (n = in->lo; n < in->hi; ++n) {
        double b[4], f[4], bmax = -1e300;
        acc_t one = {0, 0}, none = {0, 0};
        if (in->gamma && n == m) continue;
        for (i = 0; i < 4; ++i) {
          b[i] = Eq[cq[i] * in->nb + n] - in->ef;
          if (b[i] > bmax) bmax = b[i];
        }
        if (!(bmax > 0.0)) continue;
        for (i = 0; i < 4; ++i) f[i] = in->cma ? 1.0 : msq(in, c[i], cq[i], in->C, Cq, m, n);
        tet_pair(a, b, f, vol, 0, NULL, &one, &none);
        acc_add(&P[((size_t)tid * w + (m - in->lo)) * w + (n - in->lo)], acc_val(&one));
      }
    }
  }

  sgn = in->sign ? -1.0 : 1.0;
  {
    int k, th;
    for (k = 0; k < w * w; ++k) {
      acc_t R = {0, 0};
      for (th = 0; th < nth; ++th) acc_add(&R, acc_val(&P[(size_t)th * w * w + k]));
      pairs[k] = sgn * 2.0 * acc_val(&R);
    }
  }
  if (in->gamma) {
    int m;
    for (m = in->lo; m < in->hi; ++m) {
      acc_t G = {0, 0};
      for (t = 0; t < ntet; ++t) {
        int64_t c[4];
        double vol, a[4];
        int i;
        if (in->ntet > 0) {
          for (i = 0; i < 4; ++i) c[i] = in->tet[4 * t + i];
          vol = in->tvol[t];
        } else {
          builtin_tet(in, N, t, c);
          vol = vol_builtin;
        }
        for (i = 0; i < 4; ++i) a[i] = in->E[c[i] * in->nb + m] - in->ef;
        acc_add(&G, vol * oracle_tet_dos(a));
      }
      pairs[(m - in->lo) * (w + 1)] += sgn * 2.0 * acc_val(&G);
    }
  }
  free(P);
  return 0;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int oracle_input_size(void) { return (int)sizeof(oracle_input); }
