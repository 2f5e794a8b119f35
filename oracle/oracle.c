/*
 * ORACLE -- test infrastructure only.
 *
 * Plain, slow, FP64 (x87 long double where conditioning demands it) CPU
 * implementation of what the particle-wise higher-order SPH field
 * approximation (arXiv 2401.02896) computes.  Only the test-suite, the
 * package's smoke check and the benchmark's CPU-baseline leg may load this
 * file's shared library.  It shares no code with the CUDA path.
 *
 * Parts, in the paper's order:
 *   1. SPH kernels (Sec. 1, eq. "cubic-kernel"; Wendland C2/C4 and the poly6
 *      test kernel stand in for "any kernel with compact support").
 *   2. Optimal approximation of the unit-particle ray restriction
 *      B_L(t) = w(sqrt(L^2 + t^2)) (Sec. 3.1) by an even, continuous,
 *      compactly supported piecewise polynomial with K non-trivial pieces of
 *      degree <= D (Sec. 3.2): the non-orthogonal basis A~_kd, Gram-Schmidt
 *      in lexicographic order, the sum of projections (eq.
 *      "optimal-approx-for-given-knots"), and a global search over the
 *      positive knots (Sec. 3.4).  The result is the look-up table of Sec. 3.1.
 *   3. Per-ray field: candidates by brute force over all particles, the
 *      nearest table entry per candidate, the union of all knots, and on each
 *      resulting piece the field's localized coefficients by DIRECT summation
 *      of the overlapping contributions (Sec. 4.1, last alternative, and the
 *      localized-coefficient formula of Sec. 2).
 *   4. Classification and emission-absorption compositing (Sec. 1, DVR), done
 *      exactly: pieces are split at transfer-function node crossings (bisection
 *      on monotone sub-intervals), optical depth is integrated in closed form,
 *      emission by adaptive Gauss-Kronrod.  No early ray termination.
 *   5. Gradients (Conclusion: the scheme carries over to any feature that is a
 *      sum of particle contributions).  A particle's gradient at x(t) is
 *      (c / h^2) (w'(rho) / rho) ((t - t_chi) v - d) with d the vector from the
 *      ray to the particle (perpendicular to v) and rho = |x - chi| / h: along
 *      v it is the derivative of its contribution, across the ray it is
 *      -(c / h^2) d G_L((t - t_chi) / h) with G_L(s) = w'(rho) / rho, which is
 *      even and compactly supported like B_L.  G_L is approximated by the same
 *      projection (Sec. 3.3) on the table entry's own knots, so the
 *      perpendicular gradient of the ray is a piecewise polynomial with the
 *      same knots; the along-ray part is the derivative of the field's pieces.
 *      Shading (a reading: the paper names no model): the emitted colour is
 *      scaled by ka + kd |grad . v| / sqrt(|grad|^2 + g0^2) (a light along the ray;
 *      g0 >= 0 softens the cosine where the gradient is small, a reading).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef long double ld;

#define ORC_PI 3.14159265358979323846264338327950288L

enum { ORC_M4 = 0, ORC_WENDLAND_C2 = 1, ORC_WENDLAND_C4 = 2, ORC_POLY6 = 3 };

#define ORC_MAXM 4           /* positive knots per particle (K <= 8)      */
#define ORC_MAXD 7           /* polynomial degree                          */
#define ORC_MAXB (ORC_MAXM * ORC_MAXD)

/* ------------------------------------------------------------------------ */
/* 1. Kernels                                                                */
/* ------------------------------------------------------------------------ */

/* Support bound q of w (w(r) = 0 for r >= q), in units of the smoothing length. */
double orc_kernel_support(int kernel) { return kernel == ORC_POLY6 ? 1.0 : 2.0; }

/* w(r): Sec. 1 eq. (cubic-kernel) for M4; the other three are normalised in 3-D. */
static ld kernel_w(int kernel, ld r) {
  if (r < 0) r = -r;
  switch (kernel) {
    case ORC_M4:
      if (r < 1) return ((2 - r) * (2 - r) * (2 - r) - 4 * (1 - r) * (1 - r) * (1 - r)) / (4 * ORC_PI);
      if (r < 2) return (2 - r) * (2 - r) * (2 - r) / (4 * ORC_PI);
      return 0;
    case ORC_WENDLAND_C2:
      if (r < 2) { ld a = 1 - r / 2; return 21.0L / (16 * ORC_PI) * a * a * a * a * (2 * r + 1); }
      return 0;
    case ORC_WENDLAND_C4:
      if (r < 2) {
        ld a = 1 - r / 2, a2 = a * a;
        return 495.0L / (256 * ORC_PI) * a2 * a2 * a2 * (35.0L / 12 * r * r + 3 * r + 1);
      }
      return 0;
    case ORC_POLY6:
      if (r < 1) { ld a = 1 - r * r; return 315.0L / (64 * ORC_PI) * a * a * a; }
      return 0;
  }
  return 0;
}

double orc_kernel_w(int kernel, double r) { return (double)kernel_w(kernel, r); }

/* w'(r) / r, written in a form that is finite at r = 0 (derivatives of the
 * four kernels above). */
static ld kernel_dw_r(int kernel, ld r) {
  if (r < 0) r = -r;
  switch (kernel) {
    case ORC_M4:
      if (r < 1) return (-12 + 9 * r) / (4 * ORC_PI);
      if (r < 2) return -3 * (2 - r) * (2 - r) / (4 * ORC_PI * r);
      return 0;
    case ORC_WENDLAND_C2:
      if (r < 2) { ld a = 1 - r / 2; return -105.0L / (16 * ORC_PI) * a * a * a; }
      return 0;
    case ORC_WENDLAND_C4:
      if (r < 2) { ld a = 1 - r / 2, a2 = a * a; return -1155.0L / (256 * ORC_PI) * (5 * r + 2) * a2 * a2 * a; }
      return 0;
    case ORC_POLY6:
      if (r < 1) { ld a = 1 - r * r; return -945.0L / (32 * ORC_PI) * a * a; }
      return 0;
  }
  return 0;
}

double orc_kernel_dw_r(int kernel, double r) { return (double)kernel_dw_r(kernel, r); }

/* Radii inside (0, q) where w changes its polynomial piece. */
static int kernel_breaks(int kernel, ld* br) {
  if (kernel == ORC_M4) { br[0] = 1; return 1; }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre / Gauss-Kronrod rules                                      */
/* ------------------------------------------------------------------------ */

#define GL_N 20
static ld gl_x[GL_N], gl_w[GL_N];
static int gl_ready = 0;

/* Nodes/weights on [-1,1] by Newton iteration on the Legendre recurrence. */
static void gl_init(void) {
  if (gl_ready) return;
  for (int i = 0; i < GL_N; i++) {
    ld x = cosl(ORC_PI * (i + 0.75L) / (GL_N + 0.5L)), dp = 0;
    for (int it = 0; it < 100; it++) {
      ld p0 = 1, p1 = x;
      for (int k = 2; k <= GL_N; k++) { ld p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
      dp = GL_N * (x * p1 - p0) / (x * x - 1);
      ld dx = p1 / dp;
      x -= dx;
      if (fabsl(dx) < 1e-19L) break;
    }
    ld p0 = 1, p1 = x;
    for (int k = 2; k <= GL_N; k++) { ld p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
    dp = GL_N * (x * p1 - p0) / (x * x - 1);
    gl_x[i] = x;
    gl_w[i] = 2 / ((1 - x * x) * dp * dp);
  }
  gl_ready = 1;
}

/* Standard 7-point Gauss / 15-point Kronrod rule (abscissae on [0,1] half). */
static const double gk_x[8] = {0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
                               0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
                               0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
                               0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
static const double gk_wk[8] = {0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
                                0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
                                0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
                                0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double gk_wg[4] = {0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
                                0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

/* ------------------------------------------------------------------------ */
/* 2. Optimal approximation of B_L for given and for optimal knots           */
/* ------------------------------------------------------------------------ */

typedef struct {
  int kernel, K, D, m, middle;
  int target;             /* approximated function: 0 B_L(t) = w(rho), 1 G_L(t) = w'(rho) / rho */
  ld q, lam, T;           /* L and the half-length T = sqrt(q^2 - L^2) of supp B_L */
  int nsp;
  ld sp[96];              /* split points in (0, T]: grading near 0 + kernel breaks + T */
  ld BB;                  /* ||B_L||^2 over R */
  int nb;
  int bk[ORC_MAXB], bd[ORC_MAXB];  /* index set J in lexicographic order */
} lam_ctx;

static ld B_of(const lam_ctx* c, ld t) {
  const ld rho = sqrtl(c->lam * c->lam + t * t);
  return c->target ? kernel_dw_r(c->kernel, rho) : kernel_w(c->kernel, rho);
}

static int cmp_ld(const void* a, const void* b) {
  ld x = *(const ld*)a, y = *(const ld*)b;
  return x < y ? -1 : x > y;
}

static void lam_ctx_init(lam_ctx* c, int kernel, int K, int D, ld lam) {
  memset(c, 0, sizeof(*c));
  c->kernel = kernel; c->K = K; c->D = D;
  c->m = (K + 1) / 2; c->middle = (K % 2 == 0);
  c->q = orc_kernel_support(kernel);
  c->lam = lam;
  c->T = lam < c->q ? sqrtl(c->q * c->q - lam * lam) : 0;
  /* J: pairs (k,d), k = 1..m, d = 1..D, without (1, odd d) when K is odd (Sec. 3.3) */
  c->nb = 0;
  for (int k = 1; k <= c->m; k++)
    for (int d = 1; d <= D; d++) {
      if (k == 1 && (K % 2 == 1) && (d % 2 == 1)) continue;
      c->bk[c->nb] = k; c->bd[c->nb] = d; c->nb++;
    }
  /* B_L is analytic on [0,T] apart from kernel breaks, but sqrt(L^2+t^2) has
   * branch points at t = +-iL: grade the quadrature geometrically toward 0. */
  int n = 0;
  if (c->T > 0) {
    if (lam > 1e-9L) for (ld g = lam; g < c->T && n < 60; g *= 3) c->sp[n++] = g;
    ld br[4];
    int nbr = kernel_breaks(kernel, br);
    for (int i = 0; i < nbr; i++)
      if (br[i] > lam) { ld tb = sqrtl(br[i] * br[i] - lam * lam); if (tb > 0 && tb < c->T) c->sp[n++] = tb; }
    c->sp[n++] = c->T;
    qsort(c->sp, n, sizeof(ld), cmp_ld);
  }
  c->nsp = n;
}

/* Visit Gauss-Legendre nodes covering [a,b] ∩ [0,T], split at c->sp. */
typedef void (*node_fn)(void* u, ld t, ld w);
static void quad_nodes(const lam_ctx* c, ld a, ld b, node_fn f, void* u) {
  if (b > c->T) b = c->T;
  if (!(b > a)) return;
  ld lo = a;
  for (int i = 0; i <= c->nsp; i++) {
    ld hi = i < c->nsp ? c->sp[i] : b;
    if (hi > b) hi = b;
    if (hi > lo) {
      ld h = (hi - lo) / 2, mid = (hi + lo) / 2;
      for (int j = 0; j < GL_N; j++) f(u, mid + h * gl_x[j], h * gl_w[j]);
      lo = hi;
    }
    if (lo >= b) break;
  }
}

typedef struct { const lam_ctx* c; ld sum; } bb_acc;
static void acc_bb(void* u, ld t, ld w) { bb_acc* a = (bb_acc*)u; ld v = B_of(a->c, t); a->sum += w * v * v; }

typedef struct { const lam_ctx* c; ld t0, dt; int D; ld mom[ORC_MAXD + 1]; } mom_acc;
static void acc_mom(void* u, ld t, ld w) {
  mom_acc* a = (mom_acc*)u;
  ld v = B_of(a->c, t) * w, x = (t - a->t0) / a->dt, p = 1;
  for (int d = 0; d <= a->D; d++) { a->mom[d] += v * p; p *= x; }
}

/* Solution for fixed knots theta[0..m-1] (Sec. 3.3).  Returns the basis
 * coefficients coef[] (in J order) of the optimal S and ||B - S||^2. */
typedef struct {
  ld coef[ORC_MAXB];
  ld err2;
  int ok;
} fixed_sol;

/* S evaluated at |t| from basis coefficients (definition of A~_kd, Sec. 3.3). */
static ld basis_eval(int k, int d, const ld* th, ld t) {
  t = fabsl(t);
  ld a = k > 1 ? th[k - 2] : 0, b = th[k - 1];
  if (t <= a) return 1;
  if (t >= b) return 0;
  ld u = (t - a) / (b - a), p = 1;
  for (int i = 0; i < d; i++) p *= u;
  return 1 - p;
}

static ld S_eval(const lam_ctx* c, const ld* th, const ld* coef, ld t) {
  ld s = 0;
  for (int i = 0; i < c->nb; i++) s += coef[i] * basis_eval(c->bk[i], c->bd[i], th, t);
  return s;
}

typedef struct { const lam_ctx* c; const ld* th; const ld* coef; ld sum; } res_acc;
static void acc_res(void* u, ld t, ld w) {
  res_acc* a = (res_acc*)u;
  ld r = B_of(a->c, t) - S_eval(a->c, a->th, a->coef, t);
  a->sum += w * r * r;
}

static fixed_sol solve_fixed(const lam_ctx* c, const ld* th) {
  fixed_sol s;
  memset(&s, 0, sizeof(s));
  int nb = c->nb, m = c->m, D = c->D;
  for (int k = 0; k < m; k++) if (!(th[k] > (k ? th[k - 1] : 0))) return s;  /* 0 < th_1 < ... */
  /* Moments mu[k][d] = int_{th_{k-1}}^{th_k} ((t-th_{k-1})/Dk)^d B_L(t) dt. */
  ld mu[ORC_MAXM][ORC_MAXD + 1];
  for (int k = 0; k < m; k++) {
    mom_acc a;
    memset(&a, 0, sizeof(a));
    a.c = c; a.t0 = k ? th[k - 1] : 0; a.dt = th[k] - a.t0; a.D = D;
    quad_nodes(c, a.t0, th[k], acc_mom, &a);
    for (int d = 0; d <= D; d++) mu[k][d] = a.mom[d];
  }
  /* b_i = <A~_kd, B_L> = 2 [ int_0^{th_k} B - mu_k,d ]   (A~ = 1 below th_{k-1}) */
  ld b[ORC_MAXB], G[ORC_MAXB][ORC_MAXB];
  for (int i = 0; i < nb; i++) {
    int k = c->bk[i] - 1, d = c->bd[i];
    ld s = 0;
    for (int kk = 0; kk <= k; kk++) s += mu[kk][0];
    b[i] = 2 * (s - mu[k][d]);
  }
  /* Gram matrix <A~_kd, A~_k'd'> of the piecewise polynomial basis, integrated
   * piece by piece: both equal 1 on [0, th_{k-1}], on [th_{k-1}, th_k] the
   * lower-k function is 1-u^d, beyond th_k it vanishes. */
  for (int i = 0; i < nb; i++)
    for (int j = 0; j < nb; j++) {
      int k1 = c->bk[i], d1 = c->bd[i], k2 = c->bk[j], d2 = c->bd[j];
      int k = k1 < k2 ? k1 : k2;
      ld a0 = k > 1 ? th[k - 2] : 0, dk = th[k - 1] - a0, v;
      if (k1 != k2) {
        int dd = k1 < k2 ? d1 : d2;
        v = a0 + dk * (1 - 1.0L / (dd + 1));
      } else {
        v = a0 + dk * (1 - 1.0L / (d1 + 1) - 1.0L / (d2 + 1) + 1.0L / (d1 + d2 + 1));
      }
      G[i][j] = 2 * v;
    }
  /* Gram-Schmidt in lexicographic order of J (Sec. 3.3): phi_i = sum_l L[i][l] A~_l */
  ld L[ORC_MAXB][ORC_MAXB], gam[ORC_MAXB], beta[ORC_MAXB];
  memset(L, 0, sizeof(L));
  for (int i = 0; i < nb; i++) {
    L[i][i] = 1;
    for (int j = 0; j < i; j++) {
      ld ip = 0;  /* <A~_i, phi_j> */
      for (int l = 0; l <= j; l++) ip += L[j][l] * G[i][l];
      ld pr = ip / gam[j];
      for (int l = 0; l <= j; l++) L[i][l] -= pr * L[j][l];
    }
    ld g = 0;
    for (int l = 0; l <= i; l++)
      for (int l2 = 0; l2 <= i; l2++) g += L[i][l] * L[i][l2] * G[l][l2];
    if (!(g > 0)) return s;
    gam[i] = g;
    ld bt = 0;
    for (int l = 0; l <= i; l++) bt += L[i][l] * b[l];
    beta[i] = bt;
  }
  /* S = sum_i proj_{phi_i} B_L (eq. optimal-approx-for-given-knots) */
  for (int l = 0; l < nb; l++) s.coef[l] = 0;
  for (int i = 0; i < nb; i++) {
    ld al = beta[i] / gam[i];
    for (int l = 0; l <= i; l++) s.coef[l] += al * L[i][l];
  }
  /* error (eq. distance-related-approximation-error), evaluated directly */
  res_acc r;
  r.c = c; r.th = th; r.coef = s.coef; r.sum = 0;
  ld top = th[m - 1] > c->T ? th[m - 1] : c->T;
  /* integrate the residual over [0, top], split at knots and B's own splits */
  ld cuts[ORC_MAXM + 2];
  int nc = 0;
  for (int k = 0; k < m; k++) cuts[nc++] = th[k];
  cuts[nc++] = top;
  qsort(cuts, nc, sizeof(ld), cmp_ld);
  ld lo = 0;
  for (int i = 0; i < nc; i++) {
    if (cuts[i] > lo) {
      /* region beyond T: B = 0, residual is S alone (polynomial) */
      if (lo >= c->T) {
        ld h = (cuts[i] - lo) / 2, mid = (cuts[i] + lo) / 2;
        for (int j = 0; j < GL_N; j++) {
          ld t = mid + h * gl_x[j], v = S_eval(c, th, s.coef, t);
          r.sum += h * gl_w[j] * v * v;
        }
      } else {
        ld hi = cuts[i] < c->T ? cuts[i] : c->T;
        quad_nodes(c, lo, hi, acc_res, &r);
        if (cuts[i] > c->T) {
          ld h = (cuts[i] - c->T) / 2, mid = (cuts[i] + c->T) / 2;
          for (int j = 0; j < GL_N; j++) {
            ld t = mid + h * gl_x[j], v = S_eval(c, th, s.coef, t);
            r.sum += h * gl_w[j] * v * v;
          }
        }
      }
      lo = cuts[i];
    }
  }
  s.err2 = 2 * r.sum;
  s.ok = 1;
  return s;
}

/* Knots from search coordinates: x[0] = th_m / T, x[k>0] = th_{m-k}/th_{m-k+1}. */
static int knots_from_x(const lam_ctx* c, const ld* x, ld* th) {
  int m = c->m;
  if (!(x[0] > 0 && x[0] <= 1.6L)) return 0;
  th[m - 1] = x[0] * c->T;
  for (int k = 1; k < m; k++) {
    if (!(x[k] > 1e-6L && x[k] < 1 - 1e-9L)) return 0;
    th[m - 1 - k] = th[m - k] * x[k];
  }
  return 1;
}

static ld objective(const lam_ctx* c, const ld* x) {
  ld th[ORC_MAXM];
  if (!knots_from_x(c, x, th)) return INFINITY;
  fixed_sol s = solve_fixed(c, th);
  return s.ok ? s.err2 : INFINITY;
}

/* Damped Newton polish of the objective from x (finite-difference gradient
 * and Hessian, backtracking).  Returns the final value; x is updated. */
static ld newton_polish(const lam_ctx* c, ld* x, ld fx) {
  int m = c->m;
  const ld eps = 1e-5L;
  for (int iter = 0; iter < 60; iter++) {
    ld g[ORC_MAXM], H[ORC_MAXM][ORC_MAXM], fp[ORC_MAXM], fm[ORC_MAXM];
    int bad = 0;
    for (int k = 0; k < m && !bad; k++) {
      ld t[ORC_MAXM];
      memcpy(t, x, sizeof(t)); t[k] += eps; fp[k] = objective(c, t);
      memcpy(t, x, sizeof(t)); t[k] -= eps; fm[k] = objective(c, t);
      if (!isfinite((double)fp[k]) || !isfinite((double)fm[k])) bad = 1;
      g[k] = (fp[k] - fm[k]) / (2 * eps);
      H[k][k] = (fp[k] - 2 * fx + fm[k]) / (eps * eps);
    }
    if (bad) break;
    for (int k = 0; k < m; k++)
      for (int l = k + 1; l < m; l++) {
        ld t[ORC_MAXM], v[4];
        for (int s = 0; s < 4; s++) {
          memcpy(t, x, sizeof(t));
          t[k] += (s & 1) ? -eps : eps;
          t[l] += (s & 2) ? -eps : eps;
          v[s] = objective(c, t);
        }
        H[k][l] = H[l][k] = (v[0] - v[1] - v[2] + v[3]) / (4 * eps * eps);
      }
    /* Newton direction if H is positive definite (Cholesky), else -g */
    ld Lc[ORC_MAXM][ORC_MAXM], dir[ORC_MAXM];
    int pd = 1;
    for (int i = 0; i < m && pd; i++)
      for (int j = 0; j <= i; j++) {
        ld s = H[i][j];
        for (int k = 0; k < j; k++) s -= Lc[i][k] * Lc[j][k];
        if (i == j) { if (!(s > 0)) { pd = 0; break; } Lc[i][i] = sqrtl(s); }
        else Lc[i][j] = s / Lc[j][j];
      }
    if (pd) {
      ld y[ORC_MAXM];
      for (int i = 0; i < m; i++) { ld s = -g[i]; for (int k = 0; k < i; k++) s -= Lc[i][k] * y[k]; y[i] = s / Lc[i][i]; }
      for (int i = m - 1; i >= 0; i--) { ld s = y[i]; for (int k = i + 1; k < m; k++) s -= Lc[k][i] * dir[k]; dir[i] = s / Lc[i][i]; }
    } else {
      ld gn = 0;
      for (int k = 0; k < m; k++) gn += g[k] * g[k];
      gn = sqrtl(gn);
      if (!(gn > 0)) break;
      for (int k = 0; k < m; k++) dir[k] = -g[k] / gn * 1e-3L;
    }
    ld lam = 1, best = fx, nx[ORC_MAXM];
    int ok = 0;
    for (int ls = 0; ls < 40; ls++) {
      for (int k = 0; k < m; k++) nx[k] = x[k] + lam * dir[k];
      ld fv = objective(c, nx);
      if (fv < best) { best = fv; ok = 1; break; }
      lam *= 0.5L;
    }
    if (!ok) break;
    ld stepn = 0;
    for (int k = 0; k < m; k++) { stepn += (nx[k] - x[k]) * (nx[k] - x[k]); x[k] = nx[k]; }
    fx = best;
    if (stepn < 1e-26L) break;
  }
  return fx;
}

/* Compass search to a coarse tolerance, then Newton polish. */
static ld local_opt(const lam_ctx* c, ld* cx, ld cv, ld step0) {
  int m = c->m;
  ld step[ORC_MAXM];
  for (int k = 0; k < m; k++) step[k] = step0;
  for (int iter = 0; iter < 4000; iter++) {
    int moved = 0;
    for (int k = 0; k < m; k++)
      for (int sg = -1; sg <= 1; sg += 2) {
        ld tx[ORC_MAXM];
        memcpy(tx, cx, sizeof(tx));
        tx[k] += sg * step[k];
        ld tv = objective(c, tx);
        if (tv < cv) { cv = tv; memcpy(cx, tx, sizeof(tx)); moved = 1; }
      }
    if (!moved) {
      int small = 1;
      for (int k = 0; k < m; k++) { step[k] *= 0.5L; if (step[k] > 1e-6L) small = 0; }
      if (small) break;
    }
  }
  return newton_polish(c, cx, cv);
}

#define NSTART 8
/* Global search over the positive knots (Sec. 3.4): the objective on a
 * coarse grid over the whole feasible box, then a local optimisation from
 * the best NSTART grid-local minima; the best result is kept. */
static ld optimise_knots(const lam_ctx* c, ld* xbest) {
  int m = c->m;
  const int NG = m == 1 ? 96 : (m == 2 ? 28 : (m == 3 ? 10 : 7));
  long total = 1;
  for (int k = 0; k < m; k++) total *= NG;
  ld* vals = (ld*)malloc(total * sizeof(ld));
  ld x[ORC_MAXM];
  for (long it = 0; it < total; it++) {
    long r = it;
    for (int k = 0; k < m; k++) {
      int ik = (int)(r % NG);
      r /= NG;
      x[k] = k ? (ik + 0.5L) / NG : 1.5L * (ik + 0.5L) / NG;
    }
    vals[it] = objective(c, x);
  }
  long starts[NSTART];
  ld sv[NSTART];
  int ns = 0;
  for (long it = 0; it < total; it++) {
    if (!isfinite((double)vals[it])) continue;
    int is_min = 1;
    long stride = 1, r = it;
    for (int k = 0; k < m && is_min; k++) {
      int ik = (int)(r % NG);
      r /= NG;
      if (ik > 0 && vals[it - stride] < vals[it]) is_min = 0;
      if (ik < NG - 1 && vals[it + stride] < vals[it]) is_min = 0;
      stride *= NG;
    }
    if (!is_min) continue;
    int pos = ns;
    while (pos > 0 && sv[pos - 1] > vals[it]) pos--;
    if (pos >= NSTART) continue;
    int last = ns < NSTART ? ns : NSTART - 1;
    for (int s = last; s > pos; s--) { starts[s] = starts[s - 1]; sv[s] = sv[s - 1]; }
    starts[pos] = it; sv[pos] = vals[it];
    if (ns < NSTART) ns++;
  }
  free(vals);
  ld gbest = INFINITY, gx[ORC_MAXM];
  for (int k = 0; k < m; k++) gx[k] = 0;
  for (int s = 0; s < ns; s++) {
    ld cx[ORC_MAXM];
    long r = starts[s];
    for (int k = 0; k < m; k++) {
      int ik = (int)(r % NG);
      r /= NG;
      cx[k] = k ? (ik + 0.5L) / NG : 1.5L * (ik + 0.5L) / NG;
    }
    ld cv = local_opt(c, cx, sv[s], 0.5L / NG);
    if (cv < gbest) { gbest = cv; memcpy(gx, cx, sizeof(gx)); }
  }
  /* The outer knot often has two nearby basins, on either side of the end of
   * supp B_L (theta_m = T), closer together than the grid spacing: start a
   * local search on both sides of that ridge as well. */
  const ld ridge[4] = {0.97L, 0.995L, 1.01L, 1.04L};
  for (int s = 0; s < ns && s < 4; s++) {
    for (int rr = 0; rr < 4; rr++) {
      ld cx[ORC_MAXM];
      long r = starts[s];
      for (int k = 0; k < m; k++) {
        int ik = (int)(r % NG);
        r /= NG;
        cx[k] = k ? (ik + 0.5L) / NG : 1.5L * (ik + 0.5L) / NG;
      }
      cx[0] = ridge[rr];
      ld cv = objective(c, cx);
      if (!isfinite((double)cv)) continue;
      cv = local_opt(c, cx, cv, 0.01L);
      if (cv < gbest) { gbest = cv; memcpy(gx, cx, sizeof(gx)); }
    }
  }
  memcpy(xbest, gx, sizeof(gx));
  return gbest;
}

/* Search coordinates of given knots (inverse of knots_from_x). */
static void x_from_knots(const lam_ctx* c, const ld* th, ld* x) {
  int m = c->m;
  x[0] = th[m - 1] / c->T;
  for (int k = 1; k < m; k++) x[k] = th[m - 1 - k] / th[m - k];
}

/* Local coefficients p[k][d] of the pieces P_k on [th_{k-1}, th_k], expanded
 * at th_{k-1}, from the basis coefficients (definition of A~_kd). */
static void pieces_from_coef(const lam_ctx* c, const ld* th, const ld* coef, ld p[ORC_MAXM][ORC_MAXD + 1]) {
  for (int k = 1; k <= c->m; k++) {
    for (int d = 0; d <= c->D; d++) p[k - 1][d] = 0;
    ld a0 = k > 1 ? th[k - 2] : 0, dk = th[k - 1] - a0;
    for (int i = 0; i < c->nb; i++) {
      if (c->bk[i] >= k) p[k - 1][0] += coef[i];
      if (c->bk[i] == k) p[k - 1][c->bd[i]] -= coef[i] / powl(dk, c->bd[i]);
    }
  }
}

/*
 * Build the look-up table of Sec. 3.1 for L_j = j q / (n_lambda - 1).
 * Outputs (row-major, caller-allocated, FP64):
 *   theta [n_lambda][m]            positive knots th_1 < ... < th_m
 *   pieces[n_lambda][m][D+1]       P_k(s) = sum_d pieces[j][k-1][d] (s - th_{k-1})^d
 *   err   [n_lambda]               E_L = ||S_L - B_L||_2
 *   normB [n_lambda]               ||B_L||_2
 *   integ [n_lambda]               int_R S_L(t) dt
 * The last entry (L = q) and any entry with B_L = 0 is the zero function with
 * all knots at 0.  Returns 0 on success.
 */
int orc_lut_build(int kernel, int K, int D, int n_lambda, double* theta, double* pieces, double* err,
                  double* normB, double* integ) {
  if (K < 1 || K > 2 * ORC_MAXM || D < 1 || D > ORC_MAXD || n_lambda < 2) return 1;
  gl_init();
  int m = (K + 1) / 2;
  double q = orc_kernel_support(kernel);
  ld* TH = (ld*)calloc((size_t)n_lambda * m, sizeof(ld));
  ld* EV = (ld*)malloc((size_t)n_lambda * sizeof(ld));
  /* pass 1: independent global search per entry */
#pragma omp parallel for schedule(dynamic, 2)
  for (int j = 0; j < n_lambda; j++) {
    lam_ctx c;
    lam_ctx_init(&c, kernel, K, D, (ld)j * q / (n_lambda - 1));
    EV[j] = INFINITY;
    if (!(c.T > 0) || j == n_lambda - 1 || c.nb == 0) continue;
    ld x[ORC_MAXM];
    EV[j] = optimise_knots(&c, x);
    knots_from_x(&c, x, TH + (size_t)j * m);
  }
  /* pass 2: continuation -- restart each entry from its neighbours' optima
   * (odd/even halves in parallel), repeated while anything improves */
  for (int sweep = 0; sweep < 6; sweep++) {
    int improved = 0;
    for (int parity = 0; parity < 2; parity++) {
#pragma omp parallel for schedule(dynamic, 2) reduction(| : improved)
      for (int j = parity; j < n_lambda; j += 2) {
        if (!isfinite((double)EV[j])) continue;
        lam_ctx c;
        lam_ctx_init(&c, kernel, K, D, (ld)j * q / (n_lambda - 1));
        for (int nb = -1; nb <= 1; nb += 2) {
          int jn = j + nb;
          if (jn < 0 || jn >= n_lambda || !isfinite((double)EV[jn])) continue;
          ld x[ORC_MAXM];
          x_from_knots(&c, TH + (size_t)jn * m, x);
          ld v = objective(&c, x);
          if (!isfinite((double)v)) continue;
          v = local_opt(&c, x, v, 1e-4L);
          if (v < EV[j] * (1 - 1e-12L)) {
            EV[j] = v;
            knots_from_x(&c, x, TH + (size_t)j * m);
            improved = 1;
          }
        }
      }
    }
    if (!improved) break;
  }
  /* pass 3: final solution per entry */
#pragma omp parallel for schedule(dynamic, 4)
  for (int j = 0; j < n_lambda; j++) {
    lam_ctx c;
    lam_ctx_init(&c, kernel, K, D, (ld)j * q / (n_lambda - 1));
    double* th_o = theta + (size_t)j * m;
    double* p_o = pieces + (size_t)j * m * (D + 1);
    for (int k = 0; k < m; k++) th_o[k] = 0;
    for (int k = 0; k < m * (D + 1); k++) p_o[k] = 0;
    err[j] = 0; normB[j] = 0; integ[j] = 0;
    if (!(c.T > 0) || j == n_lambda - 1) continue;
    bb_acc ba; ba.c = &c; ba.sum = 0;
    quad_nodes(&c, 0, c.T, acc_bb, &ba);
    normB[j] = (double)sqrtl(2 * ba.sum);
    if (c.nb == 0) { err[j] = normB[j]; continue; }
    ld* th = TH + (size_t)j * m;
    fixed_sol s = solve_fixed(&c, th);
    ld p[ORC_MAXM][ORC_MAXD + 1];
    pieces_from_coef(&c, th, s.coef, p);
    for (int k = 0; k < m; k++) th_o[k] = (double)th[k];
    for (int k = 0; k < m; k++)
      for (int d = 0; d <= D; d++) p_o[k * (D + 1) + d] = (double)p[k][d];
    err[j] = (double)sqrtl(s.err2);
    ld I = 0;
    for (int k = 0; k < m; k++) {
      ld a0 = k ? th[k - 1] : 0, dk = th[k] - a0, pw = dk;
      for (int d = 0; d <= D; d++) { I += p[k][d] * pw / (d + 1); pw *= dk; }
    }
    integ[j] = (double)(2 * I);
  }
  free(TH); free(EV);
  return 0;
}

/*
 * Gradient table (part 5): for every entry of a table built above, the optimal
 * approximation of G_L(s) = w'(sqrt(L^2 + s^2)) / sqrt(L^2 + s^2) for the
 * entry's own knots theta (the projection of Sec. 3.3 with G_L in place of
 * B_L).  Outputs gpieces[n_lambda][m][D+1] (local coefficients as pieces),
 * gerr[n_lambda] = ||S_G - G_L||_2 and normG[n_lambda] = ||G_L||_2.  Entries
 * with all knots at 0 get the zero function.  Returns 0 on success.
 */
int orc_lut_build_grad(int kernel, int K, int D, int n_lambda, const double* theta, double* gpieces, double* gerr,
                       double* normG) {
  if (K < 1 || K > 2 * ORC_MAXM || D < 1 || D > ORC_MAXD || n_lambda < 2) return 1;
  gl_init();
  int m = (K + 1) / 2;
  double q = orc_kernel_support(kernel);
#pragma omp parallel for schedule(dynamic, 8)
  for (int j = 0; j < n_lambda; j++) {
    lam_ctx c;
    lam_ctx_init(&c, kernel, K, D, (ld)j * q / (n_lambda - 1));
    c.target = 1;
    double* p_o = gpieces + (size_t)j * m * (D + 1);
    for (int k = 0; k < m * (D + 1); k++) p_o[k] = 0;
    gerr[j] = 0; normG[j] = 0;
    const double* th_i = theta + (size_t)j * m;
    if (!(c.T > 0) || j == n_lambda - 1 || !(th_i[0] > 0)) continue;
    bb_acc ba; ba.c = &c; ba.sum = 0;
    quad_nodes(&c, 0, c.T, acc_bb, &ba);
    normG[j] = (double)sqrtl(2 * ba.sum);
    if (c.nb == 0) { gerr[j] = normG[j]; continue; }
    ld th[ORC_MAXM];
    for (int k = 0; k < m; k++) th[k] = th_i[k];
    fixed_sol sol = solve_fixed(&c, th);
    if (!sol.ok) { gerr[j] = normG[j]; continue; }
    ld pp[ORC_MAXM][ORC_MAXD + 1];
    pieces_from_coef(&c, th, sol.coef, pp);
    for (int k = 0; k < m; k++)
      for (int d = 0; d <= D; d++) p_o[k * (D + 1) + d] = (double)pp[k][d];
    gerr[j] = (double)sqrtl(sol.err2);
  }
  return 0;
}

/* Error of the optimal approximation for GIVEN knots (for tests of Sec. 3.3):
 * writes the pieces and returns ||S - B_L||_2, or -1 on invalid knots. */
double orc_fixed_knots(int kernel, int K, int D, double lam, const double* theta, double* pieces) {
  gl_init();
  lam_ctx c;
  lam_ctx_init(&c, kernel, K, D, lam);
  if (!(c.T > 0)) return -1;
  ld th[ORC_MAXM];
  for (int k = 0; k < c.m; k++) th[k] = theta[k];
  fixed_sol s = solve_fixed(&c, th);
  if (!s.ok) return -1;
  ld p[ORC_MAXM][ORC_MAXD + 1];
  pieces_from_coef(&c, th, s.coef, p);
  for (int k = 0; k < c.m; k++)
    for (int d = 0; d <= D; d++) pieces[k * (D + 1) + d] = (double)p[k][d];
  return (double)sqrtl(s.err2);
}

/* ||B_L||_2^2 by the same quadrature (for tests). */
double orc_ray_norm2(int kernel, double lam) {
  gl_init();
  lam_ctx c;
  lam_ctx_init(&c, kernel, 1, 1, lam);
  bb_acc ba; ba.c = &c; ba.sum = 0;
  quad_nodes(&c, 0, c.T, acc_bb, &ba);
  return (double)(2 * ba.sum);
}

/* int_R B_L(t) dt by the same quadrature (for tests). */
typedef struct { const lam_ctx* c; ld sum; } int_acc;
static void acc_int(void* u, ld t, ld w) { int_acc* a = (int_acc*)u; a->sum += w * B_of(a->c, t); }
double orc_ray_integral(int kernel, double lam) {
  gl_init();
  lam_ctx c;
  lam_ctx_init(&c, kernel, 1, 1, lam);
  int_acc a; a.c = &c; a.sum = 0;
  quad_nodes(&c, 0, c.T, acc_int, &a);
  return (double)(2 * a.sum);
}

/* ------------------------------------------------------------------------ */
/* 3. Per-ray field by direct summation                                      */
/* ------------------------------------------------------------------------ */

typedef struct {
  int projection;          /* 0 perspective, 1 orthographic */
  double eye[3], target[3], up[3];
  double fovy_deg;         /* perspective: full vertical field of view */
  double half_w, half_h;   /* orthographic: half extents of the view rectangle */
  double t_near;
  int width, height;
} orc_camera;

typedef struct {
  int n;                   /* nodes, >= 2 */
  double lo, hi;           /* node i sits at lo + i (hi-lo)/(n-1) */
  const double* rgba;      /* n*4: colour in [0,1], A = extinction per unit length */
  double sigma_scale;      /* sigma(f) = sigma_scale * A(f) */
} orc_tf;

typedef struct {
  int K, D, n_lambda, kernel;
  const double* theta;     /* [n_lambda][m] */
  const double* pieces;    /* [n_lambda][m][D+1] */
} orc_lut;

static void vnorm(double* v) {
  double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  v[0] /= n; v[1] /= n; v[2] /= n;
}
static void vcross(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

/* Viewing ray x(t) = o + t v through the centre of pixel p (row-major, row 0 on top). */
void orc_camera_ray(const orc_camera* cam, int p, double* o, double* v) {
  double f[3] = {cam->target[0] - cam->eye[0], cam->target[1] - cam->eye[1], cam->target[2] - cam->eye[2]};
  vnorm(f);
  double r[3], u[3];
  vcross(f, cam->up, r);
  vnorm(r);
  vcross(r, f, u);
  int px = p % cam->width, py = p / cam->width;
  double sx = 2.0 * (px + 0.5) / cam->width - 1.0, sy = 1.0 - 2.0 * (py + 0.5) / cam->height;
  if (cam->projection == 0) {
    double th = tan(cam->fovy_deg * M_PI / 360.0), asp = (double)cam->width / cam->height;
    sx *= th * asp; sy *= th;
    for (int i = 0; i < 3; i++) { o[i] = cam->eye[i]; v[i] = f[i] + sx * r[i] + sy * u[i]; }
    vnorm(v);
  } else {
    sx *= cam->half_w; sy *= cam->half_h;
    for (int i = 0; i < 3; i++) { o[i] = cam->eye[i] + sx * r[i] + sy * u[i]; v[i] = f[i]; }
  }
}

typedef struct { double t; int cand; int idx; } knot_ev;
static int cmp_knot(const void* a, const void* b) {
  const knot_ev* x = (const knot_ev*)a; const knot_ev* y = (const knot_ev*)b;
  if (x->t < y->t) return -1;
  if (x->t > y->t) return 1;
  if (x->cand != y->cand) return x->cand < y->cand ? -1 : 1;
  return x->idx - y->idx;
}

typedef struct {
  int64_t id;
  double tc, h, c;   /* t_chi, smoothing length, amplitude a / h^3 */
  int j;             /* table entry */
  int passed;        /* knots already passed */
  double dp[3];      /* vector from the ray's closest point to the particle (perpendicular to v) */
} cand_t;

static double binom(int n, int k) {
  double r = 1;
  for (int i = 1; i <= k; i++) r = r * (n - k + i) / i;
  return r;
}

/* Localized coefficients (Sec. 2) at ray parameter ta of one candidate's
 * piece polynomial (pc = piece index between its knots pc and pc+1), of the
 * approximation in table `tab` (the field's pieces, or the gradient's),
 * times the candidate's amplitude c. */
static void cand_piece_coef_tab(const orc_lut* L, const double* tab, const cand_t* cd, int pc, double ta, double* A) {
  int K = L->K, D = L->D, m = (K + 1) / 2;
  const double* th = L->theta + (size_t)cd->j * m;
  const double* P = tab + (size_t)cd->j * m * (D + 1);
  int k, sg;
  if (K % 2 == 0) {
    if (pc < m) { k = m - pc; sg = -1; } else { k = pc - m + 1; sg = 1; }
  } else {
    if (pc < m - 1) { k = m - pc; sg = -1; }
    else if (pc == m - 1) { k = 1; sg = 1; }
    else { k = pc - m + 2; sg = 1; }
  }
  const double* pk = P + (size_t)(k - 1) * (D + 1);
  double th0 = k > 1 ? th[k - 2] : 0.0;
  double z = sg * (ta - cd->tc) / cd->h - th0;   /* local argument of P_k at ta */
  double s = sg / cd->h, se = 1;
  for (int e = 0; e <= D; e++) {
    double acc = 0, zp = 1;
    for (int d = e; d <= D; d++) { acc += binom(d, e) * pk[d] * zp; zp *= z; }
    A[e] = cd->c * se * acc;
    se *= s;
  }
}

static void cand_piece_coef(const orc_lut* L, const cand_t* cd, int pc, double ta, double* A) {
  cand_piece_coef_tab(L, L->pieces, cd, pc, ta, A);
}

/* Sorted knot offsets (normalised s) of one table entry. */
static int entry_knots(const orc_lut* L, int j, double* s) {
  int K = L->K, m = (K + 1) / 2, n = 0;
  const double* th = L->theta + (size_t)j * m;
  for (int k = m - 1; k >= 0; k--) s[n++] = -th[k];
  if (K % 2 == 0) s[n++] = 0;
  for (int k = 0; k < m; k++) s[n++] = th[k];
  return n;
}

/* ------------------------------------------------------------------------ */
/* 4. Classification + compositing, exact                                    */
/* ------------------------------------------------------------------------ */

static double poly_eval(const double* c, int deg, double x) {
  double r = 0;
  for (int i = deg; i >= 0; i--) r = r * x + c[i];
  return r;
}

/* Sorted real roots of poly c (degree deg) in the open interval (a,b):
 * recursive isolation by the derivative's roots, then bisection. */
static int poly_roots(const double* c, int deg, double a, double b, double* out) {
  while (deg > 0 && c[deg] == 0) deg--;
  if (deg <= 0) return 0;
  if (deg == 1) {
    double x = -c[0] / c[1];
    if (x > a && x < b) { out[0] = x; return 1; }
    return 0;
  }
  double dc[ORC_MAXD + 2], crit[ORC_MAXD + 2];
  for (int i = 1; i <= deg; i++) dc[i - 1] = i * c[i];
  int nc = poly_roots(dc, deg - 1, a, b, crit);
  double pts[ORC_MAXD + 4];
  int np = 0;
  pts[np++] = a;
  for (int i = 0; i < nc; i++) pts[np++] = crit[i];
  pts[np++] = b;
  int n = 0;
  for (int i = 0; i + 1 < np; i++) {
    double x0 = pts[i], x1 = pts[i + 1], f0 = poly_eval(c, deg, x0), f1 = poly_eval(c, deg, x1);
    if (i > 0 && f0 == 0) { out[n++] = x0; continue; }
    if ((f0 < 0 && f1 > 0) || (f0 > 0 && f1 < 0)) {
      for (int it = 0; it < 200; it++) {
        double xm = 0.5 * (x0 + x1);
        if (xm <= x0 || xm >= x1) break;
        double fm = poly_eval(c, deg, xm);
        if ((fm < 0) == (f0 < 0) && fm != 0) { x0 = xm; f0 = fm; } else { x1 = xm; }
      }
      out[n++] = 0.5 * (x0 + x1);
    }
  }
  return n;
}

typedef struct {
  const double* F;   /* field polynomial, local variable y */
  int D;
  double G[ORC_MAXD + 2];  /* antiderivative of F, G(0) = 0 */
  double a0, a1;     /* sigma = a0 + a1 F  on this sub-interval */
  double c0[3], c1[3];
  double ya, Gya;
  const double* GP;  /* perpendicular gradient polynomials [3][D+1] (part 5), NULL: no shading */
  double ka, kd, g2; /* g2 = g0^2 */
} emis_ctx;

/* Shading factor ka + kd |F'(y)| / sqrt(|grad|^2 + g0^2) at y, |grad|^2 = F'^2 + |GP(y)|^2
 * (the perpendicular part is orthogonal to v); g0 = 0 gives the cosine |n . v|, and where
 * that gradient vanishes, ka + kd. */
static double shade_at(const emis_ctx* e, double y) {
  double dF = 0, yp = 1;
  for (int i = 1; i <= e->D; i++) { dF += i * e->F[i] * yp; yp *= y; }
  double n2 = dF * dF;
  for (int comp = 0; comp < 3; comp++) {
    double g = poly_eval(e->GP + comp * (e->D + 1), e->D, y);
    n2 += g * g;
  }
  n2 += e->g2;
  return n2 > 0 ? e->ka + e->kd * fabs(dF) / sqrt(n2) : e->ka + e->kd;
}

static void emis_eval(const emis_ctx* e, double y, double* out) {
  double f = poly_eval(e->F, e->D, y);
  double tau = e->a0 * (y - e->ya) + e->a1 * (poly_eval(e->G, e->D + 1, y) - e->Gya);
  double sg = e->a0 + e->a1 * f, w = sg * exp(-tau);
  if (e->GP) w *= shade_at(e, y);
  for (int ch = 0; ch < 3; ch++) out[ch] = (e->c0[ch] + e->c1[ch] * f) * w;
}

static void gk15(const emis_ctx* e, double a, double b, double* res, double* errv) {
  double c = 0.5 * (a + b), h = 0.5 * (b - a), fc[3], rk[3] = {0, 0, 0}, rg[3] = {0, 0, 0};
  emis_eval(e, c, fc);
  for (int ch = 0; ch < 3; ch++) { rk[ch] = gk_wk[7] * fc[ch]; rg[ch] = gk_wg[3] * fc[ch]; }
  for (int i = 0; i < 7; i++) {
    double f1[3], f2[3];
    emis_eval(e, c - h * gk_x[i], f1);
    emis_eval(e, c + h * gk_x[i], f2);
    for (int ch = 0; ch < 3; ch++) {
      rk[ch] += gk_wk[i] * (f1[ch] + f2[ch]);
      if (i % 2 == 1) rg[ch] += gk_wg[i / 2] * (f1[ch] + f2[ch]);
    }
  }
  *errv = 0;
  for (int ch = 0; ch < 3; ch++) {
    res[ch] = rk[ch] * h;
    double d = fabs((rk[ch] - rg[ch]) * h);
    if (d > *errv) *errv = d;
  }
}

static void gk_adapt(const emis_ctx* e, double a, double b, double tol, int depth, double* res) {
  double r[3], er;
  gk15(e, a, b, r, &er);
  if (er <= tol || depth > 40 || b - a < 1e-300) {
    for (int ch = 0; ch < 3; ch++) res[ch] += r[ch];
    return;
  }
  double m = 0.5 * (a + b);
  gk_adapt(e, a, m, tol * 0.5, depth + 1, res);
  gk_adapt(e, m, b, tol * 0.5, depth + 1, res);
}

/* TF linear pieces: value f lies in cell i (clamped ends are cells -1 and n-1). */
static void tf_cell_lin(const orc_tf* tf, double fmid, double* a0, double* a1, double* c0, double* c1) {
  double dv = (tf->hi - tf->lo) / (tf->n - 1);
  const double* R = tf->rgba;
  if (fmid <= tf->lo) {
    *a0 = tf->sigma_scale * R[3]; *a1 = 0;
    for (int ch = 0; ch < 3; ch++) { c0[ch] = R[ch]; c1[ch] = 0; }
    return;
  }
  if (fmid >= tf->hi) {
    const double* q = R + 4 * (tf->n - 1);
    *a0 = tf->sigma_scale * q[3]; *a1 = 0;
    for (int ch = 0; ch < 3; ch++) { c0[ch] = q[ch]; c1[ch] = 0; }
    return;
  }
  int i = (int)floor((fmid - tf->lo) / dv);
  if (i > tf->n - 2) i = tf->n - 2;
  if (i < 0) i = 0;
  double vi = tf->lo + i * dv;
  const double* p0 = R + 4 * i;
  const double* p1 = R + 4 * (i + 1);
  double s1 = tf->sigma_scale * (p1[3] - p0[3]) / dv;
  *a1 = s1; *a0 = tf->sigma_scale * p0[3] - s1 * vi;
  for (int ch = 0; ch < 3; ch++) {
    double k = (p1[ch] - p0[ch]) / dv;
    c1[ch] = k; c0[ch] = p0[ch] - k * vi;
  }
}

static int cmp_d(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return x < y ? -1 : x > y;
}

/* Composite one field piece F(y), y in [ya, yb] (local to the piece start);
 * with GP (perpendicular gradient polynomials, part 5) the emission is shaded. */
static void composite_piece(const orc_tf* tf, const double* F, int D, double ya, double yb, double* rgb, double* Tacc,
                            const double* GP, double ka, double kd, double g0) {
  if (!(yb > ya)) return;
  /* monotone sub-intervals: critical points of F */
  double dF[ORC_MAXD + 1], crit[ORC_MAXD + 2];
  for (int i = 1; i <= D; i++) dF[i - 1] = i * F[i];
  int nc = D >= 1 ? poly_roots(dF, D - 1, ya, yb, crit) : 0;
  double cuts[4096];
  int ncut = 0;
  double pts[ORC_MAXD + 4];
  int np = 0;
  pts[np++] = ya;
  for (int i = 0; i < nc; i++) pts[np++] = crit[i];
  pts[np++] = yb;
  double dv = (tf->hi - tf->lo) / (tf->n - 1);
  for (int s = 0; s + 1 < np; s++) {
    double x0 = pts[s], x1 = pts[s + 1];
    if (s > 0) cuts[ncut++] = x0;
    double f0 = poly_eval(F, D, x0), f1 = poly_eval(F, D, x1);
    double fl = f0 < f1 ? f0 : f1, fh = f0 < f1 ? f1 : f0;
    long ilo = (long)ceil((fl - tf->lo) / dv), ihi = (long)floor((fh - tf->lo) / dv);
    if (ilo < 0) ilo = 0;
    if (ihi > tf->n - 1) ihi = tf->n - 1;
    for (long i = ilo; i <= ihi && ncut < 4000; i++) {
      double v = tf->lo + i * dv;
      if (!(v > fl && v < fh)) continue;
      /* bisection on the monotone interval */
      double a = x0, b = x1, fa = f0 - v;
      for (int it = 0; it < 200; it++) {
        double xm = 0.5 * (a + b);
        if (xm <= a || xm >= b) break;
        double fm = poly_eval(F, D, xm) - v;
        if ((fm < 0) == (fa < 0)) { a = xm; fa = fm; } else b = xm;
      }
      cuts[ncut++] = 0.5 * (a + b);
    }
  }
  qsort(cuts, ncut, sizeof(double), cmp_d);
  emis_ctx e;
  e.F = F; e.D = D;
  e.GP = GP; e.ka = ka; e.kd = kd; e.g2 = g0 * g0;
  e.G[0] = 0;
  for (int i = 0; i <= D; i++) e.G[i + 1] = F[i] / (i + 1);
  double lo = ya;
  for (int s = 0; s <= ncut; s++) {
    double hi = s < ncut ? cuts[s] : yb;
    if (hi > yb) hi = yb;
    if (!(hi > lo)) continue;
    double fm = poly_eval(F, D, 0.5 * (lo + hi));
    tf_cell_lin(tf, fm, &e.a0, &e.a1, e.c0, e.c1);
    e.ya = lo; e.Gya = poly_eval(e.G, D + 1, lo);
    double r[3] = {0, 0, 0};
    gk_adapt(&e, lo, hi, 1e-15, 0, r);
    for (int ch = 0; ch < 3; ch++) rgb[ch] += *Tacc * r[ch];
    double tau = e.a0 * (hi - lo) + e.a1 * (poly_eval(e.G, D + 1, hi) - e.Gya);
    *Tacc *= exp(-tau);
    lo = hi;
  }
}

/*
 * Render the listed pixels.  Inputs: n particles (positions xyz FP32,
 * smoothing lengths FP32, amplitudes a_i = mass * value / density in FP64),
 * the table, camera and transfer function.  Outputs per ray r:
 *   rgba[4r..4r+3]  premultiplied colour and alpha
 *   stats[8r..]     [0] candidates, [1] knots, [2] candidates within 1e-6 h of
 *                   tangency, [3] particles within 1e-6 h of tangency (either
 *                   side), [4] candidates whose L sits within 1e-9 index units of
 *                   a table midpoint, [5] field pieces written, [6] 0, [7] 0
 *   cand_ids        if non-NULL: candidate particle indices, cand_cap per ray
 *   field           if non-NULL: per piece (t_a, t_b, A_0..A_D), field_cap per ray
 * With gpieces (the gradient table of orc_lut_build_grad, part 5) non-NULL the
 * emission is shaded with ka, kd, and gfield (if non-NULL) gets per field row
 * the perpendicular gradient's localized coefficients [3][D+1].
 * Returns 0, or 2 when a buffer capacity was too small (data truncated).
 */
int orc_render(int64_t n, const float* pos, const float* hs, const double* amp, int kernel, int K, int D,
               int n_lambda, const double* theta, const double* pieces, const orc_camera* cam, int tf_n,
               double tf_lo, double tf_hi, const double* tf_rgba, double sigma_scale, int n_rays,
               const int* pix, double* rgba, int64_t* stats, int64_t* cand_ids, int cand_cap, double* field,
               int field_cap, const double* gpieces, double shade_ka, double shade_kd, double shade_g0,
               double* gfield) {
  orc_lut L = {K, D, n_lambda, kernel, theta, pieces};
  orc_tf tf = {tf_n, tf_lo, tf_hi, tf_rgba, sigma_scale};
  double q = orc_kernel_support(kernel);
  int m = (K + 1) / 2;
  int trunc = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : trunc)
  for (int r = 0; r < n_rays; r++) {
    double o[3], v[3];
    orc_camera_ray(cam, pix[r], o, v);
    int64_t* st = stats + 8 * (size_t)r;
    for (int i = 0; i < 8; i++) st[i] = 0;
    size_t ccap = 1024, nc = 0;
    cand_t* cands = (cand_t*)malloc(ccap * sizeof(cand_t));
    for (int64_t i = 0; i < n; i++) {
      double p[3] = {(double)pos[3 * i] - o[0], (double)pos[3 * i + 1] - o[1], (double)pos[3 * i + 2] - o[2]};
      double w[3];
      vcross(p, v, w);
      double d = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
      double h = hs[i], R = q * h;
      if (fabs(d - R) <= 1e-6 * h) st[3]++;
      if (!(d < R)) continue;
      double tc = p[0] * v[0] + p[1] * v[1] + p[2] * v[2];
      if (!(tc + sqrt(R * R - d * d) > cam->t_near)) continue;
      if (nc == ccap) { ccap *= 2; cands = (cand_t*)realloc(cands, ccap * sizeof(cand_t)); }
      double x = d / h * (n_lambda - 1) / q;
      int j = (int)floor(x + 0.5);
      if (j > n_lambda - 1) j = n_lambda - 1;
      if (fabs(x - floor(x) - 0.5) <= 1e-9) st[4]++;
      if (fabs(d - R) <= 1e-6 * h) st[2]++;
      cand_t cd = {i, tc, h, amp[i] / (h * h * h), j, 0, {p[0] - tc * v[0], p[1] - tc * v[1], p[2] - tc * v[2]}};
      cands[nc++] = cd;
    }
    st[0] = (int64_t)nc;
    if (cand_ids) {
      for (size_t i = 0; i < nc && i < (size_t)cand_cap; i++) cand_ids[(size_t)r * cand_cap + i] = cands[i].id;
      if (nc > (size_t)cand_cap) trunc |= 2;
    }
    double* out = rgba + 4 * (size_t)r;
    out[0] = out[1] = out[2] = out[3] = 0;
    if (nc == 0) { free(cands); continue; }
    /* union of knots */
    size_t nk = 0;
    knot_ev* ev = (knot_ev*)malloc(nc * (K + 1) * sizeof(knot_ev));
    double s[2 * ORC_MAXM + 1];
    for (size_t c = 0; c < nc; c++) {
      int ns = entry_knots(&L, cands[c].j, s);
      for (int k = 0; k < ns; k++) { knot_ev e = {cands[c].tc + s[k] * cands[c].h, (int)c, k}; ev[nk++] = e; }
    }
    qsort(ev, nk, sizeof(knot_ev), cmp_knot);
    st[1] = (int64_t)nk;
    double t0 = ev[0].t > cam->t_near ? ev[0].t : cam->t_near, t1 = ev[nk - 1].t;
    /* sweep: active candidates are those with 1 <= passed <= K */
    int* act = (int*)malloc(nc * sizeof(int));
    int* pos_in = (int*)malloc(nc * sizeof(int));
    int na = 0;
    double rgb[3] = {0, 0, 0}, Tacc = 1;
    int64_t nf = 0;
    for (size_t k = 0; k < nk; k++) {
      cand_t* cd = &cands[ev[k].cand];
      cd->passed++;
      if (cd->passed == 1) { pos_in[ev[k].cand] = na; act[na++] = ev[k].cand; }
      if (cd->passed == K + 1) {
        int at = pos_in[ev[k].cand];
        act[at] = act[na - 1]; pos_in[act[at]] = at; na--;
      }
      if (k + 1 == nk) break;
      double ta = ev[k].t, tb = ev[k + 1].t;
      if (!(tb > ta)) continue;
      /* localized coefficients of the field on [ta, tb] by direct summation */
      double A[ORC_MAXD + 1], Ai[ORC_MAXD + 1];
      for (int e = 0; e <= D; e++) A[e] = 0;
      for (int a = 0; a < na; a++) {
        cand_t* c2 = &cands[act[a]];
        cand_piece_coef(&L, c2, c2->passed - 1, ta, Ai);
        for (int e = 0; e <= D; e++) A[e] += Ai[e];
      }
      /* part 5: the perpendicular gradient's localized coefficients, summed
       * the same way: -(c / h^2) d times each candidate's G approximation */
      double GP[3 * (ORC_MAXD + 1)];
      if (gpieces) {
        for (int e = 0; e < 3 * (D + 1); e++) GP[e] = 0;
        for (int a = 0; a < na; a++) {
          cand_t* c2 = &cands[act[a]];
          cand_piece_coef_tab(&L, gpieces, c2, c2->passed - 1, ta, Ai);
          const double sc = -1.0 / (c2->h * c2->h);
          for (int comp = 0; comp < 3; comp++)
            for (int e = 0; e <= D; e++) GP[comp * (D + 1) + e] += sc * c2->dp[comp] * Ai[e];
        }
      }
      if (field) {
        if (nf < field_cap) {
          double* fo = field + ((size_t)r * field_cap + nf) * (D + 3);
          fo[0] = ta; fo[1] = tb;
          for (int e = 0; e <= D; e++) fo[2 + e] = A[e];
          if (gpieces && gfield) {
            double* go = gfield + ((size_t)r * field_cap + nf) * 3 * (D + 1);
            for (int e = 0; e < 3 * (D + 1); e++) go[e] = GP[e];
          }
        } else trunc |= 2;
      }
      nf++;
      /* composite the part of the piece inside [t0, t1] */
      double ya = t0 > ta ? t0 - ta : 0, yb = (tb < t1 ? tb : t1) - ta;
      composite_piece(&tf, A, D, ya, yb, rgb, &Tacc, gpieces ? GP : NULL, shade_ka, shade_kd, shade_g0);
    }
    st[5] = nf;
    out[0] = rgb[0]; out[1] = rgb[1]; out[2] = rgb[2]; out[3] = 1 - Tacc;
    free(act); free(pos_in); free(ev); free(cands);
  }
  (void)m;
  return trunc;
}

/* Composite one polynomial piece alone (for tests of the compositing step). */
void orc_composite_piece(int tf_n, double tf_lo, double tf_hi, const double* tf_rgba, double sigma_scale,
                         const double* F, int D, double ya, double yb, double* rgb_inout, double* T_inout) {
  orc_tf tf = {tf_n, tf_lo, tf_hi, tf_rgba, sigma_scale};
  composite_piece(&tf, F, D, ya, yb, rgb_inout, T_inout, NULL, 1.0, 0.0, 0.0);
}

/* The same with shading (part 5): GP are the three perpendicular gradient polynomials [3][D+1]. */
void orc_composite_piece_shaded(int tf_n, double tf_lo, double tf_hi, const double* tf_rgba, double sigma_scale,
                                const double* F, const double* GP, int D, double ka, double kd, double g0, double ya,
                                double yb,
                                double* rgb_inout, double* T_inout) {
  orc_tf tf = {tf_n, tf_lo, tf_hi, tf_rgba, sigma_scale};
  composite_piece(&tf, F, D, ya, yb, rgb_inout, T_inout, GP, ka, kd, g0);
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
