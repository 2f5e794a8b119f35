// Look-up table of optimal per-particle approximations (Sec. 3.1-3.4), built on
// the host in extended precision.
//
// For a normalised distance L the unit particle's ray restriction is
// B_L(s) = w(sqrt(L^2 + s^2)) (Sec. 3.1).  Among even, continuous, compactly
// supported piecewise polynomials with K non-trivial pieces of degree <= D and
// positive knots theta_1 < ... < theta_m (m = ceil(K/2)), the L2-optimal one
// for fixed knots is the orthogonal projection of B_L onto the span of the
// basis A~_kd of Sec. 3.3 (unique, Sec. A.3).  This file solves the projection
// through the normal equations (Cholesky of the Gram matrix), evaluates the
// error ||S - B_L||_2 directly, and searches the knots globally (Sec. 3.4):
// a coarse scan, Nelder-Mead from the best scan minima, then a continuation
// pass that re-starts every entry from its neighbours' optima.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sphdvr_internal.h"

namespace sphdvr {
namespace {

typedef long double ld;
constexpr ld kPi = 3.14159265358979323846264338327950288L;
constexpr int kMaxM = 2;
constexpr int kMaxD = 6;
constexpr int kMaxB = kMaxM * kMaxD;

ld kernel_value(int kernel, ld r) {
  r = std::fabs(r);
  switch (kernel) {
    case 0: {  // cubic B-spline (Sec. 1)
      if (r >= 2) return 0;
      ld a = 2 - r, v = a * a * a;
      if (r < 1) { ld b = 1 - r; v -= 4 * b * b * b; }
      return v / (4 * kPi);
    }
    case 1: {  // Wendland C2
      if (r >= 2) return 0;
      ld a = 1 - r / 2, a2 = a * a;
      return (21.0L / 16.0L) / kPi * a2 * a2 * (1 + 2 * r);
    }
    case 2: {  // Wendland C4
      if (r >= 2) return 0;
      ld a = 1 - r / 2, a3 = a * a * a;
      return (495.0L / 256.0L) / kPi * a3 * a3 * (1 + 3 * r + (35.0L / 12.0L) * r * r);
    }
    default: {  // poly6
      if (r >= 1) return 0;
      ld a = 1 - r * r;
      return (315.0L / 64.0L) / kPi * a * a * a;
    }
  }
}

// w'(r) / r of the kernels of kernel_value, in a form that is finite at r = 0:
// the across-ray part of a particle's gradient on a ray is proportional to
// G_L(s) = w'(rho) / rho, rho = sqrt(L^2 + s^2), even in s like B_L.
ld kernel_slope_over_r(int kernel, ld r) {
  r = std::fabs(r);
  switch (kernel) {
    case 0: {  // (-3 (2-r)^2 + 12 (1-r)^2) / r = 9r - 12 below 1, -3 (2-r)^2 / r above
      if (r >= 2) return 0;
      if (r < 1) return (9 * r - 12) / (4 * kPi);
      ld a = 2 - r;
      return -3 * a * a / (r * 4 * kPi);
    }
    case 1: {
      if (r >= 2) return 0;
      ld a = 1 - r / 2;
      return (21.0L / 16.0L) / kPi * (-5) * a * a * a;
    }
    case 2: {
      if (r >= 2) return 0;
      ld a = 1 - r / 2, a2 = a * a;
      return (495.0L / 256.0L) / kPi * (-7.0L / 3.0L) * (5 * r + 2) * a2 * a2 * a;
    }
    default: {
      if (r >= 1) return 0;
      ld a = 1 - r * r;
      return (315.0L / 64.0L) / kPi * (-6) * a * a;
    }
  }
}

// 16-point Gauss-Legendre rule on [-1, 1].
struct GL16 {
  ld x[16], w[16];
  GL16() {
    const int n = 16;
    for (int i = 0; i < n; ++i) {
      ld z = std::cos(kPi * (i + 0.75L) / (n + 0.5L));
      for (int it = 0; it < 60; ++it) {
        ld pm = 1, p = z;
        for (int k = 2; k <= n; ++k) {
          ld pn = ((2 * k - 1) * z * p - (k - 1) * pm) / k;
          pm = p;
          p = pn;
        }
        ld dp = n * (pm - z * p) / (1 - z * z);
        ld dz = p / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-20L) break;
      }
      ld pm = 1, p = z;
      for (int k = 2; k <= n; ++k) {
        ld pn = ((2 * k - 1) * z * p - (k - 1) * pm) / k;
        pm = p;
        p = pn;
      }
      ld dp = n * (pm - z * p) / (1 - z * z);
      x[i] = z;
      w[i] = 2 / ((1 - z * z) * dp * dp);
    }
  }
};
const GL16& gl16() {
  static GL16 g;
  return g;
}

struct Problem {
  int kernel, K, D, m;
  int target = 0;  // approximated function: 0 B_L, 1 G_L (gradient tables)
  ld q, lam, T;
  ld tbrk;  // s where r crosses an interior kernel break (M4: r = 1), or -1
  int nb;
  int bk[kMaxB], bd[kMaxB];

  Problem(int kern, int K_, int D_, ld lam_) : kernel(kern), K(K_), D(D_), m((K_ + 1) / 2) {
    q = kern == 3 ? 1 : 2;
    lam = lam_;
    T = lam < q ? std::sqrt(q * q - lam * lam) : 0;
    tbrk = (kern == 0 && lam < 1) ? std::sqrt(1 - lam * lam) : -1;
    nb = 0;
    for (int k = 1; k <= m; ++k)
      for (int d = 1; d <= D; ++d) {
        if (k == 1 && (K & 1) && (d & 1)) continue;  // excluded pairs (Sec. 3.3)
        bk[nb] = k;
        bd[nb] = d;
        ++nb;
      }
  }

  ld B(ld s) const {
    const ld rho = std::sqrt(lam * lam + s * s);
    return target ? kernel_slope_over_r(kernel, rho) : kernel_value(kernel, rho);
  }

  // Integrate f(s) over [a, b] within [0, T].  For L > 0 the substitution
  // s = L sinh(u) turns sqrt(L^2 + s^2) = L cosh(u) into an entire function,
  // so Gauss-Legendre converges fast in u; interior kernel breaks are cut.
  template <class F>
  ld integrate(ld a, ld b, F&& f) const {
    if (b > T) b = T;
    if (!(b > a)) return 0;
    const GL16& g = gl16();
    ld cuts[8];
    int nc = 0;
    cuts[nc++] = a;
    if (tbrk > a && tbrk < b) cuts[nc++] = tbrk;
    cuts[nc++] = b;
    ld total = 0;
    const bool subst = lam > 1e-12L;
    for (int c = 0; c + 1 < nc; ++c) {
      ld lo = subst ? std::asinh(cuts[c] / lam) : cuts[c];
      ld hi = subst ? std::asinh(cuts[c + 1] / lam) : cuts[c + 1];
      ld span = hi - lo;
      int pieces = (int)std::ceil(span / (subst ? 1.0L : 0.25L));
      if (pieces < 1) pieces = 1;
      ld step = span / pieces;
      for (int p = 0; p < pieces; ++p) {
        ld u0 = lo + p * step, hh = step / 2, mid = u0 + hh;
        for (int i = 0; i < 16; ++i) {
          ld u = mid + hh * g.x[i];
          if (subst) {
            ld s = lam * std::sinh(u);
            total += hh * g.w[i] * f(s) * lam * std::cosh(u);
          } else {
            total += hh * g.w[i] * f(u);
          }
        }
      }
    }
    return total;
  }

  // Like integrate(), but hands each node and its weight to f(s, w).
  template <class F>
  void integrate_multi(ld a, ld b, F&& f) const {
    if (b > T) b = T;
    if (!(b > a)) return;
    const GL16& g = gl16();
    ld cuts[3];
    int nc = 0;
    cuts[nc++] = a;
    if (tbrk > a && tbrk < b) cuts[nc++] = tbrk;
    cuts[nc++] = b;
    const bool subst = lam > 1e-12L;
    for (int c = 0; c + 1 < nc; ++c) {
      ld lo = subst ? std::asinh(cuts[c] / lam) : cuts[c];
      ld hi = subst ? std::asinh(cuts[c + 1] / lam) : cuts[c + 1];
      ld span = hi - lo;
      int pieces = (int)std::ceil(span / (subst ? 1.0L : 0.25L));
      if (pieces < 1) pieces = 1;
      ld step = span / pieces;
      for (int p = 0; p < pieces; ++p) {
        ld hh = step / 2, mid = lo + p * step + hh;
        for (int i = 0; i < 16; ++i) {
          ld u = mid + hh * g.x[i];
          if (subst) f(lam * std::sinh(u), hh * g.w[i] * lam * std::cosh(u));
          else f(u, hh * g.w[i]);
        }
      }
    }
  }

  // Evaluate S at s >= 0 from basis coefficients (definition of A~_kd).
  ld S(const ld* th, const ld* c, ld s) const {
    s = std::fabs(s);
    ld v = 0;
    for (int i = 0; i < nb; ++i) {
      int k = bk[i];
      ld lo = k > 1 ? th[k - 2] : 0, hi = th[k - 1];
      if (s <= lo) v += c[i];
      else if (s < hi) {
        ld u = (s - lo) / (hi - lo), pw = 1;
        for (int d = 0; d < bd[i]; ++d) pw *= u;
        v += c[i] * (1 - pw);
      }
    }
    return v;
  }

  // Optimal coefficients for fixed knots; returns ||S - B||^2 (inf if invalid).
  ld solve(const ld* th, ld* coef) const {
    for (int k = 0; k < m; ++k)
      if (!(th[k] > (k ? th[k - 1] : 0)) || !(th[k] < 4 * q)) return INFINITY;
    ld mom[kMaxM][kMaxD + 1];
    for (int k = 0; k < m; ++k) {
      ld lo = k ? th[k - 1] : 0, len = th[k] - lo;
      for (int d = 0; d <= D; ++d) mom[k][d] = 0;
      // all moments int u^d B ds, u = (s - lo)/len, in one quadrature pass
      integrate_multi(lo, th[k], [&](ld s, ld w) {
        ld b = B(s) * w, u = (s - lo) / len, pw = 1;
        for (int d = 0; d <= D; ++d) { mom[k][d] += pw * b; pw *= u; }
      });
    }
    ld G[kMaxB][kMaxB], b[kMaxB];
    for (int i = 0; i < nb; ++i) {
      int k = bk[i];
      ld below = 0;
      for (int kk = 0; kk < k; ++kk) below += mom[kk][0];
      b[i] = 2 * (below - mom[k - 1][bd[i]]);
      for (int j = 0; j < nb; ++j) {
        int k2 = bk[j], kl = std::min(k, k2);
        ld lo = kl > 1 ? th[kl - 2] : 0, len = th[kl - 1] - lo;
        // both functions are 1 on [0, lo]; on [lo, lo+len] the lower-k one is 1 - u^d
        ld v;
        if (k == k2) {
          ld d1 = bd[i], d2 = bd[j];
          v = lo + len * (1 - 1 / (d1 + 1) - 1 / (d2 + 1) + 1 / (d1 + d2 + 1));
        } else {
          ld dl = (k < k2) ? bd[i] : bd[j];
          v = lo + len * (dl / (dl + 1));
        }
        G[i][j] = 2 * v;
      }
    }
    // Cholesky G = L L^T, then L L^T c = b
    ld L[kMaxB][kMaxB] = {};
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j <= i; ++j) {
        ld s = G[i][j];
        for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
        if (i == j) {
          if (!(s > 0)) return INFINITY;
          L[i][i] = std::sqrt(s);
        } else {
          L[i][j] = s / L[j][j];
        }
      }
    ld y[kMaxB];
    for (int i = 0; i < nb; ++i) {
      ld s = b[i];
      for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
      y[i] = s / L[i][i];
    }
    for (int i = nb - 1; i >= 0; --i) {
      ld s = y[i];
      for (int k = i + 1; k < nb; ++k) s -= L[k][i] * coef[k];
      coef[i] = s / L[i][i];
    }
    // residual, directly
    ld r2 = 0, lo = 0;
    for (int k = 0; k < m; ++k) {
      r2 += integrate(lo, th[k], [&](ld s) { ld e = B(s) - S(th, coef, s); return e * e; });
      if (th[k] > T) {  // part of the piece beyond supp B: S alone, a polynomial
        ld a = std::max(lo, T), bb = th[k], hh = (bb - a) / 2, mid = (a + bb) / 2;
        const GL16& g = gl16();
        for (int i = 0; i < 16; ++i) {
          ld v = S(th, coef, mid + hh * g.x[i]);
          r2 += hh * g.w[i] * v * v;
        }
      }
      lo = th[k];
    }
    if (T > th[m - 1]) r2 += integrate(th[m - 1], T, [&](ld s) { ld e = B(s); return e * e; });
    return 2 * r2;
  }

  ld objective(const ld* th) const {
    ld c[kMaxB];
    return solve(th, c);
  }

  // Piece coefficients P_k(s) = sum_d p[k][d] (s - theta_{k-1})^d.
  void pieces(const ld* th, const ld* coef, ld* out) const {
    for (int k = 1; k <= m; ++k) {
      ld* p = out + (k - 1) * (D + 1);
      for (int d = 0; d <= D; ++d) p[d] = 0;
      ld lo = k > 1 ? th[k - 2] : 0, len = th[k - 1] - lo;
      for (int i = 0; i < nb; ++i) {
        if (bk[i] >= k) p[0] += coef[i];
        if (bk[i] == k) p[bd[i]] -= coef[i] / std::pow(len, (ld)bd[i]);
      }
    }
  }
};

// Nelder-Mead on the knots, with restarts from the last best point.
ld nelder_mead(const Problem& P, ld* x, ld fx, ld scale) {
  const int n = P.m;
  for (int restart = 0; restart < 4; ++restart) {
    ld simp[kMaxM + 1][kMaxM], fv[kMaxM + 1];
    for (int i = 0; i <= n; ++i) {
      for (int k = 0; k < n; ++k) simp[i][k] = x[k];
      if (i > 0) simp[i][i - 1] += scale * (x[i - 1] > 0 ? 1 : -1);
      fv[i] = i ? P.objective(simp[i]) : fx;
    }
    for (int it = 0; it < 800; ++it) {
      int ord[kMaxM + 1];
      for (int i = 0; i <= n; ++i) ord[i] = i;
      std::sort(ord, ord + n + 1, [&](int a, int b) { return fv[a] < fv[b]; });
      int best = ord[0], worst = ord[n], second = ord[n - 1];
      ld size = 0;
      for (int i = 0; i <= n; ++i)
        for (int k = 0; k < n; ++k) size = std::max(size, std::fabs(simp[i][k] - simp[best][k]));
      if (size < 1e-13L) break;
      ld cen[kMaxM] = {};
      for (int i = 0; i <= n; ++i)
        if (i != worst)
          for (int k = 0; k < n; ++k) cen[k] += simp[i][k] / n;
      ld xr[kMaxM], xe[kMaxM], xc[kMaxM];
      for (int k = 0; k < n; ++k) xr[k] = cen[k] + (cen[k] - simp[worst][k]);
      ld fr = P.objective(xr);
      if (fr < fv[best]) {
        for (int k = 0; k < n; ++k) xe[k] = cen[k] + 2 * (cen[k] - simp[worst][k]);
        ld fe = P.objective(xe);
        if (fe < fr) { std::memcpy(simp[worst], xe, sizeof(xe)); fv[worst] = fe; }
        else { std::memcpy(simp[worst], xr, sizeof(xr)); fv[worst] = fr; }
        continue;
      }
      if (fr < fv[second]) { std::memcpy(simp[worst], xr, sizeof(xr)); fv[worst] = fr; continue; }
      bool outside = fr < fv[worst];
      for (int k = 0; k < n; ++k)
        xc[k] = outside ? cen[k] + 0.5L * (xr[k] - cen[k]) : cen[k] + 0.5L * (simp[worst][k] - cen[k]);
      ld fc = P.objective(xc);
      if (fc < (outside ? fr : fv[worst])) { std::memcpy(simp[worst], xc, sizeof(xc)); fv[worst] = fc; continue; }
      for (int i = 0; i <= n; ++i)
        if (i != best) {
          for (int k = 0; k < n; ++k) simp[i][k] = simp[best][k] + 0.5L * (simp[i][k] - simp[best][k]);
          fv[i] = P.objective(simp[i]);
        }
    }
    int b = 0;
    for (int i = 1; i <= n; ++i)
      if (fv[i] < fv[b]) b = i;
    bool improved = fv[b] < fx * (1 - 1e-14L);
    if (fv[b] < fx) { fx = fv[b]; std::memcpy(x, simp[b], sizeof(ld) * n); }
    if (!improved && restart > 0) break;
    scale *= 0.1L;
  }
  return fx;
}

// Global search for one entry: scan, then Nelder-Mead from the best scan minima.
ld search(const Problem& P, ld* best) {
  const int n = P.m;
  std::vector<std::pair<ld, std::vector<ld>>> starts;
  if (n == 1) {
    const int NG = 160;
    std::vector<ld> v(NG);
    for (int i = 0; i < NG; ++i) { ld th = P.T * 1.5L * (i + 0.5L) / NG; v[i] = P.objective(&th); }
    for (int i = 0; i < NG; ++i) {
      bool mn = (i == 0 || v[i] <= v[i - 1]) && (i == NG - 1 || v[i] <= v[i + 1]);
      if (mn && std::isfinite((double)v[i])) starts.push_back({v[i], {P.T * 1.5L * (i + 0.5L) / NG}});
    }
  } else {
    // scan the box (theta_2 / T, theta_1 / theta_2), which keeps both knots
    // ordered and resolves narrow basins near theta_2 ~ T
    const int NA = 48, NR = 32;
    std::vector<ld> v(NA * NR, INFINITY);
    auto knots = [&](int i, int j, ld* th) {
      th[1] = P.T * 1.5L * (i + 0.5L) / NA;
      th[0] = th[1] * (j + 0.5L) / NR;
    };
    for (int i = 0; i < NA; ++i)
      for (int j = 0; j < NR; ++j) {
        ld th[2];
        knots(i, j, th);
        v[i * NR + j] = P.objective(th);
      }
    for (int i = 0; i < NA; ++i)
      for (int j = 0; j < NR; ++j) {
        ld c = v[i * NR + j];
        if (!std::isfinite((double)c)) continue;
        bool mn = true;
        for (int di = -1; di <= 1 && mn; ++di)
          for (int dj = -1; dj <= 1; ++dj) {
            int a = i + di, b = j + dj;
            if ((di || dj) && a >= 0 && a < NA && b >= 0 && b < NR && v[a * NR + b] < c) { mn = false; break; }
          }
        if (mn) {
          ld th[2];
          knots(i, j, th);
          starts.push_back({c, {th[0], th[1]}});
        }
      }
  }
  std::sort(starts.begin(), starts.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  if (starts.size() > 8) starts.resize(8);
  // the outer knot may have two basins straddling the end of the support
  // (theta_m = T) closer than the scan resolves: seed both sides explicitly
  {
    const size_t nbest = std::min<size_t>(starts.size(), 3);
    for (size_t s = 0; s < nbest; ++s)
      for (ld f : {0.975L, 1.0L, 1.02L, 1.05L}) {
        std::vector<ld> x = starts[s].second;
        ld scale = f * P.T / x[n - 1];
        for (int k = 0; k < n; ++k) x[k] *= scale;
        ld v = P.objective(x.data());
        if (std::isfinite((double)v)) starts.push_back({v, x});
      }
  }
  ld fbest = INFINITY;
  for (auto& s : starts) {
    ld x[kMaxM];
    for (int k = 0; k < n; ++k) x[k] = s.second[k];
    ld f = nelder_mead(P, x, s.first, P.T * 0.02L);
    if (f < fbest) { fbest = f; std::memcpy(best, x, sizeof(ld) * n); }
  }
  return fbest;
}

}  // namespace

// Per-particle relative error of a table of optimal approximations: the error
// along every ray of one direction, integrated over the rays and divided by
// the L2 norm of a normalised particle's contribution (the paper's combined
// accuracy measure, approximation part):
//   E = (1 / kappa) (2 pi int_0^q L err(L)^2 dL)^(1/2),
//   kappa^2 = int w(|x|)^2 dV = 4 pi int_0^q r^2 w(r)^2 dr.
// kappa by 16-point Gauss-Legendre on [0, 1] and [1, q] (exact for these
// piecewise polynomial kernels); the L integral by composite Simpson over the
// table's uniform entries (the last interval by the trapezoid rule when the
// entry count is even).
int lut_error_measure_host(int kernel, int n_lambda, const double* err, double* E) {
  if (kernel < 0 || kernel > 3 || n_lambda < 3 || !err || !E) return 1;
  for (int j = 0; j < n_lambda; ++j)
    if (!(err[j] >= 0) || !std::isfinite(err[j])) return 1;
  const ld q = kernel == 3 ? 1 : 2;
  const GL16& g = gl16();
  ld k2 = 0;
  const ld ends[3] = {0, 1, q};
  for (int seg = 0; seg < 2; ++seg) {
    const ld a = ends[seg], b = ends[seg + 1];
    if (!(b > a)) continue;
    for (int i = 0; i < 16; ++i) {
      const ld r = 0.5L * (a + b) + 0.5L * (b - a) * g.x[i];
      const ld w = kernel_value(kernel, r);
      k2 += 0.5L * (b - a) * g.w[i] * r * r * w * w;
    }
  }
  k2 *= 4 * kPi;
  const ld hstep = q / (n_lambda - 1);
  auto f = [&](int j) { return (ld)j * hstep * (ld)err[j] * (ld)err[j]; };
  const int nodd = (n_lambda % 2 == 1) ? n_lambda : n_lambda - 1;
  ld I = 0;
  for (int j = 0; j + 2 < nodd; j += 2) I += hstep / 3 * (f(j) + 4 * f(j + 1) + f(j + 2));
  if (nodd < n_lambda) I += 0.5L * hstep * (f(n_lambda - 2) + f(n_lambda - 1));
  *E = (double)(std::sqrt(2 * kPi * I) / std::sqrt(k2));
  return 0;
}

// dw/dr of the kernels of kernel_value
static ld kernel_slope(int kernel, ld r) {
  r = std::fabs(r);
  switch (kernel) {
    case 0: {
      if (r >= 2) return 0;
      ld a = 2 - r, v = -3 * a * a;
      if (r < 1) { ld b = 1 - r; v += 12 * b * b; }
      return v / (4 * kPi);
    }
    case 1: {  // d/dr [a^4 (1 + 2r)] = -5 r a^3, a = 1 - r/2
      if (r >= 2) return 0;
      ld a = 1 - r / 2;
      return (21.0L / 16.0L) / kPi * (-5 * r) * a * a * a;
    }
    case 2: {  // d/dr [a^6 (1 + 3r + 35/12 r^2)] = -(7/3) r (5r + 2) a^5
      if (r >= 2) return 0;
      ld a = 1 - r / 2, a2 = a * a;
      return (495.0L / 256.0L) / kPi * (-7.0L / 3.0L) * r * (5 * r + 2) * a2 * a2 * a;
    }
    default: {
      if (r >= 1) return 0;
      ld a = 1 - r * r;
      return (315.0L / 64.0L) / kPi * (-6 * r) * a * a;
    }
  }
}

// kappa (L2 norm of w over R^3) and kappa' (App. A.4) by GL16 on the kernel's
// polynomial pieces (exact up to rounding).  kappa'^2 is the paper's integral
// over s of s * int_R [d/dt w(sqrt(s^2 + t^2))]^2 dt; in polar coordinates of
// the (s, t) half-plane it is (2/3) int_0^q r^2 w'(r)^2 dr.
static void quant_constants(int kernel, ld* kappa, ld* kappa_p) {
  const ld q = kernel == 3 ? 1 : 2;
  const GL16& g = gl16();
  const ld ends[3] = {0, 1, q};
  ld k2 = 0, kp2 = 0;
  for (int seg = 0; seg < 2; ++seg) {
    const ld a = ends[seg], b = ends[seg + 1];
    if (!(b > a)) continue;
    for (int i = 0; i < 16; ++i) {
      const ld r = 0.5L * (a + b) + 0.5L * (b - a) * g.x[i], wt = 0.5L * (b - a) * g.w[i];
      const ld w = kernel_value(kernel, r), dw = kernel_slope(kernel, r);
      k2 += wt * r * r * w * w;
      kp2 += wt * r * r * dw * dw;
    }
  }
  *kappa = std::sqrt(4 * kPi * k2);
  *kappa_p = std::sqrt(2 * kp2 / 3);
}

// squared Q_E(tau, sigma) times (4 kappa)^2 (Sec. 4.4)
static ld quant_radicand(ld kp, ld q, int D, ld tau, ld sigma) {
  ld s = kp * kp * tau * tau;
  for (int d = 0; d <= D; ++d)
    s += 2 * std::pow(q, (ld)(2 * d + 3)) / ((2 * d + 1) * (2 * d + 3)) * sigma * sigma / std::pow(tau, (ld)(2 * d));
  return s;
}

int quant_error_host(int kernel, int D, double tau, double sigma, double* qe) {
  if (kernel < 0 || kernel > 3 || D < 0 || D > 16 || !(tau > 0) || !(sigma >= 0) || !std::isfinite(tau) ||
      !std::isfinite(sigma) || !qe)
    return 1;
  ld kap, kp;
  quant_constants(kernel, &kap, &kp);
  *qe = (double)(std::sqrt(quant_radicand(kp, kernel == 3 ? 1 : 2, D, tau, sigma)) / (4 * kap));
  return 0;
}

double kernel_peak_host(int kernel) { return (double)kernel_value(kernel, 0); }

int quant_params_host(int kernel, int D, int int_bits, double ratio, double* tau, double* sigma, double* qe) {
  if (kernel < 0 || kernel > 3 || D < 0 || D > 16 || int_bits < 8 || int_bits > 1024 || !(ratio > 0) ||
      !std::isfinite(ratio) || !tau || !sigma || !qe)
    return 1;
  ld kap, kp;
  quant_constants(kernel, &kap, &kp);
  const ld q = kernel == 3 ? 1 : 2;
  const ld sg = (ld)ratio * kernel_value(kernel, 0) / std::ldexp(1.0L, int_bits - 1);
  // the radicand is convex in tau; tau times its derivative, as a function of
  // x = log(tau), increases: bisect it for its root
  auto slope = [&](ld x) {
    const ld t = std::exp(x);
    ld v = 2 * kp * kp * t * t;
    for (int d = 1; d <= D; ++d)
      v -= 2 * d * 2 * std::pow(q, (ld)(2 * d + 3)) / ((2 * d + 1) * (2 * d + 3)) * sg * sg / std::pow(t, (ld)(2 * d));
    return v;
  };
  ld lo = -1, hi = 1;
  while (slope(lo) > 0 && lo > -4000) lo -= 4;
  while (slope(hi) < 0 && hi < 4000) hi += 4;
  for (int it = 0; it < 200; ++it) {
    const ld mid = 0.5L * (lo + hi);
    (slope(mid) < 0 ? lo : hi) = mid;
  }
  const ld t = std::exp(0.5L * (lo + hi));
  *tau = (double)t;
  *sigma = (double)sg;
  *qe = (double)(std::sqrt(quant_radicand(kp, q, D, t, sg)) / (4 * kap));
  return 0;
}

int build_lut_host(int kernel, int K, int D, int n_lambda, double* theta, double* pieces, double* err) {
  if (kernel < 0 || kernel > 3 || K < 1 || K > 2 * kMaxM || D < 1 || D > kMaxD || n_lambda < 2 ||
      n_lambda > 65536 || !theta || !pieces)
    return 1;
  const int m = (K + 1) / 2;
  const ld q = kernel == 3 ? 1 : 2;
  std::vector<ld> TH((size_t)n_lambda * m, 0), EV(n_lambda, INFINITY);
  // global search on every `stride`-th entry, continuation from the left
  // neighbour in between, then sweeps from both neighbours (below)
  const int stride = n_lambda >= 512 ? 4 : 1;
  const int last = n_lambda - 2;
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j <= last; ++j) {
    if (j % stride != 0 && j != last) continue;
    Problem P(kernel, K, D, q * j / (n_lambda - 1));
    if (!(P.T > 0) || P.nb == 0) continue;
    EV[j] = search(P, &TH[(size_t)j * m]);
  }
  if (stride > 1) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int g = 0; g <= last / stride; ++g) {
      for (int j = g * stride + 1; j < std::min(last, (g + 1) * stride); ++j) {
        Problem P(kernel, K, D, q * j / (n_lambda - 1));
        if (!(P.T > 0) || P.nb == 0 || !std::isfinite((double)EV[j - 1])) continue;
        ld x[kMaxM];
        for (int k = 0; k < m; ++k) x[k] = TH[(size_t)(j - 1) * m + k];
        ld f = P.objective(x);
        if (!std::isfinite((double)f)) { EV[j] = search(P, &TH[(size_t)j * m]); continue; }
        EV[j] = nelder_mead(P, x, f, P.T * 1e-2L);
        for (int k = 0; k < m; ++k) TH[(size_t)j * m + k] = x[k];
      }
    }
  }
  // continuation: re-start from neighbouring optima while anything improves
  for (int sweep = 0; sweep < 6; ++sweep) {
    int improved = 0;
    for (int par = 0; par < 2; ++par) {
#pragma omp parallel for schedule(dynamic, 2) reduction(| : improved)
      for (int j = par; j < n_lambda - 1; j += 2) {
        if (!std::isfinite((double)EV[j])) continue;
        Problem P(kernel, K, D, q * j / (n_lambda - 1));
        for (int nbh = -1; nbh <= 1; nbh += 2) {
          int jn = j + nbh;
          if (jn < 0 || jn >= n_lambda - 1 || !std::isfinite((double)EV[jn])) continue;
          ld x[kMaxM];
          for (int k = 0; k < m; ++k) x[k] = TH[(size_t)jn * m + k];
          ld f = P.objective(x);
          if (!std::isfinite((double)f)) continue;
          f = nelder_mead(P, x, f, P.T * 1e-3L);
          if (f < EV[j] * (1 - 1e-12L)) {
            EV[j] = f;
            for (int k = 0; k < m; ++k) TH[(size_t)j * m + k] = x[k];
            improved = 1;
          }
        }
      }
    }
    if (!improved) break;
  }
#pragma omp parallel for schedule(dynamic, 4)
  for (int j = 0; j < n_lambda; ++j) {
    double* th_o = theta + (size_t)j * m;
    double* p_o = pieces + (size_t)j * m * (D + 1);
    for (int k = 0; k < m; ++k) th_o[k] = 0;
    for (int k = 0; k < m * (D + 1); ++k) p_o[k] = 0;
    if (err) err[j] = 0;
    if (j == n_lambda - 1) continue;
    Problem P(kernel, K, D, q * j / (n_lambda - 1));
    if (!(P.T > 0)) continue;
    if (P.nb == 0) {
      if (err) err[j] = (double)std::sqrt(2 * P.integrate(0, P.T, [&](ld s) { ld b = P.B(s); return b * b; }));
      continue;
    }
    const ld* th = &TH[(size_t)j * m];
    ld coef[kMaxB], pc[kMaxM * (kMaxD + 1)];
    ld e2 = P.solve(th, coef);
    P.pieces(th, coef, pc);
    for (int k = 0; k < m; ++k) th_o[k] = (double)th[k];
    for (int k = 0; k < m * (D + 1); ++k) p_o[k] = (double)pc[k];
    if (err) err[j] = (double)std::sqrt(e2);
  }
  return 0;
}

// Gradient table: for every entry of a table (its knots theta), the optimal
// approximation of G_L(s) = w'(rho) / rho on the entry's own knots -- the same
// projection onto the basis A~_kd (Sec. 3.3) with G_L in place of B_L, so the
// across-ray gradient of a ray is a piecewise polynomial with the field's
// knots (the Conclusion: features additively generated from particle
// contributions are approximated the same way).  gerr may be NULL.
int build_grad_host(int kernel, int K, int D, int n_lambda, const double* theta, double* gpieces, double* gerr) {
  if (kernel < 0 || kernel > 3 || K < 1 || K > 2 * kMaxM || D < 1 || D > kMaxD || n_lambda < 2 ||
      n_lambda > 65536 || !theta || !gpieces)
    return 1;
  const int m = (K + 1) / 2;
  const ld q = kernel == 3 ? 1 : 2;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(| : bad)
  for (int j = 0; j < n_lambda; ++j) {
    double* p_o = gpieces + (size_t)j * m * (D + 1);
    for (int k = 0; k < m * (D + 1); ++k) p_o[k] = 0;
    if (gerr) gerr[j] = 0;
    Problem P(kernel, K, D, q * j / (n_lambda - 1));
    P.target = 1;
    const double* th_i = theta + (size_t)j * m;
    if (j == n_lambda - 1 || !(P.T > 0) || !(th_i[0] > 0)) continue;  // zero function (knots at 0)
    ld th[kMaxM], coef[kMaxB], pc[kMaxM * (kMaxD + 1)];
    for (int k = 0; k < m; ++k) th[k] = th_i[k];
    if (P.nb == 0) {
      if (gerr) gerr[j] = (double)std::sqrt(2 * P.integrate(0, P.T, [&](ld s) { ld b = P.B(s); return b * b; }));
      continue;
    }
    const ld e2 = P.solve(th, coef);
    if (!std::isfinite((double)e2)) {
      bad = 1;
      continue;
    }
    P.pieces(th, coef, pc);
    for (int k = 0; k < m * (D + 1); ++k) p_o[k] = (double)pc[k];
    if (gerr) gerr[j] = (double)std::sqrt(e2);
  }
  return bad;
}

}  // namespace sphdvr
