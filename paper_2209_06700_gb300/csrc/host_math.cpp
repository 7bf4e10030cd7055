// Host-side setup math of libirk (see host_math.h).
//
// Radau IIA (arXiv 2209.06700, Sec. 2: Q stages, order 2Q-1): the nodes are
// the zeros of P_Q(s) - P_{Q-1}(s), s = 2x - 1 (right Radau points, c_Q = 1),
// found by sign-change scanning and bisection on the Legendre recurrence; the
// coefficient matrix solves the collocation conditions
// sum_j a_ij c_j^{m-1} = c_i^m / m (m = 1..Q) and b the quadrature conditions
// sum_j b_j c_j^{m-1} = 1/m, both by long-double Gaussian elimination.
// Eq. (irk:P): A^{-1} = L U (Crout, unit-diagonal U), L = S~ Lambda~ S~^{-1}.
// Eq. (irk:Ainv) in real form (Sec. 6): the eigenvalues of A^{-1} are the
// roots of the denominator of the (Q-1, Q) Pade approximant of e^z
// (Durand-Kerner iteration), eigenvectors by inverse iteration.
#include "host_math.h"

#include <algorithm>
#include <cmath>

namespace irk {

namespace {

using cld = std::complex<ld>;

ld legendre(int n, ld s, ld* dp = nullptr) {
  ld p0 = 1, p1 = s;
  if (n == 0) { if (dp) *dp = 0; return 1; }
  for (int j = 1; j < n; ++j) {
    ld p2 = ((2 * j + 1) * s * p1 - j * p0) / (j + 1);
    p0 = p1; p1 = p2;
  }
  if (dp) *dp = (std::fabs(s * s - 1) > 1e-30L) ? n * (s * p1 - p0) / (s * s - 1) : 0;
  return p1;
}

ld radau_fn(int Q, ld x) {
  ld s = 2 * x - 1;
  return legendre(Q, s) - legendre(Q - 1, s);
}

bool solve_dense_ld(int n, std::vector<ld> a, std::vector<ld>& x) {  // a: n x (n+1) augmented
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(a[r * (n + 1) + col]) > std::fabs(a[piv * (n + 1) + col])) piv = r;
    if (a[piv * (n + 1) + col] == 0) return false;
    if (piv != col)
      for (int c = 0; c <= n; ++c) std::swap(a[col * (n + 1) + c], a[piv * (n + 1) + c]);
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      ld f = a[r * (n + 1) + col] / a[col * (n + 1) + col];
      for (int c = col; c <= n; ++c) a[r * (n + 1) + c] -= f * a[col * (n + 1) + c];
    }
  }
  x.resize(n);
  for (int r = 0; r < n; ++r) x[r] = a[r * (n + 1) + n] / a[r * (n + 1) + r];
  return true;
}

bool invert_ld(int n, const std::vector<ld>& a, std::vector<ld>& inv) {
  std::vector<ld> w(2 * n * n, 0);
  for (int r = 0; r < n; ++r) {
    for (int c = 0; c < n; ++c) w[r * 2 * n + c] = a[r * n + c];
    w[r * 2 * n + n + r] = 1;
  }
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(w[r * 2 * n + col]) > std::fabs(w[piv * 2 * n + col])) piv = r;
    if (w[piv * 2 * n + col] == 0) return false;
    if (piv != col)
      for (int c = 0; c < 2 * n; ++c) std::swap(w[col * 2 * n + c], w[piv * 2 * n + c]);
    ld d = w[col * 2 * n + col];
    for (int c = 0; c < 2 * n; ++c) w[col * 2 * n + c] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      ld f = w[r * 2 * n + col];
      if (f == 0) continue;
      for (int c = 0; c < 2 * n; ++c) w[r * 2 * n + c] -= f * w[col * 2 * n + c];
    }
  }
  inv.assign(n * n, 0);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) inv[r * n + c] = w[r * 2 * n + n + c];
  return true;
}

bool solve_complex(int n, std::vector<cld> a, std::vector<cld>& x) {  // n x (n+1)
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::abs(a[r * (n + 1) + col]) > std::abs(a[piv * (n + 1) + col])) piv = r;
    if (std::abs(a[piv * (n + 1) + col]) == 0) return false;
    if (piv != col)
      for (int c = 0; c <= n; ++c) std::swap(a[col * (n + 1) + c], a[piv * (n + 1) + c]);
    for (int r = col + 1; r < n; ++r) {
      cld f = a[r * (n + 1) + col] / a[col * (n + 1) + col];
      for (int c = col; c <= n; ++c) a[r * (n + 1) + c] -= f * a[col * (n + 1) + c];
    }
  }
  x.assign(n, 0);
  for (int r = n - 1; r >= 0; --r) {
    cld s = a[r * (n + 1) + n];
    for (int c = r + 1; c < n; ++c) s -= a[r * (n + 1) + c] * x[c];
    x[r] = s / a[r * (n + 1) + r];
  }
  return true;
}

ld factorial(int n) { ld f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }

}  // namespace

bool invert_dense(int n, const std::vector<double>& a, std::vector<double>& inv) {
  std::vector<ld> al(a.begin(), a.end()), il;
  if (!invert_ld(n, al, il)) return false;
  inv.assign(il.begin(), il.end());
  return true;
}

bool build_tableau(int Q, Tableau& t, std::string& err) {
  if (Q < 1 || Q > 9) { err = "stage count Q must be in 1..9"; return false; }
  t = Tableau();
  t.Q = Q;
  // --- nodes: sign changes of P_Q - P_{Q-1} on (0, 1], then bisection
  std::vector<ld> c;
  const int grid = 20000;
  ld xprev = 0, fprev = radau_fn(Q, 0);
  for (int i = 1; i <= grid; ++i) {
    ld x = (ld)i / grid, f = radau_fn(Q, x);
    if (i == grid) { c.push_back(1); break; }  // x = 1 is a root for every Q
    if ((f > 0) != (fprev > 0)) {
      ld lo = xprev, hi = x, flo = fprev;
      for (int it = 0; it < 200 && hi - lo > 0; ++it) {
        ld mid = 0.5L * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        ld fm = radau_fn(Q, mid);
        if ((fm > 0) == (flo > 0)) { lo = mid; flo = fm; } else { hi = mid; }
      }
      c.push_back(0.5L * (lo + hi));
    }
    xprev = x; fprev = f;
  }
  if ((int)c.size() != Q) { err = "Radau node search failed"; return false; }
  // --- A and b from the collocation / quadrature conditions
  std::vector<ld> A(Q * Q), b(Q);
  for (int i = 0; i <= Q; ++i) {
    std::vector<ld> aug(Q * (Q + 1)), sol;
    for (int m = 0; m < Q; ++m) {
      for (int j = 0; j < Q; ++j) aug[m * (Q + 1) + j] = std::pow(c[j], (ld)m);
      aug[m * (Q + 1) + Q] = (i < Q) ? std::pow(c[i], (ld)(m + 1)) / (m + 1) : 1.0L / (m + 1);
    }
    if (!solve_dense_ld(Q, aug, sol)) { err = "Vandermonde solve failed"; return false; }
    for (int j = 0; j < Q; ++j) { if (i < Q) A[i * Q + j] = sol[j]; else b[j] = sol[j]; }
  }
  std::vector<ld> Ainv;
  if (!invert_ld(Q, A, Ainv)) { err = "A_Q is singular"; return false; }
  // --- Crout: Ainv = L U, U unit upper triangular
  std::vector<ld> L(Q * Q, 0), U(Q * Q, 0);
  for (int j = 0; j < Q; ++j) {
    U[j * Q + j] = 1;
    for (int i = j; i < Q; ++i) {
      ld s = Ainv[i * Q + j];
      for (int m = 0; m < j; ++m) s -= L[i * Q + m] * U[m * Q + j];
      L[i * Q + j] = s;
    }
    if (L[j * Q + j] == 0) { err = "zero pivot in Crout factorisation"; return false; }
    for (int i = j + 1; i < Q; ++i) {
      ld s = Ainv[j * Q + i];
      for (int m = 0; m < j; ++m) s -= L[j * Q + m] * U[m * Q + i];
      U[j * Q + i] = s / L[j * Q + j];
    }
  }
  // --- eigenvectors of L: column i has zeros above i, one at i (forward substitution)
  std::vector<ld> S(Q * Q, 0), Sinv(Q * Q, 0);
  for (int i = 0; i < Q; ++i) {
    ld lam = L[i * Q + i];
    S[i * Q + i] = 1;
    for (int m = i + 1; m < Q; ++m) {
      ld s = 0;
      for (int l = i; l < m; ++l) s += L[m * Q + l] * S[l * Q + i];
      ld den = lam - L[m * Q + m];
      if (den == 0) { err = "L has a repeated eigenvalue"; return false; }
      S[m * Q + i] = s / den;
    }
  }
  // inverse of a unit lower-triangular matrix
  for (int j = 0; j < Q; ++j) {
    Sinv[j * Q + j] = 1;
    for (int i = j + 1; i < Q; ++i) {
      ld s = 0;
      for (int l = j; l < i; ++l) s += S[i * Q + l] * Sinv[l * Q + j];
      Sinv[i * Q + j] = -s;
    }
  }
  // --- real block form of Ainv: eigenvalues from the Pade (Q-1,Q) denominator
  if (Q >= 1) {
    // det(I - zA) = sum_j d_j z^j, d_j = (2Q-1-j)! Q! / ((2Q-1)! j! (Q-j)!) (-1)^j
    std::vector<ld> d(Q + 1);
    for (int j = 0; j <= Q; ++j)
      d[j] = factorial(2 * Q - 1 - j) * factorial(Q) / (factorial(2 * Q - 1) * factorial(j) * factorial(Q - j)) *
             ((j % 2) ? -1 : 1);
    std::vector<cld> roots(Q);
    for (int i = 0; i < Q; ++i) roots[i] = std::pow(cld(0.4L, 0.9L), i) * (ld)(Q + 1);
    auto poly = [&](cld z) { cld acc = 0; for (int j = Q; j >= 0; --j) acc = acc * z + d[j] / d[Q]; return acc; };
    for (int it = 0; it < 2000; ++it) {
      ld change = 0;
      for (int i = 0; i < Q; ++i) {
        cld den = 1;
        for (int j = 0; j < Q; ++j) if (j != i) den *= roots[i] - roots[j];
        cld delta = poly(roots[i]) / den;
        roots[i] -= delta;
        change = std::max(change, std::abs(delta));
      }
      if (change < 1e-30L) break;
    }
    // order: real first, then pairs with Im > 0 by ascending real part
    std::vector<cld> real_r, pair_r;
    for (auto& z : roots) {
      if (std::fabs(z.imag()) < 1e-12L * std::abs(z)) real_r.push_back(cld(z.real(), 0));
      else if (z.imag() > 0) pair_r.push_back(z);
    }
    std::sort(pair_r.begin(), pair_r.end(), [](const cld& a, const cld& b) { return a.real() < b.real(); });
    if ((int)(real_r.size() + 2 * pair_r.size()) != Q) { err = "eigenvalue split of A^{-1} failed"; return false; }
    std::vector<ld> T(Q * Q, 0), J(Q * Q, 0);
    auto eigvec = [&](cld lam, std::vector<cld>& v) -> bool {
      v.assign(Q, cld(1, 0));
      cld shift = lam * (1 + 1e-14L) + cld(1e-14L, 0);
      for (int it = 0; it < 4; ++it) {
        std::vector<cld> aug(Q * (Q + 1));
        for (int r = 0; r < Q; ++r) {
          for (int cc = 0; cc < Q; ++cc) aug[r * (Q + 1) + cc] = cld(Ainv[r * Q + cc], 0) - (r == cc ? shift : cld(0, 0));
          aug[r * (Q + 1) + Q] = v[r];
        }
        std::vector<cld> x;
        if (!solve_complex(Q, aug, x)) return false;
        ld nrm = 0; for (auto& e : x) nrm = std::max(nrm, std::abs(e));
        for (int r = 0; r < Q; ++r) v[r] = x[r] / nrm;
      }
      // normalise the phase: largest component real positive
      int imax = 0; for (int r = 1; r < Q; ++r) if (std::abs(v[r]) > std::abs(v[imax])) imax = r;
      cld ph = std::abs(v[imax]) / v[imax];
      for (auto& e : v) e *= ph;
      return true;
    };
    int col = 0;
    for (auto& z : real_r) {
      std::vector<cld> v;
      if (!eigvec(z, v)) { err = "eigenvector failed"; return false; }
      for (int r = 0; r < Q; ++r) T[r * Q + col] = v[r].real();
      J[col * Q + col] = z.real();
      t.blocks.push_back({false, (double)z.real(), 0.0, col});
      ++col;
    }
    for (auto& z : pair_r) {
      std::vector<cld> v;
      if (!eigvec(z, v)) { err = "eigenvector failed"; return false; }
      for (int r = 0; r < Q; ++r) { T[r * Q + col] = v[r].real(); T[r * Q + col + 1] = -v[r].imag(); }
      J[col * Q + col] = z.real(); J[col * Q + col + 1] = -z.imag();
      J[(col + 1) * Q + col] = z.imag(); J[(col + 1) * Q + col + 1] = z.real();
      t.blocks.push_back({true, (double)z.real(), (double)z.imag(), col});
      col += 2;
    }
    std::vector<ld> Tinv;
    if (!invert_ld(Q, T, Tinv)) { err = "real Jordan basis is singular"; return false; }
    t.T.assign(T.begin(), T.end());
    t.Tinv.assign(Tinv.begin(), Tinv.end());
    t.J.assign(J.begin(), J.end());
  }
  auto to_d = [](const std::vector<ld>& v) { return std::vector<double>(v.begin(), v.end()); };
  t.A = to_d(A); t.b = to_d(b); t.c = to_d(c); t.Ainv = to_d(Ainv);
  t.L = to_d(L); t.U = to_d(U); t.S = to_d(S); t.Sinv = to_d(Sinv);
  t.lam.resize(Q);
  for (int i = 0; i < Q; ++i) t.lam[i] = (double)L[i * Q + i];
  return true;
}

bool build_element1d(int k, Element1D& e, std::string& err) {
  if (k < 1 || k > 4) { err = "degree k must be in 1..4"; return false; }
  e = Element1D();
  e.k = k;
  const int p = k + 1;
  // GLL nodes: -1, zeros of P_k' (Newton from Chebyshev-Lobatto guesses), +1
  std::vector<ld> xs(p);
  xs[0] = -1; xs[k] = 1;
  for (int i = 1; i < k; ++i) {
    ld x = -std::cos(3.14159265358979323846264338327950288L * i / k);
    for (int it = 0; it < 100; ++it) {
      ld dp;
      ld pk = legendre(k, x, &dp);
      ld d2 = (2 * x * dp - k * (k + 1) * pk) / (1 - x * x);
      ld dx = dp / d2;
      x -= dx;
      if (std::fabs(dx) < 1e-30L) break;
    }
    xs[i] = x;
  }
  std::vector<ld> nodes(p);
  for (int i = 0; i < p; ++i) nodes[i] = 0.5L * (xs[i] + 1);
  // Gauss-Legendre with p points: zeros of P_p, weights 2 / ((1 - s^2) P_p'(s)^2)
  std::vector<ld> gq(p), gw(p);
  for (int i = 0; i < p; ++i) {
    ld s = std::cos(3.14159265358979323846264338327950288L * (i + 0.75L) / (p + 0.5L));
    for (int it = 0; it < 100; ++it) {
      ld dp;
      ld pp = legendre(p, s, &dp);
      ld ds = pp / dp;
      s -= ds;
      if (std::fabs(ds) < 1e-30L) break;
    }
    ld dp;
    legendre(p, s, &dp);
    gq[i] = 0.5L * (s + 1);
    gw[i] = 0.5L * 2 / ((1 - s * s) * dp * dp);
  }
  auto lag = [&](int i, ld x, ld* dl) {
    ld v = 1, d = 0;
    for (int m = 0; m < p; ++m) {
      if (m == i) continue;
      ld term = 1 / (nodes[i] - nodes[m]);
      for (int l = 0; l < p; ++l) {
        if (l == i || l == m) continue;
        term *= (x - nodes[l]) / (nodes[i] - nodes[l]);
      }
      d += term;
      v *= (x - nodes[m]) / (nodes[i] - nodes[m]);
    }
    if (dl) *dl = d;
    return v;
  };
  e.nodes.resize(p);
  for (int i = 0; i < p; ++i) e.nodes[i] = (double)nodes[i];
  e.Me.assign(p * p, 0);
  e.Ke.assign(p * p, 0);
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j) {
      ld sm = 0, sk = 0;
      for (int q = 0; q < p; ++q) {
        ld di, dj;
        ld vi = lag(i, gq[q], &di), vj = lag(j, gq[q], &dj);
        sm += gw[q] * vi * vj;
        sk += gw[q] * di * dj;
      }
      e.Me[i * p + j] = (double)sm;
      e.Ke[i * p + j] = (double)sk;
    }
  e.gq.resize(p);
  e.gw.resize(p);
  e.B.resize(p * p);
  e.D.resize(p * p);
  for (int q = 0; q < p; ++q) {
    e.gq[q] = (double)gq[q];
    e.gw[q] = (double)gw[q];
    for (int i = 0; i < p; ++i) {
      ld di;
      e.B[q * p + i] = (double)lag(i, gq[q], &di);
      e.D[q * p + i] = (double)di;
    }
  }
  // prolongation: fine node m (0..2k) of a coarse cell split in two
  e.Pc.assign((2 * k + 1) * p, 0);
  for (int m = 0; m <= 2 * k; ++m) {
    ld xi = (m == 2 * k) ? 1.0L : ((m / k) + nodes[m % k]) * 0.5L;
    for (int i = 0; i < p; ++i) e.Pc[m * p + i] = (double)lag(i, xi, nullptr);
  }
  return true;
}

}  // namespace irk
