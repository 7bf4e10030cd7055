// Curved-mesh geometry of libirk (host): mapping data per cell and Gauss point, the load vector
// and the initial interpolant of the manufactured solution at the mapped nodes.
#include "deform.h"

#include <cmath>

namespace irk {

namespace {

constexpr double kPi = 3.14159265358979323846;

// J = I + eps 1 grad S^T at reference point xi (d entries); returns det J, fills J^-1 J^-T (upper
// triangle in the order of DeformGeom) and the mapped point.
double metric(int d, const double* xi, double eps, double* G, double* x) {
  double s[3] = {0, 0, 0}, c[3] = {0, 0, 0}, g[3] = {0, 0, 0};
  double S = 1.0;
  for (int a = 0; a < d; ++a) {
    s[a] = std::sin(kPi * xi[a]);
    c[a] = std::cos(kPi * xi[a]);
    S *= s[a];
  }
  for (int b = 0; b < d; ++b) {
    g[b] = kPi * c[b];
    for (int a = 0; a < d; ++a)
      if (a != b) g[b] *= s[a];
  }
  for (int a = 0; a < d; ++a) x[a] = xi[a] + eps * S;
  double J[3][3];
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) J[a][b] = (a == b ? 1.0 : 0.0) + eps * g[b];
  double det, Ji[3][3];
  if (d == 2) {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    Ji[0][0] = J[1][1] / det;
    Ji[0][1] = -J[0][1] / det;
    Ji[1][0] = -J[1][0] / det;
    Ji[1][1] = J[0][0] / det;
  } else {
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    Ji[0][0] = c00 / det;
    Ji[1][0] = c01 / det;
    Ji[2][0] = c02 / det;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  }
  auto m = [&](int a, int b) {
    double t = 0;
    for (int l = 0; l < d; ++l) t += Ji[a][l] * Ji[b][l];
    return t;
  };
  if (d == 2) {
    G[0] = m(0, 0); G[1] = m(1, 1); G[2] = m(0, 1);
  } else {
    G[0] = m(0, 0); G[1] = m(1, 1); G[2] = m(2, 2); G[3] = m(0, 1); G[4] = m(0, 2); G[5] = m(1, 2);
  }
  return det;
}

double S_at(int d, const double* x) {
  double S = 1.0;
  for (int a = 0; a < d; ++a) S *= std::sin(kPi * x[a]);
  return S;
}

}  // namespace

bool deform_valid(int dim, double eps) { return eps >= 0.0 && eps * dim * kPi < 1.0; }

bool build_deform_geometry(int dim, int N, const Element1D& e, double eps, DeformGeom& g, std::string& err) {
  if (dim != 2 && dim != 3) { err = "curved mesh: dim must be 2 or 3"; return false; }
  if (!deform_valid(dim, eps)) { err = "curved mesh: need 0 <= eps < 1 / (dim pi)"; return false; }
  g = DeformGeom();
  g.dim = dim;
  g.N = N;
  g.k = e.k;
  g.p = e.k + 1;
  g.eps = eps;
  g.nq = (dim == 3) ? g.p * g.p * g.p : g.p * g.p;
  g.nf = 1 + dim * (dim + 1) / 2;
  g.ncell = (dim == 3) ? (long long)N * N * N : (long long)N * N;
  g.geo.assign((size_t)g.ncell * g.nf * g.nq, 0.0);
  const double h = 1.0 / N;
  const double hd = (dim == 3) ? h * h * h : h * h, hd2 = (dim == 3) ? h : 1.0;
  const int p = g.p;
  for (long long cell = 0; cell < g.ncell; ++cell) {
    const int cx = (int)(cell % N), cy = (int)((cell / N) % N), cz = (dim == 3) ? (int)(cell / ((long long)N * N)) : 0;
    double* gc = g.geo.data() + (size_t)cell * g.nf * g.nq;
    for (int q = 0; q < g.nq; ++q) {
      const int qx = q % p, qy = (q / p) % p, qz = (dim == 3) ? q / (p * p) : 0;
      const double xi[3] = {(cx + e.gq[qx]) * h, (cy + e.gq[qy]) * h, (cz + e.gq[qz]) * h};
      double G[6], x[3];
      const double det = metric(dim, xi, eps, G, x);
      double w = e.gw[qx] * e.gw[qy];
      if (dim == 3) w *= e.gw[qz];
      gc[q] = w * hd * det;
      for (int f = 0; f + 1 < g.nf; ++f) gc[(size_t)(1 + f) * g.nq + q] = w * hd2 * det * G[f];
    }
  }
  return true;
}

void deform_load_vector(const DeformGeom& g, const Element1D& e, std::vector<double>& G) {
  const int d = g.dim, N = g.N, k = g.k, p = g.p, nq = g.nq;
  const long long n1 = (long long)k * N + 1, n = (d == 3) ? n1 * n1 * n1 : n1 * n1;
  G.assign((size_t)n, 0.0);
  const double h = 1.0 / N;
  std::vector<double> f(nq), t1(nq), t2(nq), loc(nq);
  for (long long cell = 0; cell < g.ncell; ++cell) {
    const int cx = (int)(cell % N), cy = (int)((cell / N) % N), cz = (d == 3) ? (int)(cell / ((long long)N * N)) : 0;
    const double* gc = g.geo.data() + (size_t)cell * g.nf * nq;
    for (int q = 0; q < nq; ++q) {
      const int qx = q % p, qy = (q / p) % p, qz = (d == 3) ? q / (p * p) : 0;
      const double xi[3] = {(cx + e.gq[qx]) * h, (cy + e.gq[qy]) * h, (cz + e.gq[qz]) * h};
      double x[3];
      double S = 1.0;
      for (int a = 0; a < d; ++a) S *= std::sin(kPi * xi[a]);
      for (int a = 0; a < d; ++a) x[a] = xi[a] + g.eps * S;
      f[q] = gc[q] * S_at(d, x);  // w h^d det J times the source profile at the physical point
    }
    // loc[i] = sum_q f[q] prod_a B[q_a][i_a]: one axis at a time
    for (int t = 0; t < nq; ++t) {  // x: (ix, qy, qz)
      const int i = t % p, r = t / p;
      double s = 0;
      for (int qx = 0; qx < p; ++qx) s += e.B[qx * p + i] * f[r * p + qx];
      t1[t] = s;
    }
    for (int t = 0; t < nq; ++t) {  // y: (ix, iy, qz)
      const int ix = t % p, j = (t / p) % p, r = t / (p * p);
      double s = 0;
      for (int qy = 0; qy < p; ++qy) s += e.B[qy * p + j] * t1[(r * p + qy) * p + ix];
      t2[t] = s;
    }
    if (d == 3) {
      for (int t = 0; t < nq; ++t) {  // z
        const int rxy = t % (p * p), l = t / (p * p);
        double s = 0;
        for (int qz = 0; qz < p; ++qz) s += e.B[qz * p + l] * t2[qz * p * p + rxy];
        loc[t] = s;
      }
    } else {
      loc = t2;
    }
    for (int t = 0; t < nq; ++t) {
      const int ix = t % p, iy = (t / p) % p, iz = (d == 3) ? t / (p * p) : 0;
      const long long node = (long long)(k * cx + ix) + n1 * ((long long)(k * cy + iy) + n1 * (k * cz + iz));
      G[(size_t)node] += loc[t];
    }
  }
  for (long long node = 0; node < n; ++node) {
    const long long ix = node % n1, iy = (node / n1) % n1, iz = (d == 3) ? node / (n1 * n1) : 1;
    if (ix == 0 || ix == n1 - 1 || iy == 0 || iy == n1 - 1 || (d == 3 && (iz == 0 || iz == n1 - 1)))
      G[(size_t)node] = 0.0;
  }
}

void deform_initial_value(const DeformGeom& g, const Element1D& e, double t, std::vector<double>& y) {
  const int d = g.dim, N = g.N, k = g.k;
  const long long n1 = (long long)k * N + 1, n = (d == 3) ? n1 * n1 * n1 : n1 * n1;
  std::vector<double> x1(n1);
  for (int c = 0; c < N; ++c)
    for (int r = 0; r <= k; ++r) x1[(size_t)c * k + r] = (c + e.nodes[r]) / N;
  y.assign((size_t)n, 0.0);
  const double ct = std::cos(t);
  for (long long node = 0; node < n; ++node) {
    const long long ix = node % n1, iy = (node / n1) % n1, iz = (d == 3) ? node / (n1 * n1) : 1;
    if (ix == 0 || ix == n1 - 1 || iy == 0 || iy == n1 - 1 || (d == 3 && (iz == 0 || iz == n1 - 1))) continue;
    const double xi[3] = {x1[(size_t)ix], x1[(size_t)iy], (d == 3) ? x1[(size_t)iz] : 0.0};
    double S = 1.0;
    for (int a = 0; a < d; ++a) S *= std::sin(kPi * xi[a]);
    double x[3];
    for (int a = 0; a < d; ++a) x[a] = xi[a] + g.eps * S;
    y[(size_t)node] = S_at(d, x) * ct;
  }
}

}  // namespace irk
