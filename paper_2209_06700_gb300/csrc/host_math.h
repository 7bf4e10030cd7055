// Host-side setup math of libirk: Radau IIA tableau and its Q x Q factors,
// one-dimensional Q_k element data.  Long double internally, FP64 results.
#pragma once
#include <complex>
#include <string>
#include <vector>

namespace irk {

using ld = long double;

// Q x Q matrices are stored row-major in std::vector<double>.
struct Tableau {
  int Q = 0;
  std::vector<double> A, b, c;      // Butcher tableau
  std::vector<double> Ainv;         // A^{-1}
  std::vector<double> L, U;         // Crout factors, A^{-1} = L U, diag(U) = 1
  std::vector<double> lam;          // diag(L) = eigenvalues of L
  std::vector<double> S, Sinv;      // eigenvectors of L (unit lower triangular) and inverse
  // Real block-diagonal form A^{-1} = T J T^{-1}: blocks listed in order,
  // real eigenvalue first (odd Q), then pairs [[alpha,-beta],[beta,alpha]], beta > 0.
  std::vector<double> T, Tinv, J;
  struct Block { bool pair; double alpha, beta; int offset; };
  std::vector<Block> blocks;
};

// Builds every field; returns false with a message on failure.
bool build_tableau(int Q, Tableau& t, std::string& err);

// One-dimensional Q_k data on the reference cell [0,1] (GLL nodes, Gauss rule).
struct Element1D {
  int k = 0;
  std::vector<double> nodes;        // k+1 GLL points
  std::vector<double> Me, Ke;       // (k+1)^2 reference element mass / stiffness (row-major)
  std::vector<double> Pc;           // (2k+1) x (k+1): coarse basis i at fine node m of a split cell
  std::vector<double> gq, gw;       // k+1 Gauss-Legendre points and weights on [0, 1]
  std::vector<double> B, D;         // (k+1) x (k+1): basis i and its derivative at Gauss point q, [q][i]
};

bool build_element1d(int k, Element1D& e, std::string& err);

// Small dense helpers (long double Gauss-Jordan with partial pivoting).
bool invert_dense(int n, const std::vector<double>& a, std::vector<double>& inv);

}  // namespace irk
