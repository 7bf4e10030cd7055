// Curved-mesh geometry of libirk: the uniform mesh of [0,1]^d mapped by
// Phi(xi) = xi + eps S(xi) (1, .., 1), S = prod_a sin(pi xi_a), which fixes the boundary of the
// cube and is non-affine in every cell (one-to-one for eps d pi < 1).  arXiv 2209.06700, Sec. 3.4
// (batching of operations): on deformed cells the matrix-free cell loop loads the mapping data at
// every quadrature point, and one batched loop over all Q stages loads it once instead of Q times.
#pragma once
#include <string>
#include <vector>

#include "host_math.h"

namespace irk {

// Per cell and Gauss point (k+1)^d, unit-cell reference coordinates (d/dxi_hat = h d/dxi):
//   geo[cell][0][q]      = w_q h^d det J_q                                (mass weight)
//   geo[cell][1 + f][q]  = w_q h^(d-2) det J_q (J_q^-1 J_q^-T)_f          (stiffness metric)
// f over the upper triangle: 3D (xx, yy, zz, xy, xz, yz), 2D (xx, yy, xy).  Cells x fastest.
struct DeformGeom {
  int dim = 0, N = 0, k = 0, p = 0, nq = 0, nf = 0;
  double eps = 0;
  long long ncell = 0;
  std::vector<double> geo;   // ncell * nf * nq
};

bool deform_valid(int dim, double eps);
bool build_deform_geometry(int dim, int N, const Element1D& e, double eps, DeformGeom& g, std::string& err);
// G_j = int S(x) phi_j dx over the curved cells (zero on the boundary), x = Phi(xi) at the Gauss points
void deform_load_vector(const DeformGeom& g, const Element1D& e, std::vector<double>& G);
// nodal interpolant of u(x, t) = S(x) cos t at the mapped nodes (zero on the boundary)
void deform_initial_value(const DeformGeom& g, const Element1D& e, double t, std::vector<double>& y);

}  // namespace irk
