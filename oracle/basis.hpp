// Reference-element operators of the DGSEM and of the DG <-> FV mappings.
//
// TEST INFRASTRUCTURE ONLY (see dgfv_oracle.h).  Everything here is computed
// in long double from the defining formulas and rounded to double at the end.
//
//   Sec. 3.1.1: Legendre-Gauss nodes/weights, Lagrange basis (Eq. 18
//               langrange_basis), derivative matrix D, weighted derivative
//               matrix Dhat and l_hat = l/omega (Eq. 24 dgsem_abbrev).
//   Sec. 3.5:   the same on Legendre-Gauss-Lobatto nodes (split-form DGSEM).
//   Every function takes the node family: kind 0 Legendre-Gauss, 1 LGL.
//   Sec. 3.2:   V^{N->M} (interpolation for N<M, L2 projection for N>M),
//               V^{DG->FV} (sub-cell integration), V^{FV->DG} (pseudo-inverse).
//   Sec. 3.4:   Legendre Vandermonde V_Leg (orthonormal Legendre modes).
//   Sec. 3.2.3: mortar interpolation to the virtual small sides and L2
//               projection back, DG and FV.
#ifndef DGFV_ORACLE_BASIS_HPP
#define DGFV_ORACLE_BASIS_HPP

#include <vector>

namespace ora {

struct Basis1D {
    int N = 0;                 // polynomial degree
    int n = 0;                 // number of nodes, N+1
    std::vector<double> x, w;  // nodes (ascending) and quadrature weights of the node family
    std::vector<double> D;     // D[i*n+j] = l_j'(x_i)
    std::vector<double> Dhat;  // Dhat[i*n+j] = -(w_j / w_i) * D[j*n+i]   (reading of Eq. 24)
    std::vector<double> lm, lp;    // l_j(-1), l_j(+1)
    std::vector<double> lhm, lhp;  // l_j(-1)/w_j, l_j(+1)/w_j
};

Basis1D make_basis(int N, int kind = 0);

// (N_to+1) x (N_from+1): interpolation if N_from <= N_to, L2 projection otherwise.
std::vector<double> vmap(int N_from, int N_to, int kind = 0);
// n_fv x (N+1): mean value of the degree-N interpolant over each of n_fv equal sub-cells.
std::vector<double> dg2fv(int N, int n_fv, int kind = 0);
// (N+1) x n_fv: Moore-Penrose pseudo-inverse of dg2fv(N, n_fv).
std::vector<double> fv2dg(int N, int n_fv, int kind = 0);
// (N+1) x (N+1): V[i*n+m] = sqrt((2m+1)/2) P_m(x_i) on the nodes of degree N.
std::vector<double> leg_vandermonde(int N, int kind = 0);
// Inverse of leg_vandermonde(N) (Gauss-Jordan elimination).
std::vector<double> leg_vandermonde_inv(int N, int kind = 0);

// Sec. 3.2.3 (non-conforming interfaces), one direction of a face halved at
// xi = 0; s = 0 the half [-1, 0], s = 1 the half [0, 1].
// (N+1) x (N+1): the big side's degree-N polynomial evaluated at the nodes of
// the virtual small side (M_01, M_02: exact, a polynomial stays one on a half).
std::vector<double> mortar_interp(int N, int s, int kind = 0);
// (N+1) x (N+1): L2 projection onto degree N of a degree-N polynomial given on
// half s (zero on the other half); M_10 and M_20 add up the two halves.
std::vector<double> mortar_proj(int N, int s, int kind = 0);
// FV sub-cells (n_fv per direction on the big side and on each virtual small
// side): n_fv x n_fv sub-cell means of the virtual small side of the big side's
// piecewise constant, and the big sub-cell means of a piecewise constant given on
// half s.
std::vector<double> mortar_interp_fv(int n_fv, int s);
std::vector<double> mortar_proj_fv(int n_fv, int s);
// n_to x n_from: the piecewise-constant L2 projection between two uniform
// sub-cell grids of one face direction (the per-element sub-cell variant's
// FV/FV faces): entry (i, j) = |cell j of n_from inside cell i of n_to| / |cell i|.
std::vector<double> fv_overlap(int n_from, int n_to);
// (N+1) x n_fv: L2 projection onto degree N of n_fv sub-cell values (a piecewise
// constant); the FV -> DG map of the per-element sub-cell variant where n_fv < N+1
// (the pseudo-inverse of a non-injective V^{DG->FV} would not keep constants).
std::vector<double> fv2dg_l2(int N, int n_fv, int kind = 0);

}  // namespace ora

#endif
