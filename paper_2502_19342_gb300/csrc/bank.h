// Host computation of the reference-element operators (see bank.cpp).
#pragma once

#include <vector>

namespace dgfv {

struct Bank1D {
    int n = 0;                    // nodes per direction (N+1)
    std::vector<double> x, w;     // nodes (ascending) and weights
    std::vector<double> D;        // D[i*n+j] = l_j'(x_i)
    std::vector<double> Dhat;     // Dhat[i*n+j] = -(w_j/w_i) D[j*n+i]
    std::vector<double> lm, lp;   // l_j(-1), l_j(+1)
    std::vector<double> lhm, lhp; // l_j(-1)/w_j, l_j(+1)/w_j
    std::vector<double> vinv;     // inverse orthonormal-Legendre Vandermonde, [m*n + i]
};

// kind: node family, 0 Legendre-Gauss, 1 Legendre-Gauss-Lobatto
Bank1D make_bank(int n, int kind = 0);
std::vector<double> make_vmap(int n_from, int n_to, int kind = 0);  // n_to x n_from
std::vector<double> make_dg2fv(int n, int nfv, int kind = 0);        // nfv x n
std::vector<double> make_fv2dg(int n, int nfv, int kind = 0);        // n x nfv
// n x nfv: L2 projection onto the n-node polynomials of nfv sub-cell values (the
// V^{FV->DG} of per-element sub-cell counts coarser than the DG side, nfv < n).
std::vector<double> make_fv2dg_l2(int n, int nfv, int kind = 0);
// n_to x n_from: piecewise-constant L2 projection between uniform sub-cell grids.
std::vector<double> make_fv_overlap(int n_from, int n_to);
// Mortar maps of half s (Sec. 3.2.3), n x n: interpolation to the virtual small
// side (proj = false) or L2 projection back (proj = true); FV: on nfv sub-cells.
std::vector<double> make_mortar(int n, int s, bool proj, int kind = 0);
std::vector<double> make_mortar_fv(int nfv, int s, bool proj);

}  // namespace dgfv
