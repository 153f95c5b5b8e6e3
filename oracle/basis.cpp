// TEST INFRASTRUCTURE ONLY (see dgfv_oracle.h).  Reference-element operators.
#include <algorithm>
#include "basis.hpp"

#include <cmath>
#include <stdexcept>

namespace ora {

namespace {

using ld = long double;

// Legendre polynomial P_n(x) and its derivative by the three-term recurrence
//   k P_k = (2k-1) x P_{k-1} - (k-1) P_{k-2},   P'_k = P'_{k-2} + (2k-1) P_{k-1}.
void legendre(int n, ld x, ld& P, ld& dP) {
    if (n == 0) { P = 1; dP = 0; return; }
    ld p0 = 1, p1 = x, d0 = 0, d1 = 1;
    for (int k = 2; k <= n; ++k) {
        ld p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
        ld d2 = d0 + (2 * k - 1) * p1;
        p0 = p1; p1 = p2; d0 = d1; d1 = d2;
    }
    P = p1; dP = d1;
}

// Roots of P_n (Legendre-Gauss nodes) by Newton's method, ascending, and the
// Gauss weights w = 2 / ((1 - x^2) P_n'(x)^2).
void gauss_legendre(int n, std::vector<ld>& x, std::vector<ld>& w) {
    const ld pi = 3.14159265358979323846264338327950288L;
    x.assign(n, 0); w.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        ld xi = -std::cos(pi * (i + 0.75L) / (n + 0.5L));
        for (int it = 0; it < 200; ++it) {
            ld P, dP;
            legendre(n, xi, P, dP);
            ld dx = P / dP;
            xi -= dx;
            if (std::fabs((double)dx) < 1e-19) break;
        }
        ld P, dP;
        legendre(n, xi, P, dP);
        x[i] = xi;
        w[i] = 2 / ((1 - xi * xi) * dP * dP);
    }
}

// Legendre-Gauss-Lobatto nodes of degree N (N+1 points): -1, the roots of
// P_N' (Newton on P_N' with P_N'' from Legendre's equation
// (1 - x^2) P'' = 2 x P' - N (N+1) P), +1; weights w = 2 / (N (N+1) P_N(x)^2).
void gauss_lobatto(int N, std::vector<ld>& x, std::vector<ld>& w) {
    const ld pi = 3.14159265358979323846264338327950288L;
    const int n = N + 1;
    x.assign(n, 0); w.assign(n, 0);
    x[0] = -1;
    x[N] = 1;
    for (int i = 1; i < N; ++i) {
        ld xi = -std::cos(pi * i / N);
        for (int it = 0; it < 200; ++it) {
            ld P, dP;
            legendre(N, xi, P, dP);
            const ld d2P = (2 * xi * dP - N * (N + 1) * P) / (1 - xi * xi);
            const ld dx = dP / d2P;
            xi -= dx;
            if (std::fabs((double)dx) < 1e-19) break;
        }
        x[i] = xi;
    }
    for (int i = 0; i < n; ++i) {
        ld P, dP;
        legendre(N, x[i], P, dP);
        w[i] = 2 / ((ld)N * (N + 1) * P * P);
    }
}

// Nodes and weights of the node family (0: Legendre-Gauss, 1: Legendre-Gauss-Lobatto).
void node_set(int N, int kind, std::vector<ld>& x, std::vector<ld>& w) {
    if (kind == 1) {
        if (N < 1) throw std::runtime_error("LGL needs N >= 1");
        gauss_lobatto(N, x, w);
    } else {
        gauss_legendre(N + 1, x, w);
    }
}

// Lagrange polynomial l_j of the nodes x, evaluated at xi.
ld lagrange(const std::vector<ld>& x, int j, ld xi) {
    ld r = 1;
    for (int m = 0; m < (int)x.size(); ++m)
        if (m != j) r *= (xi - x[m]) / (x[j] - x[m]);
    return r;
}

// Derivative of the Lagrange polynomial l_j at xi (product rule).
ld lagrange_deriv(const std::vector<ld>& x, int j, ld xi) {
    ld s = 0;
    for (int k = 0; k < (int)x.size(); ++k) {
        if (k == j) continue;
        ld t = 1 / (x[j] - x[k]);
        for (int m = 0; m < (int)x.size(); ++m)
            if (m != j && m != k) t *= (xi - x[m]) / (x[j] - x[m]);
        s += t;
    }
    return s;
}

// Orthonormal Legendre polynomial sqrt((2m+1)/2) P_m.
ld legendre_orthonormal(int m, ld x) {
    ld P, dP;
    legendre(m, x, P, dP);
    return std::sqrt((2 * m + 1) / (ld)2) * P;
}

// Inverse of a square matrix by Gauss-Jordan elimination with partial pivoting.
std::vector<ld> invert(std::vector<ld> A, int n) {
    std::vector<ld> B(n * n, 0);
    for (int i = 0; i < n; ++i) B[i * n + i] = 1;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs((double)A[r * n + c]) > std::fabs((double)A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0) throw std::runtime_error("singular matrix");
        for (int k = 0; k < n; ++k) {
            std::swap(A[c * n + k], A[piv * n + k]);
            std::swap(B[c * n + k], B[piv * n + k]);
        }
        ld d = A[c * n + c];
        for (int k = 0; k < n; ++k) { A[c * n + k] /= d; B[c * n + k] /= d; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            ld f = A[r * n + c];
            if (f == 0) continue;
            for (int k = 0; k < n; ++k) {
                A[r * n + k] -= f * A[c * n + k];
                B[r * n + k] -= f * B[c * n + k];
            }
        }
    }
    return B;
}

std::vector<double> to_double(const std::vector<ld>& a) {
    return std::vector<double>(a.begin(), a.end());
}

std::vector<ld> nodes_ld(int N, int kind) {
    std::vector<ld> x, w;
    node_set(N, kind, x, w);
    return x;
}

// (N_to+1) x (N_from+1) interpolation matrix l^{from}_j(x^{to}_i).
std::vector<ld> interp_ld(int N_from, int N_to, int kind) {
    std::vector<ld> xf = nodes_ld(N_from, kind), xt = nodes_ld(N_to, kind);
    int nf = N_from + 1, nt = N_to + 1;
    std::vector<ld> M(nt * nf);
    for (int i = 0; i < nt; ++i)
        for (int j = 0; j < nf; ++j) M[i * nf + j] = lagrange(xf, j, xt[i]);
    return M;
}

std::vector<ld> leg_vandermonde_ld(int N, int kind) {
    int n = N + 1;
    std::vector<ld> x = nodes_ld(N, kind), V(n * n);
    for (int i = 0; i < n; ++i)
        for (int m = 0; m < n; ++m) V[i * n + m] = legendre_orthonormal(m, x[i]);
    return V;
}

std::vector<ld> dg2fv_ld(int N, int n_fv, int kind) {
    int n = N + 1;
    std::vector<ld> x = nodes_ld(N, kind), q, w;
    gauss_legendre(n, q, w);  // exact for the degree-N integrand
    ld l = (ld)2 / n_fv;
    std::vector<ld> A(n_fv * n);
    for (int s = 0; s < n_fv; ++s) {
        ld a = -1 + s * l;
        for (int j = 0; j < n; ++j) {
            // (1/l) * integral over [a, a+l] of l_j  =  (1/2) sum_q w_q l_j(a + (l/2)(x_q+1))
            ld sum = 0;
            for (int k = 0; k < n; ++k) sum += w[k] * lagrange(x, j, a + l / 2 * (q[k] + 1));
            A[s * n + j] = sum / 2;
        }
    }
    return A;
}

}  // namespace

Basis1D make_basis(int N, int kind) {
    if (N < 0 || N > 15) throw std::runtime_error("degree out of range");
    Basis1D b;
    b.N = N;
    b.n = N + 1;
    const int n = b.n;
    std::vector<ld> x, w;
    node_set(N, kind, x, w);
    b.x = to_double(x);
    b.w = to_double(w);
    std::vector<ld> D(n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) D[i * n + j] = lagrange_deriv(x, j, x[i]);
    b.D = to_double(D);
    b.Dhat.assign(n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) b.Dhat[i * n + j] = (double)(-(w[j] / w[i]) * D[j * n + i]);
    b.lm.resize(n); b.lp.resize(n); b.lhm.resize(n); b.lhp.resize(n);
    for (int j = 0; j < n; ++j) {
        ld a = lagrange(x, j, -1), c = lagrange(x, j, 1);
        b.lm[j] = (double)a;
        b.lp[j] = (double)c;
        b.lhm[j] = (double)(a / w[j]);
        b.lhp[j] = (double)(c / w[j]);
    }
    return b;
}

std::vector<double> vmap(int N_from, int N_to, int kind) {
    if (N_from <= N_to) return to_double(interp_ld(N_from, N_to, kind));
    // L2 projection onto degree N_to: expand in orthonormal Legendre modes
    // (inverse Vandermonde of the finer degree), keep modes 0..N_to, evaluate
    // the truncated series on the coarser nodes.
    int nf = N_from + 1, nt = N_to + 1;
    std::vector<ld> Vinv = invert(leg_vandermonde_ld(N_from, kind), nf);
    std::vector<ld> xt = nodes_ld(N_to, kind);
    std::vector<ld> M(nt * nf, 0);
    for (int i = 0; i < nt; ++i)
        for (int j = 0; j < nf; ++j) {
            ld s = 0;
            for (int m = 0; m <= N_to; ++m) s += legendre_orthonormal(m, xt[i]) * Vinv[m * nf + j];
            M[i * nf + j] = s;
        }
    return to_double(M);
}

std::vector<double> dg2fv(int N, int n_fv, int kind) { return to_double(dg2fv_ld(N, n_fv, kind)); }

std::vector<double> fv2dg_l2(int N, int n_fv, int kind) {
    // L2 projection onto degree N of the piecewise constant given by n_fv sub-cell
    // values on [-1, 1]: M c = b with the exact mass matrix M_ij = int l_i l_j and
    // b_i(s) = int over sub-cell s of l_i, by Gauss rules exact for the integrands.
    const int n = N + 1;
    std::vector<ld> x = nodes_ld(N, kind), q, w;
    gauss_legendre(n + 1, q, w);  // exact to degree 2N+1
    std::vector<ld> M(n * n, 0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            ld sum = 0;
            for (int k = 0; k < n + 1; ++k) sum += w[k] * lagrange(x, i, q[k]) * lagrange(x, j, q[k]);
            M[i * n + j] = sum;
        }
    std::vector<ld> Minv = invert(M, n), Bm(n * n_fv, 0);
    const ld l = (ld)2 / n_fv;
    for (int s = 0; s < n_fv; ++s) {
        const ld a = -1 + s * l;
        for (int i = 0; i < n; ++i) {
            ld sum = 0;
            for (int k = 0; k < n + 1; ++k) sum += w[k] * lagrange(x, i, a + l / 2 * (q[k] + 1));
            Bm[i * n_fv + s] = sum * l / 2;
        }
    }
    std::vector<ld> P(n * n_fv, 0);
    for (int i = 0; i < n; ++i)
        for (int s = 0; s < n_fv; ++s) {
            ld sum = 0;
            for (int k = 0; k < n; ++k) sum += Minv[i * n + k] * Bm[k * n_fv + s];
            P[i * n_fv + s] = sum;
        }
    return to_double(P);
}

std::vector<double> fv2dg(int N, int n_fv, int kind) {
    // Pseudo-inverse through the normal equations, (A^T A)^{-1} A^T; A has full
    // column rank whenever n_fv >= N+1.
    int n = N + 1;
    if (n_fv < n) throw std::runtime_error("n_fv < N+1: DG->FV map not injective");
    std::vector<ld> A = dg2fv_ld(N, n_fv, kind);
    std::vector<ld> AtA(n * n, 0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            ld s = 0;
            for (int r = 0; r < n_fv; ++r) s += A[r * n + i] * A[r * n + j];
            AtA[i * n + j] = s;
        }
    std::vector<ld> inv = invert(AtA, n);
    std::vector<ld> P(n * n_fv, 0);
    for (int i = 0; i < n; ++i)
        for (int r = 0; r < n_fv; ++r) {
            ld s = 0;
            for (int k = 0; k < n; ++k) s += inv[i * n + k] * A[r * n + k];
            P[i * n_fv + r] = s;
        }
    return to_double(P);
}

std::vector<double> leg_vandermonde(int N, int kind) { return to_double(leg_vandermonde_ld(N, kind)); }

// Sec. 3.2.3: half s of a mortar face (s = 0: xi in [-1, 0], s = 1: [0, 1] of the
// big side's reference coordinate); the virtual small side's coordinate eta
// maps to xi = (eta + 2s - 1)/2.
std::vector<double> mortar_interp(int N, int s, int kind) {
    if (s < 0 || s > 1) throw std::runtime_error("mortar half out of range");
    const int n = N + 1;
    std::vector<ld> x = nodes_ld(N, kind);
    std::vector<ld> M(n * n);
    for (int i = 0; i < n; ++i) {
        const ld xi = (x[i] + 2 * s - 1) / 2;
        for (int j = 0; j < n; ++j) M[i * n + j] = lagrange(x, j, xi);
    }
    return to_double(M);
}

std::vector<double> mortar_proj(int N, int s, int kind) {
    // L2 projection onto degree N over [-1, 1] of f = (the small side's interpolant
    // on half s, zero on the other half), through orthonormal Legendre modes:
    //   c_m = int_{half s} f phi_m dxi = 1/2 int_{-1}^{1} f_s(eta) phi_m(xi(eta)) deta
    // (Gauss quadrature with N+1 points, exact for the degree-2N integrand),
    //   P[i][j] = sum_m phi_m(x_i) * 1/2 sum_k w_k l_j(eta_k) phi_m(xi(eta_k)).
    if (s < 0 || s > 1) throw std::runtime_error("mortar half out of range");
    const int n = N + 1;
    std::vector<ld> x = nodes_ld(N, kind), q, w;
    gauss_legendre(n, q, w);
    std::vector<ld> P(n * n, 0);
    for (int j = 0; j < n; ++j)
        for (int m = 0; m < n; ++m) {
            ld c = 0;
            for (int k = 0; k < n; ++k) c += w[k] * lagrange(x, j, q[k]) * legendre_orthonormal(m, (q[k] + 2 * s - 1) / 2);
            c /= 2;
            for (int i = 0; i < n; ++i) P[i * n + j] += legendre_orthonormal(m, x[i]) * c;
        }
    return to_double(P);
}

std::vector<double> mortar_interp_fv(int n_fv, int s) {
    // small sub-cell i of half s spans [(s n + i)/(2n), (s n + i + 1)/(2n)] of the big
    // face (unit length); it lies inside big sub-cell floor((s n + i)/2)
    if (s < 0 || s > 1 || n_fv < 1) throw std::runtime_error("bad FV mortar");
    std::vector<double> M((size_t)n_fv * n_fv, 0.0);
    for (int i = 0; i < n_fv; ++i) M[(size_t)i * n_fv + (s * n_fv + i) / 2] = 1.0;
    return M;
}

std::vector<double> mortar_proj_fv(int n_fv, int s) {
    // mean over big sub-cell j of the piecewise constant given on half s: each small
    // sub-cell inside it covers half of it
    if (s < 0 || s > 1 || n_fv < 1) throw std::runtime_error("bad FV mortar");
    std::vector<double> P((size_t)n_fv * n_fv, 0.0);
    for (int i = 0; i < n_fv; ++i) P[(size_t)((s * n_fv + i) / 2) * n_fv + i] = 0.5;
    return P;
}

std::vector<double> fv_overlap(int n_from, int n_to) {
    // sub-cell i of n_to spans [i/n_to, (i+1)/n_to], cell j of n_from [j/n_from, (j+1)/n_from]
    // (unit length): entry = |overlap| / |cell i|, with integer arithmetic on the
    // common grid of n_from * n_to units (cell i: units [i n_from, (i+1) n_from))
    if (n_from < 1 || n_to < 1) throw std::runtime_error("bad FV overlap");
    std::vector<double> M((size_t)n_to * n_from, 0.0);
    for (int i = 0; i < n_to; ++i)
        for (int j = 0; j < n_from; ++j) {
            const long lo = std::max((long)i * n_from, (long)j * n_to);
            const long hi = std::min((long)(i + 1) * n_from, (long)(j + 1) * n_to);
            if (hi > lo) M[(size_t)i * n_from + j] = (double)(hi - lo) / (double)n_from;
        }
    return M;
}

std::vector<double> leg_vandermonde_inv(int N, int kind) {
    return to_double(invert(leg_vandermonde_ld(N, kind), N + 1));
}

}  // namespace ora
