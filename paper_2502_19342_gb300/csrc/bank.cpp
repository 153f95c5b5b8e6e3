// Reference-element operators on the host (FP64 results of long-double work),
// uploaded once per context.  Written independently of any other
// implementation in this repository:
//   Legendre-Gauss nodes      Newton on P_n from Chebyshev-Gauss starting points
//   Lagrange basis / D        barycentric formulas (weights lambda_j = 1/prod(x_j - x_k))
//   Dhat_ij                   -(w_j/w_i) D_ji  (weighted derivative matrix of the weak
//                             form; the weight ratio of Eq. 24 read so that the DGSEM
//                             preserves a free stream and is exact on polynomials)
//   V^{N->M}, N < M           barycentric interpolation at the finer nodes
//   V^{N->M}, N > M           L2 projection by exact Gauss quadrature:
//                             P_ij = w^N_j l^M_i(x^N_j) / w^M_i
//   V^{DG->FV}                sub-cell means by a Gauss rule on every sub-cell
//   V^{FV->DG}                Moore-Penrose inverse through a Householder QR factorisation
//   Legendre Vandermonde^-1   V^-1 = V^T diag(w) (discrete orthonormality, Sec. 3.4)
// Legendre-Gauss-Lobatto nodes (split form, Sec. 3.5):
//   nodes                     Newton on f = x P_N - P_{N-1} (f' = (N+1) P_N; its roots
//                             are +-1 and the zeros of P_N') from Chebyshev-Lobatto points
//   weights                   2 / (N (N+1) P_N(x)^2)
//   V^{N->M}, N > M           L2 projection with the exact mass matrix of the coarse
//                             basis (LGL quadrature under-integrates it), Cholesky solve
//   Legendre Vandermonde^-1   V^T diag(w) with the top mode rescaled by its discrete
//                             norm (the LGL rule is exact for every other mode product)
// Mortars (Sec. 3.2.3), half s of a face halved at xi = 0:
//   interpolation             barycentric, big-side basis at (x_i + 2s - 1)/2
//   projection back           exact L2 projection: mass matrix of the big-side basis
//                             times P = 1/2 int l_i(xi(eta)) l_j(eta) deta (Gauss rule
//                             exact for the products), Cholesky solve
//   FV                        sub-cell j of the big side holds the small sub-cells
//                             2j - s n and 2j + 1 - s n of half s (injection / mean)
#include "bank.h"

#include <cmath>
#include <stdexcept>

namespace dgfv {

namespace {

using ld = long double;

void legendre_pd(int n, ld x, ld& P, ld& dP) {
    ld p0 = 1, p1 = x;
    if (n == 0) { P = 1; dP = 0; return; }
    for (int k = 2; k <= n; ++k) {
        ld p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    P = p1;
    // (1 - x^2) P_n' = n (P_{n-1} - x P_n); at x = +-1, P_n'(+-1) = (+-1)^{n-1} n (n+1)/2
    if (1 - x * x == 0)
        dP = (x > 0 ? 1 : (n % 2 ? 1 : -1)) * (ld)n * (n + 1) / 2;
    else
        dP = n * (p0 - x * p1) / (1 - x * x);
}

ld legendre_orthonormal(int m, ld x) {
    ld p0 = 1, p1 = x;
    if (m == 0) return std::sqrt((ld)0.5);
    for (int k = 2; k <= m; ++k) {
        ld p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    return std::sqrt((2 * m + 1) / (ld)2) * p1;
}

struct Nodes {
    std::vector<ld> x, w, lam;
};

Nodes gauss(int n) {
    Nodes g;
    g.x.resize(n);
    g.w.resize(n);
    const ld pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < n; ++i) {
        ld x = -std::cos(pi * (2 * i + 1) / (2 * n));
        for (int it = 0; it < 100; ++it) {
            ld P, dP;
            legendre_pd(n, x, P, dP);
            const ld dx = P / dP;
            x -= dx;
            if (std::fabs((double)dx) < 1e-20) break;
        }
        ld P, dP;
        legendre_pd(n, x, P, dP);
        g.x[i] = x;
        g.w[i] = 2 / ((1 - x * x) * dP * dP);
    }
    g.lam.resize(n);
    for (int j = 0; j < n; ++j) {
        ld p = 1;
        for (int k = 0; k < n; ++k)
            if (k != j) p *= (g.x[j] - g.x[k]);
        g.lam[j] = 1 / p;
    }
    return g;
}

void barycentric_weights(Nodes& g) {
    const int n = (int)g.x.size();
    g.lam.resize(n);
    for (int j = 0; j < n; ++j) {
        ld p = 1;
        for (int k = 0; k < n; ++k)
            if (k != j) p *= (g.x[j] - g.x[k]);
        g.lam[j] = 1 / p;
    }
}

Nodes lobatto(int n) {
    if (n < 2) throw std::runtime_error("LGL needs at least two nodes");
    const int N = n - 1;
    Nodes g;
    g.x.resize(n);
    g.w.resize(n);
    const ld pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < n; ++i) {
        ld x = -std::cos(pi * i / N);
        for (int it = 0; it < 100; ++it) {
            ld PN, dPN, PM, dPM;
            legendre_pd(N, x, PN, dPN);
            legendre_pd(N - 1, x, PM, dPM);
            const ld f = x * PN - PM, df = (N + 1) * PN;
            const ld dx = f / df;
            x -= dx;
            if (std::fabs((double)dx) < 1e-20) break;
        }
        if (i == 0) x = -1;
        if (i == N) x = 1;
        ld PN, dPN;
        legendre_pd(N, x, PN, dPN);
        g.x[i] = x;
        g.w[i] = 2 / ((ld)N * (N + 1) * PN * PN);
    }
    barycentric_weights(g);
    return g;
}

Nodes node_family(int n, int kind) { return kind == 1 ? lobatto(n) : gauss(n); }

// All Lagrange polynomials of the node set at xi (barycentric formula of the second kind).
std::vector<ld> lagrange_all(const Nodes& g, ld xi) {
    const int n = (int)g.x.size();
    std::vector<ld> l(n, 0);
    for (int j = 0; j < n; ++j)
        if (xi == g.x[j]) { l[j] = 1; return l; }
    ld den = 0;
    for (int j = 0; j < n; ++j) den += g.lam[j] / (xi - g.x[j]);
    for (int j = 0; j < n; ++j) l[j] = g.lam[j] / (xi - g.x[j]) / den;
    return l;
}

std::vector<double> to_d(const std::vector<ld>& a) { return std::vector<double>(a.begin(), a.end()); }

// X = A^{-1} B for a symmetric positive definite A (n x n) and B (n x m):
// Cholesky A = L L^T, then two triangular solves per column.
std::vector<ld> chol_solve(const std::vector<ld>& A, const std::vector<ld>& Bm, int n, int m) {
    std::vector<ld> L(n * n, 0), X(n * m, 0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            ld s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = i == j ? std::sqrt(s) : s / L[j * n + j];
        }
    for (int c = 0; c < m; ++c) {
        std::vector<ld> y(n);
        for (int i = 0; i < n; ++i) {
            ld s = Bm[i * m + c];
            for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
            y[i] = s / L[i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            ld s = y[i];
            for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * X[k * m + c];
            X[i * m + c] = s / L[i * n + i];
        }
    }
    return X;
}

}  // namespace

Bank1D make_bank(int n, int kind) {
    if (n < 1 || n > 16) throw std::runtime_error("bad node count");
    Nodes g = node_family(n, kind);
    Bank1D b;
    b.n = n;
    b.x = to_d(g.x);
    b.w = to_d(g.w);
    std::vector<ld> D(n * n, 0);
    for (int i = 0; i < n; ++i) {
        ld diag = 0;
        for (int j = 0; j < n; ++j) {
            if (i == j) continue;
            D[i * n + j] = (g.lam[j] / g.lam[i]) / (g.x[i] - g.x[j]);
            diag -= D[i * n + j];
        }
        D[i * n + i] = diag;
    }
    b.D = to_d(D);
    b.Dhat.resize(n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) b.Dhat[i * n + j] = (double)(-(g.w[j] / g.w[i]) * D[j * n + i]);
    std::vector<ld> lm = lagrange_all(g, -1), lp = lagrange_all(g, 1);
    b.lm = to_d(lm);
    b.lp = to_d(lp);
    b.lhm.resize(n);
    b.lhp.resize(n);
    for (int j = 0; j < n; ++j) {
        b.lhm[j] = (double)(lm[j] / g.w[j]);
        b.lhp[j] = (double)(lp[j] / g.w[j]);
    }
    b.vinv.resize(n * n);
    for (int m = 0; m < n; ++m) {
        ld gam = 1;  // discrete norm of mode m (1 except the top LGL mode)
        if (kind == 1 && m == n - 1) {
            gam = 0;
            for (int i = 0; i < n; ++i) gam += g.w[i] * legendre_orthonormal(m, g.x[i]) * legendre_orthonormal(m, g.x[i]);
        }
        for (int i = 0; i < n; ++i) b.vinv[m * n + i] = (double)(g.w[i] * legendre_orthonormal(m, g.x[i]) / gam);
    }
    return b;
}

std::vector<double> make_vmap(int n_from, int n_to, int kind) {
    Nodes a = node_family(n_from, kind), b = node_family(n_to, kind);
    std::vector<ld> M(n_to * n_from, 0);
    if (n_from <= n_to) {
        for (int i = 0; i < n_to; ++i) {
            std::vector<ld> l = lagrange_all(a, b.x[i]);
            for (int j = 0; j < n_from; ++j) M[i * n_from + j] = l[j];
        }
    } else if (kind == 1) {
        // exact L2 projection: (integral l^to_i l^to_k) P = integral l^to_i l^from_j,
        // integrals by a Gauss rule exact for the products
        Nodes q = gauss(n_from + n_to);
        std::vector<ld> Mc(n_to * n_to, 0), Bm(n_to * n_from, 0);
        for (size_t k = 0; k < q.x.size(); ++k) {
            std::vector<ld> lt = lagrange_all(b, q.x[k]), lf = lagrange_all(a, q.x[k]);
            for (int i = 0; i < n_to; ++i) {
                for (int j = 0; j < n_to; ++j) Mc[i * n_to + j] += q.w[k] * lt[i] * lt[j];
                for (int j = 0; j < n_from; ++j) Bm[i * n_from + j] += q.w[k] * lt[i] * lf[j];
            }
        }
        M = chol_solve(Mc, Bm, n_to, n_from);
    } else {
        for (int j = 0; j < n_from; ++j) {
            std::vector<ld> l = lagrange_all(b, a.x[j]);  // coarse basis at the fine nodes
            for (int i = 0; i < n_to; ++i) M[i * n_from + j] = a.w[j] * l[i] / b.w[i];
        }
    }
    return to_d(M);
}

namespace {

std::vector<ld> dg2fv_ld(int n, int nfv, int kind) {
    Nodes g = node_family(n, kind);
    Nodes q = gauss(n + 2);  // exact for the degree n-1 integrand
    std::vector<ld> A(nfv * n, 0);
    const ld l = (ld)2 / nfv;
    for (int s = 0; s < nfv; ++s) {
        const ld a = -1 + s * l;
        for (size_t k = 0; k < q.x.size(); ++k) {
            const ld xi = a + (q.x[k] + 1) * l / 2;
            std::vector<ld> lv = lagrange_all(g, xi);
            for (int j = 0; j < n; ++j) A[s * n + j] += q.w[k] * lv[j] / 2;
        }
    }
    return A;
}

}  // namespace

std::vector<double> make_dg2fv(int n, int nfv, int kind) { return to_d(dg2fv_ld(n, nfv, kind)); }

std::vector<double> make_fv2dg_l2(int n, int nfv, int kind) {
    // M c = b: M the exact mass matrix of the node family, b_i = integral of l_i
    // over each sub-cell (Gauss rules of n + 1 points, exact for both integrands)
    Nodes g = node_family(n, kind);
    Nodes q = gauss(n + 1);
    std::vector<ld> Mc(n * n, 0), Bm(n * nfv, 0);
    for (size_t k = 0; k < q.x.size(); ++k) {
        std::vector<ld> lv = lagrange_all(g, q.x[k]);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) Mc[i * n + j] += q.w[k] * lv[i] * lv[j];
    }
    const ld l = (ld)2 / nfv;
    for (int s = 0; s < nfv; ++s)
        for (size_t k = 0; k < q.x.size(); ++k) {
            std::vector<ld> lv = lagrange_all(g, -1 + s * l + (q.x[k] + 1) * l / 2);
            for (int i = 0; i < n; ++i) Bm[i * nfv + s] += q.w[k] * lv[i] * l / 2;
        }
    return to_d(chol_solve(Mc, Bm, n, nfv));
}

std::vector<double> make_fv_overlap(int n_from, int n_to) {
    // sweep over the merged breakpoints k/n_from and k/n_to of [0, 1]: each
    // piece between two breakpoints lies in one cell of either grid
    std::vector<double> M((size_t)n_to * n_from, 0.0);
    int a = 0, b = 0;  // next breakpoint index on the source / target grid
    long x = 0;        // current position in units of 1/(n_from n_to)
    while (a < n_from && b < n_to) {
        const long xa = (long)(a + 1) * n_to, xb = (long)(b + 1) * n_from;
        const long x1 = xa < xb ? xa : xb;
        M[(size_t)b * n_from + a] += (double)(x1 - x) / (double)n_from;  // piece / |target cell|
        x = x1;
        if (x == xa) ++a;
        if (x == xb) ++b;
    }
    return M;
}

std::vector<double> make_fv2dg(int n, int nfv, int kind) {
    if (nfv < n) throw std::runtime_error("N_FV < N+1");
    // Householder QR of A (nfv x n): A = Q R, pinv(A) = R^{-1} Q^T.
    std::vector<ld> A = dg2fv_ld(n, nfv, kind);
    const int m = nfv;
    std::vector<ld> Q(m * m, 0);
    for (int i = 0; i < m; ++i) Q[i * m + i] = 1;  // accumulates Q^T
    std::vector<ld> Rm = A;
    for (int k = 0; k < n; ++k) {
        ld norm = 0;
        for (int i = k; i < m; ++i) norm += Rm[i * n + k] * Rm[i * n + k];
        norm = std::sqrt(norm);
        const ld alpha = Rm[k * n + k] > 0 ? -norm : norm;
        std::vector<ld> v(m, 0);
        for (int i = k; i < m; ++i) v[i] = Rm[i * n + k];
        v[k] -= alpha;
        ld vv = 0;
        for (int i = k; i < m; ++i) vv += v[i] * v[i];
        if (vv == 0) continue;
        for (int j = 0; j < n; ++j) {
            ld s = 0;
            for (int i = k; i < m; ++i) s += v[i] * Rm[i * n + j];
            s = 2 * s / vv;
            for (int i = k; i < m; ++i) Rm[i * n + j] -= s * v[i];
        }
        for (int j = 0; j < m; ++j) {  // Q^T <- H Q^T
            ld s = 0;
            for (int i = k; i < m; ++i) s += v[i] * Q[i * m + j];
            s = 2 * s / vv;
            for (int i = k; i < m; ++i) Q[i * m + j] -= s * v[i];
        }
    }
    // X = R^{-1} (Q^T)[0:n, :]  by back substitution, column by column
    std::vector<ld> X(n * m, 0);
    for (int c = 0; c < m; ++c)
        for (int i = n - 1; i >= 0; --i) {
            ld s = Q[i * m + c];
            for (int j = i + 1; j < n; ++j) s -= Rm[i * n + j] * X[j * m + c];
            X[i * m + c] = s / Rm[i * n + i];
        }
    return to_d(X);
}

}  // namespace dgfv

namespace dgfv {

std::vector<double> make_mortar(int n, int s, bool proj, int kind) {
    if (s < 0 || s > 1) throw std::runtime_error("bad mortar half");
    Nodes g = node_family(n, kind);
    std::vector<ld> M(n * n, 0);
    if (!proj) {
        for (int i = 0; i < n; ++i) {
            std::vector<ld> l = lagrange_all(g, (g.x[i] + 2 * s - 1) / 2);
            for (int j = 0; j < n; ++j) M[i * n + j] = l[j];
        }
        return to_d(M);
    }
    Nodes q = gauss(n + 1);
    std::vector<ld> Mc(n * n, 0), Bm(n * n, 0);
    for (size_t k = 0; k < q.x.size(); ++k) {
        std::vector<ld> lb = lagrange_all(g, q.x[k]);                      // big basis on [-1, 1]
        std::vector<ld> lh = lagrange_all(g, (q.x[k] + 2 * s - 1) / 2);    // big basis on half s
        std::vector<ld> ls = lagrange_all(g, q.x[k]);                      // small basis at eta
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) Mc[i * n + j] += q.w[k] * lb[i] * lb[j];
            for (int j = 0; j < n; ++j) Bm[i * n + j] += q.w[k] * lh[i] * ls[j] / 2;
        }
    }
    return to_d(chol_solve(Mc, Bm, n, n));
}

std::vector<double> make_mortar_fv(int nfv, int s, bool proj) {
    if (s < 0 || s > 1 || nfv < 1) throw std::runtime_error("bad FV mortar");
    std::vector<double> M((size_t)nfv * nfv, 0.0);
    for (int j = 0; j < nfv; ++j)
        for (int t = 0; t < 2; ++t) {
            const int i = 2 * j + t - s * nfv;  // small sub-cell of half s inside big sub-cell j
            if (i < 0 || i >= nfv) continue;
            if (proj)
                M[(size_t)j * nfv + i] = 0.5;
            else
                M[(size_t)i * nfv + j] = 1.0;
        }
    return M;
}

}  // namespace dgfv
