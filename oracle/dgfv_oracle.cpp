// Plain FP64 CPU oracle of the hp-adaptive hybrid DG/FV operator
// (arXiv 2502.19342).  TEST INFRASTRUCTURE ONLY (see dgfv_oracle.h): only the
// tests, the smoke check and the benchmark's CPU-baseline leg use it.
//
// The right-hand side follows the paper's steps in order, with plain loops:
//   1. face values of every element: DG traces u(+-1) = sum_i l_i(+-1) u_i
//      (LG nodes, Sec. 3.1.1); FV elements expose their boundary sub-cell means;
//   2. FV sub-cell elements (Sec. 3.1.2): minmod TVD reconstruction of
//      (rho_k, v, p), central-difference gradients, sub-cell Riemann and
//      viscous fluxes on interior sub-cell faces;
//   3. BR1 lifting interface value U* = (u- + u+)/2 (Eq. 19), on the lower
//      degree at p-interfaces and on DG data at DG/FV interfaces (Sec. 3.2.2);
//   4. lifting (Eq. 23) and volume integral (Eq. 22) of DG elements;
//   5. face flux F* = F^c*(u-,u+) + (F^v(u-,g-) + F^v(u+,g+))/2 (Eqs. 20, 21)
//      on the higher degree at p-interfaces and on FV data at DG/FV
//      interfaces, mapped back to each side (Sec. 3.2.1, 3.2.2);
//   6. surface integral and the 1/J scaling (Eqs. 22, 26).
// Readings of the paper where it is silent or garbled are marked "Reading".
#include "dgfv_oracle.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <stdexcept>
#include <type_traits>
#include <utility>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "basis.hpp"
#include "physics.hpp"

using namespace ora;
using std::vector;

namespace {

// ------------------------------------------------------------------ mesh
struct Elem {
    int dom = 0;
    int idx[3] = {0, 0, 0};
    int N = 1;        // DG degree (kept while the element is FV)
    bool fv = false;  // FV sub-cell element
    int n = 2;        // points per direction: N+1 (DG) or n_fv (FV)
    int64_t off = 0;  // offset of the element's block in the state
    int nb[6];        // neighbour across face f (0:-x 1:+x 2:-y 3:+y 4:-z 5:+z); -1 at a mortar
    int mort[6];      // mortar of face f (index into Problem::mortars) or -1
    int quad[6];      // quadrant of this element on that mortar's small side, -1 on the big side
    double h[3];      // element size
};

// Non-conforming interface (Sec. 3.2.3): one big element face against two
// (types 1, 2: halved along one tangential direction) or four (type 3: halved
// along both) small element faces.  Tangential directions a, b of an x-face:
// y and z.  Quadrant q = qa + 2 qb, qa/qb = 0 the lower half, 1 the upper.
struct Mortar {
    int big = -1;
    int fB = 0;                      // face of the big element (0: -x, 1: +x)
    int split[2] = {0, 0};           // halved along a / along b
    int small[4] = {-1, -1, -1, -1}; // small element of quadrant q
};

struct Ops {  // reference operators, built once per problem before any parallel loop
    std::map<int, Basis1D> basis;
    std::map<std::pair<int, int>, vector<double>> vm;  // (from,to) -> V^{from->to}
    std::map<std::pair<int, int>, vector<double>> d2f, f2d;  // (DG degree, sub-cells per direction)
    std::map<std::pair<int, int>, vector<double>> ov;         // (from, to) sub-cell overlap maps
    std::map<int, vector<double>> vleg_inv;
    // mortar maps per (DG degree, half): interpolation to the virtual small side, projection back
    std::map<std::pair<int, int>, vector<double>> mi, mp;
    vector<double> mi_fv[2], mp_fv[2];  // the same on FV sub-cells
    std::map<int, vector<double>> eye;  // identity of each size (a direction that is not halved)
    const Basis1D& B(int N) const { return basis.at(N); }
};

struct Problem {
    Phys ph;
    int V = 6;
    int nfv = 2;
    bool fv_own = false;  // per-element variant: an FV element of degree N has N+1 sub-cells
    int riemann = 0;
    int nodes = 0;  // 0 Legendre-Gauss, 1 Legendre-Gauss-Lobatto
    int indicator_vars = 0;  // 0: p-adaptation on rho, FV on min(p, Y_k); 1: p-adaptation on p, FV on rho
    int pp = 0;              // positivity limiter after every stage
    double pp_eps = 1e-10;
    int split = 0;  // 1: split-form volume integral with the kinetic-energy-preserving two-point flux
    vector<Elem> el;
    vector<Mortar> mortars;
    int64_t size = 0;
    Ops ops;
};

Problem make_problem(const oracle_problem* p, bool need_ops = true) {
    if (!p || p->n_domains <= 0 || p->n_species < 1 || p->n_species > MAXSP || p->n_fv < 1)
        throw std::runtime_error("bad problem");
    Problem P;
    P.ph.nk = p->n_species;
    for (int k = 0; k < p->n_species; ++k) {
        P.ph.gamma[k] = p->gamma[k];
        P.ph.R[k] = p->Rgas[k];
        P.ph.cv[k] = p->Rgas[k] / (p->gamma[k] - 1.0);
        P.ph.cp[k] = p->gamma[k] * P.ph.cv[k];
        P.ph.mu[k] = p->mu[k];
        P.ph.pr[k] = p->Pr[k];
        P.ph.D[k] = p->Dk[k];
    }
    P.V = P.ph.V();
    P.nfv = p->n_fv;
    P.fv_own = p->fv_own_n != 0;
    if (p->fv_own_n < 0 || p->fv_own_n > 1 || (P.fv_own && p->chain_x))
        throw std::runtime_error("bad per-element sub-cell flag (not with chained domains)");
    P.riemann = p->riemann;
    P.nodes = p->nodes;
    P.split = p->split;
    P.indicator_vars = p->indicator_vars;
    P.pp = p->pp_limiter;
    P.pp_eps = p->pp_eps;
    if (P.pp && !(P.pp_eps > 0.0)) throw std::runtime_error("bad positivity floor");
    P.ph.sutherland = p->sutherland != 0;
    P.ph.T_ref = p->T_ref;
    P.ph.S = p->S_sutherland;
    if (P.ph.sutherland && !(P.ph.T_ref > 0.0 && P.ph.S >= 0.0)) throw std::runtime_error("bad Sutherland law");
    if (P.indicator_vars < 0 || P.indicator_vars > 1) throw std::runtime_error("bad indicator variables");
    if (P.nodes < 0 || P.nodes > 1 || P.split < 0 || P.split > 1 || (P.split && P.nodes != 1))
        throw std::runtime_error("bad node family / split form (split form needs LGL nodes)");
    if (p->chain_x < 0 || p->chain_x > 1) throw std::runtime_error("bad chain flag");
    int64_t e0 = 0;
    vector<int64_t> first(p->n_domains + 1, 0);
    for (int d = 0; d < p->n_domains; ++d) {
        const int nx = p->dims[3 * d], ny = p->dims[3 * d + 1], nz = p->dims[3 * d + 2];
        if (nx < 1 || ny < 1 || nz < 1) throw std::runtime_error("bad domain");
        double h[3];
        for (int a = 0; a < 3; ++a)
            h[a] = (p->hi[3 * d + a] - p->lo[3 * d + a]) / p->dims[3 * d + a];
        const int dims[3] = {nx, ny, nz};
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    Elem E;
                    E.dom = d;
                    E.idx[0] = i; E.idx[1] = j; E.idx[2] = k;
                    for (int a = 0; a < 3; ++a) E.h[a] = h[a];
                    for (int f = 0; f < 6; ++f) {
                        int q[3] = {i, j, k};
                        int a = f / 2;
                        q[a] = (q[a] + (f % 2 ? 1 : -1) + dims[a]) % dims[a];
                        E.nb[f] = (int)(e0 + q[0] + nx * (q[1] + ny * q[2]));
                        E.mort[f] = -1;
                        E.quad[f] = -1;
                    }
                    P.el.push_back(E);
                }
        e0 += (int64_t)nx * ny * nz;
        first[d + 1] = e0;
    }
    if (p->chain_x) {
        // glue the +x side of domain A to the -x side of domain A+1 (cyclically)
        const int D = p->n_domains;
        for (int A = 0; A < D; ++A)
            for (int a = 1; a < 3; ++a)
                if (p->lo[3 * A + a] != p->lo[a] || p->hi[3 * A + a] != p->hi[a])
                    throw std::runtime_error("chained domains must share the y and z extents");
        auto elem = [&](int dm, int i, int j, int k) {
            const int* dd = p->dims + 3 * dm;
            return (int)(first[dm] + i + dd[0] * (j + dd[1] * k));
        };
        for (int A = 0; A < D; ++A) {
            const int Bd = (A + 1) % D;
            const int* da = p->dims + 3 * A;
            const int* db = p->dims + 3 * Bd;
            const int ra = da[1] == db[1] ? 0 : (db[1] == 2 * da[1] ? 1 : (da[1] == 2 * db[1] ? -1 : 9));
            const int rb = da[2] == db[2] ? 0 : (db[2] == 2 * da[2] ? 1 : (da[2] == 2 * db[2] ? -1 : 9));
            if (ra == 9 || rb == 9 || ra * rb < 0) throw std::runtime_error("chained domains must be 1:1 or 2:1");
            if (ra == 0 && rb == 0) {  // conforming
                for (int k = 0; k < da[2]; ++k)
                    for (int j = 0; j < da[1]; ++j) {
                        const int eA = elem(A, da[0] - 1, j, k), eB = elem(Bd, 0, j, k);
                        P.el[eA].nb[1] = eB;
                        P.el[eB].nb[0] = eA;
                    }
                continue;
            }
            // the coarser domain holds the big sides
            const bool bigA = ra > 0 || rb > 0;
            const int Dbig = bigA ? A : Bd, Dsm = bigA ? Bd : A;
            const int* dg = p->dims + 3 * Dbig;
            const int* ds = p->dims + 3 * Dsm;
            const int fB = bigA ? 1 : 0;
            const int sa = ra != 0, sb = rb != 0;
            for (int k = 0; k < dg[2]; ++k)
                for (int j = 0; j < dg[1]; ++j) {
                    Mortar M;
                    M.big = elem(Dbig, bigA ? dg[0] - 1 : 0, j, k);
                    M.fB = fB;
                    M.split[0] = sa;
                    M.split[1] = sb;
                    const int m = (int)P.mortars.size();
                    for (int qb = 0; qb <= sb; ++qb)
                        for (int qa = 0; qa <= sa; ++qa) {
                            const int q = qa + 2 * qb;
                            const int es = elem(Dsm, bigA ? 0 : ds[0] - 1, sa ? 2 * j + qa : j, sb ? 2 * k + qb : k);
                            M.small[q] = es;
                            P.el[es].nb[fB ^ 1] = -1;
                            P.el[es].mort[fB ^ 1] = m;
                            P.el[es].quad[fB ^ 1] = q;
                        }
                    P.el[M.big].nb[fB] = -1;
                    P.el[M.big].mort[fB] = m;
                    P.mortars.push_back(M);
                }
        }
    }
    for (size_t e = 0; e < P.el.size(); ++e) {
        Elem& E = P.el[e];
        E.N = p->N[e];
        E.fv = p->fv[e] != 0;
        if (E.N < 1 || E.N > 15) throw std::runtime_error("bad degree");
        E.n = E.fv ? (P.fv_own ? E.N + 1 : P.nfv) : E.N + 1;
        E.off = P.size;
        P.size += (int64_t)P.V * E.n * E.n * E.n;
    }
    if (need_ops) {
        std::vector<int> degs;
        for (auto& E : P.el) degs.push_back(E.N);
        std::sort(degs.begin(), degs.end());
        degs.erase(std::unique(degs.begin(), degs.end()), degs.end());
        for (int N : degs) {
            P.ops.basis[N] = make_basis(N, P.nodes);
            P.ops.vleg_inv[N] = leg_vandermonde_inv(N, P.nodes);
            // DG <-> FV maps between degree N and every sub-cell count in use
            // (global: n_fv; per element: N~+1 of every degree N~ present)
            for (int M : degs) {
                const int nf = P.fv_own ? M + 1 : P.nfv;
                if (!P.fv_own && nf < N + 1) continue;
                if (P.ops.d2f.count({N, nf})) continue;
                P.ops.d2f[{N, nf}] = dg2fv(N, nf, P.nodes);
                // V^{FV->DG}: the pseudo-inverse (a left inverse) on grids of at least
                // N+1 sub-cells; on coarser ones (per-element sub-cells only) the L2
                // projection of the piecewise constant, which keeps constants and
                // face integrals
                P.ops.f2d[{N, nf}] = nf >= N + 1 ? fv2dg(N, nf, P.nodes) : fv2dg_l2(N, nf, P.nodes);
            }
            for (int M : degs) P.ops.vm[{N, M}] = vmap(N, M, P.nodes);
            for (int h = 0; h < 2; ++h) {
                P.ops.mi[{N, h}] = mortar_interp(N, h, P.nodes);
                P.ops.mp[{N, h}] = mortar_proj(N, h, P.nodes);
            }
        }
        for (int h = 0; h < 2; ++h) {
            P.ops.mi_fv[h] = mortar_interp_fv(P.nfv, h);
            P.ops.mp_fv[h] = mortar_proj_fv(P.nfv, h);
        }
        if (P.fv_own)
            for (int a : degs)
                for (int b : degs) P.ops.ov[{a + 1, b + 1}] = fv_overlap(a + 1, b + 1);
        for (int n = 1; n <= 16; ++n) {
            vector<double> I((size_t)n * n, 0.0);
            for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
            P.ops.eye[n] = I;
        }
        for (auto& E : P.el)
            if (E.fv && E.n < E.N + 1) throw std::runtime_error("n_fv < N+1 for an FV element");
    }
    return P;
}

// Node index of the point with coordinate m along direction d and transverse
// coordinates (a, b) (in increasing axis order).
inline int node_index(int n, int d, int m, int a, int b) {
    if (d == 0) return m + n * (a + n * b);
    if (d == 1) return a + n * (m + n * b);
    return a + n * (b + n * m);
}

// Apply the tensor-product map M (nout x nin) in both face directions to a
// face field of nvar variables stored as in[var*nin^2 + a + nin*b]
// (first along a, then along b).
template <class T>
vector<T> map_face(const vector<T>& in, int nvar, int nin, int nout, const vector<double>& M) {
    vector<T> tmp((size_t)nvar * nout * nin, T(0.0));
    for (int v = 0; v < nvar; ++v)
        for (int bi = 0; bi < nin; ++bi)
            for (int ao = 0; ao < nout; ++ao) {
                T s = T(0.0);
                for (int ai = 0; ai < nin; ++ai)
                    s = s + T(M[ao * nin + ai]) * in[(size_t)v * nin * nin + ai + nin * bi];
                tmp[(size_t)v * nout * nin + ao + nout * bi] = s;
            }
    vector<T> out((size_t)nvar * nout * nout, T(0.0));
    for (int v = 0; v < nvar; ++v)
        for (int bo = 0; bo < nout; ++bo)
            for (int ao = 0; ao < nout; ++ao) {
                T s = T(0.0);
                for (int bi = 0; bi < nin; ++bi)
                    s = s + T(M[bo * nin + bi]) * tmp[(size_t)v * nout * nin + ao + nout * bi];
                out[(size_t)v * nout * nout + ao + nout * bo] = s;
            }
    return out;
}

// Tensor-product map with its own matrix along each face direction:
// out[var][ao + nout*bo] = sum Ma[ao][ai] Mb[bo][bi] in[var][ai + nin*bi].
template <class T>
vector<T> map_face2(const vector<T>& in, int nvar, int nin, int nout, const vector<double>& Ma,
                    const vector<double>& Mb) {
    vector<T> out((size_t)nvar * nout * nout, T(0.0));
    for (int v = 0; v < nvar; ++v)
        for (int bo = 0; bo < nout; ++bo)
            for (int ao = 0; ao < nout; ++ao) {
                T s = T(0.0);
                for (int bi = 0; bi < nin; ++bi)
                    for (int ai = 0; ai < nin; ++ai)
                        s = s + T(Ma[ao * nin + ai] * Mb[bo * nin + bi]) * in[(size_t)v * nin * nin + ai + nin * bi];
                out[(size_t)v * nout * nout + ao + nout * bo] = s;
            }
    return out;
}

// Sec. 3.2.3: the maps of quadrant q of mortar M along the face directions a
// (dir 0) and b (dir 1): interpolation from the big side to the virtual small
// side (proj = false) or L2 projection back (proj = true), on the big side's
// representation (degree N_big; FV sub-cells when the big element is FV or
// fvgrid is set); the identity along a direction that is not halved.
const vector<double>& mortar_map(const Problem& P, const Mortar& M, int q, int dir, bool proj, bool fvgrid) {
    const Elem& B = P.el[M.big];
    const bool fvg = fvgrid || B.fv;
    if (!M.split[dir]) return P.ops.eye.at(fvg ? P.nfv : B.n);
    const int h = dir == 0 ? q % 2 : q / 2;
    if (fvg) return proj ? P.ops.mp_fv[h] : P.ops.mi_fv[h];
    return proj ? P.ops.mp.at({B.N, h}) : P.ops.mi.at({B.N, h});
}

// A face field of the big side restricted to quadrant q (its virtual small side).
template <class T>
vector<T> to_virtual(const Problem& P, const Mortar& M, int q, const vector<T>& big, int nvar, bool fvgrid = false) {
    const int n = (fvgrid || P.el[M.big].fv) ? P.nfv : P.el[M.big].n;
    return map_face2(big, nvar, n, n, mortar_map(P, M, q, 0, false, fvgrid), mortar_map(P, M, q, 1, false, fvgrid));
}

// acc += the projection of a virtual small side's field of quadrant q onto the big side.
template <class T>
void add_from_virtual(const Problem& P, const Mortar& M, int q, const vector<T>& virt, int nvar, vector<T>& acc,
                      bool fvgrid = false) {
    const int n = (fvgrid || P.el[M.big].fv) ? P.nfv : P.el[M.big].n;
    vector<T> t = map_face2(virt, nvar, n, n, mortar_map(P, M, q, 0, true, fvgrid), mortar_map(P, M, q, 1, true, fvgrid));
    if (acc.empty()) acc.assign(t.size(), T(0.0));
    for (size_t i = 0; i < t.size(); ++i) acc[i] = acc[i] + t[i];
}

// V^{N_from -> N_to} on a face field; the identity when the degrees agree.
template <class T>
vector<T> map_face_deg(const Problem& P, const vector<T>& in, int nvar, int N_from, int N_to) {
    if (N_from == N_to) return in;
    return map_face(in, nvar, N_from + 1, N_to + 1, P.ops.vm.at({N_from, N_to}));
}

// Apply the tensor-product map M (nout x nin) in all three directions to a
// volume field of nvar variables (one direction at a time).
template <class T>
vector<T> map_volume(const T* in, int nvar, int nin, int nout, const vector<double>& M) {
    vector<T> a((size_t)nvar * nout * nin * nin, T(0.0));
    for (int v = 0; v < nvar; ++v)
        for (int k = 0; k < nin; ++k)
            for (int j = 0; j < nin; ++j)
                for (int i = 0; i < nout; ++i) {
                    T s = T(0.0);
                    for (int m = 0; m < nin; ++m)
                        s = s + T(M[i * nin + m]) * in[(size_t)v * nin * nin * nin + m + nin * (j + nin * k)];
                    a[(size_t)v * nout * nin * nin + i + nout * (j + nin * k)] = s;
                }
    vector<T> b((size_t)nvar * nout * nout * nin, T(0.0));
    for (int v = 0; v < nvar; ++v)
        for (int k = 0; k < nin; ++k)
            for (int j = 0; j < nout; ++j)
                for (int i = 0; i < nout; ++i) {
                    T s = T(0.0);
                    for (int m = 0; m < nin; ++m)
                        s = s + T(M[j * nin + m]) * a[(size_t)v * nout * nin * nin + i + nout * (m + nin * k)];
                    b[(size_t)v * nout * nout * nin + i + nout * (j + nout * k)] = s;
                }
    vector<T> c((size_t)nvar * nout * nout * nout, T(0.0));
    for (int v = 0; v < nvar; ++v)
        for (int k = 0; k < nout; ++k)
            for (int j = 0; j < nout; ++j)
                for (int i = 0; i < nout; ++i) {
                    T s = T(0.0);
                    for (int m = 0; m < nin; ++m)
                        s = s + T(M[k * nin + m]) * b[(size_t)v * nout * nout * nin + i + nout * (j + nout * m)];
                    c[(size_t)v * nout * nout * nout + i + nout * (j + nout * k)] = s;
                }
    return c;
}

template <class T>
struct ElemWork {
    vector<T> face_u[6];    // DG: trace of u; FV: boundary sub-cell means      (V x n^2)
    vector<T> face_layer[6];  // DG: V^{DG->FV} sub-cell means of the boundary layer (V x n_fv^2)
    vector<T> face_rec[6];  // FV: reconstructed face state at the element face (V x n^2)
    vector<T> face_g[6];    // DG: trace of the lifted gradient; FV: boundary-cell gradient (3V x n^2)
    vector<T> ustar[6];     // DG: lifting interface value U*                  (V x n^2)
    vector<T> flux[6];      // outward normal flux F*.n on the element's own representation (V x n^2)
    vector<T> div;          // volume (DG) or interior sub-cell face (FV) part of -R  (V x n^3)
};

// Convective flux choice per face (Sec. 5.1, the jet): riemann = 2 takes Roe-HH
// on faces between two DG elements and local Lax-Friedrichs on every face that
// touches FV data (FV sub-cell faces, FV/FV and DG/FV element faces).
int riemann_kind(const Problem& P, bool fv_involved) {
    if (P.riemann == 2) return fv_involved ? 0 : 1;
    return P.riemann;
}

// Face flux at one point: F* = F^c*(uL,uR) + (F^v(uL,gL) + F^v(uR,gR))/2 in +x_d direction.
template <class T>
void point_flux(const Problem& P, const T* uL, const T* gL, const T* uR, const T* gR, int d, T* F,
                bool fv_involved) {
    const int V = P.V;
    T Fc[MAXV], FvL[MAXV], FvR[MAXV];
    Prim<T> sL, sR;
    cons_to_prim(P.ph, uL, sL);
    cons_to_prim(P.ph, uR, sR);
    riemann(P.ph, riemann_kind(P, fv_involved), uL, sL, uR, sR, d, Fc);
    flux_visc(P.ph, uL, gL, sL, d, FvL);
    flux_visc(P.ph, uR, gR, sR, d, FvR);
    for (int v = 0; v < V; ++v) F[v] = Fc[v] + T(0.5) * (FvL[v] + FvR[v]);
}

// Kinetic-energy-preserving two-point flux of Pirozzoli in +x_d (Sec. 3.5):
// with arithmetic means {.} of the two states,
//   rho_k: {rho}{v_d}{Y_k},  rho v_j: {rho}{v_d}{v_j} + {p} delta_jd,  rho E: {rho}{v_d}{H},
// H = (rho E + p)/rho the total enthalpy (species: the transported mass
// fraction times the mean mass flux, so that the species fluxes add up to
// the mass flux {rho}{v_d}).
template <class T>
void kep_flux(const Phys& ph, const Prim<T>& a, const T& Ha, const Prim<T>& b, const T& Hb, int d, T* F) {
    const int nk = ph.nk;
    const T rho = T(0.5) * (a.rho + b.rho);
    const T vd = T(0.5) * (a.v[d] + b.v[d]);
    const T mass = rho * vd;
    for (int k = 0; k < nk; ++k) F[k] = mass * (T(0.5) * (a.Y[k] + b.Y[k]));
    for (int j = 0; j < 3; ++j) F[nk + j] = mass * (T(0.5) * (a.v[j] + b.v[j]));
    F[nk + d] = F[nk + d] + T(0.5) * (a.p + b.p);
    F[nk + 3] = mass * (T(0.5) * (Ha + Hb));
}

// Split form on LGL nodes (Sec. 3.5): the convective part of the volume term
// of node i along direction d is
//   sum_m 2 D_im F#(u_i, u_m) - (B_ii/w_i) F^c(u_i),   B = diag(-1, 0, .., 0, 1)
// (the strong form with the two-point flux; by summation by parts the weak
// form's sum_m Dhat_im F^c(u_m) is the same expression with F^c(u_m) in place
// of 2 F#(u_i, u_m)).  Added to div, which holds the viscous part.
template <class T>
void split_form_convective(const Problem& P, const Elem& E, const Basis1D& B, const T* u, vector<T>& div) {
    const int V = P.V, n = E.n, n3 = n * n * n;
    vector<Prim<T>> s(n3);
    vector<T> H(n3);  // total enthalpy (rho E + p) / rho
    for (int c = 0; c < n3; ++c) {
        T uc[MAXV];
        for (int v = 0; v < V; ++v) uc[v] = u[(size_t)v * n3 + c];
        cons_to_prim(P.ph, uc, s[c]);
        H[c] = (uc[P.ph.nk + 3] + s[c].p) / s[c].rho;
    }
    for (int d = 0; d < 3; ++d) {
        const T metric = T(2.0 / E.h[d]);
        for (int b = 0; b < n; ++b)
            for (int a = 0; a < n; ++a)
                for (int i = 0; i < n; ++i) {
                    const int ci = node_index(n, d, i, a, b);
                    T ui[MAXV], Fs[MAXV], acc[MAXV];
                    for (int v = 0; v < V; ++v) {
                        ui[v] = u[(size_t)v * n3 + ci];
                        acc[v] = T(0.0);
                    }
                    for (int m = 0; m < n; ++m) {
                        const int cm = node_index(n, d, m, a, b);
                        kep_flux(P.ph, s[ci], H[ci], s[cm], H[cm], d, Fs);
                        const T two_D = T(2.0 * B.D[i * n + m]);
                        for (int v = 0; v < V; ++v) acc[v] = acc[v] + two_D * Fs[v];
                    }
                    if (i == 0 || i == n - 1) {  // boundary nodes: -(B_ii/w_i) F^c(u_i)
                        T Fc[MAXV];
                        flux_conv(P.ph, ui, s[ci], d, Fc);
                        const T c = T((i == 0 ? 1.0 : -1.0) / B.w[i]);
                        for (int v = 0; v < V; ++v) acc[v] = acc[v] + c * Fc[v];
                    }
                    for (int v = 0; v < V; ++v)
                        div[(size_t)v * n3 + ci] = div[(size_t)v * n3 + ci] + metric * acc[v];
                }
    }
}

// Whether FV data lies across face f of E (at a mortar: the big element, or
// any small element).
bool fv_across(const Problem& P, const Elem& E, int f) {
    if (E.mort[f] < 0) return P.el[E.nb[f]].fv;
    const Mortar& M = P.mortars[E.mort[f]];
    if (E.quad[f] >= 0) return P.el[M.big].fv;
    for (int q = 0; q < 4; ++q)
        if (M.small[q] >= 0 && P.el[M.small[q]].fv) return true;
    return false;
}

template <class T>
T minmod(T a, T b) {
    // minmod(a,b) = 0 if a b <= 0, else the argument of smaller magnitude (a on ties)
    if (val(a) * val(b) <= 0.0) return T(0.0);
    return std::fabs(val(a)) <= std::fabs(val(b)) ? a : b;
}

// The step being counted, for the operation-counting instantiation only (the
// other instantiations may run on several threads at once).
template <class T>
inline void set_phase(int ph) {
    if constexpr (std::is_same_v<T, Counted>) flop_counter().phase = ph;
}

template <class T>
void eval_rhs_t(const Problem& P, const T* U, T* R, bool parallel = true) {
    const int V = P.V, nfv = P.nfv;
    const int nel = (int)P.el.size();
    vector<ElemWork<T>> W(nel);

    // ---- step 1: face values of every element
    set_phase<T>(1);
#pragma omp parallel for schedule(dynamic, 16) if (parallel)
    for (int e = 0; e < nel; ++e) {
        const Elem& E = P.el[e];
        const int n = E.n;
        const T* u = U + E.off;
        for (int f = 0; f < 6; ++f) {
            const int d = f / 2, s = f % 2;
            vector<T> fu((size_t)V * n * n, T(0.0));
            for (int v = 0; v < V; ++v)
                for (int b = 0; b < n; ++b)
                    for (int a = 0; a < n; ++a) {
                        T val_ = T(0.0);
                        if (E.fv) {
                            val_ = u[(size_t)v * n * n * n + node_index(n, d, s ? n - 1 : 0, a, b)];
                        } else {
                            const vector<double>& l = s ? P.ops.B(E.N).lp : P.ops.B(E.N).lm;
                            for (int m = 0; m < n; ++m)
                                val_ = val_ + T(l[m]) * u[(size_t)v * n * n * n + node_index(n, d, m, a, b)];
                        }
                        fu[(size_t)v * n * n + a + n * b] = val_;
                    }
            W[e].face_u[f] = fu;
            // the boundary layer of sub-cell means that an FV neighbour sees:
            // V^{DG->FV} in all three directions, keeping the sub-cells next to face f
            // (counted with the FV step, which is where it is needed)
            const bool fv_neighbour = fv_across(P, E, f);
            if (!E.fv && fv_neighbour && !parallel) set_phase<T>(2);
            if (!E.fv && fv_neighbour) {
                // on the neighbour's sub-cell grid (per element: its own count)
                const int nf = (P.fv_own && E.nb[f] >= 0) ? P.el[E.nb[f]].n : P.nfv;
                const vector<double>& A = P.ops.d2f.at({E.N, nf});
                const int row = s ? nf - 1 : 0;
                vector<T> q((size_t)V * n * n, T(0.0));
                for (int v = 0; v < V; ++v)
                    for (int b = 0; b < n; ++b)
                        for (int a = 0; a < n; ++a) {
                            T t = T(0.0);
                            for (int m = 0; m < n; ++m)
                                t = t + T(A[row * n + m]) * u[(size_t)v * n * n * n + node_index(n, d, m, a, b)];
                            q[(size_t)v * n * n + a + n * b] = t;
                        }
                W[e].face_layer[f] = map_face(q, V, n, nf, A);
            }
            if (!parallel) set_phase<T>(1);
        }
    }

    // ---- step 2: FV sub-cell elements (Sec. 3.1.2)
    set_phase<T>(2);
#pragma omp parallel for schedule(dynamic, 1) if (parallel)
    for (int e = 0; e < nel; ++e) {
        const Elem& E = P.el[e];
        if (!E.fv) continue;
        const int n = E.n, n3 = n * n * n;
        const double l = 2.0 / n;  // sub-cell size in reference coordinates
        const T* u = U + E.off;
        // Reading: the value beyond the element boundary is the neighbour's
        // face-adjacent sub-cell mean: an FV neighbour's own, or, for a DG
        // neighbour, its solution mapped to sub-cell means by V^{DG->FV}
        // (Sec. 3.2.1: the DG side is transformed to the FV representation).
        // The distance to the neighbour's sub-cell centre, in this element's
        // reference coordinates, is l/2 (1 + h_nb/h), l when the sizes agree.
        // Reading at a mortar (Sec. 3.2.3 maps the face data, the paper says
        // nothing of the reconstruction stencil): a small side sees the big
        // side's layer on its quadrant (M^FV_01, M^FV_02), the big side the
        // small sides' layers projected onto its sub-cells (M^FV_10, M^FV_20).
        vector<T> nbval[6];
        double nbdist[6];
        auto layer = [&](int q, int fq) -> const vector<T>& {
            return P.el[q].fv ? W[q].face_u[fq] : W[q].face_layer[fq];
        };
        for (int f = 0; f < 6; ++f) {
            const int d = f / 2;
            if (E.mort[f] < 0) {
                const Elem& Q = P.el[E.nb[f]];
                if (Q.fv && Q.n != n) {
                    // per-element sub-cells, an FV neighbour with another count: its
                    // boundary layer by the overlap map onto this element's face grid;
                    // the centre distance l/2 + (h_nb/h)(1/n_nb) in this element's
                    // reference coordinates
                    nbval[f] = map_face(layer(E.nb[f], f ^ 1), V, Q.n, n, P.ops.ov.at({Q.n, n}));
                    nbdist[f] = l / 2 + (Q.h[d] / E.h[d]) / Q.n;
                    continue;
                }
                nbval[f] = layer(E.nb[f], f ^ 1);
                nbdist[f] = l / 2 * (1.0 + Q.h[d] / E.h[d]);
                continue;
            }
            const Mortar& M = P.mortars[E.mort[f]];
            if (E.quad[f] >= 0) {
                nbval[f] = to_virtual(P, M, E.quad[f], layer(M.big, M.fB), V, true);
                nbdist[f] = l / 2 * (1.0 + P.el[M.big].h[d] / E.h[d]);
            } else {
                nbval[f].clear();
                for (int q = 0; q < 4; ++q)
                    if (M.small[q] >= 0) add_from_virtual(P, M, q, layer(M.small[q], f ^ 1), V, nbval[f], true);
                nbdist[f] = l / 2 * (1.0 + P.el[M.small[0]].h[d] / E.h[d]);
            }
        }
        // primitive reconstruction variables of every sub-cell and of the neighbour values
        vector<T> w((size_t)V * n3);
        for (int c = 0; c < n3; ++c) {
            T uc[MAXV], wc[MAXV];
            for (int v = 0; v < V; ++v) uc[v] = u[(size_t)v * n3 + c];
            cons_to_recvars(P.ph, uc, wc);
            for (int v = 0; v < V; ++v) w[(size_t)v * n3 + c] = wc[v];
        }
        vector<T> nbw[6];
        for (int f = 0; f < 6; ++f) {
            nbw[f].resize((size_t)V * n * n);
            for (int p = 0; p < n * n; ++p) {
                T uc[MAXV], wc[MAXV];
                for (int v = 0; v < V; ++v) uc[v] = nbval[f][(size_t)v * n * n + p];
                cons_to_recvars(P.ph, uc, wc);
                for (int v = 0; v < V; ++v) nbw[f][(size_t)v * n * n + p] = wc[v];
            }
        }
        // reconstructed states at the two faces of every cell along every direction
        // recm[d], recp[d]: conservative state at the cell's -d and +d face (V x n^3)
        vector<T> recm[3], recp[3];
        // central-difference gradient of the conservative variables (3V x n^3)
        vector<T> grad((size_t)3 * V * n3, T(0.0));
        for (int d = 0; d < 3; ++d) {
            recm[d].assign((size_t)V * n3, T(0.0));
            recp[d].assign((size_t)V * n3, T(0.0));
            for (int b = 0; b < n; ++b)
                for (int a = 0; a < n; ++a)
                    for (int m = 0; m < n; ++m) {
                        const int c = node_index(n, d, m, a, b);
                        const int p = a + n * b;
                        const int cl = m > 0 ? node_index(n, d, m - 1, a, b) : -1;
                        const int cr = m < n - 1 ? node_index(n, d, m + 1, a, b) : -1;
                        const double dl = cl >= 0 ? l : nbdist[2 * d];
                        const double dr = cr >= 0 ? l : nbdist[2 * d + 1];
                        T wm[MAXV], wp[MAXV];
                        for (int v = 0; v < V; ++v) {
                            T wc = w[(size_t)v * n3 + c];
                            T wl = cl >= 0 ? w[(size_t)v * n3 + cl] : nbw[2 * d][(size_t)v * n * n + p];
                            T wr = cr >= 0 ? w[(size_t)v * n3 + cr] : nbw[2 * d + 1][(size_t)v * n * n + p];
                            // second-order TVD reconstruction with the minmod limiter
                            T slope = minmod((wc - wl) / T(dl), (wr - wc) / T(dr));
                            wm[v] = wc - slope * T(l / 2);
                            wp[v] = wc + slope * T(l / 2);
                            // viscous terms: central differences of the conservative sub-cell means
                            T ucl = cl >= 0 ? u[(size_t)v * n3 + cl] : nbval[2 * d][(size_t)v * n * n + p];
                            T ucr = cr >= 0 ? u[(size_t)v * n3 + cr] : nbval[2 * d + 1][(size_t)v * n * n + p];
                            grad[((size_t)d * V + v) * n3 + c] = (ucr - ucl) / T(dl + dr) * T(2.0 / E.h[d]);
                        }
                        T um[MAXV], up[MAXV];
                        recvars_to_cons(P.ph, wm, um);
                        recvars_to_cons(P.ph, wp, up);
                        for (int v = 0; v < V; ++v) {
                            recm[d][(size_t)v * n3 + c] = um[v];
                            recp[d][(size_t)v * n3 + c] = up[v];
                        }
                    }
        }
        // interior sub-cell faces: F* = F^c*(rec-, rec+) + (F^v(rec-, g-) + F^v(rec+, g+))/2;
        // div accumulates sum over faces of (outward flux) * |face| / |cell| = (n/h_d) F.n
        vector<T> div((size_t)V * n3, T(0.0));
        for (int d = 0; d < 3; ++d) {
            const T scale = T(n / E.h[d]);
            for (int b = 0; b < n; ++b)
                for (int a = 0; a < n; ++a)
                    for (int m = 0; m + 1 < n; ++m) {
                        const int cL = node_index(n, d, m, a, b), cR = node_index(n, d, m + 1, a, b);
                        T uL[MAXV], uR[MAXV], gL[3 * MAXV], gR[3 * MAXV], F[MAXV];
                        for (int v = 0; v < V; ++v) {
                            uL[v] = recp[d][(size_t)v * n3 + cL];
                            uR[v] = recm[d][(size_t)v * n3 + cR];
                        }
                        for (int dd = 0; dd < 3; ++dd)
                            for (int v = 0; v < V; ++v) {
                                gL[dd * V + v] = grad[((size_t)dd * V + v) * n3 + cL];
                                gR[dd * V + v] = grad[((size_t)dd * V + v) * n3 + cR];
                            }
                        point_flux(P, uL, gL, uR, gR, d, F, true);
                        for (int v = 0; v < V; ++v) {
                            div[(size_t)v * n3 + cL] = div[(size_t)v * n3 + cL] + scale * F[v];
                            div[(size_t)v * n3 + cR] = div[(size_t)v * n3 + cR] - scale * F[v];
                        }
                    }
        }
        W[e].div = div;
        // element-face states and boundary-cell gradients for the coupling
        for (int f = 0; f < 6; ++f) {
            const int d = f / 2, s = f % 2;
            vector<T> fr((size_t)V * n * n), fg((size_t)3 * V * n * n);
            for (int b = 0; b < n; ++b)
                for (int a = 0; a < n; ++a) {
                    const int c = node_index(n, d, s ? n - 1 : 0, a, b);
                    for (int v = 0; v < V; ++v)
                        fr[(size_t)v * n * n + a + n * b] = s ? recp[d][(size_t)v * n3 + c] : recm[d][(size_t)v * n3 + c];
                    for (int dv = 0; dv < 3 * V; ++dv)
                        fg[(size_t)dv * n * n + a + n * b] = grad[(size_t)dv * n3 + c];
                }
            W[e].face_rec[f] = fr;
            W[e].face_g[f] = fg;
        }
    }

    // ---- step 3: BR1 lifting interface value U* = (u- + u+)/2 (Eq. 19)
    set_phase<T>(3);
#pragma omp parallel for schedule(dynamic, 16) if (parallel)
    for (int e = 0; e < nel; ++e) {
        const Elem& E = P.el[e];
        if (E.fv) continue;
        // U* on this side's degree N from this side's trace and the other side's
        // data (its degree-No trace, or its FV reconstructed face state)
        auto lift_with = [&](const vector<T>& mine, int N, bool ofv, int No, const vector<T>& other) {
            vector<T> us;
            if (ofv) {
                // Sec. 3.2.2: FV side mapped to the DG element's polynomial data by V^{FV->DG}
                const int nfo = P.fv_own ? No + 1 : nfv;
                vector<T> o = map_face(other, V, nfo, N + 1, P.ops.f2d.at({N, nfo}));
                us.resize(mine.size());
                for (size_t i = 0; i < mine.size(); ++i) us[i] = T(0.5) * (mine[i] + o[i]);
            } else {
                // Sec. 3.2.2: lifting flux on the lower degree, interpolated back up
                const int Nm = std::min(N, No);
                vector<T> a = map_face_deg(P, mine, V, N, Nm);
                vector<T> b = map_face_deg(P, other, V, No, Nm);
                vector<T> avg(a.size());
                for (size_t i = 0; i < a.size(); ++i) avg[i] = T(0.5) * (a[i] + b[i]);
                us = map_face_deg(P, avg, V, Nm, N);
            }
            return us;
        };
        auto data = [&](int q, int fq) -> const vector<T>& { return P.el[q].fv ? W[q].face_rec[fq] : W[q].face_u[fq]; };
        for (int f = 0; f < 6; ++f) {
            const vector<T>& mine = W[e].face_u[f];
            if (E.mort[f] < 0) {
                const Elem& Q = P.el[E.nb[f]];
                W[e].ustar[f] = lift_with(mine, E.N, Q.fv, Q.N, data(E.nb[f], f ^ 1));
                continue;
            }
            // Sec. 3.2.3: the lifting value on each virtual small side, by the
            // conforming rules above; the big side takes the L2 projection of the
            // virtual sides' values
            const Mortar& M = P.mortars[E.mort[f]];
            const Elem& Bg = P.el[M.big];
            if (E.quad[f] >= 0) {
                W[e].ustar[f] = lift_with(mine, E.N, Bg.fv, Bg.N, to_virtual(P, M, E.quad[f], data(M.big, M.fB), V));
            } else {
                vector<T> acc;
                for (int q = 0; q < 4; ++q) {
                    if (M.small[q] < 0) continue;
                    const Elem& S = P.el[M.small[q]];
                    vector<T> Uq = lift_with(to_virtual(P, M, q, mine, V), E.N, S.fv, S.N, data(M.small[q], f ^ 1));
                    add_from_virtual(P, M, q, Uq, V, acc);
                }
                W[e].ustar[f] = acc;
            }
        }
    }

    // ---- step 4: lifting (Eq. 23) and volume integral (Eq. 22) of DG elements.
    set_phase<T>(4);
    // Cartesian elements: J = hx hy hz / 8, metric terms J dxi_d/dx_d = J (2/h_d),
    // so contravariant quantities divided by J carry the factor 2/h_d.
    // Reading (Eq. 23): the lifted variable is the gradient, g^d = +(1/J)[...].
    // Reading (Eq. 24): Dhat_ij = -(w_j/w_i) D_ji.
#pragma omp parallel for schedule(dynamic, 4) if (parallel)
    for (int e = 0; e < nel; ++e) {
        const Elem& E = P.el[e];
        if (E.fv) continue;
        const int n = E.n, n3 = n * n * n;
        const Basis1D& B = P.ops.B(E.N);
        const T* u = U + E.off;
        vector<T> g((size_t)3 * V * n3, T(0.0));
        for (int d = 0; d < 3; ++d) {
            const T metric = T(2.0 / E.h[d]);
            for (int v = 0; v < V; ++v)
                for (int b = 0; b < n; ++b)
                    for (int a = 0; a < n; ++a)
                        for (int i = 0; i < n; ++i) {
                            T s = T(0.0);
                            for (int m = 0; m < n; ++m)
                                s = s + T(B.Dhat[i * n + m]) * u[(size_t)v * n3 + node_index(n, d, m, a, b)];
                            const int p = a + n * b;
                            s = s + T(B.lhp[i]) * W[e].ustar[2 * d + 1][(size_t)v * n * n + p]
                                  - T(B.lhm[i]) * W[e].ustar[2 * d][(size_t)v * n * n + p];
                            g[((size_t)d * V + v) * n3 + node_index(n, d, i, a, b)] = metric * s;
                        }
        }
        // fluxes at the nodes
        vector<T> F((size_t)3 * V * n3);
        for (int c = 0; c < n3; ++c) {
            T uc[MAXV], gc[3 * MAXV], Fc[MAXV], Fv[MAXV];
            for (int v = 0; v < V; ++v) uc[v] = u[(size_t)v * n3 + c];
            for (int dv = 0; dv < 3 * V; ++dv) gc[dv] = g[(size_t)dv * n3 + c];
            Prim<T> s;
            cons_to_prim(P.ph, uc, s);
            PrimGrad<T> G;
            prim_grad(P.ph, gc, s, G);  // one chain rule per node, shared by the three directions
            for (int d = 0; d < 3; ++d) {
                flux_visc(P.ph, G, s, d, Fv);
                if (P.split) {  // the convective part follows in split_form_convective
                    for (int v = 0; v < V; ++v) F[((size_t)d * V + v) * n3 + c] = Fv[v];
                } else {
                    flux_conv(P.ph, uc, s, d, Fc);
                    for (int v = 0; v < V; ++v) F[((size_t)d * V + v) * n3 + c] = Fc[v] + Fv[v];
                }
            }
        }
        // volume integral sum_m Ftilde_m Dhat_im / J
        vector<T> div((size_t)V * n3, T(0.0));
        for (int d = 0; d < 3; ++d) {
            const T metric = T(2.0 / E.h[d]);
            for (int v = 0; v < V; ++v)
                for (int b = 0; b < n; ++b)
                    for (int a = 0; a < n; ++a)
                        for (int i = 0; i < n; ++i) {
                            T s = T(0.0);
                            for (int m = 0; m < n; ++m)
                                s = s + T(B.Dhat[i * n + m]) * F[((size_t)d * V + v) * n3 + node_index(n, d, m, a, b)];
                            const int c = node_index(n, d, i, a, b);
                            div[(size_t)v * n3 + c] = div[(size_t)v * n3 + c] + metric * s;
                        }
        }
        if (P.split) split_form_convective(P, E, B, u, div);
        W[e].div = div;
        // traces of the lifted gradient on the six faces
        for (int f = 0; f < 6; ++f) {
            const int d = f / 2, s = f % 2;
            const vector<double>& lb = s ? B.lp : B.lm;
            vector<T> fg((size_t)3 * V * n * n, T(0.0));
            for (int dv = 0; dv < 3 * V; ++dv)
                for (int b = 0; b < n; ++b)
                    for (int a = 0; a < n; ++a) {
                        T t = T(0.0);
                        for (int m = 0; m < n; ++m) t = t + T(lb[m]) * g[(size_t)dv * n3 + node_index(n, d, m, a, b)];
                        fg[(size_t)dv * n * n + a + n * b] = t;
                    }
            W[e].face_g[f] = fg;
        }
    }

    // ---- step 5: face fluxes; every conforming face is visited once, from its
    // lower element L, every mortar once, from its big side
    set_phase<T>(5);
    for (int e = 0; e < nel; ++e)
        for (int f = 0; f < 6; ++f) W[e].flux[f].clear();
    // One side of a face: FV flag, degree, and its face data (DG trace of u or FV
    // reconstructed state; gradient trace).
    struct Side {
        bool fv;
        int N;
        const vector<T>* u;
        const vector<T>* g;
    };
    // F* in +x_d between a lower side L and an upper side R, returned on each
    // side's own representation (FL, FR).
    auto pair_flux = [&](int d, const Side& L, const Side& Rr, vector<T>& FL, vector<T>& FR) {
        // common representation (Sec. 3.2.1): max degree, or FV data if either side is FV
        vector<T> uL, gL, uR, gR;
        int nc;
        const bool common_fv = L.fv || Rr.fv;
        if (!common_fv) {
            const int Nc = std::max(L.N, Rr.N);
            nc = Nc + 1;
            uL = map_face_deg(P, *L.u, V, L.N, Nc);
            gL = map_face_deg(P, *L.g, 3 * V, L.N, Nc);
            uR = map_face_deg(P, *Rr.u, V, Rr.N, Nc);
            gR = map_face_deg(P, *Rr.g, 3 * V, Rr.N, Nc);
        } else {
            // FV data (Sec. 3.2.1): a DG/FV face on the FV side's sub-cell grid,
            // the DG side by V^{DG->FV} and back by V^{FV->DG}; two FV sides with
            // different counts (per-element sub-cells) on the finer grid, the
            // coarser side by the overlap map (piecewise-constant L2 projection)
            // and back by the overlap map the other way
            const int nL = L.fv ? (P.fv_own ? L.N + 1 : nfv) : 0;
            const int nR = Rr.fv ? (P.fv_own ? Rr.N + 1 : nfv) : 0;
            nc = std::max(nL, nR);
            auto to_common = [&](const Side& S, int ns, vector<T>& u, vector<T>& g) {
                if (S.fv && ns == nc) {
                    u = *S.u;
                    g = *S.g;
                } else if (S.fv) {
                    u = map_face(*S.u, V, ns, nc, P.ops.ov.at({ns, nc}));
                    g = map_face(*S.g, 3 * V, ns, nc, P.ops.ov.at({ns, nc}));
                } else {
                    u = map_face(*S.u, V, S.N + 1, nc, P.ops.d2f.at({S.N, nc}));
                    g = map_face(*S.g, 3 * V, S.N + 1, nc, P.ops.d2f.at({S.N, nc}));
                }
            };
            to_common(L, nL, uL, gL);
            to_common(Rr, nR, uR, gR);
        }
        const int np = nc * nc;
        vector<T> Fc((size_t)V * np);
        for (int p = 0; p < np; ++p) {
            T a[MAXV], b[MAXV], ga[3 * MAXV], gb[3 * MAXV], F[MAXV];
            for (int v = 0; v < V; ++v) { a[v] = uL[(size_t)v * np + p]; b[v] = uR[(size_t)v * np + p]; }
            for (int dv = 0; dv < 3 * V; ++dv) { ga[dv] = gL[(size_t)dv * np + p]; gb[dv] = gR[(size_t)dv * np + p]; }
            point_flux(P, a, ga, b, gb, d, F, common_fv);
            for (int v = 0; v < V; ++v) Fc[(size_t)v * np + p] = F[v];
        }
        // back to each side's native representation (projection / V^{FV->DG})
        auto back = [&](const Side& S) -> vector<T> {
            if (!common_fv) return map_face_deg(P, Fc, V, nc - 1, S.N);
            if (S.fv) {
                const int ns = P.fv_own ? S.N + 1 : nfv;
                return ns == nc ? Fc : map_face(Fc, V, nc, ns, P.ops.ov.at({nc, ns}));
            }
            return map_face(Fc, V, nc, S.N + 1, P.ops.f2d.at({S.N, nc}));
        };
        FL = back(L);
        FR = back(Rr);
    };
    auto side = [&](int e, int f) -> Side {
        const Elem& E = P.el[e];
        return Side{E.fv, E.N, E.fv ? &W[e].face_rec[f] : &W[e].face_u[f], &W[e].face_g[f]};
    };
#pragma omp parallel for schedule(dynamic, 16) if (parallel)
    for (int e = 0; e < nel; ++e) {
        for (int d = 0; d < 3; ++d) {
            if (P.el[e].mort[2 * d + 1] >= 0) continue;
            const int eL = e, eR = P.el[e].nb[2 * d + 1];
            const int fL = 2 * d + 1, fR = 2 * d;
            vector<T> FLs, FRs;
            pair_flux(d, side(eL, fL), side(eR, fR), FLs, FRs);
            for (auto& x : FRs) x = -x;  // outward normal of the upper element is -x_d
            W[eL].flux[fL] = FLs;
            W[eR].flux[fR] = FRs;
        }
    }
    // Sec. 3.2.3: at a mortar the big side's face data is interpolated to each
    // virtual small side (M_01, M_02, or M^FV), the flux computed there against
    // the small side by the conforming rules, and the virtual sides' fluxes
    // projected back onto the big side (M_10, M_20, or M^FV).
    const int nmort = (int)P.mortars.size();
#pragma omp parallel for schedule(dynamic, 4) if (parallel)
    for (int m = 0; m < nmort; ++m) {
        const Mortar& M = P.mortars[m];
        const Elem& Bg = P.el[M.big];
        const int fB = M.fB, fS = fB ^ 1;
        const bool big_lower = fB == 1;
        const vector<T>& bu = Bg.fv ? W[M.big].face_rec[fB] : W[M.big].face_u[fB];
        vector<T> acc;
        for (int q = 0; q < 4; ++q) {
            const int es = M.small[q];
            if (es < 0) continue;
            const vector<T> vu = to_virtual(P, M, q, bu, V);
            const vector<T> vg = to_virtual(P, M, q, W[M.big].face_g[fB], 3 * V);
            const Side vs{Bg.fv, Bg.N, &vu, &vg};
            vector<T> FL, FR;
            if (big_lower) {
                pair_flux(0, vs, side(es, fS), FL, FR);
                for (auto& x : FR) x = -x;
                W[es].flux[fS] = FR;
                add_from_virtual(P, M, q, FL, V, acc);
            } else {
                pair_flux(0, side(es, fS), vs, FL, FR);
                for (auto& x : FR) x = -x;
                W[es].flux[fS] = FL;
                add_from_virtual(P, M, q, FR, V, acc);
            }
        }
        W[M.big].flux[fB] = acc;
    }

    // ---- step 6: surface integral and -1/J (Eqs. 22, 26)
    set_phase<T>(6);
#pragma omp parallel for schedule(dynamic, 16) if (parallel)
    for (int e = 0; e < nel; ++e) {
        const Elem& E = P.el[e];
        const int n = E.n, n3 = n * n * n;
        vector<T> div = W[e].div;
        if (!E.fv) {
            const Basis1D& B = P.ops.B(E.N);
            for (int d = 0; d < 3; ++d) {
                const T metric = T(2.0 / E.h[d]);
                for (int v = 0; v < V; ++v)
                    for (int b = 0; b < n; ++b)
                        for (int a = 0; a < n; ++a)
                            for (int i = 0; i < n; ++i) {
                                const int c = node_index(n, d, i, a, b), p = a + n * b;
                                T s = T(B.lhp[i]) * W[e].flux[2 * d + 1][(size_t)v * n * n + p]
                                    + T(B.lhm[i]) * W[e].flux[2 * d][(size_t)v * n * n + p];
                                div[(size_t)v * n3 + c] = div[(size_t)v * n3 + c] + metric * s;
                            }
            }
        } else {
            for (int d = 0; d < 3; ++d) {
                const T scale = T(n / E.h[d]);
                for (int s = 0; s < 2; ++s)
                    for (int v = 0; v < V; ++v)
                        for (int b = 0; b < n; ++b)
                            for (int a = 0; a < n; ++a) {
                                const int c = node_index(n, d, s ? n - 1 : 0, a, b);
                                div[(size_t)v * n3 + c] = div[(size_t)v * n3 + c] + scale * W[e].flux[2 * d + s][(size_t)v * n * n + a + n * b];
                            }
            }
        }
        for (int i = 0; i < V * n3; ++i) R[E.off + i] = -div[i];
    }
    set_phase<T>(0);
}

// ------------------------------------------------------------------ time step, Sec. 3.3
// Reading: alpha_RK = beta_RK = 1; lambda^c / dx -> sum_d (|v_d| + c)/dx_d;
// delta^v = max(4/3 mu/rho, kappa mu/(Pr rho), max_k D_k) with sum_d 1/dx_d^2;
// DG: dx_d = h_d and the factor (2N+1); FV: dx_d = h_d/n_fv and factor 1.
void time_step(const Problem& P, const double* U, double cfl_c, double cfl_v, double out[3]) {
    double mc = INFINITY, mv = INFINITY;
    double maxD = 0.0;
    bool viscous = false;
    for (int k = 0; k < P.ph.nk; ++k) {
        maxD = std::max(maxD, P.ph.D[k]);
        if (P.ph.mu[k] != 0.0 || P.ph.D[k] != 0.0) viscous = true;
    }
    for (const Elem& E : P.el) {
        const int n3 = E.n * E.n * E.n;
        const double fac = E.fv ? 1.0 : (2.0 * E.N + 1.0);
        double dx[3];
        for (int d = 0; d < 3; ++d) dx[d] = E.fv ? E.h[d] / E.n : E.h[d];
        for (int c = 0; c < n3; ++c) {
            double uc[MAXV];
            for (int v = 0; v < P.V; ++v) uc[v] = U[E.off + (int64_t)v * n3 + c];
            Prim<double> s;
            cons_to_prim(P.ph, uc, s);
            double lam = 0.0;
            for (int d = 0; d < 3; ++d) lam += (std::fabs(s.v[d]) + s.c) / dx[d];
            mc = std::min(mc, cfl_c / (lam * fac));
            if (viscous) {
                double dv = std::max(4.0 / 3.0 * s.mu / s.rho, s.kappa * s.mu / (s.pr * s.rho));
                dv = std::max(dv, maxD);
                double sdx = 0.0;
                for (int d = 0; d < 3; ++d) sdx += 1.0 / (dx[d] * dx[d]);
                mv = std::min(mv, cfl_v / (dv * sdx * fac));
            }
        }
    }
    out[1] = mc;
    out[2] = mv;
    out[0] = viscous ? 1.0 / (1.0 / mc + 1.0 / mv) : mc;
}

// ------------------------------------------------------------------ SSP-RK3 (Shu-Osher)
//   U1 = U0 + dt R(U0);  U2 = 3/4 U0 + 1/4 (U1 + dt R(U1));  U3 = 1/3 U0 + 2/3 (U2 + dt R(U2))
// post(U) is applied to every stage state (the positivity limiter, Sec. 3.5).
template <class Rhs, class Post>
void ssp_rk3_step(int64_t n, double* U, double dt, Rhs rhs, Post post) {
    static const double a[3] = {0.0, 0.75, 1.0 / 3.0};
    static const double b[3] = {1.0, 0.25, 2.0 / 3.0};
    vector<double> U0(U, U + n), Us(U, U + n), Rv(n);
    for (int s = 0; s < 3; ++s) {
        rhs(Us.data(), Rv.data());
        for (int64_t i = 0; i < n; ++i) Us[i] = a[s] * U0[i] + b[s] * (Us[i] + dt * Rv[i]);
        post(Us.data());
    }
    std::copy(Us.begin(), Us.end(), U);
}

template <class Rhs>
void ssp_rk3_step(int64_t n, double* U, double dt, Rhs rhs) {
    ssp_rk3_step(n, U, dt, rhs, [](double*) {});
}

// ------------------------------------------------------------------ low-storage RK4 (Sec. 3.3)
// The explicit fourth-order low-storage scheme the paper cites (Kennedy and
// Carpenter), read as the five-stage 2N-storage method of Carpenter and Kennedy
// (1994), coefficients as published:
//   dU <- A_s dU + dt R(U);   U <- U + B_s dU,   s = 1..5,  A_1 = 0.
template <class Rhs, class Post>
void lsrk4_step(int64_t n, double* U, double dt, Rhs rhs, Post post) {
    static const double A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                                -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
    static const double B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                                1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                                2277821191437.0 / 14882151754819.0};
    vector<double> dU(n, 0.0), Rv(n);
    for (int s = 0; s < 5; ++s) {
        rhs(U, Rv.data());
        for (int64_t i = 0; i < n; ++i) {
            dU[i] = A[s] * dU[i] + dt * Rv[i];
            U[i] = U[i] + B[s] * dU[i];
        }
        post(U);
    }
}

template <class Rhs>
void lsrk4_step(int64_t n, double* U, double dt, Rhs rhs) {
    lsrk4_step(n, U, dt, rhs, [](double*) {});
}

// ------------------------------------------------------------------ positivity limiter (Sec. 3.5)
// Zhang and Shu's limiter on every DG element (FV elements are left alone):
// with the element mean ubar (quadrature of the element's own nodes, exact for
// its polynomial) and the check points = the nodes and the points of the six
// faces (the face values that the face fluxes use),
//  (1) every partial density: theta_k = (ubar_k - eps_k)/(ubar_k - min rho_k) if the
//      minimum is below eps_k = min(eps, ubar_k); rho_k <- ubar_k + theta_k (rho_k - ubar_k);
//  (2) the internal energy rho e = rho E - |rho v|^2/(2 rho) (positive exactly
//      when the pressure is, kappa > 1): at every check point with rho e < eps_e =
//      min(eps, rho e(ubar)), t = the root in (0, 1) of rho e(ubar + t (u - ubar))
//      = eps_e (found by bisection; rho e is concave along the segment);
//      theta = min t;  u <- ubar + theta (u - ubar), every variable.
// Reading (the paper names the limiter only): partial densities limited one by
// one; check points include the face points; applied to every stage state.
double internal_energy(int nk, const double* u) {
    double rho = 0.0;
    for (int k = 0; k < nk; ++k) rho += u[k];
    return u[nk + 3] - 0.5 * (u[nk] * u[nk] + u[nk + 1] * u[nk + 1] + u[nk + 2] * u[nk + 2]) / rho;
}

int64_t pp_limit(const Problem& P, double* U, double eps) {
    const int V = P.V, nk = P.ph.nk;
    int64_t limited = 0;
    for (const Elem& E : P.el) {
        if (E.fv) continue;
        const Basis1D& B = P.ops.B(E.N);
        const int n = E.n, n3 = n * n * n;
        double* u = U + E.off;
        auto node = [&](int v, int c) -> double& { return u[(size_t)v * n3 + c]; };
        double mean[MAXV];
        for (int v = 0; v < V; ++v) {
            double m = 0.0;
            for (int c = 0; c < n3; ++c) m += B.w[c % n] * B.w[(c / n) % n] * B.w[c / (n * n)] * node(v, c);
            mean[v] = m / 8.0;
        }
        // the check points: nodes, then the face points (linear in the nodes)
        auto points = [&](std::vector<std::array<double, MAXV>>& pts) {
            pts.clear();
            for (int c = 0; c < n3; ++c) {
                std::array<double, MAXV> q{};
                for (int v = 0; v < V; ++v) q[v] = node(v, c);
                pts.push_back(q);
            }
            for (int f = 0; f < 6; ++f) {
                const int d = f / 2;
                const vector<double>& l = (f % 2) ? B.lp : B.lm;
                for (int b = 0; b < n; ++b)
                    for (int a = 0; a < n; ++a) {
                        std::array<double, MAXV> q{};
                        for (int v = 0; v < V; ++v) {
                            double s = 0.0;
                            for (int m = 0; m < n; ++m) s += l[m] * node(v, node_index(n, d, m, a, b));
                            q[v] = s;
                        }
                        pts.push_back(q);
                    }
            }
        };
        std::vector<std::array<double, MAXV>> pts;
        bool active = false;
        points(pts);
        for (int k = 0; k < nk; ++k) {
            double mn = mean[k];
            for (auto& q : pts) mn = std::min(mn, q[k]);
            const double ek = std::min(eps, mean[k]);
            if (mn < ek) {
                const double th = (mean[k] - ek) / (mean[k] - mn);
                for (int c = 0; c < n3; ++c) node(k, c) = mean[k] + th * (node(k, c) - mean[k]);
                active = true;
            }
        }
        points(pts);
        const double ee = std::min(eps, internal_energy(nk, mean));
        double theta = 1.0;
        for (auto& q : pts) {
            if (internal_energy(nk, q.data()) >= ee) continue;
            double lo = 0.0, hi = 1.0;  // rho e(lo) >= ee > rho e(hi)
            for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
                const double t = 0.5 * (lo + hi);
                if (t <= lo || t >= hi) break;
                double x[MAXV];
                for (int v = 0; v < V; ++v) x[v] = mean[v] + t * (q[v] - mean[v]);
                (internal_energy(nk, x) >= ee ? lo : hi) = t;
            }
            theta = std::min(theta, lo);
        }
        if (theta < 1.0) {
            for (int v = 0; v < V; ++v)
                for (int c = 0; c < n3; ++c) node(v, c) = mean[v] + theta * (node(v, c) - mean[v]);
            active = true;
        }
        limited += active ? 1 : 0;
    }
    return limited;
}

// ------------------------------------------------------------------ indicator, Sec. 3.4
// Reading: orthonormal Legendre modes; fit over m = 0..N; I = min over the three
// directions of |sigma|; FV elements are mapped to their DG degree by V^{FV->DG}
// first.  The energy fractions w_m are floored at W_FLOOR = 1e-24 before the
// logarithm: modal coefficients of FP64 nodal data carry round-off of about
// 1e-15 of the largest one, i.e. energy fractions near 1e-30, so every fraction
// below the floor is round-off and the fit of a field resolved to round-off
// does not depend on it.
constexpr double W_FLOOR = 1e-24;
double modal_indicator(const vector<double>& q, int N, const vector<double>& Vinv) {
    const int n = N + 1;
    vector<double> qm = map_volume(q.data(), 1, n, n, Vinv);  // Legendre coefficients
    double total = 0.0;
    for (int i = 0; i < n * n * n; ++i) total += qm[i] * qm[i];
    double I = INFINITY;
    for (int d = 0; d < 3; ++d) {
        vector<double> y(n);
        for (int m = 0; m < n; ++m) {
            double E = 0.0;
            for (int b = 0; b < n; ++b)
                for (int a = 0; a < n; ++a) {
                    double c = qm[node_index(n, d, m, a, b)];
                    E += c * c;
                }
            double w = total > 0.0 ? E / total : 0.0;
            y[m] = std::log(std::max(w, W_FLOOR));
        }
        // least-squares fit of log w_m = log c - sigma m  (Eq. 34)
        double mbar = 0.0, ybar = 0.0;
        for (int m = 0; m < n; ++m) { mbar += m; ybar += y[m]; }
        mbar /= n; ybar /= n;
        double sxy = 0.0, sxx = 0.0;
        for (int m = 0; m < n; ++m) { sxy += (m - mbar) * (y[m] - ybar); sxx += (m - mbar) * (m - mbar); }
        double sigma = -sxy / sxx;
        I = std::min(I, std::fabs(sigma));
    }
    return I;
}

void indicator(const Problem& P, const double* U, double* Ip, double* Ih) {
    const int nel = (int)P.el.size(), nk = P.ph.nk;
#pragma omp parallel for schedule(dynamic, 16)
    for (int e = 0; e < nel; ++e) {
        const Elem& E = P.el[e];
        const int n = E.N + 1, n3 = n * n * n;
        vector<double> u;
        if (E.fv) {
            u = map_volume(U + E.off, P.V, E.n, n, P.ops.f2d.at({E.N, E.n}));
        } else {
            u.assign(U + E.off, U + E.off + (int64_t)P.V * n3);
        }
        vector<double> rho(n3), pr(n3), Y[MAXSP];
        for (int k = 0; k < nk; ++k) Y[k].resize(n3);
        for (int c = 0; c < n3; ++c) {
            double uc[MAXV];
            for (int v = 0; v < P.V; ++v) uc[v] = u[(size_t)v * n3 + c];
            Prim<double> s;
            cons_to_prim(P.ph, uc, s);
            rho[c] = s.rho;
            pr[c] = s.p;
            for (int k = 0; k < nk; ++k) Y[k][c] = s.Y[k];
        }
        const vector<double>& Vinv = P.ops.vleg_inv.at(E.N);
        if (P.indicator_vars == 1) {  // the TGV of Sec. 4.3: p-refinement on p, FV on rho
            Ip[e] = modal_indicator(pr, E.N, Vinv);
            Ih[e] = modal_indicator(rho, E.N, Vinv);
            continue;
        }
        Ip[e] = modal_indicator(rho, E.N, Vinv);
        double ih = modal_indicator(pr, E.N, Vinv);
        for (int k = 0; k + 1 < nk; ++k) ih = std::min(ih, modal_indicator(Y[k], E.N, Vinv));
        Ih[e] = ih;
    }
}

// U_bar_j = sum_i R_bar_i (R'(U) e_j)_i for every j: the adjoint by columns of
// the tangent, the problem set up once.  D carries the tangent, A the sum.
template <class D, class A>
static void adjoint_columns_t(const Problem& P, const double* U, const double* Rbar, double* Ubar) {
#pragma omp parallel
    {
        vector<D> u(P.size), r(P.size);
#pragma omp for schedule(dynamic, 1)
        for (int64_t j = 0; j < P.size; ++j) {
            for (int64_t i = 0; i < P.size; ++i) u[i] = D(U[i], i == j ? 1.0 : 0.0);
            eval_rhs_t<D>(P, u.data(), r.data(), false);
            A s = 0;
            for (int64_t i = 0; i < P.size; ++i) s += (A)Rbar[i] * r[i].d;
            Ubar[j] = (double)s;
        }
    }
}

}  // namespace

// ==================================================================== C ABI
extern "C" {

int64_t oracle_state_size(const oracle_problem* p) {
    try { return make_problem(p, false).size; } catch (...) { return -1; }
}

int oracle_elem_offsets(const oracle_problem* p, int64_t* off) {
    try {
        Problem P = make_problem(p, false);
        for (size_t e = 0; e < P.el.size(); ++e) off[e] = P.el[e].off;
        return 0;
    } catch (...) { return -1; }
}

int oracle_eval_rhs(const oracle_problem* p, const double* U, double* R) {
    try {
        Problem P = make_problem(p);
        eval_rhs_t<double>(P, U, R);
        return 0;
    } catch (...) { return -1; }
}

int oracle_eval_rhs_extended(const oracle_problem* p, const double* U, double* R) {
    try {
        Problem P = make_problem(p);
        vector<long double> u(U, U + P.size), r(P.size);
        eval_rhs_t<long double>(P, u.data(), r.data());
        for (int64_t i = 0; i < P.size; ++i) R[i] = (double)r[i];
        return 0;
    } catch (...) { return -1; }
}

int oracle_eval_rhs_jvp(const oracle_problem* p, const double* U, const double* dU, double* R, double* dR) {
    try {
        Problem P = make_problem(p);
        vector<Dual> u(P.size), r(P.size);
        for (int64_t i = 0; i < P.size; ++i) u[i] = Dual(U[i], dU[i]);
        eval_rhs_t<Dual>(P, u.data(), r.data());
        for (int64_t i = 0; i < P.size; ++i) { R[i] = r[i].v; dR[i] = r[i].d; }
        return 0;
    } catch (...) { return -1; }
}

int oracle_eval_rhs_jvp_extended(const oracle_problem* p, const double* U, const double* dU, double* R,
                                 double* dR) {
    try {
        Problem P = make_problem(p);
        vector<DualL> u(P.size), r(P.size);
        for (int64_t i = 0; i < P.size; ++i) u[i] = DualL(U[i], dU[i]);
        eval_rhs_t<DualL>(P, u.data(), r.data());
        for (int64_t i = 0; i < P.size; ++i) { R[i] = (double)r[i].v; dR[i] = (double)r[i].d; }
        return 0;
    } catch (...) { return -1; }
}

int oracle_adjoint_columns(const oracle_problem* p, const double* U, const double* Rbar, int extended,
                           double* Ubar) {
    try {
        Problem P = make_problem(p);
        if (extended) adjoint_columns_t<DualL, long double>(P, U, Rbar, Ubar);
        else adjoint_columns_t<Dual, double>(P, U, Rbar, Ubar);
        return 0;
    } catch (...) { return -1; }
}

int oracle_count_flops(const oracle_problem* p, const double* U, double* out) {
    try {
        Problem P = make_problem(p);
        vector<Counted> u(P.size), r(P.size);
        for (int64_t i = 0; i < P.size; ++i) u[i] = Counted(U[i]);
        flop_counter() = FlopCounter();
        eval_rhs_t<Counted>(P, u.data(), r.data(), false);
        out[0] = flop_counter().add;
        out[1] = flop_counter().mul;
        out[2] = flop_counter().div;
        out[3] = flop_counter().sqrt;
        out[4] = 0.0;
        // per step of the right-hand side: out[8 + 4*step + {add, mul, div, sqrt}], steps 1..6
        for (int ph = 0; ph < 8; ++ph)
            for (int k = 0; k < 4; ++k) out[8 + 4 * ph + k] = flop_counter().by_phase[ph][k];
        return 0;
    } catch (...) { return -1; }
}

int oracle_dt(const oracle_problem* p, const double* U, double cfl_c, double cfl_v, double* out3) {
    try {
        Problem P = make_problem(p, false);
        time_step(P, U, cfl_c, cfl_v, out3);
        return 0;
    } catch (...) { return -1; }
}

int oracle_rk3(const oracle_problem* p, double* U, int n_steps, double dt_fixed, double cfl_c,
               double cfl_v, double* dts) {
    try {
        Problem P = make_problem(p);
        for (int it = 0; it < n_steps; ++it) {
            double dt = dt_fixed;
            if (!(dt > 0.0)) {
                double o[3];
                time_step(P, U, cfl_c, cfl_v, o);
                dt = o[0];
            }
            if (dts) dts[it] = dt;
            ssp_rk3_step(P.size, U, dt, [&](const double* x, double* r) { eval_rhs_t<double>(P, x, r); },
                         [&](double* x) { if (P.pp) pp_limit(P, x, P.pp_eps); });
        }
        return 0;
    } catch (...) { return -1; }
}

int oracle_lsrk4(const oracle_problem* p, double* U, int n_steps, double dt_fixed, double cfl_c, double cfl_v,
                 double* dts) {
    try {
        Problem P = make_problem(p);
        for (int it = 0; it < n_steps; ++it) {
            double dt = dt_fixed;
            if (!(dt > 0.0)) {
                double o[3];
                time_step(P, U, cfl_c, cfl_v, o);
                dt = o[0];
            }
            if (dts) dts[it] = dt;
            lsrk4_step(P.size, U, dt, [&](const double* x, double* r) { eval_rhs_t<double>(P, x, r); },
                       [&](double* x) { if (P.pp) pp_limit(P, x, P.pp_eps); });
        }
        return 0;
    } catch (...) { return -1; }
}

double oracle_lsrk4_scalar(int kind, double lambda, double dt, double u0) {
    double u = u0;
    if (kind == 0)
        lsrk4_step(1, &u, dt, [&](const double* x, double* r) { r[0] = lambda * x[0]; });
    else
        lsrk4_step(1, &u, dt, [&](const double* x, double* r) { r[0] = -x[0] * x[0]; });
    return u;
}

int oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int64_t oracle_pp_limit(const oracle_problem* p, double* U, double eps) {
    try {
        Problem P = make_problem(p);
        return pp_limit(P, U, eps);
    } catch (...) { return -1; }
}

double oracle_rk3_scalar_linear(double lambda, double dt, double u0) {
    double u = u0;
    ssp_rk3_step(1, &u, dt, [&](const double* x, double* r) { r[0] = lambda * x[0]; });
    return u;
}

int oracle_indicator(const oracle_problem* p, const double* U, double* Ip, double* Ih) {
    try {
        Problem P = make_problem(p);
        indicator(P, U, Ip, Ih);
        return 0;
    } catch (...) { return -1; }
}

// Reading of the threshold rule (values are configuration): DG -> FV when
// I_h < T_fv_on; FV -> DG when I_h > T_fv_off; a DG element that stays DG
// moves to N+1 when I_p < T_ref and to N-1 when I_p > T_crs, within
// [N_min, N_max], one level per call.
int oracle_adapt_decide(const oracle_problem* p, const double* Ip, const double* Ih, const double* thr,
                        int N_min, int N_max, int8_t* N_new, uint8_t* fv_new) {
    try {
        Problem P = make_problem(p, false);
        for (size_t e = 0; e < P.el.size(); ++e) {
            const Elem& E = P.el[e];
            int N = E.N;
            bool fv = E.fv;
            if (fv) {
                if (Ih[e] > thr[1]) fv = false;
            } else if (Ih[e] < thr[0]) {
                fv = true;
            } else if (Ip[e] < thr[2] && N < N_max) {
                N = N + 1;
            } else if (Ip[e] > thr[3] && N > N_min) {
                N = N - 1;
            }
            N_new[e] = (int8_t)N;
            fv_new[e] = fv ? 1 : 0;
        }
        return 0;
    } catch (...) { return -1; }
}

int oracle_remap(const oracle_problem* p_old, const int8_t* N_new, const uint8_t* fv_new,
                 const double* U_old, double* U_new) {
    try {
        Problem Po = make_problem(p_old, false);
        oracle_problem pn = *p_old;
        pn.N = N_new;
        pn.fv = fv_new;
        Problem Pn = make_problem(&pn, false);
        const int V = Po.V;
        for (size_t e = 0; e < Po.el.size(); ++e) {
            const Elem &A = Po.el[e], &B = Pn.el[e];
            const double* src = U_old + A.off;
            double* dst = U_new + B.off;
            vector<double> out;
            if (A.fv == B.fv && A.n == B.n) {
                out.assign(src, src + (int64_t)V * A.n * A.n * A.n);
            } else if (A.fv && B.fv) {
                out = map_volume(src, V, A.n, B.n, fv_overlap(A.n, B.n));  // sub-cell overlaps
            } else if (!A.fv && !B.fv) {
                out = map_volume(src, V, A.n, B.n, vmap(A.N, B.N, Po.nodes));      // V^{N->N~}
            } else if (!A.fv && B.fv) {
                out = map_volume(src, V, A.n, B.n, dg2fv(A.N, B.n, Po.nodes));  // V^{DG->FV}
            } else {
                out = map_volume(src, V, A.n, B.n, fv2dg(B.N, A.n, Po.nodes));  // V^{FV->DG}
            }
            std::copy(out.begin(), out.end(), dst);
        }
        return 0;
    } catch (...) { return -1; }
}

int oracle_basis(int N, double* x, double* w, double* D, double* Dhat, double* l_minus, double* l_plus,
                 int nodes) {
    try {
        Basis1D b = make_basis(N, nodes);
        std::copy(b.x.begin(), b.x.end(), x);
        std::copy(b.w.begin(), b.w.end(), w);
        std::copy(b.D.begin(), b.D.end(), D);
        std::copy(b.Dhat.begin(), b.Dhat.end(), Dhat);
        std::copy(b.lm.begin(), b.lm.end(), l_minus);
        std::copy(b.lp.begin(), b.lp.end(), l_plus);
        return 0;
    } catch (...) { return -1; }
}

int oracle_vmap(int N_from, int N_to, double* M, int nodes) {
    try { auto m = vmap(N_from, N_to, nodes); std::copy(m.begin(), m.end(), M); return 0; } catch (...) { return -1; }
}
int oracle_dg2fv(int N, int n_fv, double* M, int nodes) {
    try { auto m = dg2fv(N, n_fv, nodes); std::copy(m.begin(), m.end(), M); return 0; } catch (...) { return -1; }
}
int oracle_fv_overlap(int n_from, int n_to, double* M) {
    try { auto m = fv_overlap(n_from, n_to); std::copy(m.begin(), m.end(), M); return 0; } catch (...) { return -1; }
}
int oracle_fv2dg(int N, int n_fv, double* M, int nodes) {
    try {
        auto m = n_fv >= N + 1 ? fv2dg(N, n_fv, nodes) : fv2dg_l2(N, n_fv, nodes);
        std::copy(m.begin(), m.end(), M);
        return 0;
    } catch (...) { return -1; }
}
int oracle_mortar(int N, int s, int proj, int fv, double* M, int nodes) {
    try {
        auto m = fv ? (proj ? mortar_proj_fv(N, s) : mortar_interp_fv(N, s))
                    : (proj ? mortar_proj(N, s, nodes) : mortar_interp(N, s, nodes));
        std::copy(m.begin(), m.end(), M);
        return 0;
    } catch (...) { return -1; }
}
int oracle_leg_vandermonde(int N, double* V, int nodes) {
    try { auto m = leg_vandermonde(N, nodes); std::copy(m.begin(), m.end(), V); return 0; } catch (...) { return -1; }
}

static Phys phys_only(const oracle_problem* p) {
    Phys ph;
    ph.nk = p->n_species;
    for (int k = 0; k < ph.nk; ++k) {
        ph.gamma[k] = p->gamma[k];
        ph.R[k] = p->Rgas[k];
        ph.cv[k] = p->Rgas[k] / (p->gamma[k] - 1.0);
        ph.cp[k] = p->gamma[k] * ph.cv[k];
        ph.mu[k] = p->mu[k];
        ph.pr[k] = p->Pr[k];
        ph.D[k] = p->Dk[k];
    }
    ph.sutherland = p->sutherland != 0;
    ph.T_ref = p->T_ref;
    ph.S = p->S_sutherland;
    return ph;
}

int oracle_flux(const oracle_problem* p, const double* u, const double* g, int dir, double* Fc, double* Fv) {
    Phys ph = phys_only(p);
    Prim<double> s;
    cons_to_prim(ph, u, s);
    flux_conv(ph, u, s, dir, Fc);
    flux_visc(ph, u, g, s, dir, Fv);
    return 0;
}

int oracle_riemann(const oracle_problem* p, const double* uL, const double* uR, int dir, double* F) {
    Phys ph = phys_only(p);
    Prim<double> sL, sR;
    cons_to_prim(ph, uL, sL);
    cons_to_prim(ph, uR, sR);
    riemann(ph, p->riemann == 2 ? 1 : p->riemann, uL, sL, uR, sR, dir, F);
    return 0;
}

int oracle_primitives(const oracle_problem* p, const double* u, double* out) {
    Phys ph = phys_only(p);
    Prim<double> s;
    cons_to_prim(ph, u, s);
    out[0] = s.rho; out[1] = s.p; out[2] = s.temp; out[3] = s.c; out[4] = s.kappa;
    out[5] = s.cv; out[6] = s.cp; out[7] = s.mu; out[8] = s.lam;
    for (int k = 0; k < ph.nk; ++k) out[9 + k] = s.Y[k];
    return 0;
}

}  // extern "C"
