// Pointwise physics of the multi-component Navier-Stokes system (Sec. 2) as
// device functions, templated on the number of species NK (V = NK + 4).
//
// State u = (rho_1..rho_NK, rho v, rho E); flux convention u_t + div(F^c + F^v) = 0:
//   F^c_d = (rho_k v_d, rho v v_d + p e_d, (rho E + p) v_d)                 (Eq. 1)
//   F^v_d = (J_k,d, -tau_{d.}, -tau_{d.}.v + q_h,d + q_d,d)                (Eqs. 1, 4, 5)
// Mixture (Eqs. 8-12): c_v = sum Y c_v,k, c_p = sum Y c_p,k, R_mix = c_p - c_v,
// kappa = c_p/c_v, T = eps/c_v, p = rho R_mix T, mu = sum Y mu_k,
// Pr = sum Y Pr_k, lambda = mu c_p/Pr; sound speed c = sqrt(kappa p/rho).
// Fickian fluxes with the mass-conserving correction
// J_k = -rho D_k grad Y_k + rho Y_k sum_j D_j grad Y_j (sum_k J_k = 0).
#pragma once

#include <cmath>
#include <cstdint>

// Pointwise functions compile for the device and, for host-side checks of the
// hand-written adjoints, for the host.
#if defined(__CUDACC__)
#define DGFV_HD __host__ __device__ __forceinline__
#else
#define DGFV_HD inline
using std::fabs;
using std::fma;
using std::fmax;
using std::sqrt;
#endif

namespace dgfv {

constexpr int MAXSP = 3;
constexpr int MAXV = MAXSP + 4;

struct DevPhys {
    int nk;
    int viscous;
    int riemann;  // 0 LLF, 1 Roe + Harten-Hyman, 2 Roe-HH between DG elements, LLF where FV data meet
    double cv[MAXSP], cp[MAXSP], mu[MAXSP], pr[MAXSP], D[MAXSP];
    double maxD;
    int sutherland;     // viscosity by Sutherland's law (Sec. 4.3)
    double T_ref, S;    // its reference temperature and constant
};

// Sutherland factor (T/T_ref)^{3/2} (T_ref + S)/(T + S) of the viscosity.
DGFV_HD double sutherland_factor(const DevPhys& P, double T) {
    const double r = T / P.T_ref;
    return r * sqrt(r) * ((P.T_ref + P.S) / (T + P.S));
}

template <int NK>
struct Prim {
    double rho, irho, Y[NK], v[3], E, eps, cv, icv, cp, kappa, T, p, c, mu, pr, ipr, lam;
};

// Mixture state of a conserved vector.  3 divisions and 1 square root; terms
// a caller does not use are removed by the compiler after inlining.
template <int NK>
DGFV_HD void prim(const DevPhys& P, const double* u, Prim<NK>& s) {
    double rho = u[0];
#pragma unroll
    for (int k = 1; k < NK; ++k) rho += u[k];
    s.rho = rho;
    s.irho = 1.0 / rho;
    double cv = 0.0, cp = 0.0, mu = 0.0, pr = 0.0;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        s.Y[k] = u[k] * s.irho;
        cv = fma(s.Y[k], P.cv[k], cv);
        cp = fma(s.Y[k], P.cp[k], cp);
        mu = fma(s.Y[k], P.mu[k], mu);
        pr = fma(s.Y[k], P.pr[k], pr);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) s.v[i] = u[NK + i] * s.irho;
    s.E = u[NK + 3] * s.irho;
    double eps = s.E - 0.5 * (s.v[0] * s.v[0] + s.v[1] * s.v[1] + s.v[2] * s.v[2]);
    s.eps = eps;
    s.cv = cv;
    s.cp = cp;
    s.pr = pr;
    s.icv = 1.0 / cv;
    s.kappa = cp * s.icv;
    s.T = eps * s.icv;
    s.p = rho * (cp - cv) * s.T;
    s.c = sqrt(s.kappa * s.p * s.irho);
    if (P.sutherland) mu *= sutherland_factor(P, s.T);
    s.mu = mu;
    s.ipr = 1.0 / pr;  // kept for the adjoint (its reverse of lambda needs 1/Pr)
    s.lam = mu * cp * s.ipr;
}

// Convective flux in direction d.
// x[d] of a 3-vector by selects: indexed with a direction known only at run
// time, an array (and the structure holding it) would be placed in local
// memory; with a compile-time d this is x[d].
DGFV_HD double pick3(const double* x, int d) { return d == 0 ? x[0] : (d == 1 ? x[1] : x[2]); }

template <int NK>
DGFV_HD void flux_conv(const double* u, const Prim<NK>& s, int d, double* F) {
    const double vd = pick3(s.v, d);
#pragma unroll
    for (int k = 0; k < NK; ++k) F[k] = u[k] * vd;
#pragma unroll
    for (int i = 0; i < 3; ++i) F[NK + i] = fma(u[NK + i], vd, i == d ? s.p : 0.0);
    F[NK + 3] = (u[NK + 3] + s.p) * vd;
}

// Primitive gradients from the conservative gradient g[dd*V + v] (chain rule
// of the BR1 lifting variable, Eq. 14b): grad Y_k, grad v, grad T.
template <int NK>
struct PrimGrad {
    double Y[NK][3], v[3][3], T[3];
};

template <int NK>
DGFV_HD void prim_grad(const DevPhys& P, const Prim<NK>& s, const double* g,
                                          PrimGrad<NK>& G) {
    constexpr int V = NK + 4;
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
        const double* gd = g + dd * V;
        double gr = gd[0];
#pragma unroll
        for (int k = 1; k < NK; ++k) gr += gd[k];
        double gcv = 0.0;
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            G.Y[k][dd] = (gd[k] - s.Y[k] * gr) * s.irho;
            gcv = fma(P.cv[k], G.Y[k][dd], gcv);
        }
        double geps = (gd[NK + 3] - s.E * gr) * s.irho;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            G.v[i][dd] = (gd[NK + i] - s.v[i] * gr) * s.irho;
            geps -= s.v[i] * G.v[i][dd];
        }
        G.T[dd] = (geps - s.T * gcv) * s.icv;
    }
}

// Viscous flux in direction d from the primitive gradients.
template <int NK>
DGFV_HD void flux_visc(const DevPhys& P, const Prim<NK>& s, const PrimGrad<NK>& G,
                                          int d, double* F) {
    const double divv = G.v[0][0] + G.v[1][1] + G.v[2][2];
    double tau[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) tau[i] = s.mu * (G.v[d][i] + G.v[i][d]);
    tau[d] -= s.mu * (2.0 / 3.0) * divv;
    double corr = 0.0;
#pragma unroll
    for (int k = 0; k < NK; ++k) corr = fma(P.D[k], G.Y[k][d], corr);
    double qd = 0.0;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const double J = s.rho * (s.Y[k] * corr - P.D[k] * G.Y[k][d]);
        F[k] = J;
        qd = fma(P.cp[k], J, qd);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) F[NK + i] = -tau[i];
    const double tv = tau[0] * s.v[0] + tau[1] * s.v[1] + tau[2] * s.v[2];
    F[NK + 3] = -tv - s.lam * G.T[d] + s.T * qd;
}

// Viscous flux in direction D (a compile-time constant) straight from the
// conservative gradient, computing only what that direction needs: gx(dd, v)
// returns d u_v / d x_dd.  Of direction D every variable's gradient is used
// (species and temperature gradients, the column dv_i/dx_D); of the other two
// directions A, B only the densities and the momenta along D and along A (B):
// tau_{D.} needs dv_D/dx_A, dv_D/dx_B and div v the diagonal.  The same
// formulas as prim_grad + flux_visc (Eqs. 4a-4c, 5), with about two thirds of
// their FP64 work when the direction is not known before the call.  Every
// primitive gradient of the chain rule carries the factor 1/rho; it is kept
// out of the gradients below (they are rho times the primitive gradients) and
// applied once each in the viscosity (mu/rho), in the temperature gradient and,
// as rho/rho = 1, not at all in the diffusion fluxes.
template <int NK, int D, class GX>
DGFV_HD void flux_visc_dir(const DevPhys& P, const Prim<NK>& s, GX gx, double* F) {
    constexpr int A = D == 0 ? 1 : 0, B = D == 2 ? 1 : 2;
    double grD = gx(D, 0), grA = gx(A, 0), grB = gx(B, 0);
#pragma unroll
    for (int k = 1; k < NK; ++k) {
        grD += gx(D, k);
        grA += gx(A, k);
        grB += gx(B, k);
    }
    double vD[3];  // rho dv_i/dx_D
#pragma unroll
    for (int i = 0; i < 3; ++i) vD[i] = fma(-s.v[i], grD, gx(D, NK + i));
    const double vDA = fma(-s.v[D], grA, gx(A, NK + D));  // rho dv_D/dx_A
    const double vDB = fma(-s.v[D], grB, gx(B, NK + D));  // rho dv_D/dx_B
    const double vAA = fma(-s.v[A], grA, gx(A, NK + A));
    const double vBB = fma(-s.v[B], grB, gx(B, NK + B));
    const double divv = vD[D] + vAA + vBB;
    const double mr = s.mu * s.irho;
    double tau[3];
    tau[D] = mr * fma(-2.0 / 3.0, divv, 2.0 * vD[D]);
    tau[A] = mr * (vDA + vD[A]);
    tau[B] = mr * (vDB + vD[B]);
    double GY[NK], corr = 0.0, gcv = 0.0;  // rho dY_k/dx_D and its sums
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        GY[k] = fma(-s.Y[k], grD, gx(D, k));
        corr = fma(P.D[k], GY[k], corr);
        gcv = fma(P.cv[k], GY[k], gcv);
    }
    double geps = fma(-s.E, grD, gx(D, NK + 3));  // rho d(eps)/dx_D, eps = E - |v|^2/2
#pragma unroll
    for (int i = 0; i < 3; ++i) geps = fma(-s.v[i], vD[i], geps);
    const double GT = fma(-s.T, gcv, geps) * (s.irho * s.icv);
    double qd = 0.0;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const double J = fma(s.Y[k], corr, -P.D[k] * GY[k]);  // rho (Y_k corr - D_k dY_k/dx_D)
        F[k] = J;
        qd = fma(P.cp[k], J, qd);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) F[NK + i] = -tau[i];
    const double tv = fma(tau[2], s.v[2], fma(tau[1], s.v[1], tau[0] * s.v[0]));
    F[NK + 3] = fma(s.T, qd, fma(-s.lam, GT, -tv));
}

// F += F^v_d: the viscous flux of flux_visc added into F with fused
// multiply-adds (the volume kernel's nodal flux F^c + F^v).
template <int NK>
DGFV_HD void flux_visc_add(const DevPhys& P, const Prim<NK>& s, const PrimGrad<NK>& G, int d, double* F) {
    const double divv = G.v[0][0] + G.v[1][1] + G.v[2][2];
    double tau[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) tau[i] = s.mu * (G.v[d][i] + G.v[i][d]);
    tau[d] -= s.mu * (2.0 / 3.0) * divv;
    double corr = 0.0;
#pragma unroll
    for (int k = 0; k < NK; ++k) corr = fma(P.D[k], G.Y[k][d], corr);
    double qd = 0.0;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const double J = s.rho * fma(s.Y[k], corr, -P.D[k] * G.Y[k][d]);
        F[k] += J;
        qd = fma(P.cp[k], J, qd);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) F[NK + i] -= tau[i];
    double e = fma(s.T, qd, F[NK + 3]);
    e = fma(-s.lam, G.T[d], e);
#pragma unroll
    for (int i = 0; i < 3; ++i) e = fma(-tau[i], s.v[i], e);
    F[NK + 3] = e;
}

// Local Lax-Friedrichs flux in +x_d: (F_L + F_R)/2 - s_max (u_R - u_L)/2.
template <int NK>
DGFV_HD void riemann_llf(const double* uL, const Prim<NK>& sL, const double* uR,
                                            const Prim<NK>& sR, int d, double* F) {
    constexpr int V = NK + 4;
    double FL[V], FR[V];
    flux_conv<NK>(uL, sL, d, FL);
    flux_conv<NK>(uR, sR, d, FR);
    const double aL = fabs(pick3(sL.v, d)) + sL.c, aR = fabs(pick3(sR.v, d)) + sR.c;
    const double smax = aL > aR ? aL : aR;
#pragma unroll
    for (int v = 0; v < V; ++v) F[v] = 0.5 * fma(-smax, uR[v] - uL[v], FL[v] + FR[v]);
}

// Roe flux with the Harten-Hyman entropy fix for the ideal-gas mixture, with
// the average that linearises the mixture pressure exactly (Roe's property U,
// A~ (u_R - u_L) = F(u_R) - F(u_L)): sqrt(rho)-weighted v~, H~, Y~;
// kappa~ - 1 = sum R_k rho_k,bar / sum c_v,k rho_k,bar and
// psi_k = T_bar (c_p,k - kappa~ c_v,k) from the arithmetic means of the partial
// densities and temperatures, so that dp = (kappa~ - 1)(d(rho E) - v~.d(rho v)
// + |v~|^2/2 d rho) + sum psi_k d rho_k holds exactly;
// c~^2 = sum Y~_k psi_k + (kappa~ - 1)(H~ - |v~|^2/2); waves v_n - c,
// v_n (contact per species with energy entry |v~|^2/2 - psi_k/(kappa~ - 1),
// shear), v_n + c; Harten-Hyman fix on the acoustic waves.
template <int NK>
DGFV_HD void riemann_roe(const DevPhys& P, const double* uL, const Prim<NK>& sL,
                                            const double* uR, const Prim<NK>& sR, int d, double* F) {
    constexpr int V = NK + 4;
    double FL[V], FR[V];
    flux_conv<NK>(uL, sL, d, FL);
    flux_conv<NK>(uR, sR, d, FR);
    const double rL = sqrt(sL.rho), rR = sqrt(sR.rho);
    const double iw = 1.0 / (rL + rR);
    const double wl = rL * iw, wr = rR * iw;
    double vt[3], Yt[NK];
#pragma unroll
    for (int i = 0; i < 3; ++i) vt[i] = wl * sL.v[i] + wr * sR.v[i];
#pragma unroll
    for (int k = 0; k < NK; ++k) Yt[k] = wl * sL.Y[k] + wr * sR.Y[k];
    const double HL = sL.E + sL.p * sL.irho, HR = sR.E + sR.p * sR.irho;
    const double Ht = wl * HL + wr * HR;
    // kappa~ - 1 from the arithmetic-mean partial densities (the factor 1/2 cancels)
    double cvb = 0.0, Rb = 0.0;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const double rs = uL[k] + uR[k];
        cvb = fma(rs, P.cv[k], cvb);
        Rb = fma(rs, P.cp[k] - P.cv[k], Rb);
    }
    const double km1 = Rb / cvb;
    const double kt = km1 + 1.0;
    const double Tbar = 0.5 * (sL.T + sR.T);
    double ypsi = 0.0;  // sum_k Y~_k (c_p,k - kappa~ c_v,k)
#pragma unroll
    for (int k = 0; k < NK; ++k) ypsi = fma(Yt[k], P.cp[k] - kt * P.cv[k], ypsi);
    const double q2 = vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2];
    const double c2 = km1 * (Ht - 0.5 * q2) + Tbar * ypsi;
    const double ct = sqrt(c2);
    const double ic2 = 1.0 / c2;
    const double rt = rL * rR;
    const double vn = pick3(vt, d);
    const double dp = sR.p - sL.p;
    double dv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) dv[i] = sR.v[i] - sL.v[i];
    const double dvn = pick3(dv, d);
    const double am = 0.5 * (dp - rt * ct * dvn) * ic2;
    const double ap = 0.5 * (dp + rt * ct * dvn) * ic2;
    auto hh = [](double lt, double lL, double lR) {
        double delta = 0.0;
        delta = fmax(delta, lt - lL);
        delta = fmax(delta, lR - lt);
        const double a = fabs(lt);
        return a < delta ? delta : a;
    };
    const double vLn = pick3(sL.v, d), vRn = pick3(sR.v, d);
    const double lm = hh(vn - ct, vLn - sL.c, vRn - sR.c);
    const double lp = hh(vn + ct, vLn + sL.c, vRn + sR.c);
    const double l0 = fabs(vn);
    const double sa = lm * am + lp * ap;
    const double sd = (lp * ap - lm * am) * ct;
    double Dis[V];
#pragma unroll
    for (int k = 0; k < NK; ++k) Dis[k] = sa * Yt[k];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        Dis[NK + i] = sa * vt[i];
        if (i == d) Dis[NK + i] += sd;
    }
    Dis[NK + 3] = sa * Ht + sd * vn;
    // contact waves
    const double ecoef = -Tbar / km1;
    double scon = 0.0, econ = 0.0;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const double ak = (uR[k] - uL[k]) - Yt[k] * dp * ic2;
        const double s = l0 * ak;
        Dis[k] += s;
        scon += s;
        econ += s * (0.5 * q2 + ecoef * (P.cp[k] - kt * P.cv[k]));
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) Dis[NK + i] += scon * vt[i];
    Dis[NK + 3] += econ;
    // shear waves
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (i == d) continue;
        const double s = l0 * rt * dv[i];
        Dis[NK + i] += s;
        Dis[NK + 3] += s * vt[i];
    }
#pragma unroll
    for (int v = 0; v < V; ++v) F[v] = 0.5 * ((FL[v] + FR[v]) - Dis[v]);
}

// Convective flux of a face: riemann 0 LLF, 1 Roe-HH, 2 Roe-HH between DG
// elements and LLF on every face that touches FV data (the jet set-up of
// Sec. 5.1).  fv_involved: an FV sub-cell face, or an element face with an FV side.
DGFV_HD bool use_roe(const DevPhys& P, bool fv_involved) {
    return P.riemann == 1 || (P.riemann == 2 && !fv_involved);
}

// Interface flux at one point in +x_d: F* = F^c*(uL,uR) + (F^v(uL,gL) + F^v(uR,gR))/2
// (Eqs. 20, 21).
template <int NK>
DGFV_HD void interface_flux(const DevPhys& P, const double* uL, const double* gL,
                                               const double* uR, const double* gR, int d, double* F,
                                               bool fv_involved) {
    constexpr int V = NK + 4;
    Prim<NK> sL, sR;
    prim<NK>(P, uL, sL);
    prim<NK>(P, uR, sR);
    if (use_roe(P, fv_involved))
        riemann_roe<NK>(P, uL, sL, uR, sR, d, F);
    else
        riemann_llf<NK>(uL, sL, uR, sR, d, F);
    if (P.viscous) {
        double FvL[V], FvR[V];
        PrimGrad<NK> G;
        prim_grad<NK>(P, sL, gL, G);
        flux_visc<NK>(P, sL, G, d, FvL);
        prim_grad<NK>(P, sR, gR, G);
        flux_visc<NK>(P, sR, G, d, FvR);
#pragma unroll
        for (int v = 0; v < V; ++v) F[v] += 0.5 * (FvL[v] + FvR[v]);
    }
}

// Split form (Sec. 3.5): per-node tuple of the two-point flux,
// t = (rho, v_1, v_2, v_3, p, H, Y_1..Y_NK), H = (rho E + p)/rho.
template <int NK>
DGFV_HD void kep_tuple(const Prim<NK>& s, double* t) {
    t[0] = s.rho;
#pragma unroll
    for (int i = 0; i < 3; ++i) t[1 + i] = s.v[i];
    t[4] = s.p;
    t[5] = s.E + s.p * s.irho;
#pragma unroll
    for (int k = 0; k < NK; ++k) t[6 + k] = s.Y[k];
}

// Kinetic-energy-preserving two-point flux of Pirozzoli in +x_d from two tuples:
// arithmetic means {.};  rho_k: {rho}{v_d}{Y_k},  rho v_j: {rho}{v_d}{v_j} + {p} delta_jd,
// rho E: {rho}{v_d}{H}.  Symmetric in its arguments, equal to F^c on equal states.
template <int NK>
DGFV_HD void kep_flux(const double* a, const double* b, int d, double* F) {
    const double mass = (0.5 * (a[0] + b[0])) * (0.5 * (a[1 + d] + b[1 + d]));
#pragma unroll
    for (int k = 0; k < NK; ++k) F[k] = mass * (0.5 * (a[6 + k] + b[6 + k]));
#pragma unroll
    for (int j = 0; j < 3; ++j) F[NK + j] = mass * (0.5 * (a[1 + j] + b[1 + j]));
    F[NK + d] += 0.5 * (a[4] + b[4]);
    F[NK + 3] = mass * (0.5 * (a[5] + b[5]));
}

// FV reconstruction variables w = (rho_1..rho_NK, v, p) and back.
template <int NK>
DGFV_HD void cons_to_w(const DevPhys& P, const double* u, double* w) {
    double rho = u[0];
#pragma unroll
    for (int k = 1; k < NK; ++k) rho += u[k];
    const double irho = 1.0 / rho;
    double cvr = 0.0, cpr = 0.0;  // rho c_v, rho c_p
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        w[k] = u[k];
        cvr = fma(u[k], P.cv[k], cvr);
        cpr = fma(u[k], P.cp[k], cpr);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) w[NK + i] = u[NK + i] * irho;
    const double ke = 0.5 * fma(u[NK + 2], w[NK + 2], fma(u[NK + 1], w[NK + 1], u[NK] * w[NK]));
    w[NK + 3] = ((cpr - cvr) / cvr) * (u[NK + 3] - ke);
}

template <int NK>
DGFV_HD void w_to_cons(const DevPhys& P, const double* w, double* u) {
    double rho = w[0];
#pragma unroll
    for (int k = 1; k < NK; ++k) rho += w[k];
    double cvr = 0.0, cpr = 0.0;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        u[k] = w[k];
        cvr = fma(w[k], P.cv[k], cvr);
        cpr = fma(w[k], P.cp[k], cpr);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) u[NK + i] = rho * w[NK + i];
    const double ke = 0.5 * rho * fma(w[NK + 2], w[NK + 2], fma(w[NK + 1], w[NK + 1], w[NK] * w[NK]));
    // rho E = p / (kappa - 1) + rho |v|^2 / 2,  1/(kappa - 1) = c_v / (c_p - c_v)
    u[NK + 3] = fma(w[NK + 3], cvr / (cpr - cvr), ke);
}

DGFV_HD double minmod(double a, double b) {
    if (a * b <= 0.0) return 0.0;
    return fabs(a) <= fabs(b) ? a : b;
}

#if defined(__CUDACC__)
// minmod on the bit patterns, with no FP64 instruction: 0 when the signs
// differ (a signed zero counts by its sign bit, and a zero argument gives 0
// either way), else the argument of smaller magnitude, a on ties (for finite
// doubles |a| <= |b| is the unsigned order of the bits without the sign).
__device__ __forceinline__ double minmod_bits(double a, double b) {
    const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    if ((ia ^ ib) < 0) return 0.0;
    return (unsigned long long)(ia & 0x7fffffffffffffffLL) <= (unsigned long long)(ib & 0x7fffffffffffffffLL) ? a
                                                                                                          : b;
}
#endif

// Conservative state u and mixture state s of a reconstructed FV face value
// w = (rho_1..rho_NK, v, p), the same quantities as w_to_cons followed by
// prim, with one division: with A = rho c_v, B = rho c_p, Rr = B - A = rho R_mix
// and Q = rho Pr_mix, the reciprocals of rho, A, Rr and Q all come from
// 1/(rho A Rr Q); then rho E = p A/Rr + rho |v|^2/2, T = p/Rr, kappa = B/A,
// lambda = mu B/Q.
template <int NK>
DGFV_HD void face_state(const DevPhys& P, const double* w, double* u, Prim<NK>& s) {
    double rho = w[0], A = w[0] * P.cv[0], Bc = w[0] * P.cp[0], Mu = w[0] * P.mu[0], Q = w[0] * P.pr[0];
#pragma unroll
    for (int k = 1; k < NK; ++k) {
        rho += w[k];
        A = fma(w[k], P.cv[k], A);
        Bc = fma(w[k], P.cp[k], Bc);
        Mu = fma(w[k], P.mu[k], Mu);
        Q = fma(w[k], P.pr[k], Q);
    }
    const double Rr = Bc - A;
    const double AR = A * Rr, rQ = rho * Q;
    const double inv = 1.0 / (AR * rQ);
    const double irho = AR * Q * inv;
    const double iAR = rQ * inv;  // 1/(A Rr)
    const double iA = iAR * Rr, iR = iAR * A;
    s.rho = rho;
    s.irho = irho;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        u[k] = w[k];
        s.Y[k] = w[k] * irho;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        s.v[i] = w[NK + i];
        u[NK + i] = rho * w[NK + i];
    }
    const double p = w[NK + 3];
    const double q2 = fma(w[NK], w[NK], fma(w[NK + 1], w[NK + 1], w[NK + 2] * w[NK + 2]));
    const double rE = fma(p * A, iR, 0.5 * rho * q2);
    u[NK + 3] = rE;
    s.E = rE * irho;
    s.cv = A * irho;
    s.icv = rho * iA;
    s.cp = Bc * irho;
    s.kappa = Bc * iA;
    s.T = p * iR;
    s.eps = s.cv * s.T;
    s.p = p;
    s.c = sqrt(s.kappa * p * irho);
    double mu = Mu * irho;
    if (P.sutherland) mu *= sutherland_factor(P, s.T);
    s.mu = mu;
    s.pr = Q * irho;
    const double iQ = AR * rho * inv;  // 1/Q
    s.ipr = rho * iQ;
    s.lam = mu * Bc * iQ;  // mu c_p / Pr = mu B / Q
}

}  // namespace dgfv
