// Pointwise physics of the multi-component Navier-Stokes system, Sec. 2.
//
// TEST INFRASTRUCTURE ONLY (see dgfv_oracle.h).
//
// State u = (rho_1..rho_Nk, rho v_x, rho v_y, rho v_z, rho E); rho = sum rho_k
// (Eq. 3 species_closure with every partial density evolved).  The flux is
// written as u_t + div(F^c + F^v) = 0, so F^v is the negative of the
// right-hand sides of Eq. 1 (ns_equation):
//   F^v[rho_k] = J_k,  F^v[rho v] = -tau,  F^v[rho E] = -tau.v + q_h + q_d.
#ifndef DGFV_ORACLE_PHYSICS_HPP
#define DGFV_ORACLE_PHYSICS_HPP

#include "scalar_types.hpp"

namespace ora {

constexpr int MAXSP = 3;
constexpr int MAXV = MAXSP + 4;

struct Phys {
    int nk = 2;
    double gamma[MAXSP], R[MAXSP], cv[MAXSP], cp[MAXSP], mu[MAXSP], pr[MAXSP], D[MAXSP];
    bool sutherland = false;    // temperature-dependent viscosity (Sec. 4.3)
    double T_ref = 1.0, S = 0.0;  // Sutherland reference temperature and constant
    int V() const { return nk + 4; }
};

template <class T>
struct Prim {
    T rho, Y[MAXSP], v[3], E, eps, cv, cp, Rm, kappa, temp, p, c, mu, pr, lam;
};

// Mixture state from the conserved variables, Eqs. 6-12:
//   eps = E - |v|^2/2,  c_v,mix = sum Y c_v,  c_p,mix = sum Y c_p   (Eq. 10)
//   R_mix = c_p,mix - c_v,mix,  kappa = c_p,mix / c_v,mix            (Eq. 9)
//   T = eps / c_v,mix,  p = rho R_mix T                              (Eq. 8)
//   mu = sum Y mu_k,  Pr = sum Y Pr_k (Eq. 11),  lambda = mu c_p / Pr (Eq. 12)
//   c = sqrt(kappa p / rho)   (frozen-composition sound speed of the ideal-gas mixture)
// With Sutherland's law (the TGV of Sec. 4.3) the mixture viscosity is scaled by
//   (T/T_ref)^{3/2} (T_ref + S) / (T + S).
template <class T>
void cons_to_prim(const Phys& P, const T* u, Prim<T>& s) {
    const int nk = P.nk;
    s.rho = u[0];
    for (int k = 1; k < nk; ++k) s.rho = s.rho + u[k];
    for (int k = 0; k < nk; ++k) s.Y[k] = u[k] / s.rho;
    for (int i = 0; i < 3; ++i) s.v[i] = u[nk + i] / s.rho;
    s.E = u[nk + 3] / s.rho;
    s.eps = s.E - T(0.5) * (s.v[0] * s.v[0] + s.v[1] * s.v[1] + s.v[2] * s.v[2]);
    s.cv = s.Y[0] * T(P.cv[0]);
    s.cp = s.Y[0] * T(P.cp[0]);
    s.mu = s.Y[0] * T(P.mu[0]);
    s.pr = s.Y[0] * T(P.pr[0]);
    for (int k = 1; k < nk; ++k) {
        s.cv = s.cv + s.Y[k] * T(P.cv[k]);
        s.cp = s.cp + s.Y[k] * T(P.cp[k]);
        s.mu = s.mu + s.Y[k] * T(P.mu[k]);
        s.pr = s.pr + s.Y[k] * T(P.pr[k]);
    }
    s.Rm = s.cp - s.cv;
    s.kappa = s.cp / s.cv;
    s.temp = s.eps / s.cv;
    s.p = s.rho * s.Rm * s.temp;
    s.c = sqrt_(s.kappa * s.p / s.rho);
    if (P.sutherland) {
        const T r = s.temp / T(P.T_ref);
        s.mu = s.mu * (r * sqrt_(r)) * (T(P.T_ref + P.S) / (s.temp + T(P.S)));
    }
    s.lam = s.mu * s.cp / s.pr;
}

// Convective flux in direction d (Eq. 1, left-hand sides).
template <class T>
void flux_conv(const Phys& P, const T* u, const Prim<T>& s, int d, T* F) {
    const int nk = P.nk;
    for (int k = 0; k < nk; ++k) F[k] = u[k] * s.v[d];
    for (int i = 0; i < 3; ++i) F[nk + i] = u[nk + i] * s.v[d];
    F[nk + d] = F[nk + d] + s.p;
    F[nk + 3] = (u[nk + 3] + s.p) * s.v[d];
}

// Primitive gradients from the state's physical gradient g[dd*V + v] =
// d u_v / d x_dd (the BR1 lifting variable, Eq. 14b), by the chain rule:
//   grad Y_k = (grad rho_k - Y_k grad rho)/rho,  grad v = (grad(rho v) - v grad rho)/rho,
//   grad eps = (grad(rho E) - E grad rho)/rho - sum_i v_i grad v_i,
//   grad T = (grad eps - T grad c_v,mix)/c_v,mix,  grad c_v,mix = sum_k c_v,k grad Y_k.
template <class T>
struct PrimGrad {
    T Y[MAXSP][3], v[3][3], temp[3];
};

template <class T>
void prim_grad(const Phys& P, const T* g, const Prim<T>& s, PrimGrad<T>& G) {
    const int nk = P.nk, V = P.V();
    for (int dd = 0; dd < 3; ++dd) {
        const T* gd = g + dd * V;
        T gr = gd[0];
        for (int k = 1; k < nk; ++k) gr = gr + gd[k];
        for (int k = 0; k < nk; ++k) G.Y[k][dd] = (gd[k] - s.Y[k] * gr) / s.rho;
        for (int i = 0; i < 3; ++i) G.v[i][dd] = (gd[nk + i] - s.v[i] * gr) / s.rho;
        T geps = (gd[nk + 3] - s.E * gr) / s.rho;
        for (int i = 0; i < 3; ++i) geps = geps - s.v[i] * G.v[i][dd];
        T gcv = T(P.cv[0]) * G.Y[0][dd];
        for (int k = 1; k < nk; ++k) gcv = gcv + T(P.cv[k]) * G.Y[k][dd];
        G.temp[dd] = (geps - s.temp * gcv) / s.cv;
    }
}

// Viscous flux in direction d from the primitive gradients.
// Transport (Eqs. 4a-4c, 5):
//   tau = mu (grad v + grad v^T - 2/3 div v I),  q_h = -lambda grad T,
//   J_k = -rho D_k grad Y_k + rho Y_k sum_j D_j grad Y_j   (the sign and range of
//         the correction sum chosen so that sum_k J_k = 0, as Sec. 2 requires),
//   q_d = sum_k h_k J_k with h_k = c_p,k T.
template <class T>
void flux_visc(const Phys& P, const PrimGrad<T>& G, const Prim<T>& s, int d, T* F) {
    const int nk = P.nk;
    T divv = G.v[0][0] + G.v[1][1] + G.v[2][2];
    // row d of the stress tensor: tau_{d i}
    T tau[3];
    for (int i = 0; i < 3; ++i) {
        tau[i] = s.mu * (G.v[d][i] + G.v[i][d]);
        if (i == d) tau[i] = tau[i] - s.mu * T(2.0 / 3.0) * divv;
    }
    // species diffusion fluxes in direction d
    T corr = T(P.D[0]) * G.Y[0][d];
    for (int k = 1; k < nk; ++k) corr = corr + T(P.D[k]) * G.Y[k][d];
    T J[MAXSP] = {T(0.0), T(0.0), T(0.0)};
    for (int k = 0; k < nk; ++k)
        J[k] = -(s.rho * T(P.D[k]) * G.Y[k][d]) + s.rho * s.Y[k] * corr;
    T qh = -(s.lam * G.temp[d]);
    T qd = T(P.cp[0]) * s.temp * J[0];
    for (int k = 1; k < nk; ++k) qd = qd + T(P.cp[k]) * s.temp * J[k];
    for (int k = 0; k < nk; ++k) F[k] = J[k];
    for (int i = 0; i < 3; ++i) F[nk + i] = -tau[i];
    T tv = tau[0] * s.v[0] + tau[1] * s.v[1] + tau[2] * s.v[2];
    F[nk + 3] = -tv + qh + qd;
}

// Viscous flux in direction d from the state's physical gradient g.
template <class T>
void flux_visc(const Phys& P, const T* u, const T* g, const Prim<T>& s, int d, T* F) {
    (void)u;
    PrimGrad<T> G;
    prim_grad(P, g, s, G);
    flux_visc(P, G, s, d, F);
}

// Local Lax-Friedrichs (Rusanov) flux in direction d (used in Sec. 5 at FV
// and mixed faces):  F* = (F(uL) + F(uR))/2 - s_max (uR - uL)/2,
// s_max = max(|v_d,L| + c_L, |v_d,R| + c_R).
template <class T>
void riemann_llf(const Phys& P, const T* uL, const Prim<T>& sL, const T* uR, const Prim<T>& sR,
                 int d, T* F) {
    const int V = P.V();
    T FL[MAXV], FR[MAXV];
    flux_conv(P, uL, sL, d, FL);
    flux_conv(P, uR, sR, d, FR);
    T aL = abs_(sL.v[d]) + sL.c, aR = abs_(sR.v[d]) + sR.c;
    T smax = aL > aR ? aL : aR;
    for (int v = 0; v < V; ++v) F[v] = T(0.5) * (FL[v] + FR[v]) - T(0.5) * smax * (uR[v] - uL[v]);
}

// Roe flux with the Harten-Hyman entropy fix (Sec. 3.1.1, the default
// convective interface flux), written for the ideal-gas mixture.  The paper
// does not state the mixture average.  This oracle takes the one that makes the
// linearisation exact (Roe's property U: A~ (u_R - u_L) = F(u_R) - F(u_L)).
// With p = sum_k rho_k R_k T and rho e = sum_k rho_k c_v,k T, the jump rule
// d(ab) = a_bar db + b_bar da (arithmetic means) gives exactly
//   dp = (kappa~ - 1) [d(rho E) - v~.d(rho v) + |v~|^2/2 d rho] + sum_k psi_k d rho_k,
//   kappa~ - 1 = sum_k R_k rho_k,bar / sum_k c_v,k rho_k,bar,
//   psi_k = T_bar (c_p,k - kappa~ c_v,k),
// where rho_k,bar and T_bar are the arithmetic means of the two sides and
// v~, H~ (H = E + p/rho), Y~ the sqrt(rho)-weighted averages, rho~ = sqrt(rho_L rho_R).
// The sound speed of that linearisation is
//   c~^2 = sum_k Y~_k psi_k + (kappa~ - 1)(H~ - |v~|^2/2)
// (for one species, or species of equal gamma, every psi_k is 0: the textbook
// Roe average).  The jump is decomposed on the eigenvectors of A~:
//   acoustic  v_n -+ c:  r = (Y~_k; v~ -+ c~ n; H~ -+ c~ v~_n),  a = (dp -+ rho~ c~ dv_n)/(2 c~^2)
//   contact, species k:  r = (e_k; v~; |v~|^2/2 - psi_k/(kappa~ - 1)),  a = d(rho_k) - Y~_k dp/c~^2
//   shear, t != n:       r = (0; t; v~_t),                       a = rho~ dv_t
// (the contact vector carries no pressure change).  The Harten-Hyman fix
// replaces |lambda| by delta = max(0, lambda~ - lambda_L, lambda_R - lambda~)
// where |lambda| < delta, on the two acoustic waves.
template <class T>
void riemann_roe(const Phys& P, const T* uL, const Prim<T>& sL, const T* uR, const Prim<T>& sR,
                 int d, T* F) {
    const int nk = P.nk, V = P.V();
    T FL[MAXV], FR[MAXV];
    flux_conv(P, uL, sL, d, FL);
    flux_conv(P, uR, sR, d, FR);
    T rL = sqrt_(sL.rho), rR = sqrt_(sR.rho);
    T wsum = rL + rR;
    T vt[3], Yt[MAXSP];
    for (int i = 0; i < 3; ++i) vt[i] = (rL * sL.v[i] + rR * sR.v[i]) / wsum;
    for (int k = 0; k < nk; ++k) Yt[k] = (rL * sL.Y[k] + rR * sR.Y[k]) / wsum;
    T HL = (uL[nk + 3] + sL.p) / sL.rho, HR = (uR[nk + 3] + sR.p) / sR.rho;
    T Ht = (rL * HL + rR * HR) / wsum;
    // kappa~ from the arithmetic-mean partial densities; T_bar the mean temperature
    T rbar = T(0.5) * (uL[0] + uR[0]);
    T cvb = rbar * T(P.cv[0]), Rb = rbar * T(P.R[0]);
    for (int k = 1; k < nk; ++k) {
        rbar = T(0.5) * (uL[k] + uR[k]);
        cvb = cvb + rbar * T(P.cv[k]);
        Rb = Rb + rbar * T(P.R[k]);
    }
    T km1 = Rb / cvb;
    T kt = km1 + T(1.0);
    T Tbar = T(0.5) * (sL.temp + sR.temp);
    T psi[MAXSP];
    for (int k = 0; k < nk; ++k) psi[k] = Tbar * (T(P.cp[k]) - kt * T(P.cv[k]));
    T q2 = vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2];
    T c2 = km1 * (Ht - T(0.5) * q2);
    for (int k = 0; k < nk; ++k) c2 = c2 + Yt[k] * psi[k];
    T ct = sqrt_(c2);
    T rt = rL * rR;
    T vn = vt[d];
    T dp = sR.p - sL.p;
    T dv[3];
    for (int i = 0; i < 3; ++i) dv[i] = sR.v[i] - sL.v[i];
    // acoustic wave strengths and Harten-Hyman-fixed speeds
    T am = (dp - rt * ct * dv[d]) / (T(2.0) * c2);
    T ap = (dp + rt * ct * dv[d]) / (T(2.0) * c2);
    auto hh = [](T lt, T lL, T lR) {
        T delta = T(0.0);
        T a1 = lt - lL, a2 = lR - lt;
        if (a1 > delta) delta = a1;
        if (a2 > delta) delta = a2;
        T a = abs_(lt);
        return a < delta ? delta : a;
    };
    T lm = hh(vn - ct, sL.v[d] - sL.c, sR.v[d] - sR.c);
    T lp = hh(vn + ct, sL.v[d] + sL.c, sR.v[d] + sR.c);
    T l0 = abs_(vn);
    T Dis[MAXV];
    for (int v = 0; v < V; ++v) Dis[v] = T(0.0);
    // acoustic waves
    T sa = lm * am + lp * ap;
    for (int k = 0; k < nk; ++k) Dis[k] = Dis[k] + sa * Yt[k];
    for (int i = 0; i < 3; ++i) Dis[nk + i] = Dis[nk + i] + sa * vt[i];
    Dis[nk + d] = Dis[nk + d] + (lp * ap - lm * am) * ct;
    Dis[nk + 3] = Dis[nk + 3] + sa * Ht + (lp * ap - lm * am) * ct * vn;
    // contact waves, one per species
    for (int k = 0; k < nk; ++k) {
        T ak = (uR[k] - uL[k]) - Yt[k] * dp / c2;
        T epsk = -(psi[k] / km1);
        T s = l0 * ak;
        Dis[k] = Dis[k] + s;
        for (int i = 0; i < 3; ++i) Dis[nk + i] = Dis[nk + i] + s * vt[i];
        Dis[nk + 3] = Dis[nk + 3] + s * (T(0.5) * q2 + epsk);
    }
    // shear waves
    for (int i = 0; i < 3; ++i) {
        if (i == d) continue;
        T s = l0 * rt * dv[i];
        Dis[nk + i] = Dis[nk + i] + s;
        Dis[nk + 3] = Dis[nk + 3] + s * vt[i];
    }
    for (int v = 0; v < V; ++v) F[v] = T(0.5) * (FL[v] + FR[v]) - T(0.5) * Dis[v];
}

template <class T>
void riemann(const Phys& P, int kind, const T* uL, const Prim<T>& sL, const T* uR,
             const Prim<T>& sR, int d, T* F) {
    if (kind == 1)
        riemann_roe(P, uL, sL, uR, sR, d, F);
    else
        riemann_llf(P, uL, sL, uR, sR, d, F);
}

// Reconstruction variables of the FV sub-cell scheme: w = (rho_1..rho_Nk, v, p).
template <class T>
void cons_to_recvars(const Phys& P, const T* u, T* w) {
    const int nk = P.nk;
    T rho = u[0];
    for (int k = 1; k < nk; ++k) rho = rho + u[k];
    T cv = T(0.0), cp = T(0.0);
    for (int k = 0; k < nk; ++k) {
        T Y = u[k] / rho;
        cv = cv + Y * T(P.cv[k]);
        cp = cp + Y * T(P.cp[k]);
    }
    for (int k = 0; k < nk; ++k) w[k] = u[k];
    for (int i = 0; i < 3; ++i) w[nk + i] = u[nk + i] / rho;
    T ke = T(0.5) * rho * (w[nk] * w[nk] + w[nk + 1] * w[nk + 1] + w[nk + 2] * w[nk + 2]);
    // p = (kappa - 1)(rho E - rho |v|^2 / 2), kappa = c_p,mix / c_v,mix   (Eqs. 8-10)
    w[nk + 3] = (cp / cv - T(1.0)) * (u[nk + 3] - ke);
}

template <class T>
void recvars_to_cons(const Phys& P, const T* w, T* u) {
    const int nk = P.nk;
    T rho = w[0];
    for (int k = 1; k < nk; ++k) rho = rho + w[k];
    T cv = T(0.0), cp = T(0.0);
    for (int k = 0; k < nk; ++k) {
        T Y = w[k] / rho;
        cv = cv + Y * T(P.cv[k]);
        cp = cp + Y * T(P.cp[k]);
    }
    T kappa = cp / cv;
    for (int k = 0; k < nk; ++k) u[k] = w[k];
    for (int i = 0; i < 3; ++i) u[nk + i] = rho * w[nk + i];
    T ke = T(0.5) * rho * (w[nk] * w[nk] + w[nk + 1] * w[nk + 1] + w[nk + 2] * w[nk + 2]);
    u[nk + 3] = w[nk + 3] / (kappa - T(1.0)) + ke;
}

}  // namespace ora

#endif
