// Reverse-mode (vector-Jacobian) versions of the pointwise physics in
// physics.cuh, written statement by statement from the forward functions:
// every forward assignment y = f(x) becomes x_bar += (df/dx)^T y_bar, in
// reverse order.  Branches (the larger wave speed of the local Lax-Friedrichs
// flux, the sign of |v_d|) follow the forward evaluation.  These serve the
// adjoint of R(U) on DG elements with the local Lax-Friedrichs or the Roe-HH
// flux, constant or Sutherland viscosity.
#pragma once

#include "physics.cuh"

namespace dgfv {

template <int NK>
struct PrimBar {
    double rho, irho, Y[NK], v[3], E, eps, cv, icv, cp, kappa, T, p, c, mu, pr, lam;
};

template <int NK>
DGFV_HD void zero(PrimBar<NK>& b) {
    b.rho = b.irho = b.E = b.eps = b.cv = b.icv = b.cp = b.kappa = b.T = b.p = b.c = b.mu = b.pr = b.lam = 0.0;
    for (int k = 0; k < NK; ++k) b.Y[k] = 0.0;
    for (int i = 0; i < 3; ++i) b.v[i] = 0.0;
}

// u_bar += (d prim / d u)^T s_bar
template <int NK>
DGFV_HD void prim_rev(const DevPhys& P, const double* u, const Prim<NK>& s, PrimBar<NK> b, double* ub) {
    // lam = mu cp / pr
    const double lb = b.lam * s.ipr;
    b.mu += lb * s.cp;
    b.cp += lb * s.mu;
    b.pr -= lb * s.lam;
    // Sutherland (Sec. 4.3): mu = mu_mix f(T), f = (T/T_ref)^{3/2} (T_ref + S)/(T + S),
    // f'/f = 3/(2T) - 1/(T + S); b.mu becomes the adjoint of mu_mix
    if (P.sutherland) {
        b.T += b.mu * s.mu * (1.5 / s.T - 1.0 / (s.T + P.S));
        b.mu *= sutherland_factor(P, s.T);
    }
    // c = sqrt(kappa p irho)
    if (s.c > 0.0) {
        const double qb = 0.5 * b.c / s.c;
        b.kappa += qb * s.p * s.irho;
        b.p += qb * s.kappa * s.irho;
        b.irho += qb * s.kappa * s.p;
    }
    // p = rho (cp - cv) T
    const double Rm = s.cp - s.cv;
    b.rho += b.p * Rm * s.T;
    b.cp += b.p * s.rho * s.T;
    b.cv -= b.p * s.rho * s.T;
    b.T += b.p * s.rho * Rm;
    // T = eps icv
    b.eps += b.T * s.icv;
    b.icv += b.T * s.eps;
    // kappa = cp icv
    b.cp += b.kappa * s.icv;
    b.icv += b.kappa * s.cp;
    // icv = 1/cv
    b.cv -= b.icv * s.icv * s.icv;
    // eps = E - |v|^2/2
    b.E += b.eps;
#pragma unroll
    for (int i = 0; i < 3; ++i) b.v[i] -= b.eps * s.v[i];
    // E = u_E irho;  v_i = u_{m_i} irho
    ub[NK + 3] += b.E * s.irho;
    b.irho += b.E * u[NK + 3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        ub[NK + i] += b.v[i] * s.irho;
        b.irho += b.v[i] * u[NK + i];
    }
    // mixture sums and Y_k = u_k irho
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const double Yb = b.Y[k] + b.cv * P.cv[k] + b.cp * P.cp[k] + b.mu * P.mu[k] + b.pr * P.pr[k];
        ub[k] += Yb * s.irho;
        b.irho += Yb * u[k];
    }
    // irho = 1/rho;  rho = sum u_k
    b.rho -= b.irho * s.irho * s.irho;
#pragma unroll
    for (int k = 0; k < NK; ++k) ub[k] += b.rho;
}

// reverse of flux_conv: u_bar, s_bar += (dF/d(u, s))^T F_bar
template <int NK>
DGFV_HD void flux_conv_rev(const double* u, const Prim<NK>& s, int d, const double* Fb, double* ub,
                           PrimBar<NK>& b) {
    const double vd = s.v[d];
    double vdb = 0.0;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        ub[k] += Fb[k] * vd;
        vdb += Fb[k] * u[k];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        ub[NK + i] += Fb[NK + i] * vd;
        vdb += Fb[NK + i] * u[NK + i];
    }
    b.p += Fb[NK + d];
    ub[NK + 3] += Fb[NK + 3] * vd;
    b.p += Fb[NK + 3] * vd;
    vdb += Fb[NK + 3] * (u[NK + 3] + s.p);
    b.v[d] += vdb;
}

template <int NK>
struct PrimGradBar {
    double Y[NK][3], v[3][3], T[3];
};

template <int NK>
DGFV_HD void zero(PrimGradBar<NK>& b) {
    for (int d = 0; d < 3; ++d) {
        for (int k = 0; k < NK; ++k) b.Y[k][d] = 0.0;
        for (int i = 0; i < 3; ++i) b.v[i][d] = 0.0;
        b.T[d] = 0.0;
    }
}

// reverse of flux_visc: (G, s)_bar += (dF^v_d/d(G, s))^T F_bar
template <int NK>
DGFV_HD void flux_visc_rev(const DevPhys& P, const Prim<NK>& s, const PrimGrad<NK>& G, int d, const double* Fb,
                           PrimGradBar<NK>& Gb, PrimBar<NK>& b) {
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
    for (int k = 0; k < NK; ++k) qd = fma(P.cp[k], s.rho * (s.Y[k] * corr - P.D[k] * G.Y[k][d]), qd);
    // F_E = -tau.v - lam GT_d + T qd
    const double FE = Fb[NK + 3];
    b.lam -= FE * G.T[d];
    Gb.T[d] -= FE * s.lam;
    b.T += FE * qd;
    const double qdb = FE * s.T;
    double taub[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        taub[i] = -FE * s.v[i] - Fb[NK + i];  // from -tau.v and F_{m_i} = -tau_i
        b.v[i] -= FE * tau[i];
    }
    // J_k (= F_k) with qd = sum cp_k J_k
    double corrb = 0.0;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const double Jb = Fb[k] + qdb * P.cp[k];
        b.rho += Jb * (s.Y[k] * corr - P.D[k] * G.Y[k][d]);
        b.Y[k] += Jb * s.rho * corr;
        corrb += Jb * s.rho * s.Y[k];
        Gb.Y[k][d] -= Jb * s.rho * P.D[k];
    }
#pragma unroll
    for (int k = 0; k < NK; ++k) Gb.Y[k][d] += corrb * P.D[k];
    // tau_i = mu (Gv[d][i] + Gv[i][d]) - delta_id mu 2/3 divv
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        b.mu += taub[i] * (G.v[d][i] + G.v[i][d]);
        Gb.v[d][i] += taub[i] * s.mu;
        Gb.v[i][d] += taub[i] * s.mu;
    }
    b.mu -= taub[d] * (2.0 / 3.0) * divv;
    const double divvb = -taub[d] * s.mu * (2.0 / 3.0);
#pragma unroll
    for (int i = 0; i < 3; ++i) Gb.v[i][i] += divvb;
}

// reverse of prim_grad: g_bar, s_bar += (dG/d(g, s))^T G_bar
template <int NK>
DGFV_HD void prim_grad_rev(const DevPhys& P, const Prim<NK>& s, const double* g, const PrimGrad<NK>& G,
                           const PrimGradBar<NK>& Gb, double* gb, PrimBar<NK>& b) {
    constexpr int V = NK + 4;
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
        const double* gd = g + dd * V;
        double* gbd = gb + dd * V;
        double gr = gd[0];
#pragma unroll
        for (int k = 1; k < NK; ++k) gr += gd[k];
        double gcv = 0.0;
#pragma unroll
        for (int k = 0; k < NK; ++k) gcv = fma(P.cv[k], G.Y[k][dd], gcv);
        double geps = (gd[NK + 3] - s.E * gr) * s.irho;
#pragma unroll
        for (int i = 0; i < 3; ++i) geps -= s.v[i] * G.v[i][dd];
        // GT = (geps - T gcv) icv
        const double GTb = Gb.T[dd];
        const double gepsb = GTb * s.icv;
        b.T -= GTb * gcv * s.icv;
        const double gcvb = -GTb * s.T * s.icv;
        b.icv += GTb * (geps - s.T * gcv);
        // geps = (g_E - E gr) irho - sum_i v_i Gv_i
        double grb = 0.0;
        gbd[NK + 3] += gepsb * s.irho;
        b.E -= gepsb * gr * s.irho;
        grb -= gepsb * s.E * s.irho;
        b.irho += gepsb * (gd[NK + 3] - s.E * gr);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            b.v[i] -= gepsb * G.v[i][dd];
            const double Gvb = Gb.v[i][dd] - gepsb * s.v[i];
            // Gv_i = (g_{m_i} - v_i gr) irho
            gbd[NK + i] += Gvb * s.irho;
            b.v[i] -= Gvb * gr * s.irho;
            grb -= Gvb * s.v[i] * s.irho;
            b.irho += Gvb * (gd[NK + i] - s.v[i] * gr);
        }
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            // gcv = sum cv_k GY_k;  GY_k = (g_k - Y_k gr) irho
            const double GYb = Gb.Y[k][dd] + gcvb * P.cv[k];
            gbd[k] += GYb * s.irho;
            b.Y[k] -= GYb * gr * s.irho;
            grb -= GYb * s.Y[k] * s.irho;
            b.irho += GYb * (gd[k] - s.Y[k] * gr);
        }
        // gr = sum_k g_k
#pragma unroll
        for (int k = 0; k < NK; ++k) gbd[k] += grb;
    }
}

// prim_grad_rev after the viscous flux reverse of a face in direction D (a
// compile-time constant): flux_visc_rev leaves nonzero adjoints only on
// direction D's entries, on dv_D/dx_dd and on the diagonal dv_dd/dx_dd, so for
// the two other directions dd only those two velocity entries are reversed
// (the products with the zero adjoints of the rest are not formed; the
// compiler may not drop a product with 0.0 by itself).
template <int NK, int D>
DGFV_HD void prim_grad_rev_dir(const DevPhys& P, const Prim<NK>& s, const double* g, const PrimGrad<NK>& G,
                               const PrimGradBar<NK>& Gb, double* gb, PrimBar<NK>& b) {
    constexpr int V = NK + 4;
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
        if (dd == D) continue;
        const double* gd = g + dd * V;
        double* gbd = gb + dd * V;
        double gr = gd[0];
#pragma unroll
        for (int k = 1; k < NK; ++k) gr += gd[k];
        double grb = 0.0;
        auto vrev = [&](int i) {
            // Gv_i = (g_{m_i} - v_i gr) irho
            const double Gvb = Gb.v[i][dd];
            gbd[NK + i] += Gvb * s.irho;
            b.v[i] -= Gvb * gr * s.irho;
            grb -= Gvb * s.v[i] * s.irho;
            b.irho += Gvb * (gd[NK + i] - s.v[i] * gr);
        };
        vrev(D);
        vrev(dd);
#pragma unroll
        for (int k = 0; k < NK; ++k) gbd[k] += grb;
    }
    // direction D itself: every entry, as prim_grad_rev
    PrimGradBar<NK> GbD;
    zero(GbD);
#pragma unroll
    for (int i = 0; i < 3; ++i) GbD.v[i][D] = Gb.v[i][D];
#pragma unroll
    for (int k = 0; k < NK; ++k) GbD.Y[k][D] = Gb.Y[k][D];
    GbD.T[D] = Gb.T[D];
    {
        const double* gd = g + D * V;
        double* gbd = gb + D * V;
        double gr = gd[0];
#pragma unroll
        for (int k = 1; k < NK; ++k) gr += gd[k];
        double gcv = 0.0;
#pragma unroll
        for (int k = 0; k < NK; ++k) gcv = fma(P.cv[k], G.Y[k][D], gcv);
        double geps = (gd[NK + 3] - s.E * gr) * s.irho;
#pragma unroll
        for (int i = 0; i < 3; ++i) geps -= s.v[i] * G.v[i][D];
        const double GTb = GbD.T[D];
        const double gepsb = GTb * s.icv;
        b.T -= GTb * gcv * s.icv;
        const double gcvb = -GTb * s.T * s.icv;
        b.icv += GTb * (geps - s.T * gcv);
        double grb = 0.0;
        gbd[NK + 3] += gepsb * s.irho;
        b.E -= gepsb * gr * s.irho;
        grb -= gepsb * s.E * s.irho;
        b.irho += gepsb * (gd[NK + 3] - s.E * gr);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            b.v[i] -= gepsb * G.v[i][D];
            const double Gvb = GbD.v[i][D] - gepsb * s.v[i];
            gbd[NK + i] += Gvb * s.irho;
            b.v[i] -= Gvb * gr * s.irho;
            grb -= Gvb * s.v[i] * s.irho;
            b.irho += Gvb * (gd[NK + i] - s.v[i] * gr);
        }
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const double GYb = GbD.Y[k][D] + gcvb * P.cv[k];
            gbd[k] += GYb * s.irho;
            b.Y[k] -= GYb * gr * s.irho;
            grb -= GYb * s.Y[k] * s.irho;
            b.irho += GYb * (gd[k] - s.Y[k] * gr);
        }
#pragma unroll
        for (int k = 0; k < NK; ++k) gbd[k] += grb;
    }
}

// The gradient reverse of a face in direction d: specialised when the caller
// knows d at compile time (DC = d), the general one otherwise (DC = -1).
template <int NK, int DC>
DGFV_HD void prim_grad_rev_face(const DevPhys& P, const Prim<NK>& s, const double* g, const PrimGrad<NK>& G,
                                const PrimGradBar<NK>& Gb, double* gb, PrimBar<NK>& b) {
    if constexpr (DC >= 0)
        prim_grad_rev_dir<NK, DC>(P, s, g, G, Gb, gb, b);
    else
        prim_grad_rev<NK>(P, s, g, G, Gb, gb, b);
}

// Adjoint of the nodal volume fluxes F_d = F^c_d(u) + F^v_d(u, g), d = 0..2:
// given F_bar[d*V + v], accumulate u_bar (V) and g_bar (3V).
template <int NK>
DGFV_HD void volume_point_rev(const DevPhys& P, const double* u, const double* g, const double* Fb, double* ub,
                              double* gb, bool conv = true) {
    Prim<NK> s;
    prim<NK>(P, u, s);
    PrimBar<NK> b;
    zero(b);
    PrimGrad<NK> G;
    PrimGradBar<NK> Gb;
    if (P.viscous) {
        prim_grad<NK>(P, s, g, G);
        zero(Gb);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (conv) flux_conv_rev<NK>(u, s, d, Fb + d * (NK + 4), ub, b);
        if (P.viscous) flux_visc_rev<NK>(P, s, G, d, Fb + d * (NK + 4), Gb, b);
    }
    if (P.viscous) prim_grad_rev<NK>(P, s, g, G, Gb, gb, b);
    prim_rev<NK>(P, u, s, b, ub);
}

// Reverse of cons_to_w (physics.cuh): u_bar += (dw/du)^T w_bar for the FV
// reconstruction variables w = (rho_k, v, p).
template <int NK>
DGFV_HD void cons_to_w_rev(const DevPhys& P, const double* u, const double* wb, double* ub) {
    double rho = u[0];
    for (int k = 1; k < NK; ++k) rho += u[k];
    const double irho = 1.0 / rho;
    double cvr = 0.0, cpr = 0.0;
    for (int k = 0; k < NK; ++k) {
        cvr = fma(u[k], P.cv[k], cvr);
        cpr = fma(u[k], P.cp[k], cpr);
    }
    double wv[3];
    for (int i = 0; i < 3; ++i) wv[i] = u[NK + i] * irho;
    const double ke = 0.5 * (u[NK] * wv[0] + u[NK + 1] * wv[1] + u[NK + 2] * wv[2]);
    const double icvr = 1.0 / cvr, q = (cpr - cvr) * icvr;  // one division for q and its derivatives
    // w_p = q (u_E - ke)
    const double wpb = wb[NK + 3];
    const double qb = wpb * (u[NK + 3] - ke);
    ub[NK + 3] += wpb * q;
    const double keb = -wpb * q;
    // ke = 1/2 sum_i u_mi wv_i;  wv_i = u_mi irho
    double irhob = 0.0;
    for (int i = 0; i < 3; ++i) {
        const double wvb = wb[NK + i] + 0.5 * keb * u[NK + i];
        ub[NK + i] += 0.5 * keb * wv[i] + wvb * irho;
        irhob += wvb * u[NK + i];
    }
    // q = cpr/cvr - 1;  sums;  irho = 1/rho;  rho = sum u_k;  w_k = u_k
    const double cprb = qb * icvr, cvrb = -qb * cpr * (icvr * icvr);
    const double rhob = -irhob * irho * irho;
    for (int k = 0; k < NK; ++k) ub[k] += wb[k] + cvrb * P.cv[k] + cprb * P.cp[k] + rhob;
}

// Reverse of w_to_cons: w_bar += (du/dw)^T u_bar.
template <int NK>
DGFV_HD void w_to_cons_rev(const DevPhys& P, const double* w, const double* ubar, double* wb) {
    double rho = w[0];
    for (int k = 1; k < NK; ++k) rho += w[k];
    double cvr = 0.0, cpr = 0.0;
    for (int k = 0; k < NK; ++k) {
        cvr = fma(w[k], P.cv[k], cvr);
        cpr = fma(w[k], P.cp[k], cpr);
    }
    const double Dn = cpr - cvr, iDn = 1.0 / Dn, r = cvr * iDn;  // one division for r and its derivatives
    // u_E = w_p r + ke;  ke = 1/2 rho |v|^2;  u_mi = rho v_i
    const double ueb = ubar[NK + 3];
    wb[NK + 3] += ueb * r;
    const double rb = ueb * w[NK + 3];
    double v2 = 0.0, rhob = 0.0;
    for (int i = 0; i < 3; ++i) {
        v2 += w[NK + i] * w[NK + i];
        wb[NK + i] += ueb * rho * w[NK + i] + ubar[NK + i] * rho;
        rhob += ubar[NK + i] * w[NK + i];
    }
    rhob += 0.5 * ueb * v2;
    // r = cvr / (cpr - cvr)
    const double rbD = rb * (iDn * iDn), cvrb = rbD * cpr, cprb = -rbD * cvr;
    for (int k = 0; k < NK; ++k) wb[k] += ubar[k] + cvrb * P.cv[k] + cprb * P.cp[k] + rhob;
}

// Reverse of kep_flux (physics.cuh): the flux is a function of the arithmetic
// means of the two tuples, so both tuples receive half of each mean's adjoint;
// tb += that half (call once per argument).
template <int NK>
DGFV_HD void kep_flux_rev(const double* a, const double* b, int d, const double* Fb, double* tb) {
    const double r = 0.5 * (a[0] + b[0]), vd = 0.5 * (a[1 + d] + b[1 + d]);
    const double mass = r * vd;
    double massb = 0.0;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        massb += Fb[k] * 0.5 * (a[6 + k] + b[6 + k]);
        tb[6 + k] += 0.5 * Fb[k] * mass;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        massb += Fb[NK + j] * 0.5 * (a[1 + j] + b[1 + j]);
        tb[1 + j] += 0.5 * Fb[NK + j] * mass;
    }
    tb[4] += 0.5 * Fb[NK + d];
    massb += Fb[NK + 3] * 0.5 * (a[5] + b[5]);
    tb[5] += 0.5 * Fb[NK + 3] * mass;
    tb[0] += 0.5 * massb * vd;
    tb[1 + d] += 0.5 * massb * r;
}

// Reverse of kep_tuple: t = (rho, v, p, H = E + p/rho, Y_k).
template <int NK>
DGFV_HD void kep_tuple_rev(const Prim<NK>& s, const double* tb, PrimBar<NK>& b) {
    b.rho += tb[0];
#pragma unroll
    for (int i = 0; i < 3; ++i) b.v[i] += tb[1 + i];
    b.p += tb[4] + tb[5] * s.irho;
    b.E += tb[5];
    b.irho += tb[5] * s.p;
#pragma unroll
    for (int k = 0; k < NK; ++k) b.Y[k] += tb[6 + k];
}

// Adjoint of the interface flux F* = LLF(uL, uR) + (F^v(uL,gL) + F^v(uR,gR))/2 in +x_d:
// given F_bar (V), accumulate uL_bar, gL_bar, uR_bar, gR_bar.
// Reverse of riemann_roe (physics.cuh), statement by statement backwards:
// u_bar, s_bar += (dF/d(u, s))^T F_bar for the Roe flux with the Harten-Hyman
// fix.  The branches of the fix (which of |lambda~| and delta is taken, and
// which term gives delta) and of |v_n| follow the forward evaluation.
template <int NK>
DGFV_HD void riemann_roe_rev(const DevPhys& P, const double* uL, const Prim<NK>& sL, const double* uR,
                             const Prim<NK>& sR, int d, const double* Fb, double* uLb, PrimBar<NK>& bL, double* uRb,
                             PrimBar<NK>& bR) {
    constexpr int V = NK + 4;
    // ---- forward, keeping the intermediates
    const double rL = sqrt(sL.rho), rR = sqrt(sR.rho);
    const double iw = 1.0 / (rL + rR);
    const double wl = rL * iw, wr = rR * iw;
    double vt[3], Yt[NK];
    for (int i = 0; i < 3; ++i) vt[i] = wl * sL.v[i] + wr * sR.v[i];
    for (int k = 0; k < NK; ++k) Yt[k] = wl * sL.Y[k] + wr * sR.Y[k];
    const double HL = sL.E + sL.p * sL.irho, HR = sR.E + sR.p * sR.irho;
    const double Ht = wl * HL + wr * HR;
    double cvb = 0.0, Rb = 0.0;
    for (int k = 0; k < NK; ++k) {
        const double rs = uL[k] + uR[k];
        cvb = fma(rs, P.cv[k], cvb);
        Rb = fma(rs, P.cp[k] - P.cv[k], Rb);
    }
    const double km1 = Rb / cvb;
    const double kt = km1 + 1.0;
    const double Tbar = 0.5 * (sL.T + sR.T);
    double ypsi = 0.0, ycv = 0.0;
    for (int k = 0; k < NK; ++k) {
        ypsi = fma(Yt[k], P.cp[k] - kt * P.cv[k], ypsi);
        ycv = fma(Yt[k], P.cv[k], ycv);
    }
    const double q2 = vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2];
    const double c2 = km1 * (Ht - 0.5 * q2) + Tbar * ypsi;
    const double ct = sqrt(c2);
    const double ic2 = 1.0 / c2;
    const double rt = rL * rR;
    const double vn = vt[d];
    const double dp = sR.p - sL.p;
    double dv[3];
    for (int i = 0; i < 3; ++i) dv[i] = sR.v[i] - sL.v[i];
    const double Xm = 0.5 * (dp - rt * ct * dv[d]), Xp = 0.5 * (dp + rt * ct * dv[d]);
    const double am = Xm * ic2, ap = Xp * ic2;
    // Harten-Hyman: value and the branch taken (0: |lt|, 1: lt - lL, 2: lR - lt)
    auto hh = [](double lt, double lL, double lR, int& br) {
        double delta = 0.0;
        int dbr = 0;
        if (lt - lL > delta) { delta = lt - lL; dbr = 1; }
        if (lR - lt > delta) { delta = lR - lt; dbr = 2; }
        const double a = fabs(lt);
        br = a < delta ? dbr : 0;
        return a < delta ? delta : a;
    };
    int bm, bp;
    const double lm = hh(vn - ct, sL.v[d] - sL.c, sR.v[d] - sR.c, bm);
    const double lp = hh(vn + ct, sL.v[d] + sL.c, sR.v[d] + sR.c, bp);
    const double l0 = fabs(vn);
    const double sa = lm * am + lp * ap;
    const double sd = (lp * ap - lm * am) * ct;
    const double ecoef = -Tbar / km1;
    double ak[NK], sk[NK], scon = 0.0;
    for (int k = 0; k < NK; ++k) {
        ak[k] = (uR[k] - uL[k]) - Yt[k] * dp * ic2;
        sk[k] = l0 * ak[k];
        scon += sk[k];
    }
    // ---- reverse.  F = (F_L + F_R)/2 - Dis/2
    double half[V], Db[V];
    for (int v = 0; v < V; ++v) {
        half[v] = 0.5 * Fb[v];
        Db[v] = -0.5 * Fb[v];
    }
    flux_conv_rev<NK>(uL, sL, d, half, uLb, bL);
    flux_conv_rev<NK>(uR, sR, d, half, uRb, bR);
    double vtb[3] = {0.0, 0.0, 0.0}, Ytb[NK], dvb[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < NK; ++k) Ytb[k] = 0.0;
    double l0b = 0.0, rtb = 0.0, q2b = 0.0, ktb = 0.0, ecoefb = 0.0, dpb = 0.0, ic2b = 0.0, sab = 0.0, sdb = 0.0;
    double Htb = 0.0, vnb = 0.0, lmb = 0.0, lpb = 0.0, amb = 0.0, apb = 0.0, ctb = 0.0, c2b = 0.0;
    double km1b = 0.0, Tbarb = 0.0;
    // shear waves: s = l0 rt dv_i; Dis[m_i] += s; Dis[E] += s vt_i
    for (int i = 0; i < 3; ++i) {
        if (i == d) continue;
        const double sh = l0 * rt * dv[i];
        const double shb = Db[NK + i] + Db[NK + 3] * vt[i];
        vtb[i] += Db[NK + 3] * sh;
        l0b += shb * rt * dv[i];
        rtb += shb * l0 * dv[i];
        dvb[i] += shb * l0 * rt;
    }
    // contact waves: Dis[m_i] += scon vt_i; Dis[E] += econ
    double sconb = 0.0;
    for (int i = 0; i < 3; ++i) {
        sconb += Db[NK + i] * vt[i];
        vtb[i] += Db[NK + i] * scon;
    }
    const double econb = Db[NK + 3];
    for (int k = 0; k < NK; ++k) {
        const double ck = P.cp[k] - kt * P.cv[k];
        const double skb = Db[k] + sconb + econb * (0.5 * q2 + ecoef * ck);
        q2b += econb * sk[k] * 0.5;
        ecoefb += econb * sk[k] * ck;
        ktb -= econb * sk[k] * ecoef * P.cv[k];
        l0b += skb * ak[k];
        const double akb = skb * l0;
        uRb[k] += akb;
        uLb[k] -= akb;
        Ytb[k] -= akb * dp * ic2;
        dpb -= akb * Yt[k] * ic2;
        ic2b -= akb * Yt[k] * dp;
    }
    // ecoef = -Tbar / km1
    Tbarb -= ecoefb / km1;
    km1b += ecoefb * Tbar / (km1 * km1);
    // main waves: Dis[k] = sa Yt_k; Dis[m_i] = sa vt_i (+ sd for i = d); Dis[E] = sa Ht + sd vn
    for (int k = 0; k < NK; ++k) {
        sab += Db[k] * Yt[k];
        Ytb[k] += Db[k] * sa;
    }
    for (int i = 0; i < 3; ++i) {
        sab += Db[NK + i] * vt[i];
        vtb[i] += Db[NK + i] * sa;
    }
    sdb += Db[NK + d];
    sab += Db[NK + 3] * Ht;
    Htb += Db[NK + 3] * sa;
    sdb += Db[NK + 3] * vn;
    vnb += Db[NK + 3] * sd;
    // sd = (lp ap - lm am) ct;  sa = lm am + lp ap
    lpb += sdb * ap * ct + sab * ap;
    apb += sdb * lp * ct + sab * lp;
    lmb += -sdb * am * ct + sab * am;
    amb += -sdb * lm * ct + sab * lm;
    ctb += sdb * (lp * ap - lm * am);
    // l0 = |vn|
    vnb += l0b * (vn > 0.0 ? 1.0 : (vn < 0.0 ? -1.0 : 0.0));
    // lp = hh(vn + ct, vL + cL, vR + cR);  lm = hh(vn - ct, vL - cL, vR - cR)
    {
        double ltb = 0.0, lLb = 0.0, lRb = 0.0;
        if (bp == 0) ltb = lpb * ((vn + ct) > 0.0 ? 1.0 : ((vn + ct) < 0.0 ? -1.0 : 0.0));
        else if (bp == 1) { ltb = lpb; lLb = -lpb; }
        else { lRb = lpb; ltb = -lpb; }
        vnb += ltb;
        ctb += ltb;
        bL.v[d] += lLb;
        bL.c += lLb;
        bR.v[d] += lRb;
        bR.c += lRb;
    }
    {
        double ltb = 0.0, lLb = 0.0, lRb = 0.0;
        if (bm == 0) ltb = lmb * ((vn - ct) > 0.0 ? 1.0 : ((vn - ct) < 0.0 ? -1.0 : 0.0));
        else if (bm == 1) { ltb = lmb; lLb = -lmb; }
        else { lRb = lmb; ltb = -lmb; }
        vnb += ltb;
        ctb -= ltb;
        bL.v[d] += lLb;
        bL.c -= lLb;
        bR.v[d] += lRb;
        bR.c -= lRb;
    }
    // am = Xm ic2, ap = Xp ic2;  Xm/p = (dp -/+ rt ct dv_d)/2
    ic2b += amb * Xm + apb * Xp;
    const double Xmb = amb * ic2, Xpb = apb * ic2;
    dpb += 0.5 * (Xmb + Xpb);
    const double tb = 0.5 * (Xpb - Xmb);  // adjoint of rt ct dv_d
    rtb += tb * ct * dv[d];
    ctb += tb * rt * dv[d];
    dvb[d] += tb * rt * ct;
    // dv = vR - vL;  dp = pR - pL;  vn = vt_d;  rt = rL rR
    for (int i = 0; i < 3; ++i) {
        bR.v[i] += dvb[i];
        bL.v[i] -= dvb[i];
    }
    bR.p += dpb;
    bL.p -= dpb;
    vtb[d] += vnb;
    double rLb = rtb * rR, rRb = rtb * rL;
    // ic2 = 1/c2;  ct = sqrt(c2);  c2 = km1 (Ht - q2/2) + Tbar ypsi
    c2b -= ic2b * ic2 * ic2;
    c2b += ctb * 0.5 / ct;
    km1b += c2b * (Ht - 0.5 * q2);
    Htb += c2b * km1;
    q2b -= c2b * 0.5 * km1;
    Tbarb += c2b * ypsi;
    // ypsi = sum_k Yt_k (cp_k - kt cv_k)
    const double ypsib = c2b * Tbar;
    for (int k = 0; k < NK; ++k) Ytb[k] += ypsib * (P.cp[k] - kt * P.cv[k]);
    ktb -= ypsib * ycv;
    // kt = km1 + 1;  km1 = Rb / cvb;  Rb, cvb = sum_k (uL_k + uR_k) (R_k, cv_k)
    km1b += ktb;
    const double Rbb = km1b / cvb, cvbb = -km1b * km1 / cvb;
    for (int k = 0; k < NK; ++k) {
        const double rsb = Rbb * (P.cp[k] - P.cv[k]) + cvbb * P.cv[k];
        uLb[k] += rsb;
        uRb[k] += rsb;
    }
    // Tbar = (TL + TR)/2
    bL.T += 0.5 * Tbarb;
    bR.T += 0.5 * Tbarb;
    // q2 = |vt|^2;  Ht = wl HL + wr HR;  H = E + p irho
    for (int i = 0; i < 3; ++i) vtb[i] += q2b * 2.0 * vt[i];
    double wlb = Htb * HL, wrb = Htb * HR;
    const double HLb = Htb * wl, HRb = Htb * wr;
    bL.E += HLb;
    bL.p += HLb * sL.irho;
    bL.irho += HLb * sL.p;
    bR.E += HRb;
    bR.p += HRb * sR.irho;
    bR.irho += HRb * sR.p;
    // Yt = wl YL + wr YR;  vt = wl vL + wr vR
    for (int k = 0; k < NK; ++k) {
        wlb += Ytb[k] * sL.Y[k];
        wrb += Ytb[k] * sR.Y[k];
        bL.Y[k] += Ytb[k] * wl;
        bR.Y[k] += Ytb[k] * wr;
    }
    for (int i = 0; i < 3; ++i) {
        wlb += vtb[i] * sL.v[i];
        wrb += vtb[i] * sR.v[i];
        bL.v[i] += vtb[i] * wl;
        bR.v[i] += vtb[i] * wr;
    }
    // wl = rL iw, wr = rR iw, iw = 1/(rL + rR);  r = sqrt(rho)
    const double iwb = wlb * rL + wrb * rR;
    rLb += wlb * iw - iwb * iw * iw;
    rRb += wrb * iw - iwb * iw * iw;
    bL.rho += rLb * 0.5 / rL;
    bR.rho += rRb * 0.5 / rR;
}

// Reverse of the interface flux with the two viscous sides one after the
// other: getg(side, g) supplies a side's gradient (side 0 = L, 1 = R) just
// before its reverse and putgb(side, gb) receives its adjoint right after, so
// only one side's gradient and gradient adjoint are live at a time.
// The same with the two mixture states given (sL, sR the states of uL, uR,
// e.g. built by face_state from reconstructed variables).
template <int NK, int DC = -1, class GetG, class PutGb>
DGFV_HD void face_point_rev_seq_s(const DevPhys& P, const double* uL, const Prim<NK>& sL, const double* uR,
                                  const Prim<NK>& sR, int d, const double* Fb, double* uLb, double* uRb,
                                  bool fv_involved, GetG getg, PutGb putgb) {
    constexpr int V = NK + 4;
    PrimBar<NK> bL, bR;
    zero(bL);
    zero(bR);
    double half[V];
#pragma unroll
    for (int v = 0; v < V; ++v) half[v] = 0.5 * Fb[v];
    if (use_roe(P, fv_involved)) {
        riemann_roe_rev<NK>(P, uL, sL, uR, sR, d, Fb, uLb, bL, uRb, bR);
    } else {
        // local Lax-Friedrichs: F = (F_L + F_R)/2 - smax (uR - uL)/2
        const double aL = fabs(sL.v[d]) + sL.c, aR = fabs(sR.v[d]) + sR.c;
        const double smax = aL > aR ? aL : aR;
        double smaxb = 0.0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            uRb[v] -= half[v] * smax;
            uLb[v] += half[v] * smax;
            smaxb -= half[v] * (uR[v] - uL[v]);
        }
        flux_conv_rev<NK>(uL, sL, d, half, uLb, bL);
        flux_conv_rev<NK>(uR, sR, d, half, uRb, bR);
        if (aL > aR) {
            bL.v[d] += smaxb * (sL.v[d] > 0.0 ? 1.0 : (sL.v[d] < 0.0 ? -1.0 : 0.0));
            bL.c += smaxb;
        } else {
            bR.v[d] += smaxb * (sR.v[d] > 0.0 ? 1.0 : (sR.v[d] < 0.0 ? -1.0 : 0.0));
            bR.c += smaxb;
        }
    }
    if (P.viscous) {
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const Prim<NK>& s = side ? sR : sL;
            PrimBar<NK>& b = side ? bR : bL;
            double g[3 * V], gb[3 * V];
            getg(side, g);
#pragma unroll
            for (int x = 0; x < 3 * V; ++x) gb[x] = 0.0;
            PrimGrad<NK> G;
            PrimGradBar<NK> Gb;
            prim_grad<NK>(P, s, g, G);
            zero(Gb);
            flux_visc_rev<NK>(P, s, G, d, half, Gb, b);
            prim_grad_rev_face<NK, DC>(P, s, g, G, Gb, gb, b);
            putgb(side, gb);
        }
    }
    prim_rev<NK>(P, uL, sL, bL, uLb);
    prim_rev<NK>(P, uR, sR, bR, uRb);
}

template <int NK, int DC = -1, class GetG, class PutGb>
DGFV_HD void face_point_rev_seq(const DevPhys& P, const double* uL, const double* uR, int d, const double* Fb,
                                double* uLb, double* uRb, bool fv_involved, GetG getg, PutGb putgb) {
    Prim<NK> sL, sR;
    prim<NK>(P, uL, sL);
    prim<NK>(P, uR, sR);
    face_point_rev_seq_s<NK, DC>(P, uL, sL, uR, sR, d, Fb, uLb, uRb, fv_involved, getg, putgb);
}

// The same with both gradients given and both gradient adjoints accumulated
// into gLb, gRb.
template <int NK, int DC = -1>
DGFV_HD void face_point_rev(const DevPhys& P, const double* uL, const double* gL, const double* uR,
                            const double* gR, int d, const double* Fb, double* uLb, double* gLb, double* uRb,
                            double* gRb, bool fv_involved = false) {
    constexpr int V = NK + 4;
    face_point_rev_seq<NK, DC>(
        P, uL, uR, d, Fb, uLb, uRb, fv_involved,
        [&](int side, double* g) {
            const double* src = side ? gR : gL;
#pragma unroll
            for (int x = 0; x < 3 * V; ++x) g[x] = src[x];
        },
        [&](int side, const double* gb) {
            double* dst = side ? gRb : gLb;
#pragma unroll
            for (int x = 0; x < 3 * V; ++x) dst[x] += gb[x];
        });
}

}  // namespace dgfv
