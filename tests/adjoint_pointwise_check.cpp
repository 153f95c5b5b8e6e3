// Host check of the hand-written pointwise adjoints of the CUDA path
// (physics_adj.cuh) against central finite differences of the forward
// functions (physics.cuh), compiled for the host by the test suite: volume
// node and face point (LLF and Roe-HH, transonic states for the entropy fix,
// constant and Sutherland viscosity) and the split form's two-point flux.
#include <cstdio>
#include <cstdlib>
#include <random>

#include "../paper_2502_19342_gb300/csrc/physics_adj.cuh"

using namespace dgfv;

// The face reverse specialised on a compile-time direction (the face kernels'
// form) against the general one: the same adjoint up to rounding.
template <int NK>
int compare_dir(const DevPhys& P, const double* uL, const double* gL, const double* uR, const double* gR, int d,
                const double* Fb, const double* uLb, const double* gLb, const double* uRb, const double* gRb) {
    constexpr int V = NK + 4;
    double a[V] = {}, b[3 * V] = {}, c[V] = {}, e[3 * V] = {};
    if (d == 0) face_point_rev<NK, 0>(P, uL, gL, uR, gR, d, Fb, a, b, c, e);
    else if (d == 1) face_point_rev<NK, 1>(P, uL, gL, uR, gR, d, Fb, a, b, c, e);
    else face_point_rev<NK, 2>(P, uL, gL, uR, gR, d, Fb, a, b, c, e);
    double diff = 0.0, mag = 1e-300;
    for (int v = 0; v < V; ++v) {
        diff = std::fmax(diff, std::fabs(a[v] - uLb[v]) + std::fabs(c[v] - uRb[v]));
        mag = std::fmax(mag, std::fabs(uLb[v]) + std::fabs(uRb[v]));
    }
    for (int x = 0; x < 3 * V; ++x) {
        diff = std::fmax(diff, std::fabs(b[x] - gLb[x]) + std::fabs(e[x] - gRb[x]));
        mag = std::fmax(mag, std::fabs(gLb[x]) + std::fabs(gRb[x]));
    }
    if (diff > 1e-13 * mag) {
        std::printf("direction-specialised face reverse NK=%d d=%d differs: %.3e of %.3e\n", NK, d, diff, mag);
        return 1;
    }
    return 0;
}

template <int NK>
DevPhys phys(bool visc, bool suth = false, int riemann = 0) {
    DevPhys P{};
    P.nk = NK;
    P.viscous = visc;
    P.riemann = riemann;
    P.sutherland = suth ? 1 : 0;
    P.T_ref = 1.3;
    P.S = 0.45;
    const double gam[3] = {1.4, 1.3, 1.67}, R[3] = {1.0 / 29, 1.0 / 44, 1.0 / 4};
    for (int k = 0; k < NK; ++k) {
        P.cv[k] = R[k] / (gam[k] - 1);
        P.cp[k] = gam[k] * P.cv[k];
        P.mu[k] = 1e-2 * (1 + 0.3 * k);
        P.pr[k] = 0.72 - 0.02 * k;
        P.D[k] = 3e-3 * (1 + 0.5 * k);
    }
    return P;
}

template <int NK>
void state(std::mt19937& rng, const DevPhys& P, double* u) {
    std::uniform_real_distribution<double> U(0.0, 1.0);
    double rho = 0.0, cv = 0.0;
    for (int k = 0; k < NK; ++k) {
        u[k] = 0.2 + 0.5 * U(rng);
        rho += u[k];
        cv += u[k] * P.cv[k];
    }
    double v[3], ke = 0.0;
    for (int i = 0; i < 3; ++i) {
        v[i] = U(rng) - 0.5;
        u[NK + i] = rho * v[i];
        ke += 0.5 * rho * v[i] * v[i];
    }
    u[NK + 3] = cv * (20.0 + 10 * U(rng)) + ke;  // rho c_v T + kinetic energy
}

template <int NK>
double vol_dot(const DevPhys& P, const double* u, const double* g, const double* Fb) {
    constexpr int V = NK + 4;
    Prim<NK> s;
    prim<NK>(P, u, s);
    PrimGrad<NK> G;
    if (P.viscous) prim_grad<NK>(P, s, g, G);
    double acc = 0.0;
    for (int d = 0; d < 3; ++d) {
        double F[V], Fv[V];
        flux_conv<NK>(u, s, d, F);
        if (P.viscous) {
            flux_visc<NK>(P, s, G, d, Fv);
            for (int v = 0; v < V; ++v) F[v] += Fv[v];
        }
        for (int v = 0; v < V; ++v) acc += Fb[d * V + v] * F[v];
    }
    return acc;
}

template <int NK>
double face_dot(const DevPhys& P, const double* uL, const double* gL, const double* uR, const double* gR, int d,
                const double* Fb) {
    constexpr int V = NK + 4;
    double F[V];
    interface_flux<NK>(P, uL, gL, uR, gR, d, F, false);
    double acc = 0.0;
    for (int v = 0; v < V; ++v) acc += Fb[v] * F[v];
    return acc;
}

template <int NK>
int check(bool visc, int seed, bool suth = false, int riemann = 0) {
    constexpr int V = NK + 4;
    std::mt19937 rng(seed);
    std::normal_distribution<double> N01(0.0, 1.0);
    DevPhys P = phys<NK>(visc, suth, riemann);
    int bad = 0;
    for (int trial = 0; trial < 20; ++trial) {
        double u[V], g[3 * V], Fb[3 * V], du[V], dg[3 * V];
        state<NK>(rng, P, u);
        for (int x = 0; x < 3 * V; ++x) { g[x] = 0.3 * N01(rng); Fb[x] = N01(rng); dg[x] = N01(rng); }
        for (int v = 0; v < V; ++v) du[v] = 0.05 * N01(rng) * std::fabs(u[v]);
        double ub[V] = {}, gb[3 * V] = {};
        volume_point_rev<NK>(P, u, g, Fb, ub, gb);
        const double eps = 1e-6;
        double up[V], um[V], gp[3 * V], gm[3 * V];
        for (int v = 0; v < V; ++v) { up[v] = u[v] + eps * du[v]; um[v] = u[v] - eps * du[v]; }
        for (int x = 0; x < 3 * V; ++x) { gp[x] = g[x] + eps * dg[x]; gm[x] = g[x] - eps * dg[x]; }
        const double fd = (vol_dot<NK>(P, up, gp, Fb) - vol_dot<NK>(P, um, gm, Fb)) / (2 * eps);
        double ad = 0.0;
        for (int v = 0; v < V; ++v) ad += ub[v] * du[v];
        for (int x = 0; x < 3 * V; ++x) ad += gb[x] * dg[x];
        if (std::fabs(fd - ad) > 1e-7 + 1e-6 * std::fabs(fd)) {
            std::printf("volume NK=%d visc=%d suth=%d trial %d: fd %.12e adjoint %.12e\n", NK, visc, suth, trial, fd, ad);
            ++bad;
        }
        // face
        double uR[V], gR[3 * V], FbF[V], duR[V], dgR[3 * V];
        state<NK>(rng, P, uR);
        for (int x = 0; x < 3 * V; ++x) { gR[x] = 0.3 * N01(rng); dgR[x] = N01(rng); }
        for (int v = 0; v < V; ++v) { FbF[v] = N01(rng); duR[v] = 0.05 * N01(rng) * std::fabs(uR[v]); }
        const int d = trial % 3;
        double uLb[V] = {}, gLb[3 * V] = {}, uRb[V] = {}, gRb[3 * V] = {};
        face_point_rev<NK>(P, u, g, uR, gR, d, FbF, uLb, gLb, uRb, gRb);
        bad += compare_dir<NK>(P, u, g, uR, gR, d, FbF, uLb, gLb, uRb, gRb);
        double uRp[V], uRm[V], gRp[3 * V], gRm[3 * V];
        for (int v = 0; v < V; ++v) { uRp[v] = uR[v] + eps * duR[v]; uRm[v] = uR[v] - eps * duR[v]; }
        for (int x = 0; x < 3 * V; ++x) { gRp[x] = gR[x] + eps * dgR[x]; gRm[x] = gR[x] - eps * dgR[x]; }
        const double fdf = (face_dot<NK>(P, up, gp, uRp, gRp, d, FbF) - face_dot<NK>(P, um, gm, uRm, gRm, d, FbF)) / (2 * eps);
        double adf = 0.0;
        for (int v = 0; v < V; ++v) adf += uLb[v] * du[v] + uRb[v] * duR[v];
        for (int x = 0; x < 3 * V; ++x) adf += gLb[x] * dg[x] + gRb[x] * dgR[x];
        if (std::fabs(fdf - adf) > 1e-7 + 1e-6 * std::fabs(fdf)) {
            std::printf("face NK=%d visc=%d suth=%d riemann=%d trial %d: fd %.12e adjoint %.12e\n", NK, visc, suth,
                        riemann, trial, fdf, adf);
            ++bad;
        }
    }
    return bad;
}

// Sets the normal velocity of u to f times its sound speed, keeping density,
// the other velocity components and the temperature.
template <int NK>
void set_normal_mach(const DevPhys& P, double* u, int d, double f) {
    Prim<NK> s;
    prim<NK>(P, u, s);
    const double vn = f * s.c;
    u[NK + 3] += 0.5 * s.rho * (vn * vn - s.v[d] * s.v[d]);
    u[NK + d] = s.rho * vn;
}

// Face adjoint of the Roe flux at transonic states, where the Harten-Hyman fix
// is active on the u - c wave (even trials) or the u + c wave (odd trials).
template <int NK>
int check_transonic(bool visc, int seed) {
    constexpr int V = NK + 4;
    std::mt19937 rng(seed);
    std::normal_distribution<double> N01(0.0, 1.0);
    DevPhys P = phys<NK>(visc, false, 1);
    int bad = 0;
    for (int trial = 0; trial < 20; ++trial) {
        const int d = trial % 3;
        double uL[V], uR[V], gL[3 * V], gR[3 * V], Fb[V], duL[V], duR[V], dgL[3 * V], dgR[3 * V];
        state<NK>(rng, P, uL);
        state<NK>(rng, P, uR);
        if (trial % 2 == 0) {
            set_normal_mach<NK>(P, uL, d, 0.8);
            set_normal_mach<NK>(P, uR, d, 1.2);
        } else {
            set_normal_mach<NK>(P, uL, d, -1.2);
            set_normal_mach<NK>(P, uR, d, -0.8);
        }
        for (int x = 0; x < 3 * V; ++x) {
            gL[x] = 0.3 * N01(rng); gR[x] = 0.3 * N01(rng); dgL[x] = N01(rng); dgR[x] = N01(rng);
        }
        for (int v = 0; v < V; ++v) {
            Fb[v] = N01(rng);
            duL[v] = 0.05 * N01(rng) * std::fabs(uL[v]);
            duR[v] = 0.05 * N01(rng) * std::fabs(uR[v]);
        }
        double uLb[V] = {}, gLb[3 * V] = {}, uRb[V] = {}, gRb[3 * V] = {};
        face_point_rev<NK>(P, uL, gL, uR, gR, d, Fb, uLb, gLb, uRb, gRb);
        bad += compare_dir<NK>(P, uL, gL, uR, gR, d, Fb, uLb, gLb, uRb, gRb);
        const double eps = 1e-6;
        double a[V], b[V], c[V], e[V], ga[3 * V], gb[3 * V], gc[3 * V], ge[3 * V];
        for (int v = 0; v < V; ++v) { a[v] = uL[v] + eps * duL[v]; b[v] = uL[v] - eps * duL[v];
                                      c[v] = uR[v] + eps * duR[v]; e[v] = uR[v] - eps * duR[v]; }
        for (int x = 0; x < 3 * V; ++x) { ga[x] = gL[x] + eps * dgL[x]; gb[x] = gL[x] - eps * dgL[x];
                                          gc[x] = gR[x] + eps * dgR[x]; ge[x] = gR[x] - eps * dgR[x]; }
        const double fd = (face_dot<NK>(P, a, ga, c, gc, d, Fb) - face_dot<NK>(P, b, gb, e, ge, d, Fb)) / (2 * eps);
        double ad = 0.0;
        for (int v = 0; v < V; ++v) ad += uLb[v] * duL[v] + uRb[v] * duR[v];
        for (int x = 0; x < 3 * V; ++x) ad += gLb[x] * dgL[x] + gRb[x] * dgR[x];
        if (std::fabs(fd - ad) > 1e-7 + 1e-6 * std::fabs(fd)) {
            std::printf("transonic Roe NK=%d visc=%d trial %d: fd %.12e adjoint %.12e\n", NK, visc, trial, fd, ad);
            ++bad;
        }
    }
    return bad;
}

// Split form (Sec. 3.5): the two-point KEP flux of two states through their
// tuples, reversed with kep_flux_rev (half of each mean's adjoint per tuple),
// kep_tuple_rev and prim_rev.
template <int NK>
int check_kep(int seed) {
    constexpr int V = NK + 4, NT = 6 + NK;
    std::mt19937 rng(seed);
    std::normal_distribution<double> N01(0.0, 1.0);
    DevPhys P = phys<NK>(false);
    auto flux = [&](const double* ua, const double* ub, int d, double* F) {
        Prim<NK> sa, sb;
        prim<NK>(P, ua, sa);
        prim<NK>(P, ub, sb);
        double ta[NT], tb[NT];
        kep_tuple<NK>(sa, ta);
        kep_tuple<NK>(sb, tb);
        kep_flux<NK>(ta, tb, d, F);
    };
    int bad = 0;
    for (int trial = 0; trial < 30; ++trial) {
        const int d = trial % 3;
        double ua[V], ub[V], Fb[V], da[V], db[V];
        state<NK>(rng, P, ua);
        state<NK>(rng, P, ub);
        for (int v = 0; v < V; ++v) {
            Fb[v] = N01(rng);
            da[v] = 0.05 * N01(rng) * std::fabs(ua[v]);
            db[v] = 0.05 * N01(rng) * std::fabs(ub[v]);
        }
        Prim<NK> sa, sb;
        prim<NK>(P, ua, sa);
        prim<NK>(P, ub, sb);
        double ta[NT], tb[NT], tab[NT] = {}, tbb[NT] = {};
        kep_tuple<NK>(sa, ta);
        kep_tuple<NK>(sb, tb);
        kep_flux_rev<NK>(ta, tb, d, Fb, tab);
        kep_flux_rev<NK>(ta, tb, d, Fb, tbb);
        double uab[V] = {}, ubb[V] = {};
        PrimBar<NK> ba, bb;
        zero(ba);
        zero(bb);
        kep_tuple_rev<NK>(sa, tab, ba);
        kep_tuple_rev<NK>(sb, tbb, bb);
        prim_rev<NK>(P, ua, sa, ba, uab);
        prim_rev<NK>(P, ub, sb, bb, ubb);
        const double eps = 1e-6;
        double ap[V], am[V], bp[V], bm[V], Fp[V], Fm[V];
        for (int v = 0; v < V; ++v) {
            ap[v] = ua[v] + eps * da[v]; am[v] = ua[v] - eps * da[v];
            bp[v] = ub[v] + eps * db[v]; bm[v] = ub[v] - eps * db[v];
        }
        flux(ap, bp, d, Fp);
        flux(am, bm, d, Fm);
        double fd = 0.0, ad = 0.0;
        for (int v = 0; v < V; ++v) {
            fd += Fb[v] * (Fp[v] - Fm[v]) / (2 * eps);
            ad += uab[v] * da[v] + ubb[v] * db[v];
        }
        if (std::fabs(fd - ad) > 1e-7 + 1e-6 * std::fabs(fd)) {
            std::printf("KEP NK=%d trial %d: fd %.12e adjoint %.12e\n", NK, trial, fd, ad);
            ++bad;
        }
    }
    return bad;
}

// FV reconstruction variables (Sec. 3.1.2): cons_to_w and w_to_cons reversed.
template <int NK>
int check_fv_maps(int seed) {
    constexpr int V = NK + 4;
    std::mt19937 rng(seed);
    std::normal_distribution<double> N01(0.0, 1.0);
    DevPhys P = phys<NK>(false);
    int bad = 0;
    for (int trial = 0; trial < 30; ++trial) {
        double u[V], du[V], wb[V], w[V], dw[V], ub_[V];
        state<NK>(rng, P, u);
        for (int v = 0; v < V; ++v) {
            du[v] = 0.05 * N01(rng) * std::fabs(u[v]);
            wb[v] = N01(rng);
            ub_[v] = N01(rng);
        }
        cons_to_w<NK>(P, u, w);
        for (int v = 0; v < V; ++v) dw[v] = 0.05 * N01(rng) * std::fabs(w[v]);
        const double eps = 1e-6;
        double up[V], um[V], wp[V], wm[V];
        for (int v = 0; v < V; ++v) { up[v] = u[v] + eps * du[v]; um[v] = u[v] - eps * du[v]; }
        cons_to_w<NK>(P, up, wp);
        cons_to_w<NK>(P, um, wm);
        double fd = 0.0, ad = 0.0, g[V] = {};
        for (int v = 0; v < V; ++v) fd += wb[v] * (wp[v] - wm[v]) / (2 * eps);
        cons_to_w_rev<NK>(P, u, wb, g);
        for (int v = 0; v < V; ++v) ad += g[v] * du[v];
        if (std::fabs(fd - ad) > 1e-7 + 1e-6 * std::fabs(fd)) {
            std::printf("cons_to_w NK=%d trial %d: fd %.12e adjoint %.12e\n", NK, trial, fd, ad);
            ++bad;
        }
        double a[V], b[V], ua[V], ubb[V], h[V] = {};
        for (int v = 0; v < V; ++v) { a[v] = w[v] + eps * dw[v]; b[v] = w[v] - eps * dw[v]; }
        w_to_cons<NK>(P, a, ua);
        w_to_cons<NK>(P, b, ubb);
        fd = 0.0;
        ad = 0.0;
        for (int v = 0; v < V; ++v) fd += ub_[v] * (ua[v] - ubb[v]) / (2 * eps);
        w_to_cons_rev<NK>(P, w, ub_, h);
        for (int v = 0; v < V; ++v) ad += h[v] * dw[v];
        if (std::fabs(fd - ad) > 1e-7 + 1e-6 * std::fabs(fd)) {
            std::printf("w_to_cons NK=%d trial %d: fd %.12e adjoint %.12e\n", NK, trial, fd, ad);
            ++bad;
        }
    }
    return bad;
}

int main() {
    int bad = 0;
    for (int visc = 0; visc < 2; ++visc) {
        bad += check<1>(visc, 1 + visc);
        bad += check<2>(visc, 3 + visc);
        bad += check<3>(visc, 5 + visc);
    }
    // Sutherland viscosity (Sec. 4.3)
    bad += check<1>(true, 7, true);
    bad += check<2>(true, 8, true);
    bad += check<3>(true, 9, true);
    // Roe flux with the Harten-Hyman fix
    for (int visc = 0; visc < 2; ++visc) {
        bad += check<1>(visc, 11 + visc, false, 1);
        bad += check<2>(visc, 13 + visc, false, 1);
        bad += check<3>(visc, 15 + visc, false, 1);
        bad += check_transonic<1>(visc, 21 + visc);
        bad += check_transonic<2>(visc, 23 + visc);
        bad += check_transonic<3>(visc, 25 + visc);
    }
    bad += check_fv_maps<1>(41);
    bad += check_fv_maps<2>(42);
    bad += check_fv_maps<3>(43);
    bad += check_kep<1>(31);
    bad += check_kep<2>(32);
    bad += check_kep<3>(33);
    std::printf("%s (%d mismatches)\n", bad ? "FAIL" : "OK", bad);
    return bad ? 1 : 0;
}
