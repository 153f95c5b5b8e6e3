"""Pins of the oracle's pointwise physics (Sec. 2) and Riemann solvers
(Sec. 3.1.1) against closed forms, symmetries and a textbook Roe solver."""
import numpy as np
import pytest

from paper_2502_19342_gb300 import workloads as W


def _prob(nk, riemann=0, mu=1e-2, D=3e-3, Pr=(0.72, 0.7, 0.68)):
    specs = [W.AIR, W.CO2, W.HELIUM][:nk]
    sp = W.species_set(specs, mu=mu)
    sp["Pr"] = np.array(Pr[:nk])
    sp["Dk"] = np.array([D, 2 * D, 0.5 * D][:nk])
    sp["mu"] = np.array([mu, 0.7 * mu, 1.3 * mu][:nk])
    sp["riemann"] = riemann
    return sp


def _state(rng, nk, rho=(0.6, 0.3, 0.2), v=None, p=1.3, prob=None):
    rk = np.array(rho[:nk]) * (1 + 0.1 * rng.random(nk))
    v = rng.standard_normal(3) * 0.4 if v is None else np.asarray(v, float)
    rhot = rk.sum()
    cv = prob["Rgas"] / (prob["gamma"] - 1)
    kap = (rk @ (prob["gamma"] * cv)) / (rk @ cv)
    rE = p / (kap - 1) + 0.5 * rhot * v @ v
    return np.concatenate([rk, rhot * v, [rE]])


def test_single_species_reduces_to_gamma_law(oracle):
    prob = _prob(1)
    u = np.array([1.3, 0.4, -0.2, 0.1, 3.0])
    s = oracle.primitives(prob, u)
    g, R = prob["gamma"][0], prob["Rgas"][0]
    p = (g - 1) * (u[4] - 0.5 * (u[1] ** 2 + u[2] ** 2 + u[3] ** 2) / u[0])
    assert abs(s["p"] - p) < 1e-14
    assert abs(s["T"] - p / (u[0] * R)) < 1e-12
    assert abs(s["c"] - np.sqrt(g * p / u[0])) < 1e-14
    assert abs(s["kappa"] - g) < 1e-15


def test_identical_species_equal_single_species(oracle):
    p1 = _prob(1)
    p2 = dict(p1)
    for k in ("gamma", "Rgas", "mu", "Pr", "Dk"):
        p2[k] = np.array([p1[k][0], p1[k][0]])
    rng = np.random.default_rng(3)
    u1 = _state(rng, 1, prob=p1)
    u2 = np.concatenate([[0.3 * u1[0], 0.7 * u1[0]], u1[1:]])
    g1 = rng.standard_normal(3 * 5)
    # split the density gradient between the two (identical) species
    g2 = np.zeros(3 * 6)
    for d in range(3):
        g2[d * 6 + 0] = 0.3 * g1[d * 5]
        g2[d * 6 + 1] = 0.7 * g1[d * 5]
        g2[d * 6 + 2:d * 6 + 6] = g1[d * 5 + 1:d * 5 + 5]
    for d in range(3):
        Fc1, Fv1 = oracle.flux(p1, u1, g1, d)
        Fc2, Fv2 = oracle.flux(p2, u2, g2, d)
        np.testing.assert_allclose(Fc2[0] + Fc2[1], Fc1[0], rtol=1e-14)
        np.testing.assert_allclose(Fc2[2:], Fc1[1:], rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(Fv2[0] + Fv2[1], Fv1[0], atol=1e-15)
        np.testing.assert_allclose(Fv2[2:], Fv1[1:], rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("nk", [1, 2, 3])
def test_species_diffusion_fluxes_sum_to_zero(oracle, nk):
    prob = _prob(nk)
    rng = np.random.default_rng(nk)
    for _ in range(5):
        u = _state(rng, nk, prob=prob)
        g = rng.standard_normal(3 * (nk + 4))
        for d in range(3):
            _, Fv = oracle.flux(prob, u, g, d)
            assert abs(Fv[:nk].sum()) < 1e-15


def _permute(u, g, nk, perm):
    """Relabel the axes: new axis perm[i] carries old axis i."""
    V = nk + 4
    u2 = u.copy()
    for i in range(3):
        u2[nk + perm[i]] = u[nk + i]
    g2 = np.zeros_like(g)
    for d in range(3):
        gd = g[d * V:(d + 1) * V].copy()
        gd2 = gd.copy()
        for i in range(3):
            gd2[nk + perm[i]] = gd[nk + i]
        g2[perm[d] * V:(perm[d] + 1) * V] = gd2
    return u2, g2


@pytest.mark.parametrize("perm", [(1, 2, 0), (2, 0, 1), (1, 0, 2), (0, 2, 1)])
def test_fluxes_are_covariant_under_axis_relabelling(oracle, perm):
    nk = 3
    prob = _prob(nk)
    rng = np.random.default_rng(11)
    u = _state(rng, nk, prob=prob)
    g = rng.standard_normal(3 * (nk + 4))
    u2, g2 = _permute(u, g, nk, perm)
    for d in range(3):
        Fc, Fv = oracle.flux(prob, u, g, d)
        Fc2, Fv2 = oracle.flux(prob, u2, g2, perm[d])
        Fc_p, _ = _permute(Fc, np.zeros(3 * (nk + 4)), nk, perm)
        Fv_p, _ = _permute(Fv, np.zeros(3 * (nk + 4)), nk, perm)
        np.testing.assert_allclose(Fc2, Fc_p, rtol=1e-14, atol=1e-15)
        np.testing.assert_allclose(Fv2, Fv_p, rtol=1e-13, atol=1e-15)


def test_viscous_flux_closed_forms(oracle):
    nk = 2
    prob = _prob(nk, D=2e-3)
    prob["Dk"] = np.array([2e-3, 2e-3])
    mu = prob["mu"]
    rk = np.array([0.7, 0.5])
    rho = rk.sum()
    Y = rk / rho
    p = 1.1
    cv = prob["Rgas"] / (prob["gamma"] - 1)
    cp = prob["gamma"] * cv
    cvm, cpm = Y @ cv, Y @ cp
    kap = cpm / cvm
    u = np.concatenate([rk, [0, 0, 0], [p / (kap - 1)]])
    V = nk + 4
    mum = Y @ mu
    prm = Y @ prob["Pr"]
    T = p / (rho * (cpm - cvm))
    # shear: only d(rho v_y)/dx = a
    g = np.zeros(3 * V)
    a = 0.37
    g[0 * V + nk + 1] = a
    _, Fx = oracle.flux(prob, u, g, 0)
    _, Fy = oracle.flux(prob, u, g, 1)
    assert abs(Fx[nk + 1] - (-mum * a / rho)) < 1e-16
    assert abs(Fy[nk + 0] - (-mum * a / rho)) < 1e-16
    # dilatation: only d(rho v_x)/dx = a: tau_xx = 4/3 mu a/rho, tau_yy = -2/3 mu a/rho
    g = np.zeros(3 * V)
    g[0 * V + nk + 0] = a
    _, Fx = oracle.flux(prob, u, g, 0)
    _, Fy = oracle.flux(prob, u, g, 1)
    assert abs(Fx[nk] - (-4.0 / 3.0 * mum * a / rho)) < 1e-15
    assert abs(Fy[nk + 1] - (2.0 / 3.0 * mum * a / rho)) < 1e-15
    # heat conduction at rest: only d(rho E)/dz = q -> grad T = q/(rho cv)
    g = np.zeros(3 * V)
    q = 0.21
    g[2 * V + nk + 3] = q
    _, Fz = oracle.flux(prob, u, g, 2)
    lam = mum * cpm / prm
    assert abs(Fz[nk + 3] - (-lam * q / (rho * cvm))) < 1e-15  # F^v = q_h = -lambda grad T
    # Fickian diffusion at rest and fixed rho: d(rho_1)/dy = s = -d(rho_2)/dy,
    # equal D: J_1 = -D s; q_d = (cp_1 - cp_2) T J_1 plus heat conduction from grad c_v.
    g = np.zeros(3 * V)
    s = 0.3
    g[1 * V + 0] = s
    g[1 * V + 1] = -s
    _, Fy = oracle.flux(prob, u, g, 1)
    D = prob["Dk"][0]
    assert abs(Fy[0] - (-D * s)) < 1e-16
    assert abs(Fy[1] - (D * s)) < 1e-16
    dYdy = s / rho
    dTdy = -T * (cv[0] - cv[1]) * dYdy / cvm
    expected_E = -lam * dTdy + (cp[0] - cp[1]) * T * (-D * s)
    assert abs(Fy[nk + 3] - expected_E) < 1e-14


def _mirror(u, nk, d):
    m = u.copy()
    m[nk + d] = -m[nk + d]
    return m


@pytest.mark.parametrize("riemann", [0, 1])
@pytest.mark.parametrize("nk", [1, 2, 3])
def test_riemann_consistency_and_mirror_symmetry(oracle, riemann, nk):
    prob = _prob(nk, riemann=riemann)
    rng = np.random.default_rng(5 + nk)
    for _ in range(4):
        uL = _state(rng, nk, prob=prob, p=1.0 + rng.random())
        uR = _state(rng, nk, prob=prob, p=1.0 + rng.random())
        for d in range(3):
            Fc, _ = oracle.flux(prob, uL, np.zeros(3 * (nk + 4)), d)
            np.testing.assert_allclose(oracle.riemann(prob, uL, uL, d), Fc, rtol=1e-13, atol=1e-14)
            # reflecting the normal: F*(uL,uR) = -M F*(M uR, M uL)
            F = oracle.riemann(prob, uL, uR, d)
            Fm = oracle.riemann(prob, _mirror(uR, nk, d), _mirror(uL, nk, d), d)
            np.testing.assert_allclose(F, -_mirror(Fm, nk, d), rtol=1e-12, atol=1e-13)


def _textbook_roe(uL, uR, gamma, d, hh=True):
    """Single-gas Roe flux with Harten-Hyman fix (standard textbook form)."""
    def prim(u):
        rho = u[0]
        v = u[1:4] / rho
        p = (gamma - 1) * (u[4] - 0.5 * rho * v @ v)
        return rho, v, p

    def flux(u):
        rho, v, p = prim(u)
        F = u * v[d]
        F[1 + d] += p
        F[4] += p * v[d]
        return F

    rL, vL, pL = prim(uL)
    rR, vR, pR = prim(uR)
    HL = (uL[4] + pL) / rL
    HR = (uR[4] + pR) / rR
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    v = (sL * vL + sR * vR) / (sL + sR)
    H = (sL * HL + sR * HR) / (sL + sR)
    a = np.sqrt((gamma - 1) * (H - 0.5 * v @ v))
    rt = sL * sR
    dp, drho, dv = pR - pL, rR - rL, vR - vL
    un = v[d]
    n = np.zeros(3)
    n[d] = 1
    waves = []
    a1 = (dp - rt * a * dv[d]) / (2 * a * a)
    waves.append((un - a, a1, np.concatenate([[1], v - a * n, [H - un * a]])))
    a2 = drho - dp / (a * a)
    waves.append((un, a2, np.concatenate([[1], v, [0.5 * v @ v]])))
    for t in range(3):
        if t == d:
            continue
        et = np.zeros(3)
        et[t] = 1
        waves.append((un, rt * dv[t], np.concatenate([[0], et, [v[t]]])))
    a5 = (dp + rt * a * dv[d]) / (2 * a * a)
    waves.append((un + a, a5, np.concatenate([[1], v + a * n, [H + un * a]])))
    cL, cR = np.sqrt(gamma * pL / rL), np.sqrt(gamma * pR / rR)
    lam_side = {0: (vL[d] - cL, vR[d] - cR), len(waves) - 1: (vL[d] + cL, vR[d] + cR)}
    diss = np.zeros(5)
    for i, (lam, al, K) in enumerate(waves):
        aa = abs(lam)
        if hh and i in lam_side:
            lL, lR = lam_side[i]
            delta = max(0.0, lam - lL, lR - lam)
            if aa < delta:
                aa = delta
        diss += aa * al * K
    return 0.5 * (flux(uL) + flux(uR)) - 0.5 * diss


def test_roe_single_species_equals_textbook(oracle):
    prob = _prob(1, riemann=1)
    g = prob["gamma"][0]
    rng = np.random.default_rng(9)
    for case in range(8):
        uL = _state(rng, 1, prob=prob, p=1.0 + rng.random())
        uR = _state(rng, 1, prob=prob, p=0.5 + rng.random())
        if case == 0:  # transonic rarefaction: exercises the entropy fix
            uL = _state(rng, 1, v=(-0.2, 0.1, 0), prob=prob, p=3.0)
            uR = _state(rng, 1, v=(1.6, 0.1, 0), prob=prob, p=0.3)
        for d in range(3):
            np.testing.assert_allclose(oracle.riemann(prob, uL, uR, d), _textbook_roe(uL, uR, g, d),
                                       rtol=1e-12, atol=1e-13)


def test_llf_textbook_form(oracle):
    prob = _prob(2, riemann=0)
    rng = np.random.default_rng(2)
    uL = _state(rng, 2, prob=prob)
    uR = _state(rng, 2, prob=prob, p=0.6)
    for d in range(3):
        FL, _ = oracle.flux(prob, uL, np.zeros(18), d)
        FR, _ = oracle.flux(prob, uR, np.zeros(18), d)
        sL, sR = oracle.primitives(prob, uL), oracle.primitives(prob, uR)
        smax = max(abs(uL[2 + d] / sL["rho"]) + sL["c"], abs(uR[2 + d] / sR["rho"]) + sR["c"])
        np.testing.assert_allclose(oracle.riemann(prob, uL, uR, d), 0.5 * (FL + FR) - 0.5 * smax * (uR - uL),
                                   rtol=1e-14, atol=1e-15)


def _euler_flux(prob, u, d):
    """Convective flux of one state in direction d, written out from Eq. 1 with
    the ideal-gas mixture law p = (kappa - 1)(rho E - rho|v|^2/2), kappa = c_p/c_v."""
    nk = len(prob["gamma"])
    rk = u[:nk]
    rho = rk.sum()
    v = u[nk:nk + 3] / rho
    cv = prob["Rgas"] / (prob["gamma"] - 1)
    kap = (rk @ (cv * prob["gamma"])) / (rk @ cv)
    p = (kap - 1) * (u[nk + 3] - 0.5 * rho * v @ v)
    F = u * v[d]
    F[nk + d] += p
    F[nk + 3] += p * v[d]
    return F, p


def _mixture_state(prob, rho_k, v, p):
    nk = len(rho_k)
    rho_k = np.asarray(rho_k, float)
    v = np.asarray(v, float)
    cv = prob["Rgas"][:nk] / (prob["gamma"][:nk] - 1)
    kap = (rho_k @ (cv * prob["gamma"][:nk])) / (rho_k @ cv)
    return np.concatenate([rho_k, rho_k.sum() * v, [p / (kap - 1) + 0.5 * rho_k.sum() * v @ v]])


@pytest.mark.parametrize("nk", [2, 3])
def test_roe_mixture_property_u_supersonic(oracle, nk):
    """Roe's property U for the mixture average (Sec. 3.1.1): when every wave
    of the linearisation moves the same way and the entropy fix is inactive,
    |A~| = +-A~ and A~(u_R - u_L) = F(u_R) - F(u_L) make the Roe flux the
    upwind flux exactly: F* = F(u_L) for v_n - c > 0 on both sides, F(u_R) for
    v_n + c < 0.  Species of different gamma and R, unequal compositions and
    temperatures on the two sides.  (The mixture average with kappa~ taken
    from the sqrt(rho)-weighted mass fractions misses this by 2e-4 .. 1e-3.)"""
    prob = _prob(nk, riemann=1)
    rng = np.random.default_rng(40 + nk)
    for trial in range(6):
        rkL = np.array([0.6, 0.3, 0.2][:nk]) * (0.5 + rng.random(nk))
        rkR = np.array([0.2, 0.7, 0.1][:nk]) * (0.5 + rng.random(nk))
        for d in range(3):
            for sign in (1.0, -1.0):
                vL = rng.standard_normal(3) * 0.2
                vR = vL + rng.standard_normal(3) * 0.05
                vL[d] = sign * (3.0 + 0.1 * rng.random())
                vR[d] = sign * (3.0 + 0.1 * rng.random())
                uL = _mixture_state(prob, rkL, vL, 1.0 + 0.2 * rng.random())
                uR = _mixture_state(prob, rkR, vR, 1.0 + 0.2 * rng.random())
                sL, sR = oracle.primitives(prob, uL), oracle.primitives(prob, uR)
                if sign > 0:
                    assert vL[d] - sL["c"] > 0 and vR[d] - sR["c"] > 0
                else:
                    assert vL[d] + sL["c"] < 0 and vR[d] + sR["c"] < 0
                F = oracle.riemann(prob, uL, uR, d)
                Fup, _ = _euler_flux(prob, uL if sign > 0 else uR, d)
                np.testing.assert_allclose(F, Fup, rtol=0, atol=1e-14 * np.abs(Fup).max())


@pytest.mark.parametrize("nk", [2, 3])
def test_roe_mixture_contact_discontinuities(oracle, nk):
    """Contact between two mixtures of different gamma and R at equal pressure
    and velocity (different compositions and temperatures), Sec. 3.1.1.
    At rest the exact flux carries no mass, species or energy and the momentum
    flux is p n; moving with v_n != 0 the jump lies entirely in the contact
    waves of an exact linearisation, so the Roe flux is the upwind flux."""
    prob = _prob(nk, riemann=1)
    rng = np.random.default_rng(60 + nk)
    for trial in range(6):
        rkL = np.array([0.9, 0.1, 0.3][:nk]) * (0.5 + rng.random(nk))
        rkR = np.array([0.1, 0.8, 0.05][:nk]) * (0.5 + rng.random(nk))
        p = 0.5 + rng.random()
        for d in range(3):
            uL = _mixture_state(prob, rkL, (0, 0, 0), p)
            uR = _mixture_state(prob, rkR, (0, 0, 0), p)
            F = oracle.riemann(prob, uL, uR, d)
            expect = np.zeros(nk + 4)
            expect[nk + d] = p
            np.testing.assert_allclose(F, expect, rtol=0, atol=1e-14 * p)
            v = rng.standard_normal(3) * 0.3
            uL = _mixture_state(prob, rkL, v, p)
            uR = _mixture_state(prob, rkR, v, p)
            F = oracle.riemann(prob, uL, uR, d)
            Fup, _ = _euler_flux(prob, uL if v[d] > 0 else uR, d)
            np.testing.assert_allclose(F, Fup, rtol=0, atol=1e-14 * np.abs(Fup).max())


def _at_temperature(prob, T, rho=1.0):
    """Single-species state at rest with temperature T."""
    cv = prob["Rgas"][0] / (prob["gamma"][0] - 1)
    return np.array([rho, 0.0, 0.0, 0.0, rho * cv * T])


def test_sutherland_viscosity_limits_and_log_slope(oracle):
    """Sutherland's law (the TGV of Sec. 4.3): mu(T_ref) = mu_0; the logarithmic
    slope d ln mu / d ln T = 3/2 - T/(T + S) (3/2 far below S, 1/2 far above);
    lambda = mu c_p / Pr follows mu.  Slopes by central differences."""
    prob = _prob(1, mu=2e-3)
    prob.update(sutherland=1, T_ref=0.8, S_sutherland=0.3)
    s0 = oracle.primitives(prob, _at_temperature(prob, 0.8))
    assert abs(s0["mu"] - 2e-3) < 1e-18
    for T in (0.01, 0.3, 0.8, 2.5, 300.0):
        h = 1e-5
        mp = oracle.primitives(prob, _at_temperature(prob, T * (1 + h)))["mu"]
        mm = oracle.primitives(prob, _at_temperature(prob, T * (1 - h)))["mu"]
        slope = (np.log(mp) - np.log(mm)) / (np.log(1 + h) - np.log(1 - h))
        assert abs(slope - (1.5 - T / (T + 0.3))) < 1e-6, (T, slope)
        s = oracle.primitives(prob, _at_temperature(prob, T))
        assert abs(s["lam"] / s["mu"] - s["cp"] / prob["Pr"][0]) < 1e-12 * s["cp"] / prob["Pr"][0]
    plain = _prob(1, mu=2e-3)
    assert oracle.primitives(plain, _at_temperature(plain, 2.5))["mu"] == 2e-3


def test_indicator_variable_choice_swaps_the_roles(oracle):
    """indicator_vars = 1 (Sec. 4.3): p-refinement on the pressure indicator and
    FV on the density indicator.  With one species the default takes I(rho) and
    I(p) the other way round, so the two outputs swap exactly."""
    sp = W.species_set([W.AIR], mu=1e-3)
    prob = W.make_problem([((3, 2, 2), (0, 0, 0), (1, 1, 1))], sp, n_fv=6, N=W.random_degrees(12, 1, 5, 3),
                          fv=W.random_fv(12, 0.25, 3))
    U = W.smooth_random_state(prob, 3, amp=0.2)
    Ip0, Ih0 = oracle.indicator(prob, U)
    Ip1, Ih1 = oracle.indicator(dict(prob, indicator_vars=1), U)
    np.testing.assert_array_equal(Ip1, Ih0)
    np.testing.assert_array_equal(Ih1, Ip0)


# ---------------------------------------------------------------- sensitivity of the Roe pins
def _roe_matrix(prob, uL, uR, d, average):
    """Roe matrix A~ of the mixture Euler flux in direction d, written from
    the product rule for jumps: with sqrt(rho)-weighted v~, H~, Y~,
      d(rho_k v_d)  = Y~_k dm_d + v~_d drho_k - Y~_k v~_d drho,
      d(m_i v_d)    = v~_i dm_d + v~_d dm_i - v~_i v~_d drho,
      d(rho H v_d)  = H~ dm_d + v~_d (d(rho E) + dp) - H~ v~_d drho,
    and the pressure jump
      dp = (kappa~ - 1)[d(rho E) - v~.dm + |v~|^2/2 drho] + sum_k psi_k drho_k.
    `average` picks kappa~ and psi_k:
      "exact"  - kappa~ - 1 = sum R_k rhobar_k / sum c_v,k rhobar_k (arithmetic
                 means of the partial densities), psi_k = Tbar (c_p,k - kappa~ c_v,k);
                 the product rule applied to p = sum rho_k R_k T and
                 rho e = sum rho_k c_v,k T makes dp exact;
      "frozen" - kappa~ = c_p(Y~)/c_v(Y~), psi_k = 0: the single-gas average with
                 the species carried as passive scalars."""
    nk = len(prob["gamma"])
    Rk = prob["Rgas"]
    cv = Rk / (prob["gamma"] - 1)
    cp = cv + Rk

    def parts(u):
        rk = u[:nk]
        rho = rk.sum()
        v = u[nk:nk + 3] / rho
        T = (u[nk + 3] - 0.5 * rho * v @ v) / (rk @ cv)
        p = T * (rk @ Rk)
        return rk, rho, v, T, p, (u[nk + 3] + p) / rho

    rkL, rL, vL, TL, pL, HL = parts(uL)
    rkR, rR, vR, TR, pR, HR = parts(uR)
    wL, wR = np.sqrt(rL), np.sqrt(rR)
    avg = lambda a, b: (wL * a + wR * b) / (wL + wR)
    v, H, Y = avg(vL, vR), avg(HL, HR), avg(rkL / rL, rkR / rR)
    if average == "exact":
        rbar = 0.5 * (rkL + rkR)
        km1 = (rbar @ Rk) / (rbar @ cv)
        psi = 0.5 * (TL + TR) * (cp - (1.0 + km1) * cv)
    else:
        km1 = (Y @ cp) / (Y @ cv) - 1.0
        psi = np.zeros(nk)
    V = nk + 4
    iM, iE = nk, nk + 3
    # pressure row: dp = P . du
    P = np.zeros(V)
    P[:nk] = km1 * 0.5 * (v @ v) + psi
    P[iM:iM + 3] = -km1 * v
    P[iE] = km1
    drho = np.zeros(V)
    drho[:nk] = 1.0
    A = np.zeros((V, V))
    for k in range(nk):
        A[k, k] += v[d]
        A[k] -= Y[k] * v[d] * drho
        A[k, iM + d] += Y[k]
    for i in range(3):
        A[iM + i, iM + d] += v[i]
        A[iM + i, iM + i] += v[d]
        A[iM + i] -= v[i] * v[d] * drho
        if i == d:
            A[iM + i] += P
    A[iE, iM + d] += H
    A[iE, iE] += v[d]
    A[iE] += v[d] * P
    A[iE] -= H * v[d] * drho
    return A


def _abs_matrix(A, at_rest):
    """|A~| in the two cases the pins use.  Supersonic: every eigenvalue
    positive, so |A~| = A~.  At rest: the eigenvalues are 0 (the species,
    shear and contact waves) and +-c~, so |A~| = A~^2 / c~ on every
    eigenvector."""
    lam = np.linalg.eigvals(A)
    assert np.abs(lam.imag).max() < 1e-8 * np.abs(lam).max()
    lam = np.sort(lam.real)
    if not at_rest:
        assert lam[0] > 0
        return A
    c = lam[-1]
    assert abs(lam[0] + c) < 1e-12 * c and np.abs(lam[1:-1]).max() < 1e-6 * c
    return A @ A / c


def test_roe_pins_reject_the_frozen_kappa_average():
    """The property-U and resting-contact pins above would catch a Roe flux
    built on the single-gas average: for species of different gamma its
    matrix misses A~ du = dF, so in every supersonic case its flux
    (F_L + F_R)/2 - |A~| du/2 differs from F(u_L) (by 0.5-2 % here, against
    the pin's 1e-14), and at every resting contact it carries mass (2-12 % of
    the partial densities); the exact mixture linearisation meets both to
    round-off.  For species of equal gamma both averages coincide."""
    rng = np.random.default_rng(81)
    for nk, specs in ((2, [W.AIR, W.HELIUM]), (3, [W.AIR, W.CO2, W.HELIUM]), (2, [W.AIR, dict(W.AIR, M=4.0)])):
        prob = W.species_set(specs)
        same_gamma = len({s["gamma"] for s in specs}) == 1
        best_frozen = np.inf
        for trial in range(4):
            rkL = np.array([0.6, 0.3, 0.2][:nk]) * (0.5 + rng.random(nk))
            rkR = np.array([0.2, 0.7, 0.1][:nk]) * (0.5 + rng.random(nk))
            for d in range(3):
                # supersonic: every wave to the right, the Roe flux must be F(u_L)
                vL = rng.standard_normal(3) * 0.2
                vR = vL + rng.standard_normal(3) * 0.05
                vL[d], vR[d] = 3.0 + 0.1 * rng.random(), 3.0 + 0.1 * rng.random()
                uL = _mixture_state(prob, rkL, vL, 1.0 + 0.2 * rng.random())
                uR = _mixture_state(prob, rkR, vR, 1.0 + 0.2 * rng.random())
                FL, _ = _euler_flux(prob, uL, d)
                FR, _ = _euler_flux(prob, uR, d)
                du, dF = uR - uL, FR - FL
                for average in ("exact", "frozen"):
                    Ab = _abs_matrix(_roe_matrix(prob, uL, uR, d, average), at_rest=False)
                    err = np.abs(0.5 * (FL + FR) - 0.5 * Ab @ du - FL).max() / np.abs(FL).max()
                    if average == "exact" or same_gamma:
                        assert err < 1e-13, (nk, average, err)
                    else:
                        best_frozen = min(best_frozen, err)
                # resting contact at equal pressure: no mass, species or energy flux
                p = 0.5 + rng.random()
                uL = _mixture_state(prob, rkL, (0, 0, 0), p)
                uR = _mixture_state(prob, rkR, (0, 0, 0), p)
                for average in ("exact", "frozen"):
                    Ab = _abs_matrix(_roe_matrix(prob, uL, uR, d, average), at_rest=True)
                    diss = 0.5 * Ab @ (uR - uL)
                    mass = np.abs(diss[:nk]).max() / np.abs(uL[:nk]).max()
                    if average == "exact" or same_gamma:
                        assert mass < 1e-13, (nk, average, mass)
                    else:
                        best_frozen = min(best_frozen, mass)
        if not same_gamma:
            assert best_frozen > 1e-3, (nk, best_frozen)  # every case fails its pin
