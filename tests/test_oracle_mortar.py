"""Pins of the oracle's non-conforming (mortar) interfaces, Sec. 3.2.3: the
mortar matrices against their definitions (exact interpolation to a half, L2
projection computed independently with numpy, FV overlaps counted by hand), a
chain of equal domains against one periodic box, free-stream preservation and
discrete conservation through mortars of types 1-3 with random hp/FV patterns
(Sec. 4.1 uses a non-conforming mesh: one half at twice the resolution), the
convergence of the advected density wave of Sec. 4.2 on that mesh, and a
viscous shear flow whose right-hand side is known in closed form."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2502_19342_gb300 import workloads as W

from test_oracle_rhs import GOLDEN, _advected_l2, _per_var, _weights


def _nodes(n, kind):
    return W.dg_points(n, kind)


def _lagrange_eval(x, vals, t):
    """Value at t of the interpolant of vals on the nodes x (barycentric-free, plain products)."""
    out = np.zeros_like(t, dtype=float)
    for j in range(len(x)):
        l = np.ones_like(t, dtype=float)
        for m in range(len(x)):
            if m != j:
                l *= (t - x[m]) / (x[j] - x[m])
        out += vals[j] * l
    return out


# ---------------------------------------------------------------- mortar matrices
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("N", [1, 2, 4, 7])
def test_mortar_interpolation_is_exact_on_each_half(oracle, kind, N):
    """M_01, M_02: the big side's degree-N polynomial restricted to a half is a
    degree-N polynomial of the small side's coordinate eta, xi = (eta + 2s - 1)/2."""
    rng = np.random.default_rng(N + 10 * kind)
    c = rng.normal(size=N + 1)
    x = _nodes(N + 1, kind)
    p = np.polynomial.polynomial.polyval(x, c)
    for s in (0, 1):
        M = oracle.mortar(N, s, nodes=kind)
        exact = np.polynomial.polynomial.polyval((x + 2 * s - 1) / 2, c)
        assert np.abs(M @ p - exact).max() < 1e-13


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_mortar_projection_is_the_l2_projection(oracle, kind, N):
    """M_10 f_1 + M_20 f_2 is the degree-N polynomial g with int (g - f) phi = 0
    for every polynomial phi of degree <= N, f the piecewise polynomial given on
    the two halves (normal equations solved here in numpy with 30-point Gauss
    quadrature on each half, monomial basis)."""
    rng = np.random.default_rng(3 * N + kind)
    x = _nodes(N + 1, kind)
    f = [rng.normal(size=N + 1) for _ in range(2)]  # nodal values of the two small sides
    got = sum(oracle.mortar(N, s, proj=True, nodes=kind) @ f[s] for s in (0, 1))
    q, w = np.polynomial.legendre.leggauss(30)
    G = np.zeros((N + 1, N + 1))
    b = np.zeros(N + 1)
    for s in (0, 1):
        xi = (q + 2 * s - 1) / 2          # points of half s in the big coordinate
        fv = _lagrange_eval(x, f[s], q)   # f_s at the small coordinate eta = q
        for a in range(N + 1):
            b[a] += 0.5 * np.sum(w * fv * xi ** a)
            for c in range(N + 1):
                G[a, c] += 0.5 * np.sum(w * xi ** a * xi ** c)
    coef = np.linalg.solve(G, b)
    expect = np.polynomial.polynomial.polyval(x, coef)
    assert np.abs(got - expect).max() < 1e-10 * max(1.0, np.abs(expect).max())
    # the projection of the two restrictions of one polynomial gives it back
    I = sum(oracle.mortar(N, s, proj=True, nodes=kind) @ oracle.mortar(N, s, nodes=kind) for s in (0, 1))
    assert np.abs(I - np.eye(N + 1)).max() < 1e-13


@pytest.mark.parametrize("n", [2, 5, 7, 8])
def test_fv_mortar_matrices_are_sub_cell_overlaps(oracle, n):
    """M^FV: small sub-cell i of half s covers [(s n + i)/(2n), (s n + i + 1)/(2n)]
    of the unit big face, big sub-cell j covers [j/n, (j+1)/n]; interpolation =
    the big value of the cell containing the small one, projection = overlap
    length / big cell length (exact fractions)."""
    for s in (0, 1):
        Mi = oracle.mortar(n, s, fv=True)
        Mp = oracle.mortar(n, s, proj=True, fv=True)
        for i in range(n):
            a, b = Fraction(s * n + i, 2 * n), Fraction(s * n + i + 1, 2 * n)
            for j in range(n):
                lo, hi = Fraction(j, n), Fraction(j + 1, n)
                ov = max(Fraction(0), min(b, hi) - max(a, lo))
                assert Mi[i, j] == float(ov / (b - a))
                assert Mp[j, i] == float(ov / (hi - lo))
    I = sum(oracle.mortar(n, s, proj=True, fv=True) @ oracle.mortar(n, s, fv=True) for s in (0, 1))
    assert np.array_equal(I, np.eye(n))


# ---------------------------------------------------------------- meshes
def _all_types_chain():
    """Types 1 (y halved, big side left), 2 (z halved), 3 (both, big side right),
    and a conforming interface between domains of different x spacing."""
    return W.chain_domains([(2, 2, 2, 0.5), (2, 4, 2, 0.25), (1, 4, 4, 0.25), (2, 2, 2, 0.5)])


def _half_refined(k, L=1.0):
    """Sec. 4.1 / 4.2 layout on a Cartesian cube: the lower half in x at twice the
    resolution of the upper half (type-3 mortars on both x interfaces)."""
    return W.chain_domains([(k, 2 * k, 2 * k, L / 2), (k // 2, k, k, L / 2)], L=(L, L))


def test_chain_of_equal_domains_is_one_periodic_box(oracle):
    """Two equal domains glued along x give exactly the right-hand side of one
    periodic box with the same elements (random degrees and FV elements)."""
    sp = W.species_set([W.AIR, W.HELIUM], mu=2e-3)
    rng = np.random.default_rng(5)
    Nb = rng.integers(1, 5, (3, 3, 4)).astype(np.int8)     # [k, j, i]
    fb = (rng.random((3, 3, 4)) < 0.3).astype(np.uint8)
    one = W.make_problem([((4, 3, 3), (0, 0, 0), (1, 1, 1))], sp, n_fv=6, N=Nb.ravel(), fv=fb.ravel(), riemann=2)
    two = W.make_problem(W.chain_domains([(2, 3, 3, 0.5), (2, 3, 3, 0.5)]), sp, n_fv=6,
                         N=np.concatenate([Nb[:, :, :2].ravel(), Nb[:, :, 2:].ravel()]),
                         fv=np.concatenate([fb[:, :, :2].ravel(), fb[:, :, 2:].ravel()]), chain=1, riemann=2)
    R1 = oracle.eval_rhs(one, W.smooth_random_state(one, 3, amp=0.1))
    R2 = oracle.eval_rhs(two, W.smooth_random_state(two, 3, amp=0.1))
    off1, _ = W.offsets(one)
    off2, _ = W.offsets(two)
    _, _, c1, _ = W.element_index(one)
    _, _, c2, _ = W.element_index(two)
    where = {tuple(np.round(c, 9)): e for e, c in enumerate(c1)}
    n1 = W.points_per_dir(one)
    for e2 in range(len(c2)):
        e1 = where[tuple(np.round(c2[e2], 9))]
        m = 6 * int(n1[e1]) ** 3
        assert np.array_equal(R1[off1[e1]:off1[e1] + m], R2[off2[e2]:off2[e2] + m])


@pytest.mark.parametrize("riemann,nodes,split", [(0, 0, 0), (2, 0, 0), (1, 1, 1)])
def test_freestream_preserved_on_nonconforming_mesh(oracle, riemann, nodes, split):
    """Sec. 4.1: a uniform state on the half-refined cube with random degrees
    N in [2,5] and FV elements (N_FV = 8) stays uniform to the level of Table 1
    after 60 steps; the pattern is redrawn every 20 steps (random in space and
    time)."""
    rows = {l.split()[0]: [float(x) for x in l.split()[1:]] for l in open(GOLDEN) if l[0] != "#" and l.strip()}
    sp = W.species_set([W.AIR, W.HELIUM], mu=2e-3)
    doms = _half_refined(2, L=2.0)
    base = W.make_problem(doms, sp, n_fv=8, N=2, chain=1, riemann=riemann, nodes=nodes, split=split)
    ne = W.n_elements(base)
    U = None
    for rnd in range(3):
        prob = dict(base, N=W.random_degrees(ne, 2, 5, 11 + rnd), fv=W.random_fv(ne, 0.3, 11 + rnd))
        U0 = W.constant_state(prob, [0.7, 0.3], (1.0, 1.0, 1.0), 1.0)
        if rnd == 0:
            assert np.abs(oracle.eval_rhs(prob, U0)).max() < 5e-12
        U, _ = oracle.rk3(prob, U0, 20, cfl_c=0.9, cfl_v=0.9)
        err = _per_var(prob, U - U0)
        assert max(np.abs(e).max() for e in err) < 10 * max(rows["Linf"])


@pytest.mark.parametrize("nk,riemann,seed,nodes,split", [(2, 0, 1, 0, 0), (3, 1, 2, 0, 0), (3, 2, 3, 1, 0),
                                                          (2, 2, 4, 1, 1)])
def test_conservation_through_all_mortar_types(oracle, nk, riemann, seed, nodes, split):
    """Sum of J w R over DG nodes plus sub-cell volume x R over FV cells vanishes
    on a chain with mortars of types 1, 2 and 3 (big side on either side) and
    random hp/FV patterns: the L2 projection back to the big side keeps the face
    integral of the virtual sides' fluxes."""
    specs = [W.AIR, W.HELIUM, W.CO2][:nk]
    sp = W.species_set(specs, mu=2e-3)
    doms = _all_types_chain()
    ne = sum(int(np.prod(d[0])) for d in doms)
    prob = W.make_problem(doms, sp, n_fv=7, N=W.random_degrees(ne, 1, 6, seed), fv=W.random_fv(ne, 0.3, seed),
                          chain=1, riemann=riemann, nodes=nodes, split=split)
    U = W.smooth_random_state(prob, seed, amp=0.1)
    R = oracle.eval_rhs(prob, U)
    wts = _weights(prob)
    tot = [np.sum(r * w) for r, w in zip(_per_var(prob, R), _per_var(prob, wts))]
    scale = np.abs(R).max() * wts.sum() / W.n_vars(prob)
    assert max(abs(t) for t in tot) < 1e-14 * scale


# ---------------------------------------------------------------- convergence (Sec. 4.2)
def _mortar_l2(oracle, k, N_fine, N_coarse, fv_fine=None, T=0.05, n_fv=7, fv_coarse=None):
    """L2 error in rho_1 of the diagonal density wave of Sec. 4.2 after time T on
    the half-refined cube (k elements along x in the fine half); fv_fine /
    fv_coarse map element positions of the two halves to FV flags."""
    sp = W.species_set([W.AIR, W.HELIUM], mu=0.0)
    doms = _half_refined(k)
    base = W.make_problem(doms, sp, n_fv=n_fv, N=1, chain=1)
    dom, pos, _, _ = W.element_index(base)
    N = np.where(dom == 0, N_fine, N_coarse).astype(np.int8)
    fv = np.zeros(len(dom), np.uint8)
    pick = {0: fv_fine, 1: fv_coarse}
    fv = np.array([pick[d](*p) if pick[d] else 0 for d, p in zip(dom, pos)], np.uint8)
    prob = W.make_problem(doms, sp, n_fv=n_fv, N=N, fv=fv, chain=1)
    wave = (1, 1, 1)
    vel = (0.5, 0.5, 0.5)
    c = 1.5

    def fn_t(t):
        def fn(x, y, z):
            s = 2 * np.pi * (x + y + z - c * t)
            rho = 1 + 0.2 * np.sin(s)
            Y = 0.5 + 0.2 * np.cos(s)
            return [rho * Y, rho * (1 - Y)], vel, np.ones_like(x)
        return fn

    U0 = W.build_state(prob, fn_t(0.0))
    steps = int(np.ceil(T / (0.1 * (0.5 / k) / (2 * int(N.max()) + 1))))
    U, _ = oracle.rk3(prob, U0, steps, dt_fixed=T / steps)
    e = _per_var(prob, U - W.build_state(prob, fn_t(T)))[0]
    w = _per_var(prob, _weights(prob))[0]
    return np.sqrt((e ** 2 * w).sum() / w.sum())


def test_convergence_on_half_refined_cube():
    """Sec. 4.2 on the non-conforming cube: the error with the fine half at h and
    the coarse half at 2h lies between the errors of uniform meshes of h and 2h
    (a wrong quadrant or projection leaves an O(1) error at the mortars), and
    falls at least with order N when h halves."""
    import oracle as O
    N = 3
    e = [_mortar_l2(O, k, N, N) for k in (2, 4)]
    conf = [_advected_l2(O, (m, m, m), lambda i, j, k_: N, wave=(1, 1, 1)) for m in (2, 4, 8)]
    assert conf[1] < e[0] < conf[0], (e, conf)
    assert conf[2] < e[1] < conf[1], (e, conf)
    assert np.log2(e[0] / e[1]) > N - 0.1, e


def test_convergence_with_different_degrees_across_the_mortar():
    """Fine half N = 4, coarse half N = 2 (p- and h-non-conforming at once): the
    error stays below that of the uniform N = 2 mesh at the coarse spacing and
    falls with (at least) the pre-asymptotic order of N = 2 on these meshes."""
    import oracle as O
    e = [_mortar_l2(O, k, 4, 2) for k in (2, 4)]
    conf = [_advected_l2(O, (m, m, m), lambda i, j, k_: 2, wave=(1, 1, 1)) for m in (2, 4)]
    assert e[0] < conf[0] and e[1] < conf[1], (e, conf)
    assert np.log2(e[0] / e[1]) > 2.0, e


@pytest.mark.parametrize("half", ["fine", "coarse"])
def test_convergence_with_fv_elements_at_the_mortar(half):
    """FV elements (N_FV = 7) in a checkerboard in the fine half (FV small sides)
    or in the coarse half (FV big sides), DG N = 2 elsewhere: below the error of
    the conforming checkerboard at the coarse spacing, and the (pre-asymptotic)
    order of the FV scheme."""
    import oracle as O
    cb = lambda i, j, k_: (i + j + k_) % 2  # noqa: E731
    kw = {"fv_fine": cb} if half == "fine" else {"fv_coarse": cb}
    e = [_mortar_l2(O, k, 2, 2, **kw) for k in (2, 4)]
    conf = [_advected_l2(O, (m, m, m), lambda i, j, k_: 2, fv_of=cb, wave=(1, 1, 1)) for m in (2, 4)]
    assert e[0] < conf[0] and e[1] < conf[1], (e, conf)
    # the conforming checkerboard reaches 1.55 between these two spacings
    assert np.log2(e[0] / e[1]) > 1.5, e


# ---------------------------------------------------------------- viscous closed form
def _node_coords(prob):
    """x, y, z of every point of every element, in the state's point order."""
    _, _, corner, h = W.element_index(prob)
    n = W.points_per_dir(prob)
    out = []
    for e in range(len(n)):
        m = int(n[e])
        r = (_nodes(m, int(prob.get("nodes", 0))) + 1) / 2
        k, j, i = np.meshgrid(r, r, r, indexing="ij")
        out.append(np.stack([corner[e, 0] + h[e, 0] * i.ravel(), corner[e, 1] + h[e, 1] * j.ravel(),
                             corner[e, 2] + h[e, 2] * k.ravel()]))
    return out


def _shear_errors(oracle, N, mortar=True):
    mu, A, k2 = 2e-2, 0.05, 2 * np.pi
    sp = W.species_set([W.AIR, W.AIR], mu=mu)
    doms = _half_refined(2) if mortar else W.chain_domains([(2, 2, 2, 1.0)])
    prob = W.make_problem(doms, sp, n_fv=8, N=N, chain=1)
    Rg = sp["Rgas"][0]

    def vx(y, z):
        return A * np.sin(k2 * y + 0.3) * np.cos(k2 * z + 0.1)

    def fn(x, y, z):
        return [0.5 + 0 * x, 0.5 + 0 * x], (vx(y, z), 0 * x, 0 * x), np.ones_like(x) * Rg * 1.0

    U = W.build_state(prob, fn)
    R = oracle.eval_rhs(prob, U)
    off, _ = W.offsets(prob)
    n = W.points_per_dir(prob)
    err = {2: 0.0, 5: 0.0}
    scale = {2: 0.0, 5: 0.0}
    for e, (x, y, z) in enumerate(_node_coords(prob)):
        m3 = int(n[e]) ** 3
        blk = R[off[e]:off[e] + 6 * m3].reshape(6, m3)
        v = vx(y, z)
        vy = A * k2 * np.cos(k2 * y + 0.3) * np.cos(k2 * z + 0.1)
        vz = -A * k2 * np.sin(k2 * y + 0.3) * np.sin(k2 * z + 0.1)
        lap = -2 * k2 ** 2 * v
        exact = {2: mu * lap, 5: mu * (vy ** 2 + vz ** 2 + v * lap)}
        for q, ex in exact.items():
            err[q] = max(err[q], np.abs(blk[q] - ex).max())
            scale[q] = max(scale[q], np.abs(ex).max())
        for q in (0, 1, 3, 4):  # mass, y- and z-momentum: zero
            err.setdefault(("zero", q), 0.0)
            err[("zero", q)] = max(err[("zero", q)], np.abs(blk[q]).max())
    return {q: err[q] / scale[q] for q in (2, 5)}, max(v for q, v in err.items() if isinstance(q, tuple))


def test_viscous_shear_across_mortars_matches_closed_form(oracle):
    """v_x(y, z) at uniform density, pressure and temperature: R(rho v_x) =
    mu Lap v_x, R(rho E) = mu (|grad v_x|^2 + v_x Lap v_x), the rest 0.  The
    mortar planes cut across the shear, so the virtual-side lifting values and
    viscous fluxes enter.  R(rho v_x) converges spectrally in N; R(rho E)
    converges more slowly on any mesh (the discrete temperature gradient carries
    the interpolation error of |v|^2), so it is held to the error of the
    conforming mesh at the coarse half's spacing."""
    e5, z5 = _shear_errors(oracle, 5)
    e7, z7 = _shear_errors(oracle, 7)
    c5, _ = _shear_errors(oracle, 5, mortar=False)
    c7, _ = _shear_errors(oracle, 7, mortar=False)
    assert e7[2] < 2e-3 and e7[2] < 0.25 * e5[2], (e5, e7)
    assert e7[5] < 0.25 * e5[5], (e5, e7)
    assert e5[5] < 1.25 * c5[5] and e7[5] < 1.25 * c7[5], (e5, e7, c5, c7)
    assert z7 < 2e-4 and z7 < 0.2 * z5, (z5, z7)


def _fv_shear_error(oracle, k, n_fv=4, mu=20.0):
    """All-FV half-refined cube, v_y = A sin(2 pi x) across the mortar planes:
    max error of R(rho v_y) against mu v_y'' at the sub-cell centres (mu large,
    so that the numerical dissipation of the convective flux stays small next to
    the viscous term)."""
    A = 0.05
    sp = W.species_set([W.AIR, W.AIR], mu=mu)
    doms = _half_refined(k)
    prob = W.make_problem(doms, sp, n_fv=n_fv, N=2, fv=1, chain=1)
    Rg = sp["Rgas"][0]

    def fn(x, y, z):
        return [0.5 + 0 * x, 0.5 + 0 * x], (0 * x, A * np.sin(2 * np.pi * x), 0 * x), np.ones_like(x) * Rg

    R = oracle.eval_rhs(prob, W.build_state(prob, fn))
    off, _ = W.offsets(prob)
    _, _, corner, h = W.element_index(prob)
    c = (np.arange(n_fv) + 0.5) / n_fv
    err = 0.0
    for e in range(len(off)):
        m3 = n_fv ** 3
        x = corner[e, 0] + h[e, 0] * np.tile(c, n_fv * n_fv)
        blk = R[off[e]:off[e] + 6 * m3].reshape(6, m3)
        err = max(err, np.abs(blk[3] + mu * (2 * np.pi) ** 2 * A * np.sin(2 * np.pi * x)).max())
    return err / (mu * (2 * np.pi) ** 2 * A)


def test_fv_viscous_gradient_across_mortars_converges(oracle):
    """FV sub-cells on both sides of the mortars: the central-difference
    gradient across the interface uses the true distance between the sub-cell
    centres (l/2 (1 + h_nb/h) in the element's reference coordinates), so the
    viscous term converges across the 2:1 jump in spacing (first order there:
    a central difference on unequal spacing; second order on the conforming
    mesh).  Taking the distance as l instead makes the error grow with
    refinement."""
    e = [_fv_shear_error(oracle, k) for k in (2, 4)]
    assert e[1] < 0.6 * e[0] and e[1] < 0.15, e
