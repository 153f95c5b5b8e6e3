"""Pins of the oracle's per-element sub-cell variant: an FV element of degree N
has N+1 sub-cells per direction (the common-DOF scheme the paper sets itself
apart from, Sec. 1), so switching an element between DG and FV keeps its
number of DOFs.  A DG/FV face couples on the FV side's sub-cell grid
(Sec. 3.2.1: the DG side is transformed to the FV representation); where that
grid is coarser than the DG side's N+1 the map back, V^{FV->DG}, is the L2
projection of the sub-cell piecewise constant onto degree N (the
pseudo-inverse of a non-injective V^{DG->FV} would not keep constants).  Two FV
sides of different counts meet on the finer grid, the coarser side entering by
the exact overlaps of its sub-cells (piecewise-constant L2 projection).  The
1D brute-force comparison lives with the other brute-force checks
(tests/test_oracle_rhs.py)."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2502_19342_gb300 import workloads as W


def _overlap_exact(n_from, n_to):
    M = np.zeros((n_to, n_from))
    for i in range(n_to):
        for j in range(n_from):
            lo = max(Fraction(i, n_to), Fraction(j, n_from))
            hi = min(Fraction(i + 1, n_to), Fraction(j + 1, n_from))
            if hi > lo:
                M[i, j] = float((hi - lo) / Fraction(1, n_to))
    return M


@pytest.mark.parametrize("n_from", range(2, 10))
def test_overlap_maps_are_exact_fractions(oracle, n_from):
    for n_to in range(2, 10):
        M = oracle.fv_overlap(n_from, n_to)
        np.testing.assert_array_equal(M, _overlap_exact(n_from, n_to))
        # rows are averages (sum 1); the map back preserves integrals
        np.testing.assert_allclose(M.sum(1), 1.0, rtol=0, atol=1e-15)


@pytest.mark.parametrize("N", [2, 4, 6])
def test_coarse_fv_to_dg_map_is_the_l2_projection(oracle, N):
    """V^{FV->DG} from fewer than N+1 sub-cells: the L2 projection onto degree N
    of the piecewise constant, computed here from numpy's orthonormal Legendre
    series and Gauss rule (x: the element's LG nodes); it keeps constants and the
    integral."""
    x = np.polynomial.legendre.leggauss(N + 1)[0]
    for nf in range(1, N + 1):
        M = oracle.fv2dg(N, nf)
        assert M.shape == (N + 1, nf)
        q, wq = np.polynomial.legendre.leggauss(N + 2)
        ref = np.zeros((N + 1, nf))
        for s in range(nf):
            a, b = -1 + 2 * s / nf, -1 + 2 * (s + 1) / nf
            xs = a + (b - a) * (q + 1) / 2
            for m in range(N + 1):
                Pm = np.polynomial.legendre.Legendre.basis(m)
                c = np.sqrt((2 * m + 1) / 2) * np.dot(wq, Pm(xs)) * (b - a) / 2
                ref[:, s] += c * np.sqrt((2 * m + 1) / 2) * Pm(x)
        np.testing.assert_allclose(M, ref, rtol=0, atol=1e-13)
        np.testing.assert_allclose(M.sum(1), 1.0, rtol=0, atol=1e-13)
        wg = np.polynomial.legendre.leggauss(N + 1)[1]
        np.testing.assert_allclose(wg @ M, np.full(nf, 2.0 / nf), rtol=0, atol=1e-13)


def _problem(seed, nk=2, dims=(3, 3, 4), Nlo=1, Nhi=5, fv_frac=0.4, riemann=0, mu=2e-3, own=1, n_fv=2):
    sp = W.species_set([W.AIR, W.HELIUM, W.CO2][:nk], mu=mu)
    n = int(np.prod(dims))
    N = W.random_degrees(n, Nlo, Nhi, seed)
    fv = W.random_fv(n, fv_frac, seed)
    return W.make_problem([(dims, (0, 0, 0), (1.0, 0.9, 1.2))], sp, n_fv=n_fv, N=N, fv=fv, riemann=riemann,
                          fv_own_n=own)


@pytest.mark.parametrize("riemann", [0, 1, 2])
def test_uniform_degree_is_the_global_count_bit_for_bit(oracle, riemann):
    """With one degree N everywhere every FV element has N+1 sub-cells, which is
    the global variant with n_fv = N+1: R, the time step and the indicator agree
    bit for bit."""
    p_own = _problem(3, Nlo=3, Nhi=3, riemann=riemann)
    p_glob = dict(p_own, fv_own_n=0, n_fv=4)
    U = W.smooth_random_state(p_glob, 3, amp=0.1)
    np.testing.assert_array_equal(oracle.eval_rhs(p_own, U), oracle.eval_rhs(p_glob, U))
    np.testing.assert_array_equal(oracle.dt(p_own, U, 0.5, 0.5), oracle.dt(p_glob, U, 0.5, 0.5))
    a, b = oracle.indicator(p_own, U), oracle.indicator(p_glob, U)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("seed,nk,riemann", [(1, 2, 0), (2, 3, 1), (3, 2, 2), (4, 1, 0)])
def test_free_stream_with_per_element_sub_cells(oracle, seed, nk, riemann):
    """R(const) = 0 to round-off on random degrees 1..6 and FV elements: FV/FV
    faces between unequal counts, DG/FV faces with the FV side finer and coarser
    than the DG side's N+1."""
    prob = _problem(seed, nk=nk, Nlo=1, Nhi=6, riemann=riemann)
    rho = [0.5, 0.3, 0.2][:nk]
    U = W.constant_state(prob, rho, (0.7, -0.4, 0.25), 1.3)
    R = oracle.eval_rhs(prob, U)
    # the summed terms are (2/h) |Dhat| |F| ~ 10^2 .. 10^3 (N <= 6, h ~ 0.3):
    # round-off level is ~1e-14 of that
    _, _, _, h = W.element_index(prob)
    Fmax = np.abs(U).max() * 1.0 + 1.3
    term = 2.0 / h.min() * 2.0 * (int(prob["N"].max()) + 1) ** 2 * Fmax
    assert np.abs(R).max() < 1e-14 * term, (np.abs(R).max(), term)


def _weights(prob):
    """Quadrature weight x Jacobian of every DOF (DG: Gauss weights; FV: sub-cell volume)."""
    off, size = W.offsets(prob)
    _, _, _, h = W.element_index(prob)
    V = W.n_vars(prob)
    n = W.points_per_dir(prob)
    wts = np.zeros(size)
    for e in range(W.n_elements(prob)):
        m = int(n[e])
        if prob["fv"][e]:
            w3 = np.full(m ** 3, (2.0 / m) ** 3)
        else:
            w = np.polynomial.legendre.leggauss(m)[1]
            w3 = np.einsum("k,j,i->kji", w, w, w).ravel()
        J = np.prod(h[e]) / 8.0
        wts[off[e]:off[e] + V * m ** 3] = np.tile(w3 * J, V)
    return wts


@pytest.mark.parametrize("seed,nk,riemann", [(5, 2, 0), (6, 3, 1), (7, 2, 2)])
def test_conservation_with_per_element_sub_cells(oracle, seed, nk, riemann):
    """Every conserved variable's integral of R vanishes on the periodic mesh:
    the overlap maps and the DG/FV maps keep face integrals."""
    prob = _problem(seed, nk=nk, Nlo=1, Nhi=6, riemann=riemann)
    U = W.smooth_random_state(prob, seed, amp=0.15)
    R = oracle.eval_rhs(prob, U)
    wts = _weights(prob)
    off, _ = W.offsets(prob)
    V = W.n_vars(prob)
    n = W.points_per_dir(prob)
    for v in range(V):
        tot, mag = 0.0, 0.0
        for e in range(W.n_elements(prob)):
            m3 = int(n[e]) ** 3
            sl = slice(off[e] + v * m3, off[e] + (v + 1) * m3)
            tot += float(np.dot(wts[sl], R[sl]))
            mag += float(np.dot(wts[sl], np.abs(R[sl])))
        assert abs(tot) <= 1e-13 * mag, (v, tot, mag)


def test_switching_keeps_the_dofs_and_round_trips(oracle):
    """DG -> FV -> DG per element with N+1 sub-cells: the state size does not
    change, and V^{FV->DG} V^{DG->FV} = I (a square invertible map) returns the
    DG state."""
    prob = _problem(8, Nlo=1, Nhi=7, fv_frac=0.0)
    U = W.smooth_random_state(prob, 8, amp=0.2)
    rng = np.random.default_rng(8)
    sel = (rng.random(len(prob["N"])) < 0.5).astype(np.uint8)
    p_fv = dict(prob, fv=sel)
    U_fv = oracle.remap(prob, prob["N"], sel, U)
    assert U_fv.size == U.size == oracle.state_size(p_fv)
    U_back = oracle.remap(p_fv, prob["N"], np.zeros_like(sel), U_fv)
    np.testing.assert_allclose(U_back, U, rtol=0, atol=1e-13 * np.abs(U).max())


def test_rejected_with_chained_domains(oracle):
    sp = W.species_set([W.AIR, W.HELIUM], mu=1e-3)
    doms = W.chain_domains([(2, 2, 2, 0.5), (2, 2, 2, 0.5)])
    prob = W.make_problem(doms, sp, n_fv=4, N=2, chain=1, fv_own_n=1)
    with pytest.raises(RuntimeError):
        oracle.state_size(prob)


def _physical(prob, U):
    """Every density positive and every internal energy positive, at the nodes
    and sub-cells, and no value non-finite."""
    import oracle
    nk = len(prob["gamma"])
    V = nk + 4
    if not np.isfinite(U).all():
        return False
    off = [int(o) for o in oracle.elem_offsets(prob)] + [U.size]
    for e in range(len(prob["N"])):
        u = U[off[e]:off[e + 1]].reshape(V, -1)
        rho = u[:nk].sum(0)
        if (rho <= 0).any() or (u[nk + 3] - 0.5 * (u[nk:nk + 3] ** 2).sum(0) / rho <= 0).any():
            return False
    return True


def _shock_cycles(oracle, limiter, cycles, own=True):
    """The hp-mixed shock case (16^3 elements, N in 2..6, Mach 1.5 shock into a
    heavy-gas bubble) with per-element sub-cell counts: `cycles` times the
    indicator's adaptation and 5 SSP-RK3 steps at CFL 0.5.  Returns the number
    of steps that ended in a physical state."""
    prob, U = W.hp_shock(0, y_bg=0.01)
    prob = dict(prob, fv_own_n=int(own), pp_limiter=int(limiter))
    done = 0
    for _ in range(cycles):
        Ip, Ih = oracle.indicator(prob, U)
        N, fv = oracle.adapt_decide(prob, Ip, Ih, W.THRESHOLDS, 2, 6)
        U = oracle.remap(prob, N, fv, U)
        prob = dict(prob, N=N, fv=fv)
        for _ in range(5):
            U, _ = oracle.rk3(prob, U, 1, cfl_c=0.5, cfl_v=0.5)
            if not _physical(prob, U):
                return done
            done += 1
    return done


def test_shock_case_with_per_element_sub_cells_needs_the_positivity_limiter(oracle):
    """Per-element sub-cell counts let a DG element of degree N meet FV
    neighbours of fewer than N+1 sub-cells, whose coupling fluxes reach it as
    L2 projections of piecewise constants.  On the shock case a DG element at
    the expansion of the periodic wrap, fed so, gets face traces of negative
    pressure and the run turns non-finite within the first five cycles; the
    Zhang-Shu limiter (nodal and face-point positivity, Sec. 3.5) carries the
    same run through them.  With the global sub-cell count, N_FV = 7 >=
    N_max + 1, no such projection occurs and the case runs without the
    limiter."""
    assert _shock_cycles(oracle, limiter=False, cycles=5) < 25
    assert _shock_cycles(oracle, limiter=True, cycles=5) == 25
    assert _shock_cycles(oracle, limiter=False, cycles=5, own=False) == 25
