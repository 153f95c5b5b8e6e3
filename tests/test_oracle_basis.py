"""Pins of the oracle's reference-element operators (Sec. 3.1.1, 3.2, 3.4)
against closed forms and numpy's own polynomial routines."""
import numpy as np
import numpy.polynomial.legendre as npleg
import pytest

DEGREES = list(range(1, 8))


@pytest.mark.parametrize("N", DEGREES)
def test_nodes_weights_match_numpy_gauss_rule(oracle, N):
    b = oracle.basis(N)
    x, w = npleg.leggauss(N + 1)
    np.testing.assert_allclose(b["x"], x, atol=1e-15)
    np.testing.assert_allclose(b["w"], w, atol=1e-15)


@pytest.mark.parametrize("N", DEGREES)
def test_quadrature_exact_to_degree_2N_plus_1(oracle, N):
    b = oracle.basis(N)
    for k in range(0, 2 * N + 2):
        exact = (1 - (-1) ** (k + 1)) / (k + 1)
        assert abs(np.dot(b["w"], b["x"] ** k) - exact) < 1e-14


@pytest.mark.parametrize("N", DEGREES)
def test_derivative_matrix_exact_on_polynomials(oracle, N):
    b = oracle.basis(N)
    x = b["x"]
    for k in range(0, N + 1):
        dp = k * x ** (k - 1) if k > 0 else 0 * x
        np.testing.assert_allclose(b["D"] @ x ** k, dp, atol=1e-12)


@pytest.mark.parametrize("N", DEGREES)
def test_boundary_values_exact_on_polynomials(oracle, N):
    b = oracle.basis(N)
    for k in range(0, N + 1):
        assert abs(b["lp"] @ b["x"] ** k - 1.0) < 1e-13
        assert abs(b["lm"] @ b["x"] ** k - (-1.0) ** k) < 1e-13


@pytest.mark.parametrize("N", DEGREES)
def test_weak_derivative_reproduces_polynomial_derivative(oracle, N):
    """Dhat u + l_hat(1) u(1) - l_hat(-1) u(-1) is the exact derivative of any
    degree-N polynomial: integration by parts with exact LG quadrature.  This
    fixes the weight ratio of Dhat (Eq. 24) and the sign of the lifting
    surface terms (Eq. 23)."""
    b = oracle.basis(N)
    x, w = b["x"], b["w"]
    lhp, lhm = b["lp"] / w, b["lm"] / w
    for k in range(0, N + 1):
        u = x ** k
        du = b["Dhat"] @ u + lhp * 1.0 - lhm * (-1.0) ** k
        exact = k * x ** (k - 1) if k > 0 else 0 * x
        np.testing.assert_allclose(du, exact, atol=1e-11)


@pytest.mark.parametrize("N", DEGREES)
def test_dhat_row_sums_cancel_surface_terms(oracle, N):
    """Free-stream identity: sum_m Dhat_im = -(l_i(1) - l_i(-1)) / w_i."""
    b = oracle.basis(N)
    np.testing.assert_allclose(b["Dhat"].sum(1), -(b["lp"] - b["lm"]) / b["w"], atol=1e-12)


@pytest.mark.parametrize("N,M", [(a, c) for a in DEGREES for c in DEGREES if a < c])
def test_interpolation_up_is_exact(oracle, N, M):
    V = oracle.vmap(N, M)
    xN, xM = oracle.basis(N)["x"], oracle.basis(M)["x"]
    rng = np.random.default_rng(N * 10 + M)
    c = rng.standard_normal(N + 1)
    np.testing.assert_allclose(V @ np.polyval(c, xN), np.polyval(c, xM), atol=1e-12)


@pytest.mark.parametrize("N,M", [(a, c) for a in DEGREES for c in DEGREES if a > c])
def test_projection_down_equals_truncated_legendre_series(oracle, N, M):
    V = oracle.vmap(N, M)
    xN, xM = oracle.basis(N)["x"], oracle.basis(M)["x"]
    rng = np.random.default_rng(N * 10 + M)
    u = rng.standard_normal(N + 1)
    coef = npleg.legfit(xN, u, N)  # interpolating Legendre series
    np.testing.assert_allclose(V @ u, npleg.legval(xM, coef[:M + 1]), atol=1e-12)


@pytest.mark.parametrize("N,M", [(a, c) for a in DEGREES for c in DEGREES if a < c])
def test_project_after_interpolate_is_identity(oracle, N, M):
    np.testing.assert_allclose(oracle.vmap(M, N) @ oracle.vmap(N, M), np.eye(N + 1), atol=1e-12)


@pytest.mark.parametrize("N,nfv", [(N, nfv) for N in DEGREES for nfv in (N + 1, 8, 9)])
def test_dg_to_fv_is_subcell_mean(oracle, N, nfv):
    A = oracle.dg2fv(N, nfv)
    x = oracle.basis(N)["x"]
    rng = np.random.default_rng(N + 100 * nfv)
    c = rng.standard_normal(N + 1)
    P = np.polyint(c)
    edges = np.linspace(-1, 1, nfv + 1)
    means = (np.polyval(P, edges[1:]) - np.polyval(P, edges[:-1])) / (2.0 / nfv)
    np.testing.assert_allclose(A @ np.polyval(c, x), means, atol=1e-12)


@pytest.mark.parametrize("N,nfv", [(N, nfv) for N in DEGREES for nfv in (N + 1, 8, 9)])
def test_fv_to_dg_is_moore_penrose_inverse(oracle, N, nfv):
    A = oracle.dg2fv(N, nfv)
    X = oracle.fv2dg(N, nfv)
    np.testing.assert_allclose(A @ X @ A, A, atol=1e-12)
    np.testing.assert_allclose(X @ A @ X, X, atol=1e-11)
    np.testing.assert_allclose((A @ X).T, A @ X, atol=1e-12)
    np.testing.assert_allclose((X @ A).T, X @ A, atol=1e-12)
    np.testing.assert_allclose(X @ A, np.eye(N + 1), atol=1e-11)
    np.testing.assert_allclose(X, np.linalg.pinv(A), atol=1e-10)


@pytest.mark.parametrize("N,nfv", [(N, nfv) for N in DEGREES for nfv in (N + 1, 8, 9)])
def test_fv_to_dg_preserves_the_mean(oracle, N, nfv):
    """w^T V^{FV->DG} = l 1^T: the integral of the mapped polynomial equals the
    integral of the piecewise constants (conservation at DG/FV interfaces)."""
    w = oracle.basis(N)["w"]
    X = oracle.fv2dg(N, nfv)
    np.testing.assert_allclose(w @ X, np.full(nfv, 2.0 / nfv), atol=1e-13)


@pytest.mark.parametrize("N", DEGREES)
def test_legendre_vandermonde_orthonormal(oracle, N):
    b = oracle.basis(N)
    V = oracle.leg_vandermonde(N)
    np.testing.assert_allclose(V.T @ np.diag(b["w"]) @ V, np.eye(N + 1), atol=1e-13)
    # columns are sqrt((2m+1)/2) P_m
    for m in range(N + 1):
        e = np.zeros(m + 1)
        e[m] = 1
        np.testing.assert_allclose(V[:, m], np.sqrt((2 * m + 1) / 2) * npleg.legval(b["x"], e), atol=1e-13)
