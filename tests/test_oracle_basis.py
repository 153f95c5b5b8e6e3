"""Pins of the oracle's reference-element operators (Sec. 3.1.1, 3.2, 3.4, and
the LGL nodes of the split form, Sec. 3.5) against closed forms and numpy's own
polynomial routines.  nodes = 0: Legendre-Gauss, 1: Legendre-Gauss-Lobatto."""
import numpy as np
import numpy.polynomial.legendre as npleg
import pytest

from paper_2502_19342_gb300 import workloads as W

DEGREES = list(range(1, 8))
NODES = [0, 1]


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


@pytest.mark.parametrize("nodes", NODES)
@pytest.mark.parametrize("N", DEGREES)
def test_derivative_matrix_exact_on_polynomials(oracle, N, nodes):
    b = oracle.basis(N, nodes)
    x = b["x"]
    for k in range(0, N + 1):
        dp = k * x ** (k - 1) if k > 0 else 0 * x
        np.testing.assert_allclose(b["D"] @ x ** k, dp, atol=1e-12)


@pytest.mark.parametrize("nodes", NODES)
@pytest.mark.parametrize("N", DEGREES)
def test_boundary_values_exact_on_polynomials(oracle, N, nodes):
    b = oracle.basis(N, nodes)
    for k in range(0, N + 1):
        assert abs(b["lp"] @ b["x"] ** k - 1.0) < 1e-13
        assert abs(b["lm"] @ b["x"] ** k - (-1.0) ** k) < 1e-13


@pytest.mark.parametrize("nodes", NODES)
@pytest.mark.parametrize("N", DEGREES)
def test_weak_derivative_reproduces_polynomial_derivative(oracle, N, nodes):
    """Dhat u + l_hat(1) u(1) - l_hat(-1) u(-1) is the exact derivative of any
    degree-N polynomial: integration by parts with exact LG quadrature.  This
    fixes the weight ratio of Dhat (Eq. 24) and the sign of the lifting
    surface terms (Eq. 23)."""
    b = oracle.basis(N, nodes)
    x, w = b["x"], b["w"]
    lhp, lhm = b["lp"] / w, b["lm"] / w
    for k in range(0, N + 1):
        u = x ** k
        du = b["Dhat"] @ u + lhp * 1.0 - lhm * (-1.0) ** k
        exact = k * x ** (k - 1) if k > 0 else 0 * x
        np.testing.assert_allclose(du, exact, atol=1e-11)


@pytest.mark.parametrize("nodes", NODES)
@pytest.mark.parametrize("N", DEGREES)
def test_dhat_row_sums_cancel_surface_terms(oracle, N, nodes):
    """Free-stream identity: sum_m Dhat_im = -(l_i(1) - l_i(-1)) / w_i."""
    b = oracle.basis(N, nodes)
    np.testing.assert_allclose(b["Dhat"].sum(1), -(b["lp"] - b["lm"]) / b["w"], atol=1e-12)


@pytest.mark.parametrize("nodes", NODES)
@pytest.mark.parametrize("N,M", [(a, c) for a in DEGREES for c in DEGREES if a < c])
def test_interpolation_up_is_exact(oracle, N, M, nodes):
    V = oracle.vmap(N, M, nodes)
    xN, xM = oracle.basis(N, nodes)["x"], oracle.basis(M, nodes)["x"]
    rng = np.random.default_rng(N * 10 + M)
    c = rng.standard_normal(N + 1)
    np.testing.assert_allclose(V @ np.polyval(c, xN), np.polyval(c, xM), atol=1e-12)


@pytest.mark.parametrize("nodes", NODES)
@pytest.mark.parametrize("N,M", [(a, c) for a in DEGREES for c in DEGREES if a > c])
def test_projection_down_equals_truncated_legendre_series(oracle, N, M, nodes):
    V = oracle.vmap(N, M, nodes)
    xN, xM = oracle.basis(N, nodes)["x"], oracle.basis(M, nodes)["x"]
    rng = np.random.default_rng(N * 10 + M)
    u = rng.standard_normal(N + 1)
    coef = npleg.legfit(xN, u, N)  # interpolating Legendre series
    np.testing.assert_allclose(V @ u, npleg.legval(xM, coef[:M + 1]), atol=1e-12)


@pytest.mark.parametrize("nodes", NODES)
@pytest.mark.parametrize("N,M", [(a, c) for a in DEGREES for c in DEGREES if a < c])
def test_project_after_interpolate_is_identity(oracle, N, M, nodes):
    np.testing.assert_allclose(oracle.vmap(M, N, nodes) @ oracle.vmap(N, M, nodes), np.eye(N + 1), atol=1e-12)


@pytest.mark.parametrize("nodes", NODES)
@pytest.mark.parametrize("N,nfv", [(N, nfv) for N in DEGREES for nfv in (N + 1, 8, 9)])
def test_dg_to_fv_is_subcell_mean(oracle, N, nfv, nodes):
    A = oracle.dg2fv(N, nfv, nodes)
    x = oracle.basis(N, nodes)["x"]
    rng = np.random.default_rng(N + 100 * nfv)
    c = rng.standard_normal(N + 1)
    P = np.polyint(c)
    edges = np.linspace(-1, 1, nfv + 1)
    means = (np.polyval(P, edges[1:]) - np.polyval(P, edges[:-1])) / (2.0 / nfv)
    np.testing.assert_allclose(A @ np.polyval(c, x), means, atol=1e-12)


@pytest.mark.parametrize("nodes", NODES)
@pytest.mark.parametrize("N,nfv", [(N, nfv) for N in DEGREES for nfv in (N + 1, 8, 9)])
def test_fv_to_dg_is_moore_penrose_inverse(oracle, N, nfv, nodes):
    A = oracle.dg2fv(N, nfv, nodes)
    X = oracle.fv2dg(N, nfv, nodes)
    np.testing.assert_allclose(A @ X @ A, A, atol=1e-12)
    np.testing.assert_allclose(X @ A @ X, X, atol=1e-11)
    np.testing.assert_allclose((A @ X).T, A @ X, atol=1e-12)
    np.testing.assert_allclose((X @ A).T, X @ A, atol=1e-12)
    np.testing.assert_allclose(X @ A, np.eye(N + 1), atol=1e-11)
    np.testing.assert_allclose(X, np.linalg.pinv(A), atol=1e-10)


@pytest.mark.parametrize("nodes", NODES)
@pytest.mark.parametrize("N,nfv", [(N, nfv) for N in DEGREES for nfv in (N + 1, 8, 9)])
def test_fv_to_dg_preserves_the_mean(oracle, N, nfv, nodes):
    """w^T V^{FV->DG} = l 1^T: the integral of the mapped polynomial equals the
    integral of the piecewise constants (conservation at DG/FV interfaces)."""
    w = oracle.basis(N, nodes)["w"]
    X = oracle.fv2dg(N, nfv, nodes)
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


# ---------------------------------------------------------------- LGL nodes (Sec. 3.5)
@pytest.mark.parametrize("N", DEGREES)
def test_lgl_nodes_are_the_endpoints_and_the_roots_of_the_legendre_derivative(oracle, N):
    b = oracle.basis(N, 1)
    np.testing.assert_allclose(b["x"], W.lgl_nodes(N + 1), atol=1e-15)


@pytest.mark.parametrize("N", DEGREES)
def test_lgl_quadrature_exact_to_degree_2N_minus_1_and_not_2N(oracle, N):
    """Exactness up to degree N alone fixes the weights of given nodes."""
    w, x = oracle.basis(N, 1)["w"], oracle.basis(N, 1)["x"]
    for k in range(0, 2 * N):
        exact = (1 - (-1) ** (k + 1)) / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14
    assert abs(np.dot(w, x ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-5


@pytest.mark.parametrize("N", DEGREES)
def test_lgl_summation_by_parts(oracle, N):
    """W D + (W D)^T = B = diag(-1, 0, .., 0, 1) and Dhat = D - W^{-1} B: the
    weak form on LGL nodes is the strong form with a boundary correction."""
    b = oracle.basis(N, 1)
    Q = np.diag(b["w"]) @ b["D"]
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[N, N] = -1.0, 1.0
    np.testing.assert_allclose(Q + Q.T, B, atol=1e-13)
    np.testing.assert_allclose(b["Dhat"], b["D"] - np.diag(1.0 / b["w"]) @ B, atol=1e-12)
    np.testing.assert_array_equal(b["lm"], np.eye(N + 1)[0])
    np.testing.assert_array_equal(b["lp"], np.eye(N + 1)[N])


@pytest.mark.parametrize("N", DEGREES)
def test_lgl_legendre_vandermonde_discrete_norms(oracle, N):
    """The LGL rule is exact for the products of two modes except the top mode
    with itself: V^T W V = diag(1, .., 1, (2N+1)/N)."""
    b = oracle.basis(N, 1)
    V = oracle.leg_vandermonde(N, 1)
    G = np.eye(N + 1)
    G[N, N] = (2 * N + 1) / N
    np.testing.assert_allclose(V.T @ np.diag(b["w"]) @ V, G, atol=1e-13)
