"""Pin of the coupling between DG elements of different degree (Sec. 3.2.1,
Sec. 3.2.2) against a separate brute-force numpy implementation.

The state is chosen so that the full multi-component right-hand side reduces
exactly to a scalar linear operator: two identical species (same gamma, R, mu,
Pr, D), at rest, with uniform total density, pressure and temperature, and
only the composition varying.  Then every convective flux vanishes (or is the
constant p n), the stress, heat flux and diffusion enthalpy flux vanish, and
for the first partial density q = rho_1

    dq/dt = -div J_1,   J_1 = -D grad q,

discretised by BR1 (Eqs. 14a-14b, 19-23).  The face flux of q is
-D (g^- + g^+)/2 plus, with the local Lax-Friedrichs flux, the penalty
-c (q^+ - q^-)/2 (the Roe flux adds nothing at a contact at rest).

The brute force below writes this scalar scheme in the strong form (interior
derivative D q plus the jump between the face value and the element's own
trace, lifted by l_i(+-1)/w_i), which equals the oracle's weak form for
exact quadrature, and applies the paper's p-coupling rules literally:
  - BR1 lifting value on the lower degree: the higher side's trace L2-projected
    onto min(N, N~), averaged, and interpolated back to the higher side;
  - face flux on the higher degree: the lower side's traces of q and g
    interpolated to max(N, N~) points, the flux evaluated there, and
    L2-projected back onto the lower side.
A swap of min and max in either rule changes R at the level of the
projection error of the non-polynomial test field and fails this pin.
Operators come from numpy's Gauss-Legendre rule and product-form Lagrange
polynomials.
"""
import numpy as np
import pytest

from paper_2502_19342_gb300 import workloads as W


def _lagrange(nodes, x):
    """L[a, j] = l_j(x_a) for the Lagrange polynomials of `nodes`."""
    x = np.atleast_1d(np.asarray(x, float))
    L = np.ones((len(x), len(nodes)))
    for j in range(len(nodes)):
        for m in range(len(nodes)):
            if m != j:
                L[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return L


def _dlagrange(nodes):
    """Dm[a, j] = l_j'(x_a), by differentiating the product form."""
    n = len(nodes)
    Dm = np.zeros((n, n))
    for j in range(n):
        for a in range(n):
            s = 0.0
            for m in range(n):
                if m == j:
                    continue
                term = 1.0 / (nodes[j] - nodes[m])
                for l in range(n):
                    if l != j and l != m:
                        term *= (nodes[a] - nodes[l]) / (nodes[j] - nodes[l])
                s += term
            Dm[a, j] = s
    return Dm


class _Ops:
    def __init__(self, n):
        self.x, self.w = np.polynomial.legendre.leggauss(n)
        self.D = _dlagrange(self.x)
        self.lm = _lagrange(self.x, -1.0)[0]
        self.lp = _lagrange(self.x, 1.0)[0]


def _interp(na, nb):
    """Interpolation of degree na-1 data on na Gauss points to nb Gauss points."""
    xa = np.polynomial.legendre.leggauss(na)[0]
    xb = np.polynomial.legendre.leggauss(nb)[0]
    return _lagrange(xa, xb)


def _project(nb, na):
    """L2 projection of degree nb-1 data on nb Gauss points onto degree na-1
    (na < nb): M_a^{-1} int l^a_i l^b_j, both integrals exact on nb points."""
    xa, wa = np.polynomial.legendre.leggauss(na)
    xb, wb = np.polynomial.legendre.leggauss(nb)
    return (_lagrange(xa, xb).T * wb[None, :]) / wa[:, None]


def _map2(A, F):
    return A @ F @ A.T


def _to(n_from, n_to, F):
    if n_from == n_to:
        return F
    return _map2(_interp(n_from, n_to) if n_to > n_from else _project(n_from, n_to), F)


def _trace(q, d, side, op):
    """Face values of the element array q[k, j, i] at xi_d = side (+-1)."""
    l = op.lp if side > 0 else op.lm
    axis = 2 - d
    return np.tensordot(q, l, axes=([axis], [0]))


def _apply_dir(q, d, M):
    """Apply the matrix M along direction d of q[k, j, i]."""
    axis = 2 - d
    return np.moveaxis(np.tensordot(M, q, axes=([1], [axis])), 0, axis)


def _lift_face(q, d, side, op, val):
    """Strong-form surface term along d: l_i(side)/w_i times the face array val."""
    l = (op.lp if side > 0 else op.lm) / op.w
    axis = 2 - d
    shape = [1, 1, 1]
    shape[axis] = len(l)
    return np.expand_dims(val, axis) * l.reshape(shape)


def brute_force_rhs(dims, h, Ns, q, Dcoef, c_llf, mode="paper"):
    """R of dq/dt = div(D grad q) by BR1 on a periodic Cartesian mesh with a
    degree per element.  mode "paper": lifting on min, flux on max degree;
    "swapped": the opposite (for the check that the pin can fail)."""
    nx, ny, nz = dims
    ne = nx * ny * nz
    n = [int(N) + 1 for N in Ns]
    ops = {m: _Ops(m) for m in set(n)}

    def nb(e, d):
        i, j, k = e % nx, (e // nx) % ny, e // (nx * ny)
        p = [i, j, k]
        p[d] = (p[d] + 1) % dims[d]
        return p[0] + nx * (p[1] + ny * p[2])

    # BR1 lifting values per element face: ustar[e][(d, side)]
    ustar = [dict() for _ in range(ne)]
    for e in range(ne):
        for d in range(3):
            f = nb(e, d)
            qa = _trace(q[e], d, +1, ops[n[e]])
            qb = _trace(q[f], d, -1, ops[n[f]])
            nc = min(n[e], n[f]) if mode == "paper" else max(n[e], n[f])
            s = 0.5 * (_to(n[e], nc, qa) + _to(n[f], nc, qb))
            ustar[e][(d, +1)] = _to(nc, n[e], s)
            ustar[f][(d, -1)] = _to(nc, n[f], s)
    # gradient g^d = (2/h_d)[D q + surface jumps], strong form
    g = []
    for e in range(ne):
        op = ops[n[e]]
        ge = []
        for d in range(3):
            gd = _apply_dir(q[e], d, op.D)
            gd = gd + _lift_face(q[e], d, +1, op, ustar[e][(d, +1)] - _trace(q[e], d, +1, op))
            gd = gd - _lift_face(q[e], d, -1, op, ustar[e][(d, -1)] - _trace(q[e], d, -1, op))
            ge.append(gd * (2.0 / h[d]))
        g.append(ge)
    # face fluxes of F = -D g (in +x_d), with the LLF penalty
    fstar = [dict() for _ in range(ne)]
    for e in range(ne):
        for d in range(3):
            f = nb(e, d)
            nc = max(n[e], n[f]) if mode == "paper" else min(n[e], n[f])
            qa = _to(n[e], nc, _trace(q[e], d, +1, ops[n[e]]))
            qb = _to(n[f], nc, _trace(q[f], d, -1, ops[n[f]]))
            ga = _to(n[e], nc, _trace(g[e][d], d, +1, ops[n[e]]))
            gb = _to(n[f], nc, _trace(g[f][d], d, -1, ops[n[f]]))
            F = -Dcoef * 0.5 * (ga + gb) - 0.5 * c_llf * (qb - qa)
            fstar[e][(d, +1)] = _to(nc, n[e], F)
            fstar[f][(d, -1)] = _to(nc, n[f], F)
    R = []
    for e in range(ne):
        op = ops[n[e]]
        Re = np.zeros_like(q[e])
        for d in range(3):
            Fd = -Dcoef * g[e][d]
            div = _apply_dir(Fd, d, op.D)
            div = div + _lift_face(Fd, d, +1, op, fstar[e][(d, +1)] - _trace(Fd, d, +1, op))
            div = div - _lift_face(Fd, d, -1, op, fstar[e][(d, -1)] - _trace(Fd, d, -1, op))
            Re = Re - div * (2.0 / h[d])
        R.append(Re)
    return R


def _problem(dims, L, Ns, riemann):
    sp = W.species_set([W.AIR, W.AIR], mu=2e-2, Pr=0.72, Sc=0.8)
    return W.make_problem([(dims, (0, 0, 0), L)], sp, n_fv=4, N=np.array(Ns, np.int8), riemann=riemann)


def _state(prob, L):
    rho0, p0 = 1.3, 0.9

    def fn(x, y, z):
        Y = (0.5 + 0.25 * np.sin(2 * np.pi * x / L[0] + 0.7) * np.cos(2 * np.pi * y / L[1] - 0.3)
             + 0.15 * np.sin(4 * np.pi * z / L[2] + 0.2) * np.cos(2 * np.pi * x / L[0]))
        return [rho0 * Y, rho0 * (1.0 - Y)], (0.0, 0.0, 0.0), np.full(x.shape, p0)

    return W.build_state(prob, fn), np.sqrt(1.4 * p0 / rho0)


@pytest.mark.parametrize("riemann", [0, 1])
@pytest.mark.parametrize("dims,Ns", [((2, 1, 1), (2, 5)), ((3, 2, 2), (2, 5, 3, 4, 5, 2, 3, 2, 4, 5, 2, 3))])
def test_p_interface_coupling_matches_brute_force(oracle, riemann, dims, Ns):
    L = (1.5, 1.0, 0.8)
    prob = _problem(dims, L, Ns, riemann)
    U, c = _state(prob, L)
    R = oracle.eval_rhs(prob, U)
    off, _ = W.offsets(prob)
    V = 6
    q, Ro = [], []
    for e, N in enumerate(Ns):
        n = N + 1
        blk = U[off[e]:off[e] + V * n ** 3].reshape(V, n, n, n)
        q.append(blk[0].copy())
        Ro.append(R[off[e]:off[e] + V * n ** 3].reshape(V, n, n, n))
    h = [L[d] / dims[d] for d in range(3)]
    Dk = float(prob["Dk"][0])
    c_llf = c if riemann == 0 else 0.0
    Rb = brute_force_rhs(dims, h, Ns, q, Dk, c_llf)
    scale = max(np.abs(r).max() for r in Rb)
    err = max(np.abs(Ro[e][0] - Rb[e]).max() for e in range(len(Ns)))
    assert err < 1e-12 * scale, (err, scale)
    # the other fields: rho_2 mirrors rho_1; momentum and energy stay at rest
    for e in range(len(Ns)):
        np.testing.assert_allclose(Ro[e][1], -Ro[e][0], rtol=0, atol=1e-12 * scale)
        assert np.abs(Ro[e][2:]).max() < 1e-11 * scale
    # the swapped rule differs from the paper's by far more than the tolerance
    Rs = brute_force_rhs(dims, h, Ns, q, Dk, c_llf, mode="swapped")
    assert max(np.abs(Rs[e] - Rb[e]).max() for e in range(len(Ns))) > 1e-6 * scale


def test_brute_force_reduces_to_textbook_on_uniform_degree():
    """The brute force on a uniform degree with a separable sine field: BR1
    with central fluxes is consistent, so R -> D lap q spectrally (a check of
    the brute force itself, independent of the oracle)."""
    L = (1.0, 1.0, 1.0)
    dims = (3, 3, 3)
    errs = []
    for N in (3, 5, 7):
        n = N + 1
        x = np.polynomial.legendre.leggauss(n)[0]
        q = []
        for e in range(27):
            i, j, k = e % 3, (e // 3) % 3, e // 9
            X = (i + (x + 1) / 2) / 3
            Y = (j + (x + 1) / 2) / 3
            Z = (k + (x + 1) / 2) / 3
            zz, yy, xx = np.meshgrid(Z, Y, X, indexing="ij")
            q.append(np.sin(2 * np.pi * xx) * np.cos(2 * np.pi * yy) + 0.5 * np.sin(2 * np.pi * zz))
        R = brute_force_rhs(dims, [1 / 3] * 3, [N] * 27, q, 0.1, 0.0)
        err = 0.0
        for e in range(27):
            i, j, k = e % 3, (e // 3) % 3, e // 9
            X = (i + (x + 1) / 2) / 3
            Y = (j + (x + 1) / 2) / 3
            Z = (k + (x + 1) / 2) / 3
            zz, yy, xx = np.meshgrid(Z, Y, X, indexing="ij")
            lap = -0.1 * 4 * np.pi ** 2 * (2 * np.sin(2 * np.pi * xx) * np.cos(2 * np.pi * yy)
                                           + 0.5 * np.sin(2 * np.pi * zz))
            err = max(err, np.abs(R[e] - lap).max())
        errs.append(err)
    scale = 0.1 * 4 * np.pi ** 2 * 2.5
    assert errs[0] < 0.15 * scale and errs[1] < errs[0] / 10 and errs[2] < errs[1] / 10, errs
