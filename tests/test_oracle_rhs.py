"""Pins of the oracle's right-hand side R(U) (Sec. 3.1-3.4) against what the
paper and the mathematics fix: free-stream preservation (Sec. 4.1, Table 1),
discrete conservation, a brute-force one-dimensional DG/FV code, the N+1
convergence order (Sec. 4.2), viscous closed forms, the SSP-RK3 stability
polynomial, the modal indicator on synthetic spectra and the remap identities."""
import os

import numpy as np
import pytest

from paper_2502_19342_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "freestream_table.txt")


def _dg_weights(n, nodes):
    """Quadrature weights of n DG nodes: numpy's Gauss rule (LG), or for LGL the
    weights that make the rule exact up to degree n-1 on the LGL points
    (a Vandermonde solve)."""
    if nodes == 0:
        return np.polynomial.legendre.leggauss(n)[1]
    x = W.lgl_nodes(n)
    mom = np.array([(1 - (-1) ** (k + 1)) / (k + 1) for k in range(n)])
    return np.linalg.solve(np.vander(x, n, increasing=True).T, mom)


def _weights(prob):
    """Quadrature weight x Jacobian of every DOF (DG: weights of the node family; FV: sub-cell volume)."""
    off, size = W.offsets(prob)
    _, _, _, h = W.element_index(prob)
    V = W.n_vars(prob)
    wts = np.zeros(size)
    for e in range(W.n_elements(prob)):
        if prob["fv"][e]:
            m = int(prob["n_fv"])
            w3 = np.full(m ** 3, (2.0 / m) ** 3)
        else:
            m = int(prob["N"][e]) + 1
            w = _dg_weights(m, int(prob.get("nodes", 0)))
            w3 = np.einsum("k,j,i->kji", w, w, w).ravel()
        J = np.prod(h[e]) / 8.0
        wts[off[e]:off[e] + V * m ** 3] = np.tile(w3 * J, V)
    return wts


def _per_var(prob, x):
    off, _ = W.offsets(prob)
    V = W.n_vars(prob)
    n = W.points_per_dir(prob)
    out = [[] for _ in range(V)]
    for e in range(len(off)):
        m3 = int(n[e]) ** 3
        blk = x[off[e]:off[e] + V * m3].reshape(V, m3)
        for v in range(V):
            out[v].append(blk[v])
    return [np.concatenate(o) for o in out]


def _mixed_problem(seed, nk=2, nel=(3, 3, 3), Nlo=1, Nhi=5, fv_frac=0.3, n_fv=6, riemann=0, mu=2e-3,
                   box=(1.0, 1.0, 1.0), nodes=0, split=0):
    specs = [W.AIR, W.HELIUM, W.CO2][:nk]
    sp = W.species_set(specs, mu=mu)
    n = nel[0] * nel[1] * nel[2]
    N = W.random_degrees(n, Nlo, Nhi, seed)
    fv = W.random_fv(n, fv_frac, seed)
    return W.make_problem([(nel, (0, 0, 0), box)], sp, n_fv=n_fv, N=N, fv=fv, riemann=riemann, nodes=nodes,
                          split=split)


# ---------------------------------------------------------------- free stream
def test_golden_freestream_table_parses():
    rows = {l.split()[0]: [float(x) for x in l.split()[1:]] for l in open(GOLDEN) if l[0] != "#" and l.strip()}
    assert len(rows["L2"]) == 5 and len(rows["Linf"]) == 5
    assert max(rows["Linf"]) < 1e-13


@pytest.mark.parametrize("riemann,nodes,split", [(0, 0, 0), (1, 0, 0), (2, 0, 0), (0, 1, 0), (1, 1, 1)])
def test_freestream_preserved_on_random_hp_fv_pattern(oracle, riemann, nodes, split):
    """Sec. 4.1: a uniform state stays uniform to round-off after 180 steps on a
    random distribution of degrees N in [2,5] and FV elements (N_FV = 8).  The
    errors must stay at the level the paper reports in Table 1 (scaled by the
    state's magnitude, which is O(1) in both)."""
    rows = {l.split()[0]: [float(x) for x in l.split()[1:]] for l in open(GOLDEN) if l[0] != "#" and l.strip()}
    prob = _mixed_problem(3, nel=(3, 3, 3), Nlo=2, Nhi=5, fv_frac=0.3, n_fv=8, riemann=riemann, nodes=nodes,
                          split=split)
    U0 = W.constant_state(prob, [0.7, 0.3], (1.0, 1.0, 1.0), 1.0)
    R = oracle.eval_rhs(prob, U0)
    assert np.abs(R).max() < 5e-12
    U, dts = oracle.rk3(prob, U0, 180, cfl_c=0.9, cfl_v=0.9)
    wts = _weights(prob)
    vol = wts.sum() / W.n_vars(prob)
    err = _per_var(prob, U - U0)
    ww = _per_var(prob, wts)
    l2 = [np.sqrt((e ** 2 * w).sum() / vol) for e, w in zip(err, ww)]
    linf = [np.abs(e).max() for e in err]
    assert max(l2) < 10 * max(rows["L2"]), l2
    assert max(linf) < 10 * max(rows["Linf"]), linf


# ---------------------------------------------------------------- conservation
@pytest.mark.parametrize("nk,riemann,seed,nodes,split", [(2, 0, 1, 0, 0), (3, 1, 2, 0, 0), (2, 1, 4, 0, 0),
                                                          (3, 0, 5, 0, 0), (3, 2, 6, 0, 0), (3, 1, 7, 1, 0),
                                                          (3, 0, 8, 1, 1), (2, 2, 9, 1, 1)])
def test_discrete_conservation_periodic(oracle, nk, riemann, seed, nodes, split):
    """Sum of J w R over DG nodes plus sub-cell volume x R over FV cells vanishes
    for every conserved variable on a periodic mesh, through p- and DG/FV
    interfaces (the L2 projection and the pseudo-inverse preserve face integrals)."""
    prob = _mixed_problem(seed, nk=nk, nel=(3, 4, 3), Nlo=1, Nhi=6, fv_frac=0.3, n_fv=7, riemann=riemann,
                          box=(1.0, 1.3, 0.8), nodes=nodes, split=split)
    U = W.smooth_random_state(prob, seed, amp=0.1)
    R = oracle.eval_rhs(prob, U)
    wts = _weights(prob)
    tot = [np.sum(r * w) for r, w in zip(_per_var(prob, R), _per_var(prob, wts))]
    scale = np.abs(R).max() * wts.sum() / W.n_vars(prob)
    assert max(abs(t) for t in tot) < 1e-14 * scale


def test_flux_choice_per_face_type(oracle):
    """Sec. 5.1: Roe-HH between DG elements, local Lax-Friedrichs wherever FV
    data meet (FV sub-cell faces, FV/FV and DG/FV faces).  An element's R uses
    only its own faces, so on a mixed pattern the result equals the all-Roe
    result on every DG element with six DG neighbours and the all-LLF result
    on every FV element with six FV neighbours; elements on the DG/FV border
    differ from both."""
    nel = (4, 4, 3)
    prob = _mixed_problem(7, nk=3, nel=nel, Nlo=1, Nhi=5, fv_frac=0.35, n_fv=6)
    U = W.smooth_random_state(prob, 7, amp=0.15)
    R = {k: oracle.eval_rhs(dict(prob, riemann=k), U) for k in (0, 1, 2)}
    _, pos, _, _ = W.element_index(prob)
    lin = {tuple(p): e for e, p in enumerate(pos)}
    off, _ = W.offsets(prob)
    size = np.diff(np.append(off, R[2].size))
    fv = prob["fv"]
    n_in = {0: 0, 1: 0, "border": 0}
    for e, p in enumerate(pos):
        nb = [lin[tuple((p + s * np.eye(3, dtype=int)[d]) % nel)] for d in range(3) for s in (-1, 1)]
        sl = slice(off[e], off[e] + size[e])
        if not fv[e] and not any(fv[q] for q in nb):
            np.testing.assert_array_equal(R[2][sl], R[1][sl])
            n_in[1] += 1
        elif fv[e] and all(fv[q] for q in nb):
            np.testing.assert_array_equal(R[2][sl], R[0][sl])
            n_in[0] += 1
        elif not fv[e]:
            assert np.abs(R[2][sl] - R[1][sl]).max() > 0 and np.abs(R[2][sl] - R[0][sl]).max() > 0
            n_in["border"] += 1
    assert n_in[1] > 0 and n_in["border"] > 0
    # all-DG and all-FV patterns reduce to the single solvers
    dg = dict(prob, fv=np.zeros_like(fv), riemann=2)
    Udg = W.smooth_random_state(dg, 8, amp=0.15)
    np.testing.assert_array_equal(oracle.eval_rhs(dg, Udg), oracle.eval_rhs(dict(dg, riemann=1), Udg))
    allfv = dict(prob, fv=np.ones_like(fv), riemann=2)
    Ufv = W.smooth_random_state(allfv, 9, amp=0.15)
    np.testing.assert_array_equal(oracle.eval_rhs(allfv, Ufv), oracle.eval_rhs(dict(allfv, riemann=0), Ufv))


# ---------------------------------------------------------------- 1D brute force
def _cons_to_w(prob, u):
    nk = len(prob["gamma"])
    cv = prob["Rgas"] / (prob["gamma"] - 1)
    cp = prob["gamma"] * cv
    rho = u[:nk].sum(0)
    kap = (u[:nk].T @ cp) / (u[:nk].T @ cv)
    v = u[nk:nk + 3] / rho
    p = (kap - 1) * (u[nk + 3] - 0.5 * rho * (v ** 2).sum(0))
    return np.concatenate([u[:nk], v, p[None]])


def _w_to_cons(prob, w):
    nk = len(prob["gamma"])
    cv = prob["Rgas"] / (prob["gamma"] - 1)
    cp = prob["gamma"] * cv
    rho = w[:nk].sum(0)
    kap = (w[:nk].T @ cp) / (w[:nk].T @ cv)
    v = w[nk:nk + 3]
    return np.concatenate([w[:nk], rho * v, (w[nk + 3] / (kap - 1) + 0.5 * rho * (v ** 2).sum(0))[None]])


def _minmod(a, b):
    return np.where(a * b <= 0, 0.0, np.where(np.abs(a) <= np.abs(b), a, b))


def _rhs_1d(oracle, prob, chain, u, h, axis, own=False):
    """Brute-force 1D hybrid DG/FV operator on a periodic chain of elements.
    chain[e] = (N, fv); u[e] is (V, n) nodal values / cell means along `axis`.
    own: an FV element of degree N has N+1 sub-cells (else n_fv); the centre
    distance to an FV neighbour with another count is 1/n + 1/n_nb."""
    K = len(chain)
    V = len(prob["gamma"]) + 4
    nf_of = [(N + 1 if own else int(prob["n_fv"])) for N, _ in chain]
    B = {}
    for N, fv in chain:
        if not fv and N not in B:
            B[N] = oracle.basis(N)

    def flux(uu, gg):
        g3 = np.zeros(3 * V)
        g3[axis * V:(axis + 1) * V] = gg
        Fc, Fv = oracle.flux(prob, uu, g3, axis)
        return Fc + Fv

    def vflux(uu, gg):
        g3 = np.zeros(3 * V)
        g3[axis * V:(axis + 1) * V] = gg
        return oracle.flux(prob, uu, g3, axis)[1]

    left, right = [], []   # face values of each element (DG trace / FV boundary mean)
    for e, (N, fv) in enumerate(chain):
        if fv:
            left.append(u[e][:, 0]); right.append(u[e][:, -1])
        else:
            left.append(u[e] @ B[N]["lm"]); right.append(u[e] @ B[N]["lp"])
    rec_l, rec_r, g_l, g_r, div = {}, {}, {}, {}, {}
    for e, (N, fv) in enumerate(chain):
        if not fv:
            continue
        em, ep = (e - 1) % K, (e + 1) % K
        nfv = nf_of[e]
        l = 2.0 / nfv
        # neighbour sub-cell mean next to the face: FV cell, or V^{DG->FV} of the DG solution
        wl = right[em] if chain[em][1] else (oracle.dg2fv(chain[em][0], nfv) @ u[em].T)[-1]
        wr = left[ep] if chain[ep][1] else (oracle.dg2fv(chain[ep][0], nfv) @ u[ep].T)[0]
        dl = l if not chain[em][1] or nf_of[em] == nfv else 1.0 / nfv + 1.0 / nf_of[em]
        dr = l if not chain[ep][1] or nf_of[ep] == nfv else 1.0 / nfv + 1.0 / nf_of[ep]
        ext = np.concatenate([wl[:, None], u[e], wr[:, None]], axis=1)
        dist_l = np.array([dl] + [l] * (nfv - 1))
        dist_r = np.array([l] * (nfv - 1) + [dr])
        W_ = _cons_to_w(prob, ext)
        s = _minmod((W_[:, 1:-1] - W_[:, :-2]) / dist_l, (W_[:, 2:] - W_[:, 1:-1]) / dist_r)
        wm = _w_to_cons(prob, W_[:, 1:-1] - s * l / 2)
        wp = _w_to_cons(prob, W_[:, 1:-1] + s * l / 2)
        grad = (ext[:, 2:] - ext[:, :-2]) / (dist_l + dist_r) * (2.0 / h)
        d = np.zeros((V, nfv))
        for c in range(nfv - 1):
            F = oracle.riemann(prob, wp[:, c], wm[:, c + 1], axis) + 0.5 * (
                vflux(wp[:, c], grad[:, c]) + vflux(wm[:, c + 1], grad[:, c + 1]))
            d[:, c] += nfv / h * F
            d[:, c + 1] -= nfv / h * F
        div[e] = d
        rec_l[e], rec_r[e], g_l[e], g_r[e] = wm[:, 0], wp[:, -1], grad[:, 0], grad[:, -1]
    ustar_l, ustar_r = {}, {}
    for e, (N, fv) in enumerate(chain):
        if fv:
            continue
        em, ep = (e - 1) % K, (e + 1) % K
        ol = rec_r[em] if chain[em][1] else right[em]
        orr = rec_l[ep] if chain[ep][1] else left[ep]
        ustar_l[e] = 0.5 * (left[e] + ol)
        ustar_r[e] = 0.5 * (right[e] + orr)
    for e, (N, fv) in enumerate(chain):
        if fv:
            continue
        b = B[N]
        lhp, lhm = b["lp"] / b["w"], b["lm"] / b["w"]
        g = (2.0 / h) * (u[e] @ b["Dhat"].T + np.outer(ustar_r[e], lhp) - np.outer(ustar_l[e], lhm))
        F = np.stack([flux(u[e][:, i], g[:, i]) for i in range(N + 1)], axis=1)
        div[e] = (2.0 / h) * (F @ b["Dhat"].T)
        g_l[e], g_r[e] = g @ b["lm"], g @ b["lp"]
    for e, (N, fv) in enumerate(chain):
        ep = (e + 1) % K
        uL = rec_r[e] if fv else right[e]
        uR = rec_l[ep] if chain[ep][1] else left[ep]
        F = oracle.riemann(prob, uL, uR, axis) + 0.5 * (vflux(uL, g_r[e]) + vflux(uR, g_l[ep]))
        if fv:
            div[e][:, -1] += nf_of[e] / h * F
        else:
            b = B[N]
            div[e] += (2.0 / h) * np.outer(F, b["lp"] / b["w"])
        N2, fv2 = chain[ep]
        if fv2:
            div[ep][:, 0] -= nf_of[ep] / h * F
        else:
            b = B[N2]
            div[ep] -= (2.0 / h) * np.outer(F, b["lm"] / b["w"])
    return [-div[e] for e in range(K)]


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("riemann", [0, 1])
def test_matches_brute_force_1d_code(oracle, axis, riemann):
    """Data varying along one axis only: the 3D operator equals a separate 1D
    DG/FV code (traces, lifting, surface terms, minmod reconstruction,
    central-difference gradients and DG/FV coupling), along x, y and z."""
    chain = [(3, 0), (2, 1), (4, 0), (4, 0), (5, 1), (2, 0)]
    K = len(chain)
    sp = W.species_set([W.AIR, W.HELIUM], mu=3e-3)
    dims = [1, 1, 1]
    dims[axis] = K
    hi = [0.7, 0.7, 0.7]
    hi[axis] = 1.2
    N = np.array([c[0] for c in chain], np.int8)
    fv = np.array([c[1] for c in chain], np.uint8)
    prob = W.make_problem([(tuple(dims), (0, 0, 0), tuple(hi))], sp, n_fv=6, N=N, fv=fv, riemann=riemann)
    L = hi[axis]

    def fn(x, y, z):
        s = (x, y, z)[axis] / L
        Y1 = 0.5 + 0.3 * np.sin(2 * np.pi * s)
        rho = 1.0 + 0.2 * np.cos(2 * np.pi * s + 0.3)
        v = [0.1 + 0 * s, -0.2 + 0 * s, 0.15 + 0 * s]
        v[axis] = 0.4 + 0.2 * np.sin(2 * np.pi * s + 1.0)
        v[(axis + 1) % 3] = 0.3 * np.cos(2 * np.pi * s)
        return [rho * Y1, rho * (1 - Y1)], v, 1.0 + 0.1 * np.sin(2 * np.pi * s + 2.0)

    U = W.build_state(prob, fn)
    R = oracle.eval_rhs(prob, U)
    off, _ = W.offsets(prob)
    V = 6
    h = L / K
    u1, r3 = [], []
    for e, (Ne, f) in enumerate(chain):
        n = 6 if f else Ne + 1
        blk = U[off[e]:off[e] + V * n ** 3].reshape(V, n, n, n)  # [v][k][j][i]
        rb = R[off[e]:off[e] + V * n ** 3].reshape(V, n, n, n)
        sl = [0, 0, 0]
        if axis == 0:
            u1.append(blk[:, 0, 0, :]); r3.append(rb)
        elif axis == 1:
            u1.append(blk[:, 0, :, 0]); r3.append(rb)
        else:
            u1.append(blk[:, :, 0, 0]); r3.append(rb)
        del sl
    R1 = _rhs_1d(oracle, prob, chain, u1, h, axis)
    scale = max(np.abs(r).max() for r in R1)
    for e in range(K):
        r1 = R1[e]
        # broadcast the 1D result over the two transverse directions
        if axis == 0:
            ref = np.broadcast_to(r1[:, None, None, :], r3[e].shape)
        elif axis == 1:
            ref = np.broadcast_to(r1[:, None, :, None], r3[e].shape)
        else:
            ref = np.broadcast_to(r1[:, :, None, None], r3[e].shape)
        np.testing.assert_allclose(r3[e], ref, atol=1e-11 * scale, rtol=0)


@pytest.mark.parametrize("axis", [0, 2])
@pytest.mark.parametrize("riemann", [0, 1])
def test_per_element_sub_cells_match_brute_force_1d_code(oracle, axis, riemann):
    """The per-element sub-cell variant (an FV element of degree N has N+1
    sub-cells, Sec. 1) with data along one axis: FV/FV faces between unequal
    counts (centre distance 1/n + 1/n_nb), FV elements coarser and finer than
    their DG neighbours' N+1, against the 1D brute-force code."""
    chain = [(3, 0), (2, 1), (5, 1), (4, 0), (1, 1), (2, 1), (6, 0), (3, 1)]
    K = len(chain)
    sp = W.species_set([W.AIR, W.HELIUM], mu=3e-3)
    dims = [1, 1, 1]
    dims[axis] = K
    hi = [0.7, 0.7, 0.7]
    hi[axis] = 1.6
    N = np.array([c[0] for c in chain], np.int8)
    fv = np.array([c[1] for c in chain], np.uint8)
    prob = W.make_problem([(tuple(dims), (0, 0, 0), tuple(hi))], sp, n_fv=2, N=N, fv=fv, riemann=riemann,
                          fv_own_n=1)
    L = hi[axis]

    def fn(x, y, z):
        s = (x, y, z)[axis] / L
        Y1 = 0.5 + 0.3 * np.sin(2 * np.pi * s)
        rho = 1.0 + 0.2 * np.cos(2 * np.pi * s + 0.3)
        v = [0.1 + 0 * s, -0.2 + 0 * s, 0.15 + 0 * s]
        v[axis] = 0.4 + 0.2 * np.sin(2 * np.pi * s + 1.0)
        v[(axis + 1) % 3] = 0.3 * np.cos(2 * np.pi * s)
        return [rho * Y1, rho * (1 - Y1)], v, 1.0 + 0.1 * np.sin(2 * np.pi * s + 2.0)

    U = W.build_state(prob, fn)
    R = oracle.eval_rhs(prob, U)
    off, _ = W.offsets(prob)
    V = 6
    h = L / K
    u1, r3 = [], []
    for e, (Ne, f) in enumerate(chain):
        n = Ne + 1
        blk = U[off[e]:off[e] + V * n ** 3].reshape(V, n, n, n)
        r3.append(R[off[e]:off[e] + V * n ** 3].reshape(V, n, n, n))
        u1.append(blk[:, 0, 0, :] if axis == 0 else blk[:, :, 0, 0])
    R1 = _rhs_1d(oracle, prob, chain, u1, h, axis, own=True)
    scale = max(np.abs(r).max() for r in R1)
    for e in range(K):
        r1 = R1[e]
        ref = np.broadcast_to(r1[:, None, None, :] if axis == 0 else r1[:, :, None, None], r3[e].shape)
        np.testing.assert_allclose(r3[e], ref, atol=1e-11 * scale, rtol=0)


def test_all_fv_mesh_is_a_plain_muscl_scheme(oracle):
    """All elements FV and data along x: the operator is a uniform periodic 1D
    MUSCL-minmod scheme on K*N_FV cells (element boundaries are invisible)."""
    K, nfv = 4, 5
    chain = [(2, 1)] * K
    sp = W.species_set([W.AIR, W.HELIUM], mu=0.0)
    prob = W.make_problem([((K, 1, 1), (0, 0, 0), (1, 0.5, 0.5))], sp, n_fv=nfv, N=2, fv=1)

    def fn(x, y, z):
        Y1 = 0.5 + 0.4 * np.sin(2 * np.pi * x)
        return [Y1, (1 - Y1) * 0.5], (0.3 + 0 * x, 0 * x, 0 * x), 1.0 + 0.2 * np.cos(2 * np.pi * x)

    U = W.build_state(prob, fn)
    R = oracle.eval_rhs(prob, U)
    V = 6
    n3 = nfv ** 3
    cells = np.concatenate([U[e * V * n3:(e + 1) * V * n3].reshape(V, nfv, nfv, nfv)[:, 0, 0, :] for e in range(K)], axis=1)
    Rc = np.concatenate([R[e * V * n3:(e + 1) * V * n3].reshape(V, nfv, nfv, nfv)[:, 0, 0, :] for e in range(K)], axis=1)
    M = K * nfv
    dx = 1.0 / M
    w = _cons_to_w(prob, cells)
    s = _minmod(w - np.roll(w, 1, axis=1), np.roll(w, -1, axis=1) - w)
    wl = _w_to_cons(prob, w + 0.5 * s)  # left state of face i+1/2
    wr = _w_to_cons(prob, np.roll(w - 0.5 * s, -1, axis=1))
    F = np.stack([oracle.riemann(prob, wl[:, i], wr[:, i], 0) for i in range(M)], axis=1)
    ref = -(F - np.roll(F, 1, axis=1)) / dx
    np.testing.assert_allclose(Rc, ref, atol=1e-12 * np.abs(ref).max())


# ---------------------------------------------------------------- species closure
def test_sum_of_species_equations_is_continuity(oracle):
    """Two identical species in a spatially varying split: sum_k R(rho_k) equals
    R(rho) of the single-species problem, i.e. sum_k J_k = 0 holds discretely.
    DG elements only: the minmod limiter acts on each partial density, which
    is not additive, so FV elements reconstruct the sum differently."""
    sp1 = W.species_set([W.AIR], mu=4e-3)
    sp2 = W.species_set([W.AIR, W.AIR], mu=4e-3)
    N = W.random_degrees(27, 2, 4, 8)
    fv = np.zeros(27, np.uint8)
    p1 = W.make_problem([((3, 3, 3), (0, 0, 0), (1, 1, 1))], sp1, n_fv=5, N=N, fv=fv)
    p2 = W.make_problem([((3, 3, 3), (0, 0, 0), (1, 1, 1))], sp2, n_fv=5, N=N, fv=fv)

    def f2(x, y, z):
        rho = 1 + 0.1 * np.sin(2 * np.pi * (x + y))
        Y = 0.5 + 0.3 * np.cos(2 * np.pi * (y - z))
        return [rho * Y, rho * (1 - Y)], (0.2 + 0.1 * np.sin(2 * np.pi * z), -0.1 + 0 * x, 0.3 + 0 * x), 1 + 0.1 * np.cos(2 * np.pi * x)

    U2 = W.build_state(p2, f2)
    U1 = W.build_state(p1, lambda x, y, z: ([sum(f2(x, y, z)[0])], f2(x, y, z)[1], f2(x, y, z)[2]))
    R1 = oracle.eval_rhs(p1, U1)
    R2 = oracle.eval_rhs(p2, U2)
    v1, v2 = _per_var(p1, R1), _per_var(p2, R2)
    scale = np.abs(R1).max()
    np.testing.assert_allclose(v2[0] + v2[1], v1[0], atol=1e-12 * scale)
    for a, b in zip(v2[2:], v1[1:]):
        np.testing.assert_allclose(a, b, atol=1e-12 * scale)


# ---------------------------------------------------------------- viscous closed forms
def _viscous_errors(oracle, N):
    sp = W.species_set([W.AIR, W.AIR], mu=2e-2)
    prob = W.make_problem([((4, 1, 1), (0, 0, 0), (1, 0.5, 0.5))], sp, n_fv=8, N=N)
    A = 0.05
    k = 2 * np.pi
    mu = 2e-2
    Rg = sp["Rgas"][0]
    g = sp["gamma"][0]
    cv = Rg / (g - 1)
    cp = g * cv
    lam = mu * cp / 0.72
    T0 = 1.0 / Rg

    def fn(x, y, z):
        T = T0 * (1 + A * np.sin(k * x))
        rho = 1.0 / (Rg * T)
        Y = 0.5 + A * np.cos(k * x)
        return [rho * Y, rho * (1 - Y)], (0 * x, A * np.sin(k * x), 0 * x), np.ones_like(x)

    U = W.build_state(prob, fn)
    R = oracle.eval_rhs(prob, U)
    V, n = 6, N + 1
    xg = (np.polynomial.legendre.leggauss(n)[0] + 1) / 2
    x = np.concatenate([(e + xg) / 4 for e in range(4)])
    Rx = np.concatenate([R[e * V * n ** 3:(e + 1) * V * n ** 3].reshape(V, n, n, n)[:, 0, 0, :] for e in range(4)],
                        axis=1)
    T = T0 * (1 + A * np.sin(k * x))
    Tx = T0 * A * k * np.cos(k * x)
    Txx = -T0 * A * k ** 2 * np.sin(k * x)
    rho = 1 / (Rg * T)
    rhox = -Tx / (Rg * T ** 2)
    Yx = -A * k * np.sin(k * x)
    Yxx = -A * k ** 2 * np.cos(k * x)
    vy = A * np.sin(k * x)
    vyx = A * k * np.cos(k * x)
    vyxx = -A * k ** 2 * np.sin(k * x)
    exact = {
        3: mu * vyxx,                                  # momentum y: (mu v_y')'
        0: mu * (rhox * Yx + rho * Yxx),               # species 1: (rho D Y')', D = mu
        1: -mu * (rhox * Yx + rho * Yxx),              # species 2
        5: lam * Txx + mu * (vyx ** 2 + vy * vyxx),    # energy: (lambda T')' + (v_y mu v_y')'
    }
    return {v: np.abs(Rx[v] - ex).max() / np.abs(ex).max() for v, ex in exact.items()}


def test_viscous_terms_converge_to_analytic_derivatives(oracle):
    """At rest with smooth profiles along x, R tends spectrally to the analytic
    right-hand sides: shear (mu v_y')', heat conduction (lambda T')' with the
    work of the viscous stress, and Fickian species diffusion."""
    e5 = _viscous_errors(oracle, 5)
    e7 = _viscous_errors(oracle, 7)
    for v in e7:
        assert e7[v] < 2e-3, (v, e7[v])
        assert e7[v] < 0.2 * e5[v], (v, e5[v], e7[v])


# ---------------------------------------------------------------- convergence order
def _advected_l2(oracle, nel, N_of, fv_of=None, wave=(1, 0, 0), T=0.05, n_fv=7, nodes=0, split=0):
    """L2 error in rho_1 of an advected density/species wave (Euler limit)
    after time T; nel = elements per direction, N_of/fv_of map element
    positions (i, j, k) to the degree / FV flag (checkerboards)."""
    sp = W.species_set([W.AIR, W.HELIUM], mu=0.0)
    dims = tuple(nel)
    _, pos, _, _ = W.element_index(W.make_problem([(dims, (0, 0, 0), (1, 1, 1))], sp, n_fv=n_fv, N=1))
    N = np.array([N_of(*p) for p in pos], np.int8)
    fv = np.array([fv_of(*p) if fv_of else 0 for p in pos], np.uint8)
    hi = tuple(1.0 if wave[a] else 1.0 / nel[a] for a in range(3))
    prob = W.make_problem([(dims, (0, 0, 0), hi)], sp, n_fv=n_fv, N=N, fv=fv, nodes=nodes, split=split)
    vel = tuple(0.5 * wv for wv in wave)
    c = 0.5 * sum(wv * wv for wv in wave)

    def fn_t(t):
        def fn(x, y, z):
            s = 2 * np.pi * (wave[0] * x + wave[1] * y + wave[2] * z - c * t)
            rho = 1 + 0.2 * np.sin(s)
            Y = 0.5 + 0.2 * np.cos(s)
            return [rho * Y, rho * (1 - Y)], vel, np.ones_like(x)
        return fn

    U0 = W.build_state(prob, fn_t(0.0))
    hmin = 1.0 / max(nel)
    steps = int(np.ceil(T / (0.1 * hmin / (2 * int(N.max()) + 1))))
    U, _ = oracle.rk3(prob, U0, steps, dt_fixed=T / steps)
    Ue = W.build_state(prob, fn_t(T))
    e = _per_var(prob, U - Ue)[0]
    w = _per_var(prob, _weights(prob))[0]
    return np.sqrt((e ** 2 * w).sum() / w.sum())


def _order(e1, e2, k1, k2):
    return np.log(e1 / e2) / np.log(k2 / k1)


def test_convergence_uniform_degree_2():
    """Sec. 4.2: order N+1 = 3 (wave along x on an extruded mesh)."""
    import oracle as O
    e = [_advected_l2(O, (k, 1, 1), lambda i, j, k_: 2) for k in (32, 64)]
    assert _order(e[0], e[1], 32, 64) > 2.65, e


def test_convergence_uniform_degree_3_diagonal_wave():
    """Sec. 4.2 setup: the wave travels along [1,1,1] on a 3D mesh; order N+1 = 4."""
    import oracle as O
    e = [_advected_l2(O, (k, k, k), lambda i, j, k_: 3, wave=(1, 1, 1)) for k in (4, 6)]
    assert _order(e[0], e[1], 4, 6) > 3.65, e


@pytest.mark.parametrize("Ns,nels,wave,expect", [
    ((2, 4), (32, 64), (1, 0, 0), 2.65),   # limited by the lowest degree: 3, not 5
    ((3, 5), (8, 16), (1, 1, 0), 3.65),    # 4, not 6
])
def test_convergence_checkerboard_degrees(Ns, nels, wave, expect):
    """Sec. 4.2: checkerboard degrees; the order is that of the lowest degree
    present (and clearly below that of the highest)."""
    import oracle as O
    dims = [tuple(k if wave[a] else 1 for a in range(3)) for k in nels]
    e = [_advected_l2(O, tuple(d), lambda i, j, k_: Ns[(i + j + k_) % 2], wave=wave) for d in dims]
    order = _order(e[0], e[1], nels[0], nels[1])
    assert expect < order < Ns[1] + 1 - 0.5, (e, order)


def test_convergence_hybrid_dg_fv_checkerboard():
    """Sec. 4.2: N = 2 DG elements and N_FV = 7 FV elements in a checkerboard
    converge with the second order of the FV scheme (the paper's figure)."""
    import oracle as O
    e = [_advected_l2(O, (k, 1, 1), lambda i, j, k_: 2, fv_of=lambda i, j, k_: i % 2) for k in (32, 64)]
    assert _order(e[0], e[1], 32, 64) > 1.8, e


# ---------------------------------------------------------------- time stepping
def test_ssp_rk3_stability_polynomial(oracle):
    for z in (-0.3, -1.0, -2.4, 0.5):
        u = oracle.rk3_scalar_linear(z, 1.0, 1.0)
        assert abs(u - (1 + z + z * z / 2 + z ** 3 / 6)) < 1e-15


def test_time_step_of_uniform_state(oracle):
    sp = W.species_set([W.AIR], mu=1e-3)
    prob = W.make_problem([((2, 2, 2), (0, 0, 0), (1, 2, 4))], sp, n_fv=5, N=3, fv=np.array([0, 1] * 4, np.uint8))
    U = W.constant_state(prob, [1.0], (0.5, -0.25, 0.1), 1.0)
    dt, dtc, dtv = oracle.dt(prob, U, 0.5, 0.4)
    c = np.sqrt(1.4)
    h = np.array([0.5, 1.0, 2.0])
    lam_dg = ((np.abs([0.5, -0.25, 0.1]) + c) / h).sum()
    lam_fv = ((np.abs([0.5, -0.25, 0.1]) + c) / (h / 5)).sum()
    dtc_ref = min(0.5 / (lam_dg * 7), 0.5 / lam_fv)
    dv = max(4 / 3 * 1e-3, 1.4 * 1e-3 / 0.72, 1e-3)
    dtv_ref = min(0.4 / (dv * (1 / h ** 2).sum() * 7), 0.4 / (dv * (25 / h ** 2).sum()))
    assert abs(dtc - dtc_ref) < 1e-15 * dtc_ref
    assert abs(dtv - dtv_ref) < 1e-14 * dtv_ref
    assert abs(dt - 1 / (1 / dtc_ref + 1 / dtv_ref)) < 1e-14 * dt


# ---------------------------------------------------------------- indicator
@pytest.mark.parametrize("N,sigma", [(3, 1.7), (5, 0.6), (7, 3.3), (1, 2.0)])
def test_indicator_recovers_exponential_decay_rate(oracle, N, sigma):
    """rho(x) = sum_m a_m L_m(x) with a_m^2 = exp(-sigma m) along x only: the
    modal energies decay exactly like exp(-sigma m), so I(rho) = sigma; p and
    Y are uniform, so I_h is large."""
    sp = W.species_set([W.AIR, W.HELIUM], mu=0.0)
    prob = W.make_problem([((1, 1, 1), (0, 0, 0), (1, 1, 1))], sp, n_fv=8, N=N)
    # orthonormal amplitude a_m multiplies sqrt((2m+1)/2) P_m
    coef = np.array([np.sqrt(np.exp(-sigma * m)) * np.sqrt((2 * m + 1) / 2) for m in range(N + 1)])

    def fn(x, y, z):
        xi = 2 * x - 1
        rho = np.polynomial.legendre.legval(xi, coef) + 3.0
        return [0.6 * rho, 0.4 * rho], (0 * x, 0 * x, 0 * x), np.ones_like(x)

    # the constant 3.0 adds to mode 0; correct the expected fit accordingly
    U = W.build_state(prob, fn)
    Ip, Ih = oracle.indicator(prob, U)
    a = coef / np.sqrt([(2 * m + 1) / 2 for m in range(N + 1)])
    a[0] += 3.0 * np.sqrt(2.0)  # the constant 3 = 3 sqrt(2) times the orthonormal mode 0
    w = a ** 2 / (a ** 2).sum()
    m = np.arange(N + 1)
    y = np.log(w)
    slope = ((m - m.mean()) * (y - y.mean())).sum() / ((m - m.mean()) ** 2).sum()
    assert abs(Ip[0] - abs(slope)) < 1e-10
    assert Ih[0] > 4  # uniform p and Y: all higher modes at the energy floor


def test_indicator_pure_exponential_spectrum(oracle):
    sp = W.species_set([W.AIR, W.HELIUM], mu=0.0)
    N, sigma = 4, 2.5
    prob = W.make_problem([((1, 1, 1), (0, 0, 0), (1, 1, 1))], sp, n_fv=8, N=N)
    amp = np.sqrt(np.exp(-sigma * np.arange(N + 1))) * 0.01

    def fn(x, y, z):
        xi = 2 * z - 1  # along z this time
        norm = np.array([np.sqrt((2 * m + 1) / 2) for m in range(N + 1)])
        p = 1.0 + np.polynomial.legendre.legval(xi, amp * norm) - amp[0] * norm[0] + amp[0] * norm[0]
        return [0.5 + 0 * x, 0.5 + 0 * x], (0 * x, 0 * x, 0 * x), p

    U = W.build_state(prob, fn)
    Ip, Ih = oracle.indicator(prob, U)
    assert Ip[0] > 10  # density uniform (round-off only)
    # pressure has mode 0 = 1*sqrt(2) + amp0*norm0... check against the direct fit
    a = amp.copy()
    a[0] = np.sqrt(2.0) + amp[0]
    w = a ** 2 / (a ** 2).sum()
    y = np.log(w)
    m = np.arange(N + 1)
    slope = ((m - m.mean()) * (y - y.mean())).sum() / ((m - m.mean()) ** 2).sum()
    assert abs(Ih[0] - abs(slope)) < 1e-9


def test_adapt_decision_rule(oracle):
    sp = W.species_set([W.AIR, W.HELIUM], mu=0.0)
    N = np.array([3, 3, 3, 3, 1, 7, 4, 4], np.int8)
    fv = np.array([0, 0, 0, 0, 0, 0, 1, 1], np.uint8)
    prob = W.make_problem([((8, 1, 1), (0, 0, 0), (1, 1, 1))], sp, n_fv=8, N=N, fv=fv)
    thr = (1.0, 1.6, 3.0, 7.0)
    Ih = np.array([0.5, 5.0, 5.0, 5.0, 5.0, 5.0, 1.2, 2.0])
    Ip = np.array([0.1, 2.0, 8.0, 5.0, 8.0, 2.0, 2.0, 2.0])
    Nn, fn = oracle.adapt_decide(prob, Ip, Ih, thr, 1, 7)
    assert list(fn) == [1, 0, 0, 0, 0, 0, 1, 0]
    assert list(Nn) == [3, 4, 2, 3, 1, 7, 4, 4]


# ---------------------------------------------------------------- remap
def test_remap_identities(oracle):
    sp = W.species_set([W.AIR, W.HELIUM], mu=0.0)
    prob = W.make_problem([((2, 2, 1), (0, 0, 0), (1, 1, 0.5))], sp, n_fv=7, N=np.array([2, 3, 4, 5], np.int8))
    U = W.smooth_random_state(prob, 4)
    # up then down: identity
    up = np.array([3, 4, 5, 6], np.int8)
    U1 = oracle.remap(prob, up, prob["fv"], U)
    p_up = dict(prob, N=up)
    U2 = oracle.remap(p_up, prob["N"], prob["fv"], U1)
    np.testing.assert_allclose(U2, U, atol=1e-12)
    # DG -> FV -> DG: identity (the pseudo-inverse is a left inverse)
    fv1 = np.ones(4, np.uint8)
    Uf = oracle.remap(prob, prob["N"], fv1, U)
    p_fv = dict(prob, fv=fv1)
    Ub = oracle.remap(p_fv, prob["N"], prob["fv"], Uf)
    np.testing.assert_allclose(Ub, U, atol=1e-11)
    # DG -> FV preserves each element's integral
    wd = _weights(prob)
    wf = _weights(p_fv)
    np.testing.assert_allclose(sum(_per_var(prob, U * wd)[0]), sum(_per_var(p_fv, Uf * wf)[0]), rtol=1e-13)


# ---------------------------------------------------------------- dual numbers
def test_jvp_matches_central_differences(oracle):
    prob = _mixed_problem(6, nel=(2, 2, 2), Nlo=1, Nhi=3, fv_frac=0.3, n_fv=5)
    U = W.smooth_random_state(prob, 6, amp=0.1)
    rng = np.random.default_rng(0)
    dU = rng.standard_normal(U.size) * 1e-2 * np.abs(U).mean()
    R, dR = oracle.eval_rhs_jvp(prob, U, dU)
    np.testing.assert_array_equal(R, oracle.eval_rhs(prob, U))
    eps = 1e-6
    fd = (oracle.eval_rhs(prob, U + eps * dU) - oracle.eval_rhs(prob, U - eps * dU)) / (2 * eps)
    assert np.abs(fd - dR).max() < 1e-6 * np.abs(dR).max()


def test_extended_jvp_is_the_tangent_in_long_double(oracle):
    """The long-double tangent (the rounding reference of adjoint parity) has
    the extended evaluation's value, agrees with the FP64 tangent to rounding
    and is linear in the direction (hybrid pattern, Roe-HH, Sutherland)."""
    prob = _mixed_problem(7, nel=(2, 2, 2), Nlo=1, Nhi=4, fv_frac=0.3, n_fv=5)
    prob.update(riemann=1, sutherland=1, T_ref=29.0, S_sutherland=11.7)
    U = W.smooth_random_state(prob, 7, amp=0.1)
    rng = np.random.default_rng(1)
    dU = rng.standard_normal(U.size) * 1e-2 * np.abs(U).mean()
    R, dR = oracle.eval_rhs_jvp(prob, U, dU)
    Rx, dRx = oracle.eval_rhs_jvp_extended(prob, U, dU)
    np.testing.assert_array_equal(Rx, oracle.eval_rhs_extended(prob, U))
    assert np.abs(dRx - dR).max() < 1e-13 * np.abs(dRx).max()
    _, d3 = oracle.eval_rhs_jvp_extended(prob, U, 3.0 * dU)
    assert np.abs(d3 - 3.0 * dRx).max() < 1e-15 * np.abs(d3).max()


# ---------------------------------------------------------------- split form on LGL nodes (Sec. 3.5)
def _lgl_derivative_matrix(n):
    """D_ij = l_j'(x_i) on the LGL points from the monomial coefficients of the
    Lagrange polynomials (inverse Vandermonde)."""
    x = W.lgl_nodes(n)
    C = np.linalg.inv(np.vander(x, n, increasing=True))  # column j: coefficients of l_j
    k = np.arange(n)
    return np.array([[np.sum(k[1:] * C[1:, j] * xi ** (k[1:] - 1)) for j in range(n)] for xi in x])


def _prims(prob, blk):
    """rho, v (3), p, H, Y_k per node of one element block (V, n^3)."""
    nk = len(prob["gamma"])
    cv = prob["Rgas"] / (prob["gamma"] - 1.0)
    rho = blk[:nk].sum(0)
    Y = blk[:nk] / rho
    v = blk[nk:nk + 3] / rho
    eps = blk[nk + 3] / rho - 0.5 * (v ** 2).sum(0)
    cvm, cpm = Y.T @ cv, Y.T @ (prob["gamma"] * cv)
    p = rho * (cpm - cvm) / cvm * eps
    H = (blk[nk + 3] + p) / rho
    return rho, v, p, H, Y


def test_split_form_volume_term_equals_the_quadratic_and_cubic_split_forms(oracle):
    """With arithmetic means, sum_m 2 D_im {a}{b} = (D(ab) + a Db + b Da)_i / 2 and
    sum_m 2 D_im {a}{b}{c} = (D(abc) + a D(bc) + b D(ac) + c D(ab) + ab Dc + ac Db
    + bc Da)_i / 4 (D 1 = 0).  The split-form R minus the standard LGL R on a
    DG element is therefore, per direction d with metric 2/h_d, minus the
    metric times [split(rho Y_k v_d) - D(rho_k v_d)], [split(rho v_d v_j) +
    D p delta_jd - D(rho v_d v_j + p delta_jd)], [split(rho v_d H) - D(rho H v_d)]
    along every line; zero on FV elements.  D comes from numpy (monomials)."""
    prob = _mixed_problem(11, nk=3, nel=(2, 3, 2), Nlo=1, Nhi=6, fv_frac=0.25, n_fv=7, nodes=1, mu=1e-3)
    U = W.smooth_random_state(prob, 11, amp=0.2)
    Rstd = oracle.eval_rhs(prob, U)
    Rspl = oracle.eval_rhs(dict(prob, split=1), U)
    nk = 3
    V = nk + 4
    off, _ = W.offsets(prob)
    npd = W.points_per_dir(prob)
    _, _, _, h = W.element_index(prob)
    checked = 0
    for e in range(len(off)):
        n = int(npd[e])
        blk = U[off[e]:off[e] + V * n ** 3].reshape(V, n, n, n)  # (v, k, j, i)
        diff = (Rspl - Rstd)[off[e]:off[e] + V * n ** 3].reshape(V, n, n, n)
        if prob["fv"][e]:
            assert np.abs(diff).max() == 0.0
            continue
        D = _lgl_derivative_matrix(n)
        rho, v, p, H, Y = _prims(prob, blk.reshape(V, -1).T.T.reshape(V, -1))
        sh = (n, n, n)
        rho, p, H = rho.reshape(sh), p.reshape(sh), H.reshape(sh)
        v, Y = v.reshape(3, *sh), Y.reshape(nk, *sh)
        expect = np.zeros((V, n, n, n))
        for d in range(3):
            ax = 2 - d  # array axis of direction d in (k, j, i) order

            def Dd(f):
                return np.moveaxis(np.tensordot(D, np.moveaxis(f, ax, 0), axes=(1, 0)), 0, ax)

            def s2(a, b):
                return 0.5 * (Dd(a * b) + a * Dd(b) + b * Dd(a))

            def s3(a, b, c):
                return 0.25 * (Dd(a * b * c) + a * Dd(b * c) + b * Dd(a * c) + c * Dd(a * b)
                               + a * b * Dd(c) + a * c * Dd(b) + b * c * Dd(a))
            vd = v[d]
            terms = [s3(rho, vd, Y[k]) - Dd(rho * Y[k] * vd) for k in range(nk)]
            terms += [s3(rho, vd, v[j]) - Dd(rho * vd * v[j]) for j in range(3)]
            terms += [s3(rho, vd, H) - Dd(rho * H * vd)]
            expect -= (2.0 / h[e][d]) * np.array(terms)
        scale = np.abs(Rstd).max()
        np.testing.assert_allclose(diff, expect, atol=1e-11 * scale)
        checked += 1
    assert checked > 4


@pytest.mark.parametrize("split", [0, 1])
def test_convergence_lgl_uniform_degree_3(split):
    """Order N+1 on LGL nodes, standard and split form (advected wave, Euler);
    the LGL scheme reaches its asymptotic order on finer meshes than LG (at
    K = 4 -> 8 the observed order is 3.3-3.5)."""
    import oracle
    e1 = _advected_l2(oracle, (16, 1, 1), lambda i, j, k: 3, nodes=1, split=split)
    e2 = _advected_l2(oracle, (32, 1, 1), lambda i, j, k: 3, nodes=1, split=split)
    assert _order(e1, e2, 16, 32) > 3.7, (e1, e2)


# ---------------------------------------------------------------- low-storage RK4 (Sec. 3.3)
def test_lsrk4_linear_stability_polynomial(oracle):
    """Five stages: the amplification factor of u' = z u is a degree-5
    polynomial in z whose first five coefficients are 1/k! (fourth order)."""
    zs = np.linspace(-2.0, 0.5, 9)
    amp = np.array([oracle.lsrk4_scalar(0, z, 1.0, 1.0) for z in zs])
    coef = np.polynomial.polynomial.polyfit(zs, amp, 5)
    np.testing.assert_allclose(coef[:5], [1.0, 1.0, 0.5, 1 / 6, 1 / 24], atol=1e-12)
    assert abs(coef[5]) < 0.01 and abs(coef[5]) > 1e-4


def test_lsrk4_fourth_order_on_a_nonlinear_ode(oracle):
    """u' = -u^2, u(0) = 1 has u(1) = 1/2; the global error falls 16x per halving
    of the step (the nonlinear order conditions, not only the linear ones)."""
    def solve(m):
        u = 1.0
        for _ in range(m):
            u = oracle.lsrk4_scalar(1, 0.0, 1.0 / m, u)
        return abs(u - 0.5)
    e = [solve(m) for m in (4, 8, 16)]
    assert np.log2(e[0] / e[1]) > 3.8 and np.log2(e[1] / e[2]) > 3.8, e


def test_lsrk4_on_the_dg_operator_is_fourth_order_in_time(oracle):
    """The plain tiny case (viscous, two species) advanced to t = 4e-3 with
    1, 2 and 4 steps against 32 steps: errors fall at order 4."""
    prob, U = W.plain_tiny(0)
    T = 4e-3
    ref, _ = oracle.lsrk4(prob, U, 32, dt_fixed=T / 32)
    e = [np.abs(oracle.lsrk4(prob, U, m, dt_fixed=T / m)[0] - ref).max() for m in (1, 2, 4)]
    assert np.log2(e[0] / e[1]) > 3.6 and np.log2(e[1] / e[2]) > 3.6, e


# ---------------------------------------------------------------- positivity limiter (Sec. 3.5)
def _rarefaction():
    """Two streams pulled apart (v_x up to 12, p = 0.4) on 16 x 1 x 1 elements,
    N = 3, air/helium, inviscid: the unlimited scheme loses positivity."""
    sp = W.species_set([W.AIR, W.HELIUM], mu=0.0)
    prob = W.make_problem([((16, 1, 1), (0, 0, 0), (1, 1.0 / 16, 1.0 / 16))], sp, n_fv=6, N=3)

    def fn(x, y, z):
        v = 12.0 * np.tanh((x - 0.5) / 0.05) * np.sin(2 * np.pi * x) ** 2
        return [0.5 + 0 * x, 0.5 + 0 * x], (v, 0 * x, 0 * x), 0.4 + 0 * x
    return prob, W.build_state(prob, fn)


def _check_points(prob, U, e):
    """Nodes and the six faces' points of DG element e (numpy's LG basis)."""
    off, _ = W.offsets(prob)
    V = W.n_vars(prob)
    n = int(prob["N"][e]) + 1
    blk = U[off[e]:off[e] + V * n ** 3].reshape(V, n, n, n)  # (v, k, j, i)
    x = np.polynomial.legendre.leggauss(n)[0]
    C = np.linalg.inv(np.vander(x, n, increasing=True))
    lm, lp = np.vander([-1.0], n, increasing=True) @ C, np.vander([1.0], n, increasing=True) @ C
    pts = [blk.reshape(V, -1)]
    for ax in (1, 2, 3):
        for l in (lm[0], lp[0]):
            pts.append(np.tensordot(blk, l, axes=([ax], [0])).reshape(V, -1))
    return np.concatenate(pts, axis=1)


def _mean(prob, U, e):
    off, _ = W.offsets(prob)
    V = W.n_vars(prob)
    n = int(prob["N"][e]) + 1
    w = np.polynomial.legendre.leggauss(n)[1]
    blk = U[off[e]:off[e] + V * n ** 3].reshape(V, n, n, n)
    return np.einsum("vkji,k,j,i->v", blk, w, w, w) / 8.0


def _rho_e(q, nk):
    return q[nk + 3] - 0.5 * (q[nk] ** 2 + q[nk + 1] ** 2 + q[nk + 2] ** 2) / q[:nk].sum(0)


def test_pp_limiter_keeps_positivity_means_and_is_a_no_op_on_positive_states(oracle):
    prob, U = _rarefaction()
    nk, eps = 2, 1e-10
    same, n0 = oracle.pp_limit(prob, U, eps)
    assert n0 == 0 and np.array_equal(same, U)
    # a state that lost positivity: 46 unlimited steps (still positive), then the
    # deviations from every element mean amplified sixfold (means unchanged)
    X, _ = oracle.rk3(prob, U, 46, cfl_c=0.3, cfl_v=0.3)
    off, _ = W.offsets(prob)
    for e in range(16):
        blk = X[off[e]:off[e] + 6 * 64].reshape(6, 64)
        m = _mean(prob, X, e)
        blk[:] = m[:, None] + 6.0 * (blk - m[:, None])
    bad = [e for e in range(16) if (_check_points(prob, X, e)[:nk] < 0).any()
           or (_rho_e(_check_points(prob, X, e), nk) < 0).any()]
    assert bad, "the unlimited run should have lost positivity by now"
    L, nl = oracle.pp_limit(prob, X, eps)
    assert nl >= len(bad)
    for e in range(16):
        m0, m1 = _mean(prob, X, e), _mean(prob, L, e)
        np.testing.assert_allclose(m1, m0, rtol=1e-13, atol=1e-14 * np.abs(m0).max())
        q = _check_points(prob, L, e)
        for k in range(nk):
            assert q[k].min() >= min(eps, m0[k]) * (1 - 1e-9) - 1e-15
        re = _rho_e(q, nk)
        assert re.min() >= min(eps, _rho_e(m0, nk)) - 1e-12
        if e in bad and (_rho_e(_check_points(prob, X, e), nk) < 0).any():
            # the internal-energy step is tight: the smallest value sits on the floor
            assert re.min() < min(eps, _rho_e(m0, nk)) + 1e-9
        # momentum and energy move on one line towards the mean (one theta per element)
        d0 = (_check_points(prob, X, e) - m0[:, None])[nk:]
        d1 = (q - m0[:, None])[nk:]
        big = np.abs(d0) > 1e-8 * np.abs(d0).max()
        ratios = d1[big] / d0[big]
        assert ratios.max() - ratios.min() < 1e-9


def test_pp_limiter_keeps_a_rarefaction_alive(oracle):
    """Without the limiter the rarefaction breaks down (non-finite values
    within 60 SSP-RK3 steps); with it the run stays finite and every partial
    density and internal energy at the check points stays non-negative."""
    prob, U = _rarefaction()
    X, _ = oracle.rk3(prob, U, 60, cfl_c=0.3, cfl_v=0.3)
    assert not np.isfinite(X).all()
    Y, _ = oracle.rk3(dict(prob, pp_limiter=1, pp_eps=1e-10), U, 60, cfl_c=0.3, cfl_v=0.3)
    assert np.isfinite(Y).all()
    for e in range(16):
        q = _check_points(prob, Y, e)
        assert q[:2].min() >= -1e-14 and _rho_e(q, 2).min() >= -1e-12
