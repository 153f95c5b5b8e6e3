"""The hand-written adjoint of the CUDA path (dgfv_rhs_vjp, dgfv_rk_step_vjp)
against the oracle: the dot-product test <R_bar, J v> (oracle, exact dual
numbers) = <J^T R_bar (CUDA), v> on DG and hybrid DG/FV patterns (LG, LGL,
split form; LLF, Roe-HH, hybrid flux), whole adjoint matrices on tiny meshes,
the SSP-RK3 and low-storage RK4 step adjoints against exact stage-by-stage
tangents or central differences, and the gradient of a
kinetic-energy-plus-species-variance functional after a short rollout."""
import numpy as np
import pytest

from paper_2502_19342_gb300 import workloads as W
from tests.gpu_helpers import assert_adjoint_close, ctx_for, per_field, to_dev

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _dg_problem(seed, nk=3, nel=(3, 2, 3), Nlo=1, Nhi=5, mu=3e-3, uniform=None, nodes=0, sutherland=False,
                riemann=0):
    specs = [W.AIR, W.HELIUM, W.CO2][:nk]
    sp = W.species_set(specs, mu=mu)
    n = nel[0] * nel[1] * nel[2]
    N = np.full(n, uniform, np.int8) if uniform else W.random_degrees(n, Nlo, Nhi, seed)
    prob = W.make_problem([(nel, (0, 0, 0), (1.0, 0.8, 1.1))], sp, n_fv=8, N=N, riemann=riemann, nodes=nodes)
    if sutherland:  # T ~ p / (rho R) ~ 29 in these states; Sutherland constants of air scaled to it
        prob.update(sutherland=1, T_ref=29.0, S_sutherland=29.0 * 110.4 / 273.15)
    return prob, W.smooth_random_state(prob, seed, amp=0.1)


@pytest.mark.parametrize("nk,mu,seed,uniform,nodes,suth,riemann", [
    (3, 3e-3, 1, None, 0, False, 0), (2, 0.0, 2, None, 0, False, 0), (1, 1e-3, 3, None, 0, False, 0),
    (3, 2e-3, 4, 4, 0, False, 0), (3, 2e-3, 5, None, 1, False, 0), (3, 3e-3, 6, None, 0, True, 0),
    (2, 2e-3, 7, None, 1, True, 0), (3, 3e-3, 8, None, 0, False, 1), (2, 0.0, 9, None, 0, False, 1),
    (3, 2e-3, 10, None, 1, True, 2)])
def test_rhs_vjp_dot_product_with_oracle_jvp(oracle, nk, mu, seed, uniform, nodes, suth, riemann):
    """Constant and Sutherland viscosity (Sec. 4.3), LG and LGL nodes, the LLF
    and the Roe-HH flux (hybrid = Roe-HH on a DG-only pattern)."""
    prob, U = _dg_problem(seed, nk=nk, mu=mu, uniform=uniform, nodes=nodes, sutherland=suth, riemann=riemann)
    rng = np.random.default_rng(seed)
    Rbar = rng.standard_normal(U.size)
    ctx = ctx_for(prob, N_min=1, N_max=7)
    Ubar = ctx.rhs_vjp(to_dev(U), to_dev(Rbar)).cpu().numpy()
    for _ in range(3):
        v = rng.standard_normal(U.size) * 1e-2 * np.abs(U).mean()
        _, Jv = oracle.eval_rhs_jvp(prob, U, v)
        lhs = float(np.dot(Rbar, Jv))
        rhs = float(np.dot(Ubar, v))
        scale = float(np.abs(Rbar * Jv).sum())
        assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs, scale)
    ctx.close()


def test_rhs_vjp_full_adjoint_against_oracle_columns(oracle):
    """On a tiny mesh the whole matrix J^T R_bar is checked entry by entry: the
    oracle's JVP along every unit vector gives the columns of J."""
    prob, U = _dg_problem(5, nk=2, nel=(2, 1, 2), Nlo=1, Nhi=2)
    rng = np.random.default_rng(5)
    Rbar = rng.standard_normal(U.size)
    ctx = ctx_for(prob, N_min=1, N_max=7)
    Ubar = ctx.rhs_vjp(to_dev(U), to_dev(Rbar)).cpu().numpy()
    assert_adjoint_close(oracle, prob, U, Rbar, Ubar)
    ctx.close()


def test_rk_step_vjp_against_central_differences(oracle):
    prob, U = _dg_problem(6, nk=3, uniform=3)
    dt = 2e-4
    ctx = ctx_for(prob, N_min=1, N_max=7)
    rng = np.random.default_rng(6)
    lam = rng.standard_normal(U.size)
    Ubar = ctx.rk_step_vjp(to_dev(U), dt, to_dev(lam)).cpu().numpy()
    eps = 1e-6
    for _ in range(6):
        v = rng.standard_normal(U.size) * np.abs(U).mean()
        up, _ = oracle.rk3(prob, U + eps * v, 1, dt_fixed=dt)
        um, _ = oracle.rk3(prob, U - eps * v, 1, dt_fixed=dt)
        fd = float(np.dot(lam, (up - um) / (2 * eps)))
        ad = float(np.dot(Ubar, v))
        assert abs(fd - ad) <= 1e-6 * abs(fd) + 1e-9 * float(np.abs(lam).sum() * np.abs(v).mean()), (fd, ad)
    ctx.close()


# Carpenter and Kennedy's five-stage 2N-storage RK4 (the published coefficients)
_LSRK4_A = (0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
            -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0)
_LSRK4_B = (1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
            1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
            2277821191437.0 / 14882151754819.0)


def _lsrk4_step_tangent(oracle, prob, U, v, dt):
    """One low-storage RK4 step and its exact tangent along v, stage by stage
    with the oracle's R and its dual-number JVP."""
    Uc, Vc = U.copy(), v.copy()
    dU, dV = np.zeros_like(U), np.zeros_like(U)
    for a, b in zip(_LSRK4_A, _LSRK4_B):
        R, JR = oracle.eval_rhs_jvp(prob, Uc, Vc)
        dU = a * dU + dt * R
        dV = a * dV + dt * JR
        Uc = Uc + b * dU
        Vc = Vc + b * dV
    return Uc, Vc


@pytest.mark.parametrize("mu,seed", [(3e-3, 16), (0.0, 17)])
def test_lsrk4_step_vjp_dot_product(oracle, mu, seed):
    """Adjoint of one five-stage low-storage RK4 step (Sec. 3.3), stages
    recomputed: <lambda, (dU1/dU0) v> with the exact stage-by-stage tangent of
    the oracle equals <(dU1/dU0)^T lambda, v> of the CUDA path.  The step
    itself is checked against the oracle's integrator first."""
    prob, U = _dg_problem(seed, nk=2, mu=mu, Nlo=1, Nhi=4)
    dt = 2e-4
    ctx = ctx_for(prob, N_min=1, N_max=7, opts={"integrator": 1})
    rng = np.random.default_rng(seed)
    lam = rng.standard_normal(U.size)
    Ubar = ctx.rk_step_vjp(to_dev(U), dt, to_dev(lam)).cpu().numpy()
    U1, _ = oracle.lsrk4(prob, U, 1, dt_fixed=dt)
    for _ in range(3):
        v = rng.standard_normal(U.size) * np.abs(U).mean()
        Uc, Jv = _lsrk4_step_tangent(oracle, prob, U, v, dt)
        assert np.abs(Uc - U1).max() <= 1e-13 * np.abs(U1).max()
        lhs, rhs = float(np.dot(lam, Jv)), float(np.dot(Ubar, v))
        scale = float(np.abs(lam * Jv).sum())
        assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs, scale)
    ctx.close()


def _functional(prob, U, Ybar):
    """sum over nodes of w J [rho |v|^2 / 2 + sum_{k<Nk} (Y_k - Ybar_k)^2] (DG elements)."""
    f = per_field(prob, U)
    nk = len(prob["gamma"])
    rho = sum(f[:nk])
    ke = 0.5 * (f[nk] ** 2 + f[nk + 1] ** 2 + f[nk + 2] ** 2) / rho
    var = sum((f[k] / rho - Ybar[k]) ** 2 for k in range(nk - 1))
    wts = np.concatenate([np.einsum("k,j,i->kji", *(np.polynomial.legendre.leggauss(int(N) + 1)[1],) * 3).ravel()
                          for N in prob["N"]])
    return float(np.sum(wts * (ke + var)))


def test_rollout_gradient_against_central_differences(oracle):
    """Gradient of the functional after 4 SSP-RK3 steps with respect to the
    initial state (stage checkpointing), against central differences of the
    oracle's rollout along seeded directions."""
    from paper_2502_19342_gb300 import dgfv
    prob, U = _dg_problem(7, nk=3, nel=(2, 2, 2), uniform=3, mu=2e-3)
    Ybar = [0.3, 0.3]
    dt, steps = 3e-4, 4
    ctx = ctx_for(prob, N_min=1, N_max=7)
    nk = 3

    def loss_grad(Uf):
        X = Uf.detach().clone().requires_grad_(True)
        f = per_field_torch(prob, X)
        rho = f[0] + f[1] + f[2]
        ke = 0.5 * (f[nk] ** 2 + f[nk + 1] ** 2 + f[nk + 2] ** 2) / rho
        var = sum((f[k] / rho - Ybar[k]) ** 2 for k in range(nk - 1))
        w = torch.from_numpy(_weights(prob)).cuda()
        (w * (ke + var)).sum().backward()
        return X.grad.contiguous()

    grad, _ = dgfv.rollout_gradient(ctx, to_dev(U), steps, dt, loss_grad)
    grad = grad.cpu().numpy()
    rng = np.random.default_rng(7)
    eps = 1e-6
    for _ in range(5):
        v = rng.standard_normal(U.size) * np.abs(U).mean()
        Jp = _functional(prob, oracle.rk3(prob, U + eps * v, steps, dt_fixed=dt)[0], Ybar)
        Jm = _functional(prob, oracle.rk3(prob, U - eps * v, steps, dt_fixed=dt)[0], Ybar)
        fd = (Jp - Jm) / (2 * eps)
        ad = float(np.dot(grad, v))
        assert abs(fd - ad) <= 1e-6 * abs(fd) + 1e-10, (fd, ad)
    ctx.close()


def _weights(prob):
    """Per-point LG weights (x fastest) of every element, repeated for no variable."""
    return np.concatenate([np.einsum("k,j,i->kji", *(np.polynomial.legendre.leggauss(int(N) + 1)[1],) * 3).ravel()
                           for N in prob["N"]])


def per_field_torch(prob, X):
    off, _ = W.offsets(prob)
    V = W.n_vars(prob)
    n = W.points_per_dir(prob)
    out = [[] for _ in range(V)]
    for e in range(len(off)):
        m3 = int(n[e]) ** 3
        blk = X[int(off[e]):int(off[e]) + V * m3].reshape(V, m3)
        for v in range(V):
            out[v].append(blk[v])
    return [torch.cat(o) for o in out]


def test_autograd_function_backward_is_the_adjoint():
    from paper_2502_19342_gb300 import dgfv
    prob, U = _dg_problem(8, nk=2, uniform=2)
    ctx = ctx_for(prob, N_min=1, N_max=7)
    X = to_dev(U).requires_grad_(True)
    R = dgfv.rhs_function().apply(X, ctx)
    Rbar = torch.randn_like(R)
    (R * Rbar).sum().backward()
    ref = ctx.rhs_vjp(to_dev(U), Rbar.detach().contiguous())
    torch.testing.assert_close(X.grad, ref, rtol=0, atol=0)
    ctx.close()


@pytest.mark.parametrize("nk,mu,seed,riemann", [(2, 2e-3, 12, 0), (3, 0.0, 13, 1), (1, 1e-3, 14, 0), (3, 3e-3, 15, 2)])
def test_split_form_rhs_vjp_dot_product(oracle, nk, mu, seed, riemann):
    """Split form on LGL nodes (Sec. 3.5): the two-point volume term's reverse
    (k_adj_split) with the standard viscous part, against the oracle's exact
    dual-number JVP of its split form."""
    prob, U = _dg_problem(seed, nk=nk, mu=mu, nodes=1, riemann=riemann, Nlo=1, Nhi=6)
    prob["split"] = 1
    rng = np.random.default_rng(seed)
    Rbar = rng.standard_normal(U.size)
    ctx = ctx_for(prob, N_min=1, N_max=7)
    Ubar = ctx.rhs_vjp(to_dev(U), to_dev(Rbar)).cpu().numpy()
    for _ in range(3):
        v = rng.standard_normal(U.size) * 1e-2 * np.abs(U).mean()
        _, Jv = oracle.eval_rhs_jvp(prob, U, v)
        lhs, rhs = float(np.dot(Rbar, Jv)), float(np.dot(Ubar, v))
        scale = float(np.abs(Rbar * Jv).sum())
        assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs, scale)
    ctx.close()


def _hybrid_problem(seed, nk=2, nel=(3, 2, 3), Nlo=1, Nhi=5, fv_frac=0.35, n_fv=6, mu=3e-3, riemann=0, nodes=0):
    specs = [W.AIR, W.HELIUM, W.CO2][:nk]
    sp = W.species_set(specs, mu=mu)
    n = nel[0] * nel[1] * nel[2]
    prob = W.make_problem([(nel, (0, 0, 0), (1.0, 0.8, 1.1))], sp, n_fv=n_fv, N=W.random_degrees(n, Nlo, Nhi, seed),
                          fv=W.random_fv(n, fv_frac, seed), riemann=riemann, nodes=nodes)
    return prob, W.smooth_random_state(prob, seed, amp=0.1)


@pytest.mark.parametrize("nk,mu,seed,riemann,n_fv,nodes,fv_frac", [
    (2, 3e-3, 31, 0, 6, 0, 0.35), (3, 0.0, 32, 0, 7, 0, 0.35), (2, 2e-3, 33, 1, 6, 0, 0.35),
    (3, 3e-3, 34, 2, 8, 0, 0.35), (1, 1e-3, 35, 0, 6, 1, 0.35), (2, 2e-3, 36, 2, 6, 0, 1.0),
    (2, 2e-3, 38, 0, 9, 0, 0.35)])
def test_rhs_vjp_with_fv_elements_dot_product(oracle, nk, mu, seed, riemann, n_fv, nodes, fv_frac):
    """Hybrid DG/FV patterns frozen in the backward (Sec. 3.1.2, 3.2): the FV
    sub-cell operator reversed (minmod along the forward's branches, central
    differences, sub-cell Riemann and viscous fluxes), the DG/FV face and lifting
    maps transposed, against the oracle's exact dual-number JVP; LLF, Roe-HH
    and the hybrid flux choice; an all-FV mesh.  N_FV = 6, 7 run the FV reverse
    with the sub-cell gradients kept in shared memory, 8 and 9 with the
    gradients formed at each face (two CTAs of 128 threads per SM, and one of
    256)."""
    prob, U = _hybrid_problem(seed, nk=nk, mu=mu, riemann=riemann, n_fv=n_fv, nodes=nodes, fv_frac=fv_frac)
    rng = np.random.default_rng(seed)
    Rbar = rng.standard_normal(U.size)
    ctx = ctx_for(prob, N_min=1, N_max=int(prob["N"].max()))
    Ubar = ctx.rhs_vjp(to_dev(U), to_dev(Rbar)).cpu().numpy()
    for _ in range(3):
        v = rng.standard_normal(U.size) * 1e-2 * np.abs(U).mean()
        _, Jv = oracle.eval_rhs_jvp(prob, U, v)
        lhs, rhs = float(np.dot(Rbar, Jv)), float(np.dot(Ubar, v))
        scale = float(np.abs(Rbar * Jv).sum())
        assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs, scale)
    ctx.close()


def test_rhs_vjp_with_fv_elements_columns(oracle):
    """A 2x1x2 mesh with one FV element (N_FV = 3) among DG elements of degree
    1-2: the whole J^T R_bar entry by entry against the oracle's JVP columns."""
    sp = W.species_set([W.AIR, W.HELIUM], mu=2e-3)
    prob = W.make_problem([((2, 1, 2), (0, 0, 0), (1.0, 0.5, 1.0))], sp, n_fv=3,
                          N=np.array([2, 1, 2, 1], np.int8), fv=np.array([0, 1, 0, 0], np.uint8))
    U = W.smooth_random_state(prob, 4, amp=0.1)
    rng = np.random.default_rng(4)
    Rbar = rng.standard_normal(U.size)
    ctx = ctx_for(prob, N_min=1, N_max=2)
    Ubar = ctx.rhs_vjp(to_dev(U), to_dev(Rbar)).cpu().numpy()
    assert_adjoint_close(oracle, prob, U, Rbar, Ubar)
    ctx.close()


@pytest.mark.parametrize("nk,riemann,nodes,split,suth,n_fv,seed,fv", [
    (3, 1, 0, 0, False, 4, 41, [0, 1, 0, 0]), (2, 2, 0, 0, True, 4, 42, [0, 1, 0, 0]),
    (2, 0, 1, 1, False, 4, 43, [1, 0, 0, 0]), (3, 2, 1, 1, True, 4, 44, [0, 1, 1, 0])])
def test_rhs_vjp_columns_per_field(oracle, nk, riemann, nodes, split, suth, n_fv, seed, fv):
    """Small hybrid meshes (2x2x1 elements of degree 1-3, one or two FV):
    Roe-HH and the hybrid flux, Sutherland viscosity, LG and LGL nodes, the
    standard and the split-form volume term; the whole U_bar field by field
    against the oracle's adjoint by columns, with the bar of R(U)."""
    prob, _ = _hybrid_problem(seed, nk=nk, nel=(2, 2, 1), Nlo=1, Nhi=3, n_fv=n_fv, mu=3e-3, riemann=riemann,
                              nodes=nodes)
    prob.update(fv=np.array(fv, np.uint8), split=split)
    if suth:
        prob.update(sutherland=1, T_ref=29.0, S_sutherland=29.0 * 110.4 / 273.15)
    U = W.smooth_random_state(prob, seed, amp=0.1)
    rng = np.random.default_rng(seed)
    Rbar = rng.standard_normal(U.size)
    ctx = ctx_for(prob, N_min=1, N_max=3)
    Ubar = ctx.rhs_vjp(to_dev(U), to_dev(Rbar)).cpu().numpy()
    assert_adjoint_close(oracle, prob, U, Rbar, Ubar)
    ctx.close()


def test_rk_step_vjp_with_fv_elements_dot_product(oracle):
    """One SSP-RK3 step of a hybrid pattern, stages recomputed: against the
    exact stage-by-stage tangent built from the oracle's JVP."""
    prob, U = _hybrid_problem(37, nk=2, mu=2e-3, n_fv=6)
    dt = 2e-4
    ctx = ctx_for(prob, N_min=1, N_max=int(prob["N"].max()))
    rng = np.random.default_rng(37)
    lam = rng.standard_normal(U.size)
    Ubar = ctx.rk_step_vjp(to_dev(U), dt, to_dev(lam)).cpu().numpy()
    for _ in range(2):
        v = rng.standard_normal(U.size) * np.abs(U).mean()
        # U1 = U + dt R(U); U2 = 3/4 U + 1/4 (U1 + dt R(U1)); U3 = 1/3 U + 2/3 (U2 + dt R(U2))
        R0, J0 = oracle.eval_rhs_jvp(prob, U, v)
        U1, V1 = U + dt * R0, v + dt * J0
        R1, J1 = oracle.eval_rhs_jvp(prob, U1, V1)
        U2, V2 = 0.75 * U + 0.25 * (U1 + dt * R1), 0.75 * v + 0.25 * (V1 + dt * J1)
        R2, J2 = oracle.eval_rhs_jvp(prob, U2, V2)
        V3 = v / 3.0 + 2.0 / 3.0 * (V2 + dt * J2)
        lhs, rhs = float(np.dot(lam, V3)), float(np.dot(Ubar, v))
        scale = float(np.abs(lam * V3).sum())
        assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs, scale)
    ctx.close()


def test_stored_stage_adjoint_matches_recomputed_stages():
    """dgfv_rk_step_save advances the state exactly as dgfv_rk_step and keeps
    U1, U2; the adjoint from those stored stages equals, bit for bit, the
    adjoint that recomputes them (same kernels on the same inputs); so does a
    rollout gradient from segment checkpoints (every k-th state kept, the
    others stepped again in the backward pass)."""
    from paper_2502_19342_gb300 import dgfv
    prob, U = _dg_problem(10, nk=3, nel=(3, 2, 2), uniform=None, mu=2e-3)
    dt = 2e-4
    ctx = ctx_for(prob, N_min=1, N_max=7)
    U0 = to_dev(U)
    ctx.set_state(U0)
    ctx.rk_step(dt, want_dt=False)
    ref = ctx.get_state()
    ctx.set_state(U0)
    s1, s2 = torch.empty_like(U0), torch.empty_like(U0)
    ctx.rk_step_save(dt, s1, s2)
    assert torch.equal(ctx.get_state(), ref)
    lam = to_dev(np.random.default_rng(10).standard_normal(U.size))
    a = ctx.rk_step_vjp(U0, dt, lam)
    b = ctx.rk_step_vjp_stages((U0, s1, s2), dt, lam)
    assert torch.equal(a, b)
    with pytest.raises(dgfv.DgfvError):
        ctx.rk_step_vjp_stages((U0, s1, s2), dt, lam, Ubar=s1)
    g1, _ = dgfv.rollout_gradient(ctx, U0, 3, dt, lambda Uf: torch.ones_like(Uf))
    g2, _ = dgfv.rollout_gradient(ctx, U0, 3, dt, lambda Uf: torch.ones_like(Uf), keep_stages=True)
    assert torch.equal(g1, g2)
    # segment checkpoints (every 2nd, every 3rd state, one for the whole
    # rollout): the step states recomputed bitwise, so the same gradient
    w = to_dev(np.random.default_rng(11).standard_normal(U.size))
    ref, Uf = dgfv.rollout_gradient(ctx, U0, 7, dt, lambda X: w * X)
    for k in (2, 3, 7, 9):
        g, Ufk = dgfv.rollout_gradient(ctx, U0, 7, dt, lambda X: w * X, checkpoint_every=k)
        assert torch.equal(g, ref), k
        assert torch.equal(Ufk, Uf) and torch.equal(ctx.get_state(), Uf)
    with pytest.raises(ValueError):
        dgfv.rollout_gradient(ctx, U0, 3, dt, lambda X: X, keep_stages=True, checkpoint_every=2)
    ctx.close()


@pytest.mark.parametrize("integrator", [0, 1])
def test_rk_step_autograd_function_matches_rollout_gradient(integrator):
    """The RK step behind torch.autograd.Function (SSP-RK3, low-storage RK4):
    a chain of four steps and a torch loss on the final state backpropagate,
    step by step through the hand-written step adjoint, to the same gradient as
    rollout_gradient (bit for bit: the same adjoints on the same states); the
    forward chain reproduces the context's own rollout."""
    from paper_2502_19342_gb300 import dgfv
    prob, U = _dg_problem(12, nk=2, nel=(2, 3, 2), uniform=None, mu=2e-3)
    dt = 2e-4
    ctx = ctx_for(prob, opts=dict(integrator=integrator), N_min=1, N_max=7)
    w = to_dev(np.random.default_rng(12).standard_normal(U.size))
    step = dgfv.rk_step_function()
    X = to_dev(U).requires_grad_(True)
    Y = X
    for _ in range(4):
        Y = step.apply(Y, ctx, dt)
    (0.5 * (w * Y * Y).sum()).backward()
    g_ref, Uf = dgfv.rollout_gradient(ctx, to_dev(U), 4, dt, lambda Z: w * Z)
    assert torch.equal(Y.detach(), Uf)
    assert torch.equal(X.grad, g_ref)
    ctx.close()
