"""The rollout adjoint at the adjoint workload's full configuration: the
temporal mixing layer on 16^3 elements, N = 4, 3 species, viscous, 50 SSP-RK3
steps at the frozen initial CFL step, with stage checkpointing (one state per
step is kept, the stage states are recomputed in the backward pass).

The gradient of J = sum over nodes of w J_geo [rho |v|^2/2 + sum_{k<Nk} (Y_k -
Ybar_k)^2] of the final state with respect to the initial state is checked
  - against central differences (eps = 1e-6) of the CUDA forward rollout along
    20 seeded random directions, to 1e-6 relative;
  - against the oracle's exact directional derivative along 2 of them: the
    oracle's dual-number tangent of R carried through the 150 stages of its
    own SSP-RK3 rollout (no difference quotient), to 1e-8 relative.
"""
import numpy as np
import pytest

from paper_2502_19342_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

STEPS = 50
NK, V, NP = 3, 7, 125  # species, variables, nodes per element (N = 4)


def _setup():
    prob, U = W.mixing_layer()
    h = 1.0 / 16
    jgeo = h ** 3 / 8
    w1 = np.polynomial.legendre.leggauss(5)[1]
    w = np.einsum("k,j,i->kji", w1, w1, w1).ravel() * jgeo
    blk = U.reshape(-1, V, NP)
    rho0 = blk[:, :NK].sum(1)
    Ybar = [float((blk[:, k] / rho0).mean()) for k in range(NK - 1)]
    return prob, U, w, Ybar


def _J_torch(X, w, Ybar):
    blk = X.view(-1, V, NP)
    rho = blk[:, :NK].sum(1)
    ke = 0.5 * (blk[:, NK] ** 2 + blk[:, NK + 1] ** 2 + blk[:, NK + 2] ** 2) / rho
    var = sum((blk[:, k] / rho - Ybar[k]) ** 2 for k in range(NK - 1))
    return (w[None, :] * (ke + var)).sum()


def _dJ_numpy(Uf, dUf, w, Ybar):
    """Directional derivative of J at Uf along dUf, written out."""
    b, db = Uf.reshape(-1, V, NP), dUf.reshape(-1, V, NP)
    rho, drho = b[:, :NK].sum(1), db[:, :NK].sum(1)
    m2 = sum(b[:, NK + i] ** 2 for i in range(3))
    dm2 = sum(2 * b[:, NK + i] * db[:, NK + i] for i in range(3))
    dke = 0.5 * (dm2 / rho - m2 * drho / rho ** 2)
    dvar = sum(2 * (b[:, k] / rho - Ybar[k]) * (db[:, k] / rho - b[:, k] * drho / rho ** 2) for k in range(NK - 1))
    return float((w[None, :] * (dke + dvar)).sum())


def test_mixing_layer_rollout_gradient_at_full_configuration(oracle):
    from paper_2502_19342_gb300 import dgfv
    prob, U, w, Ybar = _setup()
    ctx = dgfv.Context(prob, N_min=4, N_max=4)
    U0 = torch.from_numpy(U).cuda()
    dt = ctx.compute_dt(U0)[0]
    wd = torch.from_numpy(w).cuda()

    def loss_grad(Uf):
        X = Uf.detach().clone().requires_grad_(True)
        _J_torch(X, wd, Ybar).backward()
        return X.grad.contiguous()

    grad, _ = dgfv.rollout_gradient(ctx, U0, STEPS, dt, loss_grad)  # stage checkpointing
    grad = grad.cpu().numpy()
    assert np.isfinite(grad).all()

    def J_of(Ustart):
        ctx.set_state(torch.from_numpy(Ustart).cuda())
        ctx.rk_steps(STEPS, dt, want_dt=False)
        return float(_J_torch(ctx.get_state(), wd, Ybar).item())

    rng = np.random.default_rng(2502)
    eps = 1e-6
    dirs = []
    for i in range(20):
        v = rng.standard_normal(U.size) * np.abs(U)  # relative perturbation of every entry
        fd = (J_of(U + eps * v) - J_of(U - eps * v)) / (2 * eps)
        ad = float(np.dot(grad, v))
        assert abs(fd - ad) <= 1e-6 * abs(fd), (i, fd, ad)
        dirs.append((v, ad))
    ctx.close()

    # the oracle's exact tangent of its own rollout along two of the directions
    a = (0.0, 0.75, 1.0 / 3.0)
    b = (1.0, 0.25, 2.0 / 3.0)
    for v, ad in dirs[:2]:
        X, dX = U.copy(), v.copy()
        for _ in range(STEPS):
            X0, dX0 = X.copy(), dX.copy()
            for s in range(3):
                R, dR = oracle.eval_rhs_jvp(prob, X, dX)
                X = a[s] * X0 + b[s] * (X + dt * R)
                dX = a[s] * dX0 + b[s] * (dX + dt * dR)
        exact = _dJ_numpy(X, dX, w, Ybar)
        assert abs(exact - ad) <= 1e-8 * abs(exact), (exact, ad)
