"""Bookkeeping of dgfv.rollout_gradient's checkpoint schemes, on the host: a
stand-in context with a nonlinear step U <- U + dt sin(U) and its exact
adjoint lam <- lam (1 + dt cos(U)) (the state each step adjoint receives must
be that step's start state).  Every scheme gives the chain-rule gradient; with
a checkpoint every k steps the backward pass steps each segment forward again
from its checkpoint (n_steps - ceil(n_steps / k) extra steps)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2502_19342_gb300 import dgfv


class _Ctx:
    def __init__(self):
        self.U = None
        self.forward_steps = 0

    def set_state(self, U):
        self.U = U.clone()

    def get_state(self, out=None):
        return self.U.clone()

    def rk_step(self, dt, want_dt=True):
        self.U = self.U + dt * torch.sin(self.U)
        self.forward_steps += 1

    def rk_step_save(self, dt, s1, s2):
        s1.copy_(self.U)
        s2.copy_(self.U)
        self.rk_step(dt)

    def rk_step_vjp(self, U0, dt, lam):
        return lam * (1.0 + dt * torch.cos(U0))

    def rk_step_vjp_stages(self, stages, dt, lam):
        return self.rk_step_vjp(stages[0], dt, lam)


def _reference(U0, n, dt, w):
    U, states = U0.clone(), []
    for _ in range(n):
        states.append(U.clone())
        U = U + dt * torch.sin(U)
    lam = w * U
    for s in range(n - 1, -1, -1):
        lam = lam * (1.0 + dt * torch.cos(states[s]))
    return lam, U


@pytest.mark.parametrize("n", [0, 1, 5, 12])
@pytest.mark.parametrize("k", [1, 2, 3, 5, 12, 20])
def test_checkpoint_every_k_steps(n, k):
    rng = np.random.default_rng(n * 31 + k)
    U0 = torch.from_numpy(rng.standard_normal(17))
    w = torch.from_numpy(rng.standard_normal(17))
    dt = 0.3
    ref, Uf_ref = _reference(U0, n, dt, w)
    ctx = _Ctx()
    g, Uf = dgfv.rollout_gradient(ctx, U0, n, dt, lambda X: w * X, checkpoint_every=k)
    assert torch.equal(Uf, Uf_ref)
    assert torch.allclose(g, ref, rtol=1e-14, atol=0)
    assert torch.equal(ctx.get_state(), Uf)
    assert ctx.forward_steps == n + (n - -(-n // k))  # the rollout, then each segment but its first step


def test_stored_stages_and_argument_checks():
    U0 = torch.linspace(-1.0, 2.0, 9, dtype=torch.float64)
    w = torch.ones(9, dtype=torch.float64)
    ref, _ = _reference(U0, 4, 0.2, w)
    g, _ = dgfv.rollout_gradient(_Ctx(), U0, 4, 0.2, lambda X: w * X, keep_stages=True)
    assert torch.allclose(g, ref, rtol=1e-14, atol=0)
    with pytest.raises(ValueError):
        dgfv.rollout_gradient(_Ctx(), U0, 4, 0.2, lambda X: X, checkpoint_every=0)
    with pytest.raises(ValueError):
        dgfv.rollout_gradient(_Ctx(), U0, 4, 0.2, lambda X: X, keep_stages=True, checkpoint_every=3)
