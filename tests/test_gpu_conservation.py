"""Conservation at scale: on periodic meshes the integral of every conserved
variable (every species' mass, the momentum, the energy) is constant.  The
face fluxes enter both neighbours with opposite signs (Eqs. 22, 26); the maps
of the p-coupling, the DG/FV coupling and the mortars keep face integrals
(Sec. 3.2); the remaps of an adaptation keep element integrals (L2
projections, and the sub-cell means of V^{DG->FV} and its mean-preserving
inverse); the Runge-Kutta stages combine states linearly.  So through steps
and adaptations the integrals may move by round-off only: checked here on the
GPU path with the pattern the indicator drives, on the hp-mixed shock case at
its full size and on a non-conforming (mortar) mesh."""
import numpy as np
import pytest

from paper_2502_19342_gb300 import workloads as W
from tests.gpu_helpers import record, to_dev

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _integrals(prob, U):
    """Per conserved variable: sum over elements of the quadrature of the state
    (DG: Gauss weights at the nodes; FV: sub-cell volumes) times the element
    Jacobian, and the same of |U| (the scale of the round-off)."""
    off, _ = W.offsets(prob)
    _, _, _, h = W.element_index(prob)
    V = W.n_vars(prob)
    n = W.points_per_dir(prob)
    weights = {}
    tot, mag = np.zeros(V), np.zeros(V)
    for e in range(W.n_elements(prob)):
        m = int(n[e])
        fv = bool(prob["fv"][e])
        if (fv, m) not in weights:
            if fv:
                weights[(fv, m)] = np.full(m ** 3, (2.0 / m) ** 3)
            else:
                w = np.polynomial.legendre.leggauss(m)[1]
                weights[(fv, m)] = np.einsum("k,j,i->kji", w, w, w).ravel()
        wj = weights[(fv, m)] * (np.prod(h[e]) / 8.0)
        blk = U[off[e]:off[e] + V * m ** 3].reshape(V, m ** 3)
        tot += blk @ wj
        mag += np.abs(blk) @ wj
    return tot, mag


def _run(prob, U, ctx, cycles, steps):
    I0, M0 = _integrals(prob, U)
    seen_fv = 0
    for c in range(cycles):
        ctx.adapt()
        ctx.rk_steps(steps, -1.0, want_dt=False)
        N, fv = ctx.get_degrees()
        seen_fv = max(seen_fv, int(fv.sum()))
        I, M = _integrals(dict(prob, N=N, fv=fv), ctx.get_state().cpu().numpy())
        # the scale of a variable's round-off: its |U| integral now or at the
        # start (the transverse momenta start at zero), at least 1e-3 of the
        # largest variable's
        scale = np.maximum(np.maximum(M0, M), 1e-3 * M0.max())
        drift = np.abs(I - I0) / scale
        record(f"conserved integrals after cycle {c + 1}", drift, 1e-12)
        assert np.all(drift <= 1e-12), (c, drift)
    return seen_fv


def test_conservation_hp_shock_full_size_with_adaptation():
    """The hp-mixed shock case (16^3 elements, N in 2..6, FV sub-cells by the
    indicator): 8 cycles of adaptation + 5 SSP-RK3 steps at CFL 0.5."""
    from paper_2502_19342_gb300 import dgfv
    prob, U = W.hp_shock(0, y_bg=0.01)
    ctx = dgfv.Context(prob, N_min=2, N_max=6, opts=dict(cfl_c=0.5, cfl_v=0.5, thresholds=W.THRESHOLDS))
    ctx.set_state(to_dev(U))
    assert _run(prob, U, ctx, cycles=8, steps=5) > 0  # FV elements took part
    ctx.close()


def test_conservation_on_mortar_mesh_with_adaptation():
    """The half-refined cube (type-3 mortars on both x interfaces, random
    degrees and FV elements): 4 cycles of adaptation + 3 steps."""
    from paper_2502_19342_gb300 import dgfv
    prob, U = W.half_refined_wave(8)
    ctx = dgfv.Context(prob, N_min=1, N_max=7, opts=dict(cfl_c=0.5, cfl_v=0.5, thresholds=W.THRESHOLDS))
    ctx.set_state(to_dev(U))
    _run(prob, U, ctx, cycles=4, steps=3)
    ctx.close()
