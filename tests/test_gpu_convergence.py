"""Convergence order of the CUDA path (Sec. 4.2): an advected density/species
wave (Euler limit, exact solution known) stepped with SSP-RK3 on the GPU at a
fixed small time step; the L2 error of rho_1 over two meshes gives order N+1
on uniform degrees, the order of the lowest degree present on a checkerboard
of degrees, and the second order of the FV scheme on a DG/FV checkerboard.
The same cases pin the oracle in tests/test_oracle_rhs.py."""
import numpy as np
import pytest

from paper_2502_19342_gb300 import workloads as W
from tests.gpu_helpers import to_dev
from tests.test_oracle_rhs import _order, _per_var, _weights

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _gpu_advected_l2(nel, N_of, fv_of=None, wave=(1, 0, 0), T=0.05, n_fv=7):
    from paper_2502_19342_gb300 import dgfv
    sp = W.species_set([W.AIR, W.HELIUM], mu=0.0)
    dims = tuple(nel)
    _, pos, _, _ = W.element_index(W.make_problem([(dims, (0, 0, 0), (1, 1, 1))], sp, n_fv=n_fv, N=1))
    N = np.array([N_of(*p) for p in pos], np.int8)
    fv = np.array([fv_of(*p) if fv_of else 0 for p in pos], np.uint8)
    hi = tuple(1.0 if wave[a] else 1.0 / nel[a] for a in range(3))
    prob = W.make_problem([(dims, (0, 0, 0), hi)], sp, n_fv=n_fv, N=N, fv=fv)
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
    ctx = dgfv.Context(prob, N_min=int(N.min()), N_max=int(N.max()))
    ctx.set_state(to_dev(U0))
    ctx.rk_steps(steps, T / steps, want_dt=False)
    U = ctx.get_state().cpu().numpy()
    ctx.close()
    Ue = W.build_state(prob, fn_t(T))
    e = _per_var(prob, U - Ue)[0]
    w = _per_var(prob, _weights(prob))[0]
    return np.sqrt((e ** 2 * w).sum() / w.sum())


def test_uniform_degree_3_diagonal_wave():
    e = [_gpu_advected_l2((k, k, k), lambda i, j, k_: 3, wave=(1, 1, 1)) for k in (4, 6)]
    assert _order(e[0], e[1], 4, 6) > 3.65, e


def test_uniform_degree_5():
    e = [_gpu_advected_l2((k, 1, 1), lambda i, j, k_: 5) for k in (8, 12)]
    assert _order(e[0], e[1], 8, 12) > 5.5, e


def test_checkerboard_degrees_take_the_lowest_order():
    dims = [(k, k, 1) for k in (8, 16)]
    e = [_gpu_advected_l2(d, lambda i, j, k_: (3, 5)[(i + j + k_) % 2], wave=(1, 1, 0)) for d in dims]
    order = _order(e[0], e[1], 8, 16)
    assert 3.65 < order < 5.5, (e, order)


def test_dg_fv_checkerboard_is_second_order():
    e = [_gpu_advected_l2((k, 1, 1), lambda i, j, k_: 2, fv_of=lambda i, j, k_: i % 2) for k in (32, 64)]
    assert _order(e[0], e[1], 32, 64) > 1.8, e
