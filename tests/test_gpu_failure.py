"""Failure detection of the CUDA path, in forms that fault no GPU: a state
corrupted on the host goes in through the C ABI, the Runge-Kutta stage kernel
notices it at a node and records the first error and its element in the
device status word, and the next synchronising call returns the error code.
Nothing traps or waits; a clean state set afterwards goes on as before.
"""
import numpy as np
import pytest

from paper_2502_19342_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

NONPHYSICAL, NONFINITE = -4, -5


def _element_of(msg):
    tail = msg.split("(element ")[1]
    return int(tail.split(")")[0])


def test_nonfinite_state_is_reported_and_a_clean_state_recovers():
    from paper_2502_19342_gb300 import dgfv
    prob, U = W.plain_tiny(0)
    ctx = dgfv.Context(prob)
    Ud = torch.from_numpy(U).cuda()
    ctx.set_state(Ud)
    dt = ctx.rk_step(-1.0)
    ref = ctx.get_state().cpu().numpy()
    # a NaN in one node of element 37
    off, _ = W.offsets(prob)
    bad = U.copy()
    n3 = (int(prob["N"][37]) + 1) ** 3
    bad[off[37] + 3 * n3 + 5] = np.nan
    ctx.set_state_host(bad)
    with pytest.raises(dgfv.DgfvError) as ei:
        ctx.rk_step(dt)
    assert ei.value.code == NONFINITE
    assert _element_of(str(ei.value)) >= 0
    ctx.sync_status()  # the report cleared the status word
    # a clean state: the same step as before the corruption
    ctx.set_state(Ud)
    assert ctx.rk_step(dt) == dt
    np.testing.assert_array_equal(ctx.get_state().cpu().numpy(), ref)
    ctx.close()


def test_nonphysical_stage_is_reported_with_its_element(oracle):
    """One element with a strong velocity divergence and a fixed step of about
    3.4 CFL steps: the first stage U + dt R(U) stays finite, but its internal
    energy rho E - |rho v|^2/(2 rho) (and so p) drops below zero.  The oracle
    names the elements where that happens; the reported element is one of them."""
    from paper_2502_19342_gb300 import dgfv
    sp = W.species_set([W.AIR, W.HELIUM], mu=1e-3)
    prob = W.make_problem([((4, 4, 4), (0, 0, 0), (1, 1, 1))], sp, n_fv=4, N=2)

    def fn(x, y, z):
        inside = (np.abs(x - 0.375) < 0.125) & (np.abs(y - 0.375) < 0.125) & (np.abs(z - 0.375) < 0.125)
        vx = np.where(inside, 6.0 * (x - 0.375) / 0.125, 0.0)
        return [0.7 + 0 * x, 0.3 + 0 * x], (vx, 0 * x, 0 * x), 1.0 + 0 * x

    U = W.build_state(prob, fn)
    dt = 0.01
    U1 = U + dt * oracle.eval_rhs(prob, U)  # the first SSP-RK3 stage
    assert np.isfinite(U1).all()
    off, _ = W.offsets(prob)
    expect = set()
    for e in range(W.n_elements(prob)):
        b = U1[off[e]:off[e] + 6 * 27].reshape(6, 27)
        rho = b[:2].sum(0)
        if (rho <= 0).any() or ((2 * rho * b[5] - (b[2:5] ** 2).sum(0)) <= 0).any():
            expect.add(e)
    assert expect, "the input must drive the first stage non-physical"
    ctx = dgfv.Context(prob)
    ctx.set_state(torch.from_numpy(U).cuda())
    with pytest.raises(dgfv.DgfvError) as ei:
        ctx.rk_step(dt)
    assert ei.value.code == NONPHYSICAL
    assert _element_of(str(ei.value)) in expect
    # recovery: a uniform state steps cleanly
    U0 = W.constant_state(prob, [0.7, 0.3], (0.2, 0.1, 0.0), 1.0)
    ctx.set_state(torch.from_numpy(U0).cuda())
    ctx.rk_step(-1.0)
    got = ctx.get_state().cpu().numpy()
    np.testing.assert_allclose(got, U0, rtol=0, atol=1e-13)
    ctx.close()
