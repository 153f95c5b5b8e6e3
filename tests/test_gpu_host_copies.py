"""State copies between the context and host buffers: page-locked buffers go
through the SM copy kernel (16-byte accesses when both pointers allow them,
8-byte ones otherwise, the odd last element of an odd-sized state), pageable
ones through cudaMemcpyAsync.  Every path returns the state bit for bit."""
import numpy as np
import pytest

from paper_2502_19342_gb300 import workloads as W
from tests.gpu_helpers import ctx_for, to_dev

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _odd_problem():
    sp = W.species_set([W.AIR], mu=1e-3)
    prob = W.make_problem([((3, 1, 1), (0, 0, 0), (1.0, 0.4, 0.4))], sp, n_fv=4, N=2)
    U = W.smooth_random_state(prob, 3, amp=0.1)
    assert U.size % 2 == 1  # 3 elements x 27 nodes x 5 variables
    return prob, U


@pytest.mark.parametrize("kind", ["pinned", "pinned_offset", "pageable"])
def test_host_state_round_trip(kind):
    prob, U = _odd_problem()
    ctx = ctx_for(prob, N_min=1, N_max=2)
    n = ctx.state_size
    assert n == U.size
    if kind == "pinned":
        src = torch.from_numpy(U.copy()).pin_memory()
        dst = torch.zeros(n, dtype=torch.float64).pin_memory()
        assert src.data_ptr() % 16 == 0 and dst.data_ptr() % 16 == 0
    elif kind == "pinned_offset":
        a = torch.zeros(n + 1, dtype=torch.float64).pin_memory()
        a[1:] = torch.from_numpy(U)
        src = a[1:]
        b = torch.zeros(n + 1, dtype=torch.float64).pin_memory()
        dst = b[1:]
        assert src.data_ptr() % 16 == 8 and src.is_pinned()
    else:
        src = torch.from_numpy(U.copy())
        dst = torch.zeros(n, dtype=torch.float64)
        assert not src.is_pinned()
    ctx.set_state_host(src)
    np.testing.assert_array_equal(ctx.get_state().cpu().numpy(), U)
    ctx.get_state_host(dst)
    np.testing.assert_array_equal(dst.numpy(), U)
    ctx.close()


def test_host_copy_of_a_full_size_state():
    """The 28^3 turbulence state (tens of millions of doubles) through a pinned
    buffer, after a few steps of GPU work: bit for bit both ways."""
    from paper_2502_19342_gb300 import dgfv
    import bench
    prob, U = bench.workload(28, seed=1)
    ctx = dgfv.Context(prob, N_min=1, N_max=7, opts=dict(cfl_c=0.5, cfl_v=0.5))
    Ud = to_dev(U)
    ctx.set_state(Ud)
    ctx.rk_steps(2, -1.0, want_dt=False)
    ref = ctx.get_state().cpu()
    host = torch.empty(ref.numel(), dtype=torch.float64).pin_memory()
    ctx.get_state_host(host)
    assert torch.equal(host, ref)
    host.mul_(-1.0)
    ctx.set_state_host(host)
    assert torch.equal(ctx.get_state().cpu(), -ref)
    ctx.close()
