"""The allocation-free time step (dgfv_compute_dt_noalloc) against the regular
one (dgfv_compute_dt).

Some callers cannot allocate device memory at the moment they need a time
step -- a latency-critical loop where cudaMalloc would synchronise the
device, or a host that owns all device memory after start-up -- so the
library offers this one entry point whose scratch is a fixed device array.
This file is collected last, so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2502_19342_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

RTOL = 1e-14  # the same kernel and reduction order as dgfv_compute_dt


def _problem(seed, nk):
    sp = W.species_set([W.AIR, W.HELIUM, W.CO2][:nk], mu=2e-3)
    n = 4 * 3 * 5
    prob = W.make_problem([((4, 3, 5), (0, 0, 0), (1.0, 0.8, 1.2))], sp, n_fv=8,
                          N=W.random_degrees(n, 1, 7, seed), fv=W.random_fv(n, 0.25, seed))
    return prob, W.smooth_random_state(prob, seed, amp=0.1)


def test_noalloc_time_step_matches_regular_entry_point_twice_in_a_row():
    from paper_2502_19342_gb300 import dgfv
    L = dgfv.lib()
    prob, U1 = _problem(3, 3)
    ctx = dgfv.Context(prob, N_min=1, N_max=7, opts=dict(cfl_c=0.5, cfl_v=0.4))
    U2 = W.smooth_random_state(prob, 4, amp=0.2)  # a second input for the second call
    out = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
    for U in (U1, U2):
        Ud = torch.from_numpy(U).cuda()
        ref = ctx.compute_dt(Ud)
        stream = torch.cuda.current_stream()
        rc = L.dgfv_compute_dt_noalloc(ctx.h, ctypes.c_void_p(Ud.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, dgfv.lib().dgfv_last_error(ctx.h)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, np.array(ref), rtol=RTOL)
    # a warm call takes no device memory: the free bytes the driver reports
    # are the same before and after it
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    rc = L.dgfv_compute_dt_noalloc(ctx.h, ctypes.c_void_p(Ud.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0
    assert torch.cuda.mem_get_info()[0] == free0
    ctx.close()


def test_noalloc_time_step_refuses_more_work_tiles_than_its_scratch():
    """The fixed scratch holds the partial results of 65536 blocks (one per
    work tile).  At N = 7 every element is a tile of its own, so 41 x 40 x 40
    = 65600 elements need more: the call returns DGFV_ERR_ARG with a message
    and launches nothing; the regular entry point still works."""
    from paper_2502_19342_gb300 import dgfv
    L = dgfv.lib()
    sp = W.species_set([W.AIR], mu=1e-3)
    prob = W.make_problem([((41, 40, 40), (0, 0, 0), (1.0, 1.0, 1.0))], sp, n_fv=8, N=7)
    ctx = dgfv.Context(prob, N_min=7, N_max=7)
    U = torch.zeros(ctx.state_size, dtype=torch.float64, device="cuda")
    U.view(-1, 5, 512)[:, 0] = 1.0           # rho
    U.view(-1, 5, 512)[:, 4] = 2.5           # rho E: p = 1 at rest
    out = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
    rc = L.dgfv_compute_dt_noalloc(ctx.h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1  # DGFV_ERR_ARG
    msg = L.dgfv_last_error(ctx.h).decode()
    assert "65600" in msg and "65536" in msg, msg
    torch.cuda.synchronize()
    assert (out.cpu().numpy() == -1.0).all()
    dt = ctx.compute_dt(U)
    assert np.isfinite(dt[0]) and dt[0] > 0
    ctx.close()
