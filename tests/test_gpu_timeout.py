"""Bounded device waits report DC_ERR_TIMEOUT and leave the context usable.

The tensor-core M2L of the chosen form's inner operator waits for its MMAs'
commit on an mbarrier with a time and poll limit.  The test hook
dc_aux_test_skip_mma_tile makes one CTA hold back the MMAs and the commit of
one tile, so nothing arrives on that mbarrier and the wait runs out (nothing
is in flight, nothing faults).  The solve must end with DC_ERR_TIMEOUT within
seconds, and once the hook is off the next solve must give the same density
as before, bit for bit."""
import time

import numpy as np
import pytest

from dc_synth import drawing_by_name

pytestmark = pytest.mark.gpu


def test_tensor_core_wait_limit_reports_timeout(dcmod, cuda_ok):
    P = dcmod
    d = drawing_by_name("mixed16")
    ctx = P.Context(form="fmm32", g=d.g, s_per_panel=d.s_per_panel, p=24, leaf_size=32,
                    gmres_tol=1e-10, p_inner=12, m2l_engine=P.DC_M2L_TENSOR)
    ctx.build_drawing(d)
    st = ctx.solve_density()
    assert st.converged == 1
    sig0 = ctx.get_density()
    ctx.test_skip_mma_tile(0)
    t0 = time.perf_counter()
    with pytest.raises(P.DcError) as e:
        ctx.solve_density()
    dt = time.perf_counter() - t0
    print(f"timed-out solve returned after {dt:.2f} s: {e.value}")
    assert e.value.status == P.DC_ERR_TIMEOUT
    assert dt < 10.0
    # the single operator application reports it too
    import torch
    x = torch.ones((ctx.sizes().n_nodes, 3), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(P.DcError) as e2:
        ctx.apply_operator(x, y, 0, 2)
    assert e2.value.status == P.DC_ERR_TIMEOUT
    ctx.test_skip_mma_tile(-1)
    st = ctx.solve_density()
    assert st.converged == 1
    assert np.array_equal(ctx.get_density(), sig0)
    ctx.close()


def test_skip_hook_argument_checks(dcmod, cuda_ok):
    P = dcmod
    d = drawing_by_name("closed4")
    ctx = P.Context(form="fmm32", g=d.g, s_per_panel=d.s_per_panel, m2l_engine=P.DC_M2L_CUDA_CORES)
    ctx.build_drawing(d)
    with pytest.raises(P.DcError) as e:
        ctx.test_skip_mma_tile(-2)
    assert e.value.status == P.DC_ERR_ARG
    with pytest.raises(P.DcError) as e:
        ctx.test_skip_mma_tile(0)
    assert e.value.status == P.DC_ERR_UNSUPPORTED
    ctx.close()
