"""dc_eval_points_noalloc: the allocation-free variant of dc_eval_points.

Some callers cannot allocate device memory while they run (a frame loop
whose memory another framework owns, code held to a fixed budget); this
entry point keeps its scratch in a fixed device array instead.  Its results
must equal those of dc_eval_points through the ordinary path (the plain
FP64 direct sum), on consecutive calls and across contexts that share the
array, and oversize drawings must be refused.  This file is collected last
so that a failure here cannot hide failures elsewhere.
"""
import numpy as np
import pytest

from dc_synth import drawing_by_name, random_node_values

pytestmark = pytest.mark.gpu

TOL = 1e-10


def dense_ctx(P, name, **kw):
    d = drawing_by_name(name)
    ctx = P.Context(form="dense64", g=d.g, s_per_panel=kw.pop("s_per_panel", d.s_per_panel),
                    gmres_tol=1e-12, gmres_restart=400, **kw)
    ctx.build_drawing(d)
    return d, ctx


def points(seed, n):
    import torch
    rng = np.random.default_rng(seed)
    return torch.tensor(rng.uniform(0.0, 1.0, (n, 2)), dtype=torch.float64, device="cuda")


def reference(ctx, xy):
    import torch
    out = torch.empty((xy.shape[0], 3), dtype=torch.float64, device="cuda")
    ctx.eval_points(xy, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def noalloc(ctx, xy):
    import torch
    out = torch.full((xy.shape[0], 3), float("nan"), dtype=torch.float64, device="cuda")
    ctx.eval_points_noalloc(xy, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_eval_points_on_consecutive_calls(dcmod, cuda_ok):
    import torch
    _, ctx = dense_ctx(dcmod, "closed4")
    ctx.solve_density()
    xy1, xy2 = points(1, 777), points(2, 1500)
    ref1, ref2 = reference(ctx, xy1), reference(ctx, xy2)
    # the first call on a device looks up the scratch array (the runtime may
    # load the array's module then); memory is compared after it
    noalloc(ctx, points(9, 4))
    # every tensor is allocated before the first reading, so only the
    # library's two calls fall between the readings
    out1 = torch.full((xy1.shape[0], 3), float("nan"), dtype=torch.float64, device="cuda")
    out2 = torch.full((xy2.shape[0], 3), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ctx.eval_points_noalloc(xy1, out1)
    ctx.eval_points_noalloc(xy2, out2)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    np.testing.assert_allclose(out1.cpu().numpy(), ref1, rtol=TOL, atol=TOL)
    np.testing.assert_allclose(out2.cpu().numpy(), ref2, rtol=TOL, atol=TOL)
    assert free1 == free0          # nothing was allocated on the device


def test_noalloc_shared_scratch_across_contexts(dcmod, cuda_ok):
    _, a = dense_ctx(dcmod, "closed4")
    a.solve_density()
    d, b = dense_ctx(dcmod, "mixed16")
    b.set_density(random_node_values(d.n_nodes, seed=4))
    xy = points(3, 600)
    ra, rb = reference(a, xy), reference(b, xy)
    np.testing.assert_allclose(noalloc(a, xy), ra, rtol=TOL, atol=TOL)
    np.testing.assert_allclose(noalloc(b, xy), rb, rtol=TOL, atol=TOL)
    np.testing.assert_allclose(noalloc(a, xy), ra, rtol=TOL, atol=TOL)


def test_noalloc_refuses_oversize_drawings(dcmod, cuda_ok):
    import torch
    P = dcmod
    d, ctx = dense_ctx(P, "mixed16", s_per_panel=1800)     # 151 panels x 1800 > 262,144
    assert ctx.sizes().n_segments > 262144
    ctx.set_density(random_node_values(d.n_nodes, seed=5))
    xy = points(6, 16)
    out = torch.zeros((16, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(P.DcError) as e:
        ctx.eval_points_noalloc(xy, out)
    assert e.value.status == P.DC_ERR_ARG
    assert "262144" in str(e.value)
