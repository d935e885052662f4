"""The FP32 inner operator of the chosen form through the C ABI: G_H at order
p_i (M2L on the tensor cores, tcgen05 TF32 with the three-term split, for
p_i <= 15; on the CUDA cores above or when asked) against the FP64 operator at order p on
the same vector, and the captured graph G_H M against the FP32 operator
applied to the preconditioner's output."""
import numpy as np
import pytest

from dc_synth import drawing_by_name, random_node_values

pytestmark = pytest.mark.gpu


def _ctx(P, d, p_inner, engine=0):
    ctx = P.Context(form="fmm32", g=d.g, s_per_panel=d.s_per_panel, p=24, leaf_size=32,
                    gmres_tol=1e-10, gmres_restart=200, gmres_max_iter=3000, p_inner=p_inner,
                    m2l_engine=engine)
    ctx.build_drawing(d)
    return ctx


@pytest.mark.parametrize("p_inner,engine", [(12, 0), (15, 0), (12, 1), (16, 0)])
def test_fp32_operator_matches_fp64(dcmod, cuda_ok, p_inner, engine):
    import torch
    d = drawing_by_name("mixed16")
    ctx = _ctx(dcmod, d, p_inner, engine)
    n = ctx.sizes().n_nodes
    x = torch.from_numpy(random_node_values(n, seed=31, scale=1.0)).cuda()
    y64 = torch.empty_like(x)
    y32 = torch.empty_like(x)
    ctx.apply_operator(x, y64, 0, 0)
    ctx.apply_operator(x, y32, 0, 2)
    torch.cuda.synchronize()
    rel = (torch.linalg.norm(y32 - y64, dim=0) / torch.linalg.norm(y64, dim=0)).cpu().numpy()
    print(f"p_inner {p_inner} engine {engine}: FP32 operator vs FP64, relative error per channel {rel}")
    assert np.all(rel < 2e-6)


def test_graph_equals_operator_after_preconditioner(dcmod, cuda_ok):
    import torch
    d = drawing_by_name("mixed16")
    ctx = _ctx(dcmod, d, 12)
    n = ctx.sizes().n_nodes
    v = torch.from_numpy(random_node_values(n, seed=32, scale=1.0)).cuda()
    w = torch.empty_like(v)
    y_graph = torch.empty_like(v)
    y_two = torch.empty_like(v)
    ctx.apply_operator(v, y_graph, 0, 1)      # G_H M v in one captured graph
    ctx.apply_operator(v, w, 0, 3)            # M v
    ctx.apply_operator(w, y_two, 0, 2)        # G_H (M v)
    torch.cuda.synchronize()
    scale = torch.linalg.norm(y_two).item()
    assert torch.isfinite(y_graph).all()
    assert torch.linalg.norm(y_graph - y_two).item() <= 1e-12 * scale
