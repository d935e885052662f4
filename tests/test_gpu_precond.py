"""The FMM forms' two-level preconditioner M (panel blocks of G_H inverted
plus a coarse space of panel constants; no counterpart in the paper): its
application through the ABI against its definition written out with numpy
from the oracle's dense G_H rows, and its effect on the solve."""
import numpy as np
import pytest

from dc_synth import drawing_by_name

pytestmark = pytest.mark.gpu

INV4PI = np.float32(0.0795774715459476679)


def reference_M(oracle_mod, d):
    """M v = P y + B (v - A~ P y), y = Ac^-1 R v: R sums a panel's nodes, P
    spreads, A~ P = exact (G_H 1_j) for near panel pairs (centroid distance
    below 1.5 (l_i + l_j)) and l_j G(q, c_j) with FP32 positions otherwise,
    Ac = R A~ P, B = inverse diagonal panel blocks."""
    disc = oracle_mod.discretise(d)
    AG, _ = oracle_mod.hybrid_rows(disc)
    N, g, P = disc.n_nodes, disc.g, disc.n_panels
    xy = disc.node_xy.reshape(P, g, 2)
    cen = xy.mean(axis=1)
    seg = disc.seg_xy.reshape(P, disc.nseg, 4)
    plen = (disc.seg_w.reshape(P, -1) * np.hypot(seg[..., 2] - seg[..., 0], seg[..., 3] - seg[..., 1])).sum(1)
    D = np.linalg.norm(cen[:, None] - cen[None], axis=2)
    near = D < 1.5 * (plen[:, None] + plen[None, :])
    APx = AG.reshape(N, P, g).sum(axis=2)
    q32 = disc.node_xy.astype(np.float32)
    c32 = cen.astype(np.float32)
    dxy = q32[:, None, :] - c32[None]
    mono = (-INV4PI * np.log(np.maximum((dxy * dxy).sum(2), np.float32(1e-30)))).astype(np.float64)
    AP = np.where(np.repeat(near, g, axis=0), APx, plen[None, :] * mono)
    Ac = AP.reshape(P, g, P).sum(axis=1)
    Aci = np.linalg.inv(Ac)
    blocks = np.stack([np.linalg.inv(AG[j * g:(j + 1) * g, j * g:(j + 1) * g]) for j in range(P)])

    def M(v):
        y = Aci @ v.reshape(P, g, -1).sum(axis=1)
        r = v - AP @ y
        return np.repeat(y, g, axis=0) + np.einsum("pij,pjc->pic", blocks, r.reshape(P, g, -1)).reshape(N, -1)
    return M, N


@pytest.mark.parametrize("form", ["fmm32", "fmm64"])
def test_two_level_preconditioner_matches_definition(dcmod, cuda_ok, oracle_mod, form):
    import torch
    d = drawing_by_name("mixed16")
    ctx = dcmod.Context(form=form, g=d.g, s_per_panel=d.s_per_panel, p=24, leaf_size=32)
    ctx.build_drawing(d)
    info = ctx.precond_info()
    print(info)
    assert info["two_level"] == 1.0 and info["panels"] == d.n_panels
    assert info["inverse_check"] < 1e-3
    M, N = reference_M(oracle_mod, d)
    v = np.random.default_rng(51).standard_normal((N, 3))
    got = torch.empty((N, 3), dtype=torch.float64, device="cuda")
    ctx.apply_operator(torch.from_numpy(v).cuda(), got, 0, 3)
    torch.cuda.synchronize()
    ref = M(v)
    rel = np.linalg.norm(got.cpu().numpy() - ref) / np.linalg.norm(ref)
    print(f"two-level M: relative difference to the definition {rel:.2e}")
    assert rel < 1e-3


def reference_M_aggregated(oracle_mod, d, coarse_max):
    """The aggregated form: K = ceil(P / (coarse_max - 32)) panels per
    aggregate, consecutive in the Morton order of the panel centroids (16
    bits per axis over the centroids' bounding box, y bit above x bit, ties
    by panel index); Ac = R_agg A~ P_agg with A~ as above; y = Ac^-1 R_agg v
    and M v = P_agg y + B (v - G_H P_agg y) with the exact G_H."""
    disc = oracle_mod.discretise(d)
    AG, _ = oracle_mod.hybrid_rows(disc)
    N, g, P = disc.n_nodes, disc.g, disc.n_panels
    cen = np.zeros((P, 2))
    for j in range(P):                  # node sums in node order, as written
        sx = sy = 0.0
        for m in range(g):
            sx += disc.node_xy[j * g + m, 0]
            sy += disc.node_xy[j * g + m, 1]
        cen[j] = (sx / g, sy / g)
    seg = disc.seg_xy.reshape(P, disc.nseg, 4)
    plen = (disc.seg_w.reshape(P, -1) * np.hypot(seg[..., 2] - seg[..., 0], seg[..., 3] - seg[..., 1])).sum(1)
    D = np.linalg.norm(cen[:, None] - cen[None], axis=2)
    near = D < 1.5 * (plen[:, None] + plen[None, :])
    APx = AG.reshape(N, P, g).sum(axis=2)
    q32 = disc.node_xy.astype(np.float32)
    c32 = cen.astype(np.float32)
    dxy = q32[:, None, :] - c32[None]
    mono = (-INV4PI * np.log(np.maximum((dxy * dxy).sum(2), np.float32(1e-30)))).astype(np.float64)
    AP = np.where(np.repeat(near, g, axis=0), APx, plen[None, :] * mono)
    K = -(-P // (coarse_max - 32))
    lo, hi = cen.min(0), cen.max(0)
    keys = []
    for j in range(P):
        q = [min(65535, int(np.floor((cen[j, a] - lo[a]) / (hi[a] - lo[a]) * 65536.0))) for a in range(2)]
        k = 0
        for b in range(15, -1, -1):
            k = (k << 2) | (((q[1] >> b) & 1) << 1) | ((q[0] >> b) & 1)
        keys.append((k, j))
    order = [j for _, j in sorted(keys)]
    nA = -(-P // K)
    agg_of = np.zeros(P, int)
    for u, j in enumerate(order):
        agg_of[j] = u // K
    S = np.zeros((P, nA))
    S[np.arange(P), agg_of] = 1.0                       # panel -> aggregate
    Ac = S.T @ (AP @ S).reshape(P, g, nA).sum(axis=1)   # [nA, nA]
    Aci = np.linalg.inv(Ac)
    blocks = np.stack([np.linalg.inv(AG[j * g:(j + 1) * g, j * g:(j + 1) * g]) for j in range(P)])

    def M(v):
        y = Aci @ (S.T @ v.reshape(P, g, -1).sum(axis=1))
        py = np.repeat(S @ y, g, axis=0)
        r = v - AG @ py
        return py + np.einsum("pij,pjc->pic", blocks, r.reshape(P, g, -1)).reshape(N, -1)
    return M, N, K, nA


@pytest.mark.parametrize("form", ["fmm32", "fmm64"])
def test_aggregated_preconditioner_matches_definition(dcmod, cuda_ok, oracle_mod, form):
    import torch
    d = drawing_by_name("mixed16")
    ctx = dcmod.Context(form=form, g=d.g, s_per_panel=d.s_per_panel, p=24, leaf_size=32, coarse_max=64)
    ctx.build_drawing(d)
    info = ctx.precond_info()
    M, N, K, nA = reference_M_aggregated(oracle_mod, d, 64)
    print(info, "reference K", K, "aggregates", nA)
    assert info["two_level"] == 1.0 and info["aggregate"] == K and info["panels"] == nA and K > 1
    v = np.random.default_rng(52).standard_normal((N, 3))
    got = torch.empty((N, 3), dtype=torch.float64, device="cuda")
    ctx.apply_operator(torch.from_numpy(v).cuda(), got, 0, 3)
    torch.cuda.synchronize()
    ref = M(v)
    rel = np.linalg.norm(got.cpu().numpy() - ref) / np.linalg.norm(ref)
    print(f"{form} aggregated M: relative difference to the definition {rel:.2e}")
    assert rel < 1e-3
    st = ctx.solve_density()
    assert st.converged == 1
