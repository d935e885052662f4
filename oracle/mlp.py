"""FP64 CPU oracle of the learned warm start: the panel features and the
4-layer GELU perceptron with its mean-squared-error gradient.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, never by the product
path, and shares no code with the CUDA library.

The warm start has no counterpart in the paper (whose warm start, Sec. 6.1,
re-uses an earlier solution); the definitions below are the library's own,
as its C header states them:

  * features of panel j, colour channel c, in the panel frame (origin at the
    centroid of the panel's nodes, x axis along the chord from its first to
    its last node, lengths divided by the panel's arc length l_j, the sum of
    its segments' arc lengths, App. A):
      own nodes (x, y, n_x, n_y) node by node, n the right-hand normal of
      the node's own segment; own u+ then u- of channel c at the g nodes;
      for each of the 8 nearest other panels by node centroid, nearest
      first: its u+ then u- of channel c; then for each of them its centroid
      offset and chord direction (2 + 2) in the frame;
  * target: l_j sigma of channel c at the panel's g nodes;
  * network: n_in -> H -> H -> H -> n_out, GELU(z) = z Phi(z) after the
    first three layers, parameters W_l [out][in] then b_l [out] per layer;
    the network reads the weights rounded to BF16 (round to nearest even)
    and the biases unrounded; loss = mean over rows and outputs of
    (y - t)^2.

Pins (tests/test_oracle_mlp.py): the gradient against FP64 central finite
differences, GELU against its closed values, the features' invariance under
rotation, translation and uniform scaling of the drawing (and their change
under a reflection), the arc lengths against the curve lengths, the Adam
step's first move, and the nearest-panel lists on a hand-checked layout.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

N_NBR = 8
LAYERS = 4


def n_features(g: int) -> int:
    return 22 * g + 32


# ------------------------------------------------------------- network --
def bf16_round(a) -> np.ndarray:
    """float32 values rounded to the nearest BF16 (ties to even), as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def dims(n_in: int, hidden: int, n_out: int):
    return [n_in, hidden, hidden, hidden, n_out]


def param_count(n_in: int, hidden: int, n_out: int) -> int:
    d = dims(n_in, hidden, n_out)
    return sum(d[l + 1] * d[l] + d[l + 1] for l in range(LAYERS))


def unpack(params, n_in, hidden, n_out):
    d = dims(n_in, hidden, n_out)
    out, o = [], 0
    for l in range(LAYERS):
        W = params[o:o + d[l + 1] * d[l]].reshape(d[l + 1], d[l])
        o += d[l + 1] * d[l]
        b = params[o:o + d[l + 1]]
        o += d[l + 1]
        out.append((W, b))
    return out


def forward(params, x, n_in, hidden, n_out, round_bf16=True):
    """Network output [rows][n_out] and the per-layer values for backward."""
    p = np.asarray(params, dtype=np.float64)
    layers = unpack(p, n_in, hidden, n_out)
    a = np.asarray(x, dtype=np.float64)
    acts, pre, Ws = [a], [], []
    for l, (W, b) in enumerate(layers):
        Wr = bf16_round(W) if round_bf16 else W
        z = a @ Wr.T + b
        pre.append(z)
        Ws.append(Wr)
        a = gelu(z) if l + 1 < LAYERS else z
        acts.append(a)
    return a, (acts, pre, Ws)


def loss_grad(params, x, target, n_in, hidden, n_out, round_bf16=True):
    """Loss and its gradient with respect to the parameters (the weights as
    the network reads them), by the chain rule layer by layer."""
    y, (acts, pre, Ws) = forward(params, x, n_in, hidden, n_out, round_bf16)
    t = np.asarray(target, dtype=np.float64)
    n = y.size
    loss = np.sum((y - t) ** 2) / n
    d = 2.0 * (y - t) / n                         # dL/dz of the last layer
    grads = []
    for l in range(LAYERS - 1, -1, -1):
        if l + 1 < LAYERS:
            d = d * gelu_grad(pre[l])
        grads.append((d.T @ acts[l], d.sum(axis=0)))
        d = d @ Ws[l]
    g = []
    for dW, db in reversed(grads):
        g.append(dW.ravel())
        g.append(db)
    return loss, np.concatenate(g)


def adam_step(p, g, m, v, lr, beta1, beta2, eps, step):
    """One Adam update (Kingma and Ba 2015, Algorithm 1) in place on m and v;
    returns the new parameters."""
    m *= beta1
    m += (1.0 - beta1) * g
    v *= beta2
    v += (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps)


# ------------------------------------------------------------ features --
def panel_frames(disc):
    """Per panel: node centroid [P,2], chord direction [P,2], arc length [P]."""
    P, g, s = disc.n_panels, disc.g, disc.nseg
    nodes = disc.node_xy.reshape(P, g, 2)
    cen = nodes.mean(axis=1)
    chord = nodes[:, -1] - nodes[:, 0]
    seg = disc.seg_xy.reshape(P, s, 4)
    if g == 1:
        chord = seg[:, -1, 2:4] - seg[:, 0, 0:2]
    tdir = chord / np.linalg.norm(chord, axis=1, keepdims=True)
    seglen = np.hypot(seg[..., 2] - seg[..., 0], seg[..., 3] - seg[..., 1])
    plen = (disc.seg_w.reshape(P, s) * seglen).sum(axis=1)
    return cen, tdir, plen


def nearest_panels(cen, k=N_NBR):
    """Indices of the k nearest other centroids, nearest first (brute force)."""
    d2 = ((cen[:, None, :] - cen[None, :, :]) ** 2).sum(axis=2)
    np.fill_diagonal(d2, np.inf)
    order = np.argsort(d2, axis=1, kind="stable")[:, :k]
    out = np.full((cen.shape[0], k), -1, dtype=np.int64)
    m = min(k, cen.shape[0] - 1)
    out[:, :m] = order[:, :m]
    return out


def node_normals(disc):
    seg = disc.seg_xy[disc.node_seg]
    dx, dy = seg[:, 2] - seg[:, 0], seg[:, 3] - seg[:, 1]
    d = np.hypot(dx, dy)
    return np.stack([dy / d, -dx / d], axis=1)


def panel_features(disc, u_plus, u_minus, sigma=None):
    """Features [3P, 22g+32] and, with sigma, targets [3P, g] (FP64)."""
    P, g = disc.n_panels, disc.g
    cen, tdir, plen = panel_frames(disc)
    nbr = nearest_panels(cen)
    nrm = node_normals(disc).reshape(P, g, 2)
    xy = disc.node_xy.reshape(P, g, 2)
    up = u_plus.reshape(P, g, 3)
    um = u_minus.reshape(P, g, 3)
    F = n_features(g)
    feat = np.zeros((3 * P, F))
    target = np.zeros((3 * P, g)) if sigma is not None else None

    def to_frame(v, j):                      # v [..., 2] direction in panel j's frame
        tx, ty = tdir[j]
        return np.stack([v[..., 0] * tx + v[..., 1] * ty, -v[..., 0] * ty + v[..., 1] * tx], axis=-1)

    for j in range(P):
        own_p = to_frame((xy[j] - cen[j]) / plen[j], j)
        own_n = to_frame(nrm[j], j)
        geo_own = np.concatenate([own_p, own_n], axis=1).ravel()        # node by node x y nx ny
        geo_nb = np.zeros(4 * N_NBR)
        for k in range(N_NBR):
            q = nbr[j, k]
            if q >= 0:
                geo_nb[4 * k:4 * k + 2] = to_frame((cen[q] - cen[j]) / plen[j], j)
                geo_nb[4 * k + 2:4 * k + 4] = to_frame(tdir[q], j)
        for c in range(3):
            r = 3 * j + c
            col_nb = np.zeros(2 * g * N_NBR)
            for k in range(N_NBR):
                q = nbr[j, k]
                if q >= 0:
                    col_nb[2 * g * k:2 * g * k + g] = up[q, :, c]
                    col_nb[2 * g * k + g:2 * g * (k + 1)] = um[q, :, c]
            feat[r] = np.concatenate([geo_own, up[j, :, c], um[j, :, c], col_nb, geo_nb])
            if sigma is not None:
                target[r] = sigma.reshape(P, g, 3)[j, :, c] * plen[j]
    return feat, target
