"""Seeded generators of cubic-Bezier diffusion-curve drawings.

Conventions shared by every consumer of a :class:`Drawing`:

* ``ctrl[i]`` holds the four control points C0..C3 of curve i; a closed
  curve has C3 == C0 exactly.
* ``colours[i, side, end, rgb]``: side 0 is the "+" side (to the right of the
  direction of travel, where the right-hand normal points), side 1 the "-"
  side; end 0 is the colour at Bezier parameter t = 0, end 1 at t = 1.  The
  colour along a curve is linear in t between the two ends.
* Panels of curve i are ``panel_start[panel_ptr[i]:panel_ptr[i+1]]``:
  increasing arc-length fractions in [0, 1) where each panel begins; a panel
  ends where the next begins (or at 1).  All fractions are dyadic rationals,
  so they are exact in binary floating point.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_POLY_SAMPLES = 256          # polyline points per curve for acceptance tests


@dataclass
class Drawing:
    name: str
    ctrl: np.ndarray          # [n, 4, 2] float64
    closed: np.ndarray        # [n] bool
    colours: np.ndarray       # [n, 2, 2, 3] float64
    panel_ptr: np.ndarray     # [n + 1] int32
    panel_start: np.ndarray   # [n_panels] float64
    g: int = 16               # Gauss-Legendre nodes per panel
    s_per_panel: int = 80     # solve segments per panel (5 g)
    meta: dict = field(default_factory=dict)

    @property
    def n_curves(self) -> int:
        return int(self.ctrl.shape[0])

    @property
    def n_panels(self) -> int:
        return int(self.panel_start.shape[0])

    @property
    def n_nodes(self) -> int:
        return self.n_panels * self.g

    @property
    def n_segments(self) -> int:
        return self.n_panels * self.s_per_panel


# ---------------------------------------------------------------- sampling --
def _polyline(c: np.ndarray, m: int = _POLY_SAMPLES) -> np.ndarray:
    """Dense sample of one cubic Bezier curve (acceptance tests only)."""
    t = np.linspace(0.0, 1.0, m)[:, None]
    u = 1.0 - t
    return (u ** 3) * c[0] + 3 * t * u * u * c[1] + 3 * t * t * u * c[2] + (t ** 3) * c[3]


def _speed_samples(c: np.ndarray, m: int = _POLY_SAMPLES) -> np.ndarray:
    t = np.linspace(0.0, 1.0, m)[:, None]
    u = 1.0 - t
    d = 3 * (u * u * (c[1] - c[0]) + 2 * t * u * (c[2] - c[1]) + t * t * (c[3] - c[2]))
    return np.hypot(d[:, 0], d[:, 1])


def _seg_intersect(a0, a1, b0, b1) -> np.ndarray:
    """Proper intersection test between segment sets (broadcast)."""
    def orient(p, q, r):
        return (q[..., 0] - p[..., 0]) * (r[..., 1] - p[..., 1]) - \
               (q[..., 1] - p[..., 1]) * (r[..., 0] - p[..., 0])
    d1 = orient(b0, b1, a0)
    d2 = orient(b0, b1, a1)
    d3 = orient(a0, a1, b0)
    d4 = orient(a0, a1, b1)
    return (d1 * d2 < 0) & (d3 * d4 < 0)


def _self_intersects(poly: np.ndarray, closed: bool) -> bool:
    a0, a1 = poly[:-1], poly[1:]
    n = a0.shape[0]
    hit = _seg_intersect(a0[:, None], a1[:, None], a0[None, :], a1[None, :])
    idx = np.arange(n)
    near = np.abs(idx[:, None] - idx[None, :]) <= 1
    if closed:
        near |= (idx[:, None] == 0) & (idx[None, :] == n - 1)
        near |= (idx[:, None] == n - 1) & (idx[None, :] == 0)
    return bool(np.any(hit & ~near))


def _point_seg_dist(p: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Distances from points p[:, None] to segments (a, b)[None, :]."""
    ab = b - a
    ap = p[:, None, :] - a[None, :, :]
    den = np.maximum(np.sum(ab * ab, axis=-1), 1e-300)
    t = np.clip(np.sum(ap * ab[None], axis=-1) / den[None], 0.0, 1.0)
    d = ap - t[..., None] * ab[None]
    return np.hypot(d[..., 0], d[..., 1])


def _poly_dist(pa: np.ndarray, pb: np.ndarray) -> float:
    d1 = _point_seg_dist(pa, pb[:-1], pb[1:]).min()
    d2 = _point_seg_dist(pb, pa[:-1], pa[1:]).min()
    return float(min(d1, d2))


def _closer_than(pa: np.ndarray, pb: np.ndarray, gap: float) -> bool:
    """_poly_dist(pa, pb) < gap, evaluated on the parts of the polylines that
    can decide it: points of one within the other's bounding box grown by
    gap, against the segments of the other whose boxes come within gap of
    those points (any pair closer than gap survives this restriction)."""
    def part(p, q):
        lo, hi = q.min(0) - gap, q.max(0) + gap
        pts = p[np.all((p >= lo) & (p <= hi), axis=1)]
        if pts.size == 0:
            return np.inf
        a, b = q[:-1], q[1:]
        slo, shi = np.minimum(a, b), np.maximum(a, b)
        plo, phi = pts.min(0) - gap, pts.max(0) + gap
        keep = np.all((shi >= plo) & (slo <= phi), axis=1)
        if not keep.any():
            return np.inf
        return float(_point_seg_dist(pts, a[keep], b[keep]).min())
    return min(part(pa, pb), part(pb, pa)) < gap


def _acceptable_shape(c: np.ndarray, closed: bool, poly: np.ndarray, check_samples: int = 0) -> bool:
    sp = _speed_samples(c)
    if sp.min() < 0.15 * sp.mean():              # avoid (near-)cusps
        return False
    if closed:
        v1, v2 = c[1] - c[0], c[2] - c[0]
        cosang = np.dot(v1, v2) / (np.linalg.norm(v1) * np.linalg.norm(v2) + 1e-300)
        if cosang > np.cos(np.deg2rad(20.0)):    # corner too sharp
            return False
    if check_samples:                            # a coarser polyline for the crossing test
        poly = _polyline(c, check_samples)
    return not _self_intersects(poly, closed)


class _Placer:
    """Accepts curves one at a time if they keep a minimum gap to the others.
    Candidates are found through a uniform grid of bounding boxes (the same
    box test and distance test as a scan over every placed curve, in the
    same order, so the decisions do not depend on the grid)."""

    def __init__(self, min_gap: float, cell: float = 0.05):
        self.min_gap = min_gap
        self.cell = cell
        self.polys: list[np.ndarray] = []
        self.boxes: list[np.ndarray] = []
        self.grid: dict[tuple[int, int], list[int]] = {}

    def _cells(self, lo, hi):
        i0, j0 = np.floor(lo / self.cell).astype(int)
        i1, j1 = np.floor(hi / self.cell).astype(int)
        for i in range(i0, i1 + 1):
            for j in range(j0, j1 + 1):
                yield (i, j)

    def fits(self, poly: np.ndarray, ignore: int = -1) -> bool:
        lo, hi = poly.min(0) - self.min_gap, poly.max(0) + self.min_gap
        cand = set()
        for key in self._cells(lo, hi):
            cand.update(self.grid.get(key, ()))
        for k in sorted(cand):
            if k == ignore:
                continue
            q, (qlo, qhi) = self.polys[k], self.boxes[k]
            if np.any(hi < qlo) or np.any(qhi < lo):
                continue
            if _closer_than(poly, q, self.min_gap):
                return False
        return True

    def add(self, poly: np.ndarray) -> None:
        k = len(self.polys)
        self.polys.append(poly)
        box = np.stack([poly.min(0), poly.max(0)])
        self.boxes.append(box)
        for key in self._cells(box[0], box[1]):
            self.grid.setdefault(key, []).append(k)


def _colours(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.uniform(0.0, 1.0, size=(n, 2, 2, 3))


def _uniform_panels(n: int, per_curve: int):
    ptr = np.arange(n + 1, dtype=np.int32) * per_curve
    start = np.tile(np.arange(per_curve, dtype=np.float64) / per_curve, n)
    return ptr, start


def _nearest_other_curve(polys: list[np.ndarray]) -> list[np.ndarray]:
    """For every polyline sample, the distance to the nearest sample of
    another curve (infinite for a single curve).  Per curve, only curves
    whose bounding box lies within a radius R of its own are searched (a k-d
    tree over their samples); R doubles until every sample's nearest is
    within R, so the result is the exact minimum over all other curves."""
    from scipy.spatial import cKDTree
    n = len(polys)
    if n == 1:
        return [np.full(polys[0].shape[0], np.inf)]
    lo = np.array([p.min(0) for p in polys])
    hi = np.array([p.max(0) for p in polys])
    span = float(max((hi - lo).max(), 1e-12))
    out = []
    for i, p in enumerate(polys):
        gap = np.maximum(0.0, np.maximum(lo - hi[i], lo[i] - hi))   # box-to-box gaps [n, 2]
        bd = np.hypot(gap[:, 0], gap[:, 1])
        bd[i] = np.inf
        R = max(float(bd.min()), 0.0) + span
        while True:
            cand = np.flatnonzero(bd <= R)
            d, _ = cKDTree(np.concatenate([polys[j] for j in cand])).query(p)
            if d.max() <= R or cand.size == n - 1:
                break
            R *= 2.0
        out.append(d)
    return out


def _adaptive_panels(polys: list[np.ndarray], ratio: float, max_level: int,
                     min_panels: int, max_len: float):
    """Bisect panels (in arc-length fraction) until each panel's length is at
    most ``ratio`` x its distance to the nearest other curve.  Lengths and
    distances are measured on the dense polylines (point-to-point, so within
    one sample spacing); break points are dyadic."""
    dists = _nearest_other_curve(polys)
    ptr = [0]
    starts: list[float] = []
    for i, p in enumerate(polys):
        seg = np.hypot(*np.diff(p, axis=0).T)
        cum = np.concatenate([[0.0], np.cumsum(seg)])
        L = cum[-1]
        frac = cum / L
        dpt = dists[i]
        stack = [(0.0, 1.0, 0)]
        out: list[float] = []
        while stack:
            a, b, lev = stack.pop()
            ia = int(np.searchsorted(frac, a, side="left"))
            ib = int(np.searchsorted(frac, b, side="right"))
            lo_i, hi_i = max(ia - 1, 0), min(ib + 1, len(frac))
            d = float(dpt[lo_i:hi_i].min())
            length = (b - a) * L
            need = lev < max_level and (
                (b - a) > 1.0 / min_panels + 1e-15
                or length > max_len
                or length > ratio * d)
            if need:
                mid = 0.5 * (a + b)
                stack.append((mid, b, lev + 1))
                stack.append((a, mid, lev + 1))
            else:
                out.append(a)
        out.sort()
        starts.extend(out)
        ptr.append(len(starts))
    return np.asarray(ptr, dtype=np.int32), np.asarray(starts, dtype=np.float64)


# ------------------------------------------------------------- generators --
def make_closed_set(seed: int, n_curves: int = 4, panels_per_curve: int = 16,
                    g: int = 16, s_per_panel: int | None = None,
                    min_gap: float = 0.01, name: str | None = None) -> Drawing:
    """Closed single-cubic loops (C3 = C0) with C0, C1, C2 uniform in [0,1]^2,
    mutually separated by ``min_gap`` (nesting allowed), simple, without
    cusps; ``panels_per_curve`` equal-arc-length panels each."""
    rng = np.random.default_rng(seed)
    placer = _Placer(min_gap)
    ctrl = []
    tries = 0
    while len(ctrl) < n_curves:
        tries += 1
        if tries > 20000:
            raise RuntimeError("closed-set rejection sampling did not converge")
        c = rng.uniform(0.0, 1.0, size=(3, 2))
        c = np.vstack([c, c[:1]])
        poly = _polyline(c)
        if not _acceptable_shape(c, True, poly) or not placer.fits(poly):
            continue
        placer.add(poly)
        ctrl.append(c)
    ctrl = np.asarray(ctrl)
    ptr, start = _uniform_panels(n_curves, panels_per_curve)
    return Drawing(name or f"closed{n_curves}_s{seed}", ctrl,
                   np.ones(n_curves, bool), _colours(rng, n_curves), ptr, start,
                   g=g, s_per_panel=s_per_panel or 5 * g,
                   meta={"seed": seed, "tries": tries})


def _near_partner(rng, host: np.ndarray, gap: float, size: float):
    """An open cubic that starts at distance ``gap`` from the host curve (on
    the host's normal at a random interior parameter) and leaves it along
    that normal, bending at most 30 degrees: a near-touching pair."""
    t = rng.uniform(0.2, 0.8)
    u = 1.0 - t
    p = (u ** 3) * host[0] + 3 * t * u * u * host[1] + 3 * t * t * u * host[2] + (t ** 3) * host[3]
    d = 3 * (u * u * (host[1] - host[0]) + 2 * t * u * (host[2] - host[1]) + t * t * (host[3] - host[2]))
    d /= np.linalg.norm(d)
    n = np.array([d[1], -d[0]]) * (1.0 if rng.uniform() < 0.5 else -1.0)
    ang = np.deg2rad(rng.uniform(-30.0, 30.0))
    dirv = np.array([np.cos(ang) * n[0] - np.sin(ang) * n[1], np.sin(ang) * n[0] + np.cos(ang) * n[1]])
    p0 = p + gap * n
    L = size * rng.uniform(1.0, 2.0)
    side = np.array([-dirv[1], dirv[0]]) * L * rng.uniform(-0.3, 0.3)
    return np.array([p0, p0 + dirv * L / 3 + side, p0 + 2 * dirv * L / 3 - side, p0 + dirv * L])


def make_mixed_set(seed: int, n_curves: int = 200, open_frac: float = 0.6,
                   g: int = 16, s_per_panel: int | None = None,
                   size_range=(0.006, 0.025), min_gap: float = 5e-3,
                   ratio: float = 0.2, max_level: int = 8, min_panels: int = 2,
                   max_len: float = 0.5, panels: str = "adaptive",
                   panels_per_curve: int = 4, name: str | None = None,
                   near_frac: float = 0.0, near_gap: float = 1e-4,
                   check_samples: int = 0) -> Drawing:
    """Open and closed cubics scattered over the unit canvas.  Each curve's
    control points are centre + size * U[-1,1]^2 with the centre uniform in
    [0.06, 0.94]^2 and size log-uniform in ``size_range``; curves keep
    ``min_gap`` from each other.  With ``near_frac`` > 0, that fraction of
    the curves are open partners planted ``near_gap`` from an earlier curve
    (near-touching pairs; only the pair itself is closer than ``min_gap``).
    Panels are bisected until their length is at most ``ratio`` x the
    distance to the nearest other curve.  ``check_samples`` > 0 runs the
    self-crossing test on a polyline of that many points (for large sets)."""
    rng = np.random.default_rng(seed)
    n_near = int(round(near_frac * n_curves))
    n_base = n_curves - n_near
    n_open = int(round(open_frac * n_base))
    kinds = np.array([False] * n_open + [True] * (n_base - n_open))
    rng.shuffle(kinds)
    placer = _Placer(min_gap, cell=max(0.05, 4 * size_range[1]) if n_curves <= 1000 else 4 * size_range[1])
    ctrl, polys = [], []
    lo_s, hi_s = np.log(size_range[0]), np.log(size_range[1])
    for closed in kinds:
        tries = 0
        while True:
            tries += 1
            if tries > 5000:
                raise RuntimeError("mixed-set rejection sampling did not converge")
            centre = rng.uniform(0.06, 0.94, size=2)
            size = np.exp(rng.uniform(lo_s, hi_s))
            if closed:
                c = centre + size * rng.uniform(-1.5, 1.5, size=(3, 2))
                c = np.vstack([c, c[:1]])
            else:
                c = centre + size * rng.uniform(-1.0, 1.0, size=(4, 2))
            c = np.clip(c, 0.005, 0.995)
            poly = _polyline(c)
            if not _acceptable_shape(c, bool(closed), poly, check_samples) or not placer.fits(poly):
                continue
            placer.add(poly)
            ctrl.append(c)
            polys.append(poly)
            break
    closed_flags = list(kinds)
    for _ in range(n_near):
        tries = 0
        while True:
            tries += 1
            if tries > 20000:
                raise RuntimeError("near-pair rejection sampling did not converge")
            host = int(rng.integers(0, n_base))
            c = _near_partner(rng, ctrl[host], near_gap, np.exp(rng.uniform(lo_s, hi_s)))
            if np.any(c < 0.002) or np.any(c > 0.998):
                continue
            poly = _polyline(c)
            if not _acceptable_shape(c, False, poly, check_samples) or not placer.fits(poly, ignore=host):
                continue
            if _closer_than(poly, polys[host], 0.5 * near_gap):
                continue
            placer.add(poly)
            ctrl.append(c)
            polys.append(poly)
            closed_flags.append(False)
            break
    kinds = np.asarray(closed_flags, bool)
    ctrl = np.asarray(ctrl)
    if panels == "adaptive":
        ptr, start = _adaptive_panels(polys, ratio, max_level, min_panels, max_len)
    else:
        ptr, start = _uniform_panels(n_curves, panels_per_curve)
    return Drawing(name or f"mixed{n_curves}_s{seed}", ctrl, kinds.copy(),
                   _colours(rng, n_curves), ptr, start, g=g,
                   s_per_panel=s_per_panel or 5 * g, meta={"seed": seed})


# Named workloads.  "closed4" is the plain FP64 case: 4 closed cubics,
# 16 panels x 16 nodes = 1024 unknowns per channel, rendered at 128^2.
# "mixed200" is the plain-vs-precision case: 200 open+closed cubics with
# adaptive panels (27,888 unknowns per channel at the default seed), rendered
# at 2048^2.  "mixed16" is a small mixed case (1208 unknowns, g = 8).
# "batched2000" is the batched-render case (2000 curves, 285,328 unknowns
# per channel) and "near20k" the large case (20,000 curves of which 2,000
# start 1e-4 from another; 1,409,808 unknowns per channel).
def drawing_by_name(name: str, seed: int | None = None) -> Drawing:
    if name == "closed4":
        return make_closed_set(20231125 if seed is None else seed, name="closed4")
    if name == "mixed200":
        return make_mixed_set(20231126 if seed is None else seed, name="mixed200")
    if name == "mixed16":       # small mixed case the oracle solves in seconds
        return make_mixed_set(7 if seed is None else seed, n_curves=16,
                              size_range=(0.03, 0.1), min_gap=0.02, g=8,
                              max_level=4, name="mixed16")
    if name == "batched2000":   # 2000 curves, about 285k unknowns per channel
        r = np.sqrt(10.0)
        return make_mixed_set(20231127 if seed is None else seed, n_curves=2000,
                              size_range=(0.006 / r, 0.025 / r), min_gap=5e-3 / r,
                              check_samples=64, name="batched2000")
    if name == "near20k":       # 20k curves, 10% planted 1e-4 from another
        return make_mixed_set(20231128 if seed is None else seed, n_curves=20000,
                              size_range=(0.0008, 0.0032), min_gap=6e-4, ratio=1.0,
                              near_frac=0.1, near_gap=1e-4, check_samples=64, name="near20k")
    raise KeyError(name)


# Cubic Bezier quarter arcs: control arm 4/3 tan(pi/8) of the radius (the
# standard tangent-matching construction; radial error below 3e-4 r).
_ARC_ARM = 4.0 / 3.0 * np.tan(np.pi / 8.0)


def circle_loops(loops, panels_per_arc: int = 4, g: int = 8, s_per_panel: int | None = None,
                 seed: int = 0, name: str = "loops") -> Drawing:
    """Closed loops of four cubic quarter arcs each, for regions bounded by
    curves: ``loops`` lists (cx, cy, r, ccw); ccw = True traverses the loop
    counter-clockwise (an outer boundary), False clockwise (a hole).  Panels
    are equal arc-length quarters of each arc; colours are seeded uniform."""
    ctrl = []
    for cx, cy, r, ccw in loops:
        c = np.array([cx, cy], float)
        arcs = []
        for k in range(4):
            a0, a1 = 0.5 * np.pi * k, 0.5 * np.pi * (k + 1)
            p0 = c + r * np.array([np.cos(a0), np.sin(a0)])
            p3 = c + r * np.array([np.cos(a1), np.sin(a1)])
            p1 = p0 + _ARC_ARM * r * np.array([-np.sin(a0), np.cos(a0)])
            p2 = p3 - _ARC_ARM * r * np.array([-np.sin(a1), np.cos(a1)])
            arcs.append(np.array([p0, p1, p2, p3]))
        if not ccw:
            arcs = [a[::-1] for a in arcs[::-1]]
        ctrl.extend(arcs)
    ctrl = np.asarray(ctrl)
    n = ctrl.shape[0]
    ptr, start = _uniform_panels(n, panels_per_arc)
    rng = np.random.default_rng(seed)
    return Drawing(name, ctrl, np.zeros(n, bool), _colours(rng, n), ptr, start,
                   g=g, s_per_panel=s_per_panel or 5 * g, meta={"loops": list(loops)})


def curve_tangent(drawing: Drawing, i, t) -> np.ndarray:
    """dB/dt of curve(s) i at Bezier parameter(s) t (input generation only)."""
    c = drawing.ctrl[np.asarray(i)]
    t = np.asarray(t, float)[..., None]
    u = 1.0 - t
    return 3 * u * u * (c[..., 1, :] - c[..., 0, :]) + 6 * u * t * (c[..., 2, :] - c[..., 1, :]) \
        + 3 * t * t * (c[..., 3, :] - c[..., 2, :])


def curve_point(drawing: Drawing, i: int, t: float) -> np.ndarray:
    """Point of curve i at Bezier parameter t (input generation only)."""
    c = drawing.ctrl[i]
    u = 1.0 - t
    return (u ** 3) * c[0] + 3 * t * u * u * c[1] + 3 * t * t * u * c[2] + (t ** 3) * c[3]


def viewport_set(drawing: Drawing, seed: int, n: int = 64, side=(256, 4096), zoom=(1.0, 1e6)):
    """n square viewports (x0, y0, x1, y1, w, h): side log-uniform in
    ``side`` pixels, zoom log-uniform in ``zoom`` (world width 1 / zoom of
    the unit canvas), each centred on a uniformly drawn point of a uniformly
    drawn curve."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        w = int(round(np.exp(rng.uniform(np.log(side[0]), np.log(side[1])))))
        z = float(np.exp(rng.uniform(np.log(zoom[0]), np.log(zoom[1]))))
        c = curve_point(drawing, int(rng.integers(0, drawing.n_curves)), float(rng.uniform()))
        h = 0.5 / z
        out.append((float(c[0] - h), float(c[1] - h), float(c[0] + h), float(c[1] + h), w, w))
    return out


def random_node_values(n: int, seed: int, channels: int = 3,
                       scale: float = 1.0) -> np.ndarray:
    """Seeded smooth-free test values (e.g. densities) at n nodes."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal((n, channels))


def pixel_sample(width: int, height: int, count: int, seed: int) -> np.ndarray:
    """Seeded distinct pixel indices (row-major, row 0 at the viewport's
    bottom edge) for sampled parity checks at full image size."""
    rng = np.random.default_rng(seed)
    count = min(count, width * height)
    return np.sort(rng.choice(width * height, size=count, replace=False)).astype(np.int64)
