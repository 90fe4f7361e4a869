"""CPU oracle for the IWPP reconstruction and distance transform.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA library (``paper_1209_3314_gb300``) and imports
nothing from it; both sides only consume the same seeded inputs.

What it provides (paper = Teodoro et al., arXiv:1209.3314):

* ``fh(marker, mask, conn)`` -- fast hybrid reconstruction, Algorithm 2
  (Section 2.1), sequential C (``iwpp_oracle.c``).
* ``edt(binary, feature_nonzero)`` -- wavefront distance transform,
  Algorithm 3 (Section 2.2), sequential C, FIFO order as published;
  ``edt(..., policy=1|2)`` re-runs it with LIFO / random pop order.
* ``edt_exact`` -- exact squared EDT (Meijster et al. 2000), sequential C.
* ``recon_bruteforce`` -- the definition of reconstruction (Section 2.1):
  elementary geodesic dilations, each clipped by the mask, to stability.
* ``recon_threshold_decomposition`` -- the textbook binary decomposition:
  for each level t, {out >= t} is the union of the connected components of
  {mask >= t} that meet {marker and mask >= t}.  Independent of Algorithm 2.
* ``edt_bruteforce`` -- the definition of the distance map (Section 2.2):
  minimum squared distance to any feature pixel.
* ``gdt`` / ``gdt_bellman_ford`` -- shortest paths on a grid with obstacles
  (Section 1): Dijkstra's algorithm, and plain relaxation to a fixpoint.
* ``skiz`` / ``skiz_per_label`` -- influence zones and their skeleton of
  labelled sources inside a mask (Section 1), with the shortest-path metric
  above: sequential C, and a restatement from one distance map per label.
* ``watershed`` -- marker-controlled watershed by flooding (Section 1), the
  image foresting transform with the highest-value path cost, sequential C;
  ``watershed_levels_threshold`` / ``watershed_pdist_relax`` /
  ``watershed_labels_reach`` restate its three parts independently
  (threshold decomposition, relaxation to a fixpoint, per-label
  reachability) for small images.
* certificate checks of a result against the propagation rules.

Every function takes and returns numpy arrays; the C part is built by
``oracle/build.py`` (``gcc -O2 -shared``) on first use.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build_oracle

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def _load():
    global _lib
    if _lib is None:
        path = build_oracle()
        lib = ctypes.CDLL(path)
        i32, i64p = ctypes.c_int, ctypes.POINTER(ctypes.c_int64)
        vp = ctypes.c_void_p
        lib.oracle_fh_i32.argtypes = [i32, i32, vp, vp, i32, i64p]
        lib.oracle_fh_u8.argtypes = [i32, i32, vp, vp, i32, i64p]
        lib.oracle_edt.argtypes = [i32, i32, vp, i32, vp, vp, i64p]
        lib.oracle_edt_policy.argtypes = [i32, i32, vp, i32, vp, vp, i64p, i32,
                                          ctypes.c_uint64]
        lib.oracle_edt_exact.argtypes = [i32, i32, vp, i32, vp]
        lib.oracle_gdt.argtypes = [i32, i32, vp, vp, vp, i64p]
        lib.oracle_watershed.argtypes = [i32, i32, vp, vp, vp, vp, vp, i64p]
        lib.oracle_skiz.argtypes = [i32, i32, vp, vp, vp, vp, vp]
        for f in ("oracle_fh_i32", "oracle_fh_u8", "oracle_edt",
                  "oracle_edt_policy", "oracle_edt_exact"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def fh(marker: np.ndarray, mask: np.ndarray, conn: int = 8, stats: dict | None = None):
    """Reconstruction of ``mask`` from ``marker`` by Algorithm 2 (FH).

    uint8 or int32 2-D arrays of identical shape; returns a new array.
    ``stats`` (optional dict) receives 'initial' and 'pushes' queue counts.
    """
    assert marker.shape == mask.shape and marker.ndim == 2
    assert marker.dtype == mask.dtype
    lib = _load()
    h, w = mask.shape
    I = np.ascontiguousarray(mask)
    J = np.ascontiguousarray(marker).copy()
    cnt = (ctypes.c_int64 * 2)()
    if I.dtype == np.uint8:
        rc = lib.oracle_fh_u8(h, w, _ptr(I), _ptr(J), conn, cnt)
    elif I.dtype == np.int32:
        rc = lib.oracle_fh_i32(h, w, _ptr(I), _ptr(J), conn, cnt)
    else:
        raise TypeError(f"unsupported dtype {I.dtype}")
    if rc != 0:
        raise RuntimeError("oracle_fh failed")
    if stats is not None:
        stats["initial"], stats["pushes"] = int(cnt[0]), int(cnt[1])
    return J


def edt(binary: np.ndarray, feature_nonzero: bool = False, policy: int = 0,
        seed: int = 0, stats: dict | None = None):
    """Algorithm 3: returns (sqdist int32, nearest int32 linear index).

    Features are pixels equal to 0 (the paper's background) unless
    ``feature_nonzero``.  No feature: sqdist INT32_MAX, nearest -1.
    """
    lib = _load()
    b = np.ascontiguousarray(binary, dtype=np.uint8)
    h, w = b.shape
    nearest = np.empty((h, w), np.int32)
    sq = np.empty((h, w), np.int32)
    cnt = (ctypes.c_int64 * 2)()
    rc = lib.oracle_edt_policy(h, w, _ptr(b), int(bool(feature_nonzero)),
                               _ptr(nearest), _ptr(sq), cnt, int(policy), int(seed))
    if rc != 0:
        raise RuntimeError("oracle_edt failed")
    if stats is not None:
        stats["initial"], stats["pushes"] = int(cnt[0]), int(cnt[1])
    return sq, nearest


def edt_exact(binary: np.ndarray, feature_nonzero: bool = False) -> np.ndarray:
    """Exact squared EDT (Meijster et al. 2000); INT32_MAX where no feature."""
    lib = _load()
    b = np.ascontiguousarray(binary, dtype=np.uint8)
    h, w = b.shape
    out = np.empty((h, w), np.int32)
    if lib.oracle_edt_exact(h, w, _ptr(b), int(bool(feature_nonzero)), _ptr(out)) != 0:
        raise RuntimeError("oracle_edt_exact failed")
    return out


# ---------------------------------------------------------------- definitions

def gdt(mask: np.ndarray, seeds: np.ndarray, stats: dict | None = None) -> np.ndarray:
    """Geodesic (shortest-path) distance through free pixels (mask != 0)
    from sources (free pixels with seeds != 0); 8 moves, cost 5 straight and
    7 diagonal; INT32_MAX for obstacles and unreachable pixels (Section 1's
    shortest paths on a grid with obstacles; Dijkstra's algorithm)."""
    lib = _load()
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    s = np.ascontiguousarray(seeds, dtype=np.uint8)
    assert m.shape == s.shape and m.ndim == 2
    h, w = m.shape
    out = np.empty((h, w), np.int32)
    st = np.zeros(2, np.int64)
    rc = lib.oracle_gdt(h, w, _ptr(m), _ptr(s), _ptr(out), st.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if rc != 0:
        raise MemoryError("oracle_gdt")
    if stats is not None:
        stats.update(pops=int(st[0]), improvements=int(st[1]))
    return out


def gdt_bellman_ford(mask: np.ndarray, seeds: np.ndarray) -> np.ndarray:
    """The same distances by plain relaxation to a fixpoint (every free pixel
    takes the least neighbour distance plus the step cost, repeated until
    nothing changes): a brute-force check of gdt on small grids."""
    m = np.asarray(mask) != 0
    INF = np.iinfo(np.int64).max // 4
    d = np.where(m & (np.asarray(seeds) != 0), 0, INF).astype(np.int64)
    h, w = d.shape
    while True:
        best = d.copy()
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dy == 0 and dx == 0:
                    continue
                cost = 7 if dy and dx else 5
                sh = np.full_like(d, INF)
                sh[max(dy, 0):h + min(dy, 0), max(dx, 0):w + min(dx, 0)] = \
                    d[max(-dy, 0):h + min(-dy, 0), max(-dx, 0):w + min(-dx, 0)]
                best = np.minimum(best, np.where(sh < INF, sh + cost, INF))
        best = np.where(m, best, INF)
        if np.array_equal(best, d):
            break
        d = best
    return np.where(d >= INF, np.iinfo(np.int32).max, d).astype(np.int32)


def watershed(relief: np.ndarray, markers: np.ndarray, stats: dict | None = None,
              with_pdist: bool = False):
    """Marker-controlled watershed by flooding (Section 1 names it as an
    IWPP algorithm; the definition is in ``oracle_watershed`` in the C file):
    returns (label int32, level in the relief's dtype[, plateau distance]).
    Without markers the level is the dtype's maximum and the label 0."""
    lib = _load()
    f = np.asarray(relief)
    assert f.dtype in (np.uint8, np.int32) and f.ndim == 2
    m = np.ascontiguousarray(markers, dtype=np.int32)
    assert m.shape == f.shape
    h, w = f.shape
    f32 = np.ascontiguousarray(f, dtype=np.int32)
    label = np.empty((h, w), np.int32)
    level = np.empty((h, w), np.int32)
    pdist = np.empty((h, w), np.int32)
    st = np.zeros(4, np.int64)
    rc = lib.oracle_watershed(h, w, _ptr(f32), _ptr(m), _ptr(label), _ptr(level), _ptr(pdist),
                              st.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if rc != 0:
        raise MemoryError("oracle_watershed")
    if stats is not None:
        stats.update(pops=int(st[0]), improvements=int(st[1]), plateau_pushes=int(st[2]),
                     label_pushes=int(st[3]))
    if f.dtype == np.uint8:
        level = np.minimum(level, 255).astype(np.uint8)
    return (label, level, pdist) if with_pdist else (label, level)


def skiz(mask: np.ndarray, labels: np.ndarray):
    """Influence zones of labelled sources (free pixels with labels != 0)
    inside a mask (mask != 0 is free), with the shortest-path metric of
    ``gdt``: returns (zones int32: the least label whose sources are
    nearest, 0 at obstacles and unreachable pixels; skiz uint8: 1 where two
    or more labels are nearest; dist int32 as ``gdt``)."""
    lib = _load()
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    assert m.shape == lab.shape and m.ndim == 2
    h, w = m.shape
    zones = np.empty((h, w), np.int32)
    sk = np.empty((h, w), np.uint8)
    dist = np.empty((h, w), np.int32)
    if lib.oracle_skiz(h, w, _ptr(m), _ptr(lab), _ptr(zones), _ptr(sk), _ptr(dist)) != 0:
        raise MemoryError("oracle_skiz")
    return zones, sk, dist


def skiz_per_label(mask: np.ndarray, labels: np.ndarray):
    """The same zones and skeleton from their definition: one distance map
    per label (relaxation to a fixpoint, ``gdt_bellman_ford``); a label
    reaches p when its map equals the least map at p.  Small images."""
    m = np.asarray(mask) != 0
    lab = np.asarray(labels).astype(np.int64)
    IMAX = np.iinfo(np.int32).max
    vals = np.unique(lab[m & (lab != 0)])
    maps = [oracle_gdt_map(m, lab == L) for L in vals]
    h, w = m.shape
    if not maps:
        return (np.zeros((h, w), np.int32), np.zeros((h, w), np.uint8),
                np.full((h, w), IMAX, np.int32))
    stack = np.stack(maps).astype(np.int64)
    best = stack.min(axis=0)
    reach = (stack == best) & (best < IMAX)
    count = reach.sum(axis=0)
    first = np.where(reach.any(axis=0), vals[np.argmax(reach, axis=0)], 0)
    return first.astype(np.int32), (count >= 2).astype(np.uint8), best.astype(np.int32)


def oracle_gdt_map(free: np.ndarray, sources: np.ndarray) -> np.ndarray:
    """One label's distance map by relaxation (``gdt_bellman_ford``)."""
    return gdt_bellman_ford(free.astype(np.uint8), sources.astype(np.uint8))


def _shifted(a: np.ndarray, dy: int, dx: int, fill) -> np.ndarray:
    """out[y, x] = a[y + dy, x + dx], fill outside the image."""
    h, w = a.shape
    out = np.full_like(a, fill)
    out[max(-dy, 0):h + min(-dy, 0), max(-dx, 0):w + min(-dx, 0)] = \
        a[max(dy, 0):h + min(dy, 0), max(dx, 0):w + min(dx, 0)]
    return out


_OFF8 = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if dy or dx]


def watershed_levels_threshold(relief: np.ndarray, markers: np.ndarray) -> np.ndarray:
    """Flooding levels by threshold decomposition: level(p) is the least t
    such that p lies in an 8-connected component of {relief <= t} that holds
    a marker pixel (a path whose highest value is <= t exists exactly then).
    int64; INT32_MAX where no marker exists."""
    from scipy import ndimage

    f = np.asarray(relief).astype(np.int64)
    mk = np.asarray(markers) != 0
    out = np.full(f.shape, np.iinfo(np.int32).max, np.int64)
    if not mk.any():
        return out
    unset = np.ones(f.shape, bool)
    for t in np.unique(f):
        lab, n = ndimage.label(f <= t, structure=np.ones((3, 3), bool))
        hit = np.zeros(n + 1, bool)
        hit[lab[mk & (f <= t)]] = True
        hit[0] = False
        reached = hit[lab] & unset
        out[reached] = t
        unset &= ~reached
    return out


def watershed_pdist_relax(level: np.ndarray, markers: np.ndarray) -> np.ndarray:
    """Plateau distances by relaxation to a fixpoint: 0 at marker pixels and
    at pixels with a lower neighbour, else 1 + the least value over the
    neighbours of equal level, repeated until nothing changes."""
    lv = np.asarray(level).astype(np.int64)
    TOP = np.iinfo(np.int64).max
    INF = np.iinfo(np.int32).max
    entry = np.asarray(markers) != 0
    for dy, dx in _OFF8:
        entry |= _shifted(lv, dy, dx, TOP) < lv
    d = np.where(entry, 0, INF).astype(np.int64)
    while True:
        best = d.copy()
        for dy, dx in _OFF8:
            nd = _shifted(d, dy, dx, INF)
            same = _shifted(lv, dy, dx, TOP) == lv
            best = np.where(same & (nd < INF), np.minimum(best, nd + 1), best)
        if np.array_equal(best, d):
            return d
        d = best


def watershed_labels_reach(level: np.ndarray, pdist: np.ndarray, markers: np.ndarray) -> np.ndarray:
    """Labels by reachability: for every marker value separately, the set of
    pixels reachable from its marker pixels along optimal edges (p -> q, q
    not a marker: level(p) < level(q) with pdist(q) = 0, or equal levels
    with pdist(p) + 1 = pdist(q)) grown to a fixpoint; each pixel takes the
    least value that reaches it, marker pixels keep theirs, 0 if none."""
    lv = np.asarray(level).astype(np.int64)
    pd = np.asarray(pdist).astype(np.int64)
    mk = np.asarray(markers).astype(np.int64)
    TOP = np.iinfo(np.int64).max
    edges = []
    for dy, dx in _OFF8:  # edge from the neighbour at (dy, dx) into p
        nl = _shifted(lv, dy, dx, TOP)
        npd = _shifted(pd, dy, dx, TOP)
        rise = (nl < lv) & (pd == 0)
        flat = (nl == lv) & (npd + 1 == pd)
        edges.append((dy, dx, (rise | flat) & (mk == 0)))
    out = mk.copy()
    best = np.full(mk.shape, TOP, np.int64)
    for L in np.unique(mk[mk != 0]):
        r = mk == L
        while True:
            grow = r.copy()
            for dy, dx, e in edges:
                grow |= e & _shifted(r, dy, dx, False)
            if np.array_equal(grow, r):
                break
            r = grow
        best = np.where(r & (mk == 0), np.minimum(best, L), best)
    out = np.where((mk == 0) & (best < TOP), best, out)
    return out.astype(np.int32)


def _neighbour_max(J: np.ndarray, conn: int) -> np.ndarray:
    """max over N_G(p) u {p}; pixels outside the image do not exist."""
    if J.dtype == np.uint8:
        low = 0
    else:
        low = np.iinfo(J.dtype).min
    h, w = J.shape
    P = np.full((h + 2, w + 2), low, dtype=J.dtype)
    P[1:-1, 1:-1] = J
    m = J.copy()
    if conn == 8:
        offs = [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]
    else:
        offs = [(-1, 0), (0, -1), (0, 1), (1, 0)]
    for dy, dx in offs:
        np.maximum(m, P[1 + dy:1 + dy + h, 1 + dx:1 + dx + w], out=m)
    return m


def recon_bruteforce(marker: np.ndarray, mask: np.ndarray, conn: int = 8,
                     max_iter: int | None = None) -> np.ndarray:
    """Section 2.1 definition: J <- (max over N_G(p) u {p} of J) and I(p),
    starting from marker and mask, repeated until nothing changes."""
    J = np.minimum(marker, mask)
    it = 0
    while True:
        Jn = np.minimum(_neighbour_max(J, conn), mask)
        it += 1
        if np.array_equal(Jn, J):
            return J
        J = Jn
        if max_iter is not None and it >= max_iter:
            raise RuntimeError("brute force did not converge")


def recon_threshold_decomposition(marker: np.ndarray, mask: np.ndarray,
                                  conn: int = 8) -> np.ndarray:
    """uint8 reconstruction by threshold decomposition and component labels.

    out(p) = number of levels t in 1..255 at which p lies in a connected
    component of {mask >= t} that contains a pixel with min(marker, mask) >= t.
    """
    from scipy import ndimage

    assert mask.dtype == np.uint8
    J0 = np.minimum(marker, mask)
    structure = np.ones((3, 3), bool) if conn == 8 else ndimage.generate_binary_structure(2, 1)
    out = np.zeros(mask.shape, np.int32)
    lo = int(J0.min())
    hi = int(J0.max())
    out += lo  # every pixel's own component meets {J0 >= t} for t <= min(J0)
    for t in range(max(lo + 1, 1), hi + 1):
        lab, n = ndimage.label(mask >= t, structure=structure)
        if n == 0:
            break
        hit = np.zeros(n + 1, bool)
        hit[lab[J0 >= t]] = True
        hit[0] = False
        out += hit[lab]
    return out.astype(np.uint8)


def edt_bruteforce(binary: np.ndarray, feature_nonzero: bool = False) -> np.ndarray:
    """Section 2.2 definition: squared distance to the nearest feature pixel."""
    b = np.asarray(binary)
    feat = (b != 0) if feature_nonzero else (b == 0)
    h, w = b.shape
    fy, fx = np.nonzero(feat)
    if fy.size == 0:
        return np.full((h, w), np.iinfo(np.int32).max, np.int32)
    yy, xx = np.mgrid[0:h, 0:w]
    d = (yy.reshape(-1, 1) - fy.reshape(1, -1)) ** 2 + (xx.reshape(-1, 1) - fx.reshape(1, -1)) ** 2
    return d.min(axis=1).reshape(h, w).astype(np.int32)


# ---------------------------------------------------------------- certificates

def recon_unstable_pairs(out: np.ndarray, mask: np.ndarray, conn: int = 8) -> int:
    """Number of (p, q) neighbour pairs where q could still be raised:
    out(q) < min(out(p), mask(q)).  Zero exactly at a fixpoint of the
    propagation rule of Algorithms 2 and 5."""
    o = out.astype(np.int64)
    m = mask.astype(np.int64)
    return int((o < np.minimum(_neighbour_max(out, conn).astype(np.int64), m)).sum())


def edt_certificate(binary: np.ndarray, sqdist: np.ndarray, nearest: np.ndarray,
                    feature_nonzero: bool = False) -> dict:
    """Checks a distance-transform result against the propagation rule.

    Returns counts of violations of: nearest is a feature (or -1 with no
    feature at all); sqdist equals |p - nearest(p)|^2; features have 0;
    local optimality (no 8-neighbour's feature is strictly closer to p).
    """
    b = np.asarray(binary)
    feat = (b != 0) if feature_nonzero else (b == 0)
    h, w = b.shape
    n = np.asarray(nearest).astype(np.int64)
    sq = np.asarray(sqdist).astype(np.int64)
    res = {}
    valid = n >= 0
    if not feat.any():
        res["bad_nearest"] = int((n != -1).sum())
        res["bad_sqdist"] = int((sq != np.iinfo(np.int32).max).sum())
        res["feature_nonzero_dist"] = 0
        res["not_locally_optimal"] = 0
        return res
    ny, nx = np.where(valid, n // w, 0), np.where(valid, n % w, 0)
    in_range = valid & (n < h * w)
    ff = feat.reshape(-1)[np.clip(n, 0, h * w - 1)].reshape(h, w)
    res["bad_nearest"] = int((~in_range | ~ff).sum())
    yy, xx = np.mgrid[0:h, 0:w]
    d = (yy - ny) ** 2 + (xx - nx) ** 2
    res["bad_sqdist"] = int((valid & (d != sq)).sum())
    res["feature_nonzero_dist"] = int((feat & (sq != 0)).sum())
    worse = 0
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dy == 0 and dx == 0:
                continue
            ys = slice(max(dy, 0), h + min(dy, 0))
            xs = slice(max(dx, 0), w + min(dx, 0))
            yd = slice(max(-dy, 0), h + min(-dy, 0))
            xd = slice(max(-dx, 0), w + min(-dx, 0))
            # candidate for pixel at (yd, xd) is the feature of its neighbour at (ys, xs)
            cn = n[ys, xs]
            cy, cx = cn // w, cn % w
            py, px = yy[yd, xd], xx[yd, xd]
            cd = (py - cy) ** 2 + (px - cx) ** 2
            better = (cn >= 0) & ((sq[yd, xd] > cd) | (n[yd, xd] < 0))
            worse += int(better.sum())
    res["not_locally_optimal"] = worse
    return res
