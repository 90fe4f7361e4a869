"""Plants plausible mistakes in a copy of the oracle's C source and checks
that the pins catch each one.  The mutated copy is built in a temporary
directory; the oracle itself is untouched.  Every mutant keeps the
propagation monotone (each update strictly improves a fixed per-pixel
measure), so every mutant still terminates quickly."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle.build import SRC, build_oracle

MUTATIONS = {
    # reconstruction (Algorithm 2)
    "raster_without_mask_clip": ("            J[p] = m < I[p] ? m : I[p];\n        }\n\n    /* Anti-raster",
                                 "            J[p] = m;\n        }\n\n    /* Anti-raster"),
    "seed_test_on_wrong_half": ("            for (int k = half; k < conn; k++) {\n                int yy = y + nb[k][0], xx = x + nb[k][1];\n                if (!inside(yy, xx, h, w)) continue;",
                                "            for (int k = 0; k < half; k++) {\n                int yy = y + nb[k][0], xx = x + nb[k][1];\n                if (!inside(yy, xx, h, w)) continue;"),
    "propagate_without_mask_clip": ("J[qq] = J[p] < I[qq] ? J[p] : I[qq];", "J[qq] = J[p];"),
    "queue_drops_diagonals": ("        for (int k = 0; k < conn; k++) {\n            int yy = y + nb[k][0], xx = x + nb[k][1];\n            if (!inside(yy, xx, h, w)) continue;\n            int64_t qq = (int64_t)yy * w + xx;\n            if (J[qq] < J[p]",
                              "        for (int k = 1; k < conn; k += 2) {\n            int yy = y + nb[k][0], xx = x + nb[k][1];\n            if (!inside(yy, xx, h, w)) continue;\n            int64_t qq = (int64_t)yy * w + xx;\n            if (J[qq] < J[p]"),
    "mirrored_left_neighbour": ("{0, -1},\n                              {1, 1}", "{0, 1},\n                              {1, 1}"),
    # distance transform (Algorithm 3)
    "edt_four_neighbours": ("            int yy = y + NB8[k][0], xx = x + NB8[k][1];\n            if (!inside(yy, xx, h, w)) continue;\n            int64_t qq = (int64_t)yy * w + xx;\n            int64_t dnew",
                            "            if (k % 2 == 0) continue;\n            int yy = y + NB8[k][0], xx = x + NB8[k][1];\n            if (!inside(yy, xx, h, w)) continue;\n            int64_t qq = (int64_t)yy * w + xx;\n            int64_t dnew"),
    "edt_seed_inverted": ("if (inside(yy, xx, h, w) && !IS_FEATURE((int64_t)yy * w + xx))",
                          "if (inside(yy, xx, h, w) && IS_FEATURE((int64_t)yy * w + xx))"),
    "edt_output_skips_self_feature": ("else { nearest[p] = (int32_t)VR[p]; sqdist[p] = (int32_t)sqd(p, VR[p], w); }",
                                      "else { nearest[p] = (int32_t)VR[p]; sqdist[p] = VR[p] == p ? 1 : (int32_t)sqd(p, VR[p], w); }"),
    "edt_distance_typo": ("return dy * dy + dx * dx;", "return dy * dy + dx * dy;"),
    # exact EDT (Meijster)
    "exact_column_scan_off_by_one": ("if (below < g[(int64_t)y * w + x]) g[(int64_t)y * w + x] = 1 + below;",
                                     "if (below < g[(int64_t)y * w + x]) g[(int64_t)y * w + x] = below;"),
    # watershed (Section 1): levels, plateau distances, labels
    "ws_level_ignores_relief": ("const int64_t c = it.key > f[qq] ? it.key : f[qq];",
                                "const int64_t c = it.key;"),
    "ws_entry_from_higher": ("lv[(int64_t)qy * w + qx] < lv[i]) entry = 1;",
                             "lv[(int64_t)qy * w + qx] > lv[i]) entry = 1;"),
    "ws_rise_from_equal_level": ("const int rise = lv[p] < lv[qq] && pdist[qq] == 0;",
                                 "const int rise = lv[p] <= lv[qq] && pdist[qq] == 0;"),
    "ws_flat_sideways": ("(int64_t)pdist[p] + 1 == pdist[qq];", "(int64_t)pdist[p] <= pdist[qq];"),
    "ws_largest_label_first": ("if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;",
                               "if (x[0] != y[0]) return x[0] < y[0] ? 1 : -1;"),
    # influence zones / SKIZ (Section 1)
    "skiz_any_shorter_edge": ("if ((int64_t)dist[p] + cost == dist[qq]) {", "if ((int64_t)dist[p] + cost >= dist[qq]) {"),
    "skiz_swapped_costs": ("const int64_t cost = (NB8[k][0] != 0 && NB8[k][1] != 0) ? 7 : 5;\n                if ((int64_t)dist[p]",
                           "const int64_t cost = (NB8[k][0] != 0 && NB8[k][1] != 0) ? 5 : 7;\n                if ((int64_t)dist[p]"),
    "skiz_max_pass_ascending": ("skiz_sweep(h, w, mask, dist, pairs, np, 1, zmax, done, &q);",
                                "skiz_sweep(h, w, mask, dist, pairs, np, 0, zmax, done, &q);"),
    "exact_separator_sign": ("int64_t num = (int64_t)u * u - i * i + gy[u] * gy[u] - gy[i] * gy[i];",
                             "int64_t num = (int64_t)u * u - i * i - gy[u] * gy[u] + gy[i] * gy[i];"),
}


def _mutant(tmp_path, name):
    src = open(SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not unique/found"
    p = tmp_path / f"{name}.c"
    p.write_text(src.replace(old, new))
    so = build_oracle(force=True, src=str(p), out=str(tmp_path / f"lib{name}.so"))
    lib = ctypes.CDLL(so)
    return lib


def _fh(lib, J, I, conn):
    J = J.copy()
    lib.oracle_fh_u8(ctypes.c_int(J.shape[0]), ctypes.c_int(J.shape[1]), I.ctypes.data_as(ctypes.c_void_p),
                     J.ctypes.data_as(ctypes.c_void_p), ctypes.c_int(conn), None)
    return J


def _edt(lib, b):
    h, w = b.shape
    sq = np.empty((h, w), np.int32)
    nn = np.empty((h, w), np.int32)
    lib.oracle_edt(ctypes.c_int(h), ctypes.c_int(w), b.ctypes.data_as(ctypes.c_void_p), ctypes.c_int(0),
                   nn.ctypes.data_as(ctypes.c_void_p), sq.ctypes.data_as(ctypes.c_void_p), None)
    return sq, nn


def _exact(lib, b):
    h, w = b.shape
    out = np.empty((h, w), np.int32)
    lib.oracle_edt_exact(ctypes.c_int(h), ctypes.c_int(w), b.ctypes.data_as(ctypes.c_void_p), ctypes.c_int(0),
                         out.ctypes.data_as(ctypes.c_void_p))
    return out


def _recon_pins_fail(lib):
    rng = np.random.default_rng(77)
    for it in range(200):
        h, w = rng.integers(2, 14, 2)
        I = rng.integers(0, 256, (h, w)).astype(np.uint8)
        J = rng.integers(0, 256, (h, w)).astype(np.uint8)
        conn = 8 if it % 2 else 4
        if not np.array_equal(_fh(lib, J, I, conn), oracle.recon_bruteforce(J, I, conn)):
            return True
    return False


def _edt_pins_fail(lib):
    rng = np.random.default_rng(78)
    for _ in range(100):
        h, w = rng.integers(2, 25, 2)
        b = (rng.random((h, w)) < rng.random()).astype(np.uint8)
        sq, nn = _edt(lib, b)
        cert = oracle.edt_certificate(b, sq, nn)
        if any(v for v in cert.values()) or (sq < oracle.edt_bruteforce(b)).any():
            return True
    return False


def _exact_pins_fail(lib):
    rng = np.random.default_rng(79)
    for _ in range(100):
        h, w = rng.integers(2, 25, 2)
        b = (rng.random((h, w)) < rng.random()).astype(np.uint8)
        if not np.array_equal(_exact(lib, b), oracle.edt_bruteforce(b)):
            return True
    return False


def _ws_pins_fail(lib):
    rng = np.random.default_rng(80)
    for it in range(150):
        h, w = (int(v) for v in rng.integers(1, 16, 2))
        f = rng.integers(0, (2, 4, 256)[it % 3], (h, w)).astype(np.int32)
        m = np.zeros((h, w), np.int32)
        for _ in range(int(rng.integers(1, 6))):
            m[rng.integers(0, h), rng.integers(0, w)] = rng.integers(1, 6)
        label, level, pdist = (np.empty((h, w), np.int32) for _ in range(3))
        vp = ctypes.c_void_p
        lib.oracle_watershed(ctypes.c_int(h), ctypes.c_int(w), f.ctypes.data_as(vp), m.ctypes.data_as(vp),
                             label.ctypes.data_as(vp), level.ctypes.data_as(vp), pdist.ctypes.data_as(vp), None)
        t = oracle.watershed_levels_threshold(f, m)
        pr = oracle.watershed_pdist_relax(t, m)
        if (not np.array_equal(level, t) or not np.array_equal(pdist, pr)
                or not np.array_equal(label, oracle.watershed_labels_reach(t, pr, m))):
            return True
    return False


def _skiz_pins_fail(lib):
    rng = np.random.default_rng(81)
    for _ in range(120):
        h, w = (int(v) for v in rng.integers(1, 16, 2))
        m = (rng.random((h, w)) >= 0.25).astype(np.uint8)
        lab = np.zeros((h, w), np.int32)
        for _ in range(int(rng.integers(1, 6))):
            lab[rng.integers(0, h), rng.integers(0, w)] = rng.integers(1, 5)
        z, d = np.empty((h, w), np.int32), np.empty((h, w), np.int32)
        s = np.empty((h, w), np.uint8)
        vp = ctypes.c_void_p
        lib.oracle_skiz(ctypes.c_int(h), ctypes.c_int(w), m.ctypes.data_as(vp), lab.ctypes.data_as(vp),
                        z.ctypes.data_as(vp), s.ctypes.data_as(vp), d.ctypes.data_as(vp))
        z2, s2, d2 = oracle.skiz_per_label(m, lab)
        if not (np.array_equal(z, z2) and np.array_equal(s, s2) and np.array_equal(d, d2)):
            return True
    return False


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    lib = _mutant(tmp_path, name)
    if name.startswith("edt_"):
        assert _edt_pins_fail(lib), f"mutation {name} not detected"
    elif name.startswith("skiz_"):
        assert _skiz_pins_fail(lib), f"mutation {name} not detected"
    elif name.startswith("ws_"):
        assert _ws_pins_fail(lib), f"mutation {name} not detected"
    elif name.startswith("exact_"):
        assert _exact_pins_fail(lib), f"mutation {name} not detected"
    else:
        assert _recon_pins_fail(lib), f"mutation {name} not detected"
