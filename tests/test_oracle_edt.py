"""Pins of the distance-transform oracles: the exact EDT (Meijster et al.)
against the Section 2.2 definition (brute force) and scipy's exact EDT, and
the wavefront EDT (Algorithm 3) against its propagation rule, the exact
distance where the rule is exact, closed-form special cases, and the
departure phenomenon of Figure 3."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1209_3314_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
IMAX = np.iinfo(np.int32).max


@pytest.mark.parametrize("fnz", [False, True])
def test_exact_equals_bruteforce_tiny(fnz):
    rng = np.random.default_rng(11 + fnz)
    for _ in range(200):
        h, w = rng.integers(1, 25, 2)
        b = (rng.random((h, w)) < rng.random()).astype(np.uint8)
        np.testing.assert_array_equal(oracle.edt_exact(b, fnz), oracle.edt_bruteforce(b, fnz))


def test_exact_equals_scipy():
    from scipy import ndimage

    img, _ = synth.disks_binary(700, 513, 4, 40, 0.3, seed=5)
    ex = oracle.edt_exact(img, False)
    # scipy: distance of each non-zero pixel to the nearest zero pixel
    ref = np.rint(ndimage.distance_transform_edt(img) ** 2).astype(np.int64)
    np.testing.assert_array_equal(ex.astype(np.int64), ref)


@pytest.mark.parametrize("fnz", [False, True])
def test_alg3_certificate_and_bounds(fnz):
    img, _ = synth.disks_binary(512, 384, 4, 40, 0.3, seed=17)
    sq, nn = oracle.edt(img, fnz)
    cert = oracle.edt_certificate(img, sq, nn, fnz)
    assert all(v == 0 for v in cert.values()), cert
    ex = oracle.edt_exact(img, fnz)
    assert (sq >= ex).all()
    dep = int((sq != ex).sum())
    assert dep < 0.005 * sq.size  # approximation errors are rare (Section 2.2)


def test_alg3_exact_on_tiny_random_mostly():
    rng = np.random.default_rng(23)
    total = dep = 0
    for _ in range(300):
        h, w = rng.integers(1, 25, 2)
        b = (rng.random((h, w)) < rng.random()).astype(np.uint8)
        sq, nn = oracle.edt(b)
        bf = oracle.edt_bruteforce(b)
        assert (sq >= bf).all()
        cert = oracle.edt_certificate(b, sq, nn)
        assert all(v == 0 for v in cert.values()), cert
        total += sq.size
        dep += int((sq != bf).sum())
    assert dep < 0.01 * total


def test_alg3_special_cases():
    # a single feature pixel: exact everywhere
    b = np.ones((31, 45), np.uint8)
    b[12, 30] = 0
    sq, nn = oracle.edt(b)
    yy, xx = np.mgrid[0:31, 0:45]
    np.testing.assert_array_equal(sq, (yy - 12) ** 2 + (xx - 30) ** 2)
    assert (nn == 12 * 45 + 30).all()
    # a full column of features at x0: (x - x0)^2
    b = np.ones((20, 27), np.uint8)
    b[:, 9] = 0
    sq, _ = oracle.edt(b)
    np.testing.assert_array_equal(sq, np.broadcast_to((np.arange(27) - 9) ** 2, (20, 27)))
    # all pixels but one are features: the lone one is at distance 1
    b = np.zeros((9, 14), np.uint8)
    b[4, 13] = 1
    sq, nn = oracle.edt(b)
    assert sq[4, 13] == 1 and sq.sum() == 1
    # no feature at all: nearest -1, distance INT32_MAX
    sq, nn = oracle.edt(np.ones((5, 6), np.uint8))
    assert (nn == -1).all() and (sq == IMAX).all()
    # polarity flag selects the other class
    sq, _ = oracle.edt(np.zeros((4, 4), np.uint8), feature_nonzero=True)
    assert (sq == IMAX).all()


def test_figure3_departure_fixture():
    """Figure 3: neighbourhood propagation can assign sqrt(170) where the
    exact distance is sqrt(169) = 13.  The fixture (written by
    tests/golden/make_golden.py, which calls only the oracle) is a small
    image where Algorithm 3 departs in exactly that way; brute force
    confirms 169 there."""
    with open(os.path.join(GOLDEN, "edt_departure_170.json")) as f:
        g = json.load(f)
    b = np.array(g["binary"], np.uint8)
    y, x = g["pixel"]
    sq, nn = oracle.edt(b)
    assert oracle.edt_bruteforce(b)[y, x] == 169
    assert sq[y, x] == 170
    cert = oracle.edt_certificate(b, sq, nn)
    assert all(v == 0 for v in cert.values())


def test_order_dependence_probe():
    """Where propagation is exact, pop order cannot change the distance; at
    departure pixels it may.  Every difference between pop orders must sit
    on a pixel that departs from the exact EDT in one of the runs."""
    img, _ = synth.disks_binary(256, 256, 4, 40, 0.3, seed=31)
    ex = oracle.edt_exact(img)
    runs = [oracle.edt(img, policy=p, seed=s)[0] for p, s in ((0, 0), (1, 0), (2, 1), (2, 2))]
    for r in runs[1:]:
        diff = r != runs[0]
        assert (~diff | (r != ex) | (runs[0] != ex)).all()


def test_departures_counted_on_config_workload():
    wl = synth.config_workload("edt4096", size=1024)
    st = {}
    sq, _ = oracle.edt(wl.binary, stats=st)
    ex = oracle.edt_exact(wl.binary)
    dep = int((sq != ex).sum())
    assert 0 < dep < 0.002 * sq.size
    assert st["pushes"] >= st["initial"] > 0
