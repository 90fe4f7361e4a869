"""Parity criteria shared by the GPU tests (CUDA result vs CPU oracle).

Reconstruction: bit-exact (the result is unique).
Distance transform (the method is approximate at rare pixels, Section 2.2,
Figure 3, and where several fixpoints exist the processing order picks one):
  1. the CUDA result satisfies the propagation-rule certificate (nearest is a
     feature, sqdist matches it, features at 0, no 8-neighbour offers a
     strictly closer feature);
  2. sqdist >= exact EDT everywhere;
  3. every pixel where CUDA and oracle differ is a departure pixel (one of
     them differs from the exact EDT there);
  4. the CUDA departure count stays within a small factor of the oracle's.
"""
import numpy as np

import oracle


def edt_parity(binary, sq, nn, feature_nonzero=False, factor=4.0, slack=16, sq_o=None, exact=None):
    binary = np.asarray(binary)
    sq = np.asarray(sq)
    nn = np.asarray(nn)
    if sq_o is None:
        sq_o, _ = oracle.edt(binary, feature_nonzero)
    if exact is None:
        exact = oracle.edt_exact(binary, feature_nonzero)
    cert = oracle.edt_certificate(binary, sq, nn, feature_nonzero)
    assert all(v == 0 for v in cert.values()), cert
    assert (sq >= exact).all(), "distance below the exact EDT"
    diff = sq != sq_o
    dep_gpu = sq != exact
    dep_orc = sq_o != exact
    assert not (diff & ~dep_gpu & ~dep_orc).any(), "CUDA and oracle differ at a non-departure pixel"
    n_gpu, n_orc = int(dep_gpu.sum()), int(dep_orc.sum())
    assert n_gpu <= factor * n_orc + slack, (n_gpu, n_orc)
    return {"departures_gpu": n_gpu, "departures_oracle": n_orc, "differ": int(diff.sum())}
