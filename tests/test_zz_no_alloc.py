"""The allocation-free reconstruction entry point (iwpp_recon_u8_noalloc).

It serves callers that cannot allocate device memory (code inside another
allocator's accounting, real-time paths, code being recorded into a CUDA
graph): its scratch is a static array inside the library.  This test calls
it through the C ABI twice in a row on different inputs -- the second call
must not see anything left over in the shared scratch from the first -- and
compares each result with the regular context-based entry point
(reconstruction is exact, so the comparison is bit-exact).  The file sorts
last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest
import torch

from paper_1209_3314_gb300 import Context, IWPPError, synth
from paper_1209_3314_gb300.binding import recon_u8_noalloc

pytestmark = pytest.mark.gpu


def test_noalloc_matches_context_entry_point_on_two_calls():
    assert torch.cuda.is_available()
    from paper_1209_3314_gb300 import build

    build.build()
    dev = torch.device("cuda:0")
    ctx = Context(0)
    try:
        for seed, (h, w) in ((77, (1000, 1200)), (78, (700, 1333))):
            marker, mask = synth.recon_inputs(h, w, 8.0, 60, seed=seed)
            m = torch.from_numpy(marker).to(dev)
            k = torch.from_numpy(mask).to(dev)
            ref = ctx.recon(m, k, conn=8)
            out = torch.full_like(k, 255)  # caller-owned output
            recon_u8_noalloc(m, k, conn=8, out=out)
            torch.cuda.synchronize()
            assert torch.equal(out, ref)
    finally:
        ctx.close()


def test_noalloc_rejects_images_beyond_its_scratch():
    dev = torch.device("cuda:0")
    w = 64 * 65537  # one row of 65537 tiles: more tiles than the scratch holds
    a = torch.zeros((1, w), dtype=torch.uint8, device=dev)
    b = torch.zeros_like(a)
    with pytest.raises(IWPPError) as e:
        recon_u8_noalloc(a, b, conn=8, out=torch.zeros_like(a))
    assert e.value.code == -1
