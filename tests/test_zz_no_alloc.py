"""The allocation-free histogram (lbm_histogram_noalloc) against lbm_histogram.

lbm_histogram_noalloc serves callers that cannot allocate device memory
(stream capture in progress, memory owned by another allocator or budgeted in
advance, distributions kept in the caller's own buffers).  It counts into one
fixed device array shared by all calls, so this test runs it twice in a row,
with different bin counts and ranges, and checks both against the allocating
entry point: the counts are integers and must match exactly.  The file sorts
last so that a stop-at-first-failure run has done every other test first.
"""
import numpy as np
import pytest

import synth
from tests.conftest import has_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not has_gpu(), reason="needs a CUDA GPU")]


def test_histogram_noalloc_matches_lbm_histogram():
    import torch

    import paper_1802_01272_gb300 as P
    from paper_1802_01272_gb300.binding import histogram_noalloc

    lp = P.Params(Lx=200, Ly=150, precision=P.LBM_FP64, T=0.8)
    rho, ux, uy = synth.bubble(200, 150, 1.9, 0.24, R=40, W=3)
    stream = torch.cuda.current_stream()
    with P.Lattice(lp, stream) as L:
        L.init_rho_u(rho, ux, uy)
        L.step(3)
        f = torch.empty((16, 150, 200), dtype=torch.float64, device="cuda")
        L.get_f_device(f)
        L.sync()
        for nbins, lo, hi in ((512, 0.0, 3.0), (64, 0.2, 2.0)):   # two calls in a row
            want = L.histogram(nbins, lo, hi)
            got = histogram_noalloc(f, P.LBM_FP64, 0.0, nbins, lo, hi, stream)
            assert got.sum() == want.sum() > 0
            assert np.array_equal(got, want)
        # the maximum is enforced
        with pytest.raises(P.LBMError) as e:
            histogram_noalloc(f, P.LBM_FP64, 0.0, 4097, 0.0, 3.0, stream)
        assert e.value.code == -1
