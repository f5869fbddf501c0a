"""The allocation-free histogram (lbm_histogram_noalloc) against lbm_histogram.

lbm_histogram_noalloc serves callers that cannot allocate device memory
(memory owned by another allocator or budgeted in advance, loops that cannot
afford an allocation's synchronisation, distributions kept in the caller's own
buffers).  It counts into one fixed device array shared by all calls, so this
test runs it twice in a row, with different bin counts and ranges, and checks
both against the allocating entry point for each storage precision (FP64,
FP32 shifted, FP16 shifted: the caller passes the stored deviations and
rho_ref): the counts are integers and must match exactly.  The file sorts last
so that a stop-at-first-failure run has done every other test first.
"""
import math

import numpy as np
import pytest

import synth
from tests.conftest import has_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not has_gpu(), reason="needs a CUDA GPU")]


def table_weights():
    """Table I weights in the library's velocity order (four groups of four)."""
    s6 = math.sqrt(6.0)
    wt = [(5 + 2 * s6) / 48, 1 / 48, 1 / 48, (5 - 2 * s6) / 48]
    return [wt[k // 4] for k in range(16)]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_histogram_noalloc_matches_lbm_histogram(prec):
    import torch

    import paper_1802_01272_gb300 as P
    from paper_1802_01272_gb300.binding import histogram_noalloc

    precision = {"fp64": P.LBM_FP64, "fp32": P.LBM_FP32_SHIFTED, "fp16": P.LBM_FP16_SHIFTED}[prec]
    rho_ref = 0.0 if prec == "fp64" else 1.9
    lp = P.Params(Lx=200, Ly=150, precision=precision, T=0.8, rho_ref=rho_ref if rho_ref else 1.0)
    rho, ux, uy = synth.bubble(200, 150, 1.9, 0.24, R=40, W=3)
    stream = torch.cuda.current_stream()
    with P.Lattice(lp, stream) as L:
        L.init_rho_u(rho, ux, uy)
        L.step(3)
        f = torch.empty((16, 150, 200), dtype=torch.float64, device="cuda")
        L.get_f_device(f)
        L.sync()
        if prec != "fp64":
            # the stored deviations f - w rho_ref, recovered exactly in their own type
            w = torch.tensor(table_weights(), dtype=torch.float64, device="cuda")
            dt = torch.float32 if prec == "fp32" else torch.float16
            f = (f - w[:, None, None] * rho_ref).to(dt).contiguous()
        for nbins, lo, hi in ((512, 0.0, 3.0), (64, 0.2, 2.0)):   # two calls in a row
            want = L.histogram(nbins, lo, hi)
            got = histogram_noalloc(f, precision, rho_ref, nbins, lo, hi, stream)
            assert got.sum() == want.sum() > 0
            assert np.array_equal(got, want)
        # the maximum is enforced
        with pytest.raises(P.LBMError) as e:
            histogram_noalloc(f, precision, rho_ref, 4097, 0.0, 3.0, stream)
        assert e.value.code == -1
