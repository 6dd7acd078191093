"""The in-library FMA issue-rate probe (fizzy_probe_fma_rate), which bench.py
uses as the measured peak of its FP64-bound kernels (needs a B300)."""
import pytest

import paper_2502_04189_b300 as F

pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible(cuda_ok):
    d, ms_d = F.probe_fma_rate(F.FP64, iters=200)
    s, ms_s = F.probe_fma_rate(F.MIXED, iters=2000)
    assert ms_d > 0 and ms_s > 0
    # FP64 FMA issue on this part is a small fraction of FP32's; both are
    # within a decade of the nominal figures (0.625 T DFMA/s, 38 T FFMA/s)
    assert 0.06e12 < d < 6e12, d
    assert 3.8e12 < s < 380e12, s
    assert s > 10 * d
    for op in (1, 2, 3):
        r, _ = F.probe_fma_rate(F.FP64, iters=200, op=op, chains=16)
        assert 0.06e12 < r < 6e12, (op, r)
    for bad in (dict(iters=0), dict(iters=10, op=6), dict(iters=10, chains=5)):
        with pytest.raises(F.FizzyError):
            F.probe_fma_rate(F.FP64, **bad)
