"""The float64 FMA rate probe that bench.py uses as the float64 solver's
arithmetic peak computes what it claims: every thread's eight chains
a <- a b + c match the closed form b^n a0 + c (1 - b^n) / (1 - b)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_fp64_probe_chains_match_closed_form(lib):
    import torch
    psatd = lib
    blocks, threads, iters = 3, 64, 1000
    out = torch.full((blocks * threads,), np.nan, dtype=torch.float64, device="cuda")
    psatd.fp64_fma_probe(out, blocks, threads, iters)
    got = out.cpu().numpy()
    b, c = 1.0 - 2.0 ** -20, 2.0 ** -24
    t = np.arange(blocks * threads)
    bn = b ** iters
    want = sum(bn * (1e-6 * (t & 1023) + k) + c * (1.0 - bn) / (1.0 - b) for k in range(8))
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)
