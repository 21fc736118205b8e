"""The sum at three times the benchmark on every loop (B=1536, P=4915, G=98304, nw=3;
15.5 GB of (igp, ig) arrays, ~0.94 M tiles), drawn on the device.

The full FP64 sum at this size takes over a minute, so the FP64 checks run on the first
16 bands at full P and G: the GPU result against the oracle on sampled columns (computed
one by one on the host), and the full launch against the sum of four launches over column
ranges (a property that holds at any size and fails on an indexing or tile-count error).
The FP32-bulk path runs the full instance and is held to the same additivity, and on 64
columns with every band (the B = 1536 band loop) to the FP64 result of the same columns.
"""

import numpy as np
import pytest

import oracle
from paper_2008_11326_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def large():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11326_gb300 import gpp
    dp = gpp.DeviceProblem(**inputs.make_device_arrays(**inputs.CONFIGS["large"], device="cuda"))
    yield gpp, dp
    del dp
    torch.cuda.empty_cache()


def bands(gpp, dp, n):
    return gpp.DeviceProblem(n, dp.nvband, dp.ncouls, dp.ngpown, dp.nw, dp.aqsmtemp[:n],
                             dp.aqsntemp[:n], dp.I_eps_array, dp.wtilde_array, dp.vcoul,
                             dp.inv_igp_index, dp.indinv, dp.wx_array[:n],
                             None if dp.aqsntemp_c64 is None else dp.aqsntemp_c64[:n])


def column_sum(gpp, dp, nchunks, **opts):
    from paper_2008_11326_gb300 import shard
    tot = None
    for r in range(nchunks):
        lo, hi = shard.column_range(dp.ngpown, r, nchunks)
        a, s = gpp.sigma(shard.restrict_columns(dp, lo, hi), **opts)
        v = np.concatenate([a.cpu().numpy(), s.cpu().numpy()])
        tot = v if tot is None else tot + v
    return tot


def host_columns(dp, cols):
    """The host problem of the given local columns (all bands and G-vectors of dp)."""
    c = [int(p) for p in cols]
    h = lambda t: t.cpu().numpy()  # noqa: E731
    return inputs.GppProblem(dp.number_bands, dp.nvband, dp.ncouls, len(c), dp.nw,
                             h(dp.aqsmtemp), h(dp.aqsntemp), h(dp.I_eps_array[c]),
                             h(dp.wtilde_array[c]), h(dp.vcoul), h(dp.inv_igp_index[c]),
                             h(dp.indinv), h(dp.wx_array))


def rel(got, ref):
    return float(np.max(np.abs(got - ref) / np.abs(ref)))


def test_fp64_band_subset(large):
    import torch
    gpp, dp = large
    sub = bands(gpp, dp, 16)
    a, s = gpp.sigma(sub)
    full = np.concatenate([a.cpu().numpy(), s.cpu().numpy()])
    assert np.all(np.isfinite(full))
    assert rel(column_sum(gpp, sub, 4), full) <= 1e-13
    cols = [0, 1, 2457, dp.ngpown - 1]
    idx = torch.tensor(cols, device=dp.wtilde_array.device)
    pick = gpp.DeviceProblem(sub.number_bands, sub.nvband, sub.ncouls, len(cols), sub.nw,
                             sub.aqsmtemp, sub.aqsntemp, sub.I_eps_array[idx].contiguous(),
                             sub.wtilde_array[idx].contiguous(), sub.vcoul,
                             sub.inv_igp_index[idx].contiguous(), sub.indinv, sub.wx_array)
    ga, gs = gpp.sigma(pick)
    ref = np.concatenate(oracle.sigma(host_columns(sub, cols)))
    assert rel(np.concatenate([ga.cpu().numpy(), gs.cpu().numpy()]), ref) <= 1e-12


def test_fp32_bulk_full_instance(large):
    gpp, dp = large
    dp.make_c64()
    a, s = gpp.sigma(dp, precision="fp32_bulk")
    full = np.concatenate([a.cpu().numpy(), s.cpu().numpy()])
    assert np.all(np.isfinite(full))
    assert rel(column_sum(gpp, dp, 3, precision="fp32_bulk"), full) <= 1e-6
    # every band (the B = 1536 loop) on 64 columns, against the FP64 path on the same
    # columns (the FP64 path matches the oracle to 1e-12)
    cols = gpp.DeviceProblem(dp.number_bands, dp.nvband, dp.ncouls, 64, dp.nw, dp.aqsmtemp,
                             dp.aqsntemp, dp.I_eps_array[:64], dp.wtilde_array[:64], dp.vcoul,
                             dp.inv_igp_index[:64], dp.indinv, dp.wx_array, dp.aqsntemp_c64)
    a32, s32 = gpp.sigma(cols, precision="fp32_bulk")
    a64, s64 = gpp.sigma(cols)
    assert rel(np.concatenate([a32.cpu().numpy(), s32.cpu().numpy()]),
               np.concatenate([a64.cpu().numpy(), s64.cpu().numpy()])) <= 1e-6
