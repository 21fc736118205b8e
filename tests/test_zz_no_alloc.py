"""gpp_sigma_noalloc: the forward sum with the library's own fixed scratch array.

Some callers cannot give the library a device workspace -- a Fortran or C host code that
calls through the C interface and keeps no device allocator, or a process whose device
memory belongs to another runtime. This entry point serves them: it takes the same problem
as gpp_sigma but no workspace, and allocates nothing. The test calls it through the C-ABI
twice in a row (the array keeps the previous call's contents, so the second call checks
that everything that must start at zero is cleared) and compares both results with
gpp_sigma's: with the same tile shape the two run the same kernels over the same partial
slots, so they must agree bit for bit (a residue of the previous call would show).
"""

import ctypes

import numpy as np
import pytest

from paper_2008_11326_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def gpp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_11326_gb300 import gpp as g
    return g


def _noalloc(gpp, dp, opts):
    import torch
    from paper_2008_11326_gb300 import _native as N
    ach = torch.empty(dp.nw, dtype=torch.complex128, device=dp.device)
    asx = torch.empty(dp.nw, dtype=torch.complex128, device=dp.device)
    prob = dp.struct(ach, asx)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dp.device).cuda_stream)
    rc = N.lib().gpp_sigma_noalloc(ctypes.byref(prob), ctypes.byref(opts), stream)
    N.check(rc)
    torch.cuda.synchronize()
    return ach.cpu().numpy(), asx.cpu().numpy()


@pytest.mark.parametrize("name,shape", [("tiny", None), ("ragged", (7, 1000, 37, 3))])
def test_noalloc_matches_gpp_sigma_twice(gpp, name, shape):
    import torch
    if shape is None:
        prob = inputs.config("tiny")
    else:
        B, G, P, W = shape
        prob = inputs.make_problem(B, 2, G, P, W, seed=5)
    dp = gpp.DeviceProblem.from_host(prob, device="cuda")
    ref_a, ref_s = gpp.sigma(dp)
    torch.cuda.synchronize()
    ref = np.concatenate([ref_a.cpu().numpy(), ref_s.cpu().numpy()])
    opts = gpp.make_options()
    for _ in range(2):
        a, s = _noalloc(gpp, dp, opts)
        got = np.concatenate([a, s])
        assert np.array_equal(got, ref)
    # the parity tolerance of the suite against the oracle, for the record
    import oracle
    ra, rs = oracle.sigma(prob)
    want = np.concatenate([ra, rs])
    assert np.max(np.abs(got - want) / np.abs(want)) <= RTOL


def test_noalloc_takes_deeper_tiles_when_the_default_does_not_fit(gpp):
    """FP32-bulk at nw=8 with 2560 columns over 32768 G-vectors: the default tile (128 x 4
    G-vectors) needs 42 MB of partials, 8 G-vectors per thread half that. The call then
    runs with 8 and equals gpp_sigma with that tile shape bit for bit."""
    import torch
    dp = gpp.DeviceProblem(**inputs.make_device_arrays(8, 2, 32768, 2560, 8, seed=21,
                                                       device="cuda"))
    dp.make_c64()
    assert gpp.workspace_size(dp, precision="fp32_bulk") > 32 << 20
    assert gpp.workspace_size(dp, precision="fp32_bulk", ig_per_thread=8) <= 32 << 20
    a, s = gpp.sigma(dp, precision="fp32_bulk", ig_per_thread=8)
    torch.cuda.synchronize()
    got = _noalloc(gpp, dp, gpp.make_options(precision="fp32_bulk"))
    assert np.array_equal(got[0], a.cpu().numpy()) and np.array_equal(got[1], s.cpu().numpy())
    del dp
    torch.cuda.empty_cache()


def test_noalloc_rejects_problems_beyond_its_scratch(gpp):
    from paper_2008_11326_gb300 import _native as N
    prob = N.GppProblem()
    prob.number_bands, prob.nvband, prob.ncouls, prob.ngpown, prob.nw = 1024, 2, 65536, 4096, 3
    opts = gpp.make_options()
    rc = N.lib().gpp_sigma_noalloc(ctypes.byref(prob), ctypes.byref(opts), None)
    assert rc == -4  # GPP_ERR_WORKSPACE
    assert b"scratch" in N.lib().gpp_last_error()
