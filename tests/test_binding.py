"""The Python binding's own checks (no GPU needed): before it hands pointers to libgpp, it
checks every tensor's dtype, shape, device and layout against the problem's sizes, since
the library reads exactly the extents that include/gpp.h gives for those sizes."""

import pytest
import torch

from paper_2008_11326_gb300 import gpp, inputs


def host_problem(B=5, G=64, P=3, W=3, c64=True):
    return gpp.DeviceProblem.from_host(inputs.make_problem(B, 2, G, P, W, seed=1),
                                       device="cpu", c64=c64)


def test_consistent_problems_pass():
    hp = host_problem()
    out = torch.empty(3, dtype=torch.complex128)
    hp.check(out, out.clone())
    hp.struct(None, None)
    host_problem(B=0).check()          # empty sums keep consistent (zero-size) shapes
    host_problem(B=3, G=0, P=0).check()


@pytest.mark.parametrize("field,bad", [
    ("wx_array", lambda t: t[:, :2].contiguous()),            # wrong nw extent
    ("aqsntemp", lambda t: t.to(torch.complex64)),             # wrong dtype
    ("indinv", lambda t: t[:-1]),                              # missing sentinel
    ("I_eps_array", lambda t: t.t()),                          # transposed view
    ("inv_igp_index", lambda t: t.to(torch.int64)),            # 64-bit indices
    ("aqsntemp_c64", lambda t: t[:, :-1].contiguous()),        # short FP32 copy
])
def test_mismatched_tensors_are_rejected(field, bad):
    hp = host_problem()
    setattr(hp, field, bad(getattr(hp, field)))
    with pytest.raises(ValueError, match=field):
        hp.struct(None, None)


def test_short_outputs_are_rejected():
    hp = host_problem()
    with pytest.raises(ValueError, match="achtemp"):
        hp.struct(torch.empty(2, dtype=torch.complex128), None)
    with pytest.raises(ValueError, match="asxtemp"):
        hp.struct(None, torch.empty(3, dtype=torch.complex64))
