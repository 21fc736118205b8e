"""The seeded input generator: determinism, shapes, ranges and index structure."""

import numpy as np

from paper_2008_11326_gb300 import inputs


def test_deterministic_and_seed_dependent():
    a = inputs.make_problem(4, 2, 64, 8, 3, seed=7)
    b = inputs.make_problem(4, 2, 64, 8, 3, seed=7)
    c = inputs.make_problem(4, 2, 64, 8, 3, seed=8)
    for f in ("aqsmtemp", "aqsntemp", "I_eps_array", "wtilde_array", "vcoul",
              "inv_igp_index", "indinv", "wx_array"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    assert not np.array_equal(a.aqsmtemp, c.aqsmtemp)


def test_shapes_ranges_and_indices():
    p = inputs.config("tiny")
    B, G, P, W = p.number_bands, p.ncouls, p.ngpown, p.nw
    assert (B, G, P, W) == (32, 512, 64, 3)
    assert p.aqsmtemp.shape == (B, G) and p.aqsmtemp.dtype == np.complex128
    assert p.wtilde_array.shape == (P, G) and p.I_eps_array.shape == (P, G)
    assert p.wx_array.shape == (B, W) and p.indinv.shape == (G + 1,)
    assert np.all(np.abs(p.aqsmtemp.real) <= 1) and np.all(np.abs(p.aqsntemp.imag) <= 1)
    assert np.all((p.I_eps_array.real >= 0.5) & (p.I_eps_array.real <= 1.5))
    assert np.all(np.abs(p.I_eps_array.imag) <= 0.1)
    assert np.all((p.wtilde_array.real >= 0.2) & (p.wtilde_array.real <= 3.0))
    assert np.all(np.abs(p.wtilde_array.imag) <= 0.05)
    assert np.all((p.vcoul >= 0.1) & (p.vcoul <= 10))
    assert len(set(p.inv_igp_index.tolist())) == P and p.inv_igp_index.max() < G
    assert sorted(p.indinv[:G].tolist()) == list(range(G)) and p.indinv[G] == G
    # wx = e_lk - e_n1 + iw * dw with e_n1 in [0, 10): steps of dw along iw
    assert np.allclose(np.diff(p.wx_array, axis=1), inputs.DW)
    assert np.all((p.wx_array[:, 0] > 0) & (p.wx_array[:, 0] <= inputs.E_LK))


def test_band_and_column_subsets():
    p = inputs.make_problem(6, 2, 32, 5, 3, seed=2)
    q = p.bands(slice(0, 2))
    assert q.number_bands == 2 and np.array_equal(q.aqsmtemp, p.aqsmtemp[:2])
    assert np.array_equal(q.wx_array, p.wx_array[:2])
    r = p.columns([1, 3])
    assert r.ngpown == 2 and np.array_equal(r.wtilde_array, p.wtilde_array[[1, 3]])


def test_batched_shapes():
    shapes = inputs.batched_shapes()
    assert len(shapes) == 64
    for s in shapes:
        assert 2048 <= s["ncouls"] <= 32768 and s["ngpown"] == s["ncouls"] // 20
        assert 64 <= s["number_bands"] <= 512 and s["nw"] == 3
    assert len({s["seed"] for s in shapes}) == 64


def test_model_flops():
    assert inputs.model_flops(512, 1638, 32768, 3) == 512 * 1638 * 32768 * 159
