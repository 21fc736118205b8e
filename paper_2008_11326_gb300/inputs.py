"""Seeded synthetic inputs for the GPP self-energy summation.

This module only draws arrays; it holds none of the summation's arithmetic. Both the
CUDA path and the CPU oracle are fed from it, so it imports neither.

The paper benchmarks BerkeleyGW's Si-214 and Si-510 systems (paper §II-A), whose data
sets are not available here. Synthetic arrays of the benchmark shape stand in for them,
drawn with ``numpy.random.Generator(PCG64(seed))`` in a fixed order:

    aqsmtemp.re, aqsmtemp.im, aqsntemp.re, aqsntemp.im, I_eps.re, I_eps.im,
    wtilde.re, wtilde.im, vcoul, inv_igp_index, indinv permutation, e_n1

with the distributions

    aqsmtemp, aqsntemp : re, im ~ U(-1, 1)
    I_eps_array        : re ~ U(0.5, 1.5), im ~ U(-0.1, 0.1)
    wtilde_array       : re ~ U(0.2, 3.0), im ~ U(-0.05, 0.05)
    vcoul              : U(0.1, 10)
    inv_igp_index      : ngpown distinct columns drawn from [0, ncouls)
    indinv             : a permutation of 0..ncouls-1 followed by the sentinel ncouls
    wx_array[b][iw]    : e_lk - e_n1[b] + iw * dw, e_n1 ~ U(0, 10), e_lk = 10, dw = 1

Layout: C row-major, last index contiguous; complex arrays are complex128 (interleaved
re, im), i.e. aqsmtemp/aqsntemp [B][G], I_eps_array/wtilde_array [P][G], wx_array [B][W].
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

E_LK = 10.0
DW = 1.0


@dataclasses.dataclass
class GppProblem:
    """Host-side arrays of one GPP instance (names follow the paper's kernel)."""

    number_bands: int
    nvband: int
    ncouls: int
    ngpown: int
    nw: int
    aqsmtemp: np.ndarray      # complex128 [B][G]
    aqsntemp: np.ndarray      # complex128 [B][G]
    I_eps_array: np.ndarray   # complex128 [P][G]
    wtilde_array: np.ndarray  # complex128 [P][G]
    vcoul: np.ndarray         # float64 [G]
    inv_igp_index: np.ndarray  # int32 [P]
    indinv: np.ndarray        # int32 [G + 1]
    wx_array: np.ndarray      # float64 [B][W]

    @property
    def shape(self):
        return (self.number_bands, self.ngpown, self.ncouls, self.nw)

    def bands(self, sel) -> "GppProblem":
        """The same instance restricted to the bands ``sel`` (a slice or index array)."""
        aqsm = np.ascontiguousarray(self.aqsmtemp[sel])
        return dataclasses.replace(
            self,
            number_bands=aqsm.shape[0],
            aqsmtemp=aqsm,
            aqsntemp=np.ascontiguousarray(self.aqsntemp[sel]),
            wx_array=np.ascontiguousarray(self.wx_array[sel]),
        )

    def columns(self, sel) -> "GppProblem":
        """The same instance restricted to the local columns ``sel`` (igp)."""
        inv = np.ascontiguousarray(self.inv_igp_index[sel])
        return dataclasses.replace(
            self,
            ngpown=inv.shape[0],
            inv_igp_index=inv,
            I_eps_array=np.ascontiguousarray(self.I_eps_array[sel]),
            wtilde_array=np.ascontiguousarray(self.wtilde_array[sel]),
        )

    def replace(self, **kw) -> "GppProblem":
        return dataclasses.replace(self, **kw)

    def nbytes(self) -> int:
        return sum(getattr(self, f).nbytes for f in _ARRAY_FIELDS)


_ARRAY_FIELDS = ("aqsmtemp", "aqsntemp", "I_eps_array", "wtilde_array", "vcoul",
                 "inv_igp_index", "indinv", "wx_array")


def _complex(rng, shape, re_lo, re_hi, im_lo, im_hi):
    out = np.empty(shape, dtype=np.complex128)
    out.real = rng.uniform(re_lo, re_hi, size=shape)
    out.imag = rng.uniform(im_lo, im_hi, size=shape)
    return out


def make_problem(number_bands: int, nvband: int, ncouls: int, ngpown: int, nw: int,
                 seed: int, e_lk: float = E_LK, dw: float = DW) -> GppProblem:
    """Draw one seeded instance with the distributions in the module docstring."""
    B, G, P, W = int(number_bands), int(ncouls), int(ngpown), int(nw)
    if min(B, G, P, W) < 0 or P > G:
        raise ValueError(f"bad sizes B={B} G={G} P={P} W={W}")
    rng = np.random.Generator(np.random.PCG64(seed))
    aqsm = _complex(rng, (B, G), -1.0, 1.0, -1.0, 1.0)
    aqsn = _complex(rng, (B, G), -1.0, 1.0, -1.0, 1.0)
    I_eps = _complex(rng, (P, G), 0.5, 1.5, -0.1, 0.1)
    wtilde = _complex(rng, (P, G), 0.2, 3.0, -0.05, 0.05)
    vcoul = rng.uniform(0.1, 10.0, size=G)
    inv = rng.choice(G, size=P, replace=False).astype(np.int32) if P else np.zeros(0, np.int32)
    indinv = np.empty(G + 1, dtype=np.int32)
    indinv[:G] = rng.permutation(G).astype(np.int32)
    indinv[G] = G
    e_n1 = rng.uniform(0.0, 10.0, size=B)
    wx = (e_lk - e_n1)[:, None] + dw * np.arange(W, dtype=np.float64)[None, :]
    return GppProblem(B, int(nvband), G, P, W, aqsm, aqsn, I_eps, wtilde, vcoul,
                      inv, indinv, np.ascontiguousarray(wx))


def make_device_arrays(number_bands: int, nvband: int, ncouls: int, ngpown: int, nw: int,
                       seed: int, device, e_lk: float = E_LK, dw: float = DW) -> dict:
    """The same distributions as :func:`make_problem`, drawn on ``device`` with a seeded
    ``torch.Generator`` (different values from the numpy draw of the same seed). For
    workloads too large to draw on the host each run; returns a dict of torch tensors with
    the field names of :class:`GppProblem`."""
    import torch
    B, G, P, W = int(number_bands), int(ncouls), int(ngpown), int(nw)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f64 = dict(dtype=torch.float64, device=device)

    def u(shape, lo, hi):
        return torch.rand(shape, generator=g, **f64) * (hi - lo) + lo

    def c(shape, rl, rh, il, ih):
        return torch.complex(u(shape, rl, rh), u(shape, il, ih))
    out = dict(number_bands=B, nvband=int(nvband), ncouls=G, ngpown=P, nw=W)
    out["aqsmtemp"] = c((B, G), -1.0, 1.0, -1.0, 1.0)
    out["aqsntemp"] = c((B, G), -1.0, 1.0, -1.0, 1.0)
    out["I_eps_array"] = c((P, G), 0.5, 1.5, -0.1, 0.1)
    out["wtilde_array"] = c((P, G), 0.2, 3.0, -0.05, 0.05)
    out["vcoul"] = u((G,), 0.1, 10.0)
    out["inv_igp_index"] = torch.randperm(G, generator=g, device=device)[:P].to(torch.int32)
    ind = torch.empty(G + 1, dtype=torch.int32, device=device)
    ind[:G] = torch.randperm(G, generator=g, device=device).to(torch.int32)
    ind[G] = G
    out["indinv"] = ind
    e_n1 = u((B,), 0.0, 10.0)
    out["wx_array"] = ((e_lk - e_n1)[:, None] + dw * torch.arange(W, **f64)[None, :]).contiguous()
    return out


def cotangents(seed: int, nw: int):
    """Loss weights a_iw, b_iw ~ N(0, 1) for L = sum_iw a_iw Re ach[iw] + b_iw Im asx[iw].

    Drawn from their own stream ``PCG64([seed, 7])`` so the problem draws stay as above.
    Returned as torch-convention complex cotangents of achtemp and asxtemp:
    g_ach = a + 0i, g_asx = 0 + i b.
    """
    rng = np.random.Generator(np.random.PCG64([seed, 7]))
    a = rng.standard_normal(nw)
    b = rng.standard_normal(nw)
    return a.astype(np.complex128), (1j * b).astype(np.complex128)


# Named workloads. "tiny" is small enough for the oracle in seconds; "benchmark" is the
# paper-shaped benchmark (band O(1000), igp O(1000), ig O(10000), paper §II-A) used for the
# FP64 throughput number; "mixed" is the same shape for the FP32-bulk path; "adjoint" is the
# gradient workload; "large" scales every loop by 3.
CONFIGS = {
    "tiny": dict(number_bands=32, nvband=2, ncouls=512, ngpown=64, nw=3, seed=0),
    "benchmark": dict(number_bands=512, nvband=2, ncouls=32768, ngpown=1638, nw=3, seed=1),
    "mixed": dict(number_bands=512, nvband=2, ncouls=32768, ngpown=1638, nw=3, seed=2),
    "adjoint": dict(number_bands=128, nvband=2, ncouls=8192, ngpown=410, nw=3, seed=3),
    # three times the benchmark on every loop (the paper's larger system is 3-4x its
    # smaller one on each, §II-A); drawn on the device with make_device_arrays
    "large": dict(number_bands=1536, nvband=2, ncouls=98304, ngpown=4915, nw=3, seed=5),
}


def config(name: str, **override) -> GppProblem:
    kw = dict(CONFIGS[name])
    kw.update(override)
    return make_problem(**kw)


def batched_shapes(n: int = 64, seed: int = 4):
    """Uneven instance shapes for the batched workload.

    ncouls = round(exp(U(ln 2048, ln 32768))), ngpown = ncouls // 20,
    number_bands ~ U{64..512}, nvband = 2, nw = 3; instance i is drawn with seed 1000 + i.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        G = int(round(math.exp(rng.uniform(math.log(2048.0), math.log(32768.0)))))
        B = int(rng.integers(64, 513))
        out.append(dict(number_bands=B, nvband=2, ncouls=G, ngpown=G // 20, nw=3,
                        seed=1000 + i))
    return out


def model_flops(number_bands: int, ngpown: int, ncouls: int, nw: int) -> float:
    """Fixed model FLOP count: 51 per (band, igp, ig, iw) plus 6 per (band, igp, ig).

    Counted with FMA = 2 and mul/add/reciprocal = 1 on the branch-1 path: wdiff 1,
    |wdiff|^2 3, reciprocal 1, delw 8, |delw|^2 3, sch 6, cden 1, |cden|^2 3, reciprocal 1,
    ssx 8, two complex multiply-accumulates 16; the weight M is a complex product (6).
    """
    return float(number_bands) * ngpown * ncouls * (51.0 * nw + 6.0)
