"""ctypes wrapper of the plain FP64 C oracle (``gpp_oracle.c``). Test infrastructure.

The C source states what is computed and from which parts of the paper; this wrapper
only builds the shared library with gcc and marshals numpy arrays.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "gpp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle_gpp.so")
_lock = threading.Lock()
_default = None

OCC_ALL = 0
OCC_OCCUPIED = 1

CFLAGS = ["-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
          "-shared"]


def lib_path() -> str:
    return _LIB


def compile_oracle(src: str, out: str) -> str:
    """Compile one oracle source with gcc: -O2, no FMA contraction, no fast-math, OpenMP."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(SOURCE)):
        return _LIB
    return compile_oracle(SOURCE, _LIB)


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


class Oracle:
    """One loaded copy of the oracle library."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        lib.oracle_gpp_sigma.restype = i32
        dbl = ctypes.c_double
        lib.oracle_gpp_sigma.argtypes = [i64, i64, i64, i64, i64, i32, i32, dbl,
                                         vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32]
        lib.oracle_gpp_sigma_adjoint.restype = i32
        lib.oracle_gpp_sigma_adjoint.argtypes = [i64, i64, i64, i64, i64, i32, i32, dbl,
                                                 vp, vp, vp, vp, vp, vp, vp, vp,
                                                 vp, vp, vp, vp, vp, vp, i32]
        lib.oracle_gpp_branch.restype = i32
        lib.oracle_gpp_branch.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        self.lib = lib
        self.path = path

    @staticmethod
    def _inputs(prob):
        keep, ptrs = [], []
        B, G, P, W = prob.number_bands, prob.ncouls, prob.ngpown, prob.nw
        spec = (("aqsmtemp", np.complex128, (B, G)), ("aqsntemp", np.complex128, (B, G)),
                ("I_eps_array", np.complex128, (P, G)),
                ("wtilde_array", np.complex128, (P, G)), ("vcoul", np.float64, (G,)),
                ("inv_igp_index", np.int32, (P,)), ("indinv", np.int32, (G + 1,)),
                ("wx_array", np.float64, (B, W)))
        for name, dt, shp in spec:
            a, p = _c(getattr(prob, name), dt)
            if a.shape != shp:
                raise ValueError(f"oracle input {name} has shape {a.shape}, want {shp}")
            keep.append(a)
            ptrs.append(p)
        return keep, ptrs

    def sigma(self, prob, occ_mode: int = OCC_ALL, nthreads: int = 0, ch_half: bool = False,
              sexcut: float = 0.0):
        """Return (achtemp, asxtemp) as complex128 arrays of length nw. ``ch_half`` and
        ``sexcut`` are the Sigma-code options described in the C source (off by default)."""
        keep, ptrs = self._inputs(prob)
        W = prob.nw
        ach = np.zeros(W, np.complex128)
        asx = np.zeros(W, np.complex128)
        rc = self.lib.oracle_gpp_sigma(prob.number_bands, prob.nvband, prob.ncouls,
                                       prob.ngpown, W, occ_mode, int(bool(ch_half)),
                                       float(sexcut), *ptrs, ach.ctypes.data,
                                       asx.ctypes.data, nthreads)
        if rc != 0:
            raise RuntimeError(f"oracle_gpp_sigma failed with {rc}")
        del keep
        return ach, asx

    def sigma_adjoint(self, prob, g_ach, g_asx, occ_mode: int = OCC_ALL, nthreads: int = 0,
                      want=("wtilde", "I_eps", "aqsm", "aqsn"), ch_half: bool = False,
                      sexcut: float = 0.0):
        """Gradients of L with dL = Re(sum conj(g_ach) d ach + conj(g_asx) d asx).

        Returns a dict of complex128 arrays (torch convention dL/dRe + i dL/dIm) for the
        requested inputs: wtilde [P][G], I_eps [P][G], aqsm [B][G], aqsn [B][G].
        """
        keep, ptrs = self._inputs(prob)
        B, G, P, W = prob.number_bands, prob.ncouls, prob.ngpown, prob.nw
        ga, gap = _c(np.asarray(g_ach).reshape(W), np.complex128)
        gs, gsp = _c(np.asarray(g_asx).reshape(W), np.complex128)
        shapes = {"wtilde": (P, G), "I_eps": (P, G), "aqsm": (B, G), "aqsn": (B, G)}
        out = {k: np.zeros(shapes[k], np.complex128) for k in want}
        ptr = {k: (out[k].ctypes.data if k in out else None) for k in shapes}
        rc = self.lib.oracle_gpp_sigma_adjoint(B, prob.nvband, G, P, W, occ_mode,
                                               int(bool(ch_half)), float(sexcut), *ptrs,
                                               gap, gsp, ptr["wtilde"], ptr["I_eps"],
                                               ptr["aqsm"], ptr["aqsn"], nthreads)
        if rc != 0:
            raise RuntimeError(f"oracle_gpp_sigma_adjoint failed with {rc}")
        del keep, ga, gs
        return out

    def branch(self, w: complex, x: float) -> int:
        """The branch (1, 2 or 3) the oracle takes for one (w, x)."""
        return int(self.lib.oracle_gpp_branch(float(np.real(w)), float(np.imag(w)), float(x)))


def default() -> Oracle:
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
        return _default


def sigma(prob, occ_mode: int = OCC_ALL, nthreads: int = 0, ch_half: bool = False,
          sexcut: float = 0.0):
    return default().sigma(prob, occ_mode, nthreads, ch_half, sexcut)


def sigma_adjoint(prob, g_ach, g_asx, occ_mode: int = OCC_ALL, nthreads: int = 0,
                  want=("wtilde", "I_eps", "aqsm", "aqsn"), ch_half: bool = False,
                  sexcut: float = 0.0):
    return default().sigma_adjoint(prob, g_ach, g_asx, occ_mode, nthreads, want, ch_half,
                                   sexcut)


def branch(w: complex, x: float) -> int:
    return default().branch(w, x)
