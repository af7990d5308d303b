"""FP64 CPU oracle of the QTB / QTB-PIMD hot path.

TEST INFRASTRUCTURE.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU baseline of ``bench.py`` may import, call or execute anything in this
package.  The product path never does, and the two share no code.

The oracle has two halves:

* ``qtb_oracle.c`` (plain C, FP64): Philox4x32-10 white noise, the direct
  coloured-noise convolution, the normal-mode matrix, brute-force periodic
  pair forces, the BAOAB ring-polymer integrator and the observables of Eq. 5.
* ``spectra.py`` (numpy, FP64): theta of Eq. 1, kappa_P of Eq. 10, the cutoff
  and the filter taps.

``build()`` compiles the C half into ``oracle/_build/libqtb_oracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from . import spectra  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qtb_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libqtb_oracle.so")
NREC = 23

POT_PAIR, POT_HARMONIC, POT_DOUBLEWELL = 0, 1, 2


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = np.ctypeslib.ndpointer(np.float64, flags="C")
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C")
        L.ora_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.ora_white.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int64]
        L.ora_white.restype = C.c_double
        L.ora_white_block.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, C.c_int64, C.c_int, dp]
        L.ora_colored_block.argtypes = [C.c_uint64, C.c_uint32, C.c_int, C.c_int64, C.c_int, C.c_int, dp, dp]
        L.ora_nm_matrix.argtypes = [C.c_int, dp]
        L.ora_nm_freqs.argtypes = [C.c_int, C.c_double, dp]
        L.ora_pair_forces.argtypes = [C.c_int, dp, C.c_void_p, dp, C.c_int, dp, dp, dp, dp,
                                      C.c_double, C.c_double, C.c_int, C.c_void_p, dp,
                                      C.POINTER(C.c_double), dp]
        L.ora_sim_create.argtypes = [C.c_void_p]
        L.ora_sim_create.restype = C.c_void_p
        L.ora_sim_destroy.argtypes = [C.c_void_p]
        L.ora_sim_step.argtypes = [C.c_void_p, C.c_int64, C.c_void_p]
        L.ora_sim_observe.argtypes = [C.c_void_p, dp]
        L.ora_sim_get.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)]
        L.ora_sim_set.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]
        L.ora_sim_cell.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.ora_sim_set_cell.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_int]
        _lib = L
    return _lib


def philox(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().ora_philox4x32_10(np.ascontiguousarray(ctr, np.uint32), np.ascontiguousarray(key, np.uint32), out)
    return out


def white(seed, sys, dof, n, stream=0):
    return lib().ora_white(seed, sys, dof, stream, n)


def white_block(seed, sys, ndof, n0, nsteps, stream=0):
    out = np.zeros((ndof, nsteps))
    lib().ora_white_block(seed, sys, stream, ndof, n0, nsteps, out)
    return out


def colored_block(seed, sys, ndof, n0, nsteps, h):
    h = np.ascontiguousarray(h, np.float64)
    out = np.zeros((ndof, nsteps))
    lib().ora_colored_block(seed, sys, ndof, n0, nsteps, len(h) - 1, h, out)
    return out


def nm_matrix(P):
    Cm = np.zeros((P, P))
    lib().ora_nm_matrix(P, Cm)
    return Cm


def nm_freqs(P, T):
    w = np.zeros(P)
    lib().ora_nm_freqs(P, T, w)
    return w


def pair_forces(x, types, box, pot, sel=None):
    """Forces (on ``sel`` atoms, or all), energy and virial of one periodic replica."""
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
    N = x.shape[0]
    types = np.ascontiguousarray(types, np.int32)
    box = np.ascontiguousarray(box, np.float64)
    nt = len(pot["mass"])
    arr = lambda k, n: np.ascontiguousarray(np.asarray(pot[k], np.float64).reshape(n))  # noqa: E731
    if sel is not None:
        sel = np.ascontiguousarray(sel, np.int32)
    nsel = N if sel is None else len(sel)
    f = np.zeros((nsel, 3))
    e = C.c_double(0.0)
    vir = np.zeros(9)
    lib().ora_pair_forces(N, x, types.ctypes.data, box, nt, arr("charge", nt), arr("buck_A", nt * nt),
                          arr("buck_rho", nt * nt), arr("buck_C", nt * nt), float(pot["dsf_alpha"]),
                          float(pot["r_cut"]), nsel, None if sel is None else sel.ctypes.data, f,
                          C.byref(e), vir)
    return f, e.value, vir.reshape(3, 3)


class _Params(C.Structure):
    _fields_ = [("N", C.c_int), ("P", C.c_int), ("ntypes", C.c_int), ("potential", C.c_int),
                ("noise", C.c_int), ("box", C.c_double * 3), ("T", C.c_double), ("gamma", C.c_double),
                ("dt", C.c_double), ("alpha", C.c_double), ("rc", C.c_double), ("ext_w0", C.c_double),
                ("ext_V0", C.c_double), ("ext_a", C.c_double), ("seed", C.c_uint64), ("sys", C.c_uint32),
                ("pad0", C.c_int32), ("mass", C.c_void_p), ("charge", C.c_void_p), ("bA", C.c_void_p),
                ("brho", C.c_void_p), ("bC", C.c_void_p), ("type", C.c_void_p), ("x0", C.c_void_p),
                ("v0", C.c_void_p), ("K", C.c_int), ("pad1", C.c_int32), ("h", C.c_void_p),
                ("npt", C.c_int), ("pad2", C.c_int32), ("pext", C.c_double), ("wmass", C.c_double),
                ("gamma_e", C.c_double)]


class Sim:
    """One system (N atoms x P beads) advanced by the oracle's BAOAB integrator.

    ``pos``/``vel`` are [P, N, 3]; ``taps`` (h_0..h_K) selects coloured noise,
    ``None`` white Langevin noise at temperature T.  ``npt`` = dict(pressure
    (eV/A^3), mass (eV fs^2), gamma (1/fs)) makes the run isothermal-isobaric
    (pair potential; ring polymers through their centroids; see qtb_oracle.c).
    """

    def __init__(self, pos, vel, types, pot, box, T, gamma, dt, seed, sys=0, taps=None,
                 potential=POT_PAIR, ext=None, npt=None):
        pos = np.ascontiguousarray(pos, np.float64)
        P, N = pos.shape[0], pos.shape[1]
        vel = np.zeros_like(pos) if vel is None else np.ascontiguousarray(vel, np.float64)
        nt = len(pot["mass"])
        keep = {
            "mass": np.ascontiguousarray(pot["mass"], np.float64),
            "charge": np.ascontiguousarray(pot.get("charge", np.zeros(nt)), np.float64),
            "bA": np.ascontiguousarray(np.asarray(pot.get("buck_A", np.zeros((nt, nt)))).reshape(-1), np.float64),
            "brho": np.ascontiguousarray(np.asarray(pot.get("buck_rho", np.ones((nt, nt)))).reshape(-1), np.float64),
            "bC": np.ascontiguousarray(np.asarray(pot.get("buck_C", np.zeros((nt, nt)))).reshape(-1), np.float64),
            "type": np.ascontiguousarray(types, np.int32),
            "x0": pos, "v0": vel,
        }
        if taps is not None:
            keep["h"] = np.ascontiguousarray(taps, np.float64)
        self._keep = keep
        ext = ext or {}
        p = _Params()
        p.N, p.P, p.ntypes, p.potential = N, P, nt, potential
        p.noise = 0 if taps is None else 1
        for c in range(3):
            p.box[c] = float(box[c]) if box is not None else 0.0
        p.T, p.gamma, p.dt = float(T), float(gamma), float(dt)
        p.alpha = float(pot.get("dsf_alpha", 0.0))
        p.rc = float(pot.get("r_cut", 0.0))
        p.ext_w0 = float(ext.get("omega", 0.0))
        p.ext_V0 = float(ext.get("V0", 0.0))
        p.ext_a = float(ext.get("a", 1.0))
        p.seed, p.sys = int(seed), int(sys)
        for k in ("mass", "charge", "bA", "brho", "bC", "type", "x0", "v0"):
            setattr(p, k, keep[k].ctypes.data)
        if taps is not None:
            p.K = len(taps) - 1
            p.h = keep["h"].ctypes.data
        if npt is not None:
            assert potential == POT_PAIR
            p.npt = 1
            p.pext, p.wmass, p.gamma_e = float(npt["pressure"]), float(npt["mass"]), float(npt["gamma"])
        self.N, self.P = N, P
        self._p = p
        self._s = lib().ora_sim_create(C.byref(p))

    def __del__(self):
        if getattr(self, "_s", None):
            lib().ora_sim_destroy(self._s)
            self._s = None

    def step(self, n, record=True):
        rec = np.zeros((n, NREC)) if record else None
        lib().ora_sim_step(self._s, n, None if rec is None else rec.ctypes.data)
        return rec

    def observe(self):
        rec = np.zeros(NREC)
        lib().ora_sim_observe(self._s, rec)
        return rec

    def state(self):
        shp = (self.P, self.N, 3)
        x, v, f = np.zeros(shp), np.zeros(shp), np.zeros(shp)
        st = C.c_int64(0)
        lib().ora_sim_get(self._s, x.ctypes.data, v.ctypes.data, f.ctypes.data, C.byref(st))
        return x, v, f, st.value

    def cell(self):
        """(cell edges [3] in A, cell momentum p_e in eV fs)."""
        box = np.zeros(3)
        pe = C.c_double(0.0)
        lib().ora_sim_cell(self._s, box.ctypes.data, C.byref(pe))
        return box, pe.value

    def set_cell(self, box, peps, pending=1):
        box = np.ascontiguousarray(box, np.float64)
        lib().ora_sim_set_cell(self._s, box.ctypes.data, float(peps), int(pending))

    def set_state(self, x, v, step):
        x = np.ascontiguousarray(x, np.float64)
        v = np.ascontiguousarray(v, np.float64)
        lib().ora_sim_set(self._s, x.ctypes.data, v.ctypes.data, int(step))
