"""CPU oracle for the Line Segment Tracking hot path: ctypes binding and build step.

TEST INFRASTRUCTURE ONLY. The product path (the CUDA library and its Python binding) never imports
this package; only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg do.
The oracle itself is ``lst_oracle.cpp``: plain FP64 loops written from the paper's description of
each stage. Parity-pinned by ``tests/test_oracle_pins.py`` and ``tests/test_oracle_bruteforce.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lst_oracle.cpp")
_LIB = os.path.join(_HERE, "liblst_oracle.so")
_lock = threading.Lock()
_lib = None

# table ids and column layouts of the C interface
T_ORDER, T_OFFSETS, T_MD, T_LS, T_T3, T_T5, T_PLSBIN, T_PT3, T_PT5, T_TC, T_T5KEPT, T_TCEXT = range(12)
I_COLS = {
    T_MD: ["hit_lo", "hit_up", "module", "pass", "definite"],
    T_LS: ["md_in", "md_out", "pass", "definite"],
    T_T3: ["ls_in", "ls_out", "pass", "definite", "md0", "md1", "md2"],
    T_T5: ["t3_in", "t3_out", "pass", "definite", "md0", "md1", "md2", "md3", "md4"],
    T_PT3: ["pls", "obj", "pass", "definite"],
    T_PT5: ["pls", "obj", "pass", "definite"],
    T_TC: ["type", "obj"] + [f"hit{k}" for k in range(14)],
    T_TCEXT: ["t3", "n_add", "definite"] + [f"hit{k}" for k in range(4)],
}
F_COLS = {
    T_MD: ["dphichange", "pt_est", "x", "y", "z", "r"],
    T_LS: ["z0", "dphi"],
    T_T3: ["R", "xc", "yc", "chi2_rz", "pt_est"],
    T_T5: ["kappa_in", "kappa_out", "kappa_fit", "chi2_c", "chi2_rz", "eta", "phi", "pt"],
    T_PT3: ["chi2_xy", "chi2_rz", "score"],
    T_PT5: ["chi2_xy", "chi2_rz", "score"],
    T_TC: ["pt", "eta", "phi"],
    T_TCEXT: ["chi2_c", "chi2_rz"],
}
TABLE_NAMES = {T_MD: "md", T_LS: "ls", T_T3: "t3", T_T5: "t5", T_PT3: "pt3", T_PT5: "pt5", T_TC: "tc",
               T_TCEXT: "tc_ext"}


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP64, no fused multiply-add contraction, no fast-math)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        tmp = f"{_LIB}.{os.getpid()}.tmp"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_run.restype = ctypes.c_void_p
        L.orc_run.argtypes = [ctypes.c_double, ctypes.c_void_p, ctypes.c_int32] + [ctypes.c_void_p] * 4 + \
            [ctypes.c_int32] + [ctypes.c_void_p] * 4 + [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]
        L.orc_free.argtypes = [ctypes.c_void_p]
        L.orc_count.restype = ctypes.c_int64
        L.orc_count.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        L.orc_get_i32.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
        L.orc_get_f64.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
        L.orc_constants.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_constants.restype = ctypes.c_int
        L.orc_circumcircle.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.orc_karimaki.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_line_fit.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_line_fit.restype = ctypes.c_double
        L.orc_pixel_bin.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_int32]
        L.orc_pixel_bin.restype = ctypes.c_int32
        L.orc_seed_terms.argtypes = [ctypes.c_void_p, ctypes.c_int32] + [ctypes.c_void_p] * 6
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def constants() -> np.ndarray:
    out = np.zeros(64, dtype=np.float64)
    n = lib().orc_constants(_p(out), 64)
    return out[:n]


def run(det, ev, brute_force: bool = False) -> dict:
    """Run the whole chain on one event; returns {table: {column: ndarray}}."""
    L = lib()
    mods = np.ascontiguousarray(det.geom.module_records())
    co = np.ascontiguousarray(det.conn_off, dtype=np.int32)
    ct = np.ascontiguousarray(det.conn_tgt, dtype=np.int32)
    po = np.ascontiguousarray(det.pix_off, dtype=np.int32)
    pt = np.ascontiguousarray(det.pix_tgt, dtype=np.int32)
    n_pix = int(po.size - 1) if pt.size else 0
    x = np.ascontiguousarray(ev.x, dtype=np.float32)
    y = np.ascontiguousarray(ev.y, dtype=np.float32)
    z = np.ascontiguousarray(ev.z, dtype=np.float32)
    s = np.ascontiguousarray(ev.sensor, dtype=np.int32)
    pls = np.ascontiguousarray(ev.pls)
    if pt.size == 0:
        pt = np.zeros(1, dtype=np.int32)
    h = L.orc_run(float(np.float32(det.pt_thr)), _p(mods), det.n_mods, _p(co), _p(ct), _p(po), _p(pt), n_pix,
                  _p(x), _p(y), _p(z), _p(s), int(x.size), _p(pls) if pls.size else None, int(pls.size),
                  1 if brute_force else 0)
    try:
        out = {}
        n = L.orc_count(h, T_ORDER)
        a = np.zeros(n, dtype=np.int32)
        L.orc_get_i32(h, T_ORDER, 0, _p(a))
        out["order"] = a
        n = L.orc_count(h, T_OFFSETS)
        a = np.zeros(n, dtype=np.int32)
        L.orc_get_i32(h, T_OFFSETS, 0, _p(a))
        out["offsets"] = a
        n = L.orc_count(h, T_PLSBIN)
        a = np.zeros(n, dtype=np.int32)
        if n:
            L.orc_get_i32(h, T_PLSBIN, 0, _p(a))
        out["pls_bin"] = a
        n = L.orc_count(h, T_T5KEPT)
        a = np.zeros(n, dtype=np.int32)
        if n:
            L.orc_get_i32(h, T_T5KEPT, 0, _p(a))
        out["t5_kept"] = a.astype(bool)
        for t, name in TABLE_NAMES.items():
            n = int(L.orc_count(h, t))
            tab = {}
            for c, col in enumerate(I_COLS[t]):
                a = np.zeros(n, dtype=np.int32)
                if n:
                    L.orc_get_i32(h, t, c, _p(a))
                tab[col] = a
            for c, col in enumerate(F_COLS[t]):
                a = np.zeros(n, dtype=np.float64)
                if n:
                    L.orc_get_f64(h, t, c, _p(a))
                tab[col] = a
            for col in ("pass", "definite"):
                if col in tab:
                    tab[col] = tab[col].astype(bool)
            out[name] = tab
        return out
    finally:
        L.orc_free(h)


def circumcircle(p):
    out = np.zeros(3)
    lib().orc_circumcircle(_p(np.ascontiguousarray(p, dtype=np.float64)), _p(out))
    return out


def karimaki(x, y):
    """(rho, phi, d, sum of squared geometric residuals) of Karimaki's fit with equal weights."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    out = np.zeros(4)
    lib().orc_karimaki(int(x.size), _p(x), _p(y), _p(out))
    return out


def line_fit(s, z, sig):
    s = np.ascontiguousarray(s, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    sig = np.ascontiguousarray(sig, dtype=np.float64)
    slope = np.zeros(1)
    chi2 = lib().orc_line_fit(int(s.size), _p(s), _p(z), _p(sig), _p(slope))
    return chi2, float(slope[0])


def pixel_bin(eta, phi, charge):
    return int(lib().orc_pixel_bin(float(eta), float(phi), int(charge)))


def seed_terms(seed, x, y, z, endcap):
    """Per-anchor pT3 / pT5 terms of one seed (a PLS_DTYPE record) against anchors (x, y, z, endcap):
    returns (terms [n, 4] = distance from the seed circle, its variance, z offset from the seed's
    r-z line, its variance; (chi2_xy, chi2_rz))."""
    rec = np.ascontiguousarray(np.asarray(seed).reshape(1))
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    ec = np.ascontiguousarray(endcap, dtype=np.int32)
    terms = np.zeros((x.size, 4))
    chi2 = np.zeros(2)
    lib().orc_seed_terms(_p(rec), int(x.size), _p(x), _p(y), _p(z), _p(ec), _p(terms), _p(chi2))
    return terms, (float(chi2[0]), float(chi2[1]))
