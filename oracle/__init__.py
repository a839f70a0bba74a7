"""CPU oracle of the cluster-preserving correction pass (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does: it runs
only the CUDA library and fails loudly when that library is missing.

The arithmetic lives in ``oracle.cpp`` (plain C++17, float64 for the
optimisation, the canonical float32 link test); this module compiles it on
demand with g++ and wraps it with ctypes and numpy.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.cpp`` into ``liboracle.so`` (no fused multiply-add; OpenMP, whose
    thread count changes the speed and never the results)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("b", C.c_double), ("xi", C.c_double), ("box_lo", C.c_double * 3),
                ("box_hi", C.c_double * 3), ("periodic", C.c_int32), ("mode", C.c_int32),
                ("m_bits", C.c_int32), ("t_max", C.c_int32), ("alpha_rel", C.c_double),
                ("beta1", C.c_double), ("beta2", C.c_double), ("eps_rel", C.c_double),
                ("loss_tol", C.c_double), ("replay_iters", C.c_int32), ("stall_patience", C.c_int32)]


class Consts(C.Structure):
    _fields_ = [("b2", C.c_float), ("lo2", C.c_float), ("hi2", C.c_float), ("L", C.c_float * 3),
                ("w2", C.c_double), ("eps_q", C.c_double), ("u", C.c_double),
                ("xi_box", C.c_double), ("dt", C.c_double), ("thr_link", C.c_double),
                ("thr_non", C.c_double), ("alpha", C.c_double), ("eps_adam", C.c_double),
                ("M", C.c_double), ("tau", C.c_double)]


class PgdStats(C.Structure):
    _fields_ = [("iters", C.c_int64), ("loss_evals", C.c_int64), ("viol0", C.c_int64),
                ("viol_final", C.c_int64), ("loss0", C.c_double), ("loss_final", C.c_double),
                ("n_editable", C.c_int64), ("converged", C.c_int32), ("pad_", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


DEFAULTS = dict(b=1.0, xi=0.1, box_lo=(0.0, 0.0, 0.0), box_hi=(1.0, 1.0, 1.0), periodic=0,
                mode=0, m_bits=16, t_max=10000, alpha_rel=0.2, beta1=0.9, beta2=0.999,
                eps_rel=2e-6, loss_tol=0.0, replay_iters=-1, stall_patience=0)


def make_params(**kw) -> Params:
    d = dict(DEFAULTS)
    d.update(kw)
    p = Params()
    for k, v in d.items():
        if k in ("box_lo", "box_hi"):
            getattr(p, k)[:] = [float(x) for x in v]
        else:
            setattr(p, k, v)
    return p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            f32p, u32p, u8p, i32p, f64p = (C.POINTER(C.c_float), C.POINTER(C.c_uint32),
                                           C.POINTER(C.c_uint8), C.POINTER(C.c_int32),
                                           C.POINTER(C.c_double))
            P = C.POINTER(Params)
            L.or_threads.argtypes = [C.c_int32]
            L.or_threads.restype = C.c_int32
            L.or_constants.argtypes = [P, f32p, f32p, C.c_int64, C.POINTER(Consts)]
            L.or_dist2.argtypes = [f32p, C.c_int64, C.c_int64, P]
            L.or_dist2.restype = C.c_float
            L.or_pairs.argtypes = [f32p, C.c_int64, P, C.c_int32, u32p, u32p, u8p, C.c_int64]
            L.or_pairs.restype = C.c_int64
            L.or_fof_labels.argtypes = [f32p, C.c_int64, P, i32p, i32p]
            L.or_fof_labels.restype = C.c_int64
            L.or_select.argtypes = [f32p, C.c_int64, P, C.c_int32, u32p, u32p, u8p, C.c_int64,
                                    C.POINTER(C.c_int64)]
            L.or_select.restype = C.c_int64
            L.or_pgd.argtypes = [f32p, f32p, C.c_int64, P, u32p, u32p, u8p, C.c_int64, f32p,
                                 f64p, i32p, C.POINTER(PgdStats)]
            L.or_pgd.restype = C.c_int32
            L.or_pgd_thr.argtypes = [f32p, f32p, C.c_int64, P, u32p, u32p, u8p, f64p, C.c_int64, f32p,
                                     f64p, i32p, C.POINTER(PgdStats)]
            L.or_pgd_thr.restype = C.c_int32
            L.or_encode.argtypes = [f32p, f32p, C.c_int64, P, u8p, C.c_int64]
            L.or_encode.restype = C.c_int64
            L.or_decode.argtypes = [f32p, C.c_int64, u8p, C.c_int64, f32p]
            L.or_decode.restype = C.c_int32
            L.or_correct.argtypes = [f32p, f32p, C.c_int64, P, f32p, C.POINTER(PgdStats),
                                     C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
            L.or_correct.restype = C.c_int32
            L.or_count_flips.argtypes = [f32p, C.c_int64, P, u32p, u32p, u8p, C.c_int64]
            L.or_count_flips.restype = C.c_int64
            _lib = L
    return _lib


def threads(n: int = 0) -> int:
    """Sets the oracle's OpenMP thread count (n > 0) and returns the count in use."""
    return int(lib().or_threads(int(n)))


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(C.POINTER(C.c_float))


def _ptr(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def constants(orig, recon=None, **kw) -> dict:
    o, op = _f32(orig)
    rp = None
    if recon is not None:
        r, rp = _f32(recon)
    c = Consts()
    lib().or_constants(C.byref(make_params(**kw)), op, rp, o.shape[0], C.byref(c))
    out = {k: getattr(c, k) for k, _ in Consts._fields_}
    out["L"] = tuple(c.L)
    return out


def dist2(P, i, j, **kw) -> np.float32:
    p, pp = _f32(P)
    return np.float32(lib().or_dist2(pp, i, j, C.byref(make_params(**kw))))


CLS_SAFE, CLS_PB, CLS_PC = 1, 2, 3


def classify(P, i, j, **kw) -> np.ndarray:
    """Class of each pair (i[k], j[k]): 0 far, 1 safe, 2 potentially broken, 3 potentially created."""
    p, pp = _f32(P)
    i = np.ascontiguousarray(i, np.uint32)
    j = np.ascontiguousarray(j, np.uint32)
    out = np.empty(len(i), np.uint8)
    lib().or_classify(pp, p.shape[0], C.byref(make_params(**kw)), _ptr(i, C.c_uint32), _ptr(j, C.c_uint32),
                      len(i), _ptr(out, C.c_uint8))
    return out


def pairs(P, brute=False, **kw):
    """All classified pairs (i < j) sorted by (i, j): returns (i, j, cls)."""
    p, pp = _f32(P)
    n = p.shape[0]
    prm = make_params(**kw)
    cnt = lib().or_pairs(pp, n, C.byref(prm), int(brute), None, None, None, 0)
    i = np.empty(cnt, np.uint32)
    j = np.empty(cnt, np.uint32)
    c = np.empty(cnt, np.uint8)
    lib().or_pairs(pp, n, C.byref(prm), int(brute), _ptr(i, C.c_uint32), _ptr(j, C.c_uint32),
                   _ptr(c, C.c_uint8), cnt)
    return i, j, c


def fof_labels(P, **kw):
    """(labels, safe_labels, n_halos): label = smallest id of the component."""
    p, pp = _f32(P)
    n = p.shape[0]
    lab = np.empty(n, np.int32)
    safe = np.empty(n, np.int32)
    nc = lib().or_fof_labels(pp, n, C.byref(make_params(**kw)), _ptr(lab, C.c_int32),
                             _ptr(safe, C.c_int32))
    return lab, safe, int(nc)


def select(P, mode=None, **kw):
    """Active pairs of ``mode`` sorted by (i, j): (i, j, link, n_vulnerable)."""
    p, pp = _f32(P)
    n = p.shape[0]
    kw = dict(kw)
    if mode is None:
        mode = kw.get("mode", 0)
    kw["mode"] = int(mode)
    prm = make_params(**kw)
    nv = C.c_int64(0)
    cnt = lib().or_select(pp, n, C.byref(prm), int(mode), None, None, None, 0, C.byref(nv))
    i = np.empty(cnt, np.uint32)
    j = np.empty(cnt, np.uint32)
    lk = np.empty(cnt, np.uint8)
    lib().or_select(pp, n, C.byref(prm), int(mode), _ptr(i, C.c_uint32), _ptr(j, C.c_uint32),
                    _ptr(lk, C.c_uint8), cnt, C.byref(nv))
    return i, j, lk, int(nv.value)


def pgd(orig, recon, ai, aj, alink, **kw):
    """Run the PGD loop on the active set: (corrected f32, delta f64 (n,3), editable mask, stats)."""
    o, op = _f32(orig)
    r, rp = _f32(recon)
    n = o.shape[0]
    ai = np.ascontiguousarray(ai, np.uint32)
    aj = np.ascontiguousarray(aj, np.uint32)
    al = np.ascontiguousarray(alink, np.uint8)
    out = np.empty_like(o)
    delta = np.zeros((n, 3), np.float64)
    ed = np.zeros(n, np.int32)
    st = PgdStats()
    rc = lib().or_pgd(op, rp, n, C.byref(make_params(**kw)), _ptr(ai, C.c_uint32),
                      _ptr(aj, C.c_uint32), _ptr(al, C.c_uint8), len(ai), _ptr(out, C.c_float),
                      _ptr(delta, C.c_double), _ptr(ed, C.c_int32), C.byref(st))
    if rc != 0:
        raise ValueError("oracle: empty projection box (xi too small for float32 coordinates)")
    return out, delta, ed.astype(bool), st.as_dict()


def select_multi(P, b_list, mode=None, **kw):
    """Union of the active sets of several linking lengths (Sec. 1 and Sec. 5: a range of
    thresholds is supported by enforcing the union of their selected pairs).  Returns
    (ai, aj, alink, ab) in threshold order, then (i, j) order: alink is the link flag
    at the pair's own linking length ab."""
    out = [[], [], [], []]
    for b in b_list:
        ai, aj, al, _ = select(P, mode=mode, **dict(kw, b=b))
        out[0].append(ai)
        out[1].append(aj)
        out[2].append(al)
        out[3].append(np.full(len(ai), float(b)))
    return tuple(np.concatenate(x) for x in out)


def pgd_multi(orig, recon, ai, aj, alink, ab, **kw):
    """PGD on an active set whose pairs carry their own linking length ab (the union of
    several thresholds): (corrected f32, delta f64 (n,3), editable mask, stats)."""
    o, op = _f32(orig)
    r, rp = _f32(recon)
    n = o.shape[0]
    ai = np.ascontiguousarray(ai, np.uint32)
    aj = np.ascontiguousarray(aj, np.uint32)
    al = np.ascontiguousarray(alink, np.uint8)
    ab = np.ascontiguousarray(ab, np.float64)
    out = np.empty_like(o)
    delta = np.zeros((n, 3), np.float64)
    ed = np.zeros(n, np.int32)
    st = PgdStats()
    rc = lib().or_pgd_thr(op, rp, n, C.byref(make_params(**kw)), _ptr(ai, C.c_uint32), _ptr(aj, C.c_uint32),
                          _ptr(al, C.c_uint8), _ptr(ab, C.c_double), len(ai), _ptr(out, C.c_float),
                          _ptr(delta, C.c_double), _ptr(ed, C.c_int32), C.byref(st))
    if rc != 0:
        raise ValueError("oracle: empty projection box (xi too small for float32 coordinates)")
    return out, delta, ed.astype(bool), st.as_dict()


def encode(recon, corrected, **kw) -> bytes:
    r, rp = _f32(recon)
    c, cp = _f32(corrected)
    prm = make_params(**kw)
    size = lib().or_encode(rp, cp, r.shape[0], C.byref(prm), None, 0)
    buf = np.zeros(size, np.uint8)
    lib().or_encode(rp, cp, r.shape[0], C.byref(prm), _ptr(buf, C.c_uint8), size)
    return buf.tobytes()


def decode(recon, stream: bytes):
    r, rp = _f32(recon)
    b = np.frombuffer(stream, np.uint8).copy()
    out = np.empty_like(r)
    rc = lib().or_decode(rp, r.shape[0], _ptr(b, C.c_uint8), len(b), _ptr(out, C.c_float))
    if rc != 0:
        raise ValueError("oracle: malformed edit stream")
    return out


def correct(orig, recon, **kw):
    """Whole pass: (corrected, stats incl. n_vulnerable / n_active)."""
    o, op = _f32(orig)
    r, rp = _f32(recon)
    out = np.empty_like(o)
    st = PgdStats()
    nv = C.c_int64(0)
    na = C.c_int64(0)
    rc = lib().or_correct(op, rp, o.shape[0], C.byref(make_params(**kw)), _ptr(out, C.c_float),
                          C.byref(st), C.byref(nv), C.byref(na))
    if rc != 0:
        raise ValueError("oracle: empty projection box")
    d = st.as_dict()
    d["n_vulnerable"] = int(nv.value)
    d["n_active"] = int(na.value)
    return out, d


def count_flips(P, ai, aj, alink, **kw) -> int:
    p, pp = _f32(P)
    ai = np.ascontiguousarray(ai, np.uint32)
    aj = np.ascontiguousarray(aj, np.uint32)
    al = np.ascontiguousarray(alink, np.uint8)
    return int(lib().or_count_flips(pp, p.shape[0], C.byref(make_params(**kw)),
                                    _ptr(ai, C.c_uint32), _ptr(aj, C.c_uint32),
                                    _ptr(al, C.c_uint8), len(ai)))
