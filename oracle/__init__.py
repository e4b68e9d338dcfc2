"""FP64 CPU oracle for the per-track Kalman step (p2z / p2r), paper section 2.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports, links or calls it.

The arithmetic lives in ``kf_oracle.c`` (plain C, double precision); this
module compiles it with gcc into ``oracle/_build/liboracle.so`` and marshals
numpy arrays in and out with ctypes.  Array layouts here are the oracle's own:
array-of-structures, one row per track, float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kf_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

NO_INTERSECT = 1
S_NOT_PD = 2
BAD_K = 4
NONFINITE = 8

FORM_STANDARD = 0
FORM_JOSEPH = 1

P2Z = 0
P2R = 1

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (x86_64 here, aarch64 on the GPU host)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    hdr = os.path.join(_HERE, "kf_oracle.h")
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(hdr))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        i8p = ctypes.POINTER(ctypes.c_int8)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.kfo_propagate_to_z.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]
        lib.kfo_propagate_to_z.restype = ctypes.c_uint
        lib.kfo_propagate_to_r.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]
        lib.kfo_propagate_to_r.restype = ctypes.c_uint
        lib.kfo_path_to_z.argtypes = [dp, ctypes.c_double, dp]
        lib.kfo_path_to_z.restype = ctypes.c_int
        lib.kfo_path_to_r.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
        lib.kfo_path_to_r.restype = ctypes.c_int
        lib.kfo_helix_at.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
        lib.kfo_helix_at.restype = None
        lib.kfo_kalman_update.argtypes = [dp, dp, dp, dp, dp, ctypes.c_int, dp, dp, dp]
        lib.kfo_kalman_update.restype = ctypes.c_uint
        for name in ("kfo_p2z_step", "kfo_p2r_step"):
            fn = getattr(lib, name)
            fn.argtypes = [dp, dp, ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double,
                           ctypes.c_int, dp, dp, dp]
            fn.restype = ctypes.c_uint
        lib.kfo_step_batch.argtypes = [ctypes.c_int, ctypes.c_int64, dp, dp, i8p, dp, dp, dp,
                                       ctypes.c_double, ctypes.c_int, dp, dp, u8p, dp]
        lib.kfo_step_batch.restype = None
        lib.kfo_chain_batch.argtypes = [ctypes.c_int64, ctypes.c_int, ip, dp, dp, dp, i8p, dp, dp,
                                        ctypes.c_double, ctypes.c_int, u8p]
        lib.kfo_chain_batch.restype = None
        _lib = lib
        return lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None) -> np.ndarray:
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        out = out.reshape(shape)
    return out


# ----------------------------------------------------------- single tracks

def propagate_to_z(p, q: int, bz: float, zt: float):
    """Returns (p', J, status) for one track propagated to the plane z = zt."""
    lib = _load()
    p = _f64(p, (6,))
    out = np.zeros(6)
    J = np.zeros((6, 6))
    st = lib.kfo_propagate_to_z(_dptr(p), int(q), float(bz), float(zt), _dptr(out), _dptr(J))
    return out, J, int(st)


def propagate_to_r(p, q: int, bz: float, R: float):
    """Returns (p', J, status) for one track propagated to the cylinder r = R."""
    lib = _load()
    p = _f64(p, (6,))
    out = np.zeros(6)
    J = np.zeros((6, 6))
    st = lib.kfo_propagate_to_r(_dptr(p), int(q), float(bz), float(R), _dptr(out), _dptr(J))
    return out, J, int(st)


def path_to_z(p, zt: float):
    lib = _load()
    p = _f64(p, (6,))
    s = np.zeros(1)
    ok = lib.kfo_path_to_z(_dptr(p), float(zt), _dptr(s))
    return float(s[0]) if ok else None


def path_to_r(p, q: int, bz: float, R: float):
    lib = _load()
    p = _f64(p, (6,))
    s = np.zeros(1)
    ok = lib.kfo_path_to_r(_dptr(p), int(q), float(bz), float(R), _dptr(s))
    return float(s[0]) if ok else None


def helix_at(p, q: int, bz: float, s: float) -> np.ndarray:
    lib = _load()
    p = _f64(p, (6,))
    out = np.zeros(6)
    lib.kfo_helix_at(_dptr(p), int(q), float(bz), float(s), _dptr(out))
    return out


def kalman_update(p, C21, H, V3, r, form: int = FORM_STANDARD):
    """Generic 2-row update. Returns (p'', C''21, chi2, status)."""
    lib = _load()
    p = _f64(p, (6,))
    C21 = _f64(C21, (21,))
    H = _f64(H, (12,))
    V3 = _f64(V3, (3,))
    r = _f64(r, (2,))
    pout = np.zeros(6)
    cout = np.zeros(21)
    chi2 = np.zeros(1)
    st = lib.kfo_kalman_update(_dptr(p), _dptr(C21), _dptr(H), _dptr(V3), _dptr(r), int(form),
                               _dptr(pout), _dptr(cout), _dptr(chi2))
    return pout, cout, float(chi2[0]), int(st)


def step(kind: int, p, C21, q: int, hit, hitcov, bz: float, surf: float,
         form: int = FORM_STANDARD):
    """One p2z (kind 0) or p2r (kind 1) step. Returns (p'', C''21, chi2, status)."""
    lib = _load()
    p = _f64(p, (6,))
    C21 = _f64(C21, (21,))
    hit = _f64(hit, (3,))
    hitcov = _f64(hitcov, (6,))
    pout = np.zeros(6)
    cout = np.zeros(21)
    chi2 = np.zeros(1)
    fn = lib.kfo_p2z_step if kind == P2Z else lib.kfo_p2r_step
    st = fn(_dptr(p), _dptr(C21), int(q), _dptr(hit), _dptr(hitcov), float(bz), float(surf),
            int(form), _dptr(pout), _dptr(cout), _dptr(chi2))
    return pout, cout, float(chi2[0]), int(st)


# ------------------------------------------------------------------ batches

def step_batch(kind: int, state, cov, charge, hit, hitcov, surf, bz: float,
               form: int = FORM_STANDARD, threads: int = 1):
    """Batched step over n tracks (AoS float64 arrays, one row per track).

    state [n,6], cov [n,21], charge [n] int8, hit [n,3], hitcov [n,6],
    surf: scalar or [n].  Returns (state_out, cov_out, status, chi2).
    ``threads`` > 1 splits the tracks into contiguous chunks run concurrently
    (ctypes releases the GIL during the call).
    """
    lib = _load()
    state = _f64(state)
    n = state.shape[0]
    cov = _f64(cov, (n, 21))
    hit = _f64(hit, (n, 3))
    hitcov = _f64(hitcov, (n, 6))
    charge = np.ascontiguousarray(np.asarray(charge, dtype=np.int8).reshape(n))
    surf = np.ascontiguousarray(np.broadcast_to(np.asarray(surf, dtype=np.float64), (n,)))
    s_out = np.empty((n, 6))
    c_out = np.empty((n, 21))
    status = np.empty(n, dtype=np.uint8)
    chi2 = np.empty(n)

    def run(lo: int, hi: int):
        m = hi - lo
        if m <= 0:
            return
        lib.kfo_step_batch(int(kind), m, _dptr(state[lo:hi]), _dptr(cov[lo:hi]),
                           charge[lo:hi].ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                           _dptr(hit[lo:hi]), _dptr(hitcov[lo:hi]), _dptr(surf[lo:hi]),
                           float(bz), int(form), _dptr(s_out[lo:hi]), _dptr(c_out[lo:hi]),
                           status[lo:hi].ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                           _dptr(chi2[lo:hi]))

    threads = max(1, int(threads))
    if threads == 1 or n < 2 * threads:
        run(0, n)
    else:
        bounds = np.linspace(0, n, threads + 1).astype(np.int64)
        ts = [threading.Thread(target=run, args=(int(bounds[t]), int(bounds[t + 1])))
              for t in range(threads)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
    return s_out, c_out, status, chi2


def chain_batch(kinds, pos, state, cov, charge, hit, hitcov, bz: float,
                form: int = FORM_STANDARD, threads: int = 1):
    """Multi-layer chain over n tracks.  hit [L,n,3], hitcov [L,n,6].

    Returns (state_out [n,6], cov_out [n,21], status [n])."""
    lib = _load()
    kinds = np.ascontiguousarray(np.asarray(kinds, dtype=np.int32))
    L = kinds.shape[0]
    pos = _f64(pos, (L,))
    state = _f64(state).copy()
    n = state.shape[0]
    cov = _f64(cov, (n, 21)).copy()
    hit = _f64(hit, (L, n, 3))
    hitcov = _f64(hitcov, (L, n, 6))
    charge = np.ascontiguousarray(np.asarray(charge, dtype=np.int8).reshape(n))
    status = np.zeros(n, dtype=np.uint8)

    def run(lo: int, hi: int):
        m = hi - lo
        if m <= 0:
            return
        h = np.ascontiguousarray(hit[:, lo:hi])
        hc = np.ascontiguousarray(hitcov[:, lo:hi])
        st_chunk = np.ascontiguousarray(state[lo:hi])
        cv_chunk = np.ascontiguousarray(cov[lo:hi])
        stat = np.zeros(m, dtype=np.uint8)
        lib.kfo_chain_batch(m, L, kinds.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(pos),
                            _dptr(st_chunk), _dptr(cv_chunk),
                            charge[lo:hi].ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                            _dptr(h), _dptr(hc), float(bz), int(form),
                            stat.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
        state[lo:hi] = st_chunk
        cov[lo:hi] = cv_chunk
        status[lo:hi] = stat

    threads = max(1, int(threads))
    if threads == 1 or n < 2 * threads:
        run(0, n)
    else:
        bounds = np.linspace(0, n, threads + 1).astype(np.int64)
        ts = [threading.Thread(target=run, args=(int(bounds[t]), int(bounds[t + 1])))
              for t in range(threads)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
    return state, cov, status
