"""ctypes wrapper of the C oracle (naive r x n and Aho-Corasick) -- TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check and bench.py's CPU-baseline leg may use this.
The shared object is compiled from ``mpm_oracle.c`` with the host C compiler;
it shares nothing with the CUDA library.

Both searches return the occurrence list of the problem statement (Section 1):
every (i, p) with T[i..i+m) == P_p, sorted by position then pattern id.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force=False):
    """Compiles the C oracle into oracle/_build/liboracle.so (gcc, -O2)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                           _SRC, "-o", tmp])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_SO)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_naive.restype = ctypes.c_int64
    lib.oracle_naive.argtypes = [u8p, ctypes.c_uint64, u8p, ctypes.c_uint64, ctypes.c_uint64,
                                 u32p, u32p, ctypes.c_uint64]
    lib.oracle_ac_build.restype = ctypes.c_void_p
    lib.oracle_ac_build.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64]
    lib.oracle_ac_build_var.restype = ctypes.c_void_p
    lib.oracle_ac_build_var.argtypes = [u8p, ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint64]
    lib.oracle_ac_search.restype = ctypes.c_int64
    lib.oracle_ac_search.argtypes = [ctypes.c_void_p, u8p, ctypes.c_uint64, ctypes.c_int,
                                     u32p, u32p, ctypes.c_uint64]
    lib.oracle_ac_free.restype = None
    lib.oracle_ac_free.argtypes = [ctypes.c_void_p]
    lib.oracle_ac_nodes.restype = ctypes.c_int64
    lib.oracle_ac_nodes.argtypes = [ctypes.c_void_p]
    _lib = lib
    return lib


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _u32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _as_text(T):
    return np.ascontiguousarray(np.frombuffer(bytes(T), np.uint8) if isinstance(T, (bytes, bytearray))
                                else np.asarray(T, dtype=np.uint8).ravel())


def _as_patterns(P):
    if isinstance(P, (list, tuple)):
        if len(P) == 0:
            return np.zeros((0, 0), np.uint8)
        P = np.stack([np.frombuffer(bytes(p), np.uint8) for p in P])
    P = np.ascontiguousarray(np.asarray(P, dtype=np.uint8))
    assert P.ndim == 2, "patterns: an (r, m) uint8 array (all of length m)"
    return P


def naive(T, P, cap=None):
    """All occurrences by direct r x n comparison; returns (pos, pid) uint32 arrays."""
    lib = _load()
    T, P = _as_text(T), _as_patterns(P)
    r, m = P.shape
    if r == 0 or m == 0:
        return np.zeros(0, np.uint32), np.zeros(0, np.uint32)
    cap = 1024 if cap is None else cap
    while True:
        pos = np.zeros(max(cap, 1), np.uint32)
        pid = np.zeros(max(cap, 1), np.uint32)
        z = lib.oracle_naive(_u8(T), T.size, _u8(P), r, m, _u32(pos), _u32(pid), cap)
        if z <= cap:
            return pos[:z].copy(), pid[:z].copy()
        cap = int(z)


def _variable(P):
    """A list of patterns of different lengths -> (concatenation, offsets)."""
    rows = [np.frombuffer(bytes(p), np.uint8) for p in P]
    off = np.zeros(len(rows) + 1, np.uint64)
    off[1:] = np.cumsum([r.size for r in rows])
    cat = np.concatenate(rows) if rows else np.zeros(0, np.uint8)
    return np.ascontiguousarray(cat), off


class AhoCorasick:
    """Textbook Aho-Corasick automaton over bytes (Section 1.1); P is an
    (r, m) array or a list of patterns, which may differ in length."""

    def __init__(self, P):
        self._lib = _load()
        self.variable = (isinstance(P, (list, tuple)) and
                         len(set(len(bytes(p)) for p in P)) > 1)
        if self.variable:
            self.cat, self.off = _variable(P)
            self.r = len(P)
            self.m = int(min(self.off[1:] - self.off[:-1]))
            self._h = self._lib.oracle_ac_build_var(
                _u8(self.cat), self.off.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), self.r)
        else:
            self.P = _as_patterns(P)
            self.r, self.m = self.P.shape
            self._h = self._lib.oracle_ac_build(_u8(self.P), self.r, self.m)
        if not self._h:
            raise MemoryError("oracle_ac_build failed")

    @property
    def nodes(self):
        return int(self._lib.oracle_ac_nodes(self._h))

    def search(self, T, threads=1, cap=None):
        T = _as_text(T)
        if self.r == 0 or self.m == 0:
            return np.zeros(0, np.uint32), np.zeros(0, np.uint32)
        cap = 1 << 16 if cap is None else cap
        while True:
            pos = np.zeros(max(cap, 1), np.uint32)
            pid = np.zeros(max(cap, 1), np.uint32)
            z = self._lib.oracle_ac_search(self._h, _u8(T), T.size, int(threads),
                                           _u32(pos), _u32(pid), cap)
            if z < 0:
                raise MemoryError("oracle_ac_search failed")
            if z <= cap:
                pos, pid = pos[:z].copy(), pid[:z].copy()
                if self.variable:  # reported in order of end position
                    order = np.lexsort((pid, pos))
                    pos, pid = pos[order], pid[order]
                return pos, pid
            cap = int(z)

    def close(self):
        if self._h:
            self._lib.oracle_ac_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def aho_corasick(T, P, threads=1):
    """All occurrences via Aho-Corasick; returns (pos, pid) uint32 arrays."""
    ac = AhoCorasick(P)
    try:
        return ac.search(T, threads=threads)
    finally:
        ac.close()
