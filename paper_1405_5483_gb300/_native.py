"""ctypes declarations of the C ABI in include/mpm.h.

Loads paper_1405_5483_gb300/_build/libmpm.so and fails loudly when it is
missing: there is no other implementation to fall back to.
"""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmpm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "mpm.h")

(MPM_OK, MPM_EINVAL, MPM_ENOMEM, MPM_ECUDA, MPM_ECAPACITY, MPM_ETIMEOUT, MPM_ENOTSUP,
 MPM_ESCRATCH) = range(8)
NOALLOC_MAX_CANDIDATES = 1 << 21
NOALLOC_MAX_OCCURRENCES = 8192
MAP_AUTO, MAP_RANK, MAP_GREEDY, MAP_LOWBITS, MAP_QHASH = range(5)
TABLE_AUTO, TABLE_SMEM, TABLE_GLOBAL = range(3)
KERNEL_AUTO, KERNEL_GENERIC, KERNEL_SPECIALISED, KERNEL_SPLIT = range(4)


class Params(ctypes.Structure):
    _fields_ = [("q", ctypes.c_int), ("sigma_r", ctypes.c_int), ("k", ctypes.c_int),
                ("map_kind", ctypes.c_int), ("map_shift", ctypes.c_int),
                ("table_place", ctypes.c_int), ("smag", ctypes.c_int), ("chunk", ctypes.c_int),
                ("kernel", ctypes.c_int), ("overlap", ctypes.c_int), ("wide", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class TableInfo(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("mprime", ctypes.c_int), ("positions", ctypes.c_int),
                ("entry_bytes", ctypes.c_int), ("entries", ctypes.c_uint64),
                ("table_bytes", ctypes.c_uint64), ("est_candidate_rate", ctypes.c_double),
                ("entry_bits", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("sampled", ctypes.c_uint64),
                ("candidates", ctypes.c_uint64), ("z", ctypes.c_uint64),
                ("launches", ctypes.c_uint32), ("retries", ctypes.c_uint32),
                ("ms_scan", ctypes.c_float), ("ms_verify", ctypes.c_float),
                ("specialised", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class TuneOpts(ctypes.Structure):
    _fields_ = [("max_q", ctypes.c_int), ("max_k", ctypes.c_int), ("reps", ctypes.c_int),
                ("kernels", ctypes.c_int), ("max_sets", ctypes.c_int),
                ("max_rate", ctypes.c_double), ("max_positions", ctypes.c_int),
                ("grid", ctypes.c_int), ("max_table_kib", ctypes.c_int),
                ("overlap", ctypes.c_int), ("batch_generic", ctypes.c_int)]


MODEL_INPUTS, MODEL_HIDDEN, MODEL_PARAMS = 8, 64, 4801
BATCH_SMEM_TABLE_BYTES = 128 << 10


class TrainOpts(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("epochs", ctypes.c_int), ("batch", ctypes.c_int),
                ("seed", ctypes.c_uint64)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("params", Params), ("info", TableInfo), ("ms", ctypes.c_double),
                ("candidates", ctypes.c_uint64), ("z", ctypes.c_uint64),
                ("status", ctypes.c_int)]

    def as_dict(self):
        return {"params": self.params.as_dict(), "info": self.info.as_dict(), "ms": self.ms,
                "candidates": self.candidates, "z": self.z, "status": self.status}


class BatchOpts(ctypes.Structure):
    _fields_ = [("lane_bytes", ctypes.c_int), ("no_graph", ctypes.c_int),
                ("unit_kib", ctypes.c_int), ("generic", ctypes.c_int)]


class BatchStats(ctypes.Structure):
    _fields_ = [("bytes", ctypes.c_uint64), ("candidates", ctypes.c_uint64),
                ("z", ctypes.c_uint64), ("tiles", ctypes.c_uint32),
                ("launches", ctypes.c_uint32), ("ms", ctypes.c_float),
                ("scan_ms", ctypes.c_float), ("variants", ctypes.c_uint32),
                ("pad", ctypes.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class MpmError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s: %s (code %d)" % (what, _strerror(code), code))


_lib = None


def _strerror(code):
    try:
        return lib().mpm_strerror(code).decode()
    except Exception:
        return "error"


def lib():
    """The loaded libmpm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libmpm.so is not built (%s); run __graft_entry__.build() or "
                          "python -m paper_1405_5483_gb300.build_lib" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, sz, u8p = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p
    Pp, Ip, Sp = ctypes.POINTER(Params), ctypes.POINTER(TableInfo), ctypes.POINTER(Stats)
    szp = ctypes.POINTER(ctypes.c_size_t)
    fp = ctypes.POINTER(ctypes.c_float)
    sig = {
        "mpm_build": (vp, [u8p, sz, sz, ctypes.c_int, Pp]),
        "mpm_build_var": (vp, [u8p, ctypes.POINTER(ctypes.c_size_t), sz, ctypes.c_int, Pp]),
        "mpm_search": (ctypes.c_int, [vp, u8p, sz, vp, vp, szp]),
        "mpm_free": (None, [vp]),
        "mpm_last_error": (ctypes.c_int, []),
        "mpm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "mpm_set_stream": (ctypes.c_int, [vp, vp]),
        "mpm_get_params": (ctypes.c_int, [vp, Pp, Ip]),
        "mpm_get_stats": (ctypes.c_int, [vp, Sp]),
        "mpm_set_timing": (ctypes.c_int, [vp, ctypes.c_int]),
        "mpm_plan": (ctypes.c_int, [u8p, sz, sz, ctypes.c_int, Pp, Pp, Ip]),
        "mpm_host_tables": (ctypes.c_int, [u8p, sz, sz, ctypes.c_int, Pp, vp, vp, sz]),
        "mpm_encode": (ctypes.c_int, [vp, u8p, sz, vp]),
        "mpm_scan": (ctypes.c_int, [vp, u8p, sz, vp, szp]),
        "mpm_search_noalloc": (ctypes.c_int, [vp, u8p, sz, vp, vp, szp]),
        "mpm_search_async": (ctypes.c_int, [vp, u8p, sz, vp, vp, sz, vp]),
        "mpm_sync": (ctypes.c_int, [vp]),
        "mpm_join": (ctypes.c_int, [vp]),
        "mpm_test_inject": (ctypes.c_int, [ctypes.c_int]),
        "mpm_reset_stats": (ctypes.c_int, [vp]),
        "mpm_batch_create": (vp, [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp),
                                  ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_uint32),
                                  ctypes.c_int, ctypes.POINTER(BatchOpts)]),
        "mpm_batch_run": (ctypes.c_int, [vp, vp, vp, vp, szp]),
        "mpm_batch_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(BatchStats)]),
        "mpm_batch_free": (None, [vp]),
        "mpm_search_batch": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp),
                                            ctypes.POINTER(ctypes.c_size_t),
                                            ctypes.POINTER(ctypes.c_uint32), ctypes.c_int,
                                            vp, vp, vp, szp]),
        "mpm_jit_compile": (ctypes.c_int, [u8p, sz, sz, ctypes.c_int, Pp, ctypes.c_char_p, sz]),
        "mpm_batch_jit_compile": (ctypes.c_int, [ctypes.POINTER(vp), szp, szp,
                                                 ctypes.POINTER(ctypes.c_int), Pp, ctypes.c_int,
                                                 ctypes.c_char_p, sz]),
        "mpm_autotune": (ctypes.c_int, [u8p, sz, sz, ctypes.c_int, u8p, sz,
                                        ctypes.POINTER(TuneOpts), Pp, ctypes.POINTER(TuneEntry),
                                        sz, szp]),
        "mpm_model_create": (vp, [ctypes.c_uint64]),
        "mpm_model_free": (None, [vp]),
        "mpm_model_set_norm": (ctypes.c_int, [vp, fp, fp, ctypes.c_float, ctypes.c_float]),
        "mpm_model_get_norm": (ctypes.c_int, [vp, fp, fp, fp, fp]),
        "mpm_model_get_params": (ctypes.c_int, [vp, fp]),
        "mpm_model_set_params": (ctypes.c_int, [vp, fp]),
        "mpm_model_predict": (ctypes.c_int, [vp, vp, sz, vp]),
        "mpm_model_loss_grad": (ctypes.c_int, [vp, vp, vp, sz, fp, fp]),
        "mpm_model_adam_step": (ctypes.c_int, [vp, fp, ctypes.POINTER(TrainOpts)]),
        "mpm_model_train": (ctypes.c_int, [vp, vp, vp, sz, ctypes.POINTER(TrainOpts), fp]),
        "mpm_model_save": (ctypes.c_int, [vp, ctypes.c_char_p]),
        "mpm_model_load": (vp, [ctypes.c_char_p]),
        "mpm_model_grid": (ctypes.c_int, [u8p, sz, sz, ctypes.c_int, ctypes.c_int, Pp, Ip, sz,
                                          szp]),
        "mpm_model_features": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, sz, sz, sz, Pp, sz,
                                              fp]),
        "mpm_model_choose": (ctypes.c_int, [vp, u8p, sz, sz, ctypes.c_int, ctypes.c_double, sz,
                                            sz, Pp, fp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def declared_functions():
    """Names of the functions include/mpm.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mpm_[a-z_0-9]+)\s*\(", text)))
