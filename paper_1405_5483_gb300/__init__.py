"""Exact multiple pattern matching on GB300: MAG / SMAG (arXiv 1405.5483).

A thin Python binding of the C ABI in include/mpm.h: every step of a search
runs in the library's CUDA kernels; this module only marshals arguments.
PyTorch supplies device memory and the current CUDA stream.

    import paper_1405_5483_gb300 as mpm
    m = mpm.Matcher(P, sigma=20)          # P: uint8 (r, m), host memory
    pos, pid = m.search(T)                # T: uint8 CUDA tensor (or numpy)
"""
import ctypes

import numpy as np

from ._native import (KERNEL_AUTO, KERNEL_GENERIC, KERNEL_SPECIALISED, KERNEL_SPLIT,  # noqa: F401,E501
                      MAP_AUTO, MAP_GREEDY, MAP_LOWBITS, MAP_QHASH, MAP_RANK, MPM_ECAPACITY, MPM_EINVAL,
                      MPM_ENOTSUP, MPM_OK, TABLE_AUTO, TABLE_GLOBAL, TABLE_SMEM, MpmError,
                      Params, Stats, TableInfo, declared_functions, lib)

__all__ = ["Matcher", "Batch", "plan", "host_tables", "autotune", "jit_compile",
           "batch_jit_compile", "MpmError", "lib", "declared_functions"]


def _torch():
    import torch
    return torch


def make_params(q=0, sigma_r=0, k=0, map_kind=MAP_AUTO, map_shift=-1, table_place=TABLE_AUTO,
                smag=0, chunk=0, kernel=KERNEL_AUTO, overlap=0, wide=0):
    return Params(q, sigma_r, k, map_kind, map_shift, table_place, smag, chunk, kernel,
                  overlap, wide)


def jit_compile(P, sigma, **kw):
    """Host-only: compiles the specialised scan for these parameters;
    returns (code, compiler log)."""
    P = _patterns(P)
    buf = ctypes.create_string_buffer(1 << 16)
    rc = lib().mpm_jit_compile(P.ctypes.data, P.shape[0], P.shape[1], sigma,
                               ctypes.byref(make_params(**kw)), buf, len(buf))
    return rc, buf.value.decode(errors="replace")


def batch_jit_compile(sets, sigmas, params=None):
    """Host-only: compiles the batched kernel that a Batch of these pattern
    sets (uint8 (r, m) arrays) with these parameters (dicts, or None for
    automatic) would run; returns (code, compiler log)."""
    sets = [_patterns(P) for P in sets]
    n = len(sets)
    ptrs = (ctypes.c_void_p * n)(*[P.ctypes.data for P in sets])
    rs = (ctypes.c_size_t * n)(*[P.shape[0] for P in sets])
    ms = (ctypes.c_size_t * n)(*[P.shape[1] for P in sets])
    sg = (ctypes.c_int * n)(*sigmas)
    ps = (Params * n)(*[make_params(**(params[i] if params else {})) for i in range(n)])
    buf = ctypes.create_string_buffer(1 << 16)
    rc = lib().mpm_batch_jit_compile(ptrs, rs, ms, sg, ps, n, buf, len(buf))
    return rc, buf.value.decode(errors="replace")


def _patterns(P):
    if isinstance(P, (list, tuple)):
        P = np.stack([np.frombuffer(bytes(p), np.uint8) for p in P])
    if hasattr(P, "detach"):
        P = P.detach().cpu().numpy()
    P = np.ascontiguousarray(np.asarray(P, dtype=np.uint8))
    if P.ndim != 2:
        raise ValueError("patterns must be an (r, m) uint8 array")
    return P


def plan(P, sigma, **kw):
    """Parameters mpm_build would choose, and the sizes that follow (host only)."""
    P = _patterns(P)
    out, info = Params(), TableInfo()
    rc = lib().mpm_plan(P.ctypes.data, P.shape[0], P.shape[1], sigma,
                        ctypes.byref(make_params(**kw)), ctypes.byref(out), ctypes.byref(info))
    if rc:
        raise MpmError(rc, "mpm_plan")
    return out.as_dict(), info.as_dict()


def host_tables(P, sigma, **kw):
    """(mu uint8[256], mask table uint8[table_bytes], info) built on the host."""
    P = _patterns(P)
    params, info = plan(P, sigma, **kw)
    mu = np.zeros(256, np.uint8)
    table = np.zeros(int(info["table_bytes"]), np.uint8)
    rc = lib().mpm_host_tables(P.ctypes.data, P.shape[0], P.shape[1], sigma,
                               ctypes.byref(make_params(**kw)), mu.ctypes.data,
                               table.ctypes.data, table.size)
    if rc:
        raise MpmError(rc, "mpm_host_tables")
    return mu, table, dict(info, **params)


def autotune(P, sigma, T, max_q=0, max_k=0, reps=0, kernels=0, max_sets=0, max_rate=0.0,
             max_positions=0, grid=0, max_table_kib=0, overlap=0, batch_generic=0):
    """Exhaustive parameter search timed on the sample text T (CUDA tensor or
    numpy).  grid=1 times every point of the cost model's grid; overlap=1
    also times overlapping-q-gram filters (2: only those); batch_generic=1
    times the precompiled batched kernel for kernels bit 3.  Returns
    (best params dict, list of timed sets)."""
    from ._native import TuneEntry, TuneOpts
    P = _patterns(P)
    opts = TuneOpts(max_q, max_k, reps, kernels, max_sets, max_rate, max_positions, grid,
                    max_table_kib, overlap, batch_generic)
    cap = 4096
    entries = (TuneEntry * cap)()
    best = Params()
    count = ctypes.c_size_t(0)
    if hasattr(T, "is_cuda") and T.is_cuda:
        tp, tn = T.data_ptr(), T.numel()
    else:
        T = np.ascontiguousarray(np.asarray(T, dtype=np.uint8))
        tp, tn = T.ctypes.data, T.size
    rc = lib().mpm_autotune(P.ctypes.data, P.shape[0], P.shape[1], sigma, tp, tn,
                            ctypes.byref(opts), ctypes.byref(best), entries, cap,
                            ctypes.byref(count))
    if rc:
        raise MpmError(rc, "mpm_autotune")
    out = [entries[i].as_dict() for i in range(min(count.value, cap))]
    return best.as_dict(), out


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def _numel(x):
    return x.numel() if hasattr(x, "numel") else x.size


class Matcher:
    """A built pattern set (mpm_build) and searches over texts (mpm_search)."""

    def __init__(self, P, sigma=256, **params):
        """P: an (r, m) uint8 array, or a list of byte strings, which may
        differ in length (mpm_build_var; m is then the shortest)."""
        self.sigma = sigma
        rows = None
        if isinstance(P, (list, tuple)):
            rows = [bytes(p) for p in P]
            if len(set(len(x) for x in rows)) <= 1:
                rows = None
        if rows is None:
            P = _patterns(P)
            self.r, self.m = P.shape
            self._h = lib().mpm_build(P.ctypes.data, self.r, self.m, sigma,
                                      ctypes.byref(make_params(**params)))
        else:
            cat = np.frombuffer(b"".join(rows), np.uint8)
            off = (ctypes.c_size_t * (len(rows) + 1))()
            at = 0
            for i, x in enumerate(rows):
                off[i] = at
                at += len(x)
            off[len(rows)] = at
            self.r, self.m = len(rows), min(len(x) for x in rows)
            self._h = lib().mpm_build_var(cat.ctypes.data, off, self.r, sigma,
                                          ctypes.byref(make_params(**params)))
        if not self._h:
            raise MpmError(lib().mpm_last_error(), "mpm_build")
        self._cap = max(1024, 4 * self.r)

    # -------------------------------------------------------------- info
    @property
    def params(self):
        p, i = Params(), TableInfo()
        self._check(lib().mpm_get_params(self._h, ctypes.byref(p), ctypes.byref(i)), "params")
        return p.as_dict()

    @property
    def info(self):
        p, i = Params(), TableInfo()
        self._check(lib().mpm_get_params(self._h, ctypes.byref(p), ctypes.byref(i)), "params")
        return i.as_dict()

    @property
    def stats(self):
        s = Stats()
        self._check(lib().mpm_get_stats(self._h, ctypes.byref(s)), "stats")
        return s.as_dict()

    def set_timing(self, on=True):
        """Device times of the scan and verification kernels in .stats."""
        self._check(lib().mpm_set_timing(self._h, 1 if on else 0), "mpm_set_timing")

    def _check(self, rc, what):
        if rc:
            raise MpmError(rc, what)

    def _stream(self, T):
        # the current PyTorch stream for device texts, the default stream
        # otherwise; the library is told only when it changes
        if getattr(T, "is_cuda", False):
            cur = _torch().cuda.current_stream().cuda_stream
        else:
            cur = None
        if cur != getattr(self, "_cur_stream", 0):
            lib().mpm_set_stream(self._h, ctypes.c_void_p(cur) if cur else None)
            self._cur_stream = cur

    # ------------------------------------------------------------ search
    def search_into(self, T, out_pos, out_pid):
        """Writes the sorted occurrences into out_pos/out_pid (device or host,
        32-bit); returns z.  Raises MpmError(MPM_ECAPACITY) with .z set when
        they are too small."""
        self._stream(T)
        z = ctypes.c_size_t(min(_numel(out_pos), _numel(out_pid)))
        rc = lib().mpm_search(self._h, _ptr(T), _numel(T), _ptr(out_pos), _ptr(out_pid),
                              ctypes.byref(z))
        if rc:
            e = MpmError(rc, "mpm_search")
            e.z = z.value
            raise e
        return z.value

    def search_async(self, T, out_pos, out_pid, status):
        """Enqueues the search of device text T on the current stream without
        waiting (mpm_search_async); status is a 4-entry int32 CUDA tensor (or
        mapped host memory) that receives [candidates, z, error, complete]."""
        self._stream(T)
        rc = lib().mpm_search_async(self._h, _ptr(T), _numel(T), _ptr(out_pos), _ptr(out_pid),
                                    min(_numel(out_pos), _numel(out_pid)), _ptr(status))
        if rc:
            raise MpmError(rc, "mpm_search_async")

    def join(self):
        """Orders later work on the handle's stream after the pipelined
        searches so far (mpm_join)."""
        self._check(lib().mpm_join(self._h), "mpm_join")

    def sync(self):
        """Waits for the handle's stream and the pipelined searches (mpm_sync)."""
        self._check(lib().mpm_sync(self._h), "mpm_sync")

    def reset_stats(self):
        self._check(lib().mpm_reset_stats(self._h), "mpm_reset_stats")

    def search(self, T):
        """All occurrences in T as (pos, pid), 32-bit, sorted by (pos, pid).
        CUDA tensor in -> int32 CUDA tensors out (values are unsigned);
        numpy in -> uint32 numpy out."""
        on_dev = hasattr(T, "is_cuda") and T.is_cuda
        while True:
            if on_dev:
                torch = _torch()
                pos = torch.empty(self._cap, dtype=torch.int32, device=T.device)
                pid = torch.empty(self._cap, dtype=torch.int32, device=T.device)
            else:
                T = np.ascontiguousarray(np.asarray(T, dtype=np.uint8))
                pos = np.empty(self._cap, np.uint32)
                pid = np.empty(self._cap, np.uint32)
            try:
                z = self.search_into(T, pos, pid)
            except MpmError as e:
                if e.code == MPM_ECAPACITY:
                    self._cap = int(e.z) + 1024
                    continue
                raise
            return pos[:z], pid[:z]

    def scan(self, T, cap=None):
        """The filter alone: candidate records ((fired << 32) | h) as an int64
        CUDA tensor, in no particular order."""
        torch = _torch()
        cap = cap or max(1 << 16, _numel(T) // 16)
        while True:
            cand = torch.empty(cap, dtype=torch.int64, device=T.device)
            self._stream(T)
            cnt = ctypes.c_size_t(cap)
            rc = lib().mpm_scan(self._h, _ptr(T), _numel(T), _ptr(cand), ctypes.byref(cnt))
            if rc == MPM_ECAPACITY:
                cap = int(cnt.value) + 1024
                continue
            self._check(rc, "mpm_scan")
            return cand[:cnt.value]

    def encode(self, T):
        """SMAG encoding: the code of every non-overlapping q-gram of T."""
        torch = _torch()
        q = self.params["q"]
        codes = torch.empty(max(1, _numel(T) // q), dtype=torch.int32, device=T.device)
        self._stream(T)
        self._check(lib().mpm_encode(self._h, _ptr(T), _numel(T), _ptr(codes)), "mpm_encode")
        return codes[: _numel(T) // q]

    def close(self):
        if getattr(self, "_h", None):
            lib().mpm_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many texts (CUDA uint8 tensors), each against one of several Matchers,
    in one persistent launch replayed from a CUDA graph (mpm_batch_*)."""

    def __init__(self, matchers, texts, set_of_text, lane_bytes=0, graph=True, unit_kib=0,
                 generic=False):
        """generic=True: the precompiled batched kernel instead of the one
        compiled for the batch's parameter sets."""
        from ._native import BatchOpts
        self._keep = (list(matchers), list(texts))
        n = len(texts)
        hs = (ctypes.c_void_p * len(matchers))(*[m._h for m in matchers])
        tp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in texts])
        ln = (ctypes.c_size_t * n)(*[t.numel() for t in texts])
        st = (ctypes.c_uint32 * n)(*[int(s) for s in set_of_text])
        opts = BatchOpts(lane_bytes, 0 if graph else 1, unit_kib, 1 if generic else 0)
        self._b = lib().mpm_batch_create(hs, len(matchers), tp, ln, st, n, ctypes.byref(opts))
        if not self._b:
            raise MpmError(lib().mpm_last_error(), "mpm_batch_create")
        self._cap = 1 << 16

    def run(self):
        """(text index, position, pattern id) as int32 CUDA tensors, sorted."""
        torch = _torch()
        dev = self._keep[1][0].device
        while True:
            out = torch.empty(3 * self._cap, dtype=torch.int32, device=dev)
            z = ctypes.c_size_t(self._cap)
            rc = lib().mpm_batch_run(self._b, out[: self._cap].data_ptr(),
                                     out[self._cap: 2 * self._cap].data_ptr(),
                                     out[2 * self._cap:].data_ptr(), ctypes.byref(z))
            if rc == MPM_ECAPACITY:
                self._cap = int(z.value) + 1024
                continue
            if rc:
                raise MpmError(rc, "mpm_batch_run")
            zz = z.value
            return out[:zz], out[self._cap: self._cap + zz], out[2 * self._cap: 2 * self._cap + zz]

    @property
    def stats(self):
        from ._native import BatchStats
        s = BatchStats()
        if lib().mpm_batch_get_stats(self._b, ctypes.byref(s)):
            raise MpmError(lib().mpm_last_error(), "mpm_batch_get_stats")
        return s.as_dict()

    def close(self):
        if getattr(self, "_b", None):
            lib().mpm_batch_free(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

