"""The learned cost model: an MLP that predicts the batched scan's time for a
pattern set and a parameter set, so parameters can be proposed per set
without timing them.  The paper fixes q from log_sigma(rm) and k by a closed
form (Section 3.2); the model is not in the paper.  Its forward, gradient and
Adam kernels are the library's (mpm_model_*); this module holds the Python
side: features, the timing database, training and regret.

Features of one (pattern set, parameter set) pair, as mpm_model_features
computes them: [sigma, entropy of the text in bits, log2 m, log10 r, log2 n,
q, log2 sigma', k]; the target is ln(ms) of the batched kernel (the one
compiled for the set's parameters, as a batch runs it) over the set's
text of n bytes, measured with the whole GPU busy (the text repeated until at
least 128 MiB are scanned; the time divided by the copies).  The grid
(mpm_model_grid) is q in 2..6 with sigma' in {2, 4, 8, 16} and q in 2..5
with q-gram hashing into 2^12, 2^14 or 2^16 bins, every feasible k <= 8, at
most 32 filter positions (the batched kernel's limit).

Command line (run where a GPU is):
  python -m paper_1405_5483_gb300.cost_model collect OUT.npz --first 0 --count 400
  python -m paper_1405_5483_gb300.cost_model train DB.npz MODEL.bin
  python -m paper_1405_5483_gb300.cost_model evaluate DB.npz MODEL.bin
"""
import argparse
import ctypes
import json
import math
import os
import time

import numpy as np

from . import _native
from ._native import MpmError, Params, TableInfo, TrainOpts, lib

N_IN = _native.MODEL_INPUTS
N_PARAMS = _native.MODEL_PARAMS
FEATURES = ("sigma", "entropy", "log2_m", "log10_r", "log2_n", "q", "log2_sigma_r", "k")
DATA_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
DB_PATH = os.path.join(DATA_DIR, "cost_timings.npz")
MODEL_PATH = os.path.join(DATA_DIR, "cost_model.bin")
TRAIN_SETS = range(0, 200)      # pattern sets whose timings train the model
HELDOUT_SETS = range(200, 400)  # pattern sets it is evaluated on


def _check(rc, what):
    if rc:
        raise MpmError(rc, what)


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _f32(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if shape is not None:
        a = a.reshape(shape)
    return a


def entropy_bits(T):
    """Symbol entropy (bits) of a byte text (numpy array or tensor)."""
    if hasattr(T, "is_cuda"):
        import torch
        h = torch.bincount(T.reshape(-1).to(torch.int64), minlength=256).double().cpu().numpy()
    else:
        h = np.bincount(np.asarray(T, np.uint8).reshape(-1), minlength=256).astype(np.float64)
    p = h[h > 0] / h.sum()
    return float(-(p * np.log2(p)).sum())


def grid(P, sigma, max_positions=32):
    """The model's feasible grid for pattern set P: list of (params, info) dicts."""
    P = np.ascontiguousarray(np.asarray(P, dtype=np.uint8))
    r, m = P.shape
    L = lib()
    count = ctypes.c_size_t(0)
    _check(L.mpm_model_grid(P.ctypes.data, r, m, sigma, max_positions, None, None, 0,
                            ctypes.byref(count)), "mpm_model_grid")
    n = count.value
    ps, infos = (Params * max(1, n))(), (TableInfo * max(1, n))()
    _check(L.mpm_model_grid(P.ctypes.data, r, m, sigma, max_positions, ps, infos, n,
                            ctypes.byref(count)), "mpm_model_grid")
    return [(ps[i].as_dict(), infos[i].as_dict()) for i in range(n)]


def features(sigma, entropy, m, r, n, params):
    """Model inputs (float32, len(params) x 8) for parameter dicts `params`."""
    k = len(params)
    arr = (Params * max(1, k))()
    for i, p in enumerate(params):
        for f, _ in Params._fields_:
            setattr(arr[i], f, int(p.get(f, -1 if f == "map_shift" else 0)))
    X = np.zeros((k, N_IN), np.float32)
    _check(lib().mpm_model_features(int(sigma), float(entropy), int(m), int(r), int(n), arr, k,
                                    _fptr(X)), "mpm_model_features")
    return X


class Model:
    """One mpm_model: parameters, normalisation and Adam state."""

    def __init__(self, seed=0, _handle=None):
        self._h = _handle if _handle is not None else lib().mpm_model_create(seed)
        if not self._h:
            raise MpmError(lib().mpm_last_error(), "mpm_model_create")

    @classmethod
    def load(cls, path=MODEL_PATH):
        h = lib().mpm_model_load(os.fsencode(path))
        if not h:
            raise MpmError(lib().mpm_last_error(), "mpm_model_load")
        return cls(_handle=h)

    def save(self, path):
        _check(lib().mpm_model_save(self._h, os.fsencode(path)), "mpm_model_save")

    def close(self):
        if self._h:
            lib().mpm_model_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def params(self):
        out = np.zeros(N_PARAMS, np.float32)
        _check(lib().mpm_model_get_params(self._h, _fptr(out)), "mpm_model_get_params")
        return out

    @params.setter
    def params(self, theta):
        theta = _f32(theta, (N_PARAMS,))
        _check(lib().mpm_model_set_params(self._h, _fptr(theta)), "mpm_model_set_params")

    @property
    def norm(self):
        mean, std = np.zeros(N_IN, np.float32), np.zeros(N_IN, np.float32)
        om, osd = ctypes.c_float(), ctypes.c_float()
        _check(lib().mpm_model_get_norm(self._h, _fptr(mean), _fptr(std), ctypes.byref(om),
                                        ctypes.byref(osd)), "mpm_model_get_norm")
        return mean, std, om.value, osd.value

    def set_norm(self, in_mean, in_std, out_mean, out_std):
        in_mean, in_std = _f32(in_mean, (N_IN,)), _f32(in_std, (N_IN,))
        _check(lib().mpm_model_set_norm(self._h, _fptr(in_mean), _fptr(in_std), float(out_mean),
                                        float(out_std)), "mpm_model_set_norm")

    def fit_norm(self, X, y):
        """Standardise with the training data's mean and deviation (inputs that
        do not vary get deviation 1)."""
        X = np.asarray(X, np.float64)
        y = np.asarray(y, np.float64)
        sd = X.std(axis=0)
        sd[sd < 1e-6] = 1.0
        self.set_norm(X.mean(axis=0), sd, y.mean(), max(y.std(), 1e-6))

    def predict(self, X):
        """Predicted ln(ms) for raw features X (N x 8, numpy or CUDA tensor)."""
        if hasattr(X, "is_cuda") and X.is_cuda:
            import torch
            X = X.to(torch.float32).contiguous()
            y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
            _check(lib().mpm_model_predict(self._h, X.data_ptr(), X.shape[0], y.data_ptr()),
                   "mpm_model_predict")
            return y
        X = _f32(X).reshape(-1, N_IN)
        y = np.zeros(X.shape[0], np.float32)
        _check(lib().mpm_model_predict(self._h, X.ctypes.data, X.shape[0], y.ctypes.data),
               "mpm_model_predict")
        return y

    def loss_grad(self, X, y):
        X = _f32(X).reshape(-1, N_IN)
        y = _f32(y, (X.shape[0],))
        loss = ctypes.c_float()
        g = np.zeros(N_PARAMS, np.float32)
        _check(lib().mpm_model_loss_grad(self._h, X.ctypes.data, y.ctypes.data, X.shape[0],
                                         ctypes.byref(loss), _fptr(g)), "mpm_model_loss_grad")
        return loss.value, g

    def adam_step(self, grad, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        grad = _f32(grad, (N_PARAMS,))
        opts = TrainOpts(lr, beta1, beta2, eps, 0, 0, 0)
        _check(lib().mpm_model_adam_step(self._h, _fptr(grad), ctypes.byref(opts)),
               "mpm_model_adam_step")

    def train(self, X, y, epochs=200, batch=256, lr=1e-3, seed=0, beta1=0.9, beta2=0.999,
              eps=1e-8):
        """Mini-batch Adam on the GPU; returns each epoch's mean loss."""
        X = _f32(X).reshape(-1, N_IN)
        y = _f32(y, (X.shape[0],))
        opts = TrainOpts(lr, beta1, beta2, eps, epochs, batch, seed)
        losses = np.zeros(epochs, np.float32)
        _check(lib().mpm_model_train(self._h, X.ctypes.data, y.ctypes.data, X.shape[0],
                                     ctypes.byref(opts), _fptr(losses)), "mpm_model_train")
        return losses

    def choose(self, P, sigma, entropy, n, max_table_bytes=0):
        """Grid point with the smallest predicted time among those whose mask
        table has at most max_table_bytes (0: any): (params dict, ln ms)."""
        P = np.ascontiguousarray(np.asarray(P, dtype=np.uint8))
        best = Params()
        pred = ctypes.c_float()
        _check(lib().mpm_model_choose(self._h, P.ctypes.data, P.shape[0], P.shape[1], sigma,
                                      float(entropy), int(n), int(max_table_bytes),
                                      ctypes.byref(best), ctypes.byref(pred)),
               "mpm_model_choose")
        return best.as_dict(), pred.value


# ------------------------------------------------------- batched workloads

def batch_matcher(P, sigma, params):
    """A Matcher for one set of a batch: the given parameters, or, when they
    exceed the batched kernel's 32 filter positions, 16 greedy bins with
    q = 4 and k = 1."""
    from . import Matcher
    m = Matcher(P, sigma=sigma, **params)
    if m.info["positions"] > 32:
        m.close()
        m = Matcher(P, sigma=sigma, map_kind=2, sigma_r=16, q=4, k=1)
    return m


def learned_batch_params(batch, model, max_table_bytes=_native.BATCH_SMEM_TABLE_BYTES):
    """The model's parameters for every pattern set of a batch (workloads.Batch):
    features from the set's texts (entropy of their first 64 KiB each, the
    mean length held to [2^20, 2^23] as in the training data), grid points
    whose mask table fits max_table_bytes.  A set without texts gets {}."""
    out = []
    for sidx, P in enumerate(batch.sets):
        mine = np.flatnonzero(batch.set_of_text == sidx)
        if mine.size == 0:
            out.append({})
            continue
        ent = entropy_bits(np.concatenate([batch.texts[i][:1 << 16] for i in mine]))
        n = int(np.clip(np.mean([batch.texts[i].size for i in mine]), 1 << 20, 1 << 23))
        out.append(model.choose(P, batch.sigma, ent, n, max_table_bytes=max_table_bytes)[0])
    return out


# ---------------------------------------------------------- timing database

def default_params(P, sigma):
    """The library's own plan (mpm_build with every parameter left 0), held
    to the batched kernel's 32 filter positions by taking k = 1 when needed."""
    from . import plan
    p, info = plan(P, sigma)
    if info["positions"] > 32:
        p, info = plan(P, sigma, q=p["q"], sigma_r=p["sigma_r"], map_kind=p["map_kind"], k=1)
    if info["positions"] > 32:
        return None
    return p


def time_batched(P, sigma, T, params, reps=3, generic=False):
    """The tuner's measurement of the batched kernel (the one compiled for
    the set; generic=True: the precompiled one): text T (a CUDA tensor)
    repeated until at least 128 MiB are scanned (at most 256 copies), median
    device ms of reps runs divided by the number of copies."""
    from . import Batch, Matcher
    n = int(T.numel())
    copies = min(256, max(1, -(-(128 << 20) // n)))
    m = Matcher(P, sigma=sigma, **{k: v for k, v in params.items() if k != "kernel"})
    b = Batch([m], [T] * copies, np.zeros(copies, np.uint32), generic=generic)
    b.run()
    ms = []
    for _ in range(reps):
        b.run()
        ms.append(b.stats["ms"] / copies)
    b.close()
    return float(np.median(ms))


def collect(first, count, reps=3, log=print):
    """Time every grid point of pattern sets first .. first+count-1 with the
    batched kernel (median of reps device-timed runs), plus the default
    parameters.  Returns a dict of numpy arrays (one row per timed point)."""
    import torch
    from . import autotune
    from . import workloads as W
    rows = {k: [] for k in ("set", "X", "y", "q", "sigma_r", "k", "map_kind", "candidates")}
    per_set = {k: [] for k in ("set", "n", "r", "m", "entropy", "default_ms", "default_q",
                               "default_sigma_r", "default_k", "default_map")}
    t0 = time.time()
    for idx in range(first, first + count):
        case = W.config5_set(idx)
        T = torch.from_numpy(case.T).cuda()
        ent = entropy_bits(case.T)
        _, entries = autotune(case.P, case.sigma, T, kernels=8, grid=1, max_positions=32,
                              reps=reps)
        ok = [e for e in entries if e["status"] == 0 and e["ms"] > 0]
        if not ok:
            continue
        ps = [e["params"] for e in ok]
        X = features(case.sigma, ent, case.m, case.r, case.n, ps)
        rows["set"].append(np.full(len(ok), idx, np.int32))
        rows["X"].append(X)
        rows["y"].append(np.log(np.array([e["ms"] for e in ok], np.float64)).astype(np.float32))
        for f in ("q", "sigma_r", "k", "map_kind"):
            rows[f].append(np.array([p[f] for p in ps], np.int32))
        rows["candidates"].append(np.array([e["candidates"] for e in ok], np.int64))
        dp = default_params(case.P, case.sigma)
        dms = time_batched(case.P, case.sigma, T, dp, reps) if dp else float("nan")
        per_set["set"].append(idx)
        per_set["n"].append(case.n)
        per_set["r"].append(case.r)
        per_set["m"].append(case.m)
        per_set["entropy"].append(ent)
        per_set["default_ms"].append(dms)
        for f, key in (("q", "default_q"), ("sigma_r", "default_sigma_r"), ("k", "default_k"),
                       ("map_kind", "default_map")):
            per_set[key].append(dp[f] if dp else -1)
        if log:
            log("set %d r=%d m=%d n=%d: %d points, best %.3f ms, default %.3f ms (%.0f s)" % (
                idx, case.r, case.m, case.n, len(ok), min(e["ms"] for e in ok), dms,
                time.time() - t0))
        del T
    out = {k: np.concatenate(v) for k, v in rows.items()}
    out.update({"set_" + k if k != "set" else "sets": np.array(v) for k, v in per_set.items()})
    return out


def load_db(path=DB_PATH):
    with np.load(path) as z:
        return {k: z[k] for k in z.files}


def split(db, sets):
    """Rows of the database whose pattern set is in `sets`."""
    keep = np.isin(db["set"], np.asarray(list(sets)))
    return {k: db[k][keep] for k in ("set", "X", "y", "q", "sigma_r", "k", "map_kind")}


def evaluate(predict, db, sets=HELDOUT_SETS):
    """Regret of argmin(predict) per pattern set against the best measured
    point of its grid, and the gain over the default parameters.
    predict: function X -> predicted ln(ms)."""
    d = split(db, sets)
    regrets, gains, chosen_ms, best_ms, default_ms = [], [], [], [], []
    set_ids = list(db["sets"])
    for s in np.unique(d["set"]):
        rows = np.flatnonzero(d["set"] == s)
        ms = np.exp(d["y"][rows].astype(np.float64))
        pred = np.asarray(predict(d["X"][rows]))
        pick = ms[int(np.argmin(pred))]
        regrets.append(pick / ms.min() - 1.0)
        chosen_ms.append(pick)
        best_ms.append(ms.min())
        dm = db["set_default_ms"][set_ids.index(s)]
        default_ms.append(dm)
        if np.isfinite(dm):
            gains.append(dm / pick)
    regrets = np.array(regrets)
    return {
        "sets": int(regrets.size),
        "mean_regret": float(regrets.mean()),
        "median_regret": float(np.median(regrets)),
        "p90_regret": float(np.quantile(regrets, 0.9)),
        "sum_chosen_ms": float(np.sum(chosen_ms)),
        "sum_best_ms": float(np.sum(best_ms)),
        "sum_default_ms": float(np.nansum(default_ms)),
        "mean_speedup_over_default": float(np.mean(gains)) if gains else float("nan"),
        "geomean_speedup_over_default": float(np.exp(np.mean(np.log(gains)))) if gains else
        float("nan"),
    }


# training settings chosen by mean regret on a validation split of the
# training sets (0-159 trained, 160-199 validated; three seeds each of
# 300/600/1200 epochs x lr 1e-3/3e-3 x batch 128/256); the held-out sets
# 200-399 only evaluate the model trained on all 200 training sets
TRAIN_EPOCHS, TRAIN_LR, TRAIN_BATCH = 600, 3e-3, 256


def train_model(db, sets=TRAIN_SETS, epochs=TRAIN_EPOCHS, batch=TRAIN_BATCH, lr=TRAIN_LR, seed=1):
    d = split(db, sets)
    model = Model(seed)
    model.fit_norm(d["X"], d["y"])
    losses = model.train(d["X"], d["y"], epochs=epochs, batch=batch, lr=lr, seed=seed)
    return model, losses


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_1405_5483_gb300.cost_model")
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("collect")
    c.add_argument("out")
    c.add_argument("--first", type=int, default=0)
    c.add_argument("--count", type=int, default=400)
    c.add_argument("--reps", type=int, default=3)
    t = sub.add_parser("train")
    t.add_argument("db")
    t.add_argument("model")
    t.add_argument("--epochs", type=int, default=TRAIN_EPOCHS)
    t.add_argument("--seed", type=int, default=1)
    e = sub.add_parser("evaluate")
    e.add_argument("db")
    e.add_argument("model")
    a = ap.parse_args(argv)
    if a.cmd == "collect":
        db = collect(a.first, a.count, a.reps)
        np.savez_compressed(a.out, **db)
        print("wrote %s: %d rows" % (a.out, db["y"].size))
    elif a.cmd == "train":
        db = load_db(a.db)
        t0 = time.time()
        model, losses = train_model(db, epochs=a.epochs, seed=a.seed)
        model.save(a.model)
        print(json.dumps({"epochs": a.epochs, "first_loss": float(losses[0]),
                          "last_loss": float(losses[-1]), "seconds": round(time.time() - t0, 2),
                          "heldout": evaluate(model.predict, db)}))
    else:
        db = load_db(a.db)
        model = Model.load(a.model)
        print(json.dumps(evaluate(model.predict, db)))


if __name__ == "__main__":
    main()
