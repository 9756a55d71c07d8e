"""GB300-native ALS-WR / ALS-NCG (arXiv 1508.03110) behind a C ABI.

The Python layer only marshals arguments to the entry points declared in
include/als.h; every step of the computation runs in the library's CUDA
kernels.  PyTorch supplies device memory (its caching allocator is passed to
the library as the allocation hook) and the CUDA stream.
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import (ALS_FP64, ALS_MIXED, ALS_LS_BACKTRACK, ALS_LS_EXACT, ALS_DT_F64, ALS_DT_F32,  # noqa: F401
                   ALS_GRAM_AUTO, ALS_GRAM_FMA, ALS_GRAM_TC, ALSError, IterInfo)

__all__ = ["ALS", "ALSBatch", "ALSGroup", "Server", "ALSError", "load", "info_dict", "make_config",
           "probe_alu_peaks"]


def load():
    return _lib.load()


def probe_alu_peaks():
    """Measured dense FMA peaks of the current device (als_probe_alu_peaks):
    (FP32 TFLOP/s, FP64 TFLOP/s)."""
    f32, f64 = ctypes.c_double(), ctypes.c_double()
    _lib.check(_lib.load().als_probe_alu_peaks(ctypes.byref(f32), ctypes.byref(f64)), "als_probe_alu_peaks")
    return f32.value, f64.value


def _torch():
    import torch
    return torch


def info_dict(info: IterInfo) -> dict:
    return dict(k=info.k, f=info.f, gnorm=info.gnorm, gnorm0=info.gnorm0, alpha=info.alpha,
                beta=info.beta, c=list(info.c), shrinks=info.shrinks, fallback=bool(info.fallback),
                fallbacks=info.fallbacks, notspd=info.notspd, kernels=info.kernels)


class _Buf:
    """A host (numpy) or device (torch) buffer handed to the C ABI."""

    def __init__(self, arr, np_dtype):
        torch = _torch()
        if isinstance(arr, torch.Tensor):
            want = {np.float64: torch.float64, np.float32: torch.float32, np.int32: torch.int32,
                    np.int64: torch.int64}[np_dtype]
            t = arr.contiguous()
            if t.dtype != want:
                t = t.to(want)
            self.keep = t
            self.ptr = t.data_ptr()
            self.on_device = 1 if t.is_cuda else 0
        else:
            a = np.ascontiguousarray(arr, dtype=np_dtype)
            self.keep = a
            self.ptr = a.ctypes.data
            self.on_device = 0


BETA_FORMS = {"pr": _lib.ALS_BETA_PR, "fr": _lib.ALS_BETA_FR, "hs": _lib.ALS_BETA_HS,
              "prplus": _lib.ALS_BETA_PR_PLUS}
# the More-Thuente search with the paper's serial settings (§IV) unless given
MT_DEFAULTS = dict(ls_alpha0=1.0, ls_c=1e-4, ls_c2=1e-2, ls_max_shrinks=20)


def make_config(n_f, lam, precision="fp64", ls_mode="backtrack", refine_steps=2, gram_path="auto",
                hbm_budget_bytes=0, ls_alpha0=None, ls_tau=0.9, ls_c=None, ls_max_shrinks=None,
                beta="pr", precond="als", ls_c2=None):
    """An als_config with the library defaults and the given fields.
    ls_mode: "backtrack" (Algorithm 3), "exact" or "more-thuente"; beta: one
    of BETA_FORMS; precond: "als" (ALS-NCG) or "none" (plain NCG)."""
    cfg = _lib.Config()
    _lib.load().als_config_default(ctypes.byref(cfg))
    cfg.n_f = int(n_f)
    cfg.lam = float(lam)
    cfg.precision = {"fp64": ALS_FP64, "mixed": ALS_MIXED}[precision]
    cfg.ls_mode = {"backtrack": ALS_LS_BACKTRACK, "exact": ALS_LS_EXACT,
                   "more-thuente": _lib.ALS_LS_MORE_THUENTE}[ls_mode]
    dflt = MT_DEFAULTS if ls_mode == "more-thuente" else dict(ls_alpha0=10.0, ls_c=0.5, ls_c2=1e-2,
                                                               ls_max_shrinks=200)
    ls_alpha0 = dflt["ls_alpha0"] if ls_alpha0 is None else ls_alpha0
    ls_c = dflt["ls_c"] if ls_c is None else ls_c
    ls_c2 = dflt["ls_c2"] if ls_c2 is None else ls_c2
    ls_max_shrinks = dflt["ls_max_shrinks"] if ls_max_shrinks is None else ls_max_shrinks
    cfg.ls_alpha0, cfg.ls_tau, cfg.ls_c, cfg.ls_c2 = float(ls_alpha0), float(ls_tau), float(ls_c), float(ls_c2)
    cfg.ls_max_shrinks = int(ls_max_shrinks)
    cfg.beta_form = BETA_FORMS[beta]
    cfg.preconditioner = {"als": _lib.ALS_PRECOND_ALS, "none": _lib.ALS_PRECOND_NONE}[precond]
    cfg.refine_steps = int(refine_steps)
    cfg.gram_path = {"auto": ALS_GRAM_AUTO, "fma": ALS_GRAM_FMA, "tc": ALS_GRAM_TC}[gram_path]
    cfg.hbm_budget_bytes = int(hbm_budget_bytes)
    return cfg


class ALS:
    """One factorisation problem R ~ U^T M on the current CUDA device.

    precision: "fp64" (parity form) or "mixed" (BF16/FP32 Gram, FP32
    Cholesky with refinement, FP64 reductions).
    """

    def __init__(self, n_u, n_m, rows, cols, vals, n_f, lam, precision="fp64", ls_mode="backtrack",
                 refine_steps=2, gram_path="auto", hbm_budget_bytes=0, stream=None, rowptr=None,
                 ls_alpha0=None, ls_tau=0.9, ls_c=None, ls_max_shrinks=None, beta="pr", precond="als",
                 ls_c2=None):
        torch = _torch()
        self.lib = _lib.load()
        self.n_u, self.n_m, self.n_f = int(n_u), int(n_m), int(n_f)
        cfg = make_config(self.n_f, lam, precision, ls_mode, refine_steps, gram_path, hbm_budget_bytes,
                          ls_alpha0, ls_tau, ls_c, ls_max_shrinks, beta, precond, ls_c2)
        # device memory comes from torch's caching allocator
        self._blocks = {}

        def _alloc(nbytes, stream_, user):
            dev = torch.cuda.current_device()
            ptr = torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream_ or 0)
            return ptr

        def _free(ptr, nbytes, stream_, user):
            torch.cuda.caching_allocator_delete(ptr)

        self._alloc_cb = _lib.ALLOC_FN(_alloc)
        self._free_cb = _lib.FREE_FN(_free)
        cfg.alloc = self._alloc_cb
        cfg.free = self._free_cb
        self.cfg = cfg
        self.precision = precision
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        nnz = int(len(cols))
        self.nnz = nnz
        cb = _Buf(cols, np.int32)
        vb = _Buf(vals, np.float32)
        if rowptr is not None:
            rp = _Buf(rowptr, np.int64)
            rb_ptr, rp_ptr = None, rp.ptr
            on_dev = rp.on_device
        else:
            rb = _Buf(rows, np.int32)
            rb_ptr, rp_ptr = rb.ptr, None
            on_dev = rb.on_device
        if not (cb.on_device == vb.on_device == on_dev):
            raise ValueError("ratings arrays must all be on the host or all on the device")
        ctx = ctypes.c_void_p()
        st = self.lib.als_create(ctypes.byref(cfg), self.n_u, self.n_m, nnz, rb_ptr, rp_ptr, cb.ptr,
                                 vb.ptr, on_dev, ctypes.c_void_p(self.stream.cuda_stream),
                                 ctypes.byref(ctx))
        _lib.check(st, "als_create")
        self.ctx = ctx

    # -- lifetime -----------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.als_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def ratings(self):
        """The device-built by-user / by-item structures and degree orders."""
        nnz = self.nnz
        out = dict(uptr=np.empty(self.n_u + 1, np.int64), uidx=np.empty(nnz, np.int32),
                   uval=np.empty(nnz, np.float32), mptr=np.empty(self.n_m + 1, np.int64),
                   midx=np.empty(nnz, np.int32), mval=np.empty(nnz, np.float32),
                   uorder=np.empty(self.n_u, np.int32), morder=np.empty(self.n_m, np.int32))
        _lib.check(self.lib.als_get_ratings(self.ctx, *[out[k].ctypes.data for k in
                                                        ("uptr", "uidx", "uval", "mptr", "midx", "mval",
                                                         "uorder", "morder")]), "als_get_ratings")
        return out

    # -- factors ----------------------------------------------------------------
    def set_factors(self, U, M):
        dt = ALS_DT_F64
        if not isinstance(U, np.ndarray) and getattr(U, "dtype", None) is not None and "float32" in str(U.dtype):
            dt = ALS_DT_F32
        npdt = np.float64 if dt == ALS_DT_F64 else np.float32
        ub, mb = _Buf(U, npdt), _Buf(M, npdt)
        if ub.on_device != mb.on_device:
            raise ValueError("U and M must both be on the host or both on the device")
        _lib.check(self.lib.als_set_factors(self.ctx, ub.ptr, mb.ptr, dt, ub.on_device), "als_set_factors")
        if ub.on_device:
            self.sync()

    def set_x(self, x):
        x = np.asarray(x, np.float64).reshape(self.n_u + self.n_m, self.n_f)
        self.set_factors(x[:self.n_u], x[self.n_u:])

    def get_factors(self, dtype="float64", device=False, out=None):
        """U (n_u x n_f) and M (n_m x n_f) as `dtype`, on the device (torch)
        or the host (numpy).  `out` = (U, M): contiguous arrays of that dtype
        and shape to write into instead, numpy arrays or torch tensors (CPU,
        for example pinned, or CUDA); returned as given."""
        torch = _torch()
        if out is not None:
            U, M = out
            want = (self.n_u, self.n_f), (self.n_m, self.n_f)
            dt = ALS_DT_F64 if dtype == "float64" else ALS_DT_F32
            ptrs, devs = [], []
            for a, shape in zip((U, M), want):
                if isinstance(a, torch.Tensor):
                    ok = (a.is_contiguous() and tuple(a.shape) == shape
                          and a.dtype == (torch.float64 if dt == ALS_DT_F64 else torch.float32))
                    ptrs.append(a.data_ptr()); devs.append(1 if a.is_cuda else 0)
                else:
                    ok = (isinstance(a, np.ndarray) and a.flags.c_contiguous and a.shape == shape
                          and a.dtype == (np.float64 if dt == ALS_DT_F64 else np.float32))
                    ptrs.append(a.ctypes.data if ok else 0); devs.append(0)
                if not ok:
                    raise ValueError(f"get_factors: out arrays must be contiguous {dtype} of shapes {want}")
            if devs[0] != devs[1]:
                raise ValueError("get_factors: out arrays must both be on the host or both on the device")
            _lib.check(self.lib.als_get_factors(self.ctx, ptrs[0], ptrs[1], dt, devs[0]), "als_get_factors")
            if devs[0]:
                self.sync()
            return U, M
        if device:
            tdt = torch.float64 if dtype == "float64" else torch.float32
            U = torch.empty((self.n_u, self.n_f), dtype=tdt, device="cuda")
            M = torch.empty((self.n_m, self.n_f), dtype=tdt, device="cuda")
            dt = ALS_DT_F64 if dtype == "float64" else ALS_DT_F32
            _lib.check(self.lib.als_get_factors(self.ctx, U.data_ptr(), M.data_ptr(), dt, 1), "als_get_factors")
            self.sync()
            return U, M
        npdt = np.float64 if dtype == "float64" else np.float32
        U = np.empty((self.n_u, self.n_f), npdt)
        M = np.empty((self.n_m, self.n_f), npdt)
        dt = ALS_DT_F64 if dtype == "float64" else ALS_DT_F32
        _lib.check(self.lib.als_get_factors(self.ctx, U.ctypes.data, M.ctypes.data, dt, 0), "als_get_factors")
        return U, M

    def get_x(self):
        U, M = self.get_factors()
        return np.concatenate([U.reshape(-1), M.reshape(-1)])

    def get_state(self):
        """Algorithm 2 state: dict of x, p, g, gbar, xbar (float64, flat) and scalars."""
        n = (self.n_u + self.n_m) * self.n_f
        v = {k: np.empty(n, np.float64) for k in ("x", "p", "g", "gbar", "xbar")}
        sc = (ctypes.c_double * 4)()
        _lib.check(self.lib.als_get_state(self.ctx, v["x"].ctypes.data, v["p"].ctypes.data, v["g"].ctypes.data,
                                          v["gbar"].ctypes.data, v["xbar"].ctypes.data, sc, ALS_DT_F64, 0),
                   "als_get_state")
        v.update(s=sc[0], gg0=sc[1], k=int(sc[2]), fallbacks=int(sc[3]))
        return v

    def set_state(self, x, p, g, gbar, xbar, s, gg0, k=0, fallbacks=0):
        arrs = [np.ascontiguousarray(a, np.float64).reshape(-1) for a in (x, p, g, gbar, xbar)]
        sc = (ctypes.c_double * 4)(float(s), float(gg0), float(k), float(fallbacks))
        _lib.check(self.lib.als_set_state(self.ctx, *[a.ctypes.data for a in arrs], sc, ALS_DT_F64, 0),
                   "als_set_state")

    # -- algorithms -------------------------------------------------------------
    def sweep(self, n=1):
        _lib.check(self.lib.als_sweep(self.ctx, int(n)), "als_sweep")

    def step(self, info=True):
        if not info:
            _lib.check(self.lib.alsncg_step(self.ctx, None), "alsncg_step")
            return None
        it = IterInfo()
        _lib.check(self.lib.alsncg_step(self.ctx, ctypes.byref(it)), "alsncg_step")
        return info_dict(it)

    def run(self, max_iter, rel_tol=0.0, check_every=10):
        it = IterInfo()
        done = ctypes.c_int32(0)
        _lib.check(self.lib.alsncg_run(self.ctx, int(max_iter), float(rel_tol), int(check_every),
                                       ctypes.byref(it), ctypes.byref(done)), "alsncg_run")
        d = info_dict(it)
        d["iters"] = done.value
        return d

    def loss(self):
        f = ctypes.c_double()
        _lib.check(self.lib.als_loss(self.ctx, ctypes.byref(f)), "als_loss")
        return f.value

    def grad(self, want_vector=True):
        gn = ctypes.c_double()
        if want_vector:
            g = np.empty((self.n_u + self.n_m) * self.n_f, np.float64)
            _lib.check(self.lib.als_grad(self.ctx, g.ctypes.data, ALS_DT_F64, 0, ctypes.byref(gn)), "als_grad")
            return g, gn.value
        _lib.check(self.lib.als_grad(self.ctx, None, ALS_DT_F64, 0, ctypes.byref(gn)), "als_grad")
        return None, gn.value

    def linesearch_coeffs(self, p=None):
        c = (ctypes.c_double * 5)()
        if p is None:
            _lib.check(self.lib.als_linesearch_coeffs(self.ctx, None, ALS_DT_F64, 0, c), "als_linesearch_coeffs")
        else:
            pb = _Buf(p, np.float64)
            _lib.check(self.lib.als_linesearch_coeffs(self.ctx, pb.ptr, ALS_DT_F64, pb.on_device, c),
                       "als_linesearch_coeffs")
        return np.array(list(c))

    def foldin(self, req_ptr, items, vals, dtype="float64"):
        n_req = len(req_ptr) - 1
        pb, ib, vb = _Buf(req_ptr, np.int64), _Buf(items, np.int32), _Buf(vals, np.float32)
        npdt = np.float64 if dtype == "float64" else np.float32
        out = np.empty((n_req, self.n_f), npdt)
        dt = ALS_DT_F64 if dtype == "float64" else ALS_DT_F32
        _lib.check(self.lib.als_foldin(self.ctx, n_req, pb.ptr, ib.ptr, vb.ptr, pb.on_device,
                                       out.ctypes.data, dt, 0), "als_foldin")
        return out

    def autotune(self, reps=3):
        """Time candidate launch shapes on this problem and keep the fastest
        (als_autotune); returns the shapes kept and the before/after times."""
        r = _lib.TuneReport()
        _lib.check(self.lib.als_autotune(self.ctx, int(reps), ctypes.byref(r)), "als_autotune")
        out = {k: getattr(r, k) for k, _ in r._fields_ if k != "chosen"}
        out.update({k: getattr(r.chosen, k) for k, _ in r.chosen._fields_})
        return out

    def rank_topt(self, t):
        """The first t items of every user's ranking by the current factors
        (als_rank_topt): int32 array n_u x t."""
        out = np.empty((self.n_u, int(t)), np.int32)
        _lib.check(self.lib.als_rank_topt(self.ctx, int(t), out.ctypes.data, 0), "als_rank_topt")
        return out

    def rank_accuracy(self, top_ref, per_user=False):
        """Mean top-t ranking accuracy q against reference lists (n_u x t)
        (als_rank_accuracy); with per_user also the n_u values q_i."""
        ref = np.ascontiguousarray(top_ref, np.int32)
        qm = ctypes.c_double()
        qu = np.empty(self.n_u, np.float64) if per_user else None
        _lib.check(self.lib.als_rank_accuracy(self.ctx, int(ref.shape[1]), ref.ctypes.data, 0, ctypes.byref(qm),
                                              qu.ctypes.data if per_user else None), "als_rank_accuracy")
        return (qm.value, qu) if per_user else qm.value

    def time_sweep(self, reps=5):
        """Per-kernel-class launch times of one sweep (als_time_sweep): dict
        with sweep_ms and, per class name, ms / launches / rows / ratings."""
        t = _lib.SweepTiming()
        _lib.check(self.lib.als_time_sweep(self.ctx, int(reps), ctypes.byref(t)), "als_time_sweep")
        out = {"sweep_ms": t.sweep_ms}
        for i, name in enumerate(_lib.SWEEP_CLASSES):
            out[name] = {"ms": t.ms[i], "launches": t.launches[i], "rows": t.rows[i], "ratings": t.ratings[i]}
        return out

    def get_launch(self):
        l = _lib.Launch()
        _lib.check(self.lib.als_get_launch(self.ctx, ctypes.byref(l)), "als_get_launch")
        return {k: getattr(l, k) for k, _ in l._fields_}

    def set_launch(self, **shape):
        """Set launch shapes (als_set_launch); unspecified fields keep their value."""
        l = _lib.Launch()
        _lib.check(self.lib.als_get_launch(self.ctx, ctypes.byref(l)), "als_get_launch")
        for k, v in shape.items():
            if k == "gram_path" and isinstance(v, str):
                v = {"fma": ALS_GRAM_FMA, "tc": ALS_GRAM_TC}[v]
            setattr(l, k, int(v))
        _lib.check(self.lib.als_set_launch(self.ctx, ctypes.byref(l)), "als_set_launch")

    def sync(self):
        _lib.check(self.lib.als_sync(self.ctx), "als_sync")


class ALSBatch(ALS):
    """Many independent problems (list of (n_u, n_m, rows, cols, vals) with
    local ids) sharing n_f, lambda and precision, solved in the same launches.
    Vectors use the global layout: every problem's U rows, then every
    problem's M rows."""

    def __init__(self, problems, n_f, lam, precision="fp64", ls_mode="backtrack", refine_steps=2,
                 gram_path="auto", hbm_budget_bytes=0, stream=None, **variant):
        """variant: make_config's line-search, beta and preconditioner keywords."""
        torch = _torch()
        self.lib = _lib.load()
        self.n_prob = len(problems)
        self.sizes = [(int(p[0]), int(p[1])) for p in problems]
        self.n_u = sum(s[0] for s in self.sizes)
        self.n_m = sum(s[1] for s in self.sizes)
        self.n_f = int(n_f)
        cfg = make_config(self.n_f, lam, precision, ls_mode, refine_steps, gram_path, hbm_budget_bytes,
                          **variant)

        def _alloc(nbytes, stream_, user):
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream_ or 0)

        def _free(ptr, nbytes, stream_, user):
            torch.cuda.caching_allocator_delete(ptr)

        self._alloc_cb = _lib.ALLOC_FN(_alloc)
        self._free_cb = _lib.FREE_FN(_free)
        cfg.alloc, cfg.free = self._alloc_cb, self._free_cb
        self.cfg = cfg
        self.precision = precision
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        nu = np.array([s[0] for s in self.sizes], np.int64)
        nm = np.array([s[1] for s in self.sizes], np.int64)
        nz = np.array([len(p[3]) for p in problems], np.int64)
        rows = np.ascontiguousarray(np.concatenate([np.asarray(p[2], np.int32) for p in problems]), np.int32)
        cols = np.ascontiguousarray(np.concatenate([np.asarray(p[3], np.int32) for p in problems]), np.int32)
        vals = np.ascontiguousarray(np.concatenate([np.asarray(p[4], np.float32) for p in problems]), np.float32)
        self.nnz = int(nz.sum())
        ctx = ctypes.c_void_p()
        st = self.lib.als_create_batched(ctypes.byref(cfg), self.n_prob, nu.ctypes.data, nm.ctypes.data,
                                         nz.ctypes.data, rows.ctypes.data, cols.ctypes.data, vals.ctypes.data,
                                         0, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx))
        _lib.check(st, "als_create_batched")
        self.ctx = ctx
        self._uoff = np.concatenate([[0], np.cumsum(nu)])
        self._moff = np.concatenate([[0], np.cumsum(nm)])

    def join_x(self, xs):
        """Global x from per-problem x vectors (Eq. 5 layout each)."""
        us, ms = [], []
        for (nu, nm), x in zip(self.sizes, xs):
            x = np.asarray(x, np.float64).reshape(nu + nm, self.n_f)
            us.append(x[:nu]); ms.append(x[nu:])
        return np.concatenate(us + ms).reshape(-1)

    def split_x(self, x):
        x = np.asarray(x).reshape(self.n_u + self.n_m, self.n_f)
        out = []
        for q in range(self.n_prob):
            U = x[self._uoff[q]:self._uoff[q + 1]]
            M = x[self.n_u + self._moff[q]:self.n_u + self._moff[q + 1]]
            out.append(np.concatenate([U.reshape(-1), M.reshape(-1)]))
        return out

    def infos(self):
        arr = (IterInfo * self.n_prob)()
        _lib.check(self.lib.als_batch_info(self.ctx, self.n_prob, arr), "als_batch_info")
        return [info_dict(a) for a in arr]

    def grad_norms(self):
        """|grad f| of every problem at the current factors (als_batch_grad_norms)."""
        out = (ctypes.c_double * self.n_prob)()
        _lib.check(self.lib.als_batch_grad_norms(self.ctx, self.n_prob, out), "als_batch_grad_norms")
        return np.array(out[:])


class Server:
    """Continuous-batching server over a model's M (als_server_* in the C ABI).

    Fold-in requests (one new user's items and ratings) are packed into device
    batches by the library's worker thread as they arrive; factorisation jobs
    are admitted by device-memory budget and advanced one ALS-NCG iteration at
    a time between the batches.  The model must not be used by other calls
    while the server exists.
    """

    def __init__(self, model, max_batch=256, max_batch_ratings=1 << 20, slots=4, max_jobs=4,
                 hbm_budget_bytes=0):
        self.lib = _lib.load()
        self.model = model
        cfg = _lib.ServerConfig()
        self.lib.als_server_config_default(ctypes.byref(cfg))
        cfg.max_batch, cfg.max_batch_ratings, cfg.slots = int(max_batch), int(max_batch_ratings), int(slots)
        cfg.max_jobs, cfg.hbm_budget_bytes = int(max_jobs), int(hbm_budget_bytes)
        srv = ctypes.c_void_p()
        _lib.check(self.lib.als_server_create(model.ctx, ctypes.byref(cfg), ctypes.byref(srv)),
                   "als_server_create")
        self.srv = srv
        self._kind = {}   # ticket -> result shape

    def close(self):
        if getattr(self, "srv", None):
            self.lib.als_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit_foldin(self, items, vals):
        items = np.ascontiguousarray(items, np.int32)
        vals = np.ascontiguousarray(vals, np.float32)
        if items.shape != vals.shape:
            raise ValueError("items and vals must have the same length")
        t = ctypes.c_int64()
        _lib.check(self.lib.als_server_submit_foldin(self.srv, len(items), items.ctypes.data, vals.ctypes.data,
                                                     ctypes.byref(t)), "als_server_submit_foldin")
        self._kind[t.value] = ("foldin", (self.model.n_f,), np.float32)
        return t.value

    def replay(self, t_arrival, req_ptr, items, vals):
        """Native open-loop load generator (als_server_replay): submit request q
        at t_arrival[q] seconds; returns (tickets, largest lag behind schedule)."""
        t_arrival = np.ascontiguousarray(t_arrival, np.float64)
        req_ptr = np.ascontiguousarray(req_ptr, np.int64)
        items = np.ascontiguousarray(items, np.int32)
        vals = np.ascontiguousarray(vals, np.float32)
        n = t_arrival.shape[0]
        tickets = np.empty(n, np.int64)
        lag = ctypes.c_double()
        _lib.check(self.lib.als_server_replay(self.srv, n, t_arrival.ctypes.data, req_ptr.ctypes.data,
                                              items.ctypes.data, vals.ctypes.data, tickets.ctypes.data,
                                              ctypes.byref(lag)), "als_server_replay")
        for t in tickets:
            self._kind[int(t)] = ("foldin", (self.model.n_f,), np.float32)
        return tickets, lag.value

    def submit_job(self, n_u, n_m, rows, cols, vals, x0, iters, n_f, lam, **config):
        """x0: (n_u + n_m) x n_f float64 initial factors; config: make_config's keywords."""
        cfg = make_config(n_f, lam, **config)
        rows = np.ascontiguousarray(rows, np.int32)
        cols = np.ascontiguousarray(cols, np.int32)
        vals = np.ascontiguousarray(vals, np.float32)
        x0 = np.ascontiguousarray(x0, np.float64).reshape(int(n_u) + int(n_m), int(n_f))
        t = ctypes.c_int64()
        _lib.check(self.lib.als_server_submit_job(self.srv, ctypes.byref(cfg), int(n_u), int(n_m), len(vals),
                                                  rows.ctypes.data, cols.ctypes.data, vals.ctypes.data,
                                                  x0.ctypes.data, int(iters), ctypes.byref(t)),
                   "als_server_submit_job")
        self._kind[t.value] = ("job", x0.shape, np.float64)
        return t.value

    def wait(self, ticket, timeout=60.0):
        """(result, latency in seconds) of a ticket; raises ALSError (ALS_ETIMEOUT) if not done in time."""
        _, shape, dt = self._kind[ticket]
        out = np.empty(shape, dt)
        lat = ctypes.c_double()
        st = self.lib.als_server_wait(self.srv, ticket, float(timeout), out.ctypes.data, ctypes.byref(lat))
        if st != _lib.ALS_ETIMEOUT:
            del self._kind[ticket]
        _lib.check(st, "als_server_wait")
        return out, lat.value

    def stats(self):
        p50, p99, rps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int64()
        _lib.check(self.lib.als_server_stats(self.srv, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(n),
                                             ctypes.byref(rps)), "als_server_stats")
        return {"p50_s": p50.value, "p99_s": p99.value, "completed": n.value, "requests_per_s": rps.value}


class ALSGroup:
    """A collection of independent problems with different n_f: one batched
    context per n_f value (all its problems in the same launches), iterated
    together by als_group_run.

    problems: list of (n_u, n_m, rows, cols, vals) with local ids; n_fs: the
    n_f of each problem."""

    def __init__(self, problems, n_fs, lam, precision="mixed", autotune=True, priorities=True,
                 schedule="concurrent", **kw):
        """schedule: "serial" puts every member on one stream, so that each
        iteration runs the members' graphs one after another (each one's
        launches fill the GPU by themselves); "concurrent" gives each member a
        stream of its own, so that their kernels may overlap.  priorities
        (concurrent only): the member with the most work per iteration
        (ratings x n_f^2) gets the highest stream priority, the next one the
        next."""
        if schedule not in ("serial", "concurrent"):
            raise ValueError("schedule: 'serial' or 'concurrent'")
        torch = _torch()
        self.lib = _lib.load()
        self.order = {}
        for q, nf in enumerate(n_fs):
            self.order.setdefault(int(nf), []).append(q)
        self.n_prob = len(problems)
        work = {nf: sum(len(problems[q][4]) for q in qs) * nf * nf for nf, qs in self.order.items()}
        ranked = sorted(self.order, key=lambda nf: -work[nf])
        if schedule == "serial":
            one = torch.cuda.Stream()
            self.streams = {nf: one for nf in self.order}
        else:
            if priorities:
                least, greatest = torch.cuda.Stream.priority_range()
                span = (list(range(greatest, least + 1)) if greatest <= least
                        else list(range(greatest, least - 1, -1)))
                prio = {nf: span[min(i, len(span) - 1)] for i, nf in enumerate(ranked)}
            else:
                prio = {nf: 0 for nf in ranked}
            self.streams = {nf: torch.cuda.Stream(priority=prio[nf]) for nf in self.order}
        self.batches = {nf: ALSBatch([problems[q] for q in qs], nf, lam, precision=precision,
                                     stream=self.streams[nf], **kw)
                        for nf, qs in self.order.items()}
        self.autotune_reports = {}
        self._autotune = autotune

    def close(self):
        for b in self.batches.values():
            b.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_x(self, xs):
        """xs: the n_f-wide x_0 of every problem, in problem order."""
        for nf, qs in self.order.items():
            b = self.batches[nf]
            b.set_x(b.join_x([xs[q] for q in qs]))
        if self._autotune and not self.autotune_reports:
            self.autotune_reports = {nf: b.autotune(reps=1) for nf, b in self.batches.items()}

    def get_x(self):
        out = [None] * self.n_prob
        for nf, qs in self.order.items():
            parts = self.batches[nf].split_x(self.batches[nf].get_x())
            for q, x in zip(qs, parts):
                out[q] = x
        return out

    def run(self, max_iter, rel_tol=0.0, check_every=10):
        members = list(self.batches.values())
        arr = (ctypes.c_void_p * len(members))(*[b.ctx.value for b in members])
        infos = (IterInfo * len(members))()
        done = ctypes.c_int32()
        _lib.check(self.lib.als_group_run(arr, len(members), int(max_iter), float(rel_tol), int(check_every),
                                          infos, ctypes.byref(done)), "als_group_run")
        return {"iters": done.value, "kernels": sum(i.kernels for i in infos)}

    def infos(self):
        out = [None] * self.n_prob
        for nf, qs in self.order.items():
            for q, info in zip(qs, self.batches[nf].infos()):
                out[q] = info
        return out
