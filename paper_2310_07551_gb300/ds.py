"""Thin Python binding of the ds3 C ABI (include/ds.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  PyTorch supplies device memory and streams.  If the compiled
library is missing this module raises at import of `lib()`: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libds3.so")

DS_OK, DS_ERR_INVALID_ARG, DS_ERR_UNSUPPORTED, DS_ERR_OOM, DS_ERR_CUDA, DS_ERR_NONFINITE, DS_ERR_TIMEOUT = range(7)
STATUS_NAMES = ["DS_OK", "DS_ERR_INVALID_ARG", "DS_ERR_UNSUPPORTED", "DS_ERR_OOM", "DS_ERR_CUDA",
                "DS_ERR_NONFINITE", "DS_ERR_TIMEOUT"]
PREC = {"f64": 0, "bf16x6": 1, "f32": 2, "bf16x6c": 3, "f16x10": 4, "f16x13": 5}
MODELS = {"schnakenberg": 0, "fhn": 1, "linear": 2}
SCHEMES = {"exprk3ds_real": 0, "etd2rkds": 1, "exprk3ds_cplx": 2, "exprk3_dense": 3}


class DsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("n", ctypes.c_int64 * 4)]


class Params(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("p", ctypes.c_double * 8)]


_lib = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        gp, pp = ctypes.POINTER(Grid), ctypes.POINTER(Params)
        sig = {
            "ds_phi_setup": ([gp, _vp, ctypes.c_int, ctypes.c_double, ctypes.POINTER(_vp), _vp], ctypes.c_int),
            "ds_phi_setup_ex": ([gp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.POINTER(_vp), _vp],
                                ctypes.c_int),
            "ds_phi_set_destroy": ([_vp], ctypes.c_int),
            "ds_phi_get": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp], ctypes.c_int),
            "ds_phi_get_ex": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp],
                              ctypes.c_int),
            "ds_tucker": ([gp, _vp, _vp, ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, _vp], ctypes.c_int),
            "ds_kronsum": ([_vp, ctypes.c_int, _vp, _vp, _vp], ctypes.c_int),
            "ds_tucker_static": ([gp, _vp, _vp, ctypes.POINTER(_vp), ctypes.c_int, _vp], ctypes.c_int),
            "ds_plan_create": ([gp, pp, _vp, ctypes.c_int, ctypes.POINTER(_vp)], ctypes.c_int),
            "ds_step": ([_vp, _vp, _vp], ctypes.c_int),
            "ds_integrate": ([_vp, _vp, ctypes.c_int64, _vp], ctypes.c_int),
            "ds_integrate_ckpt": ([_vp, _vp, ctypes.c_int64, ctypes.c_int64, _vp, _vp], ctypes.c_int),
            "ds_step_backward": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
            "ds_plan_sync": ([_vp, _vp, ctypes.c_int], ctypes.c_int),
            "ds_plan_kernels_per_step": ([_vp], ctypes.c_int64),
            "ds_plan_profile": ([_vp, ctypes.c_int], ctypes.c_int),
            "ds_plan_tuning": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
            "ds_plan_profile_read": ([_vp, _dp, ctypes.POINTER(ctypes.c_int64), _dp], ctypes.c_int),
            "ds_plan_set_fusion": ([_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
            "ds_plan_set_tiles": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
            "ds_plan_tuning_ex": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
            "ds_plan_set_tile_order": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
            "ds_plan_tile_order": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
            "ds_plan_streamk_times": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
            "ds_plan_fusion": ([_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float),
                                ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
            "ds_plan_profile_read_ex": ([_vp, _dp, ctypes.POINTER(ctypes.c_int64), _dp, _dp], ctypes.c_int),
            "ds_plan_profile_kinds": ([_vp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_int64), _dp, _dp],
                                      ctypes.c_int),
            "ds_plan_destroy": ([_vp], ctypes.c_int),
            "ds_batch_create": ([ctypes.c_int, gp, ctypes.POINTER(_vp), _dp, pp, ctypes.c_int,
                                 ctypes.POINTER(_vp)], ctypes.c_int),
            "ds_batch_integrate": ([_vp, ctypes.POINTER(_vp), ctypes.c_int64, _vp], ctypes.c_int),
            "ds_batch_sync": ([_vp], ctypes.c_int),
            "ds_batch_kernels_per_step": ([_vp], ctypes.c_int64),
            "ds_batch_destroy": ([_vp], ctypes.c_int),
            "ds_batch_fusion": ([_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float),
                                 ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
            "ds_batch_set_fusion": ([_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
            "ds_batch_tile_order": ([_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)],
                                    ctypes.c_int),
            "ds_last_error": ([], ctypes.c_char_p),
            "ds_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def check(status: int):
    if status != DS_OK:
        raise DsError(status, lib().ds_last_error().decode())


def make_grid(dims) -> Grid:
    g = Grid()
    g.d = len(dims)
    for q, n in enumerate(dims):
        g.n[q] = int(n)
    return g


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t) -> ctypes.c_void_p:
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


def pack_A(As) -> np.ndarray:
    """As[c][mu] as (n, n) arrays -> concatenated column-major blocks (the
    ds_phi_setup layout)."""
    return np.concatenate([np.ascontiguousarray(np.asarray(As[c][mu], dtype=np.float64).T).ravel()
                           for c in range(2) for mu in range(len(As[c]))])


class PhiSet:
    """ds_phi_set: FP64 phi-matrices of Algorithms 1/2 for both components."""

    def __init__(self, dims, As, tau: float, stream=None, scheme: str = "exprk3ds_real"):
        self.dims = tuple(int(n) for n in dims)
        self.grid = make_grid(self.dims)
        self.tau = float(tau)
        self.scheme = scheme
        host = pack_A(As)
        self._h = _vp()
        check(lib().ds_phi_setup_ex(ctypes.byref(self.grid), host.ctypes.data_as(_vp), 0, self.tau,
                                    SCHEMES[scheme], ctypes.byref(self._h), _stream_ptr(stream)))

    def get(self, c: int, slot: int, term: int, mu: int, part: int = 0) -> np.ndarray:
        """phi-matrix (part 0; real part for the complex scheme), its imaginary
        part (1) or its derivative w.r.t. a scaling of A (2), as (n, n).  The
        dense scheme has one N x N matrix per (c, slot): term = mu = 0."""
        n = int(np.prod(self.dims)) if self.scheme == "exprk3_dense" else self.dims[mu]
        out = np.empty(n * n)
        check(lib().ds_phi_get_ex(self._h, c, slot, term, mu, part, out.ctypes.data_as(_dp)))
        return out.reshape(n, n).T.copy()

    def kronsum(self, c: int, X, stream=None):
        import torch
        Y = torch.empty_like(X)
        check(lib().ds_kronsum(self._h, c, _dptr(X), _dptr(Y), _stream_ptr(stream)))
        return Y

    def close(self):
        if self._h:
            lib().ds_phi_set_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """ds_plan: an EXPRK3DS_REAL stepper bound to a phi-set and a model."""

    def __init__(self, phiset: PhiSet, model: str, p, precision: str = "f64"):
        self.phiset = phiset
        self.dims = phiset.dims
        self.precision = precision
        prm = Params()
        prm.model = MODELS[model]
        for q, v in enumerate(p):
            prm.p[q] = float(v)
        self._h = _vp()
        check(lib().ds_plan_create(ctypes.byref(phiset.grid), ctypes.byref(prm), phiset._h,
                                   PREC[precision], ctypes.byref(self._h)))

    def step(self, U, stream=None):
        check(lib().ds_step(self._h, _dptr(U), _stream_ptr(stream)))
        return U

    def step_backward(self, U, lam, dparams=None, dscale=None, stream=None):
        """dL/dU_n for lam = dL/dU_{n+1} at the step that started from U;
        adds dL/dp (3 model parameters) into dparams and dL/ds (relative
        scaling of each component's A) into dscale if given."""
        import torch
        out = torch.empty_like(lam)
        check(lib().ds_step_backward(self._h, _dptr(U), _dptr(lam), _dptr(out),
                                     _dptr(dparams) if dparams is not None else None,
                                     _dptr(dscale) if dscale is not None else None,
                                     _stream_ptr(stream)))
        return out

    def integrate(self, U, nsteps: int, stream=None):
        check(lib().ds_integrate(self._h, _dptr(U), int(nsteps), _stream_ptr(stream)))
        return U

    def integrate_ckpt(self, U, nsteps: int, ckpt_every: int, stream=None):
        """Advance U by nsteps; returns the checkpoints, a tensor of shape
        (nsteps // ckpt_every, *U.shape): entry j is the state after
        (j + 1) * ckpt_every steps."""
        import torch
        nck = int(nsteps) // int(ckpt_every) if ckpt_every > 0 else 0
        ck = torch.empty((nck,) + tuple(U.shape), dtype=torch.float64, device=U.device)
        check(lib().ds_integrate_ckpt(self._h, _dptr(U), int(nsteps), int(ckpt_every),
                                      _dptr(ck) if nck else None, _stream_ptr(stream)))
        return ck

    def fusion(self):
        """[(group, fused, ms_fused, ms_separate)] for split-BF16 plans: whether
        each group's last mode product finishes the stage in its epilogue."""
        out = []
        for g in range(3):
            fz = ctypes.c_int()
            a = ctypes.c_float()
            b = ctypes.c_float()
            check(lib().ds_plan_fusion(self._h, g, ctypes.byref(fz), ctypes.byref(a), ctypes.byref(b)))
            out.append((g, bool(fz.value), float(a.value), float(b.value)))
        return out

    def set_tiles(self, group: int, mode: int, tile_n: int, ksplit: int = 1):
        """Override the autotuner for the launch of group (0 F, 1 D2, 2 D3)
        and mode (1-based): output tile width 256 or 128, split-K factor
        (0: stream-K)."""
        check(lib().ds_plan_set_tiles(self._h, int(group), int(mode) - 1, int(tile_n), int(ksplit)))

    def set_tile_order(self, group: int, mode: int, order: int):
        """Tile order of a launch (0 or 1; see ds_plan_tile_order).  Without
        stream-K the results are the same."""
        check(lib().ds_plan_set_tile_order(self._h, int(group), int(mode) - 1, int(order)))

    def set_fusion(self, group: int, fused: bool):
        check(lib().ds_plan_set_fusion(self._h, int(group), int(bool(fused))))

    def sync(self, U=None, check_state: bool = False):
        check(lib().ds_plan_sync(self._h, _dptr(U) if U is not None else None, int(check_state)))

    def tuning(self):
        """Autotuner record: [(group, mode, ksplit, tiles, tile_n, {"<tile_n>x<split>": ms})]
        for split-BF16 plans; ksplit 0 and the keys "<tile_n>xsk" stand for stream-K,
        "order0" / "order1" are the two tile orders' times and "order": 1 marks the
        second order."""
        out = []
        for g in range(3):
            for mu in range(len(self.dims)):
                k = ctypes.c_int()
                t = ctypes.c_int64()
                tn = ctypes.c_int()
                ms = (ctypes.c_float * 16)()
                check(lib().ds_plan_tuning_ex(self._h, g, mu, ctypes.byref(k), ctypes.byref(t),
                                              ctypes.byref(tn), ms))
                sk = (ctypes.c_float * 2)()
                check(lib().ds_plan_streamk_times(self._h, g, mu, sk))
                cand = {f"{256 if i < 8 else 128}x{i % 8 + 1}": round(ms[i], 4) for i in range(16) if ms[i] > 0}
                cand.update({f"{(256, 128)[i]}xsk": round(sk[i], 4) for i in range(2) if sk[i] > 0})
                od = ctypes.c_int()
                ot = (ctypes.c_float * 2)()
                check(lib().ds_plan_tile_order(self._h, g, mu, ctypes.byref(od), ot))
                cand.update({f"order{i}": round(ot[i], 4) for i in range(2) if ot[i] > 0})
                if od.value:
                    cand["order"] = 1
                out.append((g, mu + 1, k.value, t.value, tn.value, cand))
        return out

    def profile(self, enable: bool = True):
        check(lib().ds_plan_profile(self._h, int(enable)))

    def profile_read(self, with_bytes: bool = False):
        """{kind: (ms, launches, useful_flops[, algorithmic_bytes])} for kinds
        'tc' (split-BF16 mode products), 'f64', 'pointwise' and 'fx' (FX mode
        products of f16x10 plans)."""
        ms = (ctypes.c_double * 4)()
        n = (ctypes.c_int64 * 4)()
        fl = (ctypes.c_double * 4)()
        by = (ctypes.c_double * 4)()
        check(lib().ds_plan_profile_kinds(self._h, 4, ms, n, fl, by))
        kinds = ("tc", "f64", "pointwise", "fx")
        if with_bytes:
            return {k: (ms[i], n[i], fl[i], by[i]) for i, k in enumerate(kinds)}
        return {k: (ms[i], n[i], fl[i]) for i, k in enumerate(kinds)}

    @property
    def kernels_per_step(self) -> int:
        return int(lib().ds_plan_kernels_per_step(self._h))

    def close(self):
        if self._h:
            lib().ds_plan_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tucker(X, Ls, transpose: bool = False, precision: str = "f64", stream=None):
    """Y = X x_1 L_1 ... x_d L_d on the GPU; X shape (n_d, ..., n_1) float64
    CUDA tensor; Ls[mu] (n_mu, n_mu) float64 CUDA tensors (row/col as usual)."""
    import torch
    dims = tuple(reversed(X.shape))
    g = make_grid(dims)
    cm = [L.t().contiguous() for L in Ls]   # column-major storage
    arr = (_vp * len(cm))(*[c.data_ptr() for c in cm])
    Y = torch.empty_like(X)
    check(lib().ds_tucker(ctypes.byref(g), _dptr(X), _dptr(Y), arr, int(transpose), PREC[precision],
                          _stream_ptr(stream)))
    return Y


def tucker_static(X, Ls, transpose: bool = False, stream=None):
    """FP64 Tucker operator through ds_tucker_static, the entry point that
    allocates no device memory (its intermediates live in a fixed device
    array of the library; grids of at most 1,048,576 points)."""
    import torch
    dims = tuple(reversed(X.shape))
    g = make_grid(dims)
    cm = [L.t().contiguous() for L in Ls]   # column-major storage
    arr = (_vp * len(cm))(*[c.data_ptr() for c in cm])
    Y = torch.empty_like(X)
    check(lib().ds_tucker_static(ctypes.byref(g), _dptr(X), _dptr(Y), arr, int(transpose),
                                 _stream_ptr(stream)))
    return Y


class Batch:
    """ds_batch: independent instances stepped together (one CUDA graph with
    a captured stream per instance)."""

    def __init__(self, dims_list, As_list, taus, model: str, params_list, precision: str = "bf16x6"):
        n = len(dims_list)
        grids = (Grid * n)(*[make_grid(dm) for dm in dims_list])
        self._packed = [pack_A(As) for As in As_list]
        Aptr = (_vp * n)(*[a.ctypes.data for a in self._packed])
        tau = (ctypes.c_double * n)(*[float(t) for t in taus])
        prms = (Params * n)()
        for i, pr in enumerate(params_list):
            prms[i].model = MODELS[model]
            for q, v in enumerate(pr):
                prms[i].p[q] = float(v)
        self.n = n
        self._h = _vp()
        check(lib().ds_batch_create(n, grids, Aptr, tau, prms, PREC[precision], ctypes.byref(self._h)))

    def integrate(self, Us, nsteps: int, stream=None):
        arr = (_vp * self.n)(*[_dptr(U).value for U in Us])
        check(lib().ds_batch_integrate(self._h, arr, int(nsteps), _stream_ptr(stream)))

    def sync(self):
        check(lib().ds_batch_sync(self._h))

    @property
    def kernels_per_step(self) -> int:
        return int(lib().ds_batch_kernels_per_step(self._h))

    def fusion(self):
        """[(group, fused, ms_fused, ms_separate)] of the grouped launches of the
        last captured split-BF16 graph (after an integrate)."""
        out = []
        for g in range(3):
            fz = ctypes.c_int()
            a = ctypes.c_float()
            b = ctypes.c_float()
            check(lib().ds_batch_fusion(self._h, g, ctypes.byref(fz), ctypes.byref(a), ctypes.byref(b)))
            out.append((g, bool(fz.value), float(a.value), float(b.value)))
        return out

    def tile_order(self):
        """[(group, order, ms_order0, ms_order1)] of the grouped mode-1 products
        of the last captured split-BF16 graph."""
        out = []
        for g in range(3):
            od = ctypes.c_int()
            t = (ctypes.c_float * 2)()
            check(lib().ds_batch_tile_order(self._h, g, ctypes.byref(od), t))
            out.append((g, od.value, float(t[0]), float(t[1])))
        return out

    def set_fusion(self, group: int, fused):
        """Fix group's choice: True fused epilogue, False grouped stage kernel,
        None timed (default)."""
        check(lib().ds_batch_set_fusion(self._h, int(group), -1 if fused is None else int(bool(fused))))

    def close(self):
        if self._h:
            lib().ds_batch_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
