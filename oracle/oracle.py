"""ctypes front end of the FP64 CPU oracle (ds_oracle.c).

TEST INFRASTRUCTURE: imported only by tests/, __graft_entry__.smoke() and
bench.py's cpu_baseline / reference legs.  The CUDA library never uses it.

Array conventions: tensors are numpy arrays of shape (n_d, ..., n_1)
(C-contiguous, so mode 1 is fastest, the paper's column-stacking vec);
matrices are ordinary numpy (n, n) arrays indexed [row, col] and are handed
to C in column-major order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ds_oracle.c")
_LIB = os.path.join(_HERE, "libds_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with the host gcc (OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_coeffs.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _dp, _dp]
            L.orc_coeffs.restype = ctypes.c_int
            L.orc_phi.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp]
            L.orc_phi.restype = ctypes.c_int
            L.orc_mode_product.argtypes = [ctypes.c_int, _i64p, _dp, ctypes.c_int, _dp, _dp]
            L.orc_mode_product.restype = None
            L.orc_step_dense.argtypes = [ctypes.c_int, _i64p, _dp, ctypes.c_int, _dp, ctypes.c_double,
                                         _dp, ctypes.c_int]
            L.orc_step_dense.restype = ctypes.c_int
            L.orc_set_sum_order.argtypes = [ctypes.c_int]
            L.orc_set_sum_order.restype = None
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_set_threads.restype = ctypes.c_int
            L.orc_tucker.argtypes = [ctypes.c_int, _i64p, _dp, ctypes.POINTER(_dp), _dp]
            L.orc_tucker.restype = ctypes.c_int
            L.orc_kronsum.argtypes = [ctypes.c_int, _i64p, _dp, ctypes.POINTER(_dp), _dp]
            L.orc_kronsum.restype = ctypes.c_int
            L.orc_g.argtypes = [ctypes.c_int, _dp, ctypes.c_int64, _dp, _dp]
            L.orc_g.restype = ctypes.c_int
            L.orc_phi_set_size.argtypes = [ctypes.c_int, _i64p]
            L.orc_phi_set_size.restype = ctypes.c_int64
            L.orc_phi_set.argtypes = [ctypes.c_int, _i64p, _dp, ctypes.c_double, _dp]
            L.orc_phi_set.restype = ctypes.c_int
            L.orc_step.argtypes = [ctypes.c_int, _i64p, _dp, _dp, ctypes.c_int, _dp,
                                   ctypes.c_double, _dp, ctypes.c_int]
            L.orc_step.restype = ctypes.c_int
            L.orc_coeffs_cplx.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp]
            L.orc_coeffs_cplx.restype = ctypes.c_int
            L.orc_phi_cplx.argtypes = [ctypes.c_int, _dp, ctypes.c_int, _dp]
            L.orc_phi_cplx.restype = ctypes.c_int
            L.orc_phi_set_cplx_size.argtypes = [ctypes.c_int, _i64p]
            L.orc_phi_set_cplx_size.restype = ctypes.c_int64
            L.orc_phi_set_cplx.argtypes = [ctypes.c_int, _i64p, _dp, ctypes.c_double, _dp]
            L.orc_phi_set_cplx.restype = ctypes.c_int
            L.orc_step_cplx.argtypes = [ctypes.c_int, _i64p, _dp, _dp, ctypes.c_int, _dp, ctypes.c_double,
                                        _dp, ctypes.c_int]
            L.orc_step_cplx.restype = ctypes.c_int
            L.orc_phi_set2_size.argtypes = [ctypes.c_int, _i64p]
            L.orc_phi_set2_size.restype = ctypes.c_int64
            L.orc_phi_set2.argtypes = [ctypes.c_int, _i64p, _dp, ctypes.c_double, _dp]
            L.orc_phi_set2.restype = ctypes.c_int
            L.orc_step2.argtypes = [ctypes.c_int, _i64p, _dp, _dp, ctypes.c_int, _dp, ctypes.c_double,
                                    _dp, ctypes.c_int]
            L.orc_step2.restype = ctypes.c_int
            L.orc_step_adjoint.argtypes = [ctypes.c_int, _i64p, _dp, _dp, ctypes.c_int, _dp,
                                           ctypes.c_double, _dp, _dp, _dp, _dp, _dp]
            L.orc_step_adjoint.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _dims(dims):
    arr = (ctypes.c_int64 * len(dims))(*dims)
    return arr


def _colmajor(M: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(M, dtype=np.float64).T)


MODELS = {"schnakenberg": 0, "fhn": 1, "linear": 2}


def coeffs(d: int, ell: int):
    """(ell_i[k], eta[k], alpha[k, d]) of the split for phi_ell in dimension d."""
    ell_i = (ctypes.c_int * 3)()
    eta = np.zeros(3)
    alpha = np.zeros(12)
    k = lib().orc_coeffs(d, ell, ell_i, _ptr(eta), _ptr(alpha))
    if k < 0:
        raise ValueError("bad (d, ell)")
    return list(ell_i)[:k], eta[:k].copy(), alpha.reshape(3, 4)[:k, :d].copy()


def phi(X: np.ndarray, lmax: int) -> list[np.ndarray]:
    """[phi_0(X), ..., phi_lmax(X)] of a dense square matrix."""
    n = X.shape[0]
    out = np.zeros((lmax + 1) * n * n)
    s = lib().orc_phi(n, _ptr(_colmajor(X)), lmax, _ptr(out))
    if s < 0:
        raise RuntimeError("orc_phi failed")
    return [out[k * n * n:(k + 1) * n * n].reshape(n, n).T.copy() for k in range(lmax + 1)]


def mode_product(X: np.ndarray, mu: int, L: np.ndarray) -> np.ndarray:
    """X x_mu L with mu 1-based (paper notation); X shape (n_d, ..., n_1)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    dims = tuple(reversed(X.shape))
    Y = np.empty_like(X)
    lib().orc_mode_product(len(dims), _dims(dims), _ptr(X), mu - 1, _ptr(_colmajor(L)), _ptr(Y))
    return Y


def _matlist(Ls):
    cm = [_colmajor(L) for L in Ls]
    arr = (_dp * len(cm))(*[_ptr(c) for c in cm])
    return arr, cm


def tucker(X: np.ndarray, Ls) -> np.ndarray:
    """X x_1 L_1 x_2 ... x_d L_d; Ls[0] is L_1."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    dims = tuple(reversed(X.shape))
    Y = np.empty_like(X)
    arr, keep = _matlist(Ls)
    if lib().orc_tucker(len(dims), _dims(dims), _ptr(X), arr, _ptr(Y)) != 0:
        raise RuntimeError("orc_tucker failed")
    return Y


def kronsum(X: np.ndarray, As) -> np.ndarray:
    """sum_mu X x_mu A_mu."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    dims = tuple(reversed(X.shape))
    Y = np.empty_like(X)
    arr, keep = _matlist(As)
    if lib().orc_kronsum(len(dims), _dims(dims), _ptr(X), arr, _ptr(Y)) != 0:
        raise RuntimeError("orc_kronsum failed")
    return Y


def g(model: str, p, U: np.ndarray) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    G = np.empty_like(U)
    pp = np.asarray(list(p) + [0.0] * (8 - len(p)), dtype=np.float64)
    lib().orc_g(MODELS[model], _ptr(pp), U[0].size, _ptr(U), _ptr(G))
    return G


def _pack_A(As):
    """As[c][mu] dense (n_mu, n_mu) -> concatenated column-major blocks."""
    return np.concatenate([_colmajor(As[c][mu]).ravel() for c in range(2) for mu in range(len(As[c]))])


def phi_set(dims, As, tau: float) -> np.ndarray:
    """Flat phi-set in the order [c][slot][i][mu] (see ds_oracle.c)."""
    d = len(dims)
    size = lib().orc_phi_set_size(d, _dims(dims))
    P = np.zeros(size)
    Ap = _pack_A(As)
    if lib().orc_phi_set(d, _dims(dims), _ptr(Ap), float(tau), _ptr(P)) != 0:
        raise RuntimeError("orc_phi_set failed")
    return P


def phi_set_blocks(dims, P: np.ndarray):
    """Unpack a flat phi-set into blocks[c][slot][i][mu] as (n, n) arrays."""
    d = len(dims)
    k = 2 if d == 2 else 3
    out, off = [], 0
    for c in range(2):
        cs = []
        for q in range(5):
            qs = []
            for i in range(k):
                ms = []
                for mu in range(d):
                    m = dims[mu]
                    ms.append(P[off:off + m * m].reshape(m, m).T.copy())
                    off += m * m
                qs.append(ms)
            cs.append(qs)
        out.append(cs)
    return out


def step(dims, As, P, model: str, p, tau: float, U: np.ndarray, nsteps: int = 1) -> np.ndarray:
    """nsteps EXPRK3DS_REAL steps; returns the new state (input untouched)."""
    d = len(dims)
    Uo = np.array(U, dtype=np.float64, order="C", copy=True)
    pp = np.asarray(list(p) + [0.0] * (8 - len(p)), dtype=np.float64)
    Ap = _pack_A(As)
    rc = lib().orc_step(d, _dims(dims), _ptr(Ap), _ptr(np.ascontiguousarray(P)), MODELS[model],
                        _ptr(pp), float(tau), _ptr(Uo), int(nsteps))
    if rc != 0:
        raise RuntimeError("orc_step failed")
    return Uo


def step_adjoint(dims, As, P, model: str, p, tau: float, U: np.ndarray, lam: np.ndarray,
                 with_scale: bool = False):
    """Reverse-mode adjoint of one step at U = U_n: returns (dL/dU_n, dL/dp[3])
    for lam = dL/dU_{n+1}; with_scale adds dL/ds[2], the derivative with
    respect to a relative scaling s_c of component c's matrices A_{c,mu}."""
    d = len(dims)
    Uc = np.ascontiguousarray(U, dtype=np.float64)
    lc = np.ascontiguousarray(lam, dtype=np.float64)
    out = np.zeros_like(Uc)
    dp = np.zeros(3)
    dsc = np.zeros(2)
    pp = np.asarray(list(p) + [0.0] * (8 - len(p)), dtype=np.float64)
    Ap = _pack_A(As)
    rc = lib().orc_step_adjoint(d, _dims(dims), _ptr(Ap), _ptr(np.ascontiguousarray(P)), MODELS[model],
                                _ptr(pp), float(tau), _ptr(Uc), _ptr(lc), _ptr(out), _ptr(dp),
                                _ptr(dsc) if with_scale else None)
    if rc != 0:
        raise RuntimeError("orc_step_adjoint failed")
    return (out, dp, dsc) if with_scale else (out, dp)


def phi_set2(dims, As, tau: float) -> np.ndarray:
    """ETD2RKDS phi-set: [c][l - 1][mu] blocks of phi_l(tau A_{c,mu})."""
    d = len(dims)
    P = np.zeros(lib().orc_phi_set2_size(d, _dims(dims)))
    if lib().orc_phi_set2(d, _dims(dims), _ptr(_pack_A(As)), float(tau), _ptr(P)) != 0:
        raise RuntimeError("orc_phi_set2 failed")
    return P


def step2(dims, As, P, model: str, p, tau: float, U: np.ndarray, nsteps: int = 1) -> np.ndarray:
    """nsteps ETD2RKDS steps; returns the new state."""
    d = len(dims)
    Uo = np.array(U, dtype=np.float64, order="C", copy=True)
    pp = np.asarray(list(p) + [0.0] * (8 - len(p)), dtype=np.float64)
    rc = lib().orc_step2(d, _dims(dims), _ptr(_pack_A(As)), _ptr(np.ascontiguousarray(P)), MODELS[model],
                         _ptr(pp), float(tau), _ptr(Uo), int(nsteps))
    if rc != 0:
        raise RuntimeError("orc_step2 failed")
    return Uo


def coeffs_cplx(d: int, ell: int):
    """(eta[2], alpha[2]) complex coefficients of Table 2 (same alpha in every mu)."""
    eta = np.zeros(4)
    alpha = np.zeros(4)
    if lib().orc_coeffs_cplx(d, ell, _ptr(eta), _ptr(alpha)) < 0:
        raise ValueError("bad (d, ell)")
    return eta[0::2] + 1j * eta[1::2], alpha[0::2] + 1j * alpha[1::2]


def phi_cplx(X: np.ndarray, lmax: int):
    n = X.shape[0]
    Xc = np.ascontiguousarray(np.asarray(X, dtype=np.complex128).T)
    out = np.zeros((lmax + 1) * n * n, dtype=np.complex128)
    if lib().orc_phi_cplx(n, Xc.view(np.float64).ctypes.data_as(_dp), lmax,
                          out.view(np.float64).ctypes.data_as(_dp)) < 0:
        raise RuntimeError("orc_phi_cplx failed")
    return [out[k * n * n:(k + 1) * n * n].reshape(n, n).T.copy() for k in range(lmax + 1)]


def phi_set_cplx(dims, As, tau: float) -> np.ndarray:
    """Complex phi-set [c][slot][i][mu] (complex128, flat)."""
    d = len(dims)
    P = np.zeros(lib().orc_phi_set_cplx_size(d, _dims(dims)))
    if lib().orc_phi_set_cplx(d, _dims(dims), _ptr(_pack_A(As)), float(tau), _ptr(P)) != 0:
        raise RuntimeError("orc_phi_set_cplx failed")
    return P.view(np.complex128)


def step_cplx(dims, As, P, model: str, p, tau: float, U: np.ndarray, nsteps: int = 1) -> np.ndarray:
    d = len(dims)
    Uo = np.array(U, dtype=np.float64, order="C", copy=True)
    pp = np.asarray(list(p) + [0.0] * (8 - len(p)), dtype=np.float64)
    Pf = np.ascontiguousarray(P).view(np.float64)
    rc = lib().orc_step_cplx(d, _dims(dims), _ptr(_pack_A(As)), _ptr(Pf), MODELS[model], _ptr(pp),
                             float(tau), _ptr(Uo), int(nsteps))
    if rc != 0:
        raise RuntimeError("orc_step_cplx failed")
    return Uo


def set_sum_order(reverse: bool) -> None:
    """Mode-product summation order of later calls: j ascending (default) or
    descending.  The difference of the two runs is the FP64 rounding floor."""
    lib().orc_set_sum_order(1 if reverse else 0)


def set_threads(n: int = 0) -> int:
    """OpenMP threads of later calls (n <= 0 leaves it); returns the count in use."""
    return int(lib().orc_set_threads(int(n)))


def noise_floor(dims, As, model, p, tau, U0, m):
    """max over components of the relative max-norm difference between m steps
    with ascending and with descending summation in every mode product."""
    P = phi_set(dims, As, tau)
    a = step(dims, As, P, model, p, tau, U0, m)
    set_sum_order(True)
    try:
        P2 = phi_set(dims, As, tau)
        b = step(dims, As, P2, model, p, tau, U0, m)
    finally:
        set_sum_order(False)
    return max(float(np.abs(a[c] - b[c]).max() / np.abs(a[c]).max()) for c in range(2)), a


def step_dense(dims, As, model, p, tau, U0, nsteps):
    """nsteps of the unsplit EXPRK3 with dense phi(c tau K) (orc_step_dense);
    small grids only."""
    d = len(dims)
    A = _pack_A(As)
    U = np.array(U0, dtype=np.float64, order="C", copy=True)
    pp = np.asarray(list(p) + [0.0] * (8 - len(p)), dtype=np.float64)
    rc = lib().orc_step_dense(d, _dims(dims), _ptr(A), MODELS[model], _ptr(pp), float(tau), _ptr(U), int(nsteps))
    if rc != 0:
        raise RuntimeError("orc_step_dense failed")
    return U
