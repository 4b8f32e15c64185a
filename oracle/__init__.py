"""Oracle for the replica-parallel Metropolis sweep with parallel tempering.

TEST INFRASTRUCTURE ONLY.  A plain, slow CPU restatement (``ising_oracle.c``)
of Figure 1 of Dickson, Karimi & Hamze (arXiv:1004.0024) with the Figure 6
neighbour update, MT19937 (the paper's ref [9]), Philox4x32-10 and standard
replica exchange.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s cpu_baseline / reference leg may import this package; the
library under ``paper_1004_0024_gb300`` never does.

The C source is compiled with gcc into ``oracle/_build/`` on first use (or by
``__graft_entry__.build()``).  This wrapper only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = [os.path.join(_HERE, "ising_oracle.c"), os.path.join(_HERE, "mlp_oracle.c")]
_LIB_PATH = os.path.join(_BUILD, "libising_oracle.so")
_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i8p = ctypes.POINTER(ctypes.c_int8)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain -O2, no intrinsics)."""
    srcs = [s for s in _SRC if os.path.exists(s)]
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in srcs)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, *srcs,
               "-lm", "-lpthread"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_mt_stream.argtypes = [ctypes.c_uint32, ctypes.c_int64, _u32p]
        lib.orc_philox.argtypes = [_u32p, _u32p, _u32p]
        lib.orc_flip_threshold.argtypes = [ctypes.c_double, ctypes.c_int64]
        lib.orc_flip_threshold.restype = ctypes.c_uint32
        lib.orc_swap_threshold.argtypes = [ctypes.c_double, ctypes.c_int64]
        lib.orc_swap_threshold.restype = ctypes.c_uint32
        lib.orc_exp_approx.argtypes = [ctypes.c_float, ctypes.c_int32]
        lib.orc_exp_approx.restype = ctypes.c_float
        lib.orc_flip_threshold_mode.argtypes = [ctypes.c_double, ctypes.c_int64, ctypes.c_int32]
        lib.orc_flip_threshold_mode.restype = ctypes.c_uint32
        lib.orc_sim_set_acceptance.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        lib.orc_sim_set_acceptance.restype = None
        lib.orc_fields.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, _i32p, _i8p, _i64p]
        lib.orc_energy.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, _i32p, _i8p]
        lib.orc_energy.restype = ctypes.c_int64
        lib.orc_sim_create.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, _i32p,
                                       ctypes.c_int32, ctypes.c_int32, _f64p,
                                       ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int32,
                                       ctypes.c_int32]
        lib.orc_sim_create.restype = ctypes.c_void_p
        lib.orc_sim_sweep.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        lib.orc_sim_pt.argtypes = [ctypes.c_void_p]
        lib.orc_sim_run.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32]
        lib.orc_sim_read.argtypes = [ctypes.c_void_p, _i8p, _i64p, _i64p, _i32p, _u64p, _u64p]
        lib.orc_sim_threads.argtypes = [ctypes.c_void_p]
        lib.orc_sim_threads.restype = ctypes.c_int32
        lib.orc_sim_destroy.argtypes = [ctypes.c_void_p]
        lib.orc_sim_set_spins.argtypes = [ctypes.c_void_p, ctypes.c_int32, _i8p]
        lib.orc_exp_det.argtypes = [ctypes.c_double]
        lib.orc_exp_det.restype = ctypes.c_double
        lib.orc_trotter_flip_threshold.argtypes = [ctypes.c_double, ctypes.c_double,
                                                   ctypes.c_int64, ctypes.c_int64]
        lib.orc_trotter_flip_threshold.restype = ctypes.c_uint32
        lib.orc_trotter_swap_threshold.argtypes = [ctypes.c_double, ctypes.c_double,
                                                   ctypes.c_int64, ctypes.c_int64]
        lib.orc_trotter_swap_threshold.restype = ctypes.c_uint32
        lib.orc_sim_set_trotter.argtypes = [ctypes.c_void_p, _f64p]
        lib.orc_sim_set_trotter.restype = None
        lib.orc_sim_read_trotter.argtypes = [ctypes.c_void_p, _i64p]
        lib.orc_sim_read_trotter.restype = None
        if hasattr(lib, "orc_mlp_forward"):
            _bind_mlp(lib)
        _lib = lib
        return lib


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ----------------------------------------------------------------- RNGs
def mt_stream(seed: int, n: int) -> np.ndarray:
    """First n outputs of MT19937 seeded with init_genrand(seed)."""
    lib = _load()
    out = np.empty(n, dtype=np.uint32)
    lib.orc_mt_stream(ctypes.c_uint32(seed & 0xFFFFFFFF), n, _ptr(out, _u32p))
    return out


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 128-bit counter under one 64-bit key."""
    lib = _load()
    c = _c(np.asarray(ctr, dtype=np.uint64) & 0xFFFFFFFF, np.uint32)
    k = _c(np.asarray(key, dtype=np.uint64) & 0xFFFFFFFF, np.uint32)
    out = np.empty(4, dtype=np.uint32)
    lib.orc_philox(_ptr(c, _u32p), _ptr(k, _u32p), _ptr(out, _u32p))
    return out


def flip_threshold(beta: float, k: int) -> int:
    """floor(2^32 exp(-2 beta k)), k >= 1."""
    return int(_load().orc_flip_threshold(beta, k))


ACCEPT_MODES = {"exact": 0, "fast": 1, "accurate": 2}


def exp_approx(x: float, accurate: bool = False) -> float:
    """The paper's fast (or accurate) approximation of e^x (section 2.4)."""
    return float(_load().orc_exp_approx(x, 1 if accurate else 0))


def flip_threshold_mode(beta: float, k: int, mode: str = "exact") -> int:
    """floor(2^32 min(1, e(-2 beta k))) with the mode's exponential."""
    return int(_load().orc_flip_threshold_mode(beta, k, ACCEPT_MODES[mode]))


def swap_threshold(dbeta: float, d: int) -> int:
    """floor(2^32 exp(-dbeta d)), d >= 1."""
    return int(_load().orc_swap_threshold(dbeta, d))


def exp_det(x: float) -> float:
    """Deterministic e^x (Cody-Waite reduction, degree-13 Taylor, unfused FP64)."""
    return float(_load().orc_exp_det(x))


def trotter_flip_threshold(beta: float, K: float, ks: int, kt: int) -> int:
    """Split couplings: floor(2^32 exp(-z)), z = 2 (beta ks + K kt) > 0."""
    return int(_load().orc_trotter_flip_threshold(beta, K, ks, kt))


def trotter_swap_threshold(dbeta: float, dK: float, dE: int, dC: int) -> int:
    """Split couplings: floor(2^32 exp_det(-z)), z = dbeta dE + dK dC > 0."""
    return int(_load().orc_trotter_swap_threshold(dbeta, dK, dE, dC))


# ----------------------------------------------------------- graph helpers
def fields(g, s: np.ndarray) -> np.ndarray:
    lib = _load()
    rp, col, J, h = (_c(g.row_ptr, np.int32), _c(g.col, np.int32), _c(g.J, np.int32),
                     _c(g.h, np.int32))
    s = _c(s, np.int8)
    out = np.empty(g.n, dtype=np.int64)
    lib.orc_fields(g.n, _ptr(rp, _i32p), _ptr(col, _i32p), _ptr(J, _i32p), _ptr(h, _i32p),
                   _ptr(s, _i8p), _ptr(out, _i64p))
    return out


def energy(g, s: np.ndarray) -> int:
    lib = _load()
    rp, col, J, h = (_c(g.row_ptr, np.int32), _c(g.col, np.int32), _c(g.J, np.int32),
                     _c(g.h, np.int32))
    s = _c(s, np.int8)
    return int(lib.orc_energy(g.n, _ptr(rp, _i32p), _ptr(col, _i32p), _ptr(J, _i32p),
                              _ptr(h, _i32p), _ptr(s, _i8p)))


class Sim:
    """Oracle simulation of one instance: R replicas of graph ``g``.

    ``g`` is any object with ``n, row_ptr, col, J, h`` (CSR, both directions
    of every edge) and optionally ``slice_size`` (the Philox counter map's S;
    the whole graph when absent).
    """

    def __init__(self, g, betas, seed: int, rng: str = "mt19937", instance: int = 0,
                 threads: int = 0, accept: str = "exact"):
        lib = _load()
        self._lib = lib
        self.n = int(g.n)
        self.betas = _c(betas, np.float64)
        self.R = int(self.betas.size)
        self._keep = [_c(g.row_ptr, np.int32), _c(g.col, np.int32), _c(g.J, np.int32),
                      _c(g.h, np.int32)]
        if self._keep[1].size == 0:
            self._keep[1] = np.zeros(1, np.int32)
            self._keep[2] = np.zeros(1, np.int32)
        if self._keep[3].size == 0:
            self._keep[3] = np.zeros(1, np.int32)
        rp, col, J, h = self._keep
        slice_size = int(getattr(g, "slice_size", 0) or self.n)
        mode = {"mt19937": 0, "philox": 1}[rng]
        self._h = lib.orc_sim_create(self.n, _ptr(rp, _i32p), _ptr(col, _i32p), _ptr(J, _i32p),
                                     _ptr(h, _i32p), slice_size, self.R,
                                     _ptr(self.betas, _f64p), ctypes.c_uint32(seed & 0xFFFFFFFF),
                                     ctypes.c_uint32(instance & 0xFFFFFFFF), mode, threads)
        self.threads = int(lib.orc_sim_threads(self._h))
        if accept != "exact":
            lib.orc_sim_set_acceptance(self._h, ACCEPT_MODES[accept])

    def sweep(self, n: int = 1):
        self._lib.orc_sim_sweep(self._h, n)

    def pt_swap(self):
        self._lib.orc_sim_pt(self._h)

    def run(self, n: int, swap_every: int = 1):
        self._lib.orc_sim_run(self._h, n, swap_every)

    def read(self):
        R, n = self.R, self.n
        spins = np.empty((R, n), dtype=np.int8)
        fields_ = np.empty((R, n), dtype=np.int64)
        E = np.empty(R, dtype=np.int64)
        temp = np.empty(R, dtype=np.int32)
        counters = np.empty(2, dtype=np.uint64)
        acc = np.zeros(max(R - 1, 1), dtype=np.uint64)
        self._lib.orc_sim_read(self._h, _ptr(spins, _i8p), _ptr(fields_, _i64p), _ptr(E, _i64p),
                               _ptr(temp, _i32p), _ptr(counters, _u64p), _ptr(acc, _u64p))
        return dict(spins=spins, fields=fields_, energy=E, temp_of_slot=temp,
                    sweeps=int(counters[0]), passes=int(counters[1]), swap_acc=acc[:max(R - 1, 0)])

    def set_trotter(self, K):
        """Split couplings: temperature k weights exp(-beta_k E_space - K_k C);
        fields and energies become the spatial ones (rebuilt from the spins)."""
        self._K = _c(K, np.float64)
        assert self._K.size == self.R
        self._lib.orc_sim_set_trotter(self._h, _ptr(self._K, _f64p))

    def read_trotter(self) -> np.ndarray:
        """C = -sum over Trotter pairs of s s', per slot (split couplings)."""
        out = np.empty(self.R, dtype=np.int64)
        self._lib.orc_sim_read_trotter(self._h, _ptr(out, _i64p))
        return out

    def set_spins(self, spins: np.ndarray):
        """Set every slot's spins ([R, n] or [n] broadcast); fields/energy recomputed."""
        sp = np.broadcast_to(np.asarray(spins, dtype=np.int8), (self.R, self.n))
        for r in range(self.R):
            row = np.ascontiguousarray(sp[r])
            self._lib.orc_sim_set_spins(self._h, r, _ptr(row, _i8p))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_sim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _bind_mlp(lib):
    d = ctypes.c_int
    lib.orc_mlp_forward.argtypes = [d, d, d, d] + [_f64p] * 10
    lib.orc_mlp_backward.argtypes = [d, d, d, d] + [_f64p] * 15
    lib.orc_mlp_backward.restype = ctypes.c_double
    lib.orc_column_energy.argtypes = [d, d, _i32p, _i8p]
    lib.orc_column_energy.restype = ctypes.c_int64
    lib.orc_log_q.argtypes = [d, _f64p, _i8p]
    lib.orc_log_q.restype = ctypes.c_double
    lib.orc_column_log_accept.argtypes = [d, d, _i32p, _i8p, _i8p, _f64p, ctypes.c_double, _i64p]
    lib.orc_column_log_accept.restype = ctypes.c_double
    lib.orc_column_log_accept_mix.argtypes = [d, d, _i32p, _i8p, _i8p, _f64p, ctypes.c_double, _i64p]
    lib.orc_column_log_accept_mix.restype = ctypes.c_double
    lib.orc_log_q_mix.argtypes = [d, _f64p, _i8p]
    lib.orc_log_q_mix.restype = ctypes.c_double


# --------------------------------------------------- learned column proposal
def mlp_forward(X, W1, b1, W2, b2, W3, b3):
    """FP64 forward: returns (H1, H2, logits) for X [B, IN]."""
    lib = _load()
    X = _c(X, np.float64)
    B, IN = X.shape
    H, OUT = W1.shape[0], W3.shape[0]
    ws = [_c(w, np.float64) for w in (W1, b1, W2, b2, W3, b3)]
    H1 = np.empty((B, H)); H2 = np.empty((B, H)); L = np.empty((B, OUT))
    lib.orc_mlp_forward(B, IN, H, OUT, _ptr(X, _f64p), *[_ptr(w, _f64p) for w in ws],
                        _ptr(H1, _f64p), _ptr(H2, _f64p), _ptr(L, _f64p))
    return H1, H2, L


def mlp_backward(X, Y, W1, b1, W2, b2, W3, b3):
    """FP64 mean BCE-with-logits loss and gradients (dW1, db1, dW2, db2, dW3, db3)."""
    lib = _load()
    X = _c(X, np.float64)
    Y = _c(Y, np.float64)
    B, IN = X.shape
    H, OUT = W1.shape[0], W3.shape[0]
    ws = [_c(w, np.float64) for w in (W1, b1, W2, b2, W3, b3)]
    grads = [np.empty_like(w) for w in ws]
    scratch = np.empty(B * (2 * H + OUT) + OUT + 2 * H)
    loss = lib.orc_mlp_backward(B, IN, H, OUT, _ptr(X, _f64p), _ptr(Y, _f64p),
                                *[_ptr(w, _f64p) for w in ws],
                                *[_ptr(g, _f64p) for g in grads], _ptr(scratch, _f64p))
    return float(loss), grads


def column_energy(M, jtau, phi, s):
    lib = _load()
    phi = _c(phi, np.int32); s = _c(s, np.int8)
    return int(lib.orc_column_energy(M, jtau, _ptr(phi, _i32p), _ptr(s, _i8p)))


def log_q(logits, s):
    lib = _load()
    lg = _c(logits, np.float64); s = _c(s, np.int8)
    return float(lib.orc_log_q(lg.size, _ptr(lg, _f64p), _ptr(s, _i8p)))


def log_q_mix(logits, s):
    """log of the flip-symmetric mixture (q(s) + q(-s)) / 2."""
    lib = _load()
    lg = _c(logits, np.float64); s = _c(s, np.int8)
    return float(lib.orc_log_q_mix(lg.size, _ptr(lg, _f64p), _ptr(s, _i8p)))


def column_log_accept(M, jtau, phi, s, s2, logits, beta, mixture=False):
    """(log A, dE) of the column move s -> s2 under the given logits (with
    mixture: the flip-symmetric mixture proposal)."""
    lib = _load()
    phi = _c(phi, np.int32); s = _c(s, np.int8); s2 = _c(s2, np.int8)
    lg = _c(logits, np.float64)
    dE = ctypes.c_int64(0)
    fn = lib.orc_column_log_accept_mix if mixture else lib.orc_column_log_accept
    la = fn(M, jtau, _ptr(phi, _i32p), _ptr(s, _i8p), _ptr(s2, _i8p), _ptr(lg, _f64p), float(beta),
            ctypes.byref(dE))
    return float(la), int(dE.value)
