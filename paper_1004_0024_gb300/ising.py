"""ctypes binding of the C ABI in ``include/ising_gb300.h``.

Argument marshalling only: every step of the sampler runs in the CUDA library
``libising_gb300.so`` built in-tree by ``paper_1004_0024_gb300/build.py``.
Importing this module loads that library and raises ``ImportError`` when it
has not been built; there is no CPU fallback.

The functions keep the C names (``ising_create``, ``ising_replicas_init``,
``ising_sweep``, ``ising_pt_swap``, ``ising_run``, ``ising_read_state`` ...);
:class:`Ising` bundles one handle with numpy-friendly methods.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libising_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")

_lib = ctypes.CDLL(LIB_PATH)

ISING_OK = 0
ERRORS = {
    -1: "INVALID_ARG", -2: "ASYMMETRIC_J", -3: "SELF_LOOP_OR_DUP", -4: "FIELD_OVERFLOW",
    -5: "NOT_INITIALISED", -6: "OOM", -7: "CUDA", -8: "TIMEOUT", -9: "UNSUPPORTED",
}
RNG = {"mt19937": 0, "philox": 1}

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i8p = ctypes.POINTER(ctypes.c_int8)
_f64p = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


class IsingInfo(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int32) for name in (
        "n", "slices", "slice_size", "levels", "slice_depth", "replicas",
        "replicas_per_block", "threads_per_block", "blocks", "smem_bytes", "persistent_ok",
        "field_bits", "rng_mode", "kmax", "fast_kernel")]


class IsingStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("sweep_launches", ctypes.c_int64),
                ("timed_launches", ctypes.c_int64), ("kernel_ms", ctypes.c_double)]


class IsingInstance(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("row_ptr", _i32p), ("col", _i32p), ("J", _i32p),
                ("h", _i32p), ("n_slices", ctypes.c_int32), ("replicas", ctypes.c_int32),
                ("betas", _f64p), ("seed", ctypes.c_uint32)]


class LearnedTrace(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64), ("replica", _i32p), ("site", _i32p), ("phi", _i32p),
                ("logits", ctypes.POINTER(ctypes.c_float)), ("old_bits", ctypes.POINTER(ctypes.c_uint32)),
                ("prop_bits", ctypes.POINTER(ctypes.c_uint32)), ("accepted", ctypes.POINTER(ctypes.c_uint8))]


class MlpStats(ctypes.Structure):
    _fields_ = [("network_launches", ctypes.c_int64), ("network_rows", ctypes.c_int64),
                ("network_ms", ctypes.c_double)]


class LearnedStats(ctypes.Structure):
    _fields_ = [("proposed", ctypes.c_uint64), ("accepted", ctypes.c_uint64), ("changed", ctypes.c_uint64),
                ("exact_decisions", ctypes.c_uint64)]


_f32p = ctypes.POINTER(ctypes.c_float)
_u32p = ctypes.POINTER(ctypes.c_uint32)
LEARNED_FP64_ONLY = 1
LEARNED_MIXTURE = 2
COLLECT_ORIENTED = 1

_SIGS = {
    "ising_last_error": ([], ctypes.c_char_p),
    "ising_create": ([ctypes.c_int32, _i32p, _i32p, _i32p, _i32p, ctypes.c_int32, ctypes.c_uint32,
                      ctypes.POINTER(_vp)], ctypes.c_int32),
    "ising_set_stream": ([_vp, _vp], ctypes.c_int32),
    "ising_replicas_init": ([_vp, ctypes.c_int32, _f64p, ctypes.c_uint32, ctypes.c_int32,
                             ctypes.c_int32], ctypes.c_int32),
    "ising_sweep": ([_vp, ctypes.c_int64], ctypes.c_int32),
    "ising_pt_swap": ([_vp], ctypes.c_int32),
    "ising_run": ([_vp, ctypes.c_int64, ctypes.c_int32], ctypes.c_int32),
    "ising_read_state": ([_vp, _i8p, _i32p, _i64p, _i32p, _u64p], ctypes.c_int32),
    "ising_read_swap_stats": ([_vp, _u64p], ctypes.c_int32),
    "ising_save": ([_vp, _vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int32),
    "ising_load": ([_vp, _vp, ctypes.c_size_t], ctypes.c_int32),
    "ising_set_seed": ([_vp, ctypes.c_uint32], ctypes.c_int32),
    "ising_get_info": ([_vp, ctypes.POINTER(IsingInfo)], ctypes.c_int32),
    "ising_set_launch": ([_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32], ctypes.c_int32),
    "ising_run_noalloc": ([_vp, ctypes.c_int64, ctypes.c_int32], ctypes.c_int32),
    "ising_set_profiling": ([_vp, ctypes.c_int32], ctypes.c_int32),
    "ising_get_stats": ([_vp, ctypes.POINTER(IsingStats)], ctypes.c_int32),
    "ising_destroy": ([_vp], ctypes.c_int32),
    "ising_batch_create": ([ctypes.c_int32, ctypes.POINTER(IsingInstance), ctypes.c_int32,
                            ctypes.c_int32, ctypes.c_uint32, ctypes.POINTER(_vp)], ctypes.c_int32),
    "ising_batch_set_stream": ([_vp, _vp], ctypes.c_int32),
    "ising_batch_autotune": ([_vp, ctypes.c_uint32], ctypes.c_int32),
    "ising_batch_run": ([_vp, ctypes.c_int64, ctypes.c_int32], ctypes.c_int32),
    "ising_batch_read_state": ([_vp, ctypes.c_int32, _i8p, _i32p, _i64p, _i32p, _u64p],
                               ctypes.c_int32),
    "ising_batch_read_swap_stats": ([_vp, ctypes.c_int32, _u64p], ctypes.c_int32),
    "ising_batch_get_info": ([_vp, ctypes.c_int32, ctypes.POINTER(IsingInfo),
                              ctypes.POINTER(ctypes.c_int32)], ctypes.c_int32),
    "ising_batch_destroy": ([_vp], ctypes.c_int32),
    "ising_tc_gemm": ([ctypes.c_int32] * 3 + [_vp, ctypes.c_int32, _vp, ctypes.c_int32, _f32p, _vp,
                                             ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_int32,
                                             ctypes.c_int32, _vp], ctypes.c_int32),
    "ising_mlp_create": ([ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64, ctypes.POINTER(_vp)],
                         ctypes.c_int32),
    "ising_mlp_set_stream": ([_vp, _vp], ctypes.c_int32),
    "ising_mlp_n_params": ([_vp], ctypes.c_int64),
    "ising_mlp_get_params": ([_vp, _f32p], ctypes.c_int32),
    "ising_mlp_set_params": ([_vp, _f32p], ctypes.c_int32),
    "ising_mlp_forward": ([_vp, ctypes.c_int32, _f32p, _f32p], ctypes.c_int32),
    "ising_mlp_grad": ([_vp, ctypes.c_int32, _f32p, _u32p, _f32p, _f32p], ctypes.c_int32),
    "ising_mlp_collect": ([_vp, _vp], ctypes.c_int32),
    "ising_mlp_collect_flags": ([_vp, _vp, ctypes.c_uint32], ctypes.c_int32),
    "ising_mlp_get_records": ([_vp, ctypes.c_int64, ctypes.c_int64, _f32p, _u32p], ctypes.c_int32),
    "ising_mlp_n_records": ([_vp], ctypes.c_int64),
    "ising_mlp_clear_records": ([_vp], ctypes.c_int32),
    "ising_mlp_train": ([_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, _f32p], ctypes.c_int32),
    "ising_learned_pass": ([_vp, _vp, ctypes.c_uint32, ctypes.POINTER(LearnedStats),
                            ctypes.POINTER(LearnedTrace)], ctypes.c_int32),
    "ising_mlp_destroy": ([_vp], ctypes.c_int32),
    "ising_mlp_set_profiling": ([_vp, ctypes.c_int32], ctypes.c_int32),
    "ising_mlp_get_stats": ([_vp, ctypes.POINTER(MlpStats)], ctypes.c_int32),
    "ising_read_observables": ([_vp, _i64p, _i64p], ctypes.c_int32),
    "ising_set_alloc_cap": ([ctypes.c_uint64], ctypes.c_int32),
    "ising_release_cached_memory": ([], ctypes.c_int32),
    "ising_set_acceptance": ([_vp, ctypes.c_int32], ctypes.c_int32),
    "ising_set_trotter": ([_vp, _f64p], ctypes.c_int32),
    "ising_read_trotter": ([_vp, _i64p], ctypes.c_int32),
    "ising_split_flip_table": ([ctypes.c_int32, _f64p, _f64p, ctypes.c_int32, _u32p], ctypes.c_int32),
    "ising_split_exp": ([ctypes.c_double], ctypes.c_double),
    "ising_swap_thresholds": ([ctypes.c_int32, _f64p, ctypes.c_int64, _u32p, ctypes.c_int64, _i64p, _i32p,
                               _i64p, _i32p], ctypes.c_int32),
    "ising_split_swap_threshold": ([ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_int64],
                                   ctypes.c_uint32),
    "ising_selftest_wait": ([ctypes.c_int32, _vp], ctypes.c_int32),
    "ising_measure_latencies": ([_f64p], ctypes.c_int32),
}
for _name, (_args, _res) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res


class IsingError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


def _check(rc: int):
    if rc != ISING_OK:
        raise IsingError(rc, _lib.ising_last_error().decode(errors="replace"))


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a, t):
    return a.ctypes.data_as(t)


# ------------------------------------------------------------ C-named calls
def ising_last_error() -> str:
    return _lib.ising_last_error().decode(errors="replace")


def ising_create(n, row_ptr, col, J, h, n_slices=1, flags=0):
    rp, c, j, hh = _arr(row_ptr, np.int32), _arr(col, np.int32), _arr(J, np.int32), _arr(h, np.int32)
    if c.size == 0:
        c = np.zeros(1, np.int32)
        j = np.zeros(1, np.int32)
    out = _vp()
    _check(_lib.ising_create(int(n), _p(rp, _i32p), _p(c, _i32p), _p(j, _i32p), _p(hh, _i32p),
                             int(n_slices), int(flags), ctypes.byref(out)))
    return out


def ising_set_stream(h, stream):
    """`stream`: a cudaStream_t as int (e.g. torch.cuda.current_stream().cuda_stream) or None."""
    _check(_lib.ising_set_stream(h, _vp(int(stream) if stream else None)))


def ising_replicas_init(h, R, betas, seed, rng_mode=0, field_bits=32):
    b = _arr(betas, np.float64)
    if isinstance(rng_mode, str):
        rng_mode = RNG[rng_mode]
    _check(_lib.ising_replicas_init(h, int(R), _p(b, _f64p), int(seed) & 0xFFFFFFFF, int(rng_mode),
                                    int(field_bits)))


def ising_sweep(h, n):
    _check(_lib.ising_sweep(h, int(n)))


def ising_pt_swap(h):
    _check(_lib.ising_pt_swap(h))


def ising_run(h, n, swap_every=1):
    _check(_lib.ising_run(h, int(n), int(swap_every)))


def ising_run_noalloc(h, n, swap_every=1):
    """ising_run without any device allocation (Philox handles only)."""
    _check(_lib.ising_run_noalloc(h, int(n), int(swap_every)))


def ising_read_state(h, R, n):
    spins = np.empty((R, n), dtype=np.int8)
    fields = np.empty((R, n), dtype=np.int32)
    E = np.empty(R, dtype=np.int64)
    temp = np.empty(R, dtype=np.int32)
    cnt = np.empty(2, dtype=np.uint64)
    _check(_lib.ising_read_state(h, _p(spins, _i8p), _p(fields, _i32p), _p(E, _i64p),
                                 _p(temp, _i32p), _p(cnt, _u64p)))
    return dict(spins=spins, fields=fields, energy=E, temp_of_slot=temp, sweeps=int(cnt[0]),
                passes=int(cnt[1]))


def ising_read_swap_stats(h, R):
    acc = np.zeros(max(R - 1, 1), dtype=np.uint64)
    _check(_lib.ising_read_swap_stats(h, _p(acc, _u64p)))
    return acc[:max(R - 1, 0)]


def ising_set_trotter(h, K):
    K = np.ascontiguousarray(K, dtype=np.float64)
    _check(_lib.ising_set_trotter(h, _p(K, _f64p)))


def ising_read_trotter(h, R):
    C = np.empty(R, dtype=np.int64)
    _check(_lib.ising_read_trotter(h, _p(C, _i64p)))
    return C


def split_flip_table(betas, K, ks: int) -> np.ndarray:
    """The flip tables ising_set_trotter builds, as [R][2 ks + 1][3] (k_s, k_tau / 2 + 1)."""
    betas = np.ascontiguousarray(betas, dtype=np.float64)
    K = np.ascontiguousarray(K, dtype=np.float64)
    out = np.empty((betas.size, 2 * ks + 1, 3), dtype=np.uint32)
    _check(_lib.ising_split_flip_table(betas.size, _p(betas, _f64p), _p(K, _f64p), ks, _p(out, _u32p)))
    return out


def swap_thresholds(betas, dmax: int):
    """The PT swap tables of a ladder as ising_replicas_init builds them:
    (thr, off, len, pt_ok), pair k's S_k(d) = thr[off[k] + d] for 1 <= d < len[k]."""
    betas = np.ascontiguousarray(betas, dtype=np.float64)
    R = betas.size
    n = ctypes.c_int64(0)
    ok = ctypes.c_int32(0)
    off = np.zeros(max(R - 1, 1), dtype=np.int64)
    ln = np.zeros(max(R - 1, 1), dtype=np.int32)
    _check(_lib.ising_swap_thresholds(R, _p(betas, _f64p), int(dmax), None, 0, _p(off, _i64p), _p(ln, _i32p),
                                      ctypes.byref(n), ctypes.byref(ok)))
    thr = np.zeros(max(n.value, 1), dtype=np.uint32)
    _check(_lib.ising_swap_thresholds(R, _p(betas, _f64p), int(dmax), _p(thr, _u32p), thr.size, None, None,
                                      ctypes.byref(n), None))
    return thr[:n.value], off[:max(R - 1, 0)], ln[:max(R - 1, 0)], bool(ok.value)


def split_exp(x: float) -> float:
    """The device's fixed FP64 exponential of the split-coupling swap rule (host build)."""
    return float(_lib.ising_split_exp(float(x)))


def split_swap_threshold(dbeta: float, dK: float, dE: int, dC: int) -> int:
    return int(_lib.ising_split_swap_threshold(dbeta, dK, int(dE), int(dC)))


def ising_save(h) -> bytes:
    size = ctypes.c_size_t(0)
    _check(_lib.ising_save(h, None, 0, ctypes.byref(size)))
    buf = ctypes.create_string_buffer(size.value)
    _check(_lib.ising_save(h, ctypes.cast(buf, _vp), size.value, ctypes.byref(size)))
    return buf.raw[: size.value]


def ising_load(h, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(_lib.ising_load(h, ctypes.cast(buf, _vp), len(blob)))


def ising_set_seed(h, seed):
    _check(_lib.ising_set_seed(h, int(seed) & 0xFFFFFFFF))


def ising_get_info(h) -> dict:
    info = IsingInfo()
    _check(_lib.ising_get_info(h, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in IsingInfo._fields_}


LAUNCH_PERSISTENT = 1
LAUNCH_GENERIC = 2
LAUNCH_NO_LEAN = 4
LAUNCH_TRACK = 8
LAUNCH_NO_PACKED = 16
BATCH_PER_SWEEP = 1


def ising_set_launch(h, replicas_per_block=0, threads_per_block=0, launch_flags=LAUNCH_PERSISTENT):
    _check(_lib.ising_set_launch(h, int(replicas_per_block), int(threads_per_block),
                                 int(launch_flags)))


def ising_set_profiling(h, on=True):
    _check(_lib.ising_set_profiling(h, 1 if on else 0))


def ising_get_stats(h) -> dict:
    st = IsingStats()
    _check(_lib.ising_get_stats(h, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in IsingStats._fields_}


def ising_set_alloc_cap(nbytes):
    """Cap every later device allocation of the library at `nbytes` (0: none)."""
    _check(_lib.ising_set_alloc_cap(int(nbytes)))


ACCEPT_MODES = {"exact": 0, "fast": 1, "accurate": 2}  # ISING_ACCEPT_*


def ising_release_cached_memory():
    """Free the MT19937 word buffers that destroyed handles left for reuse."""
    _check(_lib.ising_release_cached_memory())


def ising_measure_latencies() -> dict:
    """Cycles per dependent operation on the current GPU (shared load,
    integer multiply-add, warp shuffle, 8-warp block barrier)."""
    out = np.zeros(4, dtype=np.float64)
    _check(_lib.ising_measure_latencies(_p(out, _f64p)))
    return dict(zip(("shared_load", "int_mad", "shuffle", "barrier_8_warps"), (float(x) for x in out)))


def ising_selftest_wait(kind, stream=None):
    """Run a kernel whose bounded wait runs out; returns the status code."""
    return int(_lib.ising_selftest_wait(int(kind), _vp(stream) if stream else None))


def ising_destroy(h):
    if h:
        _check(_lib.ising_destroy(h))


# ------------------------------------------------------------------ wrapper
class Ising:
    """One model with its replicas: ``Ising(graph, betas, seed, rng, field_bits)``.

    ``graph`` has ``n, row_ptr, col, J, h`` and ``n_slices`` (see
    ``paper_1004_0024_gb300.workloads.Graph``).
    """

    def __init__(self, graph, betas=None, seed=5489, rng="mt19937", field_bits=32, stream=None,
                 accept="exact"):
        self.n = int(graph.n)
        self.h = ising_create(graph.n, graph.row_ptr, graph.col, graph.J, graph.h,
                              getattr(graph, "n_slices", 1))
        if stream is not None:
            ising_set_stream(self.h, stream)
        if accept != "exact":
            self.set_acceptance(accept)
        self.R = 0
        if betas is not None:
            self.replicas_init(betas, seed, rng, field_bits)

    def replicas_init(self, betas, seed=5489, rng="mt19937", field_bits=32):
        betas = np.asarray(betas, dtype=np.float64)
        ising_replicas_init(self.h, betas.size, betas, seed, rng, field_bits)
        self.R = int(betas.size)

    def set_acceptance(self, mode):
        """Flip thresholds from the exact exponential ("exact") or the paper's
        fast / accurate approximation, for the next replicas_init."""
        _check(_lib.ising_set_acceptance(self.h, ACCEPT_MODES[mode]))

    def set_trotter(self, K):
        """Split couplings: temperature k weights exp(-beta_k E_space - K[k] C);
        fields and energies become the spatial ones."""
        K = np.asarray(K, dtype=np.float64)
        if K.shape != (self.R,):
            raise ValueError("K needs one value per temperature index")
        ising_set_trotter(self.h, K)

    def read_trotter(self):
        """C = -sum over Trotter pairs of s s', per slot (zeros without split couplings)."""
        return ising_read_trotter(self.h, self.R)

    def set_stream(self, stream):
        ising_set_stream(self.h, stream)

    def sweep(self, n=1):
        ising_sweep(self.h, n)

    def pt_swap(self):
        ising_pt_swap(self.h)

    def run(self, n, swap_every=1):
        ising_run(self.h, n, swap_every)

    def read_state(self):
        return ising_read_state(self.h, self.R, self.n)

    def swap_stats(self):
        return ising_read_swap_stats(self.h, self.R)

    def observables(self):
        """(E, m) of the replica at each temperature index, m = sum of spins."""
        E = np.empty(self.R, dtype=np.int64)
        m = np.empty(self.R, dtype=np.int64)
        _check(_lib.ising_read_observables(self.h, _p(E, _i64p), _p(m, _i64p)))
        return E, m

    def save(self) -> bytes:
        return ising_save(self.h)

    def load(self, blob: bytes):
        ising_load(self.h, blob)

    def set_seed(self, seed):
        """Philox: later random words use ``seed``; the state is kept."""
        ising_set_seed(self.h, seed)

    def info(self) -> dict:
        return ising_get_info(self.h)

    def set_launch(self, replicas_per_block=0, threads_per_block=0, launch_flags=LAUNCH_PERSISTENT):
        ising_set_launch(self.h, replicas_per_block, threads_per_block, launch_flags)

    def set_profiling(self, on=True):
        ising_set_profiling(self.h, on)

    def stats(self) -> dict:
        return ising_get_stats(self.h)

    def close(self):
        if getattr(self, "h", None):
            ising_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


# ------------------------------------------------------------------- batches
class Batch:
    """Ragged batch: ``Batch([(graph, betas, seed), ...], rng, field_bits)``.

    Instance b is sampled exactly like ``Ising(graph, betas, seed, ...)``
    except that its Philox counters use instance = b.
    """

    def __init__(self, instances, rng="mt19937", field_bits=16, stream=None, per_sweep=False):
        self._keep = []
        arr = (IsingInstance * len(instances))()
        self.sizes = []
        for k, (g, betas, seed) in enumerate(instances):
            rp, c, j, hh = (_arr(g.row_ptr, np.int32), _arr(g.col, np.int32), _arr(g.J, np.int32),
                            _arr(g.h, np.int32))
            if c.size == 0:
                c = np.zeros(1, np.int32)
                j = np.zeros(1, np.int32)
            b = _arr(betas, np.float64)
            self._keep += [rp, c, j, hh, b]
            arr[k] = IsingInstance(int(g.n), _p(rp, _i32p), _p(c, _i32p), _p(j, _i32p),
                                   _p(hh, _i32p), int(getattr(g, "n_slices", 1)), int(b.size),
                                   _p(b, _f64p), int(seed) & 0xFFFFFFFF)
            self.sizes.append((int(g.n), int(b.size)))
        out = _vp()
        _check(_lib.ising_batch_create(len(instances), arr, RNG[rng] if isinstance(rng, str) else rng,
                                       int(field_bits), BATCH_PER_SWEEP if per_sweep else 0, ctypes.byref(out)))
        self.h = out
        self._keep = []  # inputs are copied by the library
        if stream is not None:
            _check(_lib.ising_batch_set_stream(self.h, _vp(int(stream) if stream else None)))

    def __len__(self):
        return len(self.sizes)

    def autotune(self):
        _check(_lib.ising_batch_autotune(self.h, 0))

    def run(self, n, swap_every=1):
        _check(_lib.ising_batch_run(self.h, int(n), int(swap_every)))

    def read_state(self, inst):
        n, R = self.sizes[inst]
        spins = np.empty((R, n), dtype=np.int8)
        fields = np.empty((R, n), dtype=np.int32)
        E = np.empty(R, dtype=np.int64)
        temp = np.empty(R, dtype=np.int32)
        cnt = np.empty(2, dtype=np.uint64)
        _check(_lib.ising_batch_read_state(self.h, int(inst), _p(spins, _i8p), _p(fields, _i32p),
                                           _p(E, _i64p), _p(temp, _i32p), _p(cnt, _u64p)))
        return dict(spins=spins, fields=fields, energy=E, temp_of_slot=temp, sweeps=int(cnt[0]),
                    passes=int(cnt[1]))

    def swap_stats(self, inst):
        R = self.sizes[inst][1]
        acc = np.zeros(max(R - 1, 1), dtype=np.uint64)
        _check(_lib.ising_batch_read_swap_stats(self.h, int(inst), _p(acc, _u64p)))
        return acc[:max(R - 1, 0)]

    def info(self, inst):
        info = IsingInfo()
        res = ctypes.c_int32(0)
        _check(_lib.ising_batch_get_info(self.h, int(inst), ctypes.byref(info), ctypes.byref(res)))
        d = {name: getattr(info, name) for name, _ in IsingInfo._fields_}
        d["resident"] = int(res.value)
        return d

    def close(self):
        if getattr(self, "h", None):
            _check(_lib.ising_batch_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


# ------------------------------------------------------ learned column proposal
class Mlp:
    """The learned Trotter-column proposal network (``ising_mlp_*``).

    ``Mlp(n_slices, seed, capacity)``; parameters are a flat float32 vector in
    the layout W1 [256][M+1], b1, W2 [256][256], b2, W3 [M][256], b3.
    """

    def __init__(self, n_slices, seed=1, capacity=0, stream=None):
        self.M = int(n_slices)
        h = _vp()
        _check(_lib.ising_mlp_create(self.M, ctypes.c_uint32(seed & 0xFFFFFFFF), int(capacity),
                                     ctypes.byref(h)))
        self.m = h
        if stream is not None:
            _check(_lib.ising_mlp_set_stream(self.m, _vp(stream)))

    @property
    def n_params(self) -> int:
        return int(_lib.ising_mlp_n_params(self.m))

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _check(_lib.ising_mlp_get_params(self.m, _p(out, _f32p)))
        return out

    def set_params(self, p):
        p = _arr(p, np.float32)
        if p.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {p.size}")
        _check(_lib.ising_mlp_set_params(self.m, _p(p, _f32p)))

    def unpack(self, p=None) -> dict:
        """Split a flat parameter (or gradient) vector into its six tensors."""
        p = self.get_params() if p is None else np.asarray(p)
        M, H = self.M, 256
        sizes = [("W1", (H, M + 1)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (M, H)), ("b3", (M,))]
        out, o = {}, 0
        for name, shape in sizes:
            n = int(np.prod(shape))
            out[name] = p[o:o + n].reshape(shape)
            o += n
        return out

    def forward(self, X) -> np.ndarray:
        X = _arr(X, np.float32)
        B = X.shape[0]
        L = np.empty((B, self.M), dtype=np.float32)
        _check(_lib.ising_mlp_forward(self.m, B, _p(X, _f32p), _p(L, _f32p)))
        return L

    def grad(self, X, Y):
        X, Y = _arr(X, np.float32), _arr(Y, np.uint32)
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_float()
        _check(_lib.ising_mlp_grad(self.m, X.shape[0], _p(X, _f32p), _p(Y, _u32p), _p(g, _f32p),
                                   ctypes.byref(loss)))
        return g, float(loss.value)

    def collect(self, sim: "Ising", oriented=False):
        """Record sim's columns; oriented=True stores each in the orientation
        its spatial field prefers (training set for the mixture proposal)."""
        _check(_lib.ising_mlp_collect_flags(self.m, sim.h, COLLECT_ORIENTED if oriented else 0))

    @property
    def n_records(self) -> int:
        return int(_lib.ising_mlp_n_records(self.m))

    def clear_records(self):
        _check(_lib.ising_mlp_clear_records(self.m))

    def records(self, start=0, n=None):
        """(X [n][M + 1] float32, Y [n] uint32) of recorded rows."""
        n = self.n_records - start if n is None else n
        X = np.empty((n, self.M + 1), np.float32)
        Y = np.empty(n, np.uint32)
        _check(_lib.ising_mlp_get_records(self.m, start, n, _p(X, _f32p), _p(Y, _u32p)))
        return X, Y

    def train(self, epochs=1, batch=4096, lr=1e-3) -> float:
        loss = ctypes.c_float()
        _check(_lib.ising_mlp_train(self.m, int(epochs), int(batch), ctypes.c_float(lr), ctypes.byref(loss)))
        return float(loss.value)

    def learned_pass(self, sim: "Ising", trace=False, fp64_only=False, sync=True, mixture=False):
        """One learned pass over ``sim``.  Returns a dict of its counts
        (proposed, accepted, changed, exact_decisions) and, with trace=True,
        the per-row record as a second value.  sync=False only enqueues the
        pass and returns None.  mixture=True proposes from the flip-symmetric
        mixture (q(s') + q(-s')) / 2."""
        flags = (LEARNED_FP64_ONLY if fp64_only else 0) | (LEARNED_MIXTURE if mixture else 0)
        if not sync and not trace:
            _check(_lib.ising_learned_pass(sim.h, self.m, flags, None, None))
            return None
        st = LearnedStats()
        tr = None
        if trace:
            rows = sim.R * (sim.n // self.M)
            t = {"replica": np.empty(rows, np.int32), "site": np.empty(rows, np.int32),
                 "phi": np.empty((rows, 32), np.int32), "logits": np.empty((rows, 32), np.float32),
                 "old_bits": np.empty(rows, np.uint32), "prop_bits": np.empty(rows, np.uint32),
                 "accepted": np.empty(rows, np.uint8)}
            tr = LearnedTrace(rows, _p(t["replica"], _i32p), _p(t["site"], _i32p), _p(t["phi"], _i32p),
                              _p(t["logits"], _f32p), _p(t["old_bits"], _u32p), _p(t["prop_bits"], _u32p),
                              _p(t["accepted"], ctypes.POINTER(ctypes.c_uint8)))
        _check(_lib.ising_learned_pass(sim.h, self.m, flags, ctypes.byref(st),
                                       ctypes.byref(tr) if tr is not None else None))
        stats = {k: int(getattr(st, k)) for k in ("proposed", "accepted", "changed", "exact_decisions")}
        return (stats, t) if trace else stats

    def set_profiling(self, on=True):
        _check(_lib.ising_mlp_set_profiling(self.m, int(bool(on))))

    def stats(self) -> dict:
        st = MlpStats()
        _check(_lib.ising_mlp_get_stats(self.m, ctypes.byref(st)))
        return {"network_launches": int(st.network_launches), "network_rows": int(st.network_rows),
                "network_ms": float(st.network_ms)}

    def close(self):
        if getattr(self, "m", None):
            _lib.ising_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False
