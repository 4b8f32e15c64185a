"""The C-ABI library: loads without a GPU, exports every declared entry point,
and rejects invalid models on the host before any device work (no GPU)."""
import os
import re

import numpy as np
import pytest

from conftest import ROOT

HEADER_DIR = os.path.join(ROOT, "include")


def _declared():
    names = set()
    for fn in os.listdir(HEADER_DIR):
        if fn.endswith(".h"):
            text = open(os.path.join(HEADER_DIR, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(ising_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1004_0024_gb300 import build
    build.build()
    from paper_1004_0024_gb300 import ising
    return ising


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("ising_create", "ising_replicas_init", "ising_sweep", "ising_pt_swap",
                 "ising_run", "ising_read_state", "ising_save", "ising_load", "ising_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in sorted(_declared()):
        assert hasattr(lib._lib, name), name


def _graph(edges, n, h=None, n_slices=1):
    from paper_1004_0024_gb300 import workloads as W
    return W.graph_from_edges(n, edges, np.zeros(n) if h is None else h, n_slices)


@pytest.mark.parametrize("case,code", [
    ("asym", "ASYMMETRIC_J"), ("self", "SELF_LOOP_OR_DUP"), ("dup", "SELF_LOOP_OR_DUP"),
    ("range", "INVALID_ARG"), ("slices", "INVALID_ARG"), ("bigJ", "INVALID_ARG"),
])
def test_host_validation_errors(lib, case, code):
    g = _graph({(0, 1): 1, (1, 2): -2}, 4)
    rp, col, J = g.row_ptr.copy(), g.col.copy(), g.J.copy()
    n_slices = 1
    if case == "asym":
        J[0] = 3
    elif case == "self":
        col[0] = 0
    elif case == "dup":
        col[2] = col[1]
    elif case == "range":
        col[0] = 7
    elif case == "slices":
        n_slices = 2  # spins 0..1 and 2..3 are not identical slices
    elif case == "bigJ":
        J[:] = 40000
    with pytest.raises(lib.IsingError) as ei:
        lib.ising_create(g.n, rp, col, J, g.h, n_slices)
    assert ei.value.name == code
    assert lib.ising_last_error()


@pytest.mark.parametrize("faults,code,where", [
    ({"self": 9000, "range": 200}, "INVALID_ARG", "row 200"),
    ({"range": 9000, "self": 200}, "SELF_LOOP_OR_DUP", "spin 200"),
    ({"asym": 150, "dup": 9100}, "SELF_LOOP_OR_DUP", "row 9100"),
    ({"asym": 9500}, "ASYMMETRIC_J", "J(9499,9500)"),  # first seen from row 9499
])
def test_host_validation_of_large_graphs_reports_the_first_row(lib, faults, code, where):
    """A ring of 12000 spins (rows checked in parallel chunks): of several
    faults, the error reported is the one a row-by-row check meets first
    (index faults in any row before asymmetry, then the lowest row)."""
    n = 12000
    g = _graph({(i, (i + 1) % n): 1 + (i % 3) for i in range(n)}, n)
    rp, col, J = g.row_ptr.copy(), g.col.copy(), g.J.copy()
    for kind, row in faults.items():
        e = rp[row]
        if kind == "self":
            col[e] = row
        elif kind == "range":
            col[e] = n + 5
        elif kind == "dup":
            col[e + 1] = col[e]
        elif kind == "asym":
            J[e] = J[e] + 1
    with pytest.raises(lib.IsingError) as ei:
        lib.ising_create(g.n, rp, col, J, g.h, 1)
    assert ei.value.name == code
    assert where in lib.ising_last_error(), lib.ising_last_error()


# ------------------------------------------ split couplings, host side
def test_split_flip_table_matches_the_oracle(lib):
    """The tables ising_set_trotter uploads, entry by entry against the
    oracle's split flip rule (k_s in [-ks, ks], k_tau in {-2, 0, 2})."""
    import oracle
    from paper_1004_0024_gb300 import workloads as W
    betas = W.geometric_betas(16, 0.05, 5.0)
    K = W.trotter_couplings(betas, 2.0, 32)
    ks = 20
    tab = lib.split_flip_table(betas, K, ks)
    for t in range(betas.size):
        for k in range(-ks, ks + 1):
            for j, kt in enumerate((-2, 0, 2)):
                assert tab[t, k + ks, j] == oracle.trotter_flip_threshold(betas[t], K[t], k, kt), (t, k, kt)
    with pytest.raises(lib.IsingError):
        lib.split_flip_table(betas, K, 1365)


def test_split_device_exponential_matches_the_oracle(lib):
    """The swap rule's fixed FP64 exponential, compiled from the device source
    for the host, equals the oracle's on 200000 arguments, and so do the swap
    thresholds built from it."""
    import oracle
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.uniform(-708, 0, 120000), rng.uniform(-1, 0, 60000),
                         -np.logspace(-18, 2.85, 20000), [0.0, -708.5, -745.0]])
    got = np.array([lib.split_exp(x) for x in xs.tolist()])
    want = np.array([oracle.exp_det(x) for x in xs.tolist()])
    assert np.array_equal(got, want)
    for dbeta, dK in [(0.02, -0.1), (0.3, 0.05), (1e-3, -2.0), (0.0123, 0.77)]:
        for dE in range(-50, 400, 13):
            for dC in range(-40, 41, 5):
                assert lib.split_swap_threshold(dbeta, dK, dE, dC) == \
                    oracle.trotter_swap_threshold(dbeta, dK, dE, dC), (dbeta, dK, dE, dC)


def test_header_is_plain_c():
    """The boundary header compiles as ISO C11 (no C++ or CUDA types leak
    into the ABI) and as C++17."""
    import shutil
    import subprocess
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    hdr = os.path.join(HEADER_DIR, "ising_gb300.h")
    for lang, std in (("c", "-std=c11"), ("c++", "-std=c++17")):
        r = subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", lang, hdr],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def _layered_with_fault(L, M, spin_offset):
    """A layered model whose slice t = 3 differs from slice 0 in h at one
    site: ising_create must reject it at spin 3 S + spin_offset."""
    from paper_1004_0024_gb300 import workloads as W
    g = W.layered_graph(L, M, graph_seed=7)
    S = g.n // M
    h = g.h.copy()
    h[3 * S + spin_offset] += 1
    return g, h, 3 * S + spin_offset


def test_host_worker_threads_serve_concurrent_callers(lib):
    """The library's host loops share one set of worker threads: eight Python
    threads creating models (rejected in slice extraction, which runs on the
    workers) and building flip tables at once all get their own, correct
    answers."""
    import threading
    import oracle
    from paper_1004_0024_gb300 import workloads as W
    betas = W.geometric_betas(1024, 0.05, 5.0)
    K = W.trotter_couplings(betas, 2.0, 32)
    want = lib.split_flip_table(betas, K, 20)
    assert want[517, 21, 2] == oracle.trotter_flip_threshold(betas[517], K[517], 1, 2)
    cases = [_layered_with_fault(32, 16, off) for off in (5, 77, 300, 901)]
    errors = []

    def worker(k):
        try:
            for rep in range(6):
                g, h, spin = cases[(k + rep) % len(cases)]
                with pytest.raises(lib.IsingError) as e:
                    lib.ising_create(g.n, g.row_ptr, g.col, g.J, h, g.n_slices)
                assert f"declared slices differ in h at spin {spin}" in str(e.value), str(e.value)
                assert np.array_equal(lib.split_flip_table(betas, K, 20), want)
        except BaseException as exc:  # reported on the main thread
            errors.append(repr(exc))

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(8)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=120)
    assert not any(t.is_alive() for t in threads), "a host loop did not return"
    assert not errors, errors


def _forked_table(q):
    from paper_1004_0024_gb300 import ising
    from paper_1004_0024_gb300 import workloads as W
    betas = W.geometric_betas(1024, 0.05, 5.0)
    K = W.trotter_couplings(betas, 2.0, 32)
    q.put(ising.split_flip_table(betas, K, 20).sum(dtype=np.uint64))


@pytest.mark.filterwarnings("ignore:This process .* is multi-threaded:DeprecationWarning")
def test_host_loops_work_in_a_forked_child(lib):
    """A child forked after the parent's worker threads exist has none of
    them: its host loops run on fresh threads instead of waiting forever."""
    import multiprocessing as mp
    from paper_1004_0024_gb300 import workloads as W
    betas = W.geometric_betas(1024, 0.05, 5.0)
    K = W.trotter_couplings(betas, 2.0, 32)
    want = lib.split_flip_table(betas, K, 20).sum(dtype=np.uint64)  # parent's workers now exist
    ctx = mp.get_context("fork")
    q = ctx.Queue()
    p = ctx.Process(target=_forked_table, args=(q,))
    p.start()
    p.join(timeout=60)
    if p.is_alive():
        p.kill()
        p.join()
        pytest.fail("host loop in the forked child did not return")
    assert p.exitcode == 0
    assert q.get(timeout=5) == want


@pytest.mark.parametrize("R,lo,hi,dmax", [(32, 0.1, 3.0, 67789), (2, 0.4, 0.9, 5000), (9, 0.2, 2.0, 40)])
def test_swap_tables_match_the_oracle(lib, R, lo, hi, dmax):
    """The PT swap tables ising_replicas_init uploads, entry by entry against
    the oracle's floor(2^32 exp(-dbeta d)), with each table ending at the
    first zero threshold or at the energy bound dmax."""
    import oracle
    from paper_1004_0024_gb300 import workloads as W
    betas = W.geometric_betas(R, lo, hi)
    thr, off, ln, ok = lib.swap_thresholds(betas, dmax)
    assert ok
    for k in range(R - 1):
        db = betas[k + 1] - betas[k]
        L = int(ln[k])
        got = thr[off[k] + 1: off[k] + L]
        want = [oracle.swap_threshold(db, d) for d in range(1, L)]
        assert np.array_equal(got, np.array(want, dtype=np.uint32)), k
        assert L == dmax or oracle.swap_threshold(db, L) == 0
        assert L == 1 or got[-1] > 0


def test_swap_tables_beyond_2p28_entries_refuse_pt(lib):
    """The 65536-temperature ladder of the many-replica workload needs far
    more than 2^28 FP64 thresholds: PT is refused at once (one placeholder
    entry), as ising_pt_swap then reports."""
    from paper_1004_0024_gb300 import workloads as W
    thr, off, ln, ok = lib.swap_thresholds(W.geometric_betas(65536, 0.1, 3.0), 60001)
    assert not ok and thr.size == 1 and np.all(off == 0) and np.all(ln == 1)


def test_noalloc_refuses_a_pt_group_longer_than_a_launch(lib):
    # an argument check taken before any handle or device work: a PT group of
    # more than 2^30 sweeps cannot run in one launch (it used to loop forever)
    with pytest.raises(lib.IsingError) as ei:
        lib.ising_run_noalloc(None, (1 << 30) + 5, (1 << 30) + 1)
    assert ei.value.name == "INVALID_ARG"
    assert "2^30" in lib.ising_last_error()
    # fewer sweeps than one group: no fused group, so the handle is checked next
    with pytest.raises(lib.IsingError) as ei:
        lib.ising_run_noalloc(None, 5, (1 << 30) + 1)
    assert "2^30" not in lib.ising_last_error()
