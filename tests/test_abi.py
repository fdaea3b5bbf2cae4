"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports
every function include/prot.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"\b(pr_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2203_03732_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("pr_assign", "pr_assign_workspace", "pr_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(libpath):
    from paper_2203_03732_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_workspace_query_without_gpu(libpath):
    from paper_2203_03732_gb300 import _lib
    L = _lib.load(libpath)
    assert L.pr_assign_workspace(0, 10) == 0
    assert L.pr_assign_workspace(11, 10) == 0
    w = L.pr_assign_workspace(10000, 10000)
    assert w >= 10000 * 10000 * 2 and w % 256 == 0
    assert L.pr_status_string(-3) == b"PR_ERR_TIMEOUT"


def test_host_argument_errors_without_gpu(libpath):
    from paper_2203_03732_gb300 import _lib
    L = _lib.load(libpath)
    st = _lib.PrStats()
    rc = L.pr_assign(None, 1, 10, 10, 10, 0.1, None, None, None, None, None, ctypes.byref(st),
                     None, 0, None)
    assert rc == _lib.PR_ERR_INVALID
    assert b"NULL" in L.pr_last_error()


def test_staged_and_ot_argument_errors_without_gpu(libpath):
    """pr_assign_staged and pr_ot check their arguments on the host before
    any CUDA call: each bad argument returns PR_ERR_INVALID with a message."""
    from paper_2203_03732_gb300 import _lib
    L = _lib.load(libpath)
    buf = ctypes.create_string_buffer(4096)
    p = ctypes.cast(buf, ctypes.c_void_p).value
    outs = (p, p, p, p, p)
    cases = [
        ((None, p, 1, 10, 10, 10, 0.1), b"NULL"),
        ((p, None, 1, 10, 10, 10, 0.1), b"NULL"),
        ((p, p, 7, 10, 10, 10, 0.1), b"dtype"),
        ((p, p, 1, 9, 10, 10, 0.1), b"ldc"),
    ]
    for head, msg in cases:
        rc = L.pr_assign_staged(*head, *outs, None, p, 4096, None)
        assert rc == _lib.PR_ERR_INVALID
        assert msg in L.pr_last_error()
    f64 = (ctypes.c_double * 4)()
    dp = ctypes.cast(f64, ctypes.c_void_p).value
    ot_cases = [
        (dict(C=None), b"NULL"),
        (dict(dt=7), b"dtype"),
        (dict(n_sup=0), b"n_sup"),
        (dict(ldc=1), b"ldc"),
        (dict(eps=1.5), b"eps"),
        (dict(eps=1e-6), b"eps"),
        (dict(plan_cap=0), b"plan_cap"),
        (dict(ws=None), b"workspace"),
    ]
    for change, msg in ot_cases:
        a = dict(C=p, dt=1, ldc=4, n_sup=2, n_dem=2, supply=dp, demand=dp, eps=0.1, plan_cap=8, ws=p)
        a.update(change)
        rc = L.pr_ot(a["C"], a["dt"], a["ldc"], a["n_sup"], a["n_dem"], a["supply"], a["demand"], a["eps"],
                     a["plan_cap"], p, p, p, p, p, p, p, p, p, None, a["ws"], 1 if a["ws"] else 0, None)
        expect = _lib.PR_ERR_WORKSPACE if msg == b"workspace" else _lib.PR_ERR_INVALID
        assert rc == expect, (change, rc)
        assert msg in L.pr_last_error(), (change, L.pr_last_error())


def test_other_entry_points_argument_errors_without_gpu(libpath):
    """The host-side argument checks of the remaining entry points, each
    before any CUDA call: PR_ERR_INVALID and a message naming the argument."""
    from paper_2203_03732_gb300 import _lib
    L = _lib.load(libpath)
    buf = ctypes.create_string_buffer(4096)
    p = ctypes.cast(buf, ctypes.c_void_p).value
    n_host = (ctypes.c_int32 * 2)(64, 64)
    calls = [
        (lambda: L.pr_assign_rule(5, p, 1, 10, 10, 10, 0.1, p, p, p, p, p, None, p, 4096, None), b"rule"),
        (lambda: L.pr_assign_points(None, p, 2, 1, 10, 10, 0.1, p, p, p, p, p, None, p, 4096, None), b"NULL"),
        (lambda: L.pr_assign_points(p, p, 0, 1, 10, 10, 0.1, p, p, p, p, p, None, p, 4096, None), b"dim"),
        (lambda: L.pr_assign_points(p, p, 2, 9, 10, 10, 0.1, p, p, p, p, p, None, p, 4096, None), b"metric"),
        (lambda: L.pr_assign_points(p, p, 2, 1, 11, 10, 0.1, p, p, p, p, p, None, p, 4096, None), b"n_rows"),
        (lambda: L.pr_assign_points(p, p, 2, 1, 10, 10, 0.0, p, p, p, p, p, None, p, 4096, None), b"eps"),
        (lambda: L.pr_assign_batched(None, 1, 2, n_host, 0.1, p, p, p, p, p, p, None, None, p, 4096, None),
         b"NULL"),
        (lambda: L.pr_assign_batched(p, 7, 2, n_host, 0.1, p, p, p, p, p, p, None, None, p, 4096, None),
         b"dtype"),
        (lambda: L.pr_assign_batched_points(None, p, 3, 0, 2, n_host, 0.1, p, p, p, p, p, p, None, None, p,
                                            4096, None), b"NULL"),
        (lambda: L.pr_assign_batched_points(p, p, 0, 0, 2, n_host, 0.1, p, p, p, p, p, p, None, None, p,
                                            4096, None), b"dim"),
        (lambda: L.pr_assign_batched_points(p, p, 3, 9, 2, n_host, 0.1, p, p, p, p, p, p, None, None, p,
                                            4096, None), b"metric"),
        (lambda: L.pr_assign_backward(None, p, p, 1, 8, 3, p, p, p, None, None), b"NULL"),
        (lambda: L.pr_assign_backward(p, p, p, 0, 8, 3, p, p, p, None, None), b"batch"),
        (lambda: L.pr_assign_backward(p, p, p, 1, 8, 5000, p, p, p, None, None), b"dim"),
        (lambda: L.pr_dual_bound(None, p, 4, 4, 0.1, p, p, None), b"NULL"),
        (lambda: L.pr_dual_bound(p, p, 5, 4, 0.1, p, p, None), b"n_rows"),
        (lambda: L.pr_dual_bound(p, p, 4, 4, 1.0, p, p, None), b"eps"),
        (lambda: L.pr_assign_noalloc(None, 1, 10, 10, 10, 0.1, p, p, p, p, p, None, None), b"NULL"),
        (lambda: L.pr_assign_noalloc(p, 7, 10, 10, 10, 0.1, p, p, p, p, p, None, None), b"dtype"),
        (lambda: L.pr_assign_noalloc(p, 1, 2000, 2000, 2000, 0.1, p, p, p, p, p, None, None), b"1024"),
        (lambda: L.pr_assign_noalloc(p, 1, 9, 10, 10, 0.1, p, p, p, p, p, None, None), b"ldc"),
        (lambda: L.pr_assign_noalloc(p, 1, 10, 10, 10, 2.0, p, p, p, p, p, None, None), b"eps"),
    ]
    for call, msg in calls:
        assert call() == _lib.PR_ERR_INVALID, msg
        assert msg in L.pr_last_error(), (msg, L.pr_last_error())


def test_missing_library_fails_loudly(tmp_path):
    from paper_2203_03732_gb300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(ImportError):
            _lib.load(str(tmp_path / "nope.so"))
    finally:
        _lib._lib = saved


def test_no_oracle_import_in_product_path():
    pkg = os.path.join(ROOT, "paper_2203_03732_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "prot_oracle" not in txt, f


def test_assign_within_refuses_delta_without_gpu(libpath):
    """pr_assign_within checks delta (0 < delta < 3) before anything else."""
    from paper_2203_03732_gb300 import _lib
    L = _lib.load(libpath)
    st = _lib.PrStats()
    for delta in (0.0, -1.0, 3.0, float("nan")):
        rc = L.pr_assign_within(None, 1, 10, 10, 10, delta, None, None, None, None, None,
                                ctypes.byref(st), None, 0, None)
        assert rc == _lib.PR_ERR_INVALID
        assert b"delta" in L.pr_last_error()


def test_ot_workspace_is_linear_beyond_the_rounded_costs(libpath):
    """pr_ot keeps its matched copy counts in per-demand lists: apart from
    the rounded costs (n_sup x ldq 16-bit values at most) the workspace grows
    like n_sup + n_dem, not n_sup x n_dem."""
    L = ctypes.CDLL(libpath)
    L.pr_ot_workspace.restype = ctypes.c_size_t
    L.pr_ot_workspace.argtypes = [ctypes.c_int32, ctypes.c_int32]
    for nB, nA in ((10000, 10000), (2000, 30000), (30000, 2000), (1, 1)):
        ldq = (nA + 15) // 16 * 16
        rest = L.pr_ot_workspace(nB, nA) - 2 * nB * ldq
        assert 0 < rest <= 1024 * (nB + nA) + (1 << 20), (nB, nA, rest)
