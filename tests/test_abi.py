"""CPU checks of the C ABI: the library loads, exports every function that
include/elbm.h declares, the binding's signature table covers them, and
argument validation that needs no GPU behaves as documented."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "elbm.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"ELBM_API\s+[\w\s\*]*?\b(elbm_\w+)\s*\(",
                                 text)))


@pytest.fixture(scope="module")
def elbm():
    import __graft_entry__ as g
    from paper_1904_00866_gb300 import _build
    if not os.path.exists(os.path.join(ROOT, "paper_1904_00866_gb300",
                                       "libelbm.so")):
        _build.build()
    import paper_1904_00866_gb300 as e
    e.lib()
    return e


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["elbm_create", "elbm_init_fields", "elbm_step",
                 "elbm_moments", "elbm_alpha_map", "elbm_entropy_stats"]:
        assert must in names


def test_library_exports_every_declared_symbol(elbm):
    L = elbm.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(declared_functions()) == set(elbm.SIGNATURES)


def test_stats_struct_layout_matches_header(elbm):
    text = open(HEADER).read()
    body = text[text.index("typedef struct {"):text.index(
        "} elbm_entropy_stats_t;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(\w+)(?:\[3\])?\s*[;,]", body)
    py = [n for n, _ in elbm.EntropyStats._fields_]
    assert fields == py


def test_create_validates_arguments_without_gpu(elbm):
    L = elbm.lib()
    h = ctypes.c_void_p()
    assert L.elbm_create(ctypes.byref(h), 7, 8, 8, 1, 0.01, 0) == 1
    assert b"lattice" in L.elbm_last_error(None)
    assert L.elbm_create(ctypes.byref(h), 0, 8, 8, 2, 0.01, 0) == 1   # D2Q9 nz
    assert L.elbm_create(ctypes.byref(h), 1, 0, 8, 8, 0.01, 0) == 1
    assert L.elbm_create(ctypes.byref(h), 1, 8, 8, 8, -1.0, 0) == 1
    assert L.elbm_create(ctypes.byref(h), 1, 8, 8, 8, 0.01, 9) == 1
    assert L.elbm_create(ctypes.byref(h), 1, 8, 8, 8, 0.01, 2) == 0
    assert L.elbm_step_count(h) == 0
    # stepping before initialisation is a state error, not a crash
    assert L.elbm_step(h, 1, 0) == 7
    assert L.elbm_set_diagnostics(h, -1, 0, 0, 4) == 1
    assert L.elbm_set_diagnostics(h, 1, 0, 0, 4) == 0
    L.elbm_destroy(h)
    # D1Q3: one row of nodes, FP64 storage only
    assert L.elbm_create(ctypes.byref(h), 2, 8, 2, 1, 0.01, 0) == 1
    assert L.elbm_create(ctypes.byref(h), 2, 8, 1, 2, 0.01, 0) == 1
    for dtype in (1, 2, 3):
        assert L.elbm_create(ctypes.byref(h), 2, 8, 1, 1, 0.01, dtype) == 1
        assert b"FP64" in L.elbm_last_error(None)
    assert L.elbm_create(ctypes.byref(h), 2, 1602, 1, 1, 1e-5, 0) == 0
    assert L.elbm_step(h, 1, 0) == 7
    L.elbm_destroy(h)


def test_batch_and_static_entry_points_reject_d1q3_without_gpu(elbm):
    L = elbm.lib()
    st = L.elbm_step_static(2, 64, 1, 1, 1e-4, 1.0, None, None, None, None,
                            None)
    assert st == 1 and b"D2Q9 and D3Q27" in L.elbm_last_error(None)
    b = ctypes.c_void_p()
    assert L.elbm_batch_create(ctypes.byref(b), 4) == 0
    spec = elbm.MemberSpec(lattice=2, nx=64, ny=1, nz=1, nu=1e-4)
    rho = (ctypes.c_double * 64)(*([1.0] * 64))
    u = (ctypes.c_double * 64)()
    mid = ctypes.c_int(7)
    assert L.elbm_batch_add(b, ctypes.byref(spec), rho, u,
                            ctypes.byref(mid)) == 1
    assert mid.value == -1
    assert b"D2Q9 or D3Q27" in L.elbm_batch_last_error(b)
    L.elbm_batch_destroy(b)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_1904_00866_gb300 as e
    monkeypatch.setattr(e, "_lib", None)
    monkeypatch.setattr(e, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        e.lib()


def test_beta_comes_from_the_library(elbm):
    """The binding reads beta from the C ABI; it matches the oracle's Eq. (2)
    and needs no device."""
    import oracle
    L = elbm.lib()
    h = ctypes.c_void_p()
    for nu in (1e-5, 2.546e-3, 0.01, 0.5):
        assert L.elbm_create(ctypes.byref(h), 1, 8, 8, 8, nu, 2) == 0
        assert abs(L.elbm_beta(h) - oracle.beta_from_nu(nu)) <= 1e-15
        L.elbm_destroy(h)
    assert L.elbm_beta(None) != L.elbm_beta(None)        # NaN for NULL


def test_binding_restates_no_method_arithmetic():
    """The Python binding is marshalling only: no Eq. (2) (beta from nu) or
    other method formula is evaluated there."""
    src = open(os.path.join(ROOT, "paper_1904_00866_gb300",
                            "__init__.py")).read()
    code = re.sub(r'""".*?"""', "", src, flags=re.S)
    code = "\n".join(l.split("#")[0] for l in code.splitlines())
    for pattern in [r"1\.0\s*/\s*3", r"cs2", r"2\.0\s*\*\s*self\.nu",
                    r"\bnp\.log", r"\bmath\.", r"\bsqrt\b"]:
        assert not re.search(pattern, code), pattern
