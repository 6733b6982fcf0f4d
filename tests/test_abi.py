"""libtsqr's C ABI on the CPU: the library builds and loads, exports every symbol the header
declares, and rejects bad arguments on the host before touching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1002_4250_gb300 import _build
    _build.build()
    import paper_1002_4250_gb300 as T
    return T


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "tsqr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tsqr_[a-z_]+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = _declared_functions()
    for must in ("tsqr_r", "tsqr_r_batched", "tsqr_r_ex", "tsqr_qr_uppers"):
        assert must in names


def test_every_entry_point_is_documented():
    """Each declaration in the header is preceded by its own comment block, and the compute
    entry points cite the passage of the paper they implement (a Section, Table or Fig.)."""
    text = open(os.path.join(ROOT, "include", "tsqr.h")).read()
    decl = re.compile(r"(?:tsqr_status_t|int32_t|const char \*|void)\s+(tsqr_[a-z_]+)\s*\(")
    cited = re.compile(r"Section \d|Table \d|Fig\. \d")
    compute = {"tsqr_r", "tsqr_r_ex", "tsqr_r_host", "tsqr_qr", "tsqr_qr_uppers", "tsqr_lstsq",
               "tsqr_caqr_r", "tsqr_r_batched"}
    seen = set()
    for mt in decl.finditer(text):
        name = mt.group(1)
        comment_end = text.rfind("*/", 0, mt.start())
        comment_start = text.rfind("/*", 0, comment_end)
        between = text[comment_end + 2:mt.start()]
        assert comment_end > 0 and ";" not in between, f"{name} has no comment of its own"
        if name in compute:
            assert cited.search(text[comment_start:comment_end]), f"{name} cites no passage"
        seen.add(name)
    assert compute <= seen


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(lib.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(raw, name), name
    assert set(_declared_functions()) == set(lib.ABI_SYMBOLS)


def test_status_strings(lib):
    for s in range(7):
        assert lib.capi.tsqr_status_string(s)
    assert b"unknown" in lib.capi.tsqr_status_string(99)


def test_host_side_argument_errors(lib):
    c = lib.capi
    bad = [  # (A, m, n, lda, R, ldr)
        (None, -1, 4, 10, None, 4),      # m < 0
        (None, 10, -2, 10, None, 4),     # n < 0
        (None, 10, 4, 9, None, 4),       # lda < m
        (None, 10, 4, 10, None, 3),      # ldr < n
        (None, 10, 4, 10, None, 4),      # NULL pointers with work to do
    ]
    for A, m, n, lda, R, ldr in bad:
        assert c.tsqr_r(A, m, n, lda, R, ldr, None) == lib.ERR_INVALID_ARG
    # above TSQR_MAX_N columns only tall matrices (by panels) are supported
    assert c.tsqr_r(None, 10, 129, 10, None, 129, None) == lib.ERR_UNSUPPORTED
    # n == 0 is a no-op
    assert c.tsqr_r(None, 10, 0, 10, None, 1, None) == lib.SUCCESS
    # bad dtype / precision pairs
    assert c.tsqr_r_ex(None, 7, 0, 10, 4, 10, None, 4, None, None) == lib.ERR_INVALID_ARG
    assert c.tsqr_r_ex(None, lib.F32, lib.PREC_F64, 10, 4, 10, None, 4, None, None) == lib.ERR_INVALID_ARG
    assert c.tsqr_qr_uppers(4, None, 3, None, 4, None, 4, 0, None) == lib.ERR_INVALID_ARG
    assert c.tsqr_qr_uppers(200, None, 200, None, 200, None, 200, 0, None) == lib.ERR_UNSUPPORTED
    assert c.tsqr_r_batched(None, None, None, None, -1, None, 0, 0, None) == lib.ERR_INVALID_ARG
    assert c.tsqr_r_batched(None, None, None, None, 0, None, 0, 0, None) == lib.SUCCESS
    assert lib.tsqr_last_launch_count() == 0


def test_package_has_no_cpu_fallback():
    src = open(os.path.join(ROOT, "paper_1002_4250_gb300", "__init__.py")).read()
    assert "import oracle" not in src and "from oracle" not in src
    for f in os.listdir(os.path.join(ROOT, "paper_1002_4250_gb300", "csrc")):
        body = open(os.path.join(ROOT, "paper_1002_4250_gb300", "csrc", f)).read()
        assert "oracle" not in body.lower(), f
