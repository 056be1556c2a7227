"""The C-ABI library builds, loads and exports every declared symbol; host-side
argument checks and workspace sizing answer without a GPU (no compute calls)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_1006_1744_gb300 import build
    return build.build()


def declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gf2_[a-z_0-9]+)\s*\(", text)))


def test_headers_declare_the_boundary():
    names = declared("gf2.h")
    for want in ("gf2_pls", "gf2_rref", "gf2_rank", "gf2_mul", "gf2_workspace_bytes", "gf2_strerror"):
        assert want in names


@pytest.mark.parametrize("header,lib", [("gf2.h", "libgf2.so"), ("gf2_synth.h", "libgf2synth.so")])
def test_library_exports_every_declared_symbol(built, header, lib):
    L = ctypes.CDLL(built[lib])
    for name in declared(header):
        assert hasattr(L, name), f"{lib} does not export {name}"


def test_binding_covers_the_header(built):
    from paper_1006_1744_gb300 import gf2
    assert set(declared("gf2.h")) == set(gf2.SYMBOLS)
    assert gf2.lib().gf2_version() >= 100
    assert gf2.lib().gf2_strerror(0) == b"ok"
    assert b"align" in gf2.lib().gf2_strerror(2)


def test_workspace_bytes_host_only(built):
    from paper_1006_1744_gb300 import gf2
    small = gf2.workspace_bytes(gf2.OP_PLS, 64, 64)
    big = gf2.workspace_bytes(gf2.OP_PLS, 16384, 16384)
    assert 0 < small < big
    assert big >= 16384 * 256 * 8  # at least one copy of the matrix (rows in final order)
    assert gf2.workspace_bytes(gf2.OP_RREF, 1024, 1024) > gf2.workspace_bytes(gf2.OP_PLS, 1024, 1024)
    assert gf2.workspace_bytes(gf2.OP_PLS, -1, 5) == 0
    assert gf2.workspace_bytes(99, 5, 5) == 0
    bad = gf2.Opts()
    bad.k = 5
    assert gf2.workspace_bytes(gf2.OP_PLS, 64, 64, bad) == 0


def test_argument_checks_reject_before_any_device_work(built):
    """Invalid arguments are refused on the host: nothing is dereferenced."""
    from paper_1006_1744_gb300 import gf2
    L = gf2.lib()
    fake = 1 << 40          # 128-byte aligned, never touched
    rank = 1 << 41
    P, Q = 1 << 42, 1 << 43
    EINVAL, EALIGN = 1, 2
    assert L.gf2_pls(None, 8, 8, 16, P, Q, rank, None, 0, None, None) == EINVAL
    assert L.gf2_pls(fake + 8, 8, 8, 16, P, Q, rank, None, 0, None, None) == EALIGN
    assert L.gf2_pls(fake, 8, 8, 15, P, Q, rank, None, 0, None, None) == EALIGN
    assert L.gf2_pls(fake, 8, 130, 2, P, Q, rank, None, 0, None, None) == EINVAL  # stride < ceil(n/64)
    assert L.gf2_pls(fake, -1, 8, 16, P, Q, rank, None, 0, None, None) == EINVAL
    assert L.gf2_pls(fake, 8, 8, 16, None, Q, rank, None, 0, None, None) == EINVAL
    assert L.gf2_pls(fake, 8, 8, 16, P, Q, None, None, 0, None, None) == EINVAL
    bad = gf2.Opts()
    bad.tile_words = 3
    assert L.gf2_pls(fake, 8, 8, 16, P, Q, rank, None, 0, ctypes.byref(bad), None) == EINVAL
    bad = gf2.Opts()
    bad.reserved[2] = 1
    assert L.gf2_rref(fake, 8, 8, 16, rank, None, None, 0, ctypes.byref(bad), None) == EINVAL
    # table width: 4 and 8 only; 4 only on the 16-word PLS-form sweep
    for k, extra in [(6, {}), (16, {}), (4, {"rref_method": 2}), (4, {"rref_method": 3}), (4, {"tile_words": 8}),
                     (4, {"batch_mode": 2})]:
        bad = gf2.Opts()
        bad.k = k
        for f, v in extra.items():
            setattr(bad, f, v)
        assert L.gf2_rref(fake, 8, 8, 16, rank, None, None, 0, ctypes.byref(bad), None) == EINVAL, (k, extra)
    # route and schedule codes
    for f, v in [("rref_method", 4), ("rref_method", -1), ("hybrid_permille", 1001), ("batch_mode", 3)]:
        bad = gf2.Opts()
        setattr(bad, f, v)
        assert L.gf2_rref(fake, 8, 8, 16, rank, None, None, 0, ctypes.byref(bad), None) == EINVAL, (f, v)
    assert L.gf2_rank(fake, 8, 8, 16, None, None, 0, None, None) == EINVAL
    # misaligned or undersized caller workspace
    assert L.gf2_pls(fake, 8, 8, 16, P, Q, rank, fake + 64, 1 << 30, None, None) == EALIGN
    assert L.gf2_pls(fake, 8, 8, 16, P, Q, rank, fake, 16, None, None) == 5  # GF2_ENOSPACE
    # product: bad strides
    assert L.gf2_mul(fake, 16, fake, 16, fake, 7, 8, 8, 8, 0, None, 0, None, None) == EALIGN


def test_product_path_refuses_without_library(tmp_path, monkeypatch):
    """A missing build fails loudly instead of falling back to the CPU."""
    import importlib
    import paper_1006_1744_gb300.gf2 as g
    mod = importlib.reload(g)
    monkeypatch.setattr(mod, "_LIBPATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(mod, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        mod.lib()
    importlib.reload(g)


def test_batched_workspace_and_checks_host_only(built):
    """Batched PLS: workspace sizing reads only sizes; invalid items are refused
    on the host before anything is enqueued."""
    from paper_1006_1744_gb300 import gf2
    one = gf2.pls_batched_workspace_bytes([(300, 700, 16)])
    two = gf2.pls_batched_workspace_bytes([(300, 700, 16), (300, 700, 16)])
    assert one >= gf2.workspace_bytes(gf2.OP_PLS, 300, 700)
    assert two > one
    assert gf2.pls_batched_workspace_bytes([]) > 0 or gf2.pls_batched_workspace_bytes([]) == 0
    assert gf2.pls_batched_workspace_bytes([(10, 100, 1)]) == 0  # stride < ceil(n/64)
    assert gf2.pls_batched_workspace_bytes([(-1, 5, 16)]) == 0
    L = gf2.lib()
    items = (gf2.BatchItem * 1)()
    items[0] = gf2.BatchItem(None, 10, 10, 16, None, None)  # null A with m, n > 0
    assert L.gf2_pls_batched(items, 1, None, None, 0, None, None) == 1
    items[0] = gf2.BatchItem(0x1040, 10, 10, 16, 0x2000, 0x3000)  # A not 128-byte aligned
    assert L.gf2_pls_batched(items, 1, None, None, 0, None, None) == 2
    items[0] = gf2.BatchItem(0x1000, 10, 10, 16, None, 0x3000)  # P missing
    assert L.gf2_pls_batched(items, 1, None, None, 0, None, None) == 1
    assert L.gf2_pls_batched(items, -1, None, None, 0, None, None) == 1
    assert L.gf2_pls_batched(None, 0, None, None, 0, None, None) == 0


def test_status_codes_have_text(built):
    from paper_1006_1744_gb300 import gf2
    assert b"wait" in gf2.lib().gf2_strerror(8)


def test_autotune_argument_checks_host_only(built):
    from paper_1006_1744_gb300 import gf2
    L = gf2.lib()
    o = gf2.Opts()
    ms = __import__("ctypes").c_double()
    byref = __import__("ctypes").byref
    assert L.gf2_autotune(99, 64, 64, 0.5, byref(o), byref(ms), None) == 1
    assert L.gf2_autotune(gf2.OP_PLS, 0, 64, 0.5, byref(o), byref(ms), None) == 1
    assert L.gf2_autotune(gf2.OP_PLS, 64, 64, 0.0, byref(o), byref(ms), None) == 1
    assert L.gf2_autotune(gf2.OP_PLS, 64, 64, 1.5, byref(o), byref(ms), None) == 1
    assert L.gf2_autotune(gf2.OP_PLS, 64, 64, 0.5, None, byref(ms), None) == 1


def test_mul_workspace_bytes_by_product_form():
    """The product's workspace query: none for the XOR-table form, B^T for the
    tensor-core form, and for the Strassen forms a size that grows with the
    recursion and is zero-cost only when no level is taken."""
    from paper_1006_1744_gb300 import gf2
    assert gf2.mul_workspace_bytes(4096, 4096, 4096, {"product": 1}) == 0
    tc = gf2.mul_workspace_bytes(4096, 4096, 4096, {"product": 2})
    assert tc >= 4096 * 4096 // 8
    one = gf2.mul_workspace_bytes(4096, 4096, 4096, {"product": 3, "cutoff_cols": 2048})   # one level
    two = gf2.mul_workspace_bytes(4096, 4096, 4096, {"product": 3, "cutoff_cols": 1024})   # two levels
    assert 0 < one < two
    # the accumulation product (m x n) plus at least the top level's three blocks
    assert one >= 4096 * 4096 // 8 + 3 * (2048 * 2048 // 8)
    assert gf2.mul_workspace_bytes(4096, 3000, 4096, {"product": 3, "cutoff_cols": 1024}) == 0  # no split
    assert gf2.mul_workspace_bytes(4096, 4096, 4096, {"product": 4, "cutoff_cols": 1024}) > two
    assert gf2.mul_workspace_bytes(-1, 4, 4, None) == 0
    assert gf2.mul_workspace_bytes(64, 64, 64, {"product": 5}) == 0


def test_panels_per_sweep_option_host_only(built):
    """panels_per_sweep: 0 (the library's choice), 1 or 2; other values are refused before any
    device work, and two panels per sweep size the workspace for the coordinates of every row over
    both panels' pivot rows and two buffers of four panel words per row (8 more words per row)."""
    from paper_1006_1744_gb300 import gf2
    m, n = 1000, 3000
    one = gf2.workspace_bytes(gf2.OP_PLS, m, n, {"panels_per_sweep": 1})
    two = gf2.workspace_bytes(gf2.OP_PLS, m, n, {"panels_per_sweep": 2})
    assert one > 0 and two >= one + 8 * 8 * m and two <= one + 8 * 8 * m + 512
    assert gf2.workspace_bytes(gf2.OP_PLS, m, n) == one  # small: one panel per sweep by default
    big = 30000
    assert gf2.workspace_bytes(gf2.OP_RANK, big, big) == gf2.workspace_bytes(gf2.OP_RANK, big, big,
                                                                             {"panels_per_sweep": 2})
    # the reduced-form routes of gf2_rref sweep one panel at a time whatever the option says
    assert gf2.workspace_bytes(gf2.OP_RREF, m, n, {"panels_per_sweep": 2, "rref_method": gf2.RREF_M4RI}) == \
        gf2.workspace_bytes(gf2.OP_RREF, m, n, {"panels_per_sweep": 1, "rref_method": gf2.RREF_M4RI})
    for bad in (-1, 3, 64):
        assert gf2.workspace_bytes(gf2.OP_PLS, m, n, {"panels_per_sweep": bad}) == 0
    L = gf2.lib()
    o = gf2.Opts()
    o.panels_per_sweep = 3
    fake = ctypes.c_void_p(1 << 20)
    P = Q = rank = ctypes.c_void_p(1 << 21)
    assert L.gf2_pls(fake, 8, 8, 16, P, Q, rank, None, 0, ctypes.byref(o), None) == 1  # GF2_EINVAL
