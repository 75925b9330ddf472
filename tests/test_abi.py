"""Host-side checks of libcbaa.so that need no GPU: exports, geometry rules, sizes."""
import glob
import os
import re

import pytest

import geometries as GEO
from paper_1901_06207_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def C():
    B.build()
    from paper_1901_06207_b300 import cbaa
    return cbaa


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(cbaa_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(C):
    names = _declared_functions()
    assert "cbaa_cube_update" in names and "cbaa_detect" in names
    lib = C.lib()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # every entry point is declared to ctypes: an undeclared one would pass
    # 64-bit pointers as masked C ints
    undeclared = [n for n in names if getattr(lib, n).argtypes is None]
    assert not undeclared, undeclared


def test_named_geometries_are_valid(C, oracle):
    for name, d in GEO.ALL.items():
        assert C.validate(d) == 0, name
        assert C.cube_bytes(d) == oracle.cube_words(d) * 4
    # Section V.C: the paper's setting is 128 MiB
    assert C.cube_bytes(GEO.PAPER) == 128 * 2 ** 20


def test_make_params_matches_table(C):
    assert C.make_params(4, 3, 1, 12, [12]) == GEO.with_form(GEO.PAPER, 0)
    assert C.make_params(5, 3, 1, 10, [12]) == GEO.with_form(GEO.L2, 0)
    assert C.make_params(6, 3, 1, 10, [13]) == GEO.with_form(GEO.SERVE, 0)
    assert C.make_params(6, 3, 1, 7, [10]) == GEO.with_form(GEO.TINY, 0)


def _bad(d, **kw):
    e = {k: (list(v) if isinstance(v, list) else v) for k, v in d.items()}
    e.update(kw)
    return e


@pytest.mark.parametrize("change", [
    dict(r=0), dict(r=17), dict(n_ra=1), dict(n_ra=7), dict(n_va=6), dict(log2_g=6), dict(log2_g=16),
    dict(threshold_form=2),
    dict(cbn=[4, 12, 12, 12, 0, 0, 0, 0]),
    dict(cbn=[12, 12, 8, 12, 0, 0, 0, 0]),          # |CP(2)| < 0
    dict(ring_off=[1, 10, 19, 0, 0, 0, 0, 0]),       # must start at 0
    dict(ring_off=[0, 19, 10, 0, 0, 0, 0, 0]),       # must increase
    dict(ring_off=[0, 10, 28, 0, 0, 0, 0, 0]),       # must stay inside LP
    dict(ring_off=[0, 3, 19, 0, 0, 0, 0, 0]),        # EP = (3, 16, 9): |CP(1)| = 12 - 16 < 0
    dict(ring_off=[0, 9, 12, 0, 0, 0, 0, 0], cbn=[16, 16, 16, 12, 0, 0, 0, 0]),  # |CP(0)| = 7 > |EP(1)| = 3
    dict(cbn=[12, 12, 12, 17, 0, 0, 0, 0]),          # column index wider than 16 bits
])
def test_invalid_geometries_rejected(C, change):
    d = _bad(GEO.PAPER, **change)
    assert C.validate(d) == C.ERR_INVALID_ARG
    assert C.cube_bytes(d) == 0
    assert C.workspace_bytes(d, 1024) == 0


def test_workspace_grows_with_candidates(C):
    a = C.workspace_bytes(GEO.L2, 1 << 10)
    b = C.workspace_bytes(GEO.L2, 1 << 20)
    assert 0 < a < b
    assert b - a >= ((1 << 20) - (1 << 10)) * 16 * 4   # two tuple buffers, hosts, sorted hosts


def test_status_strings(C):
    for st in range(0, -8, -1):
        assert C.status_str(st) and C.status_str(st) != "unknown status"
    assert C.status_str(-99) == "unknown status"


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1901_06207_b300 import cbaa
    monkeypatch.setattr(cbaa, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(cbaa, "_lib", None)
    with pytest.raises(ImportError):
        cbaa.lib()


def test_update_workspace_limits(C):
    """The partitioned update covers cubes up to 512 MiB; larger ones get no workspace size."""
    # A + 2 words per packet: A codes (column tiles), or a residual entry of the heavy split plus a
    # record and an overflow entry (row tiles)
    assert C.update_workspace_bytes(GEO.L2, 1 << 20) >= (1 << 20) * 4 * 6
    assert C.update_workspace_bytes(GEO.SERVE, 1) > 0
    big = C.make_params(8, 3, 1, 10, [13])          # 1 GiB cube
    assert C.validate(big) == C.OK and C.update_workspace_bytes(big, 1024) == 0
    assert C.update_workspace_bytes(GEO.L2, 0) == 0


def test_tuning_roundtrip_and_limits(C):
    before = C.get_tuning()
    C.set_tuning(scatter_shape=3, count_blocks_per_sm=4, apply_items_per_sm=16, direct_blocks_per_sm=2,
                 tile_kind=1, heavy=2, split_blocks=74)
    assert C.get_tuning() == dict(scatter_shape=3, count_blocks_per_sm=4, apply_items_per_sm=16,
                                  direct_blocks_per_sm=2, tile_kind=1, heavy=2, split_blocks=74)
    with pytest.raises(C.CbaaError):
        C.set_tuning(split_blocks=4097)
    with pytest.raises(C.CbaaError):
        C.set_tuning(tile_kind=4)
    with pytest.raises(C.CbaaError):
        C.set_tuning(heavy=4)
    with pytest.raises(C.CbaaError):
        C.set_tuning(scatter_shape=9)
    C.set_tuning(**before)
    assert C.get_tuning() == before


def test_multi_workspace_limits(C):
    assert C.update_multi_workspace_bytes(GEO.L2, 8, 1 << 20) > C.update_multi_workspace_bytes(GEO.L2, 1, 1 << 20)
    assert C.update_multi_workspace_bytes(GEO.L2, 9, 1 << 20) == 0        # 9 x 64 MiB > 512 MiB
    assert C.update_multi_workspace_bytes(GEO.TINY, 16, 1 << 10) > 0
    assert C.update_multi_workspace_bytes(GEO.TINY, 17, 1 << 10) == 0


def test_update_entry_points_reject_a_null_cube_before_any_device_work(C):
    """Argument checks that come before anything is enqueued (no device is touched): a null cube,
    for the plain, the partitioned and the assigning partitioned update."""
    lib = C.lib()
    assert lib.cbaa_cube_update(None, None, 1, None) == C.ERR_INVALID_ARG
    assert lib.cbaa_cube_update_binned(None, None, 1, None, 0, None) == C.ERR_INVALID_ARG
    assert lib.cbaa_cube_update_binned_assign(None, None, 1, None, 0, None) == C.ERR_INVALID_ARG
    assert lib.cbaa_cube_update_binned_assign(None, None, 0, None, 0, None) == C.ERR_INVALID_ARG
