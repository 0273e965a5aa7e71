"""CPU-side checks of the C ABI: the library builds, loads and exports every symbol the
header declares; the binding's config structure matches the header's field order."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    src = open(os.path.join(ROOT, "include", "ugks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ugks_[a-z_]+)\s*\(", src)))


def test_header_declares_expected_calls():
    syms = header_symbols()
    for s in ("ugks_create", "ugks_set_state", "ugks_step", "ugks_moments", "ugks_destroy"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_1810_08137_gb300 import build, ugks
    build.build()
    L = ugks.lib()
    missing = [s for s in header_symbols() if not hasattr(L, s)]
    assert not missing, missing
    assert sorted(ugks.EXPORTS) == header_symbols()


def test_config_struct_matches_header():
    from paper_1810_08137_gb300 import ugks
    src = open(os.path.join(ROOT, "include", "ugks.h")).read()
    body = re.search(r"typedef struct \{([^{}]*)\} ugks_config;", src).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        parts = decl.replace(",", " ").split()
        ty, rest = parts[0], parts[1:]
        names += [n.split("[")[0] for n in rest]
    assert names == [f[0] for f in ugks._Config._fields_]


def test_create_rejects_bad_config_without_gpu():
    """Validation happens before any CUDA call, so it runs here without a GPU."""
    from paper_1810_08137_gb300 import inputs as I
    from paper_1810_08137_gb300 import ugks
    bad = I.channel_config(nx=0)
    with pytest.raises(ugks.UGKSError) as e:
        ugks.Solver(bad)
    assert e.value.status == 1
    bad = I.channel_config(n_vel=600)
    with pytest.raises(ugks.UGKSError):
        ugks.Solver(bad)
    bad = I.channel_config()
    bad.bc = [I.BC(I.BC_PERIODIC), I.BC(I.BC_WALL), I.BC(I.BC_WALL), I.BC(I.BC_WALL)]
    with pytest.raises(ugks.UGKSError):
        ugks.Solver(bad)
