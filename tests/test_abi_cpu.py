"""CPU-side checks of the C ABI: the library builds, loads and exports every symbol the
header declares; the binding's config structure matches the header's field order."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    src = open(os.path.join(ROOT, "include", "ugks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ugks_[a-z0-9_]+)\s*\(", src)))


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


def test_state_bytes_without_gpu():
    """ugks_state_bytes is host arithmetic (no CUDA call): 0 for an invalid configuration;
    otherwise the f copies dominate it (FP64: plus the slope and face-flux buffers), with
    O(cells + faces) bytes of records on top, and it grows with the mesh."""
    from paper_1810_08137_gb300 import inputs as I
    from paper_1810_08137_gb300 import ugks
    assert ugks.state_bytes(I.channel_config(nx=0)) == 0
    cfg = I.channel_config(nx=40, ny=20, n_vel=20)
    nq, nx, ny = 400, 40, 20
    ring, wring = (nx + 4) * (ny + 4), (nx + 2) * (ny + 2)
    faces = (nx + 1) * ny + nx * (ny + 1)
    big64 = 2 * ring * nq * 16 + wring * nq * 32 + faces * nq * 16
    b64 = ugks.state_bytes(cfg, ugks.FP64)
    assert big64 < b64 < big64 + 2000 * (ring + faces)
    fs = 10 * 20  # 20 rows: 10 per half of the v axis, 5 row pairs each; 20 u values
    big32 = 2 * ring * fs * 16
    b32 = ugks.state_bytes(cfg, ugks.FP32F)
    stage = 2 * (32 << 20)  # the two staging halves of the host-state conversion
    assert big32 < b32 < big32 + stage + 2000 * (ring + faces)
    assert ugks.state_bytes(I.channel_config(nx=80, ny=40, n_vel=20), ugks.FP64) > b64


def test_shakhov_configuration_without_gpu():
    """The Prandtl number is validated before any CUDA call: a non-finite pr and the
    Shakhov model in the DF64 form are rejected; the Shakhov model adds its heat-flux
    moment sums (56 doubles per cell of the sums ring) and, in the FP32-f form, the cells'
    Shakhov records (96 bytes per cell) to the device bytes."""
    import math

    from paper_1810_08137_gb300 import inputs as I
    from paper_1810_08137_gb300 import ugks
    cfg = I.channel_config(nx=40, ny=20, n_vel=20)
    for pr, prec in ((math.nan, ugks.FP64), (2.0 / 3.0, ugks.DF64)):
        with pytest.raises(ugks.UGKSError) as e:
            ugks.Solver(cfg.replace(pr=pr), prec)
        assert e.value.status == 1
    wring, nc = 42 * 22, 40 * 20
    shk = cfg.replace(pr=2.0 / 3.0)
    assert ugks.state_bytes(shk, ugks.FP64) - ugks.state_bytes(cfg, ugks.FP64) == 56 * 8 * wring
    assert (ugks.state_bytes(shk, ugks.FP32F) - ugks.state_bytes(cfg, ugks.FP32F)
            == 56 * 8 * wring + 96 * nc)
    # a zero-initialised pr (<= 0) is BGK
    assert ugks.state_bytes(cfg.replace(pr=0.0), ugks.FP64) == ugks.state_bytes(cfg, ugks.FP64)
