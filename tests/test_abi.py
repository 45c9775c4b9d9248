"""The C-ABI library loads and exports every symbol include/dm.h declares.

No compute call needs a GPU here: only the host-side geometry is exercised,
and compared with the oracle's independent geometry.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "dm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:dm_status|void|const char\*)\s+(dm_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1506_07656_gb300 import build, dm
    build.build()
    return dm.load()


def test_header_declares_expected_calls():
    names = _declared()
    for must in ("dm_create", "dm_descriptors", "dm_correlate_pyramid", "dm_backtrack", "dm_match"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1506_07656_gb300 import dm
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(dm.exported_symbols()) == _declared()


def test_geometry_matches_oracle(lib, oracle_mod):
    from paper_1506_07656_gb300 import dm
    for (W1, H1, W2, H2) in [(64, 48, 64, 48), (37, 29, 41, 23), (1024, 436, 1024, 436), (1242, 375, 1242, 375),
                             (512, 224, 512, 224), (5, 4, 1, 1), (320, 240, 320, 240), (7, 5, 3, 2),
                             (621, 188, 621, 188), (80, 20, 80, 20), (20, 80, 20, 80), (256, 112, 300, 90),
                             (5, 100, 5, 100), (130, 70, 130, 70)]:
        a = dm.dm_geometry(W1, H1, W2, H2)
        b = oracle_mod.geometry(W1, H1, W2, H2)
        assert a["L"] == b.L and a["n_patch0"] == b.P0x * b.P0y and a["n_patch"] == b.Lx * b.Ly
        assert a["dw"] == b.dw and a["dh"] == b.dh


def test_geometry_rejects_degenerate_sizes(lib):
    from paper_1506_07656_gb300 import dm
    for bad in [(3, 10, 5, 5), (4, 4, 5, 5), (10, 10, 0, 5), (0, 0, 0, 0)]:
        with pytest.raises(dm.DmError) as e:
            dm.dm_geometry(*bad)
        assert e.value.status == dm.DM_EINVAL
    # merge keys beyond 32 bits take 64-bit keys: a 4096 x 4096 pair is accepted;
    # atomic indices (patch * 16 + offset) beyond 32 bits and more than 14
    # levels (fixed-point path scores) are refused
    assert dm.dm_geometry(4096, 4096, 4096, 4096)["L"] == 10
    for big in [(70000, 70000, 8, 8), (8, 8, 70000, 70000)]:
        with pytest.raises(dm.DmError) as e:
            dm.dm_geometry(*big)
        assert e.value.status == dm.DM_EUNSUPPORTED


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    from paper_1506_07656_gb300 import dm
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(dm.DmError) as e:
        dm.dm_create(dm.dm_config_default(), 0)
    assert e.value.status == dm.DM_EINVAL


def test_config_defaults_are_the_papers(lib):
    from paper_1506_07656_gb300 import dm
    c = dm.dm_config_default()
    vals = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_constants.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    assert abs(c.lambda_ - vals["lambda"]) < 1e-6 and abs(c.mu - vals["mu"]) < 1e-6
    assert abs(c.slope - vals["slope"]) < 1e-6
    assert (c.nu1, c.nu2, c.nu3) == (vals["nu1"], vals["nu2"], vals["nu3"])
    assert c.precision == dm.DM_FP32
    assert c.compensated == 1
