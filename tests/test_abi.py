"""The C-ABI library builds, loads and exports every entry point that
include/eco.h declares; configuration errors are reported without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "eco.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eco_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libeco():
    from paper_2510_18221_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(libeco):
    names = _declared()
    assert "eco_create" in names and "eco_step" in names and "eco_read_stats" in names
    for n in names:
        assert hasattr(libeco, n), n


def test_binding_wraps_every_declared_symbol():
    from paper_2510_18221_gb300 import eco
    src = open(eco.__file__).read()
    for n in _declared():
        assert n in src, n


def test_config_validation_without_gpu(libeco):
    from paper_2510_18221_gb300 import eco, workloads
    eco._lib = None
    cfg, keep = eco.make_config([workloads.get("small")])
    assert eco.eco_workspace_bytes(cfg) > 0
    P, D = eco.eco_param_count(cfg)
    assert (P, D) == (3814, 79)
    bad, keep2 = eco.make_config([workloads.get("small", side=63)])
    with pytest.raises(eco.EcoError) as ex:
        eco.eco_workspace_bytes(bad)
    assert ex.value.code == eco.ECO_EINVAL and "side" in str(ex.value)
    bad, keep3 = eco.make_config([workloads.get("small", hidden=48)])
    with pytest.raises(eco.EcoError):
        eco.eco_param_count(bad)
    cfg.abi_version = 99
    with pytest.raises(eco.EcoError) as ex:
        eco.eco_param_count(cfg)
    assert ex.value.code == eco.ECO_EABI


def test_workspace_sizes_paper_scale(libeco):
    from paper_2510_18221_gb300 import eco, workloads
    cfg, keep = eco.make_config([workloads.get("paper")])
    n = eco.eco_workspace_bytes(cfg)
    # FP32 masters (>= 28,553 * 4 B) + BF16 copy (>= 57,380 B) per slot
    assert n >= 65536 * (28553 * 4 + 57380)
    assert n < 65536 * (28553 * 4 + 57380) * 1.02 + 64 * 2**20


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2510_18221_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "eco_oracle" not in txt, f
