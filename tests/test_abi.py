"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/*.h declares (no compute calls here)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(dcg_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2511_23030_b300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["dcg_create", "dcg_chunk_table_update", "dcg_cull_chunks", "dcg_gather_active", "dcg_render_fwd",
              "dcg_render_bwd", "dcg_scatter_back"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.check_output(["nm", "-D", "--defined-only", libpath]).decode()
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_without_gpu(libpath):
    from paper_2511_23030_b300 import dcg

    L = dcg.lib()
    for n in declared_functions():
        assert hasattr(L, n)
    c = dcg.config()
    assert c.sh_degree == 3 and c.tile_w == 16 and c.page_gaussians == 2048


def test_no_library_means_no_fallback(tmp_path, monkeypatch):
    from paper_2511_23030_b300 import dcg

    monkeypatch.setattr(dcg, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(dcg, "_lib", None)
    with pytest.raises(ImportError):
        dcg.lib()


def test_build_targets_sm_103a_only():
    from paper_2511_23030_b300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_fault_specification_parses_on_the_host(libpath):
    """DCG_FAULT=kind[:skip], read at dcg_create, parsed by a host-only call."""
    from paper_2511_23030_b300 import dcg

    assert dcg.dcg_fault_parse("h2d_fail") == (1, 0)
    assert dcg.dcg_fault_parse("short_copy:3") == (2, 3)
    assert dcg.dcg_fault_parse("budget:0") == (3, 0)
    assert dcg.dcg_fault_parse("none") == (0, 0)
    for bad in ("h2d", "budget:", "budget:-1", "short_copy:1x", "budget:12345678901"):
        with pytest.raises(dcg.DcgError) as e:
            dcg.dcg_fault_parse(bad)
        assert e.value.status == 1


def test_bounds_check_build_exports_the_same_symbols(libpath):
    """libdcg_checks.so (-DDCG_CHECKS=1) is the same library with index checks in its kernels."""
    from paper_2511_23030_b300 import build

    checks = build.build(checks=True)
    assert checks.endswith("libdcg_checks.so")

    def exported(p):
        out = subprocess.check_output(["nm", "-D", "--defined-only", p]).decode()
        return {l.split()[-1] for l in out.splitlines() if " T " in l and l.split()[-1].startswith("dcg_")}

    assert exported(checks) == exported(libpath)
    assert not [n for n in declared_functions() if n not in exported(checks)]
