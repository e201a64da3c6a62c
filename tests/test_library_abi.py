"""CPU checks of the C ABI: the library builds, loads, and exports every
entry point that include/cfneb.h declares (no GPU calls)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "cfneb.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cfneb_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libmod():
    import paper_2510_16721_gb300 as g
    g.build()
    return g


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("cfneb_create_band", "cfneb_step", "cfneb_relax", "cfneb_insert_image",
                     "cfneb_delete_image", "cfneb_get_path", "cfneb_destroy_band"):
        assert required in names


def test_library_exports_every_declared_symbol(libmod):
    exported = subprocess.run(["nm", "-D", "--defined-only", libmod.LIB_PATH],
                              capture_output=True, text=True, check=True).stdout
    syms = set(re.findall(r"\bT (cfneb_\w+)", exported))
    missing = [n for n in _declared() if n not in syms]
    assert not missing, missing
    L = libmod.lib()
    for n in _declared():
        getattr(L, n)
    assert sorted(libmod.EXPORTS) == _declared()


def test_host_only_calls(libmod):
    """Calls that touch no device: argument validation and names."""
    assert libmod.status_string(libmod.ERR_NOT_SPD).startswith("lattice")
    o = libmod.default_options()
    assert o.k_spring == 0.1 and o.climb == 1 and o.dt == 0.1 and o.alpha_ins == 1.5
    L = libmod.lib()
    assert L.cfneb_kernel_count() >= 10
    names = [L.cfneb_kernel_name(k).decode() for k in range(L.cfneb_kernel_count())]
    assert "tersoff_partials" in names and "fire_update" in names
    # NULL arguments are rejected before any CUDA call
    assert L.cfneb_create_band(None, None, 7, None, None, None, None, None) == \
        libmod.ERR_INVALID_ARG
    assert L.cfneb_step(None, 1) == libmod.ERR_INVALID_ARG
    assert L.cfneb_destroy_band(None) == libmod.ERR_INVALID_ARG


def test_sources_target_sm103a_only():
    from paper_2510_16721_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
