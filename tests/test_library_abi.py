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


def test_nep_arguments_are_validated_on_the_host(libmod):
    """A NEP-style potential with a wrong weight count, non-finite weights,
    a missing weight array or a non-positive cutoff is rejected before any
    CUDA call."""
    import ctypes

    import numpy as np

    import cfneb_inputs as ci
    g = libmod
    with pytest.raises(ValueError):
        g.nep_potential(np.zeros(5), 2.1)
    R0, h0, R1, h1 = ci.graphite_hexdiamond_path((2, 2, 1))
    keep = []
    A = g.make_structure(R0, h0, keep)
    B = g.make_structure(R1, h1, keep)
    opt = g.default_options()
    out = ctypes.c_void_p()
    bad = []
    w = ci.nep_weights(3)
    w[10] = np.inf
    bad.append(g.nep_potential(w, 2.1))
    bad.append(g.nep_potential(ci.nep_weights(3), 0.0))
    bad.append(g.nep_potential(ci.nep_weights(3), float("nan")))
    p = g.Potential()
    p.kind, p.nep_rc = g.NEP, 2.1
    bad.append(p)
    for pot in bad:
        st = g.lib().cfneb_create_band(ctypes.byref(A), ctypes.byref(B), 5, ctypes.byref(pot),
                                       None, ctypes.byref(opt), None, ctypes.byref(out))
        assert st == g.ERR_INVALID_ARG
    # control: valid arguments pass the host checks (and then need a device)
    import torch
    if not torch.cuda.is_available():
        good = g.nep_potential(ci.nep_weights(3), 2.1)
        st = g.lib().cfneb_create_band(ctypes.byref(A), ctypes.byref(B), 5, ctypes.byref(good),
                                       None, ctypes.byref(opt), None, ctypes.byref(out))
        assert st != g.ERR_INVALID_ARG and st < 0


@pytest.mark.parametrize("case", ["inf_cell", "nan_eps", "inf_rc", "narrow_cell", "singular"])
def test_noalloc_rejects_invalid_input_before_gpu_work(libmod, case):
    """cfneb_lj_evaluate_noalloc validates its host arguments first: a
    non-finite cell entry or potential constant, a singular cell or a cell
    narrower than rc / 7 along a lattice direction (the cell list reaches 7
    bins to each side) return INVALID_ARG without touching the device (the
    device pointers here are never dereferenced)."""
    import numpy as np
    h = np.eye(3) * 10.0
    eps, sigma, rc = 1.0, 1.0, 2.5
    if case == "inf_cell":
        h[1, 2] = np.inf
    elif case == "nan_eps":
        eps = float("nan")
    elif case == "inf_rc":
        rc = float("inf")
    elif case == "narrow_cell":
        h[2, 2] = 0.3  # rc / 7 = 0.357
    else:
        h[2] = h[1]
    st = libmod.lj_evaluate_noalloc(16, 4, h, eps, sigma, rc, 1, 0, 0, 0)
    assert st == libmod.ERR_INVALID_ARG


def test_coincident_endpoints_are_rejected_on_the_host(libmod):
    """Endpoints with every atom on the same periodic site (here: the final
    structure is the initial one with a few atoms shifted by whole lattice
    vectors), and the same cell, leave no path: cfneb_create_band returns
    INVALID_ARG before any CUDA call, with the cell filter on or off."""
    import ctypes

    import numpy as np

    import cfneb_inputs as ci
    g = libmod
    R0, h0, _, _ = ci.lj_vacancy_hop(ci.LJ_A, (2, 2, 2))
    R1 = R0.copy()
    R1[:5] += h0[0]
    R1[7] -= h0[2]
    keep = []
    A = g.make_structure(R0, h0, keep)
    B = g.make_structure(R1, h0, keep)
    opt = g.default_options()
    pot = g.lj_potential()
    out = ctypes.c_void_p()
    for enabled in (0, 1):
        cf = g.CellFilter(enabled, g.ROTFREE_B, 0.0, 0.0)
        st = g.lib().cfneb_create_band(ctypes.byref(A), ctypes.byref(B), 5, ctypes.byref(pot),
                                       ctypes.byref(cf), ctypes.byref(opt), None,
                                       ctypes.byref(out))
        assert st == g.ERR_INVALID_ARG
    # control: one atom off its site passes the host checks (and then needs
    # a device)
    import torch
    if not torch.cuda.is_available():
        R2 = R1.copy()
        R2[3] += 0.1
        C = g.make_structure(R2, h0, keep)
        st = g.lib().cfneb_create_band(ctypes.byref(A), ctypes.byref(C), 5, ctypes.byref(pot),
                                       None, ctypes.byref(opt), None, ctypes.byref(out))
        assert st != g.ERR_INVALID_ARG and st < 0


def test_empty_and_short_bands_are_rejected_on_the_host(libmod):
    """A structure without atoms, endpoints of different sizes, and a band
    of fewer than three images (no moving image) are refused before any
    CUDA call."""
    import ctypes

    import numpy as np

    import cfneb_inputs as ci
    g = libmod
    R0, h0, R1, h1 = ci.lj_vacancy_hop(ci.LJ_A, (2, 2, 2))
    keep = []
    A = g.make_structure(R0, h0, keep)
    B = g.make_structure(R1, h1, keep)
    E = g.make_structure(np.zeros((0, 3)), h0, keep)
    S = g.make_structure(R1[:-1], h1, keep)
    opt = g.default_options()
    pot = g.lj_potential()
    out = ctypes.c_void_p()
    create = g.lib().cfneb_create_band
    for (a, b, n, want) in ((E, E, 5, g.ERR_INVALID_ARG), (A, B, 2, g.ERR_INVALID_ARG),
                            (A, S, 5, g.ERR_SHAPE_MISMATCH)):
        st = create(ctypes.byref(a), ctypes.byref(b), n, ctypes.byref(pot), None,
                    ctypes.byref(opt), None, ctypes.byref(out))
        assert st == want, (n, st)
