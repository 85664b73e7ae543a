"""The C ABI library builds for sm_103a, loads, and exports every entry point include/mk.h declares (no GPU)."""
import ctypes
import subprocess

import pytest

from paper_2103_02824_gb300 import build, mk


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_declares_the_boundary():
    names = mk.header_symbols()
    for required in ("mk_mesh_upload", "mk_assemble_rhs", "mk_hartree_poisson", "mk_correction_solve",
                     "mk_augmented_project", "mk_small_eigensolve"):
        assert required in names


def test_library_exports_every_header_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in mk.header_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    for name in mk.header_symbols():
        assert f" T {name}" in out, name


def test_binding_covers_header(libpath):
    assert set(mk.header_symbols()) <= set(mk._SIGS)
    lib = mk.load(libpath)
    assert b"sm_103a" in lib.mk_version()


def test_no_device_fails_loudly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(mk.MkError) as e:
        mk.Context(0)
    assert e.value.code == mk.MK_ERR_CUDA


def test_binding_constants_match_header():
    """Every integer constant the header defines (#define or enum) that the binding also names has the same value
    there (the profiling kinds are PROF_* in the binding, MK_PROF_* in the header)."""
    import os
    import re
    text = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mk.h")).read()
    consts = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(MK_\w+)\s+(-?\d+)\s*$", text, re.M)}
    for body in re.findall(r"enum\s*\{([^}]*)\}", text):
        for m in re.finditer(r"(MK_\w+)\s*=\s*(-?\d+)", body):
            consts[m.group(1)] = int(m.group(2))
    checked = 0
    for name, value in consts.items():
        alias = name[3:] if name.startswith("MK_PROF_") else name
        if hasattr(mk, alias):
            assert getattr(mk, alias) == value, (name, getattr(mk, alias), value)
            checked += 1
    # the binding's string maps
    for table, prefix, names in ((mk.MK_XC, "MK_XC_", {"none": "NONE", "slater": "SLATER", "xalpha": "XALPHA",
                                                       "lda": "LDA_PZ"}),
                                 (mk.MK_PRECOND, "MK_PRECOND_", {k: k.upper() for k in mk.MK_PRECOND}),
                                 (mk.MK_BC, "MK_BC_", {k: k.upper() for k in mk.MK_BC})):
        for key, value in table.items():
            assert consts[prefix + names[key]] == value, (prefix, key)
            checked += 1
    for needed in ("MK_OPT_DECOMPOSE_CTAS", "MK_OPT_PAIR_RESIDUAL", "MK_PREC_PAIRS", "MK_PROF_PAIRS"):
        assert needed in consts, needed
    assert checked >= 25, checked
