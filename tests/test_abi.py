"""CPU checks of the C ABI boundary: the library builds, loads without a GPU, and exports
every function include/ttm.h declares. No compute call is made here."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "ttm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(ttm_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import paper_2410_19747_gb300 as pkg
    pkg.build()
    return pkg.load_library()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ["ttm_create", "ttm_destroy", "ttm_multiply", "ttm_multiply_batched", "ttm_backward"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    import paper_2410_19747_gb300 as pkg
    names = _declared_functions()
    assert sorted(names) == sorted(pkg.EXPORTED)
    for n in names:
        assert hasattr(lib, n), n
    assert lib.ttm_version().decode().startswith("ttm-gb300")


def test_invalid_arguments_are_rejected_without_gpu(lib):
    import ctypes
    import paper_2410_19747_gb300.binding as b
    # NULL handle and NULL descriptors are rejected before any CUDA call
    assert lib.ttm_multiply(None, None, None, None, None) == -1
    assert lib.ttm_create(None, 0, None, None) == -1
    o = b.make_options(eps=1.5)
    h = ctypes.c_void_p()
    assert lib.ttm_create(ctypes.byref(h), 0, None, ctypes.byref(o)) == -1
    assert b"eps" in lib.ttm_last_error()
    # shape validation in ttm_output_capacity (host-only planning)
    import numpy as np
    A = [np.zeros((1, 2, 2)), np.zeros((2, 2, 1))]
    B = [np.zeros((1, 2, 2)), np.zeros((2, 2, 1))]
    assert b.output_capacity(A, B) == 2 * 2 * 2 or b.output_capacity(A, B) > 0
    bad = [np.zeros((2, 2, 3)), np.zeros((3, 2, 1))]   # boundary bond 2 != 1
    assert b.output_capacity(bad, B) == -1


def test_option_validation_without_gpu(lib):
    """ttm_create validates the options before its first CUDA call."""
    import ctypes
    import paper_2410_19747_gb300.binding as b
    h = ctypes.c_void_p()
    for kw, status in ((dict(jacobi_kernel=5), -1), (dict(f32_passes=9), -1), (dict(f32_passes=-1), -1),
                       (dict(newton_steps=9), -1), (dict(newton_steps=-1), -1), (dict(use_graph=2), -1),
                       (dict(use_graph=1, profile=1), -9)):
        o = b.make_options(**kw)
        assert lib.ttm_create(ctypes.byref(h), 0, None, ctypes.byref(o)) == status, kw
    # accepted options get past validation: without a GPU the next step is a CUDA error
    for kw in (dict(jacobi_kernel=8), dict(jacobi_kernel=16), dict(f32_passes=1), dict(chi_max=16, chi_out=8),
               dict(chi_max=0, chi_out=8), dict(newton_steps=1, chi_max=16), dict(use_graph=1)):
        o = b.make_options(**kw)
        st = lib.ttm_create(ctypes.byref(h), 0, None, ctypes.byref(o))
        assert st not in (-1, -9), (kw, st, lib.ttm_last_error())
        if st == 0:
            lib.ttm_destroy(h)


def test_planner_schedules_the_final_rounding_without_gpu(lib):
    """The host planner walks the whole schedule, final rounding included, with no GPU."""
    import numpy as np
    import paper_2410_19747_gb300.binding as b
    import ttgen
    A = ttgen.rand_tt(10, 2, 16, 1, canon="left")
    B = ttgen.rand_tt(10, 2, 16, 2, canon="left")
    plain = b.output_capacity(A, B, chi_max=32, chi_out=32)
    assert plain > 0
    for kw in (dict(chi_max=32, chi_out=12), dict(chi_max=32, chi_out=1), dict(chi_max=0, chi_out=12)):
        cap = b.output_capacity(A, B, **kw)
        assert cap >= min(plain, 32 * 2 * 32), kw
    # the kept/dropped polish adds bond ids to the plan but no carriage
    assert b.output_capacity(A, B, chi_max=32, chi_out=32, newton_steps=2) == plain
    assert np.isfinite(plain)


def test_header_is_plain_c_and_links(lib, tmp_path):
    """A C99 program that includes only include/ttm.h compiles warning-free, links against
    libttm.so and passes the calls that need no GPU."""
    import shutil
    import subprocess
    import paper_2410_19747_gb300 as pkg
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    libpath = pkg.library_path()
    exe = str(tmp_path / "abi_check")
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "abi_check.c"),
           "-o", exe, libpath, "-Wl,-rpath," + os.path.dirname(libpath)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "c abi check ok" in r.stdout
    # the ctypes mirrors in the binding have the header's layout, field by field
    import ctypes
    import paper_2410_19747_gb300.binding as b
    mirrors = {"ttm_tt": b.c_tt, "ttm_options": b.c_options, "ttm_report": b.c_report}
    seen = {k: set() for k in mirrors}
    for line in r.stdout.splitlines():
        if not line.startswith("layout "):
            continue
        _, name, off, size = line.split()
        struct, field = name.split(".")
        py = mirrors[struct]
        if field == "sizeof":
            assert ctypes.sizeof(py) == int(size), (struct, ctypes.sizeof(py), size)
            continue
        desc = getattr(py, field)
        assert (desc.offset, desc.size) == (int(off), int(size)), (name, desc.offset, desc.size, off, size)
        seen[struct].add(field)
    for struct, py in mirrors.items():
        assert seen[struct] == {f for f, _ in py._fields_}, struct
