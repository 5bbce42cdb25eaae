"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/fetidp.h declares
(no compute call: this runs without a GPU)."""
import os
import re

import pytest

from paper_2308_11371_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "fetidp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fetidp_[A-Za-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_header_declares_the_hot_path_entry_points():
    syms = declared_symbols()
    for s in ("fetidp_setup", "fetidp_apply_F", "fetidp_precond", "fetidp_solve", "fetidp_grad",
              "fetidp_destroy"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_symbols()) <= set(binding.SYMBOLS)


def test_default_options_and_status_strings(lib):
    o = binding.default_options()
    assert o.tol_outer == 1e-8 and o.tol_inner == 1e-11 and o.precision == binding.FETIDP_FP64
    assert o.tol_inner_mixed == 1e-6 and o.gram_drop_mixed == 1e-9 and o.tc_split == 3
    assert o.profile_mask == 0
    assert o.max_outer == 100 and o.restart == 0 and o.wait_budget_ns == 10 ** 9 and o.check_inputs == 1
    assert o.tc_bn == 0
    assert lib.fetidp_status_string(-4) == b"not converged"
    assert lib.fetidp_status_string(0) == b"ok"


def test_kernel_classes_match_the_header():
    with open(os.path.join(ROOT, "include", "fetidp.h")) as f:
        hdr = f.read()
    enum = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"FETIDP_K_(\w+)\s*=\s*(\d+)", hdr)}
    enum.pop("nclass")
    assert enum == {k.lower(): v for k, v in binding.KCLASS.items()}
    assert binding.class_mask(["sweep", "tc_gemm"]) == (1 << 9) | (1 << 7)
    assert binding.default_options(profile=["greedy"]).profile_mask == 1 << 11


def test_problem_struct_marshalling():
    from paper_2308_11371_gb300 import workloads as W
    p = W.bcc_3d_32x32x16()
    s, keep = binding.make_problem_struct(p)
    assert (s.dim, list(s.cells), s.elems, s.n_loads, s.n_rb) == (3, [32, 32, 16], 6, 6, 16)
    assert s.load_kind[3] == W.LOAD_BODY and s.load_dir[3 * 3 + 0] == 1.0
    assert abs(s.r_cell[0] - p.r_cell[0]) == 0.0


def test_setup_rejects_bad_input_without_gpu(lib):
    """Argument checks run before any CUDA call."""
    import ctypes
    from paper_2308_11371_gb300 import workloads as W
    p = W.frame_2d_4x4()
    p.n_rb = 0
    s, keep = binding.make_problem_struct(p)
    h = ctypes.c_void_p()
    st = lib.fetidp_setup(ctypes.byref(s), 2, None, None, ctypes.byref(h))
    assert st == -1 and not h.value


@pytest.mark.parametrize("case", ["batch_elems", "batch_loads", "tc_split", "gram_drop", "clamp_axis", "nu",
                                  "iterations", "restart", "wait_budget", "nan_radius", "inf_load", "nan_map",
                                  "nan_tol", "negative_E", "tc_bn"])
def test_setup_validation_without_gpu(lib, case):
    """Every argument and batch-compatibility check of fetidp_setup runs before any CUDA call and
    answers FETIDP_EINVAL (-1) with no context."""
    import ctypes
    from paper_2308_11371_gb300 import workloads as W
    a = W.frame_2d_4x4()
    probs = [a]
    opts = {}
    if case == "batch_elems":
        probs = [a, W.lattice_2d(3, 3, 6, n_rb=2)]             # 8 vs 6 elements per cell edge
    elif case == "batch_loads":
        b = W.frame_2d_4x4()
        b.loads = b.loads + b.loads                              # 1 vs 2 load cases
        probs = [a, b]
    elif case == "tc_split":
        opts = {"precision": binding.FETIDP_MIXED_BF16, "tc_split": 2}
    elif case == "gram_drop":
        opts = {"precision": binding.FETIDP_MIXED_BF16, "gram_drop_mixed": 1.5}
    elif case == "clamp_axis":
        a.clamp_axis = 2                                         # 2D lattice
    elif case == "nu":
        a.nu = 0.5
    elif case == "iterations":
        opts = {"max_outer": 0}
    elif case == "restart":
        opts = {"restart": -1}
    elif case == "wait_budget":
        opts = {"wait_budget_ns": 0}
    elif case == "nan_radius":
        a.r_cell = a.r_cell.copy(); a.r_cell[5] = float("nan")
    elif case == "inf_load":
        a.loads = [W.Load(W.LOAD_TRACTION, (0.0, float("inf")), axis=0, side=1)]
    elif case == "nan_map":
        a.map_params = (float("nan"), 4.0)
    elif case == "nan_tol":
        opts = {"tol_outer": float("nan")}
    elif case == "negative_E":
        a.E_void = -1e-3
    elif case == "tc_bn":
        opts = {"precision": binding.FETIDP_MIXED_BF16, "tc_bn": 96}
    arr = (binding.Problem * len(probs))()
    keep = []
    for i, q in enumerate(probs):
        s, k = binding.make_problem_struct(q)
        arr[i] = s
        keep.append(k)
    o = binding.default_options(**opts)
    h = ctypes.c_void_p()
    st = lib.fetidp_setup(arr, len(probs), ctypes.byref(o), None, ctypes.byref(h))
    assert st == -1 and not h.value
    expect = {"batch_elems": "must share", "batch_loads": "must share", "tc_split": "tc_split",
              "gram_drop": "gram_drop_mixed", "clamp_axis": "clamp axis", "nu": "nu out of range",
              "iterations": "iteration limits", "restart": "iteration limits",
              "wait_budget": "wait_budget_ns", "nan_radius": "non-finite", "inf_load": "non-finite",
              "nan_map": "non-finite", "nan_tol": "tolerances", "negative_E": "negative",
              "tc_bn": "tc_bn"}[case]
    assert expect in lib.fetidp_last_error().decode()


def test_zero_material_is_singular_without_gpu(lib):
    """E_solid = E_void = 0 leaves every cell stiffness zero: FETIDP_ESINGULAR (-6), no context."""
    import ctypes
    from paper_2308_11371_gb300 import workloads as W
    a = W.frame_2d_4x4()
    a.E_solid = 0.0
    a.E_void = 0.0
    s, keep = binding.make_problem_struct(a)
    h = ctypes.c_void_p()
    st = lib.fetidp_setup(ctypes.byref(s), 1, None, None, ctypes.byref(h))
    assert st == -6 and not h.value
    assert "zero" in lib.fetidp_last_error().decode()


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "fetidp.h"
int main(void) {
  fetidp_options o;
  fetidp_ctx *h = 0;
  fetidp_default_options(&o);
  if (o.tol_outer != 1e-8 || o.tc_split != 3 || o.profile_mask != 0u) return 1;
  if (strcmp(fetidp_status_string(FETIDP_ENOTCONV), "not converged") != 0) return 2;
  /* no lattice: EINVAL before any CUDA call, no context */
  if (fetidp_setup(0, 0, &o, 0, &h) != FETIDP_EINVAL || h) return 3;
  printf("%s\n", fetidp_last_error());
  return 0;
}
"""


def test_c_program_links_the_library(lib, tmp_path):
    """The boundary is a plain C ABI: a C99 program compiled against include/fetidp.h links the
    library and calls the entry points that need no GPU."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(build.LIB)
    libname = os.path.basename(build.LIB)[3:-3]          # libfetidp.so -> fetidp
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-L", libdir, f"-l{libname}", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, (run.returncode, run.stderr)
    assert "problem" in run.stdout
