"""The C-ABI libraries load and export every symbol include/*.h declares.

No compute call is made (no GPU needed).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kkt_schur.h")


def declared_functions(header=HEADER):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kkt_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ["kkt_analyze", "kkt_factor", "kkt_solve", "kkt_get_info", "kkt_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1907_05420_gb300 import binding

    try:
        lib = binding.load()
    except OSError as e:  # the CUDA runtime library itself is missing
        pytest.skip(f"cannot load libkkt_schur.so here: {e}")
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert sorted(binding.EXPORTS) == declared_functions()


def test_symbolic_library_exports_its_header():
    from paper_1907_05420_gb300 import build as lib_build

    lib = ctypes.CDLL(lib_build.build_symbolic())
    names = declared_functions(os.path.join(ROOT, "include", "kkt_symbolic.h"))
    assert names == ["kkt_symbolic_choose_tail", "kkt_symbolic_create", "kkt_symbolic_destroy",
                     "kkt_symbolic_error", "kkt_symbolic_get"]
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_without_gpu():
    from paper_1907_05420_gb300 import binding

    lib = binding.load()
    assert lib.kkt_status_string(0) == b"ok"
    assert lib.kkt_status_string(6) == b"refinement did not converge"
    opt = binding.kkt_default_options()
    assert opt.refine_tol == 1e-10 and opt.max_refine == 10 and opt.prec == 0
    assert opt.tail_ratio == 0.0 and opt.dense_tail == -1 and opt.use_graphs == 1
    assert opt.refine_mode == 0 and opt.gmres_restart == 8 and opt.device_refine == 0


def test_inertia_defaults_without_gpu():
    """The documented trial constants of the inertia correction."""
    from paper_1907_05420_gb300 import binding

    o = binding.kkt_default_inertia_options()
    assert (o.delta_w_init, o.delta_w_min, o.delta_w_max) == (1e-4, 1e-20, 1e40)
    assert (o.grow_first, o.grow, o.delta_c, o.max_trials) == (100.0, 8.0, 1e-8, 40)
    assert o.shrink == 1.0 / 3.0


def test_struct_layouts_match_header(tmp_path):
    """ctypes structures have the C compiler's sizes and offsets for the header."""
    import subprocess

    from paper_1907_05420_gb300 import binding

    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "kkt_schur.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\","
        "sizeof(kkt_pattern), offsetof(kkt_pattern, a_vals_hint),"
        "sizeof(kkt_options), offsetof(kkt_options, reduced_contraction),"
        "offsetof(kkt_options, dense_tail), offsetof(kkt_options, tail_ratio),"
        "offsetof(kkt_options, device_refine),"
        "sizeof(kkt_info), offsetof(kkt_info, n_launches), offsetof(kkt_info, tail_ratio),"
        "sizeof(kkt_inertia_options), offsetof(kkt_inertia_options, max_trials),"
        "sizeof(kkt_inertia_result), offsetof(kkt_inertia_result, trials));"
        "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [ctypes.sizeof(binding.kkt_pattern), binding.kkt_pattern.a_vals_hint.offset,
            ctypes.sizeof(binding.kkt_options), binding.kkt_options.reduced_contraction.offset,
            binding.kkt_options.dense_tail.offset, binding.kkt_options.tail_ratio.offset,
            binding.kkt_options.device_refine.offset,
            ctypes.sizeof(binding.kkt_info), binding.kkt_info.n_launches.offset,
            binding.kkt_info.tail_ratio.offset,
            ctypes.sizeof(binding.kkt_inertia_options), binding.kkt_inertia_options.max_trials.offset,
            ctypes.sizeof(binding.kkt_inertia_result), binding.kkt_inertia_result.trials.offset]
    assert got == want


def test_kernel_families_agree_with_the_header():
    """kkt_kernel_stats' families: the binding's names, the header's documented
    range and the library's family enumeration have the same count, in the
    header's order (each documented family names its kernel)."""
    from paper_1907_05420_gb300 import binding

    enum = open(os.path.join(ROOT, "paper_1907_05420_gb300", "csrc", "handle.h")).read()
    body = re.search(r"enum KernelFamily \{(.*?)\};", enum, flags=re.S).group(1)
    members = [m.strip().split("=")[0].strip() for m in body.split(",") if m.strip()]
    assert members[-1] == "kNumFamilies"
    count = len(members) - 1
    assert len(binding.KERNEL_FAMILIES) == count
    header = open(HEADER).read()
    assert f"(0..{count - 1})" in header
    doc = header[header.index("Families:"):header.index("typedef struct", header.index("Families:"))]
    for f, name in enumerate(binding.KERNEL_FAMILIES):
        # "<f> the ... (name" or "<f> the ... (name, ...": each number precedes its kernel's name
        pos_f = re.search(rf"\b{f} (the|an?) ", doc)
        assert pos_f, (f, name)
        assert name in doc[pos_f.start():], (f, name)
