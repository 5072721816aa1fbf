"""The C-ABI library builds, loads, and exports every entry point include/lq.h declares.

CPU only: no call here touches a GPU (argument validation fails before any
CUDA call is made).
"""
import ctypes
import os
import re

import pytest

from helpers import ROOT, ensure_library


def header_functions():
    src = open(os.path.join(ROOT, "include", "lq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lq_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ["lq_create_lattice", "lq_load_gauge", "lq_load_clover", "lq_dslash_apply", "lq_solve",
                     "lq_submit", "lq_poll"]:
        assert required in names


def declaration_comments():
    """Each declared entry point with the comment text that precedes its declaration
    (back to the previous declaration, or to a blank line above its comment)."""
    src = open(os.path.join(ROOT, "include", "lq.h")).read()
    # the same text with every ';' inside a comment blanked, so that only code ends a declaration
    code = re.sub(r"/\*.*?\*/", lambda c: c.group(0).replace(";", " "), src, flags=re.S)
    out = {}
    for m in re.finditer(r"^(?:int|int64_t|const char\*)\s+(lq_[a-z_0-9]+)\s*\(", src, flags=re.M):
        before = src[: m.start()]
        end = code[: m.start()].rfind(";")
        chunk = before[end + 1:]
        out[m.group(1)] = " ".join(re.findall(r"/\*(.*?)\*/", chunk, flags=re.S))
    return out


def test_every_entry_point_names_its_passage():
    """Every exported call's comment says which passage of the paper defines what it
    computes (a section, equation or table), or that the paper has no counterpart."""
    comments = declaration_comments()
    assert sorted(comments) == header_functions()
    for name, text in comments.items():
        cited = re.search(r"Paper:.*?(Sec\. \d|Eq\. \d|Table \d)", text, flags=re.S)
        none = "no counterpart" in text
        assert cited or none, name


def test_library_exports_every_declared_symbol():
    ensure_library()
    from paper_2201_09004_b300 import lib
    L = lib.lib()
    names = header_functions()
    assert sorted(lib.EXPORTS) == names
    for n in names:
        assert hasattr(L, n), n


def test_invalid_lattice_is_rejected_without_gpu():
    ensure_library()
    from paper_2201_09004_b300 import lib
    h = ctypes.c_void_p()
    code = lib.lib().lq_create_lattice((ctypes.c_int * 4)(4, 4, 5, 8), ctypes.c_int(-1), ctypes.byref(h))
    assert code == lib.LQ_EINVAL
    assert b"even" in lib.lib().lq_last_error()
    code = lib.lib().lq_create_lattice((ctypes.c_int * 4)(4, 4, 4, 8), ctypes.c_int(3), ctypes.byref(h))
    assert code == lib.LQ_EINVAL
    code = lib.lib().lq_server_create(ctypes.c_size_t(1 << 30), ctypes.c_int(0), ctypes.byref(h))
    assert code == lib.LQ_EINVAL
    with pytest.raises(lib.LqError):
        lib.Lattice((2, 2, 2, 3))


def test_null_handles_and_bad_arguments_are_rejected_without_gpu():
    """Every entry point that takes a lattice checks it (and its arguments) before
    touching the GPU: a null handle or a bad enum is LQ_EINVAL with a message."""
    ensure_library()
    from paper_2201_09004_b300 import lib
    L = lib.lib()
    buf = (ctypes.c_double * 8)()
    info = lib.SignInfo()
    assert L.lq_gamma5_dw_apply(None, ctypes.c_double(1.5), 0, 0, buf, buf, None) == lib.LQ_EINVAL
    assert L.lq_overlap_sign_apply(None, ctypes.c_double(1.5), ctypes.c_double(0.1), ctypes.c_double(8.0),
                                   ctypes.c_double(1e-5), 0, 0, buf, buf, ctypes.byref(info), None) == lib.LQ_EINVAL
    assert b"lattice" in L.lq_last_error()
    op = lib.op_params(lib.WILSON_TM, 0.1, 0.05)
    sp = lib.solve_params(solver=lib.BICGSTAB)
    ptrs = (ctypes.POINTER(ctypes.c_double) * 1)()
    assert L.lq_solve(None, ctypes.byref(op), ctypes.byref(sp), 1, ptrs, ptrs, 0, None, None) == lib.LQ_EINVAL
    assert L.lq_tune_force(-1) == lib.LQ_EINVAL
    assert L.lq_tune_force(0) == lib.LQ_OK
    assert L.lq_lattice_release_workspace(None, None) == lib.LQ_EINVAL
    ep = lib.EigParams(4, 0, 0, 1.0, 10.5, 1e-8, 0)
    evals = (ctypes.c_double * 4)()
    assert L.lq_hw_eigensolve(None, ctypes.c_double(1.5), ctypes.byref(ep), 0, evals, None, None, None) == lib.LQ_EINVAL
    assert L.lq_overlap_sign_apply_deflated(None, ctypes.c_double(1.5), ctypes.c_double(0.5), ctypes.c_double(10.5),
                                            ctypes.c_double(1e-8), 0, None, None, 0, buf, buf, None,
                                            None) == lib.LQ_EINVAL


def test_ctypes_structures_match_the_header_layout(tmp_path):
    """Every struct the binding marshals has the header's size and field offsets
    (a C program compiled against include/lq.h prints them)."""
    import subprocess
    from paper_2201_09004_b300 import lib
    structs = {"lq_op_params": lib.OpParams, "lq_solve_params": lib.SolveParams, "lq_solve_info": lib.SolveInfo,
               "lq_sign_info": lib.SignInfo, "lq_request": lib.Request, "lq_request_times": lib.RequestTimes,
               "lq_eig_params": lib.EigParams, "lq_eig_info": lib.EigInfo}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lq.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
