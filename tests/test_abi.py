"""The C ABI: libwd.so builds for sm_103a, loads without a GPU and exports every
function include/wd.h declares; the Python binding declares each of them."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "wd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:wd_status|size_t|long long|const char \*)\s*(wd_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1810_04201_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared()
    for n in ("wd_apply", "wd_apply_dagger", "wd_normal_apply", "wd_cg_solve", "wd_create", "wd_set_gauge",
              "wd_pack", "wd_unpack", "wd_cg_solve_batched", "wd_autotune"):
        assert n in names
    assert len(names) >= 18


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol(lib):
    from paper_1810_04201_gb300 import wd
    src = open(wd.__file__).read()
    missing = [n for n in declared() if f'"{n}"' not in src]
    assert not missing, missing


def test_status_strings_and_argument_checks_without_gpu(lib):
    lib.wd_status_string.restype = ctypes.c_char_p
    assert lib.wd_status_string(0) == b"ok"
    assert lib.wd_status_string(7) == b"device-side wait timed out"
    ctx = ctypes.c_void_p()
    bad = (ctypes.c_int * 4)(4, 1, 4, 4)
    assert lib.wd_create(ctypes.byref(ctx), bad, 1, None) == 1  # WD_ERR_ARG before touching the device
    assert lib.wd_create(None, bad, 1, None) == 1
    assert lib.wd_destroy(None) == 1


def test_sources_name_no_batched_memcpy():
    """The batched-memcpy runtime calls are not used anywhere in the library sources."""
    d = os.path.join(ROOT, "paper_1810_04201_gb300", "csrc")
    pat = re.compile("Memcpy" + "(3D)?" + "Batch")
    for n in os.listdir(d):
        assert not pat.search(open(os.path.join(d, n)).read()), n


def test_header_is_plain_c_and_links(lib, tmp_path):
    """A C99 program that includes wd.h, takes the address of every declared function,
    links against libwd.so and calls the entry points that need no GPU."""
    import subprocess
    from paper_1810_04201_gb300 import build
    so = build.build()
    names = declared()
    prog = ["#include <stdio.h>", '#include "wd.h"', "int main(void) {",
            "    void *fns[] = {" + ", ".join(f"(void *)&{n}" for n in names) + "};",
            "    int dims[4] = {4, 1, 4, 4};",
            "    wd_ctx *ctx = 0;",
            "    if (wd_create(&ctx, dims, 1, 0) != WD_ERR_ARG) return 1;",
            "    if (!wd_status_string(WD_OK)) return 2;",
            '    printf("%d %s\\n", (int)(sizeof fns / sizeof fns[0]), wd_status_string(WD_ERR_ARG));',
            "    return 0;", "}"]
    c = tmp_path / "abi_check.c"
    c.write_text("\n".join(prog) + "\n")
    exe = tmp_path / "abi_check"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe),
                    "-L", os.path.dirname(so), "-lwd", "-Wl,-rpath," + os.path.dirname(so)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert int(out[0]) == len(names)


def test_struct_layouts_match_the_binding(tmp_path):
    """Every struct of wd.h has the size and field offsets of its ctypes mirror in the
    binding (a field added on one side only would shift the others)."""
    import subprocess
    from paper_1810_04201_gb300 import wd
    mirrors = {"wd_cg_params": wd.CGParams, "wd_cg_result": wd.CGResult, "wd_comm": wd.Comm}
    prog = ["#include <stdio.h>", "#include <stddef.h>", '#include "wd.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        prog.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            prog.append(f'    printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    prog += ["    return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(prog) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(c), "-o",
                    str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, value = line.split()
        got[cname, field] = int(value)
    for cname, py in mirrors.items():
        assert got[cname, "size"] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[cname, field] == getattr(py, field).offset, (cname, field)
