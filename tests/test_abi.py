"""The C-ABI library builds, loads and exports every symbol include/mx.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(mx_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libmx():
    from paper_2602_12242_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path():
    names = declared_functions()
    for n in ("mx_create", "mx_build_demag_kernel", "mx_heff", "mx_llg_rhs", "mx_rk_step", "mx_energy",
              "mx_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(libmx):
    missing = [n for n in sorted(declared_functions()) if not hasattr(libmx, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2602_12242_gb300 import _lib
    assert set(_lib.SIGNATURES) >= declared_functions()


def test_params_struct_layout_matches_header(tmp_path):
    """Field offsets of the ctypes mirror equal those a C compiler gives the header."""
    from paper_2602_12242_gb300 import _lib
    fields = [f for f, _ in _lib.mx_params._fields_]
    src = tmp_path / "layout.c"
    body = "".join(f'printf("%zu ", offsetof(mx_params, {f}));' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mx.h"\n'
                   'int main(void){' + body + 'printf("%zu", sizeof(mx_params)); return 0;}')
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [getattr(_lib.mx_params, f).offset for f in fields] + [ctypes.sizeof(_lib.mx_params)]
    assert got == want


def test_version_string_without_gpu(libmx):
    libmx.mx_version.restype = ctypes.c_char_p
    assert b"sm_103a" in libmx.mx_version()


def test_null_arguments_rejected_without_gpu(libmx):
    from paper_2602_12242_gb300 import _lib
    L = _lib.lib()
    assert L.mx_create(None, None) == _lib.MX_ERR_INVALID_ARG
    assert b"NULL" in L.mx_last_error()
    assert L.mx_heff(None, None, None, 31, None) == _lib.MX_ERR_INVALID_ARG
    assert L.mx_destroy(None) == _lib.MX_OK


def test_header_is_strict_c99_and_cxx11(tmp_path):
    """include/mx.h is usable from plain C (C99, pedantic, warnings as errors)
    and from C++ with no CUDA or torch headers."""
    import subprocess
    c = tmp_path / "use.c"
    c.write_text('#include "mx.h"\nint main(void) { mx_ctx *c = 0; return mx_destroy(c); }\n')
    subprocess.run(["gcc", "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-I",
                    os.path.join(ROOT, "include"), str(c)], check=True)
    cc = tmp_path / "use.cpp"
    cc.write_text('#include "mx.h"\nint main() { mx_ctx *c = nullptr; return mx_destroy(c); }\n')
    subprocess.run(["g++", "-std=c++11", "-pedantic", "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-I",
                    os.path.join(ROOT, "include"), str(cc)], check=True)


def test_plain_c_program_links_and_calls_the_library(tmp_path, libmx):
    """A C program (no Python, no torch) links libmx.so and makes the calls
    that need no device: version, parameter counts, argument refusals."""
    import subprocess
    from paper_2602_12242_gb300 import build
    src = tmp_path / "client.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "mx.h"
int main(void) {
  mx_params p;
  mx_ctx *ctx = 0;
  mx_fno *net = 0;
  memset(&p, 0, sizeof p);
  p.nx = 0; p.ny = 8; p.nz = 1; p.dx = p.dy = p.dz = 2e-9; p.Ms = 8e5; p.gamma = 2.211e5;
  if (mx_create(&ctx, &p) != MX_ERR_UNSUPPORTED || ctx) return 1;
  if (mx_fno_create(&net, 30, 20, 12, 1) != MX_ERR_INVALID_ARG || net) return 2;
  printf("%s|%d|%d|%s\n", mx_version(), mx_cnn_num_params(), mx_fno_num_params(12), mx_last_error());
  return 0;
}
''')
    lib = build.LIB
    exe = tmp_path / "client"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), lib,
                    "-Wl,-rpath," + os.path.dirname(lib), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.strip().split("|")
    assert "sm_103a" in out[0] and out[1] == "115907" and out[2] == "2368259" and "mx_fno_create" in out[3]


def test_schedule_and_mode_enums_match_the_binding(tmp_path):
    """The demag schedules and FFT modes of mx.h equal the binding's constants."""
    from paper_2602_12242_gb300 import _lib
    names = ["MX_DEMAG_AUTO", "MX_DEMAG_GENERIC", "MX_DEMAG_PLANE", "MX_DEMAG_PLANE_PAIR", "MX_DEMAG_PLANE_XLOCAL",
             "MX_FFT_FP32", "MX_FFT_SPLIT_BF16"]
    src = tmp_path / "enums.c"
    src.write_text('#include <stdio.h>\n#include "mx.h"\nint main(void){' +
                   "".join(f'printf("%d ", (int){n});' for n in names) + "return 0;}")
    exe = tmp_path / "enums"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == [getattr(_lib, n) for n in names]


def test_timing_slots_name_the_fused_stage(libmx):
    """mx_kernel_slot needs no device: every slot has a name, the fused
    inverse-x + local stage included, and out-of-range slots are empty."""
    libmx.mx_kernel_slot.restype = ctypes.c_char_p
    slots = []
    q = 0
    while True:
        s = libmx.mx_kernel_slot(q).decode()
        if not s:
            break
        slots.append(s)
        q += 1
    assert {"x_fwd", "yz_fused", "x_inv", "local_stage", "x_inv_local"} <= set(slots)
    assert libmx.mx_kernel_slot(-1).decode() == ""
