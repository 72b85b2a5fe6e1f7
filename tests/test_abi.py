"""The C ABI: every function include/eb.h declares is exported by the built library (no GPU needed),
struct layouts of the binding match the header, and the product path refuses to run without its
library (there is no CPU fallback)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "eb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eb_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1411_4283_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "eb_build_stencils" in names and "eb_solve" in names and "eb_lsq_batch_noalloc" in names
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layouts_match_header(tmp_path):
    import paper_1411_4283_gb300 as P
    c = tmp_path / "sz.c"
    c.write_text('#include <stdio.h>\n#include "%s"\nint main(){printf("%%zu %%zu %%zu %%zu %%zu %%zu\\n", sizeof(eb_geom), '
                 'sizeof(eb_params), sizeof(eb_build_info), sizeof(eb_solve_opts), sizeof(eb_solve_info), '
                 'sizeof(eb_adjoint_info));}\n'
                 % os.path.join(ROOT, "include", "eb.h"))
    exe = tmp_path / "sz"
    subprocess.run(["gcc", str(c), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(t) for t in (P.EbGeom, P.EbParams, P.EbBuildInfo, P.EbSolveOpts, P.EbSolveInfo,
                                       P.EbAdjointInfo)]
    assert got == want


def test_status_strings(lib):
    lib.eb_status_string.restype = ctypes.c_char_p
    assert lib.eb_status_string(0) == b"ok"
    assert b"rank" in lib.eb_status_string(2)
    lib.eb_abi_version.restype = ctypes.c_int32
    assert lib.eb_abi_version() == 3


def test_invalid_arguments_rejected_without_gpu(lib):
    """Argument checks run before any CUDA call: a NULL descriptor and an oversized no-alloc
    request are refused with their status codes."""
    import paper_1411_4283_gb300 as P
    P.load()
    h = ctypes.c_void_p()
    assert P._LIB.eb_build_stencils(None, None, ctypes.byref(h), None, None) == 1
    hs = (ctypes.c_void_p * 2)()
    assert P._LIB.eb_build_stencils_batch(None, 2, None, hs, None, None) == 1
    assert P._LIB.eb_build_stencils_batch(None, 0, None, hs, None, None) == 1
    assert P._LIB.eb_lsq_batch_noalloc(None, None, None, None, 1, 15, 300, None, None, None) == 8
    assert P._LIB.eb_lsq_batch_noalloc(None, None, None, None, 1, 40, 10, None, None, None) == 1
    # batched solve: empty batch, null handles; FP64 probe and the adjoint entry points: null arguments
    sv = ctypes.c_void_p()
    assert P._LIB.eb_batch_solver_create(None, 0, None, ctypes.byref(sv), None) == 1
    assert P._LIB.eb_batch_solver_create((ctypes.c_void_p * 1)(None), 1, None, ctypes.byref(sv), None) == 1
    assert P._LIB.eb_batch_solve(None, None, None, None, 1e-12, None, None, None) == 1
    assert P._LIB.eb_fp64_fma_rate(0, 1, None, None) == 1
    J = ctypes.c_double()
    assert P._LIB.eb_adjoint_shape(None, None, None, 0, None, ctypes.byref(J), None, None, None, None) == 1
    assert P._LIB.eb_adjoint_radii(None, None, None, ctypes.byref(J), None, None) == 1
    nb = ctypes.c_int64()
    assert P._LIB.eb_geometry_shape_table(None, 0, 0, None, 2, 0, None, 0, ctypes.byref(nb)) == 1
    # one stencil set twice in a batch (refused before any handle is read)
    opts1 = P.EbSolveOpts(1, 1e-5, 100, 10, 1000, 1, 1)
    assert P._LIB.eb_batch_solver_create((ctypes.c_void_p * 3)(8, 16, 8), 3, ctypes.byref(opts1), ctypes.byref(sv),
                                         None) == 1
    assert "twice" in P._LIB.eb_last_error_message().decode()
    opts = P.EbSolveOpts(0, 1e-5, 100, 10, 1000, 1, 1)  # mixed = 0: the batch is the refinement only
    assert P._LIB.eb_batch_solver_create((ctypes.c_void_p * 1)(1), 1, ctypes.byref(opts), ctypes.byref(sv),
                                         None) == 1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_1411_4283_gb300 as P
    monkeypatch.setattr(P, "_LIB", None)
    monkeypatch.setattr(P._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        P.load()


def test_binding_checks_vectors_before_the_call():
    """The binding passes raw pointers, so it checks each vector's type, device, layout and length
    first: a CPU tensor, a float32 tensor, a non-contiguous view or a short vector is refused on the
    host, and an empty vector is accepted where the length is 0 (a geometry with no cut cells)."""
    import torch
    import paper_1411_4283_gb300 as P
    for bad in (torch.zeros(8, dtype=torch.float64),  # host memory
                torch.zeros(8, dtype=torch.float32),
                torch.zeros(16, dtype=torch.float64)[::2],
                np.zeros(8)):
        with pytest.raises(ValueError):
            P._vec64(bad, 8, "rho")
    with pytest.raises(ValueError):
        P._vec64(None, 3, "g_eb")
    assert P._vec64(None, 0, "g_eb").value is None


def test_plain_c_program_links_every_entry_point(tmp_path, lib):
    """The boundary is consumable from C alone: a C99 program that includes eb.h (warnings as errors,
    pedantic), takes the address of every declared entry point, links against the built library and
    calls the entry points that need no GPU."""
    from paper_1411_4283_gb300 import build
    libdir = os.path.dirname(build.build())
    refs = "\n".join(f"  fn = (void (*)(void))&{n}; (void)fn;" for n in _declared())
    src = tmp_path / "use.c"
    src.write_text('#include <stdio.h>\n#include "eb.h"\nint main(void) {\n  void (*fn)(void);\n' + refs +
                   '\n  printf("%d %s\\n", (int)eb_abi_version(), eb_status_string(EB_ERR_RANK_DEFICIENT));\n'
                   '  return 0;\n}\n')
    exe = tmp_path / "use"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        str(src), "-I", os.path.join(ROOT, "include"), "-L", libdir, "-leb_gb300",
                        "-Wl,-rpath," + libdir, "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    ver, msg = out.stdout.split(" ", 1)
    assert int(ver) == 3 and msg.strip()


def test_struct_field_offsets_match_header(tmp_path):
    """Every field of the binding's structures sits at the header's offset (sizes alone would not
    catch two fields swapped)."""
    import paper_1411_4283_gb300 as P
    structs = {"eb_geom": P.EbGeom, "eb_params": P.EbParams, "eb_build_info": P.EbBuildInfo,
               "eb_solve_opts": P.EbSolveOpts, "eb_solve_info": P.EbSolveInfo, "eb_adjoint_info": P.EbAdjointInfo}
    lines, want = [], []
    for cname, ct in structs.items():
        for f in ct._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {f[0]}));')
            want.append(getattr(ct, f[0]).offset)
    c = tmp_path / "off.c"
    c.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "%s"\nint main(void) {\n%s\n  return 0;\n}\n'
                 % (os.path.join(ROOT, "include", "eb.h"), "\n".join(lines)))
    exe = tmp_path / "off"
    r = subprocess.run(["gcc", str(c), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert got == want
