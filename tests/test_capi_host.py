"""Host-side checks of the C ABI, no GPU needed: the library builds for sm_103a,
loads, exports every entry point declared in include/*.h, and rejects bad
arguments before touching the device.  Also checks the closed-form constants
compiled into the kernels."""
import ctypes as C
import glob
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(qed_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2110_00256_gb300 import build, _lib
    build.build()
    return _lib.lib()


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert len(declared) >= 14
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_declared_symbols():
    from paper_2110_00256_gb300 import _lib
    assert _declared() <= set(_lib.SIGNATURES)


def test_version_and_error_message(lib):
    assert b"sm_103a" in lib.qed_version()
    assert lib.qed_last_error_message() is not None


def test_argument_validation_without_gpu(lib):
    from paper_2110_00256_gb300 import _lib
    out = C.c_void_p()
    # NULL params
    assert lib.qed_tables_generate(None, C.byref(out), None) == 1
    assert b"params" in lib.qed_last_error_message()
    # bad axes
    bad = _lib.TableParams(_lib.TableAxis(1.0, 0.5, 64, 64, 1e-12), _lib.TableAxis(0.02, 1e3, 64, 64, 0.0))
    assert lib.qed_tables_generate(C.byref(bad), C.byref(out), None) == 1
    too_big = _lib.TableParams(_lib.TableAxis(1e-3, 1e3, 4096, 64, 1e-12), _lib.TableAxis(0.02, 1e3, 64, 64, 0.0))
    assert lib.qed_tables_generate(C.byref(too_big), C.byref(out), None) == 1
    no_xi = _lib.TableParams(_lib.TableAxis(1e-3, 1e3, 64, 64, 0.0), _lib.TableAxis(0.02, 1e3, 64, 64, 0.0))
    assert lib.qed_tables_generate(C.byref(no_xi), C.byref(out), None) == 1
    # NULL handles / species
    assert lib.qed_evolve_optical_depth(None, 0, None, 1.0, 0, None, None, None) == 1
    assert lib.qed_substep(None, None, None, None, 1.0, 0, 0, None, 0, None, None) == 1
    assert lib.qed_tables_load(b"/nonexistent/qed.tab", C.byref(out), None) == 6
    assert lib.qed_tables_destroy(None) == 0


def _fnv1a64(b: bytes) -> int:
    h = 0xcbf29ce484222325
    for x in b:
        h = ((h ^ x) * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def _mlp_file(params=None, magic=b"QEDMLP\0\1", version=1, n_params=None, ranges=(1e-3, 0.02, 1e3, 1e3)):
    import struct
    import numpy as np
    from paper_2110_00256_gb300 import _lib
    n = _lib.QED_MLP_PARAMS if n_params is None else n_params
    p = np.zeros(2 * _lib.QED_MLP_PARAMS, np.float32) if params is None else params
    body = magic + struct.pack("<II4d", version, n, *ranges) + p.tobytes()
    return body + struct.pack("<Q", _fnv1a64(body))


def test_network_file_rejected_before_the_device(lib, tmp_path):
    """qed_mlp_load refuses missing, short, foreign, corrupted and non-finite
    files with QED_ERR_IO before it allocates anything on the device."""
    import numpy as np
    from paper_2110_00256_gb300 import _lib
    out = C.c_void_p(1)
    assert lib.qed_mlp_load(b"/nonexistent/qed.mlp", C.byref(out), None) == 6 and not out.value
    assert lib.qed_mlp_load(None, C.byref(out), None) == 1
    assert lib.qed_mlp_save(None, b"x") == 1
    good = _mlp_file()
    cases = {
        "short": good[:-9],
        "long": good + b"\0",
        "magic": _mlp_file(magic=b"QEDTAB\0\1"),
        "version": _mlp_file(version=2),
        "params": _mlp_file(n_params=4416),
        "checksum": good[:100] + bytes([good[100] ^ 1]) + good[101:],
        "range": _mlp_file(ranges=(1e-3, 0.02, 1e-4, 1e3)),
        "nonfinite": _mlp_file(params=np.full(2 * _lib.QED_MLP_PARAMS, np.nan, np.float32)),
    }
    for name, data in cases.items():
        path = tmp_path / f"{name}.mlp"
        path.write_bytes(data)
        out = C.c_void_p(1)
        assert lib.qed_mlp_load(str(path).encode(), C.byref(out), None) == 6, name
        assert not out.value, name
        msg = lib.qed_last_error_message()
        assert str(path).encode() in msg, (name, msg)


def test_kernel_asymptote_constants_match_closed_forms():
    src = open(os.path.join(ROOT, "paper_2110_00256_gb300", "csrc", "physics.cuh")).read()
    ts = float(re.search(r"kTSmall\s*=\s*([0-9.eE+-]+)", src).group(1))
    tl = float(re.search(r"kTLarge\s*=\s*([0-9.eE+-]+)", src).group(1))
    assert ts == pytest.approx(3 * math.sqrt(3) / (16 * math.sqrt(2)), rel=1e-15)
    g23, g13 = math.gamma(2 / 3), math.gamma(1 / 3)
    assert tl == pytest.approx(15 * 3 ** (2 / 3) * g23 ** 3 / (14 * math.pi * math.sqrt(3) * g13), rel=1e-15)
    gen = open(os.path.join(ROOT, "paper_2110_00256_gb300", "csrc", "tablegen.cu")).read()
    c = float(re.search(r"\(([0-9.]+) /\* sqrt\(3\) / \(2 pi\) \*/\)", gen).group(1))
    assert c == pytest.approx(math.sqrt(3) / (2 * math.pi), rel=1e-15)


def test_binding_struct_layouts_match_header(tmp_path):
    """Every ctypes Structure of the binding has the size and field offsets
    that a C compiler gives the matching struct of include/qed.h."""
    import subprocess
    from paper_2110_00256_gb300 import _lib
    pairs = {"qed_table_axis": _lib.TableAxis, "qed_table_params": _lib.TableParams, "qed_species": _lib.Species,
             "qed_fire_list": _lib.FireList, "qed_substep_opts": _lib.SubstepOpts, "qed_patch": _lib.Patch,
             "qed_plane_wave": _lib.PlaneWave, "qed_cells": _lib.Cells, "qed_unit_scales": _lib.UnitScales}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "qed.h"', 'int main(void) {']
    for cname, py in pairs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    for cname, py in pairs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_binding_enums_match_header(tmp_path):
    """The status, statistics and evolution-variant constants of the binding
    equal the header's."""
    import subprocess
    from paper_2110_00256_gb300 import _lib
    names = [n for n in dir(_lib) if n.startswith(("QED_STAT_", "QED_EVOLVE_", "QED_MAX_", "QED_NOALLOC_"))
             or n in ("QED_OK", "QED_F32", "QED_F64", "QED_PROC_QS", "QED_PROC_BW", "QED_MLP_PARAMS")]
    lines = ['#include <stdio.h>', '#include "qed.h"', "int main(void) {"]
    lines += ['printf("%s %%lld\\n", (long long)(%s));' % (n, n) for n in names]
    lines += ["return 0;", "}"]
    src = tmp_path / "enums.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "enums"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    assert len(names) >= 20
    for n in names:
        assert int(got[n]) == getattr(_lib, n), n
