"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a and exports every entry point that include/tidegs.h declares."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "tidegs.h")) as f:
        txt = f.read()
    return sorted(set(re.findall(r"\b(tgs_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    import paper_2605_20150_b300 as m
    from paper_2605_20150_b300 import build
    lib = build.build()
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib], text=True)
    exported = set(re.findall(r" T (tgs_\w+)", out))
    declared = _declared()
    assert declared, "no declarations found"
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    # the binding declares a signature for every exported entry point
    assert set(m.declared_symbols()) >= set(declared)


def test_library_loads_without_gpu():
    import ctypes
    from paper_2605_20150_b300 import build
    lib = ctypes.CDLL(build.build())
    lib.tgs_last_error.restype = ctypes.c_char_p
    assert lib.tgs_last_error() == b""


def test_struct_layouts_match_header():
    """ctypes mirrors of the ABI structs have the C sizes (compiled probe)."""
    import ctypes
    import tempfile
    import paper_2605_20150_b300 as m
    src = ('#include "tidegs.h"\n#include <stdio.h>\nint main(){printf("%zu %zu %zu\\n", sizeof(tgs_camera), '
           'sizeof(tgs_config), sizeof(tgs_stats));return 0;}\n')
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        with open(c, "w") as f:
            f.write(src)
        exe = os.path.join(d, "p")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        sizes = [int(x) for x in subprocess.check_output([exe], text=True).split()]
    assert sizes == [ctypes.sizeof(m.tgs_camera), ctypes.sizeof(m.tgs_config), ctypes.sizeof(m.tgs_stats)]


def test_struct_field_offsets_match_header():
    """Every field of the ctypes mirrors sits at the C offset of the field of
    the same name (a reordered or mistyped field would corrupt configs
    silently)."""
    import tempfile
    import paper_2605_20150_b300 as m
    structs = [("tgs_camera", m.tgs_camera), ("tgs_config", m.tgs_config), ("tgs_stats", m.tgs_stats)]
    lines, want = [], []
    for cname, py in structs:
        for name, _ in py._fields_:
            # Python keywords carry a trailing underscore in the mirror (lambda_)
            lines.append(f'printf("%zu\\n", offsetof({cname}, {name.rstrip("_")}));')
            want.append(getattr(py, name).offset)
    src = '#include "tidegs.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(){' + "".join(lines) + "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        with open(c, "w") as f:
            f.write(src)
        exe = os.path.join(d, "p")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(x) for x in subprocess.check_output([exe], text=True).split()]
    assert got == want
