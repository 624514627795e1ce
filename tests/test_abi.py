"""The C-ABI library loads and exports every symbol include/jt.h declares (CPU only)."""
import ctypes
import os
import re

import paper_2212_04241_gb300.jt as J

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"JT_API\s+[\w\s\*]*?\b(jt_\w+)\s*\(", src)
    return names


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert "jt_compile" in names and "jt_infer" in names and "jt_infer_device" in names
    lib = ctypes.CDLL(J.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(J.EXPORTS) <= set(names)


def test_status_strings_and_defaults():
    for s in range(9):
        assert J.lib.jt_status_string(s)
    o = J.default_opts()
    assert o.root_rule == J.JT_ROOT_MIN_HEIGHT and o.use_graphs == 1 and o.host_only == 0


def test_host_only_plan_refuses_inference():
    import numpy as np
    from synth import configs
    net = configs.network("bn20")
    p = J.Plan(net, host_only=1)
    try:
        p.infer(np.full((1, net.n), -1, dtype=np.int32))
        raise AssertionError("expected an error")
    except J.JTError as e:
        assert e.status == J.JT_EINVAL


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of jt_compile_opts and jt_plan_info_t have the
    header's field offsets and sizes (a C program compiled against
    include/jt.h prints them)."""
    import shutil
    import subprocess
    import pytest
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "jt.h"', "int main(void) {"]
    for cname, py in (("jt_compile_opts", J.CompileOpts), ("jt_plan_info_t", J.PlanInfo)):
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in (("jt_compile_opts", J.CompileOpts), ("jt_plan_info_t", J.PlanInfo)):
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)
