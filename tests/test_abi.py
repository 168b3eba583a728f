"""CPU checks of the C ABI: the library builds, loads and exports every
function include/wilson.h declares; host-only calls validate arguments."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M))
    return names


def test_build_and_exports():
    import subprocess
    import __graft_entry__ as ge
    ge.build()
    declared = _declared()
    assert declared, "no declarations parsed"
    # the library and its bounds-checked build export the same ABI
    for name in ("libwilson.so", "libwilson_checked.so"):
        lib = os.path.join(ROOT, "paper_1103_5103_gb300", name)
        out = subprocess.check_output(["nm", "-D", "--defined-only", lib]).decode()
        exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
        missing = declared - exported
        assert not missing, f"{name}: declared but not exported: {sorted(missing)}"


def test_checked_build_is_the_checked_one():
    """WL_LIBRARY=checked loads libwilson_checked.so, which says so; the
    ordinary library does not (host-only calls, no GPU needed)."""
    import subprocess
    import sys
    code = "from paper_1103_5103_gb300 import api; print(api.LIB_PATH, api.is_checked_build())"
    for env, name, flag in ((None, "libwilson.so", "False"), ("checked", "libwilson_checked.so", "True")):
        e = dict(os.environ)
        e.pop("WL_LIBRARY", None)
        if env:
            e["WL_LIBRARY"] = env
        out = subprocess.check_output([sys.executable, "-c", code], env=e, cwd=ROOT).decode().split()
        assert out[0].endswith(name) and out[1] == flag, out


def test_host_only_calls():
    from paper_1103_5103_gb300 import api
    p = api.params()
    assert p.tol == 1e-10 and p.inner_prec == api.F32 and p.eo == 1
    # the fields after the pointer member land where the C struct has them
    assert p.outer_prec == api.F64 and p.shadow is None and p.guess_max == 0 and p.reliable == 0
    assert p.inner_solver == api.SOLVER_BICGSTAB and p.verify_full == 0
    assert p.guess == api.GUESS_POLY and p.mode == api.MODE_GRAPH and p.graph_iters == 8
    lat = api.Lattice((4, 4, 4, 8))
    assert lat.spinor_bytes("f64") == 192 * 256 and lat.spinor_bytes("f32") == 96 * 256
    assert lat.spinor_bytes("f16") == 52 * 256
    # index arithmetic is 32-bit: 12 V must stay below 2^31
    for bad in [(3, 4, 4, 4), (4, 4, 0, 4), (4, 4, 4, 5), (512, 512, 512, 2)]:
        with pytest.raises(api.WilsonError) as e:
            api.Lattice(bad)
        assert e.value.status == api.WL_ERR_ARG
    with pytest.raises(api.WilsonError):
        lat.spinor_bytes(3)


def test_oracle_and_library_are_independent():
    """The oracle never imports the library; the library never imports the oracle."""
    src = open(os.path.join(ROOT, "oracle", "oracle.py")).read()
    assert "import paper_1103_5103_gb300" not in src and "from paper_1103_5103_gb300" not in src
    assert "libwilson" not in src
    pkg = os.path.join(ROOT, "paper_1103_5103_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "wilson_oracle" not in text, f
