"""The C-ABI library builds, loads, and exports every entry point the headers in include/
declare (CPU only: no compute call needs a GPU here)."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

from paper_2311_08050_gb300 import build as B
from paper_2311_08050_gb300 import inla

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header=None):
    names = [header] if header else sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
    found = set()
    for h in names:
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        found |= set(re.findall(r"\b(inla_[a-z0-9_]+)\s*\(", txt))
    return sorted(found)


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_header_declares_the_binding_entry_points():
    assert set(inla.EXPORTED) <= set(_declared("inla.h"))
    assert {"inla_mlp_create", "inla_mlp_train", "inla_mlp_predict", "inla_mlp_loss_grad"} <= set(
        _declared("inla_surrogate.h"))


def test_surrogate_parameter_count_and_argument_checks_without_a_gpu(libpath):
    from oracle import mlp_oracle
    L = inla.lib()
    L.inla_mlp_num_params.restype = ctypes.c_int64
    for d in (1, 4, 8):
        assert L.inla_mlp_num_params(d) == mlp_oracle.n_params(d, 128)
    h = ctypes.c_void_p()
    assert L.inla_mlp_create(0, 16, ctypes.byref(h)) == inla.E_BADARG
    assert L.inla_mlp_create(9, 16, ctypes.byref(h)) == inla.E_BADARG


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(inla_[a-z0-9_]+)", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing


def test_library_loads_and_answers_without_a_gpu(libpath):
    L = inla.lib()
    assert inla.status_string(0) == "ok"
    assert inla.status_string(inla.E_NOT_SPD) == "matrix not positive definite"
    o = inla.Opts()
    assert L.inla_opts_default(ctypes.byref(o)) == 0
    assert o.newton_tol == 1e-8 and o.newton_max == 50 and o.precision == 0
    # NULL arguments are rejected before any device work
    assert L.inla_model_create(None, None) == inla.E_BADARG
    assert L.inla_model_destroy(None) == 0


def test_struct_layout_matches_header(tmp_path):
    """The ctypes mirrors have the sizes and field offsets a C compiler gives the header."""
    structs = {"inla_factor": inla.Factor, "inla_block": inla.BlockS, "inla_model_desc": inla.ModelDesc,
               "inla_opts": inla.Opts}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "inla.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} __sizeof__ %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        cname, field, val = line.split()
        got[(cname, field)] = int(val)
    for cname, cls in structs.items():
        assert got[(cname, "__sizeof__")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_outer_block_pin_and_tile_width_hook_without_a_gpu(libpath):
    """INLA_OUTER_BLOCK pins the mixed Cholesky's outer block (read once per process, so each
    case runs in a fresh interpreter); unset, nothing is decided before a factorisation ran.
    The GEMM tile-width hook accepts 0, 64 and 128 only."""
    code = ("import ctypes, sys; L = ctypes.CDLL(sys.argv[1]); "
            "print(L.inla_test_outer_block(16384, 4), L.inla_test_outer_block(512, 5))")
    for pin, want in (("512", "512 512"), ("256", "256 256"), ("300", "0 0"), (None, "0 0")):
        env = {k: v for k, v in os.environ.items() if k != "INLA_OUTER_BLOCK"}
        if pin is not None:
            env["INLA_OUTER_BLOCK"] = pin
        out = subprocess.run([sys.executable, "-c", code, libpath], capture_output=True, text=True, env=env)
        assert out.returncode == 0, out.stderr
        assert out.stdout.split() == want.split(), (pin, out.stdout)
    L = inla.lib()
    for bn in (0, 64, 128):
        assert L.inla_test_gemm_tile_width(bn) == 0
    for bn in (32, 96, 256, -1):
        assert L.inla_test_gemm_tile_width(bn) == inla.E_BADARG
    assert L.inla_test_gemm_tile_width(0) == 0
