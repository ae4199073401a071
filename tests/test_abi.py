"""CPU checks of the C ABI: the library builds, loads and exports every function
include/pins.h declares, and the ctypes structures match the C layout."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pins.h")


@pytest.fixture(scope="module")
def libpath():
    from paper_2502_03749_gb300 import build
    return build.build()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pins_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("pins_create", "pins_solve", "pins_solve_batch", "pins_submit", "pins_poll",
                 "pins_destroy", "pins_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pins_[a-z_]+)\b", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_covers_exports(libpath):
    from paper_2502_03749_gb300 import pins
    lib = pins.load(libpath)
    for name in _declared():
        assert hasattr(lib, name)
    assert set(pins.EXPORTED) == set(_declared())


def test_config_default_matches_paper_hyperparameters(libpath):
    """Appendix E.1: eta 1e-2, T1 100, T2 50, K 250, beta 0.5, c1 1e-4, CG 1e-6, tol 1e-9."""
    from paper_2502_03749_gb300 import pins
    c = pins.pins_config_default()
    assert (c.eta, c.T1, c.T2, c.K) == (1e-2, 100, 50, 250)
    assert (c.armijo_beta, c.armijo_c1, c.cg_rtol, c.tol_marg) == (0.5, 1e-4, 1e-6, 1e-9)
    assert c.sparsify_gamma == 1.0


def test_ctypes_layout_matches_c(tmp_path):
    """sizeof/offsetof of the ABI structs from a C compiler equal the ctypes layout."""
    from paper_2502_03749_gb300 import pins
    src = tmp_path / "layout.c"
    fields = {"pins_config": [f for f, _ in pins.pins_config._fields_],
              "pins_problem": [f for f, _ in pins.pins_problem._fields_],
              "pins_result": [f for f, _ in pins.pins_result._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for s, fs in fields.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f in fs:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-o", str(exe), str(src)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    import ctypes
    for s, fs in fields.items():
        cls = getattr(pins, s)
        assert int(got[s]) == ctypes.sizeof(cls), s
        for f in fs:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, f"{s}.{f}"


def test_create_without_gpu_fails_loudly(libpath):
    """No CPU fallback: without a CUDA device pins_create reports an error."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2502_03749_gb300 import pins
    with pytest.raises(RuntimeError):
        pins.Pins()
