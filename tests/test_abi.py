"""The C-ABI library builds, loads and exports every symbol its header
declares (no compute calls: this runs without a GPU)."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "paulinet.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pn_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1909_08423_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["pn_init_system", "pn_eval_logpsi", "pn_eval_local_energy", "pn_metropolis_step",
              "pn_grad_logpsi", "pn_submit", "pn_poll", "pn_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pn_[a-z_0-9]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_loads_library_and_resolves_symbols(libpath):
    import ctypes
    from paper_1909_08423_gb300 import binding
    lib = ctypes.CDLL(libpath)
    for n in _declared():
        getattr(lib, n)
    for n in binding.EXPORTS:
        assert n in _declared(), n
    # a pure host call: the parameter count of the layout
    from paper_1909_08423_gb300 import synth
    s = synth.n2()
    assert lib.pn_num_params_for(128, 64, 32, 4, 2, 11) == synth.n_params(s)


def test_missing_library_fails_loudly(tmp_path):
    """No fallback: without the compiled library the binding raises."""
    import sys
    code = ("from paper_1909_08423_gb300 import binding\n"
            f"binding.load({str(tmp_path / 'libpaulinet.so')!r})\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert out.returncode != 0
    assert "not built" in out.stderr


def test_product_package_never_imports_the_oracle():
    """The oracle is test infrastructure: no module of the package imports it."""
    pkg = os.path.join(ROOT, "paper_1909_08423_gb300")
    offenders = []
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                src = open(os.path.join(dirpath, f)).read()
                if re.search(r"^\s*(from|import)\s+oracle\b", src, flags=re.M):
                    offenders.append(f)
    assert not offenders, offenders
