"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/*.h declares (no compute call: no GPU needed)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names |= set(re.findall(r"VDS_API\s+[\w\s\*]*?\b((?:vds|pod)_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2603_12550_gb300 import build
    return build.build()


def test_header_declares_api():
    names = _declared()
    for must in ("vds_create", "vds_destroy", "vds_energy_grad", "vds_step", "vds_stress"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(\S+)$", out, re.M))
    missing = _declared() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_library_loads_and_binds(libpath):
    from paper_2603_12550_gb300 import vds
    syms = set(vds.exported_symbols())
    assert _declared() <= set(vds._SIGS) | syms
    assert vds.strerror(vds.VDS_EDOMAIN).startswith("FENE")
