"""The C-ABI library without a GPU: it builds, loads, exports every symbol include/lbm.h
declares, and its host-side validation accepts and rejects what it should."""
import ctypes
import os
import re

import pytest

from paper_1402_6019_gb300 import lbm as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    """Every function declared in include/*.h (lbm_* and the three-dimensional lbm3_*)."""
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm3?_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    lib = L.load()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
        assert n in L.SIGNATURES, n
    assert set(L.SIGNATURES) == set(names)
    assert L.lbm_abi_version() == 5


def test_struct_layouts_match_header(tmp_path):
    """Every field offset of the ctypes mirrors equals the C compiler's layout of include/lbm.h."""
    import subprocess

    structs = {"lbm_desc": L.lbm_desc, "lbm_params": L.lbm_params, "lbm_obs": L.lbm_obs, "lbm3_desc": L.lbm3_desc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbm.h"', '#include "lbm3d.h"', "int main(void) {"]
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} sizeof %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{sname} {fname} %zu\\n", offsetof({sname}, {fname}));')
    lines.append("return 0; }")
    (tmp_path / "lay.c").write_text("\n".join(lines))
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(tmp_path / "lay.c"), "-o",
                    str(tmp_path / "lay")], check=True)
    out = subprocess.run([str(tmp_path / "lay")], capture_output=True, text=True, check=True).stdout
    for line in out.strip().splitlines():
        sname, fname, val = line.split()
        cls = structs[sname]
        want = ctypes.sizeof(cls) if fname == "sizeof" else getattr(cls, fname).offset
        assert int(val) == want, (sname, fname)


def test_validate_desc():
    d = L.lbm_default_desc()
    assert L.lbm_validate_desc(d) == L.LBM_OK
    for field, bad in [("nx", 0), ("nz", -1), ("nx", 70000), ("n_species", 3), ("precision", 7),
                       ("z_boundary", 2), ("kernel", 9), ("device", -1), ("rows_per_warp", -2)]:
        d = L.lbm_default_desc()
        setattr(d, field, bad)
        assert L.lbm_validate_desc(d) == L.LBM_EINVAL, field
        assert L.lbm_last_error(None)
    d = L.lbm_default_desc()
    d.nx, d.nz = 65536, 65536
    assert L.lbm_validate_desc(d) == L.LBM_EINVAL  # nx * nz > 2^30


def test_validate_params():
    p = L.lbm_default_params()
    assert L.lbm_validate_params(p, 2) == L.LBM_OK
    assert p.weight_norm == pytest.approx(1 / 3)
    cases = [("tau", [0.5, 1.0]), ("tau", [1.0, 0.4]), ("rho0", [0.0, 1.0]), ("G1", [float("nan"), 0.0]),
             ("psi_form", 5), ("weight_preset", 3), ("weight_norm", 0.0), ("psi_wall", 2),
             ("body_force", float("inf"))]
    for k, v in cases:
        p = L.make_params(**{k: v})
        assert L.lbm_validate_params(p, 2) == L.LBM_EINVAL, (k, v)
    # species B is not checked for one species
    p = L.make_params(tau=[1.0, 0.1])
    assert L.lbm_validate_params(p, 1) == L.LBM_OK
    assert L.lbm_validate_params(p, 3) == L.LBM_EINVAL


def test_create_reports_missing_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(L.LbmError) as e:
        L.lbm_create(L.lbm_default_desc())
    assert e.value.code == L.LBM_ECUDA
    assert "cuda" in str(e.value).lower()
