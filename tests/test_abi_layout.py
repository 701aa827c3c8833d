"""The ctypes structures of the binding have the size and field offsets of the C structures in
include/sexpe.h (host-only: a small C program compiled with the system compiler prints them)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "sexpe_grid": ("Grid", ["geometry", "n", "rho_star", "z_star", "z_bc", "rho_op", ("lambda", "lam")]),
    "sexpe_species": ("Species", ["n_species", "d_host", "reaction", "n_params", "params_host", "offset_host"]),
    "sexpe_coupling": ("Coupling", ["kind", "zeta", "eta", "alpha3", "beta3", "u_top", "v_top"]),
    "sexpe_plan_info": ("PlanInfo", ["geometry", "precision", "n_species", "ndim", "n", "n_instances",
                                     "kernels_per_step", "npts", "state_elems", "workspace_bytes", "setup_ms",
                                     "stencil_tile_j", "ring_slots", "stencil_tile_us", "stencil_planes",
                                     "stencil_ctas_per_sm", "theta_split", "batch_order", "batch_step_us"]),
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sexpe.h"', "int main(void) {"]
    for cname, (_, fields) in STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in fields:
            cf = f[0] if isinstance(f, tuple) else f
            lines.append(f'  printf("{cname} {cf} %zu\\n", offsetof({cname}, {cf}));')
    lines += ["  return 0;", "}"]
    src = d / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "abi"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        name, field, value = line.split()
        table[(name, field)] = int(value)
    return table


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_struct_layout_matches_header(c_layout, cname):
    from paper_2604_11558_gb300 import binding
    pyname, fields = STRUCTS[cname]
    cls = getattr(binding, pyname)
    assert ctypes.sizeof(cls) == c_layout[(cname, "size")], cname
    for f in fields:
        cf, pf = f if isinstance(f, tuple) else (f, f)
        assert getattr(cls, pf).offset == c_layout[(cname, cf)], (cname, cf)
