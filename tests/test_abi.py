"""CPU checks of the C ABI: the library builds, loads, and exports every
entry point include/*.h declares; host-only calls validate arguments.
No kernel is launched here."""
import ctypes as C
import os
import re

import pytest

from paper_2310_00810_gb300 import build as B
from paper_2310_00810_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lbm.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:LBM_API\s+)?(?:lbm_status|const char\s*\*)\s+((?:lbm|unet)_\w+)\s*\(",
                                    text, re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert "lbm_forward" in declared and "lbm_adjoint" in declared
    assert declared == set(lbm.ENTRY_POINTS), "binding and header disagree"
    for name in declared:
        assert hasattr(lib, name), name


def test_nothing_else_is_exported(lib):
    out = os.popen(f"nm -D --defined-only {B.LIB}").read()
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert {n for n in exported if n.startswith(("lbm_", "unet_"))} == set(lbm.ENTRY_POINTS)


@pytest.mark.parametrize("bad", [
    dict(q=7), dict(precision=2), dict(nx=1), dict(ny=0), dict(nz=2), dict(n_steps=0), dict(ckpt_stride=-1),
    dict(loss_kind=5), dict(inlet_kind=3), dict(ny=65536),
    dict(q=19, nx=4, ny=4, nz=65536),
])
def test_plan_create_rejects_bad_descriptors(lib, bad):
    args = dict(q=9, nx=64, ny=32, nz=1, precision=4, n_steps=10, ckpt_stride=0, loss_kind=0, loss_norm=0,
                inlet_kind=0)
    args.update(bad)
    with pytest.raises(lbm.LBMError) as e:
        lbm.Plan(**args)
    assert e.value.status == lbm.LBM_ERR_INVALID_ARG


def test_plan_create_accepts_the_largest_grid_rows(lib):
    """ny = 65535 (nz = 65535) is the last row (layer) count a launch grid holds."""
    lbm.Plan(9, 2, 65535, 1, 4, n_steps=1)
    lbm.Plan(19, 2, 2, 65535, 4, n_steps=1)


def test_workspace_size_counts_checkpoints(lib):
    st = 9 * 64 * 32 * 4
    p1 = lbm.Plan(9, 64, 32, 1, 4, n_steps=100, ckpt_stride=1)
    p10 = lbm.Plan(9, 64, 32, 1, 4, n_steps=100, ckpt_stride=10)
    p0 = lbm.Plan(9, 64, 32, 1, 4, n_steps=100)  # sqrt(T) = 10
    s1, s10, s0 = (lbm.lbm_workspace_size(p) for p in (p1, p10, p0))
    assert s10 == s0
    # stride 1 keeps T - 1 checkpoints + two 1-state segment buffers; stride 10 keeps 9 + 2 x 10
    assert s1 - s10 == (99 + 2 - 9 - 20) * st
    assert s1 > 100 * st


def test_calls_without_geometry_are_rejected(lib):
    p = lbm.Plan(9, 64, 32, 1, 4, n_steps=4)
    st = lib.lbm_forward(p.handle, None, None, 1.0, None, None, None)
    assert st == lbm.LBM_ERR_INVALID_ARG
    assert lbm.lbm_error_string(lbm.LBM_ERR_NONFINITE) == "non-finite loss or gradient"


def test_spline_basis_host_call_matches_the_oracle(lib):
    """lbm_spline_basis is host code: it runs here, against the spline oracle."""
    import numpy as np

    from oracle import spline_oracle as S

    for K, n in [(1, 5), (2, 9), (3, 17), (6, 64), (16, 128), (33, 256), (7, 7)]:
        np.testing.assert_allclose(lbm.lbm_spline_basis(K, n), S.basis(K, n), rtol=0, atol=1e-13)
    for K, n in [(0, 5), (6, 5), (2, 0)]:
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_spline_basis(K, n)
        assert e.value.status == lbm.LBM_ERR_INVALID_ARG


def test_option_setters_validate_on_the_host(lib):
    """The option calls are host-only: argument checks without a GPU."""
    p9 = lbm.Plan(9, 64, 32, 1, 4, n_steps=4)
    p19 = lbm.Plan(19, 32, 16, 16, 4, n_steps=4)

    def status(fn):
        try:
            fn()
        except lbm.LBMError as e:
            return e.status
        return lbm.LBM_OK

    # MRT: D2Q9 only, rates in (0, 2)
    assert status(lambda: lbm.lbm_set_collision(p19, lbm.LBM_COLLISION_MRT, 1.6, 1.5, 1.9)) == lbm.LBM_ERR_UNSUPPORTED
    assert status(lambda: lbm.lbm_set_collision(p9, lbm.LBM_COLLISION_MRT, 2.0, 1.5, 1.9)) == lbm.LBM_ERR_INVALID_ARG
    assert status(lambda: lbm.lbm_set_collision(p9, 2)) == lbm.LBM_ERR_INVALID_ARG
    assert status(lambda: lbm.lbm_set_collision(p9, lbm.LBM_COLLISION_MRT, 1.6, 1.5, 1.9)) == lbm.LBM_OK
    mode, rates = lbm.lbm_get_collision(p9)
    assert mode == lbm.LBM_COLLISION_MRT and rates == (1.6, 1.5, 1.9)
    assert status(lambda: lbm.lbm_set_collision(p9, lbm.LBM_COLLISION_BGK)) == lbm.LBM_OK
    assert lbm.lbm_get_collision(p9) == (lbm.LBM_COLLISION_BGK, (0.0, 0.0, 0.0))
    # Eq. 6 velocity
    assert status(lambda: lbm.lbm_set_abb_velocity(p9, 3)) == lbm.LBM_ERR_INVALID_ARG
    assert status(lambda: lbm.lbm_set_abb_velocity(p9, lbm.LBM_ABB_U_EXTRAP)) == lbm.LBM_OK
    assert lbm.lbm_get_abb_velocity(p9) == lbm.LBM_ABB_U_EXTRAP
    # velocity inlet: finite, no u_z on D2Q9
    assert status(lambda: lbm.lbm_set_velocity_inlet(p9, (0.05, 0.0, 0.01))) == lbm.LBM_ERR_INVALID_ARG
    assert status(lambda: lbm.lbm_set_velocity_inlet(p9, (float("nan"), 0.0))) == lbm.LBM_ERR_INVALID_ARG
    assert status(lambda: lbm.lbm_set_velocity_inlet(p19, (0.05, 0.0, 0.01))) == lbm.LBM_OK
    # periodic y before any geometry
    assert status(lambda: lbm.lbm_set_periodic_y(p9, True)) == lbm.LBM_OK
    assert lib.lbm_set_periodic_y(p9.handle, 2) == lbm.LBM_ERR_INVALID_ARG
    # splines need a profile inlet and at most ny knots; probes need a workspace and geometry
    assert lib.lbm_spline_profile(p9.handle, 4, 1, None, None, None, 1.0, None, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_spline_grad(p9.handle, 4, 1, None, None, None, None, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_probe_loss_grad(p9.handle, None, -1, None, None, 1.0, None, None, None, None) == \
        lbm.LBM_ERR_INVALID_ARG


STRUCTS = [("lbm_desc", "lbm.h"), ("lbm_geom_desc", "lbm.h"), ("lbm_kernel_choice", "lbm.h"), ("unet_desc", "unet.h")]


def test_ctypes_structures_match_the_c_headers(tmp_path):
    """The binding's ctypes structures have the C structs' size and every
    field's offset (a field added to a header but not to the binding, or in
    another place, would shift the fields after it)."""
    import ctypes
    import shutil
    import subprocess

    from paper_2310_00810_gb300 import lbm as L
    from paper_2310_00810_gb300 import unet as UN

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    py = {"lbm_desc": L.lbm_desc, "lbm_geom_desc": L.lbm_geom_desc, "lbm_kernel_choice": L.lbm_kernel_choice,
          "unet_desc": UN.unet_desc}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lbm.h"', '#include "unet.h"', "int main(void) {"]
    for name, _ in STRUCTS:
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in py[name]._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    include = os.path.join(ROOT, "include")
    subprocess.run([cc, "-std=c11", "-I", include, str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, what, value = line.split()
        got[(name, what)] = int(value)
    for name, _ in STRUCTS:
        s = py[name]
        assert got[(name, "size")] == ctypes.sizeof(s), name
        for field, _ in s._fields_:
            assert got[(name, field)] == getattr(s, field).offset, (name, field)
