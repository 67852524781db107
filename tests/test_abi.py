"""The C-ABI library: it builds for sm_103a, loads, exports every entry point the
public header declares, and validates configurations on the host (no GPU)."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ap_pic.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ap_pic_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2608_15249_b300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("ap_pic_create", "ap_pic_load", "ap_pic_gather_push", "ap_pic_deposit",
                     "ap_pic_sort", "ap_pic_step", "ap_pic_get_rho", "ap_pic_get_E",
                     "ap_pic_get_diag"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(ap_pic_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for n in _declared():
        getattr(lib, n)


def test_binding_lists_every_declared_symbol():
    import paper_2608_15249_b300 as pk
    assert sorted(pk.EXPORTS) == sorted(n for n in _declared()
                                        if n in pk.EXPORTS or not n.startswith("ap_pic_batch"))


def test_config_defaults_and_validation(libpath):
    import paper_2608_15249_b300 as pk
    c = pk.ap_pic_config()
    pk.lib().ap_pic_config_default(ctypes.byref(c))
    assert c.ndim == 1 and c.n[0] == 64 and c.q == -1.0 and c.sort_every == 20
    # invalid configurations are rejected before any device work
    for bad in (dict(ndim=4), dict(ndim=2, n=(1, 8)), dict(ndim=1, dt=-1.0),
                dict(ndim=3, n=(8, 8, 8), nv=2, B0=(0, 0, 1.0)), dict(ndim=2, n=(8, 8), nv=1)):
        kw = dict(ndim=1, n=(8,))
        kw.update(bad)
        cfg = pk.make_config(**kw)
        h = ctypes.c_void_p()
        st = pk.lib().ap_pic_create(ctypes.byref(cfg), None, None, ctypes.byref(h))
        assert st == -1, (bad, st)
        assert pk.lib().ap_pic_last_error(h)
        pk.lib().ap_pic_destroy(h)
    cfg = pk.make_config(ndim=1, n=(8,))
    cfg.bc = 1
    h = ctypes.c_void_p()
    assert pk.lib().ap_pic_create(ctypes.byref(cfg), None, None, ctypes.byref(h)) == -2
    pk.lib().ap_pic_destroy(h)
    # the solver: unknown values are rejected; the spectral solve needs the FP32 form
    # and every axis within its longest transform
    for bad, want in ((dict(solver=7), -1),
                      (dict(solver=pk.AP_PIC_SOLVER_FFT, precision=pk.AP_PIC_FP64_PLAIN), -2),
                      (dict(solver=pk.AP_PIC_SOLVER_FFT, n=(pk.AP_PIC_FFT_MAX_N + 1,)), -2),
                      (dict(pusher=5), -1), (dict(c_light=-1.0), -1),
                      (dict(pusher=pk.AP_PIC_PUSHER_HIGUERA_CARY,
                            precision=pk.AP_PIC_FP64_PLAIN), -2)):
        kw = dict(ndim=1, n=(8,))
        kw.update(bad)
        cfg = pk.make_config(**kw)
        h = ctypes.c_void_p()
        assert pk.lib().ap_pic_create(ctypes.byref(cfg), None, None, ctypes.byref(h)) == want
        pk.lib().ap_pic_destroy(h)


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the binding mirrors has the C compiler's size and field offsets."""
    import paper_2608_15249_b300 as pk
    structs = {"ap_pic_config": pk.ap_pic_config, "ap_pic_diag": pk.ap_pic_diag,
               "ap_pic_batch_tuning": pk.ap_pic_batch_tuning, "ap_pic_mcc": pk.ap_pic_mcc,
               "ap_pic_allocator": pk.ap_pic_allocator}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ap_pic.h"', "int main(void){"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True,
                                                        text=True, check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[f"{name}.{field}"]) == getattr(cls, field).offset, (name, field)


def test_electromagnetic_configuration_is_validated_on_the_host(libpath):
    """The electromagnetic step's configuration is checked before any device work: the
    2D3V or 3D FP32 form with Boris, c > 0 and a Courant number below 1; the absorbing
    layer only with em = 1 on a 2D grid and with layers thinner than half the grid on
    each axis."""
    import paper_2608_15249_b300 as pk
    base = dict(ndim=2, n=(32, 32), dt=0.1, nv=3, em=1, c_light=2.0)
    cases = (
        (dict(em=2), -1),
        (dict(ndim=1, n=(32,)), -2),
        (dict(ndim=3, n=(8, 8, 8), c_light=6.0), -1),  # 3D: c dt sqrt(3) = 1.04
        (dict(ndim=3, n=(16, 16, 16), em_boundary=1, pml_cells=4), -2),
        (dict(nv=2), -2),
        (dict(precision=pk.AP_PIC_FP64_PLAIN), -2),
        (dict(pusher=pk.AP_PIC_PUSHER_HIGUERA_CARY), -2),
        (dict(c_light=0.0), -1),
        (dict(c_light=10.0), -1),  # c dt sqrt(2) = 1.41: past the Courant limit
        (dict(em_boundary=2), -1),
        (dict(em=0, em_boundary=1), -1),
        (dict(em_boundary=1, pml_cells=16), -1),  # 2 * 16 = n: no interior left
    )
    for bad, want in cases:
        kw = dict(base)
        kw.update(bad)
        cfg = pk.make_config(**kw)
        h = ctypes.c_void_p()
        st = pk.lib().ap_pic_create(ctypes.byref(cfg), None, None, ctypes.byref(h))
        assert st == want, (bad, st)
        assert pk.lib().ap_pic_last_error(h)
        pk.lib().ap_pic_destroy(h)
