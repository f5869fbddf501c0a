"""CPU checks of the C ABI: the library builds, loads, exports every entry
point declared in include/*.h, its structs match the header, and parameter
validation answers without a GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import paper_1802_01272_gb300 as P
    P.lib()
    return P


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(P):
    names = declared_functions()
    assert len(names) >= 17
    out = subprocess.run(["nm", "-D", "--defined-only", P.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lbm_\w+)", out))
    assert names <= exported, names - exported
    for n in names:
        getattr(P.lib(), n)


def test_struct_layout_matches_header(P, tmp_path):
    from paper_1802_01272_gb300.binding import lbm_diag, lbm_kernel_info, lbm_params
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "ctulbm.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(lbm_params),'
                   ' sizeof(lbm_diag), offsetof(lbm_params, rho_ref), offsetof(lbm_diag, theta),'
                   ' sizeof(lbm_kernel_info), offsetof(lbm_kernel_info, tensor_copies));'
                   'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    vals = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                        check=True).stdout.split()))
    assert vals == [C.sizeof(lbm_params), C.sizeof(lbm_diag), lbm_params.rho_ref.offset,
                    lbm_diag.theta.offset, C.sizeof(lbm_kernel_info),
                    lbm_kernel_info.tensor_copies.offset]


def test_defaults_are_the_papers(P):
    p = P.lbm_default_params(512, 256)
    assert (p.Lx, p.Ly) == (512, 256)
    assert p.a == 9 / 8 and p.b == 1 / 3 and p.kappa == 1e-4
    assert p.tau == 1e-3 and p.dt == 1e-4 and p.ds == 1 / 256
    assert p.ctu_order == 2 and p.limiter == P.LBM_LIM_MC and p.regularize == 0


@pytest.mark.parametrize("field,value,code", [
    ("Lx", 0, -1), ("ctu_order", 3, -1), ("limiter", 7, -1), ("boundary", 5, -1),
    ("precision", 9, -4), ("velset", 1, -4), ("tau", 0.0, -1), ("tau", 4e-5, -1),
])
def test_validation_without_gpu(P, field, value, code):
    p = P.Params(Lx=16, Ly=16)
    setattr(p, field, value)
    with pytest.raises(P.LBMError) as e:
        P.lbm_create(p)
    assert e.value.code == code


def test_cfl_is_checked(P):
    p = P.Params(Lx=16, Ly=16, tau=1.0, dt=2e-3)   # max|xi| dt = 4.7e-3 > ds = 3.9e-3
    with pytest.raises(P.LBMError) as e:
        P.lbm_create(p)
    assert e.value.code == -2


def test_density_range_is_checked(P):
    p = P.Params(Lx=16, Ly=16, boundary=P.LBM_BC_SHEAR_WALLS, rho_ext=3.5)  # 1/b = 3
    with pytest.raises(P.LBMError) as e:
        P.lbm_create(p)
    assert e.value.code == -3


def test_strerror(P):
    L = P.lib()
    assert L.lbm_strerror(0) == b"success"
    assert b"CFL" in L.lbm_strerror(-2)
    assert L.lbm_strerror(-99) == b"unknown error"


def test_batch_server_argument_checks(P):
    """lbm_batch_* reject bad arguments before touching the GPU."""
    import ctypes as C
    from paper_1802_01272_gb300.binding import lbm_batch_info, lbm_job_result
    L = P.lib()
    b = C.c_void_p()
    assert L.lbm_batch_create(0, 10, None, C.byref(b)) == -1
    assert L.lbm_batch_create(1 << 20, 0, None, C.byref(b)) == -1
    assert L.lbm_batch_create(1 << 20, 10, None, None) == -1
    assert L.lbm_batch_poll(None, 0, C.byref(lbm_job_result())) == -1
    assert L.lbm_batch_get_info(None, C.byref(lbm_batch_info())) == -1
    assert L.lbm_batch_wait(None, -1, 0.0, None) == -1
    assert L.lbm_batch_fetch(None, 0, None, None, None) == -1
    L.lbm_batch_destroy(None)
    assert L.lbm_tune(None, 3, None) == -1
    assert L.lbm_measure_peaks(None, None, None) == -1
    assert L.lbm_set_launch(None, 96, 2) == -1
