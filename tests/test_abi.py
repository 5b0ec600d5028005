"""The C ABI without a GPU: the library loads, exports every symbol include/ch.h declares,
the ctypes mirrors match the C struct layouts, and host-side argument checks fire
before any device work."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2204_03575_gb300 import ch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ch.h")


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(ch.LIB_PATH):
        from paper_2204_03575_gb300 import build
        build.build()
    return ch.lib()


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ch_[A-Za-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_binding_surface():
    decl = declared_functions()
    assert set(decl) == set(ch.exported_symbols())


def test_library_exports_every_declared_symbol(L):
    out = subprocess.run(["nm", "-D", "--defined-only", ch.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (ch_[A-Za-z_0-9]+)", out))
    missing = set(declared_functions()) - exported
    assert not missing, missing


def _c_layout(struct, fields):
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"ch.h\"\nint main(void){\n"
    src += f'printf("%zu\\n", sizeof({struct}));\n'
    for f in fields:
        src += f'printf("%zu\\n", offsetof({struct}, {f}));\n'
    src += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    return vals[0], vals[1:]


@pytest.mark.parametrize("cls,cname", [(ch.Params, "ch_params"), (ch.StepStats, "ch_step_stats"),
                                       (ch.ProfEntry, "ch_prof_entry")])
def test_struct_layout_matches_c(cls, cname):
    names = [n for n, _ in cls._fields_]
    size, offs = _c_layout(cname, names)
    assert ctypes.sizeof(cls) == size
    assert [getattr(cls, n).offset for n in names] == offs


def test_defaults_are_the_papers(L):
    p = ch.Params()
    assert (p.tau, p.eps, p.k_evap, p.g_p, p.g_nfa, p.h_p) == (1e-4, 1e-3, 5e-3, 0.01, 0.01, 0.0)
    assert p.rtol == 1e-8 and p.bc_mode == 1 and p.evap_sign == 1 and p.precision == 0
    assert p.cheb_degree == 0 and p.vcycles_H == 2 and p.vcycles_M == 1 and p.autotune == 1
    assert p.coarse_max == 0 and p.cheb_degree_coarse == 0 and p.krylov == 0
    assert p.cheb_degree_M == 0 and p.pattern == 0
    assert p.precond_M == 0 and p.cheb_M_steps == 0
    assert (p.chi_pn, p.chi_ps, p.chi_ns, p.N_p, p.N_nfa, p.N_s) == (1.0, 0.3, 0.3, 20.0, 20.0, 1.0)
    assert p.fh_delta == 1e-10 and p.pdl == 1 and p.gs_reorth == 0


def test_status_strings(L):
    for code in range(9):
        assert L.ch_status_str(code)


@pytest.mark.parametrize("bad", [dict(dim=4), dict(nx=0), dict(tau=-1.0), dict(eps=0.0), dict(restart=0),
                                 dict(restart=65), dict(rtol=2.0), dict(precision=3), dict(bc_mode=2),
                                 dict(evap_sign=0), dict(coarse_max=-1), dict(coarse_max=4097),
                                 dict(cheb_degree_coarse=-1), dict(cheb_degree_coarse=17),
                                 dict(cheb_degree=-1), dict(cheb_degree=17),
                                 dict(krylov=2), dict(cheb_degree_M=-1), dict(cheb_degree_M=17),
                                 dict(pattern=2), dict(pattern=-1), dict(potential=4),
                                 dict(precond_M=2), dict(cheb_M_steps=17), dict(cheb_M_steps=-1),
                                 dict(N_p=0.0), dict(N_s=-1.0), dict(fh_delta=0.0), dict(fh_delta=1.0),
                                 dict(chi_pn=float("nan")), dict(pdl=2), dict(pdl=-1),
                                 dict(gs_reorth=2), dict(gs_reorth=-1)])
def test_invalid_params_rejected_on_host(L, bad):
    p = ch.Params(**bad)
    h = ctypes.c_void_p()
    st = L.ch_mesh(ctypes.byref(p), None, ctypes.byref(h))
    assert st == ch.ERR_ARG and not h.value
    assert L.ch_last_error()


def test_null_handles_rejected(L):
    assert L.ch_step(None, None, None) == ch.ERR_ARG
    assert L.ch_precond_apply(None, None, None, None) == ch.ERR_ARG
    assert L.ch_apply_A(None, None, None, None) == ch.ERR_ARG
    assert L.ch_precond_level(None, 0, 0, *([None] * 12), None) == ch.ERR_ARG
    L.ch_state_destroy(None)
    L.ch_mesh_destroy(None)


def test_profile_counters_without_gpu(L):
    ch.profile_enable(False)
    assert isinstance(ch.profile_read(reset=True), dict)
