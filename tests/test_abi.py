"""CPU checks of the C ABI: the library loads, exports every function the
header declares, the ctypes structs match the C layout, and argument
validation fails with LBM_E_INVALID before any device call."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2609_28679_b300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2609_28679_b300 import build

    build.build()
    return lbm.load_library()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_function_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layout_matches_header():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "lbm.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(lbm_lattice), sizeof(lbm_eos), sizeof(lbm_force), sizeof(lbm_heat));
  printf("%zu %zu %zu %zu %zu\n", offsetof(lbm_eos, kappa), offsetof(lbm_eos, t_solver), offsetof(lbm_lattice, phi_scheme), offsetof(lbm_eos, mu), offsetof(lbm_eos, isothermal));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    sizes = [int(x) for x in out]
    assert sizes[:4] == [ctypes.sizeof(lbm.lbm_lattice), ctypes.sizeof(lbm.lbm_eos),
                         ctypes.sizeof(lbm.lbm_force), ctypes.sizeof(lbm.lbm_heat)]
    assert sizes[4] == lbm.lbm_eos.kappa.offset
    assert sizes[5] == lbm.lbm_eos.t_solver.offset
    assert sizes[6] == lbm.lbm_lattice.phi_scheme.offset
    assert sizes[7] == lbm.lbm_eos.mu.offset
    assert sizes[8] == lbm.lbm_eos.isothermal.offset


def _create(lib, lat, eos, tau=0.8):
    h = ctypes.c_void_p()
    rc = lib.lbm_create(ctypes.byref(lat), ctypes.byref(eos), tau, tau, None, None, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("lat_kw,eos_kw,tau,why", [
    (dict(dim=4), {}, 0.8, "dim"),
    (dict(nx=0), {}, 0.8, "nx"),
    (dict(nz=2), {}, 0.8, "nz"),
    (dict(zwalls=1), {}, 0.8, "walls"),
    (dict(storage=7), {}, 0.8, "storage"),
    (dict(phi_scheme=5), {}, 0.8, "phi"),
    ({}, dict(kind=9), 0.8, "kind"),
    ({}, dict(R=0.0), 0.8, "R"),
    ({}, {}, 0.0, "tau"),
    ({}, dict(kind=lbm.LBM_PR, Tc=0.0), 0.8, "Tc"),
    ({}, dict(mu=-1.0), 0.8, "mu"),
    ({}, dict(mu=float("nan")), 0.8, "mu nan"),
    ({}, dict(isothermal=2), 0.8, "isothermal flag"),
    ({}, dict(kind=lbm.LBM_PR, Tc=0.5, Pc=0.15, t_solver=lbm.LBM_T_MLP, isothermal=1), 0.8, "isothermal learned"),
    (dict(dim=3, nz=8, zwalls=3), {}, 0.8, "zwalls value"),
    (dict(dim=3, nz=3, zwalls=2), {}, 0.8, "extrapolation walls need nz >= 4"),
    (dict(dim=3, nz=8, zwalls=2), dict(isothermal=1), 0.8, "extrapolation walls set T"),
])
def test_invalid_arguments_rejected_without_device(lib, lat_kw, eos_kw, tau, why):
    lat = lbm.lbm_lattice(**{**dict(dim=2, nx=8, ny=8, nz=1, zwalls=0, storage=0, phi_scheme=0), **lat_kw})
    eos = lbm.lbm_eos(**{**dict(kind=0, R=1.0, cv=2.5), **eos_kw})
    rc, h = _create(lib, lat, eos, tau)
    assert rc == lbm.LBM_E_INVALID
    assert not h.value
    assert lib.lbm_last_error(None)


def test_isothermal_with_heat_source_rejected_without_device(lib):
    lat = lbm.lbm_lattice(dim=2, nx=8, ny=8, nz=1, zwalls=0, storage=0, phi_scheme=0)
    eos = lbm.lbm_eos(kind=0, R=1.0, cv=2.5, isothermal=1)
    heat = lbm.lbm_heat(1e-6, 0, 0)
    h = ctypes.c_void_p()
    rc = lib.lbm_create(ctypes.byref(lat), ctypes.byref(eos), 0.8, 0.8, None, ctypes.byref(heat), ctypes.byref(h))
    assert rc == lbm.LBM_E_INVALID and not h.value


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.lbm_step(None, 1) == lbm.LBM_E_INVALID
    assert lib.lbm_set_force(None, None) == lbm.LBM_E_INVALID
    assert lib.lbm_set_walls(None, None, 1.0, None, 1.0, 0) == lbm.LBM_E_INVALID
    assert lib.lbm_set_face(None, 0, lbm.LBM_FACE_OUTLET_P, None, 1.0, 1.0) == lbm.LBM_E_INVALID


@pytest.mark.parametrize("friction", [-1e-3, float("nan")])
def test_invalid_friction_rejected_without_device(lib, friction):
    lat = lbm.lbm_lattice(dim=3, nx=1, ny=1, nz=8, zwalls=0, storage=0, phi_scheme=0)
    eos = lbm.lbm_eos(kind=0, R=1.0, cv=2.5)
    force = lbm.lbm_force((ctypes.c_double * 3)(0.0, 0.0, 0.0), friction)
    h = ctypes.c_void_p()
    rc = lib.lbm_create(ctypes.byref(lat), ctypes.byref(eos), 0.8, 0.8, ctypes.byref(force), None, ctypes.byref(h))
    assert rc == lbm.LBM_E_INVALID and not h.value
    assert lib.lbm_invariants(None, None) == lbm.LBM_E_INVALID
    lib.lbm_destroy(None)
