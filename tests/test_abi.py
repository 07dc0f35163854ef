"""Host-side checks of the C ABI: the library builds, loads without a GPU and
exports every entry point that include/ek.h declares; the binding validates."""
import ctypes
import os
import re

import pytest

from paper_1607_04572_gb300 import build as ekbuild
from paper_1607_04572_gb300 import ek

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    text = open(os.path.join(ROOT, "include", "ek.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ek_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    path = ekbuild.build()
    return ctypes.CDLL(path)


def test_header_declares_the_api():
    names = declared_entry_points()
    for n in ("ek_create", "ek_add_particle", "ek_set_field", "ek_step", "ek_get_fields",
              "ek_get_particles", "ek_poisson_solve"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    assert set(declared_entry_points()) == set(ek.EXPORTS)


def test_lattice_dirs_without_gpu():
    c = ek.lattice_dirs()
    assert c.shape == (19, 3)
    assert (c[0] == 0).all()
    # every direction has its opposite; 6 faces and 12 edges
    for v in c:
        assert any((w == -v).all() for w in c)
    assert sorted((c ** 2).sum(1).tolist()) == [0] + [1] * 6 + [2] * 12


def test_struct_layout_matches_header():
    # ek_params: 3 ints, pad, 4 doubles, int, 4 ints, pad, 8 doubles, unsigned
    assert ctypes.sizeof(ek.Params) == 4 * 3 + 4 + 8 * 4 + 4 + 4 * 4 + 4 + 8 * 8 + 8
    assert ctypes.sizeof(ek.ParticleRec) == 8 * 15 + 8 * 3 + 8


def test_new_entry_points_check_arguments_without_gpu(lib):
    """Argument checks that return before any CUDA call."""
    import ctypes as C
    lib.ek_get_state.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    lib.ek_set_state.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t]
    lib.ek_poisson_solve_mg.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                        C.c_double, C.c_double, C.c_int, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p]
    assert lib.ek_get_state(None, None, None) == -1
    assert lib.ek_set_state(None, None, 0) == -1
    assert lib.ek_poisson_solve_mg(None, None, 32, 32, 32, 0.7, 1e-12, 10, None, None, None,
                                   None) == -1


def test_multigrid_scratch_size_without_gpu():
    # 32^3: levels 32^3 and 16^3 (the coarsest, solved by FFT); scratch = b
    # and r of the box (8 B each per node), phi, b and r of 16^3, the
    # half spectrum of 16^3 (9 x 16 x 16 complex doubles) and 516 doubles
    # of reduction slots, every part rounded up to 256 bytes
    up = lambda b: (b + 255) // 256 * 256
    want = 2 * up(32 ** 3 * 8) + 3 * up(16 ** 3 * 8) + up(9 * 16 * 16 * 16) + up(516 * 8)
    assert ek.poisson_mg_scratch_bytes((32, 32, 32)) == want
    # a box that cannot be coarsened keeps only its own level
    assert ek.poisson_mg_scratch_bytes((12, 96, 27)) == (
        2 * up(12 * 96 * 27 * 8) + up(7 * 96 * 27 * 16) + up(516 * 8))
    assert ek.poisson_mg_scratch_bytes((10, 32, 32)) == 0  # 10 is not 2^a 3^b
