"""Parity of the CUDA FP64 path with the FP64 oracle where the nearest-surface
partition of the solute force decides (ties and near-ties between particles)
and on a crowded box shaped like the many-colloid workload (several spheres
of radius 5, three species with valences +1, -1, +2).  Tolerance 1e-11
relative per element (tests/pairs.py)."""
import numpy as np
import pytest

import workloads
from pairs import compare, make_pair

pytestmark = pytest.mark.gpu


def _tie_case():
    """Four spheres R = 3: 0 and 1 mirror images about the plane x = 16 (exact
    FP64 ties on the plane: the lower index), 2 and 3 the same with 3 moved
    3e-10 towards the plane (it wins in FP64, while the float distances tie)."""
    case = workloads.small_case(n=(32, 24, 32), radius=3.0, charge=-10.0, nparticles=0)
    pos = [(8.375, 5.5, 6.25), (23.625, 5.5, 6.25), (8.375, 17.5, 20.25),
           (23.625 - 3e-10, 17.5, 20.25)]
    case["particles"] = [dict(pos=list(p), radius=3.0, charge=c)
                         for p, c in zip(pos, (-10.0, -7.0, -12.0, -9.0))]
    return case


def test_nearest_surface_ties_fixed_spheres(gpu_lib):
    """Fixed spheres keep their ties every step; the particle forces (which
    hold the solute force summed over each particle's region) must match."""
    ek = gpu_lib
    case = _tie_case()
    o, s = make_pair(ek, case, fixed=True)
    for _ in range(3):
        o.step(2)
        s.step(2)
        compare(ek, o, s)
    nearest, _ = o.nearest_particle()
    nx, ny = 32, 24
    assert nearest[16 + nx * (5 + ny * 6)] == 0
    assert nearest[16 + nx * (17 + ny * 20)] == 3


def test_nearest_surface_ties_free_spheres(gpu_lib):
    ek = gpu_lib
    case = _tie_case()
    o, s = make_pair(ek, case, vel=[(0.01, 0.0, 0.0), (-0.01, 0.0, 0.0), (0.0, 0.01, 0.0),
                                    (0.0, -0.01, 0.0)])
    for _ in range(3):
        o.step(3)
        s.step(3)
        compare(ek, o, s)


def _crowded_case():
    """64^3, six spheres R = 5 by random sequential addition (centre gap >= 2R + 2)
    with charges in [-99, -33], plus a pair 12.25 - 2e-10 apart whose mid-plane
    nodes are a near-tie; three species z = +1, -1, +2 (D = 0.2, 0.3, 0.15,
    bulk 1e-3), E = 0.005 along x."""
    case = workloads.small_case(n=(64, 64, 64), radius=5.0, charge=-66.0, nparticles=6, seed=23,
                                E=0.005)
    case["valence"], case["D"], case["bulk"] = (1, -1, 2), (0.2, 0.3, 0.15), (1e-3, 1e-3, 1e-3)
    # a free spot for the pair: the first on a coarse grid clear of the others
    parts = case["particles"]

    def clear(c):
        for q in parts:
            d2 = 0.0
            for a in range(3):
                d = abs(c[a] - q["pos"][a])
                d = min(d, 64 - d)
                d2 += d * d
            if d2 < 12.0 ** 2:
                return False
        return True

    for x in range(8, 64, 4):
        for y in range(4, 64, 4):
            for z in range(4, 64, 4):
                a = (x - 6.125, y + 0.5, z + 0.25)
                b = (x + 6.125 - 2e-10, y + 0.5, z + 0.25)
                if clear(a) and clear(b):
                    parts += [dict(pos=list(a), radius=5.0, charge=-80.0),
                              dict(pos=list(b), radius=5.0, charge=-95.0)]
                    return case
    raise RuntimeError("no room for the pair")


def test_crowded_three_species_100_steps(gpu_lib):
    ek = gpu_lib
    case = _crowded_case()
    assert len(case["particles"]) == 8
    o, s = make_pair(ek, case, perturb=0.0)
    N0 = o.total_species().copy()
    for _ in range(4):
        o.step(25)
        s.step(25)
        compare(ek, o, s)
    tot = np.array([s.get_fields(ek.FIELD_SPECIES, k).sum() for k in range(3)])
    assert np.allclose(tot, N0, rtol=1e-12, atol=0)
