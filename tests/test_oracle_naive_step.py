"""Brute force: the oracle's whole time step against a second restatement
written node by node with plain loops (tests/naive_step.py), on a small box
with two moving, spinning, charged spheres whose widened boxes overlap, for
several steps: populations, species, particle state, boundary flags and Psi
agree to rounding.  The two share nothing but the state they start from."""
import numpy as np
import pytest

from oracle import ek_oracle as O
from oracle.ek_oracle import EKOracle
from naive_step import C, State


def _order():
    return [int(np.where((O.CV == np.array(c)).all(axis=1))[0][0]) for c in C]


@pytest.mark.parametrize("flags,magic,nx", [(O.PV | O.NEUTRALIZE, 3.0 / 16.0, 12),
                                            (O.NEUTRALIZE, None, 12),
                                            (O.PV | O.NEUTRALIZE | O.VACATE_ZERO | O.CHARGE_NORM_VP, None, 12),
                                            (O.PV | O.NEUTRALIZE, None, 36)])
def test_full_step_against_naive_restatement(flags, magic, nx):
    """nx = 36 leaves fluid outside both widened boxes (the shared remainder)."""
    o = EKOracle(nx, 10, 11, bulk=(2e-3, 1e-3), flags=flags, magic=magic)
    o.E = np.array([0.01, 0.002, -0.004])
    o.g = np.array([1e-5, 0.0, 2e-5])
    o.add_particle((3.6, 4.9, 5.3), vel=(0.06, -0.02, 0.03), omega=(0.004, 0.006, -0.005),
                   radius=1.7, charge=-3.0, rho_p=1.2)
    o.add_particle((8.9, 4.4, 5.8), vel=(-0.05, 0.03, -0.02), omega=(-0.003, 0.002, 0.004),
                   radius=1.6, charge=-2.0, rho_p=1.3)
    rng = np.random.default_rng(5)
    o.set_populations(o.f * (1 + 0.01 * rng.standard_normal(o.f.shape)) * (o.owner == -1))
    for k in range(2):
        o.set_species(k, o.rho[k] * (1 + 0.2 * rng.random(o.shape)))
    order = _order()
    s = State(o, order)
    flips = 0
    for step in range(6):
        old = o.owner.copy()
        o.step()
        s.step()
        flips += int((old != o.owner).sum())
        assert np.array_equal(s.owner, o.owner), step
        assert np.max(np.abs(s.psi_field() - o.psi)) == 0.0
        fo = np.array([o.f[order[i]] for i in range(19)])
        assert np.max(np.abs(s.f - fo)) < 1e-14 * np.max(np.abs(fo)), step
        assert np.max(np.abs(s.rho - o.rho)) < 1e-13 * np.max(np.abs(o.rho)), step
        for p, q in zip(s.parts, o.particles):
            assert np.allclose(p["pos"], q.pos, rtol=0, atol=1e-13)
            assert np.allclose(p["vel"], q.vel, rtol=1e-10, atol=1e-15)
            assert np.allclose(p["om"], q.omega, rtol=1e-10, atol=1e-15)
            assert np.allclose(p["force"], q.force, rtol=1e-10, atol=1e-15)
            assert np.allclose(p["torque"], q.torque, rtol=1e-10, atol=1e-15)
            assert np.allclose(p["ftr"], q.f_trans, rtol=1e-10, atol=1e-15)
        # the naive state continues from the oracle's (the sums differ in order)
        s = State(o, order)
    assert flips > 0  # the spheres claimed and released cells
