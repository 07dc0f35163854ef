"""Pins of the oracle's particle coupling against what the paper and the
mathematics fix, independently of the oracle's own code:

- the nearest-surface partition of the solute force regions against exact
  rational arithmetic (ties to the lower index);
- the moving bounce-back term 6 w_i rho_0 c_i . v_b (Sec. III.B, Eq. 12): a
  fluid in uniform motion past a sphere whose surface moves with it is a steady
  state, and next to a spinning sphere every bounced population is the
  equilibrium population of the local rigid-body velocity;
- the torque arm, the torque sums and I = 2/5 m R^2: total angular momentum of
  fluid and a free spinning sphere is conserved exactly while the disturbance
  has not reached the periodic images; the steady torque on a spinning sphere
  against Stokes' -8 pi eta R^3 omega;
- the refill and expel weights of Eqs. 17-18 on a hand-worked example;
- the two other charge normalisations (Eq. 21 with the literal V_p, and the
  simple scheme's even spread over the boundary nodes).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import ek_oracle as O
from oracle.ek_oracle import EKOracle

# D3Q19 written out here (not taken from the oracle): rest, faces, edges
C19 = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
       (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1),
       (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
W19 = [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12


def equilibrium(rho, u, c, w):
    """Second-order lattice equilibrium of one direction (textbook D3Q19)."""
    cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2]
    uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
    return w * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu)


def oracle_dir(c):
    """Index of direction c in the oracle's velocity table."""
    return int(np.where((O.CV == np.array(c)).all(axis=1))[0][0])


# --------------------------------------------------------------------------
# nearest-surface partition (the reading of the solute force's regions)
# --------------------------------------------------------------------------
def test_nearest_particle_matches_exact_arithmetic():
    """Four fixed spheres of equal radius: A and B mirror images about the plane
    x = 16 (every node of that plane is an exact tie: it goes to A, the lower
    index); C and D the same but D moved 3e-10 towards the plane (the nodes of
    the plane go to D, although float distances would call them ties).  Every
    node in two or more widened boxes is decided again with exact rationals:
    surface distances of equal radii order like squared centre distances."""
    n = (32, 24, 32)
    R = 3.0
    pos = [(8.375, 5.5, 6.25), (23.625, 5.5, 6.25), (8.375, 17.5, 20.25),
           (23.625 - 3e-10, 17.5, 20.25)]
    o = EKOracle(*n, bulk=(0.0, 0.0))
    for p in pos:
        o.add_particle(p, radius=R, charge=0.0, fixed=True)
    nearest, regions = o.nearest_particle()
    nx, ny, nz = n
    cand = {}
    for pid, (flat, _, _, _) in enumerate(regions):
        for f in flat.tolist():
            cand.setdefault(f, []).append(pid)
    checked = 0
    for f, ps in cand.items():
        x, y, z = f % nx, (f // nx) % ny, f // (nx * ny)
        best = None
        for pid in ps:
            d2 = Fraction(0)
            for coord, c, L in ((x, pos[pid][0], nx), (y, pos[pid][1], ny), (z, pos[pid][2], nz)):
                d = Fraction(coord) - Fraction(c)
                if d > Fraction(L, 2):
                    d -= L
                if d < -Fraction(L, 2):
                    d += L
                d2 += d * d
            if best is None or d2 < best[0]:
                best = (d2, pid)
        assert nearest[f] == best[1], (x, y, z, ps)
        checked += len(ps) > 1
    assert checked > 1000
    # the planes themselves
    for y in range(2, 9):
        assert nearest[16 + nx * (y + ny * 6)] == 0
    for y in range(14, 21):
        assert nearest[16 + nx * (y + ny * 20)] == 3


# --------------------------------------------------------------------------
# moving bounce-back (Sec. III.B, Eq. 12)
# --------------------------------------------------------------------------
def test_uniform_flow_past_comoving_sphere_is_steady():
    """Fluid in uniform motion V around a fixed sphere whose surface moves at V:
    the reflected population f*_i - 6 w_i rho_0 c_i.V equals the equilibrium of
    the opposite direction, so one full step leaves every fluid population at
    the equilibrium of V and density rho_0 (a factor other than 6 breaks it)."""
    V = np.array([0.01, -0.004, 0.006])
    o = EKOracle(16, 16, 16, bulk=(0.0, 0.0))
    o.add_particle((7.7, 8.2, 8.45), vel=V, radius=3.0, charge=0.0, fixed=True)
    fluid = o.owner == O.FLUID
    f0 = np.zeros_like(o.f)
    for i, c in enumerate(O.CV):
        f0[i] = np.where(fluid, equilibrium(1.0, V, c, O.WT[i]), 0.0)
    o.set_populations(f0)
    o.step()
    assert np.array_equal(o.owner, np.where(o.owner == O.FLUID, O.FLUID, o.owner))
    err = np.max(np.abs(o.f - f0)[:, fluid])
    assert err < 1e-15, err


def test_spinning_sphere_reflects_local_equilibrium():
    """Fluid in rigid motion u(x) = v + omega x (x - r_p) next to a fixed sphere
    that moves and spins with the same v and omega: since c_i . (omega x c_i) = 0,
    the wall velocity at the boundary node x + c_i has the same component along
    c_i as u(x), and every population bounced back into a fluid node is the
    equilibrium of the opposite direction at u(x).  A wrong sign of the
    rotation term or a factor other than 6 w_i rho_0 breaks it."""
    v = np.array([0.003, 0.001, -0.002])
    w = np.array([0.004, -0.003, 0.005])
    rp = np.array([8.3, 7.6, 8.15])
    o = EKOracle(16, 16, 16, bulk=(0.0, 0.0))
    o.add_particle(rp, vel=v, omega=w, radius=3.5, charge=0.0, fixed=True)
    nz, ny, nx = o.shape
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    d = [X - rp[0], Y - rp[1], Z - rp[2]]
    u = [v[0] + w[1] * d[2] - w[2] * d[1], v[1] + w[2] * d[0] - w[0] * d[2],
         v[2] + w[0] * d[1] - w[1] * d[0]]
    fluid = o.owner == O.FLUID
    f0 = np.zeros_like(o.f)
    for i, c in enumerate(O.CV):
        f0[i] = np.where(fluid, equilibrium(1.0, u, c, O.WT[i]), 0.0)
    o.set_populations(f0)
    fnew, _, _, _ = o.lb_step(np.zeros((3,) + o.shape))
    nlinks = 0
    for (z, y, x) in zip(*np.nonzero(fluid)):
        for c in C19[1:]:
            if o.owner[(z + c[2]) % nz, (y + c[1]) % ny, (x + c[0]) % nx] < 0:
                continue
            cb = (-c[0], -c[1], -c[2])
            ib = oracle_dir(cb)
            ux = [u[a][z, y, x] for a in range(3)]
            want = equilibrium(1.0, ux, cb, W19[C19.index(cb)])
            assert abs(fnew[ib, z, y, x] - want) < 1e-16, (x, y, z, c)
            nlinks += 1
    assert nlinks > 200


def _angular_momentum(o, r0):
    """Total angular momentum about r0 of the fluid (populations after
    streaming, positions as minimum-image offsets from r0) and of the
    particles (spin I omega with I = 2/5 m R^2, and orbit m (r_p - r0) x v)."""
    nz, ny, nx = o.shape
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")

    def mi(a, c, L):
        d = a - c
        return np.where(d > L / 2, d - L, np.where(d < -L / 2, d + L, d))

    d = [mi(X, r0[0], nx), mi(Y, r0[1], ny), mi(Z, r0[2], nz)]
    j = [sum(c[a] * o.f[oracle_dir(c)] for c in C19 if c[a]) for a in range(3)]
    L = np.array([(d[1] * j[2] - d[2] * j[1]).sum(), (d[2] * j[0] - d[0] * j[2]).sum(),
                  (d[0] * j[1] - d[1] * j[0]).sum()])
    P = np.array([j[a].sum() for a in range(3)])
    for p in o.particles:
        m = p.radius ** 3 * 4.0 / 3.0 * math.pi * p.rho_p
        inertia = 0.4 * m * p.radius ** 2
        rp = [mi(p.pos[a], r0[a], (nx, ny, nz)[a]) for a in range(3)]
        L = L + inertia * p.omega + m * np.cross(rp, p.vel)
        P = P + m * p.vel
    return L, P


def test_angular_momentum_conserved_spinning_free_sphere():
    """A free sphere set spinning in fluid at rest: the momentum exchange hands
    the fluid's angular momentum to the particle through the torque arm and
    I = 2/5 m R^2, so fluid + spin + orbit is conserved exactly as long as the
    disturbance has not reached the minimum-image planes (the rest fluid there
    carries no net angular momentum across).  A wrong arm, a sign or an inertia
    other than 2/5 m R^2 breaks it."""
    n = 24
    o = EKOracle(n, n, n, bulk=(0.0, 0.0))
    r0 = np.array([11.3, 12.6, 11.8])
    o.add_particle(r0, omega=(0.002, -0.003, 0.004), radius=3.0, charge=0.0, rho_p=1.5)
    owner0 = o.owner.copy()
    L0, P0 = _angular_momentum(o, r0)
    scale = float(np.abs(L0).max())
    for _ in range(6):  # disturbance within R + 1 + 6 < n / 2 of the centre
        o.step()
        L, P = _angular_momentum(o, r0)
        assert np.allclose(L, L0, rtol=0, atol=1e-13 * scale), (L - L0) / scale
        assert np.allclose(P, P0, rtol=0, atol=1e-13)
    assert np.array_equal(o.owner, owner0)  # no cell changed hands
    p = o.particles[0]
    assert np.all(np.sign(p.omega) == np.sign([0.002, -0.003, 0.004]))
    assert np.abs(p.omega).max() < 0.004  # the fluid slowed the spin down


@pytest.mark.slow
def test_spinning_sphere_torque_against_stokes():
    """Steady torque on a fixed sphere spinning at omega in a periodic 16^3 box
    against Stokes' -8 pi eta R_h^3 omega (eta = rho_0 nu = 1/6).  The lattice
    sphere of the 'centre strictly inside' rule is a little smaller than R and
    the periodic images add O(phi) (phi = 2.8% here); the ratio to the
    geometric radius's value must lie in [0.65, 1.0] and the torque must oppose
    the spin along the axis."""
    R = 3.0
    om = np.array([0.0, 0.0, 0.002])
    o = EKOracle(16, 16, 16, bulk=(0.0, 0.0))
    o.add_particle((8.0, 8.0, 8.0), omega=om, radius=R, charge=0.0, fixed=True)
    hist = []
    for _ in range(40):
        o.step(10)
        hist.append(o.particles[0].torque[2])
    Tz = hist[-1]
    assert abs(hist[-1] - hist[-5]) < 1e-3 * abs(Tz)  # steady
    stokes = -8.0 * math.pi * (1.0 / 6.0) * R ** 3 * om[2]
    ratio = Tz / stokes
    assert 0.65 <= ratio <= 1.0, ratio
    T = o.particles[0].torque
    assert abs(T[0]) < 1e-3 * abs(Tz) and abs(T[1]) < 1e-3 * abs(Tz)


# --------------------------------------------------------------------------
# refill and expel (Sec. III.D.1, Eqs. 17-18), hand-worked
# --------------------------------------------------------------------------
def _transition_case(flags):
    o = EKOracle(12, 12, 12, bulk=(1e-3, 1e-3), flags=flags)
    o.add_particle((3.2, 3.1, 3.3), radius=2.5, charge=0.0, fixed=True)
    old = o.owner.copy()
    A = (8, 8, 8)     # (x, y, z): vacated, all 18 neighbours stay fluid
    B = (9, 3, 9)     # claimed; three of its neighbours are boundary before and after
    blocked = [(10, 3, 9), (10, 4, 9), (10, 2, 9)]
    old[A[2], A[1], A[0]] = 0
    o.owner[B[2], B[1], B[0]] = 0
    old[B[2], B[1], B[0]] = O.FLUID
    for (x, y, z) in blocked:
        old[z, y, x] = 0
        o.owner[z, y, x] = 0
    rho = np.full((2,) + o.shape, 1e-3)
    rho[:, A[2], A[1], A[0]] = 0.0
    for i, c in enumerate(C19[1:], start=1):
        rho[0, A[2] + c[2], A[1] + c[1], A[0] + c[0]] = 1e-4 * (1 + i)
        rho[1, A[2] + c[2], A[1] + c[1], A[0] + c[0]] = 2e-4 * (19 - i)
    rho[:, B[2], B[1], B[0]] = (3e-3, 6e-3)
    for (x, y, z) in blocked:
        rho[:, z, y, x] = 0.0
    o.rho = rho.copy()
    return o, old, rho, A, B, blocked


def test_refill_and_expel_hand_example():
    """Vacated cell A with 18 fluid neighbours of densities 1e-4 (1 + i) (species
    0) and 2e-4 (19 - i) (species 1): Eq. 17 puts sum / 19 into A (0.0189 / 19
    and 0.0342 / 19) and Eq. 18 leaves each neighbour 18/19 of its density.
    Claimed cell B (3e-3, 6e-3) with 15 fluid neighbours (three are boundary):
    each receives 1/15 of B's solute (2e-4, 4e-4)."""
    o, old, rho, A, B, blocked = _transition_case(O.PV | O.NEUTRALIZE)
    o.transitions(old)
    r = o.rho
    assert r[0, A[2], A[1], A[0]] == pytest.approx(0.0189 / 19, rel=1e-14)
    assert r[1, A[2], A[1], A[0]] == pytest.approx(0.0342 / 19, rel=1e-14)
    for i, c in enumerate(C19[1:], start=1):
        z, y, x = A[2] + c[2], A[1] + c[1], A[0] + c[0]
        assert r[0, z, y, x] == pytest.approx(1e-4 * (1 + i) * 18 / 19, rel=1e-14)
        assert r[1, z, y, x] == pytest.approx(2e-4 * (19 - i) * 18 / 19, rel=1e-14)
    assert r[0, B[2], B[1], B[0]] == 0.0 and r[1, B[2], B[1], B[0]] == 0.0
    got = 0
    for c in C19[1:]:
        x, y, z = B[0] + c[0], B[1] + c[1], B[2] + c[2]
        if (x, y, z) in blocked:
            assert r[0, z, y, x] == 0.0
            continue
        assert r[0, z, y, x] == pytest.approx(1e-3 + 2e-4, rel=1e-14)
        assert r[1, z, y, x] == pytest.approx(1e-3 + 4e-4, rel=1e-14)
        got += 1
    assert got == 15
    # every other node unchanged
    touched = np.zeros(o.shape, dtype=bool)
    for P0 in (A, B):
        touched[P0[2], P0[1], P0[0]] = True
        for c in C19[1:]:
            touched[P0[2] + c[2], P0[1] + c[1], P0[0] + c[0]] = True
    assert np.array_equal(r[:, ~touched], rho[:, ~touched])


def test_vacate_zero_hand_example():
    """With vacated cells left empty the vacated cell stays at 0 and its
    neighbours keep their solute; the claimed cell still expels."""
    o, old, rho, A, B, blocked = _transition_case(O.PV | O.NEUTRALIZE | O.VACATE_ZERO)
    o.transitions(old)
    r = o.rho
    assert r[0, A[2], A[1], A[0]] == 0.0
    for i, c in enumerate(C19[1:], start=1):
        assert r[0, A[2] + c[2], A[1] + c[1], A[0] + c[0]] == 1e-4 * (1 + i)
    x, y, z = B[0] - 1, B[1], B[2]
    assert r[0, z, y, x] == pytest.approx(1.2e-3, rel=1e-14)


# --------------------------------------------------------------------------
# charge normalisations of the particle (Eq. 21 and the simple scheme)
# --------------------------------------------------------------------------
def _particle_charge_field(flags, Z=-12.0, R=3.3, pos=(8.21, 7.63, 8.48)):
    """Charge density of one sphere in a box without ions (no neutralisation)."""
    o = EKOracle(16, 16, 16, bulk=(0.0, 0.0), flags=flags)
    o.add_particle(pos, radius=R, charge=Z, fixed=True)
    return o, o.charge_density(), Z, R, np.array(pos)


def test_charge_literal_volume_normalisation():
    """Eq. 21 as printed: rho_b = Z Psi / V_p with V_p = 4/3 pi R^3, so the
    charge follows Psi with the factor Z / V_p, and the total is Z times the
    Psi volume over V_p (within the octree's depth-4 bound of 1)."""
    o, q, Z, R, _ = _particle_charge_field(O.PV | O.CHARGE_NORM_VP)
    Vp = 4.0 / 3.0 * math.pi * R ** 3
    on = o.psi > 0
    assert np.allclose(q[on], Z * o.psi[on] / Vp, rtol=1e-14, atol=0)
    assert np.all(q[~on] == 0.0)
    assert abs(q.sum() / Z - 1.0) < 0.02
    o2, q2, _, _, _ = _particle_charge_field(O.PV)
    assert abs(q2.sum() - Z) < 1e-13 * abs(Z)  # the default: divided by sum Psi


def test_charge_simple_scheme_even_spread():
    """Without partial volumes the charge Z is spread evenly over the boundary
    nodes, the lattice nodes whose centre is strictly inside the sphere
    (counted here by brute force in exact arithmetic)."""
    o, q, Z, R, rp = _particle_charge_field(0)
    inside = np.zeros(o.shape, dtype=bool)
    for z in range(16):
        for y in range(16):
            for x in range(16):
                d2 = sum((Fraction(a) - Fraction(float(c))) ** 2 for a, c in zip((x, y, z), rp))
                inside[z, y, x] = d2 < Fraction(R) ** 2
    nb = int(inside.sum())
    assert nb > 100
    assert np.allclose(q[inside], Z / nb, rtol=1e-15, atol=0)
    assert np.all(q[~inside] == 0.0)
    assert abs(q.sum() - Z) < 1e-12 * abs(Z)


# --------------------------------------------------------------------------
# Stokes drag in a periodic array (Hasimoto), on the oracle itself
# --------------------------------------------------------------------------
def _hasimoto_K(phi):
    """Hasimoto's correction for a simple cubic array of spheres: the drag is
    6 pi eta a U / K with K = 1 - 1.7601 phi^(1/3) + phi - 1.5593 phi^2."""
    return 1.0 - 1.7601 * phi ** (1.0 / 3.0) + phi - 1.5593 * phi ** 2


def _steady_drag(n, R, g, steps):
    """A fixed sphere in an n^3 periodic box, fluid driven by the body force g
    along x (nu = 1, TRT 3/16, no ions): the drag on the sphere and the mean
    fluid velocity at steady state."""
    o = EKOracle(n, n, n, nu=1.0, bulk=(0.0, 0.0), magic=3.0 / 16.0)
    o.add_particle((n / 2 + 0.3, n / 2 - 0.2, n / 2 + 0.1), radius=R, charge=0.0, fixed=True)
    o.g = np.array([g, 0.0, 0.0])
    hist = []
    for _ in range(steps // 50):
        o.step(50)
        hist.append(o.particles[0].force[0])
    fluid = o.owner == O.FLUID
    U = float(o.u[0][fluid].mean())
    return hist, U, o


@pytest.mark.slow
def test_stokes_drag_with_hasimoto_correction():
    """At steady state the momentum exchange carries the whole body force
    (g times the fluid nodes).  The hydrodynamic radius fitted to the 12^3
    box's drag through Hasimoto's law predicts the 16^3 box's within 5%."""
    eta = 1.0
    R, g = 2.5, 2e-6
    h12, U12, o12 = _steady_drag(12, R, g, 600)
    h16, U16, o16 = _steady_drag(16, R, g, 1200)
    for h, o in ((h12, o12), (h16, o16)):
        assert abs(h[-1] - h[-2]) < 1e-4 * abs(h[-1])  # steady
        nf = int((o.owner == O.FLUID).sum())
        assert abs(h[-1] - g * nf) < 2e-3 * g * nf     # the drag balances the body force

    def drag(a, n, U):
        phi = 4.0 / 3.0 * math.pi * a ** 3 / n ** 3
        return 6.0 * math.pi * eta * a * U / _hasimoto_K(phi)

    # fit a on the 12^3 box (bisection: the drag grows with a)
    lo, hi = 1.5, 3.5
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if drag(mid, 12, U12) < h12[-1]:
            lo = mid
        else:
            hi = mid
    a = 0.5 * (lo + hi)
    pred = drag(a, 16, U16)
    assert 1.8 < a < 2.8
    assert abs(pred / h16[-1] - 1.0) < 0.05, (a, pred, h16[-1])
