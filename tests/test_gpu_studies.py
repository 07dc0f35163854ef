"""The paper's single-colloid validation (Sec. IV.A) on the GPU, at the
paper's parameters converted to lattice units (a = 1 nm, tau = 3.1 ps, the
energy unit k_BT, so the fluid density is rho_0 = 1 / 0.0397 in those units):
R = 4, Z = 30, 1e-3 mol/l of a monovalent salt (6.02e-4 per cell and species),
D = 2e-9 m^2/s (0.0062), nu = 2.78, l_B = 0.714, E = 256.9 kV/m (0.00998),
TRT with Lambda = 3/16, a 64^3 periodic box.  FP32-storage form (its mobility
follows the FP64 form's within 1e-3, tests/test_gpu_fp32.py).

- the reduced mobility mu = 6 pi eta l_B v / (e E) of a sphere moved by the
  partial-volume scheme oscillates with the period of one cell of motion by
  less than the simple scheme's (the paper: 1.7% against 20.3%; here about 1%
  against 3%);
- the effective radius (the time-averaged number of cells completely inside
  the moving sphere, set equal to 4/3 pi R_eff^3) calibrates a fixed sphere
  whose electro-osmotic mobility then matches the moving one (the paper: 1.4%
  and 2.4%);
- the double layer around the moving sphere matches the fixed sphere's;
- the paper's low-charge colloid (Z = 3) moves with Henry's mobility.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KT_PAPER = 0.0397      # k_BT in units of rho_fluid a^5 / tau^2 (Table I: a = 1 nm, tau = 0.2 dt)
RHO0 = 1.0 / KT_PAPER  # fluid density in units with k_BT = 1
NU = 2.78
D = 0.0062
SALT = 6.02e-4
LB = 0.714
E = 0.00998
Z = 30.0
N = 64
FP32 = 16


def system(ek, radius, pv=True, fixed=False, pos=(32.3, 31.8, 32.1)):
    flags = ek.EK_NEUTRALIZE | (ek.EK_PV if pv else 0) | FP32
    s = ek.EKSystem((N, N, N), nu=NU, rho0=RHO0, bjerrum=LB, valence=(1, -1), D=(D, D),
                    bulk=(SALT, SALT), flags=flags, magic=3.0 / 16.0)
    s.add_particle(pos, radius=radius, charge=Z, rho_p=2.0 * RHO0, fixed=fixed)
    s.set_field(ek.FIELD_E_EXT, np.array([E, 0.0, 0.0]))
    return s


def mobility(ek, s):
    """Reduced mobility of the particle relative to the mean fluid velocity."""
    v = s.get_particles()[0]["vel"][0]
    fluid = s.get_fields(ek.FIELD_OWNER) == -1
    u = s.get_fields(ek.FIELD_VELOCITY)[0][fluid].mean()
    eta = RHO0 * NU
    return 6.0 * math.pi * eta * LB * (v - u) / E


def run_moving(ek, pv, settle=40000, cells=2.0, every=25, fluid_every=20):
    """Mobility samples every `every` steps over `cells` cells of motion after
    `settle` steps (the particle answers a cell's flip within a few steps, the
    fluid's mean velocity changes slowly: it is read every `fluid_every`
    samples), and the cells completely inside (Psi = 1) at those reads."""
    s = system(ek, 4.0, pv=pv)
    s.step(settle)
    x0 = s.get_particles()[0]["pos"][0]
    eta = RHO0 * NU
    mus, inside = [], []
    u = 0.0
    while True:
        if len(mus) % fluid_every == 0:
            fluid = s.get_fields(ek.FIELD_OWNER) == -1
            u = s.get_fields(ek.FIELD_VELOCITY)[0][fluid].mean()
            inside.append(int((s.get_fields(ek.FIELD_PSI) >= 1.0).sum()))
        s.step(every)
        p = s.get_particles()[0]
        mus.append(6.0 * math.pi * eta * LB * (p["vel"][0] - u) / E)
        if (p["pos"][0] - x0) % N >= cells or len(mus) > 20000:
            break
    return np.array(mus), np.array(inside), s


def amplitude(mus):
    """Half the peak-to-peak range about the linear trend (the double layer's
    slow build-up still moves the mean), relative to the mean."""
    t = np.arange(len(mus), dtype=np.float64)
    res = mus - np.polyval(np.polyfit(t, mus, 1), t)
    return 0.5 * (res.max() - res.min()) / abs(mus.mean())


@pytest.fixture(scope="module")
def runs(gpu_lib):
    ek = gpu_lib
    mu_pv, in_pv, s_pv = run_moving(ek, True)
    mu_s, _, s_s = run_moving(ek, False)
    s_s.close()
    return dict(mu_pv=mu_pv, in_pv=in_pv, s_pv=s_pv, mu_simple=mu_s)


def test_partial_volumes_damp_the_oscillation(gpu_lib, runs):
    a_pv, a_s = amplitude(runs["mu_pv"]), amplitude(runs["mu_simple"])
    print(f"\nmobility {runs['mu_pv'].mean():.4f} (PV) {runs['mu_simple'].mean():.4f} (simple); "
          f"oscillation amplitude {100 * a_pv:.2f}% (PV) {100 * a_s:.2f}% (simple)")
    print("PV     " + " ".join(f"{v:.4f}" for v in runs["mu_pv"][::80]))
    print("simple " + " ".join(f"{v:.4f}" for v in runs["mu_simple"][::80]))
    assert runs["mu_pv"].mean() > 0.0  # a positive sphere moves along E
    # the paper: 1.7% with partial volumes, 20.3% without; here the simple
    # scheme's oscillation is much smaller than the paper's (about 3%), so the
    # test asks for the partial-volume amplitude and a clear reduction
    assert a_pv < 0.02
    assert a_s > 2.0 * a_pv


def test_effective_radius_calibrates_the_fixed_sphere(gpu_lib, runs):
    ek = gpu_lib
    nbar = runs["in_pv"].mean()
    r_eff = (3.0 * nbar / (4.0 * math.pi)) ** (1.0 / 3.0)
    # a fixed sphere with the same number of cells completely inside
    best = None
    for r in np.arange(3.6, 4.6, 0.02):
        s = system(ek, float(r), fixed=True)
        n_in = int((s.get_fields(ek.FIELD_PSI) >= 1.0).sum())
        s.close()
        if best is None or abs(n_in - nbar) < abs(best[1] - nbar):
            best = (float(r), n_in)
    s = system(ek, best[0], fixed=True)
    s.step(30000)
    mu_fixed = np.mean([(s.step(500), mobility(ek, s))[1] for _ in range(10)])
    mu_moving = runs["mu_pv"].mean()
    print(f"\ncells inside {nbar:.1f} -> R_eff {r_eff:.3f}; fixed sphere R = {best[0]:.2f} "
          f"({best[1]} cells inside): mobility {mu_fixed:.4f} fixed, {mu_moving:.4f} moving, "
          f"{100 * abs(mu_moving / mu_fixed - 1):.2f}% apart")
    assert 3.0 < r_eff < 4.0
    assert abs(mu_moving / mu_fixed - 1.0) < 0.03
    runs["fixed"] = s


def _radial_charge(ek, s, centre):
    """Ion charge density averaged over shells of unit width around `centre`."""
    q = s.get_fields(ek.FIELD_SPECIES, 0) - s.get_fields(ek.FIELD_SPECIES, 1)
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")

    def mi(a, c):
        d = a - c
        return np.where(d > N / 2, d - N, np.where(d < -N / 2, d + N, d))

    r = np.sqrt(mi(x, centre[0]) ** 2 + mi(y, centre[1]) ** 2 + mi(z, centre[2]) ** 2)
    fluid = s.get_fields(ek.FIELD_OWNER) == -1
    edges = np.arange(4.0, 20.0, 1.0)
    prof = []
    for lo in edges:
        m = fluid & (r >= lo) & (r < lo + 1.0)
        prof.append(q[m].mean())
    return edges, np.array(prof)


def test_double_layer_of_the_moving_sphere_matches_the_fixed_one(gpu_lib, runs):
    ek = gpu_lib
    if "fixed" not in runs:
        pytest.skip("needs the calibrated fixed sphere")
    s_m, s_f = runs["s_pv"], runs["fixed"]
    _, pm = _radial_charge(ek, s_m, s_m.get_particles()[0]["pos"])
    edges, pf = _radial_charge(ek, s_f, s_f.get_particles()[0]["pos"])
    scale = np.abs(pf).max()
    diff = np.abs(pm - pf) / scale
    print("\nshell  " + " ".join(f"{e:5.0f}" for e in edges))
    print("fixed  " + " ".join(f"{v / scale:5.2f}" for v in pf))
    print("moving " + " ".join(f"{v / scale:5.2f}" for v in pm))
    assert pf[0] < 0.0 and pm[0] < 0.0   # counter-ions (negative) next to the positive sphere
    assert diff[2:].max() < 0.05          # beyond the first shells: the same layer
    assert diff.max() < 0.25              # next to the surface: the radii differ slightly


def henry_reduced_mobility(Z, a, kappa):
    """Henry's mobility of a weakly charged sphere (Debye-Hueckel zeta), with
    Ohshima's closed form of Henry's function, as the reduced mobility
    6 pi eta l_B mu / e = l_B Z f(kappa a) / (a (1 + kappa a))."""
    ka = kappa * a
    delta = 2.5 / (1.0 + 2.0 * math.exp(-ka))
    f = 1.0 + 1.0 / (2.0 * (1.0 + delta / ka) ** 3)
    return LB * Z * f / (a * (1.0 + ka))


def test_low_charge_mobility_against_henry(gpu_lib):
    """The paper's low-charge colloid (Z = 3, R = 4, zeta ~ 0.4 k_BT/e: the
    linear regime) in the FP64 form: the stationary reduced mobility against
    Henry's, with the lattice sphere's radius taken as R.  This pins the force
    on the particle as a whole (momentum exchange plus the reading of the
    solute's force on it) at first order in the charge."""
    ek = gpu_lib
    s = ek.EKSystem((N, N, N), nu=NU, rho0=RHO0, bjerrum=LB, valence=(1, -1), D=(D, D),
                    bulk=(SALT, SALT), flags=ek.EK_PV | ek.EK_NEUTRALIZE, magic=3.0 / 16.0)
    s.add_particle((32.3, 31.8, 32.1), radius=4.0, charge=3.0, rho_p=2.0 * RHO0)
    s.set_field(ek.FIELD_E_EXT, np.array([E, 0.0, 0.0]))
    s.step(30000)
    mus = []
    for _ in range(10):
        s.step(1000)
        mus.append(mobility(ek, s))
    mu = float(np.mean(mus))
    kappa = math.sqrt(4.0 * math.pi * LB * 2.0 * SALT)
    ref = henry_reduced_mobility(3.0, 4.0, kappa)
    bare = LB * 3.0 / 4.0  # Z E / (6 pi eta R) in reduced units
    print(f"\nreduced mobility {mu:.4f}, Henry {ref:.4f} ({100 * (mu / ref - 1):+.2f}%), "
          f"unscreened {bare:.4f}; drift over the window {100 * (max(mus) - min(mus)) / mu:.2f}%")
    assert (max(mus) - min(mus)) < 0.02 * mu
    assert abs(mu / ref - 1.0) < 0.08
