"""Helpers of the GPU parity tests: build the CUDA system and the FP64 oracle
from the same seeded inputs, and compare their fields.

Tolerance (the parity metric for the FP64 path): per element
    |x_gpu - x_ref| <= TOL * max(|x_ref|, 1e-3 * max|x_ref|),  TOL = 1e-11,
the floor keeps zero crossings of Phi from dividing by ~0.  The fluid velocity
u = (sum_i f_i c_i + f/2)/rho is a difference of populations of size w_i rho,
so its per-node rounding grows like rho/|u| (~1e3 and more); it is compared
normwise instead: max|u_gpu - u_ref| <= TOL * max|u_ref|.
"""
import numpy as np

import workloads
from oracle import ek_oracle as O
from oracle.ek_oracle import EKOracle

TOL = 1e-11


def perm_to_oracle(ek):
    """Index map: oracle direction i -> library direction perm[i]."""
    c = ek.lattice_dirs()
    perm = []
    for v in O.CV:
        perm.append(int(np.where((c == v).all(axis=1))[0][0]))
    return np.array(perm)


def make_pair(ek, case, flags=O.PV | O.NEUTRALIZE, magic=None, perturb=0.01, seed=11,
              walls=None, wall_charge=None, fixed=False, vel=None, rho_p=None, omega=None,
              g=(0.0, 0.0, 0.0)):
    nx, ny, nz = case["shape"]
    kw = dict(nu=case["nu"], rho0=case["rho0"], bjerrum=case["bjerrum"],
              valence=case["valence"], D=case["D"], bulk=case["bulk"], flags=flags)
    o = EKOracle(nx, ny, nz, magic=magic, **kw)
    s = ek.EKSystem((nx, ny, nz), magic=magic or 0.0, **kw)
    if wall_charge is not None:
        o.set_wall_charge(wall_charge)
        s.set_field(ek.FIELD_WALL_CHARGE, wall_charge)
    if walls is not None:
        o.set_walls(walls)
        s.set_field(ek.FIELD_WALL, walls.astype(np.float64))
    for j, p in enumerate(case["particles"]):
        v = vel[j] if vel is not None else (0.0, 0.0, 0.0)
        w = omega[j] if omega is not None else (0.0, 0.0, 0.0)
        rp = rho_p if rho_p is not None else case["rho_p"]
        o.add_particle(p["pos"], vel=v, radius=p["radius"], charge=p["charge"], rho_p=rp,
                       fixed=fixed, omega=w)
        s.add_particle(p["pos"], vel=v, radius=p["radius"], charge=p["charge"], rho_p=rp,
                       fixed=fixed, omega=w)
    E = np.array(case["E"], dtype=np.float64)
    o.E = E.copy()
    s.set_field(ek.FIELD_E_EXT, E)
    o.g = np.array(g, dtype=np.float64)
    s.set_field(ek.FIELD_BODY_FORCE, np.array(g, dtype=np.float64))
    if perturb:
        fluid = o.owner == O.FLUID
        noise = workloads.perturbation(o.f.size, perturb, seed).reshape(o.f.shape)
        f = np.where(fluid[None], o.f * (1.0 + noise), 0.0)
        o.set_populations(f)
        perm = perm_to_oracle(ek)
        flib = np.empty_like(f)
        flib[perm] = f
        s.set_field(ek.FIELD_POPULATIONS, flib.ravel())
        for k in range(o.K):
            nk = workloads.perturbation(o.rho[k].size, 0.2, seed + 1 + k).reshape(o.shape)
            r = o.rho[k] * (1.0 + nk)
            o.set_species(k, r)
            s.set_field(ek.FIELD_SPECIES, r.ravel(), component=k)
    return o, s


def rel_err(a, b, floor=1e-3):
    """max over elements of |a - b| / max(|b|, floor * max|b|) (0 for b == 0 == a)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.max(np.abs(b)) if b.size else 0.0
    if scale == 0.0:
        return float(np.max(np.abs(a))) if a.size else 0.0
    den = np.maximum(np.abs(b), floor * scale)
    return float(np.max(np.abs(a - b) / den))


def compare(ek, o, s, tol=TOL, what=("species", "populations", "velocity", "phi", "owner",
                                       "psi", "particles")):
    """Assert parity of every listed field; returns the error per field."""
    errs = {}
    owner_g = s.get_fields(ek.FIELD_OWNER)
    if "owner" in what:
        assert np.array_equal(owner_g, o.owner.astype(np.float64)), "boundary flags differ"
    fluid = o.owner == O.FLUID
    if "species" in what:
        for k in range(o.K):
            errs[f"rho{k}"] = rel_err(s.get_fields(ek.FIELD_SPECIES, k), o.rho[k])
    if "populations" in what:
        perm = perm_to_oracle(ek)
        fg = s.get_fields(ek.FIELD_POPULATIONS)[perm]
        errs["f"] = rel_err(fg[:, fluid], o.f[:, fluid])
    if "velocity" in what:
        errs["u"] = rel_err(s.get_fields(ek.FIELD_VELOCITY)[:, fluid], o.u[:, fluid], floor=1.0)
    if "phi" in what:
        errs["phi"] = rel_err(s.get_fields(ek.FIELD_PHI), o.phi)
    if "psi" in what:
        errs["psi"] = rel_err(s.get_fields(ek.FIELD_PSI), o.psi)
    if "particles" in what:
        pg = s.get_particles()
        for j, p in enumerate(o.particles):
            q = pg[j]
            errs[f"p{j}.pos"] = float(np.max(np.abs(q["pos"] - p.pos)) / max(1.0, np.max(np.abs(p.pos))))
            # absolute floors far below the magnitudes of the test cases keep
            # quantities that are zero up to rounding from dividing by ~0
            floors = {"vel": 1e-6, "omega": 1e-6 / p.radius, "force": 1e-6, "torque": 1e-6 * p.radius}
            for key, ref in (("vel", p.vel), ("omega", p.omega), ("force", p.force), ("torque", p.torque)):
                sc = max(float(np.max(np.abs(ref))), floors[key])
                errs[f"p{j}.{key}"] = float(np.max(np.abs(q[key] - ref)) / sc)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"parity errors above {tol}: {bad}"
    return errs
