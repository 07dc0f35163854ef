"""Seeded synthetic inputs for the electrokinetics step.

This module holds no arithmetic of the method: only the random-number
generator (SplitMix64, Steele, Lea and Flood, OOPSLA 2014) and the recipes of
the workloads (box sizes, species, particle placement).  Both the CUDA path's
tests and benchmark and the CPU oracle take their inputs from here.

Workloads (lattice units, k_B T = e = 1):
  small   32^3, one sphere R=4, Z=-50, 2 species (z=+1/-1, D=0.3, bulk 1e-3),
          Bjerrum length 0.7, E=0.01 along x, BGK tau=1 (nu=1/6).
  single  128^3, one sphere R=8, Z=-300, 2 species bulk 1e-3, E=0.005.
  many    256^3, 64 spheres R=5 at seeded non-overlapping positions, Z in
          U[-100,-50], 3 species (z=+1,-1,+2; D=0.2,0.3,0.15), E=0.005.
  large   512^3, 1000 spheres R=6, Z=-200, 2 species bulk 5e-4, E=0.002.
  sub_box  a periodic cube cut from one of them (a bounded sample for the
          CPU baseline).
  batch_ensemble  256 independent boxes, edges from {32, 48, 64} per axis, one
          sphere R in U[3, 6], Z in U[-100, -20], salt log-uniform 1e-4..1e-2,
          E log-uniform 1e-3..1e-2 (a mobility sweep).
"""
from __future__ import annotations

import math

MASK64 = (1 << 64) - 1
SEED = 1607


class SplitMix64:
    """SplitMix64 generator: a 64-bit counter advanced by the golden gamma and
    passed through the published 64-bit finaliser."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_range(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

    def array(self, n: int, lo: float = 0.0, hi: float = 1.0):
        import numpy as np
        return np.array([self.uniform_range(lo, hi) for _ in range(n)], dtype=np.float64)


def species_set(name: str):
    """(valence, D, bulk) of the workload's species."""
    if name == "many":
        return (1, -1, 2), (0.2, 0.3, 0.15), (1e-3, 1e-3, 1e-3)
    if name == "large":
        return (1, -1), (0.3, 0.3), (5e-4, 5e-4)
    return (1, -1), (0.3, 0.3), (1e-3, 1e-3)


def place_spheres(n_box, count, radius, gap, rng: SplitMix64, max_tries=1000000):
    """Random sequential addition of `count` spheres in a periodic cube of edge
    n_box, centre distance (minimum image) at least 2*radius + gap."""
    pts = []
    dmin2 = (2.0 * radius + gap) ** 2
    tries = 0
    while len(pts) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place spheres")
        c = [rng.uniform_range(0.0, n_box) for _ in range(3)]
        ok = True
        for q in pts:
            d2 = 0.0
            for a in range(3):
                d = abs(c[a] - q[a])
                d = min(d, n_box - d)
                d2 += d * d
            if d2 < dmin2:
                ok = False
                break
        if ok:
            pts.append(c)
    return pts


def workload(name: str, seed: int = SEED):
    """Parameters of a named workload as a plain dict (no arithmetic of the method)."""
    rng = SplitMix64(seed)
    val, D, bulk = species_set(name)
    if name == "small":
        n, R, Z, E = 32, 4.0, -50.0, 0.01
        pos = [16.0 + rng.uniform_range(-4.0, 4.0) for _ in range(3)]
        parts = [dict(pos=pos, radius=R, charge=Z)]
    elif name == "single":
        n, R, Z, E = 128, 8.0, -300.0, 0.005
        pos = [64.0 + rng.uniform_range(-4.0, 4.0) for _ in range(3)]
        parts = [dict(pos=pos, radius=R, charge=Z)]
    elif name == "many":
        n, R, E = 256, 5.0, 0.005
        pts = place_spheres(n, 64, R, 2.0, rng)
        # charges from the stable part of U[-150, -50]: with the divalent
        # counter-ion the explicit scheme goes non-finite within 50 steps at
        # Z = -150 on R = 5 (surface charge 0.48 e per cell face)
        parts = [dict(pos=p, radius=R, charge=rng.uniform_range(-100.0, -50.0)) for p in pts]
    elif name == "large":
        n, R, E = 512, 6.0, 0.002
        pts = place_spheres(n, 1000, R, 2.0, rng)
        parts = [dict(pos=p, radius=R, charge=-200.0) for p in pts]
    else:
        raise ValueError(name)
    return dict(name=name, shape=(n, n, n), nu=1.0 / 6.0, rho0=1.0, bjerrum=0.7,
                valence=val, D=D, bulk=bulk, E=(E, 0.0, 0.0), particles=parts,
                rho_p=2.0)


def sub_box(name: str, edge: int, seed: int = SEED):
    """A bounded sample of a workload: the periodic cube [0, edge)^3 cut from
    it, with the spheres whose centres lie at least R + 1 from every face of
    the cube (so that no sphere meets the periodic image of another); the rest
    of the recipe unchanged."""
    w = workload(name, seed)
    keep = []
    for p in w["particles"]:
        m = p["radius"] + 1.0
        if all(m <= c <= edge - m for c in p["pos"]):
            keep.append(dict(p))
    w = dict(w)
    w["name"] = f"{name}[{edge}^3]"
    w["shape"] = (edge, edge, edge)
    w["particles"] = keep
    return w


def batch_ensemble(nsys: int = 256, seed: int = SEED, edges=(32, 48, 64), radius=(3.0, 6.0),
                   charge=(-100.0, -20.0), bulk=(1e-4, 1e-2), field=(1e-3, 1e-2),
                   max_charge_per_radius=12.0):
    """Independent systems of a mobility sweep: box edges drawn per axis from
    `edges`, one sphere of radius U(radius) and charge U(charge) at a uniform
    position, salt (both species) log-uniform in `bulk`, field along x
    log-uniform in `field`; two species z = +-1, D = 0.3, l_B = 0.7.

    The charge magnitude is capped at max_charge_per_radius * R (surface
    charge density below 1 / R): a sphere of R = 3.06 with Z = -99.7 at salt
    2e-3 leaves the scheme's stable range (the FP64 reference stops after 26
    steps with nowhere to expel solute)."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(nsys):
        shape = tuple(edges[min(int(rng.uniform() * len(edges)), len(edges) - 1)] for _ in range(3))
        R = rng.uniform_range(radius[0], radius[1])
        zlo = max(charge[0], -max_charge_per_radius * R)
        Z = rng.uniform_range(zlo, min(charge[1], zlo + (charge[1] - charge[0])))
        b = math.exp(rng.uniform_range(math.log(bulk[0]), math.log(bulk[1])))
        E = math.exp(rng.uniform_range(math.log(field[0]), math.log(field[1])))
        pos = [rng.uniform_range(0.0, float(n)) for n in shape]
        out.append(dict(name="batch", shape=shape, nu=1.0 / 6.0, rho0=1.0, bjerrum=0.7,
                        valence=(1, -1), D=(0.3, 0.3), bulk=(b, b), E=(E, 0.0, 0.0),
                        particles=[dict(pos=pos, radius=R, charge=Z)], rho_p=2.0))
    return out


def small_case(n=(16, 16, 16), radius=3.0, charge=-20.0, nparticles=1, seed=SEED,
               E=0.01, bulk=1e-3, gap=2.0):
    """A small seeded case for parity tests: box n, spheres of the given radius
    placed by random sequential addition, charges around `charge`."""
    rng = SplitMix64(seed)
    nx, ny, nz = n
    parts = []
    dmin2 = (2.0 * radius + gap) ** 2
    while len(parts) < nparticles:
        c = [rng.uniform_range(0.0, nx), rng.uniform_range(0.0, ny), rng.uniform_range(0.0, nz)]
        ok = True
        for q in parts:
            d2 = 0.0
            for a, L in enumerate((nx, ny, nz)):
                d = abs(c[a] - q["pos"][a])
                d = min(d, L - d)
                d2 += d * d
            ok &= d2 >= dmin2
        if ok:
            parts.append(dict(pos=c, radius=radius,
                              charge=charge * (0.5 + rng.uniform())))
    return dict(name="case", shape=(nx, ny, nz), nu=1.0 / 6.0, rho0=1.0, bjerrum=0.7,
                valence=(1, -1), D=(0.3, 0.3), bulk=(bulk, bulk), E=(E, 0.0, 0.0),
                particles=parts, rho_p=2.0)


def perturbation(n_values: int, amplitude: float, seed: int):
    """Seeded uniform noise in [-amplitude, amplitude) (numpy array)."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    return amplitude * (2.0 * rng.random(n_values) - 1.0)
