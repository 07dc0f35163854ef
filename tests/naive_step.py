"""A second restatement of the whole time step, written node by node with
plain loops and Python floats, for the brute-force pin of the oracle.  It
shares nothing with oracle/ but the state it is handed: its own velocity set,
equilibrium, Fourier matrices, partial volumes (from the level-4 cubes), flux,
collision, bounce-back, advection, partition, integration and transitions,
each following the paper's equations under the same readings.  Small boxes
only (about a thousand nodes)."""
import math

import numpy as np

# D3Q19: rest, faces, edges; weights 1/3, 1/18, 1/36
C = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
     (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1),
     (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
W = [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12
OPPOSITE = [C.index((-c[0], -c[1], -c[2])) for c in C]
A0 = 1 + 2 * math.sqrt(2)
FLUID = -1


class State:
    """nx, ny, nz; f[19][z][y][x]; rho[K][z][y][x]; particles as dicts."""

    def __init__(self, o, order):
        """Copy the oracle's state; `order` maps our directions to its rows."""
        self.nx, self.ny, self.nz = (int(v) for v in o.n)
        self.f = np.array([o.f[order[i]] for i in range(19)])
        self.rho = o.rho.copy()
        self.owner = o.owner.copy()
        self.val = [float(v) for v in o.valence]
        self.D = [float(v) for v in o.D]
        self.rho0, self.lB, self.nu, self.magic = o.rho0, o.bjerrum, o.nu, o.magic
        self.E = [float(v) for v in o.E]
        self.g = [float(v) for v in o.g]
        self.pv = bool(o.flags & 1)
        self.vacate_zero = bool(o.flags & 2)
        self.norm_vp = bool(o.flags & 4)
        self.parts = [dict(pos=list(p.pos), vel=list(p.vel), om=list(p.omega), R=p.radius,
                           Z=p.charge, m=p.mass, I=0.4 * p.mass * p.radius ** 2,
                           fixed=p.fixed, ftr=list(p.f_trans)) for p in o.particles]
        self.psi_p = [self.psi_box(p) for p in self.parts]

    # ---- geometry -------------------------------------------------------------
    def mi(self, d, n):
        if d > 0.5 * n:
            return d - n
        if d < -0.5 * n:
            return d + n
        return d

    def offset(self, p, x, y, z):
        return (self.mi(x - p["pos"][0], self.nx), self.mi(y - p["pos"][1], self.ny),
                self.mi(z - p["pos"][2], self.nz))

    def box(self, p, widen=0):
        lo = [math.floor(p["pos"][a] - p["R"]) - 1 - widen for a in range(3)]
        hi = [math.floor(p["pos"][a] + p["R"]) + 2 + widen for a in range(3)]
        return lo, hi

    def cells(self, lo, hi):
        seen = set()
        for Z in range(lo[2], hi[2]):
            for Y in range(lo[1], hi[1]):
                for X in range(lo[0], hi[0]):
                    w = (X % self.nx, Y % self.ny, Z % self.nz)
                    if w not in seen:
                        seen.add(w)
                        yield X, Y, Z, w

    def psi_cell(self, X, Y, Z, p):
        """Psi of cell (X, Y, Z) (unwrapped box coordinates): the level-4 cubes
        one by one, all corners strictly inside 1, closest point at >= R 0,
        otherwise 1/2; squares summed x, y, z."""
        R2 = p["R"] * p["R"]
        pl = [[c + k / 16.0 - 0.5 - p["pos"][a] for k in range(17)] for a, c in enumerate((X, Y, Z))]
        far = [[max(abs(pl[a][k]), abs(pl[a][k + 1])) for k in range(16)] for a in range(3)]
        near = [[0.0 if pl[a][k] <= 0.0 <= pl[a][k + 1] else min(abs(pl[a][k]), abs(pl[a][k + 1]))
                 for k in range(16)] for a in range(3)]
        fx, fy, fz = (np.array(v) for v in far)
        ex, ey, ez = (np.array(v) for v in near)
        # cube (i, j, k): x from i, y from j, z from k, squares summed x, y, z
        dfar = (fx[:, None, None] * fx[:, None, None] + fy[None, :, None] * fy[None, :, None]) + \
            fz[None, None, :] * fz[None, None, :]
        dnear = (ex[:, None, None] * ex[:, None, None] + ey[None, :, None] * ey[None, :, None]) + \
            ez[None, None, :] * ez[None, None, :]
        ins = dfar < R2
        units = 2 * int(ins.sum()) + int(((dnear < R2) & ~ins).sum())
        return units / 8192.0

    def psi_box(self, p):
        lo, hi = self.box(p)
        return {w: self.psi_cell(X, Y, Z, p) for X, Y, Z, w in self.cells(lo, hi)}

    def inside(self, p, x, y, z):
        dx, dy, dz = (X - p["pos"][a] for a, X in enumerate((x, y, z)))
        return dx * dx + dy * dy + dz * dz < p["R"] * p["R"]

    # ---- fields ----------------------------------------------------------------
    def psi_field(self):
        psi = np.zeros((self.nz, self.ny, self.nx))
        for pp in self.psi_p:
            for (x, y, z), v in pp.items():
                psi[z, y, x] += v
        return np.minimum(psi, 1.0)

    def particle_charge(self, pid):
        p, pp = self.parts[pid], self.psi_p[pid]
        if self.pv:
            norm = 4.0 / 3.0 * math.pi * p["R"] ** 3 if self.norm_vp else sum(pp.values())
            return {w: p["Z"] * v / norm for w, v in pp.items() if v}
        own = [w for w in pp if self.owner[w[2], w[1], w[0]] == pid]
        return {w: p["Z"] / len(own) for w in own}

    def poisson(self, q):
        """lap Phi = -4 pi l_B (q - mean q), by explicit Fourier matrices."""
        def dft(n):
            k = np.arange(n)
            return np.exp(-2j * math.pi * np.outer(k, k) / n)
        Fx, Fy, Fz = dft(self.nx), dft(self.ny), dft(self.nz)
        qh = np.einsum("az,by,cx,zyx->abc", Fz, Fy, Fx, q)
        lam = np.zeros(qh.shape)
        for a in range(self.nz):
            for b in range(self.ny):
                for c in range(self.nx):
                    lam[a, b, c] = (2 - 2 * math.cos(2 * math.pi * a / self.nz)) + \
                        (2 - 2 * math.cos(2 * math.pi * b / self.ny)) + \
                        (2 - 2 * math.cos(2 * math.pi * c / self.nx))
        ph = np.where(lam > 0, 4 * math.pi * self.lB * qh / np.where(lam > 0, lam, 1), 0)
        n = self.nx * self.ny * self.nz
        return np.einsum("az,by,cx,abc->zyx", Fz.conj(), Fy.conj(), Fx.conj(), ph).real / n

    def feq(self, rho, u):
        uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
        out = []
        for i in range(19):
            cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2]
            out.append(W[i] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu))
        return out

    def wall_velocity(self, pid, x, y, z):
        p = self.parts[pid]
        d = self.offset(p, x, y, z)
        w = p["om"]
        return [p["vel"][0] + w[1] * d[2] - w[2] * d[1], p["vel"][1] + w[2] * d[0] - w[0] * d[2],
                p["vel"][2] + w[0] * d[1] - w[1] * d[0]]

    # ---- one step -----------------------------------------------------------------
    def step(self):
        nx, ny, nz, K = self.nx, self.ny, self.nz, len(self.val)
        nodes = [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx)]
        isf = lambda x, y, z: self.owner[z % nz, y % ny, x % nx] == FLUID  # noqa: E731
        psi = self.psi_field()
        P = len(self.parts)
        # S1: charge and Poisson
        q = np.tensordot(np.array(self.val), self.rho, axes=(0, 0)) if K else np.zeros((nz, ny, nx))
        for pid in range(P):
            for (x, y, z), v in self.particle_charge(pid).items():
                q[z, y, x] += v
        phi = self.poisson(q)
        # S2a: link fluxes and coupling force
        J = {}
        fext = {n: [0.0, 0.0, 0.0] for n in nodes}
        for (x, y, z) in nodes:
            if not isf(x, y, z):
                continue
            for i in range(1, 19):
                cx, cy, cz = C[i]
                X, Y, Z = (x + cx) % nx, (y + cy) % ny, (z + cz) % nz
                if not isf(X, Y, Z):
                    continue
                pa = psi[z, y, x] if self.pv else 0.0
                pb = psi[Z, Y, X] if self.pv else 0.0
                dphi = phi[z, y, x] - phi[Z, Y, X] + self.E[0] * cx + self.E[1] * cy + self.E[2] * cz
                for k in range(K):
                    a = self.rho[k, z, y, x] / (1 - pa)
                    b = self.rho[k, Z, Y, X] / (1 - pb)
                    j = self.D[k] / (A0 * math.sqrt(cx * cx + cy * cy + cz * cz)) * \
                        ((a - b) + self.val[k] * (a + b) / 2 * dphi) * (1 - pa) * (1 - pb)
                    J[(k, i, x, y, z)] = j
                    for ax, c in enumerate((cx, cy, cz)):
                        fext[(x, y, z)][ax] += 0.5 * j * c / self.D[k]
        # S4 (part): the solute's force on the particles
        Fs = [[0.0] * 3 for _ in range(P)]
        Ts = [[0.0] * 3 for _ in range(P)]
        if P:
            cand = {}
            for pid, p in enumerate(self.parts):
                lo, hi = self.box(p, widen=math.ceil(p["R"]) + 4)
                for X, Y, Z, w in self.cells(lo, hi):
                    cand.setdefault(w, []).append(pid)
            inner = {}
            for (x, y, z) in nodes:
                if not isf(x, y, z):
                    continue
                qi = sum(self.val[k] * self.rho[k, z, y, x] for k in range(K))
                inner[(x, y, z)] = [fext[(x, y, z)][a] - qi * self.E[a] for a in range(3)]
            assigned = [0.0, 0.0, 0.0]
            for w, ps in cand.items():
                if w not in inner:
                    continue
                best = None
                for pid in sorted(ps):
                    d = self.offset(self.parts[pid], *w)
                    s = math.sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - self.parts[pid]["R"]
                    if best is None or s < best[0]:
                        best = (s, pid, d)
                _, pid, d = best
                iv = inner[w]
                for a in range(3):
                    Fs[pid][a] -= iv[a]
                    assigned[a] += iv[a]
                Ts[pid][0] -= d[1] * iv[2] - d[2] * iv[1]
                Ts[pid][1] -= d[2] * iv[0] - d[0] * iv[2]
                Ts[pid][2] -= d[0] * iv[1] - d[1] * iv[0]
            total = [sum(v[a] for v in inner.values()) for a in range(3)]
            for pid, p in enumerate(self.parts):
                qp = self.particle_charge(pid)
                Q = sum(qp.values())
                for a in range(3):
                    Fs[pid][a] += Q * self.E[a] - (total[a] - assigned[a]) / P
                for w, v in qp.items():
                    d = self.offset(p, *w)
                    Ts[pid][0] += v * (d[1] * self.E[2] - d[2] * self.E[1])
                    Ts[pid][1] += v * (d[2] * self.E[0] - d[0] * self.E[2])
                    Ts[pid][2] += v * (d[0] * self.E[1] - d[1] * self.E[0])
        # S2b: collision (TRT with the force term) and push streaming with bounce-back
        tau_e = 3 * self.nu + 0.5
        le = -1 / tau_e
        lo_ = le if self.magic is None else -1 / (0.5 + self.magic / (tau_e - 0.5))
        fstar = {}
        u_field = np.zeros((3, nz, ny, nx))
        for (x, y, z) in nodes:
            if not isf(x, y, z):
                continue
            fl = [self.f[i, z, y, x] for i in range(19)]
            F = [fext[(x, y, z)][a] + self.g[a] for a in range(3)]
            rho = sum(fl)
            j = [sum(fl[i] * C[i][a] for i in range(19)) for a in range(3)]
            u = [(j[a] + F[a] / 2) / rho for a in range(3)]
            u_field[:, z, y, x] = u
            uu = sum(v * v for v in u)
            uF = sum(u[a] * F[a] for a in range(3))
            gg = 1 + le / 2
            out = []
            for i in range(19):
                ib = OPPOSITE[i]
                cu = sum(C[i][a] * u[a] for a in range(3))
                cj = sum(C[i][a] * j[a] for a in range(3))
                cF = sum(C[i][a] * F[a] for a in range(3))
                eq_e = W[i] * rho * (1 + 4.5 * cu * cu - 1.5 * uu)
                eq_o = W[i] * 3 * cj
                delta = W[i] * (3 * cF + 4.5 * 2 * gg * cu * cF - 1.5 * 2 * gg * uF)
                out.append(fl[i] + le * ((fl[i] + fl[ib]) / 2 - eq_e) +
                           lo_ * ((fl[i] - fl[ib]) / 2 - eq_o) + delta)
            fstar[(x, y, z)] = out
        fnew = np.zeros_like(self.f)
        Fh = [[0.0] * 3 for _ in range(P)]
        Th = [[0.0] * 3 for _ in range(P)]
        for (x, y, z), fs in fstar.items():
            fnew[0, z, y, x] += fs[0]
            for i in range(1, 19):
                cx, cy, cz = C[i]
                X, Y, Z = (x + cx) % nx, (y + cy) % ny, (z + cz) % nz
                if isf(X, Y, Z):
                    fnew[i, Z, Y, X] += fs[i]
                    continue
                own = int(self.owner[Z, Y, X])
                vb = self.wall_velocity(own, X, Y, Z) if own >= 0 else [0.0, 0.0, 0.0]
                refl = fs[i] - 6 * W[i] * self.rho0 * (cx * vb[0] + cy * vb[1] + cz * vb[2])
                fnew[OPPOSITE[i], z, y, x] += refl
                if own >= 0:
                    dp = [c * (fs[i] + refl) for c in (cx, cy, cz)]
                    d = self.offset(self.parts[own], X, Y, Z)
                    for a in range(3):
                        Fh[own][a] += dp[a]
                    Th[own][0] += d[1] * dp[2] - d[2] * dp[1]
                    Th[own][1] += d[2] * dp[0] - d[0] * dp[2]
                    Th[own][2] += d[0] * dp[1] - d[1] * dp[0]
        # S3: flux divergence and volume-of-fluid advection
        rho = self.rho.copy()
        for (k, i, x, y, z), j in J.items():
            rho[k, z, y, x] -= j
        for (x, y, z) in nodes:
            if not isf(x, y, z):
                continue
            u = u_field[:, z, y, x]
            for sz in (-1, 0, 1):
                for sy in (-1, 0, 1):
                    for sx in (-1, 0, 1):
                        if (sx, sy, sz) == (0, 0, 0):
                            continue
                        frac = 1.0
                        for s, ua in zip((sx, sy, sz), u):
                            if s == 0:
                                frac *= 1 - abs(ua)
                            elif (ua > 0 and s > 0) or (ua < 0 and s < 0):
                                frac *= abs(ua)
                            else:
                                frac = 0.0
                        X, Y, Z = (x + sx) % nx, (y + sy) % ny, (z + sz) % nz
                        if frac == 0.0 or not isf(X, Y, Z):
                            continue
                        for k in range(K):
                            amt = self.rho[k, z, y, x] * frac
                            rho[k, z, y, x] -= amt
                            rho[k, Z, Y, X] += amt
        self.rho = rho
        self.f = fnew
        # S4: integration
        for pid, p in enumerate(self.parts):
            F = [Fh[pid][a] + Fs[pid][a] + p["ftr"][a] for a in range(3)]
            T = [Th[pid][a] + Ts[pid][a] for a in range(3)]
            p["force"], p["torque"], p["ftr"] = F, T, [0.0, 0.0, 0.0]
            if p["fixed"]:
                continue
            for a, n in enumerate((nx, ny, nz)):
                p["vel"][a] += F[a] / p["m"]
                p["om"][a] += T[a] / p["I"]
                p["pos"][a] += p["vel"][a]
                if p["pos"][a] >= n:
                    p["pos"][a] -= n
                elif p["pos"][a] < 0:
                    p["pos"][a] += n
        # S5: re-flag, Psi, transitions
        old = self.owner.copy()
        new = np.full_like(old, FLUID)
        for pid, p in enumerate(self.parts):
            lo, hi = self.box(p)
            for X, Y, Z, (x, y, z) in self.cells(lo, hi):
                if self.inside(p, X, Y, Z):
                    new[z, y, x] = pid
        self.owner = new
        self.psi_p = [self.psi_box(p) for p in self.parts]
        steady = lambda x, y, z: old[z % nz, y % ny, x % nx] == FLUID and new[z % nz, y % ny, x % nx] == FLUID  # noqa: E731
        f_old, rho_old = self.f.copy(), self.rho.copy()
        drho = np.zeros_like(self.rho)
        for (x, y, z) in nodes:
            o_, n_ = old[z, y, x], new[z, y, x]
            nb = [((x + c[0]) % nx, (y + c[1]) % ny, (z + c[2]) % nz) for c in C[1:]
                  if steady(x + c[0], y + c[1], z + c[2])]
            if o_ == FLUID and n_ >= 0:      # covered: momentum to the particle, solute out
                mom = [sum(C[i][a] * f_old[i, z, y, x] for i in range(19)) for a in range(3)]
                for a in range(3):
                    self.parts[n_]["ftr"][a] += mom[a]
                for k in range(K):
                    drho[k, z, y, x] -= rho_old[k, z, y, x]
                    for (X, Y, Z) in nb:
                        drho[k, Z, Y, X] += rho_old[k, z, y, x] / len(nb)
                self.f[:, z, y, x] = 0.0
            elif o_ >= 0 and n_ == FLUID:    # uncovered: fluid created, solute refilled
                rbar = (sum(f_old[:, Z, Y, X].sum() for (X, Y, Z) in nb) / len(nb)) if nb else self.rho0
                vb = self.wall_velocity(int(o_), x, y, z)
                fe = self.feq(rbar, vb)
                self.f[:, z, y, x] = fe
                for a in range(3):
                    self.parts[int(o_)]["ftr"][a] -= sum(C[i][a] * fe[i] for i in range(19))
                if self.vacate_zero:
                    continue
                for k in range(K):
                    for (X, Y, Z) in nb:
                        share = rho_old[k, Z, Y, X] / (len(nb) + 1)
                        drho[k, z, y, x] += share
                        drho[k, Z, Y, X] -= share
        self.rho = self.rho + drho
