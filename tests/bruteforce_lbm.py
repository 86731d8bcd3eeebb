"""Brute-force restatement of one reactive-mixture lattice Boltzmann step in
multi-precision arithmetic (mpmath), for tiny periodic lattices.

Written independently of the oracle, straight from the paper: populations
live in dictionaries keyed by lattice node and discrete velocity, every sum
is an explicit loop, the Stefan-Maxwell system is solved with mpmath's LU
routine, the temperature of constant heat capacities is taken in closed
form, and exponentials come from mpmath.  It supports constant-cp
thermodynamics, a constant kinematic viscosity and irreversible mass-action
reactions (the configuration of the three-gas workload).

Equation references are to arXiv 2101.01702.
"""
from __future__ import annotations

import mpmath as mp

VELS = [(cx, cy, cz) for cx in (-1, 0, 1) for cy in (-1, 0, 1) for cz in (-1, 0, 1)]
THETA = mp.mpf(1) / 3


def _w1(c):
    return 1 - THETA if c == 0 else THETA / 2


def weight(c):
    return _w1(c[0]) * _w1(c[1]) * _w1(c[2])


def psi(c, xi, zeta):                                   # Eq. (phis)
    s = xi * xi + zeta
    if c == 0:
        return 1 - s
    return (c * xi + s) / 2


def prod_form(rho, v, zeta):                            # Eqs. (feq), (fstar), (feqmix)
    return {c: rho * psi(c[0], v[0], zeta) * psi(c[1], v[1], zeta) * psi(c[2], v[2], zeta)
            for c in VELS}


def grad_form(rhoE, q, R):                              # Eqs. (gieq), (giqeq)
    out = {}
    for c in VELS:
        first = sum(q[a] * c[a] for a in range(3)) / THETA
        second = mp.mpf(0)
        for a in range(3):
            for b in range(3):
                d = 1 if a == b else 0
                second += (R[a][b] - rhoE * THETA * d) * (c[a] * c[b] - THETA * d)
        out[c] = weight(c) * (rhoE + first + second / (2 * THETA * THETA))
    return out


class BruteForce:
    """params: dict with W, cp_R, h_form, T0, D (MxM), nu, Pr, r_lat and the
    irreversible reactions as lists of (log_A, b, theta, nu_f, nu_r, T_ref)."""

    def __init__(self, shape, params, dps=30, bc_x=0):
        mp.mp.dps = dps
        self.nx, self.ny, self.nz = shape
        self.bc_x = bc_x
        P = params
        self.M = len(P["W"])
        self.W = [mp.mpf(float(x)) for x in P["W"]]
        self.r = mp.mpf(float(P["r_lat"]))
        self.Ra = [self.r / x for x in self.W]
        self.T0 = mp.mpf(float(P["T0"]))
        self.cv = [(mp.mpf(float(P["cp_R"][a])) - 1) * self.Ra[a] for a in range(self.M)]
        # U_a = U0_a + cv_a (T - T0), U0_a = H0_a - R_a T0          Eq. (specHa)
        self.U0 = [mp.mpf(float(P["h_form"][a])) - self.Ra[a] * self.T0 for a in range(self.M)]
        self.D = [[mp.mpf(float(P["D"][a][b])) for b in range(self.M)] for a in range(self.M)]
        self.nu = mp.mpf(float(P["nu"]))
        self.Pr = mp.mpf(float(P["Pr"]))
        self.reactions = P["reactions"]

    def nodes(self):
        return [(x, y, z) for z in range(self.nz) for y in range(self.ny) for x in range(self.nx)]

    def U(self, a, T):
        return self.U0[a] + self.cv[a] * (T - self.T0)

    def H(self, a, T):
        return self.U(a, T) + self.Ra[a] * T

    def rates(self, rho_a, T):
        conc = [rho_a[a] / self.W[a] for a in range(self.M)]
        wdot = [mp.mpf(0)] * self.M
        for (logA, b, theta, nu_f, nu_r, T_ref) in self.reactions:
            k = mp.exp(mp.mpf(logA) + mp.mpf(b) * mp.log(T / mp.mpf(T_ref)) - mp.mpf(theta) / T)
            q = k
            for a in range(self.M):
                for _ in range(int(nu_f[a])):
                    q *= conc[a]
            for a in range(self.M):
                wdot[a] += self.W[a] * (int(nu_r[a]) - int(nu_f[a])) * q
        return wdot

    def equilibria(self, rho_a, u, T):
        """Every set at equilibrium for species densities, velocity and T."""
        M = self.M
        rho = sum(rho_a)
        Y = [ra / rho for ra in rho_a]
        Rm = self.r * sum(Y[a] / self.W[a] for a in range(M))
        usq = sum(x * x for x in u)
        sets = [prod_form(rho_a[a], u, self.Ra[a] * T) for a in range(M - 1)]
        sets.append(prod_form(rho, u, Rm * T))
        H = sum(Y[a] * self.H(a, T) for a in range(M))
        Um = sum(Y[a] * self.U(a, T) for a in range(M))
        P = rho * Rm * T
        qeq = [(H + usq / 2) * rho * u[k] for k in range(3)]
        Req = [[(H + usq / 2) * ((P if a == b else 0) + rho * u[a] * u[b]) + P * u[a] * u[b]
                for b in range(3)] for a in range(3)]
        sets.append(grad_form(rho * (Um + usq / 2), qeq, Req))
        return sets

    def ghost(self, post, xb, y, z, zero_velocity):
        """Sec. 5a: equilibrium populations at the moments of the adjacent
        boundary node (post-collision), zero velocity on the left end."""
        M = self.M
        sets = post[(xb, y, z)]
        rho = sum(sets[M - 1].values())
        rho_a = [sum(sets[a].values()) for a in range(M - 1)]
        rho_a.append(rho - sum(rho_a))
        u = [sum(sets[M - 1][c] * c[k] for c in VELS) / rho for k in range(3)]
        rhoE = sum(sets[M].values())
        Y = [ra / rho for ra in rho_a]
        e = rhoE / rho - sum(x * x for x in u) / 2
        T = self.T0 + (e - sum(Y[a] * self.U0[a] for a in range(M))) / sum(Y[a] * self.cv[a] for a in range(M))
        if zero_velocity:
            u = [mp.mpf(0)] * 3
        return self.equilibria(rho_a, u, T)

    def step(self, post):
        """post[node] = list of S dicts (species 0..M-2, f, g) -> new post."""
        M = self.M
        nxyz = (self.nx, self.ny, self.nz)
        ghosts = {}
        if self.bc_x == 1:
            for z in range(self.nz):
                for y in range(self.ny):
                    ghosts[(-1, y, z)] = self.ghost(post, 0, y, z, True)
                    ghosts[(self.nx, y, z)] = self.ghost(post, self.nx - 1, y, z, False)
        pre = {}
        for n in self.nodes():
            sets = []
            for s in range(M + 1):
                d = {}
                for c in VELS:
                    xs = n[0] - c[0]
                    ys, zs = (n[1] - c[1]) % nxyz[1], (n[2] - c[2]) % nxyz[2]
                    if 0 <= xs < self.nx:
                        d[c] = post[(xs, ys, zs)][s][c]
                    elif self.bc_x == 0:
                        d[c] = post[(xs % self.nx, ys, zs)][s][c]
                    else:
                        d[c] = ghosts[(xs, ys, zs)][s][c]
                sets.append(d)
            pre[n] = sets
        fld = {}
        for n in self.nodes():
            sets = pre[n]
            f, g = sets[M - 1], sets[M]
            fs = [sets[a] for a in range(M - 1)]
            fs.append({c: f[c] - sum(sets[a][c] for a in range(M - 1)) for c in VELS})   # Eq. (strongest)
            rho_a = [sum(fa.values()) for fa in fs]
            j_a = [[sum(fa[c] * c[k] for c in VELS) for k in range(3)] for fa in fs]
            rho = sum(f.values())
            j = [sum(f[c] * c[k] for c in VELS) for k in range(3)]
            Pt = [[sum(f[c] * c[a] * c[b] for c in VELS) for b in range(3)] for a in range(3)]
            rhoE = sum(g.values())
            q = [sum(g[c] * c[k] for c in VELS) for k in range(3)]
            u = [jk / rho for jk in j]
            usq = sum(x * x for x in u)
            Y = [ra / rho for ra in rho_a]
            inv_m = sum(Y[a] / self.W[a] for a in range(M))
            Rm = self.r * inv_m
            e = rhoE / rho - usq / 2
            T = self.T0 + (e - sum(Y[a] * self.U0[a] for a in range(M))) / sum(Y[a] * self.cv[a] for a in range(M))
            Phi = [rho * u[k] * (1 - 3 * Rm * T) - rho * u[k] ** 3 for k in range(3)]
            fld[n] = dict(fs=fs, f=f, g=g, rho_a=rho_a, j_a=j_a, rho=rho, j=j, Pt=Pt, rhoE=rhoE, q=q,
                          u=u, usq=usq, Y=Y, inv_m=inv_m, Rm=Rm, T=T, Phi=Phi, nup=self.nu / (Rm * T))

        def nb(n, c):
            x = n[0] + c[0]
            if self.bc_x == 1:
                x = min(max(x, 0), self.nx - 1)        # zero-gradient continuation
            return (x % self.nx, (n[1] + c[1]) % nxyz[1], (n[2] + c[2]) % nxyz[2])

        def lattice_grad(n, getter, comp):
            return sum(weight(c) * c[comp] * getter(nb(n, c)) for c in VELS) / THETA

        G = {}
        gY = {}
        for n in self.nodes():
            G[n] = [fld[n]["nup"] * lattice_grad(n, lambda m_, k=k: fld[m_]["Phi"][k], k) for k in range(3)]
            gY[n] = [[lattice_grad(n, lambda m_, a=a: fld[m_]["Y"][a], k) for k in range(3)] for a in range(M)]
        new = {}
        for n in self.nodes():
            F_ = fld[n]
            Xc = [-lattice_grad(n, lambda m_, k=k: G[m_][k], k) for k in range(3)]     # Eq. (Xalpha)
            rho, T, u, Y, Rm = F_["rho"], F_["T"], F_["u"], F_["Y"], F_["Rm"]
            m = 1 / F_["inv_m"]
            P = rho * Rm * T
            omega = 1 / (mp.mpf(1) / 2 + F_["nup"])
            omega1 = 1 / (mp.mpf(1) / 2 + F_["nup"] / self.Pr)
            itab = [[(m * self.r * T / (self.W[a] * self.W[b] * self.D[a][b]) if a != b else mp.mpf(0))
                     for b in range(M)] for a in range(M)]                              # Eq. (tauab)
            ita = [sum(Y[b] * itab[a][b] for b in range(M) if b != a) for a in range(M)]
            beta = [1 / (2 / ita[a] + 1) for a in range(M)]                              # Eq. (fStar)
            A = mp.matrix(M, M)
            for a in range(M):
                for b in range(M):
                    A[a, b] = 1 + ita[a] / 2 if a == b else -itab[a][b] * Y[b] / 2      # Eq. (transform1)
            du = [[mp.mpf(0)] * 3 for _ in range(M)]
            for k in range(3):
                rhs = mp.matrix([F_["j_a"][a][k] / F_["rho_a"][a] - u[k] for a in range(M)])
                sol = mp.lu_solve(A, rhs)
                for a in range(M):
                    du[a][k] = sol[a]
            wdot = self.rates(F_["rho_a"], T)
            out = []
            eq = [prod_form(F_["rho_a"][b], u, self.Ra[b] * T) for b in range(M)]
            st = [prod_form(F_["rho_a"][b], [u[k] + du[b][k] for k in range(3)], self.Ra[b] * T) for b in range(M)]
            for a in range(M - 1):
                src = prod_form(wdot[a], u, self.Ra[a] * T)                              # Eq. (fsource)
                d = {}
                for c in VELS:
                    Fai = Y[a] * sum(itab[a][b] * (eq[b][c] - st[b][c]) for b in range(M) if b != a)
                    fa = F_["fs"][a][c]
                    d[c] = fa + 2 * beta[a] * (eq[a][c] - fa) + (beta[a] - 1) * Fai + src[c]
                out.append(d)
            feq = prod_form(rho, u, Rm * T)
            d = {}
            for c in VELS:
                AX = sum(c[k] * Xc[k] for k in range(3)) / 2 if sum(x * x for x in c) == 1 else 0
                d[c] = F_["f"][c] + omega * (feq[c] - F_["f"][c]) + AX                       # Eq. (f)
            out.append(d)
            Hs = [self.H(a, T) for a in range(M)]
            H = sum(Y[a] * Hs[a] for a in range(M))
            usq = F_["usq"]
            Peq = [[(P if a == b else 0) + rho * u[a] * u[b] for b in range(3)] for a in range(3)]
            Req = [[(H + usq / 2) * Peq[a][b] + P * u[a] * u[b] for b in range(3)] for a in range(3)]
            qeq = [(H + usq / 2) * rho * u[k] for k in range(3)]
            qst = []
            for b in range(3):
                uP = sum(u[a] * (F_["Pt"][a][b] - Peq[a][b]) for a in range(3))
                qdiff = omega1 / (omega - omega1) * rho * sum(Hs[a] * Y[a] * du[a][b] for a in range(M))
                qcorr = (omega1 - 2) / (omega1 - omega) / 2 * P * sum(Hs[a] * gY[n][a][b] for a in range(M))
                qst.append(F_["q"][b] - uP + qdiff + qcorr)
            geq = grad_form(F_["rhoE"], qeq, Req)
            gst = grad_form(F_["rhoE"], qst, Req)
            out.append({c: F_["g"][c] + omega1 * (geq[c] - F_["g"][c]) + (omega - omega1) * (gst[c] - F_["g"][c])
                        for c in VELS})
            new[n] = out
        return new
