"""ctypes binding of the plain FP64 CPU oracle (oracle/lbm_oracle.c).

TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU
baseline leg of the benchmark.  The product library never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "lbm_oracle.c"
BUILD = HERE / "_build"
LIB = BUILD / "liblbm_oracle.so"

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class OrcParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("bc_x", C.c_int),
        ("M", C.c_int), ("W", _dp), ("thermo", C.c_int), ("cp_R", _dp), ("h_form", _dp),
        ("T0", C.c_double), ("poly7", _dp), ("D", _dp), ("nu", C.c_double), ("Pr", C.c_double),
        ("r_lat", C.c_double), ("visc_model", C.c_int), ("R", C.c_int), ("nu_f", _ip), ("nu_r", _ip), ("log_A", _dp),
        ("b", _dp), ("theta", _dp), ("rtype", _ip), ("eff", _dp), ("low", _dp),
        ("reversible", _ip), ("T_ref", C.c_double), ("P0", C.c_double),
        ("transport", C.c_int), ("mu0", _dp), ("mu_exp", _dp), ("T_tr", C.c_double), ("D_exp", C.c_double),
        ("P_tr", C.c_double),
    ]


def _compile(src: Path, out: Path) -> None:
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           str(src), "-o", str(out), "-lm"]
    subprocess.run(cmd, check=True)


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (-O2, no fast-math, OpenMP over nodes)."""
    BUILD.mkdir(exist_ok=True)
    if LIB.exists() and not force and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    tmp = BUILD / f"liblbm_oracle.{os.getpid()}.so"
    _compile(SRC, tmp)
    os.replace(tmp, LIB)
    return LIB


def _bind(L):
    L.orc_create.restype = C.c_void_p
    L.orc_create.argtypes = [C.POINTER(OrcParams)]
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_init.argtypes = [C.c_void_p, _dp, _dp, _dp, C.c_double]
    L.orc_step.argtypes = [C.c_void_p, C.c_int]
    L.orc_moments.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, _dp]
    L.orc_get_pop.argtypes = [C.c_void_p, _dp]
    L.orc_set_pop.argtypes = [C.c_void_p, _dp]
    L.orc_get_T.argtypes = [C.c_void_p, _dp]
    L.orc_set_T.argtypes = [C.c_void_p, _dp]
    L.orc_thermo.argtypes = [C.c_void_p, C.c_double, _dp, _dp, _dp, _dp]
    L.orc_temperature.argtypes = [C.c_void_p, _dp, C.c_double, C.c_double, _dp]
    L.orc_rates.argtypes = [C.c_void_p, _dp, C.c_double, _dp]
    L.orc_heat_release.restype = C.c_double
    L.orc_heat_release.argtypes = [C.c_void_p, _dp, C.c_double]
    L.orc_total_heat_release.restype = C.c_double
    L.orc_total_heat_release.argtypes = [C.c_void_p, _ip]
    L.orc_diffusion_velocities.argtypes = [C.c_void_p, _dp, _dp, C.c_double, _dp]
    L.orc_equilibrium_sets.argtypes = [C.c_void_p, _dp, _dp, C.c_double, _dp]
    L.orc_transport.argtypes = [C.c_void_p, _dp, C.c_double, C.c_double, _dp]
    L.orc_flame_speeds.argtypes = [C.c_void_p, _dp, _dp]
    L.orc_isoline_means.argtypes = [C.c_void_p, _dp, C.c_double, C.c_double, C.c_double, C.c_int, _dp, _dp]
    L.orc_product_form.argtypes = [C.c_double, _dp, C.c_double, _dp]
    L.orc_grad_pop.argtypes = [C.c_double, _dp, _dp, _dp]
    return L


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(C.CDLL(str(build())))
    return _lib


def load_variant(source_text: str, workdir) -> C.CDLL:
    """Compiles a modified copy of the oracle source (a test plants a
    mistake in it to show that a pin catches it) and returns its bound
    library, for Oracle(..., library=...)."""
    workdir = Path(workdir)
    src = workdir / "lbm_oracle_variant.c"
    out = workdir / "liblbm_oracle_variant.so"
    src.write_text(source_text)
    _compile(src, out)
    return _bind(C.CDLL(str(out)))


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _i(a):
    return a.ctypes.data_as(_ip) if a is not None else None


class Oracle:
    """One oracle instance bound to a workload.Problem (or its parts)."""

    def __init__(self, lattice, species, mech, library=None):
        self.lattice, self.species, self.mech = lattice, species, mech
        self._L = library if library is not None else lib()
        self.M = species.M
        self.S = self.M + 1
        self.N = lattice.nx * lattice.ny * lattice.nz
        keep = {}

        def d(name, a):
            keep[name] = np.ascontiguousarray(a, dtype=np.float64)
            return _d(keep[name])

        def i(name, a):
            keep[name] = np.ascontiguousarray(a, dtype=np.int32)
            return _i(keep[name])

        p = OrcParams(
            nx=lattice.nx, ny=lattice.ny, nz=lattice.nz, bc_x=lattice.bc_x, M=self.M,
            W=d("W", species.W), thermo=species.thermo, cp_R=d("cp_R", species.cp_R),
            h_form=d("h_form", species.h_form), T0=species.T0, poly7=d("poly7", species.poly7),
            D=d("D", species.D), nu=species.nu, Pr=species.Pr, r_lat=species.r_lat,
            visc_model=species.visc_model,
            R=mech.R, nu_f=i("nu_f", mech.nu_f), nu_r=i("nu_r", mech.nu_r),
            log_A=d("log_A", mech.log_A), b=d("b", mech.b), theta=d("theta", mech.theta),
            rtype=i("rtype", mech.rtype), eff=d("eff", mech.eff), low=d("low", mech.low),
            reversible=i("reversible", mech.reversible), T_ref=mech.T_ref, P0=mech.P0,
            transport=species.transport,
            mu0=d("mu0", species.mu0) if species.mu0 is not None else None,
            mu_exp=d("mu_exp", species.mu_exp) if species.mu_exp is not None else None,
            T_tr=species.T_tr, D_exp=species.D_exp, P_tr=species.P_tr)
        self._h = self._L.orc_create(C.byref(p))
        if not self._h:
            raise ValueError("oracle rejected the parameters")

    @classmethod
    def from_problem(cls, prob, init: bool = True, library=None):
        o = cls(prob.lattice, prob.species, prob.mech, library=library)
        if init:
            o.init(prob.init.X, prob.init.T, prob.init.u, prob.init.P)
        return o

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_destroy(h)
            self._h = None

    def init(self, X, T, u, P):
        X = np.ascontiguousarray(X, dtype=np.float64)
        T = np.ascontiguousarray(T, dtype=np.float64)
        u = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
        return self._L.orc_init(self._h, _d(X), _d(T), _d(u), float(P))

    def step(self, n: int = 1) -> int:
        return self._L.orc_step(self._h, int(n))

    def moments(self):
        M, N = self.M, self.N
        out = dict(rho_a=np.empty((M, N)), rhou=np.empty((3, N)), rhoE=np.empty(N),
                   T=np.empty(N), j_a=np.empty((M, 3, N)))
        st = self._L.orc_moments(self._h, _d(out["rho_a"]), _d(out["rhou"]), _d(out["rhoE"]),
                               _d(out["T"]), _d(out["j_a"]))
        out["status"] = st
        rho = out["rho_a"].sum(axis=0)
        out["rho"] = rho
        out["Y"] = out["rho_a"] / rho
        return out

    def get_pop(self):
        a = np.empty((self.N, self.S, 27))
        self._L.orc_get_pop(self._h, _d(a))
        return a

    def set_pop(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        assert a.shape == (self.N, self.S, 27)
        self._L.orc_set_pop(self._h, _d(a))

    def get_T(self):
        a = np.empty(self.N)
        self._L.orc_get_T(self._h, _d(a))
        return a

    def set_T(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        self._L.orc_set_T(self._h, _d(a))

    # point-wise pieces -------------------------------------------------
    def thermo(self, T):
        M = self.M
        U, H, Cv, g = (np.empty(M) for _ in range(4))
        self._L.orc_thermo(self._h, float(T), _d(U), _d(H), _d(Cv), _d(g))
        return dict(U=U, H=H, Cv=Cv, gRT=g)

    def temperature(self, Y, e, T_guess):
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        T = np.zeros(1)
        st = self._L.orc_temperature(self._h, _d(Y), float(e), float(T_guess), _d(T))
        return float(T[0]), st

    def rates(self, rho_a, T):
        rho_a = np.ascontiguousarray(rho_a, dtype=np.float64)
        w = np.empty(self.M)
        self._L.orc_rates(self._h, _d(rho_a), float(T), _d(w))
        return w

    def heat_release(self, rho_a, T):
        """hdot^c = -sum_a H_a rho_dot_a at one node state (Sec. 5b)."""
        rho_a = np.ascontiguousarray(rho_a, dtype=np.float64)
        return float(self._L.orc_heat_release(self._h, _d(rho_a), float(T)))

    def total_heat_release(self):
        """Sum over the lattice of hdot^c at the current time level (Sec. 5b)."""
        st = C.c_int(0)
        J = float(self._L.orc_total_heat_release(self._h, C.byref(st)))
        assert st.value == 0, st.value
        return J

    def flame_speeds(self):
        """S_d (Eq. (sd)) and S_a = S_d + u.n at every node of the current time level."""
        Sd, Sa = np.empty(self.N), np.empty(self.N)
        st = self._L.orc_flame_speeds(self._h, _d(Sd), _d(Sa))
        assert st == 0, st
        return Sd, Sa

    def isoline_means(self, T, T_iso, cx, cy, fields=()):
        """{A, R, means of fields} along T = T_iso in the plane z = 0 (Eq. (rmean))."""
        T = np.ascontiguousarray(T, dtype=np.float64)
        K = len(fields)
        assert K <= 16
        F = np.ascontiguousarray(np.stack(fields) if K else np.zeros((1, self.N)), dtype=np.float64)
        out = np.zeros(2 + K)
        self._L.orc_isoline_means(self._h, _d(T), float(T_iso), float(cx), float(cy), K, _d(F), _d(out))
        return out

    def transport(self, Y, T, P):
        """dict nup (1/omega - 1/2), nup1 (1/omega_1 - 1/2), mu, lam, dfac at a node state."""
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        out = np.zeros(5)
        self._L.orc_transport(self._h, _d(Y), float(T), float(P), _d(out))
        return dict(zip(("nup", "nup1", "mu", "lam", "dfac"), out.tolist()))

    def diffusion_velocities(self, Y, ua_minus_u, T):
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        r = np.ascontiguousarray(ua_minus_u, dtype=np.float64).reshape(self.M, 3)
        du = np.empty((self.M, 3))
        st = self._L.orc_diffusion_velocities(self._h, _d(Y), _d(r), float(T), _d(du))
        return du, st

    def equilibrium_sets(self, rho_a, u, T):
        rho_a = np.ascontiguousarray(rho_a, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.empty((self.S, 27))
        self._L.orc_equilibrium_sets(self._h, _d(rho_a), _d(u), float(T), _d(out))
        return out


def product_form(rho, v, zeta):
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.empty(27)
    lib().orc_product_form(float(rho), _d(v), float(zeta), _d(out))
    return out


def grad_pop(rhoE, q, R):
    q = np.ascontiguousarray(q, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(9)
    out = np.empty(27)
    lib().orc_grad_pop(float(rhoE), _d(q), _d(R), _d(out))
    return out


# Direction convention of the oracle: i = (cx+1) + 3 (cy+1) + 9 (cz+1).
C_VEL = np.array([[i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1] for i in range(27)])
