"""ctypes wrapper around the FP64 CPU oracle (``pic_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  The product path never
imports this module, and this module imports nothing from the product
package: the two are independent implementations of the method of
Ngirmang et al., "Particle-In-Cell Simulations of Quantum Plasmas"
(arXiv 2501.07465), Secs. 2-5 and Appendix A.

Units: positions in cell units (X = x / dx), velocities in m/s, displacements
of bound particles in metres, fields in SI units.  Arrays of fields have shape
(nz, ny, nx) (nz = 1 in 2D).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_LIB_OMP = os.path.join(_LIB_DIR, "liboracle_omp.so")

KIND_FREE, KIND_BOUND, KIND_DIRAC = 0, 1, 2
BC_PERIODIC, BC_PML = 0, 1


def build(force: bool = False, parallel: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off so that x86 and Arm
    hosts round identically).  parallel: the OpenMP build (all host cores),
    used only to time the oracle; the checks use the serial build."""
    out = _LIB_OMP if parallel else _LIB
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", *(["-fopenmp"] if parallel else []), _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


_lib = None
_lib_omp = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


def lib_omp():
    """The OpenMP build (timing only)."""
    global _lib_omp
    if _lib_omp is None:
        _lib_omp = C.CDLL(build(parallel=True))
        _declare(_lib_omp)
    return _lib_omp


def threads(parallel: bool = True) -> int:
    """Threads the oracle's step runs on."""
    return (lib_omp() if parallel else lib()).orc_threads()


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_u32p = C.POINTER(C.c_uint32)
_i32p = C.POINTER(C.c_int32)
_u8p = C.POINTER(C.c_uint8)
_i64p = C.POINTER(C.c_longlong)


def _declare(L):
    L.orc_create.restype = C.c_void_p
    L.orc_create.argtypes = [C.c_int, _ip, _dp, C.c_double, _ip, C.c_int, C.c_double, C.c_int,
                             C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                             C.c_double, C.c_double]
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_set_mask.argtypes = [C.c_void_p, _u8p]
    L.orc_set_permittivity.argtypes = [C.c_void_p, _dp]
    L.orc_set_external_field.argtypes = [C.c_void_p, _dp, _dp, _dp]
    L.orc_work_function_field.argtypes = [C.c_void_p, C.c_double, _dp, _dp, _dp]
    L.orc_set_particle_bc.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_uint64]
    L.orc_set_shape_order.argtypes = [C.c_void_p, C.c_int]
    L.orc_set_binding_offdiag.argtypes = [C.c_void_p, C.c_int, _dp]
    L.orc_push_bound_tensor.argtypes = [_dp, _dp, _dp, _dp, C.c_double, C.c_double, C.c_double,
                                        _dp, _dp, _dp]
    L.orc_add_species.restype = C.c_int
    L.orc_add_species.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double, _dp,
                                  _dp, C.c_double, C.c_long, _dp, _dp, _dp, C.c_int]
    L.orc_step.argtypes = [C.c_void_p, C.c_int]
    L.orc_threads.restype = C.c_int
    L.orc_threads.argtypes = []
    L.orc_get_field.argtypes = [C.c_void_p, C.c_int, _dp]
    L.orc_set_field.argtypes = [C.c_void_p, C.c_int, _dp]
    L.orc_get_J.argtypes = [C.c_void_p, C.c_int, _dp]
    L.orc_clear_J.argtypes = [C.c_void_p]
    L.orc_species_count.restype = C.c_long
    L.orc_species_count.argtypes = [C.c_void_p, C.c_int]
    L.orc_get_species.argtypes = [C.c_void_p, C.c_int, _dp, _dp, _dp, _i64p]
    L.orc_cell_counts.argtypes = [C.c_void_p, C.c_int, _i32p]
    L.orc_energy_histogram.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_int,
                                       C.POINTER(C.c_uint64)]
    L.orc_diag.argtypes = [C.c_void_p, _dp]
    L.orc_rho.argtypes = [C.c_void_p, _dp]
    L.orc_gather.argtypes = [C.c_void_p, _dp, _dp, _dp]
    L.orc_deposit_one.argtypes = [C.c_void_p, _dp, _dp, C.c_double, C.c_double]
    L.orc_push_free.argtypes = [_dp, _dp, _dp, C.c_double, C.c_double, C.c_double]
    L.orc_push_bound.argtypes = [_dp, _dp, _dp, _dp, C.c_double, C.c_double, C.c_double, _dp, _dp]
    L.orc_push_dirac.argtypes = [_dp, _dp, _dp, C.c_double, C.c_double, C.c_double, C.c_double]
    L.orc_fermi_energy.restype = C.c_double
    L.orc_fermi_energy.argtypes = [C.c_double, C.c_double]
    L.orc_dt_limit.restype = C.c_double
    L.orc_dt_limit.argtypes = [C.c_int, _dp, C.c_double, C.c_double]
    L.orc_philox.argtypes = [_u32p, _u32p, _u32p]
    L.orc_particle_uniforms.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64, _dp]
    L.orc_fd_invert.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_long,
                                _dp, _dp]
    L.orc_fd_load.restype = C.c_long
    L.orc_fd_load.argtypes = [C.c_int, _ip, _u8p, C.c_int, C.c_double, C.c_double, C.c_double,
                              C.c_double, C.c_int, C.c_int, C.c_uint64, C.c_uint32, _i32p, _dp,
                              _dp]


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


# --------------------------------------------------------------------------
# single operations (pinned individually by the CPU tests)
# --------------------------------------------------------------------------

def push_free(v, E, B, q, m, dt):
    """Boris push of one free particle (Appendix A.1); returns v_{n+1/2}."""
    v, pv = _d(np.array(v, dtype=np.float64))
    _, pE = _d(E)
    _, pB = _d(B)
    lib().orc_push_free(pv, pE, pB, q, m, dt)
    return v


def push_bound(v, D, E, B, q, m, dt, omega0, gamma):
    """Modified Boris push of one bound particle (Appendix A.2); returns
    (v_{n+1/2}, D_{n+1})."""
    v, pv = _d(np.array(v, dtype=np.float64))
    D, pD = _d(np.array(D, dtype=np.float64))
    _, pE = _d(E)
    _, pB = _d(B)
    _, pw = _d(np.broadcast_to(np.asarray(omega0, dtype=np.float64), (3,)).copy())
    _, pg = _d(np.broadcast_to(np.asarray(gamma, dtype=np.float64), (3,)).copy())
    lib().orc_push_bound(pv, pD, pE, pB, q, m, dt, pw, pg)
    return v, D


def push_bound_tensor(v, D, E, B, q, m, dt, omega0, w2off, gamma):
    """push_bound with the binding tensor diag(omega0^2) + off-diagonal
    w2off = (xy, xz, yz) in s^-2."""
    v, pv = _d(np.array(v, dtype=np.float64))
    D, pD = _d(np.array(D, dtype=np.float64))
    _, pE = _d(E)
    _, pB = _d(B)
    _, pw = _d(np.broadcast_to(np.asarray(omega0, dtype=np.float64), (3,)).copy())
    _, po = _d(np.asarray(w2off, dtype=np.float64).copy())
    _, pg = _d(np.broadcast_to(np.asarray(gamma, dtype=np.float64), (3,)).copy())
    lib().orc_push_bound_tensor(pv, pD, pE, pB, q, m, dt, pw, po, pg)
    return v, D


def push_dirac(v, E, B, q, m, dt, vF):
    """Dirac-carrier push (Sec. 5); returns v_{n+1/2} with |v| = v_F."""
    v, pv = _d(np.array(v, dtype=np.float64))
    _, pE = _d(E)
    _, pB = _d(B)
    lib().orc_push_dirac(pv, pE, pB, q, m, dt, vF)
    return v


def fermi_energy(n, m):
    return lib().orc_fermi_energy(n, m)


def dt_limit(dims, d, omega_b, omega_p):
    _, pd = _d(np.asarray(d, dtype=np.float64))
    return lib().orc_dt_limit(dims, pd, omega_b, omega_p)


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(c.ctypes.data_as(_u32p), k.ctypes.data_as(_u32p), out.ctypes.data_as(_u32p))
    return out


def particle_uniforms(seed, stream, pid):
    u = np.zeros(6)
    lib().orc_particle_uniforms(seed, stream, pid, u.ctypes.data_as(_dp))
    return u


def fd_invert(dirac, m, EF, T, vF, u):
    u, pu = _d(u)
    p = np.zeros(u.size)
    lib().orc_fd_invert(int(dirac), m, EF, T, vF, u.size, pu, p.ctypes.data_as(_dp))
    return p


def fd_load(dims, n, mask, kind, m, EF, T, vF, ppc, quiet, seed, stream):
    """The Fermi-Dirac loader (Sec. 2).  Returns (cell int32, off float64 (N,3),
    v float64 (N,3)) in particle-id order."""
    nn = np.ascontiguousarray(n, dtype=np.int32)
    pn = nn.ctypes.data_as(_ip)
    if mask is not None:
        mask = np.ascontiguousarray(mask, dtype=np.uint8).ravel()
        pm = mask.ctypes.data_as(_u8p)
    else:
        pm = None
    L = lib()
    np_ = L.orc_fd_load(dims, pn, pm, kind, m, EF, T, vF, ppc, int(quiet), seed, stream, None,
                        None, None)
    cell = np.zeros(max(np_, 1), dtype=np.int32)
    off = np.zeros((max(np_, 1), 3))
    v = np.zeros((max(np_, 1), 3))
    r = L.orc_fd_load(dims, pn, pm, kind, m, EF, T, vF, ppc, int(quiet), seed, stream,
                      cell.ctypes.data_as(_i32p), off.ctypes.data_as(_dp), v.ctypes.data_as(_dp))
    if r < 0:
        raise ValueError("quiet loading needs ppc to be a perfect power of dims")
    return cell[:np_], off[:np_], v[:np_]


# --------------------------------------------------------------------------
# the simulation
# --------------------------------------------------------------------------

class OracleSim:
    """One FP64 simulation.

    grid keys: dims, n (3 ints), d (3 floats, metres; d[2] is the slab depth
    in 2D), dt, bc (3 ints, 0 periodic / 1 PML), pml_cells, pml_R0, pml_order,
    and optionally a plane-wave source: src (bool), inc_axis, pol_axis,
    src_index, E0, omega, tau (intensity FWHM), t0.  parallel=True runs the
    step on the OpenMP build (all host cores; only the summation order of J
    differs from the serial build), for timing.
    """

    def __init__(self, parallel=False, **g):
        self._L = lib_omp() if parallel else lib()
        self.dims = int(g["dims"])
        n = list(g["n"]) + [1] * (3 - len(g["n"]))
        if self.dims == 2:
            n[2] = 1
        self.n = tuple(int(x) for x in n)
        self.shape = (self.n[2], self.n[1], self.n[0])
        nn = np.array(self.n, dtype=np.int32)
        d = np.array(g["d"], dtype=np.float64)
        bc = np.array(g.get("bc", [0, 0, 0]), dtype=np.int32)
        self.dt = float(g["dt"])
        self._h = self._L.orc_create(
            self.dims, nn.ctypes.data_as(_ip), d.ctypes.data_as(_dp), self.dt,
            bc.ctypes.data_as(_ip), int(g.get("pml_cells", 0)), float(g.get("pml_R0", 1e-8)),
            int(g.get("pml_order", 3)), int(bool(g.get("src", False))), int(g.get("inc_axis", 0)),
            int(g.get("pol_axis", 1)), int(g.get("src_index", 0)), float(g.get("E0", 0.0)),
            float(g.get("omega", 0.0)), float(g.get("tau", 1.0)), float(g.get("t0", 0.0)))
        self.nsp = 0

    def close(self):
        if self._h:
            self._L.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_mask(self, mask):
        m = np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        assert m.size == np.prod(self.shape)
        self._L.orc_set_mask(self._h, m.ctypes.data_as(_u8p))

    def set_permittivity(self, eps_r):
        """Relative permittivity per cell, [nz][ny][nx] (None: vacuum)."""
        if eps_r is None:
            self._L.orc_set_permittivity(self._h, None)
            return
        e = np.ascontiguousarray(eps_r, dtype=np.float64).reshape(-1)
        assert e.size == np.prod(self.shape)
        self._eps = e
        self._L.orc_set_permittivity(self._h, e.ctypes.data_as(_dp))

    def set_external_field(self, E):
        """External electrostatic field (Ex, Ey, Ez), each [nz][ny][nx] on the
        E stagger, seen by the particles only (None: remove)."""
        if E is None:
            self._L.orc_set_external_field(self._h, None, None, None)
            self._eext = None
            return
        arrs = [np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(self.shape))
                for c in E]
        self._eext = arrs
        self._L.orc_set_external_field(self._h, *[a.ctypes.data_as(_dp) for a in arrs])

    def work_function_field(self, W_eV):
        """The work-function barrier field of height W_eV built from the mask
        (returned, not set)."""
        out = [np.zeros(self.shape) for _ in range(3)]
        self._L.orc_work_function_field(self._h, float(W_eV), *[a.ctypes.data_as(_dp) for a in out])
        return out

    def set_binding_offdiag(self, k, w2off):
        """Off-diagonal (xy, xz, yz) entries of bound species k's Omega^2 (s^-2)."""
        a = np.ascontiguousarray(w2off, dtype=np.float64)
        self._off = a
        self._L.orc_set_binding_offdiag(self._h, int(k), a.ctypes.data_as(_dp))

    def set_shape_order(self, order):
        """1 CIC, 2 TSC for the free and Dirac particles (before add_species)."""
        self._L.orc_set_shape_order(self._h, int(order))

    def set_particle_bc(self, open_edges=False, p_diffuse=0.0, seed=0):
        self._L.orc_set_particle_bc(self._h, int(bool(open_edges)), float(p_diffuse), int(seed))

    def add_species(self, kind, q, m, w, X, V, D=None, omega0=(0, 0, 0), gamma=(0, 0, 0),
                    vF=0.0, bg=0):
        X, pX = _d(np.asarray(X, dtype=np.float64).reshape(-1, 3))
        V, pV = _d(np.asarray(V, dtype=np.float64).reshape(-1, 3))
        if D is None:
            D = np.zeros_like(X)
        D, pD = _d(np.asarray(D, dtype=np.float64).reshape(-1, 3))
        _, pw = _d(np.asarray(omega0, dtype=np.float64))
        _, pg = _d(np.asarray(gamma, dtype=np.float64))
        k = self._L.orc_add_species(self._h, kind, q, m, w, pw, pg, vF, X.shape[0], pX, pV, pD, bg)
        if k < 0:
            raise RuntimeError("too many species")
        self.nsp += 1
        return k

    def step(self, n=1):
        self._L.orc_step(self._h, int(n))

    def field(self, comp):
        """comp 0..2 E, 3..5 B (half step), 6..8 J of the last step, 9..11 B^n
        used by the last gather."""
        out = np.zeros(self.shape)
        self._L.orc_get_field(self._h, comp, out.ctypes.data_as(_dp))
        return out

    def set_field(self, comp, arr):
        a, pa = _d(np.asarray(arr, dtype=np.float64).reshape(self.shape))
        self._L.orc_set_field(self._h, comp, pa)

    def J(self, comp):
        out = np.zeros(self.shape)
        self._L.orc_get_J(self._h, comp, out.ctypes.data_as(_dp))
        return out

    def clear_J(self):
        self._L.orc_clear_J(self._h)

    def species(self, k):
        n = self._L.orc_species_count(self._h, k)
        X = np.zeros((max(n, 1), 3))
        V = np.zeros((max(n, 1), 3))
        D = np.zeros((max(n, 1), 3))
        nr = C.c_longlong(0)
        self._L.orc_get_species(self._h, k, X.ctypes.data_as(_dp), V.ctypes.data_as(_dp),
                              D.ctypes.data_as(_dp), C.byref(nr))
        return X[:n], V[:n], D[:n], int(nr.value)

    def cell_counts(self, k):
        out = np.zeros(self.shape, dtype=np.int32)
        self._L.orc_cell_counts(self._h, k, out.ctypes.data_as(_i32p))
        return out

    def energy_histogram(self, k, e_max, nbins):
        """Kinetic-energy histogram of species k: nbins bins of width
        e_max / nbins, then the count of E >= e_max (uint64, nbins + 1)."""
        out = np.zeros(nbins + 1, dtype=np.uint64)
        self._L.orc_energy_histogram(self._h, k, float(e_max), int(nbins),
                                   out.ctypes.data_as(C.POINTER(C.c_uint64)))
        return out

    def rho(self):
        out = np.zeros(self.shape)
        self._L.orc_rho(self._h, out.ctypes.data_as(_dp))
        return out

    def diag(self):
        out = np.zeros(13)
        self._L.orc_diag(self._h, out.ctypes.data_as(_dp))
        return {"kinetic": out[:self.nsp].copy(), "field_E": out[8], "field_B": out[9],
                "gauss_max": out[10], "gauss_rms": out[11], "rho_max": out[12]}

    def gather(self, X):
        _, pX = _d(np.asarray(X, dtype=np.float64))
        E = np.zeros(3)
        B = np.zeros(3)
        self._L.orc_gather(self._h, pX, E.ctypes.data_as(_dp), B.ctypes.data_as(_dp))
        return E, B

    def deposit_one(self, X0, X1, qw, vz=0.0):
        _, p0 = _d(np.asarray(X0, dtype=np.float64))
        _, p1 = _d(np.asarray(X1, dtype=np.float64))
        self._L.orc_deposit_one(self._h, p0, p1, qw, vz)
