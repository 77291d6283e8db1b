"""Seeded synthetic inputs shared by the tests, the smoke check and the
benchmark: grid and species parameters of the workloads, material masks,
random particle sets, initial fields.

This module holds none of the PIC method's arithmetic (no push, gather,
deposit, field update or Fermi-Dirac sampling) and imports nothing from the
CUDA binding or the oracle, so that both sides can be fed the same arrays.

Workloads (the paper's metal / graphene settings, Secs. 2-5):
  langmuir2d  2D3V periodic 64 x 64, dx = 0.1 nm, 16 ppc free electrons
              (n = 8.5e28 m^-3, E_F = 7.0 eV, 300 K, quiet 4 x 4 lattice),
              uniform ions, 1 % sinusoidal density ripple along x,
              dt = 0.5 dx / (c sqrt 2), 1000 steps.
  sphere3d    256^3, dx = 0.5 nm, CPML 16 on all faces, sphere of radius
              20 nm: 8 ppc free electrons (n = 5.9e28, E_F = 5.5 eV, 300 K)
              + 8 ppc bound electrons (w0 = 2 pi c / 400 nm, gamma = 1e14,
              N_b = 0.5 n), pulse lambda = 520 nm, 10 fs FWHM, 1e8 V/m,
              dt = 0.5 dx / (c sqrt 3), 4000 steps.
  graphene3d  512 x 512 x 64, dx = 1 nm, periodic x/y, CPML 16 along z, a
              one-cell sheet at z = 32 with 32 ppc Dirac carriers
              (v_F = 1e6, n_s = 1e16 m^-2, E_F = 0.2 eV, 300 K), normally
              incident 10 THz pulse of 1e6 V/m, dt = 0.5 dx / (c sqrt 3),
              2000 steps.
  batch2d     256 independent 2D nanostructures: N x N grids with N drawn
              log-uniformly in [64, 512], dx = 0.5 nm, CPML min(16, N/8);
              a disk, rod or bowtie (gap 2-10 nm) holding 4-16 ppc FD free
              electrons (langmuir2d's n, E_F, T) + as many bound electrons
              (sphere3d's w0, gamma, N_b = 0.5 n); pulse lambda uniform in
              400-900 nm; 500-3000 steps each.
  serve_jobs  a Poisson stream of jobs: 70 % 2D (64^2-512^2), 30 % 3D
              (64^3-192^3), each taking the species mix of one of the three
              settings above, 100-5000 steps.
"""
from __future__ import annotations

import math

import numpy as np

QE = 1.602176634e-19
ME = 9.1093837015e-31
C_LIGHT = 299792458.0
EPS0 = 8.8541878128e-12
HBAR = 1.054571817e-34
SEED_BASE = 250107465

FREE, BOUND, DIRAC = 0, 1, 2


def grid_shape(n):
    """(nz, ny, nx) array shape of a grid with n = (nx, ny, nz)."""
    return (n[2], n[1], n[0])


# ---------------------------------------------------------------------------
# masks
# ---------------------------------------------------------------------------

def sphere_mask(n, radius_cells, center=None):
    """1 inside a sphere (cell centres within radius_cells of center)."""
    nx, ny, nz = n
    c = center if center is not None else (nx / 2, ny / 2, nz / 2)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r2 = (i + 0.5 - c[0]) ** 2 + (j + 0.5 - c[1]) ** 2 + (k + 0.5 - c[2]) ** 2
    return (r2 < radius_cells ** 2).astype(np.uint8)


def sheet_mask(n, k0):
    """1 on the plane of cells z = k0."""
    m = np.zeros(grid_shape(n), np.uint8)
    m[k0] = 1
    return m


def disk_mask2d(n, center, radius):
    nx, ny = n[0], n[1]
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    return (((i + 0.5 - center[0]) ** 2 + (j + 0.5 - center[1]) ** 2) < radius ** 2).astype(
        np.uint8)[None]


def rod_mask2d(n, center, length, width):
    nx, ny = n[0], n[1]
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    return ((np.abs(i + 0.5 - center[0]) < length / 2) &
            (np.abs(j + 0.5 - center[1]) < width / 2)).astype(np.uint8)[None]


def bowtie_mask2d(n, center, size, gap):
    """Two triangles pointing at each other along x with a gap (cells)."""
    nx, ny = n[0], n[1]
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    x = i + 0.5 - center[0]
    y = j + 0.5 - center[1]
    ax = np.abs(x) - gap / 2
    inside = (ax >= 0) & (ax <= size) & (np.abs(y) <= ax * 0.6)
    return inside.astype(np.uint8)[None]


# ---------------------------------------------------------------------------
# particles
# ---------------------------------------------------------------------------

def cell_coords(cell, n):
    """Linear cell index -> (N, 3) integer coordinates (x fastest)."""
    cell = np.asarray(cell, np.int64)
    cz, rem = np.divmod(cell, n[0] * n[1])
    cy, cx = np.divmod(rem, n[0])
    return np.stack([cx, cy, cz], 1)


def positions(cell, off, n):
    """Cell index + in-cell offset -> position in cell units (float64)."""
    return cell_coords(cell, n).astype(np.float64) + np.asarray(off, np.float64)


def random_particles(rng, n, count, mask=None, vscale=1e6, dims=3, cells=None):
    """`count` particles in uniformly chosen (material) cells: int32 cell,
    float32 offsets in [0,1), float32 Gaussian velocities of scale vscale.
    In 2D the z offset is 0.5 and v_z is kept (2D3V)."""
    if cells is None:
        ncell = n[0] * n[1] * n[2]
        pool = np.arange(ncell) if mask is None else np.flatnonzero(np.asarray(mask).ravel())
        cells = rng.choice(pool, size=count)
    cell = np.asarray(cells, np.int32)
    off = rng.random((count, 3)).astype(np.float32)
    off = np.minimum(off, np.float32(np.nextafter(np.float32(1), np.float32(0))))
    if dims == 2:
        off[:, 2] = 0.5
    v = (rng.normal(size=(count, 3)) * vscale).astype(np.float32)
    return cell, off, v


def random_bound(rng, n, count, mask=None, dscale=1e-12, vscale=1e4):
    """Bound particles: int32 anchor cell, float64 anchor offsets,
    float32 displacements (m) and velocities."""
    ncell = n[0] * n[1] * n[2]
    pool = np.arange(ncell) if mask is None else np.flatnonzero(np.asarray(mask).ravel())
    cell = rng.choice(pool, size=count).astype(np.int32)
    anchor = rng.random((count, 3))
    disp = (rng.normal(size=(count, 3)) * dscale).astype(np.float32)
    v = (rng.normal(size=(count, 3)) * vscale).astype(np.float32)
    return cell, anchor, disp, v


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def dirac_sheet_ring(nx, ny, k0, q, dx, vF, ppc_side=4, drift=0.1):
    """Quiet start of a sheet of Dirac carriers in the node plane z = k0 of
    an nx x ny x nz grid: a ppc_side x ppc_side lattice per cell (z offset
    exactly 0, so the sheet stays one node plane thick), in-plane directions
    evenly spaced over the circle (no net current per cell), each then
    tilted toward +x by drift * cos(q x) and set back to speed v_F.  The
    sheet starts with a current ripple ~ (drift / 2) v_F cos(q x), uniform
    density and v_z = 0.  Returns (cell int32, off float32 (N,3), v float32
    (N,3), ppc)."""
    ppc = ppc_side * ppc_side
    a, b = np.meshgrid(np.arange(ppc_side), np.arange(ppc_side), indexing="ij")
    a, b = a.ravel(), b.ravel()
    th = 2 * math.pi * (a * ppc_side + b + 0.5) / ppc
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    i, j = i.ravel(), j.ravel()
    fx = (a + 0.5) / ppc_side
    fy = (b + 0.5) / ppc_side
    x = (i[:, None] + fx[None, :]) * dx
    ux = np.cos(th)[None, :] + drift * np.cos(q * x)
    uy = np.broadcast_to(np.sin(th)[None, :], ux.shape)
    nrm = np.hypot(ux, uy)
    cell = ((k0 * ny + j) * nx + i)[:, None] + np.zeros((1, ppc), np.int64)
    off = np.stack([np.broadcast_to(fx, ux.shape), np.broadcast_to(fy, ux.shape),
                    np.zeros(ux.shape)], -1)
    v = np.stack([vF * ux / nrm, vF * uy / nrm, np.zeros(ux.shape)], -1)
    return (cell.reshape(-1).astype(np.int32), off.reshape(-1, 3).astype(np.float32),
            v.reshape(-1, 3).astype(np.float32), ppc)


def fermi_velocity(E_F, m=ME):
    return math.sqrt(2 * E_F / m)


def langmuir2d(nx=64, ny=64, ppc=16, steps=1000):
    dx = 0.1e-9
    dt = 0.5 * dx / (C_LIGHT * math.sqrt(2))
    n0 = 8.5e28
    return {
        "name": f"langmuir2d {nx}x{ny} {ppc}ppc",
        "grid": dict(dims=2, n=(nx, ny, 1), d=(dx, dx, dx), dt=dt, bc=(0, 0, 0), pml_cells=0),
        "species": [dict(kind=FREE, q=-QE, m=ME, density=n0, E_F=7.0 * QE, T=300.0, ppc=ppc,
                         quiet=1, background=2, seed=SEED_BASE + 0, stream=0)],
        "mask": None,
        "steps": steps,
        "ripple": 0.01,
    }


def langmuir_ripple(X, nx, dx, amplitude):
    """Displace x by -(A/k) sin(kx) (cell units), k = 2 pi / (nx dx): a
    density ripple n0 (1 + A cos kx) to first order."""
    k = 2 * math.pi / (nx * dx)
    Y = np.array(X, dtype=np.float64, copy=True)
    Y[:, 0] = Y[:, 0] - amplitude / (k * dx) * np.sin(k * Y[:, 0] * dx)
    Y[:, 0] = np.mod(Y[:, 0], nx)
    return Y


def langmuir_initial_Ex(nx, ny, dx, n0, amplitude):
    """E_x(i+1/2) = -(e n0 A / (eps0 k)) sin(k (i+1/2) dx) for electrons of
    charge -e (Gauss's law of the ripple with a uniform ion background)."""
    k = 2 * math.pi / (nx * dx)
    i = np.arange(nx)
    ex = -(QE * n0 * amplitude / (EPS0 * k)) * np.sin(k * (i + 0.5) * dx)
    return np.broadcast_to(ex, (1, ny, nx)).copy()


def sphere3d(n=256, radius_nm=20.0, ppc=8, steps=4000, pml=16):
    dx = 0.5e-9
    dt = 0.5 * dx / (C_LIGHT * math.sqrt(3))
    lam = 520e-9
    nfree = 5.9e28
    w0 = 2 * math.pi * C_LIGHT / 400e-9
    return {
        "name": f"sphere3d {n}^3 r={radius_nm}nm {ppc}+{ppc}ppc",
        "grid": dict(dims=3, n=(n, n, n), d=(dx, dx, dx), dt=dt, bc=(1, 1, 1), pml_cells=pml,
                     src=dict(inc_axis=0, pol_axis=1, src_index=pml + 2, E0=1e8,
                              omega=2 * math.pi * C_LIGHT / lam, tau=10e-15, t0=1.0e-15)),
        "mask": sphere_mask((n, n, n), radius_nm * 1e-9 / dx),
        "species": [
            dict(kind=FREE, q=-QE, m=ME, density=nfree, E_F=5.5 * QE, T=300.0, ppc=ppc, quiet=0,
                 background=1, seed=SEED_BASE + 1, stream=0),
            dict(kind=BOUND, q=-QE, m=ME, density=0.5 * nfree, E_F=0.0, T=0.0, ppc=ppc,
                 quiet=1, background=1, seed=SEED_BASE + 1, stream=1, omega0=(w0, w0, w0),
                 gamma=(1e14, 1e14, 1e14)),
        ],
        "steps": steps,
    }


def graphene3d(nx=512, ny=512, nz=64, ppc=32, steps=2000, pml=16):
    dx = 1e-9
    dt = 0.5 * dx / (C_LIGHT * math.sqrt(3))
    vF = 1e6
    E_F = 0.2 * QE
    m_d = (E_F / vF) / (2 * vF)  # averaged transverse mass p_F / (2 v_F), Sec. 5
    n_s = 1e16
    return {
        "name": f"graphene3d {nx}x{ny}x{nz} {ppc}ppc",
        "grid": dict(dims=3, n=(nx, ny, nz), d=(dx, dx, dx), dt=dt, bc=(0, 0, 1), pml_cells=pml,
                     src=dict(inc_axis=2, pol_axis=0, src_index=pml + 2, E0=1e6,
                              omega=2 * math.pi * 10e12, tau=200e-15, t0=0.0)),
        "mask": sheet_mask((nx, ny, nz), nz // 2),
        "species": [dict(kind=DIRAC, q=-QE, m=m_d, v_F=vF, density=n_s / dx, E_F=E_F, T=300.0,
                         ppc=ppc, quiet=0, background=1, seed=SEED_BASE + 2, stream=0)],
        "steps": steps,
    }


def fermi_energy(n, m=ME):
    """E_F = hbar^2 / (2 m) (3 pi^2 n)^(2/3) (Sec. 2, exponent read as 2/3)."""
    return HBAR ** 2 / (2 * m) * (3 * math.pi ** 2 * n) ** (2.0 / 3.0)


def bulk_cube(n_e, ppc, side_nm=2.0, cell_nm=0.2, T_eV=0.0375, steps=104000, seed=SEED_BASE + 5):
    """The Fermi-Dirac relaxation workload (Sec. 2): a periodic cube of bulk
    electron plasma, side 2 nm, fixed uniform ions, electrons placed at
    random with FD momenta at T = 0.0375 eV and E_F from the density.  The
    cell (0.2 nm) and the run length (104000 steps = 20 fs at 0.5 x CFL) are
    chosen here: the paper's supplementary parameters are not given."""
    n = int(round(side_nm / cell_nm))
    dx = cell_nm * 1e-9
    dt = 0.5 * dx / (C_LIGHT * math.sqrt(3))
    return {
        "name": f"bulk cube {side_nm}nm n={n_e:.1e} {ppc}ppc",
        "grid": dict(dims=3, n=(n, n, n), d=(dx, dx, dx), dt=dt, bc=(0, 0, 0), pml_cells=0),
        "mask": None,
        "species": [dict(kind=FREE, q=-QE, m=ME, density=n_e, E_F=fermi_energy(n_e),
                         T=T_eV * QE / 1.380649e-23, ppc=ppc, quiet=0, background=2,
                         seed=seed, stream=0)],
        "steps": steps,
    }


# ---------------------------------------------------------------------------
# batched sweep and served job stream
# ---------------------------------------------------------------------------

def _log_uniform_side(rng, lo, hi, mult=8):
    n = math.exp(rng.uniform(math.log(lo), math.log(hi)))
    return int(min(hi, max(lo, mult * round(n / mult))))


def _pulse(lam, pml, E0=1e8, fwhm=0.5e-15):
    return dict(inc_axis=0, pol_axis=1, src_index=pml + 2, E0=E0,
                omega=2 * math.pi * C_LIGHT / lam, tau=fwhm, t0=1.5 * fwhm)


def nanostructure2d(k, N, shape, size_frac, gap_nm, ppc, lam, steps, seed=SEED_BASE + 3):
    """One 2D nanostructure: N x N cells of 0.5 nm, CPML min(16, N/8) on the
    four sides, a disk / rod / bowtie mask centred in the box, FD free
    electrons (n = 8.5e28, E_F = 7.0 eV, 300 K) and bound Lorentz electrons
    (w0 = 2 pi c / 400 nm, gamma = 1e14, N_b = 0.5 n), ppc of each, a
    y-polarised pulse entering along x."""
    dx = 0.5e-9
    dt = 0.5 * dx / (C_LIGHT * math.sqrt(2))
    pml = min(16, N // 8)
    L = N - 2 * pml
    n = (N, N, 1)
    c = (N / 2, N / 2)
    if shape == "disk":
        mask = disk_mask2d(n, c, max(2.0, size_frac * L))
    elif shape == "rod":
        mask = rod_mask2d(n, c, max(4.0, 2 * size_frac * L), max(2.0, 0.4 * size_frac * L))
    else:
        gap = gap_nm * 1e-9 / dx
        size = max(3.0, min(size_frac * L, (0.8 * L - gap) / 2))
        mask = bowtie_mask2d(n, c, size, gap)
    nfree = 8.5e28
    w0 = 2 * math.pi * C_LIGHT / 400e-9
    return {
        "name": f"nano2d[{k}] {N}^2 {shape} {ppc}+{ppc}ppc",
        "grid": dict(dims=2, n=n, d=(dx, dx, dx), dt=dt, bc=(1, 1, 0), pml_cells=pml,
                     src=_pulse(lam, pml)),
        "mask": mask,
        "species": [
            dict(kind=FREE, q=-QE, m=ME, density=nfree, E_F=7.0 * QE, T=300.0, ppc=ppc, quiet=0,
                 background=1, seed=seed, stream=2 * k),
            dict(kind=BOUND, q=-QE, m=ME, density=0.5 * nfree, E_F=0.0, T=0.0, ppc=ppc, quiet=0,
                 background=1, seed=seed, stream=2 * k + 1, omega0=(w0, w0, w0),
                 gamma=(1e14, 1e14, 1e14)),
        ],
        "steps": steps,
    }


def batch2d(count=256, seed=SEED_BASE + 3):
    """The batched sweep: `count` independent 2D nanostructures (seeded)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        N = _log_uniform_side(rng, 64, 512)
        shape = ("disk", "rod", "bowtie")[int(rng.integers(3))]
        size_frac = float(rng.uniform(0.15, 0.3))
        gap_nm = float(rng.uniform(2.0, 10.0))
        ppc = int(rng.integers(4, 17))
        lam = float(rng.uniform(400e-9, 900e-9))
        steps = int(rng.integers(500, 3001))
        out.append(nanostructure2d(k, N, shape, size_frac, gap_nm, ppc, lam, steps, seed))
    return out


def _periodic_plasma(k, dims, N, steps, seed):
    """The Langmuir setting's species on an N^dims periodic box (quiet
    lattice, uniform ions; 16 ppc in 2D, 8 ppc in 3D)."""
    dx = 0.1e-9
    dt = 0.5 * dx / (C_LIGHT * math.sqrt(dims))
    ppc = 16 if dims == 2 else 8
    n = (N, N, 1 if dims == 2 else N)
    return {
        "name": f"job[{k}] plasma{dims}d {N}^{dims}",
        "grid": dict(dims=dims, n=n, d=(dx, dx, dx), dt=dt, bc=(0, 0, 0), pml_cells=0),
        "mask": None,
        "species": [dict(kind=FREE, q=-QE, m=ME, density=8.5e28, E_F=7.0 * QE, T=300.0, ppc=ppc,
                         quiet=1, background=2, seed=seed, stream=k)],
        "steps": steps,
    }


def _metal3d(k, N, steps, seed):
    wl = sphere3d(n=N, radius_nm=20.0 * N / 256, pml=min(16, N // 8), steps=steps)
    wl["name"] = f"job[{k}] metal3d {N}^3"
    for q, sp in enumerate(wl["species"]):
        sp["seed"] = seed
        sp["stream"] = 2 * k + q
    return wl


def _graphene(k, N, steps, seed):
    nz = max(32, N // 4)
    wl = graphene3d(nx=N, ny=N, nz=nz, pml=min(16, nz // 4), steps=steps)
    wl["name"] = f"job[{k}] graphene {N}x{N}x{nz}"
    wl["species"][0]["seed"] = seed
    wl["species"][0]["stream"] = k
    return wl


def serve_jobs(count, rate, seed=SEED_BASE + 4):
    """A seeded Poisson job stream at `rate` jobs/s: 70 % 2D grids (N log-
    uniform in [64, 512]), 30 % 3D (N in [64, 192]); each job takes the
    species mix of the Langmuir plasma, the metal nanostructure (free +
    bound) or, in 3D, the graphene sheet; 100-5000 steps.  Returns the jobs
    with their arrival times (s) in "arrival"."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += float(rng.exponential(1.0 / rate))
        steps = int(rng.integers(100, 5001))
        if rng.random() < 0.7:
            N = _log_uniform_side(rng, 64, 512)
            if rng.random() < 0.5:
                wl = _periodic_plasma(k, 2, N, steps, seed)
            else:
                wl = nanostructure2d(k, N, ("disk", "rod", "bowtie")[int(rng.integers(3))],
                                     float(rng.uniform(0.15, 0.3)), float(rng.uniform(2, 10)),
                                     int(rng.integers(4, 17)), float(rng.uniform(400e-9, 900e-9)),
                                     steps, seed)
                wl["name"] = f"job[{k}] " + wl["name"]
        else:
            N = _log_uniform_side(rng, 64, 192)
            mix = int(rng.integers(3))
            wl = (_periodic_plasma(k, 3, N, steps, seed) if mix == 0 else
                  _metal3d(k, N, steps, seed) if mix == 1 else _graphene(k, N, steps, seed))
        wl["arrival"] = t
        wl["job"] = k
        out.append(wl)
    return out
