"""Python binding of the C ABI in include/pic.h (libpic.so).

Argument marshalling only: every step of the PIC path runs in the CUDA
kernels behind the ABI.  The functions keep the ABI's names.  Importing
this module loads the in-tree libpic.so and fails loudly if it is missing;
there is no fallback.  PyTorch serves only as the device-memory allocator
(``use_torch_allocator``) and as the source of CUDA streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpic.so")

PIC_OK, PIC_EINVAL, PIC_ENOMEM, PIC_EDTLIMIT, PIC_ECUDA = 0, 1, 2, 3, 4
PIC_ETIMEOUT, PIC_ESTATE, PIC_EBOUNDS, PIC_EBUDGET = 5, 6, 7, 8
STATUS_NAMES = {0: "PIC_OK", 1: "PIC_EINVAL", 2: "PIC_ENOMEM", 3: "PIC_EDTLIMIT",
                4: "PIC_ECUDA", 5: "PIC_ETIMEOUT", 6: "PIC_ESTATE", 7: "PIC_EBOUNDS",
                8: "PIC_EBUDGET"}
PIC_BC_PERIODIC, PIC_BC_PML = 0, 1
PIC_FREE, PIC_BOUND, PIC_DIRAC = 0, 1, 2
PIC_BG_NONE, PIC_BG_AT_PARTICLES, PIC_BG_UNIFORM = 0, 1, 2
PIC_EX, PIC_EY, PIC_EZ, PIC_BX, PIC_BY, PIC_BZ = 1, 2, 4, 8, 16, 32
PIC_JX, PIC_JY, PIC_JZ = 64, 128, 256
PIC_EXTX, PIC_EXTY, PIC_EXTZ = 512, 1024, 2048
PIC_EDGE_REFLECT, PIC_EDGE_OPEN = 0, 1
PIC_MAX_SPECIES = 8


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class pic_grid_desc(C.Structure):
    _fields_ = [("dims", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("dt", C.c_double),
                ("bc", C.c_int * 3), ("pml_cells", C.c_int), ("pml_R0", C.c_double),
                ("pml_order", C.c_int), ("src_on", C.c_int), ("inc_axis", C.c_int),
                ("pol_axis", C.c_int), ("src_index", C.c_int), ("E0", C.c_double),
                ("omega", C.c_double), ("tau", C.c_double), ("t0", C.c_double)]


class pic_species_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("q", C.c_double), ("m", C.c_double),
                ("weight", C.c_double), ("omega0", C.c_double * 3), ("gamma", C.c_double * 3),
                ("v_F", C.c_double), ("background", C.c_int)]


class pic_particles(C.Structure):
    _fields_ = [("n", C.c_int64), ("cell", C.POINTER(C.c_int32)), ("off", C.POINTER(C.c_float)),
                ("v", C.POINTER(C.c_float)), ("anchor_off", C.POINTER(C.c_double)),
                ("disp", C.POINTER(C.c_float)), ("density", C.c_double), ("E_F", C.c_double),
                ("T", C.c_double), ("ppc", C.c_int), ("quiet", C.c_int), ("seed", C.c_uint64),
                ("stream", C.c_uint32)]


class pic_tuning(C.Structure):
    _fields_ = [("tile", C.c_int * 3), ("sort_interval", C.c_int), ("field_zchunk", C.c_int),
                ("particle_ctas", C.c_int), ("keep_J", C.c_int), ("timing", C.c_int),
                ("field_plain", C.c_int), ("tile_order", C.c_int), ("no_overlap", C.c_int),
                ("field_mode", C.c_int), ("wait_polls", C.c_int64), ("field_overlap", C.c_int)]


class pic_diag(C.Structure):
    _fields_ = [("step", C.c_int64), ("time", C.c_double), ("nspecies", C.c_int),
                ("count", C.c_int64 * PIC_MAX_SPECIES),
                ("reflections", C.c_uint64 * PIC_MAX_SPECIES),
                ("kinetic", C.c_double * PIC_MAX_SPECIES), ("field_E", C.c_double),
                ("field_B", C.c_double), ("gauss_max", C.c_double), ("gauss_rms", C.c_double),
                ("rho_max", C.c_double)]


class pic_timing(C.Structure):
    _fields_ = [("particle_ms", C.c_double), ("field_ms", C.c_double), ("sort_ms", C.c_double),
                ("particle_launches", C.c_int64), ("field_launches", C.c_int64),
                ("sort_launches", C.c_int64), ("kernel_launches", C.c_int64),
                ("fieldb_ms", C.c_double), ("fieldb_launches", C.c_int64)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

# every exported symbol of include/pic.h with (restype, argtypes)
_H = C.c_void_p
SIGNATURES = {
    "pic_set_allocator": (C.c_int, [ALLOC_FN, FREE_FN, C.c_void_p]),
    "pic_create": (C.c_int, [C.POINTER(pic_grid_desc), C.c_void_p, C.POINTER(C.c_void_p)]),
    "pic_destroy": (C.c_int, [_H]),
    "pic_set_material_mask": (C.c_int, [_H, C.POINTER(C.c_uint8), C.c_size_t]),
    "pic_set_permittivity": (C.c_int, [_H, C.POINTER(C.c_float), C.c_size_t]),
    "pic_set_external_field": (C.c_int, [_H, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                         C.POINTER(C.c_double), C.c_size_t]),
    "pic_set_work_function": (C.c_int, [_H, C.c_double]),
    "pic_set_particle_bc": (C.c_int, [_H, C.c_int, C.c_double, C.c_uint64]),
    "pic_set_shape_order": (C.c_int, [_H, C.c_int]),
    "pic_set_binding_tensor": (C.c_int, [_H, C.c_int, C.POINTER(C.c_double)]),
    "pic_load_species": (C.c_int, [_H, C.POINTER(pic_species_desc), C.POINTER(pic_particles),
                                   C.POINTER(C.c_int)]),
    "pic_set_tuning": (C.c_int, [_H, C.POINTER(pic_tuning)]),
    "pic_step": (C.c_int, [_H, C.c_int]),
    "pic_sync": (C.c_int, [_H]),
    "pic_read_fields": (C.c_int, [_H, C.c_int, C.POINTER(C.c_double), C.c_size_t]),
    "pic_write_fields": (C.c_int, [_H, C.c_int, C.POINTER(C.c_double), C.c_size_t]),
    "pic_read_species": (C.c_int, [_H, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_float),
                                   C.POINTER(C.c_float), C.POINTER(C.c_double),
                                   C.POINTER(C.c_float), C.c_size_t]),
    "pic_cell_counts": (C.c_int, [_H, C.c_int, C.POINTER(C.c_int32), C.c_size_t]),
    "pic_diagnostics": (C.c_int, [_H, C.POINTER(pic_diag)]),
    "pic_energy_histogram": (C.c_int, [_H, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_uint64),
                                       C.c_size_t]),
    "pic_get_timing": (C.c_int, [_H, C.POINTER(pic_timing)]),
    "pic_memory_bytes": (C.c_int, [_H, C.POINTER(C.c_size_t)]),
    "pic_last_error": (C.c_char_p, [_H]),
    "pic_cell_counts_noalloc": (C.c_int, [_H, C.c_int, C.POINTER(C.c_int32), C.c_size_t]),
    "pic_group_create": (C.c_int, [C.c_int, C.c_size_t, C.c_void_p, C.c_int,
                                   C.POINTER(C.c_void_p)]),
    "pic_group_destroy": (C.c_int, [_H]),
    "pic_group_add": (C.c_int, [_H, _H, C.c_int64]),
    "pic_group_remove": (C.c_int, [_H, _H]),
    "pic_group_step": (C.c_int, [_H, C.c_int]),
    "pic_group_sync": (C.c_int, [_H]),
    "pic_group_progress": (C.c_int, [_H, _H, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "pic_group_info": (C.c_int, [_H, C.POINTER(C.c_int), C.POINTER(C.c_size_t),
                                 C.POINTER(C.c_int64)]),
}
PIC_NOALLOC_MAX_CELLS = 1 << 22

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libpic.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_2501_07465_gb300.build")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(st, h=None):
    if st != PIC_OK:
        msg = load_library().pic_last_error(h)
        raise PicError(st, msg.decode() if msg else "")


def _ptr(a, ctype):
    return None if a is None else a.ctypes.data_as(C.POINTER(ctype))


# ---------------------------------------------------------------------------
# device memory through PyTorch's caching allocator
# ---------------------------------------------------------------------------

_hooks = None


def use_torch_allocator():
    """Route every device allocation of the library through
    torch.cuda.caching_allocator_alloc / caching_allocator_delete."""
    global _hooks
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream or 0))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    _hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(load_library().pic_set_allocator(_hooks[0], _hooks[1], None))


def use_cuda_allocator():
    """Back to the library's own cudaMalloc / cudaFree."""
    global _hooks
    _check(load_library().pic_set_allocator(ALLOC_FN(), FREE_FN(), None))
    _hooks = None


# ---------------------------------------------------------------------------
# ABI calls
# ---------------------------------------------------------------------------

def make_grid(dims, n, d, dt, bc=(0, 0, 0), pml_cells=0, pml_R0=0.0, pml_order=0, src=None):
    """pic_grid_desc from Python values; src = dict(inc_axis, pol_axis,
    src_index, E0, omega, tau, t0) or None."""
    g = pic_grid_desc()
    g.dims = dims
    g.nx, g.ny, g.nz = (list(n) + [1, 1])[:3]
    g.dx, g.dy, g.dz = d
    g.dt = dt
    g.bc = (C.c_int * 3)(*bc)
    g.pml_cells, g.pml_R0, g.pml_order = pml_cells, pml_R0, pml_order
    if src:
        g.src_on = 1
        g.inc_axis, g.pol_axis, g.src_index = src["inc_axis"], src["pol_axis"], src["src_index"]
        g.E0, g.omega, g.tau, g.t0 = src["E0"], src["omega"], src["tau"], src["t0"]
    return g


def pic_create(grid: pic_grid_desc, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(load_library().pic_create(C.byref(grid), C.c_void_p(stream), C.byref(h)))
    return h.value


def pic_destroy(h):
    _check(load_library().pic_destroy(h))


def pic_set_material_mask(h, mask):
    m = np.ascontiguousarray(mask, dtype=np.uint8).ravel()
    _check(load_library().pic_set_material_mask(h, _ptr(m, C.c_uint8), m.size), h)


def pic_set_permittivity(h, eps_r):
    """Relative permittivity per cell, [nz][ny][nx] (None: vacuum)."""
    if eps_r is None:
        _check(load_library().pic_set_permittivity(h, None, 0), h)
        return
    e = np.ascontiguousarray(eps_r, dtype=np.float32).ravel()
    _check(load_library().pic_set_permittivity(h, _ptr(e, C.c_float), e.size), h)


def pic_set_external_field(h, E):
    """External electrostatic field (Ex, Ey, Ez), each [nz][ny][nx] in V/m on
    the E stagger, seen by the particles only (None: remove)."""
    if E is None:
        _check(load_library().pic_set_external_field(h, None, None, None, 0), h)
        return
    arrs = [np.ascontiguousarray(c, dtype=np.float64).ravel() for c in E]
    _check(load_library().pic_set_external_field(h, *[_ptr(a, C.c_double) for a in arrs],
                                                 arrs[0].size), h)


def pic_set_work_function(h, W_eV):
    """The work-function barrier of height W_eV built from the mask."""
    _check(load_library().pic_set_work_function(h, float(W_eV)), h)


def pic_set_binding_tensor(h, k, w2off):
    """Off-diagonal entries (xy, xz, yz, s^-2) of bound species k's binding
    tensor; the diagonal stays omega0^2."""
    a = np.ascontiguousarray(w2off, dtype=np.float64).ravel()
    _check(load_library().pic_set_binding_tensor(h, int(k), _ptr(a, C.c_double)), h)


def pic_set_shape_order(h, order):
    """1 CIC (default), 2 TSC for the free and Dirac particles (before
    loading species)."""
    _check(load_library().pic_set_shape_order(h, int(order)), h)


def pic_set_particle_bc(h, edges=0, p_diffuse=0.0, seed=0):
    """PIC_EDGE_REFLECT (with a diffuse share p_diffuse) or PIC_EDGE_OPEN."""
    _check(load_library().pic_set_particle_bc(h, int(edges), float(p_diffuse), int(seed)), h)


def species_desc(kind, q, m, weight=0.0, omega0=(0, 0, 0), gamma=(0, 0, 0), v_F=0.0,
                 background=PIC_BG_NONE):
    d = pic_species_desc()
    d.kind, d.q, d.m, d.weight = kind, q, m, weight
    d.omega0 = (C.c_double * 3)(*omega0)
    d.gamma = (C.c_double * 3)(*gamma)
    d.v_F, d.background = v_F, background
    return d


def pic_load_species(h, desc: pic_species_desc, cell=None, off=None, v=None, anchor_off=None,
                     disp=None, density=0.0, E_F=0.0, T=0.0, ppc=0, quiet=0, seed=0, stream=0):
    """Explicit particles (cell int32 (n,), off/v float32 (n,3), anchor_off
    float64 (n,3), disp float32 (n,3)) or, with cell=None, the Fermi-Dirac
    loader.  Returns the species id."""
    p = pic_particles()
    keep = []
    if cell is not None:
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        p.n = cell.size
        p.cell = _ptr(cell, C.c_int32)
        keep.append(cell)
        for name, arr, ct, dt in (("off", off, C.c_float, np.float32),
                                  ("v", v, C.c_float, np.float32),
                                  ("anchor_off", anchor_off, C.c_double, np.float64),
                                  ("disp", disp, C.c_float, np.float32)):
            if arr is not None:
                a = np.ascontiguousarray(arr, dtype=dt).reshape(-1)
                keep.append(a)
                setattr(p, name, _ptr(a, ct))
    p.density, p.E_F, p.T, p.ppc, p.quiet = density, E_F, T, ppc, quiet
    p.seed, p.stream = seed, stream
    sid = C.c_int(-1)
    _check(load_library().pic_load_species(h, C.byref(desc), C.byref(p), C.byref(sid)), h)
    return sid.value


def pic_set_tuning(h, tile=(0, 0, 0), sort_interval=0, field_zchunk=0, particle_ctas=0,
                   keep_J=0, timing=0, field_plain=0, tile_order=0, no_overlap=0, field_mode=0,
                   wait_polls=0, field_overlap=0):
    t = pic_tuning()
    t.tile = (C.c_int * 3)(*tile)
    t.sort_interval, t.field_zchunk, t.particle_ctas = sort_interval, field_zchunk, particle_ctas
    t.keep_J, t.timing, t.field_plain, t.tile_order = keep_J, timing, field_plain, tile_order
    t.no_overlap = no_overlap
    t.field_mode = field_mode  # 0 keeps the current mode
    t.wait_polls = wait_polls  # 0: the library's bound
    t.field_overlap = field_overlap  # 0 keeps the current choice
    _check(load_library().pic_set_tuning(h, C.byref(t)), h)


def pic_step(h, nsteps=1):
    _check(load_library().pic_step(h, int(nsteps)), h)


def pic_sync(h):
    _check(load_library().pic_sync(h), h)


def pic_read_fields(h, which, shape, out=None):
    """Returns float64 array (ncomp, nz, ny, nx) of the selected components;
    `out`, if given, is a C-contiguous float64 array of that many elements
    (e.g. a view of pinned host memory) that receives them."""
    ncomp = bin(which).count("1")
    size = ncomp * int(np.prod(shape))
    if out is None:
        out = np.zeros((ncomp,) + tuple(shape))
    elif out.dtype != np.float64 or not out.flags.c_contiguous or out.size != size:
        raise ValueError("out must be a C-contiguous float64 array of %d elements" % size)
    _check(load_library().pic_read_fields(h, which, _ptr(out, C.c_double), out.size), h)
    return out.reshape((ncomp,) + tuple(shape))


def pic_write_fields(h, which, arr):
    a = np.ascontiguousarray(arr, dtype=np.float64)
    _check(load_library().pic_write_fields(h, which, _ptr(a, C.c_double), a.size), h)


def pic_read_species(h, k, n, bound=False):
    """Species k in load order: dict(cell, off | anchor_off + disp, v)."""
    cell = np.zeros(max(n, 1), np.int32)
    v = np.zeros((max(n, 1), 3), np.float32)
    off = anchor = disp = None
    if bound:
        anchor = np.zeros((max(n, 1), 3), np.float64)
        disp = np.zeros((max(n, 1), 3), np.float32)
    else:
        off = np.zeros((max(n, 1), 3), np.float32)
    _check(load_library().pic_read_species(h, k, _ptr(cell, C.c_int32), _ptr(off, C.c_float),
                                           _ptr(v, C.c_float), _ptr(anchor, C.c_double),
                                           _ptr(disp, C.c_float), n), h)
    out = {"cell": cell[:n], "v": v[:n]}
    if bound:
        out["anchor_off"], out["disp"] = anchor[:n], disp[:n]
    else:
        out["off"] = off[:n]
    return out


def pic_cell_counts(h, k, shape):
    out = np.zeros(tuple(shape), np.int32)
    _check(load_library().pic_cell_counts(h, k, _ptr(out, C.c_int32), out.size), h)
    return out


def pic_cell_counts_noalloc(h, k, shape):
    """pic_cell_counts without device allocation (fixed in-library array of
    PIC_NOALLOC_MAX_CELLS cells; larger grids raise PicError)."""
    out = np.zeros(tuple(shape), np.int32)
    _check(load_library().pic_cell_counts_noalloc(h, k, _ptr(out, C.c_int32), out.size), h)
    return out


def pic_energy_histogram(h, k, e_max, nbins):
    """Kinetic-energy histogram of species k (uint64, nbins + 1: nbins bins
    of width e_max / nbins, then the count of E >= e_max)."""
    out = np.zeros(int(nbins) + 1, dtype=np.uint64)
    _check(load_library().pic_energy_histogram(h, int(k), float(e_max), int(nbins),
                                               _ptr(out, C.c_uint64), out.size), h)
    return out


def pic_diagnostics(h):
    d = pic_diag()
    _check(load_library().pic_diagnostics(h, C.byref(d)), h)
    n = d.nspecies
    return {"step": d.step, "time": d.time, "count": list(d.count[:n]),
            "reflections": list(d.reflections[:n]), "kinetic": list(d.kinetic[:n]),
            "field_E": d.field_E, "field_B": d.field_B, "gauss_max": d.gauss_max,
            "gauss_rms": d.gauss_rms, "rho_max": d.rho_max}


def pic_get_timing(h):
    t = pic_timing()
    _check(load_library().pic_get_timing(h, C.byref(t)), h)
    return {"particle_ms": t.particle_ms, "field_ms": t.field_ms, "sort_ms": t.sort_ms,
            "particle_launches": t.particle_launches, "field_launches": t.field_launches,
            "sort_launches": t.sort_launches, "kernel_launches": t.kernel_launches,
            "fieldb_ms": t.fieldb_ms, "fieldb_launches": t.fieldb_launches}


def pic_memory_bytes(h):
    b = C.c_size_t()
    _check(load_library().pic_memory_bytes(h, C.byref(b)), h)
    return b.value


def pic_last_error(h=None):
    m = load_library().pic_last_error(h)
    return m.decode() if m else ""


# ---------------------------------------------------------------------------
# batch engine
# ---------------------------------------------------------------------------

def pic_group_create(capacity, hbm_budget=0, stream=0, use_graph=1):
    g = C.c_void_p()
    _check(load_library().pic_group_create(int(capacity), int(hbm_budget), C.c_void_p(stream),
                                           int(use_graph), C.byref(g)))
    return g.value


def pic_group_destroy(g):
    _check(load_library().pic_group_destroy(g))


def pic_group_add(g, h, nsteps):
    _check(load_library().pic_group_add(g, h, int(nsteps)))


def pic_group_remove(g, h):
    _check(load_library().pic_group_remove(g, h))


def pic_group_step(g, nsteps):
    _check(load_library().pic_group_step(g, int(nsteps)))


def pic_group_sync(g):
    _check(load_library().pic_group_sync(g))


def pic_group_progress(g, h):
    d, l = C.c_int64(), C.c_int64()
    _check(load_library().pic_group_progress(g, h, C.byref(d), C.byref(l)))
    return d.value, l.value


def pic_group_info(g):
    m, b, n = C.c_int(), C.c_size_t(), C.c_int64()
    _check(load_library().pic_group_info(g, C.byref(m), C.byref(b), C.byref(n)))
    return {"members": m.value, "member_bytes": b.value, "launches": n.value}
