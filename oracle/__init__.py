"""FP64 CPU oracle of the nonlocal hydrodynamic FDTD method (arXiv 2005.06997).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_2005_06997_gb300``; the two meet only in the
seeded problem descriptions of ``paper_2005_06997_gb300.workloads``.

The arithmetic lives in ``oracle.c`` (plain C, FP64), written from Sec. II-III
of the paper; this module compiles it with gcc and exposes numpy views of its
arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

BC = {"pec": 0, "cpml": 1, "periodic": 2}
SHAPE = {"sphere": 1, "box": 2, "cube_tips": 3}
WAVE = {"gaussian": 1, "raised_cos": 2}


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double),
                ("courant", C.c_double), ("pml", C.c_int), ("bc", C.c_int * 3), ("eps_b", C.c_double)]


class _Material(C.Structure):
    _fields_ = [("eps_inf", C.c_double), ("wp", C.c_double), ("gamma", C.c_double),
                ("beta", C.c_double), ("diff", C.c_double), ("n_poles", C.c_int),
                ("A", C.c_double * 4), ("Om", C.c_double * 4), ("Ga", C.c_double * 4),
                ("phi", C.c_double * 4)]


class _Shape(C.Structure):
    _fields_ = [("kind", C.c_int), ("material", C.c_int), ("c", C.c_int * 3), ("radius", C.c_int),
                ("half", C.c_int * 3), ("side", C.c_int), ("tip_base", C.c_int),
                ("tip_height", C.c_int), ("tip_radius", C.c_int), ("tip_center", C.c_int),
                ("tip_cut", C.c_int)]


class _Source(C.Structure):
    _fields_ = [("enabled", C.c_int), ("tf_lo", C.c_int * 3), ("tf_hi", C.c_int * 3),
                ("waveform", C.c_int), ("w0", C.c_double), ("tau", C.c_double),
                ("t0", C.c_double), ("amp", C.c_double)]


class _Plane(C.Structure):
    _fields_ = [("axis", C.c_int), ("index", C.c_int), ("nf", C.c_int), ("omega", C.POINTER(C.c_double)),
                ("K", C.c_int)]


class _Monitors(C.Structure):
    _fields_ = [("nf", C.c_int), ("omega", C.POINTER(C.c_double)), ("abs_lo", C.c_int * 3),
                ("abs_hi", C.c_int * 3), ("sca_lo", C.c_int * 3), ("sca_hi", C.c_int * 3),
                ("K", C.c_int)]


GCC_FLAGS = ["-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
             "-ffp-contract=off"]


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, -O2, OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", *GCC_FLAGS, src, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB: a separately built copy of oracle.c (the planted-mistake
            # tests build mutated copies and check that some pin fails)
            path = os.environ.get("ORACLE_LIB") or build()
            L = C.CDLL(path)
            L.orc_create.restype = C.c_void_p
            L.orc_create.argtypes = [C.POINTER(_Grid), C.POINTER(_Material), C.c_int,
                                     C.POINTER(_Shape), C.c_int, C.c_void_p,
                                     C.POINTER(_Source), C.POINTER(_Monitors)]
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_error.restype = C.c_char_p
            L.orc_step.argtypes = [C.c_void_p, C.c_longlong]
            L.orc_time_index.restype = C.c_longlong
            L.orc_time_index.argtypes = [C.c_void_p]
            L.orc_dt.restype = C.c_double
            L.orc_dt.argtypes = [C.c_void_p]
            L.orc_array.restype = C.POINTER(C.c_double)
            L.orc_array.argtypes = [C.c_void_p, C.c_int]
            L.orc_material_map.restype = C.POINTER(C.c_uint8)
            L.orc_material_map.argtypes = [C.c_void_p, C.c_int]
            L.orc_inc_array.restype = C.POINTER(C.c_double)
            L.orc_inc_array.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int)]
            L.orc_inc_offset.restype = C.c_int
            L.orc_inc_offset.argtypes = [C.c_void_p]
            L.orc_graddiv.argtypes = [C.c_void_p, C.POINTER(C.POINTER(C.c_double)),
                                      C.POINTER(C.POINTER(C.c_double))]
            L.orc_coefficients.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_double),
                                           C.POINTER(C.c_double)]
            L.orc_num_records.restype = C.c_int
            L.orc_num_records.argtypes = [C.c_void_p]
            L.orc_records.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)]
            L.orc_dft.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.orc_spectra.argtypes = [C.c_void_p] + [C.POINTER(C.c_double)] * 4
            L.orc_set_plane.restype = C.c_int
            L.orc_set_plane.argtypes = [C.c_void_p, C.POINTER(_Plane)]
            L.orc_plane_dft.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_double)]
            L.orc_density.argtypes = [C.c_void_p, C.POINTER(C.c_double)]
            _lib = L
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


FIELDS = {"Ex": 0, "Ey": 1, "Ez": 2, "Hx": 3, "Hy": 4, "Hz": 5, "Px": 6, "Py": 7, "Pz": 8,
          "Ex_prev": 9, "Ey_prev": 10, "Ez_prev": 11, "Px_prev": 12, "Py_prev": 13, "Pz_prev": 14,
          "Pcpx": 15, "Pcpy": 16, "Pcpz": 17, "Pcpx_prev": 18, "Pcpy_prev": 19, "Pcpz_prev": 20,
          "GDx_1": 21, "GDy_1": 22, "GDz_1": 23, "GDx_2": 24, "GDy_2": 25, "GDz_2": 26}


class _SimView(np.ndarray):
    """A view of memory that an oracle simulation owns (holds it alive)."""


class Sim:
    """One oracle simulation built from a problem dict (see workloads.py)."""

    def __init__(self, prob: dict, material_map: np.ndarray | None = None):
        L = lib()
        self.prob = prob
        g = _Grid()
        g.nx, g.ny, g.nz = prob["shape"]
        g.dx = prob["dx"]
        g.courant = prob["courant"]
        g.pml = prob.get("pml", 0)
        for a, b in enumerate(prob.get("bc", ("pec",) * 3)):
            g.bc[a] = BC[b]
        g.eps_b = prob.get("eps_b", 1.0)
        mats = prob.get("materials", [])
        marr = (_Material * max(1, len(mats)))()
        for q, m in enumerate(mats):
            marr[q].eps_inf = m.get("eps_inf", 1.0)
            marr[q].wp = m.get("wp", 0.0)
            marr[q].gamma = m.get("gamma", 0.0)
            marr[q].beta = m.get("beta", 0.0)
            marr[q].diff = m.get("diff", 0.0)
            poles = m.get("poles", [])
            marr[q].n_poles = len(poles)
            for p, (A, Om, Ga, ph) in enumerate(poles):
                marr[q].A[p], marr[q].Om[p], marr[q].Ga[p], marr[q].phi[p] = A, Om, Ga, ph
        shapes = prob.get("shapes", [])
        sarr = (_Shape * max(1, len(shapes)))()
        for q, sh in enumerate(shapes):
            o = sarr[q]
            o.kind = SHAPE[sh["kind"]]
            o.material = sh["material"]
            for a in range(3):
                o.c[a] = sh["c"][a]
                o.half[a] = sh.get("half", (0, 0, 0))[a]
            o.radius = sh.get("radius", 0)
            o.side = sh.get("side", 0)
            o.tip_base = sh.get("tip_base", 0)
            o.tip_height = sh.get("tip_height", 0)
            o.tip_radius = sh.get("tip_radius", 0)
            o.tip_center = sh.get("tip_center", 0)
            o.tip_cut = sh.get("tip_cut", 0)
        src = _Source()
        s = prob.get("source")
        if s is not None:
            src.enabled = 1
            for a in range(3):
                src.tf_lo[a] = s["tf_lo"][a]
                src.tf_hi[a] = s["tf_hi"][a]
            src.waveform = WAVE[s.get("waveform", "gaussian")]
            src.w0, src.tau, src.t0, src.amp = s["w0"], s.get("tau", 0.0), s.get("t0", 0.0), s.get("amp", 1.0)
        mon = _Monitors()
        mo = prob.get("monitors")
        self._omega = None
        if mo is not None:
            self._omega = np.ascontiguousarray(mo["omega"], dtype=np.float64)
            mon.nf = len(self._omega)
            mon.omega = _dptr(self._omega)
            for a in range(3):
                mon.abs_lo[a], mon.abs_hi[a] = mo["abs_lo"][a], mo["abs_hi"][a]
                mon.sca_lo[a], mon.sca_hi[a] = mo["sca_lo"][a], mo["sca_hi"][a]
            mon.K = mo.get("K", 16)
        mp = None
        if material_map is not None:
            self._map = np.ascontiguousarray(material_map, dtype=np.uint8)
            mp = self._map.ctypes.data
        self._h = L.orc_create(C.byref(g), marr, len(mats), sarr, len(shapes), mp,
                               C.byref(src), C.byref(mon))
        if not self._h:
            raise ValueError("oracle: " + L.orc_error().decode())
        self.shape3 = (g.nz, g.ny, g.nx)
        self.ncell = g.nx * g.ny * g.nz

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- stepping -----------------------------------------------------------
    def step(self, n: int = 1):
        lib().orc_step(self._h, int(n))

    @property
    def n(self) -> int:
        return lib().orc_time_index(self._h)

    @property
    def dt(self) -> float:
        return lib().orc_dt(self._h)

    # -- state --------------------------------------------------------------
    def array(self, name: str) -> np.ndarray:
        """Writable numpy view [nz, ny, nx] of an oracle array (SI units).
        The view (and any array derived from it without a copy) keeps this
        simulation, which owns the memory, alive."""
        p = lib().orc_array(self._h, FIELDS[name])
        if not p:
            raise KeyError(name)
        v = np.ctypeslib.as_array(p, shape=(self.ncell,)).reshape(self.shape3).view(_SimView)
        v._owner = self
        return v

    def material_map(self) -> np.ndarray:
        out = np.empty((3,) + self.shape3, dtype=np.uint8)
        for c in range(3):
            p = lib().orc_material_map(self._h, c)
            out[c] = np.ctypeslib.as_array(p, shape=(self.ncell,)).reshape(self.shape3)
        return out

    def inc(self):
        n = C.c_int()
        e = lib().orc_inc_array(self._h, 0, C.byref(n))
        h = lib().orc_inc_array(self._h, 1, C.byref(n))
        if not e:
            return None, None, 0
        return (np.ctypeslib.as_array(e, shape=(n.value,)), np.ctypeslib.as_array(h, shape=(n.value,)),
                lib().orc_inc_offset(self._h))

    def graddiv(self, P):
        P = [np.ascontiguousarray(p, dtype=np.float64) for p in P]
        out = [np.zeros(self.shape3) for _ in range(3)]
        pin = (C.POINTER(C.c_double) * 3)(*[_dptr(p) for p in P])
        pout = (C.POINTER(C.c_double) * 3)(*[_dptr(o) for o in out])
        lib().orc_graddiv(self._h, pin, pout)
        return out

    def coefficients(self, material: int):
        d = np.zeros(7)
        c = np.zeros(24)
        lib().orc_coefficients(self._h, material, _dptr(d), _dptr(c))
        names = ["Dd", "D1", "D2", "D3", "DNL", "DG1", "DG2"]
        out = dict(zip(names, d))
        np_ = len(self.prob["materials"][material - 1].get("poles", []))
        out["poles"] = [dict(zip(["Cp", "C1", "C2", "C3", "C4", "C5"], c[6 * p:6 * p + 6])) for p in range(np_)]
        return out

    # -- monitors -----------------------------------------------------------
    @property
    def nrec(self) -> int:
        return lib().orc_num_records(self._h)

    def records(self):
        n = self.nrec
        rec = np.zeros((n, 10), dtype=np.int32)
        coef = np.zeros(n)
        lib().orc_records(self._h, rec.ctypes.data_as(C.POINTER(C.c_int)), _dptr(coef))
        return rec, coef

    def dft(self):
        nf = len(self._omega)
        aE = np.zeros((self.nrec + 1, nf, 2))
        aH = np.zeros((self.nrec + 1, nf, 2))
        lib().orc_dft(self._h, _dptr(aE), _dptr(aH))
        return aE, aH

    def spectra(self):
        nf = len(self._omega)
        out = [np.zeros(nf) for _ in range(4)]
        lib().orc_spectra(self._h, *[_dptr(o) for o in out])
        return dict(ext=out[0], abs=out[1], sca=out[2], inc=out[3])

    def set_plane(self, axis: int, index: int, omega, K: int):
        """Single-frequency maps on the plane normal to `axis` at node `index`
        (E_x, E_y, E_z and div P_f, running DFT every K steps)."""
        self._pl_omega = np.ascontiguousarray(omega, dtype=np.float64)
        p = _Plane(axis, index, len(self._pl_omega), _dptr(self._pl_omega), K)
        if lib().orc_set_plane(self._h, C.byref(p)) != 0:
            raise ValueError("plane monitor rejected")
        nz, ny, nx = self.shape3
        self._pl_ext = (nz, ny) if axis == 0 else ((nz, nx) if axis == 1 else (ny, nx))

    def plane_dft(self, which: int) -> np.ndarray:
        """Complex [nf][n1][n2] map: which 0..2 E_x..E_z (V/m s), 3 div P_f (C/m^3 s)."""
        n1, n2 = self._pl_ext
        out = np.zeros((len(self._pl_omega), n1, n2, 2))
        lib().orc_plane_dft(self._h, which, _dptr(out))
        return out[..., 0] + 1j * out[..., 1]

    def density(self) -> np.ndarray:
        """div P_f at every node (C/m^3), [nz][ny][nx]."""
        out = np.zeros(self.shape3)
        lib().orc_density(self._h, _dptr(out))
        return out


def run(prob: dict, steps: int | None = None, material_map=None) -> Sim:
    """Create a simulation for ``prob`` and advance it ``steps`` (default: prob['steps'])."""
    s = Sim(prob, material_map)
    s.step(prob.get("steps", 0) if steps is None else steps)
    return s
