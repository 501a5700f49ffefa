"""GB300 (sm_103a) entropic lattice Boltzmann library: Python binding.

Thin ctypes marshalling over the C ABI declared in ``include/elbm.h``; every
step of the method runs in the CUDA kernels of ``libelbm.so``.  PyTorch is
used only as plumbing: its caching allocator provides the device buffers and
its current stream orders the work.  There is no CPU fallback: importing
this package without the compiled library raises.

Usage::

    import paper_1904_00866_gb300 as elbm
    lat = elbm.Lattice("D3Q27", 128, 128, 128, nu=2.5e-3, dtype="fp32_shifted")
    lat.init_fields(rho, u)            # numpy (host) or CUDA tensors
    lat.step(100, mode="formula")
    rho, u = lat.moments()
    print(lat.entropy_stats())
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libelbm.so")

D2Q9, D3Q27, D1Q3 = 0, 1, 2
FP64, FP32, FP32_SHIFTED, FP16_SHIFTED = 0, 1, 2, 3
FORMULA, ROOT, SECANT = 0, 1, 2
LATTICES = {"D2Q9": D2Q9, "D3Q27": D3Q27, "D1Q3": D1Q3}
DTYPES = {"fp64": FP64, "fp32": FP32, "fp32_shifted": FP32_SHIFTED,
          "fp16_shifted": FP16_SHIFTED}
MODES = {"formula": FORMULA, "root": ROOT, "secant": SECANT}
Q = {D2Q9: 9, D3Q27: 27, D1Q3: 3}
DIM = {D2Q9: 2, D3Q27: 3, D1Q3: 1}

EROOT_CAP = 6
STATUS = {0: "ELBM_OK", 1: "ELBM_EINVAL", 2: "ELBM_ENOMEM", 3: "ELBM_ECUDA",
          4: "ELBM_ENONFINITE", 5: "ELBM_ENEGATIVE", 6: "ELBM_EROOT_CAP",
          7: "ELBM_ESTATE"}


class ElbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


class EntropyStats(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_longlong),
        ("n_nodes", ctypes.c_longlong),
        ("mass", ctypes.c_double),
        ("momentum", ctypes.c_double * 3),
        ("kinetic_energy", ctypes.c_double),
        ("alpha_min", ctypes.c_double),
        ("alpha_max", ctypes.c_double),
        ("alpha_sum", ctypes.c_double),
        ("n_accept_two", ctypes.c_longlong),
        ("n_accept_star", ctypes.c_longlong),
        ("n_formula", ctypes.c_longlong),
        ("n_band", ctypes.c_longlong),
        ("n_far", ctypes.c_longlong),
        ("n_degenerate", ctypes.c_longlong),
        ("n_root_iters", ctypes.c_longlong),
        ("n_root_cap", ctypes.c_longlong),
        ("n_no_root", ctypes.c_longlong),
        ("checked", ctypes.c_int),
        ("reserved", ctypes.c_int),
        ("h_total", ctypes.c_double),
        ("n_violations", ctypes.c_longlong),
        ("n_decision_mismatch", ctypes.c_longlong),
        ("alpha_dev_max", ctypes.c_double),
    ]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            if name == "reserved":
                continue
            v = getattr(self, name)
            out[name] = list(v) if name == "momentum" else v
        return out


class MemberSpec(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("nx", ctypes.c_int),
                ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("nu", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_FP = ctypes.POINTER(ctypes.c_float)
_LLP = ctypes.POINTER(ctypes.c_longlong)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

# name: (restype, argtypes) for every function of include/elbm.h
SIGNATURES = {
    "elbm_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_int]),
    "elbm_destroy": (None, [_P]),
    "elbm_last_error": (ctypes.c_char_p, [_P]),
    "elbm_set_stream": (ctypes.c_int, [_P, _P]),
    "elbm_set_allocator": (ctypes.c_int, [_P, ALLOC_FN, FREE_FN, _P]),
    "elbm_set_diagnostics": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int]),
    "elbm_init_fields": (ctypes.c_int, [_P, _DP, _DP]),
    "elbm_init_fields_device": (ctypes.c_int, [_P, _P, _P]),
    "elbm_set_populations": (ctypes.c_int, [_P, _DP]),
    "elbm_step": (ctypes.c_int, [_P, ctypes.c_longlong, ctypes.c_int]),
    "elbm_sync": (ctypes.c_int, [_P]),
    "elbm_moments": (ctypes.c_int, [_P, _DP, _DP]),
    "elbm_get_populations": (ctypes.c_int, [_P, _DP]),
    "elbm_get_populations_nodes": (ctypes.c_int, [_P, _LLP, ctypes.c_int,
                                                  _DP]),
    "elbm_alpha_map": (ctypes.c_int, [_P, _FP]),
    "elbm_entropy_stats": (ctypes.c_int, [_P, ctypes.POINTER(EntropyStats)]),
    "elbm_enstrophy": (ctypes.c_int, [_P, _DP]),
    "elbm_step_count": (ctypes.c_longlong, [_P]),
    "elbm_device_bytes": (ctypes.c_size_t, [_P]),
    "elbm_launch_count": (ctypes.c_longlong, []),
    "elbm_rho0": (ctypes.c_double, [_P]),
    "elbm_beta": (ctypes.c_double, [_P]),
    "elbm_set_decision": (ctypes.c_int, [_P, ctypes.c_int]),
    "elbm_step_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double, _P,
                                        _P, _P, _P,
                                        ctypes.POINTER(EntropyStats)]),
    "elbm_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int]),
    "elbm_batch_destroy": (None, [_P]),
    "elbm_batch_last_error": (ctypes.c_char_p, [_P]),
    "elbm_batch_set_stream": (ctypes.c_int, [_P, _P]),
    "elbm_batch_set_allocator": (ctypes.c_int, [_P, ALLOC_FN, FREE_FN, _P]),
    "elbm_batch_set_options": (ctypes.c_int, [_P] + [ctypes.c_int] * 4),
    "elbm_batch_add": (ctypes.c_int, [_P, ctypes.POINTER(MemberSpec), _DP,
                                      _DP, ctypes.POINTER(ctypes.c_int)]),
    "elbm_batch_remove": (ctypes.c_int, [_P, ctypes.c_int]),
    "elbm_batch_set_steps": (ctypes.c_int, [_P, ctypes.c_int,
                                            ctypes.c_longlong]),
    "elbm_batch_member_info": (ctypes.c_int, [_P, ctypes.c_int, _LLP, _LLP]),
    "elbm_batch_record_alpha": (ctypes.c_int, [_P, ctypes.c_int,
                                               ctypes.c_int]),
    "elbm_batch_step": (ctypes.c_int, [_P, ctypes.c_longlong]),
    "elbm_batch_sync": (ctypes.c_int, [_P]),
    "elbm_batch_moments": (ctypes.c_int, [_P, ctypes.c_int, _DP, _DP]),
    "elbm_batch_get_populations": (ctypes.c_int, [_P, ctypes.c_int, _DP]),
    "elbm_batch_alpha_map": (ctypes.c_int, [_P, ctypes.c_int, _FP]),
    "elbm_batch_entropy_stats": (ctypes.c_int, [_P, ctypes.c_int,
                                                ctypes.POINTER(EntropyStats)]),
    "elbm_batch_set_decision": (ctypes.c_int, [_P, ctypes.c_int]),
    "elbm_batch_tuning": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int)]),
    "elbm_batch_device_bytes": (ctypes.c_size_t, [_P]),
    "elbm_set_profiling": (ctypes.c_int, [_P, ctypes.c_int]),
    "elbm_profile": (ctypes.c_int, [_P, _DP, _LLP]),
}


def lib():
    """Load libelbm.so (raises when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            "libelbm.so is missing: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` "
            "(the library has no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def launch_count():
    """Kernel launches issued by the library so far (all handles)."""
    return lib().elbm_launch_count()


def _dptr(a):
    return a.ctypes.data_as(_DP)


def _torch_cuda():
    try:
        import torch
    except ImportError:
        return None
    return torch if torch.cuda.is_available() else None


class Lattice:
    """One periodic lattice advanced on the GPU.

    lattice: "D2Q9" | "D3Q27" | "D1Q3" (FP64 only); dtype: "fp64" | "fp32" |
    "fp32_shifted" | "fp16_shifted";
    allocator: "torch" (PyTorch caching allocator, the default when PyTorch
    sees a GPU) or "cuda" (cudaMalloc inside the library).
    """

    def __init__(self, lattice, nx, ny, nz=1, nu=1e-2, dtype="fp32_shifted",
                 allocator=None, stream=None):
        L = lib()
        self.lattice = LATTICES[lattice] if isinstance(lattice, str) else int(
            lattice)
        self.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.q = Q[self.lattice]
        self.d = DIM[self.lattice]
        self.nu = float(nu)
        h = _P()
        st = L.elbm_create(ctypes.byref(h), self.lattice, self.nx, self.ny,
                           self.nz, self.nu, self.dtype)
        if st:
            raise ElbmError(st, L.elbm_last_error(None).decode())
        self._h = h
        torch = _torch_cuda()
        if allocator is None:
            allocator = "torch" if torch is not None else "cuda"
        self._cb = None
        if allocator == "torch":
            if torch is None:
                raise RuntimeError("allocator='torch' needs a CUDA PyTorch")
            dev = torch.cuda.current_device()

            def _alloc(size, ctx):
                try:
                    return torch.cuda.caching_allocator_alloc(int(size), dev)
                except Exception:
                    return None

            def _free(ptr, ctx):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._cb = (ALLOC_FN(_alloc), FREE_FN(_free))
            self._check(L.elbm_set_allocator(h, self._cb[0], self._cb[1],
                                             None))
        if stream is None and torch is not None:
            stream = torch.cuda.current_stream().cuda_stream
        if stream is not None:
            self._check(L.elbm_set_stream(h, _P(int(stream))))

    # -- helpers -----------------------------------------------------------
    def _check(self, st):
        if st:
            raise ElbmError(st, lib().elbm_last_error(self._h).decode())

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def close(self):
        if getattr(self, "_h", None):
            lib().elbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- API ---------------------------------------------------------------
    def set_diagnostics(self, diag_every=1, check_every=0, alpha_map_every=0,
                        secant_iters=4):
        self._check(lib().elbm_set_diagnostics(self._h, int(diag_every),
                                               int(check_every),
                                               int(alpha_map_every),
                                               int(secant_iters)))

    def init_fields(self, rho, u):
        """f^0 = f^eq(rho, u).  numpy arrays (host) or CUDA float64 tensors
        (device); rho (nz, ny, nx), u (d, nz, ny, nx)."""
        if hasattr(rho, "is_cuda") and rho.is_cuda:
            r = rho.contiguous()
            v = u.contiguous()
            assert r.dtype == v.dtype and str(r.dtype) == "torch.float64"
            assert r.numel() == self.n and v.numel() == self.d * self.n
            self._check(lib().elbm_init_fields_device(
                self._h, _P(r.data_ptr()), _P(v.data_ptr())))
            return
        r = np.ascontiguousarray(np.broadcast_to(rho, self.shape),
                                 dtype=np.float64)
        v = np.ascontiguousarray(u, dtype=np.float64)
        if v.size != self.d * self.n:
            raise ValueError("u must have d * nx * ny * nz entries")
        self._check(lib().elbm_init_fields(self._h, _dptr(r), _dptr(v)))

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        if f.size != self.q * self.n:
            raise ValueError("f must have Q * nx * ny * nz entries")
        self._check(lib().elbm_set_populations(self._h, _dptr(f)))

    def set_decision(self, decision="exact"):
        """'exact' (default): undecided FP32 entropy tests are retaken in
        double-float arithmetic; 'certified': they keep the certified
        alpha."""
        d = {"exact": 0, "certified": 1}[decision]
        self._check(lib().elbm_set_decision(self._h, d))

    def set_stream(self, stream):
        self._check(lib().elbm_set_stream(self._h, _P(int(stream))))

    def step(self, nsteps=1, mode="formula"):
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        self._check(lib().elbm_step(self._h, int(nsteps), m))

    def sync(self):
        self._check(lib().elbm_sync(self._h))

    def moments(self):
        rho = np.empty(self.shape)
        u = np.empty((self.d,) + self.shape)
        self._check(lib().elbm_moments(self._h, _dptr(rho), _dptr(u)))
        return rho, u

    def populations(self):
        f = np.empty((self.q,) + self.shape)
        self._check(lib().elbm_get_populations(self._h, _dptr(f)))
        return f

    def populations_at(self, nodes):
        nodes = np.ascontiguousarray(nodes, dtype=np.int64)
        out = np.empty((len(nodes), self.q))
        self._check(lib().elbm_get_populations_nodes(
            self._h, nodes.ctypes.data_as(_LLP), len(nodes), _dptr(out)))
        return out

    def alpha_map(self):
        a = np.empty(self.shape, dtype=np.float32)
        self._check(lib().elbm_alpha_map(self._h, a.ctypes.data_as(_FP)))
        return a

    def entropy_stats(self):
        """Statistics of the last diagnostic step.  A step where ROOT
        bisection hit its iteration cap still returns its statistics (with
        n_root_cap > 0) and raises a RuntimeWarning."""
        s = EntropyStats()
        st = lib().elbm_entropy_stats(self._h, ctypes.byref(s))
        if st == EROOT_CAP:
            import warnings
            warnings.warn(lib().elbm_last_error(self._h).decode(),
                          RuntimeWarning)
        else:
            self._check(st)
        return s.as_dict()

    def enstrophy(self):
        out = ctypes.c_double()
        self._check(lib().elbm_enstrophy(self._h, ctypes.byref(out)))
        return out.value

    def set_profiling(self, enable=True):
        self._check(lib().elbm_set_profiling(self._h, int(bool(enable))))

    def profile(self):
        """(total ms, launches) of the stream-collide kernels recorded since
        the last call."""
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        self._check(lib().elbm_profile(self._h, ctypes.byref(ms),
                                       ctypes.byref(n)))
        return ms.value, n.value

    @property
    def step_count(self):
        return lib().elbm_step_count(self._h)

    @property
    def device_bytes(self):
        return lib().elbm_device_bytes(self._h)

    @property
    def rho0(self):
        return lib().elbm_rho0(self._h)

    @property
    def beta(self):
        """The relaxation factor beta the library steps with."""
        return lib().elbm_beta(self._h)


class Batch:
    """Many independent periodic lattices (FP32-shifted storage, FORMULA
    alpha) advanced together by the batched persistent kernel.

    Members are added with ``add(lattice, nx, ny, nz, nu, rho, u)`` and get
    an integer id; ``step(n)`` advances every member that still has steps
    (``set_steps(id, k)`` limits a member to k more steps).
    """

    def __init__(self, max_members=256, burst=16, use_graphs=True,
                 autotune=True, diag_every=0, allocator=None, stream=None):
        L = lib()
        h = _P()
        st = L.elbm_batch_create(ctypes.byref(h), int(max_members))
        if st:
            raise ElbmError(st, L.elbm_last_error(None).decode())
        self._h = h
        torch = _torch_cuda()
        if allocator is None:
            allocator = "torch" if torch is not None else "cuda"
        self._cb = None
        if allocator == "torch":
            dev = torch.cuda.current_device()

            def _alloc(size, ctx):
                try:
                    return torch.cuda.caching_allocator_alloc(int(size), dev)
                except Exception:
                    return None

            def _free(ptr, ctx):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._cb = (ALLOC_FN(_alloc), FREE_FN(_free))
            self._check(L.elbm_batch_set_allocator(h, self._cb[0],
                                                   self._cb[1], None))
        if stream is None and torch is not None:
            stream = torch.cuda.current_stream().cuda_stream
        if stream is not None:
            self._check(L.elbm_batch_set_stream(h, _P(int(stream))))
        self.set_options(diag_every, burst, use_graphs, autotune)
        self.members = {}

    def _check(self, st):
        if st:
            raise ElbmError(st, lib().elbm_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().elbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, diag_every=0, burst=16, use_graphs=True,
                    autotune=True):
        self._check(lib().elbm_batch_set_options(
            self._h, int(diag_every), int(burst), int(bool(use_graphs)),
            int(bool(autotune))))

    def set_decision(self, decision="exact"):
        """As Lattice.set_decision, for every member."""
        d = {"exact": 0, "certified": 1}[decision]
        self._check(lib().elbm_batch_set_decision(self._h, d))

    def add(self, lattice, nx, ny, nz, nu, rho, u):
        lat = LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
        spec = MemberSpec(lat, int(nx), int(ny), int(nz), float(nu))
        shape = (int(nz), int(ny), int(nx))
        r = np.ascontiguousarray(np.broadcast_to(rho, shape), dtype=np.float64)
        v = np.ascontiguousarray(u, dtype=np.float64)
        mid = ctypes.c_int()
        self._check(lib().elbm_batch_add(self._h, ctypes.byref(spec),
                                         _dptr(r), _dptr(v),
                                         ctypes.byref(mid)))
        self.members[mid.value] = (lat, shape)
        return mid.value

    def remove(self, mid):
        self._check(lib().elbm_batch_remove(self._h, int(mid)))
        self.members.pop(mid, None)

    def set_steps(self, mid, remaining):
        self._check(lib().elbm_batch_set_steps(self._h, int(mid),
                                               int(remaining)))

    def info(self, mid):
        done = ctypes.c_longlong()
        rem = ctypes.c_longlong()
        self._check(lib().elbm_batch_member_info(
            self._h, int(mid), ctypes.byref(done), ctypes.byref(rem)))
        return done.value, rem.value

    def record_alpha(self, mid, enable=True):
        self._check(lib().elbm_batch_record_alpha(self._h, int(mid),
                                                  int(bool(enable))))

    def step(self, nsteps):
        self._check(lib().elbm_batch_step(self._h, int(nsteps)))

    def sync(self):
        self._check(lib().elbm_batch_sync(self._h))

    def moments(self, mid):
        lat, shape = self.members[mid]
        rho = np.empty(shape)
        u = np.empty((DIM[lat],) + shape)
        self._check(lib().elbm_batch_moments(self._h, int(mid), _dptr(rho),
                                             _dptr(u)))
        return rho, u

    def populations(self, mid):
        lat, shape = self.members[mid]
        f = np.empty((Q[lat],) + shape)
        self._check(lib().elbm_batch_get_populations(self._h, int(mid),
                                                     _dptr(f)))
        return f

    def alpha_map(self, mid):
        lat, shape = self.members[mid]
        a = np.empty(shape, dtype=np.float32)
        self._check(lib().elbm_batch_alpha_map(self._h, int(mid),
                                               a.ctypes.data_as(_FP)))
        return a

    def entropy_stats(self, mid):
        s = EntropyStats()
        self._check(lib().elbm_batch_entropy_stats(self._h, int(mid),
                                                   ctypes.byref(s)))
        return s.as_dict()

    def tuning(self):
        t, b, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(lib().elbm_batch_tuning(self._h, ctypes.byref(t),
                                            ctypes.byref(b), ctypes.byref(k)))
        return {"threads": t.value, "blocks_per_sm": b.value,
                "burst": k.value}

    @property
    def device_bytes(self):
        return lib().elbm_batch_device_bytes(self._h)
