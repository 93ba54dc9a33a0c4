"""Python binding of the C ABI in ``include/pic.h`` (argument marshalling only).

Every step of the PIC method runs in the CUDA kernels of ``libpic.so``; this
module only converts numpy arrays to pointers and error codes to exceptions.
There is no CPU fallback: when the library is missing or no GPU is present,
calls raise :class:`PicError`.

Names follow the C ABI: :func:`pic_create`, :meth:`Sim.pic_load_particles`,
:meth:`Sim.pic_step`, :meth:`Sim.pic_fields`, :meth:`Sim.pic_diagnostics` ...
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpic.so")

PIC_OK = 0
ERRORS = {-1: "PIC_ERR_ARG", -2: "PIC_ERR_CFL", -3: "PIC_ERR_CUDA", -4: "PIC_ERR_CAPACITY",
          -5: "PIC_ERR_NONFINITE", -6: "PIC_ERR_NOMEM", -7: "PIC_ERR_STATE", -8: "PIC_ERR_TIMEOUT"}
PERIODIC, ABSORB = 0, 1
FP32_CELLOFF, FP64_PLAIN = 0, 1
PUSH_AUTO, PUSH_SIMPLE, PUSH_MLP_TC, PUSH_TILE_AGG = 0, 1, 2, 3
PUSHER_BORIS, PUSHER_VAY = 0, 1
EX, EY, EZ, BX, BY, BZ, JX, JY, JZ, RHO = range(10)
MAX_SPECIES = 8

# every symbol include/pic.h declares
EXPORTS = ["pic_create", "pic_destroy", "pic_last_error", "pic_load_particles", "pic_set_laser",
           "pic_set_field", "pic_step", "pic_fields", "pic_particle_count", "pic_get_particles",
           "pic_get_cells", "pic_diagnostics", "pic_gather", "pic_sync", "pic_profile", "pic_profile_read",
           "pic_field_energy_noalloc", "pic_set_qed", "pic_qed_eval", "pic_get_qed_state", "pic_mlp_train",
           "pic_mlp_validate", "pic_mlp_get", "pic_mlp_set", "pic_mlp_eval", "pic_mlp_eval_tc", "pic_mlp_grad",
           "pic_field_device", "pic_save", "pic_restore", "pic_profile_read_species", "pic_measure_ceilings"]
KIND_MASSIVE, KIND_PHOTON = 0, 1
QED_OFF, QED_TABLE, QED_SURROGATE = 0, 1, 2
MLP_NPARAMS = 8642
QED_EMISSION, QED_PAIR = 0, 1
PHASES = ("sort", "fields", "push", "fold")


class PicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class pic_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int64 * 3), ("dx", C.c_double * 3), ("bc", C.c_int * 3),
                ("order", C.c_int)]


class pic_species(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("w", C.c_double), ("capacity", C.c_int64),
                ("kind", C.c_int), ("qed", C.c_int)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class pic_options(C.Structure):
    _fields_ = [("struct_size", C.c_int), ("precision", C.c_int), ("sort_interval", C.c_int),
                ("tile", C.c_int * 3), ("rho_bg", C.c_double), ("stream", C.c_void_p), ("push_variant", C.c_int),
                ("seed", C.c_uint64), ("pusher", C.c_int), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", C.c_void_p)]


class pic_field_view(C.Structure):
    _fields_ = [("data", C.c_void_p), ("elem_bytes", C.c_int), ("origin", C.c_int64), ("stride", C.c_int64 * 3),
                ("lo", C.c_int64 * 3), ("hi", C.c_int64 * 3)]


class pic_qed(C.Structure):
    _fields_ = [("mode", C.c_int), ("photon_sp", C.c_int), ("electron_sp", C.c_int), ("positron_sp", C.c_int),
                ("lambda_r_m", C.c_double), ("photon_emin", C.c_double), ("method", C.c_int)]


class pic_laser(C.Structure):
    _fields_ = [("a0", C.c_double), ("waist", C.c_double), ("fwhm", C.c_double), ("t_peak", C.c_double),
                ("x_focus", C.c_double), ("yc", C.c_double), ("zc", C.c_double), ("pol", C.c_int)]


class pic_diag(C.Structure):
    _fields_ = [("step", C.c_int64), ("t", C.c_double), ("U_E", C.c_double), ("U_B", C.c_double),
                ("U_kin", C.c_double * MAX_SPECIES), ("charge", C.c_double), ("gauss_max", C.c_double),
                ("E_absorbed", C.c_double), ("n_alive", C.c_int64 * MAX_SPECIES), ("E_photon_lost", C.c_double)]


class pic_mlp_train_opts(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("batch", C.c_int64), ("lr", C.c_double), ("lr_final", C.c_double),
                ("chi_min", C.c_double), ("chi_max", C.c_double), ("rate_weight", C.c_double),
                ("seed", C.c_uint64), ("keep", C.c_int)]


class pic_mlp_report(C.Structure):
    _fields_ = [("loss", C.c_double), ("max_err_lnG", C.c_double), ("max_err_s", C.c_double),
                ("rms_err_s", C.c_double), ("ms", C.c_double), ("iterations", C.c_int64),
                ("table_bytes", C.c_int64), ("net_bytes", C.c_int64), ("max_err_mean", C.c_double)]


class pic_mlp_info(C.Structure):
    _fields_ = [("chi_min", C.c_double), ("chi_max", C.c_double), ("mu", C.c_double), ("sd", C.c_double)]


def _report(r):
    return {k: getattr(r, k) for k, _ in pic_mlp_report._fields_}


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libpic.so (it must have been built: see ``build.py``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise PicError(-3, f"{path} is not built (run paper_2104_00642_gb300/build.py)")
    L = C.CDLL(path)
    P, I, D, I64 = C.c_void_p, C.c_int, C.c_double, C.c_int64
    L.pic_create.argtypes = [C.POINTER(pic_grid), D, C.POINTER(pic_species), I, C.POINTER(pic_options),
                             C.POINTER(P)]
    L.pic_create.restype = I
    L.pic_destroy.argtypes = [P]
    L.pic_destroy.restype = None
    L.pic_last_error.argtypes = [P]
    L.pic_last_error.restype = C.c_char_p
    L.pic_load_particles.argtypes = [P, I, I64, P, P, P, P, P, P]
    L.pic_load_particles.restype = I
    L.pic_set_laser.argtypes = [P, C.POINTER(pic_laser)]
    L.pic_set_laser.restype = I
    L.pic_set_field.argtypes = [P, I, P]
    L.pic_set_field.restype = I
    L.pic_step.argtypes = [P, I64]
    L.pic_step.restype = I
    L.pic_fields.argtypes = [P, I, P]
    L.pic_fields.restype = I
    L.pic_particle_count.argtypes = [P, I]
    L.pic_particle_count.restype = I64
    L.pic_get_particles.argtypes = [P, I, I64, C.POINTER(I64), P, P, P, P, P, P, P]
    L.pic_get_particles.restype = I
    L.pic_get_cells.argtypes = [P, I, I64, P, P]
    L.pic_get_cells.restype = I
    L.pic_diagnostics.argtypes = [P, C.POINTER(pic_diag)]
    L.pic_diagnostics.restype = I
    L.pic_gather.argtypes = [P, I, I64, P]
    L.pic_gather.restype = I
    L.pic_sync.argtypes = [P]
    L.pic_sync.restype = I
    L.pic_profile.argtypes = [P, I]
    L.pic_profile.restype = I
    L.pic_profile_read.argtypes = [P, P, P, P]
    L.pic_profile_read.restype = I
    L.pic_field_energy_noalloc.argtypes = [C.POINTER(C.c_void_p), I64, D, P, P]
    L.pic_field_energy_noalloc.restype = I
    L.pic_set_qed.argtypes = [P, C.POINTER(pic_qed)]
    L.pic_set_qed.restype = I
    L.pic_qed_eval.argtypes = [P, I, I64, P, P, P]
    L.pic_qed_eval.restype = I
    L.pic_get_qed_state.argtypes = [P, I, I64, P, P]
    L.pic_get_qed_state.restype = I
    L.pic_mlp_train.argtypes = [P, I, C.POINTER(pic_mlp_train_opts), C.POINTER(pic_mlp_report)]
    L.pic_mlp_validate.argtypes = [P, I, C.POINTER(pic_mlp_report)]
    L.pic_mlp_get.argtypes = [P, I, P, C.POINTER(pic_mlp_info)]
    L.pic_mlp_set.argtypes = [P, I, P, C.POINTER(pic_mlp_info)]
    L.pic_mlp_eval.argtypes = [P, I, I64, P, P]
    L.pic_mlp_eval_tc.argtypes = [P, I, I64, P, P]
    L.pic_mlp_grad.argtypes = [P, I, I64, P, P, P, C.POINTER(D)]
    L.pic_field_device.argtypes = [P, I, C.POINTER(pic_field_view)]
    L.pic_profile_read_species.argtypes = [P, P, P]
    L.pic_save.argtypes = [P, C.c_char_p]
    L.pic_measure_ceilings.argtypes = [P]
    L.pic_measure_ceilings.restype = I
    L.pic_restore.argtypes = [P, C.c_char_p]
    for name in ("pic_mlp_train", "pic_mlp_validate", "pic_mlp_get", "pic_mlp_set", "pic_mlp_eval", "pic_mlp_eval_tc",
                 "pic_mlp_grad", "pic_field_device", "pic_save", "pic_restore", "pic_profile_read_species"):
        getattr(L, name).restype = I
    _lib = L
    return L


def pic_measure_ceilings():
    """throughput ceilings of the push kernels' instruction mixes on the
    current device (see include/pic.h): dict of per-second rates"""
    L = load_library()
    out = np.zeros(5)
    rc = L.pic_measure_ceilings(_p(out))
    if rc:
        raise PicError(rc, L.pic_last_error(None).decode())
    return {"fp32_flops": out[0], "fp64_flops": out[1], "shared_atomics_distinct": out[2],
            "shared_atomics_same_word": out[3], "warp_reduce_then_atomic_values": out[4]}


def pic_field_energy_noalloc(dev_fields, n, dV, dev_out2, stream=None):
    """Field energy of six caller-owned device FP64 arrays (Ex..Bz) into two
    device doubles, for callers that cannot allocate device memory: the
    library allocates nothing for this call (its scratch is a static device
    array).  Arguments are raw device addresses (ints)."""
    L = load_library()
    ptrs = (C.c_void_p * 6)(*[C.c_void_p(int(p)) for p in dev_fields])
    rc = L.pic_field_energy_noalloc(ptrs, int(n), float(dV), C.c_void_p(int(dev_out2)),
                                    None if stream is None else C.c_void_p(int(stream)))
    if rc != PIC_OK:
        raise PicError(rc, L.pic_last_error(None).decode())


class TorchAllocator:
    """Device memory for a simulation from PyTorch's caching allocator
    (pic_options.alloc/free): the library's blocks then live in the same pool
    as the caller's tensors.  Counts the blocks handed out and returned."""

    def __init__(self, device=None):
        import torch
        self._torch = torch
        self.device = torch.cuda.current_device() if device is None else device
        self.allocated = 0
        self.freed = 0
        self.live = {}
        self.errors = []  # exceptions the callbacks caught (the library sees a refusal)
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)

    def _do_alloc(self, ctx, nbytes, stream):
        try:
            ptr = self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream=int(stream or 0))
        except Exception as e:  # e.g. out of memory: the library reports PIC_ERR_NOMEM
            self.errors.append(repr(e))
            return None
        self.allocated += 1
        self.live[int(ptr)] = int(nbytes)
        return ptr

    def _do_free(self, ctx, ptr, stream):
        self._torch.cuda.caching_allocator_delete(int(ptr))
        self.live.pop(int(ptr), None)
        self.freed += 1


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class Sim:
    """One simulation (a ``pic_sim*``)."""

    def __init__(self, dim, n, dx, dt, species, bc=(PERIODIC, PERIODIC, PERIODIC), precision=FP32_CELLOFF,
                 sort_interval=0, tile=(0, 0, 0), rho_bg=0.0, stream=None, push_variant=0, seed=0, pusher=0,
                 allocator=None, order=2):
        L = load_library()
        g = pic_grid()
        g.dim = int(dim)
        for d in range(3):
            g.n[d] = int(n[d]) if d < len(n) else 1
            g.dx[d] = float(dx[d]) if d < len(dx) else 1.0
            g.bc[d] = int(bc[d]) if d < len(bc) else PERIODIC
        g.order = int(order)
        sp = (pic_species * max(1, len(species)))()
        for i, s in enumerate(species):
            sp[i].q, sp[i].m, sp[i].w, sp[i].capacity = float(s[0]), float(s[1]), float(s[2]), int(s[3])
            sp[i].kind = int(s[4]) if len(s) > 4 else KIND_MASSIVE
            sp[i].qed = int(s[5]) if len(s) > 5 else 0
        o = pic_options()
        o.struct_size = C.sizeof(pic_options)
        o.precision = int(precision)
        o.sort_interval = int(sort_interval)
        for d in range(3):
            o.tile[d] = int(tile[d]) if d < len(tile) else 0
        o.rho_bg = float(rho_bg)
        o.stream = stream
        o.push_variant = int(push_variant)
        o.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        o.pusher = int(pusher)
        self.allocator = allocator  # the callbacks must outlive the simulation
        if allocator is not None:
            o.alloc = allocator._alloc
            o.free = allocator._free
        h = C.c_void_p()
        rc = L.pic_create(C.byref(g), float(dt), sp, len(species), C.byref(o), C.byref(h))
        if rc != PIC_OK:
            raise PicError(rc, L.pic_last_error(None).decode())
        self._h = h
        self.dim = int(dim)
        self.n = [int(g.n[d]) for d in range(3)]
        self.bc = [int(g.bc[d]) for d in range(3)]
        self.dt = float(dt)
        self.nsp = len(species)
        self.precision = precision

    # -- lifetime ---------------------------------------------------------
    def close(self):
        h = getattr(self, "_h", None)
        if h:
            load_library().pic_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc):
        if rc != PIC_OK:
            raise PicError(rc, load_library().pic_last_error(self._h).decode())

    # -- C ABI --------------------------------------------------------------
    def box(self):
        m = [1, 1, 1]
        for d in range(self.dim):
            m[d] = self.n[d] + (1 if self.bc[d] == ABSORB else 0)
        return (m[2], m[1], m[0])

    def pic_load_particles(self, sp, x, y, z, ux, uy, uz):
        arrs = [_f64(a) for a in (x, y, z, ux, uy, uz)]
        n = len(arrs[3])
        self._check(load_library().pic_load_particles(self._h, int(sp), n, *[_p(a) for a in arrs]))

    def pic_set_laser(self, a0, waist, fwhm, t_peak, x_focus, yc=0.0, zc=0.0, pol=0):
        lz = pic_laser(a0, waist, fwhm, t_peak, x_focus, yc, zc, pol)
        self._check(load_library().pic_set_laser(self._h, C.byref(lz)))

    def pic_set_field(self, comp, arr):
        a = _f64(np.broadcast_to(arr, self.box()))
        self._check(load_library().pic_set_field(self._h, int(comp), _p(a)))

    def pic_step(self, nsteps=1):
        self._check(load_library().pic_step(self._h, int(nsteps)))

    def pic_fields(self, comp):
        out = np.zeros(self.box())
        self._check(load_library().pic_fields(self._h, int(comp), _p(out)))
        return out

    def pic_field_device(self, comp):
        """borrowed device view of a resident component: dict with the device
        address, element size, origin and strides (elements), index range"""
        v = pic_field_view()
        self._check(load_library().pic_field_device(self._h, int(comp), C.byref(v)))
        return {"data": int(v.data or 0), "elem_bytes": v.elem_bytes, "origin": v.origin, "stride": tuple(v.stride),
                "lo": tuple(v.lo), "hi": tuple(v.hi)}

    def pic_profile_read_species(self):
        """per-species push time (ms) and push count gathered by the last
        pic_profile_read"""
        ms = np.zeros(max(self.nsp, 1))
        n = np.zeros(max(self.nsp, 1), dtype=np.int64)
        self._check(load_library().pic_profile_read_species(self._h, _p(ms), _p(n)))
        return ms[: self.nsp].tolist(), n[: self.nsp].tolist()

    def pic_save(self, path):
        self._check(load_library().pic_save(self._h, os.fsencode(path)))

    def pic_restore(self, path):
        self._check(load_library().pic_restore(self._h, os.fsencode(path)))

    def pic_particle_count(self, sp):
        n = load_library().pic_particle_count(self._h, int(sp))
        if n < 0:
            self._check(-1)
        return n

    def pic_get_particles(self, sp):
        n = self.pic_particle_count(sp)
        out = {k: np.zeros(n) for k in ("x", "y", "z", "ux", "uy", "uz")}
        alive = np.zeros(n, dtype=np.uint8)
        nn = C.c_int64()
        self._check(load_library().pic_get_particles(self._h, int(sp), n, C.byref(nn),
                                                     *[_p(out[k]) for k in ("x", "y", "z", "ux", "uy", "uz")],
                                                     _p(alive)))
        out["alive"] = alive
        return out

    def pic_get_cells(self, sp):
        n = self.pic_particle_count(sp)
        cells = np.zeros(n, dtype=np.uint32)
        bits = (C.c_int * 3)()
        self._check(load_library().pic_get_cells(self._h, int(sp), n, _p(cells), bits))
        return cells, tuple(bits)

    def pic_gather(self, sp):
        n = self.pic_particle_count(sp)
        out = np.zeros((n, 6))
        self._check(load_library().pic_gather(self._h, int(sp), n, _p(out)))
        return out

    def pic_diagnostics(self):
        d = pic_diag()
        self._check(load_library().pic_diagnostics(self._h, C.byref(d)))
        return {"step": d.step, "t": d.t, "U_E": d.U_E, "U_B": d.U_B, "U_kin": list(d.U_kin[: self.nsp]),
                "charge": d.charge, "gauss_max": d.gauss_max, "E_absorbed": d.E_absorbed,
                "n_alive": list(d.n_alive[: self.nsp]), "E_photon_lost": d.E_photon_lost}

    def pic_set_qed(self, photon_sp=-1, electron_sp=-1, positron_sp=-1, lambda_r_m=1e-6, photon_emin=0.0,
                    mode=QED_TABLE, method=1):
        q = pic_qed(int(mode), int(photon_sp), int(electron_sp), int(positron_sp), float(lambda_r_m),
                    float(photon_emin), int(method))
        self._check(load_library().pic_set_qed(self._h, C.byref(q)))

    def pic_qed_eval(self, process, chi, r=None):
        chi = _f64(np.atleast_1d(chi))
        rr = None if r is None else _f64(np.atleast_1d(r))
        out = np.zeros(len(chi))
        self._check(load_library().pic_qed_eval(self._h, int(process), len(chi), _p(chi), _p(rr), _p(out)))
        return out

    def pic_mlp_train(self, process, iterations=0, batch=0, lr=0.0, lr_final=0.0, chi_min=0.0, chi_max=0.0,
                      rate_weight=0.0, seed=0, keep=False):
        o = pic_mlp_train_opts(int(iterations), int(batch), float(lr), float(lr_final), float(chi_min),
                               float(chi_max), float(rate_weight), int(seed) & 0xFFFFFFFFFFFFFFFF, int(bool(keep)))
        r = pic_mlp_report()
        self._check(load_library().pic_mlp_train(self._h, int(process), C.byref(o), C.byref(r)))
        return _report(r)

    def pic_mlp_validate(self, process):
        r = pic_mlp_report()
        self._check(load_library().pic_mlp_validate(self._h, int(process), C.byref(r)))
        return _report(r)

    def pic_mlp_get(self, process):
        P = np.zeros(MLP_NPARAMS, dtype=np.float32)
        info = pic_mlp_info()
        self._check(load_library().pic_mlp_get(self._h, int(process), _p(P), C.byref(info)))
        return P, {k: getattr(info, k) for k, _ in pic_mlp_info._fields_}

    def pic_mlp_set(self, process, params, chi_min, chi_max, mu, sd):
        P = np.ascontiguousarray(params, dtype=np.float32)
        if P.size != MLP_NPARAMS:
            raise ValueError("pic_mlp_set: wrong parameter count")
        info = pic_mlp_info(float(chi_min), float(chi_max), float(mu), float(sd))
        self._check(load_library().pic_mlp_set(self._h, int(process), _p(P), C.byref(info)))

    def pic_mlp_eval(self, process, x):
        X = np.ascontiguousarray(np.asarray(x, dtype=np.float32).reshape(-1, 2))
        Y = np.zeros_like(X)
        self._check(load_library().pic_mlp_eval(self._h, int(process), X.shape[0], _p(X), _p(Y)))
        return Y

    def pic_mlp_eval_tc(self, process, x):
        X = np.ascontiguousarray(np.asarray(x, dtype=np.float32).reshape(-1, 2))
        Y = np.zeros_like(X)
        self._check(load_library().pic_mlp_eval_tc(self._h, int(process), X.shape[0], _p(X), _p(Y)))
        return Y

    def pic_mlp_grad(self, process, x, t):
        X = np.ascontiguousarray(np.asarray(x, dtype=np.float32).reshape(-1, 2))
        T = np.ascontiguousarray(np.asarray(t, dtype=np.float32).reshape(-1, 2))
        G = np.zeros(MLP_NPARAMS, dtype=np.float32)
        loss = C.c_double(0.0)
        self._check(load_library().pic_mlp_grad(self._h, int(process), X.shape[0], _p(X), _p(T), _p(G),
                                                C.byref(loss)))
        return loss.value, G

    def pic_get_qed_state(self, sp):
        n = self.pic_particle_count(sp)
        ids = np.zeros(max(n, 1), dtype=np.uint64)
        tau = np.zeros(max(n, 1))
        self._check(load_library().pic_get_qed_state(self._h, int(sp), n, _p(ids), _p(tau)))
        return ids[:n], tau[:n]

    def pic_sync(self):
        self._check(load_library().pic_sync(self._h))

    def pic_profile(self, enable=True):
        self._check(load_library().pic_profile(self._h, int(bool(enable))))

    def pic_profile_read(self):
        ms = np.zeros(len(PHASES))
        ln = np.zeros(len(PHASES), dtype=np.int64)
        pl = C.c_int64()
        self._check(load_library().pic_profile_read(self._h, _p(ms), _p(ln), C.byref(pl)))
        return {"ms": dict(zip(PHASES, ms.tolist())), "launches": dict(zip(PHASES, ln.tolist())),
                "push_launches": int(pl.value)}


def pic_create(dim, n, dx, dt, species, **kw) -> Sim:
    """pic_create(grid, dt, species): species is a list of (q, m, w, capacity)."""
    return Sim(dim, n, dx, dt, species, **kw)


def from_workload(w, precision=FP32_CELLOFF, sort_interval=0, capacity_scale=1.0, load=True, stream=None,
                  tile=None, push_variant=0, seed=0, pusher=0, allocator=None, order=2) -> Sim:
    """Create a simulation for a :class:`workloads.Workload` and load its particles
    (QED workloads: the Monte Carlo is configured in table mode first)."""
    sp = [(s.q, s.m, s.w, max(1, int(s.capacity * capacity_scale)), s.kind, s.qed) for s in w.species]
    t = tile if tile is not None else tuple(w.tile)
    sim = Sim(w.dim, w.n, w.dx, w.dt, sp, bc=w.bc, precision=precision, sort_interval=sort_interval, tile=t,
              rho_bg=w.rho_bg, stream=stream, push_variant=push_variant, seed=seed, pusher=pusher,
              allocator=allocator, order=order)
    if w.laser is not None:
        L = w.laser
        sim.pic_set_laser(L.a0, L.waist, L.fwhm, L.t_peak, L.x_focus, L.yc, L.zc, L.pol)
    if w.qed is not None:
        sim.pic_set_qed(mode=QED_TABLE, **w.qed)
    if load:
        for i, s in enumerate(w.species):
            if s.n:
                sim.pic_load_particles(i, s.x, s.y if w.dim > 1 else None, s.z if w.dim > 2 else None, s.ux, s.uy,
                                       s.uz)
    return sim
