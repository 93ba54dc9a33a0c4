"""ctypes wrapper of the FP64 CPU oracle (``liboracle.so``).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this module; the product path never does.
The C sources next to this file follow the paper's equations (Song, Wang & Li,
arXiv:2104.00642, Secs. II and IV); this wrapper only marshals arguments.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liboracle.so")
SOURCES = ["pic_oracle.c", "philox.c", "qed.c", "mlp.c"]

EX, EY, EZ, BX, BY, BZ, JX, JY, JZ = range(9)
PERIODIC, ABSORB, SLAB = 0, 1, 2  # SLAB: a slab of a larger periodic grid (domain-decomposition tests)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no contraction, no fast-math)."""
    srcs = [os.path.join(_HERE, s) for s in SOURCES if os.path.exists(os.path.join(_HERE, s))]
    if not force and os.path.exists(LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "pic_oracle.h")])
        if os.path.getmtime(LIB_PATH) >= newest:
            return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-Wno-unused-function", *srcs, "-lm", "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB_PATH)
        P, D, I, LG = C.c_void_p, C.c_double, C.c_int, C.c_long
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        L.or_create.restype = P
        L.or_create.argtypes = [I, P, P, P, D, D, I, P]
        L.or_destroy.argtypes = [P]
        L.or_add_species.argtypes = [P, D, D, D, LG]
        L.or_add_species.restype = I
        L.or_load.argtypes = [P, I, LG, P, P, P, P, P, P]
        L.or_load.restype = I
        L.or_set_ids.argtypes = [P, I, LG, LG, P]
        L.or_set_ids.restype = I
        L.or_get_field.argtypes = [P, I, P]
        L.or_set_field.argtypes = [P, I, P]
        L.or_get_ghost.argtypes = [P, I, LG, LG, LG, P]
        L.or_set_laser.argtypes = [P, I, D, D, D, D, D, D, D]
        L.or_weights2.argtypes = [D, P]
        L.or_gather.argtypes = [P, P, P]
        L.or_boris.argtypes = [D, D, P, P, P]
        L.or_vay.argtypes = [D, D, P, P, P]
        L.or_set_pusher.argtypes = [P, I]
        L.or_set_order.argtypes = [P, I]
        L.or_set_order.restype = I
        L.or_weights4.argtypes = [D, P]
        L.or_deposit_one.argtypes = [P, P, P, P, D]
        L.or_sort_species.argtypes = [P, I, P]
        L.or_sort_species.restype = LG
        L.or_step.argtypes = [P, LG]
        L.or_step_phase.argtypes = [P, I]
        L.or_step_phase.restype = I
        L.or_field_raw_size.argtypes = [P, P]
        L.or_field_raw_size.restype = LG
        L.or_get_field_raw.argtypes = [P, I, P]
        L.or_set_field_raw.argtypes = [P, I, P]
        L.or_take_outbox.argtypes = [P, I, P, P, P, P]
        L.or_take_outbox.restype = LG
        L.or_load_state.argtypes = [P, I, LG, P, P, P, P]
        L.or_load_state.restype = I
        L.or_get_particles.argtypes = [P, I, P, P, P, P, P, P, P]
        L.or_get_particles.restype = LG
        L.or_get_rho.argtypes = [P, P]
        L.or_diagnostics.argtypes = [P, P]
        L.or_diagnostics.restype = I
        L.or_step_count.argtypes = [P]
        L.or_step_count.restype = LG
        L.or_add_species2.argtypes = [P, D, D, D, LG, I, I]
        L.or_add_species2.restype = I
        L.or_set_qed.argtypes = [P, I, I, I, D, D, C.c_uint64]
        L.or_Es.argtypes = [P]
        L.or_Es.restype = D
        L.or_set_qed_method.argtypes = [P, I]
        L.or_set_qed_method.restype = I
        L.or_method2_over.argtypes = [P]
        L.or_method2_over.restype = LG
        L.or_chi.argtypes = [P, D, P, P]
        L.or_chi.restype = D
        L.or_photon_lost.argtypes = [P]
        L.or_photon_lost.restype = D
        L.or_get_qed_state.argtypes = [P, I, P, P]
        L.or_get_qed_state.restype = LG
        L.or_mlp_nparams.restype = LG
        L.or_mlp_forward.argtypes = [P, LG, P, P]
        L.or_mlp_loss_grad.argtypes = [P, LG, P, P, P]
        L.or_mlp_loss_grad.restype = D
        L.or_philox4x32_10.argtypes = [P, P, P]
        L.or_uniform24.argtypes = [C.c_uint32]
        L.or_uniform24.restype = D
        _lib = L
        _bind_extras(L)
    return _lib


def _bind_extras(L):
    """QED and MLP entry points (present once those sources exist)."""
    P, D, I, LG = C.c_void_p, C.c_double, C.c_int, C.c_long
    for name, argt, rt in [
        ("or_bessel_k", [D, D], D),
        ("or_int_k13", [D], D),
        ("or_qed_Frad", [D, D], D),
        ("or_qed_Fpair", [D, D], D),
        ("or_qed_Grad", [D], D),
        ("or_qed_Gpair", [D], D),
        ("or_qed_Prad", [D], D),
        ("or_qed_cdf_rad", [D, D], D),
        ("or_qed_cdf_pair", [D, D], D),
        ("or_qed_sample_rad", [D, D], D),
        ("or_qed_sample_pair", [D, D], D),
        ("or_qed_method2_rad", [D, D, D, D], D),
    ]:
        if hasattr(L, name):
            f = getattr(L, name)
            f.argtypes = argt
            f.restype = rt


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def weights2(delta: float) -> np.ndarray:
    w = np.zeros(3)
    lib().or_weights2(float(delta), _ptr(w))
    return w


def weights4(delta: float) -> np.ndarray:
    w = np.zeros(5)
    lib().or_weights4(float(delta), _ptr(w))
    return w


def boris(qm: float, dt: float, E, B, u) -> np.ndarray:
    E, B = _f64(E), _f64(B)
    uu = _f64(np.array(u, dtype=np.float64).copy())
    lib().or_boris(float(qm), float(dt), _ptr(E), _ptr(B), _ptr(uu))
    return uu


def vay(qm: float, dt: float, E, B, u) -> np.ndarray:
    E, B = _f64(E), _f64(B)
    uu = _f64(np.array(u, dtype=np.float64).copy())
    lib().or_vay(float(qm), float(dt), _ptr(E), _ptr(B), _ptr(uu))
    return uu


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform24(x: int) -> float:
    return lib().or_uniform24(C.c_uint32(int(x) & 0xFFFFFFFF))


class OracleSim:
    """The FP64 CPU reference simulation (absolute positions, no ghosts)."""

    def __init__(self, dim, n, dx, dt, bc=(PERIODIC, PERIODIC, PERIODIC), rho_bg=0.0,
                 sort_interval=0, tile=(8, 8, 8)):
        L = lib()
        n3 = np.array(list(n) + [1] * (3 - len(n)), dtype=np.int64)
        dx3 = np.array(list(dx) + [1.0] * (3 - len(dx)), dtype=np.float64)
        bc3 = np.array(list(bc) + [0] * (3 - len(bc)), dtype=np.int32)
        t3 = np.array(list(tile) + [1] * (3 - len(tile)), dtype=np.int32)
        self.dim = dim
        self.n = n3
        self.dx = dx3
        self.bc = bc3
        self.dt = float(dt)
        self._h = L.or_create(int(dim), _ptr(n3), _ptr(dx3), _ptr(bc3), float(dt), float(rho_bg),
                              int(sort_interval), _ptr(t3))
        if not self._h:
            raise ValueError("oracle: bad grid")
        self.nsp = 0
        self._keep = [n3, dx3, bc3, t3]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    def box(self):
        """Field output shape (z, y, x): N per periodic axis, N+1 per absorbing axis."""
        m = [1, 1, 1]
        for d in range(self.dim):
            m[d] = int(self.n[d]) + (1 if self.bc[d] == ABSORB else 0)
        return (m[2], m[1], m[0])

    def add_species(self, q, m, w, cap, kind=0, qed=0):
        i = lib().or_add_species2(self._h, float(q), float(m), float(w), int(cap), int(kind), int(qed))
        if i < 0:
            raise ValueError("oracle: too many species")
        self.nsp += 1
        return i

    def set_qed(self, photon_sp=-1, electron_sp=-1, positron_sp=-1, lambda_r_m=1e-6, photon_emin=0.0, seed=0):
        lib().or_set_qed(self._h, int(photon_sp), int(electron_sp), int(positron_sp), float(lambda_r_m),
                         float(photon_emin), C.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF))

    def set_qed_method(self, method):
        """1: Method I (optical depth, default), 2: Method II"""
        if lib().or_set_qed_method(self._h, int(method)):
            raise ValueError("oracle: QED method must be 1 or 2")

    def method2_over(self):
        """Method II draws whose acceptance probability exceeded one"""
        return lib().or_method2_over(self._h)

    @property
    def Es(self):
        return lib().or_Es(self._h)

    def chi(self, gamma, u, eb):
        """the quantum parameter the Monte Carlo uses for momentum u (or k) with
        gamma (or |k|) in the fields eb = (Ex, Ey, Ez, Bx, By, Bz)"""
        uu, e = _f64(np.asarray(u, dtype=np.float64)), _f64(np.asarray(eb, dtype=np.float64))
        return lib().or_chi(self._h, float(gamma), _ptr(uu), _ptr(e))

    def photon_lost(self):
        return lib().or_photon_lost(self._h)

    def qed_state(self, isp):
        n = lib().or_get_qed_state(self._h, int(isp), None, None)
        ids = np.zeros(max(n, 1), dtype=np.uint64)
        tau = np.zeros(max(n, 1))
        lib().or_get_qed_state(self._h, int(isp), _ptr(ids), _ptr(tau))
        return ids[:n], tau[:n]

    def load(self, isp, x, y, z, ux, uy, uz):
        n = len(ux)
        arrs = [_f64(a) if a is not None else None for a in (x, y, z, ux, uy, uz)]
        rc = lib().or_load(self._h, int(isp), int(n), *[_ptr(a) for a in arrs])
        if rc != 0:
            raise ValueError(f"oracle: load failed ({rc})")

    def set_ids(self, isp, ids, first=0):
        """identities of particles [first, first + len(ids)) (their optical
        depths restart from the identities' initial draws)"""
        a = np.ascontiguousarray(ids, dtype=np.uint64)
        rc = lib().or_set_ids(self._h, int(isp), int(first), len(a), _ptr(a))
        if rc:
            raise ValueError(f"or_set_ids failed ({rc})")

    def set_order(self, order):
        """shape order of gather, deposit and charge density: 2 or 4"""
        if lib().or_set_order(self._h, int(order)):
            raise ValueError("oracle: order must be 2 or 4")

    def set_pusher(self, pusher):
        """0: Boris, 1: Vay"""
        lib().or_set_pusher(self._h, int(pusher))

    def set_laser(self, a0, waist, fwhm, t_peak, x_focus, yc=0.0, zc=0.0, pol=0):
        lib().or_set_laser(self._h, int(pol), float(a0), float(waist), float(fwhm), float(t_peak),
                           float(x_focus), float(yc), float(zc))

    def field(self, c) -> np.ndarray:
        out = np.zeros(self.box())
        lib().or_get_field(self._h, int(c), _ptr(out))
        return out

    def set_field(self, c, arr):
        a = _f64(np.broadcast_to(arr, self.box()))
        lib().or_set_field(self._h, int(c), _ptr(a))

    def ghost(self, c, i, j=0, k=0) -> float:
        v = np.zeros(1)
        rc = lib().or_get_ghost(self._h, int(c), int(i), int(j), int(k), _ptr(v))
        if rc != 0:
            raise IndexError("not stored")
        return float(v[0])

    def gather(self, x) -> np.ndarray:
        xx = _f64(np.array(list(x) + [0.0] * (3 - len(x))))
        out = np.zeros(6)
        lib().or_gather(self._h, _ptr(xx), _ptr(out))
        return out

    def deposit_one(self, x0, x1, v, qw):
        a = [_f64(np.array(list(t) + [0.0] * (3 - len(t)))) for t in (x0, x1, v)]
        lib().or_deposit_one(self._h, *[_ptr(t) for t in a], float(qw))
        return self.field(JX), self.field(JY), self.field(JZ)

    def sort(self, isp):
        n = self.particles(isp)["ux"].shape[0]
        perm = np.zeros(max(n, 1), dtype=np.int64)
        m = lib().or_sort_species(self._h, int(isp), _ptr(perm))
        return perm[:m]

    def step(self, n=1):
        lib().or_step(self._h, int(n))

    def step_phase(self, phase):
        """one of the split step's five phases (0: E half, 1: B half, 2: push,
        3: B half, 4: E half and n -> n+1)"""
        if lib().or_step_phase(self._h, int(phase)):
            raise ValueError("oracle: bad phase")

    # --- slab sub-domains (bc SLAB along x): raw arrays with ghost layers ---
    def field_raw(self, c):
        """component c with its ghost layers, shape (len_z, len_y, len_x)
        (along a SLAB axis index i sits at i + 4)"""
        ln = np.zeros(3, dtype=np.int64)
        L = lib()
        n = L.or_field_raw_size(self._h, _ptr(ln))
        out = np.zeros(n)
        L.or_get_field_raw(self._h, int(c), _ptr(out))
        return out.reshape(ln[2], ln[1], ln[0])

    def set_field_raw(self, c, a):
        a = _f64(np.asarray(a, dtype=np.float64))
        lib().or_set_field_raw(self._h, int(c), _ptr(a))

    def take_outbox(self, isp):
        """particles of species isp that left the slab since the last call:
        (x (n, 3), u (n, 3), id, tau)"""
        L = lib()
        n = L.or_take_outbox(self._h, int(isp), None, None, None, None)
        x, u = np.zeros((n, 3)), np.zeros((n, 3))
        ids, tau = np.zeros(n, dtype=np.uint64), np.zeros(n)
        if n:
            L.or_take_outbox(self._h, int(isp), _ptr(x), _ptr(u), _ptr(ids), _ptr(tau))
        return x, u, ids, tau

    def load_state(self, isp, x, u, ids, tau):
        """append particles with their identities and optical depths"""
        n = len(ids)
        if n == 0:
            return
        xa, ua = _f64(np.asarray(x, dtype=np.float64).reshape(n, 3)), _f64(np.asarray(u, dtype=np.float64).reshape(n, 3))
        ia, ta = np.ascontiguousarray(ids, dtype=np.uint64), _f64(np.asarray(tau, dtype=np.float64))
        rc = lib().or_load_state(self._h, int(isp), n, _ptr(xa), _ptr(ua), _ptr(ia), _ptr(ta))
        if rc:
            raise ValueError(f"oracle: load_state failed ({rc})")

    def particles(self, isp):
        L = lib()
        n = L.or_get_particles(self._h, int(isp), None, None, None, None, None, None, None)
        out = {k: np.zeros(n) for k in ("x", "y", "z", "ux", "uy", "uz")}
        alive = np.zeros(n, dtype=np.uint8)
        L.or_get_particles(self._h, int(isp), *[_ptr(out[k]) for k in ("x", "y", "z", "ux", "uy", "uz")],
                           _ptr(alive))
        out["alive"] = alive
        return out

    def rho(self) -> np.ndarray:
        out = np.zeros(self.box())
        lib().or_get_rho(self._h, _ptr(out))
        return out

    def diagnostics(self) -> dict:
        out = np.zeros(7 + 8)
        m = lib().or_diagnostics(self._h, _ptr(out))
        return {"step": int(out[0]), "t": out[1], "U_E": out[2], "U_B": out[3], "charge": out[4],
                "gauss_max": out[5], "E_absorbed": out[6], "U_kin": list(out[7:m])}

    @property
    def step_count(self):
        return lib().or_step_count(self._h)


def mlp_nparams() -> int:
    return int(lib().or_mlp_nparams())


def mlp_forward(params, x):
    P = _f64(params)
    X = _f64(np.asarray(x).reshape(-1, 2))
    out = np.zeros((X.shape[0], 2))
    lib().or_mlp_forward(_ptr(P), X.shape[0], _ptr(X), _ptr(out))
    return out


def mlp_loss_grad(params, x, t):
    P = _f64(params)
    X = _f64(np.asarray(x).reshape(-1, 2))
    T = _f64(np.asarray(t).reshape(-1, 2))
    G = np.zeros(mlp_nparams())
    loss = lib().or_mlp_loss_grad(_ptr(P), X.shape[0], _ptr(X), _ptr(T), _ptr(G))
    return loss, G
