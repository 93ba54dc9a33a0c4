"""Throughput benchmark of the GB300 PIC hot path.

Default workload: the strong-field QED collision (2D3V, grid 2048x512,
dx = lambda/32; LP laser a0 = 200 from x-min against a 1 GeV beam of 10^7
macro-electrons; nonlinear Compton and Breit-Wheeler Monte Carlo with
per-particle optical depth), the configuration the metric -- FP32 cell+offset
with the surrogate network vs the plain FP64 form at equal error -- is quoted
on.  Each form is advanced untimed to the collision, then W warm-up and K
timed steps run through it.  A "step" is one full PIC step of every species
(both field half steps, gather + push + QED Monte Carlo + drift + Esirkepov
deposit, current fold, spawn of photons and pairs, tile sort every K steps).

Prints one JSON line.  ``value`` is particle-steps/s of the FP32+surrogate
form (live particles of all species), CUDA events on the simulation's stream
around one ``pic_step(K)`` call, inputs resident in HBM (each step touches
more bytes than the L2 holds).  The line carries the FP32+tables and plain
FP64 forms on the same window, the errors of every form against the FP64
oracle on the collision's QED regime (tests/golden/qed_field_sample.json),
the roofline of the dominant push kernel, ``e2e`` (the state at the window's
start restored from a host file through the C ABI, K steps, diagnostics read
back, host wall clock) and the oracle's CPU throughput on that sample.

``--workload laser_foil_2d | thermal_3d`` time the plain PIC step (no QED)
through the laser-slab interaction or the thermal steady state, with the
push-kernel roofline.  ``--impl reference`` times the FP64 CPU oracle
(host cores) on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s on 1 GB300: FP32+surrogate vs plain FP64 form at same error"
UNIT = "particle-steps/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def max_over_ranks(t_local, dist, device="cuda"):
    """the slowest rank's time: the replicas run independently, and the job
    takes as long as its slowest one"""
    if not dist:
        return t_local
    import torch
    tt = torch.tensor([t_local], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def make_workload(name, rank=0, sample=None, beam=10_000_000):
    from paper_2104_00642_gb300 import workloads as W
    if name == "laser_foil_2d":
        ny = 1024 if sample is None else sample
        return W.laser_foil_2d(ny=ny, seed=W.SEED0 + 2 + 1000 * rank)
    if name == "thermal_3d":
        n = (256, 256, 256) if sample is None else (256, 256, sample)
        return W.thermal_3d(n=n, seed=W.SEED0 + 3 + 1000 * rank)
    if name == "langmuir_1d":
        return W.langmuir_1d()
    if name == "qed_collision_2d":
        return W.qed_collision_2d(seed=W.SEED0 + 7 + 1000 * rank, n_beam=beam)
    if name == "qed_foil_3d":
        return W.qed_foil_3d(seed=W.SEED0 + 8 + 1000 * rank)
    raise SystemExit(f"unknown workload {name}")


def describe(w):
    return (f"{w.name} {'x'.join(str(v) for v in w.n[:w.dim])} cells, {w.n_particles} particles "
            f"({', '.join(s.name for s in w.species)})")


def bytes_per_particle(dim, precision):
    """algorithmic HBM bytes of one particle in the push kernel (read + write
    of the particle state once)"""
    if precision == 0:
        return 2 * (4 + 4 * dim + 12)
    return 2 * (4 + 8 * dim + 24)


L2_BYTES = 126 * 1024 * 1024  # GB300 L2

# steps between tile sorts, chosen by measurement on a GB300 (ms per step):
# laser_foil_2d at steps 0-64 / 1928-1992 / 3792-3856 (laser on the slab):
# K = 8: 0.338 / 0.339 / 0.370, K = 16: 0.310 / 0.317 / 0.367, K = 32: 0.298 /
# 0.306 / 0.410; thermal_3d: K = 4: 19.6, K = 8: 20.7
SORT_INTERVAL = {"laser_foil_2d": 16, "thermal_3d": 4}
# untimed steps before the timed window: the laser-foil run is timed while
# the pulse sits on the slab (its peak reaches the slab front, x = 1024 dx,
# at t = t_peak + 1024 dx, step 3674 of 4000)
PRE_STEPS = {"laser_foil_2d": 3680}


def step_bytes(w, precision=0):
    """bytes one step touches at least: the particle state of every species
    (read and written once) and the nine field components of the padded grid"""
    ext = 1
    for d in range(w.dim):
        ext *= w.n[d] + 8
    state = bytes_per_particle(w.dim, precision) // 2
    return sum(s.n for s in w.species) * state + 9 * (8 if precision else 4) * ext


def occupied_cells(w):
    cells = set()
    for s in w.species:
        c = np.floor(s.x / w.dx[0]).astype(np.int64)
        if w.dim > 1:
            c = c + w.n[0] * np.floor(s.y / w.dx[1]).astype(np.int64)
        if w.dim > 2:
            c = c + w.n[0] * w.n[1] * np.floor(s.z / w.dx[2]).astype(np.int64)
        cells.update(np.unique(c).tolist())
    return len(cells)


class Clocks:
    """SM clock and throttle reasons sampled DURING the timed region: a
    thread polls NVML (read-only queries through ctypes) every ~2 ms, so a
    window of a few milliseconds still has samples; without NVML it falls
    back to nvidia-smi at 100 ms."""

    # clocks-event reason bits of NVML
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, dev):
        self.dev = dev
        self.rows = []
        self.nvml = None
        self.thread = None
        self.stop = False
        self.smi = None

    def _nvml_open(self):
        import ctypes as C
        for name in ("libnvidia-ml.so.1", "libnvidia-ml.so"):
            try:
                L = C.CDLL(name)
                break
            except OSError:
                L = None
        if L is None or L.nvmlInit_v2() != 0:
            return None
        h = C.c_void_p()
        n = C.c_uint()
        L.nvmlDeviceGetCount_v2(C.byref(n))
        idx = self.dev if n.value > self.dev else 0
        if n.value > 1:
            try:  # the CUDA device's own NVML handle, by PCI bus id
                import torch
                pr = torch.cuda.get_device_properties(self.dev)
                bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0".encode()
                if L.nvmlDeviceGetHandleByPciBusId_v2(bus, C.byref(h)) == 0:
                    return L, h
            except Exception:
                pass
        if L.nvmlDeviceGetHandleByIndex_v2(idx, C.byref(h)) != 0:
            return None
        return L, h

    def _poll(self):
        import ctypes as C
        L, h = self.nvml
        sm, mx, rs = C.c_uint(), C.c_uint(), C.c_ulonglong()
        L.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(mx))
        get_reasons = getattr(L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            L.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop:
            if L.nvmlDeviceGetClockInfo(h, 1, C.byref(sm)) == 0 and get_reasons(h, C.byref(rs)) == 0:
                self.rows.append((sm.value, mx.value, rs.value))
            time.sleep(0.002)

    def __enter__(self):
        try:
            self.nvml = self._nvml_open()
        except Exception:
            self.nvml = None
        if self.nvml is not None:
            import threading
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            return self
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.smi = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={q}",
                                         "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                        stderr=subprocess.DEVNULL)
        except Exception:
            self.smi = None
        return self

    def __exit__(self, *a):
        if self.thread is not None:
            self.stop = True
            self.thread.join(timeout=5)
        if self.smi is not None:
            self.smi.terminate()
            try:
                self.smi.wait(timeout=5)
            except Exception:
                self.smi.kill()
            self.f.close()
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for ln in open(self.path):
                t = [x.strip() for x in ln.split(",")]
                if len(t) >= 9 and t[1].replace(".", "").isdigit():
                    bits = 0
                    for i, nm in enumerate(names):
                        if t[5 + i].lower() == "active":
                            bits |= {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40, "sw_thermal_slowdown": 0x20,
                                     "sw_power_cap": 0x4}[nm]
                    self.rows.append((float(t[1]), float(t[2]) if t[2].replace(".", "").isdigit() else 0.0, bits))

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None,
                    "reasons": ["no samples" if (self.nvml or self.smi) else "no NVML and no nvidia-smi"]}
        sm = [r[0] for r in self.rows]
        reasons = sorted({nm for r in self.rows for bit, nm in self.REASONS.items() if r[2] & bit})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(r[1] for r in self.rows)),
                "reasons": reasons, "samples": len(self.rows),
                "source": "nvml (2 ms polling)" if self.nvml else "nvidia-smi (100 ms)"}


def source_sha256(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()


def traffic_record(workload):
    """dram bytes per push launch of this workload from the committed ncu
    summary, if it was taken on the current kernel source (else None)"""
    path = os.path.join(ROOT, "profiles", "push_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(workload)
    if not rec or rec.get("source_sha256") != source_sha256(rec["source_files"]):
        return None
    return rec


def oracle_rate(wname, min_seconds=10.0, max_steps=50, steps=None, sample_rows=32):
    """FP64 CPU oracle on a y-strip sample of the workload (same x structure,
    periodic y): particle-steps/s on one host core"""
    from tests.helpers import oracle_from_workload
    w = make_workload(wname, sample=sample_rows)
    o = oracle_from_workload(w, sort_interval=0)
    npart = w.n_particles
    t0 = time.perf_counter()
    done = 0
    per = []
    while True:
        a = time.perf_counter()
        o.step(1)
        per.append(time.perf_counter() - a)
        done += 1
        if steps is not None and done >= steps:
            break
        if steps is None and (time.perf_counter() - t0 >= min_seconds or done >= max_steps):
            break
    el = time.perf_counter() - t0
    return npart * done / el, {"sample": f"{describe(w)}: y-strip of {sample_rows} rows of the full workload, "
                                         f"{done} steps", "seconds": el, "steps": done, "per_step_s": per,
                               "particles": npart}


def cpu_model():
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu model")):
                return ln.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def _oracle_qed_chunk(args):
    """the FP64 oracle on electrons [lo, hi) of the QED field sample (their
    full-load identities), `steps` steps: (particle-steps, seconds)"""
    lo, hi, steps, seed = args
    from oracle import oracle as O
    from paper_2104_00642_gb300 import workloads as W
    w = W.qed_field_sample()
    o = O.OracleSim(1, (16,), (1.0,), w.dt)
    for sp in w.species:
        o.add_species(sp.q, sp.m, sp.w, sp.capacity, kind=sp.kind, qed=sp.qed)
    o.set_qed(seed=seed, **w.qed)
    o.set_field(O.BZ, np.full(o.box(), w.notes["B0"]))
    e = w.species[0]
    o.load(0, e.x[lo:hi], None, None, e.ux[lo:hi], e.uy[lo:hi], e.uz[lo:hi])
    o.set_ids(0, np.arange(lo, hi, dtype=np.uint64))
    done = 0
    t0 = time.perf_counter()
    per = []
    for _ in range(steps):
        n = sum(int(np.sum(o.particles(i)["alive"])) for i in range(3))
        a = time.perf_counter()
        o.step(1)
        per.append((n, time.perf_counter() - a))
        done += n
    return done, time.perf_counter() - t0, per


def oracle_qed_rate(n_e=64, steps=8, all_cores=False, seed=0x5A3D1E):
    """FP64 oracle throughput on the collision's QED regime (the field
    sample): one core on n_e electrons, or every host core on its own chunk
    of n_e electrons each (processes started with spawn)"""
    if not all_cores:
        ps, sec, per = _oracle_qed_chunk((0, n_e, steps, seed))
        return ps / sec, {"cores": 1, "particle_steps": ps, "seconds": sec, "per_step": per}
    import multiprocessing as mp
    nc = os.cpu_count() or 1
    jobs = [(i * n_e, (i + 1) * n_e, steps, seed) for i in range(nc)]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(nc) as pool:
        res = pool.map(_oracle_qed_chunk, jobs)
    wall = time.perf_counter() - t0
    ps = sum(r[0] for r in res)
    return ps / wall, {"cores": nc, "particle_steps": ps, "seconds": wall}


def run_reference(args):
    """--impl reference: the FP64 CPU oracle, as it stands, on the host cores"""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    for _ in range(args.warmup):
        pass
    w = args.workload
    if w in ("qed_collision_2d", "qed_foil_3d"):
        # a bounded sample: the oracle takes ~2.7 s per step for 128 electrons
        # and the photons they make (more every step), so the sample shrinks
        # with the step count to keep the whole run near two minutes
        n_ref = max(16, int(128 * min(1.0, 20.0 / max(1, args.warmup + args.steps))))
        ps_w, sec_w, per = _oracle_qed_chunk((0, n_ref, args.warmup + args.steps, 0x5A3D1E))
        per = per[args.warmup:]
        t = float(sum(x[1] for x in per))
        value = float(sum(x[0] for x in per)) / t
        sample = (f"the collision's QED regime, {n_ref} electrons of the qed_field_sample (gamma 1957 +- 1 %, "
                  "chi ~ 1.9, photons and pairs they create), FP64 oracle")
        out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / len(per),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": sample, "precision": "fp64 absolute positions, QED rates and spectra by "
                          "quadrature (CPU oracle)"},
               "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                                "cpu": cpu_model()},
               "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return
    v, info = oracle_rate(w, steps=args.warmup + args.steps)
    per = info["per_step_s"][args.warmup:]
    t = float(np.sum(per))
    value = info["particles"] * len(per) / t
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / len(per), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": info["sample"], "precision": "fp64 absolute positions (CPU oracle)"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": info["sample"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def photon_spectrum(sim, sp, edges):
    p = sim.pic_get_particles(sp)
    a = p["alive"] == 1
    k = np.sqrt(p["ux"][a] ** 2 + p["uy"][a] ** 2 + p["uz"][a] ** 2)
    return np.histogram(k, edges)[0]


def qed_bytes_per_particle(dim, photon=False):
    """algorithmic HBM bytes of one particle in a QED push: the FP32 state
    read and written once (a photon's momentum is only read: it moves at c
    along k), the FP64 optical depth read and written, the event flag
    written"""
    if photon:
        return (4 + 4 * dim + 12) + (4 + 4 * dim) + 16 + 4
    return 2 * (4 + 4 * dim + 12) + 16 + 4


def run_qed_sample(pic, mode, nets, golden):
    """one form on the QED field sample (the stored FP64 oracle run's seeded
    inputs): its errors against the oracle"""
    from paper_2104_00642_gb300 import workloads as W
    from tests import qed_setup as Q
    ws = W.qed_field_sample()
    prec = pic.FP64_PLAIN if mode == "fp64" else pic.FP32_CELLOFF
    sim = pic.from_workload(ws, precision=prec, seed=golden["seed"])
    if mode == "surrogate":
        for p_, (P, info) in nets.items():
            sim.pic_mlp_set(p_, P, info["chi_min"], info["chi_max"], info["mu"], info["sd"])
        sim.pic_set_qed(mode=pic.QED_SURROGATE, **ws.qed)
    sim.pic_set_field(pic.BZ, np.full(sim.box(), ws.notes["B0"]))
    hist = []
    for _ in range(ws.steps):
        sim.pic_step(1)
        e = sim.pic_get_particles(0)
        a = e["alive"] == 1
        hist.append(float(np.sum(np.sqrt(1.0 + e["ux"][a] ** 2 + e["uy"][a] ** 2 + e["uz"][a] ** 2))))
    d = sim.pic_diagnostics()
    fin = Q.sample_observables([sim.pic_get_particles(i) for i in range(3)], d["E_photon_lost"])
    sim.close()
    return Q.sample_errors({"history": hist, "final": fin}, golden)


PUSHER = {"boris": 0, "vay": 1}


def run_qed(args, w, pic, torch, stream, timed, rank, world, dist, local, l2_note):
    """The strong-field QED collision: the same seeded beam through three
    forms, each advanced untimed to the collision, then W warm-up and K timed
    steps around the pulse peak: FP32 cell+offset with the surrogate networks
    (trained on the device first, untimed), FP32 with the tables, and the
    plain FP64 form with the tables.  Particle-steps count the live particles
    of all species (trapezoid over the window).  Errors: every form against
    the FP64 oracle on the collision's QED regime (stored run), and the FP32
    forms against the FP64 run of the window."""
    from tests import qed_setup as Q
    K = args.steps
    if args.qed_pre is not None:
        pre = args.qed_pre
    elif "steps_to_collision" in w.notes:
        pre = max(0, w.notes["steps_to_collision"] - K // 2 - args.warmup)
    else:
        pre = 0
    iph, iel, ipo = w.qed["photon_sp"], w.qed["electron_sp"], w.qed["positron_sp"]
    edges = np.logspace(np.log10(w.qed["photon_emin"]), np.log10(3000.0), 25)
    runs = {}
    nets = {}
    modes = [m for m in args.qed_modes.split(",") if m]
    e2e = None
    peak, peak_kind = _peaks()
    for mode in modes:
        prec = pic.FP64_PLAIN if mode == "fp64" else pic.FP32_CELLOFF
        sim = pic.from_workload(w, precision=prec, sort_interval=args.sort_interval, pusher=PUSHER[args.pusher], stream=stream.cuda_stream,
                                seed=0x5EED + rank, push_variant=args.push_variant)
        train = None
        if mode == "surrogate":
            cmin = {pic.QED_EMISSION: 0.0, pic.QED_PAIR: args.qed_pair_chi_min}
            train = {p: sim.pic_mlp_train(p, iterations=args.qed_train_iters, seed=17, chi_min=cmin[p])
                     for p in (pic.QED_EMISSION, pic.QED_PAIR)}
            nets = {p: sim.pic_mlp_get(p) for p in (pic.QED_EMISSION, pic.QED_PAIR)}
            sim.pic_set_qed(mode=pic.QED_SURROGATE, **w.qed)
        with torch.cuda.stream(stream):
            sim.pic_step(pre)
        timed(sim, args.warmup)
        d0 = sim.pic_diagnostics()
        n0 = sum(d0["n_alive"])
        ckpt = None
        if mode == modes[0] and not args.no_e2e and world == 1:
            # the state at the window's start, in a host file (untimed)
            fd, ckpt = tempfile.mkstemp(prefix="pic_window_", suffix=".ckpt",
                                        dir="/dev/shm" if os.path.isdir("/dev/shm") else None)
            os.close(fd)
            sim.pic_save(ckpt)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with Clocks(local) as clk:
            ms, prof = timed(sim, K, profile=True)
        sp_ms, sp_n = sim.pic_profile_read_species()
        d = sim.pic_diagnostics()
        n1 = sum(d["n_alive"])
        t = max_over_ranks(float(np.sum(ms)) / 1e3, dist)
        alive_mid = [0.5 * (a + b) for a, b in zip(d0["n_alive"], d["n_alive"])]
        runs[mode] = {"value": world * 0.5 * (n0 + n1) * K / t, "ms_per_step": 1e3 * t / K, "n_alive": d["n_alive"],
                      "U_kin": d["U_kin"], "U_EM": d["U_E"] + d["U_B"], "E_photon_lost": d["E_photon_lost"],
                      "spectrum": photon_spectrum(sim, w.qed["photon_sp"], edges), "prof": prof, "clocks": clk.summary(),
                      "train": train, "species_ms": sp_ms, "species_pushes": sp_n, "alive_mid": alive_mid}
        if ckpt is not None:
            # end to end through the C ABI: restore the window's start from the
            # host file, K steps, diagnostics read back (host wall clock)
            size = os.path.getsize(ckpt)
            sim.close()
            sim = None
            sim_e = pic.from_workload(w, precision=prec, sort_interval=args.sort_interval, pusher=PUSHER[args.pusher], stream=stream.cuda_stream,
                                      seed=0x5EED + rank, push_variant=args.push_variant, load=False)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sim_e.pic_restore(ckpt)
            sim_e.pic_step(K)
            de = sim_e.pic_diagnostics()
            el = time.perf_counter() - t0
            os.unlink(ckpt)
            assert math.isfinite(de["U_E"])
            e2e = {"value": 0.5 * (n0 + sum(de["n_alive"])) * K / el, "unit": UNIT, "h2d_bytes_per_step": size / K,
                   "d2h_bytes_per_step": 8 * (16 + 2 * len(w.species)) / K, "seconds": el,
                   "note": "pic_restore of the window's start from a host file (fields, particles, networks) + "
                           "pic_step(K) + pic_diagnostics, host wall clock"}
            sim_e.close()
        if sim is not None:
            sim.close()
    ref = runs.get("fp64")

    def errors(r):
        if ref is None or r is None:
            return None
        e_tot = lambda x: sum(x["U_kin"]) + x["U_EM"] + x["E_photon_lost"]
        big = ref["spectrum"] >= 1000
        spec = np.abs(r["spectrum"][big] / ref["spectrum"][big] - 1.0)
        return {"total_energy_rel": abs(e_tot(r) / e_tot(ref) - 1.0),
                "photon_energy_rel": abs(r["U_kin"][iph] / ref["U_kin"][iph] - 1.0) if ref["U_kin"][iph] else None,
                "electron_energy_rel": abs(r["U_kin"][iel] / ref["U_kin"][iel] - 1.0),
                "photon_count_rel": abs(r["n_alive"][iph] / max(ref["n_alive"][iph], 1) - 1.0),
                "pairs": (int(r["n_alive"][ipo]), int(ref["n_alive"][ipo])),
                "photon_spectrum_max_bin_rel": float(spec.max()) if big.any() else None,
                "photon_spectrum_bins": int(big.sum())}

    # errors against the FP64 oracle on the collision's QED regime (stored run)
    vs_oracle = None
    gpath = os.path.join(ROOT, "tests", "golden", "qed_field_sample.json")
    if rank == 0 and os.path.exists(gpath):
        golden = json.load(open(gpath))
        vs_oracle = {m: run_qed_sample(pic, m, nets, golden) for m in modes if m != "surrogate" or nets}
        vs_oracle["sample"] = ("workloads.qed_field_sample: 2048 electrons at gamma 1957 +- 1 % in a uniform B_z "
                               "(chi ~ 1.9, the collision's peak), 48 steps, photons >= 2 m c^2 and pairs; "
                               "oracle run stored by tests/golden/make_qed_field_sample.py")

    # roofline of the first form's dominant kernel: the species push that takes
    # the most device time (per-species CUDA events in the timed region)
    s0 = runs[modes[0]]
    i_dom = int(np.argmax(s0["species_ms"]))
    per_launch_s = s0["species_ms"][i_dom] / 1e3 / max(1, s0["species_pushes"][i_dom])
    bpp = qed_bytes_per_particle(w.dim, photon=w.species[i_dom].kind == 1)
    alg = s0["alive_mid"][i_dom] * bpp
    achieved = alg / per_launch_s / 1e9
    kind = "photon push (pair rate" if w.species[i_dom].kind == 1 else "lepton push (gather, push, emission rate"
    kind += ", Monte Carlo" + (", surrogate network)" if modes[0] == "surrogate" else ", tables)")
    # DRAM bytes per particle of the dominant push from the committed ncu
    # summary (taken on a smaller beam, on the current kernel source), scaled
    # by the particles of one launch here
    trec = traffic_record(w.name)
    traffic = None
    if (trec and trec.get("form") == modes[0] and trec.get("species_kind") == w.species[i_dom].kind
            and "bytes_per_particle" in trec):
        traffic = trec["bytes_per_particle"] * s0["alive_mid"][i_dom]
    roof = {"bound": "hbm", "kernel": f"{kind}, species {w.species[i_dom].name}", "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_kind": f"{peak_kind} hbm_gbs",
            "traffic": traffic, "algorithmic_bytes_per_launch": alg, "avg_launch_ms": per_launch_s * 1e3,
            "bytes_per_particle": bpp, "particles_per_launch": s0["alive_mid"][i_dom],
            "share_of_step": s0["species_ms"][i_dom] / max(1e-30, float(sum(s0["prof"]["ms"].values())))}
    if modes[0] == "surrogate" and w.species[i_dom].kind == 1:
        # the network's arithmetic: 2*(2*64 + 64*64 + 64*64 + 64*2) flops per evaluation
        fl = s0["alive_mid"][i_dom] * 2.0 * (2 * 64 + 64 * 64 * 2 + 64 * 2)
        roof["tensor_tflops_if_every_photon_evaluates"] = fl / per_launch_s / 1e12

    # CPU baseline: the oracle on the collision's QED regime
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v1, i1 = oracle_qed_rate(n_e=64, steps=8)
        va, ia = oracle_qed_rate(n_e=32, steps=6, all_cores=True)
        cpu = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "the collision's QED regime: electrons of the qed_field_sample (gamma 1957 +- 1 %, chi ~ "
                         "1.9) with the photons and pairs they create, FP64 oracle (QED rates and spectra by "
                         "quadrature), 64 electrons, 8 steps", "seconds": i1["seconds"],
               "all_cores": {"value": va, "cores": ia["cores"], "seconds": ia["seconds"],
                             "sample": "32 electrons per core, 6 steps, one process per core"},
               "cpu": cpu_model(), "nproc": os.cpu_count()}

    if "steps_to_collision" in w.notes:
        where = f"the collision is at step {w.notes['steps_to_collision']}"
    else:
        where = f"the pulse peak reaches the foil at step {w.notes['steps_to_peak_at_foil']}"
    window = f"steps {pre + args.warmup}..{pre + args.warmup + K} ({where})"
    if rank == 0:
        s = runs[modes[0]]
        prof = s["prof"]
        tr = s["train"] or {}
        tab, f64 = runs.get("table"), runs.get("fp64")
        out = {"metric": METRIC, "value": s["value"], "unit": UNIT, "n_gpus": world, "steps": K,
               "warmup": args.warmup, "ms_per_step": s["ms_per_step"], "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": describe(w), "form": modes[0],
                          "precision": "fp32 cell+offset, QED by the surrogate networks inside their chi range "
                          "(tables outside); FP64 islands: optical depth, gamma above 1e4, diagnostics"
                          if modes[0] == "surrogate" else modes[0],
                          "window": window, "pusher": args.pusher,
                          "sort_interval": args.sort_interval, "replicas": world,
                          "l2": l2_note()},
               "fp32_table": tab and {"value": tab["value"], "ms_per_step": tab["ms_per_step"],
                                      "error_vs_fp64": errors(tab)},
               "fp64_plain": f64 and {"value": f64["value"], "ms_per_step": f64["ms_per_step"],
                                      "first_form_over_fp64": s["value"] / f64["value"]},
               "surrogate_error_vs_fp64": errors(runs.get("surrogate")),
               "error_vs_oracle": vs_oracle,
               "surrogate_training": {str(p): {k: v for k, v in r.items()} for p, r in tr.items()},
               "n_alive_end": {m: [int(v) for v in r["n_alive"]] for m, r in runs.items()},
               "gpu_launches": int(sum(prof["launches"].values())), "clocks": s["clocks"],
               "phases_ms_per_step": {k: v / K for k, v in prof["ms"].items()},
               "species_push_ms_per_step": {w.species[i].name: v / K for i, v in enumerate(s["species_ms"])},
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e}
        print(json.dumps(out))


def run_mlp_rows(n):
    """the two evaluations of the surrogate network (warp-level mma.sync,
    CTA-level tcgen05) on the same random network and inputs, twice each"""
    from paper_2104_00642_gb300 import pic
    sim = pic.pic_create(1, (16,), (1.0,), 0.02, [(-1.0, 1.0, 1e-12, 16, 0, 1), (0.0, 0.0, 1e-12, 16, 1, 0)])
    sim.pic_set_qed(photon_sp=1, electron_sp=0, lambda_r_m=1e-6)
    rng = np.random.default_rng(1)
    sim.pic_mlp_set(0, (rng.standard_normal(pic.MLP_NPARAMS) * 0.2).astype(np.float32), 1e-3, 1e2, 0.0, 1.0)
    x = rng.uniform(-1.0, 1.0, (n, 2)).astype(np.float32)
    out = {}
    for name in ("pic_mlp_eval", "pic_mlp_eval_tc") * 2:
        t = time.perf_counter()
        out[name] = getattr(sim, name)(0, x)
        out[name + "_s"] = time.perf_counter() - t
    d = np.abs(out["pic_mlp_eval"] - out["pic_mlp_eval_tc"])
    print(json.dumps({"rows": n, "wall_s_mma_sync": out["pic_mlp_eval_s"], "wall_s_tcgen05": out["pic_mlp_eval_tc_s"],
                      "max_abs_diff": float(d.max()), "frac_within_1e-5": float(np.mean(d <= 1e-5))}))
    sim.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=140)  # the QED collision: a timed region above one second
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="qed_collision_2d",
                    choices=["laser_foil_2d", "thermal_3d", "langmuir_1d", "qed_collision_2d", "qed_foil_3d"])
    ap.add_argument("--sort-interval", type=int, default=None,
                    help="steps between tile sorts (default: the measured best of the workload)")
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--pre", type=int, default=None,
                    help="untimed steps before the window (laser_foil_2d default: to the laser on the slab)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--per-step", action="store_true",
                    help="time single-step calls with the L2 flushed before each, whatever the workload size")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 form")
    ap.add_argument("--qed-beam", type=int, default=10_000_000, help="beam macro-electrons (qed_collision_2d)")
    ap.add_argument("--rows", type=int, default=None,
                    help="smaller case for profiling: ny of laser_foil_2d, nz of thermal_3d (not a bench line)")
    ap.add_argument("--qed-modes", default="surrogate,table,fp64", help="forms run by the QED workloads")
    ap.add_argument("--pusher", default="boris", choices=["boris", "vay"],
                    help="momentum update of every push (Sec. II.C: Boris, or Vay's for nearly cancelling forces)")
    ap.add_argument("--push-variant", type=int, default=0,
                    help="0: default kernels, 2: surrogate of the photon push per CTA on tcgen05 (QED workloads), "
                         "3: warp-aggregated deposit in the 2D tiled push")
    ap.add_argument("--mlp-rows", type=int, default=0,
                    help="instead of a PIC workload: evaluate a random surrogate network on this many rows with "
                         "the mma.sync and the tcgen05 kernels (profiling aid; kernel times come from ncu)")
    ap.add_argument("--qed-pair-chi-min", type=float, default=0.0,
                    help="lower end of the pair network's chi range (0: library default)")
    ap.add_argument("--qed-pre", type=int, default=None,
                    help="untimed steps before the window (default: to the collision; 0 for qed_foil_3d)")
    ap.add_argument("--qed-train-iters", type=int, default=0, help="surrogate training steps (0: library default)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.sort_interval is None:
        args.sort_interval = SORT_INTERVAL.get(args.workload, 8)
    if args.impl == "reference":
        run_reference(args)
        return
    if args.mlp_rows:
        run_mlp_rows(args.mlp_rows)
        return

    import torch

    from paper_2104_00642_gb300 import pic

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    stream = torch.cuda.Stream()
    w = make_workload(args.workload, rank, sample=args.rows, beam=args.qed_beam)
    npart = w.n_particles
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    continuous = not args.per_step and step_bytes(w) > L2_BYTES

    def l2_note():
        if continuous:
            return (f"not flushed: inputs larger than L2 (each step touches {step_bytes(w) / 1e6:.0f} MB, "
                    f"L2 {L2_BYTES / 1e6:.0f} MB); K steps in one pic_step call")
        return "flushed (256 MiB write) before every timed step" if not args.no_flush else "not flushed"

    def timed(sim, K, profile=False, per_step=None):
        """K steps between CUDA events on the simulation's stream: one
        pic_step(K) call when the workload outgrows the L2 (continuous),
        else K single-step calls with the L2 flushed before each.
        profile: the timed region proper; per-phase events on, and the CUDA
        profiler range opened (an ncu run with --profile-from-start off
        captures these launches only)."""
        one_call = continuous if per_step is None else not per_step
        if profile:
            sim.pic_profile(True)
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
        evs = []
        with torch.cuda.stream(stream):
            if one_call:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sim.pic_step(K)
                b.record(stream)
                evs.append((a, b))
            else:
                for _ in range(K):
                    if not args.no_flush:
                        flush.fill_(1.0)  # evict L2 between steps
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    sim.pic_step(1)
                    b.record(stream)
                    evs.append((a, b))
        torch.cuda.synchronize()
        if profile:
            torch.cuda.profiler.stop()
        ms = [a.elapsed_time(b) for a, b in evs]
        prof = sim.pic_profile_read() if profile else None
        if profile:
            sim.pic_profile(False)
        return ms, prof

    if args.workload in ("qed_collision_2d", "qed_foil_3d"):
        run_qed(args, w, pic, torch, stream, timed, rank, world, dist, local, l2_note)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    # ---- FP32 cell+offset: the headline ----------------------------------
    pre = args.pre
    if pre is None:
        pre = PRE_STEPS.get(args.workload, 0) if args.rows is None else 0
    sim = pic.from_workload(w, precision=pic.FP32_CELLOFF, sort_interval=args.sort_interval,
                            pusher=PUSHER[args.pusher], stream=stream.cuda_stream, push_variant=args.push_variant)
    if pre:
        with torch.cuda.stream(stream):
            sim.pic_step(pre)  # untimed: to the phase the window measures
    npart = sum(sim.pic_diagnostics()["n_alive"])
    timed(sim, args.warmup)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        ms, prof = timed(sim, args.steps, profile=True)
    t = max_over_ranks(float(np.sum(ms)) / 1e3, dist)
    value = world * npart * args.steps / t
    flushed = None
    if continuous:
        ms_f, _ = timed(sim, args.steps, per_step=True)
        flushed = {"value": npart * args.steps / (float(np.sum(ms_f)) / 1e3), "unit": UNIT,
                   "ms_per_step": float(np.mean(ms_f)), "note": "this rank, one step per call, L2 flushed before each"}
    diag = sim.pic_diagnostics()
    if not all(math.isfinite(v) for v in (diag["U_E"], diag["U_B"])):
        raise SystemExit("non-finite diagnostics")

    # roofline of the dominant kernel (the push kernel)
    peak, peak_kind = _peaks()
    push_ms = prof["ms"]["push"]
    push_launches = max(1, prof["push_launches"])
    per_launch_s = push_ms / 1e3 / push_launches
    occ = occupied_cells(w)
    bpp = bytes_per_particle(w.dim, 0)
    grid_b = (24 + 12) * occ  # gather 6 comps + deposit 3 comps, once per occupied cell
    alg_bytes_launch = (npart * bpp + len(w.species) * grid_b) / len(w.species)
    achieved = alg_bytes_launch / per_launch_s / 1e9
    trec = traffic_record(w.name)
    roof = {"bound": "hbm", "kernel": "push (gather+Boris+drift+Esirkepov)", "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_kind": f"{peak_kind} hbm_gbs",
            "traffic": (trec["bytes_per_launch"] if trec else None),
            "algorithmic_bytes_per_launch": alg_bytes_launch, "avg_launch_ms": per_launch_s * 1e3,
            "bytes_per_particle": bpp, "occupied_cells": occ}

    # ---- plain FP64 form on the same workload ------------------------------
    fp64 = None
    if not args.no_fp64:
        sim64 = pic.from_workload(w, precision=pic.FP64_PLAIN, sort_interval=args.sort_interval,
                                  pusher=PUSHER[args.pusher], stream=stream.cuda_stream)
        if pre:
            with torch.cuda.stream(stream):
                sim64.pic_step(pre)
        timed(sim64, 3)
        ms64, _ = timed(sim64, args.fp64_steps)
        v64 = npart * args.fp64_steps / (float(np.sum(ms64)) / 1e3)
        sim64.close()
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": float(np.sum(ms64)) / args.fp64_steps,
                "fp32_over_fp64": value / world / v64}

    # ---- end to end through the C ABI: the window's start state from a host
    # file (pic_restore), K steps, diagnostics read back, host wall clock ----
    e2e = None
    if not args.no_e2e and world == 1:
        fd, ckpt = tempfile.mkstemp(prefix="pic_window_", suffix=".ckpt",
                                    dir="/dev/shm" if os.path.isdir("/dev/shm") else None)
        os.close(fd)
        sim.pic_save(ckpt)  # the state after the timed window: the next window starts here
        size = os.path.getsize(ckpt)
        sim.close()
        sim_e = pic.from_workload(w, precision=pic.FP32_CELLOFF, sort_interval=args.sort_interval,
                                  pusher=PUSHER[args.pusher], stream=stream.cuda_stream, load=False, push_variant=args.push_variant)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim_e.pic_restore(ckpt)
        sim_e.pic_step(args.steps)
        d = sim_e.pic_diagnostics()
        el = time.perf_counter() - t0
        os.unlink(ckpt)
        d2h = 8 * (16 + 2 * len(w.species))
        e2e = {"value": npart * args.steps / el, "unit": UNIT,
               "h2d_bytes_per_step": size / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "seconds": el, "note": "pic_restore of the window's state from a host file (fields, particles) + "
                                      "pic_step(K) + pic_diagnostics, host wall clock"}
        assert math.isfinite(d["U_E"])
        sim_e.close()
    else:
        sim.close()

    # ---- CPU baseline (oracle, bounded sample, rank 0, N = 1) ---------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v_cpu, info = oracle_rate(args.workload, min_seconds=10.0)
        cpu = {"value": v_cpu, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": info["sample"]}

    if rank == 0:
        launches = int(sum(prof["launches"].values()))
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": describe(w), "precision": "fp32 cell+offset (FP64 islands: diagnostics)",
                          "sort_interval": args.sort_interval, "pusher": args.pusher,
                          "window": f"steps {pre + args.warmup}..{pre + args.warmup + args.steps}"
                                    + (" (the laser on the slab)" if args.workload == "laser_foil_2d" else ""),
                          "l2": l2_note(), "replicas": world, "qed": "off (no QED in this workload)"},
               "per_step_l2_flushed": flushed,
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clk.summary(),
               "fp64_plain": fp64,
               "phases_ms_per_step": {k: v / args.steps for k, v in prof["ms"].items()},
               "launches_per_step": {k: v / args.steps for k, v in prof["launches"].items()}}
        print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
