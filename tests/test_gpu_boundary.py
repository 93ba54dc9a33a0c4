"""The boundary calls around the step: pic_save / pic_restore, the borrowed
device view of a field (pic_field_device) and the caller's device allocator
(pic_options.alloc/free), through the C ABI on the GPU."""
import ctypes as C
import filecmp

import numpy as np
import pytest

from paper_2104_00642_gb300 import pic, workloads as W
from tests import qed_setup as Q
from tests.helpers import boundary_ambiguous

pytestmark = pytest.mark.gpu


def _laser_foil_small():
    return W.laser_foil_2d(nx=256, ny=64, cells_per_lambda=32, slab=(128, 144), ppc=8, fwhm_fs=5.0,
                           x_focus_cell=128)


def _jscale(w):
    """the summed size of the current terms at a node: every particle of a
    cell's neighbourhood adds up to |q w| dx/dt"""
    return sum(abs(s.q * s.w) for s in w.species) * 8 * max(w.dx[:w.dim]) / w.dt


def _compare_runs(a, b, nsp, dx, tol=1e-5, jscale=None):
    """two simulations after the same steps: the same particles in the same
    order (positions within tol of a cell, cells equal away from faces),
    momenta within tol (|u| + the species' rms |u|), fields within tol of
    their maximum, currents within tol of jscale (the size of the terms they
    sum: the order of the atomic sums moves a node by a few ulp of each
    term, and the fields it drives move every particle's momentum by about
    that fraction of the typical momentum, not of its own)"""
    for sp in range(nsp):
        pa, pb = a.pic_get_particles(sp), b.pic_get_particles(sp)
        assert len(pa["ux"]) == len(pb["ux"]), sp
        if not len(pa["ux"]):
            continue
        assert np.array_equal(pa["alive"], pb["alive"])
        umag = np.sqrt(pb["ux"] ** 2 + pb["uy"] ** 2 + pb["uz"] ** 2)
        urms = float(np.sqrt(np.mean(umag ** 2)))
        for k in ("ux", "uy", "uz"):
            assert np.all(np.abs(pa[k] - pb[k]) <= tol * (umag + urms) + 1e-12), (sp, k)
        ca, bits = a.pic_get_cells(sp)
        cb, _ = b.pic_get_cells(sp)
        amb = np.zeros(len(ca), dtype=bool)
        for d, k in enumerate(("x", "y", "z")[:len(dx)]):
            amb |= boundary_ambiguous(pb[k], dx[d])
        assert np.array_equal(ca[~amb], cb[~amb]), sp
    # fields against the scale of all field components (a small component
    # carries the others' rounding), currents against the currents' scale
    fa = [a.pic_fields(c) for c in range(9)]
    fb = [b.pic_fields(c) for c in range(9)]
    emax = max(np.max(np.abs(f)) for f in fb[:6])
    jmax = jscale if jscale is not None else max(max(np.max(np.abs(f)) for f in fb[6:]), 1e-30)
    for c in range(9):
        scale = emax if c < 6 else jmax
        assert np.max(np.abs(fa[c] - fb[c])) <= tol * scale, c


@pytest.mark.parametrize("prec", [pic.FP32_CELLOFF, pic.FP64_PLAIN])
def test_save_restore_continues_the_run(prec, tmp_path):
    """N steps + save + restore into a fresh simulation + N steps equals 2N
    steps taken as N + N: same particles in the same order, same cells, same
    sort phase (the interval is 4 and the save falls between sorts), fields
    and momenta within the tolerance of the atomic summation order."""
    w = _laser_foil_small()
    kw = dict(precision=prec, sort_interval=4)
    ref = pic.from_workload(w, **kw)
    run = pic.from_workload(w, **kw)
    ref.pic_step(10)
    ref.pic_step(10)
    run.pic_step(10)
    path = str(tmp_path / "a.ckpt")
    run.pic_save(path)
    run.close()
    new = pic.from_workload(w, load=False, **kw)
    new.pic_restore(path)
    assert new.pic_diagnostics()["step"] == 10
    new.pic_step(10)
    _compare_runs(new, ref, len(w.species), w.dx[:2], tol=1e-5 if prec == pic.FP32_CELLOFF else 1e-10,
                  jscale=_jscale(w))
    dn, dr = new.pic_diagnostics(), ref.pic_diagnostics()
    assert dn["step"] == dr["step"] == 20
    assert abs(dn["U_E"] - dr["U_E"]) <= 1e-5 * dr["U_E"]


def test_save_restore_round_trip_is_byte_exact(tmp_path):
    """restoring a file and saving again writes the same bytes"""
    w = _laser_foil_small()
    s = pic.from_workload(w, sort_interval=4)
    s.pic_step(6)
    a, b = str(tmp_path / "a.ckpt"), str(tmp_path / "b.ckpt")
    s.pic_save(a)
    t = pic.from_workload(w, sort_interval=4, load=False)
    t.pic_restore(a)
    t.pic_save(b)
    assert filecmp.cmp(a, b, shallow=False)


@pytest.mark.parametrize("prec", [pic.FP32_CELLOFF, pic.FP64_PLAIN])
def test_save_restore_keeps_the_qed_monte_carlo(prec, tmp_path):
    """QED on: after the restore the same electrons emit the same photons
    (identities from the parents' Philox counters at the restored step) with
    the same optical depths as the run that did not stop."""
    def make():
        s = pic.pic_create(1, (16,), (1.0,), Q.DT, Q.species_spec(), seed=Q.SEED, precision=prec)
        s.pic_set_qed(photon_sp=2, electron_sp=0, positron_sp=1, lambda_r_m=Q.LAMBDA)
        return s
    ref, run = make(), make()
    for s in (ref, run):
        s.pic_set_field(pic.BZ, np.full(s.box(), Q.B0))
        s.pic_load_particles(0, *Q.electrons())
        s.pic_step(12)
    ref.pic_step(12)
    path = str(tmp_path / "q.ckpt")
    run.pic_save(path)
    new = make()
    new.pic_restore(path)
    new.pic_step(12)
    for sp in range(3):
        ia, ta = new.pic_get_qed_state(sp)
        ib, tb = ref.pic_get_qed_state(sp)
        assert np.array_equal(ia, ib), sp
        assert np.all(np.abs(ta - tb) <= 1e-5 * np.abs(tb) + 1e-12), sp
    assert len(ref.pic_get_qed_state(2)[0]) > 30


def test_restore_refuses_another_configuration(tmp_path):
    w = _laser_foil_small()
    s = pic.from_workload(w, sort_interval=4)
    path = str(tmp_path / "c.ckpt")
    s.pic_save(path)
    other = pic.from_workload(w, sort_interval=8, load=False)
    with pytest.raises(pic.PicError) as e:
        other.pic_restore(path)
    assert e.value.code == -1 and "configuration" in str(e.value)
    with pytest.raises(pic.PicError) as e:
        other.pic_restore(str(tmp_path / "missing.ckpt"))
    assert e.value.code == -1


# ----------------------------------------------------------------------
# borrowed device view: read with the CUDA runtime's cudaMemcpy (ctypes)
# ----------------------------------------------------------------------

def _cudart():
    import glob
    import os
    cands = glob.glob("/usr/local/cuda/lib64/libcudart.so*")
    try:
        import nvidia
        for p in nvidia.__path__:
            cands += glob.glob(os.path.join(p, "*", "lib", "libcudart.so*"))
    except Exception:
        pass
    for c in sorted(cands):
        try:
            return C.CDLL(c)
        except OSError:
            continue
    pytest.fail("no CUDA runtime library to read device memory with")


def _read_device(ptr, n, elem_bytes):
    """n elements at device address ptr, copied to the host (not owned)"""
    rt = _cudart()
    out = np.zeros(n, dtype=np.float64 if elem_bytes == 8 else np.float32)
    rt.cudaMemcpy.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]
    rc = rt.cudaMemcpy(out.ctypes.data_as(C.c_void_p), C.c_void_p(ptr), n * elem_bytes, 2)  # device to host
    assert rc == 0, rc
    return out


@pytest.mark.parametrize("prec", [pic.FP32_CELLOFF, pic.FP64_PLAIN])
def test_field_device_view_reads_the_resident_arrays(prec):
    """pic_field_device: element origin + i + j sy + k sz of the borrowed
    array is the value pic_fields copies out at (i, j, k), for every
    component, including the periodic ghost layers' images."""
    w = _laser_foil_small()
    s = pic.from_workload(w, precision=prec, sort_interval=4)
    s.pic_step(30)
    s.pic_sync()
    for c in range(9):
        v = s.pic_field_device(c)
        assert v["elem_bytes"] == (8 if prec == pic.FP64_PLAIN else 4)
        host = s.pic_fields(c)[0]  # (ny, nx + 1): absorbing x, periodic y
        ny, nx1 = host.shape
        # one past the last element of the padded box (the component's
        # allocation may end right there)
        span = v["origin"] + v["hi"][1] * v["stride"][1] + v["hi"][0] + 1
        t = _read_device(v["data"], span, v["elem_bytes"])
        jj, ii = np.meshgrid(np.arange(ny), np.arange(nx1), indexing="ij")
        got = t[v["origin"] + ii + jj * v["stride"][1]].astype(np.float64)
        assert np.array_equal(got, host), c
        # a periodic ghost row holds its image
        assert v["lo"][1] == -4 and v["hi"][1] == ny + 3
        g = t[v["origin"] + np.arange(nx1) + (-1) * v["stride"][1]].astype(np.float64)
        assert np.array_equal(g, host[ny - 1]), c


def test_caller_allocator_serves_every_block():
    """With PyTorch's caching allocator passed as pic_options.alloc/free the
    simulation runs as with cudaMalloc (same results within the atomic order
    tolerance), every block it takes comes from that allocator (temporary
    ones of pic_get_particles included), and pic_destroy returns them all."""
    import torch
    w = _laser_foil_small()
    A = pic.TorchAllocator()
    before = torch.cuda.memory_allocated()
    s = pic.from_workload(w, sort_interval=4, allocator=A)
    r = pic.from_workload(w, sort_interval=4)
    assert not A.errors, A.errors
    assert A.allocated > 10 and torch.cuda.memory_allocated() > before
    n_state = len(A.live)  # blocks held by the simulation (the upload's staging came and went)
    for t in (s, r):
        t.pic_step(12)
    a0 = A.allocated
    _compare_runs(s, r, len(w.species), w.dx[:2], jscale=_jscale(w))
    assert A.allocated > a0 and len(A.live) == n_state  # temporaries of the read-backs came back
    s.close()
    assert A.freed == A.allocated and not A.live
