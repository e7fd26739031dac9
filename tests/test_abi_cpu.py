"""The C ABI library loads, exports every declared entry point and rejects
invalid requests on the host before touching a device (CPU only)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gpjc.h")


@pytest.fixture(scope="module")
def gpjc():
    import __graft_entry__ as ge

    ge.build()
    from paper_2601_05418_gb300 import gpjc as m

    return m


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(gpjc_[A-Za-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_five_hot_path_calls():
    names = declared_functions()
    for n in ("gpjc_build_groups", "gpjc_compress", "gpjc_apply_E", "gpjc_apply_EH", "gpjc_recon"):
        assert n in names


def test_every_declared_symbol_is_exported(gpjc):
    lib = gpjc.lib()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_version(gpjc):
    lib = gpjc.lib()
    for s in range(7):
        assert lib.gpjc_strerror(s)
    assert b"sm_103a" in lib.gpjc_version()


def _geom(gpjc, **kw):
    from paper_2601_05418_gb300 import synth

    g = synth.tiny_geometry(nx=8, ny=6, nz=1, nc=2, os=2, cycles=2.0, n_groups=2, keep=3, lines="regular")
    for k, v in kw.items():
        setattr(g, k, v)
    return g


@pytest.mark.parametrize("change,needle", [
    (dict(nx=7), "even"),
    (dict(ny=0), "even"),
    (dict(nc=0), "nc"),
    (dict(w=3), "w must divide"),
    (dict(nx=22), "products of 2, 3, 5, 7"),
    (dict(keep=np.array([0, 3], np.int32)), "keep"),
    (dict(keep=np.array([3, 99], np.int32)), "keep"),
    (dict(patch_group=np.array([0, 0, 0, 0], np.int32)), "no patch"),
    (dict(patch_group=np.array([0, 1, 2, 0], np.int32)), "out of range"),
    (dict(line_ky=np.array([2, 0, 4], np.int32), line_kz=np.zeros(3, np.int32)), "sorted"),
    (dict(line_ky=np.array([0, 6], np.int32), line_kz=np.zeros(2, np.int32)), "outside"),
    (dict(cycles=float("nan")), "finite"),
])
def test_plan_validation_rejects_before_launch(gpjc, change, needle):
    g = _geom(gpjc, **change)
    with pytest.raises(gpjc.GpjcError) as ei:
        gpjc.Plan(g)
    assert ei.value.status == gpjc.GPJC_EINVAL
    assert needle in str(ei.value)


def test_null_arguments(gpjc):
    lib = gpjc.lib()
    out = C.c_void_p()
    assert lib.gpjc_plan_create(None, C.byref(out)) == gpjc.GPJC_EINVAL
    assert lib.gpjc_apply_E(None, None, None, None) == gpjc.GPJC_EINVAL
    assert lib.gpjc_apply_EH(None, None, None, None) == gpjc.GPJC_EINVAL
    assert lib.gpjc_compress(None, None, None, 0, None) == gpjc.GPJC_EINVAL
    assert lib.gpjc_recon(None, None, None, None, None, None) == gpjc.GPJC_EINVAL
    assert lib.gpjc_build_groups(None, None, None, None, None, None, C.byref(out)) == gpjc.GPJC_EINVAL
    assert b"null" in lib.gpjc_last_error()


def test_keep_from_energy_matches_oracle(gpjc):
    """The host-only keep policy of the C ABI takes the same integer decision
    as the oracle (same FP64 running sums in index order) on random spectra
    with ties, zeros and tiny negative values, with and without a trace."""
    import oracle as O

    rng = np.random.default_rng(11)
    for trial in range(300):
        G, m = int(rng.integers(1, 6)), int(rng.integers(1, 40))
        ev = -np.sort(-np.round(rng.exponential(1.0, (G, m)), int(rng.integers(1, 4))), axis=1)
        ev[:, -1] -= 1e-16 * rng.integers(0, 2, G)
        tau = float(rng.choice([0.25, 0.5, 0.9, 0.99, 1.0, rng.uniform(0.01, 1.0)]))
        trace = None if trial % 3 == 0 else float(np.sum(np.maximum(ev, 0), axis=1).max() * rng.uniform(1.0, 1.5))
        got = gpjc.keep_from_energy(ev, tau, trace)
        want = O.keep_from_energy(ev, tau, trace)
        assert np.array_equal(got, want.astype(np.int32)), (trial, got, want)


def test_keep_from_energy_rejects_bad_input(gpjc):
    ev = np.array([[3.0, 2.0, 1.0]])
    for tau in (0.0, -0.1, 1.5, float("nan")):
        with pytest.raises(gpjc.GpjcError) as ei:
            gpjc.keep_from_energy(ev, tau)
        assert ei.value.status == gpjc.GPJC_EINVAL
    with pytest.raises(gpjc.GpjcError) as ei:
        gpjc.keep_from_energy(np.array([[3.0, float("inf")]]), 0.5)
    assert ei.value.status == gpjc.GPJC_ENONFINITE
    with pytest.raises(gpjc.GpjcError) as ei:
        gpjc.keep_from_energy(ev, 0.5, trace=-1.0)
    assert ei.value.status == gpjc.GPJC_EINVAL


def test_tv_grad_rejects_bad_input_before_launch(gpjc):
    lib = gpjc.lib()
    buf = C.c_void_p(16)  # never dereferenced: every call below fails validation first
    assert lib.gpjc_tv_grad(None, 1, 4, 4, 0.1, buf, None) == gpjc.GPJC_EINVAL
    assert lib.gpjc_tv_grad(buf, 1, 4, 4, 0.1, None, None) == gpjc.GPJC_EINVAL
    assert lib.gpjc_tv_grad(buf, 0, 4, 4, 0.1, C.c_void_p(32), None) == gpjc.GPJC_EINVAL
    assert lib.gpjc_tv_grad(buf, 1, 4, 4, 0.0, C.c_void_p(32), None) == gpjc.GPJC_EINVAL
    assert lib.gpjc_tv_grad(buf, 1, 4, 4, float("nan"), C.c_void_p(32), None) == gpjc.GPJC_EINVAL
    assert lib.gpjc_tv_grad(buf, 1, 4, 4, 0.1, buf, None) == gpjc.GPJC_EINVAL
