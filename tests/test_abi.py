"""The C-ABI library builds, loads and exports every symbol include/fpd.h
declares; host-side parameter validation works without a GPU (no compute
call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(fpd_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2212_14153_gb300 import build, fpd
    build.build()
    return fpd.load_library()


def test_library_exports_every_declared_symbol(lib):
    declared = _declared_symbols()
    assert {"fpd_create", "fpd_step", "fpd_read_fields", "fpd_read_beads", "fpd_destroy"} <= declared
    raw = ctypes.CDLL(os.path.join(ROOT, "paper_2212_14153_gb300", "libfpd.so"))
    for name in sorted(declared):
        assert hasattr(raw, name), name
    from paper_2212_14153_gb300 import fpd
    assert set(fpd.SIGNATURES) == declared


def test_version_and_defaults(lib):
    from paper_2212_14153_gb300 import fpd
    assert fpd.fpd_version() == 4
    assert fpd.fpd_sweep_variants() == 5
    p = fpd.fpd_default_params()
    assert (p.nx, p.ny, p.u_bottom, p.u_top, p.visc_ratio, p.phi_cut) == (80, 40, -0.01, 0.01, 50.0, 8.0)
    assert p.precision == fpd.FPD_F64 and p.collision == fpd.FPD_MRT_MAGIC


@pytest.mark.parametrize("field,value,needle", [
    ("nx", 0, "nx and ny"),
    ("precision", 7, "precision"),
    ("collision", 5, "collision"),
    ("n_beads", 300, "at most"),
    ("visc_ratio", -1.0, "visc_ratio"),
    ("xi", 0.0, "xi"),
    ("periodic_y", 2, "periodic_y"),
    ("bead_force_x", float("nan"), "bead_force"),
    ("sandwich_zl", 5.0, "sandwich"),      # with periodic_y below
])
def test_invalid_parameters_rejected_before_any_device_call(lib, field, value, needle):
    from paper_2212_14153_gb300 import fpd
    import numpy as np
    p = fpd.fpd_default_params()
    p.n_beads, p.n_fibers = 8, 1
    cen = np.array([40.0, 20.0]); th = np.array([0.5])
    p.centre_xy = cen.ctypes.data_as(fpd._DP)
    p.theta0 = th.ctypes.data_as(fpd._DP)
    setattr(p, field, value)
    if field == "sandwich_zl":
        p.sandwich_zr, p.periodic_y = 10.0, 1
    with pytest.raises(fpd.FpdError) as e:
        fpd.fpd_create(p, None)
    assert e.value.code == fpd.FPD_EINVAL
    assert needle in str(e.value)


def test_missing_fiber_placement_rejected(lib):
    from paper_2212_14153_gb300 import fpd
    p = fpd.fpd_default_params()
    p.n_beads, p.n_fibers = 4, 1
    with pytest.raises(fpd.FpdError) as e:
        fpd.fpd_create(p, None)
    assert "centre_xy" in str(e.value)


def test_viscosity_derivation_needs_re_and_shear(lib):
    from paper_2212_14153_gb300 import fpd
    p = fpd.fpd_default_params()
    p.u_bottom = p.u_top = 0.0   # no shear, no fiber, nu_f <= 0
    with pytest.raises(fpd.FpdError) as e:
        fpd.fpd_create(p, None)
    assert "nu_f" in str(e.value)


def test_missing_library_fails_loudly(tmp_path):
    from paper_2212_14153_gb300 import fpd
    with pytest.raises(RuntimeError, match="missing"):
        fpd.load_library.__wrapped__(str(tmp_path / "nope.so")) if hasattr(fpd.load_library, "__wrapped__") \
            else _load_fresh(fpd, str(tmp_path / "nope.so"))


def _load_fresh(fpd, path):
    saved = fpd._lib
    fpd._lib = None
    try:
        return fpd.load_library(path)
    finally:
        fpd._lib = saved


def test_workspace_bytes_without_a_device(lib):
    # the size query is host-only: the state layout of the parameters
    from paper_2212_14153_gb300 import fpd
    import numpy as np
    p = fpd.fpd_default_params()
    p.n_beads, p.n_fibers = 8, 1
    cen = np.array([40.0, 20.0]); th = np.array([0.5])
    p.centre_xy = cen.ctypes.data_as(fpd._DP)
    p.theta0 = th.ctypes.data_as(fpd._DP)
    for prec, es in ((0, 8), (1, 4), (2, 2)):
        p.precision = prec
        n = fpd.fpd_workspace_bytes(p)
        pitch = -(-p.nx // 32) * 32  # width padded to whole 32-column strips
        assert n % 256 == 0 and n >= 9 * pitch * p.ny * es
    p.nx = 0
    with pytest.raises(fpd.FpdError) as e:
        fpd.fpd_workspace_bytes(p)
    assert e.value.code == fpd.FPD_EINVAL


def test_async_bead_reads_reject_a_null_handle(lib):
    # host-only argument checks of the stream-ordered bead read
    t = ctypes.c_uint64(0)
    buf = (ctypes.c_double * 7)()
    from paper_2212_14153_gb300 import fpd
    assert lib.fpd_read_beads_async(None, ctypes.cast(buf, ctypes.c_void_p), ctypes.byref(t)) == fpd.FPD_EINVAL
    assert lib.fpd_wait_read(None, ctypes.c_uint64(0)) == fpd.FPD_EINVAL


def test_bead_export_rejects_a_null_handle(lib):
    from paper_2212_14153_gb300 import fpd
    buf = (ctypes.c_double * 7)()
    assert lib.fpd_export_beads(None, 4) == fpd.FPD_EINVAL
    assert lib.fpd_take_beads(None, 2, ctypes.cast(buf, fpd._DP)) == fpd.FPD_EINVAL


def test_autotune_cache_key_names_the_library_build(tmp_path, monkeypatch):
    # cached launch-shape timings belong to one build of the kernels: a
    # rebuilt library (another stamp) must not reuse them
    from paper_2212_14153_gb300 import autotune, build
    from paper_2212_14153_gb300 import workloads as wl
    cfg = wl.couette_only(40, 24, precision=1)
    monkeypatch.setattr(build, "OUT_DIR", str(tmp_path))
    assert "|libunbuilt|" in autotune._key(cfg, "GPU")
    (tmp_path / "stamp").write_text("a" * 64)
    k1 = autotune._key(cfg, "GPU")
    (tmp_path / "stamp").write_text("b" * 64)
    k2 = autotune._key(cfg, "GPU")
    assert k1 != k2 and "|p1|40x24|" in k1
