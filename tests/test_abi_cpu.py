"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every
symbol include/sic.h declares, and rejects bad input before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sic.h")


@pytest.fixture(scope="module")
def sic():
    from paper_1506_07207_gb300 import build
    build.build()
    from paper_1506_07207_gb300 import sic as binding
    return binding


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sic_[a-z_]+)\s*\(", text)))


def test_header_symbols_are_exported(sic):
    names = _declared()
    assert len(names) >= 14
    lib = ctypes.CDLL(sic.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(sic.EXPORTS) == names


def test_header_constants_match_the_binding(sic):
    """Every integer constant the header defines has the same value in the
    binding wherever the binding names it (error codes, limits, deposit
    schemes, the autotuner's candidate count)."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    consts = {}
    for name, val in re.findall(r"^#define\s+(SIC_[A-Z0-9_]+)\s+(\(?-?\d+\)?)\s*$", text, flags=re.M):
        consts[name] = int(val.strip("()"))
    assert {"SIC_OK", "SIC_NX_MAX", "SIC_AUTOTUNE_CANDIDATES", "SIC_DEPOSIT_PIC_CIC"} <= set(consts)
    checked = 0
    for name, val in consts.items():
        if hasattr(sic, name):
            assert getattr(sic, name) == val, name
            checked += 1
    assert checked >= 12


def test_library_is_built_for_sm103a_only(sic):
    """Every compile and the link name one target, sm_103a (real code for
    that architecture, no PTX for others)."""
    from paper_1506_07207_gb300 import build
    cmds = [build.compile_command(s) for s in build.SOURCES] + [build.link_command(build.LIB)]
    for cmd in cmds:
        gencodes = [cmd[i + 1] for i, a in enumerate(cmd) if a == "-gencode"]
        assert gencodes == ["arch=compute_103a,code=sm_103a"], cmd
        assert not any(a.startswith(("-arch", "--gpu-architecture")) for a in cmd), cmd


def test_strerror(sic):
    assert sic.sic_strerror(0) == "ok"
    for code in range(-8, 0):
        assert sic.sic_strerror(code) not in ("ok", "unknown error")
    assert sic.sic_strerror(-99) == "unknown error"


def _base(**kw):
    args = dict(nx=8, L=1.0, dt=0.1, counts=[4], closed=[1], winding=[1],
                x=np.arange(4) / 4.0, v=np.zeros(4), w=np.full(4, 0.25))
    args.update(kw)
    return args


@pytest.mark.parametrize("bad", [
    dict(nx=1), dict(nx=8193), dict(L=0.0), dict(L=float("nan")), dict(dt=-1.0),
    dict(counts=[1], x=[0.0], v=[0.0], w=[1.0]),
    dict(x=np.array([0.0, float("inf"), 0.5, 0.7])),
    dict(v=np.array([0.0, float("nan"), 0.0, 0.0])),
    dict(w=np.array([0.25, 0.0, 0.25, 0.25])),
    dict(w=np.array([0.25, -1.0, 0.25, 0.25])),
])
def test_invalid_input_is_rejected(sic, bad):
    a = _base(**bad)
    with pytest.raises(sic.SicError) as e:
        sic.Sim.sic_create(a["nx"], a["L"], a["dt"], a["counts"], a["closed"], a["winding"],
                           a["x"], a["v"], a["w"])
    assert e.value.code == sic.SIC_EINVAL


def test_position_out_of_fixed_point_range(sic):
    a = _base(x=np.array([0.0, 0.25, 0.5, 2.0 ** 27]))   # 2^30 cells
    with pytest.raises(sic.SicError) as e:
        sic.Sim.sic_create(a["nx"], a["L"], a["dt"], a["counts"], a["closed"], a["winding"],
                           a["x"], a["v"], a["w"])
    assert e.value.code == sic.SIC_ERANGE


def test_bad_config_fields(sic):
    a = _base()
    for kw in (dict(qm=0.0), dict(history_len=0), dict(qm=float("inf"))):
        with pytest.raises(sic.SicError) as e:
            sic.Sim.sic_create(a["nx"], a["L"], a["dt"], a["counts"], a["closed"], a["winding"],
                               a["x"], a["v"], a["w"], **kw)
        assert e.value.code == sic.SIC_EINVAL
    with pytest.raises(sic.SicError):
        sic.Sim.sic_create_horizontal(8, 1.0, 0.1, [0.0], [0.0], [1.0])   # one tracer
    with pytest.raises(sic.SicError):
        sic.Sim.sic_create_horizontal(8, 1.0, 0.1, [0.0, 0.5], [0.0], [-1.0])


def test_server_rejects_bad_config(sic):
    for kw in (dict(hbm_budget=0), dict(max_active=0), dict(chunk_steps=0)):
        args = dict(hbm_budget=1 << 30, max_active=4, chunk_steps=8)
        args.update(kw)
        with pytest.raises(sic.SicError) as e:
            sic.Server(**args)
        assert e.value.code == sic.SIC_EINVAL


def test_bad_deposit_scheme(sic):
    a = _base()
    for dep in (-1, 5, 99):
        with pytest.raises(sic.SicError) as e:
            sic.Sim.sic_create(a["nx"], a["L"], a["dt"], a["counts"], a["closed"], a["winding"],
                               a["x"], a["v"], a["w"], order=dep)
        assert e.value.code == sic.SIC_EINVAL


def test_null_handles_are_rejected(sic):
    """Every entry point that takes a simulation refuses a null one before it
    touches the GPU."""
    lib = ctypes.CDLL(sic.LIB_PATH)
    lib.sic_refine.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
    lib.sic_moments.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    lib.sic_sheet_counts.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.sic_history.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    lib.sic_step.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    lib.sic_step_batch_static.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    assert lib.sic_refine(None, 1.0, None) == sic.SIC_EINVAL
    assert lib.sic_moments(None, 0, None, None) == sic.SIC_EINVAL
    assert lib.sic_sheet_counts(None, None) == sic.SIC_EINVAL
    assert lib.sic_history(None, None, 4, None) == sic.SIC_EINVAL
    assert lib.sic_step(None, 1) == sic.SIC_EINVAL
    assert lib.sic_step_batch_static(None, 1, None) == sic.SIC_EINVAL


def test_refinement_settings_are_checked(sic):
    """refine_length at least 2^-10 of a cell, refine_split within
    (0, refine_length], max_tracers within [0, SIC_TRACERS_MAX]; rejected
    before anything reaches the GPU."""
    a = _base()
    for kw in (dict(refine=-1.0), dict(refine=float("nan")), dict(refine=1e-7),
               dict(refine=0.2, refine_split=0.3), dict(refine=0.2, refine_split=-0.1),
               dict(refine=0.2, max_tracers=-1), dict(refine=0.2, max_tracers=(1 << 28) + 1),
               dict(refine=0.2, order=2)):
        with pytest.raises(sic.SicError) as e:
            sic.Sim.sic_create(a["nx"], a["L"], a["dt"], a["counts"], a["closed"], a["winding"],
                               a["x"], a["v"], a["w"], **kw)
        assert e.value.code == sic.SIC_EINVAL, kw
    assert sic.sic_strerror(sic.SIC_ELIMIT) != "unknown error"


def test_charge_unit_is_checked(sic):
    """A given fixed-point unit must be positive and coarse enough that every
    particle's charge fits 2^28 units; checked before the GPU is touched."""
    a = _base()
    with pytest.raises(sic.SicError) as e:
        sic.Sim.sic_create(a["nx"], a["L"], a["dt"], a["counts"], a["closed"], a["winding"],
                           a["x"], a["v"], a["w"], charge_unit=-1.0)
    assert e.value.code == sic.SIC_EINVAL
    with pytest.raises(sic.SicError) as e:
        sic.Sim.sic_create(a["nx"], a["L"], a["dt"], a["counts"], a["closed"], a["winding"],
                           a["x"], a["v"], a["w"], charge_unit=1e-12)
    assert e.value.code == sic.SIC_ERANGE


def test_fourier_mode_is_checked(sic):
    """mode_k within [0, nx/2], rejected before the GPU is touched; the
    diagnostic calls reject null handles and unknown fields."""
    a = _base()
    for k in (-1, a["nx"] // 2 + 1):
        with pytest.raises(sic.SicError) as e:
            sic.Sim.sic_create(a["nx"], a["L"], a["dt"], a["counts"], a["closed"], a["winding"],
                               a["x"], a["v"], a["w"], mode_k=k)
        assert e.value.code == sic.SIC_EINVAL, k
    lib = sic._lib
    rows = ctypes.c_int32()
    buf = np.zeros(4)
    assert lib.sic_mode_history(None, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 4,
                                ctypes.byref(rows)) == sic.SIC_EINVAL
    assert lib.sic_spectrum(None, 0, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == sic.SIC_EINVAL
