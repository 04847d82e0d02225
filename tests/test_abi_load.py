"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/frost.h declares (no compute call: this runs without a GPU)."""

import os
import re

from paper_2011_14984_gb300 import build, frost

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(frost_[a-z_0-9]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("frost_init", "frost_accel_gradient", "frost_timesteps", "frost_step",
                     "frost_energy_momentum", "frost_partition", "frost_kick", "frost_drift",
                     "frost_destroy", "frost_last_error"):
        assert required in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    lib = frost.load()
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing
    assert "sm_103a" in frost.frost_version()
    opts = frost.frost_default_opts()
    assert opts.precision == frost.FROST_PREC_MIXED and opts.max_depth == 40


def test_binding_wraps_every_declared_function():
    for name in declared_functions():
        assert hasattr(frost, name), name


def test_init_rejects_bad_options_before_touching_the_device():
    """Argument checks of frost_init run on the host before any CUDA call, so they can be
    exercised here: bad sizes, G, eta, precision, symmetrisation, integrator and team size."""
    import numpy as np
    import pytest

    m = np.ones(4)
    x = np.zeros((4, 3))
    v = np.zeros((4, 3))
    cases = [dict(subtree_blocks=9), dict(subtree_blocks=-1), dict(precision=7), dict(sym=3),
             dict(integrator=5)]
    for fields in cases:
        o = frost.frost_default_opts()
        for k, val in fields.items():
            setattr(o, k, val)
        with pytest.raises(frost.FrostError) as e:
            frost.frost_init(m, x, v, 1.0, 0.2, o)
        assert e.value.code == frost.FROST_EINVAL, (fields, str(e.value))
    with pytest.raises(frost.FrostError):
        frost.frost_init(m, x, v, -1.0, 0.2)
