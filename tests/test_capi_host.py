"""CPU checks of the C-ABI library: it builds, loads, exports every symbol
that include/mpcgpu.h declares, and the binding's struct layouts match C.
No compute call is made (no GPU here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpcgpu.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2510_12717_b300 import mpcgpu
    return mpcgpu.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpc_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_2510_12717_b300 import mpcgpu
    assert set(_declared()) == set(mpcgpu.SIGNATURES)


def test_struct_layouts_match(lib):
    from paper_2510_12717_b300 import mpcgpu
    assert mpcgpu.MODEL_DTYPE.itemsize == C.sizeof(mpcgpu.MpcAgentModel)
    for name in mpcgpu.MODEL_DTYPE.names:
        assert mpcgpu.MODEL_DTYPE.fields[name][1] == getattr(mpcgpu.MpcAgentModel, name).offset, name
    assert mpcgpu.TREE_DTYPE.itemsize == C.sizeof(mpcgpu.MpcTreeModel)
    for name in mpcgpu.TREE_DTYPE.names:
        assert mpcgpu.TREE_DTYPE.fields[name][1] == getattr(mpcgpu.MpcTreeModel, name).offset, name


def test_pack_trees_roundtrip():
    from paper_2510_12717_b300 import mpcgpu
    from workload import make_trees
    t = make_trees("small", np.arange(3))
    recs = mpcgpu.pack_trees(t, [2, 0])
    np.testing.assert_array_equal(recs["axis"][0], t["tree_axis"][2])
    np.testing.assert_array_equal(recs["inertia"][1], t["tree_inertia"][0])
    assert np.allclose(np.linalg.norm(recs["axis"], axis=-1), 1.0)


def test_default_config_and_argument_errors(lib):
    from paper_2510_12717_b300 import mpcgpu
    cfg = mpcgpu.MpcConfig()
    assert lib.mpc_default_config(C.byref(cfg)) == 0
    assert cfg.max_horizon == 20 and abs(cfg.rho0 - 0.1) < 1e-7 and cfg.polish == 1
    assert cfg.kin_rows == 0 and abs(cfg.swing_height - 0.075) < 1e-7
    assert abs(cfg.v_takeoff - 0.1) < 1e-7 and abs(cfg.v_touchdown + 0.1) < 1e-7
    h = C.c_void_p()
    bad = mpcgpu.MpcConfig()
    lib.mpc_default_config(C.byref(bad))
    bad.max_agents = 0
    assert lib.mpc_create(C.byref(bad), C.byref(h)) == mpcgpu.MPC_ERR_INVALID
    bad.max_agents = 16
    bad.max_horizon = 99
    assert lib.mpc_create(C.byref(bad), C.byref(h)) == mpcgpu.MPC_ERR_INVALID
    bad.max_horizon = 20
    bad.precision = 7                 # not a precision
    assert lib.mpc_create(C.byref(bad), C.byref(h)) == mpcgpu.MPC_ERR_INVALID
    bad.precision = mpcgpu.BF16
    bad.refine_steps = 9              # out of range
    assert lib.mpc_create(C.byref(bad), C.byref(h)) == mpcgpu.MPC_ERR_INVALID
    bad.refine_steps = -1
    bad.precision = mpcgpu.FP32
    bad.kin_rows = 1                  # the kinematic rows: literal form only
    assert lib.mpc_create(C.byref(bad), C.byref(h)) == mpcgpu.MPC_ERR_INVALID
    bad.form = mpcgpu.FORM_LDL
    bad.ruiz_iters = 5                # ... and not with the Ruiz scaling
    assert lib.mpc_create(C.byref(bad), C.byref(h)) == mpcgpu.MPC_ERR_INVALID
    bad.ruiz_iters = 0
    bad.swing_height = float("nan")
    assert lib.mpc_create(C.byref(bad), C.byref(h)) == mpcgpu.MPC_ERR_INVALID
    bad.swing_height = 0.075
    bad.kin_rows = 0
    bad.form = mpcgpu.FORM_FUSED
    bad.hbm_budget_bytes = 1024       # far below what 16 agents need
    assert lib.mpc_create(C.byref(bad), C.byref(h)) == mpcgpu.MPC_ERR_BUDGET
    assert lib.mpc_destroy(None) == mpcgpu.MPC_ERR_INVALID
    assert lib.mpc_last_error(None) == b"NULL context"
    assert lib.mpc_set_trees(None, 0, None, None) == mpcgpu.MPC_ERR_INVALID
    tf = C.c_double(0.0)
    assert lib.mpc_measure_peak(9, None, C.byref(tf), None) == mpcgpu.MPC_ERR_INVALID
    assert lib.mpc_measure_peak(mpcgpu.PEAK_FP32_FMA, None, None, None) == mpcgpu.MPC_ERR_INVALID


def test_pack_models_roundtrip():
    from paper_2510_12717_b300 import mpcgpu
    from workload import make_agents
    m, _ = make_agents("uneven", np.arange(5))
    recs = mpcgpu.pack_models(m)
    assert np.array_equal(recs["N"], m["N"])
    assert np.array_equal(recs["J_leg"], m["J_leg"])
    assert np.array_equal(recs["duty"], m["duty"])


def test_form_values_match_header():
    from paper_2510_12717_b300 import mpcgpu
    src = open(HEADER).read()
    m = re.search(r"MPC_FORM_PLAIN = (\d+), MPC_FORM_FUSED = (\d+), MPC_FORM_LDL = (\d+)", src)
    assert m and tuple(int(v) for v in m.groups()) == (mpcgpu.FORM_PLAIN, mpcgpu.FORM_FUSED, mpcgpu.FORM_LDL)


def test_max_horizon_matches_header():
    import re
    from paper_2510_12717_b300 import mpcgpu
    src = open(os.path.join(ROOT, "include", "mpcgpu.h")).read()
    m = re.search(r"#define MPC_MAX_HORIZON (\d+)", src)
    assert m and int(m.group(1)) == mpcgpu.MAX_HORIZON
