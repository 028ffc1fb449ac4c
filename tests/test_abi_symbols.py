"""The C-ABI library loads on the host and exports every declared entry point.

No compute call is made here (no GPU needed): the library is opened with
dlopen and each function that include/*.h declares is looked up.
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(pm_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pm_create", "pm_set_distance_field", "pm_smpc_iterate", "pm_replan",
                     "pm_destroy", "pm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2512_22575_b300 as pm
    lib = ctypes.CDLL(pm.lib_path())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_every_symbol():
    from paper_2512_22575_b300 import _abi
    assert set(declared_functions()) <= set(_abi.SIGNATURES)


def test_version_and_error_strings_without_gpu():
    import paper_2512_22575_b300 as pm
    assert "sm_103a" in pm.version()
    assert isinstance(pm.last_error(None), str)


def test_invalid_create_is_rejected_on_host():
    """Argument checks run before any CUDA call."""
    import numpy as np
    import paper_2512_22575_b300 as pm
    import workloads
    from workloads.scenes import GridDesc
    rb = workloads.panda_robot()
    cp = workloads.default_cost_params(workloads.READY_POSE)
    bad = dict(rb)
    bad["n_joints"] = 6
    with pytest.raises(pm.PmError) as e:
        pm.create(bad, GridDesc(8, 8, 8, 0.1, (0, 0, 0)), cp)
    assert e.value.name == "PM_EINVAL"
    with pytest.raises(pm.PmError) as e:
        pm.create(rb, GridDesc(1, 8, 8, 0.1, (0, 0, 0)), cp)
    assert e.value.name == "PM_EINVAL"
    cp2 = dict(cp)
    cp2["w_env"] = np.float32(np.nan)
    with pytest.raises(pm.PmError) as e:
        pm.create(rb, GridDesc(8, 8, 8, 0.1, (0, 0, 0)), cp2)
    assert e.value.name == "PM_EINVAL"
