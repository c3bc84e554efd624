"""The C ABI without a GPU: the library loads, exports every symbol the
header declares, the ctypes struct matches the C layout, and configuration
errors come back as status codes with a reason."""

import ctypes
import os
import re
import subprocess

import pytest

import synthetic


@pytest.fixture(scope="module")
def B():
    from paper_2609_32892_b300 import build

    build.build()
    from paper_2609_32892_b300 import binding

    return binding


def test_exports_every_declared_symbol(B, root):
    hdr = open(os.path.join(root, "include", "lbm.h")).read()
    declared = sorted(set(re.findall(r"^int (lbm_\w+)\(", hdr, flags=re.M)))
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = sorted(set(re.findall(r" T (lbm_\w+)$", out, flags=re.M)))
    assert declared == exported
    assert sorted(B.EXPORTED) == declared


def test_struct_layout_matches_c(B, root, tmp_path):
    fields = [f for f, _ in B.lbm_config._fields_]
    src = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{root}/include/lbm.h"', "int main(void){",
           'printf("%zu\\n", sizeof(lbm_config));']
    src += [f'printf("%zu\\n", offsetof(lbm_config, {f}));' for f in fields]
    src += ["return 0;}"]
    (tmp_path / "l.c").write_text("\n".join(src))
    subprocess.run(["gcc", "-o", str(tmp_path / "l"), str(tmp_path / "l.c")], check=True)
    vals = [int(v) for v in subprocess.run([str(tmp_path / "l")], capture_output=True, text=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(B.lbm_config)
    for f, off in zip(fields, vals[1:]):
        assert getattr(B.lbm_config, f).offset == off, f


def test_required_bytes_and_config_errors(B):
    for name in ("C1", "C2", "C3", "C4", "C4_TO"):
        cfg = B.config_from_workload(synthetic.workload(name))
        assert B.lbm_required_bytes(cfg) > 0
    bad = B.config_from_workload(synthetic.workload("C1", tau=0.5))
    with pytest.raises(B.LbmError) as e:
        B.lbm_required_bytes(bad)
    assert e.value.code == B.LBM_ERR_ARG and "tau" in str(e.value)
    bad = B.config_from_workload(synthetic.workload("C2", n_mp=6))
    with pytest.raises(B.LbmError):
        B.lbm_required_bytes(bad)
    cfg = B.config_from_workload(synthetic.workload("C3"))
    assert B.lbm_qoi_row_len(cfg) == 2 + 3 * 12


def test_projection_shapes_without_gpu(B):
    """phi_m's LF grid is host arithmetic: the channel of Sec. 7.1 (phi_5) and
    the 2048^2 Kolmogorov run onto the 256^2 LF grid (phi_8)."""
    assert B.lbm_project_shape(B.config_from_workload(synthetic.workload("HF_CHANNEL")), 5) == (295, 49, 98)
    lf = synthetic.workload("LF_CHANNEL")
    assert (lf["nx"], lf["ny"], lf["nz"]) == (295, 49, 98)
    assert B.lbm_project_shape(B.config_from_workload(synthetic.workload("HF_KOLMO")), 8) == (256, 256, 1)
    for name, m in [("HF_CHANNEL", 4), ("HF_CHANNEL", 3), ("HF_KOLMO", 3), ("C4", 0)]:
        with pytest.raises(B.LbmError) as e:
            B.lbm_project_shape(B.config_from_workload(synthetic.workload(name)), m)
        assert e.value.args and "m" in str(e.value)


def test_set_to_coeffs_without_gpu(B):
    """lbm_set_to_coeffs checks its handle before any device work, and the
    fixed-gamma mode is a valid configuration (its buffer holds the N gamma_i)."""
    with pytest.raises(B.LbmError) as e:
        B.lbm_set_to_coeffs(None, "fixed", gamma_fixed=[0.0, 0.0])
    assert e.value.code == B.LBM_ERR_ARG
    fixed = B.config_from_workload(synthetic.workload("C3", to_mode="fixed"))
    observe = B.config_from_workload(synthetic.workload("C3", to_mode="observe"))
    assert B.lbm_required_bytes(fixed) >= B.lbm_required_bytes(observe)
    bad = B.config_from_workload(synthetic.workload("C3"))
    bad.to_mode = 6
    with pytest.raises(B.LbmError) as e:
        B.lbm_required_bytes(bad)
    assert e.value.code == B.LBM_ERR_ARG


def test_batch_mode_arguments_without_gpu(B):
    """lbm_batch_set_persistent refuses a missing batch and out-of-range lanes
    or node limits before touching the device."""
    for lanes, max_nodes in ((1, 16384), (-1, 16384), (65, 16384), (1, -1)):
        with pytest.raises(B.LbmError) as e:
            B.lbm_batch_set_persistent(None, lanes, max_nodes)
        assert e.value.code == B.LBM_ERR_ARG
