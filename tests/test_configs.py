"""The workload table: parameter counts of the five model shapes (host-only library calls) and
the sizes of the small inputs."""
import pytest

from paper_2304_13144_gb300 import configs


@pytest.mark.parametrize("name,m", [("C1", 26), ("C2", 222), ("C3", 383), ("C4", 651), ("C5", 1636)])
def test_parameter_counts(native_lib, name, m):
    from paper_2304_13144_gb300 import api
    w = configs.workload(name)
    assert api.mtp_describe(w.desc())["n_params"] == m
    assert w.theta().shape == (m,)


def test_small_inputs():
    b = configs.workload("C1").inputs()
    assert len(b["type"]) == 108 and b["cell"].shape == (1, 3, 3)
    t = configs.workload("C3").inputs()
    assert len(t["atom_offset"]) == 513
